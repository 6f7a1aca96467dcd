"""Pins of the oracle's staggered operator against facts fixed by the paper and
by the mathematics (no GPU).

* free-field closed form: on unit links, with antiperiodic time, the even
  restriction of a plane wave is an eigenvector of m^2 + sigma - D_eo D_oe with
  eigenvalue m^2 + sigma + sum_mu sin^2 p_mu;
* the dense 4^4 spectrum equals that closed-form multiset;
* anti-Hermiticity D_oe^dag = -D_eo (Sec. 2);
* gauge covariance under a random SU(3) transform;
* A_sigma Hermitian and bounded below by m^2 + sigma (positive definite, Eq. shift_eo).
Negative controls show that plausible mistakes (transposed links, periodic
time, dropped phases) fail these pins.
"""
import numpy as np
import pytest

import oracle
import synthetic as S
from tests import latutil as lu

LATTICES = [(4, 4, 4, 4), (6, 4, 2, 8), (2, 4, 6, 4)]


@pytest.mark.parametrize("dims", LATTICES)
@pytest.mark.parametrize("n", [(0, 0, 0, 0), (1, 2, 0, 1), (2, 1, 1, 3), (1, 3, 1, 0)])
def test_free_field_plane_wave(dims, n):
    n = tuple(k % d for k, d in zip(n, dims))
    mass, sigma = 0.1, 0.03
    psi = lu.plane_wave_even(dims, n, [1.0, 0.5j, -0.3 + 0.2j])
    out = oracle.normal_op(dims, S.unit_links(dims), mass, sigma, psi)
    lam = mass ** 2 + sigma + np.sum(np.sin(lu.momentum(dims, n)) ** 2)
    assert np.abs(out - lam * psi).max() <= 1e-13 * np.abs(psi).max() * max(lam, 1.0)


def test_free_field_dense_spectrum():
    dims, mass = (4, 4, 4, 4), 0.2
    vh3 = S.volume(dims) // 2 * 3
    u = S.unit_links(dims)
    a = lu.dense_normal_op(lambda e: oracle.normal_op(dims, u, mass, 0.0, e), vh3)
    ev = np.linalg.eigvalsh(0.5 * (a + a.conj().T))
    assert np.abs(a - a.conj().T).max() < 1e-14
    np.testing.assert_allclose(ev, lu.free_eigenvalues(dims, mass), atol=1e-12)


@pytest.mark.parametrize("dims", LATTICES)
def test_anti_hermiticity(dims):
    u = S.gauge_links(dims, "haar", 11)
    a = S.gaussian_field(dims, 12)  # odd-site vector
    b = S.gaussian_field(dims, 13)  # even-site vector
    lhs = np.vdot(a, oracle.dslash_oe(dims, u, b))
    rhs = -np.vdot(oracle.dslash_eo(dims, u, a), b)
    assert abs(lhs - rhs) <= 1e-13 * abs(lhs)


def test_full_operator_anti_hermitian_and_blocks():
    dims = (4, 2, 4, 4)
    v = S.volume(dims)
    u = S.gauge_links(dims, "haar", 21)
    d = lu.dense_normal_op(lambda e: oracle.dslash_full(dims, u, e), v * 3)
    assert np.abs(d + d.conj().T).max() < 1e-14
    # D connects only opposite parities: even-even and odd-odd blocks vanish
    par = np.repeat(lu.parity(dims), 3)
    assert np.abs(d[np.ix_(par == 0, par == 0)]).max() == 0.0
    assert np.abs(d[np.ix_(par == 1, par == 1)]).max() == 0.0


@pytest.mark.parametrize("dims", LATTICES)
@pytest.mark.parametrize("out_parity", [0, 1])
def test_gauge_covariance(dims, out_parity):
    u = S.gauge_links(dims, "haar", 31)
    om = S.haar_gauge_transform(dims, 4001)
    psi = S.gaussian_field(dims, 32)
    in_par = 1 - out_parity
    up = lu.gauge_transform_links(dims, u, om)
    psip = lu.gauge_transform_half(dims, psi, om, in_par)
    lhs = oracle.dslash(dims, up, out_parity, psip)
    rhs = lu.gauge_transform_half(dims, oracle.dslash(dims, u, out_parity, psi), om, out_parity)
    assert np.abs(lhs - rhs).max() <= 1e-13 * np.abs(rhs).max()


def test_normal_op_hermitian_positive():
    dims, mass, sigma = (4, 4, 4, 4), 0.1, 1e-3
    u = S.gauge_links(dims, "haar", 1001)
    n = S.volume(dims) // 2 * 3
    a = lu.dense_normal_op(lambda e: oracle.normal_op(dims, u, mass, sigma, e), n)
    assert np.abs(a - a.conj().T).max() < 1e-14
    ev = np.linalg.eigvalsh(a)
    assert ev.min() >= mass ** 2 + sigma - 1e-13
    # -D_eo D_oe = D_oe^dag D_oe, and each of the 4 directions of D has norm <= 1
    assert ev.max() <= mass ** 2 + sigma + 16.0


# ---------------------------------------------------------------- negative controls


def test_transposed_links_break_covariance():
    """Using U^T in place of U (a transposed operand) fails the covariance pin."""
    dims = (4, 4, 4, 4)
    u = S.gauge_links(dims, "haar", 31)
    ut = np.ascontiguousarray(np.swapaxes(u, 2, 3))
    om = S.haar_gauge_transform(dims, 4001)
    psi = S.gaussian_field(dims, 32)
    lhs = oracle.dslash(dims, lu.gauge_transform_links(dims, u, om) .swapaxes(2, 3).copy(), 1,
                        lu.gauge_transform_half(dims, psi, om, 0))
    rhs = lu.gauge_transform_half(dims, oracle.dslash(dims, ut, 1, psi), om, 1)
    assert np.abs(lhs - rhs).max() > 1e-3 * np.abs(rhs).max()


def test_periodic_time_breaks_closed_form():
    """Dropping the antiperiodic sign fails the antiperiodic-momentum closed form."""
    dims, mass = (4, 4, 4, 4), 0.1
    n = (1, 0, 0, 0)
    psi = lu.plane_wave_even(dims, n, [1.0, 0.0, 0.0])
    out = oracle.normal_op(dims, S.unit_links(dims), mass, 0.0, psi, antiperiodic=False)
    lam = mass ** 2 + np.sum(np.sin(lu.momentum(dims, n)) ** 2)
    assert np.abs(out - lam * psi).max() > 1e-2


def test_dropped_phases_break_closed_form():
    """Without staggered phases (all links +1 but eta folded away by using a
    sign-compensating link field) the plane wave stops being an eigenvector."""
    dims, mass = (4, 4, 4, 4), 0.1
    c = lu.coords(dims)
    u = S.unit_links(dims)
    # multiply each link by eta_mu(x) so that the oracle's phase cancels
    for mu in range(4):
        eta = (-1.0) ** (c[:, :mu].sum(axis=1))
        u[mu] *= eta[:, None, None]
    n = (1, 1, 0, 0)
    psi = lu.plane_wave_even(dims, n, [1.0, 0.0, 0.0])
    out = oracle.normal_op(dims, u, mass, 0.0, psi)
    lam = mass ** 2 + np.sum(np.sin(lu.momentum(dims, n)) ** 2)
    assert np.abs(out - lam * psi).max() > 1e-2
