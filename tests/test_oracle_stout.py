"""Pins of the oracle's stout smearing and its force chain rule (no GPU).

* the smeared links stay in SU(3) (unitary, det 1), rho = 0 is the identity;
* gauge covariance: smearing Omega(x) U_mu(x) Omega(x+mu)^dag gives
  Omega(x) U'_mu(x) Omega(x+mu)^dag;
* the staple sum against the independent plaquette sum: sum over links of
  Re tr(C U^dag) counts each plaquette once per link, 4 P;
* a stout step is an ascent step of the plaquette sum P: dP/drho at rho = 0
  equals sum over links |TA(C U^dag)|^2 (first-order change of P along
  U -> exp(rho X) U with X = TA(C U^dag));
* the pulled-back gradient against central finite differences of
  S(U^(k)(U^(0))), for a linear S along su(3) and along arbitrary complex
  directions, and for the pseudofermion action evaluated by dense LAPACK
  solves (its gradient at U^(k) from the oracle's fermion force).
"""
import numpy as np
import pytest

import oracle
import synthetic as S
from oracle import stout as ost
from tests import latutil as lu

DIMS = (4, 4, 4, 4)
RHO = 0.15


@pytest.fixture(scope="module")
def links():
    return S.gauge_links(DIMS, "haar", 71)


def _rand_algebra(g, n):
    m = g.standard_normal((n, 3, 3)) + 1j * g.standard_normal((n, 3, 3))
    x = 0.5 * (m - np.conj(np.swapaxes(m, 1, 2)))
    return x - np.trace(x, axis1=1, axis2=2)[:, None, None] / 3.0 * np.eye(3)


def test_smeared_links_special_unitary(links):
    for lev in ost.stout(DIMS, links, RHO, 2)[1:]:
        m = lev.reshape(-1, 3, 3)
        err = np.abs(m @ np.conj(np.swapaxes(m, 1, 2)) - np.eye(3)).max()
        assert err < 1e-13
        assert np.abs(np.linalg.det(m) - 1.0).max() < 1e-13
    assert np.array_equal(ost.stout_step(DIMS, links, 0.0), links) or \
        np.abs(ost.stout_step(DIMS, links, 0.0) - links).max() < 1e-15


def test_gauge_covariance(links):
    v = lu.coords(DIMS).shape[0]
    om = S.haar_su3(np.random.default_rng(72), v)
    a = ost.stout(DIMS, lu.gauge_transform_links(DIMS, links, om), RHO, 2)[-1]
    b = lu.gauge_transform_links(DIMS, ost.stout(DIMS, links, RHO, 2)[-1], om)
    assert np.abs(a - b).max() < 1e-13


def test_staples_count_each_plaquette_four_times(links):
    c = ost.staples(DIMS, links)
    lhs = np.einsum("lsab,lsab->", c, links.conj()).real  # sum Re tr(C U^dag)
    assert lhs == pytest.approx(4.0 * lu.plaquette_sum(DIMS, links), rel=1e-12)


def test_stout_step_ascends_plaquette(links):
    omega = ost.staples(DIMS, links) @ np.conj(np.swapaxes(links, -1, -2))
    slope = np.sum(np.abs(ost.ta(omega)) ** 2)
    eps = 1e-5
    fd = (lu.plaquette_sum(DIMS, ost.stout_step(DIMS, links, eps))
          - lu.plaquette_sum(DIMS, ost.stout_step(DIMS, links, -eps))) / (2 * eps)
    assert fd == pytest.approx(slope, rel=1e-8)
    assert lu.plaquette_sum(DIMS, ost.stout_step(DIMS, links, RHO)) > lu.plaquette_sum(DIMS, links)


def _directional(f, u, du, eps=1e-5):
    return (f(u + eps * du) - f(u - eps * du)) / (2 * eps)


@pytest.mark.parametrize("direction", ["algebra", "complex"])
def test_backward_linear_functional(links, direction):
    g = np.random.default_rng(73)
    z = g.standard_normal(links.shape) + 1j * g.standard_normal(links.shape)

    def s(u):
        return np.sum(np.conj(z) * ost.stout(DIMS, u, RHO, 2)[-1]).real  # Re tr(Z^dag U^(2))

    levels = ost.stout(DIMS, links, RHO, 2)
    g0 = ost.stout_backward(DIMS, levels, RHO, z)
    if direction == "algebra":
        du = _rand_algebra(g, 4 * links.shape[1]).reshape(links.shape) @ links
    else:
        du = g.standard_normal(links.shape) + 1j * g.standard_normal(links.shape)
    want = _directional(s, links, du)
    got = np.sum(np.conj(g0) * du).real
    assert got == pytest.approx(want, rel=1e-8)
    # Lie-algebra form: dS/deps = sum tr(X F) along U -> exp(eps X) U
    if direction == "algebra":
        x = du @ np.conj(np.swapaxes(links, -1, -2))
        f = ost.lie_force(links, g0)
        assert np.einsum("lsab,lsba->", x, f).real == pytest.approx(want, rel=1e-8)


def test_backward_pseudofermion_action():
    dims, mass = DIMS, 0.1
    shifts, res = np.array([2e-2, 0.3]), np.array([0.6, 0.3])
    u0 = S.gauge_links(dims, "haar", 74)
    b = S.gaussian_field(dims, 75)
    n = b.size

    def action(u):
        uk = ost.stout(dims, u, RHO, 2)[-1]
        a = lu.dense_normal_op(lambda e: oracle.normal_op(dims, uk, mass, 0.0, e), n)
        bb = b.reshape(-1)
        return sum(r * np.vdot(bb, np.linalg.solve(a + s * np.eye(n), bb)).real for r, s in zip(res, shifts))

    levels = ost.stout(dims, u0, RHO, 2)
    sol = oracle.mscg(dims, levels[-1], mass, shifts, b, tol=1e-13)
    gk = oracle.force(dims, levels[-1], res, sol["x"], kind=1)
    g0 = ost.stout_backward(dims, levels, RHO, gk)
    g = np.random.default_rng(76)
    du = _rand_algebra(g, 4 * u0.shape[1]).reshape(u0.shape) @ u0
    want = _directional(action, u0, du)
    assert np.sum(np.conj(g0) * du).real == pytest.approx(want, rel=1e-7)
