"""Pins of the oracle with a U(1) phase field theta_mu(x) on the links (no GPU).

* imaginary chemical potential / constant field: on unit links with theta_mu(x) = a_mu, even
  plane waves are eigenvectors of m^2 + sigma - D_eo D_oe with eigenvalue
  m^2 + sigma + sum_mu sin^2(p_mu + a_mu) (the phase shifts every momentum);
* the antiperiodic time boundary is a phase: theta_t = pi on the t-links with x_t = Lt - 1 and a
  periodic lattice gives the antiperiodic operator with theta = 0;
* U(1) gauge covariance: theta'_mu(x) = theta_mu(x) + alpha(x) - alpha(x+mu), psi' = exp(i alpha) psi;
* the force with phases against central finite differences of the action (dense LAPACK solves)
  along su(3) directions (kind 0) and complex link directions (kind 1).
"""
import numpy as np
import pytest

import oracle
import synthetic as S
from tests import latutil as lu

DIMS = (4, 4, 4, 4)
MASS = 0.1


def _unit(v):
    return np.broadcast_to(np.eye(3, dtype=np.complex128), (4, v, 3, 3)).copy()


@pytest.mark.parametrize("n", [(0, 0, 0, 0), (1, 0, 2, 1), (1, 3, 1, 0)])
def test_constant_phase_shifts_momenta(n):
    v = int(np.prod(DIMS))
    a = np.array([0.3, -0.7, 0.2, 0.45])
    theta = np.broadcast_to(a[:, None], (4, v)).copy()
    psi = lu.plane_wave_even(DIMS, n, [1.0, 0.5j, -0.25])
    out = oracle.normal_op(DIMS, oracle.u1_links(_unit(v), theta), MASS, 0.02, psi)
    lam = MASS ** 2 + 0.02 + np.sum(np.sin(lu.momentum(DIMS, n) + a) ** 2)
    assert np.abs(out - lam * psi).max() < 1e-13


def test_antiperiodic_boundary_is_a_phase():
    u = S.gauge_links(DIMS, "haar", 171)
    v = u.shape[1]
    c = lu.coords(DIMS)
    theta = np.zeros((4, v))
    theta[3] = np.where(c[:, 3] == DIMS[3] - 1, np.pi, 0.0)
    psi = S.gaussian_field(DIMS, 172)
    a = oracle.dslash_oe(DIMS, oracle.u1_links(u, theta), psi, antiperiodic=False)
    b = oracle.dslash_oe(DIMS, u, psi, antiperiodic=True)
    assert np.abs(a - b).max() < 1e-14


def test_u1_gauge_covariance():
    u = S.gauge_links(DIMS, "haar", 173)
    v = u.shape[1]
    g = np.random.default_rng(174)
    theta = g.uniform(-np.pi, np.pi, (4, v))
    alpha = g.uniform(-np.pi, np.pi, v)
    theta2 = np.stack([theta[mu] + alpha - alpha[lu.shift_index(DIMS, mu, 1)] for mu in range(4)])
    psi = S.gaussian_field(DIMS, 175)
    ph_e = np.exp(1j * lu.to_half(DIMS, alpha, 0))
    ph_o = np.exp(1j * lu.to_half(DIMS, alpha, 1))
    a = oracle.dslash_oe(DIMS, oracle.u1_links(u, theta2), ph_e[:, None] * psi)
    b = ph_o[:, None] * oracle.dslash_oe(DIMS, oracle.u1_links(u, theta), psi)
    assert np.abs(a - b).max() < 1e-13


SHIFTS = np.array([2e-2, 0.3])
RES = np.array([0.6, 0.3])


def _dense_action(u, theta, b):
    n = b.size
    vl = oracle.u1_links(u, theta)
    a = lu.dense_normal_op(lambda e: oracle.normal_op(DIMS, vl, MASS, 0.0, e), n)
    bb = b.reshape(-1)
    return sum(r * np.vdot(bb, np.linalg.solve(a + s * np.eye(n), bb)).real for r, s in zip(RES, SHIFTS))


@pytest.mark.parametrize("direction", ["algebra", "complex"])
def test_force_with_phases_finite_differences(direction):
    u = S.gauge_links(DIMS, "haar", 176)
    v = u.shape[1]
    g = np.random.default_rng(177)
    theta = g.uniform(-np.pi, np.pi, (4, v))
    b = S.gaussian_field(DIMS, 178)
    x = oracle.mscg(DIMS, oracle.u1_links(u, theta), MASS, SHIFTS, b, tol=1e-13)["x"]
    if direction == "algebra":
        m = g.standard_normal(u.shape) + 1j * g.standard_normal(u.shape)
        xa = 0.5 * (m - np.conj(np.swapaxes(m, -1, -2)))
        xa -= (np.trace(xa, axis1=-2, axis2=-1) / 3.0)[..., None, None] * np.eye(3)
        du = xa @ u
        f = oracle.force_u1(DIMS, u, theta, RES, x, kind=0)
        an = np.einsum("lsab,lsba->", xa, f).real
    else:
        du = g.standard_normal(u.shape) + 1j * g.standard_normal(u.shape)
        an = np.sum(np.conj(oracle.force_u1(DIMS, u, theta, RES, x, kind=1)) * du).real
    eps = 1e-5
    fd = (_dense_action(u + eps * du, theta, b) - _dense_action(u - eps * du, theta, b)) / (2 * eps)
    assert an == pytest.approx(fd, rel=1e-6)
