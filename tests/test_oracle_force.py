"""Pins of the oracle's fermion force (no GPU).

S = sum_i r_i Re(b^dag (A + sigma_i)^-1 b) is evaluated by dense LAPACK solves
on 4^4, independently of the oracle's solver, and differentiated by central
finite differences (eps = 1e-5):
* along U -> exp(eps X) U, X in su(3):   dS/deps = tr(X F),  F = TA(U W);
* along real / imaginary link entries:    dS/dRe U + i dS/dIm U = W^dag.
Also: F is traceless anti-Hermitian, and it transforms covariantly,
F'(x) = Omega(x) F(x) Omega(x)^dag, when links and source are gauge transformed.
"""
import numpy as np
import pytest

import oracle
import synthetic as S
from tests import latutil as lu

DIMS = (4, 4, 4, 4)
MASS = 0.1
SHIFTS = np.array([1e-3, 2e-2, 0.3])
RES = np.array([0.7, 0.4, 0.25])


def dense_action(u, b):
    n = b.size
    a = lu.dense_normal_op(lambda e: oracle.normal_op(DIMS, u, MASS, 0.0, e), n)
    bb = b.reshape(-1)
    return sum(r * np.vdot(bb, np.linalg.solve(a + s * np.eye(n), bb)).real for r, s in zip(RES, SHIFTS))


@pytest.fixture(scope="module")
def setup():
    u = S.gauge_links(DIMS, "haar", 51)
    b = S.gaussian_field(DIMS, 52)
    res = oracle.mscg(DIMS, u, MASS, SHIFTS, b, tol=1e-13)
    f = oracle.force(DIMS, u, RES, res["x"], kind=0)
    g = oracle.force(DIMS, u, RES, res["x"], kind=1)
    return u, b, res, f, g


def _links_to_test():
    v = S.volume(DIMS)
    lx, ly, lz, lt = DIMS
    t_boundary = 0 + lx * (1 + ly * (2 + lz * (lt - 1)))  # x=0, y=1, z=2, t=Lt-1
    # (mu, site): even site, odd site, t-boundary link, x-wrap link
    return [(0, 0), (2, 1), (3, t_boundary), (0, lx - 1), (1, v - 2)]


@pytest.mark.parametrize("link", _links_to_test())
def test_force_matches_finite_differences(setup, link):
    u, b, _, f, _ = setup
    mu, z = link
    g = np.random.default_rng(1000 * mu + z)
    x = lu.random_su3_algebra(g)
    eps = 1e-5
    up, um = u.copy(), u.copy()
    up[mu, z] = lu.expm_su3(eps * x) @ u[mu, z]
    um[mu, z] = lu.expm_su3(-eps * x) @ u[mu, z]
    fd = (dense_action(up, b) - dense_action(um, b)) / (2 * eps)
    an = np.trace(x @ f[mu, z]).real
    assert abs(np.trace(x @ f[mu, z]).imag) < 1e-12
    assert abs(fd - an) <= 1e-6 * abs(an), (fd, an)


@pytest.mark.parametrize("entry", [(0, 1), (2, 2)])
def test_link_entry_gradient(setup, entry):
    u, b, _, _, g = setup
    mu, z = 1, 5
    a, c = entry
    eps = 1e-5
    out = []
    for d in (1.0, 1j):
        up, um = u.copy(), u.copy()
        up[mu, z, a, c] += eps * d
        um[mu, z, a, c] -= eps * d
        out.append((dense_action(up, b) - dense_action(um, b)) / (2 * eps))
    fd = out[0] + 1j * out[1]
    assert abs(fd - g[mu, z, a, c]) <= 1e-6 * abs(g[mu, z, a, c])


def test_force_in_algebra(setup):
    f = setup[3]
    assert np.abs(f + np.conj(np.swapaxes(f, 2, 3))).max() < 1e-13 * np.abs(f).max()
    assert np.abs(np.trace(f, axis1=2, axis2=3)).max() < 1e-13 * np.abs(f).max()


def test_force_gauge_covariance(setup):
    u, b, res, f, _ = setup
    om = S.haar_gauge_transform(DIMS, 4005)
    up = lu.gauge_transform_links(DIMS, u, om)
    bp = lu.gauge_transform_half(DIMS, b, om, 0)
    resp = oracle.mscg(DIMS, up, MASS, SHIFTS, bp, tol=1e-13)
    fp = oracle.force(DIMS, up, RES, resp["x"], kind=0)
    expect = np.einsum("sab,msbc,scd->msad", om, f, np.conj(np.swapaxes(om, 1, 2)))
    assert np.abs(fp - expect).max() <= 1e-9 * np.abs(f).max()
