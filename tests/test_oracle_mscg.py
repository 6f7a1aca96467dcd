"""Pins of the oracle's multi-shift CG (no GPU).

* brute force: dense LAPACK solves of (A + sigma_i) x = b on 4^4;
* free field: a plane-wave source gives x_i = psi / (m^2 + sigma_i + sum sin^2 p);
* first-iteration closed forms of the shifted recurrences;
* agreement with an independent single-shift CG per sigma_i;
* every shift's FP64 true residual at or below the requested tolerance.
"""
import numpy as np
import pytest

import oracle
import synthetic as S
from tests import latutil as lu


@pytest.fixture(scope="module")
def small():
    cfg = S.CONFIGS["small_4x4x4x4"]
    dims = cfg["dims"]
    u = S.gauge_links(dims, cfg["links"], 1000 + cfg["k"])
    b = S.gaussian_field(dims, 2000 + cfg["k"])
    shifts = cfg["shifts"]()
    res = oracle.mscg(dims, u, cfg["mass"], shifts, b, tol=cfg["tol"], log_rows=30)
    n = b.size
    a = lu.dense_normal_op(lambda e: oracle.normal_op(dims, u, cfg["mass"], 0.0, e), n)
    return dict(dims=dims, u=u, b=b, shifts=shifts, res=res, a=a, mass=cfg["mass"], tol=cfg["tol"])


def test_true_residuals_below_tol(small):
    assert np.all(small["res"]["true_resid"] <= small["tol"])
    assert small["res"]["iters"] > 50  # a real Krylov solve, not a trivial one


def test_matches_dense_solves(small):
    a, b = small["a"], small["b"].reshape(-1)
    n = a.shape[0]
    ev = np.linalg.eigvalsh(a)
    for i, s in enumerate(small["shifts"]):
        xd = np.linalg.solve(a + s * np.eye(n), b)
        err = np.linalg.norm(small["res"]["x"][i].reshape(-1) - xd) / np.linalg.norm(xd)
        kappa = (ev.max() + s) / (ev.min() + s)
        assert err <= kappa * small["tol"], (i, err, kappa)


def test_first_iteration_closed_form(small):
    """alpha_0 = |b|^2 / b^dag A_sigma0 b and zeta_i^1 = 1 / (1 + s_i alpha_0)."""
    b = small["b"].reshape(-1)
    s0 = small["shifts"].min()
    ab = small["a"] @ b + s0 * b
    alpha0 = np.vdot(b, b).real / np.vdot(b, ab).real
    row = small["res"]["scalar_log"][0]
    assert abs(row[0] - alpha0) <= 1e-13 * alpha0
    z1 = 1.0 / (1.0 + (small["shifts"] - s0) * alpha0)
    np.testing.assert_allclose(row[2:], z1, rtol=1e-13)
    # beta_0 = |r_1|^2 / |r_0|^2 with r_1 = b - alpha0 A b
    r1 = b - alpha0 * ab
    assert abs(row[1] - np.vdot(r1, r1).real / np.vdot(b, b).real) <= 1e-12 * row[1]


def test_zeta_monotone(small):
    """For non-negative relative shifts 0 < zeta_i^{k+1} <= zeta_i^k <= 1."""
    log = small["res"]["scalar_log"]
    z = log[:, 2:]
    nz = z > 0
    assert np.all(z[nz] <= 1.0 + 1e-15)
    for i in range(z.shape[1]):
        zi = z[nz[:, i], i]
        assert np.all(np.diff(zi) <= 1e-15)


def test_free_field_plane_wave_solution():
    dims, mass = (4, 4, 4, 4), 0.1
    shifts = S.log_poles(1e-4, 1.0, 6)
    n = (1, 2, 3, 1)
    psi = lu.plane_wave_even(dims, n, [0.3, 1.0j, -0.5])
    res = oracle.mscg(dims, S.unit_links(dims), mass, shifts, psi, tol=1e-12)
    lam = mass ** 2 + np.sum(np.sin(lu.momentum(dims, n)) ** 2)
    for i, s in enumerate(shifts):
        np.testing.assert_allclose(res["x"][i], psi / (lam + s), rtol=0, atol=1e-12 * np.abs(psi).max() / (lam + s))
    # an eigenvector source converges in one iteration
    assert res["iters"] == 1


def test_agrees_with_single_shift_cg(small):
    dims, u, b, mass, tol = small["dims"], small["u"], small["b"], small["mass"], small["tol"]
    ev = np.linalg.eigvalsh(small["a"])
    for i in (0, 3, 7):
        s = small["shifts"][i]
        x, _ = oracle.cg(dims, u, mass, s, b, tol=tol)
        kappa = (ev.max() + s) / (ev.min() + s)
        err = np.linalg.norm(x - small["res"]["x"][i]) / np.linalg.norm(x)
        assert err <= 2 * kappa * tol


@pytest.mark.parametrize("dims", [(6, 4, 2, 8), (2, 2, 2, 4)])
def test_ragged_lattices(dims):
    u = S.gauge_links(dims, "expih", 7)
    b = S.gaussian_field(dims, 8)
    shifts = np.array([0.0, 0.05, 0.5])
    res = oracle.mscg(dims, u, 0.1, shifts, b, tol=1e-11)
    assert np.all(res["true_resid"] <= 1e-11)
