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


# ---------------------------------------------------------------------------- the true residual
# oracle.true_residual is the pass/fail gate of every mixed-precision GPU solve, so it is pinned
# here against quantities fixed by the algebra alone: the relative residual |b - A_sigma x| / |b|
# (Sec. 2, per shift) of x = 0, of a multiple of the exact solution, and of an arbitrary x against
# the dense matrix.


def _dense_solution(small, i):
    a, b = small["a"], small["b"].reshape(-1)
    return np.linalg.solve(a + small["shifts"][i] * np.eye(a.shape[0]), b)


def test_true_residual_of_zero_guess_is_one(small):
    """x = 0 leaves r = b, so the relative residual is exactly 1 for every shift."""
    x0 = np.zeros_like(small["b"])
    for s in small["shifts"]:
        assert oracle.true_residual(small["dims"], small["u"], small["mass"], s, small["b"], x0) == 1.0


@pytest.mark.parametrize("t", [0.5, 1.25, -1.0, 3.0])
def test_true_residual_of_scaled_solution(small, t):
    """x = t x* with A x* = b gives r = (1 - t) b: the residual is |1 - t| (a square, a missing
    sqrt, a division by |b|^2 or a sign flip b + A x would each give another number)."""
    for i in (0, 4, 7):
        xs = _dense_solution(small, i).reshape(small["b"].shape)
        got = oracle.true_residual(small["dims"], small["u"], small["mass"], small["shifts"][i], small["b"], t * xs)
        assert abs(got - abs(1.0 - t)) <= 1e-12, (i, t, got)


def test_true_residual_of_dense_solution_vanishes(small):
    for i in range(len(small["shifts"])):
        xs = _dense_solution(small, i).reshape(small["b"].shape)
        got = oracle.true_residual(small["dims"], small["u"], small["mass"], small["shifts"][i], small["b"], xs)
        assert got <= 1e-13, (i, got)


def test_true_residual_of_perturbed_solution_matches_dense(small):
    """Any x: the oracle's value equals |b - (A + sigma) x| / |b| from the dense 4^4 matrix."""
    rng = np.random.default_rng(99)
    a, b = small["a"], small["b"].reshape(-1)
    n = a.shape[0]
    for i, eps in ((0, 1e-6), (3, 1e-3), (7, 0.3)):
        s = small["shifts"][i]
        xs = _dense_solution(small, i)
        x = xs + eps * np.linalg.norm(xs) / np.sqrt(n) * (rng.standard_normal(n) + 1j * rng.standard_normal(n))
        want = np.linalg.norm(b - (a + s * np.eye(n)) @ x) / np.linalg.norm(b)
        got = oracle.true_residual(small["dims"], small["u"], small["mass"], s, small["b"], x.reshape(small["b"].shape))
        assert abs(got - want) <= 1e-12 * want + 1e-15, (i, got, want)


def test_refinement_branch_finishes_capped_shifts(small):
    """With the multi-shift phase capped at 150 iterations the five smallest shifts stop above tol;
    the oracle then finishes each with plain CG from its x_i.  Every shift must end at or below
    tol by the dense residual, and within kappa_i tol of the dense solution."""
    dims, u, b, mass, tol = small["dims"], small["u"], small["b"], small["mass"], small["tol"]
    res = oracle.mscg(dims, u, mass, small["shifts"], b, tol=tol, max_iter=150)
    assert res["iters"] == 150 and res["refine_iters"] > 0
    assert np.sum(res["shift_iters"] == 150) >= 3
    a, bb = small["a"], b.reshape(-1)
    n = a.shape[0]
    ev = np.linalg.eigvalsh(a)
    for i, s in enumerate(small["shifts"]):
        x = res["x"][i].reshape(-1)
        dense_r = np.linalg.norm(bb - (a + s * np.eye(n)) @ x) / np.linalg.norm(bb)
        assert dense_r <= tol, (i, dense_r)
        assert abs(res["true_resid"][i] - dense_r) <= 1e-13
        xd = _dense_solution(small, i)
        kappa = (ev.max() + s) / (ev.min() + s)
        assert np.linalg.norm(x - xd) / np.linalg.norm(xd) <= kappa * tol, i


def test_action_equals_spectral_rational_function(small):
    """oracle.action with the msCG solutions equals b^dag R(A) b computed from the eigenvectors of
    the dense 4^4 operator, R(l) = alpha0 + sum_i r_i / (l + sigma_i) (Sec. 2's rational form)."""
    a, b = small["a"], small["b"].reshape(-1)
    lam, vec = np.linalg.eigh(a)
    c2 = np.abs(vec.conj().T @ b) ** 2
    res = S.positive_residues(3001, len(small["shifts"]))
    alpha0 = 0.21
    want = float(np.sum(c2 * (alpha0 + sum(r / (lam + s) for r, s in zip(res, small["shifts"])))))
    got = oracle.action(res, small["b"], small["res"]["x"], alpha0=alpha0)
    ev = lam.min() + small["shifts"].min()
    assert abs(got - want) <= 1e-9 * abs(want) + small["tol"] * np.linalg.norm(b) ** 2 / ev, (got, want)
    # the residue-weighted terms alone: a sign flip of Re(b^dag x) or a dropped residue fails
    got0 = oracle.action(res, small["b"], small["res"]["x"])
    assert abs(got0 - (want - alpha0 * np.sum(c2))) <= 1e-8 * abs(want)
