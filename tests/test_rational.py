"""Pins of the Remez rational approximation (no GPU; needs mpmath).

* equioscillation: the relative error x**p -> R(x) has at least 2n+2 alternating extrema of equal
  size |E| on [lo, hi] (the characterisation of the minimax approximation), and the dense-sampled
  maximum equals the reported one;
* optimality against an independent method: the best relative error on a fine grid, found by
  bisection on E with a linear-programming feasibility test (|P - f Q| <= E f Q, Q >= 1, a library LP
  solver), agrees with Remez's E;
* structure: real positive poles, positive residues for power in (-1, 0) (a Stieltjes function);
* applied to a dense SPD matrix (the 4^4 normal operator): R(A) b against A**p b from the Hermitian
  eigendecomposition, within the approximation's error bound.
"""
import numpy as np
import pytest

pytest.importorskip("mpmath")

import oracle  # noqa: E402
import synthetic as S  # noqa: E402
from paper_1801_01473_gb300.rational import remez  # noqa: E402
from tests import latutil as lu  # noqa: E402


@pytest.mark.parametrize("power,n,lo,hi", [(-0.25, 6, 1e-3, 16.0), (-0.5, 5, 1e-2, 1.0), (0.125, 6, 1e-4, 16.0)])
def test_equioscillation(power, n, lo, hi):
    r = remez(power, n, lo, hi)
    x = np.exp(np.linspace(np.log(lo), np.log(hi), 200001))
    e = r(x) / x ** power - 1
    assert np.abs(e).max() == pytest.approx(r.max_rel_error, rel=1e-3)
    # extrema between sign changes: count the alternating runs whose peak reaches |E|
    sign = np.sign(e)
    runs = np.split(np.abs(e), np.nonzero(np.diff(sign))[0] + 1)
    peaks = [run.max() for run in runs]
    assert len(peaks) >= 2 * n + 2
    assert min(peaks) >= 0.999 * r.max_rel_error


def test_poles_and_residues_positive_for_inverse_roots():
    r = remez(-0.25, 8, 1e-4, 16.0)
    assert min(r.poles) > 0 and min(r.residues) > 0 and r.alpha0 > 0
    assert len(r.poles) == 8 and np.all(np.diff(r.poles) > 0)


def _lp_minimax(f, n, x):
    from scipy.optimize import linprog
    fx = f(x)
    V = np.vander(x, n + 1, increasing=True)
    lo_e, hi_e = 0.0, 1.0
    for _ in range(40):
        E = 0.5 * (lo_e + hi_e)
        # variables [a_0..a_n, b_0..b_n]; P - f(1+E)Q <= 0, -P + f(1-E)Q <= 0, -Q <= -1
        A1 = np.hstack([V, -(fx * (1 + E))[:, None] * V])
        A2 = np.hstack([-V, (fx * (1 - E))[:, None] * V])
        A3 = np.hstack([np.zeros_like(V), -V])
        A = np.vstack([A1, A2, A3])
        b = np.concatenate([np.zeros(len(x)), np.zeros(len(x)), -np.ones(len(x))])
        res = linprog(np.zeros(2 * n + 2), A_ub=A, b_ub=b, bounds=[(None, None)] * (2 * n + 2), method="highs")
        if res.status == 0:
            hi_e = E
        else:
            lo_e = E
    return hi_e


def test_optimal_error_matches_linear_programming():
    power, n, lo, hi = -0.25, 3, 0.05, 1.0
    r = remez(power, n, lo, hi)
    x = np.exp(np.linspace(np.log(lo), np.log(hi), 600))
    e_lp = _lp_minimax(lambda t: t ** power, n, x)
    # the grid optimum can only be below the continuous one, and the grid is fine
    assert e_lp <= r.max_rel_error * (1 + 1e-6)
    assert e_lp == pytest.approx(r.max_rel_error, rel=2e-2)


def test_matrix_function_within_error_bound():
    dims, mass = (4, 4, 4, 4), 0.3
    u = S.gauge_links(dims, "expih", 191)
    b = S.gaussian_field(dims, 192).reshape(-1)
    a = lu.dense_normal_op(lambda v: oracle.normal_op(dims, u, mass, 0.0, v), b.size)
    w, v = np.linalg.eigh(0.5 * (a + a.conj().T))
    assert w.min() > 0.05 and w.max() < 16.0
    for power in (-0.25, 0.125):
        r = remez(power, 8, 0.05, 16.0)
        exact = v @ ((w ** power) * (v.conj().T @ b))
        approx = r.alpha0 * b + sum(res * np.linalg.solve(a + s * np.eye(b.size), b)
                                    for res, s in zip(r.residues, r.poles))
        # |R(A) b - A^p b| <= max_x |R/f - 1| |A^p b| (eigenvector by eigenvector)
        assert np.linalg.norm(approx - exact) <= 1.01 * r.max_rel_error * np.linalg.norm(exact)


def test_stored_rhmc_coefficients_are_remez_output():
    import json
    import os
    stored = json.load(open(os.path.join(os.path.dirname(os.path.dirname(__file__)), "paper_1801_01473_gb300", "data",
                                         "rhmc_rational_m0.3.json")))
    for name, power in (("heatbath", 0.125), ("action", -0.25)):
        r = remez(power, 10, 0.05, 16.5)
        d = stored[name]
        assert d["power"] == power and d["lo"] == 0.05 and d["hi"] == 16.5
        assert np.allclose(d["poles"], r.poles, rtol=1e-9) and np.allclose(d["residues"], r.residues, rtol=1e-9)
        assert d["alpha0"] == pytest.approx(r.alpha0, rel=1e-9) and d["max_rel_error"] < 1e-10
