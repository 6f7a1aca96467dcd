"""The unrolled form of the multi-shift updates used by the mixed solver's deferred update (no GPU).

Per iteration t = 1..n of a window, every shift does
    x <- x + ax_t p ;   p <- pr_t r_t + pp_t p
(a converged shift: ax = pr = 0, pp = 1 after its last update; the base shift: pr = 1, pp = beta).
Unrolled over the window with P0 the p at the window start:
    x_n = x_0 + sum_t a_t r_t + e P0 ,   p_n = sum_t d_t r_t + f P0 ,
    a_t = pr_t S_t ,  d_t = pr_t P_t ,  S_{t-1} = ax_t + pp_t S_t ,  P_{t-1} = pp_t P_t ,
    S_n = 0 ,  P_n = 1 ,  e = S_0 ,  f = P_0 .
The test runs the per-iteration recurrence on random scalars and vectors and checks the unrolled
form against it, including shifts that stop inside the window and an empty window.
"""
import numpy as np
import pytest


def _per_iteration(ax, pr, pp, r, x0, p0):
    x, p = x0.copy(), p0.copy()
    for t in range(len(ax)):
        x = x + ax[t] * p
        p = pr[t] * r[t] + pp[t] * p
    return x, p


def _unrolled(ax, pr, pp, r, x0, p0):
    n = len(ax)
    a, d = np.zeros(n), np.zeros(n)
    s_acc, p_acc = 0.0, 1.0
    for t in range(n - 1, -1, -1):
        a[t], d[t] = pr[t] * s_acc, pr[t] * p_acc
        s_acc = ax[t] + pp[t] * s_acc
        p_acc = pp[t] * p_acc
    x = x0 + sum(a[t] * r[t] for t in range(n)) + s_acc * p0
    p = sum(d[t] * r[t] for t in range(n)) + p_acc * p0
    return x, p


@pytest.mark.parametrize("n,stop", [(37, None), (64, 20), (8, 0), (1, None), (0, None)])
def test_unrolled_window_equals_per_iteration(n, stop):
    rng = np.random.default_rng(1000 + n)
    m = 60
    ax = rng.uniform(0.1, 2.0, n)
    pr = rng.uniform(0.2, 1.0, n)
    pp = rng.uniform(0.0, 0.9, n)
    if stop is not None:  # the shift converges at iteration `stop` (its last x update), then idles
        pr[stop:] = 0.0
        pp[stop:] = 1.0
        ax[stop + 1:] = 0.0
    r = rng.standard_normal((max(n, 1), m)) + 1j * rng.standard_normal((max(n, 1), m))
    x0 = rng.standard_normal(m) + 1j * rng.standard_normal(m)
    p0 = rng.standard_normal(m) + 1j * rng.standard_normal(m)
    xw, pw = _per_iteration(ax, pr, pp, r, x0, p0)
    xu, pu = _unrolled(ax, pr, pp, r, x0, p0)
    scale = max(1.0, np.abs(xw).max())
    assert np.abs(xu - xw).max() <= 1e-12 * scale
    assert np.abs(pu - pw).max() <= 1e-12 * max(1.0, np.abs(pw).max())


def test_windows_compose():
    """Two consecutive windows (p materialised at the boundary) equal one window over both."""
    rng = np.random.default_rng(7)
    n, m = 40, 30
    ax, pr, pp = rng.uniform(0.1, 2, n), rng.uniform(0.2, 1, n), rng.uniform(0, 0.9, n)
    r = rng.standard_normal((n, m)) + 1j * rng.standard_normal((n, m))
    x0 = np.zeros(m, complex)
    p0 = rng.standard_normal(m) + 1j * rng.standard_normal(m)
    x1, p1 = _unrolled(ax[:16], pr[:16], pp[:16], r[:16], x0, p0)
    x2, p2 = _unrolled(ax[16:], pr[16:], pp[16:], r[16:], x1, p1)
    xa, pa = _unrolled(ax, pr, pp, r, x0, p0)
    assert np.abs(x2 - xa).max() <= 1e-12 * np.abs(xa).max()
    assert np.abs(p2 - pa).max() <= 1e-12 * np.abs(pa).max()
