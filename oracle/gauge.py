"""FP64 CPU oracle of the tree-level Symanzik gauge action and its force (numpy).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the CPU-baseline leg
of the benchmark use this module; the product path never imports it.  It
shares no code with the CUDA library.

The gauge part S_g of the action (Sec. 2) is the tree-level Symanzik improved
discretisation: Wilson loops around 1x1 plaquettes and 1x2 rectangles of the
unsmeared links U^(0).  Read with the coefficients of that discretisation,
c0 = 5/6 on every ordered plaquette and c1 = -1/12 on every ordered rectangle:

    S_g = -(beta/3) sum_x sum_{mu != nu} [ 5/6 Re tr P_{mu nu}(x) - 1/12 Re tr R_{mu nu}(x) ]
    P_{mu nu}(x) = U_mu(x) U_nu(x+mu) U_mu(x+nu)^dag U_nu(x)^dag
    R_{mu nu}(x) = U_mu(x) U_mu(x+mu) U_nu(x+2mu) U_mu(x+mu+nu)^dag U_mu(x+nu)^dag U_nu(x)^dag

(ordered pairs: every plaquette twice, every 2x1 rectangle once).  Links are
periodic in all four directions.

Every loop is a closed path of steps +d (link U_d(y), then y -> y+d) and -d
(link U_d(y-d)^dag, then y -> y-d).  The gradient in torch's convention,
G = dS/dRe U + i dS/dIm U, follows from Re tr(... U ...) = Re tr(U B) with B
the product of the rest of the loop taken cyclically: a +d step contributes
B^dag to G_d(y), a -d step (U^dag B) contributes B to G_d(y-d).  The Lie-algebra
force is F = TA(U G^dag), so that dS/deps = tr(X F) along U -> exp(eps X) U.
"""
from __future__ import annotations

import numpy as np

C_PLAQ = 5.0 / 6.0
C_RECT = -1.0 / 12.0


def _grid(dims, links):
    lx, ly, lz, lt = dims
    return np.asarray(links, dtype=np.complex128).reshape(4, lt, lz, ly, lx, 3, 3)


def _shift(a, d: int, step: int):
    """a(x + step * d) for a site field with axes (t, z, y, x, ...)."""
    return np.roll(a, -step, axis=3 - d) if step else a


def _dag(a):
    return np.swapaxes(a.conj(), -1, -2)


def _ta(x):
    y = 0.5 * (x - _dag(x))
    return y - (np.trace(y, axis1=-2, axis2=-1) / 3.0)[..., None, None] * np.eye(3)


def loops(mu: int, nu: int, c0: float = C_PLAQ, c1: float = C_RECT):
    """The two loop shapes of the action in the ordered plane (mu, nu) as step lists."""
    plaq = [(mu, 1), (nu, 1), (mu, -1), (nu, -1)]
    rect = [(mu, 1), (mu, 1), (nu, 1), (mu, -1), (mu, -1), (nu, -1)]
    return [(c0, plaq), (c1, rect)]


def _path_factors(u, path):
    """Per step: (direction, offset of the link's site from x, daggered, the factor as a field over x)."""
    pos = np.zeros(4, dtype=int)
    out = []
    for d, s in path:
        if s > 0:
            site = pos.copy()
            m = u[d]
            for k in range(4):
                m = _shift(m, k, int(site[k]))
            out.append((d, site, False, m))
            pos[d] += 1
        else:
            pos[d] -= 1
            site = pos.copy()
            m = u[d]
            for k in range(4):
                m = _shift(m, k, int(site[k]))
            out.append((d, site, True, _dag(m)))
    assert not pos.any(), "path must close"
    return out


def action(dims, links, beta: float, c0: float = C_PLAQ, c1: float = C_RECT) -> float:
    """S_g of the links [4][V][3][3] (c0, c1: loop coefficients, tree-level Symanzik by default)."""
    u = _grid(dims, links)
    s = 0.0
    for mu in range(4):
        for nu in range(4):
            if mu == nu:
                continue
            for c, path in loops(mu, nu, c0, c1):
                prod = None
                for _, _, _, m in _path_factors(u, path):
                    prod = m if prod is None else prod @ m
                s += c * np.trace(prod, axis1=-2, axis2=-1).real.sum()
    return -beta / 3.0 * s


def gradient(dims, links, beta: float, c0: float = C_PLAQ, c1: float = C_RECT) -> np.ndarray:
    """G = dS_g/dRe U + i dS_g/dIm U, [4][V][3][3]."""
    u = _grid(dims, links)
    g = np.zeros_like(u)
    for mu in range(4):
        for nu in range(4):
            if mu == nu:
                continue
            for c, path in loops(mu, nu, c0, c1):
                f = _path_factors(u, path)
                n = len(f)
                for k in range(n):
                    rest = None
                    for j in list(range(k + 1, n)) + list(range(k)):
                        rest = f[j][3] if rest is None else rest @ f[j][3]
                    d, site, dag, _ = f[k]
                    contrib = rest if dag else _dag(rest)
                    # the factor is the link at x + site: move the contribution there
                    for kk in range(4):
                        contrib = _shift(contrib, kk, -int(site[kk]))
                    g[d] += (-beta / 3.0 * c) * contrib
    return g.reshape(4, -1, 3, 3)


def force(dims, links, beta: float, c0: float = C_PLAQ, c1: float = C_RECT) -> np.ndarray:
    """F = TA(U G^dag) per link, [4][V][3][3]."""
    u = np.asarray(links, dtype=np.complex128).reshape(4, -1, 3, 3)
    return _ta(u @ _dag(gradient(dims, links, beta, c0, c1)))


def _site_step(dims, site: int, d: int, step: int) -> int:
    c = [site % dims[0], (site // dims[0]) % dims[1], (site // (dims[0] * dims[1])) % dims[2],
         site // (dims[0] * dims[1] * dims[2])]
    c[d] = (c[d] + step) % dims[d]
    return c[0] + dims[0] * (c[1] + dims[1] * (c[2] + dims[2] * c[3]))


def link_gradient(dims, links, beta: float, mu: int, site: int) -> np.ndarray:
    """G_mu(site) alone (for sampled checks on lattices too large for `gradient`): every loop of
    the action that passes through the link, walked site by site, contributes its rest B^dag (or
    B for a daggered passage), as in `gradient`."""
    u = np.asarray(links).reshape(4, -1, 3, 3)
    g = np.zeros((3, 3), np.complex128)
    for a in range(4):
        for b in range(4):
            if a == b:
                continue
            for c, path in loops(a, b):
                n = len(path)
                # every base point whose loop uses the link: walk the path from each candidate
                # base y = site - (offset of step k), k over the steps along mu
                for k in range(n):
                    d, s = path[k]
                    if d != mu:
                        continue
                    off = np.zeros(4, dtype=int)
                    for j in range(k):
                        off[path[j][0]] += path[j][1]
                    if s < 0:
                        off[d] -= 1  # a -mu step uses U_mu at (position - mu)
                    y = site
                    for e in range(4):
                        y = _site_step(dims, y, e, -int(off[e]))
                    # factors of the loop based at y
                    facs, pos = [], y
                    for dd, ss in path:
                        if ss > 0:
                            facs.append(u[dd, pos])
                            pos = _site_step(dims, pos, dd, 1)
                        else:
                            pos = _site_step(dims, pos, dd, -1)
                            facs.append(u[dd, pos].conj().T)
                    rest = np.eye(3, dtype=np.complex128)
                    for j in list(range(k + 1, n)) + list(range(k)):
                        rest = rest @ facs[j]
                    g += (-beta / 3.0 * c) * (rest if s < 0 else rest.conj().T)
    return g
