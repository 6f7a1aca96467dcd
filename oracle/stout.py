"""FP64 CPU oracle of stout smearing and of its force chain rule (numpy).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the CPU-baseline leg
of the benchmark use this module; the product path never imports it.  It
shares no code with the CUDA library.

Stout smearing (the k-times smeared links U^(k) that the Dirac operator uses,
Sec. 2; the smearing step is Morningstar and Peardon's, cited there):

    C_mu(x)  = rho * sum_{nu != mu} [ U_nu(x) U_mu(x+nu) U_nu(x+mu)^dag
                                     + U_nu(x-nu)^dag U_mu(x-nu) U_nu(x-nu+mu) ]
    Omega    = C_mu(x) U_mu(x)^dag
    i Q      = TA(Omega) = (Omega - Omega^dag)/2 - tr(Omega - Omega^dag)/6
    U'_mu(x) = exp(i Q) U_mu(x)

Links are periodic in all four directions (the antiperiodic sign belongs to
the fermion phases, not to the gauge field).  The matrix exponential of the
Hermitian Q is taken from numpy's Hermitian eigendecomposition.

Force chain rule (Sec. 3: the MD evolves U^(0) while the fermion action
depends on U^(k)): gradients use torch's convention for a real function S of
complex matrices, G = dS/dRe U + i dS/dIm U, so that dS = Re tr(G^dag dU).  One
smearing step is pulled back by reverse-mode differentiation of the four
formulas above, in their order:
* U' = E U:              G_E = G' U^dag,  G_U += E^dag G'
* E = exp(A), A = i Q:   G_A = L_exp(A^dag, G_E), the adjoint of the Frechet
                         derivative of exp (scipy.linalg.expm_frechet)
* A = TA(Omega):         G_Omega = TA(G_A)  (TA is an orthogonal projection)
* Omega = C U^dag:       G_C = G_Omega U,  G_U += G_Omega^dag C
* C = rho sum(staples):  each staple product A B C^dag / A^dag B C passes G_C
                         on to its three links by the product rule.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg


def _grid(dims, links):
    lx, ly, lz, lt = dims
    return np.asarray(links, dtype=np.complex128).reshape(4, lt, lz, ly, lx, 3, 3)


def _flat(dims, u):
    return u.reshape(4, -1, 3, 3)


def _shift(a, nu: int, step: int):
    """a(x + step * nu) for a site field with axes (t, z, y, x, ...)."""
    return np.roll(a, -step, axis=3 - nu)


def _dag(a):
    return np.swapaxes(a.conj(), -1, -2)


def ta(x):
    """Traceless anti-Hermitian part (X - X^dag)/2 - tr(X - X^dag)/6."""
    y = 0.5 * (x - _dag(x))
    tr = np.trace(y, axis1=-2, axis2=-1) / 3.0
    return y - tr[..., None, None] * np.eye(3)


def staples(dims, links):
    """Unweighted staple sum C_mu(x)/rho, links and result [4][V][3][3]."""
    u = _grid(dims, links)
    c = np.zeros_like(u)
    for mu in range(4):
        for nu in range(4):
            if nu == mu:
                continue
            up = u[nu] @ _shift(u[mu], nu, 1) @ _dag(_shift(u[nu], mu, 1))
            dn_at = _dag(u[nu]) @ u[mu] @ _shift(u[nu], mu, 1)  # staple of C_mu(x + nu)
            c[mu] += up + _shift(dn_at, nu, -1)
    return _flat(dims, c)


def _exp_i_hermitian(q):
    """exp(i Q) for stacked Hermitian 3x3 Q."""
    w, v = np.linalg.eigh(q)
    return (v * np.exp(1j * w)[..., None, :]) @ _dag(v)


def stout_step(dims, links, rho: float):
    """One stout smearing step U -> exp(i Q) U; links [4][V][3][3]."""
    u = np.asarray(links, dtype=np.complex128).reshape(4, -1, 3, 3)
    omega = rho * staples(dims, u) @ _dag(u)
    q = -1j * ta(omega)
    return _exp_i_hermitian(q) @ u


def stout(dims, links, rho: float, nstep: int):
    """[U^(0), U^(1), ..., U^(nstep)], each [4][V][3][3]."""
    levels = [np.asarray(links, dtype=np.complex128).reshape(4, -1, 3, 3)]
    for _ in range(nstep):
        levels.append(stout_step(dims, levels[-1], rho))
    return levels


def _staple_backward(dims, links, gc):
    """dS/dU from G_C = dS/dC0 with C0 = staples(U) (unweighted)."""
    u = _grid(dims, links)
    g = _grid(dims, gc)
    out = np.zeros_like(u)
    for mu in range(4):
        for nu in range(4):
            if nu == mu:
                continue
            # upper staple A B C^dag at x: A = U_nu(x), B = U_mu(x+nu), C = U_nu(x+mu)
            a, b, cc = u[nu], _shift(u[mu], nu, 1), _shift(u[nu], mu, 1)
            gx = g[mu]
            out[nu] += gx @ cc @ _dag(b)                        # -> U_nu(x)
            out[mu] += _shift(_dag(a) @ gx @ cc, nu, -1)         # -> U_mu(x+nu)
            out[nu] += _shift(_dag(gx) @ a @ b, mu, -1)          # -> U_nu(x+mu)
            # lower staple of C_mu(x+nu): A^dag B C, A = U_nu(x), B = U_mu(x), C = U_nu(x+mu)
            a, b, cc = u[nu], u[mu], _shift(u[nu], mu, 1)
            gx = _shift(g[mu], nu, 1)
            out[nu] += b @ cc @ _dag(gx)                        # -> U_nu(x)
            out[mu] += a @ gx @ _dag(cc)                        # -> U_mu(x)
            out[nu] += _shift(_dag(b) @ a @ gx, mu, -1)          # -> U_nu(x+mu)
    return _flat(dims, out)


def stout_step_backward(dims, links, rho: float, grad_out):
    """dS/dU given dS/dU' for U' = stout_step(U); torch's complex-gradient convention."""
    u = np.asarray(links, dtype=np.complex128).reshape(4, -1, 3, 3)
    gp = np.asarray(grad_out, dtype=np.complex128).reshape(4, -1, 3, 3)
    c = rho * staples(dims, u)
    omega = c @ _dag(u)
    a = ta(omega)
    e = _exp_i_hermitian(-1j * a)
    g_e = gp @ _dag(u)
    g_a = np.empty_like(a)
    for mu in range(4):
        for i in range(a.shape[1]):
            g_a[mu, i] = scipy.linalg.expm_frechet(_dag(a[mu, i]), g_e[mu, i], compute_expm=False)
    g_omega = ta(g_a)
    g_u = _dag(e) @ gp + _dag(g_omega) @ c
    g_u += rho * _staple_backward(dims, u, g_omega @ u)
    return g_u


def stout_backward(dims, levels, rho: float, grad_top):
    """dS/dU^(0) given the levels [U^(0)..U^(k)] and dS/dU^(k)."""
    g = np.asarray(grad_top, dtype=np.complex128).reshape(4, -1, 3, 3)
    for lev in reversed(levels[:-1]):
        g = stout_step_backward(dims, lev, rho, g)
    return g


def lie_force(links, grad):
    """F = TA(U G^dag): dS/deps = tr(X F) along U -> exp(eps X) U, X in su(3)."""
    u = np.asarray(links, dtype=np.complex128).reshape(4, -1, 3, 3)
    return ta(u @ _dag(np.asarray(grad).reshape(u.shape)))


def _neighbour(dims, site: int, mu: int, step: int) -> int:
    c = [site % dims[0], (site // dims[0]) % dims[1], (site // (dims[0] * dims[1])) % dims[2],
         site // (dims[0] * dims[1] * dims[2])]
    c[mu] = (c[mu] + step) % dims[mu]
    return c[0] + dims[0] * (c[1] + dims[1] * (c[2] + dims[2] * c[3]))


def smeared_link(dims, links, rho: float, nstep: int, mu: int, site: int, _memo=None) -> np.ndarray:
    """U^(nstep)_mu(site) alone, from the links it depends on (for sampled checks on lattices
    too large for the whole-lattice routines); same formulas as stout_step."""
    memo = {} if _memo is None else _memo
    key = (nstep, mu, site)
    if key in memo:
        return memo[key]
    u = np.asarray(links).reshape(4, -1, 3, 3)
    if nstep == 0:
        return u[mu, site]

    def lk(nu, s):
        return smeared_link(dims, u, rho, nstep - 1, nu, s, memo)

    c = np.zeros((3, 3), np.complex128)
    for nu in range(4):
        if nu == mu:
            continue
        xp_nu, xp_mu = _neighbour(dims, site, nu, 1), _neighbour(dims, site, mu, 1)
        c += lk(nu, site) @ lk(mu, xp_nu) @ lk(nu, xp_mu).conj().T
        xm = _neighbour(dims, site, nu, -1)
        c += lk(nu, xm).conj().T @ lk(mu, xm) @ lk(nu, _neighbour(dims, xm, mu, 1))
    u_prev = lk(mu, site)
    q = -1j * ta(rho * c @ u_prev.conj().T)
    out = _exp_i_hermitian(q) @ u_prev
    memo[key] = out
    return out
