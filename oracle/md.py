"""FP64 CPU oracle of the RHMC molecular dynamics (numpy over the other oracle modules).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the CPU-baseline leg
of the benchmark use this module; the product path never imports it.  It
shares no code with the CUDA library.

The MD of Sec. 2-3 evolves links U and traceless Hermitian momenta H under
(1/2) sum tr H^2 + S(U): U' = i H U, H' = -i F with F = TA(U G^dag) the
Lie-algebra force (G = dS/dRe U + i dS/dIm U).  S = S_g (tree-level Symanzik,
oracle.gauge) + sum over pseudofermions of sum_i r_i Re(b^dag x_i) on the
k-times stout-smeared links (oracle.stout, oracle.mscg, oracle.force).
Momenta from standard normal numbers: H = sum_a xi_a lambda_a / sqrt(2).
"""
from __future__ import annotations

import numpy as np

import oracle
from oracle import gauge as og
from oracle import stout as ost

OMELYAN_LAMBDA = 0.1931833275037836


def gell_mann() -> np.ndarray:
    lam = np.zeros((8, 3, 3), np.complex128)
    lam[0][0, 1] = lam[0][1, 0] = 1
    lam[1][0, 1], lam[1][1, 0] = -1j, 1j
    lam[2][0, 0], lam[2][1, 1] = 1, -1
    lam[3][0, 2] = lam[3][2, 0] = 1
    lam[4][0, 2], lam[4][2, 0] = -1j, 1j
    lam[5][1, 2] = lam[5][2, 1] = 1
    lam[6][1, 2], lam[6][2, 1] = -1j, 1j
    lam[7] = np.diag([1, 1, -2]) / np.sqrt(3)
    return lam


def momenta(xi) -> np.ndarray:
    """H [4][V][3][3] from xi [4][V][8]."""
    return np.einsum("lsa,aij->lsij", np.asarray(xi), gell_mann()) / np.sqrt(2.0)


def kinetic(h) -> float:
    return 0.5 * float(np.einsum("lsij,lsji->", h, h).real)


def update_links(u, h, eps):
    w, v = np.linalg.eigh(eps * h)
    e = (v * np.exp(1j * w)[..., None, :]) @ np.conj(np.swapaxes(v, -1, -2))
    return e @ u


class Action:
    def __init__(self, dims, beta, mass=0.0, pseudofermions=(), stout_rho=0.0, stout_steps=0, tol=1e-13, theta=None):
        self.dims, self.beta, self.mass = dims, beta, mass
        self.pf = list(pseudofermions)  # (b, shifts, residues)
        self.rho, self.nstout, self.tol = stout_rho, stout_steps, tol
        self.theta = theta  # U(1) phases of the fermion links [4][V] (None: none)

    def _dirac_links(self, uk):
        return uk if self.theta is None else oracle.u1_links(uk, self.theta)

    def _levels(self, u):
        return ost.stout(self.dims, u, self.rho, self.nstout)

    def value(self, u) -> float:
        s = og.action(self.dims, u, self.beta) if self.beta != 0.0 else 0.0
        if self.pf:
            uk = self._dirac_links(self._levels(u)[-1])
            for b, shifts, res in self.pf:
                x = oracle.mscg(self.dims, uk, self.mass, np.asarray(shifts), b, tol=self.tol)["x"]
                s += oracle.action(np.asarray(res), b, x)
        return s

    def gauge_force(self, u) -> np.ndarray:
        return og.force(self.dims, u, self.beta) if self.beta != 0.0 else np.zeros_like(u)

    def fermion_force(self, u) -> np.ndarray:
        f = np.zeros_like(u)
        if self.pf:
            levels = self._levels(u)
            for b, shifts, res in self.pf:
                x = oracle.mscg(self.dims, self._dirac_links(levels[-1]), self.mass, np.asarray(shifts), b,
                                tol=self.tol)["x"]
                if self.theta is None:
                    gk = oracle.force(self.dims, levels[-1], np.asarray(res), x, kind=1)
                else:
                    gk = oracle.force_u1(self.dims, levels[-1], self.theta, np.asarray(res), x, kind=1)
                f = f + ost.lie_force(u, ost.stout_backward(self.dims, levels, self.rho, gk))
        return f

    def force(self, u) -> np.ndarray:
        return self.gauge_force(u) + self.fermion_force(u)


def _kick(h, f, eps):
    return h - eps * 1j * f


def leapfrog(action: Action, u, h, tau, nsteps):
    eps = tau / nsteps
    h = _kick(h, action.force(u), 0.5 * eps)
    for k in range(nsteps):
        u = update_links(u, h, eps)
        h = _kick(h, action.force(u), eps if k < nsteps - 1 else 0.5 * eps)
    return u, h


def omelyan(action: Action, u, h, tau, nsteps, lam=OMELYAN_LAMBDA):
    eps = tau / nsteps
    h = _kick(h, action.force(u), lam * eps)
    for k in range(nsteps):
        u = update_links(u, h, 0.5 * eps)
        h = _kick(h, action.force(u), (1.0 - 2.0 * lam) * eps)
        u = update_links(u, h, 0.5 * eps)
        h = _kick(h, action.force(u), (2.0 if k < nsteps - 1 else 1.0) * lam * eps)
    return u, h


def omelyan_multiscale(action: Action, u, h, tau, nsteps, gauge_substeps, lam=OMELYAN_LAMBDA):
    """Nested Omelyan: the fermion force on the outer level, each outer link update an Omelyan
    integration under the gauge force with gauge_substeps steps."""
    state = {"u": u, "h": h}

    def omel(kick, drift, t, n):
        eps = t / n
        kick(lam * eps)
        for k in range(n):
            drift(0.5 * eps)
            kick((1.0 - 2.0 * lam) * eps)
            drift(0.5 * eps)
            kick((2.0 if k < n - 1 else 1.0) * lam * eps)

    def kick_g(e):
        state["h"] = _kick(state["h"], action.gauge_force(state["u"]), e)

    def kick_f(e):
        state["h"] = _kick(state["h"], action.fermion_force(state["u"]), e)

    def drift_u(e):
        state["u"] = update_links(state["u"], state["h"], e)

    omel(kick_f, lambda t: omel(kick_g, drift_u, t, gauge_substeps), tau, nsteps)
    return state["u"], state["h"]
