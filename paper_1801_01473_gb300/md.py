"""Molecular dynamics of the RHMC (Sec. 2: exp(-H^2/2 - S_g - S_f) sampled by MD plus an
accept/reject step; Sec. 3: each MD iteration computes the forces, evolves the momenta, then
the links).  Host-side sequencing only: every arithmetic step is a libstg kernel (gauge action and
force, stout smearing and its chain rule, multi-shift CG, fermion force, the MD link/momentum
updates, the kinetic energy and the pseudofermion action); Python only adds the few resulting
scalars of the Hamiltonian and takes the Metropolis decision.

The fermion part is S_f = sum_pf sum_i r_i Re(b^dag x_i), x_i = (m^2 + sigma_i - D_eo D_oe)^-1 b
on the k-times stout-smeared links (the pole part of the rational approximation; a constant
term has no force).  Forces are Lie-algebra forces F = TA(U G^dag) on the unsmeared links.

precision "f32" runs the molecular dynamics in single precision as Sec. 5.4 does: the gauge force,
the stout smearing and its chain rule on complex64 copies of the links (GB300 issues FP32 ~64x
faster than FP64), the fermion solve with the mixed solver on the smeared links; the MD state
(links, momenta) and its updates stay FP64, and the Hamiltonian of the Metropolis test is FP64.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Sequence

import torch

from .api import (Gauge, Lattice, complex_convert, fermion_force, gauge_action, gauge_force, md_kinetic, md_momenta,
                  md_update_links_, md_update_momenta_, mscg, mscg_batched, pseudofermion_action_value, rational_apply,
                  stout_force, stout_smear)

# Omelyan's second-order minimum-norm parameter
OMELYAN_LAMBDA = 0.1931833275037836


@dataclass
class Pseudofermion:
    b: torch.Tensor                 # even-site source [Vh, 3] complex128 (cuda)
    shifts: Sequence[float]
    residues: Sequence[float]
    alpha0: float = 0.0             # constant term of the rational approximation (no force)
    md_shifts: Sequence[float] | None = None    # optional cheaper approximation for the MD force
    md_residues: Sequence[float] | None = None  # (Sec. 2: different orders in different parts)

    def force_poles(self):
        if self.md_shifts is not None:
            return list(self.md_shifts), list(self.md_residues)
        return list(self.shifts), list(self.residues)


@dataclass
class Action:
    lattice: Lattice
    beta: float
    mass: float = 0.0
    pseudofermions: list = field(default_factory=list)
    stout_rho: float = 0.0
    stout_steps: int = 0
    tol: float = 1e-12              # stopping residual of the action (Metropolis) and heatbath solves
    md_tol: float | None = None     # stopping residual of the MD force solves (None: tol); Sec. 2 uses
                                    # different residuals in different parts of the RHMC
    inner: str | None = None        # None: FP64 solve; "f32": mixed FP32-inner solve
    precision: str = "f64"          # forces in "f64" or "f32" (the Hamiltonian is always FP64)
    theta: torch.Tensor | None = None  # U(1) phase field [4, V] on the fermion links (chemical potential, ...)

    def _smeared(self, links):
        if self.stout_steps > 0:
            levels = stout_smear(self.lattice, links, self.stout_rho, self.stout_steps)
            return levels, levels[-1].contiguous()
        return None, links

    def _gauges(self, uk):
        """The action's F64 (and FP32 inner) gauges holding uk: created once, then refreshed in place
        (no allocation per force evaluation)."""
        cache = self.__dict__.setdefault("_gauge_cache", {})
        key = (self.theta is None, self.inner)
        if cache.get("key") != key:
            cache.clear()
            cache["key"] = key
        if "g64" not in cache:
            cache["g64"] = Gauge(self.lattice, uk, "f64", 18, theta=self.theta)
            cache["gi"] = Gauge(self.lattice, uk, "f32", 12, theta=self.theta) if self.inner == "f32" else None
        else:
            cache["g64"].update(uk, self.theta)
            if cache["gi"] is not None:
                cache["gi"].update(uk, self.theta)
        return cache["g64"], cache["gi"]

    def _solve_all(self, g64, gi, tol, md=False):
        """x_i for every pseudofermion (with its MD poles if md); pseudofermions sharing a pole set
        are solved together in one batched multi-shift solve (their link loads shared, Sec. 2's
        multiple pseudofermions)."""
        groups = {}
        for k, pf in enumerate(self.pseudofermions):
            shifts = pf.force_poles()[0] if md else pf.shifts
            groups.setdefault(tuple(float(v) for v in shifts), []).append(k)
        xs = [None] * len(self.pseudofermions)
        # loose (MD) mixed solves stop their FP32 multi-shift phase at 0.3 tol rather than the library's
        # default (then 1e-9): at 32^4, m = 0.3, 10 poles, tol 1e-7 this cut the solve from 13.0 to
        # 11.4 ms with the same refinement (the certified residual is unchanged; only the split
        # between phases moves)
        itol = max(1e-9, 0.3 * tol) if (md and gi is not None) else 0.0
        for shifts, ks in groups.items():
            if len(ks) == 1:
                xs[ks[0]], _ = mscg(g64, self.pseudofermions[ks[0]].b, list(shifts), self.mass, tol=tol, g_inner=gi,
                                    inner_tol=itol)
            else:
                (x, _), = mscg_batched([(g64, gi, [self.pseudofermions[k].b for k in ks])], list(shifts), self.mass,
                                       tol=tol, inner_tol=itol)
                for j, k in enumerate(ks):
                    xs[k] = x[j]
        return xs

    def value(self, links: torch.Tensor) -> float:
        """S_g + S_f of the links."""
        s = gauge_action(self.lattice, links, self.beta)["action"] if self.beta != 0.0 else 0.0
        if self.pseudofermions:
            _, uk = self._smeared(links)
            g64, gi = self._gauges(uk)
            for pf, x in zip(self.pseudofermions, self._solve_all(g64, gi, self.tol)):
                s += pseudofermion_action_value(self.lattice, pf.b, x, pf.residues, pf.alpha0)
        return s

    def apply_force(self, links: torch.Tensor, mom: torch.Tensor, eps: float) -> None:
        """mom <- mom - eps i F(links), F the total Lie-algebra force.  The fermion forces of all
        pseudofermions are one force evaluation over the union of their (solution, residue) pairs
        (up to 32 per launch)."""
        self.apply_gauge_force(links, mom, eps)
        self.apply_fermion_force(links, mom, eps)

    def apply_gauge_force(self, links: torch.Tensor, mom: torch.Tensor, eps: float) -> None:
        """mom <- mom - eps i F_g(links), the gauge part alone (the inner time scale of multi-step MD)."""
        if self.beta == 0.0:
            return
        u = complex_convert(links, torch.complex64) if self.precision == "f32" else links
        md_update_momenta_(self.lattice, eps, gauge_force(self.lattice, u, self.beta, kind=0), mom)

    def apply_fermion_force(self, links: torch.Tensor, mom: torch.Tensor, eps: float) -> None:
        """mom <- mom - eps i F_f(links), the fermion part alone."""
        if not self.pseudofermions:
            return
        f32 = self.precision == "f32"
        u = complex_convert(links, torch.complex64) if f32 else links
        if self.stout_steps > 0:
            levels = stout_smear(self.lattice, u, self.stout_rho, self.stout_steps)
            uk = complex_convert(levels[-1], torch.complex128) if f32 else levels[-1].contiguous()
        else:
            levels, uk = None, links
        g64, gi = self._gauges(uk)
        xs = self._solve_all(g64, gi, self.md_tol if self.md_tol is not None else self.tol, md=True)
        xall = torch.cat(xs) if len(xs) > 1 else xs[0]
        rall = [float(r) for pf in self.pseudofermions for r in pf.force_poles()[1]]
        fprec = "f32" if f32 else "f64"
        for c0 in range(0, len(rall), 32):
            x, r = xall[c0:c0 + 32], rall[c0:c0 + 32]
            if levels is None:
                f = fermion_force(g64, r, x, kind=0, prec=fprec)
            else:
                gk = fermion_force(g64, r, x, kind=1, prec=fprec)
                f = stout_force(self.lattice, u, levels, self.stout_rho, gk, kind=0)
            md_update_momenta_(self.lattice, eps, f, mom)


def pseudofermion_heatbath(action: Action, links: torch.Tensor, eta: torch.Tensor, heat, act) -> Pseudofermion:
    """Pseudofermion heatbath (Sec. 2: pseudofermions are drawn at the start of the trajectory):
    phi = R_heat(A) eta on the (smeared) links, with eta complex Gaussian (density exp(-eta^dag eta),
    drawn by the caller) and R_heat ~ A^(+1/8) per rooted staggered flavour, so that phi^dag R_act(A) phi
    with R_act ~ A^(-1/4) has the distribution exp(-S_f).  heat, act: rational.RationalApprox (or any
    object with alpha0, residues, poles).  Returns the pseudofermion carrying act's poles and residues."""
    _, uk = action._smeared(links)
    g64, gi = action._gauges(uk)
    phi, _ = rational_apply(g64, eta, heat.alpha0, list(heat.residues), list(heat.poles), action.mass,
                            tol=action.tol, g_inner=gi)
    return Pseudofermion(phi, list(act.poles), list(act.residues), float(act.alpha0))


def hamiltonian(action: Action, links: torch.Tensor, mom: torch.Tensor) -> float:
    return md_kinetic(action.lattice, mom) + action.value(links)


def leapfrog(action: Action, links: torch.Tensor, mom: torch.Tensor, tau: float, nsteps: int) -> None:
    """Second-order leapfrog over trajectory length tau, in place: half momentum steps at both ends."""
    eps = tau / nsteps
    lat = action.lattice
    action.apply_force(links, mom, 0.5 * eps)
    for k in range(nsteps):
        md_update_links_(lat, eps, mom, links)
        action.apply_force(links, mom, eps if k < nsteps - 1 else 0.5 * eps)


def omelyan(action: Action, links: torch.Tensor, mom: torch.Tensor, tau: float, nsteps: int,
            lam: float = OMELYAN_LAMBDA) -> None:
    """Omelyan's second-order minimum-norm integrator (forces at lam, 1 - 2 lam, lam of each step;
    consecutive end forces merged), in place."""
    eps = tau / nsteps
    lat = action.lattice
    action.apply_force(links, mom, lam * eps)
    for k in range(nsteps):
        md_update_links_(lat, 0.5 * eps, mom, links)
        action.apply_force(links, mom, (1.0 - 2.0 * lam) * eps)
        md_update_links_(lat, 0.5 * eps, mom, links)
        action.apply_force(links, mom, (2.0 if k < nsteps - 1 else 1.0) * lam * eps)


def _omelyan_steps(kick, drift, tau: float, nsteps: int, lam: float = OMELYAN_LAMBDA) -> None:
    """Omelyan 2MN over tau in nsteps: kick(h) updates the momenta by a force step of size h,
    drift(h) evolves the links (and, in a nested integrator, everything faster) over time h."""
    eps = tau / nsteps
    kick(lam * eps)
    for k in range(nsteps):
        drift(0.5 * eps)
        kick((1.0 - 2.0 * lam) * eps)
        drift(0.5 * eps)
        kick((2.0 if k < nsteps - 1 else 1.0) * lam * eps)


def omelyan_multiscale(action: Action, links: torch.Tensor, mom: torch.Tensor, tau: float, nsteps: int,
                       gauge_substeps: int, lam: float = OMELYAN_LAMBDA) -> None:
    """Multi-step (nested time-scale) Omelyan integrator, in place: the fermion force, the expensive
    one, drives the outer level with nsteps steps; every outer link update is itself an Omelyan
    integration of the links under the gauge force alone with gauge_substeps steps (Sec. 2 lists
    multi-step integrators among the RHMC's improvements)."""
    lat = action.lattice

    def inner(h):
        _omelyan_steps(lambda e: action.apply_gauge_force(links, mom, e),
                       lambda e: md_update_links_(lat, e, mom, links), h, gauge_substeps, lam)

    _omelyan_steps(lambda e: action.apply_fermion_force(links, mom, e), inner, tau, nsteps, lam)


def trajectory(action: Action, links: torch.Tensor, xi: torch.Tensor, tau: float, nsteps: int,
               uniform: float, integrator: str = "omelyan", gauge_substeps: int = 1) -> dict:
    """One RHMC trajectory from links (not modified): momentum heatbath from the standard normal
    numbers xi [4, V, 8], MD to tau, Metropolis test against the uniform number in [0, 1).
    Returns the new links (the old ones if rejected), dH and the decision."""
    mom = md_momenta(action.lattice, xi)
    h0 = hamiltonian(action, links, mom)
    u = links.clone()
    if integrator == "omelyan" and gauge_substeps > 1:
        omelyan_multiscale(action, u, mom, tau, nsteps, gauge_substeps)
    else:
        (omelyan if integrator == "omelyan" else leapfrog)(action, u, mom, tau, nsteps)
    h1 = hamiltonian(action, u, mom)
    dh = h1 - h0
    accept = uniform < math.exp(min(0.0, -dh))
    return {"links": u if accept else links, "dH": dh, "accepted": accept}
