"""Rational approximations for the RHMC (Sec. 2: the fractional power of the Dirac operator is
approximated to machine precision by a rational function, applied as a sum over poles by the
multi-shift solver, Eq. shift_eo).

remez(power, n, lo, hi) returns the minimax approximation, in relative error on [lo, hi], of
x**power by a rational function of type (n, n), in the partial-fraction form the solver needs:

    x**power ~= alpha0 + sum_i residues[i] / (x + poles[i])

found with Remez's exchange algorithm for rational functions: on 2n+2 alternation points the
linearised equations N(x_j) - f(x_j) D(x_j) = (-1)^j E f(x_j) D(x_j) are solved for the 2n+1 free
coefficients of the numerator N and the monic denominator D and the levelled error E (iterating on
E), then the alternation set moves to the extrema of the error, until the extrema equal |E|.  The
arithmetic is mpmath's arbitrary precision (the normal equations of a wide-range approximation are
far too ill-conditioned for FP64); the host-side cost is seconds and the result is reused for a
whole simulation.  The heatbath uses power = +1/(2 n_f) type roots, the action and the force -1/4
and similar; for power in (-1, 0) and (0, 1) the poles come out real and positive.
"""
from __future__ import annotations

import math
from dataclasses import dataclass


@dataclass
class RationalApprox:
    power: float
    lo: float
    hi: float
    alpha0: float
    residues: list
    poles: list
    max_rel_error: float

    def __call__(self, x):
        """Evaluate the partial-fraction form (numpy arrays or floats)."""
        out = self.alpha0
        for r, s in zip(self.residues, self.poles):
            out = out + r / (x + s)
        return out


def _mp():
    try:
        import mpmath
    except ImportError as e:  # pragma: no cover - depends on the host image
        raise ImportError("rational.remez needs mpmath for its extended-precision arithmetic") from e
    return mpmath


def remez(power: float, n: int, lo: float, hi: float, digits: int = 0, max_iter: int = 60,
          tol: float = 1e-6) -> RationalApprox:
    """Minimax relative approximation of x**power on [lo, hi] by a type-(n, n) rational function."""
    if not (0 < lo < hi) or n < 1:
        raise ValueError("remez: need 0 < lo < hi and n >= 1")
    mp = _mp()
    old = mp.mp.dps
    mp.mp.dps = digits or max(40, 12 + 4 * n)
    try:
        return _remez(mp, power, n, lo, hi, max_iter, tol)
    finally:
        mp.mp.dps = old


def _remez(mp, power, n, lo, hi, max_iter, tol):
    mpf = mp.mpf
    p = mpf(power)
    a, b = mpf(lo), mpf(hi)
    la, lb = mp.log(a), mp.log(b)

    def f(x):
        return x ** p

    m = 2 * n + 2
    # initial alternation set: Chebyshev extrema in log x
    xs = [mp.exp(la + (lb - la) * (1 - mp.cos(mp.pi * j / (m - 1))) / 2) for j in range(m)]

    def solve(xs):
        # unknowns: a_0..a_n (numerator), b_0..b_{n-1} (denominator, b_n = 1), E
        E = mpf(0)
        dprev = [mpf(1)] * m
        num = den = None
        for _ in range(50):
            A = mp.matrix(m, m)
            rhs = mp.matrix(m, 1)
            for j, x in enumerate(xs):
                fx = f(x)
                s = 1 if j % 2 == 0 else -1
                xp = mpf(1)
                for k in range(n + 1):
                    A[j, k] = xp
                    xp *= x
                xp = mpf(1)
                for k in range(n):
                    A[j, n + 1 + k] = -fx * xp
                    xp *= x
                A[j, m - 1] = -s * fx * dprev[j]
                rhs[j] = fx * x ** n
            sol = mp.lu_solve(A, rhs)
            num = [sol[k] for k in range(n + 1)]
            den = [sol[n + 1 + k] for k in range(n)] + [mpf(1)]
            E_new = sol[m - 1]
            dprev = [mp.polyval(den[::-1], x) for x in xs]
            if abs(E_new - E) <= abs(E_new) * mpf(10) ** (-(mp.mp.dps // 2)):
                E = E_new
                break
            E = E_new
        return num, den, E

    def err(num, den, x):
        return mp.polyval(num[::-1], x) / (mp.polyval(den[::-1], x) * f(x)) - 1

    for _ in range(max_iter):
        num, den, E = solve(xs)
        # locate the zeros of the error between consecutive alternation points (bisection in log x)
        zeros = []
        for j in range(m - 1):
            u0, u1 = mp.log(xs[j]), mp.log(xs[j + 1])
            e0 = err(num, den, mp.exp(u0))
            for _b in range(80):
                um = (u0 + u1) / 2
                em = err(num, den, mp.exp(um))
                if (em > 0) == (e0 > 0):
                    u0, e0 = um, em
                else:
                    u1 = um
            zeros.append((u0 + u1) / 2)
        # extremum of |error| on each interval between zeros (golden section in log x)
        bounds = [la] + zeros + [lb]
        new = []
        gr = (mp.sqrt(5) - 1) / 2
        for j in range(m):
            u0, u1 = bounds[j], bounds[j + 1]
            c = u1 - gr * (u1 - u0)
            d = u0 + gr * (u1 - u0)
            fc, fd = abs(err(num, den, mp.exp(c))), abs(err(num, den, mp.exp(d)))
            for _g in range(90):
                if fc > fd:
                    u1, d, fd = d, c, fc
                    c = u1 - gr * (u1 - u0)
                    fc = abs(err(num, den, mp.exp(c)))
                else:
                    u0, c, fc = c, d, fd
                    d = u0 + gr * (u1 - u0)
                    fd = abs(err(num, den, mp.exp(d)))
            best = (c + d) / 2
            cand = [best]
            if j == 0:
                cand.append(la)
            if j == m - 1:
                cand.append(lb)
            best = max(cand, key=lambda u: abs(err(num, den, mp.exp(u))))
            new.append(mp.exp(best))
        emax = max(abs(err(num, den, x)) for x in new)
        xs = new
        if emax - abs(E) <= mpf(tol) * abs(E):
            break
    else:
        raise RuntimeError("remez: no convergence")

    # partial fractions: D has n real negative roots -poles; residues N(-s)/D'(-s)
    roots = mp.polyroots(den[::-1], maxsteps=400, extraprec=4 * mp.mp.dps)
    dder = [k * den[k] for k in range(1, n + 1)]
    poles, residues = [], []
    for r in roots:
        r = mp.re(r) if abs(mp.im(r)) < mpf(10) ** (-(mp.mp.dps // 3)) else r
        if not isinstance(r, type(mpf(0))):
            raise RuntimeError("remez: complex pole; the function is not a Stieltjes-type power")
        poles.append(-r)
        residues.append(mp.polyval(num[::-1], r) / mp.polyval(dder[::-1], r))
    order = sorted(range(n), key=lambda k: poles[k])
    alpha0 = num[n]  # D is monic and deg N = deg D
    return RationalApprox(power=float(power), lo=float(lo), hi=float(hi), alpha0=float(alpha0),
                          residues=[float(residues[k]) for k in order], poles=[float(poles[k]) for k in order],
                          max_rel_error=float(emax))


def load_table(name: str = "rhmc_rational_m0.3.json") -> dict:
    """Stored approximations written by data/make_rational.py (for hosts without mpmath):
    {"heatbath": RationalApprox, "action": RationalApprox}."""
    import json
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "data", name)
    with open(path) as f:
        raw = json.load(f)
    return {k: RationalApprox(power=v["power"], lo=v["lo"], hi=v["hi"], alpha0=v["alpha0"], residues=list(v["residues"]),
                              poles=list(v["poles"]), max_rel_error=v["max_rel_error"]) for k, v in raw.items()}
