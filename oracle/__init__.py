"""Python bindings of the FP64 CPU oracle (oracle.c).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the CPU-baseline
leg of the benchmark use this package; the product path never imports it.
It shares no code with the CUDA library.  The shared object is built with
gcc by ``build()`` (plain -O2, no fast-math).

All fields are numpy complex128 in the canonical layouts documented in
``synthetic``: links [4][V][3][3], half fields [Vh][3].
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (OpenMP over sites, -O2, no fast-math)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.run(["gcc", "-O2", "-std=c99", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"],
                       check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        I = ctypes.c_int
        D = ctypes.c_double
        lib.oracle_dslash_full.argtypes = [P, I, P, P, P]
        lib.oracle_dslash_eo.argtypes = [P, I, P, I, P, P]
        lib.oracle_normal_op.argtypes = [P, I, P, D, D, P, P]
        lib.oracle_true_residual.argtypes = [P, I, P, D, D, P, P]
        lib.oracle_true_residual.restype = D
        lib.oracle_cg.argtypes = [P, I, P, D, D, D, I, P, P]
        lib.oracle_mscg.argtypes = [P, I, P, D, I, P, D, I, P, P, P, P, P, P, I, I]
        lib.oracle_set_num_threads.argtypes = [I]
        lib.oracle_force.argtypes = [P, I, P, I, P, P, P, I]
        lib.oracle_num_threads.restype = I
        _lib = lib
    return _lib


def _dims(dims) -> np.ndarray:
    d = np.ascontiguousarray(np.asarray(dims, dtype=np.int32))
    if d.shape != (4,) or np.any(d < 2) or np.any(d % 2):
        raise ValueError("dims must be four even extents >= 2")
    return d


def _c128(a, shape=None) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(a, dtype=np.complex128))
    if shape is not None and a.shape != tuple(shape):
        a = a.reshape(shape)
    return a


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def volume(dims) -> int:
    d = _dims(dims)
    return int(np.prod(d.astype(np.int64)))


def num_threads() -> int:
    return int(_load().oracle_num_threads())


def set_num_threads(n: int) -> None:
    """OpenMP threads of the following oracle calls."""
    _load().oracle_set_num_threads(int(n))


def dslash_full(dims, links, psi, antiperiodic: bool = True) -> np.ndarray:
    """D psi on the full lattice, psi [V][3]."""
    d = _dims(dims)
    v = volume(d)
    u = _c128(links, (4, v, 3, 3))
    x = _c128(psi, (v, 3))
    out = np.empty((v, 3), np.complex128)
    _load().oracle_dslash_full(_ptr(d), int(antiperiodic), _ptr(u), _ptr(x), _ptr(out))
    return out


def dslash(dims, links, out_parity: int, psi, antiperiodic: bool = True) -> np.ndarray:
    """D_eo psi_o (out_parity 0) or D_oe psi_e (out_parity 1); psi [Vh][3]."""
    d = _dims(dims)
    v = volume(d)
    u = _c128(links, (4, v, 3, 3))
    x = _c128(psi, (v // 2, 3))
    out = np.empty((v // 2, 3), np.complex128)
    rc = _load().oracle_dslash_eo(_ptr(d), int(antiperiodic), _ptr(u), int(out_parity), _ptr(x), _ptr(out))
    if rc:
        raise MemoryError("oracle_dslash_eo")
    return out


def dslash_eo(dims, links, psi_odd, antiperiodic: bool = True) -> np.ndarray:
    return dslash(dims, links, 0, psi_odd, antiperiodic)


def dslash_oe(dims, links, psi_even, antiperiodic: bool = True) -> np.ndarray:
    return dslash(dims, links, 1, psi_even, antiperiodic)


def normal_op(dims, links, mass: float, sigma: float, psi_even, antiperiodic: bool = True) -> np.ndarray:
    """(m^2 + sigma) psi - D_eo D_oe psi on even sites."""
    d = _dims(dims)
    v = volume(d)
    u = _c128(links, (4, v, 3, 3))
    x = _c128(psi_even, (v // 2, 3))
    out = np.empty((v // 2, 3), np.complex128)
    rc = _load().oracle_normal_op(_ptr(d), int(antiperiodic), _ptr(u), float(mass), float(sigma), _ptr(x), _ptr(out))
    if rc:
        raise MemoryError("oracle_normal_op")
    return out


def true_residual(dims, links, mass, sigma, b, x, antiperiodic: bool = True) -> float:
    d = _dims(dims)
    v = volume(d)
    u = _c128(links, (4, v, 3, 3))
    bb = _c128(b, (v // 2, 3))
    xx = _c128(x, (v // 2, 3))
    return float(_load().oracle_true_residual(_ptr(d), int(antiperiodic), _ptr(u), float(mass), float(sigma),
                                              _ptr(bb), _ptr(xx)))


def cg(dims, links, mass, sigma, b, x0=None, tol=1e-10, max_iter=10000, antiperiodic: bool = True):
    """Plain CG on A_sigma x = b from x0; returns (x, iterations)."""
    d = _dims(dims)
    v = volume(d)
    u = _c128(links, (4, v, 3, 3))
    bb = _c128(b, (v // 2, 3))
    x = np.zeros((v // 2, 3), np.complex128) if x0 is None else _c128(x0, (v // 2, 3)).copy()
    it = _load().oracle_cg(_ptr(d), int(antiperiodic), _ptr(u), float(mass), float(sigma), float(tol),
                           int(max_iter), _ptr(bb), _ptr(x))
    if it < 0:
        raise MemoryError("oracle_cg")
    return x, int(it)


def mscg(dims, links, mass, shifts, b, tol=1e-10, max_iter=20000, log_rows: int = 0, antiperiodic: bool = True,
         finish: bool = True):
    """Multi-shift CG.  Returns dict(x [nshift][Vh][3], true_resid, shift_iters,
    iters, refine_iters, scalar_log [log_rows][2+nshift] or None).  finish=False stops after the
    multi-shift iterations (no true residuals, which are then -1, and no refinement)."""
    d = _dims(dims)
    v = volume(d)
    u = _c128(links, (4, v, 3, 3))
    bb = _c128(b, (v // 2, 3))
    sig = np.ascontiguousarray(np.asarray(shifts, dtype=np.float64))
    ns = sig.size
    x = np.empty((ns, v // 2, 3), np.complex128)
    tr = np.empty(ns, np.float64)
    si = np.empty(ns, np.int32)
    ri = np.zeros(1, np.int32)
    log = np.zeros((max(log_rows, 1), 2 + ns), np.float64)
    it = _load().oracle_mscg(_ptr(d), int(antiperiodic), _ptr(u), float(mass), ns, _ptr(sig), float(tol),
                             int(max_iter), _ptr(bb), _ptr(x), _ptr(tr), _ptr(si), _ptr(ri),
                             _ptr(log) if log_rows > 0 else None, int(log_rows), int(bool(finish)))
    if it < 0:
        raise MemoryError("oracle_mscg")
    return dict(x=x, true_resid=tr, shift_iters=si, iters=int(it), refine_iters=int(ri[0]),
                scalar_log=log[:min(log_rows, it)] if log_rows > 0 else None)


def force(dims, links, residues, x, kind: int = 0, antiperiodic: bool = True) -> np.ndarray:
    """Fermion force per link [4][V][3][3]: kind 0 -> TA(U W), kind 1 -> W^dag."""
    d = _dims(dims)
    v = volume(d)
    u = _c128(links, (4, v, 3, 3))
    res = np.ascontiguousarray(np.asarray(residues, dtype=np.float64))
    xs = _c128(x, (res.size, v // 2, 3))
    out = np.empty((4, v, 3, 3), np.complex128)
    rc = _load().oracle_force(_ptr(d), int(antiperiodic), _ptr(u), int(res.size), _ptr(res), _ptr(xs), _ptr(out),
                              int(kind))
    if rc:
        raise MemoryError("oracle_force")
    return out


def action(residues, b, x, alpha0: float = 0.0) -> float:
    """S = alpha0 |b|^2 + sum_i r_i Re(b^dag x_i) (Sec. 2: the pseudofermion action b^dag R(A) b with
    the rational function R written as a constant plus poles, x_i the solutions of the shifted
    systems)."""
    b = np.asarray(b).reshape(-1)
    s = alpha0 * np.vdot(b, b).real
    return float(s + sum(r * np.vdot(b, np.asarray(xi).reshape(-1)).real for r, xi in zip(residues, x)))


def u1_links(links, theta) -> np.ndarray:
    """Links times their U(1) phases: exp(i theta_mu(x)) U_mu(x), theta [4][V] in radians (the
    per-flavour phase field u_mu = exp(i theta_mu) of Sec. 4.1, on top of the staggered signs)."""
    return _c128(links).reshape(4, -1, 3, 3) * np.exp(1j * np.asarray(theta, dtype=np.float64))[..., None, None]


def force_u1(dims, links, theta, residues, x, kind: int = 0, antiperiodic: bool = True) -> np.ndarray:
    """Fermion force with respect to U when D uses exp(i theta) U: kind 0 -> TA(U W) (equal to the
    force of the phased links V = exp(i theta) U), kind 1 -> dS/dRe U + i dS/dIm U =
    exp(-i theta) times the gradient with respect to V (V = exp(i theta) U, dV = exp(i theta) dU)."""
    v = u1_links(links, theta)
    f = force(dims, v, residues, x, kind=kind, antiperiodic=antiperiodic)
    if kind == 1:
        f = f * np.exp(-1j * np.asarray(theta, dtype=np.float64))[..., None, None]
    return f
