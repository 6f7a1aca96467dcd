"""Python binding of the C ABI (include/stg.h) on torch tensors.

Argument marshalling only: every arithmetic step runs in libstg's CUDA
kernels.  Torch supplies device memory and the current CUDA stream.

Tensors:
  links      complex128 [4, V, 3, 3] (or [4, Lt, Lz, Ly, Lx, 3, 3]) on the GPU
  fields     complex128 [Vh, 3] canonical, half-index order of one parity
  internal   float64 [6*Vh] (F64) or float32 [6*Vh] (F32) in the library's layout
A host (CPU) tensor passed where a canonical field is expected is copied to the
device first and results are copied back: that is the end-to-end path.
"""
from __future__ import annotations

import ctypes
from typing import Sequence

import torch

from .lib import (PREC, STG_ERR_NOCONV, STG_F32, STG_F64, STG_RECON12, STG_RECON18, Instance, MscgParams,
                  MscgStats, check, lib)


# internal field tensors: dtype and elements per site for each vector precision
_FIELD = {"f64": (torch.float64, 6), "f32": (torch.float32, 6), "ds": (torch.float32, 12)}


def _stream(stream=None) -> ctypes.c_void_p:
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t: torch.Tensor) -> ctypes.c_void_p:
    return ctypes.c_void_p(t.data_ptr())


def _dev(t, dtype=torch.complex128) -> torch.Tensor:
    if not isinstance(t, torch.Tensor):
        t = torch.as_tensor(t)
    if not t.is_cuda:
        t = t.to("cuda", non_blocking=True)
    if t.dtype != dtype:
        raise TypeError(f"expected {dtype}, got {t.dtype}")
    return t.contiguous()


class Lattice:
    """Lattice geometry: dims (Lx, Ly, Lz, Lt), all even; antiperiodic in time by default."""

    def __init__(self, dims: Sequence[int], antiperiodic: bool = True):
        self.dims = tuple(int(d) for d in dims)
        arr = (ctypes.c_int32 * 4)(*self.dims)
        h = ctypes.c_void_p()
        check(lib().stg_lattice_create(arr, int(bool(antiperiodic)), ctypes.byref(h)), "stg_lattice_create")
        self._h = h
        self.antiperiodic = bool(antiperiodic)
        self.V = int(lib().stg_lattice_sites(h, -1))
        self.Vh = int(lib().stg_lattice_sites(h, 0))

    @classmethod
    def slab(cls, dims_local: Sequence[int], t0: int, lt_global: int, antiperiodic: bool = True) -> "Lattice":
        """The slab of global time slices [t0, t0 + Lt_loc) of a lattice split along t
        (stg_lattice_create_slab): stored with two halo-side slices below and above."""
        self = cls.__new__(cls)
        dl = tuple(int(d) for d in dims_local)
        arr = (ctypes.c_int32 * 4)(*dl)
        h = ctypes.c_void_p()
        check(lib().stg_lattice_create_slab(arr, int(t0), int(lt_global), int(bool(antiperiodic)), ctypes.byref(h)),
              "stg_lattice_create_slab")
        self._h = h
        self.antiperiodic = bool(antiperiodic)
        self.dims = (dl[0], dl[1], dl[2], dl[3] + 4)  # stored extents
        self.dims_local = dl
        self.t0 = int(t0)
        self.lt_global = int(lt_global)
        self.V = int(lib().stg_lattice_sites(h, -1))
        self.Vh = int(lib().stg_lattice_sites(h, 0))
        return self

    @property
    def handle(self):
        return self._h

    def field_bytes(self, prec: str) -> int:
        return int(lib().stg_field_bytes(self._h, PREC[prec]))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            lib().stg_lattice_destroy(h)
            self._h = None


class Gauge:
    """Library-owned copy of the links at precision prec ('f64', 'f32', 'bf16', 'f16', 'ds'),
    18-real or 12-real (recon=12: rows 1, 2 stored, row 3 rebuilt); theta [4, V] float64 (optional)
    attaches a U(1) phase field exp(i theta) to the links."""

    def __init__(self, lattice: Lattice, links: torch.Tensor, prec: str = "f64", recon: int = 18, stream=None,
                 theta: torch.Tensor | None = None):
        links = _dev(links).reshape(4, lattice.V, 3, 3)
        h = ctypes.c_void_p()
        rc = STG_RECON12 if recon == 12 else STG_RECON18
        if theta is None:
            check(lib().stg_gauge_create(lattice.handle, _ptr(links), PREC[prec], rc, _stream(stream), ctypes.byref(h)),
                  "stg_gauge_create")
        else:
            th = _dev(theta, torch.float64).reshape(4, lattice.V)
            check(lib().stg_gauge_create_u1(lattice.handle, _ptr(links), _ptr(th), PREC[prec], rc, _stream(stream),
                                            ctypes.byref(h)), "stg_gauge_create_u1")
        torch.cuda.current_stream().synchronize() if stream is None else stream.synchronize()
        self._h = h
        self.lattice = lattice
        self.prec = prec
        self.recon = recon
        self.vec_prec = prec if prec in ("f64", "ds") else "f32"
        self.nbytes = int(lib().stg_gauge_bytes(h))

    @property
    def handle(self):
        return self._h

    def update(self, links: torch.Tensor, theta: torch.Tensor | None = None, stream=None) -> "Gauge":
        """Replace the links (and, for a gauge created with theta, the phases) in place, without
        allocating (stg_gauge_update)."""
        links = _dev(links).reshape(4, self.lattice.V, 3, 3)
        th = _dev(theta, torch.float64).reshape(4, self.lattice.V) if theta is not None else None
        check(lib().stg_gauge_update(self._h, _ptr(links), _ptr(th) if th is not None else None, _stream(stream)),
              "stg_gauge_update")
        torch.cuda.current_stream().synchronize() if stream is None else stream.synchronize()
        return self

    def new_field(self, n: int | None = None) -> torch.Tensor:
        """Uninitialised internal-layout field(s) at this gauge's vector precision."""
        dt, per = _FIELD[self.vec_prec]
        shape = (per * self.lattice.Vh,) if n is None else (n, per * self.lattice.Vh)
        return torch.empty(shape, dtype=dt, device="cuda")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            lib().stg_gauge_destroy(h)
            self._h = None


# ------------------------------------------------------------------ fields

def pack(lattice: Lattice, canon: torch.Tensor, prec: str = "f64", stream=None) -> torch.Tensor:
    """Canonical complex128 [Vh, 3] -> internal layout (float64 [6*Vh] for f64, float32 [6*Vh]
    for f32, float32 [12*Vh] for ds)."""
    canon = _dev(canon).reshape(lattice.Vh, 3)
    dt, per = _FIELD[prec]
    out = torch.empty(per * lattice.Vh, dtype=dt, device="cuda")
    check(lib().stg_field_pack(lattice.handle, PREC[prec], _ptr(canon), _ptr(out), _stream(stream)), "stg_field_pack")
    return out


def unpack(lattice: Lattice, internal: torch.Tensor, stream=None) -> torch.Tensor:
    if internal.dtype == torch.float64:
        prec = "f64"
    else:
        prec = "ds" if internal.numel() == 12 * lattice.Vh else "f32"
    out = torch.empty((lattice.Vh, 3), dtype=torch.complex128, device="cuda")
    check(lib().stg_field_unpack(lattice.handle, PREC[prec], _ptr(internal), _ptr(out), _stream(stream)),
          "stg_field_unpack")
    return out


# ------------------------------------------------------------------ operator (internal layout)

def dslash_eo_(gauge: Gauge, out: torch.Tensor, inp: torch.Tensor, stream=None) -> torch.Tensor:
    check(lib().stg_dslash_eo(gauge.handle, _ptr(out), _ptr(inp), _stream(stream)), "stg_dslash_eo")
    return out


def dslash_oe_(gauge: Gauge, out: torch.Tensor, inp: torch.Tensor, stream=None) -> torch.Tensor:
    check(lib().stg_dslash_oe(gauge.handle, _ptr(out), _ptr(inp), _stream(stream)), "stg_dslash_oe")
    return out


def dslash_multi_(gauge: Gauge, out_parity: int, out: torch.Tensor, inp: torch.Tensor, stream=None) -> torch.Tensor:
    """out[j] = D inp[j] for each row j (2-D internal tensors), link loads shared across rows."""
    n = inp.shape[0]
    stride = inp.stride(0) * inp.element_size()
    if out.stride(0) != inp.stride(0):
        raise ValueError("out and inp need the same row stride")
    check(lib().stg_dslash_multi(gauge.handle, int(out_parity), int(n), _ptr(out), _ptr(inp), stride, _stream(stream)),
          "stg_dslash_multi")
    return out


def normal_op_(gauge: Gauge, mass: float, shift: float, out: torch.Tensor, inp: torch.Tensor, tmp: torch.Tensor,
               pq: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    check(lib().stg_normal_op(gauge.handle, float(mass), float(shift), _ptr(out), _ptr(inp), _ptr(tmp),
                              _ptr(pq) if pq is not None else None, _stream(stream)), "stg_normal_op")
    return out


def normal_op_noalloc_(gauge: Gauge, mass: float, shift: float, out: torch.Tensor, inp: torch.Tensor,
                       pq: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """stg_normal_op_noalloc: like normal_op_ but without a caller temporary; the library keeps
    its scratch in a fixed 32 MiB device array and allocates nothing (see include/stg.h)."""
    check(lib().stg_normal_op_noalloc(gauge.handle, float(mass), float(shift), _ptr(out), _ptr(inp),
                                      _ptr(pq) if pq is not None else None, _stream(stream)), "stg_normal_op_noalloc")
    return out


# ------------------------------------------------------------------ operator (canonical layout)

def _to_host(t: torch.Tensor) -> torch.Tensor:
    """Device -> pinned host copy (torch caches pinned buffers), synchronised on the current stream."""
    out = torch.empty(t.shape, dtype=t.dtype, pin_memory=True)
    out.copy_(t, non_blocking=True)
    torch.cuda.current_stream().synchronize()
    return out


def _canon_apply(gauge: Gauge, canon: torch.Tensor, fn) -> torch.Tensor:
    host = not canon.is_cuda
    lat = gauge.lattice
    x = pack(lat, canon, gauge.vec_prec)
    y = fn(x)
    out = unpack(lat, y)
    return _to_host(out) if host else out


def dslash_eo(gauge: Gauge, psi_odd: torch.Tensor) -> torch.Tensor:
    """D_eo psi_odd on canonical complex128 [Vh, 3] fields (host or device)."""
    return _canon_apply(gauge, psi_odd, lambda x: dslash_eo_(gauge, torch.empty_like(x), x))


def dslash_host(gauge: Gauge, out_parity: int, fields: torch.Tensor, out: torch.Tensor | None = None,
                stream=None) -> torch.Tensor:
    """D_eo (out_parity 0) or D_oe (1) of a batch of canonical host fields [n, Vh, 3], complex128
    or complex64 (pinned for overlap), streamed through the device by stg_dslash_host; returns
    host fields of the same dtype."""
    if fields.is_cuda or fields.dtype not in (torch.complex128, torch.complex64):
        raise TypeError("dslash_host: fields must be complex128 or complex64 host tensors")
    src = fields.contiguous().reshape(-1, gauge.lattice.Vh, 3)
    n = src.shape[0]
    if out is None:
        out = torch.empty(src.shape, dtype=src.dtype, pin_memory=src.is_pinned())
    if out.dtype != src.dtype:
        raise TypeError("dslash_host: out must have the dtype of fields")
    hp = PREC["f64"] if src.dtype == torch.complex128 else PREC["f32"]
    pi = (ctypes.c_void_p * n)(*[src[k].data_ptr() for k in range(n)])
    po = (ctypes.c_void_p * n)(*[out[k].data_ptr() for k in range(n)])
    check(lib().stg_dslash_host(gauge.handle, int(out_parity), hp, n, ctypes.cast(pi, ctypes.POINTER(ctypes.c_void_p)),
                                ctypes.cast(po, ctypes.POINTER(ctypes.c_void_p)), _stream(stream)), "stg_dslash_host")
    return out


def dslash(gauge: Gauge, out_parity: int, psi: torch.Tensor) -> torch.Tensor:
    """D_eo psi (out_parity 0: odd input, even output) or D_oe psi (out_parity 1: even input, odd
    output) on canonical complex128 [Vh, 3] fields (host or device)."""
    if out_parity not in (0, 1):
        raise ValueError("dslash: out_parity must be 0 (D_eo) or 1 (D_oe)")
    return dslash_eo(gauge, psi) if out_parity == 0 else dslash_oe(gauge, psi)


def dslash_oe(gauge: Gauge, psi_even: torch.Tensor) -> torch.Tensor:
    """D_oe psi_even on canonical complex128 [Vh, 3] fields (host or device)."""
    return _canon_apply(gauge, psi_even, lambda x: dslash_oe_(gauge, torch.empty_like(x), x))


def normal_op(gauge: Gauge, mass: float, shift: float, psi_even: torch.Tensor) -> torch.Tensor:
    """(m^2 + shift) psi - D_eo D_oe psi on canonical complex128 [Vh, 3] fields."""
    return _canon_apply(gauge, psi_even,
                        lambda x: normal_op_(gauge, mass, shift, torch.empty_like(x), x, torch.empty_like(x)))


# ------------------------------------------------------------------ multi-shift CG

def _params(shifts, mass, tol, max_iter, inner_tol, reliable_delta, log_rows, history=0):
    sh = (ctypes.c_double * len(shifts))(*[float(s) for s in shifts])
    log = (ctypes.c_double * max(1, log_rows * (2 + len(shifts))))()
    p = MscgParams(len(shifts), ctypes.cast(sh, ctypes.POINTER(ctypes.c_double)), float(mass), float(tol),
                   int(max_iter), float(inner_tol), float(reliable_delta), int(log_rows),
                   ctypes.cast(log, ctypes.POINTER(ctypes.c_double)) if log_rows > 0 else None, int(history))
    return p, sh, log


def _stats(nshift):
    tr = (ctypes.c_double * nshift)()
    si = (ctypes.c_int32 * nshift)()
    ir = (ctypes.c_double * nshift)()
    rs = (ctypes.c_int32 * nshift)()
    ru = (ctypes.c_int32 * nshift)()
    i32p = ctypes.POINTER(ctypes.c_int32)
    st = MscgStats(0, 0, 0, ctypes.cast(tr, ctypes.POINTER(ctypes.c_double)), ctypes.cast(si, i32p),
                   ctypes.cast(ir, ctypes.POINTER(ctypes.c_double)), 0, ctypes.cast(rs, i32p), ctypes.cast(ru, i32p))
    return st, tr, (si, ir, rs, ru)


def _stats_dict(st, tr, extra):
    si, ir, rs, ru = extra
    return dict(iters=st.iters, reliable_updates=st.reliable_updates, refine_iters=st.refine_iters,
                true_resid=list(tr), shift_iters=list(si), inner_resid=list(ir), fp64_fallback=st.fp64_fallback,
                refine_shift_iters=list(rs), shift_reliable_updates=list(ru))


def mscg(g_f64: Gauge, b: torch.Tensor, shifts, mass: float, tol: float = 1e-10, g_inner: Gauge | None = None,
         max_iter: int = 20000, inner_tol: float = 0.0, reliable_delta: float = 0.0, log_rows: int = 0,
         allow_noconv: bool = False, out: torch.Tensor | None = None, history: int = 0, stream=None):
    """Multi-shift CG: x_i = (m^2 + sigma_i - D_eo D_oe)^-1 b.  b canonical complex128 [Vh, 3].
    history: residuals per window of the deferred multi-shift update of mixed solves (0 automatic,
    1 per-iteration updates).  Returns (x [nshift, Vh, 3] complex128, stats dict)."""
    host = not b.is_cuda
    bd = _dev(b).reshape(g_f64.lattice.Vh, 3)
    ns = len(shifts)
    x = out if out is not None else torch.empty((ns, g_f64.lattice.Vh, 3), dtype=torch.complex128, device="cuda")
    xp = (ctypes.c_void_p * ns)(*[x[i].data_ptr() for i in range(ns)])
    p, _sh, log = _params(shifts, mass, tol, max_iter, inner_tol, reliable_delta, log_rows, history)
    st, tr, si = _stats(ns)
    rc = lib().stg_mscg_solve(g_f64.handle, g_inner.handle if g_inner is not None else None, ctypes.byref(p), _ptr(bd),
                              ctypes.cast(xp, ctypes.POINTER(ctypes.c_void_p)), ctypes.byref(st), _stream(stream))
    check(rc, "stg_mscg_solve", allow=(STG_ERR_NOCONV,) if allow_noconv else ())
    stats = _stats_dict(st, tr, si)
    stats["status"] = rc
    if log_rows > 0:
        import numpy as np
        stats["scalar_log"] = np.array(log[:]).reshape(log_rows, 2 + ns)[:min(log_rows, st.iters)]
    return (_to_host(x) if host else x), stats


def rational_apply(g_f64: Gauge, b: torch.Tensor, alpha0: float, residues, poles, mass: float, tol: float = 1e-10,
                   g_inner: Gauge | None = None, max_iter: int = 20000, stream=None):
    """alpha0 b + sum_i residues[i] (m^2 + poles[i] - D_eo D_oe)^-1 b on a canonical complex128 even
    field (stg_rational_apply).  Returns (out [Vh, 3] complex128 on cuda, stats dict)."""
    bd = _dev(b).reshape(g_f64.lattice.Vh, 3)
    ns = len(poles)
    out = torch.empty_like(bd)
    p, _sh, _log = _params(poles, mass, tol, max_iter, 0.0, 0.0, 0)
    res = (ctypes.c_double * ns)(*[float(r) for r in residues])
    st, tr, si = _stats(ns)
    check(lib().stg_rational_apply(g_f64.handle, g_inner.handle if g_inner is not None else None, ctypes.byref(p),
                                   float(alpha0), ctypes.cast(res, ctypes.POINTER(ctypes.c_double)), _ptr(bd), _ptr(out),
                                   ctypes.byref(st), _stream(stream)), "stg_rational_apply")
    return out, _stats_dict(st, tr, si)


def pseudofermion_action_value(lattice: Lattice, b: torch.Tensor, x: torch.Tensor, residues, alpha0: float = 0.0,
                         stream=None) -> float:
    """S = alpha0 |b|^2 + sum_i residues[i] Re(b^dag x_i) (stg_pseudofermion_action): b canonical
    complex128 [Vh, 3], x [nshift, Vh, 3] (e.g. the output of mscg).  Synchronises to read S."""
    bb = _dev(b).reshape(lattice.Vh, 3)
    res = [float(r) for r in residues]
    n = len(res)
    xs = _dev(x).reshape(n, lattice.Vh, 3) if n else None
    xp = (ctypes.c_void_p * max(n, 1))(*[xs[i].data_ptr() for i in range(n)])
    rp = (ctypes.c_double * max(n, 1))(*res)
    out = torch.empty(1, dtype=torch.float64, device="cuda")
    check(lib().stg_pseudofermion_action(lattice.handle, n, float(alpha0), rp, _ptr(bb), xp, _ptr(out),
                                         _stream(stream)), "stg_pseudofermion_action")
    return float(_to_host(out)[0])


def mscg_batched(instances, shifts, mass: float, tol: float = 1e-10, max_iter: int = 20000, inner_tol: float = 0.0,
                 reliable_delta: float = 0.0, history: int = 0, stream=None):
    """instances: list of (g_f64, g_inner or None, [b_r canonical [Vh,3] cuda tensors]).
    Returns list of (x [nrhs, nshift, Vh, 3], [stats per rhs])."""
    ns = len(shifts)
    keep = []
    arr = (Instance * len(instances))()
    outs = []
    for k, (gf, gi, bs) in enumerate(instances):
        bs = [_dev(b).reshape(gf.lattice.Vh, 3) for b in bs]
        x = torch.empty((len(bs), ns, gf.lattice.Vh, 3), dtype=torch.complex128, device="cuda")
        bp = (ctypes.c_void_p * len(bs))(*[t.data_ptr() for t in bs])
        xp = (ctypes.c_void_p * (len(bs) * ns))(*[x[r, i].data_ptr() for r in range(len(bs)) for i in range(ns)])
        sts = (MscgStats * len(bs))()
        bufs = []
        for r in range(len(bs)):
            st, tr, si = _stats(ns)
            sts[r] = st
            bufs.append((tr, si))
        arr[k] = Instance(gf.handle, gi.handle if gi is not None else None, len(bs),
                          ctypes.cast(bp, ctypes.POINTER(ctypes.c_void_p)),
                          ctypes.cast(xp, ctypes.POINTER(ctypes.c_void_p)),
                          ctypes.cast(sts, ctypes.POINTER(MscgStats)))
        keep += [bs, bp, xp, sts, bufs]
        outs.append((x, sts, bufs))
    p, _sh, _log = _params(shifts, mass, tol, max_iter, inner_tol, reliable_delta, 0, history)
    check(lib().stg_mscg_solve_batched(len(instances), arr, ctypes.byref(p), _stream(stream)), "stg_mscg_solve_batched")
    res = []
    for x, sts, bufs in outs:
        res.append((x, [_stats_dict(sts[r], bufs[r][0], bufs[r][1]) for r in range(len(bufs))]))
    return res


# ------------------------------------------------------------------ fermion force

def fermion_force(g_f64: Gauge, residues, x: torch.Tensor, kind: int = 0, prec: str = "f64",
                  stream=None) -> torch.Tensor:
    """Per-link force [4, V, 3, 3] from solutions x [nshift, Vh, 3]:
    kind 0 -> TA(U W) (Lie-algebra force), kind 1 -> W^dag (gradient wrt link entries).
    prec "f64": complex128 (double-single operator, FP64-class); "f32": complex64, FP32 operator
    and gather (single-precision MD forces)."""
    ns = len(residues)
    xd = _dev(x).reshape(ns, g_f64.lattice.Vh, 3)
    res = (ctypes.c_double * ns)(*[float(r) for r in residues])
    xp = (ctypes.c_void_p * ns)(*[xd[i].data_ptr() for i in range(ns)])
    dt = torch.complex128 if prec == "f64" else torch.complex64
    out = torch.empty((4, g_f64.lattice.V, 3, 3), dtype=dt, device="cuda")
    check(lib().stg_fermion_force_prec(g_f64.handle, PREC[prec], ns, res, ctypes.cast(xp, ctypes.POINTER(ctypes.c_void_p)),
                                       _ptr(out), int(kind), _stream(stream)), "stg_fermion_force_prec")
    return out


def _cprec(t: torch.Tensor) -> int:
    """Library precision of a complex link array: complex128 -> F64, complex64 -> F32."""
    if t.dtype == torch.complex128:
        return PREC["f64"]
    if t.dtype == torch.complex64:
        return PREC["f32"]
    raise TypeError(f"expected complex128 or complex64 links, got {t.dtype}")


def _links(t, lattice: Lattice) -> torch.Tensor:
    if not torch.is_tensor(t):
        t = torch.as_tensor(t)
    if not t.is_cuda:
        t = t.cuda()
    _cprec(t)
    return t.contiguous().reshape(4, lattice.V, 3, 3)


def stout_smear(lattice: Lattice, links: torch.Tensor, rho: float, nstep: int, stream=None) -> torch.Tensor:
    """Stout-smeared levels U^(1) .. U^(nstep), [nstep, 4, V, 3, 3], from U^(0) [4, V, 3, 3]
    (canonical layout): complex128 links run in FP64, complex64 links in FP32."""
    u = _links(links, lattice)
    out = torch.empty((int(nstep), 4, lattice.V, 3, 3), dtype=u.dtype, device="cuda")
    check(lib().stg_stout_smear(lattice.handle, _cprec(u), int(nstep), float(rho), _ptr(u), _ptr(out),
                                _stream(stream)), "stg_stout_smear")
    return out


def stout_force(lattice: Lattice, links: torch.Tensor, levels: torch.Tensor, rho: float, grad: torch.Tensor,
                kind: int = 1, stream=None) -> torch.Tensor:
    """Pulls dS/dU^(k) (torch convention, [4, V, 3, 3]) back through k = len(levels) stout steps:
    kind 1 -> dS/dRe U^(0) + i dS/dIm U^(0), kind 0 -> TA(U^(0) G^dag) (Lie-algebra force).
    All arrays complex128 (FP64) or all complex64 (FP32)."""
    u = _links(links, lattice)
    lv = levels.contiguous()
    nstep = int(lv.shape[0])
    gr = grad.contiguous().reshape(4, lattice.V, 3, 3)
    if lv.dtype != u.dtype or gr.dtype != u.dtype:
        raise TypeError("stout_force: links, levels and grad must share one dtype")
    out = torch.empty((4, lattice.V, 3, 3), dtype=u.dtype, device="cuda")
    check(lib().stg_stout_force(lattice.handle, _cprec(u), nstep, float(rho), _ptr(u), _ptr(lv), _ptr(gr), _ptr(out),
                                int(kind), _stream(stream)), "stg_stout_force")
    return out


def complex_convert(src: torch.Tensor, dtype, stream=None) -> torch.Tensor:
    """complex128 <-> complex64 copy of a device array by the library's conversion kernel."""
    s = src.contiguous()
    out = torch.empty(s.shape, dtype=dtype, device="cuda")
    check(lib().stg_complex_convert(s.numel(), _cprec(s), _ptr(s), _cprec(out), _ptr(out), _stream(stream)),
          "stg_complex_convert")
    return out


def gauge_action(lattice: Lattice, links: torch.Tensor, beta: float, stream=None) -> dict:
    """Tree-level Symanzik S_g of the links [4, V, 3, 3] complex128, with the plaquette sum (each
    plaquette once) and the rectangle sum (each 2x1 rectangle once).  Synchronises to read them."""
    u = _dev(links).reshape(4, lattice.V, 3, 3)
    out = torch.empty(3, dtype=torch.float64, device="cuda")
    check(lib().stg_gauge_action(lattice.handle, float(beta), _ptr(u), _ptr(out), _stream(stream)), "stg_gauge_action")
    s, p, r = _to_host(out).tolist()
    return {"action": s, "plaquette_sum": p, "rectangle_sum": r}


def gauge_force(lattice: Lattice, links: torch.Tensor, beta: float, kind: int = 0, stream=None) -> torch.Tensor:
    """Per-link gradient of S_g [4, V, 3, 3]: kind 1 -> dS/dRe U + i dS/dIm U, kind 0 -> TA(U G^dag)
    (Lie-algebra force); complex128 links run in FP64, complex64 links in FP32."""
    u = _links(links, lattice)
    out = torch.empty((4, lattice.V, 3, 3), dtype=u.dtype, device="cuda")
    check(lib().stg_gauge_force(lattice.handle, _cprec(u), float(beta), _ptr(u), _ptr(out), int(kind),
                                _stream(stream)), "stg_gauge_force")
    return out


def md_momenta(lattice: Lattice, xi: torch.Tensor, stream=None) -> torch.Tensor:
    """Momenta H [4, V, 3, 3] from standard normal numbers xi [4, V, 8] (float64)."""
    x = _dev(xi, torch.float64).reshape(4, lattice.V, 8)
    out = torch.empty((4, lattice.V, 3, 3), dtype=torch.complex128, device="cuda")
    check(lib().stg_md_momenta(lattice.handle, _ptr(x), _ptr(out), _stream(stream)), "stg_md_momenta")
    return out


def md_update_links_(lattice: Lattice, eps: float, mom: torch.Tensor, links: torch.Tensor, stream=None) -> torch.Tensor:
    """links <- exp(i eps H) links, in place (complex128 [4, V, 3, 3] on cuda)."""
    check(lib().stg_md_update_links(lattice.handle, float(eps), _ptr(mom), _ptr(links), _stream(stream)),
          "stg_md_update_links")
    return links


def md_update_momenta_(lattice: Lattice, eps: float, force: torch.Tensor, mom: torch.Tensor, stream=None) -> torch.Tensor:
    """mom <- mom - eps i F, in place (F: Lie-algebra force, kind 0 format, complex128 or complex64)."""
    f = force.contiguous()
    check(lib().stg_md_update_momenta(lattice.handle, _cprec(f), float(eps), _ptr(f), _ptr(mom), _stream(stream)),
          "stg_md_update_momenta")
    return mom


def md_kinetic(lattice: Lattice, mom: torch.Tensor, stream=None) -> float:
    """(1/2) sum tr H^2 (synchronises to read it)."""
    out = torch.empty(1, dtype=torch.float64, device="cuda")
    check(lib().stg_md_kinetic(lattice.handle, _ptr(mom), _ptr(out), _stream(stream)), "stg_md_kinetic")
    return float(_to_host(out)[0])
