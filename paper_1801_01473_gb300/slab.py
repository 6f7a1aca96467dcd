"""Lattice split into slabs along t, one per process (Sec. 3.1: one-dimensional tiling; Sec. 4.1:
halo slices next to each slab, contiguous in memory; Sec. 4.2 and Alg. 1: D on the local sites
once the 1-site halos of its input are current; the scalar products summed over processes).

The library computes (stg_dslash on a slab lattice, stg_slab_dslash_xpay, stg_slab_axpy_norm,
stg_slab_shift_update, and the FP64 scalar recurrences stg_mscg_state_*); this module moves halo
slices and sums reductions through a transport, and sequences the multi-shift CG:

    DistTransport    torch.distributed point-to-point messages and all_reduce (NCCL between GPUs,
                     gloo between CPU processes), one process per slab;
    LoopbackGroup    the slabs of one process (threads), for emulating a decomposition on one GPU.

No device code waits on another process: every exchange is host-ordered between launches.
Layout: a slab of Lt_loc local slices is stored over Lt_loc + 4 slices (stg_lattice_create_slab):
stored slice 1 is the lower halo, Lt_loc + 2 the upper one, 2 and Lt_loc + 1 the borders.
"""
from __future__ import annotations

import ctypes
import threading
from typing import Sequence

import numpy as np
import torch

from .api import Gauge, Lattice, _ptr, _stream
from .lib import PREC, MscgState, check, lib


class Slab:
    """Global lattice dims (Lx, Ly, Lz, Lt) split into nranks slabs along t; this is slab `rank`."""

    def __init__(self, dims_global: Sequence[int], rank: int, nranks: int, antiperiodic: bool = True):
        lx, ly, lz, lt = (int(d) for d in dims_global)
        if nranks < 1 or lt % nranks or (lt // nranks) % 2:
            raise ValueError("Lt must split into nranks slabs of an even number of slices")
        self.dims_global = (lx, ly, lz, lt)
        self.rank, self.nranks = int(rank), int(nranks)
        self.lt_loc = lt // nranks
        self.t0 = self.rank * self.lt_loc
        self.lattice = Lattice.slab((lx, ly, lz, self.lt_loc), self.t0, lt, antiperiodic)
        self.half_slice = lx * ly * lz // 2  # sites of one parity in one time slice
        self._layout = {}

    # ------------------------------------------------------------------ layout
    def chunks(self, prec: str):
        """[(byte offset, bytes per site)] of the internal field arrays, and sites per half slice."""
        if prec not in self._layout:
            n = ctypes.c_int32()
            off = (ctypes.c_int64 * 3)()
            elem = (ctypes.c_int32 * 3)()
            ss = ctypes.c_int64()
            check(lib().stg_slab_layout(self.lattice.handle, PREC[prec], ctypes.byref(n), off, elem, ctypes.byref(ss)),
                  "stg_slab_layout")
            self._layout[prec] = ([(int(off[k]), int(elem[k])) for k in range(n.value)], int(ss.value))
        return self._layout[prec]

    def slice_views(self, field: torch.Tensor, prec: str, stored_slice: int):
        """Byte views (one per array) of one stored time slice of an internal field."""
        chunks, ss = self.chunks(prec)
        raw = field.reshape(-1).view(torch.uint8)
        return [raw[o + e * ss * stored_slice:o + e * ss * (stored_slice + 1)] for o, e in chunks]

    # ------------------------------------------------------------------ stored canonical arrays
    def stored_slices(self):
        """Global time of every stored slice (t0 - 2 .. t0 + Lt_loc + 1, wrapped)."""
        lt = self.dims_global[3]
        return [(self.t0 - 2 + k) % lt for k in range(self.lt_loc + 4)]

    def stored_links(self, links_global):
        """Canonical stored links [4][V_stored][3][3] of this slab from the global ones
        [4][V][3][3] (numpy or torch): halo and padding slices hold the neighbours' links."""
        lx, ly, lz, lt = self.dims_global
        vs = lx * ly * lz
        u = links_global.reshape(4, lt, vs, 3, 3)
        idx = self.stored_slices()
        if isinstance(u, torch.Tensor):
            return u[:, torch.as_tensor(idx, device=u.device)].reshape(4, -1, 3, 3).contiguous()
        return np.ascontiguousarray(u[:, idx].reshape(4, -1, 3, 3))

    def stored_field(self, half_global):
        """Canonical stored half field [Vh_stored][3] from a global one [Vh][3] (one parity)."""
        lt = self.dims_global[3]
        f = half_global.reshape(lt, self.half_slice, 3)
        idx = self.stored_slices()
        if isinstance(f, torch.Tensor):
            return f[torch.as_tensor(idx, device=f.device)].reshape(-1, 3).contiguous()
        return np.ascontiguousarray(f[idx].reshape(-1, 3))

    def local_part(self, half_stored):
        """The local slices [Lt_loc * half_slice][3] of a canonical stored half field."""
        f = half_stored.reshape(self.lt_loc + 4, self.half_slice, 3)
        return f[2:self.lt_loc + 2].reshape(-1, 3)


# ---------------------------------------------------------------------- transports

class DistTransport:
    """Halo messages and sums over torch.distributed (one process per slab, ranks in t order).
    Messages going up carry tag 1, going down tag 2; sends are posted up then down and receives
    from below then from above, so that two slabs (whose neighbours coincide) still match
    under a backend that orders messages per peer instead of by tag."""

    def __init__(self, group=None):
        import torch.distributed as dist
        self.dist = dist
        self.group = group
        self.rank = dist.get_rank(group)
        self.size = dist.get_world_size(group)

    def exchange(self, to_lower: torch.Tensor, to_upper: torch.Tensor):
        if self.size == 1:
            return to_upper.clone(), to_lower.clone()
        d = self.dist
        lo, hi = (self.rank - 1) % self.size, (self.rank + 1) % self.size
        from_lower, from_upper = torch.empty_like(to_upper), torch.empty_like(to_lower)
        ops = [d.P2POp(d.isend, to_upper, hi, self.group, 1), d.P2POp(d.isend, to_lower, lo, self.group, 2),
               d.P2POp(d.irecv, from_lower, lo, self.group, 1), d.P2POp(d.irecv, from_upper, hi, self.group, 2)]
        for r in d.batch_isend_irecv(ops):
            r.wait()
        return from_lower, from_upper

    def allreduce(self, values: torch.Tensor) -> torch.Tensor:
        out = values.clone()
        if self.size > 1:
            self.dist.all_reduce(out, op=self.dist.ReduceOp.SUM, group=self.group)
        return out


class LoopbackGroup:
    """n slabs served by threads of one process: transport(rank) is slab rank's endpoint.  Each
    exchange and sum is a rendezvous of all n threads (host barriers, after each thread has
    finished its device work); sums run in rank order."""

    def __init__(self, n: int, timeout: float = 120.0):
        self.n = n
        self.barrier = threading.Barrier(n, timeout=timeout)  # a failed slab breaks it for the others
        self.slots = [None] * n

    def transport(self, rank: int) -> "_LoopbackTransport":
        return _LoopbackTransport(self, rank)


class _LoopbackTransport:
    def __init__(self, group: LoopbackGroup, rank: int):
        self.g, self.rank, self.size = group, rank, group.n

    def _sync(self, t: torch.Tensor):
        if t.is_cuda:
            torch.cuda.current_stream(t.device).synchronize()

    def exchange(self, to_lower: torch.Tensor, to_upper: torch.Tensor):
        g = self.g
        self._sync(to_lower)
        g.slots[self.rank] = (to_lower.clone(), to_upper.clone())
        self._sync(to_lower)
        g.barrier.wait()
        below, above = g.slots[(self.rank - 1) % g.n], g.slots[(self.rank + 1) % g.n]
        out = (below[1].clone(), above[0].clone())
        self._sync(to_lower)
        g.barrier.wait()
        return out

    def allreduce(self, values: torch.Tensor) -> torch.Tensor:
        g = self.g
        self._sync(values)
        g.slots[self.rank] = values.clone()
        g.barrier.wait()
        total = g.slots[0].clone()
        for r in range(1, g.n):
            total += g.slots[r]
        g.barrier.wait()
        return total


def exchange_halos(slab: Slab, field: torch.Tensor, prec: str, transport) -> None:
    """Fills the two halo slices of a slab field (internal layout) from the neighbours' borders."""
    lt = slab.lt_loc
    lo_b, hi_b = slab.slice_views(field, prec, 2), slab.slice_views(field, prec, lt + 1)
    send_lo, send_hi = torch.cat(lo_b), torch.cat(hi_b)
    from_lower, from_upper = transport.exchange(send_lo, send_hi)
    for views, buf in ((slab.slice_views(field, prec, 1), from_lower), (slab.slice_views(field, prec, lt + 2), from_upper)):
        k = 0
        for v in views:
            v.copy_(buf[k:k + v.numel()])
            k += v.numel()


# ---------------------------------------------------------------------- operators and solver

class LibraryOps:
    """The compute steps of the slab solver on one GPU, each a libstg call."""

    def __init__(self, slab: Slab, gauge: Gauge):
        self.slab, self.g = slab, gauge
        self.prec = gauge.vec_prec
        if self.prec not in ("f64", "f32"):
            raise ValueError("the slab solver runs on F64 or F32 gauges")
        self._d = torch.empty(1, dtype=torch.float64, device="cuda")

    def new_field(self) -> torch.Tensor:
        return self.g.new_field().zero_()

    def dslash(self, out_parity: int, out: torch.Tensor, inp: torch.Tensor) -> None:
        check(lib().stg_dslash(self.g.handle, int(out_parity), _ptr(out), _ptr(inp), _stream()), "stg_dslash")

    def dslash_part(self, out_parity: int, part: int, out: torch.Tensor, inp: torch.Tensor) -> None:
        check(lib().stg_slab_dslash_part(self.g.handle, int(out_parity), int(part), _ptr(out), _ptr(inp), _stream()),
              "stg_slab_dslash_part")

    def dslash_xpay(self, out_parity: int, coef: float, out, inp, p) -> float:
        check(lib().stg_slab_dslash_xpay(self.g.handle, int(out_parity), float(coef), _ptr(out), _ptr(inp), _ptr(p),
                                         _ptr(self._d), _stream()), "stg_slab_dslash_xpay")
        return float(self._d.item())

    def axpy_norm(self, alpha: float, x, y) -> float:
        check(lib().stg_slab_axpy_norm(self.slab.lattice.handle, PREC[self.prec], float(alpha), _ptr(x), _ptr(y),
                                       _ptr(self._d), _stream()), "stg_slab_axpy_norm")
        return float(self._d.item())

    def shift_update(self, st: MscgState, xs, ps, r) -> None:
        n = st.nshift
        xp = (ctypes.c_void_p * n)(*[x.data_ptr() for x in xs])
        pp = (ctypes.c_void_p * n)(*[p.data_ptr() for p in ps])
        check(lib().stg_slab_shift_update(self.slab.lattice.handle, PREC[self.prec], n, st.cx, st.cr, st.cp,
                                          st.upd_x, st.upd_p, xp, pp, _ptr(r), _stream()), "stg_slab_shift_update")


def dslash(slab: Slab, ops, out_parity: int, out: torch.Tensor, inp: torch.Tensor, transport) -> torch.Tensor:
    """D_eo (out_parity 0) or D_oe (1) on the local slices, after the halo exchange of inp (Alg. 1
    without the border/bulk overlap: the exchange is host-ordered before the launch)."""
    exchange_halos(slab, inp, ops.prec, transport)
    ops.dslash(out_parity, out, inp)
    return out


def dslash_overlapped(slab: Slab, ops, out_parity: int, out: torch.Tensor, inp: torch.Tensor, transport) -> torch.Tensor:
    """D on the local slices with the schedule of Alg. 1, for an input whose halos are current:
    the two border slices first, then the bulk on a second stream while the border outputs go to
    the neighbours, so that `out` leaves with its own halos current (the next operator's input)."""
    if not out.is_cuda:
        ops.dslash_part(out_parity, 1, out, inp)
        ops.dslash_part(out_parity, 2, out, inp)
        exchange_halos(slab, out, ops.prec, transport)
        return out
    main = torch.cuda.current_stream()
    side = getattr(ops, "_side", None)
    if side is None:
        side = ops._side = torch.cuda.Stream()
    ops.dslash_part(out_parity, 1, out, inp)  # borders on the main stream
    side.wait_stream(main)
    with torch.cuda.stream(side):
        ops.dslash_part(out_parity, 2, out, inp)  # bulk, concurrently with the exchange below
    exchange_halos(slab, out, ops.prec, transport)
    main.wait_stream(side)
    return out


def mscg(slab: Slab, ops, b: torch.Tensor, shifts: Sequence[float], mass: float, transport, tol: float = 1e-10,
         max_iter: int = 10000, overlap: bool = True):
    """Multi-shift CG (Sec. 2, Eq. shift_eo) for (m^2 + sigma_i - D_eo D_oe) x_i = b across the slabs:
    b an internal even field of this slab (halos need not be set); returns the solutions (internal
    fields, local slices valid) and the statistics.  Per iteration: the halo exchange of p, D_oe
    (with overlap: borders, then the bulk while t's borders travel, Alg. 1), the halo exchange of t
    otherwise, q = (m^2 + sigma_0) p - D_eo t with Re<p, q>, one sum over slabs, the alpha step,
    r -= alpha q with |r|^2, one sum, the beta step, the shift update."""
    L = lib()
    ns = len(shifts)
    sig = (ctypes.c_double * ns)(*[float(s) for s in shifts])
    st = MscgState()
    r = b.clone()

    def total(v: float) -> float:  # sum over the slabs
        return float(transport.allreduce(torch.tensor([v], dtype=torch.float64, device=b.device))[0])

    bb = total(ops.axpy_norm(0.0, b, r))
    check(L.stg_mscg_state_init(ctypes.byref(st), ns, sig, float(tol), bb, int(max_iter)), "stg_mscg_state_init")
    xs = [ops.new_field() for _ in range(ns)]
    ps = [b.clone() for _ in range(ns)]
    t, q = ops.new_field(), ops.new_field()
    coef = mass * mass + float(min(shifts))
    p0 = ps[st.i0]
    while st.running:
        exchange_halos(slab, p0, ops.prec, transport)
        if overlap:
            dslash_overlapped(slab, ops, 1, t, p0, transport)
        else:
            ops.dslash(1, t, p0)
            exchange_halos(slab, t, ops.prec, transport)
        pq = total(ops.dslash_xpay(0, coef, q, t, p0))
        check(L.stg_mscg_state_alpha(ctypes.byref(st), pq), "stg_mscg_state_alpha")
        rr = total(ops.axpy_norm(-st.alpha, q, r))
        check(L.stg_mscg_state_beta(ctypes.byref(st), rr), "stg_mscg_state_beta")
        ops.shift_update(st, xs, ps, r)
    stats = {"iters": st.iters, "shift_iters": list(st.shift_iters)[:ns], "rr": st.rr, "bnorm2": bb}
    return xs, stats
