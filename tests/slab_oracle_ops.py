"""CPU stand-in for the compute steps of the slab solver (test infrastructure only).

Same interface as paper_1801_01473_gb300.slab.LibraryOps, on CPU torch tensors in the library's
internal F64 layout (three arrays of Vh complex numbers, one per colour), with every step written
from the FP64 oracle: D on the stored slab lattice is the oracle's D there with the antiperiodic
sign moved onto the t-links at global time Lt - 1 (the oracle would put it on the stored lattice's
last slice), and only the local slices of an output are written, as the library does.  With it,
the host logic of the decomposition (layout, halo exchange, sums over slabs, the library's host
scalar recurrences) runs under gloo on CPU processes.
"""
from __future__ import annotations

import numpy as np
import torch

import oracle


def to_canon(t: torch.Tensor, vh: int) -> np.ndarray:
    a = t.reshape(3, vh, 2).numpy()
    return np.ascontiguousarray((a[..., 0] + 1j * a[..., 1]).T)


def from_canon(c: np.ndarray, out: torch.Tensor, rows=None) -> None:
    vh = c.shape[0]
    a = out.reshape(3, vh, 2)
    sel = slice(None) if rows is None else rows
    a[:, sel, 0] = torch.from_numpy(np.ascontiguousarray(c[sel].real.T))
    a[:, sel, 1] = torch.from_numpy(np.ascontiguousarray(c[sel].imag.T))


class OracleOps:
    prec = "f64"

    def __init__(self, slab, links_global, antiperiodic: bool = True):
        self.slab = slab
        lx, ly, lz, lt = slab.dims_global
        self.dims = (lx, ly, lz, slab.lt_loc + 4)
        u = slab.stored_links(np.asarray(links_global)).reshape(4, slab.lt_loc + 4, lx * ly * lz, 3, 3).copy()
        if antiperiodic:
            for k, tg in enumerate(slab.stored_slices()):
                if tg == lt - 1:
                    u[3, k] *= -1.0
        self.u = u.reshape(4, -1, 3, 3)
        self.vh = lx * ly * lz * (slab.lt_loc + 4) // 2
        hs = slab.half_slice
        self.local = slice(2 * hs, (slab.lt_loc + 2) * hs)

    def new_field(self) -> torch.Tensor:
        return torch.zeros(6 * self.vh, dtype=torch.float64)

    def _d(self, out_parity, inp):
        return oracle.dslash(self.dims, self.u, out_parity, to_canon(inp, self.vh), antiperiodic=False)

    def dslash(self, out_parity, out, inp):
        from_canon(self._d(out_parity, inp), out, self.local)

    def dslash_part(self, out_parity, part, out, inp):
        hs, lt = self.slab.half_slice, self.slab.lt_loc
        rows = {0: [self.local], 1: [slice(2 * hs, 3 * hs), slice((lt + 1) * hs, (lt + 2) * hs)],
                2: [slice(3 * hs, (lt + 1) * hs)]}[part]
        d = self._d(out_parity, inp)
        for r in rows:
            from_canon(d, out, r)

    def dslash_xpay(self, out_parity, coef, out, inp, p):
        pc = to_canon(p, self.vh)
        o = coef * pc - self._d(out_parity, inp)
        from_canon(o, out, self.local)
        return float(np.vdot(pc[self.local], o[self.local]).real)

    def axpy_norm(self, alpha, x, y):
        xc, yc = to_canon(x, self.vh), to_canon(y, self.vh)
        yc[self.local] += alpha * xc[self.local]
        from_canon(yc, y, self.local)
        return float(np.vdot(yc[self.local], yc[self.local]).real)

    def shift_update(self, st, xs, ps, r):
        rc = to_canon(r, self.vh)
        for i in range(st.nshift):
            if not st.upd_x[i] and not st.upd_p[i]:
                continue
            pc = to_canon(ps[i], self.vh)
            if st.upd_x[i]:
                xc = to_canon(xs[i], self.vh)
                xc[self.local] += st.cx[i] * pc[self.local]
                from_canon(xc, xs[i], self.local)
            if st.upd_p[i]:
                pc[self.local] = st.cr[i] * rc[self.local] + st.cp[i] * pc[self.local]
                from_canon(pc, ps[i], self.local)
