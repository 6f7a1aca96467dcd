"""The slab decomposition along t (Sec. 3.1, 4.1, 4.2, Alg. 1) on CPU: the library's host calls
(slab lattice, halo layout, the multi-shift scalar recurrences) and the binding's halo exchange and
solver sequencing, with the FP64 oracle standing in for the GPU compute steps
(tests/slab_oracle_ops.py).  Two slabs run as threads of one process (loopback transport) and as
two gloo processes (torch.distributed), and must reproduce the single-domain oracle's D_eo, D_oe
and multi-shift solutions element by element."""
import ctypes
import os
import sys

import numpy as np
import pytest

import oracle
import synthetic as S

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

DIMS = (4, 4, 4, 8)  # the 4^4 x 8 lattice split into two slabs of 4 slices
MASS = 0.1
SHIFTS = [1e-3, 0.02, 0.3, 1.5]
TOL = 1e-10


def _slab(rank, n, dims=DIMS):
    from paper_1801_01473_gb300.slab import Slab
    return Slab(dims, rank, n)


def _inputs(dims=DIMS):
    u = S.gauge_links(dims, "haar", 1301)
    b = S.gaussian_field(dims, 1302)
    return u, b


def _stored_internal(slab, ops, half_global):
    from tests.slab_oracle_ops import from_canon
    t = ops.new_field()
    from_canon(slab.stored_field(half_global), t)
    # halo and padding slices cleared: the exchange must fill what D reads
    hs = slab.half_slice
    a = t.reshape(3, -1, 2)
    a[:, :2 * hs] = 0.0
    a[:, (slab.lt_loc + 2) * hs:] = 0.0
    return t


def test_slab_layout_and_arguments():
    from paper_1801_01473_gb300.lib import STG_ERR_ARG, STG_ERR_SHAPE, lib
    L = lib()
    s = _slab(1, 2)
    assert s.t0 == 4 and s.lt_loc == 4
    assert s.lattice.dims == (4, 4, 4, 8) and s.lattice.Vh == 4 * 4 * 4 * 8 // 2
    ch, ss = s.chunks("f64")
    assert ss == 32 and ch == [(0, 16), (16 * s.lattice.Vh, 16), (32 * s.lattice.Vh, 16)]
    ch, ss = s.chunks("f32")
    assert ch == [(0, 16), (16 * s.lattice.Vh, 8)]
    assert s.stored_slices() == [2, 3, 4, 5, 6, 7, 0, 1]
    # one stored slice of a field spans slice_sites sites in every array
    f = torch.zeros(6 * s.lattice.Vh, dtype=torch.float64)
    assert sum(v.numel() for v in s.slice_views(f, "f64", 3)) == 48 * ss
    n, off, el, sl = ctypes.c_int32(), (ctypes.c_int64 * 3)(), (ctypes.c_int32 * 3)(), ctypes.c_int64()
    assert L.stg_slab_layout(s.lattice.handle, 2, ctypes.byref(n), off, el, ctypes.byref(sl)) == STG_ERR_ARG
    h = ctypes.c_void_p()
    for dims, t0, lt in [((4, 4, 4, 4), 1, 8), ((4, 4, 4, 4), 6, 8), ((4, 4, 4, 3), 0, 8), ((4, 4, 4, 4), 0, 7)]:
        assert L.stg_lattice_create_slab((ctypes.c_int32 * 4)(*dims), t0, lt, 1, ctypes.byref(h)) == STG_ERR_SHAPE
    with pytest.raises(ValueError):
        _slab(0, 3)


def test_scalar_state_rejects_misuse():
    from paper_1801_01473_gb300.lib import STG_ERR_ARG, MscgState, lib
    L = lib()
    st = MscgState()
    sig = (ctypes.c_double * 2)(0.1, 0.01)
    assert L.stg_mscg_state_init(ctypes.byref(st), 2, sig, 1e-8, 4.0, 100) == 0
    assert st.i0 == 1 and abs(st.s[0] - 0.09) < 1e-15 and st.running == 1
    assert L.stg_mscg_state_beta(ctypes.byref(st), 1.0) == STG_ERR_ARG  # beta before alpha
    assert L.stg_mscg_state_alpha(ctypes.byref(st), 2.0) == 0 and st.alpha == 2.0
    assert L.stg_mscg_state_alpha(ctypes.byref(st), 2.0) == STG_ERR_ARG
    bad = (ctypes.c_double * 2)(0.1, -1.0)
    assert L.stg_mscg_state_init(ctypes.byref(st), 2, bad, 1e-8, 4.0, 100) == STG_ERR_ARG
    assert L.stg_mscg_state_init(ctypes.byref(st), 33, sig, 1e-8, 4.0, 100) == STG_ERR_ARG


def _run_slab(rank, n, transport, u, b, psi_odd):
    """D_eo of an odd field, D_oe of b, and the msCG of b on slab `rank`: local parts."""
    from paper_1801_01473_gb300 import slab as sl
    from tests.slab_oracle_ops import OracleOps, to_canon
    s = _slab(rank, n)
    ops = OracleOps(s, u)
    vh = ops.vh
    out = {}
    for name, par, src in (("eo", 0, psi_odd), ("oe", 1, b)):
        inp = _stored_internal(s, ops, src)
        res = ops.new_field()
        sl.dslash(s, ops, par, res, inp, transport)
        out[name] = s.local_part(to_canon(res, vh))
    xs, st = sl.mscg(s, ops, _stored_internal(s, ops, b), SHIFTS, MASS, transport, tol=TOL)
    out["x"] = [s.local_part(to_canon(x, vh)) for x in xs]
    out["iters"] = st["iters"]
    out["shift_iters"] = st["shift_iters"]
    return out


def _check(results, u, b, psi_odd):
    lt = DIMS[3]
    hs = DIMS[0] * DIMS[1] * DIMS[2] // 2
    n = len(results)
    ref_eo = oracle.dslash_eo(DIMS, u, psi_odd)
    ref_oe = oracle.dslash_oe(DIMS, u, b)
    ref = oracle.mscg(DIMS, u, MASS, SHIFTS, b, tol=TOL)
    for rank, out in enumerate(results):
        rows = slice(rank * (lt // n) * hs, (rank + 1) * (lt // n) * hs)
        assert np.abs(out["eo"] - ref_eo[rows]).max() <= 1e-14 * np.abs(ref_eo).max()
        assert np.abs(out["oe"] - ref_oe[rows]).max() <= 1e-14 * np.abs(ref_oe).max()
        # the same recurrences with the reductions split over slabs: a shift may stop one
        # iteration apart from the oracle's near its threshold
        assert abs(out["iters"] - ref["iters"]) <= 1
        assert all(abs(a - r) <= 1 for a, r in zip(out["shift_iters"], ref["shift_iters"]))
    # the assembled solutions: FP64 true residuals at the requested tolerance (no refinement runs
    # here) and within kappa_i tol of the oracle's
    for i, sgm in enumerate(SHIFTS):
        x = np.concatenate([out["x"][i] for out in results])
        res = oracle.true_residual(DIMS, u, MASS, sgm, b, x)
        assert res <= 2 * TOL, (i, res)
        kappa = (MASS ** 2 + sgm + 16.0) / (MASS ** 2 + sgm)
        err = np.linalg.norm(x - ref["x"][i]) / np.linalg.norm(ref["x"][i])
        assert err <= 2 * kappa * TOL, (i, err)


def test_two_slabs_loopback_match_single_domain_oracle():
    import threading

    from paper_1801_01473_gb300.slab import LoopbackGroup
    u, b = _inputs()
    psi = S.gaussian_field(DIMS, 1303)
    grp = LoopbackGroup(2, timeout=300)
    results, errors = [None, None], []

    def run(rank):
        try:
            results[rank] = _run_slab(rank, 2, grp.transport(rank), u, b, psi)
        except Exception as e:  # surfaced below
            errors.append(e)
            grp.barrier.abort()

    th = [threading.Thread(target=run, args=(r,)) for r in range(2)]
    for t in th:
        t.start()
    for t in th:
        t.join(600)
    assert not errors, errors
    _check(results, u, b, psi)


def _gloo_worker(rank, ws, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), OMP_NUM_THREADS="1")
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        import synthetic as S2
        from paper_1801_01473_gb300.slab import DistTransport
        u = S2.gauge_links(DIMS, "haar", 1301)
        b = S2.gaussian_field(DIMS, 1302)
        psi = S2.gaussian_field(DIMS, 1303)
        q.put((rank, _run_slab(rank, ws, DistTransport(), u, b, psi)))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_slabs_gloo_world2_match_single_domain_oracle():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 31500 + os.getpid() % 1000
    procs = [ctx.Process(target=_gloo_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=600) for _ in range(2))
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    u, b = _inputs()
    _check([got[0], got[1]], u, b, S.gaussian_field(DIMS, 1303))
