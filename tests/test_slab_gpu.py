"""The slab decomposition along t on the GPU: two slabs of a lattice served by two threads of one
process (loopback transport: each halo exchange and each sum is a host rendezvous after both
threads' device work has finished, so no kernel ever waits on another), every compute step a
libstg kernel on its slab lattice.  D_eo / D_oe must match the single-domain oracle on every local
site (FP64 1e-12, FP32 2e-6 relative), and the multi-shift CG across the slabs must reach the
requested FP64 true residual on the assembled solutions."""
import threading

import numpy as np
import pytest

import oracle
import synthetic as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {("f64", 18): 1e-12, ("f64", 12): 1e-12, ("f32", 12): 2e-6, ("f32", 18): 2e-6}


def _stored(p, slab, canon_global, prec):
    """Internal stored field of one slab, its halo and padding slices zeroed (the exchange must fill
    what D reads)."""
    x = p.pack(slab.lattice, torch.from_numpy(slab.stored_field(canon_global)).cuda(), prec)
    for s in (0, 1, slab.lt_loc + 2, slab.lt_loc + 3):
        for v in slab.slice_views(x, prec, s):
            v.zero_()
    return x


def _run_threads(n, fn):
    from paper_1801_01473_gb300.slab import LoopbackGroup
    grp = LoopbackGroup(n, timeout=300)
    out, errors = [None] * n, []

    def run(rank):
        try:
            out[rank] = fn(rank, grp.transport(rank))
        except Exception as e:  # surfaced below
            errors.append(e)
            grp.barrier.abort()

    th = [threading.Thread(target=run, args=(r,)) for r in range(n)]
    for t in th:
        t.start()
    for t in th:
        t.join(600)
    assert not errors, errors
    return out


@pytest.mark.parametrize("variant", list(TOL))
@pytest.mark.parametrize("dims,nslab", [((4, 4, 4, 8), 2), ((6, 4, 2, 12), 3), ((8, 8, 8, 16), 2)])
def test_slab_dslash_matches_oracle(variant, dims, nslab):
    import paper_1801_01473_gb300 as p
    from paper_1801_01473_gb300 import slab as sl
    prec, recon = variant
    u = S.gauge_links(dims, "haar", 1401)
    psi = {0: S.gaussian_field(dims, 1402), 1: S.gaussian_field(dims, 1403)}  # input parity 1 - out_parity
    ut = torch.from_numpy(u).cuda()

    def fn(rank, tr):
        slab = sl.Slab(dims, rank, nslab)
        g = p.Gauge(slab.lattice, slab.stored_links(ut), prec, recon)
        ops = sl.LibraryOps(slab, g)
        res = {}
        for out_par in (0, 1):
            x = _stored(p, slab, psi[out_par], g.vec_prec)
            y = g.new_field().zero_()
            sl.dslash(slab, ops, out_par, y, x, tr)
            res[out_par] = slab.local_part(p.unpack(slab.lattice, y).cpu().numpy())
        return res

    out = _run_threads(nslab, fn)
    for out_par in (0, 1):
        ref = oracle.dslash(dims, u, out_par, psi[out_par])
        got = np.concatenate([o[out_par] for o in out])
        assert np.abs(got - ref).max() <= TOL[variant] * np.abs(ref).max(), (variant, out_par)


@pytest.mark.parametrize("lt_loc", [2, 4, 8])
def test_border_and_bulk_parts_cover_the_slab(lt_loc):
    """Alg. 1's split: the border launch and the bulk launch together write bitwise what one launch
    over all local slices writes, and the overlapped schedule leaves the output's halos current."""
    import paper_1801_01473_gb300 as p
    from paper_1801_01473_gb300 import slab as sl
    dims = (6, 4, 4, 2 * lt_loc)
    u = S.gauge_links(dims, "haar", 1407)
    psi = S.gaussian_field(dims, 1408)
    ut = torch.from_numpy(u).cuda()

    def fn(rank, tr):
        slab = sl.Slab(dims, rank, 2)
        g = p.Gauge(slab.lattice, slab.stored_links(ut), "f64", 12)
        ops = sl.LibraryOps(slab, g)
        x = _stored(p, slab, psi, "f64")
        sl.exchange_halos(slab, x, "f64", tr)
        whole, split = g.new_field().zero_(), g.new_field().zero_()
        ops.dslash(1, whole, x)
        sl.dslash_overlapped(slab, ops, 1, split, x, tr)
        torch.cuda.synchronize()
        loc = slice(2 * slab.half_slice, (slab.lt_loc + 2) * slab.half_slice)
        a, b = whole.reshape(3, -1, 2)[:, loc], split.reshape(3, -1, 2)[:, loc]
        assert torch.equal(a, b)
        return p.unpack(slab.lattice, split).cpu().numpy()

    out = _run_threads(2, fn)
    # the halos of each slab's output now hold the neighbour's border outputs
    ref = oracle.dslash_oe(dims, u, psi)
    hs = dims[0] * dims[1] * dims[2] // 2
    for rank in range(2):
        st = out[rank].reshape(lt_loc + 4, hs, 3)
        gl = ref.reshape(dims[3], hs, 3)
        t_lo, t_hi = (rank * lt_loc - 1) % dims[3], ((rank + 1) * lt_loc) % dims[3]
        assert np.abs(st[1] - gl[t_lo]).max() <= 1e-12 * np.abs(ref).max()
        assert np.abs(st[lt_loc + 2] - gl[t_hi]).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("overlap", [True, False])
def test_slab_mscg_matches_oracle(overlap):
    import paper_1801_01473_gb300 as p
    from paper_1801_01473_gb300 import slab as sl
    dims, mass, shifts, tol = (8, 8, 8, 16), 0.1, [1e-3, 0.02, 0.3, 1.5], 1e-10
    u = S.gauge_links(dims, "expih", 1404)
    b = S.gaussian_field(dims, 1405)
    ut = torch.from_numpy(u).cuda()

    def fn(rank, tr):
        slab = sl.Slab(dims, rank, 2)
        g = p.Gauge(slab.lattice, slab.stored_links(ut), "f64", 18)
        ops = sl.LibraryOps(slab, g)
        xs, st = sl.mscg(slab, ops, _stored(p, slab, b, "f64"), shifts, mass, tr, tol=tol, overlap=overlap)
        return [slab.local_part(p.unpack(slab.lattice, x).cpu().numpy()) for x in xs], st

    out = _run_threads(2, fn)
    ref = oracle.mscg(dims, u, mass, shifts, b, tol=tol)
    assert abs(out[0][1]["iters"] - ref["iters"]) <= 1 and out[0][1]["iters"] == out[1][1]["iters"]
    for i, sg in enumerate(shifts):
        x = np.concatenate([o[0][i] for o in out])
        assert oracle.true_residual(dims, u, mass, sg, b, x) <= 2 * tol, i
        kappa = (mass ** 2 + sg + 16.0) / (mass ** 2 + sg)
        assert np.linalg.norm(x - ref["x"][i]) / np.linalg.norm(ref["x"][i]) <= 2 * kappa * tol, i


def test_slab_lattice_rejected_outside_the_operator():
    import paper_1801_01473_gb300 as p
    from paper_1801_01473_gb300 import slab as sl
    from paper_1801_01473_gb300.lib import STG_ERR_SHAPE
    dims = (4, 4, 4, 8)
    slab = sl.Slab(dims, 0, 2)
    g = p.Gauge(slab.lattice, slab.stored_links(torch.from_numpy(S.gauge_links(dims, "haar", 1406)).cuda()), "f64", 18)
    x = g.new_field().zero_()
    with pytest.raises(p.StgError) as e:
        p.normal_op_(g, 0.1, 0.0, g.new_field(), x, g.new_field())
    assert e.value.status == STG_ERR_SHAPE
    with pytest.raises(p.StgError):
        p.mscg(g, torch.zeros((slab.lattice.Vh, 3), dtype=torch.complex128, device="cuda"), [0.1], 0.1)
