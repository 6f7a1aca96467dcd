"""Parity of the CUDA multi-shift CG with the FP64 oracle.

Every returned solution is re-checked with the oracle's own FP64 normal
operator: the bar is the true residual |b - A_i x_i| / |b| <= tol for every
shift (spec bar for the mixed paths), and for the pure FP64 path also
agreement of the first multi-shift recurrences with the oracle's (1e-12
relative) and of the solutions with the oracle's within the condition-number
bound kappa_i * tol.
"""
import os

import numpy as np
import pytest

import oracle
import synthetic as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
INNER = [None, ("f32", 12), ("f32", 18), ("f16", 12), ("bf16", 12)]


def stg():
    import paper_1801_01473_gb300 as p
    return p


def gauges(p, dims, u, inner):
    lat = p.Lattice(dims)
    ut = torch.from_numpy(u).cuda()
    g64 = p.Gauge(lat, ut, "f64", 18)
    gi = p.Gauge(lat, ut, inner[0], inner[1]) if inner else None
    return lat, g64, gi


def oracle_true_resid(dims, u, mass, shifts, b, x):
    return np.array([oracle.true_residual(dims, u, mass, s, b, x[i]) for i, s in enumerate(shifts)])


@pytest.fixture(scope="module")
def small():
    cfg = S.CONFIGS["small_4x4x4x4"]
    dims = cfg["dims"]
    u = S.gauge_links(dims, cfg["links"], 1000 + cfg["k"])
    b = S.gaussian_field(dims, 2000 + cfg["k"])
    return cfg, dims, u, b


@pytest.mark.parametrize("inner", INNER)
def test_small_true_residuals(small, inner):
    cfg, dims, u, b = small
    p = stg()
    shifts = cfg["shifts"]()
    _, g64, gi = gauges(p, dims, u, inner)
    x, st = p.mscg(g64, torch.from_numpy(b).cuda(), shifts, cfg["mass"], tol=cfg["tol"], g_inner=gi)
    x = x.cpu().numpy()
    tr = oracle_true_resid(dims, u, cfg["mass"], shifts, b, x)
    assert np.all(tr <= cfg["tol"]), (inner, tr, st)
    np.testing.assert_allclose(st["true_resid"], tr, rtol=1e-3, atol=1e-14)


def test_fp64_recurrences_match_oracle(small):
    cfg, dims, u, b = small
    p = stg()
    ref = np.loadtxt(os.path.join(GOLDEN, "mscg_4x4x4x4_scalars.txt"))
    _, g64, _ = gauges(p, dims, u, None)
    x, st = p.mscg(g64, torch.from_numpy(b).cuda(), cfg["shifts"](), cfg["mass"], tol=cfg["tol"], log_rows=25)
    log = st["scalar_log"]
    assert log.shape == ref.shape
    np.testing.assert_allclose(log[:20], ref[:20], rtol=1e-12)
    o = oracle.mscg(dims, u, cfg["mass"], cfg["shifts"](), b, tol=cfg["tol"])
    assert abs(st["iters"] - o["iters"]) <= 1
    # solutions agree within kappa_i * tol
    a_min, a_max = cfg["mass"] ** 2, cfg["mass"] ** 2 + 16.0
    for i, s in enumerate(cfg["shifts"]()):
        err = np.linalg.norm(x[i].cpu().numpy() - o["x"][i]) / np.linalg.norm(o["x"][i])
        assert err <= 2 * (a_max + s) / (a_min + s) * cfg["tol"]


@pytest.mark.parametrize("dims", [(6, 4, 2, 8), (2, 6, 4, 10), (12, 10, 6, 4)])
@pytest.mark.parametrize("inner", [None, ("f32", 12)])
def test_ragged_lattices(dims, inner):
    p = stg()
    u = S.gauge_links(dims, "expih", 77)
    b = S.gaussian_field(dims, 78)
    shifts = [0.0, 1e-3, 0.1, 2.0, 0.05]  # unsorted, base shift first
    _, g64, gi = gauges(p, dims, u, inner)
    x, st = p.mscg(g64, torch.from_numpy(b).cuda(), shifts, 0.05, tol=1e-10, g_inner=gi)
    tr = oracle_true_resid(dims, u, 0.05, shifts, b, x.cpu().numpy())
    assert np.all(tr <= 1e-10), tr


def test_free_field_plane_wave():
    from tests import latutil as lu
    p = stg()
    dims, mass = (8, 4, 4, 6), 0.1
    n = (1, 2, 3, 1)
    psi = lu.plane_wave_even(dims, n, [0.3, 1.0j, -0.5])
    lam = mass ** 2 + np.sum(np.sin(lu.momentum(dims, n)) ** 2)
    shifts = [1e-4, 0.01, 0.3]
    _, g64, _ = gauges(p, dims, S.unit_links(dims), None)
    x, st = p.mscg(g64, torch.from_numpy(psi).cuda(), shifts, mass, tol=1e-12)
    for i, s in enumerate(shifts):
        np.testing.assert_allclose(x[i].cpu().numpy(), psi / (lam + s), rtol=0, atol=1e-12 / (lam + s))
    assert st["iters"] == 1


def test_zero_source():
    p = stg()
    dims = (4, 4, 4, 4)
    _, g64, gi = gauges(p, dims, S.gauge_links(dims, "haar", 3), ("f32", 12))
    b = torch.zeros((128, 3), dtype=torch.complex128, device="cuda")
    x, st = p.mscg(g64, b, [0.0, 0.1], 0.1, g_inner=gi)
    assert torch.count_nonzero(x) == 0 and st["true_resid"] == [0.0, 0.0]


def test_max_iter_reports_noconv(small):
    cfg, dims, u, b = small
    p = stg()
    _, g64, _ = gauges(p, dims, u, None)
    from paper_1801_01473_gb300.lib import STG_ERR_NOCONV
    x, st = p.mscg(g64, torch.from_numpy(b).cuda(), cfg["shifts"](), cfg["mass"], tol=1e-10, max_iter=5,
                   allow_noconv=True)
    assert st["status"] == STG_ERR_NOCONV
    assert st["iters"] == 5 and max(st["true_resid"]) > 1e-10
    with pytest.raises(p.StgError):
        p.mscg(g64, torch.from_numpy(b).cuda(), cfg["shifts"](), cfg["mass"], tol=1e-10, max_iter=5)


def test_invalid_arguments_rejected():
    p = stg()
    dims = (4, 4, 4, 4)
    lat, g64, gi = gauges(p, dims, S.gauge_links(dims, "haar", 3), ("f32", 12))
    b = torch.from_numpy(S.gaussian_field(dims, 1)).cuda()
    with pytest.raises(p.StgError):
        p.mscg(g64, b, [-1.0], 0.1)              # negative shift
    with pytest.raises(p.StgError):
        p.mscg(g64, b, [0.0] * 33, 0.1)          # too many shifts
    with pytest.raises(p.StgError):
        p.mscg(gi, b, [0.0], 0.1)                # inner gauge passed as the FP64 gauge
    other = p.Gauge(p.Lattice((4, 4, 4, 6)), torch.from_numpy(S.gauge_links((4, 4, 4, 6), "haar", 4)).cuda(), "f32", 12)
    with pytest.raises(p.StgError):
        p.mscg(g64, b, [0.0], 0.1, g_inner=other)  # lattices differ
    with pytest.raises(p.StgError):
        p.mscg(g64, b, [0.0], 0.1, g_inner=gi, history=-1)  # negative history length


@pytest.mark.parametrize("inner", [("f32", 12), ("bf16", 12)])
def test_full_size_32x32x32x32_mixed(inner):
    """The benchmarked msCG workload: 32^4, 16 poles 1e-5..10, m = 0.01, true residual 1e-10.
    True residuals of four shifts (the hardest, two middle, the easiest) re-checked by the oracle."""
    p = stg()
    cfg = S.CONFIGS["mscg_32x32x32x32"]
    dims = cfg["dims"]
    u = S.gauge_links(dims, cfg["links"], 1000 + cfg["k"])
    b = S.gaussian_field(dims, 2000 + cfg["k"])
    shifts = cfg["shifts"]()
    _, g64, gi = gauges(p, dims, u, inner)
    x, st = p.mscg(g64, torch.from_numpy(b).cuda(), shifts, cfg["mass"], tol=cfg["tol"], g_inner=gi)
    assert max(st["true_resid"]) <= cfg["tol"]
    x = x.cpu().numpy()
    for i in (0, 5, 10, 15):
        assert oracle.true_residual(dims, u, cfg["mass"], shifts[i], b, x[i]) <= cfg["tol"]


def test_batched_uneven_matches_separate_solves():
    """Four lattices of different sizes, 4 sources each, 16 shifts, solved in one batch;
    every system's true residual <= tol; each instance agrees with its separate solve."""
    p = stg()
    cfg = S.CONFIGS["batched_uneven"]
    shifts = cfg["shifts"]()
    insts, keep = [], []
    for li, dims in enumerate(cfg["dims_list"]):
        u = S.gauge_links(dims, cfg["links"], 1000 + 10 * cfg["k"] + li)
        lat, g64, gi = gauges(p, dims, u, ("f32", 12))
        bs = [torch.from_numpy(S.gaussian_field(dims, 2000 + 10 * cfg["k"] + 4 * li + r)).cuda()
              for r in range(cfg["nrhs"])]
        insts.append((g64, gi, bs))
        keep.append((dims, u, lat))
    res = p.mscg_batched(insts, shifts, cfg["mass"], tol=cfg["tol"])
    for (x, stats), (g64, gi, bs), (dims, u, _) in zip(res, insts, keep):
        for r in range(len(bs)):
            assert max(stats[r]["true_resid"]) <= cfg["tol"]
        # one sampled system per lattice re-checked by the oracle, and vs a separate solve
        xs, _ = p.mscg(g64, bs[1], shifts, cfg["mass"], tol=cfg["tol"], g_inner=gi)
        b1 = bs[1].cpu().numpy()
        for i in (0, 15):
            assert oracle.true_residual(dims, u, cfg["mass"], shifts[i], b1, x[1, i].cpu().numpy()) <= cfg["tol"]
            rel = (torch.linalg.vector_norm(x[1, i] - xs[i]) / torch.linalg.vector_norm(xs[i])).item()
            assert rel <= 1e-7


def test_ill_conditioned_mixed_verified_in_fp64():
    """A shift whose condition number (~1.6e5: Haar links, m = 0.01, sigma = 0) puts the
    double-single residual error near tol: the mixed solve must still return every shift with an
    FP64 true residual <= tol (re-checked by the oracle), falling back to FP64 reliable updates
    when the FP64 verification fails."""
    p = stg()
    dims = (4, 4, 4, 4)
    u = S.gauge_links(dims, "haar", 1001)
    b = S.gaussian_field(dims, 2001)
    shifts = [0.0, 1e-3, 0.1]
    _, g64, gi = gauges(p, dims, u, ("f32", 12))
    x, st = p.mscg(g64, torch.from_numpy(b).cuda(), shifts, 0.01, tol=1e-10, g_inner=gi)
    tr = oracle_true_resid(dims, u, 0.01, shifts, b, x.cpu().numpy())
    assert np.all(tr <= 1e-10), (tr, st)
    assert st["fp64_fallback"] in (0, 1)


@pytest.mark.parametrize("inner", [None, ("f32", 12)])
def test_many_rhs_and_max_shifts(inner):
    """Limits of the batch: 10 sources on one lattice (two link-sharing groups of the multi-shift
    phase) and the maximum of 32 shifts, on a ragged lattice; every system checked by the oracle."""
    p = stg()
    dims = (6, 4, 4, 8)
    u = S.gauge_links(dims, "expih", 91)
    shifts = list(S.log_poles(1e-4, 5.0, 32))
    lat, g64, gi = gauges(p, dims, u, inner)
    bs = [torch.from_numpy(S.gaussian_field(dims, 920 + r)).cuda() for r in range(10)]
    (x, stats), = p.mscg_batched([(g64, gi, bs)], shifts, 0.05, tol=1e-10)
    assert x.shape == (10, 32, lat.Vh, 3)
    for r in (0, 9):
        b = bs[r].cpu().numpy()
        tr = oracle_true_resid(dims, u, 0.05, shifts, b, x[r].cpu().numpy())
        assert np.all(tr <= 1e-10), (r, tr.max())
        assert max(stats[r]["true_resid"]) <= 1e-10


def test_batched_fp64_matches_single():
    """Pure-FP64 batch of two lattices: each system's solution equals its single solve bitwise
    (the per-system arithmetic and reduction order do not depend on the batch)."""
    p = stg()
    shifts = [1e-3, 0.05, 1.0]
    insts, singles = [], []
    for li, dims in enumerate([(4, 4, 4, 4), (6, 4, 2, 8)]):
        u = S.gauge_links(dims, "haar", 95 + li)
        _, g64, _ = gauges(p, dims, u, None)
        bs = [torch.from_numpy(S.gaussian_field(dims, 960 + 2 * li + r)).cuda() for r in range(2)]
        insts.append((g64, None, bs))
        singles.append([p.mscg(g64, b, shifts, 0.1, tol=1e-11)[0] for b in bs])
    res = p.mscg_batched(insts, shifts, 0.1, tol=1e-11)
    for (x, _), ref in zip(res, singles):
        for r in range(2):
            assert torch.equal(x[r], ref[r])


def test_mixed_batch_bitwise_across_launch_shapes(monkeypatch):
    """A mixed batch (4 sources sharing link loads, refinement in groups of 4 rhs, converged
    members skipped) run with the shared-link multi-rhs operator, the one-hop-lookahead operator
    and the 128-thread register operator: bitwise equal solutions and statistics (the operators
    round identically), every system <= tol."""
    p = stg()
    dims = (8, 4, 6, 6)
    u = S.gauge_links(dims, "expih", 93)
    shifts = [1e-3, 2e-2, 0.3, 2.0]
    lat, g64, gi = gauges(p, dims, u, ("f32", 12))
    bs = [torch.from_numpy(S.gaussian_field(dims, 930 + r)).cuda() for r in range(4)]
    out = {}
    for shape in ("128", "shared", "ahead"):
        monkeypatch.setenv("STG_DSLASH_SHAPE", shape)
        (x, stats), = p.mscg_batched([(g64, gi, bs)], shifts, 0.05, tol=1e-10)
        out[shape] = (x.clone(), [(s["iters"], s["refine_iters"], s["reliable_updates"]) for s in stats])
        for r in range(4):
            assert max(stats[r]["true_resid"]) <= 1e-10
    for shape in ("shared", "ahead"):
        assert torch.equal(out["128"][0], out[shape][0]), shape
        assert out["128"][1] == out[shape][1], shape


@pytest.mark.parametrize("mass,tol", [(0.3, 1e-7), (0.05, 1e-6), (0.01, 1e-7)])
def test_loose_tolerance_double_single_certified(mass, tol):
    """At loose tolerances (MD force solves) the double-single residual certifies a shift without
    the FP64 operator when tol is ten times its rounding-error bound; where the bound is too large
    (m = 0.01, sigma = 0) the FP64 check still runs.  Either way the oracle's FP64 residual of every
    shift is within tol and the reported residual matches it."""
    p = stg()
    dims = (4, 4, 6, 8)
    u = S.gauge_links(dims, "expih", 1011)
    b = S.gaussian_field(dims, 2011)
    shifts = [0.0, 0.01, 0.5, 4.0]
    _, g64, gi = gauges(p, dims, u, ("f32", 12))
    x, st = p.mscg(g64, torch.from_numpy(b).cuda(), shifts, mass, tol=tol, g_inner=gi)
    tr = oracle_true_resid(dims, u, mass, shifts, b, x.cpu().numpy())
    assert np.all(tr <= tol), (tr, st)
    np.testing.assert_allclose(st["true_resid"], tr, rtol=1e-3, atol=1e-14)


@pytest.mark.parametrize("history", [0, 8, 24])
def test_deferred_update_matches_per_iteration(small, history):
    """The deferred multi-shift update (x_i, p_i formed once per window of stored FP32 residuals)
    against per-iteration updates (history=1): the multi-shift recurrences do not depend on x_i, so
    the scalar log and iteration counts agree bitwise; every shift meets tol in the oracle's FP64
    residual and the two solutions agree to the solve's accuracy.  history=8 flushes (and
    materialises p_i) every 8 iterations."""
    cfg, dims, u, b = small
    p = stg()
    shifts = cfg["shifts"]()
    _, g64, gi = gauges(p, dims, u, ("f32", 12))
    bt = torch.from_numpy(b).cuda()
    x1, st1 = p.mscg(g64, bt, shifts, cfg["mass"], tol=cfg["tol"], g_inner=gi, log_rows=40, history=1)
    xh, sth = p.mscg(g64, bt, shifts, cfg["mass"], tol=cfg["tol"], g_inner=gi, log_rows=40, history=history)
    assert st1["iters"] == sth["iters"] and st1["iters"] > 16
    np.testing.assert_array_equal(st1["scalar_log"], sth["scalar_log"])
    trh = oracle_true_resid(dims, u, cfg["mass"], shifts, b, xh.cpu().numpy())
    assert np.all(trh <= cfg["tol"]), (trh, sth)
    for i in range(len(shifts)):
        d = (x1[i] - xh[i]).abs().max().item() / x1[i].abs().max().item()
        assert d < 1e-8, (i, d)


def test_deferred_update_batched_uneven_windows():
    """Windows of 8 residuals over a batch of lattices of different sizes and several sources:
    every system within tol (oracle), iteration counts equal to per-iteration updates."""
    p = stg()
    shifts = [0.0, 0.02, 0.3, 2.0, 9.0]
    insts, data = [], []
    for k, dims in enumerate([(4, 4, 4, 4), (4, 4, 6, 8), (6, 6, 6, 4)]):
        u = S.gauge_links(dims, "expih", 1030 + k)
        bs = [S.gaussian_field(dims, 2030 + 10 * k + r) for r in range(2)]
        _, g64, gi = gauges(p, dims, u, ("f32", 12))
        insts.append((g64, gi, [torch.from_numpy(b).cuda() for b in bs]))
        data.append((dims, u, bs))
    res8 = p.mscg_batched(insts, shifts, 0.1, tol=1e-10, history=8)
    res1 = p.mscg_batched(insts, shifts, 0.1, tol=1e-10, history=1)
    for (dims, u, bs), (x8, st8), (_, st1) in zip(data, res8, res1):
        for r, b in enumerate(bs):
            assert st8[r]["iters"] == st1[r]["iters"]
            tr = oracle_true_resid(dims, u, 0.1, shifts, b, x8[r].cpu().numpy())
            assert np.all(tr <= 1e-10), tr


@pytest.mark.parametrize("dims,mass", [((12, 10, 6, 4), 0.05), ((6, 4, 2, 8), 0.01)])
def test_anchored_refinement_reports_true_residuals(dims, mass):
    """Tight mixed solves anchor each shift's residual in FP64 once and then update it by - A y in
    double-single for every refinement correction y: the reported residuals must equal the oracle's
    FP64 recomputation from the returned solutions (to 1e-3 tol), on the first solve of a process
    (the in-place update launch must run once, untuned) and on a second one."""
    p = stg()
    u = S.gauge_links(dims, "expih", 79)
    b = S.gaussian_field(dims, 80)
    shifts = [0.0, 1e-4, 3e-3, 0.1, 2.0]
    _, g64, gi = gauges(p, dims, u, ("f32", 12))
    for _ in range(2):
        x, st = p.mscg(g64, torch.from_numpy(b).cuda(), shifts, mass, tol=1e-10, g_inner=gi)
        tr = oracle_true_resid(dims, u, mass, shifts, b, x.cpu().numpy())
        assert np.all(tr <= 1e-10), tr
        assert np.abs(np.asarray(st["true_resid"]) - tr).max() <= 1e-13, (st["true_resid"], tr)
