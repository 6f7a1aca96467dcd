"""Benchmark of the staggered hot path on GB300 (one JSON line on stdout).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference] [--batch B] [--no-extras]

Headline metric (metric string as the project defines it):
  "D_eo GB/s (% HBM peak); msCG s/solve to 1e-10, mixed vs FP64 on 1 GB300"
value = effective D_eo bandwidth on the 32^4 workload (exp(i 0.3 H) links stored FP32
12-real, complex64 vectors): algorithmic bytes (all 4V links once + one input and one
output vector = 432 B per even site) / device time.  One step applies D_eo to a batch of
B distinct even-site vectors (B launches of the kernel), alternating between two copies of
the links, so that no step finds its links or vectors in L2 (inputs larger than L2).

The same JSON line carries (measured in the same run, outside the timed steps):
  e2e        the metric through the public API with host tensors: pinned host fields streamed
             through stg_dslash_host (host -> device copy of each canonical complex64 input --
             the workload computes in FP32 -- pack, D_eo, unpack, device -> host, pipelined on
             three streams; the complex128 figure beside it);
  roofline   D_eo FP32-12 against the measured HBM copy bandwidth;
  sweep      16^4 and 32^4 D_eo for every link storage (and 32^4 D_oe for FP64-18, FP32-12 and
             BF16-12): single launches after an L2 flush that leaves clean lines (median of 50),
             and back-to-back launches over distinct sources alternating two link copies; GB/s
             and fraction of the measured HBM bandwidth;
  mscg       32^4 msCG (16 poles 1e-5..10, m = 0.01, true residual 1e-10): mixed
             (FP32, FP16, BF16 inner; double-single reliable updates, FP64-verified) vs pure
             FP64, s/solve, and the effective bandwidth of the algorithmic bytes; the FP32-inner
             solve also end to end through stg.mscg with a pinned host source;
  batched    the uneven batch (16^4, 24^3x8, 32^3x8, 24^4, 4 sources x 16 shifts) in one
             solve vs the sum of separate solves, with per-instance iteration counts;
  force      48^4 fermion force (12 shifts): whole call, its double-single D_oe part and the
             per-link gather, with fractions of the measured HBM bandwidth;
  slab       the slab decomposition's D on one of two slabs of the 32^4 lattice (local sites, and
             its border and bulk launches), one GPU;
  cpu_baseline  the FP64 oracle on the host cores: D_eo at 16^4 and 32^4 and capped msCG
             iterations at 32^4, on one thread and on all of them.
--impl reference times that oracle as the reference arm (the paper ships no code).
Multi-GPU: replicas only (independent copies of the workload on every rank).
"""
from __future__ import annotations

import argparse
import json
import os
import re
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synthetic as S  # noqa: E402

METRIC = "D_eo GB/s (% HBM peak); msCG s/solve to 1e-10, mixed vs FP64 on 1 GB300"
UNIT = "GB/s"
WORKLOAD = "32^4 D_eo, exp(i0.3H) links FP32 12-real, complex64 vectors, batch of distinct sources"
LINK_BYTES = {("f64", 18): 144, ("f64", 12): 96, ("ds", 18): 144, ("ds", 12): 96, ("f32", 18): 72,
              ("f32", 12): 48, ("bf16", 12): 24, ("f16", 12): 24}


_LINKS = {}


def links_cached(dims, kind, seed):
    """Seeded synthetic links, generated once per (dims, kind, seed) in this process."""
    key = (tuple(dims), kind, seed)
    if key not in _LINKS:
        _LINKS[key] = S.gauge_links(dims, kind, seed)
    return _LINKS[key]


def workload_config(batch, ws=1):
    """The `config` object of the JSON line (shared by both arms)."""
    return {"workload": WORKLOAD, "lattice": "32x32x32x32", "links": "f32-12", "vectors": "c64",
            "batch_per_step": batch, "bytes_per_site": bytes_per_site("f32", 12),
            "l2": "inputs larger than L2: distinct source per launch, two alternating 201 MB link copies",
            "parallelism": f"replicas x{ws}"}


def bytes_per_site(prec, recon):
    """Algorithmic bytes of one D_eo output site: 8 links (all 4V links once over the
    lattice) + one input and one output colour vector."""
    vec = 48 if prec in ("f64", "ds") else 24
    return 8 * LINK_BYTES[(prec, recon)] + 2 * vec


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(t: float) -> float:
    """The largest of the ranks' timed-region durations (every rank gets it); t itself on one rank."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return t
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    tt = torch.tensor([t], dtype=torch.float64, device=dev)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return float(tt.item())


def replica_throughput(bytes_per_rank: float, t_max: float, ws: int) -> float:
    """Whole-job GB/s of `ws` independent replicas that each moved bytes_per_rank in at most t_max s."""
    return ws * bytes_per_rank / t_max / 1e9


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def profile_traffic(name):
    """dram bytes per launch from a committed ncu summary (profiles/<name>.md), or None."""
    path = os.path.join(ROOT, "profiles", name)
    if not os.path.exists(path):
        return None
    m = re.search(r"dram_bytes_per_launch:\s*([0-9.eE+]+)", open(path).read())
    return float(m.group(1)) if m else None


class ClockSampler:
    """nvidia-smi clock/throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index=0):
        self.idx = gpu_index
        self.proc = None
        self.path = os.path.join("/tmp", f"stg_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        rows = [r.split(",") for r in open(self.path).read().strip().splitlines() if r.strip()]
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if len(r) > 5 + k and "Active" in r[5 + k]
                          and "Not" not in r[5 + k]})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------------------- reference arm


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    dims = S.CONFIGS["bandwidth_32x32x32x32"]["dims"]
    u = links_cached(dims, "expih", 1000 + 2)
    psi = S.gaussian_field(dims, 2000 + 2)
    vh = S.volume(dims) // 2
    alg = bytes_per_site("f32", 12) * vh
    for _ in range(args.warmup):
        oracle.dslash_eo(dims, u, psi)
    ts = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.dslash_eo(dims, u, psi)
        ts.append(time.perf_counter() - t0)
    t = float(np.sum(ts))
    v = alg * args.steps / t / 1e9
    line = {"metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": workload_config(args.batch, ws),
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                             "sample": f"one FP64 oracle D_eo application at 32^4 per step ({args.steps} steps), "
                                       "bytes counted as the FP32-12 workload"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def cpu_baseline(d_budget_s=2.0, mscg_iters=(12, 4)):
    """The FP64 oracle on the host cores: D_eo at 16^4 and 32^4, and the 32^4 msCG workload's
    multi-shift iterations (capped, reported per iteration), each on one thread and on all of them.
    `value` (the line's unit) is D_eo at 32^4 on all threads, bytes counted as the FP32-12
    workload.  About 15 s of CPU work in all."""
    import oracle
    oracle.build()
    nall = os.cpu_count() or 1
    cases = []
    value = None
    for key in ("bandwidth_16x16x16x16", "bandwidth_32x32x32x32"):
        cfg = S.CONFIGS[key]
        dims = cfg["dims"]
        u = links_cached(dims, cfg["links"], 1000 + cfg["k"])
        psi = S.gaussian_field(dims, 2000 + cfg["k"])
        vh = S.volume(dims) // 2
        for nthr in (1, nall):
            oracle.set_num_threads(nthr)
            oracle.dslash_eo(dims, u, psi)
            n, t = 0, 0.0
            while (t < d_budget_s and n < 50) or n < 2:
                t0 = time.perf_counter()
                oracle.dslash_eo(dims, u, psi)
                t += time.perf_counter() - t0
                n += 1
            gbs = bytes_per_site("f32", 12) * vh * n / t / 1e9
            cases.append({"case": f"D_eo {'x'.join(map(str, dims))}", "threads": nthr, "calls": n,
                          "ms_per_call": round(1e3 * t / n, 2), "GBs_f32r12_equiv": round(gbs, 3)})
            if key == "bandwidth_32x32x32x32" and nthr == nall:
                value = gbs
    cfg = S.CONFIGS["mscg_32x32x32x32"]
    dims = cfg["dims"]
    u = links_cached(dims, cfg["links"], 1000 + cfg["k"])
    b = S.gaussian_field(dims, 2000 + cfg["k"])
    for nthr, cap in ((nall, mscg_iters[0]), (1, mscg_iters[1])):
        oracle.set_num_threads(nthr)
        t0 = time.perf_counter()
        r = oracle.mscg(dims, u, cfg["mass"], cfg["shifts"](), b, tol=cfg["tol"], max_iter=cap, finish=False)
        t = time.perf_counter() - t0
        cases.append({"case": "msCG 32x32x32x32, 16 shifts, multi-shift iterations", "threads": nthr,
                      "iters": r["iters"], "ms_per_iter": round(1e3 * t / r["iters"], 1),
                      "note": f"capped at {cap} iterations; the GPU solve needs ~210 plus refinement"})
    oracle.set_num_threads(nall)
    return {"value": value, "unit": UNIT, "cores": nall, "kind": "oracle",
            "sample": "FP64 oracle D_eo at 32^4 on all host threads (bytes counted as the FP32-12 workload); "
                      "cases: D_eo at 16^4 and 32^4 and capped msCG iterations at 32^4, on 1 and all threads",
            "cases": cases}


# ---------------------------------------------------------------------------- GPU arm


def events(torch):
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


class L2Flush:
    """Evicts L2 between timed launches and leaves it holding clean lines: writes one 256 MB
    buffer (> the 129 MB L2), then reads another.  A write alone leaves up to an L2 of dirty lines
    that the next kernel must write back to HBM, which would be charged to that kernel."""

    def __init__(self, torch):
        self.w = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
        self.r = torch.ones(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
        self.sink = torch.zeros((), dtype=torch.float32, device="cuda")
        self.k = 0

    def __call__(self):
        self.k += 1
        self.w.fill_(float(self.k))
        self.sink.copy_(self.r.sum())


def time_deo_sweep(torch, p, dims, peak, reps=50, b2b_batch=32, doe=()):
    """D_eo per storage kind at `dims`: single launches after an L2 flush (median of reps), and
    back-to-back launches over distinct sources alternating two copies of the links (the
    configuration of the headline number; replayed from a CUDA graph).  D_oe is timed the same way
    for the storage kinds listed in `doe` ((prec, recon) pairs, no phase field)."""
    cfg_links = links_cached(dims, "expih", 1000 + 2)
    ut = torch.from_numpy(cfg_links).cuda()
    lat = p.Lattice(dims)
    psi = torch.from_numpy(S.gaussian_field(dims, 2000 + 2)).cuda()
    flush = L2Flush(torch)
    out = []
    theta = torch.from_numpy(np.random.default_rng(4000 + 2).uniform(-np.pi, np.pi, (4, lat.V))).cuda()

    def time_op(fn, gs, x, y, src, dst):
        for _ in range(5):
            fn(gs[0], y, x)
        ts = []
        for _ in range(reps):
            flush()
            e0, e1 = events(torch)
            e0.record()
            fn(gs[0], y, x)
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1) * 1e-3)
        t = float(np.median(ts))
        # back to back: the launches captured once into a CUDA graph, so that host launch overhead
        # (~10 us per ctypes call) cannot starve the small lattices
        for j in range(b2b_batch):
            fn(gs[j & 1], dst[j], src[j])
        torch.cuda.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            for j in range(b2b_batch):
                fn(gs[j & 1], dst[j], src[j])
        graph.replay()
        e0, e1 = events(torch)
        e0.record()
        for _ in range(3):
            graph.replay()
        e1.record()
        torch.cuda.synchronize()
        del graph
        return t, e0.elapsed_time(e1) * 1e-3 / (3 * b2b_batch)

    for prec, recon, u1 in [("f64", 18, False), ("f64", 12, False), ("ds", 18, False), ("ds", 12, False),
                            ("f32", 18, False), ("f32", 12, False), ("f16", 12, False), ("bf16", 12, False),
                            ("f64", 18, True), ("ds", 18, True), ("f32", 12, True), ("f16", 12, True)]:
        gs = [p.Gauge(lat, ut, prec, recon, theta=theta if u1 else None) for _ in range(2)]
        x = p.pack(lat, psi, gs[0].vec_prec)
        src = x.unsqueeze(0).repeat(b2b_batch, 1)
        dst = torch.empty_like(src)
        y = torch.empty_like(x)
        # a U(1) phase field adds one stored phase per link ((cos, sin) doubles for f64/ds, a float angle otherwise)
        byt = (bytes_per_site(prec, recon) + (8 * (16 if prec in ("f64", "ds") else 4) if u1 else 0)) * lat.Vh
        ops = [("D_eo", p.dslash_eo_)] + ([("D_oe", p.dslash_oe_)] if (prec, recon) in doe and not u1 else [])
        for name, fn in ops:
            t, tb = time_op(fn, gs, x, y, src, dst)
            out.append({"lattice": "x".join(map(str, dims)), "op": name,
                        "links": f"{prec}-{recon}" + ("+u1" if u1 else ""),
                        "us": round(t * 1e6, 2), "GBs": round(byt / t / 1e9, 1),
                        "frac": round(byt / t / 1e9 / peak, 3),
                        "b2b_us": round(tb * 1e6, 2), "b2b_GBs": round(byt / tb / 1e9, 1),
                        "b2b_frac": round(byt / tb / 1e9 / peak, 3)})
        del gs, src, dst
    return out


def mscg_standard_bytes(vh, st, inner):
    """Standard per-iteration byte count of one msCG solve on one system (a figure of merit: the
    traffic of a multi-shift CG that reads each operand once per iteration, shift and right-hand
    side, without the solver's shared link loads and deferred shift updates).
    Multi-shift phase, per iteration and even site: 2 (8 links + 2 v) for D_oe and D_eo, 5 v for
    r, p, q, and 4 v for x_i, p_i of each active shift -- summed with the real number of active
    shifts of every iteration.  Refinement, per CG iteration of a shift: 2 (8 links + 2 v) + 7 v on
    the FP32 12-real operator; per reliable update the double-single residual,
    2 (8 x 144 + 2 x 48) + 4 x 48.  inner: (link bytes, vector bytes) of the multi-shift phase."""
    lb, v = inner
    p1 = st["iters"] * (2 * (8 * lb + 2 * v) + 5 * v) + 4 * v * sum(st["shift_iters"])
    if lb >= 144:  # pure FP64 solve: no refinement
        return vh * p1
    ref = sum(st["refine_shift_iters"]) * (2 * (8 * 48 + 2 * 24) + 7 * 24)
    rel = sum(st["shift_reliable_updates"]) * (2 * (8 * 144 + 2 * 48) + 4 * 48)
    return vh * (p1 + ref + rel)


# launch grouping of the solver (solver.cu): right-hand sides per multi-shift D launch group,
# (rhs, shift) pairs per refinement group, residuals per deferred-update window, shifts per flush block
SOLVER_RHS_GROUP, SOLVER_REFINE_GROUP, SOLVER_HIST_MAX, SOLVER_FLUSH_SHIFTS = 8, 4, 256, 8


def mscg_moved_bytes(insts, lb_inner, mixed, nshift):
    """Bytes the kernels of one msCG call must move, from its per-system statistics: every field
    a kernel touches read or written once (neighbours from cache), links once per launch group and
    iteration in which any member of the group is live (the group's longest member: a lower bound).
    insts: [(Vh, [stats of each right-hand side])]; lb_inner: link bytes of the multi-shift phase.
    Mixed solves: FP32 vectors (24 B a site), double-single solutions (48 B), deferred shift
    updates, refinement on FP32 12-real links (48 B), double-single residual operator (144 B),
    FP64 anchor (144 B), i.e. the anchored refinement these tolerances select.  FP64 solves: FP64
    vectors (48 B), per-iteration shift updates, one FP64 residual check per shift.
    Returns (bytes, bytes of the FP64-arithmetic D launches, their FP64 FMAs): FP64 D is bound by
    GB300's FP64 pipe (DFMA_PER_SITE FMAs a site and right-hand side), not by HBM."""
    v, vh, l64, lr, lh = (24, 48, 144, 48, 144) if mixed else (48, 48, 144, 144, 144)
    f64_b, f64_fma = 0, 0
    W = 0
    if mixed:
        ring = sum(len(sts) * n * 24 for n, sts in insts)
        fit = (16 << 30) // max(ring, 1)
        W = min(SOLVER_HIST_MAX, fit - 1) if fit > 1 else 8
        W = max(8, W - W % 8)
    total = 0
    for n, sts in insts:
        b = 0
        fb, ff = 0, 0  # this lattice's FP64 D bytes and FMAs (per even site)
        for g0 in range(0, len(sts), SOLVER_RHS_GROUP):  # multi-shift D: links per rhs group
            b += 2 * 8 * lb_inner * max(s["iters"] for s in sts[g0:g0 + SOLVER_RHS_GROUP])
            if not mixed:
                fb += 2 * 8 * lb_inner * max(s["iters"] for s in sts[g0:g0 + SOLVER_RHS_GROUP])
        for s in sts:
            it, si = s["iters"], list(s["shift_iters"])
            if not mixed:
                fb += it * 5 * v
                ff += it * 2 * DFMA_PER_SITE
            # start: canonical b; r, every p_i (and the window's base copy); x_i = 0; b in FP64/DS
            b += 48 + v + nshift * (v + vh) + (v if W else 0) + vh
            # per iteration: D_oe p->t (2v), D_eo t,p->q (3v), r -= alpha q (3v)
            b += it * 8 * v
            if W:
                b += it * 3 * v  # base direction p = r + beta p
                for w0 in range(0, it, W):  # window flushes
                    w1 = min(w0 + W, it)
                    live = [i for i in range(nshift) if si[i] > w0]
                    pmat = [i for i in range(nshift) if si[i] > w1 and w1 < it]
                    chunks = {i // SOLVER_FLUSH_SHIFTS for i in live + pmat}
                    b += len(chunks) * (w1 - w0) * v        # residual ring
                    b += len(live) * (v + 2 * vh)          # P0_i read, x_i read and written
                    b += len(pmat) * v + (v if w1 < it else 0)  # p_i (and the base copy) written
            else:
                b += it * v + sum(si) * (2 * v + 2 * vh)  # r once, then p_i and x_i per live shift
        # refinement and residuals: (rhs, shift) pairs in groups of SOLVER_REFINE_GROUP
        pairs = [(s, i) for s in sts for i in range(nshift)]
        for q0 in range(0, len(pairs), SOLVER_REFINE_GROUP):
            grp = pairs[q0:q0 + SOLVER_REFINE_GROUP]
            rit = [s["refine_shift_iters"][i] if mixed else 0 for s, i in grp]
            rel = [s["shift_reliable_updates"][i] if mixed else 0 for s, i in grp]
            res_d = 2 * v + 3 * v  # the D pair of one residual, vector part (precision of the pass)
            # first true residual of every pair: FP64 anchor (mixed) or FP64 check, links once
            b += 2 * 8 * l64 + len(grp) * 6 * vh
            fb += 2 * 8 * l64 + len(grp) * 6 * vh
            ff += len(grp) * 2 * DFMA_PER_SITE
            if mixed:
                b += len(grp) * (2 * vh + 2 * vh + 2 * vh)  # x to FP64 and back, r to DS
                b += 2 * 8 * lr * max(rit) + sum(rit) * (res_d + 3 * v + 5 * v)
                # reliable updates: fold (y, x, y_hi, y=0), r_hi -= A y_hi (DS), r = r_hi
                b += 2 * 8 * lh * max(rel) + sum(rel) * ((v + 2 * vh + vh + v) + 6 * vh + (vh + v))
            b += len(grp) * (vh + 3 * v)  # r = r_hi, p = r, y = 0 after the first residual
            b += len(grp) * 2 * vh        # solution to the output layout
        if mixed:
            b += len(sts) * 3 * 2 * vh    # b between DS and FP64 around the anchor and at the end
        total += n * b
        f64_b += n * fb
        f64_fma += n * ff
    return total, f64_b, f64_fma


# FP64 FMAs of one staggered D application per output site and right-hand side: 8 hops, each a
# 3 x 3 complex matrix times a colour vector (36 real FMAs) and its signed accumulation (6)
DFMA_PER_SITE = 8 * (36 + 6)
# GB300 FP64 FMA rate: 2 per clock and SM (ncu sm__sass_thread_inst_executed_op_dfma_pred_on
# .peak_sustained), 152 SMs, 2070 MHz: the nominal 1.25 TFLOP/s
FP64_FMA_PER_S = 2 * 152 * 2.07e9


def mscg_bound_s(moved, hbm_gbs):
    """Lower bound of a solve's time from (bytes, FP64 D bytes, FP64 D FMAs): HBM time of all other
    bytes plus, for the FP64 D launches, the larger of their HBM and FP64-pipe times."""
    total, fb, ff = moved
    return (total - fb) / (hbm_gbs * 1e9) + max(fb / (hbm_gbs * 1e9), ff / FP64_FMA_PER_S)


def time_mscg(torch, p, peak, reps=3):
    cfg = S.CONFIGS["mscg_32x32x32x32"]
    dims = cfg["dims"]
    ut = torch.from_numpy(links_cached(dims, cfg["links"], 1000 + cfg["k"])).cuda()
    b = torch.from_numpy(S.gaussian_field(dims, 2000 + cfg["k"])).cuda()
    lat = p.Lattice(dims)
    g64 = p.Gauge(lat, ut, "f64", 18)
    shifts = cfg["shifts"]()
    res = {}
    for name, inner, ib in [("fp32", ("f32", 12), (48, 24)), ("fp16", ("f16", 12), (24, 24)),
                            ("bf16", ("bf16", 12), (24, 24)), ("fp64", None, (144, 48))]:
        gi = p.Gauge(lat, ut, inner[0], inner[1]) if inner else None
        p.mscg(g64, b, shifts, cfg["mass"], tol=cfg["tol"], g_inner=gi, allow_noconv=True)  # autotune, untimed
        ts = []
        st = None
        for _ in range(reps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            _, st = p.mscg(g64, b, shifts, cfg["mass"], tol=cfg["tol"], g_inner=gi, allow_noconv=True)
            torch.cuda.synchronize()
            ts.append(time.perf_counter() - t0)
        t = float(np.median(ts))
        moved = mscg_moved_bytes([(lat.Vh, [st])], ib[0], inner is not None, len(shifts))
        alg, bound = moved[0], mscg_bound_s(moved, peak)
        std = mscg_standard_bytes(lat.Vh, st, ib)
        res[name] = {"s_per_solve": round(t, 5), "iters": st["iters"],
                     "refine_iters": st["refine_iters"], "reliable_updates": st["reliable_updates"],
                     "max_true_resid": float(max(st["true_resid"])), "converged": st["status"] == 0,
                     "alg_GB": round(alg / 1e9, 2), "eff_GBs": round(alg / t / 1e9, 1),
                     "frac": round(alg / t / 1e9 / peak, 3),
                     "fp64_d_GFMA": round(moved[2] / 1e9, 2), "bound_s": round(bound, 5),
                     "frac_of_bound": round(bound / t, 3),
                     "std_GB": round(std / 1e9, 2), "std_eff_GBs": round(std / t / 1e9, 1),
                     "shift_iters": list(st["shift_iters"]), "refine_shift_iters": list(st["refine_shift_iters"]),
                     "shift_reliable_updates": list(st["shift_reliable_updates"])}
        if name == "fp32":
            # end to end through the public call with host tensors: b copied in from pinned host
            # memory, the solutions copied back to pinned host memory, inside the timed region
            bh = b.cpu().pin_memory()
            xh, _ = p.mscg(g64, bh, shifts, cfg["mass"], tol=cfg["tol"], g_inner=gi, allow_noconv=True)
            nb_out = int(xh.numel() * xh.element_size())
            del xh  # untimed call: torch's pinned host allocator keeps the result buffer for reuse
            ts = []
            for _ in range(reps):
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                xh, _ = p.mscg(g64, bh, shifts, cfg["mass"], tol=cfg["tol"], g_inner=gi, allow_noconv=True)
                ts.append(time.perf_counter() - t0)
                del xh
            res[name]["e2e"] = {"s_per_solve": round(float(np.median(ts)), 5),
                                "h2d_bytes": int(bh.numel() * bh.element_size()), "d2h_bytes": nb_out,
                                "note": "stg.mscg with a pinned host source: copy in, solve, all solutions "
                                        "copied back to pinned host memory, inside the timed region"}
        del gi
    res["mixed_speedup_vs_fp64"] = round(res["fp64"]["s_per_solve"] / min(
        res[k]["s_per_solve"] for k in ("fp32", "fp16", "bf16") if res[k]["converged"]), 3)
    res["note"] = ("alg_GB: bytes the solver's kernels must move (links once per launch group, deferred shift "
                   "updates, grouped refinement, anchor and reliable updates; bench.py mscg_moved_bytes); "
                   "eff_GBs = alg_GB / solve time, frac of measured HBM; bound_s: HBM time of those bytes with "
                   "the FP64-arithmetic D launches (FP64 solve, FP64 anchor) at the larger of their HBM and "
                   "FP64-pipe times (2 DFMA per clock and SM, 152 SMs, 2070 MHz), frac_of_bound = bound_s / "
                   "solve time; std_GB: the standard per-iteration, per-shift count (mscg_standard_bytes), "
                   "a figure of merit only")
    return res


def time_batched(torch, p, peak, reps=2):
    cfg = S.CONFIGS["batched_uneven"]
    shifts = cfg["shifts"]()
    insts = []
    for li, dims in enumerate(cfg["dims_list"]):
        ut = torch.from_numpy(links_cached(dims, cfg["links"], 1000 + 10 * cfg["k"] + li)).cuda()
        lat = p.Lattice(dims)
        bs = [torch.from_numpy(S.gaussian_field(dims, 2000 + 10 * cfg["k"] + 4 * li + r)).cuda()
              for r in range(cfg["nrhs"])]
        insts.append((p.Gauge(lat, ut, "f64", 18), p.Gauge(lat, ut, "f32", 12), bs))
    # one untimed call of each shape first: the library autotunes launch shapes on first use
    p.mscg_batched(insts, shifts, cfg["mass"], tol=cfg["tol"])
    for g64, gi, bs in insts:
        p.mscg(g64, bs[0], shifts, cfg["mass"], tol=cfg["tol"], g_inner=gi)
    tb = []
    for _ in range(reps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        out = p.mscg_batched(insts, shifts, cfg["mass"], tol=cfg["tol"])
        torch.cuda.synchronize()
        tb.append(time.perf_counter() - t0)
    worst = max(max(s["true_resid"]) for _, sts in out for s in sts)
    moved = mscg_moved_bytes([(g64.lattice.Vh, sts) for (g64, _, _), (_, sts) in zip(insts, out)], 48, True,
                             len(shifts))
    alg = moved[0]
    std = sum(mscg_standard_bytes(g64.lattice.Vh, s, (48, 24)) for (g64, _, _), (_, sts) in zip(insts, out) for s in sts)
    per_inst = [{"lattice": "x".join(map(str, g64.lattice.dims)), "iters": [s["iters"] for s in sts],
                 "refine_iters": [s["refine_iters"] for s in sts]} for (g64, _, _), (_, sts) in zip(insts, out)]
    ts = 0.0
    for k, (g64, gi, bs) in enumerate(insts):
        sep = 0.0
        for b in bs:
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            p.mscg(g64, b, shifts, cfg["mass"], tol=cfg["tol"], g_inner=gi)
            torch.cuda.synchronize()
            sep += time.perf_counter() - t0
        ts += sep
        # the lattice's four sources as a batch of their own (link loads shared, no other lattice)
        p.mscg_batched([(g64, gi, bs)], shifts, cfg["mass"], tol=cfg["tol"])
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        p.mscg_batched([(g64, gi, bs)], shifts, cfg["mass"], tol=cfg["tol"])
        torch.cuda.synchronize()
        per_inst[k].update({"separate_s": round(sep, 5), "own_batch_s": round(time.perf_counter() - t0, 5)})
    t = float(np.median(tb))
    return {"s_per_batch": round(t, 5), "sum_of_separate_s": round(ts, 5),
            "speedup": round(ts / t, 3), "systems": 16, "shifts": 16,
            "max_true_resid": worst, "alg_GB": round(alg / 1e9, 2), "eff_GBs": round(alg / t / 1e9, 1),
            "frac": round(alg / t / 1e9 / peak, 3), "bound_s": round(mscg_bound_s(moved, peak), 5),
            "frac_of_bound": round(mscg_bound_s(moved, peak) / t, 3), "std_GB": round(std / 1e9, 2),
            "std_eff_GBs": round(std / t / 1e9, 1),
            "per_instance": per_inst}


def time_slab(torch, p, peak, reps=32):
    """The device part of the slab decomposition along t: one of two slabs of the 32^4 workload
    (32^3 x 16 local slices, stored with 2 + 2 halo slices), FP32-12 links: D_oe on the local sites
    back to back (graph replay), and its border (2 slices) and bulk (14 slices) launches of Alg. 1;
    GB/s over the local sites' algorithmic bytes."""
    from paper_1801_01473_gb300 import slab as sl
    dims = (32, 32, 32, 32)
    slab = sl.Slab(dims, 0, 2)
    lat = slab.lattice
    ut = torch.from_numpy(links_cached(dims, "expih", 1002)).cuda()
    g = p.Gauge(lat, slab.stored_links(ut), "f32", 12)
    del ut
    ops = sl.LibraryOps(slab, g)
    gen = torch.Generator(device="cuda").manual_seed(2002)
    x = torch.randn((2,) + tuple(g.new_field().shape), dtype=torch.float32, device="cuda", generator=gen)
    y = torch.zeros_like(x)
    out = {"global": "32x32x32x32", "local": "32x32x32x16", "stored": "32x32x32x20", "links": "f32-12"}
    local = 32 * 32 * 32 * 16 // 2
    for name, fn, sites in (("whole", lambda j: ops.dslash(1, y[j], x[j]), local),
                            ("borders", lambda j: ops.dslash_part(1, 1, y[j], x[j]), 2 * 32 * 32 * 32 // 2),
                            ("bulk", lambda j: ops.dslash_part(1, 2, y[j], x[j]), 14 * 32 * 32 * 32 // 2)):
        for j in range(2):
            fn(j)
        torch.cuda.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            for r in range(reps):
                fn(r & 1)
        graph.replay()
        e0, e1 = events(torch)
        e0.record()
        for _ in range(3):
            graph.replay()
        e1.record()
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1) * 1e-3 / (3 * reps)
        byt = bytes_per_site("f32", 12) * sites
        out[name] = {"us": round(t * 1e6, 2), "GBs": round(byt / t / 1e9, 1), "frac": round(byt / t / 1e9 / peak, 3)}
        del graph
    out["note"] = ("D_oe on one slab's local sites, reading the halo slices of its input; border + bulk is the "
                   "split Alg. 1 overlaps with the halo exchange; one GPU, so no exchange is timed")
    return out


# Fermion force per link (48^4, 12 shifts): the link (144 B), the output (144 B) and, with every
# vector read once per site, 12 x 48 B of x_i or y_i per site over its 4 links = 144 B.
FORCE_BYTES_PER_LINK = 3 * 144


def time_force(torch, p, peak):
    """48^4 fermion force: the whole call, and apart from it the 12 double-single D_oe
    applications y_i = D_oe x_i it contains (the rest is the per-link gather of W and F)."""
    cfg = S.CONFIGS["force_48x48x48x48"]
    dims = cfg["dims"]
    lat = p.Lattice(dims)
    ut = torch.from_numpy(links_cached(dims, cfg["links"], 1000 + cfg["k"])).cuda()
    g64 = p.Gauge(lat, ut, "f64", 18)
    gds = p.Gauge(lat, ut, "ds", 18)
    del ut
    res = S.positive_residues(3000 + cfg["k"], 12)
    g = torch.Generator(device="cuda").manual_seed(2000 + cfg["k"])
    x = torch.randn((12, lat.Vh, 3), dtype=torch.complex128, device="cuda", generator=g)
    p.fermion_force(g64, res, x)
    torch.cuda.synchronize()
    e0, e1 = events(torch)
    e0.record()
    for _ in range(3):
        f = p.fermion_force(g64, res, x)
    e1.record()
    torch.cuda.synchronize()
    t = e0.elapsed_time(e1) * 1e-3 / 3
    del f
    xd = p.pack(lat, x[0], "ds")
    yd = torch.empty_like(xd)
    p.dslash_oe_(gds, yd, xd)
    e0, e1 = events(torch)
    e0.record()
    for _ in range(12):
        p.dslash_oe_(gds, yd, xd)
    e1.record()
    torch.cuda.synchronize()
    t_d = e0.elapsed_time(e1) * 1e-3
    links = 4 * lat.V
    t_g = max(t - t_d, 1e-9)
    d_bytes = 12 * bytes_per_site("ds", 18) * lat.Vh
    return {"lattice": "48^4", "shifts": 12, "ms": round(t * 1e3, 3),
            "doe_ms": round(t_d * 1e3, 3), "doe_GBs": round(d_bytes / t_d / 1e9, 1),
            "doe_frac": round(d_bytes / t_d / 1e9 / peak, 3),
            "gather_ms": round(t_g * 1e3, 3), "gather_GBs": round(FORCE_BYTES_PER_LINK * links / t_g / 1e9, 1),
            "gather_frac": round(FORCE_BYTES_PER_LINK * links / t_g / 1e9 / peak, 3),
            "note": "double-single D_oe on the 12 solutions (FP32-pipe bound) + per-link gather of W in "
                    "double-single and F in FP64 (FP32/FP64-pipe bound); fractions are of measured HBM bandwidth"}


# Algorithmic FP64 flops per link of one stout step (complex 3x3 product = 27 complex
# multiply-adds = 216 flops): forward = 12 staple products + C U^dag + Q^2 + exp(iQ) U = 15
# products; the chain rule = the forward's 14 before the exp, E^dag G', G' U^dag, M Q + Q M,
# G_Omega^dag C, G_Omega U (6 more) + the 18 two-product staple terms (36).
STOUT_FWD_FLOPS = 15 * 216
STOUT_BWD_FLOPS = (14 + 6 + 36) * 216


def time_stout(torch, p):
    cfg = S.CONFIGS["force_48x48x48x48"]
    dims = cfg["dims"]
    lat = p.Lattice(dims)
    u64 = torch.from_numpy(links_cached(dims, cfg["links"], 1000 + cfg["k"])).cuda()
    rho, nstep = 0.15, 2
    out = {"lattice": "48^4", "steps": nstep, "rho": rho}
    for tag, ut in (("fp64", u64), ("fp32", p.complex_convert(u64, torch.complex64))):
        g = torch.Generator(device="cuda").manual_seed(3000 + cfg["k"])
        z = torch.randn(ut.shape, dtype=ut.dtype, device="cuda", generator=g)
        levels = p.stout_smear(lat, ut, rho, nstep)
        f = p.stout_force(lat, ut, levels, rho, z, kind=1)
        torch.cuda.synchronize()
        e0, e1, e2 = events(torch) + (torch.cuda.Event(enable_timing=True),)
        e0.record()
        for _ in range(3):
            levels = p.stout_smear(lat, ut, rho, nstep)
        e1.record()
        for _ in range(3):
            f = p.stout_force(lat, ut, levels, rho, z, kind=1)
        e2.record()
        torch.cuda.synchronize()
        t_s, t_f = e0.elapsed_time(e1) / 3, e1.elapsed_time(e2) / 3
        links = 4 * lat.V * nstep
        out[tag] = {"smear_ms": round(t_s, 3), "force_ms": round(t_f, 3),
                    "smear_tflops": round(links * STOUT_FWD_FLOPS / t_s / 1e9, 3),
                    "force_tflops": round(links * STOUT_BWD_FLOPS / t_f / 1e9, 3)}
        del f, levels, z
    out["note"] = "canonical link layout; fp32 = complex64 links (single-precision MD); flops algorithmic"
    return out


# Tree-level Symanzik gauge force: 6 plaquette + 18 rectangle staples per link = 84 complex 3x3
# products; action: per site and plane one plaquette and two rectangles = 10 products + 3 traces.
GAUGE_FORCE_FLOPS = 84 * 216
GAUGE_ACTION_FLOPS = 6 * (10 * 216 + 3 * 36)


def time_gauge(torch, p):
    cfg = S.CONFIGS["force_48x48x48x48"]
    dims = cfg["dims"]
    lat = p.Lattice(dims)
    u64 = torch.from_numpy(links_cached(dims, cfg["links"], 1000 + cfg["k"])).cuda()
    beta = 5.6
    out = {"lattice": "48^4"}
    for tag, ut in (("fp64", u64), ("fp32", p.complex_convert(u64, torch.complex64))):
        f = p.gauge_force(lat, ut, beta, kind=0)
        torch.cuda.synchronize()
        e0, e1 = events(torch)
        e0.record()
        for _ in range(3):
            f = p.gauge_force(lat, ut, beta, kind=0)
        e1.record()
        torch.cuda.synchronize()
        t_f = e0.elapsed_time(e1) / 3
        out[tag] = {"force_ms": round(t_f, 3), "force_tflops": round(4 * lat.V * GAUGE_FORCE_FLOPS / t_f / 1e9, 3)}
        del f
    p.gauge_action(lat, u64, beta)
    res = torch.empty(3, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    e0, e1 = events(torch)
    e0.record()
    for _ in range(3):
        p.lib().stg_gauge_action(lat.handle, beta, u64.data_ptr(), res.data_ptr(),
                                 torch.cuda.current_stream().cuda_stream)
    e1.record()
    torch.cuda.synchronize()
    t_a = e0.elapsed_time(e1) / 3
    out["fp64"].update({"action_ms": round(t_a, 3), "action_tflops": round(lat.V * GAUGE_ACTION_FLOPS / t_a / 1e9, 3)})
    out["note"] = "tree-level Symanzik, canonical link layout; fp32 = complex64 links (single-precision MD)"
    return out


RHMC_ACTION = dict(beta=5.6, mass=0.3, tol=1e-10, md_tol=1e-7, inner="f32", precision="f32",
                   stout_rho=0.15, stout_steps=2)


def mean_plaquette(p, lat, u):
    """Average Re tr P / 3 over the 6 V plaquettes of the links."""
    return p.gauge_action(lat, u, 1.0)["plaquette_sum"] / (18.0 * lat.V)


def thermalised_start(torch, p, tab, ntraj=40, nfree=20, small=(8, 8, 8, 8), reps=4):
    """A near-equilibrium 32^4 configuration: RHMC trajectories of the benchmark's action (tau = 0.5,
    8 Omelyan steps) on a small lattice, starting from smoothed random links (10 stout steps of
    0.1); the first nfree trajectories are kept whatever their dH (molecular dynamics with momentum
    refresh), the others pass the Metropolis test.  The small lattice's links are then repeated
    `reps` times along every direction (links are periodic; the staggered and boundary signs come
    from the coordinates)."""
    t0 = time.perf_counter()
    lat = p.Lattice(small)
    u = p.stout_smear(lat, torch.from_numpy(links_cached(small, "expih", 1002)).cuda(), 0.1, 10)[-1].contiguous()
    plaq0 = mean_plaquette(p, lat, u)
    act = p.md.Action(lat, **RHMC_ACTION)
    gen = torch.Generator(device="cuda").manual_seed(5002)
    uni = np.random.default_rng(5002).uniform(size=ntraj)
    dhs, acc = [], 0
    for k in range(ntraj):
        eta = torch.from_numpy(S.gaussian_field(small, 6000 + k)).cuda()
        act.pseudofermions = [p.md.pseudofermion_heatbath(act, u, eta, tab["heatbath"], tab["action"])]
        xi = torch.randn((4, lat.V, 8), dtype=torch.float64, device="cuda", generator=gen)
        res = p.md.trajectory(act, u, xi, 0.5, 8, uniform=0.0 if k < nfree else float(uni[k]))
        if not np.isfinite(res["dH"]):
            raise RuntimeError(f"thermalisation trajectory {k}: dH = {res['dH']}")
        u = res["links"]
        if k >= nfree:
            dhs.append(res["dH"])
            acc += bool(res["accepted"])
    torch.cuda.synchronize()
    info = {"lattice": "x".join(map(str, small)), "trajectories": ntraj, "unconditional": nfree,
            "acceptance": round(acc / max(1, ntraj - nfree), 3),
            "mean_abs_dH": round(float(np.mean(np.abs(dhs))), 4) if dhs else None,
            "plaquette_start": round(plaq0, 5), "plaquette_end": round(mean_plaquette(p, lat, u), 5),
            "s": round(time.perf_counter() - t0, 2)}
    return tile_links(u, small, reps), info


def tile_links(u, dims, reps):
    """Links [4, V, 3, 3] (site x + Lx (y + Ly (z + Lz t))) of a lattice dims = (Lx, Ly, Lz, Lt)
    repeated `reps` times along every direction: the links of the (reps Lx, ..., reps Lt) lattice."""
    big = u.reshape(4, dims[3], dims[2], dims[1], dims[0], 3, 3).repeat(1, reps, reps, reps, reps, 1, 1)
    return big.reshape(4, -1, 3, 3).contiguous()


def time_rhmc(torch, p):
    """One RHMC trajectory on 32^4 (Sec. 2-3): pseudofermion heatbath, Omelyan MD (tau = 0.5, 8 steps,
    17 force evaluations) with the gauge force, 2-step stout smearing and its chain rule and the
    fermion force in single precision (mixed solves), then the FP64 Hamiltonian and the Metropolis
    test; stored 10-pole Remez approximations of x^(1/8), x^(-1/4) for m = 0.3.  The start is an
    8^4 configuration thermalised by the same RHMC and repeated 4 times along every direction."""
    from paper_1801_01473_gb300.rational import load_table
    dims = (32, 32, 32, 32)
    lat = p.Lattice(dims)
    tab = load_table()
    u, therm = thermalised_start(torch, p, tab)
    act = p.md.Action(lat, **RHMC_ACTION)
    eta = torch.from_numpy(S.gaussian_field(dims, 2002)).cuda()
    g = torch.Generator(device="cuda").manual_seed(4002)
    xi = torch.randn((4, lat.V, 8), dtype=torch.float64, device="cuda", generator=g)

    def timed(fn):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = fn()
        torch.cuda.synchronize()
        return r, time.perf_counter() - t0

    p.md.pseudofermion_heatbath(act, u, eta, tab["heatbath"], tab["action"])  # warm-up: tuned launch shapes
    pf, t_hb = timed(lambda: p.md.pseudofermion_heatbath(act, u, eta, tab["heatbath"], tab["action"]))
    act.pseudofermions = [pf]
    mom = p.md_momenta(lat, xi)

    def median3(fn):
        fn()  # warm-up: first-call launch-shape tuning and companion gauges are not timed
        return sorted(timed(fn)[1] for _ in range(3))[1]

    t_h = median3(lambda: p.md.hamiltonian(act, u, mom))
    t_f = median3(lambda: act.apply_force(u.clone(), mom.clone(), 0.01))
    res, t_traj = timed(lambda: p.md.trajectory(act, u, xi, 0.5, 8, uniform=0.5))
    return {"lattice": "32^4", "mass": 0.3, "stout": "2 x 0.15", "integrator": "omelyan, tau 0.5, 8 steps",
            "start": "8^4 RHMC-thermalised links repeated 4 times along every direction",
            "thermalisation": therm, "plaquette": round(mean_plaquette(p, lat, u), 5),
            "forces": "fp32 (gauge, stout chain), mixed solves to 1e-7; FP64 Hamiltonian, solves to 1e-10",
            "poles": len(pf.shifts),
            "trajectory_s": round(t_traj, 3), "heatbath_ms": round(1e3 * t_hb, 1),
            "force_eval_ms": round(1e3 * t_f, 1), "hamiltonian_ms": round(1e3 * t_h, 1),
            "dH": round(res["dH"], 6), "dH_per_link": round(res["dH"] / (4 * lat.V), 6),
            "accepted": bool(res["accepted"]),
            "timing": "heatbath and trajectory: one call each after a warm-up heatbath; force evaluation and "
                      "Hamiltonian: median of 3 calls after one untimed call",
            "note": "energy conservation at O(eps^2) and the acceptance logic are tested at 4^4 and 8^4"}


def run_gpu(args):
    import torch
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    import paper_1801_01473_gb300 as p

    cfg = S.CONFIGS["bandwidth_32x32x32x32"]
    dims = cfg["dims"]
    lat = p.Lattice(dims)
    u = links_cached(dims, cfg["links"], 1000 + cfg["k"])
    ut = torch.from_numpy(u).cuda()
    gauges = [p.Gauge(lat, ut, "f32", 12), p.Gauge(lat, ut, "f32", 12)]
    del ut
    B = args.batch
    gen = torch.Generator(device="cuda").manual_seed(2000 + cfg["k"] + rank)
    src = torch.randn((B, 6 * lat.Vh), dtype=torch.float32, device="cuda", generator=gen)
    dst = torch.empty_like(src)
    alg = bytes_per_site("f32", 12) * lat.Vh

    def step():
        for j in range(B):
            p.dslash_eo_(gauges[j & 1], dst[j], src[j])

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    clk = ClockSampler(local)
    clk.start()
    time.sleep(0.3)
    e0, e1 = events(torch)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(args.steps):
        step()
    e1.record()
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    clocks = clk.stop()
    t = max_over_ranks(e0.elapsed_time(e1) * 1e-3)
    launches = args.steps * B
    value = replica_throughput(alg * launches, t, ws)
    per_launch = t / launches
    peak, peak_kind = measured_peaks()
    achieved = alg / per_launch / 1e9

    # end to end through the public API with host tensors: pinned host fields streamed through
    # stg_dslash_host (host->device copy, pack, D_eo, unpack, device->host copy, pipelined on three
    # streams), every copy inside the timed region
    n_e2e = max(8, min(64, B))
    one = torch.from_numpy(S.gaussian_field(dims, 2000 + cfg["k"]))
    e2e_rates = {}
    for dt in (torch.complex64, torch.complex128):
        host_in = torch.empty((n_e2e,) + tuple(one.shape), dtype=dt, pin_memory=True)
        host_in.copy_(one.to(dt).unsqueeze(0).expand_as(host_in))
        host_out = torch.empty_like(host_in, pin_memory=True)
        p.dslash_host(gauges[0], 0, host_in[:4], host_out[:4])  # warm-up: tuned launch shape, staging
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for j in range(2):
            p.dslash_host(gauges[j], 0, host_in, host_out)
        e2e_rates[dt] = (time.perf_counter() - t0) / (2 * n_e2e)
        del host_in, host_out
    e2e_t = e2e_rates[torch.complex64]
    # one e2e step = one dslash_host call on n_e2e complex64 fields: every field is copied host ->
    # device and its result device -> host inside the timed region
    e2e = {"value": round(ws * alg / e2e_t / 1e9, 2), "unit": UNIT,
           "h2d_bytes_per_step": int(one.numel() * 8 * n_e2e), "d2h_bytes_per_step": int(one.numel() * 8 * n_e2e),
           "steps": 2, "fields_per_step": n_e2e,
           "note": f"2 steps, each one call of dslash_host on {n_e2e} pinned host complex64 fields (copy in, pack, "
                   "D_eo, unpack, copy out; three-stage pipeline)",
           "complex128_host_fields": round(ws * alg / e2e_rates[torch.complex128] / 1e9, 2)}
    del gauges, src, dst

    line = {"metric": METRIC, "value": round(value, 2), "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(1e3 * t / args.steps, 4), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": workload_config(B, ws),
            "pct_of_hbm_peak": round(100 * achieved / peak, 2),
            "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                         "frac": round(achieved / peak, 4), "peak_kind": peak_kind,
                         "traffic": profile_traffic("deo_32x32x32x32_f32r12.md"),
                         "kernel": "k_dslash<LinkF32R12,1,0,128,0>"},
            "gpu_launches": launches, "clocks": clocks, "e2e": e2e}
    if rank == 0 and not args.no_extras:
        extras = [
            ("sweep", lambda: time_deo_sweep(torch, p, (16, 16, 16, 16), peak) + time_deo_sweep(
                torch, p, (32, 32, 32, 32), peak, doe=(("f64", 18), ("f32", 12), ("bf16", 12)))),
            ("mscg", lambda: time_mscg(torch, p, peak)),
            ("batched", lambda: time_batched(torch, p, peak)),
            ("force", lambda: time_force(torch, p, peak)),
            ("slab", lambda: time_slab(torch, p, peak)),
            ("stout", lambda: time_stout(torch, p)),
            ("gauge", lambda: time_gauge(torch, p)),
            ("rhmc", lambda: time_rhmc(torch, p)),
            ("cpu_baseline", cpu_baseline),
        ]
        for name, fn in extras:
            # a failing side measurement is reported in its own key (and on stderr) instead of
            # costing the headline line; the headline above has already been measured
            try:
                line[name] = fn()
            except Exception as e:  # noqa: BLE001
                print(f"bench: {name} failed: {e!r}", file=sys.stderr, flush=True)
                line[name] = {"error": repr(e)}
    if ws > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def run_case(name):
    """One small workload for a profiler to capture (no timing, no JSON line): `deo32_<storage>`
    four D_eo launches at 32^4 on that link storage (e.g. deo32_bf16r12); `deo32x<n>_<storage>` four
    D_oe launches on n right-hand sides sharing each link load (e.g. deo32x4_f32r12); `batched` two
    batched uneven solves (the time_batched workload); `mscg` runs two mixed
    FP32-inner solves of the 32^4 msCG workload; `force32` three double-single D_eo applications and
    one 4-shift fermion force at 32^4; `stout24` one stout step and its chain rule at 24^4;
    `gauge24` the gauge force and action at 24^4; `fp32links24` the single-precision gauge force,
    stout step and chain rule at 24^4; `rhmc_force32` one MD force evaluation of the 32^4 RHMC
    trajectory (inside the NVTX range "force_eval")."""
    import torch
    import paper_1801_01473_gb300 as p
    if name.startswith("deo32x"):
        # deo32x<n>_<storage>: four D_oe launches at 32^4 on n right-hand sides sharing each link load
        nrhs, kind = name[len("deo32x"):].split("_", 1)
        prec, recon = kind[:-3], int(kind[-2:])
        dims = (32, 32, 32, 32)
        lat = p.Lattice(dims)
        g = p.Gauge(lat, torch.from_numpy(links_cached(dims, "expih", 1002)).cuda(), prec, recon)
        gen = torch.Generator(device="cuda").manual_seed(2002)
        f = g.new_field()
        src = torch.randn((int(nrhs),) + tuple(f.shape), dtype=f.dtype, device="cuda", generator=gen)
        dst = torch.empty_like(src)
        for _ in range(4):
            p.dslash_multi_(g, 1, dst, src)
        torch.cuda.synchronize()
        print(name, float(dst.abs().max()))
        return 0
    if name.startswith("deo32_"):
        # four D_eo launches at 32^4 on one link storage (f32r12, f32r18, bf16r12, f16r12, dsr18, f64r18)
        kind = name[len("deo32_"):]
        prec, recon = kind[:-3] if kind[-3:-2] == "r" else kind[:-2], int(kind[-2:])
        dims = (32, 32, 32, 32)
        lat = p.Lattice(dims)
        g = p.Gauge(lat, torch.from_numpy(links_cached(dims, "expih", 1002)).cuda(), prec, recon)
        gen = torch.Generator(device="cuda").manual_seed(2002)
        src = torch.randn((4,) + tuple(g.new_field().shape), dtype=g.new_field().dtype, device="cuda", generator=gen)
        dst = torch.empty_like(src)
        for j in range(4):
            p.dslash_eo_(g, dst[j], src[j])
        torch.cuda.synchronize()
        print(name, float(dst.abs().max()))
        return 0
    if name == "mscg":
        cfg = S.CONFIGS["mscg_32x32x32x32"]
        dims = cfg["dims"]
        lat = p.Lattice(dims)
        ut = torch.from_numpy(links_cached(dims, cfg["links"], 1000 + cfg["k"])).cuda()
        b = torch.from_numpy(S.gaussian_field(dims, 2000 + cfg["k"])).cuda()
        g64, gi = p.Gauge(lat, ut, "f64", 18), p.Gauge(lat, ut, "f32", 12)
        for _ in range(2):
            x, st = p.mscg(g64, b, cfg["shifts"](), cfg["mass"], tol=1e-10, g_inner=gi)
        print("mscg", json.dumps({k: (list(v) if hasattr(v, "__len__") else v) for k, v in st.items()
                                  if k in ("iters", "refine_iters", "reliable_updates", "shift_iters",
                                           "refine_shift_iters", "shift_reliable_updates", "true_resid")}))
    elif name == "batched":
        # the batched uneven solve of time_batched (16^4, 24^3x8, 32^3x8, 24^4; 4 sources x 16 poles), twice
        cfg = S.CONFIGS["batched_uneven"]
        insts = []
        for li, dims in enumerate(cfg["dims_list"]):
            ut = torch.from_numpy(links_cached(dims, cfg["links"], 1000 + 10 * cfg["k"] + li)).cuda()
            lat = p.Lattice(dims)
            bs = [torch.from_numpy(S.gaussian_field(dims, 2000 + 10 * cfg["k"] + 4 * li + r)).cuda()
                  for r in range(cfg["nrhs"])]
            insts.append((p.Gauge(lat, ut, "f64", 18), p.Gauge(lat, ut, "f32", 12), bs))
        for _ in range(2):
            out = p.mscg_batched(insts, cfg["shifts"](), cfg["mass"], tol=cfg["tol"])
        torch.cuda.synchronize()
        print("batched", json.dumps([[(s["iters"], s["refine_iters"]) for s in sts] for _, sts in out]))
    elif name == "force32":
        dims = (32, 32, 32, 32)
        lat = p.Lattice(dims)
        ut = torch.from_numpy(links_cached(dims, "expih", 1002)).cuda()
        g64, gds = p.Gauge(lat, ut, "f64", 18), p.Gauge(lat, ut, "ds", 18)
        x = p.pack(lat, torch.from_numpy(S.gaussian_field(dims, 2002)).cuda(), "ds")
        y = torch.empty_like(x)
        for _ in range(3):
            p.dslash_eo_(gds, y, x)
        gen = torch.Generator(device="cuda").manual_seed(2002)
        xs = torch.randn((4, lat.Vh, 3), dtype=torch.complex128, device="cuda", generator=gen)
        f = p.fermion_force(g64, [0.5, 0.4, 0.3, 0.2], xs)
        print("force32", float(f.abs().max()))
    elif name == "stout24":
        dims = (24, 24, 24, 24)
        lat = p.Lattice(dims)
        ut = torch.from_numpy(links_cached(dims, "expih", 1005)).cuda()
        levels = p.stout_smear(lat, ut, 0.15, 1)
        gen = torch.Generator(device="cuda").manual_seed(3005)
        z = torch.randn(ut.shape, dtype=torch.complex128, device="cuda", generator=gen)
        g = p.stout_force(lat, ut, levels, 0.15, z, kind=1)
        print("stout24", float(g.abs().max()))
    elif name == "gauge24":
        dims = (24, 24, 24, 24)
        lat = p.Lattice(dims)
        ut = torch.from_numpy(links_cached(dims, "expih", 1005)).cuda()
        f = p.gauge_force(lat, ut, 5.6, kind=0)
        print("gauge24", p.gauge_action(lat, ut, 5.6)["action"], float(f.abs().max()))
    elif name == "rhmc_force32":
        # one MD force evaluation of the 32^4 trajectory workload (gauge force, 2-step stout
        # smearing and chain rule, 10-pole mixed solve to 1e-7, fermion force) after one warm-up
        # evaluation; the second one runs inside the NVTX range "force_eval"
        from paper_1801_01473_gb300.rational import load_table
        dims = (32, 32, 32, 32)
        lat = p.Lattice(dims)
        u = p.stout_smear(lat, torch.from_numpy(links_cached(dims, "expih", 1002)).cuda(), 0.1, 10)[-1].contiguous()
        ra = load_table()["action"]
        b = torch.from_numpy(S.gaussian_field(dims, 2002)).cuda()
        act = p.md.Action(lat, beta=5.6, mass=0.3, tol=1e-10, md_tol=1e-7, inner="f32", precision="f32",
                          stout_rho=0.15, stout_steps=2,
                          pseudofermions=[p.md.Pseudofermion(b, ra.poles, ra.residues, ra.alpha0)])
        mom = torch.zeros((4, lat.V, 3, 3), dtype=torch.complex128, device="cuda")
        act.apply_force(u, mom, 0.01)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("force_eval")
        act.apply_force(u, mom, 0.01)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        print("rhmc_force32", float(mom.abs().max()))
    elif name == "fp32links24":
        dims = (24, 24, 24, 24)
        lat = p.Lattice(dims)
        u32 = p.complex_convert(torch.from_numpy(links_cached(dims, "expih", 1005)).cuda(), torch.complex64)
        f = p.gauge_force(lat, u32, 5.6, kind=0)
        levels = p.stout_smear(lat, u32, 0.15, 1)
        gen = torch.Generator(device="cuda").manual_seed(3005)
        z = torch.randn(u32.shape, dtype=torch.complex64, device="cuda", generator=gen)
        g = p.stout_force(lat, u32, levels, 0.15, z, kind=1)
        print("fp32links24", float(f.abs().max()), float(g.abs().max()))
    else:
        raise SystemExit(f"unknown case {name}")
    torch.cuda.synchronize()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--batch", type=int, default=256)
    ap.add_argument("--impl", default="stg", choices=["stg", "reference"])
    ap.add_argument("--no-extras", action="store_true")
    ap.add_argument("--case", default=None,
                    choices=["mscg", "force32", "stout24", "gauge24", "fp32links24", "rhmc_force32", "deo32_f32r12",
                             "deo32_f32r18", "deo32_bf16r12", "deo32_f16r12", "deo32_dsr18", "deo32_f64r18",
                             "deo32x2_f32r12", "deo32x4_f32r12", "deo32x8_f32r12", "batched"],
                    help="run one small workload for a profiler instead of the benchmark")
    args = ap.parse_args()
    if args.case:
        return run_case(args.case)
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
