"""stg_normal_op_noalloc: the shifted normal operator for callers that cannot
allocate device memory when they call it (a framework that owns all device
memory through its own pool, or a loop that must not call cudaMalloc/cudaFree
because they can synchronize the device or fail once memory is partitioned).
It keeps its scratch in a fixed 32 MiB device array instead of taking a
temporary from the caller.

Called here through the C ABI (ctypes on libstg.so), twice in a row with
different inputs, and compared with stg_normal_op, the entry point that takes
a caller temporary (output fields within the FP64 / double-single (1e-12) and
FP32 (2e-6) relative tolerances of the operator tests, and the fused Re<in, out>
reduction as well), and with the FP64 oracle's normal operator.  F64, DS and
F32 gauges are covered, and an F32 gauge with a U(1) phase field.  Oversized
lattices and overlapping in/out fields are rejected before any launch.

This file is named to be collected last, so a run that stops at the first
failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

import oracle
import synthetic as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "ds": 1e-12, "f32": 2e-6}


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


@pytest.mark.parametrize("prec,recon,u1", [("f64", 18, False), ("ds", 12, False), ("f32", 12, False),
                                           ("f32", 12, True)])
def test_noalloc_matches_normal_op_twice(prec, recon, u1):
    import paper_1801_01473_gb300 as stg
    from paper_1801_01473_gb300.lib import lib

    L = lib()
    dims = (8, 6, 4, 10)
    lat = stg.Lattice(dims)
    u = S.gauge_links(dims, "haar", 901)
    theta = np.random.default_rng(904).uniform(-np.pi, np.pi, (4, lat.V)) if u1 else None
    g = stg.Gauge(lat, torch.from_numpy(u).cuda(), prec, recon,
                  theta=torch.from_numpy(theta).cuda() if u1 else None)
    u_oracle = oracle.u1_links(u, theta) if u1 else u
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call, (seed, mass, shift) in enumerate([(902, 0.1, 0.03), (903, 0.05, 0.7)]):
        psi = S.gaussian_field(dims, seed)
        x = stg.pack(lat, torch.from_numpy(psi).cuda(), g.vec_prec)
        ref, tmp, got = torch.empty_like(x), torch.empty_like(x), torch.full_like(x, float("nan"))
        pq_ref = torch.zeros(1, dtype=torch.float64, device="cuda")
        pq = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
        assert L.stg_normal_op(g.handle, mass, shift, _p(ref), _p(x), _p(tmp), _p(pq_ref), stream) == 0
        assert L.stg_normal_op_noalloc(g.handle, mass, shift, _p(got), _p(x), _p(pq), stream) == 0, \
            L.stg_last_error()
        torch.cuda.synchronize()
        err = (got - ref).abs().max().item() / ref.abs().max().item()
        assert err <= TOL[prec], (call, err)
        assert abs(pq.item() - pq_ref.item()) <= TOL[prec] * abs(pq_ref.item()), call
        # and against the FP64 oracle's normal operator (the tolerance of the operator tests)
        want = oracle.normal_op(dims, u_oracle, mass, shift, psi)
        have = stg.unpack(lat, got).cpu().numpy()
        assert np.abs(have - want).max() <= 4 * TOL[prec] * np.abs(want).max(), call
    # without the reduction
    out = torch.empty_like(x)
    assert L.stg_normal_op_noalloc(g.handle, 0.1, 0.0, _p(out), _p(x), None, stream) == 0
    assert L.stg_normal_op(g.handle, 0.1, 0.0, _p(ref), _p(x), _p(tmp), None, stream) == 0
    torch.cuda.synchronize()
    assert (out - ref).abs().max().item() <= TOL[prec] * ref.abs().max().item()


def test_noalloc_rejects_lattice_beyond_limit():
    import paper_1801_01473_gb300 as stg
    from paper_1801_01473_gb300.lib import STG_ERR_ARG, lib

    L = lib()
    dims = (96, 96, 96, 4)  # 1769472 sites per parity: above both limits
    lat = stg.Lattice(dims)
    links = torch.zeros((4, lat.V, 3, 3), dtype=torch.complex128, device="cuda")
    links[:, :, 0, 0] = links[:, :, 1, 1] = links[:, :, 2, 2] = 1.0
    g = stg.Gauge(lat, links, "f32", 12)
    del links
    x = torch.zeros(6 * lat.Vh, dtype=torch.float32, device="cuda")
    out = torch.zeros_like(x)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert L.stg_normal_op_noalloc(g.handle, 0.1, 0.0, _p(out), _p(x), None, stream) == STG_ERR_ARG
    assert b"32 MiB" in L.stg_last_error()


def test_noalloc_rejects_overlapping_fields():
    import paper_1801_01473_gb300 as stg
    from paper_1801_01473_gb300.lib import STG_ERR_ARG, lib

    L = lib()
    dims = (4, 4, 4, 4)
    lat = stg.Lattice(dims)
    g = stg.Gauge(lat, torch.from_numpy(S.gauge_links(dims, "haar", 905)).cuda(), "f64", 18)
    buf = torch.zeros(2 * 6 * lat.Vh, dtype=torch.float64, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    base = buf.data_ptr()
    for shift_bytes in (0, 16, 48 * lat.Vh - 16):  # same field, and partial overlaps either way
        a, b = ctypes.c_void_p(base), ctypes.c_void_p(base + shift_bytes)
        assert L.stg_normal_op_noalloc(g.handle, 0.1, 0.0, b, a, None, stream) == STG_ERR_ARG
        assert L.stg_normal_op_noalloc(g.handle, 0.1, 0.0, a, b, None, stream) == STG_ERR_ARG
        assert b"overlap" in L.stg_last_error()
    # adjacent fields do not overlap
    a, b = ctypes.c_void_p(base), ctypes.c_void_p(base + 48 * lat.Vh)
    assert L.stg_normal_op_noalloc(g.handle, 0.1, 0.0, b, a, None, stream) == 0
    torch.cuda.synchronize()
