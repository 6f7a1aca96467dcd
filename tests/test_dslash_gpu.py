"""Parity of the CUDA D_eo / D_oe / normal operator with the FP64 oracle.

Tolerances (relative max-norm error over the output vector):
  F64 links, 18 or 12 real    1e-12  (spec bar for FP64 paths)
  DS (FP32 pairs), 18 or 12   1e-12  (48-bit significand; measured well below this)
  F32 links                   2e-6   (FP32 rounding of links, vectors and 8-term sums)
  F16 links                   4e-3   (11-bit mantissa of the stored link rows)
  BF16 links                  3e-2   (8-bit mantissa of the stored link rows)
"""
import numpy as np
import pytest

import oracle
import synthetic as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {("f64", 18): 1e-12, ("f64", 12): 1e-12, ("ds", 18): 1e-12, ("ds", 12): 1e-12, ("f32", 18): 2e-6,
       ("f32", 12): 2e-6, ("f16", 12): 4e-3, ("bf16", 12): 3e-2}
VARIANTS = list(TOL)
# several tiles of 128 sites plus ragged tails; odd-shaped extents
LATTICES = [(4, 4, 4, 4), (6, 4, 2, 8), (2, 6, 4, 10), (8, 8, 8, 8), (12, 10, 6, 4)]


def stg():
    import paper_1801_01473_gb300 as p
    return p


def rel(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return np.abs(a - b).max() / np.abs(b).max()


_links_cache = {}


def links_for(dims, kind="haar", seed=101):
    key = (dims, kind, seed)
    if key not in _links_cache:
        _links_cache[key] = S.gauge_links(dims, kind, seed)
    return _links_cache[key]


@pytest.mark.parametrize("dims", LATTICES)
@pytest.mark.parametrize("variant", VARIANTS)
def test_dslash_matches_oracle(dims, variant):
    p = stg()
    prec, recon = variant
    u = links_for(dims)
    lat = p.Lattice(dims)
    g = p.Gauge(lat, torch.from_numpy(u).cuda(), prec, recon)
    for out_par in (0, 1):
        psi = S.gaussian_field(dims, 200 + out_par)
        ref = oracle.dslash(dims, u, out_par, psi)
        fn = p.dslash_eo if out_par == 0 else p.dslash_oe
        got = fn(g, torch.from_numpy(psi).cuda()).cpu().numpy()
        assert rel(got, ref) <= TOL[variant], (dims, variant, out_par, rel(got, ref))


@pytest.mark.parametrize("variant", VARIANTS)
def test_normal_op_and_fused_dot(variant):
    p = stg()
    prec, recon = variant
    dims, mass, shift = (6, 4, 2, 8), 0.1, 0.03
    u = links_for(dims)
    lat = p.Lattice(dims)
    g = p.Gauge(lat, torch.from_numpy(u).cuda(), prec, recon)
    psi = S.gaussian_field(dims, 301)
    ref = oracle.normal_op(dims, u, mass, shift, psi)
    x = p.pack(lat, torch.from_numpy(psi).cuda(), g.vec_prec)
    out, tmp = torch.empty_like(x), torch.empty_like(x)
    pq = torch.zeros(1, dtype=torch.float64, device="cuda")
    p.normal_op_(g, mass, shift, out, x, tmp, pq)
    got = p.unpack(lat, out).cpu().numpy()
    assert rel(got, ref) <= 4 * TOL[variant]
    pq_ref = np.vdot(psi, ref).real
    assert abs(pq.item() - pq_ref) <= 4 * TOL[variant] * abs(pq_ref)


@pytest.mark.parametrize("variant", [("f64", 18), ("ds", 12), ("f32", 12), ("bf16", 12)])
@pytest.mark.parametrize("nrhs", [1, 3, 8, 11, 45])
def test_multi_rhs_matches_single(variant, nrhs):
    """Shared link loads over nrhs right-hand sides give bitwise the single-rhs results (45 rhs:
    six groups of up to 8 in one launch; double-single splits them into 45 one-rhs groups, three
    launches of up to 16)."""
    p = stg()
    prec, recon = variant
    dims = (8, 4, 6, 4)
    lat = p.Lattice(dims)
    g = p.Gauge(lat, torch.from_numpy(links_for(dims)).cuda(), prec, recon)
    srcs = [S.gaussian_field(dims, 400 + j) for j in range(nrhs)]
    inp = torch.stack([p.pack(lat, torch.from_numpy(s).cuda(), g.vec_prec) for s in srcs])
    for out_par in (0, 1):
        out = torch.empty_like(inp)
        p.dslash_multi_(g, out_par, out, inp)
        for j in range(nrhs):
            one = torch.empty_like(inp[j])
            (p.dslash_eo_ if out_par == 0 else p.dslash_oe_)(g, one, inp[j].contiguous())
            assert torch.equal(one, out[j])


@pytest.mark.parametrize("variant", [("f32", 12), ("f32", 18), ("f16", 12), ("bf16", 12)])
@pytest.mark.parametrize("nrhs", [2, 3, 8])
@pytest.mark.parametrize("shape", ["shared", "64", "256", "ahead"])
def test_multi_rhs_launch_shapes_bitwise(variant, nrhs, shape, monkeypatch):
    """Every launch shape of the multi-rhs operator -- including the shared-link kernel, which
    stages each block's links in shared memory once for all rhs, and the one-hop-lookahead loop
    (FP32 12-real, 3-4 rhs; other cases fall back to the tuned shape) -- gives bitwise the
    single-rhs results, on a lattice whose last 64-site block is ragged (Vh = 1000)."""
    p = stg()
    prec, recon = variant
    dims = (10, 10, 4, 10)
    lat = p.Lattice(dims)
    g = p.Gauge(lat, torch.from_numpy(links_for(dims)).cuda(), prec, recon)
    inp = torch.stack([p.pack(lat, torch.from_numpy(S.gaussian_field(dims, 500 + j)).cuda(), g.vec_prec)
                       for j in range(nrhs)])
    monkeypatch.setenv("STG_DSLASH_SHAPE", "128")
    ref = []
    for out_par in (0, 1):
        for j in range(nrhs):
            one = torch.empty_like(inp[j])
            (p.dslash_eo_ if out_par == 0 else p.dslash_oe_)(g, one, inp[j].contiguous())
            ref.append(one)
    monkeypatch.setenv("STG_DSLASH_SHAPE", shape)
    k = 0
    for out_par in (0, 1):
        out = torch.empty_like(inp)
        p.dslash_multi_(g, out_par, out, inp)
        for j in range(nrhs):
            assert torch.equal(ref[k], out[j]), (out_par, j)
            k += 1
    # the fused epilogue (normal operator, Re<p,q> partials) through the same shapes
    for j in range(min(nrhs, 2)):
        x = inp[j].contiguous()
        monkeypatch.setenv("STG_DSLASH_SHAPE", "128")
        a1, pq1 = torch.empty_like(x), torch.zeros(1, dtype=torch.float64, device="cuda")
        p.normal_op_(g, 0.1, 0.01, a1, x, g.new_field(), pq1)
        monkeypatch.setenv("STG_DSLASH_SHAPE", shape)
        a2, pq2 = torch.empty_like(x), torch.zeros(1, dtype=torch.float64, device="cuda")
        p.normal_op_(g, 0.1, 0.01, a2, x, g.new_field(), pq2)
        assert torch.equal(a1, a2) and torch.equal(pq1, pq2)


def test_pack_unpack_roundtrip():
    p = stg()
    dims = (6, 4, 2, 8)
    lat = p.Lattice(dims)
    psi = torch.from_numpy(S.gaussian_field(dims, 5)).cuda()
    assert torch.equal(p.unpack(lat, p.pack(lat, psi, "f64")), psi)
    back = p.unpack(lat, p.pack(lat, psi, "f32"))
    assert torch.equal(back, psi.to(torch.complex64).to(torch.complex128))
    back = p.unpack(lat, p.pack(lat, psi, "ds"))  # hi + lo keeps 48 of the 53 significand bits
    assert ((back - psi).abs() <= 2.0 ** -47 * psi.abs()).all()


def test_full_size_32x32x32x32_sampled():
    """The benchmarked workload (32^4, exp(i 0.3 H) links, FP32 12-real and FP64 18-real):
    D_eo and D_oe over the full lattice against the oracle evaluated on every output site."""
    p = stg()
    cfg = S.CONFIGS["bandwidth_32x32x32x32"]
    dims = cfg["dims"]
    u = S.gauge_links(dims, cfg["links"], 1000 + cfg["k"])
    psi = S.gaussian_field(dims, 2000 + cfg["k"], parity_sites=True)
    refs = {0: oracle.dslash(dims, u, 0, psi), 1: oracle.dslash(dims, u, 1, psi)}
    lat = p.Lattice(dims)
    ut = torch.from_numpy(u).cuda()
    x = torch.from_numpy(psi).cuda()
    for prec, recon in [("f32", 12), ("f64", 18), ("ds", 18), ("bf16", 12)]:
        g = p.Gauge(lat, ut, prec, recon)
        for out_par, fn in ((0, p.dslash_eo), (1, p.dslash_oe)):
            got = fn(g, x).cpu().numpy()
            assert rel(got, refs[out_par]) <= TOL[(prec, recon)], (prec, recon, out_par, rel(got, refs[out_par]))
        del g


@pytest.mark.parametrize("variant", [("f64", 18), ("f32", 12), ("ds", 12), ("bf16", 12)])
@pytest.mark.parametrize("out_par", [0, 1])
def test_dslash_host_pipeline(variant, out_par):
    """stg_dslash_host streams host fields through pack / D / unpack with two staging slots per
    stage: 5 fields (slots reused), results bitwise equal to the device API and within the
    variant's tolerance of the oracle."""
    p = stg()
    prec, recon = variant
    dims = (8, 4, 6, 4)
    u = links_for(dims)
    lat = p.Lattice(dims)
    g = p.Gauge(lat, torch.from_numpy(u).cuda(), prec, recon)
    fields = np.stack([S.gaussian_field(dims, 300 + k) for k in range(5)])
    host = torch.from_numpy(fields).pin_memory()
    got = p.dslash_host(g, out_par, host)
    assert not got.is_cuda and got.shape == host.shape
    fn = p.dslash_eo if out_par == 0 else p.dslash_oe
    for k in range(5):
        dev = fn(g, torch.from_numpy(fields[k]).cuda()).cpu()
        assert torch.equal(got[k], dev), k
        assert rel(got[k].numpy(), oracle.dslash(dims, u, out_par, fields[k])) <= TOL[variant]
    empty = torch.empty((0, lat.Vh, 3), dtype=torch.complex128)
    assert p.dslash_host(g, out_par, empty).shape[0] == 0
    if prec in ("f32", "bf16"):
        # complex64 host fields: half the bytes over the host link, same FP32 arithmetic
        h32 = host.to(torch.complex64).pin_memory()
        got32 = p.dslash_host(g, out_par, h32)
        assert got32.dtype == torch.complex64
        for k in range(5):
            dev = fn(g, h32[k].to(torch.complex128).cuda()).cpu().to(torch.complex64)
            assert torch.equal(got32[k], dev), k


def test_generic_dslash_dispatch():
    """stg.dslash(gauge, out_parity, psi) is D_eo for parity 0 and D_oe for parity 1, bitwise."""
    p = stg()
    dims = (4, 4, 4, 6)
    lat = p.Lattice(dims)
    g = p.Gauge(lat, torch.from_numpy(links_for(dims)).cuda(), "f64", 18)
    psi = torch.from_numpy(S.gaussian_field(dims, 205)).cuda()
    assert torch.equal(p.dslash(g, 0, psi), p.dslash_eo(g, psi))
    assert torch.equal(p.dslash(g, 1, psi), p.dslash_oe(g, psi))
    # the C entry stg_dslash on internal-layout fields
    x = p.pack(lat, psi, "f64")
    for par, fn in ((0, p.dslash_eo_), (1, p.dslash_oe_)):
        want = fn(g, torch.empty_like(x), x)
        got = torch.empty_like(x)
        assert p.lib().stg_dslash(g.handle, par, got.data_ptr(), x.data_ptr(),
                                  torch.cuda.current_stream().cuda_stream) == 0
        torch.cuda.synchronize()
        assert torch.equal(got, want)
