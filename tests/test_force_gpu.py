"""Parity of the CUDA fermion force with the FP64 oracle, and checks of the
autograd path against finite differences.

* force kernel vs the oracle's force on the same solutions: 1e-12 relative;
* torch.autograd: PseudofermionAction's gradient (W^dag per link) against
  directional central differences of S and torch.autograd.gradcheck;
* 48^4 (the differentiation workload): tr(X F) against central finite
  differences (eps = 1e-5) of S along exp(eps X) U on 32 random links, 1e-6
  relative.  S(+eps) - S(-eps) is evaluated through the resolvent identity
  sum_i r_i x_i(+eps)^dag [A_i(-eps) - A_i(+eps)] x_i(-eps), which equals the
  difference of the two actions exactly but does not cancel catastrophically.
"""
import numpy as np
import pytest

import oracle
import synthetic as S
from tests import latutil as lu

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def stg():
    import paper_1801_01473_gb300 as p
    return p


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (6, 4, 2, 8), (8, 8, 4, 6)])
@pytest.mark.parametrize("recon", [18, 12])
@pytest.mark.parametrize("kind", [0, 1])
def test_force_matches_oracle(dims, recon, kind):
    p = stg()
    u = S.gauge_links(dims, "haar", 61)
    b = S.gaussian_field(dims, 62)
    shifts = [1e-3, 0.02, 0.3, 1.5]
    res = [0.7, 0.4, 0.25, 0.1]
    sol = oracle.mscg(dims, u, 0.1, shifts, b, tol=1e-12)
    ref = oracle.force(dims, u, res, sol["x"], kind=kind)
    g = p.Gauge(p.Lattice(dims), torch.from_numpy(u).cuda(), "f64", recon)
    got = p.fermion_force(g, res, torch.from_numpy(sol["x"]).cuda(), kind=kind).cpu().numpy()
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()


def _action(p, lat, links, b, shifts, res, mass):
    return p.pseudofermion_action(links, b, lat, shifts, res, mass)


def test_autograd_directional_derivative():
    p = stg()
    dims = (4, 4, 4, 4)
    lat = p.Lattice(dims)
    u = torch.from_numpy(S.gauge_links(dims, "haar", 71)).cuda().requires_grad_(True)
    b = torch.from_numpy(S.gaussian_field(dims, 72)).cuda()
    shifts, res, mass = [1e-3, 0.05, 0.5], [0.6, 0.3, 0.2], 0.1
    s = _action(p, lat, u, b, shifts, res, mass)
    (grad,) = torch.autograd.grad(s, u)
    g = np.random.default_rng(5)
    d = torch.from_numpy(g.standard_normal(u.shape) + 1j * g.standard_normal(u.shape)).cuda()
    eps = 1e-6
    with torch.no_grad():
        sp = _action(p, lat, u + eps * d, b, shifts, res, mass).item()
        sm = _action(p, lat, u - eps * d, b, shifts, res, mass).item()
    fd = (sp - sm) / (2 * eps)
    an = torch.sum(grad.real * d.real + grad.imag * d.imag).item()
    assert abs(fd - an) <= 1e-5 * abs(an), (fd, an)


def test_autograd_gradcheck_4x4x4x4():
    """torch.autograd.gradcheck of the pseudofermion action on a 4^4 FP64 lattice (complex links,
    real loss: the W^dag gradient in torch's convention)."""
    p = stg()
    dims = (4, 4, 4, 4)
    lat = p.Lattice(dims)
    u = torch.from_numpy(S.gauge_links(dims, "haar", 81)).cuda().requires_grad_(True)
    b = torch.from_numpy(S.gaussian_field(dims, 82)).cuda()
    fn = lambda links: _action(p, lat, links, b, [0.01, 0.2], [0.5, 0.5], 0.2)
    assert torch.autograd.gradcheck(fn, (u,), eps=1e-6, atol=1e-6, rtol=1e-4, fast_mode=True)


@pytest.mark.slow
def test_force_48x48x48x48_finite_differences():
    p = stg()
    cfg = S.CONFIGS["force_48x48x48x48"]
    dims, mass, tol = cfg["dims"], cfg["mass"], cfg["tol"]
    shifts = cfg["shifts"]()
    res = S.positive_residues(3000 + cfg["k"], len(shifts))
    lat = p.Lattice(dims)
    ut = torch.from_numpy(S.gauge_links(dims, cfg["links"], 1000 + cfg["k"])).cuda()
    b = torch.from_numpy(S.gaussian_field(dims, 2000 + cfg["k"])).cuda()
    g64 = p.Gauge(lat, ut, "f64", 18)
    g32 = p.Gauge(lat, ut, "f32", 12)
    x, st = p.mscg(g64, b, shifts, mass, tol=tol, g_inner=g32)
    f = p.fermion_force(g64, res, x, kind=0)
    del g32
    rng = np.random.default_rng(9)
    v = lat.V
    tmp = torch.empty(6 * lat.Vh, dtype=torch.float64, device="cuda")
    eps = 1e-5
    worst = 0.0
    for trial in range(32):
        mu, z = int(rng.integers(4)), int(rng.integers(v))
        xa = lu.random_su3_algebra(rng)
        u0 = ut[mu, z].clone()
        xs = {}
        gs = {}
        for sgn in (+1, -1):
            ut[mu, z] = torch.from_numpy(lu.expm_su3(sgn * eps * xa)).cuda() @ u0
            gs[sgn] = p.Gauge(lat, ut, "f64", 18)
            gi = p.Gauge(lat, ut, "f32", 12)
            xs[sgn], _ = p.mscg(gs[sgn], b, shifts, mass, tol=tol, g_inner=gi)
            del gi
        ut[mu, z] = u0
        ds = 0.0
        for i, s in enumerate(shifts):
            xm = p.pack(lat, xs[-1][i], "f64")
            am = torch.empty_like(xm)
            ap = torch.empty_like(xm)
            p.normal_op_(gs[-1], mass, s, am, xm, tmp)
            p.normal_op_(gs[+1], mass, s, ap, xm, tmp)
            dv = p.unpack(lat, am) - p.unpack(lat, ap)
            ds += res[i] * torch.vdot(xs[+1][i].reshape(-1), dv.reshape(-1)).real.item()
        fd = ds / (2 * eps)
        an = np.trace(xa @ f[mu, z].cpu().numpy()).real
        err = abs(fd - an) / abs(an)
        worst = max(worst, err)
        assert err <= 1e-6, (trial, mu, z, fd, an)
        del gs
    print("48^4 force vs FD: worst relative error %.2e over 32 links" % worst)


@pytest.mark.parametrize("recon", [18, 12])
@pytest.mark.parametrize("kind", [0, 1])
def test_double_single_gather_matches_fp64_gather(recon, kind, monkeypatch):
    """The default double-single accumulation of W (FP32 pipes) against the FP64 accumulation
    (STG_FORCE_FP64=1) on the same solutions: 1e-13 relative."""
    import paper_1801_01473_gb300 as p
    dims = (6, 4, 4, 8)
    u = S.gauge_links(dims, "expih", 221)
    lat = p.Lattice(dims)
    g = p.Gauge(lat, torch.from_numpy(u).cuda(), "f64", recon)
    gen = torch.Generator(device="cuda").manual_seed(222)
    x = torch.randn((5, lat.Vh, 3), dtype=torch.complex128, device="cuda", generator=gen)
    res = [0.9, 0.5, 0.3, 0.2, 0.1]
    ds = p.fermion_force(g, res, x, kind=kind)
    monkeypatch.setenv("STG_FORCE_FP64", "1")
    f64 = p.fermion_force(g, res, x, kind=kind)
    assert float((ds - f64).abs().max()) <= 1e-13 * float(f64.abs().max())


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (6, 4, 2, 8), (8, 8, 4, 6)])
@pytest.mark.parametrize("kind", [0, 1])
@pytest.mark.parametrize("phases", [False, True])
def test_single_precision_force_matches_oracle(dims, kind, phases):
    """prec="f32" (FP32 12-real links, FP32 fields and gather, complex64 out) against the oracle's
    FP64 force on the same solutions: 5e-6 relative (FP32 rounding of links, fields and sums)."""
    p = stg()
    u = S.gauge_links(dims, "haar", 63)
    b = S.gaussian_field(dims, 64)
    shifts = [1e-3, 0.02, 0.3, 1.5]
    res = [0.7, 0.4, 0.25, 0.1]
    lat = p.Lattice(dims)
    theta = np.random.default_rng(65).uniform(-np.pi, np.pi, (4, lat.V)) if phases else None
    if phases:
        sol = oracle.mscg(dims, oracle.u1_links(u, theta), 0.1, shifts, b, tol=1e-12)
        ref = oracle.force_u1(dims, u, theta, res, sol["x"], kind=kind)
    else:
        sol = oracle.mscg(dims, u, 0.1, shifts, b, tol=1e-12)
        ref = oracle.force(dims, u, res, sol["x"], kind=kind)
    g = p.Gauge(lat, torch.from_numpy(u).cuda(), "f64", 18,
                theta=torch.from_numpy(theta).cuda() if phases else None)
    got = p.fermion_force(g, res, torch.from_numpy(sol["x"]).cuda(), kind=kind, prec="f32")
    assert got.dtype == torch.complex64
    got = got.cpu().numpy()
    assert np.abs(got - ref).max() <= 5e-6 * np.abs(ref).max()


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (6, 4, 2, 8), (16, 8, 8, 12)])
@pytest.mark.parametrize("nshift", [0, 1, 5, 32])
def test_pseudofermion_action_matches_oracle(dims, nshift):
    """stg_pseudofermion_action: S = alpha0 |b|^2 + sum_i r_i Re(b^dag x_i) against the oracle's
    definition on arbitrary fields (the formula holds for any x_i), 1e-13 relative; two calls give
    bitwise the same value (fixed-order reduction)."""
    p = stg()
    lat = p.Lattice(dims)
    b = S.gaussian_field(dims, 90)
    rng = np.random.default_rng(91)
    x = (rng.standard_normal((nshift, lat.Vh, 3)) + 1j * rng.standard_normal((nshift, lat.Vh, 3))) / np.sqrt(2)
    res = S.positive_residues(92, nshift) if nshift else []
    alpha0 = 0.37
    want = oracle.action(res, b, x, alpha0=alpha0)
    xd = torch.from_numpy(x).cuda()
    got = p.pseudofermion_action_value(lat, torch.from_numpy(b).cuda(), xd, res, alpha0)
    assert abs(got - want) <= 1e-13 * abs(want), (got, want)
    assert got == p.pseudofermion_action_value(lat, torch.from_numpy(b).cuda(), xd, res, alpha0)


def test_pseudofermion_action_rejects_bad_arguments():
    p = stg()
    lat = p.Lattice((4, 4, 4, 4))
    b = torch.zeros((lat.Vh, 3), dtype=torch.complex128, device="cuda")
    x = torch.zeros((33, lat.Vh, 3), dtype=torch.complex128, device="cuda")
    with pytest.raises(p.StgError):
        p.pseudofermion_action_value(lat, b, x, [1.0] * 33)
