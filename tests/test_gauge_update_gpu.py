"""In-place link replacement (stg_gauge_update): a gauge created from links u1 and updated to u2
behaves bitwise like a gauge created from u2 -- for D in every storage variant, with and without a
U(1) phase field, and for the solves and forces whose double-single and FP32 companions were
created from u1 before the update."""
import numpy as np
import pytest

import synthetic as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

DIMS = (4, 6, 4, 8)


@pytest.fixture(scope="module")
def p():
    import paper_1801_01473_gb300 as p
    return p


def _links(seed):
    return torch.from_numpy(S.gauge_links(DIMS, "expih", seed)).cuda()


def _theta(seed):
    lat_v = int(np.prod(DIMS))
    return torch.from_numpy(np.random.default_rng(seed).uniform(-np.pi, np.pi, (4, lat_v))).cuda()


@pytest.mark.parametrize("prec,recon", [("f64", 18), ("f64", 12), ("ds", 18), ("f32", 12), ("f32", 18), ("bf16", 12)])
@pytest.mark.parametrize("phases", [False, True])
def test_dslash_after_update_bitwise(p, prec, recon, phases):
    lat = p.Lattice(DIMS)
    u1, u2 = _links(51), _links(52)
    th1, th2 = (_theta(53), _theta(54)) if phases else (None, None)
    g = p.Gauge(lat, u1, prec, recon, theta=th1)
    fresh = p.Gauge(lat, u2, prec, recon, theta=th2)
    g.update(u2, th2)
    psi = torch.from_numpy(S.gaussian_field(DIMS, 55)).cuda()
    assert torch.equal(p.dslash_oe(g, psi), p.dslash_oe(fresh, psi))
    assert torch.equal(p.dslash_eo(g, psi), p.dslash_eo(fresh, psi))


@pytest.mark.parametrize("inner", [("f32", 12), ("bf16", 12)])
def test_companions_refreshed(p, inner):
    """The mixed solve builds a double-single companion of the F64 gauge (and, for a 16-bit inner
    gauge, an FP32 one); after an update the solve and the force equal those on fresh gauges."""
    lat = p.Lattice(DIMS)
    u1, u2 = _links(61), _links(62)
    b = torch.from_numpy(S.gaussian_field(DIMS, 63)).cuda()
    shifts = [0.0, 0.1, 1.0]
    g64, gi = p.Gauge(lat, u1, "f64", 18), p.Gauge(lat, u1, *inner)
    p.mscg(g64, b, shifts, 0.1, tol=1e-10, g_inner=gi)              # companions from u1
    p.fermion_force(g64, [0.3, 0.2, 0.1], torch.zeros((3, lat.Vh, 3), dtype=torch.complex128, device="cuda"))
    g64.update(u2)
    gi.update(u2)
    f64, fi = p.Gauge(lat, u2, "f64", 18), p.Gauge(lat, u2, *inner)
    x_upd, st_upd = p.mscg(g64, b, shifts, 0.1, tol=1e-10, g_inner=gi)
    x_new, st_new = p.mscg(f64, b, shifts, 0.1, tol=1e-10, g_inner=fi)
    assert st_upd["iters"] == st_new["iters"] and torch.equal(x_upd, x_new)
    assert torch.equal(p.fermion_force(g64, [0.3, 0.2, 0.1], x_upd), p.fermion_force(f64, [0.3, 0.2, 0.1], x_new))


def test_update_argument_errors(p):
    lat = p.Lattice(DIMS)
    u = _links(71)
    g = p.Gauge(lat, u, "f32", 12)
    gp = p.Gauge(lat, u, "f32", 12, theta=_theta(72))
    with pytest.raises(p.StgError):
        g.update(u, _theta(73))   # phases on a gauge created without them
    with pytest.raises(p.StgError):
        gp.update(u)              # phases missing
