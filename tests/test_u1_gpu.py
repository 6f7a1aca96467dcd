"""D, the solvers and the fermion force with a U(1) phase field theta_mu(x) on the GPU, against
the oracle on the phased links exp(i theta) U.

Tolerances as for D without phases (relative max-norm): F64 / DS 1e-12, F32 2e-6 (the angles
are stored as FP32 and turned into cos + i sin on line), F16 4e-3, BF16 3e-2.
* D_eo, D_oe for every storage variant, lattices with ragged thread-block tails;
* the imaginary-chemical-potential closed form on unit links with constant theta;
* FP64 and mixed FP32-inner multi-shift solves to 1e-10 true residual with the oracle's operator;
* the fermion force (kinds 0 and 1) vs oracle.force_u1 (1e-12).
"""
import numpy as np
import pytest
import torch

import oracle
import synthetic as S
from tests import latutil as lu

pytestmark = pytest.mark.gpu

TOL = {("f64", 18): 1e-12, ("f64", 12): 1e-12, ("ds", 18): 1e-12, ("ds", 12): 1e-12, ("f32", 18): 2e-6,
       ("f32", 12): 2e-6, ("f16", 12): 4e-3, ("bf16", 12): 3e-2}
LATTICES = [(4, 4, 4, 4), (6, 4, 2, 8), (12, 10, 6, 4)]


@pytest.fixture(scope="module")
def p():
    import paper_1801_01473_gb300 as p
    return p


def _gpu(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def rel(a, b):
    return np.abs(np.asarray(a) - b).max() / np.abs(b).max()


def _theta(dims, seed):
    return np.random.default_rng(seed).uniform(-np.pi, np.pi, (4, int(np.prod(dims))))


@pytest.mark.parametrize("dims", LATTICES)
@pytest.mark.parametrize("variant", list(TOL))
def test_dslash_with_phases(p, dims, variant):
    prec, recon = variant
    u = S.gauge_links(dims, "haar", 181)
    th = _theta(dims, 182)
    lat = p.Lattice(dims)
    g = p.Gauge(lat, _gpu(u), prec, recon, theta=_gpu(th))
    v = oracle.u1_links(u, th)
    for out_par in (0, 1):
        psi = S.gaussian_field(dims, 183 + out_par)
        fn = p.dslash_eo if out_par == 0 else p.dslash_oe
        got = fn(g, _gpu(psi)).cpu().numpy()
        assert rel(got, oracle.dslash(dims, v, out_par, psi)) <= TOL[variant], (dims, variant, out_par)


@pytest.mark.parametrize("prec,recon", [("f64", 18), ("f32", 12), ("ds", 12)])
def test_constant_phase_closed_form(p, prec, recon):
    dims = (6, 4, 4, 8)
    v = int(np.prod(dims))
    a = np.array([0.3, -0.7, 0.2, 0.45])
    th = np.broadcast_to(a[:, None], (4, v)).copy()
    unit = np.broadcast_to(np.eye(3, dtype=np.complex128), (4, v, 3, 3)).copy()
    lat = p.Lattice(dims)
    g = p.Gauge(lat, _gpu(unit), prec, recon, theta=_gpu(th))
    n = (1, 2, 0, 3)
    psi = lu.plane_wave_even(dims, n, [1.0, 0.5j, -0.25])
    lam = 0.01 + 0.02 + np.sum(np.sin(lu.momentum(dims, n) + a) ** 2)
    got = p.normal_op(g, 0.1, 0.02, _gpu(psi)).cpu().numpy()
    assert rel(got, lam * psi) <= (1e-12 if prec != "f32" else 2e-6)


@pytest.mark.parametrize("mixed", [False, True])
def test_mscg_with_phases(p, mixed):
    dims = (8, 4, 4, 8)
    u = S.gauge_links(dims, "expih", 184)
    th = _theta(dims, 185)
    b = S.gaussian_field(dims, 186)
    shifts = [1e-3, 2e-2, 0.3, 2.0]
    lat = p.Lattice(dims)
    g64 = p.Gauge(lat, _gpu(u), "f64", 18, theta=_gpu(th))
    gi = p.Gauge(lat, _gpu(u), "f32", 12, theta=_gpu(th)) if mixed else None
    x, st = p.mscg(g64, _gpu(b), shifts, 0.1, tol=1e-10, g_inner=gi)
    v = oracle.u1_links(u, th)
    xs = x.cpu().numpy()
    for i, s in enumerate(shifts):
        assert oracle.true_residual(dims, v, 0.1, s, b, xs[i]) <= 1e-10, (i, s)


@pytest.mark.parametrize("recon", [18, 12])
@pytest.mark.parametrize("kind", [0, 1])
def test_force_with_phases(p, recon, kind):
    dims = (4, 4, 4, 6)
    u = S.gauge_links(dims, "haar", 187)
    th = _theta(dims, 188)
    b = S.gaussian_field(dims, 189)
    shifts, res = np.array([2e-2, 0.3]), np.array([0.6, 0.3])
    x = oracle.mscg(dims, oracle.u1_links(u, th), 0.1, shifts, b, tol=1e-13)["x"]
    want = oracle.force_u1(dims, u, th, res, x, kind=kind)
    lat = p.Lattice(dims)
    g = p.Gauge(lat, _gpu(u), "f64", recon, theta=_gpu(th))
    got = p.fermion_force(g, list(res), _gpu(x), kind=kind).cpu().numpy()
    assert rel(got, want) <= 1e-12
