"""Stout smearing and its force chain rule on the GPU against the FP64 oracle.

* smeared levels vs oracle.stout element by element (FP64: 1e-13 absolute on
  entries of modulus <= 1), several lattices including ragged thread-block
  tails, both signs of rho, 1..3 steps;
* the pulled-back gradient (kind 1) and the Lie-algebra force (kind 0) vs
  oracle.stout_backward (1e-12 relative);
* the smeared pseudofermion force: GPU solve + fermion force on U^(k) +
  chain rule vs the oracle's chain, and vs finite differences of the action;
* torch autograd through StoutSmear (gradcheck) and through the composed action;
* rho = 0 is the identity (bitwise), and at 48^4 (2 steps, rho = 0.15):
  32 sampled smeared links vs the oracle's single-link smearing, SU(3)
  unitarity of every link, and finite differences of a linear functional on
  32 sampled links.
"""
import numpy as np
import pytest
import torch

import oracle
import synthetic as S
from oracle import stout as ost

pytestmark = pytest.mark.gpu

CASES = [  # dims, link kind, seed, rho, nstep
    ((4, 4, 4, 4), "haar", 81, 0.15, 2),
    ((6, 4, 6, 10), "expih", 82, 0.1, 3),   # V = 1440: ragged last block of 128
    ((4, 6, 4, 8), "haar", 83, 0.5, 1),
    ((4, 4, 4, 6), "haar", 84, -0.2, 2),
]


@pytest.fixture(scope="module")
def p():
    import paper_1801_01473_gb300 as p
    return p


def _gpu(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("dims,kind,seed,rho,nstep", CASES)
def test_smear_matches_oracle(p, dims, kind, seed, rho, nstep):
    u = S.gauge_links(dims, kind, seed)
    want = ost.stout(dims, u, rho, nstep)[1:]
    lat = p.Lattice(dims)
    got = p.stout_smear(lat, _gpu(u), rho, nstep).cpu().numpy()
    assert got.shape == (nstep, 4, u.shape[1], 3, 3)
    for k in range(nstep):
        assert np.abs(got[k] - want[k]).max() < 1e-13, k


@pytest.mark.parametrize("dims,kind,seed,rho,nstep", CASES)
@pytest.mark.parametrize("out_kind", [1, 0])
def test_force_chain_matches_oracle(p, dims, kind, seed, rho, nstep, out_kind):
    u = S.gauge_links(dims, kind, seed)
    g = np.random.default_rng(seed + 100)
    z = g.standard_normal(u.shape) + 1j * g.standard_normal(u.shape)
    want = ost.stout_backward(dims, ost.stout(dims, u, rho, nstep), rho, z)
    if out_kind == 0:
        want = ost.lie_force(u, want)
    lat = p.Lattice(dims)
    ud = _gpu(u)
    levels = p.stout_smear(lat, ud, rho, nstep)
    got = p.stout_force(lat, ud, levels, rho, _gpu(z), kind=out_kind).cpu().numpy()
    assert np.abs(got - want).max() <= 1e-12 * np.abs(want).max()


def test_rho_zero_is_identity(p):
    dims = (4, 4, 4, 6)
    u = S.gauge_links(dims, "haar", 85)
    lat = p.Lattice(dims)
    ud = _gpu(u)
    levels = p.stout_smear(lat, ud, 0.0, 2)
    assert torch.equal(levels[0], ud) and torch.equal(levels[1], ud)
    z = _gpu(np.random.default_rng(86).standard_normal(u.shape) + 0j)
    assert torch.equal(p.stout_force(lat, ud, levels, 0.0, z, kind=1), z)


def test_many_steps(p):
    dims = (4, 4, 4, 4)
    u = S.gauge_links(dims, "haar", 87)
    want = ost.stout(dims, u, 0.1, 16)[-1]
    got = p.stout_smear(p.Lattice(dims), _gpu(u), 0.1, 16)[-1].cpu().numpy()
    assert np.abs(got - want).max() < 1e-12


def _action_setup(dims, seed):
    u = S.gauge_links(dims, "haar", seed)
    b = S.gaussian_field(dims, seed + 1)
    return u, b


def test_smeared_fermion_force_matches_oracle_chain(p):
    dims, rho, nstep, mass = (4, 4, 4, 4), 0.15, 2, 0.1
    shifts, res = [2e-2, 0.3], [0.6, 0.3]
    u, b = _action_setup(dims, 88)
    levels_o = ost.stout(dims, u, rho, nstep)
    sol = oracle.mscg(dims, levels_o[-1], mass, np.array(shifts), b, tol=1e-13)
    want = ost.stout_backward(dims, levels_o, rho, oracle.force(dims, levels_o[-1], np.array(res), sol["x"], kind=1))

    lat = p.Lattice(dims)
    ud = _gpu(u)
    levels = p.stout_smear(lat, ud, rho, nstep)
    gk = p.Gauge(lat, levels[-1].contiguous(), "f64", 18)
    x, _ = p.mscg(gk, _gpu(b), shifts, mass, tol=1e-13)
    got = p.stout_force(lat, ud, levels, rho, p.fermion_force(gk, res, x, kind=1), kind=1).cpu().numpy()
    assert np.abs(got - want).max() <= 1e-9 * np.abs(want).max()


def test_autograd_smeared_action_finite_differences(p):
    dims, rho, nstep, mass = (4, 4, 4, 4), 0.15, 2, 0.1
    shifts, res = [2e-2, 0.3], [0.6, 0.3]
    u, b = _action_setup(dims, 89)
    lat = p.Lattice(dims)
    bd = _gpu(b)

    def action(links):
        return p.pseudofermion_action(p.stout_smear_links(links, lat, rho, nstep), bd, lat, shifts, res, mass, 1e-13)

    ud = _gpu(u).requires_grad_(True)
    action(ud).backward()
    grad = ud.grad.cpu().numpy()
    g = np.random.default_rng(90)
    m = g.standard_normal(u.shape) + 1j * g.standard_normal(u.shape)
    x = 0.5 * (m - np.conj(np.swapaxes(m, -1, -2)))
    x -= np.trace(x, axis1=-2, axis2=-1)[..., None, None] / 3.0 * np.eye(3)
    du = x @ u
    eps = 1e-5
    with torch.no_grad():
        sp = float(action(_gpu(u + eps * du)))
        sm = float(action(_gpu(u - eps * du)))
    fd = (sp - sm) / (2 * eps)
    assert np.sum(np.conj(grad) * du).real == pytest.approx(fd, rel=1e-6)


def test_autograd_gradcheck(p):
    dims, rho = (4, 4, 4, 4), 0.15
    u = S.gauge_links(dims, "haar", 91)
    lat = p.Lattice(dims)
    z = _gpu(np.random.default_rng(92).standard_normal(u.shape) + 0j)

    def f(links):
        return (p.stout_smear_links(links, lat, rho, 2) * z.conj()).real.sum()

    ud = _gpu(u).requires_grad_(True)
    assert torch.autograd.gradcheck(f, (ud,), eps=1e-6, atol=1e-7, rtol=1e-6, fast_mode=True)


# ---------------------------------------------------------------- 48^4, the force workload's links

DIMS48 = (48, 48, 48, 48)


@pytest.fixture(scope="module")
def big(p):
    cfg = S.CONFIGS["force_48x48x48x48"]
    u = S.gauge_links(DIMS48, cfg["links"], 1000 + cfg["k"])
    lat = p.Lattice(DIMS48)
    ud = _gpu(u)
    return u, lat, ud


def _sample(n, seed):
    g = np.random.default_rng(seed)
    v = int(np.prod(DIMS48))
    return [(int(g.integers(4)), int(g.integers(v))) for _ in range(n)]


def test_48_sampled_links_and_unitarity(p, big):
    u, lat, ud = big
    levels = p.stout_smear(lat, ud, 0.15, 2)
    top = levels[-1]
    for mu, s in _sample(32, 93):
        want = ost.smeared_link(DIMS48, u, 0.15, 2, mu, s)
        assert np.abs(top[mu, s].cpu().numpy() - want).max() < 1e-13
    for k in range(2):
        m = levels[k].reshape(-1, 3, 3)
        for c in range(0, m.shape[0], 1 << 22):
            blk = m[c:c + (1 << 22)]
            err = (blk @ blk.conj().transpose(-1, -2) - torch.eye(3, dtype=blk.dtype, device=blk.device)).abs().max()
            assert float(err) < 1e-13


def test_48_force_finite_differences(p, big):
    u, lat, ud = big
    rho, nstep = 0.15, 2
    gen = torch.Generator(device="cuda").manual_seed(94)
    z = torch.complex(torch.randn(ud.shape, dtype=torch.float64, device="cuda", generator=gen),
                      torch.randn(ud.shape, dtype=torch.float64, device="cuda", generator=gen))
    levels = p.stout_smear(lat, ud, rho, nstep)
    grad = p.stout_force(lat, ud, levels, rho, z, kind=1)
    del levels
    g = np.random.default_rng(95)
    eps = 1e-5
    for mu, s in _sample(32, 96):
        m = g.standard_normal((3, 3)) + 1j * g.standard_normal((3, 3))
        x = 0.5 * (m - m.conj().T)
        x -= np.trace(x) / 3.0 * np.eye(3)
        du = torch.from_numpy(x @ u[mu, s]).cuda()
        up = ud.clone()
        up[mu, s] += eps * du
        lp = p.stout_smear(lat, up, rho, nstep)[-1]
        up[mu, s] -= 2 * eps * du
        lm = p.stout_smear(lat, up, rho, nstep)[-1]
        fd = float(((lp - lm) * z.conj()).real.sum()) / (2 * eps)  # only the link's neighbourhood differs
        an = float((grad[mu, s].conj() * du).real.sum())
        assert an == pytest.approx(fd, rel=1e-6, abs=1e-9)
        del lp, lm, up


@pytest.mark.parametrize("dims,kind,seed,rho,nstep", CASES[:2])
@pytest.mark.parametrize("out_kind", [1, 0])
def test_fp32_smear_and_chain(p, dims, kind, seed, rho, nstep, out_kind):
    """Single-precision variants (complex64 arrays, FP32 arithmetic) against the FP64 oracle at
    FP32 tolerances: links 5e-6 absolute, pulled-back gradient 2e-5 relative."""
    u = S.gauge_links(dims, kind, seed)
    g = np.random.default_rng(seed + 200)
    z = g.standard_normal(u.shape) + 1j * g.standard_normal(u.shape)
    lat = p.Lattice(dims)
    u32 = p.complex_convert(_gpu(u), torch.complex64)
    levels = p.stout_smear(lat, u32, rho, nstep)
    assert levels.dtype == torch.complex64
    want = ost.stout(dims, u, rho, nstep)
    for k in range(nstep):
        assert np.abs(levels[k].cpu().numpy().astype(np.complex128) - want[k + 1]).max() < 5e-6
    gw = ost.stout_backward(dims, want, rho, z)
    if out_kind == 0:
        gw = ost.lie_force(u, gw)
    got = p.stout_force(lat, u32, levels, rho, p.complex_convert(_gpu(z), torch.complex64), kind=out_kind)
    assert np.abs(got.cpu().numpy().astype(np.complex128) - gw).max() <= 2e-5 * np.abs(gw).max()


def test_complex_convert_round_trip(p):
    x = torch.randn(1000, dtype=torch.complex64, device="cuda")
    y = p.complex_convert(x, torch.complex128)
    assert torch.equal(y, x.to(torch.complex128))
    assert torch.equal(p.complex_convert(y, torch.complex64), x)
