"""Tree-level Symanzik gauge action and force on the GPU against the FP64 oracle.

* action, plaquette and rectangle sums vs oracle.gauge (1e-13 relative), lattices with ragged
  thread-block tails and Haar / exp(i 0.3 H) links;
* the gradient (kind 1) and the Lie-algebra force (kind 0) vs the oracle element by element
  (1e-12 relative);
* unit links: S = -9 beta V exactly and F = 0; a constant magnetic flux: the closed form;
* 48^4 (the force workload's links): 32 sampled links of the gradient vs the oracle's single-link
  gradient; unit links give S = -9 beta V at full size.
"""
import numpy as np
import pytest
import torch

import synthetic as S
from oracle import gauge as og
from tests import latutil as lu

pytestmark = pytest.mark.gpu

BETA = 3.7
CASES = [((4, 4, 4, 6), "haar", 131), ((6, 4, 6, 10), "expih", 132), ((8, 4, 4, 4), "haar", 133)]


@pytest.fixture(scope="module")
def p():
    import paper_1801_01473_gb300 as p
    return p


def _gpu(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("dims,kind,seed", CASES)
def test_action_matches_oracle(p, dims, kind, seed):
    u = S.gauge_links(dims, kind, seed)
    got = p.gauge_action(p.Lattice(dims), _gpu(u), BETA)
    assert got["action"] == pytest.approx(og.action(dims, u, BETA), rel=1e-13)
    assert got["plaquette_sum"] == pytest.approx(og.action(dims, u, -3.0 / 2.0, 1.0, 0.0), rel=1e-13)
    assert got["rectangle_sum"] == pytest.approx(og.action(dims, u, -3.0, 0.0, 1.0), rel=1e-13)


@pytest.mark.parametrize("dims,kind,seed", CASES)
@pytest.mark.parametrize("out_kind", [1, 0])
def test_force_matches_oracle(p, dims, kind, seed, out_kind):
    u = S.gauge_links(dims, kind, seed)
    want = og.gradient(dims, u, BETA) if out_kind == 1 else og.force(dims, u, BETA)
    got = p.gauge_force(p.Lattice(dims), _gpu(u), BETA, kind=out_kind).cpu().numpy()
    assert np.abs(got - want).max() <= 1e-12 * np.abs(want).max()


def test_unit_links_and_flux():
    import paper_1801_01473_gb300 as p
    dims = (6, 4, 4, 4)
    v = int(np.prod(dims))
    lat = p.Lattice(dims)
    unit = np.broadcast_to(np.eye(3, dtype=np.complex128), (4, v, 3, 3)).copy()
    assert p.gauge_action(lat, _gpu(unit), BETA)["action"] == pytest.approx(-9.0 * BETA * v, rel=1e-15)
    assert float(p.gauge_force(lat, _gpu(unit), BETA, kind=0).abs().max()) < 1e-14
    # constant flux B = 2 pi / (Lx Ly) in the (x, y) plane, charges (+1, -1, 0)
    b = 2 * np.pi / (dims[0] * dims[1])
    c = lu.coords(dims)
    u = unit.copy()
    for a, q in enumerate((1.0, -1.0, 0.0)):
        u[0, :, a, a] = np.exp(-1j * q * b * c[:, 1])
        u[1, :, a, a] = np.where(c[:, 1] == dims[1] - 1, np.exp(1j * q * b * dims[1] * c[:, 0]), 1.0)
    want = -BETA / 3.0 * v * (5.0 / 6.0 * (2 * (2 * np.cos(b) + 1) + 30)
                              - 1.0 / 12.0 * (2 * (2 * np.cos(2 * b) + 1) + 30))
    assert p.gauge_action(lat, _gpu(u), BETA)["action"] == pytest.approx(want, rel=1e-13)


DIMS48 = (48, 48, 48, 48)


def test_48_sampled_gradient_and_unit_action(p):
    cfg = S.CONFIGS["force_48x48x48x48"]
    u = S.gauge_links(DIMS48, cfg["links"], 1000 + cfg["k"])
    lat = p.Lattice(DIMS48)
    ud = _gpu(u)
    grad = p.gauge_force(lat, ud, BETA, kind=1)
    g = np.random.default_rng(134)
    v = int(np.prod(DIMS48))
    for _ in range(32):
        mu, s = int(g.integers(4)), int(g.integers(v))
        want = og.link_gradient(DIMS48, u, BETA, mu, s)
        assert np.abs(grad[mu, s].cpu().numpy() - want).max() <= 1e-12 * np.abs(want).max()
    del grad
    ud.copy_(torch.eye(3, dtype=torch.complex128, device="cuda").expand(4, v, 3, 3))
    assert p.gauge_action(lat, ud, BETA)["action"] == pytest.approx(-9.0 * BETA * v, rel=1e-14)


@pytest.mark.parametrize("dims,kind,seed", CASES)
@pytest.mark.parametrize("out_kind", [1, 0])
def test_fp32_force_matches_oracle(p, dims, kind, seed, out_kind):
    """Single-precision gauge force (complex64 links, FP32 arithmetic): 2e-5 relative."""
    u = S.gauge_links(dims, kind, seed)
    want = og.gradient(dims, u, BETA) if out_kind == 1 else og.force(dims, u, BETA)
    u32 = p.complex_convert(_gpu(u), torch.complex64)
    got = p.gauge_force(p.Lattice(dims), u32, BETA, kind=out_kind)
    assert got.dtype == torch.complex64
    assert np.abs(got.cpu().numpy().astype(np.complex128) - want).max() <= 2e-5 * np.abs(want).max()
