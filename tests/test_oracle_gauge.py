"""Pins of the oracle's tree-level Symanzik gauge action and force (no GPU).

* unit links: every loop has Re tr = 3, so S = -(beta/3) V 12 (5/6 - 1/12) 3 = -9 beta V, F = 0;
* a constant U(1) x U(1) magnetic flux B per plaquette in the (x, y) plane (charges +1, -1, 0 on
  the colour diagonal, B = 2 pi n / (Lx Ly), twisted links on the y boundary): closed form
  S = -(beta/3) V [5/6 (2 (2 cos B + 1) + 30) - 1/12 (2 (2 cos 2B + 1) + 30)]
  (the two ordered (x, y) pairs see flux B on plaquettes, 2B on 2x1 rectangles);
* the plaquette part of the gradient against the stout oracle's staple sum, G = -(beta/3)(5/3) C;
* gauge invariance of S and covariance of F;
* the gradient against central finite differences of S along su(3) and complex directions.
"""
import numpy as np
import pytest

import synthetic as S
from oracle import gauge as og
from oracle import stout as ost
from tests import latutil as lu

DIMS = (4, 4, 4, 6)
BETA = 3.7


@pytest.fixture(scope="module")
def links():
    return S.gauge_links(DIMS, "haar", 121)


def test_unit_links():
    v = int(np.prod(DIMS))
    u = np.broadcast_to(np.eye(3, dtype=np.complex128), (4, v, 3, 3)).copy()
    assert og.action(DIMS, u, BETA) == pytest.approx(-9.0 * BETA * v, rel=1e-14)
    assert np.abs(og.force(DIMS, u, BETA)).max() < 1e-14


def _flux_links(dims, n):
    lx, ly = dims[0], dims[1]
    b = 2 * np.pi * n / (lx * ly)
    c = lu.coords(dims)
    v = c.shape[0]
    q = np.array([1.0, -1.0, 0.0])
    u = np.broadcast_to(np.eye(3, dtype=np.complex128), (4, v, 3, 3)).copy()
    for a in range(3):
        u[0, :, a, a] = np.exp(-1j * q[a] * b * c[:, 1])
        u[1, :, a, a] = np.where(c[:, 1] == ly - 1, np.exp(1j * q[a] * b * ly * c[:, 0]), 1.0)
    return u, b


@pytest.mark.parametrize("n", [1, 3])
def test_constant_flux_closed_form(n):
    u, b = _flux_links(DIMS, n)
    v = u.shape[1]
    want = -BETA / 3.0 * v * (5.0 / 6.0 * (2 * (2 * np.cos(b) + 1) + 30) - 1.0 / 12.0 * (2 * (2 * np.cos(2 * b) + 1) + 30))
    assert og.action(DIMS, u, BETA) == pytest.approx(want, rel=1e-13)


def test_plaquette_gradient_is_staple_sum(links):
    g = og.gradient(DIMS, links, BETA, c1=0.0)
    want = -BETA / 3.0 * (5.0 / 3.0) * ost.staples(DIMS, links)
    assert np.abs(g - want).max() < 1e-12


def test_gauge_invariance_and_covariance(links):
    v = links.shape[1]
    om = S.haar_su3(np.random.default_rng(122), v)
    ut = lu.gauge_transform_links(DIMS, links, om)
    assert og.action(DIMS, ut, BETA) == pytest.approx(og.action(DIMS, links, BETA), rel=1e-12)
    f, ft = og.force(DIMS, links, BETA), og.force(DIMS, ut, BETA)
    want = om[None] @ f @ np.conj(np.swapaxes(om, 1, 2))[None]
    assert np.abs(ft - want).max() < 1e-12


@pytest.mark.parametrize("direction", ["algebra", "complex"])
def test_gradient_finite_differences(links, direction):
    g = np.random.default_rng(123)
    grad = og.gradient(DIMS, links, BETA)
    if direction == "algebra":
        m = g.standard_normal(links.shape) + 1j * g.standard_normal(links.shape)
        x = 0.5 * (m - np.conj(np.swapaxes(m, -1, -2)))
        x -= (np.trace(x, axis1=-2, axis2=-1) / 3.0)[..., None, None] * np.eye(3)
        du = x @ links
    else:
        du = g.standard_normal(links.shape) + 1j * g.standard_normal(links.shape)
    eps = 1e-5
    fd = (og.action(DIMS, links + eps * du, BETA) - og.action(DIMS, links - eps * du, BETA)) / (2 * eps)
    assert np.sum(np.conj(grad) * du).real == pytest.approx(fd, rel=1e-8)
    if direction == "algebra":
        f = og.force(DIMS, links, BETA)
        assert np.einsum("lsab,lsba->", x, f).real == pytest.approx(fd, rel=1e-8)


def test_link_gradient_matches_whole_lattice(links):
    g = og.gradient(DIMS, links, BETA)
    v = links.shape[1]
    for mu, s in [(0, 0), (1, 5), (2, v - 1), (3, 77), (0, 143)]:
        assert np.abs(og.link_gradient(DIMS, links, BETA, mu, s) - g[mu, s]).max() < 1e-12
