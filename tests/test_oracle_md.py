"""Pins of the MD oracle (no GPU).

* momenta from standard normals are traceless Hermitian with (1/2) tr H^2 = (1/2) sum xi^2
  (the Gell-Mann matrices are orthogonal with tr(lambda_a lambda_b) = 2 delta_ab);
* Hamiltonian dynamics: a second-order integrator conserves H = (1/2) sum tr H^2 + S up to
  O(eps^2), so halving eps divides |dH| by ~4 -- this holds only if the force is the exact
  gradient of the action with the right sign and normalisation, for the gauge action alone and
  for gauge + stout-smeared pseudofermion actions;
* reversibility: integrating, negating the momenta and integrating again returns the start.
"""
import numpy as np
import pytest

import synthetic as S
from oracle import md as omd

DIMS = (4, 4, 4, 4)


def _xi(seed, v):
    return np.random.default_rng(seed).standard_normal((4, v, 8))


def test_momenta_algebra():
    v = int(np.prod(DIMS))
    xi = _xi(141, v)
    h = omd.momenta(xi)
    assert np.abs(h - np.conj(np.swapaxes(h, -1, -2))).max() < 1e-15
    assert np.abs(np.trace(h, axis1=-2, axis2=-1)).max() < 1e-14
    assert omd.kinetic(h) == pytest.approx(0.5 * np.sum(xi ** 2), rel=1e-13)


def _dh(action, u, h, tau, nsteps, integ):
    h0 = omd.kinetic(h) + action.value(u)
    u1, h1 = integ(action, u, h, tau, nsteps)
    return omd.kinetic(h1) + action.value(u1) - h0


def test_gauge_leapfrog_energy_scaling_and_reversibility():
    u = S.gauge_links(DIMS, "expih", 142)
    h = omd.momenta(_xi(143, u.shape[1]))
    act = omd.Action(DIMS, beta=5.6)
    d1 = _dh(act, u, h, 0.5, 10, omd.leapfrog)
    d2 = _dh(act, u, h, 0.5, 20, omd.leapfrog)
    assert abs(d1) > 1e-6
    assert 3.4 < d1 / d2 < 4.6
    u1, h1 = omd.leapfrog(act, u, h, 0.5, 10)
    u2, h2 = omd.leapfrog(act, u1, -h1, 0.5, 10)
    assert np.abs(u2 - u).max() < 1e-12 and np.abs(h2 + h).max() < 1e-11


def test_full_action_omelyan_energy_scaling():
    u = S.gauge_links(DIMS, "expih", 144)
    b = S.gaussian_field(DIMS, 145)
    h = omd.momenta(_xi(146, u.shape[1]))
    act = omd.Action(DIMS, beta=5.6, mass=0.2, pseudofermions=[(b, [0.05, 0.5], [0.4, 0.3])],
                     stout_rho=0.15, stout_steps=1)
    d1 = _dh(act, u, h, 0.4, 3, omd.omelyan)
    d2 = _dh(act, u, h, 0.4, 6, omd.omelyan)
    assert abs(d1) > 1e-7
    assert 3.2 < d1 / d2 < 4.8


def test_full_action_with_u1_phases_energy_scaling():
    """With an imaginary chemical potential on the time links the MD force must still be the
    exact gradient of the action (phases enter D and the force, not the gauge part)."""
    u = S.gauge_links(DIMS, "expih", 147)
    b = S.gaussian_field(DIMS, 148)
    h = omd.momenta(_xi(149, u.shape[1]))
    theta = np.zeros((4, u.shape[1]))
    theta[3] = 0.2
    act = omd.Action(DIMS, beta=5.6, mass=0.2, pseudofermions=[(b, [0.05, 0.5], [0.4, 0.3])],
                     stout_rho=0.15, stout_steps=1, theta=theta)
    d1 = _dh(act, u, h, 0.4, 3, omd.omelyan)
    d2 = _dh(act, u, h, 0.4, 6, omd.omelyan)
    assert 3.2 < d1 / d2 < 4.8


def test_multiscale_integrator_energy_scaling():
    """Nested Omelyan (fermion force outer, gauge force inner with 3 substeps): second order in the
    outer step."""
    u = S.gauge_links(DIMS, "expih", 150)
    b = S.gaussian_field(DIMS, 151)
    h = omd.momenta(_xi(152, u.shape[1]))
    act = omd.Action(DIMS, beta=5.6, mass=0.2, pseudofermions=[(b, [0.05, 0.5], [0.4, 0.3])])

    def dh(n):
        h0 = omd.kinetic(h) + act.value(u)
        u1, h1 = omd.omelyan_multiscale(act, u, h, 0.4, n, 3)
        return omd.kinetic(h1) + act.value(u1) - h0

    d1, d2 = dh(3), dh(6)
    assert 3.2 < d1 / d2 < 4.8
