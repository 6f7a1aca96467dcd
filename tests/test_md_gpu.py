"""Molecular dynamics on the GPU against the MD oracle.

* momenta from standard normals, the link update exp(i eps H) U, the momentum update and the
  kinetic energy vs oracle.md (FP64: 1e-13 .. 1e-15);
* a whole Omelyan trajectory (gauge + one stout-smeared pseudofermion, 4^4) vs the oracle's
  trajectory: final links and momenta to 1e-9, dH to 1e-8 (solver tolerance 1e-13 on both sides);
* energy conservation: halving eps divides |dH| by ~4 (leapfrog, gauge only, 8^4 and Omelyan with
  fermions, 4^4); reversibility of a gauge trajectory to 1e-12;
* the Metropolis decision of md.trajectory.
"""
import math

import numpy as np
import pytest
import torch

import synthetic as S
from oracle import md as omd

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def p():
    import paper_1801_01473_gb300 as p
    return p


def _gpu(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _xi(seed, v):
    return np.random.default_rng(seed).standard_normal((4, v, 8))


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (6, 4, 6, 10)])
def test_md_kernels_match_oracle(p, dims):
    lat = p.Lattice(dims)
    v = int(np.prod(dims))
    xi = _xi(151, v)
    h = p.md_momenta(lat, _gpu(xi))
    hw = omd.momenta(xi)
    assert np.abs(h.cpu().numpy() - hw).max() < 1e-15
    assert p.md_kinetic(lat, h) == pytest.approx(omd.kinetic(hw), rel=1e-13)
    u = S.gauge_links(dims, "haar", 152)
    ud = _gpu(u)
    p.md_update_links_(lat, 0.13, h, ud)
    assert np.abs(ud.cpu().numpy() - omd.update_links(u, hw, 0.13)).max() < 1e-13
    f = np.random.default_rng(153).standard_normal(u.shape) + 1j * np.random.default_rng(154).standard_normal(u.shape)
    p.md_update_momenta_(lat, 0.07, _gpu(f), h)
    assert np.abs(h.cpu().numpy() - (hw - 0.07j * f)).max() < 1e-14


def _actions(p, dims, lat, stout=True):
    u = S.gauge_links(dims, "expih", 155)
    b = S.gaussian_field(dims, 156)
    pf = ([0.05, 0.5], [0.4, 0.3])
    kw = dict(stout_rho=0.15, stout_steps=1) if stout else {}
    a_gpu = p.md.Action(lat, beta=5.6, mass=0.2, pseudofermions=[p.md.Pseudofermion(_gpu(b), *pf)], tol=1e-13, **kw)
    a_ora = omd.Action(dims, beta=5.6, mass=0.2, pseudofermions=[(b, *pf)], tol=1e-13, **kw)
    return u, a_gpu, a_ora


def test_trajectory_matches_oracle(p):
    dims = (4, 4, 4, 4)
    lat = p.Lattice(dims)
    u, a_gpu, a_ora = _actions(p, dims, lat)
    xi = _xi(157, u.shape[1])
    ud = _gpu(u)
    h = p.md_momenta(lat, _gpu(xi))
    h0 = p.md.hamiltonian(a_gpu, ud, h)
    p.md.omelyan(a_gpu, ud, h, 0.4, 3)
    dh = p.md.hamiltonian(a_gpu, ud, h) - h0
    hw = omd.momenta(xi)
    hw0 = omd.kinetic(hw) + a_ora.value(u)
    uw, hw = omd.omelyan(a_ora, u, hw, 0.4, 3)
    dhw = omd.kinetic(hw) + a_ora.value(uw) - hw0
    assert np.abs(ud.cpu().numpy() - uw).max() < 1e-9
    assert np.abs(h.cpu().numpy() - hw).max() < 1e-9
    assert dh == pytest.approx(dhw, abs=1e-8)


def test_energy_scaling_and_reversibility(p):
    dims = (8, 8, 8, 8)
    lat = p.Lattice(dims)
    u = S.gauge_links(dims, "expih", 158)
    act = p.md.Action(lat, beta=5.6)
    xi = _gpu(_xi(159, u.shape[1]))

    def dh(n):
        ud, h = _gpu(u), p.md_momenta(lat, xi)
        h0 = p.md.hamiltonian(act, ud, h)
        p.md.leapfrog(act, ud, h, 0.5, n)
        return p.md.hamiltonian(act, ud, h) - h0

    d1, d2 = dh(10), dh(20)
    assert 3.4 < d1 / d2 < 4.6
    ud, h = _gpu(u), p.md_momenta(lat, xi)
    p.md.leapfrog(act, ud, h, 0.5, 10)
    h.neg_()
    p.md.leapfrog(act, ud, h, 0.5, 10)
    assert float((ud - _gpu(u)).abs().max()) < 1e-12
    assert float((h + p.md_momenta(lat, xi)).abs().max()) < 1e-11


def test_full_action_energy_scaling(p):
    dims = (4, 4, 4, 4)
    lat = p.Lattice(dims)
    u, a_gpu, _ = _actions(p, dims, lat)
    xi = _gpu(_xi(160, u.shape[1]))

    def dh(n):
        ud, h = _gpu(u), p.md_momenta(lat, xi)
        h0 = p.md.hamiltonian(a_gpu, ud, h)
        p.md.omelyan(a_gpu, ud, h, 0.4, n)
        return p.md.hamiltonian(a_gpu, ud, h) - h0

    d1, d2 = dh(3), dh(6)
    assert 3.2 < d1 / d2 < 4.8


def test_metropolis_decision(p):
    dims = (4, 4, 4, 4)
    lat = p.Lattice(dims)
    u = _gpu(S.gauge_links(dims, "expih", 161))
    act = p.md.Action(lat, beta=5.6)
    xi = _gpu(_xi(162, 256))
    r0 = p.md.trajectory(act, u, xi, 0.5, 10, uniform=0.0)
    assert r0["accepted"] and r0["links"] is not u
    r1 = p.md.trajectory(act, u, xi, 0.5, 10, uniform=math.nextafter(1.0, 0.0))
    assert r1["dH"] == pytest.approx(r0["dH"], rel=1e-12)
    assert r1["accepted"] == (r1["dH"] <= 0.0 or math.nextafter(1.0, 0.0) < math.exp(-r1["dH"]))
    if not r1["accepted"]:
        assert r1["links"] is u


def test_single_precision_forces(p):
    """MD with single-precision forces (gauge force, smearing and chain rule in FP32): the
    Hamiltonian is still conserved to O(eps^2), and a trajectory stays within FP32 rounding of the
    FP64 one."""
    dims = (4, 4, 4, 4)
    lat = p.Lattice(dims)
    u, a64, _ = _actions(p, dims, lat)
    a32 = p.md.Action(lat, beta=a64.beta, mass=a64.mass, pseudofermions=a64.pseudofermions, tol=a64.tol,
                      stout_rho=a64.stout_rho, stout_steps=a64.stout_steps, precision="f32")
    xi = _gpu(_xi(163, u.shape[1]))

    def run(act, n):
        ud, h = _gpu(u), p.md_momenta(lat, xi)
        h0 = p.md.hamiltonian(act, ud, h)
        p.md.omelyan(act, ud, h, 0.4, n)
        return p.md.hamiltonian(act, ud, h) - h0, ud

    d1, u1 = run(a32, 3)
    d2, _ = run(a32, 6)
    assert 3.2 < d1 / d2 < 4.8
    d64, u64 = run(a64, 3)
    assert float((u1 - u64).abs().max()) < 1e-5
    assert d1 == pytest.approx(d64, rel=1e-4, abs=1e-5)


def test_trajectory_with_u1_phases_matches_oracle(p):
    """Rows f1-f3 together: an Omelyan trajectory of gauge + stout-smeared pseudofermion with an
    imaginary chemical potential (constant U(1) phase 0.2 on the time links) against the oracle's
    trajectory (1e-9), and energy conservation at O(eps^2)."""
    dims = (4, 4, 4, 4)
    lat = p.Lattice(dims)
    u = S.gauge_links(dims, "expih", 164)
    b = S.gaussian_field(dims, 165)
    theta = np.zeros((4, u.shape[1]))
    theta[3] = 0.2
    pf = ([0.05, 0.5], [0.4, 0.3])
    a_gpu = p.md.Action(lat, beta=5.6, mass=0.2, pseudofermions=[p.md.Pseudofermion(_gpu(b), *pf)], tol=1e-13,
                        stout_rho=0.15, stout_steps=1, theta=_gpu(theta))
    a_ora = omd.Action(dims, beta=5.6, mass=0.2, pseudofermions=[(b, *pf)], tol=1e-13, stout_rho=0.15,
                       stout_steps=1, theta=theta)
    xi = _xi(166, u.shape[1])
    ud, h = _gpu(u), p.md_momenta(lat, _gpu(xi))
    h0 = p.md.hamiltonian(a_gpu, ud, h)
    p.md.omelyan(a_gpu, ud, h, 0.4, 3)
    dh3 = p.md.hamiltonian(a_gpu, ud, h) - h0
    hw = omd.momenta(xi)
    uw, hw = omd.omelyan(a_ora, u, hw, 0.4, 3)
    assert np.abs(ud.cpu().numpy() - uw).max() < 1e-9
    assert np.abs(h.cpu().numpy() - hw).max() < 1e-9
    ud, h = _gpu(u), p.md_momenta(lat, _gpu(xi))
    p.md.omelyan(a_gpu, ud, h, 0.4, 6)
    dh6 = p.md.hamiltonian(a_gpu, ud, h) - h0
    assert 3.2 < dh3 / dh6 < 4.8


def test_two_pseudofermions_batched_match_oracle(p):
    """Two pseudofermions with one pole set: solved in one batched multi-shift solve and forced by
    one force evaluation over both sets of solutions; the trajectory matches the oracle's (1e-9)."""
    dims = (4, 4, 4, 4)
    lat = p.Lattice(dims)
    u = S.gauge_links(dims, "expih", 167)
    b1, b2 = S.gaussian_field(dims, 168), S.gaussian_field(dims, 169)
    pf = ([0.05, 0.5], [0.4, 0.3])
    a_gpu = p.md.Action(lat, beta=5.6, mass=0.2, tol=1e-13, stout_rho=0.15, stout_steps=1,
                        pseudofermions=[p.md.Pseudofermion(_gpu(b1), *pf), p.md.Pseudofermion(_gpu(b2), *pf)])
    a_ora = omd.Action(dims, beta=5.6, mass=0.2, pseudofermions=[(b1, *pf), (b2, *pf)], tol=1e-13,
                       stout_rho=0.15, stout_steps=1)
    xi = _xi(170, u.shape[1])
    ud, h = _gpu(u), p.md_momenta(lat, _gpu(xi))
    p.md.omelyan(a_gpu, ud, h, 0.4, 3)
    uw, hw = omd.omelyan(a_ora, u, omd.momenta(xi), 0.4, 3)
    assert np.abs(ud.cpu().numpy() - uw).max() < 1e-9
    assert np.abs(h.cpu().numpy() - hw).max() < 1e-9
    assert p.md.hamiltonian(a_gpu, ud, h) == pytest.approx(omd.kinetic(hw) + a_ora.value(uw), rel=1e-10)


def test_multiscale_integrator_matches_oracle(p):
    """Nested Omelyan (fermion force outer, gauge force inner with 3 substeps): GPU vs oracle
    trajectory (1e-9)."""
    dims = (4, 4, 4, 4)
    lat = p.Lattice(dims)
    u, a_gpu, a_ora = _actions(p, dims, lat)
    xi = _xi(171, u.shape[1])
    ud, h = _gpu(u), p.md_momenta(lat, _gpu(xi))
    p.md.omelyan_multiscale(a_gpu, ud, h, 0.4, 2, 3)
    uw, hw = omd.omelyan_multiscale(a_ora, u, omd.momenta(xi), 0.4, 2, 3)
    assert np.abs(ud.cpu().numpy() - uw).max() < 1e-9
    assert np.abs(h.cpu().numpy() - hw).max() < 1e-9


def test_md_force_uses_its_own_approximation(p):
    """A pseudofermion with a separate (cheaper) MD approximation: the momentum update of
    apply_fermion_force is the fermion force of the MD poles and residues, not of the action's."""
    dims = (4, 4, 4, 4)
    lat = p.Lattice(dims)
    u = _gpu(S.gauge_links(dims, "expih", 172))
    b = _gpu(S.gaussian_field(dims, 173))
    pf = p.md.Pseudofermion(b, [0.05, 0.5, 3.0], [0.4, 0.3, 0.2], md_shifts=[0.1], md_residues=[0.7])
    act = p.md.Action(lat, beta=0.0, mass=0.2, tol=1e-13, pseudofermions=[pf])
    h = torch.zeros((4, lat.V, 3, 3), dtype=torch.complex128, device="cuda")
    act.apply_fermion_force(u, h, 1.0)
    g = p.Gauge(lat, u, "f64", 18)
    x, _ = p.mscg(g, b, [0.1], 0.2, tol=1e-13)
    f = p.fermion_force(g, [0.7], x, kind=0)
    assert float((h + 1j * f).abs().max()) <= 1e-12 * float(f.abs().max())
