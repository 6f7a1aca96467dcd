"""RHMC pieces on the GPU: a rational function of the operator applied to a field, the
pseudofermion heatbath, and a full trajectory (heatbath, Omelyan MD with gauge + stout-smeared
fermion forces, Metropolis) with the stored Remez approximations of paper_1801_01473_gb300/data.

* stg_rational_apply vs the oracle's alpha0 b + sum_i r_i x_i (multi-shift solve at 1e-13): 1e-10;
* heatbath identity: phi = R_{1/8}(A) eta gives phi^dag R_{-1/4}(A) phi = eta^dag eta up to the
  approximation errors (2 E_heat + E_act) and the solver tolerance;
* a trajectory from a heatbath pseudofermion conserves the Hamiltonian to O(eps^2) (Omelyan: halving
  eps divides dH by ~4) and the Metropolis test accepts at dH < 0 with uniform 0.999.
"""
import json
import os

import numpy as np
import pytest
import torch

import oracle
import synthetic as S

pytestmark = pytest.mark.gpu

RAT = json.load(open(os.path.join(os.path.dirname(os.path.dirname(__file__)), "paper_1801_01473_gb300", "data",
                               "rhmc_rational_m0.3.json")))
MASS = 0.3


class _Approx:
    def __init__(self, d):
        self.alpha0, self.residues, self.poles, self.err = d["alpha0"], d["residues"], d["poles"], d["max_rel_error"]


HEAT, ACT = _Approx(RAT["heatbath"]), _Approx(RAT["action"])


@pytest.fixture(scope="module")
def p():
    import paper_1801_01473_gb300 as p
    return p


def _gpu(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (6, 4, 4, 10)])
def test_rational_apply_matches_oracle(p, dims):
    u = S.gauge_links(dims, "expih", 201)
    b = S.gaussian_field(dims, 202)
    lat = p.Lattice(dims)
    g = p.Gauge(lat, _gpu(u), "f64", 18)
    out, st = p.rational_apply(g, _gpu(b), ACT.alpha0, ACT.residues, ACT.poles, MASS, tol=1e-13)
    x = oracle.mscg(dims, u, MASS, np.array(ACT.poles), b, tol=1e-13)["x"]
    want = ACT.alpha0 * b + sum(r * x[i] for i, r in enumerate(ACT.residues))
    got = out.cpu().numpy()
    assert np.abs(got - want).max() <= 1e-10 * np.abs(want).max()
    assert max(st["true_resid"]) <= 1e-13


@pytest.mark.parametrize("mixed", [False, True])
def test_heatbath_identity(p, mixed):
    dims = (6, 4, 4, 6)
    u = S.gauge_links(dims, "expih", 203)
    lat = p.Lattice(dims)
    act = p.md.Action(lat, beta=5.6, mass=MASS, tol=1e-12, inner="f32" if mixed else None,
                      stout_rho=0.15, stout_steps=2)
    eta = _gpu(S.gaussian_field(dims, 204))
    pf = p.md.pseudofermion_heatbath(act, _gpu(u), eta, HEAT, ACT)
    # the fermion action alone (beta = 0)
    fermion_only = p.md.Action(lat, beta=0.0, mass=MASS, tol=1e-12, pseudofermions=[pf], stout_rho=0.15, stout_steps=2)
    s_f = fermion_only.value(_gpu(u))
    e2 = float(torch.vdot(eta.reshape(-1), eta.reshape(-1)).real)
    assert abs(s_f / e2 - 1) <= 2 * HEAT.err + ACT.err + 1e-9


def test_rhmc_trajectory(p):
    dims = (4, 4, 4, 4)
    u = _gpu(S.gauge_links(dims, "expih", 205))
    lat = p.Lattice(dims)
    act = p.md.Action(lat, beta=5.6, mass=MASS, tol=1e-12, stout_rho=0.15, stout_steps=1)
    act.pseudofermions = [p.md.pseudofermion_heatbath(act, u, _gpu(S.gaussian_field(dims, 206)), HEAT, ACT)]
    xi = _gpu(np.random.default_rng(207).standard_normal((4, lat.V, 8)))
    d = []
    for n in (4, 8):
        r = p.md.trajectory(act, u, xi, 0.3, n, uniform=0.999)
        d.append(r["dH"])
        assert r["accepted"] == (r["dH"] <= 0 or 0.999 < np.exp(-r["dH"]))
    assert 3.2 < d[0] / d[1] < 4.8
