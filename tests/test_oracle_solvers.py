"""Pins of the Rusanov and HLL solvers of Sec. 2.3 (selectable like HLLD).

  * consistency F(U, U) = F(U) and reflection symmetry;
  * HLL: exact upwinding when supersonic, and the Rankine-Hugoniot relations across both
    outer waves with the single HLL state U* = (S_R U_R - S_L U_L - F_R + F_L)/(S_R - S_L)
    (the defining property of the HLL approximate solution, checked against the flux
    returned, not re-derived from it);
  * the paper orders its solvers "from most to least diffusive": Rusanov, HLL, HLLC/HLLD.
    At a stationary contact the mass fluxes are ordered the same way (HLLD exact), and so
    are the L1 errors of the Sod tube against its exact solution;
  * second-order convergence of the linear MHD waves with each solver (Sec. 4.2).
"""
import math
import os
import sys

import numpy as np
import pytest

import oracle
from paper_2304_13746_b300 import inputs

sys.path.insert(0, os.path.dirname(__file__))
import exact_riemann  # noqa: E402
from test_oracle_units import G53, cons_of, random_state, rel  # noqa: E402


@pytest.mark.parametrize("solver", ["rusanov", "hll"])
def test_consistency_and_speeds(solver):
    rng = np.random.default_rng(51)
    for _ in range(300):
        w = random_state(rng)
        bn = rng.normal()
        F, sL, sR = oracle.riemann(solver, w, w, bn, G53)
        assert rel(F, oracle.phys_flux(w, bn, G53)) < 1e-13
        _, hL, hR = oracle.hlld(w, w, bn, G53)
        assert (sL, sR) == (hL, hR)  # the CFL speeds do not depend on the solver


def test_hll_rankine_hugoniot_across_both_outer_waves():
    rng = np.random.default_rng(53)
    for _ in range(500):
        wL, wR = random_state(rng), random_state(rng)
        bn = rng.normal()
        F, SL, SR = oracle.riemann("hll", wL, wR, bn, G53)
        if not (SL < 0 < SR):
            continue
        UL, UR = cons_of(wL, bn, G53), cons_of(wR, bn, G53)
        FL, FR = oracle.phys_flux(wL, bn, G53), oracle.phys_flux(wR, bn, G53)
        Us = (SR * UR - SL * UL - FR + FL) / (SR - SL)
        np.testing.assert_allclose(F, FL + SL * (Us - UL), rtol=1e-12, atol=1e-12)
        np.testing.assert_allclose(F, FR + SR * (Us - UR), rtol=1e-12, atol=1e-12)


def test_hll_supersonic_upwinding():
    rng = np.random.default_rng(57)
    for _ in range(100):
        wL, wR = random_state(rng), random_state(rng)
        wL[1] = wR[1] = 25.0
        bn = rng.normal()
        F, _, _ = oracle.riemann("hll", wL, wR, bn, G53)
        assert np.array_equal(F, oracle.phys_flux(wL, bn, G53))


@pytest.mark.parametrize("solver", ["rusanov", "hll"])
def test_reflection_symmetry(solver):
    rng = np.random.default_rng(59)
    parity = np.array([-1, 1, -1, -1, -1, -1, -1])
    for _ in range(300):
        wL, wR = random_state(rng), random_state(rng)
        bn = rng.normal()
        F, _, _ = oracle.riemann(solver, wL, wR, bn, G53)
        a, b = list(wR), list(wL)
        a[1], b[1] = -a[1], -b[1]
        Fm, _, _ = oracle.riemann(solver, a, b, -bn, G53)
        assert np.max(np.abs(Fm - parity * F)) < 1e-12 * max(np.max(np.abs(F)), 1.0)


def test_hll_equals_rusanov_when_outer_speeds_are_symmetric():
    # u_L = u_R = 0 gives S_L = -S_R = S_max: the HLL formula reduces to Rusanov's
    rng = np.random.default_rng(61)
    for _ in range(100):
        wL, wR = random_state(rng), random_state(rng)
        wL[1] = wR[1] = 0.0
        bn = rng.normal()
        Fh, _, _ = oracle.riemann("hll", wL, wR, bn, G53)
        Fr, _, _ = oracle.riemann("rusanov", wL, wR, bn, G53)
        assert rel(Fh, Fr) < 1e-13


def test_diffusivity_order_at_a_moving_contact():
    # a density jump advected at u: HLLD is exact (upwind flux), HLL and Rusanov smear it,
    # Rusanov the most, as the paper's ordering of its solvers states
    rng = np.random.default_rng(67)
    for _ in range(100):
        w = random_state(rng)
        w[1] = rng.choice([-1, 1]) * rng.uniform(0.2, 0.8)
        wL, wR = list(w), list(w)
        wR[0] = w[0] * rng.uniform(1.5, 4.0)
        bn = rng.normal()
        exact = oracle.phys_flux(wL if w[1] > 0 else wR, bn, G53)
        dev = {s: abs(oracle.riemann(s, wL, wR, bn, G53)[0][0] - exact[0])
               for s in ("rusanov", "hll", "hlld")}
        assert dev["hlld"] < 1e-13
        assert dev["rusanov"] > dev["hll"] > 1e-6


def sod_l1(n_per_unit, solver):
    ic = inputs.sod_double_tube(n_per_unit, axis=0)
    sim = oracle.Sim.from_prims(ic.prim, ic.lengths, ic.gamma, 0.4, solver=solver)
    sim.advance(0.2)
    rho = sim.u[0][0, 0, :]
    x = (np.arange(rho.size) + 0.5) * (2.0 / rho.size)
    sel = (x >= 1.0) & (x < 2.0)
    ex, _, _ = exact_riemann.sample((x[sel] - 1.5) / 0.2, 1.0, 0.0, 1.0, 0.125, 0.0, 0.1, 1.4)
    return float(np.mean(np.abs(rho[sel] - ex)))


def test_sod_errors_follow_the_papers_diffusivity_order():
    e = {s: sod_l1(100, s) for s in ("rusanov", "hll", "hlld")}
    assert e["rusanov"] > e["hll"] > e["hlld"], e
    for s in ("rusanov", "hll"):
        assert sod_l1(200, s) < e[s]


def lw_error(ic, solver):
    sim = oracle.Sim.from_prims(ic.prim, ic.lengths, ic.gamma, 0.4, solver=solver)
    q0 = oracle.prims(sim.u, ic.lengths, ic.gamma)
    sim.advance(ic.meta["t_cross"])
    q1 = oracle.prims(sim.u, ic.lengths, ic.gamma)
    eps, acc, nc = ic.meta["eps"], 0.0, 0
    for f in range(8):
        if np.max(np.abs(q0[f] - np.mean(q0[f]))) < 1e-3 * eps:
            continue
        nc += 1
        acc += (np.sum(np.abs(q0[f] - q1[f])) / (eps * ic.ncells)) ** 2
    return math.sqrt(acc) / nc


@pytest.mark.parametrize("solver", ["rusanov", "hll"])
@pytest.mark.parametrize("mode", ["fast", "alfven"])
def test_linear_wave_second_order(solver, mode):
    e = [lw_error(inputs.linear_wave_1d(n, mode), solver) for n in (32, 64, 128)]
    assert math.log2(e[1] / e[2]) >= 1.9, e
