"""Pins of the oracle's operation counter, which supplies the numerator of every roofline.

Each expected count below is a hand count of the operations the oracle's formula performs,
read off the published formula it restates (paper Sec. 2.3 for the van Leer slope and the
HLLD solver of Miyoshi & Kusano 2005, Eq. 1 for the physical flux, Sec. 2.4 for the E^c
EMF of Gardiner & Stone 2005, Eqs. 5, 6, 9, 10 for the update, RK combine and time step).
A counter that dropped or doubled an operation kind, counted a sign operation, or lost a
part of the cycle fails one of them.  Every add/sub, mul, div and sqrt counts 1 (the oracle
has no fused operations); compares are counted but are not flops.
"""
import numpy as np
import pytest

import oracle
from paper_2304_13746_b300 import inputs

GAMMA = 5.0 / 3.0


def c5(add=0, mul=0, div=0, sqrt=0, cmp=0):
    return {"add": add, "mul": mul, "div": div, "sqrt": sqrt, "cmp": cmp}


def plus(*cs, k=1):
    return {op: k * sum(c[op] for c in cs) for op in oracle.OPS}


def times(c, k):
    return {op: k * c[op] for op in oracle.OPS}


# van Leer slope 2 dL dR / (dL + dR) when dL dR > 0: dL, dR, dL + dR (3 add), dL dR,
# 2 (dL dR) (2 mul), one division, one compare; otherwise only dL, dR, dL dR and the compare.
VL_SLOPE = c5(add=3, mul=2, div=1, cmp=1)
VL_FLAT = c5(add=2, mul=1, cmp=1)
# face value w +- slope / 2: one mul, one add
FACE_VALUE = c5(add=1, mul=1)
# E = P / (gamma - 1) + rho |v|^2 / 2 + |B|^2 / 2: 1 div; 0.5 rho, three squares, the
# product (5 mul) and two adds; three squares and 0.5 x (4 mul) and two adds; two adds
ENERGY = c5(add=6, mul=9, div=1)
# physical flux with E given: pT (4 mul, 3 add), v.B (3 mul, 2 add), the seven components
# rho u (1 mul); rho u u + pT - Bx^2 (3 mul, 2 add); two transverse momenta (3 mul, 1 add
# each); (E + pT) u - Bx v.B (2 mul, 2 add); two induction fluxes (2 mul, 1 add each)
PHYS_FLUX = c5(add=13, mul=23)
# fast speed sqrt((a + sqrt(a^2 - 4 gamma P Bx^2)) / (2 rho)), a = gamma P + |B|^2:
# 9 mul, 5 add, 1 div, 2 sqrt and the compare that clips the discriminant at 0
FAST_SPEED = c5(add=5, mul=9, div=1, sqrt=2, cmp=1)
# total pressure P + |B|^2 / 2 with Bx^2 shared: 3 mul, 3 add
PT = c5(add=3, mul=3)
# supersonic HLLD face (S_L > 0): both energies, Bx^2, both total pressures, both fast
# speeds, max of the fast speeds, S_L and S_R (2 compares, 2 add), both physical fluxes
# and the test S_L > 0
HLLD_SUPERSONIC_L = plus(ENERGY, ENERGY, c5(mul=1), PT, PT, FAST_SPEED, FAST_SPEED,
                         c5(cmp=3, add=2), PHYS_FLUX, PHYS_FLUX, c5(cmp=1))
# with S_R < 0 instead, the test S_L > 0 fails first: one compare more
HLLD_SUPERSONIC_R = plus(HLLD_SUPERSONIC_L, c5(cmp=1))
# E^c edge: four one-sided derivatives 2 (a - b) / d (1 add, 1 mul, 1 div each, both
# upwind candidates formed) chosen by the sign of a mass flux (1 compare when > 0, 2
# otherwise, and 0.5 (up + dn) when it is 0); then (X0 + X1 + Y0 + Y1) / 4 (3 add, 1 mul)
# and two corrections (d / 8) (q3 - q1) (1 div, 1 add, 1 mul) added (1 add each)
EC_BLOCK = c5(add=2, mul=2, div=2)
EC_TAIL = c5(add=7, mul=3, div=2)


def EC(n_pos, n_neg, n_zero):
    assert n_pos + n_neg + n_zero == 4
    return plus(times(EC_BLOCK, 4), EC_TAIL,
                c5(cmp=n_pos + 2 * n_neg + 2 * n_zero, add=n_zero, mul=n_zero))


def test_hand_counts_of_single_calls():
    assert oracle.count_vanleer(0.0, 1.0, 3.0) == VL_SLOPE
    assert oracle.count_vanleer(0.0, -1.0, -1.5) == VL_SLOPE
    assert oracle.count_vanleer(0.0, 1.0, 0.5) == VL_FLAT   # extremum
    assert oracle.count_vanleer(2.0, 2.0, 2.0) == VL_FLAT   # flat
    w = [1.1, 2.0, 0.3, -0.2, 0.6, 0.4, 0.1]
    assert oracle.count_energy_flux(w, 0.7, GAMMA) == (ENERGY, PHYS_FLUX)
    left = [1.0, 6.0, 0.1, 0.2, 0.6, 0.1, 0.2]
    right = [1.2, 5.5, -0.1, 0.3, 0.7, 0.2, -0.1]
    assert oracle.count_hlld(left, right, 0.3, GAMMA) == HLLD_SUPERSONIC_L
    neg = lambda s: [s[0], -s[1]] + s[2:]  # noqa: E731
    assert oracle.count_hlld(neg(right), neg(left), 0.3, GAMMA) == HLLD_SUPERSONIC_R
    X, Y, C = [1.0, 2.0], [3.0, 4.0], [[1.0, 2.0], [3.0, 4.0]]
    assert oracle.count_emf_ec(X, Y, C, [1, 1], [1, 1], 0.1, 0.2) == EC(4, 0, 0)
    assert oracle.count_emf_ec(X, Y, C, [-1, -1], [-1, -1], 0.1, 0.2) == EC(0, 4, 0)
    assert oracle.count_emf_ec(X, Y, C, [0, 0], [0, 0], 0.1, 0.2) == EC(0, 0, 4)
    assert oracle.count_emf_ec(X, Y, C, [1, -1], [0, 2], 0.1, 0.2) == EC(2, 1, 1)


def test_subsonic_hlld_costs_more_than_the_supersonic_face():
    # the star states and the fan add divisions, one square root per side and many products
    left = [1.0, 0.1, 0.1, 0.2, 0.6, 0.5, 0.2]
    right = [1.2, -0.2, -0.1, 0.3, 0.7, 0.2, -0.1]
    c = oracle.count_hlld(left, right, 0.8, GAMMA)
    s = HLLD_SUPERSONIC_L
    assert c["sqrt"] == s["sqrt"] + 2
    assert c["div"] > s["div"] and c["mul"] > s["mul"] + 60 and c["add"] > s["add"] + 40


def supersonic_box(shape=(3, 4, 5)):
    """Uniform state moving faster than the fast speed along +x, +y and +z: every face is
    upwinded from the left, every slope is flat, every mass flux positive."""
    nz, ny, nx = shape
    one = np.ones(shape)
    prim = [1.0 * one, 3.0 * one, 2.5 * one, 2.0 * one, 0.6 * one, 0.3 * one, 0.2 * one,
            0.1 * one]
    lengths = (1.0, 0.8, 0.6)
    return oracle.cons_from_prims(prim, lengths, GAMMA), lengths


def expected_cycle_parts(shape):
    """Per cell-update counts of one RK2 cycle on the uniform supersonic box, part by part."""
    nz, ny, nx = shape
    n = nx * ny * nz
    faces = 2 * 3          # stages x directions, one face per cell each
    e = {p: c5() for p in oracle.PARTS}
    e["prims"] = times(c5(div=1, mul=16, add=9), 2)   # 1/rho; v (3 mul); B_c (3 add, 3 mul);
    #                                                   kinetic (5 mul, 2 add); magnetic
    #                                                   (4 mul, 2 add); P (2 add, 1 mul)
    e["slope"] = times(VL_FLAT, faces * 14)           # 7 variables x 2 sides per face
    e["face"] = times(FACE_VALUE, faces * 14)
    e["riemann"] = times(HLLD_SUPERSONIC_L, faces)
    e["speed"] = c5(cmp=faces)                        # max(|S_L|, |S_R|)
    # per cell and direction: max of two faces, / dl, + ; the cell's max; and per stage
    # the max over the nz plane maxima
    e["invdt"] = plus(times(c5(cmp=4, div=3, add=3), 2), c5(cmp=2 * nz / n))
    e["cell_emf"] = times(c5(mul=2, add=1), 2 * 3 * 4)  # v_a B_b - v_b B_a at 4 edges x 3
    e["edge"] = times(EC(4, 0, 0), 2 * 3)
    # 5 cell fields x 3 directions of (difference, / dl, running sum); 3 face fields x 2
    # EMF differences of the same form
    e["diff"] = times(c5(add=2 * 15 + 2 * 6, div=15 + 6), 2)
    e["accum"] = times(c5(mul=8, add=8), 2)            # U - dt x (...) for 8 fields
    e["combine"] = c5(mul=16, add=8)                  # (1/2) U* + (1/2) U0, stage 2 only
    e["dt"] = c5(div=1 / n, cmp=2 / n)                # cfl / inv; max over the two stages
    return e


def test_whole_cycle_count_on_a_supersonic_box_is_the_sum_of_hand_counts():
    shape = (3, 4, 5)
    cons, lengths = supersonic_box(shape)
    parts = oracle.count_cycle_parts(cons, lengths, GAMMA, 0.4)
    exp = expected_cycle_parts(shape)
    for p in oracle.PARTS:
        for op in oracle.OPS:
            assert parts[p][op] == pytest.approx(exp[p][op], rel=1e-12, abs=1e-12), (p, op)
    total = oracle.count_cycle(cons, lengths, GAMMA, 0.4)
    for op in oracle.OPS:
        assert total[op] == pytest.approx(sum(parts[p][op] for p in oracle.PARTS), rel=1e-12)
    # per face of each direction: the HLLD solve and the two reconstructed states
    for d in range(3):
        h, r = oracle.count_faces(cons, lengths, GAMMA, d)
        assert h == HLLD_SUPERSONIC_L
        assert r == plus(times(VL_FLAT, 14), times(FACE_VALUE, 14))
        split = oracle.count_faces_parts(cons, lengths, GAMMA, d)
        assert split == {"riemann": HLLD_SUPERSONIC_L, "slope": times(VL_FLAT, 14),
                         "face": times(FACE_VALUE, 14)}
        # per face, each of the 7 + 7 slopes counted once: 7 of the 14 evaluations
        assert oracle.algorithmic_face_flops(split) == (oracle.flops(HLLD_SUPERSONIC_L) +
                                                        14 * oracle.flops(FACE_VALUE) +
                                                        7 * oracle.flops(VL_FLAT))


def test_algorithmic_count_removes_exactly_the_repeated_slopes_and_cell_emfs():
    # brute force on a small turbulent box: every (cell, direction, variable) van Leer
    # slope of both stages' primitives counted once through the single-call counter; the
    # cycle's slope part must be exactly twice that, and the cell-centre EMFs four times
    # one evaluation (2 mul, 1 add) per cell, component and stage
    ic = inputs.turbulent_box(6, seed=3)
    u0 = oracle.cons_from_prims(ic.prim, ic.lengths, ic.gamma)
    inv = oracle.speed_pass(u0, ic.lengths, ic.gamma)
    dt = 0.4 / inv
    u1, _ = oracle.stage(u0, ic.lengths, ic.gamma, dt)
    once = c5()
    for u in (u0, u1):
        w = oracle.prims(u, ic.lengths, ic.gamma)
        for d, ax in ((0, 2), (1, 1), (2, 0)):
            t1, t2 = (d + 1) % 3, (d + 2) % 3
            for q in (0, 1 + d, 1 + t1, 1 + t2, 4, 5 + t1, 5 + t2):
                f = w[q]
                fm, fp = np.roll(f, 1, ax), np.roll(f, -1, ax)
                for a, b, c in zip(fm.ravel(), f.ravel(), fp.ravel()):
                    once = plus(once, oracle.count_vanleer(a, b, c))
    n = u0[0].size
    once = times(once, 1.0 / n)
    parts = oracle.count_cycle_parts(u0, ic.lengths, ic.gamma, 0.4, inv_dt=inv)
    for op in oracle.OPS:
        assert parts["slope"][op] == pytest.approx(2 * once[op], rel=1e-12), op
    assert parts["cell_emf"] == times(c5(mul=2, add=1), 4 * 3 * 2)
    alg = oracle.algorithmic_flops(parts)
    total = sum(oracle.flops(c) for c in parts.values())
    cell_emf_once = 3 * 3 * 2  # 3 flops, 3 components, 2 stages
    assert alg == pytest.approx(total - oracle.flops(once) - (4 - 1) * cell_emf_once, rel=1e-12)


def test_turbulent_box_counts():
    # the figures the rooflines use, on a 32^3 box of the benchmark's recipe
    ic = inputs.turbulent_box(32, seed=0)
    cons = oracle.cons_from_prims(ic.prim, ic.lengths, ic.gamma)
    parts = oracle.count_cycle_parts(cons, ic.lengths, ic.gamma, 0.4)
    total = sum(oracle.flops(c) for c in parts.values())
    alg = oracle.algorithmic_flops(parts)
    assert 3000 < total < 3300
    assert 2800 < alg < 3000
    # HLLD dominates: about 70 % of the algorithmic flops
    assert 0.65 < oracle.flops(parts["riemann"]) / alg < 0.8
    assert oracle.fp64_island_flops(parts) == 52 + 32 + 24
