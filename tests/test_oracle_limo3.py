"""The oracle's LimO3 reconstruction (Sec. 2.3; the compact third-order limiter of Cada &
Torrilhon 2009) against what the mathematics fixes, independently of its own formula.

* Exactness: from the cell averages of a parabola, the unlimited third-order face value is
  the parabola's point value at the face.  Where the limiter leaves it alone -- ratio t of
  the difference behind the cell to the one toward the face in [0.4, 2.5] on monotone data,
  or in [-2, -0.8] at an extremum -- LimO3 must return that point value.  Linear data give
  the midpoint value at every face.
* Bounds: a face value lies between the cell's value and the neighbour's on that side, and
  on monotone data it moves by at most the difference behind the cell.
* Jumps: a cell next to a flat run keeps its value at the face beyond the jump.
* Scheme: with RK3 on the smooth linear waves of Sec. 4.2 the error falls faster than
  second order at high resolution (the paper's convergence figure) and stays well below
  PLM's with RK2.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2304_13746_b300 import inputs


def cell_averages(c0, c1, c2, centres, h):
    """Exact averages of c0 + c1 x + c2 x^2 over cells [x - h/2, x + h/2]."""
    return [c0 + c1 * x + c2 * (x * x + h * h / 12.0) for x in centres]


def parabola(c0, c1, c2, x):
    return c0 + c1 * x + c2 * x * x


def ratios(am, a0, ap):
    """t at the upper face and at the lower face of the middle cell."""
    return (a0 - am) / (ap - a0), (a0 - ap) / (am - a0)


@pytest.mark.parametrize("regime", ["monotone", "extremum"])
def test_parabola_face_values_are_exact_where_unlimited(regime):
    rng = np.random.default_rng(11 if regime == "monotone" else 12)
    checked = 0
    while checked < 200:
        h = float(rng.uniform(0.01, 1.0))
        c0 = float(rng.normal())
        c1 = float(rng.normal())
        c2 = float(rng.normal()) / h * (0.3 if regime == "monotone" else 3.0)
        xc = float(rng.uniform(-1, 1))
        am, a0, ap = cell_averages(c0, c1, c2, (xc - h, xc, xc + h), h)
        tu, tl = ratios(am, a0, ap)
        lo, hi = (0.4, 2.5) if regime == "monotone" else (-2.0, -0.8)
        if not (lo + 1e-6 < tu < hi - 1e-6 and lo + 1e-6 < tl < hi - 1e-6):
            continue
        up = oracle.limo3_face(am, a0, ap)
        down = oracle.limo3_face(ap, a0, am)
        scale = abs(a0) + abs(ap - a0) + abs(a0 - am)
        assert abs(up - parabola(c0, c1, c2, xc + h / 2)) <= 1e-13 * scale
        assert abs(down - parabola(c0, c1, c2, xc - h / 2)) <= 1e-13 * scale
        checked += 1


def test_linear_data_give_midpoints():
    for am, a0, ap in ((0.0, 1.0, 2.0), (3.0, 1.5, 0.0), (-1e3, 2e3, 5e3)):
        assert oracle.limo3_face(am, a0, ap) == pytest.approx(0.5 * (a0 + ap), rel=1e-15)
        assert oracle.limo3_face(ap, a0, am) == pytest.approx(0.5 * (a0 + am), rel=1e-15)


def test_face_values_stay_between_neighbours():
    rng = np.random.default_rng(13)
    for _ in range(5000):
        am, a0, ap = (float(v) for v in rng.normal(size=3) * rng.choice([1e-3, 1.0, 1e3]))
        for back, face in ((am, ap), (ap, am)):
            v = oracle.limo3_face(back, a0, face)
            lo, hi = min(a0, face), max(a0, face)
            tol = 1e-15 * (abs(a0) + abs(face))
            assert lo - tol <= v <= hi + tol, (back, a0, face, v)
            if (a0 - back) * (face - a0) > 0:  # monotone: moves by at most the difference behind
                assert abs(v - a0) <= abs(a0 - back) * (1 + 1e-15), (back, a0, face, v)


def test_jumps_and_flat_runs():
    # a flat run behind the cell (t = 0): no change toward the jump
    assert oracle.limo3_face(1.0, 1.0, 5.0) == 1.0
    assert oracle.limo3_face(5.0, 5.0, 1.0) == 5.0
    # a flat run toward the face (t infinite): the cell value
    assert oracle.limo3_face(0.0, 1.0, 1.0) == 1.0
    # beyond a jump of the opposite sign twice as large (t <= -2): the cell value
    assert oracle.limo3_face(0.0, 2.0, 1.0) == 2.0
    assert oracle.limo3_face(-3.0, 2.0, 1.0) == 2.0


def lw_error(ic, recon, rk, cfl=0.4):
    """Eq. (14) error of one crossing time (the measure of the linear-wave tests)."""
    sim = oracle.Sim.from_prims(ic.prim, ic.lengths, ic.gamma, cfl, rk_order=rk, recon=recon)
    q0 = oracle.prims(sim.u, ic.lengths, ic.gamma)
    sim.advance(ic.meta["t_cross"])
    q1 = oracle.prims(sim.u, ic.lengths, ic.gamma)
    eps = ic.meta["eps"]
    acc, ncomp = 0.0, 0
    for f in range(8):
        if np.max(np.abs(q0[f] - np.mean(q0[f]))) < 1e-3 * eps:
            continue
        ncomp += 1
        acc += (np.sum(np.abs(q0[f] - q1[f])) / (eps * ic.ncells)) ** 2
    return math.sqrt(acc) / max(ncomp, 1)


@pytest.mark.parametrize("mode", ["fast", "alfven", "slow", "entropy"])
def test_limo3_rk3_converges_faster_than_second_order(mode):
    e64 = lw_error(inputs.linear_wave_1d(64, mode), "limo3", 3)
    e128 = lw_error(inputs.linear_wave_1d(128, mode), "limo3", 3)
    plm128 = lw_error(inputs.linear_wave_1d(128, mode), "plm", 2)
    assert math.log2(e64 / e128) > 2.05, (e64, e128)
    assert e128 < 0.6 * plm128, (e128, plm128)


def test_limo3_first_dt_and_conservation():
    # the speed pass reconstructs with LimO3 as well; a cycle conserves mass, momentum and
    # energy and keeps div B at rounding (the reconstruction feeds the same CT update)
    ic = inputs.random_smooth((6, 5, 7), seed=21)
    cons = oracle.cons_from_prims(ic.prim, ic.lengths, ic.gamma)
    inv_plm = oracle.speed_pass(cons, ic.lengths, ic.gamma, "plm")
    inv_l3 = oracle.speed_pass(cons, ic.lengths, ic.gamma, "limo3")
    assert inv_l3 != inv_plm
    sim = oracle.Sim(cons, ic.lengths, ic.gamma, 0.4, recon="limo3", rk_order=3)
    assert sim.inv_dt == inv_l3
    tot0 = [float(np.sum(sim.u[f])) for f in range(5)]
    for _ in range(3):
        sim.step()
    for f in range(5):
        assert abs(float(np.sum(sim.u[f])) - tot0[f]) <= 1e-12 * max(1.0, abs(tot0[f]))
    nz, ny, nx = ic.shape
    dx, dy, dz = ic.lengths[0] / nx, ic.lengths[1] / ny, ic.lengths[2] / nz
    bx, by, bz = sim.u[5], sim.u[6], sim.u[7]
    div = ((np.roll(bx, -1, 2) - bx) / dx + (np.roll(by, -1, 1) - by) / dy +
           (np.roll(bz, -1, 0) - bz) / dz)
    assert float(np.max(np.abs(div))) < 1e-11


def test_scheme_entry_points_keep_plm_bitwise_and_reject_bad_codes():
    # every oracle cycle now goes through ora_cycle_scheme; with recon = PLM it must give
    # the bits of the solver/RK entry point it replaced, and unknown codes are refused
    import ctypes
    ic = inputs.random_smooth((6, 5, 7), seed=3)
    cons = oracle.cons_from_prims(ic.prim, ic.lengths, ic.gamma)
    L = oracle.lib()
    g = ctypes.byref(oracle._grid(cons[0].shape, ic.lengths))
    for solver, rk in (("hlld", 2), ("hll", 3), ("rusanov", 2)):
        a = [c.copy() for c in cons]
        b = [c.copy() for c in cons]
        inv0 = oracle.speed_pass(cons, ic.lengths, ic.gamma)
        ia, ib = ctypes.c_double(inv0), ctypes.c_double(inv0)
        da, db = ctypes.c_double(), ctypes.c_double()
        bad = ctypes.c_long(-1)
        assert L.ora_cycle_rk(g, ic.gamma, 0.4, oracle.SOLVERS[solver], rk, oracle._ptrs(a),
                              ctypes.byref(ia), 1e9, ctypes.byref(da), ctypes.byref(bad)) == 0
        assert L.ora_cycle_scheme(g, ic.gamma, 0.4, 1, oracle.SOLVERS[solver], rk,
                                  oracle._ptrs(b), None, None, ctypes.byref(ib), 1e9,
                                  ctypes.byref(db), ctypes.byref(bad)) == 0
        assert da.value == db.value and ia.value == ib.value
        for f in range(8):
            assert np.array_equal(a[f], b[f])
    u = [c.copy() for c in cons]
    inv = ctypes.c_double(1.0)
    dt = ctypes.c_double()
    bad = ctypes.c_long(-1)
    for recon in (0, 2, 4):
        assert L.ora_cycle_scheme(g, ic.gamma, 0.4, recon, 4, 2, oracle._ptrs(u), None, None,
                                  ctypes.byref(inv), 1e9, ctypes.byref(dt),
                                  ctypes.byref(bad)) == oracle.EINVAL
        assert L.ora_speed_pass_recon(g, ic.gamma, recon, oracle._ptrs(u), ctypes.byref(inv),
                                      ctypes.byref(bad)) == oracle.EINVAL
