"""Batched stepping (idx_batch_*): every sim gives the same result alone and in the mix.

Each member keeps its own grid, dt (its own CFL reduction) and end time; members join
and leave between batched cycles.  The batched kernels run the same per-cell device
code as idx_step, but in other kernel instantiations (other sweep shapes, another
wrapper), where the compiler may contract different products into FMAs; so alone and
in the mix agree to rounding, not bit for bit.  The bound is the stated FP64 one for runs
of up to 100 cycles, 1e-10 of each field's scale, and for the FP32-bulk variant its own
rounding level, 1e-5; the time reached is exactly equal."""
import math

import numpy as np
import pytest

import oracle
from paper_2304_13746_b300 import build as idx_build
from paper_2304_13746_b300 import idx, inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    idx_build.build()
    idx.lib()


def mix():
    """(IC, t_end) pairs of different shapes, dimensions and lengths of run."""
    return [
        (inputs.orszag_tang_2d(64), 0.05),
        (inputs.turbulent_box(24, seed=2), 0.02),
        (inputs.random_smooth((6, 5, 7), seed=3, lengths=(1.0, 1.3, 0.7)), 0.03),
        (inputs.sod_double_tube(40, axis=1), 0.04),
        (inputs.orszag_tang_3d(16), 0.03),
        (inputs.linear_wave(8, "alfven"), 0.06),
        (inputs.turbulent_box(40, seed=7), 0.015),   # large enough to be tuned alone
        (inputs.turbulent_box(64, seed=9), 0.008),   # 2^18 cells: stepped by its own kernels
    ]


def new_sim(ic, precision):
    s = idx.Sim(ic.shape, ic.lengths, ic.gamma, 0.4, precision)
    s.set_primitive(ic.prim)
    return s


TOL = {"fp64": 1e-10, "fp32": 1e-5}


def scaled_error(got, ref):
    rho, E = np.abs(ref[0]), np.abs(ref[4])
    msc = float(np.max(np.sqrt(2.0 * rho * E)))
    bsc = float(np.max(np.sqrt(2.0 * E)))
    own = [float(np.max(np.abs(ref[f]))) for f in range(8)]
    sc = [own[0], max(own[1], msc), max(own[2], msc), max(own[3], msc), own[4],
          max(own[5], bsc), max(own[6], bsc), max(own[7], bsc)]
    return max(float(np.max(np.abs(got[f] - ref[f]))) / sc[f] for f in range(8))


def run_alone(cases, precision):
    out = []
    for ic, t_end in cases:
        s = new_sim(ic, precision)
        n = s.advance(t_end)
        out.append((s.get_state(), n, s.time()[0]))
        s.close()
    return out


def run_batch_until_done(b, sims):
    done = set()
    for _ in range(10000):
        b.step(4)
        fin, active = b.poll()
        done.update(id(s) for s in fin)
        if active == 0:
            break
    assert all(id(s) in done for s in sims)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_alone_equals_mix(precision):
    cases = mix()
    alone = run_alone(cases, precision)
    b = idx.Batch(precision)
    sims = [new_sim(ic, precision) for ic, _ in cases]
    n0 = [s.time() for s in sims]
    for s, (_, t_end) in zip(sims, cases):
        b.add(s, t_end)
    run_batch_until_done(b, sims)
    shapes = b.shapes()
    for s, (ic, t_end), (ref, n_ref, t_ref) in zip(sims, cases, alone):
        t, _ = s.time()
        assert t == t_ref == t_end
        got = s.get_state()
        err = scaled_error(got, ref)
        print(f"{precision} {ic.name}: alone vs mix max err {err:.2e}")
        assert err <= TOL[precision], (ic.name, err)
    for s in sims:
        b.remove(s)
        s.close()
    b.close()
    assert all(v != 0 for v in shapes)
    assert all(t == 0.0 for t, _ in n0)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("shapes", [(-1, 116, 116), (16, 132, 132)])
def test_staged_batch_sweeps(precision, shapes):
    # staged tiles for the members that fit them (nx % 32 == 0, n_d a multiple of the
    # tile), marching for the others, in one batched cycle
    cases = [
        (inputs.turbulent_box(32, seed=5), 0.01),             # fits 16 and 32
        (inputs.random_smooth((16, 32, 64), seed=8), 0.02),   # z fits 16 only
        (inputs.orszag_tang_2d(64), 0.03),                     # 2D: y only
        (inputs.turbulent_box(24, seed=2), 0.01),             # nx = 24: marches
        (inputs.sod_double_tube(40, axis=2), 0.03),           # 1D along z: marches
    ]
    alone = run_alone(cases, precision)
    b = idx.Batch(precision)
    b.set_shapes(shapes)
    sims = [new_sim(ic, precision) for ic, _ in cases]
    for s, (_, t_end) in zip(sims, cases):
        b.add(s, t_end)
    run_batch_until_done(b, sims)
    assert b.shapes() == list(shapes)
    for s, (ic, t_end), (ref, n_ref, t_ref) in zip(sims, cases, alone):
        assert s.time()[0] == t_ref == t_end
        err = scaled_error(s.get_state(), ref)
        print(f"{precision} {shapes} {ic.name}: alone vs staged batch {err:.2e}")
        assert err <= TOL[precision], (ic.name, err)
    for s in sims:
        b.remove(s)
        s.close()
    b.close()


def test_members_join_and_leave():
    cases = mix()
    alone = run_alone(cases, "fp64")
    b = idx.Batch("fp64")
    sims = [new_sim(ic, "fp64") for ic, _ in cases]
    # three members first, the others join after a few cycles
    for s, (_, t_end) in list(zip(sims, cases))[:3]:
        b.add(s, t_end)
    b.step(5)
    b.poll()
    for s, (_, t_end) in list(zip(sims, cases))[3:]:
        b.add(s, t_end)
    # one member leaves early and finishes alone
    b.step(3)
    b.poll()
    leaver = sims[1]
    b.remove(leaver)
    leaver.advance(cases[1][1])
    rest = [s for s in sims if s is not leaver]
    run_batch_until_done(b, rest)
    for s, (ic, t_end), (ref, _, _) in zip(sims, cases, alone):
        got = s.get_state()
        assert s.time()[0] == t_end
        err = scaled_error(got, ref)
        assert err <= TOL["fp64"], (ic.name, err)
    b.close()
    for s in sims:
        s.close()


def test_batched_result_matches_oracle():
    ic, t_end = inputs.orszag_tang_2d(32), 0.02
    o = oracle.Sim.from_prims(ic.prim, ic.lengths, ic.gamma, 0.4)
    n = o.advance(t_end)
    b = idx.Batch("fp64")
    s = new_sim(ic, "fp64")
    b.add(s, t_end)
    run_batch_until_done(b, [s])
    got = s.get_state()
    err = max(float(np.max(np.abs(got[f] - o.u[f]))) /
              max(float(np.max(np.abs(o.u[f]))), float(np.max(np.sqrt(2 * np.abs(o.u[4]))))) for f in range(8))
    assert err <= 1e-11, (err, n)
    b.close()
    s.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_solo_members_match_alone(precision):
    # members whose cycle the work-list kernels do not run (RK3, potential, LimO3) step with
    # their own kernels inside the batched cycle, next to ordinary members
    ics = [(inputs.orszag_tang_2d(32), dict(rk_order=3), 0.02),
           (inputs.random_smooth((8, 8, 8), seed=4), dict(induction="potential"), 0.02),
           (inputs.random_smooth((6, 5, 7), seed=8), dict(recon="limo3"), 0.02),
           (inputs.turbulent_box(16, seed=3), dict(), 0.02)]
    alone = []
    for ic, kw, t_end in ics:
        s = idx.Sim(ic.shape, ic.lengths, ic.gamma, 0.4, precision, **kw)
        s.set_primitive(ic.prim)
        s.advance(t_end)
        alone.append(s.get_state())
        s.close()
    b = idx.Batch(precision)
    sims = []
    for ic, kw, t_end in ics:
        s = idx.Sim(ic.shape, ic.lengths, ic.gamma, 0.4, precision, **kw)
        s.set_primitive(ic.prim)
        b.add(s, t_end)
        sims.append(s)
    run_batch_until_done(b, sims)
    for s, (ic, kw, t_end), ref in zip(sims, ics, alone):
        assert s.time()[0] == t_end
        err = scaled_error(s.get_state(), ref)
        assert err <= TOL[precision], (ic.name, kw, err)
    for s in sims:
        b.remove(s)
        s.close()
    b.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_solo_member_replaced_at_a_reused_address(precision):
    # A finished solo member (>= 2^18 cells: its own kernels, captured into the batch's
    # graph) is removed and destroyed, and a new one of the same size joins; the allocator
    # usually hands the new sim the old one's host address.  The batch must capture its
    # cycle again for the new member's buffers: each newcomer's result equals its run alone.
    n, t_end = 64, 0.004
    ref = {}
    for seed in (11, 12, 13):
        ic = inputs.turbulent_box(n, seed=seed)
        s = idx.Sim(ic.shape, ic.lengths, ic.gamma, 0.4, precision)
        s.set_primitive(ic.prim)
        s.advance(t_end)
        ref[seed] = s.get_state()
        s.close()
    small = inputs.random_smooth((8, 8, 8), seed=5)
    b = idx.Batch(precision)
    keep = idx.Sim(small.shape, small.lengths, small.gamma, 0.4, precision)
    keep.set_primitive(small.prim)
    b.add(keep, 1e9)               # a work-list member that stays throughout
    handles = []
    for seed in (11, 12, 13):
        ic = inputs.turbulent_box(n, seed=seed)
        s = idx.Sim(ic.shape, ic.lengths, ic.gamma, 0.4, precision)
        s.set_primitive(ic.prim)
        handles.append(s.handle)
        b.add(s, t_end)
        for _ in range(1000):
            b.step(4)
            fin, _ = b.poll()
            if any(f is s for f in fin):
                break
        b.remove(s)
        assert s.time()[0] == t_end
        assert scaled_error(s.get_state(), ref[seed]) <= TOL[precision]
        s.close()
    b.remove(keep)
    keep.close()
    b.close()
    print("handles", handles)
