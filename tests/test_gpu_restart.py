"""Restart from a dump (paper Sec. 3.3) and the bounded device wait, on the GPU.

A dump of a run is its 8 fields (idx_get_state) and its clock (idx_get_clock: t, the
inverse CFL time carried from the last cycle -- Eq. 10 takes the next dt from it -- and
the cycle count).  Stopping, dumping, starting a new sim from the dump and continuing
must give the uninterrupted run bit for bit.  Every device wait of the library is
bounded; idx_probe_bounded_wait runs that wait in a block whose copy never arrives, which
must end with IDX_ETIMEOUT and leave the device usable.
"""
import numpy as np
import pytest

import oracle
from paper_2304_13746_b300 import build as idx_build
from paper_2304_13746_b300 import idx, inputs

pytestmark = pytest.mark.gpu

CASES = {
    "turb_32cube": lambda: inputs.turbulent_box(32, seed=2),      # tuned sweep shapes
    "ot2d_64": lambda: inputs.orszag_tang_2d(64),                 # small-grid launches
    "smooth_24x20x16": lambda: inputs.random_smooth((16, 20, 24), seed=6),
}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    idx_build.build()
    idx.lib()


def _sim(ic, **kw):
    s = idx.Sim(ic.shape, ic.lengths, ic.gamma, 0.4, **kw)
    s.set_primitive(ic.prim)
    return s


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_restart_continues_bit_for_bit(name, precision):
    ic = CASES[name]()
    whole = _sim(ic, precision=precision)
    for _ in range(40):
        whole.step()
    want = whole.get_state()
    want_clock = whole.get_clock()
    whole.close()

    first = _sim(ic, precision=precision)
    for _ in range(17):
        first.step()
    dump = first.get_state()
    clock = first.get_clock()
    first.close()
    assert clock[2] == 17 and clock[0] > 0 and clock[1] > 0

    second = idx.Sim(ic.shape, ic.lengths, ic.gamma, 0.4, precision)
    second.set_state(dump)
    assert second.get_clock()[2] == 0          # a new state starts a new clock ...
    second.set_clock(clock)                    # ... which the dump's replaces
    assert second.get_clock() == clock
    for _ in range(40 - 17):
        second.step()
    got = second.get_state()
    assert second.get_clock() == want_clock
    second.close()
    for f in range(8):
        assert np.array_equal(got[f], want[f]), f


def test_restart_inside_an_advance_and_against_the_oracle():
    # a stop at t = 0.025 clamps the dt that reaches it, so the run without a restart
    # makes the same stop
    ic = inputs.orszag_tang_2d(48)
    o = oracle.Sim.from_prims(ic.prim, ic.lengths, ic.gamma, 0.4)
    n_o = o.advance(0.025) + o.advance(0.06)
    whole = _sim(ic)
    n_w = whole.advance(0.025) + whole.advance(0.06)
    want = whole.get_state()
    whole.close()
    a = _sim(ic)
    n_a = a.advance(0.025)
    dump, clock = a.get_state(), a.get_clock()
    a.close()
    b = idx.Sim(ic.shape, ic.lengths, ic.gamma, 0.4)
    b.set_state(dump)
    b.set_clock(clock)
    n_b = b.advance(0.06)                       # the end time is absolute
    assert n_a + n_b == n_w == n_o
    assert b.time()[0] == 0.06
    got = b.get_state()
    for f in range(8):
        assert np.array_equal(got[f], want[f]), f
    scale = [max(float(np.max(np.abs(x))), 1e-300) for x in o.u]
    assert max(float(np.max(np.abs(got[f] - o.u[f]))) / scale[f] for f in range(8)) <= 1e-10
    b.close()


def test_set_clock_rejects_invalid_clocks():
    ic = inputs.random_smooth((4, 5, 6), seed=3)
    s = _sim(ic)
    good = s.get_clock()
    for bad in [(float("nan"), good[1], 0), (0.1, 0.0, 0), (0.1, -1.0, 0),
                (0.1, float("inf"), 0), (0.1, good[1], -1)]:
        with pytest.raises(idx.IdxError) as e:
            s.set_clock(bad)
        assert e.value.code == idx.IDX_EINVAL
    assert s.get_clock() == good
    s.close()


def test_bounded_wait_expires_with_etimeout_and_the_device_stays_usable():
    import torch
    # nothing announced: the barrier completes, no timeout
    assert idx.probe_bounded_wait(0, 1.0) == idx.IDX_OK
    # bytes announced, no copy issued: the bounded wait gives up after ~1 ms
    assert idx.probe_bounded_wait(4096, 1.0) == idx.IDX_ETIMEOUT
    side = torch.cuda.Stream()
    assert idx.probe_bounded_wait(7 * 20 * 32 * 8, 2.0, stream=side.cuda_stream) == idx.IDX_ETIMEOUT
    assert idx.probe_bounded_wait(0, 2.0, stream=side.cuda_stream) == idx.IDX_OK
    # the context is intact: a cycle afterwards still matches the oracle
    ic = inputs.turbulent_box(32, seed=7)
    o = oracle.Sim.from_prims(ic.prim, ic.lengths, ic.gamma, 0.4)
    s = _sim(ic)
    o.step()
    s.step()
    g = s.get_state()
    scale = [max(float(np.max(np.abs(x))), 1e-300) for x in o.u]
    # B_y, B_z start at 0 here: held to the field-energy bound like the parity tests
    bsc = float(np.max(np.sqrt(2.0 * np.abs(o.u[4]))))
    for f in (5, 6, 7):
        scale[f] = max(scale[f], bsc)
    assert max(float(np.max(np.abs(g[f] - o.u[f]))) / scale[f] for f in range(8)) <= 1e-12
    s.close()
