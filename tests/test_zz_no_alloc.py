"""The allocation-free entry point idx_step_noalloc against the allocating one (idx_step).

idx_step_noalloc serves callers that cannot allocate device memory (another framework's
pool, a device budget, a latency-bound path): its scratch is a fixed device array in
the library.  Two calls in a row on caller-owned device state must match two idx_step
cycles of a sim made from the same state, within the parity bound used for the GPU
path (1e-12 of each field's scale), including the carried inverse CFL time -- also for a
2D grid right after a 3D one, a non-cubic grid and a side stream, with the device's free
memory and torch's allocations unchanged across calls; a grid above IDX_NOALLOC_MAX_CELLS
and a capturing stream must be refused.  The same calls also match the oracle's own cycles
directly.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2304_13746_b300 import build as idx_build
from paper_2304_13746_b300 import idx, inputs

pytestmark = pytest.mark.gpu

IDX_ETOOLARGE = -6
MAX_CELLS = 195072


def _lib():
    idx_build.build()
    L = idx.lib()
    L.idx_step_noalloc.argtypes = [ctypes.POINTER(idx.Grid), ctypes.c_double, ctypes.c_double,
                                   idx.P8, ctypes.POINTER(ctypes.c_double),
                                   ctypes.POINTER(ctypes.c_double), ctypes.c_void_p]
    return L


def _scales(o):
    rho, E = np.abs(o[0]), np.abs(o[4])
    msc = float(np.max(np.sqrt(2.0 * rho * E)))
    bsc = float(np.max(np.sqrt(2.0 * E)))
    own = [float(np.max(np.abs(o[f]))) for f in range(8)]
    return [own[0], max(own[1], msc), max(own[2], msc), max(own[3], msc), own[4],
            max(own[5], bsc), max(own[6], bsc), max(own[7], bsc)]


def test_noalloc_two_cycles_match_idx_step():
    import torch
    L = _lib()
    ic = inputs.turbulent_box(40, seed=11)          # 64000 cells, below the limit
    cons = oracle.cons_from_prims(ic.prim, ic.lengths, ic.gamma)
    nz, ny, nx = ic.shape
    grid = idx.Grid(nx, ny, nz, *ic.lengths)

    ref = idx.Sim(ic.shape, ic.lengths, ic.gamma, 0.4)
    ref.set_state(cons)
    state = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in cons]
    torch.cuda.synchronize()
    ptrs = idx.P8(*[t.data_ptr() for t in state])
    inv = ctypes.c_double(0.0)
    for call in range(2):
        dt_ref = ref.step(want_dt=True)
        want = ref.get_state()
        dt = ctypes.c_double()
        rc = L.idx_step_noalloc(ctypes.byref(grid), ic.gamma, 0.4, ptrs, ctypes.byref(inv),
                                ctypes.byref(dt), None)
        assert rc == idx.IDX_OK, rc
        got = [t.cpu().numpy() for t in state]
        sc = _scales(want)
        err = max(float(np.max(np.abs(got[f] - want[f]))) / sc[f] for f in range(8))
        assert err <= 1e-12, (call, err)
        assert dt.value == pytest.approx(dt_ref, rel=1e-14)
        assert ref.time()[1] == pytest.approx(0.4 / inv.value, rel=1e-14)
    ref.close()


def _noalloc_cycles(L, ic, ncycles, stream=None):
    """ncycles calls of idx_step_noalloc on device copies of ic's state against idx_step;
    returns the worst field error and asserts dt and the carried bound each call."""
    import torch
    cons = oracle.cons_from_prims(ic.prim, ic.lengths, ic.gamma)
    nz, ny, nx = ic.shape
    grid = idx.Grid(nx, ny, nz, *ic.lengths)
    ref = idx.Sim(ic.shape, ic.lengths, ic.gamma, 0.4)
    ref.set_state(cons)
    state = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in cons]
    torch.cuda.synchronize()
    ptrs = idx.P8(*[t.data_ptr() for t in state])
    inv = ctypes.c_double(0.0)
    worst = 0.0
    free_before = alloc_before = None
    for call in range(ncycles):
        dt_ref = ref.step(want_dt=True)
        want = ref.get_state()
        torch.cuda.synchronize()
        if call == 1:
            # from the second call on, nothing new may appear on the device
            free_before = torch.cuda.mem_get_info()[0]
            alloc_before = torch.cuda.memory_allocated()
        dt = ctypes.c_double()
        rc = L.idx_step_noalloc(ctypes.byref(grid), ic.gamma, 0.4, ptrs, ctypes.byref(inv),
                                ctypes.byref(dt), stream)
        assert rc == idx.IDX_OK, rc
        got = [t.cpu().numpy() for t in state]
        sc = _scales(want)
        err = max(float(np.max(np.abs(got[f] - want[f]))) / sc[f] for f in range(8))
        assert err <= 1e-12, (call, err)
        worst = max(worst, err)
        assert dt.value == pytest.approx(dt_ref, rel=1e-14)
        assert ref.time()[1] == pytest.approx(0.4 / inv.value, rel=1e-14)
    torch.cuda.synchronize()
    if free_before is not None:
        assert torch.cuda.mem_get_info()[0] == free_before
        assert torch.cuda.memory_allocated() == alloc_before
    ref.close()
    return worst


def test_noalloc_cycles_match_the_oracle():
    # the same calls against the oracle's own cycles (no path shared with idx_step): a 2D
    # and a non-cubic 3D grid, two cycles each, state within the parity bound and each dt
    # and carried inverse CFL time to rounding
    import torch
    L = _lib()
    cases = (inputs.orszag_tang_2d(32),
             inputs.random_smooth((12, 10, 8), seed=3, lengths=(1.0, 0.9, 0.7)))
    for ic in cases:
        o = oracle.Sim.from_prims(ic.prim, ic.lengths, ic.gamma, 0.4)
        cons = oracle.cons_from_prims(ic.prim, ic.lengths, ic.gamma)
        nz, ny, nx = ic.shape
        grid = idx.Grid(nx, ny, nz, *ic.lengths)
        state = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in cons]
        torch.cuda.synchronize()
        ptrs = idx.P8(*[t.data_ptr() for t in state])
        inv = ctypes.c_double(0.0)
        for call in range(2):
            dt_o = o.step()
            dt = ctypes.c_double()
            rc = L.idx_step_noalloc(ctypes.byref(grid), ic.gamma, 0.4, ptrs, ctypes.byref(inv),
                                    ctypes.byref(dt), None)
            assert rc == idx.IDX_OK, rc
            got = [t.cpu().numpy() for t in state]
            want = [np.asarray(a) for a in o.u]
            sc = _scales(want)
            err = max(float(np.max(np.abs(got[f] - want[f]))) / sc[f] for f in range(8))
            print(ic.name, call, f"noalloc vs oracle {err:.2e}")
            assert err <= 1e-12, (ic.name, call, err)
            assert dt.value == pytest.approx(dt_o, rel=1e-14)
            assert 0.4 / inv.value == pytest.approx(o.next_dt(), rel=1e-14)


def test_noalloc_after_a_3d_call_runs_2d_non_cubic_and_side_stream_grids():
    # the shared array keeps the previous call's contents: a 2D grid right after a 3D one
    # (its inactive direction's arrays hold 3D leftovers), a non-cubic grid, and calls on
    # a side stream must each match idx_step
    import torch
    L = _lib()
    _noalloc_cycles(L, inputs.turbulent_box(40, seed=11), 2)
    _noalloc_cycles(L, inputs.orszag_tang_2d(64), 3)
    _noalloc_cycles(L, inputs.random_smooth((20, 24, 28), seed=8, lengths=(1.0, 0.9, 0.7)), 3)
    side = torch.cuda.Stream()
    _noalloc_cycles(L, inputs.turbulent_box(32, seed=12), 3, stream=side.cuda_stream)


def test_noalloc_refuses_a_capturing_stream():
    import torch
    L = _lib()
    ic = inputs.random_smooth((8, 8, 8), seed=2)
    nz, ny, nx = ic.shape
    grid = idx.Grid(nx, ny, nz, *ic.lengths)
    inv = ctypes.c_double(0.0)
    dummy = idx.P8(*([1] * 8))                       # never dereferenced: refused first
    side = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(side):
        with torch.cuda.graph(g, stream=side):
            rc = L.idx_step_noalloc(ctypes.byref(grid), ic.gamma, 0.4, dummy, ctypes.byref(inv),
                                    None, ctypes.c_void_p(side.cuda_stream))
            torch.zeros(1, device="cuda")          # something for the graph to hold
    assert rc == idx.IDX_EINVAL
    assert inv.value == 0.0


def test_noalloc_refuses_grids_above_its_limit():
    L = _lib()
    grid = idx.Grid(64, 64, 64, 1.0, 1.0, 1.0)      # 262144 > limit
    assert 64 ** 3 > MAX_CELLS
    inv = ctypes.c_double(0.0)
    dummy = idx.P8(*([1] * 8))                       # never dereferenced: refused first
    rc = L.idx_step_noalloc(ctypes.byref(grid), 5 / 3, 0.4, dummy, ctypes.byref(inv), None, None)
    assert rc == IDX_ETOOLARGE
