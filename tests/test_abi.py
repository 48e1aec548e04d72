"""The C-ABI library loads on the CPU, exports every entry point include/idx.h declares,
and rejects invalid arguments before touching the GPU (no compute call is made here)."""
import ctypes
import os
import re

import pytest

from paper_2304_13746_b300 import build as idx_build
from paper_2304_13746_b300 import idx

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "idx.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(idx_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def L():
    idx_build.build()
    return idx.lib()


def test_every_declared_symbol_is_exported(L):
    names = declared_symbols()
    assert len(names) >= 12
    for n in names:
        assert hasattr(L, n), n


def test_strerror_covers_codes(L):
    for code in (0, -1, -2, -3, -4, -5):
        assert idx.strerror(code) not in ("", "unknown error")
    assert idx.strerror(-99) == "unknown error"


def _create(L, grid, gamma=5 / 3, solver=None):
    s = solver or idx.Solver(1, 4, 2, 2, 0.4, 0)
    h = ctypes.c_void_p()
    rc = L.idx_create(ctypes.byref(grid) if grid is not None else None, gamma,
                      ctypes.byref(s), None, ctypes.byref(h))
    return rc, h


@pytest.mark.parametrize("grid,gamma,solver", [
    (idx.Grid(0, 4, 4, 1, 1, 1), 5 / 3, None),
    (idx.Grid(4, 4, 4, 1, -1, 1), 5 / 3, None),
    (idx.Grid(4, 4, 4, 1, 1, 1), 1.0, None),
    (idx.Grid(4, 4, 4, 1, 1, 1), float("nan"), None),
    (idx.Grid(2048, 2048, 1024, 1, 1, 1), 5 / 3, None),           # >= 2^31 cells
    (idx.Grid(4, 4, 4, 1, 1, 1), 5 / 3, idx.Solver(2, 4, 2, 2, 0.4, 0)),  # recon
    (idx.Grid(4, 4, 4, 1, 1, 1), 5 / 3, idx.Solver(1, 3, 2, 2, 0.4, 0)),  # riemann
    (idx.Grid(4, 4, 4, 1, 1, 1), 5 / 3, idx.Solver(1, 0, 2, 2, 0.4, 0)),  # riemann
    (idx.Grid(4, 4, 4, 1, 1, 1), 5 / 3, idx.Solver(1, 4, 1, 2, 0.4, 0)),  # emf
    (idx.Grid(4, 4, 4, 1, 1, 1), 5 / 3, idx.Solver(1, 4, 2, 4, 0.4, 0)),  # rk order
    (idx.Grid(4, 4, 4, 1, 1, 1), 5 / 3, idx.Solver(1, 4, 2, 2, 1.0, 0)),  # cfl
    (idx.Grid(4, 4, 4, 1, 1, 1), 5 / 3, idx.Solver(1, 4, 2, 2, 0.4, 7)),  # precision
    (idx.Grid(4, 4, 4, 1, 1, 1), 5 / 3, idx.Solver(1, 4, 2, 2, 0.4, 0, 2)),  # induction
    (idx.Grid(4, 4, 4, 1, 1, 1, (ctypes.c_int * 3)(3, 0, 0)), 5 / 3, None),   # boundary kind
    (idx.Grid(4, 4, 4, 1, 1, 1, (ctypes.c_int * 3)(0, 1, 0)), 5 / 3,
     idx.Solver(1, 4, 2, 2, 0.4, 0, 1)),                                      # potential + walls
])
def test_create_rejects_invalid_arguments(L, grid, gamma, solver):
    rc, h = _create(L, grid, gamma, solver)
    assert rc == idx.IDX_EINVAL and not h.value


def test_null_arguments(L):
    assert L.idx_create(None, 5 / 3, None, None, None) == idx.IDX_EINVAL
    rc, _ = _create(L, None)
    assert rc == idx.IDX_EINVAL
    assert L.idx_step(None, None) == idx.IDX_EINVAL
    assert L.idx_advance(None, 1.0, None) == idx.IDX_EINVAL
    assert L.idx_set_state(None, idx.P8(), 0) == idx.IDX_EINVAL
    assert L.idx_pipe_rates(None) == idx.IDX_EINVAL
    b = (ctypes.c_double * 3)(0.0, 0.0, 0.0)
    assert L.idx_set_potential(None, idx.P8(), b, 0) == idx.IDX_EINVAL
    assert L.idx_get_potential(None, idx.P3(), 0) == idx.IDX_EINVAL
    L.idx_destroy(None)


@pytest.mark.parametrize("precision,rk,induction,per_cell", [
    ("fp64", 2, "field", 432), ("fp32", 2, "field", 304),
    ("fp64", 3, "field", 496), ("fp64", 2, "potential", 504),
    ("fp64", 3, "potential", 592), ("fp32", 2, "potential", 352),
])
def test_footprint_per_cell(L, precision, rk, induction, per_cell):
    # 64^3 cells: every array is a multiple of 256 B, so the count is exact bar the
    # 256-byte control block
    n = 64 ** 3
    got = idx.footprint((64, 64, 64), precision, rk_order=rk, induction=induction)
    assert got == per_cell * n + 256
    if rk == 2 and induction == "field":
        out = ctypes.c_uint64()
        assert L.idx_footprint(ctypes.byref(idx.Grid(64, 64, 64, 1, 1, 1)), idx.PRECISIONS[precision],
                               ctypes.byref(out)) == idx.IDX_OK
        assert out.value == got


def test_footprint_of_the_carried_primitive_stages():
    # FP32 bulk with RK2, the field form and a periodic grid keeps the stage-1 face fields
    # (3 FP64 arrays) for the carried-primitive stages; RK3 and padded grids do not
    n = 64 ** 3
    assert idx.footprint((64, 64, 64), "fp32") == 304 * n + 256
    assert idx.footprint((64, 64, 64), "fp32", rk_order=3) == 280 * n + 256 + 8 * 8 * n
    padded = 64 * 64 * 68
    assert idx.footprint((64, 64, 64), "fp32", bc=(1, 0, 0)) == 280 * padded + 256


def test_footprint_rejects_invalid_solver(L):
    out = ctypes.c_uint64()
    s = idx.Solver(1, 4, 2, 2, 0.4, 0, 5)
    assert L.idx_footprint_solver(ctypes.byref(idx.Grid(8, 8, 8, 1, 1, 1)), ctypes.byref(s),
                                  ctypes.byref(out)) == idx.IDX_EINVAL
    for recon in (0, 2, 4):  # 1 PLM and 3 LimO3 are the reconstructions
        s = idx.Solver(recon, 4, 2, 2, 0.4, 0, 0)
        assert L.idx_footprint_solver(ctypes.byref(idx.Grid(8, 8, 8, 1, 1, 1)), ctypes.byref(s),
                                      ctypes.byref(out)) == idx.IDX_EINVAL


def test_limo3_needs_no_extra_memory(L):
    for precision in ("fp64", "fp32"):
        for rk in (2, 3):
            assert idx.footprint((64, 64, 64), precision, rk_order=rk, recon="limo3") == \
                idx.footprint((64, 64, 64), precision, rk_order=rk)


def test_binding_refuses_to_run_without_library(tmp_path):
    saved = idx._lib
    idx._lib = None
    try:
        with pytest.raises(RuntimeError, match="no CPU fallback"):
            idx.lib(str(tmp_path / "missing.so"))
    finally:
        idx._lib = saved


def test_footprint_of_a_padded_grid(L):
    # two ghost cells per side along each non-periodic direction; a one-cell direction
    # takes no boundary
    base = idx.footprint((8, 16, 32))
    per_cell = (base - 256) / (8 * 16 * 32)
    got = idx.footprint((8, 16, 32), bc=("outflow", "reflecting", "periodic"))
    padded = 8 * 20 * 36
    assert got == pytest.approx(per_cell * padded + 256, rel=1e-3)
    assert idx.footprint((1, 16, 32), bc=(0, 0, 1)) == idx.footprint((1, 16, 32))


def test_clock_and_probe_reject_bad_arguments_without_a_gpu(L):
    c = idx.Clock(0.0, 1.0, 0)
    assert L.idx_get_clock(None, ctypes.byref(c)) == idx.IDX_EINVAL
    assert L.idx_set_clock(None, ctypes.byref(c)) == idx.IDX_EINVAL
    # limits are checked before any device call
    assert L.idx_probe_bounded_wait(None, 64, 0.0) == idx.IDX_EINVAL
    assert L.idx_probe_bounded_wait(None, 64, 2000.0) == idx.IDX_EINVAL
    assert L.idx_probe_bounded_wait(None, 1 << 20, 1.0) == idx.IDX_EINVAL


def test_strict_rounding_build_exports_the_same_entry_points():
    # the test build of tests/test_gpu_strict_rounding.py; loaded here by ctypes alone
    path = idx_build.build(variant="strict")
    S = ctypes.CDLL(path)
    for n in declared_symbols():
        assert hasattr(S, n), n
