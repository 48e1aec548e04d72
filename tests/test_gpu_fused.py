"""The fused FP32-bulk stage kernel against the oracle and against the split kernels (GPU).

The fused kernel (idx_set_stage_kernels) forms a stage's reconstruction, Riemann fluxes,
E^c edge EMFs and update of a 32 x 8 tile of cells, plane by plane, from primitives staged
in shared memory by bulk tensor copies with a 2-cell periodic halo.  Per face, edge and
cell it does the split kernels' arithmetic, so the two agree to FP32 rounding order, and
both meet the FP32-bulk bar against the FP64 oracle.  The grids put tiles at both
periodic ends in x, y and z, use one tile across a whole direction (both halos wrap into
the same tile), several z-chunks, RK3 weights (w != w0), another Riemann solver and a
padded grid with outflow and reflecting walls.
"""
import numpy as np
import pytest

import oracle
from paper_2304_13746_b300 import build as idx_build
from paper_2304_13746_b300 import idx, inputs
from test_gpu_sweeps import field_errors  # noqa: E402

pytestmark = pytest.mark.gpu

TOL_ORACLE = 1e-5    # FP32 bulk against the FP64 oracle after one cycle
TOL_SPLIT = 3e-6     # fused against split, a few cycles (FP32 rounding order)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    idx_build.build()
    idx.lib()


CASES = {
    "turb_32cube": lambda: inputs.turbulent_box(32, seed=8),
    "smooth_16x16x32": lambda: inputs.random_smooth((16, 16, 32), seed=21),   # one x tile
    "smooth_8x8x64": lambda: inputs.random_smooth((8, 8, 64), seed=22),       # one y tile
    "smooth_12x24x96": lambda: inputs.random_smooth((12, 24, 96), seed=23,
                                                    lengths=(1.0, 0.8, 0.5)),
    "ot3d_32": lambda: inputs.orszag_tang_3d(32),
}


def run(ic, mode, cycles, prim=None, **kw):
    s = idx.Sim(ic.shape, ic.lengths, ic.gamma, 0.4, "fp32", **kw)
    s.set_primitive(ic.prim if prim is None else prim)
    s.set_stage_kernels(mode)
    assert s.stage_kernels() == mode
    for _ in range(cycles):
        s.step()
    out = s.get_state()
    s.close()
    return out


@pytest.mark.parametrize("name", list(CASES))
def test_fused_one_cycle_matches_oracle(name):
    ic = CASES[name]()
    o = oracle.Sim.from_prims(ic.prim, ic.lengths, ic.gamma, 0.4)
    o.step()
    err = field_errors(run(ic, "fused", 1), o.u)
    print(name, f"fused vs oracle {max(err):.2e}")
    assert max(err) <= TOL_ORACLE, err


@pytest.mark.parametrize("name", list(CASES))
def test_fused_matches_split(name):
    ic = CASES[name]()
    a, b = run(ic, "fused", 5), run(ic, "split", 5)
    err = field_errors(a, b)
    print(name, f"fused vs split {max(err):.2e}")
    assert max(err) <= TOL_SPLIT, err


@pytest.mark.parametrize("kw", [{"rk_order": 3}, {"riemann": "hll"}, {"riemann": "rusanov"}])
def test_fused_with_rk3_and_other_solvers(kw):
    ic = inputs.random_smooth((16, 16, 32), seed=31)
    a, b = run(ic, "fused", 4, **kw), run(ic, "split", 4, **kw)
    err = field_errors(a, b)
    assert max(err) <= TOL_SPLIT, (kw, err)


def test_fused_on_a_padded_grid_with_walls():
    # x outflow, y reflecting: the padded grid is 32 x 8 x 16 and fits the tiles
    from test_gpu_boundaries import with_faces  # noqa: E402
    ic = inputs.random_smooth((16, 4, 28), seed=33)
    bc = ("outflow", "reflecting", "periodic")
    prim = with_faces(ic.prim, [idx.BC[b] for b in bc])
    a = run(ic, "fused", 4, prim=prim, bc=bc)
    b = run(ic, "split", 4, prim=prim, bc=bc)
    err = field_errors(a, b)
    assert max(err) <= TOL_SPLIT, err


def test_stage_kernel_choice():
    big = inputs.random_smooth((64, 64, 64), seed=1)
    s = idx.Sim(big.shape, big.lengths, big.gamma, 0.4, "fp32")
    assert s.stage_kernels() == "carry"          # the default for FP32 bulk, RK2, periodic
    s.set_stage_kernels("fused")
    assert s.stage_kernels() == "fused"
    s.set_stage_kernels("split")
    assert s.stage_kernels() == "split"
    s.set_stage_kernels("auto")
    assert s.stage_kernels() == "carry"
    s.close()
    small = inputs.random_smooth((32, 32, 32), seed=1)
    s = idx.Sim(small.shape, small.lengths, small.gamma, 0.4, "fp32")
    assert s.stage_kernels() == "carry"
    s.close()
    # the carried primitives need RK2, the field form and a periodic grid; FP64 stays split
    for kw in [dict(rk_order=3), dict(induction="potential"), dict(bc=("outflow", "periodic", "periodic"))]:
        s = idx.Sim((32, 8, 8), (1.0, 1.0, 1.0), 5.0 / 3.0, 0.4, "fp32", **kw)
        assert s.stage_kernels() == "split", kw
        with pytest.raises(idx.IdxError) as e:
            s.set_stage_kernels("carry")
        assert e.value.code == idx.IDX_EINVAL
        s.close()
    s = idx.Sim((32, 32, 32), (1.0, 1.0, 1.0), 5.0 / 3.0, 0.4, "fp64")
    assert s.stage_kernels() == "split"
    with pytest.raises(idx.IdxError):
        s.set_stage_kernels("carry")
    s.close()
    for shape, prec in [((32, 32, 40), "fp32"), ((32, 12, 32), "fp32"), ((1, 32, 32), "fp32"),
                        ((32, 32, 32), "fp64")]:
        s = idx.Sim(shape, (1.0, 1.0, 1.0), 5.0 / 3.0, 0.4, prec)
        with pytest.raises(idx.IdxError) as e:
            s.set_stage_kernels("fused")
        assert e.value.code == idx.IDX_EINVAL
        s.close()


def test_fused_kernel_times_and_advance():
    ic = inputs.turbulent_box(64, seed=9)
    s = idx.Sim(ic.shape, ic.lengths, ic.gamma, 0.4, "fp32")
    s.set_primitive(ic.prim)
    s.set_stage_kernels("fused")
    kt = s.kernel_times(reps=1)
    assert kt["prims"] > 0 and kt["update"] > 0
    # nothing runs between the events of the split kernels' slots (timer resolution only)
    assert max(kt["sweep_x"], kt["sweep_y"], kt["sweep_z"], kt["emf"]) < 0.01 * kt["update"] + 0.005
    t0 = s.time()[0]
    n = s.advance(t0 + 0.01)
    assert n > 0 and s.time()[0] == pytest.approx(t0 + 0.01, abs=0)
    g = s.get_state()
    assert all(np.isfinite(a).all() for a in g)
    s.close()
