"""Every sweep shape against the oracle and against each other (GPU).

The shapes (idx_sweep_shapes) differ only in how faces are assigned to threads and how
primitives reach the registers: marching segments loading from HBM, the warp-shuffle x
sweep, and the TMA-staged y/z tiles of 16 or 32 faces with a periodic halo copied by bulk
tensor copies.  Each must give the oracle's fluxes to the parity bar.  The grids put the
staged tiles at both periodic ends, use a single tile per pencil (both halos wrapped),
and a 2D plane.
"""
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


def field_errors(g, o):
    rho, E = np.abs(o[0]), np.abs(o[4])
    msc = float(np.max(np.sqrt(2.0 * rho * E)))
    bsc = float(np.max(np.sqrt(2.0 * E)))
    own = [float(np.max(np.abs(o[f]))) for f in range(8)]
    sc = [own[0], max(own[1], msc), max(own[2], msc), max(own[3], msc), own[4],
          max(own[5], bsc), max(own[6], bsc), max(own[7], bsc)]
    return [float(np.max(np.abs(np.asarray(g[f]) - o[f]))) / max(sc[f], 1e-300) for f in range(8)]


CASES = [
    ((32, 48, 64), (-1, 116, 132)),
    ((32, 48, 64), (16, 116, 116)),
    ((16, 16, 32), (-1, 116, 116)),   # one tile per pencil: both halos wrap
    ((64, 32, 32), (32, 132, 132)),
    ((1, 64, 32), (-1, 132, 0)),      # 2D
    ((32, 48, 64), (-2, 116, 132)),   # staged x tiles too
    ((16, 16, 32), (-2, 116, 116)),   # one x tile per row: both x halos wrap
    ((1, 64, 32), (-2, 132, 0)),
]


@pytest.mark.parametrize("shape,sweeps", CASES)
def test_staged_sweeps_match_oracle(shape, sweeps):
    ic = inputs.random_smooth(shape, seed=sum(shape))
    o = oracle.Sim.from_prims(ic.prim, ic.lengths, ic.gamma, 0.4)
    s = idx.Sim(ic.shape, ic.lengths, ic.gamma, 0.4, "fp64")
    s.set_primitive(ic.prim)
    s.set_sweep_shapes(sweeps)
    expect = [v if n > 1 else 0 for v, n in zip(sweeps, shape[::-1])]
    assert s.sweep_shapes() == expect
    for _ in range(3):
        dt_o = o.step()
        assert s.step(want_dt=True) == pytest.approx(dt_o, rel=1e-12)
    err = field_errors(s.get_state(), o.u)
    print(shape, sweeps, f"{max(err):.2e}")
    assert max(err) <= 3e-12, err
    s.close()


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-11), ("fp32", 3e-6)])
def test_staged_and_marching_agree_on_turbulent_box(precision, tol):
    ic = inputs.turbulent_box(64, seed=6)
    out = []
    for sweeps in ((16, 16, 16), (-1, 132, 132), (32, 116, 116), (-2, 116, 116)):
        s = idx.Sim(ic.shape, ic.lengths, ic.gamma, 0.4, precision)
        s.set_primitive(ic.prim)
        s.set_sweep_shapes(sweeps)
        for _ in range(5):
            s.step()
        out.append(s.get_state())
        s.close()
    for other in out[1:]:
        err = field_errors(other, out[0])
        assert max(err) <= tol, err


def test_invalid_shapes_are_refused():
    ic = inputs.random_smooth((32, 48, 64), seed=1)
    s = idx.Sim(ic.shape, ic.lengths, ic.gamma, 0.4, "fp64")
    s.set_primitive(ic.prim)
    for bad in ((116, 116, 116), (-1, -1, 16), (16, 132, 16), (7, 16, 16), (16, 16, 0),
                (16, -2, 16)):
        with pytest.raises(idx.IdxError) as e:
            s.set_sweep_shapes(bad)
        assert e.value.code == idx.IDX_EINVAL
    s.close()
    # staged tiles need nx % 32 == 0; staged x tiles also ny % 8 == 0
    ic = inputs.random_smooth((16, 16, 40), seed=2)
    s = idx.Sim(ic.shape, ic.lengths, ic.gamma, 0.4, "fp64")
    with pytest.raises(idx.IdxError):
        s.set_sweep_shapes((16, 116, 16))
    s.close()
    ic = inputs.random_smooth((16, 12, 32), seed=2)
    s = idx.Sim(ic.shape, ic.lengths, ic.gamma, 0.4, "fp64")
    with pytest.raises(idx.IdxError):
        s.set_sweep_shapes((-2, 16, 16))
    s.close()
