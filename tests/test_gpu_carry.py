"""The carried-primitive FP32-bulk stages against the oracle and the split kernels (GPU).

With FP32 bulk, RK2, the field form and a periodic grid, each stage's update also recovers
the primitives of the state it forms (k_update_carry), so the stages run no primitive-
recovery kernel of their own, and the RK2 combine is carried as the half sum
S = (U^n + U*)/2 (Eq. 9 regrouped).  That changes FP64 rounding order only, so the carried
stages must meet the FP32-bulk bar against the FP64 oracle and agree with the split
kernels to FP32 rounding.  The grids cover 3D, 2D and 1D shapes, a cell count that is not
a multiple of the block size, tuned and small-grid launches, and whole runs through
idx_advance.  A state that turns non-physical must fail on the same cycle and cell as with
the split kernels, both inside a cycle and at its end (where the next cycle reports it).
The primitives stay valid across a switch of stage kernels and a spell inside a batch.
"""
import numpy as np
import pytest

import oracle
from paper_2304_13746_b300 import build as idx_build
from paper_2304_13746_b300 import idx, inputs
from test_gpu_sweeps import field_errors  # noqa: E402

pytestmark = pytest.mark.gpu

TOL_ORACLE = 1e-5    # FP32 bulk against the FP64 oracle after one cycle
TOL_SPLIT = 3e-6     # carried against split, a few cycles (FP32 rounding order)
TOL_MIX = 1e-5       # a run with cycles in a batch against one alone (as for batches)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    idx_build.build()
    idx.lib()


CASES = {
    "turb_32cube": lambda: inputs.turbulent_box(32, seed=8),           # tuned shapes
    "turb_64cube": lambda: inputs.turbulent_box(64, seed=4),           # 2^18 cells
    "smooth_12x20x28": lambda: inputs.random_smooth((12, 20, 28), seed=23,
                                                    lengths=(1.0, 0.8, 0.5)),  # 6720 cells
    "ot2d_64": lambda: inputs.orszag_tang_2d(64),                     # 2D, small grid
    "wave1d_x": lambda: inputs.linear_wave_1d(48, "alfven", eps=1e-3),  # 1D
}


def _sim(ic, mode, prim=None, **kw):
    s = idx.Sim(ic.shape, ic.lengths, ic.gamma, 0.4, "fp32", **kw)
    s.set_primitive(ic.prim if prim is None else prim)
    s.set_stage_kernels(mode)
    assert s.stage_kernels() == mode
    return s


def run(ic, mode, cycles, prim=None, **kw):
    s = _sim(ic, mode, prim, **kw)
    for _ in range(cycles):
        s.step()
    out = s.get_state()
    s.close()
    return out


@pytest.mark.parametrize("name", list(CASES))
def test_carry_one_cycle_matches_oracle(name):
    ic = CASES[name]()
    o = oracle.Sim.from_prims(ic.prim, ic.lengths, ic.gamma, 0.4)
    o.step()
    err = field_errors(run(ic, "carry", 1), o.u)
    print(name, f"carry vs oracle {max(err):.2e}")
    assert max(err) <= TOL_ORACLE, err


@pytest.mark.parametrize("name", list(CASES))
def test_carry_matches_split(name):
    ic = CASES[name]()
    a, b = run(ic, "carry", 6), run(ic, "split", 6)
    err = field_errors(a, b)
    print(name, f"carry vs split {max(err):.2e}")
    assert max(err) <= TOL_SPLIT, err


@pytest.mark.parametrize("kw", [{"recon": "limo3"}, {"riemann": "hll"}, {"riemann": "rusanov"}])
def test_carry_with_limo3_and_other_solvers(kw):
    # the carried primitives change only the update, so every reconstruction and solver of
    # the sweeps runs with them; one cycle against the oracle, five against the split kernels
    ic = inputs.turbulent_box(32, seed=12)
    o = oracle.Sim.from_prims(ic.prim, ic.lengths, ic.gamma, 0.4,
                              solver=kw.get("riemann", "hlld"),
                              recon=kw.get("recon", "plm"))
    o.step()
    assert max(field_errors(run(ic, "carry", 1, **kw), o.u)) <= TOL_ORACLE, kw
    err = field_errors(run(ic, "carry", 5, **kw), run(ic, "split", 5, **kw))
    assert max(err) <= TOL_SPLIT, (kw, err)


def test_carry_advance_matches_split_and_oracle():
    ic = inputs.orszag_tang_2d(32)
    t_end = 0.05
    out = {}
    for mode in ("carry", "split"):
        s = _sim(ic, mode)
        n = s.advance(t_end)
        assert s.time()[0] == t_end
        out[mode] = (n, s.get_state())
        s.close()
    o = oracle.Sim.from_prims(ic.prim, ic.lengths, ic.gamma, 0.4)
    n_o = o.advance(t_end)
    assert out["carry"][0] == out["split"][0] == n_o
    assert max(field_errors(out["carry"][1], out["split"][1])) <= TOL_SPLIT
    assert max(field_errors(out["carry"][1], o.u)) <= 1e-4


def _low_beta(seed, p_scale, b_scale):
    ic = inputs.random_smooth((8, 8, 16), seed=seed, amp=0.5)
    prim = [np.array(a, dtype=np.float64, copy=True) for a in ic.prim]
    prim[4] = prim[4] * p_scale
    for f in (5, 6, 7):
        prim[f] = prim[f] * b_scale
    return ic, prim


def _fail_point(ic, prim, mode, cycles=40):
    s = _sim(ic, mode, prim)
    for n in range(cycles):
        try:
            s.step(want_dt=True)
        except idx.IdxError as e:
            assert e.code == idx.IDX_ENONPHYS
            s.close()
            return n, e.cell
    s.close()
    return None


@pytest.mark.parametrize("case", [(3, 0.3, 2.0), (3, 0.3, 3.0), (3, 0.1, 2.0), (3, 0.1, 3.0)])
def test_nonphysical_state_fails_on_the_same_cycle_and_cell(case):
    # low-beta states whose pressure recovery fails after a few cycles: the split kernels
    # find it at the start of a stage, the carried stages at the end of the one before
    ic, prim = _low_beta(*case)
    a = _fail_point(ic, prim, "carry")
    b = _fail_point(ic, prim, "split")
    print(case, "carry", a, "split", b)
    assert b is not None
    assert a == b


def test_primitives_follow_mode_switches_and_batches():
    # carried cycles, split cycles, a spell as a batch work-list member (the batch steps the
    # state and leaves W behind), carried again: every switch recovers the primitives anew
    ic = inputs.turbulent_box(16, seed=5)

    def sequence(first, second):
        s = _sim(ic, first)
        for _ in range(2):
            s.step()
        s.set_stage_kernels(second)
        for _ in range(2):
            s.step()
        s.set_stage_kernels(first)
        b = idx.Batch("fp32")
        s.step()  # one more cycle alone, then 3 in the batch
        b.add(s, 1e9)
        b.step(3)
        b.poll()
        b.remove(s)
        b.close()
        for _ in range(2):
            s.step()
        assert s.step_count() == 10
        out = s.get_state()
        s.close()
        return out

    a = sequence("carry", "split")
    c = sequence("split", "carry")
    ref = run(ic, "split", 10)
    assert max(field_errors(a, ref)) <= TOL_MIX
    assert max(field_errors(c, ref)) <= TOL_MIX
    o = oracle.Sim.from_prims(ic.prim, ic.lengths, ic.gamma, 0.4)
    for _ in range(10):
        o.step()
    assert max(field_errors(a, o.u)) <= 1e-4


def test_carry_kernel_times():
    ic = inputs.turbulent_box(64, seed=9)
    s = _sim(ic, "carry")
    kt = s.kernel_times(reps=1)
    # no primitive-recovery kernel: nothing runs between its events (timer resolution only)
    assert kt["prims"] < 0.01 * kt["update"] + 0.005
    assert min(kt["sweep_x"], kt["sweep_y"], kt["sweep_z"], kt["emf"], kt["update"]) > 0
    n = s.step_count()
    assert n == 1
    s.step()
    g = s.get_state()
    assert all(np.isfinite(a).all() for a in g)
    s.close()
