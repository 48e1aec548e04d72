"""Outflow and reflecting boundaries on the GPU against the oracle (oracle/boundaries.py).

The GPU pads a non-periodic direction with two ghost cells per side and refills them
before every stage with its own kernel; the oracle does the same in numpy around its
periodic stage.  Parity bar as for the periodic path; the run lengths reach the
boundaries (reflected and outgoing waves)."""
import numpy as np
import pytest

import oracle
from oracle import boundaries as bd
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
    out = []
    for f in range(8):
        own = float(np.max(np.abs(o[f])))
        sc = own if f in (0, 4) else max(own, msc if f < 5 else bsc)
        out.append(float(np.max(np.abs(np.asarray(g[f]) - o[f]))) / max(sc, 1e-300))
    return out


def with_faces(prim, bc):
    """Periodic-layout primitives -> user layout with n + 1 normal faces along non-periodic
    directions (the extra face repeats the first)."""
    out = [np.ascontiguousarray(a) for a in prim[:5]]
    for d, ax in ((0, 2), (1, 1), (2, 0)):
        a = prim[5 + d]
        if bc[d] and a.shape[ax] > 1:
            first = np.take(a, [0], axis=ax)
            a = np.concatenate([a, first], axis=ax)
        out.append(np.ascontiguousarray(a))
    return out


def run_pair(prim, lengths, gamma, bc, cycles, precision="fp64", t_end=None, recon="plm",
             rk_order=2):
    o = oracle.SimBC(prim, lengths, gamma, 0.4, bc, rk_order=rk_order, recon=recon)
    nz, ny, nx = prim[0].shape
    s = idx.Sim((nz, ny, nx), lengths, gamma, 0.4, precision, bc=bc, recon=recon,
                rk_order=rk_order)
    s.set_primitive(prim)
    rel = 1e-12 if precision == "fp64" else 1e-5   # FP32 bulk: signal speeds in FP32
    assert s.time()[1] == pytest.approx(o.cfl / o.inv_dt, rel=rel)
    if t_end is not None:
        n_o, n_g = o.advance(t_end), s.advance(t_end)
        assert n_o == n_g
    else:
        for _ in range(cycles):
            dt = o.step()
            assert s.step(want_dt=True) == pytest.approx(dt, rel=rel)
    return o, s


def sod_part(npu, lo, hi):
    ic = inputs.sod_double_tube(npu, axis=0)
    prim = [np.ascontiguousarray(a[..., lo:hi]) for a in ic.prim]
    prim[5] = np.zeros((1, 1, hi - lo + 1))
    return prim, ic.gamma


def test_reflecting_sod():
    prim, gamma = sod_part(60, 60, 120)
    o, s = run_pair(prim, (1.0, 1.0, 1.0), gamma, (bd.REFLECTING, 0, 0), 60)
    err = field_errors(s.get_state(), o.state())
    assert max(err) <= 1e-12, err
    s.close()


def test_outflow_sod_past_the_boundary():
    prim, gamma = sod_part(60, 0, 60)
    o, s = run_pair(prim, (1.0, 1.0, 1.0), gamma, (bd.OUTFLOW, 0, 0), 0, t_end=0.35)
    err = field_errors(s.get_state(), o.state())
    assert max(err) <= 1e-11, err
    s.close()


@pytest.mark.parametrize("bc", [(bd.OUTFLOW, bd.REFLECTING, bd.PERIODIC),
                                (bd.REFLECTING, bd.PERIODIC, bd.OUTFLOW),
                                (bd.OUTFLOW, bd.OUTFLOW, bd.OUTFLOW)])
def test_mixed_boundaries_3d(bc):
    ic = inputs.random_smooth((10, 12, 14), seed=6)
    prim = with_faces(ic.prim, bc)
    o, s = run_pair(prim, ic.lengths, ic.gamma, bc, 12)
    err = field_errors(s.get_state(), o.state())
    print(bc, f"{max(err):.2e}")
    assert max(err) <= 1e-12, err
    s.close()


@pytest.mark.parametrize("rk_order", [2, 3])
def test_limo3_with_boundaries(rk_order):
    bc = (bd.OUTFLOW, bd.REFLECTING, bd.PERIODIC)
    ic = inputs.random_smooth((10, 12, 14), seed=7)
    prim = with_faces(ic.prim, bc)
    o, s = run_pair(prim, ic.lengths, ic.gamma, bc, 10, recon="limo3", rk_order=rk_order)
    err = field_errors(s.get_state(), o.state())
    print(bc, rk_order, f"{max(err):.2e}")
    assert max(err) <= 1e-12, err
    s.close()


def test_mixed_boundaries_2d_fp32():
    bc = (bd.OUTFLOW, bd.REFLECTING, bd.PERIODIC)
    ic = inputs.random_smooth((1, 24, 20), seed=8)
    prim = with_faces(ic.prim, bc)
    o, s = run_pair(prim, ic.lengths, ic.gamma, bc, 10, precision="fp32")
    err = field_errors(s.get_state(), o.state())
    assert max(err) <= 1e-5, err
    s.close()


def test_closed_box_blast_is_symmetric_and_conservative():
    ic = inputs.sedov_blast(32)
    n = 32
    prim = [a.copy() for a in ic.prim[:5]]
    prim += [np.zeros((n, n, n + 1)), np.zeros((n, n + 1, n)), np.zeros((n + 1, n, n))]
    s = idx.Sim((n, n, n), ic.lengths, ic.gamma, 0.4, "fp64", bc=("reflecting",) * 3)
    s.set_primitive(prim)
    u0 = s.get_state()
    s.advance(0.1)                      # the blast has hit the walls by now
    u = s.get_state()
    for f in (0, 4):
        assert abs(u[f].sum() - u0[f].sum()) <= 1e-12 * np.abs(u0[f]).sum(), f
    rho = u[0]
    for axes in ((0, 2, 1), (1, 0, 2), (2, 1, 0)):
        assert np.abs(rho - rho.transpose(axes)).max() <= 1e-10 * rho.max()
    s.close()


def test_bounded_member_in_a_batch_and_error_cell():
    bc = (bd.OUTFLOW, bd.REFLECTING, bd.PERIODIC)
    ic = inputs.random_smooth((6, 8, 10), seed=3)
    prim = with_faces(ic.prim, bc)
    alone = idx.Sim(ic.shape, ic.lengths, ic.gamma, 0.4, "fp64", bc=bc)
    alone.set_primitive(prim)
    alone.advance(0.02)
    ref = alone.get_state()
    s = idx.Sim(ic.shape, ic.lengths, ic.gamma, 0.4, "fp64", bc=bc)
    s.set_primitive(prim)
    b = idx.Batch("fp64")
    b.add(s, 0.02)
    for _ in range(200):
        b.step(2)
        if b.poll()[1] == 0:
            break
    assert s.time()[0] == 0.02
    assert max(field_errors(s.get_state(), ref)) <= 1e-12
    b.remove(s)
    b.close()
    # a non-physical cell is reported in the user's layout
    cons = s.get_state()
    cons[4][2, 3, 4] = -1.0
    with pytest.raises(idx.IdxError) as e:
        alone.set_state(cons)
    assert e.value.code == idx.IDX_ENONPHYS and e.value.cell == (2 * 8 + 3) * 10 + 4
    s.close()
    alone.close()
