"""Pins of the oracle's vector-potential induction (Sec. 2.4, Eqs. 7-8).

  * B = curl A on the faces (discrete Stokes): closed forms for single-component
    sinusoidal potentials (sign, index placement and cell size of every curl term),
    and a vanishing discrete divergence for a random potential.
  * Stepping A with -E and recomputing B = Bref + curl A is the field-form CT update
    (Eq. 6) rearranged, so both forms agree to rounding on 3D, 2D and 1D grids (the
    thin-direction rule included), for each Riemann solver and RK order.  The field
    form is itself pinned against exact solutions in test_oracle_scheme.py.
  * A uniform state with v x B != 0 has a uniform EMF E = -v x B, so A grows as
    t (v x B) while B stays exactly the mean field (the unbounded gauge growth the
    paper warns about for a constant large-scale EMF).
  * The divergence of B stays at the rounding of one curl evaluation, cycle after
    cycle, instead of accumulating.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2304_13746_b300 import inputs


def div_b(B, lengths):
    nz, ny, nx = B[0].shape
    dx, dy, dz = lengths[0] / nx, lengths[1] / ny, lengths[2] / nz
    return ((np.roll(B[0], -1, 2) - B[0]) / dx + (np.roll(B[1], -1, 1) - B[1]) / dy +
            (np.roll(B[2], -1, 0) - B[2]) / dz)


def test_curl_of_az_closed_form():
    nz, ny, nx = 3, 4, 16
    L = (2.0, 1.0, 1.0)
    dx = L[0] / nx
    a = 0.7
    xe = np.arange(nx) * dx                       # A_z sits at x_{i-1/2} = i dx
    Az = np.broadcast_to(a * np.sin(2 * math.pi * xe / L[0]), (nz, ny, nx)).copy()
    zero = np.zeros((nz, ny, nx))
    B = oracle.b_from_potential([zero, zero, Az], (0.1, -0.2, 0.3), L)
    xc = (np.arange(nx) + 0.5) * dx               # B_y sits at x_i
    By = 0.3 * 0 - 0.2 - (2 * a / dx) * np.cos(2 * math.pi * xc / L[0]) * math.sin(math.pi * dx / L[0])
    np.testing.assert_allclose(B[0], 0.1, rtol=0, atol=1e-15)
    np.testing.assert_allclose(B[1], np.broadcast_to(By, B[1].shape), rtol=0, atol=2e-14)
    np.testing.assert_allclose(B[2], 0.3, rtol=0, atol=1e-15)


def test_curl_of_ax_closed_form():
    nz, ny, nx = 4, 8, 3
    L = (1.0, 1.5, 1.0)
    dy = L[1] / ny
    a = -0.4
    ye = np.arange(ny) * dy                       # A_x sits at y_{j-1/2}
    Ax = np.broadcast_to((a * np.cos(2 * math.pi * ye / L[1]))[None, :, None], (nz, ny, nx)).copy()
    zero = np.zeros((nz, ny, nx))
    B = oracle.b_from_potential([Ax, zero, zero], (0.0, 0.0, 0.0), L)
    yc = (np.arange(ny) + 0.5) * dy
    Bz = (2 * a / dy) * np.sin(2 * math.pi * yc / L[1]) * math.sin(math.pi * dy / L[1])
    np.testing.assert_allclose(B[2], np.broadcast_to(Bz[None, :, None], B[2].shape), rtol=0,
                               atol=2e-14)
    np.testing.assert_array_equal(B[0], 0.0)
    np.testing.assert_array_equal(B[1], 0.0)   # dA_x/dz: A_x does not vary along z


def test_curl_has_no_divergence():
    ic = inputs.random_smooth((6, 7, 8), seed=5)
    A, bmean = ic.meta["A"], ic.meta["bmean"]
    B = oracle.b_from_potential(A, bmean, ic.lengths)
    scale = max(np.abs(b).max() for b in B) * 8
    assert np.abs(div_b(B, ic.lengths)).max() < 1e-13 * scale
    # the input generator's own curl of the same potential gives the same faces
    for d in range(3):
        np.testing.assert_allclose(B[d], ic.prim[5 + d], rtol=0, atol=1e-14)


def _field_vs_potential(ic, cycles, solver="hlld", rk_order=2, from_potential=False):
    if from_potential:
        prim5 = ic.prim[:5]
        f = oracle.Sim.from_potential(prim5, ic.meta["A"], ic.meta["bmean"], ic.lengths, ic.gamma,
                                      0.4, solver, rk_order, induction="field")
        p = oracle.Sim.from_potential(prim5, ic.meta["A"], ic.meta["bmean"], ic.lengths, ic.gamma,
                                      0.4, solver, rk_order, induction="potential")
    else:
        f = oracle.Sim.from_prims(ic.prim, ic.lengths, ic.gamma, 0.4, solver, rk_order)
        p = oracle.Sim.from_prims(ic.prim, ic.lengths, ic.gamma, 0.4, solver, rk_order,
                                  induction="potential")
    for _ in range(cycles):
        dt_f = f.step()
        dt_p = p.step()
        assert abs(dt_f - dt_p) <= 1e-12 * dt_f
    E = max(np.abs(f.u[4]).max(), 1e-300)
    for q in range(8):
        # momenta and fields against their energy bounds, the rest against their own scale
        scale = math.sqrt(2 * f.u[0].max() * E) if 1 <= q <= 3 else \
            (math.sqrt(2 * E) if q >= 5 else np.abs(f.u[q]).max())
        assert np.abs(f.u[q] - p.u[q]).max() <= 1e-12 * scale, q
    return f, p


@pytest.mark.parametrize("solver,rk", [("hlld", 2), ("hll", 2), ("rusanov", 3), ("hlld", 3)])
def test_potential_matches_field_form_3d(solver, rk):
    _field_vs_potential(inputs.random_smooth((8, 6, 10), seed=2), 12, solver, rk,
                        from_potential=True)


def test_potential_matches_field_form_orszag_tang_2d():
    _field_vs_potential(inputs.orszag_tang_2d(32), 30)


def test_potential_matches_field_form_turbulent_3d():
    _field_vs_potential(inputs.turbulent_box(12, seed=4), 10)


@pytest.mark.parametrize("shape", [(1, 1, 24), (1, 24, 1), (24, 1, 1), (1, 12, 10), (9, 1, 11),
                                   (10, 8, 1)])
def test_potential_matches_field_form_thin_grids(shape):
    # every thin configuration: 1D along each axis and 2D in each plane
    _field_vs_potential(inputs.random_smooth(shape, seed=7), 15, from_potential=True)


def test_uniform_emf_grows_potential_linearly():
    v, B = (0.3, -0.2, 0.1), (0.4, -0.5, 0.25)
    ic = inputs.uniform((4, 5, 6), lengths=(1.0, 1.3, 0.7), v=v, B=B)
    sim = oracle.Sim.from_prims(ic.prim, ic.lengths, ic.gamma, 0.4, induction="potential")
    b0 = [b.copy() for b in sim.u[5:]]
    t = 0.0
    for _ in range(7):
        t += sim.step()
    vxb = np.cross(v, B)
    tol = 1e-13 * t * np.linalg.norm(v) * np.linalg.norm(B)
    for e in range(3):
        np.testing.assert_allclose(sim.A[e], t * vxb[e], rtol=0, atol=tol)
        np.testing.assert_array_equal(sim.u[5 + e], b0[e])


def test_uniform_emf_thin_grid():
    # 1D along x: A_y and A_z follow t (v x B); A_x enters no face field and stays 0
    v, B = (0.3, -0.2, 0.1), (0.4, -0.5, 0.25)
    ic = inputs.uniform((1, 1, 8), v=v, B=B)
    sim = oracle.Sim.from_prims(ic.prim, ic.lengths, ic.gamma, 0.4, induction="potential")
    t = sum(sim.step() for _ in range(5))
    vxb = np.cross(v, B)
    tol = 1e-13 * t * np.linalg.norm(v) * np.linalg.norm(B)
    np.testing.assert_array_equal(sim.A[0], 0.0)
    np.testing.assert_allclose(sim.A[1], t * vxb[1], rtol=0, atol=tol)
    np.testing.assert_allclose(sim.A[2], t * vxb[2], rtol=0, atol=tol)


def test_divergence_does_not_accumulate():
    ic = inputs.random_smooth((8, 8, 8), seed=11)
    sim = oracle.Sim.from_potential(ic.prim[:5], ic.meta["A"], ic.meta["bmean"], ic.lengths,
                                    ic.gamma, 0.4)
    h = min(l / n for l, n in zip(ic.lengths, ic.shape[::-1]))
    eps = np.finfo(float).eps
    worst = 0.0
    for n in range(120):
        sim.step()
        if n % 20 == 19:
            amax = max(np.abs(a).max() for a in sim.A)
            bmax = max(np.abs(b).max() for b in sim.u[5:])
            # one curl: each face value carries a few roundings of |Bref| + 4 |A| / h
            bound = 64 * eps * (bmax + 4 * amax / h) / h
            d = np.abs(div_b(sim.u[5:], ic.lengths)).max()
            assert d <= bound, (n, d, bound)
            worst = max(worst, d / bound)
    assert worst > 0.0
