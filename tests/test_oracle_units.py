"""Pins of the oracle's single-interface / single-edge pieces against properties the
mathematics fixes (not against a retyped copy of the same formulas).

  * van Leer limiter (Sec. 2.3): identity on linear data, zero at extrema, TVD bounds,
    reflection symmetry, homogeneity.
  * Physical flux (Eqs. 1-4): the eigenvalues of its numerical Jacobian are the MHD
    characteristic speeds u, u +- c_A, u +- c_s, u +- c_f from their closed forms; at the
    linear-wave background of Sec. 4.2 they are 0, +-1/2, +-1, +-2.
  * HLLD (Sec. 2.3, Miyoshi & Kusano 2005): consistency, upwinding, exact resolution of
    isolated contacts, tangential and rotational discontinuities, reduction to Toro's
    HLLC form at B = 0, reflection symmetry, continuity of the fan.
  * E^c EMF (Sec. 2.4, Gardiner & Stone 2005): reduction to the face EMF for 1D data,
    uniform states, tie-break at zero mass flux, symmetry under swapping the two
    transverse directions, upwind direction.
"""
import math

import numpy as np
import pytest

import oracle

G53 = 5.0 / 3.0


def rel(a, b):
    a, b = np.asarray(a, float), np.asarray(b, float)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


# ---------------------------------------------------------------- van Leer
@pytest.mark.parametrize("a,b", [(0.3, 1.7), (-2.0, 0.125), (5.0, -3.0), (1e-8, 7e-9)])
def test_vanleer_linear_data_exact(a, b):
    assert oracle.vanleer(a - b, a, a + b) == b


def test_vanleer_extremum_and_flat():
    assert oracle.vanleer(1.0, 2.0, 1.0) == 0.0
    assert oracle.vanleer(3.0, 2.0, 3.0) == 0.0
    assert oracle.vanleer(2.0, 2.0, 5.0) == 0.0
    assert oracle.vanleer(2.0, 2.0, 2.0) == 0.0


def test_vanleer_tvd_bounds_symmetry_homogeneity():
    rng = np.random.default_rng(1)
    for _ in range(2000):
        wm, w0, wp = rng.normal(size=3)
        s = oracle.vanleer(wm, w0, wp)
        dl, dr = w0 - wm, wp - w0
        # reconstructed face values stay between the neighbours (TVD)
        lo, hi = min(w0, wp), max(w0, wp)
        assert lo - 1e-15 <= w0 + 0.5 * s <= hi + 1e-15
        lo, hi = min(wm, w0), max(wm, w0)
        assert lo - 1e-15 <= w0 - 0.5 * s <= hi + 1e-15
        assert abs(s) <= 2 * min(abs(dl), abs(dr)) + 1e-15
        assert oracle.vanleer(wp, w0, wm) == pytest.approx(-s, rel=1e-15, abs=1e-300)
        assert oracle.vanleer(3 * wm, 3 * w0, 3 * wp) == pytest.approx(3 * s, rel=1e-14)


# ---------------------------------------------------------------- physical flux
def fast_slow_alfven(rho, P, bx, by, bz, gamma):
    """Closed forms of the MHD characteristic speeds (no 4 pi in the units)."""
    a2 = gamma * P / rho
    b2 = (bx * bx + by * by + bz * bz) / rho
    ca = abs(bx) / math.sqrt(rho)
    disc = math.sqrt(max((a2 + b2) ** 2 - 4 * a2 * bx * bx / rho, 0.0))
    cf = math.sqrt(0.5 * (a2 + b2 + disc))
    cs = math.sqrt(max(0.5 * (a2 + b2 - disc), 0.0))
    return cf, ca, cs


def cons_of(w, bn, gamma):
    rho, u, v, ww, P, by, bz = w
    E = P / (gamma - 1) + 0.5 * rho * (u * u + v * v + ww * ww) + 0.5 * (bn * bn + by * by + bz * bz)
    return np.array([rho, rho * u, rho * v, rho * ww, E, by, bz])


def prim_of(U, bn, gamma):
    rho, mx, my, mz, E, by, bz = U
    u, v, w = mx / rho, my / rho, mz / rho
    P = (gamma - 1) * (E - 0.5 * rho * (u * u + v * v + w * w) - 0.5 * (bn * bn + by * by + bz * bz))
    return np.array([rho, u, v, w, P, by, bz])


def flux_jacobian_eigs(w, bn, gamma, h=1e-6):
    U0 = cons_of(w, bn, gamma)
    J = np.zeros((7, 7))
    for c in range(7):
        dU = np.zeros(7)
        dU[c] = h * max(1.0, abs(U0[c]))
        Fp = oracle.phys_flux(prim_of(U0 + dU, bn, gamma), bn, gamma)
        Fm = oracle.phys_flux(prim_of(U0 - dU, bn, gamma), bn, gamma)
        J[:, c] = (Fp - Fm) / (2 * dU[c])
    return np.sort(np.real(np.linalg.eigvals(J)))


def test_phys_flux_characteristic_speeds_linear_wave_background():
    # Sec. 4.2: rho = 1, P = 3/5, B1 = 1, B2 = 3/2 -> c_f = 2, c_A = 1, c_s = 1/2
    w = [1.0, 0.0, 0.0, 0.0, 0.6, 1.5, 0.0]
    eig = flux_jacobian_eigs(w, 1.0, G53)
    np.testing.assert_allclose(eig, [-2, -1, -0.5, 0, 0.5, 1, 2], atol=1e-6)
    cf, ca, cs = fast_slow_alfven(1.0, 0.6, 1.0, 1.5, 0.0, G53)
    assert cf == pytest.approx(2.0, rel=1e-14)
    assert ca == pytest.approx(1.0, rel=1e-14)
    assert cs == pytest.approx(0.5, rel=1e-14)


def test_phys_flux_characteristic_speeds_random_states():
    rng = np.random.default_rng(7)
    for _ in range(20):
        rho = rng.uniform(0.5, 2.0)
        P = rng.uniform(0.3, 2.0)
        u, v, w = rng.normal(size=3)
        bn, by, bz = rng.normal(size=3)
        eig = flux_jacobian_eigs([rho, u, v, w, P, by, bz], bn, G53)
        cf, ca, cs = fast_slow_alfven(rho, P, bn, by, bz, G53)
        want = np.sort([u - cf, u - ca, u - cs, u, u + cs, u + ca, u + cf])
        np.testing.assert_allclose(eig, want, atol=2e-6 * (1 + cf))


# ---------------------------------------------------------------- HLLD
def random_state(rng, bmag=1.0):
    return [rng.uniform(0.3, 2.0), *rng.normal(size=3), rng.uniform(0.2, 2.0),
            *(bmag * rng.normal(size=2))]


def test_hlld_consistency_equal_states():
    rng = np.random.default_rng(11)
    for _ in range(500):
        w = random_state(rng)
        bn = rng.normal()
        F, sL, sR = oracle.hlld(w, w, bn, G53)
        assert rel(F, oracle.phys_flux(w, bn, G53)) < 1e-13
        cf, _, _ = fast_slow_alfven(w[0], w[4], bn, w[5], w[6], G53)
        assert sL == pytest.approx(w[1] - cf, rel=1e-13, abs=1e-13)
        assert sR == pytest.approx(w[1] + cf, rel=1e-13, abs=1e-13)


def test_hlld_outer_speeds_linear_wave_background():
    w = [1.0, 0.0, 0.0, 0.0, 0.6, 1.5, 0.0]
    _, sL, sR = oracle.hlld(w, w, 1.0, G53)
    assert sL == pytest.approx(-2.0, rel=1e-14) and sR == pytest.approx(2.0, rel=1e-14)


def test_hlld_supersonic_upwinding_is_exact():
    rng = np.random.default_rng(3)
    for _ in range(200):
        wL, wR = random_state(rng), random_state(rng)
        wL[1] = wR[1] = 20.0
        bn = rng.normal()
        F, sL, _ = oracle.hlld(wL, wR, bn, G53)
        assert sL > 0
        assert np.array_equal(F, oracle.phys_flux(wL, bn, G53))
        wL[1] = wR[1] = -20.0
        F, _, sR = oracle.hlld(wL, wR, bn, G53)
        assert sR < 0
        assert np.array_equal(F, oracle.phys_flux(wR, bn, G53))


def test_hlld_resolves_isolated_contact():
    # density jump only, Bn != 0: an entropy wave moving with u; the exact interface
    # flux is that of the upwind state
    rng = np.random.default_rng(5)
    for u in (0.0, 0.37, -0.52):
        for _ in range(50):
            base = random_state(rng)
            base[1] = u
            wL, wR = list(base), list(base)
            wR[0] = base[0] * rng.uniform(0.2, 5.0)
            bn = rng.normal()
            F, _, _ = oracle.hlld(wL, wR, bn, G53)
            want = oracle.phys_flux(wL if u >= 0 else wR, bn, G53)
            assert rel(F, want) < 1e-12


def test_hlld_resolves_stationary_tangential_discontinuity():
    # Bn = 0, u = 0, total pressure continuous, everything else jumps
    rng = np.random.default_rng(9)
    n = 0
    for _ in range(200):
        wL, wR = random_state(rng), random_state(rng)
        wL[1] = wR[1] = 0.0
        pTL = wL[4] + 0.5 * (wL[5] ** 2 + wL[6] ** 2)
        wR[4] = pTL - 0.5 * (wR[5] ** 2 + wR[6] ** 2)
        if wR[4] <= 0.05:
            continue
        n += 1
        F, _, _ = oracle.hlld(wL, wR, 0.0, G53)
        want = np.array([0.0, pTL, 0, 0, 0, 0, 0])
        assert np.max(np.abs(F - want)) < 1e-13 * pTL
    assert n > 50


@pytest.mark.parametrize("direction", [+1, -1])
def test_hlld_resolves_isolated_rotational_discontinuity(direction):
    # An Alfven (rotational) discontinuity: |B_t| fixed, B_t rotated, v_t jumps by
    # -+ sign(Bn) dB_t / sqrt(rho); rho, u, P unchanged.  It moves at u +- c_A, so for
    # u = 0 the exact interface flux is F(U_L) (right-going) or F(U_R) (left-going).
    rng = np.random.default_rng(17)
    for _ in range(100):
        rho = rng.uniform(0.5, 2.0)
        P = rng.uniform(0.3, 2.0)
        bn = rng.choice([-1, 1]) * rng.uniform(0.4, 1.5)
        bt = rng.uniform(0.3, 1.5)
        th0, th1 = rng.uniform(0, 2 * math.pi, 2)
        BL = np.array([bt * math.cos(th0), bt * math.sin(th0)])
        BR = np.array([bt * math.cos(th1), bt * math.sin(th1)])
        vL = rng.normal(size=2)
        s = 1.0 if bn >= 0 else -1.0
        vR = vL - direction * s * (BR - BL) / math.sqrt(rho)
        wL = [rho, 0.0, vL[0], vL[1], P, BL[0], BL[1]]
        wR = [rho, 0.0, vR[0], vR[1], P, BR[0], BR[1]]
        F, _, _ = oracle.hlld(wL, wR, bn, G53)
        want = oracle.phys_flux(wL if direction > 0 else wR, bn, G53)
        assert rel(F, want) < 1e-12


def hllc_toro(wL, wR, gamma):
    """HLLC for the Euler equations in Toro's star-state form (Toro 2009, ch. 10),
    with the same outer wave speeds; an independent formula for the B = 0 limit."""
    def parts(w):
        rho, u, v, ww, P = w[:5]
        E = P / (gamma - 1) + 0.5 * rho * (u * u + v * v + ww * ww)
        U = np.array([rho, rho * u, rho * v, rho * ww, E])
        F = np.array([rho * u, rho * u * u + P, rho * u * v, rho * u * ww, (E + P) * u])
        return rho, u, v, ww, P, E, U, F, math.sqrt(gamma * P / rho)
    rL, uL, vL, wL_, PL, EL, UL, FL, cL = parts(wL)
    rR, uR, vR, wR_, PR, ER, UR, FR, cR = parts(wR)
    SL = min(uL, uR) - max(cL, cR)
    SR = max(uL, uR) + max(cL, cR)
    Ss = (PR - PL + rL * uL * (SL - uL) - rR * uR * (SR - uR)) / (rL * (SL - uL) - rR * (SR - uR))

    def ustar(r, u, v, ww, P, E, S):
        f = r * (S - u) / (S - Ss)
        return f * np.array([1.0, Ss, v, ww, E / r + (Ss - u) * (Ss + P / (r * (S - u)))])
    if SL >= 0:
        return FL
    if SR <= 0:
        return FR
    if Ss >= 0:
        return FL + SL * (ustar(rL, uL, vL, wL_, PL, EL, SL) - UL)
    return FR + SR * (ustar(rR, uR, vR, wR_, PR, ER, SR) - UR)


def test_hlld_reduces_to_toro_hllc_without_field():
    rng = np.random.default_rng(23)
    for _ in range(500):
        wL, wR = random_state(rng, bmag=0.0), random_state(rng, bmag=0.0)
        F, _, _ = oracle.hlld(wL, wR, 0.0, G53)
        assert rel(F[:5], hllc_toro(wL, wR, G53)) < 1e-12
        assert np.all(F[5:] == 0.0)
    F, _, _ = oracle.hlld([1, 0, 0, 0, 1, 0, 0], [0.125, 0, 0, 0, 0.1, 0, 0], 0.0, 1.4)
    assert rel(F[:5], hllc_toro([1, 0, 0, 0, 1], [0.125, 0, 0, 0, 0.1], 1.4)) < 1e-13


def test_hlld_reflection_symmetry():
    # x -> -x: u -> -u, Bn -> -Bn; each flux component picks up its parity
    rng = np.random.default_rng(29)
    parity = np.array([-1, 1, -1, -1, -1, -1, -1])

    def reflect(w):
        w = list(w)
        w[1] = -w[1]
        return w
    for _ in range(500):
        wL, wR = random_state(rng), random_state(rng)
        bn = rng.normal()
        F, sL, sR = oracle.hlld(wL, wR, bn, G53)
        Fm, sLm, sRm = oracle.hlld(reflect(wR), reflect(wL), -bn, G53)
        scale = max(np.max(np.abs(F)), 1.0)
        assert np.max(np.abs(Fm - parity * F)) < 1e-12 * scale
        assert sLm == pytest.approx(-sR, rel=1e-14) and sRm == pytest.approx(-sL, rel=1e-14)


def test_hlld_flux_continuous_across_wave_speeds():
    # Galilean sweep: as a uniform shift moves each wave speed across zero the flux
    # must stay continuous (the fan has no jump at x/t = S).
    rng = np.random.default_rng(31)
    wL, wR = random_state(rng), random_state(rng)
    prev = None
    jumps = []
    for U in np.linspace(-4, 4, 4001):
        a, b = list(wL), list(wR)
        a[1] += U
        b[1] += U
        F, _, _ = oracle.hlld(a, b, 0.8, G53)
        if prev is not None:
            jumps.append(np.max(np.abs(F - prev)))
        prev = F
    jumps = np.array(jumps)
    assert np.max(jumps) < 50 * np.median(jumps)


# ---------------------------------------------------------------- E^c
def test_emf_reduces_to_face_value_for_1d_data():
    rng = np.random.default_rng(41)
    for _ in range(500):
        F = rng.normal()
        Ci, Cim = rng.normal(size=2)
        Fa = rng.normal(size=2)
        Fb = rng.choice([-1.0, 0.0, 1.0], size=2) * rng.uniform(0.1, 1, 2)
        da, db = rng.uniform(0.01, 1, 2)
        E = oracle.emf_ec([F, F], [Ci, Cim], [[Ci, Ci], [Cim, Cim]], Fa, Fb, da, db)
        assert E == pytest.approx(F, rel=1e-13, abs=1e-13 * (abs(Ci) + abs(Cim)))


def test_emf_uniform_state():
    for fa in (-1.0, 0.0, 1.0):
        for fb in (-1.0, 0.0, 1.0):
            E = oracle.emf_ec([0.7, 0.7], [0.7, 0.7], [[0.7, 0.7], [0.7, 0.7]], [fa, fa],
                              [fb, fb], 0.1, 0.2)
            assert E == pytest.approx(0.7, rel=1e-15)


def test_emf_zero_mass_flux_is_mean_of_upwind_choices():
    rng = np.random.default_rng(43)
    for _ in range(200):
        X, Y = rng.normal(size=2), rng.normal(size=2)
        C = rng.normal(size=(2, 2))
        da, db = rng.uniform(0.01, 1, 2)
        Fb = rng.normal(size=2)
        e0 = oracle.emf_ec(X, Y, C, [0.0, 0.3], Fb, da, db)
        ep = oracle.emf_ec(X, Y, C, [1.0, 0.3], Fb, da, db)
        em = oracle.emf_ec(X, Y, C, [-1.0, 0.3], Fb, da, db)
        assert e0 == pytest.approx(0.5 * (ep + em), rel=1e-13, abs=1e-14)


def test_emf_swap_of_transverse_directions():
    rng = np.random.default_rng(47)
    for _ in range(200):
        X, Y = rng.normal(size=2), rng.normal(size=2)
        C = rng.normal(size=(2, 2))
        Fa, Fb = rng.normal(size=2), rng.normal(size=2)
        da, db = rng.uniform(0.01, 1, 2)
        e1 = oracle.emf_ec(X, Y, C, Fa, Fb, da, db)
        e2 = oracle.emf_ec(Y, X, C.T, Fb, Fa, db, da)
        assert e1 == pytest.approx(e2, rel=1e-13, abs=1e-14)


def test_emf_upwind_column_follows_mass_flux():
    # Perturb only the cell-centre EMF of cell (I-1, J).  It lies upstream of the
    # edge's a-face at row J when that face's mass flux is positive, and upstream of
    # the b-face at column I-1 when that face's mass flux is negative; otherwise the
    # edge must not see it.
    X, Y = [0.0, 0.0], [0.0, 0.0]
    C = [[0.0, 0.0], [1.0, 0.0]]  # C[c][r]: c = 0 -> I, 1 -> I-1; r = 0 -> J, 1 -> J-1

    def e(fa, fb):
        return oracle.emf_ec(X, Y, C, [fa, fa], [fb, fb], 1.0, 1.0)
    assert e(-1.0, +1.0) == 0.0          # downstream on both faces: invisible
    assert e(+1.0, +1.0) != 0.0          # upstream along a
    assert e(-1.0, -1.0) != 0.0          # upstream along b
    assert e(+1.0, -1.0) == pytest.approx(e(+1.0, +1.0) + e(-1.0, -1.0), rel=1e-15)
