"""Exact solution of the 1D Riemann problem for the Euler equations of an ideal gas.

Closed-form pin for the Sod test of Sec. 4.1.  Written from the standard exact
solver (Toro, "Riemann Solvers and Numerical Methods for Fluid Dynamics",
ch. 4): Newton iteration on f_L(p) + f_R(p) + du = 0, then sampling of the
self-similar solution.  Test infrastructure only.
"""
import math

import numpy as np


def _f_and_df(p, rho, pk, gamma):
    a = math.sqrt(gamma * pk / rho)
    if p > pk:  # shock branch
        A = 2.0 / ((gamma + 1.0) * rho)
        B = (gamma - 1.0) / (gamma + 1.0) * pk
        q = math.sqrt(A / (p + B))
        return (p - pk) * q, q * (1.0 - 0.5 * (p - pk) / (p + B))
    # rarefaction branch
    e = (gamma - 1.0) / (2.0 * gamma)
    return (2.0 * a / (gamma - 1.0) * ((p / pk) ** e - 1.0),
            (1.0 / (rho * a)) * (p / pk) ** (-(gamma + 1.0) / (2.0 * gamma)))


def star_state(rhoL, uL, pL, rhoR, uR, pR, gamma):
    """(p*, u*) by Newton iteration from the two-rarefaction guess."""
    aL, aR = math.sqrt(gamma * pL / rhoL), math.sqrt(gamma * pR / rhoR)
    e = (gamma - 1.0) / (2.0 * gamma)
    p = ((aL + aR - 0.5 * (gamma - 1.0) * (uR - uL)) / (aL / pL ** e + aR / pR ** e)) ** (1.0 / e)
    for _ in range(100):
        fL, dL = _f_and_df(p, rhoL, pL, gamma)
        fR, dR = _f_and_df(p, rhoR, pR, gamma)
        pn = max(p - (fL + fR + (uR - uL)) / (dL + dR), 1e-14)
        done = abs(pn - p) <= 1e-15 * (pn + p)
        p = pn
        if done:
            break
    fL, _ = _f_and_df(p, rhoL, pL, gamma)
    fR, _ = _f_and_df(p, rhoR, pR, gamma)
    return p, 0.5 * (uL + uR) + 0.5 * (fR - fL)


def sample(xi, rhoL, uL, pL, rhoR, uR, pR, gamma):
    """(rho, u, p) at similarity coordinate xi = x / t (arrays allowed)."""
    ps, us = star_state(rhoL, uL, pL, rhoR, uR, pR, gamma)
    g = gamma
    xi = np.asarray(xi, dtype=float)
    rho = np.empty_like(xi); u = np.empty_like(xi); p = np.empty_like(xi)
    aL, aR = math.sqrt(g * pL / rhoL), math.sqrt(g * pR / rhoR)
    for n, s in np.ndenumerate(xi):
        if s <= us:  # left of the contact
            if ps > pL:  # left shock
                SL = uL - aL * math.sqrt((g + 1) / (2 * g) * ps / pL + (g - 1) / (2 * g))
                if s <= SL:
                    r, v, pp = rhoL, uL, pL
                else:
                    r = rhoL * ((ps / pL + (g - 1) / (g + 1)) / ((g - 1) / (g + 1) * ps / pL + 1))
                    v, pp = us, ps
            else:  # left rarefaction
                head = uL - aL
                tail = us - aL * (ps / pL) ** ((g - 1) / (2 * g))
                if s <= head:
                    r, v, pp = rhoL, uL, pL
                elif s >= tail:
                    r, v, pp = rhoL * (ps / pL) ** (1 / g), us, ps
                else:
                    c = 2 / (g + 1) + (g - 1) / ((g + 1) * aL) * (uL - s)
                    r = rhoL * c ** (2 / (g - 1))
                    v = 2 / (g + 1) * (aL + (g - 1) / 2 * uL + s)
                    pp = pL * c ** (2 * g / (g - 1))
        else:  # right of the contact
            if ps > pR:  # right shock
                SR = uR + aR * math.sqrt((g + 1) / (2 * g) * ps / pR + (g - 1) / (2 * g))
                if s >= SR:
                    r, v, pp = rhoR, uR, pR
                else:
                    r = rhoR * ((ps / pR + (g - 1) / (g + 1)) / ((g - 1) / (g + 1) * ps / pR + 1))
                    v, pp = us, ps
            else:  # right rarefaction
                head = uR + aR
                tail = us + aR * (ps / pR) ** ((g - 1) / (2 * g))
                if s >= head:
                    r, v, pp = rhoR, uR, pR
                elif s <= tail:
                    r, v, pp = rhoR * (ps / pR) ** (1 / g), us, ps
                else:
                    c = 2 / (g + 1) - (g - 1) / ((g + 1) * aR) * (uR - s)
                    r = rhoR * c ** (2 / (g - 1))
                    v = 2 / (g + 1) * (-aR + (g - 1) / 2 * uR + s)
                    pp = pR * c ** (2 * g / (g - 1))
        rho[n], u[n], p[n] = r, v, pp
    return rho, u, p
