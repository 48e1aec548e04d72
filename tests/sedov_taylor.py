"""Sedov-Taylor point explosion: the self-similar solution of the 3D Euler equations for a
strong spherical shock in a uniform gas at rest (Sedov 1959; Taylor 1950).

With R(t) = xi0 (E t^2 / rho0)^(1/5), xi = r / R and a = 2/5, write
    v = a (r/t) V(xi),   rho = rho0 G(xi),   p = rho0 (a R / t)^2 Q(xi).
Substituting these into mass, momentum and entropy conservation gives, with g = ln G,
    xi (V-1) g' + xi V'                          = -3 V
    G xi^2 (V-1) V' + Q'                         = G xi (V - a V^2) / a
    a xi (V-1) (Q'/Q - gamma g')                 = 2 (1 - a)
Strong-shock jump conditions at xi = 1: G = (gamma+1)/(gamma-1), V = Q = 2/(gamma+1).
Energy E = 4 pi rho0 a^2 R^5 / t^2 * I,  I = int_0^1 (xi^4 G V^2 / 2 + xi^2 Q / (gamma-1)) dxi,
so xi0 = (4 pi a^2 I)^(-1/5).  Written from the conservation laws, not from tables.
"""
import math

import numpy as np
from scipy.integrate import solve_ivp


def xi0(gamma, xi_min=1e-3):
    a = 0.4

    def rhs(xi, y):
        lg, V, Q, _ = y
        G = math.exp(lg)
        A = np.array([[xi * (V - 1), xi, 0.0],
                      [0.0, G * xi * xi * (V - 1), 1.0],
                      [-a * xi * (V - 1) * gamma, 0.0, a * xi * (V - 1) / Q]])
        b = np.array([-3 * V, G * xi * (V - a * V * V) / a, 2 * (1 - a)])
        dlg, dV, dQ = np.linalg.solve(A, b)
        return [dlg, dV, dQ, -(xi ** 4 * G * V * V / 2 + xi ** 2 * Q / (gamma - 1))]

    y0 = [math.log((gamma + 1) / (gamma - 1)), 2 / (gamma + 1), 2 / (gamma + 1), 0.0]
    sol = solve_ivp(rhs, [1.0, xi_min], y0, rtol=1e-10, atol=1e-13, max_step=0.05)
    assert sol.status == 0
    return (4 * math.pi * a * a * sol.y[3, -1]) ** -0.2


def shock_radius(E, rho0, t, gamma):
    return xi0(gamma) * (E * t * t / rho0) ** 0.2


def density_peak_radius(rho, centre=(0.5, 0.5, 0.5), nbins=None):
    """Radius of the peak of the shell-averaged density of a cubic box of unit side:
    cells binned by centre radius, peak located by a parabola through the top 3 bins."""
    n = rho.shape[0]
    h = 1.0 / n
    c = (np.arange(n) + 0.5) * h
    Z, Y, X = np.meshgrid(c, c, c, indexing="ij")
    r = np.sqrt((X - centre[0]) ** 2 + (Y - centre[1]) ** 2 + (Z - centre[2]) ** 2)
    nbins = nbins or n // 2
    edges = np.linspace(0.0, 0.5, nbins + 1)
    idx = np.digitize(r.ravel(), edges) - 1
    ok = (idx >= 0) & (idx < nbins)
    s = np.bincount(idx[ok], weights=rho.ravel()[ok], minlength=nbins)
    k = np.bincount(idx[ok], minlength=nbins)
    prof = s / np.maximum(k, 1)
    mid = 0.5 * (edges[1:] + edges[:-1])
    j = int(np.argmax(prof[1:-1])) + 1
    y0, y1, y2 = prof[j - 1], prof[j], prof[j + 1]
    den = y0 - 2 * y1 + y2
    off = 0.5 * (y0 - y2) / den if den != 0 else 0.0
    return mid[j] + off * (edges[1] - edges[0])
