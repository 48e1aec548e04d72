"""Seeded synthetic inputs for the ideal-MHD stage (shared by the CUDA path and the oracle).

This module only *generates initial conditions*: primitive cell-centre fields
(rho, vx, vy, vz, P) and face-centred magnetic field (Bx on x-faces at i-1/2,
By on y-faces at j-1/2, Bz on z-faces at k-1/2).  It holds none of the method's
arithmetic: the conversion to conserved variables, and everything after it, is
done separately by each consumer.

Every generator returns an ``IC``: ``prim`` is a list of 8 float64 arrays of shape
(nz, ny, nx) in the order (rho, vx, vy, vz, P, Bx, By, Bz); ``lengths`` is the
box (lx, ly, lz); ``gamma`` the adiabatic index.

Workloads (IDEFIX paper, Sec. 4-5):
  * orszag_tang_2d   -- Sec. 4.2 "Orszag Tang vortex" (periodic unit square).
  * orszag_tang_3d   -- Sec. 5 performance problem (3D extension, unit cube).
  * turbulent_box    -- seeded random-phase solenoidal velocity, E(k) ~ k^-2 for
                        1 <= |k| <= 8, rms Mach 1, uniform B0 along x at beta = 1.
  * linear_wave      -- Sec. 4.2 "Linear MHD wave convergence": box (3, 1.5, 1.5),
                        2N x N x N, background rho = 1, P = 3/5, B1 = 1, B2 = 3/2.
  * sod_double_tube  -- Sec. 4.1 Sod tube on a periodic domain (two mirrored tubes).
  * random_smooth    -- smooth random states for parity tests.
"""
from dataclasses import dataclass, field
import math

import numpy as np


@dataclass
class IC:
    prim: list
    lengths: tuple
    gamma: float
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def shape(self):
        return self.prim[0].shape

    @property
    def ncells(self):
        return int(np.prod(self.shape))


def _centres(n, length):
    return (np.arange(n, dtype=np.float64) + 0.5) * (length / n)


def _faces(n, length):
    return np.arange(n, dtype=np.float64) * (length / n)


def _mesh(xs, ys, zs):
    """Broadcastable coordinate arrays for the (nz, ny, nx) layout."""
    return xs[None, None, :], ys[None, :, None], zs[:, None, None]


def _full(shape, value):
    return np.full(shape, value, dtype=np.float64)


def _up(a, axis):
    """Value at index + 1 along ``axis`` (periodic)."""
    return np.roll(a, -1, axis=axis)


def _curl_faces(Ax, Ay, Az, d):
    """Face B = discrete curl of an edge vector potential (Ax on x-edges at (i, j-1/2,
    k-1/2), Ay at (i-1/2, j, k-1/2), Az at (i-1/2, j-1/2, k)), periodic.  Its discrete
    divergence cancels term by term."""
    dx, dy, dz = d
    Bx = (_up(Az, 1) - Az) / dy - (_up(Ay, 0) - Ay) / dz
    By = (_up(Ax, 0) - Ax) / dz - (_up(Az, 2) - Az) / dx
    Bz = (_up(Ay, 2) - Ay) / dx - (_up(Ax, 1) - Ax) / dy
    return Bx, By, Bz


def orszag_tang_2d(n=128, gamma=5.0 / 3.0):
    """rho = 25/(36 pi), P = 5/(12 pi), v = (-sin 2pi y, sin 2pi x, 0),
    B = B0 (-sin 2pi y, sin 4pi x, 0), B0 = 1/sqrt(4 pi).  Bx depends on y only
    and By on x only, so point values at face centres are divergence-free."""
    shape = (1, n, n)
    B0 = 1.0 / math.sqrt(4.0 * math.pi)
    c = _centres(n, 1.0)
    X, Y, _ = _mesh(c, c, np.zeros(1))
    rho = _full(shape, 25.0 / (36.0 * math.pi))
    P = _full(shape, 5.0 / (12.0 * math.pi))
    vx = np.broadcast_to(-np.sin(2 * math.pi * Y), shape).copy()
    vy = np.broadcast_to(np.sin(2 * math.pi * X), shape).copy()
    vz = np.zeros(shape)
    # Bx sits on x-faces (its y coordinate is a cell centre); By on y-faces
    # (its x coordinate is a cell centre).
    Bx = np.broadcast_to(-B0 * np.sin(2 * math.pi * Y), shape).copy()
    By = np.broadcast_to(B0 * np.sin(4 * math.pi * X), shape).copy()
    Bz = np.zeros(shape)
    return IC([rho, vx, vy, vz, P, Bx, By, Bz], (1.0, 1.0, 1.0), gamma, "orszag_tang_2d",
              {"n": n})


def orszag_tang_3d(n=64, gamma=5.0 / 3.0):
    """Sec. 5 problem: v = (-sin 2pi y, sin 2pi x + cos 2pi z, cos 2pi x),
    B = B0 (-sin 2pi y, sin 4pi x, cos 2pi x + sin 2pi y).  Bx depends on y,
    By on x, Bz on (x, y): point values at face centres are divergence-free."""
    shape = (n, n, n)
    B0 = 1.0 / math.sqrt(4.0 * math.pi)
    c = _centres(n, 1.0)
    X, Y, Z = _mesh(c, c, c)
    tp = 2 * math.pi
    rho = _full(shape, 25.0 / (36.0 * math.pi))
    P = _full(shape, 5.0 / (12.0 * math.pi))
    vx = np.broadcast_to(-np.sin(tp * Y), shape).copy()
    vy = np.broadcast_to(np.sin(tp * X) + np.cos(tp * Z), shape).copy()
    vz = np.broadcast_to(np.cos(tp * X), shape).copy()
    Bx = np.broadcast_to(-B0 * np.sin(tp * Y), shape).copy()
    By = np.broadcast_to(B0 * np.sin(2 * tp * X), shape).copy()
    Bz = np.broadcast_to(B0 * (np.cos(tp * X) + np.sin(tp * Y)), shape).copy()
    return IC([rho, vx, vy, vz, P, Bx, By, Bz], (1.0, 1.0, 1.0), gamma, "orszag_tang_3d",
              {"n": n})


def _solenoidal_modes(seed, kmax=8, slope=-2.0):
    """Random-phase Fourier amplitudes a(n) (complex 3-vectors) for integer
    wavevectors 1 <= |n| <= kmax, amplitude |n|^slope, projected normal to n."""
    rng = np.random.Generator(np.random.PCG64(seed))
    r = np.arange(-kmax, kmax + 1)
    nx, ny, nz = np.meshgrid(r, r, r, indexing="ij")
    kk = np.sqrt(nx ** 2 + ny ** 2 + nz ** 2)
    mask = (kk >= 1.0) & (kk <= kmax)
    n = np.stack([nx[mask], ny[mask], nz[mask]], axis=1).astype(np.float64)
    k = kk[mask]
    vec = rng.standard_normal((n.shape[0], 3))           # isotropic random direction
    phase = rng.uniform(0.0, 2 * math.pi, n.shape[0])    # uniform random phase
    unit = n / k[:, None]
    vec = vec - unit * np.sum(vec * unit, axis=1)[:, None]  # project normal to n
    vec = vec / np.maximum(np.linalg.norm(vec, axis=1), 1e-300)[:, None]
    amp = (k ** slope)[:, None] * vec * np.exp(1j * phase)[:, None]
    return n.astype(np.int64), amp


def _synth(n_int, amp, N, comp):
    """Real part of sum_n amp[n, comp] exp(2 pi i n . x) at the cell centres of an
    N^3 unit box, by separable contraction over the small set of wavenumbers."""
    kmax = int(np.max(np.abs(n_int)))
    L = 2 * kmax + 1
    A = np.zeros((L, L, L), dtype=np.complex128)
    np.add.at(A, (n_int[:, 0] + kmax, n_int[:, 1] + kmax, n_int[:, 2] + kmax), amp[:, comp])
    x = _centres(N, 1.0)
    ph = np.exp(2j * math.pi * np.outer(np.arange(-kmax, kmax + 1), x))  # (L, N)
    t = np.einsum("abc,ax->bcx", A, ph)          # (ny-modes, nz-modes, x)
    t = np.einsum("bcx,by->cyx", t, ph)          # (nz-modes, y, x)
    out = np.empty((N, N, N), dtype=np.float64)
    for z0 in range(0, N, 64):
        z1 = min(N, z0 + 64)
        out[z0:z1] = np.real(np.einsum("cyx,cz->zyx", t, ph[:, z0:z1]))
    return out


def turbulent_box(n=64, seed=0, gamma=5.0 / 3.0, mach=1.0, kmax=8):
    """rho = 1, P = 1/gamma (sound speed 1), B = (sqrt(2P), 0, 0) so beta = 2P/B0^2 = 1;
    v solenoidal random-phase, |amplitude| ~ |n|^-2 (shell energy ~ k^-2), rms |v| = mach."""
    shape = (n, n, n)
    n_int, amp = _solenoidal_modes(seed, kmax=kmax)
    v = [_synth(n_int, amp, n, c) for c in range(3)]
    rms = math.sqrt(float(np.mean(v[0] ** 2 + v[1] ** 2 + v[2] ** 2)))
    v = [c * (mach / rms) for c in v]
    P0 = 1.0 / gamma
    B0 = math.sqrt(2.0 * P0)
    return IC([_full(shape, 1.0), v[0], v[1], v[2], _full(shape, P0), _full(shape, B0),
               np.zeros(shape), np.zeros(shape)], (1.0, 1.0, 1.0), gamma, "turbulent_box",
              {"n": n, "seed": seed, "mach": mach, "kmax": kmax})


# ---------------------------------------------------------------------------
# Linear MHD waves.  The eigenvectors come from the linearised ideal-MHD
# equations in primitive variables along the wave normal (a numerical
# eigen-decomposition of the quasi-linear matrix below).
# ---------------------------------------------------------------------------
def _prim_jacobian(rho, u, v, w, P, bx, by, bz, gamma):
    """A(W) with dW/dt + A dW/dx1 = 0 for W = (rho, u, v, w, P, By, Bz), Bx const."""
    A = np.zeros((7, 7))
    A[0, 0] = u; A[0, 1] = rho
    A[1, 1] = u; A[1, 4] = 1.0 / rho; A[1, 5] = by / rho; A[1, 6] = bz / rho
    A[2, 2] = u; A[2, 5] = -bx / rho
    A[3, 3] = u; A[3, 6] = -bx / rho
    A[4, 1] = gamma * P; A[4, 4] = u
    A[5, 1] = by; A[5, 2] = -bx; A[5, 5] = u
    A[6, 1] = bz; A[6, 3] = -bx; A[6, 6] = u
    return A


WAVE_SPEEDS = {"fast": 2.0, "alfven": 1.0, "slow": 0.5, "entropy": 1.0}


def linear_wave_eigen(mode, gamma=5.0 / 3.0):
    """Background and the right eigenvector (primitive variables) of the right-going
    ``mode`` along x1: returns (background dict, eigenvalue, vector)."""
    rho, P, b1, b2 = 1.0, 3.0 / 5.0, 1.0, 1.5
    u = 1.0 if mode == "entropy" else 0.0
    A = _prim_jacobian(rho, u, 0.0, 0.0, P, b1, b2, 0.0, gamma)
    lam, R = np.linalg.eig(A)
    lam = np.real(lam)
    R = np.real(R)
    target = {"fast": u + 2.0, "alfven": u + 1.0, "slow": u + 0.5, "entropy": u}[mode]
    idx = [i for i in range(7) if abs(lam[i] - target) < 1e-9]
    if mode == "alfven":
        i = max(idx, key=lambda q: abs(R[3, q]) + abs(R[6, q]))
    elif mode == "entropy":
        i = max(idx, key=lambda q: abs(R[0, q]) - abs(R[4, q]))
    else:
        i = int(np.argmin(np.abs(lam - target)))
    vec = R[:, i]
    vec = vec / vec[np.argmax(np.abs(vec))]
    bg = dict(rho=rho, u=u, v=0.0, w=0.0, P=P, b1=b1, b2=b2, b3=0.0)
    return bg, float(lam[i]), vec


def _plane_wave(shape, lengths, kvec, e1, e2, mode, eps, gamma):
    """Primitive fields of a small-amplitude eigenmode eps * r * sin(k.x) on the grid;
    face B = background on faces + discrete curl of a periodic edge potential."""
    nz, ny, nx = shape
    lx, ly, lz = lengths
    e3 = np.cross(e1, e2)
    bg, _, r = linear_wave_eigen(mode, gamma)
    d = (lx / nx, ly / ny, lz / nz)
    xc, yc, zc = _centres(nx, lx), _centres(ny, ly), _centres(nz, lz)
    xf, yf, zf = _faces(nx, lx), _faces(ny, ly), _faces(nz, lz)

    def phase(x, y, z):
        return kvec[0] * x + kvec[1] * y + kvec[2] * z

    X, Y, Z = _mesh(xc, yc, zc)
    s = np.sin(phase(X, Y, Z))
    dq = eps * r
    rho = np.broadcast_to(bg["rho"] + dq[0] * s, shape).copy()
    P = np.broadcast_to(bg["P"] + dq[4] * s, shape).copy()
    v1, v2, v3 = bg["u"] + dq[1] * s, dq[2] * s, dq[3] * s
    vel = [np.broadcast_to(v1 * e1[c] + v2 * e2[c] + v3 * e3[c], shape).copy() for c in range(3)]
    B0 = bg["b1"] * e1 + bg["b2"] * e2 + bg["b3"] * e3
    # dB = eps b_hat sin(k.x) = curl dA with dA = eps (k x b_hat) cos(k.x) / |k|^2
    bhat = r[5] * e2 + r[6] * e3
    avec = np.cross(kvec, bhat) / float(np.dot(kvec, kvec)) * eps
    Xf, Yf, Zf = _mesh(xf, yf, zf)
    Ax = np.broadcast_to(avec[0] * np.cos(phase(X, Yf, Zf)), shape)
    Ay = np.broadcast_to(avec[1] * np.cos(phase(Xf, Y, Zf)), shape)
    Az = np.broadcast_to(avec[2] * np.cos(phase(Xf, Yf, Z)), shape)
    dBx, dBy, dBz = _curl_faces(Ax, Ay, Az, d)
    prim = [rho, vel[0], vel[1], vel[2], P, np.ascontiguousarray(B0[0] + dBx),
            np.ascontiguousarray(B0[1] + dBy), np.ascontiguousarray(B0[2] + dBz)]
    return prim, bg, r


def linear_wave(N=16, mode="fast", eps=1e-6, gamma=5.0 / 3.0):
    """Sec. 4.2 linear-wave test: box (3, 1.5, 1.5), grid 2N x N x N, wave vector
    k = 2 pi (1/3, 2/3, 2/3) (wavelength 1, periodic in the box), eigenmode of
    amplitude eps, integrated for one crossing time of the wavelength."""
    lengths = (3.0, 1.5, 1.5)
    shape = (N, N, 2 * N)
    e1 = np.array([1.0, 2.0, 2.0]) / 3.0
    e2 = np.array([-2.0, 2.0, -1.0]) / 3.0
    kvec = 2 * math.pi * e1          # |k| = 2 pi: wavelength 1
    prim, bg, r = _plane_wave(shape, lengths, kvec, e1, e2, mode, eps, gamma)
    speed = bg["u"] if mode == "entropy" else WAVE_SPEEDS[mode]
    return IC(prim, lengths, gamma, "linear_wave",
              {"N": N, "mode": mode, "eps": eps, "eigen": r.copy(), "t_cross": 1.0 / speed})


def linear_wave_1d(N=32, mode="fast", eps=1e-6, gamma=5.0 / 3.0):
    """The same eigenmode along x on an N x 1 x 1 grid of the unit box (wavelength 1)."""
    shape = (1, 1, N)
    e1 = np.array([1.0, 0.0, 0.0])
    e2 = np.array([0.0, 1.0, 0.0])
    prim, bg, r = _plane_wave(shape, (1.0, 1.0, 1.0), 2 * math.pi * e1, e1, e2, mode, eps, gamma)
    speed = bg["u"] if mode == "entropy" else WAVE_SPEEDS[mode]
    return IC(prim, (1.0, 1.0, 1.0), gamma, "linear_wave_1d",
              {"N": N, "mode": mode, "eps": eps, "eigen": r.copy(), "t_cross": 1.0 / speed})


def sod_double_tube(n_per_unit=200, axis=0, gamma=1.4):
    """Sod states (rho, P) = (1, 1) | (0.125, 0.1), v = 0, B = 0 on a periodic
    domain of length 2 along ``axis`` (one cell across the other two directions):
    the left state fills [0.5, 1.5), so an L|R interface sits at 1.5 and a mirrored
    R|L one at 0.5."""
    n = 2 * n_per_unit
    c = _centres(n, 2.0)
    left = (c >= 0.5) & (c < 1.5)
    shape = [1, 1, 1]
    shape[2 - axis] = n
    shape = tuple(shape)
    rho = np.where(left, 1.0, 0.125).reshape(shape).copy()
    P = np.where(left, 1.0, 0.1).reshape(shape).copy()
    z = np.zeros(shape)
    lengths = [1.0, 1.0, 1.0]
    lengths[axis] = 2.0
    return IC([rho, z.copy(), z.copy(), z.copy(), P, z.copy(), z.copy(), z.copy()],
              tuple(lengths), gamma, "sod_double_tube", {"n_per_unit": n_per_unit, "axis": axis})


def brio_wu_double_tube(n_per_unit=200, axis=0, gamma=5.0 / 3.0):
    """Brio-Wu MHD shock tube (Sec. 4.1; gamma = 5/3 as the paper runs it): (rho, P, B_t) =
    (1, 1, 1) | (0.125, 0.1, -1), v = 0, normal field 0.75, as a periodic double tube of
    length 2 along ``axis`` like ``sod_double_tube`` (left state in [0.5, 1.5)).  The normal
    field is the component along ``axis``, the transverse one the next component in cyclic
    order, so the three orientations are the same problem rotated."""
    n = 2 * n_per_unit
    c = _centres(n, 2.0)
    left = (c >= 0.5) & (c < 1.5)
    shape = [1, 1, 1]
    shape[2 - axis] = n
    shape = tuple(shape)
    rho = np.where(left, 1.0, 0.125).reshape(shape).copy()
    P = np.where(left, 1.0, 0.1).reshape(shape).copy()
    bt = np.where(left, 1.0, -1.0).reshape(shape).copy()
    z = np.zeros(shape)
    B = [z.copy(), z.copy(), z.copy()]
    B[axis] = _full(shape, 0.75)
    B[(axis + 1) % 3] = bt
    lengths = [1.0, 1.0, 1.0]
    lengths[axis] = 2.0
    return IC([rho, z.copy(), z.copy(), z.copy(), P] + B, tuple(lengths), gamma,
              "brio_wu_double_tube", {"n_per_unit": n_per_unit, "axis": axis})


def sedov_blast(n=64, energy=1.0, r_in=None, rho0=1.0, P0=1e-2, gamma=5.0 / 3.0):
    """Sedov-Taylor blast (Sec. 4.1): a uniform gas at rest, rho = 1, P = 1e-2, on the periodic
    unit cube, with the thermal energy E = sum over cells with centre inside r < r_in of
    P dV / (gamma - 1) = energy deposited at the centre (0.5, 0.5, 0.5).  r_in defaults to 3.5
    cells; no magnetic field."""
    h = 1.0 / n
    if r_in is None:
        r_in = 3.5 * h
    xc = _centres(n, 1.0)
    X, Y, Z = _mesh(xc, xc, xc)
    r2 = (X - 0.5) ** 2 + (Y - 0.5) ** 2 + (Z - 0.5) ** 2
    inside = np.broadcast_to(r2 < r_in * r_in, (n, n, n))
    n_in = int(inside.sum())
    P_in = (gamma - 1.0) * energy / (n_in * h ** 3)
    shape = (n, n, n)
    P = np.where(inside, P_in, P0).astype(np.float64)
    z = np.zeros(shape)
    return IC([_full(shape, rho0), z.copy(), z.copy(), z.copy(), P, z.copy(), z.copy(), z.copy()],
              (1.0, 1.0, 1.0), gamma, "sedov_blast",
              {"n": n, "energy": energy, "r_in": r_in, "cells_in": n_in, "P0": P0, "rho0": rho0})


def uniform(shape=(4, 4, 4), lengths=(1.0, 1.0, 1.0), gamma=5.0 / 3.0,
            rho=1.3, v=(0.3, -0.2, 0.1), P=0.7, B=(0.4, -0.5, 0.25)):
    p = [_full(shape, rho), _full(shape, v[0]), _full(shape, v[1]), _full(shape, v[2]),
         _full(shape, P), _full(shape, B[0]), _full(shape, B[1]), _full(shape, B[2])]
    return IC(p, tuple(lengths), gamma, "uniform", {})


def random_smooth(shape=(8, 8, 8), seed=0, lengths=(1.0, 1.0, 1.0), gamma=5.0 / 3.0,
                  amp=0.3, kmax=2):
    """Smooth random periodic state with O(1) variations: a few low Fourier modes per
    field around a positive background; face B = uniform part + discrete curl of a
    periodic edge vector potential, so the discrete divergence vanishes."""
    rng = np.random.Generator(np.random.PCG64(seed))
    nz, ny, nx = shape
    lx, ly, lz = lengths
    xc, yc, zc = _centres(nx, lx), _centres(ny, ly), _centres(nz, lz)
    xf, yf, zf = _faces(nx, lx), _faces(ny, ly), _faces(nz, lz)

    def field_at(x, y, z, base, a):
        out = np.zeros(np.broadcast_shapes(np.shape(x), np.shape(y), np.shape(z))) + base
        for _ in range(3):
            kx = rng.integers(0, kmax + 1) if nx > 1 else 0
            ky = rng.integers(0, kmax + 1) if ny > 1 else 0
            kz = rng.integers(0, kmax + 1) if nz > 1 else 0
            ph = rng.uniform(0, 2 * math.pi)
            c = rng.uniform(-a, a)
            out = out + c * np.sin(2 * math.pi * (kx * x / lx + ky * y / ly + kz * z / lz) + ph)
        return out

    X, Y, Z = _mesh(xc, yc, zc)
    rho = np.broadcast_to(field_at(X, Y, Z, 1.0, amp), shape).copy()
    P = np.broadcast_to(field_at(X, Y, Z, 0.8, amp), shape).copy()
    vx = np.broadcast_to(field_at(X, Y, Z, 0.1, 0.5), shape).copy()
    vy = np.broadcast_to(field_at(X, Y, Z, -0.1, 0.5), shape).copy()
    vz = np.broadcast_to(field_at(X, Y, Z, 0.05, 0.5), shape).copy()
    Xf, Yf, Zf = _mesh(xf, yf, zf)
    Ax = np.broadcast_to(field_at(X, Yf, Zf, 0.0, 0.05), shape)
    Ay = np.broadcast_to(field_at(Xf, Y, Zf, 0.0, 0.05), shape)
    Az = np.broadcast_to(field_at(Xf, Yf, Z, 0.0, 0.05), shape)
    dBx, dBy, dBz = _curl_faces(Ax, Ay, Az, (lx / nx, ly / ny, lz / nz))
    b0 = rng.uniform(-0.6, 0.6, 3)
    # the potential itself rides along for runs that start from (A, mean field)
    A = tuple(np.ascontiguousarray(a) for a in (Ax, Ay, Az))
    return IC([rho, vx, vy, vz, P, np.ascontiguousarray(b0[0] + dBx),
               np.ascontiguousarray(b0[1] + dBy), np.ascontiguousarray(b0[2] + dBz)],
              tuple(lengths), gamma, "random_smooth",
              {"seed": seed, "A": A, "bmean": tuple(float(x) for x in b0)})
