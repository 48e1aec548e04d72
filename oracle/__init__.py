"""FP64 CPU oracle for one RK2 cycle of ideal MHD -- TEST INFRASTRUCTURE ONLY.

Only the tests, the smoke check and the benchmark's CPU-baseline leg may import
this package.  It shares no code with the CUDA path; both consume the seeded
inputs of ``paper_2304_13746_b300.inputs`` and nothing else.

Method: IDEFIX paper (Lesur et al. 2023), Eqs. (1)-(6), (9), (10), Table 1,
Secs. 2.3, 2.4, 2.7; HLLD of Miyoshi & Kusano (2005); E^c EMF of Gardiner &
Stone (2005); LimO3 reconstruction of Cada & Torrilhon (2009).  Every array is numpy float64 with shape (nz, ny, nx), periodic.
"""
import ctypes
import math

import numpy as np

from .build import build as _build

_lib = None

OK, EINVAL, ENONPHYS = 0, -1, -3
FIELDS = ("rho", "mx", "my", "mz", "E", "Bx", "By", "Bz")
PRIM_FIELDS = ("rho", "vx", "vy", "vz", "P", "Bx", "By", "Bz")


class OracleError(RuntimeError):
    def __init__(self, code, bad_cell=-1):
        super().__init__(f"oracle error {code} (bad cell {bad_cell})")
        self.code = code
        self.bad_cell = bad_cell


class _Grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("lx", ctypes.c_double), ("ly", ctypes.c_double), ("lz", ctypes.c_double)]


_P8 = ctypes.c_void_p * 8
_P3 = ctypes.c_void_p * 3
_D = ctypes.POINTER(ctypes.c_double)


def lib():
    global _lib
    if _lib is None:
        path = _build()
        L = ctypes.CDLL(path)
        G = ctypes.POINTER(_Grid)
        L.ora_cons_from_prims.argtypes = [G, ctypes.c_double, _P8, _P8]
        L.ora_prims.argtypes = [G, ctypes.c_double, _P8, _P8, ctypes.POINTER(ctypes.c_long)]
        L.ora_vanleer.argtypes = [ctypes.c_double] * 3
        L.ora_vanleer.restype = ctypes.c_double
        L.ora_hlld.argtypes = [_D, _D, ctypes.c_double, ctypes.c_double, _D, _D, _D]
        L.ora_phys_flux.argtypes = [_D, ctypes.c_double, ctypes.c_double, _D]
        L.ora_emf_ec.argtypes = [_D, _D, _D, _D, _D, ctypes.c_double, ctypes.c_double]
        L.ora_emf_ec.restype = ctypes.c_double
        L.ora_speed_pass.argtypes = [G, ctypes.c_double, _P8, _D, ctypes.POINTER(ctypes.c_long)]
        L.ora_stage.argtypes = [G, ctypes.c_double, ctypes.c_double, _P8, _P8, ctypes.c_double,
                                ctypes.c_double, _P8, _D, ctypes.POINTER(ctypes.c_long)]
        L.ora_cycle.argtypes = [G, ctypes.c_double, ctypes.c_double, _P8, _D, ctypes.c_double, _D,
                                ctypes.POINTER(ctypes.c_long)]
        L.ora_count_cycle.argtypes = [G, ctypes.c_double, ctypes.c_double, _P8, ctypes.c_double, _D]
        L.ora_riemann.argtypes = [ctypes.c_int, _D, _D, ctypes.c_double, ctypes.c_double, _D, _D, _D]
        L.ora_cycle_solver.argtypes = [G, ctypes.c_double, ctypes.c_double, ctypes.c_int, _P8, _D,
                                       ctypes.c_double, _D, ctypes.POINTER(ctypes.c_long)]
        L.ora_cycle_rk.argtypes = [G, ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                   _P8, _D, ctypes.c_double, _D, ctypes.POINTER(ctypes.c_long)]
        L.ora_count_faces.argtypes = [G, ctypes.c_double, _P8, ctypes.c_int, _D, _D]
        L.ora_count_faces_parts.argtypes = [G, ctypes.c_double, _P8, ctypes.c_int, _D]
        L.ora_count_cycle_parts.argtypes = [G, ctypes.c_double, ctypes.c_double, _P8,
                                            ctypes.c_double, _D]
        L.ora_count_vanleer.argtypes = [ctypes.c_double] * 3 + [_D]
        L.ora_count_energy_flux.argtypes = [_D, ctypes.c_double, ctypes.c_double, _D, _D]
        L.ora_count_hlld.argtypes = [_D, _D, ctypes.c_double, ctypes.c_double, _D]
        L.ora_count_emf_ec.argtypes = [_D, _D, _D, _D, _D, ctypes.c_double, ctypes.c_double, _D]
        L.ora_b_from_potential.argtypes = [G, _P3, _D, _P3]
        L.ora_cycle_vp.argtypes = [G, ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                   _P8, _P3, _P3, _D, ctypes.c_double, _D,
                                   ctypes.POINTER(ctypes.c_long)]
        L.ora_limo3_face.argtypes = [ctypes.c_double] * 3
        L.ora_limo3_face.restype = ctypes.c_double
        L.ora_speed_pass_recon.argtypes = [G, ctypes.c_double, ctypes.c_int, _P8, _D,
                                           ctypes.POINTER(ctypes.c_long)]
        L.ora_stage_scheme.argtypes = [G, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                       ctypes.c_int, _P8, _P8, ctypes.c_double, ctypes.c_double,
                                       _P8, _D, ctypes.POINTER(ctypes.c_long)]
        L.ora_cycle_scheme.argtypes = [G, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                       ctypes.c_int, ctypes.c_int, _P8, ctypes.c_void_p,
                                       ctypes.c_void_p, _D, ctypes.c_double, _D,
                                       ctypes.POINTER(ctypes.c_long)]
        L.ora_threads.restype = ctypes.c_int
        _lib = L
    return _lib


def _grid(shape, lengths):
    nz, ny, nx = shape
    lx, ly, lz = lengths
    return _Grid(nx, ny, nz, lx, ly, lz)


def _ptrs(arrays):
    for a in arrays:
        assert a.dtype == np.float64 and a.flags.c_contiguous
    return (_P8 if len(arrays) == 8 else _P3)(*[a.ctypes.data for a in arrays])


def _new(shape):
    return [np.zeros(shape, dtype=np.float64) for _ in range(8)]


def _c(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _check(code, bad=None):
    if code != OK:
        raise OracleError(code, -1 if bad is None else bad.value)


def cons_from_prims(prim, lengths, gamma):
    """(rho, vx, vy, vz, P, Bx_face, By_face, Bz_face) -> conserved 8-list."""
    prim = [_c(a) for a in prim]
    out = _new(prim[0].shape)
    _check(lib().ora_cons_from_prims(ctypes.byref(_grid(prim[0].shape, lengths)), gamma,
                                     _ptrs(prim), _ptrs(out)))
    return out


def prims(cons, lengths, gamma):
    cons = [_c(a) for a in cons]
    out = _new(cons[0].shape)
    bad = ctypes.c_long(-1)
    _check(lib().ora_prims(ctypes.byref(_grid(cons[0].shape, lengths)), gamma, _ptrs(cons),
                           _ptrs(out), ctypes.byref(bad)), bad)
    return out


def vanleer(wm, w0, wp):
    return lib().ora_vanleer(float(wm), float(w0), float(wp))


RECONS = {"plm": 1, "limo3": 3}


def limo3_face(w_back, w0, w_face):
    """LimO3 value of a cell (value w0) at its face toward w_face (Sec. 2.3)."""
    return lib().ora_limo3_face(float(w_back), float(w0), float(w_face))


def _arr(x, n):
    return (ctypes.c_double * n)(*[float(v) for v in x])


def hlld(wL, wR, bn, gamma):
    """Single interface.  wL, wR = (rho, u, v, w, P, Bt1, Bt2); returns (F[7], sL, sR)."""
    F = (ctypes.c_double * 7)()
    sL, sR = ctypes.c_double(), ctypes.c_double()
    _check(lib().ora_hlld(_arr(wL, 7), _arr(wR, 7), float(bn), float(gamma), F,
                          ctypes.byref(sL), ctypes.byref(sR)))
    return np.array(F[:]), sL.value, sR.value


SOLVERS = {"rusanov": 1, "hll": 2, "hlld": 4}


def riemann(solver, wL, wR, bn, gamma):
    """Single interface with solver 'rusanov', 'hll' or 'hlld'; returns (F[7], sL, sR)."""
    F = (ctypes.c_double * 7)()
    sL, sR = ctypes.c_double(), ctypes.c_double()
    _check(lib().ora_riemann(SOLVERS[solver], _arr(wL, 7), _arr(wR, 7), float(bn), float(gamma), F,
                             ctypes.byref(sL), ctypes.byref(sR)))
    return np.array(F[:]), sL.value, sR.value


def phys_flux(w, bn, gamma):
    F = (ctypes.c_double * 7)()
    _check(lib().ora_phys_flux(_arr(w, 7), float(bn), float(gamma), F))
    return np.array(F[:])


def emf_ec(X, Y, C, Fa, Fb, da, db):
    """C indexed C[c][r]: c = 0 (I), 1 (I-1); r = 0 (J), 1 (J-1)."""
    Cf = _arr(np.asarray(C, dtype=float).ravel(), 4)
    return lib().ora_emf_ec(_arr(X, 2), _arr(Y, 2), Cf, _arr(Fa, 2), _arr(Fb, 2), float(da),
                            float(db))


def speed_pass(cons, lengths, gamma, recon="plm"):
    cons = [_c(a) for a in cons]
    inv = ctypes.c_double()
    bad = ctypes.c_long(-1)
    _check(lib().ora_speed_pass_recon(ctypes.byref(_grid(cons[0].shape, lengths)), gamma,
                                      RECONS[recon], _ptrs(cons), ctypes.byref(inv),
                                      ctypes.byref(bad)), bad)
    return inv.value


def stage(uin, lengths, gamma, dt, u0=None, w=1.0, w0=0.0, recon="plm", solver="hlld"):
    uin = [_c(a) for a in uin]
    out = _new(uin[0].shape)
    keep = [_c(a) for a in u0] if u0 is not None else None
    p0 = _ptrs(keep) if keep is not None else _P8()
    inv = ctypes.c_double()
    bad = ctypes.c_long(-1)
    _check(lib().ora_stage_scheme(ctypes.byref(_grid(uin[0].shape, lengths)), gamma, dt,
                                  RECONS[recon], SOLVERS[solver], _ptrs(uin), p0, w, w0,
                                  _ptrs(out), ctypes.byref(inv), ctypes.byref(bad)), bad)
    return out, inv.value


def b_from_potential(A, bmean, lengths):
    """Face field (Bx, By, Bz) = bmean + curl A (Sec. 2.4, Eq. 8); A = (Ax, Ay, Az) on edges."""
    A = [_c(a) for a in A]
    out = [np.zeros(A[0].shape) for _ in range(3)]
    _check(lib().ora_b_from_potential(ctypes.byref(_grid(A[0].shape, lengths)), _ptrs(A),
                                      _arr(bmean, 3), _ptrs(out)))
    return out


INDUCTION = ("field", "potential")


class Sim:
    """Oracle simulation: state, time, and the inverse CFL time carried between cycles.

    induction="field" steps the face field with the curl of the edge EMFs (Eq. 6);
    induction="potential" steps an edge vector potential A with -E and sets the face
    field to bref + curl A every stage (Eqs. 7-8).  Without an explicit A the potential
    starts at 0 and bref is the initial face field.
    """

    def __init__(self, cons, lengths, gamma, cfl, solver="hlld", rk_order=2, induction="field",
                 A=None, bref=None, recon="plm"):
        if induction not in INDUCTION:
            raise ValueError(induction)
        self.solver = SOLVERS[solver]
        self.recon_name = recon
        self.recon = RECONS[recon]
        self.rk_order = int(rk_order)
        self.u = [_c(a).copy() for a in cons]
        self.lengths = tuple(float(x) for x in lengths)
        self.gamma = float(gamma)
        self.cfl = float(cfl)
        self.t = 0.0
        self.nsteps = 0
        self.induction = induction
        if induction == "potential":
            shape = self.u[0].shape
            self.A = [np.zeros(shape) for _ in range(3)] if A is None else [_c(a).copy() for a in A]
            self.bref = [self.u[5 + d].copy() for d in range(3)] if bref is None else \
                [_c(b).copy() for b in bref]
        self.inv_dt = speed_pass(self.u, self.lengths, self.gamma, recon)

    @classmethod
    def from_prims(cls, prim, lengths, gamma, cfl, solver="hlld", rk_order=2, induction="field",
                   recon="plm"):
        return cls(cons_from_prims(prim, lengths, gamma), lengths, gamma, cfl, solver, rk_order,
                   induction, recon=recon)

    @classmethod
    def from_potential(cls, prim5, A, bmean, lengths, gamma, cfl, solver="hlld", rk_order=2,
                       induction="potential", recon="plm"):
        """Cells from (rho, vx, vy, vz, P), faces from bmean + curl A."""
        B = b_from_potential(A, bmean, lengths)
        cons = cons_from_prims(list(prim5) + B, lengths, gamma)
        if induction == "field":
            return cls(cons, lengths, gamma, cfl, solver, rk_order, recon=recon)
        bref = [np.full(B[0].shape, float(bmean[d])) for d in range(3)]
        return cls(cons, lengths, gamma, cfl, solver, rk_order, "potential", A, bref, recon)

    def step(self, dt_max=math.inf):
        inv = ctypes.c_double(self.inv_dt)
        dt = ctypes.c_double()
        bad = ctypes.c_long(-1)
        g = ctypes.byref(_grid(self.u[0].shape, self.lengths))
        if self.induction == "potential":
            pa, pb = _ptrs(self.A), _ptrs(self.bref)
            A, bref = ctypes.cast(pa, ctypes.c_void_p), ctypes.cast(pb, ctypes.c_void_p)
        else:
            A = bref = None
        rc = lib().ora_cycle_scheme(g, self.gamma, self.cfl, self.recon, self.solver,
                                    self.rk_order, _ptrs(self.u), A, bref, ctypes.byref(inv),
                                    float(dt_max), ctypes.byref(dt), ctypes.byref(bad))
        _check(rc, bad)
        self.inv_dt = inv.value
        self.nsteps += 1
        return dt.value

    def advance(self, t_end, max_steps=10**7):
        """Cycles until t == t_end; the last dt is clamped to t_end - t."""
        n = 0
        while self.t < t_end and n < max_steps:
            remaining = t_end - self.t
            dt = self.step(dt_max=remaining)
            if dt >= remaining:
                self.t = t_end
            else:
                self.t += dt
            n += 1
        return n

    def next_dt(self):
        return self.cfl / self.inv_dt


def count_cycle(cons, lengths, gamma, cfl):
    """Per cell-update counts: dict(add, mul, div, sqrt, cmp) for one RK2 cycle."""
    cons = [_c(a) for a in cons]
    inv = speed_pass(cons, lengths, gamma)
    out = (ctypes.c_double * 5)()
    _check(lib().ora_count_cycle(ctypes.byref(_grid(cons[0].shape, lengths)), gamma, cfl,
                                 _ptrs(cons), inv, out))
    return dict(zip(("add", "mul", "div", "sqrt", "cmp"), out[:]))


def count_faces(cons, lengths, gamma, d):
    """Per-face op counts of direction d: (hlld dict, reconstruction dict)."""
    cons = [_c(a) for a in cons]
    a, b = (ctypes.c_double * 5)(), (ctypes.c_double * 5)()
    _check(lib().ora_count_faces(ctypes.byref(_grid(cons[0].shape, lengths)), gamma, _ptrs(cons),
                                 int(d), a, b))
    keys = ("add", "mul", "div", "sqrt", "cmp")
    return dict(zip(keys, a[:])), dict(zip(keys, b[:]))


OPS = ("add", "mul", "div", "sqrt", "cmp")
# parts of the method the op counts are split into (ORA_PART_* of oracle.h)
PARTS = ("prims", "slope", "face", "riemann", "speed", "invdt", "cell_emf", "edge", "diff",
         "accum", "combine", "dt", "potential")


def count_cycle_parts(cons, lengths, gamma, cfl, inv_dt=None):
    """Per cell-update op counts of one RK2 cycle split by part: {part: {op: count}}.
    inv_dt: the inverse CFL time the cycle starts from (default: the speed pass's)."""
    cons = [_c(a) for a in cons]
    inv = speed_pass(cons, lengths, gamma) if inv_dt is None else float(inv_dt)
    out = (ctypes.c_double * (5 * len(PARTS)))()
    _check(lib().ora_count_cycle_parts(ctypes.byref(_grid(cons[0].shape, lengths)), gamma, cfl,
                                       _ptrs(cons), inv, out))
    return {p: dict(zip(OPS, out[5 * q:5 * q + 5])) for q, p in enumerate(PARTS)}


def flops(counts):
    """Floating-point operations of an op-count dict: add + mul + div + sqrt (compares and
    sign operations are not flops; the oracle has no fused operations)."""
    return counts["add"] + counts["mul"] + counts["div"] + counts["sqrt"]


def algorithmic_flops(parts):
    """Flops per cell-update with each piece of the method's work counted once: the oracle
    forms each cell's van Leer slope for both faces that use it and each cell-centre EMF at
    the four edges around it, so half of the slope part and three quarters of the
    cell-centre EMF part are repeats."""
    total = sum(flops(c) for c in parts.values())
    return total - 0.5 * flops(parts["slope"]) - 0.75 * flops(parts["cell_emf"])


def fp64_island_flops(parts):
    """Flops per cell-update that the FP32-bulk variant keeps in FP64: the primitive
    recovery (energy to pressure), the accumulation into the state and the RK combine."""
    return flops(parts["prims"]) + flops(parts["accum"]) + flops(parts["combine"])


def _counts5(arr):
    return dict(zip(OPS, arr[:]))


def count_vanleer(wm, w0, wp):
    out = (ctypes.c_double * 5)()
    _check(lib().ora_count_vanleer(float(wm), float(w0), float(wp), out))
    return _counts5(out)


def count_energy_flux(w, bn, gamma):
    """(counts of the total energy, counts of the physical flux) of one face state w."""
    w = (ctypes.c_double * 7)(*[float(x) for x in w])
    a, b = (ctypes.c_double * 5)(), (ctypes.c_double * 5)()
    _check(lib().ora_count_energy_flux(w, float(bn), float(gamma), a, b))
    return _counts5(a), _counts5(b)


def count_hlld(wL, wR, bn, gamma):
    a = (ctypes.c_double * 7)(*[float(x) for x in wL])
    b = (ctypes.c_double * 7)(*[float(x) for x in wR])
    out = (ctypes.c_double * 5)()
    _check(lib().ora_count_hlld(a, b, float(bn), float(gamma), out))
    return _counts5(out)


def count_emf_ec(X, Y, C, Fa, Fb, da, db):
    arr = [(ctypes.c_double * 2)(*[float(x) for x in v]) for v in (X, Y)]
    c = (ctypes.c_double * 4)(C[0][0], C[0][1], C[1][0], C[1][1])
    fa = (ctypes.c_double * 2)(*[float(x) for x in Fa])
    fb = (ctypes.c_double * 2)(*[float(x) for x in Fb])
    out = (ctypes.c_double * 5)()
    _check(lib().ora_count_emf_ec(arr[0], arr[1], c, fa, fb, float(da), float(db), out))
    return _counts5(out)


def count_faces_parts(cons, lengths, gamma, d):
    """Per-face op counts of direction d split into {"riemann", "slope", "face"}."""
    cons = [_c(a) for a in cons]
    out = (ctypes.c_double * 15)()
    _check(lib().ora_count_faces_parts(ctypes.byref(_grid(cons[0].shape, lengths)), gamma,
                                       _ptrs(cons), int(d), out))
    return {p: dict(zip(OPS, out[5 * q:5 * q + 5])) for q, p in enumerate(("riemann", "slope",
                                                                           "face"))}


def algorithmic_face_flops(parts):
    """Flops per face with each cell's slope counted once (half the slope part)."""
    return flops(parts["riemann"]) + flops(parts["face"]) + 0.5 * flops(parts["slope"])


def threads():
    return lib().ora_threads()


class SimBC:
    """Oracle simulation with non-periodic boundaries (oracle/boundaries.py): the padded
    grid is stepped stage by stage with ora_stage_scheme (E^c), the ghosts refilled before
    every stage.  bc = (kind_x, kind_y, kind_z) of boundaries.PERIODIC / OUTFLOW /
    REFLECTING.  Fields in the user layout (normal field n + 1 faces along a non-periodic
    direction); every array numpy float64 of shape (nz, ny, nx) (+1 along that axis)."""

    def __init__(self, prim, lengths, gamma, cfl, bc, rk_order=2, recon="plm", solver="hlld"):
        from . import boundaries as bd
        self.bd = bd
        self.bc = tuple(int(b) for b in bc)
        self.cell_shape = prim[0].shape
        self.lengths = tuple(float(x) for x in lengths)
        self.plengths = bd.padded_lengths(self.lengths, self.cell_shape, self.bc)
        self.gamma = float(gamma)
        self.cfl = float(cfl)
        self.rk_order = int(rk_order)
        self.recon_name, self.solver_name = recon, solver
        w = bd.fill_ghosts(bd.pad([_c(a) for a in prim], self.bc), self.bc)
        self.u = bd.fill_ghosts(cons_from_prims(w, self.plengths, self.gamma), self.bc)
        self.t = 0.0
        self.nsteps = 0
        self.inv_dt = speed_pass(self.u, self.plengths, self.gamma, recon)

    def state(self):
        return self.bd.unpad(self.u, self.bc, self.cell_shape)

    def step(self, dt_max=math.inf):
        dt = min(self.cfl / self.inv_dt, dt_max)
        weights = [(1.0, 0.0), (0.5, 0.5)] if self.rk_order == 2 else \
            [(1.0, 0.0), (0.25, 0.75), (2.0 / 3.0, 1.0 / 3.0)]
        u0 = self.u
        prev = u0
        inv = 0.0
        for w, w0 in weights:
            out, inv_s = stage(prev, self.plengths, self.gamma, dt, u0=u0 if w0 else None, w=w,
                               w0=w0, recon=self.recon_name, solver=self.solver_name)
            prev = self.bd.fill_ghosts(out, self.bc)
            inv = max(inv, inv_s)
        self.u = prev
        self.inv_dt = inv
        self.nsteps += 1
        return dt

    def advance(self, t_end, max_steps=10**7):
        n = 0
        while self.t < t_end and n < max_steps:
            remaining = t_end - self.t
            dt = self.step(dt_max=remaining)
            self.t = t_end if dt >= remaining else self.t + dt
            n += 1
        return n
