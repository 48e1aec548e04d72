"""Python binding of libidx.so (include/idx.h): argument marshalling only.

Every step of the method runs in the library's CUDA kernels; this module converts
numpy arrays / torch CUDA tensors to pointers and return codes to exceptions.
There is no fallback: if libidx.so cannot be loaded, ``lib()`` raises.
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libidx.so")

IDX_OK, IDX_EINVAL, IDX_ENOMEM, IDX_ENONPHYS, IDX_ECUDA, IDX_ETIMEOUT = 0, -1, -2, -3, -4, -5
IDX_ETOOLARGE = -6
IDX_FP64, IDX_FP32_BULK = 0, 1
PRECISIONS = {"fp64": IDX_FP64, "fp32": IDX_FP32_BULK, "fp32_bulk": IDX_FP32_BULK}
RIEMANN = {"rusanov": 1, "hll": 2, "hlld": 4}

_lib = None


class IdxError(RuntimeError):
    def __init__(self, code, where, cell=-1):
        msg = f"{where}: {strerror(code) if _lib else code} (code {code})"
        if cell >= 0:
            msg += f", cell {cell}"
        super().__init__(msg)
        self.code = code
        self.cell = cell


class Grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("lx", ctypes.c_double), ("ly", ctypes.c_double), ("lz", ctypes.c_double),
                ("bc", ctypes.c_int * 3)]


BC = {"periodic": 0, "outflow": 1, "reflecting": 2}


def _bc_codes(bc):
    return [BC[b] if isinstance(b, str) else int(b) for b in bc]


class Solver(ctypes.Structure):
    _fields_ = [("recon", ctypes.c_int), ("riemann", ctypes.c_int), ("emf", ctypes.c_int),
                ("rk_order", ctypes.c_int), ("cfl", ctypes.c_double), ("precision", ctypes.c_int),
                ("induction", ctypes.c_int)]


class Clock(ctypes.Structure):
    """idx_clock: simulated time, carried inverse CFL time (Eq. 10), cycle count."""
    _fields_ = [("t", ctypes.c_double), ("inv_dt", ctypes.c_double), ("nsteps", ctypes.c_int64)]


P8 = ctypes.c_void_p * 8
P3 = ctypes.c_void_p * 3
INDUCTION = {"field": 0, "potential": 1}
RECON = {"plm": 1, "limo3": 3}


def lib(path=LIB_PATH):
    """Load libidx.so (built by paper_2304_13746_b300.build); raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libidx.so not found at {path}: build it with "
                           "python -m paper_2304_13746_b300.build (no CPU fallback exists)")
    L = ctypes.CDLL(path)
    vp = ctypes.c_void_p
    L.idx_create.argtypes = [ctypes.POINTER(Grid), ctypes.c_double, ctypes.POINTER(Solver), vp,
                             ctypes.POINTER(vp)]
    L.idx_set_state.argtypes = [vp, P8, ctypes.c_int]
    L.idx_set_primitive.argtypes = [vp, P8, ctypes.c_int]
    L.idx_get_state.argtypes = [vp, P8, ctypes.c_int]
    L.idx_step.argtypes = [vp, ctypes.POINTER(ctypes.c_double)]
    L.idx_advance.argtypes = [vp, ctypes.c_double, ctypes.POINTER(ctypes.c_int64)]
    L.idx_time.argtypes = [vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
    L.idx_last_error_cell.argtypes = [vp, ctypes.POINTER(ctypes.c_int64)]
    L.idx_destroy.argtypes = [vp]
    L.idx_destroy.restype = None
    L.idx_strerror.argtypes = [ctypes.c_int]
    L.idx_strerror.restype = ctypes.c_char_p
    L.idx_pipe_rates.argtypes = [ctypes.POINTER(ctypes.c_double)]
    L.idx_kernel_times.argtypes = [vp, ctypes.c_int, ctypes.POINTER(ctypes.c_double)]
    L.idx_sweep_shapes.argtypes = [vp, ctypes.POINTER(ctypes.c_int)]
    L.idx_set_sweep_shapes.argtypes = [vp, ctypes.POINTER(ctypes.c_int)]
    L.idx_step_count.argtypes = [vp, ctypes.POINTER(ctypes.c_int64)]
    L.idx_footprint.argtypes = [ctypes.POINTER(Grid), ctypes.c_int, ctypes.POINTER(ctypes.c_uint64)]
    L.idx_footprint_solver.argtypes = [ctypes.POINTER(Grid), ctypes.POINTER(Solver),
                                       ctypes.POINTER(ctypes.c_uint64)]
    L.idx_set_potential.argtypes = [vp, P8, ctypes.POINTER(ctypes.c_double), ctypes.c_int]
    L.idx_get_potential.argtypes = [vp, P3, ctypes.c_int]
    L.idx_batch_create.argtypes = [ctypes.c_int, vp, ctypes.POINTER(vp)]
    L.idx_batch_add.argtypes = [vp, vp, ctypes.c_double]
    L.idx_batch_remove.argtypes = [vp, vp]
    L.idx_batch_step.argtypes = [vp, ctypes.c_int]
    L.idx_batch_poll.argtypes = [vp, ctypes.POINTER(vp), ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                 ctypes.POINTER(ctypes.c_int)]
    L.idx_batch_shapes.argtypes = [vp, ctypes.POINTER(ctypes.c_int)]
    L.idx_batch_set_shapes.argtypes = [vp, ctypes.POINTER(ctypes.c_int)]
    L.idx_batch_destroy.argtypes = [vp]
    L.idx_batch_destroy.restype = None
    L.idx_set_stage_kernels.argtypes = [vp, ctypes.c_int]
    L.idx_stage_kernels.argtypes = [vp, ctypes.POINTER(ctypes.c_int)]
    L.idx_get_clock.argtypes = [vp, ctypes.POINTER(Clock)]
    L.idx_set_clock.argtypes = [vp, ctypes.POINTER(Clock)]
    L.idx_probe_bounded_wait.argtypes = [vp, ctypes.c_uint32, ctypes.c_double]
    _lib = L
    return L


def strerror(code):
    return lib().idx_strerror(code).decode()


def pipe_rates():
    """Measured FP64/FP32 pipe throughputs (ops/s): fma64, div64, sqrt64, fma32, div32, sqrt32."""
    out = (ctypes.c_double * 6)()
    rc = lib().idx_pipe_rates(out)
    if rc != IDX_OK:
        raise IdxError(rc, "idx_pipe_rates")
    keys = ("fma64", "div64", "sqrt64", "fma32", "div32", "sqrt32")
    return dict(zip(keys, out[:]))


def probe_bounded_wait(announce_bytes, limit_ms, stream=None):
    """Run the library's bounded mbarrier wait alone (idx_probe_bounded_wait); returns the
    code it ends with: IDX_ETIMEOUT when bytes were announced and never arrive, else IDX_OK."""
    return lib().idx_probe_bounded_wait(ctypes.c_void_p(stream) if stream else None,
                                        int(announce_bytes), float(limit_ms))


def footprint(shape, precision="fp64", rk_order=2, induction="field", riemann="hlld",
              bc=(0, 0, 0), recon="plm"):
    """Device bytes a sim of this shape (nz, ny, nx) and configuration allocates."""
    nz, ny, nx = (int(v) for v in shape)
    out = ctypes.c_uint64()
    s = Solver(RECON[recon], RIEMANN[riemann], 2, int(rk_order), 0.4, PRECISIONS[precision],
               INDUCTION[induction])
    g = Grid(nx, ny, nz, 1.0, 1.0, 1.0, (ctypes.c_int * 3)(*_bc_codes(bc)))
    rc = lib().idx_footprint_solver(ctypes.byref(g), ctypes.byref(s), ctypes.byref(out))
    if rc != IDX_OK:
        raise IdxError(rc, "idx_footprint_solver")
    return int(out.value)


def _is_torch(a):
    return type(a).__module__.startswith("torch")


def _torch_sync():
    import torch
    torch.cuda.current_stream().synchronize()


class Sim:
    """One periodic MHD box on the current CUDA device.

    shape = (nz, ny, nx); lengths = (lx, ly, lz).  Fields are 8 arrays of that shape:
    numpy float64 (host) or contiguous torch float64 CUDA tensors (device).
    """

    def __init__(self, shape, lengths, gamma=5.0 / 3.0, cfl=0.4, precision="fp64", stream=None,
                 riemann="hlld", rk_order=2, induction="field", bc=(0, 0, 0), recon="plm"):
        """bc: boundary kind per direction x, y, z ("periodic", "outflow", "reflecting" or
        0/1/2); along a non-periodic direction of more than one cell the normal face field
        has one more face than cells (see include/idx.h)."""
        L = lib()
        nz, ny, nx = (int(s) for s in shape)
        self.shape = (nz, ny, nx)
        self.bc = _bc_codes(bc)
        # per-field shapes in the user layout
        self.field_shapes = [self.shape] * 5
        for d, ax in ((0, 2), (1, 1), (2, 0)):
            fs = list(self.shape)
            if self.bc[d] and self.shape[ax] > 1:
                fs[ax] += 1
            self.field_shapes.append(tuple(fs))
        self.lengths = tuple(float(x) for x in lengths)
        self.gamma = float(gamma)
        self.cfl = float(cfl)
        self.precision = precision
        g = Grid(nx, ny, nz, *self.lengths, (ctypes.c_int * 3)(*self.bc))
        self.induction = induction
        s = Solver(RECON[recon], RIEMANN[riemann], 2, int(rk_order), self.cfl,
                   PRECISIONS[precision], INDUCTION[induction])
        h = ctypes.c_void_p()
        rc = L.idx_create(ctypes.byref(g), self.gamma, ctypes.byref(s),
                          ctypes.c_void_p(stream) if stream else None, ctypes.byref(h))
        if rc != IDX_OK:
            raise IdxError(rc, "idx_create")
        self._h = h

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None):
            lib().idx_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc, where):
        if rc != IDX_OK:
            cell = ctypes.c_int64(-1)
            lib().idx_last_error_cell(self._h, ctypes.byref(cell))
            raise IdxError(rc, where, cell.value)

    def _ptrs(self, fields, writable=False):
        assert len(fields) in (3, 8)
        P = P8 if len(fields) == 8 else P3
        shapes = self.field_shapes if len(fields) == 8 else [self.shape] * 3
        if all(_is_torch(a) for a in fields):
            import torch
            for a, sh in zip(fields, shapes):
                assert a.is_cuda and a.dtype == torch.float64 and a.is_contiguous()
                assert tuple(a.shape) == sh
            _torch_sync()
            return P(*[a.data_ptr() for a in fields]), 1, fields
        arrs = []
        for a, sh in zip(fields, shapes):
            a = np.asarray(a)
            assert a.dtype == np.float64 and a.flags.c_contiguous and a.shape == sh, \
                (a.dtype, a.shape, sh)
            if writable:
                assert a.flags.writeable
            arrs.append(a)
        return P(*[a.ctypes.data for a in arrs]), 0, arrs

    def set_state(self, cons):
        p, dev, keep = self._ptrs(cons)
        self._check(lib().idx_set_state(self._h, p, dev), "idx_set_state")

    def set_primitive(self, prim):
        p, dev, keep = self._ptrs([np.ascontiguousarray(a, dtype=np.float64)
                                   if not _is_torch(a) else a for a in prim])
        self._check(lib().idx_set_primitive(self._h, p, dev), "idx_set_primitive")

    def set_potential(self, prim5, A, bmean):
        """Cells from (rho, vx, vy, vz, P), faces from bmean + curl A; A = (Ax, Ay, Az) on
        the cell edges (layout of idx_set_potential)."""
        fields = [a if _is_torch(a) else np.ascontiguousarray(a, dtype=np.float64)
                  for a in list(prim5) + list(A)]
        p, dev, keep = self._ptrs(fields)
        b = (ctypes.c_double * 3)(*[float(x) for x in bmean])
        self._check(lib().idx_set_potential(self._h, p, b, dev), "idx_set_potential")

    def get_potential(self, out=None, device=False):
        """Edge potential (Ax, Ay, Az) of a vector-potential sim."""
        if out is None:
            if device:
                import torch
                out = [torch.empty(self.shape, dtype=torch.float64, device="cuda")
                       for _ in range(3)]
            else:
                out = [np.empty(self.shape, dtype=np.float64) for _ in range(3)]
        p, dev, keep = self._ptrs(out, writable=True)
        self._check(lib().idx_get_potential(self._h, p, dev), "idx_get_potential")
        return out

    def get_state(self, out=None, device=False):
        if out is None:
            if device:
                import torch
                out = [torch.empty(sh, dtype=torch.float64, device="cuda")
                       for sh in self.field_shapes]
            else:
                out = [np.empty(sh, dtype=np.float64) for sh in self.field_shapes]
        p, dev, keep = self._ptrs(out, writable=True)
        self._check(lib().idx_get_state(self._h, p, dev), "idx_get_state")
        return out

    def step(self, want_dt=False):
        if want_dt:
            dt = ctypes.c_double()
            self._check(lib().idx_step(self._h, ctypes.byref(dt)), "idx_step")
            return dt.value
        self._check(lib().idx_step(self._h, None), "idx_step")
        return None

    def advance(self, t_end):
        n = ctypes.c_int64()
        self._check(lib().idx_advance(self._h, float(t_end), ctypes.byref(n)), "idx_advance")
        return n.value

    def kernel_times(self, reps=2):
        """Per-launch device ms of each kernel (events between launches); advances reps cycles."""
        out = (ctypes.c_double * 6)()
        self._check(lib().idx_kernel_times(self._h, int(reps), out), "idx_kernel_times")
        return dict(zip(("prims", "sweep_x", "sweep_y", "sweep_z", "emf", "update"), out[:]))

    def sweep_shapes(self):
        """Sweep shape per direction: faces per thread, -1 warp x-sweep, 116/132 TMA-staged tile,
        0 inactive."""
        out = (ctypes.c_int * 3)()
        self._check(lib().idx_sweep_shapes(self._h, out), "idx_sweep_shapes")
        return list(out)

    def set_sweep_shapes(self, shapes):
        """Fix the sweep shapes (x, y, z) instead of autotuning them (see idx_sweep_shapes)."""
        arr = (ctypes.c_int * 3)(*[int(v) for v in shapes])
        self._check(lib().idx_set_sweep_shapes(self._h, arr), "idx_set_sweep_shapes")

    STAGE_KERNELS = {"auto": 0, "split": 1, "fused": 2, "carry": 3}

    def set_stage_kernels(self, mode):
        """FP32 bulk: "auto", "split" (six kernels per stage), "fused" (one stage kernel) or
        "carry" (the update also recovers the next stage's primitives); idx_set_stage_kernels."""
        self._check(lib().idx_set_stage_kernels(self._h, self.STAGE_KERNELS[mode]),
                    "idx_set_stage_kernels")

    def stage_kernels(self):
        """The stage kernels in use: "split", "fused" or "carry" (idx_stage_kernels)."""
        v = ctypes.c_int()
        self._check(lib().idx_stage_kernels(self._h, ctypes.byref(v)), "idx_stage_kernels")
        return {1: "split", 2: "fused", 3: "carry"}[v.value]

    def step_count(self):
        n = ctypes.c_int64()
        self._check(lib().idx_step_count(self._h, ctypes.byref(n)), "idx_step_count")
        return n.value

    def get_clock(self):
        """(t, inv_dt, nsteps): the time-stepping state to store beside the fields."""
        c = Clock()
        self._check(lib().idx_get_clock(self._h, ctypes.byref(c)), "idx_get_clock")
        return c.t, c.inv_dt, c.nsteps

    def set_clock(self, clock):
        """Restore (t, inv_dt, nsteps) after set_state, to continue a stored run."""
        c = Clock(*clock)
        self._check(lib().idx_set_clock(self._h, ctypes.byref(c)), "idx_set_clock")

    def time(self):
        t, dt = ctypes.c_double(), ctypes.c_double()
        self._check(lib().idx_time(self._h, ctypes.byref(t), ctypes.byref(dt)), "idx_time")
        return t.value, dt.value


class Batch:
    """Many sims stepped together (idx_batch_*): each keeps its own dt and end time."""

    def __init__(self, precision="fp64", stream=None):
        L = lib()
        h = ctypes.c_void_p()
        rc = L.idx_batch_create(PRECISIONS[precision], ctypes.c_void_p(stream) if stream else None,
                                ctypes.byref(h))
        if rc != IDX_OK:
            raise IdxError(rc, "idx_batch_create")
        self._h = h
        self.members = {}

    def _check(self, rc, where):
        if rc != IDX_OK:
            raise IdxError(rc, where)

    def add(self, sim, t_end=float("inf")):
        self._check(lib().idx_batch_add(self._h, sim.handle, float(t_end)), "idx_batch_add")
        self.members[sim.handle.value] = sim

    def remove(self, sim):
        self._check(lib().idx_batch_remove(self._h, sim.handle), "idx_batch_remove")
        self.members.pop(sim.handle.value, None)

    def step(self, ncycles=1):
        self._check(lib().idx_batch_step(self._h, int(ncycles)), "idx_batch_step")

    def poll(self):
        """Synchronise; returns (members that reached their end time or failed, n_active)."""
        cap = max(1, len(self.members))
        arr = (ctypes.c_void_p * cap)()
        nf, na = ctypes.c_int(), ctypes.c_int()
        self._check(lib().idx_batch_poll(self._h, arr, cap, ctypes.byref(nf), ctypes.byref(na)),
                    "idx_batch_poll")
        return [self.members[arr[i]] for i in range(min(nf.value, cap))], na.value

    def shapes(self):
        out = (ctypes.c_int * 3)()
        self._check(lib().idx_batch_shapes(self._h, out), "idx_batch_shapes")
        return list(out)

    def set_shapes(self, shapes):
        """Fix the batch's sweep shapes (x, y, z) instead of autotuning them."""
        arr = (ctypes.c_int * 3)(*[int(v) for v in shapes])
        self._check(lib().idx_batch_set_shapes(self._h, arr), "idx_batch_set_shapes")

    def close(self):
        if getattr(self, "_h", None):
            lib().idx_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
