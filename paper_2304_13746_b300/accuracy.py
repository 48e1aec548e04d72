"""Error budget of the FP32-bulk variant against the scheme's own discretisation error.

For a box of N^3 cells advanced to a fixed time t:
  e_fp32[f] = mean |u32_N[f] - u64_N[f]|              (FP32 bulk vs FP64, same grid)
  e_disc[f] = mean |R2(u64_N)[f] - u64_{N/2}[f]| / (2^p - 1),  p = 2
where R2 restricts a fine field to the coarse grid conservatively: the mean of the 2^3
fine cells for cell fields, the mean of the 2 x 2 fine faces that tile a coarse face for
the face-centred B components.  The requirement is e_fp32[f] < 0.1 e_disc[f] per field.
All runs go through the C ABI (idx_set_primitive, idx_advance, idx_get_state).
"""
import numpy as np

FIELDS = ("rho", "mx", "my", "mz", "E", "Bx", "By", "Bz")


def restrict(u):
    """Fine (2n)^3 state -> coarse n^3: cell means, and face means over the coarse face."""
    out = []
    for f, a in enumerate(u):
        nz, ny, nx = a.shape
        if f < 5:
            b = a.reshape(nz // 2, 2, ny // 2, 2, nx // 2, 2).mean(axis=(1, 3, 5))
        elif f == 5:  # x-faces at even i coincide with coarse faces; mean over (y, z) pairs
            b = a[:, :, 0::2].reshape(nz // 2, 2, ny // 2, 2, nx // 2).mean(axis=(1, 3))
        elif f == 6:
            b = a[:, 0::2, :].reshape(nz // 2, 2, ny // 2, nx // 2, 2).mean(axis=(1, 4))
        else:
            b = a[0::2, :, :].reshape(nz // 2, ny // 2, 2, nx // 2, 2).mean(axis=(2, 4))
        out.append(b)
    return out


def run(ic, precision, t_end, cfl=0.4):
    from . import idx
    s = idx.Sim(ic.shape, ic.lengths, ic.gamma, cfl, precision)
    try:
        s.set_primitive(ic.prim)
        n = s.advance(t_end)
        return s.get_state(), n
    finally:
        s.close()


def fp32_error_budget(n, t_end, seed=0, p=2):
    """Per-field e_fp32, e_disc and their ratio for the turbulent box at n^3, time t_end."""
    from . import inputs
    fine = inputs.turbulent_box(n, seed=seed)
    coarse = inputs.turbulent_box(n // 2, seed=seed)
    u64, n64 = run(fine, "fp64", t_end)
    u32, n32 = run(fine, "fp32", t_end)
    uc, nc = run(coarse, "fp64", t_end)
    rf = restrict(u64)
    out = {}
    for f, name in enumerate(FIELDS):
        e32 = float(np.mean(np.abs(u32[f] - u64[f])))
        ed = float(np.mean(np.abs(rf[f] - uc[f]))) / (2 ** p - 1)
        out[name] = {"e_fp32": e32, "e_disc": ed, "ratio": e32 / ed if ed > 0 else float("inf")}
    return {"n": n, "t_end": t_end, "cycles_fp64": n64, "cycles_fp32": n32,
            "cycles_coarse": nc, "fields": out,
            "max_ratio": max(v["ratio"] for v in out.values())}
