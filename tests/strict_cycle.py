"""Child process of tests/test_gpu_strict_rounding.py: one RK2 cycle through the
strict-rounding test build of the library (libidx_strict.so), written to an .npz file.

The binding loads one library per process, so the strict build runs here, apart from
the test process that holds libidx.so.

    python tests/strict_cycle.py <case> <out.npz>
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_2304_13746_b300 import build as idx_build  # noqa: E402
from paper_2304_13746_b300 import idx, inputs  # noqa: E402

CASES = {
    "turb256": lambda: inputs.turbulent_box(256, seed=0),
    "turb40": lambda: inputs.turbulent_box(40, seed=3),
    "ot3d32": lambda: inputs.orszag_tang_3d(32),
    "ot2d64": lambda: inputs.orszag_tang_2d(64),
}


def main():
    case, out = sys.argv[1], sys.argv[2]
    idx.lib(idx_build.build(variant="strict"))
    ic = CASES[case]()
    s = idx.Sim(ic.shape, ic.lengths, ic.gamma, 0.4, "fp64")
    s.set_primitive(ic.prim)
    dt = s.step(want_dt=True)
    g = s.get_state()
    s.close()
    np.savez(out, dt=dt, **{f"f{f}": g[f] for f in range(8)})


if __name__ == "__main__":
    main()
