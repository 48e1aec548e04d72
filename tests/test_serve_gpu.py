"""The serving loop on the GPU: every served result equals the same request advanced
alone (idx_advance) within the stated tolerance; a request with a non-physical initial
state fails on its own without disturbing the others; memory stays within the budget."""
import numpy as np
import pytest

from paper_2304_13746_b300 import build as idx_build
from paper_2304_13746_b300 import idx, serve

pytestmark = pytest.mark.gpu


def _scaled_error(got, ref):
    rho, E = np.abs(ref[0]), np.abs(ref[4])
    msc = float(np.max(np.sqrt(2.0 * rho * E)))
    bsc = float(np.max(np.sqrt(2.0 * E)))
    own = [float(np.max(np.abs(ref[f]))) for f in range(8)]
    sc = [own[0], max(own[1], msc), max(own[2], msc), max(own[3], msc), own[4],
          max(own[5], bsc), max(own[6], bsc), max(own[7], bsc)]
    return max(float(np.max(np.abs(got[f] - ref[f]))) / sc[f] for f in range(8))


def test_served_results_equal_alone_and_failures_are_isolated():
    idx_build.build()
    reqs = serve.make_payloads(serve.poisson_stream(10, 200.0, seed=11, sizes_2d=(16, 64),
                                                    sizes_3d=(8, 24), t_end=(0.005, 0.02)))
    bad = reqs[3]
    bad.payload.prim[4][0, 0, 0] = -1.0                 # negative pressure
    budget = 3 * max(idx.footprint(r.payload.shape) for r in reqs)
    be = serve.IdxBackend("fp64")
    srv = serve.Server(be, budget, cycles_per_poll=4)
    st = srv.run(reqs)
    be.close()
    assert bad.status == "failed" and "non-physical" in bad.error
    assert st["done"] == len(reqs) - 1 and srv.peak <= budget and srv.used == 0
    seq = serve.IdxSequential("fp64")
    for r in reqs:
        if r is bad:
            continue
        ref, n = seq.serve_one(r)
        assert r.cycles == n
        assert _scaled_error(r.state, ref) <= 1e-10, r.rid
