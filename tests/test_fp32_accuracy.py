"""FP32-bulk variant: its per-field L1 difference from the FP64 path stays below 10% of
the scheme's own discretisation error (Richardson estimate against the half-resolution
run, p = 2) at that resolution -- here the turbulent box at 128^3 advanced to t = 0.02."""
import pytest

from paper_2304_13746_b300 import accuracy
from paper_2304_13746_b300 import build as idx_build

pytestmark = pytest.mark.gpu


def test_fp32_error_below_tenth_of_discretisation_error():
    idx_build.build()
    r = accuracy.fp32_error_budget(128, 0.02)
    for name, v in r["fields"].items():
        print(f"{name}: e_fp32 {v['e_fp32']:.3e} e_disc {v['e_disc']:.3e} ratio {v['ratio']:.2e}")
    assert r["max_ratio"] < 0.1, r
