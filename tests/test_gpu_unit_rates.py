"""The unit-rate probe that sets the assembly's roofline: every rate is
finite, none exceeds what the SM's units can issue at the highest SM clock
(a probe whose work was folded away would), and the units rank as their
widths say (FP32 FMA over the MUFU over FP64 FMA over any FP64 library
call built from several FP64 operations)."""
import math

import pytest
import torch

from paper_2203_11733_gb300 import build as B
from paper_2203_11733_gb300 import gbem

pytestmark = pytest.mark.gpu

MAX_SM_HZ = 2.2e9   # above the part's 2.07 GHz maximum SM clock


@pytest.fixture(scope="module")
def rates():
    B.build()
    gbem.load()
    torch.cuda.set_device(0)
    ctx = gbem.Context(0)
    r = ctx.unit_rates(torch.cuda.Stream())
    ctx.close()
    return r


def test_rates_finite_and_below_issue_limit(rates):
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    assert set(rates) == set(gbem.UNIT_RATE_NAMES)
    for k, v in rates.items():
        assert math.isfinite(v) and v > 0, k
    # 128 FP32 lanes and 16 MUFU lanes per SM per clock
    assert rates["ffma"] <= sms * 128 * MAX_SM_HZ
    assert rates["mufu_rsqrt"] <= sms * 16 * MAX_SM_HZ
    assert rates["ffma"] >= 0.25 * sms * 128 * 1.0e9


def test_rates_rank_as_the_units(rates):
    assert rates["ffma"] > rates["mufu_rsqrt"] > rates["dfma"]
    for k in ("dsqrt", "dlog", "datan", "drsqrt"):
        assert rates[k] < rates["dfma"], k
