"""Arithmetic-rate probes run and give plausible GB300 figures."""
import json
import os

import pytest

pytestmark = pytest.mark.gpu


def test_probe_peaks():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1612_08792_gb300 as gm
    r = gm.gmmsp_probe_peaks()
    assert r["sm_count"] >= 100
    assert 10.0 < r["fp32_fma_tflops"] < 200.0
    assert 10.0 < r["fp32x2_fma_tflops"] < 400.0
    assert 0.1 < r["fp64_fma_tflops"] < 100.0
    assert r["mufu_ex2_tops"] > 1.0
    assert r["fp32_fma_latency_clk"] > 1.0 and r["fp64_fma_latency_clk"] > 1.0
    out = os.environ.get("GMMSP_PROBE_OUT")
    if out:
        with open(out, "w") as fh:
            json.dump(r, fh, indent=1)


def test_fp64_helpers_within_their_error_bounds():
    """The finalize's FP64 helpers (gmmsp_math.cuh) against correctly rounded IEEE results on 10^6
    inputs over the finalize's range (weights, variances, determinants): 1/x and sqrt(x) from an FP32
    estimate and two Newton-Raphson steps, within 2 and 4 FP64 ulps; log2(x) as the exponent plus the
    FP32 log2 of the mantissa, within 3e-7 plus half an FP32 ulp of the result (the fast FP32 log2 is
    within 2^-22.6 on [1, 2), the mantissa's rounding to FP32 adds 2^-24 / ln 2)."""
    import numpy as np
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_1612_08792_gb300 as gm
    rng = np.random.default_rng(7)
    x = np.concatenate([10.0 ** rng.uniform(-30, 30, 1_000_000),
                        2.0 ** np.arange(-99, 100, dtype=np.float64),
                        np.nextafter(2.0 ** np.arange(-99, 100, dtype=np.float64), 0.0),
                        rng.uniform(1e-8, 1e4, 10_000), [1.0, 2.0, 3.0, 1e-8, 64.0, 8.0]])
    rcp, sq, lg = (t.cpu().numpy() for t in gm.gmmsp_probe_fp64_helpers(torch.from_numpy(x).cuda()))
    r_rcp, r_sq = 1.0 / x, np.sqrt(x)
    assert np.all(np.abs(rcp - r_rcp) <= 2 * np.spacing(r_rcp))
    assert np.all(np.abs(sq - r_sq) <= 4 * np.spacing(r_sq))
    r_lg = np.log2(x)
    bound = 3e-7 + 0.5 * np.spacing(np.abs(r_lg).astype(np.float32)).astype(np.float64)
    assert np.all(np.abs(lg.astype(np.float64) - r_lg) <= bound)
