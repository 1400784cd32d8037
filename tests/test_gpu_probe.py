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


def test_probe_smem_patterns_run():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1612_08792_gb300 as gm
    gm.gmmsp_probe_smem_patterns()
