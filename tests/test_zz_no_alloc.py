"""The allocation-free entry point, gmmsp_segment_lab_noalloc.

It serves callers that cannot allocate device memory where they run (a
memory pool or caching allocator that owns the device memory, code that must
not cause the synchronisation cudaMalloc/cudaFree can, plug-ins handed only
their buffers): the library keeps its working memory in one fixed device
array.  This test calls it through the C ABI twice in a row, on two
different images, and checks each result against the context-based entry
points (gmmsp_init + gmmsp_em_iters + gmmsp_labels).  Both run the same
kernels on the same FP32 values, so the labels must be identical; against the
FP64 oracle they meet the parity bar of the other tests.  The file is named
so that pytest collects it last.
"""
import numpy as np
import pytest

import oracle
from synth import voronoi_image
from tests import parity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gm():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_1612_08792_gb300 as gm
    torch.cuda.set_device(0)
    return gm


def lab_image(W, H, seed):
    return oracle.rgb2lab(voronoi_image(W, H, 150, 8.0, seed)).astype(np.float32)


def reference_labels(gm, lab, K, iters):
    sp = gm.Superpixels(lab, K=K)
    sp.em_iters(iters)
    out = sp.labels().cpu().numpy()
    sp.close()
    return out


def test_noalloc_matches_context_path_twice(gm):
    import torch
    W, H, K, T = 481, 321, 1000, 10
    p = gm.gmmsp_default_params()
    p.K = K
    out = torch.full((H, W), -1, dtype=torch.int32, device="cuda")
    for seed in (0, 1):  # two calls in a row share the scratch array
        lab = lab_image(W, H, seed)
        dev = torch.from_numpy(lab).cuda()
        gm.gmmsp_segment_lab_noalloc(dev, W, H, W * 12, p, T, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        np.testing.assert_array_equal(got, reference_labels(gm, dev, K, T))
        ref = oracle.em(lab.astype(np.float64), W, H, K=K, T=T)
        agree, ndiff, worst = parity.label_report(got, ref.labels, ref.margin)
        assert agree >= parity.LABEL_AGREE and worst < parity.MARGIN_TOL, (seed, agree, ndiff, worst)


def test_noalloc_pitched_rows(gm):
    """Rows further apart than 12 W bytes; the padding holds NaN, which must never be read."""
    import torch
    W, H, T = 200, 150, 6
    p = gm.gmmsp_default_params()
    p.spacing = 12
    lab = lab_image(W, H, 5)
    padded = np.full((H, W + 7, 3), np.nan, dtype=np.float32)
    padded[:, :W] = lab
    dev = torch.from_numpy(padded).cuda()
    out = torch.full((H, W), -1, dtype=torch.int32, device="cuda")
    gm.gmmsp_segment_lab_noalloc(dev, W, H, (W + 7) * 12, p, T, out)
    torch.cuda.synchronize()
    sp = gm.Superpixels(torch.from_numpy(lab).cuda(), spacing=12)
    sp.em_iters(T)
    np.testing.assert_array_equal(out.cpu().numpy(), sp.labels().cpu().numpy())
    sp.close()


def test_noalloc_rejects_bad_parameters(gm):
    import torch
    W, H = 64, 48
    lab = torch.zeros((H, W, 3), dtype=torch.float32, device="cuda")
    out = torch.empty((H, W), dtype=torch.int32, device="cuda")
    for field, value in (("eps_s", float("inf")), ("eps_c", float("nan")), ("lambda_c", 0.0)):
        p = gm.gmmsp_default_params()
        p.spacing = 8
        setattr(p, field, value)
        with pytest.raises(gm.GmmspError) as ei:
            gm.gmmsp_segment_lab_noalloc(lab, W, H, W * 12, p, 2, out)
        assert ei.value.status == 1


def test_noalloc_rejects_grids_beyond_its_limit(gm):
    import torch
    W, H = 1920, 1080
    p = gm.gmmsp_default_params()
    p.spacing = 4  # 480 x 270 cells > 4096
    lab = torch.zeros((H, W, 3), dtype=torch.float32, device="cuda")
    out = torch.empty((H, W), dtype=torch.int32, device="cuda")
    with pytest.raises(gm.GmmspError) as ei:
        gm.gmmsp_segment_lab_noalloc(lab, W, H, W * 12, p, 2, out)
    assert ei.value.status == 1 and "4096" in str(ei.value)
