"""The allocation-free entry point, gmmsp_segment_lab_noalloc.

It serves callers that cannot allocate device memory where they run (a
memory pool or caching allocator that owns the device memory, code that must
not cause the synchronisation cudaMalloc/cudaFree can, plug-ins handed only
their buffers): the library keeps its working memory in one fixed device
array.  This test calls it through the C ABI twice in a row, on two
different images, and checks each result against the context-based entry
points (gmmsp_init + gmmsp_em_iters + gmmsp_labels) with the label tolerance
the other parity tests use.  The file is named so that pytest collects it
last.
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


def lab_tensor(W, H, seed):
    import torch
    lab = oracle.rgb2lab(voronoi_image(W, H, 150, 8.0, seed)).astype(np.float32)
    return torch.from_numpy(lab).cuda()


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
        lab = lab_tensor(W, H, seed)
        gm.gmmsp_segment_lab_noalloc(lab, W, H, W * 12, p, T, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        ref = reference_labels(gm, lab, K, T)
        agree = (got == ref).mean()
        assert agree >= parity.LABEL_AGREE, (seed, agree)
        # labels name superpixels of the grid
        assert got.min() >= 0 and got.max() < 40 * 26


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
