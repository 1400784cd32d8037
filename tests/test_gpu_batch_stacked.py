"""The batch context's stacked-input entry and its label buffer.

segment_stacked takes the n images of a batch of one size as one (n, H, W, C)
tensor and computes their addresses from its strides; it must give exactly the
labels segment gives on the same images as a list, and the context's
labels_buffer must hold every image's labels, image after image (what a caller
copies to the host in one transfer).  Covers RGB8 and float32 CIELAB input,
packed rows and rows wider than the image.
"""
import numpy as np
import pytest

from synth import voronoi_image

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gm():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_1612_08792_gb300 as gm
    torch.cuda.set_device(0)
    return gm


@pytest.mark.parametrize("lab_input,pad", [(False, 0), (False, 5), (True, 0), (True, 3)])
def test_segment_stacked_matches_segment(gm, lab_input, pad):
    import oracle
    import torch
    W, H, B, v = 97, 61, 4, 8
    imgs = [voronoi_image(W + pad, H, 12, 8.0, 9_100_000 + i) for i in range(B)]
    if lab_input:
        imgs = [oracle.rgb2lab(x).astype(np.float32) for x in imgs]
    stacked = torch.from_numpy(np.stack(imgs)).cuda()[:, :, :W]   # rows pitch (W + pad) C
    listed = [stacked[i] for i in range(B)]

    a = gm.SuperpixelsBatch([(H, W)] * B, spacing=v, lab_input=lab_input)
    ref = [x.clone() for x in a.segment(listed, iters=3)]
    got = a.segment_stacked(stacked, iters=3)
    torch.cuda.synchronize()
    for i in range(B):
        assert torch.equal(got[i], ref[i]), i
    flat = a.labels_buffer.cpu().numpy()
    assert np.array_equal(flat, np.concatenate([r.cpu().numpy().ravel() for r in ref]))
    with pytest.raises(ValueError):
        a.segment_stacked(stacked[:, :, : W - 1], iters=1)
    a.close()
