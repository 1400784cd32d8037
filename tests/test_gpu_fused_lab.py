"""The learned start's converting first kernel against the plain conversion.

With a network set and RGB8 input, the batch converts the pixels of the
n_x v x n_y v cell region inside the network's first kernel (it reads them
for the 3 x 3 patches anyway) and the conversion pass only the rest.  Both
must give the CIELAB planes of the conversion pass bit for bit, and the
network must see the same inputs: theta_0 from RGB8 input equals theta_0 from
those CIELAB planes given as float32 input (the unfused path), exactly.
Cases cover the spacings 3 (128 cells per block), 12, 15 and 33 (one cell
per block), sizes with remainder strips on both sides and with none, a
partial last block, row pitches wider than the image and images whose
first byte is not 4-byte aligned.
"""
import numpy as np
import pytest

from synth import voronoi_image

pytestmark = pytest.mark.gpu

CASES = [
    (15, 481, 321, 3, 0),
    (15, 487, 331, 2, 16),
    (15, 480, 315, 2, 3),
    (3, 64, 37, 2, 0),
    (12, 97, 61, 3, 5),
    (15, 481, 321, 2, 7),
    (33, 100, 70, 2, 0),
]


@pytest.fixture(scope="module")
def gm():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_1612_08792_gb300 as gm
    torch.cuda.set_device(0)
    return gm


def rgb_images(W, H, B, pad, seed):
    """B RGB8 CUDA tensors of W x H; with pad > 0 each is a view of a wider image (pitch 3 (W + pad))
    that starts pad // 2 columns in, so that its first byte is not 4-byte aligned when pad // 2 is
    odd (the converting kernel reads the patch rows as aligned words)."""
    import torch
    out = []
    for i in range(B):
        img = voronoi_image(W + pad, H, 40, 8.0, seed + i)
        x0 = pad // 2
        out.append(torch.from_numpy(img).cuda()[:, x0:x0 + W])
    return out


@pytest.mark.parametrize("v,W,H,B,pad", CASES)
def test_fused_conversion_and_learned_start_match_unfused(gm, v, W, H, B, pad):
    import torch
    from paper_1612_08792_gb300.learned_init import InitNet
    imgs = rgb_images(W, H, B, pad, 7_000_000 + 31 * v + W)
    shapes = [(H, W)] * B
    K = (W // v) * (H // v)

    plain = gm.SuperpixelsBatch(shapes, spacing=v)
    plain.segment(imgs, iters=0)
    torch.cuda.synchronize()
    lab_ref = [plain.get_lab(i) for i in range(B)]
    plain.close()

    net = InitNet(v, seed=11)
    fused = gm.SuperpixelsBatch(shapes, spacing=v)
    fused.set_init_net(net)
    fused.segment(imgs, iters=0)
    torch.cuda.synchronize()
    for i in range(B):
        lab = fused.get_lab(i)
        assert np.array_equal(lab.view(np.uint32), lab_ref[i].view(np.uint32)), (v, W, H, i)
    th_fused = [fused.get_params(i, K) for i in range(B)]
    fused.close()

    unfused = gm.SuperpixelsBatch(shapes, spacing=v, lab_input=True)
    unfused.set_init_net(net)
    unfused.segment([torch.from_numpy(np.ascontiguousarray(x)).cuda() for x in lab_ref], iters=0)
    torch.cuda.synchronize()
    for i in range(B):
        for a, b in zip(th_fused[i], unfused.get_params(i, K)):
            assert np.array_equal(a, b), (v, W, H, i)
    net.check()
    unfused.close()
    net.close()
