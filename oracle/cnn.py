"""FP64 CPU oracle of the learned initialiser's network.

TEST INFRASTRUCTURE ONLY: used by ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s CPU legs, never by the product library, and sharing no code
with it.

The paper (Sec. III-C) starts EM from the cell-centre pixel with
Sigma_s = diag(v^2, v^2) and Sigma_c = lambda^2 I.  The learned initialiser
predicts a better start; the paper has no such network, so this module is
the plain definition of the network that the CUDA path implements:

  x0  3 x 3 pixel patches of each v x v cell (v = 3 f): 27 values
      (L/50 - 1, a/50, b/50 of the 9 pixels, channel (3 dy + dx) 3 + colour)
      and 5 zeros; f x f patches per cell
  h1 = ReLU(W1 x0 + b1), h2 = ReLU(W2 h1 + b2)        1 x 1 layers, 32 channels
  c0 = mean of h2 over the cell's patches              the n_x x n_y grid; channels
       29-31 replaced by the start point's pixel inputs (L/50 - 1, a/50, b/50)
  c_l = ReLU(conv3x3(c_{l-1}) + b_l), l = 1, 2, 3      zero padding
  out = conv3x3(c3) + b6                               16 channels, 10 used

Parameters are one flat vector W1, b1, W2, b2, ..., W6, b6 with
W[cout][tap * 32 + cin], tap = 3 dy + dx (0 for 1 x 1).  Outputs per
superpixel k, relative to the paper's start (x_c, y_c) = (k_x v + v // 2,
k_y v + v // 2) and the colour z_c there:
  0, 1  (mu_x - x_c) / v, (mu_y - y_c) / v
  2-4   (mu_colour - z_c) / 10
  5, 6  ln(Sigma_s,xx / v^2), ln(Sigma_s,yy / v^2)
  7-9   ln(Sigma_c,LL / lambda^2), ln(Sigma_c,aa / lambda^2), ln(Sigma_c,bb / lambda^2)

``emulate_bf16=True`` rounds to bfloat16 where the CUDA kernels store BF16
(inputs, weights, every hidden activation, the backward activation
gradients); arithmetic between those points stays FP64.  With it off the
module is the exact FP64 network, which the finite-difference pins check.

Pinned by tests/test_oracle_cnn.py: the 3 x 3 convolution against
scipy.signal.correlate2d, the patch layout against a brute-force index
formula, the pooling against a reshape mean, the backward pass against
central finite differences, the BF16 rounding against torch's conversion,
the target map against its inverse (theta0_from_outputs).
"""
from __future__ import annotations

import numpy as np

C = 32        # hidden channels
OUT = 16      # output channels
USED = 10     # used outputs
LAYERS = [(1, C), (1, C), (9, C), (9, C), (9, C), (9, OUT)]  # (taps, cout); cin = 32
IN_SCALE = 0.02
COLOUR_UNIT = 10.0
START_CH = 29  # c0 channels START_CH.. START_CH + 2 carry the start pixel's scaled colour


def start_inputs(x0, v: int):
    """The x0 inputs of the start pixel (k_x v + v // 2, k_y v + v // 2) of every cell:
    (B, n_y, n_x, 3), taken from the patch and the position inside it that hold it."""
    c = v // 2
    q, d = c // 3, c % 3
    ch = (d * 3 + d) * 3
    return x0[:, :, :, q, q, ch:ch + 3]


def param_count() -> int:
    return sum(cout * taps * C + cout for taps, cout in LAYERS)


def unpack(flat):
    """[(W (cout, taps*32), b (cout,)) for the six layers] (views, float64)."""
    flat = np.asarray(flat, dtype=np.float64)
    out, o = [], 0
    for taps, cout in LAYERS:
        W = flat[o:o + cout * taps * C].reshape(cout, taps * C)
        o += cout * taps * C
        b = flat[o:o + cout]
        o += cout
        out.append((W, b))
    assert o == flat.size
    return out


def pack(params) -> np.ndarray:
    return np.concatenate([np.concatenate([W.ravel(), b.ravel()]) for W, b in params])


def bf16(x):
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    x32 = np.asarray(x, dtype=np.float64).astype(np.float32)
    u = x32.view(np.uint32).astype(np.uint64)
    rounding = ((u >> 16) & 1) + 0x7FFF
    r = ((u + rounding) >> 16) << 16
    nan = np.isnan(x32)
    out = r.astype(np.uint32).view(np.float32).astype(np.float64)
    return np.where(nan, np.nan, out)


def grid(W: int, H: int, v: int):
    """Seed grid n_x, n_y of Eq. (nxyK) for spacing v."""
    return W // v, H // v


def patches(lab, v: int):
    """x0 of B images (lab: (B, 3, H, W) planes) -> (B, n_y, n_x, f, f, 32)."""
    lab = np.asarray(lab, dtype=np.float64)
    B, _, H, W = lab.shape
    f = v // 3
    nx, ny = grid(W, H, v)
    crop = lab[:, :, :ny * v, :nx * v]
    s = crop.reshape(B, 3, ny, f, 3, nx, f, 3)          # y = (ky, qy, dy), x = (kx, qx, dx)
    s = s.transpose(0, 2, 5, 3, 6, 4, 7, 1)            # (B, ky, kx, qy, qx, dy, dx, colour)
    s = s.reshape(B, ny, nx, f, f, 27).copy()
    s[..., 0::3] = s[..., 0::3] * IN_SCALE - 1.0
    s[..., 1::3] *= IN_SCALE
    s[..., 2::3] *= IN_SCALE
    x0 = np.zeros((B, ny, nx, f, f, C))
    x0[..., :27] = s
    return x0


def conv3x3(x, W, b):
    """Zero-padded 3 x 3 correlation: y[p] = b + sum_t W_t x[p + d_t], d_t = (dy-1, dx-1)."""
    B, H, Wd, cin = x.shape
    xp = np.zeros((B, H + 2, Wd + 2, cin))
    xp[:, 1:-1, 1:-1] = x
    y = np.broadcast_to(b, (B, H, Wd, W.shape[0])).copy()
    for dy in range(3):
        for dx in range(3):
            t = 3 * dy + dx
            y += xp[:, dy:dy + H, dx:dx + Wd, :] @ W[:, t * C:(t + 1) * C].T
    return y


def conv3x3_backward(x, W, g):
    """Gradients of sum(g * conv3x3(x, W, b)) w.r.t. x, W, b."""
    B, H, Wd, cin = x.shape
    xp = np.zeros((B, H + 2, Wd + 2, cin))
    xp[:, 1:-1, 1:-1] = x
    gxp = np.zeros_like(xp)
    gW = np.zeros_like(W)
    for dy in range(3):
        for dx in range(3):
            t = 3 * dy + dx
            Wt = W[:, t * C:(t + 1) * C]
            gW[:, t * C:(t + 1) * C] = np.einsum("bhwo,bhwc->oc", g, xp[:, dy:dy + H, dx:dx + Wd, :])
            gxp[:, dy:dy + H, dx:dx + Wd, :] += g @ Wt
    return gxp[:, 1:-1, 1:-1], gW, g.sum(axis=(0, 1, 2))


def forward(flat, lab, v: int, emulate_bf16: bool = False):
    """Network outputs (B, n_y, n_x, 16) and the activations for backward()."""
    rnd = bf16 if emulate_bf16 else (lambda a: a)
    P = unpack(flat)
    Wq = [rnd(W) for W, _ in P]
    bs = [b for _, b in P]
    x0 = rnd(patches(lab, v))
    h1 = rnd(np.maximum(x0 @ Wq[0].T + bs[0], 0.0))
    h2 = rnd(np.maximum(h1 @ Wq[1].T + bs[1], 0.0))
    c0 = h2.mean(axis=(3, 4))
    c0[..., START_CH:START_CH + 3] = start_inputs(x0, v)
    c0 = rnd(c0)
    c = [c0]
    for l in (2, 3, 4):
        c.append(rnd(np.maximum(conv3x3(c[-1], Wq[l], bs[l]), 0.0)))
    out = conv3x3(c[-1], Wq[5], bs[5])
    cache = dict(x0=x0, h1=h1, h2=h2, c=c, Wq=Wq, emulate=emulate_bf16)
    return out, cache


def loss(out, target):
    """Mean squared error over the used outputs; returns (loss, d loss / d out)."""
    out = np.asarray(out, dtype=np.float64)
    t = np.asarray(target, dtype=np.float64).reshape(out.shape[:-1] + (USED,))
    d = out[..., :USED] - t
    n = d.size
    g = np.zeros_like(out)
    g[..., :USED] = 2.0 * d / n
    return float((d * d).sum() / n), g


def backward(cache, g_out):
    """Flat gradient (the parameter layout) from d loss / d out."""
    rnd = bf16 if cache["emulate"] else (lambda a: a)
    Wq, c = cache["Wq"], cache["c"]
    grads = [None] * 6
    g = rnd(g_out)
    for l in (5, 4, 3, 2):
        x = c[l - 2]
        gx, gW, gb = conv3x3_backward(x, Wq[l], g)
        grads[l] = (gW, gb)
        g = rnd(gx * (x > 0)) if l > 2 else rnd(gx)   # c0 is a mean, without a ReLU
    h1, h2, x0 = cache["h1"], cache["h2"], cache["x0"]
    ff = h2.shape[3] * h2.shape[4]
    g = g.copy()
    g[..., START_CH:START_CH + 3] = 0.0      # those c0 channels are inputs, not pooled h2
    g2 = rnd(g[:, :, :, None, None, :] / ff * (h2 > 0))
    rows = lambda a: a.reshape(-1, a.shape[-1])  # noqa: E731  (all patch positions)
    grads[1] = (rows(g2).T @ rows(h1), rows(g2).sum(axis=0))
    g1 = rnd((g2 @ Wq[1]) * (h1 > 0))
    grads[0] = (rows(g1).T @ rows(x0), rows(g1).sum(axis=0))
    return pack(grads)


def centre(W: int, H: int, v: int):
    """Start points (x_c, y_c) of Sec. III-C for k = k_y n_x + k_x."""
    nx, ny = grid(W, H, v)
    k = np.arange(nx * ny)
    return (k % nx) * v + v // 2, (k // nx) * v + v // 2


def targets(mu, cs, cc, lab_img, v: int, lambda_c: float = 8.0):
    """Outputs that reproduce the given parameters of one image (K x 10).

    mu (K, 5), cs (K, 3) = (xx, xy, yy), cc (K, 6) = (LL, La, Lb, aa, ab, bb);
    lab_img (3, H, W)."""
    lab_img = np.asarray(lab_img, dtype=np.float64)
    _, H, W = lab_img.shape
    xc, yc = centre(W, H, v)
    zc = lab_img[:, yc, xc].T
    l2 = lambda_c * lambda_c
    t = np.zeros((len(xc), USED))
    t[:, 0] = (mu[:, 0] - xc) / v
    t[:, 1] = (mu[:, 1] - yc) / v
    t[:, 2:5] = (mu[:, 2:5] - zc) / COLOUR_UNIT
    t[:, 5] = np.log(cs[:, 0] / (v * v))
    t[:, 6] = np.log(cs[:, 2] / (v * v))
    t[:, 7] = np.log(cc[:, 0] / l2)
    t[:, 8] = np.log(cc[:, 3] / l2)
    t[:, 9] = np.log(cc[:, 5] / l2)
    return t


def theta0_from_outputs(out_img, lab_img, v: int, lambda_c: float = 8.0, eps_s: float = 2.0,
                        eps_c: float = 8.0):
    """theta_0 of one image from its outputs (K x >= 10): the inverse of targets(),
    with the spatial mean clipped to the three cells around the seed's own,
    [(k_x - 1) v, (k_x + 2) v] x [(k_y - 1) v, (k_y + 2) v] (the span of Eq. Ik's
    window without its clamp to the image, so a border seed's mean may start up
    to one cell outside the image), and the diagonal covariances floored at eps
    (Eq. mlams, mlamc); exponents limited to [-10, 10]."""
    o = np.asarray(out_img, dtype=np.float64).reshape(-1, np.shape(out_img)[-1])
    lab_img = np.asarray(lab_img, dtype=np.float64)
    _, H, W = lab_img.shape
    nx, _ = grid(W, H, v)
    xc, yc = centre(W, H, v)
    kx, ky = np.arange(len(xc)) % nx, np.arange(len(xc)) // nx
    zc = lab_img[:, yc, xc].T
    mu = np.zeros((len(xc), 5))
    mu[:, 0] = np.clip(xc + v * o[:, 0], (kx - 1) * v, (kx + 2) * v)
    mu[:, 1] = np.clip(yc + v * o[:, 1], (ky - 1) * v, (ky + 2) * v)
    mu[:, 2:5] = zc + COLOUR_UNIT * o[:, 2:5]
    e = np.exp(np.clip(o[:, 5:10].astype(np.float32), -10.0, 10.0).astype(np.float64))
    l2 = lambda_c * lambda_c
    cs = np.zeros((len(xc), 3))
    cs[:, 0] = np.maximum(v * v * e[:, 0], eps_s)
    cs[:, 2] = np.maximum(v * v * e[:, 1], eps_s)
    cc = np.zeros((len(xc), 6))
    cc[:, 0] = np.maximum(l2 * e[:, 2], eps_c)
    cc[:, 3] = np.maximum(l2 * e[:, 3], eps_c)
    cc[:, 5] = np.maximum(l2 * e[:, 4], eps_c)
    return mu, cs, cc
