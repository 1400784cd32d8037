"""Plain FP64 CPU oracle for the GMM superpixel EM (arXiv 1612.08792).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline / reference legs of ``bench.py`` may import this package.
The product library (``paper_1612_08792_gb300``) never imports, links or
runs anything here, and nothing here imports the product library.

The arithmetic lives in ``gmmsp_oracle.c`` (double precision, one routine per
equation of the paper; see its header for the equation map).  This module
only compiles it with the host C compiler (once, on first use, or from
``build()``) and marshals numpy arrays through ``ctypes``.

Every function is pinned by tests against something other than itself
(closed forms, brute-force mixtures evaluated with scipy, numpy moments and
eigen-decompositions, published CIELAB values).  No function here is
"parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gmmsp_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

MAXC = 9  # |K_i| <= 9 (Sec. III-D)

# Colour models (the `colour` argument below): the full 3x3 colour covariance
# of Eq. (BlockSigma), the L | (a, b) split of Eq. (BlockSigma1), and a
# grayscale image whose scalar colour is CIE L* (Sec. III-A, III-C).
COLOUR_FULL, COLOUR_SPLIT, COLOUR_GRAY = 0, 1, 2
_COLOUR_NAMES = {"full": COLOUR_FULL, "split": COLOUR_SPLIT, "gray": COLOUR_GRAY}


def _cm(colour) -> int:
    c = _COLOUR_NAMES.get(colour, colour) if isinstance(colour, str) else int(colour)
    if c not in (COLOUR_FULL, COLOUR_SPLIT, COLOUR_GRAY):
        raise ValueError(f"unknown colour model {colour!r}")
    return c


def build(force: bool = False) -> str:
    """Compile the C oracle into ``oracle/_build/liboracle.so`` (gcc, -O2, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        I = ctypes.c_int
        L = ctypes.c_long
        D = ctypes.c_double
        sig = {
            "orc_set_threads": (None, [I]),
            "orc_max_threads": (I, []),
            "orc_rgb2lab": (None, [P, L, P]),
            "orc_gray2l": (None, [P, L, P]),
            "orc_grid": (I, [I, I, I, I, P]),
            "orc_candidates": (I, [I, I, I, I, I, P, P]),
            "orc_eig_clamp": (I, [I, P, D, P]),
            "orc_sym_eigvals": (None, [I, P, P]),
            "orc_init": (None, [P, I, I, I, I, I, D, P, P, P, I]),
            "orc_log_gauss": (D, [P, P, P, P, I]),
            "orc_estep": (D, [P, I, I, I, P, P, P, P, P, P, P, I]),
            "orc_mstep": (I, [P, I, I, I, I, I, P, P, P, D, D, P, P, P, P, P, P, P, I]),
            "orc_labels": (None, [L, P, P, P, P, P]),
            "orc_em": (I, [P, I, I, I, I, I, D, D, D, P, P, P, P, P, P, P, P, P, P, P, P, P, I]),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
        return lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


def set_threads(n: int) -> None:
    _load().orc_set_threads(int(n))


def max_threads() -> int:
    return int(_load().orc_max_threads())


# ---------------------------------------------------------------- CIELAB
def rgb2lab(rgb: np.ndarray) -> np.ndarray:
    """sRGB uint8 (..., 3) -> CIELAB float64 (..., 3); D65 white (Sec. IV)."""
    rgb = np.ascontiguousarray(rgb, dtype=np.uint8)
    assert rgb.shape[-1] == 3
    out = np.empty(rgb.shape, dtype=np.float64)
    _load().orc_rgb2lab(_ptr(rgb), int(rgb.size // 3), _ptr(out))
    return out


def gray2l(gray: np.ndarray) -> np.ndarray:
    """Grey levels uint8 (...) -> CIE L* float64 (...): L* of Y = sRGB-decode(g / 255)."""
    gray = np.ascontiguousarray(gray, dtype=np.uint8)
    out = np.empty(gray.shape, dtype=np.float64)
    _load().orc_gray2l(_ptr(gray), int(gray.size), _ptr(out))
    return out


# ---------------------------------------------------------------- grid
@dataclass(frozen=True)
class Grid:
    W: int
    H: int
    v: int
    nx: int
    ny: int
    K: int


def grid(W: int, H: int, K: int = 0, spacing: int = 0) -> Grid:
    """Eq. (vxy) / Eq. (nxyK).  Raises ValueError when the grid is empty."""
    out = np.zeros(4, dtype=np.int32)
    rc = _load().orc_grid(int(W), int(H), int(K), int(spacing), _ptr(out))
    if rc != 0:
        raise ValueError(f"empty grid for W={W} H={H} K={K} spacing={spacing}")
    return Grid(W, H, int(out[0]), int(out[1]), int(out[2]), int(out[3]))


def candidates(g: Grid):
    """Candidate sets K_i (Eq. Ik): (cand[N, 9] ascending, ncand[N])."""
    N = g.W * g.H
    cand = np.full((N, MAXC), -1, dtype=np.int32)
    ncand = np.zeros(N, dtype=np.int32)
    rc = _load().orc_candidates(g.W, g.H, g.v, g.nx, g.ny, _ptr(cand), _ptr(ncand))
    if rc != 0:
        raise RuntimeError(f"orc_candidates failed: {rc}")
    return cand, ncand


# ---------------------------------------------------------------- model
@dataclass
class Theta:
    """theta_k = (mu_k, Sigma_k,s, Sigma_k,c) for all k, float64.

    mu: (K, 5) = (x, y, L, a, b); cs: (K, 3) = (xx, xy, yy);
    cc: (K, 6) = (LL, La, Lb, aa, ab, bb).  Split model: La = Lb = 0;
    grayscale: mu's a, b and every cc entry but LL are 0.
    """
    mu: np.ndarray
    cs: np.ndarray
    cc: np.ndarray

    def copy(self) -> "Theta":
        return Theta(self.mu.copy(), self.cs.copy(), self.cc.copy())


def init_theta(lab: np.ndarray, g: Grid, lambda_c: float = 8.0, colour="full") -> Theta:
    """Sec. III-C initialisation: centre pixels, diag(v^2, v^2), lambda^2 I."""
    lab = _f64(lab, (g.H * g.W, 3))
    th = Theta(np.zeros((g.K, 5)), np.zeros((g.K, 3)), np.zeros((g.K, 6)))
    _load().orc_init(_ptr(lab), g.W, g.H, g.v, g.nx, g.ny, float(lambda_c),
                     _ptr(th.mu), _ptr(th.cs), _ptr(th.cc), _cm(colour))
    return th


def log_gauss(z, mu, cs, cc, colour="full") -> float:
    """ln p(z; theta_k), Eq. (gaussian) with the block covariance."""
    return float(_load().orc_log_gauss(_ptr(_f64(z)), _ptr(_f64(mu)), _ptr(_f64(cs)), _ptr(_f64(cc)),
                                       _cm(colour)))


def estep(lab: np.ndarray, g: Grid, th: Theta, cand=None, ncand=None, colour="full"):
    """Eq. (Rik).  Returns (R[N, 9], ll[N], L(theta), cand, ncand)."""
    if cand is None:
        cand, ncand = candidates(g)
    lab = _f64(lab, (g.H * g.W, 3))
    N = g.W * g.H
    R = np.zeros((N, MAXC))
    ll = np.zeros(N)
    L = _load().orc_estep(_ptr(lab), g.W, g.H, g.K, _ptr(cand), _ptr(ncand),
                          _ptr(_f64(th.mu)), _ptr(_f64(th.cs)), _ptr(_f64(th.cc)), _ptr(R), _ptr(ll),
                          _cm(colour))
    return R, ll, float(L), cand, ncand


def mstep(lab: np.ndarray, g: Grid, th: Theta, R, cand, ncand, eps_s: float = 2.0, eps_c: float = 8.0,
          colour="full"):
    """Eq. (UpdateMu), (UpdateSigS), (UpdateSigC) and the floor (mlams, mlamc).

    Returns (theta_{t+1}, raw spatial cov, raw colour cov, wsum, dead, (raised_s, raised_c)).
    """
    lab = _f64(lab, (g.H * g.W, 3))
    out = th.copy()
    cs_raw = np.zeros((g.K, 3))
    cc_raw = np.zeros((g.K, 6))
    wsum = np.zeros(g.K)
    nr = np.zeros(2, dtype=np.int32)
    dead = _load().orc_mstep(_ptr(lab), g.W, g.H, g.v, g.nx, g.ny, _ptr(cand), _ptr(ncand),
                             _ptr(_f64(R)), float(eps_s), float(eps_c),
                             _ptr(out.mu), _ptr(out.cs), _ptr(out.cc), _ptr(cs_raw), _ptr(cc_raw),
                             _ptr(wsum), _ptr(nr), _cm(colour))
    return out, cs_raw, cc_raw, wsum, int(dead), (int(nr[0]), int(nr[1]))


def eig_clamp(packed: np.ndarray, eps: float) -> tuple[np.ndarray, int]:
    """Eq. (eigdecs)-(eigdecrc): floor the eigenvalues of one packed 1x1 (1), 2x2 (3) or 3x3 (6)."""
    p = _f64(packed)
    n = {1: 1, 3: 2, 6: 3}[p.size]
    out = np.zeros_like(p)
    raised = _load().orc_eig_clamp(n, _ptr(p), float(eps), _ptr(out))
    return out, int(raised)


def sym_eigvals(packed: np.ndarray) -> np.ndarray:
    p = _f64(packed)
    n = {3: 2, 6: 3}[p.size]
    lam = np.zeros(n)
    _load().orc_sym_eigvals(n, _ptr(p), _ptr(lam))
    return lam


def labels_from_posteriors(R, cand, ncand):
    """Eq. (obtLi).  Returns (labels[N] int32, margin[N])."""
    N = R.shape[0]
    labels = np.zeros(N, dtype=np.int32)
    margin = np.zeros(N)
    _load().orc_labels(N, _ptr(cand), _ptr(ncand), _ptr(_f64(R)), _ptr(labels), _ptr(margin))
    return labels, margin


@dataclass
class EMResult:
    grid: Grid
    theta: Theta
    labels: np.ndarray      # (H, W) int32
    margin: np.ndarray      # (H, W) R_(1) - R_(2) of the last E-step
    loglik: np.ndarray      # (T+1,) L(theta_t), natural log
    post: np.ndarray | None
    cand: np.ndarray | None
    ncand: np.ndarray | None
    raised: np.ndarray      # (T, 2) raised eigenvalue counts
    dead: int


def em(lab: np.ndarray, W: int, H: int, K: int = 0, spacing: int = 0, T: int = 10,
       lambda_c: float = 8.0, eps_s: float = 2.0, eps_c: float = 8.0,
       theta0: Theta | None = None, keep_post: bool = False, colour="full") -> EMResult:
    """Algorithm 1, steps 1-7, on an (H, W, 3) CIELAB image (float, any precision).

    colour: "full" (Eq. BlockSigma), "split" (Eq. BlockSigma1) or "gray" (only
    the L column of lab is read)."""
    g = grid(W, H, K, spacing)
    lab = _f64(lab, (H * W, 3))
    th = Theta(np.zeros((g.K, 5)), np.zeros((g.K, 3)), np.zeros((g.K, 6)))
    labels = np.zeros(H * W, dtype=np.int32)
    margin = np.zeros(H * W)
    loglik = np.zeros(T + 1)
    raised = np.zeros((max(T, 1), 2), dtype=np.int32)
    post = np.zeros((H * W, MAXC)) if keep_post else None
    cand = np.zeros((H * W, MAXC), dtype=np.int32) if keep_post else None
    ncand = np.zeros(H * W, dtype=np.int32) if keep_post else None
    if theta0 is not None:
        mu_in, cs_in, cc_in = _f64(theta0.mu), _f64(theta0.cs), _f64(theta0.cc)
    else:
        mu_in = cs_in = cc_in = None
    rc = _load().orc_em(_ptr(lab), W, H, int(K), int(spacing), int(T), float(lambda_c),
                        float(eps_s), float(eps_c), _ptr(mu_in), _ptr(cs_in), _ptr(cc_in),
                        _ptr(th.mu), _ptr(th.cs), _ptr(th.cc), _ptr(labels), _ptr(margin),
                        _ptr(loglik), _ptr(post), _ptr(cand), _ptr(ncand), _ptr(raised), _cm(colour))
    if rc < 0:
        raise RuntimeError(f"orc_em failed: {rc}")
    return EMResult(g, th, labels.reshape(H, W), margin.reshape(H, W), loglik, post, cand, ncand,
                    raised[:T], int(rc))
