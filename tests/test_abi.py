"""The C ABI library: it loads without a GPU, exports every function that
include/gmmsp.h declares, and rejects invalid arguments on the host before
any CUDA call (these calls return before touching the device)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if h.endswith(".h"):
            text = open(os.path.join(ROOT, "include", h)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_ ]*?\**\s*\b(gmmsp_[a-z0-9_]+)\s*\(",
                                text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_1612_08792_gb300 import build
    build.build()
    import paper_1612_08792_gb300 as gm
    return gm.load_library()


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert "gmmsp_init" in names and "gmmsp_em_iters" in names and "gmmsp_labels" in names
    for n in names:
        assert hasattr(lib, n), f"{n} declared in include/ but not exported"


def test_default_params(lib):
    import paper_1612_08792_gb300 as gm
    p = gm.gmmsp_default_params()
    assert (p.spacing, p.K, p.eps_s, p.eps_c, p.lambda_c) == (0, 0, 2.0, 8.0, 8.0)
    assert p.input_format == gm.GMMSP_RGB8 and p.precision == gm.GMMSP_PREC_MIXED
    assert p.colour_model == gm.GMMSP_COLOUR_FULL
    assert gm.gmmsp_status_string(1) == "GMMSP_E_INVALID"


@pytest.mark.parametrize("fmt,prec,cm,pitch,batch_too", [
    (0, 0, 3, 960, True),      # unknown colour model
    (0, 0, -1, 960, True),
    (0, 1, 1, 960, True),      # FP32 precision with the split model
    (1, 1, 2, 3840, True),     # FP32 precision with grayscale
    (2, 0, 0, 320, True),      # grey-level input with the full model
    (2, 0, 1, 320, True),      # ... or the split one
    (2, 0, 2, 319, False),     # grey-level rows need W bytes (a batch checks pitches when it segments)
    (3, 0, 0, 960, True),      # unknown format
])
def test_colour_model_combinations_rejected_on_host(lib, fmt, prec, cm, pitch, batch_too):
    import paper_1612_08792_gb300 as gm
    p = gm.gmmsp_default_params()
    p.spacing, p.input_format, p.precision, p.colour_model = 12, fmt, prec, cm
    ctx = ctypes.c_void_p(1234)
    assert lib.gmmsp_init(ctypes.byref(ctx), 0x1000, 320, 240, pitch, ctypes.byref(p), None) == 1
    assert not ctx.value
    if batch_too:
        b = ctypes.c_void_p(1234)
        W, H = (ctypes.c_int * 1)(320), (ctypes.c_int * 1)(240)
        assert lib.gmmsp_batch_create(ctypes.byref(b), 1, W, H, ctypes.byref(p), None) == 1
        assert not b.value


@pytest.mark.parametrize("W,H,K,sp,pitch,eps", [
    (0, 240, 0, 12, 960, 8.0),       # empty image
    (320, 240, 1, 0, 960, 8.0),      # K = 1 -> v = 277 > H: empty grid
    (320, 240, 0, 0, 960, 8.0),      # neither K nor spacing
    (320, 240, 0, 12, 959, 8.0),     # pitch < 3 W
    (320, 240, 0, 12, 960, 0.0),     # eps must be positive
    (10, 10, 0, 11, 30, 8.0),        # spacing larger than the image
])
def test_invalid_arguments_rejected_on_host(lib, W, H, K, sp, pitch, eps):
    import paper_1612_08792_gb300 as gm
    p = gm.gmmsp_default_params()
    p.K, p.spacing, p.eps_c = K, sp, eps
    ctx = ctypes.c_void_p(1234)
    st = lib.gmmsp_init(ctypes.byref(ctx), 0x1000, W, H, pitch, ctypes.byref(p), None)
    assert st == 1 and not ctx.value


def test_null_context_calls(lib):
    assert lib.gmmsp_em_iters(None, 1, None) == 1
    assert lib.gmmsp_labels(None, None, None) == 1
    assert lib.gmmsp_batch_set_first_pass(None, 6) == 1
    assert lib.gmmsp_batch_get_first_pass(None, None, None) == 1
    lib.gmmsp_destroy(None)


def test_network_host_checks(lib):
    # parameter count without a device; bad spacings and null handles rejected on the host
    assert lib.gmmsp_net_param_count() == 34480
    out = ctypes.c_void_p(1234)
    for sp in (0, 2, 14, 36):
        assert lib.gmmsp_net_create(ctypes.byref(out), sp, None) == 1
        assert out.value is None
    assert lib.gmmsp_net_set_weights(None, None, 0) == 1
    assert lib.gmmsp_net_check(None) == 1
    assert lib.gmmsp_batch_set_init_net(None, None) == 1
    assert lib.gmmsp_init_from_net(None, None) == 1


def test_bounds_status_of_the_ordinary_build(lib):
    """The ordinary library has the checks compiled out and says so without touching a device;
    the status word decodes as (1 << 63) | site << 40 | (index mod 2^40)."""
    import paper_1612_08792_gb300 as gm
    assert gm.gmmsp_bounds_status() == (False, None)
    code = (1 << 63) | (5 << 40) | 1234
    assert gm.bounds_decode(code) == {"site": "partial_read", "index": 1234}
    assert gm.bounds_decode((1 << 63) | (2 << 40) | ((-3) & ((1 << 40) - 1))) == {"site": "pixel_x", "index": -3}
    assert gm.bounds_decode(0) is None
