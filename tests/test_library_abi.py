"""CPU checks of the C-ABI library: it loads, exports every function that
include/smsm.h declares, and rejects bad arguments before touching CUDA."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "smsm.h")


@pytest.fixture(scope="module")
def lib():
    from paper_1901_01893_gb300 import _build, smsm

    _build.build()
    return smsm.lib()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(smsm_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for fn in ("smsm_plan", "smsm_forward", "smsm_adjoint", "smsm_hankel_gram", "smsm_apply_filters",
               "smsm_reconstruct"):
        assert fn in names


def test_library_exports_every_declared_symbol(lib):
    for fn in declared_functions():
        assert hasattr(lib, fn), fn


def test_default_params(lib):
    from paper_1901_01893_gb300 import smsm

    p = smsm.default_params()
    assert p.lambda_ == pytest.approx(1e-2) and p.eta == pytest.approx(1.5)
    assert p.outer_iters == 10 and p.cg_iters == 10 and p.mode == smsm.SMSM_MODE_IRLS


@pytest.mark.parametrize("args", [
    (0, 4, 8, 64, 64, 5),      # no slices
    (2, 4, 8, 64, 60, 5),      # nx != ny
    (2, 3, 8, 64, 64, 5),      # N not a multiple of the shot count
    (2, 4, 8, 70, 70, 5),      # 70 = 2*5*7 is not 2^a 3^b
    (2, 4, 8, 64, 64, 0),      # filter < 1
    (2, 4, 8, 64, 64, 13),     # filter too large
    (2, 8, 8, 64, 64, 7),      # C = 392 > 320
    (2, 16, 8, 64, 64, 2),     # more than 8 shots
])
def test_plan_rejects_bad_geometry(lib, args):
    from paper_1901_01893_gb300 import smsm

    h = ctypes.c_void_p()
    st = lib.smsm_plan(ctypes.byref(h), *args, None)
    assert st == smsm.SMSM_ERR_ARG
    assert not h.value
    assert lib.smsm_last_error().decode().startswith("smsm_plan")


def test_null_plan_is_an_error(lib):
    from paper_1901_01893_gb300 import smsm

    assert lib.smsm_forward(None, None, None, None, None) == smsm.SMSM_ERR_ARG
    assert lib.smsm_reconstruct(None, None, None, None, None, None) == smsm.SMSM_ERR_ARG
    assert lib.smsm_plan_destroy(None) == smsm.SMSM_OK


def test_group_and_sense_entry_points_check_arguments(lib):
    from paper_1901_01893_gb300 import smsm

    # no groups / missing arrays, and a NULL plan inside the list: rejected before any CUDA call
    assert lib.smsm_reconstruct_groups(0, None, None, None, None, None, None) == smsm.SMSM_ERR_ARG
    plans = (ctypes.c_void_p * 1)(None)
    ys = (ctypes.c_void_p * 1)(None)
    xs = (ctypes.c_void_p * 1)(None)
    assert lib.smsm_reconstruct_groups(1, plans, ys, xs, None, None, None) == smsm.SMSM_ERR_ARG
    assert lib.smsm_sense(None, None, None, None, 5, None, None) == smsm.SMSM_ERR_ARG


def test_plan_rejects_unknown_options(lib):
    from paper_1901_01893_gb300 import smsm

    for field, value in (("boundary", 7), ("precision", 9)):
        opts = smsm.Opts()
        setattr(opts, field, value)
        h = ctypes.c_void_p()
        assert lib.smsm_plan(ctypes.byref(h), 2, 4, 8, 64, 64, 5, ctypes.byref(opts)) == smsm.SMSM_ERR_ARG
        assert not h.value


def test_network_tuner_and_learned_start_check_arguments(lib):
    from paper_1901_01893_gb300 import smsm

    h = ctypes.c_void_p()
    # channel, width, layer, size and batch ranges are checked before any CUDA call
    for args in ((0, 64, 6, 32, 32, 1), (4, 0, 6, 32, 32, 1), (4, 64, 0, 32, 32, 1), (4, 64, 6, 0, 32, 1),
                 (4, 64, 6, 32, 32, 0), (300, 64, 6, 32, 32, 1)):
        assert lib.smsm_cnn_create(ctypes.byref(h), *args) == smsm.SMSM_ERR_ARG
        assert not h.value
    assert lib.smsm_cnn_create(None, 4, 8, 2, 16, 16, 1) == smsm.SMSM_ERR_ARG
    assert lib.smsm_cnn_param_count(None) == 0
    assert lib.smsm_cnn_destroy(None) == smsm.SMSM_OK
    assert lib.smsm_cnn_forward(None, None, None, 1, None) == smsm.SMSM_ERR_ARG
    assert lib.smsm_cnn_train_step(None, None, None, 1, ctypes.c_float(1e-3), None, None) == smsm.SMSM_ERR_ARG
    assert lib.smsm_learned_start(None, None, None, None, None) == smsm.SMSM_ERR_ARG
    assert lib.smsm_autotune(None, None, None, None, None) == smsm.SMSM_ERR_ARG
