"""The C ABI: the library loads on a machine without a GPU and exports every
entry point that include/*.h declares, with the binding covering each one.
No compute call is made here."""
import ctypes as C
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?\w+\s*\*?\s*(\w+)\s*\(", src, flags=re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def tp():
    from paper_2408_03452_gb300 import build, tpfa
    build.build()
    return tpfa


def test_header_declares_the_hot_path_calls():
    names = _declared()
    for n in ("tpfa_build_trans", "tpfa_apply", "cg_solve", "tpfa_build_rhs", "tpfa_residual64",
              "tpfa_create", "tpfa_destroy", "tpfa_strerror"):
        assert n in names


def test_library_exports_every_declared_symbol(tp):
    L = C.CDLL(tp.LIB_PATH)
    for n in _declared():
        assert hasattr(L, n), f"{n} declared in include/ but not exported"


def test_binding_covers_every_declared_symbol(tp):
    assert _declared() <= set(tp.SIGNATURES), _declared() - set(tp.SIGNATURES)
    tp.lib()


def test_abi_version_and_strerror(tp):
    hdr = open(os.path.join(ROOT, "include", "tpfa.h")).read()
    ver = int(re.search(r"#define TPFA_ABI_VERSION (\d+)", hdr).group(1))
    assert tp.abi_version() == ver
    for code in range(-7, 2):
        assert tp.strerror(code) and tp.strerror(code) != "unknown status"
    assert tp.strerror(-99) == "unknown status"


def test_status_codes_match_header(tp):
    hdr = open(os.path.join(ROOT, "include", "tpfa.h")).read()
    for name, val in [("TPFA_OK", tp.OK), ("TPFA_NOTCONV", tp.NOTCONV), ("TPFA_EINVAL", tp.EINVAL),
                      ("TPFA_ENOMEM", tp.ENOMEM), ("TPFA_ECUDA", tp.ECUDA),
                      ("TPFA_EBREAKDOWN", tp.EBREAKDOWN), ("TPFA_ENONFINITE", tp.ENONFINITE),
                      ("TPFA_EINTERNAL", tp.EINTERNAL), ("TPFA_ESTAGNATION", tp.ESTAGNATION)]:
        m = re.search(rf"{name}\s*=\s*(-?\d+)", hdr)
        assert m and int(m.group(1)) == val, name
    for name, val in tp.OPTIONS.items():
        m = re.search(rf"TPFA_OPT_{name.upper()}\s*=\s*(\d+)", hdr)
        assert m and int(m.group(1)) == val, name


def test_null_context_is_rejected_without_a_gpu(tp):
    # argument checks that happen before any CUDA call
    assert tp.lib().tpfa_set_option(None, 1, 1e-6) == tp.EINVAL
    assert tp.lib().tpfa_create(None, None) == tp.EINVAL
    assert tp.lib().tpfa_destroy(None) == tp.EINVAL


def test_unet_parameter_layout_without_a_gpu(tp):
    """The library's parameter count equals the layer table of the Python
    side (W_i[27][cout][cin] then b_i[cout] per layer), and the counter-based
    initialisation fills exactly that many values; the network's argument
    checks reject a null handle before any CUDA call."""
    from paper_2408_03452_gb300 import learned
    n = sum(27 * ci * co + co for ci, co in learned.LAYERS)
    assert tp.unet_param_count() == n == 146625
    p = learned.init_params(3)
    assert p.numel() == n and p.dtype.is_floating_point
    off = 0
    for ci, co in learned.LAYERS:  # He scale per layer, zero biases
        w = p[off:off + 27 * ci * co].double()
        assert abs(float(w.std()) / (2.0 / (27 * ci)) ** 0.5 - 1.0) < 0.25
        assert float(p[off + 27 * ci * co:off + 27 * ci * co + co].abs().sum()) == 0.0
        off += 27 * ci * co + co
    L = tp.lib()
    assert L.tpfa_unet_destroy(None) == tp.EINVAL
    assert L.tpfa_unet_set_params(None, None, None) == tp.EINVAL
    assert L.tpfa_unet_forward(None, None, None, None, None) == tp.EINVAL
    assert L.tpfa_unet_forward_samples(None, 1, None, None, None, None) == tp.EINVAL
    assert L.tpfa_restrict_levels(None, None, 8, 8, 8, 1, 0, None) == tp.EINVAL
    assert L.tpfa_tc_wait_probe(0, None) == tp.EINVAL
    assert L.tpfa_tc_wait_probe((1 << 22) + 1, None) == tp.EINVAL
    assert L.tpfa_prolong_levels(None, None, 8, 8, 8, 1, 4, None) == tp.EINVAL
    assert L.tpfa_unet_backward(None, None, None, None) == tp.EINVAL
    assert L.tpfa_conv3d_select(7) == tp.EINVAL
    assert L.tpfa_adam_step(None, None, None, None, 0, 1, 1e-3, 0.9, 0.999, 1e-8, None) == tp.EINVAL
    assert L.fcg_solve(None, None, None, None, None, None, None, 1e-8, 10, None, None,
                       None) == tp.EINVAL
    assert L.fcg_solve_batch(None, None, 0, None, None, None, None, None, None, 1e-8, 10, None,
                             None, None, None) == tp.EINVAL
