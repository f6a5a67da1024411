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
