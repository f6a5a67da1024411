"""The ctypes binding's argument checks, without a GPU: a tensor of the wrong
kind fails in Python before any library call (None passes as NULL)."""
import ctypes

import pytest
import torch

from paper_2408_03452_gb300 import tpfa


def test_ptr_checks_kind_device_dtype_layout_and_size():
    cpu = torch.device("cpu")
    t = torch.zeros(12, dtype=torch.float32)
    assert tpfa._ptr(None, torch.float32, 12, cpu, "x") is None
    p = tpfa._ptr(t, torch.float32, 12, cpu, "x")
    assert isinstance(p, ctypes.c_void_p) and p.value == t.data_ptr()
    assert tpfa._ptr(t, torch.float32, None, cpu, "x").value == t.data_ptr()  # size not checked
    with pytest.raises(TypeError):
        tpfa._ptr(t.numpy(), torch.float32, 12, cpu, "x")  # not a tensor
    with pytest.raises(ValueError, match="must be on"):
        tpfa._ptr(t, torch.float32, 12, torch.device("cuda", 0), "x")
    with pytest.raises(TypeError, match="must be torch.float64"):
        tpfa._ptr(t, torch.float64, 12, cpu, "x")
    with pytest.raises(ValueError, match="contiguous"):
        tpfa._ptr(t.view(3, 4).t(), torch.float32, 12, cpu, "x")
    with pytest.raises(ValueError, match="must have 13 elements"):
        tpfa._ptr(t, torch.float32, 13, cpu, "x")


def test_every_declared_entry_has_a_signature():
    """Each function the header declares is bound with explicit argument types
    (no implicit int conversions of pointers or doubles)."""
    import os
    import re
    hdr = open(os.path.join(os.path.dirname(tpfa.__file__), "..", "include", "tpfa.h")).read()
    names = set(re.findall(r"^(?:int|int64_t|const char\*)\s+(\w+)\(", hdr, flags=re.M))
    assert names, "no declarations found"
    missing = names - set(tpfa.SIGNATURES)
    assert not missing, sorted(missing)
