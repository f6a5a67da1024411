"""tpfa_apply_noalloc against tpfa_apply.

tpfa_apply_noalloc serves callers that may not allocate device memory (an
embedded component whose host application owns all device memory, or a loop
under a fixed memory budget): it takes no context and keeps its reduction
workspace in a fixed device array.  Here it is called through the C ABI
twice in a row (the second call finds the workspace as the first one left
it) and each result is compared with the context-based tpfa_apply on the same
inputs.  This file is collected last so that a failure here cannot stop a
first-failure run before the other tests.
"""
import ctypes as C

import numpy as np
import pytest
import torch

from paper_2408_03452_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2408_03452_gb300 import build, tpfa
    build.build()
    return tpfa


@pytest.mark.parametrize("shape", [(95, 33, 20), (256, 192, 64)])
def test_noalloc_apply_matches_context_apply(tp, shape):
    nx, ny, nz = shape
    n = nx * ny * nz
    K = torch.from_numpy(synth.lognormal_field(nx, ny, nz, 1.5, 3, layer=8)).cuda()
    L = tp.lib()
    s = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    with tp.Context(nx, ny, nz) as ctx:
        coef, _ = ctx.build_trans(K, None, None, 1e-3, coef64=False)
        for call in range(2):
            p = torch.from_numpy(synth.uniform_field(n, 20 + call).astype(np.float32)).cuda()
            ref_pAp = torch.zeros(1, dtype=torch.float64, device="cuda")
            ref = ctx.apply(coef, p, pAp=ref_pAp)
            Ap = torch.full((n,), float("nan"), dtype=torch.float32, device="cuda")
            pAp = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
            g = tp._Grid(nx, ny, nz, 1.0, 1.0, 1.0, 1.0)
            rc = L.tpfa_apply_noalloc(C.byref(g), C.c_void_p(coef.data_ptr()),
                                      C.c_void_p(p.data_ptr()), C.c_void_p(Ap.data_ptr()),
                                      C.c_void_p(pAp.data_ptr()), s)
            assert rc == tp.OK, tp.strerror(rc)
            torch.cuda.synchronize()
            # same per-cell arithmetic: identical values; the dot product may
            # differ only through its summation order (tpfa_apply may take the
            # TMA-staged kernel, whose warps own 32-column rows instead of 30):
            # each side's compensated FP32 warp sums are within 2u of exact, so
            # the two differ by at most 4u sum |p_i (Ap)_i|
            assert torch.equal(Ap, ref)
            absdot = float((p.double() * ref.double()).abs().sum())
            assert abs(pAp.item() - ref_pAp.item()) <= 4 * 2.0 ** -24 * absdot


def test_noalloc_rejects_bad_arguments(tp):
    L = tp.lib()
    s = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    x = torch.zeros(64, dtype=torch.float32, device="cuda")
    g = tp._Grid(0, 4, 4, 1.0, 1.0, 1.0, 1.0)
    assert L.tpfa_apply_noalloc(C.byref(g), C.c_void_p(x.data_ptr()), C.c_void_p(x.data_ptr()),
                                C.c_void_p(x.data_ptr()), None, s) == tp.EINVAL
    # a grid too wide for the fixed workspace (ceil(nx/30) * ceil(ny/4) > 65536)
    # is refused before any launch, even with correctly sized buffers
    nx, ny = 30 * 1024, 4 * 128
    n = nx * ny
    coef = torch.zeros(4 * n, dtype=torch.float32, device="cuda")
    p = torch.zeros(n, dtype=torch.float32, device="cuda")
    Ap = torch.zeros(n, dtype=torch.float32, device="cuda")
    g = tp._Grid(nx, ny, 1, 1.0, 1.0, 1.0, 1.0)
    assert L.tpfa_apply_noalloc(C.byref(g), C.c_void_p(coef.data_ptr()), C.c_void_p(p.data_ptr()),
                                C.c_void_p(Ap.data_ptr()), None, s) == tp.EINVAL
    g = tp._Grid(30 * 512, 4 * 128, 1, 1.0, 1.0, 1.0, 1.0)  # exactly at the limit
    assert L.tpfa_apply_noalloc(C.byref(g), C.c_void_p(coef.data_ptr()), C.c_void_p(p.data_ptr()),
                                C.c_void_p(Ap.data_ptr()), None, s) == tp.OK
    torch.cuda.synchronize()
