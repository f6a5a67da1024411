"""Tensor-core 3x3x3 convolutions (forward, input gradient, weight gradient)
against the FP64 oracle of the learned preconditioner.

Inputs and weights are BF16 values and the oracle evaluates the definition in
FP64 on exactly those values, so the kernel may differ only by FP32
accumulation (at most n 2^-24 sum|x w| for n terms) and, where the output is
BF16, by one rounding (2^-8 relative)."""
import numpy as np
import pytest
import torch

from oracle import unet_oracle as U
from paper_2408_03452_gb300 import synth

pytestmark = pytest.mark.gpu

SHAPES = [(16, 16), (16, 32), (32, 16), (32, 64), (64, 32)]
VOLS = [(8, 6, 5, 2), (40, 33, 7, 1), (16, 16, 16, 3)]


@pytest.fixture(scope="module")
def tp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2408_03452_gb300 import build, tpfa
    build.build()
    return tpfa


@pytest.fixture(params=[4, 2, 1, 0], ids=["zfold_ws", "zfold", "zmarch", "tiles"])
def kernel(tp, request):
    """Every forward kernel, forced for every layer shape: the folded z-marching
    ring with warp-specialised roles, the folded ring, the z-marching ring with
    one MMA per tap, the tile kernel (the default picks one per shape)."""
    tp.conv3d_select(request.param)
    yield request.param
    tp.conv3d_select(3)


def bf16(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(torch.bfloat16)


def rand_bf16(seed, shape, scale=1.0):
    a = synth.uniform_field(int(np.prod(shape)), seed).reshape(shape) * scale
    t = bf16(a)
    return t, t.to(torch.float64).numpy()


def to_halo(a, ns, nz, ny, nx):
    """(ns, nz, ny, nx, C) tensor -> haloed [V, C] tensor with a zero halo."""
    c = a.shape[-1]
    out = torch.zeros((ns, nz + 2, ny + 2, nx + 2, c), dtype=a.dtype)
    out[:, 1:-1, 1:-1, 1:-1] = a
    return out.reshape(-1, c)


def from_halo(t, ns, nz, ny, nx):
    c = t.shape[-1]
    return t.reshape(ns, nz + 2, ny + 2, nx + 2, c)


def check_bf16_out(got, ref, absbound):
    err = np.abs(got - ref)
    bound = 2.0 ** -8 * np.abs(ref) + absbound * (1 + 2.0 ** -8) + 1e-30
    assert np.all(err <= bound), (err.max(), (err / bound).max())


@pytest.mark.parametrize("cin,cout", SHAPES)
@pytest.mark.parametrize("vol", VOLS + [(20, 13, 70, 2)])
def test_conv_forward(tp, kernel, cin, cout, vol):
    nx, ny, nz, ns = vol
    xt, x = rand_bf16(11, (ns, nz, ny, nx, cin))
    wt, w = rand_bf16(12, (27, cout, cin), 1.0 / np.sqrt(27 * cin))
    b = synth.uniform_field(cout, 13) * 0.3
    dev = torch.device("cuda")
    X = to_halo(xt, ns, nz, ny, nx).to(dev)
    Y = torch.zeros((X.shape[0], cout), dtype=torch.bfloat16, device=dev)
    bias = torch.from_numpy(b).float().to(dev)
    b32 = bias.cpu().double().numpy()
    tp.conv3d_bf16(X, wt.to(dev), Y, vol, cin, cout, bias=bias, flags=tp.CONV_RELU)
    tp.net_status()
    got = from_halo(Y.cpu(), ns, nz, ny, nx)
    ref = U.relu(U.conv3d(x, w, b32))
    S = U.conv3d(np.abs(x), np.abs(w)) + np.abs(b32)
    check_bf16_out(got[:, 1:-1, 1:-1, 1:-1].double().numpy(), ref, 27 * cin * 2.0 ** -24 * S)
    halo = got.clone()
    halo[:, 1:-1, 1:-1, 1:-1] = 0
    assert torch.count_nonzero(halo) == 0


@pytest.mark.parametrize("cin,cout", SHAPES)
def test_conv_input_gradient_with_mask(tp, kernel, cin, cout):
    """dx = mask * conv^T(dy, w), computed by the forward kernel with the taps
    flipped and each tap's matrix transposed."""
    nx, ny, nz, ns = 20, 9, 6, 2
    dyt, dy = rand_bf16(21, (ns, nz, ny, nx, cout))
    wt, w = rand_bf16(22, (27, cout, cin), 1.0 / np.sqrt(27 * cout))
    mt, m = rand_bf16(23, (ns, nz, ny, nx, cin))
    wflip = torch.flip(wt, dims=[0]).transpose(1, 2).contiguous()  # [27][cin][cout]
    dev = torch.device("cuda")
    DY = to_halo(dyt, ns, nz, ny, nx).to(dev)
    M = to_halo(mt, ns, nz, ny, nx).to(dev)
    DX = torch.zeros((DY.shape[0], cin), dtype=torch.bfloat16, device=dev)
    tp.conv3d_bf16(DY, wflip.to(dev), DX, (nx, ny, nz, ns), cout, cin, mask=M, flags=tp.CONV_MASK)
    tp.net_status()
    got = from_halo(DX.cpu(), ns, nz, ny, nx)[:, 1:-1, 1:-1, 1:-1].double().numpy()
    ref = U.conv3d_adjoint(dy, w) * (m > 0)
    S = U.conv3d_adjoint(np.abs(dy), np.abs(w))
    check_bf16_out(got, ref, 27 * cout * 2.0 ** -24 * S)


@pytest.mark.parametrize("cin,cout", SHAPES)
@pytest.mark.parametrize("vol", [(8, 6, 5, 2), (40, 33, 7, 1)])
def test_conv_weight_gradient(tp, cin, cout, vol):
    nx, ny, nz, ns = vol
    xt, x = rand_bf16(31, (ns, nz, ny, nx, cin))
    dyt, dy = rand_bf16(32, (ns, nz, ny, nx, cout))
    dev = torch.device("cuda")
    X = to_halo(xt, ns, nz, ny, nx).to(dev)
    DY = to_halo(dyt, ns, nz, ny, nx).to(dev)
    dw = torch.full((27, cout, cin), 5.0, dtype=torch.float32, device=dev)
    tp.conv3d_wgrad_bf16(X, DY, dw, vol, cin, cout)
    tp.net_status()
    ref = U.conv3d_wgrad(x, dy)
    S = U.conv3d_wgrad(np.abs(x), np.abs(dy))
    n = ns * nz * ny * nx
    err = np.abs(dw.cpu().double().numpy() - ref)
    assert np.all(err <= n * 2.0 ** -24 * S + 2.0 ** -24 * np.abs(ref) + 1e-30), err.max()
    # accumulate adds to what is there
    tp.conv3d_wgrad_bf16(X, DY, dw, vol, cin, cout, accumulate=True)
    tp.net_status()
    err2 = np.abs(dw.cpu().double().numpy() - 2 * ref)
    assert np.all(err2 <= 2 * n * 2.0 ** -24 * S + 2.0 ** -23 * np.abs(ref) + 1e-30)


def test_conv_rejects_bad_arguments(tp):
    dev = torch.device("cuda")
    X = torch.zeros((tp.halo_voxels(4, 4, 4), 16), dtype=torch.bfloat16, device=dev)
    Y = torch.zeros((tp.halo_voxels(4, 4, 4), 16), dtype=torch.bfloat16, device=dev)
    w = torch.zeros((27, 16, 16), dtype=torch.bfloat16, device=dev)
    lib = tp.lib()
    st = tp._stream(dev)
    assert lib.tpfa_conv3d_bf16(X.data_ptr(), w.data_ptr(), None, None, Y.data_ptr(), 4, 4, 4, 1,
                                16, 24, 0, st) == tp.EINVAL
    assert lib.tpfa_conv3d_bf16(X.data_ptr(), w.data_ptr(), None, None, X.data_ptr(), 4, 4, 4, 1,
                                16, 16, 0, st) == tp.EINVAL
    assert lib.tpfa_conv3d_bf16(X.data_ptr(), w.data_ptr(), None, None, Y.data_ptr(), 4, 4, 4, 1,
                                16, 16, tp.CONV_MASK, st) == tp.EINVAL
    host = torch.zeros((tp.halo_voxels(4, 4, 4), 16), dtype=torch.bfloat16)
    assert lib.tpfa_conv3d_bf16(host.data_ptr(), w.data_ptr(), None, None, Y.data_ptr(), 4, 4, 4,
                                1, 16, 16, 0, st) == tp.EINVAL


def test_bounded_wait_timeout_is_reported_and_cleared(tp):
    """Failure path of the tensor-core kernels' bounded mbarrier waits: a wait
    that nothing completes gives up, the host reads TPFA_EINTERNAL from
    tpfa_net_status, the flag is cleared, and the context keeps working."""
    dev = torch.device("cuda")
    stream = tp._stream(dev)
    tp.net_status()  # nothing pending
    assert tp.lib().tpfa_tc_wait_probe(1000, stream) == tp.OK
    assert tp.lib().tpfa_net_status(stream) == tp.EINTERNAL
    assert tp.lib().tpfa_net_status(stream) == tp.OK  # reported once, then cleared
    # the context is still usable: a convolution runs and reports no timeout
    V = tp.halo_voxels(8, 8, 8, 1)
    x = torch.ones(V * 16, dtype=torch.bfloat16, device=dev)
    w = torch.ones(27 * 16 * 16, dtype=torch.bfloat16, device=dev)
    y = torch.zeros(V * 16, dtype=torch.bfloat16, device=dev)
    tp.conv3d_bf16(x, w, y, (8, 8, 8, 1), 16, 16)
    tp.net_status()
    assert float(y.float().max()) > 0.0
