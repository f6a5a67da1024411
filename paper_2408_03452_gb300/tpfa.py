"""Thin Python binding of ``libtpfa.so`` (the C ABI declared in include/tpfa.h).

Argument marshalling only: every step of the solve runs in the library's
CUDA kernels.  Tensors must be CUDA tensors on the context's device, C
contiguous, of the dtype stated per argument; work is enqueued on the
current torch stream.  There is no CPU fallback: if the library is missing
or fails to load, every call raises.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libtpfa.so")

OK, NOTCONV = 0, 1
EINVAL, ENOMEM, ECUDA, EBREAKDOWN, ENONFINITE, EINTERNAL, ESTAGNATION = -1, -2, -3, -4, -5, -6, -7

OPTIONS = {"inner_rtol": 1, "max_outer": 2, "loop": 3, "tile_vy": 4, "tile_zc": 5, "chunk": 6,
           "stages": 7, "inner_rtol_bf16": 11,
           "precond": 12, "fcg_m": 13, "fcg_fallback": 14, "sweep": 15, "tma_tile": 16}


class TpfaError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {strerror(code)} (status {code})")


class _Grid(C.Structure):
    _fields_ = [("nx", C.c_int64), ("ny", C.c_int64), ("nz", C.c_int64),
                ("dx", C.c_double), ("dy", C.c_double), ("dz", C.c_double), ("mu", C.c_double)]


class _Info(C.Structure):
    _fields_ = [("iters", C.c_int64), ("outer", C.c_int32), ("status", C.c_int32),
                ("rel_res_inner", C.c_double), ("rel_res_fp64", C.c_double),
                ("inner_ms", C.c_double), ("total_ms", C.c_double),
                ("kernel_launches", C.c_int64)]


_lib = None

# name -> (restype, argtypes)
_P = C.c_void_p
SIGNATURES = {
    "tpfa_create": (C.c_int, [C.POINTER(_Grid), C.POINTER(C.c_void_p)]),
    "tpfa_destroy": (C.c_int, [_P]),
    "tpfa_strerror": (C.c_char_p, [C.c_int]),
    "tpfa_abi_version": (C.c_int, []),
    "tpfa_set_option": (C.c_int, [_P, C.c_int, C.c_double]),
    "tpfa_sweep_tiling": (C.c_int, [_P, C.c_int, _P]),
    "tpfa_build_trans": (C.c_int, [_P, _P, _P, _P, C.c_double, _P, _P, _P]),
    "tpfa_build_rhs": (C.c_int, [_P, _P, _P, _P, _P, _P, _P, C.c_int64, _P, _P]),
    "tpfa_apply": (C.c_int, [_P, _P, _P, _P, _P, _P]),
    "tpfa_build_rhs_transient": (C.c_int, [_P, _P, _P, _P, _P, _P, _P, C.c_int64, _P, C.c_double,
                                           _P, _P, _P]),
    "tpfa_residual64": (C.c_int, [_P, _P, _P, _P, _P, _P, _P]),
    "cg_solve": (C.c_int, [_P, _P, _P, _P, _P, C.c_double, C.c_int64, C.POINTER(_Info), _P]),
    "tpfa_apply_noalloc": (C.c_int, [C.POINTER(_Grid), _P, _P, _P, _P, _P]),
    "tpfa_tc_gemm_bf16": (C.c_int, [_P, _P, _P, C.c_int, C.c_int, C.c_int, _P]),
    "tpfa_conv3d_bf16": (C.c_int, [_P, _P, _P, _P, _P] + [C.c_int] * 7 + [_P]),
    "tpfa_conv3d_wgrad_bf16": (C.c_int, [_P, _P, _P] + [C.c_int] * 7 + [_P]),
    "tpfa_net_status": (C.c_int, [_P]),
    "tpfa_tc_wait_probe": (C.c_int, [C.c_uint32, _P]),
    "tpfa_conv3d_select": (C.c_int, [C.c_int]),
    "tpfa_unet_param_count": (C.c_int64, []),
    "tpfa_log_perm": (C.c_int, [_P, _P, C.c_int64, _P]),
    "tpfa_unet_create": (C.c_int, [C.c_int] * 5 + [C.POINTER(C.c_void_p)]),
    "tpfa_unet_destroy": (C.c_int, [_P]),
    "tpfa_unet_shape": (C.c_int, [_P, C.POINTER(C.c_int)]),
    "tpfa_unet_set_params": (C.c_int, [_P, _P, _P]),
    "tpfa_unet_forward": (C.c_int, [_P, _P, _P, _P, _P]),
    "tpfa_unet_forward_samples": (C.c_int, [_P, C.c_int, _P, _P, _P, _P]),
    "tpfa_unet_backward": (C.c_int, [_P, _P, _P, _P]),
    "tpfa_adam_step": (C.c_int, [_P, _P, _P, _P, C.c_int64, C.c_int, C.c_double, C.c_double,
                                 C.c_double, C.c_double, _P]),
    "tpfa_anorm_loss_grad": (C.c_int, [_P] * 9),
    "tpfa_jacobi_split": (C.c_int, [_P] * 7),
    "tpfa_restrict2": (C.c_int, [_P, _P, C.c_int, C.c_int, C.c_int, C.c_int, C.c_float, _P]),
    "tpfa_prolong2": (C.c_int, [_P, _P, C.c_int, C.c_int, C.c_int, C.c_int, _P]),
    "tpfa_restrict_levels": (C.c_int, [_P, _P] + [C.c_int] * 5 + [_P]),
    "tpfa_prolong_levels": (C.c_int, [_P, _P] + [C.c_int] * 5 + [_P]),
    "fcg_solve": (C.c_int, [_P, _P, _P, _P, _P, _P, _P, C.c_double, C.c_int64,
                            C.POINTER(_Info), C.POINTER(C.c_int), _P]),
    "tpfa_build_trans_bf16": (C.c_int, [_P, _P, _P, _P, C.c_double, _P, _P]),
    "tpfa_apply_bf16": (C.c_int, [_P, _P, _P, _P, _P, _P]),
    "cg_solve_bf16": (C.c_int, [_P, _P, _P, _P, _P, C.c_double, C.c_int64, C.POINTER(_Info), _P]),
    "tpfa_batch_create": (C.c_int, [_P, C.c_int, _P, C.POINTER(C.c_void_p)]),
    "tpfa_batch_destroy": (C.c_int, [_P]),
    "tpfa_batch_offsets": (C.c_int, [_P, _P]),
    "tpfa_batch_zc": (C.c_int, [_P, _P]),
    "tpfa_batch_set_option": (C.c_int, [_P, C.c_int, C.c_double]),
    "tpfa_batch_build_trans": (C.c_int, [_P, _P, _P, _P, C.c_double, _P, _P, _P]),
    "tpfa_batch_build_rhs": (C.c_int, [_P, _P, _P, _P, _P, _P, _P]),
    "cg_solve_batch": (C.c_int, [_P, _P, _P, _P, _P, C.c_double, C.c_int64, _P,
                                 C.POINTER(_Info), _P]),
    "fcg_solve_batch": (C.c_int, [_P, _P, C.c_int, _P, _P, _P, _P, _P, _P, C.c_double,
                                  C.c_int64, _P, C.POINTER(_Info), _P, _P]),
}


def lib():
    """Load libtpfa.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "`python -m paper_2408_03452_gb300.build` (needs nvcc)")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def strerror(code: int) -> str:
    return lib().tpfa_strerror(int(code)).decode()


def abi_version() -> int:
    return lib().tpfa_abi_version()


def tc_gemm_bf16(A, Bt, C=None):
    """C = A @ Bt.T on the tensor cores (A [M,K], Bt [N,K] bfloat16; C float32)."""
    M, K = A.shape
    N = Bt.shape[0]
    if C is None:
        C = torch.empty((M, N), dtype=torch.float32, device=A.device)
    dev = A.device
    _check(lib().tpfa_tc_gemm_bf16(_ptr(A, torch.bfloat16, M * K, dev, "A"),
                                   _ptr(Bt, torch.bfloat16, N * K, dev, "Bt"),
                                   _ptr(C, torch.float32, M * N, dev, "C"), M, N, K,
                                   _stream(dev)), "tpfa_tc_gemm_bf16")
    return C


CONV_RELU, CONV_MASK = 1, 2


def halo_voxels(nx: int, ny: int, nz: int, ns: int = 1) -> int:
    """Voxels of the haloed channels-last layout of ns samples of nz x ny x nx."""
    return (nx + 2) * (ny + 2) * (nz + 2) * ns


def conv3d_bf16(x, w, y, shape, cin, cout, bias=None, mask=None, flags=0):
    """y = epilogue(conv3x3x3(x; w) + bias) on haloed BF16 volumes (tensor cores).

    shape = (nx, ny, nz, ns); x [V, cin], y [V, cout] and mask [V, cout] are
    bfloat16 with V = halo_voxels(*shape); w [27, cout, cin] bfloat16; bias
    [cout] float32.  flags: CONV_RELU, CONV_MASK (zero where mask <= 0)."""
    dev = x.device
    V = halo_voxels(*shape)
    _check(lib().tpfa_conv3d_bf16(_ptr(x, torch.bfloat16, V * cin, dev, "x"),
                                  _ptr(w, torch.bfloat16, 27 * cin * cout, dev, "w"),
                                  _ptr(bias, torch.float32, cout, dev, "bias"),
                                  _ptr(mask, torch.bfloat16, V * cout, dev, "mask"),
                                  _ptr(y, torch.bfloat16, V * cout, dev, "y"), *shape, cin, cout,
                                  flags, _stream(dev)), "tpfa_conv3d_bf16")
    return y


def conv3d_wgrad_bf16(x, dy, dw, shape, cin, cout, accumulate=False):
    """dw[t, co, ci] (+)= sum_v dy[v, co] x[v + off_t, ci] (tensor cores); dw float32."""
    dev = x.device
    V = halo_voxels(*shape)
    _check(lib().tpfa_conv3d_wgrad_bf16(_ptr(x, torch.bfloat16, V * cin, dev, "x"),
                                        _ptr(dy, torch.bfloat16, V * cout, dev, "dy"),
                                        _ptr(dw, torch.float32, 27 * cin * cout, dev, "dw"),
                                        *shape, cin, cout, int(accumulate), _stream(dev)),
           "tpfa_conv3d_wgrad_bf16")
    return dw


def conv3d_select(kernel: int):
    """Forward-convolution kernel (tpfa_conv3d_select): 0 tile, 1 z-marching,
    2 z-taps folded, 3 automatic (default: 4 except 32 -> 16, which takes 1),
    4 folded with warp-specialised roles; 64 -> 32 always takes 0."""
    _check(lib().tpfa_conv3d_select(int(kernel)), "tpfa_conv3d_select")


def net_status(device=None):
    """Synchronise and report a tensor-core wait that gave up (raises)."""
    dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
    _check(lib().tpfa_net_status(_stream(dev)), "tpfa_net_status")


def _check(code: int, where: str, allow=(OK,)):
    if code not in allow:
        raise TpfaError(code, where)
    return code


def _ptr(t: Optional[torch.Tensor], dtype, n: Optional[int], dev: torch.device, name: str):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch tensor")
    if t.device != dev:
        raise ValueError(f"{name} must be on {dev}, got {t.device}")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if n is not None and t.numel() != n:
        raise ValueError(f"{name} must have {n} elements, got {t.numel()}")
    return C.c_void_p(t.data_ptr())


def _stream(dev):
    return C.c_void_p(torch.cuda.current_stream(dev).cuda_stream)


class Context:
    """One grid on one CUDA device (wraps tpfa_create / tpfa_destroy)."""

    def __init__(self, nx, ny, nz, dx=1.0, dy=1.0, dz=1.0, mu=1.0, device=None):
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None \
            else torch.device(device)
        self.nx, self.ny, self.nz = int(nx), int(ny), int(nz)
        self.n = self.nx * self.ny * self.nz
        self._h = C.c_void_p()
        g = _Grid(self.nx, self.ny, self.nz, float(dx), float(dy), float(dz), float(mu))
        with torch.cuda.device(self.device):
            _check(lib().tpfa_create(C.byref(g), C.byref(self._h)), "tpfa_create")

    def close(self):
        if self._h:
            with torch.cuda.device(self.device):
                lib().tpfa_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_option(self, name: str, value: float):
        _check(lib().tpfa_set_option(self._h, OPTIONS[name], float(value)), f"set_option({name})")

    def tiling(self, which: int = 0) -> dict:
        """Sweep tiling: which = 0 (CG loop, FP32 records), 1 (CG loop, BF16
        records), 2 (tpfa_apply), 3 (tpfa_apply_bf16; both for 16-byte aligned
        arguments).  kernel 1 = cp.async-staged, 2 = TMA-staged."""
        out = (C.c_int64 * 6)()
        _check(lib().tpfa_sweep_tiling(self._h, int(which), C.cast(out, C.c_void_p)),
               "tpfa_sweep_tiling")
        return dict(zip(("kernel", "vy", "stages", "warps", "zc", "blocks"), list(out)))

    # -- coefficient and right-hand side construction -----------------------
    def build_trans(self, K, dirichlet=None, d=None, d_uniform=0.0, coef=None, coef64=True):
        """Returns (coef float32[N,4], coef64 float64[N,4] or None)."""
        dev, n = self.device, self.n
        if coef is None:
            coef = torch.empty((n, 4), dtype=torch.float32, device=dev)
        if coef64 is True:
            coef64 = torch.empty((n, 4), dtype=torch.float64, device=dev)
        elif coef64 is False:
            coef64 = None
        with torch.cuda.device(dev):
            _check(lib().tpfa_build_trans(
                self._h, _ptr(K, torch.float64, n, dev, "K"),
                _ptr(dirichlet, torch.uint8, n, dev, "dirichlet"),
                _ptr(d, torch.float64, n, dev, "d"), float(d_uniform),
                _ptr(coef, torch.float32, 4 * n, dev, "coef"),
                _ptr(coef64, torch.float64, 4 * n, dev, "coef64"), _stream(dev)), "tpfa_build_trans")
        return coef, coef64

    def build_trans_bf16(self, K, dirichlet=None, d=None, d_uniform=0.0, coef16=None):
        """BF16 records (Tx', Ty', Tz', E) as int16 bit patterns, shape [N, 4]."""
        dev, n = self.device, self.n
        if coef16 is None:
            coef16 = torch.empty((n, 4), dtype=torch.int16, device=dev)
        with torch.cuda.device(dev):
            _check(lib().tpfa_build_trans_bf16(
                self._h, _ptr(K, torch.float64, n, dev, "K"),
                _ptr(dirichlet, torch.uint8, n, dev, "dirichlet"),
                _ptr(d, torch.float64, n, dev, "d"), float(d_uniform),
                _ptr(coef16, torch.int16, 4 * n, dev, "coef16"), _stream(dev)),
                "tpfa_build_trans_bf16")
        return coef16

    def build_rhs(self, K, dirichlet=None, q=None, pD=None, src_idx=None, src_val=None, b=None):
        dev, n = self.device, self.n
        if b is None:
            b = torch.empty(n, dtype=torch.float64, device=dev)
        ns = 0 if src_idx is None else int(src_idx.numel())
        if (src_val is None) != (src_idx is None) or (src_val is not None and src_val.numel() != ns):
            raise ValueError("src_idx and src_val must be given together, with equal lengths")
        with torch.cuda.device(dev):
            _check(lib().tpfa_build_rhs(
                self._h, _ptr(K, torch.float64, n, dev, "K"),
                _ptr(dirichlet, torch.uint8, n, dev, "dirichlet"),
                _ptr(q, torch.float64, n, dev, "q"), _ptr(pD, torch.float64, n, dev, "pD"),
                _ptr(src_idx, torch.int64, ns, dev, "src_idx") if ns else None,
                _ptr(src_val, torch.float64, ns, dev, "src_val") if ns else None, ns,
                _ptr(b, torch.float64, n, dev, "b"), _stream(dev)), "tpfa_build_rhs")
        return b

    def build_rhs_transient(self, K, p_prev, dirichlet=None, q=None, pD=None, src_idx=None,
                            src_val=None, d=None, d_uniform=0.0, b=None):
        """Right-hand side of one backward-Euler step from p_prev (float64 [N])."""
        dev, n = self.device, self.n
        if b is None:
            b = torch.empty(n, dtype=torch.float64, device=dev)
        ns = 0 if src_idx is None else int(src_idx.numel())
        with torch.cuda.device(dev):
            _check(lib().tpfa_build_rhs_transient(
                self._h, _ptr(K, torch.float64, n, dev, "K"),
                _ptr(dirichlet, torch.uint8, n, dev, "dirichlet"),
                _ptr(q, torch.float64, n, dev, "q"), _ptr(pD, torch.float64, n, dev, "pD"),
                _ptr(src_idx, torch.int64, ns, dev, "src_idx") if ns else None,
                _ptr(src_val, torch.float64, ns, dev, "src_val") if ns else None, ns,
                _ptr(d, torch.float64, n, dev, "d"), float(d_uniform),
                _ptr(p_prev, torch.float64, n, dev, "p_prev"),
                _ptr(b, torch.float64, n, dev, "b"), _stream(dev)), "tpfa_build_rhs_transient")
        return b

    # -- operator --------------------------------------------------------------
    def apply(self, coef, p, Ap=None, pAp=None):
        """Ap = A p in FP32.  pAp: optional float64 tensor of one element that
        receives p.Ap."""
        dev, n = self.device, self.n
        if Ap is None:
            Ap = torch.empty(n, dtype=torch.float32, device=dev)
        with torch.cuda.device(dev):
            _check(lib().tpfa_apply(
                self._h, _ptr(coef, torch.float32, 4 * n, dev, "coef"),
                _ptr(p, torch.float32, n, dev, "p"), _ptr(Ap, torch.float32, n, dev, "Ap"),
                _ptr(pAp, torch.float64, 1, dev, "pAp"), _stream(dev)), "tpfa_apply")
        return Ap

    def apply_bf16(self, coef16, p, Ap=None, pAp=None):
        dev, n = self.device, self.n
        if Ap is None:
            Ap = torch.empty(n, dtype=torch.float32, device=dev)
        with torch.cuda.device(dev):
            _check(lib().tpfa_apply_bf16(
                self._h, _ptr(coef16, torch.int16, 4 * n, dev, "coef16"),
                _ptr(p, torch.float32, n, dev, "p"), _ptr(Ap, torch.float32, n, dev, "Ap"),
                _ptr(pAp, torch.float64, 1, dev, "pAp"), _stream(dev)), "tpfa_apply_bf16")
        return Ap

    def residual64(self, coef64, b, x, r=None, norms=None):
        """r = b - A x in FP64.  norms: optional float64[2] receiving
        (||r||^2, ||b||^2)."""
        dev, n = self.device, self.n
        if r is None:
            r = torch.empty(n, dtype=torch.float64, device=dev)
        with torch.cuda.device(dev):
            _check(lib().tpfa_residual64(
                self._h, _ptr(coef64, torch.float64, 4 * n, dev, "coef64"),
                _ptr(b, torch.float64, n, dev, "b"), _ptr(x, torch.float64, n, dev, "x"),
                _ptr(r, torch.float64, n, dev, "r"), _ptr(norms, torch.float64, 2, dev, "norms"),
                _stream(dev)), "tpfa_residual64")
        return r

    def cg_solve(self, coef, coef64, b, x=None, tol=1e-8, maxit=100000, check=True):
        """Solve A x = b to FP64 relative residual tol.  Returns (x, info dict).
        coef: FP32 records (float32 [N,4]) or BF16 records (int16 [N,4], the
        mixed-precision solve cg_solve_bf16)."""
        dev, n = self.device, self.n
        if x is None:
            x = torch.zeros(n, dtype=torch.float64, device=dev)
        info = _Info()
        b16 = coef.dtype == torch.int16
        fn = lib().cg_solve_bf16 if b16 else lib().cg_solve
        with torch.cuda.device(dev):
            code = fn(
                self._h, _ptr(coef, torch.int16 if b16 else torch.float32, 4 * n, dev, "coef"),
                _ptr(coef64, torch.float64, 4 * n, dev, "coef64"),
                _ptr(b, torch.float64, n, dev, "b"), _ptr(x, torch.float64, n, dev, "x"),
                float(tol), int(maxit), C.byref(info), _stream(dev))
        if check:
            _check(code, "cg_solve", allow=(OK, NOTCONV))
        out = {f: getattr(info, f) for f, _ in _Info._fields_}
        out["code"] = code
        return x, out


    def fcg_solve(self, coef, coef64, b, net=None, lnk=None, x=None, tol=1e-8, maxit=100000,
                  check=True):
        """Flexible CG preconditioned by a UNet (None: plain CG), FP64-refined.
        Returns (x, info dict with 'fell_back')."""
        dev, n = self.device, self.n
        if x is None:
            x = torch.zeros(n, dtype=torch.float64, device=dev)
        info = _Info()
        fb = C.c_int(0)
        with torch.cuda.device(dev):
            code = lib().fcg_solve(
                self._h, net._h if net is not None else None,
                _ptr(coef, torch.float32, 4 * n, dev, "coef"),
                _ptr(coef64, torch.float64, 4 * n, dev, "coef64"),
                _ptr(lnk, torch.float32, n, dev, "lnk") if net is not None else None,
                _ptr(b, torch.float64, n, dev, "b"), _ptr(x, torch.float64, n, dev, "x"),
                float(tol), int(maxit), C.byref(info), C.byref(fb), _stream(dev))
        if check:
            _check(code, "fcg_solve", allow=(OK, NOTCONV))
        out = {f: getattr(info, f) for f, _ in _Info._fields_}
        out["code"] = code
        out["fell_back"] = bool(fb.value)
        return x, out

    def anorm_loss_grad(self, coef, mr, r, eae, q, g, stats):
        """Gradient of the scale-optimal A-norm loss (see tpfa_anorm_loss_grad):
        q = A mr, stats float64[2] = (mr'r, mr'A mr), g = dL/dmr.  The loss is
        1 - stats[0]^2 / (stats[1] eae)."""
        dev, n = self.device, self.n
        with torch.cuda.device(dev):
            _check(lib().tpfa_anorm_loss_grad(
                self._h, _ptr(coef, torch.float32, 4 * n, dev, "coef"),
                _ptr(mr, torch.float32, n, dev, "mr"), _ptr(r, torch.float32, n, dev, "r"),
                _ptr(eae, torch.float64, 1, dev, "eae"), _ptr(q, torch.float32, n, dev, "q"),
                _ptr(g, torch.float32, n, dev, "g"), _ptr(stats, torch.float64, 2, dev, "stats"),
                _stream(dev)), "tpfa_anorm_loss_grad")
        return g


    def jacobi_split(self, coef, r, s=None, e=None, wAw=None):
        """s = r - A D^-1 r; with e and wAw (float64 [1]): wAw = w'Aw, w = e - D^-1 r."""
        dev, n = self.device, self.n
        if s is None:
            s = torch.empty(n, dtype=torch.float32, device=dev)
        with torch.cuda.device(dev):
            _check(lib().tpfa_jacobi_split(
                self._h, _ptr(coef, torch.float32, 4 * n, dev, "coef"),
                _ptr(r, torch.float32, n, dev, "r"), _ptr(e, torch.float32, n, dev, "e"),
                _ptr(s, torch.float32, n, dev, "s"), _ptr(wAw, torch.float64, 1, dev, "wAw"),
                _stream(dev)), "tpfa_jacobi_split")
        return s


def unet_param_count() -> int:
    return int(lib().tpfa_unet_param_count())


class UNet:
    """The U-Net preconditioner for ns samples of nx x ny x nz (wraps tpfa_unet_*).
    Parameters: one float32 tensor of unet_param_count() values."""

    def __init__(self, nx, ny, nz, ns=1, train=False, device=None):
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None \
            else torch.device(device)
        self.shape = (nx, ny, nz, ns)
        self.n = nx * ny * nz * ns
        self._h = C.c_void_p()
        with torch.cuda.device(self.device):
            _check(lib().tpfa_unet_create(nx, ny, nz, ns, int(bool(train)), C.byref(self._h)),
                   "tpfa_unet_create")

    def close(self):
        if self._h:
            with torch.cuda.device(self.device):
                lib().tpfa_unet_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, params):
        dev = self.device
        with torch.cuda.device(dev):
            _check(lib().tpfa_unet_set_params(
                self._h, _ptr(params, torch.float32, unet_param_count(), dev, "params"),
                _stream(dev)), "tpfa_unet_set_params")

    def forward(self, r, lnk, z=None, samples=None):
        """z = M(r); samples: run on the first `samples` samples only (r, lnk, z
        then hold that many)."""
        dev = self.device
        ns = self.shape[3] if samples is None else int(samples)
        n = self.n // self.shape[3] * ns
        if z is None:
            z = torch.empty(n, dtype=torch.float32, device=dev)
        with torch.cuda.device(dev):
            _check(lib().tpfa_unet_forward_samples(
                self._h, ns, _ptr(r, torch.float32, n, dev, "r"),
                _ptr(lnk, torch.float32, n, dev, "lnk"), _ptr(z, torch.float32, n, dev, "z"),
                _stream(dev)), "tpfa_unet_forward_samples")
        return z

    def backward(self, gz, grad=None):
        dev, n = self.device, self.n
        if grad is None:
            grad = torch.empty(unet_param_count(), dtype=torch.float32, device=dev)
        with torch.cuda.device(dev):
            _check(lib().tpfa_unet_backward(self._h, _ptr(gz, torch.float32, n, dev, "gz"),
                                            _ptr(grad, torch.float32, grad.numel(), dev, "grad"),
                                            _stream(dev)), "tpfa_unet_backward")
        return grad


def restrict2(fine, shape, scale=0.125, coarse=None):
    """coarse = scale * (sum of each cell's 8 children); shape = (nx, ny, nz, ns) of the fine grid."""
    nx, ny, nz, ns = shape
    dev = fine.device
    nc = (nx // 2) * (ny // 2) * (nz // 2) * ns
    if coarse is None:
        coarse = torch.empty(nc, dtype=torch.float32, device=dev)
    with torch.cuda.device(dev):
        _check(lib().tpfa_restrict2(_ptr(fine, torch.float32, nc * 8, dev, "fine"),
                                    _ptr(coarse, torch.float32, nc, dev, "coarse"), nx, ny, nz, ns,
                                    float(scale), _stream(dev)), "tpfa_restrict2")
    return coarse


def prolong2(coarse, shape, fine=None):
    """fine[c] = coarse[parent(c)]; shape = (nx, ny, nz, ns) of the fine grid."""
    nx, ny, nz, ns = shape
    dev = coarse.device
    n = nx * ny * nz * ns
    if fine is None:
        fine = torch.empty(n, dtype=torch.float32, device=dev)
    with torch.cuda.device(dev):
        _check(lib().tpfa_prolong2(_ptr(coarse, torch.float32, n // 8, dev, "coarse"),
                                   _ptr(fine, torch.float32, n, dev, "fine"), nx, ny, nz, ns,
                                   _stream(dev)), "tpfa_prolong2")
    return fine


def restrict_levels(fine, shape, levels, coarse=None):
    """The 2^levels coarser grid in one pass (block means); shape = (nx, ny, nz, ns)."""
    nx, ny, nz, ns = shape
    dev = fine.device
    nc = (nx * ny * nz * ns) >> (3 * levels)
    if coarse is None:
        coarse = torch.empty(nc, dtype=torch.float32, device=dev)
    with torch.cuda.device(dev):
        _check(lib().tpfa_restrict_levels(_ptr(fine, torch.float32, nx * ny * nz * ns, dev, "fine"),
                                          _ptr(coarse, torch.float32, nc, dev, "coarse"), nx, ny,
                                          nz, ns, int(levels), _stream(dev)), "tpfa_restrict_levels")
    return coarse


def prolong_levels(coarse, shape, levels, fine=None):
    """fine[c] = coarse value of c's ancestor on the 2^levels coarser grid."""
    nx, ny, nz, ns = shape
    dev = coarse.device
    n = nx * ny * nz * ns
    if fine is None:
        fine = torch.empty(n, dtype=torch.float32, device=dev)
    with torch.cuda.device(dev):
        _check(lib().tpfa_prolong_levels(_ptr(coarse, torch.float32, n >> (3 * levels), dev,
                                              "coarse"),
                                         _ptr(fine, torch.float32, n, dev, "fine"), nx, ny, nz, ns,
                                         int(levels), _stream(dev)), "tpfa_prolong_levels")
    return fine


def log_perm(K, lnk=None):
    """The network's permeability input ln K (FP32) from K (float64 CUDA tensor)."""
    dev, n = K.device, K.numel()
    if lnk is None:
        lnk = torch.empty(n, dtype=torch.float32, device=dev)
    with torch.cuda.device(dev):
        _check(lib().tpfa_log_perm(_ptr(K, torch.float64, n, dev, "K"),
                                   _ptr(lnk, torch.float32, n, dev, "lnk"), n, _stream(dev)),
               "tpfa_log_perm")
    return lnk


def adam_step(params, grad, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    dev, n = params.device, params.numel()
    with torch.cuda.device(dev):
        _check(lib().tpfa_adam_step(_ptr(params, torch.float32, n, dev, "params"),
                                    _ptr(grad, torch.float32, n, dev, "grad"),
                                    _ptr(m, torch.float32, n, dev, "m"),
                                    _ptr(v, torch.float32, n, dev, "v"), n, int(t), float(lr),
                                    float(b1), float(b2), float(eps), _stream(dev)),
               "tpfa_adam_step")


class BatchContext:
    """Many grids solved together (wraps tpfa_batch_*).  Per-cell tensors are
    the concatenation of the instances' arrays; `offsets` gives the split."""

    def __init__(self, grids, zc=None, device=None):
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None \
            else torch.device(device)
        self.ninst = len(grids)
        arr = (_Grid * self.ninst)()
        for i, g in enumerate(grids):
            g = tuple(g) + (1.0, 1.0, 1.0, 1.0)[len(g) - 3:] if len(g) < 7 else tuple(g)
            arr[i] = _Grid(int(g[0]), int(g[1]), int(g[2]), float(g[3]), float(g[4]),
                           float(g[5]), float(g[6]))
        zarr = None
        if zc is not None:
            zarr = (C.c_int * self.ninst)(*[int(z) for z in zc])
        self._h = C.c_void_p()
        with torch.cuda.device(self.device):
            _check(lib().tpfa_batch_create(C.cast(arr, C.c_void_p), self.ninst,
                                           C.cast(zarr, C.c_void_p) if zarr is not None else None,
                                           C.byref(self._h)), "tpfa_batch_create")
        off = (C.c_int64 * (self.ninst + 1))()
        _check(lib().tpfa_batch_offsets(self._h, C.cast(off, C.c_void_p)), "tpfa_batch_offsets")
        self.offsets = [int(v) for v in off]
        self.n = self.offsets[-1]

    @property
    def zc(self):
        """z-run length per instance of the batched sweep the options select."""
        z = (C.c_int * self.ninst)()
        _check(lib().tpfa_batch_zc(self._h, C.cast(z, C.c_void_p)), "tpfa_batch_zc")
        return [int(v) for v in z]

    def close(self):
        if self._h:
            with torch.cuda.device(self.device):
                lib().tpfa_batch_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_option(self, name, value):
        _check(lib().tpfa_batch_set_option(self._h, OPTIONS[name], float(value)),
               f"batch set_option({name})")

    def build_trans(self, K, dirichlet=None, d=None, d_uniform=0.0):
        dev, n = self.device, self.n
        coef = torch.empty((n, 4), dtype=torch.float32, device=dev)
        coef64 = torch.empty((n, 4), dtype=torch.float64, device=dev)
        with torch.cuda.device(dev):
            _check(lib().tpfa_batch_build_trans(
                self._h, _ptr(K, torch.float64, n, dev, "K"),
                _ptr(dirichlet, torch.uint8, n, dev, "dirichlet"),
                _ptr(d, torch.float64, n, dev, "d"), float(d_uniform),
                _ptr(coef, torch.float32, 4 * n, dev, "coef"),
                _ptr(coef64, torch.float64, 4 * n, dev, "coef64"), _stream(dev)),
                "tpfa_batch_build_trans")
        return coef, coef64

    def build_rhs(self, K, dirichlet=None, q=None, pD=None):
        dev, n = self.device, self.n
        b = torch.empty(n, dtype=torch.float64, device=dev)
        with torch.cuda.device(dev):
            _check(lib().tpfa_batch_build_rhs(
                self._h, _ptr(K, torch.float64, n, dev, "K"),
                _ptr(dirichlet, torch.uint8, n, dev, "dirichlet"),
                _ptr(q, torch.float64, n, dev, "q"), _ptr(pD, torch.float64, n, dev, "pD"),
                _ptr(b, torch.float64, n, dev, "b"), _stream(dev)), "tpfa_batch_build_rhs")
        return b

    def cg_solve(self, coef, coef64, b, x=None, tol=1e-8, maxit=100000, check=True):
        """Returns (x, per-instance info list, total info)."""
        dev, n = self.device, self.n
        if x is None:
            x = torch.zeros(n, dtype=torch.float64, device=dev)
        infos = (_Info * self.ninst)()
        tot = _Info()
        with torch.cuda.device(dev):
            code = lib().cg_solve_batch(
                self._h, _ptr(coef, torch.float32, 4 * n, dev, "coef"),
                _ptr(coef64, torch.float64, 4 * n, dev, "coef64"),
                _ptr(b, torch.float64, n, dev, "b"), _ptr(x, torch.float64, n, dev, "x"),
                float(tol), int(maxit), C.cast(infos, C.c_void_p), C.byref(tot), _stream(dev))
        if check:
            _check(code, "cg_solve_batch", allow=(OK, NOTCONV))
        per = [{f: getattr(infos[i], f) for f, _ in _Info._fields_} for i in range(self.ninst)]
        total = {f: getattr(tot, f) for f, _ in _Info._fields_}
        total["code"] = code
        return x, per, total

    def fcg_solve(self, coef, coef64, b, nets=(), net_of=None, lnk=None, x=None, tol=1e-8,
                  maxit=100000, check=True):
        """Flexible CG over every instance (fcg_solve_batch).  nets: UNet
        objects; net_of[i]: index into nets of instance i's network, or -1.
        Returns (x, per-instance info list with 'fell_back', total info)."""
        dev, n = self.device, self.n
        if x is None:
            x = torch.zeros(n, dtype=torch.float64, device=dev)
        nets = list(nets)
        harr = (C.c_void_p * max(1, len(nets)))(*[u._h.value for u in nets])
        oarr = None
        if nets:
            if net_of is None or len(net_of) != self.ninst:
                raise ValueError("net_of needs one entry per instance")
            oarr = (C.c_int * self.ninst)(*[int(k) for k in net_of])
        infos = (_Info * self.ninst)()
        tot = _Info()
        fb = (C.c_int * self.ninst)()
        with torch.cuda.device(dev):
            code = lib().fcg_solve_batch(
                self._h, C.cast(harr, C.c_void_p) if nets else None, len(nets),
                C.cast(oarr, C.c_void_p) if oarr is not None else None,
                _ptr(coef, torch.float32, 4 * n, dev, "coef"),
                _ptr(coef64, torch.float64, 4 * n, dev, "coef64"),
                _ptr(lnk, torch.float32, n, dev, "lnk") if nets else None,
                _ptr(b, torch.float64, n, dev, "b"), _ptr(x, torch.float64, n, dev, "x"),
                float(tol), int(maxit), C.cast(infos, C.c_void_p), C.byref(tot),
                C.cast(fb, C.c_void_p), _stream(dev))
        if check:
            _check(code, "fcg_solve_batch", allow=(OK, NOTCONV))
        per = []
        for i in range(self.ninst):
            d = {f: getattr(infos[i], f) for f, _ in _Info._fields_}
            d["fell_back"] = bool(fb[i])
            per.append(d)
        total = {f: getattr(tot, f) for f, _ in _Info._fields_}
        total["code"] = code
        return x, per, total
