"""Thin ctypes binding of libuot (include/uot.h).

Functions carry the C names and only marshal arguments: torch tensors supply
device pointers, leading dimensions and the current CUDA stream; every step of
the iteration runs in the library's CUDA kernels.  There is no fallback: if
``libuot.so`` is missing or no GPU is present the calls raise.
"""

from __future__ import annotations

import ctypes
import math
import os
from dataclasses import dataclass

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libuot.so")

UOT_OK = 0
UOT_ERR_INVALID_ARG = 1
UOT_ERR_CUDA = 2
UOT_ERR_NONFINITE = 3
UOT_ERR_ZERO_SUM = 4
UOT_ERR_TIMEOUT = 5
UOT_ERR_UNSUPPORTED = 6
UOT_ERR_WORKSPACE = 7

UOT_F32, UOT_BF16, UOT_F16 = 0, 1, 2
UOT_ALGO_FUSED, UOT_ALGO_MULTIPASS = 0, 1
UOT_RULE_PAPER, UOT_RULE_POT = 0, 1
UOT_STORAGE_INPLACE, UOT_STORAGE_KFORM = 0, 1
UOT_SCHED_AUTO, UOT_SCHED_PASSES, UOT_SCHED_PERSISTENT = 0, 1, 2
UOT_DEV_ZERO_SUM, UOT_DEV_NONFINITE, UOT_DEV_TIMEOUT = 1, 2, 4


class UotOptions(ctypes.Structure):
    _fields_ = [("dtype", ctypes.c_int32), ("algo", ctypes.c_int32),
                ("check_every", ctypes.c_int32), ("tile", ctypes.c_int32),
                ("cluster", ctypes.c_int32), ("max_ctas", ctypes.c_int32),
                ("rule", ctypes.c_int32), ("storage", ctypes.c_int32),
                ("deterministic", ctypes.c_int32), ("schedule", ctypes.c_int32),
                ("reserved", ctypes.c_int32 * 1),
                ("pass_events", ctypes.c_void_p * 2)]


class UotResult(ctypes.Structure):
    _fields_ = [("iters_done", ctypes.c_int32), ("dev_status", ctypes.c_uint32),
                ("err", ctypes.c_double)]


class UotProblem(ctypes.Structure):
    _fields_ = [("plan", ctypes.c_void_p), ("ldp", ctypes.c_int64), ("n", ctypes.c_int64),
                ("m", ctypes.c_int64), ("a", ctypes.c_void_p), ("b", ctypes.c_void_p),
                ("reg", ctypes.c_float), ("reg_m", ctypes.c_float), ("iters", ctypes.c_int32),
                ("rule", ctypes.c_int32)]


class UotBatchTuning(ctypes.Structure):
    _fields_ = [("stages", ctypes.c_int32), ("max_team", ctypes.c_int32),
                ("target_elems", ctypes.c_double), ("resident_max_cluster", ctypes.c_int32),
                ("reserved", ctypes.c_int32 * 3)]


class UotError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {uot_status_string(status)} (status {status})")


_lib = None

# (name, restype, argtypes) of every exported symbol declared in include/uot.h.
_P, _I64, _I32, _F, _D, _SZ = (ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32,
                               ctypes.c_float, ctypes.c_double, ctypes.c_size_t)
SIGNATURES = {
    "uot_default_options": (None, [ctypes.POINTER(UotOptions)]),
    "uot_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "uot_workspace_size": (_SZ, [_I64, _I64, ctypes.POINTER(UotOptions)]),
    "uot_launch_count": (ctypes.c_uint64, []),
    "uot_selftest_wait": (ctypes.c_int, [_P, _I32, _I32, _D, _P, _P]),
    "uot_selftest_factor": (ctypes.c_int, [_P, _P, _I64, _F, _P, _P, _P]),
    "uot_init_kernel": (ctypes.c_int, [_P, _I64, _P, _I64, _I64, _I64, _F,
                                       ctypes.POINTER(UotOptions), _P]),
    "uot_sinkhorn": (ctypes.c_int, [_P, _I64, _P, _P, _I64, _I64, _F, _F, _I32, _D, _P, _SZ,
                                    ctypes.POINTER(UotOptions), _P, ctypes.POINTER(UotResult)]),
    "uot_read_result": (ctypes.c_int, [_P, _I64, _I64, ctypes.POINTER(UotOptions), _P,
                                       ctypes.POINTER(UotResult)]),
    "uot_cost": (ctypes.c_int, [_P, _I64, _P, _I64, _I64, _I64, _I32, _P, _P]),
    "uot_init_kernel_scaled": (ctypes.c_int, [_P, _I64, _P, _I64, _I64, _I64, _F, _F,
                                              ctypes.POINTER(UotOptions), _P]),
    "uot_sinkhorn_kform": (ctypes.c_int, [_P, _I64, _P, _P, _I64, _I64, _F, _F, _I32, _D, _F,
                                          _P, _P, _P, _SZ, ctypes.POINTER(UotOptions), _P,
                                          ctypes.POINTER(UotResult)]),
    "uot_kform_plan": (ctypes.c_int, [_P, _I64, _I32, _P, _P, _I64, _I64, _P, _I64, _I32, _P]),
    "uot_kform_cost": (ctypes.c_int, [_P, _I64, _I32, _P, _P, _P, _I64, _I64, _I64, _P, _P]),
    "uot_grad_hist_size": (_SZ, [_I64, _I64, _I32]),
    "uot_sinkhorn_kform_save": (ctypes.c_int, [_P, _I64, _P, _P, _I64, _I64, _F, _F, _I32, _F,
                                               _P, _P, _P, _SZ, _P, _SZ,
                                               ctypes.POINTER(UotOptions), _P,
                                               ctypes.POINTER(UotResult)]),
    "uot_backward_workspace_size": (_SZ, [_I64, _I64, _I32]),
    "uot_sinkhorn_backward": (ctypes.c_int, [_P, _I64, _P, _I64, _P, _P, _I64, _I64, _F, _F,
                                             _I32, _P, _SZ, _D, _P, _P, _I64, _P, _P, _P, _SZ,
                                             ctypes.POINTER(UotOptions), _P]),
    "uot_backward_batch_workspace_size": (_SZ, [_I32, _I64, _I64, _I32]),
    "uot_sinkhorn_backward_batch": (ctypes.c_int, [_I32, _P, _I64, _I64, _P, _I64, _I64, _P, _P,
                                                   _I64, _I64, _F, _F, _I32, _P, _SZ, _D, _P,
                                                   _P, _I64, _I64, _P, _P, _P, _SZ,
                                                   ctypes.POINTER(UotOptions), _P]),
    "uot_sinkhorn_noalloc": (ctypes.c_int, [_P, _I64, _P, _P, _I64, _I64, _F, _F, _I32, _D,
                                            ctypes.POINTER(UotOptions), _P,
                                            ctypes.POINTER(UotResult)]),
    "uot_shard_pass": (ctypes.c_int, [_P, _I64, _P, _I64, _I64, _F, _F, _I32, _P, _P, _P, _SZ,
                                      ctypes.POINTER(UotOptions), _P]),
    "uot_shard_factors": (ctypes.c_int, [_P, _P, _I64, _F, _F, _P, _P, _P]),
    "uot_shard_finish": (ctypes.c_int, [_P, _I64, _I64, _I64, _I32, _P, _P]),
    "uot_tensor3_workspace_size": (_SZ, [_I64, _I64, _I64]),
    "uot_sinkhorn_tensor3": (ctypes.c_int, [_P, _I64, _I64, _I64, _P, _P, _P, _F, _F, _I32, _P,
                                            _SZ, ctypes.POINTER(UotOptions), _P,
                                            ctypes.POINTER(UotResult)]),
    "uot_batch_default_tuning": (None, [ctypes.POINTER(UotBatchTuning)]),
    "uot_batched_workspace_size": (_SZ, [ctypes.POINTER(UotProblem), _I32,
                                         ctypes.POINTER(UotOptions)]),
    "uot_batched_prepare": (ctypes.c_int, [ctypes.POINTER(UotProblem), _I32,
                                           ctypes.POINTER(UotOptions),
                                           ctypes.POINTER(UotBatchTuning), _P, _SZ, _P]),
    "uot_sinkhorn_batched": (ctypes.c_int, [_P, _P]),
    "uot_batched_results": (ctypes.c_int, [_P, _I32, ctypes.POINTER(UotResult), _P]),
    "uot_batched_placement": (_I32, [_P, _I32, ctypes.POINTER(_I32), ctypes.POINTER(_I32)]),
    "uot_fused_config": (_I32, [_I32, ctypes.POINTER(_I32), ctypes.POINTER(_I32),
                                ctypes.POINTER(_I32), ctypes.POINTER(_I32)]),
}


def load(path: str = LIB_PATH):
    """Loads libuot.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libuot.so not found at {path}; build it with "
                           "paper_2412_11079_gb300.build.build()")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def uot_status_string(status: int) -> str:
    return load().uot_status_string(int(status)).decode()


def _check(status: int, where: str):
    if status != UOT_OK:
        raise UotError(status, where)


def _torch():
    import torch
    return torch


def dtype_code(t) -> int:
    torch = _torch()
    codes = {torch.float32: UOT_F32, torch.bfloat16: UOT_BF16, torch.float16: UOT_F16}
    if t not in codes:
        raise TypeError(f"unsupported plan dtype {t}")
    return codes[t]


def _matrix(x, name):
    if not x.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if x.dim() != 2 or (x.shape[1] > 1 and x.stride(1) != 1) or x.stride(0) < x.shape[1]:
        raise ValueError(f"{name} must be a row-major 2-D tensor (unit column stride)")
    return x.data_ptr(), int(x.stride(0))


def _batch_matrix(x, name):
    """(pointer, leading dimension, batch stride) of a [batch, rows, cols]
    tensor with unit column stride."""
    if not x.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if x.dim() != 3 or (x.shape[2] > 1 and x.stride(2) != 1) or x.stride(1) < x.shape[2]:
        raise ValueError(f"{name} must be a [batch, rows, cols] tensor with unit column stride")
    return x.data_ptr(), int(x.stride(1)), int(x.stride(0))


def _batch_vector(x, name, batch, length):
    torch = _torch()
    if (not x.is_cuda or x.dtype != torch.float32 or tuple(x.shape) != (batch, length)
            or not x.is_contiguous()):
        raise ValueError(f"{name} must be a contiguous CUDA float32 tensor of shape "
                         f"({batch}, {length})")
    return x.data_ptr()


def _vector(x, name, length):
    torch = _torch()
    if not x.is_cuda or x.dtype != torch.float32 or x.dim() != 1 or x.numel() != length:
        raise ValueError(f"{name} must be a CUDA float32 vector of length {length}")
    if length > 1 and x.stride(0) != 1:
        raise ValueError(f"{name} must be contiguous")
    return x.data_ptr()


def _stream(stream):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def options(dtype: int = UOT_F32, algo: int = UOT_ALGO_FUSED, check_every: int = 1,
            tile: int = 0, cluster: int = 0, max_ctas: int = 0,
            rule: int = UOT_RULE_PAPER, storage: int = UOT_STORAGE_INPLACE,
            deterministic: bool = False, schedule: int = UOT_SCHED_AUTO) -> UotOptions:
    o = UotOptions()
    load().uot_default_options(ctypes.byref(o))
    o.dtype, o.algo, o.check_every, o.tile, o.cluster = dtype, algo, check_every, tile, cluster
    o.max_ctas = max_ctas
    o.rule = rule
    o.storage = storage
    o.deterministic = 1 if deterministic else 0
    o.schedule = schedule
    return o


def uot_workspace_size(n: int, m: int, opt: UotOptions | None = None) -> int:
    return int(load().uot_workspace_size(n, m, ctypes.byref(opt) if opt else None))


def uot_launch_count() -> int:
    return int(load().uot_launch_count())


def uot_selftest_wait(counter, target: int, complete: bool, limit_s: float, status, stream=None):
    """Runs the bounded-wait self-test: `counter` a one-element int32 device
    tensor, `status` a two-element int32 device tensor receiving
    UOT_DEV_TIMEOUT or 0 for the barrier and the counter wait.  Async."""
    torch = _torch()
    if counter.dtype != torch.int32 or status.dtype != torch.int32 or status.numel() < 2:
        raise ValueError("counter and status must be int32 device tensors (status of 2)")
    _check(load().uot_selftest_wait(counter.data_ptr(), int(target), 1 if complete else 0,
                                    float(limit_s), status.data_ptr(), _stream(stream)),
           "uot_selftest_wait")


def uot_selftest_factor(target, total, fi: float, stream=None):
    """The library's rescaling factor (target/total)^fi for float32 device
    vectors; returns (factors, status bits)."""
    torch = _torch()
    n = target.numel()
    t = target.contiguous()
    s_ = total.contiguous()
    if t.dtype != torch.float32 or s_.dtype != torch.float32 or s_.numel() != n or not t.is_cuda:
        raise ValueError("target and total must be float32 CUDA vectors of one length")
    out = torch.empty_like(t)
    st = torch.zeros(1, dtype=torch.int32, device=t.device)
    _check(load().uot_selftest_factor(t.data_ptr(), s_.data_ptr(), n, float(fi), out.data_ptr(),
                                      st.data_ptr(), _stream(stream)), "uot_selftest_factor")
    return out, int(st.item())


def uot_fused_config(k: int):
    d, t, v, c = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    total = load().uot_fused_config(k, ctypes.byref(d), ctypes.byref(t), ctypes.byref(v),
                                    ctypes.byref(c))
    if k < 0 or k >= total:
        return total, None
    return total, {"dtype": d.value, "threads": t.value, "vecs": v.value, "cols": c.value}


def workspace(n: int, m: int, opt: UotOptions | None = None, device=None):
    """A caller-owned workspace tensor for uot_sinkhorn (256-byte aligned)."""
    torch = _torch()
    size = uot_workspace_size(n, m, opt)
    if size == 0:
        raise ValueError("bad problem size")
    buf = torch.empty(size + 256, dtype=torch.uint8, device=device or "cuda")
    off = (-buf.data_ptr()) % 256
    return buf[off:off + size]


def workspace_bytes(size: int, device=None):
    """A 256-byte aligned device byte buffer of `size` bytes."""
    torch = _torch()
    if size <= 0:
        raise ValueError("bad workspace size")
    buf = torch.empty(size + 256, dtype=torch.uint8, device=device or "cuda")
    off = (-buf.data_ptr()) % 256
    return buf[off:off + size]


def uot_init_kernel(C, plan, reg: float, opt: UotOptions | None = None, stream=None):
    n, m = C.shape
    if tuple(plan.shape) != (n, m):
        raise ValueError("plan and C shapes differ")
    if C.dtype != _torch().float32:
        raise ValueError("C must be float32")
    opt = opt or options(dtype_code(plan.dtype))
    if opt.dtype != dtype_code(plan.dtype):
        raise ValueError("options dtype does not match the plan tensor")
    cp, ldc = _matrix(C, "C")
    pp, ldp = _matrix(plan, "plan")
    _check(load().uot_init_kernel(cp, ldc, pp, ldp, n, m, reg, ctypes.byref(opt),
                                  _stream(stream)), "uot_init_kernel")


def uot_init_kernel_scaled(C, K, reg: float, log2_scale: int, opt: UotOptions | None = None,
                           stream=None):
    n, m = C.shape
    if tuple(K.shape) != (n, m) or C.dtype != _torch().float32:
        raise ValueError("K must have C's shape; C must be float32")
    opt = opt or options(dtype_code(K.dtype))
    cp, ldc = _matrix(C, "C")
    kp, ldk = _matrix(K, "K")
    _check(load().uot_init_kernel_scaled(cp, ldc, kp, ldk, n, m, reg, float(log2_scale),
                                         ctypes.byref(opt), _stream(stream)),
           "uot_init_kernel_scaled")


def uot_sinkhorn_kform(K, a, b, reg: float, reg_m: float, iters: int, tol: float = 0.0,
                       k_log2_scale: int = 0, U=None, V=None, ws=None,
                       opt: UotOptions | None = None, stream=None, sync: bool = True,
                       check_status: bool = True):
    """Kernel-form iteration on read-only K; returns (U, V, SinkhornResult or None)."""
    torch = _torch()
    n, m = K.shape
    opt = opt or options(dtype_code(K.dtype))
    if opt.dtype != dtype_code(K.dtype):
        raise ValueError("options dtype does not match K")
    U = torch.empty(n, dtype=torch.float32, device=K.device) if U is None else U
    V = torch.empty(m, dtype=torch.float32, device=K.device) if V is None else V
    if ws is None:
        ws = workspace(n, m, opt, K.device)
    kp, ldk = _matrix(K, "K")
    res = UotResult()
    st = load().uot_sinkhorn_kform(kp, ldk, _vector(a, "a", n), _vector(b, "b", m), n, m,
                                   float(reg), float(reg_m), int(iters), float(tol),
                                   float(k_log2_scale), _vector(U, "U", n), _vector(V, "V", m),
                                   ws.data_ptr(), ws.numel(), ctypes.byref(opt), _stream(stream),
                                   ctypes.byref(res) if sync else None)
    if not sync:
        _check(st, "uot_sinkhorn_kform")
        return U, V, None
    if st not in (UOT_OK, UOT_ERR_NONFINITE, UOT_ERR_ZERO_SUM, UOT_ERR_TIMEOUT) or (
            check_status and st != UOT_OK):
        raise UotError(st, "uot_sinkhorn_kform")
    return U, V, SinkhornResult(res.iters_done, res.dev_status, res.err)


def uot_kform_plan(K, U, V, plan=None, stream=None):
    torch = _torch()
    n, m = K.shape
    if plan is None:
        plan = torch.empty((n, m), dtype=torch.float32, device=K.device)
    kp, ldk = _matrix(K, "K")
    pp, ldp = _matrix(plan, "plan")
    _check(load().uot_kform_plan(kp, ldk, dtype_code(K.dtype), _vector(U, "U", n),
                                 _vector(V, "V", m), n, m, pp, ldp, dtype_code(plan.dtype),
                                 _stream(stream)), "uot_kform_plan")
    return plan


def uot_kform_cost(K, U, V, C, out=None, stream=None):
    torch = _torch()
    n, m = K.shape
    if out is None:
        out = torch.empty(1, dtype=torch.float64, device=K.device)
    kp, ldk = _matrix(K, "K")
    cp, ldc = _matrix(C, "C")
    _check(load().uot_kform_cost(kp, ldk, dtype_code(K.dtype), _vector(U, "U", n),
                                 _vector(V, "V", m), cp, ldc, n, m, out.data_ptr(),
                                 _stream(stream)), "uot_kform_cost")
    return out


@dataclass
class SinkhornResult:
    iters_done: int
    dev_status: int
    err: float


def uot_sinkhorn(plan, a, b, reg: float, reg_m: float, iters: int, tol: float = 0.0,
                 ws=None, opt: UotOptions | None = None, stream=None, sync: bool = True,
                 check_status: bool = True):
    """Runs ``iters`` iterations in place on ``plan``.  With ``sync`` the call
    waits and returns a SinkhornResult; otherwise it returns None and the
    result can be read with ``uot_read_result``."""
    n, m = plan.shape
    opt = opt or options(dtype_code(plan.dtype))
    if opt.dtype != dtype_code(plan.dtype):
        raise ValueError("options dtype does not match the plan tensor")
    if ws is None:
        ws = workspace(n, m, opt, plan.device)
    pp, ldp = _matrix(plan, "plan")
    res = UotResult()
    st = load().uot_sinkhorn(pp, ldp, _vector(a, "a", n), _vector(b, "b", m), n, m,
                             float(reg), float(reg_m), int(iters), float(tol), ws.data_ptr(),
                             ws.numel(), ctypes.byref(opt), _stream(stream),
                             ctypes.byref(res) if sync else None)
    if not sync:
        _check(st, "uot_sinkhorn")
        return None
    if st not in (UOT_OK, UOT_ERR_NONFINITE, UOT_ERR_ZERO_SUM, UOT_ERR_TIMEOUT) or (
            check_status and st != UOT_OK):
        raise UotError(st, "uot_sinkhorn")
    return SinkhornResult(res.iters_done, res.dev_status, res.err)


UOT_STATIC_SCRATCH_BYTES = 2 << 20


def uot_sinkhorn_noalloc(plan, a, b, reg: float, reg_m: float, iters: int, tol: float = 0.0,
                         opt: UotOptions | None = None, stream=None,
                         check_status: bool = True):
    """uot_sinkhorn on the library's built-in scratch array (no workspace, no
    device allocation); synchronous, returns a SinkhornResult."""
    n, m = plan.shape
    opt = opt or options(dtype_code(plan.dtype))
    if opt.dtype != dtype_code(plan.dtype):
        raise ValueError("options dtype does not match the plan tensor")
    pp, ldp = _matrix(plan, "plan")
    res = UotResult()
    st = load().uot_sinkhorn_noalloc(pp, ldp, _vector(a, "a", n), _vector(b, "b", m), n, m,
                                     float(reg), float(reg_m), int(iters), float(tol),
                                     ctypes.byref(opt), _stream(stream), ctypes.byref(res))
    if st not in (UOT_OK, UOT_ERR_NONFINITE, UOT_ERR_ZERO_SUM, UOT_ERR_TIMEOUT) or (
            check_status and st != UOT_OK):
        raise UotError(st, "uot_sinkhorn_noalloc")
    return SinkhornResult(res.iters_done, res.dev_status, res.err)


def uot_read_result(ws, n: int, m: int, opt: UotOptions | None = None, stream=None):
    res = UotResult()
    st = load().uot_read_result(ws.data_ptr(), n, m, ctypes.byref(opt) if opt else None,
                                _stream(stream), ctypes.byref(res))
    if st not in (UOT_OK, UOT_ERR_NONFINITE, UOT_ERR_ZERO_SUM, UOT_ERR_TIMEOUT):
        raise UotError(st, "uot_read_result")
    return SinkhornResult(res.iters_done, res.dev_status, res.err)


def uot_cost(plan, C, out=None, stream=None):
    """Transport cost <P, C> in FP64; returns a one-element CUDA float64 tensor."""
    torch = _torch()
    n, m = plan.shape
    if tuple(C.shape) != (n, m) or C.dtype != torch.float32:
        raise ValueError("C must be float32 with the plan's shape")
    if out is None:
        out = torch.empty(1, dtype=torch.float64, device=plan.device)
    pp, ldp = _matrix(plan, "plan")
    cp, ldc = _matrix(C, "C")
    _check(load().uot_cost(pp, ldp, cp, ldc, n, m, dtype_code(plan.dtype), out.data_ptr(),
                           _stream(stream)), "uot_cost")
    return out


def solve(C, a, b, reg: float, reg_m: float = math.inf, iters: int = 100, tol: float = 0.0,
          dtype=None, algo: int = UOT_ALGO_FUSED, check_every: int = 1, stream=None):
    """Convenience: P0 = exp(-C/reg), ``iters`` iterations, cost.  Returns
    ``(plan, cost_tensor, SinkhornResult)``; all on C's device."""
    torch = _torch()
    dtype = dtype or torch.float32
    n, m = C.shape
    plan = torch.empty((n, m), dtype=dtype, device=C.device)
    opt = options(dtype_code(dtype), algo, check_every)
    uot_init_kernel(C, plan, reg, opt, stream)
    res = uot_sinkhorn(plan, a, b, reg, reg_m, iters, tol, opt=opt, stream=stream)
    cost = uot_cost(plan, C, stream=stream)
    return plan, cost, res


def uot_shard_pass(plan, a, reg: float, reg_m: float, t: int, beta_in, colsum, ws=None,
                   opt: UotOptions | None = None, stream=None):
    """One fused pass over a row block (rows of `plan`, targets `a`): applies
    beta_in (None at t = 1), writes the block's column sums to `colsum`."""
    n, m = plan.shape
    opt = opt or options(dtype_code(plan.dtype))
    if ws is None:
        ws = workspace(n, m, opt, plan.device)
    pp, ldp = _matrix(plan, "plan")
    bp = None if beta_in is None else _vector(beta_in, "beta_in", m)
    _check(load().uot_shard_pass(pp, ldp, _vector(a, "a", n), n, m, float(reg), float(reg_m),
                                 int(t), bp, _vector(colsum, "colsum", m), ws.data_ptr(),
                                 ws.numel(), ctypes.byref(opt), _stream(stream)),
           "uot_shard_pass")
    return ws


def uot_shard_factors(colsum, b, reg: float, reg_m: float, beta, status=None, stream=None):
    m = b.numel()
    sp = None if status is None else status.data_ptr()
    _check(load().uot_shard_factors(_vector(colsum, "colsum", m), _vector(b, "b", m), m,
                                    float(reg), float(reg_m), _vector(beta, "beta", m), sp,
                                    _stream(stream)), "uot_shard_factors")


def uot_shard_finish(plan, beta, stream=None):
    n, m = plan.shape
    pp, ldp = _matrix(plan, "plan")
    _check(load().uot_shard_finish(pp, ldp, n, m, dtype_code(plan.dtype),
                                   _vector(beta, "beta", m), _stream(stream)),
           "uot_shard_finish")


def uot_sinkhorn_tensor3(P, a, b, c, reg: float, reg_m: float, iters: int, ws=None,
                         opt: UotOptions | None = None, stream=None, sync: bool = True,
                         check_status: bool = True):
    """Three-way form on the contiguous n1 x n2 x n3 tensor P, in place."""
    torch = _torch()
    if not P.is_cuda or P.dim() != 3 or not P.is_contiguous():
        raise ValueError("P must be a contiguous 3-D CUDA tensor")
    n1, n2, n3 = P.shape
    opt = opt or options(dtype_code(P.dtype))
    if ws is None:
        size = int(load().uot_tensor3_workspace_size(n1, n2, n3))
        if size == 0:
            raise ValueError("bad tensor size")
        ws = workspace_bytes(size, P.device)
    res = UotResult()
    st = load().uot_sinkhorn_tensor3(P.data_ptr(), n1, n2, n3, _vector(a, "a", n1),
                                     _vector(b, "b", n2), _vector(c, "c", n3), float(reg),
                                     float(reg_m), int(iters), ws.data_ptr(), ws.numel(),
                                     ctypes.byref(opt), _stream(stream),
                                     ctypes.byref(res) if sync else None)
    if not sync:
        _check(st, "uot_sinkhorn_tensor3")
        return None
    if st not in (UOT_OK, UOT_ERR_NONFINITE, UOT_ERR_ZERO_SUM, UOT_ERR_TIMEOUT) or (
            check_status and st != UOT_OK):
        raise UotError(st, "uot_sinkhorn_tensor3")
    return SinkhornResult(res.iters_done, res.dev_status, res.err)


def batch_tuning(stages: int | None = None, max_team: int | None = None,
                 target_elems: float | None = None,
                 resident_max_cluster: int | None = None) -> UotBatchTuning:
    t = UotBatchTuning()
    load().uot_batch_default_tuning(ctypes.byref(t))
    if stages is not None:
        t.stages = stages
    if max_team is not None:
        t.max_team = max_team
    if target_elems is not None:
        t.target_elems = target_elems
    if resident_max_cluster is not None:
        t.resident_max_cluster = resident_max_cluster
    return t


def uot_batched_workspace_size(probs) -> int:
    arr = (UotProblem * len(probs))(*probs)
    return int(load().uot_batched_workspace_size(arr, len(probs), None))


def uot_batched_prepare(probs, ws, tuning: UotBatchTuning | None = None, stream=None):
    arr = (UotProblem * len(probs))(*probs)
    _check(load().uot_batched_prepare(arr, len(probs), None,
                                      ctypes.byref(tuning) if tuning else None, ws.data_ptr(),
                                      ws.numel(), _stream(stream)), "uot_batched_prepare")


def uot_sinkhorn_batched(ws, stream=None):
    _check(load().uot_sinkhorn_batched(ws.data_ptr(), _stream(stream)), "uot_sinkhorn_batched")


def uot_batched_placement(ws, nprob: int, teams: bool = False):
    """Per prepared problem: its on-chip cluster size, or 0 if it streams;
    with teams=True also the streaming team size class (0 on chip)."""
    out = (_I32 * nprob)()
    team = (_I32 * nprob)()
    k = load().uot_batched_placement(ws.data_ptr(), nprob, out, team)
    if k < 0:
        raise UotError(UOT_ERR_INVALID_ARG, "uot_batched_placement")
    k = min(k, nprob)
    if teams:
        return list(out)[:k], list(team)[:k]
    return list(out)[:k]


def uot_batched_results(ws, nprob: int, stream=None, check_status: bool = True):
    out = (UotResult * nprob)()
    st = load().uot_batched_results(ws.data_ptr(), nprob, out, _stream(stream))
    if st not in (UOT_OK, UOT_ERR_NONFINITE, UOT_ERR_ZERO_SUM, UOT_ERR_TIMEOUT) or (
            check_status and st != UOT_OK):
        raise UotError(st, "uot_batched_results")
    return [SinkhornResult(r.iters_done, r.dev_status, r.err) for r in out]


def uot_sinkhorn_kform_save(K, a, b, reg: float, reg_m: float, iters: int, U=None, V=None,
                            hist=None, ws=None, stream=None, opt: UotOptions | None = None):
    """Kernel-form solve of exactly `iters` iterations that keeps the history
    its adjoint needs; returns (U, V, hist)."""
    torch = _torch()
    n, m = K.shape
    if K.dtype != torch.float32:
        raise ValueError("the differentiable solve keeps K in FP32")
    U = torch.empty(n, device=K.device) if U is None else U
    V = torch.empty(m, device=K.device) if V is None else V
    if hist is None:
        hist = workspace_bytes(int(load().uot_grad_hist_size(n, m, iters)), K.device)
    if ws is None:
        ws = workspace(n, m, None, K.device)
    kp, ldk = _matrix(K, "K")
    res = UotResult()
    _check(load().uot_sinkhorn_kform_save(kp, ldk, _vector(a, "a", n), _vector(b, "b", m), n, m,
                                          float(reg), float(reg_m), int(iters), 0.0,
                                          _vector(U, "U", n), _vector(V, "V", m),
                                          hist.data_ptr(), hist.numel(), ws.data_ptr(),
                                          ws.numel(), ctypes.byref(opt) if opt else None,
                                          _stream(stream), None),
           "uot_sinkhorn_kform_save")
    return U, V, hist


def grad_hist_batch(batch: int, n: int, m: int, iters: int, device=None):
    """Histories of `batch` solves for the batched adjoint: a [batch, stride]
    byte tensor, 256-byte aligned rows (one uot_sinkhorn_kform_save each)."""
    size = int(load().uot_grad_hist_size(n, m, int(iters)))
    if size == 0 or batch < 1:
        raise ValueError("bad problem size")
    stride = (size + 255) // 256 * 256
    return workspace_bytes(stride * batch, device).view(batch, stride)


def uot_sinkhorn_backward_batch(K, C, a, b, reg: float, reg_m: float, iters: int, hist,
                                grad_out: float = 1.0, dC=None, da=None, db=None, ws=None,
                                stream=None, opt: UotOptions | None = None, grad_out_dev=None):
    """Adjoint of `batch` solves of one shape in one set of launches (one per
    reverse step for the whole batch).  K, C, dC: [batch, n, m] (unit column
    stride); a, da: [batch, n]; b, db: [batch, m]; hist: [batch, stride]
    bytes from grad_hist_batch; grad_out_dev: None or a CUDA float64 tensor
    of `batch` per-problem factors."""
    torch = _torch()
    B, n, m = K.shape
    gdev = None
    if grad_out_dev is not None:
        if (not grad_out_dev.is_cuda or grad_out_dev.dtype != torch.float64
                or grad_out_dev.numel() != B or not grad_out_dev.is_contiguous()):
            raise ValueError("grad_out_dev must be a contiguous CUDA float64 tensor of batch "
                             "entries")
        gdev = grad_out_dev.data_ptr()
    if dC is None:
        dC = torch.empty((B, n, (m + 3) // 4 * 4), device=K.device)[:, :, :m]
    da = torch.empty((B, n), device=K.device) if da is None else da
    db = torch.empty((B, m), device=K.device) if db is None else db
    if ws is None:
        ws = workspace_bytes(int(load().uot_backward_batch_workspace_size(B, n, m, int(iters))),
                             K.device)
    if hist.dim() != 2 or hist.shape[0] != B or hist.dtype != torch.uint8 or hist.stride(1) != 1:
        raise ValueError("hist must be a [batch, stride] uint8 tensor (grad_hist_batch)")
    kp, ldk, sk = _batch_matrix(K, "K")
    cp, ldc, sc = _batch_matrix(C, "C")
    gp, ldd, sd = _batch_matrix(dC, "dC")
    _check(load().uot_sinkhorn_backward_batch(
        B, kp, ldk, sk, cp, ldc, sc, _batch_vector(a, "a", B, n), _batch_vector(b, "b", B, m),
        n, m, float(reg), float(reg_m), int(iters), hist.data_ptr(), int(hist.stride(0)),
        float(grad_out), gdev, gp, ldd, sd, _batch_vector(da, "da", B, n),
        _batch_vector(db, "db", B, m), ws.data_ptr(), ws.numel(),
        ctypes.byref(opt) if opt else None, _stream(stream)), "uot_sinkhorn_backward_batch")
    return dC, da, db


def uot_sinkhorn_backward(K, C, a, b, reg: float, reg_m: float, iters: int, hist,
                          grad_out: float = 1.0, dC=None, da=None, db=None, ws=None,
                          stream=None, opt: UotOptions | None = None, grad_out_dev=None):
    """Adjoint of the solve recorded in `hist`.  The gradients are scaled by
    grad_out, times the one-element float64 device tensor grad_out_dev if
    given (read on the device, no synchronisation)."""
    torch = _torch()
    gdev = None
    if grad_out_dev is not None:
        if (not grad_out_dev.is_cuda or grad_out_dev.dtype != torch.float64
                or grad_out_dev.numel() != 1):
            raise ValueError("grad_out_dev must be a one-element CUDA float64 tensor")
        gdev = grad_out_dev.data_ptr()
    n, m = K.shape
    dC = torch.empty((n, (m + 3) // 4 * 4), device=K.device)[:, :m] if dC is None else dC
    da = torch.empty(n, device=K.device) if da is None else da
    db = torch.empty(m, device=K.device) if db is None else db
    if ws is None:
        ws = workspace_bytes(int(load().uot_backward_workspace_size(n, m, int(iters))), K.device)
    kp, ldk = _matrix(K, "K")
    cp, ldc = _matrix(C, "C")
    gp, ldd = _matrix(dC, "dC")
    _check(load().uot_sinkhorn_backward(kp, ldk, cp, ldc, _vector(a, "a", n), _vector(b, "b", m),
                                        n, m, float(reg), float(reg_m), int(iters),
                                        hist.data_ptr(), hist.numel(), float(grad_out), gdev, gp,
                                        ldd,
                                        _vector(da, "da", n), _vector(db, "db", m),
                                        ws.data_ptr(), ws.numel(),
                                        ctypes.byref(opt) if opt else None, _stream(stream)),
           "uot_sinkhorn_backward")
    return dC, da, db
