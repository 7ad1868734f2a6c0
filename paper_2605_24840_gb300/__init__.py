"""Python binding of librsign, the GB300 shifted matrix-sign reflector library.

Argument marshalling only: every step of the computation runs in the CUDA
kernels of ``librsign.so`` (built from ``csrc/`` for sm_103a).  There is no
CPU fallback; importing the binding without the built library raises.

Tensors may be torch tensors (CUDA or CPU) or numpy arrays; float64,
C-contiguous.  CUDA tensors are passed as device pointers on the current
torch stream; host arrays are passed as host pointers and the library copies
them in and out itself.
"""
from __future__ import annotations

import ctypes
import enum
import math
import os
import re

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "librsign.so")
HEADERS = [os.path.join(_HERE, "..", "include", h) for h in ("rsign.h", "rsign_debug.h")]


class Policy(enum.IntEnum):
    FP64 = 0
    FP16 = 1
    BF16 = 2
    FP16_POLISH = 3
    BF16_POLISH = 4
    FP16_REFINE = 5
    BF16_REFINE = 6
    FP32 = 7


class Status(enum.IntEnum):
    OK = 0
    ERR_ARG = 1
    ERR_NOCONV = 2
    ERR_CERT = 3
    ERR_GAP = 4
    ERR_CUDA = 5
    ERR_TIMEOUT = 6
    ERR_UNSUPPORTED = 7


class AlphaMode(enum.IntEnum):
    INF = 0
    POWER = 1


class Info(ctypes.Structure):
    _fields_ = [
        ("steps_low", ctypes.c_int32), ("steps_fp64", ctypes.c_int32),
        ("sweeps_refine", ctypes.c_int32), ("cert_ok", ctypes.c_int32),
        ("alpha", ctypes.c_double), ("shift", ctypes.c_double), ("gamma_est", ctypes.c_double),
        ("resid_fro", ctypes.c_double), ("trace", ctypes.c_double),
        ("correction_fro", ctypes.c_double), ("commutator_norm", ctypes.c_double),
        ("err_est", ctypes.c_double),
        ("tol_fro", ctypes.c_double), ("ms_total", ctypes.c_double), ("ms_low", ctypes.c_double),
        ("ms_fp64", ctypes.c_double), ("flops_low", ctypes.c_double),
        ("launches", ctypes.c_int64), ("workspace_bytes", ctypes.c_int64),
        ("lam_k_est", ctypes.c_double), ("lam_k1_est", ctypes.c_double), ("shift_eps", ctypes.c_double),
        ("margin_lb", ctypes.c_double), ("lanczos_iters", ctypes.c_int32), ("steps_pred", ctypes.c_int32),
        ("batch_grouped", ctypes.c_int32), ("batch_tile", ctypes.c_int32),
        ("ns_scaled_steps", ctypes.c_int32), ("refine_levels", ctypes.c_int32),
        ("err_bound", ctypes.c_double),
    ]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class Options(ctypes.Structure):
    _fields_ = [
        ("max_steps", ctypes.c_int32), ("polish_steps", ctypes.c_int32),
        ("max_sweeps", ctypes.c_int32), ("alpha_mode", ctypes.c_int32),
        ("power_steps", ctypes.c_int32), ("timing", ctypes.c_int32),
        ("low_split", ctypes.c_int32), ("lanczos_max", ctypes.c_int32),
        ("batch_graphs", ctypes.c_int32), ("batch_tile", ctypes.c_int32),
        ("ns_scaling", ctypes.c_int32), ("margin", ctypes.c_double),
        ("refine_stop", ctypes.c_int32), ("engine", ctypes.c_int32),
    ]


class Engine(enum.IntEnum):
    NS3 = 0
    NS5 = 1


class RefineStop(enum.IntEnum):
    ESTIMATE = 0
    BOUND = 1


class ShiftPolicy(enum.IntEnum):
    MIDPOINT = 0
    REUSE_REFRESH = 1
    DAMPED = 2


class ShiftState(ctypes.Structure):
    _fields_ = [
        ("shift", ctypes.c_double), ("lam_k_est", ctypes.c_double), ("lam_k1_est", ctypes.c_double),
        ("eps", ctypes.c_double), ("margin_cert", ctypes.c_double), ("drift_sum", ctypes.c_double),
        ("refreshes", ctypes.c_int32), ("reuses", ctypes.c_int32),
    ]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class ShiftReport(ctypes.Structure):
    _fields_ = [
        ("refreshed", ctypes.c_int32), ("lanczos_iters", ctypes.c_int32), ("drift_ub", ctypes.c_double),
        ("drift_est", ctypes.c_double), ("margin_cert", ctypes.c_double),
    ]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class RsignError(RuntimeError):
    def __init__(self, status, msg=""):
        self.status = Status(status)
        super().__init__("%s (%s)%s" % (self.status.name, status_str(status), (": " + msg) if msg else ""))


_lib = None


def header_functions():
    """Names of every function declared in include/*.h (the exported C ABI)."""
    names = []
    for h in HEADERS:
        with open(h) as f:
            txt = f.read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        names += re.findall(r"\b(rsign_\w+)\s*\(", txt)
    return sorted(set(names))


def load():
    """Load librsign.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError("librsign.so not built: run __graft_entry__.build() (expected at %s)" % LIB_PATH)
    lib = ctypes.CDLL(LIB_PATH)
    dp, vp, i64, i32, dbl = (ctypes.POINTER(ctypes.c_double), ctypes.c_void_p, ctypes.c_int64,
                             ctypes.c_int32, ctypes.c_double)
    lib.rsign_options_default.argtypes = [ctypes.POINTER(Options)]
    lib.rsign_options_default.restype = None
    lib.rsign_reflector.argtypes = [vp, i64, i32, dbl, dbl, ctypes.c_int, vp, ctypes.POINTER(Info), vp]
    lib.rsign_reflector.restype = ctypes.c_int
    lib.rsign_reflector_ex.argtypes = [vp, i64, i32, dbl, dbl, ctypes.c_int, ctypes.POINTER(Options), vp,
                                       ctypes.POINTER(Info), vp]
    lib.rsign_reflector_ex.restype = ctypes.c_int
    lib.rsign_apply.argtypes = [vp, i64, vp, i64, vp, vp]
    lib.rsign_apply.restype = ctypes.c_int
    lib.rsign_reflector_batched.argtypes = [i32, ctypes.POINTER(vp), ctypes.POINTER(i64), ctypes.POINTER(i32),
                                            ctypes.POINTER(dbl), dbl, ctypes.c_int, ctypes.POINTER(vp),
                                            ctypes.POINTER(Info), vp]
    lib.rsign_reflector_batched.restype = ctypes.c_int
    lib.rsign_reflector_batched_ex.argtypes = [i32, ctypes.POINTER(vp), ctypes.POINTER(i64), ctypes.POINTER(i32),
                                               ctypes.POINTER(dbl), dbl, ctypes.c_int, ctypes.POINTER(Options),
                                               ctypes.POINTER(vp), ctypes.POINTER(Info), vp]
    lib.rsign_reflector_batched_ex.restype = ctypes.c_int
    lib.rsign_shift_state_init.argtypes = [ctypes.POINTER(ShiftState)]
    lib.rsign_shift_state_init.restype = None
    lib.rsign_shift_can_reuse.argtypes = [ctypes.POINTER(ShiftState), dbl, dbl]
    lib.rsign_shift_can_reuse.restype = i32
    lib.rsign_shift_damped.argtypes = [dbl, dbl, dbl, dbl, dbl]
    lib.rsign_shift_damped.restype = dbl
    lib.rsign_shift_update.argtypes = [vp, vp, i64, i32, ctypes.c_int, dbl, dbl, dbl, ctypes.POINTER(ShiftState),
                                       ctypes.POINTER(ShiftReport), vp]
    lib.rsign_shift_update.restype = ctypes.c_int
    lib.rsign_reflector_backward.argtypes = [vp, i64, i32, dbl, ctypes.c_int, vp, vp, i32, vp]
    lib.rsign_reflector_backward.restype = ctypes.c_int
    lib.rsign_status_str.argtypes = [ctypes.c_int]
    lib.rsign_status_str.restype = ctypes.c_char_p
    lib.rsign_version.argtypes = []
    lib.rsign_version.restype = ctypes.c_char_p
    lib.rsign_trim_workspace.argtypes = []
    lib.rsign_trim_workspace.restype = ctypes.c_int
    lib.rsign_dbg_tc_gemm.argtypes = [vp, vp, i64, i32, i32, vp, vp, vp]
    lib.rsign_dbg_tc_gemm.restype = ctypes.c_int
    lib.rsign_dbg_f64_gemm.argtypes = [vp, vp, i64, i32, vp, vp]
    lib.rsign_dbg_f64_gemm.restype = ctypes.c_int
    lib.rsign_dbg_fp64grade_gemm.argtypes = [vp, vp, i64, i64, i32, vp, vp]
    lib.rsign_dbg_fp64grade_gemm.restype = ctypes.c_int
    lib.rsign_dbg_set_refine_levels.argtypes = [i32, i32, i32]
    lib.rsign_dbg_set_refine_levels.restype = i32
    lib.rsign_dbg_set_ozaki_tile.argtypes = [i32]
    lib.rsign_dbg_set_ozaki_tile.restype = i32
    lib.rsign_dbg_stage_plan.argtypes = [dbl, dbl, i32, i32, i32, dp, ctypes.POINTER(i32), ctypes.POINTER(i32)]
    lib.rsign_dbg_stage_plan.restype = ctypes.c_int
    lib.rsign_dbg_set_split_until.argtypes = [dbl]
    lib.rsign_dbg_set_split_until.restype = dbl
    lib.rsign_dbg_set_copy_streams.argtypes = [i32]
    lib.rsign_dbg_set_copy_streams.restype = i32
    lib.rsign_dbg_set_host_mapped.argtypes = [i32]
    lib.rsign_dbg_set_host_mapped.restype = i32
    lib.rsign_dbg_set_tangent_cut.argtypes = [i32]
    lib.rsign_dbg_set_tangent_cut.restype = i32
    lib.rsign_dbg_set_split_steps.argtypes = [i32]
    lib.rsign_dbg_set_split_steps.restype = i32
    lib.rsign_dbg_set_digit_fp8.argtypes = [i32]
    lib.rsign_dbg_set_digit_fp8.restype = i32
    lib.rsign_dbg_bounded_wait.argtypes = [i32, i64, vp, vp]
    lib.rsign_dbg_bounded_wait.restype = ctypes.c_int
    lib.rsign_dbg_tile_order.argtypes = [i64, i32, ctypes.POINTER(i32), ctypes.POINTER(i32)]
    lib.rsign_dbg_tile_order.restype = i32
    lib.rsign_dbg_fp64e_gemm.argtypes = [vp, vp, i64, i64, i32, vp, vp]
    lib.rsign_dbg_fp64e_gemm.restype = ctypes.c_int
    lib.rsign_dbg_gemv_df.argtypes = [vp, vp, i64, vp, vp]
    lib.rsign_dbg_gemv_df.restype = ctypes.c_int
    lib.rsign_dbg_sym_gemv_tiles.argtypes = [i64, ctypes.POINTER(i32), ctypes.POINTER(i32)]
    lib.rsign_dbg_sym_gemv_tiles.restype = i32
    lib.rsign_dbg_spectral_norm.argtypes = [vp, i64, i32, i32, ctypes.POINTER(ctypes.c_double), vp]
    lib.rsign_dbg_spectral_norm.restype = ctypes.c_int
    lib.rsign_dbg_gemv_df_sym.argtypes = [vp, vp, i64, vp, vp]
    lib.rsign_dbg_gemv_df_sym.restype = ctypes.c_int
    lib.rsign_dbg_oz_convert.argtypes = [vp, vp, i64, vp, vp, vp]
    lib.rsign_dbg_oz_convert.restype = ctypes.c_int
    lib.rsign_dbg_commutator_check.argtypes = [vp, vp, i64, i64, i32, vp, vp]
    lib.rsign_dbg_commutator_check.restype = ctypes.c_int
    lib.rsign_dbg_tridiag_ritz.argtypes = [dp, dp, i32, i32, dp, dp]
    lib.rsign_dbg_tridiag_ritz.restype = ctypes.c_int
    lib.rsign_dbg_scaled_coeffs.argtypes = [dbl, dbl, i32, dp, ctypes.POINTER(i32)]
    lib.rsign_dbg_scaled_coeffs.restype = ctypes.c_int
    lib.rsign_dbg_gamma_from_steps.argtypes = [i32, dp]
    lib.rsign_dbg_gamma_from_steps.restype = ctypes.c_int
    lib.rsign_dbg_batch_units.argtypes = [i32, ctypes.POINTER(i32), i32, i32, i32, i32, ctypes.POINTER(i32),
                                          ctypes.POINTER(i32)]
    lib.rsign_dbg_batch_units.restype = i32
    lib.rsign_dbg_refine_levels.argtypes = [dbl, dbl, dbl, i64, dbl, i32]
    lib.rsign_dbg_refine_levels.restype = i32
    lib.rsign_dbg_fp64e_beta.argtypes = [i64]
    lib.rsign_dbg_fp64e_beta.restype = i32
    ip = ctypes.POINTER(i32)
    lib.rsign_dbg_fp64e_plan.argtypes = [i32, i32, i32, i64, ip, ip, ip, ip, ip, ip]
    lib.rsign_dbg_fp64e_plan.restype = ctypes.c_int
    _lib = lib
    return lib


def status_str(code) -> str:
    return load().rsign_status_str(int(code)).decode()


def version() -> str:
    return load().rsign_version().decode()


def trim_workspace() -> None:
    """Return the workspace memory cached by earlier calls to the driver (rsign_trim_workspace)."""
    st = Status(load().rsign_trim_workspace())
    if st != Status.OK:
        raise RsignError(st)


def default_options(**kw) -> Options:
    o = Options()
    load().rsign_options_default(ctypes.byref(o))
    for k, v in kw.items():
        setattr(o, k, float(v) if k == "margin" else int(v))
    return o


# ----------------------------------------------------------------------------
# marshalling helpers
# ----------------------------------------------------------------------------
def _torch():
    import torch
    return torch


def _ptr_of(x, name, shape=None, dtype="float64"):
    """(pointer, keepalive, is_cuda) of a float64 C-contiguous array/tensor."""
    if isinstance(x, np.ndarray):
        if x.dtype != np.dtype(dtype) or not x.flags["C_CONTIGUOUS"]:
            raise TypeError("%s must be a C-contiguous %s numpy array" % (name, dtype))
        if shape is not None and tuple(x.shape) != tuple(shape):
            raise ValueError("%s has shape %s, expected %s" % (name, x.shape, shape))
        return x.ctypes.data, x, False
    torch = _torch()
    if isinstance(x, torch.Tensor):
        tdt = getattr(torch, dtype)
        if x.dtype != tdt or not x.is_contiguous():
            raise TypeError("%s must be a contiguous torch.%s tensor" % (name, dtype))
        if shape is not None and tuple(x.shape) != tuple(shape):
            raise ValueError("%s has shape %s, expected %s" % (name, tuple(x.shape), shape))
        return x.data_ptr(), x, x.is_cuda
    raise TypeError("%s: expected a numpy array or torch tensor" % name)


def _stream_ptr(stream, any_cuda):
    if stream is not None:
        return int(getattr(stream, "cuda_stream", stream))
    if any_cuda:
        return int(_torch().cuda.current_stream().cuda_stream)
    return 0


def _like(x, shape):
    if isinstance(x, np.ndarray):
        return np.empty(shape, dtype=np.float64)
    torch = _torch()
    return torch.empty(shape, dtype=torch.float64, device=x.device)


# ----------------------------------------------------------------------------
# public calls (same names as the C ABI, without the prefix)
# ----------------------------------------------------------------------------
def reflector(H, k, s, tol=1e-12, policy=Policy.FP64, out=None, options=None, stream=None,
              check=True):
    """R = sign(H - sI) = I - 2 P_k via rsign_reflector_ex.  Returns (R, Info, Status).

    With check=True a status other than OK raises RsignError (R and info are
    attached to the exception as .R and .info).
    """
    lib = load()
    d = int(H.shape[0])
    hp, hk, hc = _ptr_of(H, "H", (d, d))
    if out is None:
        out = _like(H, (d, d))
    rp, rk, rc = _ptr_of(out, "out", (d, d))
    info = Info()
    opt = options if options is not None else default_options()
    st = lib.rsign_reflector_ex(hp, d, int(k), float("nan") if s is None else float(s), float(tol),
                                int(policy), ctypes.byref(opt), rp, ctypes.byref(info),
                                _stream_ptr(stream, hc or rc))
    st = Status(st)
    if check and st != Status.OK:
        e = RsignError(st)
        e.R, e.info = out, info
        raise e
    return out, info, st


def apply(R, V, out=None, stream=None):
    """out = R V (rsign_apply); V is d x nv."""
    lib = load()
    d = int(R.shape[0])
    if V.ndim == 1:
        V = V.reshape(d, 1)
    nv = int(V.shape[1])
    rp, rk, rc = _ptr_of(R, "R", (d, d))
    vp, vk, vc = _ptr_of(V, "V", (d, nv))
    if out is None:
        out = _like(V, (d, nv))
    op, ok, oc = _ptr_of(out, "out", (d, nv))
    st = Status(lib.rsign_apply(rp, d, vp, nv, op, _stream_ptr(stream, rc or vc or oc)))
    if st != Status.OK:
        raise RsignError(st)
    return out


def reflector_batched(Hs, ks, ss, tol=1e-12, policy=Policy.FP64, outs=None, options=None, stream=None):
    """Independent reflectors for a list of matrices (rsign_reflector_batched_ex).

    Returns (outs, infos, status); status is the first non-OK status in index
    order, infos[i].batch_grouped tells whether matrix i went through the
    grouped launches."""
    lib = load()
    n = len(Hs)
    outs = outs if outs is not None else [_like(H, H.shape) for H in Hs]
    keep = []
    hp = (ctypes.c_void_p * n)()
    rp = (ctypes.c_void_p * n)()
    dd = (ctypes.c_int64 * n)()
    kk = (ctypes.c_int32 * n)()
    sv = (ctypes.c_double * n)()
    any_cuda = False
    for i, (H, R) in enumerate(zip(Hs, outs)):
        d = int(H.shape[0])
        p, kp, c1 = _ptr_of(H, "H[%d]" % i, (d, d))
        q, kq, c2 = _ptr_of(R, "R[%d]" % i, (d, d))
        keep += [kp, kq]
        any_cuda |= c1 or c2
        hp[i], rp[i], dd[i], kk[i] = p, q, d, int(ks[i])
        sv[i] = float("nan") if ss[i] is None else float(ss[i])
    infos = (Info * n)()
    optp = ctypes.byref(options) if options is not None else None
    st = Status(lib.rsign_reflector_batched_ex(n, hp, dd, kk, sv, float(tol), int(policy), optp, rp, infos,
                                               _stream_ptr(stream, any_cuda)))
    return outs, list(infos), st


def shift_state() -> ShiftState:
    """A fresh shift-policy state (no shift yet)."""
    st = ShiftState()
    load().rsign_shift_state_init(ctypes.byref(st))
    return st


def shift_can_reuse(state: ShiftState, drift_ub: float, threshold: float = 0.0) -> bool:
    """Prop. 4.2 reuse rule on the host (rsign_shift_can_reuse)."""
    return bool(load().rsign_shift_can_reuse(ctypes.byref(state), float(drift_ub), float(threshold)))


def shift_damped(s_prev, lam_k_est, lam_k1_est, eps, damping) -> float:
    """Damped midpoint clipped into the certified interval (rsign_shift_damped)."""
    return float(load().rsign_shift_damped(float(s_prev), float(lam_k_est), float(lam_k1_est), float(eps),
                                           float(damping)))


def shift_update(H_new, H_old, k, state: ShiftState, policy=ShiftPolicy.REUSE_REFRESH, threshold=0.0,
                 damping=0.5, drift_bound=None, stream=None):
    """Shift for H_new given the state left by H_old (rsign_shift_update).

    drift_bound: a caller-certified bound on ||H_new - H_old||_2, or None for
    the GPU's rigorous bound from H_old.  Updates ``state`` in place and
    returns (status, report)."""
    lib = load()
    d = int(H_new.shape[0])
    hp, hk, hc = _ptr_of(H_new, "H_new", (d, d))
    if H_old is not None:
        op, ok, oc = _ptr_of(H_old, "H_old", (d, d))
    else:
        op, ok, oc = None, None, False
    rep = ShiftReport()
    db = float("nan") if drift_bound is None else float(drift_bound)
    st = Status(lib.rsign_shift_update(hp, op, d, int(k), int(policy), float(threshold), float(damping), db,
                                       ctypes.byref(state), ctypes.byref(rep), _stream_ptr(stream, hc or oc)))
    return st, rep


def reflector_backward(H, k, s, Rbar, policy=Policy.FP64, ckpt_every=4, out=None, stream=None):
    """Hbar = dL/dH given Rbar = dL/dR (rsign_reflector_backward)."""
    lib = load()
    d = int(H.shape[0])
    hp, hk, hc = _ptr_of(H, "H", (d, d))
    bp, bk, bc = _ptr_of(Rbar, "Rbar", (d, d))
    if out is None:
        out = _like(H, (d, d))
    op, ok, oc = _ptr_of(out, "out", (d, d))
    st = Status(lib.rsign_reflector_backward(hp, d, int(k), float(s), int(policy), bp, op, int(ckpt_every),
                                             _stream_ptr(stream, hc or bc or oc)))
    if st != Status.OK:
        raise RsignError(st)
    return out


def _autograd_function():
    torch = _torch()

    class SignReflector(torch.autograd.Function):
        """R = sign(H - sI) with the hand-written Newton-Schulz adjoint as its backward.

        forward: rsign_reflector (s = None: automatic shift, then frozen);
        backward: rsign_reflector_backward with s and alpha held fixed."""

        @staticmethod
        def forward(ctx, H, k, s, policy, tol, ckpt_every):
            R, info, st = reflector(H.detach(), k, s, tol=tol, policy=policy, check=True)
            ctx.save_for_backward(H.detach())
            ctx.k, ctx.s, ctx.policy, ctx.ckpt = int(k), float(info.shift), policy, int(ckpt_every)
            return R

        @staticmethod
        def backward(ctx, Rbar):
            (H,) = ctx.saved_tensors
            Hbar = reflector_backward(H, ctx.k, ctx.s, Rbar.detach().contiguous(), policy=ctx.policy,
                                      ckpt_every=ctx.ckpt)
            return Hbar, None, None, None, None, None

    return SignReflector


_SIGN_FN = None


def sign_reflector(H, k, s=None, policy=Policy.FP64, tol=1e-12, ckpt_every=4):
    """Differentiable R_k = sign(H - sI) for a float64 CUDA tensor H (torch.autograd).

    The gradient is the adjoint of the Newton-Schulz map with s and alpha
    frozen (Gershgorin alpha, the default of the forward call)."""
    global _SIGN_FN
    if _SIGN_FN is None:
        _SIGN_FN = _autograd_function()
    return _SIGN_FN.apply(H, int(k), s, Policy(policy), float(tol), int(ckpt_every))


# debug products (kernel-level tests)
def dbg_tc_gemm(A, B, fmt=0, sym=0, out=None, stream=None):
    """out = A B^T on the tcgen05 path (A, B: dp x dp CUDA fp16/bf16 tensors)."""
    torch = _torch()
    lib = load()
    dp = int(A.shape[0])
    if out is None:
        out = torch.empty((dp, dp), dtype=torch.float32, device=A.device)
    status = torch.zeros(1, dtype=torch.int32, device=A.device)
    st = Status(lib.rsign_dbg_tc_gemm(A.data_ptr(), B.data_ptr(), dp, int(fmt), int(sym), out.data_ptr(),
                                      status.data_ptr(), _stream_ptr(stream, True)))
    if st != Status.OK:
        raise RsignError(st)
    return out, status


def dbg_f64_gemm(A, B, sym=0, out=None, stream=None):
    torch = _torch()
    lib = load()
    dp = int(A.shape[0])
    if out is None:
        out = torch.empty((dp, dp), dtype=torch.float64, device=A.device)
    st = Status(lib.rsign_dbg_f64_gemm(A.data_ptr(), B.data_ptr(), dp, int(sym), out.data_ptr(),
                                       _stream_ptr(stream, True)))
    if st != Status.OK:
        raise RsignError(st)
    return out


def dbg_tridiag_ritz(alpha, beta, j):
    """(theta_j, last component) of the symmetric tridiagonal (alpha, beta) -- host routine, no GPU."""
    a = np.ascontiguousarray(alpha, dtype=np.float64)
    b = np.ascontiguousarray(beta, dtype=np.float64)
    th, la = ctypes.c_double(), ctypes.c_double()
    p = ctypes.POINTER(ctypes.c_double)
    st = Status(load().rsign_dbg_tridiag_ritz(a.ctypes.data_as(p), b.ctypes.data_as(p), len(a), int(j),
                                               ctypes.byref(th), ctypes.byref(la)))
    if st != Status.OK:
        raise RsignError(st)
    return th.value, la.value


def dbg_scaled_coeffs(alpha_margin, u0=1.0):
    """Step scalings of the scaled steps for l0 = alpha * margin (host routine, no GPU)."""
    lib = load()
    n = ctypes.c_int32()
    buf = (ctypes.c_double * 256)()
    st = Status(lib.rsign_dbg_scaled_coeffs(float(alpha_margin), float(u0), 256, buf, ctypes.byref(n)))
    if st != Status.OK:
        raise RsignError(st)
    return [buf[i] for i in range(min(n.value, 256))]


def dbg_gamma_from_steps(m: int) -> float:
    """Margin lower bound implied by a plain trajectory stopping after m steps (host routine, no GPU)."""
    g = ctypes.c_double()
    st = Status(load().rsign_dbg_gamma_from_steps(int(m), ctypes.byref(g)))
    if st != Status.OK:
        raise RsignError(st)
    return g.value


def dbg_batch_units(dps, bn, sym=1, order=0):
    """Tile table of the grouped batched launches (host routine, no GPU):
    (list of (matrix, tile row, tile column, slot), slot_begin)."""
    lib = load()
    i32 = ctypes.c_int32
    n = len(dps)
    d = (i32 * max(n, 1))(*[int(x) for x in dps])
    cnt = lib.rsign_dbg_batch_units(n, d, int(bn), int(sym), int(order), 0, None, None)
    if cnt < 0:
        raise RsignError(Status.ERR_ARG)
    u = (i32 * (4 * max(cnt, 1)))()
    sb = (i32 * (n + 1))()
    lib.rsign_dbg_batch_units(n, d, int(bn), int(sym), int(order), cnt, u, sb)
    return [tuple(u[4 * i:4 * i + 4]) for i in range(cnt)], list(sb)


def dbg_refine_levels(tol, s_a, s_r, d, mu, k):
    """(first sweep's R A levels, polish levels) chosen by rule (host routine, no GPU)."""
    v = int(load().rsign_dbg_refine_levels(float(tol), float(s_a), float(s_r), int(d), float(mu), int(k)))
    if v < 0:
        raise RsignError(Status.ERR_ARG)
    return v & 0xFFFF, v >> 16


def dbg_fp64e_beta(k_extent: int) -> int:
    """Digit width of the FP64-emulating products for an inner extent (host routine, no GPU)."""
    return int(load().rsign_dbg_fp64e_beta(int(k_extent)))


def dbg_fp64e_plan(n_planes, beta, levels, k_extent):
    """Accumulation plan of an FP64-grade product (host routine, no GPU): a dict
    with the groups (list of (pair list, shift, super-group)), the number of
    int64 sums and the unit exponents."""
    lib = load()
    i32 = ctypes.c_int32
    meta = (i32 * 5)()
    gs, pa, pb = (i32 * 33)(), (i32 * 72)(), (i32 * 72)()
    sh, sg = (i32 * 32)(), (i32 * 32)()
    st = Status(lib.rsign_dbg_fp64e_plan(int(n_planes), int(beta), int(levels), int(k_extent), meta, gs, pa, pb,
                                         sh, sg))
    if st != Status.OK:
        raise RsignError(st)
    G = meta[0]
    groups = [([(pa[r], pb[r]) for r in range(gs[g], gs[g + 1])], sh[g], sg[g]) for g in range(G)]
    return {"groups": groups, "n_pairs": meta[1], "n_sg": meta[2], "unit_exp": meta[3], "sh01": meta[4]}




def dbg_fp64grade_gemm(A, B, d_real=None, sym=0, out=None, stream=None):
    """out = A B (FP64-grade, digit planes on the FP16 tensor cores); A, B symmetric CUDA float64."""
    torch = _torch()
    lib = load()
    dp = int(A.shape[0])
    if out is None:
        out = torch.empty((dp, dp), dtype=torch.float64, device=A.device)
    st = Status(lib.rsign_dbg_fp64grade_gemm(A.data_ptr(), B.data_ptr(), dp, int(d_real or dp), int(sym),
                                             out.data_ptr(), _stream_ptr(stream, True)))
    if st != Status.OK:
        raise RsignError(st)
    return out


def dbg_stage_plan(alpha_margin, u0=1.0, scaled=True, max_steps=100, steps_low=None):
    """(lower ends l_0..l_max_steps, n_split, m_tangent) of the REFINE stage plan (host only)."""
    lib = load()
    steps_low = max_steps if steps_low is None else steps_low
    le = np.empty(max_steps + 1)
    ns, mt = ctypes.c_int32(0), ctypes.c_int32(0)
    st = Status(lib.rsign_dbg_stage_plan(float(alpha_margin), float(u0), int(bool(scaled)), int(max_steps),
                                         int(steps_low), le.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                         ctypes.byref(ns), ctypes.byref(mt)))
    if st != Status.OK:
        raise RsignError(st)
    return le, int(ns.value), int(mt.value)


def dbg_set_split_until(l):
    """Threshold of the stage-1 split rule (pairs while the known lower end is below l); returns the
    previous threshold."""
    return float(load().rsign_dbg_set_split_until(float(l)))


def dbg_set_copy_streams(n):
    """Staged host copies split over n streams (1..8); returns the previous setting."""
    return int(load().rsign_dbg_set_copy_streams(int(n)))


def dbg_set_host_mapped(on):
    """Host buffers read/written in place by the kernels (1) or staged through copies (0); returns the
    previous setting."""
    return int(load().rsign_dbg_set_host_mapped(int(on)))


def dbg_set_tangent_cut(on):
    """Leave out tangent steps at converged stored iterates (1) or run them all (0); returns the previous setting."""
    return int(load().rsign_dbg_set_tangent_cut(int(on)))


def dbg_set_split_steps(n):
    """REFINE stage 1: iterates X_0..X_{n-1} as hi/lo pairs, later ones single planes (-2: by rule,
    -1: all pairs); returns the previous setting."""
    return int(load().rsign_dbg_set_split_steps(int(n)))


def dbg_set_digit_fp8(on):
    """Digit planes of the FP64-grade products as FP8 E4M3 (1) or FP16 (0); returns the previous setting."""
    return int(load().rsign_dbg_set_digit_fp8(int(on)))


def dbg_set_refine_levels(polish=-1, ra_first=-1, ra_later=-1):
    """Set the digit levels of the refinement's FP64-grade products (0 = by the tolerance,
    -1 keeps a setting); returns the previous settings as 100 p + 10 f + l."""
    return int(load().rsign_dbg_set_refine_levels(int(polish), int(ra_first), int(ra_later)))


def dbg_set_ozaki_tile(bn):
    """Tile width (128, 256, or 0 = by order) of the refinement's FP64-grade products; returns the
    previous setting."""
    return int(load().rsign_dbg_set_ozaki_tile(int(bn)))


def dbg_bounded_wait(arrive, limit_ns, status, stream=None):
    """One bounded mbarrier wait (limit in ns); without the arrival it gives up and sets
    *status (a device int32 tensor) to ERR_TIMEOUT.  Returns the call's status."""
    lib = load()
    return Status(lib.rsign_dbg_bounded_wait(int(arrive), int(limit_ns), status.data_ptr(), _stream_ptr(stream, True)))


def dbg_oz_convert(v, e, stream=None):
    """(a, b): the digit-plane epilogue's int64 -> FP64 conversion v 2^e done two ways on the device
    (correctly rounded conversion plus exponent shift; 128-bit integer rounding).  v int64, e int32 (CUDA)."""
    torch = _torch()
    lib = load()
    n = int(v.numel())
    a = torch.empty(n, dtype=torch.float64, device=v.device)
    b = torch.empty(n, dtype=torch.float64, device=v.device)
    st = Status(lib.rsign_dbg_oz_convert(v.data_ptr(), e.data_ptr(), n, a.data_ptr(), b.data_ptr(),
                                         _stream_ptr(stream, True)))
    if st != Status.OK:
        raise RsignError(st)
    return a, b


def dbg_sym_gemv_tiles(dp):
    """(I, J) arrays: the upper-triangle tile handled by each block of the check's symmetric GEMV (host only)."""
    lib = load()
    n = lib.rsign_dbg_sym_gemv_tiles(int(dp), None, None)
    if n < 0:
        raise RsignError(Status.ERR_ARG)
    I = (ctypes.c_int32 * n)()
    J = (ctypes.c_int32 * n)()
    m = lib.rsign_dbg_sym_gemv_tiles(int(dp), I, J)
    return np.array(I[:m]), np.array(J[:m])


def dbg_tile_order(dp, sym=0):
    """(bm, bn) arrays of the persistent GEMM's tile visiting order (host only)."""
    lib = load()
    n = lib.rsign_dbg_tile_order(int(dp), int(sym), None, None)
    if n < 0:
        raise RsignError(Status.ERR_ARG)
    bm = (ctypes.c_int32 * n)()
    bn = (ctypes.c_int32 * n)()
    m = lib.rsign_dbg_tile_order(int(dp), int(sym), bm, bn)
    return np.array(bm[:m]), np.array(bn[:m])


def dbg_fp64e_gemm(A, B, d_real=None, sym=0, out=None, stream=None):
    """out = A B with FP64-emulating digit planes (>= 54 bits) on the FP16 tensor cores."""
    torch = _torch()
    lib = load()
    dp = int(A.shape[0])
    if out is None:
        out = torch.empty((dp, dp), dtype=torch.float64, device=A.device)
    st = Status(lib.rsign_dbg_fp64e_gemm(A.data_ptr(), B.data_ptr(), dp, int(d_real or dp), int(sym),
                                         out.data_ptr(), _stream_ptr(stream, True)))
    if st != Status.OK:
        raise RsignError(st)
    return out


def dbg_spectral_norm(M, iters, per_step=False, stream=None):
    """Power-step estimate of ||M||_2 (M symmetric CUDA float64), as the alpha rule computes it."""
    lib = load()
    out = ctypes.c_double(0.0)
    st = Status(lib.rsign_dbg_spectral_norm(M.data_ptr(), int(M.shape[0]), int(iters), int(bool(per_step)),
                                            ctypes.byref(out), _stream_ptr(stream, True)))
    if st != Status.OK:
        raise RsignError(st)
    return out.value


def dbg_gemv_df_sym(M, x, stream=None):
    """y = M x for a symmetric device FP64 M read from its upper triangle (double-float arithmetic)."""
    torch = _torch()
    lib = load()
    dp = int(M.shape[0])
    y = torch.empty(dp, dtype=torch.float64, device=M.device)
    st = Status(lib.rsign_dbg_gemv_df_sym(M.data_ptr(), x.data_ptr(), dp, y.data_ptr(), _stream_ptr(stream, True)))
    if st != Status.OK:
        raise RsignError(st)
    return y


def dbg_gemv_df(M, x, stream=None):
    """y = M x (device FP64) in the double-float arithmetic of the refinement check."""
    torch = _torch()
    lib = load()
    dp = int(M.shape[0])
    y = torch.empty(dp, dtype=torch.float64, device=M.device)
    st = Status(lib.rsign_dbg_gemv_df(M.data_ptr(), x.data_ptr(), dp, y.data_ptr(), _stream_ptr(stream, True)))
    if st != Status.OK:
        raise RsignError(st)
    return y


def dbg_commutator_check(A, R, d=None, iters=12, stream=None):
    """The refinement's matrix-free check on device A, R: returns (||G||_2 est,
    ||R^2 - I||_2 est, (a11, a12, a22) of the 2 x 2 Rayleigh-Ritz projection)."""
    lib = load()
    dp = int(A.shape[0])
    out = (ctypes.c_double * 5)()
    st = Status(lib.rsign_dbg_commutator_check(A.data_ptr(), R.data_ptr(), dp, int(d or dp), int(iters), out,
                                               _stream_ptr(stream, True)))
    if st != Status.OK:
        raise RsignError(st)
    return out[0], out[1], (out[2], out[3], out[4])


def build(force=False, verbose=False):
    """Compile librsign.so (sm_103a) in-tree."""
    from . import buildlib
    return buildlib.build(force=force, verbose=verbose)
