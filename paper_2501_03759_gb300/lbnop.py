"""ctypes binding of the learned leap (the C-ABI declared in include/lbnop.h), in the same
library as lbch. Functions keep the C names and only marshal arguments; device tensors
and streams come from PyTorch. Every computation runs in the library's CUDA kernels."""
from __future__ import annotations

import ctypes
import threading

import numpy as np

from . import lbch as _lbch

MAX_BATCH = 64


class lbnop_params(ctypes.Structure):
    _fields_ = [("H", ctypes.c_int32), ("W", ctypes.c_int32), ("max_batch", ctypes.c_int32),
                ("scale", ctypes.c_double)]


class lbnop_judge(ctypes.Structure):
    _fields_ = [("leap_steps", ctypes.c_int64), ("energy_rtol", ctypes.c_double), ("mass_atol", ctypes.c_double),
                ("audit_every", ctypes.c_int64), ("phi_rtol", ctypes.c_double)]


class lbnop_judge_stats(ctypes.Structure):
    _fields_ = [("accepted", ctypes.c_int64), ("rejected", ctypes.c_int64),
                ("rejected_nonfinite", ctypes.c_int64), ("rejected_mass", ctypes.c_int64),
                ("rejected_energy", ctypes.c_int64), ("rejected_audit", ctypes.c_int64),
                ("audits", ctypes.c_int64), ("lbm_steps", ctypes.c_int64),
                ("max_audit_err", ctypes.c_double), ("max_leap_rise", ctypes.c_double),
                ("max_corr_rise", ctypes.c_double)]


def make_judge(leap_steps: int = 500, energy_rtol: float = 1e-4, mass_atol: float = 1e-6, audit_every: int = 0,
               phi_rtol: float = 1e-2) -> lbnop_judge:
    j = lbnop_judge()
    j.leap_steps, j.energy_rtol, j.mass_atol = int(leap_steps), float(energy_rtol), float(mass_atol)
    j.audit_every, j.phi_rtol = int(audit_every), float(phi_rtol)
    return j


def make_params(H: int, W: int, max_batch: int = 1, scale: float = 0.05) -> lbnop_params:
    p = lbnop_params()
    p.H, p.W, p.max_batch, p.scale = int(H), int(W), int(max_batch), float(scale)
    return p


_lock = threading.Lock()
_ready = False


def load():
    """The loaded library with the lbnop signatures registered."""
    global _ready
    lib = _lbch.load()
    with _lock:
        if _ready:
            return lib
        vp, dp, fp = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_float)
        P = ctypes.POINTER(lbnop_params)
        i32 = ctypes.c_int32
        lib.lbnop_param_count.argtypes = []
        lib.lbnop_param_count.restype = ctypes.c_int64
        lib.lbnop_workspace_bytes.argtypes = [P]
        lib.lbnop_workspace_bytes.restype = ctypes.c_size_t
        lib.lbnop_create.argtypes = [P, vp, ctypes.c_size_t, vp, ctypes.POINTER(vp)]
        lib.lbnop_create.restype = ctypes.c_int
        for name in ("lbnop_set_params", "lbnop_get_params", "lbnop_get_grads"):
            getattr(lib, name).argtypes = [vp, fp]
            getattr(lib, name).restype = ctypes.c_int
        lib.lbnop_forward.argtypes = [vp, vp, dp, i32, vp]
        lib.lbnop_forward.restype = ctypes.c_int
        lib.lbnop_backward.argtypes = [vp, vp, dp, vp, dp, i32, dp]
        lib.lbnop_backward.restype = ctypes.c_int
        lib.lbnop_adam.argtypes = [vp, ctypes.c_double]
        lib.lbnop_adam.restype = ctypes.c_int
        lib.lbnop_set_leap_turns.argtypes = [vp, i32]
        lib.lbnop_set_leap_turns.restype = ctypes.c_int
        lib.lbnop_set_clip.argtypes = [vp, ctypes.c_double]
        lib.lbnop_set_clip.restype = ctypes.c_int
        lib.lbnop_grad_norm.argtypes = [vp, dp]
        lib.lbnop_grad_norm.restype = ctypes.c_int
        lib.lbnop_train_step.argtypes = [vp, vp, dp, vp, dp, i32, ctypes.c_double, dp]
        lib.lbnop_train_step.restype = ctypes.c_int
        lib.lbnop_leap_run.argtypes = [vp, vp, ctypes.c_double, ctypes.c_int64, ctypes.c_int64]
        lib.lbnop_leap_run.restype = ctypes.c_int
        lib.lbnop_leap_run_judged.argtypes = [vp, vp, ctypes.c_double, ctypes.c_int64, ctypes.c_int64,
                                              ctypes.POINTER(lbnop_judge), ctypes.POINTER(lbnop_judge_stats)]
        lib.lbnop_leap_run_judged.restype = ctypes.c_int
        for name in ("lbnop_conv3x3_bwd_data", "lbnop_conv3x3_bwd_weight"):
            getattr(lib, name).argtypes = [vp, vp, i32, i32, i32, i32, i32, vp, vp]
            getattr(lib, name).restype = ctypes.c_int
        lib.lbnop_conv3x3.argtypes = [vp, vp, vp, i32, i32, i32, i32, i32, vp, vp]
        lib.lbnop_conv3x3.restype = ctypes.c_int
        lib.lbnop_conv3x3_packed_bytes.argtypes = [i32, i32]
        lib.lbnop_conv3x3_packed_bytes.restype = ctypes.c_size_t
        lib.lbnop_conv3x3_pack.argtypes = [vp, i32, i32, vp, vp]
        lib.lbnop_conv3x3_pack.restype = ctypes.c_int
        lib.lbnop_conv3x3_packed.argtypes = [vp, vp, vp, vp, i32, i32, i32, i32, i32, vp, vp]
        lib.lbnop_conv3x3_packed.restype = ctypes.c_int
        lib.lbnop_tc_launches.argtypes = []
        lib.lbnop_tc_launches.restype = ctypes.c_int64
        lib.lbnop_tc_fault.argtypes = []
        lib.lbnop_tc_fault.restype = ctypes.c_int32
        lib.lbnop_last_error.argtypes = [vp]
        lib.lbnop_last_error.restype = ctypes.c_char_p
        lib.lbnop_destroy.argtypes = [vp]
        lib.lbnop_destroy.restype = None
        _ready = True
        return lib


def _check(ctx, status: int, what: str):
    if status != _lbch.OK:
        detail = (load().lbnop_last_error(ctx) or b"").decode(errors="replace") if ctx else ""
        raise _lbch.LbchError(status, what, detail)


def _alpha(alpha) -> ctypes.Array:
    a = np.ascontiguousarray(np.atleast_1d(np.asarray(alpha, dtype=np.float64)))
    return (ctypes.c_double * a.size)(*a.tolist())


def _f32_host(a, n: int, what: str) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.float32)
    if a.size != n:
        raise ValueError(f"{what}: expected {n} values, got {a.size}")
    return a


# ---------------------------------------------------------------- C-ABI, same names

def lbnop_param_count() -> int:
    return int(load().lbnop_param_count())


def lbnop_workspace_bytes(p: lbnop_params) -> int:
    return int(load().lbnop_workspace_bytes(ctypes.byref(p)))


def lbnop_create(p: lbnop_params, d_workspace: int, nbytes: int, cuda_stream):
    ctx = ctypes.c_void_p()
    st = load().lbnop_create(ctypes.byref(p), ctypes.c_void_p(int(d_workspace)), int(nbytes),
                             ctypes.c_void_p(int(cuda_stream or 0)), ctypes.byref(ctx))
    _check(None, st, "lbnop_create")
    return ctx


def lbnop_set_params(ctx, theta) -> None:
    a = _f32_host(theta, lbnop_param_count(), "theta")
    _check(ctx, load().lbnop_set_params(ctx, a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))), "lbnop_set_params")


def lbnop_get_params(ctx) -> np.ndarray:
    out = np.empty(lbnop_param_count(), dtype=np.float32)
    _check(ctx, load().lbnop_get_params(ctx, out.ctypes.data_as(ctypes.POINTER(ctypes.c_float))), "lbnop_get_params")
    return out


def lbnop_get_grads(ctx) -> np.ndarray:
    out = np.empty(lbnop_param_count(), dtype=np.float32)
    _check(ctx, load().lbnop_get_grads(ctx, out.ctypes.data_as(ctypes.POINTER(ctypes.c_float))), "lbnop_get_grads")
    return out


def lbnop_forward(ctx, d_phi: int, alpha, batch: int, d_phi_out: int) -> None:
    _check(ctx, load().lbnop_forward(ctx, ctypes.c_void_p(int(d_phi)), _alpha(alpha), int(batch),
                                     ctypes.c_void_p(int(d_phi_out))), "lbnop_forward")


def lbnop_backward(ctx, d_phi: int, alpha, d_target: int, batch: int, want_loss: bool = True, weight=None):
    loss = ctypes.c_double(float("nan"))
    _check(ctx, load().lbnop_backward(ctx, ctypes.c_void_p(int(d_phi)), _alpha(alpha), ctypes.c_void_p(int(d_target)),
                                      None if weight is None else _alpha(weight), int(batch),
                                      ctypes.byref(loss) if want_loss else None), "lbnop_backward")
    return loss.value if want_loss else None


def lbnop_adam(ctx, lr: float) -> None:
    _check(ctx, load().lbnop_adam(ctx, float(lr)), "lbnop_adam")


def lbnop_set_clip(ctx, max_norm: float) -> None:
    _check(ctx, load().lbnop_set_clip(ctx, float(max_norm)), "lbnop_set_clip")


def lbnop_set_leap_turns(ctx, turns: int) -> None:
    _check(ctx, load().lbnop_set_leap_turns(ctx, int(turns)), "lbnop_set_leap_turns")


def lbnop_grad_norm(ctx) -> float:
    out = ctypes.c_double(float("nan"))
    _check(ctx, load().lbnop_grad_norm(ctx, ctypes.byref(out)), "lbnop_grad_norm")
    return out.value


def lbnop_train_step(ctx, d_phi: int, alpha, d_target: int, batch: int, lr: float, want_loss: bool = False,
                     weight=None):
    loss = ctypes.c_double(float("nan"))
    _check(ctx, load().lbnop_train_step(ctx, ctypes.c_void_p(int(d_phi)), _alpha(alpha),
                                        ctypes.c_void_p(int(d_target)), None if weight is None else _alpha(weight),
                                        int(batch), float(lr), ctypes.byref(loss) if want_loss else None),
           "lbnop_train_step")
    return loss.value if want_loss else None


def lbnop_leap_run(ctx, lbm_ctx, alpha: float, cycles: int, lbm_steps: int) -> None:
    _check(ctx, load().lbnop_leap_run(ctx, lbm_ctx, float(alpha), int(cycles), int(lbm_steps)), "lbnop_leap_run")


def lbnop_leap_run_judged(ctx, lbm_ctx, alpha: float, cycles: int, lbm_steps: int, judge: lbnop_judge) -> dict:
    """Runs the judged leap cycles; returns the judge's counts as a dict."""
    st = lbnop_judge_stats()
    _check(ctx, load().lbnop_leap_run_judged(ctx, lbm_ctx, float(alpha), int(cycles), int(lbm_steps),
                                             ctypes.byref(judge), ctypes.byref(st)), "lbnop_leap_run_judged")
    return {name: getattr(st, name) for name, _ in lbnop_judge_stats._fields_}


def lbnop_conv3x3(d_x: int, d_w: int, d_bias: int | None, B: int, H: int, W: int, c_in: int, c_out: int,
                  d_y: int, cuda_stream) -> None:
    st = load().lbnop_conv3x3(ctypes.c_void_p(int(d_x)), ctypes.c_void_p(int(d_w)),
                              ctypes.c_void_p(int(d_bias)) if d_bias else None, B, H, W, c_in, c_out,
                              ctypes.c_void_p(int(d_y)), ctypes.c_void_p(int(cuda_stream or 0)))
    _check(None, st, "lbnop_conv3x3")


def lbnop_conv3x3_packed_bytes(c_in: int, c_out: int) -> int:
    """Bytes of a layer's weights packed for the tensor-core path (0: unsupported widths)."""
    return int(load().lbnop_conv3x3_packed_bytes(c_in, c_out))


def lbnop_conv3x3_pack(d_w: int, c_in: int, c_out: int, d_packed: int, cuda_stream) -> None:
    st = load().lbnop_conv3x3_pack(ctypes.c_void_p(int(d_w)), c_in, c_out, ctypes.c_void_p(int(d_packed)),
                                   ctypes.c_void_p(int(cuda_stream or 0)))
    _check(None, st, "lbnop_conv3x3_pack")


def lbnop_conv3x3_packed(d_x: int, d_w: int, d_packed: int | None, d_bias: int | None, B: int, H: int, W: int,
                         c_in: int, c_out: int, d_y: int, cuda_stream) -> None:
    st = load().lbnop_conv3x3_packed(ctypes.c_void_p(int(d_x)), ctypes.c_void_p(int(d_w)),
                                     ctypes.c_void_p(int(d_packed)) if d_packed else None,
                                     ctypes.c_void_p(int(d_bias)) if d_bias else None, B, H, W, c_in, c_out,
                                     ctypes.c_void_p(int(d_y)), ctypes.c_void_p(int(cuda_stream or 0)))
    _check(None, st, "lbnop_conv3x3_packed")


def lbnop_conv3x3_bwd_data(d_dy: int, d_w: int, B: int, H: int, W: int, c_in: int, c_out: int, d_dx: int,
                           cuda_stream) -> None:
    st = load().lbnop_conv3x3_bwd_data(ctypes.c_void_p(int(d_dy)), ctypes.c_void_p(int(d_w)), B, H, W, c_in, c_out,
                                       ctypes.c_void_p(int(d_dx)), ctypes.c_void_p(int(cuda_stream or 0)))
    _check(None, st, "lbnop_conv3x3_bwd_data")


def lbnop_conv3x3_bwd_weight(d_x: int, d_dy: int, B: int, H: int, W: int, c_in: int, c_out: int, d_dw: int,
                             cuda_stream) -> None:
    st = load().lbnop_conv3x3_bwd_weight(ctypes.c_void_p(int(d_x)), ctypes.c_void_p(int(d_dy)), B, H, W, c_in,
                                         c_out, ctypes.c_void_p(int(d_dw)), ctypes.c_void_p(int(cuda_stream or 0)))
    _check(None, st, "lbnop_conv3x3_bwd_weight")


def lbnop_tc_fault() -> int:
    """1 if a tcgen05 convolution of this process gave up a bounded wait (its outputs are
    invalid), 0 if none did, -1 if unreadable. Read after synchronising."""
    return int(load().lbnop_tc_fault())


def lbnop_tc_launches() -> int:
    """Convolutions run on the tcgen05 tensor-core path so far in this process."""
    return int(load().lbnop_tc_launches())


def lbnop_last_error(ctx) -> str:
    return (load().lbnop_last_error(ctx) or b"").decode(errors="replace")


def lbnop_destroy(ctx) -> None:
    load().lbnop_destroy(ctx)


# ---------------------------------------------------------------- convenience owner

class Surrogate:
    """Owns an lbnop context and its device workspace on one stream. Fields are float32
    CUDA tensors of shape (batch, H, W); alpha is one anisotropy strength per field."""

    def __init__(self, H: int, W: int, max_batch: int = 1, scale: float = 0.05, device=None, stream=None):
        import torch

        self.params = make_params(H, W, max_batch, scale)
        self.H, self.W, self.max_batch = int(H), int(W), int(max_batch)
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        nbytes = lbnop_workspace_bytes(self.params)
        if nbytes == 0:
            raise _lbch.LbchError(_lbch.EINVAL, "lbnop_workspace_bytes", "invalid parameters")
        with torch.cuda.device(self.device):
            self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
            self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
            self.ctx = lbnop_create(self.params, self.workspace.data_ptr(), nbytes, self.stream.cuda_stream)

    def _on(self):
        import torch
        return torch.cuda.device(self.device)

    def _fields(self, t, what):
        import torch
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
            raise ValueError(f"{what}: expected a contiguous float32 CUDA tensor")
        if t.numel() % (self.H * self.W):
            raise ValueError(f"{what}: size is not a multiple of H*W")
        return t.numel() // (self.H * self.W)

    def set_params(self, theta) -> None:
        with self._on():
            lbnop_set_params(self.ctx, theta)

    def params_host(self) -> np.ndarray:
        with self._on():
            return lbnop_get_params(self.ctx)

    def grads_host(self) -> np.ndarray:
        with self._on():
            return lbnop_get_grads(self.ctx)

    def forward(self, phi, alpha, out=None):
        import torch
        b = self._fields(phi, "phi")
        if out is None:
            out = torch.empty_like(phi)
        with self._on():
            lbnop_forward(self.ctx, phi.data_ptr(), alpha, b, out.data_ptr())
        return out

    def backward(self, phi, alpha, target, weight=None) -> float:
        b = self._fields(phi, "phi")
        with self._on():
            return lbnop_backward(self.ctx, phi.data_ptr(), alpha, target.data_ptr(), b, weight=weight)

    def adam(self, lr: float) -> None:
        with self._on():
            lbnop_adam(self.ctx, lr)

    def set_clip(self, max_norm: float) -> None:
        """Global-norm gradient clipping for the following Adam steps (0: off)."""
        lbnop_set_clip(self.ctx, max_norm)

    def set_leap_turns(self, turns: int) -> None:
        """Leaps average the network over 1 or 4 quarter turns of the field (lbnop_set_leap_turns)."""
        lbnop_set_leap_turns(self.ctx, turns)

    def grad_norm(self) -> float:
        """L2 norm of the last backward's gradient, before clipping (synchronises)."""
        with self._on():
            return lbnop_grad_norm(self.ctx)

    def train_step(self, phi, alpha, target, lr: float, want_loss: bool = False, weight=None):
        b = self._fields(phi, "phi")
        with self._on():
            return lbnop_train_step(self.ctx, phi.data_ptr(), alpha, target.data_ptr(), b, lr, want_loss, weight)

    def leap_run(self, solver, alpha: float, cycles: int, lbm_steps: int) -> None:
        """Alternates leaps with lbm_steps steps of an lbch Solver (same stream, nx = W, ny = H)."""
        if solver.nx != self.W or solver.ny != self.H:
            raise ValueError("solver grid must match the surrogate's H x W")
        if solver.stream.cuda_stream != self.stream.cuda_stream:
            raise ValueError("solver and surrogate must share a CUDA stream")
        with self._on():
            lbnop_leap_run(self.ctx, solver.ctx, alpha, cycles, lbm_steps)

    def leap_run_judged(self, solver, alpha: float, cycles: int, lbm_steps: int, judge=None) -> dict:
        """leap_run with the plain scheme as judge and fallback (lbnop_leap_run_judged); returns
        the judge's counts. judge: an lbnop_judge (default make_judge())."""
        if solver.nx != self.W or solver.ny != self.H:
            raise ValueError("solver grid must match the surrogate's H x W")
        if solver.stream.cuda_stream != self.stream.cuda_stream:
            raise ValueError("solver and surrogate must share a CUDA stream")
        with self._on():
            return lbnop_leap_run_judged(self.ctx, solver.ctx, alpha, cycles, lbm_steps,
                                         make_judge() if judge is None else judge)

    def close(self) -> None:
        if getattr(self, "ctx", None):
            lbnop_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
