"""ctypes binding of liblbch.so (the C-ABI declared in include/lbch.h).

The functions keep the C names and only marshal arguments: host arrays become
pointers, device memory and the stream come from PyTorch. Every computation runs
in the library's CUDA kernels; there is no Python or CPU fallback. A missing
library raises ``LbchUnavailable``.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

STORE_F32, STORE_BF16_DEV, STORE_F16_DEV = 0, 1, 2
Q_LITERAL, MU_NESTED, S35_EXPLICIT = 1, 2, 4
REG_NONE, REG_WILLMORE, REG_LINEAR = 0, 1, 2

OK, EINVAL, ECUDA, ENOMEM, ENONFINITE, ESTATE = 0, -1, -2, -3, -4, -5
_STATUS = {OK: "LBCH_OK", EINVAL: "LBCH_EINVAL", ECUDA: "LBCH_ECUDA", ENOMEM: "LBCH_ENOMEM",
           ENONFINITE: "LBCH_ENONFINITE", ESTATE: "LBCH_ESTATE"}

# Bytes moved per node update by one step, by storage (9 populations read and written).
ALGORITHMIC_BYTES_PER_LU = {STORE_F32: 72, STORE_BF16_DEV: 48, STORE_F16_DEV: 48}


class LbchUnavailable(RuntimeError):
    """The CUDA library is not built or cannot be loaded."""


class LbchError(RuntimeError):
    def __init__(self, status: int, what: str, detail: str = ""):
        self.status = status
        super().__init__(f"{what}: {_STATUS.get(status, status)}" + (f" ({detail})" if detail else ""))


class lbch_params(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
        ("M", ctypes.c_double), ("sigma", ctypes.c_double), ("D", ctypes.c_double),
        ("eps", ctypes.c_double), ("alpha", ctypes.c_double),
        ("s", ctypes.c_double * 9),
        ("storage", ctypes.c_int32), ("regularization", ctypes.c_int32), ("flags", ctypes.c_uint32),
    ]


class lbch3_params(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
        ("M", ctypes.c_double), ("sigma", ctypes.c_double), ("D", ctypes.c_double),
        ("eps", ctypes.c_double), ("alpha", ctypes.c_double),
        ("s", ctypes.c_double * 15),
        ("regularization", ctypes.c_int32), ("flags", ctypes.c_uint32),
    ]


def make_params3(nx: int, ny: int, nz: int, *, M=0.1, sigma=0.01, D=5.0, eps=0.03, alpha=0.0, s=None,
                 regularization=REG_WILLMORE, flags=0) -> lbch3_params:
    """lbch3_params (D3Q15) with the defaults of Eq. 39 and Willmore G."""
    p = lbch3_params()
    p.nx, p.ny, p.nz = int(nx), int(ny), int(nz)
    p.M, p.sigma, p.D, p.eps, p.alpha = float(M), float(sigma), float(D), float(eps), float(alpha)
    rates = [1.0] * 15 if s is None else list(s)
    for i in range(15):
        p.s[i] = float(rates[i])
    p.regularization, p.flags = int(regularization), int(flags)
    return p


def make_params(nx: int, ny: int, *, M=0.1, sigma=0.01, D=5.0, eps=0.03, alpha=0.0, s=None,
                storage=STORE_F32, regularization=REG_WILLMORE, flags=0) -> lbch_params:
    """lbch_params with the defaults of Eq. 39 (M, eps, D, sigma) and Willmore G."""
    p = lbch_params()
    p.nx, p.ny = int(nx), int(ny)
    p.M, p.sigma, p.D, p.eps, p.alpha = float(M), float(sigma), float(D), float(eps), float(alpha)
    rates = [1.0] * 9 if s is None else list(s)
    for i in range(9):
        p.s[i] = float(rates[i])
    p.storage, p.regularization, p.flags = int(storage), int(regularization), int(flags)
    return p


_lock = threading.Lock()
_lib = None


def library_path() -> str:
    return _build.LIB


def load():
    """Loads liblbch.so (raises LbchUnavailable if it is not built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if not os.path.exists(path):
            raise LbchUnavailable(
                f"{path} is not built; run paper_2501_03759_gb300.build.build() (nvcc, sm_103a)")
        try:
            lib = ctypes.CDLL(path)
        except OSError as e:
            raise LbchUnavailable(f"cannot load {path}: {e}") from e
        P = ctypes.POINTER(lbch_params)
        dp = ctypes.POINTER(ctypes.c_double)
        vp = ctypes.c_void_p
        lib.lbch_workspace_bytes.argtypes = [P]
        lib.lbch_workspace_bytes.restype = ctypes.c_size_t
        lib.lbch_create.argtypes = [P, vp, ctypes.c_size_t, vp, ctypes.POINTER(vp)]
        lib.lbch_create.restype = ctypes.c_int
        for name in ("lbch_init_field", "lbch_set_state"):
            getattr(lib, name).argtypes = [vp, dp]
            getattr(lib, name).restype = ctypes.c_int
        for name in ("lbch_mass", "lbch_free_energy", "lbch_get_field", "lbch_get_state"):
            getattr(lib, name).argtypes = [vp, dp]
            getattr(lib, name).restype = ctypes.c_int
        lib.lbch_step.argtypes = [vp, ctypes.c_int64]
        lib.lbch_step.restype = ctypes.c_int
        for name in ("lbch_init_field_device", "lbch_get_phi_device"):
            getattr(lib, name).argtypes = [vp, vp]
            getattr(lib, name).restype = ctypes.c_int
        lib.lbch_batch_get_phi_device.argtypes = [vp, ctypes.c_int32, vp]
        lib.lbch_batch_get_phi_device.restype = ctypes.c_int
        lib.lbch_steps_taken.argtypes = [vp]
        lib.lbch_steps_taken.restype = ctypes.c_int64
        lib.lbch_set_steps_taken.argtypes = [vp, ctypes.c_int64]
        lib.lbch_set_steps_taken.restype = ctypes.c_int
        for name in ("lbch_mass_device", "lbch_free_energy_device"):
            getattr(lib, name).argtypes = [vp, vp]
            getattr(lib, name).restype = ctypes.c_int
        lib.lbch_field_diagnostics_device.argtypes = [vp, vp, vp]
        lib.lbch_field_diagnostics_device.restype = ctypes.c_int
        lib.lbch_state_bytes.argtypes = [P]
        lib.lbch_state_bytes.restype = ctypes.c_size_t
        for name in ("lbch_save_state_device", "lbch_restore_state_device"):
            getattr(lib, name).argtypes = [vp, vp, ctypes.c_size_t]
            getattr(lib, name).restype = ctypes.c_int
        lib.lbch_last_error.argtypes = [vp]
        lib.lbch_last_error.restype = ctypes.c_char_p
        lib.lbch_destroy.argtypes = [vp]
        lib.lbch_destroy.restype = None
        lib.lbch_free_energy_static.argtypes = [P, vp, ctypes.c_int64, vp, vp]
        lib.lbch_free_energy_static.restype = ctypes.c_int
        ip = ctypes.POINTER(ctypes.c_int32)
        lib.lbch_batch_workspace_bytes.argtypes = [P, ctypes.c_int32, ip, ip]
        lib.lbch_batch_workspace_bytes.restype = ctypes.c_size_t
        lib.lbch_batch_create.argtypes = [P, ctypes.c_int32, ip, ip, dp, vp, ctypes.c_size_t, vp,
                                          ctypes.POINTER(vp)]
        lib.lbch_batch_create.restype = ctypes.c_int
        lib.lbch_batch_init_field.argtypes = [vp, ctypes.c_int32, dp]
        lib.lbch_batch_init_field.restype = ctypes.c_int
        lib.lbch_batch_step.argtypes = [vp, ctypes.c_int64]
        lib.lbch_batch_step.restype = ctypes.c_int
        for name in ("lbch_batch_get_field", "lbch_batch_mass", "lbch_batch_free_energy"):
            getattr(lib, name).argtypes = [vp, ctypes.c_int32, dp]
            getattr(lib, name).restype = ctypes.c_int
        lib.lbch_batch_rows_target.argtypes = [vp]
        lib.lbch_batch_rows_target.restype = ctypes.c_int32
        lib.lbch_batch_steps_taken.argtypes = [vp]
        lib.lbch_batch_steps_taken.restype = ctypes.c_int64
        lib.lbch_batch_last_error.argtypes = [vp]
        lib.lbch_batch_last_error.restype = ctypes.c_char_p
        lib.lbch_batch_destroy.argtypes = [vp]
        lib.lbch_batch_destroy.restype = None
        P3 = ctypes.POINTER(lbch3_params)
        lib.lbch3_workspace_bytes.argtypes = [P3]
        lib.lbch3_workspace_bytes.restype = ctypes.c_size_t
        lib.lbch3_create.argtypes = [P3, vp, ctypes.c_size_t, vp, ctypes.POINTER(vp)]
        lib.lbch3_create.restype = ctypes.c_int
        for name in ("lbch3_init_field", "lbch3_get_field", "lbch3_mass", "lbch3_free_energy"):
            getattr(lib, name).argtypes = [vp, dp]
            getattr(lib, name).restype = ctypes.c_int
        lib.lbch3_step.argtypes = [vp, ctypes.c_int64]
        lib.lbch3_step.restype = ctypes.c_int
        lib.lbch3_last_error.argtypes = [vp]
        lib.lbch3_last_error.restype = ctypes.c_char_p
        lib.lbch3_destroy.argtypes = [vp]
        lib.lbch3_destroy.restype = None
        _lib = lib
        return lib


def _check(ctx, status: int, what: str):
    if status != OK:
        detail = ""
        if ctx:
            detail = (load().lbch_last_error(ctx) or b"").decode(errors="replace")
        raise LbchError(status, what, detail)


def _host_ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _as_host_f64(a, n: int, what: str) -> np.ndarray:
    if hasattr(a, "detach"):  # torch tensor (possibly pinned): use its memory directly
        assert a.device.type == "cpu" and a.dtype.is_floating_point, what
        a = a.detach().numpy()
    a = np.ascontiguousarray(a, dtype=np.float64)
    if a.size != n:
        raise ValueError(f"{what}: expected {n} values, got {a.size}")
    return a


def _check_device_f32(t, n: int, what: str) -> None:
    import torch

    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
        raise ValueError(f"{what}: expected a contiguous float32 CUDA tensor")
    if t.numel() != n:
        raise ValueError(f"{what}: expected {n} values, got {t.numel()}")


def _check_device_f64(t, what: str) -> None:
    import torch

    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.numel() >= 1):
        raise ValueError(f"{what}: expected a float64 CUDA tensor")


# ---------------------------------------------------------------- C-ABI, same names

def lbch_workspace_bytes(p: lbch_params) -> int:
    return int(load().lbch_workspace_bytes(ctypes.byref(p)))


def lbch_create(p: lbch_params, d_workspace: int, nbytes: int, cuda_stream: int | None):
    ctx = ctypes.c_void_p()
    st = load().lbch_create(ctypes.byref(p), ctypes.c_void_p(int(d_workspace)), int(nbytes),
                            ctypes.c_void_p(int(cuda_stream or 0)), ctypes.byref(ctx))
    _check(None, st, "lbch_create")
    return ctx


def lbch_init_field(ctx, phi0) -> None:
    _check(ctx, load().lbch_init_field(ctx, _host_ptr(phi0)), "lbch_init_field")


def lbch_init_field_device(ctx, d_phi0: int) -> None:
    _check(ctx, load().lbch_init_field_device(ctx, ctypes.c_void_p(int(d_phi0))), "lbch_init_field_device")


def lbch_get_phi_device(ctx, d_phi: int) -> None:
    _check(ctx, load().lbch_get_phi_device(ctx, ctypes.c_void_p(int(d_phi))), "lbch_get_phi_device")


def lbch_step(ctx, n: int) -> None:
    _check(ctx, load().lbch_step(ctx, int(n)), "lbch_step")


def lbch_mass(ctx) -> float:
    v = ctypes.c_double()
    _check(ctx, load().lbch_mass(ctx, ctypes.byref(v)), "lbch_mass")
    return v.value


def lbch_free_energy(ctx) -> float:
    v = ctypes.c_double()
    _check(ctx, load().lbch_free_energy(ctx, ctypes.byref(v)), "lbch_free_energy")
    return v.value


def lbch_get_field(ctx, out: np.ndarray) -> np.ndarray:
    _check(ctx, load().lbch_get_field(ctx, _host_ptr(out)), "lbch_get_field")
    return out


def lbch_get_state(ctx, out: np.ndarray) -> np.ndarray:
    _check(ctx, load().lbch_get_state(ctx, _host_ptr(out)), "lbch_get_state")
    return out


def lbch_set_state(ctx, f9: np.ndarray) -> None:
    _check(ctx, load().lbch_set_state(ctx, _host_ptr(f9)), "lbch_set_state")


def lbch_steps_taken(ctx) -> int:
    return int(load().lbch_steps_taken(ctx))


def lbch_set_steps_taken(ctx, steps: int) -> None:
    _check(ctx, load().lbch_set_steps_taken(ctx, int(steps)), "lbch_set_steps_taken")


def lbch_mass_device(ctx, d_out: int) -> None:
    _check(ctx, load().lbch_mass_device(ctx, ctypes.c_void_p(int(d_out))), "lbch_mass_device")


def lbch_free_energy_device(ctx, d_out: int) -> None:
    _check(ctx, load().lbch_free_energy_device(ctx, ctypes.c_void_p(int(d_out))), "lbch_free_energy_device")


def lbch_field_diagnostics_device(ctx, d_phi: int, d_out2: int) -> None:
    _check(ctx, load().lbch_field_diagnostics_device(ctx, ctypes.c_void_p(int(d_phi)), ctypes.c_void_p(int(d_out2))),
           "lbch_field_diagnostics_device")


def lbch_state_bytes(p: lbch_params) -> int:
    return int(load().lbch_state_bytes(ctypes.byref(p)))


def lbch_save_state_device(ctx, d_dst: int, nbytes: int) -> None:
    _check(ctx, load().lbch_save_state_device(ctx, ctypes.c_void_p(int(d_dst)), int(nbytes)),
           "lbch_save_state_device")


def lbch_restore_state_device(ctx, d_src: int, nbytes: int) -> None:
    _check(ctx, load().lbch_restore_state_device(ctx, ctypes.c_void_p(int(d_src)), int(nbytes)),
           "lbch_restore_state_device")


def lbch_last_error(ctx) -> str:
    return (load().lbch_last_error(ctx) or b"").decode(errors="replace")


def lbch_destroy(ctx) -> None:
    if ctx:
        load().lbch_destroy(ctx)


def lbch_free_energy_static(p: lbch_params, d_f9: int, plane_stride: int, d_out: int,
                            cuda_stream: int | None) -> None:
    """Free energy of caller-held FP32 populations on the device, without device allocation.

    d_f9 and d_out are device addresses (e.g. ``tensor.data_ptr()``); the result lands in
    the double at d_out, asynchronously on the stream.
    """
    st = load().lbch_free_energy_static(ctypes.byref(p), ctypes.c_void_p(int(d_f9)), int(plane_stride),
                                        ctypes.c_void_p(int(d_out)), ctypes.c_void_p(int(cuda_stream or 0)))
    _check(None, st, "lbch_free_energy_static")


# ---------------------------------------------------------------- convenience owner

class Solver:
    """Owns a context and its device workspace (a torch uint8 tensor) on one stream.

    Host inputs are float64 arrays of shape (ny, nx) (phi) or (9, ny, nx) (state);
    pinned torch CPU tensors are accepted and used in place.
    """

    def __init__(self, params: lbch_params, device=None, stream=None):
        import torch

        self.params = params
        self.nx, self.ny = params.nx, params.ny
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        nbytes = lbch_workspace_bytes(params)
        if nbytes == 0:
            raise LbchError(EINVAL, "lbch_workspace_bytes", "invalid parameters")
        with torch.cuda.device(self.device):
            self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
            self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
            self.ctx = lbch_create(params, self.workspace.data_ptr(), nbytes, self.stream.cuda_stream)

    def _on_device(self):
        import torch
        return torch.cuda.device(self.device)

    def init_field(self, phi0) -> None:
        a = _as_host_f64(phi0, self.nx * self.ny, "phi0")
        with self._on_device():
            lbch_init_field(self.ctx, a)

    def step(self, n: int) -> None:
        with self._on_device():
            lbch_step(self.ctx, n)

    def init_field_device(self, phi0) -> None:
        """f = f^eq(phi0) from a contiguous float32 CUDA tensor of shape (ny, nx)."""
        _check_device_f32(phi0, self.nx * self.ny, "phi0")
        with self._on_device():
            lbch_init_field_device(self.ctx, phi0.data_ptr())

    def phi_device(self, out=None):
        """phi = sum_i f_i into a float32 CUDA tensor (ny, nx) (allocated if out is None)."""
        import torch

        if out is None:
            out = torch.empty((self.ny, self.nx), dtype=torch.float32, device=self.device)
        _check_device_f32(out, self.nx * self.ny, "out")
        with self._on_device():
            lbch_get_phi_device(self.ctx, out.data_ptr())
        return out

    def mass(self) -> float:
        with self._on_device():
            return lbch_mass(self.ctx)

    def free_energy(self) -> float:
        with self._on_device():
            return lbch_free_energy(self.ctx)

    def field(self, out=None) -> np.ndarray:
        if out is None:
            out = np.empty((self.ny, self.nx), dtype=np.float64)
        buf = out.detach().numpy() if hasattr(out, "detach") else out
        assert buf.dtype == np.float64 and buf.flags.c_contiguous and buf.size == self.nx * self.ny
        with self._on_device():
            lbch_get_field(self.ctx, buf)
        return out

    def state(self) -> np.ndarray:
        out = np.empty((9, self.ny, self.nx), dtype=np.float64)
        with self._on_device():
            lbch_get_state(self.ctx, out)
        return out

    def set_state(self, f9) -> None:
        a = _as_host_f64(f9, 9 * self.nx * self.ny, "state")
        with self._on_device():
            lbch_set_state(self.ctx, a)

    def mass_device(self, out) -> None:
        """lbch_mass_device into out[0] (a float64 CUDA tensor), asynchronously."""
        _check_device_f64(out, "out")
        with self._on_device():
            lbch_mass_device(self.ctx, out.data_ptr())

    def free_energy_device(self, out) -> None:
        """lbch_free_energy_device into out[0] (a float64 CUDA tensor), asynchronously."""
        _check_device_f64(out, "out")
        with self._on_device():
            lbch_free_energy_device(self.ctx, out.data_ptr())

    def field_diagnostics_device(self, phi, out) -> None:
        """Mass and free energy of a float32 CUDA field (ny, nx) into out[0:2] (float64 CUDA)."""
        _check_device_f32(phi, self.nx * self.ny, "phi")
        _check_device_f64(out, "out")
        with self._on_device():
            lbch_field_diagnostics_device(self.ctx, phi.data_ptr(), out.data_ptr())

    def save_state_device(self, out=None):
        """Device-side checkpoint into a uint8 CUDA tensor of lbch_state_bytes (allocated if None)."""
        import torch

        nb = lbch_state_bytes(self.params)
        if out is None:
            out = torch.empty(nb, dtype=torch.uint8, device=self.device)
        if not (out.is_cuda and out.is_contiguous() and out.numel() * out.element_size() >= nb):
            raise ValueError(f"out: expected a contiguous CUDA tensor of at least {nb} bytes")
        with self._on_device():
            lbch_save_state_device(self.ctx, out.data_ptr(), out.numel() * out.element_size())
        return out

    def restore_state_device(self, image) -> None:
        with self._on_device():
            lbch_restore_state_device(self.ctx, image.data_ptr(), image.numel() * image.element_size())

    @property
    def steps_taken(self) -> int:
        return lbch_steps_taken(self.ctx)

    def close(self) -> None:
        if getattr(self, "ctx", None):
            lbch_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------- batches (C names)

def _i32(v):
    a = np.ascontiguousarray(v, dtype=np.int32)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def _batch_check(b, status: int, what: str):
    if status != OK:
        detail = (load().lbch_batch_last_error(b) or b"").decode(errors="replace") if b else ""
        raise LbchError(status, what, detail)


def lbch_batch_workspace_bytes(common: lbch_params, nx, ny) -> int:
    (ax, px), (ay, py) = _i32(nx), _i32(ny)
    return int(load().lbch_batch_workspace_bytes(ctypes.byref(common), len(ax), px, py))


def lbch_batch_create(common: lbch_params, nx, ny, alpha, d_workspace: int, nbytes: int, cuda_stream):
    (ax, px), (ay, py) = _i32(nx), _i32(ny)
    al = None if alpha is None else np.ascontiguousarray(alpha, dtype=np.float64)
    b = ctypes.c_void_p()
    st = load().lbch_batch_create(ctypes.byref(common), len(ax), px, py, None if al is None else _host_ptr(al),
                                  ctypes.c_void_p(int(d_workspace)), int(nbytes),
                                  ctypes.c_void_p(int(cuda_stream or 0)), ctypes.byref(b))
    _batch_check(None, st, "lbch_batch_create")
    return b


def lbch_batch_init_field(b, i: int, phi0) -> None:
    _batch_check(b, load().lbch_batch_init_field(b, int(i), _host_ptr(phi0)), "lbch_batch_init_field")


def lbch_batch_step(b, n: int) -> None:
    _batch_check(b, load().lbch_batch_step(b, int(n)), "lbch_batch_step")


def lbch_batch_get_field(b, i: int, out: np.ndarray) -> np.ndarray:
    _batch_check(b, load().lbch_batch_get_field(b, int(i), _host_ptr(out)), "lbch_batch_get_field")
    return out


def lbch_batch_get_phi_device(b, i: int, d_phi: int) -> None:
    _batch_check(b, load().lbch_batch_get_phi_device(b, int(i), ctypes.c_void_p(int(d_phi))),
                 "lbch_batch_get_phi_device")


def lbch_batch_mass(b, i: int) -> float:
    v = ctypes.c_double()
    _batch_check(b, load().lbch_batch_mass(b, int(i), ctypes.byref(v)), "lbch_batch_mass")
    return v.value


def lbch_batch_free_energy(b, i: int) -> float:
    v = ctypes.c_double()
    _batch_check(b, load().lbch_batch_free_energy(b, int(i), ctypes.byref(v)), "lbch_batch_free_energy")
    return v.value


def lbch_batch_rows_target(b) -> int:
    return int(load().lbch_batch_rows_target(b))


def lbch_batch_steps_taken(b) -> int:
    return int(load().lbch_batch_steps_taken(b))


def lbch_batch_last_error(b) -> str:
    return (load().lbch_batch_last_error(b) or b"").decode(errors="replace")


def lbch_batch_destroy(b) -> None:
    if b:
        load().lbch_batch_destroy(b)


class Batch:
    """Owns a batch of periodic fields (sizes nx[i] x ny[i], strengths alpha[i]) and its
    device workspace; the other parameters come from ``common``."""

    def __init__(self, common: lbch_params, nx, ny, alpha=None, device=None, stream=None):
        import torch

        self.nx = [int(v) for v in nx]
        self.ny = [int(v) for v in ny]
        self.count = len(self.nx)
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        nbytes = lbch_batch_workspace_bytes(common, self.nx, self.ny)
        if nbytes == 0:
            raise LbchError(EINVAL, "lbch_batch_workspace_bytes", "invalid arguments")
        with torch.cuda.device(self.device):
            self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
            self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
            self.handle = lbch_batch_create(common, self.nx, self.ny, alpha, self.workspace.data_ptr(), nbytes,
                                            self.stream.cuda_stream)

    def _on_device(self):
        import torch
        return torch.cuda.device(self.device)

    def init_field(self, i: int, phi0) -> None:
        a = _as_host_f64(phi0, self.nx[i] * self.ny[i], "phi0")
        with self._on_device():
            lbch_batch_init_field(self.handle, i, a)

    def step(self, n: int) -> None:
        with self._on_device():
            lbch_batch_step(self.handle, n)

    def phi_device(self, i: int, out) -> None:
        """phi of field i into a contiguous float32 CUDA tensor of ny[i] x nx[i] values."""
        _check_device_f32(out, self.nx[i] * self.ny[i], "out")
        with self._on_device():
            lbch_batch_get_phi_device(self.handle, i, out.data_ptr())

    def field(self, i: int) -> np.ndarray:
        out = np.empty((self.ny[i], self.nx[i]), dtype=np.float64)
        with self._on_device():
            lbch_batch_get_field(self.handle, i, out)
        return out

    def mass(self, i: int) -> float:
        with self._on_device():
            return lbch_batch_mass(self.handle, i)

    def free_energy(self, i: int) -> float:
        with self._on_device():
            return lbch_batch_free_energy(self.handle, i)

    @property
    def rows_target(self) -> int:
        return lbch_batch_rows_target(self.handle)

    @property
    def steps_taken(self) -> int:
        return lbch_batch_steps_taken(self.handle)

    def close(self) -> None:
        if getattr(self, "handle", None):
            lbch_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------- 3D (C names)

def _check3(c, status: int, what: str):
    if status != OK:
        detail = (load().lbch3_last_error(c) or b"").decode(errors="replace") if c else ""
        raise LbchError(status, what, detail)


def lbch3_workspace_bytes(p: lbch3_params) -> int:
    return int(load().lbch3_workspace_bytes(ctypes.byref(p)))


def lbch3_create(p: lbch3_params, d_workspace: int, nbytes: int, cuda_stream):
    c = ctypes.c_void_p()
    st = load().lbch3_create(ctypes.byref(p), ctypes.c_void_p(int(d_workspace)), int(nbytes),
                             ctypes.c_void_p(int(cuda_stream or 0)), ctypes.byref(c))
    _check3(None, st, "lbch3_create")
    return c


def lbch3_init_field(c, phi0) -> None:
    _check3(c, load().lbch3_init_field(c, _host_ptr(phi0)), "lbch3_init_field")


def lbch3_step(c, n: int) -> None:
    _check3(c, load().lbch3_step(c, int(n)), "lbch3_step")


def lbch3_get_field(c, out: np.ndarray) -> np.ndarray:
    _check3(c, load().lbch3_get_field(c, _host_ptr(out)), "lbch3_get_field")
    return out


def lbch3_mass(c) -> float:
    v = ctypes.c_double()
    _check3(c, load().lbch3_mass(c, ctypes.byref(v)), "lbch3_mass")
    return v.value


def lbch3_free_energy(c) -> float:
    v = ctypes.c_double()
    _check3(c, load().lbch3_free_energy(c, ctypes.byref(v)), "lbch3_free_energy")
    return v.value


def lbch3_last_error(c) -> str:
    return (load().lbch3_last_error(c) or b"").decode(errors="replace")


def lbch3_destroy(c) -> None:
    if c:
        load().lbch3_destroy(c)


class Solver3:
    """Owns a 3D (D3Q15) context and its workspace; fields are (nz, ny, nx) float64 arrays."""

    def __init__(self, params: lbch3_params, device=None, stream=None):
        import torch

        self.params = params
        self.shape = (params.nz, params.ny, params.nx)
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        nbytes = lbch3_workspace_bytes(params)
        if nbytes == 0:
            raise LbchError(EINVAL, "lbch3_workspace_bytes", "invalid parameters")
        with torch.cuda.device(self.device):
            self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
            self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
            self.ctx = lbch3_create(params, self.workspace.data_ptr(), nbytes, self.stream.cuda_stream)

    def _on_device(self):
        import torch
        return torch.cuda.device(self.device)

    def init_field(self, phi0) -> None:
        a = _as_host_f64(phi0, int(np.prod(self.shape)), "phi0")
        with self._on_device():
            lbch3_init_field(self.ctx, a)

    def step(self, n: int) -> None:
        with self._on_device():
            lbch3_step(self.ctx, n)

    def field(self) -> np.ndarray:
        out = np.empty(self.shape, dtype=np.float64)
        with self._on_device():
            lbch3_get_field(self.ctx, out)
        return out

    def mass(self) -> float:
        with self._on_device():
            return lbch3_mass(self.ctx)

    def free_energy(self) -> float:
        with self._on_device():
            return lbch3_free_energy(self.ctx)

    def close(self) -> None:
        if getattr(self, "ctx", None):
            lbch3_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
