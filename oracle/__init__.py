"""FP64 CPU oracle for the anisotropic Cahn-Hilliard MRT lattice Boltzmann scheme.

TEST INFRASTRUCTURE ONLY. Only the test suite, the smoke check and the
benchmark's CPU-baseline leg may import this package. It shares no code with the
CUDA library (the package ``paper_2501_03759_gb300``) and never imports it.

The arithmetic lives in ``lbch_oracle.cpp`` (plain C++, FP64, whole-field passes
over arrays, following Section 3 of arXiv 2501.03759 step by step). This module
only builds that file with g++ when needed and marshals numpy arrays.

State layout: ``f`` has shape (9, ny, nx), plane i in the D2Q9 order of Eq. 20a,
x fastest, holding the post-streaming distribution f_i(x, t) of Eq. 17.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbch_oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

Q_LITERAL = 1
MU_NESTED = 2
S35_EXPLICIT = 4

NONE, WILLMORE, LINEAR = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile ``liboracle.so`` with g++ (FP64, no FMA contraction, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(
        os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "lbch_oracle.h"))
    ):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["g++", "-O2", "-std=c++17", "-fno-fast-math", "-ffp-contract=off", "-fopenmp",
               "-fPIC", "-shared", _SRC, "-o", tmp]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class _Params(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
        ("M", ctypes.c_double), ("sigma", ctypes.c_double), ("D", ctypes.c_double),
        ("eps", ctypes.c_double), ("alpha", ctypes.c_double),
        ("s", ctypes.c_double * 9),
        ("regularization", ctypes.c_int32), ("flags", ctypes.c_uint32),
    ]


class _Derived(ctypes.Structure):
    _fields_ = [("k", ctypes.c_double), ("beta", ctypes.c_double), ("s", ctypes.c_double * 9)]


@dataclass
class Params:
    """Scheme parameters. Defaults are Eq. 39 (M, eps, D, sigma) with Willmore G."""
    nx: int
    ny: int
    M: float = 0.1
    sigma: float = 0.01
    D: float = 5.0
    eps: float = 0.03
    alpha: float = 0.0
    s: list = field(default_factory=lambda: [1.0] * 9)
    regularization: int = WILLMORE
    flags: int = 0

    def c(self) -> _Params:
        p = _Params()
        p.nx, p.ny = int(self.nx), int(self.ny)
        p.M, p.sigma, p.D, p.eps, p.alpha = self.M, self.sigma, self.D, self.eps, self.alpha
        for i in range(9):
            p.s[i] = float(self.s[i])
        p.regularization = int(self.regularization)
        p.flags = int(self.flags)
        return p


class _Params3(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
        ("M", ctypes.c_double), ("sigma", ctypes.c_double), ("D", ctypes.c_double),
        ("eps", ctypes.c_double), ("alpha", ctypes.c_double),
        ("s", ctypes.c_double * 15),
        ("regularization", ctypes.c_int32), ("flags", ctypes.c_uint32),
    ]


@dataclass
class Params3:
    """3D (D3Q15) scheme parameters; defaults as Params."""
    nx: int
    ny: int
    nz: int
    M: float = 0.1
    sigma: float = 0.01
    D: float = 5.0
    eps: float = 0.03
    alpha: float = 0.0
    s: list = field(default_factory=lambda: [1.0] * 15)
    regularization: int = WILLMORE
    flags: int = 0

    def c(self) -> _Params3:
        p = _Params3()
        p.nx, p.ny, p.nz = int(self.nx), int(self.ny), int(self.nz)
        p.M, p.sigma, p.D, p.eps, p.alpha = self.M, self.sigma, self.D, self.eps, self.alpha
        for i in range(15):
            p.s[i] = float(self.s[i])
        p.regularization = int(self.regularization)
        p.flags = int(self.flags)
        return p


def _load():
    global _lib
    with _lock:
        if _lib is None:
            # LBCH_ORACLE_LIB names a prebuilt copy instead (the mutation tests load
            # oracles with a planted mistake this way, each in its own process).
            lib = ctypes.CDLL(os.environ.get("LBCH_ORACLE_LIB") or build())
            dp = ctypes.POINTER(ctypes.c_double)
            pp = ctypes.POINTER(_Params)
            lib.orc_derive.argtypes = [pp, ctypes.POINTER(_Derived)]
            lib.orc_matrices.argtypes = [dp, dp]
            lib.orc_equilibrium.argtypes = [ctypes.c_double, ctypes.c_double, dp]
            lib.orc_source.argtypes = [ctypes.c_double, ctypes.c_double, dp]
            lib.orc_collide_site.argtypes = [pp, dp, ctypes.c_double, ctypes.c_double,
                                             ctypes.c_double, ctypes.c_double, dp]
            lib.orc_init.argtypes = [pp, dp, dp]
            lib.orc_step.argtypes = [pp, dp, ctypes.c_int64]
            lib.orc_phi.argtypes = [pp, dp, dp]
            lib.orc_fields.argtypes = [pp, dp, dp]
            lib.orc_mass.argtypes = [pp, dp]
            lib.orc_mass.restype = ctypes.c_double
            lib.orc_energy.argtypes = [pp, dp]
            lib.orc_energy.restype = ctypes.c_double
            lib.orc_set_threads.argtypes = [ctypes.c_int]
            lib.orc_set_threads.restype = ctypes.c_int
            p3 = ctypes.POINTER(_Params3)
            lib.orc3_matrices.argtypes = [dp, dp]
            lib.orc3_equilibrium.argtypes = [ctypes.c_double, ctypes.c_double, dp]
            lib.orc3_source.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double, dp]
            lib.orc3_collide_site.argtypes = [p3, dp, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                              ctypes.c_double, ctypes.c_double, dp]
            lib.orc3_init.argtypes = [p3, dp, dp]
            lib.orc3_fields.argtypes = [p3, dp, dp]
            lib.orc3_step.argtypes = [p3, dp, ctypes.c_int64]
            lib.orc3_phi.argtypes = [p3, dp, dp]
            lib.orc3_mass.argtypes = [p3, dp]
            lib.orc3_mass.restype = ctypes.c_double
            lib.orc3_energy.argtypes = [p3, dp]
            lib.orc3_energy.restype = ctypes.c_double
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _check(rc: int, what: str):
    if rc != 0:
        raise ValueError(f"oracle {what}: invalid parameters")


def derive(p: Params) -> dict:
    """k, beta (inverted Eq. 5) and the relaxation rates actually used."""
    d = _Derived()
    _check(_load().orc_derive(ctypes.byref(p.c()), ctypes.byref(d)), "derive")
    return {"k": d.k, "beta": d.beta, "s": [d.s[i] for i in range(9)]}


def matrices():
    """(M of Eq. 23, its Gauss-Jordan inverse) as 9x9 arrays."""
    M = np.zeros((9, 9))
    Mi = np.zeros((9, 9))
    _load().orc_matrices(_ptr(M), _ptr(Mi))
    return M, Mi


def equilibrium(phi: float, mu_alpha: float) -> np.ndarray:
    out = np.zeros(9)
    _load().orc_equilibrium(phi, mu_alpha, _ptr(out))
    return out


def source(gx: float, gy: float) -> np.ndarray:
    out = np.zeros(9)
    _load().orc_source(gx, gy, _ptr(out))
    return out


def collide_site(p: Params, f9, phi, mu_alpha, gx, gy) -> np.ndarray:
    fi = np.ascontiguousarray(f9, dtype=np.float64)
    out = np.zeros(9)
    _load().orc_collide_site(ctypes.byref(p.c()), _ptr(fi), phi, mu_alpha, gx, gy, _ptr(out))
    return out


def init(p: Params, phi0: np.ndarray) -> np.ndarray:
    phi0 = np.ascontiguousarray(phi0, dtype=np.float64)
    assert phi0.shape == (p.ny, p.nx)
    f = np.zeros((9, p.ny, p.nx))
    _check(_load().orc_init(ctypes.byref(p.c()), _ptr(phi0), _ptr(f)), "init")
    return f


def step(p: Params, f: np.ndarray, nsteps: int) -> np.ndarray:
    """Returns a new state advanced ``nsteps`` steps (the input is not modified)."""
    g = np.array(f, dtype=np.float64, order="C", copy=True)
    assert g.shape == (9, p.ny, p.nx)
    _check(_load().orc_step(ctypes.byref(p.c()), _ptr(g), int(nsteps)), "step")
    return g


def phi(p: Params, f: np.ndarray) -> np.ndarray:
    f = np.ascontiguousarray(f, dtype=np.float64)
    out = np.zeros((p.ny, p.nx))
    _check(_load().orc_phi(ctypes.byref(p.c()), _ptr(f), _ptr(out)), "phi")
    return out


FIELD_NAMES = ("phi", "dphi_x", "dphi_y", "lap_phi", "gamma", "Qx", "Qy", "w",
               "mu_alpha", "mu_beta", "gx", "gy")


def fields(p: Params, f: np.ndarray) -> dict:
    f = np.ascontiguousarray(f, dtype=np.float64)
    out = np.zeros((12, p.ny, p.nx))
    _check(_load().orc_fields(ctypes.byref(p.c()), _ptr(f), _ptr(out)), "fields")
    return {n: out[i] for i, n in enumerate(FIELD_NAMES)}


def mass(p: Params, f: np.ndarray) -> float:
    return float(_load().orc_mass(ctypes.byref(p.c()), _ptr(np.ascontiguousarray(f))))


def energy(p: Params, f: np.ndarray) -> float:
    return float(_load().orc_energy(ctypes.byref(p.c()), _ptr(np.ascontiguousarray(f))))


def set_threads(n: int) -> int:
    return int(_load().orc_set_threads(int(n)))


def run(p: Params, phi0: np.ndarray, nsteps: int) -> np.ndarray:
    """phi after ``nsteps`` steps from f = f^eq(phi0)."""
    return phi(p, step(p, init(p, phi0), nsteps))


def run_window(p: Params, phi0_full: np.ndarray, x0: int, y0: int, w: int, h: int,
               nsteps: int) -> np.ndarray:
    """phi after ``nsteps`` steps on the w x h window at (x0, y0) of a periodic field.

    Each step reads phi at most 4 nodes away (pull of f* at radius 1, whose
    collision needs phi at radius 3), and the initial state reads phi0 at radius 1,
    so a window padded by 4*nsteps + 1 nodes (taken with periodic wrap from the
    full field) gives the exact interior however the pad itself evolves.
    """
    ny, nx = phi0_full.shape
    pad = 4 * int(nsteps) + 1
    ys = (np.arange(y0 - pad, y0 + h + pad)) % ny
    xs = (np.arange(x0 - pad, x0 + w + pad)) % nx
    sub = np.ascontiguousarray(phi0_full[np.ix_(ys, xs)])
    q = Params(**{**p.__dict__, "nx": sub.shape[1], "ny": sub.shape[0]})
    out = run(q, sub, nsteps)
    return out[pad:pad + h, pad:pad + w]


# ---------------------------------------------------------------- 3D (D3Q15)

def matrices3():
    """(M of Eq. 24 as built by the oracle, its Gauss-Jordan inverse), 15x15."""
    M = np.zeros((15, 15))
    Mi = np.zeros((15, 15))
    _load().orc3_matrices(_ptr(M), _ptr(Mi))
    return M, Mi


def equilibrium3(phi: float, mu_alpha: float) -> np.ndarray:
    out = np.zeros(15)
    _load().orc3_equilibrium(phi, mu_alpha, _ptr(out))
    return out


def source3(gx: float, gy: float, gz: float) -> np.ndarray:
    out = np.zeros(15)
    _load().orc3_source(gx, gy, gz, _ptr(out))
    return out


def collide_site3(p: Params3, f15, phi, mu_alpha, gx, gy, gz) -> np.ndarray:
    fi = np.ascontiguousarray(f15, dtype=np.float64)
    out = np.zeros(15)
    _load().orc3_collide_site(ctypes.byref(p.c()), _ptr(fi), phi, mu_alpha, gx, gy, gz, _ptr(out))
    return out


def init3(p: Params3, phi0: np.ndarray) -> np.ndarray:
    phi0 = np.ascontiguousarray(phi0, dtype=np.float64)
    assert phi0.shape == (p.nz, p.ny, p.nx)
    f = np.zeros((15, p.nz, p.ny, p.nx))
    _check(_load().orc3_init(ctypes.byref(p.c()), _ptr(phi0), _ptr(f)), "init3")
    return f


def step3(p: Params3, f: np.ndarray, nsteps: int) -> np.ndarray:
    g = np.array(f, dtype=np.float64, order="C", copy=True)
    assert g.shape == (15, p.nz, p.ny, p.nx)
    _check(_load().orc3_step(ctypes.byref(p.c()), _ptr(g), int(nsteps)), "step3")
    return g


def fields3(p: Params3, f: np.ndarray) -> dict:
    """phi, gamma, mu_alpha and mu_beta of a 3D state, each (nz, ny, nx)."""
    f = np.ascontiguousarray(f, dtype=np.float64)
    out = np.zeros((4, p.nz, p.ny, p.nx))
    _check(_load().orc3_fields(ctypes.byref(p.c()), _ptr(f), _ptr(out)), "fields3")
    return {n: out[i] for i, n in enumerate(("phi", "gamma", "mu_alpha", "mu_beta"))}


def phi3(p: Params3, f: np.ndarray) -> np.ndarray:
    out = np.zeros((p.nz, p.ny, p.nx))
    _check(_load().orc3_phi(ctypes.byref(p.c()), _ptr(np.ascontiguousarray(f)), _ptr(out)), "phi3")
    return out


def mass3(p: Params3, f: np.ndarray) -> float:
    return float(_load().orc3_mass(ctypes.byref(p.c()), _ptr(np.ascontiguousarray(f))))


def energy3(p: Params3, f: np.ndarray) -> float:
    return float(_load().orc3_energy(ctypes.byref(p.c()), _ptr(np.ascontiguousarray(f))))


def run3(p: Params3, phi0: np.ndarray, nsteps: int) -> np.ndarray:
    """phi after nsteps 3D steps from f = f^eq(phi0)."""
    return phi3(p, step3(p, init3(p, phi0), nsteps))
