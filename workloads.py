"""Seeded synthetic initial fields phi0 for the anisotropic Cahn-Hilliard runs.

This module holds only input generation (the shapes of the paper's initial
conditions, Eqs. 40-42, resized), none of the lattice Boltzmann arithmetic. Both
the CUDA path and the FP64 oracle take the same float64 arrays from here, so no
random number generator has to be matched between them.

Every field is float64 with shape (ny, nx), row-major with x fastest; node (x, y)
sits at integer coordinates.
"""
from __future__ import annotations

import numpy as np


def droplet(nx: int, ny: int, radius: float, width: float, cx: float | None = None,
            cy: float | None = None) -> np.ndarray:
    """phi0 = tanh((R - r) / width), r the distance from (cx, cy) (default the grid centre).

    With width = D/2 this is the profile of Eq. 40, tanh(2(R - r)/D); with
    width = sqrt(2) * 1.5 it is the 64x64 droplet workload's profile.
    """
    cx = nx / 2.0 if cx is None else cx
    cy = ny / 2.0 if cy is None else cy
    y, x = np.meshgrid(np.arange(ny, dtype=np.float64), np.arange(nx, dtype=np.float64),
                       indexing="ij")
    r = np.sqrt((x - cx) ** 2 + (y - cy) ** 2)
    return np.tanh((radius - r) / width)


def droplet_workload(n: int = 64) -> np.ndarray:
    """n x n droplet, radius 20 (scaled 0.3125 n), profile tanh((R - r)/(sqrt(2) 1.5))."""
    return droplet(n, n, radius=20.0 * n / 64.0, width=np.sqrt(2.0) * 1.5)


def two_droplets(nx: int, ny: int, drops, width: float) -> np.ndarray:
    """Eq. 41: sum_i tanh((R_i - r_i)/width) + 1, drops = [(R, x, y), ...]."""
    y, x = np.meshgrid(np.arange(ny, dtype=np.float64), np.arange(nx, dtype=np.float64),
                       indexing="ij")
    out = np.ones((ny, nx))
    for (R, cx, cy) in drops:
        out += np.tanh((R - np.sqrt((x - cx) ** 2 + (y - cy) ** 2)) / width)
    return out


def noise(nx: int, ny: int, amplitude: float, seed: int, mean: float = 0.0) -> np.ndarray:
    """Spinodal initial field (Eq. 42 shape): mean + U[-amplitude, amplitude], i.i.d. per node."""
    rng = np.random.default_rng(seed)
    return mean + rng.uniform(-amplitude, amplitude, size=(ny, nx))


def cosine_mode(nx: int, ny: int, mx: int, my: int, amplitude: float, mean: float,
                shift: float | None = None) -> np.ndarray:
    """mean + A cos(q . x + shift), q = 2 pi (mx/nx, my/ny).

    The default shift of half a node along the dominant axis (pi |m|/n) keeps every node
    off the zeros of the gradient for modes along an axis or a diagonal, so no node has
    grad phi = 0. Other directions pass their own shift.
    """
    y, x = np.meshgrid(np.arange(ny, dtype=np.float64), np.arange(nx, dtype=np.float64),
                       indexing="ij")
    if shift is None:
        m = max(abs(mx), abs(my))
        n = nx if abs(mx) >= abs(my) else ny
        shift = np.pi * m / n
    return mean + amplitude * np.cos(2 * np.pi * (mx * x / nx + my * y / ny) + shift)


def planar_bands(nx: int, ny: int, x_left: float, x_right: float, width: float) -> np.ndarray:
    """+1 between two planar interfaces normal to x, -1 outside; tanh profiles of the given width."""
    x = np.arange(nx, dtype=np.float64)[None, :].repeat(ny, axis=0)
    return np.tanh((x - x_left) / width) - np.tanh((x - x_right) / width) - 1.0


def batch_sweep_specs(count: int = 512, seed: int = 0):
    """The parameter-sweep batch: count square fields with edges drawn uniformly from
    {64, 128, 256, 512}, alpha ~ U[0, 0.5], alternating droplet (radius 0.3 L, profile
    tanh((R - r)/(sqrt(2) 1.5))) and spinodal (U[-0.05, 0.05]) initial fields.

    Returns a list of dicts (n, alpha, kind, seed); batch_field(spec) builds phi0."""
    rng = np.random.default_rng(seed)
    sizes = rng.choice(np.array([64, 128, 256, 512]), size=count)
    alphas = rng.uniform(0.0, 0.5, size=count)
    field_seeds = rng.integers(0, 2**31 - 1, size=count)
    return [{"n": int(sizes[i]), "alpha": float(alphas[i]), "kind": "droplet" if i % 2 == 0 else "spinodal",
             "seed": int(field_seeds[i])} for i in range(count)]


def batch_field(spec) -> np.ndarray:
    n = spec["n"]
    if spec["kind"] == "droplet":
        return droplet(n, n, radius=0.3 * n, width=np.sqrt(2.0) * 1.5)
    return noise(n, n, 0.05, spec["seed"])


def bf16_exact(shape, seed: int, scale: float, levels: int = 64) -> np.ndarray:
    """Seeded values k * scale / levels with integer k in [-levels, levels]: with levels <= 128
    and scale a power of two every value has at most 8 significant bits, so it is exact in
    BF16 and products of two such values are exact in FP32 (operator test inputs)."""
    r = np.random.default_rng(seed)
    return r.integers(-levels, levels + 1, size=shape).astype(np.float64) * (scale / levels)


def surrogate_theta(seed: int, out_scale: float = 1.0) -> np.ndarray:
    """A seeded parameter vector for the learned leap (flat layout of include/lbnop.h):
    He-normal 3 x 3 weights (std sqrt(2 / (9 c_in))), those of the output layer and the
    linear path scaled by out_scale, biases N(0, 0.01), conditioning vector N(0, 0.25), rounded to float32."""
    layers = [(16, 96), (96, 96), (96, 64), (64, 64), (64, 96), (96, 96), (96, 96), (96, 96),
              (96, 96), (96, 64), (64, 64), (64, 96), (96, 96), (96, 16), (16, 16), (16, 16)]
    r = np.random.default_rng(seed)
    parts = []
    for k, (ci, co) in enumerate(layers):
        w = r.normal(0.0, (2.0 / (9 * ci)) ** 0.5, 9 * co * ci)
        if k >= 13:  # the output layer and the linear path
            w *= out_scale
        parts += [w, r.normal(0.0, 0.1, co)]
        if k == 0:
            parts.append(r.normal(0.0, 0.5, co))
    return np.concatenate(parts).astype(np.float32).astype(np.float64)
