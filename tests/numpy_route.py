"""A second, independently written FP64 route through one time step, in NumPy.

It exists only to cross-check the C++ oracle on tiny grids (a different author's
idioms: whole-array np.roll shifts, dense 9x9 operators from numpy.linalg.inv,
einsum collisions). It takes its lattice tables from the golden fixtures of
Eqs. 20 and 23 rather than from the oracle. Readings match the oracle's defaults:
k on the second term of Eq. 15, split mu_beta, n = 0 and gamma = 1 where
|grad phi|^2 < 1e-12, Willmore regularisation.
"""
import numpy as np

import golden_io

C, WT = golden_io.lattice()
MMAT = golden_io.moment_matrix()


def _at(a, cx, cy):
    """Field whose value at (x, y) is a(x + cx, y + cy), periodic."""
    return np.roll(a, shift=(-cy, -cx), axis=(0, 1))


def grad(a):
    gx = 3.0 * sum(WT[i] * C[i, 0] * _at(a, *C[i]) for i in range(9))
    gy = 3.0 * sum(WT[i] * C[i, 1] * _at(a, *C[i]) for i in range(9))
    return gx, gy


def lap(a):
    return 6.0 * sum(WT[i] * (_at(a, *C[i]) - a) for i in range(9))


def step(f, M=0.1, sigma=0.01, D=5.0, eps=0.03, alpha=0.0, s=None):
    beta = 3.0 * sigma / (4.0 * D)
    k = 3.0 * sigma * D / 8.0
    rates = np.ones(9) if s is None else np.array(s, dtype=float)
    rates[3] = rates[5] = 1.0 / (3.0 * M + 0.5)
    phi = f.sum(axis=0)
    px, py = grad(phi)
    L = lap(phi)
    g2 = px * px + py * py
    ok = g2 >= 1e-12
    nrm = np.sqrt(g2)
    safe = np.where(ok, nrm, 1.0)
    n = np.stack([np.where(ok, px / safe, 0.0), np.where(ok, py / safe, 0.0)])
    gamma = np.where(ok, 1.0 + alpha * (4.0 * (n ** 4).sum(axis=0) - 3.0), 1.0)
    dgam = 16.0 * alpha * n ** 3
    proj = np.eye(2)[:, :, None, None] - n[:, None] * n[None, :]
    pg = np.einsum("ab...,b...->a...", proj, dgam)
    Qx = (gamma - 1.0) * k * px + k * nrm * pg[0]
    Qy = (gamma - 1.0) * k * py + k * nrm * pg[1]
    fb = 4.0 * beta * phi * (phi * phi - 1.0)
    fp = 4.0 * beta * (3.0 * phi * phi - 1.0)
    w = L - fb
    mua = fb - k * L
    divq = grad(Qx)[0] + grad(Qy)[1]
    mub = (gamma - 1.0) * fb - divq + eps * (lap(w) - fp * w)
    gx, gy = grad(mub)
    feq = WT[:, None, None] * mua[None]
    feq[0] += phi - mua
    F = -WT[:, None, None] * (C[:, 0, None, None] * gx[None] + C[:, 1, None, None] * gy[None])
    Minv = np.linalg.inv(MMAT)
    A = Minv @ np.diag(rates) @ MMAT
    B = Minv @ np.diag(1.0 - rates / 2.0) @ MMAT
    post = f - np.einsum("ij,j...->i...", A, f - feq) + np.einsum("ij,j...->i...", B, F)
    return np.stack([_at(post[i], -C[i, 0], -C[i, 1]) for i in range(9)])


def init(phi0, sigma=0.01, D=5.0):
    beta = 3.0 * sigma / (4.0 * D)
    k = 3.0 * sigma * D / 8.0
    mua = 4.0 * beta * phi0 * (phi0 * phi0 - 1.0) - k * lap(phi0)
    f = WT[:, None, None] * mua[None]
    f[0] += phi0 - mua
    return f
