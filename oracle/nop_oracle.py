"""FP64 NumPy oracle for the learned leap: a periodic convolutional U-Net that maps
phi(t) to phi(t + K) for the anisotropic Cahn-Hilliard LBM, with its loss, its
gradients and the Adam update.

TEST INFRASTRUCTURE ONLY. Only the test suite, the smoke check and the benchmark
may import this module. It shares no code with the CUDA library and never imports
it; the two meet only through the flat parameter vector and the array layouts
stated below, which each side implements on its own.

The surrogate is not part of arXiv 2501.03759: it leaps K steps of the scheme of
Section 3 (Eqs. 17-26), and the scheme itself is what it is checked against. Every
operation here is written out from its textbook definition:
  - 3x3 cross-correlation on a periodic grid, y(p) = sum_d W_d x(p + d) + b,
    and its two adjoints (data and weight gradients);
  - SiLU, z sigmoid(z) (Elfwing, Uchibe, Doya 2018);
  - 2x2 average pooling and nearest-neighbour 2x upsampling, and their adjoints;
  - 4x4 space-to-depth and depth-to-space;
  - Adam (Kingma, Ba 2015, Algorithm 1, with bias correction).

Layouts:
  activations  (B, H, W, C), channels last;
  phi          (B, H, W) with H, W multiples of 32;
  conv weight  W[tap, c_out, c_in], tap = 3 (dy + 1) + (dx + 1) for the offset
               (dy, dx) in {-1, 0, 1}^2 (dy along H, dx along W);
  parameters   one flat vector: for each layer of LAYERS in order, W (9 c_out c_in
               values, tap-major), then the bias b (c_out), and for the first layer
               also the conditioning vector v (c_out) that adds alpha v to its
               pre-activation (alpha: the anisotropy strength of Eq. 6).
Parity: pinned (tests/test_nop_oracle_pins.py: FFT convolution, adjoint identities,
finite-difference gradients, closed-form Adam steps).
"""
from __future__ import annotations

import numpy as np

# name, c_in, c_out, level (resolution H/4 / 2^level), activation
LAYERS = [
    ("e0a", 16, 96, 0, True),
    ("e0b", 96, 96, 0, True),
    ("e1a", 96, 64, 1, True),
    ("e1b", 64, 64, 1, True),
    ("e2a", 64, 96, 2, True),
    ("e2b", 96, 96, 2, True),
    ("m3a", 96, 96, 3, True),
    ("m3b", 96, 96, 3, True),
    ("d2a", 96, 96, 2, True),
    ("d2b", 96, 64, 2, False),
    ("d1a", 64, 64, 1, True),
    ("d1b", 64, 96, 1, False),
    ("d0a", 96, 96, 0, True),
    ("out", 96, 16, 0, False),
    ("lin", 16, 16, 0, False),    # linear path from the network input
    ("lina", 16, 16, 0, False),   # the same, its output multiplied by alpha
]
TAPS = [(dy, dx) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]


def param_count() -> int:
    n = 0
    for name, ci, co, _, _ in LAYERS:
        n += 9 * co * ci + co + (co if name == "e0a" else 0)
    return n


def unpack(theta: np.ndarray) -> dict:
    """Flat parameter vector -> {name: (W, b[, v])}."""
    out, k = {}, 0
    for name, ci, co, _, _ in LAYERS:
        W = theta[k:k + 9 * co * ci].reshape(9, co, ci)
        k += 9 * co * ci
        b = theta[k:k + co]
        k += co
        if name == "e0a":
            v = theta[k:k + co]
            k += co
            out[name] = (W, b, v)
        else:
            out[name] = (W, b)
    assert k == theta.size
    return out


def pack(grads: dict) -> np.ndarray:
    parts = []
    for name, *_ in LAYERS:
        parts.extend(g.ravel() for g in grads[name])
    return np.concatenate(parts)


# ---------------------------------------------------------------- elementary operations

def shift(x: np.ndarray, dy: int, dx: int) -> np.ndarray:
    """Periodic shift: shift(x, dy, dx)[b, i, j] = x[b, i + dy, j + dx]."""
    return np.roll(x, shift=(-dy, -dx), axis=(1, 2))


def conv(x: np.ndarray, W: np.ndarray, b: np.ndarray | None = None) -> np.ndarray:
    """y(p) = sum_d W_d x(p + d) (+ b): 3x3 periodic cross-correlation."""
    y = sum(shift(x, dy, dx) @ W[t].T for t, (dy, dx) in enumerate(TAPS))
    return y if b is None else y + b


def conv_bwd_data(dy: np.ndarray, W: np.ndarray) -> np.ndarray:
    """Adjoint of conv in x: dx(q) = sum_d W_d^T dy(q - d)."""
    return sum(shift(dy @ W[t], -oy, -ox) for t, (oy, ox) in enumerate(TAPS))


def conv_bwd_weight(x: np.ndarray, dy: np.ndarray) -> np.ndarray:
    """Adjoint of conv in W: dW_d = sum_{b, p} dy(p) x(p + d)^T, shape (9, c_out, c_in)."""
    return np.stack([np.einsum("bhwo,bhwi->oi", dy, shift(x, oy, ox)) for oy, ox in TAPS])


def sigmoid(z):
    return 1.0 / (1.0 + np.exp(-z))


def silu(z):
    return z * sigmoid(z)


def silu_grad(z):
    s = sigmoid(z)
    return s * (1.0 + z * (1.0 - s))


def pool(x):
    """2x2 average pooling."""
    B, H, W, C = x.shape
    return x.reshape(B, H // 2, 2, W // 2, 2, C).mean(axis=(2, 4))


def pool_bwd(g):
    return np.repeat(np.repeat(g, 2, axis=1), 2, axis=2) / 4.0


def up(x):
    """Nearest-neighbour 2x upsampling."""
    return np.repeat(np.repeat(x, 2, axis=1), 2, axis=2)


def up_bwd(g):
    B, H, W, C = g.shape
    return g.reshape(B, H // 2, 2, W // 2, 2, C).sum(axis=(2, 4))


def s2d(phi):
    """(B, H, W) -> (B, H/4, W/4, 16), channel 4 di + dj holds phi[4 i + di, 4 j + dj]."""
    B, H, W = phi.shape
    return phi.reshape(B, H // 4, 4, W // 4, 4).transpose(0, 1, 3, 2, 4).reshape(B, H // 4, W // 4, 16)


def d2s(x):
    B, h, w, _ = x.shape
    return x.reshape(B, h, w, 4, 4).transpose(0, 1, 3, 2, 4).reshape(B, 4 * h, 4 * w)


# ---------------------------------------------------------------- the network

def bf16(a):
    """Round to the nearest BF16 value (ties to even) through FP32: the storage format of
    weights, activations and activation gradients in the CUDA path."""
    x = np.asarray(a, dtype=np.float32)
    u = x.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) >> 16 << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def _identity(a):
    return a


def rms(phi: np.ndarray) -> np.ndarray:
    """Root mean square of each field, shape (B, 1, 1); 1 for a zero field."""
    r = np.sqrt(np.mean(phi * phi, axis=(1, 2), keepdims=True))
    return np.where(r > 1e-30, r, 1.0)


def forward(theta: np.ndarray, phi: np.ndarray, alpha: np.ndarray, scale: float, quantize=None):
    """phi_out = phi + scale sig (D - mean D), D = d2s(U-Net(s2d(phi / sig), alpha)), sig the
    root mean square of each field (so the network sees fields of unit size).

    quantize (default: none) is applied where the CUDA path stores BF16: the weights, the
    network input (as a rounded value plus its rounded remainder), every activation, pooled
    and summed tensor, and linear layer output. Returns phi_out and the saved tensors the
    backward pass needs.
    """
    Q = quantize or _identity
    P = unpack(theta)
    alpha = np.asarray(alpha, dtype=np.float64).reshape(-1, 1, 1, 1)
    s = {"Q": Q}

    def layer(name, x):
        W, b = Q(P[name][0]), P[name][1]
        z = conv(x, W, b)
        if name == "e0a":  # the input's BF16 remainder, by the same weights (0 without quantize)
            z = z + conv(s["x0_lo"], W) + alpha * P[name][2]
        s["in_" + name], s["z_" + name] = x, z
        act = dict((l[0], l[4]) for l in LAYERS)[name]
        if name == "out":
            return z
        return Q(silu(z)) if act else Q(z)

    sig = rms(phi)
    s["sig"] = sig
    x0f = s2d(phi / sig)
    x0 = Q(x0f)
    s["x0_lo"] = Q(x0f - x0)
    h0 = layer("e0b", layer("e0a", x0))
    h1 = layer("e1b", layer("e1a", Q(pool(h0))))
    h2 = layer("e2b", layer("e2a", Q(pool(h1))))
    h3 = layer("m3b", layer("m3a", Q(pool(h2))))
    zd2 = layer("d2b", layer("d2a", Q(up(h3) + h2)))
    zd1 = layer("d1b", layer("d1a", Q(up(zd2) + h1)))
    zo = layer("out", layer("d0a", Q(up(zd1) + h0)))
    for name in ("lin", "lina"):  # linear path: W x0 + b, times alpha for lina
        Wf, b = P[name][0], P[name][1]
        W = Q(Wf)
        W_lo = Q(Wf - W)  # with BF16 storage the weights are kept as two halves too
        zl = conv(x0, W, b) + conv(s["x0_lo"], W) + conv(x0, W_lo)
        zo = zo + (alpha * zl if name == "lina" else zl)
    s["in_lin"] = s["in_lina"] = x0
    D = d2s(zo)
    D = D - D.mean(axis=(1, 2), keepdims=True)
    s["alpha"] = alpha
    return phi + scale * sig * D, s


def loss(phi_out: np.ndarray, target: np.ndarray, weight=None) -> tuple[float, np.ndarray]:
    """sum_b w_b sum_x (phi_out - target)^2 / (B H W) (w_b = 1 by default: the mean squared
    error), and its gradient in phi_out."""
    d = phi_out - target
    w = np.ones(d.shape[0]) if weight is None else np.asarray(weight, dtype=np.float64)
    w = w.reshape(-1, 1, 1)
    return float(np.sum(w * d * d) / d.size), 2.0 * w * d / d.size


def backward(theta: np.ndarray, s: dict, dphi_out: np.ndarray, scale: float) -> np.ndarray:
    """Gradient of the loss in the flat parameter vector, given d loss / d phi_out."""
    P = unpack(theta)
    Q = s["Q"]
    G = {}

    def layer_bwd(name, g_out, act):
        """g_out: gradient in the layer's output; returns the gradient in its input."""
        z, x = s["z_" + name], s["in_" + name]
        dz = Q(g_out * silu_grad(Q(z)) if act else g_out)
        W = Q(P[name][0])
        grads = [conv_bwd_weight(x, dz), dz.sum(axis=(0, 1, 2))]
        if name == "e0a":
            grads[0] = grads[0] + conv_bwd_weight(s["x0_lo"], dz)
            grads.append((dz * s["alpha"]).sum(axis=(0, 1, 2)))
        G[name] = grads
        return conv_bwd_data(dz, W)

    dD = scale * s["sig"] * (dphi_out - dphi_out.mean(axis=(1, 2), keepdims=True))
    g = s2d(dD)  # adjoint of d2s (quantised as the output layer's dz)
    for name in ("lin", "lina"):
        dz = Q(g)
        if name == "lina":
            dz = Q(s["alpha"] * dz)
        G[name] = [conv_bwd_weight(s["in_" + name], dz) + conv_bwd_weight(s["x0_lo"], dz), dz.sum(axis=(0, 1, 2))]
    g = layer_bwd("out", g, False)
    g_in_d0a = layer_bwd("d0a", g, True)
    g_h0 = g_in_d0a.copy()
    g = layer_bwd("d1b", up_bwd(g_in_d0a), False)
    g_in_d1a = layer_bwd("d1a", g, True)
    g_h1 = g_in_d1a.copy()
    g = layer_bwd("d2b", up_bwd(g_in_d1a), False)
    g_in_d2a = layer_bwd("d2a", g, True)
    g_h2 = g_in_d2a.copy()
    g = layer_bwd("m3b", up_bwd(g_in_d2a), True)
    g_h2 += pool_bwd(layer_bwd("m3a", g, True))
    g = layer_bwd("e2b", g_h2, True)
    g_h1 += pool_bwd(layer_bwd("e2a", g, True))
    g = layer_bwd("e1b", g_h1, True)
    g_h0 += pool_bwd(layer_bwd("e1a", g, True))
    g = layer_bwd("e0b", g_h0, True)
    layer_bwd("e0a", g, True)
    return pack(G)


def clip_global_norm(grad, max_norm):
    """Global-norm gradient clipping: grad scaled by min(1, max_norm / |grad|_2); max_norm 0
    leaves it unchanged."""
    nrm = float(np.sqrt(np.sum(np.asarray(grad, dtype=np.float64) ** 2)))
    if max_norm > 0.0 and nrm > max_norm:
        return grad * (max_norm / nrm)
    return grad


def adam(theta, grad, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step (Kingma, Ba 2015, Algorithm 1); t counts from 1. Returns new arrays."""
    m = beta1 * m + (1.0 - beta1) * grad
    v = beta2 * v + (1.0 - beta2) * grad * grad
    mhat = m / (1.0 - beta1 ** t)
    vhat = v / (1.0 - beta2 ** t)
    return theta - lr * mhat / (np.sqrt(vhat) + eps), m, v
