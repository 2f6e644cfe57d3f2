"""Pins of the learned-leap oracle (oracle/nop_oracle.py) against facts that do not
depend on it: FFT circular correlation, adjoint (dot-product) identities, central
finite differences of the whole network's loss, exact mass conservation of the
head, the closed form of Adam's first steps, and BF16 round-to-nearest-even cases."""
import numpy as np
import pytest

from oracle import nop_oracle as N

rng = np.random.default_rng(11)


def rand_theta(seed=0, out_scale=1.0):
    r = np.random.default_rng(seed)
    P = {}
    for name, ci, co, _, _ in N.LAYERS:
        W = r.normal(0.0, (2.0 / (9 * ci)) ** 0.5, (9, co, ci))
        if name == "out":
            W *= out_scale
        parts = [W, r.normal(0.0, 0.1, co)]
        if name == "e0a":
            parts.append(r.normal(0.0, 0.5, co))
        P[name] = parts
    return N.pack(P)


def test_conv_matches_fft_circular_correlation():
    B, H, W, ci, co = 2, 8, 12, 3, 5
    x = rng.normal(size=(B, H, W, ci))
    Wt = rng.normal(size=(9, co, ci))
    y = N.conv(x, Wt)
    # y[p, o] = sum_i sum_d K_{o,i}[d] x_i[p + d] = ifft(fft(x_i) * conj(fft(k_{o,i})))
    ref = np.zeros((B, H, W, co))
    for o in range(co):
        for i in range(ci):
            k = np.zeros((H, W))
            for t, (dy, dx) in enumerate(N.TAPS):
                k[dy % H, dx % W] += Wt[t, o, i]
            ref[..., o] += np.real(np.fft.ifft2(np.fft.fft2(x[..., i]) * np.conj(np.fft.fft2(k))))
    assert np.abs(y - ref).max() < 1e-12


def test_conv_known_offsets():
    # A single tap picks the neighbour it names: tap (dy, dx) = (1, -1) reads x[i + 1, j - 1].
    x = rng.normal(size=(1, 5, 6, 1))
    Wt = np.zeros((9, 1, 1))
    Wt[N.TAPS.index((1, -1)), 0, 0] = 1.0
    y = N.conv(x, Wt)
    assert y[0, 2, 3, 0] == x[0, 3, 2, 0]
    assert y[0, 4, 0, 0] == x[0, 0, 5, 0]  # wraps in both directions


def test_conv_adjoints():
    B, H, W, ci, co = 2, 6, 10, 4, 3
    x = rng.normal(size=(B, H, W, ci))
    dy = rng.normal(size=(B, H, W, co))
    Wt = rng.normal(size=(9, co, ci))
    lhs = np.sum(N.conv(x, Wt) * dy)
    assert abs(lhs - np.sum(x * N.conv_bwd_data(dy, Wt))) < 1e-10 * abs(lhs)
    assert abs(lhs - np.sum(Wt * N.conv_bwd_weight(x, dy))) < 1e-10 * abs(lhs)


def test_pool_up_s2d_adjoints():
    x = rng.normal(size=(2, 8, 12, 3))
    g = rng.normal(size=(2, 4, 6, 3))
    assert abs(np.sum(N.pool(x) * g) - np.sum(x * N.pool_bwd(g))) < 1e-12
    assert abs(np.sum(N.up(g) * x) - np.sum(g * N.up_bwd(x))) < 1e-12
    phi = rng.normal(size=(2, 8, 12))
    assert np.array_equal(N.d2s(N.s2d(phi)), phi)
    assert N.s2d(phi)[1, 1, 2, 4 * 1 + 3] == phi[1, 5, 11]
    assert N.pool(np.ones((1, 4, 4, 1)))[0, 1, 1, 0] == 1.0


def test_silu_values_and_derivative():
    assert N.silu(0.0) == 0.0 and N.sigmoid(0.0) == 0.5
    assert abs(N.silu(40.0) - 40.0) < 1e-12 and abs(N.silu(-40.0)) < 1e-15
    z = np.linspace(-6, 6, 25)
    h = 1e-6
    fd = (N.silu(z + h) - N.silu(z - h)) / (2 * h)
    assert np.abs(fd - N.silu_grad(z)).max() < 1e-9


def test_zero_output_layer_is_identity_and_head_conserves_mass():
    theta = rand_theta(1, out_scale=0.0)
    P = N.unpack(theta)
    for name in ("out", "lin", "lina"):  # every term of D
        P[name][0][:] = 0.0
        P[name][1][:] = 0.0
    phi = rng.uniform(-1, 1, size=(2, 64, 64))
    out, _ = N.forward(theta, phi, [0.1, 0.4], 0.1)
    assert np.array_equal(out, phi)
    out, _ = N.forward(rand_theta(2), phi, [0.1, 0.4], 0.1)
    assert np.abs(out - phi).max() > 1e-3
    assert abs(out[0].sum() - phi[0].sum()) < 1e-10 and abs(out[1].sum() - phi[1].sum()) < 1e-10


def test_network_gradient_matches_central_differences():
    theta = rand_theta(3, out_scale=0.5)
    phi = rng.uniform(-1, 1, size=(2, 64, 64))
    target = phi + 0.05 * rng.normal(size=phi.shape)
    alpha = np.array([0.2, 0.45])
    scale = 0.3

    def L(th):
        return N.loss(N.forward(th, phi, alpha, scale)[0], target)[0]

    out, saved = N.forward(theta, phi, alpha, scale)
    _, dout = N.loss(out, target)
    g = N.backward(theta, saved, dout, scale)
    # Parameters from every layer, including biases and the conditioning vector.
    idx, k = [], 0
    for name, ci, co, _, _ in N.LAYERS:
        n_w = 9 * co * ci
        idx += [k + int(rng.integers(n_w)), k + n_w + int(rng.integers(co))]
        k += n_w + co
        if name == "e0a":
            idx.append(k + int(rng.integers(co)))
            k += co
    h = 1e-5
    for i in idx:
        e = np.zeros_like(theta)
        e[i] = h
        fd = (L(theta + e) - L(theta - e)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(abs(fd), 1e-8) + 1e-11, (i, fd, g[i])


def test_pack_unpack_round_trip():
    theta = rand_theta(4)
    assert theta.size == N.param_count()
    assert np.array_equal(N.pack({k: list(v) for k, v in N.unpack(theta).items()}), theta)


def test_adam_first_steps_closed_form():
    # Step 1: m_hat = g, v_hat = g^2, so the update is -lr g / (|g| + eps).
    theta = np.array([1.0, -2.0, 0.5])
    g = np.array([0.3, -4.0, 1e-3])
    lr, eps = 1e-2, 1e-8
    t1, m, v = N.adam(theta, g, np.zeros(3), np.zeros(3), 1, lr, eps=eps)
    assert np.allclose(t1, theta - lr * g / (np.abs(g) + eps), rtol=0, atol=1e-15)
    # Step 2 with g2 = -g1 on one coordinate, by hand:
    # m = 0.9 * 0.1 g - 0.1 g = -0.01 g, m_hat = -0.01 g / 0.19;
    # v = 0.999 * 0.001 g^2 + 0.001 g^2 = 0.001999 g^2, v_hat = g^2 0.001999 / (1 - 0.999^2).
    t2, _, _ = N.adam(t1[:1], -g[:1], m[:1], v[:1], 2, lr, eps=0.0)
    mhat = -0.01 * g[0] / 0.19
    vhat = 0.001999 * g[0] ** 2 / (1 - 0.999 ** 2)
    assert abs(t2[0] - (t1[0] - lr * mhat / np.sqrt(vhat))) < 1e-15


@pytest.mark.parametrize("H,W", [(64, 64), (32, 96)])
def test_shapes(H, W):
    theta = rand_theta(5)
    out, _ = N.forward(theta, rng.uniform(-1, 1, (1, H, W)), [0.3], 0.1)
    assert out.shape == (1, H, W)


def test_bf16_rounding_is_round_to_nearest_even():
    x = np.array([1.0, 1 + 2 ** -8, 1 + 3 * 2 ** -9, 1 + 3 * 2 ** -8, -(1 + 2 ** -7 + 2 ** -9), 2.0 ** -130])
    want = np.array([1.0, 1.0, 1 + 2 ** -7, 1 + 2 ** -6, -(1 + 2 ** -7), 2.0 ** -130])
    assert np.array_equal(N.bf16(x), want)


def test_weighted_loss_and_gradient():
    r = np.random.default_rng(21)
    out, tgt = r.normal(size=(2, 4, 8)), r.normal(size=(2, 4, 8))
    w = np.array([0.5, 3.0])
    L, g = N.loss(out, tgt, w)
    sse = ((out - tgt) ** 2).sum(axis=(1, 2))
    assert abs(L - (w[0] * sse[0] + w[1] * sse[1]) / out.size) < 1e-14
    assert N.loss(out, tgt)[0] == N.loss(out, tgt, [1.0, 1.0])[0]
    e = np.zeros_like(out)
    e[1, 2, 3] = 1e-6
    fd = (N.loss(out + e, tgt, w)[0] - N.loss(out - e, tgt, w)[0]) / 2e-6
    assert abs(fd - g[1, 2, 3]) < 1e-8


def test_global_norm_clipping():
    # Above the threshold the clipped gradient keeps its direction and has norm max_norm;
    # at or below it, or with max_norm 0, the gradient is unchanged. An element-wise clip or
    # a division by the squared norm fails the norm and direction checks.
    r = np.random.default_rng(31)
    g = r.normal(size=1000) * np.exp(r.normal(size=1000))
    nrm = np.sqrt(np.sum(g * g))
    c = N.clip_global_norm(g, 0.25 * nrm)
    assert abs(np.sqrt(np.sum(c * c)) - 0.25 * nrm) < 1e-12 * nrm
    assert abs(np.dot(c, g) / (np.linalg.norm(c) * np.linalg.norm(g)) - 1.0) < 1e-12
    assert np.allclose(c, 0.25 * g, rtol=1e-13, atol=0)
    assert np.array_equal(N.clip_global_norm(g, 2.0 * nrm), g)
    assert np.array_equal(N.clip_global_norm(g, 0.0), g)
    # a gradient with one huge entry: every entry shrinks by the same factor
    h = np.ones(100)
    h[7] = 1e6
    ch = N.clip_global_norm(h, 1.0)
    assert abs(ch[7] / ch[0] - 1e6) < 1e-3 and abs(np.linalg.norm(ch) - 1.0) < 1e-12
