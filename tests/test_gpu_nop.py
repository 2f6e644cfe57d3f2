"""Parity of the learned leap's CUDA path (lbnop_*) with the FP64 oracle
(oracle/nop_oracle.py): the three convolution operators on BF16-exact inputs (FP32
accumulation is the only difference), the whole network forward and backward against the
oracle with the same BF16 storage points, Adam's update, and the leap/LBM alternation
against the same calls made one by one."""
import numpy as np
import pytest

import workloads as W
from oracle import nop_oracle as N

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2501_03759_gb300 import lbch, lbnop  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    lbnop.load()


def dev_bf16(a):
    bits = (np.ascontiguousarray(a, dtype=np.float32).view(np.uint32) >> 16).astype(np.uint16)
    return torch.from_numpy(bits.view(np.int16)).cuda()


def stream():
    return torch.cuda.current_stream().cuda_stream


SHAPES = [(2, 8, 12), (1, 1, 5), (3, 7, 3), (1, 16, 20)]
# Enough pixels (>= 152 x 16 warps of 16) that the kernel keeps every output channel in one
# block instead of slicing them by 16: the path training takes on large batches.
LARGE = (4, 96, 104)
CHANNELS = [(16, 64), (64, 64), (64, 96), (96, 96), (96, 16), (64, 16), (16, 16), (96, 64), (16, 96)]


@pytest.mark.parametrize("ci,co", CHANNELS)
@pytest.mark.parametrize("shape", SHAPES)
def test_conv_forward(ci, co, shape):
    B, H, Wd = shape
    x = W.bf16_exact((B, H, Wd, ci), 1, 1.0)
    w = W.bf16_exact((9, co, ci), 2, 0.25)
    b = W.bf16_exact((co,), 3, 1.0).astype(np.float32)
    y = torch.empty((B, H, Wd, co), dtype=torch.float32, device="cuda")
    xd, wd, bt = dev_bf16(x), dev_bf16(w), torch.from_numpy(b).cuda()  # held until the kernel has run
    lbnop.lbnop_conv3x3(xd.data_ptr(), wd.data_ptr(), bt.data_ptr(), B, H, Wd, ci, co, y.data_ptr(), stream())
    ref = N.conv(x, w, b)
    scale = N.conv(np.abs(x), np.abs(w)).max() + 1.0
    assert np.abs(y.cpu().numpy() - ref).max() <= 2e-7 * 9 * ci * scale / 64 + 1e-6


@pytest.mark.parametrize("ci,co", CHANNELS)
@pytest.mark.parametrize("shape", SHAPES)
def test_conv_bwd_data(ci, co, shape):
    B, H, Wd = shape
    dy = W.bf16_exact((B, H, Wd, co), 4, 1.0)
    w = W.bf16_exact((9, co, ci), 5, 0.25)
    dx = torch.empty((B, H, Wd, ci), dtype=torch.float32, device="cuda")
    dyd, wd = dev_bf16(dy), dev_bf16(w)
    lbnop.lbnop_conv3x3_bwd_data(dyd.data_ptr(), wd.data_ptr(), B, H, Wd, ci, co, dx.data_ptr(), stream())
    ref = N.conv_bwd_data(dy, w)
    scale = N.conv_bwd_data(np.abs(dy), np.abs(w)).max() + 1.0
    assert np.abs(dx.cpu().numpy() - ref).max() <= 1e-6 * scale


@pytest.mark.parametrize("ci,co", CHANNELS)
@pytest.mark.parametrize("shape", SHAPES + [(4, 64, 64)])
def test_conv_bwd_weight(ci, co, shape):
    B, H, Wd = shape
    x = W.bf16_exact((B, H, Wd, ci), 6, 1.0)
    dy = W.bf16_exact((B, H, Wd, co), 7, 1.0)
    dw = torch.empty((9, co, ci), dtype=torch.float32, device="cuda")
    xd, dyd = dev_bf16(x), dev_bf16(dy)
    lbnop.lbnop_conv3x3_bwd_weight(xd.data_ptr(), dyd.data_ptr(), B, H, Wd, ci, co, dw.data_ptr(), stream())
    ref = N.conv_bwd_weight(x, dy)
    scale = N.conv_bwd_weight(np.abs(x), np.abs(dy)).max() + 1.0
    assert np.abs(dw.cpu().numpy() - ref).max() <= 1e-6 * scale


def network_case(B=2, H=64, Wd=64, seed=0):
    theta = W.surrogate_theta(seed, out_scale=0.5)
    r = np.random.default_rng(seed + 100)
    phi = r.uniform(-1, 1, (B, H, Wd)).astype(np.float32).astype(np.float64)
    target = (phi + 0.05 * r.normal(size=phi.shape)).astype(np.float32).astype(np.float64)
    alpha = r.uniform(0.0, 0.5, B)
    return theta, phi, target, alpha


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("shape", [(2, 64, 64), (1, 32, 96), (3, 96, 32)])
def test_network_forward_matches_oracle(shape):
    B, H, Wd = shape
    theta, phi, _, alpha = network_case(B, H, Wd)
    scale = 0.05
    s = lbnop.Surrogate(H, Wd, max_batch=B, scale=scale)
    s.set_params(theta)
    pd = torch.from_numpy(phi.astype(np.float32)).cuda()
    out = s.forward(pd, alpha).cpu().numpy().astype(np.float64)
    ref_q, _ = N.forward(theta, phi, alpha, scale, quantize=N.bf16)
    ref, _ = N.forward(theta, phi, alpha, scale)
    d, dq, d64 = out - phi, ref_q - phi, ref - phi
    e_q, e_64 = rel_l2(d, dq), rel_l2(d, d64)
    print(f"forward {shape}: rel L2 of the update vs oracle with BF16 storage {e_q:.2e}, vs FP64 oracle {e_64:.2e}")
    # Tolerance from the arithmetic: with the same BF16 storage points, FP32 and FP64
    # accumulation alone move the update by up to 3.3e-3 (rel L2) on these and similar cases
    # (a BF16 rounding that flips early propagates); BF16 storage itself moves it by ~5e-3.
    assert e_q <= 1e-2
    assert e_64 <= 2e-2
    # the head conserves mass: sum phi_out = sum phi per field up to FP32 rounding
    for b in range(B):
        assert abs(out[b].sum() - phi[b].sum()) <= 1e-6 * np.abs(phi[b]).sum()
    s.close()


def test_network_backward_matches_oracle():
    B, H, Wd = 2, 64, 64
    theta, phi, target, alpha = network_case(B, H, Wd, seed=1)
    scale = 0.05
    s = lbnop.Surrogate(H, Wd, max_batch=B, scale=scale)
    s.set_params(theta)
    pd, td = torch.from_numpy(phi.astype(np.float32)).cuda(), torch.from_numpy(target.astype(np.float32)).cuda()
    weight = [0.5, 2.0]
    loss = s.backward(pd, alpha, td, weight=weight)
    g = s.grads_host().astype(np.float64)
    out, saved = N.forward(theta, phi, alpha, scale, quantize=N.bf16)
    loss_ref, dout = N.loss(out, target, weight)
    g_ref = N.backward(theta, saved, dout, scale)
    assert abs(loss - loss_ref) <= 1e-4 * loss_ref
    k = 0
    worst = 0.0
    for name, ci, co, _, _ in N.LAYERS:
        n = 9 * co * ci + co + (co if name == "e0a" else 0)
        e = rel_l2(g[k:k + n], g_ref[k:k + n])
        worst = max(worst, e)
        k += n
    print(f"backward: loss {loss:.6e} (oracle {loss_ref:.6e}); worst per-layer gradient rel L2 {worst:.2e}")
    assert worst <= 2e-2  # accumulation order alone moves a layer's gradient by up to ~2e-3
    s.close()


def test_first_adam_step_is_the_closed_form():
    # Adam's first bias-corrected step is -lr g / (|g| + eps) for every parameter.
    B, H, Wd = 1, 32, 32
    theta, phi, target, alpha = network_case(B, H, Wd, seed=2)
    s = lbnop.Surrogate(H, Wd, max_batch=B, scale=0.05)
    s.set_params(theta)
    pd, td = torch.from_numpy(phi.astype(np.float32)).cuda(), torch.from_numpy(target.astype(np.float32)).cuda()
    s.backward(pd, alpha, td)
    g = s.grads_host().astype(np.float64)
    th0 = s.params_host().astype(np.float64)
    lr = 1e-3
    s.adam(lr)
    th1 = s.params_host().astype(np.float64)
    assert np.abs(th1 - (th0 - lr * g / (np.abs(g) + 1e-8))).max() <= 1e-6
    assert np.count_nonzero(g) > 0.99 * g.size
    s.close()


def test_clipped_adam_steps_match_oracle():
    # Two Adam steps: the first unclipped, the second with the gradient clipped to half its
    # global norm (the first step alone is scale-invariant, so the second one shows the clip).
    B, H, Wd = 2, 32, 64
    theta, phi, target, alpha = network_case(B, H, Wd, seed=9)
    s = lbnop.Surrogate(H, Wd, max_batch=B, scale=0.05)
    s.set_params(theta)
    pd, td = torch.from_numpy(phi.astype(np.float32)).cuda(), torch.from_numpy(target.astype(np.float32)).cuda()
    lr = 1e-3
    s.backward(pd, alpha, td)
    g1 = s.grads_host().astype(np.float64)
    assert abs(s.grad_norm() - np.linalg.norm(g1)) <= 1e-9 * np.linalg.norm(g1)
    th0 = s.params_host().astype(np.float64)
    s.adam(lr)
    th1 = s.params_host().astype(np.float64)
    s.backward(pd, alpha, td)
    g2 = s.grads_host().astype(np.float64)
    n2 = s.grad_norm()
    assert abs(n2 - np.linalg.norm(g2)) <= 1e-9 * np.linalg.norm(g2)
    s.set_clip(0.5 * n2)
    s.adam(lr)
    th2 = s.params_host().astype(np.float64)
    r1, m1, v1 = N.adam(th0, g1, np.zeros_like(g1), np.zeros_like(g1), 1, lr)
    assert np.abs(th1 - r1).max() <= 1e-6
    r2, _, _ = N.adam(th1, N.clip_global_norm(g2, 0.5 * n2), m1, v1, 2, lr)
    r2u, _, _ = N.adam(th1, g2, m1, v1, 2, lr)
    err, err_u = np.abs(th2 - r2).max(), np.abs(th2 - r2u).max()
    print(f"clipped Adam: max |theta - oracle| {err:.2e} (unclipped oracle differs by {err_u:.2e})")
    assert err <= 1e-6 and err_u > 10 * err
    with pytest.raises(lbch.LbchError):
        s.set_clip(-1.0)
    with pytest.raises(lbch.LbchError):
        s.set_clip(float("nan"))
    s.close()


def test_training_reduces_the_loss():
    B, H, Wd = 4, 64, 64
    teacher = W.surrogate_theta(7, out_scale=0.5)
    t = lbnop.Surrogate(H, Wd, max_batch=B, scale=0.05)
    t.set_params(teacher)
    r = np.random.default_rng(3)
    phi = torch.from_numpy(r.uniform(-1, 1, (B, H, Wd)).astype(np.float32)).cuda()
    alpha = [0.1, 0.2, 0.3, 0.4]
    target = t.forward(phi, alpha)
    s = lbnop.Surrogate(H, Wd, max_batch=B, scale=0.05)
    s.set_params(W.surrogate_theta(8, out_scale=0.0))
    losses = [s.train_step(phi, alpha, target, 1e-3, want_loss=True) for _ in range(60)]
    print(f"training: loss {losses[0]:.3e} -> {losses[-1]:.3e}")
    assert losses[-1] < 0.5 * losses[0]
    t.close()
    s.close()


def test_device_field_entry_points_match_host_ones():
    n = 64
    phi0 = W.droplet_workload(n).astype(np.float32)
    a = lbch.Solver(lbch.make_params(n, n, alpha=0.3))
    b = lbch.Solver(lbch.make_params(n, n, alpha=0.3))
    a.init_field(phi0.astype(np.float64))
    b.init_field_device(torch.from_numpy(phi0).cuda())
    assert np.array_equal(a.state(), b.state())
    a.step(7)
    ph = a.phi_device()
    assert np.abs(ph.cpu().numpy() - a.field()).max() <= 1e-6
    a.close()
    b.close()


def test_leap_run_equals_the_calls_it_makes():
    n, alpha, cycles, steps = 64, 0.3, 3, 5
    phi0 = W.noise(n, n, 0.05, 5)
    s = lbnop.Surrogate(n, n, max_batch=1, scale=0.05)
    s.set_params(W.surrogate_theta(9, out_scale=0.5))
    a = lbch.Solver(lbch.make_params(n, n, alpha=alpha), stream=s.stream)
    b = lbch.Solver(lbch.make_params(n, n, alpha=alpha), stream=s.stream)
    a.init_field(phi0)
    b.init_field(phi0)
    s.leap_run(a, alpha, cycles, steps)
    for _ in range(cycles):
        phi = b.phi_device()
        b.init_field_device(s.forward(phi.view(1, n, n), [alpha]).view(n, n))
        b.step(steps)
    assert np.array_equal(a.field(), b.field())
    a.close()
    b.close()
    s.close()


def test_invalid_arguments():
    s = lbnop.Surrogate(32, 32, max_batch=2)
    phi = torch.zeros((3, 32, 32), dtype=torch.float32, device="cuda")
    with pytest.raises(lbch.LbchError):
        s.forward(phi, [0.1, 0.2, 0.3])  # batch 3 > max_batch 2
    with pytest.raises(lbch.LbchError):
        s.adam(1e-3)  # no gradient yet
    with pytest.raises(lbch.LbchError):
        s.grad_norm()  # no gradient yet
    bad = W.surrogate_theta(0)
    bad[5] = np.nan
    with pytest.raises(lbch.LbchError):
        s.set_params(bad)
    s.close()


@pytest.mark.parametrize("ci,co", [(16, 96), (96, 96), (96, 64), (64, 96), (64, 64), (96, 16)])
def test_conv_forward_and_data_grad_large_tiles(ci, co):
    B, H, Wd = LARGE
    x = W.bf16_exact((B, H, Wd, ci), 11, 1.0)
    w = W.bf16_exact((9, co, ci), 12, 0.25)
    dy = W.bf16_exact((B, H, Wd, co), 13, 1.0)
    y = torch.empty((B, H, Wd, co), dtype=torch.float32, device="cuda")
    dx = torch.empty((B, H, Wd, ci), dtype=torch.float32, device="cuda")
    xd, wd, dyd = dev_bf16(x), dev_bf16(w), dev_bf16(dy)
    lbnop.lbnop_conv3x3(xd.data_ptr(), wd.data_ptr(), None, B, H, Wd, ci, co, y.data_ptr(), stream())
    lbnop.lbnop_conv3x3_bwd_data(dyd.data_ptr(), wd.data_ptr(), B, H, Wd, ci, co, dx.data_ptr(), stream())
    ref = N.conv(x, w)
    assert np.abs(y.cpu().numpy() - ref).max() <= 1e-6 * (N.conv(np.abs(x), np.abs(w)).max() + 1.0)
    ref = N.conv_bwd_data(dy, w)
    assert np.abs(dx.cpu().numpy() - ref).max() <= 1e-6 * (N.conv_bwd_data(np.abs(dy), np.abs(w)).max() + 1.0)


# Mid-size layers (too many output warps for the per-tap split, too few to keep all channels
# in one block): the channel-sliced path a single 512^2 field takes at level 0.
@pytest.mark.parametrize("ci,co,shape", [(96, 96, (1, 64, 128)), (16, 96, (1, 64, 128)), (64, 64, (1, 96, 128)),
                                         (96, 64, (1, 96, 128))])
def test_conv_forward_mid_tiles(ci, co, shape):
    B, H, Wd = shape
    x = W.bf16_exact((B, H, Wd, ci), 14, 1.0)
    w = W.bf16_exact((9, co, ci), 15, 0.25)
    y = torch.empty((B, H, Wd, co), dtype=torch.float32, device="cuda")
    xd, wd = dev_bf16(x), dev_bf16(w)
    lbnop.lbnop_conv3x3(xd.data_ptr(), wd.data_ptr(), None, B, H, Wd, ci, co, y.data_ptr(), stream())
    ref = N.conv(x, w)
    assert np.abs(y.cpu().numpy() - ref).max() <= 1e-6 * (N.conv(np.abs(x), np.abs(w)).max() + 1.0)


def test_network_backward_large_batch_matches_oracle():
    # Large enough (level 0: 4 x 104 x 104 pixels) that the convolutions and their data
    # gradients keep every output channel in one block, as training does.
    B, H, Wd = 4, 416, 416
    theta, phi, target, alpha = network_case(B, H, Wd, seed=5)
    scale = 0.05
    s = lbnop.Surrogate(H, Wd, max_batch=B, scale=scale)
    s.set_params(theta)
    pd, td = torch.from_numpy(phi.astype(np.float32)).cuda(), torch.from_numpy(target.astype(np.float32)).cuda()
    loss = s.backward(pd, alpha, td)
    g = s.grads_host().astype(np.float64)
    out, saved = N.forward(theta, phi, alpha, scale, quantize=N.bf16)
    loss_ref, dout = N.loss(out, target)
    g_ref = N.backward(theta, saved, dout, scale)
    assert abs(loss - loss_ref) <= 1e-4 * loss_ref
    k, worst = 0, 0.0
    for name, ci, co, _, _ in N.LAYERS:
        n = 9 * co * ci + co + (co if name == "e0a" else 0)
        worst = max(worst, rel_l2(g[k:k + n], g_ref[k:k + n]))
        k += n
    print(f"backward large: worst per-layer gradient rel L2 {worst:.2e}")
    assert worst <= 2e-2
    s.close()


def test_leap_turns_average_the_turned_predictions():
    """With 4 turns a leap is the mean of the network's predictions on the field turned by 0,
    90, 180 and 270 degrees, each turned back (torch.rot90 as the independent route); mass
    is conserved, and the result is exactly equivariant under a quarter turn of the input."""
    n, alpha = 64, 0.3
    s = lbnop.Surrogate(n, n, max_batch=4, scale=0.05)
    s.set_params(W.surrogate_theta(9, out_scale=0.5))
    s.set_leap_turns(4)
    a = lbch.Solver(lbch.make_params(n, n, alpha=alpha), stream=s.stream)
    phi0 = W.noise(n, n, 0.05, 5)
    a.init_field(phi0)
    phi = a.phi_device()
    s.leap_run(a, alpha, 1, 0)
    got = a.phi_device().cpu().numpy()
    xs = torch.stack([torch.rot90(phi, k, (0, 1)) for k in range(4)]).contiguous()
    ys = s.forward(xs, [alpha] * 4)
    want = sum(torch.rot90(ys[k], -k, (0, 1)) for k in range(4)).cpu().numpy() * 0.25
    assert np.abs(got - want).max() <= 1e-6 * np.abs(want).max()
    assert abs(got.astype(np.float64).sum() - phi0.sum()) <= 1e-6 * np.abs(phi0).sum()
    # equivariance: leaping the turned field gives the turned leap (each prediction of the four
    # turns is one of the four of the original, so only the order of the sum differs)
    b = lbch.Solver(lbch.make_params(n, n, alpha=alpha), stream=s.stream)
    b.init_field(np.rot90(phi0).copy())
    s.leap_run(b, alpha, 1, 0)
    assert np.abs(b.phi_device().cpu().numpy() - np.rot90(got)).max() <= 1e-6 * np.abs(want).max()
    for o in (a, b, s):
        o.close()


# ---------------------------------------------------------------- the tcgen05 tensor-core path

# Rows of 128 pixels (or a multiple) with H a multiple of 4 take the tcgen05 path: input rows
# staged by cp.async, whole weight taps by bulk copies from a packed copy of the weights, FP32
# accumulators in tensor memory. The shapes cover 1, 2 and 4 output rows
# per CTA (few, some and many rows), both ends of a row (periodic wrap in x) and of the field
# (wrap in y), and rows of 256 pixels (two tiles per row).
TC_SHAPES = [(1, 4, 128), (2, 8, 256), (3, 12, 128), (10, 128, 128)]


@pytest.mark.parametrize("ci,co", [(96, 96), (96, 64), (64, 96), (64, 64), (96, 16), (16, 96), (16, 16), (64, 16)])
@pytest.mark.parametrize("shape", TC_SHAPES)
def test_conv_tc_forward(ci, co, shape):
    B, H, Wd = shape
    x = W.bf16_exact((B, H, Wd, ci), 21, 1.0)
    w = W.bf16_exact((9, co, ci), 22, 0.25)
    b = W.bf16_exact((co,), 23, 1.0).astype(np.float32)
    y = torch.empty((B, H, Wd, co), dtype=torch.float32, device="cuda")
    xd, wd, bt = dev_bf16(x), dev_bf16(w), torch.from_numpy(b).cuda()
    pk = torch.empty(lbnop.lbnop_conv3x3_packed_bytes(ci, co), dtype=torch.uint8, device="cuda")
    lbnop.lbnop_conv3x3_pack(wd.data_ptr(), ci, co, pk.data_ptr(), stream())
    before = lbnop.lbnop_tc_launches()
    lbnop.lbnop_conv3x3_packed(xd.data_ptr(), wd.data_ptr(), pk.data_ptr(), bt.data_ptr(), B, H, Wd, ci, co,
                               y.data_ptr(), stream())
    torch.cuda.synchronize()
    assert lbnop.lbnop_tc_launches() == before + 1  # the tensor-core path ran
    assert lbnop.lbnop_tc_fault() == 0  # and no bounded wait gave up
    ref = N.conv(x, w, b)
    scale = N.conv(np.abs(x), np.abs(w)).max() + 1.0
    assert np.abs(y.cpu().numpy() - ref).max() <= 2e-7 * 9 * ci * scale / 64 + 1e-6


@pytest.mark.parametrize("ci,co", [(96, 96), (16, 64)])
def test_conv_packed_weights(ci, co):
    """Weights packed once (lbnop_conv3x3_pack) drive the tensor-core path; without a packed
    copy (and through lbnop_conv3x3) the same shape runs on the mma.sync kernels. All agree
    with the oracle's conv."""
    B, H, Wd = 2, 8, 256
    x = W.bf16_exact((B, H, Wd, ci), 31, 1.0)
    w = W.bf16_exact((9, co, ci), 32, 0.25)
    xd, wd = dev_bf16(x), dev_bf16(w)
    nb = lbnop.lbnop_conv3x3_packed_bytes(ci, co)
    assert nb == 9 * (ci // 8) * (co * 16 + 16)
    assert lbnop.lbnop_conv3x3_packed_bytes(32, co) == 0
    pk = torch.empty(nb, dtype=torch.uint8, device="cuda")
    lbnop.lbnop_conv3x3_pack(wd.data_ptr(), ci, co, pk.data_ptr(), stream())
    ref = N.conv(x, w)
    bound = 2e-7 * 9 * ci * (N.conv(np.abs(x), np.abs(w)).max() + 1.0) / 64 + 1e-6
    for packed in (pk.data_ptr(), None):
        y = torch.empty((B, H, Wd, co), dtype=torch.float32, device="cuda")
        before = lbnop.lbnop_tc_launches()
        lbnop.lbnop_conv3x3_packed(xd.data_ptr(), wd.data_ptr(), packed, None, B, H, Wd, ci, co, y.data_ptr(),
                                   stream())
        torch.cuda.synchronize()
        assert lbnop.lbnop_tc_launches() - before == (1 if packed else 0)
        assert np.abs(y.cpu().numpy() - ref).max() <= bound
    y = torch.empty((B, H, Wd, co), dtype=torch.float32, device="cuda")
    before = lbnop.lbnop_tc_launches()
    lbnop.lbnop_conv3x3(xd.data_ptr(), wd.data_ptr(), None, B, H, Wd, ci, co, y.data_ptr(), stream())
    torch.cuda.synchronize()
    assert lbnop.lbnop_tc_launches() == before
    assert np.abs(y.cpu().numpy() - ref).max() <= bound
    # the packed layout itself: tap t, chunk c, output channel n holds w[t][n][8 c .. 8 c + 7]
    raw = pk.cpu().numpy().view(np.uint16).reshape(9, ci // 8, co + 1, 8)
    assert (raw[:, :, co, :] == 0).all()
    wbits = wd.cpu().numpy().view(np.uint16).reshape(9, co, ci // 8, 8)
    assert (raw[:, :, :co, :] == wbits.transpose(0, 2, 1, 3)).all()


# The weight gradient takes the tcgen05 path on rows of 128 pixels (or a multiple); H is free
# (every dz row meets its own sample's rows). Shapes: one row, a few rows across samples, an
# odd H, rows of 256 pixels, and many rows per CTA.
WG_TC_SHAPES = [(1, 1, 128), (3, 5, 128), (2, 8, 256), (10, 128, 128)]


@pytest.mark.parametrize("ci,co", CHANNELS)
@pytest.mark.parametrize("shape", WG_TC_SHAPES)
def test_conv_bwd_weight_tc(ci, co, shape):
    B, H, Wd = shape
    x = W.bf16_exact((B, H, Wd, ci), 26, 1.0)
    dy = W.bf16_exact((B, H, Wd, co), 27, 1.0)
    dw = torch.empty((9, co, ci), dtype=torch.float32, device="cuda")
    xd, dyd = dev_bf16(x), dev_bf16(dy)
    before = lbnop.lbnop_tc_launches()
    lbnop.lbnop_conv3x3_bwd_weight(xd.data_ptr(), dyd.data_ptr(), B, H, Wd, ci, co, dw.data_ptr(), stream())
    torch.cuda.synchronize()
    assert lbnop.lbnop_tc_launches() == before + 1  # the tensor-core path ran
    assert lbnop.lbnop_tc_fault() == 0
    ref = N.conv_bwd_weight(x, dy)
    scale = N.conv_bwd_weight(np.abs(x), np.abs(dy)).max() + 1.0
    assert np.abs(dw.cpu().numpy() - ref).max() <= 1e-6 * scale


def test_network_on_tensor_core_path_matches_oracle():
    """A 512^2 field: its finest level (128 x 128) runs e0a (the input and its BF16 remainder
    as K = 32), e0b, d0a and the output layer, and in the backward pass the data gradients of
    the last three and the weight gradients of all six level-0 layers, on the tcgen05 path;
    forward and gradients against the oracle with the same BF16 storage points, with the bounds
    of the mma.sync path."""
    B, H, Wd = 1, 512, 512
    theta, phi, target, alpha = network_case(B, H, Wd, seed=3)
    scale = 0.05
    s = lbnop.Surrogate(H, Wd, max_batch=B, scale=scale)
    s.set_params(theta)
    pd, td = torch.from_numpy(phi.astype(np.float32)).cuda(), torch.from_numpy(target.astype(np.float32)).cuda()
    before = lbnop.lbnop_tc_launches()
    out = s.forward(pd, alpha).cpu().numpy().astype(np.float64)
    mid = lbnop.lbnop_tc_launches()
    assert mid - before == 4  # e0a, e0b, d0a, out
    loss = s.backward(pd, alpha, td)
    # forward again, the data gradients of out, d0a, e0b, and the weight gradients of the level-0
    # layers (e0a, lin, lina twice: phi's two BF16 halves share their weights)
    assert lbnop.lbnop_tc_launches() - mid == 4 + 3 + 9
    g = s.grads_host().astype(np.float64)
    ref_q, saved = N.forward(theta, phi, alpha, scale, quantize=N.bf16)
    e_q = rel_l2(out - phi, ref_q - phi)
    loss_ref, dout = N.loss(ref_q, target)
    g_ref = N.backward(theta, saved, dout, scale)
    k, worst = 0, 0.0
    for name, ci, co, _, _ in N.LAYERS:
        n = 9 * co * ci + co + (co if name == "e0a" else 0)
        worst = max(worst, rel_l2(g[k:k + n], g_ref[k:k + n]))
        k += n
    print(f"tensor-core network 512^2: update rel L2 {e_q:.2e}, loss {loss:.6e} (oracle {loss_ref:.6e}), "
          f"worst gradient rel L2 {worst:.2e}")
    assert e_q <= 1e-2
    assert abs(loss - loss_ref) <= 1e-4 * loss_ref
    assert worst <= 2e-2
    s.close()


# ---------------------------------------------------------------- the plain scheme as judge and fallback

def _judged_pair(n, alpha, theta, scale, warm=100):
    s = lbnop.Surrogate(n, n, max_batch=1, scale=scale)
    s.set_params(theta)
    a = lbch.Solver(lbch.make_params(n, n, alpha=alpha), stream=s.stream)
    b = lbch.Solver(lbch.make_params(n, n, alpha=alpha), stream=s.stream)
    phi0 = W.noise(n, n, 0.05, 12)
    a.init_field(phi0)
    b.init_field(phi0)
    a.step(warm)
    b.step(warm)
    return s, a, b


def test_judged_leap_rejects_bad_weights_and_equals_plain_scheme():
    """A network of random weights with a large output scale adds noise of the field's own
    size: the free energy (Eq. 7) rises across every leap, the judge rejects each one, and
    the run is then the plain scheme over the same steps, bit for bit."""
    n, alpha, cycles, K, corr = 64, 0.3, 4, 100, 20
    s, a, b = _judged_pair(n, alpha, W.surrogate_theta(3, out_scale=0.5), scale=1.0)
    judge = lbnop.make_judge(leap_steps=K, energy_rtol=1e-6, mass_atol=1e-6)
    st = s.leap_run_judged(a, alpha, cycles, corr, judge)
    b.step(cycles * (K + corr))
    assert st["rejected"] == cycles and st["accepted"] == 0
    assert st["rejected_energy"] == cycles
    assert st["max_leap_rise"] > 1e-3
    assert st["lbm_steps"] == cycles * (K + corr)
    assert a.steps_taken == 100 + cycles * (K + corr)
    assert np.array_equal(a.state(), b.state())
    for o in (a, b, s):
        o.close()


def test_judged_leap_accepts_good_leaps_like_the_unjudged_run():
    """With tolerances no leap can fail (a loose energy bound), every leap is accepted and the
    judged run equals lbnop_leap_run bit for bit: saving the state and reading mass and energy
    change nothing. The step counter keeps the simulated time."""
    n, alpha, cycles, corr = 64, 0.3, 3, 10
    s, a, b = _judged_pair(n, alpha, W.surrogate_theta(9, out_scale=0.5), scale=0.05)
    judge = lbnop.make_judge(leap_steps=500, energy_rtol=1e3, mass_atol=1.0)
    st = s.leap_run_judged(a, alpha, cycles, corr, judge)
    s.leap_run(b, alpha, cycles, corr)
    assert st["accepted"] == cycles and st["rejected"] == 0 and st["audits"] == 0
    assert st["lbm_steps"] == cycles * corr
    assert a.steps_taken == 100 + cycles * (500 + corr)
    assert np.array_equal(a.state(), b.state())
    for o in (a, b, s):
        o.close()


def test_judged_leap_audits_continue_from_the_plain_scheme():
    """audit_every = 1: each cycle runs the plain K steps beside the leap and continues from
    the plain state, so the run is the plain scheme bit for bit; each audit measures the
    leap's phi error (here of random weights, so phi_rtol = 0 rejects every audited leap)."""
    n, alpha, cycles, K, corr = 64, 0.2, 3, 60, 15
    s, a, b = _judged_pair(n, alpha, W.surrogate_theta(5, out_scale=0.5), scale=0.05)
    judge = lbnop.make_judge(leap_steps=K, energy_rtol=1e-6, audit_every=1, phi_rtol=0.0)
    st = s.leap_run_judged(a, alpha, cycles, corr, judge)
    b.step(cycles * (K + corr))
    assert st["audits"] == cycles and st["rejected_audit"] == cycles
    assert 0.0 < st["max_audit_err"] < 1.0
    assert np.array_equal(a.state(), b.state())
    # phi_rtol = 1: the same audits pass
    s2, c, _ = _judged_pair(n, alpha, W.surrogate_theta(5, out_scale=0.5), scale=0.05)
    st2 = s2.leap_run_judged(c, alpha, cycles, corr, lbnop.make_judge(leap_steps=K, audit_every=1, phi_rtol=1.0))
    assert st2["accepted"] == cycles and st2["max_audit_err"] == st["max_audit_err"]
    for o in (a, b, s, c, s2):
        o.close()


@pytest.mark.parametrize("storage", [lbch.STORE_F32, lbch.STORE_BF16_DEV])
def test_device_checkpoint_and_device_diagnostics(storage):
    """lbch_save_state_device / lbch_restore_state_device give back the same continuation bit
    for bit; lbch_mass_device / lbch_free_energy_device equal the synchronous calls."""
    n = 48
    a = lbch.Solver(lbch.make_params(n, n, alpha=0.3, storage=storage))
    a.init_field(W.droplet_workload(n))
    a.step(13)
    img = a.save_state_device()
    a.step(21)
    want = a.state()
    m = torch.zeros(2, dtype=torch.float64, device="cuda")
    a.mass_device(m[0:1])
    a.free_energy_device(m[1:2])
    assert m[0].item() == a.mass() and m[1].item() == a.free_energy()
    # the fused diagnostics of a given field: the energy bit for bit, the mass as the FP64 sum of
    # the FP32 phi (the populations' sum differs by FP32 rounding of phi only)
    d = torch.zeros(2, dtype=torch.float64, device="cuda")
    a.field_diagnostics_device(a.phi_device(), d)
    assert d[1].item() == a.free_energy()
    assert abs(d[0].item() - a.mass()) <= 2.0 ** -23 * np.abs(a.field()).sum()
    a.restore_state_device(img)
    assert a.steps_taken == 34  # restore leaves the counter as it is
    a.step(21)
    assert np.array_equal(a.state(), want)
    with pytest.raises(lbch.LbchError):
        a.restore_state_device(img[:16])
    a.close()
