"""Parity of the CUDA path (through the C-ABI) with the FP64 oracle.

FP32 state: max |dphi| <= 1e-6 after 1 step and <= 1e-4 after 1000 steps on the
64x64 droplet workload; the same 1e-6 bound for up to 10 steps on every other
shape. Energies agree to 1e-5 relative; FP32 mass drifts by at most 1e-6
relative over 2000 steps.
"""
import numpy as np
import pytest

import oracle
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2501_03759_gb300 import lbch  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    lbch.load()


def solver(nx, ny, **kw):
    return lbch.Solver(lbch.make_params(nx, ny, **kw))


def oparams(nx, ny, **kw):
    kw.pop("storage", None)
    return oracle.Params(nx, ny, **kw)


def both(nx, ny, phi0, checkpoints, **kw):
    """phi from the GPU and from the oracle at each checkpoint (cumulative steps)."""
    s = solver(nx, ny, **kw)
    s.init_field(phi0)
    p = oparams(nx, ny, **kw)
    f = oracle.init(p, phi0)
    out, done = [], 0
    for t in checkpoints:
        s.step(t - done)
        f = oracle.step(p, f, t - done)
        done = t
        out.append((t, s.field(), oracle.phi(p, f), s, p, f))
    return out


def test_droplet_64_parity_over_time():
    phi0 = W.droplet_workload(64)
    bounds = {1: 1e-6, 10: 1e-6, 100: 1e-5, 1000: 1e-4, 2000: 1e-4}
    res = both(64, 64, phi0, list(bounds), alpha=0.3)
    for t, g, r, *_ in res:
        err = np.abs(g - r).max()
        print(f"droplet 64 alpha=0.3 step {t}: max|dphi| = {err:.3e}")
        assert err <= bounds[t], (t, err)


@pytest.mark.parametrize("shape", [(8, 8), (9, 7), (13, 11), (4, 4), (1, 5), (7, 1), (100, 100),
                                   (130, 67), (250, 33), (124, 9), (241, 19), (256, 40)])
@pytest.mark.parametrize("alpha", [0.0, 0.3])
def test_shapes_parity(shape, alpha):
    nx, ny = shape
    phi0 = W.noise(nx, ny, 0.6, 7)
    for t, g, r, *_ in both(nx, ny, phi0, [1, 10], alpha=alpha):
        err = np.abs(g - r).max()
        assert err <= 1e-6, (shape, t, err)


def test_spinodal_256_parity():
    phi0 = W.noise(256, 256, 0.05, 0)
    for t, g, r, *_ in both(256, 256, phi0, [1, 200], alpha=0.2):
        err = np.abs(g - r).max()
        print(f"spinodal 256 alpha=0.2 step {t}: max|dphi| = {err:.3e}")
        assert err <= (1e-6 if t == 1 else 1e-5), (t, err)


@pytest.mark.parametrize("variant", [
    dict(flags=lbch.MU_NESTED), dict(flags=lbch.Q_LITERAL), dict(regularization=lbch.REG_LINEAR),
    dict(regularization=lbch.REG_NONE), dict(eps=0.1),
    dict(s=[1.0, 0.8, 1.3, 1.0, 1.6, 1.0, 0.7, 1.1, 1.5]),
    dict(s=[1.0, 1.2, 1.2, 0.9, 1.2, 0.9, 1.2, 1.2, 1.2], flags=lbch.S35_EXPLICIT),
])
def test_variant_parity(variant):
    kw = dict(alpha=0.3)
    kw.update(variant)
    oflags = kw.get("flags", 0)
    phi0 = W.noise(64, 48, 0.5, 3)
    s = solver(64, 48, **kw)
    s.init_field(phi0)
    okw = dict(kw)
    okw["flags"] = oflags  # same bit values in both APIs
    p = oparams(64, 48, **okw)
    f = oracle.init(p, phi0)
    s.step(10)
    f = oracle.step(p, f, 10)
    err = np.abs(s.field() - oracle.phi(p, f)).max()
    assert err <= 1e-6, (variant, err)


def test_state_matches_oracle_populations():
    phi0 = W.droplet_workload(64)
    s = solver(64, 64, alpha=0.3)
    s.init_field(phi0)
    p = oparams(64, 64, alpha=0.3)
    f = oracle.init(p, phi0)
    # Initial populations differ by their FP32 rounding only.
    assert np.all(np.abs(s.state() - f) <= np.abs(f) * 2.0 ** -24 + 1e-30)
    s.step(5)
    f = oracle.step(p, f, 5)
    assert np.abs(s.state() - f).max() <= 1e-6


def test_checkpoint_resume_bitwise_f32():
    phi0 = W.noise(96, 64, 0.5, 9)
    a = solver(96, 64, alpha=0.3)
    a.init_field(phi0)
    a.step(13)
    ckpt = a.state()
    a.step(17)
    b = solver(96, 64, alpha=0.3)
    b.set_state(ckpt)
    b.step(17)
    assert np.array_equal(a.field(), b.field())
    assert np.array_equal(a.state(), b.state())


def test_mass_and_energy():
    phi0 = W.droplet_workload(64)
    s = solver(64, 64, alpha=0.3)
    s.init_field(phi0)
    p = oparams(64, 64, alpha=0.3)
    f = oracle.init(p, phi0)
    m0 = s.mass()
    # The GPU sums FP32-rounded populations (in FP64): at most 2^-24 |f| per population.
    assert abs(m0 - oracle.mass(p, f)) <= np.abs(f).sum() * 2.0 ** -24
    done = 0
    for t in (0, 10, 100, 1000, 2000):
        s.step(t - done)
        f = oracle.step(p, f, t - done)
        done = t
        e, e_ref = s.free_energy(), oracle.energy(p, f)
        print(f"step {t}: energy {e:.10f} oracle {e_ref:.10f}")
        assert abs(e - e_ref) <= 1e-5 * abs(e_ref), (t, e, e_ref)
    assert abs(s.mass() - m0) <= 1e-6 * abs(m0)


def test_energy_non_increasing_on_gpu():
    s = solver(64, 64, alpha=0.3)
    s.init_field(W.droplet_workload(64))
    E = [s.free_energy()]
    for _ in range(100):
        s.step(10)
        E.append(s.free_energy())
    E = np.array(E)
    assert np.all(np.diff(E) <= 1e-6 * np.abs(E[:-1]))


# The 16-bit storages on the spinodal amplitude U[-0.05, 0.05]: a regression guard set at
# the measured maxima with a ~2x margin (not a derived bound; see DEV_ROUGH_TOL below).
FULL_SIZE_TOL = {lbch.STORE_F32: 1e-6, lbch.STORE_BF16_DEV: 5e-5, lbch.STORE_F16_DEV: 8e-6}


@pytest.mark.parametrize("storage", [lbch.STORE_F32, lbch.STORE_BF16_DEV, lbch.STORE_F16_DEV])
def test_full_size_8192_sampled_windows(storage):
    """The 8192x8192 spinodal workload, in the launch shape the benchmark times (69 strips
    x 17 row segments for FP32, 12 warps/SM for the 16-bit storages), after 5 steps, on
    windows at the corners, the periodic seams, segment boundaries and random places,
    against the oracle on the same windows (exact: padded by the 5-step footprint)."""
    n, steps, wsz = 8192, 5, 24
    phi0 = W.noise(n, n, 0.05, 0)
    s = solver(n, n, alpha=0.3, storage=storage)
    s.init_field(phi0)
    s.step(steps)
    g = s.field()
    s.close()
    p = oparams(n, n, alpha=0.3)
    rng = np.random.default_rng(1)
    corners = [(0, 0), (n - wsz, n - wsz), (n - wsz, 0), (0, n - wsz), (4000, 4090), (116, 7000),
               (8160, 470), (3, 3848), (120 * 34 - 12, 482 * 9 - 12)]
    corners += [tuple(v) for v in rng.integers(0, n - wsz, size=(6, 2))]
    worst = 0.0
    for (x0, y0) in corners:
        ref = oracle.run_window(p, phi0, x0, y0, wsz, wsz, steps)
        worst = max(worst, np.abs(g[y0:y0 + wsz, x0:x0 + wsz] - ref).max())
    name = {lbch.STORE_F32: "f32"}.get(storage) or DEV_NAME[storage]
    print(f"{name} 8192^2 sampled windows after {steps} steps: max|dphi| = {worst:.3e}")
    assert worst <= FULL_SIZE_TOL[storage]
    assert np.isfinite(g).all()


# The 256^2 spinodal workload (alpha = 0.2, U[-0.05, 0.05]) at 1000 steps. FP32: the 1e-4
# bound of the FP32 state (measured 1.8e-8). 16-bit storages: the measured 1.1e-6 (BF16) and
# 1.8e-7 (FP16) with a ~2.7x margin (a regression guard, reported).
SPINODAL_1000_TOL = {lbch.STORE_F32: 1e-4, lbch.STORE_BF16_DEV: 3e-6, lbch.STORE_F16_DEV: 5e-7}


@pytest.mark.parametrize("storage", [lbch.STORE_F32, lbch.STORE_BF16_DEV, lbch.STORE_F16_DEV])
def test_spinodal_256_1000_steps_and_energy_law(storage):
    """The 256^2 spinodal run, 1000 steps, against the oracle; mass conserved; the energy
    sampled every 100 steps follows the small-noise alpha > 0 gate (rises between samples of
    at most 1e-4 relative, since Eq. 15 is exact only at an interface, and a falling trend)."""
    n = 256
    phi0 = W.noise(n, n, 0.05, 0)
    s = solver(n, n, alpha=0.2, storage=storage)
    s.init_field(phi0)
    m0 = s.mass()
    E = [s.free_energy()]
    for _ in range(10):
        s.step(100)
        E.append(s.free_energy())
    p = oparams(n, n, alpha=0.2)
    f = oracle.step(p, oracle.init(p, phi0), 1000)
    err = np.abs(s.field() - oracle.phi(p, f)).max()
    drift = abs(s.mass() - m0) / n / n
    name = {lbch.STORE_F32: "f32"}.get(storage) or DEV_NAME[storage]
    print(f"{name} spinodal 256 alpha=0.2 step 1000: max|dphi| = {err:.3e}, mass drift/node {drift:.2e}")
    assert err <= SPINODAL_1000_TOL[storage]
    assert drift <= 1e-8
    E = np.array(E)
    assert np.all(np.diff(E) <= 1e-4 * np.abs(E[:-1]))
    assert E[-1] < E[0]
    assert abs(E[-1] - oracle.energy(p, f)) <= 1e-5 * abs(E[-1])
    s.close()


@pytest.mark.parametrize("alpha", [0.0, 0.3])
def test_two_droplets_eq41_parity_and_energy(alpha):
    """Two droplets of Eq. 41 on 100^2 (radii 28 and 9, profile tanh(2(R - r)/D), D = 5),
    isotropic and alpha = 0.3 (the paper's two-droplet cases of Section 4): phi against the
    oracle at 1, 100 and 1000 steps within the FP32 bounds, energy non-increasing every 10
    steps (1e-6 relative: an interface case, where the dynamics is the gradient flow)."""
    n = 100
    phi0 = W.two_droplets(n, n, [(28, 35, 40), (9, 70, 70)], 2.5)
    bounds = {1: 1e-6, 100: 1e-5, 1000: 1e-4}
    for t, g, r, *_ in both(n, n, phi0, list(bounds), alpha=alpha):
        err = np.abs(g - r).max()
        print(f"two droplets alpha={alpha} step {t}: max|dphi| = {err:.3e}")
        assert err <= bounds[t], (t, err)
    s = solver(n, n, alpha=alpha)
    s.init_field(phi0)
    E = [s.free_energy()]
    for _ in range(100):
        s.step(10)
        E.append(s.free_energy())
    E = np.array(E)
    assert np.all(np.diff(E) <= 1e-6 * np.abs(E[:-1]))
    assert E[-1] < E[0]
    s.close()


def test_errors_on_gpu():
    s = solver(32, 32, alpha=0.3)
    with pytest.raises(lbch.LbchError) as e:
        s.step(1)
    assert e.value.status == lbch.EINVAL
    bad = W.noise(32, 32, 0.5, 1)
    bad[3, 4] = np.nan
    with pytest.raises(lbch.LbchError) as e:
        s.init_field(bad)
    assert e.value.status == lbch.ENONFINITE
    s.init_field(W.noise(32, 32, 0.5, 1))
    with pytest.raises(lbch.LbchError) as e:
        s.step(-1)
    assert e.value.status == lbch.EINVAL
    st = s.state()
    st[2, 1, 1] = np.inf
    with pytest.raises(lbch.LbchError) as e:
        s.set_state(st)
    assert e.value.status == lbch.ENONFINITE
    s.init_field(W.noise(32, 32, 0.5, 1))
    s.step(3)
    assert s.steps_taken == 3


# 16-bit deviation storage keeps d_i = f*_i - w_i anchor(x + c_i) to a relative 2^-9 (BF16)
# or 2^-12 (FP16, scaled). d_i is about (1/s) w_i c_i . grad mu_alpha, so its rounding grows
# with the roughness of the field: smooth interfaces lose ~1e-6 per step, the deliberately
# rough U[-0.6, 0.6] fields ~1e-4..3e-4 (BF16). Bounds: measured maxima with ~2x margin.
DEV_ROUGH_TOL = {lbch.STORE_BF16_DEV: 5e-4, lbch.STORE_F16_DEV: 8e-5}
DEV_NAME = {lbch.STORE_BF16_DEV: "bf16-dev", lbch.STORE_F16_DEV: "f16-dev"}


@pytest.mark.parametrize("storage", [lbch.STORE_BF16_DEV, lbch.STORE_F16_DEV])
def test_deviation_storage_state_and_resume(storage):
    """The canonical state of 16-bit storage tracks the oracle's populations, and a
    checkpoint taken with get_state resumes close to the uninterrupted run."""
    phi0 = W.noise(96, 64, 0.5, 9)
    a = solver(96, 64, alpha=0.3, storage=storage)
    a.init_field(phi0)
    p = oparams(96, 64, alpha=0.3)
    f = oracle.init(p, phi0)
    assert np.abs(a.state() - f).max() <= 1e-7  # initial deviations are exactly zero
    a.step(13)
    f = oracle.step(p, f, 13)
    err = np.abs(a.state() - f).max()
    print(f"{DEV_NAME[storage]} state after 13 steps (U[-0.5,0.5]): max|df| = {err:.3e}")
    assert err <= DEV_ROUGH_TOL[storage]
    ckpt = a.state()
    a.step(17)
    b = solver(96, 64, alpha=0.3, storage=storage)
    b.set_state(ckpt)
    b.step(17)
    err = np.abs(a.field() - b.field()).max()
    print(f"{DEV_NAME[storage]} resume vs uninterrupted after 17 steps: max|dphi| = {err:.3e}")
    assert err <= DEV_ROUGH_TOL[storage]
    # set_state closes the rest population on phi, so the resumed mass differs only by
    # FP32 rounding of the rest populations (at most 2^-24 |phi| per node).
    assert abs(a.mass() - b.mass()) <= 2.0 ** -24 * np.abs(a.field()).sum() * 2


@pytest.mark.parametrize("storage", [lbch.STORE_BF16_DEV, lbch.STORE_F16_DEV])
@pytest.mark.parametrize("shape", [(130, 67), (9, 7), (256, 40)])
def test_deviation_storage_shapes(storage, shape):
    nx, ny = shape
    rough = W.noise(nx, ny, 0.6, 7)
    for t, g, r, *_ in both(nx, ny, rough, [1, 10], alpha=0.3, storage=storage):
        err = np.abs(g - r).max()
        print(f"{DEV_NAME[storage]} {shape} U[-0.6,0.6] step {t}: max|dphi| = {err:.3e}")
        assert err <= DEV_ROUGH_TOL[storage], (shape, t, err)
    spin = W.noise(nx, ny, 0.05, 7)  # the spinodal workloads' amplitude
    for t, g, r, *_ in both(nx, ny, spin, [1, 10], alpha=0.3, storage=storage):
        err = np.abs(g - r).max()
        print(f"{DEV_NAME[storage]} {shape} U[-0.05,0.05] step {t}: max|dphi| = {err:.3e}")
        assert err <= DEV_ROUGH_TOL[storage] / 10, (shape, t, err)


@pytest.mark.parametrize("storage", [lbch.STORE_BF16_DEV, lbch.STORE_F16_DEV])
def test_deviation_storage_reported(storage):
    """16-bit deviation storage: error against the oracle is reported; gated loosely."""
    phi0 = W.droplet_workload(64)
    res = both(64, 64, phi0, [1, 100, 1000], alpha=0.3, storage=storage)
    name = {lbch.STORE_BF16_DEV: "bf16-dev", lbch.STORE_F16_DEV: "f16-dev"}[storage]
    bounds = {1: 2e-6, 100: 1e-5, 1000: 1e-4}  # regression guard at the FP32 bounds
    for t, g, r, s, p, f in res:
        err = np.abs(g - r).max()
        print(f"{name} droplet 64 step {t}: max|dphi| = {err:.3e}")
        assert err <= bounds[t], (t, err)
    t, g, r, s, p, f = res[-1]
    m0 = oracle.mass(p, f)  # the oracle conserves mass to 1e-13
    drift = abs(s.mass() - m0) / abs(m0)
    print(f"{name} mass drift after 1000 steps: {drift:.3e}")
    assert drift <= 1e-5


@pytest.mark.parametrize("storage", [lbch.STORE_F32, lbch.STORE_BF16_DEV])
@pytest.mark.parametrize("nx,ny", [(64, 64), (66, 50)])
def test_graph_replay_equals_single_launches(storage, nx, ny):
    """Runs of steps replayed from the context's CUDA graph (entered from the odd buffer,
    with a remainder) give the state of the same steps launched one by one, bit for bit."""
    phi0 = W.noise(nx, ny, 0.5, 3)
    a = solver(nx, ny, alpha=0.3, storage=storage)
    b = solver(nx, ny, alpha=0.3, storage=storage)
    a.init_field(phi0)
    b.init_field(phi0)
    a.step(1)
    a.step(57)  # one step back to buffer 0, three graph replays of 16, then 8 single steps
    for _ in range(58):
        b.step(1)
    assert a.steps_taken == b.steps_taken == 58
    assert np.array_equal(a.state(), b.state())
    assert np.array_equal(a.field(), b.field())
