"""Pins of the FP64 oracle against things other than itself.

Each test checks the oracle against what the paper prints (golden fixtures of
Eqs. 20, 23, 39), exact identities it states (Eq. 27, Eq. 34), closed forms
derived from its continuum equations (Eqs. 5, 10, 13, 15, 16, 38, 40), lattice
symmetries of Eq. 6 and Eq. 20, textbook special cases (single relaxation time),
or a second, separately written NumPy route.
"""
import math

import numpy as np
import pytest

import golden_io
import numpy_route
import oracle
import workloads as W

C, WT = golden_io.lattice()
MMAT = golden_io.moment_matrix()
EQ39 = golden_io.parameters()


def P(nx, ny, **kw):
    base = dict(M=EQ39["M"], sigma=EQ39["sigma"], D=EQ39["D"], eps=EQ39["eps"])
    base.update(kw)
    return oracle.Params(nx, ny, **base)


# ---------------------------------------------------------------- tables (Eqs. 20, 23, 39)

def test_lattice_tables_match_eq20():
    # f^eq(phi=0, mu_alpha=1) returns w_i for i >= 1 (Eq. 18); F(g=(1,0)) = -w_i c_ix (Eq. 19).
    feq = oracle.equilibrium(0.0, 1.0)
    assert np.array_equal(feq[1:], WT[1:])
    assert feq[0] == WT[0] - 1.0
    for axis in range(2):
        g = [0.0, 0.0]
        g[axis] = 1.0
        F = oracle.source(*g)
        assert np.array_equal(F, -WT * C[:, axis])


def test_moment_matrix_matches_eq23():
    M, _ = oracle.matrices()
    assert np.array_equal(M, MMAT)


def test_parameters_eq5_inversion():
    d = oracle.derive(P(8, 8))
    k, beta = d["k"], d["beta"]
    # Eq. 5 evaluated forward must give back sigma and D.
    assert math.isclose(4.0 * math.sqrt(2.0 * k * beta) / 3.0, EQ39["sigma"], rel_tol=1e-14)
    assert math.isclose(math.sqrt(2.0 * k / beta), EQ39["D"], rel_tol=1e-14)
    # s_3 = s_5 from M = c_s^2 (1/s - 1/2) (after Eq. 38), c_s^2 = 1/3.
    s35 = d["s"][3]
    assert d["s"][5] == s35
    assert math.isclose((1.0 / 3.0) * (1.0 / s35 - 0.5), EQ39["M"], rel_tol=1e-14)
    assert math.isclose(s35, 1.25, rel_tol=1e-15)


# ---------------------------------------------------------------- P1: Eq. 27 moment constraints

def test_lattice_moments_eq27a():
    assert math.isclose(WT.sum(), 1.0, abs_tol=1e-16)
    assert np.allclose(WT @ C, 0.0, atol=0)
    assert np.allclose(np.einsum("i,ia,ib->ab", WT, C, C), np.eye(2) / 3.0, atol=1e-16)


@pytest.mark.parametrize("seed", range(5))
def test_equilibrium_and_source_moments_eq27bc(seed):
    rng = np.random.default_rng(seed)
    phi, mua, gx, gy = rng.uniform(-1.5, 1.5, 4)
    feq = oracle.equilibrium(phi, mua)
    F = oracle.source(gx, gy)
    tol = 1e-15
    assert abs(feq.sum() - phi) <= tol * 4
    assert np.abs(feq @ C).max() <= tol
    assert np.abs(np.einsum("i,ia,ib->ab", feq, C, C) - mua * np.eye(2) / 3.0).max() <= tol
    assert abs(F.sum()) <= tol
    assert np.abs(F @ C - (-np.array([gx, gy]) / 3.0)).max() <= tol


# ---------------------------------------------------------------- P2 / P3: M and closed forms

def test_matrix_orthogonal_and_inverse():
    M, Mi = oracle.matrices()
    assert np.array_equal(M @ M.T, np.diag([9, 36, 36, 6, 12, 6, 12, 4, 4]).astype(float))
    assert np.abs(Mi @ M - np.eye(9)).max() <= 1e-15
    # Orthogonal rows: M^-1 = M^T diag(1/|row|^2).
    assert np.abs(Mi - M.T @ np.diag(1.0 / np.array([9, 36, 36, 6, 12, 6, 12, 4, 4]))).max() <= 1e-15


@pytest.mark.parametrize("seed", range(3))
def test_moment_closed_forms(seed):
    """M f^eq and M F in closed form (the forms the CUDA collision uses)."""
    rng = np.random.default_rng(100 + seed)
    phi, mua, gx, gy = rng.uniform(-1.0, 1.0, 4)
    M, _ = oracle.matrices()
    meq = M @ oracle.equilibrium(phi, mua)
    want = np.array([phi, -4 * phi + 2 * mua, 4 * phi - 3 * mua, 0, 0, 0, 0, 0, 0])
    assert np.abs(meq - want).max() <= 1e-15 * 8
    Fm = M @ oracle.source(gx, gy)
    want = np.array([0, 0, 0, -gx / 3, gx / 3, -gy / 3, gy / 3, 0, 0])
    assert np.abs(Fm - want).max() <= 1e-15


# ---------------------------------------------------------------- P6: single-relaxation reduction

@pytest.mark.parametrize("s", [0.6, 1.0, 1.7])
def test_srt_reduction(s):
    p = P(8, 8, s=[s] * 9, flags=oracle.S35_EXPLICIT)
    rng = np.random.default_rng(7)
    f = rng.uniform(-0.2, 0.8, 9)
    phi = f.sum()
    mua, gx, gy = rng.uniform(-0.1, 0.1, 3)
    out = oracle.collide_site(p, f, phi, mua, gx, gy)
    # BGK with forcing: f - s (f - f^eq) + (1 - s/2) F, with Eq. 18 / Eq. 19 from the golden tables.
    feq = WT * mua
    feq[0] = phi + (WT[0] - 1.0) * mua
    F = -WT * (C[:, 0] * gx + C[:, 1] * gy)
    bgk = f - s * (f - feq) + (1.0 - s / 2.0) * F
    assert np.abs(out - bgk).max() <= 1e-14


def test_init_is_equilibrium_of_eq16_mu_alpha():
    """Reading C5: the initial state is f^eq (Eq. 18) of phi0 and mu_alpha = f(phi0) - k lap phi0
    (Eq. 16), the Laplacian that of Eq. 26b. Recomputed here with np.roll from the printed
    Eq. 20 tables and the Eq. 39 parameters through Eq. 5."""
    ny, nx = 9, 11
    phi0 = np.random.default_rng(12).uniform(-0.9, 0.9, (ny, nx))
    f = oracle.init(P(nx, ny, alpha=0.3), phi0)
    beta = 3 * EQ39["sigma"] / (4 * EQ39["D"])
    k = beta * EQ39["D"] ** 2 / 2
    lap = 6 * sum(WT[i] * (np.roll(phi0, shift=(-C[i, 1], -C[i, 0]), axis=(0, 1)) - phi0) for i in range(9))
    mua = 4 * beta * phi0 * (phi0 * phi0 - 1) - k * lap
    want = WT[:, None, None] * mua[None]
    want[0] = phi0 - (1 - WT[0]) * mua
    assert np.abs(f - want).max() <= 1e-15


# ---------------------------------------------------------------- P4 / P5: conservation and energy

def test_mass_conserved_and_energy_decays_droplet():
    p = P(64, 64, alpha=0.3)
    f = oracle.init(p, W.droplet_workload(64))
    m0 = oracle.mass(p, f)
    E = [oracle.energy(p, f)]
    for _ in range(200):
        f = oracle.step(p, f, 10)
        E.append(oracle.energy(p, f))
    assert abs(oracle.mass(p, f) - m0) <= 1e-13 * abs(m0)
    E = np.array(E)
    assert np.all(np.diff(E) <= 1e-12 * np.abs(E[:-1]))
    assert E[-1] < E[0]


def test_energy_decays_isotropic_spinodal_and_two_droplets():
    cases = [
        (P(128, 128, alpha=0.0), W.noise(128, 128, 0.05, 0)),
        (P(64, 64, alpha=0.3), W.noise(64, 64, 1.0, 1)),  # Eq. 42: rand in [-1, 1]
        (P(100, 100, alpha=0.3), W.two_droplets(100, 100, [(28, 35, 40), (9, 70, 70)], 2.5)),
    ]
    for p, phi0 in cases:
        f = oracle.init(p, phi0)
        m0 = oracle.mass(p, f)
        E = [oracle.energy(p, f)]
        for _ in range(100):
            f = oracle.step(p, f, 10)
            E.append(oracle.energy(p, f))
        E = np.array(E)
        assert np.all(np.diff(E) <= 1e-12 * np.abs(E[:-1]))
        assert abs(oracle.mass(p, f) - m0) <= 1e-13 * max(1.0, abs(m0))


def test_energy_anisotropic_spinodal_near_monotone():
    # With alpha > 0 and small-noise spinodal fields the dynamics is not the exact gradient
    # flow of Eq. 7 (Eq. 15 replaces F by k|grad phi|^2/2, exact only at an interface),
    # so the energy may rise slightly between samples; the trend must still be down.
    p = P(128, 128, alpha=0.2)
    f = oracle.init(p, W.noise(128, 128, 0.05, 0))
    E = [oracle.energy(p, f)]
    for _ in range(200):
        f = oracle.step(p, f, 10)
        E.append(oracle.energy(p, f))
    E = np.array(E)
    assert np.all(np.diff(E) <= 1e-4 * np.abs(E[:-1]))
    assert E[-1] < 0.9 * E[0]


# ---------------------------------------------------------------- energy on closed-form fields

def _energy_axis_closed_form(n, ny, m, A, alpha, k, beta, eps):
    q = 2 * np.pi * m / n
    L = 2.0 - 2.0 * np.cos(q)            # minus the Eq. 26b symbol along x
    s1 = np.sin(q)                       # Eq. 26a symbol along x
    # Sums over a period: sin^2, cos^2 -> n/2, cos^4 -> 3n/8, cos^6 -> 5n/16.
    grad2 = A * A * s1 * s1 * n / 2
    Fsum = beta * (3 * A ** 4 * n / 8 - A * A * n + n)
    a1 = (4 * beta - L) * A              # w = a1 cos - 4 beta A^3 cos^3
    a3 = -4 * beta * A ** 3
    w2 = a1 * a1 * n / 2 + 2 * a1 * a3 * 3 * n / 8 + a3 * a3 * 5 * n / 16
    return ny * ((1 + alpha) * (0.5 * k * grad2 + Fsum) + 0.5 * eps * w2)


def _energy_diag_closed_form(n, m, A, alpha, k, beta, eps):
    q = 2 * np.pi * m / n
    s1 = (2.0 / 3.0) * np.sin(q) + (1.0 / 6.0) * np.sin(2 * q)   # Eq. 26a symbol, 45 degrees
    L = -((8.0 / 3.0) * (np.cos(q) - 1) + (1.0 / 3.0) * (np.cos(2 * q) - 1))
    N = n * n
    grad2 = 2 * A * A * s1 * s1 * N / 2
    Fsum = beta * (3 * A ** 4 * N / 8 - A * A * N + N)
    a1 = (4 * beta - L) * A
    a3 = -4 * beta * A ** 3
    w2 = a1 * a1 * N / 2 + 2 * a1 * a3 * 3 * N / 8 + a3 * a3 * 5 * N / 16
    return (1 - alpha) * (0.5 * k * grad2 + Fsum) + 0.5 * eps * w2


@pytest.mark.parametrize("alpha", [0.0, 0.3])
def test_energy_closed_form_cosines(alpha):
    n, ny, m, A = 32, 4, 1, 0.8
    p = P(n, ny, alpha=alpha)
    d = oracle.derive(p)
    phi0 = W.cosine_mode(n, ny, m, 0, A, 0.0)
    f = oracle.init(p, phi0)
    want = _energy_axis_closed_form(n, ny, m, A, alpha, d["k"], d["beta"], EQ39["eps"])
    assert math.isclose(oracle.energy(p, f), want, rel_tol=1e-12)
    p2 = P(n, n, alpha=alpha)
    phi0 = W.cosine_mode(n, n, m, m, A, 0.0)
    f = oracle.init(p2, phi0)
    want = _energy_diag_closed_form(n, m, A, alpha, d["k"], d["beta"], EQ39["eps"])
    assert math.isclose(oracle.energy(p2, f), want, rel_tol=1e-12)


# ---------------------------------------------------------------- P7: isotropic limit

def test_isotropic_limit_mu_beta_zero():
    p = P(32, 32, alpha=0.0, eps=0.0, regularization=oracle.NONE)
    f = oracle.init(p, W.noise(32, 32, 0.5, 3))
    f = oracle.step(p, f, 5)
    fl = oracle.fields(p, f)
    assert np.all(fl["mu_beta"] == 0.0)
    assert np.all(fl["gx"] == 0.0) and np.all(fl["gy"] == 0.0)


def _tanh_deviation(n, D, steps):
    p = P(n, 8, alpha=0.0, eps=0.0, D=D, regularization=oracle.NONE)
    exact = W.planar_bands(n, 8, n / 4, 3 * n / 4, width=D / 2)   # tanh(2x/D), Eq. 40 with Eq. 5
    f = oracle.step(p, oracle.init(p, exact), steps)
    fl = oracle.fields(p, f)
    return np.abs(oracle.phi(p, f) - exact).max(), np.ptp(fl["mu_alpha"])


def test_isotropic_tanh_profile_second_order():
    dev5, spread5 = _tanh_deviation(64, 5.0, 20000)
    dev10, _ = _tanh_deviation(128, 10.0, 20000)
    assert dev5 <= 2e-2
    assert spread5 <= 2e-5            # chemical potential nearly uniform: a stationary profile
    assert dev5 / dev10 >= 3.0        # second order: halving dx/W cuts the error ~4x


# ---------------------------------------------------------------- P8: linear dispersion

def _measured_rate(p, mx, my, phi0, T=400, shift=None):
    n = p.nx
    # Small enough to stay linear (the next order is ~A^2 relative), large enough that
    # |grad phi|^2 stays above the n = 0 guard (1e-12) at every node, since a guarded
    # node drops gamma(n) from the rate.
    A = 1e-3
    if shift is None:
        shift = np.pi * max(abs(mx), abs(my)) / n
    f = oracle.init(p, W.cosine_mode(n, n, mx, my, A, phi0, shift=shift))
    y, x = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    z = np.exp(-1j * (2 * np.pi * (mx * x / n + my * y / n) + shift))

    def amp(g):
        return abs(((oracle.phi(p, g) - phi0) * z).sum())

    f1 = oracle.step(p, f, T)
    f2 = oracle.step(p, f1, T)
    return math.log(amp(f2) / amp(f1)) / T


def _continuum_rate(p, mx, my, phi0):
    """lambda = -M q^2 [gamma(theta)(f'(phi0) + k q^2) + eps (q^2 + f'(phi0))^2].

    Linearising Eq. 10 with mu of Eq. 13 and Q of Eq. 15 about a uniform phi0 with
    f(phi0) = 0; on the lattice axes and diagonals P grad_n gamma = 0.
    """
    d = oracle.derive(p)
    q2 = (2 * np.pi / p.nx) ** 2 * (mx * mx + my * my)
    gam = 1 + p.alpha * np.cos(4 * np.arctan2(my, mx))
    fp = 4 * d["beta"] * (3 * phi0 ** 2 - 1)
    return -p.M * q2 * (gam * (fp + d["k"] * q2) + p.eps * (q2 + fp) ** 2)


@pytest.mark.parametrize("alpha", [0.0, 0.3])
@pytest.mark.parametrize("phi0", [-1.0, 0.0, 1.0])
@pytest.mark.parametrize("mode", [(1, 0), (2, 0), (1, 1)])
def test_linear_dispersion_small_q(alpha, phi0, mode):
    p = P(64, 64, alpha=alpha)
    lam = _measured_rate(p, *mode, phi0)
    want = _continuum_rate(p, *mode, phi0)
    assert abs(lam - want) <= 5e-3 * abs(want)


@pytest.mark.parametrize("alpha,eps", [(0.0, 0.03), (0.3, 0.03), (0.3, 0.1)])
def test_linear_dispersion_regularisation_visible(alpha, eps):
    # At q = 2 pi 4/64 about phi0 = 1 the eps term is 5-15 % of the rate, so a dropped or
    # mis-signed Willmore term fails the 2 % bound; lattice error at this q is about 1 %.
    p = P(64, 64, alpha=alpha, eps=eps)
    lam = _measured_rate(p, 4, 0, 1.0, T=200)
    want = _continuum_rate(p, 4, 0, 1.0)
    assert abs(lam - want) <= 2e-2 * abs(want)
    p0 = P(64, 64, alpha=alpha, eps=0.0)
    assert abs(_continuum_rate(p0, 4, 0, 1.0) - want) > 4e-2 * abs(want)


# ---------------------------------------------------------------- P9 / P10: symmetries

def _rot90(a):
    """Field rotated by +90 degrees about the origin (mod n): a'(x, y) = a(y, -x)."""
    n = a.shape[-1]
    idx = np.arange(n)
    return a[..., (-idx[None, :]) % n, idx[:, None]] if a.ndim == 2 else None


def _rot90_state(f):
    perm = [0, 4, 1, 2, 3, 8, 5, 6, 7]   # new plane j takes rotated old plane perm[j]: 1->2->3->4->1
    return np.stack([_rot90(f[perm[j]]) for j in range(9)])


def _mirror(a):
    n = a.shape[-1]
    return a[..., (-np.arange(n)) % n]


def _mirror_state(f):
    perm = [0, 3, 2, 1, 4, 6, 5, 8, 7]   # 1<->3, 5<->6, 7<->8
    return np.stack([_mirror(f[perm[j]]) for j in range(9)])


def test_rotation_and_mirror_equivariance():
    n = 32
    p = P(n, n, alpha=0.3)
    phi0 = W.noise(n, n, 0.5, 11)
    f0 = oracle.init(p, phi0)
    ref = oracle.step(p, f0, 100)
    # Rotation of the initial state commutes with the step (gamma is 4-fold symmetric).
    rot = oracle.step(p, _rot90_state(f0), 100)
    assert np.abs(rot - _rot90_state(ref)).max() <= 1e-13
    assert np.abs(oracle.init(p, _rot90(phi0)) - _rot90_state(f0)).max() <= 1e-15
    mir = oracle.step(p, _mirror_state(f0), 100)
    assert np.abs(mir - _mirror_state(ref)).max() <= 1e-13


def test_translation_bitwise():
    p = P(24, 20, alpha=0.3)
    phi0 = W.noise(24, 20, 0.5, 4)
    a = oracle.run(p, phi0, 20)
    b = oracle.run(p, np.roll(phi0, (5, 3), axis=(0, 1)), 20)
    assert np.array_equal(np.roll(a, (5, 3), axis=(0, 1)), b)


@pytest.mark.parametrize("c", [-1.0, -0.3, 0.0, 0.7, 1.0])
def test_constant_field_fixed_point(c):
    p = P(16, 12, alpha=0.3)
    f = oracle.init(p, np.full((12, 16), c))
    g = oracle.step(p, f, 50)
    # Every plane stays uniform, bitwise (each node computes the same thing).
    assert all(np.all(g[i] == g[i, 0, 0]) for i in range(9))
    if c in (-1.0, 0.0, 1.0):
        # mu_alpha = f(c) = 0 and f^eq = (c, 0, ..., 0): no rounding anywhere.
        assert np.array_equal(g, f)
    else:
        # sum_i f_i rounds away from c by about an ulp a step (a drift linear in steps,
        # not growth): 50 steps stay within a few ulps per step.
        assert np.abs(g - f).max() <= 50 * 4 * np.finfo(np.float64).eps


# ---------------------------------------------------------------- P11: second route

@pytest.mark.parametrize("shape", [(8, 8), (9, 7), (5, 11)])
@pytest.mark.parametrize("alpha", [0.0, 0.3])
def test_numpy_second_route(shape, alpha):
    nx, ny = shape
    p = P(nx, ny, alpha=alpha)
    phi0 = W.noise(nx, ny, 0.6, 5)
    f = oracle.init(p, phi0)
    g = numpy_route.init(phi0)
    assert np.abs(f - g).max() <= 1e-15
    for _ in range(10):
        g = numpy_route.step(g, alpha=alpha)
    f = oracle.step(p, f, 10)
    assert np.abs(f - g).max() <= 1e-13


# ---------------------------------------------------------------- generic-angle gamma (Eq. 6)

@pytest.mark.parametrize("phi0", [-1.0, 0.0, 1.0])
@pytest.mark.parametrize("mode", [(2, 1), (1, 2)])
def test_linear_dispersion_generic_angle(phi0, mode):
    """The (2, 1) mode on 64^2 sits at theta = atan(1/2), where cos 4 theta = -0.28 lies
    strictly between the axis and diagonal values, so gamma(theta) of Eq. 6 is tested at
    a value the (1, 0), (2, 0) and (1, 1) modes never reach.

    For a plane wave n = +-q/|q| is constant, so P grad_n gamma is gamma'(theta) times the
    unit tangent, a constant vector times q.grad phi; its divergence t.grad (q.grad phi)
    vanishes, on the lattice as well (the Eq. 26a divergence symbol is orthogonal to the
    tangent of the Eq. 26a gradient symbol). The rate is therefore the continuum lambda
    with gamma(theta) alone. A phase shift of pi/64 keeps every node off the gradient's
    zeros (the phase 2 pi (2x + y)/64 + pi/64 is never a multiple of pi).
    """
    p = P(64, 64, alpha=0.3)
    lam = _measured_rate(p, *mode, phi0, shift=np.pi / 64)
    want = _continuum_rate(p, *mode, phi0)
    assert abs(lam - want) <= 5e-3 * abs(want)


# ---------------------------------------------------------------- linear regularisation (Eqs. 8, 12)

def _continuum_rate_linear(p, mx, my, phi0):
    """lambda = -M q^2 [gamma(theta)(f'(phi0) + k q^2) + eps q^4].

    Linearising Eq. 10 with mu of Eq. 12 (G = (lap phi)^2 of Eq. 8, so the regularising
    part of mu is eps lap^2 phi) and Q of Eq. 15 about a uniform phi0 with f(phi0) = 0.
    """
    d = oracle.derive(p)
    q2 = (2 * np.pi / p.nx) ** 2 * (mx * mx + my * my)
    gam = 1 + p.alpha * np.cos(4 * np.arctan2(my, mx))
    fp = 4 * d["beta"] * (3 * phi0 ** 2 - 1)
    return -p.M * q2 * (gam * (fp + d["k"] * q2) + p.eps * q2 * q2)


@pytest.mark.parametrize("phi0", [-1.0, 1.0])
@pytest.mark.parametrize("alpha", [0.0, 0.3])
def test_linear_regularisation_dispersion_small_q(alpha, phi0):
    p = P(64, 64, alpha=alpha, eps=0.1, regularization=oracle.LINEAR)
    for mode in ((1, 0), (2, 0), (1, 1)):
        lam = _measured_rate(p, *mode, phi0)
        assert abs(lam - _continuum_rate_linear(p, *mode, phi0)) <= 5e-3 * abs(lam)


@pytest.mark.parametrize("alpha,eps", [(0.0, 0.1), (0.3, 0.1), (0.3, 0.2)])
def test_linear_regularisation_visible(alpha, eps):
    # At q = 2 pi 4/64 about phi0 = 1 the eps q^4 term is 11-24 % of the rate, so a dropped,
    # doubled or mis-signed Eq. 12 term fails the 3 % bound. Lattice error here: the Eq. 26b
    # symbol squared, (2 - 2 cos q)^2, falls short of q^4 by ~q^2/6 = 2.6 %, on a term that
    # is a fifth of the rate, plus ~1 % elsewhere (measured 0.8-2.0 %).
    p = P(64, 64, alpha=alpha, eps=eps, regularization=oracle.LINEAR)
    lam = _measured_rate(p, 4, 0, 1.0, T=200)
    want = _continuum_rate_linear(p, 4, 0, 1.0)
    assert abs(lam - want) <= 3e-2 * abs(want)
    p0 = P(64, 64, alpha=alpha, eps=0.0, regularization=oracle.LINEAR)
    assert abs(_continuum_rate_linear(p0, 4, 0, 1.0) - want) > 1e-1 * abs(want)


@pytest.mark.parametrize("alpha", [0.0, 0.3])
def test_energy_closed_form_cosines_linear_regularisation(alpha):
    """Eq. 7 with G = (lap phi)^2 (Eq. 8) on cosine fields: with the Eq. 26b symbol -L,
    sum (lap phi)^2 = L^2 A^2 N/2, the other sums as for the Willmore closed form."""
    n, ny, m, A, eps = 32, 4, 1, 0.8, 0.05
    p = P(n, ny, alpha=alpha, eps=eps, regularization=oracle.LINEAR)
    d = oracle.derive(p)
    k, beta = d["k"], d["beta"]
    q = 2 * np.pi * m / n
    L = 2.0 - 2.0 * np.cos(q)
    grad2 = A * A * np.sin(q) ** 2 * n / 2
    Fsum = beta * (3 * A ** 4 * n / 8 - A * A * n + n)
    want = ny * ((1 + alpha) * (0.5 * k * grad2 + Fsum) + 0.5 * eps * L * L * A * A * n / 2)
    f = oracle.init(p, W.cosine_mode(n, ny, m, 0, A, 0.0))
    assert math.isclose(oracle.energy(p, f), want, rel_tol=1e-12)
    p2 = P(n, n, alpha=alpha, eps=eps, regularization=oracle.LINEAR)
    s1 = (2.0 / 3.0) * np.sin(q) + (1.0 / 6.0) * np.sin(2 * q)
    L2 = -((8.0 / 3.0) * (np.cos(q) - 1) + (1.0 / 3.0) * (np.cos(2 * q) - 1))
    N = n * n
    grad2 = 2 * A * A * s1 * s1 * N / 2
    Fsum = beta * (3 * A ** 4 * N / 8 - A * A * N + N)
    want = (1 - alpha) * (0.5 * k * grad2 + Fsum) + 0.5 * eps * L2 * L2 * A * A * N / 2
    f = oracle.init(p2, W.cosine_mode(n, n, m, m, A, 0.0))
    assert math.isclose(oracle.energy(p2, f), want, rel_tol=1e-12)


def test_linear_regularisation_energy_decays():
    # Eq. 12 is the variational derivative of Eq. 7 with Eq. 8, so the droplet's energy
    # (an interface case, where Eq. 15 is exact) must fall.
    p = P(64, 64, alpha=0.3, regularization=oracle.LINEAR)
    f = oracle.init(p, W.droplet_workload(64))
    E = [oracle.energy(p, f)]
    for _ in range(50):
        f = oracle.step(p, f, 10)
        E.append(oracle.energy(p, f))
    E = np.array(E)
    assert np.all(np.diff(E) <= 1e-12 * np.abs(E[:-1]))
    assert E[-1] < E[0]


# ---------------------------------------------------------------- nested mu_beta (reading C2)

def _lattice_symbols(nx, ny):
    """Eq. 26a and 26b in Fourier space, written from the Eq. 20 tables: the gradient of
    e^{i q.x} is i G(q) e^{i q.x} with G = 3 sum_i w_i c_i sin(q.c_i), the Laplacian is
    L(q) e^{i q.x} with L = 6 sum_i w_i (cos(q.c_i) - 1)."""
    qy = 2 * np.pi * np.fft.fftfreq(ny)[:, None]
    qx = 2 * np.pi * np.fft.fftfreq(nx)[None, :]
    ph = [qx * C[i, 0] + qy * C[i, 1] for i in range(9)]
    Gx = 3.0 * sum(WT[i] * C[i, 0] * np.sin(ph[i]) for i in range(9))
    Gy = 3.0 * sum(WT[i] * C[i, 1] * np.sin(ph[i]) for i in range(9))
    L = 6.0 * sum(WT[i] * (np.cos(ph[i]) - 1.0) for i in range(9))
    return Gx, Gy, L


def test_nested_mu_beta_isotropic_cosine_symbol():
    """At alpha = 0 without regularisation the literal mu - mu_alpha of Eq. 16 is
    gamma f - div(k grad phi) - f + k lap phi = k (lap - div grad) phi: with nested Eq. 26a
    stencils, k (L(q) + |G(q)|^2) times a cosine mode, exactly, at any amplitude."""
    n, A = 32, 0.7
    p = P(n, n, alpha=0.0, eps=0.0, regularization=oracle.NONE, flags=oracle.MU_NESTED)
    k = oracle.derive(p)["k"]
    for mx, my in ((1, 0), (3, 0), (2, 2), (3, 1), (5, 2)):
        phi0 = W.cosine_mode(n, n, mx, my, A, 0.0, shift=0.3)
        fl = oracle.fields(p, oracle.init(p, phi0))
        q = 2 * np.pi * np.array([mx, my]) / n
        G2 = sum((3.0 * sum(WT[i] * C[i, a] * np.sin(q @ C[i]) for i in range(9))) ** 2
                 for a in range(2))
        L = 6.0 * sum(WT[i] * (np.cos(q @ C[i]) - 1.0) for i in range(9))
        want = k * (L + G2) * (phi0 - 0.0)
        assert np.abs(fl["mu_beta"] - want).max() <= 1e-14


@pytest.mark.parametrize("alpha,reg", [(0.3, oracle.WILLMORE), (0.45, oracle.NONE)])
def test_nested_minus_split_is_lattice_commutator(alpha, reg):
    """For any field and alpha, Q of Eq. 15 is Qt + k grad phi, so the literal Eq. 16
    difference (nested) exceeds the split form by k (lap phi - div grad phi) exactly; the
    test forms that from Fourier symbols of Eqs. 26a/26b (a second route)."""
    n = 24
    phi0 = W.noise(n, n, 0.6, 21)
    ps = P(n, n, alpha=alpha, regularization=reg)
    pn = P(n, n, alpha=alpha, regularization=reg, flags=oracle.MU_NESTED)
    f = oracle.init(ps, phi0)
    f = oracle.step(ps, f, 3)
    d = oracle.fields(pn, f)["mu_beta"] - oracle.fields(ps, f)["mu_beta"]
    Gx, Gy, L = _lattice_symbols(n, n)
    k = oracle.derive(ps)["k"]
    phi = oracle.phi(ps, f)
    want = np.real(np.fft.ifft2(k * (L + Gx * Gx + Gy * Gy) * np.fft.fft2(phi)))
    assert np.abs(d - want).max() <= 1e-14


# ---------------------------------------------------------------- tangential term on a curved interface

def _curved_mu_beta_error(scale, literal):
    """Largest |mu_beta(oracle) - mu_beta(continuum)| within one width of a circular
    interface phi = tanh((R - r)/W), R = 16 s, W = 3 s on a (64 s)^2 grid, and the largest
    |mu_beta| there (alpha = 0.3, no regularisation).

    Continuum, from Eqs. 2, 6, 15, 16 in polar coordinates (r, t) about the centre: n =
    -r_hat, so theta = t + pi and gamma = 1 + alpha cos 4t; the tangential term is
    c |phi'| gamma'(theta) times the unit tangent dn/dtheta = -t_hat, whose divergence is
    -c |phi'| gamma''(theta)/r with gamma'' = -16 alpha cos 4t (c = k, or 1 as printed).
    The isotropic part (gamma - 1) k phi'(r) r_hat has divergence
    alpha cos 4t k (phi'' + phi'/r). So
        mu_beta = alpha cos 4t [f(phi) - k (phi'' + phi'/r) - 16 c |phi'|/r],
    whose curvature terms are k|phi'|(gamma + gamma'' - 1)/r at c = k: the interface
    stiffness gamma + gamma'' less the isotropic part that mu_alpha carries.
    """
    N, R, Wd, alpha = 64 * scale, 16.0 * scale, 3.0 * scale, 0.3
    p = P(N, N, alpha=alpha, eps=0.0, regularization=oracle.NONE,
          flags=oracle.Q_LITERAL if literal else 0)
    d = oracle.derive(p)
    k, beta = d["k"], d["beta"]
    y, x = np.meshgrid(np.arange(N, dtype=float), np.arange(N, dtype=float), indexing="ij")
    r = np.hypot(x - N / 2, y - N / 2)
    t = np.arctan2(y - N / 2, x - N / 2)
    phi0 = W.droplet(N, N, R, Wd)
    mask = np.abs(r - R) <= Wd
    th = np.tanh((R - r[mask]) / Wd)
    dphi = -(1 - th * th) / Wd
    d2phi = -2 * th * (1 - th * th) / Wd ** 2
    c = 1.0 if literal else k
    fphi = 4 * beta * th * (th * th - 1)
    want = alpha * np.cos(4 * t[mask]) * (fphi - k * (d2phi + dphi / r[mask])
                                          - 16 * c * np.abs(dphi) / r[mask])
    got = oracle.fields(p, oracle.init(p, phi0))["mu_beta"][mask]
    return np.abs(got - want).max(), np.abs(want).max()


@pytest.mark.parametrize("literal", [False, True])
def test_tangential_term_curved_interface(literal):
    """Pins the k |grad phi| P grad_n gamma term of Eq. 15 (reading C1, and the literal
    reading without k) off the lattice axes: the oracle's mu_beta converges to the
    continuum value at second order (stencil errors scale as h^2 times the field's
    derivatives, so the error falls ~16x when R and W double)."""
    e2, m2 = _curved_mu_beta_error(2, literal)
    e4, m4 = _curved_mu_beta_error(4, literal)
    assert e4 <= 1e-2 * m4
    assert e2 / e4 >= 12.0


# ---------------------------------------------------------------- the n = 0 guard (reading C3)

def test_guard_fires_only_in_the_bulk():
    """The guard |grad phi|^2 < 1e-12 sets gamma = 1 and drops P grad_n gamma. It must never
    change an interface node. On droplets, two droplets and evolved spinodal fields every
    guarded node is a critical point inside a bulk phase (|phi| >= 0.99, where |f(phi)| is
    at most 1.2e-4, 5 % of its interface peak, so the guard moves mu_beta there by at most
    alpha 1.2e-4), and every node with |phi| < 0.9 has |grad phi|^2 at least 1000 times the
    threshold (measured minimum 2.4e-9, on the 64^2 spinodal field after 1000 steps)."""
    cases = [
        (P(64, 64, alpha=0.3), W.droplet_workload(64), [0, 100, 1000]),
        (P(100, 100, alpha=0.3), W.two_droplets(100, 100, [(28, 35, 40), (9, 70, 70)], 2.5),
         [0, 200]),
        (P(64, 64, alpha=0.2), W.noise(64, 64, 0.05, 0), [0, 1000]),
        (P(64, 64, alpha=0.3), W.noise(64, 64, 1.0, 1), [0, 500, 2000]),
    ]
    fired = 0
    for p, phi0, times in cases:
        f = oracle.init(p, phi0)
        t0 = 0
        for t in times:
            f = oracle.step(p, f, t - t0)
            t0 = t
            fl = oracle.fields(p, f)
            g2 = fl["dphi_x"] ** 2 + fl["dphi_y"] ** 2
            # With alpha > 0 an unguarded node has gamma = 1 + alpha cos 4 theta, which is
            # exactly 1 only at theta = 22.5 deg + k 45 deg; the guard sets it to 1.
            guarded = fl["gamma"] == 1.0
            fired += int(guarded.sum())
            assert np.all(guarded[g2 < 1e-12])
            assert np.all(np.abs(fl["phi"][guarded]) >= 0.99)
            interface = np.abs(fl["phi"]) < 0.9
            assert np.all(g2[interface] >= 1e-9)
    assert fired > 0   # the droplet cases do reach the guard (centre and far field)
