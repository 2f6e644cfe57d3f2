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

def _measured_rate(p, mx, my, phi0, T=400):
    n = p.nx
    # Small enough to stay linear (the next order is ~A^2 relative), large enough that
    # |grad phi|^2 stays above the n = 0 guard (1e-12) at every node, since a guarded
    # node drops gamma(n) from the rate.
    A = 1e-3
    f = oracle.init(p, W.cosine_mode(n, n, mx, my, A, phi0))
    y, x = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    m = max(abs(mx), abs(my))
    z = np.exp(-1j * (2 * np.pi * (mx * x / n + my * y / n) + np.pi * m / n))

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
