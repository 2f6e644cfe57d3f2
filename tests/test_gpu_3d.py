"""Parity of the 3D (D3Q15) CUDA path (lbch3_*) with the FP64 3D oracle: max |dphi|
<= 1e-6 after 1 step and <= 1e-5 after 50 on droplets and rough fields of several
shapes, energy within 1e-5 relative, FP32 mass drift <= 1e-6 relative."""
import math

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


def droplet3(nx, ny, nz, radius, width):
    z, y, x = np.meshgrid(np.arange(nz, dtype=float), np.arange(ny, dtype=float), np.arange(nx, dtype=float),
                          indexing="ij")
    r = np.sqrt((x - nx / 2) ** 2 + (y - ny / 2) ** 2 + (z - nz / 2) ** 2)
    return np.tanh((radius - r) / width)


def both3(shape, phi0, checkpoints, **kw):
    nx, ny, nz = shape
    s = lbch.Solver3(lbch.make_params3(nx, ny, nz, **kw))
    s.init_field(phi0)
    p = oracle.Params3(nx, ny, nz, **kw)
    f = oracle.init3(p, phi0)
    out, done = [], 0
    for t in checkpoints:
        s.step(t - done)
        f = oracle.step3(p, f, t - done)
        done = t
        out.append((t, s.field(), oracle.phi3(p, f), {"mass": s.mass(), "energy": s.free_energy()}, p, f))
    return out


def test_droplet_3d_parity():
    phi0 = droplet3(24, 24, 24, 8.0, 2.5)
    bounds = {1: 1e-6, 10: 2e-6, 50: 1e-5}
    for t, g, r, *_ in both3((24, 24, 24), phi0, list(bounds), alpha=0.3):
        err = np.abs(g - r).max()
        print(f"3D droplet 24^3 step {t}: max|dphi| = {err:.3e}")
        assert err <= bounds[t]


@pytest.mark.parametrize("shape", [(13, 11, 9), (16, 8, 4), (5, 7, 3), (32, 12, 10)])
def test_shapes_3d_parity(shape):
    rng = np.random.default_rng(4)
    phi0 = rng.uniform(-0.5, 0.5, shape[::-1])
    for t, g, r, *_ in both3(shape, phi0, [1, 10], alpha=0.4):
        assert np.abs(g - r).max() <= 2e-6, (shape, t)


@pytest.mark.parametrize("variant", [dict(flags=lbch.MU_NESTED), dict(flags=lbch.Q_LITERAL),
                                     dict(regularization=lbch.REG_LINEAR), dict(regularization=lbch.REG_NONE),
                                     dict(s=[1.0, 0.9, 1.2, 1.0, 1.4, 1.0, 0.8, 1.0, 1.1, 1.3, 0.7, 1.2,
                                             1.5, 0.9, 1.6])])
def test_variants_3d_parity(variant):
    rng = np.random.default_rng(6)
    phi0 = rng.uniform(-0.4, 0.4, (8, 10, 12))
    for t, g, r, *_ in both3((12, 10, 8), phi0, [5], alpha=0.3, **variant):
        assert np.abs(g - r).max() <= 2e-6, variant


def test_mass_energy_3d():
    phi0 = droplet3(20, 20, 20, 7.0, 2.5)
    res = both3((20, 20, 20), phi0, [0, 20, 200], alpha=0.3)
    m0 = res[0][3]["mass"]
    for t, g, r, d, p, f in res:
        e, e_ref = d["energy"], oracle.energy3(p, f)
        assert abs(e - e_ref) <= 1e-5 * abs(e_ref), (t, e, e_ref)
        assert abs(d["mass"] - math.fsum(f.ravel())) <= 1e-6 * abs(m0), t
    assert abs(res[-1][3]["mass"] - m0) <= 1e-6 * abs(m0)


def test_paper_droplet_100_cubed():
    """The 3D single-droplet case of Section 4 (Eq. 43): R = 25 on 100^3, alpha = 0.3."""
    n = 100
    phi0 = droplet3(n, n, n, 25.0, 2.5)
    for t, g, r, *_ in both3((n, n, n), phi0, [3], alpha=0.3):
        assert np.abs(g - r).max() <= 1e-6
