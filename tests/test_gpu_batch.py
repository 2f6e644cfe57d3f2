"""Batched stepping (lbch_batch_*): every field of a batch evolves exactly as it does
alone (bitwise, same kernels per node), and small fields match the FP64 oracle."""
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


FIELDS = [  # (nx, ny, alpha, kind)
    (512, 512, 0.41, "droplet"), (64, 64, 0.0, "spinodal"), (128, 96, 0.3, "droplet"),
    (256, 256, 0.12, "spinodal"), (200, 124, 0.5, "spinodal"), (64, 200, 0.25, "droplet"),
    (8, 12, 0.3, "spinodal"), (640, 128, 0.2, "spinodal"),
]


def phi0_of(nx, ny, kind, seed):
    if kind == "droplet":
        return W.droplet(nx, ny, radius=0.3 * min(nx, ny), width=np.sqrt(2.0) * 1.5)
    return W.noise(nx, ny, 0.05, seed)


def run_batch(fields, steps, storage=lbch.STORE_F32, chunks=None):
    common = lbch.make_params(8, 8, storage=storage)
    b = lbch.Batch(common, [f[0] for f in fields], [f[1] for f in fields], [f[2] for f in fields])
    for i, (nx, ny, _, kind) in enumerate(fields):
        b.init_field(i, phi0_of(nx, ny, kind, 100 + i))
    for n in (chunks or [steps]):
        b.step(n)
    return b


def run_single(nx, ny, alpha, kind, seed, steps, storage=lbch.STORE_F32):
    s = lbch.Solver(lbch.make_params(nx, ny, alpha=alpha, storage=storage))
    s.init_field(phi0_of(nx, ny, kind, seed))
    s.step(steps)
    return s


@pytest.mark.parametrize("storage", [lbch.STORE_F32, lbch.STORE_BF16_DEV])
def test_batch_matches_single_fields_bitwise(storage):
    # 131 steps in chunks: plain launches, two replays of the 64-step graph, an odd
    # parity start.
    b = run_batch(FIELDS, 131, storage, chunks=[3, 64, 1, 63])
    assert b.steps_taken == 131
    assert b.rows_target > 0
    for i, (nx, ny, alpha, kind) in enumerate(FIELDS):
        s = run_single(nx, ny, alpha, kind, 100 + i, 131, storage)
        assert np.array_equal(b.field(i), s.field()), (i, nx, ny)
        assert b.mass(i) == s.mass()
        assert b.free_energy(i) == s.free_energy()
        s.close()
    b.close()


def test_batch_scalar_path_when_a_width_is_not_multiple_of_4():
    fields = [(9, 7, 0.3, "spinodal"), (64, 64, 0.2, "droplet"), (130, 67, 0.1, "spinodal")]
    b = run_batch(fields, 70)
    for i, (nx, ny, alpha, kind) in enumerate(fields):
        s = run_single(nx, ny, alpha, kind, 100 + i, 70)
        assert np.array_equal(b.field(i), s.field()), i
    b.close()


def test_batch_small_fields_match_oracle():
    fields = [(64, 64, 0.3, "droplet"), (48, 40, 0.45, "spinodal")]
    b = run_batch(fields, 10)
    for i, (nx, ny, alpha, kind) in enumerate(fields):
        ref = oracle.run(oracle.Params(nx, ny, alpha=alpha), phi0_of(nx, ny, kind, 100 + i), 10)
        assert np.abs(b.field(i) - ref).max() <= 1e-6
    b.close()


def test_batch_call_order_errors():
    common = lbch.make_params(8, 8)
    b = lbch.Batch(common, [64, 32], [64, 32], [0.1, 0.2])
    b.init_field(0, W.noise(64, 64, 0.05, 1))
    with pytest.raises(lbch.LbchError) as e:
        b.step(1)  # field 1 not initialised
    assert e.value.status == lbch.EINVAL
    b.init_field(1, W.noise(32, 32, 0.05, 2))
    b.step(1)
    with pytest.raises(lbch.LbchError) as e:
        b.init_field(0, W.noise(64, 64, 0.05, 1))  # odd number of steps taken
    assert e.value.status == lbch.EINVAL
    b.step(1)
    b.init_field(0, W.noise(64, 64, 0.05, 1))
    b.close()


def test_batch_sweep_workload_sample():
    """A 24-field sample of the parameter-sweep workload, 40 steps, against single runs."""
    specs = W.batch_sweep_specs(24, seed=3)
    common = lbch.make_params(8, 8)
    b = lbch.Batch(common, [s["n"] for s in specs], [s["n"] for s in specs], [s["alpha"] for s in specs])
    for i, sp in enumerate(specs):
        b.init_field(i, W.batch_field(sp))
    b.step(40)
    for i in (0, 5, 11, 23):
        sp = specs[i]
        s = lbch.Solver(lbch.make_params(sp["n"], sp["n"], alpha=sp["alpha"]))
        s.init_field(W.batch_field(sp))
        s.step(40)
        assert np.array_equal(b.field(i), s.field())
        s.close()
    b.close()
