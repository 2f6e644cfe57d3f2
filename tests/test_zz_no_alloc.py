"""The allocation-free free-energy entry point, checked against lbch_free_energy.

lbch_free_energy_static exists for callers that cannot allocate device memory (all
of their memory comes from a pool fixed at start-up, or they may only launch work
on memory they already own): it keeps its scratch in a static device array instead
of a workspace. This file runs last so that, if it fails, a run that stops at the
first failure has already run every other test; it also passes in a fresh process.
"""
import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2501_03759_gb300 import lbch  # noqa: E402

REL_TOL = 1e-5  # the energy tolerance of the GPU parity tests


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    lbch.load()


def _static_energy(params, f9_host, stream):
    """Copies canonical populations to the device as FP32 and runs the static entry point."""
    ny, nx = f9_host.shape[1:]
    d_f9 = torch.from_numpy(np.ascontiguousarray(f9_host, dtype=np.float32)).cuda()
    d_out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    lbch.lbch_free_energy_static(params, d_f9.data_ptr(), nx * ny, d_out.data_ptr(), stream.cuda_stream)
    stream.synchronize()
    return float(d_out.item())


@pytest.mark.parametrize("alpha,reg", [(0.3, lbch.REG_WILLMORE), (0.0, lbch.REG_LINEAR)])
def test_static_energy_matches_context_energy_two_calls(alpha, reg):
    nx, ny = 160, 96
    params = lbch.make_params(nx, ny, alpha=alpha, regularization=reg)
    s = lbch.Solver(params)
    s.init_field(W.noise(nx, ny, 0.4, 12))
    stream = torch.cuda.current_stream()
    for steps in (7, 30):  # two calls in a row, on two different states
        s.step(steps)
        want = s.free_energy()
        got = _static_energy(params, s.state(), stream)  # state() values are exact FP32
        assert abs(got - want) <= REL_TOL * abs(want), (steps, got, want)
    s.close()


def test_static_energy_rejects_oversized_grid_and_bad_arguments():
    p = lbch.make_params(4096, 2048)  # 8,388,608 nodes > 4,194,304
    with pytest.raises(lbch.LbchError) as e:
        lbch.lbch_free_energy_static(p, 256, 4096 * 2048, 256, 0)
    assert e.value.status == lbch.EINVAL
    q = lbch.make_params(64, 64)
    with pytest.raises(lbch.LbchError) as e:
        lbch.lbch_free_energy_static(q, 256, 64 * 64 - 1, 256, 0)  # planes overlap
    assert e.value.status == lbch.EINVAL
    with pytest.raises(lbch.LbchError) as e:
        lbch.lbch_free_energy_static(q, 0, 64 * 64, 256, 0)
    assert e.value.status == lbch.EINVAL
