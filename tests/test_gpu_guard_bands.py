"""Canary guard bands: every kernel of a context or batch writes only inside the
workspace it was given. The workspace sits between two 1 MiB bands filled with a
byte pattern; after init, steps, diagnostics and state transfer the bands must be
unchanged."""
import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2501_03759_gb300 import lbch  # noqa: E402

GUARD = 1 << 20
PATTERN = 0xA5


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    lbch.load()


def guarded(nbytes):
    buf = torch.full((GUARD + nbytes + GUARD,), PATTERN, dtype=torch.uint8, device="cuda")
    assert buf.data_ptr() % 256 == 0
    return buf, buf.data_ptr() + GUARD


def bands_intact(buf, nbytes):
    torch.cuda.synchronize()
    lo = buf[:GUARD]
    hi = buf[GUARD + nbytes:]
    return bool((lo == PATTERN).all()) and bool((hi == PATTERN).all())


@pytest.mark.parametrize("shape", [(9, 7), (130, 67), (256, 40), (1, 5), (124, 9)])
@pytest.mark.parametrize("storage", [lbch.STORE_F32, lbch.STORE_BF16_DEV, lbch.STORE_F16_DEV])
def test_context_writes_stay_in_workspace(shape, storage):
    nx, ny = shape
    p = lbch.make_params(nx, ny, alpha=0.3, storage=storage)
    nbytes = lbch.lbch_workspace_bytes(p)
    buf, ptr = guarded(nbytes)
    stream = torch.cuda.current_stream()
    ctx = lbch.lbch_create(p, ptr, nbytes, stream.cuda_stream)
    try:
        lbch.lbch_init_field(ctx, np.ascontiguousarray(W.noise(nx, ny, 0.5, 1)))
        lbch.lbch_step(ctx, 9)
        lbch.lbch_mass(ctx)
        lbch.lbch_free_energy(ctx)
        st = np.empty((9, ny, nx))
        lbch.lbch_get_state(ctx, st)
        lbch.lbch_set_state(ctx, st)
        lbch.lbch_step(ctx, 4)
        lbch.lbch_get_field(ctx, np.empty((ny, nx)))
    finally:
        lbch.lbch_destroy(ctx)
    assert bands_intact(buf, nbytes)


def test_batch_writes_stay_in_workspace():
    nx, ny = [9, 64, 130, 256], [7, 64, 67, 40]
    common = lbch.make_params(8, 8)
    nbytes = lbch.lbch_batch_workspace_bytes(common, nx, ny)
    buf, ptr = guarded(nbytes)
    b = lbch.lbch_batch_create(common, nx, ny, [0.1, 0.2, 0.3, 0.4], ptr, nbytes,
                               torch.cuda.current_stream().cuda_stream)
    try:
        for i in range(4):
            lbch.lbch_batch_init_field(b, i, np.ascontiguousarray(W.noise(nx[i], ny[i], 0.5, i)))
        lbch.lbch_batch_step(b, 70)
        for i in range(4):
            lbch.lbch_batch_mass(b, i)
            lbch.lbch_batch_free_energy(b, i)
    finally:
        lbch.lbch_batch_destroy(b)
    assert bands_intact(buf, nbytes)


def test_3d_context_writes_stay_in_workspace():
    nx, ny, nz = 13, 11, 9
    p = lbch.make_params3(nx, ny, nz, alpha=0.3)
    nbytes = lbch.lbch3_workspace_bytes(p)
    buf, ptr = guarded(nbytes)
    ctx = lbch.lbch3_create(p, ptr, nbytes, torch.cuda.current_stream().cuda_stream)
    try:
        lbch.lbch3_init_field(ctx, np.ascontiguousarray(np.random.default_rng(1).uniform(-0.5, 0.5, (nz, ny, nx))))
        lbch.lbch3_step(ctx, 7)
        lbch.lbch3_mass(ctx)
        lbch.lbch3_free_energy(ctx)
        lbch.lbch3_get_field(ctx, np.empty((nz, ny, nx)))
    finally:
        lbch.lbch3_destroy(ctx)
    assert bands_intact(buf, nbytes)
