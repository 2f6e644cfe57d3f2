"""Host-side checks of the learned leap's C-ABI (no GPU): parameter count, workspace
sizing and parameter validation, and the symmetry turns of the training data."""
import numpy as np
import pytest

from oracle import nop_oracle as N
from paper_2501_03759_gb300 import lbnop


def test_param_count_matches_the_layout():
    assert lbnop.lbnop_param_count() == N.param_count() == 826096


@pytest.mark.parametrize("H,W,B,scale", [(31, 64, 1, 0.1), (64, 48, 1, 0.1), (64, 64, 0, 0.1), (64, 64, 65, 0.1),
                                         (64, 64, 1, 0.0), (64, 64, 1, float("nan")), (16, 16, 1, 0.1)])
def test_invalid_params_have_no_workspace(H, W, B, scale):
    assert lbnop.lbnop_workspace_bytes(lbnop.make_params(H, W, B, scale)) == 0


def test_workspace_grows_with_batch_and_size():
    a = lbnop.lbnop_workspace_bytes(lbnop.make_params(64, 64, 1))
    b = lbnop.lbnop_workspace_bytes(lbnop.make_params(64, 64, 4))
    c = lbnop.lbnop_workspace_bytes(lbnop.make_params(128, 128, 4))
    assert 0 < a < b < c
    # parameters, Adam state and gradients alone: 4 FP32 copies
    assert a > 4 * 4 * N.param_count()


def test_d4_turns_form_the_square_group():
    # The eight training turns are distinct, are numpy's rot90 / flip, and compose as the group.
    import torch
    from paper_2501_03759_gb300.surrogate import d4

    x = torch.arange(2 * 6 * 6, dtype=torch.float32).reshape(2, 6, 6)
    seen = set()
    for k in range(4):
        for flip in (False, True):
            y = d4(x, k, flip)
            ref = np.rot90(x.numpy(), k, axes=(1, 2))
            ref = ref[:, :, ::-1] if flip else ref
            assert np.array_equal(y.numpy(), ref) and y.is_contiguous()
            seen.add(y.numpy().tobytes())
    assert len(seen) == 8
    assert torch.equal(d4(d4(x, 1, False), 3, False), x)
    assert torch.equal(d4(d4(x, 0, True), 0, True), x)


def test_leap_turns_validated_on_the_host():
    # lbnop_create only lays out the caller's workspace (no CUDA call), so a context on a
    # placeholder address can check the setter's arguments without a GPU.
    import ctypes

    from paper_2501_03759_gb300 import lbch

    lib = lbnop.load()
    for (H, W, B), allowed in (((64, 64, 4), {1, 4}), ((64, 64, 1), {1}), ((64, 128, 4), {1})):
        p = lbnop.make_params(H, W, B)
        ctx = lbnop.lbnop_create(p, 1 << 20, lbnop.lbnop_workspace_bytes(p), 0)
        for turns in (0, 1, 2, 3, 4, 8):
            st = lib.lbnop_set_leap_turns(ctx, turns)
            assert st == (lbch.OK if turns in allowed else lbch.EINVAL), (H, W, B, turns)
        lbnop.lbnop_destroy(ctx)
    assert lib.lbnop_set_leap_turns(None, 1) == lbch.EINVAL
