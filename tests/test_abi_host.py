"""Host-side checks of the C-ABI library: it loads without a GPU, exports every
function the public headers declare, and validates parameters and workspaces
before any CUDA call."""
import ctypes
import glob
import os
import re

import pytest

from paper_2501_03759_gb300 import build, lbch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return lbch.load()


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names.update(re.findall(r"\b((?:lbch|lbch3|lbnop)_[a-z0-9_]+)\s*\(", text))
    return sorted(names)


def test_headers_declare_the_boundary():
    names = declared_functions()
    for required in ("lbch_create", "lbch_init_field", "lbch_step", "lbch_free_energy", "lbch_mass",
                     "lbch_get_field", "lbch_get_state", "lbch_set_state", "lbch_destroy"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_params_struct_layout_matches_header():
    # int32 nx, ny; 5 doubles; 9 doubles; int32 storage, regularization; uint32 flags
    assert ctypes.sizeof(lbch.lbch_params) == 8 + 5 * 8 + 9 * 8 + 3 * 4 + 4  # trailing pad to 8
    assert lbch.lbch_params.s.offset == 48


def test_workspace_bytes(lib):
    p = lbch.make_params(64, 64)
    n = 64 * 64
    b = lbch.lbch_workspace_bytes(p)
    assert b >= 2 * 9 * 4 * n + 2 * 8 * n
    for st in (lbch.STORE_BF16_DEV, lbch.STORE_F16_DEV):
        q = lbch.make_params(64, 64, storage=st)
        assert 2 * 24 * n + 2 * 8 * n <= lbch.lbch_workspace_bytes(q) < b


@pytest.mark.parametrize("bad", [
    dict(nx=0), dict(ny=0), dict(nx=70000), dict(M=0.0), dict(M=-1.0), dict(sigma=0.0), dict(D=0.0),
    dict(eps=-0.1), dict(alpha=1.0), dict(alpha=-0.1), dict(storage=3), dict(regularization=5),
    dict(flags=8), dict(s=[1, 1, 2.0, 1, 1, 1, 1, 1, 1]), dict(s=[1, 0.0, 1, 1, 1, 1, 1, 1, 1]),
    dict(M=float("nan")),
])
def test_invalid_params_rejected_before_cuda(lib, bad):
    kw = dict(nx=16, ny=16)
    kw.update(bad)
    nx, ny = kw.pop("nx"), kw.pop("ny")
    p = lbch.make_params(nx, ny, **kw)
    assert lbch.lbch_workspace_bytes(p) == 0
    with pytest.raises(lbch.LbchError) as e:
        lbch.lbch_create(p, 256, 1 << 30, 0)
    assert e.value.status == lbch.EINVAL


def test_workspace_checks_before_cuda(lib):
    p = lbch.make_params(16, 16)
    need = lbch.lbch_workspace_bytes(p)
    for ptr, nbytes in ((0, need), (256, need - 1), (256 + 8, need)):
        with pytest.raises(lbch.LbchError) as e:
            lbch.lbch_create(p, ptr, nbytes, 0)
        assert e.value.status == lbch.ENOMEM


def test_null_context_calls(lib):
    assert lib.lbch_step(None, 1) == lbch.EINVAL
    assert lib.lbch_steps_taken(None) == -1
    assert lbch.lbch_last_error(None) == "context is NULL"
    lib.lbch_destroy(None)


def test_explicit_s35_validated(lib):
    p = lbch.make_params(16, 16, s=[1, 1, 1, 0.0, 1, 1, 1, 1, 1])
    assert lbch.lbch_workspace_bytes(p) > 0  # s_3 comes from M
    q = lbch.make_params(16, 16, s=[1, 1, 1, 0.0, 1, 1, 1, 1, 1], flags=lbch.S35_EXPLICIT)
    assert lbch.lbch_workspace_bytes(q) == 0


def test_declarations_cover_all_three_headers():
    names = declared_functions()
    for required in ("lbch3_create", "lbch3_step", "lbnop_forward", "lbnop_leap_run", "lbnop_leap_run_judged",
                     "lbch_mass_device", "lbch_free_energy_device", "lbch_save_state_device",
                     "lbch_restore_state_device", "lbch_set_steps_taken", "lbch_state_bytes"):
        assert required in names


def test_state_bytes_match_storage(lib):
    n = 100 * 60
    ps = (n + 63) // 64 * 64
    assert lbch.lbch_state_bytes(lbch.make_params(100, 60)) >= 9 * 4 * ps
    for st in (lbch.STORE_BF16_DEV, lbch.STORE_F16_DEV):
        b = lbch.lbch_state_bytes(lbch.make_params(100, 60, storage=st))
        assert 2 * 4 * ps + 8 * 2 * ps <= b < 9 * 4 * ps
    assert lbch.lbch_state_bytes(lbch.make_params(0, 60)) == 0


def test_new_calls_reject_null_context(lib):
    assert lib.lbch_set_steps_taken(None, 5) == lbch.EINVAL
    assert lib.lbch_mass_device(None, None) == lbch.EINVAL
    assert lib.lbch_free_energy_device(None, None) == lbch.EINVAL
    assert lib.lbch_save_state_device(None, None, 0) == lbch.EINVAL
    assert lib.lbch_restore_state_device(None, None, 0) == lbch.EINVAL


def test_judge_struct_layout():
    from paper_2501_03759_gb300 import lbnop

    lbnop.load()
    assert ctypes.sizeof(lbnop.lbnop_judge) == 5 * 8
    assert ctypes.sizeof(lbnop.lbnop_judge_stats) == 11 * 8
    assert lbnop.lbnop_judge_stats.max_audit_err.offset == 8 * 8
    j = lbnop.make_judge()
    assert lbch.load().lbnop_leap_run_judged(None, None, 0.3, 1, 50, ctypes.byref(j), None) == lbch.EINVAL
