"""Planted mistakes in the learned-leap oracle (oracle/nop_oracle.py): each must make its pin fail.

Each case copies nop_oracle.py with one plausible mistake (a convolution where the network
correlates, a wrong adjoint shift, a dropped factor or term, truncation instead of rounding),
loads the copy in a separate process in place of oracle.nop_oracle, and runs the named pins
of tests/test_nop_oracle_pins.py there. The case passes only if those pins FAIL; the
unmodified oracle passes them in the pin file itself. CPU only.
"""
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "nop_oracle.py")
PINS = "tests/test_nop_oracle_pins.py"

# (name, original text, planted text, pins expected to fail); each original occurs once.
MUTANTS = [
    ("conv_not_correlation", "y = sum(shift(x, dy, dx) @ W[t].T for t, (dy, dx) in enumerate(TAPS))",
     "y = sum(shift(x, -dy, -dx) @ W[t].T for t, (dy, dx) in enumerate(TAPS))",
     ["test_conv_matches_fft_circular_correlation", "test_conv_known_offsets"]),
    ("bwd_data_wrong_shift", "return sum(shift(dy @ W[t], -oy, -ox) for t, (oy, ox) in enumerate(TAPS))",
     "return sum(shift(dy @ W[t], oy, ox) for t, (oy, ox) in enumerate(TAPS))", ["test_conv_adjoints"]),
    ("bwd_weight_wrong_shift", 'return np.stack([np.einsum("bhwo,bhwi->oi", dy, shift(x, oy, ox)) for oy, ox in TAPS])',
     'return np.stack([np.einsum("bhwo,bhwi->oi", dy, shift(x, -oy, -ox)) for oy, ox in TAPS])', ["test_conv_adjoints"]),
    ("silu_grad_wrong", "return s * (1.0 + z * (1.0 - s))", "return s * (1.0 + z * s)",
     ["test_silu_values_and_derivative"]),
    ("pool_bwd_unscaled", "return np.repeat(np.repeat(g, 2, axis=1), 2, axis=2) / 4.0",
     "return np.repeat(np.repeat(g, 2, axis=1), 2, axis=2)", ["test_pool_up_s2d_adjoints"]),
    ("head_keeps_mean", "D = D - D.mean(axis=(1, 2), keepdims=True)", "D = D",
     ["test_zero_output_layer_is_identity_and_head_conserves_mass"]),
    ("skip_gradient_dropped", 'g_h1 += pool_bwd(layer_bwd("e2a", g, True))', 'g_h1 = pool_bwd(layer_bwd("e2a", g, True))',
     ["test_network_gradient_matches_central_differences"]),
    ("activation_flag_m3b", 'g = layer_bwd("m3b", up_bwd(g_in_d2a), True)', 'g = layer_bwd("m3b", up_bwd(g_in_d2a), False)',
     ["test_network_gradient_matches_central_differences"]),
    ("adam_no_bias_correction", "mhat = m / (1.0 - beta1 ** t)", "mhat = m",
     ["test_adam_first_steps_closed_form"]),
    ("bf16_truncates", "u = (u + 0x7FFF + ((u >> 16) & 1)) >> 16 << 16", "u = u >> 16 << 16",
     ["test_bf16_rounding_is_round_to_nearest_even"]),
    ("clip_max_norm", "nrm = float(np.sqrt(np.sum(np.asarray(grad, dtype=np.float64) ** 2)))",
     "nrm = float(np.max(np.abs(np.asarray(grad, dtype=np.float64))))", ["test_global_norm_clipping"]),
    ("loss_ignores_weight", "return float(np.sum(w * d * d) / d.size), 2.0 * w * d / d.size",
     "return float(np.sum(d * d) / d.size), 2.0 * w * d / d.size", ["test_weighted_loss_and_gradient"]),
]

# Runs the pins with the planted copy registered as oracle.nop_oracle before the pin file
# imports it.
RUNNER = r"""
import importlib.util, sys
root, planted, pin_id = sys.argv[1], sys.argv[2], sys.argv[3]
sys.path.insert(0, root)
import oracle
spec = importlib.util.spec_from_file_location("oracle.nop_oracle", planted)
mod = importlib.util.module_from_spec(spec)
sys.modules["oracle.nop_oracle"] = mod
spec.loader.exec_module(mod)
oracle.nop_oracle = mod
import pytest
sys.exit(pytest.main(["-q", "-p", "no:cacheprovider", pin_id]))
"""


def _run(tmp, name, old, new, pins):
    src = open(SRC).read()
    assert src.count(old) == 1, old
    planted = os.path.join(tmp, f"{name}.py")
    with open(planted, "w") as fh:
        fh.write(src.replace(old, new))
    rc = {}
    for pin in pins:
        r = subprocess.run([sys.executable, "-c", RUNNER, ROOT, planted, f"{PINS}::{pin}"], cwd=ROOT,
                           capture_output=True, text=True, env=dict(os.environ, OMP_NUM_THREADS="2"))
        rc[pin] = (r.returncode, r.stdout[-2000:] + r.stderr[-1000:])
    return rc


@pytest.fixture(scope="module")
def outcomes(tmp_path_factory):
    tmp = str(tmp_path_factory.mktemp("nop_mutants"))
    with ThreadPoolExecutor(max(1, min(len(MUTANTS), (os.cpu_count() or 2) // 2))) as ex:
        futs = {m[0]: ex.submit(_run, tmp, *m) for m in MUTANTS}
        return {k: f.result() for k, f in futs.items()}


def test_runner_passes_the_unmodified_oracle(tmp_path):
    # The same loader with an unplanted copy: the pins pass (exit 0), so a failure below comes
    # from the planted mistake and not from the loading.
    rc = _run(str(tmp_path), "unplanted", "def shift(", "def shift(", ["test_conv_known_offsets", "test_conv_adjoints"])
    for pin, (code, out) in rc.items():
        assert code == 0, f"{pin}: {out}"


@pytest.mark.parametrize("name", [m[0] for m in MUTANTS])
def test_planted_mistake_is_caught(outcomes, name):
    for pin, (code, out) in outcomes[name].items():
        # pytest exit code 1: tests ran and at least one failed (not a load or collection error).
        assert code == 1, f"{name}: pin {pin} did not fail (exit {code})\n{out}"
