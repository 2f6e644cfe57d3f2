"""Planted mistakes in the FP64 oracle: each must make its pin fail.

A pin that passes whatever the oracle computes pins nothing. Each case below copies
oracle/lbch_oracle.cpp with one plausible mistake in one branch (a wrong factor, a
flipped sign, a dropped term, a wrong reading), builds that copy with g++, and runs
the named pins against it in a separate process (LBCH_ORACLE_LIB points the oracle
package at the copy): tests/test_oracle_pins.py for the 2D scheme, and
tests/test_oracle3_pins.py for the D3Q15 scheme. The case passes only if those pins FAIL
on the planted mistake; the unmodified oracle passes them in the pin files themselves.

Everything here runs on the CPU; no mistake is ever planted in the CUDA library.
"""
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "lbch_oracle.cpp")
PINS = "tests/test_oracle_pins.py"
PINS3 = "tests/test_oracle3_pins.py"

# (name, original text, planted text, pins expected to fail). Each original text must occur
# exactly once in the 2D part of the oracle source.
MUTANTS = [
    # Linear regularisation, Eq. 12 (mu) and Eq. 8 (energy).
    ("linear_mu_doubled", "reg = sc.eps * F.lap2[id];  // Eq. 12",
     "reg = 2.0 * sc.eps * F.lap2[id];", ["test_linear_regularisation_visible"]),
    ("linear_mu_sign", "reg = sc.eps * F.lap2[id];  // Eq. 12",
     "reg = -sc.eps * F.lap2[id];", ["test_linear_regularisation_visible"]),
    ("linear_energy_factor", "e += 0.5 * sc.eps * lap * lap;  // Eq. 8\n      }",
     "e += sc.eps * lap * lap;\n      }", ["test_energy_closed_form_cosines_linear_regularisation"]),
    ("linear_energy_willmore_g",
     "e += 0.5 * sc.eps * lap * lap;  // Eq. 8\n      }",
     "e += 0.5 * sc.eps * (lap - bulk_f(sc, phi[id])) * (lap - bulk_f(sc, phi[id]));\n      }",
     ["test_energy_closed_form_cosines_linear_regularisation"]),
    # Nested mu_beta (reading C2, literal Eq. 16).
    ("nested_as_split", "const double iso = nested ? a.gamma : (a.gamma - 1.0);\n      F.Qx",
     "const double iso = a.gamma - 1.0;\n      F.Qx",
     ["test_nested_mu_beta_isotropic_cosine_symbol", "test_nested_minus_split_is_lattice_commutator"]),
    ("nested_minus_f_only", "F.mub[id] = mu - F.mua[id];",
     "F.mub[id] = mu - fb;",
     ["test_nested_mu_beta_isotropic_cosine_symbol", "test_nested_minus_split_is_lattice_commutator"]),
    # The tangential term k |grad phi| P grad_n gamma of Eq. 15 (reading C1) and its literal form.
    ("tangential_drops_k", "const double kq = literal_q ? 1.0 : sc.k;  // factor",
     "const double kq = 1.0;  // factor", ["test_tangential_term_curved_interface"]),
    ("literal_keeps_k", "const double kq = literal_q ? 1.0 : sc.k;  // factor",
     "const double kq = sc.k;  // factor", ["test_tangential_term_curved_interface"]),
    ("projector_sign", "const double P11 = 1.0 - n1 * n1, P12 = -n1 * n2, P22 = 1.0 - n2 * n2;",
     "const double P11 = 1.0 + n1 * n1, P12 = n1 * n2, P22 = 1.0 + n2 * n2;",
     ["test_tangential_term_curved_interface"]),
    ("grad_n_gamma_12_alpha",
     "const double gn1 = 16.0 * sc.alpha * n1 * n1 * n1;       // grad_n gamma\n"
     "  const double gn2 = 16.0 * sc.alpha * n2 * n2 * n2;",
     "const double gn1 = 12.0 * sc.alpha * n1 * n1 * n1;\n"
     "  const double gn2 = 12.0 * sc.alpha * n2 * n2 * n2;",
     ["test_tangential_term_curved_interface"]),
    ("grad_n_gamma_swapped",
     "const double gn1 = 16.0 * sc.alpha * n1 * n1 * n1;       // grad_n gamma\n"
     "  const double gn2 = 16.0 * sc.alpha * n2 * n2 * n2;",
     "const double gn1 = 16.0 * sc.alpha * n2 * n2 * n2;\n"
     "  const double gn2 = 16.0 * sc.alpha * n1 * n1 * n1;",
     ["test_tangential_term_curved_interface"]),
    # gamma(theta) of Eq. 6 between the axis and diagonal values: c |c| equals c = cos 4 theta
    # at c = +-1 (axes and diagonals), so only a generic angle can tell them apart.
    ("gamma_generic_angle",
     "a.gamma = 1.0 + sc.alpha * (4.0 * (n1_4 + n2_4) - 3.0);  // Eq. 6, d = 2",
     "a.gamma = 1.0 + sc.alpha * (4.0 * (n1_4 + n2_4) - 3.0) * std::fabs(4.0 * (n1_4 + n2_4) - 3.0);",
     ["test_linear_dispersion_generic_angle"]),
    # The n = 0 guard (reading C3) at a threshold that reaches interface nodes.
    ("guard_too_high", "const double GUARD = 1e-12;", "const double GUARD = 1e-6;",
     ["test_guard_fires_only_in_the_bulk"]),
    # The discrete energy (reading C11: Eq. 7 with Eq. 9).
    ("energy_without_gamma", "double e = a.gamma * (0.5 * sc.k * (dx * dx + dy * dy) + bulkF(sc, phi[id]));",
     "double e = (0.5 * sc.k * (dx * dx + dy * dy) + bulkF(sc, phi[id]));", ["test_energy_closed_form_cosines"]),
    ("energy_willmore_factor", "        e += 0.5 * sc.eps * w * w;\n      } else if (sc.reg == 2) {",
     "        e += sc.eps * w * w;\n      } else if (sc.reg == 2) {", ["test_energy_closed_form_cosines"]),
    # Parameters and collision (Eqs. 5, 17-19, the rate after Eq. 38).
    ("k_without_half", "d->k = d->beta * p->D * p->D / 2.0;", "d->k = d->beta * p->D * p->D;",
     ["test_parameters_eq5_inversion"]),
    ("s35_without_cs2", "const double s35 = 1.0 / (p->M / CS2 + 0.5);", "const double s35 = 1.0 / (p->M + 0.5);",
     ["test_parameters_eq5_inversion"]),
    ("force_factor_one_minus_s", "b += sc->Minv[i][m] * (1.0 - sc->s[m] / 2.0) * MROWS[m][j];",
     "b += sc->Minv[i][m] * (1.0 - sc->s[m]) * MROWS[m][j];", ["test_srt_reduction"]),
    ("relaxation_squared", "a += sc->Minv[i][m] * sc->s[m] * MROWS[m][j];",
     "a += sc->Minv[i][m] * sc->s[m] * sc->s[m] * MROWS[m][j];", ["test_srt_reduction"]),
    ("rest_equilibrium", "feq[0] = phi + (WGT[0] - 1.0) * mua;", "feq[0] = phi - WGT[0] * mua;",
     ["test_equilibrium_and_source_moments_eq27bc"]),
    ("init_mu_alpha_sign", "const double mua = bulk_f(sc, phi0[id]) - sc.k * lap26(sc, phi0, x, y);  // Eq. 16",
     "const double mua = bulk_f(sc, phi0[id]) + sc.k * lap26(sc, phi0, x, y);",
     ["test_init_is_equilibrium_of_eq16_mu_alpha"]),
    ("source_sign", "for (int i = 0; i < 9; ++i) F[i] = -WGT[i] * (CX[i] * gx + CY[i] * gy);",
     "for (int i = 0; i < 9; ++i) F[i] = WGT[i] * (CX[i] * gx + CY[i] * gy);",
     ["test_equilibrium_and_source_moments_eq27bc"]),
]


# The same for the D3Q15 scheme (Eqs. 3, 6, 17-19, 21, 24, 26 with d = 3): each original text
# occurs exactly once in the 3D part. Most are caught by the separately written NumPy step
# (test_numpy_second_route_3d, alpha = 0.35); the tangential-term readings also by the
# spherical interface, which does not share the NumPy step's readings; the rest by the
# dispersion and mass pins.
MUTANTS3 = [
    ("grad_n_gamma_12_alpha_3d", "gn[d] = 16.0 * alpha * n[d] * n[d] * n[d];",
     "gn[d] = 12.0 * alpha * n[d] * n[d] * n[d];",
     ["test_numpy_second_route_3d", "test_tangential_term_spherical_interface"]),
    ("projector_sign_3d", "v += ((d == e ? 1.0 : 0.0) - n[d] * n[e]) * gn[e];  // P = I - n n^T",
     "v += ((d == e ? 1.0 : 0.0) + n[d] * n[e]) * gn[e];",
     ["test_numpy_second_route_3d", "test_tangential_term_spherical_interface"]),
    ("gamma_alpha_sign_3d", "a.gamma = 1.0 + alpha * (4.0 * s4 - 3.0);  // Eq. 6, d = 3",
     "a.gamma = 1.0 - alpha * (4.0 * s4 - 3.0);", ["test_linear_dispersion_3d_axis"]),
    ("jz_rate_default_3d", "sc->s[3] = sc->s[5] = sc->s[7] = sj;",
     "sc->s[3] = sc->s[5] = sj;", ["test_numpy_second_route_3d"]),
    ("laplacian_half_3d",
     "for (int i = 0; i < 15; ++i) s += 2.0 * W3[i] * (chi[idx3(sc, x + CX3[i], y + CY3[i], z + CZ3[i])] - c);",
     "for (int i = 0; i < 15; ++i) s += W3[i] * (chi[idx3(sc, x + CX3[i], y + CY3[i], z + CZ3[i])] - c);",
     ["test_numpy_second_route_3d", "test_linear_dispersion_3d_axis"]),
    ("tangential_drops_k_3d", "const double kq = literal_q ? 1.0 : sc.k;",
     "const double kq = 1.0;", ["test_numpy_second_route_3d", "test_tangential_term_spherical_interface"]),
    ("literal_keeps_k_3d", "const double kq = literal_q ? 1.0 : sc.k;",
     "const double kq = sc.k;", ["test_tangential_term_spherical_interface"]),
    ("willmore_drops_fprime_w_3d",
     "reg = sc.eps * (lap3(sc, F.w.data(), x, y, z) - fp * F.w[id]);  // Eq. 13",
     "reg = sc.eps * lap3(sc, F.w.data(), x, y, z);", ["test_numpy_second_route_3d"]),
    ("linear_regularisation_doubled_3d", "else if (sc.reg == 2) reg = sc.eps * F.lap2[id];",
     "else if (sc.reg == 2) reg = 2.0 * sc.eps * F.lap2[id];", ["test_linear_dispersion_3d_linear_regularisation"]),
    ("nested_as_split_3d", "const double iso = nested ? a.gamma : (a.gamma - 1.0);",
     "const double iso = a.gamma - 1.0;", ["test_nested_minus_split_is_lattice_commutator_3d"]),
    ("nested_minus_f_only_3d", "F.mub[id] = nested ? F.gamma[id] * fb - divQ + reg - F.mua[id]",
     "F.mub[id] = nested ? F.gamma[id] * fb - divQ + reg - fb", ["test_nested_minus_split_is_lattice_commutator_3d"]),
    ("guard_too_high_3d", "  if (g2 < GUARD) {", "  if (g2 < 1e-6) {", ["test_guard_fires_only_in_the_bulk_3d"]),
    ("init_mu_alpha_sign_3d",
     "const double mua = 4.0 * sc.beta * ph * (ph + 1.0) * (ph - 1.0) - sc.k * lap3(sc, phi0, x, y, z);",
     "const double mua = 4.0 * sc.beta * ph * (ph + 1.0) * (ph - 1.0) + sc.k * lap3(sc, phi0, x, y, z);",
     ["test_init_is_equilibrium_of_eq16_mu_alpha_3d"]),
    ("energy_without_gamma_3d",
     "double e = a.gamma * (0.5 * sc.k * (g[0] * g[0] + g[1] * g[1] + g[2] * g[2]) + F);  // Eq. 7",
     "double e = (0.5 * sc.k * (g[0] * g[0] + g[1] * g[1] + g[2] * g[2]) + F);", ["test_energy3_matches_numpy_route"]),
    ("energy_willmore_factor_3d", "e += 0.5 * sc.eps * w * w;", "e += sc.eps * w * w;",
     ["test_energy3_matches_numpy_route"]),
    ("energy_linear_factor_3d", "e += 0.5 * sc.eps * lap * lap;  // Eq. 8", "e += sc.eps * lap * lap;",
     ["test_energy3_matches_numpy_route"]),
    ("source_sign_3d", "F[i] = -W3[i] * (CX3[i] * gx + CY3[i] * gy + CZ3[i] * gz);  // Eq. 19",
     "F[i] = W3[i] * (CX3[i] * gx + CY3[i] * gy + CZ3[i] * gz);", ["test_numpy_second_route_3d"]),
    ("rest_equilibrium_3d", "feq[0] = phi + (W3[0] - 1.0) * mua;",
     "feq[0] = phi - W3[0] * mua;", ["test_mass_and_energy_droplet_3d"]),
]


def _planted_source(old, new, part="2d"):
    src = open(SRC).read()
    cut = src.index("// 3D: D3Q15")  # the 2D scheme before, the 3D scheme after
    head, tail = src[:cut], src[cut:]
    if part == "2d":
        assert head.count(old) == 1, old
        return head.replace(old, new) + tail
    assert tail.count(old) == 1, old
    return head + tail.replace(old, new)


def _build_and_run(tmp, name, old, new, pins, part="2d", pin_file=PINS):
    d = os.path.join(tmp, name)
    os.makedirs(d, exist_ok=True)
    cpp = os.path.join(d, "lbch_oracle.cpp")
    with open(cpp, "w") as fh:
        fh.write(_planted_source(old, new, part))
    lib = os.path.join(d, "liboracle.so")
    subprocess.run(["g++", "-O2", "-std=c++17", "-fno-fast-math", "-ffp-contract=off", "-fopenmp",
                    "-fPIC", "-shared", "-I", os.path.join(ROOT, "oracle"), cpp, "-o", lib], check=True)
    env = dict(os.environ, LBCH_ORACLE_LIB=lib, OMP_NUM_THREADS="2")
    rc = {}
    for pin in pins:
        r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-p", "no:cacheprovider",
                            f"{pin_file}::{pin}"], cwd=ROOT, env=env, capture_output=True, text=True)
        rc[pin] = (r.returncode, r.stdout[-2000:])
    return rc


@pytest.fixture(scope="module")
def outcomes(tmp_path_factory):
    tmp = str(tmp_path_factory.mktemp("oracle_mutants"))
    with ThreadPoolExecutor(max(1, min(len(MUTANTS) + len(MUTANTS3), (os.cpu_count() or 2) // 2))) as ex:
        futs = {m[0]: ex.submit(_build_and_run, tmp, *m) for m in MUTANTS}
        futs.update({m[0]: ex.submit(_build_and_run, tmp, *m, "3d", PINS3) for m in MUTANTS3})
        return {k: f.result() for k, f in futs.items()}


@pytest.mark.parametrize("name", [m[0] for m in MUTANTS + MUTANTS3])
def test_planted_mistake_is_caught(outcomes, name):
    for pin, (code, out) in outcomes[name].items():
        # pytest exit code 1: tests ran and at least one failed (not a build or collection error).
        assert code == 1, f"{name}: pin {pin} did not fail (exit {code})\n{out}"
