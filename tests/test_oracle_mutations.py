"""The oracle's pins are sharp: each plausible mistake planted in a copy of the
oracle's C source (on the CPU, in a temporary build) makes some pin fail.

Every mutant is a one-line slip of the kind that could hide in the oracle: a
wrong sign of i, a dropped or shifted sqrt(p+1), the atom index reversed,
w_a and w_c swapped, a wrong Taylor factor, a missing conjugate, a wrong
photon-number bin, a wrong Dicke element, a wrong tangent generator.
"""
import os
import subprocess
import tempfile

import pytest

import oracle as O
from tests import test_oracle_pins as pins

SRC = os.path.join(os.path.dirname(O.__file__), "tc_oracle.c")

MUTANTS = {
    "taylor_sign_of_i": [("term[2 * j] = f * im;\n            term[2 * j + 1] = -f * re;",
                          "term[2 * j] = -f * im;\n            term[2 * j + 1] = f * re;")],
    "dropped_sqrt": [("return g[atom0] * sqrt((double)(p + 1));", "return g[atom0];")],
    "sqrt_of_p_not_p_plus_1": [("return g[atom0] * sqrt((double)(p + 1));",
                                "return g[atom0] * sqrt((double)(p + (p > 0 ? 0 : 1)));")],
    "sqrt_p_plus_2": [("return g[atom0] * sqrt((double)(p + 1));",
                       "return g[atom0] * sqrt((double)(p + 2));")],
    "atom_bit_order_reversed": [("unsigned long bit = 1ul << (n - i);", "unsigned long bit = 1ul << (i - 1);"),
                                ("if ((s >> (n - i)) & 1ul)", "if ((s >> (i - 1)) & 1ul)")],
    "wa_wc_swapped": [("double a = wc * (double)p;\n    double b = wa * (double)pc;",
                       "double a = wa * (double)p;\n    double b = wc * (double)pc;")],
    "taylor_factor": [("double f = dt / (double)k, big = 0.0;\n        for (unsigned long j = 0; j < N; j++) {\n            double re",
                       "double f = dt / (double)(k + 1), big = 0.0;\n        for (unsigned long j = 0; j < N; j++) {\n            double re")],
    "photon_bin_reversed": [("Pm[n - pc] += d;", "Pm[pc] += d;"),
                            ("out[n + 1 + (n - pc)] += d;", "out[n + 1 + pc] += d;")],
    "dense_step_missing_conj": [("double ur = uj[2 * k], ui = -uj[2 * k + 1];",
                                 "double ur = uj[2 * k], ui = uj[2 * k + 1];")],
    "dense_step_transposed_U": [("const double* uj = U + 2 * j * N;\n            double sr = 0.0, si = 0.0;\n            for (long k = 0; k < N; k++) {\n                double xr = x[2 * k], xi = x[2 * k + 1];\n                double ur = uj[2 * k], ui = -uj[2 * k + 1];",
                                 "double sr = 0.0, si = 0.0;\n            for (long k = 0; k < N; k++) {\n                double xr = x[2 * k], xi = x[2 * k + 1];\n                double ur = U[2 * (k * N + j)], ui = -U[2 * (k * N + j) + 1];")],
    "dicke_element": [("double h = g * (double)(m + 1) * sqrt((double)(n - m));",
                       "double h = g * sqrt((double)(m + 1)) * sqrt((double)(n - m));")],
    "taylor_fixed_factorial": [("fact *= (double)k;", "fact *= (double)(k > 1 ? k - 1 : 1);")],
    "tangent_wa_wc_swapped": [("double d = (param == n) ? (double)pc : (double)(n - pc);",
                               "double d = (param == n) ? (double)(n - pc) : (double)pc;")],
    "energy_offdiag_dropped": [("*en += h * (rho[2 * (s * N + sg)] + rho[2 * (sg * N + s)]);", "(void)h;")],
    "purity_abs_not_squared": [("*pur += re * re + im * im;", "*pur += re * re;")],
}

# the pins run against each mutant (cheap ones; each takes < 1 s)
PINS = [
    pins.test_h_n2_matches_hand_expansion,
    pins.test_h_n1_is_jaynes_cummings,
    lambda o: pins.test_jaynes_cummings_rabi(o, 0.02),
    pins.test_jaynes_cummings_full_state_pins_the_sign_of_i,
    lambda o: pins.test_qubit_photon_reading_factorises(o, 3),
    pins.test_dicke_matrix_by_hand,
    lambda o: pins.test_dicke_tridiagonal_matches_full_space(o, 5),
    lambda o: pins.test_taylor_stepping_matches_diagonalisation(o, 4),
    pins.test_short_time_photon_growth,
    pins.test_invariants_of_pure_evolution,
    pins.test_paper_taylor_k10_has_the_predicted_remainder,
    pins.test_dense_step_matches_state_propagation,
    pins.test_dense_step_mixed_invariants,
    pins.test_dense_step_general_unitary,
    pins.test_observables_hand_n2,
    pins.test_observables_pure_equals_dense,
    pins.test_forward_gradient_matches_central_differences,
    pins.test_gradient_identities,
]


def _build_mutant(edits, workdir):
    src = open(SRC).read()
    for old, new in edits:
        assert old in src, "mutation anchor not found: %r" % old[:60]
        src = src.replace(old, new)
    cpath = os.path.join(workdir, "mut.c")
    with open(cpath, "w") as f:
        f.write(src)
    so = os.path.join(workdir, "libmut.so")
    subprocess.run(["gcc", "-O1", "-fopenmp", "-ffp-contract=off", "-shared", "-fPIC",
                    "-o", so, cpath, "-lm"], check=True)
    return so


def test_unmutated_oracle_passes_every_pin(oracle):
    for pin in PINS:
        pin(oracle)


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_each_mutant_is_caught(name, monkeypatch, oracle):
    with tempfile.TemporaryDirectory() as d:
        so = _build_mutant(MUTANTS[name], d)
        monkeypatch.setattr(O, "_lib", O._bind(so))
        caught = []
        for pin in PINS:
            try:
                pin(O)
            except (AssertionError, RuntimeError, FloatingPointError, ValueError):
                caught.append(pin)
                break
        assert caught, "mutant %s survived every pin" % name
