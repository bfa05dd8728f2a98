"""Planted mistakes in the oracle must fail at least one pin.

Each case copies ``oracle/lbrd_oracle.c``, plants one plausible mistake (a
dropped term, a wrong sign, a wrong index, a transposed operand, a wrong
table entry), compiles the copy on the CPU and runs the pins of
``test_oracle_pins.py`` against it.  The real oracle is never modified.
"""
import os
import shutil

import numpy as np
import pytest

import oracle.lbrd_oracle as olib
from oracle import Reaction

import test_oracle_pins as pins

SRC = os.path.join(os.path.dirname(olib.__file__), "lbrd_oracle.c")

GS = Reaction("gray_scott", F=0.04, k=0.06)
LIN = Reaction("linear", kappa=0.02)

PINS = [
    ("table", pins.test_d2q9_table_matches_eq_weights, ()),
    ("isotropy", pins.test_d2q9_isotropy_eq_app11, ()),
    ("tau1_gs", pins.test_tau1_reduces_to_explicit_stencil, ("D2Q9", GS)),
    ("tau1_lin", pins.test_tau1_reduces_to_explicit_stencil, ("D2Q9", LIN)),
    ("symbol", pins.test_fourier_decay_matches_exact_symbol, ("D2Q9", 0.8)),
    ("mass_none", pins.test_mass_conserved_without_reaction, ("D2Q9", 2)),
    ("mass_linear", pins.test_mass_linear_decay_discrete, (2,)),
    ("euler", pins.test_gs_uniform_field_is_forward_euler_of_kinetics, ()),
    ("P_decay", pins.test_gs_P_decay_eq_reac_diff21, ()),
    ("fixed_points", pins.test_gs_steady_states_are_fixed_points, ()),
    ("growth", pins.test_linear_growth_rate_vs_exact_symbol, ("-", 2.0, 22, "turing", (1e-6, 1e-6), 300, 200)),
    ("net_linear", pins.test_network_transformation_equals_linear_kind_bitwise, ()),
    ("net_gs", pins.test_network_gray_scott_matches_eqs_reac_diff10_11, ()),
    ("net_euler3", pins.test_network_three_species_uniform_field_is_forward_euler, ()),
    ("net_cycle", pins.test_network_conservative_cycle_keeps_total_mass, ()),
]

MUTATIONS = {
    "source_sign": ("+ w[i] * R[ss];", "- w[i] * R[ss];"),
    "relaxation_dropped": ("(feq - fi) * omega[ss]", "(feq - fi)"),
    "relaxation_sign": ("fi + (feq - fi) * omega[ss]", "fi - (feq - fi) * omega[ss]"),
    "gs_feed_sign": ("F * (1.0 - u)", "F * (1.0 + u)"),
    "gs_decay_term": ("(F + k) * v", "k * v"),
    "gs_autocatalysis": ("double uvv = u * v * v;", "double uvv = u * u * v;"),
    "stream_transposed": ("(x + ex[i] + nx) % nx", "(x + ey[i] + nx) % nx"),
    "density_species_index": ("r += f_in[at(nx, ny, Q, ss, i, y, x)];", "r += f_in[at(nx, ny, Q, 0, i, y, x)];"),
    "weight_diagonal": ("w[q] = 1.0 / 36.0;", "w[q] = 1.0 / 18.0;"),
    "linear_product_sign": ("R[1] = kappa * rho[0];", "R[1] = -kappa * rho[0];"),
    "velocity_table": ("{0, 0, 1, 0, -1, 1, 1, -1, -1}", "{0, 0, 1, 0, -1, 1, -1, -1, 1}"),
    "init_weight": ("f[at(nx, ny, Q, s, i, y, x)] = w[i] * rho0", "f[at(nx, ny, Q, s, i, y, x)] = w[0] * rho0"),
    "network_order_off_by_one": ("for (e = 0; e < src->order[r][j]; ++e)", "for (e = 0; e <= src->order[r][j]; ++e)"),
    "network_change_sign": ("R[s] = R[s] + (double)src->change[r][s] * p;", "R[s] = R[s] - (double)src->change[r][s] * p;"),
    "network_species_index": ("p = p * rho[j];", "p = p * rho[0];"),
    "network_rate_dropped": ("double p = src->rate[r];", "double p = 1.0;"),
}


def _failing_pins(lib):
    saved = olib._DEFAULT
    olib._DEFAULT = lib
    failed = []
    try:
        for name, fn, args in PINS:
            try:
                with np.errstate(all="ignore"):
                    fn(*args)
            except (AssertionError, ValueError, FloatingPointError, np.linalg.LinAlgError):
                failed.append(name)
    finally:
        olib._DEFAULT = saved
    return failed


def test_unmutated_copy_passes_every_pin(tmp_path):
    src = tmp_path / "lbrd_oracle.c"
    shutil.copy(SRC, src)
    lib = olib.OracleLib(olib.build(str(tmp_path / "liborc.so"), str(src)))
    assert _failing_pins(lib) == []


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(name, tmp_path):
    old, new = MUTATIONS[name]
    text = open(SRC).read()
    assert text.count(old) == 1, f"mutation anchor for {name} not unique"
    src = tmp_path / "lbrd_oracle.c"
    src.write_text(text.replace(old, new))
    lib = olib.OracleLib(olib.build(str(tmp_path / "liborc.so"), str(src)))
    failed = _failing_pins(lib)
    assert failed, f"planted mistake {name} passed every pin"
