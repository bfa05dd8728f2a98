"""Host-side analysis (paper_1007_3109_gb300.analysis) against the oracle's
independent formulation and against closed forms.

The library's classification works in lattice variables (F, k, D_u, D_v);
the oracle follows the paper's dimensionless route (eta, tau, eps of
Sec. III.B, Eq. reac_diff19 states, tr M / |M| closed forms).  Both must
label every instance of the 32 x 32 (F, k) sweep alike.
"""
import math

import numpy as np
import pytest

import oracle as orc
from paper_1007_3109_gb300 import analysis, inputs


def _oracle_label(F, k, Du, Dv):
    d = orc.gs_dimensionless(F, k, Du, Dv)
    eta, tau, eps2 = d["eta"], d["tau"], d["eps2"]
    if eta < 2.0:
        return "trivial"
    B = orc.gs_steady_states_dimensionless(eta)["-"][1]
    band = orc.turing_band(eta, eps2, B)
    turing = band is not None and band[0] > 0.0
    if orc.hopf_unstable(eta, tau):
        return "turing+hopf" if turing else "hopf"
    return "turing" if turing else "stable"


def test_point_source_and_error_match_oracle():
    for (L, D, kap, t) in ((100, 0.02, 0.01, 400), (64, 0.1, 0.033, 80), (33, 1.0 / 6.0, 0.0, 7)):
        a = analysis.point_source(L, L, L // 2, L // 2, D, kap, t)
        b = orc.point_source(L, L, L // 2, L // 2, D, kap, t)
        np.testing.assert_allclose(a, b, rtol=1e-14, atol=0)
    rng = np.random.default_rng(1)
    x, y = rng.random((40, 40)), rng.random((40, 40))
    assert analysis.relative_error(x, y) == pytest.approx(orc.relative_error(x, y), rel=1e-14)


def test_point_source_integrates_to_decayed_mass():
    rho = analysis.point_source(300, 300, 150, 150, 0.05, 0.02, 200.0)
    assert rho.sum() == pytest.approx(math.exp(-4.0), rel=1e-9)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_dominant_wavelength_matches_oracle(seed):
    L = 128
    y, x = np.mgrid[0:L, 0:L]
    rng = np.random.default_rng(seed)
    n = rng.integers(4, 20, size=2)
    field = np.cos(2 * np.pi * (n[0] * x + n[1] * y) / L) + 0.1 * rng.standard_normal((L, L))
    a = analysis.dominant_wavelength(field)
    b = orc.structure_factor_peak(field)
    assert a["shell"] == b["shell"]
    assert a["wavelength"] == pytest.approx(b["wavelength"], rel=1e-12)


def test_dominant_wavelength_exact_mode():
    L = 96
    y, x = np.mgrid[0:L, 0:L]
    res = analysis.dominant_wavelength(np.cos(2 * np.pi * (6 * x + 8 * y) / L))
    assert res["shell"] == 10 and res["wavelength"] == pytest.approx(L / 10, rel=1e-12)
    assert res["q"] == pytest.approx(orc.wave_number(6, 8, L, L), rel=1e-12)


def test_gs_states_are_fixed_points():
    for F, k in ((0.04, 0.06), (0.025, 0.055), (0.08, 0.03)):
        for u, v in analysis.gs_states(F, k):
            assert abs(-u * v * v + F * (1 - u)) < 1e-14 and abs(u * v * v - (F + k) * v) < 1e-14


def test_gs_classification_matches_oracle_on_the_sweep():
    """Every (F, k) of the phase-diagram sweep, and the Turing parameters of
    Figs. 7-8 and 11-12 (eta, tau given, D_u / D_v = 2)."""
    w = inputs.WORKLOADS["gs_sweep_256"]
    Du, Dv = w["D"]
    F, k = inputs.sweep_params()
    labels = {}
    for f, kk in zip(F, k):
        got = analysis.gs_classify(float(f), float(kk), Du, Dv)["label"]
        ref = _oracle_label(float(f), float(kk), Du, Dv)
        assert got == ref, (f, kk, got, ref)
        labels[got] = labels.get(got, 0) + 1
    assert set(labels) >= {"trivial", "hopf", "stable"}, labels
    for eta, tau in ((2.0072819, 2.742424), (2.013958, 2.73333), (2.017971, 2.707462), (2.0184336, 2.7272),
                     (2.014, 2.733)):
        f, kk = orc.gs_params_from_dimensionless(eta, tau)
        res = analysis.gs_classify(f, kk, 0.08, 0.04)
        assert res["label"] == _oracle_label(f, kk, 0.08, 0.04), (eta, tau, res)
        assert res["label"].startswith("turing") and res["band"][0] > 0.0, (eta, tau, res)


def test_turing_band_matches_eq_reac_diff32():
    """The lattice-variable band [q1^2, q2^2] in units of 1/l_A^2 equals the
    roots of Eq. reac_diff32."""
    eta, tau = 2.014, 2.733
    F, k = orc.gs_params_from_dimensionless(eta, tau)
    Du, Dv = 0.08, 0.04
    res = analysis.gs_classify(F, k, Du, Dv)
    d = orc.gs_dimensionless(F, k, Du, Dv)
    B = orc.gs_steady_states_dimensionless(eta)["-"][1]
    lo, hi = orc.turing_band(eta, d["eps2"], B)
    lA2 = d["lA"] ** 2
    assert res["band"][0] * lA2 == pytest.approx(lo, rel=1e-9)
    assert res["band"][1] * lA2 == pytest.approx(hi, rel=1e-9)
