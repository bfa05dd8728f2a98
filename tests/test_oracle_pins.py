"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Every check here is independent of the oracle's own code: closed forms of the
paper, a brute-force explicit stencil, exact Fourier symbols, conservation
laws, fixed points and exact symmetries.  ``test_oracle_mutations.py`` shows
that plausible mistakes in the oracle fail at least one of them.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle as orc
from oracle import Reaction
from paper_1007_3109_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

# Velocity set and weights written out from Eq. Weights (D2Q9) in the
# ordering used throughout, and the D2Q5 reading; used only by the checks.
E9 = [(0, 0), (1, 0), (0, 1), (-1, 0), (0, -1), (1, 1), (-1, 1), (-1, -1), (1, -1)]
W9 = [4 / 9] + [1 / 9] * 4 + [1 / 36] * 4
E5 = E9[:5]
W5 = [1 / 3] + [1 / 6] * 4
TABLES = {"D2Q9": (E9, W9), "D2Q5": (E5, W5)}


def _golden(name):
    with open(os.path.join(GOLDEN, name)) as fh:
        return json.load(fh)


# ---------------------------------------------------------------------------
# Lattice tables: Eq. Weights and the isotropy conditions of Eq. app11
# ---------------------------------------------------------------------------

def _moments(lat):
    ex, ey, w = orc.lattice(lat)
    e = np.stack([ex, ey], axis=1).astype(float)
    m0 = w.sum()
    m1 = np.einsum("i,ia->a", w, e)
    m2 = np.einsum("i,ia,ib->ab", w, e, e)
    m3 = np.einsum("i,ia,ib,ic->abc", w, e, e, e)
    m4 = np.einsum("i,ia,ib,ic,id->abcd", w, e, e, e, e)
    return m0, m1, m2, m3, m4


def _iso4(cs2):
    d = np.eye(2)
    return cs2 ** 2 * (np.einsum("ab,cd->abcd", d, d) + np.einsum("ac,bd->abcd", d, d)
                       + np.einsum("ad,bc->abcd", d, d))


def test_d2q9_table_matches_eq_weights():
    ex, ey, w = orc.lattice("D2Q9")
    assert list(zip(ex.tolist(), ey.tolist())) == E9
    np.testing.assert_array_equal(w, np.array(W9))


def test_d2q9_isotropy_eq_app11():
    m0, m1, m2, m3, m4 = _moments("D2Q9")
    cs2 = 1.0 / 3.0
    assert m0 == pytest.approx(1.0, abs=1e-15)                    # (a)
    np.testing.assert_allclose(m1, 0.0, atol=1e-16)                # (b)
    np.testing.assert_allclose(m2, cs2 * np.eye(2), atol=1e-15)    # (c)
    np.testing.assert_allclose(m3, 0.0, atol=1e-16)                # (d)
    np.testing.assert_allclose(m4, _iso4(cs2), atol=1e-15)         # (e)


def test_d2q5_isotropy_to_second_order():
    """D2Q5 (reading: w0 = 1/3, w1..4 = 1/6) meets (a)-(d) with c_s^2 = 1/3
    but not the fourth-order condition (e); pure diffusion only needs (a)-(c)."""
    m0, m1, m2, m3, m4 = _moments("D2Q5")
    assert m0 == pytest.approx(1.0, abs=1e-15)
    np.testing.assert_allclose(m1, 0.0, atol=1e-16)
    np.testing.assert_allclose(m2, np.eye(2) / 3.0, atol=1e-15)
    np.testing.assert_allclose(m3, 0.0, atol=1e-16)
    assert np.max(np.abs(m4 - _iso4(1.0 / 3.0))) > 0.05


def test_tau_diffusion_map():
    # D = c_s^2 (tau - 1/2) with c_s^2 = 1/3 (end of Sec. II.A).
    assert orc.tau_from_diffusion(1.0 / 6.0) == 1.0
    assert orc.tau_from_diffusion(0.1) == pytest.approx(0.8, abs=1e-15)
    assert orc.tau_from_diffusion(0.05) == pytest.approx(0.65, abs=1e-15)
    assert orc.diffusion_from_tau(orc.tau_from_diffusion(0.02)) == pytest.approx(0.02, abs=1e-16)


# ---------------------------------------------------------------------------
# Step algebra: tau = 1 reduces to an explicit stencil on rho
# ---------------------------------------------------------------------------

def _brute_tau1(lat, rho, reaction, steps):
    """At tau = 1 the post-collision value is w_i (rho + R), so
    rho(x, t+1) = sum_i w_i (rho + R)(x - e_i, t).  Written with np.roll."""
    E, W = TABLES[lat]
    rho = rho.copy()
    for _ in range(steps):
        R = _reaction_np(reaction, rho)
        src = rho + R
        new = np.zeros_like(rho)
        for (ex, ey), w in zip(E, W):
            new += w * np.roll(src, shift=(ey, ex), axis=(1, 2))
        rho = new
    return rho


def _reaction_np(reaction, rho):
    if reaction.kind == "none":
        return np.zeros_like(rho)
    if reaction.kind == "linear":
        R = np.zeros_like(rho)
        R[0] = -reaction.kappa * rho[0]
        if rho.shape[0] == 2:
            R[1] = reaction.kappa * rho[0]
        return R
    # Eqs. reac_diff10/11 with A0 = k1 = 1, k_f = k_0 = F, k_2 = k.
    kf, k1, k2, A0 = reaction.F, 1.0, reaction.k, 1.0
    A, B = rho
    return np.stack([kf * (A0 - A) - k1 * B * B * A, -(kf + k2) * B + k1 * B * B * A])


@pytest.mark.parametrize("lat", ["D2Q9", "D2Q5"])
@pytest.mark.parametrize("reaction", [Reaction("none"), Reaction("linear", kappa=0.02),
                                      Reaction("gray_scott", F=0.04, k=0.06)])
def test_tau1_reduces_to_explicit_stencil(lat, reaction):
    S = 2 if reaction.kind == "gray_scott" else 1
    rng = np.random.default_rng(7)
    rho0 = 0.5 + rng.random((S, 11, 13))
    if S == 2:  # stay in the physical range u in [0.4, 1], v in [0, 0.3]
        rho0 = np.stack([0.4 + 0.6 * rng.random((11, 13)), 0.3 * rng.random((11, 13))])
    f = orc.init(lat, rho0)
    f = orc.run(lat, [1.0] * S, reaction, f, 6)
    got = orc.density(lat, f)
    want = _brute_tau1(lat, rho0, reaction, 6)
    np.testing.assert_allclose(got, want, rtol=1e-14, atol=1e-15)


# ---------------------------------------------------------------------------
# Fourier-mode decay (linear decay, decay_128 workload)
# ---------------------------------------------------------------------------

def _mode_amplitude(rho, n):
    nx = rho.shape[-1]
    c = np.cos(2 * np.pi * n * np.arange(nx) / nx)
    return 2.0 * np.mean(rho[0] * c[None, :])


@pytest.mark.parametrize("lat", ["D2Q9", "D2Q5"])
def test_fourier_decay_tau1_closed_form(lat):
    """tau = 1, kappa = 1e-3, mode 2 pi / 128 along x: every step multiplies the
    mode by G = (1 - kappa)(2/3 + cos k / 3) (D2Q9 and D2Q5 alike) and the mean
    by (1 - kappa).  The continuum rate D k^2 + kappa (Eq. reac_diff3 in
    Fourier space) agrees to the discretisation gap."""
    kappa, nx, ny, t = 1e-3, 128, 4, 2000
    rho0 = inputs.rho0_cosine(nx, ny, seed=1235, noise=0.0)
    f = orc.run(lat, [1.0], Reaction("linear", kappa=kappa), orc.init(lat, rho0), t)
    rho = orc.density(lat, f)
    k = 2 * np.pi / nx
    G = (1 - kappa) * (2.0 / 3.0 + np.cos(k) / 3.0)
    assert _mode_amplitude(rho, 1) == pytest.approx(0.1 * G ** t, rel=1e-10)
    assert rho.mean() == pytest.approx((1 - kappa) ** t, rel=1e-12)
    rate = -np.log(G)
    D = 1.0 / 6.0
    assert rate == pytest.approx(1.4020956e-3, rel=1e-7)
    assert rate == pytest.approx(D * k * k + kappa, rel=5e-4)
    assert abs(rate / (D * k * k + kappa) - 1) > 1e-4  # the gap is real, not zero


@pytest.mark.parametrize("lat,tau", [("D2Q9", 0.8), ("D2Q9", 0.65), ("D2Q5", 0.8), ("D2Q9", 1.7)])
def test_fourier_decay_matches_exact_symbol(lat, tau):
    """For tau != 1 the mode decays at the leading eigenvalue of the exact
    amplification matrix of the linearised step (``lb_symbol``)."""
    kappa, nx, ny = 1e-3, 64, 3
    rho0 = inputs.rho0_cosine(nx, ny, seed=1, noise=0.0)
    f = orc.run(lat, [tau], Reaction("linear", kappa=kappa), orc.init(lat, rho0), 200)
    a1 = _mode_amplitude(orc.density(lat, f), 1)
    f = orc.run(lat, [tau], Reaction("linear", kappa=kappa), f, 300)
    a2 = _mode_amplitude(orc.density(lat, f), 1)
    lam = orc.lb_growth_rate(lat, [tau], [[-kappa]], (2 * np.pi / nx, 0.0))
    assert abs(lam.imag) < 1e-12
    assert np.log(a2 / a1) / 300 == pytest.approx(lam.real, rel=1e-9)
    D = orc.diffusion_from_tau(tau)
    k2 = (2 * np.pi / nx) ** 2
    assert -lam.real == pytest.approx(D * k2 + kappa, rel=2e-2)


# ---------------------------------------------------------------------------
# Mass balance: sum_i f_eq = rho and sum_i w_i = 1 (Eq. equili, Eq. app11a)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("lat", ["D2Q9", "D2Q5"])
@pytest.mark.parametrize("S", [1, 2])
def test_mass_conserved_without_reaction(lat, S):
    rng = np.random.default_rng(3)
    rho0 = 0.2 + rng.random((S, 24, 31))
    taus = [0.8, 0.65][:S]
    f = orc.init(lat, rho0)
    m0 = rho0.sum(axis=(1, 2))
    f = orc.run(lat, taus, Reaction("none"), f, 500)
    m = orc.density(lat, f).sum(axis=(1, 2))
    np.testing.assert_allclose(m, m0, rtol=1e-13)


@pytest.mark.parametrize("S", [1, 2])
def test_mass_linear_decay_discrete(S):
    """With R_A = -kappa rho_A the LB mass follows M_A(t) = M_A(0) (1 - kappa)^t
    exactly (not exp(-kappa t)); with species B the total is conserved."""
    kappa, t = 0.01, 400
    rng = np.random.default_rng(4)
    rho0 = rng.random((S, 20, 22))
    if S == 2:
        rho0[1] = 0.0
    f = orc.run("D2Q9", [0.56] * S, Reaction("linear", kappa=kappa), orc.init("D2Q9", rho0), t)
    m = orc.density("D2Q9", f).sum(axis=(1, 2))
    mA0 = rho0[0].sum()
    assert m[0] == pytest.approx(mA0 * (1 - kappa) ** t, rel=1e-12)
    assert m[0] != pytest.approx(mA0 * math.exp(-kappa * t), rel=1e-3)
    if S == 2:
        assert m.sum() == pytest.approx(mA0, rel=1e-13)


# ---------------------------------------------------------------------------
# Gray-Scott, homogeneous dynamics (Sec. III.A)
# ---------------------------------------------------------------------------

def test_gs_uniform_field_is_forward_euler_of_kinetics():
    """A uniform field does not stream, and sum_i w_i R = R: one LB step is one
    forward-Euler step (dt = 1) of Eqs. reac_diff10/11 without diffusion."""
    F, k = 0.03, 0.055
    rho0 = np.empty((2, 5, 7))
    rho0[0], rho0[1] = 0.61, 0.27
    f = orc.init("D2Q9", rho0)
    A, B = 0.61, 0.27
    kf, k1, k2, A0 = F, 1.0, k, 1.0
    for t in range(1, 301):
        A, B = A + (kf * (A0 - A) - k1 * B * B * A), B + (-(kf + k2) * B + k1 * B * B * A)
        f = orc.step("D2Q9", [0.8, 0.65], Reaction("gray_scott", F=F, k=k), f)
        if t % 50 == 0:
            rho = orc.density("D2Q9", f)
            assert np.ptp(rho[0]) == 0.0 and np.ptp(rho[1]) == 0.0
            assert rho[0, 0, 0] == pytest.approx(A, rel=1e-14)
            assert rho[1, 0, 0] == pytest.approx(B, rel=1e-14)


def test_gs_P_decay_eq_reac_diff21():
    """tau = tau_A / tau_B = 1 means k = 0.  Then P = eta A + B - eta
    (dimensionless) decays: exactly (1 - F)^t per LB step and exp(-t / tau_A)
    in the continuum (Eq. reac_diff21 read with +B(0), as in the definition
    of P in Eq. reac_diff20)."""
    F, k = 0.02, 0.0
    d = orc.gs_dimensionless(F, k, 1.0, 1.0)
    assert d["tau"] == 1.0
    eta, B0 = d["eta"], d["B0"]
    u0, v0 = 0.5, 0.25
    rho0 = np.empty((2, 4, 4))
    rho0[0], rho0[1] = u0, v0
    P0 = eta * u0 + v0 / B0 - eta
    f = orc.init("D2Q9", rho0)
    for t in (25, 50, 100):
        f = orc.run("D2Q9", [0.8, 0.65], Reaction("gray_scott", F=F, k=k), f, 25 if t == 25 else (25 if t == 50 else 50))
        rho = orc.density("D2Q9", f)
        P = eta * rho[0, 0, 0] + rho[1, 0, 0] / B0 - eta
        assert P == pytest.approx(P0 * (1 - F) ** t, rel=1e-12)
        cont = P0 * math.exp(-t / d["tauA"])
        assert abs(P / cont - 1) <= F * F * t / 2 * 1.05


def test_gs_steady_states_are_fixed_points():
    """The states of Eq. reac_diff19 (and the trivial state) solve
    Eq. reac_diff18 and are fixed points of the LB step."""
    g = _golden("turing_fig7.json")
    F, k = orc.gs_params_from_dimensionless(g["eta"], g["tau"])
    d = orc.gs_dimensionless(F, k, 1.0, 1.0)
    assert d["eta"] == pytest.approx(g["eta"], rel=1e-12)
    for A, B in orc.gs_steady_states_dimensionless(d["eta"]).values():
        assert -B * B * A + 1 - A == pytest.approx(0.0, abs=1e-15)
        assert d["eta"] * B * B * A - B == pytest.approx(0.0, abs=1e-15)
    for u, v in orc.gs_steady_states(F, k).values():
        rho0 = np.empty((2, 3, 4))
        rho0[0], rho0[1] = u, v
        reac = Reaction("gray_scott", F=F, k=k)
        f = orc.step("D2Q9", [0.8, 0.65], reac, orc.init("D2Q9", rho0))
        rho = orc.density("D2Q9", f)
        # one step moves a fixed point by rounding only (a few ulp) ...
        np.testing.assert_allclose(rho[0], u, rtol=1e-15, atol=1e-17)
        np.testing.assert_allclose(rho[1], v, rtol=1e-15, atol=1e-17)
        # ... and 20 steps stay within the slow growth of that rounding
        # (the + state is a saddle, the - state Hopf-unstable here).
        f = orc.run("D2Q9", [0.8, 0.65], reac, f, 19)
        rho = orc.density("D2Q9", f)
        np.testing.assert_allclose(rho[0], u, rtol=1e-14, atol=1e-16)
        np.testing.assert_allclose(rho[1], v, rtol=1e-14, atol=1e-16)


def test_gs_saddle_node_at_eta_2():
    """F = 0.04, k = 0.06 gives eta = 2 exactly: the two non-trivial states of
    Eq. reac_diff19 merge at A = 1/2, B = 1 (u = 0.5, v = 0.2)."""
    d = orc.gs_dimensionless(0.04, 0.06, 0.1, 0.05)
    assert d["eta"] == pytest.approx(2.0, rel=1e-15)
    st = orc.gs_steady_states(0.04, 0.06)
    assert st["+"][0] == pytest.approx(0.5) and st["-"][0] == pytest.approx(0.5)
    assert st["+"][1] == pytest.approx(0.2) and st["-"][1] == pytest.approx(0.2)
    assert "+" not in orc.gs_steady_states(0.037, 0.06)  # eta < 2: trivial only


def test_gs_scales_match_fig10():
    """(F, k) = (0.025, 0.06) with D_A = 0.016, D_B = 0.008 reproduces the
    printed eta = 1.86, tau = 3.40, eps = 2.61 of Sec. IV / Fig. 10, and
    the D -> lambda^2 D rescale leaves them unchanged."""
    g = _golden("gs_fig10_scales.json")
    F, k = orc.gs_params_from_dimensionless(g["eta"], g["tau"])
    assert F == pytest.approx(0.025, rel=2e-3) and k == pytest.approx(0.06, rel=2e-3)
    for DA, DB in ((g["D_A"], g["D_B"]), (g["D_A_system2"], g["D_B_system2"])):
        d = orc.gs_dimensionless(0.025, 0.06, DA, DB)
        assert round(d["eta"], 2) == g["eta"]
        assert round(d["tau"], 2) == g["tau"]
        assert round(d["eps"], 2) == g["eps"]
    d1 = orc.gs_dimensionless(0.025, 0.06, g["D_A"], g["D_B"])
    d2 = orc.gs_dimensionless(0.025, 0.06, g["D_A_system2"], g["D_B_system2"])
    assert d2["lA"] / d1["lA"] == pytest.approx(g["lambda"], rel=1e-12)


# ---------------------------------------------------------------------------
# Linear stability (Sec. III.B, III.C)
# ---------------------------------------------------------------------------

def _turing_case(ratio=2.0, Du=0.1):
    g = _golden("turing_fig7.json")
    F, k = orc.gs_params_from_dimensionless(g["eta"], g["tau"])
    d = orc.gs_dimensionless(F, k, Du, Du / ratio)
    return g, F, k, d


def test_closed_form_trace_det_match_matrix():
    """The closed forms of tr M and |M| (Sec. III.C) equal the trace and
    determinant of M (Eq. reac_diff29), and of tau_A (J - D q^2) written in
    lattice variables, at the B- state."""
    g, F, k, d = _turing_case()
    A, B = orc.gs_steady_states_dimensionless(d["eta"])["-"]
    u, v = orc.gs_steady_states(F, k)["-"]
    J = orc.gs_jacobian(F, k, u, v)
    Dm = np.diag([0.1, 0.05])
    for q2 in (0.0, 0.3, 1.2, 3.0):
        M = orc.gs_matrix_M(d["eta"], d["tau"], d["eps2"], A, B, q2)
        tr, det = orc.gs_trace_det_M(d["eta"], d["tau"], d["eps2"], B, q2)
        assert np.trace(M) == pytest.approx(tr, rel=1e-12, abs=1e-12)
        assert np.linalg.det(M) == pytest.approx(det, rel=1e-10, abs=1e-12)
        # dimensionless time t~ = t / tau_A, length l_A: q = q~ / l_A
        L = d["tauA"] * (J - Dm * (q2 / d["lA"] ** 2))
        assert np.trace(L) == pytest.approx(tr, rel=1e-10, abs=1e-12)
        assert np.linalg.det(L) == pytest.approx(det, rel=1e-9, abs=1e-12)


def test_turing_and_hopf_sides():
    """eta = 2.0139, tau = 2.733 (Fig. 7): with D_A / D_B = 2, eps^2 = 5.466
    exceeds the exact Turing bound, so |M(q^2)| < 0 on a band of real positive
    growth; with D_A / D_B = 1, eps^2 = tau is below it and only the Hopf
    mode (tr M(0) > 0, complex pair) is unstable."""
    g, F, k, d = _turing_case(2.0)
    assert d["eps2"] == pytest.approx(g["eps2"], rel=1e-4)
    bound = orc.turing_space_lower_bound(d["eta"])
    assert bound == pytest.approx(4.4375, abs=2e-3)
    B = orc.gs_steady_states_dimensionless(d["eta"])["-"][1]
    lo, hi = orc.turing_band(d["eta"], d["eps2"], B)
    assert lo == pytest.approx(0.548, abs=2e-3) and hi == pytest.approx(2.653, abs=2e-3)
    mid = 0.5 * (lo + hi)
    assert orc.gs_trace_det_M(d["eta"], d["tau"], d["eps2"], B, mid)[1] < 0
    assert orc.hopf_unstable(d["eta"], d["tau"])
    _, _, _, d1 = _turing_case(1.0)
    assert d1["eps2"] < bound
    assert orc.turing_band(d1["eta"], d1["eps2"], B) is None or \
        max(orc.turing_band(d1["eta"], d1["eps2"], B)) <= 0
    tr0, det0 = orc.gs_trace_det_M(d1["eta"], d1["tau"], d1["eps2"], B, 0.0)
    assert tr0 == pytest.approx(0.468, abs=2e-3) and tr0 * tr0 - 4 * det0 < 0


def test_fig8_parameters_lie_in_turing_space():
    g = _golden("turing_fig8.json")
    for eta, tau in g["params"]:
        eps2 = tau * g["D_ratio"]
        assert eta > 2.0
        assert eps2 > orc.turing_space_lower_bound(eta)


@pytest.mark.parametrize("state,ratio,n,kind,amp,t1,dt", [
    ("-", 2.0, 22, "turing", (1e-6, 1e-6), 300, 200),
    ("-", 2.0, 40, "decay", (1e-6, 1e-6), 300, 200),
    # at (1, 0) with v = 0 exactly the u equation is exactly linear
    ("trivial", 2.0, 10, "decay", (0.1, 0.0), 100, 200)])
def test_linear_growth_rate_vs_exact_symbol(state, ratio, n, kind, amp, t1, dt):
    """A small cosine perturbation of mode n on L = 256 about a uniform steady
    state grows or decays at the leading eigenvalue of the 2Q x 2Q linearised
    LB symbol; inside the Turing band of the B- state (Fig. 7 parameters,
    D_u = 0.1, D_u / D_v = 2) it grows at a real rate within 5 % of the
    continuum eig(J - D q^2) (the gap is the first-order time error of the
    scheme, about 4 % of the rate already at q = 0)."""
    g, F, k, d = _turing_case(ratio)
    Du, Dv = 0.1, 0.1 / ratio
    u, v = orc.gs_steady_states(F, k)[state]
    nx, ny = 256, 2
    J = orc.gs_jacobian(F, k, u, v)
    taus = [orc.tau_from_diffusion(Du), orc.tau_from_diffusion(Dv)]
    kx = 2 * np.pi * n / nx
    lam = orc.lb_growth_rate("D2Q9", taus, J, (kx, 0.0))
    cont = orc.continuum_growth_rate(J, [Du, Dv], kx * kx)
    c = cont[np.argmax(cont.real)]
    assert abs(lam.imag) < 1e-12 and abs(c.imag) < 1e-14
    if kind == "turing":
        assert lam.real > 0 and c.real > 0
        q2 = kx * kx * d["lA"] ** 2
        B = orc.gs_steady_states_dimensionless(d["eta"])["-"][1]
        lo, hi = orc.turing_band(d["eta"], d["eps2"], B)
        assert lo < q2 < hi
        assert lam.real == pytest.approx(c.real, rel=5e-2)
    else:
        assert lam.real < 0 and c.real < 0
    x = np.arange(nx)
    pert = np.cos(kx * x)[None, :]
    rho0 = np.empty((2, ny, nx))
    rho0[0] = u + amp[0] * pert
    rho0[1] = v + amp[1] * pert
    reac = Reaction("gray_scott", F=F, k=k)
    f = orc.run("D2Q9", taus, reac, orc.init("D2Q9", rho0), t1)

    def amplitude(f):
        rho = orc.density("D2Q9", f)
        cc = np.cos(kx * x)
        return np.mean((rho[0] - u) * cc[None, :]) * 2

    a1 = amplitude(f)
    f = orc.run("D2Q9", taus, reac, f, dt)
    a2 = amplitude(f)
    assert min(abs(a1), abs(a2)) > 1e-9
    assert np.log(abs(a2 / a1)) / dt == pytest.approx(lam.real, rel=1e-5)


# ---------------------------------------------------------------------------
# Exact symmetry: periodic shift equivariance
# ---------------------------------------------------------------------------

def test_periodic_shift_equivariance_bitwise():
    rho0 = inputs.rho0_square(24, 20, seed=5, side=8)
    reac = Reaction("gray_scott", F=0.04, k=0.06)
    f1 = orc.run("D2Q9", [0.8, 0.65], reac, orc.init("D2Q9", rho0), 40)
    sh = (7, -5)
    f2 = orc.run("D2Q9", [0.8, 0.65], reac, orc.init("D2Q9", np.roll(rho0, sh, axis=(1, 2))), 40)
    np.testing.assert_array_equal(np.roll(f1, sh, axis=(2, 3)), f2)


def test_oracle_threads_do_not_change_results():
    rho0 = inputs.rho0_square(40, 36, seed=9, side=10)
    reac = Reaction("gray_scott", F=0.04, k=0.06)
    f = orc.run("D2Q9", [0.8, 0.65], reac, orc.init("D2Q9", rho0), 30)
    g = orc.init("D2Q9", rho0)
    for _ in range(30):
        g = orc.step("D2Q9", [0.8, 0.65], reac, g)
    np.testing.assert_array_equal(f, g)


# ---------------------------------------------------------------------------
# Analysis helpers
# ---------------------------------------------------------------------------

def test_structure_factor_peak_exact_modes():
    L = 200
    y, x = np.mgrid[0:L, 0:L]
    field = np.cos(2 * np.pi * (3 * x + 4 * y) / L) + 0.5 * np.cos(2 * np.pi * (4 * x - 3 * y) / L)
    res = orc.structure_factor_peak(field)
    assert res["shell"] == 5
    assert res["wavelength"] == pytest.approx(L / 5, rel=1e-12)
    assert orc.wave_number(3, 4, L, L) == pytest.approx(2 * np.pi * 5 / L)


def test_point_source_normalisation_and_error_metric():
    # Eq. reac_diff5 integrates to exp(-kappa t) on a domain much wider than sqrt(D t).
    rho = orc.point_source(200, 200, 100, 100, 0.02, 0.01, 400.0)
    assert rho.sum() == pytest.approx(math.exp(-4.0), rel=1e-9)
    assert orc.relative_error(rho, rho) == 0.0
    assert orc.relative_error(rho, 1.01 * rho) == pytest.approx(0.01, rel=1e-12)


# ---------------------------------------------------------------------------
# Order of accuracy of the point-source problem (Sec. II.B, appendix)
# ---------------------------------------------------------------------------

def _point_source_error(L, D, kappa, t, lat="D2Q9"):
    rho0 = np.zeros((1, L, L))
    rho0[0, L // 2, L // 2] = 1.0
    f = orc.run(lat, [float(orc.tau_from_diffusion(D))], Reaction("linear", kappa=kappa), orc.init(lat, rho0), t)
    an = orc.point_source(L, L, L // 2, L // 2, D, kappa, t)
    return orc.relative_error(an, orc.density(lat, f)[0])


@pytest.mark.parametrize("D,kappa", [(0.02, 0.0), (0.05, 0.04), (0.1, 0.132), (1.0 / 6.0, 0.04)])
def test_point_source_second_order_under_diffusive_refinement(D, kappa):
    """The Chapman-Enskog expansion of the appendix makes the scheme a
    second-order approximation of Eq. reac_diff3 under diffusive scaling
    (dx -> dx/2, dt -> dt/4: D fixed in lattice units, kappa/4, 4 t steps).
    E_rho of one physical problem must fall by 4 per level (a wrong weight,
    tau map or source term leaves an O(1) error that does not converge)."""
    L0, t0 = 50, int(round(2.0 / D))
    e = [_point_source_error(L0 * 2 ** l, D, kappa / 4 ** l, t0 * 4 ** l) for l in range(3)]
    assert e[0] / e[1] == pytest.approx(4.0, rel=0.06), e
    assert e[1] / e[2] == pytest.approx(4.0, rel=0.03), e


def test_point_source_fourth_order_at_tau_one():
    """At tau = 1 without reaction the update is rho(t + 1) = sum_i w_i rho(x - e_i)
    whose symbol (2/3 + cos(k_x)/3)(2/3 + cos(k_y)/3) agrees with
    exp(-D |k|^2) for D = 1/6 through |k|^4 (the first difference is the k^6
    term: 1/2160 against 1/1296), so under diffusive refinement the error
    falls by 2^4 = 16 per level, not 4."""
    kx = 1e-2
    sym = 2.0 / 3.0 + math.cos(kx) / 3.0
    assert abs(sym - math.exp(-kx * kx / 6.0)) < 2e-13  # O(k^6) ~ 1e-12 * (1/1296 - 1/2160)
    D = 1.0 / 6.0
    e = [_point_source_error(50 * 2 ** l, D, 0.0, 12 * 4 ** l) for l in range(3)]
    assert e[0] / e[1] > 14.0 and e[1] / e[2] > 14.0, e


def test_point_source_decay_error_is_kappa_squared_t():
    """Reading of Eq. relax for the source: the mass of A follows
    (1 - kappa)^t, while Eq. reac_diff5 decays as exp(-kappa t).  At
    D = 1/6 the diffusion error is fourth order and small, so E_rho is
    dominated by |1 - (1 - kappa)^t exp(kappa t)| ~ kappa^2 t / 2."""
    D, L, t = 1.0 / 6.0, 100, 48
    for kappa in (0.01, 0.02, 0.04):
        e = _point_source_error(L, D, kappa, t)
        amp = abs(1.0 - (1.0 - kappa) ** t * math.exp(kappa * t))
        assert e == pytest.approx(amp, rel=0.05), (kappa, e, amp)


# ---------------------------------------------------------------------------
# Mass-action networks (Eq. reac_diff1 for N species, built from reaction
# steps like those of Sec. III: U + 2V -> 3V, V -> P, feed and removal)
# ---------------------------------------------------------------------------

def _mass_action_R(rates, order, change, rho):
    """R_s = sum_r change[r][s] k_r prod_j rho_j^order[r][j], written out with
    numpy powers (the test's own evaluation)."""
    rho = np.asarray(rho, dtype=np.float64)
    R = np.zeros_like(rho)
    for kr, a, nu in zip(rates, order, change):
        p = kr * np.prod([rho[j] ** a[j] for j in range(len(a))], axis=0)
        for s in range(len(nu)):
            R[s] = R[s] + nu[s] * p
    return R


GS_NET = dict(order=[(1, 2), (0, 0), (1, 0), (0, 1)], change=[(-1, 1), (1, 0), (-1, 0), (0, -1)])


def _gs_network(F, k):
    return Reaction.network([1.0, F, F, F + k], GS_NET["order"], GS_NET["change"])


def test_network_transformation_equals_linear_kind_bitwise():
    """A -> B as a one-step network evaluates -kappa rho_A and +kappa rho_A
    exactly as the transformation source does."""
    rng = np.random.default_rng(11)
    rho0 = 1.0 + 0.3 * rng.random((2, 12, 17))
    taus = [0.8, 1.3]
    net = Reaction.network([0.02], [(1, 0)], [(-1, 1)])
    a = orc.run("D2Q9", taus, net, orc.init("D2Q9", rho0), 40)
    b = orc.run("D2Q9", taus, Reaction("linear", kappa=0.02), orc.init("D2Q9", rho0), 40)
    np.testing.assert_array_equal(a, b)


def test_network_gray_scott_matches_eqs_reac_diff10_11():
    """Gray-Scott from its reaction steps (U + 2V -> 3V at rate 1, feed of U
    at F, removal of U at F, V -> P at F + k) gives R_u = -u v^2 + F (1 - u),
    R_v = u v^2 - (F + k) v up to rounding, and the same trajectory."""
    F, k = 0.04, 0.06
    rng = np.random.default_rng(12)
    rho = rng.random((2, 50))
    R = np.stack([orc.default().reaction(_gs_network(F, k), rho[:, j]) for j in range(rho.shape[1])], axis=1)
    u, v = rho
    np.testing.assert_allclose(R[0], -u * v * v + F * (1 - u), rtol=1e-13, atol=1e-16)
    np.testing.assert_allclose(R[1], u * v * v - (F + k) * v, rtol=1e-13, atol=1e-16)
    rho0 = inputs.rho0_square(32, 32, seed=3, side=8)
    taus = [float(t) for t in orc.tau_from_diffusion(np.array([0.1, 0.05]))]
    a = orc.density("D2Q9", orc.run("D2Q9", taus, _gs_network(F, k), orc.init("D2Q9", rho0), 200))
    b = orc.density("D2Q9", orc.run("D2Q9", taus, Reaction("gray_scott", F=F, k=k), orc.init("D2Q9", rho0), 200))
    np.testing.assert_allclose(a, b, rtol=0, atol=1e-12)


def test_network_three_species_uniform_field_is_forward_euler():
    """A uniform field does not stream: rho(t + 1) = rho + R(rho), the forward
    Euler step of the kinetics (A + B <-> C, C -> 0, 0 -> A, 2 B -> B)."""
    rates = [0.3, 0.05, 0.02, 0.01, 0.07]
    order = [(1, 1, 0), (0, 0, 1), (0, 0, 1), (0, 0, 0), (0, 2, 0)]
    change = [(-1, -1, 1), (1, 1, -1), (0, 0, -1), (1, 0, 0), (0, -1, 0)]
    net = Reaction.network(rates, order, change)
    r = np.array([0.7, 0.4, 0.2])
    f = orc.init("D2Q9", np.broadcast_to(r[:, None, None], (3, 5, 6)).copy())
    taus = [0.7, 0.9, 1.4]
    for _ in range(30):
        f = orc.step("D2Q9", taus, net, f)
        r = r + _mass_action_R(rates, order, change, r)
        np.testing.assert_allclose(orc.density("D2Q9", f)[:, 2, 3], r, rtol=1e-13)


def test_network_conservative_cycle_keeps_total_mass():
    """Four species in a cycle A -> B -> C -> D -> A plus 2 A -> A + B: every
    step has sum_s nu_rs = 0, so the total over species is conserved while
    each species' own mass changes."""
    rates = [0.02, 0.03, 0.05, 0.01, 0.04]
    order = [(1, 0, 0, 0), (0, 1, 0, 0), (0, 0, 1, 0), (0, 0, 0, 1), (2, 0, 0, 0)]
    change = [(-1, 1, 0, 0), (0, -1, 1, 0), (0, 0, -1, 1), (1, 0, 0, -1), (-1, 1, 0, 0)]
    net = Reaction.network(rates, order, change)
    rng = np.random.default_rng(13)
    rho0 = 0.5 + rng.random((4, 20, 24))
    f = orc.run("D2Q5", [0.6, 0.8, 1.0, 1.7], net, orc.init("D2Q5", rho0), 150)
    m0, m1 = rho0.sum(axis=(1, 2)), orc.density("D2Q5", f).sum(axis=(1, 2))
    assert m1.sum() == pytest.approx(m0.sum(), rel=1e-13)
    assert np.max(np.abs(m1 - m0)) > 1.0


def test_network_three_species_mode_growth_matches_symbol():
    """A small cosine mode about a uniform state of a linear three-species
    network (A -> B -> C -> A) evolves with the leading eigenvalue of the
    3Q x 3Q linearised step (the exact amplification matrix)."""
    rates = [0.03, 0.02, 0.05]
    order = [(1, 0, 0), (0, 1, 0), (0, 0, 1)]
    change = [(-1, 1, 0), (0, -1, 1), (1, 0, -1)]
    net = Reaction.network(rates, order, change)
    J = np.zeros((3, 3))
    for kr, a, nu in zip(rates, order, change):
        j = int(np.argmax(a))
        for s in range(3):
            J[s, j] += nu[s] * kr
    L, n = 64, 3
    taus = [0.9, 0.7, 1.2]
    x = np.arange(L)
    base = np.array([1.0, 1.5, 0.6])  # J base = 0: 0.03 = 0.02 * 1.5 = 0.05 * 0.6
    vec = np.array([1.0, -0.4, 0.3])
    rho0 = base[:, None, None] + 1e-6 * vec[:, None, None] * np.cos(2 * np.pi * n * x / L)[None, None, :]
    rho0 = np.broadcast_to(rho0, (3, 4, L)).copy()
    kvec = (2 * np.pi * n / L, 0.0)
    lam = np.max(np.abs(np.linalg.eigvals(orc.lb_symbol("D2Q9", taus, J, kvec))))
    f = orc.init("D2Q9", rho0)
    amps = []
    for t in range(400):
        f = orc.step("D2Q9", taus, net, f)
        if t >= 200:
            d = orc.density("D2Q9", f)[0, 0] - base[0]
            amps.append(np.abs(np.fft.rfft(d)[n]))
    rate = (amps[-1] / amps[0]) ** (1.0 / (len(amps) - 1))
    assert rate == pytest.approx(lam, rel=1e-6)


def test_network_schnakenberg_fixed_point():
    """Schnakenberg kinetics u' = c (a - u + u^2 v), v' = c (b - u^2 v) from
    its steps (0 -> U at c a, U -> 0 at c, 2U + V -> 3U at c, 0 -> V at c b):
    the uniform state u = a + b, v = b / (a + b)^2 is a fixed point of the
    step (c = 0.05 keeps the per-step Euler map stable there, so rounding does
    not grow)."""
    a, b, c = 0.1, 0.9, 0.05
    net = Reaction.network([c * a, c, c, c * b], [(0, 0), (1, 0), (2, 1), (0, 0)], [(1, 0), (-1, 0), (1, -1), (0, 1)])
    u, v = a + b, b / (a + b) ** 2
    f = orc.init("D2Q9", np.stack([np.full((6, 7), u), np.full((6, 7), v)]))
    f = orc.run("D2Q9", [0.8, 1.1], net, f, 50)
    rho = orc.density("D2Q9", f)
    assert np.max(np.abs(rho[0] - u)) < 1e-13 and np.max(np.abs(rho[1] - v)) < 1e-13


@pytest.mark.parametrize("lat", ["D2Q9", "D2Q5"])
@pytest.mark.parametrize("tau", [0.6, 0.8, 1.2, 1.5])
def test_dispersion_fourth_order_term_closed_form(lat, tau):
    """Truncation trend in tau (Chapman-Enskog, appendix): for a mode along a
    lattice axis both lattices reduce to three velocities with weights
    (2/3, 1/6, 1/6), and expanding the leading eigenvalue of that 3 x 3 BGK
    symbol in k gives the decay rate -log(lambda) = D k^2 + c4 k^4 + O(k^6)
    with D = (tau - 1/2)/3 and c4 = -tau (tau - 1/2)(tau - 1)/9 (series of the
    characteristic polynomial, done by hand and by computer algebra).  So the
    gap to the continuum rate D k^2 falls by 16 when k halves, changes sign at
    tau = 1, and vanishes to fourth order there."""
    D = (tau - 0.5) / 3.0
    c4 = -tau * (tau - 0.5) * (tau - 1.0) / 9.0
    for k in (0.04, 0.02):
        lam = np.max(np.abs(np.linalg.eigvals(orc.lb_symbol(lat, [tau], np.zeros((1, 1)), (k, 0.0)))))
        gap = -math.log(lam) - D * k * k
        assert gap / k ** 4 == pytest.approx(c4, rel=0.02), (k, gap / k ** 4, c4)


@pytest.mark.parametrize("lat", ["D2Q9", "D2Q5"])
def test_dispersion_sixth_order_at_tau_one(lat):
    """At tau = 1 the k^4 term vanishes: the gap falls by 2^6 when k halves."""
    gaps = []
    for k in (0.08, 0.04):
        lam = np.max(np.abs(np.linalg.eigvals(orc.lb_symbol(lat, [1.0], np.zeros((1, 1)), (k, 0.0)))))
        gaps.append(-math.log(lam) - k * k / 6.0)
    assert gaps[0] / gaps[1] == pytest.approx(64.0, rel=0.02), gaps
