"""Long runs: the gs_512 workload over its full 20000 steps, and the
scale-invariance experiment of Sec. IV.

* FP64: the GPU path performs the oracle's operations in the oracle's order,
  so even the chaotic 20000-step run is bit-identical.
* FP32 and 16-bit deviation storage diverge pointwise from the FP64 run after
  a short horizon (the instability amplifies rounding); after the horizon they
  are compared by the dominant pattern wavelength (structure-factor peak,
  Eq. reac_diff35 read as in the oracle's structure_factor_peak), within 2 %.
* Sec. IV: multiplying every diffusion coefficient by lambda^2 leaves eta, tau
  and eps unchanged and scales lengths by lambda; a Turing pattern grown on
  L = 256 with 4 D has twice the wavelength of the one on L = 128 with D.
"""
import numpy as np
import pytest

import oracle as orc
from oracle import Reaction
from paper_1007_3109_gb300 import binding as B
from paper_1007_3109_gb300 import inputs

pytestmark = pytest.mark.gpu

T_FULL = inputs.WORKLOADS["gs_512"]["steps"]


def _gs512_setup():
    w = inputs.WORKLOADS["gs_512"]
    rho0 = inputs.initial_density("gs_512")
    taus = [float(t) for t in orc.tau_from_diffusion(np.array(w["D"]))]
    return w, rho0, taus


@pytest.fixture(scope="module")
def oracle_20000():
    w, rho0, taus = _gs512_setup()
    f = orc.run("D2Q9", taus, Reaction("gray_scott", F=0.04, k=0.06), orc.init("D2Q9", rho0), T_FULL)
    return orc.density("D2Q9", f)


def _gpu(precision, steps):
    w, rho0, taus = _gs512_setup()
    with B.Simulation("D2Q9", 2, 512, 512, taus, "gray_scott", F=0.04, k=0.06, precision=precision) as sim:
        sim.init(rho0).step(steps)
        return sim.moments()[0]


@pytest.mark.timeout(900)
def test_gs_512_full_run_fp64_bit_identical(oracle_20000):
    np.testing.assert_array_equal(_gpu("fp64", T_FULL), oracle_20000)


@pytest.mark.timeout(900)
@pytest.mark.parametrize("precision", ["fp32", "fp32_bf16dev", "fp32_fp16dev"])
def test_gs_512_full_run_wavelength_within_2pct(oracle_20000, precision):
    ref = orc.structure_factor_peak(oracle_20000[1])
    got = orc.structure_factor_peak(_gpu(precision, T_FULL)[1])
    assert ref["shell"] > 10, "a pattern must have formed for the comparison to mean anything"
    assert got["wavelength"] == pytest.approx(ref["wavelength"], rel=0.02), (got, ref)


def test_scale_invariance_turing_pattern():
    """eta = 2.014, tau = 2.733 (Figs. 11-12), D_u / D_v = 2: the pattern of
    (L = 256, 4 D) has twice the dominant wavelength of (L = 128, D) at the
    same time (the reaction time scale is unchanged)."""
    F, k = orc.gs_params_from_dimensionless(2.014, 2.733)
    u, v = orc.gs_steady_states(F, k)["-"]
    rng = np.random.default_rng(5)
    base = rng.standard_normal((2, 64, 64))
    lam_dom = {}
    for lam, L, Du in ((1, 128, 0.08), (2, 256, 0.32)):
        d1 = orc.gs_dimensionless(F, k, 0.08, 0.04)
        d2 = orc.gs_dimensionless(F, k, Du, Du / 2)
        assert d2["eps2"] == pytest.approx(d1["eps2"]) and d2["lA"] == pytest.approx(lam * d1["lA"])
        pert = np.kron(base, np.ones((2 * lam, 2 * lam)))  # the same field on the finer grid
        pert -= pert.mean(axis=(1, 2), keepdims=True)
        rho0 = np.stack([u + 1e-3 * pert[0], v + 1e-3 * pert[1]])
        taus = [float(orc.tau_from_diffusion(Du)), float(orc.tau_from_diffusion(Du / 2))]
        with B.Simulation("D2Q9", 2, L, L, taus, "gray_scott", F=F, k=k, precision="fp32") as sim:
            sim.init(rho0).step(20000)
            lam_dom[lam] = orc.structure_factor_peak(sim.moments()[0][1])["wavelength"]
    assert lam_dom[2] / lam_dom[1] == pytest.approx(2.0, rel=0.02), lam_dom
