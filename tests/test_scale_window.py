"""Scale invariance of Sec. IV on the FP64 oracle (CPU): the window in which
the lattice keeps it, and the break-down below the resolution floor.

Multiplying every diffusion coefficient by lambda^2 leaves the Gray-Scott
scales eta, tau and eps unchanged and multiplies every length by lambda
(Sec. IV), so a Turing pattern grown on lambda L with lambda^2 D has lambda
times the wavelength.  The lattice keeps this only while the pattern is
resolved and tau stays moderate.  At eta = 2.014, tau = 2.733 (Figs. 11-12),
D_u / D_v = 2, D_u = 0.08 (L / 128)^2, 20000 steps from the B- state plus a
scale-free perturbation: L = 128 -> 192 keeps the mode number to 0.4 %
(inside the window), L = 64 (about five sites per wavelength) misses it by
12.6 %.  The tau side (L = 512, tau_u = 4.34: +10.2 %) takes minutes on the
host and is checked on the GPU path.
"""
import numpy as np
import pytest

import oracle as orc
from oracle import Reaction
from paper_1007_3109_gb300 import inputs


def _oracle_wavelength(L, Du, steps=20000):
    F, k = orc.gs_params_from_dimensionless(2.014, 2.733)
    u, v = orc.gs_steady_states(F, k)["-"]
    pert = inputs.fourier_perturbation(L, 1242)
    rho0 = np.stack([u + 1e-3 * pert[0], v + 1e-3 * pert[1]])
    taus = [float(orc.tau_from_diffusion(Du)), float(orc.tau_from_diffusion(Du / 2))]
    f = orc.run("D2Q9", taus, Reaction("gray_scott", F=F, k=k), orc.init("D2Q9", rho0), steps)
    return orc.structure_factor_peak(orc.density("D2Q9", f)[1])


@pytest.fixture(scope="module")
def base128():
    return _oracle_wavelength(128, 0.08)


def test_rescaled_pattern_inside_the_window(base128):
    got = _oracle_wavelength(192, 0.18)
    assert base128["shell"] >= 10, base128  # a Turing pattern formed
    assert got["wavelength"] / base128["wavelength"] == pytest.approx(1.5, rel=0.02), (got, base128)
    assert got["n_mean"] == pytest.approx(base128["n_mean"], rel=0.02)


def test_rescaled_pattern_breaks_below_the_resolution_floor(base128):
    got = _oracle_wavelength(64, 0.02)
    assert got["wavelength"] < 6.0  # about five sites per wavelength
    ratio = got["wavelength"] / base128["wavelength"] / 0.5
    assert ratio > 1.05, (got, base128)
