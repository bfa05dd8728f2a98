"""Host-side analysis of simulation output: the closed forms and diagnostics
the paper compares its lattice Boltzmann runs against.

* ``point_source`` / ``relative_error``: the infinite-domain solution of the
  decay problem A -> B (Sec. II.B, Eq. reac_diff5) and the relative error
  E_rho defined after it.
* ``dominant_wavelength``: the pattern wavelength from the Fourier spectrum of
  a periodic field (Sec. III.D, Eq. reac_diff35).
* ``gs_classify``: linear-stability label of a Gray-Scott parameter pair
  (Sec. III.B-C): only the trivial state exists, or the non-trivial state
  with the larger v (the paper's B-) is Hopf unstable (tr J > 0), Turing
  unstable (unstable for a band of wave numbers q > 0), both, or stable.  Worked in lattice variables with J - q^2 diag(D_u, D_v); the
  paper's dimensionless groups (eta, tau, eps) give the same sets.

numpy only; nothing here touches the device.
"""
from __future__ import annotations

import math

import numpy as np


def point_source(nx: int, ny: int, x0: float, y0: float, D: float, kappa: float, t: float) -> np.ndarray:
    """rho_A(x, y, t) of a unit point source at (x0, y0) diffusing with D and
    decaying at rate kappa on an unbounded plane, sampled at the integer
    sites of an ny x nx grid (Eq. reac_diff5)."""
    ys = np.arange(ny, dtype=np.float64)[:, None] - y0
    xs = np.arange(nx, dtype=np.float64)[None, :] - x0
    spread = 4.0 * D * t
    return np.exp(-(xs * xs + ys * ys) / spread) * (math.exp(-kappa * t) / (math.pi * spread))


def relative_error(analytic: np.ndarray, simulated: np.ndarray) -> float:
    """E_rho = ||rho_an - rho_sim||_2 / ||rho_an||_2 over all sites (Sec. II.B)."""
    a = np.asarray(analytic, dtype=np.float64).ravel()
    d = a - np.asarray(simulated, dtype=np.float64).ravel()
    return float(math.sqrt(float(d @ d) / float(a @ a)))


def dominant_wavelength(field: np.ndarray) -> dict:
    """Dominant wavelength of a periodic square field (Eq. reac_diff35).

    The power |DFT(field - mean)|^2 of every mode n = (n_x, n_y) is binned
    by the nearest integer of |n|; the bin of most power (the smaller |n| on
    a tie, |n| = 0 excluded) and its two neighbours on each side give the
    power-weighted mean |n|; the wavelength is L over that mean.  Returns
    {"shell", "n_mean", "wavelength", "q"} with q = 2 pi n_mean / L.
    """
    f = np.asarray(field, dtype=np.float64)
    ny, nx = f.shape
    if nx != ny:
        raise ValueError("dominant_wavelength expects a square field")
    power = np.abs(np.fft.fft2(f - f.mean())) ** 2
    m = np.fft.fftfreq(nx, d=1.0 / nx)
    mag = np.hypot(m[:, None], m[None, :])
    shells = np.rint(mag).astype(np.int64)
    per_shell = np.zeros(int(shells.max()) + 1)
    np.add.at(per_shell, shells.ravel(), power.ravel())
    per_shell[0] = -np.inf
    p = int(np.argmax(per_shell))
    near = (shells >= max(1, p - 2)) & (shells <= p + 2)
    n_mean = float((mag[near] * power[near]).sum() / power[near].sum())
    return {"shell": p, "n_mean": n_mean, "wavelength": nx / n_mean, "q": 2.0 * math.pi * n_mean / nx}


def gs_states(F: float, k: float) -> list[tuple[float, float]]:
    """Uniform steady states of R_u = -u v^2 + F (1 - u), R_v = u v^2 - (F + k) v:
    (1, 0) and, when F >= 4 (F + k)^2, the two states with
    v = F (1 +- sqrt(1 - 4 (F + k)^2 / F)) / (2 (F + k)), u = 1 - (F + k) v / F
    (larger v first)."""
    out = [(1.0, 0.0)]
    g = F + k
    disc = 1.0 - 4.0 * g * g / F
    if disc >= 0.0:
        r = math.sqrt(disc)
        for v in (F * (1.0 + r) / (2.0 * g), F * (1.0 - r) / (2.0 * g)):
            out.append((1.0 - g * v / F, v))
    return out


def gs_classify(F: float, k: float, Du: float, Dv: float) -> dict:
    """Linear-stability label of the Gray-Scott pair (F, k) with diffusion
    coefficients (Du, Dv).

    "trivial": only (1, 0) exists (it is stable to small perturbations for
    every q).  Otherwise the state of larger v is examined with
    J = [[-v^2 - F, -2 u v], [v^2, 2 u v - (F + k)]] (det J > 0 there):
    it is Turing unstable when det(J - q^2 D) < 0 for a band of q^2 > 0 and
    Hopf unstable when tr J > 0 (a growing oscillation at q = 0).  Labels:
    "turing", "hopf", "turing+hopf" (both) or "stable" (neither).  The
    Turing band [q1^2, q2^2] is the positive root pair of det(J - q^2 D) = 0.
    """
    states = gs_states(F, k)
    if len(states) == 1:
        return {"label": "trivial", "state": states[0], "band": None}
    u, v = states[1]
    j11, j12 = -v * v - F, -2.0 * u * v
    j21, j22 = v * v, 2.0 * u * v - (F + k)
    tr, det = j11 + j22, j11 * j22 - j12 * j21
    # det(J - q^2 D) = Du Dv q^4 - (Dv j11 + Du j22) q^2 + det J
    a, b, c = Du * Dv, -(Dv * j11 + Du * j22), det
    band = None
    disc = b * b - 4.0 * a * c
    if disc > 0.0 and -b > 0.0:
        r = math.sqrt(disc)
        lo, hi = (-b - r) / (2.0 * a), (-b + r) / (2.0 * a)
        if hi > 0.0:
            band = (max(lo, 0.0), hi)
    turing = det > 0.0 and band is not None and band[0] > 0.0
    if det <= 0.0:
        label = "saddle"
    elif tr > 0.0:
        label = "turing+hopf" if turing else "hopf"
    else:
        label = "turing" if turing else "stable"
    return {"label": label, "state": (u, v), "band": band, "trace": tr, "det": det}


def pattern_outcome(v: np.ndarray, decayed_below: float = 1e-3, uniform_below: float = 1e-3) -> dict:
    """Outcome of a Gray-Scott run from its final v field (periodic, square).

    "decayed": max v < decayed_below (back at the trivial state u = 1, v = 0);
    "uniform": v nearly constant, std(v) < uniform_below * mean(v) (a uniform
    non-trivial state); "pattern" otherwise, with the dominant wavelength of
    ``dominant_wavelength``.
    """
    v = np.asarray(v, dtype=np.float64)
    vmax, mean, std = float(v.max()), float(v.mean()), float(v.std())
    out = {"vmax": vmax, "mean": mean, "std": std, "wavelength": None}
    if vmax < decayed_below:
        out["outcome"] = "decayed"
    elif std < uniform_below * abs(mean):
        out["outcome"] = "uniform"
    else:
        out["outcome"] = "pattern"
        out["wavelength"] = dominant_wavelength(v)["wavelength"]
    return out
