"""FP64 CPU oracle: the LB reaction-diffusion step plus the paper's analysis.

TEST INFRASTRUCTURE ONLY -- imported by the tests, the smoke check and the
benchmark's CPU-baseline leg, never by the library.  Two halves:

* ``OracleLib``: ctypes front end of ``lbrd_oracle.c`` (plain scalar C, FP64,
  no FMA contraction, OpenMP over rows), which applies the LB equation of
  Sec. II.A (Eq. relax, multi-species form) literally as collide-then-push.
* Closed forms of the paper, in numpy: the D <-> tau map (end of Sec. II.A,
  Eq. app22), the Gray-Scott scalings (Sec. III, Eqs. reac_diff12 to
  reac_diff17), the homogeneous steady states (Eq. reac_diff19), the linear
  stability matrices (Eqs. reac_diff24, reac_diff29, reac_diff32), the point
  source solution (Eq. reac_diff5), the relative error E_rho (Sec. II.B), the
  excited wave numbers (Eq. reac_diff35) and the exact Fourier symbol of the
  linearised LB step used to pin the oracle.

Each function states the passage it follows.  Where the paper is garbled or
silent the reading taken is stated beside the code.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import tempfile
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbrd_oracle.c")
_LIB = os.path.join(_HERE, "liblbrd_oracle.so")

LATTICES = {"D2Q9": 0, "D2Q5": 1}
REACTIONS = {"none": 0, "linear": 1, "gray_scott": 2, "mass_action": 3}
CS2 = 1.0 / 3.0  # lattice sound speed squared, c_s^2 = dx^2 / (3 dt^2) (Sec. II.A)

__all__ = [
    "LATTICES", "REACTIONS", "CS2", "Reaction", "OracleLib", "build", "default",
    "lattice", "init", "step", "run", "density", "threads", "set_threads",
    "tau_from_diffusion", "diffusion_from_tau", "gs_dimensionless",
    "gs_params_from_dimensionless", "gs_steady_states_dimensionless",
    "gs_steady_states", "gs_jacobian", "gs_matrix_M", "gs_trace_det_M",
    "turing_band", "turing_space_lower_bound", "hopf_unstable",
    "lb_symbol", "lb_growth_rate", "continuum_growth_rate",
    "point_source", "relative_error", "wave_number", "structure_factor_peak",
]


@dataclass(frozen=True)
class Reaction:
    """Reaction source R_s(rho_1..rho_S).

    kind "none": R = 0.  kind "linear": transformation A -> B at rate kappa
    (Sec. II.B, Eq. reac_diff2): R_A = -kappa rho_A (and R_B = +kappa rho_A for
    a second species).  kind "gray_scott": Pearson's lattice form of
    Eqs. reac_diff10/11 with A0 = k1 = 1, k_f = F, k_2 = k:
    R_u = -u v^2 + F(1 - u), R_v = u v^2 - (F + k) v.
    """

    kind: str = "none"
    kappa: float = 0.0
    F: float = 0.0
    k: float = 0.0
    rates: tuple = ()
    order: tuple = ()
    change: tuple = ()

    @property
    def code(self) -> int:
        return REACTIONS[self.kind]

    @staticmethod
    def network(rates, order, change) -> "Reaction":
        """Mass-action network (Eq. reac_diff1 for N species built from
        reaction steps): step r runs at rate_r = k_r prod_j rho_j^order[r][j]
        and changes species s by change[r][s], R_s = sum_r change[r][s] rate_r.
        Evaluated in the compiled oracle as p = k_r, p *= rho_j (order[r][j]
        times, j ascending), R_s += change[r][s] * p (reactions in order,
        zero changes skipped)."""
        return Reaction("mass_action", rates=tuple(float(r) for r in rates),
                        order=tuple(tuple(int(a) for a in row) for row in order),
                        change=tuple(tuple(int(c) for c in row) for row in change))

    def _arrays(self, S):
        nr = len(self.rates)
        rate = np.ascontiguousarray(self.rates, dtype=np.float64)
        order = np.ascontiguousarray(np.asarray(self.order, dtype=np.int32).reshape(nr, S))
        change = np.ascontiguousarray(np.asarray(self.change, dtype=np.int32).reshape(nr, S))
        return nr, rate, order, change


def build(out: str = _LIB, src: str = _SRC, cc: str = "gcc") -> str:
    """Compile the oracle C file into a shared library (gcc, FP64, no FMA)."""
    cmd = [cc, "-O2", "-std=c99", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
           "-fPIC", "-shared", src, "-o", out]
    subprocess.run(cmd, check=True)
    return out


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _iptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


class OracleLib:
    """ctypes front end of one compiled copy of ``lbrd_oracle.c``."""

    def __init__(self, path: str = _LIB):
        if not os.path.exists(path) or (path == _LIB and os.path.getmtime(path) < os.path.getmtime(_SRC)):
            build(path)
        self.path = path
        L = ctypes.CDLL(path)
        i64, dp, ip, i32, f64 = ctypes.c_int64, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int), ctypes.c_int, ctypes.c_double
        L.orc_lattice.argtypes = [i32, ip, ip, dp]
        L.orc_lattice.restype = i32
        L.orc_reaction.argtypes = [i32, f64, f64, f64, i32, dp, dp]
        L.orc_reaction.restype = None
        L.orc_init.argtypes = [i32, i32, i64, i64, dp, dp]
        L.orc_init.restype = i32
        L.orc_density.argtypes = [i32, i32, i64, i64, dp, dp]
        L.orc_density.restype = i32
        L.orc_step.argtypes = [i32, i32, i64, i64, dp, i32, f64, f64, f64, dp, dp]
        L.orc_step.restype = i32
        L.orc_run.argtypes = [i32, i32, i64, i64, dp, i32, f64, f64, f64, i64, dp, dp]
        L.orc_run.restype = i32
        ip32 = ctypes.POINTER(ctypes.c_int32)
        L.orc_network_reaction.argtypes = [i32, i32, dp, ip32, ip32, dp, dp]
        L.orc_network_reaction.restype = i32
        L.orc_run_network.argtypes = [i32, i32, i64, i64, dp, i32, dp, ip32, ip32, i64, dp, dp]
        L.orc_run_network.restype = i32
        L.orc_threads.argtypes = []
        L.orc_threads.restype = i32
        L.orc_set_threads.argtypes = [i32]
        L.orc_set_threads.restype = i32
        self.L = L

    # -- lattice ----------------------------------------------------------
    def lattice(self, lat):
        """(ex, ey, w) of the velocity set (Eq. Weights for D2Q9)."""
        code = LATTICES[lat] if isinstance(lat, str) else int(lat)
        ex = (ctypes.c_int * 9)()
        ey = (ctypes.c_int * 9)()
        w = np.zeros(9)
        Q = self.L.orc_lattice(code, ex, ey, _dptr(w))
        if Q == 0:
            raise ValueError(f"unknown lattice {lat!r}")
        return np.array(ex[:Q]), np.array(ey[:Q]), w[:Q].copy()

    def reaction(self, reaction: Reaction, rho):
        rho = np.ascontiguousarray(rho, dtype=np.float64)
        R = np.zeros_like(rho)
        if reaction.kind == "mass_action":
            nr, rate, order, change = reaction._arrays(len(rho))
            _check(self.L.orc_network_reaction(len(rho), nr, _dptr(rate), _iptr(order), _iptr(change),
                                               _dptr(rho), _dptr(R)))
            return R
        self.L.orc_reaction(reaction.code, reaction.kappa, reaction.F, reaction.k, len(rho), _dptr(rho), _dptr(R))
        return R

    # -- state --------------------------------------------------------------
    def init(self, lat, rho0):
        """Equilibrium state f_i,s = w_i rho0_s (Eq. equili), shape (S, Q, ny, nx)."""
        rho0 = np.ascontiguousarray(rho0, dtype=np.float64)
        S, ny, nx = rho0.shape
        Q = len(self.lattice(lat)[2])
        f = np.empty((S, Q, ny, nx))
        rc = self.L.orc_init(_code(lat), S, nx, ny, _dptr(rho0), _dptr(f))
        _check(rc)
        return f

    def density(self, lat, f):
        """rho_s = sum_i f_i,s (the moment below Eq. relax), shape (S, ny, nx)."""
        f = np.ascontiguousarray(f, dtype=np.float64)
        S, Q, ny, nx = f.shape
        rho = np.empty((S, ny, nx))
        _check(self.L.orc_density(_code(lat), S, nx, ny, _dptr(f), _dptr(rho)))
        return rho

    def step(self, lat, taus, reaction: Reaction, f):
        """One LB time step (Eq. relax, multi-species form); returns a new array."""
        if reaction.kind == "mass_action":
            return self.run(lat, taus, reaction, f, 1)
        f = np.ascontiguousarray(f, dtype=np.float64)
        S, Q, ny, nx = f.shape
        tau = np.ascontiguousarray(np.broadcast_to(np.asarray(taus, dtype=np.float64), (S,)))
        out = np.empty_like(f)
        _check(self.L.orc_step(_code(lat), S, nx, ny, _dptr(tau), reaction.code, reaction.kappa,
                               reaction.F, reaction.k, _dptr(f), _dptr(out)))
        return out

    def run(self, lat, taus, reaction: Reaction, f, nsteps: int):
        """nsteps LB time steps; returns a new array (the input is not modified)."""
        f = np.array(f, dtype=np.float64, order="C", copy=True)
        S, Q, ny, nx = f.shape
        tau = np.ascontiguousarray(np.broadcast_to(np.asarray(taus, dtype=np.float64), (S,)))
        tmp = np.empty_like(f)
        if reaction.kind == "mass_action":
            nr, rate, order, change = reaction._arrays(S)
            _check(self.L.orc_run_network(_code(lat), S, nx, ny, _dptr(tau), nr, _dptr(rate), _iptr(order),
                                          _iptr(change), int(nsteps), _dptr(f), _dptr(tmp)))
            return f
        _check(self.L.orc_run(_code(lat), S, nx, ny, _dptr(tau), reaction.code, reaction.kappa,
                              reaction.F, reaction.k, int(nsteps), _dptr(f), _dptr(tmp)))
        return f

    def threads(self) -> int:
        return int(self.L.orc_threads())

    def set_threads(self, n: int) -> int:
        """Threads of the parallel loops from now on (timing only; results do
        not depend on it)."""
        return int(self.L.orc_set_threads(int(n)))


def _code(lat) -> int:
    return LATTICES[lat] if isinstance(lat, str) else int(lat)


def _check(rc: int):
    if rc != 0:
        raise ValueError(f"oracle rejected the arguments (status {rc})")


_DEFAULT: OracleLib | None = None


def default() -> OracleLib:
    global _DEFAULT
    if _DEFAULT is None:
        _DEFAULT = OracleLib()
    return _DEFAULT


def lattice(lat):
    return default().lattice(lat)


def init(lat, rho0):
    return default().init(lat, rho0)


def step(lat, taus, reaction, f):
    return default().step(lat, taus, reaction, f)


def run(lat, taus, reaction, f, nsteps):
    return default().run(lat, taus, reaction, f, nsteps)


def density(lat, f):
    return default().density(lat, f)


def threads() -> int:
    return default().threads()


def set_threads(n: int) -> int:
    return default().set_threads(n)


# ---------------------------------------------------------------------------
# Closed forms of the paper
# ---------------------------------------------------------------------------

def tau_from_diffusion(D):
    """tau_s = D_s / (c_s^2 dt) + 1/2 with dt = 1 (end of Sec. II.A; Eq. app22)."""
    return np.asarray(D, dtype=np.float64) / CS2 + 0.5


def diffusion_from_tau(tau):
    """D_s = c_s^2 dt (tau_s - 1/2) with dt = 1 (end of Sec. II.A; Eq. app22)."""
    return CS2 * (np.asarray(tau, dtype=np.float64) - 0.5)


def gs_dimensionless(F: float, k: float, Du: float, Dv: float) -> dict:
    """Gray-Scott scales of Sec. III, Eqs. reac_diff12/13 and the groups of
    Eqs. reac_diff15 to reac_diff17, under the reading A0 = k1 = 1, k_f = F,
    k_2 = k (Pearson's (F, k) form):

    tau_A = 1/k_f, tau_B = 1/(k_f + k_2), l = sqrt(D tau), B0 = sqrt(k_f/k1),
    eta = A0 sqrt(k1 k_f)/(k_f + k_2), tau = tau_A/tau_B,
    eps = l_A/l_B = sqrt(tau_A D_A / (tau_B D_B)).
    """
    kf, k1, k2, A0 = F, 1.0, k, 1.0
    tauA = 1.0 / kf
    tauB = 1.0 / (kf + k2)
    lA = math.sqrt(Du * tauA)
    lB = math.sqrt(Dv * tauB)
    B0 = math.sqrt(kf / k1)
    eta = A0 * math.sqrt(k1 * kf) / (kf + k2)
    return {"tauA": tauA, "tauB": tauB, "lA": lA, "lB": lB, "B0": B0, "A0": A0,
            "eta": eta, "tau": tauA / tauB, "eps": lA / lB, "eps2": (lA / lB) ** 2}


def gs_params_from_dimensionless(eta: float, tau: float) -> tuple[float, float]:
    """Inverse of ``gs_dimensionless`` for (F, k): eta = 1/(tau sqrt(F)),
    tau = (F + k)/F (same reading as above)."""
    F = 1.0 / (eta * tau) ** 2
    return F, (tau - 1.0) * F


def gs_steady_states_dimensionless(eta: float):
    """Homogeneous steady states of Eq. reac_diff18 in the variables of
    Eqs. reac_diff16/17: the trivial state (1, 0) and, for eta >= 2, the pair
    of Eq. reac_diff19, A+- = (eta +- sqrt(eta^2 - 4))/(2 eta),
    B+- = (eta -+ sqrt(eta^2 - 4))/2.  Labels follow the paper: "+" has the
    larger A and the smaller B.  Returns {"trivial", "+", "-"}."""
    out = {"trivial": (1.0, 0.0)}
    if eta >= 2.0:
        r = math.sqrt(max(eta * eta - 4.0, 0.0))
        out["+"] = ((eta + r) / (2.0 * eta), (eta - r) / 2.0)
        out["-"] = ((eta - r) / (2.0 * eta), (eta + r) / 2.0)
    return out


def gs_steady_states(F: float, k: float):
    """The states of ``gs_steady_states_dimensionless`` in lattice variables:
    u = A0 * A_tilde, v = B0 * B_tilde (Eq. reac_diff13)."""
    d = gs_dimensionless(F, k, 1.0, 1.0)
    return {key: (d["A0"] * a, d["B0"] * b)
            for key, (a, b) in gs_steady_states_dimensionless(d["eta"]).items()}


def gs_jacobian(F: float, k: float, u: float, v: float) -> np.ndarray:
    """Jacobian dR/d(u, v) of the Gray-Scott source in lattice variables
    (linearisation of Eqs. reac_diff10/11 under the (F, k) reading)."""
    return np.array([[-v * v - F, -2.0 * u * v],
                     [v * v, 2.0 * u * v - (F + k)]])


def gs_matrix_M(eta: float, tau: float, eps2: float, A: float, B: float, q2: float) -> np.ndarray:
    """Matrix M(q^2) of Eq. reac_diff29 as printed (q = 0 gives J of
    Eq. reac_diff24).  Reading: both rows and columns are ordered (B, A)
    although phi is written (phi_A, phi_B); trace and determinant, which is
    all the paper uses, do not depend on that order."""
    return np.array([[tau * (2.0 * eta * A * B - 1.0 - q2 / eps2), tau * eta * B * B],
                     [-2.0 * A * B, -(q2 + B * B + 1.0)]])


def gs_trace_det_M(eta: float, tau: float, eps2: float, B: float, q2):
    """tr M(q^2) and |M(q^2)| at a non-trivial state in the closed forms given
    after Fig. 8 in Sec. III.C:
    tr M = tau - eta B - q^2 (tau/eps^2 + 1),
    |M| = q^4 tau/eps^2 + q^2 (tau eta B/eps^2 - tau) + tau (eta B - 2)."""
    q2 = np.asarray(q2, dtype=np.float64)
    tr = tau - eta * B - q2 * (tau / eps2 + 1.0)
    det = q2 * q2 * tau / eps2 + q2 * (tau * eta * B / eps2 - tau) + tau * (eta * B - 2.0)
    return tr, det


def turing_band(eta: float, eps2: float, B: float):
    """Roots q^2_{1,2} of |M(q^2)| = 0, Eq. reac_diff32 (dimensionless q, in
    units of 1/l_A).  Returns (low, high) or None if the roots are complex."""
    b = eta * B
    disc = (b - eps2) ** 2 - 4.0 * eps2 * (b - 2.0)
    if disc < 0:
        return None
    r = math.sqrt(disc)
    return ((-(b - eps2) - r) / 2.0, (-(b - eps2) + r) / 2.0)


def turing_space_lower_bound(eta: float) -> float:
    """Smallest eps^2 for which the B- state has two distinct positive roots
    of Eq. reac_diff32 (Turing space, Eq. reac_diff33).

    Reading: the printed upper bound "-8 + 11.65 eta B" is garbled; with
    b = eta B- > 2, two positive real roots need eps^2 > b (first condition of
    Eq. reac_diff33) and a positive discriminant, which for eps^2 > b holds
    exactly when eps^2 > (3b - 4) + 2 sqrt(2 (b - 1)(b - 2)).  That is a
    lower bound on eps^2 (it exceeds b), used here in place of the printed one.
    """
    B = gs_steady_states_dimensionless(eta)["-"][1]
    b = eta * B
    return (3.0 * b - 4.0) + 2.0 * math.sqrt(2.0 * (b - 1.0) * (b - 2.0))


def hopf_unstable(eta: float, tau: float) -> bool:
    """Hopf side of the B- state: tr M(0) = tau - eta B- > 0 (Sec. III.C,
    end of the Turing-space discussion)."""
    B = gs_steady_states_dimensionless(eta)["-"][1]
    return tau - eta * B > 0.0


def lb_symbol(lat, taus, jac, kvec) -> np.ndarray:
    """Amplification matrix of one LB step for a Fourier mode exp(i k.x).

    Linearising Eq. relax (multi-species form) about a uniform state:
    the collision maps a perturbation df_{i,s} to
    (1 - w_s) df_{i,s} + w_i (w_s drho_s + sum_r J_sr drho_r), with
    drho_s = sum_j df_{j,s} and w_s = 1/tau_s; the push to x + e_i multiplies
    the mode by exp(-i k.e_i).  Size (S Q) x (S Q), index s * Q + i.
    ``jac`` is dR/drho (S x S).  The velocity set is taken from the compiled
    oracle so that this symbol describes exactly the table it uses.
    """
    ex, ey, w = lattice(lat)
    Q = len(w)
    jac = np.atleast_2d(np.asarray(jac, dtype=np.float64))
    S = jac.shape[0]
    om = 1.0 / np.broadcast_to(np.asarray(taus, dtype=np.float64), (S,))
    C = np.zeros((S * Q, S * Q))
    for s in range(S):
        for i in range(Q):
            row = s * Q + i
            C[row, row] += 1.0 - om[s]
            for r in range(S):
                coef = w[i] * ((om[s] if r == s else 0.0) + jac[s, r])
                C[row, r * Q:(r + 1) * Q] += coef
    phase = np.exp(-1j * (kvec[0] * ex + kvec[1] * ey))
    P = np.diag(np.tile(phase, S))
    return P @ C


def lb_growth_rate(lat, taus, jac, kvec) -> complex:
    """Leading eigenvalue of ``lb_symbol`` as a rate per step, log(lambda)."""
    ev = np.linalg.eigvals(lb_symbol(lat, taus, jac, kvec))
    lam = ev[np.argmax(np.abs(ev))]
    return complex(np.log(lam))


def continuum_growth_rate(jac, D, q2) -> np.ndarray:
    """Eigenvalues of J - diag(D) q^2, the linearised reaction-diffusion
    equation (Eq. reac_diff1) for a mode of wave number q."""
    jac = np.atleast_2d(np.asarray(jac, dtype=np.float64))
    D = np.broadcast_to(np.asarray(D, dtype=np.float64), (jac.shape[0],))
    return np.linalg.eigvals(jac - np.diag(D) * q2)


def point_source(nx: int, ny: int, x0: float, y0: float, D: float, kappa: float, t: float) -> np.ndarray:
    """Infinite-domain solution of Eq. reac_diff3 for a unit point source,
    Eq. reac_diff5: exp(-r^2/(4 D t)) exp(-kappa t) / (4 pi D t)."""
    y, x = np.mgrid[0:ny, 0:nx].astype(np.float64)
    r2 = (x - x0) ** 2 + (y - y0) ** 2
    return np.exp(-r2 / (4.0 * D * t)) * math.exp(-kappa * t) / (4.0 * math.pi * D * t)


def relative_error(analytic: np.ndarray, simulated: np.ndarray) -> float:
    """E_rho of Sec. II.B: sqrt(sum |an - sim|^2 / sum |an|^2)."""
    return float(np.sqrt(np.sum(np.abs(analytic - simulated) ** 2) / np.sum(np.abs(analytic) ** 2)))


def wave_number(nx_mode, ny_mode, Lx: float, Ly: float):
    """q = 2 pi sqrt((n_x/L_x)^2 + (n_y/L_y)^2), Eq. reac_diff35."""
    return 2.0 * np.pi * np.sqrt((np.asarray(nx_mode) / Lx) ** 2 + (np.asarray(ny_mode) / Ly) ** 2)


def structure_factor_peak(field: np.ndarray) -> dict:
    """Dominant pattern wavelength of a periodic square field from its Fourier
    spectrum (Sec. III.D, Eq. reac_diff35).

    Reading (integer shells alone are too coarse for a 2 % comparison):
    S(n) = |DFT(field - mean)|^2, modes grouped into shells round(|n|) with
    n = 0 excluded; p is the shell of largest total power (ties: smaller |n|);
    <|n|> = sum |n| S / sum S over the modes of shells p-2 .. p+2;
    lambda_dom = L / <|n|>.
    """
    field = np.asarray(field, dtype=np.float64)
    ny, nx = field.shape
    spec = np.abs(np.fft.fft2(field - field.mean())) ** 2
    ky = np.fft.fftfreq(ny) * ny
    kx = np.fft.fftfreq(nx) * nx
    n = np.sqrt(ky[:, None] ** 2 + kx[None, :] ** 2)
    shell = np.rint(n).astype(np.int64)
    power = np.bincount(shell.ravel(), weights=spec.ravel())
    power[0] = -1.0
    p = int(np.argmax(power))
    sel = (shell >= max(p - 2, 1)) & (shell <= p + 2)
    nmean = float(np.sum(n[sel] * spec[sel]) / np.sum(spec[sel]))
    L = float(nx)
    return {"shell": p, "n_mean": nmean, "wavelength": L / nmean}
