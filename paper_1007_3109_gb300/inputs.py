"""Seeded synthetic inputs for the reaction-diffusion workloads.

This module is shared by the library's tests and benchmark and by the oracle
checks.  It holds only input recipes -- initial density fields, seeds and the
parameters of each workload -- and none of the LB arithmetic.

Random numbers come from SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), used as a counter-based
generator: the value of site (x, y) of species s under a seed is
splitmix64(key(seed, s, y, x)), so any window of a field can be generated on
its own and every consumer sees the same bits.

Workloads (sizes, parameters and initial states follow the paper's runs:
Sec. II.B for the linear decay, Sec. III.D and Sec. IV for Gray-Scott):

=================  =====================================================
decay_128          1 species, linear decay kappa = 1e-3, D = 1/6, 128^2,
                   rho0 = 1 + 0.1 cos(2 pi x / 128) + U(-1e-6, 1e-6)
gs_512             Gray-Scott F = 0.04, k = 0.06, D_u = 0.1, D_v = 0.05,
                   512^2, u = 1, v = 0 with a centred 40x40 square
                   u = 0.5, v = 0.25, plus U(-0.01, 0.01) on every site
gs_sweep_256       1024 Gray-Scott instances of 256^2 on a 32x32 (F, k) grid,
                   F in [0.01, 0.08], k in [0.03, 0.07], same init recipe
gs_serving         Poisson stream of Gray-Scott requests, side in
                   [64, 2048], diffusion scale in {1, 2, 4}, steps in
                   [1e3, 5e4]
gs_8192            Gray-Scott F = 0.037, k = 0.06, D_u = 0.1, D_v = 0.05,
                   8192^2, 256 random 16x16 spots u = 0.5, v = 0.25 on
                   u = 1, v = 0, plus U(-0.01, 0.01)
gs2x_8192          4 species: two Gray-Scott pairs (F, k) = (0.037, 0.06)
                   and (0.03, 0.055) exchanging v at rate 0.001, as a
                   mass-action network of 10 steps; D = (0.1, 0.05) per
                   pair; 8192^2, spot init per pair (seeds 1240, 1241)
=================  =====================================================
"""
from __future__ import annotations

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(x):
    """SplitMix64 output function applied to counter values x (uint64)."""
    with np.errstate(over="ignore"):
        z = np.asarray(x, dtype=np.uint64) + _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def _key(seed: int, stream: int, y, x):
    """Counter of one draw: 14-bit seed, 2-bit stream, 24-bit y, 24-bit x."""
    base = np.uint64(((int(seed) & 0x3FFF) << 50) | ((int(stream) & 0x3) << 48))
    return base | (np.asarray(y, dtype=np.uint64) << np.uint64(24)) | np.asarray(x, dtype=np.uint64)


def uniform01(seed: int, stream: int, y, x) -> np.ndarray:
    """U[0, 1) with 53 random bits for each (y, x) pair."""
    z = splitmix64(_key(seed, stream, y, x))
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def noise_field(seed: int, stream: int, ny: int, nx: int, amp: float, y0: int = 0, x0: int = 0) -> np.ndarray:
    """Additive U(-amp, amp) on an ny x nx window whose corner is (y0, x0)."""
    y = np.arange(y0, y0 + ny, dtype=np.uint64)[:, None]
    x = np.arange(x0, x0 + nx, dtype=np.uint64)[None, :]
    return amp * (2.0 * uniform01(seed, stream, y, x) - 1.0)


def rho0_cosine(nx: int, ny: int, seed: int, amp: float = 0.1, noise: float = 1e-6) -> np.ndarray:
    """One species: 1 + amp cos(2 pi x / nx) + U(-noise, noise); shape (1, ny, nx)."""
    x = np.arange(nx, dtype=np.float64)
    base = 1.0 + amp * np.cos(2.0 * np.pi * x / nx)
    return (base[None, :] + noise_field(seed, 0, ny, nx, noise))[None]


def rho0_square(nx: int, ny: int, seed: int, side: int = 40, u_in: float = 0.5, v_in: float = 0.25,
                noise: float = 0.01) -> np.ndarray:
    """Gray-Scott u = 1, v = 0 with a centred side x side square (u_in, v_in),
    sites [n/2 - side/2, n/2 + side/2) in both directions, plus U(-noise, noise)
    on every site of both species; shape (2, ny, nx)."""
    u = np.ones((ny, nx))
    v = np.zeros((ny, nx))
    h = side // 2
    ys = slice(max(ny // 2 - h, 0), min(ny // 2 - h + side, ny))
    xs = slice(max(nx // 2 - h, 0), min(nx // 2 - h + side, nx))
    u[ys, xs] = u_in
    v[ys, xs] = v_in
    u += noise_field(seed, 0, ny, nx, noise)
    v += noise_field(seed, 1, ny, nx, noise)
    return np.stack([u, v])


def spot_positions(seed: int, nx: int, ny: int, nspots: int):
    """Lower-left corners of the random spots (stream 2 of the seed)."""
    j = np.arange(nspots, dtype=np.uint64)
    px = (splitmix64(_key(seed, 2, 0, j)) % np.uint64(nx)).astype(np.int64)
    py = (splitmix64(_key(seed, 2, 1, j)) % np.uint64(ny)).astype(np.int64)
    return px, py


def rho0_spots(nx: int, ny: int, seed: int, nspots: int = 256, side: int = 16, u_in: float = 0.5,
               v_in: float = 0.25, noise: float = 0.01, rows: slice | None = None) -> np.ndarray:
    """Gray-Scott u = 1, v = 0 with nspots side x side squares (u_in, v_in) at
    seeded positions (periodic wrap, overlaps allowed) plus U(-noise, noise).
    ``rows`` restricts the output to a band of rows (same values as the full
    field there); shape (2, nrows, nx)."""
    rows = rows or slice(0, ny)
    y0, y1 = rows.start, rows.stop
    nr = y1 - y0
    u = np.ones((nr, nx))
    v = np.zeros((nr, nx))
    px, py = spot_positions(seed, nx, ny, nspots)
    for sx, sy in zip(px.tolist(), py.tolist()):
        yy = (sy + np.arange(side)) % ny
        xx = (sx + np.arange(side)) % nx
        sel = yy[(yy >= y0) & (yy < y1)] - y0
        if sel.size:
            u[np.ix_(sel, xx)] = u_in
            v[np.ix_(sel, xx)] = v_in
    u += noise_field(seed, 0, nr, nx, noise, y0=y0)
    v += noise_field(seed, 1, nr, nx, noise, y0=y0)
    return np.stack([u, v])


def sweep_params(n: int = 32, F_range=(0.01, 0.08), k_range=(0.03, 0.07)):
    """(F, k) of the phase-diagram sweep: instance i * n + j has
    F = F0 + (F1 - F0) i / (n - 1), k = k0 + (k1 - k0) j / (n - 1)."""
    i = np.arange(n)
    F = F_range[0] + (F_range[1] - F_range[0]) * i / (n - 1)
    k = k_range[0] + (k_range[1] - k_range[0]) * i / (n - 1)
    FF, KK = np.meshgrid(F, k, indexing="ij")
    return FF.ravel(), KK.ravel()


def serving_requests(n: int, seed: int, rate: float, side_range=(64, 2048), scales=(1, 2, 4),
                     steps_range=(1000, 50000)):
    """Seeded request stream: Poisson arrival times (exponential gaps of mean
    1/rate seconds), side, diffusion scale and step count per request."""
    j = np.arange(n, dtype=np.uint64)
    u_gap = uniform01(seed, 3, 0, j)
    gaps = -np.log1p(-u_gap) / rate
    arrivals = np.cumsum(gaps) - gaps[0]
    side = side_range[0] + (splitmix64(_key(seed, 3, 1, j)) % np.uint64(side_range[1] - side_range[0] + 1)).astype(np.int64)
    scale = np.asarray(scales)[(splitmix64(_key(seed, 3, 2, j)) % np.uint64(len(scales))).astype(np.int64)]
    steps = steps_range[0] + (splitmix64(_key(seed, 3, 3, j)) % np.uint64(steps_range[1] - steps_range[0] + 1)).astype(np.int64)
    return {"arrival_s": arrivals, "side": side, "scale": scale, "steps": steps}


WORKLOADS = {
    "decay_128": dict(lattice="D2Q9", nspecies=1, nx=128, ny=128, D=(1.0 / 6.0,),
                      reaction=dict(kind="linear", kappa=1e-3), steps=2000, seed=1235,
                      init="cosine"),
    "gs_512": dict(lattice="D2Q9", nspecies=2, nx=512, ny=512, D=(0.1, 0.05),
                   reaction=dict(kind="gray_scott", F=0.04, k=0.06), steps=20000, seed=1236,
                   init="square"),
    "gs_sweep_256": dict(lattice="D2Q9", nspecies=2, nx=256, ny=256, D=(0.1, 0.05),
                         reaction=dict(kind="gray_scott"), steps=10000, seed=1237, init="square",
                         instances=1024),
    "gs_serving": dict(lattice="D2Q9", nspecies=2, D=(0.1, 0.05),
                       reaction=dict(kind="gray_scott", F=0.04, k=0.06), seed=1238, requests=256),
    "gs_8192": dict(lattice="D2Q9", nspecies=2, nx=8192, ny=8192, D=(0.1, 0.05),
                    reaction=dict(kind="gray_scott", F=0.037, k=0.06), steps=10000, seed=1239,
                    init="spots"),
    "gs2x_8192": dict(lattice="D2Q9", nspecies=4, nx=8192, ny=8192, D=(0.1, 0.05, 0.1, 0.05),
                      reaction=dict(kind="mass_action"), steps=10000, seed=1240,
                      init="spots2"),
}


def fourier_perturbation(L: int, seed: int, nmax: int = 10) -> np.ndarray:
    """Two zero-mean fields on an L x L periodic grid, shape (2, L, L): per field
    the sum over mode numbers (a, b), 0 < a^2 + b^2 <= nmax^2, b >= 0, of
    A cos(2 pi (a x + b y) / L + phi) with A = U(-1, 1) and phi = 2 pi U(0, 1)
    from SplitMix64(seed, field, mode index), scaled to max |.| = 1.  A function
    of (x / L, y / L) alone: the same perturbation at every grid size, for
    the diffusion-rescaling runs of Sec. IV."""
    x = np.arange(L, dtype=np.float64) / L
    modes = [(a, b) for a in range(-nmax, nmax + 1) for b in range(0, nmax + 1)
             if 0 < a * a + b * b <= nmax * nmax]
    idx = np.arange(len(modes), dtype=np.uint64)
    out = np.zeros((2, L, L))
    for s in range(2):
        amp = 2.0 * uniform01(seed, 10 + s, 0, idx) - 1.0
        ph = 2.0 * np.pi * uniform01(seed, 10 + s, 1, idx)
        for (a, b), A, p in zip(modes, amp, ph):
            out[s] += A * np.cos(2.0 * np.pi * (a * x[None, :] + b * x[:, None]) + p)
    out -= out.mean(axis=(1, 2), keepdims=True)
    return out / np.abs(out).max(axis=(1, 2), keepdims=True)


def coupled_gs_network(F1=0.037, k1=0.06, F2=0.03, k2=0.055, c=0.001):
    """Reaction steps of two Gray-Scott pairs (u1, v1, u2, v2) coupled by a
    slow exchange of the autocatalyst, as (rates, order, change) rows:
    U + 2V -> 3V at 1, 0 -> U at F, U -> 0 at F, V -> 0 at F + k for each pair
    (the steps of Sec. III), then V1 -> V2 and V2 -> V1 at c."""
    rates, order, change = [], [], []
    for p, (F, k) in enumerate(((F1, k1), (F2, k2))):
        u, v = 2 * p, 2 * p + 1
        for kr, a, nu in ((1.0, {u: 1, v: 2}, {u: -1, v: 1}), (F, {}, {u: 1}), (F, {u: 1}, {u: -1}),
                          (F + k, {v: 1}, {v: -1})):
            rates.append(kr)
            order.append(tuple(a.get(j, 0) for j in range(4)))
            change.append(tuple(nu.get(j, 0) for j in range(4)))
    rates += [c, c]
    order += [(0, 1, 0, 0), (0, 0, 0, 1)]
    change += [(0, -1, 0, 1), (0, 1, 0, -1)]
    return rates, order, change


def rho0_spots2(nx: int, ny: int, seed: int) -> np.ndarray:
    """Two independent spot fields (``rho0_spots`` with seeds seed and
    seed + 1), stacked as (u1, v1, u2, v2); shape (4, ny, nx)."""
    return np.concatenate([rho0_spots(nx, ny, seed), rho0_spots(nx, ny, seed + 1)])


def initial_density(name: str, nx: int | None = None, ny: int | None = None, seed: int | None = None) -> np.ndarray:
    """Initial densities of a named workload, optionally on another grid size."""
    w = WORKLOADS[name]
    nx = nx or w["nx"]
    ny = ny or w["ny"]
    seed = w["seed"] if seed is None else seed
    if w["init"] == "cosine":
        return rho0_cosine(nx, ny, seed)
    if w["init"] == "square":
        return rho0_square(nx, ny, seed)
    if w["init"] == "spots":
        return rho0_spots(nx, ny, seed)
    if w["init"] == "spots2":
        return rho0_spots2(nx, ny, seed)
    raise KeyError(w["init"])
