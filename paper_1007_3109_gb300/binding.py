"""Thin ctypes binding of the C ABI in include/lb_rd.h.

Argument marshalling only: every step of the computation runs in the CUDA
library ``lib/liblbrd.so``.  There is no CPU path; if the library is missing
the calls raise instead of computing anything here.

The functions keep the C names (``lb_rd_create``, ``lb_rd_step``, ...) and
take numpy arrays (host memory) or CUDA torch tensors (device memory) where
the C functions take a pointer plus an ``is_device`` flag.  ``Simulation`` is
a small owner of one handle built from those functions.
"""
from __future__ import annotations

import ctypes
import os
import re
import time
from ctypes import POINTER, c_double, c_int, c_int32, c_int64, c_size_t, c_void_p, c_char_p

import numpy as np

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "lib", "liblbrd.so")

LB_RD_OK, LB_RD_EINVAL, LB_RD_ENOMEM, LB_RD_ECUDA = 0, 1, 2, 3
LB_RD_EPENDING, LB_RD_ETIMEOUT, LB_RD_EBUSY, LB_RD_ENOTFOUND = 4, 5, 6, 7
STATUS_NAMES = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "EPENDING", 5: "ETIMEOUT",
                6: "EBUSY", 7: "ENOTFOUND"}

LATTICES = {"D2Q9": 0, "D2Q5": 1}
Q_OF = {"D2Q9": 9, "D2Q5": 5}
PRECISIONS = {"fp64": 0, "fp32": 1, "fp32_bf16dev": 2, "fp32_fp16dev": 3}
REACTIONS = {"none": 0, "linear": 1, "gray_scott": 2, "mass_action": 3}


class LbRdError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


MAX_SPECIES, MAX_REACTIONS = 4, 16


class lb_rd_reaction(ctypes.Structure):
    _fields_ = [("kind", c_int32), ("kappa", c_double), ("F", c_double), ("k", c_double),
                ("nreactions", c_int32), ("rate", c_double * MAX_REACTIONS),
                ("order", (ctypes.c_int8 * MAX_SPECIES) * MAX_REACTIONS),
                ("change", (ctypes.c_int8 * MAX_SPECIES) * MAX_REACTIONS)]


class lb_rd_config(ctypes.Structure):
    _fields_ = [("lattice", c_int32), ("nspecies", c_int32), ("nx", c_int64), ("ny", c_int64),
                ("tau", c_double * MAX_SPECIES), ("reaction", lb_rd_reaction), ("precision", c_int32),
                ("track_mass", c_int32), ("streaming", c_int32), ("stream", c_void_p), ("tb_depth", c_int32)]


_LIB = None

_SIGNATURES = {
    "lb_rd_last_error": ([], c_char_p),
    "lb_rd_version": ([], c_char_p),
    "lb_rd_tau_from_diffusion": ([c_double], c_double),
    "lb_rd_check_config": ([POINTER(lb_rd_config), POINTER(c_size_t)], c_int),
    "lb_rd_create": ([POINTER(lb_rd_config), POINTER(c_void_p)], c_int),
    "lb_rd_destroy": ([c_void_p], c_int),
    "lb_rd_init": ([c_void_p, c_void_p, c_int], c_int),
    "lb_rd_step": ([c_void_p, c_int64], c_int),
    "lb_rd_get_time": ([c_void_p, POINTER(c_int64)], c_int),
    "lb_rd_moments": ([c_void_p, c_void_p, c_void_p, c_int], c_int),
    "lb_rd_get_distributions": ([c_void_p, c_void_p, c_int], c_int),
    "lb_rd_state_size": ([c_void_p, POINTER(c_size_t)], c_int),
    "lb_rd_save": ([c_void_p, c_void_p, c_size_t], c_int),
    "lb_rd_restore": ([c_void_p, c_void_p, c_size_t], c_int),
    "lb_rd_set_timing": ([c_void_p, c_int], c_int),
    "lb_rd_kernel_time": ([c_void_p, POINTER(c_double), POINTER(c_int64)], c_int),
    "lb_rd_launch_count": ([c_void_p, POINTER(c_int64)], c_int),
    "lb_rd_launch_times": ([c_void_p, POINTER(c_double), POINTER(c_int32), POINTER(c_int32), c_int64,
                            POINTER(c_int64)], c_int),
    "lb_rd_step_noalloc": ([POINTER(lb_rd_config), c_void_p, c_void_p, c_void_p], c_int),
    "lb_rd_variant_count": ([c_int32, POINTER(c_int32)], c_int),
    "lb_rd_variant_name": ([c_int32, c_int32], c_char_p),
    "lb_rd_handle_variant_count": ([c_void_p, POINTER(c_int32)], c_int),
    "lb_rd_handle_variant_name": ([c_void_p, c_int32], c_char_p),
    "lb_rd_autotune": ([c_void_p, c_int32, POINTER(c_int32), POINTER(c_double), c_int32], c_int),
    "lb_rd_set_variant": ([c_void_p, c_int32], c_int),
    "lb_rd_get_variant": ([c_void_p, POINTER(c_int32)], c_int),
    "lb_rd_debug_inject_wait_timeout": ([c_void_p, c_int32], c_int),
    "lb_rd_batch_create": ([POINTER(lb_rd_config), c_int32, POINTER(c_void_p)], c_int),
    "lb_rd_batch_destroy": ([c_void_p], c_int),
    "lb_rd_batch_init": ([c_void_p, c_int32, c_void_p, c_int], c_int),
    "lb_rd_batch_step": ([c_void_p, c_int64], c_int),
    "lb_rd_batch_set_graph": ([c_void_p, c_int32], c_int),
    "lb_rd_batch_moments": ([c_void_p, c_int32, c_void_p, c_void_p, c_int], c_int),
    "lb_rd_batch_set_steps_per_launch": ([c_void_p, c_int32], c_int),
    "lb_rd_batch_get_time": ([c_void_p, POINTER(c_int64), POINTER(c_int64)], c_int),
    "lb_rd_server_create": ([ctypes.c_void_p, POINTER(c_void_p)], c_int),
    "lb_rd_server_destroy": ([c_void_p], c_int),
    "lb_rd_submit": ([c_void_p, POINTER(lb_rd_config), c_void_p, c_int64, POINTER(ctypes.c_uint64)], c_int),
    "lb_rd_poll": ([c_void_p, ctypes.c_uint64, c_void_p, c_void_p, c_void_p], c_int),
    "lb_rd_server_drain": ([c_void_p, c_int64], c_int),
    "lb_rd_server_stats": ([c_void_p, POINTER(c_int64), POINTER(c_int64), POINTER(c_int64)], c_int),
}


def lib():
    """Load liblbrd.so (once).  Raises if it has not been built."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with "
                              "`python -c 'import __graft_entry__ as g; g.build()'` (no CPU fallback exists)")
        L = ctypes.CDLL(LIB_PATH)
        for name, (args, res) in _SIGNATURES.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _LIB = L
    return _LIB


def _check(status: int):
    if status != LB_RD_OK:
        raise LbRdError(status, lib().lb_rd_last_error().decode())


def _ptr(buf, writable: bool = False):
    """(address, is_device) of a numpy array or a torch tensor (contiguous)."""
    if buf is None:
        return None, 0
    if isinstance(buf, np.ndarray):
        if not buf.flags["C_CONTIGUOUS"] or buf.dtype != np.float64:
            raise ValueError("host buffers must be C-contiguous float64 arrays")
        if writable and not buf.flags["WRITEABLE"]:
            raise ValueError("output buffer is read-only")
        return buf.ctypes.data, 0
    # torch tensor (imported lazily: torch is plumbing, not required here)
    if not buf.is_contiguous():
        raise ValueError("tensors must be contiguous")
    if str(buf.dtype) != "torch.float64":
        raise ValueError("tensors must be float64")
    return buf.data_ptr(), 1 if buf.is_cuda else 0


def make_config(lattice="D2Q9", nspecies=1, nx=64, ny=64, tau=(1.0, 1.0), reaction="none", kappa=0.0, F=0.0,
                k=0.0, precision="fp32", track_mass=False, stream=None, network=None,
                inplace=False, tb_depth=0) -> lb_rd_config:
    """Config struct.  ``network`` = (rates, order, change) for
    reaction="mass_action": rate constants per step and the per-step
    reactant exponents and net changes per species (lists of rows);
    ``tb_depth`` time steps per launch (0: the autotuner's choice)."""
    cfg = lb_rd_config()
    cfg.lattice = LATTICES[lattice] if isinstance(lattice, str) else int(lattice)
    cfg.nspecies = int(nspecies)
    cfg.nx, cfg.ny = int(nx), int(ny)
    taus = [float(t) for t in np.atleast_1d(tau)]
    if len(taus) > MAX_SPECIES:
        raise ValueError(f"at most {MAX_SPECIES} relaxation times")
    taus += [1.0] * (MAX_SPECIES - len(taus))
    for s, t in enumerate(taus):
        cfg.tau[s] = t
    cfg.reaction.kind = REACTIONS[reaction] if isinstance(reaction, str) else int(reaction)
    cfg.reaction.kappa, cfg.reaction.F, cfg.reaction.k = float(kappa), float(F), float(k)
    if network is not None:
        rates, order, change = network
        if len(rates) > MAX_REACTIONS or len(order) != len(rates) or len(change) != len(rates):
            raise ValueError(f"a network has 1 .. {MAX_REACTIONS} steps with one order and change row each")
        cfg.reaction.nreactions = len(rates)
        for r, (kr, a, nu) in enumerate(zip(rates, order, change)):
            cfg.reaction.rate[r] = float(kr)
            for j, x in enumerate(a):
                cfg.reaction.order[r][j] = int(x)
            for j, x in enumerate(nu):
                cfg.reaction.change[r][j] = int(x)
    cfg.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    cfg.track_mass = 1 if track_mass else 0
    cfg.streaming = 1 if inplace else 0
    cfg.stream = stream
    cfg.tb_depth = int(tb_depth)
    return cfg


# -- C entry points with the same names --------------------------------------

def lb_rd_version() -> str:
    return lib().lb_rd_version().decode()


def lb_rd_tau_from_diffusion(D: float) -> float:
    return lib().lb_rd_tau_from_diffusion(float(D))


def lb_rd_check_config(cfg: lb_rd_config) -> int:
    n = c_size_t(0)
    _check(lib().lb_rd_check_config(ctypes.byref(cfg), ctypes.byref(n)))
    return n.value


def lb_rd_create(cfg: lb_rd_config) -> int:
    h = c_void_p()
    _check(lib().lb_rd_create(ctypes.byref(cfg), ctypes.byref(h)))
    return h.value


def lb_rd_destroy(h: int):
    _check(lib().lb_rd_destroy(h))


def lb_rd_init(h: int, rho0):
    p, dev = _ptr(rho0)
    _check(lib().lb_rd_init(h, p, dev))


def lb_rd_step(h: int, nsteps: int):
    _check(lib().lb_rd_step(h, int(nsteps)))


def lb_rd_get_time(h: int) -> int:
    t = c_int64(0)
    _check(lib().lb_rd_get_time(h, ctypes.byref(t)))
    return t.value


def lb_rd_moments(h: int, rho_out=None, mass_out=None):
    pr, dev_r = _ptr(rho_out, True)
    pm, dev_m = _ptr(mass_out, True)
    if rho_out is not None and mass_out is not None and dev_r != dev_m:
        raise ValueError("rho_out and mass_out must both be host or both be device buffers")
    _check(lib().lb_rd_moments(h, pr, pm, dev_r if rho_out is not None else dev_m))


def lb_rd_get_distributions(h: int, f_out):
    p, dev = _ptr(f_out, True)
    _check(lib().lb_rd_get_distributions(h, p, dev))


def lb_rd_state_size(h: int) -> int:
    n = c_size_t(0)
    _check(lib().lb_rd_state_size(h, ctypes.byref(n)))
    return n.value


def lb_rd_save(h: int) -> bytearray:
    buf = bytearray(lb_rd_state_size(h))
    cbuf = (ctypes.c_char * len(buf)).from_buffer(buf)
    _check(lib().lb_rd_save(h, ctypes.addressof(cbuf), len(buf)))
    return buf


def lb_rd_restore(h: int, buf: bytes | bytearray):
    data = bytearray(buf)
    cbuf = (ctypes.c_char * len(data)).from_buffer(data)
    _check(lib().lb_rd_restore(h, ctypes.addressof(cbuf), len(data)))


def lb_rd_set_timing(h: int, enable: bool):
    _check(lib().lb_rd_set_timing(h, 1 if enable else 0))


def lb_rd_kernel_time(h: int):
    ms, n = c_double(0), c_int64(0)
    _check(lib().lb_rd_kernel_time(h, ctypes.byref(ms), ctypes.byref(n)))
    return ms.value, n.value


def lb_rd_launch_times(h: int, max_launches: int = 1 << 16):
    """Per timed launch since lb_rd_set_timing(h, True): (ms, steps, variant) lists."""
    ms = (c_double * max_launches)()
    steps = (c_int32 * max_launches)()
    var = (c_int32 * max_launches)()
    n = c_int64(0)
    _check(lib().lb_rd_launch_times(h, ms, steps, var, max_launches, ctypes.byref(n)))
    k = min(n.value, max_launches)
    return list(ms[:k]), list(steps[:k]), list(var[:k])


def lb_rd_launch_count(h: int) -> int:
    n = c_int64(0)
    _check(lib().lb_rd_launch_count(h, ctypes.byref(n)))
    return n.value


def lb_rd_step_noalloc(cfg: lb_rd_config, state_in: int, state_out: int, mass_out: int):
    """Allocation-free step between caller-owned device buffers (addresses)."""
    _check(lib().lb_rd_step_noalloc(ctypes.byref(cfg), state_in, state_out, mass_out))


def lb_rd_variant_count(precision) -> int:
    n = c_int32(0)
    _check(lib().lb_rd_variant_count(PRECISIONS.get(precision, precision), ctypes.byref(n)))
    return n.value


def lb_rd_variant_name(precision, variant: int) -> str:
    return lib().lb_rd_variant_name(PRECISIONS.get(precision, precision), int(variant)).decode()


def variant_steps(name: str) -> int:
    """Time steps per launch of a launch variant, from its name: tb2*_
    variants two, deep<K><letters>_, hdeep<K>_ and hpair<K>_ variants K, the
    others one."""
    m = re.match(r"(?:h?deep|hpair)(\d+)[a-z]*_", name)
    if m:
        return int(m.group(1))
    return 2 if name.startswith("tb2") else 1


def lb_rd_autotune(h: int, iters: int = 20, max_times: int = 0):
    """Returns (best variant, mean ms per time step of every variant of the
    handle; -1 where a variant does not fit the grid)."""
    max_times = max_times or lb_rd_handle_variant_count(h)
    best = c_int32(0)
    times = (c_double * max_times)()
    _check(lib().lb_rd_autotune(h, int(iters), ctypes.byref(best), times, max_times))
    return best.value, list(times)


def lb_rd_handle_variant_count(h: int) -> int:
    n = c_int32(0)
    _check(lib().lb_rd_handle_variant_count(h, ctypes.byref(n)))
    return n.value


def lb_rd_handle_variant_name(h: int, variant: int) -> str:
    return lib().lb_rd_handle_variant_name(h, int(variant)).decode()


def lb_rd_set_variant(h: int, variant: int):
    _check(lib().lb_rd_set_variant(h, int(variant)))


def lb_rd_debug_inject_wait_timeout(h: int, enable: bool = True):
    _check(lib().lb_rd_debug_inject_wait_timeout(h, 1 if enable else 0))


def lb_rd_get_variant(h: int) -> int:
    v = c_int32(0)
    _check(lib().lb_rd_get_variant(h, ctypes.byref(v)))
    return v.value


def lb_rd_batch_create(cfgs) -> int:
    arr = (lb_rd_config * len(cfgs))(*cfgs)
    b = c_void_p()
    _check(lib().lb_rd_batch_create(arr, len(cfgs), ctypes.byref(b)))
    return b.value


def lb_rd_batch_destroy(b: int):
    _check(lib().lb_rd_batch_destroy(b))


def lb_rd_batch_init(b: int, idx: int, rho0):
    p, dev = _ptr(rho0)
    _check(lib().lb_rd_batch_init(b, int(idx), p, dev))


def lb_rd_batch_step(b: int, nsteps: int):
    _check(lib().lb_rd_batch_step(b, int(nsteps)))


def lb_rd_batch_set_graph(b: int, steps_per_graph: int):
    _check(lib().lb_rd_batch_set_graph(b, int(steps_per_graph)))


def lb_rd_batch_moments(b: int, idx: int, rho_out=None, mass_out=None):
    pr, dev_r = _ptr(rho_out, True)
    pm, dev_m = _ptr(mass_out, True)
    _check(lib().lb_rd_batch_moments(b, int(idx), pr, pm, dev_r if rho_out is not None else dev_m))


def lb_rd_batch_set_steps_per_launch(b: int, k: int):
    _check(lib().lb_rd_batch_set_steps_per_launch(b, int(k)))


def lb_rd_batch_get_time(b: int):
    t, n = c_int64(0), c_int64(0)
    _check(lib().lb_rd_batch_get_time(b, ctypes.byref(t), ctypes.byref(n)))
    return t.value, n.value


class lb_rd_server_config(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", c_size_t), ("max_slots", c_int32), ("steps_per_tick", c_int32),
                ("lattice", c_int32), ("nspecies", c_int32), ("precision", c_int32), ("stream", c_void_p),
                ("tick_sites", c_int64)]


class lb_rd_request_stats(ctypes.Structure):
    _fields_ = [("arrival_ns", c_int64), ("start_ns", c_int64), ("end_ns", c_int64), ("steps", c_int64),
                ("status", c_int32)]


def lb_rd_server_create(hbm_budget_bytes, max_slots=64, steps_per_tick=64, lattice="D2Q9", nspecies=2,
                        precision="fp32", stream=None, tick_sites=0) -> int:
    cfg = lb_rd_server_config(int(hbm_budget_bytes), int(max_slots), int(steps_per_tick), LATTICES[lattice],
                              int(nspecies), PRECISIONS[precision], stream, int(tick_sites))
    s = c_void_p()
    _check(lib().lb_rd_server_create(ctypes.byref(cfg), ctypes.byref(s)))
    return s.value


def lb_rd_server_destroy(s: int):
    _check(lib().lb_rd_server_destroy(s))


def lb_rd_submit(s: int, cfg: lb_rd_config, rho0: np.ndarray, nsteps: int) -> int:
    rho0 = np.ascontiguousarray(rho0, dtype=np.float64)
    t = ctypes.c_uint64(0)
    _check(lib().lb_rd_submit(s, ctypes.byref(cfg), rho0.ctypes.data, int(nsteps), ctypes.byref(t)))
    return t.value


def lb_rd_poll(s: int, ticket: int, rho_out=None, mass_out=None):
    """Returns (status, stats dict); status LB_RD_EPENDING while not finished.
    A failed request's status is returned, not raised."""
    st = lb_rd_request_stats()
    pr = rho_out.ctypes.data if rho_out is not None else None
    pm = mass_out.ctypes.data if mass_out is not None else None
    rc = lib().lb_rd_poll(s, ctypes.c_uint64(ticket), pr, pm, ctypes.byref(st))
    if rc in (LB_RD_EINVAL, LB_RD_ENOTFOUND):
        _check(rc)
    return rc, {"arrival_ns": st.arrival_ns, "start_ns": st.start_ns, "end_ns": st.end_ns, "steps": st.steps,
                "status": st.status}


def lb_rd_server_drain(s: int, timeout_ms: int):
    _check(lib().lb_rd_server_drain(s, int(timeout_ms)))


def lb_rd_server_stats(s: int):
    a, b, c = c_int64(0), c_int64(0), c_int64(0)
    _check(lib().lb_rd_server_stats(s, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
    return {"launches": a.value, "ticks": b.value, "finished": c.value}


class Server:
    """Owner of one lb_rd_server (continuous batching of simulation requests)."""

    def __init__(self, hbm_budget_bytes, max_slots=64, steps_per_tick=64, lattice="D2Q9", nspecies=2,
                 precision="fp32", stream=None, tick_sites=0):
        self.nspecies = int(nspecies)
        self.s = lb_rd_server_create(hbm_budget_bytes, max_slots, steps_per_tick, lattice, nspecies, precision,
                                     stream, tick_sites)
        self._shape = {}

    def submit(self, rho0, nsteps, **config) -> int:
        """Queue a request (make_config kwargs); returns its ticket."""
        rho0 = np.ascontiguousarray(rho0, dtype=np.float64)
        t = lb_rd_submit(self.s, make_config(**config), rho0, nsteps)
        self._shape[t] = rho0.shape
        return t

    def result(self, ticket, timeout_s=600.0):
        """Block until the request finishes; returns (rho, mass, stats).
        A failed request raises LbRdError with its status."""
        shape = self._shape[ticket]
        rho = np.empty(shape)
        mass = np.empty(shape[0])
        deadline = time.monotonic() + timeout_s
        delay = 1e-4
        while True:
            rc, st = lb_rd_poll(self.s, ticket, rho, mass)
            if rc != LB_RD_EPENDING:
                del self._shape[ticket]
                if rc != LB_RD_OK:
                    raise LbRdError(rc, f"request {ticket} failed with status {rc}")
                return rho, mass, st
            if time.monotonic() > deadline:
                raise LbRdError(LB_RD_ETIMEOUT, f"request {ticket} did not finish in {timeout_s} s")
            time.sleep(delay)
            delay = min(delay * 2, 0.01)

    def drain(self, timeout_s=600.0):
        lb_rd_server_drain(self.s, int(timeout_s * 1000))
        return self

    def stats(self):
        return lb_rd_server_stats(self.s)

    def close(self):
        if self.s:
            lb_rd_server_destroy(self.s)
            self.s = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Owner of one lb_rd_batch (instances described by make_config kwargs)."""

    def __init__(self, configs):
        self.kw = [dict(c) for c in configs]
        self.cfgs = [make_config(**c) for c in configs]
        self.b = lb_rd_batch_create(self.cfgs)

    def init(self, idx, rho0):
        lb_rd_batch_init(self.b, idx, np.ascontiguousarray(rho0, dtype=np.float64)
                         if isinstance(rho0, np.ndarray) else rho0)
        return self

    def step(self, n=1):
        lb_rd_batch_step(self.b, n)
        return self

    def set_graph(self, steps):
        lb_rd_batch_set_graph(self.b, steps)
        return self

    def set_steps_per_launch(self, k):
        """Time steps per batched launch: 1, 2 (two-step kernel, every nx a
        multiple of 256) or 4, 5, 6, 8 (depth-K kernel; FP32 batches with two
        state copies default to 6 for D2Q9, 4 for D2Q5).  Bitwise the same
        results for every choice."""
        lb_rd_batch_set_steps_per_launch(self.b, k)
        return self

    def moments(self, idx):
        c = self.kw[idx]
        S = int(c.get("nspecies", 1))
        rho = np.empty((S, int(c["ny"]), int(c["nx"])))
        mass = np.empty(S)
        lb_rd_batch_moments(self.b, idx, rho, mass)
        return rho, mass

    @property
    def time(self):
        return lb_rd_batch_get_time(self.b)[0]

    def close(self):
        if self.b:
            lb_rd_batch_destroy(self.b)
            self.b = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Simulation:
    """Owner of one lb_rd handle (a convenience over the functions above)."""

    def __init__(self, lattice="D2Q9", nspecies=1, nx=64, ny=64, tau=(1.0, 1.0), reaction="none", kappa=0.0,
                 F=0.0, k=0.0, precision="fp32", track_mass=False, stream=None, network=None, inplace=False,
                 tb_depth=0):
        self.cfg = make_config(lattice, nspecies, nx, ny, tau, reaction, kappa, F, k, precision, track_mass, stream,
                               network, inplace, tb_depth)
        self.lattice = lattice
        self.S, self.nx, self.ny = int(nspecies), int(nx), int(ny)
        self.Q = Q_OF[lattice] if isinstance(lattice, str) else (9 if lattice == 0 else 5)
        self.h = lb_rd_create(self.cfg)

    def init(self, rho0):
        if isinstance(rho0, np.ndarray):
            rho0 = np.ascontiguousarray(rho0, dtype=np.float64)
            if rho0.shape != (self.S, self.ny, self.nx):
                raise ValueError(f"rho0 must have shape {(self.S, self.ny, self.nx)}, got {rho0.shape}")
        lb_rd_init(self.h, rho0)
        return self

    def step(self, n: int = 1):
        lb_rd_step(self.h, n)
        return self

    @property
    def time(self) -> int:
        return lb_rd_get_time(self.h)

    def moments(self):
        rho = np.empty((self.S, self.ny, self.nx))
        mass = np.empty(self.S)
        lb_rd_moments(self.h, rho, mass)
        return rho, mass

    def mass(self):
        m = np.empty(self.S)
        lb_rd_moments(self.h, None, m)
        return m

    def distributions(self):
        f = np.empty((self.S, self.Q, self.ny, self.nx))
        lb_rd_get_distributions(self.h, f)
        return f

    def set_variant(self, variant: int):
        lb_rd_set_variant(self.h, variant)
        return self

    def autotune(self, iters: int = 10):
        return lb_rd_autotune(self.h, iters)

    def save(self) -> bytearray:
        return lb_rd_save(self.h)

    def restore(self, buf):
        lb_rd_restore(self.h, buf)

    def close(self):
        if self.h:
            lb_rd_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
