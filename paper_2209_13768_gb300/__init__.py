"""GB300-native explicit finite-volume field-equation solver (arXiv 2209.13768).

A thin ctypes binding over the C ABI declared in ``include/wfa.h`` and
implemented in CUDA under ``csrc/`` (built into ``libwfa.so`` beside this
file). Every step of the solve runs in the library's kernels; this module only
marshals arguments. There is no CPU fallback: if the library is missing or
the GPU is absent, calls raise.

Low level: ``lib()`` returns the loaded library with every entry point typed;
the functions keep their C names (``wfa_create_grid`` ...).
High level: ``Grid`` wraps one handle; ``Server`` wraps the request server.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libwfa.so")

F32, BF16 = 0, 1
CG_CLASSIC, CG_PIPELINED = 0, 1
DIRICHLET, ZEROFLUX, PERIODIC, DIRICHLET_CELL, EXCHANGE = 0, 1, 2, 3, 4
BC_KINDS = {"dirichlet": DIRICHLET, "zeroflux": ZEROFLUX, "periodic": PERIODIC,
            "dirichlet_cell": DIRICHLET_CELL, "exchange": EXCHANGE}
PLANES_FIELD, PLANES_K, PLANES_RECIP_K = 0, 1, 2
ZLO, ZHI = 4, 5
STATUS = {0: "WFA_OK", -1: "WFA_ERR_ARG", -2: "WFA_ERR_OOM", -3: "WFA_ERR_BC", -4: "WFA_ERR_UNSTABLE",
          -5: "WFA_ERR_CUDA", -6: "WFA_ERR_TIMEOUT", -7: "WFA_ERR_STATE", -8: "WFA_ERR_BUDGET"}

# every entry point of include/wfa.h: name -> (restype, argtypes)
_vp, _i, _d, _ll, _sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_longlong, ctypes.c_size_t
_fp = ctypes.POINTER(ctypes.c_float)
_dp = ctypes.POINTER(ctypes.c_double)
_llp = ctypes.POINTER(ctypes.c_longlong)
_ip = ctypes.POINTER(ctypes.c_int)


class Request(ctypes.Structure):
    _fields_ = [("nx", _i), ("ny", _i), ("nz", _i), ("hx", _d), ("hy", _d), ("hz", _d),
                ("storage", _i), ("T0_host", _fp), ("k_host", _fp), ("k_uniform", _d),
                ("ux", _d), ("uy", _d), ("uz", _d), ("bc_kind", _i * 6), ("bc_value", _d * 6),
                ("dt", _d), ("steps", _ll), ("out_host", _fp)]


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", _ll), ("admitted", _ll), ("completed", _ll), ("rejected", _ll),
                ("ticks", _ll), ("cell_updates", _d), ("busy_seconds", _d),
                ("p50_latency_s", _d), ("p99_latency_s", _d), ("mean_latency_s", _d),
                ("resident_bytes", _sz), ("peak_resident_bytes", _sz)]


SIGNATURES = {
    "wfa_create_grid": (_i, [_i, _i, _i, _d, _d, _d, _i, _vp, ctypes.POINTER(_vp)]),
    "wfa_destroy_grid": (_i, [_vp]),
    "wfa_set_field": (_i, [_vp, _fp]),
    "wfa_set_coeffs": (_i, [_vp, _fp, _d, _d, _d, _d]),
    "wfa_set_bc": (_i, [_vp, _i, _i, _d]),
    "wfa_stability_dt": (_i, [_vp, _dp]),
    "wfa_set_dt": (_i, [_vp, _d]),
    "wfa_set_tuning": (_i, [_vp, _i, _i]),
    "wfa_set_zchunk": (_i, [_vp, _i]),
    "wfa_get_tuning": (_i, [_vp, _ip, _ip, _ip]),
    "wfa_autotune": (_i, [_vp, _ip, _ip]),
    "wfa_step": (_i, [_vp, _ll]),
    "wfa_steps_done": (_i, [_vp, _llp]),
    "wfa_read_field": (_i, [_vp, _fp]),
    "wfa_total_heat": (_i, [_vp, _dp]),
    "wfa_boundary_flux": (_i, [_vp, _dp]),
    "wfa_sync": (_i, [_vp]),
    "wfa_grid_buffer_bytes": (_i, [_vp, ctypes.POINTER(_sz), ctypes.POINTER(_sz)]),
    "wfa_grid_attach_buffers": (_i, [_vp, _vp, _vp, _vp, _vp]),
    "wfa_set_kernel_timing": (_i, [_vp, _i]),
    "wfa_kernel_time": (_i, [_vp, _dp, _llp]),
    "wfa_launch_count": (_i, [_vp, _llp]),
    "wfa_sum_f32_noalloc": (_i, [_vp, _ll, _d, _vp, _vp]),
    "wfa_last_error": (ctypes.c_char_p, []),
    "wfa_inject_alloc_failure": (_i, [_i]),
    "wfa_implicit_step": (_i, [_vp, _d, _ll, _d, _i, _llp, _dp]),
    "wfa_set_cg_method": (_i, [_vp, _i]),
    "wfa_batch_run": (_i, [ctypes.POINTER(_vp), _llp, _i]),
    "wfa_exchange_planes": (_i, [_vp, _i, _i, ctypes.POINTER(_vp), ctypes.POINTER(_vp), ctypes.POINTER(_sz)]),
    "wfa_exchange": (_i, [_vp, _vp, _i]),
    "wfa_slabs_step": (_i, [ctypes.POINTER(_vp), _i, _ll]),
    "wfa_server_create": (_i, [_sz, _i, _ll, ctypes.POINTER(_vp)]),
    "wfa_server_submit": (_i, [_vp, ctypes.POINTER(Request), _llp]),
    "wfa_server_poll": (_i, [_vp, _ll, _ip]),
    "wfa_server_wait": (_i, [_vp, _ll, _d]),
    "wfa_server_latency": (_i, [_vp, _ll, _dp]),
    "wfa_server_stats_get": (_i, [_vp, ctypes.POINTER(ServerStats)]),
    "wfa_server_destroy": (_i, [_vp]),
}

_lock = threading.Lock()
_lib = None


class WfaError(RuntimeError):
    def __init__(self, code, where, msg):
        super().__init__(f"{where}: {STATUS.get(code, code)}: {msg}")
        self.code = code


def lib():
    """Load libwfa.so (raises if it was not built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                                   "`python -m paper_2209_13768_gb300.build` (needs nvcc)")
            L = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def last_error() -> str:
    return lib().wfa_last_error().decode()


def inject_alloc_failure(n: int) -> None:
    """Make the device allocation after n further successful ones fail once
    with WFA_ERR_OOM (host-side fault injection for tests; n < 0 disarms).
    See wfa_inject_alloc_failure."""
    check(lib().wfa_inject_alloc_failure(int(n)), "wfa_inject_alloc_failure")


def check(code, where=""):
    if code != 0:
        raise WfaError(code, where, last_error())
    return code


def _host_f32(a, n):
    """Pointer to a host float32 buffer of n elements (numpy array or CPU tensor)."""
    if hasattr(a, "data_ptr"):   # torch tensor
        if a.is_cuda or str(a.dtype) != "torch.float32" or not a.is_contiguous() or a.numel() != n:
            raise ValueError("expected a contiguous CPU float32 tensor of %d elements" % n)
        return ctypes.cast(a.data_ptr(), _fp), a
    arr = np.ascontiguousarray(a, dtype=np.float32)
    if arr.size != n:
        raise ValueError(f"expected {n} elements, got {arr.size}")
    return arr.ctypes.data_as(_fp), arr


class Grid:
    """One grid handle. Arrays are indexed [z, y, x] (x fastest)."""

    def __init__(self, shape, h=(1.0, 1.0, 1.0), storage=F32, stream=None):
        self.shape = tuple(int(s) for s in shape)   # (nx, ny, nz)
        self.n = self.shape[0] * self.shape[1] * self.shape[2]
        self.storage = storage
        out = _vp()
        st = _vp(stream) if stream else None
        check(lib().wfa_create_grid(*self.shape, *[float(v) for v in h], storage, st, ctypes.byref(out)),
              "wfa_create_grid")
        self.handle = out

    def close(self):
        if getattr(self, "handle", None):
            lib().wfa_destroy_grid(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_field(self, T):
        p, keep = _host_f32(T, self.n)
        check(lib().wfa_set_field(self.handle, p), "wfa_set_field")

    def set_coeffs(self, k=1.0, u=(0.0, 0.0, 0.0)):
        if np.isscalar(k):
            check(lib().wfa_set_coeffs(self.handle, None, float(k), *[float(v) for v in u]), "wfa_set_coeffs")
        else:
            p, keep = _host_f32(k, self.n)
            check(lib().wfa_set_coeffs(self.handle, p, 0.0, *[float(v) for v in u]), "wfa_set_coeffs")

    def set_bc(self, face, kind, value=0.0):
        kind = BC_KINDS.get(kind, kind)
        check(lib().wfa_set_bc(self.handle, int(face), int(kind), float(value)), "wfa_set_bc")

    def set_bcs(self, bc):
        """bc: six (kind, value) pairs for faces -x, +x, -y, +y, -z, +z."""
        for f, (kind, val) in enumerate(bc):
            self.set_bc(f, kind, val)

    def stability_dt(self):
        v = ctypes.c_double()
        check(lib().wfa_stability_dt(self.handle, ctypes.byref(v)), "wfa_stability_dt")
        return v.value

    def set_dt(self, dt):
        check(lib().wfa_set_dt(self.handle, float(dt)), "wfa_set_dt")

    def set_tuning(self, depth=0, variant=0):
        check(lib().wfa_set_tuning(self.handle, int(depth), int(variant)), "wfa_set_tuning")

    def set_zchunk(self, planes=0):
        """Planes per z chunk of the column-march kernels (0: automatic; see wfa_set_zchunk)."""
        check(lib().wfa_set_zchunk(self.handle, int(planes)), "wfa_set_zchunk")

    def tuning(self):
        """(depth, variant, z-chunk planes) the next step uses (see wfa_get_tuning)."""
        d, v, z = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        check(lib().wfa_get_tuning(self.handle, ctypes.byref(d), ctypes.byref(v), ctypes.byref(z)), "wfa_get_tuning")
        return d.value, v.value, z.value

    def autotune(self):
        """Pick the fastest kernel configuration for this grid; returns (depth, variant)."""
        d, v = ctypes.c_int(), ctypes.c_int()
        check(lib().wfa_autotune(self.handle, ctypes.byref(d), ctypes.byref(v)), "wfa_autotune")
        return d.value, v.value

    def step(self, n):
        check(lib().wfa_step(self.handle, int(n)), "wfa_step")

    def steps_done(self):
        v = ctypes.c_longlong()
        check(lib().wfa_steps_done(self.handle, ctypes.byref(v)), "wfa_steps_done")
        return v.value

    def read_field(self, out=None):
        if out is None:
            out = np.empty(self.shape[::-1], dtype=np.float32)
        p, keep = _host_f32(out, self.n)
        check(lib().wfa_read_field(self.handle, p), "wfa_read_field")
        return out

    def total_heat(self):
        v = ctypes.c_double()
        check(lib().wfa_total_heat(self.handle, ctypes.byref(v)), "wfa_total_heat")
        return v.value

    def boundary_flux(self):
        """fp64 heat one step brings in through the Dirichlet faces (wfa_boundary_flux)."""
        v = ctypes.c_double()
        check(lib().wfa_boundary_flux(self.handle, ctypes.byref(v)), "wfa_boundary_flux")
        return v.value

    def sync(self):
        check(lib().wfa_sync(self.handle), "wfa_sync")

    def buffer_bytes(self):
        """(bytes of one padded field buffer, bytes of one padded k buffer)."""
        fb, kb = _sz(), _sz()
        check(lib().wfa_grid_buffer_bytes(self.handle, ctypes.byref(fb), ctypes.byref(kb)), "wfa_grid_buffer_bytes")
        return fb.value, kb.value

    def attach_buffers(self, Ta, Tb, k=None, r=None):
        """Hold the grid's data in caller-owned device memory (device pointers
        or CUDA tensors, kept alive by this object until close)."""
        ptr = lambda t: None if t is None else _vp(t.data_ptr() if hasattr(t, "data_ptr") else int(t))
        check(lib().wfa_grid_attach_buffers(self.handle, ptr(Ta), ptr(Tb), ptr(k), ptr(r)), "wfa_grid_attach_buffers")
        self._attached = (Ta, Tb, k, r)

    def set_kernel_timing(self, every):
        """Time the main sweep kernel of every every-th pass with CUDA events (0: off)."""
        check(lib().wfa_set_kernel_timing(self.handle, int(every)), "wfa_set_kernel_timing")

    def launch_count(self):
        """Kernels the sweeps of this grid have launched so far."""
        n = ctypes.c_longlong()
        check(lib().wfa_launch_count(self.handle, ctypes.byref(n)), "wfa_launch_count")
        return n.value

    def set_cg_method(self, method):
        """"classic" (two kernels and two reductions an iteration) or
        "pipelined" (Chronopoulos-Gear: one of each); see wfa_set_cg_method."""
        m = {"classic": CG_CLASSIC, "pipelined": CG_PIPELINED}.get(method, method)
        check(lib().wfa_set_cg_method(self.handle, int(m)), "wfa_set_cg_method")

    def implicit_step(self, dt, n=1, rtol=1e-6, max_iter=1000):
        """n backward-Euler steps of size dt, each solved by classic CG to
        ||r|| <= rtol ||b|| (see wfa_implicit_step). Returns (CG iterations of
        all steps, the last step's relative residual)."""
        it, res = ctypes.c_longlong(), ctypes.c_double()
        check(lib().wfa_implicit_step(self.handle, float(dt), int(n), float(rtol), int(max_iter),
                                      ctypes.byref(it), ctypes.byref(res)), "wfa_implicit_step")
        return it.value, res.value

    def exchange_planes(self, face, what=PLANES_FIELD):
        """(send, recv, plane_bytes): device addresses of this slab's outermost
        plane next to an exchange face and of the halo plane beyond it (see
        wfa_exchange_planes)."""
        s, r, b = _vp(), _vp(), _sz()
        check(lib().wfa_exchange_planes(self.handle, int(face), int(what), ctypes.byref(s), ctypes.byref(r),
                                        ctypes.byref(b)), "wfa_exchange_planes")
        return s.value, r.value, b.value

    def kernel_time(self):
        """(summed milliseconds, launches) of the sampled kernels since the last call."""
        ms, n = ctypes.c_double(), ctypes.c_longlong()
        check(lib().wfa_kernel_time(self.handle, ctypes.byref(ms), ctypes.byref(n)), "wfa_kernel_time")
        return ms.value, n.value


def sum_f32_noalloc(d_x, n, scale, d_out, stream=None):
    """fp64 sum (times scale) of n floats at device address d_x into the device
    double at d_out, without allocating (see wfa_sum_f32_noalloc)."""
    check(lib().wfa_sum_f32_noalloc(_vp(d_x), int(n), float(scale), _vp(d_out), _vp(stream) if stream else None),
          "wfa_sum_f32_noalloc")


def exchange(lower, upper, what=PLANES_FIELD):
    """Copy planes across lower's +z and upper's -z exchange faces (see wfa_exchange)."""
    check(lib().wfa_exchange(lower.handle, upper.handle, int(what)), "wfa_exchange")


def slabs_step(slabs, n):
    """Advance slabs of one grid (z order, one device) by n steps, exchanging
    planes before every step (see wfa_slabs_step)."""
    arr = (_vp * len(slabs))(*[g.handle for g in slabs])
    check(lib().wfa_slabs_step(arr, len(slabs), int(n)), "wfa_slabs_step")


def batch_run(grids, steps):
    """Advance grids[i] by steps[i] time steps, all grids in one CUDA-graph
    launch (see wfa_batch_run; the grids share one stream). Bitwise equal to
    stepping each grid alone."""
    arr = (_vp * len(grids))(*[g.handle for g in grids])
    st = (ctypes.c_longlong * len(steps))(*[int(s) for s in steps])
    check(lib().wfa_batch_run(arr, st, len(grids)), "wfa_batch_run")


class Server:
    """Continuous-batching request server (see wfa_server_create)."""

    def __init__(self, budget_bytes, max_resident=0, quantum=0):
        out = _vp()
        check(lib().wfa_server_create(int(budget_bytes), int(max_resident), int(quantum), ctypes.byref(out)),
              "wfa_server_create")
        self.handle = out
        self._keep = {}

    def submit(self, shape, T0, steps, *, out=None, h=(1.0, 1.0, 1.0), storage=F32, k=1.0,
               u=(0.0, 0.0, 0.0), bc=None, dt=0.0):
        nx, ny, nz = (int(s) for s in shape)
        n = nx * ny * nz
        r = Request()
        r.nx, r.ny, r.nz = nx, ny, nz
        r.hx, r.hy, r.hz = (float(v) for v in h)
        r.storage = storage
        t0p, t0 = _host_f32(T0, n)
        r.T0_host = t0p
        kk = None
        if np.isscalar(k):
            r.k_host = None
            r.k_uniform = float(k)
        else:
            r.k_host, kk = _host_f32(k, n)
        r.ux, r.uy, r.uz = (float(v) for v in u)
        bc = bc or [("zeroflux", 0.0)] * 6
        for f, (kind, val) in enumerate(bc):
            r.bc_kind[f] = BC_KINDS.get(kind, kind)
            r.bc_value[f] = float(val)
        r.dt = float(dt)
        r.steps = int(steps)
        if out is None:
            out = np.empty((nz, ny, nx), dtype=np.float32)
        r.out_host, outk = _host_f32(out, n)
        ticket = ctypes.c_longlong()
        check(lib().wfa_server_submit(self.handle, ctypes.byref(r), ctypes.byref(ticket)), "wfa_server_submit")
        self._keep[ticket.value] = (outk, t0, kk)   # the server reads the inputs later
        return ticket.value

    def poll(self, ticket):
        d = ctypes.c_int()
        check(lib().wfa_server_poll(self.handle, int(ticket), ctypes.byref(d)), "wfa_server_poll")
        return d.value

    def wait(self, ticket, timeout=60.0):
        check(lib().wfa_server_wait(self.handle, int(ticket), float(timeout)), "wfa_server_wait")
        kept = self._keep.pop(ticket, None)
        return kept[0] if kept else None

    def latency(self, ticket):
        """Seconds from submit to result on the host of a finished ticket."""
        v = ctypes.c_double()
        check(lib().wfa_server_latency(self.handle, int(ticket), ctypes.byref(v)), "wfa_server_latency")
        return v.value

    def stats(self):
        st = ServerStats()
        check(lib().wfa_server_stats_get(self.handle, ctypes.byref(st)), "wfa_server_stats_get")
        return {name: getattr(st, name) for name, _ in ServerStats._fields_}

    def close(self):
        if getattr(self, "handle", None):
            lib().wfa_server_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
