"""FP64 CPU oracle for the finite-volume sweeps of arXiv 2209.13768 (explicit
steps and implicit steps solved by CG).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` use it; the library never does. It shares no
code with the CUDA path (the C source is ``wfa_oracle.c`` beside this file).

Functions
---------
run(T0, n_steps, **problem)      -> field after n_steps (Eq. expl_form, face-flux form)
implicit(T0, n_steps, **problem) -> (field, CG iterations, relative residual) after
                                    n_steps backward-Euler steps (Eq. impl_form, classic CG;
                                    method="cgcg": Chronopoulos-Gear CG)
dt_max(**problem)                -> positivity limit of the explicit step (Sec. 1.1.1)
total_heat(T, h)                 -> sum of T times the cell volume
round_to(x, mode)                -> fp32 / bf16 nearest-even rounding used by ``run``

A problem is described by keyword arguments:
  shape (nx, ny, nz); h=(hx, hy, hz); k: scalar or array of shape (nz, ny, nx);
  u=(ux, uy, uz); bc: six (kind, value) pairs for faces -x,+x,-y,+y,-z,+z with
  kind in {"dirichlet", "zeroflux", "periodic", "dirichlet_cell"}; dt.
Arrays are numpy, indexed [z, y, x] (x fastest in memory).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "wfa_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

KINDS = {"dirichlet": 0, "zeroflux": 1, "periodic": 2, "dirichlet_cell": 3}
ROUND = {None: 0, "none": 0, "f32": 1, "bf16": 2}


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP when available). Returns the .so path."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".{os.getpid()}.tmp"
    base = ["gcc", "-O2", "-shared", "-fPIC", "-std=c11", _SRC, "-o", tmp, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(tmp, _LIB)
    return _LIB


def _bind(path):
    """Load an oracle shared library and declare its entry points."""
    lib = ctypes.CDLL(path)
    i64p = ctypes.POINTER(ctypes.c_int64)
    dp = ctypes.POINTER(ctypes.c_double)
    ip = ctypes.POINTER(ctypes.c_int)
    lib.wfa_oracle_run.argtypes = [i64p, dp, dp, ctypes.c_double, dp, ip, dp, ctypes.c_double,
                                   dp, ctypes.c_int64, ctypes.c_int, ctypes.c_int]
    lib.wfa_oracle_run.restype = ctypes.c_int
    lib.wfa_oracle_dt_max.argtypes = [i64p, dp, dp, ctypes.c_double, dp, ip]
    lib.wfa_oracle_dt_max.restype = ctypes.c_double
    lib.wfa_oracle_total_heat.argtypes = [i64p, dp, dp]
    lib.wfa_oracle_total_heat.restype = ctypes.c_double
    lib.wfa_oracle_round.argtypes = [ctypes.c_double, ctypes.c_int]
    lib.wfa_oracle_round.restype = ctypes.c_double
    if hasattr(lib, "wfa_oracle_round_array"):
        lib.wfa_oracle_round_array.argtypes = [dp, ctypes.c_int64, ctypes.c_int]
        lib.wfa_oracle_round_array.restype = None
    if hasattr(lib, "wfa_oracle_implicit"):
        lib.wfa_oracle_implicit.argtypes = [i64p, dp, ctypes.c_double, dp, ip, dp, ctypes.c_double, dp,
                                            ctypes.c_int64, ctypes.c_double, ctypes.c_int64, i64p, dp, ctypes.c_int]
        lib.wfa_oracle_implicit.restype = ctypes.c_int
    if hasattr(lib, "wfa_oracle_implicit_cgcg"):
        lib.wfa_oracle_implicit_cgcg.argtypes = lib.wfa_oracle_implicit.argtypes
        lib.wfa_oracle_implicit_cgcg.restype = ctypes.c_int
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _bind(build())
    return _lib


def _arr(vals, ctype):
    return (ctype * len(vals))(*vals)


def _ptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if a is not None else None


def _common(shape, h, u, k, bc):
    nx, ny, nz = (int(s) for s in shape)
    n = _arr([nx, ny, nz], ctypes.c_int64)
    hh = _arr([float(v) for v in h], ctypes.c_double)
    uu = _arr([float(v) for v in u], ctypes.c_double)
    if np.isscalar(k):
        k_uniform, karr = float(k), None
    else:
        karr = np.ascontiguousarray(k, dtype=np.float64)
        if karr.shape != (nz, ny, nx):
            raise ValueError(f"k has shape {karr.shape}, expected {(nz, ny, nx)}")
        k_uniform = 0.0
    if len(bc) != 6:
        raise ValueError("bc needs six (kind, value) pairs")
    kinds = _arr([KINDS[b[0]] for b in bc], ctypes.c_int)
    vals = _arr([float(b[1]) for b in bc], ctypes.c_double)
    return n, hh, uu, k_uniform, karr, kinds, vals


def run(T0, n_steps, *, shape, h=(1.0, 1.0, 1.0), k=1.0, u=(0.0, 0.0, 0.0), bc, dt,
        round_to=None, threads=0, lib=None):
    """Advance T0 (shape (nz, ny, nx)) by n_steps explicit steps in fp64.

    ``lib`` selects another build of the oracle (the mutation tests use it)."""
    lib = lib or _load()
    n, hh, uu, k_uniform, karr, kinds, vals = _common(shape, h, u, k, bc)
    T = np.array(T0, dtype=np.float64, order="C", copy=True)
    nx, ny, nz = (int(s) for s in shape)
    if T.shape != (nz, ny, nx):
        raise ValueError(f"T0 has shape {T.shape}, expected {(nz, ny, nx)}")
    rc = lib.wfa_oracle_run(n, hh, uu, k_uniform, _ptr(karr), kinds, vals, float(dt), _ptr(T),
                            int(n_steps), ROUND[round_to], int(threads))
    if rc != 0:
        raise ValueError(f"oracle rejected the problem (code {rc})")
    return T


def implicit(T0, n_steps, *, shape, h=(1.0, 1.0, 1.0), k=1.0, bc, dt, rtol=1e-12, max_iter=10000,
             threads=0, lib=None, method="classic"):
    """Advance T0 by n_steps backward-Euler steps, each solved by classic CG
    in fp64 (Sec. 1.1.2, Eq. impl_form, face-flux form, no advection).

    Returns (T, iterations of all steps, last step's relative residual
    sqrt(r.r / b.b)). rtol = 0 runs exactly max_iter iterations per step
    (fewer only if the residual becomes exactly zero). method="cgcg" runs
    Chronopoulos and Gear's single-synchronisation CG instead (the same
    iterates in exact arithmetic)."""
    lib = lib or _load()
    n, hh, _, k_uniform, karr, kinds, vals = _common(shape, h, (0.0, 0.0, 0.0), k, bc)
    T = np.array(T0, dtype=np.float64, order="C", copy=True)
    nx, ny, nz = (int(s) for s in shape)
    if T.shape != (nz, ny, nx):
        raise ValueError(f"T0 has shape {T.shape}, expected {(nz, ny, nx)}")
    iters = ctypes.c_int64()
    res = ctypes.c_double()
    fn = {"classic": lib.wfa_oracle_implicit, "cgcg": lib.wfa_oracle_implicit_cgcg}[method]
    rc = fn(n, hh, k_uniform, _ptr(karr), kinds, vals, float(dt), _ptr(T), int(n_steps),
            float(rtol), int(max_iter), ctypes.byref(iters), ctypes.byref(res), int(threads))
    if rc != 0:
        raise ValueError(f"oracle rejected the problem (code {rc})")
    return T, iters.value, res.value


def dt_max(*, shape, h=(1.0, 1.0, 1.0), k=1.0, u=(0.0, 0.0, 0.0), bc, lib=None):
    lib = lib or _load()
    n, hh, uu, k_uniform, karr, kinds, _ = _common(shape, h, u, k, bc)
    v = lib.wfa_oracle_dt_max(n, hh, uu, k_uniform, _ptr(karr), kinds)
    if v < 0:
        raise ValueError(f"oracle rejected the problem (code {v})")
    return v


def total_heat(T, h=(1.0, 1.0, 1.0)):
    lib = _load()
    T = np.ascontiguousarray(T, dtype=np.float64)
    nz, ny, nx = T.shape
    n = _arr([nx, ny, nz], ctypes.c_int64)
    return lib.wfa_oracle_total_heat(n, _arr([float(v) for v in h], ctypes.c_double), _ptr(T))


def round_to(x, mode):
    lib = _load()
    a = np.array(x, dtype=np.float64, order="C", copy=True)
    lib.wfa_oracle_round_array(_ptr(a), a.size, ROUND[mode])
    return a
