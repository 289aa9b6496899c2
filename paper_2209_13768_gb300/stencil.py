"""Expression front end: explicit field updates written as array expressions
with relative offsets, compiled into one fused CUDA kernel for sm_103a.

The WFA's Python front end (Sec. 3, Example Code) writes a time step as
NumPy-like operations on arrays whose indices are relative to the cell
(-1, 0, +1 for the neighbour on each side), and can fuse a whole step into one
kernel. The same here: a `Field` indexed with an offset triple is the value of
that field at the neighbouring cell, `Param`s are scalars given at launch, and
`compile({T: expr})` generates a column-march kernel that evaluates every
update of one time step in one pass (double-buffered fields, Jacobi order).

    T, w = Field("T"), Param("w")
    step = compile({T: T + w * (T[-1, 0, 0] + T[1, 0, 0] + T[0, -1, 0] + T[0, 1, 0]
                                + T[0, 0, -1] + T[0, 0, 1] - 6 * T)})
    step.run({"T": t}, steps=100, w=0.1)   # t: float32 CUDA tensor (nz, ny, nx)

Offsets are (dx, dy, dz). A step updates the interior cells, those whose
every referenced neighbour lies inside the grid; the outer layers (as deep
as the largest offset) keep their values, which is Eq. expl_form's held
boundary. Arithmetic is fp32 in the order the expression is written.

The kernel source is generated here and compiled with nvcc
(-gencode arch=compute_103a,code=sm_103a) into a small shared library in
`_dsl_cache/`, keyed by the source's hash; there is no interpreter or CPU
path: without nvcc or a GPU, compiling or running raises.
"""
from __future__ import annotations

import ctypes
import hashlib
import os
import platform
import shutil
import subprocess
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
CACHE = os.path.join(HERE, "_dsl_cache")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-shared", "-Xcompiler", "-fPIC", "-cudart", "static"]
MAX_RADIUS = 4
_lock = threading.Lock()


# ----------------------------------------------------------------- algebra --
class Expr:
    def __add__(self, o):
        return BinOp("+", self, _wrap(o))

    def __radd__(self, o):
        return BinOp("+", _wrap(o), self)

    def __sub__(self, o):
        return BinOp("-", self, _wrap(o))

    def __rsub__(self, o):
        return BinOp("-", _wrap(o), self)

    def __mul__(self, o):
        return BinOp("*", self, _wrap(o))

    def __rmul__(self, o):
        return BinOp("*", _wrap(o), self)

    def __truediv__(self, o):
        return BinOp("/", self, _wrap(o))

    def __rtruediv__(self, o):
        return BinOp("/", _wrap(o), self)

    def __neg__(self):
        return Neg(self)

    def children(self):
        return ()


def _wrap(v):
    if isinstance(v, Expr):
        return v
    if isinstance(v, (int, float)):
        if v != v or v in (float("inf"), float("-inf")):
            raise ValueError("stencil constants must be finite")
        return Const(float(v))
    raise TypeError(f"cannot use {type(v).__name__} in a stencil expression")


class Const(Expr):
    def __init__(self, value):
        self.value = float(value)


class Param(Expr):
    """A scalar given at launch (fp32)."""

    def __init__(self, name):
        _check_name(name)
        self.name = name


class Ref(Expr):
    """The value of `field` at the cell displaced by `offset` = (dx, dy, dz)."""

    def __init__(self, field, offset):
        self.field = field
        self.offset = tuple(int(v) for v in offset)


class Field(Ref):
    """A grid field; `F[dx, dy, dz]` is its value at the neighbouring cell."""

    def __init__(self, name):
        _check_name(name)
        super().__init__(self, (0, 0, 0))
        self.name = name

    def __getitem__(self, off):
        if not (isinstance(off, tuple) and len(off) == 3 and all(isinstance(v, int) for v in off)):
            raise IndexError("a field is indexed by an offset triple of integers (dx, dy, dz)")
        if max(abs(v) for v in off) > MAX_RADIUS:
            raise IndexError(f"offsets are limited to +-{MAX_RADIUS} cells")
        return Ref(self, off)

    def __hash__(self):
        return id(self)

    def __eq__(self, other):
        return self is other


class BinOp(Expr):
    def __init__(self, op, a, b):
        self.op, self.a, self.b = op, a, b

    def children(self):
        return (self.a, self.b)


class Neg(Expr):
    def __init__(self, a):
        self.a = a

    def children(self):
        return (self.a,)


def _check_name(name):
    if not (isinstance(name, str) and name.isidentifier() and not name.startswith("_")):
        raise ValueError(f"bad name {name!r}: an identifier not starting with '_'")


def _wname(field, dz):
    """Register of a z window: field value at plane z + dz of the own column."""
    return f"zw_{field}_{'m' if dz < 0 else 'p'}{abs(dz)}"


def _walk(e):
    yield e
    for c in e.children():
        yield from _walk(c)


# ----------------------------------------------------------------- codegen --
class Program:
    """What `compile` derives from the updates: fields read and written, the
    halo radius, the parameters, and the CUDA source."""

    def __init__(self, updates):
        if not updates:
            raise ValueError("no updates")
        for f, e in updates.items():
            if not isinstance(f, Field):
                raise TypeError("update keys are Fields")
            if not isinstance(e, Expr):
                raise TypeError("update values are stencil expressions")
        self.updates = list(updates.items())
        fields, params, radius = {}, {}, 0
        for f, e in self.updates:
            fields.setdefault(f.name, f)
            for n in _walk(e):
                if isinstance(n, Ref):
                    if n.field.name in fields and fields[n.field.name] is not n.field:
                        raise ValueError(f"two different fields are named {n.field.name!r}")
                    fields.setdefault(n.field.name, n.field)
                    radius = max(radius, max(abs(v) for v in n.offset))
                elif isinstance(n, Param):
                    params.setdefault(n.name, n)
        self.fields = sorted(fields)               # every field the step touches, by name
        self.written = [f.name for f, _ in self.updates]
        if len(set(self.written)) != len(self.written):
            raise ValueError("a field is updated twice")
        self.params = sorted(params)
        self.radius = radius   # 0: a pointwise update of every cell
        # z windows: a field read at several dz of the cell's own column keeps
        # those values in registers while the thread marches z (one new load
        # a plane instead of one a reference)
        col = {}
        for _, e in self.updates:
            for n in _walk(e):
                if isinstance(n, Ref) and n.offset[0] == 0 and n.offset[1] == 0:
                    col.setdefault(n.field.name, set()).add(n.offset[2])
        self.windows = {f: (min(d), max(d)) for f, d in col.items() if len(d) >= 2}
        self.source = self._source()
        self.key = hashlib.sha256(self.source.encode()).hexdigest()[:16]

    def _expr(self, e):
        if isinstance(e, Const):
            return f"{e.value!r}f" if "e" in repr(e.value) or "." in repr(e.value) else f"{e.value!r}.0f"
        if isinstance(e, Param):
            return f"p_{e.name}"
        if isinstance(e, Ref):
            dx, dy, dz = e.offset
            if dx == 0 and dy == 0 and e.field.name in getattr(self, "windows", {}):
                return _wname(e.field.name, dz)
            return f"__ldg(in_{e.field.name} + o + ({dx}) + ({dy}) * sy + ({dz}) * sz)"
        if isinstance(e, Neg):
            return f"(-{self._expr(e.a)})"
        if isinstance(e, BinOp):
            fn = {"+": "__fadd_rn", "-": "__fsub_rn", "*": "__fmul_rn", "/": "__fdiv_rn"}[e.op]
            return f"{fn}({self._expr(e.a)}, {self._expr(e.b)})"
        raise TypeError(type(e).__name__)

    def _source(self):
        ins = ", ".join(f"const float* __restrict__ in_{f}" for f in self.fields)
        outs = ", ".join(f"float* __restrict__ out_{f}" for f in self.written)
        prm = ", ".join(f"float p_{p}" for p in self.params)
        sig = ", ".join(x for x in (ins, outs, prm) if x)
        body = "\n".join(f"        out_{f.name}[o] = {self._expr(e)};" for f, e in self.updates)
        call_in = ", ".join(f"in[{i}]" for i in range(len(self.fields)))
        call_out = ", ".join(f"out[{i}]" for i in range(len(self.written)))
        call_p = ", ".join(f"params[{i}]" for i in range(len(self.params)))
        call = ", ".join(x for x in (call_in, call_out, call_p) if x)
        R = self.radius
        pre, top, shift = [], [], []
        for f, (lo, hi) in sorted(self.windows.items()):
            for dz in range(lo, hi):
                pre.append(f"    float {_wname(f, dz)} = __ldg(in_{f} + o0 + ({dz}) * sz);")
            top.append(f"        const float {_wname(f, hi)} = __ldg(in_{f} + o + ({hi}) * sz);")
            shift.extend(f"        {_wname(f, dz)} = {_wname(f, dz + 1)};" for dz in range(lo, hi))
        pre_s, top_s, shift_s = "\n".join(pre), "\n".join(top), "\n".join(shift)
        return f"""// generated by paper_2209_13768_gb300.stencil: one explicit step, every update fused
#include <cuda_runtime.h>
// one thread per (x, y) column of interior cells and z chunk, marching z;
// x fastest (coalesced); neighbours through the read-only cache
__global__ void __launch_bounds__(256) step_kernel({sig}, int nx, int ny, int nz, int zchunk) {{
    const int x = {R} + blockIdx.x * 32 + threadIdx.x;
    const int y = {R} + blockIdx.y * 8 + threadIdx.y;
    if (x >= nx - {R} || y >= ny - {R}) return;
    const int z0 = {R} + blockIdx.z * zchunk;
    const int z1 = min(z0 + zchunk, nz - {R});
    const long long sy = nx, sz = (long long)nx * ny;
    const long long o0 = x + y * sy + z0 * sz;
{pre_s}
    for (int z = z0; z < z1; ++z) {{
        const long long o = x + y * sy + z * sz;
{top_s}
{body}
{shift_s}
    }}
}}

extern "C" int stencil_launch(float** in, float** out, const float* params, int nx, int ny, int nz, int zchunk,
                              void* stream) {{
    (void)params;
    const int ix = nx - 2 * {R}, iy = ny - 2 * {R}, iz = nz - 2 * {R};
    if (ix <= 0 || iy <= 0 || iz <= 0) return 0;
    const dim3 block(32, 8);
    const dim3 grid((ix + 31) / 32, (iy + 7) / 8, (iz + zchunk - 1) / zchunk);
    step_kernel<<<grid, block, 0, (cudaStream_t)stream>>>({call}, nx, ny, nz, zchunk);
    return (int)cudaGetLastError();
}}
"""


def _nvcc():
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the stencil front end compiles its kernels with nvcc")


_toolchain = None


def _toolchain_key() -> str:
    """Hash of the compiler (its path and `--version`), the target and the
    flags: a cached kernel built by another toolchain or with other flags is
    not reused."""
    global _toolchain
    if _toolchain is None:
        nv = _nvcc()
        ver = subprocess.run([nv, "--version"], capture_output=True, text=True).stdout
        _toolchain = hashlib.sha256("\n".join([nv, ver] + ARCH + FLAGS).encode()).hexdigest()[:12]
    return _toolchain


def build(program: Program) -> str:
    """Compile the program's kernel into _dsl_cache/ (once per source,
    toolchain and host architecture). The source and the library are
    written under per-process names and the library renamed into place, so
    processes compiling the same program at once do not clobber each
    other's files."""
    with _lock:
        os.makedirs(CACHE, exist_ok=True)
        so = os.path.join(CACHE, f"stencil_{program.key}_{_toolchain_key()}_{platform.machine()}.so")
        if os.path.exists(so):
            return so
        src = os.path.join(CACHE, f"stencil_{program.key}.{os.getpid()}.cu")
        with open(src, "w") as f:
            f.write(program.source)
        tmp = so + f".{os.getpid()}.tmp"
        cmd = [_nvcc()] + ARCH + FLAGS + [src, "-o", tmp]
        try:
            r = subprocess.run(cmd, capture_output=True, text=True)
            if r.returncode != 0:
                raise RuntimeError(f"nvcc failed for the generated stencil:\n{r.stderr[-4000:]}")
            os.replace(tmp, so)
        finally:
            for leftover in (src, tmp):
                if os.path.exists(leftover):
                    os.remove(leftover)
        return so


class Kernel:
    """A compiled step; `run` advances CUDA float32 tensors in place."""

    def __init__(self, program: Program):
        self.program = program
        self.path = build(program)
        self.lib = ctypes.CDLL(self.path)
        self.lib.stencil_launch.restype = ctypes.c_int
        self.lib.stencil_launch.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(ctypes.c_void_p),
                                            ctypes.POINTER(ctypes.c_float), ctypes.c_int, ctypes.c_int,
                                            ctypes.c_int, ctypes.c_int, ctypes.c_void_p]
        self.launches = 0

    def run(self, arrays, steps=1, stream=None, **params):
        """Advance every updated field `steps` explicit steps. `arrays` maps
        each field name to a contiguous float32 CUDA tensor of shape
        (nz, ny, nx) (all the same shape); updated fields are overwritten
        with the result. `params` gives every Param by name."""
        import torch

        p = self.program
        missing = [f for f in p.fields if f not in arrays]
        if missing:
            raise KeyError(f"no array for field(s) {missing}")
        unknown = [k for k in params if k not in p.params]
        if unknown or len(params) != len(p.params):
            raise KeyError(f"parameters {p.params} expected, got {sorted(params)}")
        shape = None
        for f in p.fields:
            t = arrays[f]
            if not (t.is_cuda and t.dtype == torch.float32 and t.is_contiguous() and t.dim() == 3):
                raise TypeError(f"field {f}: a contiguous 3-D float32 CUDA tensor is required")
            if shape is None:
                shape = tuple(t.shape)
            elif tuple(t.shape) != shape:
                raise ValueError("all fields must have the same shape")
        nz, ny, nx = shape
        if steps < 0:
            raise ValueError("negative step count")
        if steps == 0:
            return arrays
        st = stream if stream is not None else torch.cuda.current_stream()
        cur = {f: arrays[f] for f in p.fields}
        spare = {f: arrays[f].clone() for f in p.written}   # boundary layers match from the start
        pv = (ctypes.c_float * max(1, len(p.params)))(*[float(params[k]) for k in p.params])
        # z chunks of 16 planes (one launch a step, many blocks in flight)
        zchunk = 16
        for _ in range(steps):
            ins = (ctypes.c_void_p * len(p.fields))(*[cur[f].data_ptr() for f in p.fields])
            outs = (ctypes.c_void_p * len(p.written))(*[spare[f].data_ptr() for f in p.written])
            rc = self.lib.stencil_launch(ins, outs, pv, nx, ny, nz, zchunk, ctypes.c_void_p(st.cuda_stream))
            if rc != 0:
                raise RuntimeError(f"stencil launch failed (CUDA error {rc})")
            self.launches += 1
            for f in p.written:
                cur[f], spare[f] = spare[f], cur[f]
        for f in p.written:
            if cur[f] is not arrays[f]:
                arrays[f].copy_(cur[f])
        return arrays


def compile(updates) -> Kernel:   # noqa: A001 - the front end's verb
    """Compile {Field: expression} into one fused step kernel."""
    return Kernel(Program(updates))
