"""Expression front end: explicit field updates written as array expressions
with relative offsets, compiled into one fused CUDA kernel for sm_103a.

The WFA's Python front end (Sec. 2.1, Example Code) writes a time step as
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


V = 4   # x cells a thread


def _sn(v):
    return ("m%d" % -v) if v < 0 else ("p%d" % v)


def _sname(field, dy, dz, k):
    """Register of row (field, dy, dz) at x0 + k in the generated kernel."""
    return f"s_{field}_{_sn(dy)}_{_sn(dz)}_{_sn(k)}"


def _rname(dy, dz):
    """Element offset of row (dy, dz) from the thread's cell."""
    return f"ro_{_sn(dy)}_{_sn(dz)}"


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
        # rows: every (field, dy, dz) referenced, with the x offsets it is
        # read at; a thread loads each such row's segment once a plane
        rows = {}
        for _, e in self.updates:
            for n in _walk(e):
                if isinstance(n, Ref):
                    dx, dy, dz = n.offset
                    lo, hi = rows.get((n.field.name, dy, dz), (dx, dx))
                    rows[(n.field.name, dy, dz)] = (min(lo, dx), max(hi, dx))
        # z windows: a field read in its own row (dy = 0) at several dz keeps
        # those segments in registers while the thread marches z (one new
        # segment a plane); a window's segments share the union of the x ranges
        col = {}
        for (f, dy, dz) in rows:
            if dy == 0:
                col.setdefault(f, set()).add(dz)
        self.windows = {f: (min(d), max(d)) for f, d in col.items() if len(d) >= 2}
        self.rows = {k: v for k, v in rows.items() if not (k[1] == 0 and k[0] in self.windows)}
        for f, (zlo, zhi) in self.windows.items():   # every plane of the window, one x range
            wl = min(v[0] for (g, dy, _), v in rows.items() if g == f and dy == 0)
            wh = max(v[1] for (g, dy, _), v in rows.items() if g == f and dy == 0)
            for dz in range(zlo, zhi + 1):
                self.rows[(f, 0, dz)] = (wl, wh)
        self.source = self._source()
        self.key = hashlib.sha256(self.source.encode()).hexdigest()[:16]

    def _expr(self, e, i):
        """fp32 expression of cell i (0..V-1) of the thread's group."""
        if isinstance(e, Const):
            return f"{e.value!r}f" if "e" in repr(e.value) or "." in repr(e.value) else f"{e.value!r}.0f"
        if isinstance(e, Param):
            return f"p_{e.name}"
        if isinstance(e, Ref):
            dx, dy, dz = e.offset
            return _sname(e.field.name, dy, dz, i + dx)
        if isinstance(e, Neg):
            return f"(-{self._expr(e.a, i)})"
        if isinstance(e, BinOp):
            fn = {"+": "__fadd_rn", "-": "__fsub_rn", "*": "__fmul_rn", "/": "__fdiv_rn"}[e.op]
            return f"{fn}({self._expr(e.a, i)}, {self._expr(e.b, i)})"
        raise TypeError(type(e).__name__)

    def _load_row(self, f, dy, dz, plane, indent, decl=True):
        """Statements loading row (f, dy, dz) of plane z + `plane` into its
        segment: the V cells by one 128-bit load when VEC, the x halo (and,
        without VEC, every element) cell by cell, masked to the row."""
        lo, hi = self.rows[(f, dy, dz)]
        base = f"(q_{f} + {_rname(dy, plane)})"
        out = []
        out.append(f"{indent}{{")
        out.append(f"{indent}    const float* r_ = {base};")
        out.append(f"{indent}    if (VEC) {{")
        out.append(f"{indent}        const float4 c_ = __ldg(reinterpret_cast<const float4*>(r_));")
        for k, comp in zip(range(V), "xyzw"):
            out.append(f"{indent}        {_sname(f, dy, dz, k)} = c_.{comp};")
        out.append(f"{indent}    }} else {{")
        for k in range(V):
            out.append(f"{indent}        {_sname(f, dy, dz, k)} = x0 + {k} < nx ? __ldg(r_ + {k}) : 0.0f;")
        out.append(f"{indent}    }}")
        for k in list(range(lo, 0)) + list(range(V, V + hi)):
            out.append(f"{indent}    {_sname(f, dy, dz, k)} = (unsigned)(x0 + ({k})) < (unsigned)nx ? "
                       f"__ldg(r_ + ({k})) : 0.0f;")
        out.append(f"{indent}}}")
        decls = [f"{indent}float {_sname(f, dy, dz, k)};" for k in range(lo, V + hi)] if decl else []
        return decls + out

    def _source(self):
        ins = ", ".join(f"const float* __restrict__ in_{f}" for f in self.fields)
        outs = ", ".join(f"float* __restrict__ out_{f}" for f in self.written)
        prm = ", ".join(f"float p_{p}" for p in self.params)
        sig = ", ".join(x for x in (ins, outs, prm) if x)
        call_in = ", ".join(f"in[{i}]" for i in range(len(self.fields)))
        call_out = ", ".join(f"out[{i}]" for i in range(len(self.written)))
        call_p = ", ".join(f"params[{i}]" for i in range(len(self.params)))
        call = ", ".join(x for x in (call_in, call_out, call_p) if x)
        R = self.radius
        pre, top, shift = [], [], []
        # per-thread pointers to the group's first cell at plane z (advanced
        # a plane an iteration); row offsets dy sy + dz sz are loop invariants
        for f in self.fields:
            pre.append(f"    const float* __restrict__ q_{f} = in_{f} + o0;")
        for f in self.written:
            pre.append(f"    float* __restrict__ w_{f} = out_{f} + o0;")
        offs = sorted({(dy, dz) for (_, dy, dz) in self.rows} |
                      {(0, d) for f, (lo, hi) in self.windows.items() for d in range(lo, hi + 1)})
        for dy, dz in offs:
            pre.append(f"    const long long {_rname(dy, dz)} = ({dy}) * sy + ({dz}) * sz;")
        # window segments below the top one, loaded before the march
        for f, (lo, hi) in sorted(self.windows.items()):
            for dz in range(lo, hi):
                pre.extend(self._load_row(f, 0, dz, dz, "    "))
        # every plane: the windows' top segments and the other rows
        for (f, dy, dz) in sorted(self.rows):
            if dy == 0 and f in self.windows:
                if dz == self.windows[f][1]:
                    top.extend(self._load_row(f, 0, dz, dz, "        ", decl=False))
            else:
                top.extend(self._load_row(f, dy, dz, dz, "        ", decl=False))
        # one thread per 128-byte line asks L2 for the plane three ahead of
        # the furthest one read
        zmax = max([dz for (_, _, dz) in self.rows] + [0])
        for f in self.fields:
            top.append(f"        if ((threadIdx.x & 7) == 0 && z + {zmax + 3} < nz) "
                       f"asm volatile(\"prefetch.global.L2 [%0];\" :: \"l\"(q_{f} + ({zmax + 3}) * sz));")
        body = []
        for f, e in self.updates:
            for i in range(V):
                body.append(f"        const float v_{f.name}_{i} = {self._expr(e, i)};")
        for f, _ in self.updates:
            body.append(f"        if (full) {{")
            body.append(f"            *reinterpret_cast<float4*>(w_{f.name}) = make_float4("
                        + ", ".join(f"v_{f.name}_{i}" for i in range(V)) + ");")
            body.append(f"        }} else {{")
            for i in range(V):
                body.append(f"            if (x0 + {i} >= {R} && x0 + {i} < nx - {R}) w_{f.name}[{i}] = v_{f.name}_{i};")
            body.append(f"        }}")
        for f, (lo, hi) in sorted(self.windows.items()):
            wl, wh = self.rows[(f, 0, lo)]
            for dz in range(lo, hi):
                for k in range(wl, V + wh):
                    shift.append(f"        {_sname(f, 0, dz, k)} = {_sname(f, 0, dz + 1, k)};")
        shift.extend([f"        q_{f} += sz;" for f in self.fields] + [f"        w_{f} += sz;" for f in self.written])
        top_decl = []
        for (f, dy, dz), (lo, hi) in sorted(self.rows.items()):
            if dy == 0 and f in self.windows and dz < self.windows[f][1]:
                continue   # declared before the march
            top_decl.extend(f"        float {_sname(f, dy, dz, k)};" for k in range(lo, V + hi))
        pre_s, top_s, body_s, shift_s = "\n".join(pre), "\n".join(top_decl + top), "\n".join(body), "\n".join(shift)
        return f"""// generated by paper_2209_13768_gb300.stencil: one explicit step, every update fused
#include <cuda_runtime.h>
// each thread takes {V} consecutive x cells (a 16-byte aligned group) of one
// row of a z chunk and marches z; every row it reads is loaded once a plane
// (the {V} cells by one 128-bit load when VEC, the x halo cell by cell, masked
// to the row), and updated cells that lie in the interior are stored
template <bool VEC>
__global__ void __launch_bounds__(256) step_kernel({sig}, int nx, int ny, int nz, int zchunk) {{
    const int x0 = {V} * (blockIdx.x * 32 + threadIdx.x);
    const int y = {R} + blockIdx.y * 8 + threadIdx.y;
    if (x0 + {V - 1} < {R} || x0 >= nx - {R} || y >= ny - {R}) return;
    const int z0 = {R} + blockIdx.z * zchunk;
    const int z1 = min(z0 + zchunk, nz - {R});
    const long long sy = nx, sz = (long long)nx * ny;
    const long long o0 = x0 + y * sy + z0 * sz;
    const bool full = VEC && x0 >= {R} && x0 + {V - 1} < nx - {R};   // every cell of the group is updated
{pre_s}
    for (int z = z0; z < z1; ++z) {{
{top_s}
{body_s}
{shift_s}
    }}
}}

extern "C" int stencil_launch(float** in, float** out, const float* params, int nx, int ny, int nz, int zchunk,
                              void* stream) {{
    (void)params;
    const int ix = nx - 2 * {R}, iy = ny - 2 * {R}, iz = nz - 2 * {R};
    if (ix <= 0 || iy <= 0 || iz <= 0) return 0;
    // 128-bit loads and stores when every row starts on a 16-byte boundary
    bool vec = nx % {V} == 0;
    for (int i = 0; i < {len(self.fields)}; ++i) vec = vec && ((size_t)in[i] % 16 == 0);
    for (int i = 0; i < {len(self.written)}; ++i) vec = vec && ((size_t)out[i] % 16 == 0);
    const dim3 block(32, 8);
    const dim3 grid(((nx + {V - 1}) / {V} + 31) / 32, (iy + 7) / 8, (iz + zchunk - 1) / zchunk);
    if (vec) step_kernel<true><<<grid, block, 0, (cudaStream_t)stream>>>({call}, nx, ny, nz, zchunk);
    else step_kernel<false><<<grid, block, 0, (cudaStream_t)stream>>>({call}, nx, ny, nz, zchunk);
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
