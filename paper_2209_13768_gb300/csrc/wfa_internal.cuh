// Internal declarations of the GB300 finite-volume sweep library.
//
// Device layout of a field (one "padded" array per ping-pong buffer):
//   every axis carries HALO = 8 extra cells on each side; x is padded further
//   so that a row is a multiple of 128 bytes:
//     px = round_up(nx + 2*HALO, 128 / element_size), py = ny + 2*HALO, pz = nz + 2*HALO
//   domain cell (x, y, z), -HALO <= x < nx + HALO, is element
//     ((z + HALO) * py + (y + HALO)) * px + (x + HALO)
//   Halo cells of a periodic axis hold copies of the cells one period away
//   ("twins"), kept current by every kernel that writes the field, so a tile
//   near the edge reads its wrapped neighbours as ordinary memory. Halo cells
//   of other axes are never read by an updated cell: a boundary cell takes its
//   outside neighbour from the boundary condition.
//   Per-cell conductivity k (fp32) uses the same layout (its periodic twins are
//   written once by wfa_set_coeffs).
//   Each padded array starts lead_bytes() into its allocation, so that domain
//   column x = 0 (HALO elements into a row) falls on a 128-byte line: a row's
//   4-cell vectors then fill whole lines (fewer L1 wavefronts per load).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda.h>
#include <stdint.h>

#include <nvtx3/nvToolsExt.h>

#include <string>

#include "../../include/wfa.h"

namespace wfa {

constexpr int HALO = 8;       // halo width on every side (>= the deepest temporal block)
constexpr int MAX_DEPTH = 8;  // steps fused per pass over the grid
constexpr int NUM_TILE_VARIANTS = 2;  // tile shapes compiled per (storage, k mode, depth)
constexpr int COL_VARIANT = 3;        // the one-step column-march kernel
constexpr int FUSED_VARIANT = 4;      // the two-step column-march kernel (uniform k)
constexpr int INPLACE_VARIANT = 5;    // the one-step column-march kernel, boundaries in place
constexpr int WIDE_VARIANT = 6;       // the one-step column-march kernel, 8 cells a thread (16 for bf16, uniform k)
constexpr int T2_VARIANT = 7;         // two steps per pass, TMA-staged planes (uniform k)

// NVTX range over one API call: a named span on a profiler's timeline
// (nothing happens unless a tool is attached).
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

// ---------------------------------------------------------------- errors --
void set_error(const char* fmt, ...);
int cuda_fail(cudaError_t e, const char* what);
#define WFA_STR2(x) #x
#define WFA_STR(x) WFA_STR2(x)
#define WFA_CUDA(call)                                                                      \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess) return ::wfa::cuda_fail(e_, #call " (" __FILE__ ":" WFA_STR(__LINE__) ")"); \
    } while (0)

// ------------------------------------------------------- kernel parameters --
// Everything a sweep needs, by value (coefficients already rounded to fp32 on
// the host from fp64, in a fixed way, so every kernel sees the same bits).
struct SweepCoef {
    int n[3];              // nx, ny, nz
    long long sy, sz;      // element strides of y and z in the padded layout
    int periodic[3];       // axis periodic (both faces)
    int bkind[6];          // face kind (enum wfa_bc_kind)
    float tb[6];           // Dirichlet face value (fp32)
    float w_in[6];         // uniform k: coefficient of an interior face, k dt/h^2 + A_f
    float w_bd[6];         // uniform k: coefficient of the boundary face (Dirichlet: 2k dt/h^2 + A_f; else 0)
    float tcd[3];          // 2 dt / h_a^2 (per-cell k: face coefficient = tcd / (1/k_C + 1/k_D) + A_f)
    float adv[6];          // A_f: upwind coefficient of face f: -face dt*max(u,0)/h, +face dt*max(-u,0)/h
    float s_lo[3], s_hi[3];  // self term of a cell on a zero-flux face with advection
    int held[6];           // face holds its outer cell layer (Dirichlet cell)
    int ext[6];            // exchange face (z only): the neighbour values are in the halo layer,
                           // written there by an exchange with the next slab; interior formula
    int any_self;          // some zero-flux face carries a self term
    int halo_bc;           // the halo encodes every boundary face (see build_coef): the
                           // interior formula is exact on boundary cells too
    long long px, py, pz;  // padded extents (TMA coordinates live in [0, p*))
    long long lo, hi;      // valid element offsets relative to the domain origin
};

// Self-checking build (-DWFA_CHECKED): global stores and TMA coordinates are
// checked against their allocation; a bad one is recorded in the grid's
// status words (code, x, y, z, extra) and skipped instead of performed.
#ifdef WFA_CHECKED
__device__ __forceinline__ bool wfa_chk(bool ok, int* st, int code, int x, int y, int z, int e) {
    if (!ok && st) {
        if (atomicCAS(st, 0, code) == 0) {
            st[1] = x; st[2] = y; st[3] = z; st[4] = e;
        }
    }
    return ok;
}
#define WFA_CHK(ok, st, code, x, y, z, e) ::wfa::wfa_chk((ok), (st), (code), (x), (y), (z), (e))
#else
#define WFA_CHK(ok, st, code, x, y, z, e) true
#endif

}  // namespace wfa

struct wfa_grid_s {
    int n[3];
    double h[3];
    int storage;          // WFA_F32 / WFA_BF16
    int esize;            // bytes per stored element
    cudaStream_t stream;
    long long px, py, pz; // padded extents (elements)
    void* T[2];           // ping-pong padded fields (allocation bases)
    float* k;             // padded per-cell conductivity or nullptr (fp64 stability limit)
    float* r;             // padded reciprocal conductivity 1/k (the sweeps' operand)
    int cur;              // buffer holding the current field
    double k_uniform;
    double u[3];
    int bc_kind[6];
    double bc_value[6];
    double dt;
    double limit;         // stability limit dt_max of the current coefficients and faces
    bool limit_valid;
    bool field_set, coeffs_set, dt_set, halo_dirty;
    bool k_halo_dirty;    // k twins / ghost layers and 1/k must be rebuilt before use
    long long steps_done;
    int force_depth, force_variant;   // wfa_set_tuning (0 = automatic)
    int force_zchunk;                 // wfa_set_zchunk: planes per z chunk of the column kernels (0 = automatic)
    double* d_partials;   // fp64 reduction partials (scratch)
    double* h_result;     // pinned host word for reduction results
    float* d_stage;       // dense fp32 staging buffer for set/read (scratch)
    int* d_status;        // device error word (a bounded wait that gave up)
    int* h_status;        // pinned host copy
    void* tmaps;          // wfa::TmapCache (TMA descriptors for the current tile box)
    int tuned_depth, tuned_variant;   // configuration picked by the autotuner (0 = none)
    int tuned_zchunk;                 // its z chunk length (0 = automatic)
    bool own_T, own_k;    // the library allocated T[] / k and r (else the caller attached them)
    float* ext_k;         // caller buffers for k and 1/k, used when per-cell k is set
    float* ext_r;
    long long launches;   // kernels launched by the sweeps so far (wfa_launch_count)
    int timing_every;     // wfa_set_kernel_timing: sample every n-th pass (0 = off)
    long long timing_pass;
    void* timing;         // wfa::KernelTiming (recorded event pairs)
    void* graphs;         // wfa::StepGraphs (captured runs of passes for small grids)
    void* cg;             // wfa::CgWork (work vectors and graph of the implicit solver)
    int cg_method;        // WFA_CG_CLASSIC / WFA_CG_PIPELINED (wfa_set_cg_method)
    cudaEvent_t xev;      // orders plane exchanges against this grid's stream (wfa_exchange)
    bool thin[2];         // buffer's periodic copies hold one layer without corners (a thin column
                          // pass wrote it): enough for one-step kernels, not for the tiled ones
};

namespace wfa {

inline long long domain_offset(const wfa_grid_s* g) {
    return ((long long)HALO * g->py + HALO) * g->px + HALO;
}
inline size_t field_elems(const wfa_grid_s* g) { return (size_t)g->px * g->py * g->pz; }
// Bytes between an allocation and element 0 of the padded array it holds.
inline size_t lead_bytes(int esize) { return (size_t)((128 - (HALO * esize) % 128) % 128); }
constexpr size_t LEAD_SLACK = 128;   // an allocation holds the array plus this much
inline bool has_exchange_face(const wfa_grid_s* g) {
    return g->bc_kind[4] == WFA_BC_EXCHANGE || g->bc_kind[5] == WFA_BC_EXCHANGE;
}

int build_coef(const wfa_grid_s* g, SweepCoef* c);       // host: fp64 -> fp32 coefficients
int refresh_halo(wfa_grid_s* g, int buf);                 // twins + held layers of one buffer
int launch_sweep(wfa_grid_s* g, long long nsteps);        // advance nsteps on g->stream
int check_status(wfa_grid_s* g);                          // sync + report a device-side timeout
int autotune(wfa_grid_s* g, int* depth, int* variant);    // pick the fastest kernel configuration
int prepare_coeff_halo(wfa_grid_s* g);                    // k periodic twins, then 1/k
void free_cg(wfa_grid_s* g);
void* pinned_word();                                      // a 64-byte pinned host slot
void pinned_release(void* w);
void free_tmaps(wfa_grid_s* g);
void free_timing(wfa_grid_s* g);
void free_graphs(wfa_grid_s* g);
cudaError_t dev_alloc(void** p, size_t bytes, cudaStream_t st);   // grid memory pool, stream-ordered
void dev_free(void* p, cudaStream_t st);
// a padded array of `bytes` with elements of esize bytes (see lead_bytes)
cudaError_t padded_alloc(void** p, size_t bytes, int esize, cudaStream_t st);
void padded_free(void* p, int esize, cudaStream_t st);
int grid_rebind_stream(wfa_grid_s* g, cudaStream_t st);          // move a quiet grid to another stream
int grid_move_stream(wfa_grid_s* g, cudaStream_t st);            // the same, the caller has waited already

// ----------------------------------------------------------- device math --
// The fixed per-cell arithmetic. Every kernel that updates a cell calls these
// with the same operands, so any two kernels (any tile shape, temporal depth
// or batching) produce bit-identical fields. The *_rn intrinsics are never
// contracted into other operations by the compiler.

// Face coefficient between two cells from their reciprocal conductivities
// ra = 1/k_C, rb = 1/k_D: the harmonic mean 2 k_C k_D / (k_C + k_D) equals
// 2 / (ra + rb); tcd = 2 dt / h^2. A zero conductivity (r = inf) gives 0,
// the harmonic mean's limit. Symmetric in (ra, rb) bit for bit.
// The reciprocal is the hardware approximation (PTX rcp.approx.ftz.f32,
// about 1 ulp; 1/inf = 0), one instruction.
__device__ __forceinline__ float rcp_approx(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float face_r(float ra, float rb, float tcd) {
    return __fmul_rn(tcd, rcp_approx(__fadd_rn(ra, rb)));
}

// Dirichlet face: conductance 2 k_C / h^2 (value on the face, half a cell
// away) = tcd / r_C.
__device__ __forceinline__ float dirichlet_r(float rc, float tcd) { return __fmul_rn(tcd, rcp_approx(rc)); }

// Sum of the face terms of one cell: sum_f w_f (T_f - T_C), faces in the
// order -x, +x, -y, +y, -z, +z. The update is T' = T_C + acc (plus s T_C
// first when the cell has a nonzero zero-flux self term).
__device__ __forceinline__ float flux_sum(float tc, float txm, float txp, float tym, float typ, float tzm,
                                          float tzp, float wxm, float wxp, float wym, float wyp, float wzm,
                                          float wzp) {
    float acc = __fmul_rn(wxm, __fsub_rn(txm, tc));
    acc = __fmaf_rn(wxp, __fsub_rn(txp, tc), acc);
    acc = __fmaf_rn(wym, __fsub_rn(tym, tc), acc);
    acc = __fmaf_rn(wyp, __fsub_rn(typ, tc), acc);
    acc = __fmaf_rn(wzm, __fsub_rn(tzm, tc), acc);
    return __fmaf_rn(wzp, __fsub_rn(tzp, tc), acc);
}
__device__ __forceinline__ float finish_update(float tc, float acc, float s) {
    if (s != 0.0f) acc = __fmaf_rn(s, tc, acc);
    return __fadd_rn(tc, acc);
}

// Self term of a cell from the zero-flux faces it touches (fixed order).
__device__ __forceinline__ float self_term(const SweepCoef& c, int x, int y, int z) {
    float s = 0.0f;
    if (!c.any_self) return s;
    if (x == 0) s = __fadd_rn(s, c.s_lo[0]);
    if (x == c.n[0] - 1) s = __fadd_rn(s, c.s_hi[0]);
    if (y == 0) s = __fadd_rn(s, c.s_lo[1]);
    if (y == c.n[1] - 1) s = __fadd_rn(s, c.s_hi[1]);
    if (z == 0) s = __fadd_rn(s, c.s_lo[2]);
    if (z == c.n[2] - 1) s = __fadd_rn(s, c.s_hi[2]);
    return s;
}

// Cell held by a Dirichlet-cell layer.
__device__ __forceinline__ bool is_held(const SweepCoef& c, int x, int y, int z) {
    return (c.held[0] && x == 0) || (c.held[1] && x == c.n[0] - 1) || (c.held[2] && y == 0) ||
           (c.held[3] && y == c.n[1] - 1) || (c.held[4] && z == 0) || (c.held[5] && z == c.n[2] - 1);
}

// Storage conversions.
template <typename S> __device__ __forceinline__ float to_f32(S v);
template <> __device__ __forceinline__ float to_f32<float>(float v) { return v; }
template <> __device__ __forceinline__ float to_f32<__nv_bfloat16>(__nv_bfloat16 v) {
    return __bfloat162float(v);
}
template <typename S> __device__ __forceinline__ S from_f32(float v);
template <> __device__ __forceinline__ float from_f32<float>(float v) { return v; }
template <> __device__ __forceinline__ __nv_bfloat16 from_f32<__nv_bfloat16>(float v) {
    return __float2bfloat16_rn(v);
}
// Value as stored (bf16 fields round after every step, also inside a fused block).
template <typename S> __device__ __forceinline__ float storage_round(float v) {
    return to_f32<S>(from_f32<S>(v));
}

// Twins of coordinate x along an axis of n cells inside [-HALO, n + HALO):
// the first one and how many there are (1 when the axis is not periodic or x
// is far from both ends).
__device__ __forceinline__ void twin_range(int x, int n, bool periodic, int* first, int* count) {
    if (periodic && (x < HALO || x >= n - HALO)) {
        const int lo = x - ((x + HALO) / n) * n;           // smallest twin >= -HALO
        *first = lo;
        *count = (n + HALO - 1 - lo) / n + 1;              // twins below n + HALO
    } else {
        *first = x;
        *count = 1;
    }
}

// Write v at (x, y, z) and at every periodic twin of that cell inside the halo.
template <typename S>
__device__ __forceinline__ void store_with_twins(S* origin, const SweepCoef& c, int x, int y, int z,
                                                 S v, int* st = nullptr) {
    int x0, nxt, y0, nyt, z0, nzt;
    twin_range(x, c.n[0], c.periodic[0] != 0, &x0, &nxt);
    twin_range(y, c.n[1], c.periodic[1] != 0, &y0, &nyt);
    twin_range(z, c.n[2], c.periodic[2] != 0, &z0, &nzt);
    for (int iz = 0; iz < nzt; ++iz) {
        const int zz = z0 + iz * c.n[2];
        for (int iy = 0; iy < nyt; ++iy) {
            const int yy = y0 + iy * c.n[1];
            for (int ix = 0; ix < nxt; ++ix) {
                const int xx = x0 + ix * c.n[0];
                const long long off = (long long)zz * c.sz + (long long)yy * c.sy + xx;
                if (WFA_CHK(off >= c.lo && off < c.hi, st, 11, xx, yy, zz, 0)) origin[off] = v;
            }
        }
    }
}

}  // namespace wfa
