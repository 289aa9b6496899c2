// Grid handles, field transfer (pack / unpack), halo maintenance and the fp64
// reductions (total heat, stability limit) behind the C ABI in include/wfa.h.
#include <stdarg.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <map>
#include <mutex>
#include <new>
#include <vector>

#include "wfa_internal.cuh"

namespace wfa {

static thread_local std::string g_last_error;

void set_error(const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
}

int cuda_fail(cudaError_t e, const char* what) {
    set_error("%s failed: %s", what, cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? WFA_ERR_OOM : WFA_ERR_CUDA;
}

static int fail(int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return code;
}

// ----------------------------------------------------------- device memory --
// Grid buffers come from one stream-ordered memory pool per device that keeps
// freed memory for reuse: creating and destroying a grid per request (as the
// server does) costs no device-wide synchronisation, and once the pool has
// grown no trip to the driver's allocator.
static std::mutex g_pool_mu;
static std::map<int, cudaMemPool_t> g_pools;

static cudaMemPool_t grid_pool() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
    std::lock_guard<std::mutex> lk(g_pool_mu);
    auto it = g_pools.find(dev);
    if (it != g_pools.end()) return it->second;
    cudaMemPoolProps props;
    memset(&props, 0, sizeof props);
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t pool = nullptr;
    if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) return nullptr;
    uint64_t keep = ~0ull;   // never hand freed memory back to the driver
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    g_pools[dev] = pool;
    return pool;
}

// Allocations left before an injected failure (-1: none armed).
static std::atomic<int> g_fail_countdown{-1};

static bool injected_failure() {
    static std::once_flag env_once;   // WFA_FAULT_ALLOC_AT=n: the n-th allocation of the process fails
    std::call_once(env_once, [] {
        const char* v = getenv("WFA_FAULT_ALLOC_AT");
        const long n = v ? strtol(v, nullptr, 10) : 0;
        if (n >= 1 && n < (1L << 30)) g_fail_countdown.store((int)n - 1);
    });
    int cur = g_fail_countdown.load();
    while (cur >= 0)
        if (g_fail_countdown.compare_exchange_weak(cur, cur - 1)) return cur == 0;
    return false;
}

cudaError_t dev_alloc(void** p, size_t bytes, cudaStream_t st) {
    if (injected_failure()) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    cudaMemPool_t pool = grid_pool();
    if (!pool) return cudaErrorMemoryAllocation;
    return cudaMallocFromPoolAsync(p, bytes, pool, st);
}

void dev_free(void* p, cudaStream_t st) {
    if (p) cudaFreeAsync(p, st);
}

cudaError_t padded_alloc(void** p, size_t bytes, int esize, cudaStream_t st) {
    void* raw = nullptr;
    const cudaError_t e = dev_alloc(&raw, bytes + LEAD_SLACK, st);
    *p = e == cudaSuccess ? (char*)raw + lead_bytes(esize) : nullptr;
    return e;
}

void padded_free(void* p, int esize, cudaStream_t st) {
    if (p) dev_free((char*)p - lead_bytes(esize), st);
}

// Pinned host words (reduction results, status) carved from shared slabs of
// 1024 slots of 64 bytes, so a grid costs no pinned allocation of its own.
static std::mutex g_pin_mu;
static std::vector<void*> g_pin_free;

void* pinned_word() {
    std::lock_guard<std::mutex> lk(g_pin_mu);
    if (g_pin_free.empty()) {
        char* slab = nullptr;
        if (cudaMallocHost(&slab, 1024 * 64) != cudaSuccess) return nullptr;
        for (int i = 1023; i >= 0; --i) g_pin_free.push_back(slab + 64 * i);
    }
    void* w = g_pin_free.back();
    g_pin_free.pop_back();
    return w;
}

void pinned_release(void* w) {
    if (!w) return;
    std::lock_guard<std::mutex> lk(g_pin_mu);
    g_pin_free.push_back(w);
}

// ------------------------------------------------------------ coefficients --
int build_coef(const wfa_grid_s* g, SweepCoef* c) {
    memset(c, 0, sizeof *c);
    for (int a = 0; a < 3; ++a) c->n[a] = g->n[a];
    c->sy = g->px;
    c->sz = g->px * g->py;
    c->px = g->px;
    c->py = g->py;
    c->pz = g->pz;
    c->lo = -domain_offset(g);
    c->hi = (long long)field_elems(g) - domain_offset(g);
    const double dt = g->dt;
    for (int a = 0; a < 3; ++a) {
        const int lo = g->bc_kind[2 * a], hi = g->bc_kind[2 * a + 1];
        if ((lo == WFA_BC_PERIODIC) != (hi == WFA_BC_PERIODIC))
            return fail(WFA_ERR_BC, "axis %d: a periodic face needs a periodic opposite face", a);
        if ((lo == WFA_BC_EXCHANGE || hi == WFA_BC_EXCHANGE) && a != 2)
            return fail(WFA_ERR_BC, "axis %d: exchange faces are z faces", a);
        if ((lo == WFA_BC_DIRICHLET_CELL || hi == WFA_BC_DIRICHLET_CELL) && g->n[a] < 3)
            return fail(WFA_ERR_BC, "axis %d: held boundary cells need an edge >= 3", a);
        c->periodic[a] = lo == WFA_BC_PERIODIC;
        const double h = g->h[a];
        const double cd = dt / (h * h);
        const double ap = dt * (g->u[a] > 0 ? g->u[a] : 0.0) / h;   // -face inflow weight
        const double am = dt * (g->u[a] < 0 ? -g->u[a] : 0.0) / h;  // +face inflow weight
        c->tcd[a] = (float)(2.0 * cd);
        c->adv[2 * a] = (float)ap;
        c->adv[2 * a + 1] = (float)am;
        c->w_in[2 * a] = (float)(g->k_uniform * cd + ap);
        c->w_in[2 * a + 1] = (float)(g->k_uniform * cd + am);
        for (int side = 0; side < 2; ++side) {
            const int f = 2 * a + side;
            const double A = side == 0 ? ap : am;
            c->bkind[f] = g->bc_kind[f];
            c->tb[f] = (float)g->bc_value[f];
            c->held[f] = g->bc_kind[f] == WFA_BC_DIRICHLET_CELL;
            c->ext[f] = g->bc_kind[f] == WFA_BC_EXCHANGE;
            if (g->bc_kind[f] == WFA_BC_DIRICHLET) c->w_bd[f] = (float)(2.0 * g->k_uniform * cd + A);
            else if (g->bc_kind[f] == WFA_BC_PERIODIC || c->ext[f]) c->w_bd[f] = c->w_in[f];
            else c->w_bd[f] = 0.0f;
        }
        // a zero-flux face stops the advective flux: the cell keeps (or loses)
        // the upwind transport that its interior-face weights assume
        if (lo == WFA_BC_ZEROFLUX) c->s_lo[a] = (float)(am - ap);
        if (hi == WFA_BC_ZEROFLUX) c->s_hi[a] = (float)(ap - am);
        if (c->s_lo[a] != 0.0f || c->s_hi[a] != 0.0f) c->any_self = 1;
    }
    // Boundary faces as ghost cells. With per-cell k the halo layer next to a
    // Dirichlet face holds the face value with k = inf (1/k = 0), so the
    // harmonic-mean face coefficient tcd / (1/k_C + 0) is the Dirichlet one,
    // tcd / (1/k_C), bit for bit; next to a zero-flux face it holds k = 0
    // (1/k = inf), so the coefficient is 0. The interior formula is then exact
    // on boundary cells, unless a cell is held, a zero-flux face meets
    // advection (no ghost value gives the self term), or a bf16 halo cannot
    // hold a Dirichlet value exactly.
    bool any_adv = false;
    for (int f = 0; f < 6; ++f) any_adv = any_adv || c->adv[f] != 0.0f;
    c->halo_bc = g->r != nullptr;
    for (int f = 0; f < 6; ++f) {
        const int kind = g->bc_kind[f];
        if (kind == WFA_BC_DIRICHLET_CELL) c->halo_bc = 0;
        if (kind == WFA_BC_ZEROFLUX && any_adv) c->halo_bc = 0;
        if (kind == WFA_BC_DIRICHLET && g->storage == WFA_BF16) {
            uint32_t bits;
            memcpy(&bits, &c->tb[f], sizeof bits);
            if (bits & 0xFFFFu) c->halo_bc = 0;   // low 16 bits set: not a bf16 value
        }
    }
    return WFA_OK;
}

__global__ void recip_kernel(const float* __restrict__ k, float* __restrict__ r, long long n);

// ------------------------------------------------------------ pack/unpack --
struct Geo {
    int n[3];
    long long px, py;
};

// Dense (x fastest, no halo) <-> padded layout, one warp per (y, z) row: the
// row index is split once per row in 32-bit arithmetic and the warp's
// accesses are consecutive on both sides. `dense` may be device memory or
// pinned host memory (read or written directly over the host link).
template <typename S>
__global__ void pack_kernel(const float* __restrict__ dense, S* __restrict__ origin, const __grid_constant__ Geo geo) {
    const unsigned ny = (unsigned)geo.n[1];
    const long long rows = (long long)geo.n[1] * geo.n[2];
    const long long sz = geo.px * geo.py;
    const int lane = threadIdx.x & 31;
    const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
    for (long long r = blockIdx.x * (long long)(blockDim.x >> 5) + (threadIdx.x >> 5); r < rows; r += warps) {
        const long long z = r / ny, y = r - z * ny;
        const float* src = dense + r * geo.n[0];
        S* dst = origin + z * sz + y * geo.px;
        for (int x = lane; x < geo.n[0]; x += 32) dst[x] = from_f32<S>(src[x]);
    }
}

template <typename S>
__global__ void unpack_kernel(const S* __restrict__ origin, float* __restrict__ dense, const __grid_constant__ Geo geo) {
    const unsigned ny = (unsigned)geo.n[1];
    const long long rows = (long long)geo.n[1] * geo.n[2];
    const long long sz = geo.px * geo.py;
    const int lane = threadIdx.x & 31;
    const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
    for (long long r = blockIdx.x * (long long)(blockDim.x >> 5) + (threadIdx.x >> 5); r < rows; r += warps) {
        const long long z = r / ny, y = r - z * ny;
        const S* src = origin + z * sz + y * geo.px;
        float* dst = dense + r * geo.n[0];
        for (int x = lane; x < geo.n[0]; x += 32) dst[x] = to_f32<S>(src[x]);
    }
}

// Device address of a host buffer the GPU can read and write directly
// (pinned, or mapped), or nullptr (pageable: go through the staging buffer).
static const void* host_device_view(const void* p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();   // clear: an unknown pointer is just not device-accessible
        return nullptr;
    }
    return at.type == cudaMemoryTypeHost ? at.devicePointer : nullptr;
}

struct HaloSpec {
    int n[3];
    long long px, py;
    int periodic[3];
    int held[6];
    int dirichlet[6];   // face value on the face (ghost cells hold it)
    float gam[6];       // held-layer or Dirichlet value
    int ext[6];         // exchange face: its halo planes hold the neighbour slab's values (left alone)
};

// Row (y, z) of the padded box lies in the halo planes beyond an exchange
// face, which an exchange with the neighbouring slab fills (whole planes).
__device__ __forceinline__ bool exchange_row(const HaloSpec& h, int z) {
    return (h.ext[4] && z < 0) || (h.ext[5] && z >= h.n[2]);
}

// Dirichlet face whose ghost layer holds the halo cell c (outside the domain
// on exactly one axis, and that axis not periodic), or -1.
__device__ __forceinline__ int ghost_face(const HaloSpec& h, const int c[3]) {
    int face = -1, outside = 0;
    for (int a = 0; a < 3; ++a) {
        if (c[a] < 0 || c[a] >= h.n[a]) {
            ++outside;
            face = 2 * a + (c[a] >= h.n[a]);
            if (h.periodic[a]) face = -1;
        }
    }
    return outside == 1 && face >= 0 && h.dirichlet[face] ? face : -1;
}

// Value a domain cell must hold if a held layer covers it (last face wins).
__device__ __forceinline__ bool held_value(const HaloSpec& h, int x, int y, int z, float* v) {
    bool any = false;
    const int c[3] = {x, y, z};
    for (int f = 0; f < 6; ++f) {
        if (!h.held[f]) continue;
        const int a = f >> 1;
        if (c[a] == ((f & 1) ? h.n[a] - 1 : 0)) {
            *v = h.gam[f];
            any = true;
        }
    }
    return any;
}

// One cell (x, y, z) of the padded box of a field buffer: held layers get
// their value, periodic twins a copy, the ghost layers of Dirichlet faces
// the face value, every other halo cell 0; other domain cells are left alone.
template <typename S>
__device__ __forceinline__ void halo_cell(S* __restrict__ base, const HaloSpec& h, int x, int y, int z) {
    const int c[3] = {x, y, z};
    bool outside = false, fill_zero = false;
    int w[3];
    for (int a = 0; a < 3; ++a) {
        w[a] = c[a];
        if (c[a] < 0 || c[a] >= h.n[a]) {
            outside = true;
            if (h.periodic[a]) w[a] = ((c[a] % h.n[a]) + h.n[a]) % h.n[a];
            else fill_zero = true;
        }
    }
    S* dst = base + ((long long)(z + HALO) * h.py + (y + HALO)) * h.px + (x + HALO);
    float v;
    if (!outside) {
        if (held_value(h, x, y, z, &v)) *dst = from_f32<S>(v);
        return;
    }
    if (fill_zero) {
        const int f = ghost_face(h, c);
        *dst = from_f32<S>(f >= 0 ? h.gam[f] : 0.0f);
        return;
    }
    if (held_value(h, w[0], w[1], w[2], &v)) {
        *dst = from_f32<S>(v);
    } else {
        const S* src = base + ((long long)(w[2] + HALO) * h.py + (w[1] + HALO)) * h.px + (w[0] + HALO);
        *dst = *src;
    }
}

// x positions of row (y, z) of the padded box that can need a write: all of
// them when the row lies outside the domain or on a held y / z layer, else
// the x halo and the two end cells (held x layers).
__device__ __forceinline__ bool full_row(const HaloSpec& h, int y, int z) {
    if (y < 0 || y >= h.n[1] || z < 0 || z >= h.n[2]) return true;
    return (h.held[2] && y == 0) || (h.held[3] && y == h.n[1] - 1) || (h.held[4] && z == 0) ||
           (h.held[5] && z == h.n[2] - 1);
}
__device__ __forceinline__ int row_x(const HaloSpec& h, bool full, int t) {
    if (full) return t - HALO;
    if (t < HALO) return t - HALO;                     // -HALO .. -1
    if (t < 2 * HALO) return h.n[0] + (t - HALO);      // n .. n + HALO - 1
    return t == 2 * HALO ? 0 : h.n[0] - 1;             // end cells
}

// Halo and held layers of one padded buffer, one warp per row of the padded
// box (no per-cell 64-bit index arithmetic; interior rows touch 18 cells).
template <typename S>
__global__ void halo_kernel(S* __restrict__ base, const __grid_constant__ HaloSpec h) {
    const int ey = h.n[1] + 2 * HALO;
    const long long rows = (long long)ey * (h.n[2] + 2 * HALO);
    const int lane = threadIdx.x & 31;
    const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
    for (long long r = blockIdx.x * (long long)(blockDim.x >> 5) + (threadIdx.x >> 5); r < rows; r += warps) {
        const int z = (int)(r / ey) - HALO;
        const int y = (int)(r - (long long)(z + HALO) * ey) - HALO;
        if (exchange_row(h, z)) continue;
        const bool full = full_row(h, y, z);
        const int count = full ? h.n[0] + 2 * HALO : 2 * HALO + 2;
        for (int t = lane; t < count; t += 32) halo_cell<S>(base, h, row_x(h, full, t), y, z);
    }
}

static int grid_blocks(long long n, int threads) {
    long long b = (n + threads - 1) / threads;
    if (b > 152 * 16) b = 152 * 16;
    return (int)(b < 1 ? 1 : b);
}

static HaloSpec halo_spec(const wfa_grid_s* g) {
    HaloSpec h;
    memset(&h, 0, sizeof h);
    for (int a = 0; a < 3; ++a) {
        h.n[a] = g->n[a];
        h.periodic[a] = g->bc_kind[2 * a] == WFA_BC_PERIODIC && g->bc_kind[2 * a + 1] == WFA_BC_PERIODIC;
    }
    h.px = g->px;
    h.py = g->py;
    for (int f = 0; f < 6; ++f) {
        h.held[f] = g->bc_kind[f] == WFA_BC_DIRICHLET_CELL;
        h.dirichlet[f] = g->bc_kind[f] == WFA_BC_DIRICHLET;
        h.gam[f] = (float)g->bc_value[f];
        h.ext[f] = g->bc_kind[f] == WFA_BC_EXCHANGE;
    }
    return h;
}

// Halo of buffer buf, then of the other one: a pass writes only domain cells
// and periodic twins, so the ghost layers of both must be in place. (The
// other buffer's twins and held cells are rewritten by the next pass.)
int refresh_halo(wfa_grid_s* g, int buf) {
    HaloSpec h = halo_spec(g);
    const long long rows = (long long)(g->n[1] + 2 * HALO) * (g->n[2] + 2 * HALO);
    const int thr = 256;
    for (int b : {buf, 1 - buf}) {
        if (g->storage == WFA_BF16)
            halo_kernel<__nv_bfloat16><<<grid_blocks(rows * 32, thr), thr, 0, g->stream>>>((__nv_bfloat16*)g->T[b], h);
        else
            halo_kernel<float><<<grid_blocks(rows * 32, thr), thr, 0, g->stream>>>((float*)g->T[b], h);
        WFA_CUDA(cudaGetLastError());
    }
    g->thin[0] = g->thin[1] = false;   // every periodic copy, corners included
    return WFA_OK;
}

// --------------------------------------------------------------- reductions --
constexpr int RED_BLOCKS = 304;
// the stability passes are latency-bound (divisions, seven k reads a cell):
// more warps per SM; their partials fit the 4096-double scratch below the
// word kept for the k check (index 4095)
constexpr int RATE_BLOCKS = 152 * 8;
constexpr int RATE_P2 = 1280;
constexpr int RATE_RISKY = 2560;   // pass 1's per-block flags: the block met a risky cell
static_assert(RATE_P2 > RATE_BLOCKS + 1 && RATE_P2 + RATE_BLOCKS <= RATE_RISKY && RATE_RISKY + RATE_BLOCKS < 4095,
              "scratch layout");
constexpr int RED_THREADS = 256;

template <typename S>
__global__ void __launch_bounds__(RED_THREADS) heat_partial_kernel(const S* __restrict__ origin, const __grid_constant__ Geo geo,
                                                                   double* __restrict__ partials) {
    __shared__ double sh[RED_THREADS];
    const long long N = (long long)geo.n[0] * geo.n[1] * geo.n[2];
    const long long sz = geo.px * geo.py;
    double acc = 0.0;
    for (long long i = blockIdx.x * (long long)RED_THREADS + threadIdx.x; i < N;
         i += (long long)RED_BLOCKS * RED_THREADS) {
        const int x = (int)(i % geo.n[0]);
        const long long r = i / geo.n[0];
        const int y = (int)(r % geo.n[1]);
        const int z = (int)(r / geo.n[1]);
        acc += (double)to_f32<S>(origin[z * sz + y * geo.px + x]);
    }
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int s = RED_THREADS / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) partials[blockIdx.x] = sh[0];
}

// Fixed-order finish: one block, a tree over RED_BLOCKS partials.
__global__ void __launch_bounds__(512) finish_sum_kernel(const double* __restrict__ partials, int n,
                                                         double scale, double* __restrict__ out) {
    __shared__ double sh[512];
    double acc = 0.0;
    for (int i = threadIdx.x; i < n; i += 512) acc += partials[i];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int s = 256; s > 0; s >>= 1) {
        if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = sh[0] * scale;
}

// Heat that one explicit step from the current field brings in through the
// Dirichlet faces, per unit volume and time, block partial sums in fp64 (see
// wfa_boundary_flux). blockIdx.y is the face; a block of 256 threads walks
// its plane. Diffusion through the face: 2 k_C (T_b - T_C) / h^2 (value on
// the face, half a cell away); advection: the upwind value is T_b for
// inflow and T_C for outflow.
struct FluxSpec {
    int n[3];
    long long px, py;
    int dirichlet[6];
    double tb[6];
    double inv_h2[3], u_h[3];   // 1/h^2, u / h
    double k_uniform;
};

template <typename S>
__global__ void __launch_bounds__(RED_THREADS) flux_partial_kernel(const S* __restrict__ origin,
                                                                   const float* __restrict__ korigin,
                                                                   const __grid_constant__ FluxSpec fs,
                                                                   double* __restrict__ partials) {
    __shared__ double sh[RED_THREADS];
    const int f = blockIdx.y, ax = f >> 1, side = f & 1;
    double acc = 0.0;
    if (fs.dirichlet[f]) {
        const int b = ax == 0 ? 1 : 0, d = ax == 2 ? 1 : 2;
        const unsigned nb = (unsigned)fs.n[b], plane = nb * (unsigned)fs.n[d];
        for (unsigned t = blockIdx.x * RED_THREADS + threadIdx.x; t < plane; t += gridDim.x * RED_THREADS) {
            int c[3];
            c[ax] = side ? fs.n[ax] - 1 : 0;
            c[b] = (int)(t % nb);
            c[d] = (int)(t / nb);
            const long long i = ((long long)c[2] * fs.py + c[1]) * fs.px + c[0];
            const double tc = (double)to_f32<S>(origin[i]);
            const double kc = korigin ? (double)korigin[i] : fs.k_uniform;
            const double tb = fs.tb[f], u = fs.u_h[ax];
            acc += 2.0 * kc * (tb - tc) * fs.inv_h2[ax];
            // inflow through the low face when u > 0, through the high face when u < 0
            if (side == 0) acc += u > 0 ? u * tb : u * tc;
            else acc -= u > 0 ? u * tc : u * tb;
        }
    }
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int st = RED_THREADS / 2; st > 0; st >>= 1) {
        if (threadIdx.x < st) sh[threadIdx.x] += sh[threadIdx.x + st];
        __syncthreads();
    }
    if (threadIdx.x == 0) partials[blockIdx.y * gridDim.x + blockIdx.x] = sh[0];
}

struct RateSpec {
    int n[3];
    long long px, py;
    int kind[6];
    int held[6];
    double inv_h2[3], up[3], um[3];  // 1/h^2, max(u,0)/h, max(-u,0)/h
    float inv_h2f[3], upf[3], umf[3];
    double k_uniform;
};

__device__ __forceinline__ double harm64(double a, double b) {
    const double s = a + b;
    return s > 0.0 ? 2.0 * a * b / s : 0.0;
}

__device__ __forceinline__ bool rate_held(const RateSpec& r, const int c[3]) {
    bool held = false;
    for (int f = 0; f < 6; ++f)
        if (r.held[f] && c[f >> 1] == ((f & 1) ? r.n[f >> 1] - 1 : 0)) held = true;
    return held;
}

// D_C of one cell in fp64 (see wfa_stability_dt): the sum of the cell's
// outflow coefficients per unit dt, faces in the order -x, +x, -y, +y, -z, +z.
__device__ __forceinline__ double rate64(const float* __restrict__ korigin, const RateSpec& r, const int c[3],
                                         long long idx) {
    const long long st[3] = {1, r.px, r.px * r.py};
    const double kC = korigin ? (double)korigin[idx] : r.k_uniform;
    double D = 0.0;
    for (int a = 0; a < 3; ++a) {
        for (int side = 0; side < 2; ++side) {
            const int f = 2 * a + side;
            const bool edge = side == 0 ? c[a] == 0 : c[a] == r.n[a] - 1;
            bool active = true;
            if (edge && r.kind[f] != WFA_BC_PERIODIC && r.kind[f] != WFA_BC_EXCHANGE) {
                if (r.kind[f] == WFA_BC_DIRICHLET) D += 2.0 * kC * r.inv_h2[a];
                else active = false;
            } else {
                // interior or periodic neighbour (periodic twins live in the halo)
                const double kD = korigin ? (double)korigin[idx + (side ? st[a] : -st[a])] : r.k_uniform;
                D += harm64(kC, kD) * r.inv_h2[a];
            }
            if (active) D += side ? r.up[a] : r.um[a];
        }
    }
    return D;
}

// The same sum in fp32 (only to find the candidates of the fp64 pass):
// every term is >= 0 and every operation is correctly rounded except the
// division of the harmonic mean, a fast division within 2 ulp for a
// denominator in (2^-126, 2^126). For a cell whose k values lie in
// [1e-15, 1e15] (or are 0) no operand leaves the normal range and the result
// is within 24 units of 2^-24, relative, of the fp64 one (2 roundings and
// the division per harmonic mean, 2 per product with 1/h^2 and its
// conversion, at most 12 additions). A cell with other k values is `risky`.
// A cell whose six neighbours are all cells (inside the domain, or across a
// periodic or exchange face: their copies are in the halo); never held.
__device__ __forceinline__ bool rate_inner(const RateSpec& r, const int c[3]) {
    bool in = true;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const bool wlo = r.kind[2 * a] == WFA_BC_PERIODIC || r.kind[2 * a] == WFA_BC_EXCHANGE;
        const bool whi = r.kind[2 * a + 1] == WFA_BC_PERIODIC || r.kind[2 * a + 1] == WFA_BC_EXCHANGE;
        in = in & (wlo | (c[a] > 0)) & (whi | (c[a] < r.n[a] - 1));   // no short circuit: no branches
    }
    return in;
}

// inner (rate_inner): the same operations in the same order without the
// face tests.
__device__ __forceinline__ float rate32(const float* __restrict__ korigin, const RateSpec& r, const int c[3],
                                        long long idx, bool* risky, bool inner) {
    const long long st[3] = {1, r.px, r.px * r.py};
    const float kC = korigin[idx];
    bool bad = (kC != 0.0f) & !((kC >= 1e-15f) & (kC <= 1e15f));   // bitwise: no branches
    float D = 0.0f;
    if (inner) {
        const float k2 = __fmul_rn(2.0f, kC);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
#pragma unroll
            for (int side = 0; side < 2; ++side) {
                const float kD = korigin[idx + (side ? st[a] : -st[a])];
                bad = bad | ((kD != 0.0f) & !((kD >= 1e-15f) & (kD <= 1e15f)));
                const float s2 = __fadd_rn(kC, kD);
                const float h = s2 > 0.0f ? __fdividef(__fmul_rn(k2, kD), s2) : 0.0f;
                D = __fadd_rn(D, __fmul_rn(h, r.inv_h2f[a]));
                D = __fadd_rn(D, side ? r.upf[a] : r.umf[a]);
            }
        }
        *risky = bad;
        return D;
    }
    for (int a = 0; a < 3; ++a) {
        for (int side = 0; side < 2; ++side) {
            const int f = 2 * a + side;
            const bool edge = side == 0 ? c[a] == 0 : c[a] == r.n[a] - 1;
            bool active = true;
            if (edge && r.kind[f] != WFA_BC_PERIODIC && r.kind[f] != WFA_BC_EXCHANGE) {
                if (r.kind[f] == WFA_BC_DIRICHLET) D = __fadd_rn(D, __fmul_rn(__fmul_rn(2.0f, kC), r.inv_h2f[a]));
                else active = false;
            } else {
                const float kD = korigin[idx + (side ? st[a] : -st[a])];
                bad = bad || (kD != 0.0f && !(kD >= 1e-15f && kD <= 1e15f));
                const float s2 = __fadd_rn(kC, kD);
                const float h = s2 > 0.0f ? __fdividef(__fmul_rn(__fmul_rn(2.0f, kC), kD), s2) : 0.0f;
                D = __fadd_rn(D, __fmul_rn(h, r.inv_h2f[a]));
            }
            if (active) D = __fadd_rn(D, side ? r.upf[a] : r.umf[a]);
        }
    }
    *risky = bad;
    return D;
}

// Every domain cell once: warp w of the launch takes rows (y, z) w, w + W, ...
// and its lanes the x of a row; f(c, idx) gets the cell and its padded offset.
template <typename F>
__device__ __forceinline__ void for_each_cell(const RateSpec& r, F f) {
    const long long rows = (long long)r.n[1] * r.n[2];
    const int lane = threadIdx.x & 31;
    const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
    for (long long row = blockIdx.x * (long long)(blockDim.x >> 5) + (threadIdx.x >> 5); row < rows; row += warps) {
        int c[3];
        c[2] = (int)(row / r.n[1]);
        c[1] = (int)(row - (long long)c[2] * r.n[1]);
        const long long base = (long long)c[2] * r.px * r.py + (long long)c[1] * r.px;
        for (int x = lane; x < r.n[0]; x += 32) {
            c[0] = x;
            f(c, base + x);
        }
    }
}

__device__ __forceinline__ void block_max_out(double best, double* __restrict__ out) {
    __shared__ double sh[RED_THREADS];
    sh[threadIdx.x] = best;
    __syncthreads();
    for (int s = RED_THREADS / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) sh[threadIdx.x] = fmax(sh[threadIdx.x], sh[threadIdx.x + s]);
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = sh[0];
}

// Block maxima of D_C in fp64 over every cell that is not held.
__global__ void __launch_bounds__(RED_THREADS) rate_partial_kernel(const float* __restrict__ korigin,
                                                                   const __grid_constant__ RateSpec r,
                                                                   double* __restrict__ partials) {
    double best = 0.0;
    for_each_cell(r, [&](const int c[3], long long idx) {
        if (!rate_held(r, c)) best = fmax(best, rate64(korigin, r, c, idx));
    });
    block_max_out(best, &partials[blockIdx.x]);
}

// Per-cell k, pass 1: block maxima of the fp32 D_C over the cells that are
// neither held nor risky, and per block whether it met a risky cell.
__global__ void __launch_bounds__(RED_THREADS) rate32_partial_kernel(const float* __restrict__ korigin,
                                                                     const __grid_constant__ RateSpec r,
                                                                     double* __restrict__ partials,
                                                                     double* __restrict__ risky_out) {
    float best = 0.0f;
    int any_risky = 0;
    for_each_cell(r, [&](const int c[3], long long idx) {
        const bool inner = rate_inner(r, c);
        if (!inner && rate_held(r, c)) return;
        bool risky;
        const float d = rate32(korigin, r, c, idx, &risky, inner);
        if (!risky) best = fmaxf(best, d);
        else any_risky = 1;
    });
    block_max_out((double)best, &partials[blockIdx.x]);
    any_risky = __syncthreads_or(any_risky);
    if (threadIdx.x == 0) risky_out[blockIdx.x] = any_risky ? 1.0 : 0.0;
}

// Per-cell k, pass 2: fp64 D_C of the candidates only, the cells whose fp32
// value reaches M (1 - 2^-12), M the pass-1 maximum, and the risky cells. The
// cell with the largest fp64 value is always a candidate: its fp32 value is
// at least M (1 - 2 * 24 * 2^-24) > M (1 - 2^-12). So the maximum over the
// candidates is the fp64 maximum over all cells, the same number as the
// one-pass reduction gives. Candidates lie only in the rows that pass-1
// blocks with a maximum at the threshold (or a risky cell) visited; with
// at most RATE_ACTIVE such blocks, every block of this launch takes a share
// of those rows (so the few that hold candidates do not serialise on one
// block), otherwise each block takes its pass-1 rows again.
constexpr int RATE_ACTIVE = 64;
__global__ void __launch_bounds__(RED_THREADS) rate_cand_kernel(const float* __restrict__ korigin,
                                                                const __grid_constant__ RateSpec r,
                                                                const double* __restrict__ pass1,
                                                                const double* __restrict__ risky,
                                                                const double* __restrict__ m32,
                                                                double* __restrict__ partials) {
    __shared__ int s_act[RATE_ACTIVE];
    __shared__ int s_nact;
    const float m = (float)*m32;
    const float thr = __fsub_rn(m, __fmul_rn(m, 0x1p-12f));
    const int lane = threadIdx.x & 31;
    if (threadIdx.x < 32) {   // the pass-1 blocks that may hold candidates, in order
        int n = 0;
        for (int base = 0; base < RATE_BLOCKS; base += 32) {
            const int b = base + lane;
            const bool act = b < RATE_BLOCKS && ((float)pass1[b] >= thr || risky[b] != 0.0);
            unsigned bits = __ballot_sync(0xffffffffu, act);
            while (bits) {
                const int i = __ffs(bits) - 1;
                bits &= bits - 1;
                if (lane == 0 && n < RATE_ACTIVE) s_act[n] = base + i;
                ++n;
            }
        }
        if (lane == 0) s_nact = n;
    }
    __syncthreads();
    const int nact = s_nact;
    double best = 0.0;
    auto cell = [&](const int c[3], long long idx) {
        const bool inner = rate_inner(r, c);
        if (!inner && rate_held(r, c)) return;
        bool rk;
        const float d = rate32(korigin, r, c, idx, &rk, inner);
        if (rk || d >= thr) best = fmax(best, rate64(korigin, r, c, idx));
    };
    if (nact > RATE_ACTIVE) {
        for_each_cell(r, cell);
    } else {
        // pass-1 block b took rows 8b + w + k W (w < 8 warps, W = all warps of
        // the launch); here warp g of the launch takes the j-th of those
        // rows for j = g, g + W, ..., over the active blocks in turn
        const int wpb = RED_THREADS / 32;
        const long long W = (long long)RATE_BLOCKS * wpb;
        const long long rows = (long long)r.n[1] * r.n[2];
        const long long gw = (long long)blockIdx.x * wpb + (threadIdx.x >> 5);
        for (int t = 0; t < nact; ++t) {
            const int b = s_act[t];
            const long long first = (long long)b * wpb;
            if (first >= rows) continue;
            const long long per = wpb * ((rows - first + W - 1) / W);   // an upper bound of b's rows
            for (long long j = gw; j < per; j += W) {
                const long long row = first + (j % wpb) + (j / wpb) * W;
                if (row >= rows) continue;
                int c[3];
                c[2] = (int)(row / r.n[1]);
                c[1] = (int)(row - (long long)c[2] * r.n[1]);
                const long long base = (long long)c[2] * r.px * r.py + (long long)c[1] * r.px;
                for (int x = lane; x < r.n[0]; x += 32) {
                    c[0] = x;
                    cell(c, base + x);
                }
            }
        }
    }
    block_max_out(best, &partials[blockIdx.x]);
}

__global__ void __launch_bounds__(512) finish_max_kernel(const double* __restrict__ partials, int n,
                                                         double* __restrict__ out) {
    __shared__ double sh[512];
    double m = 0.0;
    for (int i = threadIdx.x; i < n; i += 512) m = fmax(m, partials[i]);
    sh[threadIdx.x] = m;
    __syncthreads();
    for (int s = 256; s > 0; s >>= 1) {
        if (threadIdx.x < s) sh[threadIdx.x] = fmax(sh[threadIdx.x], sh[threadIdx.x + s]);
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = sh[0];
}

// k halo: periodic twins (the harmonic mean across a wrap face reads them),
// inf in the ghost layers of Dirichlet faces, 0 elsewhere (see build_coef).
// One warp per row of the padded box; interior rows touch only the x halo.
__global__ void k_halo_kernel(float* __restrict__ base, const __grid_constant__ HaloSpec h) {
    const int ey = h.n[1] + 2 * HALO;
    const long long rows = (long long)ey * (h.n[2] + 2 * HALO);
    const int lane = threadIdx.x & 31;
    const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
    for (long long r = blockIdx.x * (long long)(blockDim.x >> 5) + (threadIdx.x >> 5); r < rows; r += warps) {
        const int cz = (int)(r / ey) - HALO;
        const int cy = (int)(r - (long long)(cz + HALO) * ey) - HALO;
        if (exchange_row(h, cz)) continue;
        const bool full = cy < 0 || cy >= h.n[1] || cz < 0 || cz >= h.n[2];
        const int count = full ? h.n[0] + 2 * HALO : 2 * HALO;
        for (int t = lane; t < count; t += 32) {
            const int cx = full ? t - HALO : (t < HALO ? t - HALO : h.n[0] + (t - HALO));
            const int c[3] = {cx, cy, cz};
            bool outside = false, zero = false;
            int w[3];
            for (int a = 0; a < 3; ++a) {
                w[a] = c[a];
                if (c[a] < 0 || c[a] >= h.n[a]) {
                    outside = true;
                    if (h.periodic[a]) w[a] = ((c[a] % h.n[a]) + h.n[a]) % h.n[a];
                    else zero = true;
                }
            }
            if (!outside) continue;
            float* dst = base + ((long long)(c[2] + HALO) * h.py + (c[1] + HALO)) * h.px + (c[0] + HALO);
            *dst = zero ? (ghost_face(h, c) >= 0 ? INFINITY : 0.0f)
                        : base[((long long)(w[2] + HALO) * h.py + (w[1] + HALO)) * h.px + (w[0] + HALO)];
        }
    }
}

// Smallest index of a negative or non-finite k (bad stays at its initial
// value when every k is valid). copy: also write every k to `out` (src is
// then pinned host memory the GPU reads over the host link).
__global__ void check_k_kernel(const float* __restrict__ k, long long n, unsigned long long* bad,
                               float* __restrict__ out = nullptr) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float v = k[i];
        if (out) out[i] = v;
        if (!(v >= 0.0f && v <= 3.402823466e38f)) atomicMin(bad, (unsigned long long)i);
    }
}

int check_status(wfa_grid_s* g) {
    WFA_CUDA(cudaMemcpyAsync(g->h_status, g->d_status, 8 * sizeof(int), cudaMemcpyDeviceToHost, g->stream));
    WFA_CUDA(cudaStreamSynchronize(g->stream));
    if (g->h_status[0] != 0) {
        const int* st = g->h_status;
        const int code = st[0];
        cudaMemsetAsync(g->d_status, 0, 8 * sizeof(int), g->stream);
        cudaStreamSynchronize(g->stream);
        if (code >= 10)
            return fail(WFA_ERR_CUDA, "checked build: bad access, code %d at (%d, %d, %d) extra %d", code, st[1],
                        st[2], st[3], st[4]);
        return fail(WFA_ERR_TIMEOUT, "a device-side wait gave up after its time limit (code %d)", code);
    }
    return WFA_OK;
}

// r = 1/k (IEEE division; 1/0 = inf makes every face of that cell insulating).
__global__ void recip_kernel(const float* __restrict__ k, float* __restrict__ r, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        r[i] = __fdiv_rn(1.0f, k[i]);
}

}  // namespace wfa

using namespace wfa;

// =============================================================== C ABI ====
extern "C" {

const char* wfa_last_error(void) { return g_last_error.c_str(); }

int wfa_inject_alloc_failure(int n) {
    wfa::g_fail_countdown.store(n < 0 ? -1 : n);
    return WFA_OK;
}

int wfa_create_grid(int nx, int ny, int nz, double hx, double hy, double hz, int storage,
                    void* cuda_stream, wfa_grid* out) {
    if (!out) return fail(WFA_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (nx < 2 || ny < 2 || nz < 2) return fail(WFA_ERR_ARG, "every edge must be >= 2 (got %d %d %d)", nx, ny, nz);
    if (!(hx > 0 && hy > 0 && hz > 0) || !std::isfinite(hx) || !std::isfinite(hy) || !std::isfinite(hz))
        return fail(WFA_ERR_ARG, "cell sizes must be finite and > 0");
    if (storage != WFA_F32 && storage != WFA_BF16) return fail(WFA_ERR_ARG, "storage must be WFA_F32 or WFA_BF16");
    if ((double)nx * ny * nz > (double)(1LL << 40)) return fail(WFA_ERR_ARG, "grid too large");
    // face-wise kernels index a padded face (with its 16 halo layers) in 32 bits
    const double pfx = (double)(nx + 16), pfy = (double)(ny + 16), pfz = (double)(nz + 16);
    if (16.0 * std::max(pfx * pfy, std::max(pfx * pfz, pfy * pfz)) >= 4294967296.0)
        return fail(WFA_ERR_ARG, "a face of %d x %d x %d cells is too large (padded face x 16 must stay below 2^32)",
                    nx, ny, nz);
    wfa_grid_s* g = new (std::nothrow) wfa_grid_s();
    if (!g) return fail(WFA_ERR_OOM, "host allocation failed");
    g->n[0] = nx; g->n[1] = ny; g->n[2] = nz;
    g->h[0] = hx; g->h[1] = hy; g->h[2] = hz;
    g->storage = storage;
    g->esize = storage == WFA_BF16 ? 2 : 4;
    g->stream = (cudaStream_t)cuda_stream;
    const long long align = 128 / g->esize;
    g->px = ((nx + 2LL * HALO + align - 1) / align) * align;
    g->py = ny + 2LL * HALO;
    g->pz = nz + 2LL * HALO;
    for (int f = 0; f < 6; ++f) { g->bc_kind[f] = WFA_BC_ZEROFLUX; g->bc_value[f] = 0.0; }
    const size_t bytes = field_elems(g) * g->esize;
    cudaError_t e = cudaSuccess;
    g->own_T = true;
    g->own_k = true;
    for (int b = 0; b < 2 && e == cudaSuccess; ++b) e = padded_alloc(&g->T[b], bytes, g->esize, g->stream);
    if (e == cudaSuccess) e = dev_alloc((void**)&g->d_partials, 4096 * sizeof(double), g->stream);
    if (e == cudaSuccess) e = dev_alloc((void**)&g->d_status, 8 * sizeof(int), g->stream);
    if (e == cudaSuccess) {
        g->h_result = static_cast<double*>(pinned_word());
        g->h_status = static_cast<int*>(pinned_word());
        if (!g->h_result || !g->h_status) e = cudaErrorMemoryAllocation;
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(g->d_status, 0, 8 * sizeof(int), g->stream);
    if (e == cudaSuccess) {
        for (int b = 0; b < 2 && e == cudaSuccess; ++b) e = cudaMemsetAsync(g->T[b], 0, bytes, g->stream);
    }
    if (e != cudaSuccess) {
        int rc = cuda_fail(e, "wfa_create_grid allocation");
        wfa_destroy_grid(g);
        return rc;
    }
    *out = g;
    return WFA_OK;
}

int wfa_destroy_grid(wfa_grid g) {
    if (!g) return WFA_OK;
    cudaStreamSynchronize(g->stream);   // nothing of this grid is in flight below
    if (g->own_T)
        for (int b = 0; b < 2; ++b) padded_free(g->T[b], g->esize, g->stream);
    if (g->own_k) {
        padded_free(g->k, 4, g->stream);
        padded_free(g->r, 4, g->stream);
    }
    dev_free(g->d_partials, g->stream);
    dev_free(g->d_stage, g->stream);
    dev_free(g->d_status, g->stream);
    pinned_release(g->h_result);
    pinned_release(g->h_status);
    free_tmaps(g);
    free_timing(g);
    free_graphs(g);
    free_cg(g);
    if (g->xev) cudaEventDestroy(g->xev);
    delete g;
    return WFA_OK;
}

static int ensure_stage(wfa_grid g) {
    if (g->d_stage) return WFA_OK;
    const size_t N = (size_t)g->n[0] * g->n[1] * g->n[2];
    WFA_CUDA(dev_alloc((void**)&g->d_stage, N * sizeof(float), g->stream));
    return WFA_OK;
}

static Geo geo_of(const wfa_grid_s* g) {
    Geo geo;
    for (int a = 0; a < 3; ++a) geo.n[a] = g->n[a];
    geo.px = g->px;
    geo.py = g->py;
    return geo;
}

int wfa_set_field(wfa_grid g, const float* host_dense) {
    NvtxRange nvtx_("wfa_set_field");
    if (!g || !host_dense) return fail(WFA_ERR_ARG, "NULL argument");
    const long long N = (long long)g->n[0] * g->n[1] * g->n[2];
    // pinned host memory is read by the packing kernel itself; pageable
    // memory goes through the staging buffer
    const float* src = static_cast<const float*>(host_device_view(host_dense));
    if (!src) {
        int rc = ensure_stage(g);
        if (rc) return rc;
        WFA_CUDA(cudaMemcpyAsync(g->d_stage, host_dense, N * sizeof(float), cudaMemcpyHostToDevice, g->stream));
        src = g->d_stage;
    }
    const int thr = 256;
    const Geo geo = geo_of(g);
    const long long rows = (long long)g->n[1] * g->n[2];
    if (g->storage == WFA_BF16)
        pack_kernel<__nv_bfloat16><<<grid_blocks(rows * 32, thr), thr, 0, g->stream>>>(
            src, (__nv_bfloat16*)g->T[g->cur] + domain_offset(g), geo);
    else
        pack_kernel<float><<<grid_blocks(rows * 32, thr), thr, 0, g->stream>>>(
            src, (float*)g->T[g->cur] + domain_offset(g), geo);
    WFA_CUDA(cudaGetLastError());
    // the host buffer may be reused as soon as we return
    WFA_CUDA(cudaStreamSynchronize(g->stream));
    g->field_set = true;
    g->halo_dirty = true;
    g->steps_done = 0;
    return WFA_OK;
}


int wfa_set_coeffs(wfa_grid g, const float* k_host, double k_uniform, double ux, double uy, double uz) {
    if (!g) return fail(WFA_ERR_ARG, "NULL grid");
    if (!std::isfinite(ux) || !std::isfinite(uy) || !std::isfinite(uz))
        return fail(WFA_ERR_ARG, "velocity must be finite");
    if (!k_host && (!(k_uniform >= 0) || !std::isfinite(k_uniform)))
        return fail(WFA_ERR_ARG, "k_uniform must be finite and >= 0");
    const long long N = (long long)g->n[0] * g->n[1] * g->n[2];
    if (k_host) {
        int rc = ensure_stage(g);
        if (rc) return rc;
        // validate on the device before anything of the grid changes. Pinned
        // host memory is read by the checking kernel itself, which also
        // copies it into the staging buffer (as wfa_set_field reads its
        // input); pageable memory goes through a copy into the staging buffer
        unsigned long long* bad = reinterpret_cast<unsigned long long*>(g->d_partials + 4095);
        WFA_CUDA(cudaMemsetAsync(bad, 0xFF, sizeof(unsigned long long), g->stream));
        const float* kv = static_cast<const float*>(host_device_view(k_host));
        if (kv) {
            check_k_kernel<<<grid_blocks(N, 256), 256, 0, g->stream>>>(kv, N, bad, g->d_stage);
        } else {
            WFA_CUDA(cudaMemcpyAsync(g->d_stage, k_host, N * sizeof(float), cudaMemcpyHostToDevice, g->stream));
            check_k_kernel<<<grid_blocks(N, 256), 256, 0, g->stream>>>(g->d_stage, N, bad);
        }
        WFA_CUDA(cudaGetLastError());
        WFA_CUDA(cudaMemcpyAsync(g->h_result, bad, sizeof(unsigned long long), cudaMemcpyDeviceToHost, g->stream));
        WFA_CUDA(cudaStreamSynchronize(g->stream));
        unsigned long long first;
        memcpy(&first, g->h_result, sizeof first);
        if (first != ~0ull)
            return fail(WFA_ERR_ARG, "k[%llu] = %g is negative or not finite", first, (double)k_host[first]);
        if (!g->k) {
            if (g->ext_k) {   // the caller's buffers (wfa_grid_attach_buffers)
                g->k = g->ext_k;
                g->r = g->ext_r;
                g->own_k = false;
            } else {
                // both or neither: a grid never holds k without 1/k
                float *kb = nullptr, *rb = nullptr;
                WFA_CUDA(padded_alloc((void**)&kb, field_elems(g) * sizeof(float), 4, g->stream));
                const cudaError_t e = padded_alloc((void**)&rb, field_elems(g) * sizeof(float), 4, g->stream);
                if (e != cudaSuccess) {
                    padded_free(kb, 4, g->stream);
                    return cuda_fail(e, "conductivity allocation");
                }
                g->k = kb;
                g->r = rb;
                g->own_k = true;
            }
            WFA_CUDA(cudaMemsetAsync(g->k, 0, field_elems(g) * sizeof(float), g->stream));
        }
        const int thr = 256;
        const long long rows = (long long)g->n[1] * g->n[2];
        pack_kernel<float><<<grid_blocks(rows * 32, thr), thr, 0, g->stream>>>(g->d_stage, g->k + domain_offset(g),
                                                                                geo_of(g));
        WFA_CUDA(cudaGetLastError());
        g->k_halo_dirty = true;   // twins, ghost layers and 1/k follow before the next use
        g->k_uniform = 0.0;
    } else {
        if (g->k) {
            cudaStreamSynchronize(g->stream);
            if (g->own_k) {
                padded_free(g->k, 4, g->stream);
                padded_free(g->r, 4, g->stream);
            }
            g->k = nullptr;
            g->r = nullptr;
            free_tmaps(g);
        }
        g->k_uniform = k_uniform;
    }
    g->u[0] = ux; g->u[1] = uy; g->u[2] = uz;
    g->coeffs_set = true;
    g->dt_set = false;   // the limit may have moved
    g->limit_valid = false;
    g->halo_dirty = true;
    return WFA_OK;
}

int wfa_set_bc(wfa_grid g, int face, int kind, double value) {
    if (!g) return fail(WFA_ERR_ARG, "NULL grid");
    if (face < 0 || face > 5) return fail(WFA_ERR_ARG, "face %d out of range", face);
    if (kind < 0 || kind > WFA_BC_EXCHANGE) return fail(WFA_ERR_ARG, "boundary kind %d out of range", kind);
    if (kind == WFA_BC_EXCHANGE && face < WFA_ZLO)
        return fail(WFA_ERR_BC, "exchange faces are z faces (the grid is split into slabs along z)");
    if (!std::isfinite(value)) return fail(WFA_ERR_ARG, "boundary value must be finite");
    if (kind == WFA_BC_DIRICHLET_CELL && g->n[face / 2] < 3)
        return fail(WFA_ERR_BC, "held boundary cells need an edge >= 3");
    g->bc_kind[face] = kind;
    g->bc_value[face] = value;
    g->halo_dirty = true;
    g->k_halo_dirty = true;
    g->dt_set = false;
    g->limit_valid = false;
    return WFA_OK;
}

static RateSpec rate_spec(const wfa_grid_s* g) {
    RateSpec r;
    memset(&r, 0, sizeof r);
    for (int a = 0; a < 3; ++a) {
        r.n[a] = g->n[a];
        r.inv_h2[a] = 1.0 / (g->h[a] * g->h[a]);
        r.up[a] = (g->u[a] > 0 ? g->u[a] : 0.0) / g->h[a];
        r.um[a] = (g->u[a] < 0 ? -g->u[a] : 0.0) / g->h[a];
    }
    for (int f = 0; f < 6; ++f) {
        r.kind[f] = g->bc_kind[f];
        r.held[f] = g->bc_kind[f] == WFA_BC_DIRICHLET_CELL;
    }
    for (int a = 0; a < 3; ++a) {
        r.inv_h2f[a] = (float)r.inv_h2[a];
        r.upf[a] = (float)r.up[a];
        r.umf[a] = (float)r.um[a];
    }
    r.px = g->px;
    r.py = g->py;
    r.k_uniform = g->k_uniform;
    return r;
}

// The fp32 first pass keeps every product of a k in [1e-15, 1e15] with these
// factors inside the normal fp32 range.
static bool rate32_applies(const RateSpec& r) {
    for (int a = 0; a < 3; ++a) {
        if (!(r.inv_h2[a] >= 1e-15 && r.inv_h2[a] <= 1e15)) return false;
        for (double v : {r.up[a], r.um[a]})
            if (v != 0.0 && !(v >= 1e-30 && v <= 1e30)) return false;
    }
    return true;
}

// Uniform k: D_C depends only on which faces of the cell are boundary faces,
// so the maximum is taken over the (at most 27) cell classes on the host:
// per axis the low end, an interior position (when the edge is >= 3) and the
// high end. The expression is the device's (rate64) term for term.
static double uniform_rate_max(const RateSpec& r) {
    double best = 0.0;
    int pos[3][3], npos[3];
    for (int a = 0; a < 3; ++a) {
        npos[a] = 0;
        pos[a][npos[a]++] = 0;
        if (r.n[a] >= 3) pos[a][npos[a]++] = 1;
        pos[a][npos[a]++] = r.n[a] - 1;
    }
    for (int i = 0; i < npos[0]; ++i)
        for (int j = 0; j < npos[1]; ++j)
            for (int l = 0; l < npos[2]; ++l) {
                const int c[3] = {pos[0][i], pos[1][j], pos[2][l]};
                bool held = false;
                for (int f = 0; f < 6; ++f)
                    if (r.held[f] && c[f >> 1] == ((f & 1) ? r.n[f >> 1] - 1 : 0)) held = true;
                if (held) continue;
                const double kC = r.k_uniform;
                double D = 0.0;
                for (int a = 0; a < 3; ++a)
                    for (int side = 0; side < 2; ++side) {
                        const int f = 2 * a + side;
                        const bool edge = side == 0 ? c[a] == 0 : c[a] == r.n[a] - 1;
                        bool active = true;
                        if (edge && r.kind[f] != WFA_BC_PERIODIC && r.kind[f] != WFA_BC_EXCHANGE) {
                            if (r.kind[f] == WFA_BC_DIRICHLET) D += 2.0 * kC * r.inv_h2[a];
                            else active = false;
                        } else {
                            const double s2 = kC + kC;
                            D += (s2 > 0.0 ? 2.0 * kC * kC / s2 : 0.0) * r.inv_h2[a];
                        }
                        if (active) D += side ? r.up[a] : r.um[a];
                    }
                best = std::max(best, D);
            }
    return best;
}

// k halo (periodic twins), then r = 1/k over the whole padded buffer.
static int prepare_k_halo(wfa_grid g) {
    if (!g->k) return WFA_OK;
    if (!g->k_halo_dirty) return WFA_OK;
    HaloSpec h = halo_spec(g);
    const long long rows = (long long)(g->n[1] + 2 * HALO) * (g->n[2] + 2 * HALO);
    k_halo_kernel<<<grid_blocks(rows * 32, 256), 256, 0, g->stream>>>(g->k, h);
    WFA_CUDA(cudaGetLastError());
    const long long all = (long long)field_elems(g);
    recip_kernel<<<grid_blocks(all, 256), 256, 0, g->stream>>>(g->k, g->r, all);
    WFA_CUDA(cudaGetLastError());
    g->k_halo_dirty = false;
    return WFA_OK;
}

int wfa_stability_dt(wfa_grid g, double* dt_max) {
    NvtxRange nvtx_("wfa_stability_dt");
    if (!g || !dt_max) return fail(WFA_ERR_ARG, "NULL argument");
    if (!g->coeffs_set) return fail(WFA_ERR_STATE, "set the coefficients first");
    for (int a = 0; a < 3; ++a)
        if ((g->bc_kind[2 * a] == WFA_BC_PERIODIC) != (g->bc_kind[2 * a + 1] == WFA_BC_PERIODIC))
            return fail(WFA_ERR_BC, "axis %d: a periodic face needs a periodic opposite face", a);
    if (!g->limit_valid) {
        RateSpec r = rate_spec(g);
        double dmax;
        if (!g->k) {
            dmax = uniform_rate_max(r);
        } else {
            int rc = prepare_k_halo(g);
            if (rc) return rc;
            const float* ko = g->k + domain_offset(g);
            double* part = g->d_partials;
            if (rate32_applies(r)) {
                // partials of pass 1 at [0, RATE_BLOCKS), its maximum at RATE_BLOCKS,
                // partials of pass 2 at [RATE_P2, RATE_P2 + RATE_BLOCKS), the result at RATE_BLOCKS + 1
                rate32_partial_kernel<<<RATE_BLOCKS, RED_THREADS, 0, g->stream>>>(ko, r, part, part + RATE_RISKY);
                finish_max_kernel<<<1, 512, 0, g->stream>>>(part, RATE_BLOCKS, part + RATE_BLOCKS);
                rate_cand_kernel<<<RATE_BLOCKS, RED_THREADS, 0, g->stream>>>(ko, r, part, part + RATE_RISKY,
                                                                             part + RATE_BLOCKS, part + RATE_P2);
                finish_max_kernel<<<1, 512, 0, g->stream>>>(part + RATE_P2, RATE_BLOCKS, part + RATE_BLOCKS + 1);
            } else {
                rate_partial_kernel<<<RATE_BLOCKS, RED_THREADS, 0, g->stream>>>(ko, r, part + RATE_P2);
                finish_max_kernel<<<1, 512, 0, g->stream>>>(part + RATE_P2, RATE_BLOCKS, part + RATE_BLOCKS + 1);
            }
            WFA_CUDA(cudaGetLastError());
            WFA_CUDA(cudaMemcpyAsync(g->h_result, part + RATE_BLOCKS + 1, sizeof(double), cudaMemcpyDeviceToHost,
                                     g->stream));
            WFA_CUDA(cudaStreamSynchronize(g->stream));
            dmax = g->h_result[0];
        }
        g->limit = dmax > 0.0 ? 1.0 / dmax : INFINITY;
        g->limit_valid = true;
    }
    *dt_max = g->limit;
    return WFA_OK;
}

int wfa_set_dt(wfa_grid g, double dt) {
    if (!g) return fail(WFA_ERR_ARG, "NULL grid");
    if (!(dt > 0) || !std::isfinite(dt)) return fail(WFA_ERR_ARG, "dt must be finite and > 0");
    double lim;
    int rc = wfa_stability_dt(g, &lim);
    if (rc) return rc;
    if (dt > lim) return fail(WFA_ERR_UNSTABLE, "dt = %.17g exceeds the stability limit %.17g", dt, lim);
    g->dt = dt;
    g->dt_set = true;
    return WFA_OK;
}

int wfa_set_tuning(wfa_grid g, int depth, int variant) {
    if (!g) return fail(WFA_ERR_ARG, "NULL grid");
    if (depth < 0 || depth > MAX_DEPTH) return fail(WFA_ERR_ARG, "depth must be 0..%d", MAX_DEPTH);
    if (variant < -1 || variant > T2_VARIANT) return fail(WFA_ERR_ARG, "variant must be -1..%d", T2_VARIANT);
    g->force_depth = depth;
    g->force_variant = variant;
    return WFA_OK;
}

int wfa_set_zchunk(wfa_grid g, int planes) {
    if (!g) return fail(WFA_ERR_ARG, "NULL grid");
    if (planes < 0) return fail(WFA_ERR_ARG, "planes must be >= 0");
    g->force_zchunk = planes;
    return WFA_OK;
}

int wfa_step(wfa_grid g, long long n) {
    NvtxRange nvtx_("wfa_step");
    if (!g) return fail(WFA_ERR_ARG, "NULL grid");
    if (n < 0) return fail(WFA_ERR_ARG, "negative step count");
    if (!g->field_set || !g->coeffs_set || !g->dt_set)
        return fail(WFA_ERR_STATE, "set the field, the coefficients and dt before stepping");
    SweepCoef c;
    int rc = build_coef(g, &c);
    if (rc) return rc;
    if (n == 0) return WFA_OK;
    if (g->halo_dirty) {
        rc = refresh_halo(g, g->cur);
        if (rc) return rc;
        rc = prepare_k_halo(g);
        if (rc) return rc;
        g->halo_dirty = false;
    }
    rc = launch_sweep(g, n);
    if (rc) return rc;
    g->steps_done += n;
    return WFA_OK;
}

int wfa_autotune(wfa_grid g, int* depth, int* variant) {
    NvtxRange nvtx_("wfa_autotune");
    if (!g) return fail(WFA_ERR_ARG, "NULL grid");
    if (!g->field_set || !g->coeffs_set || !g->dt_set)
        return fail(WFA_ERR_STATE, "set the field, the coefficients and dt before tuning");
    if (g->halo_dirty) {
        int rc = refresh_halo(g, g->cur);
        if (rc) return rc;
        rc = prepare_k_halo(g);
        if (rc) return rc;
        g->halo_dirty = false;
    }
    return autotune(g, depth, variant);
}

int wfa_steps_done(wfa_grid g, long long* n) {
    if (!g || !n) return fail(WFA_ERR_ARG, "NULL argument");
    *n = g->steps_done;
    return WFA_OK;
}

int wfa_read_field(wfa_grid g, float* host_dense) {
    NvtxRange nvtx_("wfa_read_field");
    if (!g || !host_dense) return fail(WFA_ERR_ARG, "NULL argument");
    if (!g->field_set) return fail(WFA_ERR_STATE, "no field set");
    if (g->halo_dirty) {   // held layers show their value even before the first step
        int rc = refresh_halo(g, g->cur);
        if (rc) return rc;
    }
    const long long N = (long long)g->n[0] * g->n[1] * g->n[2];
    // pinned host memory is written by the unpacking kernel itself; pageable
    // memory is filled from the staging buffer
    float* dst = static_cast<float*>(const_cast<void*>(host_device_view(host_dense)));
    const bool staged = !dst;
    if (staged) {
        int rc = ensure_stage(g);
        if (rc) return rc;
        dst = g->d_stage;
    }
    const int thr = 256;
    const Geo geo = geo_of(g);
    const long long rows = (long long)g->n[1] * g->n[2];
    if (g->storage == WFA_BF16)
        unpack_kernel<__nv_bfloat16><<<grid_blocks(rows * 32, thr), thr, 0, g->stream>>>(
            (const __nv_bfloat16*)g->T[g->cur] + domain_offset(g), dst, geo);
    else
        unpack_kernel<float><<<grid_blocks(rows * 32, thr), thr, 0, g->stream>>>(
            (const float*)g->T[g->cur] + domain_offset(g), dst, geo);
    WFA_CUDA(cudaGetLastError());
    if (staged)
        WFA_CUDA(cudaMemcpyAsync(host_dense, g->d_stage, N * sizeof(float), cudaMemcpyDeviceToHost, g->stream));
    return check_status(g);   // synchronises: the host buffer is complete
}

int wfa_total_heat(wfa_grid g, double* e) {
    NvtxRange nvtx_("wfa_total_heat");
    int rc_;
    if (!g || !e) return fail(WFA_ERR_ARG, "NULL argument");
    if (!g->field_set) return fail(WFA_ERR_STATE, "no field set");
    if (g->halo_dirty) {
        int rc = refresh_halo(g, g->cur);
        if (rc) return rc;
    }
    const Geo geo = geo_of(g);
    if (g->storage == WFA_BF16)
        heat_partial_kernel<__nv_bfloat16><<<RED_BLOCKS, RED_THREADS, 0, g->stream>>>(
            (const __nv_bfloat16*)g->T[g->cur] + domain_offset(g), geo, g->d_partials);
    else
        heat_partial_kernel<float><<<RED_BLOCKS, RED_THREADS, 0, g->stream>>>(
            (const float*)g->T[g->cur] + domain_offset(g), geo, g->d_partials);
    finish_sum_kernel<<<1, 512, 0, g->stream>>>(g->d_partials, RED_BLOCKS, g->h[0] * g->h[1] * g->h[2],
                                                g->d_partials + RED_BLOCKS);
    WFA_CUDA(cudaGetLastError());
    WFA_CUDA(cudaMemcpyAsync(g->h_result, g->d_partials + RED_BLOCKS, sizeof(double), cudaMemcpyDeviceToHost,
                             g->stream));
    rc_ = check_status(g);
    *e = g->h_result[0];
    return rc_;
}

int wfa_boundary_flux(wfa_grid g, double* flux) {
    NvtxRange nvtx_("wfa_boundary_flux");
    if (!g || !flux) return fail(WFA_ERR_ARG, "NULL argument");
    if (!g->field_set || !g->coeffs_set || !g->dt_set)
        return fail(WFA_ERR_STATE, "set the field, the coefficients and dt first");
    for (int f = 0; f < 6; ++f)
        if (g->bc_kind[f] == WFA_BC_DIRICHLET_CELL)
            return fail(WFA_ERR_BC, "held boundary layers are not faces: no face flux to report");
    if (g->halo_dirty) {
        int rc = refresh_halo(g, g->cur);
        if (rc) return rc;
    }
    FluxSpec fs;
    memset(&fs, 0, sizeof fs);
    for (int a = 0; a < 3; ++a) {
        fs.n[a] = g->n[a];
        fs.inv_h2[a] = 1.0 / (g->h[a] * g->h[a]);
        fs.u_h[a] = g->u[a] / g->h[a];
    }
    for (int f = 0; f < 6; ++f) {
        fs.dirichlet[f] = g->bc_kind[f] == WFA_BC_DIRICHLET;
        fs.tb[f] = g->bc_value[f];
    }
    fs.px = g->px;
    fs.py = g->py;
    fs.k_uniform = g->k_uniform;
    // 6 faces x FLUX_BLOCKS partials, then one fixed-order sum (scaled by dt
    // and the cell volume)
    constexpr int FLUX_BLOCKS = 96;
    static_assert(6 * FLUX_BLOCKS + 1 < 4095, "scratch layout");
    const dim3 grid(FLUX_BLOCKS, 6);
    const float* ko = g->k ? g->k + domain_offset(g) : nullptr;
    if (g->storage == WFA_BF16)
        flux_partial_kernel<__nv_bfloat16><<<grid, RED_THREADS, 0, g->stream>>>(
            (const __nv_bfloat16*)g->T[g->cur] + domain_offset(g), ko, fs, g->d_partials);
    else
        flux_partial_kernel<float><<<grid, RED_THREADS, 0, g->stream>>>(
            (const float*)g->T[g->cur] + domain_offset(g), ko, fs, g->d_partials);
    finish_sum_kernel<<<1, 512, 0, g->stream>>>(g->d_partials, 6 * FLUX_BLOCKS,
                                                g->dt * g->h[0] * g->h[1] * g->h[2], g->d_partials + 6 * FLUX_BLOCKS);
    WFA_CUDA(cudaGetLastError());
    WFA_CUDA(cudaMemcpyAsync(g->h_result, g->d_partials + 6 * FLUX_BLOCKS, sizeof(double), cudaMemcpyDeviceToHost,
                             g->stream));
    const int rc = check_status(g);
    *flux = g->h_result[0];
    return rc;
}

int wfa_grid_buffer_bytes(wfa_grid g, size_t* field_bytes, size_t* k_bytes) {
    if (!g || !field_bytes || !k_bytes) return fail(WFA_ERR_ARG, "NULL argument");
    *field_bytes = field_elems(g) * g->esize + LEAD_SLACK;
    *k_bytes = field_elems(g) * sizeof(float) + LEAD_SLACK;
    return WFA_OK;
}

int wfa_grid_attach_buffers(wfa_grid g, void* d_Ta, void* d_Tb, float* d_k, float* d_r) {
    if (!g || !d_Ta || !d_Tb || d_Ta == d_Tb) return fail(WFA_ERR_ARG, "two distinct field buffers are needed");
    if ((d_k == nullptr) != (d_r == nullptr)) return fail(WFA_ERR_ARG, "give both k and 1/k buffers, or neither");
    for (const void* p : {(const void*)d_Ta, (const void*)d_Tb, (const void*)d_k, (const void*)d_r}) {
        if (!p) continue;
        if ((uintptr_t)p % 256) return fail(WFA_ERR_ARG, "attached buffers must be 256-byte aligned");
        cudaPointerAttributes at;
        if (cudaPointerGetAttributes(&at, p) != cudaSuccess || at.type != cudaMemoryTypeDevice) {
            cudaGetLastError();
            return fail(WFA_ERR_ARG, "attached buffers must be device memory");
        }
    }
    const size_t fb = field_elems(g) * g->esize, kb = field_elems(g) * sizeof(float);
    // the padded arrays start lead_bytes() into the caller's buffers, as in the grid's own
    char* ta = (char*)d_Ta + lead_bytes(g->esize);
    char* tb = (char*)d_Tb + lead_bytes(g->esize);
    float* ka = d_k ? (float*)((char*)d_k + lead_bytes(4)) : nullptr;
    float* ra = d_r ? (float*)((char*)d_r + lead_bytes(4)) : nullptr;
    // the grid's current contents move into the caller's buffers
    WFA_CUDA(cudaMemcpyAsync(ta, g->T[0], fb, cudaMemcpyDeviceToDevice, g->stream));
    WFA_CUDA(cudaMemcpyAsync(tb, g->T[1], fb, cudaMemcpyDeviceToDevice, g->stream));
    if (d_k && g->k) {
        WFA_CUDA(cudaMemcpyAsync(ka, g->k, kb, cudaMemcpyDeviceToDevice, g->stream));
        WFA_CUDA(cudaMemcpyAsync(ra, g->r, kb, cudaMemcpyDeviceToDevice, g->stream));
    }
    WFA_CUDA(cudaStreamSynchronize(g->stream));
    if (g->own_T)
        for (int b = 0; b < 2; ++b) padded_free(g->T[b], g->esize, g->stream);
    g->T[0] = ta;
    g->T[1] = tb;
    g->own_T = false;
    if (d_k) {
        if (g->k) {
            if (g->own_k) {
                padded_free(g->k, 4, g->stream);
                padded_free(g->r, 4, g->stream);
            }
            g->k = ka;
            g->r = ra;
            g->own_k = false;
        }
        g->ext_k = ka;
        g->ext_r = ra;
    }
    free_tmaps(g);   // descriptors name the old buffers
    return WFA_OK;
}

int wfa_sync(wfa_grid g) {
    if (!g) return fail(WFA_ERR_ARG, "NULL grid");
    return check_status(g);
}

}  // extern "C"

namespace wfa {
int prepare_coeff_halo(wfa_grid_s* g) { return prepare_k_halo(g); }

// Hand a grid to another stream: its own work is finished first, and later
// work goes to the new stream (device memory is not tied to a stream once
// allocated).
int grid_rebind_stream(wfa_grid_s* g, cudaStream_t st) {
    WFA_CUDA(cudaStreamSynchronize(g->stream));
    g->stream = st;
    return WFA_OK;
}

// As grid_rebind_stream, for a caller that knows no work of g is pending on
// its stream (it has waited for an event behind the last of it).
int grid_move_stream(wfa_grid_s* g, cudaStream_t st) {
    g->stream = st;
    return WFA_OK;
}
}  // namespace wfa
