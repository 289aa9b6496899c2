// Implicit (backward-Euler) time steps solved by classic conjugate gradients
// (Sec. 1.1.2, Eq. impl_form), in the same face-flux form as the explicit
// sweep, diffusion only (with advection the system is not symmetric and CG
// does not apply).
//
// One step solves, for every cell that is not held,
//   T'_C + sum_f c_f (T'_C - T'_D) + sum_{Dirichlet faces} d_f (T'_C - Tb_f) = T_C
// with c_f = dt K_f / h_a^2 (K_f the harmonic-mean face conductivity) and
// d_f = 2 dt k_C / h_a^2; held cells keep their value. Moving the known
// values (Dirichlet faces, held neighbours) to the right-hand side leaves a
// symmetric positive definite system A y = b on the free cells, solved from
// y = T by classic CG with its two inner products per iteration:
//
//   q = A p,  alpha = r.r / p.q,  x += alpha p,  r -= alpha q,
//   beta = r.r' / r.r,  p = r + beta p
//
// GB300 mapping. The field x is the grid's fp32 buffer, updated in place;
// r, p (two buffers) and q are fp32 work vectors in the same padded layout.
// Each iteration is two HBM-bound kernels:
//   cg_spmv   p = r + beta p_old on the fly (for the cell and its six
//             neighbours), q = A p, and the block partials of p.q; reads r and
//             p_old, writes p and q (16 B a cell, + 4 B of 1/k for per-cell k);
//   cg_update x += alpha p, r -= alpha q, and the block partials of r.r
//             (reads x, p, q, r, writes x, r: 24 B a cell).
// The last block of each kernel to finish (an atomic ticket, no waiting) sums
// the partials in a fixed order and computes alpha (resp. beta and the
// convergence test) on the device, so no host round trip sits between
// iterations: a whole call is one graph launch whose conditional WHILE nodes
// loop over the time steps and the iterations (device loops, below); where
// those cannot be built, captured runs of iterations are replayed with the
// host reading the convergence flag between runs, one run ahead.
// Periodic axes read the neighbour across the boundary from a twin copy
// that every writer of a boundary cell also stores one cell beyond the
// opposite face; non-periodic boundary faces take a ghost value that makes
// the interior expression exact, only in warps that hold a boundary cell.
// cg_pipe is the pipelined alternative (Chronopoulos and Gear): one kernel
// and one reduction an iteration.
// Inner products: fp32 products summed per plane, a compensated fp32 sum over
// a thread's planes, fp64 above that (the block, the fixed-order sum over
// blocks); the GPU's fp64 rate is low, so no fp64 arithmetic sits in the
// hot loops.
#include <type_traits>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <new>

#include "wfa_internal.cuh"

namespace wfa {

constexpr int CG_TX = 16, CG_TY = 16;   // cg_spmv block: 64 x 16 cells, 4 x cells a thread
constexpr int CG_THREADS = 256;
constexpr int CG_MAX_PART = 16384;      // per-block partials of one launch
constexpr bool CG_SPMV_SM_DEFAULT = false;   // cg_spmv (L1 neighbours) unless WFA_CG_SPMV=sm
constexpr int CG_NRUN = 4;              // captured runs of 1, 2, 4 and 8 iterations
constexpr int CG_RUN_LEN[CG_NRUN] = {1, 2, 4, 8};

// Solver scalars on the device (56 bytes; read back as one block).
struct CgState {   // fits one 64-byte pinned word
    double rr;        // r.r of the current residual
    double bb;        // b.b of the step's right-hand side
    double alpha, beta;
    double tol2;      // rtol^2
    int done;         // converged, iteration limit reached, or breakdown
    int iter;         // iterations of the current step
    int max_iter;
    unsigned ticket;  // blocks of the current launch that have finished
};

static_assert(sizeof(CgState) <= 64, "CgState is read back into a 64-byte pinned word");

struct CgCoef {
    int n[3];
    int periodic[3];
    int dface[6];     // face carries a Dirichlet value (on the face)
    int held[6];      // face holds its outer cell layer
    long long sy, sz; // element strides of the padded layout
    float tb[6];      // Dirichlet face values
    float cu[3];      // uniform k: dt k / h_a^2
    float du;         // uniform k: 1 + 2 (cu[0] + cu[1] + cu[2]), an interior row's diagonal
    float tcd[3];     // per-cell k: 2 dt / h_a^2 (c_f = tcd / (1/k_C + 1/k_D))
};

struct CgArgs {
    CgCoef c;
    float* x;          // domain origins (cell (0,0,0)) of the padded arrays
    const float* rk;   // 1/k, or nullptr for uniform k
    float* r;
    float* p0;
    float* p1;
    float* q;
    double* part;      // per-block partials (two arrays of CG_MAX_PART for cg_init)
    CgState* s;
    float* r2;         // pipelined CG: second r, w and s buffers (r, w and s ping-pong, read at
    float* w2;         // neighbours: r in r / r2, w in q / w2, s in p1 / s2; p in p0)
    float* s2;
    int zchunk;        // cg_spmv planes per block
    int nblk;          // blocks of this launch
    int q_twins;       // cg_spmv also writes q's periodic twins (q is the pipelined solver's first w)
};

__device__ __forceinline__ long long cg_at(const CgCoef& c, int x, int y, int z) {
    return x + (long long)y * c.sy + (long long)z * c.sz;
}

__device__ __forceinline__ bool cg_held(const CgCoef& c, int x, int y, int z) {
    return (c.held[0] && x == 0) || (c.held[1] && x == c.n[0] - 1) || (c.held[2] && y == 0) ||
           (c.held[3] && y == c.n[1] - 1) || (c.held[4] && z == 0) || (c.held[5] && z == c.n[2] - 1);
}
// The same over the faces of mask FM (bit f: face f); the caller knows that
// the cell is on no face outside FM.
template <int FM>
__device__ __forceinline__ bool cg_held_m(const CgCoef& c, int x, int y, int z) {
    return ((FM & 1) && c.held[0] && x == 0) || ((FM & 2) && c.held[1] && x == c.n[0] - 1) ||
           ((FM & 4) && c.held[2] && y == 0) || ((FM & 8) && c.held[3] && y == c.n[1] - 1) ||
           ((FM & 16) && c.held[4] && z == 0) || ((FM & 32) && c.held[5] && z == c.n[2] - 1);
}

__device__ __forceinline__ void prefetch_l2(const void* p) {
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

__device__ __forceinline__ void sts4(float* p, const float v[4]) {
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
__device__ __forceinline__ void lds4(const float* p, float v[4]) {
    const float4 t = *reinterpret_cast<const float4*>(p);
    v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
}

__device__ __forceinline__ void ld4(const float* p, float v[4]) {
    const float4 t = __ldg(reinterpret_cast<const float4*>(p));
    v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
}

// Store 4 cells of row (gx.., y, z), the ones inside the domain, plus the
// periodic twins of those on a periodic face.
__device__ __forceinline__ void st4_row(float* o, int gx, int nx, const float v[4]) {
    if (gx + 3 < nx) {
        *reinterpret_cast<float4*>(o) = make_float4(v[0], v[1], v[2], v[3]);
    } else {
#pragma unroll
        for (int i = 0; i < 4; ++i)
            if (gx + i < nx) o[i] = v[i];
    }
}

__device__ __forceinline__ void st4_twins(float* base, const CgCoef& c, int gx, int y, int z, const float v[4]) {
    const int nx = c.n[0];
    st4_row(base + cg_at(c, gx, y, z), gx, nx, v);
    if (c.periodic[1] && (y == 0 || y == c.n[1] - 1)) st4_row(base + cg_at(c, gx, y == 0 ? c.n[1] : -1, z), gx, nx, v);
    if (c.periodic[2] && (z == 0 || z == c.n[2] - 1)) st4_row(base + cg_at(c, gx, y, z == 0 ? c.n[2] : -1), gx, nx, v);
    if (c.periodic[0]) {
        if (gx == 0) base[cg_at(c, nx, y, z)] = v[0];
#pragma unroll
        for (int i = 0; i < 4; ++i)
            if (gx + i == nx - 1) base[cg_at(c, -1, y, z)] = v[i];
    }
}

// Compensated (Kahan) fp32 running sum: a thread's share of an inner product
// without per-plane fp64 arithmetic (the GPU's fp64 rate is a small fraction
// of its fp32 rate); the block and the blocks are then summed in fp64.
struct KahanF {
    float s = 0.0f, c = 0.0f;
    __device__ __forceinline__ void add(float v) {
        const float y = __fsub_rn(v, c);
        const float t = __fadd_rn(s, y);
        c = __fsub_rn(__fsub_rn(t, s), y);
        s = t;
    }
    __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};

// Block sum of one double per thread (fixed shuffle tree, then the warps in
// order); the result is valid in thread 0.
__device__ __forceinline__ double block_sum(double v, double* red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int tid = threadIdx.x + threadIdx.y * blockDim.x;
    const int nw = (blockDim.x * blockDim.y + 31) / 32;
    if ((tid & 31) == 0) red[tid >> 5] = v;
    __syncthreads();
    double t = 0.0;
    if (tid == 0)
        for (int w = 0; w < nw; ++w) t += red[w];
    __syncthreads();
    return t;
}

// Publish this block's partial; true in every thread of the last block of
// the launch to do so (which then owns the finish and resets the ticket).
__device__ __forceinline__ bool publish(const CgArgs& a, double* slot, double v, bool* last) {
    const int tid = threadIdx.x + threadIdx.y * blockDim.x;
    if (tid == 0) {
        *slot = v;
        __threadfence();
        const unsigned t = atomicAdd(&a.s->ticket, 1u);
        *last = t == (unsigned)a.nblk - 1;
    }
    __syncthreads();
    return *last;
}

// Fixed-order sum of n partials by the whole block; valid in thread 0.
__device__ __forceinline__ double sum_partials(const double* part, int n, double* red) {
    const int tid = threadIdx.x + threadIdx.y * blockDim.x;
    const int nt = blockDim.x * blockDim.y;
    __threadfence();
    double t = 0.0;
    for (int i = tid; i < n; i += nt) t += __ldcg(part + i);
    return block_sum(t, red);
}

template <bool KVAR>
struct CgOcc {
    static constexpr int blocks = KVAR ? 3 : 4;
};

// Boundary faces a thread's cells touch (non-periodic axes only). A face is
// taken as a ghost neighbour that makes the interior formula exact: across a
// Dirichlet face (value 0 in A) p_ghost = -p_C, across a zero-flux face
// p_ghost = p_C, with the ghost's conductivity that of the cell (so the face
// coefficient is tcd / (2 r_C): twice it is the Dirichlet coefficient
// 2 k_C dt / h^2). Held cells are masked (q = 0).
struct CgEdge {
    int ih;            // index 0..3 of the thread's cell on the +x face (4: none)
    unsigned bits;     // 1: cell 0 on the -x face, 2: the row on the -y face, 4: on the +y face
};

__device__ __forceinline__ CgEdge cg_edge(const CgCoef& c, int gx, int gy) {
    CgEdge e;
    const int nx = c.n[0], ny = c.n[1];
    e.ih = (!c.periodic[0] && gx <= nx - 1 && nx - 1 - gx < 4) ? nx - 1 - gx : 4;
    e.bits = ((!c.periodic[0] && gx == 0) ? 1u : 0u) | ((!c.periodic[1] && gy == 0) ? 2u : 0u) |
             ((!c.periodic[1] && gy == ny - 1) ? 4u : 0u);
    return e;
}

// ghost value across face f of a cell holding v: -v (Dirichlet face) or v
__device__ __forceinline__ float ghost(const CgCoef& c, int f, float v) { return c.dface[f] ? -v : v; }

// r = dt acc(T) and the b terms of the 4 cells of a thread at plane z. EDGE
// (warp-uniform) puts ghost values across boundary faces (2 Tb - T_C across a
// Dirichlet face, T_C across a zero-flux face, the cell's own 1/k), adds the
// known values to b (Dirichlet faces: d_f Tb; held neighbours: c_f T_D) and
// masks held cells and cells beyond the x end; without it every neighbour
// is a free cell inside the domain or across a periodic face. FM: the faces
// (bit f: face f) whose boundary or held layer may be near the warp's cells
// (x faces only for warps away from the y and z faces); the others are not
// looked at.
template <bool KVAR, bool EDGE, int FM = 63>
__device__ __forceinline__ void cg_r4(const CgCoef& c, const CgEdge& e, int gx, int gy, int z, const float tc[4],
                                      const float tm[4], const float tp[4], const float ym[4], const float yp[4],
                                      float xm, float xp, const float kc[4], const float km[4], const float kp[4],
                                      const float kym[4], const float kyp[4], float kxm, float kxp, float rv[4],
                                      float& sr, float& sb) {
    const int nx = c.n[0], ny = c.n[1], nz = c.n[2];
    const bool zlo = EDGE && (FM & 16) && !c.periodic[2] && z == 0,
               zhi = EDGE && (FM & 32) && !c.periodic[2] && z == nz - 1;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        float t[6] = {i == 0 ? xm : tc[i - 1], i == 3 ? xp : tc[i + 1], ym[i], yp[i], tm[i], tp[i]};
        float k[6] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
        if (KVAR) {
            k[0] = i == 0 ? kxm : kc[i - 1];
            k[1] = i == 3 ? kxp : kc[i + 1];
            k[2] = kym[i];
            k[3] = kyp[i];
            k[4] = km[i];
            k[5] = kp[i];
        }
        float bs = tc[i];
        if (EDGE) {
            const int xi = gx + i;
            const bool bd[6] = {(FM & 1) && i == 0 && (e.bits & 1u) != 0, (FM & 2) && i == e.ih,
                                (FM & 4) && (e.bits & 2u) != 0, (FM & 8) && (e.bits & 4u) != 0, zlo, zhi};
            // a neighbour inside the domain is held only through its own axis's face
            const bool hn[6] = {(FM & 1) && c.held[0] && xi == 1, (FM & 2) && c.held[1] && xi == nx - 2,
                                (FM & 4) && c.held[2] && gy == 1, (FM & 8) && c.held[3] && gy == ny - 2,
                                (FM & 16) && c.held[4] && z == 1, (FM & 32) && c.held[5] && z == nz - 2};
#pragma unroll
            for (int f = 0; f < 6; ++f) {
                if (!((FM >> f) & 1)) continue;
                const float cf = KVAR ? face_r(kc[i], bd[f] ? kc[i] : k[f], c.tcd[f >> 1]) : c.cu[f >> 1];
                if (hn[f]) bs = __fmaf_rn(cf, t[f], bs);
                if (bd[f]) {
                    if (c.dface[f]) bs = __fmaf_rn(__fmul_rn(2.0f, cf), c.tb[f], bs);
                    t[f] = c.dface[f] ? __fsub_rn(__fmul_rn(2.0f, c.tb[f]), tc[i]) : tc[i];
                    k[f] = kc[i];
                }
            }
        }
        float acc;
        if (KVAR) {
            acc = __fmul_rn(face_r(kc[i], k[0], c.tcd[0]), __fsub_rn(t[0], tc[i]));
            acc = __fmaf_rn(face_r(kc[i], k[1], c.tcd[0]), __fsub_rn(t[1], tc[i]), acc);
            acc = __fmaf_rn(face_r(kc[i], k[2], c.tcd[1]), __fsub_rn(t[2], tc[i]), acc);
            acc = __fmaf_rn(face_r(kc[i], k[3], c.tcd[1]), __fsub_rn(t[3], tc[i]), acc);
            acc = __fmaf_rn(face_r(kc[i], k[4], c.tcd[2]), __fsub_rn(t[4], tc[i]), acc);
            acc = __fmaf_rn(face_r(kc[i], k[5], c.tcd[2]), __fsub_rn(t[5], tc[i]), acc);
        } else {
            acc = __fmul_rn(c.cu[0], __fadd_rn(__fsub_rn(t[0], tc[i]), __fsub_rn(t[1], tc[i])));
            acc = __fmaf_rn(c.cu[1], __fadd_rn(__fsub_rn(t[2], tc[i]), __fsub_rn(t[3], tc[i])), acc);
            acc = __fmaf_rn(c.cu[2], __fadd_rn(__fsub_rn(t[4], tc[i]), __fsub_rn(t[5], tc[i])), acc);
        }
        if (EDGE) {
            const bool isfree = gx + i < nx && gy < ny && !cg_held_m<FM>(c, gx + i, gy, z);
            rv[i] = isfree ? acc : 0.0f;
            sr = __fmaf_rn(rv[i], rv[i], sr);
            if (isfree) sb = __fmaf_rn(bs, bs, sb);
        } else {
            rv[i] = acc;
            sr = __fmaf_rn(acc, acc, sr);
            sb = __fmaf_rn(bs, bs, sb);
        }
    }
}

// ---------------------------------------------------------------- cg_init --
// r = b - A T (dt times the explicit step's accumulation), b.b and r.r, on
// the column-march layout of cg_spmv (4 x cells a thread, z queue). The
// field's periodic twins are current (refresh_halo before the first step,
// cg_update after every iteration). b adds to T the known values: Dirichlet
// faces and held neighbours. O32: every array is under 4 GiB, so the loop
// addresses its planes by a 32-bit byte offset from the array's start (one
// integer add an address); otherwise by a 64-bit one.
template <bool KVAR, bool O32>
__global__ void __launch_bounds__(CG_TX * CG_TY, CgOcc<KVAR>::blocks) cg_init(const __grid_constant__ CgArgs a, double tol2,
                                                                         int max_iter) {
    __shared__ double red[CG_TX * CG_TY / 32];
    __shared__ bool last;
    const CgCoef& c = a.c;
    const float* __restrict__ xv = a.x;
    const float* __restrict__ rk = a.rk;
    const int nx = c.n[0], ny = c.n[1], nz = c.n[2];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int gx = blockIdx.x * 64 + 4 * tx, gy = blockIdx.y * CG_TY + ty;
    const int z0 = blockIdx.z * a.zchunk, z1 = min(z0 + a.zchunk, nz);
    const bool perx = c.periodic[0], pery = c.periodic[1], perz = c.periodic[2];
    KahanF rr, bb;
    if (gx < nx && gy < ny) {
        const long long sy = c.sy, sz = c.sz;
        const long long row = cg_at(c, gx, gy, 0);
        // fast cells: no boundary face and no held neighbour (two cells from
        // every non-periodic face); inner_y: the same along y only
        const bool inner_y = pery || (gy > 1 && gy < ny - 2);
        const bool inner_xy = gx + 3 < nx && (perx || (gx > 1 && gx + 5 < nx)) && inner_y;
        const CgEdge edge = cg_edge(c, gx, gy);
        float tm[4], tc[4], km[4], kc[4];
        ld4(xv + row + (long long)(z0 - 1) * sz, tm);
        ld4(xv + row + (long long)z0 * sz, tc);
        if (KVAR) {
            ld4(rk + row + (long long)(z0 - 1) * sz, km);
            ld4(rk + row + (long long)z0 * sz, kc);
        }
        using OT = typename std::conditional<O32, unsigned, unsigned long long>::type;
        const long long org = HALO * sz + HALO * sy + HALO;   // elements before the domain origin
        const char* const xB = reinterpret_cast<const char*>(xv - org);
        const char* const kB = KVAR ? reinterpret_cast<const char*>(rk - org) : nullptr;
        char* const rB = reinterpret_cast<char*>(a.r - org);
        auto F = [](const char* b, OT o) { return reinterpret_cast<const float*>(b + o); };
        OT o = (OT)((org + row + (long long)z0 * sz) * 4);   // plane z, this thread's first cell
        const OT dz = (OT)(sz * 4), dy = (OT)(sy * 4);
        const bool twins = perx || pery || perz;
        for (int z = z0; z < z1; ++z) {
            if ((tx & 7) == 0) prefetch_l2(F(xB, o + 3 * dz));
            float tp[4], ym[4], yp[4];
            ld4(F(xB, o + dz), tp);
            ld4(F(xB, o - dy), ym);
            ld4(F(xB, o + dy), yp);
            const float xm = __ldg(F(xB, o - 4u)), xp = __ldg(F(xB, o + 16u));
            float kp[4], kym[4], kyp[4], kxm = 0.0f, kxp = 0.0f;
            if (KVAR) {
                ld4(F(kB, o + dz), kp);
                ld4(F(kB, o - dy), kym);
                ld4(F(kB, o + dy), kyp);
                kxm = __ldg(F(kB, o - 4u));
                kxp = __ldg(F(kB, o + 16u));
            }
            float rv[4];
            float sr = 0.0f, sb = 0.0f;
            const bool inner_z = perz || (z > 1 && z < nz - 2);
            const bool fast = inner_xy && inner_z;
            const unsigned am = __activemask();
            if (__all_sync(am, fast))   // warp-uniform choice, as in cg_spmv
                cg_r4<KVAR, false>(c, edge, gx, gy, z, tc, tm, tp, ym, yp, xm, xp, kc, km, kp, kym, kyp, kxm, kxp, rv,
                                   sr, sb);
            else if (__all_sync(am, inner_y && inner_z))   // near an x face only
                cg_r4<KVAR, true, 3>(c, edge, gx, gy, z, tc, tm, tp, ym, yp, xm, xp, kc, km, kp, kym, kyp, kxm, kxp,
                                     rv, sr, sb);
            else
                cg_r4<KVAR, true>(c, edge, gx, gy, z, tc, tm, tp, ym, yp, xm, xp, kc, km, kp, kym, kyp, kxm, kxp, rv,
                                  sr, sb);
            if (twins)   // the same for every thread
                st4_twins(a.r, c, gx, gy, z, rv);
            else
                st4_row(reinterpret_cast<float*>(rB + o), gx, nx, rv);
            rr.add(sr);
            bb.add(sb);
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                tm[i] = tc[i];
                tc[i] = tp[i];
                if (KVAR) {
                    km[i] = kc[i];
                    kc[i] = kp[i];
                }
            }
            o += dz;
        }
    }
    const int blk = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
    const double rs = block_sum(rr.value(), red);
    const double bsum = block_sum(bb.value(), red);
    if (threadIdx.x == 0 && threadIdx.y == 0) a.part[CG_MAX_PART + blk] = bsum;
    if (!publish(a, a.part + blk, rs, &last)) return;
    const double R = sum_partials(a.part, a.nblk, red);
    const double B = sum_partials(a.part + CG_MAX_PART, a.nblk, red);
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        CgState* s = a.s;
        s->rr = R;
        s->bb = B;
        s->alpha = 0.0;
        s->beta = 0.0;
        s->tol2 = tol2;
        s->iter = 0;
        s->max_iter = max_iter;
        s->done = (R <= tol2 * B || max_iter <= 0 || !(R == R)) ? 1 : 0;
        s->ticket = 0;
    }
}

// ---------------------------------------------------------------- cg_spmv --
// p(this iteration) = r + beta p(previous), formed for each cell where it is
// read, so p is never re-read from DRAM after being written; q = A p.
struct PNew {
    const float* r;
    const float* po;
    float beta;
    bool first;   // first iteration: p = r
};

__device__ __forceinline__ void pnew4(const PNew& P, long long o, float v[4]) {
    ld4(P.r + o, v);
    if (!P.first) {
        float w[4];
        ld4(P.po + o, w);
#pragma unroll
        for (int i = 0; i < 4; ++i) v[i] = __fmaf_rn(P.beta, w[i], v[i]);
    }
}
__device__ __forceinline__ float pnew1(const PNew& P, long long o) {
    const float v = __ldg(P.r + o);
    return P.first ? v : __fmaf_rn(P.beta, __ldg(P.po + o), v);
}

// q = A p for the 4 cells of a thread at plane z, and their p.q (cells inside
// the domain). EDGE (chosen warp-uniformly) puts ghost values across
// boundary faces and masks held cells and cells beyond the x end; without
// it every neighbour is inside the domain or across a periodic face. Both
// evaluate the same expression, so an interior cell gets the same bits
// either way. FM: the faces that may be near the warp's cells (see cg_r4).
template <bool KVAR, bool EDGE, int FM = 63>
__device__ __forceinline__ float cg_q4(const CgCoef& c, const CgEdge& e, int gx, int gy, int z, const float pc[4],
                                       const float pm[4], const float pp[4], const float ym[4], const float yp[4],
                                       float xm, float xp, const float kc[4], const float km[4], const float kp[4],
                                       const float kym[4], const float kyp[4], float kxm, float kxp, float q[4]) {
    float psum = 0.0f;
    const bool zlo = EDGE && (FM & 16) && !c.periodic[2] && z == 0,
               zhi = EDGE && (FM & 32) && !c.periodic[2] && z == c.n[2] - 1;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        float pw = i == 0 ? xm : pc[i - 1], pe = i == 3 ? xp : pc[i + 1];
        float y0 = ym[i], y1 = yp[i], z0 = pm[i], z1 = pp[i];
        float kw = 0.0f, ke = 0.0f, ky0 = 0.0f, ky1 = 0.0f, kz0 = 0.0f, kz1 = 0.0f;
        if (KVAR) {
            kw = i == 0 ? kxm : kc[i - 1];
            ke = i == 3 ? kxp : kc[i + 1];
            ky0 = kym[i];
            ky1 = kyp[i];
            kz0 = km[i];
            kz1 = kp[i];
        }
        if (EDGE) {
            if ((FM & 1) && i == 0 && (e.bits & 1u)) { pw = ghost(c, 0, pc[i]); kw = kc[i]; }
            if ((FM & 2) && i == e.ih) { pe = ghost(c, 1, pc[i]); ke = kc[i]; }
            if ((FM & 4) && (e.bits & 2u)) { y0 = ghost(c, 2, pc[i]); ky0 = kc[i]; }
            if ((FM & 8) && (e.bits & 4u)) { y1 = ghost(c, 3, pc[i]); ky1 = kc[i]; }
            if (zlo) { z0 = ghost(c, 4, pc[i]); kz0 = kc[i]; }
            if (zhi) { z1 = ghost(c, 5, pc[i]); kz1 = kc[i]; }
        }
        float qi;
        if (KVAR) {
            const float r0 = kc[i];
            float acc = __fmul_rn(face_r(r0, kw, c.tcd[0]), __fsub_rn(pc[i], pw));
            acc = __fmaf_rn(face_r(r0, ke, c.tcd[0]), __fsub_rn(pc[i], pe), acc);
            acc = __fmaf_rn(face_r(r0, ky0, c.tcd[1]), __fsub_rn(pc[i], y0), acc);
            acc = __fmaf_rn(face_r(r0, ky1, c.tcd[1]), __fsub_rn(pc[i], y1), acc);
            acc = __fmaf_rn(face_r(r0, kz0, c.tcd[2]), __fsub_rn(pc[i], z0), acc);
            acc = __fmaf_rn(face_r(r0, kz1, c.tcd[2]), __fsub_rn(pc[i], z1), acc);
            qi = __fadd_rn(pc[i], acc);
        } else {
            float acc = __fmul_rn(c.du, pc[i]);
            acc = __fmaf_rn(-c.cu[0], __fadd_rn(pw, pe), acc);
            acc = __fmaf_rn(-c.cu[1], __fadd_rn(y0, y1), acc);
            qi = __fmaf_rn(-c.cu[2], __fadd_rn(z0, z1), acc);
        }
        if (EDGE) {
            const bool isfree = gx + i < c.n[0] && gy < c.n[1] && !cg_held_m<FM>(c, gx + i, gy, z);
            qi = isfree ? qi : 0.0f;
            psum = isfree ? __fmaf_rn(pc[i], qi, psum) : psum;
        } else {
            psum = __fmaf_rn(pc[i], qi, psum);
        }
        q[i] = qi;
    }
    return psum;
}

template <bool KVAR>
__global__ void __launch_bounds__(CG_TX * CG_TY, CgOcc<KVAR>::blocks) cg_spmv(const __grid_constant__ CgArgs a) {
    __shared__ double red[CG_TX * CG_TY / 32];
    __shared__ bool last;
    const CgCoef& c = a.c;
    if (a.s->done) return;
    const int par = a.s->iter & 1;   // iteration i reads p[i mod 2], writes p[(i + 1) mod 2]
    PNew P;
    P.r = a.r;
    P.po = par ? a.p1 : a.p0;
    P.beta = (float)a.s->beta;
    P.first = a.s->iter == 0;
    float* __restrict__ pn = par ? a.p0 : a.p1;
    float* __restrict__ qv = a.q;
    const float* __restrict__ rk = a.rk;
    const int nx = c.n[0], ny = c.n[1], nz = c.n[2];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int gx = blockIdx.x * 64 + 4 * tx, gy = blockIdx.y * CG_TY + ty;
    const int z0 = blockIdx.z * a.zchunk, z1 = min(z0 + a.zchunk, nz);
    const bool perx = c.periodic[0], pery = c.periodic[1], perz = c.periodic[2];
    KahanF dot;
    if (gx < nx && gy < ny) {
        const long long sy = c.sy, sz = c.sz;
        const long long row = cg_at(c, gx, gy, 0);
        const bool inner_y = pery || (gy > 0 && gy < ny - 1);
        const bool inner_xy = gx + 3 < nx && (perx || (gx > 0 && gx + 4 < nx)) && inner_y;
        const CgEdge edge = cg_edge(c, gx, gy);
        float pm[4], pc[4], km[4], kc[4];
        pnew4(P, row + (long long)(z0 - 1) * sz, pm);
        pnew4(P, row + (long long)z0 * sz, pc);
        if (KVAR) {
            ld4(rk + row + (long long)(z0 - 1) * sz, km);
            ld4(rk + row + (long long)z0 * sz, kc);
        }
        for (int z = z0; z < z1; ++z) {
            const long long o = row + (long long)z * sz;
            if ((tx & 7) == 0) {   // one thread per 128-byte line asks L2 for plane z + 3
                prefetch_l2(P.r + o + 3 * sz);
                if (!P.first) prefetch_l2(P.po + o + 3 * sz);
            }
            float pp[4], ym[4], yp[4];
            pnew4(P, o + sz, pp);
            pnew4(P, o - sy, ym);
            pnew4(P, o + sy, yp);
            const float xm = pnew1(P, o - 1), xp = pnew1(P, o + 4);
            float kp[4], kym[4], kyp[4], kxm = 0.0f, kxp = 0.0f;
            if (KVAR) {
                ld4(rk + o + sz, kp);
                ld4(rk + o - sy, kym);
                ld4(rk + o + sy, kyp);
                kxm = __ldg(rk + o - 1);
                kxp = __ldg(rk + o + 4);
            }
            float q[4];
            const bool inner_z = perz || (z > 0 && z < nz - 1);
            const bool fast = inner_xy && inner_z;
            const unsigned am = __activemask();
            const float psum =
                __all_sync(am, fast)
                    ? cg_q4<KVAR, false>(c, edge, gx, gy, z, pc, pm, pp, ym, yp, xm, xp, kc, km, kp, kym, kyp, kxm, kxp,
                                         q)
                : __all_sync(am, inner_y && inner_z)   // near an x face only
                    ? cg_q4<KVAR, true, 3>(c, edge, gx, gy, z, pc, pm, pp, ym, yp, xm, xp, kc, km, kp, kym, kyp, kxm,
                                           kxp, q)
                    : cg_q4<KVAR, true>(c, edge, gx, gy, z, pc, pm, pp, ym, yp, xm, xp, kc, km, kp, kym, kyp, kxm, kxp,
                                        q);
            dot.add(psum);
            st4_twins(pn, c, gx, gy, z, pc);
            if (a.q_twins) {
                st4_twins(qv, c, gx, gy, z, q);
            } else if (gx + 3 < nx) {
                *reinterpret_cast<float4*>(qv + o) = make_float4(q[0], q[1], q[2], q[3]);
            } else {
#pragma unroll
                for (int i = 0; i < 4; ++i)
                    if (gx + i < nx) qv[o + i] = q[i];
            }
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                pm[i] = pc[i];
                pc[i] = pp[i];
                if (KVAR) {
                    km[i] = kc[i];
                    kc[i] = kp[i];
                }
            }
        }
    }
    const double bsum = block_sum(dot.value(), red);
    const int blk = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
    if (!publish(a, a.part + blk, bsum, &last)) return;
    const double pq = sum_partials(a.part, a.nblk, red);
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        CgState* s = a.s;
        if (pq > 0.0 && pq < INFINITY) {
            s->alpha = s->rr / pq;
        } else {
            s->alpha = 0.0;
            s->done = 1;   // p = 0 (exact solution) or a breakdown
        }
        s->ticket = 0;
    }
}

// cg_spmv_sm: the same step with the x / y neighbours of p from shared
// memory. Each thread forms p for its own 4 cells of plane z + 1 (two 128-bit
// loads), edge threads also for the one-cell ring of the 64 x 16 tile, and
// writes them into a two-plane shared ring; after one barrier a plane, q at
// plane z reads its x / y neighbours there (the z neighbours stay in the
// register queue). Two global loads a thread and plane instead of ten.
constexpr int SM_W = 72;   // shared row: x = -4 .. 67 of the tile, x = 0 at index 4

template <bool KVAR>
__global__ void __launch_bounds__(CG_TX * CG_TY, CgOcc<KVAR>::blocks) cg_spmv_sm(const __grid_constant__ CgArgs a) {
    __shared__ double red[CG_TX * CG_TY / 32];
    __shared__ bool last;
    __shared__ __align__(16) float sp[2][CG_TY + 2][SM_W];
    const CgCoef& c = a.c;
    if (a.s->done) return;
    const int par = a.s->iter & 1;
    PNew P;
    P.r = a.r;
    P.po = par ? a.p1 : a.p0;
    P.beta = (float)a.s->beta;
    P.first = a.s->iter == 0;
    float* __restrict__ pn = par ? a.p0 : a.p1;
    float* __restrict__ qv = a.q;
    const float* __restrict__ rk = a.rk;
    const int nx = c.n[0], ny = c.n[1], nz = c.n[2];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int x0 = blockIdx.x * 64, y0 = blockIdx.y * CG_TY;
    const int gx = x0 + 4 * tx, gy = y0 + ty;
    const int z0 = blockIdx.z * a.zchunk, z1 = min(z0 + a.zchunk, nz);
    const bool perx = c.periodic[0], pery = c.periodic[1], perz = c.periodic[2];
    const long long sy = c.sy, sz = c.sz;
    // every load below stays within the one-cell ring of the domain
    // ([-1, n] on each axis), inside the padded arrays' halo
    const bool own = gx < nx && gy < ny;
    // threads on the one-cell ring of the domain load too: on a periodic
    // axis their cells are the twins the domain's edge cells read
    const bool ld = gx <= nx && gy <= ny;
    const int ry = ty == 0 ? y0 - 1 : y0 + CG_TY;                       // y-ring row of this thread (ty 0 / 15)
    const bool yr = (ty == 0 || ty == CG_TY - 1) && gx < nx && ry <= ny;
    const int rx = tx == 0 ? x0 - 1 : x0 + 64;                          // x-ring cell of this row (tx 0 / 15)
    const bool xr = gy < ny && (tx == 0 || (tx == CG_TX - 1 && x0 + 63 < nx));
    const int srow = ty + 1, scol = 4 + 4 * tx;
    const int yrow = ty == 0 ? 0 : CG_TY + 1, xcol = tx == 0 ? 3 : 4 + 64;
    const long long own_o = cg_at(c, gx, gy, 0), yr_o = cg_at(c, gx, ry, 0), xr_o = cg_at(c, rx, gy, 0);
    const bool inner_xy = own && gx + 3 < nx && (perx || (gx > 0 && gx + 4 < nx)) && (pery || (gy > 0 && gy < ny - 1));
    const CgEdge edge = cg_edge(c, gx, gy);

    // shared planes start at 0: cells no thread writes (outside the ring of
    // the domain) stay finite
    for (int i = threadIdx.x + CG_TX * threadIdx.y; i < 2 * (CG_TY + 2) * SM_W; i += CG_TX * CG_TY)
        (&sp[0][0][0])[i] = 0.0f;
    __syncthreads();

    float pm[4], pc[4], km[4], kc[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) pm[i] = pc[i] = km[i] = kc[i] = 0.0f;
    if (ld) {
        pnew4(P, own_o + (long long)(z0 - 1) * sz, pm);
        pnew4(P, own_o + (long long)z0 * sz, pc);
    }
    if (own) {
        if (KVAR) {
            ld4(rk + own_o + (long long)(z0 - 1) * sz, km);
            ld4(rk + own_o + (long long)z0 * sz, kc);
        }
    }
    {   // plane z0 into shared slot z0 & 1
        float* sl = &sp[z0 & 1][0][0];
        sts4(sl + srow * SM_W + scol, pc);
        if (yr) {
            float v[4];
            pnew4(P, yr_o + (long long)z0 * sz, v);
            sts4(sl + yrow * SM_W + scol, v);
        }
        if (xr) sl[srow * SM_W + xcol] = pnew1(P, xr_o + (long long)z0 * sz);
    }
    __syncthreads();

    KahanF dot;
    for (int z = z0; z < z1; ++z) {
        const int cs = z & 1;
        const long long o = own_o + (long long)z * sz;
        float pp[4];
        if (ld) {
            if ((tx & 7) == 0) {   // one thread per 128-byte line asks L2 for plane z + 3
                prefetch_l2(P.r + o + 3 * sz);
                if (!P.first) prefetch_l2(P.po + o + 3 * sz);
            }
            pnew4(P, o + sz, pp);
        } else {
#pragma unroll
            for (int i = 0; i < 4; ++i) pp[i] = 0.0f;
        }
        {   // plane z + 1 into the other slot (free since the last barrier)
            float* sl = &sp[cs ^ 1][0][0];
            sts4(sl + srow * SM_W + scol, pp);
            if (yr) {
                float v[4];
                pnew4(P, yr_o + (long long)(z + 1) * sz, v);
                sts4(sl + yrow * SM_W + scol, v);
            }
            if (xr) sl[srow * SM_W + xcol] = pnew1(P, xr_o + (long long)(z + 1) * sz);
        }
        float kp[4], kym[4], kyp[4], kxm = 0.0f, kxp = 0.0f;
        if (KVAR) {
#pragma unroll
            for (int i = 0; i < 4; ++i) kp[i] = kym[i] = kyp[i] = 1.0f;
            if (own) {
                ld4(rk + o + sz, kp);
                ld4(rk + o - sy, kym);
                ld4(rk + o + sy, kyp);
                kxm = __ldg(rk + o - 1);
                kxp = __ldg(rk + o + 4);
            }
        }
        const float* sl = &sp[cs][0][0];
        float ym[4], yp[4];
        lds4(sl + (srow - 1) * SM_W + scol, ym);
        lds4(sl + (srow + 1) * SM_W + scol, yp);
        const float xm = sl[srow * SM_W + scol - 1], xp = sl[srow * SM_W + scol + 4];
        float q[4];
        // threads without own cells do not hold the warp back from the
        // interior formula (as in cg_spmv, where they do not take part)
        const bool fast = !own || (inner_xy && (perz || (z > 0 && z < nz - 1)));
        const float psum = __all_sync(__activemask(), fast)
                               ? cg_q4<KVAR, false>(c, edge, gx, gy, z, pc, pm, pp, ym, yp, xm, xp, kc, km, kp, kym, kyp,
                                                    kxm, kxp, q)
                               : cg_q4<KVAR, true>(c, edge, gx, gy, z, pc, pm, pp, ym, yp, xm, xp, kc, km, kp, kym, kyp,
                                                   kxm, kxp, q);
        if (own) {
            dot.add(psum);
            st4_twins(pn, c, gx, gy, z, pc);
            if (gx + 3 < nx) {
                *reinterpret_cast<float4*>(qv + o) = make_float4(q[0], q[1], q[2], q[3]);
            } else {
#pragma unroll
                for (int i = 0; i < 4; ++i)
                    if (gx + i < nx) qv[o + i] = q[i];
            }
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            pm[i] = pc[i];
            pc[i] = pp[i];
            if (KVAR) {
                km[i] = kc[i];
                kc[i] = kp[i];
            }
        }
        __syncthreads();
    }
    const double bsum = block_sum(dot.value(), red);
    const int blk = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
    if (!publish(a, a.part + blk, bsum, &last)) return;
    const double pq = sum_partials(a.part, a.nblk, red);
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        CgState* s = a.s;
        if (pq > 0.0 && pq < INFINITY) {
            s->alpha = s->rr / pq;
        } else {
            s->alpha = 0.0;
            s->done = 1;
        }
        s->ticket = 0;
    }
}

// ---------------------------------------------------------------- cg_pipe --
// One iteration of Chronopoulos and Gear's CG in one kernel and one
// reduction (the reduction-limited variant Sec. 3.2 points to): with alpha,
// beta of this iteration,
//   s = w + beta s,  p = r + beta p,  x += alpha p,  r' = r - alpha s,
//   w' = A r',  gamma' = r'.r',  delta' = w'.r'
// and the last block forms beta' = gamma' / gamma and
// alpha' = gamma' / (delta' - beta' gamma' / alpha). r' is needed at the
// neighbours of each cell, so it is formed there from r, w and s (three
// arrays with their x / y halo); r, w and s ping-pong between two buffers, p
// is read and written only at its own cell.
template <bool KVAR>
struct PipeOcc {
    static constexpr int blocks = KVAR ? 2 : 3;
};

struct RNew {
    const float* r;
    const float* w;
    const float* s;
    float alpha, beta;
    bool first;   // beta = 0: s = w (s is not read)
};

// r' and s at 4 cells of one row
__device__ __forceinline__ void rnew4(const RNew& R, long long o, float rn[4], float sn[4], float rv[4]) {
    ld4(R.r + o, rv);
    ld4(R.w + o, sn);
    if (!R.first) {
        float so[4];
        ld4(R.s + o, so);
#pragma unroll
        for (int i = 0; i < 4; ++i) sn[i] = __fmaf_rn(R.beta, so[i], sn[i]);
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) rn[i] = __fmaf_rn(-R.alpha, sn[i], rv[i]);
}
__device__ __forceinline__ float rnew1(const RNew& R, long long o) {
    float sv = __ldg(R.w + o);
    if (!R.first) sv = __fmaf_rn(R.beta, __ldg(R.s + o), sv);
    return __fmaf_rn(-R.alpha, sv, __ldg(R.r + o));
}

template <bool KVAR>
__global__ void __launch_bounds__(CG_TX * CG_TY, PipeOcc<KVAR>::blocks) cg_pipe(const __grid_constant__ CgArgs a) {
    __shared__ double red[CG_TX * CG_TY / 32];
    __shared__ bool last;
    const CgCoef& c = a.c;
    if (a.s->done) return;
    const int par = a.s->iter & 1;   // iteration i reads r, w [i mod 2], writes [(i + 1) mod 2]
    RNew R;
    R.r = par ? a.r2 : a.r;
    R.w = par ? a.w2 : a.q;
    R.s = par ? a.s2 : a.p1;
    R.alpha = (float)a.s->alpha;
    R.beta = (float)a.s->beta;
    R.first = a.s->iter == 0;
    float* __restrict__ r_out = par ? a.r : a.r2;
    float* __restrict__ w_out = par ? a.q : a.w2;
    float* __restrict__ pv = a.p0;
    float* __restrict__ sv = par ? a.p1 : a.s2;
    float* __restrict__ xv = a.x;
    const float* __restrict__ rk = a.rk;
    const int nx = c.n[0], ny = c.n[1], nz = c.n[2];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int gx = blockIdx.x * 64 + 4 * tx, gy = blockIdx.y * CG_TY + ty;
    const int z0 = blockIdx.z * a.zchunk, z1 = min(z0 + a.zchunk, nz);
    const bool perx = c.periodic[0], pery = c.periodic[1], perz = c.periodic[2];
    KahanF gam, del;
    if (gx < nx && gy < ny) {
        const long long sy = c.sy, sz = c.sz;
        const long long row = cg_at(c, gx, gy, 0);
        const bool inner_xy = gx + 3 < nx && (perx || (gx > 0 && gx + 4 < nx)) && (pery || (gy > 0 && gy < ny - 1));
        const CgEdge edge = cg_edge(c, gx, gy);
        float rm[4], rc[4], sc[4], rvc[4], km[4], kc[4], tmp[4];
        rnew4(R, row + (long long)(z0 - 1) * sz, rm, tmp, rvc);
        rnew4(R, row + (long long)z0 * sz, rc, sc, rvc);
        if (KVAR) {
            ld4(rk + row + (long long)(z0 - 1) * sz, km);
            ld4(rk + row + (long long)z0 * sz, kc);
        }
        for (int z = z0; z < z1; ++z) {
            const long long o = row + (long long)z * sz;
            if ((tx & 7) == 0) {   // one thread per 128-byte line asks L2 for plane z + 3
                prefetch_l2(R.r + o + 3 * sz);
                prefetch_l2(R.w + o + 3 * sz);
                if (!R.first) prefetch_l2(R.s + o + 3 * sz);
            }
            float rp[4], sp_[4], rvp[4], ym[4], yp[4], t4[4], t5[4];
            rnew4(R, o + sz, rp, sp_, rvp);
            rnew4(R, o - sy, ym, t4, t5);
            rnew4(R, o + sy, yp, t4, t5);
            const float xm = rnew1(R, o - 1), xp = rnew1(R, o + 4);
            float kp[4], kym[4], kyp[4], kxm = 0.0f, kxp = 0.0f;
            if (KVAR) {
                ld4(rk + o + sz, kp);
                ld4(rk + o - sy, kym);
                ld4(rk + o + sy, kyp);
                kxm = __ldg(rk + o - 1);
                kxp = __ldg(rk + o + 4);
            }
            float wn[4];
            const bool fast = inner_xy && (perz || (z > 0 && z < nz - 1));
            const bool interior = __all_sync(__activemask(), fast);
            const float dsum = interior
                                   ? cg_q4<KVAR, false>(c, edge, gx, gy, z, rc, rm, rp, ym, yp, xm, xp, kc, km, kp, kym,
                                                        kyp, kxm, kxp, wn)
                                   : cg_q4<KVAR, true>(c, edge, gx, gy, z, rc, rm, rp, ym, yp, xm, xp, kc, km, kp, kym,
                                                       kyp, kxm, kxp, wn);
            float gsum = 0.0f;
#pragma unroll
            for (int i = 0; i < 4; ++i)
                gsum = (interior || gx + i < nx) ? __fmaf_rn(rc[i], rc[i], gsum) : gsum;   // held cells: r' = 0
            gam.add(gsum);
            del.add(dsum);
            // own cells at plane z: p, x, and the new s, r, w
            float pn[4], xn[4];
            ld4(xv + o, xn);
            if (R.first) {
#pragma unroll
                for (int i = 0; i < 4; ++i) pn[i] = rvc[i];
            } else {
                ld4(pv + o, pn);
#pragma unroll
                for (int i = 0; i < 4; ++i) pn[i] = __fmaf_rn(R.beta, pn[i], rvc[i]);
            }
#pragma unroll
            for (int i = 0; i < 4; ++i) xn[i] = __fmaf_rn(R.alpha, pn[i], xn[i]);
            st4_row(pv + o, gx, nx, pn);
            st4_twins(sv, c, gx, gy, z, sc);
            st4_twins(xv, c, gx, gy, z, xn);
            st4_twins(r_out, c, gx, gy, z, rc);
            st4_twins(w_out, c, gx, gy, z, wn);
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                rm[i] = rc[i];
                rc[i] = rp[i];
                sc[i] = sp_[i];
                rvc[i] = rvp[i];
                if (KVAR) {
                    km[i] = kc[i];
                    kc[i] = kp[i];
                }
            }
        }
    }
    const double gs = block_sum(gam.value(), red);
    const double ds = block_sum(del.value(), red);
    const int blk = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
    if (threadIdx.x == 0 && threadIdx.y == 0) a.part[CG_MAX_PART + blk] = ds;
    if (!publish(a, a.part + blk, gs, &last)) return;
    const double G = sum_partials(a.part, a.nblk, red);
    const double Dl = sum_partials(a.part + CG_MAX_PART, a.nblk, red);
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        CgState* st = a.s;
        const double beta = st->rr > 0.0 ? G / st->rr : 0.0;
        const double den = st->alpha > 0.0 ? Dl - beta * G / st->alpha : 0.0;
        st->iter += 1;
        st->beta = beta;
        st->rr = G;
        if (den > 0.0 && den < INFINITY) {
            st->alpha = G / den;
        } else {
            st->alpha = 0.0;
            st->done = 1;   // r' = 0 (exact solution) or a breakdown
        }
        if (G <= st->tol2 * st->bb || st->iter >= st->max_iter || !(G == G)) st->done = 1;
        st->ticket = 0;
    }
}

// -------------------------------------------------------------- cg_update --
// x += alpha p, r -= alpha q over the domain cells (4 along x per item),
// r.r partials; then beta and the convergence test.
__global__ void __launch_bounds__(CG_THREADS) cg_update(const __grid_constant__ CgArgs a) {
    __shared__ double red[CG_THREADS / 32];
    __shared__ bool last;
    const CgCoef& c = a.c;
    if (a.s->done) return;
    const int par = a.s->iter & 1;
    const float alpha = (float)a.s->alpha;
    const float* __restrict__ p = par ? a.p0 : a.p1;
    const int nx = c.n[0], ny = c.n[1], nz = c.n[2];
    const int xg = (nx + 3) / 4;
    const long long items = (long long)xg * ny * nz;
    KahanF rr;
    // item it = (x group, y, z); one division at the start, then the stride
    // is added digit by digit (no 64-bit division in the loop)
    const long long it0 = blockIdx.x * (long long)CG_THREADS + threadIdx.x;
    const long long stride = (long long)gridDim.x * CG_THREADS;
    const int dxg = (int)(stride % xg);
    const long long drow = stride / xg;
    const int dy = (int)(drow % ny), dz = (int)(drow / ny);
    int ixg = (int)(it0 % xg), y = (int)((it0 / xg) % ny), z = (int)(it0 / xg / ny);
    for (long long it = it0; it < items; it += stride) {
        const int gx = 4 * ixg;
        const long long o = cg_at(c, gx, y, z);
        float xv[4], pv[4], qv[4], rv[4];
        ld4(a.x + o, xv);
        ld4(p + o, pv);
        ld4(a.q + o, qv);
        ld4(a.r + o, rv);
        float s = 0.0f;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            xv[i] = __fmaf_rn(alpha, pv[i], xv[i]);
            rv[i] = __fmaf_rn(-alpha, qv[i], rv[i]);
            if (gx + i < nx) s = __fmaf_rn(rv[i], rv[i], s);
        }
        rr.add(s);
        st4_twins(a.x, c, gx, y, z, xv);   // the field's twins feed the next step's cg_init
        st4_twins(a.r, c, gx, y, z, rv);
        ixg += dxg;
        y += dy;
        z += dz;
        if (ixg >= xg) {
            ixg -= xg;
            ++y;
        }
        if (y >= ny) {
            y -= ny;
            ++z;
        }
    }
    const double bsum = block_sum(rr.value(), red);
    if (!publish(a, a.part + blockIdx.x, bsum, &last)) return;
    const double R = sum_partials(a.part, a.nblk, red);
    if (threadIdx.x == 0) {
        CgState* s = a.s;
        s->beta = s->rr > 0.0 ? R / s->rr : 0.0;
        s->rr = R;
        s->iter += 1;
        if (R <= s->tol2 * s->bb || s->iter >= s->max_iter || !(R == R)) s->done = 1;
        s->ticket = 0;
    }
}

// ---------------------------------------------------------- device loops --
// The whole call as one graph launch: an outer conditional WHILE node over the
// time steps, an inner one over the CG iterations of a step. One thread of a
// control kernel sets each loop's condition; both loops also stop on their
// own counters (max_iter + 2 iterations, n steps), whatever the solver
// scalars say, so neither can run on without bound.
struct CgLoop {
    long long steps_left;    // time steps still to take
    long long steps_limit;   // n: the outer loop's own bound
    long long steps_done;
    long long total_iters;   // CG iterations of all steps
    double last_rr, last_bb; // the last step's r.r and b.b
    unsigned inner_count;    // iterations run in the current step (the inner loop's own bound)
    unsigned pad;
};
static_assert(sizeof(CgLoop) <= 64, "CgLoop is read back into a 64-byte pinned word");

__global__ void cg_ctl_start(CgState* s, CgLoop* L, cudaGraphConditionalHandle inner) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        L->inner_count = 0;
        cudaGraphSetConditional(inner, s->done ? 0u : 1u);
    }
}

__global__ void cg_ctl_iter(CgState* s, CgLoop* L, cudaGraphConditionalHandle inner, int max_iter) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        const unsigned k = ++L->inner_count;
        cudaGraphSetConditional(inner, (!s->done && k < (unsigned)max_iter + 2u) ? 1u : 0u);
    }
}

__global__ void cg_ctl_step(CgState* s, CgLoop* L, cudaGraphConditionalHandle outer) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        L->total_iters += s->iter;
        L->last_rr = s->rr;
        L->last_bb = s->bb;
        L->steps_left -= 1;
        L->steps_done += 1;
        cudaGraphSetConditional(outer, (L->steps_left > 0 && L->steps_done < L->steps_limit) ? 1u : 0u);
    }
}

// ------------------------------------------------------------------ host --
struct CgWork {
    float* r = nullptr;
    float* p[2] = {nullptr, nullptr};
    float* q = nullptr;
    double* part = nullptr;
    CgState* s = nullptr;
    CgState* h[2] = {nullptr, nullptr};   // pinned read-back slots
    cudaEvent_t ev[2] = {nullptr, nullptr};
    float* extra[3] = {nullptr, nullptr, nullptr};   // pipelined CG: r2, w2, s2 (allocated on first use)
    CgLoop* loop = nullptr;            // device loop counters
    cudaGraphExec_t loop_exec = nullptr;   // the whole call as one graph (device loops)
    CgArgs loop_key;
    int loop_kvar = -1, loop_method = -1, loop_max_iter = -1;
    double loop_tol2 = -1.0;
    bool loop_broken = false;          // building it failed once: host loop from then on
    cudaGraphExec_t exec[CG_NRUN] = {nullptr, nullptr, nullptr, nullptr};
    cudaStream_t cap = nullptr;   // capture stream (the grid's own may be the legacy default stream)
    CgArgs key;        // arguments the graph was captured with
    int kvar = -1;
    int method = -1;   // WFA_CG_CLASSIC / WFA_CG_PIPELINED of the captured graphs
    int spmv_grid[3] = {0, 0, 0};
    int upd_blocks = 0;
    long long prev_iters = 0;   // iterations the last step needed (sizes the first run of the next)
    bool o32 = false;           // every array under 4 GiB: cg_init takes 32-bit byte offsets
};

void free_cg(wfa_grid_s* g) {
    CgWork* w = static_cast<CgWork*>(g->cg);
    if (!w) return;
    cudaStreamSynchronize(g->stream);
    for (cudaGraphExec_t e : w->exec)
        if (e) cudaGraphExecDestroy(e);
    if (w->cap) cudaStreamDestroy(w->cap);
    for (int b = 0; b < 2; ++b) {
        if (w->ev[b]) cudaEventDestroy(w->ev[b]);
        pinned_release(w->h[b]);
        padded_free(w->p[b], 4, g->stream);
    }
    if (w->loop_exec) cudaGraphExecDestroy(w->loop_exec);
    dev_free(w->loop, g->stream);
    for (float* e : w->extra) padded_free(e, 4, g->stream);
    padded_free(w->r, 4, g->stream);
    padded_free(w->q, 4, g->stream);
    dev_free(w->part, g->stream);
    dev_free(w->s, g->stream);
    delete w;
    g->cg = nullptr;
}

static int cg_workspace(wfa_grid_s* g, CgWork** out) {
    if (g->cg) {
        *out = static_cast<CgWork*>(g->cg);
        return WFA_OK;
    }
    CgWork* w = new (std::nothrow) CgWork();
    if (!w) {
        set_error("host allocation failed");
        return WFA_ERR_OOM;
    }
    g->cg = w;
    const size_t fb = field_elems(g) * sizeof(float);
    w->o32 = fb < ((size_t)1 << 32);
    // padded arrays in the field's layout (see lead_bytes)
    cudaError_t e = padded_alloc((void**)&w->r, fb, 4, g->stream);
    for (int b = 0; b < 2 && e == cudaSuccess; ++b) e = padded_alloc((void**)&w->p[b], fb, 4, g->stream);
    if (e == cudaSuccess) e = padded_alloc((void**)&w->q, fb, 4, g->stream);
    if (e == cudaSuccess) e = dev_alloc((void**)&w->part, 2 * CG_MAX_PART * sizeof(double), g->stream);
    if (e == cudaSuccess) e = dev_alloc((void**)&w->s, sizeof(CgState), g->stream);
    // the halos and held cells of the work vectors stay 0 (finite) for good
    for (float* v : {w->r, w->p[0], w->p[1], w->q})
        if (e == cudaSuccess) e = cudaMemsetAsync(v, 0, fb, g->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(w->s, 0, sizeof(CgState), g->stream);
    for (int b = 0; b < 2 && e == cudaSuccess; ++b) {
        w->h[b] = static_cast<CgState*>(pinned_word());
        if (!w->h[b]) e = cudaErrorMemoryAllocation;
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&w->ev[b], cudaEventDisableTiming);
    }
    if (e != cudaSuccess) {
        const int rc = cuda_fail(e, "implicit solver workspace");
        free_cg(g);
        return rc;
    }
    *out = w;
    return WFA_OK;
}

static void cg_coef(const wfa_grid_s* g, double dt, CgCoef* c) {
    memset(c, 0, sizeof *c);
    for (int a = 0; a < 3; ++a) {
        c->n[a] = g->n[a];
        c->periodic[a] = g->bc_kind[2 * a] == WFA_BC_PERIODIC;
        const double ih2 = 1.0 / (g->h[a] * g->h[a]);
        c->cu[a] = (float)(dt * g->k_uniform * ih2);
        c->tcd[a] = (float)(2.0 * dt * ih2);
    }
    c->du = 1.0f + 2.0f * (c->cu[0] + c->cu[1] + c->cu[2]);
    for (int f = 0; f < 6; ++f) {
        c->dface[f] = g->bc_kind[f] == WFA_BC_DIRICHLET;
        c->held[f] = g->bc_kind[f] == WFA_BC_DIRICHLET_CELL;
        c->tb[f] = (float)g->bc_value[f];
    }
    c->sy = g->px;
    c->sz = g->px * g->py;
}

static int cg_capture(wfa_grid_s* g, CgWork* w, const CgArgs& base, bool kvar, int method) {
    if (w->exec[0] && w->kvar == (int)kvar && w->method == method && memcmp(&w->key, &base, sizeof base) == 0)
        return WFA_OK;
    for (cudaGraphExec_t& e : w->exec)
        if (e) {
            cudaGraphExecDestroy(e);
            e = nullptr;
        }
    CgArgs sp = base, up = base;
    sp.nblk = w->spmv_grid[0] * w->spmv_grid[1] * w->spmv_grid[2];
    up.nblk = w->upd_blocks;
    const dim3 sgrid(w->spmv_grid[0], w->spmv_grid[1], w->spmv_grid[2]), sblock(CG_TX, CG_TY);
    if (!w->cap) WFA_CUDA(cudaStreamCreateWithFlags(&w->cap, cudaStreamNonBlocking));
    const cudaStream_t st = w->cap;
    // q = A p from L1-cached neighbour loads (cg_spmv) or through a shared
    // plane (cg_spmv_sm); WFA_CG_SPMV=l1|sm overrides the default
    const char* pick = getenv("WFA_CG_SPMV");
    const bool use_sm = pick ? strcmp(pick, "sm") == 0 : CG_SPMV_SM_DEFAULT;
    for (int k = 0; k < CG_NRUN; ++k) {
        WFA_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
        cudaError_t e = cudaSuccess;
        for (int it = 0; it < CG_RUN_LEN[k] && e == cudaSuccess; ++it) {
            if (method == WFA_CG_PIPELINED) {   // one kernel, one reduction an iteration
                if (kvar)
                    cg_pipe<true><<<sgrid, sblock, 0, st>>>(sp);
                else
                    cg_pipe<false><<<sgrid, sblock, 0, st>>>(sp);
                e = cudaGetLastError();
                continue;
            }
            if (kvar && use_sm)
                cg_spmv_sm<true><<<sgrid, sblock, 0, st>>>(sp);
            else if (kvar)
                cg_spmv<true><<<sgrid, sblock, 0, st>>>(sp);
            else if (use_sm)
                cg_spmv_sm<false><<<sgrid, sblock, 0, st>>>(sp);
            else
                cg_spmv<false><<<sgrid, sblock, 0, st>>>(sp);
            e = cudaGetLastError();
            if (e == cudaSuccess) {
                cg_update<<<w->upd_blocks, CG_THREADS, 0, st>>>(up);
                e = cudaGetLastError();
            }
        }
        cudaGraph_t gr = nullptr;
        const cudaError_t e2 = cudaStreamEndCapture(st, &gr);
        if (e == cudaSuccess) e = e2;
        if (e == cudaSuccess) e = cudaGraphInstantiate(&w->exec[k], gr, 0);
        if (gr) cudaGraphDestroy(gr);
        if (e != cudaSuccess) {
            w->exec[k] = nullptr;
            return cuda_fail(e, "implicit solver graph");
        }
    }
    w->key = base;
    w->kvar = kvar;
    w->method = method;
    return WFA_OK;
}

// Kernel node of `fn` with the given arguments, depending on `dep` (if any).
static cudaError_t add_kernel(cudaGraph_t gr, cudaGraphNode_t* node, cudaGraphNode_t dep, const void* fn, dim3 grid,
                              dim3 block, void** args) {
    cudaKernelNodeParams kp = {};
    kp.func = const_cast<void*>(fn);
    kp.gridDim = grid;
    kp.blockDim = block;
    kp.sharedMemBytes = 0;
    kp.kernelParams = args;
    return cudaGraphAddKernelNode(node, gr, dep ? &dep : nullptr, dep ? 1 : 0, &kp);
}

// Conditional WHILE node depending on `dep`; its body graph is returned.
static cudaError_t add_while(cudaGraph_t gr, cudaGraphNode_t* node, cudaGraphNode_t dep, cudaGraphConditionalHandle h,
                             cudaGraph_t* body) {
    cudaGraphNodeParams np = {};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = h;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaError_t e = cudaGraphAddNode(node, gr, dep ? &dep : nullptr, nullptr, dep ? 1 : 0, &np);
    if (e == cudaSuccess) *body = np.conditional.phGraph_out[0];
    return e;
}

// outer WHILE (steps) { cg_init; [pipelined: cg_spmv]; cg_ctl_start;
//   inner WHILE (iterations) { classic: cg_spmv, cg_update | pipelined: cg_pipe; cg_ctl_iter }; cg_ctl_step }
static cudaError_t build_loop_graph(CgWork* w, const CgArgs& base, bool kvar, int method, double tol2,
                                    int max_iter, cudaGraphExec_t* out) {
    cudaGraph_t top = nullptr;
    cudaError_t e = cudaGraphCreate(&top, 0);
    if (e != cudaSuccess) return e;
    cudaGraphConditionalHandle ho = 0, hi = 0;
    cudaGraph_t outer = nullptr, inner = nullptr;
    cudaGraphNode_t n_outer = nullptr, n = nullptr, prev = nullptr;
    CgArgs ia = base, sp = base, up = base;
    ia.nblk = sp.nblk = w->spmv_grid[0] * w->spmv_grid[1] * w->spmv_grid[2];
    up.nblk = w->upd_blocks;
    const dim3 sgrid(w->spmv_grid[0], w->spmv_grid[1], w->spmv_grid[2]), sblock(CG_TX, CG_TY);
    CgState* st = w->s;
    CgLoop* L = w->loop;
    void* a_init[] = {&ia, &tol2, &max_iter};
    void* a_sp[] = {&sp};
    void* a_up[] = {&up};
    void* a_start[] = {&st, &L, &hi};
    void* a_iter[] = {&st, &L, &hi, &max_iter};
    void* a_step[] = {&st, &L, &ho};
    e = cudaGraphConditionalHandleCreate(&ho, top, 1, cudaGraphCondAssignDefault);
    if (e == cudaSuccess) e = add_while(top, &n_outer, nullptr, ho, &outer);
    if (e == cudaSuccess)
        e = add_kernel(outer, &n, nullptr,
                       kvar ? (w->o32 ? (const void*)cg_init<true, true> : (const void*)cg_init<true, false>)
                            : (w->o32 ? (const void*)cg_init<false, true> : (const void*)cg_init<false, false>),
                       sgrid,
                       sblock, a_init);
    prev = n;
    if (e == cudaSuccess && method == WFA_CG_PIPELINED) {
        e = add_kernel(outer, &n, prev, kvar ? (const void*)cg_spmv<true> : (const void*)cg_spmv<false>, sgrid, sblock,
                       a_sp);
        prev = n;
    }
    if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&hi, outer, 0, 0);
    if (e == cudaSuccess) e = add_kernel(outer, &n, prev, (const void*)cg_ctl_start, dim3(1), dim3(32), a_start);
    prev = n;
    cudaGraphNode_t n_inner = nullptr;
    if (e == cudaSuccess) e = add_while(outer, &n_inner, prev, hi, &inner);
    if (e == cudaSuccess) {
        cudaGraphNode_t ip = nullptr;
        if (method == WFA_CG_PIPELINED) {
            e = add_kernel(inner, &ip, nullptr, kvar ? (const void*)cg_pipe<true> : (const void*)cg_pipe<false>, sgrid,
                           sblock, a_sp);
        } else {
            e = add_kernel(inner, &ip, nullptr, kvar ? (const void*)cg_spmv<true> : (const void*)cg_spmv<false>, sgrid,
                           sblock, a_sp);
            if (e == cudaSuccess)
                e = add_kernel(inner, &ip, ip, (const void*)cg_update, dim3(w->upd_blocks), dim3(CG_THREADS), a_up);
        }
        if (e == cudaSuccess) e = add_kernel(inner, &ip, ip, (const void*)cg_ctl_iter, dim3(1), dim3(32), a_iter);
    }
    if (e == cudaSuccess) e = add_kernel(outer, &n, n_inner, (const void*)cg_ctl_step, dim3(1), dim3(32), a_step);
    if (e == cudaSuccess) e = cudaGraphInstantiate(out, top, 0);
    cudaGraphDestroy(top);
    return e;
}

}  // namespace wfa

using namespace wfa;

int wfa_implicit_step(wfa_grid g, double dt, long long n, double rtol, int max_iter, long long* iters,
                      double* rel_res) {
    NvtxRange nvtx_("wfa_implicit_step");
    if (!g) {
        set_error("NULL grid");
        return WFA_ERR_ARG;
    }
    if (!(dt >= 0.0) || !std::isfinite(dt) || n < 0 || !(rtol >= 0.0) || !std::isfinite(rtol) || max_iter < 0) {
        set_error("wfa_implicit_step: need dt >= 0 (finite), n >= 0, rtol >= 0 (finite), max_iter >= 0");
        return WFA_ERR_ARG;
    }
    if (g->storage != WFA_F32) {
        set_error("wfa_implicit_step: the implicit solver needs fp32 storage");
        return WFA_ERR_ARG;
    }
    if (!g->field_set || !g->coeffs_set) {
        set_error("set the field and the coefficients before an implicit step");
        return WFA_ERR_STATE;
    }
    if (g->u[0] != 0.0 || g->u[1] != 0.0 || g->u[2] != 0.0) {
        set_error("wfa_implicit_step: advection makes the system non-symmetric; CG needs u = 0");
        return WFA_ERR_ARG;
    }
    for (int a = 0; a < 3; ++a)
        if ((g->bc_kind[2 * a] == WFA_BC_PERIODIC) != (g->bc_kind[2 * a + 1] == WFA_BC_PERIODIC)) {
            set_error("axis %d: a periodic face needs a periodic opposite face", a);
            return WFA_ERR_BC;
        }
    if (has_exchange_face(g)) {   // a slab's CG would need the other slabs' inner products
        set_error("wfa_implicit_step: exchange faces are for the explicit step only");
        return WFA_ERR_BC;
    }
    if (iters) *iters = 0;
    if (rel_res) *rel_res = 0.0;
    if (n == 0) return WFA_OK;
    if (g->halo_dirty) {   // held layers carry their value before the first solve
        int rc = refresh_halo(g, g->cur);
        if (rc) return rc;
        g->halo_dirty = false;
    }
    int rc = prepare_coeff_halo(g);
    if (rc) return rc;
    CgWork* w = nullptr;
    rc = cg_workspace(g, &w);
    if (rc) return rc;

    const bool kvar = g->k != nullptr;
    const long long off = domain_offset(g);
    CgArgs base;
    memset(&base, 0, sizeof base);
    cg_coef(g, dt, &base.c);
    base.x = static_cast<float*>(g->T[g->cur]) + off;
    base.rk = kvar ? g->r + off : nullptr;
    base.r = w->r + off;
    base.p0 = w->p[0] + off;
    base.p1 = w->p[1] + off;
    base.q = w->q + off;
    base.part = w->part;
    base.s = w->s;
    int nsm = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (nsm <= 0) nsm = 1;
    {   // cg_spmv / cg_init grid: 64 x 16 columns, z chunks of about 16 planes,
        // many waves of blocks so the last wave's tail is short; chunks down to
        // 2 planes only where 16 would leave SMs idle (small grids)
        const int gxb = (g->n[0] + 63) / 64, gyb = (g->n[1] + CG_TY - 1) / CG_TY;
        const long long cols = (long long)gxb * gyb;
        const long long resident = (long long)nsm * (kvar ? CgOcc<true>::blocks : CgOcc<false>::blocks);
        long long nch = std::max<long long>(1, resident * 16 / cols);
        long long cap = std::max(1, g->n[2] / 16);
        if (cols * cap < resident) cap = std::max(1, g->n[2] / 2);
        nch = std::min(nch, cap);
        nch = std::min<long long>(nch, std::max<long long>(1, CG_MAX_PART / cols));
        base.zchunk = (int)((g->n[2] + nch - 1) / nch);
        nch = (g->n[2] + base.zchunk - 1) / base.zchunk;
        if (cols * nch > CG_MAX_PART) {
            set_error("wfa_implicit_step: grid too large for the partial-sum buffer");
            return WFA_ERR_ARG;
        }
        w->spmv_grid[0] = gxb;
        w->spmv_grid[1] = gyb;
        w->spmv_grid[2] = (int)nch;
        const long long items = (long long)((g->n[0] + 3) / 4) * g->n[1] * g->n[2];
        w->upd_blocks = (int)std::max<long long>(1, std::min<long long>((items + CG_THREADS - 1) / CG_THREADS, nsm * 8LL));
    }
    const int method = g->cg_method;
    if (method == WFA_CG_PIPELINED) {   // three more work vectors: r, w and s ping-pong
        const size_t fb = field_elems(g) * sizeof(float);
        for (float*& e : w->extra)
            if (!e) {
                WFA_CUDA(padded_alloc((void**)&e, fb, 4, g->stream));
                WFA_CUDA(cudaMemsetAsync(e, 0, fb, g->stream));
            }
        base.r2 = w->extra[0] + off;
        base.w2 = w->extra[1] + off;
        base.s2 = w->extra[2] + off;
        base.q_twins = 1;
    }
    rc = cg_capture(g, w, base, kvar, method);
    if (rc) return rc;

    const int per_iter = method == WFA_CG_PIPELINED ? 1 : 2;   // kernels an iteration

    // The device-loop graph: every step and iteration without a host round
    // trip (WFA_CG_LOOP=host keeps the host-checked runs below).
    const char* loop_pick = getenv("WFA_CG_LOOP");
    if (!(loop_pick && strcmp(loop_pick, "host") == 0) && !w->loop_broken) {
        const double tol2 = rtol * rtol;
        if (!w->loop) {
            WFA_CUDA(dev_alloc((void**)&w->loop, sizeof(CgLoop), g->stream));
        }
        if (!w->loop_exec || w->loop_kvar != (int)kvar || w->loop_method != method || w->loop_max_iter != max_iter ||
            w->loop_tol2 != tol2 || memcmp(&w->loop_key, &base, sizeof base) != 0) {
            if (w->loop_exec) cudaGraphExecDestroy(w->loop_exec);
            w->loop_exec = nullptr;
            const cudaError_t e = build_loop_graph(w, base, kvar, method, tol2, max_iter, &w->loop_exec);
            if (e != cudaSuccess) {   // no conditional nodes here: host-checked runs from now on
                cudaGetLastError();
                w->loop_exec = nullptr;
                w->loop_broken = true;
            } else {
                w->loop_key = base;
                w->loop_kvar = kvar;
                w->loop_method = method;
                w->loop_max_iter = max_iter;
                w->loop_tol2 = tol2;
            }
        }
        if (w->loop_exec) {
            CgLoop L0;
            memset(&L0, 0, sizeof L0);
            L0.steps_left = n;
            L0.steps_limit = n;
            CgLoop* h = reinterpret_cast<CgLoop*>(w->h[0]);
            memcpy(h, &L0, sizeof L0);
            WFA_CUDA(cudaMemcpyAsync(w->loop, h, sizeof(CgLoop), cudaMemcpyHostToDevice, g->stream));
            WFA_CUDA(cudaGraphLaunch(w->loop_exec, g->stream));
            WFA_CUDA(cudaMemcpyAsync(h, w->loop, sizeof(CgLoop), cudaMemcpyDeviceToHost, g->stream));
            WFA_CUDA(cudaStreamSynchronize(g->stream));
            CgLoop Lr;
            memcpy(&Lr, h, sizeof Lr);
            if (Lr.steps_done != n) {
                set_error("wfa_implicit_step: the device loop ran %lld of %lld steps", Lr.steps_done, n);
                return WFA_ERR_STATE;
            }
            const int extra_per_step = method == WFA_CG_PIPELINED ? 4 : 3;   // init, [spmv], start, step
            g->launches += extra_per_step * n + (long long)(per_iter + 1) * Lr.total_iters;
            w->prev_iters = n > 0 ? Lr.total_iters / n : 0;
            g->halo_dirty = true;
            g->steps_done += n;
            if (iters) *iters = Lr.total_iters;
            if (rel_res) *rel_res = Lr.last_bb > 0.0 ? sqrt(Lr.last_rr / Lr.last_bb) : sqrt(Lr.last_rr);
            return WFA_OK;
        }
    }

    CgArgs ia = base;
    ia.nblk = w->spmv_grid[0] * w->spmv_grid[1] * w->spmv_grid[2];
    const dim3 sgrid(w->spmv_grid[0], w->spmv_grid[1], w->spmv_grid[2]), sblock(CG_TX, CG_TY);
    long long total = 0;
    double last_rel = 0.0;
    for (long long step = 0; step < n; ++step) {
        if (kvar)
            if (w->o32) cg_init<true, true><<<sgrid, sblock, 0, g->stream>>>(ia, rtol * rtol, max_iter);
            else cg_init<true, false><<<sgrid, sblock, 0, g->stream>>>(ia, rtol * rtol, max_iter);
        else
            if (w->o32) cg_init<false, true><<<sgrid, sblock, 0, g->stream>>>(ia, rtol * rtol, max_iter);
            else cg_init<false, false><<<sgrid, sblock, 0, g->stream>>>(ia, rtol * rtol, max_iter);
        WFA_CUDA(cudaGetLastError());
        g->launches += 1;
        if (method == WFA_CG_PIPELINED) {
            // w = A r, delta = w.r and alpha = r.r / delta: the first half of a
            // classic iteration (q = A p with p = r), q keeping its twins
            if (kvar)
                cg_spmv<true><<<sgrid, sblock, 0, g->stream>>>(ia);
            else
                cg_spmv<false><<<sgrid, sblock, 0, g->stream>>>(ia);
            WFA_CUDA(cudaGetLastError());
            g->launches += 1;
        }
        // Runs of captured iterations with one run queued ahead of the flag
        // check, so the GPU does not wait for the host: the first run as long
        // as the last step needed (rounded up to 1, 2, 4 or 8), then 2, then 8s.
        // Iterations after convergence are kernels that return at once.
        long long queued = 0, launched = 0;
        auto enqueue = [&]() -> int {
            int k = CG_NRUN - 1;
            if (launched == 0) {
                const long long want = w->prev_iters > 0 ? w->prev_iters : CG_RUN_LEN[CG_NRUN - 1];
                k = 0;
                while (k < CG_NRUN - 1 && CG_RUN_LEN[k] < want) ++k;
            } else if (launched == 1) {
                k = 1;
            }
            WFA_CUDA(cudaGraphLaunch(w->exec[k], g->stream));
            WFA_CUDA(cudaMemcpyAsync(w->h[launched & 1], w->s, sizeof(CgState), cudaMemcpyDeviceToHost, g->stream));
            WFA_CUDA(cudaEventRecord(w->ev[launched & 1], g->stream));
            g->launches += per_iter * CG_RUN_LEN[k];
            queued += CG_RUN_LEN[k];
            ++launched;
            return WFA_OK;
        };
        rc = enqueue();
        if (rc) return rc;
        CgState st;
        memset(&st, 0, sizeof st);
        for (long long k = 0;; ++k) {
            if (launched == k + 1 && queued < max_iter) {
                rc = enqueue();
                if (rc) return rc;
            }
            WFA_CUDA(cudaEventSynchronize(w->ev[k & 1]));
            memcpy(&st, w->h[k & 1], sizeof st);
            if (st.done) break;
            if (launched == k + 1) {   // nothing left in flight, yet not done
                set_error("wfa_implicit_step: the solver did not report completion");
                return WFA_ERR_STATE;
            }
        }
        WFA_CUDA(cudaStreamSynchronize(g->stream));   // the run queued ahead has ended (no-op kernels)
        total += st.iter;
        w->prev_iters = st.iter;
        last_rel = st.bb > 0.0 ? sqrt(st.rr / st.bb) : sqrt(st.rr);
    }
    g->halo_dirty = true;   // periodic copies and ghost layers of the field are stale
    g->steps_done += n;
    if (iters) *iters = total;
    if (rel_res) *rel_res = last_rel;
    return WFA_OK;
}

int wfa_set_cg_method(wfa_grid g, int method) {
    if (!g || (method != WFA_CG_CLASSIC && method != WFA_CG_PIPELINED)) {
        set_error("wfa_set_cg_method: NULL grid or unknown method %d", method);
        return WFA_ERR_ARG;
    }
    g->cg_method = method;
    return WFA_OK;
}
