// sweep_col<S, KVAR>: one explicit step per pass (Sec. 1.1.1,
// Eq. expl_form in face-flux form) without shared memory or barriers.
//
// Every thread owns V consecutive x cells of one row (4; 8 for the wide
// variant, 16 for bf16 with uniform k) and marches along z over a chunk of
// planes. Its own values at planes z-1, z, z+1 live in a register queue; at
// plane z it loads plane z + 1 (own cells, 128-bit along x) and the x / y
// neighbours at plane z, and asks L2 for plane z + 3, so the loads mostly
// hit L2 by the time they are issued. x / y neighbours of a thread are other
// threads' cells of the same plane, so they come from L1; every value is read
// from DRAM about once per pass. Addresses are constant byte offsets from a
// pointer to the thread's cells in each plane. The per-cell
// arithmetic is the same fixed expression as the tiled kernels (bit-identical
// results); the new values are rounded to the storage type once, at the
// store.
#pragma once

#include <algorithm>

#include "wfa_sweep.cuh"

namespace wfa {

// Ask L2 for the line holding p (no register, no completion to wait for).
__device__ __forceinline__ void prefetch_l2(const void* p) {
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}
// The same under a predicate: no branch, so the warps that do not ask pay one
// instruction and no reconvergence.
__device__ __forceinline__ void prefetch_l2_if(const void* p, bool pred) {
    asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %1, 0;\n\t@q prefetch.global.L2 [%0];\n\t}" ::"l"(p),
                 "r"((int)pred));
}

// 4 consecutive stored values -> 4 floats, and one value. COH = false reads
// through the read-only (non-coherent) path; COH = true bypasses L1 (ld.cg),
// for fields that other blocks rewrite during the same launch.
template <typename S, bool COH>
__device__ __forceinline__ void ldg4(const S* p, float v[4]);
template <>
__device__ __forceinline__ void ldg4<float, false>(const float* p, float v[4]) {
    const float4 q = __ldg(reinterpret_cast<const float4*>(p));
    v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
}
template <>
__device__ __forceinline__ void ldg4<float, true>(const float* p, float v[4]) {
    const float4 q = __ldcg(reinterpret_cast<const float4*>(p));
    v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
}
__device__ __forceinline__ void unpack_bf16x4(uint2 q, float v[4]) {
    const __nv_bfloat162 a = *reinterpret_cast<const __nv_bfloat162*>(&q.x);
    const __nv_bfloat162 b = *reinterpret_cast<const __nv_bfloat162*>(&q.y);
    v[0] = __low2float(a); v[1] = __high2float(a); v[2] = __low2float(b); v[3] = __high2float(b);
}
template <>
__device__ __forceinline__ void ldg4<__nv_bfloat16, false>(const __nv_bfloat16* p, float v[4]) {
    unpack_bf16x4(__ldg(reinterpret_cast<const uint2*>(p)), v);
}
template <>
__device__ __forceinline__ void ldg4<__nv_bfloat16, true>(const __nv_bfloat16* p, float v[4]) {
    unpack_bf16x4(__ldcg(reinterpret_cast<const uint2*>(p)), v);
}
template <typename S, bool COH>
__device__ __forceinline__ float ldg1(const S* p);
template <>
__device__ __forceinline__ float ldg1<float, false>(const float* p) {
    return __ldg(p);
}
template <>
__device__ __forceinline__ float ldg1<float, true>(const float* p) {
    return __ldcg(p);
}
template <>
__device__ __forceinline__ float ldg1<__nv_bfloat16, true>(const __nv_bfloat16* p) {
    const unsigned short b = __ldcg(reinterpret_cast<const unsigned short*>(p));
    return __uint_as_float((unsigned)b << 16);
}
template <>
__device__ __forceinline__ float ldg1<__nv_bfloat16, false>(const __nv_bfloat16* p) {
    return __bfloat162float(*p);
}

// One cell with uniform k: boundary faces, held layers and the zero-flux self
// term chosen by select, in the order and form of boundary_update, so the
// value is bitwise that of every other kernel (an interior cell reduces to
// the interior expression: w_in weights, neighbour values, no self term).
__device__ __forceinline__ float uniform_cell(const SweepCoef& c, float tc, float txm, float txp, float tym,
                                              float typ, float tzm, float tzp, int x, int y, int z) {
    const bool e0 = !c.periodic[0] && x == 0, e1 = !c.periodic[0] && x == c.n[0] - 1;
    const bool e2 = !c.periodic[1] && y == 0, e3 = !c.periodic[1] && y == c.n[1] - 1;
    const bool e4 = !c.periodic[2] && !c.ext[4] && z == 0, e5 = !c.periodic[2] && !c.ext[5] && z == c.n[2] - 1;
    auto tface = [&](int f) { return c.bkind[f] == WFA_BC_DIRICHLET ? c.tb[f] : 0.0f; };
    const float t0 = e0 ? tface(0) : txm, t1 = e1 ? tface(1) : txp;
    const float t2 = e2 ? tface(2) : tym, t3 = e3 ? tface(3) : typ;
    const float t4 = e4 ? tface(4) : tzm, t5 = e5 ? tface(5) : tzp;
    const float w0 = e0 ? c.w_bd[0] : c.w_in[0], w1 = e1 ? c.w_bd[1] : c.w_in[1];
    const float w2 = e2 ? c.w_bd[2] : c.w_in[2], w3 = e3 ? c.w_bd[3] : c.w_in[3];
    const float w4 = e4 ? c.w_bd[4] : c.w_in[4], w5 = e5 ? c.w_bd[5] : c.w_in[5];
    float s = 0.0f;
    if (c.any_self) {   // self_term: the same sum, a zero added where a face is not on the wall
        s = __fadd_rn(s, x == 0 ? c.s_lo[0] : 0.0f);
        s = __fadd_rn(s, x == c.n[0] - 1 ? c.s_hi[0] : 0.0f);
        s = __fadd_rn(s, y == 0 ? c.s_lo[1] : 0.0f);
        s = __fadd_rn(s, y == c.n[1] - 1 ? c.s_hi[1] : 0.0f);
        s = __fadd_rn(s, z == 0 ? c.s_lo[2] : 0.0f);
        s = __fadd_rn(s, z == c.n[2] - 1 ? c.s_hi[2] : 0.0f);
    }
    const float v = finish_update(tc, flux_sum(tc, t0, t1, t2, t3, t4, t5, w0, w1, w2, w3, w4, w5), s);
    return is_held(c, x, y, z) ? tc : v;
}

// Interior cell (no face on the boundary, not held, no self term).
__device__ __forceinline__ float uniform_inner(const SweepCoef& c, float tc, float txm, float txp, float tym,
                                               float typ, float tzm, float tzp) {
    return __fadd_rn(tc, flux_sum(tc, txm, txp, tym, typ, tzm, tzp, c.w_in[0], c.w_in[1], c.w_in[2], c.w_in[3],
                                  c.w_in[4], c.w_in[5]));
}

// Outside the domain on a non-periodic axis (a ghost or padding cell).
__device__ __forceinline__ bool outside_np(const SweepCoef& c, int x, int y, int z) {
    return (!c.periodic[0] && (x < 0 || x >= c.n[0])) || (!c.periodic[1] && (y < 0 || y >= c.n[1])) ||
           (!c.periodic[2] && (z < 0 || z >= c.n[2]));
}

// V consecutive stored values <-> V floats (V = 4, 8 or 16; 8 fp32 values
// are two 128-bit accesses, 8 bf16 values one).
template <typename S, bool COH, int V>
__device__ __forceinline__ void ldgv(const S* p, float v[V]) {
#pragma unroll
    for (int i = 0; i < V; i += 4) ldg4<S, COH>(p + i, v + i);
}
template <>
__device__ __forceinline__ void ldgv<__nv_bfloat16, false, 8>(const __nv_bfloat16* p, float v[8]) {
    const uint4 q = __ldg(reinterpret_cast<const uint4*>(p));
    unpack_bf16x4(make_uint2(q.x, q.y), v);
    unpack_bf16x4(make_uint2(q.z, q.w), v + 4);
}
template <>
__device__ __forceinline__ void ldgv<__nv_bfloat16, true, 8>(const __nv_bfloat16* p, float v[8]) {
    const uint4 q = __ldcg(reinterpret_cast<const uint4*>(p));
    unpack_bf16x4(make_uint2(q.x, q.y), v);
    unpack_bf16x4(make_uint2(q.z, q.w), v + 4);
}
template <>
__device__ __forceinline__ void ldgv<__nv_bfloat16, false, 16>(const __nv_bfloat16* p, float v[16]) {
    ldgv<__nv_bfloat16, false, 8>(p, v);
    ldgv<__nv_bfloat16, false, 8>(p + 8, v + 8);
}
template <>
__device__ __forceinline__ void ldgv<__nv_bfloat16, true, 16>(const __nv_bfloat16* p, float v[16]) {
    ldgv<__nv_bfloat16, true, 8>(p, v);
    ldgv<__nv_bfloat16, true, 8>(p + 8, v + 8);
}
template <typename S, int V>
__device__ __forceinline__ void stv(S* p, const float v[V]) {
#pragma unroll
    for (int i = 0; i < V; i += 4) Vec4<S>::store(p + i, v + i);
}
template <>
__device__ __forceinline__ void stv<__nv_bfloat16, 8>(__nv_bfloat16* p, const float v[8]) {
    uint4 q;
    __nv_bfloat162 h[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) h[i] = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
    q.x = *reinterpret_cast<uint32_t*>(&h[0]);
    q.y = *reinterpret_cast<uint32_t*>(&h[1]);
    q.z = *reinterpret_cast<uint32_t*>(&h[2]);
    q.w = *reinterpret_cast<uint32_t*>(&h[3]);
    *reinterpret_cast<uint4*>(p) = q;
}
template <>
__device__ __forceinline__ void stv<__nv_bfloat16, 16>(__nv_bfloat16* p, const float v[16]) {
    stv<__nv_bfloat16, 8>(p, v);
    stv<__nv_bfloat16, 8>(p + 8, v + 8);
}

// V new values rounded to S once (bf16: packed in pairs), then stored at one
// or more places; store_if is a predicated vector store (no branch). Every
// address is aligned to V elements.
__device__ __forceinline__ void st4_if(float* p, float a, float b, float c, float d, bool pred) {
    asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %5, 0;\n\t@q st.global.v4.f32 [%0], {%1, %2, %3, %4};\n\t}" ::"l"(p),
                 "f"(a), "f"(b), "f"(c), "f"(d), "r"((int)pred));
}
__device__ __forceinline__ void st4_if(void* p, unsigned a, unsigned b, unsigned c, unsigned d, bool pred) {
    asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %5, 0;\n\t@q st.global.v4.b32 [%0], {%1, %2, %3, %4};\n\t}" ::"l"(p),
                 "r"(a), "r"(b), "r"(c), "r"(d), "r"((int)pred));
}
__device__ __forceinline__ void st2_if(void* p, unsigned a, unsigned b, bool pred) {
    asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %3, 0;\n\t@q st.global.v2.b32 [%0], {%1, %2};\n\t}" ::"l"(p),
                 "r"(a), "r"(b), "r"((int)pred));
}
__device__ __forceinline__ unsigned pack_bf16x2(float a, float b) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<const unsigned*>(&h);
}
template <typename S, int V> struct StoreVec;
template <int V> struct StoreVec<float, V> {
    float v[V];
    __device__ __forceinline__ explicit StoreVec(const float* o) {
#pragma unroll
        for (int i = 0; i < V; ++i) v[i] = o[i];
    }
    __device__ __forceinline__ void store(float* p) const { stv<float, V>(p, v); }
    __device__ __forceinline__ void store_if(float* p, bool pred) const {
#pragma unroll
        for (int i = 0; i < V; i += 4) st4_if(p + i, v[i], v[i + 1], v[i + 2], v[i + 3], pred);
    }
};
template <int V> struct StoreVec<__nv_bfloat16, V> {
    unsigned u[V / 2];
    __device__ __forceinline__ explicit StoreVec(const float* o) {
#pragma unroll
        for (int i = 0; i < V / 2; ++i) u[i] = pack_bf16x2(o[2 * i], o[2 * i + 1]);
    }
    __device__ __forceinline__ void store(__nv_bfloat16* p) const {
        if constexpr (V >= 8) {
#pragma unroll
            for (int i = 0; i < V / 2; i += 4)
                *reinterpret_cast<uint4*>(p + 2 * i) = make_uint4(u[i], u[i + 1], u[i + 2], u[i + 3]);
        } else {
            *reinterpret_cast<uint2*>(p) = make_uint2(u[0], u[1]);
        }
    }
    __device__ __forceinline__ void store_if(__nv_bfloat16* p, bool pred) const {
        if constexpr (V >= 8) {
#pragma unroll
            for (int i = 0; i < V / 2; i += 4) st4_if(p + 2 * i, u[i], u[i + 1], u[i + 2], u[i + 3], pred);
        } else {
            st2_if(p, u[0], u[1], pred);
        }
    }
};

// x / y neighbours of one plane for one thread: the V cells below and above in
// y and the x neighbours of the row ends; same for 1/k. They belong to other
// threads' columns, so they come from L1 (or L2).
template <typename S, bool KVAR, bool COH, int V = 4>
struct ColNb {
    float ty_m[V], ty_p[V], tx_m, tx_p;
    float ry_m[V], ry_p[V], rx_m, rx_p;
    // tp / rp: this thread's first cell of the plane (T, 1/k); syt / syr: one row in bytes
    __device__ __forceinline__ void load(const char* tp, const char* rp, long long syt, long long syr) {
        ldgv<S, COH, V>(reinterpret_cast<const S*>(tp - syt), ty_m);
        ldgv<S, COH, V>(reinterpret_cast<const S*>(tp + syt), ty_p);
        tx_m = ldg1<S, COH>(reinterpret_cast<const S*>(tp) - 1);
        tx_p = ldg1<S, COH>(reinterpret_cast<const S*>(tp) + V);
        if (KVAR) {   // 1/k never changes during a launch: read-only path
            ldgv<float, false, V>(reinterpret_cast<const float*>(rp - syr), ry_m);
            ldgv<float, false, V>(reinterpret_cast<const float*>(rp + syr), ry_p);
            rx_m = __ldg(reinterpret_cast<const float*>(rp) - 1);
            rx_p = __ldg(reinterpret_cast<const float*>(rp) + V);
        }
    }
};

// Latency hiding: the kernel keeps few live values so that several blocks fit
// on an SM, the z extent is cut into short chunks so that thousands of blocks
// stream the grid at once, and each thread asks L2 for plane z + 3
// (prefetch.global.L2, no register cost) while it loads plane z + 1, so most
// plane loads hit L2 (measured at 512^3: +11% with per-cell k, +7% with
// uniform k). Register-level prefetch was slower: it costs the occupancy.
template <bool KVAR, bool INL = false, int ES = 4, int V = 4> struct ColOcc {
    static constexpr int blocks = V == 16 ? 3 : V == 8 ? (KVAR ? 2 : 4) : INL ? (KVAR ? 3 : 4) : (KVAR ? 4 : 6);
    // measured: uniform k prefers the z loop unrolled twice (fp32 with 4
    // cells a thread, bf16 with 8), per-cell k not
    static constexpr int unroll = KVAR ? 1 : (V == 4 && ES == 4) || (V == 8 && ES == 2) ? 2 : 1;
};

// How a column pass treats boundary cells and periodic copies.
enum ColMode {
    COL_MAIN = 0,    // every cell takes the interior formula; boundary cells and periodic copies
                     // are rewritten afterwards (the batched sweep's boundary and copy launches)
    COL_INPLACE = 1, // boundary cells in place, every periodic copy of a written cell stored (full halo)
    COL_THIN = 2     // every cell takes the interior formula, and one layer of periodic copies
                     // (no corners: all that a one-step pass reads) is stored in the pass; the
                     // boundary cells, if the ghost layers do not hold the faces, follow in a
                     // short launch (boundary_fix) that stores their copies too
};

// One thread's work: cells (gx .. gx+V-1, gy) of planes [z0, z1), one step,
// from tin into tout. Shared by the single-grid kernel and the batched one.
// MODE: see ColMode. GHOST: the caller guarantees c.halo_bc (the ghost layers
// encode every boundary face), so the boundary path is not compiled at all.
// DIR = +1 marches planes z0 .. z1-1 upwards, DIR = -1 marches z1-1 .. z0
// downwards. The single-grid kernel alternates the direction between
// neighbouring z chunks, so that the two chunks that share a boundary plane
// read it at about the same time (both at their start, or both at their end)
// and the second read hits L2 instead of DRAM. The march direction does not
// change a cell's value: the z faces are symmetric bit for bit and every
// cell takes the same operands in the same order.
template <typename S, bool KVAR, bool ADV, bool COH, int UNROLL, ColMode MODE, bool PF = false, bool GHOST = false,
          int DIR = 1, int V = 4, bool TW = true, bool HELD = false>
__device__ __forceinline__ void col_run(const SweepCoef& c, const S* __restrict__ tin, S* __restrict__ tout,
                                        const float* __restrict__ rk, int* status, int gx, int gy, int z0, int z1) {
    static_assert(V == 4 || V == 8 || V == 16, "cells per thread");
    const long long sy = c.sy, sz = c.sz;
    const long long col = (long long)gy * sy + gx;
    // plane p of T is tcol + p * sz (-1 <= p <= nz, inside the halo)
    const S* __restrict__ tcol = tin + col;
    const float* __restrict__ rcol = KVAR ? rk + col : nullptr;

    const bool perx = c.periodic[0], pery = c.periodic[1], perz = c.periodic[2];
    const bool bym = !pery && gy == 0, byp = !pery && gy == c.n[1] - 1;
    const bool full_x = gx + V - 1 < c.n[0];   // every cell of the group lies in the domain
    const bool edge_x = !perx && (gx == 0 || gx + V - 1 >= c.n[0] - 1);
    const bool inner_xy = !edge_x && !bym && !byp && full_x;
    const bool plain_xy = full_x && !(perx && (gx < HALO || gx + V - 1 >= c.n[0] - HALO)) &&
                          !(pery && (gy < HALO || gy >= c.n[1] - HALO));
    // threads per 128-byte line: one of them asks L2 for the line ahead
    constexpr int LINE_T = 128 / (V * (int)sizeof(S)) > 0 ? 128 / (V * (int)sizeof(S)) : 1;

    // register queue: tm = the plane already passed (z - DIR), tc = plane z,
    // tz = the plane ahead (z + DIR), loaded at plane z; gzm = the face
    // between the passed plane and plane z (per-cell k)
    const int zs = DIR > 0 ? z0 : z1 - 1;          // first plane of the march
    const long long dsz = DIR > 0 ? sz : -sz;      // one plane ahead
    float tm[V], tc[V], rc[V], gzm[V];
    ldgv<S, COH, V>(tcol + (long long)(zs - DIR) * sz, tm);
    ldgv<S, COH, V>(tcol + (long long)zs * sz, tc);
    if (KVAR) {
        float rb[V];
        ldgv<float, false, V>(rcol + (long long)(zs - DIR) * sz, rb);
        ldgv<float, false, V>(rcol + (long long)zs * sz, rc);
#pragma unroll
        for (int i = 0; i < V; ++i) gzm[i] = face_r(rb[i], rc[i], c.tcd[2]);
    }

    // Addresses in the loop: the start of each padded array and this
    // thread's byte offset from it (T and the new field share the layout, so
    // one offset serves both); every plane forms a pointer to the thread's
    // cells and addresses its loads and stores by constant byte offsets from
    // it (measured as fast as 32-bit offsets from the array's start, and 10%
    // faster with per-cell k than forming every address from the start).
    using OT = unsigned long long;
    const long long org = HALO * sz + HALO * sy + HALO;   // elements before the domain origin
    const char* const tB = reinterpret_cast<const char*>(tin - org);
    char* const oB = reinterpret_cast<char*>(tout - org);
    const char* const rB = KVAR ? reinterpret_cast<const char*>(rk - org) : nullptr;
    const long long cell0 = org + col + (long long)zs * sz;   // this thread's first cell, plane zs
    OT to = (OT)(cell0 * (long long)sizeof(S));
    OT ro = KVAR ? (OT)(cell0 * 4) : (OT)0;
    const OT dzt = (OT)(dsz * (long long)sizeof(S)), dzr = (OT)(dsz * 4);
    const OT syt = (OT)(sy * (long long)sizeof(S)), syr = (OT)(sy * 4);
    const int len = z1 - z0;
    const bool pf_lead = PF && (threadIdx.x & (LINE_T - 1)) == 0;
    // THIN: the periodic copies this thread stores at every plane. With
    // n_x a multiple of V the row's first and last vectors are stored whole
    // (shifted by -+n_x into the halo: every shifted cell is a copy);
    // otherwise cell by cell.
    const bool xvec = c.n[0] % V == 0;
    const bool xt_first = MODE == COL_THIN && TW && perx && gx == 0;
    const int xlast = c.n[0] - 1 - gx;   // index of cell n_x - 1 in this thread's vector (if 0 <= xlast < V)
    const bool xt_last = MODE == COL_THIN && TW && perx && xlast >= 0 && xlast < V;
    const long long yoff = MODE == COL_THIN && TW && pery ? (gy == 0 ? c.n[1] * sy : gy == c.n[1] - 1 ? -c.n[1] * sy : 0) : 0;
    // THIN with HELD (some face holds its cell layer): those cells keep
    // their value in the pass itself, so those faces need no boundary launch
    const bool held_y = HELD && ((c.held[2] && gy == 0) || (c.held[3] && gy == c.n[1] - 1));
    const OT yoffb = (OT)(yoff * (long long)sizeof(S)), xoffb = (OT)((long long)c.n[0] * (long long)sizeof(S));

#pragma unroll(UNROLL)
    for (int s = 0; s < len; ++s) {
        const int z = DIR > 0 ? z0 + s : z1 - 1 - s;
        // this plane's pointers to the thread's cells
        const char* const tP = tB + to;
        const char* const rP = KVAR ? rB + ro : nullptr;
        char* const oP = oB + to;
        float tz[V], rz[V];
        ldgv<S, COH, V>(reinterpret_cast<const S*>(tP + dzt), tz);   // own cells, plane z + DIR
        // one thread per 128-byte line asks L2 for plane z + 3 DIR, as long as
        // the chunk still needs it (the last plane read is z1 going up, z0 - 1
        // going down); the plane after that belongs to the next chunk
        if (PF) {
            prefetch_l2_if(tP + 3 * dzt, pf_lead && s + 3 <= len);
            if (KVAR) prefetch_l2_if(rP + 3 * dzr, pf_lead && s + 3 <= len);
        }
        if (KVAR) ldgv<float, false, V>(reinterpret_cast<const float*>(rP + dzr), rz);
        ColNb<S, KVAR, COH, V> nb;                       // x / y neighbours, plane z
        nb.load(tP, rP, (long long)syt, (long long)syr);
        S* const op = reinterpret_cast<S*>(oP);          // this thread's cells at plane z

        const bool bzm = !perz && !c.ext[4] && z == 0, bzp = !perz && !c.ext[5] && z == c.n[2] - 1;
        // GHOST (c.halo_bc known at compile time) or c.halo_bc: the ghost layers hold the faces
        const bool fast = GHOST || c.halo_bc || (inner_xy && !bzm && !bzp);
        float xf[V + 1], gzp[V];
        if (KVAR) {
            xf[0] = face_r(nb.rx_m, rc[0], c.tcd[0]);
#pragma unroll
            for (int i = 0; i < V - 1; ++i) xf[i + 1] = face_r(rc[i], rc[i + 1], c.tcd[0]);
            xf[V] = face_r(rc[V - 1], nb.rx_p, c.tcd[0]);
#pragma unroll
            for (int i = 0; i < V; ++i) gzp[i] = face_r(rc[i], rz[i], c.tcd[2]);
        }
        // face weights of the V cells (same values on every path below)
        float w[V][6];
#pragma unroll
        for (int i = 0; i < V; ++i) {
            if (KVAR) {
                w[i][0] = xf[i];
                w[i][1] = xf[i + 1];
                w[i][2] = face_r(nb.ry_m[i], rc[i], c.tcd[1]);
                w[i][3] = face_r(rc[i], nb.ry_p[i], c.tcd[1]);
                w[i][4] = DIR > 0 ? gzm[i] : gzp[i];   // the -z face
                w[i][5] = DIR > 0 ? gzp[i] : gzm[i];   // the +z face
                if (ADV) {
#pragma unroll
                    for (int f = 0; f < 6; ++f) w[i][f] = __fadd_rn(w[i][f], c.adv[f]);
                }
            } else {
#pragma unroll
                for (int f = 0; f < 6; ++f) w[i][f] = c.w_in[f];
            }
        }
        // the new values in fp32; every store rounds them to S once
        float out[V];
        if (MODE == COL_MAIN || MODE == COL_THIN || fast) {   // interior formula (see ColMode)
#pragma unroll
            for (int i = 0; i < V; ++i) {
                const float txm = i == 0 ? nb.tx_m : tc[i - 1];
                const float txp = i == V - 1 ? nb.tx_p : tc[i + 1];
                out[i] = __fadd_rn(tc[i], flux_sum(tc[i], txm, txp, nb.ty_m[i], nb.ty_p[i], DIR > 0 ? tm[i] : tz[i],
                                                   DIR > 0 ? tz[i] : tm[i], w[i][0], w[i][1], w[i][2], w[i][3],
                                                   w[i][4], w[i][5]));
            }
        } else {
#pragma unroll
            for (int i = 0; i < V; ++i) {
                const float txm = i == 0 ? nb.tx_m : tc[i - 1];
                const float txp = i == V - 1 ? nb.tx_p : tc[i + 1];
                const float tzm = DIR > 0 ? tm[i] : tz[i], tzp = DIR > 0 ? tz[i] : tm[i];
                const bool edge_cell = bym || byp || bzm || bzp || (!perx && (gx + i == 0 || gx + i == c.n[0] - 1));
                if (!KVAR) {   // uniform k: the boundary formula by select, inline
                    out[i] = uniform_cell(c, tc[i], txm, txp, nb.ty_m[i], nb.ty_p[i], tzm, tzp, gx + i, gy, z);
                } else if (!edge_cell) {
                    out[i] = __fadd_rn(tc[i], flux_sum(tc[i], txm, txp, nb.ty_m[i], nb.ty_p[i], tzm, tzp, w[i][0],
                                                       w[i][1], w[i][2], w[i][3], w[i][4], w[i][5]));
                } else {
                    out[i] = boundary_update<KVAR>(&c, tc[i], txm, txp, nb.ty_m[i], nb.ty_p[i], tzm, tzp, w[i][0],
                                                   w[i][1], w[i][2], w[i][3], w[i][4], w[i][5], KVAR ? rc[i] : 0.0f,
                                                   gx + i, gy, z);
                }
            }
        }
        if (MODE == COL_THIN) {
            if (HELD) {
                const bool held_yz = held_y || (c.held[4] && z == 0) || (c.held[5] && z == c.n[2] - 1);
#pragma unroll
                for (int i = 0; i < V; ++i)
                    if (held_yz || (c.held[0] && gx + i == 0) || (c.held[1] && gx + i == c.n[0] - 1)) out[i] = tc[i];
            }
            // the cells (masked at the x end: the halo there holds the x copies),
            // then one layer of periodic copies for the next one-step pass
            const StoreVec<S, V> sv(out);
            const long long zoff = TW && perz ? (z == 0 ? c.n[2] * sz : z == c.n[2] - 1 ? -c.n[2] * sz : 0) : 0;
            S* const oy = reinterpret_cast<S*>(oP + yoffb);
            S* const oz = reinterpret_cast<S*>(oP + (OT)(zoff * (long long)sizeof(S)));
            if (xvec) {
                // n_x a multiple of V (the same for every thread): every vector
                // lies in the domain, and the row ends store theirs shifted
                sv.store(op);
                if (TW && pery) sv.store_if(oy, yoff != 0);
                if (TW && perz) sv.store_if(oz, zoff != 0);
                if (TW && perx) {
                    sv.store_if(reinterpret_cast<S*>(oP + xoffb), xt_first);
                    sv.store_if(reinterpret_cast<S*>(oP - xoffb), xt_last);
                }
            } else {
                if (full_x) {
                    sv.store(op);
                    if (TW && pery) sv.store_if(oy, yoff != 0);
                    if (TW && perz) sv.store_if(oz, zoff != 0);
                } else {
#pragma unroll
                    for (int i = 0; i < V; ++i)
                        if (gx + i < c.n[0]) {
                            op[i] = from_f32<S>(out[i]);
                            if (TW && yoff != 0) oy[i] = from_f32<S>(out[i]);
                            if (TW && zoff != 0) oz[i] = from_f32<S>(out[i]);
                        }
                }
                if (TW && perx) {
                    if (xt_first) op[c.n[0]] = from_f32<S>(out[0]);
                    if (xt_last) {
#pragma unroll
                        for (int i = 0; i < V; ++i)
                            if (i == xlast) op[i - c.n[0]] = from_f32<S>(out[i]);   // cell n - 1 at x = -1
                    }
                }
            }
        } else {
            const bool plain = plain_xy && !(perz && (z < HALO || z >= c.n[2] - HALO));
            // partial vector at the x end with per-cell k: the halo keeps its ghost
            // values (uniform k never reads them, and the unmasked store is faster)
            if (MODE == COL_MAIN && KVAR && !full_x) {
#pragma unroll
                for (int i = 0; i < V; ++i)
                    if (gx + i < c.n[0]) op[i] = from_f32<S>(out[i]);
            } else if (MODE == COL_MAIN || plain) {
                stv<S, V>(op, out);
            } else if (!perx && !pery && !perz) {   // the x end of a row, no copies to store
#pragma unroll
                for (int i = 0; i < V; ++i)
                    if (gx + i < c.n[0]) op[i] = from_f32<S>(out[i]);
            } else {
#pragma unroll
                for (int i = 0; i < V; ++i)
                    if (gx + i < c.n[0]) store_twins_out_of_line<S>(tout, &c, gx + i, gy, z, out[i], status);
            }
        }
#pragma unroll
        for (int i = 0; i < V; ++i) {
            tm[i] = tc[i];
            tc[i] = tz[i];
            if (KVAR) {
                rc[i] = rz[i];
                gzm[i] = gzp[i];
            }
        }
        to += dzt;
        if (KVAR) ro += dzr;
    }
}

// ADV: per-cell k with a nonzero upwind weight on some face (uniform k folds
// the upwind weights into its constants and never needs it).
// INL: boundary cells and every periodic copy in place (variant 5, one
// launch per pass); otherwise the thin pass (variant 3 with V = 4, variant 6
// with V = 8, or V = 16 for bf16 with uniform k): interior formula and one
// layer of periodic copies, then
// boundary_fix where the ghost layers do not hold the faces.
// TW: some axis is periodic (the thin pass stores its one layer of copies;
// without a periodic axis that code is not compiled).
template <typename S, bool KVAR, bool ADV, bool INL, int V = 4, bool TW = true, bool HELD = false>
__global__ void __launch_bounds__(256, (ColOcc<KVAR, INL, sizeof(S), V>::blocks))
    sweep_col(const __grid_constant__ SweepArgs a) {
    const SweepCoef& c = a.c;
    const int gx = (blockIdx.x * blockDim.x + threadIdx.x) * V;
    const int gy = blockIdx.y * blockDim.y + threadIdx.y;
    if (gx >= c.n[0] || gy >= c.n[1]) return;
    const int z0 = blockIdx.z * a.zchunk;
    const int z1 = min(z0 + a.zchunk, c.n[2]);
    constexpr int U = ColOcc<KVAR, INL, sizeof(S), V>::unroll;
    constexpr ColMode MODE = INL ? COL_INPLACE : COL_THIN;
    if (blockIdx.z & 1)   // odd chunks march down: see col_run
        col_run<S, KVAR, ADV, false, U, MODE, true, false, -1, V, TW, HELD>(c, (const S*)a.tin, (S*)a.tout, a.rk,
                                                                           a.status, gx, gy, z0, z1);
    else
        col_run<S, KVAR, ADV, false, U, MODE, true, false, 1, V, TW, HELD>(c, (const S*)a.tin, (S*)a.tout, a.rk,
                                                                          a.status, gx, gy, z0, z1);
}

// Boundary cells (the outer layer on every non-periodic face): recomputed
// from the input field with the boundary conditions. blockIdx.y is the face
// (-x, +x, -y, +y, -z, +z; periodic axes have none); the threads of a block
// walk the face's plane x-fastest where the face has an x extent, so y and z
// faces are read and written in whole rows (cells on an edge are visited once
// per face and get the same value). Plane sizes fit 32-bit arithmetic (the
// caller checks).
// SKIPHELD: the main pass kept the cells of held faces (the thin column pass).
template <typename S, bool KVAR, bool SKIPHELD = false>
__global__ void __launch_bounds__(256) boundary_fix(const __grid_constant__ SweepArgs a) {
    const SweepCoef& c = a.c;
    const int f = blockIdx.y, ax = f >> 1;
    if (c.periodic[ax] || c.ext[f] || (SKIPHELD && c.held[f])) return;   // no boundary cells to fix on this face
    const int b = ax == 0 ? 1 : 0, d = ax == 2 ? 1 : 2;
    const unsigned nb = (unsigned)c.n[b], plane = nb * (unsigned)c.n[d];
    int pos[3];
    pos[ax] = (f & 1) ? c.n[ax] - 1 : 0;
    for (unsigned t = blockIdx.x * blockDim.x + threadIdx.x; t < plane; t += gridDim.x * blockDim.x) {
        pos[b] = (int)(t % nb);
        pos[d] = (int)(t / nb);
        const long long i = (long long)pos[2] * c.sz + (long long)pos[1] * c.sy + pos[0];
        const float v = general_cell<S, KVAR>(c, (const S*)a.tin, a.rk, i, pos[0], pos[1], pos[2], a.status);
        if (c.periodic[0] || c.periodic[1] || c.periodic[2])   // with its periodic copies
            store_with_twins<S>((S*)a.tout, c, pos[0], pos[1], pos[2], from_f32<S>(v), a.status);
        else
            ((S*)a.tout)[i] = from_f32<S>(v);
    }
}

// Periodic halo copies of one axis, over the full extent of the other two
// (their halos included, so corners are right when the axes go x, y, z).
// Element order: for x copies the 16 halo columns of a row are consecutive,
// for y and z copies whole padded rows are, so loads and stores coalesce.
// Totals fit 32-bit arithmetic (the caller checks).
template <typename S>
__global__ void __launch_bounds__(256) twin_copy(const __grid_constant__ SweepCoef c, S* origin, int ax) {
    const unsigned ex = c.n[0] + 2 * HALO, ey = c.n[1] + 2 * HALO, ez = c.n[2] + 2 * HALO;
    const unsigned total = 2u * HALO * (ax == 0 ? ey * ez : ex * (ax == 1 ? ez : ey));
    const int n = c.n[ax];
    for (unsigned t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
        int p[3], k;
        if (ax == 0) {            // (layer, y, z)
            k = (int)(t & (2 * HALO - 1));
            const unsigned r = t / (2 * HALO);
            p[1] = (int)(r % ey) - HALO;
            p[2] = (int)(r / ey) - HALO;
        } else if (ax == 1) {     // (x, layer, z)
            p[0] = (int)(t % ex) - HALO;
            const unsigned r = t / ex;
            k = (int)(r & (2 * HALO - 1));
            p[2] = (int)(r / (2 * HALO)) - HALO;
        } else {                  // (x, y, layer)
            p[0] = (int)(t % ex) - HALO;
            const unsigned r = t / ex;
            p[1] = (int)(r % ey) - HALO;
            k = (int)(r / ey);
        }
        const int dst = k < HALO ? k - HALO : n + (k - HALO);
        int src = dst % n;
        if (src < 0) src += n;
        p[ax] = dst;
        const long long od = (long long)p[2] * c.sz + (long long)p[1] * c.sy + p[0];
        p[ax] = src;
        const long long os = (long long)p[2] * c.sz + (long long)p[1] * c.sy + p[0];
        origin[od] = origin[os];
    }
}

// After a branch-free main pass: the boundary cells (unless the ghost layers
// hold the faces), then the periodic copies of the written buffer.
template <typename S, bool KVAR>
cudaError_t fix_and_twins(const SweepArgs& a, cudaStream_t st, int nsm) {
    long long plane = 0;   // the largest face
    for (int ax = 0; ax < 3; ++ax) {
        const int b = ax == 0 ? 1 : 0, d = ax == 2 ? 1 : 2;
        if (!a.c.periodic[ax]) plane = std::max(plane, (long long)a.c.n[b] * a.c.n[d]);
    }
    if (plane > 0 && !a.c.halo_bc) {
        const int nb = (int)std::min<long long>((plane + 255) / 256, (long long)nsm * 2);
        boundary_fix<S, KVAR><<<dim3(nb, 6), 256, 0, st>>>(a);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    for (int ax = 0; ax < 3; ++ax) {
        if (!a.c.periodic[ax]) continue;
        const int b = ax == 0 ? 1 : 0, d = ax == 2 ? 1 : 2;
        const long long total = 2LL * HALO * (a.c.n[b] + 2 * HALO) * (a.c.n[d] + 2 * HALO);
        const int nb = (int)std::min<long long>((total + 255) / 256, (long long)nsm * 8);
        twin_copy<S><<<nb, 256, 0, st>>>(a.c, (S*)a.tout, ax);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// One column pass (variant 3: V = 4, variant 6: V = 8, or 16 for bf16 with
// uniform k, both thin; variant 5: in place, V = 4): one launch.
template <typename S, bool KVAR, int V>
cudaError_t col_launch_v(const SweepArgs& a_in, cudaStream_t st, int nsm, const cudaEvent_t* ev, bool inl) {
    SweepArgs a = a_in;
    dim3 block(16, 16);
    const int gxb = (a.c.n[0] + 16 * V - 1) / (16 * V), gyb = (a.c.n[1] + 15) / 16;
    // z chunks of about 16 planes: many short columns stream the grid at once
    const long long cols = (long long)gxb * gyb,
                    resident = (long long)nsm * (inl ? ColOcc<KVAR, true>::blocks : ColOcc<KVAR, false, 4, V>::blocks);
    long long want = resident * 16;
    int nch = (int)std::max<long long>(1, want / cols);
    // chunks of at least 16 planes, unless that leaves SMs idle (small grids,
    // which sit in L2 anyway): then down to 2 planes
    int cap = std::max(1, a.c.n[2] / 16);
    if (cols * cap < resident) cap = std::max(1, a.c.n[2] / 2);
    nch = std::min(nch, cap);
    // a chunk length asked for by the caller (the autotuner's trials)
    if (a_in.zchunk > 0) nch = (a.c.n[2] + a_in.zchunk - 1) / a_in.zchunk;
    a.zchunk = (a.c.n[2] + nch - 1) / nch;
    nch = (a.c.n[2] + a.zchunk - 1) / a.zchunk;
    dim3 grid(gxb, gyb, nch);
    const bool adv = KVAR && (a.c.adv[0] != 0.0f || a.c.adv[1] != 0.0f || a.c.adv[2] != 0.0f ||
                              a.c.adv[3] != 0.0f || a.c.adv[4] != 0.0f || a.c.adv[5] != 0.0f);
    if (ev) cudaEventRecord(ev[0], st);
    if (inl) {
        if (adv) sweep_col<S, KVAR, true, true><<<grid, block, 0, st>>>(a);
        else sweep_col<S, KVAR, false, true><<<grid, block, 0, st>>>(a);
    } else if (a.c.held[0] || a.c.held[1] || a.c.held[2] || a.c.held[3] || a.c.held[4] || a.c.held[5]) {
        // held cell layers: kept in the pass (copies for any periodic axis too)
        if (adv) sweep_col<S, KVAR, true, false, V, true, true><<<grid, block, 0, st>>>(a);
        else sweep_col<S, KVAR, false, false, V, true, true><<<grid, block, 0, st>>>(a);
    } else if (a.c.periodic[0] || a.c.periodic[1] || a.c.periodic[2]) {
        if (adv) sweep_col<S, KVAR, true, false, V, true><<<grid, block, 0, st>>>(a);
        else sweep_col<S, KVAR, false, false, V, true><<<grid, block, 0, st>>>(a);
    } else {   // no periodic axis: no copies to store
        if (adv) sweep_col<S, KVAR, true, false, V, false><<<grid, block, 0, st>>>(a);
        else sweep_col<S, KVAR, false, false, V, false><<<grid, block, 0, st>>>(a);
    }
    if (ev) cudaEventRecord(ev[1], st);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || inl || a.c.halo_bc) return e;
    long long plane = 0;   // the largest face with boundary cells to fix (held faces are done)
    for (int ax = 0; ax < 3; ++ax) {
        const int b = ax == 0 ? 1 : 0, d = ax == 2 ? 1 : 2;
        if (!a.c.periodic[ax] && ((!a.c.ext[2 * ax] && !a.c.held[2 * ax]) || (!a.c.ext[2 * ax + 1] && !a.c.held[2 * ax + 1])))
            plane = std::max(plane, (long long)a.c.n[b] * a.c.n[d]);
    }
    if (plane == 0) return cudaSuccess;
    const int nb = (int)std::min<long long>((plane + 255) / 256, (long long)nsm * 2);
    boundary_fix<S, KVAR, true><<<dim3(nb, 6), 256, 0, st>>>(a);
    return cudaGetLastError();
}

template <typename S, bool KVAR>
cudaError_t col_launch(const SweepArgs& a, cudaStream_t st, int nsm, const cudaEvent_t* ev, bool inl, bool wide) {
    // bf16 with uniform k: 16 cells (32 bytes) a thread, measured 7% faster
    // than 8 at 3 blocks per SM (2 blocks: 7% slower than 8, 4: spills)
    if constexpr (sizeof(S) == 2 && !KVAR) {
        if (wide && !inl) return col_launch_v<S, KVAR, 16>(a, st, nsm, ev, false);
    }
    return wide && !inl ? col_launch_v<S, KVAR, 8>(a, st, nsm, ev, false) : col_launch_v<S, KVAR, 4>(a, st, nsm, ev, inl);
}

}  // namespace wfa
