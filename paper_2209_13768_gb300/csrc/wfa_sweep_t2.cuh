// sweep_t2<S>: two explicit steps per pass over the grid (Sec. 1.1.1,
// Eq. expl_form applied twice) with uniform conductivity: temporal blocking,
// so each pass reads and writes the field once for two steps (4 B per cell
// update in fp32 instead of 8; Eqs. A_eff and t_it_min with the field read
// once per two steps).
//
// A block owns a 64 x 16 output tile of one z chunk and marches z.
//  * Input planes arrive by TMA (cp.async.bulk.tensor.3d) into a ring of
//    T2_NS shared-memory slots, each an 80 x 20 box (x0 - 8 .. x0 + 72,
//    y0 - 2 .. y0 + 18), issued T2_NS - 3 planes ahead of use and completing
//    on one mbarrier per slot. No register holds a value in flight.
//  * Stage 1 (the first step) at plane q covers 72 x 18 cells (the tile, a
//    ring of one cell, and 3 more columns on each side so that every thread
//    owns 4 aligned cells): 18 x 18 threads, each 4 cells of one row, all
//    neighbours read from the input ring. It writes its plane into one of
//    four stage-1 slots.
//  * After one barrier per plane, stage 2 (the second step) updates plane
//    q - 1 of the tile from stage-1 planes q - 2, q - 1, q and stores it (a
//    cell near a periodic edge also stores its periodic copies). Four
//    stage-1 slots let a thread still in stage 2 overlap the next stage 1.
//  * Both stages evaluate the fixed per-cell expression of every other
//    kernel (the interior formula, or the select form with boundary faces,
//    held layers and zero-flux self terms when the tile touches a
//    non-periodic face) and round to the storage type after each step, so
//    the field after a pass is bitwise the field after two single steps.
// Bounded waits: a copy that does not land within about 2 s sets the grid's
// status word; the block drains the copies it issued (bounded too) and
// returns.
#pragma once

#include "wfa_sweep_col.cuh"

namespace wfa {

constexpr int T2_TX = 64, T2_TY = 16;               // output tile
constexpr int T2_EX = 80, T2_EY = 20;               // input box: x0 - 8 .. x0 + 72, y0 - 2 .. y0 + 18
constexpr int T2_GX = 18, T2_GY = 18;               // threads: 18 groups of 4 cells x 18 rows (stage 1)
constexpr int T2_NT = T2_GX * T2_GY;                // 324
constexpr int T2_SW = 72;                           // stage-1 row: x0 - 4 .. x0 + 68
constexpr int T2_SPLANE = T2_SW * T2_GY;            // stage-1 plane (floats)
constexpr int T2_NS = 6;                            // input slots (3 planes ahead of use)
constexpr int T2_BLOCKS = 3;                        // blocks per SM the register budget targets

template <typename S>
struct T2Cfg {
    static constexpr size_t SLOT = ((size_t)T2_EX * T2_EY * sizeof(S) + 127) / 128 * 128;
    static constexpr size_t IN_BYTES = SLOT * T2_NS;
    static constexpr size_t S1_BYTES = (size_t)4 * T2_SPLANE * sizeof(float);
    static constexpr size_t BAR_BYTES = 128;
    static constexpr size_t SMEM = 1024 + BAR_BYTES + IN_BYTES + S1_BYTES;   // 1024: alignment slack
    static constexpr uint32_t TX_BYTES = (uint32_t)(T2_EX * T2_EY * sizeof(S));
    static_assert(SLOT % 128 == 0 && IN_BYTES % 128 == 0, "TMA destinations 128-byte aligned");
    static_assert(SMEM <= 232448, "shared memory above the 227 KB a block may use");
};

// 4 consecutive values of a shared plane (stored type) -> floats.
template <typename S>
__device__ __forceinline__ void lds4(const S* p, float v[4]) {
    Vec4<S>::load(p, v);
}
template <typename S>
__device__ __forceinline__ float lds1(const S* p) {
    return to_f32<S>(*p);
}

template <typename S>
__device__ __forceinline__ void t2_issue(const CUtensorMap* map, unsigned char* ring, uint64_t* bars, int j,
                                         int x0, int y0, int zbase, const SweepCoef& c, int* status) {
    // box origin in padded coordinates: x0 - 8 + HALO = x0 (16-byte aligned:
    // x0 is a multiple of 64), y0 - 2 + HALO, plane zbase + j + HALO
    const int tx = x0 - 8 + HALO, ty = y0 - 2 + HALO, tz = zbase + j + HALO;
    if (!WFA_CHK(tx >= 0 && tx < c.px && ty >= 0 && ty < c.py && tz >= 0 && tz < c.pz, status, 17, tx, ty, tz, j))
        return;
    uint64_t* bar = &bars[j % T2_NS];
    mbar_expect_tx(bar, T2Cfg<S>::TX_BYTES);
    tma_load_3d(ring + (size_t)(j % T2_NS) * T2Cfg<S>::SLOT, map, bar, tx, ty, tz);
}

template <typename S>
__global__ void __launch_bounds__(T2_NT, T2_BLOCKS)
    sweep_t2(const __grid_constant__ CUtensorMap tmT, const __grid_constant__ SweepArgs a) {
    using Cfg = T2Cfg<S>;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    unsigned char* smem = smem_raw + ((1024u - (smem_addr(smem_raw) & 1023u)) & 1023u);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem);
    unsigned char* ring = smem + Cfg::BAR_BYTES;
    float* s1 = reinterpret_cast<float*>(smem + Cfg::BAR_BYTES + Cfg::IN_BYTES);

    const SweepCoef& c = a.c;
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * T2_GX + tx;
    const int x0 = blockIdx.x * T2_TX, y0 = blockIdx.y * T2_TY;
    const int z0 = blockIdx.z * a.zchunk, z1 = min(z0 + a.zchunk, c.n[2]);
    const int zbase = z0 - 2;                 // plane of ring index j = 0
    const int L = (z1 - z0) + 4;              // input planes z0 - 2 .. z1 + 1
    const bool perx = c.periodic[0], pery = c.periodic[1], perz = c.periodic[2];

    // stage-1 cells of this thread: x = x0 - 4 + 4 tx .. + 3, y = y0 - 1 + ty
    const int sx = x0 - 4 + 4 * tx, sy = y0 - 1 + ty;
    // the tile with its stage-1 ring lies at least one cell away from every
    // non-periodic face: the interior formula everywhere
    const bool plain_xy = (perx || (x0 - 4 >= 1 && x0 + 68 <= c.n[0] - 1)) &&
                          (pery || (y0 - 1 >= 1 && y0 + 17 <= c.n[1] - 1));
    // stage 2: output cells x = x0 + 4 (tx - 1) .., row y0 + ty - 1
    const bool act2 = tx >= 1 && tx <= 16 && ty >= 1 && ty <= 16;
    const int ox = x0 + 4 * (tx - 1), oy = y0 + ty - 1;
    const bool out_ok = act2 && ox < c.n[0] && oy < c.n[1];
    const bool out_full = out_ok && ox + 3 < c.n[0];
    const bool out_plain = out_full && !(perx && (ox < HALO || ox + 3 >= c.n[0] - HALO)) &&
                           !(pery && (oy < HALO || oy >= c.n[1] - HALO));
    S* __restrict__ tout = (S*)a.tout;

    if (tid == 0) {
        for (int b = 0; b < T2_NS; ++b) mbar_init(&bars[b], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        fence_proxy_async_smem();
        for (int j = 0; j < T2_NS && j < L; ++j) t2_issue<S>(&tmT, ring, bars, j, x0, y0, zbase, c, a.status);
    }
    __syncthreads();
    int issued = T2_NS < L ? T2_NS : L;   // thread 0: ring index one past the last plane issued

    bool failed = false;
    int waited = 0;                       // input planes 0 .. waited - 1 have landed
    for (int t = 0; t + 2 < L; ++t) {
        const int q = z0 - 1 + t;         // stage-1 plane; input planes t, t + 1, t + 2
        // wait for the planes stage 1 reads (each slot's phase: j / T2_NS)
        bool late = false;
        for (; waited <= t + 2; ++waited)
            late = late || !mbar_wait_bounded(&bars[waited % T2_NS], (uint32_t)(waited / T2_NS) & 1u);
        if (__syncthreads_or(late)) {
            failed = true;
            break;
        }
        const S* inm = reinterpret_cast<const S*>(ring + (size_t)(t % T2_NS) * Cfg::SLOT);
        const S* inc = reinterpret_cast<const S*>(ring + (size_t)((t + 1) % T2_NS) * Cfg::SLOT);
        const S* inp = reinterpret_cast<const S*>(ring + (size_t)((t + 2) % T2_NS) * Cfg::SLOT);
        // ---- stage 1 at plane q: row ty + 1 of the box, columns 4 + 4 tx ..
        {
            const int o = (ty + 1) * T2_EX + 4 + 4 * tx;
            float tc[4], ym[4], yp[4], zm[4], zp[4];
            lds4<S>(inc + o, tc);
            lds4<S>(inc + o - T2_EX, ym);
            lds4<S>(inc + o + T2_EX, yp);
            lds4<S>(inm + o, zm);
            lds4<S>(inp + o, zp);
            const float xm = lds1<S>(inc + o - 1), xp = lds1<S>(inc + o + 4);
            float sn[4];
            const bool plain = plain_xy && (perz || (q >= 1 && q <= c.n[2] - 2));
            if (plain) {
#pragma unroll
                for (int i = 0; i < 4; ++i)
                    sn[i] = storage_round<S>(uniform_inner(c, tc[i], i == 0 ? xm : tc[i - 1], i == 3 ? xp : tc[i + 1],
                                                           ym[i], yp[i], zm[i], zp[i]));
            } else {
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const float v = uniform_cell(c, tc[i], i == 0 ? xm : tc[i - 1], i == 3 ? xp : tc[i + 1], ym[i],
                                                 yp[i], zm[i], zp[i], sx + i, sy, q);
                    // a cell outside the domain on a non-periodic axis is never read
                    sn[i] = outside_np(c, sx + i, sy, q) ? tc[i] : storage_round<S>(v);
                }
            }
            Vec4<float>::store(s1 + (t & 3) * T2_SPLANE + ty * T2_SW + 4 * tx, sn);
        }
        __syncthreads();   // stage-1 plane q complete; input plane t is free
        if (tid == 0 && issued < L) {
            fence_proxy_async_smem();
            t2_issue<S>(&tmT, ring, bars, issued, x0, y0, zbase, c, a.status);
            ++issued;
        }
        // ---- stage 2 at plane p = q - 1 (stage-1 planes q - 2, q - 1, q)
        const int p = q - 1;
        if (t >= 2 && out_ok) {
            const float* sm = s1 + ((t - 2) & 3) * T2_SPLANE;
            const float* sc = s1 + ((t - 1) & 3) * T2_SPLANE;
            const float* sp = s1 + (t & 3) * T2_SPLANE;
            const int o = ty * T2_SW + 4 * tx;
            float tc[4], ym[4], yp[4], zm[4], zp[4], out[4];
            Vec4<float>::load(sc + o, tc);
            Vec4<float>::load(sc + o - T2_SW, ym);
            Vec4<float>::load(sc + o + T2_SW, yp);
            Vec4<float>::load(sm + o, zm);
            Vec4<float>::load(sp + o, zp);
            const float xm = sc[o - 1], xp = sc[o + 4];
            const bool plain = plain_xy && (perz || (p >= 1 && p <= c.n[2] - 2));
            if (plain) {
#pragma unroll
                for (int i = 0; i < 4; ++i)
                    out[i] = uniform_inner(c, tc[i], i == 0 ? xm : tc[i - 1], i == 3 ? xp : tc[i + 1], ym[i], yp[i],
                                           zm[i], zp[i]);
            } else {
#pragma unroll
                for (int i = 0; i < 4; ++i)
                    out[i] = uniform_cell(c, tc[i], i == 0 ? xm : tc[i - 1], i == 3 ? xp : tc[i + 1], ym[i], yp[i],
                                          zm[i], zp[i], ox + i, oy, p);
            }
            const bool plain_out = out_plain && !(perz && (p < HALO || p >= c.n[2] - HALO));
            if (plain_out) {
                Vec4<S>::store(tout + (long long)p * c.sz + (long long)oy * c.sy + ox, out);
            } else {
#pragma unroll
                for (int i = 0; i < 4; ++i)
                    if (ox + i < c.n[0]) store_twins_out_of_line<S>(tout, &c, ox + i, oy, p, out[i], a.status);
            }
        }
    }

    if (failed) {
        // drain: wait (bounded) for the copies this block issued and has not consumed
        if (tid == 0) {
            atomicExch(a.status, 1);
            for (int j = waited; j < issued; ++j) (void)mbar_wait_bounded(&bars[j % T2_NS], (uint32_t)(j / T2_NS) & 1u);
        }
        __syncthreads();
    }
}

// One pass of two steps: blocks over (x tiles, y tiles, z chunks); chunks of
// at least 32 planes (each recomputes two stage-1 planes), about four waves
// of blocks, or the length a caller asks for (a.zchunk > 0).
template <typename S>
cudaError_t t2_launch(const CUtensorMap* tmT, const SweepArgs& a_in, cudaStream_t st, int nsm, const cudaEvent_t* ev) {
    using Cfg = T2Cfg<S>;
    static bool attr_set = false;
    if (!attr_set) {
        const cudaError_t e = cudaFuncSetAttribute(sweep_t2<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cfg::SMEM);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    SweepArgs a = a_in;
    const int gxb = (a.c.n[0] + T2_TX - 1) / T2_TX, gyb = (a.c.n[1] + T2_TY - 1) / T2_TY;
    const long long tiles = (long long)gxb * gyb, resident = (long long)nsm * T2_BLOCKS;
    int nch = (int)std::max<long long>(1, (4 * resident + tiles / 2) / tiles);
    nch = std::min(nch, std::max(1, a.c.n[2] / 32));
    if (a_in.zchunk > 0) nch = (a.c.n[2] + a_in.zchunk - 1) / a_in.zchunk;
    a.zchunk = (a.c.n[2] + nch - 1) / nch;
    nch = (a.c.n[2] + a.zchunk - 1) / a.zchunk;
    if (ev) cudaEventRecord(ev[0], st);
    sweep_t2<S><<<dim3(gxb, gyb, nch), dim3(T2_GX, T2_GY), Cfg::SMEM, st>>>(*tmT, a);
    if (ev) cudaEventRecord(ev[1], st);
    return cudaGetLastError();
}

}  // namespace wfa
