// Sweep kernels: D explicit finite-volume steps per pass over the grid
// (arXiv 2209.13768, Sec. 1.1.1, Eq. expl_form in face-flux form).
//
// sweep_tb<S, KVAR, D, EX, EY, R> — the hot path.
//   * One thread block owns an extended EX x EY tile of (x, y) columns and
//     marches along z. Output is the inner (EX - 2 PX) x (EY - 2 D) tile; the
//     ring of PX >= D columns and D rows around it is recomputed redundantly
//     (overlapped tiling), so the D fused steps need no exchange with other
//     blocks.
//   * Input planes (and, for per-cell conductivity, k planes) arrive by TMA
//     (cp.async.bulk.tensor.3d) into a ring of shared-memory slots, P planes
//     ahead of use, each slot completing on its own mbarrier.
//   * Stage s (1..D) at iteration j updates plane j - s (a wavefront in z):
//     z-neighbours come from a per-thread register queue, x/y neighbours from
//     one shared-memory plane per stage written at the end of the previous
//     iteration.
//   * Every thread owns 4 consecutive x cells in R consecutive rows (128-bit
//     shared loads); face conductances between its own cells are computed
//     once and used by both cells, the z face is carried to the next plane.
//   * The last stage writes its plane straight to global memory (and to the
//     periodic twins in the halo).
// Bounded waits: a TMA that does not land within ~2 s sets the grid's status
// word, the block drains its copies (bounded again) and exits.
#pragma once

#include "wfa_internal.cuh"

namespace wfa {

struct SweepArgs {
    SweepCoef c;
    const void* tin;    // input field, domain origin
    void* tout;         // output field, domain origin
    const float* rk;    // reciprocal conductivity 1/k, domain origin (nullptr for uniform k)
    int tiles_x, tiles_y, zchunk, nzchunk, items;   // column kernels: zchunk > 0 on entry asks for
                                                     // chunks of that many planes (0: automatic)
    int* status;
};

// --------------------------------------------------------------- PTX helpers --
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Wait for one phase of an mbarrier; false after ~2 s without completion.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    while (!mbar_try_wait(bar, parity)) {
        if (global_ns() - t0 > 2000000000ull) return false;
    }
    return true;
}
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y,
                                            int z) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_addr(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_addr(bar))
        : "memory");
}

// 4 consecutive stored values <-> 4 floats.
template <typename S> struct Vec4;
template <> struct Vec4<float> {
    __device__ __forceinline__ static void load(const float* p, float v[4]) {
        const float4 q = *reinterpret_cast<const float4*>(p);
        v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
    }
    __device__ __forceinline__ static void store(float* p, const float v[4]) {
        *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
    }
};
template <> struct Vec4<__nv_bfloat16> {
    __device__ __forceinline__ static void load(const __nv_bfloat16* p, float v[4]) {
        const uint2 q = *reinterpret_cast<const uint2*>(p);
        const __nv_bfloat162 a = *reinterpret_cast<const __nv_bfloat162*>(&q.x);
        const __nv_bfloat162 b = *reinterpret_cast<const __nv_bfloat162*>(&q.y);
        v[0] = __low2float(a); v[1] = __high2float(a); v[2] = __low2float(b); v[3] = __high2float(b);
    }
    __device__ __forceinline__ static void store(__nv_bfloat16* p, const float v[4]) {
        __nv_bfloat162 a = __floats2bfloat162_rn(v[0], v[1]);
        __nv_bfloat162 b = __floats2bfloat162_rn(v[2], v[3]);
        uint2 q;
        q.x = *reinterpret_cast<uint32_t*>(&a);
        q.y = *reinterpret_cast<uint32_t*>(&b);
        *reinterpret_cast<uint2*>(p) = q;
    }
};

// ------------------------------------------------------------ one cell ------
// One cell with every boundary rule applied, neighbours read from the field
// (periodic neighbours from the halo twins). i is the cell's element offset.
template <typename S, bool KVAR>
__device__ __forceinline__ float general_cell(const SweepCoef& c, const S* __restrict__ in,
                                              const float* __restrict__ rk, long long i, int x, int y, int z,
                                              int* status) {
    const float tc = to_f32<S>(in[i]);
    if (is_held(c, x, y, z)) return tc;
    const float rc = KVAR ? rk[i] : 0.0f;
    const int pos[3] = {x, y, z};
    const long long st[3] = {1, c.sy, c.sz};
    float tn[6], w[6];
#pragma unroll
    for (int f = 0; f < 6; ++f) {
        const int ax = f >> 1, side = f & 1;
        const bool edge = side ? pos[ax] == c.n[ax] - 1 : pos[ax] == 0;
        tn[f] = 0.0f;
        w[f] = 0.0f;
        if (edge && !c.periodic[ax] && !c.ext[f]) {
            const bool dir = c.bkind[f] == WFA_BC_DIRICHLET;
            tn[f] = dir ? c.tb[f] : 0.0f;
            if (KVAR) w[f] = dir ? __fadd_rn(dirichlet_r(rc, c.tcd[ax]), c.adv[f]) : 0.0f;
            else w[f] = c.w_bd[f];
        } else {
            const long long j = i + (side ? st[ax] : -st[ax]);
            if (!WFA_CHK(j >= c.lo && j < c.hi, status, 20, x, y, z, f)) continue;
            tn[f] = to_f32<S>(in[j]);
            w[f] = KVAR ? __fadd_rn(face_r(rc, rk[j], c.tcd[ax]), c.adv[f]) : c.w_in[f];
        }
    }
    return finish_update(tc, flux_sum(tc, tn[0], tn[1], tn[2], tn[3], tn[4], tn[5], w[0], w[1], w[2], w[3], w[4], w[5]),
                         self_term(c, x, y, z));
}

// ------------------------------------------------------------ simple kernel --
// One thread per (x, y) column, neighbours read from global memory. One step.
// Used for grids too small for the tiled kernel's box and as a second,
// independent realisation of the same per-cell arithmetic.
template <typename S, bool KVAR>
__global__ void __launch_bounds__(256) sweep_simple(const __grid_constant__ SweepArgs a) {
    const SweepCoef& c = a.c;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= c.n[0] || y >= c.n[1]) return;
    const S* __restrict__ in = (const S*)a.tin;
    S* __restrict__ out = (S*)a.tout;
    const long long st[3] = {1, c.sy, c.sz};
    for (int z = 0; z < c.n[2]; ++z) {
        const long long i = z * c.sz + y * c.sy + x;
        const float v = general_cell<S, KVAR>(c, in, a.rk, i, x, y, z, a.status);
        store_with_twins<S>(out, c, x, y, z, from_f32<S>(v), a.status);
    }
}

// --------------------------------------------------------- tiled kernel ----
template <typename S, bool KVAR, int D, int EX, int EY, int R, int PF = 2>
struct TbCfg {
    static constexpr int VA = 16 / (int)sizeof(S);          // elements per 16 bytes (TMA x alignment)
    static constexpr int DEPTH = D;
    // x halo = the allocation's halo, so a box starts at allocated column x0;
    // with TX a multiple of 128 bytes every box row is line-aligned
    static constexpr int PX = HALO;
    static constexpr int TX = EX - 2 * PX;                  // output tile
    static constexpr int TY = EY - 2 * D;
    static constexpr int NTX = EX / 4, NTY = EY / R, NT = NTX * NTY;
    static constexpr int MINB = (NT <= 256 && D <= 2) ? 2 : 1;   // blocks per SM the register budget targets
    static constexpr int P = PF;                            // planes in flight ahead of use
    static constexpr int NS = P + 2;                        // input ring slots (= mbarriers)
    static constexpr int NK = KVAR ? D + P + 2 : 0;         // k ring slots
    static constexpr int PLANE = EX * EY;
    static constexpr size_t BAR_BYTES = 1024;   // mbarriers; keeps the ring 1024-byte aligned
    // slot strides padded to 128 bytes: every TMA destination stays 128-byte aligned
    static constexpr size_t SLOT_T = ((size_t)PLANE * sizeof(S) + 127) / 128 * 128;
    static constexpr size_t SLOT_K = ((size_t)PLANE * sizeof(float) + 127) / 128 * 128;
    static constexpr size_t RING_BYTES = (size_t)NS * SLOT_T;
    static constexpr size_t K_BYTES = (size_t)NK * SLOT_K;
    static constexpr size_t SBUF_BYTES = (size_t)(D > 1 ? D - 1 : 0) * PLANE * sizeof(float);
    static constexpr size_t SMEM = 1024 + BAR_BYTES + RING_BYTES + K_BYTES + SBUF_BYTES;
    static constexpr uint32_t TX_BYTES = (uint32_t)(PLANE * sizeof(S) + (KVAR ? PLANE * sizeof(float) : 0));
    static_assert(EX % 4 == 0 && EX % VA == 0 && EX <= 256 && EY <= 256, "TMA box");
    static_assert(EY % R == 0, "rows per thread");
    static_assert(TX > 0 && TY > 0, "tile too small for this depth");
    static_assert((TX * (int)sizeof(S)) % 128 == 0, "output tile width must be a multiple of 128 bytes");
    static_assert(NT <= 1024, "too many threads");
    static_assert(D >= 1 && D <= MAX_DEPTH && PX <= HALO, "depth");
    static_assert(SMEM <= 232448, "shared memory above the 227 KB a block may use");
    static_assert(SLOT_T % 128 == 0 && SLOT_K % 128 == 0 && BAR_BYTES % 1024 == 0 && RING_BYTES % 128 == 0,
                  "TMA destinations must be 128-byte aligned");
};

// Update of a cell that touches the domain boundary: the face values and
// coefficients computed for an interior face are replaced by the boundary
// condition's (Dirichlet: the face value with 2 k_C dt / h^2; zero-flux: no
// flux), held cells keep their value, and zero-flux faces with advection add
// the self term. Called only for boundary cells, so it stays out of line.
template <bool KVAR>
__device__ __noinline__ float boundary_update(const SweepCoef* cp, float tc, float txm, float txp, float tym,
                                              float typ, float tzm, float tzp, float wxm, float wxp, float wym,
                                              float wyp, float wzm, float wzp, float rc, int x, int y, int z) {
    const SweepCoef& c = *cp;
    if (is_held(c, x, y, z)) return tc;
    float t[6] = {txm, txp, tym, typ, tzm, tzp};
    float w[6] = {wxm, wxp, wym, wyp, wzm, wzp};
    const int pos[3] = {x, y, z};
#pragma unroll
    for (int f = 0; f < 6; ++f) {
        const int ax = f >> 1;
        const bool edge = (f & 1) ? pos[ax] == c.n[ax] - 1 : pos[ax] == 0;
        if (edge && !c.periodic[ax] && !c.ext[f]) {
            const bool dir = c.bkind[f] == WFA_BC_DIRICHLET;
            t[f] = dir ? c.tb[f] : 0.0f;
            if (KVAR) w[f] = dir ? __fadd_rn(dirichlet_r(rc, c.tcd[ax]), c.adv[f]) : 0.0f;
            else w[f] = c.w_bd[f];
        }
    }
    return finish_update(tc, flux_sum(tc, t[0], t[1], t[2], t[3], t[4], t[5], w[0], w[1], w[2], w[3], w[4], w[5]),
                         self_term(c, x, y, z));
}

template <typename S>
__device__ __noinline__ void store_twins_out_of_line(S* out, const SweepCoef* c, int x, int y, int z, float v,
                                                     int* st) {
    store_with_twins<S>(out, *c, x, y, z, from_f32<S>(v), st);
}

// Issue the TMA copies of input plane `plane` (and its k plane) into the ring
// slot of counter idx; both complete on the slot's mbarrier.
template <typename Cfg, bool KVAR, typename S>
__device__ __forceinline__ void issue_plane(const CUtensorMap* mT, const CUtensorMap* mK, S* ring, float* kring,
                                            uint64_t* bars, uint32_t idx, int x0, int y0, int plane,
                                            const SweepArgs& a) {
    const int tx = x0 - Cfg::PX + HALO, ty = y0 - Cfg::DEPTH + HALO, tz = plane + HALO;
    if (!WFA_CHK(tx >= 0 && tx % Cfg::VA == 0 && tx < a.c.px && ty >= 0 && ty < a.c.py && tz >= 0 && tz < a.c.pz,
                 a.status, 13, tx, ty, tz, (int)idx))
        return;
    uint64_t* bar = &bars[idx % Cfg::NS];
    mbar_expect_tx(bar, Cfg::TX_BYTES);
    tma_load_3d(reinterpret_cast<char*>(ring) + (idx % Cfg::NS) * Cfg::SLOT_T, mT, bar, tx, ty, tz);
    if (KVAR)
        tma_load_3d(reinterpret_cast<char*>(kring) + (idx % (Cfg::NK > 0 ? Cfg::NK : 1)) * Cfg::SLOT_K, mK, bar, tx, ty, tz);
}

template <typename S, bool KVAR, int D, int EX, int EY, int R, int PF>
__global__ void __launch_bounds__(TbCfg<S, KVAR, D, EX, EY, R, PF>::NT, TbCfg<S, KVAR, D, EX, EY, R, PF>::MINB)
    sweep_tb(const __grid_constant__ CUtensorMap tmT, const __grid_constant__ CUtensorMap tmK,
             const __grid_constant__ SweepArgs a) {
    using Cfg = TbCfg<S, KVAR, D, EX, EY, R, PF>;
    constexpr int PX = Cfg::PX, TX = Cfg::TX, TY = Cfg::TY, NTX = Cfg::NTX, NS = Cfg::NS, NK = Cfg::NK,
                  P = Cfg::P, PLANE = Cfg::PLANE;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    // TMA destinations: keep every slot 1024-byte aligned (SMEM reserves the slack)
    unsigned char* smem = smem_raw + ((1024u - (smem_addr(smem_raw) & 1023u)) & 1023u);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem);
    S* ring = reinterpret_cast<S*>(smem + Cfg::BAR_BYTES);
    float* kring = reinterpret_cast<float*>(smem + Cfg::BAR_BYTES + Cfg::RING_BYTES);
    float* sbuf = reinterpret_cast<float*>(smem + Cfg::BAR_BYTES + Cfg::RING_BYTES + Cfg::K_BYTES);

    const SweepCoef& c = a.c;
    const int tid = threadIdx.x;
    const int xl = 4 * (tid % NTX);   // first local x of this thread's cells
    const int yl = R * (tid / NTX);   // first local row
    const bool perx = c.periodic[0], pery = c.periodic[1], perz = c.periodic[2];

#ifdef WFA_CHECKED
    // the TMA descriptor operands must be the kernel's grid-constant parameters
    if (tid == 0) {
        WFA_CHK(__isGridConstant(&tmT) && __isGridConstant(&tmK), a.status, 14, 0, 0, 0, 0);
        WFA_CHK(__isShared(smem_raw), a.status, 15, 0, 0, 0, 0);
    }
#define SIDX(i, lim) (WFA_CHK((i) >= 0 && (i) < (lim), a.status, 16, (int)(i), (int)(lim), __LINE__, 0) ? (i) : 0)
#else
#define SIDX(i, lim) (i)
#endif
    if (tid == 0) {
        for (int b = 0; b < NS; ++b) mbar_init(&bars[b], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    uint32_t cnt = 0;        // planes this block has consumed (ring slot / barrier phase)
    uint32_t issued_hi = 0;  // thread 0: counter one past the last plane issued
    uint32_t fail_idx = 0;
    bool failed = false;

    for (int item = blockIdx.x; item < a.items && !failed; item += gridDim.x) {
        const int tix = item % a.tiles_x;
        const int rest = item / a.tiles_x;
        const int tiy = rest % a.tiles_y;
        const int zci = rest / a.tiles_y;
        const int x0 = tix * TX, y0 = tiy * TY;
        const int z0 = zci * a.zchunk;
        const int z1 = min(z0 + a.zchunk, c.n[2]);
        const int jstart = z0 - D, jend = z1 + D;   // stage-0 planes streamed through
        const int gx0 = x0 - PX + xl, gy0 = y0 - D + yl;

        if (tid == 0) {
            fence_proxy_async_smem();
            for (int p = 0; p <= P && jstart + p < jend; ++p) {
                issue_plane<Cfg, KVAR>(&tmT, &tmK, ring, kring, bars, cnt + p, x0, y0, jstart + p, a);
                issued_hi = cnt + p + 1;
            }
        }

        // per-cell constants over the march
        bool bxm[4], bxp[4], bym[R], byp[R];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            bxm[i] = !perx && gx0 + i == 0;
            bxp[i] = !perx && gx0 + i == c.n[0] - 1;
        }
#pragma unroll
        for (int r = 0; r < R; ++r) {
            bym[r] = !pery && gy0 + r == 0;
            byp[r] = !pery && gy0 + r == c.n[1] - 1;
        }
        // output rows / columns of this thread and whether they need no periodic twins
        const bool out_cols = xl >= PX && xl < PX + TX;
        bool out_row[R], plain_row[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int ly = yl + r, gy = gy0 + r;
            out_row[r] = ly >= D && ly < D + TY && gy < c.n[1];
            plain_row[r] = gx0 + 3 < c.n[0] && !(perx && (gx0 < HALO || gx0 + 3 >= c.n[0] - HALO)) &&
                           !(pery && (gy < HALO || gy >= c.n[1] - HALO));
        }
        bool thread_inner = true;   // no own cell has an x or y boundary face
#pragma unroll
        for (int i = 0; i < 4; ++i) thread_inner = thread_inner && !bxm[i] && !bxp[i];
#pragma unroll
        for (int r = 0; r < R; ++r) thread_inner = thread_inner && !bym[r] && !byp[r];
        const bool has_adv = c.adv[0] != 0.0f || c.adv[1] != 0.0f || c.adv[2] != 0.0f || c.adv[3] != 0.0f ||
                             c.adv[4] != 0.0f || c.adv[5] != 0.0f;

        float zm[D][R][4], zc[D][R][4];   // stage s-1 outputs at planes q-1, q (s = 1..D)
        float gz[D][R][4];                // per-cell k: coefficient of the z face below the next plane
#pragma unroll
        for (int s = 0; s < D; ++s)
#pragma unroll
            for (int r = 0; r < R; ++r)
#pragma unroll
                for (int i = 0; i < 4; ++i) zm[s][r][i] = zc[s][r][i] = gz[s][r][i] = 0.0f;

        for (int j = jstart; j < jend; ++j) {
            const uint32_t idx = cnt + (uint32_t)(j - jstart);
            // a copy that never lands leaves garbage in the slot; the block
            // agrees to stop at the barrier below before issuing anything new
            const bool late = !mbar_wait_bounded(&bars[idx % NS], (idx / NS) & 1u);
            const S* cur0 = reinterpret_cast<const S*>(reinterpret_cast<const char*>(ring) + (idx % NS) * Cfg::SLOT_T);  // stage-0 plane j
            const S* prev0 = reinterpret_cast<const S*>(reinterpret_cast<const char*>(ring) + ((idx + NS - 1) % NS) * Cfg::SLOT_T);  // j-1

            float nw[D + 1][R][4];
#pragma unroll
            for (int r = 0; r < R; ++r) Vec4<S>::load(cur0 + SIDX((yl + r) * EX + xl, PLANE - 3), nw[0][r]);

#pragma unroll
            for (int s = 1; s <= D; ++s) {
                const int q = j - s;   // plane this stage updates
                // only the columns later stages (or the output) depend on
                const int lo_x = PX - (D - s), hi_x = EX - PX + (D - s);
                const int lo_y = s, hi_y = EY - s;
                const bool need = xl + 4 > lo_x && xl < hi_x && yl + R > lo_y && yl < hi_y;
                if (!need) {
#pragma unroll
                    for (int r = 0; r < R; ++r)
#pragma unroll
                        for (int i = 0; i < 4; ++i) nw[s][r][i] = 0.0f;
                    continue;
                }
                // x/y neighbours of stage s-1 at plane q
                float below[4], above[4];
                {
                    const int yb = max(yl - 1, 0), ya = min(yl + R, EY - 1);
                    if (s == 1) {
                        Vec4<S>::load(prev0 + SIDX(yb * EX + xl, PLANE - 3), below);
                        Vec4<S>::load(prev0 + SIDX(ya * EX + xl, PLANE - 3), above);
                    } else {
                        Vec4<float>::load(sbuf + SIDX((s - 2) * PLANE + yb * EX + xl, (D - 1) * PLANE - 3), below);
                        Vec4<float>::load(sbuf + SIDX((s - 2) * PLANE + ya * EX + xl, (D - 1) * PLANE - 3), above);
                    }
                }
                const bool bzm = !perz && q == 0, bzp = !perz && q == c.n[2] - 1;

                // per-cell k: this stage's 1/k plane (q) and the one above (q + 1)
                constexpr uint32_t NKS = NK > 0 ? NK : 1;
                const float* kq = reinterpret_cast<const float*>(reinterpret_cast<const char*>(kring) + ((idx + 2u * NKS - (uint32_t)s) % NKS) * Cfg::SLOT_K);
                const float* kqp = reinterpret_cast<const float*>(reinterpret_cast<const char*>(kring) + ((idx + 2u * NKS - (uint32_t)s + 1u) % NKS) * Cfg::SLOT_K);
                float kc[R][4];          // 1/k of the own cells
                float gxf[R][5];         // x faces: left of cell i is gxf[r][i], right is gxf[r][i+1]
                float gyf[R + 1][4];     // y faces: below row r is gyf[r], above is gyf[r+1]
                float gzp[R][4];         // z face above plane q (carried to the next plane)
                if (KVAR) {
                    float kb[4], ka[4];
#pragma unroll
                    for (int r = 0; r < R; ++r) Vec4<float>::load(kq + SIDX((yl + r) * EX + xl, PLANE - 3), kc[r]);
                    Vec4<float>::load(kq + SIDX(max(yl - 1, 0) * EX + xl, PLANE - 3), kb);
                    Vec4<float>::load(kq + SIDX(min(yl + R, EY - 1) * EX + xl, PLANE - 3), ka);
#pragma unroll
                    for (int r = 0; r < R; ++r) {
                        const float kl = kq[SIDX((yl + r) * EX + max(xl - 1, 0), PLANE)];
                        const float kr = kq[SIDX((yl + r) * EX + min(xl + 4, EX - 1), PLANE)];
                        gxf[r][0] = face_r(kl, kc[r][0], c.tcd[0]);
#pragma unroll
                        for (int i = 0; i < 3; ++i) gxf[r][i + 1] = face_r(kc[r][i], kc[r][i + 1], c.tcd[0]);
                        gxf[r][4] = face_r(kc[r][3], kr, c.tcd[0]);
                        float kzp[4];
                        Vec4<float>::load(kqp + SIDX((yl + r) * EX + xl, PLANE - 3), kzp);
#pragma unroll
                        for (int i = 0; i < 4; ++i) gzp[r][i] = face_r(kc[r][i], kzp[i], c.tcd[2]);
                    }
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        gyf[0][i] = face_r(kb[i], kc[0][i], c.tcd[1]);
                        gyf[R][i] = face_r(kc[R - 1][i], ka[i], c.tcd[1]);
#pragma unroll
                        for (int r = 1; r < R; ++r) gyf[r][i] = face_r(kc[r - 1][i], kc[r][i], c.tcd[1]);
                    }
                }

                // fast path: no cell of this thread touches a boundary at this plane
                const bool fast = thread_inner && !bzm && !bzp;
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    // x neighbours of the row ends (clamped: only out-of-tile cells read a clamped value)
                    const int il = SIDX((yl + r) * EX + max(xl - 1, 0), PLANE);
                    const int ir = SIDX((yl + r) * EX + min(xl + 4, EX - 1), PLANE);
                    const float left = s == 1 ? to_f32<S>(prev0[il]) : sbuf[SIDX((s - 2) * PLANE + il, (D - 1) * PLANE)];
                    const float right = s == 1 ? to_f32<S>(prev0[ir]) : sbuf[SIDX((s - 2) * PLANE + ir, (D - 1) * PLANE)];
                    const int gy = gy0 + r;
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const float tc = zc[s - 1][r][i];
                        float txm = i == 0 ? left : zc[s - 1][r][i - 1];
                        float txp = i == 3 ? right : zc[s - 1][r][i + 1];
                        float tym = r == 0 ? below[i] : zc[s - 1][r - 1][i];
                        float typ = r == R - 1 ? above[i] : zc[s - 1][r + 1][i];
                        float tzm = zm[s - 1][r][i];
                        float tzp = nw[s - 1][r][i];
                        float wxm, wxp, wym, wyp, wzm, wzp;
                        if (KVAR) {
                            wxm = gxf[r][i]; wxp = gxf[r][i + 1];
                            wym = gyf[r][i]; wyp = gyf[r + 1][i];
                            wzm = gz[s - 1][r][i]; wzp = gzp[r][i];
                            if (has_adv) {
                                wxm = __fadd_rn(wxm, c.adv[0]); wxp = __fadd_rn(wxp, c.adv[1]);
                                wym = __fadd_rn(wym, c.adv[2]); wyp = __fadd_rn(wyp, c.adv[3]);
                                wzm = __fadd_rn(wzm, c.adv[4]); wzp = __fadd_rn(wzp, c.adv[5]);
                            }
                        } else {
                            wxm = c.w_in[0]; wxp = c.w_in[1]; wym = c.w_in[2];
                            wyp = c.w_in[3]; wzm = c.w_in[4]; wzp = c.w_in[5];
                        }
                        float v;
                        const bool edge_cell = !fast && (bxm[i] || bxp[i] || bym[r] || byp[r] || bzm || bzp);
                        if (!edge_cell) {
                            v = __fadd_rn(tc, flux_sum(tc, txm, txp, tym, typ, tzm, tzp, wxm, wxp, wym, wyp, wzm, wzp));
                        } else {
                            v = boundary_update<KVAR>(&c, tc, txm, txp, tym, typ, tzm, tzp, wxm, wxp, wym, wyp, wzm,
                                                      wzp, KVAR ? kc[r][i] : 0.0f, gx0 + i, gy, q);
                        }
                        nw[s][r][i] = storage_round<S>(v);
                    }
                }
                if (KVAR) {
#pragma unroll
                    for (int r = 0; r < R; ++r)
#pragma unroll
                        for (int i = 0; i < 4; ++i) gz[s - 1][r][i] = gzp[r][i];
                }
            }

            // every read of prev0 and of the stage planes is done
            if (__syncthreads_or(late)) {
                failed = true;
                fail_idx = idx;
                break;
            }
#pragma unroll
            for (int s = 1; s < D; ++s)
#pragma unroll
                for (int r = 0; r < R; ++r) Vec4<float>::store(sbuf + SIDX((s - 1) * PLANE + (yl + r) * EX + xl, (D - 1) * PLANE - 3), nw[s][r]);
#pragma unroll
            for (int s = 0; s < D; ++s)
#pragma unroll
                for (int r = 0; r < R; ++r)
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        zm[s][r][i] = zc[s][r][i];
                        zc[s][r][i] = nw[s][r][i];
                    }

            // output: stage D at plane j - D
            {
                const int q = j - D;
                if (q >= z0 && q < z1 && out_cols) {
                    S* out = (S*)a.tout;
                    const bool zplain = !(perz && (q < HALO || q >= c.n[2] - HALO));
#pragma unroll
                    for (int r = 0; r < R; ++r) {
                        if (!out_row[r]) continue;
                        const int gy = gy0 + r;
                        const int gx = gx0;
                        const bool plain = plain_row[r] && zplain;
                        if (plain) {
                            const long long off = (long long)q * c.sz + (long long)gy * c.sy + gx;
                            if (WFA_CHK(off >= c.lo && off + 3 < c.hi && (off & 3) == 0, a.status, 10, gx, gy, q, r))
                                Vec4<S>::store(out + off, nw[D][r]);
                        } else {
#pragma unroll
                            for (int i = 0; i < 4; ++i)
                                if (gx + i < c.n[0]) store_twins_out_of_line<S>(out, &c, gx + i, gy, q, nw[D][r][i], a.status);
                        }
                    }
                }
            }
            __syncthreads();   // stage planes written; the ring slot of plane j-1 is free
            if (tid == 0 && j + P + 1 < jend) {
                fence_proxy_async_smem();
                issue_plane<Cfg, KVAR>(&tmT, &tmK, ring, kring, bars, idx + P + 1, x0, y0, j + P + 1, a);
                issued_hi = idx + P + 2;
            }
        }
        if (failed) break;
        cnt += (uint32_t)(jend - jstart);
    }
#undef SIDX

    if (failed) {
        // drain: wait (bounded) for the copies this block issued and has not consumed
        if (tid == 0) {
            atomicExch(a.status, 1);
            for (uint32_t u = fail_idx; u < issued_hi; ++u) (void)mbar_wait_bounded(&bars[u % NS], (u / NS) & 1u);
        }
        __syncthreads();
    }
}

}  // namespace wfa
