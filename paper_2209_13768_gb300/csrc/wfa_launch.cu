// Host side of wfa_step: TMA descriptors, depth / tile choice, work
// decomposition of the persistent tiled sweep, ping-pong bookkeeping.
#include <cudaTypedefs.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <mutex>

#include "wfa_sweep_impl.cuh"

namespace wfa {

struct TmapCache {
    CUtensorMap t[2];
    CUtensorMap k;
    int ex, ey;
    const void* tbase[2];
    const void* kbase;
};

void free_tmaps(wfa_grid_s* g) {
    free(g->tmaps);
    g->tmaps = nullptr;
}

static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    });
    return fn;
}

// 3D tiled map over a whole padded buffer; box = one (ex x ey) plane.
static int encode_map(CUtensorMap* m, const void* base, CUtensorMapDataType dt, int esize, const wfa_grid_s* g,
                      int ex, int ey) {
    auto fn = encode_fn();
    if (!fn) {
        set_error("cuTensorMapEncodeTiled is not available from the driver");
        return WFA_ERR_CUDA;
    }
    const cuuint64_t dims[3] = {(cuuint64_t)g->px, (cuuint64_t)g->py, (cuuint64_t)g->pz};
    const cuuint64_t strides[2] = {(cuuint64_t)g->px * esize, (cuuint64_t)g->px * g->py * esize};
    const cuuint32_t box[3] = {(cuuint32_t)ex, (cuuint32_t)ey, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = fn(m, dt, 3, const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        set_error("cuTensorMapEncodeTiled failed (CUresult %d) for box %dx%d", (int)r, ex, ey);
        return WFA_ERR_CUDA;
    }
    return WFA_OK;
}

static int get_tmaps(wfa_grid_s* g, int ex, int ey, TmapCache** out) {
    TmapCache* tc = (TmapCache*)g->tmaps;
    if (tc && tc->ex == ex && tc->ey == ey && tc->tbase[0] == g->T[0] && tc->tbase[1] == g->T[1] &&
        tc->kbase == g->k) {
        *out = tc;
        return WFA_OK;
    }
    if (!tc) {
        void* p = nullptr;
        if (posix_memalign(&p, 128, sizeof(TmapCache)) != 0) {
            set_error("host allocation failed");
            return WFA_ERR_OOM;
        }
        memset(p, 0, sizeof(TmapCache));
        tc = (TmapCache*)p;
        g->tmaps = p;
    }
    const CUtensorMapDataType dt =
        g->storage == WFA_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    for (int b = 0; b < 2; ++b) {
        int rc = encode_map(&tc->t[b], g->T[b], dt, g->esize, g, ex, ey);
        if (rc) return rc;
        tc->tbase[b] = g->T[b];
    }
    if (g->k) {
        int rc = encode_map(&tc->k, g->k, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, g, ex, ey);
        if (rc) return rc;
    } else {
        tc->k = tc->t[0];   // never read
    }
    tc->kbase = g->k;
    tc->ex = ex;
    tc->ey = ey;
    *out = tc;
    return WFA_OK;
}

static int num_sms() {
    static int n = 0;
    if (!n) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 1;
    }
    return n;
}

// Depth used when nobody forced one and the autotuner has no entry.
static int default_depth(const wfa_grid_s* g) {
    if (g->tuned_depth) return g->tuned_depth;
    return g->k ? 2 : 4;
}

static TbEntry entry_for(const wfa_grid_s* g, int depth, int variant) {
    if (g->storage == WFA_BF16) return g->k ? tb_entry_bf16_k(depth, variant) : tb_entry_bf16_u(depth, variant);
    return g->k ? tb_entry_f32_k(depth, variant) : tb_entry_f32_u(depth, variant);
}

// Split the z extent so that (tiles x chunks) fills the resident blocks in
// whole waves while keeping the redundant 2*depth planes per chunk small.
static void choose_chunks(int nz, int depth, long long tiles, long long resident, int* zchunk, int* nchunk) {
    double best = 1e300;
    int bz = nz, bn = 1;
    for (int n = 1; n <= nz; ++n) {
        const int zc = (nz + n - 1) / n;
        const int nn = (nz + zc - 1) / zc;
        if (nn != n) continue;
        if (zc < 2 * depth && n > 1) break;
        const long long items = tiles * n;
        const long long waves = (items + resident - 1) / resident;
        const double t = (double)waves * (zc + 2.0 * depth);
        if (t < best * 0.999) {
            best = t;
            bz = zc;
            bn = n;
        }
    }
    *zchunk = bz;
    *nchunk = bn;
}

static SweepArgs base_args(wfa_grid_s* g, const SweepCoef& c, int in_buf) {
    SweepArgs a;
    memset(&a, 0, sizeof a);
    a.c = c;
    const long long off = domain_offset(g);
    a.tin = (const char*)g->T[in_buf] + off * g->esize;
    a.tout = (char*)g->T[1 - in_buf] + off * g->esize;
    a.k = g->k ? g->k + off : nullptr;
    a.status = g->d_status;
    return a;
}

// One pass of `depth` fused steps from buffer g->cur into the other buffer.
static int one_pass(wfa_grid_s* g, const SweepCoef& c, int depth, int variant) {
    SweepArgs a = base_args(g, c, g->cur);
    if (variant < 0) {   // one-column reference kernel, one step
        cudaError_t e;
        if (g->storage == WFA_BF16)
            e = g->k ? launch_simple_bf16_k(a, g->stream) : launch_simple_bf16_u(a, g->stream);
        else
            e = g->k ? launch_simple_f32_k(a, g->stream) : launch_simple_f32_u(a, g->stream);
        if (e != cudaSuccess) return cuda_fail(e, "sweep_simple launch");
        g->cur = 1 - g->cur;
        return WFA_OK;
    }
    const TbEntry en = entry_for(g, depth, variant);
    TmapCache* tm = nullptr;
    int rc = get_tmaps(g, en.ex, en.ey, &tm);
    if (rc) return rc;
    a.tiles_x = (c.n[0] + en.tx - 1) / en.tx;
    a.tiles_y = (c.n[1] + en.ty - 1) / en.ty;
    const long long tiles = (long long)a.tiles_x * a.tiles_y;
    const long long resident = (long long)en.occupancy() * num_sms();
    choose_chunks(c.n[2], depth, tiles, resident, &a.zchunk, &a.nzchunk);
    const long long items = tiles * a.nzchunk;
    if (items > (1LL << 30)) {
        set_error("grid too large for one pass");
        return WFA_ERR_ARG;
    }
    a.items = (int)items;
    const int blocks = (int)std::min<long long>(items, resident);
    cudaError_t e = en.launch(&tm->t[g->cur], &tm->k, a, blocks, g->stream);
    if (e != cudaSuccess) return cuda_fail(e, "sweep_tb launch");
    g->cur = 1 - g->cur;
    return WFA_OK;
}

int launch_sweep(wfa_grid_s* g, long long nsteps) {
    SweepCoef c;
    int rc = build_coef(g, &c);
    if (rc) return rc;
    const int variant = g->force_variant ? g->force_variant : (g->tuned_variant ? g->tuned_variant : 1);
    int depth = g->force_depth ? g->force_depth : default_depth(g);
    if (variant < 0) depth = 1;
    while (nsteps > 0) {
        const int d = (int)std::min<long long>(depth, nsteps);
        rc = one_pass(g, c, d, variant);
        if (rc) return rc;
        nsteps -= d;
    }
    return WFA_OK;
}

}  // namespace wfa
