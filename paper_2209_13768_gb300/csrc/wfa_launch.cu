// Host side of wfa_step: TMA descriptors, depth / tile choice, work
// decomposition of the persistent tiled sweep, ping-pong bookkeeping.
#include <cudaTypedefs.h>
#include <stdlib.h>
#include <string.h>

#include <stdio.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <string>
#include <new>
#include <vector>

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

// Event pairs bracketing the main sweep kernel of sampled passes.
constexpr int TIMING_MAX_PAIRS = 4096;
struct KernelTiming {
    std::vector<cudaEvent_t> ev;   // pair i: ev[2i] before, ev[2i + 1] after
    std::vector<int> weight;       // launches pair i brackets (a replayed run: its passes)
    int used = 0;
};

void free_timing(wfa_grid_s* g) {
    auto* t = static_cast<KernelTiming*>(g->timing);
    if (!t) return;
    for (cudaEvent_t e : t->ev) cudaEventDestroy(e);
    delete t;
    g->timing = nullptr;
}

// The pair for this pass, or null when the pass is not sampled (timing off,
// not an every-th pass, or every pair in use until the next read).
static const cudaEvent_t* timing_slot(wfa_grid_s* g, int weight = 1) {
    if (g->timing_every <= 0) return nullptr;
    if (g->timing_pass++ % g->timing_every) return nullptr;
    auto* t = static_cast<KernelTiming*>(g->timing);
    if (!t || t->used >= TIMING_MAX_PAIRS) return nullptr;
    if ((int)t->weight.size() <= t->used) t->weight.resize(t->used + 1);
    t->weight[t->used] = weight;
    if (2 * t->used == (int)t->ev.size()) {
        cudaEvent_t a, b;
        if (cudaEventCreate(&a) != cudaSuccess) return nullptr;
        if (cudaEventCreate(&b) != cudaSuccess) {
            cudaEventDestroy(a);
            return nullptr;
        }
        t->ev.push_back(a);
        t->ev.push_back(b);
    }
    return &t->ev[2 * t->used++];
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
        tc->kbase == g->r) {
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
    if (g->r) {
        int rc = encode_map(&tc->k, g->r, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, g, ex, ey);
        if (rc) return rc;
    } else {
        tc->k = tc->t[0];   // never read
    }
    tc->kbase = g->r;
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

// ------------------------------------------------------------ tuning ------
// Kernel configuration of a pass: variant (COL_VARIANT = column march, one
// step; INPLACE_VARIANT = the same with boundaries and periodic copies in the
// pass itself; FUSED_VARIANT = column march, two steps, uniform k;
// WIDE_VARIANT = column march, 8 cells a thread (16 for bf16 with uniform k);
// T2_VARIANT = two steps, TMA-staged planes, uniform k; 1..NUM_TILE_VARIANTS
// = tiled TMA kernel, `depth` fused steps; -1 = the plain one-column kernel)
// and depth.
struct Choice {
    int variant, depth;
    int zc = 0;   // column kernels: planes per z chunk (0 = automatic)
};

// Autotuned choices, per size class, shared by every grid of the process and
// optionally persisted (WFA_TUNE_CACHE = path of a small text file).
static std::mutex g_tune_mu;
static std::map<std::string, Choice> g_tune;
static bool g_tune_loaded = false;

static int ceil_log2(int v) {
    int k = 0;
    while ((1 << k) < v) ++k;
    return k;
}

// The device a choice was measured on: compute capability and SM count, so
// one cache file can serve different GPUs.
static const char* device_tag() {
    static char tag[32] = "";
    if (!tag[0]) {
        int dev = 0, major = 0, minor = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
        cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
        snprintf(tag, sizeof tag, "cc%d%d.sm%d", major, minor, num_sms());
    }
    return tag;
}

static std::string tune_key(const wfa_grid_s* g) {
    char buf[128];
    const bool adv = g->u[0] != 0.0 || g->u[1] != 0.0 || g->u[2] != 0.0;
    snprintf(buf, sizeof buf, "%s.%s.%s.%s.%d.%d.%d", device_tag(), g->storage == WFA_BF16 ? "bf16" : "f32",
             g->r ? "k" : "u", adv ? "adv" : "noadv", ceil_log2(g->n[0]), ceil_log2(g->n[1]), ceil_log2(g->n[2]));
    return buf;
}

static void tune_load_locked() {
    if (g_tune_loaded) return;
    g_tune_loaded = true;
    const char* path = getenv("WFA_TUNE_CACHE");
    if (!path) return;
    FILE* f = fopen(path, "r");
    if (!f) return;
    char key[128];
    char line[256];
    while (fgets(line, sizeof line, f)) {   // "key variant depth [zchunk]"
        int v, d, z = 0;
        if (sscanf(line, "%127s %d %d %d", key, &v, &d, &z) >= 3) g_tune[key] = Choice{v, d, z};
    }
    fclose(f);
}

static void tune_save_locked() {
    const char* path = getenv("WFA_TUNE_CACHE");
    if (!path) return;
    FILE* f = fopen(path, "w");
    if (!f) return;
    for (const auto& kv : g_tune)
        fprintf(f, "%s %d %d %d\n", kv.first.c_str(), kv.second.variant, kv.second.depth, kv.second.zc);
    fclose(f);
}

static Choice choose(const wfa_grid_s* g) {
    Choice ch{COL_VARIANT, 1};   // untuned default: the column-march kernel, one step per pass
    if (g->tuned_variant) {
        ch = Choice{g->tuned_variant, g->tuned_depth, g->tuned_zchunk};
    } else {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        tune_load_locked();
        auto it = g_tune.find(tune_key(g));
        if (it != g_tune.end()) ch = it->second;
    }
    if (g->force_variant || g->force_depth) {
        const int v = g->force_variant ? g->force_variant : (g->force_depth > 1 ? 1 : COL_VARIANT);
        int d = g->force_depth ? g->force_depth : (v == COL_VARIANT || v < 0 ? 1 : 2);
        ch = Choice{v, d};
    }
    if (g->force_zchunk) ch.zc = g->force_zchunk;
    // exchange faces: the column kernels (one step a pass, the neighbour
    // slab's plane read from the halo) or the one-column kernel
    if (has_exchange_face(g) && ch.variant != COL_VARIANT && ch.variant != INPLACE_VARIANT &&
        ch.variant != WIDE_VARIANT && ch.variant >= 0)
        ch = Choice{COL_VARIANT, 1, ch.zc};
    if (ch.variant < 0 || ch.variant == COL_VARIANT || ch.variant == INPLACE_VARIANT || ch.variant == WIDE_VARIANT)
        ch.depth = 1;
    if (ch.variant == FUSED_VARIANT || ch.variant == T2_VARIANT) ch.depth = g->k ? 1 : 2;   // per-cell k: one step
    return ch;
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

static SweepArgs base_args(wfa_grid_s* g, const SweepCoef& c, int in_buf, int zc = 0) {
    SweepArgs a;
    memset(&a, 0, sizeof a);
    a.zchunk = zc;
    a.c = c;
    const long long off = domain_offset(g);
    a.tin = (const char*)g->T[in_buf] + off * g->esize;
    a.tout = (char*)g->T[1 - in_buf] + off * g->esize;
    a.rk = g->r ? g->r + off : nullptr;
    a.status = g->d_status;
    return a;
}

// Kernels one pass launches (the column kernels add a boundary fix-up and a
// copy per periodic axis, see col_launch / col2_launch).
static int pass_launches(const wfa_grid_s* g, const SweepCoef& c, int depth, int variant) {
    const int periodic = c.periodic[0] + c.periodic[1] + c.periodic[2];
    if (variant == FUSED_VARIANT && depth == 2 && !g->r) return 1 + periodic;
    if (variant == COL_VARIANT || variant == WIDE_VARIANT || variant == FUSED_VARIANT || variant == T2_VARIANT) {   // thin pass
        // boundary cells the ghost layers do not hold: one boundary_fix launch
        // (the one-step column pass keeps held faces itself)
        const bool col = variant == COL_VARIANT || variant == WIDE_VARIANT ||
                         ((variant == FUSED_VARIANT || variant == T2_VARIANT) && !(depth == 2 && !g->r));
        bool faces = false;
        for (int f = 0; f < 6; ++f) faces = faces || (!c.periodic[f >> 1] && !c.ext[f] && !(col && c.held[f]));
        return 1 + (faces && !c.halo_bc ? 1 : 0);
    }
    return 1;
}

// The pass reads periodic copies beyond the first layer (or corner copies):
// the tiled kernels and the two-step column kernel.
static bool needs_full_twins(const wfa_grid_s* g, int depth, int variant) {
    if (variant == FUSED_VARIANT || variant == T2_VARIANT) return depth == 2 && !g->r;
    return variant >= 1 && variant <= NUM_TILE_VARIANTS;
}
// The pass writes one layer of periodic copies only (the thin column pass).
static bool writes_thin_twins(const wfa_grid_s* g, const SweepCoef& c, int depth, int variant) {
    if (!c.periodic[0] && !c.periodic[1] && !c.periodic[2]) return false;
    const bool two = (variant == FUSED_VARIANT || variant == T2_VARIANT) && depth == 2 && !g->r;
    return !two && (variant == COL_VARIANT || variant == WIDE_VARIANT || variant == FUSED_VARIANT || variant == T2_VARIANT);
}

// One pass of `depth` fused steps from buffer g->cur into the other buffer
// (zc: planes per z chunk of the column kernels, 0 = automatic).
static int one_pass(wfa_grid_s* g, const SweepCoef& c, int depth, int variant, int zc = 0) {
    if (needs_full_twins(g, depth, variant) && g->thin[g->cur]) {   // complete the copies first
        const int rc = refresh_halo(g, g->cur);
        if (rc) return rc;
    }
    g->thin[1 - g->cur] = writes_thin_twins(g, c, depth, variant);
    g->launches += pass_launches(g, c, depth, variant);
    SweepArgs a = base_args(g, c, g->cur, zc);
    const cudaEvent_t* ev = timing_slot(g);
    if (variant < 0) {   // one-column reference kernel, one step
        cudaError_t e;
        if (ev) cudaEventRecord(ev[0], g->stream);
        if (g->storage == WFA_BF16)
            e = g->k ? launch_simple_bf16_k(a, g->stream) : launch_simple_bf16_u(a, g->stream);
        else
            e = g->k ? launch_simple_f32_k(a, g->stream) : launch_simple_f32_u(a, g->stream);
        if (ev) cudaEventRecord(ev[1], g->stream);
        if (e != cudaSuccess) return cuda_fail(e, "sweep_simple launch");
        g->cur = 1 - g->cur;
        return WFA_OK;
    }
    if (variant == T2_VARIANT && depth == 2 && !g->r) {   // two steps, TMA-staged planes (uniform k)
        TmapCache* tm = nullptr;
        int rc = get_tmaps(g, 80, 20, &tm);
        if (rc) return rc;
        cudaError_t e = g->storage == WFA_BF16 ? launch_t2_bf16_u(&tm->t[g->cur], a, g->stream, num_sms(), ev)
                                               : launch_t2_f32_u(&tm->t[g->cur], a, g->stream, num_sms(), ev);
        if (e != cudaSuccess) return cuda_fail(e, "sweep_t2 launch");
        g->cur = 1 - g->cur;
        return WFA_OK;
    }
    if (variant == FUSED_VARIANT && depth == 2 && !g->r) {   // two-step column march (uniform k)
        cudaError_t e = g->storage == WFA_BF16 ? launch_col2_bf16_u(a, g->stream, num_sms(), ev)
                                               : launch_col2_f32_u(a, g->stream, num_sms(), ev);
        if (e != cudaSuccess) return cuda_fail(e, "sweep_col2 launch");
        g->cur = 1 - g->cur;
        return WFA_OK;
    }
    if (variant == COL_VARIANT || variant == FUSED_VARIANT || variant == INPLACE_VARIANT || variant == T2_VARIANT ||
        variant == WIDE_VARIANT) {   // column march, one step
        const bool inl = variant == INPLACE_VARIANT, wide = variant == WIDE_VARIANT;
        cudaError_t e;
        if (g->storage == WFA_BF16)
            e = g->r ? launch_col_bf16_k(a, g->stream, num_sms(), ev, inl, wide)
                     : launch_col_bf16_u(a, g->stream, num_sms(), ev, inl, wide);
        else
            e = g->r ? launch_col_f32_k(a, g->stream, num_sms(), ev, inl, wide)
                     : launch_col_f32_u(a, g->stream, num_sms(), ev, inl, wide);
        if (e != cudaSuccess) return cuda_fail(e, "sweep_col launch");
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
    if (ev) cudaEventRecord(ev[0], g->stream);
    cudaError_t e = en.launch(&tm->t[g->cur], &tm->k, a, blocks, g->stream);
    if (ev) cudaEventRecord(ev[1], g->stream);
    if (e != cudaSuccess) return cuda_fail(e, "sweep_tb launch");
    g->cur = 1 - g->cur;
    return WFA_OK;
}

// Small grids: a run of GRAPH_PASSES passes captured once as a CUDA graph
// and replayed, so that the per-kernel launch cost (which dominates a pass of
// a few microseconds) is paid once per run. One graph per starting buffer;
// a graph is rebuilt when anything its kernels were given changes.
constexpr int GRAPH_PASSES = 32;                // even: a run ends on the buffer it started from
constexpr long long GRAPH_MAX_CELLS = 1LL << 22;

struct StepGraph {
    SweepCoef c;
    const void* T[2];
    const float* r;
    int variant = 0, depth = 0, zc = 0;
    cudaGraphExec_t exec = nullptr;
};
struct StepGraphs {
    StepGraph slot[2];            // by starting buffer
    cudaStream_t stream = nullptr;  // capture stream
};

void free_graphs(wfa_grid_s* g) {
    auto* gs = static_cast<StepGraphs*>(g->graphs);
    if (!gs) return;
    for (auto& sl : gs->slot)
        if (sl.exec) cudaGraphExecDestroy(sl.exec);
    if (gs->stream) cudaStreamDestroy(gs->stream);
    delete gs;
    g->graphs = nullptr;
}

// The graph of GRAPH_PASSES passes from buffer g->cur with this configuration
// (captured now if the cached one was made for something else).
static int run_graph(wfa_grid_s* g, const SweepCoef& c, const Choice& ch, cudaGraphExec_t* out) {
    if (!g->graphs) g->graphs = new (std::nothrow) StepGraphs();
    auto* gs = static_cast<StepGraphs*>(g->graphs);
    if (!gs) {
        set_error("host allocation failed");
        return WFA_ERR_OOM;
    }
    StepGraph& sl = gs->slot[g->cur];
    const bool same = sl.exec && !memcmp(&sl.c, &c, sizeof c) && sl.T[0] == g->T[0] && sl.T[1] == g->T[1] &&
                      sl.r == g->r && sl.variant == ch.variant && sl.depth == ch.depth && sl.zc == ch.zc;
    if (!same) {
        if (sl.exec) cudaGraphExecDestroy(sl.exec);
        sl.exec = nullptr;
        if (!gs->stream) WFA_CUDA(cudaStreamCreateWithFlags(&gs->stream, cudaStreamNonBlocking));
        // the passes are issued on the capture stream; g->cur and the launch
        // count move back to where they were (nothing ran yet)
        const cudaStream_t user = g->stream;
        const int cur0 = g->cur;
        const long long launches0 = g->launches;
        const bool thin0[2] = {g->thin[0], g->thin[1]};
        g->stream = gs->stream;
        cudaError_t e = cudaStreamBeginCapture(gs->stream, cudaStreamCaptureModeThreadLocal);
        int rc = WFA_OK;
        for (int k = 0; k < GRAPH_PASSES && e == cudaSuccess && !rc; ++k)
            rc = one_pass(g, c, ch.depth, ch.variant, ch.zc);
        cudaGraph_t graph = nullptr;
        const cudaError_t e2 = e == cudaSuccess ? cudaStreamEndCapture(gs->stream, &graph) : e;
        g->stream = user;
        g->cur = cur0;
        g->launches = launches0;
        g->thin[0] = thin0[0];
        g->thin[1] = thin0[1];
        if (e == cudaSuccess) e = e2;
        if (e == cudaSuccess && !rc) e = cudaGraphInstantiate(&sl.exec, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        if (rc) return rc;
        if (e != cudaSuccess) return cuda_fail(e, "step graph capture");
        sl.c = c;
        sl.T[0] = g->T[0];
        sl.T[1] = g->T[1];
        sl.r = g->r;
        sl.variant = ch.variant;
        sl.depth = ch.depth;
        sl.zc = ch.zc;
    }
    *out = sl.exec;
    return WFA_OK;
}

int launch_sweep(wfa_grid_s* g, long long nsteps) {
    SweepCoef c;
    int rc = build_coef(g, &c);
    if (rc) return rc;
    const Choice ch = choose(g);
    const long long cells = (long long)g->n[0] * g->n[1] * g->n[2];
    const long long runs = nsteps / ((long long)ch.depth * GRAPH_PASSES);
    if (cells <= GRAPH_MAX_CELLS && runs >= 2) {
        cudaGraphExec_t exec = nullptr;
        if (needs_full_twins(g, ch.depth, ch.variant) && g->thin[g->cur]) {   // not inside the graph
            rc = refresh_halo(g, g->cur);
            if (rc) return rc;
        }
        const int every = g->timing_every;
        g->timing_every = 0;   // no event records inside the captured passes
        rc = run_graph(g, c, ch, &exec);
        g->timing_every = every;
        if (rc) return rc;
        for (long long r = 0; r < runs; ++r) {
            // kernel timing samples a whole run (its passes, fix-up kernels included)
            const cudaEvent_t* ev = every > 0 ? timing_slot(g, GRAPH_PASSES) : nullptr;
            if (ev) cudaEventRecord(ev[0], g->stream);
            WFA_CUDA(cudaGraphLaunch(exec, g->stream));
            if (ev) cudaEventRecord(ev[1], g->stream);
        }
        g->launches += runs * GRAPH_PASSES * pass_launches(g, c, ch.depth, ch.variant);
        nsteps -= runs * GRAPH_PASSES * ch.depth;
        g->thin[0] = g->thin[1] = writes_thin_twins(g, c, ch.depth, ch.variant);   // both written by the run
    }
    while (nsteps > 0) {
        const int d = (int)std::min<long long>(ch.depth, nsteps);
        rc = one_pass(g, c, d, ch.variant, ch.zc);
        if (rc) return rc;
        nsteps -= d;
    }
    return WFA_OK;
}

// Time every compiled configuration on a scratch copy of the grid's field
// and keep the fastest (results do not depend on the choice).
int autotune(wfa_grid_s* g, int* depth_out, int* variant_out) {
    SweepCoef c;
    int rc = build_coef(g, &c);
    if (rc) return rc;
    // trial passes are not the caller's steps: keep them out of kernel timing
    struct Pause {
        wfa_grid_s* g;
        int every;
        ~Pause() { g->timing_every = every; }
    } pause{g, g->timing_every};
    g->timing_every = 0;
    std::vector<Choice> cands = {{COL_VARIANT, 1}, {WIDE_VARIANT, 1}, {INPLACE_VARIANT, 1}, {T2_VARIANT, 2}, {FUSED_VARIANT, 2}, {1, 1}, {2, 1},
                                 {1, 2}, {2, 2}, {1, 3}, {2, 3}, {1, 4}, {2, 4}, {1, 6}, {1, 8}};
    // the column kernels with other z chunk lengths: longer ones read fewer
    // boundary planes twice (fewer, longer-lived blocks, down to two chunks:
    // one wave on large grids); shorter ones put more blocks in flight (at
    // 512^3 with per-cell k, 12-plane chunks measured 1% faster than 16)
    const int half = (c.n[2] + 1) / 2;
    for (int zc : {8, 12, 32, 64, 128})
        if (zc < half) cands.push_back(Choice{COL_VARIANT, 1, zc});
    if (half >= 32) cands.push_back(Choice{COL_VARIANT, 1, half});
    for (int zc : {12, 32})
        if (zc < half) cands.push_back(Choice{WIDE_VARIANT, 1, zc});
    const size_t bytes = field_elems(g) * g->esize;
    void* save = nullptr;
    WFA_CUDA(dev_alloc(&save, bytes, g->stream));
    const int cur0 = g->cur;
    cudaError_t e = cudaMemcpyAsync(save, g->T[cur0], bytes, cudaMemcpyDeviceToDevice, g->stream);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    const long long cells = (long long)g->n[0] * g->n[1] * g->n[2];
    const int steps = cells > (1LL << 22) ? 24 : 96;   // divisible by every depth tried
    Choice best{COL_VARIANT, 1};
    float best_ms = 1e30f;
    for (const Choice& ch : cands) {
        if (e != cudaSuccess) break;
        if ((ch.variant == FUSED_VARIANT || ch.variant == T2_VARIANT) && g->k) continue;   // uniform k only
        if (has_exchange_face(g) && ch.variant != COL_VARIANT && ch.variant != INPLACE_VARIANT &&
            ch.variant != WIDE_VARIANT)
            continue;
        // one warm-up pass, then the timed passes
        rc = one_pass(g, c, ch.depth, ch.variant, ch.zc);
        if (rc) break;
        cudaEventRecord(e0, g->stream);
        for (int s = 0; s < steps && !rc; s += ch.depth) rc = one_pass(g, c, ch.depth, ch.variant, ch.zc);
        cudaEventRecord(e1, g->stream);
        if (rc) break;
        e = cudaEventSynchronize(e1);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && ms < best_ms) {
            best_ms = ms;
            best = ch;
        }
    }
    // put the field back exactly as it was
    if (e == cudaSuccess) e = cudaMemcpyAsync(g->T[cur0], save, bytes, cudaMemcpyDeviceToDevice, g->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(g->stream);
    g->cur = cur0;
    g->halo_dirty = true;   // the other buffer's halo was rewritten by the trials
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    dev_free(save, g->stream);
    if (rc) return rc;
    if (e != cudaSuccess) return cuda_fail(e, "autotune");
    g->tuned_variant = best.variant;
    g->tuned_depth = best.depth;
    g->tuned_zchunk = best.zc;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        tune_load_locked();
        g_tune[tune_key(g)] = best;
        tune_save_locked();
    }
    if (depth_out) *depth_out = best.depth;
    if (variant_out) *variant_out = best.variant;
    return WFA_OK;
}

}  // namespace wfa

extern "C" {

int wfa_set_kernel_timing(wfa_grid g, int every) {
    if (!g) { wfa::set_error("NULL grid"); return WFA_ERR_ARG; }
    if (every < 0) { wfa::set_error("every must be >= 0"); return WFA_ERR_ARG; }
    wfa::free_timing(g);
    g->timing_every = every;
    g->timing_pass = 0;
    if (every > 0) {
        g->timing = new (std::nothrow) wfa::KernelTiming();
        if (!g->timing) {
            g->timing_every = 0;
            wfa::set_error("host allocation failed");
            return WFA_ERR_OOM;
        }
    }
    return WFA_OK;
}

int wfa_kernel_time(wfa_grid g, double* ms, long long* launches) {
    if (!g || !ms || !launches) { wfa::set_error("NULL argument"); return WFA_ERR_ARG; }
    *ms = 0.0;
    *launches = 0;
    auto* t = static_cast<wfa::KernelTiming*>(g->timing);
    if (!t) return WFA_OK;
    cudaError_t e = cudaStreamSynchronize(g->stream);
    double sum = 0.0;
    long long n = 0;
    for (int i = 0; i < t->used && e == cudaSuccess; ++i) {
        float m = 0.0f;
        e = cudaEventElapsedTime(&m, t->ev[2 * i], t->ev[2 * i + 1]);
        sum += m;
        n += t->weight[i];
    }
    t->used = 0;
    if (e != cudaSuccess) return wfa::cuda_fail(e, "wfa_kernel_time");
    *ms = sum;
    *launches = n;
    return WFA_OK;
}

}  // extern "C"

extern "C" int wfa_get_tuning(wfa_grid g, int* depth, int* variant, int* zchunk) {
    if (!g) {
        wfa::set_error("NULL grid");
        return WFA_ERR_ARG;
    }
    const wfa::Choice ch = wfa::choose(g);
    if (depth) *depth = ch.depth;
    if (variant) *variant = ch.variant;
    if (zchunk) *zchunk = ch.zc;
    return WFA_OK;
}

extern "C" int wfa_launch_count(wfa_grid g, long long* n) {
    if (!g || !n) {
        wfa::set_error("NULL argument");
        return WFA_ERR_ARG;
    }
    *n = g->launches;
    return WFA_OK;
}
