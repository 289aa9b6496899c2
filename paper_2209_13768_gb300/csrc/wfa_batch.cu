// wfa_batch_run: many grids of different sizes and step counts advanced
// together (Sec. 4.1.2: iteration rate at small workloads per processor —
// one launch per grid and step would leave most of the GPU idle for grids of
// 16^3..128^3 cells, and every launch would pay its own latency).
//
// Step s of every grid that still has more than s steps to go runs in one
// launch per class of grids (storage type x conductivity mode x advection);
// the launch boundary is the only barrier between steps, so nothing inside a
// launch waits for anything. A block works on one grid: 256 (column, z
// chunk) pairs, each a column of 4 x cells over a chunk of planes marched
// with the column-march code of the single-grid sweep (same arithmetic, so
// results are bitwise those of wfa_step). Chunks are shortened for small
// grids so that every block has 256 pairs. Within a class the grids are
// sorted by step count, so the grids still active at step s are a prefix of
// the block table and a launch is just a shorter grid of blocks.
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <vector>

#include "wfa_sweep_col.cuh"

namespace wfa {

namespace {

constexpr int MG_THREADS = 256;
// {f32, bf16} x {uniform k, per-cell k, per-cell k with advection, and the
// last two with every boundary face in the ghost layers}
constexpr int NKIND = 5;
constexpr int NCLASS = 2 * NKIND;

struct MgGrid {
    SweepCoef c;
    const void* tb[2];    // domain origins of the field buffers; step s reads tb[s & 1]
    const float* rk;      // 1/k (nullptr for uniform k)
    int ncx;              // groups of 4 x cells per row
    int ncols;            // ncx * ny
    int zchunk, nch;      // z chunk length and count
    int block0;           // first block of the grid in a launch of its class
    int nblocks;          // ceil(ncols * nch / MG_THREADS)
    long long steps;
};

// blocks per SM the register budget targets (the general boundary path keeps
// more values live than the ghost-layer one)
template <bool KVAR, bool GHOST> struct MgOcc { static constexpr int blocks = GHOST ? 4 : (KVAR ? 3 : 4); };

// One step of every active grid of one class; block b works on grid
// block_grid[b], pairs (b - block0) * 256 + thread, numbered chunk-major.
template <typename S, bool KVAR, bool ADV, bool GHOST>
__global__ void __launch_bounds__(MG_THREADS, MgOcc<KVAR, GHOST>::blocks)
    mg_sweep(const MgGrid* __restrict__ grids, const int* __restrict__ block_grid, long long step, int* status) {
    __shared__ MgGrid sg;
    static_assert(sizeof(MgGrid) % 4 == 0, "copied as words");
    const MgGrid* src = &grids[block_grid[blockIdx.x]];
    for (int i = threadIdx.x; i < (int)(sizeof(MgGrid) / 4); i += MG_THREADS)
        reinterpret_cast<int*>(&sg)[i] = reinterpret_cast<const int*>(src)[i];
    __syncthreads();
    const int p = ((int)blockIdx.x - sg.block0) * MG_THREADS + (int)threadIdx.x;
    if (p >= sg.ncols * sg.nch) return;
    const int chunk = p / sg.ncols, col = p - chunk * sg.ncols;
    const int gx = 4 * (col % sg.ncx), gy = col / sg.ncx;
    const int z0 = chunk * sg.zchunk;
    const int z1 = min(z0 + sg.zchunk, sg.c.n[2]);
    col_run<S, KVAR, ADV, false, 1, false, true, GHOST>(sg.c, (const S*)sg.tb[step & 1], (S*)sg.tb[(step + 1) & 1],
                                                        sg.rk, status, gx, gy, z0, z1);
}

template <typename S>
cudaError_t launch_kind(int kind, int blocks, const MgGrid* grids, const int* block_grid, long long step, int* status,
                        cudaStream_t st) {
    switch (kind) {
        case 0: mg_sweep<S, false, false, false><<<blocks, MG_THREADS, 0, st>>>(grids, block_grid, step, status); break;
        case 1: mg_sweep<S, true, false, false><<<blocks, MG_THREADS, 0, st>>>(grids, block_grid, step, status); break;
        case 2: mg_sweep<S, true, true, false><<<blocks, MG_THREADS, 0, st>>>(grids, block_grid, step, status); break;
        case 3: mg_sweep<S, true, false, true><<<blocks, MG_THREADS, 0, st>>>(grids, block_grid, step, status); break;
        default: mg_sweep<S, true, true, true><<<blocks, MG_THREADS, 0, st>>>(grids, block_grid, step, status); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_class(int cls, int blocks, const MgGrid* grids, const int* block_grid, long long step, int* status,
                         cudaStream_t st) {
    return cls < NKIND ? launch_kind<float>(cls, blocks, grids, block_grid, step, status, st)
                       : launch_kind<__nv_bfloat16>(cls - NKIND, blocks, grids, block_grid, step, status, st);
}

// Per (device, stream) tables: pinned host staging and its device copy.
struct BatchCtx {
    unsigned char* host = nullptr;
    unsigned char* dev = nullptr;
    size_t cap = 0;
};

std::mutex g_batch_mu;
std::map<std::pair<int, cudaStream_t>, BatchCtx*> g_batch;

BatchCtx* context_for(cudaStream_t st) {
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(g_batch_mu);
    BatchCtx*& c = g_batch[{dev, st}];
    if (!c) c = new BatchCtx();
    return c;
}

int reserve(BatchCtx* c, size_t bytes) {
    if (bytes <= c->cap) return WFA_OK;
    if (c->host) cudaFreeHost(c->host);
    if (c->dev) cudaFree(c->dev);
    c->host = nullptr;
    c->dev = nullptr;
    c->cap = 0;
    const size_t cap = std::max(bytes, (size_t)1 << 20) * 2;
    WFA_CUDA(cudaMallocHost(&c->host, cap));
    WFA_CUDA(cudaMalloc(&c->dev, cap));
    c->cap = cap;
    return WFA_OK;
}

}  // namespace

}  // namespace wfa

using namespace wfa;

extern "C" int wfa_batch_run(wfa_grid* gs, const long long* steps, int count) {
    if (count < 0 || (count > 0 && (!gs || !steps))) {
        set_error("wfa_batch_run: bad arguments");
        return WFA_ERR_ARG;
    }
    if (count == 0) return WFA_OK;
    cudaStream_t st = gs[0] ? gs[0]->stream : nullptr;
    std::vector<int> order;
    long long max_steps = 0;
    for (int i = 0; i < count; ++i) {
        wfa_grid g = gs[i];
        if (!g || steps[i] < 0) {
            set_error("wfa_batch_run: grid %d is NULL or has a negative step count", i);
            return WFA_ERR_ARG;
        }
        if (!g->field_set || !g->coeffs_set || !g->dt_set) {
            set_error("wfa_batch_run: grid %d needs its field, coefficients and dt", i);
            return WFA_ERR_STATE;
        }
        if (g->stream != st) {
            set_error("wfa_batch_run: grid %d is on another stream than grid 0", i);
            return WFA_ERR_ARG;
        }
        for (int j = 0; j < i; ++j)
            if (gs[j] == g) {
                set_error("wfa_batch_run: grid %d appears twice", i);
                return WFA_ERR_ARG;
            }
        if (steps[i] > 0) order.push_back(i);
        max_steps = std::max(max_steps, steps[i]);
    }
    if (order.empty()) return WFA_OK;
    // halos, held layers and 1/k of grids changed since their last step
    for (int i : order) {
        wfa_grid g = gs[i];
        if (g->halo_dirty) {
            int rc = refresh_halo(g, g->cur);
            if (rc) return rc;
            rc = prepare_coeff_halo(g);
            if (rc) return rc;
            g->halo_dirty = false;
        }
    }
    // descriptors, grouped by class, each class sorted by step count (descending)
    const int ng = (int)order.size();
    std::vector<MgGrid> mg(ng);
    std::vector<int> cls(ng);
    for (int k = 0; k < ng; ++k) {
        wfa_grid g = gs[order[k]];
        MgGrid& b = mg[k];
        memset(&b, 0, sizeof b);
        int rc = build_coef(g, &b.c);
        if (rc) return rc;
        const long long off = domain_offset(g);
        b.tb[0] = (const char*)g->T[g->cur] + off * g->esize;
        b.tb[1] = (const char*)g->T[1 - g->cur] + off * g->esize;
        b.rk = g->r ? g->r + off : nullptr;
        bool adv = false;
        for (int f = 0; f < 6; ++f) adv = adv || b.c.adv[f] != 0.0f;
        const int kind = g->r ? (adv ? 2 : 1) + (b.c.halo_bc ? 2 : 0) : 0;
        cls[k] = (g->storage == WFA_BF16 ? NKIND : 0) + kind;
        b.ncx = (g->n[0] + 3) / 4;
        b.ncols = b.ncx * g->n[1];
        // z chunks of about 16 planes, shorter (down to 4) while a grid has
        // fewer pairs than a block has threads
        const int nz = g->n[2];
        int nch = std::max((nz + 15) / 16, (MG_THREADS + b.ncols - 1) / b.ncols);
        nch = std::max(1, std::min(nch, nz / 4));
        b.zchunk = (nz + nch - 1) / nch;
        b.nch = (nz + b.zchunk - 1) / b.zchunk;
        const long long pairs = (long long)b.ncols * b.nch;
        if (pairs > (1LL << 30)) {
            set_error("wfa_batch_run: grid %d is too large for the batched sweep", order[k]);
            return WFA_ERR_ARG;
        }
        b.nblocks = (int)((pairs + MG_THREADS - 1) / MG_THREADS);
        b.steps = steps[order[k]];
    }
    std::vector<int> idx(ng);
    for (int k = 0; k < ng; ++k) idx[k] = k;
    std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) {
        return cls[a] != cls[b] ? cls[a] < cls[b] : mg[a].steps > mg[b].steps;
    });
    int cls_first[NCLASS + 1];   // sorted positions of each class
    for (int t = 0; t <= NCLASS; ++t) cls_first[t] = ng;
    for (int j = ng - 1; j >= 0; --j) cls_first[cls[idx[j]]] = j;
    for (int t = NCLASS - 1; t >= 0; --t) cls_first[t] = std::min(cls_first[t], cls_first[t + 1]);
    std::vector<MgGrid> sorted(ng);
    long long total_blocks = 0;
    for (int t = 0; t < NCLASS; ++t) {
        long long b0 = 0;
        for (int j = cls_first[t]; j < cls_first[t + 1]; ++j) {
            sorted[j] = mg[idx[j]];
            sorted[j].block0 = (int)b0;
            b0 += sorted[j].nblocks;
        }
        if (b0 > (1LL << 30)) {
            set_error("wfa_batch_run: too many blocks in one launch");
            return WFA_ERR_ARG;
        }
        total_blocks += b0;
    }
    // device tables: the descriptors, then per class the block -> grid map
    const size_t grid_bytes = ((size_t)ng * sizeof(MgGrid) + 255) / 256 * 256;
    const size_t bytes = grid_bytes + (size_t)total_blocks * sizeof(int);
    BatchCtx* c = context_for(st);
    // the previous call's copy out of the pinned buffer is complete: every
    // call synchronises the stream before it returns
    int rc = reserve(c, bytes);
    if (rc) return rc;
    memcpy(c->host, sorted.data(), (size_t)ng * sizeof(MgGrid));
    int* bmap = reinterpret_cast<int*>(c->host + grid_bytes);
    long long cls_map[NCLASS];   // offset of each class's block map (ints)
    {
        long long o = 0;
        for (int t = 0; t < NCLASS; ++t) {
            cls_map[t] = o;
            for (int j = cls_first[t]; j < cls_first[t + 1]; ++j)
                for (int b = 0; b < sorted[j].nblocks; ++b) bmap[o++] = j;
        }
    }
    WFA_CUDA(cudaMemcpyAsync(c->dev, c->host, bytes, cudaMemcpyHostToDevice, st));
    const MgGrid* dgrids = reinterpret_cast<const MgGrid*>(c->dev);
    const int* dmap = reinterpret_cast<const int*>(c->dev + grid_bytes);
    int* status = gs[order[0]]->d_status;
    // step s: per class, the grids with more than s steps are a prefix
    int active[NCLASS];
    for (int t = 0; t < NCLASS; ++t) active[t] = cls_first[t + 1];
    for (long long s = 0; s < max_steps; ++s) {
        for (int t = 0; t < NCLASS; ++t) {
            while (active[t] > cls_first[t] && sorted[active[t] - 1].steps <= s) --active[t];
            if (active[t] == cls_first[t]) continue;
            const MgGrid& last = sorted[active[t] - 1];
            cudaError_t e = launch_class(t, last.block0 + last.nblocks, dgrids, dmap + cls_map[t], s, status, st);
            if (e != cudaSuccess) return cuda_fail(e, "wfa_batch_run launch");
        }
    }
    rc = check_status(gs[order[0]]);   // synchronises the stream
    if (rc) return rc;
    for (int k = 0; k < ng; ++k) {
        wfa_grid g = gs[order[k]];
        g->cur = (int)((g->cur + mg[k].steps) & 1);
        g->steps_done += mg[k].steps;
    }
    return WFA_OK;
}
