// wfa_batch_run: many grids of different sizes and step counts advanced
// together (Sec. 3.1.2: iteration rate at small workloads per processor —
// one launch per grid and step would leave most of the GPU idle for grids of
// 16^3..128^3 cells, and every launch would pay its own latency).
//
// Work unit: 256 (column, z chunk) pairs of one grid, each a column of 4 x
// cells over a chunk of planes, marched with the column-march code of the
// single-grid sweep (same arithmetic, so results are bitwise those of
// wfa_step). Chunks are shortened for small grids so that a unit is full.
// Grids are sorted by step count (descending), so the grids still active at
// step (round) r are a prefix and so are their units.
//
// Default ("rounds"): every round is one launch per class of grid (storage
// type x conductivity mode x advection x ghost-layer faces) over the active
// units, one block per unit; the whole sequence is captured into one CUDA
// graph and launched once, so the launch boundary is the barrier between
// rounds and nothing inside a kernel waits on another block. Grids are
// independent, so the graph has a branch per class and group of grids
// (a class of many grids is dealt round-robin into up to two groups): one
// branch's round fills the GPU while another's drains.
// WFA_BATCH_MODE=persistent runs the rounds in one persistent kernel instead
// (replayed as a graph: descriptor copy, counter reset, kernel): every block
// the GPU can hold is launched, the blocks take the active units of round r
// from an atomic counter, then meet at a grid-wide barrier, a counter with a
// bounded spin; a wait that runs out (about 2 s) sets an abort word, every
// block stops and the call returns WFA_ERR_TIMEOUT. WFA_BATCH_MODE=stream
// issues the per-round launches directly on the stream. All three give the
// same fields bit for bit; the per-round graph was the fastest measured
// (256 grids of 16..128 cells per edge, side by side with an earlier column
// march: 200 GLUPS against 168 persistent; the per-round graph now runs
// about 305).
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <tuple>
#include <type_traits>
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
// per-round launches: the grids of a class are dealt round-robin (by step
// count) into NGROUP groups, each its own branch of the graph, so one
// group's round can fill the GPU while another's drains (the 256-grid batch:
// 2 groups 4% faster than 4, 10% faster than 1, 12% faster than 8)
constexpr int NGROUP = 2;
constexpr int NBRANCH = NCLASS * NGROUP;

struct MgGrid {
    SweepCoef c;
    const void* tb[2];    // domain origins of the field buffers; step s reads tb[s & 1]
    const float* rk;      // 1/k (nullptr for uniform k)
    int cls;              // class: storage * NKIND + kind
    int ncx;              // groups of 4 x cells per row
    int ncols;            // ncx * ny
    int zchunk, nch;      // z chunk length and count
    int nblocks;          // units: ceil(ncols * nch / MG_THREADS)
    int block0;           // first unit of the grid in a per-round launch of its class
    int unit0;            // first unit of the grid in the persistent kernel's table
    // uniform k, per-round launches: a branch-free main pass that stores one
    // layer of periodic copies, then the boundary cells in a launch of its own
    int nbu, bu0;         // boundary-cell units (256 cells) and the first in its class
    int pad;
    long long steps;
};

// One step of unit u of a grid: thread t takes pair u * 256 + t, pairs
// numbered chunk-major over (z chunk, column). COH: the field was written by
// other blocks of the same launch (persistent kernel), so it is read through
// L2 (ld.cg) instead of the read-only path.
template <typename S, bool KVAR, bool ADV, bool GHOST, bool COH>
__device__ __forceinline__ void mg_unit(const MgGrid& sg, int u, long long step, int* status) {
    const int p = u * MG_THREADS + (int)threadIdx.x;
    if (p >= sg.ncols * sg.nch) return;
    const int chunk = p / sg.ncols, col = p - chunk * sg.ncols;
    const int gx = 4 * (col % sg.ncx), gy = col / sg.ncx;
    const int z0 = chunk * sg.zchunk;
    const int z1 = min(z0 + sg.zchunk, sg.c.n[2]);
    col_run<S, KVAR, ADV, COH, 1, COL_INPLACE, true, GHOST>(sg.c, (const S*)sg.tb[step & 1], (S*)sg.tb[(step + 1) & 1],
                                                        sg.rk, status, gx, gy, z0, z1);
}

// Copy a descriptor into shared memory (all threads; callers synchronise).
__device__ __forceinline__ void load_desc(MgGrid* dst, const MgGrid* src) {
    static_assert(sizeof(MgGrid) % 4 == 0, "copied as words");
    for (int i = threadIdx.x; i < (int)(sizeof(MgGrid) / 4); i += MG_THREADS)
        reinterpret_cast<int*>(dst)[i] = reinterpret_cast<const int*>(src)[i];
}

// ------------------------------------------------------ one launch per round
template <bool KVAR, bool GHOST> struct MgOcc { static constexpr int blocks = GHOST ? 4 : (KVAR ? 3 : 4); };

template <typename S, bool KVAR, bool ADV, bool GHOST>
__global__ void __launch_bounds__(MG_THREADS, MgOcc<KVAR, GHOST>::blocks)
    mg_sweep(const MgGrid* __restrict__ grids, const int* __restrict__ block_grid, long long step, int* status) {
    __shared__ MgGrid sg;
    load_desc(&sg, &grids[block_grid[blockIdx.x]]);
    __syncthreads();
    mg_unit<S, KVAR, ADV, GHOST, false>(sg, (int)blockIdx.x - sg.block0, step, status);
}

// Uniform k, per-round launches: every cell takes the interior formula
// (branch-free, the occupancy of the single-grid main pass) and stores one
// layer of periodic copies, all that the next one-step pass reads ...
template <typename S>
__global__ void __launch_bounds__(MG_THREADS, (ColOcc<false, false, sizeof(S)>::blocks))
    mg_sweep_main(const MgGrid* __restrict__ grids, const int* __restrict__ block_grid, long long step) {
    __shared__ MgGrid sg;
    load_desc(&sg, &grids[block_grid[blockIdx.x]]);
    __syncthreads();
    const int p = ((int)blockIdx.x - sg.block0) * MG_THREADS + (int)threadIdx.x;
    if (p >= sg.ncols * sg.nch) return;
    const int chunk = p / sg.ncols, col = p - chunk * sg.ncols;
    const int gx = 4 * (col % sg.ncx), gy = col / sg.ncx;
    const int z0 = chunk * sg.zchunk;
    const int z1 = min(z0 + sg.zchunk, sg.c.n[2]);
    col_run<S, false, false, false, ColOcc<false, false, sizeof(S)>::unroll, COL_THIN, true>(
        sg.c, (const S*)sg.tb[step & 1], (S*)sg.tb[(step + 1) & 1], nullptr, nullptr, gx, gy, z0, z1);
}

// ... then the outer cell layer of every non-periodic face recomputed with
// the boundary conditions (the cells of a face in 256-cell units), with its
// periodic copies where another axis is periodic.
template <typename S>
__global__ void __launch_bounds__(MG_THREADS)
    mg_boundary(const MgGrid* __restrict__ grids, const int* __restrict__ unit_grid, long long step, int* status) {
    __shared__ MgGrid sg;
    load_desc(&sg, &grids[unit_grid[blockIdx.x]]);
    __syncthreads();
    const SweepCoef& c = sg.c;
    long long u = (long long)((int)blockIdx.x - sg.bu0) * MG_THREADS + threadIdx.x;
    int pos[3] = {0, 0, 0};
    bool found = false;
    for (int ax = 0; ax < 3 && !found; ++ax) {
        if (c.periodic[ax]) continue;
        const int b = ax == 0 ? 1 : 0, d = ax == 2 ? 1 : 2;
        const long long plane = (long long)c.n[b] * c.n[d];
        if (u >= 2 * plane) {
            u -= 2 * plane;
            continue;
        }
        pos[ax] = u >= plane ? c.n[ax] - 1 : 0;
        u %= plane;
        pos[b] = (int)(u % c.n[b]);
        pos[d] = (int)(u / c.n[b]);
        found = true;
    }
    if (!found) return;   // past the last face
    const S* tin = (const S*)sg.tb[step & 1];
    const long long i = (long long)pos[2] * c.sz + (long long)pos[1] * c.sy + pos[0];
    const S v = from_f32<S>(general_cell<S, false>(c, tin, nullptr, i, pos[0], pos[1], pos[2], status));
    S* tout = (S*)sg.tb[(step + 1) & 1];
    if (c.periodic[0] || c.periodic[1] || c.periodic[2])
        store_with_twins<S>(tout, c, pos[0], pos[1], pos[2], v, status);
    else
        tout[i] = v;
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

// One round of a uniform-k class: main pass, then boundary cells (a block
// count of 0 skips that launch).
template <typename S>
cudaError_t uniform_round(int blocks, int bblocks, const MgGrid* grids, const int* map, const int* bmap,
                          long long step, int* status, cudaStream_t st) {
    mg_sweep_main<S><<<blocks, MG_THREADS, 0, st>>>(grids, map, step);
    if (bblocks > 0) mg_boundary<S><<<bblocks, MG_THREADS, 0, st>>>(grids, bmap, step, status);
    return cudaGetLastError();
}

// ------------------------------------------------------- persistent launch
struct PHeader {
    int ngrids;
    int total_units;
    int max_steps;
    int stall;        // test hook: the first barrier waits for one arrival too many (0: off)
};

// layout of the packed descriptor buffer (pinned host copy and device copy)
struct PLayout {
    size_t header, grids, unit_grid, bytes;
    static PLayout of(int ngrids, int nunits) {
        PLayout l;
        size_t o = 0;
        l.header = o; o += 256;
        l.grids = o; o += ((size_t)ngrids * sizeof(MgGrid) + 255) / 256 * 256;
        l.unit_grid = o; o += ((size_t)nunits * sizeof(int) + 255) / 256 * 256;
        l.bytes = o;
        return l;
    }
};

__device__ __forceinline__ unsigned load_acquire_u32(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ int load_acquire_i32(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Every block of the launch arrives; returns false (everywhere) if the wait
// gave up or another block reported an abort.
__device__ bool grid_barrier(unsigned* count, unsigned target, int* status) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(count, 1u);
        int ok = 1;
        if (load_acquire_u32(count) < target) {
            const uint64_t t0 = global_ns();
            while (load_acquire_u32(count) < target) {
                if (load_acquire_i32(status) != 0 || global_ns() - t0 > 2000000000ull) {
                    ok = 0;
                    break;
                }
            }
        }
        if (!ok) atomicCAS(status, 0, 2);
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

template <typename S, bool KVAR, bool ADV, bool GHOST>
__device__ __noinline__ void unit_call(const MgGrid& sg, int u, long long step, int* status) {
    mg_unit<S, KVAR, ADV, GHOST, true>(sg, u, step, status);
}

__device__ __forceinline__ void unit_dispatch(const MgGrid& sg, int u, long long step, int* status) {
    switch (sg.cls) {
        case 0: unit_call<float, false, false, false>(sg, u, step, status); break;
        case 1: unit_call<float, true, false, false>(sg, u, step, status); break;
        case 2: unit_call<float, true, true, false>(sg, u, step, status); break;
        case 3: unit_call<float, true, false, true>(sg, u, step, status); break;
        case 4: unit_call<float, true, true, true>(sg, u, step, status); break;
        case 5: unit_call<__nv_bfloat16, false, false, false>(sg, u, step, status); break;
        case 6: unit_call<__nv_bfloat16, true, false, false>(sg, u, step, status); break;
        case 7: unit_call<__nv_bfloat16, true, true, false>(sg, u, step, status); break;
        case 8: unit_call<__nv_bfloat16, true, false, true>(sg, u, step, status); break;
        default: unit_call<__nv_bfloat16, true, true, true>(sg, u, step, status); break;
    }
}

// Class -> (storage, conductivity mode, advection, ghost-layer faces).
template <int CLS> struct ClassOf {
    using S = typename std::conditional<(CLS >= NKIND), __nv_bfloat16, float>::type;
    static constexpr int kind = CLS % NKIND;
    static constexpr bool kvar = kind != 0, adv = kind == 2 || kind == 4, ghost = kind >= 3;
};

// Blocks per SM the register budget targets: CLS < 0 dispatches every class
// per unit (its registers are the largest variant's); one class alone is
// compiled like the per-round kernels.
template <int CLS> struct PersistOcc {
    static constexpr int blocks = CLS < 0 ? 3 : MgOcc<ClassOf<(CLS < 0 ? 0 : CLS)>::kvar,
                                                      ClassOf<(CLS < 0 ? 0 : CLS)>::ghost>::blocks;
};

template <int CLS>
__global__ void __launch_bounds__(MG_THREADS, PersistOcc<CLS>::blocks)
    batch_persistent(const unsigned char* __restrict__ packed, PLayout lay, unsigned* count, int* status) {
    const PHeader& h = *reinterpret_cast<const PHeader*>(packed + lay.header);
    const MgGrid* grids = reinterpret_cast<const MgGrid*>(packed + lay.grids);
    const int* unit_grid = reinterpret_cast<const int*>(packed + lay.unit_grid);
    __shared__ MgGrid sg;
    __shared__ int s_u;
    unsigned* grab = count + 2;   // units handed out so far, over all rounds
    unsigned base = 0;            // grab count at the start of this round
    int have = -1;                // grid whose descriptor sg holds
    for (int r = 0; r < h.max_steps; ++r) {
        // grids are sorted by step count, descending: those with more than r
        // steps are the first `lo`, and their units the first `units`
        int lo = 0, hi = h.ngrids;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (grids[mid].steps > r) lo = mid + 1;
            else hi = mid;
        }
        const int units = lo < h.ngrids ? grids[lo].unit0 : h.total_units;
        // units go to whichever block asks next (their cost differs with the
        // grid's chunk length); every block asks once more than it gets, so a
        // round hands out exactly units + gridDim.x grabs
        for (;;) {
            if (threadIdx.x == 0) s_u = (int)(atomicAdd(grab, 1u) - base);
            __syncthreads();
            const int u = s_u;
            __syncthreads();   // s_u read by everyone before the next grab
            if (u >= units) break;
            const int g = unit_grid[u];
            if (g != have) {   // the previous unit's use of sg ended at the barriers above
                load_desc(&sg, &grids[g]);
                __syncthreads();
                have = g;
            }
            if constexpr (CLS < 0) {
                unit_dispatch(sg, u - sg.unit0, r, status);
            } else {
                using C = ClassOf<(CLS < 0 ? 0 : CLS)>;
                mg_unit<typename C::S, C::kvar, C::adv, C::ghost, true>(sg, u - sg.unit0, r, status);
            }
        }
        base += (unsigned)units + gridDim.x;
        if (r + 1 < h.max_steps &&
            !grid_barrier(count, (unsigned)(r + 1) * gridDim.x + (h.stall ? 1u : 0u), status))
            return;
    }
}

// Launch (or query the occupancy of) the persistent kernel of class cls
// (-1: every class). The launch is cooperative: the runtime starts it only
// with all its blocks resident at once (or refuses it), which the kernel's
// grid-wide barrier needs even while other streams keep SMs busy.
cudaError_t persistent_kernel(int cls, bool launch, int* occ, int blocks, const unsigned char* dev, const PLayout& lay,
                              unsigned* count, cudaStream_t st) {
    int* status = reinterpret_cast<int*>(count + 1);
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(blocks > 0 ? blocks : 1);
    cfg.blockDim = dim3(MG_THREADS);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
#define WFA_PERSIST_CASE(K)                                                                                   \
    case K:                                                                                                   \
        if (launch) {                                                                                         \
            const cudaError_t e = cudaLaunchKernelEx(&cfg, batch_persistent<K>, dev, lay, count, status);     \
            if (e != cudaSuccess) return e;                                                                   \
        } else {                                                                                              \
            return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, batch_persistent<K>, MG_THREADS, 0);    \
        }                                                                                                     \
        break;
    switch (cls) {
        WFA_PERSIST_CASE(-1)
        WFA_PERSIST_CASE(0)
        WFA_PERSIST_CASE(1)
        WFA_PERSIST_CASE(2)
        WFA_PERSIST_CASE(3)
        WFA_PERSIST_CASE(4)
        WFA_PERSIST_CASE(5)
        WFA_PERSIST_CASE(6)
        WFA_PERSIST_CASE(7)
        WFA_PERSIST_CASE(8)
        WFA_PERSIST_CASE(9)
        default: return cudaErrorInvalidValue;
    }
#undef WFA_PERSIST_CASE
    return cudaGetLastError();
}

// Per (device, stream, slot) context: descriptor buffers, counters and, per
// class of persistent kernel, the graph of its launch (copy descriptors in,
// clear the counters, run). Two slots let a caller issue the next batch while
// the previous one runs (batch_launch without waiting, then batch_wait).
struct BatchCtx {
    unsigned char* host = nullptr;     // pinned descriptors
    unsigned char* dev = nullptr;      // device descriptors
    size_t cap = 0;                    // bytes of both (per-round launch tables too)
    int cap_grids = 0, cap_units = 0;  // what the persistent layout holds
    PLayout lay{};
    unsigned* count = nullptr;         // barrier arrivals, the status word, units handed out
    cudaStream_t cap_stream = nullptr; // where per-round launches are captured
    cudaStream_t cls_stream[NBRANCH] = {};   // one branch per (class, group) inside the capture
    cudaEvent_t fork = nullptr, join[NBRANCH] = {};
    int blocks[NCLASS + 1] = {};       // launch size per persistent kernel (index cls + 1)
    cudaGraphExec_t exec[NCLASS + 1] = {};
    // a launch not waited for: its graph, an event behind it and its status word read back
    bool pending = false;
    cudaGraphExec_t pending_exec = nullptr;
    cudaEvent_t done = nullptr;
    int* h_status = nullptr;           // pinned, 8 words
    int* pending_status = nullptr;     // the device status word it copied
};

std::mutex g_batch_mu;
std::map<std::tuple<int, cudaStream_t, int>, BatchCtx*> g_batch;

BatchCtx* context_for(cudaStream_t st, int slot) {
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(g_batch_mu);
    BatchCtx*& c = g_batch[std::make_tuple(dev, st, slot)];
    if (!c) c = new BatchCtx();
    return c;
}

void release(BatchCtx* c) {
    for (auto& e : c->exec) {
        if (e) cudaGraphExecDestroy(e);
        e = nullptr;
    }
    if (c->host) cudaFreeHost(c->host);
    if (c->dev) cudaFree(c->dev);
    if (c->count) cudaFree(c->count);
    c->host = nullptr;
    c->dev = nullptr;
    c->count = nullptr;
    c->cap = 0;
    c->cap_grids = c->cap_units = 0;
}

// Buffers for at least `bytes` of per-round tables, or `ngrids` grids and
// `nunits` units of the persistent layout.
int reserve(BatchCtx* c, size_t bytes, int ngrids, int nunits) {
    if (bytes <= c->cap && ngrids <= c->cap_grids && nunits <= c->cap_units) return WFA_OK;
    const int cg = std::max(ngrids, std::max(64, 2 * c->cap_grids));
    const int cu = std::max(nunits, std::max(4096, 2 * c->cap_units));
    const PLayout lay = PLayout::of(cg, cu);
    const size_t cap = std::max(std::max(bytes, lay.bytes), (size_t)1 << 20) * 2;
    release(c);
    WFA_CUDA(cudaMallocHost(&c->host, cap));
    WFA_CUDA(cudaMalloc(&c->dev, cap));
    WFA_CUDA(cudaMalloc(&c->count, 4 * sizeof(unsigned)));
    c->cap = cap;
    c->cap_grids = cg;
    c->cap_units = cu;
    c->lay = lay;
    return WFA_OK;
}

// The graph of the persistent kernel of class cls over the current buffers.
int graph_for(BatchCtx* c, int cls) {
    cudaGraphExec_t& exec = c->exec[cls + 1];
    if (exec) return WFA_OK;
    int dev = 0, sms = 1, occ = 1;
    WFA_CUDA(cudaGetDevice(&dev));
    WFA_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    if (persistent_kernel(cls, false, &occ, 0, nullptr, c->lay, nullptr, nullptr) != cudaSuccess || occ < 1) occ = 1;
    c->blocks[cls + 1] = sms * occ;
    cudaStream_t cap_stream;
    WFA_CUDA(cudaStreamCreateWithFlags(&cap_stream, cudaStreamNonBlocking));
    cudaGraph_t gr = nullptr;
    cudaError_t e = cudaStreamBeginCapture(cap_stream, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->dev, c->host, c->lay.bytes, cudaMemcpyHostToDevice, cap_stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->count, 0, 4 * sizeof(unsigned), cap_stream);
    if (e == cudaSuccess)
        e = persistent_kernel(cls, true, nullptr, c->blocks[cls + 1], c->dev, c->lay, c->count, cap_stream);
    cudaError_t e2 = cudaStreamEndCapture(cap_stream, &gr);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, gr, 0);
    if (gr) cudaGraphDestroy(gr);
    cudaStreamDestroy(cap_stream);
    if (e != cudaSuccess) return cuda_fail(e, "wfa_batch_run graph build");
    return WFA_OK;
}

}  // namespace

// Waits for the launch that batch_launch(..., slot, false) left running on
// stream st, frees its graph and reports its status word (WFA_OK when none is
// pending).
int batch_wait(cudaStream_t st, int slot) {
    BatchCtx* c = context_for(st, slot);
    if (!c->pending) return WFA_OK;
    c->pending = false;
    const cudaError_t e = cudaEventSynchronize(c->done);
    if (c->pending_exec) cudaGraphExecDestroy(c->pending_exec);
    c->pending_exec = nullptr;
    if (e != cudaSuccess) return cuda_fail(e, "wfa_batch_run wait");
    const int code = c->h_status[0];
    if (code != 0) {
        cudaMemsetAsync(c->pending_status, 0, 8 * sizeof(int), st);
        cudaStreamSynchronize(st);
        if (code >= 10) {
            set_error("checked build: bad access, code %d at (%d, %d, %d) extra %d", code, c->h_status[1],
                      c->h_status[2], c->h_status[3], c->h_status[4]);
            return WFA_ERR_CUDA;
        }
        set_error("a device-side wait gave up after its time limit (code %d)", code);
        return WFA_ERR_TIMEOUT;
    }
    return WFA_OK;
}

// The batched sweep. wait = false (per-round modes only; the persistent mode
// always waits) returns once the work is queued on the grids' stream, with
// the grids' state already advanced; batch_wait(stream, slot) must follow
// before the slot is used again, and the grids must stay alive until then.
int batch_launch(wfa_grid* gs, const long long* steps, int count, int slot, bool wait) {
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
        if (has_exchange_face(g)) {
            set_error("wfa_batch_run: grid %d has an exchange face (step slabs with wfa_slabs_step)", i);
            return WFA_ERR_BC;
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
        // z chunks of about 16 planes (the 256-grid batch: 1% faster than 12,
        // 1.2% than 8, 1.5% than 24), shorter (down to 4) while a grid has
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
    // WFA_BATCH_MODE: "rounds" (default: one launch per round and class,
    // captured into one graph, a branch per class), "persistent" (one
    // persistent kernel) or "stream" (the per-round launches issued in order
    // on the stream)
    const char* mode_env = getenv("WFA_BATCH_MODE");
    const int mode = !mode_env ? 1 : !strcmp(mode_env, "persistent") ? 0 : !strcmp(mode_env, "stream") ? 2 : 1;
    BatchCtx* c = context_for(st, slot);
    int rc = batch_wait(st, slot);   // a launch of this slot still in flight
    if (rc) return rc;
    if (!wait && !c->done) {
        WFA_CUDA(cudaEventCreateWithFlags(&c->done, cudaEventDisableTiming));
        WFA_CUDA(cudaMallocHost(&c->h_status, 8 * sizeof(int)));
    }
    if (mode == 0) {
        // persistent launch: grids by step count (descending), units in that order
        std::vector<int> idx(ng);
        for (int k = 0; k < ng; ++k) idx[k] = k;
        std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return mg[a].steps > mg[b].steps; });
        long long units = 0;
        std::vector<MgGrid> sorted(ng);
        for (int j = 0; j < ng; ++j) {
            sorted[j] = mg[idx[j]];
            sorted[j].cls = cls[idx[j]];
            sorted[j].unit0 = (int)units;
            units += sorted[j].nblocks;
        }
        if (units > (1LL << 30)) {
            set_error("wfa_batch_run: too many work units");
            return WFA_ERR_ARG;
        }
        // one class alone gets its own specialised kernel
        int kcls = sorted[0].cls;
        for (int j = 1; j < ng; ++j)
            if (sorted[j].cls != kcls) kcls = -1;
        rc = reserve(c, 0, ng, (int)units);
        if (rc) return rc;
        rc = graph_for(c, kcls);
        if (rc) return rc;
        // 32-bit counters: barrier arrivals (steps x blocks) and unit grabs
        // (every grid's units once per step, plus one miss per block and step)
        unsigned long long grabs = (unsigned long long)max_steps * (unsigned long long)c->blocks[kcls + 1];
        for (int j = 0; j < ng; ++j) grabs += (unsigned long long)sorted[j].nblocks * (unsigned long long)sorted[j].steps;
        if (grabs >= (1ull << 31)) {
            set_error("wfa_batch_run: %lld steps in one call are more than the device counters hold; split the call",
                      max_steps);
            return WFA_ERR_ARG;
        }
        // the previous replay has read the pinned buffer: every call synchronises before it returns
        const PLayout& lay = c->lay;
        PHeader* h = reinterpret_cast<PHeader*>(c->host + lay.header);
        h->ngrids = ng;
        h->total_units = (int)units;
        h->max_steps = (int)max_steps;
        const char* stall = getenv("WFA_TEST_BATCH_STALL");
        h->stall = stall && stall[0] == '1';
        memcpy(c->host + lay.grids, sorted.data(), (size_t)ng * sizeof(MgGrid));
        int* ug = reinterpret_cast<int*>(c->host + lay.unit_grid);
        for (int j = 0; j < ng; ++j)
            for (int b = 0; b < sorted[j].nblocks; ++b) ug[sorted[j].unit0 + b] = j;
        WFA_CUDA(cudaGraphLaunch(c->exec[kcls + 1], st));
        int status = 0;
        WFA_CUDA(cudaMemcpyAsync(&status, c->count + 1, sizeof(int), cudaMemcpyDeviceToHost, st));
        WFA_CUDA(cudaStreamSynchronize(st));
        if (status) {
            set_error("wfa_batch_run: a device-side wait gave up after its time limit; the fields of these grids "
                      "are undefined (code %d)", status);
            return WFA_ERR_TIMEOUT;
        }
        rc = check_status(gs[order[0]]);
        if (rc) return rc;
    } else {
        // one launch per round and branch (class x group); each branch sorted
        // by step count (descending)
        std::vector<int> idx(ng);
        for (int k = 0; k < ng; ++k) idx[k] = k;
        std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) {
            return cls[a] != cls[b] ? cls[a] < cls[b] : mg[a].steps > mg[b].steps;
        });
        // groups per class: one per 32 grids, at most NGROUP (a few large
        // batches gain from overlapping rounds; a tick of the server, rebuilt
        // every time, would only pay for more graph nodes)
        int ncls[NCLASS] = {};
        for (int k = 0; k < ng; ++k) ++ncls[cls[k]];
        std::vector<int> br(ng);   // branch of each grid
        for (int j = 0, rank = 0; j < ng; ++j) {
            rank = (j > 0 && cls[idx[j]] == cls[idx[j - 1]]) ? rank + 1 : 0;
            const int groups = std::max(1, std::min(NGROUP, ncls[cls[idx[j]]] / 32));
            br[idx[j]] = cls[idx[j]] * NGROUP + rank % groups;
        }
        std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) {
            return br[a] != br[b] ? br[a] < br[b] : mg[a].steps > mg[b].steps;
        });
        int cls_first[NBRANCH + 1];   // sorted positions of each branch
        for (int t = 0; t <= NBRANCH; ++t) cls_first[t] = ng;
        for (int j = ng - 1; j >= 0; --j) cls_first[br[idx[j]]] = j;
        for (int t = NBRANCH - 1; t >= 0; --t) cls_first[t] = std::min(cls_first[t], cls_first[t + 1]);
        std::vector<MgGrid> sorted(ng);
        long long total_blocks = 0;
        auto uniform_class = [](int t) { return (t / NGROUP) % NKIND == 0; };   // t: a branch
        for (int t = 0; t < NBRANCH; ++t) {
            long long b0 = 0, bu = 0;
            for (int j = cls_first[t]; j < cls_first[t + 1]; ++j) {
                MgGrid& m = sorted[j];
                m = mg[idx[j]];
                m.cls = t / NGROUP;
                m.block0 = (int)b0;
                b0 += m.nblocks;
                if (uniform_class(t)) {   // boundary-cell units
                    long long bcells = 0;
                    for (int ax = 0; ax < 3; ++ax) {
                        const int b = ax == 0 ? 1 : 0, d = ax == 2 ? 1 : 2;
                        if (!m.c.periodic[ax]) bcells += 2LL * m.c.n[b] * m.c.n[d];
                    }
                    m.nbu = (int)((bcells + MG_THREADS - 1) / MG_THREADS);
                    m.bu0 = (int)bu;
                    bu += m.nbu;
                }
            }
            if (b0 > (1LL << 30) || bu > (1LL << 30)) {
                set_error("wfa_batch_run: too many blocks in one launch");
                return WFA_ERR_ARG;
            }
            total_blocks += b0 + bu;
        }
        // device tables: the descriptors, then per class the block -> grid
        // maps (main units; for uniform k also boundary units)
        const size_t grid_bytes = ((size_t)ng * sizeof(MgGrid) + 255) / 256 * 256;
        const size_t bytes = grid_bytes + (size_t)total_blocks * sizeof(int);
        rc = reserve(c, bytes, 0, 0);
        if (rc) return rc;
        memcpy(c->host, sorted.data(), (size_t)ng * sizeof(MgGrid));
        int* bmap = reinterpret_cast<int*>(c->host + grid_bytes);
        long long cls_map[NBRANCH], cls_bmap[NBRANCH];   // offsets (ints)
        {
            long long o = 0;
            for (int t = 0; t < NBRANCH; ++t) {
                cls_map[t] = o;
                for (int j = cls_first[t]; j < cls_first[t + 1]; ++j)
                    for (int b = 0; b < sorted[j].nblocks; ++b) bmap[o++] = j;
                cls_bmap[t] = o;
                if (uniform_class(t))
                    for (int j = cls_first[t]; j < cls_first[t + 1]; ++j)
                        for (int b = 0; b < sorted[j].nbu; ++b) bmap[o++] = j;
            }
        }
        // mode "rounds": captured on a private stream into one graph, launched
        // on the grids' stream. Branches hold different grids, so each
        // branch's chain of rounds is its own branch of the graph (forked
        // after the descriptor copy, joined at the end): their launches
        // overlap on the GPU instead of draining it between rounds.
        cudaStream_t ls = st;
        if (mode == 1) {
            if (!c->cap_stream) {
                WFA_CUDA(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
                WFA_CUDA(cudaEventCreateWithFlags(&c->fork, cudaEventDisableTiming));
                for (int t = 0; t < NBRANCH; ++t) {
                    WFA_CUDA(cudaStreamCreateWithFlags(&c->cls_stream[t], cudaStreamNonBlocking));
                    WFA_CUDA(cudaEventCreateWithFlags(&c->join[t], cudaEventDisableTiming));
                }
            }
            ls = c->cap_stream;
            WFA_CUDA(cudaStreamBeginCapture(ls, cudaStreamCaptureModeThreadLocal));
        }
        cudaError_t e = cudaMemcpyAsync(c->dev, c->host, bytes, cudaMemcpyHostToDevice, ls);
        if (mode == 1 && e == cudaSuccess) e = cudaEventRecord(c->fork, ls);
        const MgGrid* dgrids = reinterpret_cast<const MgGrid*>(c->dev);
        const int* dmap = reinterpret_cast<const int*>(c->dev + grid_bytes);
        int* status = gs[order[0]]->d_status;
        // per branch, the grids with more than s steps are a prefix
        for (int t = 0; t < NBRANCH && e == cudaSuccess; ++t) {
            if (cls_first[t] == cls_first[t + 1]) continue;
            cudaStream_t cs = mode == 1 ? c->cls_stream[t] : ls;
            if (mode == 1) e = cudaStreamWaitEvent(cs, c->fork, 0);
            int active = cls_first[t + 1];
            for (long long s = 0; s < max_steps && e == cudaSuccess; ++s) {
                while (active > cls_first[t] && sorted[active - 1].steps <= s) --active;
                if (active == cls_first[t]) break;
                const MgGrid& last = sorted[active - 1];
                const int type = t / NGROUP;
                if (uniform_class(t)) {
                    e = type < NKIND ? uniform_round<float>(last.block0 + last.nblocks, last.bu0 + last.nbu, dgrids,
                                                         dmap + cls_map[t], dmap + cls_bmap[t], s, status, cs)
                                     : uniform_round<__nv_bfloat16>(last.block0 + last.nblocks, last.bu0 + last.nbu,
                                                                    dgrids, dmap + cls_map[t], dmap + cls_bmap[t], s,
                                                                    status, cs);
                } else {
                    e = launch_class(type, last.block0 + last.nblocks, dgrids, dmap + cls_map[t], s, status, cs);
                }
            }
            if (mode == 1 && e == cudaSuccess) e = cudaEventRecord(c->join[t], cs);
            if (mode == 1 && e == cudaSuccess) e = cudaStreamWaitEvent(ls, c->join[t], 0);
        }
        cudaGraph_t gr = nullptr;
        cudaGraphExec_t ex = nullptr;
        if (mode == 1) {
            const cudaError_t e2 = cudaStreamEndCapture(ls, &gr);
            if (e == cudaSuccess) e = e2;
            if (e == cudaSuccess) e = cudaGraphInstantiate(&ex, gr, 0);
            if (e == cudaSuccess) e = cudaGraphLaunch(ex, st);
        }
        if (gr) cudaGraphDestroy(gr);   // the executable graph holds what it runs
        if (e == cudaSuccess && !wait) {
            // read back the status word behind the work, then an event for batch_wait
            e = cudaMemcpyAsync(c->h_status, status, 8 * sizeof(int), cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess) e = cudaEventRecord(c->done, st);
            if (e == cudaSuccess) {
                c->pending = true;
                c->pending_exec = ex;
                c->pending_status = status;
                ex = nullptr;
            }
        }
        rc = e != cudaSuccess ? cuda_fail(e, "wfa_batch_run launch")
                              : wait ? check_status(gs[order[0]]) : WFA_OK;   // check_status synchronises
        if (e != cudaSuccess) cudaStreamSynchronize(st);
        if (ex) cudaGraphExecDestroy(ex);
        if (rc) return rc;
    }
    for (int k = 0; k < ng; ++k) {
        wfa_grid g = gs[order[k]];
        g->cur = (int)((g->cur + mg[k].steps) & 1);
        // the persistent kernel and the per-cell-k passes write every periodic
        // copy (corners included); the per-round uniform-k passes one layer
        const bool one_layer = mode != 0 && cls[k] % NKIND == 0 &&
                               (mg[k].c.periodic[0] || mg[k].c.periodic[1] || mg[k].c.periodic[2]);
        if (mg[k].steps >= 1) g->thin[g->cur] = one_layer;
        if (mg[k].steps >= 2) g->thin[1 - g->cur] = one_layer;
        g->steps_done += mg[k].steps;
    }
    return WFA_OK;
}

}  // namespace wfa

using namespace wfa;

extern "C" int wfa_batch_run(wfa_grid* gs, const long long* steps, int count) {
    NvtxRange nvtx_("wfa_batch_run");
    return batch_launch(gs, steps, count, 0, true);
}
