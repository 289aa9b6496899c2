// wfa_batch_run: many grids of different sizes and step counts in one
// persistent launch, replayed as a CUDA graph (Sec. 4.1.2: iteration rate at
// small workloads per processor — one launch per grid and step would leave
// most of the GPU idle for grids of 16^3..128^3 cells).
//
// Work items are (round, grid, column block). They are numbered round-major
// over the grids sorted by step count, so every item of round r-1 of a grid
// is taken (by a running block) before any item of round r of that grid. A
// block takes the next item from an atomic counter, waits until the grid's
// counter shows round r-1 complete (bounded spin), computes one step of its
// column block with the column-march code, and bumps the counter. Because an
// item only ever waits for items taken earlier by running blocks, the launch
// cannot deadlock, whatever the number of resident blocks. A wait that runs
// out (about 2 s) sets an abort word; every block then stops.
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <vector>

#include "wfa_sweep_col.cuh"

namespace wfa {

namespace {

constexpr int BX = 16, BY = 16;        // block of threads: 64 x-cells x 16 rows
constexpr int ZCHUNK = 16;             // planes per work item
constexpr int BATCH_THREADS = BX * BY;

struct BatchGrid {
    SweepCoef c;
    const void* tb[2];    // domain origins of the field buffers; round r reads tb[r & 1]
    const float* rk;      // 1/k (nullptr for uniform k)
    int bf16, kvar, adv;
    int nbx, nby, nch;    // column blocks per round
    int items;            // nbx * nby * nch
    long long steps;
};

struct BatchHeader {
    int ngrids;
    int max_steps;
    int stall_grid;       // test hook: this grid's items of round >= 1 wait for a count that never comes (-1: none)
    int pad;
    long long total_items;
};

// layout of the packed descriptor buffer (host pinned copy and device copy)
struct Layout {
    size_t header, grids, prefix, round_off, bytes;
    static Layout of(int ngrids, int max_steps) {
        Layout l;
        size_t o = 0;
        l.header = o; o += 256;
        l.grids = o; o += ((size_t)ngrids * sizeof(BatchGrid) + 255) / 256 * 256;
        l.prefix = o; o += ((size_t)(ngrids + 1) * sizeof(long long) + 255) / 256 * 256;
        l.round_off = o; o += ((size_t)(max_steps + 1) * sizeof(long long) + 255) / 256 * 256;
        l.bytes = o;
        return l;
    }
};

__device__ __forceinline__ int upper_bound_ll(const long long* a, int n, long long v) {
    int lo = 0, hi = n;   // first index with a[i] > v
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (a[mid] <= v) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ int load_acquire(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

template <typename S, bool KVAR, bool ADV>
__device__ __forceinline__ void batch_item(const BatchGrid& bg, int r, int blk, int* status) {
    const int bx = blk % bg.nbx;
    const int rest = blk / bg.nbx;
    const int by = rest % bg.nby;
    const int ch = rest / bg.nby;
    const int gx = (bx * BX + (int)threadIdx.x) * 4;
    const int gy = by * BY + (int)threadIdx.y;
    if (gx >= bg.c.n[0] || gy >= bg.c.n[1]) return;
    const int z0 = ch * ZCHUNK;
    const int z1 = min(z0 + ZCHUNK, bg.c.n[2]);
    col_run<S, KVAR, ADV, true, 1, false>(bg.c, (const S*)bg.tb[r & 1], (S*)bg.tb[(r + 1) & 1], bg.rk, status, gx, gy, z0,
                              z1);
}

__global__ void __launch_bounds__(BATCH_THREADS, 2)
    batch_kernel(const unsigned char* __restrict__ packed, Layout lay, unsigned long long* work, int* done,
                 int* status) {
    const BatchHeader& h = *reinterpret_cast<const BatchHeader*>(packed + lay.header);
    const BatchGrid* grids = reinterpret_cast<const BatchGrid*>(packed + lay.grids);
    const long long* prefix = reinterpret_cast<const long long*>(packed + lay.prefix);
    const long long* round_off = reinterpret_cast<const long long*>(packed + lay.round_off);
    __shared__ long long s_item;
    __shared__ int s_ok;
    const bool lead = threadIdx.x == 0 && threadIdx.y == 0;
    for (;;) {
        if (lead) s_item = (long long)atomicAdd(work, 1ull);
        __syncthreads();
        const long long it = s_item;
        if (it >= h.total_items) break;
        // item -> (round, grid, block)
        const int r = upper_bound_ll(round_off, h.max_steps + 1, it) - 1;
        const long long j = it - round_off[r];
        const int g = upper_bound_ll(prefix, h.ngrids + 1, j) - 1;
        const int blk = (int)(j - prefix[g]);
        const BatchGrid& bg = grids[g];
        if (lead) {
            // round r - 1 of this grid complete (its items were all taken earlier)
            const int target = r * bg.items + ((g == h.stall_grid && r >= 1) ? 1 : 0);
            int ok = 1;
            if (load_acquire(&done[g]) < target) {
                const uint64_t t0 = global_ns();
                while (load_acquire(&done[g]) < target) {
                    if (load_acquire(status) != 0 || global_ns() - t0 > 2000000000ull) {
                        ok = 0;
                        break;
                    }
                }
            }
            if (!ok) atomicCAS(status, 0, 2);
            s_ok = ok;
        }
        __syncthreads();
        if (!s_ok) break;
        if (bg.bf16) {
            if (!bg.kvar) batch_item<__nv_bfloat16, false, false>(bg, r, blk, status);
            else if (bg.adv) batch_item<__nv_bfloat16, true, true>(bg, r, blk, status);
            else batch_item<__nv_bfloat16, true, false>(bg, r, blk, status);
        } else {
            if (!bg.kvar) batch_item<float, false, false>(bg, r, blk, status);
            else if (bg.adv) batch_item<float, true, true>(bg, r, blk, status);
            else batch_item<float, true, false>(bg, r, blk, status);
        }
        __threadfence();   // this thread's stores before the count below
        __syncthreads();
        if (lead) atomicAdd(&done[g], 1);
    }
}

// Per (device, stream) context: descriptor buffers and the instantiated graph
// (copy descriptors in, clear counters, run the persistent kernel).
struct BatchCtx {
    int device = 0;
    cudaStream_t stream = nullptr;     // where graphs are launched
    unsigned char* host = nullptr;     // pinned descriptors
    unsigned char* dev = nullptr;      // device descriptors
    size_t cap = 0;
    int cap_grids = 0, cap_steps = 0;
    unsigned long long* work = nullptr;
    int* done = nullptr;               // one counter per grid, then the status word
    int blocks = 0;
    cudaGraphExec_t exec = nullptr;
    Layout lay{};
};

std::mutex g_batch_mu;
std::map<std::pair<int, cudaStream_t>, BatchCtx*> g_batch;

int blocks_for_kernel() {
    int dev = 0, sms = 1, occ = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, batch_kernel, BATCH_THREADS, 0) != cudaSuccess || occ < 1)
        occ = 1;
    return sms * occ;
}

void release(BatchCtx* c) {
    if (c->exec) cudaGraphExecDestroy(c->exec);
    if (c->host) cudaFreeHost(c->host);
    if (c->dev) cudaFree(c->dev);
    if (c->work) cudaFree(c->work);
    if (c->done) cudaFree(c->done);
    c->exec = nullptr;
    c->host = nullptr;
    c->dev = nullptr;
    c->work = nullptr;
    c->done = nullptr;
}

// (Re)build buffers and the graph for at least ngrids grids and max_steps rounds.
int ensure(BatchCtx* c, int ngrids, int max_steps) {
    if (c->exec && ngrids <= c->cap_grids && max_steps <= c->cap_steps) return WFA_OK;
    release(c);
    c->cap_grids = std::max(ngrids, std::max(64, 2 * c->cap_grids));
    c->cap_steps = std::max(max_steps, std::max(1024, 2 * c->cap_steps));
    c->lay = Layout::of(c->cap_grids, c->cap_steps);
    c->cap = c->lay.bytes;
    WFA_CUDA(cudaMallocHost(&c->host, c->cap));
    WFA_CUDA(cudaMalloc(&c->dev, c->cap));
    WFA_CUDA(cudaMalloc(&c->work, sizeof(unsigned long long)));
    WFA_CUDA(cudaMalloc(&c->done, (c->cap_grids + 1) * sizeof(int)));
    memset(c->host, 0, c->cap);
    c->blocks = blocks_for_kernel();
    cudaStream_t cap_stream;
    WFA_CUDA(cudaStreamCreateWithFlags(&cap_stream, cudaStreamNonBlocking));
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(cap_stream, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->dev, c->host, c->cap, cudaMemcpyHostToDevice, cap_stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->work, 0, sizeof(unsigned long long), cap_stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->done, 0, (c->cap_grids + 1) * sizeof(int), cap_stream);
    if (e == cudaSuccess) {
        batch_kernel<<<c->blocks, dim3(BX, BY), 0, cap_stream>>>(c->dev, c->lay, c->work, c->done,
                                                                   c->done + c->cap_grids);
        e = cudaGetLastError();
    }
    cudaError_t e2 = cudaStreamEndCapture(cap_stream, &graph);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&c->exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    cudaStreamDestroy(cap_stream);
    if (e != cudaSuccess) return cuda_fail(e, "wfa_batch_run graph build");
    return WFA_OK;
}

BatchCtx* context_for(cudaStream_t st) {
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(g_batch_mu);
    BatchCtx*& c = g_batch[{dev, st}];
    if (!c) {
        c = new BatchCtx();
        c->device = dev;
        c->stream = st;
    }
    return c;
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
    if (max_steps > (1LL << 30)) {
        set_error("wfa_batch_run: too many steps");
        return WFA_ERR_ARG;
    }
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
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return steps[a] > steps[b]; });
    const int ng = (int)order.size();
    BatchCtx* c = context_for(st);
    int rc = ensure(c, ng, (int)max_steps);
    if (rc) return rc;
    const Layout& lay = c->lay;
    unsigned char* host = c->host;
    BatchHeader* h = reinterpret_cast<BatchHeader*>(host + lay.header);
    BatchGrid* bgs = reinterpret_cast<BatchGrid*>(host + lay.grids);
    long long* prefix = reinterpret_cast<long long*>(host + lay.prefix);
    long long* round_off = reinterpret_cast<long long*>(host + lay.round_off);
    // the previous replay must be done reading the pinned buffer before it is rewritten
    WFA_CUDA(cudaStreamSynchronize(st));
    prefix[0] = 0;
    for (int k = 0; k < ng; ++k) {
        wfa_grid g = gs[order[k]];
        BatchGrid& b = bgs[k];
        memset(&b, 0, sizeof b);
        rc = build_coef(g, &b.c);
        if (rc) return rc;
        const long long off = domain_offset(g);
        b.tb[0] = (const char*)g->T[g->cur] + off * g->esize;
        b.tb[1] = (const char*)g->T[1 - g->cur] + off * g->esize;
        b.rk = g->r ? g->r + off : nullptr;
        b.bf16 = g->storage == WFA_BF16;
        b.kvar = g->r != nullptr;
        for (int f = 0; f < 6; ++f) b.adv |= b.c.adv[f] != 0.0f;
        b.nbx = (g->n[0] + 4 * BX - 1) / (4 * BX);
        b.nby = (g->n[1] + BY - 1) / BY;
        b.nch = (g->n[2] + ZCHUNK - 1) / ZCHUNK;
        b.items = b.nbx * b.nby * b.nch;
        b.steps = steps[order[k]];
        prefix[k + 1] = prefix[k] + b.items;
    }
    // round r holds the grids with more than r steps: a prefix of the sorted list
    round_off[0] = 0;
    int active = ng;
    for (long long r = 0; r < max_steps; ++r) {
        while (active > 0 && bgs[active - 1].steps <= r) --active;
        round_off[r + 1] = round_off[r] + prefix[active];
    }
    h->ngrids = ng;
    h->max_steps = (int)max_steps;
    h->total_items = round_off[max_steps];
    const char* stall = getenv("WFA_TEST_BATCH_STALL");
    h->stall_grid = (stall && stall[0] == '1') ? 0 : -1;
    WFA_CUDA(cudaGraphLaunch(c->exec, st));
    int status = 0;
    WFA_CUDA(cudaMemcpyAsync(&status, c->done + c->cap_grids, sizeof(int), cudaMemcpyDeviceToHost, st));
    WFA_CUDA(cudaStreamSynchronize(st));
    for (int k = 0; k < ng; ++k) {
        wfa_grid g = gs[order[k]];
        const long long n = bgs[k].steps;
        if (!status) {
            g->cur = (int)((g->cur + n) & 1);
            g->steps_done += n;
        }
    }
    if (status) {
        set_error("wfa_batch_run: a device-side wait gave up after its time limit; the fields of these grids are "
                  "undefined (code %d)", status);
        return WFA_ERR_TIMEOUT;
    }
    return WFA_OK;
}
