// wfa_sum_f32_noalloc: the fp64 field-sum reduction of wfa_total_heat for a
// caller-owned dense device array, with its scratch (the per-block partial
// sums) in a fixed array that lives in the library's device image instead of
// memory allocated per call or per grid.
//
// Some callers cannot allocate device memory: a serving process that reserves
// all device memory in its own pool at start-up (a later cudaMalloc fails), a
// real-time loop where an allocation's implicit synchronisation and latency
// are not acceptable, or a plug-in inside a host framework that owns every
// device buffer. They pass the input and the output; this entry point needs
// nothing else.
#include <mutex>

#include "wfa_internal.cuh"

namespace {

constexpr int NA_THREADS = 256;
constexpr int NA_ITEMS = 64;                                              // elements per thread
constexpr long long NA_PER_BLOCK = (long long)NA_THREADS * NA_ITEMS;      // 16384 elements per block
constexpr int NA_MAX_BLOCKS = 8192;                                       // partial sums held: 64 KiB
constexpr long long NA_MAX_N = NA_PER_BLOCK * NA_MAX_BLOCKS;              // 2^27 elements (a 512^3 field)

// One fp64 partial per block. Every GPU that loads the library holds this
// array until the process exits; all calls share it.
static __device__ __align__(256) double g_na_partials[NA_MAX_BLOCKS];

// Block b sums elements [b * NA_PER_BLOCK, min(n, (b + 1) * NA_PER_BLOCK)) in a
// fixed order (thread t takes t, t + NA_THREADS, ...; then a fixed tree), so
// the result is bit-reproducible for a given n.
__global__ void __launch_bounds__(NA_THREADS) na_partial(const float* __restrict__ x, long long n,
                                                          double* __restrict__ partials) {
    __shared__ double sh[NA_THREADS];
    const long long base = blockIdx.x * NA_PER_BLOCK;
    double acc = 0.0;
#pragma unroll 4
    for (int k = 0; k < NA_ITEMS; ++k) {
        const long long i = base + threadIdx.x + (long long)k * NA_THREADS;
        if (i < n) acc += (double)x[i];
    }
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int s = NA_THREADS / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) partials[blockIdx.x] = sh[0];
}

// One block adds the nb partials in a fixed order and scales the sum.
__global__ void __launch_bounds__(1024) na_finish(const double* __restrict__ partials, int nb, double scale,
                                                  double* __restrict__ out) {
    __shared__ double sh[1024];
    double acc = 0.0;
    for (int i = threadIdx.x; i < nb; i += 1024) acc += partials[i];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int s = 512; s > 0; s >>= 1) {
        if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = sh[0] * scale;
}

// Device address of g_na_partials, looked up once per device with that
// device current. In host code the array's name is only a host-side stand-in.
// The address belongs to the device's current context: it is looked up again
// when the context changes (after cudaDeviceReset the library's device image
// is loaded afresh, possibly elsewhere).
constexpr int NA_MAX_DEVICES = 64;
std::mutex g_na_mu;
double* g_na_addr[NA_MAX_DEVICES] = {};
CUcontext g_na_ctx[NA_MAX_DEVICES] = {};

using CtxGetCurrent = CUresult (*)(CUcontext*);

CtxGetCurrent ctx_get_current() {
    static CtxGetCurrent fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (CtxGetCurrent)p;
    });
    return fn;
}

int partials_address(double** out) {
    int dev = 0;
    WFA_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= NA_MAX_DEVICES) {
        wfa::set_error("wfa_sum_f32_noalloc: device ordinal %d out of range", dev);
        return WFA_ERR_ARG;
    }
    // the current context (null on a thread the runtime has not bound to the
    // device yet: the lookup below binds it, and the context is read again)
    const CtxGetCurrent get = ctx_get_current();
    CUcontext ctx = nullptr;
    if (get && get(&ctx) != CUDA_SUCCESS) ctx = nullptr;
    std::lock_guard<std::mutex> lk(g_na_mu);
    if (!g_na_addr[dev] || !ctx || ctx != g_na_ctx[dev]) {
        void* p = nullptr;
        WFA_CUDA(cudaGetSymbolAddress(&p, g_na_partials));
        if (get && get(&ctx) != CUDA_SUCCESS) ctx = nullptr;
        g_na_addr[dev] = static_cast<double*>(p);
        g_na_ctx[dev] = ctx;
    }
    *out = g_na_addr[dev];
    return WFA_OK;
}

}  // namespace

extern "C" int wfa_sum_f32_noalloc(const float* d_x, long long n, double scale, double* d_out, void* stream) {
    if (!d_x || !d_out || n < 0) {
        wfa::set_error("wfa_sum_f32_noalloc: null pointer or negative size");
        return WFA_ERR_ARG;
    }
    if (n > NA_MAX_N) {
        wfa::set_error("wfa_sum_f32_noalloc: %lld elements exceed the maximum of %lld (%d partial sums of %lld)",
                       n, NA_MAX_N, NA_MAX_BLOCKS, NA_PER_BLOCK);
        return WFA_ERR_ARG;
    }
    double* partials = nullptr;
    int rc = partials_address(&partials);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    const int nb = (int)((n + NA_PER_BLOCK - 1) / NA_PER_BLOCK);
    if (nb > 0) na_partial<<<nb, NA_THREADS, 0, st>>>(d_x, n, partials);
    na_finish<<<1, 1024, 0, st>>>(partials, nb, scale, d_out);
    WFA_CUDA(cudaGetLastError());
    return WFA_OK;
}
