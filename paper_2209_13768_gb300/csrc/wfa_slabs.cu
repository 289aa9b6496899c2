// One grid split into slabs along z (domain decomposition, Sec. 1, Fig. 1b;
// Sec. 2.1's 1 x 1 x Z columns, whose neighbour values come over the fabric
// for every product, Sec. 3).
//
// A slab is an ordinary grid whose z faces towards its neighbours are
// exchange faces (WFA_BC_EXCHANGE): the kernels read the neighbour's cells
// from the halo plane beyond such a face as they read any other neighbour,
// and nothing in the library writes that plane except an exchange. Before
// every step the outermost plane of each slab is copied into the halo plane
// of the slab across the face; then every slab takes one step. Because each
// cell sees the same operands as in the undivided grid, the slabs' fields are
// bitwise the undivided grid's (tests/test_gpu_slabs.py).
//
// Planes are whole padded planes (px * py elements: the x / y halo rides
// along, so periodic copies and ghost values in x and y arrive current).
// Between slabs on one device the copies are cudaMemcpyAsync calls ordered
// against both grids' streams; across devices or processes the caller moves
// the same planes (wfa_exchange_planes gives their addresses), e.g. with NCCL
// send / receive into the receiving GPU's own memory.
#include <string.h>

#include "wfa_internal.cuh"

namespace wfa {

static int fail_arg(int code, const char* msg) {
    set_error("%s", msg);
    return code;
}

// Issue the grid's queued halo and coefficient set-up work now (it would
// otherwise run at the next step): a plane received after this call is not
// touched again before the step reads it.
static int settle(wfa_grid_s* g) {
    if (g->halo_dirty) {
        int rc = refresh_halo(g, g->cur);
        if (rc) return rc;
        rc = prepare_coeff_halo(g);
        if (rc) return rc;
        g->halo_dirty = false;
    }
    return prepare_coeff_halo(g);
}

// Base of the padded array `what` refers to, and its element size.
static int plane_base(wfa_grid_s* g, int what, char** base, size_t* esize) {
    if (what == WFA_PLANES_FIELD) {
        *base = (char*)g->T[g->cur];
        *esize = (size_t)g->esize;
        return WFA_OK;
    }
    if (what == WFA_PLANES_K || what == WFA_PLANES_RECIP_K) {
        if (!g->k) return fail_arg(WFA_ERR_STATE, "no per-cell conductivity on this grid (uniform k needs no planes)");
        *base = (char*)(what == WFA_PLANES_K ? g->k : g->r);
        *esize = sizeof(float);
        return WFA_OK;
    }
    return fail_arg(WFA_ERR_ARG, "what must be WFA_PLANES_FIELD, WFA_PLANES_K or WFA_PLANES_RECIP_K");
}

static int planes(wfa_grid_s* g, int face, int what, void** send, void** recv, size_t* bytes) {
    if (face != WFA_ZLO && face != WFA_ZHI) return fail_arg(WFA_ERR_ARG, "face must be WFA_ZLO or WFA_ZHI");
    if (g->bc_kind[face] != WFA_BC_EXCHANGE) return fail_arg(WFA_ERR_BC, "the face is not an exchange face");
    int rc = settle(g);
    if (rc) return rc;
    char* base;
    size_t es;
    rc = plane_base(g, what, &base, &es);
    if (rc) return rc;
    const size_t plane = (size_t)g->px * g->py * es;
    // padded plane p holds z = p - HALO
    const long long own = face == WFA_ZLO ? HALO : HALO + g->n[2] - 1;
    const long long halo = face == WFA_ZLO ? HALO - 1 : HALO + g->n[2];
    if (send) *send = base + own * plane;
    if (recv) *recv = base + halo * plane;
    if (bytes) *bytes = plane;
    return WFA_OK;
}

static int device_of(const void* p, int* dev) {
    cudaPointerAttributes at;
    cudaError_t e = cudaPointerGetAttributes(&at, p);
    if (e != cudaSuccess) return cuda_fail(e, "cudaPointerGetAttributes");
    *dev = at.device;
    return WFA_OK;
}

static cudaError_t order_event(wfa_grid_s* g, cudaEvent_t* ev) {
    if (!g->xev) {
        cudaError_t e = cudaEventCreateWithFlags(&g->xev, cudaEventDisableTiming);
        if (e != cudaSuccess) return e;
    }
    *ev = g->xev;
    return cudaSuccess;
}

// lower's +z exchange face against upper's -z exchange face (lower == upper:
// one slab whose z axis wraps around).
static int exchange(wfa_grid_s* lo, wfa_grid_s* up, int what) {
    if (lo->n[0] != up->n[0] || lo->n[1] != up->n[1] || lo->px != up->px || lo->py != up->py ||
        lo->storage != up->storage)
        return fail_arg(WFA_ERR_ARG, "slabs of one grid need the same nx, ny and storage");
    if (what == WFA_PLANES_K && (!lo->k) != (!up->k))
        return fail_arg(WFA_ERR_ARG, "both slabs or neither need per-cell conductivity");
    if (what == WFA_PLANES_K && !lo->k) return WFA_OK;   // uniform k: nothing to move
    int dl = 0, du = 0;
    int rc = device_of(lo->T[0], &dl);
    if (rc) return rc;
    rc = device_of(up->T[0], &du);
    if (rc) return rc;
    if (dl != du) return fail_arg(WFA_ERR_ARG, "slabs on different devices: move wfa_exchange_planes yourself");
    const int kinds[2] = {what == WFA_PLANES_K ? WFA_PLANES_K : WFA_PLANES_FIELD, WFA_PLANES_RECIP_K};
    const int nk = what == WFA_PLANES_K ? 2 : 1;
    void *ls[2], *lr[2], *us[2], *ur[2];
    size_t bytes[2];
    for (int i = 0; i < nk; ++i) {
        rc = planes(lo, WFA_ZHI, kinds[i], &ls[i], &lr[i], &bytes[i]);
        if (rc) return rc;
        rc = planes(up, WFA_ZLO, kinds[i], &us[i], &ur[i], &bytes[i]);
        if (rc) return rc;
    }
    cudaStream_t st = lo->stream;
    if (up->stream != lo->stream) {   // the copies wait for upper's queued work
        cudaEvent_t ev;
        WFA_CUDA(order_event(up, &ev));
        WFA_CUDA(cudaEventRecord(ev, up->stream));
        WFA_CUDA(cudaStreamWaitEvent(st, ev, 0));
    }
    for (int i = 0; i < nk; ++i) {
        WFA_CUDA(cudaMemcpyAsync(ur[i], ls[i], bytes[i], cudaMemcpyDeviceToDevice, st));   // lower's top plane up
        WFA_CUDA(cudaMemcpyAsync(lr[i], us[i], bytes[i], cudaMemcpyDeviceToDevice, st));   // upper's bottom plane down
    }
    if (up->stream != lo->stream) {   // upper's next work waits for the copies
        cudaEvent_t ev;
        WFA_CUDA(order_event(lo, &ev));
        WFA_CUDA(cudaEventRecord(ev, st));
        WFA_CUDA(cudaStreamWaitEvent(up->stream, ev, 0));
    }
    if (what == WFA_PLANES_K) {   // the neighbour's conductivity enters both stability limits
        lo->limit_valid = false;
        up->limit_valid = false;
    }
    return WFA_OK;
}

}  // namespace wfa

using namespace wfa;

extern "C" {

int wfa_exchange_planes(wfa_grid g, int face, int what, void** send, void** recv, size_t* plane_bytes) {
    if (!g) return fail_arg(WFA_ERR_ARG, "NULL grid");
    return planes(g, face, what, send, recv, plane_bytes);
}

int wfa_exchange(wfa_grid lower, wfa_grid upper, int what) {
    NvtxRange nvtx_("wfa_exchange");
    if (!lower || !upper) return fail_arg(WFA_ERR_ARG, "NULL grid");
    if (what != WFA_PLANES_FIELD && what != WFA_PLANES_K)
        return fail_arg(WFA_ERR_ARG, "what must be WFA_PLANES_FIELD or WFA_PLANES_K");
    if (lower->bc_kind[WFA_ZHI] != WFA_BC_EXCHANGE || upper->bc_kind[WFA_ZLO] != WFA_BC_EXCHANGE)
        return fail_arg(WFA_ERR_BC, "lower's +z face and upper's -z face must be exchange faces");
    return exchange(lower, upper, what);
}

int wfa_slabs_step(wfa_grid* gs, int count, long long n) {
    NvtxRange nvtx_("wfa_slabs_step");
    if (!gs || count < 1) return fail_arg(WFA_ERR_ARG, "need at least one slab");
    if (n < 0) return fail_arg(WFA_ERR_ARG, "negative step count");
    for (int i = 0; i < count; ++i) {
        wfa_grid g = gs[i];
        if (!g) return fail_arg(WFA_ERR_ARG, "NULL slab");
        for (int j = 0; j < i; ++j)
            if (gs[j] == g) return fail_arg(WFA_ERR_ARG, "a slab appears twice");
        if (!g->field_set || !g->coeffs_set || !g->dt_set)
            return fail_arg(WFA_ERR_STATE, "set the field, the coefficients and dt of every slab first");
        if (g->dt != gs[0]->dt) return fail_arg(WFA_ERR_ARG, "the slabs of one grid need one dt");
        const bool last = i == count - 1;
        if (!last && (g->bc_kind[WFA_ZHI] != WFA_BC_EXCHANGE || gs[i + 1]->bc_kind[WFA_ZLO] != WFA_BC_EXCHANGE))
            return fail_arg(WFA_ERR_BC, "neighbouring slabs must meet at exchange faces");
    }
    const bool wrap = gs[0]->bc_kind[WFA_ZLO] == WFA_BC_EXCHANGE;
    if (wrap != (gs[count - 1]->bc_kind[WFA_ZHI] == WFA_BC_EXCHANGE))
        return fail_arg(WFA_ERR_BC, "a wrapping z axis needs exchange faces at both ends");
    // conductivity planes once per call (they change only with wfa_set_coeffs)
    for (int i = 0; i + 1 < count; ++i) {
        int rc = exchange(gs[i], gs[i + 1], WFA_PLANES_K);
        if (rc) return rc;
    }
    if (wrap) {
        int rc = exchange(gs[count - 1], gs[0], WFA_PLANES_K);
        if (rc) return rc;
    }
    for (long long s = 0; s < n; ++s) {
        for (int i = 0; i + 1 < count; ++i) {
            int rc = exchange(gs[i], gs[i + 1], WFA_PLANES_FIELD);
            if (rc) return rc;
        }
        if (wrap) {
            int rc = exchange(gs[count - 1], gs[0], WFA_PLANES_FIELD);
            if (rc) return rc;
        }
        for (int i = 0; i < count; ++i) {
            int rc = wfa_step(gs[i], 1);
            if (rc) return rc;
        }
    }
    return WFA_OK;
}

}  // extern "C"
