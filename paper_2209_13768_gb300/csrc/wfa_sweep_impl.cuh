// Host-side glue shared by the sweep instantiation units: one table entry per
// compiled (storage, conductivity mode, depth, tile shape) kernel.
#pragma once

#include "wfa_sweep.cuh"

namespace wfa {

using TbLaunchFn = cudaError_t (*)(const CUtensorMap* tmT, const CUtensorMap* tmK, const SweepArgs& a,
                                   int blocks, cudaStream_t st);
using TbOccFn = int (*)();

struct TbEntry {
    TbLaunchFn launch;
    TbOccFn occupancy;   // resident blocks per SM
    int ex, ey, r;       // TMA box / thread mapping
    int px, tx, ty;      // x halo and output tile
    int depth;
    size_t smem;
    int threads;
};

// Defined in wfa_sweep_{f32,bf16}_{u,k}.cu (u: uniform k, k: per-cell k).
// variant in [1, NUM_TILE_VARIANTS].
TbEntry tb_entry_f32_u(int depth, int variant);
TbEntry tb_entry_f32_k(int depth, int variant);
TbEntry tb_entry_bf16_u(int depth, int variant);
TbEntry tb_entry_bf16_k(int depth, int variant);
cudaError_t launch_simple_f32_u(const SweepArgs& a, cudaStream_t st);
cudaError_t launch_simple_f32_k(const SweepArgs& a, cudaStream_t st);
cudaError_t launch_simple_bf16_u(const SweepArgs& a, cudaStream_t st);
cudaError_t launch_simple_bf16_k(const SweepArgs& a, cudaStream_t st);
// one-step column-march kernel (variant 3; inl: variant 5, boundaries and
// periodic copies in the same launch); ev (may be null): events recorded just
// before and just after the main kernel, outside its fix-up kernels
cudaError_t launch_col_f32_u(const SweepArgs& a, cudaStream_t st, int nsm, const cudaEvent_t* ev, bool inl, bool wide);
cudaError_t launch_col_f32_k(const SweepArgs& a, cudaStream_t st, int nsm, const cudaEvent_t* ev, bool inl, bool wide);
cudaError_t launch_col_bf16_u(const SweepArgs& a, cudaStream_t st, int nsm, const cudaEvent_t* ev, bool inl, bool wide);
cudaError_t launch_col_bf16_k(const SweepArgs& a, cudaStream_t st, int nsm, const cudaEvent_t* ev, bool inl, bool wide);
// two steps per pass with TMA-staged input planes (variant 7, uniform k only);
// tmT: the input buffer's tensor map with an 80 x 20 box
cudaError_t launch_t2_f32_u(const CUtensorMap* tmT, const SweepArgs& a, cudaStream_t st, int nsm, const cudaEvent_t* ev);
cudaError_t launch_t2_bf16_u(const CUtensorMap* tmT, const SweepArgs& a, cudaStream_t st, int nsm, const cudaEvent_t* ev);
// two-step column-march kernel (variant 4, uniform k only)
cudaError_t launch_col2_f32_u(const SweepArgs& a, cudaStream_t st, int nsm, const cudaEvent_t* ev);
cudaError_t launch_col2_bf16_u(const SweepArgs& a, cudaStream_t st, int nsm, const cudaEvent_t* ev);

template <typename S, bool KVAR, int D, int EX, int EY, int R, int PF>
cudaError_t tb_launch(const CUtensorMap* tmT, const CUtensorMap* tmK, const SweepArgs& a, int blocks,
                      cudaStream_t st) {
    using Cfg = TbCfg<S, KVAR, D, EX, EY, R, PF>;
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(sweep_tb<S, KVAR, D, EX, EY, R, PF>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cfg::SMEM);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    sweep_tb<S, KVAR, D, EX, EY, R, PF><<<blocks, Cfg::NT, Cfg::SMEM, st>>>(*tmT, *tmK, a);
    return cudaGetLastError();
}

template <typename S, bool KVAR, int D, int EX, int EY, int R, int PF>
int tb_occupancy() {
    using Cfg = TbCfg<S, KVAR, D, EX, EY, R, PF>;
    static int occ = -1;
    if (occ < 0) {
        cudaFuncSetAttribute(sweep_tb<S, KVAR, D, EX, EY, R, PF>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)Cfg::SMEM);
        int n = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, sweep_tb<S, KVAR, D, EX, EY, R, PF>, Cfg::NT,
                                                          Cfg::SMEM) != cudaSuccess)
            n = 1;
        occ = n > 0 ? n : 1;
    }
    return occ;
}

template <typename S, bool KVAR, int D, int EX, int EY, int R, int PF>
TbEntry make_entry() {
    using Cfg = TbCfg<S, KVAR, D, EX, EY, R, PF>;
    TbEntry e;
    e.launch = &tb_launch<S, KVAR, D, EX, EY, R, PF>;
    e.occupancy = &tb_occupancy<S, KVAR, D, EX, EY, R, PF>;
    e.ex = EX; e.ey = EY; e.r = R;
    e.px = Cfg::PX; e.tx = Cfg::TX; e.ty = Cfg::TY;
    e.depth = D;
    e.smem = Cfg::SMEM;
    e.threads = Cfg::NT;
    return e;
}

template <typename S, bool KVAR>
cudaError_t simple_launch(const SweepArgs& a, cudaStream_t st) {
    dim3 block(32, 8);
    dim3 grid((a.c.n[0] + 31) / 32, (a.c.n[1] + 7) / 8);
    sweep_simple<S, KVAR><<<grid, block, 0, st>>>(a);
    return cudaGetLastError();
}

}  // namespace wfa
