// Compiled sweep kernels: bf16 storage, uniform conductivity, depths 1..8.
#include "wfa_sweep_col.cuh"
#include "wfa_sweep_fused.cuh"
#include "wfa_sweep_t2.cuh"
#include "wfa_sweep_impl.cuh"

namespace wfa {

namespace {
using S = __nv_bfloat16;
constexpr bool KVAR = false;

// tile shape (EX, EY, R) per variant and depth, sized to the 227 KB of
// shared memory a block may hold (per-cell k keeps D + 4 k planes on chip)
// Shared-memory bytes per (x, y) column of the box: input ring (4 slots),
// k ring (D + 4 slots), one float plane per inner stage.
constexpr int col_bytes(int D) {
    return 4 * (int)sizeof(S) + (KVAR ? 4 * (D + 4) : 0) + 4 * (D - 1);
}
// Rows of the box: as many as fit the budget (two blocks per SM for depth
// <= 2, one block beyond), even, at most 64 and 512 threads, at least 2 D + 2.
constexpr int rows_for(int D, int EX) {
    const int budget = (D <= 2 ? 110 : 218) * 1024;
    int ey = budget / (col_bytes(D) * EX);
    const int ey_threads = ((D <= 2 ? 256 : 512) / (EX / 4)) * 2;   // threads: 2 blocks/SM for D <= 2
    ey = ey > 64 ? 64 : ey;
    ey = ey > ey_threads ? ey_threads : ey;
    ey -= ey % 2;
    return ey < 2 * D + 2 ? 2 * D + 2 : ey;
}

// Tile shapes; the output width TX = EX - 16 is a multiple of 128 bytes.
// Variant 1: EX = 80. Variant 2: EX = 144 where its smallest box fits the
// shared memory, else as variant 1.
template <int D>
TbEntry pick(int variant) {
    constexpr bool wide_fits = col_bytes(D) * 144 * (2 * D + 2) <= 218 * 1024;
    constexpr int WIDE = wide_fits ? 144 : 80;
    if (variant == 2) return make_entry<S, KVAR, D, WIDE, rows_for(D, WIDE), 2, 2>();
    return make_entry<S, KVAR, D, 80, rows_for(D, 80), 2, 2>();
}
}  // namespace

TbEntry tb_entry_bf16_u(int depth, int variant) {
    switch (depth) {
        case 1: return pick<1>(variant);
        case 2: return pick<2>(variant);
        case 3: return pick<3>(variant);
        case 4: return pick<4>(variant);
        case 5: return pick<5>(variant);
        case 6: return pick<6>(variant);
        case 7: return pick<7>(variant);
        default: return pick<8>(variant);
    }
}

cudaError_t launch_simple_bf16_u(const SweepArgs& a, cudaStream_t st) {
    return simple_launch<S, KVAR>(a, st);
}

cudaError_t launch_col_bf16_u(const SweepArgs& a, cudaStream_t st, int nsm, const cudaEvent_t* ev, bool inl, bool wide) {
    return col_launch<S, KVAR>(a, st, nsm, ev, inl, wide);
}

cudaError_t launch_col2_bf16_u(const SweepArgs& a, cudaStream_t st, int nsm, const cudaEvent_t* ev) {
    return col2_launch<S>(a, st, nsm, ev);
}

cudaError_t launch_t2_bf16_u(const CUtensorMap* tmT, const SweepArgs& a, cudaStream_t st, int nsm, const cudaEvent_t* ev) {
    return t2_launch<S>(tmT, a, st, nsm, ev);
}

}  // namespace wfa
