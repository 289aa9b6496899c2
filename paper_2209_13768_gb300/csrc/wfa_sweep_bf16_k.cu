// Compiled sweep kernels: bf16 storage, per-cell conductivity, depths 1..8.
#include "wfa_sweep_impl.cuh"

namespace wfa {

namespace {
using S = __nv_bfloat16;
constexpr bool KVAR = true;

// tile shape (EX, EY, R) per variant and depth, sized to the 227 KB of
// shared memory a block may hold (per-cell k keeps D + 4 k planes on chip)
template <int D>
TbEntry pick(int variant) {
    if (variant == 2) {
        constexpr int EX = (KVAR && D > 4) ? 96 : 128;
        constexpr int EY = D <= 2 ? 16 : (D <= 4 ? 24 : (KVAR ? 24 : 32));
        return make_entry<S, KVAR, D, EX, EY, 2>();
    }
    constexpr int EY = D <= 2 ? 32 : (D <= 4 ? 48 : (KVAR ? 32 : 64));
    return make_entry<S, KVAR, D, 64, EY, 2>();
}
}  // namespace

TbEntry tb_entry_bf16_k(int depth, int variant) {
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

cudaError_t launch_simple_bf16_k(const SweepArgs& a, cudaStream_t st) {
    return simple_launch<S, KVAR>(a, st);
}

}  // namespace wfa
