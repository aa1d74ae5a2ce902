// Flooding decoder kernels (weighted), all message formats.
#include "decode_kernels.cuh"

namespace ldpcx {
namespace dec {

template <int DMAX, int ALGO>
KernelFn flood_prec(int prec) {
    if (prec == kF32) return k_flooding<DMAX, ALGO, kF32>;
    if (prec == kF16) return k_flooding<DMAX, ALGO, kF16>;
    if constexpr (ALGO == kMinSum) return k_flooding<DMAX, kMinSum, kFix6>;
    return nullptr;
}

KernelFn flooding_kernel(int dmax, int algo, int prec) {
    if (dmax > 20) return nullptr;
    if (algo == kMinSum) return dmax <= 12 ? flood_prec<12, kMinSum>(prec) : flood_prec<20, kMinSum>(prec);
    return dmax <= 12 ? flood_prec<12, kSpa>(prec) : flood_prec<20, kSpa>(prec);
}

}  // namespace dec
}  // namespace ldpcx
