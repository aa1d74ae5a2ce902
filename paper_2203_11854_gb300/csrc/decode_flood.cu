// Flooding decoder kernels (weighted), all message formats, one, two or four
// threads per check node.
#include "decode_kernels.cuh"

namespace ldpcx {
namespace dec {

template <int DMAX, int ALGO, int TPC>
KernelFn flood_prec(int prec) {
    if (prec == kF32) return k_flooding<DMAX, ALGO, kF32, TPC>;
    if (prec == kF16) return k_flooding<DMAX, ALGO, kF16, TPC>;
    if constexpr (ALGO == kMinSum) return k_flooding<DMAX, kMinSum, kFix6, TPC>;
    return nullptr;
}

template <int TPC>
KernelFn flood_tpc(int dmax, int algo, int prec) {
    if (algo == kMinSum) return dmax <= 12 ? flood_prec<12, kMinSum, TPC>(prec) : flood_prec<20, kMinSum, TPC>(prec);
    return dmax <= 12 ? flood_prec<12, kSpa, TPC>(prec) : flood_prec<20, kSpa, TPC>(prec);
}

KernelFn flooding_kernel(int dmax, int algo, int prec, int tpc) {
    if (dmax > 20) return nullptr;
    if (tpc == 4) return flood_tpc<4>(dmax, algo, prec);
    if (tpc == 2) return flood_tpc<2>(dmax, algo, prec);
    if (tpc == 1) return flood_tpc<1>(dmax, algo, prec);
    return nullptr;
}

}  // namespace dec
}  // namespace ldpcx
