// Layered decoder kernels with F16 message storage.
#include "decode_kernels.cuh"

namespace ldpcx {
namespace dec {

KernelFn layered_kernel_f16(int dmax, int algo, int zpt, bool qam) {
    constexpr int PREC = kF16;
    if (dmax > 20) return nullptr;
    if (zpt != 1) return nullptr;  // one check node per thread (two measured slower here: bank conflicts)
    if (algo == kMinSum) return dmax <= 12 ? layered_ch<12, kMinSum, PREC>(qam) : layered_ch<20, kMinSum, PREC>(qam);
    return dmax <= 12 ? layered_ch<12, kSpa, PREC>(qam) : layered_ch<20, kSpa, PREC>(qam);
}

KernelFn layered_kernel_zc_f16(int dmax, int algo, int Z, bool qam) {
    constexpr int PREC = kF16;
    if (algo != kMinSum || dmax > 20) return nullptr;
    if (Z == 384) return dmax <= 12 ? layered_ch<12, kMinSum, PREC, 384>(qam) : layered_ch<20, kMinSum, PREC, 384>(qam);
    return nullptr;
}

}  // namespace dec
}  // namespace ldpcx
