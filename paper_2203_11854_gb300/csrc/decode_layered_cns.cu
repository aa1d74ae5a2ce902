// Layered min-sum kernels with check-node state (decode_cns.cuh), generic and
// specialised for Z = 384, for FP32, FP16 and 6-bit message formats, and the
// lookup of the compiled-schedule variants (decode_cns_sched_*.cu).
#include "decode_cns_sched.cuh"

namespace ldpcx {
namespace dec {

template <int PREC>
KernelFn cns_for(int dmax, int Z) {
    if (Z == 384) return dmax <= 12 ? k_layered_cns<12, PREC, 384> : k_layered_cns<20, PREC, 384>;
    return dmax <= 12 ? k_layered_cns<12, PREC, 0> : k_layered_cns<20, PREC, 0>;
}

SchedFn cns_sched_f32(int bg, int Z, int k, bool trunc, bool qam);
SchedFn cns_sched_f16(int bg, int Z, int k, bool trunc, bool qam);
SchedFn cns_sched_fix6(int bg, int Z, int k, bool trunc, bool qam);

SchedFn layered_cns_sched_kernel(int bg, int prec, int Z, int k, bool trunc, bool qam) {
    if (prec == kF32) return cns_sched_f32(bg, Z, k, trunc, qam);
    if (prec == kF16) return cns_sched_f16(bg, Z, k, trunc, qam);
    return cns_sched_fix6(bg, Z, k, trunc, qam);
}

KernelFn layered_cns_kernel(int dmax, int prec, int Z) {
    if (dmax > 20) return nullptr;
    if (prec == kF32) return cns_for<kF32>(dmax, Z);
    if (prec == kF16) return cns_for<kF16>(dmax, Z);
    return cns_for<kFix6>(dmax, Z);
}

}  // namespace dec
}  // namespace ldpcx
