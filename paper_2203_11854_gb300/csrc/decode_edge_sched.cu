// Layered sum-product with per-edge messages and a compiled-in layer schedule
// (decode_edge_sched.cuh): both base-graph shapes, FP32 and FP16 messages,
// generic Z and Z = 384.
#include "decode_edge_sched.cuh"

namespace ldpcx {
namespace dec {

template <int BG, int PREC>
SchedFn edge_sched_for(int Z, bool qam) {
    if (qam)
        return Z == 384 ? k_layered_edge_sched<BG, kSpa, PREC, 384, kChAny> : k_layered_edge_sched<BG, kSpa, PREC, 0, kChAny>;
    return Z == 384 ? k_layered_edge_sched<BG, kSpa, PREC, 384, kChLlr> : k_layered_edge_sched<BG, kSpa, PREC, 0, kChLlr>;
}

SchedFn layered_edge_sched_kernel(int bg, int algo, int prec, int Z, bool qam) {
    if (algo != kSpa || (bg != 1 && bg != 2)) return nullptr;
    if (prec == kF32) return bg == 1 ? edge_sched_for<1, kF32>(Z, qam) : edge_sched_for<2, kF32>(Z, qam);
    if (prec == kF16) return bg == 1 ? edge_sched_for<1, kF16>(Z, qam) : edge_sched_for<2, kF16>(Z, qam);
    return nullptr;
}

}  // namespace dec
}  // namespace ldpcx
