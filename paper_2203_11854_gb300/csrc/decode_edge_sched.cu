// Layered sum-product with per-edge messages and a compiled-in layer schedule
// (decode_edge_sched.cuh): both base-graph shapes, FP32 and FP16 messages,
// generic Z and Z = 384.
#include "decode_edge_sched.cuh"

namespace ldpcx {
namespace dec {

template <int BG, int PREC>
SchedFn edge_sched_for(int Z) {
    return Z == 384 ? k_layered_edge_sched<BG, kSpa, PREC, 384> : k_layered_edge_sched<BG, kSpa, PREC, 0>;
}

SchedFn layered_edge_sched_kernel(int bg, int algo, int prec, int Z) {
    if (algo != kSpa || (bg != 1 && bg != 2)) return nullptr;
    if (prec == kF32) return bg == 1 ? edge_sched_for<1, kF32>(Z) : edge_sched_for<2, kF32>(Z);
    if (prec == kF16) return bg == 1 ? edge_sched_for<1, kF16>(Z) : edge_sched_for<2, kF16>(Z);
    return nullptr;
}

}  // namespace dec
}  // namespace ldpcx
