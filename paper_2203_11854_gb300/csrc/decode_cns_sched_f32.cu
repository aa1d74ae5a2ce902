// Layered min-sum with check-node state and a compiled-in layer schedule
// (decode_cns_sched.cuh), f32 message format: both base-graph shapes,
// generic Z and Z = 384.
#include "decode_cns_sched.cuh"

namespace ldpcx {
namespace dec {

SchedFn cns_sched_f32(int bg, int Z) {
    if (bg == 1) return Z == 384 ? k_layered_cns_sched<1, kF32, 384> : k_layered_cns_sched<1, kF32, 0>;
    if (bg == 2) return Z == 384 ? k_layered_cns_sched<2, kF32, 384> : k_layered_cns_sched<2, kF32, 0>;
    return nullptr;
}

}  // namespace dec
}  // namespace ldpcx
