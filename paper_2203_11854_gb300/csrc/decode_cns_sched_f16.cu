// Layered min-sum with check-node state and a compiled-in layer schedule
// (decode_cns_sched.cuh), f16 message format: both base-graph shapes,
// generic Z and Z = 384.
#include "decode_cns_sched.cuh"

namespace ldpcx {
namespace dec {

SchedFn cns_sched_f16(int bg, int Z) {
    if (bg == 1) return Z == 384 ? k_layered_cns_sched<1, kF16, 384> : k_layered_cns_sched<1, kF16, 0>;
    if (bg == 2) return Z == 384 ? k_layered_cns_sched<2, kF16, 384> : k_layered_cns_sched<2, kF16, 0>;
    return nullptr;
}

}  // namespace dec
}  // namespace ldpcx
