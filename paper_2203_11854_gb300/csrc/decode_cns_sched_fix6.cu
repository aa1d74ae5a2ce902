// Layered min-sum with check-node state and a compiled-in layer schedule
// (decode_cns_sched.cuh), fix6 message format: both base-graph shapes,
// generic Z and Z = 384.
#include "decode_cns_sched.cuh"

namespace ldpcx {
namespace dec {

SchedFn cns_sched_fix6(int bg, int Z) {
    if (bg == 1) return Z == 384 ? k_layered_cns_sched<1, kFix6, 384> : k_layered_cns_sched<1, kFix6, 0>;
    if (bg == 2) return Z == 384 ? k_layered_cns_sched<2, kFix6, 384> : k_layered_cns_sched<2, kFix6, 0>;
    return nullptr;
}

}  // namespace dec
}  // namespace ldpcx
