// Layered min-sum with check-node state and a compiled-in layer schedule
// (decode_cns_sched.cuh), f16 message format: both base-graph shapes,
// generic Z and Z = 384, one or two check nodes per thread; truncated codes
// (generic Z, one node per thread).
#include "decode_cns_sched.cuh"

namespace ldpcx {
namespace dec {

template <int BG>
SchedFn cns_sched_f16_bg(int Z, int k, bool trunc, bool qam) {
    if (trunc) return k_layered_cns_sched<BG, kF16, 0, 1, true>;
    if (k == 2) return Z == 384 ? k_layered_cns_sched<BG, kF16, 384, 2> : k_layered_cns_sched<BG, kF16, 0, 2>;
    if (qam) return Z == 384 ? k_layered_cns_sched<BG, kF16, 384, 1, false, kChAny>
                             : k_layered_cns_sched<BG, kF16, 0, 1, false, kChAny>;
    return Z == 384 ? k_layered_cns_sched<BG, kF16, 384, 1, false, kChLlr>
                    : k_layered_cns_sched<BG, kF16, 0, 1, false, kChLlr>;
}

SchedFn cns_sched_f16(int bg, int Z, int k, bool trunc, bool qam) {
    if (bg == 1) return cns_sched_f16_bg<1>(Z, k, trunc, qam);
    if (bg == 2) return cns_sched_f16_bg<2>(Z, k, trunc, qam);
    return nullptr;
}

}  // namespace dec
}  // namespace ldpcx
