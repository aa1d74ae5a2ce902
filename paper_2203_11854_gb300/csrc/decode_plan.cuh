// Host side of ldpc_bp_decode shared with ldpc_bp_decode_noalloc: the choice
// of kernel for a code and its options (and the tuning knobs), the kernel
// parameters, and the launch. Both entry points run the same kernels with the
// same parameters, so they give the same results bit for bit; they differ
// only in where the code tables and the messages live.
#pragma once

#include "decode_edge_sched.cuh"

namespace ldpcx {
namespace dec {

struct DecodePlan {
    KernelFn fn = nullptr;  // row-table (or compile-time-Z) kernel, launched with Params only
    SchedFn sf = nullptr;   // compiled-schedule kernel (block table as a parameter), or null
    int kpt = 1;            // check nodes per thread of sf
    int zpt = 1;            // check nodes per thread of fn (layered)
    bool layered = false;
    bool cns = false;       // min-sum check-node state instead of per-edge messages
    int64_t state_bytes = 0;  // with cns: bytes of one codeword's state in the kernel's format
};

// Picks the kernel; LDPCX_E_UNSUPPORTED when none is built for the code. qam:
// the channel input is received symbols (ldpc_bp_decode_qam), which the
// per-edge kernels take in a build of their own.
int decode_plan(const ldpcx_code *c, const ldpcx_decode_opts *o, DecodePlan *pl, bool qam = false);

// Message (or check-node state) bytes one codeword needs under the plan.
int64_t decode_plan_bytes_per_cw(const ldpcx_code *c, const ldpcx_decode_opts *o, const DecodePlan &pl);

// Kernel parameters: tables blk / row_ptr on the device, messages of codeword
// cw at msg + cw * msg_stride * (bytes per message), checkpoints or null.
Params decode_params(const ldpcx_code *c, const uint32_t *blk, const int32_t *row_ptr, const float *llr_ch,
                     int64_t B, const ldpcx_decode_opts *o, float *llr_out, uint32_t *bits_out, int32_t *iters_out,
                     void *msg, int64_t msg_stride, float *ckpt, bool layered);

// Launches the planned kernel on `stream`.
int decode_launch(const DecodePlan &pl, const ldpcx_code *c, const Params &p, int64_t B, void *stream);

}  // namespace dec
}  // namespace ldpcx
