// Internal declarations shared by the translation units of libldpcx.so.
// Nothing here is part of the C ABI (include/ldpcx.h is).
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>
#include <vector>

#include "ldpcx.h"

namespace ldpcx {

// Largest lifting size the kernels accept (one thread per check node of a
// layer, at most 384 threads per CTA).
constexpr int kMaxZ = 384;
constexpr int kMaxThreads = 384;

// Device-side view of a code's tables.
struct DevCode {
    const uint32_t *blk;      // [nnz] (col << 16) | shift, sorted by base row, then column
    const int32_t *row_ptr;   // [rows + 1] first block of each base row
    const uint32_t *core_inv; // [4Z][inv_words] GF(2) inverse of the core parity part, or null
};

// Encoder structure of a code: the transmitter handles base matrices whose
// core rows 0..3 touch only the systematic and the four core parity columns
// and whose extension row r touches, past those, only its own column kb + r.
constexpr int kEncNone = 0;      // not encodable by the transmitter
constexpr int kEncDualDiag = 1;  // the 5G dual-diagonal core: the recursion
constexpr int kEncCoreInv = 2;   // any invertible core: its inverse

}  // namespace ldpcx

// The opaque code object behind ldpcx_code_t.
struct ldpcx_code {
    ldpcx_code_params params;
    int Z, rows, cols, kb, nnz, max_deg, n, k, n_tx, p0;
    int n_fill = 0;                // filler bits at positions k .. k + n_fill - 1 (qc_ldpc_shorten)
    std::vector<int16_t> S;        // rows x cols base matrix, -1 = zero block
    std::vector<uint32_t> blk;     // nonzero blocks in row-major order
    std::vector<int32_t> row_ptr;  // rows + 1
    int enc = 0;                   // ldpcx::kEnc*
    int inv_words = 0;             // words per row of core_inv
    std::vector<uint32_t> core_inv;  // [4Z][inv_words] (kEncCoreInv)
    std::mutex mu;
    int dev = -1;                  // device the tables live on
    void *d_tables = nullptr;
    ldpcx::DevCode d{};
};

namespace ldpcx {

// Upload the code's tables to the current device on first use.
int code_device(ldpcx_code_t code, DevCode *out);

// Status words latched by the kernels of each translation unit.
unsigned int take_status_decode(cudaStream_t s);
// Device address of the decoders' status word on the current device.
unsigned int *status_word_decode();
// Bytes of the adjoint checkpoints for B codewords and `iters` iterations.
size_t ckpt_bytes(const ldpcx_code *c, int64_t B, int iters);
// Floats per codeword of the APP checkpoints that follow the message checkpoints.
inline int64_t ckpt_app_stride(int n) { return ((int64_t)n + 31) / 32 * 32; }
unsigned int take_status_channel(cudaStream_t s);

// Transmitter launch (source, encoder, mapper, AWGN); cw0_dev optional;
// y_out null: codewords only (packed into cw_out); points: a constellation by
// label instead of the Gray QAM.
int launch_tx(ldpcx_code_t c, uint64_t seed, uint64_t cw0, const uint64_t *cw0_dev, int64_t B, int m,
              const float *no, int64_t no_stride, float *y_out, uint32_t *info_out, cudaStream_t stream,
              uint32_t *cw_out = nullptr, const float *points = nullptr);

// Host fault injection (ldpcx_fault_set, LDPCX_FAULT): true when the armed
// one-shot allocation failure fires for this allocation.
bool fault_alloc();

// The codewords-per-CTA tuning knob (LDPCX_TUNE_CW_PER_CTA): 0 = automatic,
// else a cap on the codewords one CTA decodes together.
int tune_cw_per_cta();

// Per-device cached attribute: SM count.
int sm_count();

inline int cuda_status(cudaError_t e) { return e == cudaSuccess ? LDPCX_OK : LDPCX_E_CUDA; }

// Codeword position of transmitted bit t: the transmit layout starts at p0 and
// skips the n_fill filler positions k .. k + n_fill - 1 of a shortened code.
__host__ __device__ __forceinline__ int tx_position(int t, int p0, int k, int n_fill) {
    const int v = p0 + t;
    return v >= k ? v + n_fill : v;
}

// Set the device status word (atomic OR) -- used for conditions only the GPU sees.
__device__ __forceinline__ void latch(unsigned int *word, unsigned int flag) { atomicOr(word, flag); }

// Counter-based Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11): ten rounds of
//   (hi0, lo0) = 0xD2511F53 * c0, (hi1, lo1) = 0xCD9E8D57 * c2,
//   c <- (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0),
// with the key advanced by (0x9E3779B9, 0xBB67AE85) between rounds.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
    for (int i = 0; i < 10; ++i) {
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
        k.x += 0x9E3779B9u;
        k.y += 0xBB67AE85u;
    }
    return c;
}

// One 128-bit draw of the simulation: counter (q, cw lo, cw hi, stream), key = seed.
__device__ __forceinline__ uint4 draw(uint64_t seed, uint64_t cw, uint32_t stream, uint32_t q) {
    return philox4x32_10(make_uint4(q, (uint32_t)cw, (uint32_t)(cw >> 32), stream),
                         make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
}

// Box-Muller on one Philox word pair: u1 = ((a>>9)+0.5) 2^-23, u2 = (b>>8) 2^-24.
__device__ __forceinline__ float2 box_muller(uint32_t a, uint32_t b) {
    const float u1 = ((float)(a >> 9) + 0.5f) * (1.0f / 8388608.0f);
    const float u2 = (float)(b >> 8) * (1.0f / 16777216.0f);
    const float r = sqrtf(-2.0f * logf(u1));
    float s, c;
    sincospif(2.0f * u2, &s, &c);
    return make_float2(r * c, r * s);
}

}  // namespace ldpcx
