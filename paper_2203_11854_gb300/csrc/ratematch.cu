// Circular-buffer rate matching of codewords and soft recovery of received
// LLRs (the rate matching of the 5G NR LDPC chain, with the start position and
// buffer size given by the caller). The buffer is the transmit layout: codeword
// positions from p0 on, without a shortened code's filler bits. Both are index work: one thread per output
// bit (ballot-packed per warp) and one thread per buffer position (a gather in
// increasing k, so no atomics and the sums run in a fixed order).
#include "common.cuh"

namespace ldpcx {
namespace {

struct RmParams {
    int64_t B;
    int p0, ncb, k0, E, qm, C;  // C = E / qm columns of the interleaver
    int k, nf;                  // a shortened code's filler positions k .. k + nf - 1 are not in the buffer
    int nw_in, nw_out;          // packed words per codeword in / out
};

// e index k -> transmitted position f: k = j C + i  ->  f = i qm + j.
__device__ __forceinline__ int64_t k_to_f(int64_t k, int C, int qm) { return (k % C) * qm + k / C; }

__global__ void __launch_bounds__(256) k_rate_match(const RmParams p, const uint32_t *__restrict__ cw,
                                                    uint32_t *__restrict__ out) {
    const int lane = threadIdx.x & 31;
    const int64_t words = p.B * p.nw_out;
    const int64_t warp0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t w = warp0; w < words; w += nwarps) {  // warp-uniform
        const int64_t b = w / p.nw_out;
        const int f = (int)(w - b * p.nw_out) * 32 + lane;
        bool bit = false;
        if (f < p.E) {
            const int i = f / p.qm, j = f - i * p.qm;  // f = i qm + j  <-  k = j C + i
            const int64_t k = (int64_t)j * p.C + i;
            const int pos = tx_position((int)((p.k0 + k) % p.ncb), p.p0, p.k, p.nf);
            bit = (cw[b * p.nw_in + (pos >> 5)] >> (pos & 31)) & 1u;
        }
        const unsigned word = __ballot_sync(0xFFFFFFFFu, bit);
        if (lane == 0) out[w] = word;
    }
}

__global__ void __launch_bounds__(256) k_rate_recover(const RmParams p, const float *__restrict__ llr,
                                                      float *__restrict__ out) {
    const int64_t total = p.B * p.ncb;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = t / p.ncb;
        const int q = (int)(t - b * p.ncb);
        // the k with (k0 + k) mod ncb = q, in increasing order
        int64_t k = q - p.k0;
        if (k < 0) k += p.ncb;
        float acc = 0.0f;
        for (; k < p.E; k += p.ncb) acc += llr[b * p.E + k_to_f(k, p.C, p.qm)];
        out[t] = acc;
    }
}

int rm_check(const ldpcx_code *c, int64_t B, int k0, int ncb, int E, int qm) {
    if (!c || B < 0) return LDPCX_E_INVAL;
    if (ncb < 1 || ncb > c->n - c->p0 - c->n_fill || k0 < 0 || k0 >= ncb || E < 1) return LDPCX_E_INVAL;
    if (!(qm == 1 || qm == 2 || qm == 4 || qm == 6 || qm == 8) || E % qm) return LDPCX_E_INVAL;
    return LDPCX_OK;
}

RmParams rm_params(const ldpcx_code *c, int64_t B, int k0, int ncb, int E, int qm) {
    RmParams p{};
    p.B = B;
    p.p0 = c->p0;
    p.k = c->k;
    p.nf = c->n_fill;
    p.ncb = ncb;
    p.k0 = k0;
    p.E = E;
    p.qm = qm;
    p.C = E / qm;
    p.nw_in = (c->n + 31) / 32;
    p.nw_out = (E + 31) / 32;
    return p;
}

}  // namespace
}  // namespace ldpcx

using namespace ldpcx;

extern "C" int rate_match(ldpcx_code_t c, const uint32_t *cw, int64_t B, int k0, int ncb, int E, int qm,
                          uint32_t *out, void *stream) {
    int st = rm_check(c, B, k0, ncb, E, qm);
    if (st) return st;
    if (B == 0) return LDPCX_OK;
    if (!cw || !out) return LDPCX_E_INVAL;
    const RmParams p = rm_params(c, B, k0, ncb, E, qm);
    const int64_t threads = p.B * p.nw_out * 32;
    int64_t blocks = (threads + 255) / 256;
    const int64_t cap = (int64_t)sm_count() * 8;
    if (blocks > cap) blocks = cap;
    k_rate_match<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(p, cw, out);
    return cuda_status(cudaGetLastError());
}

extern "C" int rate_recover(ldpcx_code_t c, const float *llr, int64_t B, int k0, int ncb, int E, int qm,
                            float *out, void *stream) {
    int st = rm_check(c, B, k0, ncb, E, qm);
    if (st) return st;
    if (B == 0) return LDPCX_OK;
    if (!llr || !out) return LDPCX_E_INVAL;
    const RmParams p = rm_params(c, B, k0, ncb, E, qm);
    int64_t blocks = (p.B * p.ncb + 255) / 256;
    const int64_t cap = (int64_t)sm_count() * 8;
    if (blocks > cap) blocks = cap;
    k_rate_recover<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(p, llr, out);
    return cuda_status(cudaGetLastError());
}
