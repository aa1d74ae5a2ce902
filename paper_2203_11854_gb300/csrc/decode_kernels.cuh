// Device code of the belief-propagation decoders (LDPC5GDecoder of the paper's
// Listing 1; min-sum BP as the custom CUDA op of Sec. IV-A), shared by the
// kernel translation units decode_*.cu.
//
// Mapping: one thread per (codeword, z): for every base row (layer) r, thread
// z owns check node r*Z + z. A base row touches each column at most once and
// every circulant is a bijection, so the check nodes of a layer touch disjoint
// variable nodes: a thread updates its check node with no communication, and
// one __syncthreads() separates layers. The APP array of each codeword lives
// in shared memory; the check-to-variable messages live in HBM in the
// circulant-contiguous layout msg[cw][blk*Z + z] (blk = nonzero base block in
// row-major order), so each block of a layer is one coalesced Z-wide stream,
// and the whole layer is one contiguous span. Each thread reads and writes only
// its own message slots, so messages need no synchronisation at all; the next
// layer's messages are loaded into registers while the current layer computes,
// and each layer runs a body specialised for its exact degree.
//
// Arithmetic is binary32 with explicit round-to-nearest intrinsics (no fused
// multiply-add), in the operation order of the decoder definition in ldpcx.h.
#pragma once

#include <math.h>

#include <type_traits>

#include "common.cuh"
#include "demap.cuh"

namespace ldpcx {
namespace dec {

enum { kMinSum = 0, kSpa = 1 };
enum { kF32 = LDPCX_MSG_F32, kF16 = LDPCX_MSG_F16, kFix6 = LDPCX_MSG_FIX6 };

template <int P> struct MsgT;
template <> struct MsgT<kF32> { using T = float; };
template <> struct MsgT<kF16> { using T = __half; };
template <> struct MsgT<kFix6> { using T = int8_t; };

template <int P> __device__ __forceinline__ float msg_load(const typename MsgT<P>::T *p);
template <> __device__ __forceinline__ float msg_load<kF32>(const float *p) { return __ldcg(p); }
template <> __device__ __forceinline__ float msg_load<kF16>(const __half *p) {
    return __half2float(__ushort_as_half(__ldcg(reinterpret_cast<const unsigned short *>(p))));
}
template <> __device__ __forceinline__ float msg_load<kFix6>(const int8_t *p) {
    return (float)(int)__ldcg(reinterpret_cast<const signed char *>(p)) * 0.5f;
}

// Round a message to its storage format; returns the value used by the decoder
// and writes the stored representation to *q.
template <int P> __device__ __forceinline__ float msg_round(float r, typename MsgT<P>::T *q);
template <> __device__ __forceinline__ float msg_round<kF32>(float r, float *q) {
    *q = r;
    return r;
}
template <> __device__ __forceinline__ float msg_round<kF16>(float r, __half *q) {
    *q = __float2half_rn(r);
    return __half2float(*q);
}
template <> __device__ __forceinline__ float msg_round<kFix6>(float r, int8_t *q) {
    int v = (int)rintf(r * 2.0f);  // step 0.5; rintf rounds half to even
    v = max(-31, min(31, v));
    *q = (int8_t)v;
    return (float)v * 0.5f;
}

template <int P> __device__ __forceinline__ void msg_store(typename MsgT<P>::T *p, typename MsgT<P>::T v);
template <> __device__ __forceinline__ void msg_store<kF32>(float *p, float v) { __stcg(p, v); }
template <> __device__ __forceinline__ void msg_store<kF16>(__half *p, __half v) {
    __stcg(reinterpret_cast<unsigned short *>(p), __half_as_ushort(v));
}
template <> __device__ __forceinline__ void msg_store<kFix6>(int8_t *p, int8_t v) {
    __stcg(reinterpret_cast<signed char *>(p), (signed char)v);
}

// phi(x) = -ln tanh(x/2) = ln(1 + 2/(e^x - 1)), for x > 0.
__device__ __forceinline__ float phi(float x) { return log1pf(__fdiv_rn(2.0f, expm1f(x))); }

// The same function from the hardware approximations of 2^x, 1/x and log2 x,
// for phi(clamp) <= x <= clamp. Where a difference of nearly equal numbers
// would cancel, the Taylor series is used instead:
//   e^x - 1 = x + x^2/2 + x^3/6 + x^4/24 + O(x^5)  for x < 1/16
//             (truncation below x^4/120 < 5e-7 relative),
//   ln(1+y) = y - y^2/2 + y^3/3 - y^4/4 + O(y^5)     for y < 1/16
//             (truncation below y^4/5 < 4e-6 relative).
// Otherwise e^x - 1 >= 0.064 loses at most a factor e^x/(e^x - 1) < 17 of the
// exponential's relative error, and ln(1+y) >= 0.06 is taken where log2 is
// accurate in absolute terms; the result stays within about 2e-5 relative.
//
// e^x = 2^(x log2 e), ln y = log2(y) ln 2 and 1/x come from the PTX ex2, lg2 and
// rcp approximations with subnormals flushed: for phi(clamp) <= x <= clamp
// every argument and result here (x, e^x, e^x - 1 >= x, 2/(e^x - 1) <= 2/x,
// 1 + y) is a normal binary32 number, so the flush changes no value.
constexpr float kLog2e = 1.44269504088896341f, kLn2 = 0.693147180559945309f;
__device__ __forceinline__ float hw_exp2(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float hw_log2(float x) {
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float hw_rcp(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float phi_fast(float x) {
    const float em1 = x < 0.0625f ? x * (1.0f + x * (0.5f + x * (1.0f / 6.0f + x * (1.0f / 24.0f))))
                                  : hw_exp2(x * kLog2e) - 1.0f;
    const float y = 2.0f * hw_rcp(em1);
    return y < 0.0625f ? y * (1.0f - y * (0.5f - y * (1.0f / 3.0f - y * 0.25f))) : hw_log2(1.0f + y) * kLn2;
}


struct Params {
    const uint32_t *blk;
    const int32_t *row_ptr;
    int Z, rows, nnz, n, k, n_tx, p0;
    int nf;                       // filler bits at positions k .. k + nf - 1 (known zeros, not transmitted)
    int iters, early_stop;
    float offset, clamp, phi_lo;  // phi_lo = phi(clamp)
    const float *llr;             // [B][n_tx]
    // fused demapper (llr unused when sym is set): received symbols [B][n_tx/m] (float2, or float for
    // m = 1), N0 [B] (sym_no_stride 1) or [1] (0), and demap_app's other arguments
    const float *sym;
    const float *sym_no;
    int64_t sym_no_stride;
    int qam_m, demap_method;
    float demap_clamp, qam_scale;
    void *msg;                    // [B][msg_stride]
    int64_t msg_stride;
    const float *weights;         // flooding: [iters][nnz] or null
    float *ckpt;                  // flooding: C^t checkpoints [iters-1][B][msg_stride] (FP32) or null
    int64_t ckpt_tstride;         // B * msg_stride
    int64_t ckpt_app_stride;      // floats per codeword of the APP checkpoints after the messages
    float *llr_out;               // [B][n] or null
    uint32_t *bits_out;           // [B][kw] or null
    int32_t *iters_out;           // [B] or null
    int64_t B;
    int G;                        // codewords per CTA
    int pf_dist;                  // L2 prefetch distance in layers (0 = off)
    int msg_size;                 // bytes per message
    unsigned int *status;         // device status word (LDPCX_FLAG_*)
    // Integer constants read from the parameter space, so that products with
    // them stay integer multiply-adds (FMA pipe) instead of being turned into
    // shifts and logic ops on the ALU pipe, which bounds the layered min-sum
    // kernels. one = 1, two = 2, four = 4, two22 = 2^22, two31 = 2^31, neg4z = -4Z.
    unsigned k_one, k_two, k_four, k_two22, k_two31, k_neg4z;
};

inline void set_int_constants(Params &p) {
    p.k_one = 1u;
    p.k_two = 2u;
    p.k_four = 4u;
    p.k_two22 = 1u << 22;
    p.k_two31 = 1u << 31;
    p.k_neg4z = (unsigned)(-4 * p.Z);
}

// Shared memory: app[G][n] (and a second APP array for flooding), blk[nnz],
// row_ptr[rows+1], flag[G], done[G].
__host__ __device__ inline size_t smem_bytes(const Params &p, int napp) {
    return sizeof(float) * (size_t)napp * p.G * p.n + sizeof(uint32_t) * p.nnz + sizeof(int32_t) * (p.rows + 1) +
           2 * sizeof(int) * p.G;
}

__device__ __forceinline__ float clamp_llr(float x, float c, bool &bad) {
    if (!(x == x)) {  // NaN
        bad = true;
        return 0.0f;
    }
    if (isinf(x)) bad = true;
    return fminf(fmaxf(x, -c), c);
}

__device__ __forceinline__ float4 clamp_llr4(float4 x, float c, bool &bad) {
    return make_float4(clamp_llr(x.x, c, bad) + 0.0f, clamp_llr(x.y, c, bad) + 0.0f, clamp_llr(x.z, c, bad) + 0.0f,
                       clamp_llr(x.w, c, bad) + 0.0f);
}

// Channel LLR of codeword position v (clamped; +0.0 for -0.0): punctured and
// untransmitted positions 0, filler bits of a shortened code +clamp (a known
// zero), the rest from the transmit layout.
__device__ __forceinline__ float channel_llr(const Params &p, int64_t cw, int v, bool &bad) {
    if (v >= p.k && v < p.k + p.nf) return p.clamp;
    const int t = v - p.p0 - (v >= p.k ? p.nf : 0);
    if (cw < p.B && v >= p.p0 && t < p.n_tx) return clamp_llr(p.llr[cw * p.n_tx + t], p.clamp, bad) + 0.0f;
    return 0.0f;
}

// The fused demapper: the channel LLRs of the CTA's codewords computed from
// the received symbols, the values demap_app writes (same arithmetic, then the
// decoder's clamp), placed as load_channel places them, so decoding is the same
// bit for bit as demap_app followed by the decoder. Out of line: one copy per
// translation unit instead of one per kernel (the kernels declare their Params
// __grid_constant__, so the function may take its address). The parameters are
// read once into registers (through the reference every shared-memory store
// would force them to be read again).
struct QamLoad {
    const float *y;  // this codeword's symbols
    float inv_n0, scale, dclamp, clamp;
    int S, p0, k, nf, method;
    bool vec;        // contiguous transmit layout from a 16-byte-aligned p0: vector stores
};
// The demapper's values are finite and within +-dclamp (fminf / fmaxf drop a NaN), so the decoder's clamp
// of its input reduces to min / max, or to nothing when dclamp <= clamp; + 0 maps -0 to +0 as it does.
__device__ __forceinline__ float qam_llr(float L, float clamp, bool clip) {
    return (clip ? fminf(fmaxf(L, -clamp), clamp) : L) + 0.0f;
}
template <int M>
__device__ __forceinline__ void qam_channel(const QamLoad q, float *a, bool &bad) {
    constexpr int W = M == 1 ? 1 : 2;  // floats per symbol
    constexpr int U = 8;               // symbols per thread in flight
    const int bd = blockDim.x;
    const bool clip = q.dclamp > q.clamp;
    for (int s0 = threadIdx.x; s0 < q.S; s0 += U * bd) {
        float v[U][W];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int s = s0 + u * bd;
#pragma unroll
            for (int w = 0; w < W; ++w) v[u][w] = 0.0f;
            if (s < q.S) {
                if constexpr (W == 1) {
                    v[u][0] = __ldcs(q.y + s);
                } else {
                    const float2 t = __ldcs(reinterpret_cast<const float2 *>(q.y) + s);
                    v[u][0] = t.x;
                    v[u][1] = t.y;
                }
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int s = s0 + u * bd;
            if (s >= q.S) break;
            float L[M];
            demap_symbol<M>(v[u][0], v[u][W - 1], q.inv_n0, q.scale, q.method, q.dclamp, L, bad);
#pragma unroll
            for (int j = 0; j < M; ++j) L[j] = qam_llr(L[j], q.clamp, clip);
            if (q.vec) {
                float *o = a + q.p0 + s * M;
                if constexpr (M == 4 || M == 8) {
#pragma unroll
                    for (int j = 0; j < M; j += 4)
                        *reinterpret_cast<float4 *>(o + j) = make_float4(L[j], L[j + 1], L[j + 2], L[j + 3]);
                } else if constexpr (M == 2 || M == 6) {
#pragma unroll
                    for (int j = 0; j < M; j += 2) *reinterpret_cast<float2 *>(o + j) = make_float2(L[j], L[j + 1]);
                } else {
                    o[0] = L[0];
                }
            } else {
#pragma unroll
                for (int j = 0; j < M; ++j) a[tx_position(s * M + j, q.p0, q.k, q.nf)] = L[j];
            }
        }
    }
}
__device__ __forceinline__ void load_channel_qam_body(const Params &p, float *app, int64_t cw_base) {
    const int G = p.G, n = p.n, k = p.k, nf = p.nf, p0 = p.p0, n_tx = p.n_tx, m = p.qam_m;
    const int64_t B = p.B;
    const float clamp = p.clamp;
    const float *sym = p.sym, *sym_no = p.sym_no;
    const bool per_cw = p.sym_no_stride != 0;
    // vector stores: no fillers to skip, p0 and the row length multiples of 4 floats (16-byte aligned rows)
    const bool vec = nf == 0 && ((p0 | n) & 3) == 0;
    QamLoad q{nullptr, 0.0f, p.qam_scale, p.demap_clamp, clamp, n_tx / m, p0, k, nf, p.demap_method, vec};
    unsigned int *status = p.status;
    bool bad = false;
    for (int g = 0; g < G; ++g) {
        const int64_t cw = cw_base + g;
        float *a = app + (size_t)g * n;
        // positions without a received bit: punctured and untransmitted (0), fillers (+clamp)
        for (int v = threadIdx.x; v < n; v += blockDim.x) {
            const bool fill = v >= k && v < k + nf;
            const int t = v - p0 - (v >= k ? nf : 0);
            if (fill) a[v] = clamp;
            else if (v < p0 || t >= n_tx || cw >= B) a[v] = 0.0f;
        }
        if (cw >= B) continue;
        q.inv_n0 = 1.0f / sym_no[per_cw ? cw : 0];
        q.y = sym + cw * q.S * (m == 1 ? 1 : 2);
        switch (m) {
            case 1: qam_channel<1>(q, a, bad); break;
            case 2: qam_channel<2>(q, a, bad); break;
            case 4: qam_channel<4>(q, a, bad); break;
            case 6: qam_channel<6>(q, a, bad); break;
            default: qam_channel<8>(q, a, bad); break;
        }
    }
    if (bad) latch(status, LDPCX_FLAG_NONFINITE);
}

static __device__ __noinline__ void load_channel_qam(const Params &p, float *app, int64_t cw_base) {
    load_channel_qam_body(p, app, cw_base);
}

// Load the channel LLRs of the CTA's codewords into app (placed: punctured and
// untransmitted positions are 0). When the row layout allows, 16-byte loads,
// four per thread in flight (streaming: the LLRs are read once).
__device__ __forceinline__ void load_channel_llr(const Params &p, float *app, int64_t cw_base) {
    bool bad = false;
    if (p.nf == 0 && ((p.p0 | p.n_tx | p.n) & 3) == 0 && (reinterpret_cast<uintptr_t>(p.llr) & 15u) == 0) {
        const int bd = blockDim.x, n4 = p.n_tx >> 2;
        for (int g = 0; g < p.G; ++g) {
            const int64_t cw = cw_base + g;
            float *a = app + (size_t)g * p.n;
            for (int v = threadIdx.x; v < p.p0; v += bd) a[v] = 0.0f;
            for (int v = p.p0 + p.n_tx + threadIdx.x; v < p.n; v += bd) a[v] = 0.0f;
            float4 *dst = reinterpret_cast<float4 *>(a + p.p0);
            if (cw >= p.B) {
                for (int i = threadIdx.x; i < n4; i += bd) dst[i] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                continue;
            }
            const float4 *src = reinterpret_cast<const float4 *>(p.llr + cw * p.n_tx);
            int i = threadIdx.x;
            for (; i + 3 * bd < n4; i += 4 * bd) {
                const float4 x0 = __ldcs(src + i), x1 = __ldcs(src + i + bd), x2 = __ldcs(src + i + 2 * bd),
                             x3 = __ldcs(src + i + 3 * bd);
                dst[i] = clamp_llr4(x0, p.clamp, bad);
                dst[i + bd] = clamp_llr4(x1, p.clamp, bad);
                dst[i + 2 * bd] = clamp_llr4(x2, p.clamp, bad);
                dst[i + 3 * bd] = clamp_llr4(x3, p.clamp, bad);
            }
            for (; i < n4; i += bd) dst[i] = clamp_llr4(__ldcs(src + i), p.clamp, bad);
        }
        if (bad) latch(p.status, LDPCX_FLAG_NONFINITE);
        return;
    }
    for (int g = 0; g < p.G; ++g) {
        const int64_t cw = cw_base + g;
        for (int v = threadIdx.x; v < p.n; v += blockDim.x) app[(size_t)g * p.n + v] = channel_llr(p, cw, v, bad);
    }
    if (bad) latch(p.status, LDPCX_FLAG_NONFINITE);
}

// The channel load of every decoder: from the received symbols (the fused
// demapper, out of line) or from the LLRs.
__device__ inline void load_channel(const Params &p, float *app, int64_t cw_base) {
    if (p.sym) {
        load_channel_qam(p, app, cw_base);
        return;
    }
    load_channel_llr(p, app, cw_base);
}

// The channel load chosen at compile time (kCh*): the per-edge kernels are
// built once per input kind, since holding the fused path at all costs their
// main loop about 9 %.
constexpr int kChAny = 0, kChLlr = 1, kChQam = 2;
template <int CH>
__device__ __forceinline__ void load_channel_as(const Params &p, float *app, int64_t cw_base) {
    if constexpr (CH == kChLlr) load_channel_llr(p, app, cw_base);
    else if constexpr (CH == kChQam) load_channel_qam_body(p, app, cw_base);
    else load_channel(p, app, cw_base);
}

// Shared-memory block table entry: (col * Z) << 16 | shift. Variable node of
// check node z of the block: col*Z + (z + shift) mod Z.
__device__ __forceinline__ int vn_at(uint32_t vb, int z, int Z) {
    int zz = z + (int)(vb & 0xFFFFu);
    zz -= (zz >= Z) ? Z : 0;
    return (int)(vb >> 16) + zz;
}

// min(|a|, |b|) with the sign bit sign(a) XOR sign(b) (inputs are never NaN).
__device__ __forceinline__ float min_xorsign_abs(float a, float b) {
    float d;
    asm("min.xorsign.abs.f32 %0, %1, %2;" : "=f"(d) : "f"(a), "f"(b));
    return d;
}

// Layered min-sum check node. The layered APP never holds -0.0 (the channel
// load maps -0.0 to +0.0, and T = APP - R, APP = T + R cannot create it), so the
// IEEE sign bit of T equals (T < 0) and the sign product is an XOR of sign bits.
// The message magnitude of edge j is m2 when |T_j| == m1, else m1: identical to
// "m2 at the first index of the minimum", because m2 == m1 when the minimum is tied.
template <int N> struct FastMinSum {
    float v1, v2;  // offset, floored and clamped smallest / second smallest |T|
    float m1;      // smallest |T|
    unsigned sx;   // XOR of the sign bits of T
    __device__ __forceinline__ void prepare(const float (&T)[N], int deg, float offset, float clamp) {
        // acc: magnitude = smallest |T| so far, sign bit = XOR of the sign bits
        // so far (min.xorsign.abs does both in one instruction)
        float acc = INFINITY, a2 = INFINITY;
#pragma unroll
        for (int j = 0; j < N; ++j) {
            if (j < deg) {
                a2 = fminf(a2, fmaxf(fabsf(acc), fabsf(T[j])));
                acc = min_xorsign_abs(acc, T[j]);
            }
        }
        const float a1 = fabsf(acc);
        sx = __float_as_uint(acc);
        m1 = a1;
        v1 = fminf(fmaxf(__fsub_rn(a1, offset), 0.0f), clamp);
        v2 = fminf(fmaxf(__fsub_rn(a2, offset), 0.0f), clamp);
    }
    __device__ __forceinline__ float value(float Tj) const {
        const float mag = (fabsf(Tj) == m1) ? v2 : v1;
        return __uint_as_float(__float_as_uint(mag) | ((sx ^ __float_as_uint(Tj)) & 0x80000000u));
    }
};

// phi in bits, g(x) = phi(x) / ln 2 = log2(1 + 2/(e^x - 1)), of an argument also
// given in bits (xb = x log2 e, so e^x = 2^xb): the approximations and series of
// phi_fast with the series' coefficients scaled, so that neither an input nor an
// output of it needs a multiplication by log2 e or ln 2.
//   e^x - 1 = xb (c1 + xb (c2 + xb (c3 + xb c4))), c_k = (ln 2)^k / k!, x < 1/16
//   log2(1 + y) = r (d1 + r (d2 + r (d3 + r d4))), y = 2r, r = 1/(e^x - 1) < 1/32
//             (2r - 2r^2 + 8r^3/3 - 4r^4 over ln 2)
// The truncation errors are those of phi_fast. Outside [phi(clamp), clamp] the
// value still lies on the right side of the clamp: e^x - 1 = 0 gives r = inf and
// g = inf; e^x = inf gives r = 0 and g = 0.
__device__ __forceinline__ float phi_bits(float xb) {
    constexpr float c1 = 0.693147180559945309f, c2 = 0.240226506959100712f, c3 = 0.0555041086648215800f,
                    c4 = 0.00961812910762847717f;
    constexpr float d1 = 2.88539008177792681f, d2 = -2.88539008177792681f, d3 = 3.84718677570390241f,
                    d4 = -5.77078016355585362f;
    const float em1 = xb < 0.0625f * kLog2e ? xb * (c1 + xb * (c2 + xb * (c3 + xb * c4))) : hw_exp2(xb) - 1.0f;
    const float r = hw_rcp(em1);
    return r < 0.03125f ? r * (d1 + r * (d2 + r * (d3 + r * d4))) : hw_log2(fmaf(2.0f, r, 1.0f));
}

// Layered sum-product check node on the variable-to-check inputs T[0..deg):
// R_j = s_j phi(sum_{i != j} phi(|T_i|)), every phi argument in [phi(clamp),
// clamp] (sum-product reading of the clamps), s_j the product of the other
// inputs' signs.
//  * The terms g_i = phi(|T_i|) are kept in bits; the exclusive sum of edge j is
//    s_rest + (g_max - g_j), where s_rest sums every term but the largest one
//    (each term is added as min(term, largest so far), the largest so far kept
//    apart): no term is ever subtracted from a sum that holds it, so nothing
//    cancels (g_max - g_j is exact for g_j >= g_max / 2, and at least g_max / 2
//    otherwise).
//  * Clamping the outer argument to [phi(clamp), clamp] equals clamping the
//    result to the same interval (phi is decreasing and its own inverse), so the
//    result is clamped instead; the inner arguments keep their clamp, which also
//    keeps every term finite.
//  * The layered T is never -0.0 (the channel load maps -0.0 to +0.0; x - x and
//    x + (-0.0) give +0.0 for x = +0.0), so the sign of T_j is its sign bit, the
//    sign product an XOR of sign bits, and s_j the sign bit of bits(T_j) + that
//    XOR (an addition flips bit 31 or not), formed by a multiply-add.
template <int N> struct SpaNode {
    float g[N];          // phi(|T_j|) in bits
    float s_rest, g_max; // sum of the terms without the largest one; the largest one
    unsigned sxs;        // XOR of the sign bits of T (bit 31)
    __device__ __forceinline__ void prepare(const float (&T)[N], int deg, float clamp, float phi_lo) {
        unsigned sx = 0;
        s_rest = 0.0f;
        g_max = 0.0f;
#pragma unroll
        for (int j = 0; j < N; ++j) {
            if (j < deg) {
                g[j] = phi_bits(fminf(fmaxf(fabsf(T[j]), phi_lo), clamp) * kLog2e);
                if (j == 0) {
                    g_max = g[0];
                } else {
                    s_rest = __fadd_rn(s_rest, fminf(g[j], g_max));
                    g_max = fmaxf(g_max, g[j]);
                }
                sx ^= __float_as_uint(T[j]);
            }
        }
        sxs = sx & 0x80000000u;
    }
    // magnitude of the message of edge j, clamped
    __device__ __forceinline__ float mag(int j, float clamp, float phi_lo) const {
        const float x = __fadd_rn(s_rest, __fsub_rn(g_max, g[j]));
        return fminf(fmaxf(phi_bits(x) * kLn2, phi_lo), clamp);
    }
    // message of edge j (input T_j), clamped, not yet rounded to the message format
    __device__ __forceinline__ float value(int j, float Tj, float clamp, float phi_lo, unsigned one) const {
        const float m = mag(j, clamp, phi_lo);
        const unsigned U = __float_as_uint(Tj) * one + sxs;
        return __uint_as_float((U & 0x80000000u) | __float_as_uint(m));
    }
};

// Write final outputs of the CTA's codewords from app.
__device__ inline void write_outputs(const Params &p, const float *app, int64_t cw_base, int iters_run, int g,
                                     bool active, int z0) {
    if (p.llr_out) {
        for (int gg = 0; gg < p.G; ++gg) {
            const int64_t cw = cw_base + gg;
            if (cw >= p.B) break;
            for (int v = threadIdx.x; v < p.n; v += blockDim.x) p.llr_out[cw * p.n + v] = app[(size_t)gg * p.n + v];
        }
    }
    if (p.bits_out) {
        const int kw = (p.k + 31) >> 5;
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
        for (int w = warp; w < p.G * kw; w += nwarps) {
            const int gg = w / kw, ww = w - gg * kw;
            const int pos = ww * 32 + lane;
            const bool bit = pos < p.k && app[(size_t)gg * p.n + pos] < 0.0f;
            const unsigned m = __ballot_sync(0xFFFFFFFFu, bit);
            const int64_t cw = cw_base + gg;
            if (lane == 0 && cw < p.B) p.bits_out[cw * kw + ww] = m;
        }
    }
    if (p.iters_out && active && z0 == 0) p.iters_out[cw_base + g] = iters_run;
}

// Parity of every check node of the thread's z over the current hard decisions.
__device__ __forceinline__ bool syndrome_bad(const Params &p, const uint32_t *s_vb, const int32_t *s_rp,
                                             const float *app, int z) {
    bool bad = false;
    for (int r = 0; r < p.rows; ++r) {
        unsigned par = 0;
        for (int b = s_rp[r]; b < s_rp[r + 1]; ++b) par ^= app[vn_at(s_vb[b], z, p.Z)] < 0.0f ? 1u : 0u;
        bad |= par != 0;
    }
    return bad;
}

// Copy the block table to shared memory as (col * Z) << 16 | shift.
__device__ __forceinline__ void load_tables(const Params &p, uint32_t *s_vb, int32_t *s_rp) {
    for (int i = threadIdx.x; i < p.nnz; i += blockDim.x) {
        const uint32_t b = p.blk[i];
        s_vb[i] = ((b >> 16) * (uint32_t)p.Z) << 16 | (b & 0xFFFFu);
    }
    for (int i = threadIdx.x; i <= p.rows; i += blockDim.x) s_rp[i] = p.row_ptr[i];
}

// Prefetch into L2 the message span of layer (r + dist) -- one contiguous span
// per codeword -- so that the register prefetch one layer ahead hits L2.
// Rounded out to 16-byte boundaries; the per-codeword stride is a multiple of
// 128 messages, so the rounded span stays inside the workspace.
__device__ __forceinline__ void l2_prefetch_layer(const Params &p, const int32_t *s_rp, int64_t cw_base, int r, int t) {
    int rr = r + p.pf_dist, tt = t;
    while (rr >= p.rows) {
        rr -= p.rows;
        ++tt;
    }
    if (tt < 1 || tt >= p.iters) return;  // iteration 0 reads no messages
    const char *base = reinterpret_cast<const char *>(p.msg);
    for (int gg = 0; gg < p.G; ++gg) {
        const int64_t cw = cw_base + gg;
        if (cw >= p.B) break;
        const int64_t e0 = cw * p.msg_stride + (int64_t)s_rp[rr] * p.Z;
        const int64_t e1 = cw * p.msg_stride + (int64_t)s_rp[rr + 1] * p.Z;
        const int64_t b0 = (e0 * p.msg_size) & ~(int64_t)15;
        const int64_t b1 = (e1 * p.msg_size + 15) & ~(int64_t)15;
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(base + b0), "r"((unsigned)(b1 - b0))
                     : "memory");
    }
}

// Message access for ZPT adjacent check nodes (z0 .. z0+ZPT-1, z0 a multiple
// of ZPT): one vector load / store per block. The per-codeword message stride
// is a multiple of 128 and Z is a multiple of ZPT, so the vectors are aligned.
template <int PREC, int ZPT> struct MsgVec;

template <int PREC> struct MsgVec<PREC, 1> {
    using MT = typename MsgT<PREC>::T;
    static __device__ __forceinline__ void load(const MT *p, float (&v)[1]) { v[0] = msg_load<PREC>(p); }
    // round r to the storage format, return the rounded values in rq, store when asked
    static __device__ __forceinline__ void round_store(MT *p, const float (&r)[1], float (&rq)[1], bool store) {
        MT q;
        rq[0] = msg_round<PREC>(r[0], &q);
        if (store) msg_store<PREC>(p, q);
    }
};

template <> struct MsgVec<kF32, 2> {
    static __device__ __forceinline__ void load(const float *p, float (&v)[2]) {
        const float2 x = __ldcg(reinterpret_cast<const float2 *>(p));
        v[0] = x.x;
        v[1] = x.y;
    }
    static __device__ __forceinline__ void round_store(float *p, const float (&r)[2], float (&rq)[2], bool store) {
        rq[0] = r[0];
        rq[1] = r[1];
        if (store) __stcg(reinterpret_cast<float2 *>(p), make_float2(r[0], r[1]));
    }
};

template <> struct MsgVec<kF16, 2> {
    static __device__ __forceinline__ void load(const __half *p, float (&v)[2]) {
        const unsigned int w = __ldcg(reinterpret_cast<const unsigned int *>(p));
        const float2 f = __half22float2(*reinterpret_cast<const __half2 *>(&w));
        v[0] = f.x;
        v[1] = f.y;
    }
    static __device__ __forceinline__ void round_store(__half *p, const float (&r)[2], float (&rq)[2], bool store) {
        const __half2 h = __floats2half2_rn(r[0], r[1]);  // round to nearest even, each half
        const float2 f = __half22float2(h);
        rq[0] = f.x;
        rq[1] = f.y;
        if (store) __stcg(reinterpret_cast<unsigned int *>(p), *reinterpret_cast<const unsigned int *>(&h));
    }
};

template <> struct MsgVec<kFix6, 2> {
    static __device__ __forceinline__ void load(const int8_t *p, float (&v)[2]) {
        const unsigned short w = __ldcg(reinterpret_cast<const unsigned short *>(p));
        v[0] = (float)(int)(signed char)(w & 0xFFu) * 0.5f;
        v[1] = (float)(int)(signed char)(w >> 8) * 0.5f;
    }
    static __device__ __forceinline__ void round_store(int8_t *p, const float (&r)[2], float (&rq)[2], bool store) {
        int8_t q0, q1;
        rq[0] = msg_round<kFix6>(r[0], &q0);
        rq[1] = msg_round<kFix6>(r[1], &q1);
        if (store)
            __stcg(reinterpret_cast<unsigned short *>(p),
                   (unsigned short)((unsigned)(uint8_t)q0 | ((unsigned)(uint8_t)q1 << 8)));
    }
};

// Variable node of check node z0 + k of a block: col*Z + (z0 + k + shift) mod Z.
template <int ZPT>
__device__ __forceinline__ void vn_vec(uint32_t vb, int z0, int Z, int (&v)[ZPT]) {
    int zz = z0 + (int)(vb & 0xFFFFu);
    zz -= (zz >= Z) ? Z : 0;
    const int colZ = (int)(vb >> 16);
    v[0] = colZ + zz;
#pragma unroll
    for (int k = 1; k < ZPT; ++k) {
        ++zz;
        zz = (zz == Z) ? 0 : zz;
        v[k] = colZ + zz;
    }
}

// Layers of degree up to kPf get an exact-degree body and have their messages
// prefetched into registers one layer ahead; denser layers (the four core rows
// of the 5G shapes) run one predicated body that loads its own messages.
constexpr int kPf = 8;

// Messages of one layer (D blocks, Z apart) into registers.
template <int D, int PREC, int ZPT>
__device__ __forceinline__ void load_layer(float (&R)[ZPT][kPf], const typename MsgT<PREC>::T *ml, int Z) {
#pragma unroll
    for (int j = 0; j < D; ++j) {
        float v[ZPT];
        MsgVec<PREC, ZPT>::load(ml + (size_t)j * Z, v);
#pragma unroll
        for (int k = 0; k < ZPT; ++k) R[k][j] = v[k];
    }
}

// Layered update of check nodes z0 .. z0+ZPT-1 of one layer of degree deg <= DM
// (D == 0: deg is a runtime value and the DM edge slots are predicated; else
// deg == D exactly). Rc holds the old messages (prefetched) when D > 0; the
// predicated body loads them itself (first iteration: zero).
// T = APP - R_old, check-node rule, APP = T + R_new (rounded), store R_new.
template <int D, int DM, int ALGO, int PREC, int ZPT, int ZC>
__device__ __forceinline__ void layer_update(const Params &p, int deg, float *app, const uint32_t *vb, int z0,
                                             typename MsgT<PREC>::T *ml, const float (&Rc)[ZPT][kPf], bool load,
                                             bool store) {
    const int ZV = ZC ? ZC : p.Z;  // lifting size (compile-time when ZC != 0)
    constexpr int N = D ? D : DM;
    constexpr bool kKeepIdx = D != 0;  // exact (sparse) bodies keep their indices in registers
    float T[ZPT][N];
    int vi[ZPT][kKeepIdx ? N : 1];
#pragma unroll
    for (int j = 0; j < N; ++j) {
        if (D || j < deg) {
            float old[ZPT];
            if (D) {
#pragma unroll
                for (int k = 0; k < ZPT; ++k) old[k] = Rc[k][j < kPf ? j : 0];
            } else if (load) {
                MsgVec<PREC, ZPT>::load(ml + (size_t)j * ZV, old);
            } else {
#pragma unroll
                for (int k = 0; k < ZPT; ++k) old[k] = 0.0f;
            }
            int v[ZPT];
            vn_vec<ZPT>(vb[j], z0, ZV, v);
#pragma unroll
            for (int k = 0; k < ZPT; ++k) {
                if constexpr (kKeepIdx) vi[k][j] = v[k];
                T[k][j] = __fsub_rn(app[v[k]], old[k]);
            }
        } else {
#pragma unroll
            for (int k = 0; k < ZPT; ++k) T[k][j] = 0.0f;
        }
    }
    using CN = typename std::conditional<ALGO == kMinSum, FastMinSum<N>, SpaNode<N>>::type;
    CN cn[ZPT];
#pragma unroll
    for (int k = 0; k < ZPT; ++k) {
        if constexpr (ALGO == kMinSum) cn[k].prepare(T[k], D ? D : deg, p.offset, p.clamp);
        else cn[k].prepare(T[k], D ? D : deg, p.clamp, p.phi_lo);
    }
#pragma unroll
    for (int j = 0; j < N; ++j) {
        if (D || j < deg) {
            float r[ZPT], rq[ZPT];
#pragma unroll
            for (int k = 0; k < ZPT; ++k) {
                if constexpr (ALGO == kMinSum) r[k] = cn[k].value(T[k][j]);
                else r[k] = cn[k].value(j, T[k][j], p.clamp, p.phi_lo, p.k_one);
            }
            MsgVec<PREC, ZPT>::round_store(ml + (size_t)j * ZV, r, rq, store);
            int v[ZPT];
            if constexpr (kKeepIdx) {
#pragma unroll
                for (int k = 0; k < ZPT; ++k) v[k] = vi[k][j];
            } else {
                vn_vec<ZPT>(vb[j], z0, ZV, v);  // dense body: recomputed, fewer live registers
            }
#pragma unroll
            for (int k = 0; k < ZPT; ++k) app[v[k]] = __fadd_rn(T[k][j], rq[k]);
        }
    }
}

// One layer step of the layered schedule: prefetch the next layer's messages
// into Rn (sparse layers), update layer r, then a block barrier.
template <int DMAX, int ALGO, int PREC, int ZPT, int ZC>
__device__ __forceinline__ void layered_step(const Params &p, const uint32_t *s_vb, const int32_t *s_rp, float *app,
                                             typename MsgT<PREC>::T *mp, int z0, int t, int r, bool done,
                                             int64_t cw_base, const float (&Rc)[ZPT][kPf], float (&Rn)[ZPT][kPf]) {
    const int ZV = ZC ? ZC : p.Z;  // lifting size (compile-time when ZC != 0)
    const int b0 = s_rp[r], deg = s_rp[r + 1] - b0;
    if (p.pf_dist > 0 && threadIdx.x == 0) l2_prefetch_layer(p, s_rp, cw_base, r, t);
    int rn = r + 1, tn = t;
    if (rn == p.rows) {
        rn = 0;
        tn = t + 1;
    }
    if (tn == 0) {
#pragma unroll
        for (int k = 0; k < ZPT; ++k)
#pragma unroll
            for (int j = 0; j < kPf; ++j) Rn[k][j] = 0.0f;  // iteration 0 starts from zero messages
    } else if (!done && tn < p.iters) {
        const int bn0 = s_rp[rn], degn = s_rp[rn + 1] - bn0;
        const auto *ml = mp + (size_t)bn0 * ZV;
        switch (degn) {
#define LDPCX_LOAD(d) \
    case d:           \
        load_layer<d, PREC, ZPT>(Rn, ml, ZV); \
        break;
            LDPCX_LOAD(1) LDPCX_LOAD(2) LDPCX_LOAD(3) LDPCX_LOAD(4)
            LDPCX_LOAD(5) LDPCX_LOAD(6) LDPCX_LOAD(7) LDPCX_LOAD(8)
#undef LDPCX_LOAD
            default: break;  // dense layer: loads its own messages
        }
    }
    if (!done) {
        const bool store = t + 1 < p.iters;  // the last iteration's messages are never read
        auto *ml = mp + (size_t)b0 * ZV;
        const uint32_t *vb = s_vb + b0;
        switch (deg) {
#define LDPCX_UPDATE(d) \
    case d:             \
        layer_update<d, d, ALGO, PREC, ZPT, ZC>(p, d, app, vb, z0, ml, Rc, t > 0, store); \
        break;
            LDPCX_UPDATE(1) LDPCX_UPDATE(2) LDPCX_UPDATE(3) LDPCX_UPDATE(4)
            LDPCX_UPDATE(5) LDPCX_UPDATE(6) LDPCX_UPDATE(7) LDPCX_UPDATE(8)
#undef LDPCX_UPDATE
            default:
                layer_update<0, DMAX, ALGO, PREC, ZPT, ZC>(p, deg, app, vb, z0, ml, Rc, t > 0, store);
                break;
        }
    }
    __syncthreads();
}

// Parity of the check nodes of z0 .. z0+ZPT-1 over the current hard decisions.
template <int ZPT, int ZC>
__device__ __forceinline__ bool syndrome_bad_vec(const Params &p, const uint32_t *s_vb, const int32_t *s_rp,
                                                 const float *app, int z0) {
    const int ZV = ZC ? ZC : p.Z;  // lifting size (compile-time when ZC != 0)
    bool bad = false;
    for (int r = 0; r < p.rows; ++r) {
        unsigned par[ZPT];
#pragma unroll
        for (int k = 0; k < ZPT; ++k) par[k] = 0;
        for (int b = s_rp[r]; b < s_rp[r + 1]; ++b) {
            int v[ZPT];
            vn_vec<ZPT>(s_vb[b], z0, ZV, v);
#pragma unroll
            for (int k = 0; k < ZPT; ++k) par[k] ^= app[v[k]] < 0.0f ? 1u : 0u;
        }
#pragma unroll
        for (int k = 0; k < ZPT; ++k) bad |= par[k] != 0;
    }
    return bad;
}

// Threads per CTA of the layered kernel: ZPT check nodes per thread.
template <int ZPT> constexpr int layered_threads() { return kMaxThreads / ZPT; }

// One tile of the layered schedule: the G codewords cw_base .. cw_base+G-1 of
// p, decoded by the whole CTA. Messages of codeword cw live at
// msg + (cw - msg_cw0) * msg_stride (msg_cw0 = 0: one slot per codeword of the
// batch; msg_cw0 = cw_base: one slot per codeword of the tile). CH: the
// channel load (kCh*).
template <int DMAX, int ALGO, int PREC, int ZPT, int ZC = 0, int CH = kChAny>
__device__ __forceinline__ void layered_tile(const Params &p, int64_t cw_base, int64_t msg_cw0,
                                             unsigned char *smem) {
    const int ZV = ZC ? ZC : p.Z;  // lifting size (compile-time when ZC != 0)
    using MT = typename MsgT<PREC>::T;
    float *s_app_all = reinterpret_cast<float *>(smem);
    uint32_t *s_vb = reinterpret_cast<uint32_t *>(s_app_all + (size_t)p.G * p.n);
    int32_t *s_rp = reinterpret_cast<int32_t *>(s_vb + p.nnz);
    int *s_flag = reinterpret_cast<int *>(s_rp + p.rows + 1);

    load_tables(p, s_vb, s_rp);
    load_channel_as<CH>(p, s_app_all, cw_base);

    const int zq = ZV / ZPT;  // threads per codeword
    const int g = threadIdx.x / zq, z0 = (threadIdx.x - g * zq) * ZPT;
    const int64_t cw = cw_base + g;
    const bool active = g < p.G && cw < p.B;
    float *app = s_app_all + (size_t)(active ? g : 0) * p.n;
    MT *mp = reinterpret_cast<MT *>(p.msg) + (active ? cw - msg_cw0 : 0) * p.msg_stride + z0;
    bool done = !active;
    int iters_run = 0;
    __syncthreads();

    // Ra / Rb alternate as current / prefetched messages (loop unrolled by two
    // layer steps so that no register copies are needed).
    float Ra[ZPT][kPf], Rb[ZPT][kPf];
#pragma unroll
    for (int k = 0; k < ZPT; ++k)
#pragma unroll
        for (int j = 0; j < kPf; ++j) Ra[k][j] = 0.0f;

    int t = 0, r = 0;
    // Advance to the next layer; at the end of an iteration run the early-stop
    // check. Returns true when every codeword of the CTA has stopped.
    auto advance = [&]() -> bool {
        if (++r < p.rows) return false;
        r = 0;
        if (!done) iters_run = t + 1;
        ++t;
        if (!p.early_stop) return false;
        if (threadIdx.x < p.G) s_flag[threadIdx.x] = 0;
        __syncthreads();
        if (!done && syndrome_bad_vec<ZPT, ZC>(p, s_vb, s_rp, app, z0)) s_flag[g] = 1;
        __syncthreads();
        if (!done && s_flag[g] == 0) done = true;
        return __syncthreads_and(done);
    };
    while (t < p.iters) {
        layered_step<DMAX, ALGO, PREC, ZPT, ZC>(p, s_vb, s_rp, app, mp, z0, t, r, done, cw_base, Ra, Rb);
        if (advance() || t >= p.iters) break;
        layered_step<DMAX, ALGO, PREC, ZPT, ZC>(p, s_vb, s_rp, app, mp, z0, t, r, done, cw_base, Rb, Ra);
        if (advance()) break;
    }
    __syncthreads();
    write_outputs(p, s_app_all, cw_base, iters_run, g, active, z0);
}

// ZC: compile-time lifting size (0 = the runtime p.Z); CH: channel input,
// LLRs (kChLlr) or received symbols (kChQam).
template <int DMAX, int ALGO, int PREC, int ZPT, int ZC = 0, int CH = kChLlr>
__global__ void __launch_bounds__(layered_threads<ZPT>(), 2) k_layered(const __grid_constant__ Params p) {
    extern __shared__ __align__(16) unsigned char smem[];
    layered_tile<DMAX, ALGO, PREC, ZPT, ZC, CH>(p, (int64_t)blockIdx.x * p.G, 0, smem);
}

using KernelFn = void (*)(Params);

// The per-edge kernel for an input kind (one check node per thread).
template <int DMAX, int ALGO, int PREC, int ZC = 0>
KernelFn layered_ch(bool qam) {
    return qam ? k_layered<DMAX, ALGO, PREC, 1, ZC, kChQam> : k_layered<DMAX, ALGO, PREC, 1, ZC, kChLlr>;
}

// Kernel lookup per translation unit (nullptr when the combination is not built).
// zpt: check nodes per thread (2 needs an even Z).
KernelFn layered_kernel_f32(int dmax, int algo, int zpt, bool qam = false);
KernelFn layered_kernel_f16(int dmax, int algo, int zpt, bool qam = false);
KernelFn layered_kernel_fix6(int dmax, int algo, int zpt, bool qam = false);
KernelFn flooding_kernel(int dmax, int algo, int prec);
// Shared memory of the flooding kernel: two APP arrays per codeword, the block
// table by rows and by columns with their row and column pointers, and three
// words per codeword.
__host__ __device__ inline size_t flood_smem_bytes(const Params &p) {
    return sizeof(float) * 2 * (size_t)p.G * p.n + sizeof(uint32_t) * 2 * (size_t)p.nnz +
           sizeof(int32_t) * (size_t)(p.rows + 1 + p.n / p.Z + 1) + 3 * sizeof(int) * (size_t)p.G;
}
// Threads per CTA of the flooding kernel: about one per variable node of its
// codewords, a multiple of 32 within 64..512.
inline int flood_threads(int G, int n) {
    const int64_t t = ((int64_t)G * n + 31) / 32 * 32;
    return t < 64 ? 64 : t > 512 ? 512 : (int)t;
}
// Layered min-sum kernels specialised for a compile-time lifting size (nullptr
// when none is built for Z): the hot loop's addresses become immediates.
KernelFn layered_kernel_zc_f32(int dmax, int algo, int Z, bool qam = false);
KernelFn layered_kernel_zc_f16(int dmax, int algo, int Z, bool qam = false);
KernelFn layered_kernel_zc_fix6(int dmax, int algo, int Z, bool qam = false);

}  // namespace dec
}  // namespace ldpcx
