// Monte-Carlo transmitter (BinarySource -> LDPC5GEncoder -> Mapper -> AWGN of
// the paper's Listing 1), APP demapper (Demapper("app")) and error counting
// (compute_ber), all on the device.
#include <math.h>

#include <algorithm>

#include "common.cuh"
#include "demap.cuh"

namespace ldpcx {
namespace {

__device__ unsigned int g_status;

struct TxParams {
    const uint32_t *blk;
    const int32_t *row_ptr;
    int Z, rows, kb, n, k, n_tx, p0, nnz;
    int nf;                    // filler bits at positions k .. k + nf - 1 (0, known, not transmitted)
    const uint32_t *core_inv;  // [4Z][inv_words] inverse of the core parity part, or null (dual diagonal)
    int inv_words;
    int m;
    float scale;         // 1/sqrt(2(4^h-1)/3): unit average symbol energy
    uint64_t seed, cw0;
    const uint64_t *cw0_dev;  // when set, *cw0_dev is added to cw0 (graph replays: the host writes it per batch)
    const float *no;
    int64_t no_stride;
    float *y;            // [B][S][2] or [B][S]
    uint32_t *info;      // [B][kw] or null
    uint32_t *cw_out;    // [B][ceil(n/32)] packed codeword bits or null
    const float2 *points;  // [2^m] constellation by label (MSB first), or null for the Gray QAM
    int64_t B;
    int G;               // codewords per CTA
};

constexpr int kTxThreads = 256;

// Gray PAM level of h label bits at stride 2 of `bits` from bit `off` (I: 0,
// Q: 1), label bit i at bit i of the word:
// A = (1-2a0)(2^(h-1) - (1-2a1)(2^(h-2) - ... (1-2a_{h-1}))).
__device__ __forceinline__ int pam_level(uint32_t bits, int h, int off) {
    int inner = 1 - 2 * (int)((bits >> (2 * (h - 1) + off)) & 1u);
    for (int i = h - 2; i >= 0; --i) inner = (1 - 2 * (int)((bits >> (2 * i + off)) & 1u)) * ((1 << (h - 1 - i)) - inner);
    return inner;
}

// k_tx keeps each codeword's bits packed, position v at bit v & 31 of word
// v >> 5, so one circulant block of a parity check is a word-wide rotation (a
// funnel shift of two words) instead of Z one-byte loads.
// Shared memory, per CTA: the block table as {column, shift} pairs and the row
// pointers, then per codeword its nLw packed words (n positions plus a padding
// word that windows read past the end), the four core-row sums lambda (4 Wz
// words; Wz = words of one block column) and, for a general core, lambda as one
// 4Z-bit vector (inv_words words).
struct TxLayout {
    int nLw, Wz, per_cw;  // words
    size_t cw_off;        // bytes before the first codeword
    size_t bytes;
};
__host__ __device__ inline TxLayout tx_layout(int G, int n, int Z, int nnz, int rows, int inv_words) {
    TxLayout t;
    t.nLw = ((n + 31) >> 5) + 1;
    t.Wz = (Z + 31) >> 5;
    t.per_cw = t.nLw + 4 * t.Wz + inv_words;
    t.cw_off = (8 * (size_t)nnz + 4 * (size_t)(rows + 1) + 15) & ~(size_t)15;
    t.bytes = t.cw_off + 4 * (size_t)G * t.per_cw;
    return t;
}

// 32 positions of a packed codeword from position pos (pos + 32 may pass the
// last position by less than one word).
__device__ __forceinline__ uint32_t tx_window(const uint32_t *L, int pos) {
    return __funnelshift_r(L[pos >> 5], L[(pos >> 5) + 1], pos & 31);
}

// Word j of block column `col` rotated by s: bit i = position col Z + (32 j + i
// + s) mod Z, for i < min(32, Z - 32 j) (the bits above are unspecified). The
// range of i wraps past the column's end at most once.
__device__ __forceinline__ uint32_t tx_rot(const uint32_t *L, int col, int s, int j, int Z) {
    int a = 32 * j + s;
    if (a >= Z) a -= Z;
    const int base = col * Z, n1 = Z - a;  // n1 positions before the wrap
    uint32_t w = tx_window(L, base + a);
    if (n1 < 32) w = (w & ((1u << n1) - 1u)) | (tx_window(L, base) << n1);
    return w;
}

// Writes bits 0 .. min(32, Z - 32 j) - 1 of v to positions col Z + 32 j ... of
// L, whose bits there are zero: a word shared with another column takes an
// atomic OR, a word of its own a plain store.
__device__ __forceinline__ void tx_put(uint32_t *L, int col, int j, uint32_t v, int Z) {
    const int nv = min(32, Z - 32 * j);
    if (nv < 32) v &= (1u << nv) - 1u;
    const int pos = col * Z + 32 * j, w = pos >> 5, o = pos & 31;
    if (o == 0 && nv == 32) {
        L[w] = v;
        return;
    }
    atomicOr(&L[w], v << o);
    if (o + nv > 32) atomicOr(&L[w + 1], v >> (32 - o));
}

// The m label bits of symbol s (label bit j at bit j): transmitted positions
// m s .. m s + m - 1 in the transmit layout (from p0, the fillers skipped).
__device__ __forceinline__ uint32_t tx_symbol_bits(const uint32_t *L, int s, int m, int p0, int k, int nf) {
    const int v = p0 + s * m, before = k - v;  // positions ahead of the fillers
    uint32_t w;
    if (nf == 0 || before >= m) w = tx_window(L, v);
    else if (before <= 0) w = tx_window(L, v + nf);
    else w = (tx_window(L, v) & ((1u << before) - 1u)) | (tx_window(L, v + nf) & ~((1u << before) - 1u));
    return w & ((1u << m) - 1u);
}

__global__ void __launch_bounds__(kTxThreads) k_tx(const TxParams p) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int Z = p.Z;
    const TxLayout lay = tx_layout(p.G, p.n, Z, p.nnz, p.rows, p.inv_words);
    const int nLw = lay.nLw, Wz = lay.Wz;
    const int kw = (p.k + 31) >> 5;
    const int nq = (kw + 3) >> 2;  // Philox blocks of source bits per codeword
    int2 *s_tab = reinterpret_cast<int2 *>(smem);  // [nnz] {column, shift}
    int32_t *s_rp = reinterpret_cast<int32_t *>(s_tab + p.nnz);
    uint32_t *s_cw = reinterpret_cast<uint32_t *>(smem + lay.cw_off);  // [G][per_cw]
    const int64_t cw_base = (int64_t)blockIdx.x * p.G;
    const int G = p.B - cw_base < p.G ? (int)(p.B - cw_base) : p.G;  // codewords of this CTA
    const uint64_t cw0 = p.cw0 + (p.cw0_dev ? *p.cw0_dev : 0ull);
    const int T = blockDim.x, tid = threadIdx.x;
    auto Lp = [&](int gg) { return s_cw + (size_t)gg * lay.per_cw; };
    auto lam = [&](int gg) { return Lp(gg) + nLw; };       // [4][Wz]
    auto lin = [&](int gg) { return Lp(gg) + nLw + 4 * Wz; };  // [inv_words]

    for (int i = tid; i < p.nnz; i += T) {
        const uint32_t bb = p.blk[i];
        s_tab[i] = make_int2((int)(bb >> 16), (int)(bb & 0xFFFFu));
    }
    for (int i = tid; i <= p.rows; i += T) s_rp[i] = p.row_ptr[i];
    // source bits (Philox stream 0) to the output and to words 0 .. kw - 1; every later word
    // (fillers, parity, padding) and the lambda vector start at zero
    for (int gg = 0; gg < G; ++gg) {
        const int64_t cw = cw_base + gg;
        uint32_t *L = Lp(gg);
        for (int q = tid; q < nq; q += T) {
            const uint4 x = draw(p.seed, cw0 + (uint64_t)cw, 0u, (uint32_t)q);
            const uint32_t w4[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int w = 4 * q + e;
                if (w >= kw) break;
                uint32_t word = w4[e];
                const int valid = min(32, p.k - 32 * w);
                if (valid < 32) word &= (1u << valid) - 1u;
                if (p.info) p.info[cw * kw + w] = word;
                L[w] = word;
            }
        }
        for (int w = kw + tid; w < nLw; w += T) L[w] = 0u;
        for (int w = tid; w < p.inv_words; w += T) lin(gg)[w] = 0u;
    }
    __syncthreads();

    // lambda_r = sum over the systematic blocks of core row r, word by word
    for (int i = tid; i < G * 4 * Wz; i += T) {
        const int gg = i / (4 * Wz), rj = i - gg * 4 * Wz, r = rj / Wz, j = rj - r * Wz;
        const uint32_t *L = Lp(gg);
        uint32_t acc = 0u;
        for (int b = s_rp[r]; b < s_rp[r + 1]; ++b) {
            const int2 e = s_tab[b];
            if (e.x < p.kb) acc ^= tx_rot(L, e.x, e.y, j, Z);
        }
        lam(gg)[rj] = acc;
        if (p.core_inv) tx_put(lin(gg), r, j, acc, Z);  // bit r Z + z of the 4Z-bit vector
    }
    __syncthreads();
    if (p.core_inv) {
        // core parity p = H_core^-1 lambda: bit i of p (position kb Z + i) is the parity of row i of the
        // inverse AND lambda
        const int N = 4 * Z;
        for (int i = tid; i < G * N; i += T) {
            const int gg = i / N, b = i - gg * N;
            const uint32_t *row = p.core_inv + (size_t)b * p.inv_words, *lw = lin(gg);
            uint32_t x = 0u;
            for (int w = 0; w < p.inv_words; ++w) x ^= __ldg(row + w) & lw[w];
            if (__popc(x) & 1) {
                const int v = p.kb * Z + b;
                atomicOr(&Lp(gg)[v >> 5], 1u << (v & 31));
            }
        }
    } else {
        // the 5G dual-diagonal core: the core rows sum to [I 0 0 0], so p_a = sum of the lambdas
        for (int i = tid; i < G * Wz; i += T) {
            const int gg = i / Wz, j = i - gg * Wz;
            const uint32_t *l = lam(gg);
            tx_put(Lp(gg), p.kb, j, l[j] ^ l[Wz + j] ^ l[2 * Wz + j] ^ l[3 * Wz + j], Z);
        }
        __syncthreads();
        for (int i = tid; i < G * Wz; i += T) {
            const int gg = i / Wz, j = i - gg * Wz;
            const uint32_t *l = lam(gg);
            uint32_t *L = Lp(gg);
            const uint32_t pa = l[j] ^ l[Wz + j] ^ l[2 * Wz + j] ^ l[3 * Wz + j];
            const uint32_t pb = l[j] ^ tx_rot(L, p.kb, 1, j, Z);  // row 0: P^1 p_a + p_b
            const uint32_t pc = l[Wz + j] ^ pa ^ pb;                // row 1: p_a + p_b + p_c
            const uint32_t pd = l[2 * Wz + j] ^ pc;                 // row 2: p_c + p_d
            tx_put(L, p.kb + 1, j, pb, Z);
            tx_put(L, p.kb + 2, j, pc, Z);
            tx_put(L, p.kb + 3, j, pd, Z);
        }
    }
    __syncthreads();
    // extension rows read only columns below kb + 4, so they are independent: check z of row r holds
    // its own column's position (z + s_own) mod Z, so own-column bit v sums the other blocks rotated
    // by s - s_own
    {
        const int items = (p.rows - 4) * Wz;
        for (int i = tid; i < G * items; i += T) {
            const int gg = i / items, rj = i - gg * items, r = 4 + rj / Wz, j = rj - (r - 4) * Wz;
            const int own = p.kb + r;
            int s_own = 0;
            for (int b = s_rp[r]; b < s_rp[r + 1]; ++b)
                if (s_tab[b].x == own) s_own = s_tab[b].y;
            uint32_t *L = Lp(gg);
            uint32_t acc = 0u;
            for (int b = s_rp[r]; b < s_rp[r + 1]; ++b) {
                const int2 e = s_tab[b];
                if (e.x == own) continue;
                int s = e.y - s_own;
                if (s < 0) s += Z;
                acc ^= tx_rot(L, e.x, s, j, Z);
            }
            tx_put(L, own, j, acc, Z);
        }
    }
    __syncthreads();

    // the codewords themselves, packed 32 positions per word (positions past n are zero)
    if (p.cw_out) {
        const int nw = (p.n + 31) >> 5;
        for (int i = tid; i < G * nw; i += T) {
            const int gg = i / nw, w = i - gg * nw;
            p.cw_out[(cw_base + gg) * nw + w] = Lp(gg)[w];
        }
    }
    if (!p.y) return;

    // Gray mapping and AWGN (Philox stream 1): four real or two complex symbols per draw; y = fma(sd, n, x)
    // in every mapper kernel, so k_tx and k_map_awgn agree bit for bit
    const int m = p.m, S = p.n_tx / m;
    const int per = m == 1 ? 4 : 2, nqs = (S + per - 1) / per;
    for (int gg = 0; gg < G; ++gg) {
        const int64_t cw = cw_base + gg;
        const uint32_t *L = Lp(gg);
        const float sd = sqrtf(p.no[cw * p.no_stride] * 0.5f);
        for (int q = tid; q < nqs; q += T) {
            const uint4 x = draw(p.seed, cw0 + (uint64_t)cw, 1u, (uint32_t)q);
            if (m == 1) {
                const float2 g01 = box_muller(x.x, x.y), g23 = box_muller(x.z, x.w);
                const float gs[4] = {g01.x, g01.y, g23.x, g23.y};
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int s = 4 * q + e;
                    if (s >= S) break;
                    const int v = tx_position(s, p.p0, p.k, p.nf);
                    p.y[cw * S + s] = __fmaf_rn(sd, gs[e], 1.0f - 2.0f * (float)((L[v >> 5] >> (v & 31)) & 1u));
                }
            } else {
                const int h = m >> 1;
                const float2 gn[2] = {box_muller(x.x, x.y), box_muller(x.z, x.w)};
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    const int s = 2 * q + e;
                    if (s >= S) break;
                    const uint32_t bits = tx_symbol_bits(L, s, m, p.p0, p.k, p.nf);
                    float xi, xq;
                    if (p.points) {
                        const float2 pt = p.points[__brev(bits) >> (32 - m)];  // label MSB first
                        xi = pt.x;
                        xq = pt.y;
                    } else {
                        xi = __fmul_rn((float)pam_level(bits, h, 0), p.scale);
                        xq = __fmul_rn((float)pam_level(bits, h, 1), p.scale);
                    }
                    reinterpret_cast<float2 *>(p.y)[cw * S + s] =
                        make_float2(__fmaf_rn(sd, gn[e].x, xi), __fmaf_rn(sd, gn[e].y, xq));
                }
            }
        }
    }
}

// Mapper and AWGN on caller bits: symbol s of row b takes bits s m .. s m + m - 1
// of the row and the Gaussians k_tx draws for symbol s of codeword cw0 + b
// (Philox stream 1; one block gives four real or two complex symbols), with the
// same arithmetic, so the symbols equal k_tx's for the same bits.
__global__ void __launch_bounds__(256) k_map_awgn(const uint32_t *__restrict__ bits, int64_t B, int E, int nw, int m,
                                                  float scale, uint64_t seed, uint64_t cw0,
                                                  const float *__restrict__ no, int64_t no_stride,
                                                  float *__restrict__ y) {
    const int S = E / m;
    const int per = m == 1 ? 4 : 2;
    const int nqs = (S + per - 1) / per;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < B * nqs; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = i / nqs;
        const int q = (int)(i - b * nqs);
        const float sd = sqrtf(no[b * no_stride] * 0.5f);
        const uint4 x = draw(seed, cw0 + (uint64_t)b, 1u, (uint32_t)q);
        const uint32_t *row = bits + b * nw;
        if (m == 1) {
            const float2 g01 = box_muller(x.x, x.y), g23 = box_muller(x.z, x.w);
            const float gs[4] = {g01.x, g01.y, g23.x, g23.y};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int s = 4 * q + e;
                if (s >= S) break;
                const uint8_t bit = (uint8_t)((row[s >> 5] >> (s & 31)) & 1u);
                y[b * S + s] = __fmaf_rn(sd, gs[e], 1.0f - 2.0f * (float)bit);
            }
        } else {
            const int h = m >> 1;
            const float2 gn[2] = {box_muller(x.x, x.y), box_muller(x.z, x.w)};
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const int s = 2 * q + e;
                if (s >= S) break;
                uint32_t lb = 0u;
                for (int j = 0; j < m; ++j) {
                    const int t = s * m + j;
                    lb |= ((row[t >> 5] >> (t & 31)) & 1u) << j;
                }
                const float xi = __fmul_rn((float)pam_level(lb, h, 0), scale);
                const float xq = __fmul_rn((float)pam_level(lb, h, 1), scale);
                reinterpret_cast<float2 *>(y)[b * S + s] = make_float2(__fmaf_rn(sd, gn[e].x, xi), __fmaf_rn(sd, gn[e].y, xq));
            }
        }
    }
}

// ---------------------------------------------------------------- demapper
template <int M>
__global__ void __launch_bounds__(256) k_demap(const float *__restrict__ y, const float *__restrict__ no,
                                               int64_t no_stride, int64_t B, int64_t S, int method, float clamp,
                                               float scale, float *__restrict__ llr) {
    const int64_t total = B * S;
    bool bad = false;
    const float inv_shared = no_stride ? 0.0f : 1.0f / no[0];  // one N0 for all: no per-symbol division
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const float inv_n0 = no_stride ? 1.0f / no[i / S] : inv_shared;
        float L[M];
        if constexpr (M == 1) {
            demap_symbol<1>(y[i], 0.0f, inv_n0, scale, method, clamp, L, bad);
        } else {
            const float2 v = reinterpret_cast<const float2 *>(y)[i];
            demap_symbol<M>(v.x, v.y, inv_n0, scale, method, clamp, L, bad);
        }
        float *o = llr + i * M;
        if constexpr (M == 1) {
            o[0] = L[0];
        } else if constexpr (M == 2) {
            reinterpret_cast<float2 *>(o)[0] = make_float2(L[0], L[1]);
        } else if constexpr (M == 4) {
            reinterpret_cast<float4 *>(o)[0] = make_float4(L[0], L[1], L[2], L[3]);
        } else {
#pragma unroll
            for (int j = 0; j < M; ++j) o[j] = L[j];
        }
    }
    if (bad) latch(&g_status, LDPCX_FLAG_NONFINITE);
}

// ------------------------------------------------------ demapper with prior
template <int M>
__global__ void __launch_bounds__(256) k_demap_prior(const float *__restrict__ y, const float *__restrict__ no,
                                                     int64_t no_stride, int64_t B, int64_t S, int method, float clamp,
                                                     float scale, const float *__restrict__ prior, int out_mode,
                                                     float *__restrict__ llr) {
    const int64_t total = B * S;
    bool bad = false;
    const float inv_shared = no_stride ? 0.0f : 1.0f / no[0];  // one N0 for all: no per-symbol division
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const float inv_n0 = no_stride ? 1.0f / no[i / S] : inv_shared;
        if constexpr (M == 1) {
            const float v = y[i], la = prior ? prior[i] : 0.0f;
            float L = 4.0f * v * inv_n0;
            if (!isfinite(v)) {
                bad = true;
                L = 0.0f;
            }
            if (out_mode == LDPCX_DEMAP_OUT_APP) L += la;
            llr[i] = fminf(fmaxf(L, -clamp), clamp);
        } else {
            constexpr int H = M / 2;
            const float2 v = reinterpret_cast<const float2 *>(y)[i];
            float lai[H], laq[H], oi[H], oq[H];
#pragma unroll
            for (int j = 0; j < H; ++j) {
                lai[j] = prior ? prior[i * M + 2 * j] : 0.0f;
                laq[j] = prior ? prior[i * M + 2 * j + 1] : 0.0f;
            }
            if (isfinite(v.x) && isfinite(v.y)) {
                demap_dim_prior<H>(v.x, inv_n0, scale, method, clamp, lai, out_mode, oi);
                demap_dim_prior<H>(v.y, inv_n0, scale, method, clamp, laq, out_mode, oq);
            } else {
                bad = true;
#pragma unroll
                for (int j = 0; j < H; ++j) oi[j] = oq[j] = 0.0f;
            }
            float *o = llr + i * M;
#pragma unroll
            for (int j = 0; j < H; ++j) {
                o[2 * j] = oi[j];
                o[2 * j + 1] = oq[j];
            }
        }
    }
    if (bad) latch(&g_status, LDPCX_FLAG_NONFINITE);
}

// ------------------------------------------- EXIT: a-priori LLRs, information
__device__ __forceinline__ unsigned bit_at(const uint32_t *row, int64_t v) {
    return (row[v >> 5] >> (v & 31)) & 1u;
}

__global__ void __launch_bounds__(256) k_apriori(const uint32_t *__restrict__ bits, int64_t bits_stride,
                                                 int64_t bit_off, int64_t B, int64_t N, float sigma, uint64_t seed,
                                                 uint64_t cw0, float *__restrict__ out) {
    const int64_t nq = (N + 3) >> 2;  // Philox blocks per row: four Gaussians each
    const float mu = 0.5f * sigma * sigma;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < B * nq; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = i / nq, q = i - b * nq;
        const uint4 x = draw(seed, cw0 + (uint64_t)b, 2u, (uint32_t)q);
        const float2 g01 = box_muller(x.x, x.y), g23 = box_muller(x.z, x.w);
        const float g[4] = {g01.x, g01.y, g23.x, g23.y};
        const uint32_t *row = bits + b * bits_stride;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int64_t t = 4 * q + e;
            if (t < N) out[b * N + t] = fmaf(sigma, g[e], bit_at(row, bit_off + t) ? -mu : mu);
        }
    }
}

__global__ void __launch_bounds__(256) k_mutual_info(const float *__restrict__ llr, int64_t B, int64_t N,
                                                     const uint32_t *__restrict__ bits, int64_t bits_stride,
                                                     int64_t bit_off, double *acc) {
    double sum = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < B * N; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = i / N, t = i - b * N;
        const float L = llr[i];
        const float x = bit_at(bits + b * bits_stride, bit_off + t) ? -L : L;  // (1 - 2c) L
        // log2(1 + e^-x) = (max(-x, 0) + ln(1 + e^-|x|)) / ln 2, without overflow
        sum += (double)(fmaxf(-x, 0.0f) + log1pf(expf(-fabsf(x)))) * 1.4426950408889634;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xFFFFFFFFu, sum, o);
    __shared__ double s_part[8];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) s_part[warp] = sum;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += s_part[w];
        atomicAdd(&acc[0], t);
        if (blockIdx.x == 0) atomicAdd(&acc[1], (double)B * (double)N);
    }
}

__global__ void __launch_bounds__(256) k_extrinsic(const float *__restrict__ app, const float *__restrict__ in,
                                                   int64_t B, int n, int p0, int n_tx, int k, int nf, float clamp,
                                                   float *__restrict__ out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < B * n_tx; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = i / n_tx, t = i - b * n_tx;
        const float x = fminf(fmaxf(in[i], -clamp), clamp);  // the input as the decoder clamped it
        out[i] = fminf(fmaxf(app[b * n + tx_position((int)t, p0, k, nf)] - x, -clamp), clamp);
    }
}

// ------------------------------------------ arbitrary constellation (next 3)
// Online log-sum-exp: (mx, s) represents mx + ln s; adding term d.
__device__ __forceinline__ void lse_add(float &mx, float &s, float d) {
    if (d > mx) {
        s = s * expf(mx - d) + 1.0f;
        mx = d;
    } else {
        s += expf(d - mx);
    }
}

// Points into shared memory (2^m float2).
__device__ __forceinline__ void load_points(const float *points, int P, float2 *s_pts) {
    for (int l = threadIdx.x; l < P; l += blockDim.x) s_pts[l] = reinterpret_cast<const float2 *>(points)[l];
    __syncthreads();
}

template <int M>
__global__ void __launch_bounds__(256) k_demap_points(const float *__restrict__ y, const float *__restrict__ no,
                                                      int64_t no_stride, int64_t B, int64_t S,
                                                      const float *__restrict__ points, int method, float clamp,
                                                      float *__restrict__ llr) {
    constexpr int P = 1 << M;
    __shared__ float2 s_pts[P];
    load_points(points, P, s_pts);
    bool bad = false;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < B * S; i += (int64_t)gridDim.x * blockDim.x) {
        const float inv_n0 = 1.0f / no[(i / S) * no_stride];
        const float2 v = reinterpret_cast<const float2 *>(y)[i];
        float out[M];
        if (isfinite(v.x) && isfinite(v.y)) {
            float mx0[M], s0[M], mx1[M], s1[M];
#pragma unroll
            for (int j = 0; j < M; ++j) {
                mx0[j] = mx1[j] = -INFINITY;
                s0[j] = s1[j] = 0.0f;
            }
            for (int l = 0; l < P; ++l) {
                const float dr = v.x - s_pts[l].x, di = v.y - s_pts[l].y;
                const float d = -(dr * dr + di * di) * inv_n0;
#pragma unroll
                for (int j = 0; j < M; ++j) {
                    const bool one = (l >> (M - 1 - j)) & 1;
                    if (method == LDPCX_DEMAP_MAXLOG) {
                        if (one) mx1[j] = fmaxf(mx1[j], d);
                        else mx0[j] = fmaxf(mx0[j], d);
                    } else if (one) {
                        lse_add(mx1[j], s1[j], d);
                    } else {
                        lse_add(mx0[j], s0[j], d);
                    }
                }
            }
#pragma unroll
            for (int j = 0; j < M; ++j) {
                float L = mx0[j] - mx1[j];
                if (method != LDPCX_DEMAP_MAXLOG) L += logf(s0[j]) - logf(s1[j]);
                out[j] = fminf(fmaxf(L, -clamp), clamp);
            }
        } else {
            bad = true;
#pragma unroll
            for (int j = 0; j < M; ++j) out[j] = 0.0f;
        }
#pragma unroll
        for (int j = 0; j < M; ++j) llr[i * M + j] = out[j];
    }
    if (bad) latch(&g_status, LDPCX_FLAG_NONFINITE);
}

// Adjoint of the exact demapper: with w^0_j(l) = exp(d_l - LSE_0j), w^1_j(l) =
// exp(d_l - LSE_1j), dL_j/dd_l = w^0_j(l) or -w^1_j(l) by bit j of l, so
// g_l = sum_j gL_j (+-w_j(l)); dd_l/dy = -2 (y - p_l)/N0 = -dd_l/dp_l. Outputs
// held at the clamp pass no gradient. Point gradients are summed per block in
// shared memory, then added to grad_points once per block.
template <int M>
__global__ void __launch_bounds__(256) k_demap_points_bwd(const float *__restrict__ y, const float *__restrict__ no,
                                                          int64_t no_stride, int64_t B, int64_t S,
                                                          const float *__restrict__ points, float clamp,
                                                          const float *__restrict__ gllr, float *__restrict__ gy,
                                                          float *__restrict__ gpts) {
    constexpr int P = 1 << M;
    __shared__ float2 s_pts[P];
    __shared__ float s_g[2 * P];
    for (int l = threadIdx.x; l < 2 * P; l += blockDim.x) s_g[l] = 0.0f;
    load_points(points, P, s_pts);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < B * S; i += (int64_t)gridDim.x * blockDim.x) {
        const float inv_n0 = 1.0f / no[(i / S) * no_stride];
        const float2 v = reinterpret_cast<const float2 *>(y)[i];
        float2 g_y = make_float2(0.0f, 0.0f);
        if (isfinite(v.x) && isfinite(v.y)) {
            float mx0[M], s0[M], mx1[M], s1[M], gl[M];
#pragma unroll
            for (int j = 0; j < M; ++j) {
                mx0[j] = mx1[j] = -INFINITY;
                s0[j] = s1[j] = 0.0f;
            }
            for (int l = 0; l < P; ++l) {
                const float dr = v.x - s_pts[l].x, di = v.y - s_pts[l].y;
                const float d = -(dr * dr + di * di) * inv_n0;
#pragma unroll
                for (int j = 0; j < M; ++j) {
                    if ((l >> (M - 1 - j)) & 1) lse_add(mx1[j], s1[j], d);
                    else lse_add(mx0[j], s0[j], d);
                }
            }
#pragma unroll
            for (int j = 0; j < M; ++j) {
                const float l0 = mx0[j] + logf(s0[j]), l1 = mx1[j] + logf(s1[j]);
                mx0[j] = l0;  // now the log-sum-exp values
                mx1[j] = l1;
                const float L = l0 - l1;
                gl[j] = (L > -clamp && L < clamp) ? gllr[i * M + j] : 0.0f;
            }
            for (int l = 0; l < P; ++l) {
                const float dr = v.x - s_pts[l].x, di = v.y - s_pts[l].y;
                const float d = -(dr * dr + di * di) * inv_n0;
                float g = 0.0f;
#pragma unroll
                for (int j = 0; j < M; ++j) {
                    if ((l >> (M - 1 - j)) & 1) g -= gl[j] * expf(d - mx1[j]);
                    else g += gl[j] * expf(d - mx0[j]);
                }
                const float c = 2.0f * g * inv_n0;
                g_y.x -= c * dr;
                g_y.y -= c * di;
                atomicAdd(&s_g[2 * l], c * dr);
                atomicAdd(&s_g[2 * l + 1], c * di);
            }
        }
        reinterpret_cast<float2 *>(gy)[i] = g_y;
    }
    __syncthreads();
    for (int l = threadIdx.x; l < 2 * P; l += blockDim.x)
        if (s_g[l] != 0.0f) atomicAdd(&gpts[l], s_g[l]);
}

// Adjoint of the mapper: grad_points[label(b, s)] += grad_x[b][s].
__global__ void __launch_bounds__(256) k_map_points_bwd(const uint32_t *__restrict__ cw, int64_t nw, int p0, int k,
                                                        int nf, int m, int64_t B, int64_t S,
                                                        const float *__restrict__ gx, float *__restrict__ gpts) {
    __shared__ float s_g[512];
    const int P = 1 << m;
    for (int l = threadIdx.x; l < 2 * P; l += blockDim.x) s_g[l] = 0.0f;
    __syncthreads();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < B * S; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = i / S, s = i - b * S;
        const uint32_t *row = cw + b * nw;
        int l = 0;
        for (int j = 0; j < m; ++j) l = (l << 1) | (int)bit_at(row, tx_position((int)(s * m + j), p0, k, nf));
        const float2 g = reinterpret_cast<const float2 *>(gx)[i];
        atomicAdd(&s_g[2 * l], g.x);
        atomicAdd(&s_g[2 * l + 1], g.y);
    }
    __syncthreads();
    for (int l = threadIdx.x; l < 2 * P; l += blockDim.x)
        if (s_g[l] != 0.0f) atomicAdd(&gpts[l], s_g[l]);
}

// Binary cross-entropy of LLRs (logits -L) and its gradient.
__global__ void __launch_bounds__(256) k_bce(const float *__restrict__ llr, int64_t B, int64_t N,
                                             const uint32_t *__restrict__ bits, int64_t bits_stride, int64_t bit_off,
                                             float scale, double *acc, float *__restrict__ grad) {
    double sum = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < B * N; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = i / N, t = i - b * N;
        const float sgn = bit_at(bits + b * bits_stride, bit_off + t) ? -1.0f : 1.0f;  // 1 - 2c
        const float x = sgn * llr[i];
        sum += (double)(fmaxf(-x, 0.0f) + log1pf(expf(-fabsf(x))));  // ln(1 + e^-x)
        if (grad) grad[i] = -scale * sgn / (1.0f + expf(x));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xFFFFFFFFu, sum, o);
    __shared__ double s_part[8];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) s_part[warp] = sum;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += s_part[w];
        atomicAdd(&acc[0], t);
    }
}

// ------------------------------------------------------------ error count
__global__ void __launch_bounds__(256) k_count(const uint32_t *__restrict__ ref, const uint32_t *__restrict__ hat,
                                               const int32_t *__restrict__ iters, int64_t B, int k,
                                               unsigned long long *counts) {
    const int kw = (k + 31) >> 5;
    const int lane = threadIdx.x & 31;
    __shared__ unsigned long long s_acc[3];
    if (threadIdx.x < 3) s_acc[threadIdx.x] = 0ull;
    __syncthreads();
    unsigned long long be = 0, blk = 0, it = 0;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t cw = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); cw < B; cw += warps) {
        unsigned e = 0;
        for (int w = lane; w < kw; w += 32) e += __popc(ref[cw * kw + w] ^ hat[cw * kw + w]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) e += __shfl_xor_sync(0xFFFFFFFFu, e, o);
        if (lane == 0) {
            be += e;
            blk += e ? 1u : 0u;
            it += iters ? (unsigned long long)iters[cw] : 0ull;
        }
    }
    if (lane == 0) {
        atomicAdd(&s_acc[0], be);
        atomicAdd(&s_acc[1], blk);
        atomicAdd(&s_acc[2], it);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        atomicAdd(&counts[1], s_acc[0]);
        atomicAdd(&counts[3], s_acc[1]);
        atomicAdd(&counts[4], s_acc[2]);
        if (blockIdx.x == 0) {
            atomicAdd(&counts[0], (unsigned long long)B * (unsigned long long)k);
            atomicAdd(&counts[2], (unsigned long long)B);
        }
    }
}


}  // namespace

unsigned int take_status_channel(cudaStream_t s) {
    unsigned int v = 0, zero = 0;
    if (cudaMemcpyFromSymbolAsync(&v, g_status, sizeof(v), 0, cudaMemcpyDeviceToHost, s) != cudaSuccess) return 0;
    cudaMemcpyToSymbolAsync(g_status, &zero, sizeof(zero), 0, cudaMemcpyHostToDevice, s);
    cudaStreamSynchronize(s);
    return v;
}

}  // namespace ldpcx

using namespace ldpcx;

namespace ldpcx {

int launch_tx(ldpcx_code_t c, uint64_t seed, uint64_t cw0, const uint64_t *cw0_dev, int64_t B, int m,
              const float *no, int64_t no_stride, float *y_out, uint32_t *info_out, cudaStream_t stream,
              uint32_t *cw_out, const float *points) {
    if (c->enc == kEncNone) return LDPCX_E_UNSUPPORTED;  // before any device work
    DevCode d;
    int st = code_device(c, &d);
    if (st) return st;
    TxParams p{};
    p.blk = d.blk;
    p.row_ptr = d.row_ptr;
    p.Z = c->Z;
    p.rows = c->rows;
    p.kb = c->kb;
    p.n = c->n;
    p.k = c->k;
    p.n_tx = c->n_tx;
    p.p0 = c->p0;
    p.nf = c->n_fill;
    p.m = m;
    p.scale = qam_scale(m);
    p.seed = seed;
    p.cw0 = cw0;
    p.cw0_dev = cw0_dev;
    p.no = no;
    p.no_stride = no_stride;
    p.y = y_out;
    p.info = info_out;
    p.cw_out = cw_out;
    p.points = reinterpret_cast<const float2 *>(points);
    p.B = B;
    p.nnz = c->nnz;
    p.core_inv = c->enc == kEncCoreInv ? d.core_inv : nullptr;
    p.inv_words = c->enc == kEncCoreInv ? c->inv_words : 0;
    // codewords per CTA: about 2048 transmitted positions of mapping work, within 48 KB of shared memory
    int G = (int)std::max<int64_t>(1, std::min<int64_t>(std::min<int64_t>(16, 2048 / std::max(1, c->n_tx)), B));
    while (G > 1 && tx_layout(G, c->n, c->Z, c->nnz, c->rows, p.inv_words).bytes > 48 * 1024) --G;
    p.G = G;
    const size_t smem = tx_layout(G, c->n, c->Z, c->nnz, c->rows, p.inv_words).bytes;
    if (smem > 227 * 1024) return LDPCX_E_UNSUPPORTED;
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(k_tx, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return LDPCX_E_CUDA;
    const int64_t grid = (B + G - 1) / G;
    if (grid > 0x7FFFFFFF) return LDPCX_E_INVAL;
    k_tx<<<(unsigned)grid, kTxThreads, smem, stream>>>(p);
    return cuda_status(cudaGetLastError());
}


}  // namespace ldpcx

extern "C" int sim_tx(ldpcx_code_t c, uint64_t seed, uint64_t cw0, int64_t B, int m, const float *no,
                      int64_t no_stride, float *y_out, uint32_t *info_out, void *stream) {
    if (!c || B < 0 || !valid_m(m) || (no_stride != 0 && no_stride != 1)) return LDPCX_E_INVAL;
    if (c->n_tx % m != 0) return LDPCX_E_INVAL;
    if (B == 0) return LDPCX_OK;
    if (!no || !y_out) return LDPCX_E_INVAL;
    return launch_tx(c, seed, cw0, nullptr, B, m, no, no_stride, y_out, info_out, (cudaStream_t)stream);
}

extern "C" int qam_map_awgn(const uint32_t *bits, int64_t B, int E, int m, uint64_t seed, uint64_t cw0,
                            const float *no, int64_t no_stride, float *y_out, void *stream) {
    if (B < 0 || E < 1 || !valid_m(m) || E % m != 0 || (no_stride != 0 && no_stride != 1)) return LDPCX_E_INVAL;
    if (B == 0) return LDPCX_OK;
    if (!bits || !no || !y_out) return LDPCX_E_INVAL;
    const int per = m == 1 ? 4 : 2;
    const int64_t work = B * (int64_t)((E / m + per - 1) / per);
    int64_t blocks = (work + 255) / 256;
    const int64_t cap = (int64_t)sm_count() * 8;
    if (blocks > cap) blocks = cap;
    k_map_awgn<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(bits, B, E, (E + 31) / 32, m, qam_scale(m), seed,
                                                                   cw0, no, no_stride, y_out);
    return cuda_status(cudaGetLastError());
}

extern "C" int demap_app(const float *y, const float *no, int64_t no_stride, int64_t B, int64_t syms, int m,
                         int method, float clamp, float *llr_out, void *stream) {
    if (B < 0 || syms < 0 || !valid_m(m) || (no_stride != 0 && no_stride != 1)) return LDPCX_E_INVAL;
    if (method != LDPCX_DEMAP_EXACT && method != LDPCX_DEMAP_MAXLOG) return LDPCX_E_INVAL;
    if (!(clamp > 0.0f)) return LDPCX_E_INVAL;
    if (B == 0 || syms == 0) return LDPCX_OK;
    if (!y || !no || !llr_out) return LDPCX_E_INVAL;
    const int64_t total = B * syms;
    int64_t blocks = (total + 255) / 256;
    const int64_t cap = (int64_t)sm_count() * 8;
    if (blocks > cap) blocks = cap;
    cudaStream_t s = (cudaStream_t)stream;
    const float sc = qam_scale(m);
    switch (m) {
        case 1: k_demap<1><<<(unsigned)blocks, 256, 0, s>>>(y, no, no_stride, B, syms, method, clamp, sc, llr_out); break;
        case 2: k_demap<2><<<(unsigned)blocks, 256, 0, s>>>(y, no, no_stride, B, syms, method, clamp, sc, llr_out); break;
        case 4: k_demap<4><<<(unsigned)blocks, 256, 0, s>>>(y, no, no_stride, B, syms, method, clamp, sc, llr_out); break;
        case 6: k_demap<6><<<(unsigned)blocks, 256, 0, s>>>(y, no, no_stride, B, syms, method, clamp, sc, llr_out); break;
        default: k_demap<8><<<(unsigned)blocks, 256, 0, s>>>(y, no, no_stride, B, syms, method, clamp, sc, llr_out); break;
    }
    return cuda_status(cudaGetLastError());
}

extern "C" int sim_count(const uint32_t *ref, const uint32_t *hat, const int32_t *iters, int64_t B, int k,
                         int64_t *counts, void *stream) {
    if (B < 0 || k < 1 || !counts) return LDPCX_E_INVAL;
    if (B == 0) return LDPCX_OK;
    if (!ref || !hat) return LDPCX_E_INVAL;
    int64_t blocks = (B + 7) / 8;
    const int64_t cap = (int64_t)sm_count() * 4;
    if (blocks > cap) blocks = cap;
    k_count<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(ref, hat, iters, B, k,
                                                                 reinterpret_cast<unsigned long long *>(counts));
    return cuda_status(cudaGetLastError());
}

extern "C" int sim_codewords(ldpcx_code_t c, uint64_t seed, uint64_t cw0, int64_t B, uint32_t *cw_out,
                             void *stream) {
    if (!c || B < 0) return LDPCX_E_INVAL;
    if (B == 0) return LDPCX_OK;
    if (!cw_out) return LDPCX_E_INVAL;
    return launch_tx(c, seed, cw0, nullptr, B, 2, nullptr, 0, nullptr, nullptr, (cudaStream_t)stream, cw_out);
}

extern "C" int demap_app_prior(const float *y, const float *no, int64_t no_stride, int64_t B, int64_t syms, int m,
                               int method, float clamp, const float *prior, int out_mode, float *llr_out,
                               void *stream) {
    if (B < 0 || syms < 0 || !valid_m(m) || (no_stride != 0 && no_stride != 1)) return LDPCX_E_INVAL;
    if (method != LDPCX_DEMAP_EXACT && method != LDPCX_DEMAP_MAXLOG) return LDPCX_E_INVAL;
    if (out_mode != LDPCX_DEMAP_OUT_APP && out_mode != LDPCX_DEMAP_OUT_EXTRINSIC) return LDPCX_E_INVAL;
    if (!(clamp > 0.0f)) return LDPCX_E_INVAL;
    if (B == 0 || syms == 0) return LDPCX_OK;
    if (!y || !no || !llr_out) return LDPCX_E_INVAL;
    int64_t blocks = (B * syms + 255) / 256;
    const int64_t cap = (int64_t)sm_count() * 8;
    if (blocks > cap) blocks = cap;
    cudaStream_t s = (cudaStream_t)stream;
    const float sc = qam_scale(m);
#define LDPCX_DP(MM) \
    k_demap_prior<MM><<<(unsigned)blocks, 256, 0, s>>>(y, no, no_stride, B, syms, method, clamp, sc, prior, out_mode, llr_out)
    switch (m) {
        case 1: LDPCX_DP(1); break;
        case 2: LDPCX_DP(2); break;
        case 4: LDPCX_DP(4); break;
        case 6: LDPCX_DP(6); break;
        default: LDPCX_DP(8); break;
    }
#undef LDPCX_DP
    return cuda_status(cudaGetLastError());
}

extern "C" int llr_apriori(const uint32_t *bits, int64_t bits_stride, int64_t bit_off, int64_t B, int64_t N,
                           float sigma, uint64_t seed, uint64_t cw0, float *out, void *stream) {
    if (B < 0 || N < 0 || bit_off < 0 || !(sigma >= 0.0f) || isinf(sigma)) return LDPCX_E_INVAL;
    if (B == 0 || N == 0) return LDPCX_OK;
    if (!bits || !out || bits_stride * 32 < bit_off + N) return LDPCX_E_INVAL;
    int64_t blocks = (B * ((N + 3) >> 2) + 255) / 256;
    const int64_t cap = (int64_t)sm_count() * 8;
    if (blocks > cap) blocks = cap;
    k_apriori<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(bits, bits_stride, bit_off, B, N, sigma, seed, cw0,
                                                                  out);
    return cuda_status(cudaGetLastError());
}

extern "C" int llr_mutual_info(const float *llr, int64_t B, int64_t N, const uint32_t *bits, int64_t bits_stride,
                               int64_t bit_off, double *acc, void *stream) {
    if (B < 0 || N < 0 || bit_off < 0 || !acc) return LDPCX_E_INVAL;
    if (B == 0 || N == 0) return LDPCX_OK;
    if (!llr || !bits || bits_stride * 32 < bit_off + N) return LDPCX_E_INVAL;
    int64_t blocks = (B * N + 255) / 256;
    const int64_t cap = (int64_t)sm_count() * 4;
    if (blocks > cap) blocks = cap;
    k_mutual_info<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(llr, B, N, bits, bits_stride, bit_off, acc);
    return cuda_status(cudaGetLastError());
}

extern "C" int ldpc_extrinsic(ldpcx_code_t c, const float *app, const float *llr_in, int64_t B, float clamp,
                              float *out, void *stream) {
    if (!c || B < 0 || !(clamp > 0.0f)) return LDPCX_E_INVAL;
    if (B == 0) return LDPCX_OK;
    if (!app || !llr_in || !out) return LDPCX_E_INVAL;
    int64_t blocks = (B * c->n_tx + 255) / 256;
    const int64_t cap = (int64_t)sm_count() * 8;
    if (blocks > cap) blocks = cap;
    k_extrinsic<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(app, llr_in, B, c->n, c->p0, c->n_tx, c->k,
                                                                     c->n_fill, clamp, out);
    return cuda_status(cudaGetLastError());
}

extern "C" int sim_tx_points(ldpcx_code_t c, uint64_t seed, uint64_t cw0, int64_t B, int m, const float *points,
                             const float *no, int64_t no_stride, float *y_out, uint32_t *cw_out, void *stream) {
    if (!c || B < 0 || (m != 2 && m != 4 && m != 6 && m != 8) || (no_stride != 0 && no_stride != 1))
        return LDPCX_E_INVAL;
    if (c->n_tx % m != 0) return LDPCX_E_INVAL;
    if (B == 0) return LDPCX_OK;
    if (!points || !no || !y_out) return LDPCX_E_INVAL;
    return launch_tx(c, seed, cw0, nullptr, B, m, no, no_stride, y_out, nullptr, (cudaStream_t)stream, cw_out,
                     points);
}

namespace {
int grid_for(int64_t work, int per_sm) {
    int64_t blocks = (work + 255) / 256;
    const int64_t cap = (int64_t)sm_count() * per_sm;
    if (blocks > cap) blocks = cap;
    return (int)(blocks < 1 ? 1 : blocks);
}
bool valid_points_m(int m) { return m == 2 || m == 4 || m == 6 || m == 8; }
}  // namespace

extern "C" int demap_points(const float *y, const float *no, int64_t no_stride, int64_t B, int64_t S, int m,
                            const float *points, int method, float clamp, float *llr_out, void *stream) {
    if (B < 0 || S < 0 || !valid_points_m(m) || (no_stride != 0 && no_stride != 1) || !(clamp > 0.0f))
        return LDPCX_E_INVAL;
    if (method != LDPCX_DEMAP_EXACT && method != LDPCX_DEMAP_MAXLOG) return LDPCX_E_INVAL;
    if (B == 0 || S == 0) return LDPCX_OK;
    if (!y || !no || !points || !llr_out) return LDPCX_E_INVAL;
    const int g = grid_for(B * S, 8);
    cudaStream_t st = (cudaStream_t)stream;
    switch (m) {
        case 2: k_demap_points<2><<<g, 256, 0, st>>>(y, no, no_stride, B, S, points, method, clamp, llr_out); break;
        case 4: k_demap_points<4><<<g, 256, 0, st>>>(y, no, no_stride, B, S, points, method, clamp, llr_out); break;
        case 6: k_demap_points<6><<<g, 256, 0, st>>>(y, no, no_stride, B, S, points, method, clamp, llr_out); break;
        default: k_demap_points<8><<<g, 256, 0, st>>>(y, no, no_stride, B, S, points, method, clamp, llr_out); break;
    }
    return cuda_status(cudaGetLastError());
}

extern "C" int demap_points_backward(const float *y, const float *no, int64_t no_stride, int64_t B, int64_t S,
                                     int m, const float *points, float clamp, const float *grad_llr, float *grad_y,
                                     float *grad_points, void *stream) {
    if (B < 0 || S < 0 || !valid_points_m(m) || (no_stride != 0 && no_stride != 1) || !(clamp > 0.0f))
        return LDPCX_E_INVAL;
    if (B == 0 || S == 0) return LDPCX_OK;
    if (!y || !no || !points || !grad_llr || !grad_y || !grad_points) return LDPCX_E_INVAL;
    const int g = grid_for(B * S, 4);
    cudaStream_t st = (cudaStream_t)stream;
#define LDPCX_DPB(MM) \
    k_demap_points_bwd<MM><<<g, 256, 0, st>>>(y, no, no_stride, B, S, points, clamp, grad_llr, grad_y, grad_points)
    switch (m) {
        case 2: LDPCX_DPB(2); break;
        case 4: LDPCX_DPB(4); break;
        case 6: LDPCX_DPB(6); break;
        default: LDPCX_DPB(8); break;
    }
#undef LDPCX_DPB
    return cuda_status(cudaGetLastError());
}

extern "C" int map_points_backward(ldpcx_code_t c, const uint32_t *cw, int64_t B, int m, const float *grad_x,
                                   float *grad_points, void *stream) {
    if (!c || B < 0 || !valid_points_m(m) || c->n_tx % m != 0) return LDPCX_E_INVAL;
    if (B == 0) return LDPCX_OK;
    if (!cw || !grad_x || !grad_points) return LDPCX_E_INVAL;
    const int64_t S = c->n_tx / m, nw = (c->n + 31) / 32;
    k_map_points_bwd<<<grid_for(B * S, 4), 256, 0, (cudaStream_t)stream>>>(cw, nw, c->p0, c->k, c->n_fill, m, B, S,
                                                                         grad_x, grad_points);
    return cuda_status(cudaGetLastError());
}

extern "C" int llr_bce(const float *llr, int64_t B, int64_t N, const uint32_t *bits, int64_t bits_stride,
                       int64_t bit_off, float scale, double *loss_acc, float *grad_llr, void *stream) {
    if (B < 0 || N < 0 || bit_off < 0 || !loss_acc) return LDPCX_E_INVAL;
    if (B == 0 || N == 0) return LDPCX_OK;
    if (!llr || !bits || bits_stride * 32 < bit_off + N) return LDPCX_E_INVAL;
    k_bce<<<grid_for(B * N, 4), 256, 0, (cudaStream_t)stream>>>(llr, B, N, bits, bits_stride, bit_off, scale,
                                                                 loss_acc, grad_llr);
    return cuda_status(cudaGetLastError());
}
