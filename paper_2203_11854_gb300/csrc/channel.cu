// Monte-Carlo transmitter (BinarySource -> LDPC5GEncoder -> Mapper -> AWGN of
// the paper's Listing 1), APP demapper (Demapper("app")) and error counting
// (compute_ber), all on the device.
#include <math.h>

#include "common.cuh"

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

// Gray PAM level of h bits taken from c at stride 2 (I: offset 0, Q: offset 1):
// A = (1-2a0)(2^(h-1) - (1-2a1)(2^(h-2) - ... (1-2a_{h-1}))).
__device__ __forceinline__ int pam_level(const uint8_t *c, int h) {
    int inner = 1 - 2 * (int)c[2 * (h - 1)];
    for (int i = h - 2; i >= 0; --i) inner = (1 - 2 * (int)c[2 * i]) * ((1 << (h - 1 - i)) - inner);
    return inner;
}


// Shared-memory layout of k_tx, per CTA: [G][ns] codeword bytes (ns = n rounded
// up to 4), [G][4 nq] packed source words, then (8-byte aligned) the block
// table as {col Z + shift, Z - shift} pairs, the row pointers and the packed
// lambda words of the general core.
__host__ __device__ inline int tx_ns(int n) { return (n + 3) & ~3; }
__host__ __device__ inline size_t tx_enc_off(int G, int n, int k) {
    const int nq = (((k + 31) >> 5) + 3) >> 2;
    return ((size_t)G * tx_ns(n) + (size_t)G * 16 * nq + 7) & ~(size_t)7;
}
__host__ __device__ inline size_t tx_smem(int G, int n, int k, int nnz, int rows, int inv_words) {
    return tx_enc_off(G, n, k) + 8 * (size_t)nnz + 4 * (size_t)(rows + 1) + 4 * (size_t)G * inv_words;
}

__global__ void __launch_bounds__(kMaxThreads) k_tx(const TxParams p) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int ns = tx_ns(p.n);
    const int kw = (p.k + 31) >> 5;
    const int nq = (kw + 3) >> 2;  // Philox blocks of source bits per codeword
    uint8_t *s_c = smem;           // [G][ns] codeword bits, one byte each
    uint32_t *s_w = reinterpret_cast<uint32_t *>(smem + (size_t)p.G * ns);  // [G][4 nq] source words
    int2 *s_enc = reinterpret_cast<int2 *>(smem + tx_enc_off(p.G, p.n, p.k));  // [nnz] {col Z + s, Z - s}
    int32_t *s_rp = reinterpret_cast<int32_t *>(s_enc + p.nnz);
    uint32_t *s_lam = reinterpret_cast<uint32_t *>(s_rp + p.rows + 1);  // [G][inv_words] packed lambda
    const int64_t cw_base = (int64_t)blockIdx.x * p.G;
    const uint64_t cw0 = p.cw0 + (p.cw0_dev ? *p.cw0_dev : 0ull);

    for (int i = threadIdx.x; i < p.nnz; i += blockDim.x) {
        const uint32_t bb = p.blk[i];
        const int sh = (int)(bb & 0xFFFFu);
        s_enc[i] = make_int2((int)(bb >> 16) * p.Z + sh, p.Z - sh);
    }
    for (int i = threadIdx.x; i <= p.rows; i += blockDim.x) s_rp[i] = p.row_ptr[i];
    for (int i = threadIdx.x; i < p.G * p.inv_words; i += blockDim.x) s_lam[i] = 0u;
    // source bits (Philox stream 0), written packed to the output and to shared memory
    for (int i = threadIdx.x; i < p.G * nq; i += blockDim.x) {
        const int gg = i / nq, q = i - gg * nq;
        const int64_t cw = cw_base + gg;
        if (cw >= p.B) continue;
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
            s_w[(size_t)gg * 4 * nq + w] = word;
        }
    }
    __syncthreads();
    // one byte per bit, four bits per 32-bit store: nibble * 0x00204081 moves bit j to bit 8j (the four
    // shifted copies of the nibble do not overlap). Bytes past k belong to parity column kb and are
    // overwritten below.
    const int k4 = (p.k + 3) >> 2;
    for (int i = threadIdx.x; i < p.G * k4; i += blockDim.x) {
        const int gg = i / k4, j = i - gg * k4;
        if (cw_base + gg >= p.B) continue;
        const uint32_t nib = (s_w[(size_t)gg * 4 * nq + (j >> 3)] >> (4 * (j & 7))) & 0xFu;
        *reinterpret_cast<uint32_t *>(s_c + (size_t)gg * ns + 4 * j) = (nib * 0x00204081u) & 0x01010101u;
    }
    if (p.nf > 0) {
        // filler bits are 0; bytes k .. 4 k4 - 1 already are (the last source word is masked)
        const int f0 = 4 * k4, f1 = p.k + p.nf, nfz = f1 > f0 ? f1 - f0 : 0;
        for (int i = threadIdx.x; i < p.G * nfz; i += blockDim.x) {
            const int gg = i / nfz, v = f0 + (i - gg * nfz);
            if (cw_base + gg < p.B) s_c[(size_t)gg * ns + v] = 0;
        }
    }
    __syncthreads();

    // systematic encoding, one thread per (codeword, z)
    const int g = threadIdx.x / p.Z, z = threadIdx.x - g * p.Z;
    const bool active = g < p.G && cw_base + g < p.B;
    uint8_t *c = s_c + (size_t)(active ? g : 0) * ns;
    const int Z = p.Z;
    // bit of check z in block e: codeword position col Z + (z + s) mod Z; blocks of columns below
    // `lim` Z are those with e.x < lim Z (s < Z)
    auto at = [&](const int2 e) -> uint8_t {
        int v = e.x + z;
        if (z >= e.y) v -= Z;
        return c[v];
    };
    uint8_t lam[4] = {0, 0, 0, 0};
    if (active) {
        // lambda_r = sum over the systematic blocks of core row r
        const int kbZ = p.kb * Z;
        for (int r = 0; r < 4; ++r) {
            uint8_t acc = 0;
#pragma unroll 4
            for (int b = s_rp[r]; b < s_rp[r + 1]; ++b) {
                const int2 e = s_enc[b];
                if (e.x < kbZ) acc ^= at(e);
            }
            lam[r] = acc;
        }
        if (p.core_inv) {
            // lambda as a 4Z-bit vector, bit r Z + z = lambda_r[z]
            uint32_t *lw = s_lam + (size_t)g * p.inv_words;
#pragma unroll
            for (int r = 0; r < 4; ++r)
                if (lam[r]) atomicOr(&lw[(r * Z + z) >> 5], 1u << ((r * Z + z) & 31));
        } else {
            c[p.kb * Z + z] = lam[0] ^ lam[1] ^ lam[2] ^ lam[3];  // p_a: the core rows sum to [I 0 0 0]
        }
    }
    __syncthreads();
    if (active && p.core_inv) {
        // core parity p = H_core^-1 lambda: bit r Z + z is the parity of (row r Z + z of the inverse) & lambda
        const uint32_t *lw = s_lam + (size_t)g * p.inv_words;
#pragma unroll 1
        for (int r = 0; r < 4; ++r) {
            const uint32_t *row = p.core_inv + (size_t)(r * Z + z) * p.inv_words;
            uint32_t x = 0u;
            for (int w = 0; w < p.inv_words; ++w) x ^= __ldg(row + w) & lw[w];
            c[(p.kb + r) * Z + z] = (uint8_t)(__popc(x) & 1);
        }
    } else if (active) {
        const uint8_t pa = c[p.kb * Z + z];
        const uint8_t pb = lam[0] ^ c[p.kb * Z + (z + 1 == Z ? 0 : z + 1)];  // row 0: P^1 p_a + p_b
        const uint8_t pc = lam[1] ^ pa ^ pb;                                  // row 1: p_a + p_b + p_c
        const uint8_t pd = lam[2] ^ pc;                                       // row 2: p_c + p_d
        c[(p.kb + 1) * Z + z] = pb;
        c[(p.kb + 2) * Z + z] = pc;
        c[(p.kb + 3) * Z + z] = pd;
    }
    __syncthreads();
    if (active) {
        // extension rows only read columns < kb + 4, so they are independent
        for (int r = 4; r < p.rows; ++r) {
            uint8_t acc = 0;
            const int ownZ = (p.kb + r) * Z;  // the row's own parity column; every other block lies below it
            int2 eo = make_int2(ownZ, Z);
#pragma unroll 4
            for (int b = s_rp[r]; b < s_rp[r + 1]; ++b) {
                const int2 e = s_enc[b];
                if (e.x < ownZ) acc ^= at(e);
                else eo = e;
            }
            // check z holds own-column bit (z + s_own) mod Z
            int v = eo.x + z;
            if (z >= eo.y) v -= Z;
            c[v] = acc;
        }
    }
    __syncthreads();

    // the codewords themselves, packed 32 positions per word by warp ballots
    if (p.cw_out) {
        const int nw = (p.n + 31) >> 5;
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
        for (int w = warp; w < p.G * nw; w += nwarps) {
            const int gg = w / nw, ww = w - gg * nw;
            const int64_t cw = cw_base + gg;
            const int pos = ww * 32 + lane;
            const bool bit = cw < p.B && pos < p.n && s_c[(size_t)gg * ns + pos] != 0;
            const unsigned word = __ballot_sync(0xFFFFFFFFu, bit);
            if (lane == 0 && cw < p.B) p.cw_out[cw * nw + ww] = word;
        }
    }
    if (!p.y) return;  // codewords only: no barrier follows

    // Gray mapping and AWGN (Philox stream 1)
    const int m = p.m, S = p.n_tx / m;
    if (m == 1) {
        const int nqs = (S + 3) >> 2;
        for (int i = threadIdx.x; i < p.G * nqs; i += blockDim.x) {
            const int gg = i / nqs, q = i - gg * nqs;
            const int64_t cw = cw_base + gg;
            if (cw >= p.B) continue;
            const float sd = sqrtf(p.no[cw * p.no_stride] * 0.5f);
            const uint4 x = draw(p.seed, cw0 + (uint64_t)cw, 1u, (uint32_t)q);
            const float2 g01 = box_muller(x.x, x.y), g23 = box_muller(x.z, x.w);
            const float gs[4] = {g01.x, g01.y, g23.x, g23.y};
            const uint8_t *cg = s_c + (size_t)gg * ns;
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int s = 4 * q + e;
                if (s < S) p.y[cw * S + s] = (1.0f - 2.0f * (float)cg[tx_position(s, p.p0, p.k, p.nf)]) + sd * gs[e];
            }
        }
    } else {
        const int h = m >> 1, nqs = (S + 1) >> 1;
        for (int i = threadIdx.x; i < p.G * nqs; i += blockDim.x) {
            const int gg = i / nqs, q = i - gg * nqs;
            const int64_t cw = cw_base + gg;
            if (cw >= p.B) continue;
            const float sd = sqrtf(p.no[cw * p.no_stride] * 0.5f);
            const uint4 x = draw(p.seed, cw0 + (uint64_t)cw, 1u, (uint32_t)q);
            const float2 gn[2] = {box_muller(x.x, x.y), box_muller(x.z, x.w)};
            const uint8_t *cb = s_c + (size_t)gg * ns + p.p0;
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const int s = 2 * q + e;
                if (s >= S) break;
                const uint8_t *bits = cb + (size_t)s * m;
                uint8_t gathered[8];
                if (p.nf > 0) {  // a shortened code: the symbol's bits skip the fillers
                    const uint8_t *cg = s_c + (size_t)gg * ns;
                    for (int j = 0; j < m; ++j) gathered[j] = cg[tx_position(s * m + j, p.p0, p.k, p.nf)];
                    bits = gathered;
                }
                float xi, xq;
                if (p.points) {
                    int l = 0;
                    for (int j = 0; j < m; ++j) l = (l << 1) | bits[j];
                    const float2 pt = p.points[l];
                    xi = pt.x;
                    xq = pt.y;
                } else {
                    xi = (float)pam_level(bits, h) * p.scale;
                    xq = (float)pam_level(bits + 1, h) * p.scale;
                }
                reinterpret_cast<float2 *>(p.y)[cw * S + s] = make_float2(xi + sd * gn[e].x, xq + sd * gn[e].y);
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
                y[b * S + s] = (1.0f - 2.0f * (float)bit) + sd * gs[e];
            }
        } else {
            const int h = m >> 1;
            const float2 gn[2] = {box_muller(x.x, x.y), box_muller(x.z, x.w)};
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const int s = 2 * q + e;
                if (s >= S) break;
                uint8_t lb[8];
                for (int j = 0; j < m; ++j) {
                    const int t = s * m + j;
                    lb[j] = (uint8_t)((row[t >> 5] >> (t & 31)) & 1u);
                }
                const float xi = (float)pam_level(lb, h) * scale;
                const float xq = (float)pam_level(lb + 1, h) * scale;
                reinterpret_cast<float2 *>(y)[b * S + s] = make_float2(xi + sd * gn[e].x, xq + sd * gn[e].y);
            }
        }
    }
}

// ---------------------------------------------------------------- demapper
// Per I/Q dimension: metrics d_l = -(y - A_l s)^2 / N0 over the 2^h PAM levels;
// bit i of the dimension gets LSE/max over levels whose label has bit i = 0,
// minus the same over bit i = 1.
template <int H>
__device__ __forceinline__ void demap_dim(float y, float inv_n0, float scale, int method, float clamp, float *out) {
    constexpr int P = 1 << H;
    float d[P];
#pragma unroll
    for (int l = 0; l < P; ++l) {
        // label bits a_i = bit (H-1-i) of l; level by the Gray recursion
        int inner = 1 - 2 * ((l >> 0) & 1);
#pragma unroll
        for (int i = H - 2; i >= 0; --i) inner = (1 - 2 * ((l >> (H - 1 - i)) & 1)) * ((1 << (H - 1 - i)) - inner);
        const float e = y - (float)inner * scale;
        d[l] = -(e * e) * inv_n0;
    }
#pragma unroll
    for (int i = 0; i < H; ++i) {
        const int bit = H - 1 - i;
        float mx0 = -INFINITY, mx1 = -INFINITY;
#pragma unroll
        for (int l = 0; l < P; ++l) {
            if ((l >> bit) & 1) mx1 = fmaxf(mx1, d[l]);
            else mx0 = fmaxf(mx0, d[l]);
        }
        float L;
        if (method == LDPCX_DEMAP_MAXLOG) {
            L = mx0 - mx1;
        } else {
            float s0 = 0.0f, s1 = 0.0f;
#pragma unroll
            for (int l = 0; l < P; ++l) {
                if ((l >> bit) & 1) s1 += expf(d[l] - mx1);
                else s0 += expf(d[l] - mx0);
            }
            L = (mx0 - mx1) + (logf(s0) - logf(s1));
        }
        out[i] = fminf(fmaxf(L, -clamp), clamp);
    }
}

template <int M>
__global__ void __launch_bounds__(256) k_demap(const float *__restrict__ y, const float *__restrict__ no,
                                               int64_t no_stride, int64_t B, int64_t S, int method, float clamp,
                                               float scale, float *__restrict__ llr) {
    const int64_t total = B * S;
    bool bad = false;
    const float inv_shared = no_stride ? 0.0f : 1.0f / no[0];  // one N0 for all: no per-symbol division
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const float inv_n0 = no_stride ? 1.0f / no[i / S] : inv_shared;
        if constexpr (M == 1) {
            float v = y[i];
            float L = 4.0f * v * inv_n0;
            if (!isfinite(v)) {
                bad = true;
                L = 0.0f;
            }
            llr[i] = fminf(fmaxf(L, -clamp), clamp);
        } else {
            constexpr int H = M / 2;
            const float2 v = reinterpret_cast<const float2 *>(y)[i];
            float oi[H], oq[H];
            if (isfinite(v.x) && isfinite(v.y)) {
                demap_dim<H>(v.x, inv_n0, scale, method, clamp, oi);
                demap_dim<H>(v.y, inv_n0, scale, method, clamp, oq);
            } else {
                bad = true;
#pragma unroll
                for (int j = 0; j < H; ++j) oi[j] = oq[j] = 0.0f;
            }
            float *o = llr + i * M;
            if constexpr (M == 2) {
                reinterpret_cast<float2 *>(o)[0] = make_float2(oi[0], oq[0]);
            } else if constexpr (M == 4) {
                reinterpret_cast<float4 *>(o)[0] = make_float4(oi[0], oq[0], oi[1], oq[1]);
            } else {
#pragma unroll
                for (int j = 0; j < H; ++j) {
                    o[2 * j] = oi[j];
                    o[2 * j + 1] = oq[j];
                }
            }
        }
    }
    if (bad) latch(&g_status, LDPCX_FLAG_NONFINITE);
}

// ------------------------------------------------------ demapper with prior
// demap_dim with a-priori LLRs la[0..H) of the dimension's bits: the metric of
// level l gains sum_i (1 - 2 a_i(l)) la_i / 2. Extrinsic output leaves bit i's
// own term out, which shifts the two sets of bit i by -la_i/2 and +la_i/2, so
// it is the a-posteriori value minus la_i.
template <int H>
__device__ __forceinline__ void demap_dim_prior(float y, float inv_n0, float scale, int method, float clamp,
                                                const float *la, int out_mode, float *out) {
    constexpr int P = 1 << H;
    float d[P];
#pragma unroll
    for (int l = 0; l < P; ++l) {
        int inner = 1 - 2 * ((l >> 0) & 1);
#pragma unroll
        for (int i = H - 2; i >= 0; --i) inner = (1 - 2 * ((l >> (H - 1 - i)) & 1)) * ((1 << (H - 1 - i)) - inner);
        const float e = y - (float)inner * scale;
        float pr = 0.0f;
#pragma unroll
        for (int i = 0; i < H; ++i) pr += ((l >> (H - 1 - i)) & 1) ? -la[i] : la[i];
        d[l] = fmaf(0.5f, pr, -(e * e) * inv_n0);
    }
#pragma unroll
    for (int i = 0; i < H; ++i) {
        const int bit = H - 1 - i;
        float mx0 = -INFINITY, mx1 = -INFINITY;
#pragma unroll
        for (int l = 0; l < P; ++l) {
            if ((l >> bit) & 1) mx1 = fmaxf(mx1, d[l]);
            else mx0 = fmaxf(mx0, d[l]);
        }
        float L;
        if (method == LDPCX_DEMAP_MAXLOG) {
            L = mx0 - mx1;
        } else {
            float s0 = 0.0f, s1 = 0.0f;
#pragma unroll
            for (int l = 0; l < P; ++l) {
                if ((l >> bit) & 1) s1 += expf(d[l] - mx1);
                else s0 += expf(d[l] - mx0);
            }
            L = (mx0 - mx1) + (logf(s0) - logf(s1));
        }
        if (out_mode == LDPCX_DEMAP_OUT_EXTRINSIC) L -= la[i];
        out[i] = fminf(fmaxf(L, -clamp), clamp);
    }
}

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


bool valid_m(int m) { return m == 1 || m == 2 || m == 4 || m == 6 || m == 8; }

float qam_scale(int m) {
    if (m == 1) return 1.0f;
    const int h = m / 2;
    return (float)(1.0 / sqrt(2.0 * (double)((1 << (2 * h)) - 1) / 3.0));
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
    int G = kMaxThreads / c->Z;
    if (G < 1) G = 1;
    while (G > 1 && tx_smem(G, c->n, c->k, c->nnz, c->rows, p.inv_words) > 96 * 1024) --G;
    p.G = G;
    const size_t smem = tx_smem(G, c->n, c->k, c->nnz, c->rows, p.inv_words);
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(k_tx, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return LDPCX_E_CUDA;
    const int threads = (G * c->Z + 31) / 32 * 32;
    const int64_t grid = (B + G - 1) / G;
    k_tx<<<(unsigned)grid, threads, smem, stream>>>(p);
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
