// Flooding decoder kernels (weighted), all message formats.
//
// An iteration runs in two phases over the CTA's G codewords, each phase a
// strided loop of the CTA's threads over independent work items:
//  1. every check node of every row: V2C_j = w_j (APP_v - C_j) from the
//     previous iteration's APP, the check-node rule, the new messages rounded
//     to the format and stored (and checkpointed for the adjoint);
//  2. every variable node: APP_v = L_v + the new messages of its column in
//     ascending row order, read back from the message array (the values just
//     stored, so the rounded ones).
// Phase 2 adds in the order the definition of flooding BP sums in (channel
// LLR first, then ascending base row), so the results equal a row-by-row
// accumulation bit for bit, with two block barriers per iteration instead of
// one per row. The messages of the last iteration are stored too (phase 2
// reads them).
#include "decode_cols.cuh"
#include "decode_kernels.cuh"

namespace ldpcx {
namespace dec {

// Check node z of row r (blocks b0 .. b0 + deg) of one codeword: the flooding
// update from the previous APP `app`, messages of the codeword at ml (edge b
// at ml[b Z + z]), weights w (or null), checkpoint ck of C^t (or null).
// Min-sum: the two smallest |T| with ties to m2, v2 for the edges whose |T|
// equals the smallest, signs by comparison (a weighted input may be -0.0).
// Sum-product: SpaNode's magnitudes (phi in bits, exclusive sums without
// cancellation, the outer clamp on phi's result), signs by comparison.
template <int DMAX, int ALGO, int PREC>
__device__ __forceinline__ void flood_check(const Params &p, const float *app, const uint32_t *vb, int deg, int z,
                                            typename MsgT<PREC>::T *ml, const float *w, bool load, float *ck) {
    using MT = typename MsgT<PREC>::T;
    float T[DMAX];
    unsigned par = 0;
#pragma unroll
    for (int j = 0; j < DMAX; ++j) {
        T[j] = 0.0f;
        if (j < deg) {
            const float old = load ? msg_load<PREC>(ml + (size_t)j * p.Z) : 0.0f;
            float v2c = __fsub_rn(app[vn_at(vb[j], z, p.Z)], old);
            if (w) v2c = __fmul_rn(w[j], v2c);
            T[j] = v2c;
            par ^= T[j] < 0.0f ? 1u : 0u;
        }
    }
    // the new message of edge j: rounded to the format, stored (and checkpointed)
    auto put = [&](int j, float val) {
        MT mq;
        const float rq = msg_round<PREC>(val, &mq);
        msg_store<PREC>(ml + (size_t)j * p.Z, mq);
        if (ck) ck[(size_t)j * p.Z] = rq;  // checkpoint of C^t for the adjoint
    };
    if constexpr (ALGO == kMinSum) {
        float m1 = INFINITY, m2 = INFINITY;
#pragma unroll
        for (int j = 0; j < DMAX; ++j) {
            if (j < deg) {
                const float a = fabsf(T[j]);
                m2 = fminf(m2, fmaxf(m1, a));
                m1 = fminf(m1, a);
            }
        }
        const float v1 = fminf(fmaxf(__fsub_rn(m1, p.offset), 0.0f), p.clamp);
        const float v2 = fminf(fmaxf(__fsub_rn(m2, p.offset), 0.0f), p.clamp);
#pragma unroll
        for (int j = 0; j < DMAX; ++j) {
            if (j < deg) {
                const float mag = fabsf(T[j]) == m1 ? v2 : v1;
                put(j, (par ^ (T[j] < 0.0f ? 1u : 0u)) ? -mag : mag);
            }
        }
    } else {
        SpaNode<DMAX> cn;
        cn.prepare(T, deg, p.clamp, p.phi_lo);
#pragma unroll
        for (int j = 0; j < DMAX; ++j) {
            if (j < deg) {
                const float mag = cn.mag(j, p.clamp, p.phi_lo);
                put(j, (par ^ (T[j] < 0.0f ? 1u : 0u)) ? -mag : mag);
            }
        }
    }
}

// The check-node update with an exact-degree body for the short rows of the
// 5G-shaped base graphs (the extension rows: degree 4 or 5, 5 or 6), where
// no edge slot is predicated off, and the predicated DMAX body for the rest
// (the dense core rows lose a slot or two): the same operations in the same
// order either way.
template <int DMAX, int ALGO, int PREC>
__device__ __forceinline__ void flood_check_any(const Params &p, const float *app, const uint32_t *vb, int deg, int z,
                                                typename MsgT<PREC>::T *ml, const float *w, bool load, float *ck) {
    constexpr int D0 = DMAX <= 12 ? 4 : 5;
    if (deg == D0) flood_check<D0, ALGO, PREC>(p, app, vb, D0, z, ml, w, load, ck);
    else if (deg == D0 + 1) flood_check<D0 + 1, ALGO, PREC>(p, app, vb, D0 + 1, z, ml, w, load, ck);
    else flood_check<DMAX, ALGO, PREC>(p, app, vb, deg, z, ml, w, load, ck);
}

// Flooding BP, G codewords per CTA (flood_threads threads); each phase is one
// strided loop over the items of all G codewords, so that small codes fill the
// CTA.
template <int DMAX, int ALGO, int PREC>
__global__ void __launch_bounds__(512, 2) k_flooding(const __grid_constant__ Params p) {
    using MT = typename MsgT<PREC>::T;
    extern __shared__ __align__(16) unsigned char smem[];
    const int cols = p.n / p.Z;
    float *s_a = reinterpret_cast<float *>(smem);
    float *s_b = s_a + (size_t)p.G * p.n;
    uint32_t *s_vb = reinterpret_cast<uint32_t *>(s_b + (size_t)p.G * p.n);
    uint32_t *s_cb = s_vb + p.nnz;  // blocks by column: b << 16 | shift, ascending b (= ascending row)
    int32_t *s_rp = reinterpret_cast<int32_t *>(s_cb + p.nnz);
    int32_t *s_cp = s_rp + p.rows + 1;
    int *s_flag = s_cp + cols + 1;
    int *s_done = s_flag + p.G;
    int *s_iters = s_done + p.G;

    load_tables(p, s_vb, s_rp);
    build_col_lists(p.blk, p.nnz, cols, s_cp, s_cb);
    const int64_t cw_base = (int64_t)blockIdx.x * p.G;
    for (int i = threadIdx.x; i < p.G; i += blockDim.x) {
        s_done[i] = (cw_base + i >= p.B) ? 1 : 0;
        s_iters[i] = 0;
    }
    load_channel_llr(p, s_a, cw_base);  // the flooding decoders take LLRs only
    float *cur = s_a, *nxt = s_b;       // APP of the previous iteration / of this one

    for (int t = 0; t < p.iters; ++t) {
        __syncthreads();
        const float *w_t = p.weights ? p.weights + (size_t)t * p.nnz : nullptr;
        const bool ckpt = p.ckpt && t + 1 < p.iters;
        // phase 1: every check node of the codewords still decoding, items (codeword, row, z) with z fastest
        {
            GZWalk it(p.Z, p.rows);
            for (; it.g < p.G; it.next(p.Z, p.rows)) {
                const int gg = it.g, r = it.q;
                if (s_done[gg]) continue;
                const int64_t cw = cw_base + gg;
                const int b0 = s_rp[r], deg = s_rp[r + 1] - b0;
                const size_t e0 = (size_t)b0 * p.Z + it.z;
                MT *mp = reinterpret_cast<MT *>(p.msg) + cw * p.msg_stride;
                float *ck = ckpt ? p.ckpt + (size_t)t * p.ckpt_tstride + (size_t)cw * p.msg_stride + e0 : nullptr;
                flood_check_any<DMAX, ALGO, PREC>(p, cur + (size_t)gg * p.n, s_vb + b0, deg, it.z, mp + e0,
                                              w_t ? w_t + b0 : nullptr, t > 0, ck);
            }
        }
        __syncthreads();
        // phase 2: every variable node, items (codeword, column, z); a stopped codeword carries its APP forward
        {
            GZWalk it(p.Z, cols);
            for (; it.g < p.G; it.next(p.Z, cols)) {
                const int gg = it.g, c = it.q;
                const int64_t cw = cw_base + gg;
                if (cw >= p.B) continue;
                const int v = c * p.Z + it.z;
                float *a1 = nxt + (size_t)gg * p.n;
                if (s_done[gg]) {
                    a1[v] = cur[(size_t)gg * p.n + v];
                    continue;
                }
                const MT *mp = reinterpret_cast<const MT *>(p.msg) + cw * p.msg_stride;
                bool bad = false;
                float a = channel_llr(p, cw, v, bad);
                // four loads in flight, then their sums in order
                const int e1 = s_cp[c + 1];
                for (int e = s_cp[c]; e < e1; e += 4) {
                    float m[4];
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        m[i] = 0.0f;
                        if (e + i < e1) {
                            const uint32_t cb = s_cb[e + i];
                            m[i] = msg_load<PREC>(mp + (size_t)(cb >> 16) * p.Z + col_check_z(cb, it.z, p.Z));
                        }
                    }
#pragma unroll
                    for (int i = 0; i < 4; ++i)
                        if (e + i < e1) a = __fadd_rn(a, m[i]);
                }
                a1[v] = a;
            }
        }
        __syncthreads();
        float *tmp = cur;
        cur = nxt;
        nxt = tmp;
        if (ckpt) {
            // APP^(t+1) for the adjoint, after the message checkpoints (no early stop here)
            float *ca = p.ckpt + (size_t)(p.iters - 1) * p.ckpt_tstride + (size_t)t * p.B * p.ckpt_app_stride;
            const bool vec = (p.n & 3) == 0;  // 16-byte rows on both sides (the stride is a multiple of 32)
            for (int gg = 0; gg < p.G; ++gg) {
                const int64_t c2 = cw_base + gg;
                if (c2 >= p.B) break;
                float *dst = ca + c2 * p.ckpt_app_stride;
                const float *a = cur + (size_t)gg * p.n;
                if (vec) {
                    for (int v = threadIdx.x; v < (p.n >> 2); v += blockDim.x)
                        reinterpret_cast<float4 *>(dst)[v] = reinterpret_cast<const float4 *>(a)[v];
                } else {
                    for (int v = threadIdx.x; v < p.n; v += blockDim.x) dst[v] = a[v];
                }
            }
        }
        for (int gg = threadIdx.x; gg < p.G; gg += blockDim.x)
            if (!s_done[gg]) s_iters[gg] = t + 1;
        if (p.early_stop) {
            for (int gg = threadIdx.x; gg < p.G; gg += blockDim.x) s_flag[gg] = 0;
            __syncthreads();
            {
                GZWalk it(p.Z, p.rows);
                for (; it.g < p.G; it.next(p.Z, p.rows)) {
                    const int gg = it.g, r = it.q;
                    if (s_done[gg]) continue;
                    const float *a = cur + (size_t)gg * p.n;
                    unsigned pr = 0;
                    for (int b = s_rp[r]; b < s_rp[r + 1]; ++b) pr ^= a[vn_at(s_vb[b], it.z, p.Z)] < 0.0f ? 1u : 0u;
                    if (pr) s_flag[gg] = 1;
                }
            }
            __syncthreads();
            bool all = true;
            for (int gg = 0; gg < p.G; ++gg) all &= s_done[gg] != 0 || s_flag[gg] == 0;
            __syncthreads();
            for (int gg = threadIdx.x; gg < p.G; gg += blockDim.x)
                if (s_flag[gg] == 0) s_done[gg] = 1;
            if (__syncthreads_and(all)) break;
        }
    }
    __syncthreads();
    write_outputs(p, cur, cw_base, 0, 0, false, 1);  // APP and bits of every codeword of the CTA
    if (p.iters_out)
        for (int gg = threadIdx.x; gg < p.G; gg += blockDim.x)
            if (cw_base + gg < p.B) p.iters_out[cw_base + gg] = s_iters[gg];
}

template <int DMAX, int ALGO>
KernelFn flood_prec(int prec) {
    if (prec == kF32) return k_flooding<DMAX, ALGO, kF32>;
    if (prec == kF16) return k_flooding<DMAX, ALGO, kF16>;
    if constexpr (ALGO == kMinSum) return k_flooding<DMAX, kMinSum, kFix6>;
    return nullptr;
}

KernelFn flooding_kernel(int dmax, int algo, int prec) {
    if (dmax > 20) return nullptr;
    if (algo == kMinSum) return dmax <= 12 ? flood_prec<12, kMinSum>(prec) : flood_prec<20, kMinSum>(prec);
    return dmax <= 12 ? flood_prec<12, kSpa>(prec) : flood_prec<20, kSpa>(prec);
}

}  // namespace dec
}  // namespace ldpcx
