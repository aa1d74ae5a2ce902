// Flooding decoder kernels (weighted), all message formats, one, two or four
// threads per check node.
#include "decode_kernels.cuh"

namespace ldpcx {
namespace dec {

// Flooding check-node update by TPC threads per check node: thread q takes
// the edges j = q, q + TPC, ... of the row (DPT at most) and the row-wide
// quantities are combined by shuffles among the node's TPC adjacent lanes.
// Every lane of the warp calls it (act = false: neutral values, no stores).
// Min-sum: the two smallest |T| merge exactly (min of the minima, min of the
// larger first minimum and the second minima), the sign parity by XOR, and an
// edge takes v2 when |T_j| equals the smallest (= the first index of it, as
// m2 = m1 on ties), so results equal the one-thread rule bit for bit.
// Sum-product: phi_fast; the row's largest term (lowest index on ties) stays
// out of the running sum as in CheckNode, the partial sums combine by shuffles.
template <int DMAX, int ALGO, int PREC, int TPC>
__device__ __forceinline__ void flood_update_tpc(const Params &p, bool act, int deg, const float *app, float *acc,
                                                 const uint32_t *vb, int z, int q, typename MsgT<PREC>::T *ml,
                                                 const float *w, bool load, bool store, float *ck) {
    using MT = typename MsgT<PREC>::T;
    constexpr int DPT = (DMAX + TPC - 1) / TPC;
    float T[DPT];
    unsigned par = 0;
#pragma unroll
    for (int i = 0; i < DPT; ++i) {
        const int j = q + TPC * i;
        T[i] = 0.0f;
        if (TPC * i < deg && act && j < deg) {  // TPC i < deg: warp-uniform, skips slots no lane uses
            const float old = load ? msg_load<PREC>(ml + (size_t)j * p.Z) : 0.0f;
            float v2c = __fsub_rn(app[vn_at(vb[j], z, p.Z)], old);
            if (w) v2c = __fmul_rn(w[j], v2c);
            T[i] = v2c;
            par ^= T[i] < 0.0f ? 1u : 0u;
        }
    }
#pragma unroll
    for (int o = 1; o < TPC; o <<= 1) par ^= __shfl_xor_sync(0xFFFFFFFFu, par, o);
    float val[DPT];
    if constexpr (ALGO == kMinSum) {
        float m1 = INFINITY, m2 = INFINITY;
#pragma unroll
        for (int i = 0; i < DPT; ++i) {
            if (act && q + TPC * i < deg) {
                const float a = fabsf(T[i]);
                m2 = fminf(m2, fmaxf(m1, a));
                m1 = fminf(m1, a);
            }
        }
#pragma unroll
        for (int o = 1; o < TPC; o <<= 1) {
            const float o1 = __shfl_xor_sync(0xFFFFFFFFu, m1, o), o2 = __shfl_xor_sync(0xFFFFFFFFu, m2, o);
            m2 = fminf(fmaxf(m1, o1), fminf(m2, o2));
            m1 = fminf(m1, o1);
        }
        const float v1 = fminf(fmaxf(__fsub_rn(m1, p.offset), 0.0f), p.clamp);
        const float v2 = fminf(fmaxf(__fsub_rn(m2, p.offset), 0.0f), p.clamp);
#pragma unroll
        for (int i = 0; i < DPT; ++i) {
            const float mag = fabsf(T[i]) == m1 ? v2 : v1;
            val[i] = (par ^ (T[i] < 0.0f ? 1u : 0u)) ? -mag : mag;
        }
    } else {
        float f[DPT];
        float fmax = -1.0f;
        int jmax = DMAX;
#pragma unroll
        for (int i = 0; i < DPT; ++i) {
            f[i] = 0.0f;
            if (TPC * i < deg && act && q + TPC * i < deg) {
                f[i] = phi_fast(fminf(fmaxf(fabsf(T[i]), p.phi_lo), p.clamp));
                if (f[i] > fmax) {
                    fmax = f[i];
                    jmax = q + TPC * i;
                }
            }
        }
#pragma unroll
        for (int o = 1; o < TPC; o <<= 1) {
            const float om = __shfl_xor_sync(0xFFFFFFFFu, fmax, o);
            const int oj = __shfl_xor_sync(0xFFFFFFFFu, jmax, o);
            if (om > fmax || (om == fmax && oj < jmax)) {
                fmax = om;
                jmax = oj;
            }
        }
        float part = 0.0f;
#pragma unroll
        for (int i = 0; i < DPT; ++i)
            if (act && q + TPC * i < deg && q + TPC * i != jmax) part = __fadd_rn(part, f[i]);
#pragma unroll
        for (int o = 1; o < TPC; o <<= 1) part = __fadd_rn(part, __shfl_xor_sync(0xFFFFFFFFu, part, o));
        const float s_rest = part, s_all = __fadd_rn(s_rest, fmax);
#pragma unroll
        for (int i = 0; i < DPT; ++i) {
            val[i] = 0.0f;
            if (TPC * i < deg) {
                float x = (q + TPC * i == jmax) ? s_rest : __fsub_rn(s_all, f[i]);
                x = fminf(fmaxf(x, p.phi_lo), p.clamp);
                const float mag = fminf(phi_fast(x), p.clamp);
                val[i] = (par ^ (T[i] < 0.0f ? 1u : 0u)) ? -mag : mag;
            }
        }
    }
#pragma unroll
    for (int i = 0; i < DPT; ++i) {
        const int j = q + TPC * i;
        if (TPC * i < deg && act && j < deg) {
            MT mq;
            const float rq = msg_round<PREC>(val[i], &mq);
            if (store) msg_store<PREC>(ml + (size_t)j * p.Z, mq);
            if (ck) ck[(size_t)j * p.Z] = rq;  // checkpoint of C^t for the adjoint
            const int v = vn_at(vb[j], z, p.Z);
            acc[v] = __fadd_rn(acc[v], rq);
        }
    }
}

// Flooding BP, G codewords per CTA of G Z TPC threads (TPC threads per check
// node of the current row). Rows add into the accumulator one after another,
// so the APP sums run in ascending row order.
template <int DMAX, int ALGO, int PREC, int TPC>
__global__ void __launch_bounds__(512, TPC > 1 ? 2 : 1) k_flooding(const __grid_constant__ Params p) {
    using MT = typename MsgT<PREC>::T;
    extern __shared__ __align__(16) unsigned char smem[];
    float *s_a = reinterpret_cast<float *>(smem);
    float *s_b = s_a + (size_t)p.G * p.n;
    uint32_t *s_vb = reinterpret_cast<uint32_t *>(s_b + (size_t)p.G * p.n);
    int32_t *s_rp = reinterpret_cast<int32_t *>(s_vb + p.nnz);
    int *s_flag = reinterpret_cast<int *>(s_rp + p.rows + 1);
    int *s_done = s_flag + p.G;

    load_tables(p, s_vb, s_rp);
    const int64_t cw_base = (int64_t)blockIdx.x * p.G;
    for (int i = threadIdx.x; i < p.G; i += blockDim.x) s_done[i] = (cw_base + i >= p.B) ? 1 : 0;
    load_channel_llr(p, s_a, cw_base);  // the flooding decoders take LLRs only

    const int node = threadIdx.x / TPC, q = threadIdx.x - node * TPC;
    const int g = node / p.Z, z = node - g * p.Z;
    const int64_t cw = cw_base + g;
    const bool active = g < p.G && cw < p.B;
    MT *mp = reinterpret_cast<MT *>(p.msg) + (active ? cw : 0) * p.msg_stride + z;
    bool done = !active;
    int iters_run = 0;
    float *cur = s_a, *nxt = s_b;  // APP of the previous iteration / accumulator

    for (int t = 0; t < p.iters; ++t) {
        const bool store = t + 1 < p.iters;
        __syncthreads();
        // the accumulator starts from the channel LLRs; a stopped codeword
        // carries its APP forward unchanged
        {
            bool bad = false;
            for (int gg = 0; gg < p.G; ++gg) {
                const int64_t c2 = cw_base + gg;
                const bool keep = s_done[gg] != 0;
                for (int v = threadIdx.x; v < p.n; v += blockDim.x)
                    nxt[(size_t)gg * p.n + v] = keep ? cur[(size_t)gg * p.n + v] : channel_llr(p, c2, v, bad);
            }
        }
        __syncthreads();
        const float *app = cur + (size_t)(active ? g : 0) * p.n;
        float *acc = nxt + (size_t)(active ? g : 0) * p.n;
        const float *w_t = p.weights ? p.weights + (size_t)t * p.nnz : nullptr;
        for (int r = 0; r < p.rows; ++r) {
            const int b0 = s_rp[r], deg = s_rp[r + 1] - b0;
            auto *ml = mp + (size_t)b0 * p.Z;
            const float *w = w_t ? w_t + b0 : nullptr;
            float *ck = (p.ckpt && store && active) ? p.ckpt + (size_t)t * p.ckpt_tstride + (size_t)cw * p.msg_stride +
                                                          (size_t)b0 * p.Z + z
                                                    : nullptr;
            flood_update_tpc<DMAX, ALGO, PREC, TPC>(p, !done, deg, app, acc, s_vb + b0, z, q, ml, w, t > 0, store,
                                                    ck);
            __syncthreads();  // rows add into the accumulator in ascending order
        }
        float *tmp = cur;
        cur = nxt;
        nxt = tmp;
        if (p.ckpt && store) {
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
        if (!done) iters_run = t + 1;
        if (p.early_stop) {
            if (threadIdx.x < p.G) s_flag[threadIdx.x] = 0;
            __syncthreads();
            // the node's TPC threads split its rows
            if (!done) {
                bool bad = false;
                const float *a = cur + (size_t)g * p.n;
                for (int r = q; r < p.rows; r += TPC) {
                    unsigned pr = 0;
                    for (int b = s_rp[r]; b < s_rp[r + 1]; ++b) pr ^= a[vn_at(s_vb[b], z, p.Z)] < 0.0f ? 1u : 0u;
                    bad |= pr != 0;
                }
                if (bad) s_flag[g] = 1;
            }
            __syncthreads();
            if (!done && s_flag[g] == 0) {
                done = true;
                if (z == 0 && q == 0) s_done[g] = 1;
            }
            if (__syncthreads_and(done)) break;
        }
    }
    __syncthreads();
    write_outputs(p, cur, cw_base, iters_run, g, active, q == 0 ? z : 1);
}


template <int DMAX, int ALGO, int TPC>
KernelFn flood_prec(int prec) {
    if (prec == kF32) return k_flooding<DMAX, ALGO, kF32, TPC>;
    if (prec == kF16) return k_flooding<DMAX, ALGO, kF16, TPC>;
    if constexpr (ALGO == kMinSum) return k_flooding<DMAX, kMinSum, kFix6, TPC>;
    return nullptr;
}

template <int TPC>
KernelFn flood_tpc(int dmax, int algo, int prec) {
    if (algo == kMinSum) return dmax <= 12 ? flood_prec<12, kMinSum, TPC>(prec) : flood_prec<20, kMinSum, TPC>(prec);
    return dmax <= 12 ? flood_prec<12, kSpa, TPC>(prec) : flood_prec<20, kSpa, TPC>(prec);
}

KernelFn flooding_kernel(int dmax, int algo, int prec, int tpc) {
    if (dmax > 20) return nullptr;
    if (tpc == 4) return flood_tpc<4>(dmax, algo, prec);
    if (tpc == 2) return flood_tpc<2>(dmax, algo, prec);
    if (tpc == 1) return flood_tpc<1>(dmax, algo, prec);
    return nullptr;
}

}  // namespace dec
}  // namespace ldpcx
