// Layered decoding with per-edge messages on the full 5G-shaped base graphs,
// with the layer schedule compiled in (decode_cns_sched.cuh gives the
// schedule; this is its counterpart for rules whose messages do not reduce to
// a check-node state, i.e. sum-product).
//
// Messages live circulant-contiguous, msg[cw][b Z + z] for block b of the
// row-major block order (= layer order), as in k_layered. Rows of degree up to
// kPf get their old messages prefetched into registers one layer ahead; the
// dense core rows load their own. The update is that of layer_update, so the
// results equal k_layered's bit for bit.
#pragma once

#include "decode_cns_sched.cuh"

namespace ldpcx {
namespace dec {

// Layered update of check node z of a row of exact degree D: T = APP - R_old,
// check-node rule, APP = T + R_new (rounded), store R_new. Rows with D <= kPf
// take their old messages from Rc and keep their APP offsets in registers;
// denser rows load the messages here (zero in the first iteration) and
// recompute the offsets in the second pass.
template <int D, int ALGO, int PREC>
__device__ __forceinline__ void edge_update(const Params &p, float *app, const int2 *at, int z,
                                            typename MsgT<PREC>::T *ml, const float (&Rc)[kPf], bool load,
                                            bool store) {
    constexpr bool kSparse = D <= kPf;
    float T[D];
    int vi[kSparse ? D : 1];
#pragma unroll
    for (int j = 0; j < D; ++j) {
        float old;
        if constexpr (kSparse) old = Rc[j];
        else old = load ? msg_load<PREC>(ml + (size_t)j * p.Z) : 0.0f;
        const int v = vn_off_mixed(p, at[j], z);
        if constexpr (kSparse) vi[j] = v;
        T[j] = __fsub_rn(app_at(app, v), old);
    }
    using CN = typename std::conditional<ALGO == kMinSum, FastMinSum<D>, SpaNode<D>>::type;
    CN cn;
    if constexpr (ALGO == kMinSum) cn.prepare(T, D, p.offset, p.clamp);
    else cn.prepare(T, D, p.clamp, p.phi_lo);
#pragma unroll
    for (int j = 0; j < D; ++j) {
        float r[1], rq[1];
        if constexpr (ALGO == kMinSum) r[0] = cn.value(T[j]);
        else r[0] = cn.value(j, T[j], p.clamp, p.phi_lo, p.k_one);
        MsgVec<PREC, 1>::round_store(ml + (size_t)j * p.Z, r, rq, store);
        int v;
        if constexpr (kSparse) v = vi[j];
        else v = vn_off_mixed(p, at[j], z);
        app_at(app, v) = __fadd_rn(T[j], rq[0]);
    }
}

// Old messages of the row r2 of the schedule into R (rows of degree <= kPf).
template <int BG, int PREC>
__device__ __forceinline__ void edge_prefetch(const Params &p, const typename MsgT<PREC>::T *mp, int z, int r2,
                                              float (&R)[kPf]) {
    using S = Sched<BG>;
    using L = SchedLayout<BG, PREC>;
    static_assert(S::d_hi <= kPf && S::d_lo <= kPf && S::dc0 > kPf && S::dc2 > kPf && S::dc3 > kPf &&
                      S::dc1 > kPf,
                  "extension rows are prefetched, core rows load their own messages");
    if (r2 < 4) return;
    if (r2 < 4 + S::n_hi) {
        const auto *ml = mp + (size_t)(L::b_hi + (r2 - 4) * S::d_hi) * p.Z + z;
#pragma unroll
        for (int j = 0; j < S::d_hi; ++j) R[j] = msg_load<PREC>(ml + (size_t)j * p.Z);
    } else {
        const auto *ml = mp + (size_t)(L::b_lo + (r2 - 4 - S::n_hi) * S::d_lo) * p.Z + z;
#pragma unroll
        for (int j = 0; j < S::d_lo; ++j) R[j] = msg_load<PREC>(ml + (size_t)j * p.Z);
    }
}

// One layer step of degree D on row r (blocks from b0): prefetch the next
// layer's messages into Rn, update from Rc, barrier.
template <int D, int BG, int ALGO, int PREC>
__device__ __forceinline__ void edge_step(const Params &p, const int2 *s_at, float *app,
                                          typename MsgT<PREC>::T *mp, int z, int t, int r, int b0, bool done,
                                          const float (&Rc)[kPf], float (&Rn)[kPf]) {
    using S = Sched<BG>;
    int rn = r + 1, tn = t;
    if (rn == S::rows) {
        rn = 0;
        ++tn;
    }
    if (tn == 0) {
#pragma unroll
        for (int j = 0; j < kPf; ++j) Rn[j] = 0.0f;  // iteration 0 starts from zero messages
    } else if (!done && tn < p.iters) {
        edge_prefetch<BG, PREC>(p, mp, z, rn, Rn);
    }
    if (!done)
        edge_update<D, ALGO, PREC>(p, app, s_at + b0, z, mp + (size_t)b0 * p.Z + z, Rc, t > 0, t + 1 < p.iters);
    __syncthreads();
}

// COUNT consecutive rows of degree D from row r0 (blocks from b0), the first
// at ring phase PH (even: current messages in Ra).
template <int D, int COUNT, int PH, int BG, int ALGO, int PREC>
__device__ __forceinline__ void edge_run(const Params &p, const int2 *s_at, float *app, typename MsgT<PREC>::T *mp,
                                         int z, int t, int r0, int b0, bool done, float (&Ra)[kPf],
                                         float (&Rb)[kPf]) {
    int r = r0, bb = b0;
    auto &R0 = PH % 2 == 0 ? Ra : Rb;
    auto &R1 = PH % 2 == 0 ? Rb : Ra;
#pragma unroll 1
    for (int i = 0; i < COUNT / 2; ++i) {
        edge_step<D, BG, ALGO, PREC>(p, s_at, app, mp, z, t, r, bb, done, R0, R1);
        edge_step<D, BG, ALGO, PREC>(p, s_at, app, mp, z, t, r + 1, bb + D, done, R1, R0);
        r += 2;
        bb += 2 * D;
    }
    if constexpr (COUNT % 2 == 1) edge_step<D, BG, ALGO, PREC>(p, s_at, app, mp, z, t, r, bb, done, R0, R1);
}

// CH: channel input, LLRs alone (kChLlr) or either (kChAny: the fused
// demapper's load out of line, for ldpc_bp_decode_qam).
template <int BG, int ALGO, int PREC, int ZC = 0, int CH = kChAny>
__global__ void __launch_bounds__(kMaxThreads, 2)
    k_layered_edge_sched(const __grid_constant__ Params p, const __grid_constant__ SchedTab tab) {
    using S = Sched<BG>;
    using L = SchedLayout<BG, PREC>;
    using MT = typename MsgT<PREC>::T;
    extern __shared__ __align__(16) unsigned char smem[];
    const int ZV = ZC ? ZC : p.Z;
    float *s_app_all = reinterpret_cast<float *>(smem);
    uint32_t *s_vb = reinterpret_cast<uint32_t *>(s_app_all + (size_t)p.G * p.n);
    int32_t *s_rp = reinterpret_cast<int32_t *>(s_vb + p.nnz);
    int *s_flag = reinterpret_cast<int *>(s_rp + p.rows + 1);
    const int2 *s_at = tab.at;

    load_tables(p, s_vb, s_rp);  // for the syndrome check
    const int64_t cw_base = (int64_t)blockIdx.x * p.G;
    load_channel_as<CH>(p, s_app_all, cw_base);
    const int g = threadIdx.x / ZV, z = threadIdx.x - g * ZV;
    const int64_t cw = cw_base + g;
    const bool active = g < p.G && cw < p.B;
    float *app = s_app_all + (size_t)(active ? g : 0) * p.n;
    MT *mp = reinterpret_cast<MT *>(p.msg) + (active ? cw : 0) * p.msg_stride;
    bool done = !active;
    int iters_run = 0;
    __syncthreads();

    float Ra[kPf], Rb[kPf];
#pragma unroll
    for (int j = 0; j < kPf; ++j) Ra[j] = Rb[j] = 0.0f;
    for (int t = 0; t < p.iters; ++t) {
        edge_run<S::dc0, 1, 0, BG, ALGO, PREC>(p, s_at, app, mp, z, t, 0, 0, done, Ra, Rb);
        edge_run<S::dc1, 1, 1, BG, ALGO, PREC>(p, s_at, app, mp, z, t, 1, S::dc0, done, Ra, Rb);
        edge_run<S::dc2, 1, 2, BG, ALGO, PREC>(p, s_at, app, mp, z, t, 2, S::dc0 + S::dc1, done, Ra, Rb);
        edge_run<S::dc3, 1, 3, BG, ALGO, PREC>(p, s_at, app, mp, z, t, 3, S::dc0 + S::dc1 + S::dc2, done, Ra, Rb);
        edge_run<S::d_hi, S::n_hi, 4, BG, ALGO, PREC>(p, s_at, app, mp, z, t, 4, L::b_hi, done, Ra, Rb);
        edge_run<S::d_lo, S::rows - 4 - S::n_hi, 4 + S::n_hi, BG, ALGO, PREC>(p, s_at, app, mp, z, t, 4 + S::n_hi,
                                                                             L::b_lo, done, Ra, Rb);
        if constexpr (S::rows % 2 == 1) {  // the next iteration's first row finds its messages in Rb
#pragma unroll
            for (int j = 0; j < kPf; ++j) {
                const float x = Ra[j];
                Ra[j] = Rb[j];
                Rb[j] = x;
            }
        }
        if (!done) iters_run = t + 1;
        if (p.early_stop) {
            if (threadIdx.x < p.G) s_flag[threadIdx.x] = 0;
            __syncthreads();
            if (!done && syndrome_bad_vec<1, ZC>(p, s_vb, s_rp, app, z)) s_flag[g] = 1;
            __syncthreads();
            if (!done && s_flag[g] == 0) done = true;
            if (__syncthreads_and(done)) break;
        }
    }
    __syncthreads();
    write_outputs(p, s_app_all, cw_base, iters_run, g, active, z);
}

// Kernel for a code whose row degrees follow the full base graph of shape bg,
// sum-product with FP32 or FP16 messages, or nullptr.
SchedFn layered_edge_sched_kernel(int bg, int algo, int prec, int Z, bool qam = false);

}  // namespace dec
}  // namespace ldpcx
