// Adjoint of unrolled weighted flooding sum-product BP: gradients of a loss on
// the output LLRs with respect to the channel LLRs and the per-iteration
// per-base-block weights ("gradients can be specified" for a custom op,
// Sec. IV-A; end-to-end learning, Sec. III-C).
//
// Forward (iteration t, edges e of check c, variable v(e)):
//   APP^0 = L (clamped channel LLRs),  APP^(t+1) = L + sum_e C^t_e over v's edges
//   V_e = w[t][blk(e)] (APP^t_v - C^(t-1)_e),  a_e = clamp(|V_e|, lo, hi),  f_e = phi(a_e)
//   S_e = sum_{e' != e in c} f_e',  x_e = clamp(S_e, lo, hi),  C^t_e = s_e phi(x_e)
// Reverse sweep, t = iters-1 .. 0, with gA^(t+1) = dLoss/dAPP^(t+1) known:
//   gC_e  = gA^(t+1)_v + carry_e          (carry = -w gV from iteration t+1)
//   u_e   = gC_e s_e phi'(x_e) [lo < S_e < hi]
//   gV_e  = phi'(a_e) sgn(V_e) [lo <= |V_e| <= hi] sum_{e' != e} u_e'
//   gw   += gV_e (APP^t_v - C^(t-1)_e),  gA^t_v += w gV_e,  carry_e = -w gV_e
//   dLoss/dL = sum_t gA^t (through the channel clamp).
// APP^t is the forward's own value, checkpointed after each iteration. phi and phi' are evaluated with
// the hardware exponential, reciprocal and logarithm (phi_fast, dphi_fast:
// within about 2e-5 and 1e-6 relative), the exclusive sums S_e as in the
// forward's check node (the largest term left out of the running sum) and the
// exclusive sums of u from prefix and suffix sums: O(d) per check node. dL/dL
// accumulates in grad_llr itself, iteration by iteration.
#include <math.h>

#include <type_traits>

#include "decode_kernels.cuh"

namespace ldpcx {
namespace {

struct BwdParams {
    const uint32_t *blk;
    const int32_t *row_ptr;
    int Z, rows, nnz, n, n_tx, p0, iters;
    float clamp, phi_lo;
    const float *llr;       // [B][n_tx]
    const float *weights;   // [iters][nnz] or null (all ones)
    const float *ckpt;      // [iters-1][B][stride]
    const float *ckpt_app;  // [iters-1][B][app_stride]: APP^(t+1) after forward iteration t
    int64_t stride, tstride, app_stride;
    const float *grad_out;  // [B][n]
    float *grad_llr;        // [B][n_tx]
    float *grad_w;          // [iters][nnz] (accumulated) or null
    float *carry;           // [B][stride]
    int64_t B;
    int G;
};

// phi'(x) = -1/sinh(x) from the hardware exponential; below x = 1/16, where
// e^x - e^-x would cancel, from the Taylor series sinh x = x (1 + x^2/6 (1 +
// x^2/20 (1 + x^2/42))) (truncation below 1e-12 relative there). Above it
// e - 1/e >= 0.125 loses at most a factor 16 of the exponential's relative
// error: about 1e-6 relative overall. The hardware approximations are those
// of phi_fast (every value here is a normal binary32 number).
__device__ __forceinline__ float dphi_fast(float x) {
    if (x < 0.0625f) {
        const float x2 = x * x;
        return -dec::hw_rcp(x * (1.0f + x2 * (1.0f / 6.0f) * (1.0f + x2 * (1.0f / 20.0f) * (1.0f + x2 * (1.0f / 42.0f)))));
    }
    const float e = dec::hw_exp2(x * dec::kLog2e);
    return -2.0f * dec::hw_rcp(e - dec::hw_rcp(e));
}

__device__ __forceinline__ int vn_of(uint32_t vb, int z, int Z) {
    int zz = z + (int)(vb & 0xFFFFu);
    zz -= (zz >= Z) ? Z : 0;
    return (int)(vb >> 16) + zz;
}

// Channel LLRs of codeword cw placed on the n positions and clamped (NaN -> 0).
__device__ __forceinline__ float placed_llr(const BwdParams &p, int64_t cw, int v) {
    const int t = v - p.p0;
    if (cw >= p.B || t < 0 || t >= p.n_tx) return 0.0f;
    const float x = p.llr[cw * p.n_tx + t];
    if (!(x == x)) return 0.0f;
    return fminf(fmaxf(x, -p.clamp), p.clamp);
}

// The values src[(b0 + j) Z] of this thread's edges j = q + TPC i of a row
// (zero where it has none): loaded one row ahead of their use, so that the
// global loads of the next row overlap the current row's arithmetic.
template <int DPT, int TPC>
__device__ __forceinline__ void row_values(const float *src, bool on, int b0, int deg, int q, int Z,
                                           float (&out)[DPT]) {
#pragma unroll
    for (int i = 0; i < DPT; ++i) {
        const int j = q + TPC * i;
        out[i] = (on && TPC * i < deg && j < deg) ? src[(size_t)(b0 + j) * Z] : 0.0f;
    }
}

// Sum over the TPC adjacent lanes of one check node (TPC a power of two <= 32).
template <int TPC> __device__ __forceinline__ float group_sum(float x) {
#pragma unroll
    for (int o = 1; o < TPC; o <<= 1) x += __shfl_xor_sync(0xFFFFFFFFu, x, o);
    return x;
}

// TPC threads per check node: thread q of node z takes the edges j = q, q +
// TPC, ... of the row (DPT of them at most), and the row-wide quantities (the
// sign parity, the largest phi term and the sums) are combined by shuffles
// among the node's TPC adjacent lanes. Threads: G Z TPC per CTA.
template <int DMAX, int TPC>
__global__ void __launch_bounds__(512, TPC == 4 ? 2 : 1) k_backward(const BwdParams p) {
    constexpr int DPT = (DMAX + TPC - 1) / TPC;
    extern __shared__ __align__(16) unsigned char smem[];
    const size_t gn = (size_t)p.G * p.n;
    float *s_app = reinterpret_cast<float *>(smem);
    float *s_gin = s_app + gn;   // gA^(t+1)
    float *s_gout = s_gin + gn;  // gA^t (accumulated)
    float *s_gw = s_gout + gn;   // [nnz] weight gradient of this iteration
    uint32_t *s_vb = reinterpret_cast<uint32_t *>(s_gw + p.nnz);
    int32_t *s_rp = reinterpret_cast<int32_t *>(s_vb + p.nnz);

    for (int i = threadIdx.x; i < p.nnz; i += blockDim.x) {
        const uint32_t b = p.blk[i];
        s_vb[i] = ((b >> 16) * (uint32_t)p.Z) << 16 | (b & 0xFFFFu);
        s_gw[i] = 0.0f;
    }
    for (int i = threadIdx.x; i <= p.rows; i += blockDim.x) s_rp[i] = p.row_ptr[i];
    const int64_t cw_base = (int64_t)blockIdx.x * p.G;
    for (int gg = 0; gg < p.G; ++gg) {
        const int64_t c2 = cw_base + gg;
        for (int v = threadIdx.x; v < p.n; v += blockDim.x)
            s_gin[(size_t)gg * p.n + v] = c2 < p.B ? p.grad_out[c2 * p.n + v] : 0.0f;
        if (c2 < p.B)
            for (int t = threadIdx.x; t < p.n_tx; t += blockDim.x) p.grad_llr[c2 * p.n_tx + t] = 0.0f;
    }
    const int node = threadIdx.x / TPC, q = threadIdx.x - node * TPC;
    const int g = node / p.Z, z = node - g * p.Z;
    const int64_t cw = cw_base + g;
    const bool active = g < p.G && cw < p.B;
    const size_t off = (size_t)(active ? g : 0) * p.n;
    float *carry = p.carry + (active ? cw : 0) * p.stride + z;
    const float lo = p.phi_lo, hi = p.clamp;
    float *gin = s_gin, *gout = s_gout;
    __syncthreads();

    for (int t = p.iters - 1; t >= 0; --t) {
        // APP^t: the clamped channel LLRs (t = 0) or the forward's own APP^t from its checkpoint
        const float *ca = t >= 1 ? p.ckpt_app + (size_t)(t - 1) * p.B * p.app_stride : nullptr;
        for (int gg = 0; gg < p.G; ++gg) {
            const int64_t c2 = cw_base + gg;
            for (int v = threadIdx.x; v < p.n; v += blockDim.x)
                s_app[(size_t)gg * p.n + v] = !ca ? placed_llr(p, c2, v) : c2 < p.B ? ca[c2 * p.app_stride + v] : 0.0f;
        }
        const float *ck = t >= 1 ? p.ckpt + (size_t)(t - 1) * p.tstride + (active ? cw : 0) * p.stride + z : nullptr;
        // dLoss/dL collects every gA^(t+1) (transmitted positions only); gA^t starts from zero
        for (int gg = 0; gg < p.G; ++gg) {
            const int64_t c2 = cw_base + gg;
            if (c2 >= p.B) break;
            for (int tt = threadIdx.x; tt < p.n_tx; tt += blockDim.x)
                p.grad_llr[c2 * p.n_tx + tt] += gin[(size_t)gg * p.n + p.p0 + tt];
        }
        for (size_t i = threadIdx.x; i < gn; i += blockDim.x) gout[i] = 0.0f;
        __syncthreads();
        const float *w_t = p.weights ? p.weights + (size_t)t * p.nnz : nullptr;
        const bool has_carry = t + 1 < p.iters;
        float ckn[DPT], cyn[DPT];  // the next row's checkpointed messages and carries
        row_values<DPT, TPC>(ck, active && ck, s_rp[0], s_rp[1] - s_rp[0], q, p.Z, ckn);
        row_values<DPT, TPC>(carry, active && has_carry, s_rp[0], s_rp[1] - s_rp[0], q, p.Z, cyn);
        for (int r = 0; r < p.rows; ++r) {
            const int b0 = s_rp[r], deg = s_rp[r + 1] - b0;
            float ckc[DPT], cyc[DPT];
#pragma unroll
            for (int i = 0; i < DPT; ++i) {
                ckc[i] = ckn[i];
                cyc[i] = cyn[i];
            }
            if (r + 1 < p.rows) {
                const int b1 = s_rp[r + 1], d1 = s_rp[r + 2] - b1;
                row_values<DPT, TPC>(ck, active && ck, b1, d1, q, p.Z, ckn);
                row_values<DPT, TPC>(carry, active && has_carry, b1, d1, q, p.Z, cyn);
            }
            // the row body for NS edge slots per lane (the row's own count: one for a degree of at most TPC), so
            // that no slot the row does not use is issued; the same operations in the same order for any NS
            auto row_body = [&](auto ns_tag) {
                constexpr int NS = decltype(ns_tag)::value;
                float gw[NS];
                float V[NS], d[NS], f[NS], u[NS];
                int vi[NS];
                // this thread's edges: the sign parity, its largest phi term and their sum
                unsigned par = 0;
                float fmax = -1.0f;
                int im = -1;
    #pragma unroll
                for (int i = 0; i < NS; ++i) {
                    const int j = q + TPC * i;
                    gw[i] = V[i] = d[i] = f[i] = u[i] = 0.0f;
                    vi[i] = 0;
                    if (TPC * i < deg && active && j < deg) {  // the first test is warp-uniform
                        vi[i] = vn_of(s_vb[b0 + j], z, p.Z);
                        d[i] = __fsub_rn(s_app[off + vi[i]], ckc[i]);
                        V[i] = w_t ? __fmul_rn(w_t[b0 + j], d[i]) : d[i];
                        f[i] = dec::phi_fast(fminf(fmaxf(fabsf(V[i]), lo), hi));
                        par ^= V[i] < 0.0f ? 1u : 0u;
                        if (f[i] > fmax) {
                            fmax = f[i];
                            im = i;
                        }
                    }
                }
                // the row's largest term (ties: the lowest edge index) leaves the running sum, as in the forward
                float rmax = fmax;
                int jmax = im >= 0 ? q + TPC * im : DMAX;
    #pragma unroll
                for (int o = 1; o < TPC; o <<= 1) {
                    const float om = __shfl_xor_sync(0xFFFFFFFFu, rmax, o);
                    const int oj = __shfl_xor_sync(0xFFFFFFFFu, jmax, o);
                    if (om > rmax || (om == rmax && oj < jmax)) {
                        rmax = om;
                        jmax = oj;
                    }
                }
    #pragma unroll
                for (int o = 1; o < TPC; o <<= 1) par ^= __shfl_xor_sync(0xFFFFFFFFu, par, o);
                float part = 0.0f;
    #pragma unroll
                for (int i = 0; i < NS; ++i)
                    if (q + TPC * i < deg && q + TPC * i != jmax) part += f[i];
                const float s_rest = group_sum<TPC>(part);
                const float s_all = s_rest + rmax;
                // u_e = gC_e s_e phi'(x_e) [lo < S_e < hi]
                float usum = 0.0f;
    #pragma unroll
                for (int i = 0; i < NS; ++i) {
                    const int j = q + TPC * i;
                    if (TPC * i < deg && active && j < deg) {  // the first test is warp-uniform
                        const float S = j == jmax ? s_rest : s_all - f[i];
                        const float gC = gin[off + vi[i]] + cyc[i];
                        const float sg = (par ^ (V[i] < 0.0f ? 1u : 0u)) ? -1.0f : 1.0f;
                        u[i] = (S > lo && S < hi) ? gC * sg * dphi_fast(S) : 0.0f;
                        usum += u[i];
                    }
                }
                const float U_all = group_sum<TPC>(usum);
                // gV_e = phi'(a_e) sgn(V_e) [lo <= |V_e| <= hi] sum_{e' != e} u_e'
    #pragma unroll
                for (int i = 0; i < NS; ++i) {
                    const int j = q + TPC * i;
                    if (TPC * i < deg && active && j < deg) {  // the first test is warp-uniform
                        const float U = U_all - u[i];
                        const float a = fabsf(V[i]);
                        const bool inside = a >= lo && a <= hi;
                        const float gV = inside ? dphi_fast(a) * (V[i] < 0.0f ? -1.0f : 1.0f) * U : 0.0f;
                        const float w = w_t ? w_t[b0 + j] : 1.0f;
                        gw[i] = gV * d[i];
                        gout[off + vi[i]] += w * gV;
                        carry[(size_t)(b0 + j) * p.Z] = -w * gV;
                    }
                }
                // weight gradient: the lanes of a warp with the same q are at the same blocks b0 + q + TPC i
                if (p.grad_w) {
    #pragma unroll
                    for (int i = 0; i < NS; ++i) {
                        if (TPC * i < deg) {  // warp-uniform: some lane of the warp has an edge in slot i
                            float x = gw[i];
    #pragma unroll
                            for (int o = TPC; o < 32; o <<= 1) x += __shfl_xor_sync(0xFFFFFFFFu, x, o);
                            const int j = q + TPC * i;
                            if ((threadIdx.x & 31) < TPC && j < deg && x != 0.0f) atomicAdd(&s_gw[b0 + j], x);
                        }
                    }
                }
            };
            const int ns = (deg + TPC - 1) / TPC;
            if constexpr (DPT >= 2) {
                if (ns == 1) row_body(std::integral_constant<int, 1>{});
                else if (ns == 2) row_body(std::integral_constant<int, 2>{});
                else row_body(std::integral_constant<int, DPT>{});
            } else {
                row_body(std::integral_constant<int, DPT>{});
            }
            __syncthreads();  // rows add into gA^t in ascending order
        }
        if (p.grad_w) {
            for (int i = threadIdx.x; i < p.nnz; i += blockDim.x) {
                atomicAdd(&p.grad_w[(size_t)t * p.nnz + i], s_gw[i]);
                s_gw[i] = 0.0f;
            }
        }
        float *tmp = gin;
        gin = gout;
        gout = tmp;
        __syncthreads();
    }
    // dLoss/dL += gA^0, then through the channel clamp (each thread revisits only its own entries)
    for (int gg = 0; gg < p.G; ++gg) {
        const int64_t c2 = cw_base + gg;
        if (c2 >= p.B) break;
        for (int t = threadIdx.x; t < p.n_tx; t += blockDim.x) {
            const float x = p.llr[c2 * p.n_tx + t];
            const bool pass = (x == x) && fabsf(x) <= p.clamp;
            const float gsum = p.grad_llr[c2 * p.n_tx + t] + gin[(size_t)gg * p.n + p.p0 + t];
            p.grad_llr[c2 * p.n_tx + t] = pass ? gsum : 0.0f;
        }
    }
}

size_t bwd_smem(int G, int n, int nnz, int rows) {
    return sizeof(float) * (3 * (size_t)G * n + nnz) + sizeof(uint32_t) * nnz + sizeof(int32_t) * (rows + 1);
}

int64_t stride_of(const ldpcx_code *c) {
    const int64_t E = (int64_t)c->nnz * c->Z;
    return (E + 127) / 128 * 128;
}

int check_bwd(const ldpcx_code *c, const ldpcx_decode_opts *o) {
    size_t tmp = 0;
    int st = ldpc_bp_workspace(const_cast<ldpcx_code *>(c), 1, o, &tmp);  // validates the options
    if (st) return st;
    if (o->algo != LDPCX_FLOOD_SPA || o->msg_prec != LDPCX_MSG_F32 || o->early_stop) return LDPCX_E_UNSUPPORTED;
    if (c->n_fill) return LDPCX_E_UNSUPPORTED;  // channel LLRs are read in the unshortened layout
    if (bwd_smem(1, c->n, c->nnz, c->rows) > 216 * 1024) return LDPCX_E_UNSUPPORTED;
    return LDPCX_OK;
}

}  // namespace
}  // namespace ldpcx

using namespace ldpcx;

extern "C" int ldpc_bp_backward_workspace(ldpcx_code_t c, int64_t B, const ldpcx_decode_opts *o, size_t *ws) {
    if (!c || !ws || B < 0 || !o) return LDPCX_E_INVAL;
    int st = check_bwd(c, o);
    if (st) return st;
    *ws = sizeof(float) * (size_t)B * (size_t)stride_of(c);
    return LDPCX_OK;
}

extern "C" int ldpc_bp_backward(ldpcx_code_t c, const float *llr_ch, int64_t B, const ldpcx_decode_opts *o,
                                const void *ckpt, size_t ckpt_bytes_in, const float *grad_llr_out,
                                float *grad_llr_ch, float *grad_weights, void *ws, size_t ws_bytes, void *stream) {
    if (!c || B < 0 || !o) return LDPCX_E_INVAL;
    int st = check_bwd(c, o);
    if (st) return st;
    if (B == 0) return LDPCX_OK;
    if (!llr_ch || !grad_llr_out || !grad_llr_ch) return LDPCX_E_INVAL;
    if (!ckpt || ckpt_bytes_in < ckpt_bytes(c, B, o->iters) || ((uintptr_t)ckpt & 15u)) return LDPCX_E_WORKSPACE;
    const size_t need = sizeof(float) * (size_t)B * (size_t)stride_of(c);
    if (!ws || ws_bytes < need || ((uintptr_t)ws & 15u)) return LDPCX_E_WORKSPACE;
    DevCode d;
    st = code_device(c, &d);
    if (st) return st;

    BwdParams p{};
    p.blk = d.blk;
    p.row_ptr = d.row_ptr;
    p.Z = c->Z;
    p.rows = c->rows;
    p.nnz = c->nnz;
    p.n = c->n;
    p.n_tx = c->n_tx;
    p.p0 = c->p0;
    p.iters = o->iters;
    p.clamp = o->clamp;
    p.phi_lo = (float)log1p(2.0 / expm1((double)o->clamp));
    p.llr = llr_ch;
    p.weights = o->weights;
    p.ckpt = (const float *)ckpt;
    p.stride = stride_of(c);
    p.tstride = B * p.stride;
    p.app_stride = ckpt_app_stride(c->n);
    p.ckpt_app = p.ckpt + (size_t)(o->iters > 1 ? o->iters - 1 : 1) * p.tstride;
    p.grad_out = grad_llr_out;
    p.grad_llr = grad_llr_ch;
    p.grad_w = grad_weights;
    p.carry = (float *)ws;
    p.B = B;
    // threads per check node: as many as keep a CTA within 512 threads
    const int tpc = c->Z <= 128 ? 4 : c->Z <= 256 ? 2 : 1;
    int G = 512 / (c->Z * tpc);
    if (G < 1) G = 1;
    const size_t cap = tpc == 4 ? 112 * 1024 : 216 * 1024;  // two CTAs per SM with four threads per node
    while (G > 1 && bwd_smem(G, c->n, c->nnz, c->rows) > cap) --G;
    p.G = G;
    const size_t smem = bwd_smem(G, c->n, c->nnz, c->rows);
    void (*fn)(BwdParams) = nullptr;
    if (c->max_deg <= 12) fn = tpc == 4 ? k_backward<12, 4> : tpc == 2 ? k_backward<12, 2> : k_backward<12, 1>;
    else fn = tpc == 4 ? k_backward<20, 4> : tpc == 2 ? k_backward<20, 2> : k_backward<20, 1>;
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return LDPCX_E_CUDA;
    const int threads = (G * c->Z * tpc + 31) / 32 * 32;
    const int64_t grid = (B + G - 1) / G;
    fn<<<(unsigned)grid, threads, smem, (cudaStream_t)stream>>>(p);
    return cudaGetLastError() == cudaSuccess ? LDPCX_OK : LDPCX_E_CUDA;
}
