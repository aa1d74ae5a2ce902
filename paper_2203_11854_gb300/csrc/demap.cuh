// Gray-QAM APP demapper of one received symbol (Demapper("app") of the
// paper's Listing 1), shared by the standalone demapper kernel and the
// decoders' fused channel load so that both compute the same LLRs bit for bit.
//
// Per I/Q dimension (exact for square Gray QAM: the other dimension's
// distance terms cancel): metrics d_l = -(y - A_l s)^2 / N0 over the 2^h PAM
// levels A_l; bit i of the dimension = LSE over levels whose label has bit i
// = 0 minus LSE over those with bit i = 1 (max instead of LSE for max-log),
// clamped to [-clamp, clamp]. Every operation is rounded on its own (no fused
// multiply-add), so the values do not depend on how a kernel is compiled.
#pragma once

#include <math.h>

#include "ldpcx.h"

namespace ldpcx {

inline bool valid_m(int m) { return m == 1 || m == 2 || m == 4 || m == 6 || m == 8; }

// 1 / sqrt(2 (4^h - 1) / 3): unit average symbol energy of the 2^(2h)-point square QAM (1 for BPSK).
inline float qam_scale(int m) {
    if (m == 1) return 1.0f;
    const int h = m / 2;
    return (float)(1.0 / sqrt(2.0 * (double)((1 << (2 * h)) - 1) / 3.0));
}

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
        const float e = __fsub_rn(y, __fmul_rn((float)inner, scale));
        d[l] = __fmul_rn(-__fmul_rn(e, e), inv_n0);
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
            L = __fsub_rn(mx0, mx1);
        } else {
            float s0 = 0.0f, s1 = 0.0f;
#pragma unroll
            for (int l = 0; l < P; ++l) {
                if ((l >> bit) & 1) s1 = __fadd_rn(s1, expf(__fsub_rn(d[l], mx1)));
                else s0 = __fadd_rn(s0, expf(__fsub_rn(d[l], mx0)));
            }
            L = __fadd_rn(__fsub_rn(mx0, mx1), __fsub_rn(logf(s0), logf(s1)));
        }
        out[i] = fminf(fmaxf(L, -clamp), clamp);
    }
}

// demap_dim with a-priori LLRs la[0..H) of the dimension's bits: the metric of
// level l gains sum_i (1 - 2 a_i(l)) la_i / 2. Extrinsic output leaves bit i's
// own term out, which shifts the two sets of bit i by -la_i/2 and +la_i/2, so
// it is the a-posteriori value minus la_i. With zero priors the values are
// demap_dim's (the same roundings; an added zero changes nothing).
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
        const float e = __fsub_rn(y, __fmul_rn((float)inner, scale));
        float pr = 0.0f;
#pragma unroll
        for (int i = 0; i < H; ++i) pr = __fadd_rn(pr, ((l >> (H - 1 - i)) & 1) ? -la[i] : la[i]);
        d[l] = __fmaf_rn(0.5f, pr, __fmul_rn(-__fmul_rn(e, e), inv_n0));
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
            L = __fsub_rn(mx0, mx1);
        } else {
            float s0 = 0.0f, s1 = 0.0f;
#pragma unroll
            for (int l = 0; l < P; ++l) {
                if ((l >> bit) & 1) s1 = __fadd_rn(s1, expf(__fsub_rn(d[l], mx1)));
                else s0 = __fadd_rn(s0, expf(__fsub_rn(d[l], mx0)));
            }
            L = __fadd_rn(__fsub_rn(mx0, mx1), __fsub_rn(logf(s0), logf(s1)));
        }
        if (out_mode == LDPCX_DEMAP_OUT_EXTRINSIC) L = __fsub_rn(L, la[i]);
        out[i] = fminf(fmaxf(L, -clamp), clamp);
    }
}

// The M LLRs of one received symbol (re, im); M = 1 reads re alone), bit i
// of the symbol at out[i]: I bits at even i, Q bits at odd i. A non-finite
// symbol gives zeros and sets bad.
template <int M>
__device__ __forceinline__ void demap_symbol(float re, float im, float inv_n0, float scale, int method, float clamp,
                                             float (&out)[M], bool &bad) {
    if constexpr (M == 1) {
        const float x = re;
        float L = __fmul_rn(__fmul_rn(4.0f, x), inv_n0);
        if (!isfinite(x)) {
            bad = true;
            L = 0.0f;
        }
        out[0] = fminf(fmaxf(L, -clamp), clamp);
    } else {
        constexpr int H = M / 2;
        const float2 s = make_float2(re, im);
        float oi[H], oq[H];
        if (isfinite(s.x) && isfinite(s.y)) {
            demap_dim<H>(s.x, inv_n0, scale, method, clamp, oi);
            demap_dim<H>(s.y, inv_n0, scale, method, clamp, oq);
        } else {
            bad = true;
#pragma unroll
            for (int j = 0; j < H; ++j) oi[j] = oq[j] = 0.0f;
        }
#pragma unroll
        for (int j = 0; j < H; ++j) {
            out[2 * j] = oi[j];
            out[2 * j + 1] = oq[j];
        }
    }
}

}  // namespace ldpcx
