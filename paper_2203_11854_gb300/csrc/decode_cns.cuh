// Layered offset min-sum with check-node state instead of per-edge messages.
//
// A min-sum check node sends only two magnitudes: v2 on the edges whose |T|
// equalled the minimum and v1 on the others, each with its own sign. So the
// messages of check node (r, z) are kept as one state slot: the two magnitudes
// rounded to the message format, and two bit masks over the row's edges -- eq
// (the edge took v2) and neg (the message is negative). Every message is
// rebuilt exactly as the per-edge store would have held it: rounding to FP16
// (RNE) and to the 6-bit format is symmetric in the sign, so
// round(+-mag) = +-round(mag); the 6-bit format carries no negative zero.
//
// Slot sizes (bytes) by format and row degree d:
//   FP32: 16  {v1, v2, eq, neg}
//   FP16:  8  {half v1 | half v2 << 16, eq | neg << 16}          (d <= 16)
//         16  {halves, eq, neg, 0}                                (d <= 32)
//   FIX6:  4  {q1 | q2 << 5 | eq << 10 | neg << 21}              (d <= 11)
//          8  {q1 | q2 << 5 | eq << 10, neg}                      (d <= 22)
//         16  {q1 | q2 << 8, eq, neg, 0}                          (d <= 32)
// (q = magnitude in steps of 0.5, 0..31). Row r's slots are contiguous:
// state[cw] + off_r + z * slot_r, so a warp's 32 slots are one coalesced access.
#pragma once

#include "decode_kernels.cuh"

namespace ldpcx {
namespace dec {

template <int PREC>
__host__ __device__ constexpr int cns_slot_bytes(int d) {
    if (PREC == kF32) return 16;
    if (PREC == kF16) return d <= 16 ? 8 : 16;
    return d <= 11 ? 4 : d <= 22 ? 8 : 16;
}

// Rounded magnitudes of a state.
template <int PREC> struct CnsMag;
template <> struct CnsMag<kF32> {
    float r1, r2;
    __device__ __forceinline__ void set(float v1, float v2) {
        r1 = v1;
        r2 = v2;
    }
    // message of an edge: +-(eq ? r2 : r1), negative zero kept
    __device__ __forceinline__ float msg(unsigned eq, unsigned neg) const {
        const float m = eq ? r2 : r1;
        return __uint_as_float(__float_as_uint(m) | (neg << 31));
    }
};
template <> struct CnsMag<kF16> {
    unsigned w;  // the two binary16 magnitudes, r1 in the low half
    float r1, r2;
    __device__ __forceinline__ void set(float v1, float v2) {
        const __half2 h = __floats2half2_rn(v1, v2);  // each rounded to nearest even
        w = *reinterpret_cast<const unsigned *>(&h);
        const float2 f = __half22float2(h);
        r1 = f.x;
        r2 = f.y;
    }
    __device__ __forceinline__ void from_bits(unsigned bits) {
        w = bits;
        const float2 f = __half22float2(*reinterpret_cast<const __half2 *>(&bits));
        r1 = f.x;
        r2 = f.y;
    }
    __device__ __forceinline__ float msg(unsigned eq, unsigned neg) const {
        const float m = eq ? r2 : r1;
        return __uint_as_float(__float_as_uint(m) | (neg << 31));
    }
};
// The 0.5 grid with FP32 adds instead of conversion instructions: adding
// 1.5 * 2^22 (whose ulp is 0.5) rounds 0 <= x < 2^21 to the nearest multiple of
// 0.5, ties to an even number of halves (= rint(2 x) / 2), and leaves that
// number of halves as an integer in the low mantissa bits; subtracting it back
// is exact.
constexpr float kHalfMagic = 6291456.0f;  // 1.5 * 2^22, bits 0x4AC00000

template <> struct CnsMag<kFix6> {
    int q1, q2;      // magnitude codes 0..31 (steps of 0.5)
    float r1, r2;    // their values
    // q = min(31, rint(2 v)) and r = q / 2 for 0 <= v <= clamp
    __device__ __forceinline__ void set(float v1, float v2) {
        const float a = fminf(__fadd_rn(v1, kHalfMagic), kHalfMagic + 15.5f);
        const float b = fminf(__fadd_rn(v2, kHalfMagic), kHalfMagic + 15.5f);
        q1 = (int)(__float_as_uint(a) & 63u);
        q2 = (int)(__float_as_uint(b) & 63u);
        r1 = __fsub_rn(a, kHalfMagic);
        r2 = __fsub_rn(b, kHalfMagic);
    }
    __device__ __forceinline__ void values() {
        r1 = __fsub_rn(__uint_as_float(0x4AC00000u | (unsigned)q1), kHalfMagic);
        r2 = __fsub_rn(__uint_as_float(0x4AC00000u | (unsigned)q2), kHalfMagic);
    }
    // The 6-bit store holds a signed integer, so it has no negative zero; a
    // zero message here may carry the sign bit. Both give the same sums: the
    // APP and T values are never -0 (the channel load maps -0 to +0, and
    // x - x = +0 under round-to-nearest), and for such x, x + (-0) = x - (-0) = x.
    __device__ __forceinline__ float msg(unsigned eq, unsigned neg) const {
        const float m = eq ? r2 : r1;
        return __uint_as_float(__float_as_uint(m) | (neg << 31));
    }
};

// Packed state <-> (magnitudes, eq, neg) for a row of degree d.
template <int PREC>
__device__ __forceinline__ uint4 cns_pack(const CnsMag<PREC> &m, unsigned eq, unsigned neg, int d) {
    if constexpr (PREC == kF32) {
        return make_uint4(__float_as_uint(m.r1), __float_as_uint(m.r2), eq, neg);
    } else if constexpr (PREC == kF16) {
        if (d <= 16) return make_uint4(m.w, neg | (eq << 16), 0u, 0u);
        return make_uint4(m.w, eq, neg, 0u);
    } else {
        if (d <= 11) return make_uint4((unsigned)m.q1 | ((unsigned)m.q2 << 5) | (eq << 10) | (neg << 21), 0u, 0u, 0u);
        if (d <= 22) return make_uint4((unsigned)m.q1 | ((unsigned)m.q2 << 5) | (eq << 10), neg, 0u, 0u);
        return make_uint4((unsigned)m.q1 | ((unsigned)m.q2 << 8), eq, neg, 0u);
    }
}

template <int PREC>
__device__ __forceinline__ void cns_unpack(const uint4 &s, int d, CnsMag<PREC> &m, unsigned &eq, unsigned &neg) {
    if constexpr (PREC == kF32) {
        m.r1 = __uint_as_float(s.x);
        m.r2 = __uint_as_float(s.y);
        eq = s.z;
        neg = s.w;
    } else if constexpr (PREC == kF16) {
        m.from_bits(s.x);
        if (d <= 16) {
            eq = s.y >> 16;
            neg = s.y & 0xFFFFu;
        } else {
            eq = s.y;
            neg = s.z;
        }
    } else {
        if (d <= 11) {
            m.q1 = (int)(s.x & 31u);
            m.q2 = (int)((s.x >> 5) & 31u);
            eq = (s.x >> 10) & 0x7FFu;
            neg = s.x >> 21;
        } else if (d <= 22) {
            m.q1 = (int)(s.x & 31u);
            m.q2 = (int)((s.x >> 5) & 31u);
            eq = s.x >> 10;
            neg = s.y;
        } else {
            m.q1 = (int)(s.x & 0xFFu);
            m.q2 = (int)((s.x >> 8) & 0xFFu);
            eq = s.y;
            neg = s.z;
        }
        m.values();
    }
}

// The same layouts as a compile-time-degree update walks them: eq bit j of a
// state is bit j + cns_eq_pos of the word eqw, and neg bit D-1 is bit 31 of wn
// with the lower neg bits below it (the bits further down are never shifted
// up to bit 31 within D steps). So neither mask is extracted.
template <int PREC, int D> constexpr int cns_eq_pos() {
    return (PREC == kF16 && D <= 16) ? 16 : (PREC == kFix6 && D <= 22) ? 10 : 0;
}
template <int PREC, int D>
__device__ __forceinline__ void cns_unpack_walk(const uint4 &s, CnsMag<PREC> &m, unsigned &eqw, unsigned &wn) {
    if constexpr (PREC == kF32) {
        m.r1 = __uint_as_float(s.x);
        m.r2 = __uint_as_float(s.y);
        eqw = s.z;
        wn = s.w << (32 - D);
    } else if constexpr (PREC == kF16) {
        m.from_bits(s.x);
        eqw = s.y;
        if constexpr (D <= 16) wn = s.y << (32 - D);  // neg in bits 0..15, eq above
        else wn = s.z << (32 - D);
    } else {
        if constexpr (D <= 22) {
            m.q1 = (int)(s.x & 31u);
            m.q2 = (int)((s.x >> 5) & 31u);
            eqw = s.x;
            if constexpr (D <= 11) wn = s.x << (11 - D);  // neg in bits 21..31
            else wn = s.y << (32 - D);
        } else {
            m.q1 = (int)(s.x & 0xFFu);
            m.q2 = (int)((s.x >> 8) & 0xFFu);
            eqw = s.y;
            wn = s.z << (32 - D);
        }
        m.values();
    }
}
// Pack with the new eq mask already at bit j + cns_eq_pos.
template <int PREC, int D>
__device__ __forceinline__ uint4 cns_pack_walk(const CnsMag<PREC> &m, unsigned eqw, unsigned neg) {
    if constexpr (PREC == kF32) {
        return make_uint4(__float_as_uint(m.r1), __float_as_uint(m.r2), eqw, neg);
    } else if constexpr (PREC == kF16) {
        if constexpr (D <= 16) return make_uint4(m.w, eqw | neg, 0u, 0u);
        else return make_uint4(m.w, eqw, neg, 0u);
    } else {
        if constexpr (D <= 11) return make_uint4((unsigned)m.q1 | ((unsigned)m.q2 << 5) | eqw | (neg << 21), 0u, 0u, 0u);
        else if constexpr (D <= 22) return make_uint4((unsigned)m.q1 | ((unsigned)m.q2 << 5) | eqw, neg, 0u, 0u);
        else return make_uint4((unsigned)m.q1 | ((unsigned)m.q2 << 8), eqw, neg, 0u);
    }
}

// Slot load / store of `bytes` (4, 8 or 16; aligned to that size).
__device__ __forceinline__ uint4 cns_load(const unsigned char *p, int bytes) {
    if (bytes == 16) return __ldcg(reinterpret_cast<const uint4 *>(p));
    if (bytes == 8) {
        const uint2 v = __ldcg(reinterpret_cast<const uint2 *>(p));
        return make_uint4(v.x, v.y, 0u, 0u);
    }
    return make_uint4(__ldcg(reinterpret_cast<const unsigned *>(p)), 0u, 0u, 0u);
}
__device__ __forceinline__ void cns_store(unsigned char *p, int bytes, const uint4 &v) {
    if (bytes == 16) __stcg(reinterpret_cast<uint4 *>(p), v);
    else if (bytes == 8) __stcg(reinterpret_cast<uint2 *>(p), make_uint2(v.x, v.y));
    else __stcg(reinterpret_cast<unsigned *>(p), v.x);
}

// Byte offset in the APP array of the variable node of check node z in a
// block with table entry at = {4 (col Z + shift), Z - shift}:
// 4 (col Z + (z + shift) mod Z) = at.x + 4z - (z >= at.y ? 4Z : 0), computed
// on the FMA pipe: f = (z + 1024 - at.y) >> 10 is 1 exactly when z >= at.y
// (both lie in [0, Z], Z <= 384), taken as the high word of a product with
// 2^22; then off = 4z + at.x - 4Z f.
__device__ __forceinline__ int vn_off_fma(const Params &p, const int2 at, int z) {
    const unsigned x = (unsigned)z * p.k_one + (unsigned)(1024 - at.y);
    const unsigned f = __umulhi(x, p.k_two22);
    return (int)((unsigned)z * p.k_four + (unsigned)at.x + f * p.k_neg4z);
}
// The same offset in three instructions, one multiply-add and two ALU
// operations: off = 4z + at.x, less 4Z when z >= at.y.
__device__ __forceinline__ int vn_off_mixed(const Params &p, const int2 at, int z) {
    unsigned off = (unsigned)z * p.k_four + (unsigned)at.x;
    if (z >= at.y) off = off * p.k_one + p.k_neg4z;  // a predicated multiply-add: the FMA pipe
    return (int)off;
}
__device__ __forceinline__ float &app_at(float *app, int off) {
    return *reinterpret_cast<float *>(reinterpret_cast<char *>(app) + off);
}

// Layered min-sum update of check node z of one layer of degree d (D = d
// exactly, or D = 0 with d <= DM at run time): rebuild the old messages from
// the old state, T = APP - R_old, check-node rule, APP = T + R_new, store the
// new state.
//
// Integer work is balanced between the ALU and FMA pipes. Both passes visit
// the edges in descending order (the updates of one row touch distinct APP
// entries, and the two-minimum rule does not depend on the order). In the
// first pass the old neg bits walk down through bit 31 of a word doubled by
// multiply-adds; in the second the sign of the new message is bit 31 of U =
// bits(T) + (sign bit of the product), an addition modulo 2^32 that flips
// exactly bit 31, and one funnel shift appends it to the neg mask.
template <int D, int DM, int PREC, int ZC>
__device__ __forceinline__ void cns_update(const Params &p, int deg, float *app, const int2 *at, int z,
                                           const uint4 &s_old, unsigned char *slot, int sbytes, bool store) {
    constexpr int N = D ? D : DM;
    const int d = D ? D : deg;
    CnsMag<PREC> mo;
    unsigned eqo, nego;
    cns_unpack<PREC>(s_old, d, mo, eqo, nego);
    float T[N];
    int vi[D ? N : 1];
    unsigned wn = d ? nego << (32 - d) : 0u;  // old neg bits walked down through bit 31 (descending edges)
#pragma unroll
    for (int j = N - 1; j >= 0; --j) {
        T[j] = 0.0f;
        if (D || j < d) {
            const int v = vn_off_mixed(p, at[j], z);
            if constexpr (D != 0) vi[j] = v;
            const float m = ((eqo >> j) & 1u) ? mo.r2 : mo.r1;
            const float old = __uint_as_float(__float_as_uint(m) | (wn & 0x80000000u));
            wn *= p.k_two;
            T[j] = __fsub_rn(app_at(app, v), old);
        }
    }
    FastMinSum<N> cn;
    cn.prepare(T, d, p.offset, p.clamp);
    CnsMag<PREC> mn;
    mn.set(cn.v1, cn.v2);
    unsigned eq = 0, neg = 0;
    const unsigned sxs = cn.sx & 0x80000000u;
    const unsigned b1 = __float_as_uint(mn.r1), b2 = __float_as_uint(mn.r2);
#pragma unroll
    for (int j = N - 1; j >= 0; --j) {
        if (D || j < d) {
            const bool e = fabsf(T[j]) == cn.m1;
            const unsigned U = __float_as_uint(T[j]) * p.k_one + sxs;
            neg = __funnelshift_l(U, neg, 1);  // (neg << 1) | (U >> 31)
            if (e) eq |= 1u << j;
            int v;
            if constexpr (D != 0) v = vi[j];
            else v = vn_off_mixed(p, at[j], z);
            app_at(app, v) = __fadd_rn(T[j], __uint_as_float((U & 0x80000000u) | (e ? b2 : b1)));
        }
    }
    if (store) cns_store(slot, sbytes, cns_pack<PREC>(mn, eq, neg, d));
}

// One layer step: prefetch the state of layer r + 2 into s_far, update layer r
// from s_cur, then a block barrier.
template <int DMAX, int PREC, int ZC>
__device__ __forceinline__ void cns_step(const Params &p, const int2 *s_at, const int32_t *s_rp,
                                         const int32_t *s_soff, float *app, unsigned char *st, int z, int t, int r,
                                         bool done, const uint4 &s_cur, uint4 &s_far) {
    const int ZV = ZC ? ZC : p.Z;
    const int b0 = s_rp[r], deg = s_rp[r + 1] - b0;
    int r2 = r + 2, t2 = t;
    while (r2 >= p.rows) {
        r2 -= p.rows;
        ++t2;
    }
    if (t2 == 0) {
        s_far = make_uint4(0u, 0u, 0u, 0u);  // iteration 0 starts from zero messages
    } else if (!done && t2 < p.iters) {
        const int d2 = s_rp[r2 + 1] - s_rp[r2], sb2 = cns_slot_bytes<PREC>(d2);
        s_far = cns_load(st + s_soff[r2] + (size_t)z * sb2, sb2);
    }
    if (!done) {
        const bool store = t + 1 < p.iters;  // the last iteration's state is never read
        const int sb = cns_slot_bytes<PREC>(deg);
        unsigned char *slot = st + s_soff[r] + (size_t)z * sb;
        const int2 *at = s_at + b0;
        switch (deg) {
#define LDPCX_CNS(dd) \
    case dd:          \
        cns_update<dd, dd, PREC, ZC>(p, dd, app, at, z, s_cur, slot, sb, store); \
        break;
            LDPCX_CNS(1) LDPCX_CNS(2) LDPCX_CNS(3) LDPCX_CNS(4)
            LDPCX_CNS(5) LDPCX_CNS(6) LDPCX_CNS(7) LDPCX_CNS(8)
#undef LDPCX_CNS
            default:
                cns_update<0, DMAX, PREC, ZC>(p, deg, app, at, z, s_cur, slot, sb, store);
                break;
        }
    }
    (void)ZV;
    __syncthreads();
}

// Bytes of the check-node state of one codeword (each row's region rounded
// to 16 bytes so that every slot is aligned to its size).
template <int PREC>
__host__ __device__ inline int64_t cns_bytes_per_cw(const int32_t *row_ptr, int rows, int Z) {
    int64_t off = 0;
    for (int r = 0; r < rows; ++r) off += (cns_slot_bytes<PREC>(row_ptr[r + 1] - row_ptr[r]) * (int64_t)Z + 15) / 16 * 16;
    return off;
}

__host__ __device__ inline size_t cns_smem_bytes(const Params &p) {
    return smem_bytes(p, 1) + sizeof(int32_t) * p.rows + sizeof(int2) * p.nnz + 8;
}

// Check-node-state layered min-sum of the G codewords cw_base .. cw_base+G-1
// of p by the whole CTA, the schedule read from the row table. The state of
// codeword cw lives at msg + (cw - msg_cw0) * msg_stride * msg_size
// (msg_cw0 = 0: one slot per codeword of the batch; msg_cw0 = cw_base: one
// slot per codeword of the tile, as in the persistent mixed-batch kernel).
template <int DMAX, int PREC, int ZC = 0>
__device__ __forceinline__ void cns_tile(const Params &p, int64_t cw_base, int64_t msg_cw0, unsigned char *smem) {
    const int ZV = ZC ? ZC : p.Z;
    float *s_app_all = reinterpret_cast<float *>(smem);
    uint32_t *s_vb = reinterpret_cast<uint32_t *>(s_app_all + (size_t)p.G * p.n);
    int32_t *s_rp = reinterpret_cast<int32_t *>(s_vb + p.nnz);
    int *s_flag = reinterpret_cast<int *>(s_rp + p.rows + 1);
    int32_t *s_soff = reinterpret_cast<int32_t *>(s_flag + 2 * p.G);
    int2 *s_at = reinterpret_cast<int2 *>((reinterpret_cast<uintptr_t>(s_soff + p.rows) + 7) & ~(uintptr_t)7);

    load_tables(p, s_vb, s_rp);
    load_channel(p, s_app_all, cw_base);
    __syncthreads();
    if (threadIdx.x == 0) {
        int32_t off = 0;
        for (int r = 0; r < p.rows; ++r) {
            s_soff[r] = off;
            off += (cns_slot_bytes<PREC>(s_rp[r + 1] - s_rp[r]) * ZV + 15) / 16 * 16;
        }
    }
    for (int i = threadIdx.x; i < p.nnz; i += blockDim.x) {
        const uint32_t vb = s_vb[i];
        const int sh = (int)(vb & 0xFFFFu);
        s_at[i] = make_int2(4 * ((int)(vb >> 16) + sh), ZV - sh);
    }
    const int g = threadIdx.x / ZV, z = threadIdx.x - g * ZV;
    const int64_t cw = cw_base + g;
    const bool active = g < p.G && cw < p.B;
    float *app = s_app_all + (size_t)(active ? g : 0) * p.n;
    unsigned char *st =
        reinterpret_cast<unsigned char *>(p.msg) + (active ? cw - msg_cw0 : 0) * p.msg_stride * p.msg_size;
    bool done = !active;
    int iters_run = 0;
    __syncthreads();

    // state ring: the current layer, the next one (loaded a step ago) and the
    // one after (loaded now); unrolled by three so no registers are copied
    uint4 sa = make_uint4(0u, 0u, 0u, 0u), sb = sa, sc = sa;
    int t = 0, r = 0;
    auto advance = [&]() -> bool {
        if (++r < p.rows) return false;
        r = 0;
        if (!done) iters_run = t + 1;
        ++t;
        if (!p.early_stop) return false;
        if (threadIdx.x < p.G) s_flag[threadIdx.x] = 0;
        __syncthreads();
        if (!done && syndrome_bad_vec<1, ZC>(p, s_vb, s_rp, app, z)) s_flag[g] = 1;
        __syncthreads();
        if (!done && s_flag[g] == 0) done = true;
        return __syncthreads_and(done);
    };
    while (t < p.iters) {
        cns_step<DMAX, PREC, ZC>(p, s_at, s_rp, s_soff, app, st, z, t, r, done, sa, sc);
        if (advance() || t >= p.iters) break;
        cns_step<DMAX, PREC, ZC>(p, s_at, s_rp, s_soff, app, st, z, t, r, done, sb, sa);
        if (advance() || t >= p.iters) break;
        cns_step<DMAX, PREC, ZC>(p, s_at, s_rp, s_soff, app, st, z, t, r, done, sc, sb);
        if (advance()) break;
    }
    __syncthreads();
    write_outputs(p, s_app_all, cw_base, iters_run, g, active, z);
}

template <int DMAX, int PREC, int ZC = 0>
__global__ void __launch_bounds__(kMaxThreads, 2) k_layered_cns(const __grid_constant__ Params p) {
    extern __shared__ __align__(16) unsigned char smem[];
    cns_tile<DMAX, PREC, ZC>(p, (int64_t)blockIdx.x * p.G, 0, smem);
}

KernelFn layered_cns_kernel(int dmax, int prec, int Z);

}  // namespace dec
}  // namespace ldpcx
