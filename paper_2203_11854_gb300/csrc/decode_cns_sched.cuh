// Layered min-sum with check-node state on the 5G-shaped base graphs (full or
// truncated to their first rows), with the layer schedule compiled in.
//
// The row degrees of a full base graph depend on its shape alone (the seed
// moves blocks within a row, never changes how many there are): four core
// rows of the systematic degree plus 2, 3, 2, 2 dual-diagonal blocks, then
// extension rows in two runs of equal degree. So one iteration is four steps
// of exact degree followed by two loops of fixed degree, and no step looks up
// a row table or dispatches on a degree. Slot offsets and table offsets
// advance by constants. Everything else -- the update, the state format, the
// prefetch of the state two layers ahead and the early stop -- is that of
// k_layered_cns, so results are the same bit for bit.
//
// A thread may own K = 2 check nodes of each row, z and z + Z/2 (Z even): the
// K updates are interleaved pass by pass (all APP loads, all check-node rules,
// all APP stores), so one warp carries two independent dependency chains and
// the per-row work (schedule, barrier, table reads) is shared. Each access of
// a warp still covers 32 consecutive APP entries, free of bank conflicts.
#pragma once

#include "decode_cns.cuh"

namespace ldpcx {
namespace dec {

template <int BG> struct Sched;
template <> struct Sched<1> {
    static constexpr int rows = 46, dc0 = 18, dc1 = 19, dc2 = 18, dc3 = 18, n_hi = 33, d_hi = 6, d_lo = 5;
};
template <> struct Sched<2> {
    static constexpr int rows = 42, dc0 = 10, dc1 = 11, dc2 = 10, dc3 = 10, n_hi = 4, d_hi = 5, d_lo = 4;
};

template <int BG, int PREC> struct SchedLayout {
    using S = Sched<BG>;
    static constexpr int sb_core = cns_slot_bytes<PREC>(S::dc1);  // slot bytes of the core rows
    static constexpr int sb_ext = cns_slot_bytes<PREC>(S::d_hi);  // and of the extension rows
    // BG1-shaped codes with FP16 or 6-bit messages (one check node per thread) keep per-edge messages
    // for the extension rows (degree 6 and 5): a node's messages in two planes of the row's region,
    // messages 0..3 in plane A, 4 and 5 in plane B; binary16 takes 8 + 4 B per node, 6-bit one byte
    // per message, 4 + 2 B. Rebuilding a message is then a conversion (FP16) or a byte permute and a
    // subtraction (6-bit) instead of a select on two masks; the core rows (degree 18 and 19) keep the
    // check-node state.
    static constexpr bool edge_ext = BG == 1 && (PREC == kF16 || PREC == kFix6);
    static constexpr int edge_a = PREC == kFix6 ? 4 : 8;     // plane A bytes per node
    static constexpr int edge_row = PREC == kFix6 ? 6 : 12;  // bytes per node of an extension row
    static constexpr int b_hi = S::dc0 + S::dc1 + S::dc2 + S::dc3;  // first block of the extension rows
    static constexpr int b_lo = b_hi + S::n_hi * S::d_hi;
    static_assert(cns_slot_bytes<PREC>(S::dc0) == sb_core && cns_slot_bytes<PREC>(S::dc2) == sb_core &&
                      cns_slot_bytes<PREC>(S::dc3) == sb_core && cns_slot_bytes<PREC>(S::d_lo) == sb_ext,
                  "one slot size per run of rows");
};

// Block table of the schedule, passed by value as a kernel parameter so that
// every lookup is a warp-uniform constant-bank read: entry b = {4 (col Z +
// shift), Z - shift} of block b in row-major order.
constexpr int kSchedMaxBlocks = 316;
struct SchedTab {
    int2 at[kSchedMaxBlocks];
};

// The three state registers of the ring by step phase (K slots each).
template <int Ph, int K>
__device__ __forceinline__ uint4 (&ring(uint4 (&a)[K], uint4 (&b)[K], uint4 (&c)[K]))[K] {
    if constexpr (Ph % 3 == 0) return a;
    else if constexpr (Ph % 3 == 1) return b;
    else return c;
}

// Geometry of one codeword's state: region bytes of a core and of an extension
// row, and (one check node per thread) the thread's slot in core row 0 and in
// extension row 0 (with per-edge extension rows: its plane A slot; its plane B
// slot lies a per-thread distance further on).
struct SchedGeo {
    int Lc, Le;
    unsigned char *core_z, *ext_z;
    __device__ __forceinline__ int off(int r) const { return r < 4 ? r * Lc : 4 * Lc + (r - 4) * Le; }
};

// Bytes of one codeword's state under the compiled schedule (each row region
// rounded to 16 B): check-node state for every row, or, for BG1-shaped codes
// with FP16 or 6-bit messages and one check node per thread, the state of the
// four core rows followed by 12 B (FP16) or 6 B (6-bit) of per-edge messages
// per node of each extension row.
__host__ inline int64_t sched_state_bytes(int bg, int prec, int kpt, const int32_t *row_ptr, int rows, int Z) {
    if (bg == 1 && (prec == kF16 || prec == kFix6) && kpt == 1) {
        const int64_t ext = prec == kFix6 ? 6 : 12;
        int64_t b = 0;
        for (int r = 0; r < rows; ++r) {
            const int d = row_ptr[r + 1] - row_ptr[r];
            const int core = prec == kFix6 ? cns_slot_bytes<kFix6>(d) : cns_slot_bytes<kF16>(d);
            b += r < 4 ? (core * (int64_t)Z + 15) / 16 * 16 : (ext * Z + 15) / 16 * 16;
        }
        return b;
    }
    if (prec == kF32) return cns_bytes_per_cw<kF32>(row_ptr, rows, Z);
    if (prec == kF16) return cns_bytes_per_cw<kF16>(row_ptr, rows, Z);
    return cns_bytes_per_cw<kFix6>(row_ptr, rows, Z);
}

// Per-edge extension rows: a node's messages (plane A: messages 0..3, plane B: 4, 5).
template <int PREC>
__device__ __forceinline__ uint4 edge_ext_load(const unsigned char *a, const unsigned char *b) {
    if constexpr (PREC == kFix6) {
        return make_uint4(__ldcg(reinterpret_cast<const unsigned *>(a)),
                          (unsigned)__ldcg(reinterpret_cast<const unsigned short *>(b)), 0u, 0u);
    } else {
        const uint2 va = __ldcg(reinterpret_cast<const uint2 *>(a));
        return make_uint4(va.x, va.y, __ldcg(reinterpret_cast<const unsigned *>(b)), 0u);
    }
}

// A 6-bit message R (a multiple of 0.5 in [-15.5, 15.5]) is stored as the byte
// 32 + 2R: that byte under the upper bytes of 1.5 * 2^22 (0x4AC00000, whose
// mantissa step is 0.5) reads as 1.5 * 2^22 + 16 + R exactly, so one byte
// permute and one subtraction rebuild R, and one addition gives the byte back.
// A zero message is the byte 32, so the first iteration starts from bytes of
// 32, not from zero bytes; it is stored as +0 (the 6-bit store has no -0, as in
// the check-node state; the sums are the same).
constexpr float kFix6Bias = 6291472.0f;  // 1.5 * 2^22 + 16
__device__ __forceinline__ float fix6_byte_value(unsigned w, unsigned j) {
    return __fsub_rn(__uint_as_float(__byte_perm(w, 0x4AC00000u, 0x7650u | j)), kFix6Bias);
}
__device__ __forceinline__ unsigned fix6_byte_of(float r) { return __float_as_uint(__fadd_rn(r, kFix6Bias)); }
__device__ __forceinline__ float half_lo(unsigned w) { return __low2float(*reinterpret_cast<const __half2 *>(&w)); }
__device__ __forceinline__ float half_hi(unsigned w) { return __high2float(*reinterpret_cast<const __half2 *>(&w)); }
__device__ __forceinline__ unsigned half_pack(float a, float b) {
    const __half2 h = __floats2half2_rn(a, b);  // exact: a and b are binary16 values
    return *reinterpret_cast<const unsigned *>(&h);
}

// Layered min-sum update of check node z of an extension row of degree D with
// per-edge FP16 or 6-bit messages: the rule of cns_update_k, the old messages
// read from the packed halves (bytes) and the new rounded ones packed back, so
// the stored values, and every APP, are the same bit for bit.
template <int D, int PREC>
__device__ __forceinline__ void edge_ext_update(const Params &p, float *app, const int2 *at, int z,
                                                const uint4 &s_old, unsigned char *slot_a, unsigned char *slot_b,
                                                bool store) {
    static_assert(D >= 5 && D <= 6, "two planes hold five or six messages");
    const unsigned w[3] = {s_old.x, s_old.y, s_old.z};
    float T[D];
    int vi[D];
#pragma unroll
    for (int j = D - 1; j >= 0; --j) {
        vi[j] = vn_off_mixed(p, at[j], z);
        const float old = PREC == kFix6 ? fix6_byte_value(w[j >> 2], (unsigned)(j & 3))
                          : (j & 1)     ? half_hi(w[j >> 1])
                                        : half_lo(w[j >> 1]);
        T[j] = __fsub_rn(app_at(app, vi[j]), old);
    }
    FastMinSum<D> cn;
    cn.prepare(T, D, p.offset, p.clamp);
    CnsMag<PREC> mn;
    mn.set(cn.v1, cn.v2);
    const unsigned sxs = cn.sx & 0x80000000u;
    const unsigned b1 = __float_as_uint(mn.r1), b2 = __float_as_uint(mn.r2);
    float R[D];
#pragma unroll
    for (int j = D - 1; j >= 0; --j) {
        const bool e = fabsf(T[j]) == cn.m1;
        // sign of the new message: bit 31 of U = bits(T) + the product's sign bit (a flip of bit 31)
        const unsigned U = __float_as_uint(T[j]) * p.k_one + sxs;
        R[j] = __uint_as_float((U & 0x80000000u) | (e ? b2 : b1));
        app_at(app, vi[j]) = __fadd_rn(T[j], R[j]);
    }
    if (store) {
        if constexpr (PREC == kFix6) {
            unsigned f[6];
#pragma unroll
            for (int j = 0; j < D; ++j) f[j] = fix6_byte_of(R[j]);
            if constexpr (D == 5) f[5] = 32u;  // a zero message in the unused slot
            const unsigned a = __byte_perm(__byte_perm(f[0], f[1], 0x0040u), __byte_perm(f[2], f[3], 0x0040u),
                                           0x5410u);
            __stcg(reinterpret_cast<unsigned *>(slot_a), a);
            __stcg(reinterpret_cast<unsigned short *>(slot_b), (unsigned short)__byte_perm(f[4], f[5], 0x0040u));
        } else {
            __stcg(reinterpret_cast<uint2 *>(slot_a), make_uint2(half_pack(R[0], R[1]), half_pack(R[2], R[3])));
            __stcg(reinterpret_cast<unsigned *>(slot_b), half_pack(R[4], D > 5 ? R[D - 1] : 0.0f));
        }
    }
}

// Layered min-sum update of the K check nodes zk[0..K) of a row of exact
// degree D (the rule of cns_update, pass by pass over the K nodes). The state
// slot of node k is row + zk[k] * slot bytes, or row itself when K = 1.
template <int D, int PREC, int K>
__device__ __forceinline__ void cns_update_k(const Params &p, float *app, const int2 *at, const int (&zk)[K],
                                             const uint4 (&s_old)[K], unsigned char *row, bool store) {
    constexpr int SB = cns_slot_bytes<PREC>(D);
    constexpr int EP = cns_eq_pos<PREC, D>();
    CnsMag<PREC> mo[K];
    // the old neg bits walked down through bit 31 of wn (edges in descending order: the row's updates
    // touch distinct APP entries, and the two-minimum rule does not depend on the order)
    unsigned eqo[K], wn[K];
#pragma unroll
    for (int k = 0; k < K; ++k) cns_unpack_walk<PREC, D>(s_old[k], mo[k], eqo[k], wn[k]);
    float T[K][D];
    int vi[K][D];
#pragma unroll
    for (int j = D - 1; j >= 0; --j) {
        const int2 a = at[j];
#pragma unroll
        for (int k = 0; k < K; ++k) {
            vi[k][j] = vn_off_mixed(p, a, zk[k]);
            const float m = ((eqo[k] >> (j + EP)) & 1u) ? mo[k].r2 : mo[k].r1;
            const float old = __uint_as_float(__float_as_uint(m) | (wn[k] & 0x80000000u));
            wn[k] *= p.k_two;
            T[k][j] = __fsub_rn(app_at(app, vi[k][j]), old);
        }
    }
    FastMinSum<D> cn[K];
    CnsMag<PREC> mn[K];
    unsigned eq[K], neg[K], sxs[K], b1[K], b2[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        cn[k].prepare(T[k], D, p.offset, p.clamp);
        mn[k].set(cn[k].v1, cn[k].v2);
        eq[k] = 0;
        neg[k] = 0;
        sxs[k] = cn[k].sx & 0x80000000u;
        b1[k] = __float_as_uint(mn[k].r1);
        b2[k] = __float_as_uint(mn[k].r2);
    }
#pragma unroll
    for (int j = D - 1; j >= 0; --j) {
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const bool e = fabsf(T[k][j]) == cn[k].m1;
            // sign of the new message: bit 31 of U = bits(T) + the product's sign bit (a flip of bit 31)
            const unsigned U = __float_as_uint(T[k][j]) * p.k_one + sxs[k];
            neg[k] = __funnelshift_l(U, neg[k], 1);  // (neg << 1) | (U >> 31)
            eq[k] |= e ? (1u << (j + EP)) : 0u;
            app_at(app, vi[k][j]) = __fadd_rn(T[k][j], __uint_as_float((U & 0x80000000u) | (e ? b2[k] : b1[k])));
        }
    }
    if (store) {
#pragma unroll
        for (int k = 0; k < K; ++k)
            cns_store(K == 1 ? row : row + zk[k] * SB, SB, cns_pack_walk<PREC, D>(mn[k], eq[k], neg[k]));
    }
}

// Where a step's row and the row it prefetches lie, when that is known at
// compile time (full base graphs): core row 0..3, an extension row whose row
// r + 2 is in the same iteration, or one of the last two rows, whose r + 2 is
// row 0 or 1 of the next iteration. kStepAny decides at run time (truncated
// codes, whose row count is a parameter).
constexpr int kStepExt = 4, kStepExtWrap = 5, kStepAny = 6;

// The row two layers on from row r of iteration t (its state is prefetched
// into the ring), its iteration, and whether it is a core row: known at
// compile time for full base graphs (MODE), at run time for truncated ones.
template <int BG, bool TRUNC, int MODE>
__device__ __forceinline__ void sched_far(const Params &p, int t, int r, int &r2, int &t2, bool &core2) {
    static_assert(MODE == kStepAny || !TRUNC, "truncated codes place their rows at run time");
    const int rows = TRUNC ? p.rows : Sched<BG>::rows;
    if constexpr (MODE == kStepAny) {
        const bool wrap = r + 2 >= rows;  // the state two layers on is the next iteration's
        r2 = wrap ? r + 2 - rows : r + 2;
        t2 = wrap ? t + 1 : t;
        core2 = r2 < 4;
    } else if constexpr (MODE == kStepExtWrap) {
        r2 = r + 2 - rows;
        t2 = t + 1;
        core2 = true;
    } else {
        r2 = r + 2;
        t2 = t;
        core2 = MODE < 2;
    }
}

// One layer step of degree D on row r (blocks from b0, the row's state region
// at st + off) for K >= 2 check nodes per thread: prefetch the state of layer
// r + 2 into s_far, update from s_cur, barrier.
template <int D, int BG, int PREC, int K, bool TRUNC, int MODE>
__device__ __forceinline__ void sched_step(const Params &p, const int2 *s_at, float *app, unsigned char *st,
                                           const int (&zk)[K], int t, int r, int b0, int off, const SchedGeo &geo,
                                           bool done, const uint4 (&s_cur)[K], uint4 (&s_far)[K]) {
    using L = SchedLayout<BG, PREC>;
    int r2, t2;
    bool core2;
    sched_far<BG, TRUNC, MODE>(p, t, r, r2, t2, core2);
    // t2 == 0 only without a wrap, and t2 < p.iters holds without one (t < p.iters)
    const bool zero = MODE == kStepExtWrap ? false : t2 == 0;
    const bool fetch = MODE == kStepAny ? t2 < p.iters : MODE == kStepExtWrap ? t + 1 < p.iters : true;
    if (zero) {
#pragma unroll
        for (int k = 0; k < K; ++k) s_far[k] = make_uint4(0u, 0u, 0u, 0u);  // iteration 0: zero messages
    } else if (!done && fetch) {
        const unsigned char *row2 = st + geo.off(r2);
#pragma unroll
        for (int k = 0; k < K; ++k) {
            if (core2) s_far[k] = cns_load(row2 + zk[k] * L::sb_core, L::sb_core);
            else s_far[k] = cns_load(row2 + zk[k] * L::sb_ext, L::sb_ext);
        }
    }
    if (!done) cns_update_k<D, PREC, K>(p, app, s_at + b0, zk, s_cur, st + off, t + 1 < p.iters);
    __syncthreads();
}

// COUNT consecutive rows of degree D from row r0, the first at ring phase PH
// (= r0 for full graphs). LAST: the run ends the iteration of a full graph, so
// its last two steps prefetch the next iteration's rows 0 and 1.
template <int D, int COUNT, int PH, int BG, int PREC, int K, bool TRUNC = false, bool LAST = false>
__device__ __forceinline__ void sched_run(const Params &p, const int2 *s_at, float *app, unsigned char *st,
                                          const int (&zk)[K], int t, int r0, int b0, int off0, int Lrow,
                                          const SchedGeo &geo, bool done, uint4 (&a)[K], uint4 (&b)[K],
                                          uint4 (&c)[K]) {
    constexpr int M = TRUNC ? kStepAny : PH < 4 ? PH : kStepExt;
    constexpr int NW = LAST ? COUNT - 2 : COUNT;  // steps without a wrap
    static_assert(!LAST || (COUNT >= 2 && !TRUNC && PH >= 4), "the last run is an extension run of a full graph");
    int r = r0, bb = b0, off = off0;
#pragma unroll 1
    for (int i = 0; i < NW / 3; ++i) {
        sched_step<D, BG, PREC, K, TRUNC, M>(p, s_at, app, st, zk, t, r, bb, off, geo, done, ring<PH, K>(a, b, c),
                                             ring<PH + 2, K>(a, b, c));
        sched_step<D, BG, PREC, K, TRUNC, M>(p, s_at, app, st, zk, t, r + 1, bb + D, off + Lrow, geo, done,
                                             ring<PH + 1, K>(a, b, c), ring<PH + 3, K>(a, b, c));
        sched_step<D, BG, PREC, K, TRUNC, M>(p, s_at, app, st, zk, t, r + 2, bb + 2 * D, off + 2 * Lrow, geo, done,
                                             ring<PH + 2, K>(a, b, c), ring<PH + 4, K>(a, b, c));
        r += 3;
        bb += 3 * D;
        off += 3 * Lrow;
    }
    if constexpr (NW % 3 >= 1)
        sched_step<D, BG, PREC, K, TRUNC, M>(p, s_at, app, st, zk, t, r, bb, off, geo, done, ring<PH, K>(a, b, c),
                                             ring<PH + 2, K>(a, b, c));
    if constexpr (NW % 3 == 2)
        sched_step<D, BG, PREC, K, TRUNC, M>(p, s_at, app, st, zk, t, r + 1, bb + D, off + Lrow, geo, done,
                                             ring<PH + 1, K>(a, b, c), ring<PH + 3, K>(a, b, c));
    if constexpr (LAST) {
        constexpr int Q = PH + NW;  // ring phase of the first wrapping step
        r += NW % 3;
        bb += (NW % 3) * D;
        off += (NW % 3) * Lrow;
        sched_step<D, BG, PREC, K, TRUNC, kStepExtWrap>(p, s_at, app, st, zk, t, r, bb, off, geo, done,
                                                        ring<Q, K>(a, b, c), ring<Q + 2, K>(a, b, c));
        sched_step<D, BG, PREC, K, TRUNC, kStepExtWrap>(p, s_at, app, st, zk, t, r + 1, bb + D, off + Lrow, geo,
                                                        done, ring<Q + 1, K>(a, b, c), ring<Q + 3, K>(a, b, c));
    }
}

// `count` (run-time) consecutive rows of degree D from row r0, starting at
// ring phase 0; the ring is rotated afterwards so that the next run starts at
// phase 0 again.
template <int D, int BG, int PREC, int K>
__device__ __forceinline__ void sched_run_n(const Params &p, const int2 *s_at, float *app, unsigned char *st,
                                            const int (&zk)[K], int t, int r0, int b0, int off0, int Lrow,
                                            int count, const SchedGeo &geo, bool done, uint4 (&a)[K],
                                            uint4 (&b)[K], uint4 (&c)[K]) {
    int r = r0, bb = b0, off = off0;
#pragma unroll 1
    for (int i = 0; i < count / 3; ++i) {
        sched_step<D, BG, PREC, K, true, kStepAny>(p, s_at, app, st, zk, t, r, bb, off, geo, done, a, c);
        sched_step<D, BG, PREC, K, true, kStepAny>(p, s_at, app, st, zk, t, r + 1, bb + D, off + Lrow, geo, done, b, a);
        sched_step<D, BG, PREC, K, true, kStepAny>(p, s_at, app, st, zk, t, r + 2, bb + 2 * D, off + 2 * Lrow, geo, done, c, b);
        r += 3;
        bb += 3 * D;
        off += 3 * Lrow;
    }
    const int rem = count - 3 * (count / 3);
    if (rem >= 1) sched_step<D, BG, PREC, K, true, kStepAny>(p, s_at, app, st, zk, t, r, bb, off, geo, done, a, c);
    if (rem == 2) sched_step<D, BG, PREC, K, true, kStepAny>(p, s_at, app, st, zk, t, r + 1, bb + D, off + Lrow, geo, done, b, a);
    if (rem == 1) {
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const uint4 x = a[k];
            a[k] = b[k];
            b[k] = c[k];
            c[k] = x;
        }
    } else if (rem == 2) {
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const uint4 x = c[k];
            c[k] = b[k];
            b[k] = a[k];
            a[k] = x;
        }
    }
}

// K >= 2 check nodes per thread: G codewords per CTA of G Z / K threads. The code
// is the full base graph of shape BG or a truncation of it to its first p.rows
// rows (the extension rows in order), so the runs have run-time lengths.
// The codewords cw_base .. cw_base+G-1 of p by the whole CTA; block table
// s_at (constant bank or shared memory); the state of codeword cw at msg +
// (cw - msg_cw0) * msg_stride * msg_size.
template <int BG, int PREC, int ZC, int K, bool TRUNC>
__device__ __forceinline__ void cns_sched_tile(const Params &p, int64_t cw_base, int64_t msg_cw0,
                                               unsigned char *smem, const int2 *s_at) {
    static_assert(K >= 2, "one check node per thread runs cns_sched_tile1");
    using S = Sched<BG>;
    using L = SchedLayout<BG, PREC>;
    const int ZV = ZC ? ZC : p.Z;
    const int H = ZV / K;  // threads per codeword
    float *s_app_all = reinterpret_cast<float *>(smem);
    uint32_t *s_vb = reinterpret_cast<uint32_t *>(s_app_all + (size_t)p.G * p.n);
    int32_t *s_rp = reinterpret_cast<int32_t *>(s_vb + p.nnz);
    int *s_flag = reinterpret_cast<int *>(s_rp + p.rows + 1);

    load_tables(p, s_vb, s_rp);  // for the syndrome check
    load_channel(p, s_app_all, cw_base);
    const int g = threadIdx.x / H, z = threadIdx.x - g * H;
    int zk[K];
#pragma unroll
    for (int k = 0; k < K; ++k) zk[k] = z + k * H;
    const int64_t cw = cw_base + g;
    const bool active = g < p.G && cw < p.B;
    float *app = s_app_all + (size_t)(active ? g : 0) * p.n;
    unsigned char *st =
        reinterpret_cast<unsigned char *>(p.msg) + (active ? cw - msg_cw0 : 0) * p.msg_stride * p.msg_size;
    bool done = !active;
    int iters_run = 0;
    SchedGeo geo;
    geo.Lc = (L::sb_core * ZV + 15) / 16 * 16;
    geo.Le = (L::sb_ext * ZV + 15) / 16 * 16;
    geo.core_z = st + zk[0] * L::sb_core;
    geo.ext_z = st + 4 * geo.Lc + zk[0] * L::sb_ext;
    __syncthreads();

    const int n_hi = min(S::n_hi, p.rows - 4), n_lo = p.rows - 4 - n_hi;
    uint4 a[K], b[K], c[K];
#pragma unroll
    for (int k = 0; k < K; ++k) a[k] = b[k] = c[k] = make_uint4(0u, 0u, 0u, 0u);
    for (int t = 0; t < p.iters; ++t) {
        sched_run<S::dc0, 1, 0, BG, PREC, K, TRUNC>(p, s_at, app, st, zk, t, 0, 0, 0, geo.Lc, geo, done, a, b, c);
        sched_run<S::dc1, 1, 1, BG, PREC, K, TRUNC>(p, s_at, app, st, zk, t, 1, S::dc0, geo.Lc, geo.Lc, geo, done,
                                                    a, b, c);
        sched_run<S::dc2, 1, 2, BG, PREC, K, TRUNC>(p, s_at, app, st, zk, t, 2, S::dc0 + S::dc1, 2 * geo.Lc, geo.Lc,
                                                    geo, done, a, b, c);
        sched_run<S::dc3, 1, 3, BG, PREC, K, TRUNC>(p, s_at, app, st, zk, t, 3, S::dc0 + S::dc1 + S::dc2,
                                                    3 * geo.Lc, geo.Lc, geo, done, a, b, c);
        if constexpr (!TRUNC) {
            // the full graph: run lengths known here, phases follow on
            sched_run<S::d_hi, S::n_hi, 4, BG, PREC, K>(p, s_at, app, st, zk, t, 4, L::b_hi, 4 * geo.Lc, geo.Le,
                                                        geo, done, a, b, c);
            sched_run<S::d_lo, S::rows - 4 - S::n_hi, 4 + S::n_hi, BG, PREC, K, false, true>(
                p, s_at, app, st, zk, t, 4 + S::n_hi, L::b_lo, 4 * geo.Lc + S::n_hi * geo.Le, geo.Le, geo, done, a,
                b, c);
            // the next iteration's first step finds its state at phase rows mod 3
#pragma unroll
            for (int k = 0; k < K; ++k) {
                if constexpr (S::rows % 3 == 1) {
                    const uint4 x = a[k];
                    a[k] = b[k];
                    b[k] = c[k];
                    c[k] = x;
                } else if constexpr (S::rows % 3 == 2) {
                    const uint4 x = c[k];
                    c[k] = b[k];
                    b[k] = a[k];
                    a[k] = x;
                }
            }
        } else {
            // a truncation: four core steps end at phase 1; rotate so that each run starts at phase 0
#pragma unroll
            for (int k = 0; k < K; ++k) {
                const uint4 x = a[k];
                a[k] = b[k];
                b[k] = c[k];
                c[k] = x;
            }
            sched_run_n<S::d_hi, BG, PREC, K>(p, s_at, app, st, zk, t, 4, L::b_hi, 4 * geo.Lc, geo.Le, n_hi, geo,
                                              done, a, b, c);
            sched_run_n<S::d_lo, BG, PREC, K>(p, s_at, app, st, zk, t, 4 + S::n_hi, L::b_lo,
                                              4 * geo.Lc + S::n_hi * geo.Le, geo.Le, n_lo, geo, done, a, b, c);
        }
        if (!done) iters_run = t + 1;
        if (p.early_stop) {
            if (threadIdx.x < p.G) s_flag[threadIdx.x] = 0;
            __syncthreads();
            bool bad = false;
#pragma unroll
            for (int k = 0; k < K; ++k) bad |= !done && syndrome_bad_vec<1, ZC>(p, s_vb, s_rp, app, zk[k]);
            if (bad) s_flag[g] = 1;
            __syncthreads();
            if (!done && s_flag[g] == 0) done = true;
            if (__syncthreads_and(done)) break;
        }
    }
    __syncthreads();
    write_outputs(p, s_app_all, cw_base, iters_run, g, active, z);
}

// ---------------------------------------------------------------------------
// One check node per thread (K = 1): the same schedule, update and prefetch
// with scalar registers throughout and the slot addresses formed from two
// per-thread bases (core and extension rows), so a step adds one row offset.
// BG1-shaped codes with FP16 or 6-bit messages keep the extension rows per
// edge (SchedLayout::edge_ext); plane B of a node lies a Z - (2a - e) z bytes
// past its plane A (a = plane A bytes per node, e = bytes per node; 8 Z - 4 z
// for FP16), an offset formed where it is used (a register held across the
// whole kernel costs more than the multiply-add).

// Layered min-sum update of check node z of a row of exact degree D from its
// check-node state (the rule of cns_update_k for one node).
template <int D, int PREC>
__device__ __forceinline__ void cns_update1(const Params &p, float *app, const int2 *at, int z, const uint4 &s_old,
                                            unsigned char *slot, bool store) {
    constexpr int EP = cns_eq_pos<PREC, D>();
    CnsMag<PREC> mo;
    unsigned eqo, wn;  // the old eq word, and the old neg bits walked down through bit 31 (descending edges)
    cns_unpack_walk<PREC, D>(s_old, mo, eqo, wn);
    float T[D];
    int vi[D];
#pragma unroll
    for (int j = D - 1; j >= 0; --j) {
        vi[j] = vn_off_mixed(p, at[j], z);
        const float m = ((eqo >> (j + EP)) & 1u) ? mo.r2 : mo.r1;
        const float old = __uint_as_float(__float_as_uint(m) | (wn & 0x80000000u));
        wn *= p.k_two;
        T[j] = __fsub_rn(app_at(app, vi[j]), old);
    }
    FastMinSum<D> cn;
    cn.prepare(T, D, p.offset, p.clamp);
    CnsMag<PREC> mn;
    mn.set(cn.v1, cn.v2);
    unsigned eq = 0, neg = 0;
    const unsigned sxs = cn.sx & 0x80000000u;
    const unsigned b1 = __float_as_uint(mn.r1), b2 = __float_as_uint(mn.r2);
#pragma unroll
    for (int j = D - 1; j >= 0; --j) {
        const bool e = fabsf(T[j]) == cn.m1;
        const unsigned U = __float_as_uint(T[j]) * p.k_one + sxs;
        neg = __funnelshift_l(U, neg, 1);  // (neg << 1) | (U >> 31)
        eq |= e ? (1u << (j + EP)) : 0u;
        app_at(app, vi[j]) = __fadd_rn(T[j], __uint_as_float((U & 0x80000000u) | (e ? b2 : b1)));
    }
    if (store) cns_store(slot, cns_slot_bytes<PREC>(D), cns_pack_walk<PREC, D>(mn, eq, neg));
}

// One layer step of degree D on row r with one check node per thread.
template <int D, int BG, int PREC, int ZC, bool TRUNC, int MODE>
__device__ __forceinline__ void sched_step1(const Params &p, const int2 *s_at, float *app, int z, int t, int r,
                                            int b0, int off, const SchedGeo &geo, bool done, const uint4 &s_cur,
                                            uint4 &s_far) {
    using L = SchedLayout<BG, PREC>;
    // plane B past plane A (per-edge extension rows): the rest of plane A, then this node's plane B slot
    const int pb = L::edge_a * (ZC ? ZC : p.Z) - (2 * L::edge_a - L::edge_row) * z;
    // an extension row: the core rows of both shapes have degree 10 or more, the extension rows 6 or less
    constexpr bool ext_row = D <= 8;
    int r2, t2;
    bool core2;
    sched_far<BG, TRUNC, MODE>(p, t, r, r2, t2, core2);
    const bool zero = MODE == kStepExtWrap ? false : t2 == 0;
    const bool fetch = MODE == kStepAny ? t2 < p.iters : MODE == kStepExtWrap ? t + 1 < p.iters : true;
    if (zero) {
        // iteration 0: zero messages (all-zero words, except per-edge 6-bit rows: bytes of 32)
        if constexpr (L::edge_ext && PREC == kFix6)
            s_far = core2 ? make_uint4(0u, 0u, 0u, 0u) : make_uint4(0x20202020u, 0x2020u, 0u, 0u);
        else
            s_far = make_uint4(0u, 0u, 0u, 0u);
    } else if (!done && fetch) {
        if (core2) {
            s_far = cns_load(geo.core_z + r2 * geo.Lc, L::sb_core);
        } else {
            const unsigned char *a = geo.ext_z + (r2 - 4) * geo.Le;
            if constexpr (L::edge_ext) s_far = edge_ext_load<PREC>(a, a + pb);
            else s_far = cns_load(a, L::sb_ext);
        }
    }
    if (!done) {
        if constexpr (L::edge_ext && ext_row) {
            unsigned char *slot = geo.ext_z - 4 * geo.Lc + off;
            edge_ext_update<D, PREC>(p, app, s_at + b0, z, s_cur, slot, slot + pb, t + 1 < p.iters);
        } else {
            unsigned char *slot = (ext_row ? geo.ext_z - 4 * geo.Lc : geo.core_z) + off;
            cns_update1<D, PREC>(p, app, s_at + b0, z, s_cur, slot, t + 1 < p.iters);
        }
    }
    __syncthreads();
}

template <int Ph>
__device__ __forceinline__ uint4 &ring1(uint4 &a, uint4 &b, uint4 &c) {
    if constexpr (Ph % 3 == 0) return a;
    else if constexpr (Ph % 3 == 1) return b;
    else return c;
}

// COUNT consecutive rows of degree D from row r0 at ring phase PH (as sched_run).
template <int D, int COUNT, int PH, int BG, int PREC, int ZC, bool TRUNC = false, bool LAST = false>
__device__ __forceinline__ void sched_run1(const Params &p, const int2 *s_at, float *app, int z, int t, int r0,
                                           int b0, int off0, int Lrow, const SchedGeo &geo, bool done, uint4 &a,
                                           uint4 &b, uint4 &c) {
    constexpr int M = TRUNC ? kStepAny : PH < 4 ? PH : kStepExt;
    constexpr int NW = LAST ? COUNT - 2 : COUNT;  // steps without a wrap
    static_assert(!LAST || (COUNT >= 2 && !TRUNC && PH >= 4), "the last run is an extension run of a full graph");
    int r = r0, bb = b0, off = off0;
#pragma unroll 1
    for (int i = 0; i < NW / 3; ++i) {
        sched_step1<D, BG, PREC, ZC, TRUNC, M>(p, s_at, app, z, t, r, bb, off, geo, done, ring1<PH>(a, b, c),
                                           ring1<PH + 2>(a, b, c));
        sched_step1<D, BG, PREC, ZC, TRUNC, M>(p, s_at, app, z, t, r + 1, bb + D, off + Lrow, geo, done,
                                           ring1<PH + 1>(a, b, c), ring1<PH + 3>(a, b, c));
        sched_step1<D, BG, PREC, ZC, TRUNC, M>(p, s_at, app, z, t, r + 2, bb + 2 * D, off + 2 * Lrow, geo, done,
                                           ring1<PH + 2>(a, b, c), ring1<PH + 4>(a, b, c));
        r += 3;
        bb += 3 * D;
        off += 3 * Lrow;
    }
    if constexpr (NW % 3 >= 1)
        sched_step1<D, BG, PREC, ZC, TRUNC, M>(p, s_at, app, z, t, r, bb, off, geo, done, ring1<PH>(a, b, c),
                                           ring1<PH + 2>(a, b, c));
    if constexpr (NW % 3 == 2)
        sched_step1<D, BG, PREC, ZC, TRUNC, M>(p, s_at, app, z, t, r + 1, bb + D, off + Lrow, geo, done,
                                           ring1<PH + 1>(a, b, c), ring1<PH + 3>(a, b, c));
    if constexpr (LAST) {
        constexpr int Q = PH + NW;  // ring phase of the first wrapping step
        r += NW % 3;
        bb += (NW % 3) * D;
        off += (NW % 3) * Lrow;
        sched_step1<D, BG, PREC, ZC, TRUNC, kStepExtWrap>(p, s_at, app, z, t, r, bb, off, geo, done,
                                                      ring1<Q>(a, b, c), ring1<Q + 2>(a, b, c));
        sched_step1<D, BG, PREC, ZC, TRUNC, kStepExtWrap>(p, s_at, app, z, t, r + 1, bb + D, off + Lrow, geo, done,
                                                      ring1<Q + 1>(a, b, c), ring1<Q + 3>(a, b, c));
    }
}

// `count` (run-time) consecutive rows of degree D of a truncated graph (as sched_run_n).
template <int D, int BG, int PREC, int ZC>
__device__ __forceinline__ void sched_run_n1(const Params &p, const int2 *s_at, float *app, int z, int t, int r0,
                                             int b0, int off0, int Lrow, int count, const SchedGeo &geo, bool done,
                                             uint4 &a, uint4 &b, uint4 &c) {
    int r = r0, bb = b0, off = off0;
#pragma unroll 1
    for (int i = 0; i < count / 3; ++i) {
        sched_step1<D, BG, PREC, ZC, true, kStepAny>(p, s_at, app, z, t, r, bb, off, geo, done, a, c);
        sched_step1<D, BG, PREC, ZC, true, kStepAny>(p, s_at, app, z, t, r + 1, bb + D, off + Lrow, geo, done, b, a);
        sched_step1<D, BG, PREC, ZC, true, kStepAny>(p, s_at, app, z, t, r + 2, bb + 2 * D, off + 2 * Lrow, geo,
                                                 done, c, b);
        r += 3;
        bb += 3 * D;
        off += 3 * Lrow;
    }
    const int rem = count - 3 * (count / 3);
    if (rem >= 1) sched_step1<D, BG, PREC, ZC, true, kStepAny>(p, s_at, app, z, t, r, bb, off, geo, done, a, c);
    if (rem == 2)
        sched_step1<D, BG, PREC, ZC, true, kStepAny>(p, s_at, app, z, t, r + 1, bb + D, off + Lrow, geo, done, b, a);
    if (rem == 1) {
        const uint4 x = a;
        a = b;
        b = c;
        c = x;
    } else if (rem == 2) {
        const uint4 x = c;
        c = b;
        b = a;
        a = x;
    }
}

// One check node per thread: G codewords per CTA of G Z threads (as cns_sched_tile).
template <int BG, int PREC, int ZC, bool TRUNC>
__device__ __forceinline__ void cns_sched_tile1(const Params &p, int64_t cw_base, int64_t msg_cw0,
                                                unsigned char *smem, const int2 *s_at) {
    using S = Sched<BG>;
    using L = SchedLayout<BG, PREC>;
    const int ZV = ZC ? ZC : p.Z;
    float *s_app_all = reinterpret_cast<float *>(smem);
    uint32_t *s_vb = reinterpret_cast<uint32_t *>(s_app_all + (size_t)p.G * p.n);
    int32_t *s_rp = reinterpret_cast<int32_t *>(s_vb + p.nnz);
    int *s_flag = reinterpret_cast<int *>(s_rp + p.rows + 1);

    load_tables(p, s_vb, s_rp);  // for the syndrome check
    load_channel(p, s_app_all, cw_base);
    const int g = threadIdx.x / ZV, z = threadIdx.x - g * ZV;
    const int64_t cw = cw_base + g;
    const bool active = g < p.G && cw < p.B;
    float *app = s_app_all + (size_t)(active ? g : 0) * p.n;
    unsigned char *st =
        reinterpret_cast<unsigned char *>(p.msg) + (active ? cw - msg_cw0 : 0) * p.msg_stride * p.msg_size;
    bool done = !active;
    int iters_run = 0;
    SchedGeo geo;
    geo.Lc = (L::sb_core * ZV + 15) / 16 * 16;
    geo.Le = L::edge_ext ? (L::edge_row * ZV + 15) / 16 * 16 : (L::sb_ext * ZV + 15) / 16 * 16;
    geo.core_z = st + z * L::sb_core;
    geo.ext_z = st + 4 * geo.Lc + z * (L::edge_ext ? L::edge_a : L::sb_ext);
    __syncthreads();

    const int n_hi = min(S::n_hi, p.rows - 4), n_lo = p.rows - 4 - n_hi;
    uint4 a = make_uint4(0u, 0u, 0u, 0u), b = a, c = a;
    for (int t = 0; t < p.iters; ++t) {
        sched_run1<S::dc0, 1, 0, BG, PREC, ZC, TRUNC>(p, s_at, app, z, t, 0, 0, 0, geo.Lc, geo, done, a, b, c);
        sched_run1<S::dc1, 1, 1, BG, PREC, ZC, TRUNC>(p, s_at, app, z, t, 1, S::dc0, geo.Lc, geo.Lc, geo, done, a,
                                                  b, c);
        sched_run1<S::dc2, 1, 2, BG, PREC, ZC, TRUNC>(p, s_at, app, z, t, 2, S::dc0 + S::dc1, 2 * geo.Lc, geo.Lc,
                                                  geo, done, a, b, c);
        sched_run1<S::dc3, 1, 3, BG, PREC, ZC, TRUNC>(p, s_at, app, z, t, 3, S::dc0 + S::dc1 + S::dc2,
                                                  3 * geo.Lc, geo.Lc, geo, done, a, b, c);
        if constexpr (!TRUNC) {
            sched_run1<S::d_hi, S::n_hi, 4, BG, PREC, ZC>(p, s_at, app, z, t, 4, L::b_hi, 4 * geo.Lc, geo.Le, geo,
                                                      done, a, b, c);
            sched_run1<S::d_lo, S::rows - 4 - S::n_hi, 4 + S::n_hi, BG, PREC, ZC, false, true>(p, s_at, app, z, t, 4 + S::n_hi, L::b_lo, 4 * geo.Lc + S::n_hi * geo.Le, geo.Le, geo, done, a,
                b, c);
            if constexpr (S::rows % 3 == 1) {  // the next iteration's first step finds its state at phase 0
                const uint4 x = a;
                a = b;
                b = c;
                c = x;
            } else if constexpr (S::rows % 3 == 2) {
                const uint4 x = c;
                c = b;
                b = a;
                a = x;
            }
        } else {
            // a truncation: four core steps end at phase 1; rotate so that each run starts at phase 0
            const uint4 x = a;
            a = b;
            b = c;
            c = x;
            sched_run_n1<S::d_hi, BG, PREC, ZC>(p, s_at, app, z, t, 4, L::b_hi, 4 * geo.Lc, geo.Le, n_hi, geo, done,
                                            a, b, c);
            sched_run_n1<S::d_lo, BG, PREC, ZC>(p, s_at, app, z, t, 4 + S::n_hi, L::b_lo,
                                            4 * geo.Lc + S::n_hi * geo.Le, geo.Le, n_lo, geo, done, a, b, c);
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

// The kernel. For a full base graph with one check node per thread the tile
// is written out in the kernel body: the same steps as cns_sched_tile1, which
// (called as a function) compiles to about 8 % more instructions on sm_103a.
// That form is built for LLR input alone (CH = kChLlr: 0.4 % faster than with
// the fused path beside it) and for either input (kChAny, calling the fused
// demapper's load out of line: inlined, it costs the main loop 1.3 %); the
// other forms take either input.
template <int BG, int PREC, int ZC = 0, int K = 1, bool TRUNC = false, int CH = kChAny>
__global__ void __launch_bounds__(kMaxThreads / K, 2)
    k_layered_cns_sched(const __grid_constant__ Params p, const __grid_constant__ SchedTab tab) {
    extern __shared__ __align__(16) unsigned char smem[];
    if constexpr (K == 1 && !TRUNC) {
        using S = Sched<BG>;
        using L = SchedLayout<BG, PREC>;
        const int ZV = ZC ? ZC : p.Z;
        const int64_t cw_base = (int64_t)blockIdx.x * p.G;
        const int2 *s_at = tab.at;
        float *s_app_all = reinterpret_cast<float *>(smem);
        uint32_t *s_vb = reinterpret_cast<uint32_t *>(s_app_all + (size_t)p.G * p.n);
        int32_t *s_rp = reinterpret_cast<int32_t *>(s_vb + p.nnz);
        int *s_flag = reinterpret_cast<int *>(s_rp + p.rows + 1);
        load_tables(p, s_vb, s_rp);  // for the syndrome check
        load_channel_as<CH>(p, s_app_all, cw_base);
        const int g = threadIdx.x / ZV, z = threadIdx.x - g * ZV;
        const int64_t cw = cw_base + g;
        const bool active = g < p.G && cw < p.B;
        float *app = s_app_all + (size_t)(active ? g : 0) * p.n;
        unsigned char *st =
            reinterpret_cast<unsigned char *>(p.msg) + (active ? cw : 0) * p.msg_stride * p.msg_size;
        bool done = !active;
        int iters_run = 0;
        SchedGeo geo;
        geo.Lc = (L::sb_core * ZV + 15) / 16 * 16;
        geo.Le = L::edge_ext ? (L::edge_row * ZV + 15) / 16 * 16 : (L::sb_ext * ZV + 15) / 16 * 16;
        geo.core_z = st + z * L::sb_core;
        geo.ext_z = st + 4 * geo.Lc + z * (L::edge_ext ? L::edge_a : L::sb_ext);
        __syncthreads();
        uint4 a = make_uint4(0u, 0u, 0u, 0u), b = a, c = a;
        for (int t = 0; t < p.iters; ++t) {
            sched_run1<S::dc0, 1, 0, BG, PREC, ZC>(p, s_at, app, z, t, 0, 0, 0, geo.Lc, geo, done, a, b, c);
            sched_run1<S::dc1, 1, 1, BG, PREC, ZC>(p, s_at, app, z, t, 1, S::dc0, geo.Lc, geo.Lc, geo, done, a, b,
                                                   c);
            sched_run1<S::dc2, 1, 2, BG, PREC, ZC>(p, s_at, app, z, t, 2, S::dc0 + S::dc1, 2 * geo.Lc, geo.Lc, geo,
                                                   done, a, b, c);
            sched_run1<S::dc3, 1, 3, BG, PREC, ZC>(p, s_at, app, z, t, 3, S::dc0 + S::dc1 + S::dc2, 3 * geo.Lc,
                                                   geo.Lc, geo, done, a, b, c);
            sched_run1<S::d_hi, S::n_hi, 4, BG, PREC, ZC>(p, s_at, app, z, t, 4, L::b_hi, 4 * geo.Lc, geo.Le, geo,
                                                          done, a, b, c);
            sched_run1<S::d_lo, S::rows - 4 - S::n_hi, 4 + S::n_hi, BG, PREC, ZC, false, true>(
                p, s_at, app, z, t, 4 + S::n_hi, L::b_lo, 4 * geo.Lc + S::n_hi * geo.Le, geo.Le, geo, done, a, b,
                c);
            if constexpr (S::rows % 3 == 1) {  // the next iteration's first step finds its state at phase 0
                const uint4 x = a;
                a = b;
                b = c;
                c = x;
            } else if constexpr (S::rows % 3 == 2) {
                const uint4 x = c;
                c = b;
                b = a;
                a = x;
            }
            if (!done) iters_run = t + 1;
            if (p.early_stop) {
                if (threadIdx.x < p.G) s_flag[threadIdx.x] = 0;
                __syncthreads();
                const bool bad = !done && syndrome_bad_vec<1, ZC>(p, s_vb, s_rp, app, z);
                if (bad) s_flag[g] = 1;
                __syncthreads();
                if (!done && s_flag[g] == 0) done = true;
                if (__syncthreads_and(done)) break;
            }
        }
        __syncthreads();
        write_outputs(p, s_app_all, cw_base, iters_run, g, active, z);
    } else if constexpr (K == 1) {
        cns_sched_tile1<BG, PREC, ZC, TRUNC>(p, (int64_t)blockIdx.x * p.G, 0, smem, tab.at);
    } else {
        cns_sched_tile<BG, PREC, ZC, K, TRUNC>(p, (int64_t)blockIdx.x * p.G, 0, smem, tab.at);
    }
}

// Host: the shape (1, 2) whose base graph's first `rows` row degrees the row
// table has, or 0.
inline int sched_shape_of(const int32_t *row_ptr, int rows, int bg_shape) {
    auto match = [&](auto tag) {
        using S = decltype(tag);
        if (rows < 4 || rows > S::rows) return false;
        for (int r = 0; r < rows; ++r) {
            const int d = row_ptr[r + 1] - row_ptr[r];
            const int want = r == 0 ? S::dc0 : r == 1 ? S::dc1 : r == 2 ? S::dc2 : r == 3 ? S::dc3
                           : r < 4 + S::n_hi ? S::d_hi : S::d_lo;
            if (d != want) return false;
        }
        return true;
    };
    if (bg_shape == 1 && match(Sched<1>{})) return 1;
    if (bg_shape == 2 && match(Sched<2>{})) return 2;
    return 0;
}

using SchedFn = void (*)(Params, SchedTab);

// Kernel for a code whose row degrees follow the base graph of shape bg (1 or
// 2), full (k check nodes per thread: 1, or 2 when Z is even) or truncated
// (trunc, one check node per thread), or nullptr.
// qam: the channel input is received symbols (ldpc_bp_decode_qam).
SchedFn layered_cns_sched_kernel(int bg, int prec, int Z, int k, bool trunc, bool qam = false);

}  // namespace dec
}  // namespace ldpcx
