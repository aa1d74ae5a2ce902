// Belief-propagation decoding of seeded QC-LDPC codes (LDPC5GDecoder of the
// paper's Listing 1; min-sum BP as the custom CUDA op of Sec. IV-A).
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
// layer's messages are loaded into registers while the current layer computes.
//
// Arithmetic is binary32 with explicit round-to-nearest intrinsics (no fused
// multiply-add), in the operation order of the decoder definition in ldpcx.h.
#include <math.h>

#include <atomic>

#include "common.cuh"

namespace ldpcx {
namespace {

__device__ unsigned int g_status;

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

struct Params {
    const uint32_t *blk;
    const int32_t *row_ptr;
    int Z, rows, nnz, n, k, n_tx, p0;
    int iters, early_stop;
    float offset, clamp, phi_lo;  // phi_lo = phi(clamp)
    const float *llr;             // [B][n_tx]
    void *msg;                    // [B][msg_stride]
    int64_t msg_stride;
    const float *weights;         // flooding: [iters][nnz] or null
    float *llr_out;               // [B][n] or null
    uint32_t *bits_out;           // [B][kw] or null
    int32_t *iters_out;           // [B] or null
    int64_t B;
    int G;                        // codewords per CTA
    int pf_dist;                  // L2 prefetch distance in layers (0 = off)
    int msg_size;                 // bytes per message
};

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

// Load the channel LLRs of the CTA's codewords into app (placed: punctured and
// untransmitted positions are 0).
__device__ void load_channel(const Params &p, float *app, int64_t cw_base) {
    bool bad = false;
    for (int g = 0; g < p.G; ++g) {
        const int64_t cw = cw_base + g;
        for (int v = threadIdx.x; v < p.n; v += blockDim.x) {
            float x = 0.0f;
            const int t = v - p.p0;
            if (cw < p.B && t >= 0 && t < p.n_tx) x = clamp_llr(p.llr[cw * p.n_tx + t], p.clamp, bad);
            app[(size_t)g * p.n + v] = x;
        }
    }
    if (bad) latch(&g_status, LDPCX_FLAG_NONFINITE);
}

__device__ __forceinline__ int vn_index(uint32_t b, int z, int Z) {
    const int col = (int)(b >> 16);
    int zz = z + (int)(b & 0xFFFFu);
    zz -= (zz >= Z) ? Z : 0;
    return col * Z + zz;
}

// Check-node rule on the variable-to-check inputs T[0..deg): prepare() reduces
// the inputs to the check's state, value(j) then gives the (clamped, not yet
// rounded) check-to-variable message of edge j.
template <int DMAX, int ALGO> struct CheckNode;

template <int DMAX> struct CheckNode<DMAX, kMinSum> {
    float v1, v2;   // offset, floored and clamped smallest / second smallest |T|
    int idx;        // first index of the smallest |T|
    unsigned neg;   // bit j: T_j < 0
    unsigned par;   // parity of the negative inputs
    __device__ __forceinline__ void prepare(const float (&T)[DMAX], int deg, float offset, float clamp, float) {
        float m1 = INFINITY, m2 = INFINITY;
        idx = 0;
        neg = 0;
#pragma unroll
        for (int j = 0; j < DMAX; ++j) {
            if (j < deg) {
                const float a = fabsf(T[j]);
                const bool lt = a < m1;
                m2 = lt ? m1 : fminf(m2, a);
                m1 = lt ? a : m1;
                idx = lt ? j : idx;
                neg |= (T[j] < 0.0f ? 1u : 0u) << j;
            }
        }
        par = __popc(neg) & 1u;
        v1 = fminf(fmaxf(__fsub_rn(m1, offset), 0.0f), clamp);
        v2 = fminf(fmaxf(__fsub_rn(m2, offset), 0.0f), clamp);
    }
    __device__ __forceinline__ float value(int j, float, float) const {
        const float mag = (j == idx) ? v2 : v1;
        return ((par ^ (neg >> j)) & 1u) ? -mag : mag;
    }
};

template <int DMAX> struct CheckNode<DMAX, kSpa> {
    float f[DMAX];       // phi(|T_j|) with the argument clamped to [phi(clamp), clamp]
    float s_rest, s_all; // sum without the largest term / with it
    int jm;              // index of the largest term
    unsigned neg, par;
    __device__ __forceinline__ void prepare(const float (&T)[DMAX], int deg, float, float clamp, float phi_lo) {
        float fmax = -1.0f;
        jm = 0;
        neg = 0;
#pragma unroll
        for (int j = 0; j < DMAX; ++j) {
            if (j < deg) {
                const float a = fminf(fmaxf(fabsf(T[j]), phi_lo), clamp);
                f[j] = phi(a);
                const bool gt = f[j] > fmax;
                fmax = gt ? f[j] : fmax;
                jm = gt ? j : jm;
                neg |= (T[j] < 0.0f ? 1u : 0u) << j;
            }
        }
        par = __popc(neg) & 1u;
        // Exclusive sums without cancellation: the largest term is left out of
        // the running sum, so s_all - f_j (f_j <= largest) loses at most a bit.
        s_rest = 0.0f;
#pragma unroll
        for (int j = 0; j < DMAX; ++j)
            if (j < deg && j != jm) s_rest = __fadd_rn(s_rest, f[j]);
        s_all = __fadd_rn(s_rest, fmax);
    }
    __device__ __forceinline__ float value(int j, float clamp, float phi_lo) const {
        float x = (j == jm) ? s_rest : __fsub_rn(s_all, f[j]);
        x = fminf(fmaxf(x, phi_lo), clamp);
        const float mag = fminf(phi(x), clamp);
        return ((par ^ (neg >> j)) & 1u) ? -mag : mag;
    }
};

// Write final outputs of the CTA's codewords from app.
__device__ void write_outputs(const Params &p, const float *app, int64_t cw_base, int iters_run, int g, bool active) {
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
    if (p.iters_out && active && (threadIdx.x % p.Z) == 0) p.iters_out[cw_base + g] = iters_run;
}

// Parity of every check node of the thread's z over the current hard decisions.
__device__ __forceinline__ bool syndrome_bad(const Params &p, const uint32_t *s_blk, const int32_t *s_rp,
                                             const float *app, int z) {
    bool bad = false;
    for (int r = 0; r < p.rows; ++r) {
        unsigned par = 0;
        for (int b = s_rp[r]; b < s_rp[r + 1]; ++b) par ^= app[vn_index(s_blk[b], z, p.Z)] < 0.0f ? 1u : 0u;
        bad |= par != 0;
    }
    return bad;
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

template <int DMAX, int ALGO, int PREC>
__global__ void __launch_bounds__(kMaxThreads, 2) k_layered(const Params p) {
    using MT = typename MsgT<PREC>::T;
    extern __shared__ __align__(16) unsigned char smem[];
    float *s_app_all = reinterpret_cast<float *>(smem);
    uint32_t *s_blk = reinterpret_cast<uint32_t *>(s_app_all + (size_t)p.G * p.n);
    int32_t *s_rp = reinterpret_cast<int32_t *>(s_blk + p.nnz);
    int *s_flag = reinterpret_cast<int *>(s_rp + p.rows + 1);

    for (int i = threadIdx.x; i < p.nnz; i += blockDim.x) s_blk[i] = p.blk[i];
    for (int i = threadIdx.x; i <= p.rows; i += blockDim.x) s_rp[i] = p.row_ptr[i];
    const int64_t cw_base = (int64_t)blockIdx.x * p.G;
    load_channel(p, s_app_all, cw_base);

    const int g = threadIdx.x / p.Z, z = threadIdx.x - g * p.Z;
    const int64_t cw = cw_base + g;
    const bool active = g < p.G && cw < p.B;
    float *app = s_app_all + (size_t)(active ? g : 0) * p.n;
    MT *mp = reinterpret_cast<MT *>(p.msg) + (active ? cw : 0) * p.msg_stride + z;
    bool done = !active;
    int iters_run = 0;
    __syncthreads();

    float Rc[DMAX];
#pragma unroll
    for (int j = 0; j < DMAX; ++j) Rc[j] = 0.0f;

    for (int t = 0; t < p.iters; ++t) {
        const bool store = t + 1 < p.iters;  // the last iteration's messages are never read
        for (int r = 0; r < p.rows; ++r) {
            const int b0 = s_rp[r], deg = s_rp[r + 1] - b0;
            if (p.pf_dist > 0 && threadIdx.x == 0) l2_prefetch_layer(p, s_rp, cw_base, r, t);
            // prefetch the next layer's messages (written one iteration ago)
            int rn = r + 1, tn = t;
            if (rn == p.rows) { rn = 0; tn = t + 1; }
            const bool pf = !done && tn > 0 && tn < p.iters;
            const int bn0 = s_rp[rn], degn = s_rp[rn + 1] - bn0;
            float Rn[DMAX];
#pragma unroll
            for (int j = 0; j < DMAX; ++j) {
                Rn[j] = 0.0f;
                if (pf && j < degn) Rn[j] = msg_load<PREC>(mp + (size_t)(bn0 + j) * p.Z);
            }
            if (!done) {
                float T[DMAX];
#pragma unroll
                for (int j = 0; j < DMAX; ++j) {
                    T[j] = 0.0f;
                    if (j < deg) T[j] = __fsub_rn(app[vn_index(s_blk[b0 + j], z, p.Z)], Rc[j]);
                }
                CheckNode<DMAX, ALGO> cn;
                cn.prepare(T, deg, p.offset, p.clamp, p.phi_lo);
#pragma unroll
                for (int j = 0; j < DMAX; ++j) {
                    if (j < deg) {
                        MT q;
                        const float rq = msg_round<PREC>(cn.value(j, p.clamp, p.phi_lo), &q);
                        if (store) msg_store<PREC>(mp + (size_t)(b0 + j) * p.Z, q);
                        app[vn_index(s_blk[b0 + j], z, p.Z)] = __fadd_rn(T[j], rq);
                    }
                }
            }
            __syncthreads();
#pragma unroll
            for (int j = 0; j < DMAX; ++j) Rc[j] = Rn[j];
        }
        if (!done) iters_run = t + 1;
        if (p.early_stop) {
            if (threadIdx.x < p.G) s_flag[threadIdx.x] = 0;
            __syncthreads();
            if (!done && syndrome_bad(p, s_blk, s_rp, app, z)) s_flag[g] = 1;
            __syncthreads();
            if (!done && s_flag[g] == 0) done = true;
            if (__syncthreads_and(done)) break;
        }
    }
    __syncthreads();
    write_outputs(p, s_app_all, cw_base, iters_run, g, active);
}

template <int DMAX, int ALGO, int PREC>
__global__ void __launch_bounds__(kMaxThreads, 1) k_flooding(const Params p) {
    using MT = typename MsgT<PREC>::T;
    extern __shared__ __align__(16) unsigned char smem[];
    float *s_a = reinterpret_cast<float *>(smem);
    float *s_b = s_a + (size_t)p.G * p.n;
    uint32_t *s_blk = reinterpret_cast<uint32_t *>(s_b + (size_t)p.G * p.n);
    int32_t *s_rp = reinterpret_cast<int32_t *>(s_blk + p.nnz);
    int *s_flag = reinterpret_cast<int *>(s_rp + p.rows + 1);
    int *s_done = s_flag + p.G;

    for (int i = threadIdx.x; i < p.nnz; i += blockDim.x) s_blk[i] = p.blk[i];
    for (int i = threadIdx.x; i <= p.rows; i += blockDim.x) s_rp[i] = p.row_ptr[i];
    const int64_t cw_base = (int64_t)blockIdx.x * p.G;
    for (int i = threadIdx.x; i < p.G; i += blockDim.x) s_done[i] = (cw_base + i >= p.B) ? 1 : 0;
    load_channel(p, s_a, cw_base);

    const int g = threadIdx.x / p.Z, z = threadIdx.x - g * p.Z;
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
                for (int v = threadIdx.x; v < p.n; v += blockDim.x) {
                    float x = 0.0f;
                    const int tt = v - p.p0;
                    if (keep) x = cur[(size_t)gg * p.n + v];
                    else if (c2 < p.B && tt >= 0 && tt < p.n_tx) x = clamp_llr(p.llr[c2 * p.n_tx + tt], p.clamp, bad);
                    nxt[(size_t)gg * p.n + v] = x;
                }
            }
        }
        __syncthreads();
        const float *app = cur + (size_t)(active ? g : 0) * p.n;
        float *acc = nxt + (size_t)(active ? g : 0) * p.n;
        const float *w_t = p.weights ? p.weights + (size_t)t * p.nnz : nullptr;
        for (int r = 0; r < p.rows; ++r) {
            const int b0 = s_rp[r], deg = s_rp[r + 1] - b0;
            if (!done) {
                float T[DMAX];
#pragma unroll
                for (int j = 0; j < DMAX; ++j) {
                    T[j] = 0.0f;
                    if (j < deg) {
                        const float old = t > 0 ? msg_load<PREC>(mp + (size_t)(b0 + j) * p.Z) : 0.0f;
                        float v2c = __fsub_rn(app[vn_index(s_blk[b0 + j], z, p.Z)], old);
                        if (w_t) v2c = __fmul_rn(w_t[b0 + j], v2c);
                        T[j] = v2c;
                    }
                }
                CheckNode<DMAX, ALGO> cn;
                cn.prepare(T, deg, p.offset, p.clamp, p.phi_lo);
#pragma unroll
                for (int j = 0; j < DMAX; ++j) {
                    if (j < deg) {
                        MT q;
                        const float rq = msg_round<PREC>(cn.value(j, p.clamp, p.phi_lo), &q);
                        if (store) msg_store<PREC>(mp + (size_t)(b0 + j) * p.Z, q);
                        const int v = vn_index(s_blk[b0 + j], z, p.Z);
                        acc[v] = __fadd_rn(acc[v], rq);
                    }
                }
            }
            __syncthreads();  // rows add into the accumulator in ascending order
        }
        float *tmp = cur;
        cur = nxt;
        nxt = tmp;
        if (!done) iters_run = t + 1;
        if (p.early_stop) {
            if (threadIdx.x < p.G) s_flag[threadIdx.x] = 0;
            __syncthreads();
            if (!done && syndrome_bad(p, s_blk, s_rp, cur + (size_t)g * p.n, z)) s_flag[g] = 1;
            __syncthreads();
            if (!done && s_flag[g] == 0) {
                done = true;
                if (z == 0) s_done[g] = 1;
            }
            if (__syncthreads_and(done)) break;
        }
    }
    __syncthreads();
    write_outputs(p, cur, cw_base, iters_run, g, active);
}

using KernelFn = void (*)(Params);

template <int DMAX, int ALGO>
KernelFn pick_prec(bool layered, int prec) {
    if (layered) {
        if (prec == kF32) return k_layered<DMAX, ALGO, kF32>;
        if (prec == kF16) return k_layered<DMAX, ALGO, kF16>;
        if (ALGO == kMinSum) return k_layered<DMAX, kMinSum, kFix6>;
    } else {
        if (prec == kF32) return k_flooding<DMAX, ALGO, kF32>;
        if (prec == kF16) return k_flooding<DMAX, ALGO, kF16>;
        if (ALGO == kMinSum) return k_flooding<DMAX, kMinSum, kFix6>;
    }
    return nullptr;
}

template <int DMAX>
KernelFn pick_algo(bool layered, int algo, int prec) {
    return algo == kMinSum ? pick_prec<DMAX, kMinSum>(layered, prec) : pick_prec<DMAX, kSpa>(layered, prec);
}

KernelFn pick_kernel(int max_deg, bool layered, int algo, int prec) {
    if (max_deg <= 12) return pick_algo<12>(layered, algo, prec);
    if (max_deg <= 20) return pick_algo<20>(layered, algo, prec);
    if (max_deg <= 32) return pick_algo<32>(layered, algo, prec);
    return nullptr;
}

size_t msg_bytes(int prec) { return prec == kF32 ? 4 : prec == kF16 ? 2 : 1; }

int64_t msg_stride(const ldpcx_code *c) {
    const int64_t E = (int64_t)c->nnz * c->Z;
    return (E + 127) / 128 * 128;
}

int check_opts(const ldpcx_code *c, const ldpcx_decode_opts *o) {
    if (!o) return LDPCX_E_INVAL;
    if (o->algo < LDPCX_LAYERED_MINSUM || o->algo > LDPCX_FLOOD_SPA) return LDPCX_E_INVAL;
    if (o->iters < 1 || o->iters > 1000) return LDPCX_E_INVAL;
    if (o->msg_prec < LDPCX_MSG_F32 || o->msg_prec > LDPCX_MSG_FIX6) return LDPCX_E_INVAL;
    if (o->early_stop != 0 && o->early_stop != 1) return LDPCX_E_INVAL;
    if (!(o->offset >= 0.0f) || !(o->clamp > 0.0f) || isinf(o->offset) || isinf(o->clamp)) return LDPCX_E_INVAL;
    const bool spa = o->algo == LDPCX_LAYERED_SPA || o->algo == LDPCX_FLOOD_SPA;
    const bool layered = o->algo == LDPCX_LAYERED_MINSUM || o->algo == LDPCX_LAYERED_SPA;
    if (spa && o->msg_prec == LDPCX_MSG_FIX6) return LDPCX_E_UNSUPPORTED;
    if (o->weights && layered) return LDPCX_E_INVAL;
    if (c->max_deg > 32) return LDPCX_E_UNSUPPORTED;
    return LDPCX_OK;
}

// Codewords per CTA: enough check-node threads to fill ~384 threads, bounded
// by the shared memory that keeps two CTAs per SM (layered) or one (flooding).
int pick_G(const ldpcx_code *c, bool layered) {
    const size_t per_cw = sizeof(float) * (size_t)c->n * (layered ? 1 : 2);
    const size_t budget = layered ? 105 * 1024 : 210 * 1024;
    int G = kMaxThreads / c->Z;
    if (G < 1) G = 1;
    while (G > 1 && per_cw * G > budget) --G;
    return G;
}

std::atomic<int> g_pf_dist{3};

}  // namespace

unsigned int take_status_decode(cudaStream_t s) {
    unsigned int v = 0, zero = 0;
    if (cudaMemcpyFromSymbolAsync(&v, g_status, sizeof(v), 0, cudaMemcpyDeviceToHost, s) != cudaSuccess) return 0;
    cudaMemcpyToSymbolAsync(g_status, &zero, sizeof(zero), 0, cudaMemcpyHostToDevice, s);
    cudaStreamSynchronize(s);
    return v;
}

}  // namespace ldpcx

using namespace ldpcx;

extern "C" int ldpc_bp_workspace(ldpcx_code_t c, int64_t B, const ldpcx_decode_opts *o, size_t *ws) {
    if (!c || !ws || B < 0) return LDPCX_E_INVAL;
    int st = check_opts(c, o);
    if (st) return st;
    *ws = (size_t)B * (size_t)msg_stride(c) * msg_bytes(o->msg_prec);
    return LDPCX_OK;
}

extern "C" int ldpc_bp_decode(ldpcx_code_t c, const float *llr_ch, int64_t B, const ldpcx_decode_opts *o,
                              float *llr_out, uint32_t *bits_out, int32_t *iters_out, void *ws, size_t ws_bytes,
                              void *stream) {
    if (!c || B < 0 || (B > 0 && !llr_ch)) return LDPCX_E_INVAL;
    int st = check_opts(c, o);
    if (st) return st;
    if (B == 0) return LDPCX_OK;
    size_t need = 0;
    ldpc_bp_workspace(c, B, o, &need);
    if (!ws || ws_bytes < need || ((uintptr_t)ws & 255u)) return LDPCX_E_WORKSPACE;
    DevCode d;
    st = code_device(c, &d);
    if (st) return st;

    const bool layered = o->algo == LDPCX_LAYERED_MINSUM || o->algo == LDPCX_LAYERED_SPA;
    const int algo = (o->algo == LDPCX_LAYERED_MINSUM || o->algo == LDPCX_FLOOD_MINSUM) ? kMinSum : kSpa;
    KernelFn fn = pick_kernel(c->max_deg, layered, algo, o->msg_prec);
    if (!fn) return LDPCX_E_UNSUPPORTED;

    Params p{};
    p.blk = d.blk;
    p.row_ptr = d.row_ptr;
    p.Z = c->Z;
    p.rows = c->rows;
    p.nnz = c->nnz;
    p.n = c->n;
    p.k = c->k;
    p.n_tx = c->n_tx;
    p.p0 = c->p0;
    p.iters = o->iters;
    p.early_stop = o->early_stop;
    p.offset = o->offset;
    p.clamp = o->clamp;
    p.phi_lo = (float)log1p(2.0 / expm1((double)o->clamp));
    p.llr = llr_ch;
    p.msg = ws;
    p.msg_stride = msg_stride(c);
    p.weights = o->weights;
    p.llr_out = llr_out;
    p.bits_out = bits_out;
    p.iters_out = iters_out;
    p.B = B;
    p.G = pick_G(c, layered);
    p.pf_dist = layered ? g_pf_dist.load() : 0;
    p.msg_size = (int)msg_bytes(o->msg_prec);

    const size_t smem = smem_bytes(p, layered ? 1 : 2);
    if (smem > 227 * 1024) return LDPCX_E_UNSUPPORTED;
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return LDPCX_E_CUDA;
    int threads = p.G * p.Z;
    threads = (threads + 31) / 32 * 32;
    const int64_t grid = (B + p.G - 1) / p.G;
    if (grid > 0x7FFFFFFF) return LDPCX_E_INVAL;
    fn<<<(unsigned)grid, threads, smem, (cudaStream_t)stream>>>(p);
    return cuda_status(cudaGetLastError());
}

extern "C" int ldpcx_tune_set(int key, int value) {
    if (key == LDPCX_TUNE_L2_PREFETCH) {
        if (value < 0 || value > 16) return LDPCX_E_INVAL;
        g_pf_dist.store(value);
        return LDPCX_OK;
    }
    return LDPCX_E_INVAL;
}

extern "C" int ldpcx_tune_get(int key, int *value) {
    if (!value) return LDPCX_E_INVAL;
    if (key == LDPCX_TUNE_L2_PREFETCH) {
        *value = g_pf_dist.load();
        return LDPCX_OK;
    }
    return LDPCX_E_INVAL;
}
