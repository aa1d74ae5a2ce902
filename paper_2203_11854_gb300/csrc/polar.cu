// Polar codes: construction (host), transmitter and CRC-aided successive-
// cancellation list decoding on the device. Conventions in ldpcx.h.
//
// Decoder layout: one CTA per codeword. Per physical path slot, shared memory
// holds the LLRs of every tree level (node size s at offset N - 2s, N - 1
// floats in all), the partial sums of the last completed left node of each
// size (same offsets, bytes), the decisions u and a combine buffer. Logical
// paths (the list in its defined order) map to physical slots, so a path
// that survives with one child keeps its slot and only a path that survives
// with two children is copied, into a slot freed by a path with none.
#include <math.h>

#include <algorithm>
#include <mutex>
#include <new>
#include <vector>

#include "common.cuh"

struct ldpcx_polar {
    int n, N, K, r;
    uint64_t g;
    std::vector<int32_t> info;
    std::vector<uint8_t> frozen;
    std::mutex mu;
    int dev = -1;
    int32_t *d_info = nullptr;
    uint8_t *d_frozen = nullptr;
};

namespace ldpcx {
namespace {

constexpr int kPolarThreads = 256;
constexpr int kPolarMaxL = 32;

int polar_device(ldpcx_polar *c, const int32_t **info, const uint8_t **frozen) {
    std::lock_guard<std::mutex> lk(c->mu);
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return LDPCX_E_CUDA;
    if (c->dev != dev) {
        if (c->d_info) {
            cudaFree(c->d_info);
            c->d_info = nullptr;
            c->d_frozen = nullptr;
        }
        void *mem = nullptr;
        const size_t bi = sizeof(int32_t) * (size_t)std::max(1, c->K), bf = (size_t)c->N;
        if (fault_alloc() || cudaMalloc(&mem, bi + bf) != cudaSuccess) {
            cudaGetLastError();
            return LDPCX_E_NOMEM;
        }
        c->d_info = (int32_t *)mem;
        c->d_frozen = (uint8_t *)mem + bi;
        if (cudaMemcpy(c->d_info, c->info.data(), sizeof(int32_t) * c->K, cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(c->d_frozen, c->frozen.data(), bf, cudaMemcpyHostToDevice) != cudaSuccess)
            return LDPCX_E_CUDA;
        c->dev = dev;
    }
    *info = c->d_info;
    *frozen = c->d_frozen;
    return LDPCX_OK;
}

// CRC remainder of bits[0..len) (bytes 0/1, read through idx) modulo g, r bits.
template <class Get>
__device__ __forceinline__ uint64_t crc_of(Get get, int len, uint64_t g, int r) {
    const uint64_t top = 1ull << (r - 1), mask = (r == 64) ? ~0ull : ((1ull << r) - 1);
    uint64_t reg = 0;
    for (int i = 0; i < len; ++i) {
        const uint64_t fb = ((reg & top) ? 1ull : 0ull) ^ (uint64_t)(get(i) & 1);
        reg = (reg << 1) & mask;
        if (fb) reg ^= g & mask;
    }
    return reg;
}

// ------------------------------------------------------------- transmitter
struct PolarTx {
    int n, N, K, r;
    uint64_t g;
    const int32_t *info;
    uint64_t seed, cw0;
    const float *no;
    int64_t no_stride;
    float *y;
    uint32_t *data;
    int64_t B;
};

__global__ void __launch_bounds__(kPolarThreads) k_polar_tx(const PolarTx p) {
    extern __shared__ __align__(16) unsigned char smem[];
    uint8_t *u = smem;  // [N]
    const int64_t b = blockIdx.x;
    const int Kd = p.K - p.r, kw = (Kd + 31) >> 5, nq = (kw + 3) >> 2;
    for (int j = threadIdx.x; j < p.N; j += blockDim.x) u[j] = 0;
    __syncthreads();
    // data bits: Philox stream 0, word w from block w/4 (as the LDPC source)
    for (int q = threadIdx.x; q < nq; q += blockDim.x) {
        const uint4 x = draw(p.seed, p.cw0 + (uint64_t)b, 0u, (uint32_t)q);
        const uint32_t w4[4] = {x.x, x.y, x.z, x.w};
        for (int e = 0; e < 4; ++e) {
            const int w = 4 * q + e;
            if (w >= kw) break;
            uint32_t word = w4[e];
            const int valid = min(32, Kd - 32 * w);
            if (valid < 32) word &= (1u << valid) - 1u;
            if (p.data) p.data[b * kw + w] = word;
            for (int t = 0; t < valid; ++t) u[p.info[32 * w + t]] = (uint8_t)((word >> t) & 1u);
        }
    }
    __syncthreads();
    if (p.r > 0 && threadIdx.x == 0) {
        const uint64_t rem = crc_of([&](int i) { return u[p.info[i]]; }, Kd, p.g, p.r);
        for (int i = 0; i < p.r; ++i) u[p.info[Kd + i]] = (uint8_t)((rem >> (p.r - 1 - i)) & 1ull);
    }
    __syncthreads();
    // x = u F^{(x)n}: butterflies of span h = 1, 2, ..., N/2
    for (int h = 1; h < p.N; h <<= 1) {
        for (int t = threadIdx.x; t < p.N / 2; t += blockDim.x) {
            const int j = (t / h) * 2 * h + (t % h);
            u[j] ^= u[j + h];
        }
        __syncthreads();
    }
    // BPSK and AWGN (Philox stream 1, as sim_tx for a real channel)
    const float sd = sqrtf(p.no[b * p.no_stride] * 0.5f);
    for (int q = threadIdx.x; q < (p.N + 3) / 4; q += blockDim.x) {
        const uint4 x = draw(p.seed, p.cw0 + (uint64_t)b, 1u, (uint32_t)q);
        const float2 g01 = box_muller(x.x, x.y), g23 = box_muller(x.z, x.w);
        const float gs[4] = {g01.x, g01.y, g23.x, g23.y};
        for (int e = 0; e < 4; ++e) {
            const int j = 4 * q + e;
            if (j < p.N) p.y[b * p.N + j] = (1.0f - 2.0f * (float)u[j]) + sd * gs[e];
        }
    }
}

}  // namespace
}  // namespace ldpcx

namespace ldpcx {
namespace {

// ---------------------------------------------------------------- decoder
struct PolarScl {
    int n, N, K, r, L;
    uint64_t g;
    const int32_t *info;
    const uint8_t *frozen;
    const float *llr;
    uint32_t *data;
    float *pm_out;
    int64_t B;
};

__device__ __forceinline__ float f_min(float a, float b) {
    const float m = fminf(fabsf(a), fabsf(b));
    return ((a < 0.0f) != (b < 0.0f)) ? -m : m;
}

// Shared-memory bytes of the decoder for (N, L).
__host__ __device__ inline size_t scl_smem(int N, int L) {
    return sizeof(float) * (size_t)N                       // channel LLRs
           + sizeof(float) * (size_t)L * (N - 1)           // alpha per slot
           + (size_t)L * (N - 1)                           // beta per slot
           + 2 * (size_t)L * N                             // u and combine buffer per slot
           + (size_t)N + 16 + sizeof(int) * ((size_t)N + 3)  // frozen flags, information positions
           + sizeof(float) * 3 * kPolarMaxL * 2            // pm, candidate metrics, leaf LLRs
           + sizeof(int) * 4 * kPolarMaxL * 2 + 64;        // slots, selection
}

// Phases of the leaf loop touch cur * s elements (cur paths, node size s = 2^ls).
// Phases of at most 32 elements run in warp 0 alone, separated by __syncwarp;
// larger ones use the whole CTA, separated by __syncthreads. `cta` records
// whether the last phase was CTA-wide, which decides the barrier a phase needs
// before it reads what the previous one wrote. Every such decision depends on
// (i, s, cur, L) only, so all threads take the same barriers.
__global__ void __launch_bounds__(kPolarThreads) k_polar_scl(const PolarScl p) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int N = p.N, L = p.L, T = blockDim.x;
    const bool w0 = threadIdx.x < 32;
    const int lane = threadIdx.x & 31;
    float *ch = reinterpret_cast<float *>(smem);
    float *alpha = ch + N;                                              // [L][N-1]
    uint8_t *beta = reinterpret_cast<uint8_t *>(alpha + (size_t)L * (N - 1));  // [L][N-1]
    uint8_t *ubuf = beta + (size_t)L * (N - 1);                         // [L][N]
    uint8_t *tmp = ubuf + (size_t)L * N;                                // [L][N]
    uint8_t *fz = tmp + (size_t)L * N;                                  // [N] frozen flags
    int *s_info = reinterpret_cast<int *>((reinterpret_cast<uintptr_t>(fz + N) + 15) & ~(uintptr_t)15);  // [K]
    float *pm = reinterpret_cast<float *>(s_info + ((p.K + 3) & ~3));
    float *cm = pm + kPolarMaxL;          // [2 L] candidate metrics
    int *slot = reinterpret_cast<int *>(cm + 2 * kPolarMaxL);  // [L] logical -> physical
    int *cpy_to = slot + kPolarMaxL;      // [L] copy destinations of this leaf
    int *cpy_from = cpy_to + kPolarMaxL;  // [L] and sources
    int *keep_c = cpy_from + kPolarMaxL;  // [L] CRC flags at the end
    __shared__ int s_cur, s_ncopy, s_best;

    const int64_t b = blockIdx.x;
    for (int j = threadIdx.x; j < N; j += T) {
        ch[j] = p.llr[b * N + j];
        fz[j] = p.frozen[j];
    }
    for (int j = threadIdx.x; j < p.K; j += T) s_info[j] = p.info[j];
    if (threadIdx.x == 0) {
        s_cur = 1;
        pm[0] = 0.0f;
        slot[0] = 0;
    }
    __syncthreads();
    bool cta = true;  // everything above is synchronised
    int cur = 1;      // equal in every thread: it changes only at info leaves, after a barrier

    auto sync_for = [&](bool wide) {
        if (wide || cta) __syncthreads();
        else if (w0) __syncwarp();
        cta = wide;
    };
    const int n = p.n;

    for (int i = 0; i < N; ++i) {
        // A: LLRs of the nodes that start at leaf i, from the largest down to the leaf
        const int llow = i == 0 ? n - 1 : min(__ffs(i) - 1, n - 1);
        for (int ls = llow; ls >= 0; --ls) {
            const int sz = 1 << ls;
            const bool wide = (cur << ls) > 32;
            sync_for(wide);
            if (!wide && !w0) continue;
            const bool right = (i >> ls) & 1;
            for (int idx = wide ? threadIdx.x : lane; idx < (cur << ls); idx += wide ? T : 32) {
                const int k = idx >> ls, j = idx & (sz - 1);
                const int ph = slot[k];
                float *a = alpha + (size_t)ph * (N - 1);
                const float *P = (2 * sz == N) ? ch : a + (N - 4 * sz);  // parent, size 2s
                const float x = P[j], y = P[j + sz];
                if (!right) {
                    a[N - 2 * sz + j] = f_min(x, y);
                } else {
                    const uint8_t ps = beta[(size_t)ph * (N - 1) + N - 2 * sz + j];
                    a[N - 2 * sz + j] = ps ? y - x : y + x;
                }
            }
        }
        // B: decision at leaf i, in warp 0
        sync_for(false);
        if (fz[i]) {
            if (w0 && lane < cur) {
                const int ph = slot[lane];
                const float l = alpha[(size_t)ph * (N - 1) + N - 2];
                if (l < 0.0f) pm[lane] = pm[lane] + fabsf(l);
                ubuf[(size_t)ph * N + i] = 0;
            }
        } else if (L == 1) {
            // one path: the decision agrees with the sign (a tie at L = 0 keeps bit 0, the smaller c)
            if (threadIdx.x == 0) {
                const float l = alpha[(size_t)slot[0] * (N - 1) + N - 2];
                ubuf[(size_t)slot[0] * N + i] = l < 0.0f ? 1 : 0;
            }
        } else {
            const int nc = 2 * cur, keep = min(nc, L);
            if (w0) {
                // candidates c = lane and lane + 32: metric, survival (the keep smallest (PM, c))
                float m[2];
                bool sv[2];
                int oslot = lane < cur ? slot[lane] : 0;
                for (int h = 0; h < 2; ++h) {
                    const int c = lane + 32 * h;
                    m[h] = 0.0f;
                    if (c < nc) {
                        const int k = c >> 1, bit = c & 1;
                        const float l = alpha[(size_t)slot[k] * (N - 1) + N - 2];
                        const int hd = l < 0.0f ? 1 : 0;
                        m[h] = (bit == hd) ? pm[k] : pm[k] + fabsf(l);
                        cm[c] = m[h];
                    }
                }
                __syncwarp();
                for (int h = 0; h < 2; ++h) {
                    const int c = lane + 32 * h;
                    int rank = 0;
                    if (c < nc)
                        for (int c2 = 0; c2 < nc; ++c2) rank += (cm[c2] < m[h] || (cm[c2] == m[h] && c2 < c)) ? 1 : 0;
                    sv[h] = c < nc && rank < keep;
                }
                const unsigned s0 = __ballot_sync(0xFFFFFFFFu, sv[0]), s1 = __ballot_sync(0xFFFFFFFFu, sv[1]);
                const unsigned long long smask = (unsigned long long)s0 | ((unsigned long long)s1 << 32);
                // duplicated paths (both children survive) and the slots in use after the selection
                const bool dup = lane < cur && ((smask >> (2 * lane)) & 3ull) == 3ull;
                const bool any = lane < cur && ((smask >> (2 * lane)) & 3ull) != 0ull;
                const unsigned used = __reduce_or_sync(0xFFFFFFFFu, any ? (1u << oslot) : 0u);
                const unsigned dmask = __ballot_sync(0xFFFFFFFFu, dup);
                const unsigned freem = ~used & (L == 32 ? 0xFFFFFFFFu : ((1u << L) - 1u));
                int srcs[2];  // old slot of each candidate's path, fetched by every lane
                for (int h = 0; h < 2; ++h) srcs[h] = __shfl_sync(0xFFFFFFFFu, oslot, (lane + 32 * h) >> 1);
                __syncwarp();
                for (int h = 0; h < 2; ++h) {
                    const int c = lane + 32 * h;
                    if (!sv[h]) continue;
                    const int k = c >> 1;
                    const int nk = __popcll(smask & ((1ull << c) - 1ull));
                    int ns;
                    const bool second = (c & 1) && ((smask >> (c - 1)) & 1ull);
                    const int srcslot = srcs[h];
                    if (!second) {
                        ns = srcslot;
                    } else {
                        const int t = __popc(dmask & ((1u << k) - 1u));  // duplicates before this one
                        ns = __fns(freem, 0, t + 1);
                        cpy_to[t] = ns;
                        cpy_from[t] = srcslot;
                    }
                    slot[nk] = ns;
                    pm[nk] = m[h];
                    ubuf[(size_t)ns * N + i] = (uint8_t)(c & 1);  // position i is not copied
                }
                if (lane == 0) {
                    s_ncopy = __popc(dmask);
                    s_cur = keep;
                }
            }
            // the copies: all threads, after the selection of warp 0
            __syncthreads();
            cur = s_cur;
            const int ncopy = s_ncopy;
            for (int q = 0; q < ncopy; ++q) {
                const int from = cpy_from[q], to = cpy_to[q];
                for (int j = threadIdx.x; j < N - 1; j += T) {
                    alpha[(size_t)to * (N - 1) + j] = alpha[(size_t)from * (N - 1) + j];
                    beta[(size_t)to * (N - 1) + j] = beta[(size_t)from * (N - 1) + j];
                }
                for (int j = threadIdx.x; j < i; j += T) ubuf[(size_t)to * N + j] = ubuf[(size_t)from * N + j];
            }
            cta = true;
        }
        // C: partial sums: leaf i closes the nodes whose last leaf it is
        for (int ls = 0; ls < n; ++ls) {
            const int sz = 1 << ls;
            const bool wide = (cur << ls) > 32;
            sync_for(wide);
            const bool right = (i >> ls) & 1;
            if (wide || w0) {
                for (int idx = wide ? threadIdx.x : lane; idx < (cur << ls); idx += wide ? T : 32) {
                    const int k = idx >> ls, j = idx & (sz - 1);
                    const int ph = slot[k];
                    uint8_t *t = tmp + (size_t)ph * N;
                    uint8_t *bt = beta + (size_t)ph * (N - 1) + N - 2 * sz;
                    const uint8_t v = (ls == 0) ? ubuf[(size_t)ph * N + i] : t[j];
                    if (!right) {
                        bt[j] = v;  // a completed left node: kept for its right sibling
                    } else {
                        t[sz + j] = v;
                        t[j] = v ^ bt[j];
                    }
                }
            }
            if (!right) break;
        }
    }

    // CRC-aided selection and output
    __syncthreads();
    if (threadIdx.x < cur) {
        const int k = threadIdx.x;
        const uint8_t *uk = ubuf + (size_t)slot[k] * N;
        int ok = 1;
        if (p.r > 0) {
            const int Kd = p.K - p.r;
            const uint64_t rem = crc_of([&](int q) { return uk[s_info[q]]; }, Kd, p.g, p.r);
            for (int q = 0; q < p.r; ++q) ok &= ((rem >> (p.r - 1 - q)) & 1ull) == uk[s_info[Kd + q]];
        }
        keep_c[k] = ok;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int best = -1;
        for (int k = 0; k < cur; ++k)
            if (keep_c[k] && (best < 0 || pm[k] < pm[best])) best = k;
        if (best < 0)
            for (int k = 0; k < cur; ++k)
                if (best < 0 || pm[k] < pm[best]) best = k;
        s_best = best;
        if (p.pm_out) p.pm_out[b] = pm[best];
    }
    __syncthreads();
    const uint8_t *ub = ubuf + (size_t)slot[s_best] * N;
    const int Kd = p.K - p.r, kw = (Kd + 31) >> 5;
    const int warp = threadIdx.x >> 5, nwarps = T >> 5;
    for (int w = warp; w < kw; w += nwarps) {
        const int q = 32 * w + lane;
        const unsigned word = __ballot_sync(0xFFFFFFFFu, q < Kd && ub[s_info[q]] != 0);
        if (lane == 0) p.data[b * kw + w] = word;
    }
}

// Successive cancellation (list of one) with one warp per codeword and
// kScWarps codewords per CTA: the same node order, f / g arithmetic, partial
// sums and path metric as k_polar_scl with L = 1 (so the same bits), but every
// phase is a warp loop separated by __syncwarp, with no CTA barrier inside the
// leaf loop. The channel LLRs are read from global memory where they are used
// (the two halves of the root, at leaves 0 and N/2). Per warp in shared
// memory: node LLRs [N-1] (node of size s at N - 2s), left-node partial sums
// [N-1], combine buffer [N], decisions [N]; per CTA: frozen flags [N] and
// information positions [K].
constexpr int kScWarps = 4;
__host__ __device__ inline size_t sc_warp_bytes(int N) {
    return ((sizeof(float) * ((size_t)N - 1) + 3 * (size_t)N + 15) / 16) * 16;
}
__host__ __device__ inline size_t sc_smem(int N, int K) {
    return kScWarps * sc_warp_bytes(N) + (((size_t)N + 15) / 16) * 16 + sizeof(int) * (size_t)K;
}

__global__ void __launch_bounds__(32 * kScWarps) k_polar_sc(const PolarScl p) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int N = p.N, n = p.n, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint8_t *fz = smem + kScWarps * sc_warp_bytes(N);
    int *s_info = reinterpret_cast<int *>(fz + ((N + 15) / 16) * 16);
    for (int j = threadIdx.x; j < N; j += blockDim.x) fz[j] = p.frozen[j];
    for (int j = threadIdx.x; j < p.K; j += blockDim.x) s_info[j] = p.info[j];
    __syncthreads();
    const int64_t b = (int64_t)blockIdx.x * kScWarps + warp;
    if (b >= p.B) return;  // a whole warp leaves; no CTA barrier follows
    unsigned char *w = smem + warp * sc_warp_bytes(N);
    const float *ch = p.llr + b * N;
    float *a = reinterpret_cast<float *>(w);                   // [N-1]
    uint8_t *beta = reinterpret_cast<uint8_t *>(a + (N - 1));  // [N-1]
    uint8_t *t = beta + (N - 1);                               // [N]
    uint8_t *u = t + N;                                        // [N]
    float pm = 0.0f;  // equal in every lane
    for (int i = 0; i < N; ++i) {
        // LLRs of the nodes that start at leaf i, from the largest down to the leaf
        const int llow = i == 0 ? n - 1 : min(__ffs(i) - 1, n - 1);
        for (int ls = llow; ls >= 0; --ls) {
            const int sz = 1 << ls;
            const bool right = (i >> ls) & 1;
            const float *P = (2 * sz == N) ? ch : a + (N - 4 * sz);  // parent, size 2s
            for (int j = lane; j < sz; j += 32) {
                const float x = (2 * sz == N) ? __ldg(P + j) : P[j], y = (2 * sz == N) ? __ldg(P + j + sz) : P[j + sz];
                if (!right) a[N - 2 * sz + j] = f_min(x, y);
                else a[N - 2 * sz + j] = beta[N - 2 * sz + j] ? y - x : y + x;
            }
            __syncwarp();
        }
        // decision at leaf i (every lane reads the same leaf LLR)
        const float l = a[N - 2];
        uint8_t ui;
        if (fz[i]) {
            ui = 0;
            if (l < 0.0f) pm = pm + fabsf(l);
        } else {
            ui = l < 0.0f ? 1 : 0;  // a tie at 0 keeps bit 0
        }
        if (lane == 0) u[i] = ui;
        // partial sums: leaf i closes the nodes whose last leaf it is
        for (int ls = 0; ls < n; ++ls) {
            const int sz = 1 << ls;
            const bool right = (i >> ls) & 1;
            uint8_t *bt = beta + N - 2 * sz;
            for (int j = lane; j < sz; j += 32) {
                const uint8_t v = (ls == 0) ? ui : t[j];
                if (!right) {
                    bt[j] = v;  // a completed left node: kept for its right sibling
                } else {
                    t[sz + j] = v;
                    t[j] = v ^ bt[j];
                }
            }
            __syncwarp();
            if (!right) break;
        }
    }
    if (p.pm_out && lane == 0) p.pm_out[b] = pm;
    const int Kd = p.K - p.r, kw = (Kd + 31) >> 5;
    for (int q0 = 0; q0 < kw; ++q0) {
        const int q = 32 * q0 + lane;
        const unsigned word = __ballot_sync(0xFFFFFFFFu, q < Kd && u[s_info[q]] != 0);
        if (lane == 0) p.data[b * kw + q0] = word;
    }
}

}  // namespace
}  // namespace ldpcx

using namespace ldpcx;

extern "C" int polar_build(int n, int K, float design_esn0_db, uint64_t crc_poly, int crc_r, ldpcx_polar_t *out) {
    if (!out || n < 2 || n > 10 || K < 1 || K > (1 << n) || crc_r < 0 || crc_r >= K || crc_r > 32) return LDPCX_E_INVAL;
    if (crc_r > 0 && !((crc_poly >> crc_r) & 1ull)) return LDPCX_E_INVAL;  // the x^r term
    ldpcx_polar *c = fault_alloc() ? nullptr : new (std::nothrow) ldpcx_polar();
    if (!c) return LDPCX_E_NOMEM;
    c->n = n;
    c->N = 1 << n;
    c->K = K;
    c->r = crc_r;
    c->g = crc_poly;
    // Bhattacharyya parameters: the transforms of the bits of i, most significant first
    const double z0 = exp(-pow(10.0, (double)design_esn0_db / 10.0));
    std::vector<double> z((size_t)c->N);
    for (int i = 0; i < c->N; ++i) {
        double v = z0;
        for (int bit = n - 1; bit >= 0; --bit) v = ((i >> bit) & 1) ? v * v : 2.0 * v - v * v;
        z[(size_t)i] = v;
    }
    std::vector<int> order((size_t)c->N);
    for (int i = 0; i < c->N; ++i) order[(size_t)i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        return z[(size_t)a] < z[(size_t)b] || (z[(size_t)a] == z[(size_t)b] && a > b);
    });
    c->frozen.assign((size_t)c->N, 1);
    for (int i = 0; i < K; ++i) c->frozen[(size_t)order[(size_t)i]] = 0;
    for (int i = 0; i < c->N; ++i)
        if (!c->frozen[(size_t)i]) c->info.push_back(i);
    *out = c;
    return LDPCX_OK;
}

extern "C" int polar_free(ldpcx_polar_t c) {
    if (!c) return LDPCX_OK;
    if (c->d_info) cudaFree(c->d_info);
    delete c;
    return LDPCX_OK;
}

extern "C" int polar_info(ldpcx_polar_t c, int *N, int *K, int *crc_r, int32_t *info_out) {
    if (!c) return LDPCX_E_INVAL;
    if (N) *N = c->N;
    if (K) *K = c->K;
    if (crc_r) *crc_r = c->r;
    if (info_out) std::copy(c->info.begin(), c->info.end(), info_out);
    return LDPCX_OK;
}

extern "C" int polar_sim_tx(ldpcx_polar_t c, uint64_t seed, uint64_t cw0, int64_t B, const float *no,
                            int64_t no_stride, float *y_out, uint32_t *data_out, void *stream) {
    if (!c || B < 0 || (no_stride != 0 && no_stride != 1)) return LDPCX_E_INVAL;
    if (B == 0) return LDPCX_OK;
    if (!no || !y_out || B > 0x7FFFFFFF) return LDPCX_E_INVAL;
    const int32_t *info;
    const uint8_t *frozen;
    int st = polar_device(c, &info, &frozen);
    if (st) return st;
    PolarTx p{};
    p.n = c->n;
    p.N = c->N;
    p.K = c->K;
    p.r = c->r;
    p.g = c->g;
    p.info = info;
    p.seed = seed;
    p.cw0 = cw0;
    p.no = no;
    p.no_stride = no_stride;
    p.y = y_out;
    p.data = data_out;
    p.B = B;
    k_polar_tx<<<(unsigned)B, kPolarThreads, (size_t)c->N, (cudaStream_t)stream>>>(p);
    return cuda_status(cudaGetLastError());
}

extern "C" int polar_scl_decode(ldpcx_polar_t c, const float *llr, int64_t B, int L, uint32_t *data_out,
                                float *pm_out, void *stream) {
    if (!c || B < 0 || L < 1 || L > kPolarMaxL) return LDPCX_E_INVAL;
    if (B == 0) return LDPCX_OK;
    if (!llr || !data_out || B > 0x7FFFFFFF) return LDPCX_E_INVAL;
    const size_t smem = scl_smem(c->N, L);
    if (smem > 227 * 1024) return LDPCX_E_UNSUPPORTED;
    const int32_t *info;
    const uint8_t *frozen;
    int st = polar_device(c, &info, &frozen);
    if (st) return st;
    PolarScl p{};
    p.n = c->n;
    p.N = c->N;
    p.K = c->K;
    p.r = c->r;
    p.L = L;
    p.g = c->g;
    p.info = info;
    p.frozen = frozen;
    p.llr = llr;
    p.data = data_out;
    p.pm_out = pm_out;
    p.B = B;
    if (L == 1) {
        // a list of one: one warp per codeword
        const size_t ssm = sc_smem(c->N, c->K);
        if (ssm > 48 * 1024 &&
            cudaFuncSetAttribute(k_polar_sc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ssm) != cudaSuccess)
            return LDPCX_E_CUDA;
        const int64_t grid = (B + kScWarps - 1) / kScWarps;
        k_polar_sc<<<(unsigned)grid, 32 * kScWarps, ssm, (cudaStream_t)stream>>>(p);
        return cuda_status(cudaGetLastError());
    }
    if (cudaFuncSetAttribute(k_polar_scl, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return LDPCX_E_CUDA;
    // small lists run mostly in warp 0: fewer threads per CTA leave room for more CTAs per SM
    const int threads = L <= 2 ? 64 : L <= 8 ? 128 : kPolarThreads;
    k_polar_scl<<<(unsigned)B, threads, smem, (cudaStream_t)stream>>>(p);
    return cuda_status(cudaGetLastError());
}
