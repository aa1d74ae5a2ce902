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
        if (cudaMalloc(&mem, bi + bf) != cudaSuccess) return LDPCX_E_NOMEM;
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
           + sizeof(float) * 3 * kPolarMaxL * 2            // pm, candidate metrics, leaf LLRs
           + sizeof(int) * 4 * kPolarMaxL * 2 + 64;        // slots, selection
}

__global__ void __launch_bounds__(kPolarThreads) k_polar_scl(const PolarScl p) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int N = p.N, L = p.L, T = blockDim.x;
    float *ch = reinterpret_cast<float *>(smem);
    float *alpha = ch + N;                                              // [L][N-1]
    uint8_t *beta = reinterpret_cast<uint8_t *>(alpha + (size_t)L * (N - 1));  // [L][N-1]
    uint8_t *ubuf = beta + (size_t)L * (N - 1);                         // [L][N]
    uint8_t *tmp = ubuf + (size_t)L * N;                                // [L][N]
    float *pm = reinterpret_cast<float *>((reinterpret_cast<uintptr_t>(tmp + (size_t)L * N) + 15) & ~(uintptr_t)15);
    float *cm = pm + kPolarMaxL;          // [2 L] candidate metrics
    float *lam = cm + 2 * kPolarMaxL;     // [L] leaf LLR per logical path
    int *slot = reinterpret_cast<int *>(lam + kPolarMaxL);  // [L] logical -> physical
    int *nslot = slot + kPolarMaxL;       // [L] new logical -> physical
    int *src = nslot + kPolarMaxL;        // [L] new logical -> old physical to copy from (-1: none)
    int *keep_c = src + kPolarMaxL;       // [2 L] survive flags, then [L] new bits at 2 kPolarMaxL
    __shared__ int s_cur, s_best;

    const int64_t b = blockIdx.x;
    for (int j = threadIdx.x; j < N; j += T) ch[j] = p.llr[b * N + j];
    if (threadIdx.x == 0) {
        s_cur = 1;
        pm[0] = 0.0f;
        slot[0] = 0;
    }
    __syncthreads();

    for (int i = 0; i < N; ++i) {
        const int cur = s_cur;
        // A: LLRs of the nodes that start at leaf i, from the largest down to the leaf
        const int low = i == 0 ? N / 2 : min(i & -i, N / 2);
        for (int s = low; s >= 1; s >>= 1) {
            const bool right = (i / s) & 1;
            for (int idx = threadIdx.x; idx < cur * s; idx += T) {
                const int k = idx / s, j = idx - k * s;
                const int ph = slot[k];
                float *a = alpha + (size_t)ph * (N - 1);
                const float *P = (2 * s == N) ? ch : a + (N - 4 * s);  // parent, size 2s
                const float x = P[j], y = P[j + s];
                if (!right) {
                    a[N - 2 * s + j] = f_min(x, y);
                } else {
                    const uint8_t ps = beta[(size_t)ph * (N - 1) + N - 2 * s + j];
                    a[N - 2 * s + j] = ps ? y - x : y + x;
                }
            }
            __syncthreads();
        }
        // B: decision at leaf i
        if (threadIdx.x < cur) lam[threadIdx.x] = alpha[(size_t)slot[threadIdx.x] * (N - 1) + N - 2];
        __syncthreads();
        if (p.frozen[i]) {
            if (threadIdx.x < cur) {
                const int k = threadIdx.x;
                if (lam[k] < 0.0f) pm[k] = pm[k] + fabsf(lam[k]);
                ubuf[(size_t)slot[k] * N + i] = 0;
            }
            __syncthreads();
        } else {
            const int nc = 2 * cur, keep = min(nc, L);
            if (threadIdx.x < nc) {
                const int c = threadIdx.x, k = c >> 1, bit = c & 1;
                const int h = lam[k] < 0.0f ? 1 : 0;
                cm[c] = (bit == h) ? pm[k] : pm[k] + fabsf(lam[k]);
            }
            __syncthreads();
            if (threadIdx.x < nc) {
                const int c = threadIdx.x;
                int rank = 0;
                for (int c2 = 0; c2 < nc; ++c2) rank += (cm[c2] < cm[c] || (cm[c2] == cm[c] && c2 < c)) ? 1 : 0;
                keep_c[c] = rank < keep ? 1 : 0;
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                // survivors in ascending c; the first child of a path keeps its slot, a second child
                // takes a slot of a path with no survivor (or an unused one) and is copied there
                int used[kPolarMaxL];
                for (int q = 0; q < L; ++q) used[q] = 0;
                for (int k = 0; k < cur; ++k)
                    if (keep_c[2 * k] || keep_c[2 * k + 1]) used[slot[k]] = 1;
                int nk = 0, freeq = 0;
                for (int c = 0; c < nc; ++c) {
                    if (!keep_c[c]) continue;
                    const int k = c >> 1;
                    const bool first = (c & 1) == 0 || !keep_c[c - 1];
                    if (first) {
                        nslot[nk] = slot[k];
                        src[nk] = -1;
                    } else {
                        while (used[freeq]) ++freeq;
                        used[freeq] = 1;
                        nslot[nk] = freeq;
                        src[nk] = slot[k];
                    }
                    lam[nk] = cm[c];           // reuse: the new metric
                    keep_c[2 * kPolarMaxL + nk] = c & 1;  // the new bit
                    ++nk;
                }
            }
            __syncthreads();
            // copy the duplicated paths' state
            for (int k = 0; k < keep; ++k) {
                if (src[k] < 0) continue;
                const int from = src[k], to = nslot[k];
                for (int j = threadIdx.x; j < N - 1; j += T) {
                    alpha[(size_t)to * (N - 1) + j] = alpha[(size_t)from * (N - 1) + j];
                    beta[(size_t)to * (N - 1) + j] = beta[(size_t)from * (N - 1) + j];
                }
                for (int j = threadIdx.x; j < i; j += T) ubuf[(size_t)to * N + j] = ubuf[(size_t)from * N + j];
            }
            __syncthreads();
            if (threadIdx.x < keep) {
                const int k = threadIdx.x;
                slot[k] = nslot[k];
                pm[k] = lam[k];
                ubuf[(size_t)nslot[k] * N + i] = (uint8_t)keep_c[2 * kPolarMaxL + k];
            }
            if (threadIdx.x == 0) s_cur = keep;
            __syncthreads();
        }
        // C: partial sums: leaf i closes the nodes whose last leaf it is
        const int cur2 = s_cur;
        if (threadIdx.x < cur2) tmp[(size_t)slot[threadIdx.x] * N] = ubuf[(size_t)slot[threadIdx.x] * N + i];
        __syncthreads();
        for (int s = 1; s < N; s <<= 1) {
            const bool right = (i / s) & 1;
            for (int idx = threadIdx.x; idx < cur2 * s; idx += T) {
                const int k = idx / s, j = idx - k * s;
                const int ph = slot[k];
                uint8_t *t = tmp + (size_t)ph * N;
                uint8_t *bt = beta + (size_t)ph * (N - 1) + N - 2 * s;
                if (!right) {
                    bt[j] = t[j];  // a completed left node: kept for its right sibling
                } else {
                    const uint8_t v = t[j];
                    t[s + j] = v;
                    t[j] = v ^ bt[j];
                }
            }
            __syncthreads();
            if (!right) break;
        }
    }

    // CRC-aided selection and output
    const int cur = s_cur;
    if (threadIdx.x < cur) {
        const int k = threadIdx.x;
        const uint8_t *uk = ubuf + (size_t)slot[k] * N;
        int ok = 1;
        if (p.r > 0) {
            const int Kd = p.K - p.r;
            const uint64_t rem = crc_of([&](int q) { return uk[p.info[q]]; }, Kd, p.g, p.r);
            for (int q = 0; q < p.r; ++q) ok &= ((rem >> (p.r - 1 - q)) & 1ull) == uk[p.info[Kd + q]];
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
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = T >> 5;
    for (int w = warp; w < kw; w += nwarps) {
        const int q = 32 * w + lane;
        const unsigned word = __ballot_sync(0xFFFFFFFFu, q < Kd && ub[p.info[q]] != 0);
        if (lane == 0) p.data[b * kw + w] = word;
    }
}

}  // namespace
}  // namespace ldpcx

using namespace ldpcx;

extern "C" int polar_build(int n, int K, float design_esn0_db, uint64_t crc_poly, int crc_r, ldpcx_polar_t *out) {
    if (!out || n < 2 || n > 10 || K < 1 || K > (1 << n) || crc_r < 0 || crc_r >= K || crc_r > 32) return LDPCX_E_INVAL;
    if (crc_r > 0 && !((crc_poly >> crc_r) & 1ull)) return LDPCX_E_INVAL;  // the x^r term
    ldpcx_polar *c = new (std::nothrow) ldpcx_polar();
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
    if (cudaFuncSetAttribute(k_polar_scl, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return LDPCX_E_CUDA;
    k_polar_scl<<<(unsigned)B, kPolarThreads, smem, (cudaStream_t)stream>>>(p);
    return cuda_status(cudaGetLastError());
}
