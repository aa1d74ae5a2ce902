// Code construction (seeded 5G-shaped QC-LDPC base matrices), code objects,
// status helpers. Host code only; the device tables are uploaded lazily.
#include <string.h>

#include <algorithm>
#include <new>

#include "common.cuh"

namespace {

// splitmix64 (Steele, Lea & Flood, OOPSLA 2014): Weyl step 0x9E3779B97F4A7C15,
// then xor-shift-multiply by 0xBF58476D1CE4E5B9 (>>30) and 0x94D049BB133111EB
// (>>27), final >>31 xor-shift.
struct SplitMix64 {
    uint64_t x;
    uint64_t next() {
        x += 0x9E3779B97F4A7C15ull;
        uint64_t z = x;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    }
    uint32_t below(uint32_t n) { return (uint32_t)(next() % n); }
};

struct Shape {
    int kb, n_ext, d_core;
    int d_ext(int j) const;
    int bg;
};

int Shape::d_ext(int j) const { return bg == 1 ? (j < 33 ? 5 : 4) : (j < 4 ? 4 : 3); }

// Draw `count` distinct values of [0, N) by a partial Fisher-Yates shuffle.
void draw_distinct(SplitMix64 &rng, int N, int count, int *out) {
    int pool[64];
    for (int i = 0; i < N; ++i) pool[i] = i;
    for (int i = 0; i < count; ++i) {
        int j = i + (int)rng.below((uint32_t)(N - i));
        std::swap(pool[i], pool[j]);
        out[i] = pool[i];
    }
}

// Full (untruncated) seeded base matrix of the BG shape; -1 = zero block.
void seeded_base(const Shape &sh, int Z, uint64_t seed, std::vector<int16_t> &S, int &M, int &C) {
    M = 4 + sh.n_ext;
    C = sh.kb + M;
    S.assign((size_t)M * C, -1);
    std::vector<uint8_t> drawn((size_t)M * C, 0);
    SplitMix64 rng{seed};
    int pick[32];
    for (int r = 0; r < 4; ++r) {
        draw_distinct(rng, sh.kb, sh.d_core, pick);
        for (int i = 0; i < sh.d_core; ++i) drawn[(size_t)r * C + pick[i]] = 1;
    }
    for (int j = 0; j < sh.n_ext; ++j) {
        const int d = sh.d_ext(j);
        draw_distinct(rng, sh.kb + 4, d, pick);
        for (int i = 0; i < d; ++i) drawn[(size_t)(4 + j) * C + pick[i]] = 1;
        S[(size_t)(4 + j) * C + sh.kb + 4 + j] = 0;  // extension identity
    }
    // dual-diagonal core: rows of blocks over columns kb..kb+3
    static const int core[4][4] = {{1, 0, -1, -1}, {0, 0, 0, -1}, {-1, -1, 0, 0}, {1, -1, -1, 0}};
    for (int r = 0; r < 4; ++r)
        for (int c = 0; c < 4; ++c)
            if (core[r][c] >= 0) S[(size_t)r * C + sh.kb + c] = (int16_t)core[r][c];
    for (int r = 0; r < M; ++r)
        for (int c = 0; c < C; ++c)
            if (drawn[(size_t)r * C + c]) S[(size_t)r * C + c] = (int16_t)rng.below((uint32_t)Z);
}

}  // namespace

extern "C" const char *ldpcx_status_str(int status) {
    switch (status) {
        case LDPCX_OK: return "LDPCX_OK";
        case LDPCX_E_INVAL: return "LDPCX_E_INVAL: invalid argument";
        case LDPCX_E_UNSUPPORTED: return "LDPCX_E_UNSUPPORTED: not supported by this build";
        case LDPCX_E_NOMEM: return "LDPCX_E_NOMEM: allocation failed";
        case LDPCX_E_WORKSPACE: return "LDPCX_E_WORKSPACE: workspace missing, too small or misaligned";
        case LDPCX_E_CUDA: return "LDPCX_E_CUDA: CUDA runtime error";
        case LDPCX_E_NONFINITE: return "LDPCX_E_NONFINITE: non-finite input sanitised";
        case LDPCX_E_TIMEOUT: return "LDPCX_E_TIMEOUT: bounded device wait gave up";
        case LDPCX_E_NODEVICE: return "LDPCX_E_NODEVICE: no CUDA device";
        default: return "unknown ldpcx status";
    }
}

extern "C" int ldpcx_sync_status(void *stream, unsigned int *flags) {
    cudaStream_t s = (cudaStream_t)stream;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return LDPCX_E_NODEVICE;
    }
    if (cudaStreamSynchronize(s) != cudaSuccess) return LDPCX_E_CUDA;
    unsigned int f = ldpcx::take_status_decode(s) | ldpcx::take_status_channel(s);
    if (flags) *flags = f;
    if (f & LDPCX_FLAG_TIMEOUT) return LDPCX_E_TIMEOUT;
    if (f & LDPCX_FLAG_NONFINITE) return LDPCX_E_NONFINITE;
    return LDPCX_OK;
}

extern "C" int qc_ldpc_build(const ldpcx_code_params *p, ldpcx_code_t *out) {
    if (!p || !out) return LDPCX_E_INVAL;
    Shape sh{};
    if (p->bg_shape == 1) sh = Shape{22, 42, 16, 1};
    else if (p->bg_shape == 2) sh = Shape{10, 38, 8, 2};
    else return LDPCX_E_INVAL;
    if (p->Z < 2 || p->Z > ldpcx::kMaxZ) return LDPCX_E_INVAL;
    const int M_full = 4 + sh.n_ext;
    const int rows = p->rows_kept == 0 ? M_full : p->rows_kept;
    if (rows < 4 || rows > M_full) return LDPCX_E_INVAL;
    if (p->punct_cols < 0 || p->punct_cols > sh.kb) return LDPCX_E_INVAL;

    ldpcx_code *c = new (std::nothrow) ldpcx_code();
    if (!c) return LDPCX_E_NOMEM;
    c->params = *p;
    std::vector<int16_t> full;
    int M = 0, C = 0;
    seeded_base(sh, p->Z, p->seed, full, M, C);
    c->Z = p->Z;
    c->rows = rows;
    c->kb = sh.kb;
    c->cols = sh.kb + rows;
    c->n = c->cols * c->Z;
    c->k = c->kb * c->Z;
    c->p0 = p->punct_cols * c->Z;
    c->n_tx = p->n_tx == 0 ? c->n - c->p0 : p->n_tx;
    if (c->n_tx < 1 || c->p0 + c->n_tx > c->n) {
        delete c;
        return LDPCX_E_INVAL;
    }
    c->S.resize((size_t)rows * c->cols);
    for (int r = 0; r < rows; ++r)
        for (int col = 0; col < c->cols; ++col) c->S[(size_t)r * c->cols + col] = full[(size_t)r * C + col];
    c->row_ptr.assign(rows + 1, 0);
    c->max_deg = 0;
    for (int r = 0; r < rows; ++r) {
        int deg = 0;
        for (int col = 0; col < c->cols; ++col) {
            const int s = c->S[(size_t)r * c->cols + col];
            if (s < 0) continue;
            c->blk.push_back(((uint32_t)col << 16) | (uint32_t)s);
            ++deg;
        }
        c->row_ptr[r + 1] = c->row_ptr[r] + deg;
        c->max_deg = std::max(c->max_deg, deg);
    }
    c->nnz = (int)c->blk.size();
    *out = c;
    return LDPCX_OK;
}

extern "C" int qc_ldpc_free(ldpcx_code_t c) {
    if (!c) return LDPCX_OK;
    if (c->d_tables) {
        int cur = -1;
        cudaGetDevice(&cur);
        if (cur != c->dev) cudaSetDevice(c->dev);
        cudaFree(c->d_tables);
        if (cur >= 0 && cur != c->dev) cudaSetDevice(cur);
    }
    delete c;
    return LDPCX_OK;
}

extern "C" int qc_ldpc_info(ldpcx_code_t c, ldpcx_code_info *info) {
    if (!c || !info) return LDPCX_E_INVAL;
    info->Z = c->Z;
    info->rows = c->rows;
    info->cols = c->cols;
    info->kb = c->kb;
    info->nnz = c->nnz;
    info->max_row_deg = c->max_deg;
    info->n = c->n;
    info->k = c->k;
    info->n_tx = c->n_tx;
    info->p0 = c->p0;
    info->edges = (int64_t)c->nnz * c->Z;
    return LDPCX_OK;
}

extern "C" int qc_ldpc_base(ldpcx_code_t c, int16_t *S_out, int capacity) {
    if (!c || !S_out || capacity < c->rows * c->cols) return LDPCX_E_INVAL;
    memcpy(S_out, c->S.data(), sizeof(int16_t) * c->S.size());
    return LDPCX_OK;
}

namespace ldpcx {

int code_device(ldpcx_code_t c, DevCode *out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return LDPCX_E_NODEVICE;
    }
    std::lock_guard<std::mutex> lock(c->mu);
    if (c->d_tables && c->dev != dev) return LDPCX_E_INVAL;  // tables live on another device
    if (!c->d_tables) {
        const size_t nb = sizeof(uint32_t) * c->blk.size();
        const size_t nr = sizeof(int32_t) * c->row_ptr.size();
        void *p = nullptr;
        if (cudaMalloc(&p, nb + nr) != cudaSuccess) {
            cudaGetLastError();
            return LDPCX_E_NOMEM;
        }
        if (cudaMemcpy(p, c->blk.data(), nb, cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy((char *)p + nb, c->row_ptr.data(), nr, cudaMemcpyHostToDevice) != cudaSuccess) {
            cudaFree(p);
            return LDPCX_E_CUDA;
        }
        c->d_tables = p;
        c->dev = dev;
        c->d.blk = (const uint32_t *)p;
        c->d.row_ptr = (const int32_t *)((char *)p + nb);
    }
    *out = c->d;
    return LDPCX_OK;
}

int sm_count() {
    static int cached[64] = {0};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) return 152;
    if (!cached[dev]) {
        int v = 0;
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
        cached[dev] = v > 0 ? v : 152;
    }
    return cached[dev];
}

}  // namespace ldpcx
