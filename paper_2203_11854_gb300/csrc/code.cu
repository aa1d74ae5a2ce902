// Code construction (seeded 5G-shaped QC-LDPC base matrices), code objects,
// status helpers. Host code only; the device tables are uploaded lazily.
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <new>
#include <string>
#include <vector>

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

// Block table, row pointers and largest row degree from c->S.
void index_blocks(ldpcx_code *c) {
    c->blk.clear();
    c->row_ptr.assign(c->rows + 1, 0);
    c->max_deg = 0;
    for (int r = 0; r < c->rows; ++r) {
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
}

// GF(2) inverse of the core parity part H_core (rows 0..3, columns kb..kb+3,
// a 4Z x 4Z matrix: block (r, kb+j) with shift s has ones at (rZ + z,
// jZ + (z+s) mod Z)) by Gauss-Jordan elimination on [H_core | I]. Row i of the
// inverse is written to inv[i * nw ..], bit j of word j/32 = entry (i, j).
// False when H_core is singular.
bool core_inverse(const ldpcx_code *c, std::vector<uint32_t> &inv, int &nw) {
    const int Z = c->Z, N = 4 * Z;
    nw = (N + 31) / 32;
    const int W = 2 * nw;  // words per augmented row
    std::vector<uint32_t> a((size_t)N * W, 0u);
    auto set = [&](int row, int col) { a[(size_t)row * W + (col >> 5)] ^= 1u << (col & 31); };
    for (int r = 0; r < 4; ++r)
        for (int j = 0; j < 4; ++j) {
            const int s = c->S[(size_t)r * c->cols + c->kb + j];
            if (s < 0) continue;
            for (int z = 0; z < Z; ++z) set(r * Z + z, j * Z + (z + s) % Z);
        }
    for (int i = 0; i < N; ++i) a[(size_t)i * W + nw + (i >> 5)] |= 1u << (i & 31);
    for (int col = 0; col < N; ++col) {
        const int w = col >> 5;
        const uint32_t bit = 1u << (col & 31);
        int piv = -1;
        for (int i = col; i < N; ++i)
            if (a[(size_t)i * W + w] & bit) {
                piv = i;
                break;
            }
        if (piv < 0) return false;
        if (piv != col)
            for (int k = 0; k < W; ++k) std::swap(a[(size_t)piv * W + k], a[(size_t)col * W + k]);
        for (int i = 0; i < N; ++i)
            if (i != col && (a[(size_t)i * W + w] & bit))
                for (int k = 0; k < W; ++k) a[(size_t)i * W + k] ^= a[(size_t)col * W + k];
    }
    inv.assign((size_t)N * nw, 0u);
    for (int i = 0; i < N; ++i)
        for (int k = 0; k < nw; ++k) inv[(size_t)i * nw + k] = a[(size_t)i * W + nw + k];
    return true;
}

// Which encoder the transmitter can use for c (ldpcx::kEnc*), with the core
// inverse when it needs one.
void analyse_encoder(ldpcx_code *c) {
    c->enc = ldpcx::kEncNone;
    c->core_inv.clear();
    c->inv_words = 0;
    const int kb = c->kb, C = c->cols;
    if (c->rows < 4 || C != kb + c->rows) return;
    auto S = [&](int r, int col) { return (int)c->S[(size_t)r * C + col]; };
    for (int r = 0; r < c->rows; ++r)
        for (int col = kb + 4; col < C; ++col)
            if (S(r, col) >= 0 && !(r >= 4 && col == kb + r)) return;  // a parity column out of order
    for (int r = 4; r < c->rows; ++r)
        if (S(r, kb + r) < 0) return;  // extension row without its own parity block
    static const int dual[4][4] = {{1, 0, -1, -1}, {0, 0, 0, -1}, {-1, -1, 0, 0}, {1, -1, -1, 0}};
    bool is_dual = true;
    for (int r = 0; r < 4; ++r)
        for (int j = 0; j < 4; ++j) is_dual = is_dual && S(r, kb + j) == dual[r][j];
    if (is_dual) {
        c->enc = ldpcx::kEncDualDiag;
        return;
    }
    int nw = 0;
    if (core_inverse(c, c->core_inv, nw)) {
        c->enc = ldpcx::kEncCoreInv;
        c->inv_words = nw;
    }
}

// Lines of text split into integer tokens (empty lines kept); false on any
// other token.
bool int_lines(const char *text, size_t len, std::vector<std::vector<long>> &lines) {
    lines.clear();
    std::vector<long> cur;
    size_t i = 0;
    auto flush = [&]() {
        lines.push_back(cur);
        cur.clear();
    };
    while (i < len && text[i] != '\0') {
        const char ch = text[i];
        if (ch == '\n') {
            flush();
            ++i;
        } else if (ch == ' ' || ch == '\t' || ch == '\r') {
            ++i;
        } else if (ch >= '0' && ch <= '9') {
            long v = 0;
            while (i < len && text[i] >= '0' && text[i] <= '9') {
                v = v * 10 + (text[i] - '0');
                if (v > 100000000L) return false;
                ++i;
            }
            cur.push_back(v);
        } else {
            return false;
        }
    }
    flush();
    return true;
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
        case LDPCX_E_IO: return "LDPCX_E_IO: checkpoint file could not be read, parsed or written";
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

    ldpcx_code *c = ldpcx::fault_alloc() ? nullptr : new (std::nothrow) ldpcx_code();
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
    index_blocks(c);
    analyse_encoder(c);
    *out = c;
    return LDPCX_OK;
}

extern "C" int qc_ldpc_build_base(const ldpcx_base_params *p, ldpcx_code_t *out) {
    if (!p || !out || !p->S) return LDPCX_E_INVAL;
    if (p->Z < 2 || p->Z > ldpcx::kMaxZ) return LDPCX_E_INVAL;
    if (p->rows < 1 || p->rows > 4096 || p->cols < 2 || p->cols > 4096) return LDPCX_E_INVAL;
    if (p->kb < 1 || p->kb >= p->cols) return LDPCX_E_INVAL;
    if (p->punct_cols < 0 || p->punct_cols > p->kb) return LDPCX_E_INVAL;
    for (int r = 0; r < p->rows; ++r) {
        int deg = 0;
        for (int col = 0; col < p->cols; ++col) {
            const int s = p->S[(size_t)r * p->cols + col];
            if (s < -1 || s >= p->Z) return LDPCX_E_INVAL;
            deg += s >= 0;
        }
        if (deg < 2) return LDPCX_E_INVAL;  // every check node needs two edges
    }
    ldpcx_code *c = ldpcx::fault_alloc() ? nullptr : new (std::nothrow) ldpcx_code();
    if (!c) return LDPCX_E_NOMEM;
    c->params = ldpcx_code_params{0, p->Z, 0ull, 0, p->punct_cols, p->n_tx};
    c->Z = p->Z;
    c->rows = p->rows;
    c->cols = p->cols;
    c->kb = p->kb;
    c->n = c->cols * c->Z;
    c->k = c->kb * c->Z;
    c->p0 = p->punct_cols * c->Z;
    c->n_tx = p->n_tx == 0 ? c->n - c->p0 : p->n_tx;
    if (c->n_tx < 1 || c->p0 + c->n_tx > c->n) {
        delete c;
        return LDPCX_E_INVAL;
    }
    c->S.assign(p->S, p->S + (size_t)p->rows * p->cols);
    index_blocks(c);
    analyse_encoder(c);
    *out = c;
    return LDPCX_OK;
}

extern "C" int qc_alist_parse(const char *text, size_t len, int Z, int16_t *S_out, int capacity, int *rows_out,
                              int *cols_out) {
    if (!text || !rows_out || !cols_out || Z < 1 || Z > ldpcx::kMaxZ) return LDPCX_E_INVAL;
    std::vector<std::vector<long>> all, L;
    if (!int_lines(text, len, all)) return LDPCX_E_INVAL;
    // the header: the first four non-empty lines
    size_t at = 0;
    while (L.size() < 4 && at < all.size()) {
        if (!all[at].empty()) L.push_back(all[at]);
        ++at;
    }
    if (L.size() < 4 || L[0].size() != 2 || L[1].size() != 2) return LDPCX_E_INVAL;
    const long N = L[0][0], M = L[0][1];
    if (N < 1 || M < 1 || N % Z || M % Z || N / Z > 4096 || M / Z > 4096) return LDPCX_E_INVAL;
    if ((long)L[2].size() != N || (long)L[3].size() != M) return LDPCX_E_INVAL;
    // the N + M lists: the non-empty lines that follow, or, when a list is
    // empty (a weight-0 column or row written without padding), every line
    // that follows up to the trailing empty ones
    std::vector<std::vector<long>> rest(all.begin() + (long)at, all.end());
    while (!rest.empty() && rest.back().empty()) rest.pop_back();
    long nonempty = 0;
    for (const auto &ln : rest) nonempty += !ln.empty();
    if (nonempty == N + M) {
        for (const auto &ln : rest)
            if (!ln.empty()) L.push_back(ln);
    } else if ((long)rest.size() == N + M) {
        L.insert(L.end(), rest.begin(), rest.end());
    } else {
        return LDPCX_E_INVAL;
    }
    // the row lists give the entries; the column lists must give the same ones
    std::vector<std::vector<int>> by_col((size_t)N);
    long entries = 0;
    for (long i = 0; i < M; ++i) {
        long cnt = 0;
        for (long v : L[4 + N + i]) {
            if (v == 0) continue;  // padding
            if (v > N) return LDPCX_E_INVAL;
            by_col[(size_t)(v - 1)].push_back((int)i);
            ++cnt;
        }
        if (cnt != L[3][(size_t)i]) return LDPCX_E_INVAL;
        entries += cnt;
    }
    long col_entries = 0;
    for (long j = 0; j < N; ++j) {
        std::vector<int> listed;
        for (long v : L[4 + j]) {
            if (v == 0) continue;
            if (v > M) return LDPCX_E_INVAL;
            listed.push_back((int)(v - 1));
        }
        if ((long)listed.size() != L[2][(size_t)j]) return LDPCX_E_INVAL;
        std::vector<int> have = by_col[(size_t)j];
        std::sort(listed.begin(), listed.end());
        std::sort(have.begin(), have.end());
        if (listed != have) return LDPCX_E_INVAL;
        col_entries += (long)listed.size();
    }
    if (col_entries != entries) return LDPCX_E_INVAL;
    const int rows = (int)(M / Z), cols = (int)(N / Z);
    *rows_out = rows;
    *cols_out = cols;
    if (!S_out) return LDPCX_OK;  // size query
    if (capacity < rows * cols) return LDPCX_E_INVAL;
    // every Z x Z block must be zero or a cyclically shifted identity: entry (z, (z + s) mod Z)
    std::vector<int> shift((size_t)rows * cols, -1), count((size_t)rows * cols, 0);
    for (long j = 0; j < N; ++j)
        for (int i : by_col[(size_t)j]) {
            const int br = i / Z, z = i % Z, bc = (int)(j / Z), w = (int)(j % Z);
            const int s = (w - z + Z) % Z;
            const size_t b = (size_t)br * cols + bc;
            if (shift[b] >= 0 && shift[b] != s) return LDPCX_E_INVAL;
            shift[b] = s;
            ++count[b];
        }
    for (size_t b = 0; b < shift.size(); ++b) {
        if (count[b] != 0 && count[b] != Z) return LDPCX_E_INVAL;
        S_out[b] = (int16_t)shift[b];
    }
    return LDPCX_OK;
}

extern "C" int qc_ldpc_alist(ldpcx_code_t c, char *buf, size_t cap, size_t *len_out) {
    if (!c || !len_out) return LDPCX_E_INVAL;
    const int Z = c->Z, R = c->rows, C = c->cols;
    std::vector<int> col_deg(C, 0);
    for (int r = 0; r < R; ++r)
        for (int col = 0; col < C; ++col) col_deg[col] += c->S[(size_t)r * C + col] >= 0;
    const int max_c = *std::max_element(col_deg.begin(), col_deg.end());
    std::string t;
    t.reserve((size_t)c->nnz * Z * 14 + 64);
    auto num = [&](long v, char end) {
        t += std::to_string(v);
        t += end;
    };
    num((long)C * Z, ' ');
    num((long)R * Z, '\n');
    num(max_c, ' ');
    num(c->max_deg, '\n');
    for (int col = 0; col < C; ++col)
        for (int w = 0; w < Z; ++w) num(col_deg[col], col == C - 1 && w == Z - 1 ? '\n' : ' ');
    for (int r = 0; r < R; ++r)
        for (int z = 0; z < Z; ++z) num(c->row_ptr[r + 1] - c->row_ptr[r], r == R - 1 && z == Z - 1 ? '\n' : ' ');
    // variable (col, w): check rows r Z + (w - s) mod Z of the blocks in base column col, ascending
    for (int col = 0; col < C; ++col)
        for (int w = 0; w < Z; ++w) {
            int k = 0;
            for (int r = 0; r < R; ++r) {
                const int s = c->S[(size_t)r * C + col];
                if (s < 0) continue;
                num((long)r * Z + (w - s + Z) % Z + 1, ++k == max_c ? '\n' : ' ');
            }
            for (; k < max_c;) num(0, ++k == max_c ? '\n' : ' ');
        }
    // check (r, z): variables col Z + (z + s) mod Z of the row's blocks, ascending
    for (int r = 0; r < R; ++r)
        for (int z = 0; z < Z; ++z) {
            int k = 0;
            for (int b = c->row_ptr[r]; b < c->row_ptr[r + 1]; ++b) {
                const int col = (int)(c->blk[b] >> 16), s = (int)(c->blk[b] & 0xFFFFu);
                num((long)col * Z + (z + s) % Z + 1, ++k == c->max_deg ? '\n' : ' ');
            }
            for (; k < c->max_deg;) num(0, ++k == c->max_deg ? '\n' : ' ');
        }
    *len_out = t.size();
    if (!buf) return LDPCX_OK;  // size query
    if (cap < t.size() + 1) return LDPCX_E_INVAL;
    memcpy(buf, t.data(), t.size());
    buf[t.size()] = '\0';
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
    info->encodable = c->enc != ldpcx::kEncNone;
    info->n_fill = c->n_fill;
    return LDPCX_OK;
}

extern "C" int qc_ldpc_shorten(ldpcx_code_t code, int k, ldpcx_code_t *out) {
    if (!code || !out) return LDPCX_E_INVAL;
    const int K = code->kb * code->Z;
    if (code->n_fill != 0 || k < code->p0 || k > K || code->p0 + code->n_tx < K) return LDPCX_E_INVAL;
    if (code->n_tx - (K - k) < 1) return LDPCX_E_INVAL;
    ldpcx_code *c = ldpcx::fault_alloc() ? nullptr : new (std::nothrow) ldpcx_code();
    if (!c) return LDPCX_E_NOMEM;
    c->params = code->params;
    c->Z = code->Z;
    c->rows = code->rows;
    c->cols = code->cols;
    c->kb = code->kb;
    c->nnz = code->nnz;
    c->max_deg = code->max_deg;
    c->n = code->n;
    c->p0 = code->p0;
    c->k = k;
    c->n_fill = K - k;
    c->n_tx = code->n_tx - c->n_fill;
    c->S = code->S;
    c->blk = code->blk;
    c->row_ptr = code->row_ptr;
    c->enc = code->enc;
    c->inv_words = code->inv_words;
    c->core_inv = code->core_inv;
    *out = c;  // device tables are uploaded on first use, as for any code
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
        const size_t ni = sizeof(uint32_t) * c->core_inv.size();
        const size_t oi = (nb + nr + 15) / 16 * 16;
        void *p = nullptr;
        if (fault_alloc() || cudaMalloc(&p, oi + ni) != cudaSuccess) {
            cudaGetLastError();
            return LDPCX_E_NOMEM;
        }
        if (cudaMemcpy(p, c->blk.data(), nb, cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy((char *)p + nb, c->row_ptr.data(), nr, cudaMemcpyHostToDevice) != cudaSuccess ||
            (ni && cudaMemcpy((char *)p + oi, c->core_inv.data(), ni, cudaMemcpyHostToDevice) != cudaSuccess)) {
            cudaFree(p);
            return LDPCX_E_CUDA;
        }
        c->d_tables = p;
        c->dev = dev;
        c->d.blk = (const uint32_t *)p;
        c->d.row_ptr = (const int32_t *)((char *)p + nb);
        c->d.core_inv = ni ? (const uint32_t *)((char *)p + oi) : nullptr;
    }
    *out = c->d;
    return LDPCX_OK;
}

namespace {
std::atomic<int> g_fault_kind{-1};  // -1: the environment not read yet
std::atomic<int> g_fault_after{0};
std::once_flag g_fault_env;

void fault_from_env() {
    const char *e = getenv("LDPCX_FAULT");
    int kind = LDPCX_FAULT_NONE, after = 0;
    if (e && strncmp(e, "alloc", 5) == 0 && (e[5] == 0 || (e[5] == ':' && sscanf(e + 6, "%d", &after) == 1))) {
        kind = after >= 0 ? LDPCX_FAULT_ALLOC : LDPCX_FAULT_NONE;
    }
    int expect = -1;
    g_fault_after.store(after < 0 ? 0 : after);
    g_fault_kind.compare_exchange_strong(expect, kind);  // an ldpcx_fault_set before this wins
}
}  // namespace

bool fault_alloc() {
    std::call_once(g_fault_env, fault_from_env);
    if (g_fault_kind.load() != LDPCX_FAULT_ALLOC) return false;
    if (g_fault_after.fetch_sub(1) > 0) return false;
    g_fault_kind.store(LDPCX_FAULT_NONE);  // one shot
    return true;
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

extern "C" int ldpcx_fault_set(int kind, int after) {
    if ((kind != LDPCX_FAULT_NONE && kind != LDPCX_FAULT_ALLOC) || after < 0) return LDPCX_E_INVAL;
    std::call_once(ldpcx::g_fault_env, ldpcx::fault_from_env);
    ldpcx::g_fault_after.store(after);
    ldpcx::g_fault_kind.store(kind);
    return LDPCX_OK;
}
