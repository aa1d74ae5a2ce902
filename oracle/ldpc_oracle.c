/*
 * ldpc_oracle.c -- plain, slow FP64 CPU oracle for the QC-LDPC Monte-Carlo
 * hot path (source -> encoder -> Gray QAM mapper -> AWGN -> APP demapper ->
 * belief-propagation decoder -> error count).
 *
 * TEST INFRASTRUCTURE ONLY. Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / --impl reference legs of bench.py load this library. It shares
 * no code, header, table or constant generator with the CUDA library in
 * paper_2203_11854_gb300/, and neither side includes or links the other.
 *
 * The Sionna white paper (arXiv 2203.11854) names every block on this path --
 * BinarySource, LDPC5GEncoder, Constellation/Mapper, AWGN, Demapper("app"),
 * LDPC5GDecoder ("belief propagation (BP) decoder and variants"), compute_ber
 * (Listing 1 and the feature list of Sec. III-B), and the min-sum BP decoder as
 * a custom CUDA op (Sec. IV-A) -- but prints no equation for any of them. Each
 * function below therefore writes out the textbook definition it cites, step
 * by step, with no blocking, fusion or reordering beyond that definition.
 *
 * Precision: everything is computed in IEEE double. A "prec = 1" switch rounds
 * the result of every arithmetic operation of the min-sum/sum-product updates
 * to binary32 ("FP32 replay"): for +, -, *, / of binary32 operands, computing
 * in binary64 and rounding once to binary32 gives the correctly rounded
 * binary32 result, so the replay equals IEEE binary32 arithmetic in the same
 * operation order. Compile with -ffp-contract=off (no fused multiply-add).
 *
 * Parity pins for every function live in tests/test_oracle_*.py. Functions
 * with no pin other than structural invariants say so in their comment.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

#define ORC_OK 0
#define ORC_E_INVAL (-1)
#define ORC_E_RANK (-2)
#define ORC_E_NOMEM (-3)

/* ------------------------------------------------------------------------- */
/* splitmix64: Steele, Lea & Flood, "Fast splittable pseudorandom number     */
/* generators" (OOPSLA 2014): a Weyl sequence with increment 0x9E3779B97F4A7C15 */
/* followed by the 64-bit finaliser with constants 0xBF58476D1CE4E5B9 and     */
/* 0x94D049BB133111EB and shifts 30, 27, 31.                                  */
/* Pinned by the first outputs of the reference implementation from state 0 */
/* (tests/test_oracle_random.py); the codes it seeds are also pinned         */
/* structurally.                                                              */
/* ------------------------------------------------------------------------- */
static uint64_t sm64_next(uint64_t *state)
{
    uint64_t z;
    *state += 0x9E3779B97F4A7C15ULL;
    z = *state;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* uniform integer in [0, n): next output reduced modulo n */
static uint32_t sm64_below(uint64_t *state, uint32_t n)
{
    return (uint32_t)(sm64_next(state) % (uint64_t)n);
}

uint64_t orc_splitmix64_next(uint64_t *state) { return sm64_next(state); }

/* ------------------------------------------------------------------------- */
/* Seeded BG-shaped base matrix.                                             */
/*                                                                           */
/* The real 3GPP TS 38.212 base graphs are not available, so codes are       */
/* seeded matrices with the 5G-NR shape (the paper's LDPC5GEncoder, Sec.     */
/* III-B): columns [0,Kb) systematic, [Kb,Kb+4) core parity, [Kb+4,cols)     */
/* extension parity.  Core 4x4 parity blocks (shift, -1 = zero):             */
/*   row0 [1 0 - -], row1 [0 0 0 -], row2 [- - 0 0], row3 [1 - - 0]           */
/* whose rows sum to [I 0 0 0] (dual diagonal, invertible).  Extension row j */
/* carries an identity at column Kb+4+j.                                      */
/* Support: core rows draw d_core distinct systematic columns, extension     */
/* rows draw d_ext(j) distinct columns of [0,Kb+4), each by a partial        */
/* Fisher-Yates shuffle driven by splitmix64(seed); then every drawn block,  */
/* in row-major order, gets a shift uniform in [0,Z) from the same stream.    */
/*   BG1: Kb=22, 42 ext rows, d_core=16, d_ext = 5 (j<33) else 4 -> 316 blocks */
/*   BG2: Kb=10, 38 ext rows, d_core=8,  d_ext = 4 (j<4)  else 3 -> 197 blocks */
/* rows_kept (4..M, 0 = all) keeps the first rows and Kb+rows_kept columns.  */
/* dims_out = {rows, cols, Kb}; S_out has room for 46*68 entries.            */
/* ------------------------------------------------------------------------- */
int orc_base_matrix(int bg, int Z, uint64_t seed, int rows_kept, int16_t *S_out, int32_t *dims_out)
{
    int Kb, n_ext, d_core, M, C, r, c, j, i;
    int16_t full[46 * 68];
    int perm[32];
    uint64_t st = seed;
    const int16_t PENDING = -2;

    if (bg == 1) { Kb = 22; n_ext = 42; d_core = 16; }
    else if (bg == 2) { Kb = 10; n_ext = 38; d_core = 8; }
    else return ORC_E_INVAL;
    if (Z < 2 || Z > 32767) return ORC_E_INVAL;
    M = 4 + n_ext;
    C = Kb + M;
    if (rows_kept == 0) rows_kept = M;
    if (rows_kept < 4 || rows_kept > M) return ORC_E_INVAL;

    for (i = 0; i < M * C; ++i) full[i] = -1;

    /* support of the core rows: d_core of the Kb systematic columns */
    for (r = 0; r < 4; ++r) {
        for (i = 0; i < Kb; ++i) perm[i] = i;
        for (i = 0; i < d_core; ++i) {
            int jj = i + (int)sm64_below(&st, (uint32_t)(Kb - i));
            int t = perm[i]; perm[i] = perm[jj]; perm[jj] = t;
            full[r * C + perm[i]] = PENDING;
        }
    }
    /* support of the extension rows: d_ext of the first Kb+4 columns */
    for (j = 0; j < n_ext; ++j) {
        int d_ext = (bg == 1) ? (j < 33 ? 5 : 4) : (j < 4 ? 4 : 3);
        int ncand = Kb + 4;
        for (i = 0; i < ncand; ++i) perm[i] = i;
        for (i = 0; i < d_ext; ++i) {
            int jj = i + (int)sm64_below(&st, (uint32_t)(ncand - i));
            int t = perm[i]; perm[i] = perm[jj]; perm[jj] = t;
            full[(4 + j) * C + perm[i]] = PENDING;
        }
        full[(4 + j) * C + Kb + 4 + j] = 0;
    }
    /* fixed dual-diagonal core */
    full[0 * C + Kb + 0] = 1; full[0 * C + Kb + 1] = 0;
    full[1 * C + Kb + 0] = 0; full[1 * C + Kb + 1] = 0; full[1 * C + Kb + 2] = 0;
    full[2 * C + Kb + 2] = 0; full[2 * C + Kb + 3] = 0;
    full[3 * C + Kb + 0] = 1; full[3 * C + Kb + 3] = 0;
    /* shifts in row-major order */
    for (r = 0; r < M; ++r)
        for (c = 0; c < C; ++c)
            if (full[r * C + c] == PENDING) full[r * C + c] = (int16_t)sm64_below(&st, (uint32_t)Z);

    {
        int cols_kept = Kb + rows_kept;
        for (r = 0; r < rows_kept; ++r)
            for (c = 0; c < cols_kept; ++c) S_out[r * cols_kept + c] = full[r * C + c];
        dims_out[0] = rows_kept;
        dims_out[1] = cols_kept;
        dims_out[2] = Kb;
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* Lifting (QC expansion): block (r,c) with shift s maps check node r*Z+z to  */
/* variable node c*Z + (z+s) mod Z.  Edges are stored check-node-major, each  */
/* check node's edges in ascending base column; check nodes r*Z..r*Z+Z-1 form */
/* layer r.  edge_cls = row-major index of the base block (weight class).     */
/* ------------------------------------------------------------------------- */
int orc_lift(const int16_t *S, int rows, int cols, int Z,
             int32_t *cn_ptr, int32_t *edge_vn, int32_t *edge_cls, int32_t *layer_ptr)
{
    int r, c, z, e = 0;
    int32_t *cls_of = (int32_t *)malloc(sizeof(int32_t) * (size_t)rows * (size_t)cols);
    int ncls = 0;
    if (!cls_of) return ORC_E_NOMEM;
    for (r = 0; r < rows; ++r)
        for (c = 0; c < cols; ++c)
            cls_of[r * cols + c] = (S[r * cols + c] >= 0) ? ncls++ : -1;
    for (r = 0; r < rows; ++r) {
        layer_ptr[r] = r * Z;
        for (z = 0; z < Z; ++z) {
            cn_ptr[r * Z + z] = e;
            for (c = 0; c < cols; ++c) {
                int s = S[r * cols + c];
                if (s < 0) continue;
                edge_vn[e] = c * Z + (z + s) % Z;
                edge_cls[e] = cls_of[r * cols + c];
                ++e;
            }
        }
    }
    cn_ptr[rows * Z] = e;
    layer_ptr[rows] = rows * Z;
    free(cls_of);
    return e;
}

/* ------------------------------------------------------------------------- */
/* Systematic encoder by GF(2) Gauss-Jordan elimination.                      */
/* H = [H_s | H_p] with H_s the k systematic columns; c = [u | p] is a        */
/* codeword iff H_p p = H_s u.  Reduce [H_p | H_s] to [I | A] (row ops over   */
/* GF(2)); then p = A u.  rank(H_p) < n-k is reported as ORC_E_RANK.          */
/* ------------------------------------------------------------------------- */
typedef struct {
    int n, k, m;       /* m = n - k parity bits (= rows of H) */
    int words;         /* 64-bit words per row of [I | A] */
    uint64_t *rows;    /* m rows; column j<m is parity j, column m+i is info bit i */
} orc_encoder;

static inline int bit_get(const uint64_t *row, int j) { return (int)((row[j >> 6] >> (j & 63)) & 1u); }
static inline void bit_flip(uint64_t *row, int j) { row[j >> 6] ^= (uint64_t)1 << (j & 63); }

void *orc_enc_prepare(const int16_t *S, int rows, int cols, int Kb, int Z, int32_t *status)
{
    orc_encoder *enc = (orc_encoder *)calloc(1, sizeof(orc_encoder));
    int r, c, z, piv;
    if (!enc) { *status = ORC_E_NOMEM; return NULL; }
    enc->n = cols * Z;
    enc->k = Kb * Z;
    enc->m = rows * Z;
    if (enc->m != enc->n - enc->k) { free(enc); *status = ORC_E_INVAL; return NULL; }
    enc->words = (enc->n + 63) / 64;
    enc->rows = (uint64_t *)calloc((size_t)enc->m * (size_t)enc->words, sizeof(uint64_t));
    if (!enc->rows) { free(enc); *status = ORC_E_NOMEM; return NULL; }
    /* column reorder: codeword position v < k (systematic) -> m + v; v >= k -> v - k */
    for (r = 0; r < rows; ++r)
        for (z = 0; z < Z; ++z) {
            uint64_t *row = enc->rows + (size_t)(r * Z + z) * (size_t)enc->words;
            for (c = 0; c < cols; ++c) {
                int s = S[r * cols + c], v, col;
                if (s < 0) continue;
                v = c * Z + (z + s) % Z;
                col = (v < enc->k) ? enc->m + v : v - enc->k;
                bit_flip(row, col);
            }
        }
    /* Gauss-Jordan on the first m columns */
    for (piv = 0; piv < enc->m; ++piv) {
        int found = -1, i, w;
        uint64_t *prow;
        for (i = piv; i < enc->m; ++i)
            if (bit_get(enc->rows + (size_t)i * enc->words, piv)) { found = i; break; }
        if (found < 0) {
            free(enc->rows); free(enc);
            *status = ORC_E_RANK;
            return NULL;
        }
        if (found != piv) {
            uint64_t *a = enc->rows + (size_t)found * enc->words, *b = enc->rows + (size_t)piv * enc->words;
            for (w = 0; w < enc->words; ++w) { uint64_t t = a[w]; a[w] = b[w]; b[w] = t; }
        }
        prow = enc->rows + (size_t)piv * enc->words;
        for (i = 0; i < enc->m; ++i) {
            uint64_t *row;
            if (i == piv) continue;
            row = enc->rows + (size_t)i * enc->words;
            if (bit_get(row, piv))
                for (w = piv >> 6; w < enc->words; ++w) row[w] ^= prow[w];
        }
    }
    *status = ORC_OK;
    return enc;
}

void orc_enc_free(void *h)
{
    orc_encoder *enc = (orc_encoder *)h;
    if (!enc) return;
    free(enc->rows);
    free(enc);
}

/* u: [B][k] bits (0/1 bytes); c: [B][n] bits. c = [u | A u]. */
int orc_enc_encode(const void *h, const uint8_t *u, int64_t B, uint8_t *cw)
{
    const orc_encoder *enc = (const orc_encoder *)h;
    int64_t b;
    uint64_t *ubits;
    if (!enc) return ORC_E_INVAL;
    ubits = (uint64_t *)calloc((size_t)enc->words, sizeof(uint64_t));
    if (!ubits) return ORC_E_NOMEM;
    for (b = 0; b < B; ++b) {
        const uint8_t *ub = u + b * enc->k;
        uint8_t *cb = cw + b * enc->n;
        int i, w;
        memset(ubits, 0, sizeof(uint64_t) * (size_t)enc->words);
        for (i = 0; i < enc->k; ++i) {
            cb[i] = ub[i] & 1u;
            if (cb[i]) bit_flip(ubits, enc->m + i);
        }
        for (i = 0; i < enc->m; ++i) {
            const uint64_t *row = enc->rows + (size_t)i * enc->words;
            uint64_t acc = 0;
            for (w = 0; w < enc->words; ++w) acc ^= row[w] & ubits[w];
            cb[enc->k + i] = (uint8_t)__builtin_parityll(acc);
        }
    }
    free(ubits);
    return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* Philox4x32-10: Salmon, Moraes, Dror & Shaw, "Parallel random numbers: as   */
/* easy as 1, 2, 3" (SC'11).  Round: (hi0,lo0) = M0*c0, (hi1,lo1) = M1*c2,    */
/* c' = (hi1^c1^k0, lo1, hi0^c3^k1, lo0) with M0 = 0xD2511F53, M1 = 0xCD9E8D57;*/
/* the key is bumped by (0x9E3779B9, 0xBB67AE85) between rounds; 10 rounds.   */
/* ------------------------------------------------------------------------- */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    int round;
    for (round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0, n1 = lo1, n2 = hi0 ^ c3 ^ k1, n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        if (round < 9) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

void orc_philox_many(int64_t count, const uint32_t *ctr /*[count][4]*/, const uint32_t key[2], uint32_t *out)
{
    int64_t i;
    for (i = 0; i < count; ++i) orc_philox4x32_10(ctr + 4 * i, key, out + 4 * i);
}

/* counter layout shared by every random draw of the simulation:
 * (block index q, codeword index low 32, codeword index high 32, stream id);
 * key = (seed low 32, seed high 32).  Stream 0: source bits; stream 1: noise. */
static void philox_block(uint64_t seed, uint64_t cw, uint32_t stream, uint32_t q, uint32_t out[4])
{
    uint32_t ctr[4] = { q, (uint32_t)cw, (uint32_t)(cw >> 32), stream };
    uint32_t key[2] = { (uint32_t)seed, (uint32_t)(seed >> 32) };
    orc_philox4x32_10(ctr, key, out);
}

/* BinarySource (Listing 1): info bit j of codeword cw = bit (j mod 32) of word
 * (j mod 128)/32 of Philox block j/128 on stream 0. u: [B][k] bytes. */
void orc_source_bits(uint64_t seed, uint64_t cw0, int64_t B, int k, uint8_t *u)
{
    int64_t b;
    for (b = 0; b < B; ++b) {
        uint32_t blk[4];
        int j;
        for (j = 0; j < k; ++j) {
            if ((j & 127) == 0) philox_block(seed, cw0 + (uint64_t)b, 0u, (uint32_t)(j >> 7), blk);
            u[b * k + j] = (uint8_t)((blk[(j & 127) >> 5] >> (j & 31)) & 1u);
        }
    }
}

/* ------------------------------------------------------------------------- */
/* Gray square QAM (Constellation("qam", m) / Mapper, Listing 1).             */
/* m = 1: BPSK x = 1 - 2b (real).  m = 2h: bits b0,b2,... go to I and         */
/* b1,b3,... to Q; per dimension the level of bits (a0..a_{h-1}) is           */
/*   A = (1-2a0) (2^{h-1} - (1-2a1) (2^{h-2} - ... - (1-2a_{h-1}) ))          */
/* (the reflected Gray labelling of 3GPP TS 38.211 Sec. 5.1), scaled by       */
/* 1/sqrt(2 (4^h - 1)/3) so that the average symbol energy is 1.              */
/* ------------------------------------------------------------------------- */
static double pam_level(const uint8_t *a, int h)
{
    /* evaluate from the innermost term outwards */
    double inner = (double)(1 - 2 * (int)a[h - 1]);
    int i;
    for (i = h - 2; i >= 0; --i) inner = (double)(1 - 2 * (int)a[i]) * ((double)(1 << (h - 1 - i)) - inner);
    return inner;
}

double orc_qam_scale(int m)
{
    int h = m / 2;
    if (m == 1) return 1.0;
    return 1.0 / sqrt(2.0 * (double)((1 << (2 * h)) - 1) / 3.0);
}

/* bits: [B][n] codeword bits; the transmitted bits are positions
 * [p0, p0 + n_tx) (punctured/truncated positions are not sent).
 * x: m = 1 -> [B][n_tx] real; else [B][n_tx/m][2] (re, im). */
int orc_map(const uint8_t *bits, int n, int p0, int n_tx, int m, int64_t B, double *x)
{
    int64_t b;
    int S, s, i, h = m / 2;
    double sc = orc_qam_scale(m);
    if (m != 1 && (m < 2 || m > 8 || (m & 1))) return ORC_E_INVAL;
    if (n_tx % m != 0 || p0 + n_tx > n) return ORC_E_INVAL;
    S = n_tx / m;
    for (b = 0; b < B; ++b) {
        const uint8_t *cb = bits + b * n + p0;
        for (s = 0; s < S; ++s) {
            if (m == 1) {
                x[b * S + s] = 1.0 - 2.0 * (double)cb[s];
            } else {
                uint8_t aI[4], aQ[4];
                for (i = 0; i < h; ++i) { aI[i] = cb[s * m + 2 * i]; aQ[i] = cb[s * m + 2 * i + 1]; }
                x[(b * S + s) * 2 + 0] = sc * pam_level(aI, h);
                x[(b * S + s) * 2 + 1] = sc * pam_level(aQ, h);
            }
        }
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* AWGN (AWGN()([x, no]), Listing 1): y = x + sqrt(N0/2) g per real dimension.*/
/* g by Box-Muller (Box & Muller 1958) on Philox stream 1: block q gives       */
/* (x0,x1,x2,x3); u1 = ((x0>>9)+0.5) 2^-23 in (0,1), u2 = (x1>>8) 2^-24 in     */
/* [0,1) -- both exact binary32 numbers, so every side draws the same pair --  */
/* g[4q] = r cos(2 pi u2), g[4q+1] = r sin(2 pi u2) with r = sqrt(-2 ln u1),  */
/* and likewise (x2,x3) -> g[4q+2], g[4q+3].  Complex symbol s takes          */
/* (g[2s], g[2s+1]); real symbol s takes g[s].                                 */
/* ------------------------------------------------------------------------- */
void orc_gauss_pair(uint32_t a, uint32_t b, double *g0, double *g1)
{
    double u1 = ((double)(a >> 9) + 0.5) * (1.0 / 8388608.0);
    double u2 = (double)(b >> 8) * (1.0 / 16777216.0);
    double r = sqrt(-2.0 * log(u1));
    double th = 2.0 * M_PI * u2;
    *g0 = r * cos(th);
    *g1 = r * sin(th);
}

/* N0 per codeword: N0[b]; x,y as in orc_map. */
void orc_awgn(const double *x, int64_t B, int S, int m, const double *N0, uint64_t seed, uint64_t cw0, double *y)
{
    int64_t b;
    int dims = (m == 1) ? 1 : 2;
    int G = S * dims; /* Gaussians per codeword */
    for (b = 0; b < B; ++b) {
        double sd = sqrt(N0[b] / 2.0);
        int i;
        uint32_t blk[4];
        double g[4];
        for (i = 0; i < G; ++i) {
            if ((i & 3) == 0) {
                philox_block(seed, cw0 + (uint64_t)b, 1u, (uint32_t)(i >> 2), blk);
                orc_gauss_pair(blk[0], blk[1], &g[0], &g[1]);
                orc_gauss_pair(blk[2], blk[3], &g[2], &g[3]);
            }
            y[b * G + i] = x[b * G + i] + sd * g[i & 3];
        }
    }
}

/* N0 = 1 / (r m 10^(EbN0/10)) with r = k / n_tx (information bits per
 * transmitted bit) and unit symbol energy. */
double orc_n0_from_ebn0(double ebn0_db, int k, int n_tx, int m)
{
    double r = (double)k / (double)n_tx;
    return 1.0 / (r * (double)m * pow(10.0, ebn0_db / 10.0));
}

/* ------------------------------------------------------------------------- */
/* APP demapper (Demapper("app"), Listing 1): with L = ln P(b=0|y)/P(b=1|y),   */
/*   L_i = ln sum_{x: b_i(x)=0} exp(-|y-x|^2/N0) - ln sum_{x: b_i(x)=1} exp(.) */
/* over all 2^m constellation points (the full 2-D sum, no separability        */
/* shortcut).  method 0 = exact (max-shifted log-sum-exp), 1 = max-log (each   */
/* log-sum-exp replaced by its largest term).  BPSK uses the real channel,     */
/* |y-x|^2 = (y-x)^2.  The result is clamped to [-clamp, clamp].              */
/* ------------------------------------------------------------------------- */
static double lse_or_max(const double *v, int cnt, int method)
{
    double mx = -INFINITY, acc = 0.0;
    int i;
    for (i = 0; i < cnt; ++i) if (v[i] > mx) mx = v[i];
    if (method == 1) return mx;
    for (i = 0; i < cnt; ++i) acc += exp(v[i] - mx);
    return mx + log(acc);
}

int orc_demap(const double *y, int64_t B, int S, int m, const double *N0, int method, double clamp, double *llr)
{
    int64_t b;
    int P = 1 << m, h = m / 2, s, i, p;
    double pts_re[256], pts_im[256];
    uint8_t lab[256][8];
    double sc = orc_qam_scale(m);
    if (m != 1 && (m < 2 || m > 8 || (m & 1))) return ORC_E_INVAL;
    /* enumerate the constellation with its labels: label bits (MSB-first index) */
    for (p = 0; p < P; ++p) {
        uint8_t bits[8], aI[4], aQ[4];
        for (i = 0; i < m; ++i) bits[i] = (uint8_t)((p >> (m - 1 - i)) & 1);
        for (i = 0; i < m; ++i) lab[p][i] = bits[i];
        if (m == 1) { pts_re[p] = 1.0 - 2.0 * bits[0]; pts_im[p] = 0.0; continue; }
        for (i = 0; i < h; ++i) { aI[i] = bits[2 * i]; aQ[i] = bits[2 * i + 1]; }
        pts_re[p] = sc * pam_level(aI, h);
        pts_im[p] = sc * pam_level(aQ, h);
    }
    for (b = 0; b < B; ++b) {
        for (s = 0; s < S; ++s) {
            double yr, yi, metric[256], v0[128], v1[128];
            if (m == 1) { yr = y[b * S + s]; yi = 0.0; }
            else { yr = y[(b * S + s) * 2]; yi = y[(b * S + s) * 2 + 1]; }
            for (p = 0; p < P; ++p) {
                double dr = yr - pts_re[p], di = yi - pts_im[p];
                metric[p] = -(dr * dr + di * di) / N0[b];
            }
            for (i = 0; i < m; ++i) {
                int c0 = 0, c1 = 0;
                double L;
                for (p = 0; p < P; ++p) {
                    if (lab[p][i]) v1[c1++] = metric[p];
                    else v0[c0++] = metric[p];
                }
                L = lse_or_max(v0, c0, method) - lse_or_max(v1, c1, method);
                if (L > clamp) L = clamp;
                if (L < -clamp) L = -clamp;
                llr[(b * S + s) * m + i] = L;
            }
        }
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* Demapper with prior (feature list of Section III: "Demapper with prior").  */
/* With a-priori LLRs La_j = ln P(b_j=0)/P(b_j=1), the prior of point x is     */
/* prod_j P(b_j(x)), and ln P(b_j) = (1 - 2 b_j) La_j / 2 - ln(e^{La_j/2} +    */
/* e^{-La_j/2}); the normaliser is the same for every x and cancels. So       */
/*   APP_i = ln sum_{x: b_i=0} exp(m(x)) - ln sum_{x: b_i=1} exp(m(x)),        */
/*   m(x) = -|y-x|^2/N0 + sum_j (1 - 2 b_j(x)) La_j / 2,                       */
/* and the extrinsic value is the same ratio with the j = i term left out of  */
/* m(x) (computed as such here, not as APP_i - La_i).  Full 2-D sums over the */
/* 2^m points; max-log replaces each log-sum-exp by its largest term.         */
/* prior: [B][S*m] (NULL = zero); mode 0 = APP, 1 = extrinsic.                */
/* ------------------------------------------------------------------------- */
int orc_demap_prior(const double *y, int64_t B, int S, int m, const double *N0, int method, double clamp,
                    const double *prior, int mode, double *llr)
{
    int64_t b;
    int P = 1 << m, h = m / 2, s, i, j, p;
    double pts_re[256], pts_im[256];
    uint8_t lab[256][8];
    double sc = orc_qam_scale(m);
    if (m != 1 && (m < 2 || m > 8 || (m & 1))) return ORC_E_INVAL;
    if (mode != 0 && mode != 1) return ORC_E_INVAL;
    for (p = 0; p < P; ++p) {
        uint8_t bits[8], aI[4], aQ[4];
        for (i = 0; i < m; ++i) bits[i] = (uint8_t)((p >> (m - 1 - i)) & 1);
        for (i = 0; i < m; ++i) lab[p][i] = bits[i];
        if (m == 1) { pts_re[p] = 1.0 - 2.0 * bits[0]; pts_im[p] = 0.0; continue; }
        for (i = 0; i < h; ++i) { aI[i] = bits[2 * i]; aQ[i] = bits[2 * i + 1]; }
        pts_re[p] = sc * pam_level(aI, h);
        pts_im[p] = sc * pam_level(aQ, h);
    }
    for (b = 0; b < B; ++b) {
        for (s = 0; s < S; ++s) {
            double yr, yi, dist[256], v0[128], v1[128];
            const double *la = prior ? prior + (b * S + s) * m : NULL;
            if (m == 1) { yr = y[b * S + s]; yi = 0.0; }
            else { yr = y[(b * S + s) * 2]; yi = y[(b * S + s) * 2 + 1]; }
            for (p = 0; p < P; ++p) {
                double dr = yr - pts_re[p], di = yi - pts_im[p];
                dist[p] = -(dr * dr + di * di) / N0[b];
            }
            for (i = 0; i < m; ++i) {
                int c0 = 0, c1 = 0;
                double L;
                for (p = 0; p < P; ++p) {
                    double mt = dist[p];
                    for (j = 0; j < m; ++j) {
                        if (!la || (mode == 1 && j == i)) continue;
                        mt += (lab[p][j] ? -0.5 : 0.5) * la[j];
                    }
                    if (lab[p][i]) v1[c1++] = mt;
                    else v0[c0++] = mt;
                }
                L = lse_or_max(v0, c0, method) - lse_or_max(v1, c1, method);
                if (L > clamp) L = clamp;
                if (L < -clamp) L = -clamp;
                llr[(b * S + s) * m + i] = L;
            }
        }
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* APP demapper over an arbitrary constellation (Listing 2's trainable        */
/* Constellation with the Demapper): point l = (pr[l], pi[l]) carries label  */
/* bits b_j = (l >> (m-1-j)) & 1, and                                        */
/*   L_i = ln sum_{l: b_i=0} exp(-|y-p_l|^2/N0) - ln sum_{l: b_i=1} exp(.)   */
/* over all 2^m points (method 1: max-log).  y: [B][S][2]; out [B][S*m].     */
/* ------------------------------------------------------------------------- */
int orc_demap_points(const double *y, int64_t B, int S, int m, const double *N0, const double *pts, int method,
                     double clamp, double *llr)
{
    int64_t b;
    int P = 1 << m, s, i, p;
    if (m < 1 || m > 8) return ORC_E_INVAL;
    for (b = 0; b < B; ++b) {
        for (s = 0; s < S; ++s) {
            double yr = y[(b * S + s) * 2], yi = y[(b * S + s) * 2 + 1], metric[256], v0[128], v1[128];
            for (p = 0; p < P; ++p) {
                double dr = yr - pts[2 * p], di = yi - pts[2 * p + 1];
                metric[p] = -(dr * dr + di * di) / N0[b];
            }
            for (i = 0; i < m; ++i) {
                int c0 = 0, c1 = 0;
                double L;
                for (p = 0; p < P; ++p) {
                    if ((p >> (m - 1 - i)) & 1) v1[c1++] = metric[p];
                    else v0[c0++] = metric[p];
                }
                L = lse_or_max(v0, c0, method) - lse_or_max(v1, c1, method);
                if (L > clamp) L = clamp;
                if (L < -clamp) L = -clamp;
                llr[(b * S + s) * m + i] = L;
            }
        }
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* A-priori LLRs of the consistent Gaussian model used for EXIT charts (ten   */
/* Brink, IEEE Trans. Commun. 2001): L = (sigma^2/2)(1 - 2c) + sigma g, g     */
/* standard Gaussian by Box-Muller on Philox stream 2, block t/4, pairs       */
/* (x0,x1) -> g[4q], g[4q+1] and (x2,x3) -> g[4q+2], g[4q+3] as orc_awgn.      */
/* bits: [B][N] unpacked reference bits; out: [B][N].                          */
/* ------------------------------------------------------------------------- */
void orc_apriori(const uint8_t *bits, int64_t B, int64_t N, double sigma, uint64_t seed, uint64_t cw0, double *out)
{
    int64_t b, t;
    double mu = 0.5 * sigma * sigma;
    for (b = 0; b < B; ++b) {
        uint32_t blk[4];
        double g[4];
        for (t = 0; t < N; ++t) {
            if ((t & 3) == 0) {
                philox_block(seed, cw0 + (uint64_t)b, 2u, (uint32_t)(t >> 2), blk);
                orc_gauss_pair(blk[0], blk[1], &g[0], &g[1]);
                orc_gauss_pair(blk[2], blk[3], &g[2], &g[3]);
            }
            out[b * N + t] = (bits[b * N + t] ? -mu : mu) + sigma * g[t & 3];
        }
    }
}

/* Puncturing / truncation: the decoder input has n positions; position v gets
 * the transmitted LLR v - p0 when p0 <= v < p0 + n_tx, else 0 (no information). */
void orc_place_llr(const double *llr_tx, int64_t B, int n_tx, int p0, int n, double *llr)
{
    int64_t b;
    int v;
    for (b = 0; b < B; ++b)
        for (v = 0; v < n; ++v)
            llr[b * n + v] = (v >= p0 && v < p0 + n_tx) ? llr_tx[b * n_tx + (v - p0)] : 0.0;
}

/* ------------------------------------------------------------------------- */
/* Belief-propagation decoding on a Tanner graph (LDPC5GDecoder, Sec. III-B;  */
/* min-sum as the custom CUDA op of Sec. IV-A).                               */
/*                                                                           */
/* Messages: R = check-to-variable (C2V).  LLR convention L = ln P0/P1.        */
/* Check-node rules for the incoming variable-to-check messages T_i:          */
/*  offset min-sum: R_j = sgn_j s max(min_{i!=j} |T_i| - beta, 0),            */
/*     min_{i!=j} taken as m2 at the first index of the smallest |T| and m1   */
/*     elsewhere (m2 = m1 on ties), s = prod sgn(T_i), sgn(x) = -1 iff x < 0.  */
/*  sum-product: R_j = sgn_j s phi(sum_{i!=j} phi(|T_i|)),                    */
/*     phi(x) = -ln tanh(x/2) = ln(1 + 2/(e^x - 1)), every phi argument       */
/*     clamped to [phi(clamp), clamp].                                        */
/*  |R| <= clamp.  The stored message is then rounded: store 1 = binary16     */
/*  round-to-nearest-even, store 2 = 6-bit fixed point (step 0.5, saturated   */
/*  to +-31 steps, round-to-nearest-even).  The rounded value is both stored  */
/*  and added to the variable node.                                           */
/* Layered schedule (layer = base row, ascending; check nodes of a layer are */
/* independent): T = APP - R_old; CN rule; APP = T + R_new.                  */
/* Flooding schedule: V2C = w_{t,cls} (APP_old - R_old); CN rule for every   */
/* check node; APP_new = L + sum of the new R over the variable's check nodes,*/
/* added in ascending check-node order.                                       */
/* Early stop: after each full iteration, stop when the hard decisions       */
/* (bit = 1 iff APP < 0) satisfy every parity check; the iteration count is  */
/* the number of full iterations run.  Channel LLRs are clamped to +-clamp;   */
/* the APP itself is never clamped.                                           */
/* ------------------------------------------------------------------------- */
typedef struct {
    int n, m, E, n_layers, n_cls;
    const int32_t *cn_ptr, *edge_vn, *edge_cls, *layer_ptr;
} orc_graph;

typedef struct {
    int algo, schedule, iters, prec, store, early_stop;
    double offset, clamp;
    const double *weights; /* [iters][n_cls] or NULL */
} orc_opts;

static inline double rnd(int prec, double x) { return prec ? (double)(float)x : x; }

double orc_to_half(double x)
{
    double a, q, r;
    int e, lead;
    if (x == 0.0 || !isfinite(x)) return x;
    a = fabs(x);
    frexp(a, &e);          /* a = f 2^e, f in [0.5, 1): leading bit 2^(e-1) */
    lead = e - 1;
    if (lead < -14) lead = -14; /* subnormal binary16 spacing is 2^-24 */
    q = ldexp(1.0, lead - 10);  /* 10 fraction bits */
    r = nearbyint(a / q) * q;   /* default rounding mode: to nearest, ties to even */
    if (r > 65504.0) r = INFINITY;
    return copysign(r, x);
}

double orc_to_fix6(double x)
{
    double q = nearbyint(x / 0.5);
    if (q > 31.0) q = 31.0;
    if (q < -31.0) q = -31.0;
    return (double)(int)q * 0.5; /* integer storage carries no negative zero */
}

static inline double store_msg(int store, double r)
{
    if (store == 1) return orc_to_half(r);
    if (store == 2) return orc_to_fix6(r);
    return r;
}

double orc_phi(double x) { return log1p(2.0 / expm1(x)); }

/* check-node rule on d inputs T[0..d-1] -> R[0..d-1] */
static void cn_rule(const orc_opts *o, int d, const double *T, double *R, double *scratch)
{
    int j, i, neg_all = 0;
    for (j = 0; j < d; ++j) if (T[j] < 0.0) neg_all ^= 1;
    if (o->algo == 0) {
        double m1 = INFINITY, m2 = INFINITY;
        int idx = -1;
        for (j = 0; j < d; ++j) {
            double a = fabs(T[j]);
            if (a < m1) { m2 = m1; m1 = a; idx = j; }
            else if (a < m2) m2 = a;
        }
        for (j = 0; j < d; ++j) {
            double mag = (j == idx) ? m2 : m1;
            int neg = neg_all ^ (T[j] < 0.0);
            mag = rnd(o->prec, mag - o->offset);
            if (mag < 0.0) mag = 0.0;
            if (mag > o->clamp) mag = o->clamp;
            R[j] = neg ? -mag : mag;
        }
    } else {
        double lo = orc_phi(o->clamp);
        double *f = scratch;
        for (i = 0; i < d; ++i) {
            double a = fabs(T[i]);
            if (a < lo) a = lo;
            if (a > o->clamp) a = o->clamp;
            f[i] = rnd(o->prec, orc_phi(a));
        }
        for (j = 0; j < d; ++j) {
            double sum = 0.0, mag;
            int neg = neg_all ^ (T[j] < 0.0);
            for (i = 0; i < d; ++i) if (i != j) sum = rnd(o->prec, sum + f[i]);
            if (sum < lo) sum = lo;
            if (sum > o->clamp) sum = o->clamp;
            mag = rnd(o->prec, orc_phi(sum));
            if (mag > o->clamp) mag = o->clamp;
            R[j] = neg ? -mag : mag;
        }
    }
}

static int syndrome_ok(const orc_graph *g, const double *app)
{
    int c, e;
    for (c = 0; c < g->m; ++c) {
        int par = 0;
        for (e = g->cn_ptr[c]; e < g->cn_ptr[c + 1]; ++e) par ^= (app[g->edge_vn[e]] < 0.0);
        if (par) return 0;
    }
    return 1;
}

static int max_degree(const orc_graph *g)
{
    int c, d = 0;
    for (c = 0; c < g->m; ++c) if (g->cn_ptr[c + 1] - g->cn_ptr[c] > d) d = g->cn_ptr[c + 1] - g->cn_ptr[c];
    return d;
}

/* one codeword; llr: [n] channel LLRs (already placed); app_out: [n] */
static int decode_one(const orc_graph *g, const orc_opts *o, const double *llr, double *app_out, int32_t *iters_out)
{
    int n = g->n, E = g->E, dmax = max_degree(g);
    double *L = (double *)malloc(sizeof(double) * (size_t)n);
    double *app = (double *)malloc(sizeof(double) * (size_t)n);
    double *app_new = (double *)malloc(sizeof(double) * (size_t)n);
    double *R = (double *)calloc((size_t)E, sizeof(double));
    double *T = (double *)malloc(sizeof(double) * (size_t)(dmax + 1));
    double *Rn = (double *)malloc(sizeof(double) * (size_t)(dmax + 1));
    double *scr = (double *)malloc(sizeof(double) * (size_t)(dmax + 1));
    int v, t, done = 0, it_run = 0;
    if (!L || !app || !app_new || !R || !T || !Rn || !scr) {
        free(L); free(app); free(app_new); free(R); free(T); free(Rn); free(scr);
        return ORC_E_NOMEM;
    }
    for (v = 0; v < n; ++v) {
        double x = llr[v];
        if (o->prec) x = (double)(float)x;
        if (x > o->clamp) x = o->clamp;
        if (x < -o->clamp) x = -o->clamp;
        L[v] = x;
        app[v] = x;
    }
    for (t = 0; t < o->iters && !done; ++t) {
        if (o->schedule == 0) {
            int l, c, e;
            for (l = 0; l < g->n_layers; ++l)
                for (c = g->layer_ptr[l]; c < g->layer_ptr[l + 1]; ++c) {
                    int e0 = g->cn_ptr[c], d = g->cn_ptr[c + 1] - e0;
                    for (e = 0; e < d; ++e) T[e] = rnd(o->prec, app[g->edge_vn[e0 + e]] - R[e0 + e]);
                    cn_rule(o, d, T, Rn, scr);
                    for (e = 0; e < d; ++e) {
                        double r = store_msg(o->store, Rn[e]);
                        R[e0 + e] = r;
                        app[g->edge_vn[e0 + e]] = rnd(o->prec, T[e] + r);
                    }
                }
        } else {
            int c, e;
            for (v = 0; v < n; ++v) app_new[v] = L[v];
            for (c = 0; c < g->m; ++c) {
                int e0 = g->cn_ptr[c], d = g->cn_ptr[c + 1] - e0;
                for (e = 0; e < d; ++e) {
                    double vm = rnd(o->prec, app[g->edge_vn[e0 + e]] - R[e0 + e]);
                    if (o->weights) vm = rnd(o->prec, o->weights[(size_t)t * g->n_cls + g->edge_cls[e0 + e]] * vm);
                    T[e] = vm;
                }
                cn_rule(o, d, T, Rn, scr);
                for (e = 0; e < d; ++e) {
                    double r = store_msg(o->store, Rn[e]);
                    int vv = g->edge_vn[e0 + e];
                    R[e0 + e] = r;
                    app_new[vv] = rnd(o->prec, app_new[vv] + r);
                }
            }
            memcpy(app, app_new, sizeof(double) * (size_t)n);
        }
        it_run = t + 1;
        if (o->early_stop && syndrome_ok(g, app)) done = 1;
    }
    memcpy(app_out, app, sizeof(double) * (size_t)n);
    *iters_out = it_run;
    free(L); free(app); free(app_new); free(R); free(T); free(Rn); free(scr);
    return ORC_OK;
}

typedef struct {
    const orc_graph *g;
    const orc_opts *o;
    const double *llr;
    double *app;
    uint8_t *hard;
    int32_t *iters;
    int64_t b0, b1;
    int status;
} dec_job;

static void *dec_worker(void *arg)
{
    dec_job *jb = (dec_job *)arg;
    int64_t b;
    int n = jb->g->n;
    for (b = jb->b0; b < jb->b1; ++b) {
        int v, st = decode_one(jb->g, jb->o, jb->llr + b * n, jb->app + b * n, jb->iters + b);
        if (st) { jb->status = st; return NULL; }
        if (jb->hard)
            for (v = 0; v < n; ++v) jb->hard[b * n + v] = (uint8_t)(jb->app[b * n + v] < 0.0);
    }
    return NULL;
}

/* Decode B codewords (threads only split the batch; results do not depend on nthreads). */
int orc_decode(int n, int m, int E, int n_layers, int n_cls,
               const int32_t *cn_ptr, const int32_t *edge_vn, const int32_t *edge_cls, const int32_t *layer_ptr,
               int algo, int schedule, int iters, int prec, int store, int early_stop,
               double offset, double clamp, const double *weights,
               const double *llr, int64_t B, double *app_out, uint8_t *hard_out, int32_t *iters_out, int nthreads)
{
    orc_graph g = { n, m, E, n_layers, n_cls, cn_ptr, edge_vn, edge_cls, layer_ptr };
    orc_opts o = { algo, schedule, iters, prec, store, early_stop, offset, clamp, weights };
    dec_job jobs[256];
    pthread_t th[256];
    int t, status = ORC_OK;
    if (algo < 0 || algo > 1 || schedule < 0 || schedule > 1 || iters < 1 || store < 0 || store > 2)
        return ORC_E_INVAL;
    if (weights && schedule != 1) return ORC_E_INVAL;
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    if ((int64_t)nthreads > B) nthreads = (int)(B > 0 ? B : 1);
    for (t = 0; t < nthreads; ++t) {
        jobs[t].g = &g; jobs[t].o = &o; jobs[t].llr = llr; jobs[t].app = app_out;
        jobs[t].hard = hard_out; jobs[t].iters = iters_out; jobs[t].status = ORC_OK;
        jobs[t].b0 = B * t / nthreads;
        jobs[t].b1 = B * (t + 1) / nthreads;
    }
    if (nthreads == 1) dec_worker(&jobs[0]);
    else {
        for (t = 0; t < nthreads; ++t) pthread_create(&th[t], NULL, dec_worker, &jobs[t]);
        for (t = 0; t < nthreads; ++t) pthread_join(th[t], NULL);
    }
    for (t = 0; t < nthreads; ++t) if (jobs[t].status) status = jobs[t].status;
    return status;
}

/* ------------------------------------------------------------------------- */
/* Bitwise MAP by enumeration (the exact result BP approximates): for a code  */
/* given by a dense parity-check matrix H [m][n] (n <= 24),                   */
/*   APP_v = ln sum_{c: Hc=0, c_v=0} exp(-sum_i c_i L_i)                      */
/*         - ln sum_{c: Hc=0, c_v=1} exp(-sum_i c_i L_i),                     */
/* since P(c | y) is proportional to prod_i exp(-c_i L_i) for L = ln P0/P1.   */
/* ------------------------------------------------------------------------- */
int orc_bitwise_map(const uint8_t *H, int m, int n, const double *L, double *app)
{
    uint32_t c, total = 1u << n;
    double *w0 = (double *)calloc((size_t)n, sizeof(double));
    double *w1 = (double *)calloc((size_t)n, sizeof(double));
    double *mets = (double *)malloc(sizeof(double) * total);
    uint8_t *valid = (uint8_t *)malloc(total);
    double mx = -INFINITY;
    int v, r;
    if (n > 24 || !w0 || !w1 || !mets || !valid) { free(w0); free(w1); free(mets); free(valid); return ORC_E_INVAL; }
    for (c = 0; c < total; ++c) {
        int ok = 1;
        double met = 0.0;
        for (r = 0; r < m && ok; ++r) {
            int par = 0;
            for (v = 0; v < n; ++v) par ^= H[r * n + v] & (int)((c >> v) & 1u);
            if (par) ok = 0;
        }
        valid[c] = (uint8_t)ok;
        if (!ok) continue;
        for (v = 0; v < n; ++v) if ((c >> v) & 1u) met -= L[v];
        mets[c] = met;
        if (met > mx) mx = met;
    }
    for (c = 0; c < total; ++c) {
        double w;
        if (!valid[c]) continue;
        w = exp(mets[c] - mx);
        for (v = 0; v < n; ++v) {
            if ((c >> v) & 1u) w1[v] += w;
            else w0[v] += w;
        }
    }
    for (v = 0; v < n; ++v) app[v] = log(w0[v]) - log(w1[v]);
    free(w0); free(w1); free(mets); free(valid);
    return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* The whole Monte-Carlo chain for codewords [cw0, cw0+B) (Listing 1):        */
/* source -> encode -> map -> AWGN -> APP demap -> place -> decode -> count.  */
/* counts[5] += {info bits, bit errors, blocks, block errors, iterations}.    */
/* Bit errors are counted over the k information bits (punctured ones        */
/* included); a block error is any information-bit error (compute_ber).       */
/* ------------------------------------------------------------------------- */
typedef struct {
    const void *enc;
    const orc_graph *g;
    const orc_opts *o;
    uint64_t seed, cw0;
    int64_t B;
    int k, n, p0, n_tx, m, demap_method;
    double N0, demap_clamp;
    int64_t counts[5];
    int status;
} sim_job;

static void *sim_worker(void *arg)
{
    sim_job *jb = (sim_job *)arg;
    int n = jb->n, k = jb->k, S = jb->n_tx / jb->m, dims = (jb->m == 1) ? 1 : 2;
    uint8_t *u = (uint8_t *)malloc((size_t)k);
    uint8_t *cw = (uint8_t *)malloc((size_t)n);
    double *x = (double *)malloc(sizeof(double) * (size_t)S * dims);
    double *y = (double *)malloc(sizeof(double) * (size_t)S * dims);
    double *ltx = (double *)malloc(sizeof(double) * (size_t)jb->n_tx);
    double *llr = (double *)malloc(sizeof(double) * (size_t)n);
    double *app = (double *)malloc(sizeof(double) * (size_t)n);
    int64_t b;
    if (!u || !cw || !x || !y || !ltx || !llr || !app) { jb->status = ORC_E_NOMEM; goto out; }
    for (b = 0; b < jb->B; ++b) {
        uint64_t cwi = jb->cw0 + (uint64_t)b;
        int32_t it;
        int j, errs = 0, st;
        orc_source_bits(jb->seed, cwi, 1, k, u);
        orc_enc_encode(jb->enc, u, 1, cw);
        orc_map(cw, n, jb->p0, jb->n_tx, jb->m, 1, x);
        orc_awgn(x, 1, S, jb->m, &jb->N0, jb->seed, cwi, y);
        orc_demap(y, 1, S, jb->m, &jb->N0, jb->demap_method, jb->demap_clamp, ltx);
        orc_place_llr(ltx, 1, jb->n_tx, jb->p0, n, llr);
        st = decode_one(jb->g, jb->o, llr, app, &it);
        if (st) { jb->status = st; goto out; }
        for (j = 0; j < k; ++j) errs += ((app[j] < 0.0) != (u[j] != 0));
        jb->counts[0] += k;
        jb->counts[1] += errs;
        jb->counts[2] += 1;
        jb->counts[3] += (errs > 0);
        jb->counts[4] += it;
    }
out:
    free(u); free(cw); free(x); free(y); free(ltx); free(llr); free(app);
    return NULL;
}

int orc_sim(const void *enc, int n, int m_cn, int E, int n_layers, int n_cls,
            const int32_t *cn_ptr, const int32_t *edge_vn, const int32_t *edge_cls, const int32_t *layer_ptr,
            int k, int p0, int n_tx, int mod_m, int demap_method, double demap_clamp,
            int algo, int schedule, int iters, int prec, int store, int early_stop, double offset, double clamp,
            uint64_t seed, uint64_t cw0, int64_t B, double ebn0_db, int64_t *counts, int nthreads)
{
    orc_graph g = { n, m_cn, E, n_layers, n_cls, cn_ptr, edge_vn, edge_cls, layer_ptr };
    orc_opts o = { algo, schedule, iters, prec, store, early_stop, offset, clamp, NULL };
    sim_job jobs[256];
    pthread_t th[256];
    int t, i, status = ORC_OK;
    double N0 = orc_n0_from_ebn0(ebn0_db, k, n_tx, mod_m);
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    if ((int64_t)nthreads > B) nthreads = (int)(B > 0 ? B : 1);
    for (t = 0; t < nthreads; ++t) {
        sim_job *jb = &jobs[t];
        memset(jb, 0, sizeof(*jb));
        jb->enc = enc; jb->g = &g; jb->o = &o; jb->seed = seed;
        jb->cw0 = cw0 + (uint64_t)(B * t / nthreads);
        jb->B = B * (t + 1) / nthreads - B * t / nthreads;
        jb->k = k; jb->n = n; jb->p0 = p0; jb->n_tx = n_tx; jb->m = mod_m;
        jb->demap_method = demap_method; jb->N0 = N0; jb->demap_clamp = demap_clamp;
    }
    if (nthreads == 1) sim_worker(&jobs[0]);
    else {
        for (t = 0; t < nthreads; ++t) pthread_create(&th[t], NULL, sim_worker, &jobs[t]);
        for (t = 0; t < nthreads; ++t) pthread_join(th[t], NULL);
    }
    for (t = 0; t < nthreads; ++t) {
        if (jobs[t].status) status = jobs[t].status;
        for (i = 0; i < 5; ++i) counts[i] += jobs[t].counts[i];
    }
    return status;
}
