/*
 * polar_oracle.c -- plain FP64 CPU oracle of polar coding (construction,
 * encoder, successive-cancellation list decoding with CRC). TEST
 * INFRASTRUCTURE ONLY: built into the oracle library next to ldpc_oracle.c;
 * only tests/ load it. It shares nothing with the CUDA library.
 *
 * The Sionna white paper lists polar codes and SC, SCL and SCL-CRC decoders
 * among its FEC features (Section III) and names the polar SCL decoder as a
 * custom CUDA kernel case (Section IV-A); it prints no equation. Definitions
 * followed here:
 *  - encoder x = u F^{(x)n}, F = [[1,0],[1,1]], natural order (no bit
 *    reversal), N = 2^n (Arikan, IEEE Trans. IT 55(7), 2009);
 *  - construction by Bhattacharyya parameters: bit channel i applies to
 *    z0 = exp(-Es/N0) the transforms z -> 2z - z^2 (bit 0 of i) or z -> z^2
 *    (bit 1) for the bits of i from the most significant down (the first
 *    transform acts on the physical channel); the K channels of smallest z
 *    carry information (ties: the larger index);
 *  - SC decoding in the LLR domain (L = ln P0/P1) with the min-sum check
 *    rule f(a, b) = sgn(a) sgn(b) min(|a|, |b|) and g(a, b, u) = b + (1-2u) a
 *    (Leroux et al., 2011); the LLR of leaf i is computed from scratch for each
 *    path from its own earlier decisions, by the recursion over the tree;
 *  - SCL (Tal & Vardy, IEEE Trans. IT 61(5), 2015) with the LLR-based path
 *    metric of Balatsoukas-Stimming et al. (IEEE Trans. SP 63(19), 2015) in
 *    its approximate form PM += |L_i| when the decision disagrees with the
 *    sign of L_i (h(L) = 1 iff L < 0); frozen bits are 0;
 *  - list selection: candidates (path l, bit b) in the order c = 2l + b; keep
 *    the L smallest (PM, c) lexicographically, the survivors kept in
 *    ascending c; the list doubles from one path until it reaches L;
 *  - CRC-aided selection: the smallest (PM, list index) among the paths whose
 *    information bits pass the CRC, else the smallest among all.
 *  - CRC: the last r information bits are the remainder of the first K - r
 *    (most significant first, zero initial state) modulo the generator
 *    polynomial g (bit r of g set, the x^r term).
 * prec = 1 rounds the result of every arithmetic operation of the decoder (g
 * and the path-metric adds; f is exact) to binary32: the FP32 replay.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define PO_OK 0
#define PO_E_INVAL -1
#define PO_E_NOMEM -3

static double rnd(double x, int prec) { return prec ? (double)(float)x : x; }

/* Bhattacharyya parameters z[N] of the bit channels for design Es/N0 (dB). */
int orc_polar_bhatt(int n, double design_esn0_db, double *z)
{
    int N = 1 << n, i, b;
    double z0;
    if (n < 1 || n > 16) return PO_E_INVAL;
    z0 = exp(-pow(10.0, design_esn0_db / 10.0));
    for (i = 0; i < N; ++i) {
        double v = z0;
        for (b = n - 1; b >= 0; --b) v = ((i >> b) & 1) ? v * v : 2.0 * v - v * v;
        z[i] = v;
    }
    return PO_OK;
}

/* Information set: the K indices of smallest z (ties: larger index first),
 * written ascending to info[K]; frozen[N] = 1 for the others. */
int orc_polar_info_set(int n, double design_esn0_db, int K, int *info, uint8_t *frozen)
{
    int N = 1 << n, i, j, c = 0;
    double *z;
    int *order;
    if (K < 0 || K > N) return PO_E_INVAL;
    z = (double *)malloc(sizeof(double) * N);
    order = (int *)malloc(sizeof(int) * N);
    if (!z || !order) { free(z); free(order); return PO_E_NOMEM; }
    orc_polar_bhatt(n, design_esn0_db, z);
    for (i = 0; i < N; ++i) order[i] = i;
    /* insertion sort by (z ascending, index descending) */
    for (i = 1; i < N; ++i) {
        int v = order[i];
        j = i - 1;
        while (j >= 0 && (z[order[j]] > z[v] || (z[order[j]] == z[v] && order[j] < v))) {
            order[j + 1] = order[j];
            --j;
        }
        order[j + 1] = v;
    }
    for (i = 0; i < N; ++i) frozen[i] = 1;
    for (i = 0; i < K; ++i) frozen[order[i]] = 0;
    for (i = 0; i < N; ++i) if (!frozen[i]) info[c++] = i;
    free(z);
    free(order);
    return PO_OK;
}

/* x = u F^{(x)n} over GF(2), in place on x (copy of u). */
void orc_polar_encode(int n, const uint8_t *u, uint8_t *x)
{
    int N = 1 << n, h, i, j;
    memcpy(x, u, (size_t)N);
    for (h = 1; h < N; h <<= 1)
        for (i = 0; i < N; i += 2 * h)
            for (j = i; j < i + h; ++j) x[j] ^= x[j + h];
}

/* CRC remainder (r bits, MSB first into out[r]) of bits[0..len) modulo g. */
void orc_crc(const uint8_t *bits, int len, uint64_t g, int r, uint8_t *out)
{
    uint64_t reg = 0, top = 1ull << (r - 1), mask = (r == 64) ? ~0ull : ((1ull << r) - 1);
    int i;
    for (i = 0; i < len; ++i) {
        uint64_t fb = ((reg & top) ? 1ull : 0ull) ^ (uint64_t)(bits[i] & 1);
        reg = (reg << 1) & mask;
        if (fb) reg ^= g & mask;
    }
    for (i = 0; i < r; ++i) out[i] = (uint8_t)((reg >> (r - 1 - i)) & 1);
}

static double f_min(double a, double b)
{
    double s = ((a < 0.0) != (b < 0.0)) ? -1.0 : 1.0;
    return s * fmin(fabs(a), fabs(b));
}

/* LLR of leaf i of the size-M subtree whose input LLRs are lam[0..M), given
 * the decisions u[0..i) of that subtree: the recursion over the tree. */
static double leaf_llr(const double *lam, int M, const uint8_t *u, int i, int prec, double *scratch)
{
    int h = M / 2, j;
    double *child = scratch, *rest = scratch + h;
    if (M == 1) return lam[0];
    if (i < h) {
        for (j = 0; j < h; ++j) child[j] = f_min(lam[j], lam[j + h]);
        return leaf_llr(child, h, u, i, prec, rest);
    } else {
        /* partial sums of the left half: its decisions re-encoded */
        uint8_t *ps = (uint8_t *)malloc((size_t)h);
        double r;
        int hh, a, c;
        memcpy(ps, u, (size_t)h);
        for (hh = 1; hh < h; hh <<= 1)
            for (a = 0; a < h; a += 2 * hh)
                for (c = a; c < a + hh; ++c) ps[c] ^= ps[c + hh];
        for (j = 0; j < h; ++j) child[j] = rnd(lam[j + h] + (ps[j] ? -lam[j] : lam[j]), prec);
        free(ps);
        r = leaf_llr(child, h, u + h, i - h, prec, rest);
        return r;
    }
}

static int crc_ok(const uint8_t *uhat, const int *info, int K, uint64_t g, int r)
{
    uint8_t data[1 << 16], rem[64];
    int i;
    if (r == 0) return 1;
    for (i = 0; i < K; ++i) data[i] = uhat[info[i]];
    orc_crc(data, K - r, g, r, rem);
    for (i = 0; i < r; ++i)
        if (rem[i] != data[K - r + i]) return 0;
    return 1;
}

/* SCL decoding of B codewords. llr [B][N]; frozen [N]; info [K] ascending;
 * L >= 1 (L = 1 is SC); CRC g of degree r (r = 0: none). Outputs: uhat
 * [B][N] (the chosen path's decisions), pm [B] (its metric). */
int orc_polar_scl(int n, const double *llr, int64_t B, const uint8_t *frozen, const int *info, int K, int L,
                  uint64_t g, int r, int prec, uint8_t *uhat, double *pm)
{
    int N = 1 << n, Lmax = L;
    int64_t b;
    uint8_t *paths, *npaths;
    double *pms, *npms, *scratch, *lam;
    if (n < 1 || n > 12 || L < 1 || L > 64 || K < 0 || K > N || r < 0 || r > K || r > 63) return PO_E_INVAL;
    paths = (uint8_t *)malloc((size_t)Lmax * N);
    npaths = (uint8_t *)malloc((size_t)Lmax * N);
    pms = (double *)malloc(sizeof(double) * Lmax);
    npms = (double *)malloc(sizeof(double) * Lmax);
    scratch = (double *)malloc(sizeof(double) * 2 * N);
    lam = (double *)malloc(sizeof(double) * N);
    if (!paths || !npaths || !pms || !npms || !scratch || !lam) {
        free(paths); free(npaths); free(pms); free(npms); free(scratch); free(lam);
        return PO_E_NOMEM;
    }
    for (b = 0; b < B; ++b) {
        int cur = 1, i, l, best = -1;
        for (i = 0; i < N; ++i) lam[i] = rnd(llr[b * N + i], prec);
        memset(paths, 0, (size_t)Lmax * N);
        pms[0] = 0.0;
        for (i = 0; i < N; ++i) {
            if (frozen[i]) {
                for (l = 0; l < cur; ++l) {
                    double li = leaf_llr(lam, N, paths + (size_t)l * N, i, prec, scratch);
                    paths[(size_t)l * N + i] = 0;
                    if (li < 0.0) pms[l] = rnd(pms[l] + fabs(li), prec);
                }
            } else {
                /* 2 cur candidates c = 2l + bit with metrics */
                int nc = 2 * cur, keep = nc < Lmax ? nc : Lmax, c, k, sel[2 * 64];
                double cm[2 * 64];
                uint8_t taken[2 * 64];
                for (l = 0; l < cur; ++l) {
                    double li = leaf_llr(lam, N, paths + (size_t)l * N, i, prec, scratch);
                    int h = li < 0.0 ? 1 : 0;
                    cm[2 * l] = h == 0 ? pms[l] : rnd(pms[l] + fabs(li), prec);
                    cm[2 * l + 1] = h == 1 ? pms[l] : rnd(pms[l] + fabs(li), prec);
                }
                memset(taken, 0, sizeof(taken));
                for (k = 0; k < keep; ++k) { /* the k-th smallest (metric, index) */
                    int bi = -1;
                    for (c = 0; c < nc; ++c)
                        if (!taken[c] && (bi < 0 || cm[c] < cm[bi])) bi = c;
                    taken[bi] = 1;
                }
                k = 0;
                for (c = 0; c < nc; ++c) if (taken[c]) sel[k++] = c; /* survivors in ascending c */
                for (k = 0; k < keep; ++k) {
                    int src = sel[k] >> 1;
                    memcpy(npaths + (size_t)k * N, paths + (size_t)src * N, (size_t)N);
                    npaths[(size_t)k * N + i] = (uint8_t)(sel[k] & 1);
                    npms[k] = cm[sel[k]];
                }
                memcpy(paths, npaths, (size_t)keep * N);
                memcpy(pms, npms, sizeof(double) * keep);
                cur = keep;
            }
        }
        for (l = 0; l < cur; ++l)
            if (crc_ok(paths + (size_t)l * N, info, K, g, r) && (best < 0 || pms[l] < pms[best])) best = l;
        if (best < 0)
            for (l = 0; l < cur; ++l)
                if (best < 0 || pms[l] < pms[best]) best = l;
        memcpy(uhat + b * N, paths + (size_t)best * N, (size_t)N);
        pm[b] = pms[best];
    }
    free(paths); free(npaths); free(pms); free(npms); free(scratch); free(lam);
    return PO_OK;
}
