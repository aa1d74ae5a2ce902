/*
 * ldpcx.h -- C ABI of the GB300 QC-LDPC Monte-Carlo library (libldpcx.so).
 *
 * The library implements the hot path of the link-level Monte-Carlo
 * simulation shown as the "Hello, World!" chain of the Sionna white paper
 * (arXiv 2203.11854, Listing 1): BinarySource -> LDPC5GEncoder -> Mapper ->
 * AWGN -> Demapper("app") -> LDPC5GDecoder -> compute_ber, with the min-sum
 * belief-propagation decoder written as a custom CUDA kernel (Sec. IV-A).
 *
 * Conventions shared by every entry point
 *  - Every function returns an int status: LDPCX_OK (0) or a negative
 *    LDPCX_E_* code. Argument errors are detected on the host before any
 *    work is queued and leave all outputs untouched.
 *  - Pointers documented as "device" must point to memory of the current CUDA
 *    device (cudaMalloc / torch CUDA tensors). The caller owns every buffer;
 *    the library only owns ldpcx_code_t objects and their internal tables.
 *  - `stream` is a cudaStream_t (NULL = legacy default stream). Work is
 *    queued asynchronously on it; results are ready once it is synchronised.
 *  - Conditions only the GPU can see (a non-finite input, a bounded wait that
 *    gave up) do not abort the kernel: they are latched in a device status
 *    word and reported by ldpcx_sync_status().
 *  - LLR convention: L = ln P(b=0 | y) / P(b=1 | y); hard decision b = 1 iff
 *    L < 0. (Listing 2 of the paper feeds LLRs to a binary cross-entropy
 *    "from logits", which is the opposite sign: logits = -L.)
 *  - Bit vectors are packed little-endian in uint32 words: bit j of a
 *    codeword's vector is bit (j mod 32) of word j/32; words per codeword =
 *    ceil(bits / 32); unused high bits of the last word are zero.
 */
#ifndef LDPCX_H
#define LDPCX_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------ status */
#define LDPCX_OK 0
#define LDPCX_E_INVAL (-1)       /* bad argument: null pointer, size or enum out of range */
#define LDPCX_E_UNSUPPORTED (-2) /* valid request this build does not implement */
#define LDPCX_E_NOMEM (-3)       /* host or device allocation failed */
#define LDPCX_E_WORKSPACE (-4)   /* workspace missing, too small or misaligned */
#define LDPCX_E_CUDA (-5)        /* a CUDA runtime call failed */
#define LDPCX_E_NONFINITE (-6)   /* device-latched: a non-finite input was sanitised */
#define LDPCX_E_TIMEOUT (-7)     /* device-latched: a bounded wait gave up */
#define LDPCX_E_NODEVICE (-8)    /* no CUDA device is visible */
#define LDPCX_E_IO (-9)          /* a checkpoint file could not be read, parsed or written */

/* Device status flags latched by kernels (ldpcx_sync_status). */
#define LDPCX_FLAG_NONFINITE 1u  /* NaN input -> treated as 0; +-inf -> +-clamp */
#define LDPCX_FLAG_TIMEOUT 2u

/* Human-readable name of a status code; never NULL. */
const char *ldpcx_status_str(int status);

/* Synchronise `stream`, then return (in *flags) the OR of the device status
 * flags latched since the previous call on this device, and clear them.
 * Returns LDPCX_E_NONFINITE / LDPCX_E_TIMEOUT when a flag was set, LDPCX_OK
 * otherwise. flags may be NULL. */
int ldpcx_sync_status(void *stream, unsigned int *flags);

/* ------------------------------------------------------------ code */
/* A seeded quasi-cyclic LDPC code with the 5G-NR base-graph shape (the
 * paper's "5G LDPC codes", Sec. III-B; LDPC5GEncoder in Listing 1). The 3GPP
 * TS 38.212 shift tables are not used: the base matrix S (rows x cols, -1 =
 * all-zero block, s >= 0 = identity cyclically shifted by s) is drawn from
 * splitmix64(seed):
 *   columns [0,Kb) systematic, [Kb,Kb+4) core parity, [Kb+4,cols) extension;
 *   core parity blocks  row0 [1 0 - -]  row1 [0 0 0 -]  row2 [- - 0 0]
 *                       row3 [1 - - 0]   (dual diagonal, rows sum to [I 0 0 0]);
 *   extension row j: identity at column Kb+4+j;
 *   support: core rows draw d_core distinct systematic columns, extension row
 *   j draws d_ext(j) distinct columns of [0,Kb+4), each by a partial
 *   Fisher-Yates shuffle (index i + next() mod (N - i)); then each drawn
 *   block in row-major order gets shift next() mod Z.
 *   bg_shape 1: Kb 22, 46 rows, 68 cols, d_core 16, d_ext 5 (j<33) / 4 -> 316 blocks.
 *   bg_shape 2: Kb 10, 42 rows, 52 cols, d_core 8,  d_ext 4 (j<4)  / 3 -> 197 blocks.
 * Block (r,c) with shift s joins check node r*Z+z to variable node
 * c*Z + (z+s) mod Z. Codeword c = [u | p], u = the k = Kb*Z information bits.
 * Transmission: the first punct_cols*Z systematic bits are not sent; the
 * n_tx bits at positions [punct_cols*Z, punct_cols*Z + n_tx) are sent.
 * rows_kept < rows keeps the first rows_kept rows and Kb+rows_kept columns
 * (rate by extension truncation). */
typedef struct ldpcx_code *ldpcx_code_t;

typedef struct {
    int bg_shape;   /* 1 or 2 */
    int Z;          /* lifting size, 2..384 */
    uint64_t seed;  /* splitmix64 seed of the support and the shifts */
    int rows_kept;  /* 4..rows, or 0 = all rows */
    int punct_cols; /* 0..Kb systematic columns not transmitted (5G uses 2) */
    int n_tx;       /* transmitted bits; 0 = every bit after the punctured ones */
} ldpcx_code_params;

typedef struct {
    int Z, rows, cols, kb;   /* base matrix shape */
    int nnz;                 /* nonzero base blocks (= weight classes) */
    int max_row_deg;         /* largest check-node degree */
    int n, k, n_tx, p0;      /* codeword, info and transmitted bits; p0 = first transmitted position */
    int64_t edges;           /* nnz * Z */
    int encodable;           /* 1 when the transmitter can encode the code (see qc_ldpc_build_base) */
    int n_fill;              /* filler bits at positions k .. k + n_fill - 1 (qc_ldpc_shorten), else 0 */
} ldpcx_code_info;

/* Build the code on the host (no device work; device tables are uploaded on
 * first use on the then-current device). *out is owned by the caller until
 * qc_ldpc_free. Errors: LDPCX_E_INVAL for a bad shape or null pointer. */
int qc_ldpc_build(const ldpcx_code_params *params, ldpcx_code_t *out);
/* Release the code and its device tables. NULL is accepted. The code must not
 * be in use by queued work. */
int qc_ldpc_free(ldpcx_code_t code);
/* Sizes of the code. */
int qc_ldpc_info(ldpcx_code_t code, ldpcx_code_info *info);
/* Copy the base matrix (row-major int16, -1 = zero block) into host memory
 * S_out of `capacity` entries (>= rows*cols, else LDPCX_E_INVAL). */
int qc_ldpc_base(ldpcx_code_t code, int16_t *S_out, int capacity);

/* A code block carrying k < kb*Z information bits (the 5G code blocks of the
 * paper's Listing 1, k = 500 bits coded into n = 1000, Sec. III-C): *out is a
 * new code object, a copy of `code` in which systematic positions k .. kb*Z-1
 * are filler bits. Fillers are 0, known to both ends, and never transmitted:
 * the transmit layout (sim_tx, sim_codewords' transmitted bits, rate_match,
 * rate_recover, the decoders' llr_ch, ldpc_extrinsic) is the list of codeword
 * positions p0 .. p0 + n_tx + n_fill - 1 without the fillers, in increasing
 * order, so n_tx shrinks by n_fill. The transmitter draws k source bits and
 * encodes [u | 0 ... 0]; the decoders give the fillers the channel LLR
 * +clamp (a known zero) and write k bits to bits_out; sim_run counts k bits
 * per block. The base matrix, the tables and every kernel are the mother
 * code's. Requires p0 <= k <= kb*Z, fillers inside the transmitted span
 * (p0 + n_tx >= kb*Z) and an unshortened `code`, else LDPCX_E_INVAL. The
 * differentiable decode (ldpc_bp_decode_ckpt, ldpc_bp_backward) accepts no
 * shortened code (LDPCX_E_UNSUPPORTED). Free *out with qc_ldpc_free; it does
 * not depend on `code` afterwards. */
int qc_ldpc_shorten(ldpcx_code_t code, int k, ldpcx_code_t *out);

/* A quasi-cyclic code from a caller-supplied base matrix (the paper's
 * Section III lists LDPC codes from user parity-check matrices, with alist
 * import, next to the 5G codes). S: host, rows x cols row-major, -1 = all-zero
 * block, s in [0, Z) = identity cyclically shifted by s (block (r,c) joins
 * check node r*Z+z to variable node c*Z + (z+s) mod Z, as for the seeded
 * codes); copied, the caller keeps ownership. The first kb columns are the
 * systematic ones (k = kb*Z); transmission as for qc_ldpc_build (punct_cols
 * systematic columns not sent, then n_tx bits; n_tx = 0: all the rest).
 * Every decoder accepts the code (within its limits: row degree <= 20,
 * n <= 65535, else LDPCX_E_UNSUPPORTED at decode time). The transmitter
 * (sim_tx, sim_codewords, sim_run) also needs cols = kb + rows >= kb + 4,
 * core rows 0..3 with no block past column kb+3, extension row r >= 4 with,
 * past column kb+3, exactly one block, at its own column kb+r (any shift), and
 * an invertible core parity part (rows 0..3 x columns kb..kb+3, 4Z x 4Z over
 * GF(2)); ldpcx_code_info.encodable says whether it holds, and the
 * transmitter returns LDPCX_E_UNSUPPORTED when it does not. The 5G
 * dual-diagonal core [[P1 I - -] [I I I -] [- - I I] [P1 - - I]] is encoded
 * by its recursion, any other invertible core through its inverse (computed
 * here by Gauss-Jordan elimination). Errors: LDPCX_E_INVAL for a null
 * pointer, Z outside [2, 384], rows or cols outside [1, 4096] / [2, 4096],
 * kb outside [1, cols), a shift outside [-1, Z), a row with fewer than two
 * blocks, or a bad puncturing / n_tx. */
typedef struct {
    int rows, cols;   /* base matrix shape */
    int kb;           /* systematic columns */
    int Z;            /* lifting size, 2..384 */
    const int16_t *S; /* host [rows][cols] */
    int punct_cols;   /* 0..kb */
    int n_tx;         /* 0 = every bit after the punctured ones */
} ldpcx_base_params;
int qc_ldpc_build_base(const ldpcx_base_params *params, ldpcx_code_t *out);

/* Parse a parity-check matrix in alist text (MacKay's format: "N M", the
 * largest column and row weights, the N column weights, the M row weights,
 * then N lines of 1-based row indices, one line per column, and M lines of
 * 1-based column indices, one per row; zeros pad a line and are skipped) into
 * the base matrix of lifting size Z. text: host, len bytes (a NUL ends it
 * early). The matrix must consist of Z x Z blocks that are zero or cyclically
 * shifted identities, and the column lists must give the same entries as the
 * row lists. Writes *rows_out = M/Z, *cols_out = N/Z, and, when S_out is
 * not NULL, the base matrix to S_out (capacity >= rows*cols entries; -1 =
 * zero block). Errors: LDPCX_E_INVAL for malformed text, inconsistent
 * lists, a non-circulant block, N or M not a multiple of Z, or a small
 * capacity. */
int qc_alist_parse(const char *text, size_t len, int Z, int16_t *S_out, int capacity, int *rows_out,
                   int *cols_out);
/* The code's parity-check matrix as alist text (the format above, lines
 * padded with zeros to the largest weight), NUL-terminated in buf (cap bytes).
 * *len_out = the text length without the NUL, always; buf = NULL is a size
 * query. Errors: LDPCX_E_INVAL for a null code or len_out, or cap <= len. */
int qc_ldpc_alist(ldpcx_code_t code, char *buf, size_t cap, size_t *len_out);

/* ------------------------------------------------ transmitter */
/* Monte-Carlo transmitter for codewords cw0 .. cw0+B-1 (BinarySource,
 * LDPC5GEncoder, Mapper, AWGN of Listing 1), all on the device:
 *  - info bit j of codeword w = bit (j mod 32) of output word (j mod 128)/32
 *    of Philox4x32-10 (Salmon et al., SC'11) with key (seed lo32, seed hi32)
 *    and counter (j/128, w lo32, w hi32, 0);
 *  - systematic encoding by the dual-diagonal recursion of the core followed
 *    by the extension parities;
 *  - Gray square QAM per dimension: bits b0,b2,.. -> I and b1,b3,.. -> Q, level
 *    (1-2a0)(2^(h-1) - (1-2a1)(2^(h-2) - ...)) scaled to unit average energy;
 *    m = 1 is BPSK x = 1-2b on a real channel;
 *  - AWGN y = x + sqrt(N0/2) g per real dimension, g by Box-Muller from
 *    Philox block q = (index of the Gaussian)/4 on stream 1: u1 = ((a>>9)+0.5)
 *    2^-23, u2 = (b>>8) 2^-24 from words (a,b) = (x0,x1) or (x2,x3),
 *    g = sqrt(-2 ln u1) (cos 2 pi u2, sin 2 pi u2); complex symbol s uses
 *    Gaussians 2s, 2s+1; real symbol s uses Gaussian s.
 * no: device float, N0 of codeword b at no[b * no_stride] (stride 0 or 1).
 * y_out (device): m = 1 -> [B][n_tx] float; else [B][n_tx/m][2] float (re, im).
 * info_out (device, or NULL): [B][ceil(k/32)] packed information bits.
 * m in {1,2,4,6,8} and n_tx divisible by m, else LDPCX_E_INVAL. A code the
 * transmitter cannot encode (ldpcx_code_info.encodable = 0; only codes of
 * qc_ldpc_build_base) gives LDPCX_E_UNSUPPORTED, here and in sim_codewords,
 * sim_tx_points and sim_run. */
int sim_tx(ldpcx_code_t code, uint64_t seed, uint64_t cw0, int64_t B, int m,
           const float *no, int64_t no_stride, float *y_out, uint32_t *info_out, void *stream);

/* Mapper and AWGN on caller bits (the Mapper and AWGN layers of Listing 1
 * applied to a rate-matched stream, Sec. III-C): bits (device)
 * [B][ceil(E/32)] packed (bit t of row b = bit t mod 32 of word t/32), E bits
 * per row, m in {1,2,4,6,8} dividing E. Symbol s of row b maps bits
 * s m .. s m + m - 1 as sim_tx maps a symbol and adds the Gaussians sim_tx
 * draws for symbol s of codeword cw0 + b, with the same arithmetic: sim_tx
 * equals sim_codewords, then rate_match with k0 = 0, ncb = E = n_tx, qm = 1,
 * then this call. no: device, N0 of row b at no[b * no_stride] (stride 0 or
 * 1). y_out (device): m = 1 -> [B][E] float; else [B][E/m][2] (re, im).
 * Errors: LDPCX_E_INVAL for B < 0, E < 1, a bad m or stride, or a null pointer
 * with B > 0. */
int qam_map_awgn(const uint32_t *bits, int64_t B, int E, int m, uint64_t seed, uint64_t cw0, const float *no,
                 int64_t no_stride, float *y_out, void *stream);

/* ----------------------------------------------------------- demap */
/* APP demapper (Demapper("app"), Listing 1) for Gray square QAM on AWGN:
 *   L_i = ln sum_{x: b_i(x)=0} exp(-|y-x|^2/N0) - ln sum_{x: b_i(x)=1} exp(...)
 * computed per I/Q dimension (exact for Gray square QAM on a circular AWGN
 * channel: the other dimension's factor cancels). method LDPCX_DEMAP_EXACT
 * uses log-sum-exp, LDPCX_DEMAP_MAXLOG the largest term. The result is
 * clamped to [-clamp, clamp]. A non-finite y gives L = 0 and latches
 * LDPCX_FLAG_NONFINITE.
 * y (device): m = 1 -> [B][syms] float; else [B][syms][2] float (re, im).
 * no (device): N0 of codeword b at no[b * no_stride] (stride 0 or 1).
 * llr_out (device): [B][syms*m] float, bit i of symbol s at s*m + i. */
#define LDPCX_DEMAP_EXACT 0
#define LDPCX_DEMAP_MAXLOG 1
int demap_app(const float *y, const float *no, int64_t no_stride, int64_t B, int64_t syms_per_cw,
              int m, int method, float clamp, float *llr_out, void *stream);

/* ------------------------------------------------ BP decoding */
/* Belief-propagation decoding (LDPC5GDecoder, "BP decoder and variants",
 * Sec. III-B; min-sum BP as the custom CUDA op of Sec. IV-A). Messages
 * R = check-to-variable; for the variable-to-check inputs T_i of a check:
 *  offset min-sum: R_j = sgn_j s max(m_j - offset, 0), m_j = second smallest
 *    |T| at the first index of the smallest, the smallest elsewhere,
 *    s = prod_i sgn(T_i), sgn(x) = -1 iff x < 0;
 *  sum-product: R_j = sgn_j s phi(sum_{i!=j} phi(|T_i|)),
 *    phi(x) = -ln tanh(x/2), each phi argument clamped to [phi(clamp), clamp];
 *  |R| <= clamp; then R is rounded to the message format (FP32 as is; FP16
 *  round-to-nearest-even; FIX6: 6-bit fixed point with step 0.5, RNE,
 *  saturated to +-31 steps) and the rounded value is stored and used.
 * Layered schedule: layer = base row in ascending order, each check node
 *  T_j = APP_v - R_j(old), CN rule, APP_v = T_j + R_j(new).
 * Flooding schedule: T_j = w[t][blk] (APP_v(old) - R_j(old)) with w = 1 when
 *  weights == NULL; APP_v(new) = L_v + sum of the new R over v's checks,
 *  added in ascending base-row order.
 * Channel LLRs are clamped to +-clamp (NaN -> 0, latching NONFINITE);
 * punctured / untransmitted positions start at 0; APP is not clamped.
 * Early stop: after each full iteration the hard decisions are checked
 * against every parity check; a codeword stops at the first iteration whose
 * syndrome is zero. Iteration count = full iterations run (1..iters).
 * Arithmetic is binary32 in the order above (no fused multiply-add), so
 * min-sum results are reproducible bit for bit. */
#define LDPCX_LAYERED_MINSUM 0
#define LDPCX_LAYERED_SPA 1
#define LDPCX_FLOOD_MINSUM 2
#define LDPCX_FLOOD_SPA 3
#define LDPCX_MSG_F32 0
#define LDPCX_MSG_F16 1
#define LDPCX_MSG_FIX6 2 /* min-sum only */

typedef struct {
    int algo;             /* LDPCX_LAYERED_MINSUM .. LDPCX_FLOOD_SPA */
    int iters;            /* 1..1000 */
    int msg_prec;         /* LDPCX_MSG_* */
    int early_stop;       /* 0 or 1 */
    float offset;         /* min-sum offset beta >= 0 (0.5 for the 5G workloads) */
    float clamp;          /* > 0; 20 for the 5G workloads */
    const float *weights; /* flooding only: device [iters][nnz] per-iteration per-base-block
                             weights (block index = row-major order of the base matrix), or NULL */
} ldpcx_decode_opts;

/* Workspace in bytes that ldpc_bp_decode needs for B codewords (message
 * storage: B * round_up(edges, 64) messages of the chosen format). */
int ldpc_bp_workspace(ldpcx_code_t code, int64_t B, const ldpcx_decode_opts *opts, size_t *ws_bytes);

/* The message storage ldpc_bp_decode will use for this code and options:
 * *cn_state = 1 when layered min-sum keeps check-node state (see
 * LDPCX_TUNE_CN_STATE), 0 for per-edge messages; *bytes_per_cw = bytes of
 * message storage one codeword reads or writes in one full iteration. */
int ldpc_bp_msg_format(ldpcx_code_t code, const ldpcx_decode_opts *opts, int *cn_state, int64_t *bytes_per_cw);

/* The sum-product check-node function phi(x) = -ln tanh(x/2) = ln(1 + 2/(e^x
 * - 1)) as the decoders evaluate it, on n device floats x (each in
 * [phi(clamp), clamp] as the decoders use it; x > 0 required). fast = 0: from
 * the CUDA library functions expm1f, IEEE division and log1pf; fast = 1: from
 * the hardware 2^x, 1/x and log2 approximations with Taylor series where a
 * difference would cancel (the adjoint of flooding sum-product); fast = 2:
 * the same approximations in bits, phi(x) / ln 2 of x log2 e, times ln 2
 * here (layered and flooding sum-product, which sum the terms in bits).
 * Exposed so that tests can bound each against FP64. Asynchronous on stream; LDPCX_E_INVAL for
 * n < 0, null pointers with n > 0 or fast outside 0..2. */
int ldpcx_phi(const float *x, float *out, int64_t n, int fast, void *stream);

/* Decode B codewords.
 * llr_ch   (device) [B][n_tx] float channel LLRs of the transmitted positions.
 * llr_out  (device, or NULL) [B][n] float final APP LLRs.
 * bits_out (device, or NULL) [B][ceil(k/32)] packed hard decisions of the k
 *          information positions (punctured ones included).
 * iters_out(device, or NULL) [B] int32 iterations run.
 * ws       (device) >= ldpc_bp_workspace bytes, 256-byte aligned; contents
 *          on entry are ignored and on exit undefined.
 * Pure function of its inputs: the same call gives the same outputs. */
int ldpc_bp_decode(ldpcx_code_t code, const float *llr_ch, int64_t B, const ldpcx_decode_opts *opts,
                   float *llr_out, uint32_t *bits_out, int32_t *iters_out,
                   void *ws, size_t ws_bytes, void *stream);

/* The demapper fused into the decoder (Demapper("app") feeding
 * LDPC5GDecoder in the paper's Listing 1, as one launch): the layered
 * decoders compute each codeword's channel LLRs from its received symbols
 * while loading them, so no LLR array is written or read. The results equal
 * demap_app(y, no, no_stride, B, n_tx/m, m, demap_method, demap_clamp, llr)
 * followed by ldpc_bp_decode(code, llr, B, opts, ...) bit for bit, the
 * NONFINITE flag included (a non-finite symbol gives zero LLRs).
 * y        (device) [B][n_tx/m] complex symbols as float pairs (re, im), or
 *          [B][n_tx] floats for m = 1; the layout sim_tx writes.
 * no       (device) N0: [B] floats (no_stride = 1) or one float (0).
 * m        1, 2, 4, 6 or 8 bits per symbol; n_tx must be a multiple of m.
 * demap_method LDPCX_DEMAP_EXACT or LDPCX_DEMAP_MAXLOG; demap_clamp finite, > 0.
 * opts, outputs, ws and ws_bytes as ldpc_bp_decode (same workspace size).
 * Errors: LDPCX_E_INVAL for a bad argument; LDPCX_E_UNSUPPORTED for the
 * flooding schedules, whose kernels read the channel LLRs in every
 * iteration; otherwise as ldpc_bp_decode. */
int ldpc_bp_decode_qam(ldpcx_code_t code, const float *y, const float *no, int64_t no_stride, int64_t B, int m,
                       int demap_method, float demap_clamp, const ldpcx_decode_opts *opts, float *llr_out,
                       uint32_t *bits_out, int32_t *iters_out, void *ws, size_t ws_bytes, void *stream);

/* Decoder tuning knobs (process-wide; read at each launch; the autotuner's
 * search space). LDPCX_TUNE_L2_PREFETCH: layered decoders prefetch into L2 the
 * message span of the layer this many layers ahead (0 = off, 0..16, default 0).
 * LDPCX_TUNE_ZPT: check nodes per thread of the layered min-sum kernels with
 * a compiled-in schedule (LDPCX_TUNE_SCHEDULE): 0 = auto = 1; 2 = check nodes
 * z and z + Z/2, honoured when Z is even. Other kernels use one.
 * LDPCX_TUNE_CW_PER_CTA: codewords decoded together by one CTA of
 * ldpc_bp_decode (0 = automatic: layered, about 384 check nodes per CTA
 * within the shared-memory budget, fewer when the batch would give the SMs
 * fewer than about four CTAs each; flooding, up to 32 codewords by the fewest
 * codewords per SM, raised where a thread would have fewer than two check
 * nodes; a smaller value gives smaller CTAs, more per SM), and
 * the cap on the codewords of one work item of ldpc_bp_decode_mixed (smaller
 * items: a finer queue, less waiting on a tile's slowest codeword).
 * LDPCX_TUNE_SPECIALISED: 1 (default) = use the layered min-sum kernels built
 * for a compile-time lifting size when one exists for the code's Z (384);
 * 0 = always the generic kernel.
 * LDPCX_TUNE_CN_STATE: 1 (default) = layered min-sum keeps, per check node,
 * the two rounded message magnitudes and per-edge "took the second minimum" and
 * sign bits instead of one stored message per edge (4, 8 or 16 bytes per check
 * node); every message is rebuilt exactly, so results are identical. Used when
 * the state fits the per-edge workspace. 0 = per-edge messages.
 * LDPCX_TUNE_SCHEDULE: 1 (default) = a code whose row degrees are those of
 * its shape's base graph (every code of qc_ldpc_build: full, or truncated by
 * rows_kept) runs a kernel with that layer schedule compiled in -- min-sum
 * with check-node state for full and truncated codes, sum-product for full
 * codes; 0 = the kernels that read the schedule from the row table.
 * Knobs change speed only, never results. */
#define LDPCX_TUNE_L2_PREFETCH 1
#define LDPCX_TUNE_ZPT 2
#define LDPCX_TUNE_CW_PER_CTA 3
#define LDPCX_TUNE_SPECIALISED 4
#define LDPCX_TUNE_CN_STATE 5
#define LDPCX_TUNE_SCHEDULE 6
int ldpcx_tune_set(int key, int value);
int ldpcx_tune_get(int key, int *value);

/* Host-side fault injection, for tests of the error paths (the library makes
 * no GPU fault on purpose). kind LDPCX_FAULT_ALLOC arms a one-shot allocation
 * failure: the allocations of the library -- a code or polar object on the host
 * (qc_ldpc_build, qc_ldpc_build_base, qc_ldpc_shorten, polar_build), and the
 * device tables a code or polar code uploads on its first use on a device
 * (sim_tx, sim_codewords, sim_tx_points, ldpc_bp_decode and its variants,
 * ldpc_bp_backward, sim_run, polar_sim_tx, polar_scl_decode) -- let `after`
 * allocations pass and fail the next one, which then returns LDPCX_E_NOMEM
 * with the caller's outputs untouched; the injector then disarms.
 * LDPCX_FAULT_NONE disarms it. The environment variable LDPCX_FAULT=alloc or
 * alloc:N (N = `after`) arms it when the library first checks it. Errors:
 * LDPCX_E_INVAL for an unknown kind or after < 0. */
#define LDPCX_FAULT_NONE 0
#define LDPCX_FAULT_ALLOC 1
int ldpcx_fault_set(int kind, int after);

/* Allocation-free decode. The paper has no counterpart: this entry point
 * exists for callers that cannot call cudaMalloc -- a receiver that allocates
 * every buffer at start-up and forbids allocation on its real-time path, a host
 * thread that must never block on the device (cudaMalloc may synchronise), or
 * a component whose device memory belongs to an allocator this library cannot
 * reach. It decodes exactly like ldpc_bp_decode (same arguments and outputs,
 * same kernel choice and tuning knobs, same results bit for bit) but keeps its
 * scratch -- the code tables and the check-to-variable messages, or for
 * layered min-sum the check-node state -- in a fixed array of
 * LDPCX_NOALLOC_SCRATCH_BYTES inside the library image, which every GPU that
 * loads the library holds until the process exits. It calls no cudaMalloc,
 * cudaFree or allocating library routine. Limits: the tables (rounded to 256
 * bytes) plus B times the per-codeword bytes of the decoder's message format
 * must fit in the array, else LDPCX_E_WORKSPACE before any work; B is bounded
 * before any product is formed. At Z = 384, BG1-shaped: layered min-sum
 * (their state format) 118 / 153 / 307 codewords with FP32 / FP16 / FIX6
 * messages; sum-product and flooding (per-edge messages) 69 / 138. The first
 * call on a device looks up the array's device address (cudaGetSymbolAddress);
 * make that first call before any stream capture. Every call on a device
 * shares the array and leaves its contents behind; nothing needs clearing
 * (tables are rewritten by each call, every message is written before it is
 * read), but calls that overlap on the GPU -- on different streams -- race on
 * it. */
#define LDPCX_NOALLOC_SCRATCH_BYTES (32u << 20)
int ldpc_bp_decode_noalloc(ldpcx_code_t code, const float *llr_ch, int64_t B, const ldpcx_decode_opts *opts,
                           float *llr_out, uint32_t *bits_out, int32_t *iters_out, void *stream);

/* -------------------------------------------- mixed-size batch */
/* One persistent launch decodes a batch mixing codes of different lifting
 * sizes, base-graph shapes and rates -- the per-example differing execution
 * the paper names as the reason for custom CUDA ops (Sec. III-D, Sec. IV-A).
 * The batch is a list of groups, one per code. Work items (up to G codewords
 * of one code, G = the codewords one CTA decodes together) are ordered by
 * nominal cost (edges x codewords, largest first) and pulled by resident CTAs
 * from a device queue with atomicAdd; a CTA decodes an item to the end
 * (including early stop) before it pulls the next. Layered schedules only.
 * Results equal ldpc_bp_decode on each group separately, bit for bit. */
typedef struct {
    ldpcx_code_t code;
    int64_t B;             /* codewords of this group (>= 0) */
    const float *llr_ch;   /* device [B][n_tx of the code] */
    float *llr_out;        /* device [B][n] or NULL */
    uint32_t *bits_out;    /* device [B][ceil(k/32)] or NULL */
    int32_t *iters_out;    /* device [B] or NULL */
} ldpcx_batch_group;

/* Workspace bytes for the groups: queue, item list, and message scratch for
 * each resident CTA (not per codeword). Needs the current device (SM count). */
int ldpc_bp_mixed_workspace(const ldpcx_batch_group *groups, int n_groups, const ldpcx_decode_opts *opts,
                            size_t *ws_bytes);
/* Decode all groups in one persistent launch. ws: device, >= the workspace
 * bytes, 256-byte aligned; it is written (queue, items) before the launch. */
int ldpc_bp_decode_mixed(const ldpcx_batch_group *groups, int n_groups, const ldpcx_decode_opts *opts, void *ws,
                         size_t ws_bytes, void *stream);

/* ------------------------------------------- differentiable BP */
/* Gradients through the unrolled decoder ("gradients can be specified" for a
 * custom op, Sec. IV-A; end-to-end learning with a binary cross-entropy loss,
 * Sec. III-C, Listing 2). Supported for weighted flooding sum-product
 * (LDPCX_FLOOD_SPA, FP32 messages, no early stop): the forward pass
 * ldpc_bp_decode_ckpt stores each iteration's check-to-variable messages C^t
 * and the APP after it, APP^(t+1) = L + sum C^t (t = 0 .. iters-2), as FP32
 * checkpoints; ldpc_bp_backward walks the iterations in reverse, takes APP^t
 * (L for t = 0) and recomputes the check-node quantities of iteration t from
 * the checkpoints, and propagates the adjoints
 *   dC_e/dV_e' = s_e phi'(x_e) [lo < S_e < hi] phi'(a_e') sgn(V_e') [lo <= |V_e'| <= hi]
 * (e' != e in the same check; x_e = clamp(S_e), a = clamp(|V|), phi'(x) =
 * -1/sinh(x)), V_e = w (APP_v - C_e(old)), APP = L + sum C, L = clamp(llr_ch).
 *
 * ckpt bytes = 4 * max(iters-1, 1) * B * (round_up(edges, 128) + round_up(n, 32)):
 * the messages [iters-1][B][round_up(edges, 128)], then the APP values
 * [iters-1][B][round_up(n, 32)]. */
int ldpc_bp_ckpt_bytes(ldpcx_code_t code, int64_t B, const ldpcx_decode_opts *opts, size_t *ckpt_bytes);
/* ldpc_bp_decode plus checkpoints (device, >= ldpc_bp_ckpt_bytes, 16-byte aligned). */
int ldpc_bp_decode_ckpt(ldpcx_code_t code, const float *llr_ch, int64_t B, const ldpcx_decode_opts *opts,
                        float *llr_out, uint32_t *bits_out, int32_t *iters_out, void *ws, size_t ws_bytes,
                        void *ckpt, size_t ckpt_bytes, void *stream);
/* Workspace of ldpc_bp_backward: 4 * B * round_up(edges, 128) bytes (adjoint carry). */
int ldpc_bp_backward_workspace(ldpcx_code_t code, int64_t B, const ldpcx_decode_opts *opts, size_t *ws_bytes);
/* Adjoint of ldpc_bp_decode_ckpt with the same code, llr_ch, B and opts.
 * grad_llr_out (device) [B][n]: dLoss/d(output APP).
 * grad_llr_ch  (device) [B][n_tx]: dLoss/d(llr_ch), overwritten.
 * grad_weights (device, or NULL) [iters][nnz]: dLoss/d(weights), ACCUMULATED
 *              (+=, float atomics: the summation order is not fixed).
 * opts->weights may be NULL (all ones). Errors: LDPCX_E_UNSUPPORTED for other
 * algorithms, message formats or early stop, or a code too long for the
 * kernel's shared memory (n > 13800). */
int ldpc_bp_backward(ldpcx_code_t code, const float *llr_ch, int64_t B, const ldpcx_decode_opts *opts,
                     const void *ckpt, size_t ckpt_bytes, const float *grad_llr_out, float *grad_llr_ch,
                     float *grad_weights, void *ws, size_t ws_bytes, void *stream);

/* ------------------------------------------------------ error count */
/* compute_ber of Listing 1: for each codeword, bit errors = popcount over
 * the k information bits of ref XOR hat; block error = any bit error.
 * counts (device int64[5]) accumulates {info bits, bit errors, blocks,
 * block errors, sum of iters} (iters may be NULL: the last term is then 0).
 * ref, hat: device [B][ceil(k/32)] packed bits. */
int sim_count(const uint32_t *ref, const uint32_t *hat, const int32_t *iters, int64_t B, int k,
              int64_t *counts, void *stream);

/* ------------------------- demapper with prior, EXIT charts */
/* The feature list of the paper names a demapper with prior and EXIT chart
 * simulations (Section III, list of FEC features). These entry points close
 * the bit-interleaved coded modulation loop with iterative demapping and
 * decoding (BICM-ID) and measure extrinsic information transfer.
 *
 * sim_codewords: the codewords sim_tx transmits for the same (code, seed, cw0,
 * B) -- same source bits, same encoder -- packed into cw_out (device)
 * [B][ceil(n/32)]: bit v of codeword b is bit (v mod 32) of word v/32 (all n
 * positions, punctured and untransmitted ones included). */
int sim_codewords(ldpcx_code_t code, uint64_t seed, uint64_t cw0, int64_t B, uint32_t *cw_out, void *stream);

/* demap_app with a-priori LLRs La (same layout as llr_out; NULL = all zero).
 * With label bits b_j(x) of point x, the metric of x is
 *   -|y-x|^2/N0 + sum_j (1 - 2 b_j(x)) La_j / 2
 * (log prior of x up to a constant, L = ln P(b=0)/P(b=1)), and
 *   out = LDPCX_DEMAP_OUT_APP:       LSE_{b_i=0} - LSE_{b_i=1} of the metric
 *         LDPCX_DEMAP_OUT_EXTRINSIC: the same with bit i's own prior term
 *                                    left out (= APP - La_i)
 * (max instead of LSE for LDPCX_DEMAP_MAXLOG), per I/Q dimension (exact for
 * Gray square QAM: the prior and distance terms of the other dimension
 * cancel), clamped to [-clamp, clamp]. Arguments as demap_app. */
#define LDPCX_DEMAP_OUT_APP 0
#define LDPCX_DEMAP_OUT_EXTRINSIC 1
int demap_app_prior(const float *y, const float *no, int64_t no_stride, int64_t B, int64_t syms_per_cw, int m,
                    int method, float clamp, const float *llr_prior, int out_mode, float *llr_out, void *stream);

/* A-priori LLRs of the consistent Gaussian model of EXIT analysis:
 *   L = (sigma^2 / 2)(1 - 2 c) + sigma g,
 * c = bit (bit_off + t) of the packed row bits[b * bits_stride + ...] (words,
 * bit order as sim_codewords), g standard Gaussian by Box-Muller from Philox
 * stream 2 with key (seed) and counter (t/4, (cw0 + b) lo32, hi32, 2), words
 * as in sim_tx (Gaussian t uses block t/4: (x0,x1) for t mod 4 in {0,1},
 * (x2,x3) for {2,3}). out (device) [B][N] float. sigma >= 0. */
int llr_apriori(const uint32_t *bits, int64_t bits_stride, int64_t bit_off, int64_t B, int64_t N, float sigma,
                uint64_t seed, uint64_t cw0, float *out, void *stream);

/* Mutual information estimate between bits and LLRs (time average, valid
 * for consistent LLRs): acc[0] += sum over b, t of log2(1 + exp(-(1 - 2c) L)),
 * acc[1] += B N, so that I = 1 - acc[0] / acc[1]. llr (device) [B][N]; bits
 * as llr_apriori; acc (device) double[2], accumulated (float64 atomics: the
 * summation order is not fixed). */
int llr_mutual_info(const float *llr, int64_t B, int64_t N, const uint32_t *bits, int64_t bits_stride,
                    int64_t bit_off, double *acc, void *stream);

/* Extrinsic LLRs of a decode on the transmitted positions:
 *   out[b][t] = app[b][p0 + t] - clip(llr_in[b][t]),  t < n_tx,
 * app (device) [B][n] from ldpc_bp_decode's llr_out, llr_in (device) [B][n_tx]
 * its channel input, clip = clamping to [-clamp, clamp] as the decoder does
 * with its input (pass the decode's clamp); out (device) [B][n_tx], clamped
 * to [-clamp, clamp]. */
int ldpc_extrinsic(ldpcx_code_t code, const float *app, const float *llr_in, int64_t B, float clamp, float *out,
                   void *stream);

/* --------------- trainable constellation, end-to-end gradients */
/* Listing 2 of the paper makes the constellation trainable and learns it
 * end to end through mapper, AWGN and demapper with a binary cross-entropy
 * loss. These entry points run that chain and its adjoint with a constellation
 * given as 2^m complex points: point l has label bits b_j = (l >> (m-1-j)) & 1
 * (b_0 the most significant; the Gray QAM of sim_tx puts its point with label
 * l there). m in {2, 4, 6, 8}; points (device) [2^m][2] float (re, im), used as
 * given (normalise them to the wanted energy first).
 *
 * sim_tx_points: sim_tx with the constellation `points` -- same source bits,
 * encoder and AWGN draws; symbol s of codeword b carries the transmitted bits
 * p0 + s m .. p0 + s m + m - 1 as its label. cw_out (device, or NULL) as
 * sim_codewords. */
int sim_tx_points(ldpcx_code_t code, uint64_t seed, uint64_t cw0, int64_t B, int m, const float *points,
                  const float *no, int64_t no_stride, float *y_out, uint32_t *cw_out, void *stream);

/* APP demapper over an arbitrary constellation (full 2-D sums, no
 * separability): L_i = LSE_{l: b_i(l)=0}(-|y - p_l|^2/N0) - LSE_{b_i(l)=1}(.)
 * (max for LDPCX_DEMAP_MAXLOG), clamped to [-clamp, clamp].
 * y (device) [B][S][2]; llr_out (device) [B][S*m]. */
int demap_points(const float *y, const float *no, int64_t no_stride, int64_t B, int64_t S, int m,
                 const float *points, int method, float clamp, float *llr_out, void *stream);

/* Adjoint of demap_points (exact method only) for the loss gradient
 * grad_llr (device) [B][S*m]: writes grad_y (device) [B][S][2] and ADDS to
 * grad_points (device) [2^m][2] (float atomics: the summation order is not
 * fixed). Outputs at the clamp have zero derivative. */
int demap_points_backward(const float *y, const float *no, int64_t no_stride, int64_t B, int64_t S, int m,
                          const float *points, float clamp, const float *grad_llr, float *grad_y,
                          float *grad_points, void *stream);

/* Adjoint of the mapper of sim_tx_points: ADDS grad_x[b][s] (device
 * [B][S][2], the gradient at the transmitted symbol; AWGN passes it
 * unchanged) to grad_points[label of symbol (b, s)]. cw (device) packed
 * codewords as sim_codewords; the labels are read from positions p0 + s m. */
int map_points_backward(ldpcx_code_t code, const uint32_t *cw, int64_t B, int m, const float *grad_x,
                        float *grad_points, void *stream);

/* Binary cross-entropy of LLRs against bits (Listing 2's loss; with
 * L = ln P0/P1 the logits are -L): loss_acc (device double[1]) +=
 * sum_{b,t} ln(1 + exp(-(1 - 2c) L)); grad_llr (device [B][N], or NULL) =
 * scale * d/dL of that sum = -scale (1 - 2c) / (1 + exp((1 - 2c) L)).
 * bits, bits_stride, bit_off as llr_apriori. */
int llr_bce(const float *llr, int64_t B, int64_t N, const uint32_t *bits, int64_t bits_stride, int64_t bit_off,
            float scale, double *loss_acc, float *grad_llr, void *stream);

/* ----------------------------------- polar codes, SC/SCL decoding */
/* The paper lists polar codes with SC, SCL and SCL-CRC decoders among its FEC
 * features (Section III) and names the polar SCL decoder as a custom CUDA
 * kernel case (Section IV-A). Conventions:
 *  - N = 2^n (n in 2..10), encoder x = u F^{(x)n}, F = [[1,0],[1,1]], natural
 *    order; BPSK x -> 1 - 2x on a real AWGN channel, L = ln P0/P1;
 *  - information set: the K bit channels of smallest Bhattacharyya parameter
 *    z_i, where z_i applies to z0 = exp(-Es/N0 at the design point) the
 *    transforms z -> 2z - z^2 (bit 0 of i) or z -> z^2 (bit 1) for the bits of
 *    i from the most significant down (ties: the larger index); the 3GPP
 *    reliability sequence is not used (not available to this build);
 *  - the K information positions carry, in ascending order, K - r data bits
 *    and their r-bit CRC (generator g with the x^r term, remainder of the data
 *    most significant first, zero initial state); r = 0: no CRC;
 *  - SCL (L = 1: SC) in the LLR domain with f(a,b) = sgn(a) sgn(b) min(|a|,|b|),
 *    g(a,b,u) = b + (1-2u) a, path metric PM += |L_i| when the decision
 *    disagrees with sign(L_i) (decision 1 iff L < 0; frozen bits are 0);
 *    candidates (path l, bit b) ordered c = 2l + b, the L smallest (PM, c)
 *    survive in ascending c; CRC-aided selection of the smallest (PM, list
 *    index) among the paths that pass the CRC, else among all. */
typedef struct ldpcx_polar *ldpcx_polar_t;
int polar_build(int n, int K, float design_esn0_db, uint64_t crc_poly, int crc_r, ldpcx_polar_t *out);
int polar_free(ldpcx_polar_t code);
/* info_out (host, or NULL) [K] ascending information positions. */
int polar_info(ldpcx_polar_t code, int *N, int *K, int *crc_r, int32_t *info_out);
/* Transmitter: data bits (Philox stream 0, word w of codeword b from block
 * w/4 with counter (w/4, (cw0+b) lo32, hi32, 0), as sim_tx), CRC, encoder,
 * BPSK and AWGN (Philox stream 1 as sim_tx for m = 1).
 * y_out (device) [B][N] float; data_out (device, or NULL) [B][ceil((K-r)/32)]. */
int polar_sim_tx(ldpcx_polar_t code, uint64_t seed, uint64_t cw0, int64_t B, const float *no, int64_t no_stride,
                 float *y_out, uint32_t *data_out, void *stream);
/* CRC-aided SCL decoding of llr (device) [B][N] with list size L in 1..32.
 * data_out (device) [B][ceil((K-r)/32)] packed data bits of the chosen path;
 * pm_out (device, or NULL) [B] its path metric. */
int polar_scl_decode(ldpcx_polar_t code, const float *llr, int64_t B, int L, uint32_t *data_out, float *pm_out,
                     void *stream);

/* ------------------------------------------------------- rate matching */
/* Circular-buffer rate matching (the paper's Section III lists 5G LDPC with
 * rate matching among its FEC features), as the parameterised procedure of
 * the 5G NR LDPC chain; the start position per redundancy version is the
 * caller's (k0), so no standard table is built in:
 *   buffer w = the first ncb bits of the transmit layout: codeword positions
 *   p0, p0 + 1, ... (p0 = the code's punctured systematic bits,
 *   ldpcx_code_info.p0) without the filler bits of a shortened code
 *   (qc_ldpc_shorten); the 5G form keeps the fillers in the buffer as <NULL>
 *   entries and skips them while reading, which selects the same bits when its
 *   start counts the fillers before it; selection e_k = w[(k0 + k) mod ncb],
 *   k = 0 .. E-1 (E > ncb repeats, E < ncb punctures); interleaving over qm
 *   rows of E/qm columns, written by rows and read by columns:
 *   f[i qm + j] = e[j (E/qm) + i].
 * rate_match: cw (device) [B][ceil(n/32)] packed codeword bits (bit v of
 *   codeword b = bit v mod 32 of word v/32, as sim_codewords writes them) ->
 *   out (device) [B][ceil(E/32)] packed transmitted bits f.
 * rate_recover (soft combining): llr (device) [B][E] received LLRs in
 *   transmission order -> out (device) [B][ncb]: buffer position p holds the
 *   sum, in increasing k, of the e_k that came from it (0 where none did).
 *   A code built with n_tx = ncb and the same punct_cols decodes it directly.
 * Errors: LDPCX_E_INVAL for a null pointer with B > 0, B < 0, ncb outside
 * [1, n - p0 - n_fill], k0 outside [0, ncb), E < 1, qm not in {1,2,4,6,8} or
 * not dividing E. */
int rate_match(ldpcx_code_t code, const uint32_t *cw, int64_t B, int k0, int ncb, int E, int qm,
               uint32_t *out, void *stream);
int rate_recover(ldpcx_code_t code, const float *llr, int64_t B, int k0, int ncb, int E, int qm,
                 float *out, void *stream);

/* -------------------------------------------------- Monte-Carlo run */
/* A BER/BLER sweep over Eb/N0 points (the loop around Listing 1): for each
 * point, batches of `batch` codewords run sim_tx -> demap_app -> ldpc_bp_decode
 * -> sim_count on the device; codeword indices continue across batches and
 * points from cw0, so every draw is reproducible. N0 = 1/(r m 10^(EbN0/10)),
 * r = k/n_tx. A point ends after max_batches batches or once it has
 * min_bit_errors bit errors (checked between batches when > 0); the sweep
 * ends early after a point whose BER is below stop_ber (> 0). With
 * use_graph, a batch runs as two captured CUDA graphs, a front (transmitter,
 * demapper) and a back (decoder, count), over two buffer sets: the next
 * batch's front runs on a lower-priority stream while the current batch
 * decodes (a front started for a batch that does not follow -- after an
 * early end of a point or of the sweep -- is discarded); the counts equal
 * those of eager mode (use_graph = 0: one stream, launch by launch).
 * The sweep synchronises `stream` first and then runs on private streams of
 * its own; it returns after all its work has finished. */
typedef struct {
    ldpcx_code_t code;
    int m;                  /* bits per symbol: 1, 2, 4, 6, 8 */
    int demap_method;       /* LDPCX_DEMAP_* */
    float demap_clamp;      /* demapper LLR clamp */
    ldpcx_decode_opts dec;  /* decoder options (weights not allowed) */
    uint64_t seed;          /* Philox key */
    uint64_t cw0;           /* first codeword index */
    int64_t batch;          /* codewords per batch, >= 1 */
    int64_t max_batches;    /* batches per point, >= 1 */
    int64_t min_bit_errors; /* 0 = always run max_batches */
    const double *ebn0_db;  /* host [n_snr] */
    int n_snr;
    double stop_ber;        /* 0 = never stop early */
    int use_graph;          /* capture and replay one batch as a CUDA graph */
    const char *ckpt_path;  /* host path of the sweep's checkpoint file, or NULL (see sim_run) */
    int max_points;         /* run at most this many points in this call (0 = no limit) */
} ldpcx_sim_config;

typedef struct {
    int64_t bits, bit_errors, blocks, block_errors, iter_sum;
} ldpcx_sim_counts;

/* Workspace bytes sim_run needs for cfg (two sets of batch buffers + decoder
 * messages). */
int sim_workspace(const ldpcx_sim_config *cfg, size_t *ws_bytes);
/* Run the sweep. out: host [n_snr] counts (points not run are zero);
 * *points_run = points executed. Synchronises `stream` once per batch check
 * and once per point. ws: device, >= sim_workspace bytes, 256-byte aligned.
 * Checkpoint / resume: with ckpt_path set, the sweep's state is written to
 * that file after every finished point -- the points done with their int64
 * counts, the index of the next codeword and whether the sweep has ended --
 * as JSON, through a temporary file renamed over the old one, so an
 * interrupted run leaves the last complete state. A call that finds the file
 * restores it and continues with the next point from the saved codeword
 * index; since every draw is counter-based, the counts equal those of an
 * uninterrupted sweep bit for bit (and a sweep already ended returns its
 * saved counts without device work). The file carries a fingerprint of
 * everything that fixes the counts (code, channel, decoder, seed, cw0, batch
 * sizes, stopping rules, Eb/N0 points; not use_graph or max_points); a file
 * of another sweep, or one this library did not write, gives LDPCX_E_IO
 * before any device work, as does a write that fails. max_points > 0 ends
 * the call after that many points of this call (a long sweep run in slices).
 * out and *points_run then cover the restored and the new points. */
int sim_run(const ldpcx_sim_config *cfg, ldpcx_sim_counts *out, int *points_run,
            void *ws, size_t ws_bytes, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* LDPCX_H */
