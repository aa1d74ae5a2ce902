// Host side of the decoders: argument checks, workspace sizing, kernel choice
// and launch of ldpc_bp_decode. Kernels live in decode_layered_*.cu and
// decode_flood.cu.
#include <math.h>

#include <algorithm>
#include <atomic>

#include "decode_plan.cuh"

namespace ldpcx {
namespace {

using namespace dec;

__device__ unsigned int g_status;

std::atomic<int> g_specialised{1};  // use compile-time-Z kernels when built
std::atomic<int> g_cns{1};          // layered min-sum keeps check-node state instead of per-edge messages
std::atomic<int> g_sched{1};        // ... with the full base graph's layer schedule compiled in

int sched_shape(const ldpcx_code *c) { return sched_shape_of(c->row_ptr.data(), c->rows, c->params.bg_shape); }

// Bytes of the check-node state of one codeword in format prec.
int64_t cns_bytes(const ldpcx_code *c, int prec) {
    const int32_t *rp = c->row_ptr.data();
    if (prec == kF32) return cns_bytes_per_cw<kF32>(rp, c->rows, c->Z);
    if (prec == kF16) return cns_bytes_per_cw<kF16>(rp, c->rows, c->Z);
    return cns_bytes_per_cw<kFix6>(rp, c->rows, c->Z);
}

KernelFn pick_kernel(int max_deg, bool layered, int algo, int prec, int zpt, int Z, bool qam) {
    if (!layered) return flooding_kernel(max_deg, algo, prec);
    if (zpt == 1 && g_specialised.load()) {
        KernelFn f = prec == kF32 ? layered_kernel_zc_f32(max_deg, algo, Z, qam)
                   : prec == kF16 ? layered_kernel_zc_f16(max_deg, algo, Z, qam)
                                  : layered_kernel_zc_fix6(max_deg, algo, Z, qam);
        if (f) return f;
    }
    if (prec == kF32) return layered_kernel_f32(max_deg, algo, zpt, qam);
    if (prec == kF16) return layered_kernel_f16(max_deg, algo, zpt, qam);
    return layered_kernel_fix6(max_deg, algo, zpt, qam);
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
    if (c->max_deg > 20 || c->n > 65535) return LDPCX_E_UNSUPPORTED;
    return LDPCX_OK;
}

std::atomic<int> g_pf_dist{0};
std::atomic<int> g_zpt{0};
std::atomic<int> g_cw_per_cta{0};  // 0 = automatic

// Flooding: the codewords per CTA, up to gmax, by a cost that follows the
// GB300 timings of Z = 8 and Z = 64 batches: the most codewords one SM decodes,
// ceil(CTAs / SMs) G (and at least its resident CTAs' G each, when the batch
// leaves an SM part empty), scaled up where a thread would have fewer than two
// check nodes per phase (latency left exposed); ties to the larger G. CTAs per
// SM from the threads (64 registers each) and the shared memory of one CTA.
int pick_G_flood(const ldpcx_code *c, int64_t B, int gmax) {
    const size_t per_cw = 2 * sizeof(float) * (size_t)c->n;
    const size_t tables = 2 * sizeof(uint32_t) * c->nnz + sizeof(int32_t) * (c->rows + c->n / c->Z + 2) + 64;
    const int64_t sms = sm_count();
    int best = 1;
    double best_cost = 1e300;
    for (int g = 1; g <= gmax; ++g) {
        const int threads = flood_threads(g, c->n);
        int per_sm = std::min(65536 / (threads * 64), 2048 / threads);
        per_sm = std::min<int>(per_sm, (int)((227 * 1024) / (per_cw * g + tables + 1024)));
        if (per_sm < 1) per_sm = 1;
        const int64_t ctas = (B + g - 1) / g;
        const int64_t on_sm = std::max<int64_t>((ctas + sms - 1) / sms, per_sm);
        const double nodes_per_thread = (double)g * c->rows * c->Z / threads;
        const double cost = (double)(on_sm * g) * std::max(1.0, 2.0 / nodes_per_thread);
        if (cost <= best_cost * (1.0 + 1e-9)) {
            best_cost = cost;
            best = g;
        }
    }
    return best;
}

// Codewords per CTA: enough check-node threads to fill ~384 threads (layered)
// or up to 32 codewords (flooding, whose threads loop over the CTA's check and
// variable nodes), bounded by the shared memory that keeps two CTAs per SM
// (layered; flooding where two fit) or one.
int pick_G(const ldpcx_code *c, bool layered, int64_t B) {
    const size_t per_cw = sizeof(float) * (size_t)c->n * (layered ? 1 : 2);
    const size_t budget = layered || per_cw <= 105 * 1024 ? 105 * 1024 : 210 * 1024;
    int G = layered ? kMaxThreads / c->Z : 32;
    if (G < 1) G = 1;
    while (G > 1 && per_cw * G > budget) --G;
    const int want = g_cw_per_cta.load();
    if (want > 0) {
        if (want < G) G = want;  // autotuner: smaller tiles, more CTAs per SM
    } else if (!layered) {
        G = pick_G_flood(c, B, G);
    } else {
        // a small batch: fewer codewords per CTA, so that its CTAs (each a serial chain of row steps) spread
        // over about four per SM instead of crowding a few
        const int64_t spread = B / (4 * (int64_t)sm_count());
        if (spread < G) G = spread < 1 ? 1 : (int)spread;
    }
    return G;
}

  // check nodes per thread of the layered kernels: 0 = auto (1), 1, 2

}  // namespace

int tune_cw_per_cta() { return g_cw_per_cta.load(); }

unsigned int take_status_decode(cudaStream_t s) {
    unsigned int v = 0, zero = 0;
    if (cudaMemcpyFromSymbolAsync(&v, g_status, sizeof(v), 0, cudaMemcpyDeviceToHost, s) != cudaSuccess) return 0;
    cudaMemcpyToSymbolAsync(g_status, &zero, sizeof(zero), 0, cudaMemcpyHostToDevice, s);
    cudaStreamSynchronize(s);
    return v;
}

// Device address of the status word on the current device (looked up once per device).
unsigned int *status_word_decode() {
    static unsigned int *addr[64] = {nullptr};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    if (!addr[dev]) {
        void *a = nullptr;
        if (cudaGetSymbolAddress(&a, g_status) != cudaSuccess) return nullptr;
        addr[dev] = (unsigned int *)a;
    }
    return addr[dev];
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

namespace ldpcx {
namespace {

// Decode, optionally storing FP32 checkpoints of C^t (flooding only).
// Launch a compiled-schedule kernel: block table as a kernel parameter, one
// CTA per p.G codewords with kpt check nodes per thread.
int launch_sched(SchedFn sf, const ldpcx_code *c, const Params &p, int64_t B, int kpt, void *stream) {
    SchedTab tab;
    for (int i = 0; i < c->nnz; ++i) {
        const int col = (int)(c->blk[(size_t)i] >> 16), sh = (int)(c->blk[(size_t)i] & 0xFFFFu);
        tab.at[i] = make_int2(4 * (col * c->Z + sh), c->Z - sh);
    }
    const size_t smem = smem_bytes(p, 1);
    if (smem > 227 * 1024) return LDPCX_E_UNSUPPORTED;
    if (cudaFuncSetAttribute(sf, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return LDPCX_E_CUDA;
    const int64_t grid = (B + p.G - 1) / p.G;
    if (grid > 0x7FFFFFFF) return LDPCX_E_INVAL;
    sf<<<(unsigned)grid, (p.G * (p.Z / kpt) + 31) / 32 * 32, smem, (cudaStream_t)stream>>>(p, tab);
    return cuda_status(cudaGetLastError());
}

int decode_impl(ldpcx_code_t c, const float *llr_ch, int64_t B, const ldpcx_decode_opts *o, float *llr_out,
                uint32_t *bits_out, int32_t *iters_out, void *ws, size_t ws_bytes, float *ckpt, void *stream) {
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
    DecodePlan pl;
    st = decode_plan(c, o, &pl);
    if (st) return st;
    // the workspace holds per-edge messages; check-node state uses the same per-codeword stride
    const Params p = decode_params(c, d.blk, d.row_ptr, llr_ch, B, o, llr_out, bits_out, iters_out, ws,
                                   msg_stride(c), ckpt, pl.layered);
    if (!p.status) return LDPCX_E_CUDA;
    return decode_launch(pl, c, p, B, stream);
}

// The adjoint supports weighted flooding sum-product with FP32 messages and a
// fixed iteration count.
int check_differentiable(const ldpcx_code *c, const ldpcx_decode_opts *o) {
    int st = check_opts(c, o);
    if (st) return st;
    if (o->algo != LDPCX_FLOOD_SPA || o->msg_prec != LDPCX_MSG_F32 || o->early_stop) return LDPCX_E_UNSUPPORTED;
    if (c->n_fill) return LDPCX_E_UNSUPPORTED;  // the adjoint reads the channel LLRs in the unshortened layout
    return LDPCX_OK;
}

}  // namespace

int dec::decode_plan(const ldpcx_code *c, const ldpcx_decode_opts *o, DecodePlan *pl, bool qam) {
    *pl = DecodePlan{};
    const bool layered = o->algo == LDPCX_LAYERED_MINSUM || o->algo == LDPCX_LAYERED_SPA;
    const int algo = (o->algo == LDPCX_LAYERED_MINSUM || o->algo == LDPCX_FLOOD_MINSUM) ? kMinSum : kSpa;
    pl->layered = layered;
    int zpt = 1;
    if (layered) {
        const int want = g_zpt.load();
        zpt = (want == 2 && c->Z % 2 == 0) ? 2 : 1;
    }
    KernelFn fn = pick_kernel(c->max_deg, layered, algo, o->msg_prec, zpt, c->Z, qam);
    if (!fn && zpt == 2) {  // two check nodes per thread not built: fall back to one
        zpt = 1;
        fn = pick_kernel(c->max_deg, layered, algo, o->msg_prec, zpt, c->Z, qam);
    }
    if (!fn) return LDPCX_E_UNSUPPORTED;
    pl->fn = fn;
    pl->zpt = zpt;
    // layered sum-product on a full base graph: per-edge messages, compiled-in schedule
    if (layered && algo == kSpa && zpt == 1 && g_sched.load()) {
        // the per-edge kernel compiles the full schedule: truncated codes take the row table
        int bg = sched_shape(c);
        if (bg && c->rows != (bg == 1 ? Sched<1>::rows : Sched<2>::rows)) bg = 0;
        SchedFn sf = bg && c->nnz <= kSchedMaxBlocks
                         ? layered_edge_sched_kernel(bg, algo, o->msg_prec, g_specialised.load() ? c->Z : 0, qam)
                         : nullptr;
        if (sf) {
            pl->sf = sf;
            pl->kpt = 1;
            return LDPCX_OK;
        }
    }
    // layered min-sum: check-node state (the compiled schedule's format, or the row-table kernel's) when it
    // fits the per-edge workspace of a codeword
    const int64_t ws_cw = msg_stride(c) * (int64_t)msg_bytes(o->msg_prec);
    if (layered && algo == kMinSum && zpt == 1 && g_cns.load()) {
        const int zs = g_specialised.load() ? c->Z : 0;
        const int bg = g_sched.load() ? sched_shape(c) : 0;
        const bool trunc = bg && c->rows != (bg == 1 ? Sched<1>::rows : Sched<2>::rows);
        const int kpt = !trunc && g_zpt.load() == 2 && c->Z % 2 == 0 ? 2 : 1;  // check nodes per thread
        SchedFn sf = bg && c->nnz <= kSchedMaxBlocks ? layered_cns_sched_kernel(bg, o->msg_prec, zs, kpt, trunc, qam)
                                                     : nullptr;
        const int64_t sb = bg ? sched_state_bytes(bg, o->msg_prec, kpt, c->row_ptr.data(), c->rows, c->Z) : 0;
        if (sf && sb <= ws_cw) {
            pl->sf = sf;
            pl->kpt = kpt;
            pl->cns = true;
            pl->state_bytes = sb;
            return LDPCX_OK;
        }
        KernelFn f = cns_bytes(c, o->msg_prec) <= ws_cw ? layered_cns_kernel(c->max_deg, o->msg_prec, zs) : nullptr;
        if (f) {
            pl->fn = f;
            pl->cns = true;
            pl->state_bytes = cns_bytes(c, o->msg_prec);
        }
    }
    return LDPCX_OK;
}

int64_t dec::decode_plan_bytes_per_cw(const ldpcx_code *c, const ldpcx_decode_opts *o, const DecodePlan &pl) {
    return pl.cns ? pl.state_bytes : msg_stride(c) * (int64_t)msg_bytes(o->msg_prec);
}

dec::Params dec::decode_params(const ldpcx_code *c, const uint32_t *blk, const int32_t *row_ptr,
                               const float *llr_ch, int64_t B, const ldpcx_decode_opts *o, float *llr_out,
                               uint32_t *bits_out, int32_t *iters_out, void *msg, int64_t stride, float *ckpt,
                               bool layered) {
    Params p{};
    p.blk = blk;
    p.row_ptr = row_ptr;
    p.Z = c->Z;
    p.rows = c->rows;
    p.nnz = c->nnz;
    p.n = c->n;
    p.k = c->k;
    p.n_tx = c->n_tx;
    p.p0 = c->p0;
    p.nf = c->n_fill;
    p.iters = o->iters;
    p.early_stop = o->early_stop;
    p.offset = o->offset;
    p.clamp = o->clamp;
    p.phi_lo = (float)log1p(2.0 / expm1((double)o->clamp));
    p.llr = llr_ch;
    p.msg = msg;
    p.msg_stride = stride;
    p.weights = o->weights;
    p.ckpt = ckpt;
    p.ckpt_tstride = B * stride;
    p.ckpt_app_stride = ckpt_app_stride(c->n);
    p.llr_out = llr_out;
    p.bits_out = bits_out;
    p.iters_out = iters_out;
    p.B = B;
    p.G = pick_G(c, layered, B);
    p.pf_dist = layered ? g_pf_dist.load() : 0;
    p.msg_size = (int)msg_bytes(o->msg_prec);
    p.status = status_word_decode();
    set_int_constants(p);
    return p;
}

int dec::decode_launch(const DecodePlan &pl, const ldpcx_code *c, const Params &p, int64_t B, void *stream) {
    if (pl.sf) return launch_sched(pl.sf, c, p, B, pl.kpt, stream);
    const size_t smem = pl.cns ? cns_smem_bytes(p) : pl.layered ? smem_bytes(p, 1) : flood_smem_bytes(p);
    if (smem > 227 * 1024) return LDPCX_E_UNSUPPORTED;
    if (cudaFuncSetAttribute(pl.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return LDPCX_E_CUDA;
    int threads = pl.layered ? (p.G * (p.Z / pl.zpt) + 31) / 32 * 32 : flood_threads(p.G, p.n);
    const int64_t grid = (B + p.G - 1) / p.G;
    if (grid > 0x7FFFFFFF) return LDPCX_E_INVAL;
    pl.fn<<<(unsigned)grid, threads, smem, (cudaStream_t)stream>>>(p);
    return cuda_status(cudaGetLastError());
}

size_t ckpt_bytes(const ldpcx_code *c, int64_t B, int iters) {
    return sizeof(float) * (size_t)(iters > 1 ? iters - 1 : 1) * (size_t)B *
           (size_t)(msg_stride(c) + ckpt_app_stride(c->n));
}

}  // namespace ldpcx

extern "C" int ldpc_bp_decode(ldpcx_code_t c, const float *llr_ch, int64_t B, const ldpcx_decode_opts *o,
                              float *llr_out, uint32_t *bits_out, int32_t *iters_out, void *ws, size_t ws_bytes,
                              void *stream) {
    return ldpcx::decode_impl(c, llr_ch, B, o, llr_out, bits_out, iters_out, ws, ws_bytes, nullptr, stream);
}

extern "C" int ldpc_bp_decode_qam(ldpcx_code_t c, const float *y, const float *no, int64_t no_stride, int64_t B,
                                  int m, int demap_method, float demap_clamp, const ldpcx_decode_opts *o,
                                  float *llr_out, uint32_t *bits_out, int32_t *iters_out, void *ws, size_t ws_bytes,
                                  void *stream) {
    using namespace ldpcx;
    using namespace ldpcx::dec;
    if (!c || B < 0 || !valid_m(m) || (no_stride != 0 && no_stride != 1)) return LDPCX_E_INVAL;
    if (demap_method != LDPCX_DEMAP_EXACT && demap_method != LDPCX_DEMAP_MAXLOG) return LDPCX_E_INVAL;
    if (!(demap_clamp > 0.0f) || isinf(demap_clamp) || c->n_tx % m != 0) return LDPCX_E_INVAL;
    int st = check_opts(c, o);
    if (st) return st;
    // the flooding kernels read the channel LLRs again in every iteration
    if (o->algo != LDPCX_LAYERED_MINSUM && o->algo != LDPCX_LAYERED_SPA) return LDPCX_E_UNSUPPORTED;
    if (B == 0) return LDPCX_OK;
    if (!y || !no) return LDPCX_E_INVAL;
    size_t need = 0;
    ldpc_bp_workspace(c, B, o, &need);
    if (!ws || ws_bytes < need || ((uintptr_t)ws & 255u)) return LDPCX_E_WORKSPACE;
    DevCode d;
    st = code_device(c, &d);
    if (st) return st;
    DecodePlan pl;
    st = decode_plan(c, o, &pl, true);
    if (st) return st;
    Params p = decode_params(c, d.blk, d.row_ptr, nullptr, B, o, llr_out, bits_out, iters_out, ws, msg_stride(c),
                             nullptr, pl.layered);
    if (!p.status) return LDPCX_E_CUDA;
    p.sym = y;
    p.sym_no = no;
    p.sym_no_stride = no_stride;
    p.qam_m = m;
    p.demap_method = demap_method;
    p.demap_clamp = demap_clamp;
    p.qam_scale = qam_scale(m);
    return decode_launch(pl, c, p, B, stream);
}

namespace ldpcx {
namespace {
__global__ void k_phi(const float *x, float *out, int64_t n, int fast) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = fast == 2 ? dec::phi_bits(x[i] * dec::kLog2e) * dec::kLn2 : fast ? dec::phi_fast(x[i]) : dec::phi(x[i]);
}
}  // namespace
}  // namespace ldpcx

extern "C" int ldpcx_phi(const float *x, float *out, int64_t n, int fast, void *stream) {
    if (n < 0 || (n > 0 && (!x || !out)) || fast < 0 || fast > 2) return LDPCX_E_INVAL;
    if (n == 0) return LDPCX_OK;
    const int64_t blocks = std::min<int64_t>((n + 255) / 256, 4096);
    ldpcx::k_phi<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(x, out, n, fast);
    return ldpcx::cuda_status(cudaGetLastError());
}

extern "C" int ldpc_bp_msg_format(ldpcx_code_t c, const ldpcx_decode_opts *o, int *cn_state,
                                  int64_t *bytes_per_cw) {
    if (!c || !cn_state || !bytes_per_cw) return LDPCX_E_INVAL;
    int st = ldpcx::check_opts(c, o);
    if (st) return st;
    // the format the decoder would run (the same choice as ldpc_bp_decode)
    ldpcx::dec::DecodePlan pl;
    st = ldpcx::dec::decode_plan(c, o, &pl);
    if (st) return st;
    *cn_state = pl.cns ? 1 : 0;
    *bytes_per_cw = pl.cns ? pl.state_bytes : (int64_t)c->nnz * c->Z * (int64_t)ldpcx::msg_bytes(o->msg_prec);
    return LDPCX_OK;
}

extern "C" int ldpc_bp_ckpt_bytes(ldpcx_code_t c, int64_t B, const ldpcx_decode_opts *o, size_t *bytes) {
    if (!c || !bytes || B < 0) return LDPCX_E_INVAL;
    int st = ldpcx::check_differentiable(c, o);
    if (st) return st;
    *bytes = ldpcx::ckpt_bytes(c, B, o->iters);
    return LDPCX_OK;
}

extern "C" int ldpc_bp_decode_ckpt(ldpcx_code_t c, const float *llr_ch, int64_t B, const ldpcx_decode_opts *o,
                                   float *llr_out, uint32_t *bits_out, int32_t *iters_out, void *ws,
                                   size_t ws_bytes, void *ckpt, size_t ckpt_bytes, void *stream) {
    if (!c || B < 0) return LDPCX_E_INVAL;
    int st = ldpcx::check_differentiable(c, o);
    if (st) return st;
    if (B == 0) return LDPCX_OK;
    if (!ckpt || ckpt_bytes < ldpcx::ckpt_bytes(c, B, o->iters) || ((uintptr_t)ckpt & 15u))
        return LDPCX_E_WORKSPACE;
    return ldpcx::decode_impl(c, llr_ch, B, o, llr_out, bits_out, iters_out, ws, ws_bytes, (float *)ckpt, stream);
}

extern "C" int ldpcx_tune_set(int key, int value) {
    if (key == LDPCX_TUNE_L2_PREFETCH) {
        if (value < 0 || value > 16) return LDPCX_E_INVAL;
        g_pf_dist.store(value);
        return LDPCX_OK;
    }
    if (key == LDPCX_TUNE_ZPT) {
        if (value < 0 || value > 2) return LDPCX_E_INVAL;
        g_zpt.store(value);
        return LDPCX_OK;
    }
    if (key == LDPCX_TUNE_CW_PER_CTA) {
        if (value < 0 || value > kMaxThreads) return LDPCX_E_INVAL;
        g_cw_per_cta.store(value);
        return LDPCX_OK;
    }
    if (key == LDPCX_TUNE_SPECIALISED) {
        if (value < 0 || value > 1) return LDPCX_E_INVAL;
        g_specialised.store(value);
        return LDPCX_OK;
    }
    if (key == LDPCX_TUNE_CN_STATE) {
        if (value < 0 || value > 1) return LDPCX_E_INVAL;
        g_cns.store(value);
        return LDPCX_OK;
    }
    if (key == LDPCX_TUNE_SCHEDULE) {
        if (value < 0 || value > 1) return LDPCX_E_INVAL;
        g_sched.store(value);
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
    if (key == LDPCX_TUNE_ZPT) {
        *value = g_zpt.load();
        return LDPCX_OK;
    }
    if (key == LDPCX_TUNE_CW_PER_CTA) {
        *value = g_cw_per_cta.load();
        return LDPCX_OK;
    }
    if (key == LDPCX_TUNE_SPECIALISED) {
        *value = g_specialised.load();
        return LDPCX_OK;
    }
    if (key == LDPCX_TUNE_CN_STATE) {
        *value = g_cns.load();
        return LDPCX_OK;
    }
    if (key == LDPCX_TUNE_SCHEDULE) {
        *value = g_sched.load();
        return LDPCX_OK;
    }
    return LDPCX_E_INVAL;
}
