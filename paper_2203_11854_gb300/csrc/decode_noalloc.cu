// ldpc_bp_decode_noalloc: the decoder for callers that cannot allocate device
// memory. Some callers cannot call cudaMalloc: a receiver that allocates every
// buffer once at start-up and forbids allocation on its real-time path, a host
// thread that must never block on the device (cudaMalloc may synchronise), or a
// component whose memory is owned by an allocator this library cannot reach.
// For them, this entry point keeps its scratch (the code tables and the
// check-to-variable messages) in a fixed array in device memory that is part
// of the library image: every GPU that loads the library holds it until the
// process exits. The caller still passes the inputs and outputs.
//
// The array is shared by every call on a device and keeps the previous call's
// contents; nothing in it needs clearing, because each call writes the tables
// first and the decoder writes every message before it reads it. Calls that
// overlap on the GPU (for example on two streams) race on the array.
#include <math.h>

#include <mutex>

#include "decode_kernels.cuh"

namespace {

using namespace ldpcx;
using namespace ldpcx::dec;

// The fixed scratch: tables, then messages (256-byte aligned sections).
static __device__ __align__(256) unsigned char g_noalloc_scratch[LDPCX_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxTableWords = 512;  // nnz + rows + 1 (a 46 x 68 base matrix needs 363)

struct TablesByValue {
    uint32_t w[kMaxTableWords];  // blk[nnz], then row_ptr[rows + 1]
    int count;
};

// Writes the code tables into the scratch; they arrive as a kernel parameter,
// so no copy from host memory and no staging buffer is needed.
__global__ void k_put_tables(const TablesByValue t, uint32_t *dst) {
    for (int i = threadIdx.x; i < t.count; i += blockDim.x) dst[i] = t.w[i];
}

// Device address of the scratch array on the current device: host code must
// not use the symbol itself (it names a host-side stand-in). Looked up once per
// device with that device current.
std::mutex g_mu;
unsigned char *g_scratch_addr[64] = {nullptr};

int scratch_address(unsigned char **out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) {
        cudaGetLastError();
        return LDPCX_E_NODEVICE;
    }
    if (dev >= 64) return LDPCX_E_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_addr[dev]) {
        void *ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) {
            cudaGetLastError();
            return LDPCX_E_CUDA;
        }
        g_scratch_addr[dev] = (unsigned char *)ptr;
    }
    *out = g_scratch_addr[dev];
    return LDPCX_OK;
}

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

// Codewords per CTA (same rule as ldpc_bp_decode): ~384 check-node threads,
// bounded by two CTAs per SM (layered) or one (flooding).
int codewords_per_cta(const ldpcx_code *c, bool layered) {
    const size_t per_cw = sizeof(float) * (size_t)c->n * (layered ? 1 : 2);
    const int tpc = layered ? 1 : flood_tpc(c->Z);
    const size_t budget = layered || tpc > 1 ? 105 * 1024 : 210 * 1024;
    int G = layered ? kMaxThreads / c->Z : 512 / (c->Z * tpc);
    if (G < 1) G = 1;
    while (G > 1 && per_cw * G > budget) --G;
    return G;
}

}  // namespace

extern "C" int ldpc_bp_decode_noalloc(ldpcx_code_t c, const float *llr_ch, int64_t B, const ldpcx_decode_opts *o,
                                      float *llr_out, uint32_t *bits_out, int32_t *iters_out, void *stream) {
    if (!c || B < 0 || (B > 0 && !llr_ch)) return LDPCX_E_INVAL;
    size_t msg_bytes = 0;
    int st = ldpc_bp_workspace(c, B, o, &msg_bytes);  // validates the options
    if (st) return st;
    if (B == 0) return LDPCX_OK;
    const int words = c->nnz + c->rows + 1;
    if (words > kMaxTableWords) return LDPCX_E_UNSUPPORTED;
    const size_t table_bytes = align256(sizeof(uint32_t) * (size_t)words);
    if (msg_bytes > (size_t)LDPCX_NOALLOC_SCRATCH_BYTES - table_bytes) return LDPCX_E_WORKSPACE;

    unsigned char *scratch = nullptr;
    st = scratch_address(&scratch);
    if (st) return st;
    unsigned int *status = status_word_decode();
    if (!status) return LDPCX_E_CUDA;

    const bool layered = o->algo == LDPCX_LAYERED_MINSUM || o->algo == LDPCX_LAYERED_SPA;
    const int algo = (o->algo == LDPCX_LAYERED_MINSUM || o->algo == LDPCX_FLOOD_MINSUM) ? kMinSum : kSpa;
    KernelFn fn = nullptr;
    if (!layered) fn = flooding_kernel(c->max_deg, algo, o->msg_prec, flood_tpc(c->Z));
    else if (o->msg_prec == kF32) fn = layered_kernel_f32(c->max_deg, algo, 1);
    else if (o->msg_prec == kF16) fn = layered_kernel_f16(c->max_deg, algo, 1);
    else fn = layered_kernel_fix6(c->max_deg, algo, 1);
    if (!fn) return LDPCX_E_UNSUPPORTED;

    cudaStream_t s = (cudaStream_t)stream;
    TablesByValue t;
    t.count = words;
    for (int i = 0; i < c->nnz; ++i) t.w[i] = c->blk[i];
    for (int i = 0; i <= c->rows; ++i) t.w[c->nnz + i] = (uint32_t)c->row_ptr[i];
    uint32_t *tables = reinterpret_cast<uint32_t *>(scratch);
    k_put_tables<<<1, 256, 0, s>>>(t, tables);
    if (cudaGetLastError() != cudaSuccess) return LDPCX_E_CUDA;

    const int64_t E = (int64_t)c->nnz * c->Z;
    Params p{};
    p.blk = tables;
    p.row_ptr = reinterpret_cast<const int32_t *>(tables + c->nnz);
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
    p.msg = scratch + table_bytes;
    p.msg_stride = (E + 127) / 128 * 128;
    p.weights = o->weights;
    p.llr_out = llr_out;
    p.bits_out = bits_out;
    p.iters_out = iters_out;
    p.B = B;
    p.G = codewords_per_cta(c, layered);
    p.pf_dist = 0;
    p.msg_size = o->msg_prec == kF32 ? 4 : o->msg_prec == kF16 ? 2 : 1;
    p.status = status;

    const size_t smem = smem_bytes(p, layered ? 1 : 2);
    if (smem > 227 * 1024) return LDPCX_E_UNSUPPORTED;
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return LDPCX_E_CUDA;
    const int threads = (p.G * p.Z * (layered ? 1 : flood_tpc(p.Z)) + 31) / 32 * 32;
    const int64_t grid = (B + p.G - 1) / p.G;
    fn<<<(unsigned)grid, threads, smem, s>>>(p);
    return cudaGetLastError() == cudaSuccess ? LDPCX_OK : LDPCX_E_CUDA;
}
