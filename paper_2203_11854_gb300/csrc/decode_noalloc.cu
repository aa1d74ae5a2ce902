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

#include "decode_plan.cuh"

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

}  // namespace

extern "C" int ldpc_bp_decode_noalloc(ldpcx_code_t c, const float *llr_ch, int64_t B, const ldpcx_decode_opts *o,
                                      float *llr_out, uint32_t *bits_out, int32_t *iters_out, void *stream) {
    if (!c || B < 0 || (B > 0 && !llr_ch)) return LDPCX_E_INVAL;
    size_t ws_unused = 0;
    int st = ldpc_bp_workspace(c, 0, o, &ws_unused);  // validates the options
    if (st) return st;
    if (B == 0) return LDPCX_OK;
    const int words = c->nnz + c->rows + 1;
    if (words > kMaxTableWords) return LDPCX_E_UNSUPPORTED;
    // the kernel ldpc_bp_decode would run, and the bytes each codeword's messages (or check-node state) take
    DecodePlan pl;
    st = decode_plan(c, o, &pl);
    if (st) return st;
    const int64_t per_cw = decode_plan_bytes_per_cw(c, o, pl);
    const int msg_size = o->msg_prec == LDPCX_MSG_F32 ? 4 : o->msg_prec == LDPCX_MSG_F16 ? 2 : 1;
    const size_t table_bytes = align256(sizeof(uint32_t) * (size_t)words);
    // B is bounded by the array before any product is formed
    const int64_t capacity =
        per_cw > 0 ? (int64_t)(((size_t)LDPCX_NOALLOC_SCRATCH_BYTES - table_bytes) / (size_t)per_cw) : 0;
    if (B > capacity) return LDPCX_E_WORKSPACE;
    if (per_cw % 16 != 0) return LDPCX_E_UNSUPPORTED;  // every codeword's state starts on a 16-byte boundary

    unsigned char *scratch = nullptr;
    st = scratch_address(&scratch);
    if (st) return st;

    cudaStream_t s = (cudaStream_t)stream;
    TablesByValue t;
    t.count = words;
    for (int i = 0; i < c->nnz; ++i) t.w[i] = c->blk[i];
    for (int i = 0; i <= c->rows; ++i) t.w[c->nnz + i] = (uint32_t)c->row_ptr[i];
    uint32_t *tables = reinterpret_cast<uint32_t *>(scratch);
    k_put_tables<<<1, 256, 0, s>>>(t, tables);
    if (cudaGetLastError() != cudaSuccess) return LDPCX_E_CUDA;

    // messages packed at the plan's own per-codeword size (check-node state for layered min-sum)
    const Params p = decode_params(c, tables, reinterpret_cast<const int32_t *>(tables + c->nnz), llr_ch, B, o,
                                   llr_out, bits_out, iters_out, scratch + table_bytes, per_cw / msg_size, nullptr,
                                   pl.layered);
    if (!p.status) return LDPCX_E_CUDA;
    return decode_launch(pl, c, p, B, stream);
}
