// Monte-Carlo BER/BLER sweep (the loop around the paper's Listing 1): for each
// Eb/N0 point, batches of codewords run transmitter -> demapper -> decoder ->
// error count on the device. The codeword index lives in device memory and is
// advanced by a kernel at the end of each batch, so one captured CUDA graph of
// a batch replays for every batch of every point.
#include <math.h>

#include <vector>

#include "common.cuh"

namespace {

struct SimLayout {
    size_t y, llr, ref, hat, iters, no, cw0, acc, dec, total;
    int64_t S, kw;
    size_t dec_bytes;
};

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

int layout(const ldpcx_sim_config *c, SimLayout *L) {
    if (!c || !c->code) return LDPCX_E_INVAL;
    const ldpcx_code *code = c->code;
    if (code->enc == ldpcx::kEncNone) return LDPCX_E_UNSUPPORTED;  // the transmitter cannot encode it
    if (!(c->m == 1 || c->m == 2 || c->m == 4 || c->m == 6 || c->m == 8)) return LDPCX_E_INVAL;
    if (code->n_tx % c->m) return LDPCX_E_INVAL;
    if (c->batch < 1 || c->max_batches < 1 || c->n_snr < 0 || c->min_bit_errors < 0) return LDPCX_E_INVAL;
    if (c->n_snr > 0 && !c->ebn0_db) return LDPCX_E_INVAL;
    if (c->dec.weights) return LDPCX_E_INVAL;
    if (c->demap_method != LDPCX_DEMAP_EXACT && c->demap_method != LDPCX_DEMAP_MAXLOG) return LDPCX_E_INVAL;
    if (!(c->demap_clamp > 0.0f)) return LDPCX_E_INVAL;
    size_t dec = 0;
    int st = ldpc_bp_workspace(c->code, c->batch, &c->dec, &dec);
    if (st) return st;
    const int64_t B = c->batch;
    L->S = code->n_tx / c->m;
    L->kw = (code->k + 31) / 32;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t at = off;
        off = align256(off + bytes);
        return at;
    };
    L->dec = take(dec);
    L->y = take(sizeof(float) * (size_t)B * L->S * (c->m == 1 ? 1 : 2));
    L->llr = take(sizeof(float) * (size_t)B * code->n_tx);
    L->ref = take(sizeof(uint32_t) * (size_t)B * L->kw);
    L->hat = take(sizeof(uint32_t) * (size_t)B * L->kw);
    L->iters = take(sizeof(int32_t) * (size_t)B);
    L->no = take(sizeof(float));
    L->cw0 = take(sizeof(uint64_t));
    L->acc = take(sizeof(int64_t) * 5);
    L->dec_bytes = dec;
    L->total = off;
    return LDPCX_OK;
}

// One batch: transmitter, demapper, decoder, counter, advance of the codeword index.
int run_batch(const ldpcx_sim_config *c, const SimLayout &L, char *ws, cudaStream_t s) {
    const ldpcx_code *code = c->code;
    const int64_t B = c->batch;
    float *y = (float *)(ws + L.y), *llr = (float *)(ws + L.llr), *no = (float *)(ws + L.no);
    uint32_t *ref = (uint32_t *)(ws + L.ref), *hat = (uint32_t *)(ws + L.hat);
    int32_t *iters = (int32_t *)(ws + L.iters);
    uint64_t *cw0 = (uint64_t *)(ws + L.cw0);
    int64_t *acc = (int64_t *)(ws + L.acc);
    int st = ldpcx::launch_tx(c->code, c->seed, 0, cw0, B, c->m, no, 0, y, ref, s);
    if (!st) st = demap_app(y, no, 0, B, L.S, c->m, c->demap_method, c->demap_clamp, llr, s);
    if (!st) st = ldpc_bp_decode(c->code, llr, B, &c->dec, nullptr, hat, iters, ws + L.dec, L.dec_bytes, s);
    if (!st) st = sim_count(ref, hat, iters, B, code->k, acc, s);
    if (!st) st = ldpcx::launch_advance(cw0, (uint64_t)B, s);
    return st;
}

}  // namespace

extern "C" int sim_workspace(const ldpcx_sim_config *cfg, size_t *ws_bytes) {
    if (!ws_bytes) return LDPCX_E_INVAL;
    SimLayout L;
    int st = layout(cfg, &L);
    if (st) return st;
    *ws_bytes = L.total;
    return LDPCX_OK;
}

extern "C" int sim_run(const ldpcx_sim_config *c, ldpcx_sim_counts *out, int *points_run, void *ws_v,
                       size_t ws_bytes, void *stream) {
    SimLayout L;
    int st = layout(c, &L);
    if (st) return st;
    if (!out) return LDPCX_E_INVAL;
    if (!ws_v || ws_bytes < L.total || ((uintptr_t)ws_v & 255u)) return LDPCX_E_WORKSPACE;
    // Work runs on a private non-blocking stream (the legacy NULL stream cannot
    // be captured into a graph), ordered after the caller's stream.
    cudaStream_t caller = (cudaStream_t)stream, s = nullptr;
    if (cudaStreamSynchronize(caller) != cudaSuccess) return LDPCX_E_CUDA;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return LDPCX_E_CUDA;
    char *ws = (char *)ws_v;
    ldpcx::DevCode d;
    st = ldpcx::code_device(c->code, &d);  // upload tables before any capture
    if (st) {
        cudaStreamDestroy(s);
        return st;
    }
    for (int i = 0; i < c->n_snr; ++i) out[i] = ldpcx_sim_counts{0, 0, 0, 0, 0};
    if (points_run) *points_run = 0;

    uint64_t cw_start = c->cw0;
    if (cudaMemcpyAsync(ws + L.cw0, &cw_start, sizeof(cw_start), cudaMemcpyHostToDevice, s) != cudaSuccess) {
        cudaStreamDestroy(s);
        return LDPCX_E_CUDA;
    }

    cudaGraphExec_t exec = nullptr;
    cudaGraph_t graph = nullptr;
    const double r = (double)c->code->k / (double)c->code->n_tx;
    int result = LDPCX_OK;
    for (int i = 0; i < c->n_snr && result == LDPCX_OK; ++i) {
        const float n0 = (float)(1.0 / (r * (double)c->m * pow(10.0, c->ebn0_db[i] / 10.0)));
        if (cudaMemcpyAsync(ws + L.no, &n0, sizeof(n0), cudaMemcpyHostToDevice, s) != cudaSuccess ||
            cudaMemsetAsync(ws + L.acc, 0, sizeof(int64_t) * 5, s) != cudaSuccess) {
            result = LDPCX_E_CUDA;
            break;
        }
        int64_t counts[5] = {0, 0, 0, 0, 0};
        for (int64_t b = 0; b < c->max_batches; ++b) {
            if (c->use_graph) {
                if (!exec) {
                    if (cudaStreamSynchronize(s) != cudaSuccess) { result = LDPCX_E_CUDA; break; }
                    if (cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
                        result = LDPCX_E_CUDA;
                        break;
                    }
                    int cs = run_batch(c, L, ws, s);
                    cudaError_t ce = cudaStreamEndCapture(s, &graph);
                    if (cs || ce != cudaSuccess) { result = cs ? cs : LDPCX_E_CUDA; break; }
                    if (cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) { result = LDPCX_E_CUDA; break; }
                }
                if (cudaGraphLaunch(exec, s) != cudaSuccess) { result = LDPCX_E_CUDA; break; }
            } else {
                result = run_batch(c, L, ws, s);
                if (result) break;
            }
            if (c->min_bit_errors > 0) {
                if (cudaMemcpyAsync(counts, ws + L.acc, sizeof(counts), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                    cudaStreamSynchronize(s) != cudaSuccess) {
                    result = LDPCX_E_CUDA;
                    break;
                }
                if (counts[1] >= c->min_bit_errors) break;
            }
        }
        if (result) break;
        if (cudaMemcpyAsync(counts, ws + L.acc, sizeof(counts), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess) {
            result = LDPCX_E_CUDA;
            break;
        }
        out[i] = ldpcx_sim_counts{counts[0], counts[1], counts[2], counts[3], counts[4]};
        if (points_run) *points_run = i + 1;
        if (c->stop_ber > 0.0 && counts[0] > 0 && (double)counts[1] / (double)counts[0] < c->stop_ber) break;
    }
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (cudaStreamSynchronize(s) != cudaSuccess && result == LDPCX_OK) result = LDPCX_E_CUDA;
    cudaStreamDestroy(s);
    return result;
}
