// Monte-Carlo BER/BLER sweep (the loop around the paper's Listing 1): for each
// Eb/N0 point, batches of codewords run transmitter -> demapper -> decoder ->
// error count on the device.
//
// Each batch's N0 and first codeword index are written by the host into the
// device copy its transmitter reads. The layered decoders demap while loading
// the channel (ldpc_bp_decode_qam); the flooding ones read the LLRs of a
// separate demapper launch. Eager mode runs a batch's launches one after
// another on one stream. Graph mode splits a batch into a front (transmitter,
// and the demapper when it is separate, into one of two buffer sets, with that
// set's N0 and first codeword index written by the host) and a back (decoder +
// error count from that set), captured once per set as four CUDA graphs. The front of the next batch runs on a second,
// lower-priority stream while the current batch decodes, so it fills the SM
// slots the decoder's last wave leaves idle. The next batch is guessed before
// the host has read the current counts (the same point, or the next point after
// its last batch); a wrong guess (a point ended by min_bit_errors or a sweep
// ended by stop_ber) discards that front and runs the right one. Codeword
// indices follow the batches actually counted, so both modes give the same
// counts.
#include <errno.h>
#include <inttypes.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <string>
#include <vector>

#include "common.cuh"

namespace {

// ---------------------------------------------------------------- checkpoints
// FNV-1a (64 bit) over everything that fixes a sweep's counts.
struct Fnv {
    uint64_t h = 0xcbf29ce484222325ull;
    void bytes(const void *p, size_t n) {
        const unsigned char *b = (const unsigned char *)p;
        for (size_t i = 0; i < n; ++i) {
            h ^= b[i];
            h *= 0x100000001b3ull;
        }
    }
    template <typename T> void put(const T &v) { bytes(&v, sizeof(v)); }
};

uint64_t fingerprint(const ldpcx_sim_config *c) {
    Fnv f;
    const ldpcx_code *code = c->code;
    const int shape[] = {code->Z, code->rows, code->cols, code->kb, code->n, code->k, code->n_tx, code->p0,
                         code->n_fill};
    f.bytes(shape, sizeof(shape));
    f.bytes(code->S.data(), sizeof(int16_t) * code->S.size());
    f.put(c->m);
    f.put(c->demap_method);
    f.put(c->demap_clamp);
    f.put(c->dec.algo);
    f.put(c->dec.iters);
    f.put(c->dec.msg_prec);
    f.put(c->dec.early_stop);
    f.put(c->dec.offset);
    f.put(c->dec.clamp);
    f.put(c->seed);
    f.put(c->cw0);
    f.put(c->batch);
    f.put(c->max_batches);
    f.put(c->min_bit_errors);
    f.put(c->stop_ber);
    f.put(c->n_snr);
    for (int i = 0; i < c->n_snr; ++i) f.put(c->ebn0_db[i]);
    return f.h;
}

struct Ckpt {
    uint64_t fp = 0, next_cw = 0;
    int next_point = 0, finished = 0;
    std::vector<ldpcx_sim_counts> pts;
};

const char *kCkptFormat = "ldpcx-sim-checkpoint";

// Write the state as JSON, one item per line, to path + ".tmp", then rename it
// over path (atomic on POSIX file systems: a reader sees the old or the new state).
int write_ckpt(const char *path, const ldpcx_sim_config *c, const Ckpt &k) {
    const std::string tmp = std::string(path) + ".tmp";
    FILE *f = fopen(tmp.c_str(), "w");
    if (!f) return LDPCX_E_IO;
    bool ok = fprintf(f, "{\n \"format\": \"%s\",\n \"version\": 1,\n \"fingerprint\": \"%016" PRIx64 "\",\n",
                      kCkptFormat, k.fp) > 0;
    ok = ok && fprintf(f, " \"next_point\": %d,\n \"next_cw\": %" PRIu64 ",\n \"finished\": %d,\n \"points\": [\n",
                       k.next_point, k.next_cw, k.finished) > 0;
    for (int i = 0; ok && i < k.next_point; ++i) {
        const ldpcx_sim_counts &q = k.pts[(size_t)i];
        ok = fprintf(f,
                     "  {\"ebn0_db\": %.17g, \"bits\": %" PRId64 ", \"bit_errors\": %" PRId64 ", \"blocks\": %" PRId64
                     ", \"block_errors\": %" PRId64 ", \"iter_sum\": %" PRId64 "}%s\n",
                     c->ebn0_db[i], q.bits, q.bit_errors, q.blocks, q.block_errors, q.iter_sum,
                     i + 1 < k.next_point ? "," : "") > 0;
    }
    ok = ok && fprintf(f, " ]\n}\n") > 0;
    ok = (fflush(f) == 0) && ok;
    ok = (fclose(f) == 0) && ok;
    if (!ok || rename(tmp.c_str(), path) != 0) {
        remove(tmp.c_str());
        return LDPCX_E_IO;
    }
    return LDPCX_OK;
}

// Read a checkpoint this library wrote for the sweep with fingerprint fp:
// LDPCX_OK (loaded), 1 (no file), LDPCX_E_IO (unreadable, malformed or of another sweep).
int read_ckpt(const char *path, const ldpcx_sim_config *c, uint64_t fp, Ckpt *k) {
    FILE *f = fopen(path, "r");
    if (!f) return errno == ENOENT ? 1 : LDPCX_E_IO;
    std::vector<std::string> lines;
    char buf[512];
    while (fgets(buf, sizeof(buf), f)) lines.emplace_back(buf);
    fclose(f);
    if (lines.size() < 9) return LDPCX_E_IO;
    char fmt[64] = {0};
    int version = 0;
    unsigned long long fpv = 0, ncw = 0;
    if (lines[0] != "{\n" || sscanf(lines[1].c_str(), " \"format\": \"%63[^\"]\",", fmt) != 1 || strcmp(fmt, kCkptFormat) ||
        sscanf(lines[2].c_str(), " \"version\": %d,", &version) != 1 || version != 1 ||
        sscanf(lines[3].c_str(), " \"fingerprint\": \"%16llx\",", &fpv) != 1 || fpv != fp ||
        sscanf(lines[4].c_str(), " \"next_point\": %d,", &k->next_point) != 1 ||
        sscanf(lines[5].c_str(), " \"next_cw\": %llu,", &ncw) != 1 ||
        sscanf(lines[6].c_str(), " \"finished\": %d,", &k->finished) != 1 || lines[7] != " \"points\": [\n")
        return LDPCX_E_IO;
    if (k->next_point < 0 || k->next_point > c->n_snr || (k->finished != 0 && k->finished != 1)) return LDPCX_E_IO;
    if (lines.size() != (size_t)k->next_point + 10) return LDPCX_E_IO;
    k->fp = fpv;
    k->next_cw = ncw;
    k->pts.assign((size_t)k->next_point, ldpcx_sim_counts{0, 0, 0, 0, 0});
    for (int i = 0; i < k->next_point; ++i) {
        double eb = 0.0;
        long long v[5] = {0, 0, 0, 0, 0};
        if (sscanf(lines[(size_t)8 + i].c_str(),
                   "  {\"ebn0_db\": %lf, \"bits\": %lld, \"bit_errors\": %lld, \"blocks\": %lld, \"block_errors\": %lld, "
                   "\"iter_sum\": %lld}",
                   &eb, &v[0], &v[1], &v[2], &v[3], &v[4]) != 6 ||
            eb != c->ebn0_db[i])
            return LDPCX_E_IO;
        k->pts[(size_t)i] = ldpcx_sim_counts{v[0], v[1], v[2], v[3], v[4]};
    }
    if (lines[(size_t)8 + k->next_point] != " ]\n" || lines[(size_t)9 + k->next_point] != "}\n") return LDPCX_E_IO;
    return LDPCX_OK;
}

struct SimLayout {
    size_t y[2], llr[2], ref[2], no[2], cw0[2];
    size_t hat, iters, acc, dec, total;
    int64_t S, kw;
    size_t dec_bytes;
};

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

// The layered decoders take the received symbols and demap them while loading
// the channel (ldpc_bp_decode_qam, the same results as demap_app then
// ldpc_bp_decode); the flooding decoders read LLRs, which the front writes.
bool fused_demap(const ldpcx_sim_config *c) {
    return c->dec.algo == LDPCX_LAYERED_MINSUM || c->dec.algo == LDPCX_LAYERED_SPA;
}

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
    for (int s = 0; s < 2; ++s) {
        L->y[s] = take(sizeof(float) * (size_t)B * L->S * (c->m == 1 ? 1 : 2));
        L->llr[s] = fused_demap(c) ? 0 : take(sizeof(float) * (size_t)B * code->n_tx);
        L->ref[s] = take(sizeof(uint32_t) * (size_t)B * L->kw);
        L->no[s] = take(sizeof(float));
        L->cw0[s] = take(sizeof(uint64_t));
    }
    L->hat = take(sizeof(uint32_t) * (size_t)B * L->kw);
    L->iters = take(sizeof(int32_t) * (size_t)B);
    L->acc = take(sizeof(int64_t) * 5);
    L->dec_bytes = dec;
    L->total = off;
    return LDPCX_OK;
}

// Front of a batch into buffer set s: transmitter (codewords from the set's
// device index) and, for the flooding decoders, the demapper.
int run_front(const ldpcx_sim_config *c, const SimLayout &L, char *ws, int s, cudaStream_t st) {
    float *y = (float *)(ws + L.y[s]), *llr = (float *)(ws + L.llr[s]), *no = (float *)(ws + L.no[s]);
    uint32_t *ref = (uint32_t *)(ws + L.ref[s]);
    const uint64_t *cw0 = (const uint64_t *)(ws + L.cw0[s]);
    int r = ldpcx::launch_tx(c->code, c->seed, 0, cw0, c->batch, c->m, no, 0, y, ref, st);
    if (!r && !fused_demap(c)) r = demap_app(y, no, 0, c->batch, L.S, c->m, c->demap_method, c->demap_clamp, llr, st);
    return r;
}

// Back of a batch from buffer set s: decoder (with the demapper fused into it
// for the layered schedules) and error count into the point's counters.
int run_back(const ldpcx_sim_config *c, const SimLayout &L, char *ws, int s, cudaStream_t st) {
    uint32_t *ref = (uint32_t *)(ws + L.ref[s]), *hat = (uint32_t *)(ws + L.hat);
    int32_t *iters = (int32_t *)(ws + L.iters);
    int r;
    if (fused_demap(c))
        r = ldpc_bp_decode_qam(c->code, (const float *)(ws + L.y[s]), (const float *)(ws + L.no[s]), 0, c->batch,
                               c->m, c->demap_method, c->demap_clamp, &c->dec, nullptr, hat, iters, ws + L.dec,
                               L.dec_bytes, st);
    else
        r = ldpc_bp_decode(c->code, (const float *)(ws + L.llr[s]), c->batch, &c->dec, nullptr, hat, iters,
                           ws + L.dec, L.dec_bytes, st);
    if (!r) r = sim_count(ref, hat, iters, c->batch, c->code->k, (int64_t *)(ws + L.acc), st);
    return r;
}

float n0_of(const ldpcx_sim_config *c, int point) {
    const double r = (double)c->code->k / (double)c->code->n_tx;
    return (float)(1.0 / (r * (double)c->m * pow(10.0, c->ebn0_db[point] / 10.0)));
}

// Owner of the streams, events and graphs of one sweep.
struct Runtime {
    cudaStream_t back = nullptr, front = nullptr;
    cudaEvent_t fdone[2] = {nullptr, nullptr}, bdone[2] = {nullptr, nullptr};
    cudaGraphExec_t fexec[2] = {nullptr, nullptr}, bexec[2] = {nullptr, nullptr};
    ~Runtime() {
        if (back) cudaStreamSynchronize(back);  // nothing of the sweep is left in flight
        if (front) cudaStreamSynchronize(front);
        for (int s = 0; s < 2; ++s) {
            if (fexec[s]) cudaGraphExecDestroy(fexec[s]);
            if (bexec[s]) cudaGraphExecDestroy(bexec[s]);
            if (fdone[s]) cudaEventDestroy(fdone[s]);
            if (bdone[s]) cudaEventDestroy(bdone[s]);
        }
        if (back) cudaStreamDestroy(back);
        if (front) cudaStreamDestroy(front);
    }
};

// Capture fn(s, stream) into an executable graph.
template <typename F> int capture(cudaStream_t st, cudaGraphExec_t *exec, F fn) {
    if (cudaStreamBeginCapture(st, cudaStreamCaptureModeRelaxed) != cudaSuccess) return LDPCX_E_CUDA;
    const int cs = fn();
    cudaGraph_t g = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(st, &g);
    if (cs || ce != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return cs ? cs : LDPCX_E_CUDA;
    }
    const cudaError_t ie = cudaGraphInstantiate(exec, g, 0);
    cudaGraphDestroy(g);
    return ie == cudaSuccess ? LDPCX_OK : LDPCX_E_CUDA;
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
    if (!out || c->max_points < 0) return LDPCX_E_INVAL;
    if (!ws_v || ws_bytes < L.total || ((uintptr_t)ws_v & 255u)) return LDPCX_E_WORKSPACE;
    // a saved state of this sweep: read it before any device work
    Ckpt ck;
    ck.fp = c->ckpt_path ? fingerprint(c) : 0;
    int first = 0;
    uint64_t cw_next = c->cw0;  // index of the next batch's first codeword
    auto restore = [&]() {
        for (int i = 0; i < c->n_snr; ++i) out[i] = i < ck.next_point ? ck.pts[(size_t)i] : ldpcx_sim_counts{0, 0, 0, 0, 0};
        if (points_run) *points_run = ck.next_point;
    };
    if (c->ckpt_path) {
        Ckpt saved;
        const int rs = read_ckpt(c->ckpt_path, c, ck.fp, &saved);
        if (rs < 0) return rs;
        if (rs == LDPCX_OK) {
            ck = saved;
            if (ck.finished || ck.next_point >= c->n_snr) {  // nothing left to run
                restore();
                return LDPCX_OK;
            }
            first = ck.next_point;
            cw_next = ck.next_cw;
        }
    }
    // Work runs on private non-blocking streams (the legacy NULL stream cannot
    // be captured into a graph), ordered after the caller's stream.
    if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return LDPCX_E_CUDA;
    Runtime rt;
    int lo = 0, hi = 0;
    cudaDeviceGetStreamPriorityRange(&lo, &hi);  // hi: the numerically smallest, highest priority
    if (cudaStreamCreateWithPriority(&rt.back, cudaStreamNonBlocking, hi) != cudaSuccess ||
        cudaStreamCreateWithPriority(&rt.front, cudaStreamNonBlocking, lo) != cudaSuccess)
        return LDPCX_E_CUDA;
    for (int s = 0; s < 2; ++s)
        if (cudaEventCreateWithFlags(&rt.fdone[s], cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&rt.bdone[s], cudaEventDisableTiming) != cudaSuccess)
            return LDPCX_E_CUDA;
    char *ws = (char *)ws_v;
    ldpcx::DevCode d;
    st = ldpcx::code_device(c->code, &d);  // upload tables before any capture
    if (st) return st;
    restore();  // outputs: the restored points, zeros for the rest
    const bool graph = c->use_graph != 0;
    const int64_t B = c->batch;

    // Launch the front of batch (point, index cw) into set s: N0 and the first
    // codeword index are written on the front stream, after the set's last back.
    std::vector<float> n0_host(2);
    std::vector<uint64_t> cw_host(2);
    auto front = [&](int s, int point, uint64_t cw) -> int {
        cudaStream_t fs = graph ? rt.front : rt.back;
        n0_host[s] = n0_of(c, point);
        cw_host[s] = cw;
        if (graph && cudaStreamWaitEvent(fs, rt.bdone[s], 0) != cudaSuccess) return LDPCX_E_CUDA;
        if (cudaMemcpyAsync(ws + L.no[s], &n0_host[s], sizeof(float), cudaMemcpyHostToDevice, fs) != cudaSuccess ||
            cudaMemcpyAsync(ws + L.cw0[s], &cw_host[s], sizeof(uint64_t), cudaMemcpyHostToDevice, fs) != cudaSuccess)
            return LDPCX_E_CUDA;
        int r;
        if (graph) {
            if (!rt.fexec[s]) {
                if (cudaStreamSynchronize(fs) != cudaSuccess) return LDPCX_E_CUDA;
                r = capture(fs, &rt.fexec[s], [&] { return run_front(c, L, ws, s, fs); });
                if (r) return r;
            }
            r = cudaGraphLaunch(rt.fexec[s], fs) == cudaSuccess ? LDPCX_OK : LDPCX_E_CUDA;
        } else {
            r = run_front(c, L, ws, s, fs);
        }
        if (!r && cudaEventRecord(rt.fdone[s], fs) != cudaSuccess) r = LDPCX_E_CUDA;
        return r;
    };
    auto back = [&](int s) -> int {
        if (graph && cudaStreamWaitEvent(rt.back, rt.fdone[s], 0) != cudaSuccess) return LDPCX_E_CUDA;
        int r;
        if (graph) {
            if (!rt.bexec[s]) {
                if (cudaStreamSynchronize(rt.back) != cudaSuccess) return LDPCX_E_CUDA;
                r = capture(rt.back, &rt.bexec[s], [&] { return run_back(c, L, ws, s, rt.back); });
                if (r) return r;
            }
            r = cudaGraphLaunch(rt.bexec[s], rt.back) == cudaSuccess ? LDPCX_OK : LDPCX_E_CUDA;
        } else {
            r = run_back(c, L, ws, s, rt.back);
        }
        if (!r && cudaEventRecord(rt.bdone[s], rt.back) != cudaSuccess) r = LDPCX_E_CUDA;
        return r;
    };
    // Pending front: the set it fills and the batch it holds (point, index in point).
    struct Pending {
        bool on = false;
        int set = 0, point = 0;
        int64_t b = 0;
    } pend;
    int set = 0;
    int result = LDPCX_OK;
    for (int i = first; i < c->n_snr && result == LDPCX_OK; ++i) {
        if (c->max_points > 0 && i - first >= c->max_points) break;  // this call's slice is done
        if (cudaMemsetAsync(ws + L.acc, 0, sizeof(int64_t) * 5, rt.back) != cudaSuccess) {
            result = LDPCX_E_CUDA;
            break;
        }
        int64_t counts[5] = {0, 0, 0, 0, 0};
        for (int64_t b = 0; b < c->max_batches; ++b) {
            // the front of this batch: pending if the guess was right, else launched now
            if (!(pend.on && pend.point == i && pend.b == b)) {
                set = pend.on ? 1 - pend.set : set;  // a wrong guess leaves its set to finish in the background
                result = front(set, i, cw_next);
                if (result) break;
            } else {
                set = pend.set;
            }
            pend.on = false;
            cw_next += (uint64_t)B;
            result = back(set);
            if (result) break;
            // guess the next batch and start its front into the other set while this one decodes (submitted
            // after the back, so the decoder's CTAs are dispatched first)
            if (graph) {
                const bool more = b + 1 < c->max_batches;
                if (more || i + 1 < c->n_snr) {
                    pend = Pending{true, 1 - set, more ? i : i + 1, more ? b + 1 : 0};
                    result = front(pend.set, pend.point, cw_next);
                    if (result) break;
                }
            }
            if (c->min_bit_errors > 0) {
                if (cudaMemcpyAsync(counts, ws + L.acc, sizeof(counts), cudaMemcpyDeviceToHost, rt.back) !=
                        cudaSuccess ||
                    cudaStreamSynchronize(rt.back) != cudaSuccess) {
                    result = LDPCX_E_CUDA;
                    break;
                }
                if (counts[1] >= c->min_bit_errors) break;
            }
        }
        if (result) break;
        if (cudaMemcpyAsync(counts, ws + L.acc, sizeof(counts), cudaMemcpyDeviceToHost, rt.back) != cudaSuccess ||
            cudaStreamSynchronize(rt.back) != cudaSuccess) {
            result = LDPCX_E_CUDA;
            break;
        }
        out[i] = ldpcx_sim_counts{counts[0], counts[1], counts[2], counts[3], counts[4]};
        if (points_run) *points_run = i + 1;
        const bool stop = c->stop_ber > 0.0 && counts[0] > 0 && (double)counts[1] / (double)counts[0] < c->stop_ber;
        if (c->ckpt_path) {
            ck.pts.resize((size_t)i + 1);
            ck.pts[(size_t)i] = out[i];
            ck.next_point = i + 1;
            ck.next_cw = cw_next;
            ck.finished = stop || i + 1 == c->n_snr;
            result = write_ckpt(c->ckpt_path, c, ck);
            if (result) break;
        }
        if (stop) break;
    }
    if (cudaStreamSynchronize(rt.front) != cudaSuccess && result == LDPCX_OK) result = LDPCX_E_CUDA;
    if (cudaStreamSynchronize(rt.back) != cudaSuccess && result == LDPCX_OK) result = LDPCX_E_CUDA;
    return result;
}
