// Mixed-size batch in one persistent launch: resident CTAs pull work items
// (up to G codewords of one code) from a device queue, longest first, and run
// a layered tile on each: for min-sum the compiled-schedule check-node-state
// tile (decode_cns_sched.cuh) when the code is one of the 5G shapes, full or
// truncated, else the row-table one (decode_cns.cuh); the per-edge tile
// (decode_kernels.cuh) for sum-product. Message scratch
// is one slot per resident CTA, sized for the largest item.
#include <math.h>

#include <algorithm>
#include <vector>

#include "decode_cns_sched.cuh"

namespace ldpcx {
namespace {

using namespace dec;

struct GroupDesc {
    const uint32_t *blk;
    const int32_t *row_ptr;
    int Z, rows, nnz, n, k, n_tx, p0, G;
    int nf;   // filler bits of a shortened code
    int cns;  // min-sum with check-node state in the message slot
    int bg;   // 1 or 2: the rows follow that shape's base graph (compiled schedule); 0: row table
    int64_t B, stride;
    const float *llr;
    float *llr_out;
    uint32_t *bits;
    int32_t *iters;
};

struct Item {
    int group;
    int pad;
    int64_t cw_base;
};

struct MixedParams {
    const GroupDesc *groups;
    const Item *items;
    int n_items;
    int *head;         // queue head (zeroed before the launch)
    char *scratch;     // [grid][slot_bytes]
    int64_t slot_bytes;
    int iters, early_stop;
    float offset, clamp, phi_lo;
    unsigned int *status;
    unsigned k_one, k_two, k_four, k_two22, k_two31;  // as Params (opaque integer constants)
};

template <int DMAX, int ALGO, int PREC>
__global__ void __launch_bounds__(kMaxThreads, 2) k_mixed(const MixedParams m) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_item;
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(m.head, 1);
        __syncthreads();
        const int it = s_item;
        if (it >= m.n_items) break;
        const Item item = m.items[it];
        const GroupDesc gd = m.groups[item.group];
        Params p{};
        p.blk = gd.blk;
        p.row_ptr = gd.row_ptr;
        p.Z = gd.Z;
        p.rows = gd.rows;
        p.nnz = gd.nnz;
        p.n = gd.n;
        p.k = gd.k;
        p.n_tx = gd.n_tx;
        p.p0 = gd.p0;
        p.nf = gd.nf;
        p.iters = m.iters;
        p.early_stop = m.early_stop;
        p.offset = m.offset;
        p.clamp = m.clamp;
        p.phi_lo = m.phi_lo;
        p.llr = gd.llr;
        p.msg = m.scratch + (size_t)blockIdx.x * m.slot_bytes;
        p.msg_stride = gd.stride;
        p.llr_out = gd.llr_out;
        p.bits_out = gd.bits;
        p.iters_out = gd.iters;
        p.B = gd.B;
        p.G = gd.G;
        p.pf_dist = 0;
        p.msg_size = PREC == kF32 ? 4 : PREC == kF16 ? 2 : 1;
        p.status = m.status;
        p.k_one = m.k_one;
        p.k_two = m.k_two;
        p.k_four = m.k_four;
        p.k_two22 = m.k_two22;
        p.k_two31 = m.k_two31;
        p.k_neg4z = (unsigned)(-4 * gd.Z) * m.k_one;
        if constexpr (ALGO == kMinSum) {
            if (gd.cns && gd.bg) {
                // block table {4 (col Z + shift), Z - shift} in shared memory past the tile's own tables
                int2 *s_at = reinterpret_cast<int2 *>(
                    (reinterpret_cast<uintptr_t>(smem + smem_bytes(p, 1)) + 7) & ~(uintptr_t)7);
                for (int i = threadIdx.x; i < p.nnz; i += blockDim.x) {
                    const uint32_t bk = p.blk[i];
                    const int sh = (int)(bk & 0xFFFFu);
                    s_at[i] = make_int2(4 * ((int)(bk >> 16) * p.Z + sh), p.Z - sh);
                }
                if (gd.bg == 1) cns_sched_tile1<1, PREC, 0, true>(p, item.cw_base, item.cw_base, smem, s_at);
                else cns_sched_tile1<2, PREC, 0, true>(p, item.cw_base, item.cw_base, smem, s_at);
            } else if (gd.cns) {
                cns_tile<DMAX, PREC, 0>(p, item.cw_base, item.cw_base, smem);
            } else {
                layered_tile<DMAX, ALGO, PREC, 1, 0, kChLlr>(p, item.cw_base, item.cw_base, smem);
            }
        } else {
            layered_tile<DMAX, ALGO, PREC, 1, 0, kChLlr>(p, item.cw_base, item.cw_base, smem);
        }
        __syncthreads();  // every thread has read s_item before it is overwritten
    }
}

using MixedFn = void (*)(MixedParams);

template <int DMAX, int ALGO>
MixedFn mixed_prec(int prec) {
    if (prec == kF32) return k_mixed<DMAX, ALGO, kF32>;
    if (prec == kF16) return k_mixed<DMAX, ALGO, kF16>;
    if constexpr (ALGO == kMinSum) return k_mixed<DMAX, kMinSum, kFix6>;
    return nullptr;
}

MixedFn pick_mixed(int dmax, int algo, int prec) {
    if (dmax > 20) return nullptr;
    if (algo == kMinSum) return dmax <= 12 ? mixed_prec<12, kMinSum>(prec) : mixed_prec<20, kMinSum>(prec);
    return dmax <= 12 ? mixed_prec<12, kSpa>(prec) : mixed_prec<20, kSpa>(prec);
}

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

// Codewords per CTA for a code (same rule as ldpc_bp_decode's layered path,
// including the LDPCX_TUNE_CW_PER_CTA cap): the codewords of one work item.
int group_G(const ldpcx_code *c) {
    const size_t per_cw = sizeof(float) * (size_t)c->n;
    int G = kMaxThreads / c->Z;
    if (G < 1) G = 1;
    while (G > 1 && per_cw * G > 105 * 1024) --G;
    const int want = tune_cw_per_cta();
    if (want > 0 && want < G) G = want;
    return G;
}

int64_t stride_of(const ldpcx_code *c) {
    const int64_t E = (int64_t)c->nnz * c->Z;
    return (E + 127) / 128 * 128;
}

size_t tile_smem(const ldpcx_code *c, int G) {
    return sizeof(float) * (size_t)G * c->n + sizeof(uint32_t) * c->nnz + sizeof(int32_t) * (c->rows + 1) +
           2 * sizeof(int) * G;
}

// Shared memory of the check-node-state tile: the per-edge tile's plus the
// row slot offsets and the {offset, wrap} block table (cns_smem_bytes).
size_t cns_tile_smem(const ldpcx_code *c, int G) {
    return tile_smem(c, G) + sizeof(int32_t) * c->rows + sizeof(int2) * c->nnz + 8;
}

// Check-node state of a codeword fits its per-edge message slot.
bool cns_fits(const ldpcx_code *c, int prec, int64_t slot_bytes) {
    const int32_t *rp = c->row_ptr.data();
    const int64_t b = prec == kF32   ? cns_bytes_per_cw<kF32>(rp, c->rows, c->Z)
                      : prec == kF16 ? cns_bytes_per_cw<kF16>(rp, c->rows, c->Z)
                                     : cns_bytes_per_cw<kFix6>(rp, c->rows, c->Z);
    return b <= slot_bytes;
}

struct Plan {
    size_t off_groups, off_items, off_scratch, total, slot_bytes, smem;
    int n_items, grid, dmax;
};

int plan(const ldpcx_batch_group *groups, int n_groups, const ldpcx_decode_opts *o, Plan *pl) {
    if (!groups || n_groups < 1 || !o) return LDPCX_E_INVAL;
    if (o->algo != LDPCX_LAYERED_MINSUM && o->algo != LDPCX_LAYERED_SPA) return LDPCX_E_UNSUPPORTED;
    if (o->weights) return LDPCX_E_INVAL;
    size_t msgb = o->msg_prec == LDPCX_MSG_F32 ? 4 : o->msg_prec == LDPCX_MSG_F16 ? 2 : 1;
    pl->n_items = 0;
    pl->slot_bytes = 0;
    pl->smem = 0;
    pl->dmax = 0;
    for (int i = 0; i < n_groups; ++i) {
        const ldpcx_batch_group &g = groups[i];
        if (!g.code || g.B < 0 || (g.B > 0 && !g.llr_ch)) return LDPCX_E_INVAL;
        size_t tmp = 0;
        int st = ldpc_bp_workspace(g.code, 1, o, &tmp);  // validates options against the code
        if (st) return st;
        const int G = group_G(g.code);
        pl->n_items += (int)((g.B + G - 1) / G);
        pl->slot_bytes = std::max(pl->slot_bytes, (size_t)G * (size_t)stride_of(g.code) * msgb);
        const bool cns = o->algo == LDPCX_LAYERED_MINSUM &&
                         cns_fits(g.code, o->msg_prec, stride_of(g.code) * (int64_t)msgb);
        pl->smem = std::max(pl->smem, cns ? cns_tile_smem(g.code, G) : tile_smem(g.code, G));
        pl->dmax = std::max(pl->dmax, g.code->max_deg);
    }
    if (pl->smem + 64 > 227 * 1024) return LDPCX_E_UNSUPPORTED;  // + the kernel's static queue slot
    pl->slot_bytes = align256(std::max<size_t>(pl->slot_bytes, 256));
    int sms = sm_count();
    pl->grid = 2 * sms;  // two resident CTAs per SM at most (shared memory / registers)
    pl->off_groups = 256;
    pl->off_items = pl->off_groups + align256(sizeof(GroupDesc) * (size_t)n_groups);
    pl->off_scratch = pl->off_items + align256(sizeof(Item) * (size_t)std::max(1, pl->n_items));
    pl->total = pl->off_scratch + (size_t)pl->grid * pl->slot_bytes;
    return LDPCX_OK;
}

}  // namespace
}  // namespace ldpcx

using namespace ldpcx;

extern "C" int ldpc_bp_mixed_workspace(const ldpcx_batch_group *groups, int n_groups, const ldpcx_decode_opts *o,
                                       size_t *ws_bytes) {
    if (!ws_bytes) return LDPCX_E_INVAL;
    Plan pl;
    int st = plan(groups, n_groups, o, &pl);
    if (st) return st;
    *ws_bytes = pl.total;
    return LDPCX_OK;
}

extern "C" int ldpc_bp_decode_mixed(const ldpcx_batch_group *groups, int n_groups, const ldpcx_decode_opts *o,
                                    void *ws, size_t ws_bytes, void *stream) {
    Plan pl;
    int st = plan(groups, n_groups, o, &pl);
    if (st) return st;
    if (!ws || ws_bytes < pl.total || ((uintptr_t)ws & 255u)) return LDPCX_E_WORKSPACE;
    if (pl.n_items == 0) return LDPCX_OK;
    const int algo = o->algo == LDPCX_LAYERED_MINSUM ? kMinSum : kSpa;
    MixedFn fn = pick_mixed(pl.dmax, algo, o->msg_prec);
    if (!fn) return LDPCX_E_UNSUPPORTED;
    unsigned int *status = status_word_decode();
    if (!status) return LDPCX_E_CUDA;

    std::vector<GroupDesc> gds((size_t)n_groups);
    std::vector<std::pair<double, Item>> items;
    items.reserve((size_t)pl.n_items);
    for (int i = 0; i < n_groups; ++i) {
        const ldpcx_batch_group &g = groups[i];
        DevCode d;
        st = code_device(g.code, &d);
        if (st) return st;
        const ldpcx_code *c = g.code;
        GroupDesc &gd = gds[(size_t)i];
        gd.blk = d.blk;
        gd.row_ptr = d.row_ptr;
        gd.Z = c->Z;
        gd.rows = c->rows;
        gd.nnz = c->nnz;
        gd.n = c->n;
        gd.k = c->k;
        gd.n_tx = c->n_tx;
        gd.p0 = c->p0;
        gd.nf = c->n_fill;
        gd.G = group_G(c);
        gd.B = g.B;
        gd.stride = stride_of(c);
        const int64_t slot_cw = gd.stride * (int64_t)(o->msg_prec == LDPCX_MSG_F32   ? 4
                                                      : o->msg_prec == LDPCX_MSG_F16 ? 2
                                                                                     : 1);
        gd.bg = sched_shape_of(c->row_ptr.data(), c->rows, c->params.bg_shape);
        if (gd.bg && c->nnz > kSchedMaxBlocks) gd.bg = 0;
        // the compiled-schedule tile's own format must fit the codeword's slot
        if (gd.bg && sched_state_bytes(gd.bg, o->msg_prec, 1, c->row_ptr.data(), c->rows, c->Z) > slot_cw) gd.bg = 0;
        gd.cns = o->algo == LDPCX_LAYERED_MINSUM && cns_fits(c, o->msg_prec, slot_cw);
        gd.llr = g.llr_ch;
        gd.llr_out = g.llr_out;
        gd.bits = g.bits_out;
        gd.iters = g.iters_out;
        for (int64_t b = 0; b < g.B; b += gd.G) {
            const int64_t cnt = std::min<int64_t>(gd.G, g.B - b);
            Item it{i, 0, b};
            items.push_back({(double)c->nnz * c->Z * (double)cnt, it});
        }
    }
    // longest first (LPT order); ties keep the group order
    std::stable_sort(items.begin(), items.end(),
                     [](const std::pair<double, Item> &a, const std::pair<double, Item> &b) { return a.first > b.first; });
    std::vector<Item> flat(items.size());
    for (size_t i = 0; i < items.size(); ++i) flat[i] = items[i].second;

    cudaStream_t s = (cudaStream_t)stream;
    char *base = (char *)ws;
    if (cudaMemsetAsync(base, 0, 256, s) != cudaSuccess ||
        cudaMemcpyAsync(base + pl.off_groups, gds.data(), sizeof(GroupDesc) * gds.size(), cudaMemcpyHostToDevice,
                        s) != cudaSuccess ||
        cudaMemcpyAsync(base + pl.off_items, flat.data(), sizeof(Item) * flat.size(), cudaMemcpyHostToDevice, s) !=
            cudaSuccess)
        return LDPCX_E_CUDA;

    MixedParams m{};
    m.groups = (const GroupDesc *)(base + pl.off_groups);
    m.items = (const Item *)(base + pl.off_items);
    m.n_items = (int)flat.size();
    m.head = (int *)base;
    m.scratch = base + pl.off_scratch;
    m.slot_bytes = (int64_t)pl.slot_bytes;
    m.iters = o->iters;
    m.early_stop = o->early_stop;
    m.offset = o->offset;
    m.clamp = o->clamp;
    m.phi_lo = (float)log1p(2.0 / expm1((double)o->clamp));
    m.status = status;
    m.k_one = 1u;
    m.k_two = 2u;
    m.k_four = 4u;
    m.k_two22 = 1u << 22;
    m.k_two31 = 1u << 31;
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pl.smem) != cudaSuccess)
        return LDPCX_E_CUDA;
    fn<<<(unsigned)pl.grid, kMaxThreads, pl.smem, s>>>(m);
    return cudaGetLastError() == cudaSuccess ? LDPCX_OK : LDPCX_E_CUDA;
}
