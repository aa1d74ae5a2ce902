// Pieces of the two-phase flooding decoder: a strided walk over the check or
// variable nodes of a CTA's codewords, and the column lists of the block
// table, which let a variable node visit its edges in ascending row order.
#pragma once

#include <cstdint>

namespace ldpcx {
namespace dec {

// Work items of a strided loop over G codewords' grids, G x rows x Z (check
// nodes) or G x columns x Z (variable nodes), z fastest: the item's codeword
// g, its row or column q (0 .. R - 1) and its z, advanced by the CTA's thread
// count without a division per item.
struct GZWalk {
    int g, q, z;
    int dg, dq, dz;  // the stride in codewords, rows (columns) and z
    __device__ __forceinline__ GZWalk(int Z, int R) {
        const int fq = threadIdx.x / Z, sq = blockDim.x / Z;
        z = threadIdx.x - fq * Z;
        dz = blockDim.x - sq * Z;
        g = fq / R;
        q = fq - g * R;
        dg = sq / R;
        dq = sq - dg * R;
    }
    __device__ __forceinline__ void next(int Z, int R) {
        z += dz;
        q += dq;
        g += dg;
        if (z >= Z) {
            z -= Z;
            ++q;
        }
        if (q >= R) {  // q < 2 R: dq < R and at most one carry from z
            q -= R;
            ++g;
        }
    }
};

// The blocks of each column in block order (= ascending row: blocks are
// numbered row by row): s_cp[c] .. s_cp[c + 1] index s_cb, whose entries are
// b << 16 | shift. blk: the code's block table (col << 16 | shift). With at
// most one column per thread, thread c scans the table for column c; with
// more columns, one thread places the blocks by a counting sort (stable, so
// ascending block order within a column): O(nnz + cols) instead of
// O(cols nnz / threads). Ends with a block barrier.
__device__ __forceinline__ void build_col_lists(const uint32_t *blk, int nnz, int cols, int32_t *s_cp,
                                                uint32_t *s_cb) {
    if (cols <= (int)blockDim.x) {
        const int c = threadIdx.x;
        int cnt = 0;
        if (c < cols)
            for (int b = 0; b < nnz; ++b) cnt += (int)(blk[b] >> 16) == c ? 1 : 0;
        if (c < cols) s_cp[c + 1] = cnt;
        if (threadIdx.x == 0) s_cp[0] = 0;
        __syncthreads();
        if (threadIdx.x == 0)
            for (int k = 0; k < cols; ++k) s_cp[k + 1] += s_cp[k];
        __syncthreads();
        if (c < cols) {
            int e = s_cp[c];
            for (int b = 0; b < nnz; ++b) {
                const uint32_t bk = blk[b];
                if ((int)(bk >> 16) == c) s_cb[e++] = (uint32_t)b << 16 | (bk & 0xFFFFu);
            }
        }
    } else if (threadIdx.x == 0) {
        for (int k = 0; k <= cols; ++k) s_cp[k] = 0;
        for (int b = 0; b < nnz; ++b) ++s_cp[(blk[b] >> 16) + 1];
        for (int k = 0; k < cols; ++k) s_cp[k + 1] += s_cp[k];
        // place with s_cp[c] as column c's cursor, then shift the pointers back by one column
        for (int b = 0; b < nnz; ++b) {
            const uint32_t bk = blk[b];
            s_cb[s_cp[bk >> 16]++] = (uint32_t)b << 16 | (bk & 0xFFFFu);
        }
        for (int k = cols; k > 0; --k) s_cp[k] = s_cp[k - 1];
        s_cp[0] = 0;
    }
    __syncthreads();
}

// Check node of the variable z of a column for column-list entry cb (b << 16 | shift).
__device__ __forceinline__ int col_check_z(uint32_t cb, int z, int Z) {
    const int zc = z - (int)(cb & 0xFFFFu);
    return zc < 0 ? zc + Z : zc;
}

}  // namespace dec
}  // namespace ldpcx
