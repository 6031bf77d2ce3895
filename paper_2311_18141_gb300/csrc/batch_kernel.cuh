// Batched persistent SpMM: many independent products C_p = beta_p*C_p + A_p*B_p.
//
// Every product keeps its own merge-path plan.  Its work units (G consecutive
// sub-chunks, column block) are numbered after those of the products before it
// (item_base).  The products are grouped by lane shape (lanes per column
// block), and each group runs as one persistent launch of the kernel compiled
// for that shape: its warps reserve items from the group's counter with
// atomicAdd (Algorithm 3's fetch-and-add, over the group's products), so a
// warp that finishes a small product moves straight on to the next item of
// any other.  Within a group the host orders products by width, then by
// decreasing work, so the largest are reserved first.  Each warp copies the
// descriptor of the product it is working on into its own slot of shared
// memory and runs the same unit code as the single-product kernel; the rows
// that chunk boundaries cut are summed afterwards, for all products in one
// launch (split_row_fixup_batched_kernel).  One shape
// per kernel keeps its register count, and so its resident warps, those of the
// single-product kernel.
#pragma once

#include "spmm_kernel.cuh"

#ifndef SPMM_BATCH_MINBLOCKS
#define SPMM_BATCH_MINBLOCKS 3   // resident 256-thread CTAs per SM the register budget targets
#endif
#ifndef SPMM_BATCH_NBUF
#define SPMM_BATCH_NBUF 2   // stage buffers per warp of the batched kernel
#endif

namespace spmm {

// One problem of a batch as the device sees it.  Scratch pointers inside `p`
// are filled in per call from the workspace base and the offsets below.
struct BatchEntry {
    Problem p;
    int64_t piece_off;   // byte offset of this problem's piece counters in the workspace
    int64_t slot_off;    // byte offset of its partial-row slots
    int32_t lpn;         // lanes per nonzero of its column blocks (2, 4, 8, 16 or 32)
    int32_t pad;
};

static_assert(sizeof(BatchEntry) % 4 == 0, "descriptor copied as 32-bit words");

constexpr int kBatchWarps = 8;

// Staging bytes per warp of the kernel for lane shape LPN.
template <class TA, class TB, int LPN>
__host__ __device__ constexpr int batch_stage_bytes() {
    return KCfg<TA, TB, LPN, 1, SPMM_BATCH_NBUF>::STAGE_BYTES;
}

// Unit u of a problem in column block j: its sub-chunks u*G .. u*G+G-1, counted
// over all row blocks, one per lane group; each group finds its own row block.
template <class TA, class TB, int LPN>
__device__ __forceinline__ void batch_unit(const Problem& p, int u, int j, int lane,
                                           uint32_t wbase) {
    using K = KCfg<TA, TB, LPN, 1, SPMM_BATCH_NBUF>;
    const LaneCols<K::VPL> lc = lane_cols<K, K::VPL, K::LPN>(p, j, lane % K::LPN);
    const int gsc = u * K::G + lane / K::LPN;
    int il = 0, cs = -1;
    if (gsc < p.blk_base[p.TR]) {
        int ih = p.TR - 1;   // largest il with blk_base[il] <= gsc
        while (il < ih) {
            const int mid = (il + ih + 1) >> 1;
            if (p.blk_base[mid] <= gsc) il = mid;
            else ih = mid - 1;
        }
        cs = gsc - p.blk_base[il];
    }
    walk_unit<K>(p, il, j, cs, lc, lane, wbase);
}

// The products of one lane shape (LPN lanes per column block) of a batch:
// table[0 .. count) with item_base[0 .. count] (the batch-wide prefix of
// their work items, so item_base[0] need not be 0).  Warps reserve items
// from `counter` and walk units of whichever product owns them.
template <class TA, class TB, int LPN>
__global__ void __launch_bounds__(kBatchWarps * 32, SPMM_BATCH_MINBLOCKS)
spmm_csr_batched_kernel(const BatchEntry* __restrict__ table,
                        const int64_t* __restrict__ item_base, int count, char* ws,
                        int* counter) {
    using K = KCfg<TA, TB, LPN, 1, SPMM_BATCH_NBUF>;
    __shared__ Problem sp[kBatchWarps];
    const int lane = threadIdx.x & 31;
    const int w = threadIdx.x >> 5;
    const uint32_t wbase = warp_staging<K>();
    const int64_t first = item_base[0];
    const int64_t total = item_base[count] - first;
    int cur = -1;   // product whose descriptor is in sp[w]
    while (true) {
        int item = 0;
        if (lane == 0) item = atomicAdd(counter, 1);
        item = __shfl_sync(kFull, item, 0);
        if ((int64_t)item >= total) break;
        const int64_t abs_item = first + item;
        // product owning the item: largest q with item_base[q] <= abs_item
        int lo = 0, hi = count - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (item_base[mid] <= abs_item) lo = mid;
            else hi = mid - 1;
        }
        const BatchEntry* e = table + lo;
        if (lo != cur) {
            __syncwarp();
            const uint32_t* src = reinterpret_cast<const uint32_t*>(&e->p);
            uint32_t* dst = reinterpret_cast<uint32_t*>(&sp[w]);
            for (int k = lane; k < (int)(sizeof(Problem) / 4); k += 32) dst[k] = src[k];
            __syncwarp();
            if (lane == 0) {
                sp[w].status = reinterpret_cast<int32_t*>(ws);
                sp[w].piece_cnt = reinterpret_cast<int32_t*>(ws + e->piece_off);
                sp[w].slots = reinterpret_cast<float*>(ws + e->slot_off);
            }
            __syncwarp();
            cur = lo;
        }
        const Problem& p = sp[w];
        const int local = (int)(abs_item - item_base[lo]);
        const int u = local / p.TC;
        const int j = local - u * p.TC;
        batch_unit<TA, TB, LPN>(p, u, j, lane, wbase);
    }
}

}  // namespace spmm
