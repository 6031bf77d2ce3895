// Work reservation of the persistent SpMM kernels (Section 3.4, Algorithm 3:
// fetch-and-add on a reservation counter; Section 3.3: staggered starting
// tiles).  Shared by every kernel shape: a walker callback does the work of one
// unit, this loop decides which unit a warp takes next.
#pragma once

#include "common.cuh"

namespace spmm {

// Launch flags of the persistent kernels (spmm_tuning.tile_order).
constexpr int kFlagOrderColumn = 1;   // steal along the tile column first
constexpr int kFlagWarpHome = 2;      // stagger home tiles per warp instead of per CTA
constexpr int kFlagSweep = 4;         // all CTAs start in column block 0, steal column-major:
                                      // one column block's B rows are live in L2 at a time
constexpr int kFlagLockstep = 8;      // all warps start on tile 0 and visit the tiles in the
                                      // same order (row- or column-major by bit 0): one tile's
                                      // B rows are live in L2 at a time
constexpr int kFlagInterleave = 16;   // one queue per tile row handing out the same chunk of
                                      // its TC tiles in turn: warps that reserve one after the
                                      // other read the same A chunk and the same B rows

__device__ __forceinline__ long long globaltimer_ns() {
    long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// The persistent loop of one warp.  A unit is G consecutive plan chunks of
// one tile, chunk c*G + g for lane group g; `walk(i, j, cs)` walks the
// group's chunk cs of row block i in column block j (cs < 0: none, the group
// still takes part in the warp's shuffles) and returns false when the warp
// must stop (a bounded wait ran out).  Called by all 32 lanes of the warp.
// With a trace buffer, lane 0 records the warp's start and end time, the units
// it walked and how many came from outside its home tile (row).
template <int G, class Walk>
__device__ __forceinline__ void persistent_schedule(const Problem& p, int flags, Walk&& walk) {
    const int lane = threadIdx.x & 31;
    const int warp = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (p.trace && lane == 0 && warp < p.trace_max) p.trace[warp].t_start_ns = globaltimer_ns();
    int units = 0, stolen = 0;
    if (flags & kFlagInterleave) {
        // ticket k of tile row i is chunk group k / TC of tile (i, k % TC);
        // the tile row's first counter is its queue
        const int home_i = (flags & kFlagLockstep) ? 0 : (int)blockIdx.x % p.TR;
        for (int step = 0; step < p.TR; ++step) {
            int i = home_i + step;
            if (i >= p.TR) i -= p.TR;
            const int nsub = p.blk_base[i + 1] - p.blk_base[i];
            const int total = (nsub + G - 1) / G * p.TC;
            int* ctr = p.tile_ctr + i * p.TC;
            if (total == 0 || ld_relaxed(ctr) >= total) continue;
            while (true) {
                int k = 0;
                if (lane == 0) k = atomicAdd(ctr, 1);
                k = __shfl_sync(kFull, k, 0);
                if (k >= total) break;
                const int c = k / p.TC;
                const int j = k - c * p.TC;
                const int cs = c * G + lane / (32 / G);
                ++units;
                stolen += step != 0;
                if (!walk(i, j, cs < nsub ? cs : -1)) goto done;
            }
        }
    } else {
        const int T = p.TR * p.TC;
        const bool sweep = (flags & kFlagSweep) != 0;
        const int home = (flags & kFlagLockstep) ? 0
                         : sweep ? (int)blockIdx.x % p.TR
                                 : ((flags & kFlagWarpHome) ? warp : (int)blockIdx.x) % T;
        for (int step = 0; step < T; ++step) {
            int t = home + step;
            if (t >= T) t -= T;
            int i, j;
            if (sweep || (flags & kFlagOrderColumn)) {
                j = t / p.TR;
                i = t - j * p.TR;
            } else {
                i = t / p.TC;
                j = t - i * p.TC;
            }
            const int tid = i * p.TC + j;
            const int nsub = p.blk_base[i + 1] - p.blk_base[i];
            const int nun = (nsub + G - 1) / G;   // units: G chunks each
            if (nun == 0) continue;
            if (ld_relaxed(p.tile_ctr + tid) >= nun) continue;
            while (true) {
                int c = 0;
                if (lane == 0) c = atomicAdd(p.tile_ctr + tid, 1);
                c = __shfl_sync(kFull, c, 0);
                if (c >= nun) break;
                const int cs = c * G + lane / (32 / G);
                ++units;
                stolen += step != 0;
                if (!walk(i, j, cs < nsub ? cs : -1)) goto done;
            }
        }
    }
done:
    if (p.trace && lane == 0 && warp < p.trace_max) {
        // the home tile (row) of the walk above, recomputed
        int home;
        if (flags & kFlagLockstep) home = 0;
        else if (flags & kFlagInterleave) home = (int)blockIdx.x % p.TR;
        else if (flags & kFlagSweep) home = (int)blockIdx.x % p.TR;
        else home = ((flags & kFlagWarpHome) ? warp : (int)blockIdx.x) % (p.TR * p.TC);
        uint32_t smid;
        asm("mov.u32 %0, %%smid;" : "=r"(smid));
        spmm_trace_record* r = p.trace + warp;
        r->t_end_ns = globaltimer_ns();
        r->units = units;
        r->stolen = stolen;
        r->home = home;
        r->smid = (int32_t)smid;
    }
}

}  // namespace spmm
