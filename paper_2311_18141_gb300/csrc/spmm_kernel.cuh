// Persistent work-stealing CSR SpMM kernel, C = beta*C + A*B.
//
// Work decomposition (Section 2.1 tile grid; Section 3.4 reservation):
//   * C is cut into TR row blocks x TC column blocks.  Tile (i, j) needs the
//     rows of row block i and the columns of column block j of B and C.
//   * The plan splits row block i's merge path -- its rows interleaved with
//     its nonzeros, a row's end counting as one item -- into sub-chunks of D
//     items, so every sub-chunk carries the same amount of work however skewed
//     the row lengths are.
//   * A warp is G = 32/LPN lane groups; LPN lanes hold one column block of a
//     B row in 16-byte vectors.  A work unit is G consecutive sub-chunks of
//     one tile, one per group.
//   * Each tile (or, in the default interleaved order, each tile row) has a
//     counter; a warp reserves the next unit with one atomicAdd (the
//     fetch-and-add of Algorithm 3).  Warps start on staggered home tiles
//     (the iteration offset of Section 3.3) and, when theirs runs dry, move
//     on to others in a locality-aware stealing order (schedule.cuh).
//   * A row cut by a sub-chunk boundary yields one partial vector per
//     sub-chunk, each left in a workspace slot.  After the persistent (or
//     batched) launch split_row_fixup sums each such row's partials (the plan
//     lists the rows) in sub-chunk order and writes C.  No atomics touch C and
//     the result is reproducible.
//
// Inside a unit every group walks its own sub-chunk item by item: a nonzero
// item gathers the B row segment and accumulates it, a row-end item writes
// the finished row (an empty row is a row end with nothing before it).  Items
// are decoded MB at a time from row pointers loaded ahead, and the gathers of
// the next stage of items are in flight, as cp.async copies into shared
// memory, while the current stage is summed.  Every group stays busy whatever
// the row lengths, and there is no per-row start-up latency.
#pragma once

#include <limits.h>

#include "common.cuh"
#include "schedule.cuh"

#ifndef SPMM_MINBLOCKS
#define SPMM_MINBLOCKS 3   // resident 256-thread CTAs per SM the register budget targets
#endif
#ifndef SPMM_MINBLOCKS_NARROW
#define SPMM_MINBLOCKS_NARROW 3   // the same for shapes with LPN <= 8 and one vector per lane
#endif
#ifndef SPMM_NBUF
#define SPMM_NBUF 2        // stage buffers per warp (stages in flight + 1)
#endif
#ifndef SPMM_STAGE_ITEMS
#define SPMM_STAGE_ITEMS 8 // items per lane group in one stage (of one 16-byte vector each)
#endif
#ifndef SPMM_DECODE_EXTRA
#define SPMM_DECODE_EXTRA 0 // batches decoded ahead beyond the two the stages need
#endif
#ifndef SPMM_WALK_UNROLL
#define SPMM_WALK_UNROLL 2 // stages per iteration of the walk loop
#endif

namespace spmm {

template <typename TA_, typename TB_, int LPN_, int VPL_, int NBUF_ = SPMM_NBUF>
struct KCfg {
    using TA = TA_;
    using TB = TB_;
    static constexpr int LPN = LPN_;                           // lanes per item
    static constexpr int VPL = VPL_;                           // 16-byte vectors per lane
    static constexpr int EPV = TB::EPV;                        // B elements per vector
    static constexpr int G = 32 / LPN;                         // lane groups per warp
    static constexpr int NE = VPL * EPV;                       // accumulated floats per lane
    static constexpr int ESZ = 16 / EPV;                       // bytes per B element
    // items decoded per group at a time (one bit each in a 32-bit mask), and
    // how many of them each lane of the group holds
    // (a lane holding VPL > 1 vectors takes MB = max(LPN, 8 / VPL) items, so a
    // stage of one batch stays 8 vectors per lane)
    static constexpr int MB = LPN >= 8 ? LPN : VPL == 1 ? 8 : (LPN > 8 / VPL ? LPN : 8 / VPL);
    static constexpr int IPL = MB / LPN;
    // a stage is SS items (SS*VPL 16-byte slots per lane); NBUF stage
    // buffers, NBUF-1 stages in flight while one is summed
    // (a lane holding several items of a batch needs the batch in one stage)
    static constexpr int SS0 = SPMM_STAGE_ITEMS / VPL < 1 ? 1 : SPMM_STAGE_ITEMS / VPL;
    static constexpr int SS = (IPL > 1 || SS0 > MB) ? MB : SS0;
    static constexpr int SPB = MB / SS;                        // stages per decoded batch
    // (shapes whose batch is a single stage keep two buffers of 8 items)
    static constexpr int NBUF = NBUF_ < 2 ? 2 : NBUF_;
    static constexpr int STAGE_BYTES = NBUF * SS * VPL * 32 * 16;  // per warp
    // the stage issued NBUF-1 stages ahead lies at most REL batches past the
    // current one; one more batch is decoded so that its column indices load
    // a batch before their gathers issue
    static constexpr int REL = (SPB - 1 + NBUF - 1) / SPB;
    static constexpr int DEPTH = REL + 2 + SPMM_DECODE_EXTRA;
    // resident CTAs per SM the register budget targets
    static constexpr int MINB = (LPN <= 8 && VPL == 1) ? SPMM_MINBLOCKS_NARROW : SPMM_MINBLOCKS;
    // stages per iteration of the walk loop: two where the accumulators and
    // decoded batches leave room in the register budget (no spills) and the
    // per-item conversion is short (B types of at most 8 elements per vector;
    // the E4M3 loop body, unrolled, ran 2.4x slower)
    static constexpr int UNROLL = (VPL == 1 && IPL <= 2 && EPV <= 8) ? SPMM_WALK_UNROLL : 1;
    static_assert(DEPTH <= 8, "at most eight decoded batches");
    static_assert(SPB == 1 || IPL == 1, "split batches need one item per lane");
};

// Dynamic shared memory of a persistent CTA of `warps` warps: the warps'
// staging regions, one after the other.
__host__ __device__ constexpr int smem_bytes(int warps, int stage_bytes) {
    return warps * stage_bytes;
}

// Dynamic shared memory of the persistent kernels (staging buffers).
extern __shared__ uint4 spmm_dyn_smem[];

// Per-lane view of a column block: where this lane's vectors start in a B
// row and a C row, and which of them fall inside the block.  Vectors outside
// the block are pointed at the block's first vector, so every gather is to a
// valid address and needs no predicate; only stores are masked.
template <int NV>
struct LaneCols {
    const char* b;         // B + this lane's vector 0 (bytes), clamped into the block
    uint32_t ldb_bytes;    // B row stride in bytes (N <= 2^20, so it fits 32 bits)
    int32_t c_off;         // element offset of this lane's vector 0 within a C row
    uint32_t ldc_bytes;    // C row stride in bytes (below 2^32)
    float* c;              // C + this lane's vector 0 in row 0
    uint32_t vmask;        // bit q set when vector q lies inside the column block
    uint32_t qoff[NV];     // byte offset of vector q from b (0 when clamped)
};

// Lane `t` of a group whose vectors are t, t + STRIDE, t + 2*STRIDE, ...
template <class K, int NV, int STRIDE>
__device__ __forceinline__ LaneCols<NV> lane_cols(const Problem& p, int j, int t) {
    LaneCols<NV> lc;
    const int64_t col_lo = (int64_t)j * p.W;
    int64_t col_hi = col_lo + p.W;
    if (col_hi > p.N) col_hi = p.N;
    const int64_t c0 = col_lo + (int64_t)t * K::EPV;
    lc.vmask = 0;
#pragma unroll
    for (int q = 0; q < NV; ++q)
        if (c0 + (int64_t)q * STRIDE * K::EPV < col_hi) lc.vmask |= 1u << q;
    const int64_t cb = (lc.vmask & 1u) ? c0 : col_lo;
    lc.b = reinterpret_cast<const char*>(p.B) + cb * K::ESZ;
    lc.ldb_bytes = (uint32_t)(p.ldb * K::ESZ);
    lc.c_off = (int32_t)c0;
    lc.ldc_bytes = (uint32_t)(p.ldc * 4);
    lc.c = p.C + c0;
#pragma unroll
    for (int q = 0; q < NV; ++q)
        lc.qoff[q] = ((lc.vmask >> q) & 1u) ? (uint32_t)(q * STRIDE * 16) : 0u;
    return lc;
}

// Address of this lane's vector 0 in B row `col`: one 32x32->64 multiply-add.
template <int NV>
__device__ __forceinline__ const char* brow(const LaneCols<NV>& lc, int col) {
    return lc.b + (uint64_t)(uint32_t)col * lc.ldb_bytes;
}

// Raw partial vector of this lane into workspace slot `slot`.
template <class K>
__device__ __forceinline__ void store_slot(const Problem& p, int64_t slot, const float2* acc,
                                           const LaneCols<K::VPL>& lc) {
    float* dst = p.slots + slot * p.N + lc.c_off;
#pragma unroll
    for (int q = 0; q < K::VPL; ++q) {
        if (!((lc.vmask >> q) & 1u)) continue;
#pragma unroll
        for (int h = 0; h < K::EPV / 4; ++h) {
            const float2 lo = acc[q * (K::EPV / 2) + 2 * h];
            const float2 hi = acc[q * (K::EPV / 2) + 2 * h + 1];
            st_cg_f4(dst + q * K::LPN * K::EPV + h * 4, make_float4(lo.x, lo.y, hi.x, hi.y));
        }
    }
}

// Row end, stored without divergent branches: every lane of the warp runs
// this; lanes whose group ends a row here (`mine`) store, the others are
// predicated off.  A tail piece (`to_slot`) goes raw to workspace slot 2*gc,
// a whole row to C as beta*C + a_scale*acc.
template <class K>
__device__ __forceinline__ void store_row_pred(const Problem& p, int row, bool mine,
                                               bool to_slot, int gc, const float2* acc,
                                               const LaneCols<K::VPL>& lc) {
    const bool to_c = mine && !to_slot;
    const bool scaled = p.a_scale != nullptr;
    float sa = 1.0f;
    if (scaled && to_c) sa = __ldg(p.a_scale + row);
    float* dst = to_slot ? p.slots + 2 * (int64_t)gc * p.N + lc.c_off
                         : reinterpret_cast<float*>(reinterpret_cast<char*>(lc.c) +
                                                    (uint64_t)(uint32_t)row * lc.ldc_bytes);
    const float beta = to_slot ? 0.0f : p.beta;
#pragma unroll
    for (int q = 0; q < K::VPL; ++q) {
        const bool st = mine && ((lc.vmask >> q) & 1u);
#pragma unroll
        for (int h = 0; h < K::EPV / 4; ++h) {
            float* d = dst + q * K::LPN * K::EPV + h * 4;
            const float2 lo = acc[q * (K::EPV / 2) + 2 * h];
            const float2 hi = acc[q * (K::EPV / 2) + 2 * h + 1];
            float4 o = make_float4(lo.x, lo.y, hi.x, hi.y);
            if (scaled) {
                o.x *= sa;
                o.y *= sa;
                o.z *= sa;
                o.w *= sa;
            }
            if (p.beta != 0.0f) {
                float4 old = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                if (st && to_c) old = __ldcg(reinterpret_cast<const float4*>(d));
                o.x = fmaf(beta, old.x, o.x);
                o.y = fmaf(beta, old.y, o.y);
                o.z = fmaf(beta, old.z, o.z);
                o.w = fmaf(beta, old.w, o.w);
            }
            if (st) st_cs_f4(d, o);
        }
    }
}

template <int BITS>
__host__ __device__ constexpr uint32_t low_bits() {
    return BITS >= 32 ? 0xffffffffu : ((1u << BITS) - 1u);
}

// MB consecutive items of a group's walk, decoded.  Lane tq of the group holds
// items tq, tq + LPN, ... (IPL of them).
template <class K>
struct ItemBatch {
    int col[K::IPL];      // column index of a nonzero item (0 for other items)
    float val[K::IPL];    // its value, times b_scale[col] (0 for other items)
    uint32_t ends;        // bit t: item t ends a row
    uint32_t nz;          // bit t: item t is a nonzero
    uint32_t any_end;     // bit t: item t ends a row in some group of the warp (warp-uniform)
};

// OR of a per-lane MB-bit mask over the lanes of each group.
template <class K>
__device__ __forceinline__ uint32_t group_or(uint32_t m, int g) {
    if constexpr (K::IPL == 1) {
        // MB == LPN: the G group masks sit side by side in one word
        const uint32_t all = __reduce_or_sync(kFull, m << (g * K::LPN));
        return K::LPN == 32 ? all : ((all >> (g * K::LPN)) & low_bits<K::LPN>());
    } else {
#pragma unroll
        for (int off = 1; off < K::LPN; off <<= 1) m |= __shfl_xor_sync(kFull, m, off);
        return m;
    }
}

// One group's walk over global sub-chunk blk_base[i] + cs of row block i, in
// column block j (cs < 0: no sub-chunk; the group still takes part in the
// warp's shuffles).  Called by the whole warp.
//
// Items of the sub-chunk from merge-path point (x0, y0) to (x1, y1): the
// nonzeros y0 .. y1-1 and the ends of rows x0 .. x1-1, in merge order.  Row
// ends come from the plan's bitmap over the merge items (see decode), a
// nonzero item's index is its position minus the row ends before it, and
// batches are decoded two ahead of use, so their column indices are in
// registers when their gathers are issued; the gathers of stage t+1 are in
// flight while stage t is summed.
//
// A row that begins in an earlier sub-chunk ends here as a tail piece, and a
// row that goes on in a later one leaves a head piece: both go to workspace
// slots, which split_row_fixup sums into C after the launch (no atomics in
// the walk).  `wbase` is the warp's staging region.
template <class K>
__device__ __forceinline__ void walk_unit(const Problem& p, int i, int j, int cs,
                                          const LaneCols<K::VPL>& lc, int lane, uint32_t wbase) {
    constexpr int LPN = K::LPN, MB = K::MB, IPL = K::IPL, SS = K::SS, SPB = K::SPB;
    constexpr int VPL = K::VPL;
    constexpr uint32_t kStage = SS * VPL * 32 * 16;   // bytes of one stage buffer
    const int g = lane / LPN;
    const int tq = lane - g * LPN;

    int gc = 0, x0 = 0, y0 = 0, x1 = 0, y1 = 0, row_hi = 0;
    if (cs >= 0) {
        gc = p.blk_base[i] + cs;
        const int bi = gc + i;
        x0 = p.bnd_row[bi];
        y0 = p.bnd_nnz[bi];
        x1 = p.bnd_row[bi + 1];
        y1 = p.bnd_nnz[bi + 1];
        const int row_lo = i * p.RB;
        row_hi = min(p.M, row_lo + p.RB);
        if (x0 > x1 || y0 > y1 || x0 < row_lo || x1 > row_hi) {
            if (tq == 0) atomicOr(p.status + 1, 1);
            x0 = x1 = y0 = y1 = row_hi = 0;
            cs = -1;
        }
    }
    const int nitems = (x1 - x0) + (y1 - y0);
    const int rs0 = (cs >= 0) ? __ldg(p.rowptr + x0) : 0;   // x0, x1 <= M
    const int rs1 = (cs >= 0) ? __ldg(p.rowptr + x1) : 0;
    // Row x0 began in an earlier sub-chunk: its end, if here, closes a tail
    // piece.  Row x1 (if inside the row block and holding items here) goes on
    // in a later sub-chunk: a head piece, left in acc when the walk ends.
    const int tail_row = (rs0 < y0 && x0 < x1) ? x0 : -1;
    const bool head = (cs >= 0) && x1 < row_hi && y1 > rs1;

    // Row ends come from the plan's bitmap over the merge items: the chunk's
    // items are global items x0 + y0 .. x1 + y1 - 1, and batch b's mask is
    // the MB bits from item x0 + y0 + b*MB on, read as a 64-bit window of two
    // words.  The words of the next batch are loaded one batch ahead.
    const uint32_t item0 = (uint32_t)x0 + (uint32_t)y0;
    uint32_t w_lo = 0, w_hi = 0;
    auto load_words = [&](int b_off) {
        const uint32_t pos = item0 + (uint32_t)b_off;
        w_lo = __ldg(p.ends + (pos >> 5));
        w_hi = __ldg(p.ends + (pos >> 5) + 1);
    };
    load_words(0);

    int beta = 0, e = y0;   // next batch: first item, first nonzero
    auto decode = [&](ItemBatch<K>& B) {
        const int left = nitems - beta;
        const uint32_t valid =
            left >= MB ? low_bits<MB>() : (left > 0 ? ((1u << left) - 1u) : 0u);
        uint32_t m = __funnelshift_r(w_lo, w_hi, (item0 + (uint32_t)beta) & 31u) & valid;
        if (beta + MB < nitems) load_words(beta + MB);
        // every lane of a group computes the same mask; the warp's OR marks the
        // items where some group ends a row
        const uint32_t any = __reduce_or_sync(kFull, m);
        // items past a group's walk are never row ends, so the warp's OR needs no mask
        B.any_end = any;
        const uint32_t nz = valid & ~m;
#pragma unroll
        for (int u = 0; u < IPL; ++u) {
            const int t = tq + u * LPN;
            int c = 0;
            float v = 0.0f;
            if ((nz >> t) & 1u) {
                const int idx = e + t - __popc(m & ((1u << t) - 1u));
                c = ld_stream_i32(p.colind + idx);
                v = aval<typename K::TA, true>(p.vals, (int64_t)idx);
                if (p.b_scale) v *= __ldg(p.b_scale + c);
            }
            B.col[u] = c;
            B.val[u] = v;
        }
        B.ends = m;
        B.nz = nz;
        e += __popc(nz);
        beta += MB;
    };

    float2 acc[K::NE / 2];
#pragma unroll
    for (int q = 0; q < K::NE / 2; ++q) acc[q] = make_float2(0.0f, 0.0f);
    // items are summed in merge order, so the next row end closes row cur_row
    int cur_row = x0;

    // Accumulate item tt of a batch from its B vectors v[q]; a row-end item
    // then writes its row (the tail piece: its slot).
    auto take_item = [&](const ItemBatch<K>& X, int tt, float a, const uint4* v) {
        const float2 a2 = make_float2(a, a);
#pragma unroll
        for (int q = 0; q < VPL; ++q) fma_vec<typename K::TB>(acc + q * (K::EPV / 2), a2, v[q]);
        // the warp-uniform test skips the row-end code on the items where no
        // group of the warp ends a row; where one does, the whole warp runs it,
        // predicated, with no divergent branch
        if ((X.any_end >> tt) & 1u) {
            const bool mine = (X.ends >> tt) & 1u;
            const int row = cur_row;
            cur_row += mine ? 1 : 0;
            store_row_pred<K>(p, row, mine, row == tail_row, gc, acc, lc);
#pragma unroll
            for (int q = 0; q < K::NE / 2; ++q) {
                acc[q].x = mine ? 0.0f : acc[q].x;
                acc[q].y = mine ? 0.0f : acc[q].y;
            }
        }
    };
    // value of item tt of stage h, from the lane that decoded it
    auto item_val = [&](const ItemBatch<K>& X, int s, int h) -> float {
        if constexpr (SPB == 1) return __shfl_sync(kFull, X.val[s / LPN], s % LPN, LPN);
        else return __shfl_sync(kFull, X.val[0], h * SS + s, LPN);
    };

    // cp.async staging: slot (s, q) of lane l at buf + (s*VPL + q)*512 + l*16
    // holds vector q of item s of the lane's group; padding slots are zeroed.
    auto issue_lsu = [&](int t, const ItemBatch<K>& X, int h) {
        const uint32_t buf = wbase + lane * 16 + (uint32_t)(t % K::NBUF) * kStage;
#pragma unroll
        for (int s = 0; s < SS; ++s) {
            int tt, cc;
            if constexpr (SPB == 1) {
                tt = s;
                cc = __shfl_sync(kFull, X.col[s / LPN], s % LPN, LPN);
            } else {
                tt = h * SS + s;
                cc = __shfl_sync(kFull, X.col[0], tt, LPN);
            }
            const char* rp = brow(lc, cc);
#pragma unroll
            for (int q = 0; q < VPL; ++q)
                cp_async16_if_set(buf + (uint32_t)((s * VPL + q) * 32 * 16), rp + lc.qoff[q],
                                  X.nz, 1u << tt);
        }
        cp_async_commit();
    };
    auto consume_lsu = [&](int t, const ItemBatch<K>& X, int h) {
        const uint32_t buf = wbase + lane * 16 + (uint32_t)(t % K::NBUF) * kStage;
#pragma unroll
        for (int s = 0; s < SS; ++s) {
            const int tt = SPB == 1 ? s : h * SS + s;
            const float a = item_val(X, s, h);
            uint4 v[VPL];
#pragma unroll
            for (int q = 0; q < VPL; ++q) v[q] = lds128(buf + (uint32_t)((s * VPL + q) * 32 * 16));
            take_item(X, tt, a, v);
        }
    };

    const int nb = (__reduce_max_sync(kFull, nitems) + MB - 1) / MB;
    const int nst = nb * SPB;
    // q[r]: batch b + r, b the batch being summed
    ItemBatch<K> q[K::DEPTH];
#pragma unroll
    for (int r = 0; r < K::DEPTH; ++r) decode(q[r]);
    ItemBatch<K>& A = q[0];
    // stage t of the walk lies in batch t / SPB; batch b, b+1, b+2 are A, B, C
    auto issue_lsu_stage = [&](int t, int b) {
        const int bt = t / SPB;
        const int ht = t - bt * SPB;
#pragma unroll
        for (int r = 0; r <= K::REL; ++r)
            if (bt == b + r) issue_lsu(t, q[r], ht);
    };
#pragma unroll
    for (int k = 0; k < K::NBUF - 1; ++k) {
        if (k < nst) issue_lsu_stage(k, 0);
        else cp_async_commit();   // empty group: the wait count stays NBUF-1
    }
    constexpr int kUnroll = K::UNROLL;
#pragma unroll kUnroll
    for (int t = 0; t < nst; ++t) {
        const int h = SPB == 1 ? 0 : (t & (SPB - 1));
        const int tn = t + K::NBUF - 1;
        if (tn < nst) {
            // one stage per batch: stage tn is batch tn, q[NBUF-1]
            if constexpr (SPB == 1) issue_lsu(tn, q[K::NBUF - 1], 0);
            else issue_lsu_stage(tn, t / SPB);
        } else {
            cp_async_commit();
        }
        cp_async_wait<K::NBUF - 1>();
        consume_lsu(t, A, h);
        if (h == SPB - 1) {
#pragma unroll
            for (int r = 0; r + 1 < K::DEPTH; ++r) q[r] = q[r + 1];
            decode(q[K::DEPTH - 1]);
        }
    }
    if (head) store_slot<K>(p, 2 * (int64_t)gc + 1, acc, lc);
}

// The warp's staging region (stage_bytes per warp, in warp order from the
// start of the CTA's dynamic shared memory).
template <class K>
__device__ __forceinline__ uint32_t warp_staging(int stage_bytes = K::STAGE_BYTES) {
    const int w = threadIdx.x >> 5;
    const uint32_t smem = (uint32_t)__cvta_generic_to_shared(spmm_dyn_smem);
    return smem + (uint32_t)(w * stage_bytes);
}

// The persistent kernel: each warp is an independent worker (see
// persistent_schedule for the reservation order and the optional trace).
// Split rows are left in workspace slots for split_row_fixup.
template <class TA, class TB, int LPN, int VPL>
__global__ void __launch_bounds__(256, (KCfg<TA, TB, LPN, VPL>::MINB))
spmm_csr_persistent(const Problem p, int flags) {
    using K = KCfg<TA, TB, LPN, VPL>;
    const int lane = threadIdx.x & 31;
    const uint32_t wbase = warp_staging<K>();
    persistent_schedule<K::G>(p, flags, [&](int i, int j, int cs) {
        const LaneCols<K::VPL> lc = lane_cols<K, K::VPL, K::LPN>(p, j, lane % K::LPN);
        walk_unit<K>(p, i, j, cs, lc, lane, wbase);
        return true;
    });
}

}  // namespace spmm
