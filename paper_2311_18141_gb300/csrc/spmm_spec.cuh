// Warp-specialised form of the staged SpMM kernel (opt-in, spmm_tuning.kernel
// = SPMM_KERNEL_SPEC).  The work decomposition, reservation order and
// arithmetic are the staged kernel's (spmm_kernel.cuh): merge-path chunks of
// a tile walked item by item, B row segments gathered by 16-byte cp.async into
// shared memory, FP32 FFMA2 accumulation, split rows left in workspace slots
// for split_row_fixup.  What differs is who does what.  The warps of a CTA
// form pairs: the producer of a pair reserves units, decodes their items and
// issues the gathers; the consumer only sums the staged B vectors and stores
// finished rows.  They hand stages over through a ring of NSLOT shared-memory
// slots, each with a "full" and an "empty" mbarrier:
//
//   producer: wait empty[s] -> write the stage's item metadata (values,
//             row-end bits, unit header) -> issue the stage's cp.async
//             gathers -> cp.async.mbarrier.arrive + mbarrier.arrive on full[s]
//   consumer: wait full[s] -> read metadata and B vectors, accumulate, store
//             rows -> mbarrier.arrive on empty[s]
//
// so the producer runs up to NSLOT stages ahead of the consumer.  Every wait is
// bounded (about a second); one that runs out records SPMM_ERR_TIMEOUT in the
// status word and the warp stops, and its partner's next wait runs out in turn.
#pragma once

#include <stddef.h>

#include "spmm_kernel.cuh"

#ifndef SPMM_SPEC_SLOTS
#define SPMM_SPEC_SLOTS 4   // ring slots per producer/consumer pair
#endif
#ifndef SPMM_SPEC_AHEAD
#define SPMM_SPEC_AHEAD 3   // batches the producer decodes ahead of the one it issues
#endif

namespace spmm {

constexpr int kSpecSlots = SPMM_SPEC_SLOTS;
constexpr int kSpecMetaBytes = 256;   // per slot: item values, row-end bits, unit header

// Stage flags (SpecMeta::flags).
constexpr uint32_t kStageFirst = 1;   // first stage of a unit: the header is valid
constexpr uint32_t kStageLast = 2;    // last stage of a unit
constexpr uint32_t kStageStop = 4;    // no stage: the producer has no more units

// Metadata of one stage, written by the producer lanes, read by the consumer.
// G <= 4 groups (LPN >= 8), SS = 8 items per group.
struct SpecMeta {
    float val[32];          // [g*8 + s]: value of item s of group g (0 for non-nonzeros)
    uint32_t ends[4];       // [g]: bit s set when item s of group g ends a row
    uint32_t any;           // bit s set when item s ends a row in some group
    uint32_t flags;         // kStage*
    int32_t i, j;           // the unit's tile (header)
    int32_t gc[4];          // [g]: global chunk of group g (-1: none) (header)
    int32_t x0[4];          // [g]: first row of the chunk (header)
    int32_t tail_row[4];    // [g]: row whose tail piece ends in the chunk, or -1 (header)
    int32_t head[4];        // [g]: 1 when the chunk's last row goes on in a later chunk (header)
};
static_assert(sizeof(SpecMeta) <= kSpecMetaBytes, "stage metadata fits its slot");

template <class K>
struct SpecCfg {
    static_assert(K::VPL == 1 && K::IPL == 1 && K::LPN >= 8 && K::SS == 8,
                  "the specialised kernel takes one 16-byte vector per lane and 8-item stages");
    static constexpr int DATA_BYTES = K::SS * 32 * 16;             // B vectors of one stage
    static constexpr int SLOT_BYTES = kSpecMetaBytes + DATA_BYTES;
    static constexpr int PAIR_BYTES = kSpecSlots * SLOT_BYTES;
};

// Dynamic shared memory of a specialised CTA of `warps` warps (warps/2 pairs):
// the pairs' mbarriers (2 per slot), then the pairs' rings.
__host__ __device__ constexpr int spec_smem_bytes(int warps, int slot_bytes) {
    return (warps / 2) * (kSpecSlots * 16 + kSpecSlots * slot_bytes);
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" :: "r"(bar) : "memory");
}
// Arrive on `bar` once this thread's earlier cp.async copies have landed.
__device__ __forceinline__ void cp_async_mbar_arrive(uint32_t bar) {
    asm volatile("cp.async.mbarrier.arrive.shared::cta.b64 [%0];" :: "r"(bar) : "memory");
}
__device__ __forceinline__ void sts32(uint32_t addr, uint32_t v) {
    asm volatile("st.shared.u32 [%0], %1;" :: "r"(addr), "r"(v) : "memory");
}
__device__ __forceinline__ uint32_t lds32(uint32_t addr) {
    uint32_t v;
    asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(addr) : "memory");
    return v;
}

// Shared-memory addresses of pair `pr`'s ring.
struct SpecRing {
    uint32_t full0, empty0;   // mbarrier of slot s: full0 + 8*s, empty0 + 8*s
    uint32_t slot0;           // slot s at slot0 + s*SLOT_BYTES: metadata, then B vectors
};

template <class K>
__device__ __forceinline__ SpecRing spec_ring(int pr) {
    const int pairs = (int)(blockDim.x >> 6);
    const uint32_t smem = (uint32_t)__cvta_generic_to_shared(spmm_dyn_smem);
    SpecRing r;
    r.full0 = smem + (uint32_t)(pr * kSpecSlots * 16);
    r.empty0 = r.full0 + kSpecSlots * 8;
    r.slot0 = smem + (uint32_t)(pairs * kSpecSlots * 16 + pr * SpecCfg<K>::PAIR_BYTES);
    return r;
}

__device__ __forceinline__ void spec_timeout(const Problem& p) {
    atomicCAS(p.status, 0, SPMM_ERR_TIMEOUT);
}

// The producer's view of one group's chunk: bounds, split-row facts and the
// batch decoder (the staged kernel's decode: row ends from the plan's bitmap,
// a nonzero's index from the popc of the row ends before it).
template <class K>
struct SpecChunk {
    int gc, x0, nitems, tail_row, head;
    uint32_t item0, w_lo, w_hi;
    int beta, e;

    __device__ __forceinline__ void load_words(const Problem& p, int b_off) {
        const uint32_t pos = item0 + (uint32_t)b_off;
        w_lo = __ldg(p.ends + (pos >> 5));
        w_hi = __ldg(p.ends + (pos >> 5) + 1);
    }

    __device__ __forceinline__ void init(const Problem& p, int i, int cs, int tq) {
        gc = -1;
        x0 = 0;
        int y0 = 0, x1 = 0, y1 = 0, row_hi = 0;
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
                gc = -1;
            }
        }
        nitems = (x1 - x0) + (y1 - y0);
        const int rs0 = (gc >= 0) ? __ldg(p.rowptr + x0) : 0;
        const int rs1 = (gc >= 0) ? __ldg(p.rowptr + x1) : 0;
        tail_row = (rs0 < y0 && x0 < x1) ? x0 : -1;
        head = (gc >= 0) && x1 < row_hi && y1 > rs1;
        item0 = (uint32_t)x0 + (uint32_t)y0;
        load_words(p, 0);
        beta = 0;
        e = y0;
    }

    __device__ __forceinline__ void decode(const Problem& p, ItemBatch<K>& B, int tq) {
        constexpr int MB = K::MB;
        const int left = nitems - beta;
        const uint32_t valid =
            left >= MB ? low_bits<MB>() : (left > 0 ? ((1u << left) - 1u) : 0u);
        const uint32_t m = __funnelshift_r(w_lo, w_hi, (item0 + (uint32_t)beta) & 31u) & valid;
        if (beta + MB < nitems) load_words(p, beta + MB);
        B.any_end = __reduce_or_sync(kFull, m);
        const uint32_t nz = valid & ~m;
        int c = 0;
        float v = 0.0f;
        if ((nz >> tq) & 1u) {
            const int idx = e + tq - __popc(m & ((1u << tq) - 1u));
            c = ld_stream_i32(p.colind + idx);
            v = aval<typename K::TA, true>(p.vals, (int64_t)idx);
            if (p.b_scale) v *= __ldg(p.b_scale + c);
        }
        B.col[0] = c;
        B.val[0] = v;
        B.ends = m;
        B.nz = nz;
        e += __popc(nz);
        beta += MB;
    }
};

// Producer side of one unit (tile (i, j), group chunk cs): publishes its stages
// into the ring, `seq` counting the pair's stages.  False when a wait ran out.
template <class K>
__device__ __forceinline__ bool spec_produce_unit(const Problem& p, int i, int j, int cs,
                                                  int lane, const SpecRing& ring,
                                                  uint32_t& seq) {
    constexpr int LPN = K::LPN, MB = K::MB, SS = K::SS, SPB = K::SPB;
    constexpr int SLOT = SpecCfg<K>::SLOT_BYTES;
    const int g = lane / LPN;
    const int tq = lane - g * LPN;
    SpecChunk<K> ch;
    ch.init(p, i, cs, tq);
    const LaneCols<1> lc = lane_cols<K, 1, LPN>(p, j, tq);
    const int nb = (__reduce_max_sync(kFull, ch.nitems) + MB - 1) / MB;
    const int nst = nb * SPB > 0 ? nb * SPB : 1;   // a unit always publishes a stage
    // q[0]: the batch being issued; q[1..]: decoded ahead, so their column
    // indices have landed by the time their stages issue
    constexpr int DQ = 1 + SPMM_SPEC_AHEAD;
    ItemBatch<K> q[DQ];
#pragma unroll
    for (int r = 0; r < DQ; ++r) ch.decode(p, q[r], tq);
    ItemBatch<K>& cur = q[0];
#pragma unroll 1
    for (int t = 0; t < nst; ++t) {
        const int h = SPB == 1 ? 0 : (t & (SPB - 1));
        const uint32_t slot = seq % kSpecSlots;
        const uint32_t k = seq / kSpecSlots;
        if (!mbar_wait_bounded(ring.empty0 + 8 * slot, (k & 1u) ^ 1u)) {
            spec_timeout(p);
            return false;
        }
        const uint32_t m = ring.slot0 + slot * SLOT;
        const uint32_t data = m + kSpecMetaBytes + (uint32_t)lane * 16;
        // item values: lane tq holds item tq of its group's batch
        const int s_my = tq - h * SS;
        if (s_my >= 0 && s_my < SS)
            sts32(m + (uint32_t)(g * 8 + s_my) * 4, __float_as_uint(cur.val[0]));
        if (tq == 0) {
            sts32(m + offsetof(SpecMeta, ends) + 4 * g, (cur.ends >> (h * SS)) & 0xffu);
            if (t == 0) {
                sts32(m + offsetof(SpecMeta, gc) + 4 * g, (uint32_t)ch.gc);
                sts32(m + offsetof(SpecMeta, x0) + 4 * g, (uint32_t)ch.x0);
                sts32(m + offsetof(SpecMeta, tail_row) + 4 * g, (uint32_t)ch.tail_row);
                sts32(m + offsetof(SpecMeta, head) + 4 * g, (uint32_t)ch.head);
            }
        }
        if (lane == 0) {
            sts32(m + offsetof(SpecMeta, any), (cur.any_end >> (h * SS)) & 0xffu);
            sts32(m + offsetof(SpecMeta, flags),
                  (t == 0 ? kStageFirst : 0u) | (t == nst - 1 ? kStageLast : 0u));
            if (t == 0) {
                sts32(m + offsetof(SpecMeta, i), (uint32_t)i);
                sts32(m + offsetof(SpecMeta, j), (uint32_t)j);
            }
        }
        // the stage's gathers: item h*SS + s of each group into row s of the slot
#pragma unroll
        for (int s = 0; s < SS; ++s) {
            const int tt = h * SS + s;
            const int cc = __shfl_sync(kFull, cur.col[0], tt, LPN);
            cp_async16_if_set(data + (uint32_t)(s * 32 * 16), brow(lc, cc), cur.nz, 1u << tt);
        }
        cp_async_mbar_arrive(ring.full0 + 8 * slot);
        mbar_arrive(ring.full0 + 8 * slot);
        ++seq;
        if (h == SPB - 1) {
#pragma unroll
            for (int r = 0; r + 1 < DQ; ++r) q[r] = q[r + 1];
            ch.decode(p, q[DQ - 1], tq);
        }
    }
    return true;
}

// The producer has no more units: publish a stop stage.
template <class K>
__device__ __forceinline__ void spec_produce_stop(const Problem& p, int lane, const SpecRing& ring,
                                                  uint32_t seq) {
    const uint32_t slot = seq % kSpecSlots;
    const uint32_t k = seq / kSpecSlots;
    if (!mbar_wait_bounded(ring.empty0 + 8 * slot, (k & 1u) ^ 1u)) {
        spec_timeout(p);
        return;
    }
    const uint32_t m = ring.slot0 + slot * SpecCfg<K>::SLOT_BYTES;
    if (lane == 0) sts32(m + offsetof(SpecMeta, flags), kStageStop);
    mbar_arrive(ring.full0 + 8 * slot);
}

// Consumer: sums the stages of the pair's ring until the stop stage.
template <class K>
__device__ __forceinline__ void spec_consume(const Problem& p, int lane, const SpecRing& ring) {
    constexpr int LPN = K::LPN, SS = K::SS;
    constexpr int SLOT = SpecCfg<K>::SLOT_BYTES;
    const int g = lane / LPN;
    const int tq = lane - g * LPN;
    float2 acc[K::NE / 2];
#pragma unroll
    for (int q = 0; q < K::NE / 2; ++q) acc[q] = make_float2(0.0f, 0.0f);
    LaneCols<1> lc = lane_cols<K, 1, LPN>(p, 0, tq);
    int gc = -1, cur_row = 0, tail_row = -1, head = 0;
#pragma unroll 1
    for (uint32_t seq = 0;; ++seq) {
        const uint32_t slot = seq % kSpecSlots;
        const uint32_t k = seq / kSpecSlots;
        if (!mbar_wait_bounded(ring.full0 + 8 * slot, k & 1u)) {
            spec_timeout(p);
            return;
        }
        const uint32_t m = ring.slot0 + slot * SLOT;
        const uint32_t flags = lds32(m + offsetof(SpecMeta, flags));
        if (flags & kStageStop) return;
        if (flags & kStageFirst) {
            const int j = (int)lds32(m + offsetof(SpecMeta, j));
            lc = lane_cols<K, 1, LPN>(p, j, tq);
            gc = (int)lds32(m + offsetof(SpecMeta, gc) + 4 * g);
            cur_row = (int)lds32(m + offsetof(SpecMeta, x0) + 4 * g);
            tail_row = (int)lds32(m + offsetof(SpecMeta, tail_row) + 4 * g);
            head = (int)lds32(m + offsetof(SpecMeta, head) + 4 * g);
        }
        const uint4 va = lds128(m + (uint32_t)(g * 8) * 4);
        const uint4 vb = lds128(m + (uint32_t)(g * 8 + 4) * 4);
        const uint32_t vals[8] = {va.x, va.y, va.z, va.w, vb.x, vb.y, vb.z, vb.w};
        const uint32_t ends = lds32(m + offsetof(SpecMeta, ends) + 4 * g);
        const uint32_t any = lds32(m + offsetof(SpecMeta, any));
        const uint32_t data = m + kSpecMetaBytes + (uint32_t)lane * 16;
#pragma unroll
        for (int s = 0; s < SS; ++s) {
            const uint4 v = lds128(data + (uint32_t)(s * 32 * 16));
            const float a = __uint_as_float(vals[s]);
            fma_vec<typename K::TB>(acc, make_float2(a, a), v);
            if ((any >> s) & 1u) {
                const bool mine = (ends >> s) & 1u;
                const int row = cur_row;
                cur_row += mine ? 1 : 0;
                store_row_pred<K>(p, row, mine, row == tail_row, gc, acc, lc);
#pragma unroll
                for (int q = 0; q < K::NE / 2; ++q) {
                    acc[q].x = mine ? 0.0f : acc[q].x;
                    acc[q].y = mine ? 0.0f : acc[q].y;
                }
            }
        }
        if (flags & kStageLast) {
            // the chunk's last row goes on later: its head piece to slot 2*gc+1
            if (head) store_slot<K>(p, 2 * (int64_t)gc + 1, acc, lc);
#pragma unroll
            for (int q = 0; q < K::NE / 2; ++q) acc[q] = make_float2(0.0f, 0.0f);
        }
        mbar_arrive(ring.empty0 + 8 * slot);
    }
}

// The warp-specialised persistent kernel: warp 2q is the producer and warp
// 2q+1 the consumer of pair q.
template <class TA, class TB, int LPN, int VPL>
__global__ void __launch_bounds__(256, (KCfg<TA, TB, LPN, VPL>::MINB))
spmm_csr_spec(const Problem p, int flags) {
    using K = KCfg<TA, TB, LPN, VPL>;
    const int lane = threadIdx.x & 31;
    const int w = threadIdx.x >> 5;
    const SpecRing ring = spec_ring<K>(w >> 1);
    if (threadIdx.x < (blockDim.x >> 6) * kSpecSlots * 2) {
        // one thread per mbarrier: full ones count the producer's 32 lanes,
        // empty ones the consumer's
        const uint32_t smem = (uint32_t)__cvta_generic_to_shared(spmm_dyn_smem);
        mbar_init(smem + 8 * threadIdx.x, 32);
    }
    mbar_init_fence();
    __syncthreads();
    if ((w & 1) == 0) {
        uint32_t seq = 0;
        bool ok = true;
        persistent_schedule<K::G>(p, flags, [&](int i, int j, int cs) {
            ok = spec_produce_unit<K>(p, i, j, cs, lane, ring, seq);
            return ok;
        });
        if (ok) spec_produce_stop<K>(p, lane, ring, seq);
        // leave no copy of this thread in flight (they land in this CTA's
        // shared memory, which the consumers still read)
        cp_async_wait<0>();
    } else {
        spec_consume<K>(p, lane, ring);
    }
}

}  // namespace spmm
