// Persistent CSR SpMM kernel with 32-byte register gathers,
// C = beta*C + A*B: the local product C_ij += A_ik B_kj of Section 2.1 for
// every tile of a TR x TC grid, units reserved as in Section 3.4.
//
// Same decomposition as spmm_csr_persistent (merge-path chunks, per-tile
// queues, split rows summed by the last piece), with a different inner walk:
//   * a B row segment (one item) is LPN lanes x NV vectors of 32 bytes, and
//     every lane loads its 32-byte vectors with one 256-bit load straight into
//     registers -- no shared-memory staging, no copy-back instruction, and half
//     the load instructions of 16-byte vectors;
//   * the loads of the next P items of every lane group are in flight (a ring
//     of P register slots) while the current item is summed;
//   * an item that is not a nonzero (a row end, or padding past the chunk)
//     loads from a zero-filled buffer, so every step is the same FMA and B
//     values that are Inf or NaN can never meet a zero weight;
//   * a finished row is written with 32-byte streaming stores.
// The kernel needs no shared memory at all, so the SM's whole L1 is cache.
#pragma once

#include <limits.h>

#include "common.cuh"
#include "schedule.cuh"

#ifndef SPMM_WIDE_DEPTH
#define SPMM_WIDE_DEPTH 4   // items in flight per lane group (a power of two, at most 8)
#endif
#ifndef SPMM_WIDE_MINB
#define SPMM_WIDE_MINB 2    // resident 256-thread CTAs per SM the register budget targets
#endif

namespace spmm {

// Zero-filled vectors read by items that are not nonzeros: 32 lanes x up to
// four 32-byte vectors.  Never written.
static __device__ __align__(256) uint4 g_zero_vecs[256];

template <typename TA_, typename TB_, int LPN_, int NV_>
struct WCfg {
    using TA = TA_;
    using TB = TB_;
    static constexpr int LPN = LPN_;              // lanes per item
    static constexpr int NV = NV_;                // 32-byte vectors per lane
    static constexpr int EPV = 2 * TB::EPV;       // B elements per 32-byte vector
    static constexpr int ESZ = 32 / EPV;          // bytes per B element
    static constexpr int G = 32 / LPN;            // lane groups per warp
    static constexpr int NE = NV * EPV;           // floats accumulated per lane
    // items decoded per group at a time (one bit each of a 32-bit mask) and
    // how many of them each lane of the group holds
    static constexpr int MB = LPN < 8 ? 8 : LPN;
    static constexpr int IPL = MB / LPN;
    static constexpr int P = SPMM_WIDE_DEPTH < MB ? SPMM_WIDE_DEPTH : MB;
    static constexpr int MINB = SPMM_WIDE_MINB;
    static_assert(MB % P == 0, "the load ring must divide a batch");
    static_assert(NV * LPN * 32 <= 4096, "zero buffer covers 4 KB of vectors");
};

// Per-lane view of a column block for 32-byte vectors: lane t holds vectors
// t, t + LPN, ... (NV of them).  A vector outside the block points at the
// block's first vector (loads stay in bounds) and is never stored.
template <int NV>
struct WideCols {
    const char* b;         // B + this lane's vector 0 (bytes), clamped into the block
    const char* zero;      // this lane's zero vectors
    uint32_t ldb_bytes;    // B row stride in bytes
    uint32_t ldc_bytes;    // C row stride in bytes
    float* c;              // C + this lane's vector 0 in row 0
    int32_t c_off;         // element offset of this lane's vector 0 within a row
    uint32_t vmask;        // bit q set when vector q lies inside the column block
    uint32_t qoff[NV];     // byte offset of vector q from b (0 when clamped)
};

template <class K>
__device__ __forceinline__ WideCols<K::NV> wide_cols(const Problem& p, int j, int t) {
    WideCols<K::NV> lc;
    const int64_t col_lo = (int64_t)j * p.W;
    int64_t col_hi = col_lo + p.W;
    if (col_hi > p.N) col_hi = p.N;
    const int64_t c0 = col_lo + (int64_t)t * K::EPV;
    lc.vmask = 0;
#pragma unroll
    for (int q = 0; q < K::NV; ++q)
        if (c0 + (int64_t)q * K::LPN * K::EPV < col_hi) lc.vmask |= 1u << q;
    const bool in0 = lc.vmask & 1u;
    lc.b = reinterpret_cast<const char*>(p.B) + (in0 ? c0 : col_lo) * K::ESZ;
    lc.zero = reinterpret_cast<const char*>(g_zero_vecs) + (in0 ? t * 32 : 0);
    lc.ldb_bytes = (uint32_t)(p.ldb * K::ESZ);
    lc.ldc_bytes = (uint32_t)(p.ldc * 4);
    lc.c_off = (int32_t)c0;
    lc.c = p.C + c0;
#pragma unroll
    for (int q = 0; q < K::NV; ++q)
        lc.qoff[q] = ((lc.vmask >> q) & 1u) ? (uint32_t)(q * K::LPN * 32) : 0u;
    return lc;
}

// acc[0 .. EPV/2) += a2 * decode(v) for one 32-byte vector.
template <class K>
__device__ __forceinline__ void fma_v32(float2* acc, float2 a2, const V32& v) {
    fma_vec<typename K::TB>(acc, a2, v.lo);
    fma_vec<typename K::TB>(acc + K::EPV / 4, a2, v.hi);
}

// C[r] = beta*C[r] + a_scale[r]*acc for this lane's vectors (callable by one
// group alone: no warp-synchronous operation).
template <class K>
__device__ __forceinline__ void wide_store_row(const Problem& p, int r, const float2* acc,
                                               const WideCols<K::NV>& lc) {
    const bool scaled = p.a_scale != nullptr;
    const float sa = scaled ? __ldg(p.a_scale + r) : 1.0f;
    float* dst = reinterpret_cast<float*>(reinterpret_cast<char*>(lc.c) +
                                          (uint64_t)(uint32_t)r * lc.ldc_bytes);
#pragma unroll
    for (int q = 0; q < K::NV; ++q) {
        if (!((lc.vmask >> q) & 1u)) continue;
#pragma unroll
        for (int h = 0; h < K::EPV / 8; ++h) {
            float* d = dst + q * K::LPN * K::EPV + h * 8;
            const float2* a = acc + q * (K::EPV / 2) + 4 * h;
            float4 o0 = make_float4(a[0].x, a[0].y, a[1].x, a[1].y);
            float4 o1 = make_float4(a[2].x, a[2].y, a[3].x, a[3].y);
            if (scaled) {
                o0.x *= sa; o0.y *= sa; o0.z *= sa; o0.w *= sa;
                o1.x *= sa; o1.y *= sa; o1.z *= sa; o1.w *= sa;
            }
            if (p.beta != 0.0f) {
                float4 c0, c1;
                ld_cg_f8(d, c0, c1);
                o0.x = fmaf(p.beta, c0.x, o0.x); o0.y = fmaf(p.beta, c0.y, o0.y);
                o0.z = fmaf(p.beta, c0.z, o0.z); o0.w = fmaf(p.beta, c0.w, o0.w);
                o1.x = fmaf(p.beta, c1.x, o1.x); o1.y = fmaf(p.beta, c1.y, o1.y);
                o1.z = fmaf(p.beta, c1.z, o1.z); o1.w = fmaf(p.beta, c1.w, o1.w);
            }
            st_cs_f8(d, o0, o1);
        }
    }
}

// Raw partial vector of this lane into workspace slot `slot`.
template <class K>
__device__ __forceinline__ void wide_store_slot(const Problem& p, int64_t slot, const float2* acc,
                                                const WideCols<K::NV>& lc) {
    float* dst = p.slots + slot * p.N + lc.c_off;
#pragma unroll
    for (int q = 0; q < K::NV; ++q) {
        if (!((lc.vmask >> q) & 1u)) continue;
#pragma unroll
        for (int h = 0; h < K::EPV / 8; ++h) {
            const float2* a = acc + q * (K::EPV / 2) + 4 * h;
            st_cg_f8(dst + q * K::LPN * K::EPV + h * 8,
                     make_float4(a[0].x, a[0].y, a[1].x, a[1].y),
                     make_float4(a[2].x, a[2].y, a[3].x, a[3].y));
        }
    }
}

// Partial row r of global chunk gc (tail piece: slot 2*gc; head piece: slot
// 2*gc+1; `acc` null when already stored).  If this is the last piece of the
// row to arrive, the group sums all pieces in chunk order and writes C.
// Called by the LPN lanes of one group (mask gmask, first lane `leader`).
template <class K>
__device__ __forceinline__ void wide_piece_row(const Problem& p, int i, int j, int gc, int r,
                                               bool tail, const float2* acc,
                                               const WideCols<K::NV>& lc, int tq,
                                               unsigned gmask, int leader) {
    if (acc) wide_store_slot<K>(p, 2 * (int64_t)gc + (tail ? 0 : 1), acc, lc);
    // __syncwarp orders the group's slot stores before the leader's release;
    // the acq_rel atomic publishes them and, for the last piece, acquires the
    // other pieces' stores, which the second __syncwarp extends to the group.
    __syncwarp(gmask);
    int ca = 0, cb = 0, last = 0;
    if (tq == 0) {
        const int row_lo = i * p.RB;
        const int nnz_lo = __ldg(p.rowptr + row_lo);
        const int rstart = __ldg(p.rowptr + r);
        const int rend = __ldg(p.rowptr + r + 1);
        ca = (int)(((int64_t)(r - row_lo) + (rstart - nnz_lo)) / p.D);
        cb = (int)(((int64_t)(r - row_lo) + (rend - nnz_lo)) / p.D);
        const int base = p.blk_base[i];
        int* cnt = p.piece_cnt + (int64_t)(base + cb) * p.TC + j;
        const int old = atom_add_acq_rel(cnt, 1);
        last = (old == cb - ca);
        ca += base;
        cb += base;
    }
    __syncwarp(gmask);
    last = __shfl_sync(gmask, last, leader);
    if (!last) return;
    ca = __shfl_sync(gmask, ca, leader);
    cb = __shfl_sync(gmask, cb, leader);
    float2 sum[K::NE / 2];
#pragma unroll
    for (int e = 0; e < K::NE / 2; ++e) sum[e] = make_float2(0.0f, 0.0f);
    for (int cc = ca; cc <= cb; ++cc) {
        const int64_t s2 = 2 * (int64_t)cc + (cc == cb ? 0 : 1);
        const float* src = p.slots + s2 * p.N + lc.c_off;
#pragma unroll
        for (int q = 0; q < K::NV; ++q) {
            if (!((lc.vmask >> q) & 1u)) continue;
#pragma unroll
            for (int h = 0; h < K::EPV / 8; ++h) {
                float4 v0, v1;
                ld_cg_f8(src + q * K::LPN * K::EPV + h * 8, v0, v1);
                float2* s = sum + q * (K::EPV / 2) + 4 * h;
                s[0].x += v0.x; s[0].y += v0.y; s[1].x += v0.z; s[1].y += v0.w;
                s[2].x += v1.x; s[2].y += v1.y; s[3].x += v1.z; s[3].y += v1.w;
            }
        }
    }
    wide_store_row<K>(p, r, sum, lc);
}

// MB consecutive items of a group's walk, decoded; lane tq of the group holds
// items tq, tq + LPN, ... (IPL of them).
template <class K>
struct WideBatch {
    int col[K::IPL];      // column index of a nonzero item (0 for other items)
    float val[K::IPL];    // its value, times b_scale[col] (0 for other items)
    uint32_t ends;        // bit t: item t ends a row
    uint32_t nz;          // bit t: item t is a nonzero
};

// OR of a per-lane MB-bit mask over the lanes of each group.
template <class K>
__device__ __forceinline__ uint32_t wide_group_or(uint32_t m, int g) {
    if constexpr (K::IPL == 1) {
        // MB == LPN: the G group masks sit side by side in one word
        const uint32_t all = __reduce_or_sync(kFull, m << (g * K::LPN));
        return K::LPN == 32 ? all
                            : ((all >> (g * K::LPN)) & (K::LPN >= 32 ? 0xffffffffu
                                                                    : ((1u << K::LPN) - 1u)));
    } else {
#pragma unroll
        for (int off = 1; off < K::LPN; off <<= 1) m |= __shfl_xor_sync(kFull, m, off);
        return m;
    }
}

// One group's walk over global chunk blk_base[i] + cs of row block i in
// column block j (cs < 0: no chunk; the group still takes part in the warp's
// shuffles).  Called by the whole warp.
//
// Items of the chunk from merge-path point (x0, y0) to (x1, y1): nonzeros
// y0 .. y1-1 and the ends of rows x0 .. x1-1 in merge order, so the end of row
// r sits at item (rowptr[r+1] - y0) + (r - x0).  Those positions are read MB
// rows at a time ("pages", three in flight) and turned into a row-end mask
// per batch of MB items; a nonzero item's index is its position minus the row
// ends before it.  Batches are decoded two ahead of use, so the column
// indices of batch b+1 are in registers when batch b issues their loads.
template <class K>
__device__ __forceinline__ void walk_unit_wide(const Problem& p, int i, int j, int cs,
                                               const WideCols<K::NV>& lc, int lane) {
    constexpr int LPN = K::LPN, MB = K::MB, IPL = K::IPL, NV = K::NV, P = K::P;
    const int g = lane / LPN;
    const int tq = lane - g * LPN;
    const int leader = g * LPN;
    const unsigned gmask = LPN == 32 ? kFull : (((1u << LPN) - 1u) << leader);

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
    // Row x0 began in an earlier chunk: its end, if here, closes a tail piece.
    // Row x1 (inside the row block, holding items here) goes on in a later
    // chunk: a head piece, left in acc when the walk ends.
    const int tail_row = (rs0 < y0 && x0 < x1) ? x0 : -1;
    const bool head = (cs >= 0) && x1 < row_hi && y1 > rs1;

    int pg_cur[IPL], pg_nxt[IPL], pg_nx2[IPL];
    auto load_page = [&](int q, int* out) {
#pragma unroll
        for (int u = 0; u < IPL; ++u) {
            const int o = q * MB + tq + u * LPN;   // row offset from x0
            out[u] = (o < x1 - x0) ? (__ldg(p.rowptr + x0 + o + 1) - y0 + o) : INT_MAX;
        }
    };
    load_page(0, pg_cur);
    load_page(1, pg_nxt);
    load_page(2, pg_nx2);
    int pq = 2;

    int beta = 0, e = y0;   // next batch: first item, first nonzero
    auto decode = [&](WideBatch<K>& X) {
        uint32_t m = 0;
#pragma unroll
        for (int u = 0; u < IPL; ++u) {
            const unsigned d0 = (unsigned)(pg_cur[u] - beta);
            const unsigned d1 = (unsigned)(pg_nxt[u] - beta);
            if (d0 < (unsigned)MB) m |= 1u << d0;
            if (d1 < (unsigned)MB) m |= 1u << d1;
        }
        m = wide_group_or<K>(m, g);
        const int left = nitems - beta;
        const uint32_t full = MB >= 32 ? 0xffffffffu : ((1u << MB) - 1u);
        const uint32_t valid = left >= MB ? full : (left > 0 ? ((1u << left) - 1u) : 0u);
        m &= valid;
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
            X.col[u] = c;
            X.val[u] = v;
        }
        X.ends = m;
        X.nz = nz;
        e += __popc(nz);
        beta += MB;
        // A batch closes at most MB rows, so at most one page runs out per batch.
        const int last = __shfl_sync(kFull, pg_cur[IPL - 1], LPN - 1, LPN);
        if (last < beta) {
#pragma unroll
            for (int u = 0; u < IPL; ++u) {
                pg_cur[u] = pg_nxt[u];
                pg_nxt[u] = pg_nx2[u];
            }
            ++pq;
            load_page(pq, pg_nx2);
        }
    };

    float2 acc[K::NE / 2];
#pragma unroll
    for (int q = 0; q < K::NE / 2; ++q) acc[q] = make_float2(0.0f, 0.0f);
    int cur_row = x0;   // items are summed in merge order: the next row end closes cur_row

    // the load ring: slot s % P holds the vectors of item s (mod P)
    V32 ring[P][NV];
    auto issue = [&](V32* slot, const WideBatch<K>& X, int n) {
        const int c = __shfl_sync(kFull, X.col[n / LPN], n % LPN, LPN);
        const char* rp = ((X.nz >> n) & 1u)
                             ? lc.b + (uint64_t)(uint32_t)c * lc.ldb_bytes
                             : lc.zero;
#pragma unroll
        for (int q = 0; q < NV; ++q) slot[q] = ld_gather32(rp + lc.qoff[q]);
    };

    const int nb = (__reduce_max_sync(kFull, nitems) + MB - 1) / MB;
    WideBatch<K> q0, q1, q2;   // batches b, b+1, b+2
    decode(q0);
    decode(q1);
    decode(q2);
#pragma unroll
    for (int s = 0; s < P; ++s) issue(ring[s], q0, s);
#pragma unroll 1
    for (int b = 0; b < nb; ++b) {
        const bool more = b + 1 < nb;
#pragma unroll
        for (int s = 0; s < MB; ++s) {
            // sum item s of this batch
            const float a = __shfl_sync(kFull, q0.val[s / LPN], s % LPN, LPN);
            const float2 a2 = make_float2(a, a);
#pragma unroll
            for (int q = 0; q < NV; ++q) fma_v32<K>(acc + q * (K::EPV / 2), a2, ring[s % P][q]);
            // refill its slot with item s + P
            if (s + P < MB) issue(ring[s % P], q0, s + P);
            else if (more) issue(ring[s % P], q1, s + P - MB);
            if ((q0.ends >> s) & 1u) {
                const int row = cur_row++;
                if (row == tail_row) wide_store_slot<K>(p, 2 * (int64_t)gc, acc, lc);
                else wide_store_row<K>(p, row, acc, lc);
#pragma unroll
                for (int q = 0; q < K::NE / 2; ++q) acc[q] = make_float2(0.0f, 0.0f);
            }
        }
        q0 = q1;
        q1 = q2;
        decode(q2);
    }
    if (tail_row >= 0)
        wide_piece_row<K>(p, i, j, gc, tail_row, true, nullptr, lc, tq, gmask, leader);
    if (head) wide_piece_row<K>(p, i, j, gc, x1, false, acc, lc, tq, gmask, leader);
}

template <class TA, class TB, int LPN, int NV>
__global__ void __launch_bounds__(256, (WCfg<TA, TB, LPN, NV>::MINB))
spmm_csr_wide(const Problem p, int flags) {
    using K = WCfg<TA, TB, LPN, NV>;
    const int lane = threadIdx.x & 31;
    persistent_schedule<K::G>(p, flags, [&](int i, int j, int cs) {
        const WideCols<NV> lc = wide_cols<K>(p, j, lane % LPN);
        walk_unit_wide<K>(p, i, j, cs, lc, lane);
        return true;
    });
}

}  // namespace spmm
