// Persistent work-stealing CSR SpMM kernel, C = beta*C + A*B.
//
// Work decomposition (Section 2.1 tile grid; Section 3.4 reservation):
//   * C is cut into TR row blocks x TC column blocks.  Tile (i, j) needs the
//     rows of row block i and the columns of column block j of B and C.
//   * The plan splits row block i's merge path -- its rows interleaved with
//     its nonzeros, a row's end counting as one item -- into chunks of D
//     items, so every chunk carries the same amount of work however skewed the
//     row lengths are.  Work unit = (tile, chunk).
//   * Each tile has a counter; a warp reserves the next chunk of a tile with
//     one atomicAdd (the fetch-and-add of Algorithm 3).  Warps start on
//     staggered home tiles (the iteration offset of Section 3.3) and, when a
//     tile runs dry, move on to other tiles, same tile row first (order 0) or
//     same tile column first (order 1): the locality-aware stealing order.
//   * A row cut by a chunk boundary yields one partial vector per chunk.  Each
//     partial goes to a workspace slot; a per-(row, column block) counter
//     tells the unit that finishes last, which sums the partials in chunk
//     order and writes C.  No atomics touch C and the result is reproducible.
//
// Inside a unit a warp loads the row pointers of 32 rows at once.  Rows with
// at most SHORT_MAX nonzeros (empty rows included) are processed SUB lanes
// per row, all such rows of the batch in parallel, each lane gathering VPS
// 16-byte vectors of B per nonzero, one nonzero at a time.  Longer rows and
// split rows are walked by the whole warp: each LPN-lane group takes its own
// run of nonzeros of every 32-nonzero batch, UB gathers in flight per lane,
// then a shuffle reduction across the groups.
#pragma once

#include "common.cuh"

#ifndef SPMM_MINBLOCKS
#define SPMM_MINBLOCKS 3   // resident 256-thread CTAs per SM the register budget targets
#endif
#ifndef SPMM_LONG_UNROLL
#define SPMM_LONG_UNROLL 4 // B gathers in flight per lane on the whole-warp path
#endif
#ifndef SPMM_STAGE
#define SPMM_STAGE 1       // stage whole-warp gathers through shared memory
#endif
#ifndef SPMM_STAGE_SHORT
#define SPMM_STAGE_SHORT 0 // stage short-row gathers too (slower on power-law rows)
#endif

namespace spmm {

// Launch flags of the persistent kernel.
constexpr int kFlagOrderColumn = 1;   // steal along the tile column first
constexpr int kFlagWarpHome = 2;      // stagger home tiles per warp instead of per CTA
constexpr int kFlagSweep = 4;         // all CTAs start in column block 0, steal column-major:
                                      // one column block's B rows are live in L2 at a time

template <typename TA_, typename TB_, int LPN_, int VPL_>
struct KCfg {
    using TA = TA_;
    using TB = TB_;
    static constexpr int LPN = LPN_;
    static constexpr int VPL = VPL_;
    static constexpr int EPV = TB::EPV;
    static constexpr int G = 32 / LPN;
    static constexpr int NE = VPL * EPV;                       // long-path floats per lane
    static constexpr int ESZ = 16 / EPV;                       // bytes per B element
    // gathers in flight per lane on the whole-warp path: up to SPMM_LONG_UNROLL
    // steps of VPL vectors, never more steps than a 32-nonzero batch has
    static constexpr int UB0 = SPMM_LONG_UNROLL / VPL < 1 ? 1 : SPMM_LONG_UNROLL / VPL;
    static constexpr int UB = LPN < UB0 ? LPN : UB0;           // steps per batch = LPN
    // Short rows: SUB lanes per row, each lane VPS vectors (about 16 floats),
    // RPP rows of a 32-row batch per pass, SUB passes per batch.
    static constexpr int WF = LPN * VPL * EPV;                 // floats of a column block
    static constexpr int SUB = (WF / 16) < 1 ? 1 : ((WF / 16) > 32 ? 32 : (WF / 16));
    static constexpr int VPS = (WF / SUB / EPV) < 1 ? 1 : (WF / SUB / EPV);
    static constexpr int RPP = 32 / SUB;
    static constexpr int NS = VPS * EPV;                       // short-path floats per lane
    static constexpr int SHORT_MAX = 16;                       // longer rows: whole warp
    // Whole-warp gathers staged through shared memory with cp.async: a stage
    // is SS steps of a 32-nonzero batch (SS*VPL 16-byte slots per lane), two
    // stages in flight per warp.
    static constexpr bool STAGED = SPMM_STAGE != 0;
    static constexpr int SS = (8 / VPL) < LPN ? (8 / VPL) : LPN;   // steps per stage
    static constexpr int SPB = LPN / SS;                           // stages per batch
    static constexpr int STAGE_BYTES0 = 2 * SS * VPL * 32 * 16;   // whole-warp path
    static constexpr int STAGE_BYTES1 = 2 * VPS * 32 * 16;        // short-row path
    static constexpr int STAGE_BYTES =
        STAGED ? (STAGE_BYTES0 > STAGE_BYTES1 ? STAGE_BYTES0 : STAGE_BYTES1) : 0;   // per warp
};

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

// C[r] = beta*C[r] + scale*acc for the NV vectors of this lane (stride STRIDE).
template <class K, int NV, int STRIDE>
__device__ __forceinline__ void store_vecs(const Problem& p, int64_t r, const float2* acc,
                                           const LaneCols<NV>& lc) {
    float sa = 1.0f;
    if (p.a_scale) sa = __ldg(p.a_scale + r);
    float* dst = p.C + r * p.ldc + lc.c_off;
#pragma unroll
    for (int q = 0; q < NV; ++q) {
        if (!((lc.vmask >> q) & 1u)) continue;
#pragma unroll
        for (int h = 0; h < K::EPV / 4; ++h) {
            float* d = dst + q * STRIDE * K::EPV + h * 4;
            const float2 lo = acc[q * (K::EPV / 2) + 2 * h];
            const float2 hi = acc[q * (K::EPV / 2) + 2 * h + 1];
            float4 o = make_float4(lo.x * sa, lo.y * sa, hi.x * sa, hi.y * sa);
            if (p.beta != 0.0f) {
                const float4 old = __ldcg(reinterpret_cast<const float4*>(d));
                o.x = fmaf(p.beta, old.x, o.x);
                o.y = fmaf(p.beta, old.y, o.y);
                o.z = fmaf(p.beta, old.z, o.z);
                o.w = fmaf(p.beta, old.w, o.w);
            }
            st_cs_f4(d, o);
        }
    }
}

// Partial row: write this unit's piece, and if it is the last piece of the
// row to arrive, sum all pieces in chunk order and write C.  Called by the
// whole warp; group 0 holds the vector.
template <class K>
__device__ __forceinline__ void piece_row(const Problem& p, int i, int j, int gc, int64_t r,
                                          bool tail, const float2* acc,
                                          const LaneCols<K::VPL>& lc, int lane) {
    const int g = lane / K::LPN;
    const int64_t slot = 2 * (int64_t)gc + (tail ? 0 : 1);
    if (g == 0) {
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
    // __syncwarp orders the group's slot stores before lane 0's release; the
    // acq_rel atomic publishes them and, for the last piece, acquires the
    // other pieces' stores, which __syncwarp then extends to the whole group.
    __syncwarp();
    int ca = 0, cb = 0, last = 0;
    if (lane == 0) {
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
    last = __shfl_sync(kFull, last, 0);
    if (!last) return;
    ca = __shfl_sync(kFull, ca, 0);
    cb = __shfl_sync(kFull, cb, 0);
    if (g != 0) return;
    float2 sum[K::NE / 2];
#pragma unroll
    for (int e = 0; e < K::NE / 2; ++e) sum[e] = make_float2(0.0f, 0.0f);
    for (int cc = ca; cc <= cb; ++cc) {
        const int64_t s2 = 2 * (int64_t)cc + (cc == cb ? 0 : 1);
        const float* src = p.slots + s2 * p.N + lc.c_off;
#pragma unroll
        for (int q = 0; q < K::VPL; ++q) {
            if (!((lc.vmask >> q) & 1u)) continue;
#pragma unroll
            for (int h = 0; h < K::EPV / 4; ++h) {
                const float4 v = ld_cg_f4(src + q * K::LPN * K::EPV + h * 4);
                float2* s = sum + q * (K::EPV / 2) + 2 * h;
                s[0].x += v.x;
                s[0].y += v.y;
                s[1].x += v.z;
                s[1].y += v.w;
            }
        }
    }
    store_vecs<K, K::VPL, K::LPN>(p, r, sum, lc);
}

// Whole-warp walk of nonzeros [rs, rs+L) of one row.  The row is taken 32
// nonzeros at a time, lane l holding nonzero l of the batch; group g owns the
// contiguous nonzeros g*LPN .. g*LPN+LPN-1 of each batch, so step s of every
// group reads lane s of its own LPN-lane segment (an immediate shuffle index).
// The next batch's column indices and values are fetched while the current
// one is gathered (Algorithm 2's prefetch of the next tile, at warp scale), and
// UB gathers per lane are in flight before their FMAs.  Returns the vector
// summed over the groups in every group.
template <class K>
__device__ __forceinline__ void row_warp(const Problem& p, int rs, int L,
                                         const LaneCols<K::VPL>& lc, float2* acc, int lane) {
    const int g = lane / K::LPN;
#pragma unroll
    for (int e = 0; e < K::NE / 2; ++e) acc[e] = make_float2(0.0f, 0.0f);
    int col_n = 0;
    float val_n = 0.0f;
    if (lane < L) {
        col_n = ld_stream_i32(p.colind + rs + lane);
        val_n = aval<typename K::TA, true>(p.vals, (int64_t)rs + lane);
    }
#pragma unroll 1
    for (int k = 0; k < L; k += 32) {
        const int cnt = min(32, L - k);
        const int col = col_n;
        float v = val_n;
        if (p.b_scale && lane < cnt) v *= __ldg(p.b_scale + col);
        if (k + 32 < L) {
            const int idx = k + 32 + lane;
            col_n = 0;
            val_n = 0.0f;
            if (idx < L) {
                col_n = ld_stream_i32(p.colind + rs + idx);
                val_n = aval<typename K::TA, true>(p.vals, (int64_t)rs + idx);
            }
        }
        if (cnt == 32) {
            // full batch: every step of every group is a nonzero
#pragma unroll
            for (int s0 = 0; s0 < K::LPN; s0 += K::UB) {
                uint4 bv[K::UB][K::VPL];
                float av[K::UB];
#pragma unroll
                for (int u = 0; u < K::UB; ++u) {
                    const int cc = __shfl_sync(kFull, col, s0 + u, K::LPN);
                    av[u] = __shfl_sync(kFull, v, s0 + u, K::LPN);
                    const char* rp = brow(lc, cc);
#pragma unroll
                    for (int q = 0; q < K::VPL; ++q) bv[u][q] = ld_b16(rp + lc.qoff[q]);
                }
#pragma unroll
                for (int u = 0; u < K::UB; ++u) {
                    const float2 a2 = make_float2(av[u], av[u]);
#pragma unroll
                    for (int q = 0; q < K::VPL; ++q)
                        fma_vec<typename K::TB>(acc + q * (K::EPV / 2), a2, bv[u][q]);
                }
            }
        } else {
            // last, partial batch: group g has cg nonzeros
            const int cg = min(max(cnt - g * K::LPN, 0), K::LPN);
            const int steps = min(cnt, K::LPN);
#pragma unroll 1
            for (int s0 = 0; s0 < steps; s0 += K::UB) {
                uint4 bv[K::UB][K::VPL];
                float av[K::UB];
#pragma unroll
                for (int u = 0; u < K::UB; ++u) {
                    const int cc = __shfl_sync(kFull, col, (s0 + u) & (K::LPN - 1), K::LPN);
                    av[u] = __shfl_sync(kFull, v, (s0 + u) & (K::LPN - 1), K::LPN);
                    const char* rp = brow(lc, cc);
                    if (s0 + u < cg) {
#pragma unroll
                        for (int q = 0; q < K::VPL; ++q) bv[u][q] = ld_b16(rp + lc.qoff[q]);
                    }
                }
#pragma unroll
                for (int u = 0; u < K::UB; ++u) {
                    if (s0 + u < cg) {
                        const float2 a2 = make_float2(av[u], av[u]);
#pragma unroll
                        for (int q = 0; q < K::VPL; ++q)
                            fma_vec<typename K::TB>(acc + q * (K::EPV / 2), a2, bv[u][q]);
                    }
                }
            }
        }
    }
#pragma unroll
    for (int off = K::LPN; off < 32; off <<= 1)
#pragma unroll
        for (int e = 0; e < K::NE / 2; ++e) {
            acc[e].x += __shfl_xor_sync(kFull, acc[e].x, off);
            acc[e].y += __shfl_xor_sync(kFull, acc[e].y, off);
        }
}

// The whole-warp walk with shared-memory staging.  The row's 32-nonzero
// batches are cut into stages of SS steps; stage t+1's gathers are issued as
// 16-byte cp.async copies into buffer (t+1)&1 while stage t is summed from the
// other buffer.  Lane l issues and later reads its own slots only, so
// cp.async.wait_group alone orders copy and read.  Slots of padding lanes are
// zero-filled and their values are 0, so no step needs a predicate.  `sbase`
// is this lane's first slot: warp region + lane * 16 bytes.
template <class K>
__device__ __forceinline__ void row_warp_staged(const Problem& p, int rs, int L,
                                                const LaneCols<K::VPL>& lc, float2* acc,
                                                int lane, uint32_t sbase) {
    const int g = lane / K::LPN;
    constexpr uint32_t kStage = K::SS * K::VPL * 32 * 16;   // bytes of one buffer
#pragma unroll
    for (int e = 0; e < K::NE / 2; ++e) acc[e] = make_float2(0.0f, 0.0f);
    const int nb = (L + 31) >> 5;
    const int nst = nb * K::SPB;
    // column indices and values of the current batch (c) and of the next (n)
    int col_c = 0, col_n = 0;
    float val_c = 0.0f, val_n = 0.0f;
    if (lane < L) {
        col_c = ld_stream_i32(p.colind + rs + lane);
        val_c = aval<typename K::TA, true>(p.vals, (int64_t)rs + lane);
        if (p.b_scale) val_c *= __ldg(p.b_scale + col_c);
    }
    if (32 + lane < L) {
        col_n = ld_stream_i32(p.colind + rs + 32 + lane);
        val_n = aval<typename K::TA, true>(p.vals, (int64_t)rs + 32 + lane);
        if (p.b_scale) val_n *= __ldg(p.b_scale + col_n);
    }
    auto issue = [&](int t, int col) {
        const int b = t / K::SPB, h = t - b * K::SPB;
        const int cnt = min(32, L - 32 * b);
        const uint32_t buf = sbase + (uint32_t)(t & 1) * kStage;
#pragma unroll
        for (int s = 0; s < K::SS; ++s) {
            const int step = h * K::SS + s;
            const int cc = __shfl_sync(kFull, col, step, K::LPN);
            const int ok = (g * K::LPN + step < cnt) ? 16 : 0;
            const char* rp = brow(lc, cc);
#pragma unroll
            for (int q = 0; q < K::VPL; ++q)
                cp_async16(buf + (uint32_t)((s * K::VPL + q) * 32 * 16), rp + lc.qoff[q], ok);
        }
        cp_async_commit();
    };
    issue(0, col_c);
#pragma unroll 1
    for (int t = 0; t < nst; ++t) {
        const int b = t / K::SPB, h = t - b * K::SPB;
        if (t + 1 < nst) {
            issue(t + 1, (h + 1 < K::SPB) ? col_c : col_n);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        const uint32_t buf = sbase + (uint32_t)(t & 1) * kStage;
#pragma unroll
        for (int s = 0; s < K::SS; ++s) {
            const float a = __shfl_sync(kFull, val_c, h * K::SS + s, K::LPN);
            const float2 a2 = make_float2(a, a);
#pragma unroll
            for (int q = 0; q < K::VPL; ++q)
                fma_vec<typename K::TB>(acc + q * (K::EPV / 2), a2,
                                        lds128(buf + (uint32_t)((s * K::VPL + q) * 32 * 16)));
        }
        if (h == K::SPB - 1 && b + 1 < nb) {   // move on to batch b+1, fetch batch b+2
            col_c = col_n;
            val_c = val_n;
            col_n = 0;
            val_n = 0.0f;
            const int idx = 32 * (b + 2) + lane;
            if (idx < L) {
                col_n = ld_stream_i32(p.colind + rs + idx);
                val_n = aval<typename K::TA, true>(p.vals, (int64_t)rs + idx);
                if (p.b_scale) val_n *= __ldg(p.b_scale + col_n);
            }
        }
    }
#pragma unroll
    for (int off = K::LPN; off < 32; off <<= 1)
#pragma unroll
        for (int e = 0; e < K::NE / 2; ++e) {
            acc[e].x += __shfl_xor_sync(kFull, acc[e].x, off);
            acc[e].y += __shfl_xor_sync(kFull, acc[e].y, off);
        }
}

// Short rows of the batch: SUB lanes per row, RPP rows per pass; the next
// column index and value are fetched one nonzero ahead.  With SPMM_STAGE_SHORT
// the B vectors of nonzero k+1 are also copied into shared memory (cp.async,
// zero-filled past the row's end) while nonzero k is summed.
template <class K>
__device__ __forceinline__ void short_rows(const Problem& p, int rb, unsigned smask, int s,
                                           int L, const LaneCols<K::VPS>& ls, int lane,
                                           uint32_t sbase) {
    constexpr uint32_t kBuf = K::VPS * 32 * 16;   // one nonzero's slots for the warp
#pragma unroll 1
    for (int pass = 0; pass < K::SUB; ++pass) {
        const unsigned pbits =
            K::RPP == 32 ? smask : ((smask >> (pass * K::RPP)) & ((1u << K::RPP) - 1u));
        if (!pbits) continue;
        const int q = pass * K::RPP + lane / K::SUB;   // row slot of this lane
        const int rs = __shfl_sync(kFull, s, q);
        int rl = __shfl_sync(kFull, L, q);
        const bool mine = (smask >> q) & 1u;
        if (!mine) rl = 0;
        const int lmax = __reduce_max_sync(kFull, rl);
        float2 acc[K::NS / 2];
#pragma unroll
        for (int e = 0; e < K::NS / 2; ++e) acc[e] = make_float2(0.0f, 0.0f);
        int c_n = 0;
        float a_n = 0.0f;
        if (rl > 0) {
            c_n = __ldg(p.colind + rs);
            a_n = aval<typename K::TA, false>(p.vals, (int64_t)rs);
            if (p.b_scale) a_n *= __ldg(p.b_scale + c_n);
        }
        if constexpr (K::STAGED && SPMM_STAGE_SHORT) {
            auto issue = [&](int k, int col) {
                const uint32_t buf = sbase + (uint32_t)(k & 1) * kBuf;
                const char* r0 = brow(ls, col);
                const int ok = (k < rl) ? 16 : 0;
#pragma unroll
                for (int v = 0; v < K::VPS; ++v)
                    cp_async16(buf + (uint32_t)(v * 32 * 16), r0 + ls.qoff[v], ok);
                cp_async_commit();
            };
            if (lmax > 0) issue(0, c_n);
            float a_c = a_n;
            c_n = 0;
            a_n = 0.0f;
            if (1 < rl) {
                c_n = __ldg(p.colind + rs + 1);
                a_n = aval<typename K::TA, false>(p.vals, (int64_t)rs + 1);
                if (p.b_scale) a_n *= __ldg(p.b_scale + c_n);
            }
#pragma unroll 1
            for (int k = 0; k < lmax; ++k) {
                if (k + 1 < lmax) {
                    issue(k + 1, c_n);
                    cp_async_wait<1>();
                } else {
                    cp_async_wait<0>();
                }
                const uint32_t buf = sbase + (uint32_t)(k & 1) * kBuf;
                const float2 a2 = make_float2(a_c, a_c);
#pragma unroll
                for (int v = 0; v < K::VPS; ++v)
                    fma_vec<typename K::TB>(acc + v * (K::EPV / 2), a2,
                                            lds128(buf + (uint32_t)(v * 32 * 16)));
                a_c = a_n;
                c_n = 0;
                a_n = 0.0f;
                if (k + 2 < rl) {
                    c_n = __ldg(p.colind + rs + k + 2);
                    a_n = aval<typename K::TA, false>(p.vals, (int64_t)rs + k + 2);
                    if (p.b_scale) a_n *= __ldg(p.b_scale + c_n);
                }
            }
        } else {
#pragma unroll 1
            for (int k = 0; k < lmax; ++k) {
                const int c0 = c_n;
                const float a0 = a_n;
                if (k + 1 < rl) {
                    c_n = __ldg(p.colind + rs + k + 1);
                    a_n = aval<typename K::TA, false>(p.vals, (int64_t)rs + k + 1);
                    if (p.b_scale) a_n *= __ldg(p.b_scale + c_n);
                }
                if (k < rl) {
                    const char* r0 = brow(ls, c0);
                    uint4 b0[K::VPS];
#pragma unroll
                    for (int v = 0; v < K::VPS; ++v) b0[v] = ld_b16(r0 + ls.qoff[v]);
                    const float2 a02 = make_float2(a0, a0);
#pragma unroll
                    for (int v = 0; v < K::VPS; ++v)
                        fma_vec<typename K::TB>(acc + v * (K::EPV / 2), a02, b0[v]);
                }
            }
        }
        // an empty row with beta == 1 and no row scale leaves C unchanged
        if (mine && !(rl == 0 && p.beta == 1.0f && p.a_scale == nullptr))
            store_vecs<K, K::VPS, K::SUB>(p, (int64_t)rb + q, acc, ls);
    }
}

// One work unit: chunk c of row block i, column block j.
template <class K>
__device__ __forceinline__ void process_unit(const Problem& p, int i, int j, int c,
                                             const LaneCols<K::VPL>& lc,
                                             const LaneCols<K::VPS>& ls, int lane,
                                             uint32_t sbase) {
    const int g = lane / K::LPN;
    const int gc = p.blk_base[i] + c;
    const int bi = gc + i;
    const int x0 = p.bnd_row[bi], y0 = p.bnd_nnz[bi];
    const int x1 = p.bnd_row[bi + 1], y1 = p.bnd_nnz[bi + 1];
    const int row_lo = i * p.RB;
    const int row_hi = min(p.M, row_lo + p.RB);
    if (x0 > x1 || y0 > y1 || x0 < row_lo || x1 > row_hi) {
        if (lane == 0) atomicOr(p.status + 1, 1);
        return;
    }
    for (int rb = x0; rb <= x1 && rb < row_hi; rb += 32) {
        const int r = rb + lane;
        bool valid = (r <= x1) && (r < row_hi);
        // rowptr[r] by this lane, rowptr[r+1] from the next lane (lane 31 loads
        // it); r <= x1 <= row_hi <= M, so rowptr[r] exists even for r == row_hi
        const int rp_here = (r <= x1) ? __ldg(p.rowptr + r) : 0;
        int rp_next = __shfl_down_sync(kFull, rp_here, 1);
        if (lane == 31 && r < x1) rp_next = __ldg(p.rowptr + r + 1);
        int s = 0, L = 0;
        bool piece = false, tail = false;
        if (valid) {
            const int rstart = rp_here;
            const int rend = (r < x1) ? rp_next : y1;
            const bool carried = rstart < y0;
            const bool head = (r == x1);
            s = max(rstart, y0);
            L = rend - s;
            if (head && !carried && y1 <= rstart) {
                valid = false;
                L = 0;
            }
            piece = carried || head;
            tail = carried && !head;
        }
        const bool is_long = valid && (piece || L > K::SHORT_MAX);
        const bool is_short = valid && !is_long;   // empty rows included

        // ---- long rows and split rows: the whole warp per row ----
        unsigned lmask = __ballot_sync(kFull, is_long);
        while (lmask) {
            const int src = __ffs(lmask) - 1;
            lmask &= lmask - 1;
            const int rs = __shfl_sync(kFull, s, src);
            const int rl = __shfl_sync(kFull, L, src);
            const unsigned flags =
                __shfl_sync(kFull, (piece ? 1u : 0u) | (tail ? 2u : 0u), src);
            float2 acc[K::NE / 2];
            if constexpr (K::STAGED) row_warp_staged<K>(p, rs, rl, lc, acc, lane, sbase);
            else row_warp<K>(p, rs, rl, lc, acc, lane);
            if (flags & 1u) {
                piece_row<K>(p, i, j, gc, (int64_t)rb + src, (flags & 2u) != 0, acc, lc, lane);
            } else if (g == 0) {
                store_vecs<K, K::VPL, K::LPN>(p, (int64_t)rb + src, acc, lc);
            }
        }

        // ---- short rows: SUB lanes per row, RPP rows per pass ----
        const unsigned smask = __ballot_sync(kFull, is_short);
        if (smask) short_rows<K>(p, rb, smask, s, L, ls, lane, sbase);
    }
}

// The persistent kernel: each warp is an independent worker.
template <class TA, class TB, int LPN, int VPL>
__global__ void __launch_bounds__(256, SPMM_MINBLOCKS)
spmm_csr_persistent(const Problem p, int flags) {
    using K = KCfg<TA, TB, LPN, VPL>;
    const int lane = threadIdx.x & 31;
    const int warp = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(spmm_dyn_smem) +
                           (uint32_t)((threadIdx.x >> 5) * K::STAGE_BYTES + lane * 16);
    const int T = p.TR * p.TC;
    const bool sweep = (flags & kFlagSweep) != 0;
    const int home = sweep ? (int)blockIdx.x % p.TR
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
        const int nch = p.blk_base[i + 1] - p.blk_base[i];
        if (nch == 0) continue;
        if (ld_relaxed(p.tile_ctr + tid) >= nch) continue;
        const LaneCols<K::VPL> lc = lane_cols<K, K::VPL, K::LPN>(p, j, lane % K::LPN);
        const LaneCols<K::VPS> ls = lane_cols<K, K::VPS, K::SUB>(p, j, lane % K::SUB);
        while (true) {
            int c = 0;
            if (lane == 0) c = atomicAdd(p.tile_ctr + tid, 1);
            c = __shfl_sync(kFull, c, 0);
            if (c >= nch) break;
            process_unit<K>(p, i, j, c, lc, ls, lane, sbase);
        }
    }
}

}  // namespace spmm
