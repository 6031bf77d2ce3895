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
// Inside a unit a warp is LPN-lane groups (G = 32/LPN of them); a group
// covers one B row slice of the column block with 16-byte loads (VPL per
// lane).  Rows with at most SHORT_MAX nonzeros are taken one per group; longer
// rows and split rows are walked by the whole warp, groups interleaved over the
// nonzeros, and reduced across groups with shuffles.
#pragma once

#include "common.cuh"

#ifndef SPMM_MINBLOCKS
#define SPMM_MINBLOCKS 3   // resident 256-thread CTAs per SM the register budget targets
#endif

namespace spmm {

template <typename Tag, int LPN_, int VPL_>
struct KCfg {
    static constexpr int LPN = LPN_;
    static constexpr int VPL = VPL_;
    static constexpr int EPV = Tag::EPV;
    static constexpr int G = 32 / LPN;
    static constexpr int NE = VPL * EPV;
    static constexpr int ESZ = 16 / EPV;                       // bytes per B element
    static constexpr int U = (32 / G) < 4 ? (32 / G) : 4;      // steps in flight, long path
    // Short rows: SUB lanes per row, each lane VPS vectors (about 16 floats),
    // RPP rows of a 32-row batch per pass, SUB passes per batch.
    static constexpr int WF = LPN * VPL * EPV;                 // floats of a column block
    static constexpr int SUB = (WF / 16) < 1 ? 1 : ((WF / 16) > 32 ? 32 : (WF / 16));
    static constexpr int VPS = (WF / SUB / EPV) < 1 ? 1 : (WF / SUB / EPV);
    static constexpr int RPP = 32 / SUB;
    static constexpr int NS = VPS * EPV;                       // short-path accumulators
    static constexpr int SHORT_MAX = 16;                       // longer rows: whole warp
};

// Per-lane view of column block j.
struct LaneCols {
    const char* b;       // B + first column of this lane's vector 0 (bytes)
    int64_t ldb_bytes;
    int32_t c_off;       // element offset of this lane's vector 0 within a C row
    uint32_t vmask;      // bit q set when vector q lies inside the column block
};

template <class K>
__device__ __forceinline__ LaneCols lane_cols(const Problem& p, int j, int sl) {
    LaneCols lc;
    const int64_t col_lo = (int64_t)j * p.W;
    int64_t col_hi = col_lo + p.W;
    if (col_hi > p.N) col_hi = p.N;
    const int64_t c0 = col_lo + (int64_t)sl * K::EPV;
    lc.b = reinterpret_cast<const char*>(p.B) + c0 * K::ESZ;
    lc.ldb_bytes = p.ldb * K::ESZ;
    lc.c_off = c0;
    lc.vmask = 0;
#pragma unroll
    for (int q = 0; q < K::VPL; ++q)
        if (c0 + (int64_t)q * K::LPN * K::EPV < col_hi) lc.vmask |= 1u << q;
    return lc;
}

// Per-lane view of column block j in the short-row layout: sub-lane t of a
// row owns vectors t, t+SUB, t+2*SUB, ... of the block.
template <class K>
__device__ __forceinline__ LaneCols lane_cols_short(const Problem& p, int j, int t) {
    LaneCols lc;
    const int64_t col_lo = (int64_t)j * p.W;
    int64_t col_hi = col_lo + p.W;
    if (col_hi > p.N) col_hi = p.N;
    const int64_t c0 = col_lo + (int64_t)t * K::EPV;
    lc.b = reinterpret_cast<const char*>(p.B) + c0 * K::ESZ;
    lc.ldb_bytes = p.ldb * K::ESZ;
    lc.c_off = c0;
    lc.vmask = 0;
#pragma unroll
    for (int v = 0; v < K::VPS; ++v)
        if (c0 + (int64_t)v * K::SUB * K::EPV < col_hi) lc.vmask |= 1u << v;
    return lc;
}

// Short-row store: C[r] = beta*C[r] + scale*acc in the short-row layout.
template <class K>
__device__ __forceinline__ void store_row_short(const Problem& p, int64_t r, const float* acc,
                                                const LaneCols& lc) {
    float sa = 1.0f;
    if (p.a_scale) sa = __ldg(p.a_scale + r);
    float* dst = p.C + r * p.ldc + lc.c_off;
#pragma unroll
    for (int v = 0; v < K::VPS; ++v) {
        if (!((lc.vmask >> v) & 1u)) continue;
#pragma unroll
        for (int h = 0; h < K::EPV / 4; ++h) {
            float* d = dst + v * K::SUB * K::EPV + h * 4;
            const float* a = acc + v * K::EPV + h * 4;
            float4 o = make_float4(a[0] * sa, a[1] * sa, a[2] * sa, a[3] * sa);
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

// Write one finished row: C[r] = beta*C[r] + scale*acc (lanes of one group).
template <class K>
__device__ __forceinline__ void store_row(const Problem& p, int64_t r, float* acc,
                                          const LaneCols& lc) {
    float sa = 1.0f;
    if (p.a_scale) sa = __ldg(p.a_scale + r);
    float* dst = p.C + r * p.ldc + lc.c_off;
#pragma unroll
    for (int q = 0; q < K::VPL; ++q) {
        if (!((lc.vmask >> q) & 1u)) continue;
#pragma unroll
        for (int h = 0; h < K::EPV / 4; ++h) {
            float* d = dst + q * K::LPN * K::EPV + h * 4;
            const float* a = acc + q * K::EPV + h * 4;
            float4 o = make_float4(a[0] * sa, a[1] * sa, a[2] * sa, a[3] * sa);
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
                                          bool tail, float* acc, const LaneCols& lc, int lane) {
    const int g = lane / K::LPN;
    const int64_t slot = 2 * (int64_t)gc + (tail ? 0 : 1);
    if (g == 0) {
        float* dst = p.slots + slot * p.N + lc.c_off;
#pragma unroll
        for (int q = 0; q < K::VPL; ++q) {
            if (!((lc.vmask >> q) & 1u)) continue;
#pragma unroll
            for (int h = 0; h < K::EPV / 4; ++h) {
                const float* a = acc + q * K::EPV + h * 4;
                st_cg_f4(dst + q * K::LPN * K::EPV + h * 4, make_float4(a[0], a[1], a[2], a[3]));
            }
        }
        __threadfence();
    }
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
        __threadfence();
        const int old = atomicAdd(cnt, 1);
        last = (old == cb - ca);
        ca += base;
        cb += base;
    }
    last = __shfl_sync(kFull, last, 0);
    if (!last) return;
    ca = __shfl_sync(kFull, ca, 0);
    cb = __shfl_sync(kFull, cb, 0);
    __threadfence();
    if (g != 0) return;
    float sum[K::NE];
#pragma unroll
    for (int e = 0; e < K::NE; ++e) sum[e] = 0.0f;
    for (int cc = ca; cc <= cb; ++cc) {
        const int64_t s2 = 2 * (int64_t)cc + (cc == cb ? 0 : 1);
        const float* src = p.slots + s2 * p.N + lc.c_off;
#pragma unroll
        for (int q = 0; q < K::VPL; ++q) {
            if (!((lc.vmask >> q) & 1u)) continue;
#pragma unroll
            for (int h = 0; h < K::EPV / 4; ++h) {
                const float4 v = ld_cg_f4(src + q * K::LPN * K::EPV + h * 4);
                float* s = sum + q * K::EPV + h * 4;
                s[0] += v.x;
                s[1] += v.y;
                s[2] += v.z;
                s[3] += v.w;
            }
        }
    }
    store_row<K>(p, r, sum, lc);
}

// Whole-warp walk of nonzeros [rs, rs+L) of one row: group g takes nonzeros
// g, g+G, g+2G, ...; returns the group-summed vector in every group.
template <class K, class Tag>
__device__ __forceinline__ void row_warp(const Problem& p, int rs, int L, const LaneCols& lc,
                                         float* acc, int lane) {
    const int g = lane / K::LPN;
#pragma unroll
    for (int e = 0; e < K::NE; ++e) acc[e] = 0.0f;
    for (int k = 0; k < L; k += 32) {
        const int cnt = min(32, L - k);
        int col = 0;
        float v = 0.0f;
        if (lane < cnt) {
            col = ld_stream_i32(p.colind + rs + k + lane);
            v = load_aval(p.vals, p.a_dtype, (int64_t)rs + k + lane);
            if (p.b_scale) v *= __ldg(p.b_scale + col);
        }
        for (int t = 0; t < cnt; t += K::G * K::U) {
            uint4 bv[K::U][K::VPL];
            float av[K::U];
#pragma unroll
            for (int u = 0; u < K::U; ++u) {
                const int src = t + u * K::G + g;
                const int cc = __shfl_sync(kFull, col, src & 31);
                av[u] = __shfl_sync(kFull, v, src & 31);
                const char* rp = lc.b + (int64_t)cc * lc.ldb_bytes;
#pragma unroll
                for (int q = 0; q < K::VPL; ++q)
                    if (src < cnt && ((lc.vmask >> q) & 1u))
                        bv[u][q] = ld_b16(rp + q * K::LPN * 16);
            }
#pragma unroll
            for (int u = 0; u < K::U; ++u) {
                if (t + u * K::G + g < cnt) {
#pragma unroll
                    for (int q = 0; q < K::VPL; ++q)
                        if ((lc.vmask >> q) & 1u) fma_vec<Tag>(acc + q * K::EPV, av[u], bv[u][q]);
                }
            }
        }
    }
#pragma unroll
    for (int off = K::LPN; off < 32; off <<= 1)
#pragma unroll
        for (int e = 0; e < K::NE; ++e) acc[e] += __shfl_xor_sync(kFull, acc[e], off);
}

// One work unit: chunk c (global gc) of row block i, column block j.
template <class K, class Tag>
__device__ __forceinline__ void process_unit(const Problem& p, int i, int j, int c,
                                             const LaneCols& lc, const LaneCols& ls, int lane) {
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
        int s = 0, L = 0;
        bool piece = false, tail = false;
        // rowptr[r] by this lane, rowptr[r+1] from the next lane (lane 31 loads it)
        const int rp_here = (r <= x1 && r < row_hi) ? __ldg(p.rowptr + r) : 0;
        int rp_next = __shfl_down_sync(kFull, rp_here, 1);
        if (lane == 31 && r < x1 && r < row_hi) rp_next = __ldg(p.rowptr + r + 1);
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
            float acc[K::NE];
            row_warp<K, Tag>(p, rs, rl, lc, acc, lane);
            if (flags & 1u) {
                piece_row<K>(p, i, j, gc, (int64_t)rb + src, (flags & 2u) != 0, acc, lc, lane);
            } else if (g == 0) {
                store_row<K>(p, (int64_t)rb + src, acc, lc);
            }
        }

        // ---- short rows: SUB lanes per row, RPP rows per pass ----
        const unsigned smask = __ballot_sync(kFull, is_short);
        if (smask) {
            const int t = lane % K::SUB;
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
                float acc[K::NS];
#pragma unroll
                for (int e = 0; e < K::NS; ++e) acc[e] = 0.0f;
                for (int k = 0; k < lmax; ++k) {
                    if (k < rl) {
                        const int c0 = __ldg(p.colind + rs + k);
                        float a0 = load_aval(p.vals, p.a_dtype, (int64_t)rs + k);
                        if (p.b_scale) a0 *= __ldg(p.b_scale + c0);
                        uint4 b0[K::VPS];
                        const char* r0 = ls.b + (int64_t)c0 * ls.ldb_bytes;
#pragma unroll
                        for (int v = 0; v < K::VPS; ++v)
                            if ((ls.vmask >> v) & 1u) b0[v] = ld_b16(r0 + v * K::SUB * 16);
#pragma unroll
                        for (int v = 0; v < K::VPS; ++v)
                            if ((ls.vmask >> v) & 1u) fma_vec<Tag>(acc + v * K::EPV, a0, b0[v]);
                    }
                }
                // an empty row with beta == 1 and no row scale leaves C unchanged
                if (mine && !(rl == 0 && p.beta == 1.0f && p.a_scale == nullptr))
                    store_row_short<K>(p, (int64_t)rb + q, acc, ls);
            }
        }
    }
}

// The persistent kernel: each warp is an independent worker.
template <class Tag, int LPN, int VPL>
__global__ void __launch_bounds__(256, SPMM_MINBLOCKS)
spmm_csr_persistent(const Problem p, int tile_order) {
    using K = KCfg<Tag, LPN, VPL>;
    const int lane = threadIdx.x & 31;
    const int warp = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int T = p.TR * p.TC;
    const int home = warp % T;
    const int sl = lane % K::LPN;
    for (int step = 0; step < T; ++step) {
        int t = home + step;
        if (t >= T) t -= T;
        int i, j;
        if (tile_order == 0) {
            i = t / p.TC;
            j = t - i * p.TC;
        } else {
            j = t / p.TR;
            i = t - j * p.TR;
        }
        const int tid = i * p.TC + j;
        const int nch = p.blk_base[i + 1] - p.blk_base[i];
        if (nch == 0) continue;
        if (ld_relaxed(p.tile_ctr + tid) >= nch) continue;
        const LaneCols lc = lane_cols<K>(p, j, sl);
        const LaneCols ls = lane_cols_short<K>(p, j, lane % K::SUB);
        while (true) {
            int c = 0;
            if (lane == 0) c = atomicAdd(p.tile_ctr + tid, 1);
            c = __shfl_sync(kFull, c, 0);
            if (c >= nch) break;
            process_unit<K, Tag>(p, i, j, c, lc, ls, lane);
        }
    }
}

}  // namespace spmm
