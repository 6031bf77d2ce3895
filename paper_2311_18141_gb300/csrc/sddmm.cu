// SDDMM at A's pattern: out[e] = sum_n dC[row_e, n] * B[col_e, n].
//
// This is the gradient of sum(dC .* (A B)) with respect to A's values.  It uses
// the SpMM plan with one column block (a lane group covers the whole row of B),
// the same per-tile reservation and stealing loop, and the same per-group walk
// over merge-path sub-chunks.  The B row of every nonzero is staged through
// shared memory by cp.async; a dC row is staged once per row, with the row's
// first nonzero, and kept in registers for the rest of the row (shapes whose
// dC slice would take more than two float4 per lane stage it per nonzero).  Every output
// is one nonzero, so rows cut by sub-chunk boundaries need no fix-up.
#include <string.h>

#include "api_internal.cuh"
#include "launch.cuh"
#include "plan.cuh"
#include "spmm_kernel.cuh"

#ifndef SPMM_SDDMM_UNROLL
#define SPMM_SDDMM_UNROLL 0   // stages per iteration of the walk loop (0: the stages of a batch)
#endif

namespace spmm {

struct SddmmProblem {
    Problem p;           // rowptr, colind, B, ldb, M, N, plan arrays, tile_ctr, status
    const float* dC;
    int64_t lddc;
    float* out;
};

// Staging shape of the SDDMM walk: each nonzero item has slots for its B row
// segment (VPL vectors per lane) and a dC row segment (VPL*DV float4 per lane;
// filled only for the first nonzero of a row), SS items per stage, two stages
// per warp.
template <class K>
struct SCfg {
    static constexpr int DV = K::EPV / 4;                       // dC float4s per B vector
    static constexpr int SLOTS = K::VPL * (1 + DV);             // 16-byte slots per item per lane
    static constexpr int SS0 = 8 / SLOTS < 1 ? 1 : 8 / SLOTS;
    static constexpr int SS = (K::IPL > 1 || SS0 > K::MB) ? K::MB : SS0;
    static constexpr int SPB = K::MB / SS;
    static constexpr int STAGE = SS * SLOTS * 32 * 16;           // bytes of one stage buffer
    static constexpr int STAGE_BYTES = 2 * STAGE;                // per warp
    // dC of the current row held in registers (at most two float4 per lane);
    // wider shapes stage and read dC for every nonzero
    static constexpr bool ROW_DC = K::VPL * DV <= 2;
    static_assert(SPB == 1 || K::IPL == 1, "split batches need one item per lane");
};

// One group's walk over sub-chunk cs of row block i (cs < 0: none), in the
// same merge order as the SpMM walk: nonzero items are dotted, row ends only
// advance the row.  Per stage, lane l of a group holds partial dot products
// of the stage's items over its own columns; a butterfly across the group
// (plain halves while the group is wider than the stage, then a transposed
// exchange) leaves item s's total in the lane that decoded item s, which
// writes out[e] (consecutive nonzeros, coalesced).
template <class K, class Tag>
__device__ __forceinline__ void sddmm_walk(const SddmmProblem& sp, int i, int cs,
                                           const LaneCols<K::VPL>& lc, int lane, uint32_t wbase) {
    using S = SCfg<K>;
    const Problem& p = sp.p;
    constexpr int LPN = K::LPN, MB = K::MB, IPL = K::IPL, VPL = K::VPL;
    constexpr int SS = S::SS, SPB = S::SPB, DV = S::DV, EPV = K::EPV;
    const int g = lane / LPN;
    const int tq = lane - g * LPN;

    int x0 = 0, y0 = 0, x1 = 0, y1 = 0;
    if (cs >= 0) {
        const int gc = p.blk_base[i] + cs;
        const int bi = gc + i;
        x0 = p.bnd_row[bi];
        y0 = p.bnd_nnz[bi];
        x1 = p.bnd_row[bi + 1];
        y1 = p.bnd_nnz[bi + 1];
        const int row_lo = i * p.RB;
        const int row_hi = min(p.M, row_lo + p.RB);
        if (x0 > x1 || y0 > y1 || x0 < row_lo || x1 > row_hi) {
            if (tq == 0) atomicOr(p.status + 1, 1);
            x0 = x1 = y0 = y1 = 0;
        }
    }
    const int nitems = (x1 - x0) + (y1 - y0);

    int pg_cur[IPL], pg_nxt[IPL], pg_nx2[IPL];
    auto load_page = [&](int q, int* out) {
#pragma unroll
        for (int u = 0; u < IPL; ++u) {
            const int o = q * MB + tq + u * LPN;
            out[u] = (o < x1 - x0) ? (__ldg(p.rowptr + x0 + o + 1) - y0 + o) : INT_MAX;
        }
    };
    load_page(0, pg_cur);
    load_page(1, pg_nxt);
    load_page(2, pg_nx2);
    int pq = 2;

    struct Batch {
        int col[IPL];
        int e[IPL];
        uint32_t ends, nz;
        uint32_t rs;     // bit t: item t is the first nonzero of its row in this walk
        int rbase;
    };
    int beta = 0, ecur = y0, r = x0;
    uint32_t prev_end = 1u;   // the item before the next batch ends a row (or the walk starts)
    auto decode = [&](Batch& B) {
        uint32_t m = 0;
#pragma unroll
        for (int u = 0; u < IPL; ++u) {
            const unsigned d0 = (unsigned)(pg_cur[u] - beta);
            const unsigned d1 = (unsigned)(pg_nxt[u] - beta);
            if (d0 < (unsigned)MB) m |= 1u << d0;
            if (d1 < (unsigned)MB) m |= 1u << d1;
        }
        m = group_or<K>(m, g);
        const int left = nitems - beta;
        const uint32_t valid = left >= MB ? low_bits<MB>() : (left > 0 ? ((1u << left) - 1u) : 0u);
        m &= valid;
        const uint32_t nz = valid & ~m;
#pragma unroll
        for (int u = 0; u < IPL; ++u) {
            const int t = tq + u * LPN;
            int c = 0, idx = 0;
            if ((nz >> t) & 1u) {
                idx = ecur + t - __popc(m & ((1u << t) - 1u));
                c = ld_stream_i32(p.colind + idx);
            }
            B.col[u] = c;
            B.e[u] = idx;
        }
        B.ends = m;
        B.nz = nz;
        B.rs = nz & ((m << 1) | prev_end);
        prev_end = (m >> (MB - 1)) & 1u;
        B.rbase = r;
        r += __popc(m);
        ecur += __popc(nz);
        beta += MB;
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

    // slots of item s in a stage buffer: B vector q at (s*SLOTS + q)*512,
    // dC float4 k of vector q at (s*SLOTS + VPL + q*DV + k)*512 (+ lane*16)
    // this lane's columns of a dC row, vector by vector; a vector past N is
    // pointed at column 0 (its copy is zero-filled, but the address stays valid)
    int64_t dcoff[VPL];
#pragma unroll
    for (int q = 0; q < VPL; ++q)
        dcoff[q] = ((lc.vmask >> q) & 1u) ? (int64_t)lc.c_off + q * LPN * EPV : 0;
    auto issue = [&](int t, const Batch& X, int h) {
        const uint32_t buf = wbase + lane * 16 + (uint32_t)(t & 1) * S::STAGE;
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
            const bool live = (X.nz >> tt) & 1u;
            const char* rp = brow(lc, cc);
#pragma unroll
            for (int q = 0; q < VPL; ++q)
                cp_async16_if_set(buf + (uint32_t)((s * S::SLOTS + q) * 512), rp + lc.qoff[q], X.nz,
                                  1u << tt);
            if (S::ROW_DC ? ((X.rs >> tt) & 1u) : live) {
                // (first) nonzero of its row: stage the row's dC segment
                const int row = X.rbase + __popc(X.ends & ((1u << tt) - 1u));
                const float* dr = sp.dC + (int64_t)row * sp.lddc;
#pragma unroll
                for (int q = 0; q < VPL; ++q)
#pragma unroll
                    for (int k = 0; k < DV; ++k)
                        cp_async16(buf + (uint32_t)((s * S::SLOTS + VPL + q * DV + k) * 512),
                                   dr + dcoff[q] + k * 4, ((lc.vmask >> q) & 1u) ? 16 : 0);
            }
        }
        cp_async_commit();
    };

    // this lane's columns of the current row of dC, loaded from the stage
    // slot of the row's first nonzero
    uint4 dcur[S::ROW_DC ? VPL * DV : 1];
#pragma unroll
    for (int k = 0; k < (S::ROW_DC ? VPL * DV : 1); ++k) dcur[k] = make_uint4(0u, 0u, 0u, 0u);

    // per-lane partial dot product of item s of the stage
    auto partial = [&](uint32_t buf, int s) -> float {
        // two FMA chains, over even and odd elements, as one packed pair
        float2 ab = make_float2(0.0f, 0.0f);
#pragma unroll
        for (int q = 0; q < VPL; ++q) {
            const uint4 bv = lds128(buf + (uint32_t)((s * S::SLOTS + q) * 512));
            float bf[EPV];
            if constexpr (EPV == 4) {
                bf[0] = __uint_as_float(bv.x); bf[1] = __uint_as_float(bv.y);
                bf[2] = __uint_as_float(bv.z); bf[3] = __uint_as_float(bv.w);
            } else {
                const uint32_t w[4] = {bv.x, bv.y, bv.z, bv.w};
#pragma unroll
                for (int k = 0; k < 4; ++k) { bf[2 * k] = bf16lo(w[k]); bf[2 * k + 1] = bf16hi(w[k]); }
            }
#pragma unroll
            for (int k = 0; k < DV; ++k) {
                const uint4 dv =
                    S::ROW_DC ? dcur[q * DV + k]
                              : lds128(buf + (uint32_t)((s * S::SLOTS + VPL + q * DV + k) * 512));
                ab = ffma2(make_float2(__uint_as_float(dv.x), __uint_as_float(dv.y)),
                           make_float2(bf[4 * k + 0], bf[4 * k + 1]), ab);
                ab = ffma2(make_float2(__uint_as_float(dv.z), __uint_as_float(dv.w)),
                           make_float2(bf[4 * k + 2], bf[4 * k + 3]), ab);
            }
        }
        return ab.x + ab.y;
    };

    auto consume = [&](int t, const Batch& X, int h) {
        const uint32_t buf = wbase + lane * 16 + (uint32_t)(t & 1) * S::STAGE;
        float v[SS];
#pragma unroll
        for (int s = 0; s < SS; ++s) {
            const int tt = (SPB == 1 ? 0 : h * SS) + s;
            if constexpr (S::ROW_DC) {
                if ((X.rs >> tt) & 1u) {
#pragma unroll
                    for (int k = 0; k < VPL * DV; ++k)
                        dcur[k] = lds128(buf + (uint32_t)((s * S::SLOTS + VPL + k) * 512));
                }
            }
            v[s] = partial(buf, s);
        }
        if constexpr (SS <= LPN) {
            // plain halves while the group is wider than the stage ...
#pragma unroll
            for (int off = LPN / 2; off >= SS; off >>= 1)
#pragma unroll
                for (int s = 0; s < SS; ++s) v[s] += __shfl_xor_sync(kFull, v[s], off);
            // ... then a transposed exchange: lane l keeps item l % SS
#pragma unroll
            for (int off = SS / 2, cnt = SS; off >= 1; off >>= 1, cnt >>= 1) {
                const bool up = (tq & off) != 0;
#pragma unroll
                for (int j = 0; j < cnt / 2; ++j) {
                    const float send = up ? v[j] : v[j + cnt / 2];
                    const float keep = up ? v[j + cnt / 2] : v[j];
                    v[j] = keep + __shfl_xor_sync(kFull, send, off);
                }
            }
            // lane h*SS + s decoded item h*SS + s and now holds its total
            const int tt = (SPB == 1 ? 0 : h * SS) + (tq % SS);
            if ((tq / SS) == (SPB == 1 ? 0 : h) && ((X.nz >> tt) & 1u)) sp.out[X.e[0]] = v[0];
        } else {
            // a stage wider than the group (lanes hold several items): sum
            // each item over the group; the lane that decoded it writes it
#pragma unroll
            for (int off = LPN / 2; off >= 1; off >>= 1)
#pragma unroll
                for (int s = 0; s < SS; ++s) v[s] += __shfl_xor_sync(kFull, v[s], off);
#pragma unroll
            for (int s = 0; s < SS; ++s)
                if ((s % LPN) == tq && ((X.nz >> s) & 1u)) sp.out[X.e[s / LPN]] = v[s];
        }
    };

    const int nb = (__reduce_max_sync(kFull, nitems) + MB - 1) / MB;
    const int nst = nb * SPB;
    Batch A, B, C;
    decode(A);
    decode(B);
    decode(C);
    if (nst > 0) issue(0, A, 0);
    // unrolled by the stages of a batch, the stage's place in its batch is a
    // constant in each copy of the body
    constexpr int kUnroll = SPMM_SDDMM_UNROLL > 0 ? SPMM_SDDMM_UNROLL : SPB;
#pragma unroll kUnroll
    for (int t = 0; t < nst; ++t) {
        const int h = SPB == 1 ? 0 : (t & (SPB - 1));
        if (t + 1 < nst) {
            if (SPB > 1 && h + 1 < SPB) issue(t + 1, A, h + 1);
            else issue(t + 1, B, 0);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        consume(t, A, h);
        if (h == SPB - 1) {
            A = B;
            B = C;
            decode(C);
        }
    }
}

#ifndef SPMM_SDDMM_MINBLOCKS
#define SPMM_SDDMM_MINBLOCKS 3   // resident 256-thread CTAs per SM the register budget targets
#endif

template <class Tag, int LPN, int VPL>
__global__ void __launch_bounds__(256, SPMM_SDDMM_MINBLOCKS) sddmm_persistent(const SddmmProblem s) {
    using K = KCfg<TagF32, Tag, LPN, VPL>;
    using SC = SCfg<K>;
    const Problem& p = s.p;
    const int lane = threadIdx.x & 31;
    const int g = lane / K::LPN;
    const int warp = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const uint32_t wbase = (uint32_t)__cvta_generic_to_shared(spmm_dyn_smem) +
                           (uint32_t)((threadIdx.x >> 5) * SC::STAGE_BYTES);
    const int T = p.TR;
    const int home = warp % T;
    const LaneCols<K::VPL> lc = lane_cols<K, K::VPL, K::LPN>(p, 0, lane % K::LPN);
    for (int step = 0; step < T; ++step) {
        int i = home + step;
        if (i >= T) i -= T;
        const int nsub = p.blk_base[i + 1] - p.blk_base[i];
        const int nun = (nsub + K::G - 1) / K::G;   // units: G sub-chunks each
        if (nun == 0) continue;
        if (ld_relaxed(p.tile_ctr + i) >= nun) continue;
        while (true) {
            int c = 0;
            if (lane == 0) c = atomicAdd(p.tile_ctr + i, 1);
            c = __shfl_sync(kFull, c, 0);
            if (c >= nun) break;
            const int cs = c * K::G + g;
            sddmm_walk<K, Tag>(s, i, cs < nsub ? cs : -1, lc, lane, wbase);
        }
    }
}

template <class Tag, int LPN, int VPL>
static cudaError_t launch_sddmm_one(const SddmmProblem& s, int64_t units, cudaStream_t st) {
    static std::atomic<int> cache[kMaxDevices][kOccSlots];
    using K = KCfg<TagF32, Tag, LPN, VPL>;
    auto kern = sddmm_persistent<Tag, LPN, VPL>;
    const size_t smem = (size_t)8 * SCfg<K>::STAGE_BYTES;
    const int per_sm = cached_ctas_per_sm(kern, 256, smem, cache);
    if (per_sm == 0) return cudaErrorInvalidValue;
    const int64_t grid = persistent_grid(per_sm, 0, (units + K::G - 1) / K::G, 8);
    kern<<<(unsigned)grid, 256, smem, st>>>(s);
    return cudaGetLastError();
}

template <class Tag>
static cudaError_t launch_sddmm_tag(int lpn, int vpl, const SddmmProblem& s, int64_t units,
                                    cudaStream_t st) {
    switch (lpn * 10 + vpl) {
        case 21: return launch_sddmm_one<Tag, 2, 1>(s, units, st);
        case 41: return launch_sddmm_one<Tag, 4, 1>(s, units, st);
        case 81: return launch_sddmm_one<Tag, 8, 1>(s, units, st);
        case 161: return launch_sddmm_one<Tag, 16, 1>(s, units, st);
        case 321: return launch_sddmm_one<Tag, 32, 1>(s, units, st);
        case 322: return launch_sddmm_one<Tag, 32, 2>(s, units, st);
        case 324: return launch_sddmm_one<Tag, 32, 4>(s, units, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace spmm

using namespace spmm;

extern "C" int spmm_sddmm_csr(const int32_t* A_rowptr, const int32_t* A_colind, const float* dC,
                              int64_t lddc, const void* B, int32_t b_dtype, int64_t ldb,
                              float* out_vals, int64_t M, int64_t K, int64_t N, int64_t nnz,
                              spmm_plan plan, void* workspace, size_t workspace_bytes,
                              void* stream) {
    if (M < 0 || K < 0 || N < 0 || nnz < 0) return SPMM_ERR_INVALID_ARG;
    if (b_dtype != SPMM_F32 && b_dtype != SPMM_BF16) return SPMM_ERR_UNSUPPORTED;
    if (nnz == 0 || M == 0) return SPMM_OK;
    if (!A_rowptr || !A_colind || !dC || !B || !out_vals) return SPMM_ERR_INVALID_ARG;
    if (N == 0) return SPMM_ERR_INVALID_ARG;
    if (lddc < N || ldb < N) return SPMM_ERR_INVALID_ARG;
    if (ldb * elem_bytes(b_dtype) >= ((int64_t)1 << 32) || lddc * 4 >= ((int64_t)1 << 32))
        return SPMM_ERR_INVALID_ARG;
    const int eb = elem_bytes(b_dtype);
    const int epv = 16 / eb;
    if (N % epv != 0 || (ldb * eb) % 16 != 0 || (lddc * 4) % 16 != 0 ||
        ((uintptr_t)B & 15u) || ((uintptr_t)dC & 15u))
        return SPMM_ERR_MISALIGNED;
    int lpn = 0, vpl = 0;
    if (!pick_shape(N / epv, &lpn, &vpl)) return SPMM_ERR_UNSUPPORTED;
    if (!workspace || ((uintptr_t)workspace & 255u)) return SPMM_ERR_WORKSPACE;
    cudaStream_t st = (cudaStream_t)stream;
    char* ws = static_cast<char*>(workspace);
    int32_t TR, TC, RB, D;
    int64_t cap;
    int32_t *blk_base, *bnd_row, *bnd_nnz;
    if (plan) {
        int rc = plan_view(plan, M, K, nnz, N, &TR, &TC, &RB, &D, &cap, &blk_base, &bnd_row,
                           &bnd_nnz);
        if (rc) return rc;
        if (TC != 1) return SPMM_ERR_PLAN_MISMATCH;
    } else {
        TR = 1; TC = 1;
        RB = (int32_t)M;
        D = plan_default_chunk(M, nnz, 1, device_sm_count(), plan_default_groups(N, 1));
        cap = plan_chunk_cap(M, nnz, TR, D);
        // layout [status, counter (256 B)][plan arrays]
        const size_t pb = plan_array_bytes(TR, cap);
        if (workspace_bytes < pb + 256) return SPMM_ERR_WORKSPACE;
        int4* split;
        int32_t* n_split;
        plan_carve(ws + 256, TR, cap, &blk_base, &bnd_row, &bnd_nnz, &split, &n_split);
        if (plan_build(A_rowptr, M, TR, RB, D, cap, blk_base, bnd_row, bnd_nnz, split, n_split,
                       st) != cudaSuccess)
            return SPMM_ERR_CUDA;
        workspace_bytes -= pb;
    }
    const size_t need = kStatusBytes + 4 * (size_t)TR;
    if (workspace_bytes < need) return SPMM_ERR_WORKSPACE;
    SddmmProblem s;
    memset(&s, 0, sizeof(s));
    Problem& p = s.p;
    p.rowptr = A_rowptr; p.colind = A_colind; p.B = B; p.ldb = ldb;
    p.M = (int32_t)M; p.N = (int32_t)N; p.TR = TR; p.TC = 1; p.RB = RB; p.W = (int32_t)N; p.D = D;
    p.blk_base = blk_base; p.bnd_row = bnd_row; p.bnd_nnz = bnd_nnz;
    p.status = reinterpret_cast<int32_t*>(ws);
    p.tile_ctr = reinterpret_cast<int32_t*>(ws + kStatusBytes);
    s.dC = dC; s.lddc = lddc; s.out = out_vals;
    if (cudaMemsetAsync(p.tile_ctr, 0, 4 * (size_t)TR, st) != cudaSuccess) return SPMM_ERR_CUDA;
    cudaError_t e = (b_dtype == SPMM_F32) ? launch_sddmm_tag<TagF32>(lpn, vpl, s, cap, st)
                                          : launch_sddmm_tag<TagBF16>(lpn, vpl, s, cap, st);
    return e == cudaSuccess ? SPMM_OK : SPMM_ERR_CUDA;
}
