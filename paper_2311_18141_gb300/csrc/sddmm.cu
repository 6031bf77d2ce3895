// SDDMM at A's pattern: out[e] = sum_n dC[row_e, n] * B[col_e, n].
//
// This is the gradient of sum(dC .* (A B)) with respect to A's values.  It uses
// the SpMM plan with one column block (each group covers the whole row of B),
// the same per-tile reservation and stealing loop, and the same split between
// rows walked by one group and rows walked by the whole warp.  Every output is
// one nonzero, so rows cut by chunk boundaries need no fix-up.
#include <string.h>

#include "api_internal.cuh"
#include "plan.cuh"
#include "spmm_kernel.cuh"

namespace spmm {

// partial dot product of this lane's columns: sum_e d[e] * decode(v)[e]
template <class Tag>
__device__ __forceinline__ float dot_vec(const float* d, const uint4& v);

template <>
__device__ __forceinline__ float dot_vec<TagF32>(const float* d, const uint4& v) {
    float a = d[0] * __uint_as_float(v.x);
    float b = d[1] * __uint_as_float(v.y);
    a = fmaf(d[2], __uint_as_float(v.z), a);
    b = fmaf(d[3], __uint_as_float(v.w), b);
    return a + b;
}
template <>
__device__ __forceinline__ float dot_vec<TagBF16>(const float* d, const uint4& v) {
    float a = d[0] * bf16lo(v.x);
    float b = d[1] * bf16hi(v.x);
    a = fmaf(d[2], bf16lo(v.y), a);
    b = fmaf(d[3], bf16hi(v.y), b);
    a = fmaf(d[4], bf16lo(v.z), a);
    b = fmaf(d[5], bf16hi(v.z), b);
    a = fmaf(d[6], bf16lo(v.w), a);
    b = fmaf(d[7], bf16hi(v.w), b);
    return a + b;
}

struct SddmmProblem {
    Problem p;           // rowptr, colind, B, ldb, M, N, plan arrays, tile_ctr, status
    const float* dC;
    int64_t lddc;
    float* out;
};

template <class K>
__device__ __forceinline__ void load_dc_row(const SddmmProblem& s, int64_t r,
                                            const LaneCols<K::VPL>& lc, float* d) {
    const float* src = s.dC + r * s.lddc + lc.c_off;
#pragma unroll
    for (int q = 0; q < K::VPL; ++q) {
#pragma unroll
        for (int h = 0; h < K::EPV / 4; ++h) {
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if ((lc.vmask >> q) & 1u) v = __ldg(reinterpret_cast<const float4*>(src + q * K::LPN * K::EPV + h * 4));
            float* o = d + q * K::EPV + h * 4;
            o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
        }
    }
}

// group-of-LPN sum; lane sl == 0 of the group ends with the total
template <int LPN>
__device__ __forceinline__ float group_sum(float x) {
#pragma unroll
    for (int off = LPN / 2; off > 0; off >>= 1) x += __shfl_xor_sync(kFull, x, off);
    return x;
}

template <class K, class Tag>
__device__ __forceinline__ void sddmm_unit(const SddmmProblem& s, int i, int c,
                                           const LaneCols<K::VPL>& lc, int lane) {
    const Problem& p = s.p;
    const int g = lane / K::LPN;
    const int sl = lane - g * K::LPN;
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
        int st = 0, L = 0;
        if (r <= x1 && r < row_hi) {
            const int rstart = __ldg(p.rowptr + r);
            const int rend = (r < x1) ? __ldg(p.rowptr + r + 1) : y1;
            st = max(rstart, y0);
            L = max(0, rend - st);
        }
        // rows with more nonzeros than groups: whole warp, groups interleaved
        unsigned lmask = __ballot_sync(kFull, L > K::G);
        while (lmask) {
            const int src = __ffs(lmask) - 1;
            lmask &= lmask - 1;
            const int rs = __shfl_sync(kFull, st, src);
            const int rl = __shfl_sync(kFull, L, src);
            float d[K::NE];
            load_dc_row<K>(s, (int64_t)rb + src, lc, d);
            for (int k = 0; k < rl; k += K::G) {
                const int e = k + g;
                float part = 0.0f;
                if (e < rl) {
                    const int col = __ldg(p.colind + rs + e);
                    const char* rp = brow(lc, col);
#pragma unroll
                    for (int q = 0; q < K::VPL; ++q)
                        if ((lc.vmask >> q) & 1u)
                            part += dot_vec<Tag>(d + q * K::EPV, ld_b16(rp + lc.qoff[q]));
                }
                part = group_sum<K::LPN>(part);
                if (e < rl && sl == 0) s.out[rs + e] = part;
            }
        }
        // short rows: one row per group
        const unsigned smask = __ballot_sync(kFull, L > 0 && L <= K::G);
        const int nshort = __popc(smask);
        for (int q0 = 0; q0 < nshort; q0 += K::G) {
            const int q = q0 + g;
            const bool act = q < nshort;
            const int pos = act ? nth_set_bit(smask, q) : 0;
            const int rs = __shfl_sync(kFull, st, pos);
            int rl = __shfl_sync(kFull, L, pos);
            if (!act) rl = 0;
            float d[K::NE];
            load_dc_row<K>(s, act ? (int64_t)rb + pos : (int64_t)rb, lc, d);
            const int tmax = __reduce_max_sync(kFull, rl);
            for (int e = 0; e < tmax; ++e) {
                float part = 0.0f;
                if (e < rl) {
                    const int col = __ldg(p.colind + rs + e);
                    const char* rp = brow(lc, col);
#pragma unroll
                    for (int qq = 0; qq < K::VPL; ++qq)
                        if ((lc.vmask >> qq) & 1u)
                            part += dot_vec<Tag>(d + qq * K::EPV, ld_b16(rp + lc.qoff[qq]));
                }
                part = group_sum<K::LPN>(part);
                if (e < rl && sl == 0) s.out[rs + e] = part;
            }
        }
    }
}

template <class Tag, int LPN, int VPL>
__global__ void __launch_bounds__(256, 2) sddmm_persistent(const SddmmProblem s) {
    using K = KCfg<TagF32, Tag, LPN, VPL>;
    const Problem& p = s.p;
    const int lane = threadIdx.x & 31;
    const int warp = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int T = p.TR;
    const int home = warp % T;
    const LaneCols<K::VPL> lc = lane_cols<K, K::VPL, K::LPN>(p, 0, lane % K::LPN);
    for (int step = 0; step < T; ++step) {
        int i = home + step;
        if (i >= T) i -= T;
        const int nch = p.blk_base[i + 1] - p.blk_base[i];
        if (nch == 0) continue;
        if (ld_relaxed(p.tile_ctr + i) >= nch) continue;
        while (true) {
            int c = 0;
            if (lane == 0) c = atomicAdd(p.tile_ctr + i, 1);
            c = __shfl_sync(kFull, c, 0);
            if (c >= nch) break;
            sddmm_unit<K, Tag>(s, i, c, lc, lane);
        }
    }
}

int device_sm_count();

template <class Tag, int LPN, int VPL>
static cudaError_t launch_sddmm_one(const SddmmProblem& s, int64_t units, cudaStream_t st) {
    auto kern = sddmm_persistent<Tag, LPN, VPL>;
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, 0);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    int64_t grid = (int64_t)device_sm_count() * per_sm;
    const int64_t need = (units + 7) / 8;
    if (grid > need) grid = need;
    if (grid < 1) grid = 1;
    kern<<<(unsigned)grid, 256, 0, st>>>(s);
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
        D = plan_default_chunk(M, nnz, 1, device_sm_count(), 1);
        cap = plan_chunk_cap(M, nnz, TR, D);
        // layout [status, counter (256 B)][plan arrays]
        const size_t pb = plan_array_bytes(TR, cap);
        if (workspace_bytes < pb + 256) return SPMM_ERR_WORKSPACE;
        plan_carve(ws + 256, TR, cap, &blk_base, &bnd_row, &bnd_nnz);
        if (plan_build(A_rowptr, M, TR, RB, D, cap, blk_base, bnd_row, bnd_nnz, st) != cudaSuccess)
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
