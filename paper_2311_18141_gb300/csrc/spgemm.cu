// Local SpGEMM, C = A * B with CSR A (M x K), CSR B (K x N) and CSR C, FP32
// values: the sparse-sparse local product of the paper's SpGEMM experiments.
//
// Expand - sort - compress:
//   1. count: every nonzero e of A (row i, column k) makes nnz(B row k)
//      products; an exclusive scan of the counts gives each its offset.
//   2. expand: one warp per nonzero of A writes (i, j, A_ik * B_kj) for the
//      nonzeros (k, j) of B's row k, in A's CSR order and then B's.
//   3. sort: when bits(M) + bits(N) <= 32 the key (i << bits(N)) | j is sorted
//      once, stably, carrying the value; otherwise the products are sorted
//      stably by column, then stably by row, carrying each product's index.
//      Either way equal (i, j) stay in expansion order.
//   4. compress: run heads are flagged and scanned into entry indices, each
//      entry's first product is recorded, and one thread per entry sums its
//      run in FP32 in that order; row pointers by lower bound over the entry
//      rows.
// An entry of C exists wherever some product is formed (explicit zeros
// count).  The order of every sum is fixed, so results are reproducible.
#include <string.h>

#include "api_internal.cuh"
#include "radix.cuh"

namespace spmm {

namespace {

size_t up256(size_t x) { return (x + 255) / 256 * 256; }

unsigned grid_for(int64_t work, int threads) {
    int64_t g = (work + threads - 1) / threads;
    const int64_t cap = (int64_t)device_sm_count() * 16;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    return (unsigned)g;
}

// cnt[e] = nnz of B's row colA[e] (0 and an error flag for a column outside [0, K))
__global__ void spgemm_count_kernel(const int32_t* __restrict__ A_colind, int64_t nnzA,
                                    const int32_t* __restrict__ B_rowptr, int64_t K,
                                    int32_t* __restrict__ cnt, int32_t* status) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnzA; e += stride) {
        const int32_t k = A_colind[e];
        int32_t c = 0;
        if (k >= 0 && k < K) c = B_rowptr[k + 1] - B_rowptr[k];
        else atomicCAS(status, 0, SPMM_ERR_BAD_CSR);
        cnt[e] = c;
    }
}

__global__ void sum_i32_kernel(const int32_t* __restrict__ x, int64_t n,
                               unsigned long long* __restrict__ total) {
    unsigned long long s = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += stride)
        s += (unsigned long long)(uint32_t)x[e];
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(kFull, s, off);
    if ((threadIdx.x & 31) == 0) atomicAdd(total, s);
}

// One warp per nonzero of A: its products, at the nonzero's offset.
__global__ void spgemm_expand_kernel(const int32_t* __restrict__ A_colind,
                                     const float* __restrict__ A_vals,
                                     const int32_t* __restrict__ row_of,
                                     const int32_t* __restrict__ off, int64_t nnzA, int64_t K,
                                     const int32_t* __restrict__ B_rowptr,
                                     const int32_t* __restrict__ B_colind,
                                     const float* __restrict__ B_vals, int64_t N,
                                     int32_t* __restrict__ prow, int32_t* __restrict__ pcol,
                                     float* __restrict__ pval, int32_t* status) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t e = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; e < nnzA; e += nw) {
        const int32_t k = A_colind[e];
        if (k < 0 || k >= K) continue;   // counted as no products
        const int32_t b0 = B_rowptr[k], b1 = B_rowptr[k + 1];
        const int32_t r = row_of[e];
        const float a = A_vals[e];
        const int64_t o = off[e];
        for (int32_t f = b0 + lane; f < b1; f += 32) {
            int32_t j = B_colind[f];
            if (j < 0 || j >= N) {
                atomicCAS(status, 0, SPMM_ERR_BAD_CSR);
                j = 0;
            }
            prow[o + (f - b0)] = r;
            pcol[o + (f - b0)] = j;
            pval[o + (f - b0)] = a * B_vals[f];
        }
    }
}

// Fused-key form (bits(M) + bits(N) <= 32): each product's key is
// (row << bN) | col and its payload the FP32 value, so one stable sort of the
// keys orders the products by (row, col) with equal pairs in expansion order.
__global__ void spgemm_expand_fused_kernel(const int32_t* __restrict__ A_colind,
                                           const float* __restrict__ A_vals,
                                           const int32_t* __restrict__ row_of,
                                           const int32_t* __restrict__ off, int64_t nnzA,
                                           int64_t K, const int32_t* __restrict__ B_rowptr,
                                           const int32_t* __restrict__ B_colind,
                                           const float* __restrict__ B_vals, int64_t N, int bN,
                                           uint32_t* __restrict__ key, float* __restrict__ val,
                                           int32_t* status) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t e = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; e < nnzA; e += nw) {
        const int32_t k = A_colind[e];
        if (k < 0 || k >= K) continue;   // counted as no products
        const int32_t b0 = B_rowptr[k], b1 = B_rowptr[k + 1];
        const uint32_t rk = (uint32_t)row_of[e] << bN;
        const float a = A_vals[e];
        const int64_t o = off[e];
        for (int32_t f = b0 + lane; f < b1; f += 32) {
            int32_t j = B_colind[f];
            if (j < 0 || j >= N) {
                atomicCAS(status, 0, SPMM_ERR_BAD_CSR);
                j = 0;
            }
            key[o + (f - b0)] = rk | (uint32_t)j;
            val[o + (f - b0)] = a * B_vals[f];
        }
    }
}

__global__ void spgemm_heads_fused_kernel(const uint32_t* __restrict__ key, int64_t P,
                                          int32_t* __restrict__ head) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p <= P; p += stride)
        head[p] = p < P && (p == 0 || key[p] != key[p - 1]);
}

// start[q] = first product of entry q (pos[p] for the run heads p), start[E] = P,
// where E = pos[P] is the entry count.
__global__ void spgemm_run_starts_kernel(const int32_t* __restrict__ pos, int64_t P,
                                         int32_t* __restrict__ start) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < P; p += stride)
        if (pos[p + 1] != pos[p]) start[pos[p]] = (int32_t)p;
    if (blockIdx.x == 0 && threadIdx.x == 0) start[pos[P]] = (int32_t)P;
}

// One thread per entry q: the FP32 sum of its products start[q] .. start[q+1]-1
// in order (the loop bounds are known before any value is loaded).
__global__ void spgemm_compress_fused_kernel(const uint32_t* __restrict__ key,
                                             const float* __restrict__ val,
                                             const int32_t* __restrict__ start,
                                             const int32_t* __restrict__ nentries, int bN,
                                             int32_t* __restrict__ crow, int32_t* __restrict__ ccol,
                                             float* __restrict__ cval) {
    const int64_t E = *nentries;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < E; q += stride) {
        const int32_t s0 = start[q], s1 = start[q + 1];
        float sum = val[s0];
        for (int32_t x = s0 + 1; x < s1; ++x) sum += val[x];
        const uint32_t kk = key[s0];
        crow[q] = (int32_t)(kk >> bN);
        ccol[q] = (int32_t)(kk & ((1u << bN) - 1u));
        cval[q] = sum;
    }
}

// rkey[p] = prow[idx[p]], icopy[p] = idx[p]
__global__ void spgemm_rowkeys_kernel(const int32_t* __restrict__ prow,
                                      const int32_t* __restrict__ idx, int64_t P,
                                      int32_t* __restrict__ rkey, int32_t* __restrict__ icopy) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < P; p += stride) {
        const int32_t i = idx[p];
        rkey[p] = prow[i];
        icopy[p] = i;
    }
}

// head[p] = 1 where (row, col) of sorted product p differs from product p-1;
// head[P] = 0 (so the exclusive scan's last element is the entry count)
__global__ void spgemm_heads_kernel(const int32_t* __restrict__ rows,
                                    const int32_t* __restrict__ idx,
                                    const int32_t* __restrict__ pcol, int64_t P,
                                    int32_t* __restrict__ head) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p <= P; p += stride) {
        int32_t h = 0;
        if (p < P) {
            h = p == 0 || rows[p] != rows[p - 1] || pcol[idx[p]] != pcol[idx[p - 1]];
        }
        head[p] = h;
    }
}

// One thread per entry q: sum its products start[q] .. start[q+1]-1 in order.
__global__ void spgemm_compress_kernel(const int32_t* __restrict__ rows,
                                       const int32_t* __restrict__ idx,
                                       const int32_t* __restrict__ pcol,
                                       const float* __restrict__ pval,
                                       const int32_t* __restrict__ start,
                                       const int32_t* __restrict__ nentries,
                                       int32_t* __restrict__ crow, int32_t* __restrict__ ccol,
                                       float* __restrict__ cval) {
    const int64_t E = *nentries;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < E; q += stride) {
        const int32_t s0 = start[q], s1 = start[q + 1];
        float sum = pval[idx[s0]];
        for (int32_t x = s0 + 1; x < s1; ++x) sum += pval[idx[x]];
        crow[q] = rows[s0];
        ccol[q] = pcol[idx[s0]];
        cval[q] = sum;
    }
}

// Workspace: [status word, 256 B][arrays ...]
struct SpgemmLayout {
    size_t row_of, off, scan, prow, pcol, pval, k0, v0, k1, v1, rkey, icopy, pos, start, radix,
        crow, ccol, cval, total;
};

// The radix scratch comes last: its size depends on the key widths (bits of M
// and N), the offsets of the output arrays do not.
SpgemmLayout spgemm_layout(int64_t nnzA, int64_t P, int64_t M, int64_t N) {
    SpgemmLayout L;
    const size_t a = up256(4 * (size_t)(nnzA > 0 ? nnzA : 1));
    const size_t b = up256(4 * (size_t)(P > 0 ? P : 1));
    size_t o = 256;
    L.row_of = o; o += a;
    L.off = o; o += a;
    L.scan = o; o += scan_scratch_bytes(nnzA);
    L.prow = o; o += b;
    L.pcol = o; o += b;
    L.pval = o; o += b;
    L.k0 = o; o += b;
    L.v0 = o; o += b;
    L.k1 = o; o += b;
    L.v1 = o; o += b;
    L.rkey = o; o += b;
    L.icopy = o; o += b;
    L.pos = o; o += up256(4 * (size_t)(P + 1));
    L.start = o; o += up256(4 * (size_t)(P + 1));
    L.crow = o; o += b;
    L.ccol = o; o += b;
    L.cval = o; o += b;
    L.radix = o;
    const int bM = bits_for(M), bN = bits_for(N);
    size_t rs = radix_scratch_bytes(P, bM + bN <= 32 ? bM + bN : bM);
    if (bM + bN > 32) {
        const size_t r2 = radix_scratch_bytes(P, bN);
        if (r2 > rs) rs = r2;
    }
    const size_t ss = scan_scratch_bytes(P + 1);
    o += rs > ss ? rs : ss;
    L.total = o;
    return L;
}

int check_spgemm_args(const int32_t* A_rowptr, const int32_t* A_colind, int64_t M, int64_t K,
                      int64_t nnzA, const int32_t* B_rowptr, int64_t N) {
    const int64_t lim = ((int64_t)1 << 31) - 1;
    if (M < 0 || K < 0 || N < 0 || nnzA < 0 || M >= lim || K >= lim || N >= lim || nnzA >= lim)
        return SPMM_ERR_INVALID_ARG;
    if (!A_rowptr || !B_rowptr || (nnzA > 0 && !A_colind)) return SPMM_ERR_INVALID_ARG;
    return SPMM_OK;
}

}  // namespace

}  // namespace spmm

using namespace spmm;

extern "C" int spmm_spgemm_analyze(const int32_t* A_rowptr, const int32_t* A_colind, int64_t M,
                                   int64_t K, int64_t nnzA, const int32_t* B_rowptr, int64_t N,
                                   int64_t* products, size_t* workspace_bytes, void* stream) {
    int st = check_spgemm_args(A_rowptr, A_colind, M, K, nnzA, B_rowptr, N);
    if (st) return st;
    if (!products || !workspace_bytes) return SPMM_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    int64_t P = 0;
    if (nnzA > 0) {
        int32_t* cnt = nullptr;
        unsigned long long* total = nullptr;
        int32_t* status = nullptr;
        if (cudaMalloc(&cnt, 4 * (size_t)nnzA) != cudaSuccess) return SPMM_ERR_CUDA;
        if (cudaMalloc(&total, 64) != cudaSuccess) {
            cudaFree(cnt);
            return SPMM_ERR_CUDA;
        }
        status = reinterpret_cast<int32_t*>(total + 1);
        int rc = SPMM_OK;
        unsigned long long h[2] = {0, 0};
        if (cudaMemsetAsync(total, 0, 64, s) != cudaSuccess) rc = SPMM_ERR_CUDA;
        if (!rc) {
            spgemm_count_kernel<<<grid_for(nnzA, 256), 256, 0, s>>>(A_colind, nnzA, B_rowptr, K,
                                                                     cnt, status);
            sum_i32_kernel<<<grid_for(nnzA, 256), 256, 0, s>>>(cnt, nnzA, total);
            if (cudaGetLastError() != cudaSuccess ||
                cudaMemcpyAsync(h, total, 16, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                cudaStreamSynchronize(s) != cudaSuccess)
                rc = SPMM_ERR_CUDA;
        }
        cudaFree(total);
        cudaFree(cnt);
        if (rc) return rc;
        if ((int32_t)(h[1] & 0xffffffffu) != 0) return SPMM_ERR_BAD_CSR;
        P = (int64_t)h[0];
    }
    if (P >= ((int64_t)1 << 31) - 1) return SPMM_ERR_UNSUPPORTED;   // products index in int32
    *products = P;
    *workspace_bytes = spgemm_layout(nnzA, P, M, N).total;
    return SPMM_OK;
}

extern "C" int spmm_spgemm(const int32_t* A_rowptr, const int32_t* A_colind, const float* A_vals,
                           int64_t M, int64_t K, int64_t nnzA, const int32_t* B_rowptr,
                           const int32_t* B_colind, const float* B_vals, int64_t N,
                           int64_t products, void* workspace, size_t workspace_bytes,
                           int64_t* entries, void* stream) {
    int st = check_spgemm_args(A_rowptr, A_colind, M, K, nnzA, B_rowptr, N);
    if (st) return st;
    if (!entries || products < 0 || products >= ((int64_t)1 << 31) - 1) return SPMM_ERR_INVALID_ARG;
    if (nnzA > 0 && !A_vals) return SPMM_ERR_INVALID_ARG;
    if (products > 0 && (!B_colind || !B_vals)) return SPMM_ERR_INVALID_ARG;
    const int64_t P = products;
    const SpgemmLayout L = spgemm_layout(nnzA, P, M, N);
    if (!workspace || workspace_bytes < L.total || ((uintptr_t)workspace & 255u))
        return SPMM_ERR_WORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    char* ws = static_cast<char*>(workspace);
    int32_t* status = reinterpret_cast<int32_t*>(ws);
    auto I = [&](size_t o) { return reinterpret_cast<int32_t*>(ws + o); };
    if (cudaMemsetAsync(ws, 0, 256, s) != cudaSuccess) return SPMM_ERR_CUDA;
    if (P > 0) {
        if (csr_rows_of(A_rowptr, M, I(L.row_of), s) != cudaSuccess) return SPMM_ERR_CUDA;
        spgemm_count_kernel<<<grid_for(nnzA, 256), 256, 0, s>>>(A_colind, nnzA, B_rowptr, K,
                                                                 I(L.off), status);
        if (scan_exclusive_i32(I(L.off), nnzA, ws + L.scan, s) != cudaSuccess) return SPMM_ERR_CUDA;
        const int bM = bits_for(M), bN = bits_for(N);
        if (bM + bN <= 32) {
            uint32_t* key = reinterpret_cast<uint32_t*>(ws + L.prow);
            float* val = reinterpret_cast<float*>(ws + L.pval);
            spgemm_expand_fused_kernel<<<grid_for(nnzA * 32, 256), 256, 0, s>>>(
                A_colind, A_vals, I(L.row_of), I(L.off), nnzA, K, B_rowptr, B_colind, B_vals, N,
                bN, key, val, status);
            int r = 0;
            if (radix_sort_pairs(reinterpret_cast<const int32_t*>(key),
                                 reinterpret_cast<const int32_t*>(val), P, bM + bN, I(L.k0),
                                 I(L.v0), I(L.k1), I(L.v1), ws + L.radix, &r, s) != cudaSuccess)
                return SPMM_ERR_CUDA;
            const uint32_t* skey = reinterpret_cast<const uint32_t*>(r ? I(L.k1) : I(L.k0));
            const float* sval = reinterpret_cast<const float*>(r ? I(L.v1) : I(L.v0));
            spgemm_heads_fused_kernel<<<grid_for(P + 1, 256), 256, 0, s>>>(skey, P, I(L.pos));
            if (scan_exclusive_i32(I(L.pos), P + 1, ws + L.radix, s) != cudaSuccess)
                return SPMM_ERR_CUDA;
            spgemm_run_starts_kernel<<<grid_for(P, 256), 256, 0, s>>>(I(L.pos), P, I(L.start));
            spgemm_compress_fused_kernel<<<grid_for(P, 256), 256, 0, s>>>(
                skey, sval, I(L.start), I(L.pos) + P, bN, I(L.crow), I(L.ccol),
                reinterpret_cast<float*>(ws + L.cval));
        } else {
        spgemm_expand_kernel<<<grid_for(nnzA * 32, 256), 256, 0, s>>>(
            A_colind, A_vals, I(L.row_of), I(L.off), nnzA, K, B_rowptr, B_colind, B_vals, N,
            I(L.prow), I(L.pcol), reinterpret_cast<float*>(ws + L.pval), status);
        // stable by column, then stable by row
        int r1 = 0, r2 = 0;
        if (radix_sort_pairs(I(L.pcol), nullptr, P, bits_for(N), I(L.k0), I(L.v0), I(L.k1),
                             I(L.v1), ws + L.radix, &r1, s) != cudaSuccess)
            return SPMM_ERR_CUDA;
        const int32_t* idx1 = r1 ? I(L.v1) : I(L.v0);
        spgemm_rowkeys_kernel<<<grid_for(P, 256), 256, 0, s>>>(I(L.prow), idx1, P, I(L.rkey),
                                                               I(L.icopy));
        if (radix_sort_pairs(I(L.rkey), I(L.icopy), P, bits_for(M), I(L.k0), I(L.v0), I(L.k1),
                             I(L.v1), ws + L.radix, &r2, s) != cudaSuccess)
            return SPMM_ERR_CUDA;
        const int32_t* rows = r2 ? I(L.k1) : I(L.k0);
        const int32_t* idx = r2 ? I(L.v1) : I(L.v0);
        spgemm_heads_kernel<<<grid_for(P + 1, 256), 256, 0, s>>>(rows, idx, I(L.pcol), P,
                                                                 I(L.pos));
        if (scan_exclusive_i32(I(L.pos), P + 1, ws + L.radix, s) != cudaSuccess)
            return SPMM_ERR_CUDA;
        spgemm_run_starts_kernel<<<grid_for(P, 256), 256, 0, s>>>(I(L.pos), P, I(L.start));
        spgemm_compress_kernel<<<grid_for(P, 256), 256, 0, s>>>(
            rows, idx, I(L.pcol), reinterpret_cast<const float*>(ws + L.pval), I(L.start),
            I(L.pos) + P, I(L.crow), I(L.ccol), reinterpret_cast<float*>(ws + L.cval));
        }
        if (cudaGetLastError() != cudaSuccess) return SPMM_ERR_CUDA;
    }
    int32_t h_status = 0;
    int32_t h_entries = 0;
    if (cudaMemcpyAsync(&h_status, status, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return SPMM_ERR_CUDA;
    if (P > 0 && cudaMemcpyAsync(&h_entries, I(L.pos) + P, 4, cudaMemcpyDeviceToHost, s) !=
                     cudaSuccess)
        return SPMM_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return SPMM_ERR_CUDA;
    if (h_status != 0) return h_status;
    *entries = h_entries;
    return SPMM_OK;
}

extern "C" int spmm_spgemm_copy(const void* workspace, int64_t M, int64_t nnzA, int64_t products,
                                int64_t entries, int32_t* C_rowptr, int32_t* C_colind,
                                float* C_vals, void* stream) {
    if (!workspace || !C_rowptr || M < 0 || entries < 0 || entries > products)
        return SPMM_ERR_INVALID_ARG;
    if (entries > 0 && (!C_colind || !C_vals)) return SPMM_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const char* ws = static_cast<const char*>(workspace);
    const SpgemmLayout L = spgemm_layout(nnzA, products, 1, 1);   // output offsets only
    const int32_t* crow = reinterpret_cast<const int32_t*>(ws + L.crow);
    if (entries == 0) {
        if (cudaMemsetAsync(C_rowptr, 0, 4 * (size_t)(M + 1), s) != cudaSuccess) return SPMM_ERR_CUDA;
        return SPMM_OK;
    }
    if (lower_bounds(crow, entries, M, C_rowptr, s) != cudaSuccess) return SPMM_ERR_CUDA;
    if (cudaMemcpyAsync(C_colind, ws + L.ccol, 4 * (size_t)entries, cudaMemcpyDeviceToDevice, s) !=
            cudaSuccess ||
        cudaMemcpyAsync(C_vals, ws + L.cval, 4 * (size_t)entries, cudaMemcpyDeviceToDevice, s) !=
            cudaSuccess)
        return SPMM_ERR_CUDA;
    return SPMM_OK;
}
