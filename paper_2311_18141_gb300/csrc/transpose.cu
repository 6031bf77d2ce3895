// CSR -> CSC (the CSR of A^T) on the device, for the backward dB = A^T dC.
//
// The nonzeros are sorted by column with a stable least-significant-digit
// radix sort (8-bit digits) carrying each nonzero's CSR position e.  The CSR
// order lists rows in increasing order, so stability leaves every column's
// rows increasing and the output is the same on every run.  Then
//   perm[p]      = e of the nonzero that lands at CSC position p,
//   rowind[p]    = row of nonzero perm[p],
//   vals_t[p]    = vals[perm[p]],
//   colptr[c]    = first p whose column >= c (binary search of the sorted keys).
// Each radix pass is per-tile digit counts, an exclusive scan over the
// digit-major count table (three small kernels), and a stable scatter in which
// every tile ranks its keys in index order (a warp-level multisplit) and
// writes each digit's keys as one contiguous run.
#include "api_internal.cuh"
#include "radix.cuh"

namespace spmm {

constexpr int kSortThreads = 256;
constexpr int kSortItems = 16;                         // keys per thread per tile
constexpr int kTile = kSortThreads * kSortItems;       // 4096 keys per tile
constexpr int kMaxDigitBits = 9;   // digits of 8 or 9 bits: wider digits leave runs of 2-4 keys per
                                   // digit and tile, whose scattered stores cost more than a pass
constexpr int kScanBlock = 1024;                       // scan: elements per block-thread group

int device_sm_count();

// row_of[e] = row containing nonzero e (one warp per row).
__global__ void expand_rows_kernel(const int32_t* __restrict__ rowptr, int64_t M,
                                   int32_t* __restrict__ row_of) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < M; r += nw) {
        const int32_t a = rowptr[r], b = rowptr[r + 1];
        for (int32_t e = a + lane; e < b; e += 32) row_of[e] = (int32_t)r;
    }
}

// counts[d * ntiles + tile] = number of keys of the tile with digit d (digits of
// DB bits).
template <int DB>
__global__ void __launch_bounds__(kSortThreads)
radix_count_kernel(const int32_t* __restrict__ keys, int64_t n, int shift, int64_t ntiles,
                   int32_t* __restrict__ counts) {
    constexpr int kRadix = 1 << DB;
    __shared__ int32_t h[kRadix];
    for (int d = threadIdx.x; d < kRadix; d += kSortThreads) h[d] = 0;
    __syncthreads();
    const int64_t tile = blockIdx.x;
    const int64_t base = tile * kTile;
    int32_t rkey[kSortItems];
#pragma unroll
    for (int k = 0; k < kSortItems; ++k) {
        const int64_t idx = base + (int64_t)k * kSortThreads + threadIdx.x;
        rkey[k] = idx < n ? keys[idx] : 0;
    }
#pragma unroll
    for (int k = 0; k < kSortItems; ++k)
        if (base + (int64_t)k * kSortThreads + threadIdx.x < n)
            atomicAdd(&h[((uint32_t)rkey[k] >> shift) & (kRadix - 1)], 1);
    __syncthreads();
    for (int d = threadIdx.x; d < kRadix; d += kSortThreads) counts[(int64_t)d * ntiles + tile] = h[d];
}

// Exclusive scan, three phases: block sums, scan of block sums, block scan.
__global__ void __launch_bounds__(1024)
scan_block_sums_kernel(const int32_t* __restrict__ in, int64_t n, int64_t per_block,
                       int64_t* __restrict__ sums) {
    __shared__ int64_t red[1024];
    const int64_t lo = (int64_t)blockIdx.x * per_block;
    const int64_t hi = min(n, lo + per_block);
    int64_t s = 0;
    for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) s += in[i];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int off = 512; off > 0; off >>= 1) {
        if ((int)threadIdx.x < off) red[threadIdx.x] += red[threadIdx.x + off];
        __syncthreads();
    }
    if (threadIdx.x == 0) sums[blockIdx.x] = red[0];
}

// Exclusive scan of the nb block sums, in place, by one block of 1024 threads:
// each thread sums a run of consecutive entries, the 1024 run totals are
// scanned in shared memory, and each thread writes its run's prefixes.
__global__ void __launch_bounds__(1024) scan_sums_serial_kernel(int64_t* sums, int64_t nb) {
    __shared__ int64_t part[1024];
    const int64_t per = (nb + 1023) / 1024;
    const int64_t a = min(nb, (int64_t)threadIdx.x * per);
    const int64_t b = min(nb, a + per);
    int64_t s = 0;
    for (int64_t i = a; i < b; ++i) s += sums[i];
    part[threadIdx.x] = s;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        const int64_t v = (int)threadIdx.x >= off ? part[threadIdx.x - off] : 0;
        __syncthreads();
        part[threadIdx.x] += v;
        __syncthreads();
    }
    int64_t run = threadIdx.x ? part[threadIdx.x - 1] : 0;
    for (int64_t i = a; i < b; ++i) {
        const int64_t v = sums[i];
        sums[i] = run;
        run += v;
    }
}

__global__ void __launch_bounds__(1024)
scan_apply_kernel(int32_t* __restrict__ data, int64_t n, int64_t per_block,
                  const int64_t* __restrict__ sums) {
    // The block's range, 1024 elements at a time: coalesced loads, a warp
    // shuffle scan, a scan of the 32 warp totals, and a running block offset.
    __shared__ int64_t wsum[32];
    __shared__ int64_t carry;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t lo = (int64_t)blockIdx.x * per_block;
    const int64_t hi = min(n, lo + per_block);
    if (threadIdx.x == 0) carry = sums[blockIdx.x];
    __syncthreads();
    for (int64_t t0 = lo; t0 < hi; t0 += 1024) {
        const int64_t i = t0 + threadIdx.x;
        const int64_t v = i < hi ? data[i] : 0;
        int64_t x = v;   // inclusive scan within the warp
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int64_t y = __shfl_up_sync(kFull, x, off);
            if (lane >= off) x += y;
        }
        if (lane == 31) wsum[warp] = x;
        __syncthreads();
        if (warp == 0) {
            int64_t w = wsum[lane];
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const int64_t y = __shfl_up_sync(kFull, w, off);
                if (lane >= off) w += y;
            }
            wsum[lane] = w;   // inclusive over warps
        }
        __syncthreads();
        const int64_t base = carry + (warp ? wsum[warp - 1] : 0);
        if (i < hi) data[i] = (int32_t)(base + x - v);
        __syncthreads();
        if (threadIdx.x == 0) carry += wsum[31];
        __syncthreads();
    }
}

// Stable scatter of one radix pass (a warp-level multisplit).  Warp w owns
// keys w*KW .. w*KW+KW-1 of the tile (KW = 32 * kSortItems), taken 32 at a
// time in index order; within each group of 32, the lanes holding the same
// digit are found with match_any, and each key's rank within its digit is the
// warp's running count of that digit plus its rank among those lanes.  Keys
// are then placed in shared memory at (tile-local start of the digit) +
// (earlier warps' count of the digit) + (rank): (digit, index) order, stable.
// The tile is written out in that order, so each digit's keys leave as one
// contiguous run at the digit's global offset (coalesced stores).  Digits of DB
// bits; the digit tables live in dynamic shared memory (scatter_smem_bytes(DB)),
// the staged keys and payloads in static shared memory.
constexpr size_t scatter_smem_bytes(int db) {
    return 4 * (size_t)(kSortThreads / 32 + 3) * ((size_t)1 << db);
}

template <int DB>
__global__ void __launch_bounds__(kSortThreads, 2)
radix_scatter_kernel(const int32_t* __restrict__ keys_in, const int32_t* __restrict__ vals_in,
                     int64_t n, int shift, int64_t ntiles, const int32_t* __restrict__ offsets,
                     int32_t* __restrict__ keys_out, int32_t* __restrict__ vals_out) {
    constexpr int kRadix = 1 << DB;
    constexpr int W = kSortThreads / 32;
    constexpr int KW = 32 * kSortItems;     // keys per warp
    extern __shared__ int32_t radix_smem[];
    // per-warp digit counts, then per-warp offsets
    int32_t(*__restrict__ wc)[kRadix] = reinterpret_cast<int32_t(*)[kRadix]>(radix_smem);
    int32_t* __restrict__ tot = radix_smem + W * kRadix;   // tile digit counts
    int32_t* __restrict__ lstart = tot + kRadix;           // tile-local start of each digit
    int32_t* __restrict__ gdelta = lstart + kRadix;        // global offset - local start
    __shared__ int32_t skey[kTile];
    __shared__ int32_t sval[kTile];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t tile = blockIdx.x;
    const int64_t t0 = tile * kTile;
    const int cnt = (int)min((int64_t)kTile, n - t0);
    for (int q = threadIdx.x; q < W * kRadix; q += kSortThreads) (&wc[0][0])[q] = 0;
    int32_t rkey[kSortItems], rval[kSortItems];
#pragma unroll
    for (int k = 0; k < kSortItems; ++k) {
        const int li = warp * KW + k * 32 + lane;
        rkey[k] = li < cnt ? keys_in[t0 + li] : 0;
        rval[k] = li < cnt ? (vals_in ? vals_in[t0 + li] : (int32_t)(t0 + li)) : 0;
    }
    __syncthreads();
    int32_t rr[kSortItems];   // rank within (warp, digit)
#pragma unroll
    for (int k = 0; k < kSortItems; ++k) {
        const bool ok = warp * KW + k * 32 + lane < cnt;
        const int d = ok ? (int)(((uint32_t)rkey[k] >> shift) & (kRadix - 1)) : kRadix;   // kRadix = none
        const unsigned peers = __match_any_sync(kFull, d);
        const int r = __popc(peers & ((1u << lane) - 1u));
        const int32_t before = ok ? wc[warp][d] : 0;
        rr[k] = before + r;
        __syncwarp();
        if (ok && r == 0) wc[warp][d] = before + __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    // per digit: offsets of the warps, and the tile total
    for (int d = threadIdx.x; d < kRadix; d += kSortThreads) {
        int32_t run = 0;
        for (int w = 0; w < W; ++w) {
            const int32_t c = wc[w][d];
            wc[w][d] = run;
            run += c;
        }
        tot[d] = run;
    }
    __syncthreads();
    if (warp == 0) {   // exclusive scan of the digit totals
        int32_t run = 0;
        for (int d0 = 0; d0 < kRadix; d0 += 32) {
            const int32_t c = tot[d0 + lane];
            int32_t x = c;
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const int32_t y = __shfl_up_sync(kFull, x, off);
                if (lane >= off) x += y;
            }
            lstart[d0 + lane] = run + x - c;
            run += __shfl_sync(kFull, x, 31);
        }
    }
    __syncthreads();
    for (int d = threadIdx.x; d < kRadix; d += kSortThreads)
        gdelta[d] = offsets[(int64_t)d * ntiles + tile] - lstart[d];
#pragma unroll
    for (int k = 0; k < kSortItems; ++k) {
        if (warp * KW + k * 32 + lane < cnt) {
            const int d = (int)(((uint32_t)rkey[k] >> shift) & (kRadix - 1));
            const int32_t lp = lstart[d] + wc[warp][d] + rr[k];
            skey[lp] = rkey[k];
            sval[lp] = rval[k];
        }
    }
    __syncthreads();
    // write out in (digit, index) order: runs of equal digits are contiguous
    for (int lp = threadIdx.x; lp < cnt; lp += kSortThreads) {
        const int32_t key = skey[lp];
        const int d = (int)(((uint32_t)key >> shift) & (kRadix - 1));
        const int64_t pos = (int64_t)gdelta[d] + lp;
        keys_out[pos] = key;
        vals_out[pos] = sval[lp];
    }
}

// colptr[c] = lower_bound(sorted_keys, c), c in [0, K].
__global__ void colptr_kernel(const int32_t* __restrict__ sorted, int64_t n, int64_t K,
                              int32_t* __restrict__ colptr) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c <= K; c += stride) {
        int64_t lo = 0, hi = n;
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            if ((int64_t)sorted[mid] < c) lo = mid + 1;
            else hi = mid;
        }
        colptr[c] = (int32_t)lo;
    }
}

template <typename T>
__global__ void finish_kernel(const int32_t* __restrict__ perm, const int32_t* __restrict__ row_of,
                              const T* __restrict__ vals, int64_t n, int32_t* __restrict__ rowind,
                              T* __restrict__ vals_t, int32_t* __restrict__ perm_out) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += stride) {
        const int32_t e = perm[p];
        rowind[p] = row_of[e];
        if (vals_t) vals_t[p] = vals[e];
        if (perm_out) perm_out[p] = e;
    }
}

static size_t up256(size_t x) { return (x + 255) / 256 * 256; }

static unsigned grid_cap(int64_t work, int threads) {
    int64_t g = (work + threads - 1) / threads;
    const int64_t cap = (int64_t)device_sm_count() * 8;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    return (unsigned)g;
}

// Scan layout for n int32 elements: blocks of per_block elements.
struct ScanLayout {
    int64_t per_block, blocks;
};
static ScanLayout scan_layout(int64_t n) {
    ScanLayout L;
    L.per_block = 8 * kScanBlock;
    L.blocks = (n + L.per_block - 1) / L.per_block;
    if (L.blocks < 1) L.blocks = 1;
    return L;
}

size_t scan_scratch_bytes(int64_t n) { return up256(8 * (size_t)scan_layout(n).blocks); }

cudaError_t scan_exclusive_i32(int32_t* data, int64_t n, void* scratch, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const ScanLayout L = scan_layout(n);
    int64_t* sums = static_cast<int64_t*>(scratch);
    scan_block_sums_kernel<<<(unsigned)L.blocks, 1024, 0, s>>>(data, n, L.per_block, sums);
    scan_sums_serial_kernel<<<1, 1024, 0, s>>>(sums, L.blocks);
    scan_apply_kernel<<<(unsigned)L.blocks, 1024, 0, s>>>(data, n, L.per_block, sums);
    return cudaGetLastError();
}

// Passes and digit width for keys of key_bits bits: the fewest passes of at
// most kMaxDigitBits bits, each digit as narrow as that allows but at least 8.
static void radix_digits(int key_bits, int* passes, int* width) {
    int p = (key_bits + kMaxDigitBits - 1) / kMaxDigitBits;
    if (p < 1) p = 1;
    int w = (key_bits + p - 1) / p;
    if (w < 8) w = 8;
    *passes = p;
    *width = w;
}

// Radix scratch: the digit-major count table (buckets x tiles) and its scan sums.
size_t radix_scratch_bytes(int64_t n, int key_bits) {
    int passes = 0, width = 0;
    radix_digits(key_bits, &passes, &width);
    const int64_t ntiles = n > 0 ? (n + kTile - 1) / kTile : 1;
    const int64_t ncounts = ntiles << width;
    return up256(4 * (size_t)ncounts) + scan_scratch_bytes(ncounts);
}

// One pass over digits of DB bits at `shift`: count, scan, scatter.
template <int DB>
static cudaError_t radix_pass(const int32_t* kin, const int32_t* vin, int64_t n, int shift,
                              int64_t ntiles, int32_t* counts, void* sums, int32_t* kout,
                              int32_t* vout, cudaStream_t s) {
    const int64_t ncounts = ntiles << DB;
    const size_t smem = scatter_smem_bytes(DB);
    cudaError_t e = cudaFuncSetAttribute(radix_scatter_kernel<DB>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    radix_count_kernel<DB><<<(unsigned)ntiles, kSortThreads, 0, s>>>(kin, n, shift, ntiles, counts);
    e = scan_exclusive_i32(counts, ncounts, sums, s);
    if (e != cudaSuccess) return e;
    radix_scatter_kernel<DB><<<(unsigned)ntiles, kSortThreads, smem, s>>>(kin, vin, n, shift, ntiles,
                                                                          counts, kout, vout);
    return cudaGetLastError();
}

cudaError_t radix_sort_pairs(const int32_t* keys, const int32_t* vals, int64_t n, int key_bits,
                             int32_t* k0, int32_t* v0, int32_t* k1, int32_t* v1, void* scratch,
                             int* out, cudaStream_t s) {
    *out = 0;
    if (n <= 0) return cudaSuccess;
    int passes = 0, width = 0;
    radix_digits(key_bits, &passes, &width);
    const int64_t ntiles = (n + kTile - 1) / kTile;
    const int64_t ncounts = ntiles << width;
    int32_t* counts = static_cast<int32_t*>(scratch);
    void* sums = static_cast<char*>(scratch) + up256(4 * (size_t)ncounts);
    int32_t* kb[2] = {k0, k1};
    int32_t* vb[2] = {v0, v1};
    const int32_t* kin = keys;
    const int32_t* vin = vals;   // nullptr: first pass carries the index
    int cur = 0;
    for (int pass = 0; pass < passes; ++pass) {
        const int shift = width * pass;
        cudaError_t e;
        if (width == 8)
            e = radix_pass<8>(kin, vin, n, shift, ntiles, counts, sums, kb[cur], vb[cur], s);
        else
            e = radix_pass<9>(kin, vin, n, shift, ntiles, counts, sums, kb[cur], vb[cur], s);
        if (e != cudaSuccess) return e;
        kin = kb[cur];
        vin = vb[cur];
        *out = cur;
        cur ^= 1;
    }
    return cudaGetLastError();
}

cudaError_t csr_rows_of(const int32_t* rowptr, int64_t M, int32_t* row_of, cudaStream_t s) {
    if (M <= 0) return cudaSuccess;
    expand_rows_kernel<<<grid_cap(M * 32, 256), 256, 0, s>>>(rowptr, M, row_of);
    return cudaGetLastError();
}

cudaError_t lower_bounds(const int32_t* sorted, int64_t n, int64_t K, int32_t* ptr,
                         cudaStream_t s) {
    colptr_kernel<<<grid_cap(K + 1, 256), 256, 0, s>>>(sorted, n, K, ptr);
    return cudaGetLastError();
}

int bits_for(int64_t n) {
    int bits = 1;
    while (bits < 31 && ((int64_t)1 << bits) < n) ++bits;
    return bits;
}

struct TransposeLayout {
    size_t row_of, keys0, keys1, vals0, vals1, scratch, total;
};

static TransposeLayout transpose_layout(int64_t nnz, int64_t K) {
    TransposeLayout L;
    size_t off = 0;
    const size_t a = up256(4 * (size_t)(nnz > 0 ? nnz : 1));
    L.row_of = off; off += a;
    L.keys0 = off; off += a;
    L.keys1 = off; off += a;
    L.vals0 = off; off += a;
    L.vals1 = off; off += a;
    L.scratch = off; off += radix_scratch_bytes(nnz, bits_for(K));
    L.total = off;
    return L;
}

}  // namespace spmm

using namespace spmm;

extern "C" int spmm_csr_transpose_workspace_size(int64_t M, int64_t K, int64_t nnz,
                                                 size_t* bytes) {
    if (!bytes || M < 0 || K < 0 || nnz < 0) return SPMM_ERR_INVALID_ARG;
    *bytes = transpose_layout(nnz, K).total;
    return SPMM_OK;
}

extern "C" int spmm_csr_transpose(const int32_t* A_rowptr, const int32_t* A_colind,
                                  const void* A_vals, int32_t val_dtype, int64_t M, int64_t K,
                                  int64_t nnz, int32_t* out_colptr, int32_t* out_rowind,
                                  void* out_vals, int32_t* out_perm, void* workspace,
                                  size_t workspace_bytes, void* stream) {
    if (M < 0 || K < 0 || nnz < 0 || nnz >= ((int64_t)1 << 31) - 1) return SPMM_ERR_INVALID_ARG;
    if (K >= ((int64_t)1 << 31) - 1) return SPMM_ERR_INVALID_ARG;
    if (!A_rowptr || !out_colptr || (nnz > 0 && (!A_colind || !out_rowind)))
        return SPMM_ERR_INVALID_ARG;
    if (out_vals && elem_bytes(val_dtype) == 0) return SPMM_ERR_UNSUPPORTED;
    if (nnz > 0 && out_vals && !A_vals) return SPMM_ERR_INVALID_ARG;
    const TransposeLayout L = transpose_layout(nnz, K);
    if (!workspace || workspace_bytes < L.total || ((uintptr_t)workspace & 255u))
        return SPMM_ERR_WORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    char* ws = static_cast<char*>(workspace);
    if (nnz == 0) {
        if (cudaMemsetAsync(out_colptr, 0, 4 * (size_t)(K + 1), s) != cudaSuccess) return SPMM_ERR_CUDA;
        return SPMM_OK;
    }
    int32_t* row_of = reinterpret_cast<int32_t*>(ws + L.row_of);
    int32_t* kb[2] = {reinterpret_cast<int32_t*>(ws + L.keys0), reinterpret_cast<int32_t*>(ws + L.keys1)};
    int32_t* vb[2] = {reinterpret_cast<int32_t*>(ws + L.vals0), reinterpret_cast<int32_t*>(ws + L.vals1)};

    if (csr_rows_of(A_rowptr, M, row_of, s) != cudaSuccess) return SPMM_ERR_CUDA;
    int res = 0;
    if (radix_sort_pairs(A_colind, nullptr, nnz, bits_for(K), kb[0], vb[0], kb[1], vb[1],
                         ws + L.scratch, &res, s) != cudaSuccess)
        return SPMM_ERR_CUDA;
    const int32_t* kin = kb[res];
    const int32_t* vin = vb[res];
    colptr_kernel<<<grid_cap(K + 1, 256), 256, 0, s>>>(kin, nnz, K, out_colptr);
    const unsigned g = grid_cap(nnz, 256);
    switch (out_vals ? elem_bytes(val_dtype) : 4) {
        case 4: finish_kernel<int32_t><<<g, 256, 0, s>>>(vin, row_of, (const int32_t*)A_vals, nnz, out_rowind, (int32_t*)out_vals, out_perm); break;
        case 2: finish_kernel<uint16_t><<<g, 256, 0, s>>>(vin, row_of, (const uint16_t*)A_vals, nnz, out_rowind, (uint16_t*)out_vals, out_perm); break;
        default: finish_kernel<uint8_t><<<g, 256, 0, s>>>(vin, row_of, (const uint8_t*)A_vals, nnz, out_rowind, (uint8_t*)out_vals, out_perm); break;
    }
    return cudaGetLastError() == cudaSuccess ? SPMM_OK : SPMM_ERR_CUDA;
}
