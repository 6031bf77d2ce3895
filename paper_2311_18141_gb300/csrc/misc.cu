// Small kernels behind the C ABI: CSR validation, row quantisation, value
// gather.
#include "api_internal.cuh"

using namespace spmm;

namespace spmm {

// rowptr[0] == 0, rowptr[M] == nnz, rowptr non-decreasing, colind in [0, K).
// Reads only rowptr[0..M] and colind[0..nnz); any violation stores
// SPMM_ERR_BAD_CSR into status[0].
__global__ void validate_kernel(const int32_t* __restrict__ rowptr,
                                const int32_t* __restrict__ colind, int64_t M, int64_t K,
                                int64_t nnz, int32_t* status) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    bool bad = false;
    for (int64_t r = t0; r <= M; r += stride) {
        const int32_t v = rowptr[r];
        if (r == 0 && v != 0) bad = true;
        if (r == M && (int64_t)v != nnz) bad = true;
        if (r < M && rowptr[r + 1] < v) bad = true;
        if (v < 0 || (int64_t)v > nnz) bad = true;
    }
    for (int64_t e = t0; e < nnz; e += stride) {
        const int32_t c = colind[e];
        if (c < 0 || (int64_t)c >= K) bad = true;
    }
    if (bad) atomicExch(status, SPMM_ERR_BAD_CSR);
}

__device__ __forceinline__ uint8_t f32_to_e4m3_sat(float x) {
    uint16_t two;
    asm("cvt.rn.satfinite.e4m3x2.f32 %0, %1, %2;" : "=h"(two) : "f"(0.0f), "f"(x));
    return (uint8_t)(two & 0xffu);
}

// One warp per row.  E4M3: s = amax/448 (FP32 division, 1 for a zero row),
// q = E4M3(x / s); F16/BF16: round to nearest even, no scale.
__global__ void quantize_rows_kernel(const float* __restrict__ X, int64_t rows, int64_t cols,
                                     int64_t ldx, int dtype, void* __restrict__ Xq, int64_t ldq,
                                     float* __restrict__ scale) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t r = warp; r < rows; r += nwarps) {
        const float* x = X + r * ldx;
        if (dtype == SPMM_E4M3) {
            float amax = 0.0f;
            for (int64_t c = lane; c < cols; c += 32) amax = fmaxf(amax, fabsf(x[c]));
#pragma unroll
            for (int off = 16; off > 0; off >>= 1)
                amax = fmaxf(amax, __shfl_xor_sync(kFull, amax, off));
            float s = __fdiv_rn(amax, 448.0f);
            if (amax == 0.0f) s = 1.0f;
            if (lane == 0) scale[r] = s;
            uint8_t* q = static_cast<uint8_t*>(Xq) + r * ldq;
            for (int64_t c = lane; c < cols; c += 32) q[c] = f32_to_e4m3_sat(__fdiv_rn(x[c], s));
        } else if (dtype == SPMM_BF16) {
            __nv_bfloat16* q = static_cast<__nv_bfloat16*>(Xq) + r * ldq;
            for (int64_t c = lane; c < cols; c += 32) q[c] = __float2bfloat16_rn(x[c]);
            if (scale && lane == 0) scale[r] = 1.0f;
        } else {
            __half* q = static_cast<__half*>(Xq) + r * ldq;
            for (int64_t c = lane; c < cols; c += 32) q[c] = __float2half_rn(x[c]);
            if (scale && lane == 0) scale[r] = 1.0f;
        }
    }
}

template <typename T>
__global__ void gather_kernel(const T* __restrict__ in, const int32_t* __restrict__ perm,
                              int64_t n, T* __restrict__ out) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        out[i] = in[perm[i]];
}

// Bounded-wait self-test.  One thread initialises an mbarrier that expects one
// arrival, never arrives on it, and waits on its first phase for at most
// `limit` SM cycles -- the wait the bulk-copy staging does for its copies.
// When the wait runs out it records SPMM_ERR_TIMEOUT in the status word, the
// way a kernel whose copies never land reports it and returns.
__global__ void wait_timeout_selftest_kernel(int32_t* status, long long limit) {
    __shared__ __align__(8) unsigned long long bar_mem;
    if (threadIdx.x != 0) return;
    const uint32_t bar = (uint32_t)__cvta_generic_to_shared(&bar_mem);
    mbar_init(bar, 1);
    mbar_init_fence();
    bool done = mbar_try_wait(bar, 0);
    const long long t0 = clock64();
    while (!done && clock64() - t0 <= limit) done = mbar_try_wait(bar, 0);
    if (!done) atomicCAS(status, 0, SPMM_ERR_TIMEOUT);
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" :: "r"(bar) : "memory");
}

int device_sm_count();

static unsigned grid_for(int64_t work, int threads) {
    int64_t g = (work + threads - 1) / threads;
    const int64_t cap = (int64_t)device_sm_count() * 16;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    return (unsigned)g;
}

}  // namespace spmm

extern "C" {

int spmm_csr_validate(const int32_t* A_rowptr, const int32_t* A_colind, int64_t M, int64_t K,
                      int64_t nnz, void* workspace, size_t workspace_bytes, void* stream) {
    if (!A_rowptr || M < 0 || K < 0 || nnz < 0 || (nnz > 0 && !A_colind)) return SPMM_ERR_INVALID_ARG;
    if (!workspace || workspace_bytes < kStatusBytes) return SPMM_ERR_WORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    const int threads = 256;
    validate_kernel<<<grid_for((M + 1 > nnz ? M + 1 : nnz), threads), threads, 0, s>>>(
        A_rowptr, A_colind, M, K, nnz, static_cast<int32_t*>(workspace));
    return cudaGetLastError() == cudaSuccess ? SPMM_OK : SPMM_ERR_CUDA;
}

int spmm_quantize_rows(const float* X, int64_t rows, int64_t cols, int64_t ldx, int32_t dtype,
                       void* Xq, int64_t ldq, float* scale, void* stream) {
    if (rows < 0 || cols < 0 || ldx < cols || ldq < cols) return SPMM_ERR_INVALID_ARG;
    if (dtype != SPMM_E4M3 && dtype != SPMM_BF16 && dtype != SPMM_F16) return SPMM_ERR_UNSUPPORTED;
    if (rows == 0 || cols == 0) return SPMM_OK;
    if (!X || !Xq || (dtype == SPMM_E4M3 && !scale)) return SPMM_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const int threads = 256;
    quantize_rows_kernel<<<grid_for(rows * 32, threads), threads, 0, s>>>(X, rows, cols, ldx, dtype,
                                                                         Xq, ldq, scale);
    return cudaGetLastError() == cudaSuccess ? SPMM_OK : SPMM_ERR_CUDA;
}

int spmm_selftest_wait_timeout(void* workspace, size_t workspace_bytes, int64_t limit_cycles,
                               void* stream) {
    if (!workspace || workspace_bytes < kStatusBytes) return SPMM_ERR_WORKSPACE;
    if (limit_cycles < 1 || limit_cycles > ((int64_t)1 << 31)) return SPMM_ERR_INVALID_ARG;
    wait_timeout_selftest_kernel<<<1, 32, 0, (cudaStream_t)stream>>>(
        static_cast<int32_t*>(workspace), (long long)limit_cycles);
    return cudaGetLastError() == cudaSuccess ? SPMM_OK : SPMM_ERR_CUDA;
}

int spmm_gather_values(const void* vals, int32_t val_dtype, const int32_t* perm, int64_t nnz,
                       void* out_vals, void* stream) {
    if (nnz < 0) return SPMM_ERR_INVALID_ARG;
    if (nnz == 0) return SPMM_OK;
    if (!vals || !perm || !out_vals) return SPMM_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const int threads = 256;
    const unsigned g = grid_for(nnz, threads);
    switch (elem_bytes(val_dtype)) {
        case 4: gather_kernel<int32_t><<<g, threads, 0, s>>>((const int32_t*)vals, perm, nnz, (int32_t*)out_vals); break;
        case 2: gather_kernel<uint16_t><<<g, threads, 0, s>>>((const uint16_t*)vals, perm, nnz, (uint16_t*)out_vals); break;
        case 1: gather_kernel<uint8_t><<<g, threads, 0, s>>>((const uint8_t*)vals, perm, nnz, (uint8_t*)out_vals); break;
        default: return SPMM_ERR_UNSUPPORTED;
    }
    return cudaGetLastError() == cudaSuccess ? SPMM_OK : SPMM_ERR_CUDA;
}

}  // extern "C"
