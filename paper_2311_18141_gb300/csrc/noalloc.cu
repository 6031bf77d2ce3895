// spmm_csr_noalloc: spmm_csr for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc at the point where they need the
// product: code running inside a memory pool they do not own, plugins whose
// host application forbids device allocation, or code paths that must not
// synchronise the device (cudaMalloc/cudaFree can).  This entry point needs
// no workspace from them: its scratch (plan arrays, work counters and partial
// rows) lives in one file-scope device array of fixed size that every GPU
// loading this library holds until the process exits.
#include <mutex>

#include "api_internal.cuh"

namespace {

constexpr size_t kStaticScratchBytes = size_t(16) << 20;   // 16 MiB per device
constexpr int kMaxDevices = 64;

// In host code this name is only a host-side stand-in for the device array;
// its device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

std::mutex g_mutex;
void* g_scratch_ptr[kMaxDevices] = {};

// Device address of g_static_scratch on the current device, looked up once per
// device (with that device current) and cached.
int static_scratch(void** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return SPMM_ERR_CUDA;
    if (dev < 0 || dev >= kMaxDevices) return SPMM_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || !p) return SPMM_ERR_CUDA;
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return SPMM_OK;
}

}  // namespace

extern "C" int spmm_csr_noalloc(const int32_t* A_rowptr, const int32_t* A_colind,
                                const void* A_vals, int32_t a_dtype, const float* A_row_scale,
                                const void* B, int32_t b_dtype, const float* B_row_scale,
                                int64_t ldb, float* C, int64_t ldc, int64_t M, int64_t K,
                                int64_t N, int64_t nnz, int32_t tile_rows, int32_t tile_cols,
                                float beta, void* stream) {
    if (M == 0 || N == 0) return SPMM_OK;
    size_t need = 0;
    int st = spmm_csr_workspace_size(M, nnz, N, tile_rows, tile_cols, nullptr, &need);
    if (st != SPMM_OK) return st;
    if (need > kStaticScratchBytes) return SPMM_ERR_WORKSPACE;   // problem too large
    void* ws = nullptr;
    st = static_scratch(&ws);
    if (st != SPMM_OK) return st;
    // the array keeps the previous call's contents: clear its status word
    if (cudaMemsetAsync(ws, 0, spmm::kStatusBytes, (cudaStream_t)stream) != cudaSuccess)
        return SPMM_ERR_CUDA;
    return spmm_csr(A_rowptr, A_colind, A_vals, a_dtype, A_row_scale, B, b_dtype, B_row_scale,
                    ldb, C, ldc, M, K, N, nnz, tile_rows, tile_cols, beta, nullptr, ws,
                    kStaticScratchBytes, stream);
}

extern "C" int spmm_csr_noalloc_status(int32_t* status, void* stream) {
    if (!status) return SPMM_ERR_INVALID_ARG;
    void* ws = nullptr;
    const int st = static_scratch(&ws);
    if (st != SPMM_OK) return st;
    // the same read-and-clear as spmm_get_device_status, on the array's words
    return spmm_get_device_status(ws, status, stream);
}
