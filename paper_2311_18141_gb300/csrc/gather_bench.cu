// B-gather microbenchmark: the B term of the local product C_ij += A_ik B_kj
// (Section 2.1) without the rest of the product.  Section 4's local-SpMM byte
// count reads B once, and the paper notes that rows of B may have to be
// reloaded; this kernel measures what that reloading costs on its own.  It
// reads, for every nonzero of A and every column block, the block's segment
// of B row colind[e] -- exactly the gathers the SpMM kernels issue, in the
// same order as their interleaved tile-row queue -- and nothing else: no row
// pointers, no values, no C.  Its time is a floor for any SpMM that gathers a
// B row segment per nonzero, and an ncu capture of it gives B's own L2 hit
// rate.
#include "api_internal.cuh"
#include "launch.cuh"

namespace spmm {

namespace {

constexpr int kGatherInFlight = 4;   // 32-byte loads in flight per lane

// Ticket k (warp-strided) is chunk c = k / TC of column block j = k % TC.
// Chunk c covers nonzero positions [c*CH, c*CH + CH), CH = G*S; lane group g
// of the warp reads positions c*CH + g*S .. + S - 1 in order, each as LPN
// lanes x 32 bytes (the block's segment; lanes past the segment re-read its
// first vector).  Every value read is added into a per-lane sum, and the
// warp's sums go into *out with one atomic add, so no load can be dropped.
template <int LPN>
__global__ void __launch_bounds__(256)
gather_bench_kernel(const char* __restrict__ B, uint32_t ldb_bytes, uint32_t seg_bytes,
                    const int32_t* __restrict__ colind, int nnz, int TC, int S, float* out) {
    constexpr int G = 32 / LPN;
    constexpr int U = kGatherInFlight;
    const int lane = threadIdx.x & 31;
    const int g = lane / LPN, t = lane % LPN;
    const int warp = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int nwarps = gridDim.x * (blockDim.x >> 5);
    const int CH = G * S;
    const int nchunks = (nnz + CH - 1) / CH;
    const int64_t tickets = (int64_t)nchunks * TC;
    const uint32_t lane_off = (uint32_t)t * 32 < seg_bytes ? (uint32_t)t * 32 : 0u;
    float acc[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) acc[q] = 0.0f;
    for (int64_t k = warp; k < tickets; k += nwarps) {
        const int c = (int)(k / TC);
        const int j = (int)(k - (int64_t)c * TC);
        const char* bj = B + (uint64_t)j * seg_bytes + lane_off;
        const int first = c * CH + g * S;
        const int end = min(first + S, nnz);
        for (int pos = first; pos < first + S; pos += U) {
            V32 r[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                // positions past the end re-read the group's last position
                const int pp = pos + u < end ? pos + u : max(end - 1, 0);
                const int col = __ldg(colind + pp);   // L1-cached: a group reads its positions in order
                r[u] = ld_gather32(bj + (uint64_t)(uint32_t)col * ldb_bytes);
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const bool live = pos + u < end;
                acc[0] += live ? __uint_as_float(r[u].lo.x) : 0.0f;
                acc[1] += live ? __uint_as_float(r[u].lo.y) : 0.0f;
                acc[2] += live ? __uint_as_float(r[u].lo.z) : 0.0f;
                acc[3] += live ? __uint_as_float(r[u].lo.w) : 0.0f;
                acc[4] += live ? __uint_as_float(r[u].hi.x) : 0.0f;
                acc[5] += live ? __uint_as_float(r[u].hi.y) : 0.0f;
                acc[6] += live ? __uint_as_float(r[u].hi.z) : 0.0f;
                acc[7] += live ? __uint_as_float(r[u].hi.w) : 0.0f;
            }
        }
    }
    // lanes whose 32 bytes lie past the segment read the segment's first
    // vector again: they take part in the traffic, not in the sum
    float s = 0.0f;
    if ((uint32_t)t * 32 < seg_bytes) {
#pragma unroll
        for (int q = 0; q < 8; ++q) s += acc[q];
    }
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) s += __shfl_xor_sync(kFull, s, off);
    if (lane == 0) atomicAdd(out, s);
}

template <int LPN>
cudaError_t launch_gather(const char* B, uint32_t ldb_bytes, uint32_t seg_bytes,
                          const int32_t* colind, int nnz, int TC, int S, float* out,
                          int ctas_per_sm, cudaStream_t s) {
    static std::atomic<int> cache[kMaxDevices][kOccSlots];
    auto kern = gather_bench_kernel<LPN>;
    const int per_sm = cached_ctas_per_sm(kern, 256, 0, cache);
    if (per_sm == 0) return cudaErrorInvalidValue;
    constexpr int G = 32 / LPN;
    const int64_t tickets = ((int64_t)nnz + (int64_t)G * S - 1) / ((int64_t)G * S) * TC;
    const int64_t grid = persistent_grid(per_sm, ctas_per_sm, tickets, 8);
    kern<<<(unsigned)grid, 256, 0, s>>>(B, ldb_bytes, seg_bytes, colind, nnz, TC, S, out);
    return cudaGetLastError();
}

}  // namespace

}  // namespace spmm

using namespace spmm;

extern "C" int spmm_bench_gather(const int32_t* A_colind, int64_t nnz, const void* B,
                                 int32_t b_dtype, int64_t ldb, int64_t K, int64_t N,
                                 int32_t tile_cols, int32_t items_per_group,
                                 int32_t ctas_per_sm, float* out, void* stream) {
    (void)K;
    const int eb = elem_bytes(b_dtype);
    if (eb == 0) return SPMM_ERR_UNSUPPORTED;
    if (nnz < 0 || N <= 0 || tile_cols < 1 || ldb < N || items_per_group < 4 ||
        items_per_group > 4096 || items_per_group % kGatherInFlight != 0 || ctas_per_sm < 0)
        return SPMM_ERR_INVALID_ARG;
    // chunk offsets (up to nnz plus two chunks of 16 x 4096 positions) stay in int32
    if (nnz >= ((int64_t)1 << 31) - ((int64_t)1 << 18) || ldb * eb >= ((int64_t)1 << 32))
        return SPMM_ERR_INVALID_ARG;
    if (!out || (nnz > 0 && (!A_colind || !B))) return SPMM_ERR_INVALID_ARG;
    if (N % tile_cols != 0) return SPMM_ERR_INVALID_ARG;
    const int64_t seg = N / tile_cols * eb;   // bytes of one column block's segment
    if (seg % 32 != 0 || seg < 64 || seg > 1024 || (ldb * eb) % 32 != 0 ||
        ((uintptr_t)B & 31u))
        return SPMM_ERR_MISALIGNED;
    if (nnz == 0) return SPMM_OK;
    int lpn = 2;
    while (lpn * 32 < seg) lpn <<= 1;
    cudaStream_t s = (cudaStream_t)stream;
    const char* b = static_cast<const char*>(B);
    const uint32_t ldb_bytes = (uint32_t)(ldb * eb);
    cudaError_t e;
    switch (lpn) {
        case 2: e = launch_gather<2>(b, ldb_bytes, (uint32_t)seg, A_colind, (int)nnz, tile_cols,
                                     items_per_group, out, ctas_per_sm, s); break;
        case 4: e = launch_gather<4>(b, ldb_bytes, (uint32_t)seg, A_colind, (int)nnz, tile_cols,
                                     items_per_group, out, ctas_per_sm, s); break;
        case 8: e = launch_gather<8>(b, ldb_bytes, (uint32_t)seg, A_colind, (int)nnz, tile_cols,
                                     items_per_group, out, ctas_per_sm, s); break;
        case 16: e = launch_gather<16>(b, ldb_bytes, (uint32_t)seg, A_colind, (int)nnz,
                                       tile_cols, items_per_group, out, ctas_per_sm, s); break;
        default: e = launch_gather<32>(b, ldb_bytes, (uint32_t)seg, A_colind, (int)nnz,
                                       tile_cols, items_per_group, out, ctas_per_sm, s); break;
    }
    return e == cudaSuccess ? SPMM_OK : SPMM_ERR_CUDA;
}
