// Plan construction: merge-path chunk boundaries for every C row block.
//
// Row block i holds rows [i*RB, min(M, (i+1)*RB)).  Its merge path walks the
// block's row ends and nonzeros in order (a row's nonzeros first, then its
// end), items = rows + nonzeros.  Chunk c of the block covers path steps
// [c*D, (c+1)*D).  Boundary c is the path coordinate (x rows finished,
// y nonzeros consumed) with x + y = c*D; the step at diagonal x + rowend(x)
// finishes row x.  Boundaries that would cut a light row are moved to its
// start, so a row is split between chunks only when it is heavy.  The search
// is the merge-path partition of Merrill and Garland (SC'16) applied per
// block; it balances work the way Section 1 of the paper asks of a schedule
// under skewed (R-MAT) row lengths.
#include "common.cuh"
#include "plan.cuh"

namespace spmm {

// One block of 1024 threads: chunk counts per row block and their exclusive
// prefix, blk_base[0..TR].
__global__ void __launch_bounds__(1024)
plan_blocks_kernel(const int32_t* __restrict__ rowptr, int M, int TR, int RB, int D,
                   int32_t* __restrict__ blk_base) {
    __shared__ int64_t part[1024];
    const int t = threadIdx.x;
    const int per = (TR + 1023) / 1024;
    const int b0 = min(TR, t * per), b1 = min(TR, b0 + per);
    int64_t sum = 0;
    for (int i = b0; i < b1; ++i) {
        const int lo = min(M, i * RB), hi = min(M, lo + RB);
        const int64_t items = (int64_t)(hi - lo) + (rowptr[hi] - rowptr[lo]);
        sum += (items + D - 1) / D;
    }
    part[t] = sum;
    __syncthreads();
    if (t == 0) {
        int64_t run = 0;
        for (int k = 0; k < 1024; ++k) {
            const int64_t v = part[k];
            part[k] = run;
            run += v;
        }
    }
    __syncthreads();
    int64_t run = part[t];
    for (int i = b0; i < b1; ++i) {
        blk_base[i] = (int32_t)run;
        const int lo = min(M, i * RB), hi = min(M, lo + RB);
        const int64_t items = (int64_t)(hi - lo) + (rowptr[hi] - rowptr[lo]);
        run += (items + D - 1) / D;
    }
    if (b1 == TR && b0 < b1) blk_base[TR] = (int32_t)run;
    if (TR == 0 && t == 0) blk_base[0] = 0;
}

// One thread per boundary slot b in [0, blk_base[TR] + TR).  Slot b belongs to
// the block i with blk_base[i] + i <= b < blk_base[i+1] + i + 1; it is boundary
// c = b - blk_base[i] - i (0 <= c <= chunks of block i).
__global__ void plan_bounds_kernel(const int32_t* __restrict__ rowptr, int M, int TR, int RB,
                                   int D, const int32_t* __restrict__ blk_base, int64_t cap,
                                   int32_t* __restrict__ bnd_row, int32_t* __restrict__ bnd_nnz,
                                   int4* __restrict__ split, int32_t* __restrict__ n_split) {
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= cap) return;
    const int64_t total = (int64_t)blk_base[TR] + TR;
    if (b >= total) return;
    int lo = 0, hi = TR - 1;  // largest i with blk_base[i] + i <= b
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if ((int64_t)blk_base[mid] + mid <= b) lo = mid;
        else hi = mid - 1;
    }
    const int i = lo;
    const int64_t c = b - blk_base[i] - i;
    const int row_lo = min(M, i * RB), row_hi = min(M, row_lo + RB);
    const int nnz_lo = rowptr[row_lo];
    const int64_t R = row_hi - row_lo;
    const int64_t Z = (int64_t)rowptr[row_hi] - nnz_lo;
    int64_t d = c * D;
    if (d > R + Z) d = R + Z;
    // first x in [max(0, d - Z), min(d, R)] whose row end lies at or after d
    int64_t xl = d - Z > 0 ? d - Z : 0;
    int64_t xh = d < R ? d : R;
    while (xl < xh) {
        const int64_t mid = (xl + xh) >> 1;
        const int64_t rowend = (int64_t)rowptr[row_lo + mid + 1] - nnz_lo;
        if (rowend <= d - mid - 1) xl = mid + 1;
        else xh = mid;
    }
    // A boundary inside a light row (fewer than D/8 items) moves to that row's
    // start, so only rows of D/8 items or more are ever cut between chunks.
    // The moved boundary stays on the merge path and moves back by less than
    // D/8 (chunks stay within 1/8 of D), and boundaries inside heavier rows
    // stay on exact diagonals.
    int64_t y = d - xl;
    if (xl < R) {
        const int64_t rs = (int64_t)rowptr[row_lo + xl] - nnz_lo;
        const int64_t re = (int64_t)rowptr[row_lo + xl + 1] - nnz_lo;
        if (y > rs && 8 * (re - rs + 1) < D) y = rs;
        // Still inside the row: the row is cut.  The first boundary inside it
        // (the one that ends the chunk where the row's first item lies) lists
        // it, with the chunks of its first item and of its end.
        if (y > rs && c >= 1) {
            const int64_t ca = (xl + rs) / D;
            if (c == ca + 1) {
                const int64_t cb = (xl + re) / D;
                const int k = atomicAdd(n_split, 1);
                split[k] = make_int4(row_lo + (int)xl, blk_base[i] + (int)ca,
                                     blk_base[i] + (int)cb, 0);
            }
        }
    }
    bnd_row[b] = (int32_t)(row_lo + xl);
    bnd_nnz[b] = (int32_t)(nnz_lo + y);
}

// One thread per row: set the bit of the row's end item.
__global__ void plan_ends_kernel(const int32_t* __restrict__ rowptr, int M,
                                 uint32_t* __restrict__ ends) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= M) return;
    const int64_t item = (int64_t)r + rowptr[r + 1];
    atomicOr(ends + (item >> 5), 1u << (item & 31));
}

static int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

size_t plan_ends_bytes(int64_t items) {
    return ((size_t)(ceil_div(items, 32) + 2) * 4 + 255) / 256 * 256;
}

cudaError_t plan_build_ends(const int32_t* rowptr, int64_t M, int64_t items, uint32_t* ends,
                            cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(ends, 0, plan_ends_bytes(items), s);
    if (e != cudaSuccess || M == 0) return e;
    plan_ends_kernel<<<(unsigned)ceil_div(M, 256), 256, 0, s>>>(rowptr, (int)M, ends);
    return cudaGetLastError();
}

int64_t plan_chunk_cap(int64_t M, int64_t nnz, int32_t TR, int32_t D) {
    return ceil_div(M + nnz, D) + TR;
}

int32_t plan_default_chunk(int64_t M, int64_t nnz, int32_t TC, int sms, int groups) {
    const int64_t nwarps = (int64_t)(sms > 0 ? sms : 148) * 32;
    if (groups < 1) groups = 1;
    const int64_t work = (M + nnz) * (int64_t)TC;
    // about 16 units per warp of the full grid, a unit being `groups` chunks
    int64_t d = ceil_div(work, 16 * nwarps * groups);
    // Longer chunks, up to 16 mean rows (M + nnz) / M, while the grid keeps at
    // least 4 units per warp: a boundary cuts only rows of D/8 items or more,
    // and every cut row costs its pieces' slot stores and the fix-up's reads.
    if (M > 0) {
        const int64_t rows16 = ceil_div(16 * (M + nnz), M);
        const int64_t d4 = work / (4 * nwarps * groups);
        const int64_t want = rows16 < d4 ? rows16 : d4;
        if (want > d) d = want;
    }
    if (d < 32) d = 32;   // small problems: enough units to spread over the SMs
    if (d > 16384) d = 16384;
    d = ceil_div(d, 32) * 32;
    return (int32_t)d;
}

int plan_default_groups(int64_t N, int32_t TC) {
    if (TC < 1) TC = 1;
    const int64_t nvec = ((N + TC - 1) / TC + 3) / 4;   // FP32 vectors of a column block
    if (nvec >= 32) return 1;
    int lpn = 2;
    while (lpn < nvec) lpn <<= 1;
    return 32 / lpn;
}

size_t plan_array_bytes(int32_t TR, int64_t cap) {
    size_t a = ((size_t)(TR + 1) * 4 + 255) / 256 * 256;
    size_t b = ((size_t)(cap + TR) * 4 + 255) / 256 * 256;
    size_t l = ((size_t)(cap + TR) * 16 + 255) / 256 * 256;
    return a + 2 * b + l + 256;
}

void plan_carve(void* base, int32_t TR, int64_t cap, int32_t** blk_base, int32_t** bnd_row,
                int32_t** bnd_nnz, int4** split, int32_t** n_split) {
    char* p = static_cast<char*>(base);
    size_t a = ((size_t)(TR + 1) * 4 + 255) / 256 * 256;
    size_t b = ((size_t)(cap + TR) * 4 + 255) / 256 * 256;
    size_t l = ((size_t)(cap + TR) * 16 + 255) / 256 * 256;
    *blk_base = reinterpret_cast<int32_t*>(p);
    *bnd_row = reinterpret_cast<int32_t*>(p + a);
    *bnd_nnz = reinterpret_cast<int32_t*>(p + a + b);
    *split = reinterpret_cast<int4*>(p + a + 2 * b);
    *n_split = reinterpret_cast<int32_t*>(p + a + 2 * b + l);
}

cudaError_t plan_build(const int32_t* rowptr, int64_t M, int32_t TR, int32_t RB, int32_t D,
                       int64_t cap, int32_t* blk_base, int32_t* bnd_row, int32_t* bnd_nnz,
                       int4* split, int32_t* n_split, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(n_split, 0, sizeof(int32_t), s);
    if (e != cudaSuccess) return e;
    plan_blocks_kernel<<<1, 1024, 0, s>>>(rowptr, (int)M, TR, RB, D, blk_base);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int64_t slots = cap + TR;
    const int threads = 256;
    const int64_t blocks = ceil_div(slots, threads);
    plan_bounds_kernel<<<(unsigned)blocks, threads, 0, s>>>(rowptr, (int)M, TR, RB, D, blk_base,
                                                           slots, bnd_row, bnd_nnz, split,
                                                           n_split);
    return cudaGetLastError();
}

}  // namespace spmm
