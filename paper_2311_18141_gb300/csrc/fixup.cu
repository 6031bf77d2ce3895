// Split rows of the staged product, summed after the persistent launch.
//
// The plan cuts a row block's merge path into chunks; a chunk boundary inside
// a (heavy) row splits it.  While walking, the chunk where such a row begins
// and every chunk fully inside it leave a head piece in workspace slot
// 2*gc + 1, and the chunk where it ends leaves a tail piece in slot 2*gc (gc
// the global chunk).  Once the launch is over, this kernel sums each split
// row's pieces in chunk order and writes C = beta*C + a_scale*sum: the same
// sums, in the same order, that the last-arriving piece would form inside the
// walk, without the acquire-release atomics that ordering needs there.
#include "api_internal.cuh"
#include "launch.cuh"

namespace spmm {

namespace {

constexpr int kFixupInFlight = 16;   // slot loads in flight per lane

// Lane l of warp w tests plan boundary b = 32*w + l (the boundaries of row
// block i sit at blk_base[i] + i + c, c = 0 .. chunks of the block).  The
// first boundary strictly inside a row r -- the one that ends the chunk where
// r begins -- marks r; the warp then sums its marked rows one after another,
// each across its lanes.  One lane per boundary keeps the chain of dependent
// loads of the test to one per warp of 32 boundaries.
__global__ void __launch_bounds__(256) split_row_fixup_kernel(const Problem p) {
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    const int64_t total = (int64_t)p.blk_base[p.TR] + p.TR;
    if (warp * 32 >= total) return;
    const int64_t b64 = warp * 32 + lane;
    bool mine = false;
    int r = 0, ca = 0, cb = 0, base = 0;
    if (b64 < total) {
        const int b = (int)b64;
        int lo = 0, hi = p.TR - 1;   // largest i with blk_base[i] + i <= b
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (p.blk_base[mid] + mid <= b) lo = mid;
            else hi = mid - 1;
        }
        const int i = lo;
        base = p.blk_base[i];
        const int c = b - base - i;
        r = p.bnd_row[b];
        const int row_lo = i * p.RB;
        const int row_hi = min(p.M, row_lo + p.RB);
        // interior boundaries only, inside the row block
        if (c >= 1 && c < p.blk_base[i + 1] - base && r >= row_lo && r < row_hi) {
            const int rs = __ldg(p.rowptr + r);
            if (p.bnd_nnz[b] > rs) {   // not at a row start: r is split here
                const int re = __ldg(p.rowptr + r + 1);
                const int nnz_lo = __ldg(p.rowptr + row_lo);
                // chunks holding r's first item and its end (chunk c spans
                // merge-path items [c*D, (c+1)*D) of the block; boundaries
                // inside a split row are never moved, so these are exact)
                ca = (int)(((int64_t)(r - row_lo) + (rs - nnz_lo)) / p.D);
                cb = (int)(((int64_t)(r - row_lo) + (re - nnz_lo)) / p.D);
                mine = (c == ca + 1);
            }
        }
    }
    const bool scaled = p.a_scale != nullptr;
    uint32_t todo = __ballot_sync(kFull, mine);
    while (todo) {
        const int src = __ffs(todo) - 1;
        todo &= todo - 1;
        const int rr = __shfl_sync(kFull, r, src);
        const int ra = __shfl_sync(kFull, ca, src);
        const int rb = __shfl_sync(kFull, cb, src);
        const int rbase = __shfl_sync(kFull, base, src);
        const float sa = scaled ? __ldg(p.a_scale + rr) : 1.0f;
        float* crow = p.C + (int64_t)rr * p.ldc;
        // the slot loads of a row go out kFixupInFlight at a time; the adds
        // stay in chunk order, so the sum is the same however many are in flight
        for (int v = lane; v < p.N / 4; v += 32) {
            float4 s = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            for (int c0 = ra; c0 <= rb; c0 += kFixupInFlight) {
                float4 t[kFixupInFlight];
#pragma unroll
                for (int u = 0; u < kFixupInFlight; ++u) {
                    const int cc = c0 + u;
                    if (cc <= rb) {
                        const int64_t slot = 2 * (int64_t)(rbase + cc) + (cc == rb ? 0 : 1);
                        t[u] = ld_cg_f4(p.slots + slot * p.N + 4 * v);
                    }
                }
#pragma unroll
                for (int u = 0; u < kFixupInFlight; ++u) {
                    if (c0 + u <= rb) {
                        s.x += t[u].x;
                        s.y += t[u].y;
                        s.z += t[u].z;
                        s.w += t[u].w;
                    }
                }
            }
            if (scaled) {
                s.x *= sa;
                s.y *= sa;
                s.z *= sa;
                s.w *= sa;
            }
            float* d = crow + 4 * v;
            if (p.beta != 0.0f) {
                const float4 old = __ldcg(reinterpret_cast<const float4*>(d));
                s.x = fmaf(p.beta, old.x, s.x);
                s.y = fmaf(p.beta, old.y, s.y);
                s.z = fmaf(p.beta, old.z, s.z);
                s.w = fmaf(p.beta, old.w, s.w);
            }
            st_cs_f4(d, s);
        }
    }
}

}  // namespace

cudaError_t launch_split_row_fixup(const Problem& p, int64_t max_boundaries, cudaStream_t s) {
    if (max_boundaries <= 0) return cudaSuccess;
    const int64_t blocks = (max_boundaries + 255) / 256;   // one lane per boundary
    split_row_fixup_kernel<<<(unsigned)blocks, 256, 0, s>>>(p);
    return cudaGetLastError();
}

}  // namespace spmm
