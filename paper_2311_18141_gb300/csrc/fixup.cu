// Split rows of the staged product, summed after the persistent launch.
//
// The plan cuts a row block's merge path into chunks; a chunk boundary inside
// a (heavy) row splits it, and the plan lists every such row once.  While
// walking, the chunk where such a row begins and every chunk fully inside it
// leave a head piece in workspace slot 2*gc + 1, and the chunk where it ends
// leaves a tail piece in slot 2*gc (gc the global chunk).  Once the launch is
// over, this kernel sums each listed row's pieces in chunk order and writes
// C = beta*C + a_scale*sum: the same sums, in the same order, that the
// last-arriving piece would form inside the walk, without the acquire-release
// atomics that ordering needs there.
#include "api_internal.cuh"
#include "batch_kernel.cuh"
#include "launch.cuh"

namespace spmm {

namespace {

constexpr int kFixupInFlight = 16;   // slot loads in flight per thread
constexpr int kFixupThreads = 256;
constexpr int kFixupMaxBlocks = 2048;

// Split row k of the plan's list, 16-byte column vector v: the row's pieces
// are its head pieces in slots 2*cc + 1 of chunks cc = first .. last-1 and its
// tail piece in slot 2*last; their sum, in chunk order, is scaled and written
// to C.
__device__ __forceinline__ void fixup_row_vector(const Problem& p, const float* slots, int k,
                                                 int v) {
    const int4 ent = __ldg(p.split + k);
    const int r = ent.x, first = ent.y, last = ent.z;
    // the slot loads go out kFixupInFlight at a time; the adds stay in chunk
    // order, so the sum is the same however many are in flight
    float4 s = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    for (int c0 = first; c0 <= last; c0 += kFixupInFlight) {
        float4 t[kFixupInFlight];
#pragma unroll
        for (int u = 0; u < kFixupInFlight; ++u) {
            const int cc = c0 + u;
            if (cc <= last) {
                const int64_t slot = 2 * (int64_t)cc + (cc == last ? 0 : 1);
                t[u] = ld_cg_f4(slots + slot * p.N + 4 * v);
            }
        }
#pragma unroll
        for (int u = 0; u < kFixupInFlight; ++u) {
            if (c0 + u <= last) {
                s.x += t[u].x;
                s.y += t[u].y;
                s.z += t[u].z;
                s.w += t[u].w;
            }
        }
    }
    if (p.a_scale != nullptr) {
        const float sa = __ldg(p.a_scale + r);
        s.x *= sa;
        s.y *= sa;
        s.z *= sa;
        s.w *= sa;
    }
    float* d = p.C + (int64_t)r * p.ldc + 4 * v;
    if (p.beta != 0.0f) {
        const float4 old = __ldcg(reinterpret_cast<const float4*>(d));
        s.x = fmaf(p.beta, old.x, s.x);
        s.y = fmaf(p.beta, old.y, s.y);
        s.z = fmaf(p.beta, old.z, s.z);
        s.w = fmaf(p.beta, old.w, s.w);
    }
    st_cs_f4(d, s);
}

// One thread per (split row, 16-byte column vector) of one product.
__global__ void __launch_bounds__(kFixupThreads) split_row_fixup_kernel(const Problem p) {
    const int n = *p.n_split;
    const int V4 = p.N / 4;
    const int64_t items = (int64_t)n * V4;
    for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < items;
         w += (int64_t)gridDim.x * blockDim.x) {
        const int k = (int)(w / V4);
        fixup_row_vector(p, p.slots, k, (int)(w - (int64_t)k * V4));
    }
}

// The products of a batch: blockIdx.y is the product, and the gridDim.x
// blocks of a product share out its (split row, vector) pairs.  A product's
// slots lie at ws + slot_off.
__global__ void __launch_bounds__(kFixupThreads)
split_row_fixup_batched_kernel(const BatchEntry* __restrict__ table, char* ws) {
    const BatchEntry& e = table[blockIdx.y];
    const Problem& p = e.p;
    const int n = *p.n_split;
    const int V4 = p.N / 4;
    const int64_t items = (int64_t)n * V4;
    const float* slots = reinterpret_cast<const float*>(ws + e.slot_off);
    for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < items;
         w += (int64_t)gridDim.x * blockDim.x) {
        const int k = (int)(w / V4);
        fixup_row_vector(p, slots, k, (int)(w - (int64_t)k * V4));
    }
}

}  // namespace

cudaError_t launch_split_row_fixup(const Problem& p, int64_t max_rows, cudaStream_t s) {
    if (max_rows <= 0 || p.N < 4) return cudaSuccess;
    // grid-stride over the rows the plan listed (at most max_rows of them)
    const int64_t items = max_rows * (p.N / 4);
    int64_t blocks = (items + kFixupThreads - 1) / kFixupThreads;
    if (blocks > kFixupMaxBlocks) blocks = kFixupMaxBlocks;
    split_row_fixup_kernel<<<(unsigned)blocks, kFixupThreads, 0, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_split_row_fixup_batched(const BatchEntry* table, int count, char* ws,
                                           int64_t max_items, cudaStream_t s) {
    if (count <= 0 || max_items <= 0) return cudaSuccess;
    // enough blocks per product for its largest possible list, at most 64
    int64_t bx = (max_items + kFixupThreads - 1) / kFixupThreads;
    if (bx > 64) bx = 64;
    // gridDim.y holds at most 65535 products per launch
    for (int q0 = 0; q0 < count; q0 += 65535) {
        const int nq = count - q0 < 65535 ? count - q0 : 65535;
        split_row_fixup_batched_kernel<<<dim3((unsigned)bx, (unsigned)nq), kFixupThreads, 0, s>>>(
            table + q0, ws);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace spmm
