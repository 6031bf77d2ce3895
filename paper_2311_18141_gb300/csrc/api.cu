// C ABI entry points: argument checks, plans, workspace layout and dispatch.
#include <atomic>
#include <stdlib.h>
#include <string.h>

#include "api_internal.cuh"
#include "launch.cuh"
#include "plan.cuh"

using namespace spmm;

struct spmm_plan_s {
    int device;
    int64_t M, K, nnz, N;
    int32_t TR, TC, RB, D;
    int64_t cap;          // chunk capacity (upper bound of chunks)
    spmm_tuning tuning;
    void* mem;            // device plan arrays
    int32_t* blk_base;
    int32_t* bnd_row;
    int32_t* bnd_nnz;
    uint32_t* ends;       // row-end bitmap over the merge items
    int4* split;          // rows cut by a chunk boundary (see plan_build)
    int32_t* n_split;
    spmm_trace_record* trace;   // caller-owned per-warp trace records (null: off)
    int32_t trace_max;
};

namespace spmm {

int device_sm_count() {
    // cached per device: the hot calls ask for it on every launch
    static std::atomic<int> cache[kMaxDevices];
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 148;
    if (dev >= 0 && dev < kMaxDevices) {
        n = cache[dev].load(std::memory_order_relaxed);
        if (n > 0) return n;
    }
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 148;
    if (dev >= 0 && dev < kMaxDevices) cache[dev].store(n, std::memory_order_relaxed);
    return n;
}

int elem_bytes(int dt) {
    switch (dt) {
        case SPMM_F32: return 4;
        case SPMM_F16: case SPMM_BF16: return 2;
        case SPMM_E4M3: return 1;
        default: return 0;
    }
}

static bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

// Scratch layout of one call: [status 64 B][tile_ctr T][piece_cnt cap*TC] pad
// 256 [slots 2*cap*N floats].
struct Scratch {
    size_t counters_off, counters_bytes, slots_off, total;
};

static Scratch scratch_layout(int32_t TR, int32_t TC, int64_t cap, int64_t N) {
    Scratch s;
    s.counters_off = kStatusBytes;
    s.counters_bytes = 4 * ((size_t)TR * TC + (size_t)cap * TC);
    s.slots_off = (s.counters_off + s.counters_bytes + 255) / 256 * 256;
    s.total = s.slots_off + 4 * (size_t)2 * cap * N;
    s.total = (s.total + 255) / 256 * 256;
    return s;
}

void resolve_tuning(const spmm_tuning* in, spmm_tuning* out) {
    memset(out, 0, sizeof(*out));
    if (in) *out = *in;
    if (out->warps_per_cta < 0 || out->warps_per_cta > 8) out->warps_per_cta = 0;
    if (out->ctas_per_sm < 0) out->ctas_per_sm = 0;
    if (out->tile_order < 0 || out->tile_order > 31) out->tile_order = 0;
    if (out->chunk_items < 0) out->chunk_items = 0;
    if (out->kernel < SPMM_KERNEL_AUTO || out->kernel > SPMM_KERNEL_SPEC)
        out->kernel = SPMM_KERNEL_AUTO;
    if (out->lanes_per_item != 2 && out->lanes_per_item != 4) out->lanes_per_item = 0;
}

// Column-block width for N split in TC blocks of B type `dt`: ceil(N/TC)
// rounded up to whole 16-byte vectors.  0 if the grid leaves a block empty.
int64_t column_block_width(int64_t N, int32_t TC, int dt) {
    const int epv = 16 / elem_bytes(dt);
    int64_t w = (N + TC - 1) / TC;
    w = (w + epv - 1) / epv * epv;
    if (w <= 0 || (int64_t)(TC - 1) * w >= N) return 0;
    return w;
}

// Pick (lanes per nonzero, vectors per lane) covering `nvec` 16-byte vectors.
bool pick_shape(int64_t nvec, int* lpn, int* vpl) {
    if (nvec <= 0) return false;
    if (nvec <= 32) {
        int l = 2;
        while (l < nvec) l <<= 1;
        *lpn = l;
        *vpl = 1;
        return true;
    }
    *lpn = 32;
    if (nvec <= 64) { *vpl = 2; return true; }
    if (nvec <= 128) { *vpl = 4; return true; }
    return false;
}

// Shape of the 32-byte-lane kernel for a column block of `bytes` bytes: lanes
// per item and 32-byte vectors per lane.  Built for blocks of 2 to 32 whole
// 32-byte vectors (64 bytes to 1 KB); others run the staged kernel.
bool pick_wide_shape(int64_t bytes, int* lpn, int* nv) {
    const int64_t nvec = bytes / 32;
    if (bytes % 32 != 0 || nvec < 2 || nvec > 32) return false;
    int l = 2;
    while (l < nvec) l <<= 1;
    *lpn = l;
    *nv = 1;
    return true;
}

// The same with the lanes per item asked for by the tuning (2 or 4): a block
// of 4 or 8 vectors can also be walked by fewer lanes holding 2 or 4 vectors
// each (fewer instructions per byte, more registers per lane).  Other requests
// keep the default shape.
bool pick_shape_lanes(int64_t nvec, int32_t lanes, int* lpn, int* vpl) {
    if (!pick_shape(nvec, lpn, vpl)) return false;
    if ((lanes == 2 || lanes == 4) && *vpl == 1 && (nvec == 4 || nvec == 8) &&
        *lpn == nvec && lanes < nvec && nvec / lanes <= 4) {
        *vpl = (int)(nvec / lanes);
        *lpn = lanes;
    }
    return true;
}

int plan_view(spmm_plan plan, int64_t M, int64_t K, int64_t nnz, int64_t N, int32_t* TR,
              int32_t* TC, int32_t* RB, int32_t* D, int64_t* cap, int32_t** blk_base,
              int32_t** bnd_row, int32_t** bnd_nnz) {
    if (!plan) return SPMM_ERR_INVALID_ARG;
    if (plan->M != M || plan->K != K || plan->nnz != nnz || plan->N != N)
        return SPMM_ERR_PLAN_MISMATCH;
    *TR = plan->TR; *TC = plan->TC; *RB = plan->RB; *D = plan->D; *cap = plan->cap;
    *blk_base = plan->blk_base; *bnd_row = plan->bnd_row; *bnd_nnz = plan->bnd_nnz;
    return SPMM_OK;
}

int plan_shape(spmm_plan plan, int64_t* M, int64_t* K, int64_t* nnz, int64_t* N, int32_t* TR,
               int32_t* TC) {
    if (!plan) return SPMM_ERR_INVALID_ARG;
    if (M) *M = plan->M;
    if (K) *K = plan->K;
    if (nnz) *nnz = plan->nnz;
    if (N) *N = plan->N;
    if (TR) *TR = plan->TR;
    if (TC) *TC = plan->TC;
    return SPMM_OK;
}

}  // namespace spmm

extern "C" {

const char* spmm_status_string(int status) {
    switch (status) {
        case SPMM_OK: return "ok";
        case SPMM_ERR_INVALID_ARG: return "invalid argument";
        case SPMM_ERR_MISALIGNED: return "misaligned pointer, stride or width";
        case SPMM_ERR_UNSUPPORTED: return "unsupported dtype or width";
        case SPMM_ERR_CUDA: return "CUDA runtime error";
        case SPMM_ERR_BAD_CSR: return "malformed CSR";
        case SPMM_ERR_TIMEOUT: return "device wait timed out";
        case SPMM_ERR_WORKSPACE: return "workspace missing or too small";
        case SPMM_ERR_PLAN_MISMATCH: return "plan does not match the call";
        case SPMM_ERR_INTERNAL: return "internal plan check failed";
        default: return "unknown status";
    }
}

int spmm_version(void) { return 100; }

static int check_shape(int64_t M, int64_t K, int64_t nnz, int64_t N, int32_t TR, int32_t TC) {
    const int64_t lim = (int64_t)1 << 30;
    if (M < 0 || K < 0 || nnz < 0 || N < 0) return SPMM_ERR_INVALID_ARG;
    if (M >= lim * 2 - (1 << 20) || K >= lim * 2 - (1 << 20) || nnz >= lim * 2 - 1)
        return SPMM_ERR_INVALID_ARG;
    if (N > (1 << 20)) return SPMM_ERR_INVALID_ARG;
    if (TR < 1 || TR > 65536 || TC < 1 || TC > 4096) return SPMM_ERR_INVALID_ARG;
    if (M > 0 && nnz > 0 && K == 0) return SPMM_ERR_INVALID_ARG;
    return SPMM_OK;
}

int spmm_plan_create(spmm_plan* plan, const int32_t* A_rowptr, int64_t M, int64_t K,
                     int64_t nnz, int64_t N, int32_t tile_rows, int32_t tile_cols,
                     const spmm_tuning* tuning, void* stream) {
    if (!plan) return SPMM_ERR_INVALID_ARG;
    *plan = nullptr;
    int st = check_shape(M, K, nnz, N, tile_rows, tile_cols);
    if (st) return st;
    if (!A_rowptr) return SPMM_ERR_INVALID_ARG;
    spmm_plan_s* p = (spmm_plan_s*)calloc(1, sizeof(spmm_plan_s));
    if (!p) return SPMM_ERR_INVALID_ARG;
    if (cudaGetDevice(&p->device) != cudaSuccess) { free(p); return SPMM_ERR_CUDA; }
    p->M = M; p->K = K; p->nnz = nnz; p->N = N;
    p->TR = tile_rows; p->TC = tile_cols;
    p->RB = (int32_t)((M + tile_rows - 1) / tile_rows);
    if (p->RB < 1) p->RB = 1;
    resolve_tuning(tuning, &p->tuning);
    p->D = p->tuning.chunk_items > 0 ? p->tuning.chunk_items
                                    : plan_default_chunk(M, nnz, tile_cols, device_sm_count(),
                                                         plan_default_groups(N, tile_cols));
    p->tuning.chunk_items = p->D;
    p->cap = plan_chunk_cap(M, nnz, tile_rows, p->D);
    const size_t arrays = plan_array_bytes(tile_rows, p->cap);
    const size_t bytes = arrays + plan_ends_bytes(M + nnz);
    if (cudaMalloc(&p->mem, bytes) != cudaSuccess) { free(p); return SPMM_ERR_CUDA; }
    plan_carve(p->mem, tile_rows, p->cap, &p->blk_base, &p->bnd_row, &p->bnd_nnz, &p->split,
               &p->n_split);
    p->ends = reinterpret_cast<uint32_t*>(static_cast<char*>(p->mem) + arrays);
    cudaError_t e = plan_build_ends(A_rowptr, M, M + nnz, p->ends, (cudaStream_t)stream);
    if (e == cudaSuccess)
        e = plan_build(A_rowptr, M, p->TR, p->RB, p->D, p->cap, p->blk_base, p->bnd_row,
                       p->bnd_nnz, p->split, p->n_split, (cudaStream_t)stream);
    if (e != cudaSuccess) { cudaFree(p->mem); free(p); return SPMM_ERR_CUDA; }
    *plan = p;
    return SPMM_OK;
}

int spmm_plan_destroy(spmm_plan plan) {
    if (!plan) return SPMM_OK;
    cudaDeviceSynchronize();
    cudaFree(plan->mem);
    free(plan);
    return SPMM_OK;
}

int spmm_plan_get_boundaries(spmm_plan plan, int32_t* blk_base, int32_t* bnd_row,
                             int32_t* bnd_nnz) {
    if (!plan) return SPMM_ERR_INVALID_ARG;
    int32_t n = 0;
    if (cudaMemcpy(&n, plan->blk_base + plan->TR, sizeof(n), cudaMemcpyDeviceToHost) != cudaSuccess)
        return SPMM_ERR_CUDA;
    const size_t nb = (size_t)n + plan->TR;
    if ((blk_base && cudaMemcpy(blk_base, plan->blk_base, 4 * ((size_t)plan->TR + 1),
                                cudaMemcpyDeviceToHost) != cudaSuccess) ||
        (bnd_row && cudaMemcpy(bnd_row, plan->bnd_row, 4 * nb, cudaMemcpyDeviceToHost) !=
                        cudaSuccess) ||
        (bnd_nnz && cudaMemcpy(bnd_nnz, plan->bnd_nnz, 4 * nb, cudaMemcpyDeviceToHost) !=
                        cudaSuccess))
        return SPMM_ERR_CUDA;
    return SPMM_OK;
}

int spmm_plan_set_trace(spmm_plan plan, spmm_trace_record* records, int32_t max_records) {
    if (!plan || max_records < 0) return SPMM_ERR_INVALID_ARG;
    plan->trace = max_records > 0 ? records : nullptr;
    plan->trace_max = plan->trace ? max_records : 0;
    return SPMM_OK;
}

int spmm_plan_workspace_size(spmm_plan plan, size_t* bytes) {
    if (!plan || !bytes) return SPMM_ERR_INVALID_ARG;
    *bytes = scratch_layout(plan->TR, plan->TC, plan->cap, plan->N).total;
    return SPMM_OK;
}

int spmm_plan_units(spmm_plan plan, int64_t* chunks, int64_t* units) {
    if (!plan) return SPMM_ERR_INVALID_ARG;
    int32_t n = 0;
    if (cudaMemcpy(&n, plan->blk_base + plan->TR, sizeof(n), cudaMemcpyDeviceToHost) != cudaSuccess)
        return SPMM_ERR_CUDA;
    if (chunks) *chunks = n;
    if (units) *units = (int64_t)n * plan->TC;
    return SPMM_OK;
}

int spmm_csr_workspace_size(int64_t M, int64_t nnz, int64_t N, int32_t tile_rows,
                            int32_t tile_cols, const spmm_tuning* tuning, size_t* bytes) {
    if (!bytes) return SPMM_ERR_INVALID_ARG;
    int st = check_shape(M, 1, nnz, N, tile_rows, tile_cols);
    if (st) return st;
    (void)tuning;  // a call without a plan always uses the default tuning
    const int32_t D = plan_default_chunk(M, nnz, tile_cols, device_sm_count(),
                                         plan_default_groups(N, tile_cols));
    const int64_t cap = plan_chunk_cap(M, nnz, tile_rows, D);
    *bytes = plan_array_bytes(tile_rows, cap) + plan_ends_bytes(M + nnz) +
             scratch_layout(tile_rows, tile_cols, cap, N).total;
    return SPMM_OK;
}

int spmm_csr(const int32_t* A_rowptr, const int32_t* A_colind, const void* A_vals,
             int32_t a_dtype, const float* A_row_scale, const void* B, int32_t b_dtype,
             const float* B_row_scale, int64_t ldb, float* C, int64_t ldc, int64_t M,
             int64_t K, int64_t N, int64_t nnz, int32_t tile_rows, int32_t tile_cols,
             float beta, spmm_plan plan, void* workspace, size_t workspace_bytes,
             void* stream) {
    if (plan) {
        if (tile_rows == 0) tile_rows = plan->TR;
        if (tile_cols == 0) tile_cols = plan->TC;
    }
    int st = check_shape(M, K, nnz, N, tile_rows, tile_cols);
    if (st) return st;
    if (elem_bytes(a_dtype) == 0 || elem_bytes(b_dtype) == 0) return SPMM_ERR_UNSUPPORTED;
    if (M == 0 || N == 0) return SPMM_OK;
    if (!A_rowptr || !C || (nnz > 0 && (!A_colind || !A_vals || !B))) return SPMM_ERR_INVALID_ARG;
    if (ldb < N || ldc < N) return SPMM_ERR_INVALID_ARG;
    // the kernels keep row strides in bytes as 32-bit values
    if (ldb * elem_bytes(b_dtype) >= ((int64_t)1 << 32) || ldc * 4 >= ((int64_t)1 << 32))
        return SPMM_ERR_INVALID_ARG;
    const int eb = elem_bytes(b_dtype);
    const int epv = 16 / eb;
    if (N % epv != 0 || (ldb * eb) % 16 != 0 || (ldc * 4) % 16 != 0 || !aligned16(C) ||
        (B && !aligned16(B)))
        return SPMM_ERR_MISALIGNED;
    const int64_t W = column_block_width(N, tile_cols, b_dtype);
    if (W == 0) return SPMM_ERR_INVALID_ARG;
    // The 32-byte-lane kernel needs every B row segment and C row segment on
    // 32-byte boundaries; otherwise the 16-byte staged kernel runs.
    const bool wide_ok = (W * eb) % 32 == 0 && (N * eb) % 32 == 0 && (ldb * eb) % 32 == 0 &&
                         (ldc * 4) % 32 == 0 && ((uintptr_t)C & 31u) == 0 &&
                         (!B || ((uintptr_t)B & 31u) == 0);
    int lpn = 0, vpl = 0;
    if (!pick_shape(W / epv, &lpn, &vpl)) return SPMM_ERR_UNSUPPORTED;
    const int32_t lanes_req = plan ? plan->tuning.lanes_per_item : 0;
    pick_shape_lanes(W / epv, lanes_req, &lpn, &vpl);
    int wlpn = 0, wnv = 0;
    const bool wide_shape = wide_ok && pick_wide_shape(W * eb, &wlpn, &wnv);
    if (!workspace || ((uintptr_t)workspace & 255u)) return SPMM_ERR_WORKSPACE;

    cudaStream_t s = (cudaStream_t)stream;
    char* ws = static_cast<char*>(workspace);
    int32_t TR = tile_rows, TC = tile_cols, RB, D;
    int64_t cap;
    int32_t *blk_base, *bnd_row, *bnd_nnz, *n_split;
    int4* split;
    uint32_t* ends;
    spmm_tuning tun;
    if (plan) {
        if (plan->M != M || plan->nnz != nnz || plan->N != N || plan->TR != TR ||
            plan->TC != TC || plan->K != K)
            return SPMM_ERR_PLAN_MISMATCH;
        RB = plan->RB; D = plan->D; cap = plan->cap;
        blk_base = plan->blk_base; bnd_row = plan->bnd_row; bnd_nnz = plan->bnd_nnz;
        ends = plan->ends;
        split = plan->split; n_split = plan->n_split;
        tun = plan->tuning;
    } else {
        resolve_tuning(nullptr, &tun);
        RB = (int32_t)((M + TR - 1) / TR);
        D = plan_default_chunk(M, nnz, TC, device_sm_count(), plan_default_groups(N, TC));
        cap = plan_chunk_cap(M, nnz, TR, D);
        // layout [scratch: status, counters, slots][plan arrays]: the status
        // word stays at the start of the caller's workspace
        const size_t pa = plan_array_bytes(TR, cap);
        const size_t pb = pa + plan_ends_bytes(M + nnz);
        const Scratch sc = scratch_layout(TR, TC, cap, N);
        if (workspace_bytes < pb + sc.total) return SPMM_ERR_WORKSPACE;
        plan_carve(ws + sc.total, TR, cap, &blk_base, &bnd_row, &bnd_nnz, &split, &n_split);
        ends = reinterpret_cast<uint32_t*>(ws + sc.total + pa);
        if (plan_build_ends(A_rowptr, M, M + nnz, ends, s) != cudaSuccess ||
            plan_build(A_rowptr, M, TR, RB, D, cap, blk_base, bnd_row, bnd_nnz, split, n_split,
                       s) != cudaSuccess)
            return SPMM_ERR_CUDA;
        workspace_bytes -= pb;
    }
    const Scratch sc = scratch_layout(TR, TC, cap, N);
    if (workspace_bytes < sc.total) return SPMM_ERR_WORKSPACE;

    Problem p;
    memset(&p, 0, sizeof(p));
    p.rowptr = A_rowptr; p.colind = A_colind; p.vals = A_vals; p.a_scale = A_row_scale;
    p.B = B; p.b_scale = B_row_scale; p.C = C; p.ldb = ldb; p.ldc = ldc;
    p.M = (int32_t)M; p.N = (int32_t)N; p.a_dtype = a_dtype; p.beta = beta;
    p.TR = TR; p.TC = TC; p.RB = RB; p.W = (int32_t)W; p.D = D;
    p.blk_base = blk_base; p.bnd_row = bnd_row; p.bnd_nnz = bnd_nnz; p.ends = ends;
    p.split = split; p.n_split = n_split;
    p.status = reinterpret_cast<int32_t*>(ws);
    p.tile_ctr = reinterpret_cast<int32_t*>(ws + sc.counters_off);
    p.piece_cnt = p.tile_ctr + (size_t)TR * TC;
    p.slots = reinterpret_cast<float*>(ws + sc.slots_off);
    if (plan) {
        p.trace = plan->trace;
        p.trace_max = plan->trace_max;
    }
    if (cudaMemsetAsync(ws + sc.counters_off, 0, sc.counters_bytes, s) != cudaSuccess)
        return SPMM_ERR_CUDA;
    LaunchOpts o;
    o.warps_per_cta = tun.warps_per_cta;
    o.ctas_per_sm = tun.ctas_per_sm;
    o.flags = tun.tile_order;
    o.units = cap * TC;
    if (tun.kernel == SPMM_KERNEL_WIDE && !wide_shape) return SPMM_ERR_MISALIGNED;
    cudaError_t e;
    if (tun.kernel == SPMM_KERNEL_WIDE && wide_shape) {
        const WideLaunchFn fn = wide_launcher(a_dtype, b_dtype);
        if (!fn) return SPMM_ERR_UNSUPPORTED;
        e = fn(wlpn, wnv, p, o, s);
    } else if (tun.kernel == SPMM_KERNEL_SPEC) {
        const SpecLaunchFn fn = spec_launcher(a_dtype, b_dtype);
        if (!fn || vpl != 1 || lpn < 8) return SPMM_ERR_UNSUPPORTED;
        e = fn(lpn, p, o, s);
        // like the staged kernel, it leaves split rows in the slots
        if (e == cudaSuccess) e = launch_split_row_fixup(p, cap + TR, s);
    } else {
        const LaunchFn fn = spmm_launcher(a_dtype, b_dtype);
        if (!fn) return SPMM_ERR_UNSUPPORTED;
        e = fn(lpn, vpl, p, o, s);
        // the staged kernel leaves split rows in the slots
        if (e == cudaSuccess) e = launch_split_row_fixup(p, cap + TR, s);
    }
    return e == cudaSuccess ? SPMM_OK : SPMM_ERR_CUDA;
}

int spmm_get_device_status(void* workspace, int32_t* status, void* stream) {
    if (!workspace || !status) return SPMM_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    int32_t h[2] = {0, 0};
    if (cudaMemcpyAsync(h, workspace, sizeof(h), cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return SPMM_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return SPMM_ERR_CUDA;
    if (cudaMemsetAsync(workspace, 0, sizeof(h), s) != cudaSuccess) return SPMM_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return SPMM_ERR_CUDA;
    if (h[0] != 0) *status = h[0];
    else if (h[1] != 0) *status = SPMM_ERR_INTERNAL;
    else *status = SPMM_OK;
    return SPMM_OK;
}

}  // extern "C"
