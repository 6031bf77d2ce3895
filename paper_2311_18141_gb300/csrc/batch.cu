// Batched SpMM host side: per-problem plans, the device descriptor table, the
// per-call workspace, CUDA-graph replay and the shape autotuner.
#include <algorithm>
#include <numeric>
#include <string.h>
#include <vector>

#include "api_internal.cuh"
#include "batch_kernel.cuh"
#include "launch.cuh"
#include "plan.cuh"

using namespace spmm;

namespace {

constexpr int32_t kBatchMinChunk = 256;   // smallest sub-chunk the autotuner may choose
constexpr int32_t kBatchMaxTC = 2;        // widest column split the autotuner may choose

size_t up256(size_t x) { return (x + 255) / 256 * 256; }

// item_base[q+1] = item_base[q] + units(q) * TC(q), a unit being G = 32/lpn
// sub-chunks of the plan.
__global__ void item_base_kernel(const BatchEntry* table, int count, int64_t* item_base) {
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    int64_t run = 0;
    item_base[0] = 0;
    for (int q = 0; q < count; ++q) {
        const Problem& p = table[q].p;
        const int G = 32 / table[q].lpn;
        run += (int64_t)((p.blk_base[p.TR] + G - 1) / G) * p.TC;
        item_base[q + 1] = run;
    }
}

}  // namespace

struct spmm_batch_s {
    int device = 0;
    int32_t count = 0, a_dtype = 0, b_dtype = 0;
    std::vector<spmm_problem> probs;     // in execution order (largest work first)
    std::vector<int32_t> user_index;     // execution slot -> caller's index
    std::vector<int32_t> TR, TC, D, lpn;
    std::vector<int64_t> cap;
    void* plan_mem = nullptr;
    size_t plan_bytes = 0;
    BatchEntry* d_table = nullptr;
    int64_t* d_item_base = nullptr;
    std::vector<BatchEntry> h_table;
    size_t ws_needed = 0;                // for the current shapes
    size_t ws_bound = 0;                 // for any shapes the autotuner may pick
    int64_t max_items = 0;               // upper bound of work items
    int64_t fixup_items = 0;             // bound of any product's (split row, vector) pairs
    // device table order: products grouped by lane shape (one persistent launch
    // per group), each group in execution order; exec[k] = index into probs
    std::vector<int32_t> exec;
    struct Group {
        int32_t start, count, lpn;
        int64_t max_items;
    };
    std::vector<Group> groups;
    int32_t ctas_per_sm = 0;             // 0: occupancy limit (autotuned)
    cudaGraphExec_t graph = nullptr;
    const void* graph_ws = nullptr;
    cudaStream_t graph_stream = nullptr;
};

namespace {

int64_t problem_cap(const spmm_problem& q, int32_t TR, int32_t D) {
    return plan_chunk_cap(q.M, q.nnz, TR, D);
}

// Scratch bytes of one problem: piece counters (cap*TC ints) and slots
// (2*cap*N floats), each 256-byte padded.
size_t problem_scratch(const spmm_problem& q, int64_t cap, int32_t TC) {
    return up256(4 * (size_t)cap * TC) + up256(4 * (size_t)2 * cap * q.N);
}

// Lanes per nonzero for a column block of B type `dt` with N split TC ways;
// 0 if the block is wider than one warp covers with one vector per lane.
int32_t shape_lpn(int64_t N, int32_t TC, int dt) {
    const int64_t W = column_block_width(N, TC, dt);
    if (W == 0) return 0;
    const int epv = 16 / elem_bytes(dt);
    int lpn = 0, vpl = 0;
    if (!pick_shape(W / epv, &lpn, &vpl) || vpl != 1) return 0;
    return lpn;
}

// (Re)build every plan and the descriptor table for the current shapes.
int batch_build(spmm_batch b, cudaStream_t s) {
    const int n = b->count;
    b->cap.assign(n, 0);
    b->lpn.assign(n, 0);
    size_t plan_total = 0, ws = kStatusBytes + 256, ws_bound = kStatusBytes + 256;
    std::vector<size_t> plan_off(n);
    std::vector<int64_t> piece_off(n), slot_off(n);
    b->max_items = 0;
    b->fixup_items = 0;
    for (int q = 0; q < n; ++q) {
        const spmm_problem& P = b->probs[q];
        b->lpn[q] = shape_lpn(P.N, b->TC[q], b->b_dtype);
        if (b->lpn[q] == 0) return SPMM_ERR_UNSUPPORTED;
        b->cap[q] = problem_cap(P, b->TR[q], b->D[q]);
        plan_off[q] = plan_total;
        plan_total += plan_array_bytes(b->TR[q], b->cap[q]) + plan_ends_bytes(P.M + P.nnz);
        const size_t sc = problem_scratch(P, b->cap[q], b->TC[q]);
        piece_off[q] = (int64_t)ws;
        slot_off[q] = (int64_t)(ws + up256(4 * (size_t)b->cap[q] * b->TC[q]));
        ws += sc;
        const int32_t tr_any = std::max<int32_t>(b->TR[q], 16);
        ws_bound += problem_scratch(P, problem_cap(P, tr_any, kBatchMinChunk), kBatchMaxTC);
        b->max_items += b->cap[q] * b->TC[q];
        // a product lists at most one split row per plan boundary
        b->fixup_items =
            std::max<int64_t>(b->fixup_items, (b->cap[q] + b->TR[q]) * (int64_t)(P.N / 4));
    }
    b->ws_needed = ws;
    b->ws_bound = std::max(ws_bound, ws);
    if (plan_total > b->plan_bytes) {
        if (b->plan_mem) cudaFree(b->plan_mem);
        b->plan_mem = nullptr;
        b->plan_bytes = 0;
        if (cudaMalloc(&b->plan_mem, plan_total) != cudaSuccess) return SPMM_ERR_CUDA;
        b->plan_bytes = plan_total;
    }
    // group the device table by lane shape, widest items first; the stable
    // sort keeps the execution order inside a group
    b->exec.resize(n);
    std::iota(b->exec.begin(), b->exec.end(), 0);
    std::stable_sort(b->exec.begin(), b->exec.end(),
                     [&](int x, int y) { return b->lpn[x] > b->lpn[y]; });
    b->groups.clear();
    for (int k = 0; k < n; ++k) {
        const int q = b->exec[k];
        if (b->groups.empty() || b->groups.back().lpn != b->lpn[q])
            b->groups.push_back({k, 0, b->lpn[q], 0});
        b->groups.back().count += 1;
        b->groups.back().max_items += b->cap[q] * b->TC[q];
    }
    b->h_table.assign(n, BatchEntry{});
    for (int k = 0; k < n; ++k) {
        const int q = b->exec[k];
        const spmm_problem& P = b->probs[q];
        BatchEntry& e = b->h_table[k];
        memset(&e, 0, sizeof(e));
        Problem& p = e.p;
        int32_t *blk_base, *bnd_row, *bnd_nnz, *n_split;
        int4* split;
        plan_carve(static_cast<char*>(b->plan_mem) + plan_off[q], b->TR[q], b->cap[q], &blk_base,
                   &bnd_row, &bnd_nnz, &split, &n_split);
        const int32_t RB = (int32_t)std::max<int64_t>(1, (P.M + b->TR[q] - 1) / b->TR[q]);
        uint32_t* ends = reinterpret_cast<uint32_t*>(static_cast<char*>(b->plan_mem) + plan_off[q] +
                                                     plan_array_bytes(b->TR[q], b->cap[q]));
        if (plan_build_ends(P.rowptr, P.M, P.M + P.nnz, ends, s) != cudaSuccess ||
            plan_build(P.rowptr, P.M, b->TR[q], RB, b->D[q], b->cap[q], blk_base, bnd_row, bnd_nnz,
                       split, n_split, s) != cudaSuccess)
            return SPMM_ERR_CUDA;
        p.rowptr = P.rowptr; p.colind = P.colind; p.vals = P.vals; p.a_scale = P.a_scale;
        p.B = P.B; p.b_scale = P.b_scale; p.C = P.C; p.ldb = P.ldb; p.ldc = P.ldc;
        p.M = (int32_t)P.M; p.N = (int32_t)P.N; p.a_dtype = b->a_dtype; p.beta = P.beta;
        p.TR = b->TR[q]; p.TC = b->TC[q]; p.RB = RB;
        p.W = (int32_t)column_block_width(P.N, b->TC[q], b->b_dtype); p.D = b->D[q];
        p.blk_base = blk_base; p.bnd_row = bnd_row; p.bnd_nnz = bnd_nnz; p.ends = ends;
        p.split = split; p.n_split = n_split;
        e.piece_off = piece_off[q];
        e.slot_off = slot_off[q];
        e.lpn = b->lpn[q];
    }
    if (!b->d_table) {
        if (cudaMalloc(&b->d_table, sizeof(BatchEntry) * n) != cudaSuccess) return SPMM_ERR_CUDA;
        if (cudaMalloc(&b->d_item_base, sizeof(int64_t) * (n + 1)) != cudaSuccess)
            return SPMM_ERR_CUDA;
    }
    if (cudaMemcpyAsync(b->d_table, b->h_table.data(), sizeof(BatchEntry) * n,
                        cudaMemcpyHostToDevice, s) != cudaSuccess)
        return SPMM_ERR_CUDA;
    item_base_kernel<<<1, 32, 0, s>>>(b->d_table, n, b->d_item_base);
    if (cudaGetLastError() != cudaSuccess) return SPMM_ERR_CUDA;
    // the table upload reads pageable host memory: finish it before h_table changes
    if (cudaStreamSynchronize(s) != cudaSuccess) return SPMM_ERR_CUDA;
    if (b->graph) {
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
        b->graph_ws = nullptr;
    }
    return SPMM_OK;
}

int check_problem(const spmm_problem& q, int b_dtype) {
    if (q.M <= 0 || q.K <= 0 || q.N <= 0 || q.nnz < 0) return SPMM_ERR_INVALID_ARG;
    if (q.M >= (1ll << 31) - (1 << 20) || q.nnz >= (1ll << 31) - 1) return SPMM_ERR_INVALID_ARG;
    if (!q.rowptr || !q.C || (q.nnz > 0 && (!q.colind || !q.vals || !q.B)))
        return SPMM_ERR_INVALID_ARG;
    if (q.ldb < q.N || q.ldc < q.N) return SPMM_ERR_INVALID_ARG;
    if (q.ldb * elem_bytes(b_dtype) >= ((int64_t)1 << 32) || q.ldc * 4 >= ((int64_t)1 << 32))
        return SPMM_ERR_INVALID_ARG;
    const int eb = elem_bytes(b_dtype);
    const int epv = 16 / eb;
    if (q.N % epv != 0 || (q.ldb * eb) % 16 != 0 || (q.ldc * 4) % 16 != 0 ||
        ((uintptr_t)q.C & 15u) || ((uintptr_t)q.B & 15u))
        return SPMM_ERR_MISALIGNED;
    if (q.tile_rows < 0 || q.tile_rows > 65536 || q.tile_cols < 0 || q.chunk_items < 0)
        return SPMM_ERR_INVALID_ARG;
    return SPMM_OK;
}

}  // namespace

extern "C" {

int spmm_batch_create(spmm_batch* out, const spmm_problem* problems, int32_t count,
                      int32_t a_dtype, int32_t b_dtype, void* stream) {
    if (!out || !problems || count <= 0) return SPMM_ERR_INVALID_ARG;
    *out = nullptr;
    if (elem_bytes(a_dtype) == 0 || elem_bytes(b_dtype) == 0) return SPMM_ERR_UNSUPPORTED;
    for (int q = 0; q < count; ++q) {
        const int st = check_problem(problems[q], b_dtype);
        if (st) return st;
    }
    spmm_batch b = new spmm_batch_s();
    if (cudaGetDevice(&b->device) != cudaSuccess) { delete b; return SPMM_ERR_CUDA; }
    b->count = count;
    b->a_dtype = a_dtype;
    b->b_dtype = b_dtype;
    // execution order: by width (so the warps of an SM mostly run one kernel
    // shape at a time), each width by decreasing work (nonzeros x width, plus
    // rows), ties by index
    b->user_index.resize(count);
    std::iota(b->user_index.begin(), b->user_index.end(), 0);
    auto work = [&](int q) {
        return (double)(problems[q].nnz + problems[q].M) * (double)problems[q].N;
    };
    std::stable_sort(b->user_index.begin(), b->user_index.end(), [&](int x, int y) {
        if (problems[x].N != problems[y].N) return problems[x].N > problems[y].N;
        return work(x) > work(y);
    });
    b->probs.resize(count);
    b->TR.resize(count);
    b->TC.resize(count);
    b->D.resize(count);
    for (int k = 0; k < count; ++k) {
        const spmm_problem& P = problems[b->user_index[k]];
        b->probs[k] = P;
        b->TR[k] = P.tile_rows > 0 ? P.tile_rows : 1;
        int32_t tc = P.tile_cols > 0 ? P.tile_cols : 1;
        while (shape_lpn(P.N, tc, b_dtype) == 0 && tc < 4096) tc *= 2;   // fit one warp
        b->TC[k] = tc;
        // default sub-chunk: a unit (32/lpn sub-chunks) of about 4096 items
        const int32_t lpn = shape_lpn(P.N, tc, b_dtype);
        const int32_t groups = lpn > 0 ? 32 / lpn : 1;
        b->D[k] = P.chunk_items > 0 ? P.chunk_items
                                    : std::min<int32_t>(2048, std::max<int32_t>(kBatchMinChunk,
                                                                               4096 / groups));
    }
    const int st = batch_build(b, (cudaStream_t)stream);
    if (st) {
        spmm_batch_destroy(b);
        return st;
    }
    *out = b;
    return SPMM_OK;
}

int spmm_batch_destroy(spmm_batch b) {
    if (!b) return SPMM_OK;
    cudaDeviceSynchronize();
    if (b->graph) cudaGraphExecDestroy(b->graph);
    if (b->plan_mem) cudaFree(b->plan_mem);
    if (b->d_table) cudaFree(b->d_table);
    if (b->d_item_base) cudaFree(b->d_item_base);
    delete b;
    return SPMM_OK;
}

int spmm_batch_workspace_size(spmm_batch b, size_t* bytes) {
    if (!b || !bytes) return SPMM_ERR_INVALID_ARG;
    *bytes = b->ws_bound;
    return SPMM_OK;
}

int spmm_batch_set_shapes(spmm_batch b, const int32_t* tile_rows, const int32_t* tile_cols,
                          const int32_t* chunk_items, void* stream) {
    if (!b) return SPMM_ERR_INVALID_ARG;
    for (int k = 0; k < b->count; ++k) {
        const int u = b->user_index[k];
        if (tile_rows && tile_rows[u] > 0) b->TR[k] = std::min(tile_rows[u], 65536);
        if (tile_cols && tile_cols[u] > 0) {
            if (shape_lpn(b->probs[k].N, tile_cols[u], b->b_dtype) == 0)
                return SPMM_ERR_UNSUPPORTED;
            b->TC[k] = tile_cols[u];
        }
        if (chunk_items && chunk_items[u] > 0) b->D[k] = chunk_items[u];
    }
    return batch_build(b, (cudaStream_t)stream);
}

int spmm_batch_get_shapes(spmm_batch b, int32_t* tile_rows, int32_t* tile_cols,
                          int32_t* chunk_items) {
    if (!b) return SPMM_ERR_INVALID_ARG;
    for (int k = 0; k < b->count; ++k) {
        const int u = b->user_index[k];
        if (tile_rows) tile_rows[u] = b->TR[k];
        if (tile_cols) tile_cols[u] = b->TC[k];
        if (chunk_items) chunk_items[u] = b->D[k];
    }
    return SPMM_OK;
}

static int batch_enqueue(spmm_batch b, void* workspace, size_t bytes, cudaStream_t s) {
    if (!workspace || ((uintptr_t)workspace & 255u)) return SPMM_ERR_WORKSPACE;
    if (bytes < b->ws_needed) return SPMM_ERR_WORKSPACE;
    char* ws = static_cast<char*>(workspace);
    // reset the global counter and every problem's piece counters (slots need no reset)
    if (cudaMemsetAsync(ws + kStatusBytes, 0, b->ws_needed - kStatusBytes, s) != cudaSuccess)
        return SPMM_ERR_CUDA;
    const BatchLaunchFn fn = batched_launcher(b->a_dtype, b->b_dtype);
    if (!fn) return SPMM_ERR_UNSUPPORTED;
    // one persistent launch per lane shape, each with its own work counter
    int* counters = reinterpret_cast<int*>(ws + kStatusBytes);
    for (size_t g = 0; g < b->groups.size(); ++g) {
        const spmm_batch_s::Group& G = b->groups[g];
        const cudaError_t e = fn(G.lpn, b->d_table + G.start, b->d_item_base + G.start, G.count,
                                 ws, counters + g, G.max_items, b->ctas_per_sm, s);
        if (e != cudaSuccess) return SPMM_ERR_CUDA;
    }
    // the rows that chunk boundaries cut, summed from their slots
    if (launch_split_row_fixup_batched(b->d_table, (int)b->count, ws, b->fixup_items, s) !=
        cudaSuccess)
        return SPMM_ERR_CUDA;
    return SPMM_OK;
}

int spmm_csr_batched(spmm_batch b, void* workspace, size_t workspace_bytes, void* stream) {
    if (!b) return SPMM_ERR_INVALID_ARG;
    return batch_enqueue(b, workspace, workspace_bytes, (cudaStream_t)stream);
}

int spmm_batch_graph_launch(spmm_batch b, void* workspace, size_t workspace_bytes, void* stream) {
    if (!b) return SPMM_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (!workspace || workspace_bytes < b->ws_needed) return SPMM_ERR_WORKSPACE;
    if (!b->graph || b->graph_ws != workspace) {
        if (b->graph) {
            cudaGraphExecDestroy(b->graph);
            b->graph = nullptr;
        }
        cudaStream_t cap = s;
        bool own = false;
        if (!cap) {   // the legacy default stream cannot be captured
            if (cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess)
                return SPMM_ERR_CUDA;
            own = true;
        }
        cudaGraph_t g = nullptr;
        if (cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
            if (own) cudaStreamDestroy(cap);
            return SPMM_ERR_CUDA;
        }
        const int st = batch_enqueue(b, workspace, workspace_bytes, cap);
        const cudaError_t e = cudaStreamEndCapture(cap, &g);
        if (own) cudaStreamDestroy(cap);
        if (st != SPMM_OK || e != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            return st != SPMM_OK ? st : SPMM_ERR_CUDA;
        }
        const cudaError_t ie = cudaGraphInstantiate(&b->graph, g, 0);
        cudaGraphDestroy(g);
        if (ie != cudaSuccess) {
            b->graph = nullptr;
            return SPMM_ERR_CUDA;
        }
        b->graph_ws = workspace;
    }
    return cudaGraphLaunch(b->graph, s) == cudaSuccess ? SPMM_OK : SPMM_ERR_CUDA;
}

}  // extern "C"

namespace {

// Average milliseconds of `reps` batched launches on `s` (after one warm-up).
int time_batch(spmm_batch b, void* ws, size_t bytes, int reps, cudaStream_t s, float* ms) {
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return SPMM_ERR_CUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); return SPMM_ERR_CUDA; }
    int st = batch_enqueue(b, ws, bytes, s);
    if (st == SPMM_OK && cudaEventRecord(e0, s) != cudaSuccess) st = SPMM_ERR_CUDA;
    for (int r = 0; st == SPMM_OK && r < reps; ++r) st = batch_enqueue(b, ws, bytes, s);
    if (st == SPMM_OK && cudaEventRecord(e1, s) != cudaSuccess) st = SPMM_ERR_CUDA;
    if (st == SPMM_OK && cudaEventSynchronize(e1) != cudaSuccess) st = SPMM_ERR_CUDA;
    float t = 0.0f;
    if (st == SPMM_OK && cudaEventElapsedTime(&t, e0, e1) != cudaSuccess) st = SPMM_ERR_CUDA;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st == SPMM_OK) *ms = t / (float)reps;
    return st;
}

}  // namespace

extern "C" int spmm_batch_autotune(spmm_batch b, void* workspace, size_t workspace_bytes,
                                   int32_t reps, void* stream, float* best_ms) {
    if (!b) return SPMM_ERR_INVALID_ARG;
    if (!workspace || workspace_bytes < b->ws_bound) return SPMM_ERR_WORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    if (reps < 1) reps = 3;
    // size classes: (N, rows below 10k / 50k / above)
    auto bucket = [](int64_t M) { return M < 10000 ? 0 : (M < 50000 ? 1 : 2); };
    std::vector<std::pair<int64_t, int>> keys;
    std::vector<int> cls(b->count);
    for (int k = 0; k < b->count; ++k) {
        const std::pair<int64_t, int> key(b->probs[k].N, bucket(b->probs[k].M));
        auto it = std::find(keys.begin(), keys.end(), key);
        cls[k] = (int)(it - keys.begin());
        if (it == keys.end()) keys.push_back(key);
    }
    float best = 0.0f;
    int st = time_batch(b, workspace, workspace_bytes, reps, s, &best);
    if (st) return st;
    const int32_t tr_c[] = {1, 4};
    const int32_t tc_c[] = {1, 2};
    const int32_t d_c[] = {kBatchMinChunk, 512, 1024, 2048};
    for (int c = 0; c < (int)keys.size(); ++c) {
        int32_t bt = -1, bc = -1, bd = -1;
        for (int k = 0; k < b->count; ++k)
            if (cls[k] == c) { bt = b->TR[k]; bc = b->TC[k]; bd = b->D[k]; break; }
        for (int32_t tr : tr_c)
            for (int32_t tc : tc_c)
                for (int32_t d : d_c) {
                    if (tr == bt && tc == bc && d == bd) continue;
                    bool ok = true;
                    for (int k = 0; k < b->count; ++k)
                        if (cls[k] == c && shape_lpn(b->probs[k].N, tc, b->b_dtype) == 0) ok = false;
                    if (!ok) continue;
                    for (int k = 0; k < b->count; ++k)
                        if (cls[k] == c) { b->TR[k] = tr; b->TC[k] = tc; b->D[k] = d; }
                    st = batch_build(b, s);
                    float ms = 0.0f;
                    if (st == SPMM_OK) st = time_batch(b, workspace, workspace_bytes, reps, s, &ms);
                    if (st) return st;
                    if (ms < best) {
                        best = ms;
                        bt = tr; bc = tc; bd = d;
                    }
                }
        for (int k = 0; k < b->count; ++k)
            if (cls[k] == c) { b->TR[k] = bt; b->TC[k] = bc; b->D[k] = bd; }
        st = batch_build(b, s);
        if (st) return st;
    }
    // then the resident CTAs per SM of the launches (fewer CTAs leave each
    // warp more of the L2 and the memory pipes)
    const int32_t cps_c[] = {2, 1};
    int32_t best_cps = b->ctas_per_sm;
    for (int32_t cps : cps_c) {
        if (cps == best_cps) continue;
        b->ctas_per_sm = cps;
        float ms = 0.0f;
        st = time_batch(b, workspace, workspace_bytes, reps, s, &ms);
        if (st) return st;
        if (ms < best) {
            best = ms;
            best_cps = cps;
        }
    }
    b->ctas_per_sm = best_cps;
    if (b->graph) {   // the captured launch carries the grid size
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
        b->graph_ws = nullptr;
    }
    if (best_ms) *best_ms = best;
    return SPMM_OK;
}
