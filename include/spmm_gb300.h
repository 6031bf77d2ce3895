/*
 * spmm_gb300.h -- C ABI of the GB300 CSR sparse-times-dense product library.
 *
 * The library computes the local tile product of Brock, Bulu\c{c} and Yelick,
 * "RDMA-Based Algorithms for Sparse Matrix Multiplication on GPUs" (ICS'24):
 * C_ij = C_ij + sum_k A_ik B_kj (Section 2.1), where A is a CSR matrix and B, C
 * are dense.  The paper's distributed, asynchronous, work-stealing schedule
 * (Sections 3.2-3.4, Algorithms 2 and 3) is re-expressed inside one GPU: the
 * C-row-block x B-column-block tiles of a 2D tile grid are work queues that a
 * persistent kernel's warps reserve from with atomic fetch-and-add, and a warp
 * whose own tile is empty steals from other tiles, same tile row first.
 *
 * Conventions for every entry point:
 *   - Pointers marked "device" are CUDA device (or managed) pointers owned by
 *     the caller; pointers marked "host" are ordinary host pointers.  The
 *     library never frees caller memory and never keeps a caller pointer past
 *     the call, except that a plan keeps nothing but its own device arrays.
 *   - `stream` is a cudaStream_t passed as void*; NULL means the legacy
 *     default stream.  All device work is enqueued asynchronously on it; the
 *     calls do not synchronise unless documented.
 *   - Dense matrices are row-major with a leading dimension in ELEMENTS
 *     (ldb >= N, ldc >= N, and a row stride below 2^32 bytes: larger
 *     strides return SPMM_ERR_INVALID_ARG).  Vector paths need B, C,
 *     ldb*elem_size and ldc*4 to be 16-byte aligned and N a multiple of the
 *     elements in 16 bytes of B's type (4 for F32, 8 for F16/BF16, 16 for
 *     E4M3); otherwise the call returns SPMM_ERR_MISALIGNED and enqueues
 *     nothing.
 *   - Indices are int32; nnz < 2^31.  CSR rows may be in any column order and
 *     may repeat a column (repeats are summed); rowptr must be non-decreasing
 *     with rowptr[0] = 0 and rowptr[M] = nnz, and every column index must lie
 *     in [0, K).  Compute calls trust this; spmm_csr_validate checks it.
 *   - Every entry point returns an int status: SPMM_OK (0) or a negative code
 *     below.  No entry point exits, traps or throws.  Errors found by device
 *     code are written to a status word in the caller's workspace and read
 *     with spmm_get_device_status.
 *   - The hot calls (spmm_csr with a plan, spmm_sddmm_csr with a plan,
 *     spmm_csr_batched) allocate no memory: all scratch comes from the
 *     caller's workspace.  Plan creation allocates (cudaMalloc) and is meant
 *     to happen once per sparsity pattern.
 */
#ifndef SPMM_GB300_H
#define SPMM_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---- */
#define SPMM_OK 0
#define SPMM_ERR_INVALID_ARG (-1)   /* null pointer, negative size, bad enum    */
#define SPMM_ERR_MISALIGNED (-2)    /* vector-path alignment rule broken         */
#define SPMM_ERR_UNSUPPORTED (-3)   /* dtype or width combination not built      */
#define SPMM_ERR_CUDA (-4)          /* a CUDA runtime call failed                */
#define SPMM_ERR_BAD_CSR (-5)       /* validator found a malformed CSR           */
#define SPMM_ERR_TIMEOUT (-6)       /* a bounded device wait ran out             */
#define SPMM_ERR_WORKSPACE (-7)     /* workspace missing or too small            */
#define SPMM_ERR_PLAN_MISMATCH (-8) /* plan built for another shape or grid      */
#define SPMM_ERR_INTERNAL (-9)      /* device sanity check on the plan failed    */

/* ---- element types ---- */
#define SPMM_F32 0   /* IEEE binary32                                   */
#define SPMM_F16 1   /* IEEE binary16                                   */
#define SPMM_BF16 2  /* bfloat16                                        */
#define SPMM_E4M3 3  /* OCP FP8 E4M3 (finite variant, max 448)          */

typedef struct spmm_plan_s* spmm_plan;

/* Tuning knobs; a zero field means "library default".  Host struct. */
typedef struct spmm_tuning {
    int32_t chunk_items;   /* merge-path items (rows + nonzeros) per plan chunk; a
                              warp's work unit is 32/LPN chunks, one per lane group     */
    int32_t warps_per_cta; /* 1 to 8; 0 = 7 where four 7-warp CTAs fit on an SM, else 8 */
    int32_t ctas_per_sm;   /* persistent CTAs per SM; 0 = as many as fit              */
    int32_t tile_order;    /* bit 0: steal along the tile column first (else the row);
                              bit 1: stagger home tiles per warp (else per CTA);
                              bit 2: column sweep -- every CTA starts in column block 0
                              and steals column-major, so one column block of B is
                              live at a time;
                              bit 3: lockstep -- every warp starts on tile 0 and visits
                              the tiles in the same order (bit 0 picks column-major),
                              so one tile's B rows are live at a time;
                              bit 4: interleave -- one queue per tile row hands out the
                              same chunk of its tiles in turn (bit 3: all warps start
                              on tile row 0)                                           */
    int32_t kernel;        /* SPMM_KERNEL_AUTO (0): the library's choice, today the
                              16-byte staged kernel (it measured faster everywhere);
                              SPMM_KERNEL_STAGED (1): the staged kernel;
                              SPMM_KERNEL_WIDE (2): the 32-byte-lane register-gather
                              kernel, or SPMM_ERR_MISALIGNED when B, C, their strides
                              or the column blocks are not whole 32-byte vectors of
                              2..32 vectors per block;
                              SPMM_KERNEL_SPEC (3): the warp-specialised staged kernel
                              (producer warps decode and gather, consumer warps sum;
                              FP32 A with FP32 or BF16 B, FP16 A with FP32, FP16 or
                              BF16 B, column blocks of 8..32 16-byte vectors), else
                              SPMM_ERR_UNSUPPORTED                                      */
    int32_t lanes_per_item; /* 0: the default, one 16-byte vector per lane (a column
                              block of 8 vectors is walked by 8 lanes); 2 or 4: a block
                              of 4 or 8 vectors is walked by that many lanes holding
                              several vectors each (staged kernel only)               */
    int32_t reserved[2];
} spmm_tuning;

/* spmm_tuning.kernel values */
#define SPMM_KERNEL_AUTO 0
#define SPMM_KERNEL_STAGED 1
#define SPMM_KERNEL_WIDE 2
#define SPMM_KERNEL_SPEC 3

/* Human-readable name of a status code (static storage). */
const char* spmm_status_string(int status);

/* Library version as major*10000 + minor*100 + patch. */
int spmm_version(void);

/*
 * spmm_plan_create -- cut A into work units for a tile_rows x tile_cols grid.
 *   Section 2.1 tiles C into a grid of row blocks x column blocks; Section 3.4
 *   (Algorithm 3) reserves work inside a tile with fetch-and-add.  The plan
 *   splits each C row block's merge path (its rows interleaved with its
 *   nonzeros) into runs ("chunks") of about `chunk_items` items; a boundary
 *   inside a row of fewer than chunk_items/8 items moves to the row's start.
 *   The kernel reserves, in one column block, 32/LPN consecutive chunks at a
 *   time (LPN lanes hold one column block of a B row), one per lane group;
 *   a heavy row is shared by several chunks.
 *   A_rowptr  device int32[M+1], read on `stream` during this call.
 *   M, K, nnz, N  problem shape (N = columns of B and C).
 *   tile_rows, tile_cols  grid shape, 1 <= tile_rows <= 65536,
 *                 1 <= tile_cols <= N/vector width.  Column blocks are ceil(N /
 *                 tile_cols) rounded up to whole 16-byte vectors; the last one
 *                 may be narrower.
 *   tuning    host, nullable.
 *   On success *plan owns device memory; the plan arrays are complete once
 *   `stream` reaches this point.  Free with spmm_plan_destroy.
 */
int spmm_plan_create(spmm_plan* plan, const int32_t* A_rowptr, int64_t M, int64_t K,
                     int64_t nnz, int64_t N, int32_t tile_rows, int32_t tile_cols,
                     const spmm_tuning* tuning, void* stream);

/* Release a plan (synchronises the device first).  NULL is accepted. */
int spmm_plan_destroy(spmm_plan plan);

/* Bytes of per-call scratch a call with this plan needs (host out-param). */
int spmm_plan_workspace_size(spmm_plan plan, size_t* bytes);

/* Chunks of a plan and chunks x column blocks (the (chunk, tile) pairs), for
 * reporting. */
int spmm_plan_units(spmm_plan plan, int64_t* chunks, int64_t* units);

/*
 * spmm_plan_get_boundaries -- copy a plan's partition to host buffers
 *   (synchronous).  blk_base[TR+1]: chunks before row block i; for row block
 *   i, boundary c (0 <= c <= chunks of the block) sits at index
 *   blk_base[i] + i + c of bnd_row / bnd_nnz (int32[chunks + TR]), the merge-
 *   path point (rows finished, nonzeros consumed) where chunk c starts.  Any
 *   output may be NULL.  Meant for inspection and tests.
 */
int spmm_plan_get_boundaries(spmm_plan plan, int32_t* blk_base, int32_t* bnd_row,
                             int32_t* bnd_nnz);

/*
 * Per-warp trace of the persistent SpMM kernel: the on-chip counterpart of the
 * paper's split of run time into computation and load imbalance (Section 6).
 * Each warp of a spmm_csr launch with a traced plan writes one record, warp w
 * (= blockIdx.x * warps_per_cta + warp in CTA) to records[w] when w <
 * max_records; records past the launched warps are left untouched.
 */
typedef struct spmm_trace_record {
    int64_t t_start_ns;   /* %globaltimer when the warp started               */
    int64_t t_end_ns;     /* %globaltimer when it ran out of work             */
    int32_t units;        /* work units (32/LPN chunks of one tile) it walked */
    int32_t stolen;       /* of those, units outside its home tile (row)      */
    int32_t home;         /* its home tile (or tile row, interleaved order)   */
    int32_t smid;         /* the SM it ran on                                 */
} spmm_trace_record;

/*
 * spmm_plan_set_trace -- make spmm_csr calls with `plan` write trace records
 *   to `records` (device, spmm_trace_record[max_records], caller-owned; the
 *   buffer must outlive those calls).  records == NULL or max_records == 0
 *   turns tracing off.  A traced launch does the same work; each warp adds one
 *   32-byte store at its end.
 */
int spmm_plan_set_trace(spmm_plan plan, spmm_trace_record* records, int32_t max_records);

/* Bytes of workspace a spmm_csr call with plan == NULL needs: the plan arrays
 * plus the per-call scratch.  Such calls use the default tuning; `tuning` is
 * reserved and should be NULL. */
int spmm_csr_workspace_size(int64_t M, int64_t nnz, int64_t N, int32_t tile_rows,
                            int32_t tile_cols, const spmm_tuning* tuning, size_t* bytes);

/*
 * spmm_csr -- C = beta*C + diag(A_row_scale) * A * (diag(B_row_scale) * B).
 *   This is the local product C_ij = C_ij + sum_k A_ik B_kj of Section 2.1
 *   (the "local_c += local_a*local_b" step of Algorithm 2) computed for all
 *   tiles of the grid by one persistent launch; beta = 1 is the paper's
 *   accumulate, beta = 0 overwrites (C is then never read, NaNs included).
 *   A_rowptr, A_colind  device int32 CSR arrays.
 *   A_vals     device, nnz values of type a_dtype (F32, F16, BF16 or E4M3).
 *   A_row_scale device float[M] or NULL: row r of A is multiplied by it.
 *   B          device, K x N of type b_dtype (F32, F16, BF16 or E4M3), row
 *              stride ldb elements.
 *   B_row_scale device float[K] or NULL: row k of B is multiplied by it.
 *   C          device float, M x N, row stride ldc.  Accumulation is FP32.
 *   tile_rows, tile_cols  must equal the plan's (or be 0 to take the plan's).
 *   plan       from spmm_plan_create for the same rowptr/shape, or NULL to build
 *              the plan inside `workspace` on every call.
 *   workspace  device scratch of at least spmm_plan_workspace_size (plan) or
 *              spmm_csr_workspace_size (NULL plan) bytes, 256-byte aligned.
 *              Calls that share a workspace must not overlap on the GPU.
 *   Rows that the plan splits between work units are summed through the
 *   workspace in a fixed order by whichever unit finishes last, so results
 *   are bitwise reproducible run to run for a given plan and launch shape.
 */
int spmm_csr(const int32_t* A_rowptr, const int32_t* A_colind, const void* A_vals,
             int32_t a_dtype, const float* A_row_scale, const void* B, int32_t b_dtype,
             const float* B_row_scale, int64_t ldb, float* C, int64_t ldc, int64_t M,
             int64_t K, int64_t N, int64_t nnz, int32_t tile_rows, int32_t tile_cols,
             float beta, spmm_plan plan, void* workspace, size_t workspace_bytes,
             void* stream);

/* ---------------- batched products ---------------- */

/* One product of a batch: C = beta*C + diag(a_scale) * A * (diag(b_scale) * B).
 * All pointers are device pointers owned by the caller; layout and alignment
 * rules are those of spmm_csr.  tile_rows, tile_cols and chunk_items of 0 let
 * the library choose (tile_cols grows until one column block fits a warp). */
typedef struct spmm_problem {
    const int32_t* rowptr;
    const int32_t* colind;
    const void* vals;
    const float* a_scale;      /* nullable */
    const void* B;
    const float* b_scale;      /* nullable */
    float* C;
    int64_t M, K, N, nnz, ldb, ldc;
    float beta;
    int32_t tile_rows, tile_cols, chunk_items;
} spmm_problem;

typedef struct spmm_batch_s* spmm_batch;

/*
 * spmm_batch_create -- plans for `count` independent products run as one
 *   persistent launch.  The batch form of Section 3.4's reservation: every
 *   product keeps its own merge-path plan, its units (32/LPN chunks in one
 *   column block) are numbered after those of the products before it, and the
 *   warps of one grid reserve units from a single counter, so warps that finish
 *   one product move on to any other.  Products run by width (so the warps of an
 *   SM mostly share one kernel shape), each width largest first.  All products share A's value
 *   type `a_dtype` and B's type `b_dtype`.  `problems` is a host array copied at
 *   creation; the device arrays it points to must stay valid while the batch is
 *   used.  Allocates device memory for plans and the descriptor table and
 *   synchronises `stream`.
 */
int spmm_batch_create(spmm_batch* batch, const spmm_problem* problems, int32_t count,
                      int32_t a_dtype, int32_t b_dtype, void* stream);
int spmm_batch_destroy(spmm_batch batch);

/* Workspace bytes for spmm_csr_batched / spmm_batch_graph_launch under any
 * shapes spmm_batch_autotune may choose (chunks of at least 256 items, at most
 * two column blocks, up to 16 row blocks). */
int spmm_batch_workspace_size(spmm_batch batch, size_t* bytes);

/* Per-product shapes (host arrays of `count`, in the caller's order; an entry
 * of 0 or a NULL array keeps the current value).  Rebuilds the plans. */
int spmm_batch_set_shapes(spmm_batch batch, const int32_t* tile_rows, const int32_t* tile_cols,
                          const int32_t* chunk_items, void* stream);
int spmm_batch_get_shapes(spmm_batch batch, int32_t* tile_rows, int32_t* tile_cols,
                          int32_t* chunk_items);

/* All products of the batch in one persistent launch (after one counter-reset
 * memset).  No allocation; calls sharing a workspace must not overlap. */
int spmm_csr_batched(spmm_batch batch, void* workspace, size_t workspace_bytes, void* stream);

/* The same work replayed from a CUDA graph: the first call (and the first call
 * after a shape change or with another workspace) captures the memset and the
 * launch into a graph held by the batch; later calls only launch that graph. */
int spmm_batch_graph_launch(spmm_batch batch, void* workspace, size_t workspace_bytes,
                            void* stream);

/* Choose row blocks {1,4}, column blocks {1,2} and chunk size {256..2048} per
 * size class (same N, rows below 10k / 50k / above) by coordinate descent,
 * then the resident CTAs per SM of the launches (as many as fit, 2 or 1),
 * timing `reps` batched launches per candidate with CUDA events; leaves the
 * batch planned with the best choices and returns the best time in *best_ms. */
int spmm_batch_autotune(spmm_batch batch, void* workspace, size_t workspace_bytes, int32_t reps,
                        void* stream, float* best_ms);

/*
 * spmm_csr_noalloc -- spmm_csr for callers that cannot allocate device memory.
 *   The paper has no counterpart: this is a library convenience.  Some callers
 *   cannot call cudaMalloc where they need the product (code inside a memory
 *   pool they do not own, plug-ins whose host forbids device allocation, paths
 *   that must not synchronise the device, which cudaMalloc/cudaFree can do).
 *   This call takes no plan and no workspace: it builds the plan and keeps its
 *   counters and partial rows in one fixed 16 MiB device array that every GPU
 *   loading this library holds until the process exits.  It computes the same
 *   C = beta*C + diag(A_row_scale) * A * (diag(B_row_scale) * B) as spmm_csr
 *   with plan == NULL; all other arguments are as there.
 *   It allocates nothing (no cudaMalloc, cudaFree or allocating library call).
 *   Problems whose spmm_csr_workspace_size exceeds 16 MiB are rejected with
 *   SPMM_ERR_WORKSPACE before any device work.  The first call on a device
 *   looks up the array's device address (cudaGetSymbolAddress) with that
 *   device current; make that first call before any stream capture.  All
 *   calls on a device share the one array, so calls that overlap on the GPU
 *   (other streams, other host threads) race and give wrong results: order
 *   them on one stream or synchronise between them.
 */
int spmm_csr_noalloc(const int32_t* A_rowptr, const int32_t* A_colind, const void* A_vals,
                     int32_t a_dtype, const float* A_row_scale, const void* B, int32_t b_dtype,
                     const float* B_row_scale, int64_t ldb, float* C, int64_t ldc, int64_t M,
                     int64_t K, int64_t N, int64_t nnz, int32_t tile_rows, int32_t tile_cols,
                     float beta, void* stream);

/*
 * spmm_csr_noalloc_status -- the device status of spmm_csr_noalloc calls on
 *   the current device.  Errors that device code finds during such a call (an
 *   inconsistent plan, SPMM_ERR_INTERNAL; a bounded wait that ran out,
 *   SPMM_ERR_TIMEOUT) land in the status word of the fixed array, which no
 *   workspace pointer reaches.  This call synchronises `stream`, copies that
 *   word into *status (host) and clears it, like spmm_get_device_status does
 *   for a caller workspace.  Each spmm_csr_noalloc call clears the word when
 *   it starts, so read it after the call whose result you check and before the
 *   next one.  Allocates nothing.
 */
int spmm_csr_noalloc_status(int32_t* status, void* stream);

/*
 * spmm_csr_validate -- check the CSR invariants listed above on the device.
 *   Writes SPMM_OK or SPMM_ERR_BAD_CSR into the workspace status word (the
 *   first 64 bytes of `workspace`, which must hold at least 64 bytes); read it
 *   with spmm_get_device_status.  Never faults on a bad CSR: it reads only
 *   rowptr[0..M] and colind[0..nnz).
 */
int spmm_csr_validate(const int32_t* A_rowptr, const int32_t* A_colind, int64_t M, int64_t K,
                      int64_t nnz, void* workspace, size_t workspace_bytes, void* stream);

/*
 * Local SpGEMM, C = A * B: the sparse-sparse local product of the paper's
 *   SpGEMM experiments (Section 5), here for CSR A (M x K), CSR B (K x N) and
 *   CSR C with FP32 values.  Row i of C holds column j wherever some product
 *   A_ik * B_kj is formed (explicit zeros count), columns increasing; each
 *   value is the FP32 sum of its products taken in A's CSR order, then B's,
 *   so results are reproducible.  Three calls:
 *
 * spmm_spgemm_analyze -- number of products (sum over A's nonzeros of the
 *   length of B's row) and the workspace bytes spmm_spgemm needs.  Allocates
 *   and frees temporary device memory and synchronises `stream`.  Errors:
 *   SPMM_ERR_INVALID_ARG, SPMM_ERR_BAD_CSR (a column of A outside [0, K)),
 *   SPMM_ERR_UNSUPPORTED (2^31 - 1 products or more), SPMM_ERR_CUDA.
 */
int spmm_spgemm_analyze(const int32_t* A_rowptr, const int32_t* A_colind, int64_t M, int64_t K,
                        int64_t nnzA, const int32_t* B_rowptr, int64_t N, int64_t* products,
                        size_t* workspace_bytes, void* stream);

/* spmm_spgemm -- the product into `workspace` (256-byte aligned, at least the
 * analyzed size; no allocation); *entries := nnz of C.  Synchronises
 * `stream`.  Errors: SPMM_ERR_INVALID_ARG, SPMM_ERR_WORKSPACE, SPMM_ERR_BAD_CSR
 * (a column of B outside [0, N)), SPMM_ERR_CUDA. */
int spmm_spgemm(const int32_t* A_rowptr, const int32_t* A_colind, const float* A_vals, int64_t M,
                int64_t K, int64_t nnzA, const int32_t* B_rowptr, const int32_t* B_colind,
                const float* B_vals, int64_t N, int64_t products, void* workspace,
                size_t workspace_bytes, int64_t* entries, void* stream);

/* spmm_spgemm_copy -- C from the workspace of the spmm_spgemm call with the
 * same (M, nnzA, products) into caller buffers: C_rowptr[M+1], C_colind and
 * C_vals of `entries` elements (device).  Enqueued on `stream`. */
int spmm_spgemm_copy(const void* workspace, int64_t M, int64_t nnzA, int64_t products,
                     int64_t entries, int32_t* C_rowptr, int32_t* C_colind, float* C_vals,
                     void* stream);

/*
 * spmm_bench_gather -- measurement kernel: the B gathers of spmm_csr alone.
 *   Section 4 counts B's bytes once in the local product and notes that B
 *   values may have to be reloaded; a CSR product reads, for every nonzero e
 *   and every column block j, the block's segment of B row A_colind[e].  This
 *   call issues exactly those reads (32 bytes per lane, the interleaved order
 *   of spmm_csr's default tile order: chunk c of column blocks 0..TC-1 in
 *   turn) and nothing else -- no row pointers, values or C -- so its time is a
 *   floor for a product that gathers a B segment per nonzero, and a profile of
 *   it shows B's own L2 hit rate.
 *   A_colind  device int32[nnz], entries in [0, K) (trusted, as in spmm_csr).
 *   B         device, K x N of b_dtype, row stride ldb elements, 32-byte
 *             aligned; N split into tile_cols equal blocks of 64..1024 bytes,
 *             each a multiple of 32 bytes, and ldb*elem_size a multiple of 32
 *             (else SPMM_ERR_MISALIGNED).
 *   items_per_group  positions each lane group reads per chunk (4..4096, a
 *             multiple of 4); ctas_per_sm 0 = as many as fit.
 *   out       device float[1]: the sum of every value read, taken as FP32
 *             words, is ADDED to it (float atomics, so the low bits vary run to
 *             run).  It keeps the loads from being dropped; for F32 B it also
 *             checks that they read the right rows.
 *   Returns SPMM_ERR_INVALID_ARG for bad sizes or nnz >= 2^31 - 2^18.
 */
int spmm_bench_gather(const int32_t* A_colind, int64_t nnz, const void* B, int32_t b_dtype,
                      int64_t ldb, int64_t K, int64_t N, int32_t tile_cols,
                      int32_t items_per_group, int32_t ctas_per_sm, float* out, void* stream);

/* Synchronise `stream`, then copy the device status word of `workspace` into
 * *status (host) and clear it. */
int spmm_get_device_status(void* workspace, int32_t* status, void* stream);

/*
 * spmm_selftest_wait_timeout -- exercise the bounded device wait.  One thread
 *   waits on an mbarrier phase that nothing completes, for at most
 *   limit_cycles SM cycles (1 .. 2^31; 2^20 is about half a millisecond),
 *   then writes SPMM_ERR_TIMEOUT into the status word of `workspace` (device,
 *   at least 64 bytes) and returns; the CUDA context stays usable.  This is
 *   how a product reports copies that never arrive, without faulting or
 *   hanging the GPU.  Read the result with spmm_get_device_status.
 */
int spmm_selftest_wait_timeout(void* workspace, size_t workspace_bytes, int64_t limit_cycles,
                               void* stream);

/*
 * Host-buffer pipeline -- the local product C = A B of Section 2.1 for
 * operands that live in host memory, one product per submitted step.  Each
 * step copies A (rowptr, colind, vals) and B from the host to the device,
 * runs spmm_csr with the pipeline's plan, and copies C back to the host.  The
 * pipeline owns `depth` device slots (one set of A, B and C arrays each), one
 * workspace and two streams of its own (copy-in, copy-out); the products run
 * on the caller's `stream`.  Step k uses slot k mod depth: its inputs copy in
 * once the product of step k - depth has finished reading that slot, and its
 * product starts once step k - depth's C has left the slot.  With depth >= 2
 * the upload of step k+1 and the download of step k-1 overlap the product of
 * step k, the way the paper's prefetching overlaps tile transfers with local
 * multiplies (Section 3.3).  depth = 1 runs the steps one after the other.
 */
typedef struct spmm_host_pipe_s* spmm_host_pipe;

/*
 * spmm_host_pipe_create -- allocate a pipeline for `plan`'s shape (M, K, nnz,
 *   N and tile grid): depth (1..4) slots of (M+1) + nnz int32, nnz elements
 *   of a_dtype, K x N elements of b_dtype (dense, ldb = N) and M x N float
 *   (ldc = N), plus the plan's workspace.  N must meet the vector-path rule of
 *   b_dtype.  No row scales are carried: b_dtype E4M3 returns
 *   SPMM_ERR_UNSUPPORTED.  The plan must outlive the pipeline.  Allocates device memory and
 *   creates two streams and 3 * depth events; *pipe is NULL on failure.
 */
int spmm_host_pipe_create(spmm_host_pipe* pipe, spmm_plan plan, int32_t a_dtype,
                          int32_t b_dtype, int32_t depth, void* stream);

/*
 * spmm_host_pipe_submit -- enqueue one step: A_rowptr int32[M+1], A_colind
 *   int32[nnz], A_vals (a_dtype)[nnz] and B (b_dtype)[K*N] are host inputs;
 *   C float[M*N] receives A B (host).  All five are host pointers.  The call
 *   only enqueues work and returns: the inputs must stay unchanged and C
 *   unread until spmm_host_pipe_wait returns.  The copies overlap other work
 *   only when the host buffers are page-locked (cudaHostAlloc or
 *   cudaHostRegister); pageable buffers are copied synchronously.
 */
int spmm_host_pipe_submit(spmm_host_pipe pipe, const int32_t* A_rowptr, const int32_t* A_colind,
                          const void* A_vals, const void* B, float* C);

/*
 * spmm_host_pipe_wait -- block until every submitted step's C is in host
 *   memory.  Returns SPMM_OK, SPMM_ERR_CUDA, or the first error a product's
 *   device code reported (e.g. SPMM_ERR_TIMEOUT, SPMM_ERR_INTERNAL), which it
 *   then clears.
 */
int spmm_host_pipe_wait(spmm_host_pipe pipe);

/* spmm_host_pipe_destroy -- wait for outstanding steps, then free the slots,
 * the workspace, the streams and the events.  NULL is a no-op. */
int spmm_host_pipe_destroy(spmm_host_pipe pipe);

/*
 * spmm_csr_transpose -- CSR of A (M x K) -> CSR of A^T (K x M), i.e. A's CSC.
 *   Needed by the backward pass dB = A^T dC.  Built on the device by a stable
 *   least-significant-digit radix sort of the nonzeros by column, so each
 *   column lists its rows in increasing order and the output is identical run
 *   to run.
 *   out_colptr device int32[K+1]; out_rowind device int32[nnz];
 *   out_vals   device, nnz elements of val_dtype (may be NULL);
 *   out_perm   device int32[nnz] or NULL: CSR position of each CSC entry, so
 *              values can be re-gathered later without a new sort.
 *   workspace  at least spmm_csr_transpose_workspace_size bytes.
 */
int spmm_csr_transpose_workspace_size(int64_t M, int64_t K, int64_t nnz, size_t* bytes);
int spmm_csr_transpose(const int32_t* A_rowptr, const int32_t* A_colind, const void* A_vals,
                       int32_t val_dtype, int64_t M, int64_t K, int64_t nnz,
                       int32_t* out_colptr, int32_t* out_rowind, void* out_vals,
                       int32_t* out_perm, void* workspace, size_t workspace_bytes,
                       void* stream);

/* Gather out_vals[p] = vals[perm[p]] for p < nnz (elements of val_dtype). */
int spmm_gather_values(const void* vals, int32_t val_dtype, const int32_t* perm, int64_t nnz,
                       void* out_vals, void* stream);

/*
 * spmm_sddmm_csr -- out_vals[e] = sum_n dC[row_e, n] * B[col_e, n] for every
 *   nonzero e of A's pattern: the gradient of sum(dC .* (A B)) with respect to
 *   A's values.  dC device float M x N (stride lddc); B device of b_dtype
 *   (F32 or BF16) K x N (stride ldb); out_vals device float[nnz].
 *   plan: a plan of the same A with tile_cols == 1 (or NULL: built inside the
 *   workspace, sized by spmm_csr_workspace_size with tile grid 1 x 1).
 */
int spmm_sddmm_csr(const int32_t* A_rowptr, const int32_t* A_colind, const float* dC,
                   int64_t lddc, const void* B, int32_t b_dtype, int64_t ldb, float* out_vals,
                   int64_t M, int64_t K, int64_t N, int64_t nnz, spmm_plan plan,
                   void* workspace, size_t workspace_bytes, void* stream);

/*
 * spmm_quantize_rows -- store a float32 matrix in a narrower type.
 *   X device float rows x cols (stride ldx).  dtype F16 or BF16: Xq = round-
 *   to-nearest-even of X, `scale` ignored (may be NULL).  dtype E4M3: per row,
 *   s = amax|X[r,:]| / 448 computed in FP32 (s = 1 for an all-zero row),
 *   Xq = E4M3(X / s) rounded to nearest even with saturation to +-448, and
 *   scale[r] = s (device float[rows], required).  Xq stride ldq elements.
 */
int spmm_quantize_rows(const float* X, int64_t rows, int64_t cols, int64_t ldx, int32_t dtype,
                       void* Xq, int64_t ldq, float* scale, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* SPMM_GB300_H */
