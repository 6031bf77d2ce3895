// Declarations shared by the C ABI translation units.
#pragma once

#include "common.cuh"

namespace spmm {

int elem_bytes(int dt);
void resolve_tuning(const spmm_tuning* in, spmm_tuning* out);
int64_t column_block_width(int64_t N, int32_t TC, int dt);
bool pick_shape(int64_t nvec, int* lpn, int* vpl);
int device_sm_count();
// Shape check and array view of a plan; SPMM_ERR_PLAN_MISMATCH if the plan was
// built for another (M, K, nnz, N).
int plan_view(spmm_plan plan, int64_t M, int64_t K, int64_t nnz, int64_t N, int32_t* TR,
              int32_t* TC, int32_t* RB, int32_t* D, int64_t* cap, int32_t** blk_base,
              int32_t** bnd_row, int32_t** bnd_nnz);
// Sum the split rows of a staged product (left in workspace slots by
// spmm_csr_persistent) into C; `max_rows` bounds the length of the plan's
// split-row list (chunk capacity + TR).  Enqueued on `s` after the product.
cudaError_t launch_split_row_fixup(const Problem& p, int64_t max_rows, cudaStream_t s);
// The same for the `count` products of a batch table (device array), whose
// slots lie in the batch workspace `ws`; `max_items` bounds any product's
// (split row, 16-byte vector) pairs.  Enqueued on `s` after the products.
struct BatchEntry;
cudaError_t launch_split_row_fixup_batched(const BatchEntry* table, int count, char* ws,
                                           int64_t max_items, cudaStream_t s);
// Shape of a plan (any output may be null).
int plan_shape(spmm_plan plan, int64_t* M, int64_t* K, int64_t* nnz, int64_t* N, int32_t* TR,
               int32_t* TC);

}  // namespace spmm
