// Host-side helpers for plan construction (merge-path chunk boundaries).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace spmm {

// Upper bound on the number of chunks of all row blocks.
int64_t plan_chunk_cap(int64_t M, int64_t nnz, int32_t TR, int32_t D);
// Default merge-path items per chunk: about 16 units per warp of the grid, or
// longer (up to 16 mean rows, keeping 4 units per warp) so that few rows are cut.
int32_t plan_default_chunk(int64_t M, int64_t nnz, int32_t TC, int sms, int groups);
// Lane groups per warp of the staged kernel's FP32 shape for N columns in TC
// blocks (the default kernel).
int plan_default_groups(int64_t N, int32_t TC);
// Bytes of the plan arrays (blk_base, bnd_row, bnd_nnz, the split-row list
// and its count), 256-byte padded.
size_t plan_array_bytes(int32_t TR, int64_t cap);
// Split a plan-array region into its arrays.
void plan_carve(void* base, int32_t TR, int64_t cap, int32_t** blk_base, int32_t** bnd_row,
                int32_t** bnd_nnz, int4** split, int32_t** n_split);
// Row-end bitmap over the merge path of the whole matrix: the merge item of
// row r's end is r + rowptr[r+1] (the item of nonzero e of row r is r + e),
// and bit (r + rowptr[r+1]) is set for every row.  Bytes for M + nnz items
// (two words of padding, so a 64-bit window read never leaves the array).
size_t plan_ends_bytes(int64_t items);
// Clear the bitmap and set the row ends (enqueued on `s`).
cudaError_t plan_build_ends(const int32_t* rowptr, int64_t M, int64_t items, uint32_t* ends,
                            cudaStream_t s);
// Enqueue the two plan kernels on `s`.  Besides the boundaries they list the
// rows that a boundary cuts, one entry per row: {row, global chunk where it
// begins, global chunk where it ends, 0}, in no particular order.
cudaError_t plan_build(const int32_t* rowptr, int64_t M, int32_t TR, int32_t RB, int32_t D,
                       int64_t cap, int32_t* blk_base, int32_t* bnd_row, int32_t* bnd_nnz,
                       int4* split, int32_t* n_split, cudaStream_t s);

}  // namespace spmm
