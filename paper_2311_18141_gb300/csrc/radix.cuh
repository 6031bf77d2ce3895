// Device building blocks shared by the CSR -> CSC transpose and the SpGEMM:
// a stable LSD radix sort of int32 keys with int32 payloads, an in-place
// exclusive scan of an int32 array, and the row of every CSR nonzero.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace spmm {

// Scratch (bytes) of radix_sort_pairs for n keys of key_bits bits, and of
// scan_exclusive_i32 for n elements; the caller provides it 256-byte aligned.
size_t radix_scratch_bytes(int64_t n, int key_bits);
size_t scan_scratch_bytes(int64_t n);

// Stable sort of n keys (key_bits significant bits; keys >= 0 and < 2^key_bits)
// carrying a payload (vals == nullptr: the payload is the element's index).
// The passes -- the fewest of at most 9-bit digits, each digit at least 8
// bits -- ping-pong between (k0, v0) and (k1, v1), which must not alias the
// inputs; *out is set to 0 or 1, the pair that holds the result.  Enqueued on s.
cudaError_t radix_sort_pairs(const int32_t* keys, const int32_t* vals, int64_t n, int key_bits,
                             int32_t* k0, int32_t* v0, int32_t* k1, int32_t* v1, void* scratch,
                             int* out, cudaStream_t s);

// data[0..n) := exclusive prefix sums of data (int32; the caller guarantees
// that every partial sum fits in int32).  Enqueued on s.
cudaError_t scan_exclusive_i32(int32_t* data, int64_t n, void* scratch, cudaStream_t s);

// row_of[e] = row of CSR nonzero e.
cudaError_t csr_rows_of(const int32_t* rowptr, int64_t M, int32_t* row_of, cudaStream_t s);

// ptr[c] = first index of sorted[0..n) whose value is >= c, for c in [0, K].
cudaError_t lower_bounds(const int32_t* sorted, int64_t n, int64_t K, int32_t* ptr,
                         cudaStream_t s);

// Bits needed for values in [0, n): at least 1.
int bits_for(int64_t n);

}  // namespace spmm
