// Device helpers shared by the sm_103a kernels: cache-hinted loads and
// stores, element decode, packed FP32 FMA, and the argument blocks.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include "spmm_gb300.h"

namespace spmm {

constexpr unsigned kFull = 0xffffffffu;

// ---------------------------------------------------------------- loads ----

// Streaming 32-bit load that skips L1 (CSR arrays are touched once per unit;
// they stay in L2 for the other column blocks of the same chunk).
__device__ __forceinline__ int32_t ld_stream_i32(const int32_t* p) {
    int32_t v;
    asm volatile("ld.global.nc.L1::no_allocate.b32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ uint32_t ld_stream_u16(const void* p) {
    uint16_t v;
    asm volatile("ld.global.nc.L1::no_allocate.u16 %0, [%1];" : "=h"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ uint32_t ld_stream_u8(const void* p) {
    uint16_t v;
    asm volatile("ld.global.nc.L1::no_allocate.u8 %0, [%1];" : "=h"(v) : "l"(p));
    return v;
}

// 16-byte read-only load of a B row vector (L1-cacheable: hot rows repeat).
__device__ __forceinline__ uint4 ld_b16(const void* p) {
    return __ldg(reinterpret_cast<const uint4*>(p));
}

// 16-byte asynchronous copy global -> shared; copies `src_bytes` (16 or 0)
// and zero-fills the rest of the 16 bytes.  SPMM_CP_ASYNC_CA=1 allocates the
// line in L1 (.ca); the default bypasses L1 (.cg): gathered B rows are
// rarely re-read from the same SM.
#ifndef SPMM_CP_ASYNC_CA
#define SPMM_CP_ASYNC_CA 0
#endif
__device__ __forceinline__ void cp_async16(uint32_t smem_addr, const void* gptr, int src_bytes) {
#if SPMM_CP_ASYNC_CA
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16, %2;"
                 :: "r"(smem_addr), "l"(gptr), "r"(src_bytes) : "memory");
#else
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;"
                 :: "r"(smem_addr), "l"(gptr), "r"(src_bytes) : "memory");
#endif
}
// 16-byte cp.async that zero-fills instead of reading when `mask & bit` is
// 0: the test is part of the asm (a constant `bit` folds into it), so no 0/1
// value is formed first.
__device__ __forceinline__ void cp_async16_if_set(uint32_t smem_addr, const void* gptr,
                                                  uint32_t mask, uint32_t bit) {
    asm volatile("{\n\t.reg .pred q;\n\t.reg .b32 t;\n\t"
                 "and.b32 t, %2, %3;\n\tsetp.eq.b32 q, t, 0;\n\t"
#if SPMM_CP_ASYNC_CA
                 "cp.async.ca.shared.global [%0], [%1], 16, q;\n\t}"
#else
                 "cp.async.cg.shared.global [%0], [%1], 16, q;\n\t}"
#endif
                 :: "r"(smem_addr), "l"(gptr), "r"(mask), "r"(bit) : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
    asm volatile("cp.async.commit_group;" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" :: "n"(N) : "memory");
}

// ---- mbarriers, waited on with a bound ----
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" :: "r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_init_fence() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile("{\n\t.reg .pred p;\n\t"
                 "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(ok) : "r"(bar), "r"(parity) : "memory");
    return ok != 0;
}
// Wait for phase `parity` of `bar` to complete, for at most about a second
// (2^31 SM cycles); false when the wait ran out.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > (1ll << 31)) return false;
    return true;
}

__device__ __forceinline__ uint4 lds128(uint32_t smem_addr) {
    uint4 v;
    asm volatile("ld.shared.v4.u32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "r"(smem_addr));
    return v;
}

// Relaxed GPU-scope read of a work counter.
__device__ __forceinline__ int32_t ld_relaxed(const int32_t* p) {
    int32_t v;
    asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
}

// GPU-scope fetch-and-add with acquire-release semantics.
__device__ __forceinline__ int atom_add_acq_rel(int* p, int v) {
    int old;
    asm volatile("atom.add.acq_rel.gpu.global.s32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v)
                 : "memory");
    return old;
}

// 16-byte L2 (coherent) load, used to read partial rows written by other SMs.
__device__ __forceinline__ float4 ld_cg_f4(const float* p) {
    return __ldcg(reinterpret_cast<const float4*>(p));
}

// Streaming 16-byte store (C is written once).
__device__ __forceinline__ void st_cs_f4(float* p, float4 v) {
    __stcs(reinterpret_cast<float4*>(p), v);
}
__device__ __forceinline__ void st_cg_f4(float* p, float4 v) {
    __stcg(reinterpret_cast<float4*>(p), v);
}

// ---- 32-byte (256-bit) accesses, sm_100 and later ----
// One lane moves a whole 32-byte sector per instruction: half the load
// instructions of 16-byte vectors for the same bytes.
struct V32 {
    uint4 lo, hi;
};

// B-row gather into registers.  SPMM_GATHER_L1=1 lets the line allocate in
// L1 (hot rows may then hit there); the default bypasses L1.
#ifndef SPMM_GATHER_L1
#define SPMM_GATHER_L1 0
#endif
__device__ __forceinline__ V32 ld_gather32(const void* p) {
    V32 v;
#if SPMM_GATHER_L1
    asm("ld.global.nc.v8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
        : "=r"(v.lo.x), "=r"(v.lo.y), "=r"(v.lo.z), "=r"(v.lo.w),
          "=r"(v.hi.x), "=r"(v.hi.y), "=r"(v.hi.z), "=r"(v.hi.w) : "l"(p));
#else
    asm("ld.global.nc.L1::no_allocate.v8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
        : "=r"(v.lo.x), "=r"(v.lo.y), "=r"(v.lo.z), "=r"(v.lo.w),
          "=r"(v.hi.x), "=r"(v.hi.y), "=r"(v.hi.z), "=r"(v.hi.w) : "l"(p));
#endif
    return v;
}
// Coherent (L2) 32-byte load of partial rows written by other SMs.
__device__ __forceinline__ void ld_cg_f8(const float* p, float4& a, float4& b) {
    asm volatile("ld.global.cg.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=f"(a.x), "=f"(a.y), "=f"(a.z), "=f"(a.w),
                   "=f"(b.x), "=f"(b.y), "=f"(b.z), "=f"(b.w) : "l"(p) : "memory");
}
// Streaming 32-byte store (C is written once) and an L2 store (partial rows).
__device__ __forceinline__ void st_cs_f8(float* p, const float4& a, const float4& b) {
    asm volatile("st.global.cs.v8.f32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};"
                 :: "l"(p), "f"(a.x), "f"(a.y), "f"(a.z), "f"(a.w),
                    "f"(b.x), "f"(b.y), "f"(b.z), "f"(b.w) : "memory");
}
__device__ __forceinline__ void st_cg_f8(float* p, const float4& a, const float4& b) {
    asm volatile("st.global.cg.v8.f32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};"
                 :: "l"(p), "f"(a.x), "f"(a.y), "f"(a.z), "f"(a.w),
                    "f"(b.x), "f"(b.y), "f"(b.z), "f"(b.w) : "memory");
}

// ---------------------------------------------------------------- math ----

// c += a * b on two FP32 lanes at once (packed FFMA2 on sm_100 and later).
__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c) {
#if defined(__CUDA_ARCH__) && (__CUDA_ARCH__ >= 1000) && !defined(SPMM_SCALAR_FMA)
    return __ffma2_rn(a, b, c);
#else
    return make_float2(fmaf(a.x, b.x, c.x), fmaf(a.y, b.y, c.y));
#endif
}

// -------------------------------------------------------------- decode ----

// Element traits of a storage type: EPV = elements per 16-byte vector.
struct TagF32 { static constexpr int EPV = 4;  static constexpr int dtype = SPMM_F32; };
struct TagF16 { static constexpr int EPV = 8;  static constexpr int dtype = SPMM_F16; };
struct TagBF16 { static constexpr int EPV = 8; static constexpr int dtype = SPMM_BF16; };
struct TagE4M3 { static constexpr int EPV = 16; static constexpr int dtype = SPMM_E4M3; };

__device__ __forceinline__ float bf16lo(uint32_t w) { return __uint_as_float(w << 16); }
__device__ __forceinline__ float bf16hi(uint32_t w) { return __uint_as_float(w & 0xffff0000u); }

__device__ __forceinline__ float2 h2f2(uint32_t w) {
    __half2 h = *reinterpret_cast<const __half2*>(&w);
    return __half22float2(h);
}

// two E4M3 codes (low 16 bits of w) -> two floats, exactly (E4M3 is a subset of f16)
__device__ __forceinline__ float2 e4m3x2_to_f2(uint16_t w) {
    uint32_t h2;
    asm("cvt.rn.f16x2.e4m3x2 %0, %1;" : "=r"(h2) : "h"(w));
    return h2f2(h2);
}

// acc[0 .. EPV/2) += a2 * decode(v), a2 = (a, a)
template <typename Tag>
__device__ __forceinline__ void fma_vec(float2* acc, float2 a2, const uint4& v);

template <>
__device__ __forceinline__ void fma_vec<TagF32>(float2* acc, float2 a2, const uint4& v) {
    acc[0] = ffma2(a2, make_float2(__uint_as_float(v.x), __uint_as_float(v.y)), acc[0]);
    acc[1] = ffma2(a2, make_float2(__uint_as_float(v.z), __uint_as_float(v.w)), acc[1]);
}
template <>
__device__ __forceinline__ void fma_vec<TagBF16>(float2* acc, float2 a2, const uint4& v) {
    acc[0] = ffma2(a2, make_float2(bf16lo(v.x), bf16hi(v.x)), acc[0]);
    acc[1] = ffma2(a2, make_float2(bf16lo(v.y), bf16hi(v.y)), acc[1]);
    acc[2] = ffma2(a2, make_float2(bf16lo(v.z), bf16hi(v.z)), acc[2]);
    acc[3] = ffma2(a2, make_float2(bf16lo(v.w), bf16hi(v.w)), acc[3]);
}
template <>
__device__ __forceinline__ void fma_vec<TagF16>(float2* acc, float2 a2, const uint4& v) {
    acc[0] = ffma2(a2, h2f2(v.x), acc[0]);
    acc[1] = ffma2(a2, h2f2(v.y), acc[1]);
    acc[2] = ffma2(a2, h2f2(v.z), acc[2]);
    acc[3] = ffma2(a2, h2f2(v.w), acc[3]);
}
template <>
__device__ __forceinline__ void fma_vec<TagE4M3>(float2* acc, float2 a2, const uint4& v) {
    const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        acc[2 * q + 0] = ffma2(a2, e4m3x2_to_f2((uint16_t)(w[q] & 0xffffu)), acc[2 * q + 0]);
        acc[2 * q + 1] = ffma2(a2, e4m3x2_to_f2((uint16_t)(w[q] >> 16)), acc[2 * q + 1]);
    }
}

// A's value e of storage type TagA, as FP32.  `stream` skips L1 allocation.
template <typename TagA, bool stream>
__device__ __forceinline__ float aval(const void* vals, int64_t e);

template <> __device__ __forceinline__ float aval<TagF32, true>(const void* v, int64_t e) {
    return __int_as_float(ld_stream_i32(reinterpret_cast<const int32_t*>(v) + e));
}
template <> __device__ __forceinline__ float aval<TagF32, false>(const void* v, int64_t e) {
    return __ldg(reinterpret_cast<const float*>(v) + e);
}
template <> __device__ __forceinline__ float aval<TagF16, true>(const void* v, int64_t e) {
    return __half2float(__ushort_as_half((unsigned short)ld_stream_u16(reinterpret_cast<const uint16_t*>(v) + e)));
}
template <> __device__ __forceinline__ float aval<TagF16, false>(const void* v, int64_t e) {
    return __half2float(__ldg(reinterpret_cast<const __half*>(v) + e));
}
template <> __device__ __forceinline__ float aval<TagBF16, true>(const void* v, int64_t e) {
    return __uint_as_float(ld_stream_u16(reinterpret_cast<const uint16_t*>(v) + e) << 16);
}
template <> __device__ __forceinline__ float aval<TagBF16, false>(const void* v, int64_t e) {
    return __uint_as_float((uint32_t)__ldg(reinterpret_cast<const unsigned short*>(v) + e) << 16);
}
template <> __device__ __forceinline__ float aval<TagE4M3, true>(const void* v, int64_t e) {
    return e4m3x2_to_f2((uint16_t)ld_stream_u8(reinterpret_cast<const uint8_t*>(v) + e)).x;
}
template <> __device__ __forceinline__ float aval<TagE4M3, false>(const void* v, int64_t e) {
    return e4m3x2_to_f2((uint16_t)__ldg(reinterpret_cast<const unsigned char*>(v) + e)).x;
}


// ----------------------------------------------------------- arguments ----

// One SpMM problem as the persistent kernel sees it.
struct Problem {
    const int32_t* rowptr;
    const int32_t* colind;
    const void* vals;
    const float* a_scale;   // nullable, [M]
    const void* B;
    const float* b_scale;   // nullable, [K]
    float* C;
    int64_t ldb;            // elements
    int64_t ldc;            // elements
    int32_t M, N;
    int32_t a_dtype;
    float beta;
    // plan
    int32_t TR, TC, RB, W, D;
    const int32_t* blk_base;  // [TR+1] chunk prefix per row block
    const int32_t* bnd_row;   // boundary (row, nnz) at index blk_base[i] + i + c
    const int32_t* bnd_nnz;
    const uint32_t* ends;     // row-end bitmap over the merge items (see plan_ends_bytes)
    const int4* split;        // rows cut by a chunk boundary: {row, first chunk, last chunk, 0}
    const int32_t* n_split;   // how many entries of `split` the plan wrote
    // per-call scratch
    int32_t* tile_ctr;        // [TR*TC]
    int32_t* piece_cnt;       // [chunks*TC]
    float* slots;             // [2*chunks][N]
    int32_t* status;          // status words
    // optional per-warp trace (null: off)
    spmm_trace_record* trace;
    int32_t trace_max;
};

// Workspace layout (offsets in bytes from the workspace base).
constexpr size_t kStatusBytes = 64;      // status[0]: first error code, status[1]: internal

}  // namespace spmm
