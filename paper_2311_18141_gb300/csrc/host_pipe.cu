// Host-buffer pipeline: the local product of Section 2.1 with A, B and C in
// host memory.  Step k copies its inputs into device slot k mod depth on the
// copy-in stream, multiplies on the caller's stream with the pipeline's plan,
// and copies C out on the copy-out stream.  Events order each slot's reuse:
// inputs overwrite a slot only after the product that read it is done, and a
// product writes a slot's C only after the previous C has left it.  With two
// or more slots the three streams overlap, the upload of step k+1 and the
// download of step k-1 running while step k multiplies (the prefetching of
// Section 3.3, between host and device instead of between GPUs).
#include <stdlib.h>
#include <string.h>

#include <new>

#include "api_internal.cuh"

using namespace spmm;

namespace {

constexpr int kMaxDepth = 4;

struct Slot {
    int32_t* rowptr = nullptr;
    int32_t* colind = nullptr;
    void* vals = nullptr;
    void* B = nullptr;
    float* C = nullptr;
    cudaEvent_t in_done = nullptr;    // inputs are on the device
    cudaEvent_t comp_done = nullptr;  // the product has read the inputs and written C
    cudaEvent_t out_done = nullptr;   // C is in host memory
    bool used = false;
};

size_t round256(size_t b) { return (b + 255) / 256 * 256; }

// Copies go out in pieces of at most kCopyPiece bytes, so that uploads and
// downloads on the two copy streams interleave finely instead of one copy
// engine holding a multi-gigabyte transfer.
constexpr size_t kCopyPiece = (size_t)64 << 20;

cudaError_t copy_pieces(void* dst, const void* src, size_t bytes, cudaMemcpyKind kind,
                        cudaStream_t s) {
    for (size_t off = 0; off < bytes; off += kCopyPiece) {
        const size_t n = bytes - off < kCopyPiece ? bytes - off : kCopyPiece;
        const cudaError_t e = cudaMemcpyAsync(static_cast<char*>(dst) + off,
                                              static_cast<const char*>(src) + off, n, kind, s);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace

struct spmm_host_pipe_s {
    spmm_plan plan = nullptr;
    int64_t M = 0, K = 0, nnz = 0, N = 0;
    int32_t a_t = 0, b_t = 0;
    int depth = 0;
    cudaStream_t comp = nullptr, in = nullptr, out = nullptr;
    size_t rp_bytes = 0, ci_bytes = 0, v_bytes = 0, b_bytes = 0, c_bytes = 0;
    void* mem = nullptr;   // all slots, carved in 256-byte aligned pieces
    void* ws = nullptr;
    size_t ws_bytes = 0;
    int64_t submitted = 0;
    Slot slot[kMaxDepth];
};

static void pipe_free(spmm_host_pipe_s* p) {
    if (!p) return;
    for (int b = 0; b < kMaxDepth; ++b) {
        if (p->slot[b].in_done) cudaEventDestroy(p->slot[b].in_done);
        if (p->slot[b].comp_done) cudaEventDestroy(p->slot[b].comp_done);
        if (p->slot[b].out_done) cudaEventDestroy(p->slot[b].out_done);
    }
    if (p->in) cudaStreamDestroy(p->in);
    if (p->out) cudaStreamDestroy(p->out);
    if (p->mem) cudaFree(p->mem);
    if (p->ws) cudaFree(p->ws);
    delete p;
}

extern "C" {

int spmm_host_pipe_create(spmm_host_pipe* pipe, spmm_plan plan, int32_t a_dtype,
                          int32_t b_dtype, int32_t depth, void* stream) {
    if (!pipe) return SPMM_ERR_INVALID_ARG;
    *pipe = nullptr;
    if (!plan || depth < 1 || depth > kMaxDepth) return SPMM_ERR_INVALID_ARG;
    const int ea = elem_bytes(a_dtype), eb = elem_bytes(b_dtype);
    // E4M3 B only means something with its per-row scales, which the pipeline
    // does not carry
    if (ea == 0 || eb == 0 || b_dtype == SPMM_E4M3) return SPMM_ERR_UNSUPPORTED;
    spmm_host_pipe_s* p = new (std::nothrow) spmm_host_pipe_s();
    if (!p) return SPMM_ERR_INVALID_ARG;
    plan_shape(plan, &p->M, &p->K, &p->nnz, &p->N, nullptr, nullptr);
    if (p->N % (16 / eb) != 0) {
        delete p;
        return SPMM_ERR_MISALIGNED;
    }
    p->plan = plan;
    p->a_t = a_dtype;
    p->b_t = b_dtype;
    p->depth = depth;
    p->comp = (cudaStream_t)stream;
    p->rp_bytes = (size_t)(p->M + 1) * 4;
    p->ci_bytes = (size_t)p->nnz * 4;
    p->v_bytes = (size_t)p->nnz * ea;
    p->b_bytes = (size_t)p->K * p->N * eb;
    p->c_bytes = (size_t)p->M * p->N * 4;
    const size_t per_slot = round256(p->rp_bytes) + round256(p->ci_bytes) +
                            round256(p->v_bytes) + round256(p->b_bytes) + round256(p->c_bytes);
    int st = spmm_plan_workspace_size(plan, &p->ws_bytes);
    if (st) {
        delete p;
        return st;
    }
    if (cudaMalloc(&p->mem, per_slot * depth) != cudaSuccess ||
        cudaMalloc(&p->ws, p->ws_bytes) != cudaSuccess ||
        cudaMemsetAsync(p->ws, 0, p->ws_bytes, p->comp) != cudaSuccess ||
        cudaStreamCreateWithFlags(&p->in, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&p->out, cudaStreamNonBlocking) != cudaSuccess) {
        pipe_free(p);
        return SPMM_ERR_CUDA;
    }
    char* m = static_cast<char*>(p->mem);
    for (int b = 0; b < depth; ++b) {
        Slot& s = p->slot[b];
        s.rowptr = reinterpret_cast<int32_t*>(m);
        m += round256(p->rp_bytes);
        s.colind = reinterpret_cast<int32_t*>(m);
        m += round256(p->ci_bytes);
        s.vals = m;
        m += round256(p->v_bytes);
        s.B = m;
        m += round256(p->b_bytes);
        s.C = reinterpret_cast<float*>(m);
        m += round256(p->c_bytes);
        if (cudaEventCreateWithFlags(&s.in_done, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&s.comp_done, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&s.out_done, cudaEventDisableTiming) != cudaSuccess) {
            pipe_free(p);
            return SPMM_ERR_CUDA;
        }
    }
    *pipe = p;
    return SPMM_OK;
}

int spmm_host_pipe_submit(spmm_host_pipe p, const int32_t* A_rowptr, const int32_t* A_colind,
                          const void* A_vals, const void* B, float* C) {
    if (!p || !A_rowptr || !C) return SPMM_ERR_INVALID_ARG;
    if (p->nnz > 0 && (!A_colind || !A_vals || !B)) return SPMM_ERR_INVALID_ARG;
    Slot& s = p->slot[p->submitted % p->depth];
    const auto ok = [](cudaError_t e) { return e == cudaSuccess; };
    // copy-in: the slot's inputs are free once step k - depth's product is done
    if (s.used && !ok(cudaStreamWaitEvent(p->in, s.comp_done, 0))) return SPMM_ERR_CUDA;
    if (!ok(copy_pieces(s.rowptr, A_rowptr, p->rp_bytes, cudaMemcpyHostToDevice, p->in)))
        return SPMM_ERR_CUDA;
    if (p->nnz > 0 &&
        (!ok(copy_pieces(s.colind, A_colind, p->ci_bytes, cudaMemcpyHostToDevice, p->in)) ||
         !ok(copy_pieces(s.vals, A_vals, p->v_bytes, cudaMemcpyHostToDevice, p->in)) ||
         !ok(copy_pieces(s.B, B, p->b_bytes, cudaMemcpyHostToDevice, p->in))))
        return SPMM_ERR_CUDA;
    if (!ok(cudaEventRecord(s.in_done, p->in))) return SPMM_ERR_CUDA;
    // product: needs this step's inputs, and step k - depth's C out of the slot
    if (!ok(cudaStreamWaitEvent(p->comp, s.in_done, 0))) return SPMM_ERR_CUDA;
    if (s.used && !ok(cudaStreamWaitEvent(p->comp, s.out_done, 0))) return SPMM_ERR_CUDA;
    const int st = spmm_csr(s.rowptr, s.colind, s.vals, p->a_t, nullptr, s.B, p->b_t, nullptr,
                            p->N, s.C, p->N, p->M, p->K, p->N, p->nnz, 0, 0, 0.0f, p->plan, p->ws,
                            p->ws_bytes, p->comp);
    if (st) return st;
    if (!ok(cudaEventRecord(s.comp_done, p->comp))) return SPMM_ERR_CUDA;
    // copy-out
    if (!ok(cudaStreamWaitEvent(p->out, s.comp_done, 0)) ||
        !ok(copy_pieces(C, s.C, p->c_bytes, cudaMemcpyDeviceToHost, p->out)) ||
        !ok(cudaEventRecord(s.out_done, p->out)))
        return SPMM_ERR_CUDA;
    s.used = true;
    ++p->submitted;
    return SPMM_OK;
}

int spmm_host_pipe_wait(spmm_host_pipe p) {
    if (!p) return SPMM_ERR_INVALID_ARG;
    if (cudaStreamSynchronize(p->in) != cudaSuccess ||
        cudaStreamSynchronize(p->comp) != cudaSuccess ||
        cudaStreamSynchronize(p->out) != cudaSuccess)
        return SPMM_ERR_CUDA;
    int32_t status = SPMM_OK;
    const int st = spmm_get_device_status(p->ws, &status, p->comp);
    if (st) return st;
    return status;
}

int spmm_host_pipe_destroy(spmm_host_pipe p) {
    if (!p) return SPMM_OK;
    cudaStreamSynchronize(p->in);
    cudaStreamSynchronize(p->comp);
    cudaStreamSynchronize(p->out);
    pipe_free(p);
    return SPMM_OK;
}

}  // extern "C"
