// cw_lsqr_precond_host: the preconditioned LSQR of cw_lsqr_precond for a CSR
// matrix and right-hand side held in host memory.
//
// The host -> device copy of A is the longest step of such a call (GB300's
// link from host memory runs at a few percent of HBM bandwidth), so it is
// overlapped with the sketch.  The rows are cut into kHostChunks row ranges of
// about equal nonzero count.  A second stream copies chunk after chunk (row_ptr,
// b, then the chunk's col and val); as each chunk lands, the call's stream
// sketches it as a row shard with its global row offset (S A = sum over the
// shards of S_k A_k, the hash evaluated at global row indices: Section 2's S
// applied block by block), adding its S_k A_k and S_k b_k to SA and Sb in chunk
// order.  When the last chunk is in, the preconditioner, the start and the
// LSQR iterations run on the full device copy, and x is copied back.
#include <algorithm>
#include <vector>

#include "cw_common.cuh"
#include "cw_internal.h"

namespace cw {
namespace {

constexpr int kHostChunks = 8;

// The copy stream and its events; on leaving the call the call's stream first
// waits for every copy, so the device buffers are released after them.
struct CopyLane {
    cudaStream_t call = nullptr;
    cudaStream_t copy = nullptr;
    cudaEvent_t ready = nullptr;               // the buffers exist
    std::vector<cudaEvent_t> landed;           // chunk k is on the device
    cudaEvent_t all = nullptr;                 // every copy issued so far is done
    ~CopyLane() {
        if (copy) {
            if (all && cudaEventRecord(all, copy) == cudaSuccess) cudaStreamWaitEvent(call, all, 0);
            cudaStreamDestroy(copy);
        }
        for (cudaEvent_t e : landed)
            if (e) cudaEventDestroy(e);
        if (ready) cudaEventDestroy(ready);
        if (all) cudaEventDestroy(all);
        (void)cudaGetLastError();
    }
};

}  // namespace
}  // namespace cw

using namespace cw;

extern "C" int cw_lsqr_precond_host(const cw_csr* A, const float* b, int64_t m, uint64_t seed, double rtol,
                                    int32_t max_iter, double* x, int32_t* iters, double* final_test,
                                    cw_stream stream) {
    if (!A || !b || !x) return CW_ERR_ARG;
    if (!(rtol > 0.0) || max_iter < 0) return CW_ERR_ARG;
    int st = validate_common(A->n, A->d, m);
    if (st != CW_OK) return st;
    if (A->d < 1 || A->d > 1024 || A->d > m) return CW_ERR_SHAPE;
    if (A->nnz < 0 || A->nnz > 0x7FFFFFFFll) return CW_ERR_OVERFLOW;
    if (!A->row_ptr || (A->nnz > 0 && (!A->col || !A->val))) return CW_ERR_ARG;
    const int64_t n = A->n, nnz = A->nnz, d = A->d;
    if (A->row_ptr[0] != 0 || (int64_t)A->row_ptr[n] != nnz) return CW_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;

    Scratch ws(s);
    const size_t oRp = ws.reserve(sizeof(int32_t) * (size_t)(n + 1));
    const size_t oCol = ws.reserve(sizeof(int32_t) * (size_t)std::max<int64_t>(nnz, 1));
    const size_t oVal = ws.reserve(sizeof(float) * (size_t)std::max<int64_t>(nnz, 1));
    const size_t oB = ws.reserve(sizeof(float) * (size_t)std::max<int64_t>(n, 1));
    const size_t oSA = ws.reserve(sizeof(float) * (size_t)m * (size_t)d);
    const size_t oSb = ws.reserve(sizeof(float) * (size_t)m);
    const size_t oX = ws.reserve(sizeof(double) * (size_t)d);
    CW_CUDA_TRY(ws.alloc());
    int32_t* rp_d = ws.at<int32_t>(oRp);
    int32_t* col_d = ws.at<int32_t>(oCol);
    float* val_d = ws.at<float>(oVal);
    float* b_d = ws.at<float>(oB);
    float* SA = ws.at<float>(oSA);
    float* Sb = ws.at<float>(oSb);
    double* x_d = ws.at<double>(oX);

    // row chunks of about equal nonzero count; their nonzero ranges partition
    // [0, nnz) even when row_ptr is not monotone (the kernels flag that)
    const int K = n > 0 ? (int)std::min<int64_t>(kHostChunks, n) : 0;
    std::vector<int64_t> r(K + 1, 0), z(K + 1, 0);
    for (int k = 1; k < K; ++k) {
        const int64_t target = nnz * k / K;
        int64_t lo = r[k - 1] + 1, hi = n - (K - k);  // at least one row per chunk
        while (lo < hi) {
            const int64_t mid = (lo + hi) / 2;
            if ((int64_t)A->row_ptr[mid] < target) lo = mid + 1; else hi = mid;
        }
        r[k] = lo;
        z[k] = std::min<int64_t>(nnz, std::max<int64_t>(z[k - 1], (int64_t)A->row_ptr[lo]));
    }
    if (K > 0) {
        r[K] = n;
        z[K] = nnz;
    }

    CopyLane lane;
    lane.call = s;
    CW_CUDA_TRY(cudaStreamCreateWithFlags(&lane.copy, cudaStreamNonBlocking));
    CW_CUDA_TRY(cudaEventCreateWithFlags(&lane.ready, cudaEventDisableTiming));
    CW_CUDA_TRY(cudaEventCreateWithFlags(&lane.all, cudaEventDisableTiming));
    lane.landed.assign((size_t)K, nullptr);
    for (int k = 0; k < K; ++k) CW_CUDA_TRY(cudaEventCreateWithFlags(&lane.landed[k], cudaEventDisableTiming));
    CW_CUDA_TRY(cudaEventRecord(lane.ready, s));
    CW_CUDA_TRY(cudaStreamWaitEvent(lane.copy, lane.ready, 0));
    for (int k = 0; k < K; ++k) {
        const int64_t r0 = r[k], r1 = r[k + 1];
        CW_CUDA_TRY(cudaMemcpyAsync(rp_d + r0, A->row_ptr + r0, sizeof(int32_t) * (size_t)(r1 - r0 + 1),
                                    cudaMemcpyHostToDevice, lane.copy));
        CW_CUDA_TRY(cudaMemcpyAsync(b_d + r0, b + r0, sizeof(float) * (size_t)(r1 - r0), cudaMemcpyHostToDevice,
                                    lane.copy));
        if (z[k + 1] > z[k]) {
            const size_t cnt = (size_t)(z[k + 1] - z[k]);
            CW_CUDA_TRY(cudaMemcpyAsync(col_d + z[k], A->col + z[k], sizeof(int32_t) * cnt, cudaMemcpyHostToDevice,
                                        lane.copy));
            CW_CUDA_TRY(cudaMemcpyAsync(val_d + z[k], A->val + z[k], sizeof(float) * cnt, cudaMemcpyHostToDevice,
                                        lane.copy));
        }
        CW_CUDA_TRY(cudaEventRecord(lane.landed[k], lane.copy));
    }
    if (K == 0) CW_CUDA_TRY(cudaMemcpyAsync(rp_d, A->row_ptr, sizeof(int32_t), cudaMemcpyHostToDevice, lane.copy));
    CW_CUDA_TRY(cudaEventRecord(lane.all, lane.copy));

    // sketch each chunk as it lands: chunk 0 writes SA and Sb, the others add
    for (int k = 0; k < K; ++k) {
        CW_CUDA_TRY(cudaStreamWaitEvent(s, lane.landed[k], 0));
        st = sketch_impl(kSketchCSR, r[k + 1] - r[k], d, 0, r[k], rp_d + r[k], col_d, val_d, nullptr, b_d + r[k], m,
                         seed, SA, Sb, nullptr, s, nullptr, nullptr, nullptr, nullptr, k > 0);
        if (st != CW_OK) return st;
    }
    CW_CUDA_TRY(cudaStreamWaitEvent(s, lane.all, 0));
    const cw_csr Ad{n, d, nnz, rp_d, col_d, val_d};
    st = lsqr_run(&Ad, b_d, m, seed, rtol, max_iter, x_d, iters, final_test, s, K > 0 ? SA : nullptr,
                  K > 0 ? Sb : nullptr);
    if (st != CW_OK && st != CW_ERR_NOCONV) return st;
    CW_CUDA_TRY(cudaMemcpyAsync(x, x_d, sizeof(double) * (size_t)d, cudaMemcpyDeviceToHost, s));
    CW_CUDA_TRY(cudaStreamSynchronize(s));
    return st;
}
