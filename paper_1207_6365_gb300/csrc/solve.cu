// Sketch-and-solve least squares (Theorem "lin reg": compute Phi D A and Phi D b,
// output argmin_x ||Phi D A x - Phi D b||), solved as R^-1 Q^T S b with the
// float64 Householder QR of [SA | Sb] (proof of Theorem "renRegAlg").
#include "cw_common.cuh"
#include "cw_internal.h"

namespace cw {

int solve_from_sketch(const float* SA, const float* Sb, int64_t m, int d, double* x, double* R_out,
                             cudaStream_t stream) {
    Scratch ws(stream);
    const size_t oR = R_out ? 0 : ws.reserve(sizeof(double) * (size_t)d * d);
    const size_t oc = ws.reserve(sizeof(double) * (size_t)d);
    CW_CUDA_TRY(ws.alloc());
    double* R = R_out ? R_out : ws.at<double>(oR);
    double* c = ws.at<double>(oc);
    int st = qr64(SA, m, d, Sb, R, c, stream);
    if (st != CW_OK) return st;
    st = trsv_upper(R, d, c, x, stream);
    if (st != CW_OK) return st;
    CW_CUDA_TRY(cudaStreamSynchronize(stream));
    return CW_OK;
}

}  // namespace cw

using namespace cw;

extern "C" int cw_solve_sketch(const cw_csr* A, const float* b, int64_t m, uint64_t seed, double* x, double* R,
                               cw_stream stream) {
    if (!A || !b || !x) return CW_ERR_ARG;
    int st = validate_common(A->n, A->d, m);
    if (st != CW_OK) return st;
    if (A->d < 1 || A->d > 1024 || A->d > m) return CW_ERR_SHAPE;
    if (A->nnz < 0 || A->nnz > 0x7FFFFFFFll) return CW_ERR_OVERFLOW;
    if (A->n > 0 && (!A->row_ptr || (A->nnz > 0 && (!A->col || !A->val)))) return CW_ERR_ARG;
    const int d = (int)A->d;
    Scratch ws(stream);
    const size_t oSA = ws.reserve(sizeof(float) * (size_t)m * d);
    const size_t oSb = ws.reserve(sizeof(float) * (size_t)m);
    CW_CUDA_TRY(ws.alloc());
    float* SA = ws.at<float>(oSA);
    float* Sb = ws.at<float>(oSb);
    st = sketch_impl(kSketchCSR, A->n, d, 0, 0, A->row_ptr, A->col, A->val, nullptr, b, m, seed, SA, Sb, nullptr,
                     stream);
    if (st != CW_OK) return st;
    return solve_from_sketch(SA, Sb, m, d, x, R, stream);
}

extern "C" int cw_solve_sketch_dense(const float* A, int64_t n, int64_t d, int64_t lda, const float* b, int64_t m,
                                     uint64_t seed, double* x, double* R, cw_stream stream) {
    if (!b || !x || (n > 0 && !A)) return CW_ERR_ARG;
    int st = validate_common(n, d, m);
    if (st != CW_OK) return st;
    if (d < 1 || d > 1024 || d > m || lda < d) return CW_ERR_SHAPE;
    Scratch ws(stream);
    const size_t oSA = ws.reserve(sizeof(float) * (size_t)m * d);
    const size_t oSb = ws.reserve(sizeof(float) * (size_t)m);
    CW_CUDA_TRY(ws.alloc());
    float* SA = ws.at<float>(oSA);
    float* Sb = ws.at<float>(oSb);
    st = sketch_impl(kSketchDense, n, d, lda, 0, nullptr, nullptr, nullptr, A, b, m, seed, SA, Sb, nullptr, stream);
    if (st != CW_OK) return st;
    return solve_from_sketch(SA, Sb, m, (int)d, x, R, stream);
}
