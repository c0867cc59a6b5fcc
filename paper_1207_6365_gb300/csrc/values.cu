// Sketches with given values at the hash positions, and their backward.
//
// S(v) has the single entry of column i at row h(i) (the bucket map of
// Section 2) with value v_i instead of the sign sigma(i); S(sigma) is the
// sparse embedding itself.  SA(v) = S(v) A and Sb(v) = S(v) b are linear in v:
//   SA(v)[k, :] = sum over i with h(i) = k of v_i A_i,   Sb(v)[k] = sum v_i b_i,
// so for a loss L with gradients G = dL/dSA (m x d) and g = dL/dSb (m),
//   dL/dv_i = <G[h(i), :], A_i> + g[h(i)] b_i,
// a gather of the gradient rows of each row's bucket.  The backward kernels
// stream over the rows of A (one pass, each output written once, no atomics),
// recomputing h(i) from the same bucket polynomial as the forward sort.
#include <cmath>

#include "cw_common.cuh"
#include "cw_internal.h"

namespace cw {

// Buckets of rows r0 + lane (lane < 32) for a warp's 32-row group.
__device__ __forceinline__ int group_bucket(const HashParams& hp, int64_t r0, int64_t n, int lane) {
    return r0 + lane < n ? (int)bucket_of(horner61(hp.cb, (uint64_t)(r0 + lane)), hp) : 0;
}

// Dense A: a warp per 32-row group; for each row the warp forms
// <G[h(i), :], A_i> over its columns (16-byte loads when allowed) and reduces
// across lanes.
__global__ void __launch_bounds__(256) k_values_backward_dense(HashParams hp, const float* __restrict__ A, int64_t n,
                                                               int d, int64_t lda, const float* __restrict__ b,
                                                               const float* __restrict__ gSA,
                                                               const float* __restrict__ gSb, float* __restrict__ gv,
                                                               int vec4) {
    const int lane = threadIdx.x & 31;
    const int64_t wglobal = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t grp = wglobal; grp * 32 < n; grp += nwarps) {
        const int64_t r0 = grp * 32;
        const int bk_l = group_bucket(hp, r0, n, lane);
        const int nr = (n - r0) < 32 ? (int)(n - r0) : 32;
        for (int t = 0; t < nr; ++t) {
            const int64_t r = r0 + t;
            const int bk = __shfl_sync(0xFFFFFFFFu, bk_l, t);
            const float* ar = A + r * lda;
            const float* gr = gSA + (int64_t)bk * d;
            float acc = 0.f;
            if (vec4) {
                for (int c = lane * 4; c < d; c += 128) {
                    const float4 x = __ldg(reinterpret_cast<const float4*>(ar + c));
                    const float4 y = __ldg(reinterpret_cast<const float4*>(gr + c));
                    acc = fmaf(x.x, y.x, acc);
                    acc = fmaf(x.y, y.y, acc);
                    acc = fmaf(x.z, y.z, acc);
                    acc = fmaf(x.w, y.w, acc);
                }
            } else {
                for (int c = lane; c < d; c += 32) acc = fmaf(__ldg(ar + c), __ldg(gr + c), acc);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xFFFFFFFFu, acc, o);
            if (lane == 0) {
                if (gSb && b) acc = fmaf(__ldg(gSb + bk), __ldg(b + r), acc);
                gv[r] = acc;
            }
        }
    }
}

// CSR A: a half-warp per row (two rows at a time); lanes take the row's
// nonzeros k, k + 16, ... and gather G[h(i), col_k].
__global__ void __launch_bounds__(256) k_values_backward_csr(HashParams hp, const int32_t* __restrict__ row_ptr,
                                                             const int32_t* __restrict__ col,
                                                             const float* __restrict__ val, int64_t n, int d,
                                                             const float* __restrict__ b,
                                                             const float* __restrict__ gSA,
                                                             const float* __restrict__ gSb, float* __restrict__ gv,
                                                             unsigned* status) {
    const int lane = threadIdx.x & 31, half = lane >> 4, hl = lane & 15;
    const int64_t wglobal = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t grp = wglobal; grp * 32 < n; grp += nwarps) {
        const int64_t r0 = grp * 32;
        const int bk_l = group_bucket(hp, r0, n, lane);
        const int nr = (n - r0) < 32 ? (int)(n - r0) : 32;
        for (int t0 = 0; t0 < nr; t0 += 2) {
            const int t = t0 + half;
            const int bk = __shfl_sync(0xFFFFFFFFu, bk_l, t & 31);
            float acc = 0.f;
            if (t < nr) {
                const int64_t r = r0 + t;
                const int s = __ldg(row_ptr + r), e = __ldg(row_ptr + r + 1);
                const float* gr = gSA + (int64_t)bk * d;
                for (int k = s + hl; k < e; k += 16) {
                    const int c = __ldg(col + k);
                    if ((unsigned)c < (unsigned)d) acc = fmaf(__ldg(val + k), __ldg(gr + c), acc);
                    else flag_error(status, kDevBadColumn);
                }
            }
#pragma unroll
            for (int o = 8; o > 0; o >>= 1) acc += __shfl_xor_sync(0xFFFFFFFFu, acc, o);
            if (hl == 0 && t < nr) {
                const int64_t r = r0 + t;
                if (gSb && b) acc = fmaf(__ldg(gSb + bk), __ldg(b + r), acc);
                gv[r] = acc;
            }
        }
    }
}

namespace {

int grid_for(int64_t n) {
    const int64_t groups = (n + 31) / 32;
    const int64_t blocks = (groups + 7) / 8;
    const int64_t cap = (int64_t)num_sms() * 8;
    return (int)std::max<int64_t>(1, std::min(blocks, cap));
}

}  // namespace

}  // namespace cw

using namespace cw;

extern "C" int cw_sketch_csr_values(const cw_csr* A, const float* b, int64_t m, uint64_t seed, const float* v,
                                    float* SA, float* Sb, cw_stream stream) {
    if (!A || !SA) return CW_ERR_ARG;
    int st = validate_common(A->n, A->d, m);
    if (st != CW_OK) return st;
    if (A->d < 1) return CW_ERR_SHAPE;
    if (A->nnz < 0 || A->nnz > 0x7FFFFFFFll) return CW_ERR_OVERFLOW;
    if (A->n > 0 && (!v || !A->row_ptr || (A->nnz > 0 && (!A->col || !A->val)))) return CW_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (A->n == 0) {
        CW_CUDA_TRY(cudaMemsetAsync(SA, 0, sizeof(float) * (size_t)m * (size_t)A->d, s));
        if (b && Sb) CW_CUDA_TRY(cudaMemsetAsync(Sb, 0, sizeof(float) * (size_t)m, s));
        return CW_OK;
    }
    st = sketch_impl(kSketchCSR, A->n, A->d, 0, 0, A->row_ptr, A->col, A->val, nullptr, nullptr, m, seed, SA,
                     nullptr, nullptr, s, nullptr, nullptr, nullptr, v);
    if (st != CW_OK || !b || !Sb) return st;
    return sketch_impl(kSketchVec, A->n, 0, 0, 0, nullptr, nullptr, nullptr, nullptr, b, m, seed, nullptr, Sb,
                       nullptr, s, nullptr, nullptr, nullptr, v);
}

extern "C" int cw_sketch_dense_values(const float* A, int64_t n, int64_t d, int64_t lda, const float* b, int64_t m,
                                      uint64_t seed, const float* v, float* SA, float* Sb, cw_stream stream) {
    if (!SA || (n > 0 && (!A || !v))) return CW_ERR_ARG;
    int st = validate_common(n, d, m);
    if (st != CW_OK) return st;
    if (d < 1 || lda < d) return CW_ERR_SHAPE;
    return sketch_impl(kSketchDense, n, d, lda, 0, nullptr, nullptr, nullptr, A, b, m, seed, SA, b ? Sb : nullptr,
                       nullptr, (cudaStream_t)stream, nullptr, nullptr, nullptr, v);
}

extern "C" int cw_sketch_values_backward_csr(const cw_csr* A, const float* b, int64_t m, uint64_t seed,
                                             const float* gSA, const float* gSb, float* gv, cw_stream stream) {
    if (!A || !gSA || !gv) return CW_ERR_ARG;
    int st = validate_common(A->n, A->d, m);
    if (st != CW_OK) return st;
    if (A->d < 1) return CW_ERR_SHAPE;
    if (A->nnz < 0 || A->nnz > 0x7FFFFFFFll) return CW_ERR_OVERFLOW;
    if (A->n > 0 && (!A->row_ptr || (A->nnz > 0 && (!A->col || !A->val)))) return CW_ERR_ARG;
    if (A->n == 0) return CW_OK;
    unsigned* status = device_status_word();
    if (!status) return CW_ERR_CUDA;
    const HashParams hp = make_hash_params(seed, m);
    cudaStream_t s = (cudaStream_t)stream;
    {
        CW_PROF("k_values_backward_csr", s);
        k_values_backward_csr<<<grid_for(A->n), 256, 0, s>>>(hp, A->row_ptr, A->col, A->val, A->n, (int)A->d, b, gSA,
                                                              gSb, gv, status);
    }
    CW_LAUNCH_CHECK();
    return CW_OK;
}

extern "C" int cw_sketch_values_backward_dense(const float* A, int64_t n, int64_t d, int64_t lda, const float* b,
                                               int64_t m, uint64_t seed, const float* gSA, const float* gSb,
                                               float* gv, cw_stream stream) {
    if (!gSA || !gv || (n > 0 && !A)) return CW_ERR_ARG;
    int st = validate_common(n, d, m);
    if (st != CW_OK) return st;
    if (d < 1 || lda < d) return CW_ERR_SHAPE;
    if (n == 0) return CW_OK;
    const HashParams hp = make_hash_params(seed, m);
    const int vec4 = (d % 4 == 0) && (lda % 4 == 0) && ((reinterpret_cast<uintptr_t>(A) & 15) == 0) &&
                     ((reinterpret_cast<uintptr_t>(gSA) & 15) == 0);
    cudaStream_t s = (cudaStream_t)stream;
    {
        CW_PROF("k_values_backward_dense", s);
        k_values_backward_dense<<<grid_for(n), 256, 0, s>>>(hp, A, n, (int)d, lda, b, gSA, gSb, gv, vec4);
    }
    CW_LAUNCH_CHECK();
    return CW_OK;
}
