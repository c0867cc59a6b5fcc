// Approximate leverage scores (Section 6, Theorem "icml"): with R from the QR
// of SA (S a sparse embedding) and Pi_2 = G / sqrt(k), G ~ N(0,1)^{d x k},
//     u'_i = ||(A R^-1 Pi_2)_i||^2 = ||A_i M||^2 / k,   M = R^-1 G.
// The product A M is never stored: each warp streams rows of A and keeps the k
// outputs of a row in its lanes.
//
// Precision: for an ill-conditioned A the terms A_ij M_jl are many orders of
// magnitude larger than their sum (M carries R^-1), so float32 accumulation
// would lose the result.  Each product is formed exactly in two float32 words
// (fma), M is kept as a float32 pair (hi + lo), and the sum is a compensated
// (two-word) float32 accumulation; only the final squared norms are rounded to
// float32.
#include "cw_common.cuh"
#include "cw_internal.h"

namespace cw {

constexpr int kLevRPW = 4;      // rows per warp in flight
constexpr int kLevJC = 512;     // columns of A (rows of M) per shared-memory chunk
constexpr int kLevWarps = 8;

__global__ void k_split_m(const double* __restrict__ M, int64_t cnt, float* __restrict__ hi, float* __restrict__ lo) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= cnt) return;
    const double v = M[q];
    const float h = (float)v;
    hi[q] = h;
    lo[q] = (float)(v - (double)h);
}

__global__ void __launch_bounds__(kLevWarps * 32) k_leverage(const float* __restrict__ A, int64_t n, int d,
                                                            int64_t lda, const float* __restrict__ Mhi,
                                                            const float* __restrict__ Mlo, int k,
                                                            float* __restrict__ lev) {
    extern __shared__ __align__(16) float sm[];
    float* sMh = sm;                            // [kLevJC][32]
    float* sMl = sMh + kLevJC * 32;             // [kLevJC][32]
    float* sA = sMl + kLevJC * 32;              // [warps][RPW][kLevJC]
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float* myA = sA + (size_t)warp * kLevRPW * kLevJC;
    const int nlc = (k + 31) / 32, njc = (d + kLevJC - 1) / kLevJC;
    const bool resident = (nlc == 1 && njc == 1);

    auto load_m = [&](int lc, int jc) {
        const int j0 = jc * kLevJC;
        for (int q = threadIdx.x; q < kLevJC * 32; q += blockDim.x) {
            const int jj = q / 32, l = q % 32;
            const int j = j0 + jj, col = lc * 32 + l;
            const bool ok = j < d && col < k;
            sMh[q] = ok ? Mhi[(size_t)j * k + col] : 0.f;
            sMl[q] = ok ? Mlo[(size_t)j * k + col] : 0.f;
        }
    };
    if (resident) {
        load_m(0, 0);
        __syncthreads();
    }
    const int64_t rows_per_cta = (int64_t)kLevWarps * kLevRPW;
    for (int64_t g0 = (int64_t)blockIdx.x * rows_per_cta; g0 < n; g0 += (int64_t)gridDim.x * rows_per_cta) {
        const int64_t rw = g0 + (int64_t)warp * kLevRPW;
        float levacc[kLevRPW];
#pragma unroll
        for (int r = 0; r < kLevRPW; ++r) levacc[r] = 0.f;
        for (int lc = 0; lc < nlc; ++lc) {
            float s[kLevRPW], comp[kLevRPW];
#pragma unroll
            for (int r = 0; r < kLevRPW; ++r) {
                s[r] = 0.f;
                comp[r] = 0.f;
            }
            for (int jc = 0; jc < njc; ++jc) {
                const int j0 = jc * kLevJC;
                const int jn = min(kLevJC, d - j0);
                if (!resident) {
                    __syncthreads();
                    load_m(lc, jc);
                    __syncthreads();
                }
#pragma unroll
                for (int r = 0; r < kLevRPW; ++r) {
                    const int64_t row = rw + r;
                    for (int jj = lane; jj < jn; jj += 32)
                        myA[r * kLevJC + jj] = row < n ? __ldg(A + row * lda + j0 + jj) : 0.f;
                }
                __syncwarp();
#pragma unroll 4
                for (int jj = 0; jj < jn; ++jj) {
                    const float mh = sMh[jj * 32 + lane], ml = sMl[jj * 32 + lane];
#pragma unroll
                    for (int r = 0; r < kLevRPW; ++r) {
                        const float a = myA[r * kLevJC + jj];
                        const float p = a * mh;
                        float e = fmaf(a, mh, -p);
                        e = fmaf(a, ml, e);
                        const float t = s[r] + p;
                        const float bp = t - s[r];
                        const float err = (s[r] - (t - bp)) + (p - bp);
                        s[r] = t;
                        comp[r] += err + e;
                    }
                }
                __syncwarp();
            }
#pragma unroll
            for (int r = 0; r < kLevRPW; ++r) {
                const float y = (lc * 32 + lane < k) ? s[r] + comp[r] : 0.f;
                levacc[r] = fmaf(y, y, levacc[r]);
            }
        }
#pragma unroll
        for (int r = 0; r < kLevRPW; ++r) {
            float v = levacc[r];
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
            const int64_t row = rw + r;
            if (lane == 0 && row < n) lev[row] = v / (float)k;
        }
    }
}

}  // namespace cw

using namespace cw;

extern "C" int cw_leverage(const float* A, int64_t n, int64_t d, int64_t lda, int64_t m, uint64_t seed, int32_t k,
                           const double* G, float* lev, cw_stream stream) {
    if (!G || !lev || (n > 0 && !A)) return CW_ERR_ARG;
    int st = validate_common(n, d, m);
    if (st != CW_OK) return st;
    if (d < 1 || d > 1024 || d > m || lda < d || k < 1 || k > 4096) return CW_ERR_SHAPE;
    const int di = (int)d;
    Scratch ws(stream);
    const size_t oSA = ws.reserve(sizeof(double) * (size_t)m * di);
    const size_t oR = ws.reserve(sizeof(double) * (size_t)di * di);
    const size_t oM = ws.reserve(sizeof(double) * (size_t)di * k);
    const size_t oH = ws.reserve(sizeof(float) * (size_t)di * k);
    const size_t oL = ws.reserve(sizeof(float) * (size_t)di * k);
    CW_CUDA_TRY(ws.alloc());
    double* SA64 = ws.at<double>(oSA);
    double* R = ws.at<double>(oR);
    double* M = ws.at<double>(oM);
    float* Mhi = ws.at<float>(oH);
    float* Mlo = ws.at<float>(oL);
    // SA exact to ~2^-48 (two-word sums): R then carries no float32 error of SA,
    // which an ill-conditioned A would amplify by its condition number
    st = sketch_impl(kSketchDense, n, d, lda, 0, nullptr, nullptr, nullptr, A, nullptr, m, seed, nullptr, nullptr,
                     nullptr, stream, SA64);
    if (st != CW_OK) return st;
    st = qr64(nullptr, m, di, nullptr, R, nullptr, stream, SA64);
    if (st != CW_OK) return st;
    st = trsm_upper(R, di, G, k, M, stream);
    if (st != CW_OK) return st;
    const int64_t cnt = (int64_t)di * k;
    {
        CW_PROF("k_split_m", stream);
        k_split_m<<<(unsigned)((cnt + 255) / 256), 256, 0, stream>>>(M, cnt, Mhi, Mlo);
    }
    CW_LAUNCH_CHECK();
    if (n > 0) {
        const size_t smem = sizeof(float) * ((size_t)kLevJC * 32 * 2 + (size_t)kLevWarps * kLevRPW * kLevJC);
        CW_CUDA_TRY(cudaFuncSetAttribute(k_leverage, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        int per = 1;
        CW_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_leverage, kLevWarps * 32, smem));
        const int64_t groups = (n + kLevWarps * kLevRPW - 1) / (kLevWarps * kLevRPW);
        int64_t grid = (int64_t)num_sms() * (per > 0 ? per : 1);
        if (grid > groups) grid = groups;
        {
            CW_PROF("k_leverage", stream);
            k_leverage<<<(unsigned)grid, kLevWarps * 32, smem, stream>>>(A, n, di, lda, Mhi, Mlo, k, lev);
        }
        CW_LAUNCH_CHECK();
    }
    CW_CUDA_TRY(cudaStreamSynchronize(stream));
    return CW_OK;
}
