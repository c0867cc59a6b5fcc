// Training a sketch: the sketched solve, its backward, the exact-solution
// constants of the loss, and values tied per bucket.
//
// Sketch-and-solve (Theorem "lin reg") returns x' = argmin ||M x - y|| for the
// sketched system M = S A (m x d), y = S b, computed as R^-1 Q^T y from the
// Householder QR M = Q R (proof of Theorem "renRegAlg").  Training the values
// of S needs dL/dM and dL/dy for a loss L(x').  With the sketched residual
// r = y - M x' and z = (M^T M)^-1 dL/dx' = R^-1 R^-T dL/dx', differentiating
// the normal equations M^T M x' = M^T y gives
//     dL/dM = r z^T - (M z) x'^T,        dL/dy = M z,
// so the backward costs two triangular solves with R and one pass over M.
//
// The loss judges x' on the full problem: rho^2 - 1 with
//     rho = ||A x' - b|| / ||A x* - b||,   rho^2 - 1 = (x' - x*)^T A^T A (x' - x*) / ||A x* - b||^2
// (the residual of x* is orthogonal to the range of A), so per matrix only the
// bordered Gram matrix G = [A b]^T [A b], x* and ||A x* - b||^2 are kept.  The
// upper Cholesky factor of G is [[R, c], [0, rho*]] with R^T R = A^T A,
// R^T c = A^T b and rho*^2 = ||A x* - b||^2, and x* = R^-1 c: the same numbers
// a QR of [A | b] gives.
//
// Tied values: a sketch whose value at row i is w_{h(i)} sigma(i) (one free
// value per bucket) is diag(w) S, so its sketch of A is the plain sketch with
// row k scaled by w_k, and dL/dw_k = <dL/dM_k, (S A)_k> + dL/dy_k (S b)_k.
#include <algorithm>
#include <cmath>

#include "cw_common.cuh"
#include "cw_internal.h"

namespace cw {
namespace {

constexpr int kLnThreads = 1024;
constexpr int kNsThreads = 512;  // k_normal_solve: a warp per trailing row
constexpr size_t kLnSmemMax = 200 * 1024;

// Upper Cholesky factor of the n x n symmetric W (row-major, upper triangle
// used, overwritten with the factor), one CTA.  bad[0] = first column whose
// pivot is not above 1e-14 of its original diagonal G_kk (left at n when
// none); the last column (b) may end with a zero pivot, b then lying in the
// range of A.
// Thread 0 forms each pivot's square root and reciprocal (float64 square roots
// and divisions are long sequences on this part) and the block reads them.
__device__ void chol_upper_block(double* W, int n, const double* G, int* bad) {
    const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    __shared__ double s_piv[3];
    for (int k = 0; k < n; ++k) {
        if (threadIdx.x == 0) {
            const double piv = W[(int64_t)k * n + k];
            const double tol = k < n - 1 ? 1e-14 * G[(int64_t)k * n + k] : -INFINITY;
            const bool okp = piv > tol;   // also false for NaN
            const double rk = sqrt(piv > 0.0 ? piv : 0.0);
            s_piv[0] = okp ? 1.0 : 0.0;
            s_piv[1] = rk;
            s_piv[2] = rk > 0.0 ? 1.0 / rk : 0.0;
        }
        __syncthreads();
        if (s_piv[0] == 0.0) {
            if (threadIdx.x == 0) *bad = k;
            return;
        }
        const double rk = s_piv[1];
        const double inv = s_piv[2];
        for (int j = k + threadIdx.x; j < n; j += blockDim.x)
            W[(int64_t)k * n + j] = j == k ? rk : W[(int64_t)k * n + j] * inv;
        __syncthreads();
        // trailing update of the upper triangle, W_ij -= R_ki R_kj for
        // k < i <= j: a warp per row i, its lanes along j
        for (int i = k + 1 + (threadIdx.x >> 5); i < n; i += nw) {
            const double rki = W[(int64_t)k * n + i];
            for (int j = i + lane; j < n; j += 32) W[(int64_t)i * n + j] -= rki * W[(int64_t)k * n + j];
        }
        __syncthreads();
    }
}

// x = R^-1 c for the leading d x d block of the n x n factor W (ldw = n),
// c = column d of W; one CTA.  sw (shared, d doubles) is the work vector and
// sx (shared, d doubles) receives x.  Step j: every thread forms x_j from the
// settled sw[j] (unchanged during the step), the owner of j stores it, the
// owners of i < j subtract R_ij x_j: one barrier a step.
// rinv (shared, d doubles) receives the reciprocals of the diagonal first, one
// division per thread in parallel (float64 divisions are long on this part).
__device__ void back_substitute(const double* W, int d, int ldw, const double* c, double* sw, double* sx,
                                double* rinv) {
    for (int i = threadIdx.x; i < d; i += blockDim.x) {
        sw[i] = c[(int64_t)i * ldw];
        rinv[i] = 1.0 / W[(int64_t)i * ldw + i];
    }
    __syncthreads();
    for (int j = d - 1; j >= 0; --j) {
        const double xj = sw[j] * rinv[j];
        for (int i = threadIdx.x; i < d; i += blockDim.x) {
            if (i == j) sx[i] = xj;
            else if (i < j) sw[i] -= W[(int64_t)i * ldw + j] * xj;
        }
        __syncthreads();
    }
}

// x* and ||A x* - b||^2 (and R, when Rout is given) from the bordered Gram
// matrix G ((d+1) x (d+1)).  SMEM: the factor is formed in shared memory
// (n^2 + 3 d doubles), otherwise in the global workspace Wg (n^2 doubles;
// shared memory then holds 3 d doubles).
template <bool SMEM>
__global__ void __launch_bounds__(kLnThreads) k_normal_solve(const double* __restrict__ G, int d, double* Wg,
                                                             double* __restrict__ x, double* __restrict__ r2,
                                                             double* __restrict__ Rout, int* __restrict__ bad) {
    extern __shared__ double sh[];
    const int n = d + 1;
    double* W = SMEM ? sh : Wg;
    double* sx = SMEM ? sh + (size_t)n * n : sh;
    if (threadIdx.x == 0) *bad = n;
    for (int64_t e = threadIdx.x; e < (int64_t)n * n; e += blockDim.x) W[e] = G[e];
    __syncthreads();
    chol_upper_block(W, n, G, bad);
    __syncthreads();
    if (*bad != n) return;
    back_substitute(W, d, n, W + d, sx + d, sx, sx + 2 * d);
    for (int i = threadIdx.x; i < d; i += blockDim.x) x[i] = sx[i];
    if (Rout)
        for (int64_t e = threadIdx.x; e < (int64_t)d * d; e += blockDim.x) {
            const int i = (int)(e / d), j = (int)(e % d);
            Rout[e] = j >= i ? W[(int64_t)i * n + j] : 0.0;
        }
    if (threadIdx.x == 0) {
        const double rr = W[(int64_t)d * n + d];
        *r2 = rr * rr;
    }
}

// loss = e^T G_AA e / r2 and gx = 2 G_AA e / r2 with e = x - x*; one CTA,
// a warp per row of G_AA.  se = shared 2 d + 32 doubles.
__global__ void __launch_bounds__(kLnThreads) k_excess(const double* __restrict__ G, int d,
                                                       const double* __restrict__ xstar,
                                                       const double* __restrict__ r2, const double* __restrict__ x,
                                                       double* __restrict__ loss, double* __restrict__ gx) {
    extern __shared__ double se[];
    double* e = se;
    double* Ge = se + d;
    double* red = se + 2 * d;
    const int ldg = d + 1;
    for (int i = threadIdx.x; i < d; i += blockDim.x) e[i] = x[i] - xstar[i];
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int i = warp; i < d; i += nw) {
        double acc = 0.0;
        for (int j = lane; j < d; j += 32) acc = fma(G[(int64_t)i * ldg + j], e[j], acc);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xFFFFFFFFu, acc, o);
        if (lane == 0) Ge[i] = acc;
    }
    if (threadIdx.x == 0) red[0] = 1.0 / *r2;   // one division for the block
    __syncthreads();
    const double inv = red[0];
    __syncthreads();   // red is reused below
    double part = 0.0;
    for (int i = threadIdx.x; i < d; i += blockDim.x) {
        part = fma(e[i], Ge[i], part);
        if (gx) gx[i] = 2.0 * Ge[i] * inv;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xFFFFFFFFu, part, o);
    if (lane == 0) red[warp] = part;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < nw; ++w) s += red[w];
        *loss = s * inv;
    }
}

// z = R^-1 R^-T g (R upper, row-major d x d); one CTA, shared memory: two
// d-vectors (SMEM: then R, d^2 more doubles, and the reciprocals of its
// diagonal, d more).
template <bool SMEM>
__global__ void __launch_bounds__(kLnThreads) k_gram_inv_apply(const double* __restrict__ Rg, int d,
                                                               const double* __restrict__ g, double* __restrict__ z) {
    extern __shared__ double sz[];
    double* yv = sz + d;
    const double* R = Rg;
    if (SMEM) {
        double* Rs = sz + 2 * d;
        for (int64_t e = threadIdx.x; e < (int64_t)d * d; e += blockDim.x) Rs[e] = Rg[e];
        R = Rs;
    }
    double* rinv = SMEM ? sz + 2 * d + (size_t)d * d : nullptr;
    for (int i = threadIdx.x; i < d; i += blockDim.x) {
        sz[i] = g[i];
        if (SMEM) rinv[i] = 1.0 / R[(int64_t)i * d + i];   // one division per thread, in parallel
    }
    __syncthreads();
    // R^T y = g: forward substitution along the rows of R.  Step j: every
    // thread forms y_j from the settled sz[j] (left unchanged during the
    // step), the owner of entry j stores it in yv, the owners of i > j subtract
    // R_ji y_j from sz[i]: one barrier a step.
    for (int j = 0; j < d; ++j) {
        const double yj = SMEM ? sz[j] * rinv[j] : sz[j] / R[(int64_t)j * d + j];
        for (int i = threadIdx.x; i < d; i += blockDim.x) {
            if (i == j) yv[i] = yj;
            else if (i > j) sz[i] -= R[(int64_t)j * d + i] * yj;
        }
        __syncthreads();
    }
    // R z = y: back substitution along the columns of R, yv the work vector
    // and sz the result
    for (int j = d - 1; j >= 0; --j) {
        const double zj = SMEM ? yv[j] * rinv[j] : yv[j] / R[(int64_t)j * d + j];
        for (int i = threadIdx.x; i < d; i += blockDim.x) {
            if (i == j) sz[i] = zj;
            else if (i < j) yv[i] -= R[(int64_t)i * d + j] * zj;
        }
        __syncthreads();
    }
    for (int i = threadIdx.x; i < d; i += blockDim.x) z[i] = sz[i];
}

// Row i of the backward: r_i = y_i - M_i x, u_i = M_i z (float64 sums),
// gM_i = r_i z^T - u_i x^T, gy_i = u_i; a warp per row, x and z in shared memory.
__global__ void __launch_bounds__(256) k_solve_backward_rows(const float* __restrict__ M, const float* __restrict__ y,
                                                             int64_t m, int d, const double* __restrict__ x,
                                                             const double* __restrict__ z, float* __restrict__ gM,
                                                             float* __restrict__ gy) {
    extern __shared__ double sv[];
    double* sxv = sv;
    double* szv = sv + d;
    for (int i = threadIdx.x; i < d; i += blockDim.x) {
        sxv[i] = x[i];
        szv[i] = z[i];
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = w0; i < m; i += nw) {
        const float* Mi = M + i * d;
        double mx = 0.0, mz = 0.0;
        for (int c = lane; c < d; c += 32) {
            const double a = (double)__ldg(Mi + c);
            mx = fma(a, sxv[c], mx);
            mz = fma(a, szv[c], mz);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            mx += __shfl_xor_sync(0xFFFFFFFFu, mx, o);
            mz += __shfl_xor_sync(0xFFFFFFFFu, mz, o);
        }
        const double r = (double)__ldg(y + i) - mx;
        float* gi = gM + i * d;
        for (int c = lane; c < d; c += 32) gi[c] = (float)(r * szv[c] - mz * sxv[c]);
        if (lane == 0) gy[i] = (float)mz;
    }
}

// M_k = w_k P_k for k < ms, M_k = P_k otherwise (and the same for y from Pb).
__global__ void __launch_bounds__(256) k_scale_rows(const float* __restrict__ P, const float* __restrict__ Pb,
                                                    int64_t m, int d, int64_t ms, const float* __restrict__ w,
                                                    float* __restrict__ M, float* __restrict__ y) {
    const int64_t total = m * d;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += stride) {
        const int64_t k = e / d;
        const float p = __ldg(P + e);
        M[e] = k < ms ? __ldg(w + k) * p : p;
    }
    if (Pb && y)
        for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < m; k += stride) {
            const float p = __ldg(Pb + k);
            y[k] = k < ms ? __ldg(w + k) * p : p;
        }
}

// gw_k = <gM_k, P_k> + gy_k Pb_k for k < ms; a warp per row, float64 sums.
__global__ void __launch_bounds__(256) k_scale_rows_backward(const float* __restrict__ P, const float* __restrict__ Pb,
                                                             int64_t ms, int d, const float* __restrict__ gM,
                                                             const float* __restrict__ gy, float* __restrict__ gw) {
    const int lane = threadIdx.x & 31;
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t k = w0; k < ms; k += nw) {
        double acc = 0.0;
        for (int c = lane; c < d; c += 32) acc = fma((double)__ldg(gM + k * d + c), (double)__ldg(P + k * d + c), acc);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xFFFFFFFFu, acc, o);
        if (lane == 0) {
            if (Pb && gy) acc = fma((double)__ldg(gy + k), (double)__ldg(Pb + k), acc);
            gw[k] = (float)acc;
        }
    }
}

int grid_for(int64_t work, int threads) {
    int64_t g = (work + threads - 1) / threads;
    const int64_t cap = (int64_t)num_sms() * 8;
    if (g > cap) g = cap;
    return (int)(g < 1 ? 1 : g);
}

}  // namespace
}  // namespace cw

using namespace cw;

extern "C" int cw_solve_sketched(const float* SA, const float* Sb, int64_t m, int64_t d, double* x, double* R,
                                 cw_stream stream) {
    if (!SA || !Sb || !x) return CW_ERR_ARG;
    if (d < 1 || d > 1024 || m < d) return CW_ERR_SHAPE;
    if (m > 0x7FFFFFFFll) return CW_ERR_OVERFLOW;
    return solve_from_sketch(SA, Sb, m, (int)d, x, R, (cudaStream_t)stream);
}

extern "C" int cw_solve_sketched_backward(const float* SA, const float* Sb, int64_t m, int64_t d, const double* R,
                                          const double* x, const double* gx, float* gSA, float* gSb,
                                          cw_stream stream) {
    if (!SA || !Sb || !R || !x || !gx || !gSA || !gSb) return CW_ERR_ARG;
    if (d < 1 || d > 1024 || m < d) return CW_ERR_SHAPE;
    if (m > 0x7FFFFFFFll) return CW_ERR_OVERFLOW;
    cudaStream_t s = (cudaStream_t)stream;
    Scratch ws(s);
    const size_t oz = ws.reserve(sizeof(double) * (size_t)d);
    CW_CUDA_TRY(ws.alloc());
    double* z = ws.at<double>(oz);
    const size_t sm = sizeof(double) * (size_t)(3 * d + d * d);
    // one thread per entry of z (fewer warps make the barriers cheaper)
    const int th = (int)std::min<int64_t>(kLnThreads, (d + 31) & ~31ll);
    if (sm <= kLnSmemMax) {
        CW_CUDA_TRY(cudaFuncSetAttribute(k_gram_inv_apply<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        CW_PROF("k_gram_inv_apply", s);
        k_gram_inv_apply<true><<<1, th, sm, s>>>(R, (int)d, gx, z);
    } else {
        CW_PROF("k_gram_inv_apply", s);
        k_gram_inv_apply<false><<<1, th, sizeof(double) * 2 * (size_t)d, s>>>(R, (int)d, gx, z);
    }
    CW_LAUNCH_CHECK();
    {
        CW_PROF("k_solve_backward_rows", s);
        k_solve_backward_rows<<<grid_for(m * 32, 256), 256, sizeof(double) * 2 * (size_t)d, s>>>(SA, Sb, m, (int)d, x, z,
                                                                                                gSA, gSb);
    }
    CW_LAUNCH_CHECK();
    return CW_OK;
}

extern "C" int cw_normal_solve(const double* G, int64_t d, double* x, double* r2, double* R, cw_stream stream) {
    if (!G || !x || !r2) return CW_ERR_ARG;
    if (d < 1 || d > 1024) return CW_ERR_SHAPE;
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t n = d + 1;
    const size_t sm = sizeof(double) * (size_t)(n * n + 3 * d);
    const bool in_smem = sm <= kLnSmemMax;
    Scratch ws(s);
    const size_t oW = in_smem ? 0 : ws.reserve(sizeof(double) * (size_t)(n * n));
    const size_t oB = ws.reserve(sizeof(int));
    CW_CUDA_TRY(ws.alloc());
    int* bad = ws.at<int>(oB);
    if (in_smem) {
        CW_CUDA_TRY(cudaFuncSetAttribute(k_normal_solve<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        CW_PROF("k_normal_solve", s);
        k_normal_solve<true><<<1, kNsThreads, sm, s>>>(G, (int)d, nullptr, x, r2, R, bad);
    } else {
        CW_PROF("k_normal_solve", s);
        k_normal_solve<false><<<1, kNsThreads, sizeof(double) * 3 * (size_t)d, s>>>(G, (int)d, ws.at<double>(oW), x,
                                                                                   r2, R, bad);
    }
    CW_LAUNCH_CHECK();
    int bad_h = 0;
    CW_CUDA_TRY(cudaMemcpyAsync(&bad_h, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
    CW_CUDA_TRY(cudaStreamSynchronize(s));
    return bad_h == (int)n ? CW_OK : CW_ERR_RANK;
}

extern "C" int cw_excess_residual(const double* G, int64_t d, const double* xstar, const double* r2, const double* x,
                                  double* loss, double* gx, cw_stream stream) {
    if (!G || !xstar || !r2 || !x || !loss) return CW_ERR_ARG;
    if (d < 1 || d > 1024) return CW_ERR_SHAPE;
    cudaStream_t s = (cudaStream_t)stream;
    {
        CW_PROF("k_excess", s);
        k_excess<<<1, kLnThreads, sizeof(double) * (2 * (size_t)d + 32), s>>>(G, (int)d, xstar, r2, x, loss, gx);
    }
    CW_LAUNCH_CHECK();
    return CW_OK;
}

extern "C" int cw_scale_rows(const float* P, const float* Pb, int64_t m, int64_t d, int64_t ms, const float* w,
                             float* M, float* y, cw_stream stream) {
    if (!P || !M || (ms > 0 && !w) || (!Pb != !y)) return CW_ERR_ARG;
    if (d < 1 || m < 0 || ms < 0 || ms > m) return CW_ERR_SHAPE;
    if (m * d > 0x7FFFFFFFFFFFll) return CW_ERR_OVERFLOW;
    if (m == 0) return CW_OK;
    cudaStream_t s = (cudaStream_t)stream;
    {
        CW_PROF("k_scale_rows", s);
        k_scale_rows<<<grid_for(m * d, 256), 256, 0, s>>>(P, Pb, m, (int)d, ms, w, M, y);
    }
    CW_LAUNCH_CHECK();
    return CW_OK;
}

extern "C" int cw_scale_rows_backward(const float* P, const float* Pb, int64_t ms, int64_t d, const float* gM,
                                      const float* gy, float* gw, cw_stream stream) {
    if (!P || !gM || !gw || (!Pb != !gy)) return CW_ERR_ARG;
    if (d < 1 || ms < 0) return CW_ERR_SHAPE;
    if (ms * d > 0x7FFFFFFFFFFFll) return CW_ERR_OVERFLOW;
    if (ms == 0) return CW_OK;
    cudaStream_t s = (cudaStream_t)stream;
    {
        CW_PROF("k_scale_rows_backward", s);
        k_scale_rows_backward<<<grid_for(ms * 32, 256), 256, 0, s>>>(P, Pb, ms, (int)d, gM, gy, gw);
    }
    CW_LAUNCH_CHECK();
    return CW_OK;
}
