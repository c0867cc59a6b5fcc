// Least squares by LSQR (Paige and Saunders, 1982) on the preconditioned
// operator y -> A M y with M = R^-1, R from the sketch SA (Section 7.6 of the
// paper: a CG-like method on A R, whose condition number is at most
// (1+e0)^2/(1-e0)^2 for an e0-subspace embedding; Theorem "it reg").
//
// Per iteration one fused pass streams A once (rows in natural order):
//     z_i = (A vhat)_i - coef * z_i          (vhat = M v, float32)
//     ||z||^2 and A^T z                      (per-CTA partials, fixed order)
// which gives both halves of the Golub-Kahan step: beta u = A M v - alpha u
// and A^T u = A^T z / beta.  A single-CTA kernel then finishes the step in
// float64 (M^T A^T u, alpha, the plane rotation, y, w, the stopping tests and
// the next vhat).  The loop runs in batches on the device; the host reads the
// done flag once per batch.
//
// R: upper Cholesky factor of the Gram matrix of SA (float32 products, float64
// sums), which makes SA R^-1 orthonormal up to kappa^2 * 2^-24; when the
// diagonal of that R suggests kappa is too large for it, the float64
// Householder R of SA is used instead.  The start x0 is the sketch-and-solve
// solution R^-1 R^-T SA^T Sb (Theorem "lin reg").
#include <cmath>
#include <vector>

#include "cw_common.cuh"
#include "cw_internal.h"

namespace cw {

struct LsqrState {
    double alpha, beta, rhobar, phibar, anorm2, bnorm, s, coef, test2, rnorm;
    int iters, done, converged, pad;
};

struct PassArgs {
    const int32_t* row_ptr;
    const int32_t* col;
    const float* val;
    const float* vhat;     // d
    const float* zin;      // n (z of the previous step, or b for the first pass)
    float* zout;           // n
    double* gpart;         // [grid][d]
    double* zpart;         // [grid]
    double* bpart;         // [grid] (sum of zin^2; first pass only)
    const LsqrState* st;   // coef, done
    unsigned* status;
    int64_t n;
    int d, dpad;
    float coef_first;      // used when st == nullptr
};

template <int LPR, int U>
__global__ void __launch_bounds__(512, 2) k_lsqr_pass(PassArgs a) {
    constexpr int COPIES = 32 / LPR;
    extern __shared__ __align__(16) float sm[];
    if (a.st && a.st->done) return;
    const float coef = a.st ? (float)a.st->coef : a.coef_first;
    const int nwarps = blockDim.x >> 5;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int sub = lane / LPR, sl = lane % LPR;
    const int NS = nwarps * COPIES;
    const int sw = warp * COPIES + sub;
    float* vh = sm;
    float* acc = sm + a.dpad;
    for (int j = threadIdx.x; j < a.d; j += blockDim.x) vh[j] = a.vhat[j];
    for (int q = threadIdx.x; q < NS * a.dpad; q += blockDim.x) acc[q] = 0.f;
    __syncthreads();
    float* myacc = acc + (size_t)sw * a.dpad;

    const int64_t per = (a.n + gridDim.x - 1) / gridDim.x;
    const int64_t r0 = (per * blockIdx.x < a.n) ? per * blockIdx.x : a.n;
    const int64_t r1 = (r0 + per < a.n) ? r0 + per : a.n;
    float zz = 0.f, bb = 0.f;
    for (int64_t base = r0; base < r1; base += (int64_t)NS * U) {
        int st[U], ln[U];
        float zo[U];
        int cc[U];
        float vv[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t r = base + sw + (int64_t)NS * u;
            st[u] = 0;
            ln[u] = 0;
            zo[u] = 0.f;
            if (r < r1) {
                st[u] = __ldg(a.row_ptr + r);
                ln[u] = __ldg(a.row_ptr + r + 1) - st[u];
                zo[u] = __ldg(a.zin + r);
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            cc[u] = 0;
            vv[u] = 0.f;
            if (sl < ln[u]) {
                cc[u] = __ldg(a.col + st[u] + sl);
                vv[u] = __ldg(a.val + st[u] + sl);
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t r = base + sw + (int64_t)NS * u;
            // w_r = sum_k val_k * vhat[col_k]
            float p = 0.f;
            for (int t = sl; t < ln[u]; t += LPR) {
                int c;
                float v;
                if (t == sl) {
                    c = cc[u];
                    v = vv[u];
                } else {
                    c = __ldg(a.col + st[u] + t);
                    v = __ldg(a.val + st[u] + t);
                }
                if ((unsigned)c < (unsigned)a.d)
                    p = fmaf(v, vh[c], p);
                else
                    flag_error(a.status, kDevBadColumn);
            }
#pragma unroll
            for (int o = LPR / 2; o > 0; o >>= 1) p += __shfl_xor_sync(0xFFFFFFFFu, p, o);
            const float z = p - coef * zo[u];
            if (r < r1) {
                if (sl == 0) {
                    a.zout[r] = z;
                    zz = fmaf(z, z, zz);
                    bb = fmaf(zo[u], zo[u], bb);
                }
                // A^T z: this sub-warp's accumulator (distinct columns within a row)
                for (int t = sl; t < ln[u]; t += LPR) {
                    int c;
                    float v;
                    if (t == sl) {
                        c = cc[u];
                        v = vv[u];
                    } else {
                        c = __ldg(a.col + st[u] + t);
                        v = __ldg(a.val + st[u] + t);
                    }
                    if ((unsigned)c < (unsigned)a.d) myacc[c] = fmaf(v, z, myacc[c]);
                }
            }
            __syncwarp();
        }
    }
    __syncthreads();
    // per-CTA partials in float64, sub-warps summed in a fixed order
    for (int j = threadIdx.x; j < a.d; j += blockDim.x) {
        double s = 0.0;
        for (int q = 0; q < NS; ++q) s += (double)acc[(size_t)q * a.dpad + j];
        a.gpart[(size_t)blockIdx.x * a.d + j] = s;
    }
    __shared__ double rz[32], rb[32];
    double zd = (double)zz, bd = (double)bb;
    for (int o = 16; o > 0; o >>= 1) {
        zd += __shfl_xor_sync(0xFFFFFFFFu, zd, o);
        bd += __shfl_xor_sync(0xFFFFFFFFu, bd, o);
    }
    if (lane == 0) {
        rz[warp] = zd;
        rb[warp] = bd;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0, tb = 0.0;
        for (int w = 0; w < nwarps; ++w) {
            t += rz[w];
            tb += rb[w];
        }
        a.zpart[blockIdx.x] = t;
        if (a.bpart) a.bpart[blockIdx.x] = tb;
    }
}

struct PostArgs {
    const double* gpart;
    const double* zpart;
    const double* bpart;  // first step only
    int nblk;
    int d;
    const double* M;      // row-major d x d, upper triangular
    const float* M32T;    // column-major float32 copy of M
    const double* y0;     // R x0
    double* v;
    double* w;
    double* dy;
    double* g;            // scratch d
    float* vhat;          // out: M v (float32)
    LsqrState* st;
    double rtol;
    int max_iter;
    int first;
};

__device__ double block_sum(double v, double* red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double t = 0.0;
    for (int w = 0; w < nw; ++w) t += red[w];  // every thread, same order
    return t;
}

__global__ void __launch_bounds__(1024) k_lsqr_post(PostArgs a) {
    __shared__ double red[32];
    __shared__ double sg[1024];
    __shared__ double sv[1024];
    LsqrState* st = a.st;
    if (st->done) return;
    const int d = a.d;
    // reduce the pass partials (fixed order)
    for (int j = threadIdx.x; j < d; j += blockDim.x) {
        double s = 0.0;
        for (int b = 0; b < a.nblk; ++b) s += a.gpart[(size_t)b * d + j];
        sg[j] = s;
    }
    double zz = 0.0, bb = 0.0;
    for (int b = threadIdx.x; b < a.nblk; b += blockDim.x) {
        zz += a.zpart[b];
        if (a.first) bb += a.bpart[b];
    }
    zz = block_sum(zz, red);
    if (a.first) bb = block_sum(bb, red);
    __syncthreads();
    const double beta = sqrt(zz);
    // scale of u = z * s_new: z = A x0 - b = -r0 on the first step
    const double s_new = beta > 0.0 ? (a.first ? -1.0 / beta : 1.0 / beta) : 0.0;
    // t = M^T (A^T z); gvec = s_new * t - beta * v
    double loc = 0.0;
    for (int j = threadIdx.x; j < d; j += blockDim.x) {
        double t = 0.0;
        for (int i = 0; i <= j; ++i) t += a.M[(size_t)i * d + j] * sg[i];
        double gv = s_new * t;
        if (!a.first) gv -= beta * a.v[j];
        sv[j] = gv;
        loc += gv * gv;
    }
    const double alpha = sqrt(block_sum(loc, red));
    __syncthreads();
    if (a.first) {
        for (int j = threadIdx.x; j < d; j += blockDim.x) {
            const double vj = alpha > 0.0 ? sv[j] / alpha : 0.0;
            a.v[j] = vj;
            a.w[j] = vj;
            a.dy[j] = 0.0;
            sv[j] = vj;
        }
        if (threadIdx.x == 0) {
            st->bnorm = sqrt(bb);
            st->beta = beta;
            st->alpha = alpha;
            st->phibar = beta;
            st->rhobar = alpha;
            st->anorm2 = 0.0;
            st->iters = 0;
            st->rnorm = beta;
            st->s = s_new;
            st->coef = alpha * s_new;
            st->test2 = 1.0;
            if (alpha * beta == 0.0) {
                st->done = 1;
                st->converged = 1;
                st->test2 = 0.0;
            } else if (a.max_iter <= 0) {
                st->done = 1;
            }
        }
    } else {
        const double alpha_old = st->alpha;
        const double anorm2 = st->anorm2 + alpha_old * alpha_old + beta * beta;
        const double rho = hypot(st->rhobar, beta);
        const double c = st->rhobar / rho, sn = beta / rho;
        const double theta = sn * alpha;
        const double phi = c * st->phibar;
        const double phibar = sn * st->phibar;
        double yl = 0.0;
        for (int j = threadIdx.x; j < d; j += blockDim.x) {
            const double vj = alpha > 0.0 ? sv[j] / alpha : 0.0;
            const double wj = a.w[j];
            const double dyj = a.dy[j] + (phi / rho) * wj;
            a.dy[j] = dyj;
            a.w[j] = vj - (theta / rho) * wj;
            a.v[j] = vj;
            sv[j] = vj;
            const double yj = a.y0[j] + dyj;
            yl += yj * yj;
        }
        const double ynorm = sqrt(block_sum(yl, red));
        if (threadIdx.x == 0) {
            const double anorm = sqrt(anorm2);
            const double rnorm = phibar;
            const double arnorm = phibar * alpha * fabs(c);
            const double test2 = rnorm > 0.0 ? arnorm / (anorm * rnorm) : 0.0;
            st->anorm2 = anorm2;
            st->rhobar = -c * alpha;
            st->phibar = phibar;
            st->alpha = alpha;
            st->beta = beta;
            st->s = s_new;
            st->coef = alpha * s_new;
            st->rnorm = rnorm;
            st->test2 = test2;
            st->iters += 1;
            const bool conv = test2 <= a.rtol || rnorm <= a.rtol * (st->bnorm + anorm * ynorm) || beta == 0.0 ||
                              alpha == 0.0;
            if (conv) {
                st->converged = 1;
                st->done = 1;
            } else if (st->iters >= a.max_iter) {
                st->done = 1;
            }
        }
    }
    __syncthreads();
    // next vhat = M v (float32; it feeds the float32 pass)
    for (int i = threadIdx.x; i < d; i += blockDim.x) {
        float s = 0.f;
        for (int j = i; j < d; ++j) s = fmaf(a.M32T[(size_t)j * d + i], (float)sv[j], s);
        a.vhat[i] = s;
    }
}

__global__ void k_to_f32_transposed(const double* __restrict__ M, int d, float* __restrict__ MT,
                                    float* __restrict__ x32, const double* __restrict__ x) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q < (int64_t)d * d) {
        const int i = (int)(q / d), j = (int)(q % d);
        MT[(size_t)j * d + i] = (float)M[q];
    }
    if (q < d && x32) x32[q] = (float)x[q];
}

// y = R x (upper triangular, float64, one thread per row)
__global__ void k_upper_matvec(const double* __restrict__ R, int d, const double* __restrict__ x,
                               double* __restrict__ y, const double* __restrict__ add) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < d; i += gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int j = i; j < d; ++j) s += R[(size_t)i * d + j] * x[j];
        y[i] = (add ? add[i] : 0.0) + s;
    }
}

}  // namespace cw

using namespace cw;

extern "C" int cw_lsqr_precond(const cw_csr* A, const float* b, int64_t m, uint64_t seed, double rtol,
                               int32_t max_iter, double* x, int32_t* iters, double* final_test, cw_stream stream) {
    if (!A || !b || !x) return CW_ERR_ARG;
    if (!(rtol > 0.0) || max_iter < 0) return CW_ERR_ARG;
    int st = validate_common(A->n, A->d, m);
    if (st != CW_OK) return st;
    if (A->d < 1 || A->d > 1024 || A->d > m) return CW_ERR_SHAPE;
    if (A->nnz < 0 || A->nnz > 0x7FFFFFFFll) return CW_ERR_OVERFLOW;
    if (A->n > 0 && (!A->row_ptr || (A->nnz > 0 && (!A->col || !A->val)))) return CW_ERR_ARG;
    unsigned* status = device_status_word();
    if (!status) return CW_ERR_CUDA;
    const int d = (int)A->d;
    const int64_t n = A->n;
    const int nsm = num_sms();
    const int grid = 2 * nsm;
    const int threads = 512;
    const int lpr = 16;
    const int dpad = ((d + 31) & ~31) + 1;
    const int nsub = (threads / 32) * (32 / lpr);

    Scratch ws(stream);
    const size_t oSA = ws.reserve(sizeof(float) * (size_t)m * d);
    const size_t oSb = ws.reserve(sizeof(float) * (size_t)m);
    const size_t oR = ws.reserve(sizeof(double) * (size_t)d * d);
    const size_t oM = ws.reserve(sizeof(double) * (size_t)d * d);
    const size_t oM32 = ws.reserve(sizeof(float) * (size_t)d * d);
    const size_t oc = ws.reserve(sizeof(double) * (size_t)d);
    const size_t ox0 = ws.reserve(sizeof(double) * (size_t)d);
    const size_t oy0 = ws.reserve(sizeof(double) * (size_t)d);
    const size_t ov = ws.reserve(sizeof(double) * (size_t)d);
    const size_t ow = ws.reserve(sizeof(double) * (size_t)d);
    const size_t ody = ws.reserve(sizeof(double) * (size_t)d);
    const size_t og = ws.reserve(sizeof(double) * (size_t)d);
    const size_t ovh = ws.reserve(sizeof(float) * (size_t)d);
    const size_t oz = ws.reserve(sizeof(float) * (size_t)(n > 0 ? n : 1));
    const size_t ogp = ws.reserve(sizeof(double) * (size_t)grid * d);
    const size_t ozp = ws.reserve(sizeof(double) * (size_t)grid);
    const size_t obp = ws.reserve(sizeof(double) * (size_t)grid);
    const size_t ost = ws.reserve(sizeof(LsqrState));
    CW_CUDA_TRY(ws.alloc());
    float* SA = ws.at<float>(oSA);
    float* Sb = ws.at<float>(oSb);
    double* R = ws.at<double>(oR);
    double* M = ws.at<double>(oM);
    float* M32T = ws.at<float>(oM32);
    double* c = ws.at<double>(oc);
    double* x0 = ws.at<double>(ox0);
    double* y0 = ws.at<double>(oy0);
    float* vhat = ws.at<float>(ovh);
    float* z = ws.at<float>(oz);
    LsqrState* state = ws.at<LsqrState>(ost);
    CW_CUDA_TRY(cudaMemsetAsync(state, 0, sizeof(LsqrState), stream));

    st = sketch_impl(kSketchCSR, n, d, 0, 0, A->row_ptr, A->col, A->val, nullptr, b, m, seed, SA, Sb, nullptr,
                     stream);
    if (st != CW_OK) return st;
    // preconditioner R: Cholesky of the Gram matrix, float64 Householder when that is not safe
    bool use_qr = false;
    st = gram_cholesky(SA, m, d, Sb, R, c, stream);
    if (st == CW_ERR_RANK) {
        use_qr = true;
    } else if (st != CW_OK) {
        return st;
    } else {
        std::vector<double> Rh((size_t)d * d);
        CW_CUDA_TRY(cudaMemcpy(Rh.data(), R, sizeof(double) * (size_t)d * d, cudaMemcpyDeviceToHost));
        double mx = 0.0, mn = INFINITY;
        for (int j = 0; j < d; ++j) {
            const double v = fabs(Rh[(size_t)j * d + j]);
            mx = v > mx ? v : mx;
            mn = v < mn ? v : mn;
        }
        // kappa(SA) >= max/min |R_jj|; the Gram route loses kappa^2 * 2^-24
        if (!(mn > 0.0) || mx / mn > 300.0) use_qr = true;
    }
    if (use_qr) {
        st = qr64(SA, m, d, Sb, R, c, stream);
        if (st != CW_OK) return st;
    }
    st = trsv_upper(R, d, c, x0, stream);  // x0 = R^-1 c: sketch-and-solve start
    if (st != CW_OK) return st;
    st = trsm_upper(R, d, nullptr, d, M, stream);  // M = R^-1
    if (st != CW_OK) return st;
    const int64_t dd = (int64_t)d * d;
    {
        CW_PROF("k_to_f32_transposed", stream);
        k_to_f32_transposed<<<(unsigned)((dd + 255) / 256), 256, 0, stream>>>(M, d, M32T, vhat, x0);
    }
    CW_LAUNCH_CHECK();
    {
        CW_PROF("k_upper_matvec", stream);
        k_upper_matvec<<<(d + 127) / 128, 128, 0, stream>>>(R, d, x0, y0, nullptr);
    }
    CW_LAUNCH_CHECK();

    const size_t pass_smem = sizeof(float) * (size_t)dpad * (1 + nsub);
    auto pk = k_lsqr_pass<16, 4>;
    CW_CUDA_TRY(cudaFuncSetAttribute(pk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pass_smem));
    PassArgs pa{A->row_ptr, A->col, A->val, vhat, b, z, ws.at<double>(ogp), ws.at<double>(ozp), ws.at<double>(obp),
                nullptr, status, n, d, dpad, 1.0f};
    {
        CW_PROF("k_lsqr_pass", stream);
        pk<<<grid, threads, pass_smem, stream>>>(pa);  // z = A x0 - b
    }
    CW_LAUNCH_CHECK();
    PostArgs qa{ws.at<double>(ogp), ws.at<double>(ozp), ws.at<double>(obp), grid, d, M, M32T, y0,
                ws.at<double>(ov), ws.at<double>(ow), ws.at<double>(ody), ws.at<double>(og), vhat, state, rtol,
                max_iter, 1};
    {
        CW_PROF("k_lsqr_post", stream);
        k_lsqr_post<<<1, 1024, 0, stream>>>(qa);
    }
    CW_LAUNCH_CHECK();
    pa.zin = z;
    pa.st = state;
    pa.bpart = nullptr;
    qa.first = 0;
    qa.bpart = nullptr;
    LsqrState hs{};
    int launched = 0;
    const int batch = 4;
    for (;;) {
        CW_CUDA_TRY(cudaMemcpyAsync(&hs, state, sizeof(LsqrState), cudaMemcpyDeviceToHost, stream));
        CW_CUDA_TRY(cudaStreamSynchronize(stream));
        if (hs.done || launched >= max_iter) break;
        const int nb = (max_iter - launched) < batch ? (max_iter - launched) : batch;
        for (int q = 0; q < nb; ++q) {
            {
                CW_PROF("k_lsqr_pass", stream);
                pk<<<grid, threads, pass_smem, stream>>>(pa);
            }
            {
                CW_PROF("k_lsqr_post", stream);
                k_lsqr_post<<<1, 1024, 0, stream>>>(qa);
            }
        }
        CW_LAUNCH_CHECK();
        launched += nb;
    }
    // x = x0 + M dy
    {
        CW_PROF("k_upper_matvec", stream);
        k_upper_matvec<<<(d + 127) / 128, 128, 0, stream>>>(M, d, ws.at<double>(ody), x, x0);
    }
    CW_LAUNCH_CHECK();
    CW_CUDA_TRY(cudaStreamSynchronize(stream));
    if (iters) *iters = hs.iters;
    if (final_test) *final_test = hs.test2;
    return hs.converged ? CW_OK : CW_ERR_NOCONV;
}
