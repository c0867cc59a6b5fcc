// Least squares by LSQR (Paige and Saunders, 1982) on the preconditioned
// operator y -> A M y with M = R^-1, R from the sketch SA (Section 7.6 of the
// paper: a CG-like method on A R, whose condition number is at most
// (1+e0)^2/(1-e0)^2 for an e0-subspace embedding; Theorem "it reg").
//
// Per iteration one fused pass streams A once (rows in natural order):
//     z_i = (A vhat)_i - coef * z_i          (vhat = M v, float32)
//     ||z||^2 and A^T z                      (per-CTA partials, fixed order)
// which gives both halves of the Golub-Kahan step: beta u = A M v - alpha u
// and A^T u = A^T z / beta.  A cooperative kernel on 32 CTAs then finishes
// the step (M^T A^T u in two-word float32, alpha, the plane rotation, y, w and
// the stopping tests in float64, the next vhat).  The loop runs in batches on
// the device; the host reads the done flag once per batch.
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
#include "lsqr_pass.cuh"

namespace cw {

struct PostArgs {
    const float2* gpart;
    const double* zpart;
    const double* bpart;  // first step only
    int nblk;
    int d;
    const float* M32T;    // M = R^-1 (float32 values), column-major: M32T[j * d + i] = M_ij
    const double* M;      // the same values, float64 row-major
    const double* y0;     // R x0
    double* v;
    double* w;
    double* dy;
    float* vhat;          // out: M v (float32)
    LsqrState* st;
    double rtol;
    int max_iter;
    int first;
};

// One LSQR step on P CTAs (one cooperative launch, three bounded grid
// barriers), CTA c owning the columns [c * per, (c + 1) * per) of every
// length-d vector:
//   1. g_j = sum over pass blocks of the two-word partials (A^T z)_j;
//   2. t_j = (M^T g)_j (two-word products and sums), gv_j = s t_j - beta v_j,
//      and the CTA's share of ||gv||^2;
//   3. alpha from the shares (every CTA adds them in the same order), the
//      plane rotation from the state (every CTA alike), v, w, dy, and the
//      share of ||y0 + dy||^2;
//   4. CTA 0 updates the state; vhat_i = (M v)_i in float32 for the CTA's rows.
// Every sum has a fixed order, so the results are the same in every run.
struct PostMcArgs {
    PostArgs p;
    float2* gsum;       // d: g as (hi, lo)
    double* tv;         // d: gv
    double* share;      // [2][P]: shares of ||gv||^2 and ||y||^2
    unsigned* bar;      // grid barrier words (zero at the first launch)
    unsigned* tflag;    // set when a barrier wait gave up
};

__device__ __forceinline__ void two_add(float& hi, float& lo, float xh, float xl) {
    const float t = __fadd_rn(hi, xh);
    const float bp = __fsub_rn(t, hi);
    lo = __fadd_rn(lo, __fadd_rn(__fadd_rn(__fsub_rn(hi, __fsub_rn(t, bp)), __fsub_rn(xh, bp)), xl));
    hi = t;
}

// sum of x[0..cnt) in float64 in a fixed order, the same value on every lane
__device__ __forceinline__ double warp_sum_fixed(const double* x, int cnt, int lane) {
    double v = 0.0;
    for (int k = lane; k < cnt; k += 32) v += __ldcg(x + k);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    return v;
}

__global__ void __launch_bounds__(256) k_lsqr_post_mc(PostMcArgs a) {
    const PostArgs& q = a.p;
    LsqrState* st = q.st;
    if (st->done || *reinterpret_cast<volatile unsigned*>(a.tflag)) return;
    const int d = q.d, P = gridDim.x, cta = blockIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    const int per = (d + P - 1) / P, j0 = cta * per, j1 = min(d, j0 + per);
    __shared__ double s_sc[8], s_a2;
    __shared__ double s_col[32];
    __shared__ float vf[1024];

    // 1. g for the CTA's columns (warp per column, lanes over the pass blocks)
    for (int j = j0 + warp; j < j1; j += nwarp) {
        float hi = 0.f, lo = 0.f;
        for (int b0 = lane; b0 < q.nblk; b0 += 32 * 8) {   // blocks b0, b0 + 32, ... (loads ahead of the adds)
            float2 x[8];
#pragma unroll
            for (int u = 0; u < 8; ++u)
                x[u] = b0 + 32 * u < q.nblk ? __ldg(q.gpart + (size_t)(b0 + 32 * u) * d + j) : make_float2(0.f, 0.f);
#pragma unroll
            for (int u = 0; u < 8; ++u)
                if (b0 + 32 * u < q.nblk) two_add(hi, lo, x[u].x, x[u].y);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float oh = __shfl_xor_sync(0xFFFFFFFFu, hi, o);
            const float ol = __shfl_xor_sync(0xFFFFFFFFu, lo, o);
            two_add(hi, lo, oh, ol);
        }
        if (lane == 0) a.gsum[j] = make_float2(hi, lo);
    }
    // ||z||^2 (and ||b||^2 on the first step): every CTA the same sums
    // (beta and its reciprocal formed by one thread: float64 square roots and
    // divisions are long sequences on this part)
    __shared__ double s_beta[2];
    if (warp == 0) {
        const double zz = warp_sum_fixed(q.zpart, q.nblk, lane);
        const double bb = q.first ? warp_sum_fixed(q.bpart, q.nblk, lane) : 0.0;
        if (lane == 0) {
            s_sc[6] = zz;
            s_sc[7] = bb;
            const double be = sqrt(zz);
            s_beta[0] = be;
            s_beta[1] = be > 0.0 ? (q.first ? -1.0 / be : 1.0 / be) : 0.0;
        }
    }
    if (!grid_barrier(a.bar, (unsigned)P, a.tflag)) return;
    const double beta = s_beta[0];
    const double s_new = s_beta[1];

    // 2. t = M^T g for the CTA's columns (warp per column, lanes over rows i <= j)
    for (int j = j0 + warp; j < j1; j += nwarp) {
        const float* mcol = q.M32T + (size_t)j * d;
        float sh = 0.f, sl = 0.f;
        for (int i0 = lane; i0 <= j; i0 += 32 * 4) {   // rows i0, i0 + 32, ... (loads ahead of the adds)
            float m[4];
            float2 g[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const bool ok = i0 + 32 * u <= j;
                m[u] = ok ? __ldg(mcol + i0 + 32 * u) : 0.f;
                g[u] = ok ? __ldcg(a.gsum + i0 + 32 * u) : make_float2(0.f, 0.f);
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                if (i0 + 32 * u > j) break;
                const float p = __fmul_rn(m[u], g[u].x);
                float e = fmaf(m[u], g[u].x, -p);
                e = fmaf(m[u], g[u].y, e);
                two_add(sh, sl, p, e);
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float oh = __shfl_xor_sync(0xFFFFFFFFu, sh, o);
            const float ol = __shfl_xor_sync(0xFFFFFFFFu, sl, o);
            two_add(sh, sl, oh, ol);
        }
        if (lane == 0) {
            double gv = s_new * ((double)sh + (double)sl);
            if (!q.first) gv -= beta * q.v[j];
            a.tv[j] = gv;
            s_col[j - j0] = gv * gv;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double loc = 0.0;
        for (int j = j0; j < j1; ++j) loc += s_col[j - j0];
        a.share[cta] = loc;
    }
    if (!grid_barrier(a.bar, (unsigned)P, a.tflag)) return;

    // 3. alpha, the rotation, the vector updates for the CTA's columns
    if (warp == 0) {
        const double t = warp_sum_fixed(a.share, P, lane);
        if (lane == 0) s_a2 = sqrt(t);
    }
    __syncthreads();
    const double alpha = s_a2;
    if (q.first) {
        for (int j = j0 + threadIdx.x; j < j1; j += blockDim.x) {
            const double vj = alpha > 0.0 ? a.tv[j] / alpha : 0.0;
            q.v[j] = vj;
            q.w[j] = vj;
            q.dy[j] = 0.0;
        }
    } else {
        if (threadIdx.x == 0) {
            const double alpha_old = st->alpha;
            const double anorm2 = st->anorm2 + alpha_old * alpha_old + beta * beta;
            const double rho = hypot(st->rhobar, beta);
            const double c = st->rhobar / rho, sn = beta / rho;
            const double rinv = 1.0 / rho;
            s_sc[0] = c * st->phibar * rinv;   // phi / rho
            s_sc[1] = sn * alpha * rinv;       // theta / rho
            s_sc[2] = alpha > 0.0 ? 1.0 / alpha : 0.0;
            s_sc[3] = anorm2;
            s_sc[4] = c;
            s_sc[5] = sn * st->phibar;         // phibar
        }
        __syncthreads();
        const double k_dy = s_sc[0], k_w = s_sc[1], ainv = s_sc[2];
        for (int j = j0 + threadIdx.x; j < j1; j += blockDim.x) {
            const double vj = a.tv[j] * ainv;
            const double wj = q.w[j];
            const double dyj = fma(k_dy, wj, q.dy[j]);
            q.dy[j] = dyj;
            q.w[j] = fma(-k_w, wj, vj);
            q.v[j] = vj;
            const double yj = q.y0[j] + dyj;
            s_col[j - j0] = yj * yj;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            double yl = 0.0;
            for (int j = j0; j < j1; ++j) yl += s_col[j - j0];
            a.share[P + cta] = yl;
        }
    }
    if (!grid_barrier(a.bar, (unsigned)P, a.tflag)) return;

    // 4. the state (CTA 0) and vhat = M v for the CTA's rows
    if (cta == 0 && warp == 0) {
        const double ynorm = q.first ? 0.0 : sqrt(warp_sum_fixed(a.share + P, P, lane));
        if (lane == 0) {
            if (q.first) {
                st->bnorm = sqrt(s_sc[7]);
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
                } else if (q.max_iter <= 0) {
                    st->done = 1;
                }
            } else {
                const double anorm2 = s_sc[3], c = s_sc[4], phibar = s_sc[5];
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
                const bool conv = test2 <= q.rtol || rnorm <= q.rtol * (st->bnorm + anorm * ynorm) || beta == 0.0 ||
                                  alpha == 0.0;
                if (conv) {
                    st->converged = 1;
                    st->done = 1;
                } else if (st->iters >= q.max_iter) {
                    st->done = 1;
                }
            }
        }
    }
    if (j0 >= j1) return;
    for (int j = j0 + threadIdx.x; j < d; j += blockDim.x) vf[j] = (float)__ldcg(q.v + j);
    __syncthreads();
    // row i: lanes over j >= i (M row-major float64 holds the float32 values), fixed tree
    for (int i = j0 + warp; i < j1; i += nwarp) {
        const double* mrow = q.M + (size_t)i * d;
        float s0 = 0.f;
        for (int jb = i + lane; jb < d; jb += 32 * 4) {   // columns jb, jb + 32, ... (loads ahead of the FMAs)
            double mv[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) mv[u] = jb + 32 * u < d ? __ldg(mrow + jb + 32 * u) : 0.0;
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (jb + 32 * u < d) s0 = fmaf((float)mv[u], vf[jb + 32 * u], s0);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s0 += __shfl_xor_sync(0xFFFFFFFFu, s0, o);
        if (lane == 0) q.vhat[i] = s0;
    }
}

// MT = float32 transpose of M (column-major copy); M itself is rounded to the
// same float32 values so that every use of the preconditioner agrees.
__global__ void k_to_f32_transposed(double* __restrict__ M, int d, float* __restrict__ MT) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q < (int64_t)d * d) {
        const int i = (int)(q / d), j = (int)(q % d);
        const float v = (float)M[q];
        MT[(size_t)j * d + i] = v;
        M[q] = (double)v;
    }
}

// y = add + R x (R upper triangular, float64 row-major): one warp per row,
// lane l taking columns i + l, i + 32 + l, ..., then a fixed shuffle tree.
// Rows spread over many SMs: float64 issues slowly on this part.
__global__ void __launch_bounds__(256) k_upper_matvec(const double* __restrict__ R, int d,
                                                     const double* __restrict__ x, double* __restrict__ y,
                                                     const double* __restrict__ add) {
    const int lane = threadIdx.x & 31;
    const int i = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if (i >= d) return;
    double s = 0.0;
    for (int j = i + lane; j < d; j += 32) s = fma(R[(size_t)i * d + j], x[j], s);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xFFFFFFFFu, s, o);
    if (lane == 0) y[i] = (add ? add[i] : 0.0) + s;
}

// The start of the iteration in one launch: x0 = M c (the sketch-and-solve
// solution, computed as k_upper_matvec does), vhat = x0 in float32 (the first
// pass's input) and y0 = c (= R x0).
__global__ void __launch_bounds__(256) k_lsqr_start(const double* __restrict__ M, int d,
                                                   const double* __restrict__ c, double* __restrict__ x0,
                                                   float* __restrict__ vhat, double* __restrict__ y0) {
    const int lane = threadIdx.x & 31;
    const int i = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if (i >= d) return;
    double s = 0.0;
    for (int j = i + lane; j < d; j += 32) s = fma(M[(size_t)i * d + j], c[j], s);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xFFFFFFFFu, s, o);
    if (lane == 0) {
        const double v = 0.0 + s;
        x0[i] = v;
        vhat[i] = (float)v;
        y0[i] = c[i];
    }
}

}  // namespace cw

namespace cw {

// The preconditioned LSQR of cw_lsqr_precond; with SA_in / Sb_in given (device,
// the sketch of A and b with `seed`, already formed), the sketch step is skipped.
int lsqr_run(const cw_csr* A, const float* b, int64_t m, uint64_t seed, double rtol, int32_t max_iter, double* x,
             int32_t* iters, double* final_test, cudaStream_t stream, const float* SA_in, const float* Sb_in) {
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
    const int grid = nsm;
    // warps per CTA: the most (from 24, 16, 12, 8, 4) whose vhat + eight
    // accumulator copies of d floats per warp fit in shared memory; 24 warps
    // measured fastest at d = 256 (more leave too little L1 for the loads in flight)
    const int dpad = ((d + 31) & ~31) + 1;
    auto pass_bytes = [&](int w) { return sizeof(float) * (size_t)dpad * (1 + 8 * (size_t)w); };
    int pass_warps = 4;
    for (int w : {24, 16, 12, 8})
        if (pass_bytes(w) <= 220 * 1024) {
            pass_warps = w;
            break;
        }
    const int threads = pass_warps * 32;
    const size_t pass_smem = pass_bytes(pass_warps);
    if (pass_smem > 227 * 1024) return CW_ERR_SHAPE;

    Scratch ws(stream);
    const bool given = SA_in && Sb_in;
    const size_t oSA = given ? 0 : ws.reserve(sizeof(float) * (size_t)m * d);
    const size_t oSb = given ? 0 : ws.reserve(sizeof(float) * (size_t)m);
    const size_t oR = ws.reserve(sizeof(double) * (size_t)d * d);
    const size_t oM = ws.reserve(sizeof(double) * (size_t)d * d);
    const size_t oM32 = ws.reserve(sizeof(float) * (size_t)d * d);
    const size_t oc = ws.reserve(sizeof(double) * (size_t)d);
    const size_t ox0 = ws.reserve(sizeof(double) * (size_t)d);
    const size_t oy0 = ws.reserve(sizeof(double) * (size_t)d);
    const size_t ov = ws.reserve(sizeof(double) * (size_t)d);
    const size_t ow = ws.reserve(sizeof(double) * (size_t)d);
    const size_t ody = ws.reserve(sizeof(double) * (size_t)d);
    const size_t ovh = ws.reserve(sizeof(float) * (size_t)d);
    const size_t oz = ws.reserve(sizeof(float) * (size_t)(n > 0 ? n : 1));
    const size_t ogp = ws.reserve(sizeof(float2) * (size_t)grid * d);
    const size_t ozp = ws.reserve(sizeof(double) * (size_t)grid);
    const size_t obp = ws.reserve(sizeof(double) * (size_t)grid);
    const size_t ost = ws.reserve(sizeof(LsqrState));
    const size_t ogf = ws.reserve(16);   // the Cholesky route's flags
    const size_t opb = ws.reserve(16);   // the LSQR step's grid barrier and its timeout flag
    const size_t ogs = ws.reserve(sizeof(float2) * (size_t)d);
    const size_t otv = ws.reserve(sizeof(double) * (size_t)d);
    const size_t osh = ws.reserve(sizeof(double) * 2 * (size_t)(nsm > 0 ? nsm : 1));
    CW_CUDA_TRY(ws.alloc());
    float* SA = given ? const_cast<float*>(SA_in) : ws.at<float>(oSA);
    float* Sb = given ? const_cast<float*>(Sb_in) : ws.at<float>(oSb);
    double* R = ws.at<double>(oR);
    double* M = ws.at<double>(oM);
    float* M32T = ws.at<float>(oM32);
    double* c = ws.at<double>(oc);
    double* x0 = ws.at<double>(ox0);
    double* y0 = ws.at<double>(oy0);
    float* vhat = ws.at<float>(ovh);
    float* z = ws.at<float>(oz);
    LsqrState* state = ws.at<LsqrState>(ost);

    if (!given) {
        st = sketch_impl(kSketchCSR, n, d, 0, 0, A->row_ptr, A->col, A->val, nullptr, b, m, seed, SA, Sb, nullptr,
                         stream);
        if (st != CW_OK) return st;
    }
    // preconditioner M = R^-1: R from the Cholesky factor of the Gram matrix of
    // SA (one shared-memory kernel), or from the float64 Householder QR of SA
    // when the Cholesky route is not safe (large diagonal ratio, a failed
    // pivot, or d too large for the shared-memory kernel).  c = Q^T Sb.  The
    // Cholesky route's flags are read back with the first LSQR state, after
    // the first batch of iterations has been queued; if they reject it, the
    // iterations are redone from the QR preconditioner.
    unsigned* gflags = ws.at<unsigned>(ogf);
    CW_CUDA_TRY(cudaMemsetAsync(gflags, 0, 16, stream));
    float klb = 0.f;
    st = gram_chol_inverse(SA, m, d, Sb, M, M32T, c, &klb, stream, gflags);
    if (st != CW_OK && st != CW_ERR_SHAPE) return st;
    bool precond_checked = st != CW_OK;   // CW_ERR_SHAPE: straight to the QR route
    auto qr_precond = [&]() -> int {
        int r = qr64(SA, m, d, Sb, R, c, stream);
        if (r != CW_OK) return r;
        r = tri_inverse(R, d, M, stream);
        if (r != CW_OK) return r;
        const int64_t dd0 = (int64_t)d * d;
        {
            CW_PROF("k_to_f32_transposed", stream);
            k_to_f32_transposed<<<(unsigned)((dd0 + 255) / 256), 256, 0, stream>>>(M, d, M32T);
        }
        CW_LAUNCH_CHECK();
        return CW_OK;
    };
    if (precond_checked) {
        st = qr_precond();
        if (st != CW_OK) return st;
    }
    auto pk = pass_warps == 24   ? k_lsqr_pass<24>
              : pass_warps == 16 ? k_lsqr_pass<16>
              : pass_warps == 12 ? k_lsqr_pass<12>
              : pass_warps == 8  ? k_lsqr_pass<8>
                                 : k_lsqr_pass<4>;
    CW_CUDA_TRY(cudaFuncSetAttribute(pk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pass_smem));
    PassArgs pa{};
    PostArgs qa{};
    // the LSQR step on P CTAs (cooperative), each owning at most 32 columns
    const int post_P = std::min(nsm, (d + 7) / 8);
    if ((d + post_P - 1) / post_P > 32) return CW_ERR_SHAPE;
    unsigned* pbar = ws.at<unsigned>(opb);   // [0, 1] barrier, [2] barrier wait gave up
    auto post = [&]() -> int {
        PostMcArgs qm{qa, ws.at<float2>(ogs), ws.at<double>(otv), ws.at<double>(osh), pbar, pbar + 2};
        void* args[] = {&qm};
        CW_PROF("k_lsqr_post_mc", stream);
        CW_CUDA_TRY(cudaLaunchCooperativeKernel((void*)k_lsqr_post_mc, dim3((unsigned)post_P), dim3(256), args, 0,
                                                stream));
        CW_LAUNCH_CHECK();
        return CW_OK;
    };
    // from M and c: the start x0 = M c, the first pass (z = A x0 - b) and the
    // first post step (LSQR's initial bidiagonalisation)
    auto start = [&]() -> int {
        CW_CUDA_TRY(cudaMemsetAsync(state, 0, sizeof(LsqrState), stream));
        {
            CW_PROF("k_lsqr_start", stream);  // x0 = M c, vhat = x0 (float32), y0 = c
            k_lsqr_start<<<(d + 7) / 8, 256, 0, stream>>>(M, d, c, x0, vhat, y0);
        }
        CW_LAUNCH_CHECK();
        pa = PassArgs{A->row_ptr, A->col, A->val, vhat, b, z, ws.at<float2>(ogp), ws.at<double>(ozp),
                      ws.at<double>(obp), nullptr, status, n, d, dpad, 1.0f};
        {
            CW_PROF("k_lsqr_pass", stream);
            pk<<<grid, threads, pass_smem, stream>>>(pa);  // z = A x0 - b
        }
        CW_LAUNCH_CHECK();
        qa = PostArgs{ws.at<float2>(ogp), ws.at<double>(ozp), ws.at<double>(obp), grid, d, M32T, M, y0,
                      ws.at<double>(ov), ws.at<double>(ow), ws.at<double>(ody), vhat, state, rtol,
                      max_iter, 1};
        CW_CUDA_TRY(cudaMemsetAsync(pbar, 0, 16, stream));
        int r = post();
        if (r != CW_OK) return r;
        pa.zin = z;
        pa.st = state;
        pa.bpart = nullptr;
        qa.first = 0;
        qa.bpart = nullptr;
        return CW_OK;
    };
    st = start();
    if (st != CW_OK) return st;
    // iterations in batches of four: each pass and post step returns at once
    // when the state says done, so a batch may run past convergence at the
    // cost of a few empty launches; the host reads the state between batches.
    // x = x0 + M dy is queued behind every batch, before the state is read, so
    // a call that converges within a batch waits on the device only once (a
    // later batch overwrites x).
    struct Flags {
        unsigned rank, timeout;
        float klb, pad;
    };
    LsqrState hs{};
    Flags hf{};
    int launched = 0;
    const int batch = 4;
    for (;;) {
        const int nb = (max_iter - launched) < batch ? (max_iter - launched) : batch;
        for (int q = 0; q < nb; ++q) {
            {
                CW_PROF("k_lsqr_pass", stream);
                pk<<<grid, threads, pass_smem, stream>>>(pa);
            }
            st = post();
            if (st != CW_OK) return st;
        }
        {
            CW_PROF("k_upper_matvec", stream);
            k_upper_matvec<<<(d + 7) / 8, 256, 0, stream>>>(M, d, ws.at<double>(ody), x, x0);
        }
        CW_LAUNCH_CHECK();
        launched += nb;
        unsigned ptimeout = 0;
        CW_CUDA_TRY(cudaMemcpyAsync(&hs, state, sizeof(LsqrState), cudaMemcpyDeviceToHost, stream));
        CW_CUDA_TRY(cudaMemcpyAsync(&ptimeout, pbar + 2, sizeof(unsigned), cudaMemcpyDeviceToHost, stream));
        if (!precond_checked)
            CW_CUDA_TRY(cudaMemcpyAsync(&hf, gflags, sizeof(Flags), cudaMemcpyDeviceToHost, stream));
        CW_CUDA_TRY(cudaStreamSynchronize(stream));
        if (ptimeout) return CW_ERR_TIMEOUT;
        if (!precond_checked) {
            precond_checked = true;
            if (hf.timeout) return CW_ERR_TIMEOUT;
            if (hf.rank || !(hf.klb <= 300.f)) {   // redo from the QR preconditioner
                st = qr_precond();
                if (st != CW_OK) return st;
                st = start();
                if (st != CW_OK) return st;
                launched = 0;
                continue;
            }
        }
        if (hs.done || launched >= max_iter) break;
    }
    if (iters) *iters = hs.iters;
    if (final_test) *final_test = hs.test2;
    return hs.converged ? CW_OK : CW_ERR_NOCONV;
}

}  // namespace cw

using namespace cw;

extern "C" int cw_lsqr_precond(const cw_csr* A, const float* b, int64_t m, uint64_t seed, double rtol,
                               int32_t max_iter, double* x, int32_t* iters, double* final_test, cw_stream stream) {
    return lsqr_run(A, b, m, seed, rtol, max_iter, x, iters, final_test, (cudaStream_t)stream, nullptr, nullptr);
}
