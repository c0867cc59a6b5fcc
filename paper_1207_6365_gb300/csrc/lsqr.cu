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
    float2* gpart;         // [grid][d] two-word (hi, lo) partial sums of A^T z
    double* zpart;         // [grid]
    double* bpart;         // [grid] (sum of zin^2; first pass only)
    const LsqrState* st;   // coef, done
    unsigned* status;
    int64_t n;
    int d, dpad;
    float coef_first;      // used when st == nullptr
};

constexpr int kPassBatch = 32;     // rows per warp batch (lane l holds row_ptr / z of row l)

// Streaming 16-byte loads that do not allocate in L1 (each nonzero is read
// once per pass; L1 is left to the shared-memory accumulators).
__device__ __forceinline__ int4 ld_stream_i4(const int32_t* p) {
    int4 r;
    asm volatile("ld.global.nc.L1::no_allocate.v4.s32 {%0, %1, %2, %3}, [%4];\n"
                 : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
                 : "l"(p));
    return r;
}
__device__ __forceinline__ float4 ld_stream_f4(const float* p) {
    float4 r;
    asm volatile("ld.global.nc.L1::no_allocate.v4.f32 {%0, %1, %2, %3}, [%4];\n"
                 : "=f"(r.x), "=f"(r.y), "=f"(r.z), "=f"(r.w)
                 : "l"(p));
    return r;
}

// One CTA per SM, kW warps; warp w owns a contiguous block of rows and walks
// it in batches of 32.  Shared memory holds only vhat and eight accumulator
// copies of A^T z per warp, so many warps fit on the SM; nonzeros go straight
// from global memory to registers.
//
// Quad batches (every row starts on a 4-element boundary and has a multiple
// of 4, at most 16, entries): four lanes per row, four entries per lane,
// eight rows per step; all four steps' 16-byte loads are issued before the
// first is used.  Row slot q of a step accumulates into copy q, so no two
// lanes ever update the same address in one instruction and every address is
// updated in program order: the sums are the same in every run.
// Other batches: a half-warp per row (16 lanes, longer rows loop), four rows
// at a time, two accumulator copies.
template <int kW>
__global__ void __launch_bounds__(kW * 32, 1) k_lsqr_pass(PassArgs a) {
    extern __shared__ __align__(16) float sm[];
    if (a.st && a.st->done) return;
    constexpr int LPR = 16, HALVES = 32 / LPR, RPH = kPassBatch / HALVES, COPIES = 8;
    const float coef = a.st ? (float)a.st->coef : a.coef_first;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int sub = lane / LPR, sl = lane % LPR;
    float* vh = sm;                      // [dpad], zero past d
    float* acc = vh + a.dpad;            // [kW][COPIES][dpad]
    const bool vec16 = ((reinterpret_cast<uintptr_t>(a.col) | reinterpret_cast<uintptr_t>(a.val)) & 15) == 0;
    for (int j = threadIdx.x; j < a.dpad; j += blockDim.x) vh[j] = j < a.d ? a.vhat[j] : 0.f;
    for (int q = threadIdx.x; q < kW * COPIES * a.dpad; q += blockDim.x) acc[q] = 0.f;
    __syncthreads();
    float* myacc = acc + (size_t)(warp * COPIES + sub) * a.dpad;
    const int qd = lane >> 2, ql = lane & 3;   // quad batches: row slot, lane in quad
    float* qacc = acc + (size_t)(warp * COPIES + qd) * a.dpad;

    const int64_t nw = (int64_t)gridDim.x * kW;
    const int64_t gw = (int64_t)blockIdx.x * kW + warp;
    const int64_t per = (((a.n + nw - 1) / nw) + kPassBatch - 1) / kPassBatch * kPassBatch;
    const int64_t w0 = gw * per < a.n ? gw * per : a.n;
    const int64_t w1 = w0 + per < a.n ? w0 + per : a.n;
    const int nbatch = (int)((w1 - w0 + kPassBatch - 1) / kPassBatch);

    auto load_meta = [&](int k, int32_t& rp, int32_t& rend, float& zo) {
        rp = 0;
        rend = 0;
        zo = 0.f;
        if (k < nbatch) {
            const int64_t r0 = w0 + (int64_t)k * kPassBatch;
            const int64_t rl = (r0 + kPassBatch < w1) ? r0 + kPassBatch : w1;
            if (r0 + lane < rl) {
                rp = __ldg(a.row_ptr + r0 + lane);
                zo = __ldg(a.zin + r0 + lane);
            }
            rend = __ldg(a.row_ptr + rl);
        }
    };
    int32_t rpA, reA, rpB, reB;
    float zoA, zoB;
    load_meta(0, rpA, reA, zoA);
    float zz = 0.f, bb = 0.f;
    for (int k = 0; k < nbatch; ++k) {
        load_meta(k + 1, rpB, reB, zoB);   // next batch's rows, in flight during this one
        const int64_t r0 = w0 + (int64_t)k * kPassBatch;
        const int nrows = (int)((r0 + kPassBatch < w1 ? r0 + kPassBatch : w1) - r0);
        float zreg = 0.f;
        // every lane takes part in the shuffle and the vote (full masks)
        const int32_t nxt = __shfl_down_sync(0xFFFFFFFFu, rpA, 1);
        const int32_t myl = (lane < nrows) ? ((lane + 1 < nrows) ? nxt : reA) - rpA : 0;
        const bool okq = (lane >= nrows) || (((rpA & 3) == 0) && ((myl & 3) == 0) && myl <= 16);
        const bool quad = __all_sync(0xFFFFFFFFu, okq) && vec16;
        if (quad) {
            int4 c4[4];
            float4 v4[4];
            int lens[4];
            float zolds[4];
#pragma unroll
            for (int step = 0; step < 4; ++step) {
                const int row = step * 8 + qd;
                const int32_t rs = __shfl_sync(0xFFFFFFFFu, rpA, row);
                lens[step] = __shfl_sync(0xFFFFFFFFu, myl, row);
                zolds[step] = __shfl_sync(0xFFFFFFFFu, zoA, row);
                c4[step] = make_int4(0, 0, 0, 0);
                v4[step] = make_float4(0.f, 0.f, 0.f, 0.f);
                if (4 * ql < lens[step]) {
                    c4[step] = ld_stream_i4(a.col + rs + 4 * ql);
                    v4[step] = ld_stream_f4(a.val + rs + 4 * ql);
                }
            }
#pragma unroll
            for (int step = 0; step < 4; ++step) {
                const bool act = 4 * ql < lens[step];
                int4 c = c4[step];
                float4 v = v4[step];
                if (act) {
                    const unsigned cmax = max(max((unsigned)c.x, (unsigned)c.y), max((unsigned)c.z, (unsigned)c.w));
                    if (cmax >= (unsigned)a.d) {
                        flag_error(a.status, kDevBadColumn);
                        c = make_int4(0, 0, 0, 0);
                        v = make_float4(0.f, 0.f, 0.f, 0.f);
                    }
                }
                float p = 0.f;
                if (act) {
                    p = v.x * vh[c.x];
                    p = fmaf(v.y, vh[c.y], p);
                    p = fmaf(v.z, vh[c.z], p);
                    p = fmaf(v.w, vh[c.w], p);
                }
                p += __shfl_xor_sync(0xFFFFFFFFu, p, 1);
                p += __shfl_xor_sync(0xFFFFFFFFu, p, 2);
                const float z = p - coef * zolds[step];
                const float zt = __shfl_sync(0xFFFFFFFFu, z, (lane & 7) * 4);
                if ((lane >> 3) == step) zreg = zt;
                if (act) {
                    qacc[c.x] = fmaf(v.x, z, qacc[c.x]);
                    qacc[c.y] = fmaf(v.y, z, qacc[c.y]);
                    qacc[c.z] = fmaf(v.z, z, qacc[c.z]);
                    qacc[c.w] = fmaf(v.w, z, qacc[c.w]);
                }
                __syncwarp();
            }
        } else {
            // RI rows of this half-warp at a time: independent dot products and
            // reductions interleave; the A^T z updates then go row by row in order
            constexpr int RI = 4;
#pragma unroll 1
            for (int t0 = 0; t0 < RPH; t0 += RI) {
                int32_t rs[RI];
                int len[RI];
                float zold[RI], p[RI];
                int c0[RI];
                float v0[RI];
#pragma unroll
                for (int u = 0; u < RI; ++u) {
                    const int row = sub * RPH + t0 + u;
                    rs[u] = __shfl_sync(0xFFFFFFFFu, rpA, row & 31);
                    len[u] = __shfl_sync(0xFFFFFFFFu, myl, row & 31);
                    zold[u] = __shfl_sync(0xFFFFFFFFu, zoA, row & 31);
                    c0[u] = 0;
                    v0[u] = 0.f;
                    if (sl < len[u]) {
                        c0[u] = __ldg(a.col + rs[u] + sl);
                        v0[u] = __ldg(a.val + rs[u] + sl);
                    }
                }
#pragma unroll
                for (int u = 0; u < RI; ++u) {
                    p[u] = 0.f;
                    if (sl < len[u]) {
                        if ((unsigned)c0[u] < (unsigned)a.d)
                            p[u] = v0[u] * vh[c0[u]];
                        else
                            flag_error(a.status, kDevBadColumn);
                    }
                    for (int q = sl + LPR; q < len[u]; q += LPR) {  // rows longer than LPR
                        const int c = __ldg(a.col + rs[u] + q);
                        const float v = __ldg(a.val + rs[u] + q);
                        if ((unsigned)c < (unsigned)a.d)
                            p[u] = fmaf(v, vh[c], p[u]);
                        else
                            flag_error(a.status, kDevBadColumn);
                    }
                }
#pragma unroll
                for (int o = LPR / 2; o > 0; o >>= 1)
#pragma unroll
                    for (int u = 0; u < RI; ++u) p[u] += __shfl_xor_sync(0xFFFFFFFFu, p[u], o);
#pragma unroll
                for (int u = 0; u < RI; ++u) {
                    const float z = p[u] - coef * zold[u];
                    if (sl == t0 + u) zreg = z;
                    if (sl < len[u] && (unsigned)c0[u] < (unsigned)a.d) myacc[c0[u]] = fmaf(v0[u], z, myacc[c0[u]]);
                    for (int q = sl + LPR; q < len[u]; q += LPR) {
                        const int c = __ldg(a.col + rs[u] + q);
                        const float v = __ldg(a.val + rs[u] + q);
                        if ((unsigned)c < (unsigned)a.d) myacc[c] = fmaf(v, z, myacc[c]);
                    }
                    __syncwarp();
                }
            }
        }
        // quad batches: lane l holds z of row l; others: lane l of half h
        // holds z of row h*RPH + l (l < RPH)
        const int myrow = quad ? lane : sub * RPH + sl;
        if ((quad || sl < RPH) && myrow < nrows) {
            a.zout[r0 + myrow] = zreg;
            zz = fmaf(zreg, zreg, zz);
        }
        if (lane < nrows) bb = fmaf(zoA, zoA, bb);
        rpA = rpB;
        reA = reB;
        zoA = zoB;
    }
    __syncthreads();
    // per-CTA partials: the accumulator copies summed in a fixed order with an
    // exact two-sum (float32 hi + lo), so no float64 pipe work per CTA
    const int NS = kW * COPIES;
    for (int j = threadIdx.x; j < a.d; j += blockDim.x) {
        float hi = 0.f, lo = 0.f;
        for (int q = 0; q < NS; ++q) {
            const float x = acc[(size_t)q * a.dpad + j];
            const float t = hi + x;
            const float bp = t - hi;
            lo += (hi - (t - bp)) + (x - bp);
            hi = t;
        }
        a.gpart[(size_t)blockIdx.x * a.d + j] = make_float2(hi, lo);
    }
    __shared__ double rz[kW], rb[kW];
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
        for (int w = 0; w < kW; ++w) {
            t += rz[w];
            tb += rb[w];
        }
        a.zpart[blockIdx.x] = t;
        if (a.bpart) a.bpart[blockIdx.x] = tb;
    }
}

struct PostArgs {
    const float2* gpart;
    const double* zpart;
    const double* bpart;  // first step only
    int nblk;
    int d;
    const float* M32T;    // M = R^-1 (float32 values), column-major: M32T[j * d + i] = M_ij
    const float* M32P;    // the same, packed by columns: M_ij (i <= j) at j (j + 1) / 2 + i
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

// Sum over the block, the same on every thread and in every run: a shuffle
// tree in each warp (skipped by warps whose values are all zero), then warp 0
// adds the per-warp sums the same way.  float64 issues slowly on this part,
// so only these few warp instructions use it.  red: 33 doubles.
__device__ double block_sum(double v, double* red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    if (__any_sync(0xFFFFFFFFu, v != 0.0))
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    if (lane == 0) red[warp] = v;
    __syncthreads();
    if (warp == 0) {
        double t = lane < nw ? red[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xFFFFFFFFu, t, o);
        if (lane == 0) red[32] = t;
    }
    __syncthreads();
    return red[32];
}

// SMEM_M: the packed triangle of M is copied to shared memory at the start
// (one round of 16-byte copies, overlapped with the partial-sum reduction),
// and both products with M read it from there.
template <bool SMEM_M>
__global__ void __launch_bounds__(1024) k_lsqr_post(PostArgs a) {
    extern __shared__ __align__(16) float Ms[];
    __shared__ double red[33];
    __shared__ double sg[1024];
    __shared__ double sv[1024];
    LsqrState* st = a.st;
    if (st->done) return;
    const int d = a.d;
    if (SMEM_M) {
        const int nq = (d * (d + 1) / 2 + 3) / 4;
        for (int q = threadIdx.x; q < nq; q += blockDim.x) cp_async16(Ms + 4 * q, a.M32P + 4 * q);
        cp_async_commit();
    }
    // reduce the pass partials (two-word sums) -> g = A^T z as float32 (hi, lo)
    // pairs in shared memory: `gp` threads per column, thread g taking blocks
    // g, g + gp, ... in order, eight independent loads in flight (the next
    // eight issued before the current ones are added); the gp sums combined in order
    __shared__ float ghi[1024], glo[1024];
    {
        __shared__ float2 gstripe[1024];
        const int gp = blockDim.x / d >= 4 ? 4 : (blockDim.x / d >= 2 ? 2 : 1);
        constexpr int U = 8;
        for (int tq = threadIdx.x; tq < d * gp; tq += blockDim.x) {
            const int j = tq % d, g = tq / d;
            const int nb = (a.nblk - g + gp - 1) / gp;   // blocks g + gp * t, t < nb
            float hi = 0.f, lo = 0.f;
            float2 cur[U], nxt[U];
#pragma unroll
            for (int u = 0; u < U; ++u)
                cur[u] = u < nb ? a.gpart[(size_t)(g + gp * u) * d + j] : make_float2(0.f, 0.f);
            for (int t0 = 0; t0 < nb; t0 += U) {
#pragma unroll
                for (int u = 0; u < U; ++u)
                    nxt[u] = t0 + U + u < nb ? a.gpart[(size_t)(g + gp * (t0 + U + u)) * d + j] : make_float2(0.f, 0.f);
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    if (t0 + u < nb) {
                        const float t = hi + cur[u].x;
                        const float bp = t - hi;
                        lo += (hi - (t - bp)) + (cur[u].x - bp) + cur[u].y;
                        hi = t;
                    }
                }
#pragma unroll
                for (int u = 0; u < U; ++u) cur[u] = nxt[u];
            }
            gstripe[g * d + j] = make_float2(hi, lo);
        }
        __syncthreads();
        for (int j = threadIdx.x; j < d; j += blockDim.x) {
            float hi = 0.f, lo = 0.f;
            for (int g = 0; g < gp; ++g) {
                const float2 x = gstripe[g * d + j];
                const float t = hi + x.x;
                const float bp = t - hi;
                lo += (hi - (t - bp)) + (x.x - bp) + x.y;
                hi = t;
            }
            ghi[j] = hi;
            glo[j] = lo;
        }
        if (SMEM_M) cp_async_wait_all();
        __syncthreads();
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
    // t = M^T (A^T z): exact float32 products (fma two-product) and two-word
    // sums; one warp per column (columns w, w + 32, ...), lane l taking rows
    // l, l + 32, ... in order, then a fixed shuffle tree of two-word sums
    {
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
        for (int j = warp; j < d; j += nwarp) {
            const float* mcol = SMEM_M ? Ms + j * (j + 1) / 2 : a.M32T + (size_t)j * d;
            float sh = 0.f, sl2 = 0.f;
            for (int i = lane; i <= j; i += 32) {
                const float m = mcol[i];
                const float p = m * ghi[i];
                float e = fmaf(m, ghi[i], -p);
                e = fmaf(m, glo[i], e);
                const float t = sh + p;
                const float bp = t - sh;
                sl2 += (sh - (t - bp)) + (p - bp) + e;
                sh = t;
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const float oh = __shfl_xor_sync(0xFFFFFFFFu, sh, o);
                const float ol = __shfl_xor_sync(0xFFFFFFFFu, sl2, o);
                const float t = sh + oh;
                const float bp = t - sh;
                sl2 += (sh - (t - bp)) + (oh - bp) + ol;
                sh = t;
            }
            if (lane == 0) sv[j] = (double)sh + (double)sl2;
        }
        __syncthreads();
    }
    double loc = 0.0;
    for (int j = threadIdx.x; j < d; j += blockDim.x) {
        double gv = s_new * sv[j];
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
        // the plane rotation and its scalars once (thread 0), then the vector updates
        __shared__ double sc[8];
        if (threadIdx.x == 0) {
            const double alpha_old = st->alpha;
            const double anorm2 = st->anorm2 + alpha_old * alpha_old + beta * beta;
            const double rho = hypot(st->rhobar, beta);
            const double c = st->rhobar / rho, sn = beta / rho;
            const double rinv = 1.0 / rho;
            sc[0] = c * st->phibar * rinv;     // phi / rho
            sc[1] = sn * alpha * rinv;         // theta / rho
            sc[2] = alpha > 0.0 ? 1.0 / alpha : 0.0;
            sc[3] = anorm2;
            sc[4] = c;
            sc[5] = sn * st->phibar;           // phibar
        }
        __syncthreads();
        const double k_dy = sc[0], k_w = sc[1], ainv = sc[2];
        double yl = 0.0;
        for (int j = threadIdx.x; j < d; j += blockDim.x) {
            const double vj = sv[j] * ainv;
            const double wj = a.w[j];
            const double dyj = fma(k_dy, wj, a.dy[j]);
            a.dy[j] = dyj;
            a.w[j] = fma(-k_w, wj, vj);
            a.v[j] = vj;
            sv[j] = vj;
            const double yj = a.y0[j] + dyj;
            yl = fma(yj, yj, yl);
        }
        const double ynorm = sqrt(block_sum(yl, red));
        if (threadIdx.x == 0) {
            const double anorm2 = sc[3], c = sc[4], phibar = sc[5];
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
    {
        // vhat = M v in float32, `gper` threads per row (fixed slices, fixed combine order)
        __shared__ float vf[1024];
        for (int j = threadIdx.x; j < d; j += blockDim.x) vf[j] = (float)sv[j];
        __syncthreads();
        const int gper = blockDim.x / d >= 4 ? 4 : (blockDim.x / d >= 2 ? 2 : 1);
        float* vpart = reinterpret_cast<float*>(sg);  // sg no longer needed
        for (int tq = threadIdx.x; tq < d * gper; tq += blockDim.x) {
            const int i = tq % d, g = tq / d;
            const int len = d - i, lo = i + (int)((int64_t)len * g / gper), hi = i + (int)((int64_t)len * (g + 1) / gper);
            float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
            int j = lo;
            if (SMEM_M) {
                for (; j + 3 < hi; j += 4) {
                    s0 = fmaf(Ms[j * (j + 1) / 2 + i], vf[j], s0);
                    s1 = fmaf(Ms[(j + 1) * (j + 2) / 2 + i], vf[j + 1], s1);
                    s2 = fmaf(Ms[(j + 2) * (j + 3) / 2 + i], vf[j + 2], s2);
                    s3 = fmaf(Ms[(j + 3) * (j + 4) / 2 + i], vf[j + 3], s3);
                }
                for (; j < hi; ++j) s0 = fmaf(Ms[j * (j + 1) / 2 + i], vf[j], s0);
            } else {
                for (; j + 3 < hi; j += 4) {
                    s0 = fmaf(a.M32T[(size_t)j * d + i], vf[j], s0);
                    s1 = fmaf(a.M32T[(size_t)(j + 1) * d + i], vf[j + 1], s1);
                    s2 = fmaf(a.M32T[(size_t)(j + 2) * d + i], vf[j + 2], s2);
                    s3 = fmaf(a.M32T[(size_t)(j + 3) * d + i], vf[j + 3], s3);
                }
                for (; j < hi; ++j) s0 = fmaf(a.M32T[(size_t)j * d + i], vf[j], s0);
            }
            vpart[g * d + i] = (s0 + s1) + (s2 + s3);
        }
        __syncthreads();
        for (int i = threadIdx.x; i < d; i += blockDim.x) {
            float t = 0.f;
            for (int g = 0; g < gper; ++g) t += vpart[g * d + i];
            a.vhat[i] = t;
        }
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

// M32P = the upper triangle of M (float32, column-major M32T) packed by columns.
__global__ void k_pack_upper_f32(const float* __restrict__ M32T, int d, float* __restrict__ M32P) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= (int64_t)d * d) return;
    const int j = (int)(q / d), i = (int)(q % d);
    if (i <= j) M32P[(int64_t)j * (j + 1) / 2 + i] = M32T[q];
}

// y = float32 copy of x (n entries).
__global__ void k_copy_f32(const double* __restrict__ x, int n, float* __restrict__ y) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q < n) y[q] = (float)x[q];
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
    const size_t oSA = ws.reserve(sizeof(float) * (size_t)m * d);
    const size_t oSb = ws.reserve(sizeof(float) * (size_t)m);
    const size_t oR = ws.reserve(sizeof(double) * (size_t)d * d);
    const size_t oM = ws.reserve(sizeof(double) * (size_t)d * d);
    const size_t oM32 = ws.reserve(sizeof(float) * (size_t)d * d);
    const size_t packed_floats = ((size_t)d * (d + 1) / 2 + 3) & ~size_t(3);
    const size_t oM32P = ws.reserve(sizeof(float) * packed_floats);
    const size_t oc = ws.reserve(sizeof(double) * (size_t)d);
    const size_t ox0 = ws.reserve(sizeof(double) * (size_t)d);
    const size_t oy0 = ws.reserve(sizeof(double) * (size_t)d);
    const size_t ov = ws.reserve(sizeof(double) * (size_t)d);
    const size_t ow = ws.reserve(sizeof(double) * (size_t)d);
    const size_t ody = ws.reserve(sizeof(double) * (size_t)d);
    const size_t og = ws.reserve(sizeof(double) * (size_t)d);
    const size_t ovh = ws.reserve(sizeof(float) * (size_t)d);
    const size_t oz = ws.reserve(sizeof(float) * (size_t)(n > 0 ? n : 1));
    const size_t ogp = ws.reserve(sizeof(float2) * (size_t)grid * d);
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
    // preconditioner M = R^-1: R from the Cholesky factor of the Gram matrix of
    // SA (one shared-memory kernel), or from the float64 Householder QR of SA
    // when the Cholesky route is not safe (large diagonal ratio, a failed
    // pivot, or d too large for the shared-memory kernel).  c = Q^T Sb.
    float klb = 0.f;
    st = gram_chol_inverse(SA, m, d, Sb, M, M32T, c, &klb, stream);
    const bool fast_ok = (st == CW_OK) && klb <= 300.f;
    if (st != CW_OK && st != CW_ERR_RANK && st != CW_ERR_SHAPE) return st;
    if (!fast_ok) {
        st = qr64(SA, m, d, Sb, R, c, stream);
        if (st != CW_OK) return st;
        st = tri_inverse(R, d, M, stream);
        if (st != CW_OK) return st;
        const int64_t dd0 = (int64_t)d * d;
        {
            CW_PROF("k_to_f32_transposed", stream);
            k_to_f32_transposed<<<(unsigned)((dd0 + 255) / 256), 256, 0, stream>>>(M, d, M32T);
        }
        CW_LAUNCH_CHECK();
    }
    float* M32P = ws.at<float>(oM32P);
    {
        const int64_t dd1 = (int64_t)d * d;
        CW_PROF("k_pack_upper_f32", stream);
        k_pack_upper_f32<<<(unsigned)((dd1 + 255) / 256), 256, 0, stream>>>(M32T, d, M32P);
    }
    {
        CW_PROF("k_upper_matvec", stream);  // x0 = M c: the sketch-and-solve start
        k_upper_matvec<<<(d + 7) / 8, 256, 0, stream>>>(M, d, c, x0, nullptr);
    }
    CW_LAUNCH_CHECK();
    // first pass input: vhat = x0 (float32); y0 = R x0 = c
    {
        CW_PROF("k_copy_f32", stream);
        k_copy_f32<<<(d + 255) / 256, 256, 0, stream>>>(x0, d, vhat);
    }
    CW_CUDA_TRY(cudaMemcpyAsync(y0, c, sizeof(double) * d, cudaMemcpyDeviceToDevice, stream));
    CW_LAUNCH_CHECK();

    auto pk = pass_warps == 24   ? k_lsqr_pass<24>
              : pass_warps == 16 ? k_lsqr_pass<16>
              : pass_warps == 12 ? k_lsqr_pass<12>
              : pass_warps == 8  ? k_lsqr_pass<8>
                                 : k_lsqr_pass<4>;
    CW_CUDA_TRY(cudaFuncSetAttribute(pk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pass_smem));
    PassArgs pa{A->row_ptr, A->col, A->val, vhat, b, z, ws.at<float2>(ogp), ws.at<double>(ozp), ws.at<double>(obp),
                nullptr, status, n, d, dpad, 1.0f};
    {
        CW_PROF("k_lsqr_pass", stream);
        pk<<<grid, threads, pass_smem, stream>>>(pa);  // z = A x0 - b
    }
    CW_LAUNCH_CHECK();
    // the post kernel keeps the packed triangle of M in shared memory when it fits
    const size_t post_smem = sizeof(float) * packed_floats;
    const bool post_sm = post_smem <= 160 * 1024;
    auto postk = post_sm ? k_lsqr_post<true> : k_lsqr_post<false>;
    if (post_sm)
        CW_CUDA_TRY(cudaFuncSetAttribute(postk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)post_smem));
    const size_t post_dyn = post_sm ? post_smem : 0;
    PostArgs qa{ws.at<float2>(ogp), ws.at<double>(ozp), ws.at<double>(obp), grid, d, M32T, M32P, y0,
                ws.at<double>(ov), ws.at<double>(ow), ws.at<double>(ody), ws.at<double>(og), vhat, state, rtol,
                max_iter, 1};
    {
        CW_PROF("k_lsqr_post", stream);
        postk<<<1, 1024, post_dyn, stream>>>(qa);
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
                postk<<<1, 1024, post_dyn, stream>>>(qa);
            }
        }
        CW_LAUNCH_CHECK();
        launched += nb;
    }
    // x = x0 + M dy
    {
        CW_PROF("k_upper_matvec", stream);
        k_upper_matvec<<<(d + 7) / 8, 256, 0, stream>>>(M, d, ws.at<double>(ody), x, x0);
    }
    CW_LAUNCH_CHECK();
    CW_CUDA_TRY(cudaStreamSynchronize(stream));
    if (iters) *iters = hs.iters;
    if (final_test) *final_test = hs.test2;
    return hs.converged ? CW_OK : CW_ERR_NOCONV;
}
