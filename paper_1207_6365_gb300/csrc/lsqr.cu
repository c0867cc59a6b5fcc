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

constexpr int kPassBatch = 32;     // rows per warp batch (one per lane for row_ptr / z)
constexpr int kPassCap = 640;      // staged nnz per batch (multiple of 4)
constexpr int kPassStages = 2;

// Copies col/val[s, e) into the stage buffers (element base = s & ~3 at offset
// 0).  16-byte copies for whole aligned chunks inside [0, nnz), 4-byte copies
// for the rest.  Every lane of the warp calls this.
// vec16: col and val are 16-byte aligned (scol / sval always are).
__device__ __forceinline__ void stage_nnz(const int32_t* __restrict__ col, const float* __restrict__ val,
                                          int64_t nnz, int64_t s, int64_t e, int32_t* scol, float* sval,
                                          int lane, bool vec16) {
    const int64_t base = s & ~3ll;
    const int64_t end4 = (e + 3) & ~3ll;
    const int64_t nchunk = (end4 - base) >> 2;
    for (int64_t q = lane; q < nchunk; q += 32) {
        const int64_t g = base + 4 * q;
        if (vec16 && g + 4 <= nnz) {
            cp_async16(scol + 4 * q, col + g);
            cp_async16(sval + 4 * q, val + g);
        } else {
            for (int t = 0; t < 4; ++t)
                if (g + t < nnz) {
                    cp_async4(scol + 4 * q + t, col + g + t);
                    cp_async4(sval + 4 * q + t, val + g + t);
                }
        }
    }
}

template <int LPR, int kPassWarps>
__global__ void __launch_bounds__(kPassWarps * 32, 1) k_lsqr_pass(PassArgs a) {
    extern __shared__ __align__(16) float sm[];
    if (a.st && a.st->done) return;
    constexpr int HALVES = 32 / LPR;          // rows processed side by side (scalar path)
    constexpr int RPH = kPassBatch / HALVES;  // rows per sub-warp per batch
    constexpr int COPIES = 8;                 // accumulator copies per warp (quad path: one per row slot)
    static_assert(HALVES <= COPIES, "copies");
    const float coef = a.st ? (float)a.st->coef : a.coef_first;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int sub = lane / LPR, sl = lane % LPR;
    float* vh = sm;                                         // [dpad]
    float* acc = vh + a.dpad;                               // [warps][COPIES][dpad]
    // stage buffers start on a 128-byte boundary (16-byte cp.async targets)
    const size_t stage_off = (((size_t)(1 + kPassWarps * COPIES) * a.dpad * sizeof(float)) + 127) & ~size_t(127);
    int32_t* stage = reinterpret_cast<int32_t*>(reinterpret_cast<char*>(sm) + stage_off);
    const bool vec16 = ((reinterpret_cast<uintptr_t>(a.col) | reinterpret_cast<uintptr_t>(a.val)) & 15) == 0;
    int32_t* wst = stage + (size_t)warp * kPassStages * 2 * (kPassCap + 8);
    for (int j = threadIdx.x; j < a.d; j += blockDim.x) vh[j] = a.vhat[j];
    for (int q = threadIdx.x; q < kPassWarps * COPIES * a.dpad; q += blockDim.x) acc[q] = 0.f;
    __syncthreads();
    float* myacc = acc + (size_t)(warp * COPIES + sub) * a.dpad;
    const int qd = lane >> 2, ql = lane & 3;                // quad path: row slot, lane in quad
    float* qacc = acc + (size_t)(warp * COPIES + qd) * a.dpad;

    // this warp's contiguous rows
    const int64_t nw = (int64_t)gridDim.x * kPassWarps;
    const int64_t gw = (int64_t)blockIdx.x * kPassWarps + warp;
    const int64_t per = (((a.n + nw - 1) / nw) + kPassBatch - 1) / kPassBatch * kPassBatch;
    const int64_t w0 = gw * per < a.n ? gw * per : a.n;
    const int64_t w1 = w0 + per < a.n ? w0 + per : a.n;
    const int64_t nbatch = (w1 - w0 + kPassBatch - 1) / kPassBatch;
    const int64_t nnz = a.row_ptr[a.n];

    // batch registers: lane l holds row_ptr[r0 + l], the batch end, z_in[r0 + l]
    auto load_meta = [&](int64_t k, int32_t& rp, int32_t& rend, float& zo) {
        rp = 0;
        rend = 0;
        zo = 0.f;
        if (k < nbatch) {
            const int64_t r0 = w0 + k * kPassBatch;
            const int64_t r = r0 + lane;
            const int64_t rl = (r0 + kPassBatch < w1) ? r0 + kPassBatch : w1;
            if (r < rl) {
                rp = __ldg(a.row_ptr + r);
                zo = __ldg(a.zin + r);
            }
            rend = __ldg(a.row_ptr + rl);
        }
    };
    auto issue = [&](int64_t k, int32_t rp, int32_t rend) {
        if (k < nbatch) {
            const int32_t s0 = __shfl_sync(0xFFFFFFFFu, rp, 0);
            int32_t* scol = wst + (size_t)(k % kPassStages) * 2 * (kPassCap + 8);
            float* sval = reinterpret_cast<float*>(scol + kPassCap + 8);
            if (rend - s0 <= kPassCap) stage_nnz(a.col, a.val, nnz, s0, rend, scol, sval, lane, vec16);
        }
        cp_async_commit();
    };

    int32_t rpA, reA, rpB, reB, rpC, reC;
    float zoA, zoB, zoC;
    load_meta(0, rpA, reA, zoA);
    load_meta(1, rpB, reB, zoB);
    issue(0, rpA, reA);
    float zz = 0.f, bb = 0.f;
    for (int64_t k = 0; k < nbatch; ++k) {
        load_meta(k + 2, rpC, reC, zoC);
        issue(k + 1, rpB, reB);
        cp_async_wait<1>();
        __syncwarp();
        const int64_t r0 = w0 + k * kPassBatch;
        const int nrows = (int)((r0 + kPassBatch < w1 ? r0 + kPassBatch : w1) - r0);
        const int32_t s0 = __shfl_sync(0xFFFFFFFFu, rpA, 0);
        const bool staged = reA - s0 <= kPassCap;
        const int32_t base = s0 & ~3;
        const int32_t* scol = wst + (size_t)(k % kPassStages) * 2 * (kPassCap + 8);
        const float* sval = reinterpret_cast<const float*>(scol + kPassCap + 8);
        float zreg = 0.f;
        // quad path: every row of the batch starts on a 4-element boundary and
        // has a multiple of 4 (at most 16) entries -> 4 lanes per row, 4 entries
        // per lane from 16-byte shared loads, 8 rows per warp step, row slot q
        // of each step accumulating into copy q (rows in ascending order).
        bool quad = false;
        {
            // every lane takes part in the shuffle and the vote (full masks)
            const int32_t nxt = __shfl_down_sync(0xFFFFFFFFu, rpA, 1);
            const int32_t myl = (lane < nrows) ? ((lane + 1 < nrows) ? nxt : reA) - rpA : 0;
            const bool ok = (lane >= nrows) || (((rpA & 3) == 0) && ((myl & 3) == 0) && myl <= 16);
            quad = __all_sync(0xFFFFFFFFu, ok) && staged && vec16;
        }
        if (quad) {
#pragma unroll 1
            for (int step = 0; step < kPassBatch / 8; ++step) {
                const int row = step * 8 + qd;
                const int32_t rs = __shfl_sync(0xFFFFFFFFu, rpA, row);
                const int32_t rn = __shfl_sync(0xFFFFFFFFu, rpA, (row + 1) & 31);
                const float zold = __shfl_sync(0xFFFFFFFFu, zoA, row);
                const int32_t re = (row + 1 < nrows) ? rn : reA;
                const int len = row < nrows ? re - rs : 0;
                const bool act = 4 * ql < len;
                int4 c4 = make_int4(0, 0, 0, 0);
                float4 v4 = make_float4(0.f, 0.f, 0.f, 0.f);
                if (act) {
                    c4 = *reinterpret_cast<const int4*>(scol + (rs - base) + 4 * ql);
                    v4 = *reinterpret_cast<const float4*>(sval + (rs - base) + 4 * ql);
                    const unsigned cmax = max(max((unsigned)c4.x, (unsigned)c4.y), max((unsigned)c4.z, (unsigned)c4.w));
                    if (cmax >= (unsigned)a.d) {
                        flag_error(a.status, kDevBadColumn);
                        c4 = make_int4(0, 0, 0, 0);
                        v4 = make_float4(0.f, 0.f, 0.f, 0.f);
                    }
                }
                float p = 0.f;
                if (act) {
                    p = v4.x * vh[c4.x];
                    p = fmaf(v4.y, vh[c4.y], p);
                    p = fmaf(v4.z, vh[c4.z], p);
                    p = fmaf(v4.w, vh[c4.w], p);
                }
                p += __shfl_xor_sync(0xFFFFFFFFu, p, 1);
                p += __shfl_xor_sync(0xFFFFFFFFu, p, 2);
                const float z = p - coef * zold;
                const float zt = __shfl_sync(0xFFFFFFFFu, z, (lane & 7) * 4);
                if ((lane >> 3) == step) zreg = zt;
                if (act) {
                    qacc[c4.x] = fmaf(v4.x, z, qacc[c4.x]);
                    qacc[c4.y] = fmaf(v4.y, z, qacc[c4.y]);
                    qacc[c4.z] = fmaf(v4.z, z, qacc[c4.z]);
                    qacc[c4.w] = fmaf(v4.w, z, qacc[c4.w]);
                }
                __syncwarp();
            }
        }
        // scalar path: RI rows of this sub-warp at a time: independent dot
        // products and reductions interleave; the A^T z updates then go row by
        // row in order
        constexpr int RI = 4;
#pragma unroll 1
        for (int t0 = 0; t0 < (quad ? 0 : RPH); t0 += RI) {
            int32_t rs[RI];
            int len[RI];
            float zold[RI], p[RI];
            int c0[RI];
            float v0[RI];
#pragma unroll
            for (int u = 0; u < RI; ++u) {
                const int row = sub * RPH + t0 + u;
                rs[u] = __shfl_sync(0xFFFFFFFFu, rpA, row & 31);
                const int32_t rn = __shfl_sync(0xFFFFFFFFu, rpA, (row + 1) & 31);
                zold[u] = __shfl_sync(0xFFFFFFFFu, zoA, row & 31);
                const int32_t re = (row + 1 < nrows) ? rn : reA;
                len[u] = row < nrows ? re - rs[u] : 0;
                c0[u] = 0;
                v0[u] = 0.f;
                if (sl < len[u]) {
                    if (staged) {
                        c0[u] = scol[rs[u] - base + sl];
                        v0[u] = sval[rs[u] - base + sl];
                    } else {
                        c0[u] = __ldg(a.col + rs[u] + sl);
                        v0[u] = __ldg(a.val + rs[u] + sl);
                    }
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
                    int c;
                    float v;
                    if (staged) {
                        c = scol[rs[u] - base + q];
                        v = sval[rs[u] - base + q];
                    } else {
                        c = __ldg(a.col + rs[u] + q);
                        v = __ldg(a.val + rs[u] + q);
                    }
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
                    int c;
                    float v;
                    if (staged) {
                        c = scol[rs[u] - base + q];
                        v = sval[rs[u] - base + q];
                    } else {
                        c = __ldg(a.col + rs[u] + q);
                        v = __ldg(a.val + rs[u] + q);
                    }
                    if ((unsigned)c < (unsigned)a.d) myacc[c] = fmaf(v, z, myacc[c]);
                }
                __syncwarp();
            }
        }
        // scalar path: lane l of sub-warp h holds z of row h*RPH + l (l < RPH);
        // quad path: lane l holds z of row l
        const int myrow = quad ? lane : sub * RPH + sl;
        if ((quad || sl < RPH) && myrow < nrows) {
            a.zout[r0 + myrow] = zreg;
            zz = fmaf(zreg, zreg, zz);
        }
        if (lane < nrows) bb = fmaf(zoA, zoA, bb);
        __syncwarp();
        rpA = rpB; reA = reB; zoA = zoB;
        rpB = rpC; reB = reC; zoB = zoC;
    }
    cp_async_wait<0>();
    __syncthreads();
    // per-CTA partials: the accumulator copies summed in a fixed order with an
    // exact two-sum (float32 hi + lo), so no float64 pipe work per CTA
    const int NS = kPassWarps * COPIES;
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
    __shared__ double rz[kPassWarps], rb[kPassWarps];
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
        for (int w = 0; w < kPassWarps; ++w) {
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
    // reduce the pass partials (two-word sums) -> g = A^T z as float32 (hi, lo)
    // pairs in shared memory; `gp` threads per column take fixed stripes of
    // blocks, four independent loads in flight, stripes combined in order
    __shared__ float ghi[1024], glo[1024];
    {
        __shared__ float2 gstripe[1024];
        const int gp = blockDim.x / d >= 4 ? 4 : (blockDim.x / d >= 2 ? 2 : 1);
        for (int tq = threadIdx.x; tq < d * gp; tq += blockDim.x) {
            const int j = tq % d, g = tq / d;
            float hi = 0.f, lo = 0.f;
            int b = g;
            for (; b + 3 * gp < a.nblk; b += 4 * gp) {
                float2 x[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) x[u] = a.gpart[(size_t)(b + u * gp) * d + j];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const float t = hi + x[u].x;
                    const float bp = t - hi;
                    lo += (hi - (t - bp)) + (x[u].x - bp) + x[u].y;
                    hi = t;
                }
            }
            for (; b < a.nblk; b += gp) {
                const float2 x = a.gpart[(size_t)b * d + j];
                const float t = hi + x.x;
                const float bp = t - hi;
                lo += (hi - (t - bp)) + (x.x - bp) + x.y;
                hi = t;
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
    // sums; `gper` threads per column over fixed slices, combined in order
    __shared__ float2 tpart[1024];
    {
        const int gper = blockDim.x / d >= 4 ? 4 : (blockDim.x / d >= 2 ? 2 : 1);
        for (int tq = threadIdx.x; tq < d * gper; tq += blockDim.x) {
            const int j = tq % d, g = tq / d;
            const int len = j + 1, lo = (int)((int64_t)len * g / gper), hi = (int)((int64_t)len * (g + 1) / gper);
            const float* mcol = a.M32T + (size_t)j * d;
            float sh = 0.f, sl2 = 0.f;
            int i = lo;
            for (; i < hi; i += 8) {
                float mv[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) mv[u] = (i + u < hi) ? mcol[i + u] : 0.f;
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    if (i + u >= hi) break;
                    const float p = mv[u] * ghi[i + u];
                    float e = fmaf(mv[u], ghi[i + u], -p);
                    e = fmaf(mv[u], glo[i + u], e);
                    const float t = sh + p;
                    const float bp = t - sh;
                    sl2 += (sh - (t - bp)) + (p - bp) + e;
                    sh = t;
                }
            }
            tpart[g * d + j] = make_float2(sh, sl2);
        }
        __syncthreads();
        for (int j = threadIdx.x; j < d; j += blockDim.x) {
            double t = 0.0;
            for (int g = 0; g < gper; ++g) t += (double)tpart[g * d + j].x + (double)tpart[g * d + j].y;
            sv[j] = t;
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
            for (; j + 3 < hi; j += 4) {
                s0 = fmaf(a.M32T[(size_t)j * d + i], vf[j], s0);
                s1 = fmaf(a.M32T[(size_t)(j + 1) * d + i], vf[j + 1], s1);
                s2 = fmaf(a.M32T[(size_t)(j + 2) * d + i], vf[j + 2], s2);
                s3 = fmaf(a.M32T[(size_t)(j + 3) * d + i], vf[j + 3], s3);
            }
            for (; j < hi; ++j) s0 = fmaf(a.M32T[(size_t)j * d + i], vf[j], s0);
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

// y = float32 copy of x (n entries).
__global__ void k_copy_f32(const double* __restrict__ x, int n, float* __restrict__ y) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q < n) y[q] = (float)x[q];
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
    const int grid = nsm;
    // warps per CTA: as many as the per-warp shared memory (8 accumulator
    // copies of d floats + two cp.async stages) allows, from {12, 8, 4}
    const size_t per_warp = sizeof(float) * 8 * (size_t)(((d + 31) & ~31) + 1) +
                            sizeof(int32_t) * kPassStages * 2 * (kPassCap + 8);
    const int fit = (int)((220 * 1024) / per_warp);
    const int pass_warps = fit >= 12 ? 12 : (fit >= 8 ? 8 : 4);
    const int threads = pass_warps * 32;
    const int lpr = 16;
    const int dpad = ((d + 31) & ~31) + 1;
    const int nsub = pass_warps * 8;  // accumulator copies

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
    {
        CW_PROF("k_upper_matvec", stream);  // x0 = M c: the sketch-and-solve start
        k_upper_matvec<<<(d + 127) / 128, 128, 0, stream>>>(M, d, c, x0, nullptr);
    }
    CW_LAUNCH_CHECK();
    // first pass input: vhat = x0 (float32); y0 = R x0 = c
    {
        CW_PROF("k_copy_f32", stream);
        k_copy_f32<<<(d + 255) / 256, 256, 0, stream>>>(x0, d, vhat);
    }
    CW_CUDA_TRY(cudaMemcpyAsync(y0, c, sizeof(double) * d, cudaMemcpyDeviceToDevice, stream));
    CW_LAUNCH_CHECK();

    const size_t pass_smem = ((sizeof(float) * (size_t)dpad * (1 + nsub) + 127) & ~size_t(127)) +
                             sizeof(int32_t) * (size_t)pass_warps * kPassStages * 2 * (kPassCap + 8);
    if (pass_smem > 227 * 1024) return CW_ERR_SHAPE;
    auto pk = pass_warps == 12 ? k_lsqr_pass<16, 12> : (pass_warps == 8 ? k_lsqr_pass<16, 8> : k_lsqr_pass<16, 4>);
    CW_CUDA_TRY(cudaFuncSetAttribute(pk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pass_smem));
    PassArgs pa{A->row_ptr, A->col, A->val, vhat, b, z, ws.at<float2>(ogp), ws.at<double>(ozp), ws.at<double>(obp),
                nullptr, status, n, d, dpad, 1.0f};
    {
        CW_PROF("k_lsqr_pass", stream);
        pk<<<grid, threads, pass_smem, stream>>>(pa);  // z = A x0 - b
    }
    CW_LAUNCH_CHECK();
    PostArgs qa{ws.at<float2>(ogp), ws.at<double>(ozp), ws.at<double>(obp), grid, d, M32T, y0,
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
