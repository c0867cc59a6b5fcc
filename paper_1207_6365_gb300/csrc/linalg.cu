// Small dense linear algebra on the sketch SA (m x d, m >> d):
//
//  * Householder QR of [SA | Sb] in float64 (the solve of the proof of
//    Theorem "renRegAlg": a QR factorisation of SA, then R^-1 Q^T SB).  One
//    persistent cooperative kernel; each CTA owns a contiguous block of rows of
//    the column-major float64 copy and every column step uses three grid-wide
//    barriers (norm -> reflector dots -> update).  Barriers spin with an
//    iteration limit and report CW_ERR_TIMEOUT instead of hanging.
//  * Gram matrix [SA | Sb]^T [SA | Sb] (float32 products, per-chunk float32
//    partial sums combined in float64 in a fixed order) and its Cholesky
//    factor: the fast R used to precondition LSQR, whose quality only needs to
//    be a constant factor (Section 7.6: kappa(R^T A^T A R) <= (1+e0)^2/(1-e0)^2).
//  * Triangular solves and the triangular inverse in float64.
#include <cmath>
#include <cstring>

#include "cw_common.cuh"
#include "cw_internal.h"

namespace cw {

// ---------------------------------------------------------------- bounded grid barrier

constexpr long long kBarrierSpinLimit = 1ll << 24;  // ~1 s with 64 ns sleeps

// bar[0] = arrival count, bar[1] = generation.  Returns false (after flagging
// the status word) when the wait exceeded its limit; the caller must return.
__device__ bool grid_barrier(unsigned* bar, unsigned nblocks, unsigned* timeout_flag) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        ok = 1;
        __threadfence();
        const unsigned gen = atomicAdd(&bar[1], 0u);
        const unsigned arrived = atomicAdd(&bar[0], 1u) + 1u;
        if (arrived == nblocks) {
            atomicExch(&bar[0], 0u);
            __threadfence();
            atomicAdd(&bar[1], 1u);
        } else {
            long long it = 0;
            while (atomicAdd(&bar[1], 0u) == gen) {
                __nanosleep(64);
                if (++it > kBarrierSpinLimit) {
                    atomicExch(timeout_flag, 1u);
                    ok = 0;
                    break;
                }
            }
            if (ok && atomicAdd(timeout_flag, 0u)) ok = 0;
        }
        __threadfence();
    }
    __syncthreads();
    return ok != 0;
}

// ---------------------------------------------------------------- layout conversion

// W (column-major m x nc, float64) <- [SA | Sb] (SA row-major float32).
template <class T>
__global__ void k_to_colmajor64(const T* __restrict__ SA, const float* __restrict__ Sb, int64_t m, int d,
                                int nc, double* __restrict__ W) {
    __shared__ double tile[32][33];
    const int64_t r0 = (int64_t)blockIdx.x * 32;
    const int c0 = blockIdx.y * 32;
    for (int q = threadIdx.y; q < 32; q += blockDim.y) {
        const int64_t r = r0 + q;
        const int c = c0 + threadIdx.x;
        double v = 0.0;
        if (r < m) {
            if (c < d) v = (double)SA[r * d + c];
            else if (c == d && Sb) v = (double)Sb[r];
        }
        tile[q][threadIdx.x] = v;
    }
    __syncthreads();
    for (int q = threadIdx.y; q < 32; q += blockDim.y) {
        const int c = c0 + q;
        const int64_t r = r0 + threadIdx.x;
        if (c < nc && r < m) W[(int64_t)c * m + r] = tile[threadIdx.x][q];
    }
}

// ---------------------------------------------------------------- Householder QR (float64)

struct QrArgs {
    double* W;        // column-major m x nc
    int64_t m;
    int d;            // columns to factor
    int nc;           // d or d + 1 (the last one is carried: c = Q^T Sb)
    double* normp;    // [grid] partial squared norms
    double* dotp;     // [grid][nc] partial reflector dots
    double* wv;       // [nc] tau * (v^T W[:, k])
    unsigned* bar;    // barrier words (2)
    unsigned* tflag;  // timeout flag
};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    return v;
}

__global__ void __launch_bounds__(256) k_qr_householder(QrArgs a) {
    extern __shared__ double sv[];  // this block's reflector entries (rows r0..r1)
    __shared__ double s_red[8];
    const unsigned G = gridDim.x;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
    const int64_t per = (a.m + G - 1) / G;
    const int64_t r0 = (per * blockIdx.x < a.m) ? per * blockIdx.x : a.m;
    const int64_t r1 = (r0 + per < a.m) ? r0 + per : a.m;
    const int64_t rows = r1 - r0;

    // squared norm of column 0 over this block's rows
    {
        double s = 0.0;
        for (int64_t i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
            const double x = a.W[i];
            s += x * x;
        }
        s = warp_sum(s);
        if (lane == 0) s_red[warp] = s;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int w = 0; w < nwarps; ++w) t += s_red[w];
            a.normp[blockIdx.x] = t;
        }
    }
    if (!grid_barrier(a.bar, G, a.tflag)) return;

    for (int j = 0; j < a.d; ++j) {
        // reflector for column j: every block forms the same scalars
        double sig2 = 0.0;
        for (unsigned c = 0; c < G; ++c) sig2 += a.normp[c];  // fixed order
        const double ajj = a.W[(int64_t)j * a.m + j];
        double beta, tau, vscale;
        if (sig2 == 0.0) {
            beta = 0.0;
            tau = 0.0;
            vscale = 0.0;
        } else {
            const double sig = sqrt(sig2);
            beta = ajj >= 0.0 ? -sig : sig;
            tau = (beta - ajj) / beta;
            vscale = 1.0 / (ajj - beta);
        }
        // v for my rows (0 above the diagonal, 1 at it)
        const double* colj = a.W + (int64_t)j * a.m;
        for (int64_t q = threadIdx.x; q < rows; q += blockDim.x) {
            const int64_t i = r0 + q;
            sv[q] = (i < j) ? 0.0 : (i == j ? 1.0 : colj[i] * vscale);
        }
        __syncthreads();
        // partial dots v^T W[:, k] for k > j
        for (int k = j + 1 + warp; k < a.nc; k += nwarps) {
            const double* colk = a.W + (int64_t)k * a.m;
            double s = 0.0;
            for (int64_t q = lane; q < rows; q += 32) s += sv[q] * colk[r0 + q];
            s = warp_sum(s);
            if (lane == 0) a.dotp[(size_t)blockIdx.x * a.nc + k] = s;
        }
        if (!grid_barrier(a.bar, G, a.tflag)) return;
        // distributed reduction over blocks (fixed order)
        for (int k = j + 1 + blockIdx.x * nwarps + warp; k < a.nc; k += G * nwarps) {
            double s = 0.0;
            for (unsigned c = lane; c < G; c += 32) s += a.dotp[(size_t)c * a.nc + k];
            s = warp_sum(s);
            if (lane == 0) a.wv[k] = tau * s;
        }
        if (!grid_barrier(a.bar, G, a.tflag)) return;
        // update W[:, k] -= v * wv[k]; norm of the next column
        double nrm = 0.0;
        for (int k = j + 1 + warp; k < a.nc; k += nwarps) {
            double* colk = a.W + (int64_t)k * a.m;
            const double wk = a.wv[k];
            double s = 0.0;
            for (int64_t q = lane; q < rows; q += 32) {
                const int64_t i = r0 + q;
                double x = colk[i];
                if (i >= j) {
                    x -= sv[q] * wk;
                    colk[i] = x;
                }
                if (k == j + 1 && i >= j + 1) s += x * x;
            }
            if (k == j + 1) nrm = warp_sum(s);
        }
        if (lane == 0) s_red[warp] = nrm;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int w = 0; w < nwarps; ++w) t += s_red[w];
            a.normp[blockIdx.x] = t;
            if (j >= r0 && j < r1) a.W[(int64_t)j * a.m + j] = beta;  // R_jj
        }
        if (!grid_barrier(a.bar, G, a.tflag)) return;
    }
}

// R (row-major d x d, positive diagonal) and c = Q^T Sb from the factored W;
// flags rank deficiency |R_jj| <= d * 2^-52 * max |R_ii|.
__global__ void k_qr_finalize(const double* __restrict__ W, int64_t m, int d, int nc, double* __restrict__ R,
                              double* __restrict__ c, unsigned* rank_flag) {
    __shared__ double dmax;
    if (threadIdx.x == 0) {
        double mx = 0.0;
        for (int j = 0; j < d; ++j) mx = fmax(mx, fabs(W[(int64_t)j * m + j]));
        dmax = mx;
    }
    __syncthreads();
    for (int j = threadIdx.x; j < d; j += blockDim.x) {
        const double rjj = W[(int64_t)j * m + j];
        const double s = rjj < 0.0 ? -1.0 : 1.0;
        if (fabs(rjj) <= (double)d * 2.220446049250313e-16 * dmax) atomicExch(rank_flag, 1u);
        if (R)
            for (int k = 0; k < d; ++k) R[(int64_t)j * d + k] = (k < j) ? 0.0 : s * W[(int64_t)k * m + j];
        if (c && nc > d) c[j] = s * W[(int64_t)d * m + j];
    }
}

// ---------------------------------------------------------------- triangular solves (float64)

// x = R^-1 rhs for upper-triangular row-major R (one CTA, column sweep).
__global__ void k_trsv_upper(const double* __restrict__ R, int d, const double* __restrict__ rhs,
                             double* __restrict__ x) {
    extern __shared__ double sx[];
    for (int i = threadIdx.x; i < d; i += blockDim.x) sx[i] = rhs[i];
    __syncthreads();
    for (int j = d - 1; j >= 0; --j) {
        if (threadIdx.x == 0) sx[j] = sx[j] / R[(int64_t)j * d + j];
        __syncthreads();
        const double xj = sx[j];
        for (int i = threadIdx.x; i < j; i += blockDim.x) sx[i] -= R[(int64_t)i * d + j] * xj;
        __syncthreads();
    }
    for (int i = threadIdx.x; i < d; i += blockDim.x) x[i] = sx[i];
}

// X = R^-1 B for upper-triangular R (d x d) and B (d x k), both row-major; one
// CTA per column of B.
__global__ void k_trsm_upper(const double* __restrict__ R, int d, const double* __restrict__ B, int k,
                             double* __restrict__ X) {
    extern __shared__ double sx[];
    const int col = blockIdx.x;
    for (int i = threadIdx.x; i < d; i += blockDim.x) sx[i] = B ? B[(int64_t)i * k + col] : (i == col ? 1.0 : 0.0);
    __syncthreads();
    for (int j = d - 1; j >= 0; --j) {
        if (threadIdx.x == 0) sx[j] = sx[j] / R[(int64_t)j * d + j];
        __syncthreads();
        const double xj = sx[j];
        if (xj != 0.0)
            for (int i = threadIdx.x; i < j; i += blockDim.x) sx[i] -= R[(int64_t)i * d + j] * xj;
        __syncthreads();
    }
    for (int i = threadIdx.x; i < d; i += blockDim.x) X[(int64_t)i * k + col] = sx[i];
}

// ---- Gram matrix SA^T SA: 128 x 128 output tiles, 8 x 8 per thread ----------
//
// CTA (ti <= tj, chunk) accumulates sum over its rows of SA[r, ti*128 + a] *
// SA[r, tj*128 + b] in float32 and writes a float64 partial tile; partials are
// added over chunks in a fixed order.  The diagonal tiles also accumulate
// SA^T Sb for their columns, tile (0, 0) also Sb^T Sb.

constexpr int kGT = 128;         // tile edge
constexpr int kGK = 16;          // rows per shared-memory stage

__global__ void __launch_bounds__(256) k_gram_tile(const float* __restrict__ SA, const float* __restrict__ Sb,
                                                   int64_t m, int d, int ntile, int rows, double* __restrict__ part,
                                                   double* __restrict__ vpart) {
    __shared__ __align__(16) float As[kGK][kGT + 4];
    __shared__ __align__(16) float Bs[kGK][kGT + 4];
    __shared__ float Ss[kGK];
    int t = blockIdx.x, ti = 0;
    while (t >= ntile - ti) {
        t -= ntile - ti;
        ++ti;
    }
    const int tj = ti + t;
    const int64_t r0 = (int64_t)blockIdx.y * rows;
    const int64_t r1 = (r0 + rows < m) ? r0 + rows : m;
    const int ty = threadIdx.x >> 4, tx = threadIdx.x & 15;
    const bool vec = (d % 4 == 0) && ((reinterpret_cast<uintptr_t>(SA) & 15) == 0);
    float acc[8][8];
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int b = 0; b < 8; ++b) acc[a][b] = 0.f;
    // diagonal tiles also form SA^T Sb for their columns (lanes with tx == 0)
    // and tile (0, 0) forms Sb^T Sb (thread 0)
    const bool vrow = Sb && ti == tj && tx == 0;
    float vacc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    float sbb = 0.f;
    const int ci0 = ti * kGT, cj0 = tj * kGT;
    for (int64_t rb = r0; rb < r1; rb += kGK) {
        if (Sb && ti == tj && threadIdx.x < kGK) Ss[threadIdx.x] = (rb + threadIdx.x < r1) ? Sb[rb + threadIdx.x] : 0.f;
        // stage: 16 rows x 128 columns of each operand; thread loads 2 x 4 floats per operand
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int q = threadIdx.x + 256 * h;   // 0..511 -> (row kk, column quad cq)
            const int kk = q >> 5, cq = (q & 31) * 4;
            const int64_t r = rb + kk;
            float4 va = make_float4(0.f, 0.f, 0.f, 0.f), vb = make_float4(0.f, 0.f, 0.f, 0.f);
            if (r < r1) {
                const float* row = SA + r * d;
                if (vec && ci0 + cq + 3 < d) {
                    va = *reinterpret_cast<const float4*>(row + ci0 + cq);
                } else {
                    va.x = ci0 + cq < d ? row[ci0 + cq] : 0.f;
                    va.y = ci0 + cq + 1 < d ? row[ci0 + cq + 1] : 0.f;
                    va.z = ci0 + cq + 2 < d ? row[ci0 + cq + 2] : 0.f;
                    va.w = ci0 + cq + 3 < d ? row[ci0 + cq + 3] : 0.f;
                }
                if (vec && cj0 + cq + 3 < d) {
                    vb = *reinterpret_cast<const float4*>(row + cj0 + cq);
                } else {
                    vb.x = cj0 + cq < d ? row[cj0 + cq] : 0.f;
                    vb.y = cj0 + cq + 1 < d ? row[cj0 + cq + 1] : 0.f;
                    vb.z = cj0 + cq + 2 < d ? row[cj0 + cq + 2] : 0.f;
                    vb.w = cj0 + cq + 3 < d ? row[cj0 + cq + 3] : 0.f;
                }
            }
            *reinterpret_cast<float4*>(&As[kk][cq]) = va;
            *reinterpret_cast<float4*>(&Bs[kk][cq]) = vb;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < kGK; ++kk) {
            const float4 a0 = *reinterpret_cast<const float4*>(&As[kk][ty * 8]);
            const float4 a1 = *reinterpret_cast<const float4*>(&As[kk][ty * 8 + 4]);
            const float4 b0 = *reinterpret_cast<const float4*>(&Bs[kk][tx * 8]);
            const float4 b1 = *reinterpret_cast<const float4*>(&Bs[kk][tx * 8 + 4]);
            const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
            for (int a = 0; a < 8; ++a)
#pragma unroll
                for (int b = 0; b < 8; ++b) acc[a][b] = fmaf(av[a], bv[b], acc[a][b]);
            if (vrow) {
                const float sb = Ss[kk];
#pragma unroll
                for (int a = 0; a < 8; ++a) vacc[a] = fmaf(av[a], sb, vacc[a]);
                sbb = fmaf(sb, sb, sbb);
            }
        }
        __syncthreads();
    }
    double* out = part + ((size_t)blockIdx.y * gridDim.x + blockIdx.x) * kGT * kGT;
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int b = 0; b < 8; ++b) out[(ty * 8 + a) * kGT + tx * 8 + b] = (double)acc[a][b];
    if (vrow) {
        double* vo = vpart + (size_t)blockIdx.y * (d + 1);
#pragma unroll
        for (int a = 0; a < 8; ++a)
            if (ci0 + ty * 8 + a < d) vo[ci0 + ty * 8 + a] = (double)vacc[a];
        if (ti == 0 && ty == 0) vo[d] = (double)sbb;
    }
}

// Gm (nc x nc, full, float64) from the tile and vector partials, fixed order.
__global__ void k_gram_reduce2(const double* __restrict__ tpart, const double* __restrict__ vpart, int nchunk,
                               int ntile, int d, int nc, double* __restrict__ Gm) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)nc * nc) return;
    const int ci = (int)(idx / nc), cj = (int)(idx % nc);
    if (ci > cj) return;
    double s = 0.0;
    if (cj < d) {
        const int ti = ci / kGT, tj = cj / kGT;
        int tl = 0;
        for (int q = 0; q < ti; ++q) tl += ntile - q;
        tl += tj - ti;
        const int ntl = ntile * (ntile + 1) / 2;
        const int off = (ci % kGT) * kGT + (cj % kGT);
        for (int c = 0; c < nchunk; ++c) s += tpart[((size_t)c * ntl + tl) * kGT * kGT + off];
    } else {
        for (int c = 0; c < nchunk; ++c) s += vpart[(size_t)c * (d + 1) + ci];
    }
    Gm[(int64_t)ci * nc + cj] = s;
    Gm[(int64_t)cj * nc + ci] = s;
}

// ---- blocked Cholesky + inverse on many SMs (LSQR preconditioner) --------
//
// W (float32, nc x nc, row-major) starts as the Gram matrix; after the panel
// loop its upper triangle holds R (G = R^T R) and its column d holds
// c = R^-T SA^T Sb.  Panels of 32 columns: one CTA factors the diagonal block
// and solves the panel's rows to the right, then one CTA per 32 x 32 tile of
// the trailing upper triangle subtracts the rank-32 update.

constexpr int kCholB = 32;

__global__ void k_gram_to_f32(const double* __restrict__ Gm, int64_t cnt, float* __restrict__ W) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q < cnt) W[q] = (float)Gm[q];
}

// Cholesky of a pb x pb (pb <= 32) diagonal block held by one warp, lane k
// holding column k in registers (entries 0..k): right-looking, the pivot and
// row j of R reach the other lanes by shuffles.  Returns false, the same on
// every lane, when a pivot is not positive.
__device__ __forceinline__ bool chol_block32(float (&col)[kCholB], int pb) {
    const int lane = threadIdx.x & 31;
    bool ok = true;
#pragma unroll
    for (int j = 0; j < kCholB; ++j) {
        const float piv = __shfl_sync(0xFFFFFFFFu, col[j], j);
        if (j < pb) {
            if (!(piv > 0.f)) ok = false;
            const float r = sqrtf(piv);
            if (lane == j) col[j] = r;
            else if (lane > j) col[j] = col[j] / r;
        }
        const float rjk = col[j];
#pragma unroll
        for (int i = 0; i < kCholB; ++i) {   // constant trip count keeps col[] in registers
            if (i > j) {
                const float rji = __shfl_sync(0xFFFFFFFFu, col[j], i);
                if (j < pb && lane >= i) col[i] = fmaf(-rji, rjk, col[i]);
            }
        }
    }
    return ok;
}

__global__ void __launch_bounds__(512) k_chol_panel(float* __restrict__ W, int d, int nc, int p0,
                                                   unsigned* bad) {
    __shared__ float D[kCholB][kCholB + 1];
    __shared__ int fail;
    const int tid = threadIdx.x, nt = blockDim.x;
    const int pb = min(kCholB, d - p0);
    for (int q = tid; q < kCholB * kCholB; q += nt) {
        const int i = q / kCholB, j = q % kCholB;
        D[i][j] = (i < pb && j < pb) ? W[(int64_t)(p0 + i) * nc + p0 + j] : 0.f;
    }
    if (tid == 0) fail = 0;
    __syncthreads();
    if (tid < 32) {
        float col[kCholB];
#pragma unroll
        for (int q = 0; q < kCholB; ++q) col[q] = D[q][tid];
        const bool ok = chol_block32(col, pb);
        if (!ok && tid == 0) {
            fail = 1;
            atomicExch(bad, 1u);
        }
#pragma unroll
        for (int q = 0; q < kCholB; ++q)
            if (q <= tid) D[q][tid] = col[q];
    }
    __syncthreads();
    if (fail) return;
    for (int q = tid; q < pb * pb; q += nt) {
        const int i = q / pb, k = q % pb;
        if (k >= i) W[(int64_t)(p0 + i) * nc + p0 + k] = D[i][k];
    }
    // rows p0..p0+pb-1 of R to the right of the block: R_pp^T X = W[p0.., k]
    for (int k = p0 + pb + tid; k < nc; k += nt) {
        float x[kCholB];
#pragma unroll
        for (int i = 0; i < kCholB; ++i) x[i] = (i < pb) ? W[(int64_t)(p0 + i) * nc + k] : 0.f;
#pragma unroll
        for (int i = 0; i < kCholB; ++i) {
            if (i < pb) {
                float sacc = x[i];
#pragma unroll
                for (int q = 0; q < kCholB; ++q)
                    if (q < i) sacc -= D[q][i] * x[q];
                x[i] = sacc / D[i][i];
            }
        }
#pragma unroll
        for (int i = 0; i < kCholB; ++i)
            if (i < pb) W[(int64_t)(p0 + i) * nc + k] = x[i];
    }
}

// W[i][k] -= sum_q R[p0+q][i] R[p0+q][k] over the trailing block (i < d, k >= i).
__global__ void __launch_bounds__(256) k_chol_update(float* __restrict__ W, int d, int nc, int p0) {
    __shared__ float Ri[kCholB][kCholB + 1];
    __shared__ float Rk[kCholB][kCholB + 1];
    const int s0 = p0 + kCholB;
    const int ntk = (nc - s0 + kCholB - 1) / kCholB;
    int t = blockIdx.x, ti = 0;
    while (t >= ntk - ti) {
        t -= ntk - ti;
        ++ti;
    }
    const int tk = ti + t;
    const int i0 = s0 + kCholB * ti, k0 = s0 + kCholB * tk;
    for (int q = threadIdx.x; q < kCholB * kCholB; q += blockDim.x) {
        const int r = q / kCholB, c = q % kCholB;
        const float* row = W + (int64_t)(p0 + r) * nc;
        Ri[r][c] = (i0 + c < d) ? row[i0 + c] : 0.f;
        Rk[r][c] = (k0 + c < nc) ? row[k0 + c] : 0.f;
    }
    __syncthreads();
    const int ty = threadIdx.x >> 5, tx = threadIdx.x & 31;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        const int r = ty * 4 + a;
        const int i = i0 + r, k = k0 + tx;
        if (i < d && k < nc && k >= i) {
            float acc = 0.f;
#pragma unroll 8
            for (int q = 0; q < kCholB; ++q) acc = fmaf(Ri[q][r], Rk[q][tx], acc);
            W[(int64_t)i * nc + k] -= acc;
        }
    }
}

// The whole factorization in one CTA when the packed upper triangle of W fits
// in shared memory: for each panel of 32 columns, warp 0 factors the diagonal
// block, one thread per column to the right solves the panel's rows, and all
// warps subtract the rank-32 update from the trailing triangle (warp = 4 rows
// x 128 columns, lane = 4 columns 32 apart).  W is read once and written once.
// Packed row i holds columns i..nc-1 at P[i*nc - i*(i+1)/2 + k].  The three
// phases are separate non-inlined functions so that each one's unrolled
// register arrays get the whole register budget.
__device__ __forceinline__ int chol_off(int i, int nc) { return i * nc - (i * (i + 1)) / 2; }

// warp 0: diagonal block of panel p0 (pb columns) into Dg and back into P;
// returns false on a non-positive pivot (the same on every lane)
__device__ __noinline__ bool chol_small_factor(float* P, float (*Dg)[kCholB + 1], int nc, int p0, int pb) {
    const int lane = threadIdx.x & 31;
    float col[kCholB];
#pragma unroll
    for (int q = 0; q < kCholB; ++q) col[q] = (q <= lane && lane < pb) ? P[chol_off(p0 + q, nc) + p0 + lane] : 0.f;
    const bool ok = chol_block32(col, pb);
#pragma unroll
    for (int q = 0; q < kCholB; ++q) {
        if (q <= lane && lane < pb) P[chol_off(p0 + q, nc) + p0 + lane] = col[q];
        Dg[q][lane] = col[q];
    }
    return ok;
}

// column k to the right of the block: R_pp^T x = P[p0.., k], rows in two halves of 16
__device__ __noinline__ void chol_small_panel(float* P, const float (*Dg)[kCholB + 1], int nc, int p0, int pb,
                                              int k) {
    float x[16], y[16];
    int o = chol_off(p0, nc) + k;   // P index of (p0 + i, k), advanced row by row
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        x[i] = (i < pb) ? P[o] : 0.f;
        o += nc - (p0 + i) - 1;
    }
#pragma unroll
    for (int q = 0; q < 16; ++q) {
        x[q] = (q < pb) ? x[q] / Dg[q][q] : 0.f;
#pragma unroll
        for (int i = 0; i < 16; ++i)
            if (i > q) x[i] = fmaf(-Dg[q][i], x[q], x[i]);
    }
    const int o16 = o;
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        y[i] = (16 + i < pb) ? P[o] : 0.f;
        o += nc - (p0 + 16 + i) - 1;
    }
#pragma unroll
    for (int q = 0; q < 16; ++q)
#pragma unroll
        for (int i = 0; i < 16; ++i) y[i] = fmaf(-Dg[q][16 + i], x[q], y[i]);
#pragma unroll
    for (int q = 0; q < 16; ++q) {
        y[q] = (16 + q < pb) ? y[q] / Dg[16 + q][16 + q] : 0.f;
#pragma unroll
        for (int i = 0; i < 16; ++i)
            if (i > q) y[i] = fmaf(-Dg[16 + q][16 + i], y[q], y[i]);
    }
    o = chol_off(p0, nc) + k;
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        if (i < pb) P[o] = x[i];
        o += nc - (p0 + i) - 1;
    }
    o = o16;
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        if (16 + i < pb) P[o] = y[i];
        o += nc - (p0 + 16 + i) - 1;
    }
}

// P[i][k] -= sum_q R[p0+q][i] R[p0+q][k] for i in [i0, i0 + 4) (< d), the lane's
// four columns kb + lane + 32c (>= i, < nc)
__device__ __noinline__ void chol_small_update(float* P, int d, int nc, int p0, int pb, int i0, int kb) {
    const int lane = threadIdx.x & 31;
    float acc[4][4];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c] = 0.f;
    int o = chol_off(p0, nc);
    for (int q = 0; q < pb; ++q) {
        const float* Rq = P + o;
        float a[4], b[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) a[r] = (i0 + r < d) ? Rq[i0 + r] : 0.f;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int k = kb + lane + 32 * c;
            b[c] = (k < nc) ? Rq[k] : 0.f;
        }
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[r][c] = fmaf(a[r], b[c], acc[r][c]);
        o += nc - (p0 + q) - 1;
    }
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int i = i0 + r, k = kb + lane + 32 * c;
            if (i < d && k < nc && k >= i) P[chol_off(i, nc) + k] -= acc[r][c];
        }
}

__global__ void __launch_bounds__(512) k_chol_small(float* __restrict__ W, int d, int nc, unsigned* bad) {
    extern __shared__ float P[];
    __shared__ float Dg[kCholB][kCholB + 1];   // R of the current diagonal block
    __shared__ int fail;
    const int tid = threadIdx.x, nt = blockDim.x, warp = tid >> 5, nw = nt >> 5;
    for (int q = tid; q < nc * nc; q += nt) {
        const int i = q / nc, k = q - i * nc;
        if (k >= i) cp_async4(P + chol_off(i, nc) + k, W + q);
    }
    cp_async_wait_all();
    if (tid == 0) fail = 0;
    __syncthreads();
    for (int p0 = 0; p0 < d; p0 += kCholB) {
        const int pb = min(kCholB, d - p0);
        if (warp == 0) {
            const bool ok = chol_small_factor(P, Dg, nc, p0, pb);
            if (!ok && tid == 0) {
                fail = 1;
                atomicExch(bad, 1u);
            }
        }
        __syncthreads();
        if (fail) return;
        const int s0 = p0 + pb;
        for (int k = s0 + tid; k < nc; k += nt) chol_small_panel(P, Dg, nc, p0, pb, k);
        __syncthreads();
        const int nbi = (d - s0 + 3) / 4, ng = (nc - s0 + 127) / 128;
        for (int wt = warp; wt < nbi * ng; wt += nw) {
            const int bi = wt / ng, g = wt - bi * ng;
            const int i0 = s0 + 4 * bi, kb = s0 + 128 * g;
            if (kb + 127 >= i0) chol_small_update(P, d, nc, p0, pb, i0, kb);   // else below the diagonal
        }
        __syncthreads();
    }
    for (int q = tid; q < nc * nc; q += nt) {
        const int i = q / nc, k = q - i * nc;
        if (k >= i) W[q] = P[chol_off(i, nc) + k];
    }
}

// diagonal ratio (lower bound of kappa) and c = W[0:d, d] in float64
__global__ void k_chol_finish(const float* __restrict__ W, int d, int nc, double* __restrict__ c,
                              float* __restrict__ kappa_lb) {
    __shared__ float smx[32], smn[32];
    float mx = 0.f, mn = 3.4e38f;
    for (int j = threadIdx.x; j < d; j += blockDim.x) {
        const float v = fabsf(W[(int64_t)j * nc + j]);
        mx = fmaxf(mx, v);
        mn = fminf(mn, v);
        if (c && nc > d) c[j] = (double)W[(int64_t)j * nc + d];
    }
    for (int o = 16; o > 0; o >>= 1) {
        mx = fmaxf(mx, __shfl_xor_sync(0xFFFFFFFFu, mx, o));
        mn = fminf(mn, __shfl_xor_sync(0xFFFFFFFFu, mn, o));
    }
    if ((threadIdx.x & 31) == 0) {
        smx[threadIdx.x >> 5] = mx;
        smn[threadIdx.x >> 5] = mn;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
            mx = fmaxf(mx, smx[w]);
            mn = fminf(mn, smn[w]);
        }
        mx = fmaxf(mx, smx[0]);
        mn = fminf(mn, smn[0]);
        *kappa_lb = mn > 0.f ? mx / mn : 3.4e38f;
    }
}

// M = R^-1 (float32 arithmetic, R = upper triangle of W), one warp per column:
// x_i = (delta_ij - sum_{i<k<=j} R_ik x_k) / R_ii for i = j .. 0, R rows read
// from a shared-memory copy of the packed triangle when it fits (PACKED).
template <bool PACKED>
__global__ void __launch_bounds__(256) k_tri_inv_f32(const float* __restrict__ W, int d, int nc,
                                                    double* __restrict__ M, float* __restrict__ M32T) {
    extern __shared__ float sh[];
    float* xs = sh;                                   // [8][1024]
    float* T = sh + 8 * 1024;                         // packed triangle (PACKED)
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (PACKED) {
        for (int q = threadIdx.x; q < d * d; q += blockDim.x) {
            const int i = q / d, k = q - i * d;
            if (k >= i) cp_async4(T + i * d - (i * (i - 1)) / 2 + (k - i), W + (int64_t)i * nc + k);
        }
        cp_async_wait_all();
        __syncthreads();
    }
    const int col = blockIdx.x * 8 + warp;
    if (col >= d) return;
    float* x = xs + warp * 1024;
    for (int i = lane; i < d; i += 32) x[i] = 0.f;
    __syncwarp();
    for (int i = col; i >= 0; --i) {
        float part = 0.f;
        if (PACKED) {
            const float* Ri = T + i * d - (i * (i - 1)) / 2 - i;
            for (int k = i + 1 + lane; k <= col; k += 32) part = fmaf(Ri[k], x[k], part);
        } else {
            const float* Ri = W + (int64_t)i * nc;
            for (int k = i + 1 + lane; k <= col; k += 32) part = fmaf(Ri[k], x[k], part);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xFFFFFFFFu, part, o);
        if (lane == 0) {
            const float rii = PACKED ? T[i * d - (i * (i - 1)) / 2] : W[(int64_t)i * nc + i];
            x[i] = ((i == col ? 1.f : 0.f) - part) / rii;
        }
        __syncwarp();
    }
    for (int i = lane; i < d; i += 32) {
        const float v = (i <= col) ? x[i] : 0.f;
        M[(int64_t)i * d + col] = (double)v;
        M32T[(int64_t)col * d + i] = v;
    }
}

// M = R^-1 for upper-triangular row-major R (float64); one warp per column of
// M, RT = R^T (column j of R contiguous) for coalesced reads.
__global__ void k_tri_inverse(const double* __restrict__ RT, int d, double* __restrict__ M) {
    const int lane = threadIdx.x & 31;
    const int col = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if (col >= d) return;
    constexpr int kMaxPer = 32;  // d <= 1024
    double s[kMaxPer];
    const int per = (d + 31) / 32;
#pragma unroll
    for (int q = 0; q < kMaxPer; ++q) s[q] = 0.0;
#pragma unroll
    for (int q = 0; q < kMaxPer; ++q)
        if (q < per && lane + 32 * q == col) s[q] = 1.0;
    for (int j = col; j >= 0; --j) {
        const int oj = j & 31, qj = j >> 5;
        double sj = 0.0;
#pragma unroll
        for (int q = 0; q < kMaxPer; ++q)
            if (q == qj) sj = s[q];
        const double xj = __shfl_sync(0xFFFFFFFFu, sj, oj) / RT[(int64_t)j * d + j];
#pragma unroll
        for (int q = 0; q < kMaxPer; ++q) {
            if (q < per) {
                const int i = lane + 32 * q;
                if (i == j)
                    s[q] = xj;
                else if (i < j)
                    s[q] -= RT[(int64_t)j * d + i] * xj;
            }
        }
    }
#pragma unroll
    for (int q = 0; q < kMaxPer; ++q) {
        const int i = lane + 32 * q;
        if (q < per && i < d) M[(int64_t)i * d + col] = (i <= col) ? s[q] : 0.0;
    }
}

__global__ void k_transpose64(const double* __restrict__ A, int d, double* __restrict__ AT) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= (int64_t)d * d) return;
    const int i = (int)(q / d), j = (int)(q % d);
    AT[(int64_t)j * d + i] = A[q];
}

// ---------------------------------------------------------------- host drivers

namespace {

int qr_grid(int64_t m, int threads, size_t smem) {
    int dev = 0, per = 0;
    cudaGetDevice(&dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_qr_householder, threads, smem) != cudaSuccess)
        per = 1;
    per = per < 1 ? 1 : (per > 2 ? 2 : per);
    int g = num_sms() * per;
    const int64_t want = (m + 63) / 64;  // at least 64 rows per block
    if (want < g) g = (int)(want < 1 ? 1 : want);
    return g;
}

}  // namespace

// Householder QR of [SA | Sb] in float64.  R (device, row-major d x d) and c
// (device, d) may be NULL.  Synchronises the stream.  Returns CW_ERR_RANK for
// a numerically rank-deficient SA (outputs still written).
int qr64(const float* SA, int64_t m, int d, const float* Sb, double* R, double* c, cudaStream_t stream,
         const double* SA64) {
    const int nc = d + (Sb ? 1 : 0);
    const int threads = 256;
    int G = qr_grid(m, threads, 48 * 1024);
    const size_t smem = sizeof(double) * (size_t)((m + G - 1) / G);
    if (smem > 200 * 1024) return CW_ERR_SHAPE;  // m too large for the resident-grid design
    Scratch ws(stream);
    const size_t oW = ws.reserve(sizeof(double) * (size_t)m * nc);
    const size_t oN = ws.reserve(sizeof(double) * (size_t)G);
    const size_t oD = ws.reserve(sizeof(double) * (size_t)G * nc);
    const size_t oV = ws.reserve(sizeof(double) * (size_t)nc);
    const size_t oB = ws.reserve(sizeof(unsigned) * 4);
    CW_CUDA_TRY(ws.alloc());
    double* W = ws.at<double>(oW);
    unsigned* bar = ws.at<unsigned>(oB);
    CW_CUDA_TRY(cudaMemsetAsync(bar, 0, sizeof(unsigned) * 4, stream));
    dim3 tb(32, 8), tg((unsigned)((m + 31) / 32), (unsigned)((nc + 31) / 32));
    if (SA64)
        {
            CW_PROF("k_to_colmajor64", stream);
            k_to_colmajor64<double><<<tg, tb, 0, stream>>>(SA64, Sb, m, d, nc, W);
        }
    else
        {
            CW_PROF("k_to_colmajor64", stream);
            k_to_colmajor64<float><<<tg, tb, 0, stream>>>(SA, Sb, m, d, nc, W);
        }
    CW_LAUNCH_CHECK();
    QrArgs a{W, m, d, nc, ws.at<double>(oN), ws.at<double>(oD), ws.at<double>(oV), bar, bar + 2};
    CW_CUDA_TRY(cudaFuncSetAttribute(k_qr_householder, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    CW_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_qr_householder, threads, smem));
    if ((int64_t)per_sm * num_sms() < G) G = per_sm * num_sms();
    if (G < 1) return CW_ERR_CUDA;
    void* args[] = {&a};
    {
        CW_PROF("k_qr_householder", stream);
        CW_CUDA_TRY(cudaLaunchCooperativeKernel((void*)k_qr_householder, dim3(G), dim3(threads), args, smem, stream));
    }
    {
        CW_PROF("k_qr_finalize", stream);
        k_qr_finalize<<<1, 256, 0, stream>>>(W, m, d, nc, R, c, bar + 3);
    }
    CW_LAUNCH_CHECK();
    unsigned flags[2] = {0, 0};
    CW_CUDA_TRY(cudaMemcpyAsync(flags, bar + 2, sizeof(unsigned) * 2, cudaMemcpyDeviceToHost, stream));
    CW_CUDA_TRY(cudaStreamSynchronize(stream));
    if (flags[0]) return CW_ERR_TIMEOUT;
    if (flags[1]) return CW_ERR_RANK;
    return CW_OK;
}

// Gram + Cholesky + inverse for the LSQR preconditioner.  M (float64 d x d,
// float32 values), M32T (float32, column-major) and c = R^-T SA^T Sb; *kappa_lb
// receives the diagonal ratio of R.  Returns CW_ERR_RANK on a non-positive
// pivot.  Synchronises (the caller needs the ratio on the host).
int gram_chol_inverse(const float* SA, int64_t m, int d, const float* Sb, double* M, float* M32T, double* c,
                      float* kappa_lb_host, cudaStream_t stream) {
    const int nc = d + (Sb ? 1 : 0);
    if (d > 1024) return CW_ERR_SHAPE;
    const int ntile = (d + kGT - 1) / kGT;
    const int ntl = ntile * (ntile + 1) / 2;
    // rows per chunk: about one CTA per SM in one wave (146 registers a thread)
    int64_t rows = (m * ntl + num_sms() - 1) / num_sms();
    rows = ((rows + kGK - 1) / kGK) * kGK;
    if (rows < 256) rows = 256;
    const int nchunk = (int)((m + rows - 1) / rows);
    Scratch ws(stream);
    const size_t oP = ws.reserve(sizeof(double) * (size_t)nchunk * ntl * kGT * kGT);
    const size_t oV = ws.reserve(sizeof(double) * (size_t)nchunk * (d + 1));
    const size_t oG = ws.reserve(sizeof(double) * (size_t)nc * nc);
    const size_t oW = ws.reserve(sizeof(float) * (size_t)nc * nc);
    const size_t oF = ws.reserve(sizeof(unsigned) * 2 + sizeof(float) * 2);
    CW_CUDA_TRY(ws.alloc());
    double* part = ws.at<double>(oP);
    double* vpart = ws.at<double>(oV);
    double* Gm = ws.at<double>(oG);
    float* W = ws.at<float>(oW);
    unsigned* bad = ws.at<unsigned>(oF);
    float* klb = reinterpret_cast<float*>(bad + 2);
    CW_CUDA_TRY(cudaMemsetAsync(bad, 0, sizeof(unsigned) * 2 + sizeof(float) * 2, stream));
    {
        CW_PROF("k_gram_tile", stream);
        k_gram_tile<<<dim3((unsigned)ntl, (unsigned)nchunk), 256, 0, stream>>>(SA, Sb, m, d, ntile, (int)rows, part,
                                                                             vpart);
    }
    const int64_t tot = (int64_t)nc * nc;
    {
        CW_PROF("k_gram_reduce", stream);
        k_gram_reduce2<<<(unsigned)((tot + 255) / 256), 256, 0, stream>>>(part, vpart, nchunk, ntile, d, nc, Gm);
    }
    {
        CW_PROF("k_gram_to_f32", stream);
        k_gram_to_f32<<<(unsigned)((tot + 255) / 256), 256, 0, stream>>>(Gm, tot, W);
    }
    const size_t psm = sizeof(float) * ((size_t)nc * (nc + 1) / 2);
    const bool small = psm + 1024 <= 227 * 1024;
    if (small) {
        CW_CUDA_TRY(cudaFuncSetAttribute(k_chol_small, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)psm));
        CW_PROF("k_chol_small", stream);
        k_chol_small<<<1, 512, psm, stream>>>(W, d, nc, bad);
    }
    for (int p0 = 0; !small && p0 < d; p0 += kCholB) {
        {
            CW_PROF("k_chol_panel", stream);
            k_chol_panel<<<1, 512, 0, stream>>>(W, d, nc, p0, bad);
        }
        const int s0 = p0 + kCholB;
        if (s0 < d) {
            const int nti = (d - s0 + kCholB - 1) / kCholB, ntk = (nc - s0 + kCholB - 1) / kCholB;
            int tiles = 0;
            for (int ti = 0; ti < nti; ++ti) tiles += ntk - ti;
            CW_PROF("k_chol_update", stream);
            k_chol_update<<<tiles, 256, 0, stream>>>(W, d, nc, p0);
        }
    }
    {
        CW_PROF("k_chol_finish", stream);
        k_chol_finish<<<1, 1024, 0, stream>>>(W, d, nc, c, klb);
    }
    const size_t packed = sizeof(float) * ((size_t)d * (d + 1) / 2);
    const size_t xs = sizeof(float) * 8 * 1024;
    if (xs + packed <= 200 * 1024) {
        CW_CUDA_TRY(cudaFuncSetAttribute(k_tri_inv_f32<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(xs + packed)));
        CW_PROF("k_tri_inv_f32", stream);
        k_tri_inv_f32<true><<<(d + 7) / 8, 256, xs + packed, stream>>>(W, d, nc, M, M32T);
    } else {
        CW_PROF("k_tri_inv_f32", stream);
        k_tri_inv_f32<false><<<(d + 7) / 8, 256, xs, stream>>>(W, d, nc, M, M32T);
    }
    CW_LAUNCH_CHECK();
    unsigned h[2] = {0, 0};
    float kl[2] = {0.f, 0.f};
    CW_CUDA_TRY(cudaMemcpyAsync(h, bad, sizeof(unsigned) * 2, cudaMemcpyDeviceToHost, stream));
    CW_CUDA_TRY(cudaMemcpyAsync(kl, klb, sizeof(float) * 2, cudaMemcpyDeviceToHost, stream));
    CW_CUDA_TRY(cudaStreamSynchronize(stream));
    if (kappa_lb_host) *kappa_lb_host = kl[0];
    return h[0] ? CW_ERR_RANK : CW_OK;
}

int trsv_upper(const double* R, int d, const double* rhs, double* x, cudaStream_t stream) {
    {
        CW_PROF("k_trsv_upper", stream);
        k_trsv_upper<<<1, 256, sizeof(double) * d, stream>>>(R, d, rhs, x);
    }
    CW_LAUNCH_CHECK();
    return CW_OK;
}

// M = R^-1 (upper triangular, float64), one warp per column.
int tri_inverse(const double* R, int d, double* M, cudaStream_t stream) {
    if (d > 1024) return CW_ERR_SHAPE;
    double* RT = nullptr;
    CW_CUDA_TRY(cudaMallocAsync(&RT, sizeof(double) * (size_t)d * d, stream));
    const int64_t dd = (int64_t)d * d;
    {
        CW_PROF("k_transpose64", stream);
        k_transpose64<<<(unsigned)((dd + 255) / 256), 256, 0, stream>>>(R, d, RT);
    }
    {
        CW_PROF("k_tri_inverse", stream);
        k_tri_inverse<<<(unsigned)((d + 7) / 8), 256, 0, stream>>>(RT, d, M);
    }
    cudaError_t e = cudaGetLastError();
    cudaFreeAsync(RT, stream);
    return e == cudaSuccess ? CW_OK : CW_ERR_CUDA;
}

// X = R^-1 B (B d x k row-major; B == NULL gives the inverse, k == d).
int trsm_upper(const double* R, int d, const double* B, int k, double* X, cudaStream_t stream) {
    {
        CW_PROF("k_trsm_upper", stream);
        k_trsm_upper<<<k, 256, sizeof(double) * d, stream>>>(R, d, B, k, X);
    }
    CW_LAUNCH_CHECK();
    return CW_OK;
}

}  // namespace cw

using namespace cw;

extern "C" int cw_qr(const float* SA, int64_t m, int64_t d, const float* Sb, double* R, double* c,
                     cw_stream stream) {
    if (!SA) return CW_ERR_ARG;
    if (d < 1 || d > 1024 || m < d) return CW_ERR_SHAPE;
    if (m > 0x7FFFFFFFll) return CW_ERR_OVERFLOW;
    return qr64(SA, m, (int)d, c ? Sb : nullptr, R, c, stream);
}
