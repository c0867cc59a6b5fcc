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

// ---------------------------------------------------------------- Gram matrix (fast R)

constexpr int kGramTile = 64;
constexpr int kGramRowsPerChunk = 2048;

// Partial Gram of the columns [ti*64, ti*64+64) x [tj*64, tj*64+64) of
// X = [SA | Sb] over one chunk of rows; float32 products and sums within the
// chunk, stored as float64 partials [chunk][nc][nc].
__global__ void __launch_bounds__(256) k_gram_partial(const float* __restrict__ SA, const float* __restrict__ Sb,
                                                     int64_t m, int d, int nc, int ntile,
                                                     double* __restrict__ part) {
    __shared__ float Xi[32][kGramTile + 1];
    __shared__ float Xj[32][kGramTile + 1];
    // upper-triangular tile index -> (ti, tj)
    int t = blockIdx.x, ti = 0;
    while (t >= ntile - ti) {
        t -= ntile - ti;
        ++ti;
    }
    const int tj = ti + t;
    const int chunk = blockIdx.y;
    const int64_t rb = (int64_t)chunk * kGramRowsPerChunk;
    const int64_t re = (rb + kGramRowsPerChunk < m) ? rb + kGramRowsPerChunk : m;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;  // 16 x 16 threads, 4 x 4 outputs each
    float acc[4][4] = {};
    for (int64_t r = rb; r < re; r += 32) {
        for (int q = threadIdx.x; q < 32 * kGramTile; q += blockDim.x) {
            const int rr = q / kGramTile, cc = q % kGramTile;
            const int64_t row = r + rr;
            const int ci = ti * kGramTile + cc, cj = tj * kGramTile + cc;
            float vi = 0.f, vj = 0.f;
            if (row < re) {
                vi = ci < d ? SA[row * d + ci] : (ci == d && Sb ? Sb[row] : 0.f);
                vj = cj < d ? SA[row * d + cj] : (cj == d && Sb ? Sb[row] : 0.f);
            }
            Xi[rr][cc] = vi;
            Xj[rr][cc] = vj;
        }
        __syncthreads();
#pragma unroll 4
        for (int rr = 0; rr < 32; ++rr) {
            float a[4], b[4];
#pragma unroll
            for (int p = 0; p < 4; ++p) {
                a[p] = Xi[rr][ty * 4 + p];
                b[p] = Xj[rr][tx * 4 + p];
            }
#pragma unroll
            for (int p = 0; p < 4; ++p)
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[p][q] = fmaf(a[p], b[q], acc[p][q]);
        }
        __syncthreads();
    }
    double* out = part + (size_t)chunk * nc * nc;
#pragma unroll
    for (int p = 0; p < 4; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int ci = ti * kGramTile + ty * 4 + p, cj = tj * kGramTile + tx * 4 + q;
            if (ci < nc && cj < nc && ci <= cj) out[(size_t)ci * nc + cj] = (double)acc[p][q];
        }
}

__global__ void k_gram_reduce(const double* __restrict__ part, int nchunk, int nc, double* __restrict__ Gm) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)nc * nc) return;
    const int ci = (int)(idx / nc), cj = (int)(idx % nc);
    if (ci > cj) return;
    double s = 0.0;
    for (int c = 0; c < nchunk; ++c) s += part[(size_t)c * nc * nc + idx];
    Gm[(int64_t)ci * nc + cj] = s;
    Gm[(int64_t)cj * nc + ci] = s;
}

// Upper Cholesky G = R^T R of the leading d x d block of the float64 Gram
// matrix, computed in float32 by one CTA (right-looking, 32 x 32 thread grid
// over the trailing block).  The carried column d becomes c = R^-T SA^T Sb.
// float32 is enough here: this R only preconditions LSQR (any R with
// SA R^-1 near-orthonormal works), and callers fall back to the float64
// Householder R when the diagonal signals a large condition number.
// W: float32 working copy (nc x nc, row-major).  Flags a non-positive pivot.
__global__ void __launch_bounds__(1024) k_cholesky_f32(const double* __restrict__ Gm, float* __restrict__ W, int d,
                                                      int nc, double* __restrict__ R, double* __restrict__ c,
                                                      unsigned* bad) {
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    for (int64_t q = threadIdx.x; q < (int64_t)nc * nc; q += blockDim.x) W[q] = (float)Gm[q];
    __syncthreads();
    __shared__ float rowj[1025];
    __shared__ int fail;
    if (threadIdx.x == 0) fail = 0;
    for (int j = 0; j < d; ++j) {
        __syncthreads();
        const float piv = W[(int64_t)j * nc + j];
        if (!(piv > 0.f)) {
            if (threadIdx.x == 0) {
                fail = 1;
                atomicExch(bad, 1u);
            }
            break;
        }
        const float rjj = sqrtf(piv);
        const float inv = 1.0f / rjj;
        for (int k = j + threadIdx.x; k < nc; k += blockDim.x) {
            const float v = (k == j) ? rjj : W[(int64_t)j * nc + k] * inv;
            W[(int64_t)j * nc + k] = v;
            rowj[k] = v;
        }
        __syncthreads();
        // W[i, k] -= R[j, i] * R[j, k] for j < i <= k
        for (int i = j + 1 + ty; i < d; i += 32) {
            const float rji = rowj[i];
            float* wi = W + (int64_t)i * nc;
            for (int k = i + tx; k < nc; k += 32) wi[k] -= rji * rowj[k];
        }
    }
    __syncthreads();
    if (fail) return;
    for (int64_t q = threadIdx.x; q < (int64_t)d * d; q += blockDim.x) {
        const int i = (int)(q / d), k = (int)(q % d);
        R[q] = (k < i) ? 0.0 : (double)W[(int64_t)i * nc + k];
    }
    if (c && nc > d)
        for (int i = threadIdx.x; i < d; i += blockDim.x) c[i] = (double)W[(int64_t)i * nc + d];
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
    for (int j = 0; j < pb; ++j) {
        if (tid == 0) {
            const float piv = D[j][j];
            if (!(piv > 0.f)) {
                fail = 1;
                atomicExch(bad, 1u);
            } else {
                D[j][j] = sqrtf(piv);
            }
        }
        __syncthreads();
        if (fail) return;
        const float r = D[j][j];
        if (tid > j && tid < pb) D[j][tid] /= r;
        __syncthreads();
        for (int q = tid; q < pb * pb; q += nt) {
            const int i = q / pb, k = q % pb;
            if (i > j && k >= i) D[i][k] -= D[j][i] * D[j][k];
        }
        __syncthreads();
    }
    for (int q = tid; q < pb * pb; q += nt) {
        const int i = q / pb, k = q % pb;
        if (k >= i) W[(int64_t)(p0 + i) * nc + p0 + k] = D[i][k];
    }
    // rows p0..p0+pb-1 of R to the right of the block: R_pp^T X = W[p0.., k]
    for (int k = p0 + pb + tid; k < nc; k += nt) {
        float x[kCholB];
#pragma unroll
        for (int i = 0; i < kCholB; ++i) {
            if (i < pb) {
                float sacc = W[(int64_t)(p0 + i) * nc + k];
#pragma unroll
                for (int q = 0; q < kCholB; ++q)
                    if (q < i) sacc -= D[q][i] * x[q];
                x[i] = sacc / D[i][i];
                W[(int64_t)(p0 + i) * nc + k] = x[i];
            }
        }
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
        for (int i = 0; i < d; ++i)
            for (int k = i + threadIdx.x; k < d; k += blockDim.x)
                T[i * d - (i * (i - 1)) / 2 + (k - i)] = W[(int64_t)i * nc + k];
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

// Fast R: upper Cholesky factor of the Gram matrix of SA (float32 products,
// float64 accumulation across row chunks), and c = R^-T SA^T Sb when Sb is
// given.  Returns CW_ERR_RANK when a pivot is not positive.  Asynchronous
// except for the final flag read (synchronises).
int gram_cholesky(const float* SA, int64_t m, int d, const float* Sb, double* R, double* c, cudaStream_t stream) {
    const int nc = d + (Sb ? 1 : 0);
    const int ntile = (nc + kGramTile - 1) / kGramTile;
    const int nchunk = (int)((m + kGramRowsPerChunk - 1) / kGramRowsPerChunk);
    Scratch ws(stream);
    const size_t oP = ws.reserve(sizeof(double) * (size_t)nchunk * nc * nc);
    const size_t oG = ws.reserve(sizeof(double) * (size_t)nc * nc);
    const size_t oW = ws.reserve(sizeof(float) * (size_t)nc * nc);
    const size_t oF = ws.reserve(sizeof(unsigned) * 2);
    CW_CUDA_TRY(ws.alloc());
    double* part = ws.at<double>(oP);
    double* Gm = ws.at<double>(oG);
    unsigned* bad = ws.at<unsigned>(oF);
    CW_CUDA_TRY(cudaMemsetAsync(bad, 0, sizeof(unsigned) * 2, stream));
    dim3 gg((unsigned)(ntile * (ntile + 1) / 2), (unsigned)nchunk);
    {
        CW_PROF("k_gram_partial", stream);
        k_gram_partial<<<gg, 256, 0, stream>>>(SA, Sb, m, d, nc, ntile, part);
    }
    CW_LAUNCH_CHECK();
    const int64_t tot = (int64_t)nc * nc;
    {
        CW_PROF("k_gram_reduce", stream);
        k_gram_reduce<<<(unsigned)((tot + 255) / 256), 256, 0, stream>>>(part, nchunk, nc, Gm);
    }
    CW_LAUNCH_CHECK();
    {
        CW_PROF("k_cholesky_f32", stream);
        k_cholesky_f32<<<1, 1024, 0, stream>>>(Gm, ws.at<float>(oW), d, nc, R, c, bad);
    }
    CW_LAUNCH_CHECK();
    unsigned h = 0;
    CW_CUDA_TRY(cudaMemcpyAsync(&h, bad, sizeof(unsigned), cudaMemcpyDeviceToHost, stream));
    CW_CUDA_TRY(cudaStreamSynchronize(stream));
    return h ? CW_ERR_RANK : CW_OK;
}

// Gram + Cholesky + inverse for the LSQR preconditioner.  M (float64 d x d),
// M32T (float32, column-major) and c = R^-T SA^T Sb; *kappa_lb receives the
// diagonal ratio of R.  Returns CW_ERR_RANK on a non-positive pivot and
// CW_ERR_SHAPE when the packed triangle does not fit in shared memory.
int gram_chol_inverse(const float* SA, int64_t m, int d, const float* Sb, double* M, float* M32T, double* c,
                      float* kappa_lb_host, cudaStream_t stream) {
    const int nc = d + (Sb ? 1 : 0);
    if (d > 1024) return CW_ERR_SHAPE;
    const int ntile = (nc + kGramTile - 1) / kGramTile;
    const int nchunk = (int)((m + kGramRowsPerChunk - 1) / kGramRowsPerChunk);
    Scratch ws(stream);
    const size_t oP = ws.reserve(sizeof(double) * (size_t)nchunk * nc * nc);
    const size_t oG = ws.reserve(sizeof(double) * (size_t)nc * nc);
    const size_t oW = ws.reserve(sizeof(float) * (size_t)nc * nc);
    const size_t oF = ws.reserve(sizeof(unsigned) * 2 + sizeof(float) * 2);
    CW_CUDA_TRY(ws.alloc());
    double* part = ws.at<double>(oP);
    double* Gm = ws.at<double>(oG);
    float* W = ws.at<float>(oW);
    unsigned* bad = ws.at<unsigned>(oF);
    float* klb = reinterpret_cast<float*>(bad + 2);
    CW_CUDA_TRY(cudaMemsetAsync(bad, 0, sizeof(unsigned) * 2 + sizeof(float) * 2, stream));
    dim3 gg((unsigned)(ntile * (ntile + 1) / 2), (unsigned)nchunk);
    {
        CW_PROF("k_gram_partial", stream);
        k_gram_partial<<<gg, 256, 0, stream>>>(SA, Sb, m, d, nc, ntile, part);
    }
    const int64_t tot = (int64_t)nc * nc;
    {
        CW_PROF("k_gram_reduce", stream);
        k_gram_reduce<<<(unsigned)((tot + 255) / 256), 256, 0, stream>>>(part, nchunk, nc, Gm);
    }
    {
        CW_PROF("k_gram_to_f32", stream);
        k_gram_to_f32<<<(unsigned)((tot + 255) / 256), 256, 0, stream>>>(Gm, tot, W);
    }
    for (int p0 = 0; p0 < d; p0 += kCholB) {
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
