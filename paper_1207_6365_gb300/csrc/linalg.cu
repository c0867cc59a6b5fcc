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

__global__ void __launch_bounds__(1024) k_qr_householder(QrArgs a) {
    extern __shared__ double sv[];  // this block's reflector entries (rows r0..r1)
    __shared__ double s_red[32];
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
        // reflector for column j: every block forms the same scalars (lanes
        // over blocks, then the warp's tree: the same fixed order everywhere)
        // (the scalars formed by one thread: float64 square roots and divisions
        // are long sequences on this part)
        if (warp == 0) {
            double t = 0.0;
            for (unsigned c = lane; c < G; c += 32) t += a.normp[c];
            t = warp_sum(t);
            if (lane == 0) {
                const double sig2 = t;
                const double ajj = a.W[(int64_t)j * a.m + j];
                double beta = 0.0, tau = 0.0, vscale = 0.0;
                if (sig2 != 0.0) {
                    const double sig = sqrt(sig2);
                    beta = ajj >= 0.0 ? -sig : sig;
                    tau = (beta - ajj) / beta;
                    vscale = 1.0 / (ajj - beta);
                }
                s_red[0] = beta;
                s_red[1] = tau;
                s_red[2] = vscale;
            }
        }
        __syncthreads();
        const double beta = s_red[0], tau = s_red[1], vscale = s_red[2];
        __syncthreads();
        // v for my rows (0 above the diagonal, 1 at it)
        const double* colj = a.W + (int64_t)j * a.m;
        for (int64_t q = threadIdx.x; q < rows; q += blockDim.x) {
            const int64_t i = r0 + q;
            sv[q] = (i < j) ? 0.0 : (i == j ? 1.0 : colj[i] * vscale);
        }
        __syncthreads();
        // partial dots v^T W[:, k] for k > j
        for (int k = j + 1 + warp; k < a.nc; k += nwarps) {
            const double* colk = a.W + (int64_t)k * a.m + r0;
            double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;   // four independent chains
            int64_t q = lane;
            for (; q + 96 < rows; q += 128) {
                s0 = fma(sv[q], colk[q], s0);
                s1 = fma(sv[q + 32], colk[q + 32], s1);
                s2 = fma(sv[q + 64], colk[q + 64], s2);
                s3 = fma(sv[q + 96], colk[q + 96], s3);
            }
            for (; q < rows; q += 32) s0 = fma(sv[q], colk[q], s0);
            const double s = warp_sum((s0 + s1) + (s2 + s3));
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
            double* colk = a.W + (int64_t)k * a.m + r0;
            const double wk = a.wv[k];
            // rows i < j of this block are untouched (sv = 0 there)
            double s = 0.0;
            int64_t q = lane;
            for (; q + 96 < rows; q += 128) {
                double x[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) x[u] = colk[q + 32 * u];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int64_t i = r0 + q + 32 * u;
                    if (i >= j) {
                        x[u] = fma(-sv[q + 32 * u], wk, x[u]);
                        colk[q + 32 * u] = x[u];
                    }
                    if (k == j + 1 && i >= j + 1) s = fma(x[u], x[u], s);
                }
            }
            for (; q < rows; q += 32) {
                const int64_t i = r0 + q;
                double x = colk[q];
                if (i >= j) {
                    x = fma(-sv[q], wk, x);
                    colk[q] = x;
                }
                if (k == j + 1 && i >= j + 1) s = fma(x, x, s);
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

// ---------------------------------------------------------------- blocked Householder QR (float64)
//
// The same reflectors in panels of kQrB columns (compact WY form, as in
// LAPACK's dgeqrf / dlarft / dlarfb): the panel's columns are factored one at
// a time as above, but each reflector is applied only to the rest of the
// panel; then the panel's product Q_p = I - V T V^T is applied to all trailing
// columns at once, W_t <- W_t - V (T^T (V^T W_t)).  Each CTA keeps the
// reflectors' entries for its own rows in shared memory (V, rows x kQrB), so
// the trailing matrix is read and written once per panel instead of once per
// column.  Reductions over CTAs are in a fixed order (deterministic).
constexpr int kQrB = 32;         // panel width
constexpr int kQrVs = kQrB + 1;  // row stride of V in shared memory (doubles)

struct QrbArgs {
    double* W;        // column-major m x nc
    int64_t m;
    int d, nc;
    double* normp;    // [2][grid] partial squared norms (double-buffered by column parity)
    double* dotp;     // [2][grid][kQrB] partial raw dots inside a panel
    double* rowv;     // [2][kQrB] row j of the panel, published by its owner block
    double* Pp;       // [grid][nc][kQrB] partial V^T W_t
    double* VtVp;     // [grid][kQrB][kQrB] partial V^T V
    double* P;        // [nc][kQrB] V^T W_t
    double* T;        // [kQrB][kQrB] the panel's T
    double* Y;        // [nc][kQrB] T^T V^T W_t
    unsigned* bar;
    unsigned* tflag;
};

__global__ void __launch_bounds__(1024) k_qr_blocked(QrbArgs a) {
    extern __shared__ double V[];  // [rows][kQrVs]: this block's rows of the panel's reflectors
    __shared__ double s_red[32];
    __shared__ double stau[kQrB];
    __shared__ double swv[kQrB];
    __shared__ double sT[kQrB][kQrB + 1];
    __shared__ double sVV[kQrB][kQrB + 1];
    const unsigned G = gridDim.x;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, nwarps = blockDim.x >> 5;
    const int64_t per = (a.m + G - 1) / G;
    const int64_t r0 = (per * blockIdx.x < a.m) ? per * blockIdx.x : a.m;
    const int64_t r1 = (r0 + per < a.m) ? r0 + per : a.m;
    const int rows = (int)(r1 - r0);

    // Partials of column j for its reflector, over this block's rows, into
    // buffer (j & 1): ||W[i >= j, j]||^2 and, for k in (j, kend), the raw dots
    // sum_{i > j} W[i][j] W[i][k].  With v = (1 at j, W[i][j] * vscale below),
    // v^T W[:, k] = W[j][k] + vscale * (raw dot), so the dots are formed before
    // the column's scale is known and one grid barrier per column suffices.
    auto column_partials = [&](int j, int kend) {
        const int buf = j & 1;
        const double* colj = a.W + (int64_t)j * a.m + r0;
        double s = 0.0;
        if (warp * 32 < rows) {   // warps without rows skip the float64 shuffle tree
            for (int q = tid; q < rows; q += blockDim.x) {
                const int64_t i = r0 + q;
                if (i >= j) s = fma(colj[q], colj[q], s);
            }
            s = warp_sum(s);
        }
        if (lane == 0) s_red[warp] = s;
        for (int k = j + 1 + warp; k < kend; k += nwarps) {
            const double* colk = a.W + (int64_t)k * a.m + r0;
            double t0 = 0.0, t1 = 0.0;
            for (int q = lane; q < rows; q += 64) {
                if (r0 + q > j) t0 = fma(colj[q], colk[q], t0);
                if (q + 32 < rows && r0 + q + 32 > j) t1 = fma(colj[q + 32], colk[q + 32], t1);
            }
            const double t = warp_sum(t0 + t1);
            if (lane == 0) a.dotp[((size_t)buf * G + blockIdx.x) * kQrB + (k - (j / kQrB) * kQrB)] = t;
        }
        // the block owning row j publishes W[j][j .. kend): every block reads
        // them after the barrier while the owner goes on to overwrite row j
        if (j >= r0 && j < r1)
            for (int k = j + tid; k < kend; k += blockDim.x)
                a.rowv[buf * kQrB + (k - (j / kQrB) * kQrB)] = a.W[(int64_t)k * a.m + j];
        __syncthreads();
        if (tid == 0) {
            double t = 0.0;
            for (int w = 0; w < nwarps; ++w) t += s_red[w];
            a.normp[buf * G + blockIdx.x] = t;
        }
    };

    column_partials(0, min(kQrB, a.d));
    if (!grid_barrier(a.bar, G, a.tflag)) return;

    for (int j0 = 0; j0 < a.d; j0 += kQrB) {
        const int bb = min(kQrB, a.d - j0);
        const int jend = j0 + bb;
        // ---- the panel, one column (one grid barrier) at a time
        for (int j = j0; j < jend; ++j) {
            const int jl = j - j0, buf = j & 1;
            // ||column j||^2: lanes over blocks, then the warp's tree (the same
            // fixed order in every block)
            // and the reflector's scalars, formed once: float64 square roots and
            // divisions are long sequences on a part with little float64 rate, so
            // one thread forms them and the block reads them from shared memory
            if (warp == 0) {
                double t = 0.0;
                for (unsigned c = lane; c < G; c += 32) t += a.normp[buf * G + c];
                t = warp_sum(t);
                if (lane == 0) {
                    const double sig2 = t;
                    const double ajj = a.rowv[buf * kQrB + jl];
                    double beta = 0.0, tau = 0.0, vscale = 0.0;
                    if (sig2 != 0.0) {
                        const double sig = sqrt(sig2);
                        beta = ajj >= 0.0 ? -sig : sig;
                        tau = (beta - ajj) / beta;
                        vscale = 1.0 / (ajj - beta);
                    }
                    s_red[0] = beta;
                    s_red[1] = tau;
                    s_red[2] = vscale;
                    stau[jl] = tau;
                }
            }
            __syncthreads();
            const double beta = s_red[0], tau = s_red[1], vscale = s_red[2];
            const double* colj = a.W + (int64_t)j * a.m;
            for (int q = tid; q < rows; q += blockDim.x) {
                const int64_t i = r0 + q;
                V[q * kQrVs + jl] = (i < j) ? 0.0 : (i == j ? 1.0 : colj[i] * vscale);
            }
            // tau * v^T W[:, k] for k in (j, jend), the same in every block
            for (int k = j + 1 + warp; k < jend; k += nwarps) {
                double t = 0.0;
                for (unsigned c = lane; c < G; c += 32) t += a.dotp[((size_t)buf * G + c) * kQrB + (k - j0)];
                t = warp_sum(t);
                if (lane == 0) swv[k - j0] = tau * (a.rowv[buf * kQrB + (k - j0)] + vscale * t);
            }
            __syncthreads();
            // apply the reflector to the rest of the panel (this block's rows i >= j)
            for (int k = j + 1 + warp; k < jend; k += nwarps) {
                double* colk = a.W + (int64_t)k * a.m + r0;
                const double wk = swv[k - j0];
                for (int q = lane; q < rows; q += 32)
                    if (r0 + q >= j) colk[q] = fma(-V[q * kQrVs + jl], wk, colk[q]);
            }
            if (tid == 0 && j >= r0 && j < r1) a.W[(int64_t)j * a.m + j] = beta;  // R_jj
            __syncthreads();
            if (j + 1 < jend) {
                column_partials(j + 1, jend);
                if (!grid_barrier(a.bar, G, a.tflag)) return;
            }
        }
        const int ntr = a.nc - jend;  // trailing columns (with the carried Sb)
        if (ntr <= 0) break;
        __syncthreads();
        // ---- partial V^T V and V^T W_t over this block's rows
        for (int ap = warp; ap < bb; ap += nwarps) {
            double acc = 0.0;
            if (lane < bb)
                for (int q = 0; q < rows; ++q) acc = fma(V[q * kQrVs + lane], V[q * kQrVs + ap], acc);
            a.VtVp[((size_t)blockIdx.x * kQrB + ap) * kQrB + lane] = acc;
        }
        for (int t = warp; t < ntr; t += nwarps) {
            const int k = jend + t;
            const double* colk = a.W + (int64_t)k * a.m + r0;
            double acc = 0.0;
            for (int q0 = 0; q0 < rows; q0 += 32) {
                const double w = (q0 + lane < rows) ? colk[q0 + lane] : 0.0;
                const int nq = min(32, rows - q0);
                for (int u = 0; u < nq; ++u) {
                    const double wu = __shfl_sync(0xFFFFFFFFu, w, u);
                    if (lane < bb) acc = fma(V[(q0 + u) * kQrVs + lane], wu, acc);
                }
            }
            a.Pp[((size_t)blockIdx.x * a.nc + k) * kQrB + lane] = acc;
        }
        if (!grid_barrier(a.bar, G, a.tflag)) return;
        // ---- reductions over blocks; block 0 also forms T
        for (int t = blockIdx.x * nwarps + warp; t < ntr; t += G * nwarps) {
            const int k = jend + t;
            double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;  // four chains, fixed order
            unsigned c = 0;
            for (; c + 3 < G; c += 4) {
                s0 += a.Pp[((size_t)c * a.nc + k) * kQrB + lane];
                s1 += a.Pp[((size_t)(c + 1) * a.nc + k) * kQrB + lane];
                s2 += a.Pp[((size_t)(c + 2) * a.nc + k) * kQrB + lane];
                s3 += a.Pp[((size_t)(c + 3) * a.nc + k) * kQrB + lane];
            }
            for (; c < G; ++c) s0 += a.Pp[((size_t)c * a.nc + k) * kQrB + lane];
            a.P[(size_t)k * kQrB + lane] = (s0 + s1) + (s2 + s3);
        }
        if (blockIdx.x == 0) {
            __syncthreads();
            for (int ap = warp; ap < bb; ap += nwarps) {
                double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
                unsigned c = 0;
                for (; c + 3 < G; c += 4) {
                    s0 += a.VtVp[((size_t)c * kQrB + ap) * kQrB + lane];
                    s1 += a.VtVp[((size_t)(c + 1) * kQrB + ap) * kQrB + lane];
                    s2 += a.VtVp[((size_t)(c + 2) * kQrB + ap) * kQrB + lane];
                    s3 += a.VtVp[((size_t)(c + 3) * kQrB + ap) * kQrB + lane];
                }
                for (; c < G; ++c) s0 += a.VtVp[((size_t)c * kQrB + ap) * kQrB + lane];
                sVV[ap][lane] = (s0 + s1) + (s2 + s3);
            }
            __syncthreads();
            if (warp == 0) {
                // T upper triangular: T_aa = tau_a, T[0:a, a] = -tau_a T[0:a, 0:a] (V^T v_a)[0:a]
                for (int c2 = 0; c2 < bb; ++c2) {
                    double z = 0.0;
                    if (lane < c2)
                        for (int x = lane; x < c2; ++x) z = fma(sT[lane][x], sVV[x][c2], z);
                    __syncwarp();
                    if (lane < c2) sT[lane][c2] = -stau[c2] * z;
                    else if (lane == c2) sT[c2][c2] = stau[c2];
                    else sT[lane][c2] = 0.0;
                    __syncwarp();
                }
                for (int x = 0; x < kQrB; ++x) a.T[x * kQrB + lane] = (x < bb && lane < bb) ? sT[x][lane] : 0.0;
            }
        }
        if (!grid_barrier(a.bar, G, a.tflag)) return;
        // ---- Y = T^T P for the trailing columns (distributed)
        for (int e = tid; e < kQrB * kQrB; e += blockDim.x) sT[e / kQrB][e % kQrB] = a.T[e];
        __syncthreads();
        for (int t = blockIdx.x * nwarps + warp; t < ntr; t += G * nwarps) {
            const int k = jend + t;
            const double p = a.P[(size_t)k * kQrB + lane];
            double y = 0.0;
            for (int x = 0; x < bb; ++x) {
                const double px = __shfl_sync(0xFFFFFFFFu, p, x);
                if (x <= lane) y = fma(sT[x][lane], px, y);
            }
            a.Y[(size_t)k * kQrB + lane] = (lane < bb) ? y : 0.0;
        }
        if (!grid_barrier(a.bar, G, a.tflag)) return;
        // ---- W_t -= V Y over this block's rows, then the next panel's first
        // column partials
        for (int t = warp; t < ntr; t += nwarps) {
            const int k = jend + t;
            const double yl = a.Y[(size_t)k * kQrB + lane];
            double* colk = a.W + (int64_t)k * a.m + r0;
            for (int q0 = 0; q0 < rows; q0 += 32) {
                const int q = q0 + lane;
                double acc = 0.0;
                for (int x = 0; x < bb; ++x) {
                    const double yx = __shfl_sync(0xFFFFFFFFu, yl, x);
                    if (q < rows) acc = fma(V[q * kQrVs + x], yx, acc);
                }
                if (q < rows) colk[q] -= acc;
            }
        }
        __syncthreads();
        if (jend < a.d) column_partials(jend, min(jend + kQrB, a.d));
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

// x = R^-1 rhs for upper-triangular row-major R (one CTA, column sweep).  The
// reciprocals of the diagonal are formed first, one division per thread in
// parallel (float64 divisions are long sequences on this part).
__global__ void k_trsv_upper(const double* __restrict__ R, int d, const double* __restrict__ rhs,
                             double* __restrict__ x) {
    extern __shared__ double sx[];
    double* rinv = sx + d;
    for (int i = threadIdx.x; i < d; i += blockDim.x) {
        sx[i] = rhs[i];
        rinv[i] = 1.0 / R[(int64_t)i * d + i];
    }
    __syncthreads();
    for (int j = d - 1; j >= 0; --j) {
        if (threadIdx.x == 0) sx[j] = sx[j] * rinv[j];
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
    double* rinv = sx + d;   // reciprocals of the diagonal, formed in parallel
    const int col = blockIdx.x;
    for (int i = threadIdx.x; i < d; i += blockDim.x) {
        sx[i] = B ? B[(int64_t)i * k + col] : (i == col ? 1.0 : 0.0);
        rinv[i] = 1.0 / R[(int64_t)i * d + i];
    }
    __syncthreads();
    for (int j = d - 1; j >= 0; --j) {
        if (threadIdx.x == 0) sx[j] = sx[j] * rinv[j];
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
    // the stage of 16 rows x 128 columns of each operand: a thread holds 2 x 4
    // floats of each; the next stage's loads are in flight during this one's products
    float4 va[2], vb[2];
    float sbv = 0.f;
    auto load_stage = [&](int64_t rb) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int q = threadIdx.x + 256 * h;   // 0..511 -> (row kk, column quad cq)
            const int kk = q >> 5, cq = (q & 31) * 4;
            const int64_t r = rb + kk;
            va[h] = make_float4(0.f, 0.f, 0.f, 0.f);
            vb[h] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (r < r1) {
                const float* row = SA + r * d;
                if (vec && ci0 + cq + 3 < d) {
                    va[h] = *reinterpret_cast<const float4*>(row + ci0 + cq);
                } else {
                    va[h].x = ci0 + cq < d ? row[ci0 + cq] : 0.f;
                    va[h].y = ci0 + cq + 1 < d ? row[ci0 + cq + 1] : 0.f;
                    va[h].z = ci0 + cq + 2 < d ? row[ci0 + cq + 2] : 0.f;
                    va[h].w = ci0 + cq + 3 < d ? row[ci0 + cq + 3] : 0.f;
                }
                if (vec && cj0 + cq + 3 < d) {
                    vb[h] = *reinterpret_cast<const float4*>(row + cj0 + cq);
                } else {
                    vb[h].x = cj0 + cq < d ? row[cj0 + cq] : 0.f;
                    vb[h].y = cj0 + cq + 1 < d ? row[cj0 + cq + 1] : 0.f;
                    vb[h].z = cj0 + cq + 2 < d ? row[cj0 + cq + 2] : 0.f;
                    vb[h].w = cj0 + cq + 3 < d ? row[cj0 + cq + 3] : 0.f;
                }
            }
        }
        if (Sb && ti == tj && threadIdx.x < kGK) sbv = (rb + threadIdx.x < r1) ? Sb[rb + threadIdx.x] : 0.f;
    };
    if (r0 < r1) load_stage(r0);
    for (int64_t rb = r0; rb < r1; rb += kGK) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int q = threadIdx.x + 256 * h;
            const int kk = q >> 5, cq = (q & 31) * 4;
            *reinterpret_cast<float4*>(&As[kk][cq]) = va[h];
            *reinterpret_cast<float4*>(&Bs[kk][cq]) = vb[h];
        }
        if (Sb && ti == tj && threadIdx.x < kGK) Ss[threadIdx.x] = sbv;
        __syncthreads();
        if (rb + kGK < r1) load_stage(rb + kGK);
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
// row j of R reach the other lanes by shuffles; 1 / R_jj from one reciprocal
// square root (two roundings; the factor is a preconditioner).  Returns false,
// the same on every lane, when a pivot is not positive.  rinv_out (lane j)
// receives 1 / R_jj.
__device__ __forceinline__ bool chol_block32(float (&col)[kCholB], int pb, float& rinv_out) {
    const int lane = threadIdx.x & 31;
    bool ok = true;
    rinv_out = 1.f;
#pragma unroll
    for (int j = 0; j < kCholB; ++j) {
        const float piv = __shfl_sync(0xFFFFFFFFu, col[j], j);
        if (j < pb) {
            if (!(piv > 0.f)) ok = false;
            const float rinv = rsqrtf(piv);
            if (lane == j) {
                col[j] = piv * rinv;
                rinv_out = rinv;
            } else if (lane > j) {
                col[j] *= rinv;
            }
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

// Rows of the shared-memory copy of a diagonal block: 16-byte aligned, so that
// a row can be read back as 16-byte broadcasts.
constexpr int kDgStride = kCholB + 4;

// chol_block32 with the scaled row j published to Dg[j][.] in shared memory at
// each pivot and read back by every lane as 16-byte broadcasts for the update
// (one store and at most eight loads per pivot instead of 31 shuffles); the
// arithmetic and its order are those of chol_block32.  Dg ends up holding R.
__device__ __forceinline__ bool chol_block32_rows(float (&col)[kCholB], int pb, float& rinv_out,
                                                  float (*Dg)[kDgStride]) {
    const int lane = threadIdx.x & 31;
    bool ok = true;
    rinv_out = 1.f;
#pragma unroll
    for (int j = 0; j < kCholB; ++j) {
        const float piv = __shfl_sync(0xFFFFFFFFu, col[j], j);
        if (j < pb) {
            if (!(piv > 0.f)) ok = false;
            const float rinv = rsqrtf(piv);
            if (lane == j) {
                col[j] = piv * rinv;
                rinv_out = rinv;
            } else if (lane > j) {
                col[j] *= rinv;
            }
        }
        Dg[j][lane] = col[j];
        __syncwarp();
        if (j < pb) {
            const float rjk = col[j];
#pragma unroll
            for (int i4 = (j + 1) & ~3; i4 < kCholB; i4 += 4) {
                const float4 r = *reinterpret_cast<const float4*>(&Dg[j][i4]);
                const float rv[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int i = i4 + u;
                    if (i > j && lane >= i) col[i] = fmaf(-rv[u], rjk, col[i]);
                }
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
        float rinv_unused;
        const bool ok = chol_block32(col, pb, rinv_unused);
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

// Warp 0: the diagonal block of panel p0 (pb columns) from P into registers,
// factored by chol_block32_rows (which leaves R in Dg), written back to P, with 1 / R_jj in
// Dinv.  Not inlined, so its 32 registers of column do not add to the
// kernel's peak.  Returns false (every lane) on a non-positive pivot.
__device__ __noinline__ bool chol_small_diag(float* P, float (*Dg)[kDgStride], float* Dinv, int nc, int p0,
                                             int pb) {
    const int lane = threadIdx.x & 31;
    float col[kCholB];
#pragma unroll
    for (int q = 0; q < kCholB; ++q) col[q] = (q <= lane && lane < pb) ? P[chol_off(p0 + q, nc) + p0 + lane] : 0.f;
    float rinv;
    const bool ok = chol_block32_rows(col, pb, rinv, Dg);
#pragma unroll
    for (int q = 0; q < kCholB; ++q)
        if (q <= lane && lane < pb) P[chol_off(p0 + q, nc) + p0 + lane] = col[q];
    Dinv[lane] = rinv;
    return ok;
}

// Column k (>= s0) of the panel rows right of the diagonal block: R_pp^T x =
// P[p0.., k] by forward substitution in registers, rows 0..15 then 16..31;
// the result goes to P and densely to Pan (zero past the last column, nc <= k
// < s0 + tp, and below row pb).  Not inlined: the caller's loop would
// otherwise hoist the Dg loads and spill.
__device__ __noinline__ void chol_small_panel(float* P, float* Pan, const float (*Dg)[kDgStride],
                                              const float* Dinv, int nc, int p0, int pb, int s0, int tp, int k) {
    // rows 0..15 of the panel, then rows 16..31 (fewer live registers)
    float x[16], y[16];
    const bool live = k < nc;
    int o = chol_off(p0, nc) + k;
#pragma unroll
    for (int q = 0; q < 16; ++q) {
        x[q] = (live && q < pb) ? P[o] : 0.f;
        o += nc - (p0 + q) - 1;
    }
    const int o16 = o;
#pragma unroll
    for (int q = 0; q < 16; ++q) {
        x[q] *= Dinv[q];
#pragma unroll
        for (int i = 0; i < 16; ++i)
            if (i > q) x[i] = fmaf(-Dg[q][i], x[q], x[i]);
    }
#pragma unroll
    for (int q = 0; q < 16; ++q) {
        y[q] = (live && 16 + q < pb) ? P[o] : 0.f;
        o += nc - (p0 + 16 + q) - 1;
    }
#pragma unroll
    for (int q = 0; q < 16; ++q)
#pragma unroll
        for (int i = 0; i < 16; ++i) y[i] = fmaf(-Dg[q][16 + i], x[q], y[i]);
#pragma unroll
    for (int q = 0; q < 16; ++q) {
        y[q] *= Dinv[16 + q];
#pragma unroll
        for (int i = 0; i < 16; ++i)
            if (i > q) y[i] = fmaf(-Dg[16 + q][16 + i], y[q], y[i]);
    }
    o = chol_off(p0, nc) + k;
#pragma unroll
    for (int q = 0; q < 16; ++q) {
        if (live && q < pb) P[o] = x[q];
        o += nc - (p0 + q) - 1;
        Pan[q * tp + (k - s0)] = (q < pb) ? x[q] : 0.f;
    }
    o = o16;
#pragma unroll
    for (int q = 0; q < 16; ++q) {
        if (live && 16 + q < pb) P[o] = y[q];
        o += nc - (p0 + 16 + q) - 1;
        Pan[(16 + q) * tp + (k - s0)] = (16 + q < pb) ? y[q] : 0.f;
    }
}

// Pan: the panel's rows of R right of the diagonal block, dense (row q at
// Pan + q * tp, column k - s0), zero past the last column; the trailing
// update is then a rank-32 product with 8 x 8 register tiles and 16-byte
// shared-memory operand loads.
__global__ void __launch_bounds__(512) k_chol_small(float* __restrict__ W, int d, int nc, int tpmax,
                                                   unsigned* bad) {
    extern __shared__ __align__(16) float P[];
    __shared__ __align__(16) float Dg[kCholB][kDgStride];   // R of the current diagonal block
    __shared__ float Dinv[kCholB];             // 1 / its diagonal
    __shared__ int fail;
    const int tid = threadIdx.x, nt = blockDim.x, warp = tid >> 5, lane = tid & 31, nw = nt >> 5;
    const int psz = ((nc * (nc + 1) / 2) + 3) & ~3;
    float* Pan = P + psz;                      // [kCholB][tpmax]
    for (int i = warp; i < nc; i += nw) {      // row i of the upper triangle, one warp per row
        float* dst = P + chol_off(i, nc);
        const float* src = W + (int64_t)i * nc;
        for (int k = i + lane; k < nc; k += 32) cp_async4(dst + k, src + k);
    }
    cp_async_wait_all();
    if (tid == 0) fail = 0;
    __syncthreads();
    for (int p0 = 0; p0 < d; p0 += kCholB) {
        const int pb = min(kCholB, d - p0);
        const int s0 = p0 + pb;
        if (warp == 0 && !chol_small_diag(P, Dg, Dinv, nc, p0, pb) && lane == 0) {
            fail = 1;
            atomicExch(bad, 1u);
        }
        __syncthreads();
        if (fail) return;
        if (s0 >= nc) break;
        // panel rows right of the block: R_pp^T x = P[p0.., k] by forward
        // substitution in registers (thread = column); the result goes to P and
        // densely to Pan (zero past the last column and below row pb)
        const int T = nc - s0, tp = (T + 7) & ~7;
        for (int k = s0 + tid; k < s0 + tp; k += nt) chol_small_panel(P, Pan, Dg, Dinv, nc, p0, pb, s0, tp, k);
        __syncthreads();
        if (s0 >= d) break;
        // 8 x 8 tiles (ti <= tk) of the trailing upper triangle, rows < d
        const int nti = (d - s0 + 7) / 8, ntk = tp / 8;
        const int ntiles = nti * ntk - nti * (nti - 1) / 2;
        for (int t = tid; t < ntiles; t += nt) {
            int ti = 0, rem = t;
            while (rem >= ntk - ti) {
                rem -= ntk - ti;
                ++ti;
            }
            const int tk = ti + rem;
            float acc[8][8];
#pragma unroll
            for (int r = 0; r < 8; ++r)
#pragma unroll
                for (int c = 0; c < 8; ++c) acc[r][c] = 0.f;
            const float* pa = Pan + 8 * ti;
            const float* pk = Pan + 8 * tk;
            for (int q = 0; q < pb; ++q) {
                const float4 a0 = *reinterpret_cast<const float4*>(pa + q * tp);
                const float4 a1 = *reinterpret_cast<const float4*>(pa + q * tp + 4);
                const float4 b0 = *reinterpret_cast<const float4*>(pk + q * tp);
                const float4 b1 = *reinterpret_cast<const float4*>(pk + q * tp + 4);
                const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
                const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
                for (int r = 0; r < 8; ++r)
#pragma unroll
                    for (int c = 0; c < 8; ++c) acc[r][c] = fmaf(av[r], bv[c], acc[r][c]);
            }
#pragma unroll
            for (int r = 0; r < 8; ++r) {
                const int i = s0 + 8 * ti + r;
                if (i >= d) break;
                float* row = P + chol_off(i, nc);
                float cur[8];
#pragma unroll
                for (int c = 0; c < 8; ++c) {   // the row's eight values first, then the stores
                    const int k = s0 + 8 * tk + c;
                    cur[c] = (k >= i && k < nc) ? row[k] : 0.f;
                }
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    const int k = s0 + 8 * tk + c;
                    if (k >= i && k < nc) row[k] = cur[c] - acc[r][c];
                }
            }
        }
        __syncthreads();
    }
    for (int i = warp; i < nc; i += nw) {
        const float* src = P + chol_off(i, nc);
        float* dst = W + (int64_t)i * nc;
        for (int k = i + lane; k < nc; k += 32) dst[k] = src[k];
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

// ---- blocked inverse of the float32 Cholesky factor (blocks of 32) -------
//
// With R = [R_IK] in 32 x 32 blocks, the blocks of M = R^-1 satisfy
// M_II = R_II^-1 and, for I < J, M_IJ = -M_II sum_{K=I+1..J} R_IK M_KJ.
// k_tri_diag_inv forms every M_II (one warp each, lane c back-substitutes
// column c); k_tri_inv_blk then builds block column J in one CTA, from block
// row J - 1 up to block row 0, each step a 32 x 32 product over the blocks
// already found and a multiply by M_II.

__global__ void __launch_bounds__(32) k_tri_diag_inv(const float* __restrict__ W, int d, int nc,
                                                    float* __restrict__ Dinv) {
    __shared__ float Rb[kCholB][kCholB + 1];
    __shared__ float X[kCholB][kCholB + 1];
    const int I = blockIdx.x, lane = threadIdx.x;
    const int i0 = I * kCholB, ib = min(kCholB, d - i0);
    for (int r = 0; r < kCholB; ++r)
        Rb[r][lane] = (r < ib && lane < ib && lane >= r) ? W[(int64_t)(i0 + r) * nc + i0 + lane] : 0.f;
    __syncwarp();
    // column c = lane of R_II^-1: x_c = 1 / R_cc, x_i = -(sum_{i<k<=c} R_ik x_k) / R_ii
    const int c = lane;
    for (int r = 0; r < kCholB; ++r) X[r][c] = 0.f;
    if (c < ib) {
        X[c][c] = 1.f / Rb[c][c];
        for (int i = c - 1; i >= 0; --i) {
            float sacc = 0.f;
            for (int k = i + 1; k <= c; ++k) sacc = fmaf(Rb[i][k], X[k][c], sacc);
            X[i][c] = -sacc / Rb[i][i];
        }
    }
    __syncwarp();
    float* out = Dinv + (size_t)I * kCholB * kCholB;
    for (int r = 0; r < kCholB; ++r) out[r * kCholB + lane] = X[r][lane];
}

__global__ void __launch_bounds__(256) k_tri_inv_blk(const float* __restrict__ W, int d, int nc,
                                                    const float* __restrict__ Dinv, double* __restrict__ M,
                                                    float* __restrict__ M32T) {
    extern __shared__ __align__(16) float sh[];
    const int J = blockIdx.x, tid = threadIdx.x;
    const int j0 = J * kCholB, jb = min(kCholB, d - j0);
    const int rows = j0 + kCholB;                 // block rows 0..J of the column block
    const int rw = j0 + 1;
    float* Mc = sh;                               // [rows][32]: M_KJ, K <= J
    float* T = Mc + (size_t)rows * kCholB;        // [32][33]
    float* Dv = T + kCholB * (kCholB + 1);        // [J + 1][32][32]: M_II
    float* Rb0 = Dv + (size_t)(J + 1) * kCholB * kCholB;   // two buffers [32][rw]: block row I of R
    float* Rb1 = Rb0 + (size_t)kCholB * rw;
    // block row I of R, columns 32 (I + 1) .. j0 + jb - 1, into buf (4-byte async copies)
    auto load_row = [&](int I, float* buf) {
        const int i0 = I * kCholB, k0 = i0 + kCholB, w = j0 + jb - k0;
        for (int q = tid; q < kCholB * w; q += blockDim.x) {
            const int r = q / w, k = q - r * w;
            cp_async4(buf + r * rw + k, W + (int64_t)(i0 + r) * nc + k0 + k);
        }
    };
    for (int q = tid; q < (J + 1) * kCholB * kCholB; q += blockDim.x) cp_async4(Dv + q, Dinv + q);
    if (J >= 1) load_row(J - 1, Rb0);
    cp_async_commit();
    for (int q = tid; q < rows * kCholB; q += blockDim.x) {
        const int r = q / kCholB, c = q % kCholB;
        Mc[q] = (r >= j0 && r - j0 < jb && c < jb) ? Dinv[(size_t)J * kCholB * kCholB + (r - j0) * kCholB + c] : 0.f;
    }
    const int tr = tid >> 3, tc = (tid & 7) * 4;  // T rows tr, columns tc .. tc + 3
    int buf = 0;
    for (int I = J - 1; I >= 0; --I) {
        float* Rb = buf ? Rb1 : Rb0;
        if (I >= 1) load_row(I - 1, buf ? Rb0 : Rb1);   // next block row, in flight during this step
        cp_async_commit();
        cp_async_wait<1>();
        __syncthreads();
        const int i0 = I * kCholB;
        const int k0 = i0 + kCholB, w = j0 + jb - k0;
        float t0 = 0.f, t1 = 0.f, t2 = 0.f, t3 = 0.f;
        const float* rrow = Rb + tr * rw;
        const float* mrow = Mc + (size_t)k0 * kCholB + tc;
#pragma unroll 4
        for (int k = 0; k < w; ++k) {
            const float rv = rrow[k];
            const float4 mv = *reinterpret_cast<const float4*>(mrow + (size_t)k * kCholB);
            t0 = fmaf(rv, mv.x, t0);
            t1 = fmaf(rv, mv.y, t1);
            t2 = fmaf(rv, mv.z, t2);
            t3 = fmaf(rv, mv.w, t3);
        }
        T[tr * (kCholB + 1) + tc] = t0;
        T[tr * (kCholB + 1) + tc + 1] = t1;
        T[tr * (kCholB + 1) + tc + 2] = t2;
        T[tr * (kCholB + 1) + tc + 3] = t3;
        __syncthreads();
        const float* dinv = Dv + (size_t)I * kCholB * kCholB + tr * kCholB;
        float m0 = 0.f, m1 = 0.f, m2 = 0.f, m3 = 0.f;
        for (int q = tr; q < kCholB; ++q) {
            const float dv = dinv[q];
            m0 = fmaf(dv, T[q * (kCholB + 1) + tc], m0);
            m1 = fmaf(dv, T[q * (kCholB + 1) + tc + 1], m1);
            m2 = fmaf(dv, T[q * (kCholB + 1) + tc + 2], m2);
            m3 = fmaf(dv, T[q * (kCholB + 1) + tc + 3], m3);
        }
        float* out = Mc + (size_t)(i0 + tr) * kCholB + tc;
        out[0] = -m0;
        out[1] = -m1;
        out[2] = -m2;
        out[3] = -m3;
        buf ^= 1;
    }
    cp_async_wait_all();
    __syncthreads();
    // column block J of M (float64, row-major) and of M32T (float32, column-major)
    for (int q = tid; q < d * kCholB; q += blockDim.x) {
        const int i = q / kCholB, c = q % kCholB;
        if (c >= jb) continue;
        const float v = (i < rows) ? Mc[(size_t)i * kCholB + c] : 0.f;
        M[(int64_t)i * d + j0 + c] = (double)v;
    }
    for (int q = tid; q < jb * d; q += blockDim.x) {
        const int c = q / d, i = q % d;
        M32T[(int64_t)(j0 + c) * d + i] = (i < rows) ? Mc[(size_t)i * kCholB + c] : 0.f;
    }
}

// M = R^-1 for upper-triangular row-major R (float64); one warp per column of
// M, RT = R^T (column j of R contiguous) for coalesced reads.
__global__ void k_tri_inverse(const double* __restrict__ RT, int d, double* __restrict__ M) {
    // reciprocals of the diagonal, one division per thread in parallel (float64
    // divisions are long sequences on this part; the sweep below multiplies)
    __shared__ double rinv[1024];
    for (int i = threadIdx.x; i < d; i += blockDim.x) rinv[i] = 1.0 / RT[(int64_t)i * d + i];
    __syncthreads();
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
        const double xj = __shfl_sync(0xFFFFFFFFu, sj, oj) * rinv[j];
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
    int g = num_sms() * per;   // one CTA of 32 warps per SM in practice
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
    const int threads = 1024;
    int G = qr_grid(m, threads, 48 * 1024);
    const size_t smem = sizeof(double) * (size_t)((m + G - 1) / G);
    if (smem > 200 * 1024) return CW_ERR_SHAPE;  // m too large for the resident-grid design
    // the blocked kernel when this block's rows of a panel fit in shared memory
    // (one CTA of 1024 threads per SM)
    int Gb = num_sms();
    if ((int64_t)Gb > (m + 63) / 64) Gb = (int)std::max<int64_t>(1, (m + 63) / 64);
    const size_t bsmem = sizeof(double) * (size_t)((m + Gb - 1) / Gb) * kQrVs;
    bool blocked = bsmem <= 180 * 1024;
    if (blocked) {
        int per_sm = 0;
        if (cudaFuncSetAttribute(k_qr_blocked, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bsmem) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_qr_blocked, threads, bsmem) != cudaSuccess ||
            per_sm < 1) {
            (void)cudaGetLastError();
            blocked = false;
        }
    }
    const int Gn = blocked ? Gb : G;
    Scratch ws(stream);
    const size_t oW = ws.reserve(sizeof(double) * (size_t)m * nc);
    const size_t oN = ws.reserve(sizeof(double) * (size_t)Gn * 2);
    const size_t oD = blocked ? 0 : ws.reserve(sizeof(double) * (size_t)G * nc);
    const size_t oV = blocked ? 0 : ws.reserve(sizeof(double) * (size_t)nc);
    const size_t oBd = blocked ? ws.reserve(sizeof(double) * (size_t)Gb * kQrB * 2) : 0;
    const size_t oBw = blocked ? ws.reserve(sizeof(double) * kQrB * 2) : 0;
    const size_t oPp = blocked ? ws.reserve(sizeof(double) * (size_t)Gb * nc * kQrB) : 0;
    const size_t oVV = blocked ? ws.reserve(sizeof(double) * (size_t)Gb * kQrB * kQrB) : 0;
    const size_t oP = blocked ? ws.reserve(sizeof(double) * (size_t)nc * kQrB) : 0;
    const size_t oT = blocked ? ws.reserve(sizeof(double) * kQrB * kQrB) : 0;
    const size_t oY = blocked ? ws.reserve(sizeof(double) * (size_t)nc * kQrB) : 0;
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
    if (blocked) {
        QrbArgs b{W, m, d, nc, ws.at<double>(oN), ws.at<double>(oBd), ws.at<double>(oBw), ws.at<double>(oPp),
                  ws.at<double>(oVV), ws.at<double>(oP), ws.at<double>(oT), ws.at<double>(oY), bar, bar + 2};
        CW_CUDA_TRY(cudaFuncSetAttribute(k_qr_blocked, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bsmem));
        void* args[] = {&b};
        {
            CW_PROF("k_qr_blocked", stream);
            CW_CUDA_TRY(cudaLaunchCooperativeKernel((void*)k_qr_blocked, dim3(Gb), dim3(threads), args, bsmem, stream));
        }
    } else {
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

// [SA | Sb]^T [SA | Sb] (float64, nc x nc, nc = d + (Sb != NULL)).  Does not
// synchronise; an MMA wait of the tensor-core kernel that gave up sets *tflag.
int gram_f64(const float* SA, int64_t m, int d, const float* Sb, double* Gm, unsigned* tflag, cudaStream_t stream,
             float* W32) {
    if (d < 1 || d > 1024) return CW_ERR_SHAPE;
    if (d <= 256) return gram_tc(SA, m, d, Sb, Gm, tflag, stream, W32);
    const int nc = d + (Sb ? 1 : 0);
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
    CW_CUDA_TRY(ws.alloc());
    double* part = ws.at<double>(oP);
    double* vpart = ws.at<double>(oV);
    const int64_t tot = (int64_t)nc * nc;
    {
        CW_PROF("k_gram_tile", stream);
        k_gram_tile<<<dim3((unsigned)ntl, (unsigned)nchunk), 256, 0, stream>>>(SA, Sb, m, d, ntile, (int)rows, part,
                                                                             vpart);
    }
    {
        CW_PROF("k_gram_reduce", stream);
        k_gram_reduce2<<<(unsigned)((tot + 255) / 256), 256, 0, stream>>>(part, vpart, nchunk, ntile, d, nc, Gm);
    }
    if (W32) {
        CW_PROF("k_gram_to_f32", stream);
        k_gram_to_f32<<<(unsigned)((tot + 255) / 256), 256, 0, stream>>>(Gm, tot, W32);
    }
    CW_LAUNCH_CHECK();
    return CW_OK;
}

// Gram + Cholesky + inverse for the LSQR preconditioner.  M (float64 d x d,
// float32 values), M32T (float32, column-major) and c = R^-T SA^T Sb; *kappa_lb
// receives the diagonal ratio of R.  Returns CW_ERR_RANK on a non-positive
// pivot.  Synchronises (the caller needs the ratio on the host).
int gram_chol_inverse(const float* SA, int64_t m, int d, const float* Sb, double* M, float* M32T, double* c,
                      float* kappa_lb_host, cudaStream_t stream, unsigned* flags_dev) {
    const int nc = d + (Sb ? 1 : 0);
    if (d > 1024) return CW_ERR_SHAPE;
    Scratch ws(stream);
    const size_t oG = ws.reserve(sizeof(double) * (size_t)nc * nc);
    const size_t oW = ws.reserve(sizeof(float) * (size_t)nc * nc);
    const size_t oF = ws.reserve(sizeof(unsigned) * 2 + sizeof(float) * 2);
    const int nb = (d + kCholB - 1) / kCholB;
    const size_t oD = ws.reserve(sizeof(float) * (size_t)nb * kCholB * kCholB);   // diagonal block inverses
    CW_CUDA_TRY(ws.alloc());
    double* Gm = ws.at<double>(oG);
    float* W = ws.at<float>(oW);
    float* Dinv = ws.at<float>(oD);
    unsigned* bad = ws.at<unsigned>(oF);
    float* klb = reinterpret_cast<float*>(bad + 2);
    CW_CUDA_TRY(cudaMemsetAsync(bad, 0, sizeof(unsigned) * 2 + sizeof(float) * 2, stream));
    // the Gram matrix in Gm (float64) and W (float32); bad[1]: an MMA wait of
    // the tensor-core Gram gave up
    int gst = gram_f64(SA, m, d, Sb, Gm, bad + 1, stream, W);
    if (gst != CW_OK) return gst;
    // one-CTA factorization when the packed triangle and a dense 32-row panel fit
    const int tpmax = (nc + 7) & ~7;
    const size_t psm = sizeof(float) * ((((size_t)nc * (nc + 1) / 2) + 3) & ~size_t(3)) +
                       sizeof(float) * (size_t)kCholB * tpmax;
    const bool small = psm + 6 * 1024 <= 227 * 1024 && nc <= 512;
    if (small) {
        CW_CUDA_TRY(cudaFuncSetAttribute(k_chol_small, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)psm));
        CW_PROF("k_chol_small", stream);
        k_chol_small<<<1, 512, psm, stream>>>(W, d, nc, tpmax, bad);
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
    // M = R^-1: diagonal block inverses, then one CTA per block column
    {
        {
            CW_PROF("k_tri_diag_inv", stream);
            k_tri_diag_inv<<<nb, 32, 0, stream>>>(W, d, nc, Dinv);
        }
        // Mc + T + the diagonal inverses + two block rows of R
        const size_t ism = sizeof(float) * ((size_t)nb * kCholB * kCholB + kCholB * (kCholB + 1) +
                                            (size_t)nb * kCholB * kCholB +
                                            2 * (size_t)kCholB * ((nb - 1) * kCholB + 1));
        if (ism <= 200 * 1024) {
            CW_CUDA_TRY(cudaFuncSetAttribute(k_tri_inv_blk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ism));
            CW_PROF("k_tri_inv_blk", stream);
            k_tri_inv_blk<<<nb, 256, ism, stream>>>(W, d, nc, Dinv, M, M32T);
        } else {   // large d: one warp per column of M, R read from global memory
            CW_PROF("k_tri_inv_f32", stream);
            k_tri_inv_f32<false><<<(d + 7) / 8, 256, sizeof(float) * 8 * 1024, stream>>>(W, d, nc, M, M32T);
        }
    }
    CW_LAUNCH_CHECK();
    if (flags_dev) {   // the caller reads the flags later
        CW_CUDA_TRY(cudaMemcpyAsync(flags_dev, bad, sizeof(unsigned) * 2 + sizeof(float) * 2, cudaMemcpyDeviceToDevice,
                                    stream));
        return CW_OK;
    }
    unsigned h[2] = {0, 0};
    float kl[2] = {0.f, 0.f};
    CW_CUDA_TRY(cudaMemcpyAsync(h, bad, sizeof(unsigned) * 2, cudaMemcpyDeviceToHost, stream));
    CW_CUDA_TRY(cudaMemcpyAsync(kl, klb, sizeof(float) * 2, cudaMemcpyDeviceToHost, stream));
    CW_CUDA_TRY(cudaStreamSynchronize(stream));
    if (kappa_lb_host) *kappa_lb_host = kl[0];
    if (h[1]) return CW_ERR_TIMEOUT;
    return h[0] ? CW_ERR_RANK : CW_OK;
}

int trsv_upper(const double* R, int d, const double* rhs, double* x, cudaStream_t stream) {
    {
        CW_PROF("k_trsv_upper", stream);
        k_trsv_upper<<<1, 256, sizeof(double) * 2 * (size_t)d, stream>>>(R, d, rhs, x);
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
        k_trsm_upper<<<k, 256, sizeof(double) * 2 * (size_t)d, stream>>>(R, d, B, k, X);
    }
    CW_LAUNCH_CHECK();
    return CW_OK;
}

}  // namespace cw

using namespace cw;

extern "C" int cw_gram(const float* SA, int64_t m, int64_t d, const float* Sb, double* G, cw_stream stream) {
    if (!SA || !G) return CW_ERR_ARG;
    if (d < 1 || d > 1024 || m < 1) return CW_ERR_SHAPE;
    if (m > 0x7FFFFFFFll) return CW_ERR_OVERFLOW;
    cudaStream_t s = (cudaStream_t)stream;
    unsigned* flag = nullptr;
    CW_CUDA_TRY(cudaMallocAsync(reinterpret_cast<void**>(&flag), sizeof(unsigned), s));
    int st = CW_OK;
    unsigned h = 0;
    if (cudaMemsetAsync(flag, 0, sizeof(unsigned), s) != cudaSuccess) st = CW_ERR_CUDA;
    if (st == CW_OK) st = gram_f64(SA, m, (int)d, Sb, G, flag, s);
    if (st == CW_OK && cudaMemcpyAsync(&h, flag, sizeof(unsigned), cudaMemcpyDeviceToHost, s) != cudaSuccess)
        st = CW_ERR_CUDA;
    cudaFreeAsync(flag, s);
    if (cudaStreamSynchronize(s) != cudaSuccess && st == CW_OK) st = CW_ERR_CUDA;
    if (st == CW_OK && h) st = CW_ERR_TIMEOUT;
    return st;
}

extern "C" int cw_qr(const float* SA, int64_t m, int64_t d, const float* Sb, double* R, double* c,
                     cw_stream stream) {
    if (!SA) return CW_ERR_ARG;
    if (d < 1 || d > 1024 || m < d) return CW_ERR_SHAPE;
    if (m > 0x7FFFFFFFll) return CW_ERR_OVERFLOW;
    return qr64(SA, m, (int)d, c ? Sb : nullptr, R, c, stream);
}
