// Batched sketch-and-solve: many independent least-squares problems of uneven
// n and d, each x'_p = argmin ||S_p A_p x - S_p b_p|| (Theorem "lin reg", one
// sparse embedding S_p of Section 2 per problem, its own m_p and seed).
//
// One plan per batch (cw_batch_create): problem descriptors, scratch, and a
// CUDA graph that holds the whole batch:
//   1. the batched sketch (sketch.cu): the eight stages of the single-problem
//      sketch, each launched once over all problems;
//   2. one persistent cooperative kernel, k_batch_solve, whose phases are
//      separated by bounded grid barriers:
//        A  Gram units: (problem, slab of S bucket rows) -> partial
//           SA^T SA and SA^T Sb of the slab's non-empty rows (float32
//           products and sums within the slab, float64 across slabs);
//        B  per problem: sum of its partials (fixed order), float64
//           Cholesky SA^T SA = L L^T, x0 = L^-T L^-1 SA^T Sb;
//        C  refinement units: r = Sb - SA x and the partial g = SA^T r over
//           the slab's rows in double-word float32 (~48-bit) arithmetic;
//        D  per problem: g summed in fixed order, delta = L^-T L^-1 g,
//           x += delta, converged when |delta|_inf <= 1e-13 |x|_inf or the
//           contraction over two steps puts the remaining error there;
//      C and D repeat up to `steps` times.
// L L^T is the Cholesky factorisation of the Gram matrix, so L^T is the R of a
// QR factorisation of SA with a positive diagonal (the factorisation of the
// proof of Theorem "renRegAlg"); the refinement with ~48-bit residuals (the
// corrected semi-normal equations of Bjorck, 1987) removes the float32 error
// of the Gram products, so x' is the least-squares solution of the float32 SA
// to about 1e-12.  A problem whose Cholesky pivot fails or whose refinement does
// not converge is flagged and re-solved by cw_batch_finish with the float64
// Householder QR.
//
// Slab size and CTAs per SM are chosen by timing candidates on the batch
// itself (CW_BATCH_AUTOTUNE); the choice can be cached in a text file named by
// the CW_TUNE_CACHE environment variable, keyed by a hash of the shapes.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "batch.h"
#include "cw.h"

namespace cw {

constexpr int kSolveThreads = 256;
constexpr int kMaxBatchD = 128;
constexpr int kMaxSlab = 4096;
constexpr int kChunkRows = 32;
constexpr int kStages = 4;      // row chunks in flight per work unit
constexpr int kMaxSteps = 4;  // refinement steps at most

struct SolveProb {
    int32_t d, m;
    int32_t unit0, nunits;  // this problem's units (contiguous in `units`)
    const float* SA;
    const float* Sb;
    const int32_t* bptr;  // m + 1 bucket starts (empty bucket <=> zero SA row)
    double* x;            // d (caller's)
    double* L;            // packed lower Cholesky factor, d (d + 1) / 2
    double* dprev;        // |delta|_inf of the previous refinement step
    int32_t* rowlist;     // m: per unit, its non-empty rows from position r0 (phase A)
    int32_t vec;          // SA rows can be copied in 16-byte pieces
    int64_t g0, gstride;  // partial Gram of unit unit0 + u at Gp + g0 + u * gstride
    int64_t v0, vstride;  // partial vector of unit unit0 + u at Vp + v0 + u * vstride
};

// sum over the problem's units of part[base + u * stride + e], four chains in a
// fixed order
__device__ __forceinline__ double sum_units(const double* __restrict__ part, int64_t base, int64_t stride, int n,
                                            int64_t e) {
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
    const double* p = part + base + e;
    int u = 0;
    for (; u + 3 < n; u += 4) {
        s0 += __ldg(p + (int64_t)u * stride);
        s1 += __ldg(p + (int64_t)(u + 1) * stride);
        s2 += __ldg(p + (int64_t)(u + 2) * stride);
        s3 += __ldg(p + (int64_t)(u + 3) * stride);
    }
    for (; u < n; ++u) s0 += __ldg(p + (int64_t)u * stride);
    return (s0 + s1) + (s2 + s3);
}

struct SolveUnit {
    int32_t p, r0, r1;
    int64_t goff;  // partial Gram (packed lower) in Gp
    int64_t voff;  // partial vector (c or g) in Vp
};

struct SolveArgs {
    const SolveProb* probs;
    const SolveUnit* units;
    const int32_t* uorder;  // units in decreasing estimated cost
    const int32_t* porder;  // problems in decreasing d
    int32_t count, nunits, steps;
    double* Gp;
    double* Vp;
    int32_t* status;        // per problem: 0 ok, 1 Cholesky failed, 2 not converged
    unsigned* conv;         // per problem: 1 when refinement is done
    unsigned* qctr;         // one work counter per phase (zeroed before launch)
    unsigned* bar;          // grid barrier words
    unsigned* tflag;        // barrier timeout flag
    unsigned long long* stamps;  // globaltimer (ns) at the start and after each phase, by CTA 0
    int32_t* ucount;        // per unit: number of non-empty rows (phase A)
};

__device__ __forceinline__ void stamp(const SolveArgs& S, int k) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        unsigned long long t;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
        S.stamps[k] = t;
    }
}

__device__ __forceinline__ int64_t tri(int64_t i) { return i * (i + 1) / 2; }

// Next item of a phase's queue for the whole CTA (-1 when none is left).
__device__ __forceinline__ int next_item(unsigned* ctr, int total, int* sh) {
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned v = atomicAdd(ctr, 1u);
        *sh = v < (unsigned)total ? (int)v : -1;
    }
    __syncthreads();
    return *sh;
}

// ---------------------------------------------------------------- row staging (phases A and C)

// Shared-memory layout of a unit: the slab's non-empty rows (compacted, in
// order), two buffers of 32 staged SA rows with their Sb, warp counts.
struct UnitSmem {
    int* rows;   // [kMaxSlab]
    float* tile; // [kStages][kChunkRows][ldt]
    float* tsb;  // [kStages][kChunkRows]
    int* wcnt;   // [16]
    int ldt;
};

__device__ __forceinline__ UnitSmem unit_smem(char* smem, int ldt) {
    UnitSmem u;
    u.rows = reinterpret_cast<int*>(smem);
    u.tile = reinterpret_cast<float*>(u.rows + kMaxSlab);
    u.tsb = u.tile + kStages * kChunkRows * ldt;
    u.wcnt = reinterpret_cast<int*>(u.tsb + kStages * kChunkRows);
    u.ldt = ldt;
    return u;
}

// Indices of the non-empty rows r0 <= r < r1 (bucket_ptr[r] < bucket_ptr[r + 1])
// in ascending order; returns their number.
__device__ int compact_rows(const SolveProb& P, int r0, int r1, const UnitSmem& u) {
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    int total = 0;
    for (int base = r0; base < r1; base += kSolveThreads) {
        const int r = base + tid;
        const bool ne = r < r1 && P.bptr[r] < P.bptr[r + 1];
        const unsigned bal = __ballot_sync(0xFFFFFFFFu, ne);
        if (lane == 0) u.wcnt[warp] = __popc(bal);
        __syncthreads();
        int off = total;
        for (int w = 0; w < warp; ++w) off += u.wcnt[w];
        if (ne) u.rows[off + __popc(bal & ((1u << lane) - 1u))] = r;
        int add = 0;
        for (int w = 0; w < kSolveThreads / 32; ++w) add += u.wcnt[w];
        __syncthreads();
        total += add;
    }
    return total;
}

// Asynchronous copy of compact rows c0 .. c0 + nr - 1 (d floats each) and
// their Sb into buffer `buf` (16-byte pieces when the rows allow it).
__device__ __forceinline__ void stage_rows(const SolveProb& P, const UnitSmem& u, int c0, int nr, int buf) {
    const int d = P.d, tid = threadIdx.x;
    float* tile = u.tile + buf * kChunkRows * u.ldt;
    if (P.vec) {
        const int q4 = d >> 2;
        for (int e = tid; e < nr * q4; e += kSolveThreads) {
            const int i = e / q4, j = (e - i * q4) * 4;
            cp_async16(tile + i * u.ldt + j, P.SA + (size_t)u.rows[c0 + i] * d + j);
        }
    } else {
        for (int e = tid; e < nr * d; e += kSolveThreads) {
            const int i = e / d, j = e - i * d;
            cp_async4(tile + i * u.ldt + j, P.SA + (size_t)u.rows[c0 + i] * d + j);
        }
    }
    if (tid < nr) cp_async4(u.tsb + buf * kChunkRows + tid, P.Sb + u.rows[c0 + tid]);
}

// Runs body(tile, tsb, nr) over the unit's non-empty rows, 32 at a time, with
// the copies of the next kStages - 1 chunks in flight while one is used (one
// commit group per chunk, empty past the end, so the wait count is fixed).
template <class F>
__device__ __forceinline__ void over_rows(const SolveProb& P, const UnitSmem& u, int total, F&& body) {
    const int nch = (total + kChunkRows - 1) / kChunkRows;
    if (nch == 0) return;
#pragma unroll
    for (int c = 0; c < kStages - 1; ++c) {
        if (c < nch) stage_rows(P, u, c * kChunkRows, min(kChunkRows, total - c * kChunkRows), c);
        cp_async_commit();
    }
    for (int c = 0; c < nch; ++c) {
        const int cn = c + kStages - 1;
        if (cn < nch) stage_rows(P, u, cn * kChunkRows, min(kChunkRows, total - cn * kChunkRows), cn % kStages);
        cp_async_commit();
        cp_async_wait<kStages - 1>();
        __syncthreads();
        const int b = c % kStages;
        body(u.tile + b * kChunkRows * u.ldt, u.tsb + b * kChunkRows, min(kChunkRows, total - c * kChunkRows));
        __syncthreads();
    }
    cp_async_wait<0>();
}

// ---------------------------------------------------------------- phase A

// Partial Gram of the unit's non-empty rows in T x T blocks of the lower
// triangle (16 block rows at most), spread over the warps so that no
// scheduler issues much more than one off-diagonal block's multiply-adds per
// row (warp w runs on scheduler w % 4): threads 0..119 take the off-diagonal
// blocks (jb > kb, T*T FMAs per row), threads 128..143 the lower triangles of
// the diagonal blocks (T(T+1)/2 FMAs), threads 160..255 form c = SA^T Sb
// (thread 160 + j for column j, then j + 96).  float32 sums over the slab;
// padding columns of the tiles are zero.
template <int T>
__device__ __noinline__ void gram_unit(const SolveArgs& S, int ui, const SolveUnit& U, char* smem) {
    constexpr int NT = T * T;  // accumulators: T*T (off-diagonal) or T(T+1)/2 (diagonal)
    const SolveProb& P = S.probs[U.p];
    const int d = P.d, tid = threadIdx.x;
    const int ldt = 16 * T + 4;
    const UnitSmem u = unit_smem(smem, ldt);
    const int total = compact_rows(P, U.r0, U.r1, u);
    // keep the list for the refinement passes
    for (int k = tid; k < total; k += kSolveThreads) P.rowlist[U.r0 + k] = u.rows[k];
    if (tid == 0) S.ucount[ui] = total;
    // zero the padding columns of all buffers once (copies never touch them)
    for (int e = tid; e < kStages * kChunkRows * (ldt - d); e += kSolveThreads) {
        const int i = e / (ldt - d), j = d + (e - i * (ldt - d));
        u.tile[i * ldt + j] = 0.f;
    }
    const int nbd = (d + T - 1) / T;
    const int nod = nbd * (nbd - 1) / 2;
    // role: 1 off-diagonal block (jb, kb), 2 diagonal blocks db, db + 1, 0 none
    int role = 0, jb = 0, kb = 0;
    if (tid < nod) {
        role = 1;
        jb = 1;
        while (jb * (jb + 1) / 2 <= tid) ++jb;  // tid in [jb (jb - 1) / 2, jb (jb + 1) / 2)
        kb = tid - jb * (jb - 1) / 2;
    } else if (tid >= 128 && tid < 128 + nbd) {
        role = 2;
        jb = tid - 128;
    }
    float acc[NT];
#pragma unroll
    for (int e = 0; e < NT; ++e) acc[e] = 0.f;
    float cacc = 0.f, cacc2 = 0.f;
    const int cj = tid - 160;  // columns cj and cj + 96
    over_rows(P, u, total, [&](const float* tile, const float* tsb, int nr) {
        if (role == 1) {
#pragma unroll 1
            for (int i = 0; i < nr; ++i) {
                const float* tr = tile + i * ldt;
                float aj[T], ak[T];
                if constexpr (T >= 4) {
#pragma unroll
                    for (int a = 0; a < T; a += 4) {
                        const float4 v = *reinterpret_cast<const float4*>(tr + jb * T + a);
                        const float4 w = *reinterpret_cast<const float4*>(tr + kb * T + a);
                        aj[a] = v.x; aj[a + 1] = v.y; aj[a + 2] = v.z; aj[a + 3] = v.w;
                        ak[a] = w.x; ak[a + 1] = w.y; ak[a + 2] = w.z; ak[a + 3] = w.w;
                    }
                } else {
#pragma unroll
                    for (int a = 0; a < T; ++a) {
                        aj[a] = tr[jb * T + a];
                        ak[a] = tr[kb * T + a];
                    }
                }
#pragma unroll
                for (int a = 0; a < T; ++a)
#pragma unroll
                    for (int b = 0; b < T; ++b) acc[a * T + b] = fmaf(aj[a], ak[b], acc[a * T + b]);
            }
        } else if (role == 2) {
#pragma unroll 1
            for (int i = 0; i < nr; ++i) {
                const float* tr = tile + i * ldt;
                float x[T];
                if constexpr (T >= 4) {
#pragma unroll
                    for (int a = 0; a < T; a += 4) {
                        const float4 v = *reinterpret_cast<const float4*>(tr + jb * T + a);
                        x[a] = v.x; x[a + 1] = v.y; x[a + 2] = v.z; x[a + 3] = v.w;
                    }
                } else {
#pragma unroll
                    for (int a = 0; a < T; ++a) x[a] = tr[jb * T + a];
                }
#pragma unroll
                for (int a = 0; a < T; ++a)
#pragma unroll
                    for (int b = 0; b <= a; ++b) acc[a * (a + 1) / 2 + b] = fmaf(x[a], x[b], acc[a * (a + 1) / 2 + b]);
            }
        }
        if (cj >= 0 && cj < d)
            for (int i = 0; i < nr; ++i) cacc = fmaf(tile[i * ldt + cj], tsb[i], cacc);
        if (cj >= 0 && cj + 96 < d)
            for (int i = 0; i < nr; ++i) cacc2 = fmaf(tile[i * ldt + cj + 96], tsb[i], cacc2);
    });
    double* G = S.Gp + U.goff;
    if (role == 1) {
#pragma unroll
        for (int a = 0; a < T; ++a) {
            const int j = jb * T + a;
            if (j < d) {
                double* g = G + (j * (j + 1) / 2 + kb * T);
#pragma unroll
                for (int b = 0; b < T; ++b) g[b] = (double)acc[a * T + b];
            }
        }
    } else if (role == 2) {
#pragma unroll
        for (int a = 0; a < T; ++a)
#pragma unroll
            for (int b = 0; b <= a; ++b) {
                const int j = jb * T + a, k = jb * T + b;
                if (j < d) G[tri(j) + k] = (double)acc[a * (a + 1) / 2 + b];
            }
    }
    if (cj >= 0 && cj < d) S.Vp[U.voff + cj] = (double)cacc;
    if (cj >= 0 && cj + 96 < d) S.Vp[U.voff + cj + 96] = (double)cacc2;
}

// ---------------------------------------------------------------- phase B

// Sum of the problem's partials, Cholesky in shared memory, x0.  Returns
// false when a pivot is not positive (status 1; the problem is skipped by the
// refinement).
__device__ void chol_solve(const SolveArgs& S, int p, double* sm) {
    const SolveProb& P = S.probs[p];
    const int d = P.d, tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    const int64_t nt = tri(d);
    double* G = sm;         // packed lower [nt]
    double* v = sm + nt;    // [d]
    double* dinv = v + kMaxBatchD + 16;   // [d] reciprocals of L's diagonal
    __shared__ int ok;
    for (int64_t e = tid; e < nt; e += kSolveThreads) G[e] = sum_units(S.Gp, P.g0, P.gstride, P.nunits, e);
    for (int j = tid; j < d; j += kSolveThreads) v[j] = sum_units(S.Vp, P.v0, P.vstride, P.nunits, j);
    if (tid == 0) ok = 1;
    __syncthreads();
    __shared__ double s_rl;
    for (int j = 0; j < d; ++j) {
        // thread 0 forms the pivot's root and its reciprocal: float64 square roots
        // and divisions are long sequences on this part, so the block reads them
        if (tid == 0) {
            const double piv = G[tri(j) + j];
            if (!(piv > 0.0)) ok = 0;
            else {
                const double r = sqrt(piv);
                G[tri(j) + j] = r;
                s_rl = 1.0 / r;
                dinv[j] = s_rl;
            }
        }
        __syncthreads();
        if (!ok) break;
        const double rl = s_rl;
        for (int i = j + 1 + tid; i < d; i += kSolveThreads) G[tri(i) + j] *= rl;
        __syncthreads();
        for (int i = j + 1 + warp; i < d; i += kSolveThreads / 32) {
            const double lij = G[tri(i) + j];
            for (int k = j + 1 + lane; k <= i; k += 32) G[tri(i) + k] -= lij * G[tri(k) + j];
        }
        __syncthreads();
    }
    if (!ok) {
        for (int j = tid; j < d; j += kSolveThreads) P.x[j] = 0.0;
        if (tid == 0) {
            S.status[p] = 1;
            S.conv[p] = 1;
        }
        return;
    }
    // L y = v, then L^T x = y (v overwritten)
    for (int j = 0; j < d; ++j) {
        if (tid == 0) v[j] *= dinv[j];
        __syncthreads();
        for (int i = j + 1 + tid; i < d; i += kSolveThreads) v[i] -= G[tri(i) + j] * v[j];
        __syncthreads();
    }
    for (int j = d - 1; j >= 0; --j) {
        if (tid == 0) v[j] *= dinv[j];
        __syncthreads();
        for (int i = tid; i < j; i += kSolveThreads) v[i] -= G[tri(j) + i] * v[j];
        __syncthreads();
    }
    for (int j = tid; j < d; j += kSolveThreads) P.x[j] = v[j];
    for (int64_t e = tid; e < nt; e += kSolveThreads) P.L[e] = G[e];
    if (tid == 0) {
        S.status[p] = 0;
        S.conv[p] = 0;
    }
}

// ---------------------------------------------------------------- phase C

// Double-word float32 arithmetic (float64 issues at 1/64 of the float32 rate
// on this part, and so do float32 <-> float64 conversions): a value is an
// unevaluated sum hi + lo of two floats.  dw_mac adds the product of a float
// a and a double-word y = (yh, yl) to the double-word accumulator (sh, sl):
// a * yh exactly by TwoProd (the product rounded, its error by a fused
// multiply-add), a * yl rounded (it is 2^-24 of the product), and the sum by
// TwoSum (Knuth), so each step keeps about 48 bits.
// (The _rn intrinsics keep the compiler from fusing the product into the
// sums, which would break the error terms.)
__device__ __forceinline__ void dw_mac(float& sh, float& sl, float a, float yh, float yl) {
    const float p = __fmul_rn(a, yh);
    const float e = fmaf(a, yh, -p);
    const float s = __fadd_rn(sh, p);
    const float bp = __fsub_rn(s, sh);
    const float err = __fadd_rn(__fsub_rn(sh, __fsub_rn(s, bp)), __fsub_rn(p, bp));
    sh = s;
    sl = fmaf(a, yl, __fadd_rn(sl, __fadd_rn(err, e)));
}

__device__ __forceinline__ void dw_split(double v, float& h, float& l) {
    h = (float)v;
    l = (float)(v - (double)h);
}

// (sh, sl) += (oh, ol) for double-word values (TwoSum of the high parts).
__device__ __forceinline__ void dw_add(float& sh, float& sl, float oh, float ol) {
    const float s = __fadd_rn(sh, oh);
    const float bp = __fsub_rn(s, sh);
    const float err = __fadd_rn(__fsub_rn(sh, __fsub_rn(s, bp)), __fsub_rn(oh, bp));
    sh = s;
    sl = __fadd_rn(sl, __fadd_rn(ol, err));
}

// g = SA_slab^T (Sb_slab - SA_slab x) over the slab's non-empty rows, staged
// 32 at a time, in double-word float32: eight threads per row form r_i
// (columns q, q + 8, ...; the eight partial sums combined by TwoSum), then
// thread t accumulates column t & 127 of rows (t >> 7) * 16 .. + 15 times r_i;
// the two halves are added in float64 at the end.  The tile's row stride is
// 8 mod 32 words, so the eight-lane row reads hit 32 distinct banks.
__device__ void refine_unit(const SolveArgs& S, int ui, const SolveUnit& U, char* smem) {
    const SolveProb& P = S.probs[U.p];
    const int d = P.d, tid = threadIdx.x;
    const int ldt = ((d + 31) / 32) * 32 + 8;
    const UnitSmem u = unit_smem(smem, ldt);
    float2* xs = reinterpret_cast<float2*>(u.wcnt + 16);  // [kMaxBatchD] x as (hi, lo)
    float2* rr = xs + kMaxBatchD;                         // [kChunkRows] r as (hi, lo)
    double* red = reinterpret_cast<double*>(rr + kChunkRows);  // [2][kMaxBatchD]
    for (int j = tid; j < d; j += kSolveThreads) {
        float h, l;
        dw_split(P.x[j], h, l);
        xs[j] = make_float2(h, l);
    }
    const int total = S.ucount[ui];                       // the list phase A kept
    for (int k = tid; k < total; k += kSolveThreads) u.rows[k] = P.rowlist[U.r0 + k];
    __syncthreads();                                      // (publishes xs and rows)
    const int ri = tid >> 3, q = tid & 7;
    const int col = tid & (kMaxBatchD - 1), half = tid >> 7;
    float gh = 0.f, gl = 0.f;
    over_rows(P, u, total, [&](const float* tile, const float* tsb, int nr) {
        float sh = 0.f, sl = 0.f;
        if (ri < nr) {
            const float* tr = tile + ri * ldt;
            for (int j = q; j < d; j += 8) {
                const float2 x2 = xs[j];
                dw_mac(sh, sl, tr[j], x2.x, x2.y);
            }
        }
#pragma unroll
        for (int o = 4; o > 0; o >>= 1) {
            const float oh = __shfl_xor_sync(0xFFFFFFFFu, sh, o);
            const float ol = __shfl_xor_sync(0xFFFFFFFFu, sl, o);
            dw_add(sh, sl, oh, ol);
        }
        if (q == 0 && ri < nr) {
            // r_i = Sb_i - dot as a double-word value
            float rh = tsb[ri], rl = 0.f;
            dw_add(rh, rl, -sh, -sl);
            {   // renormalise (TwoSum of the two parts): |rl| <= ulp(rh) / 2 for dw_mac
                const float t = __fadd_rn(rh, rl);
                const float bp = __fsub_rn(t, rh);
                rl = __fadd_rn(__fsub_rn(rh, __fsub_rn(t, bp)), __fsub_rn(rl, bp));
                rh = t;
            }
            rr[ri] = make_float2(rh, rl);
        }
        __syncthreads();
        if (col < d) {
            const int i1 = min(nr, half * 16 + 16);
            for (int i = half * 16; i < i1; ++i) {
                const float2 r2 = rr[i];
                dw_mac(gh, gl, tile[i * ldt + col], r2.x, r2.y);
            }
        }
    });
    if (col < d) red[half * kMaxBatchD + col] = (double)gh + (double)gl;
    __syncthreads();
    for (int j = tid; j < d; j += kSolveThreads) S.Vp[U.voff + j] = red[j] + red[kMaxBatchD + j];
}

// ---------------------------------------------------------------- phase D

__device__ void refine_update(const SolveArgs& S, int p, bool first, bool last, double* sm) {
    const SolveProb& P = S.probs[p];
    const int d = P.d, tid = threadIdx.x;
    const int64_t nt = tri(d);
    double* G = sm;
    double* v = sm + nt;
    double* red = v + kMaxBatchD;  // [2 * 8]
    double* dinv = red + 16;       // [d] reciprocals of L's diagonal, one division per thread
    for (int64_t e = tid; e < nt; e += kSolveThreads) G[e] = P.L[e];
    for (int j = tid; j < d; j += kSolveThreads) dinv[j] = 1.0 / P.L[tri(j) + j];
    for (int j = tid; j < d; j += kSolveThreads) v[j] = sum_units(S.Vp, P.v0, P.vstride, P.nunits, j);
    __syncthreads();
    for (int j = 0; j < d; ++j) {
        if (tid == 0) v[j] *= dinv[j];
        __syncthreads();
        for (int i = j + 1 + tid; i < d; i += kSolveThreads) v[i] -= G[tri(i) + j] * v[j];
        __syncthreads();
    }
    for (int j = d - 1; j >= 0; --j) {
        if (tid == 0) v[j] *= dinv[j];
        __syncthreads();
        for (int i = tid; i < j; i += kSolveThreads) v[i] -= G[tri(j) + i] * v[j];
        __syncthreads();
    }
    double dmax = 0.0, xmax = 0.0;
    for (int j = tid; j < d; j += kSolveThreads) {
        const double xn = P.x[j] + v[j];
        P.x[j] = xn;
        dmax = fmax(dmax, fabs(v[j]));
        xmax = fmax(xmax, fabs(xn));
    }
    const int warp = tid >> 5, lane = tid & 31;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        dmax = fmax(dmax, __shfl_xor_sync(0xFFFFFFFFu, dmax, o));
        xmax = fmax(xmax, __shfl_xor_sync(0xFFFFFFFFu, xmax, o));
    }
    if (lane == 0) {
        red[warp] = dmax;
        red[8 + warp] = xmax;
    }
    __syncthreads();
    if (tid == 0) {
        double a = 0.0, b = 0.0;
        for (int w = 0; w < kSolveThreads / 32; ++w) {
            a = fmax(a, red[w]);
            b = fmax(b, red[8 + w]);
        }
        // Stop once the correction is at rounding level, or once the
        // contraction seen over two steps (rho = a / previous correction)
        // puts the remaining error, about rho * a, there.  After the last step
        // a correction above 1e-10 |x| marks the problem for the fallback.
        const double prev = *P.dprev;
        const bool small = a <= 1e-13 * b;
        const bool contracting = !first && a < prev && a * a <= 1e-14 * b * prev;
        if (small || contracting) S.conv[p] = 1;
        else if (last && !(a <= 1e-10 * b)) S.status[p] = 2;
        *P.dprev = a;
    }
}

// ---------------------------------------------------------------- the persistent kernel

__global__ void __launch_bounds__(kSolveThreads, 2) k_batch_solve(SolveArgs S) {
    extern __shared__ __align__(16) double smd[];
    __shared__ int item;
    const unsigned G = gridDim.x;
    stamp(S, 0);
    // A: Gram units
    for (;;) {
        const int q = next_item(S.qctr + 0, S.nunits, &item);
        if (q < 0) break;
        const int ui = S.uorder[q];
        const SolveUnit U = S.units[ui];
        const int d = S.probs[U.p].d;
        if (d <= 16) gram_unit<1>(S, ui, U, reinterpret_cast<char*>(smd));
        else if (d <= 32) gram_unit<2>(S, ui, U, reinterpret_cast<char*>(smd));
        else if (d <= 64) gram_unit<4>(S, ui, U, reinterpret_cast<char*>(smd));
        else gram_unit<8>(S, ui, U, reinterpret_cast<char*>(smd));
    }
    if (!grid_barrier(S.bar, G, S.tflag)) return;
    stamp(S, 1);
    // B: Cholesky and x0 per problem
    for (;;) {
        const int q = next_item(S.qctr + 1, S.count, &item);
        if (q < 0) break;
        chol_solve(S, S.porder[q], smd);
    }
    for (int step = 0; step < S.steps; ++step) {
        if (!grid_barrier(S.bar, G, S.tflag)) return;
        stamp(S, 2 + 2 * step);
        // C: residual units
        for (;;) {
            const int q = next_item(S.qctr + 2 + 2 * step, S.nunits, &item);
            if (q < 0) break;
            const int ui = S.uorder[q];
            const SolveUnit U = S.units[ui];
            if (*(volatile unsigned*)(S.conv + U.p)) continue;
            refine_unit(S, ui, U, reinterpret_cast<char*>(smd));
        }
        if (!grid_barrier(S.bar, G, S.tflag)) return;
        stamp(S, 3 + 2 * step);
        // D: corrections
        for (;;) {
            const int q = next_item(S.qctr + 3 + 2 * step, S.count, &item);
            if (q < 0) break;
            const int p = S.porder[q];
            if (*(volatile unsigned*)(S.conv + p)) continue;
            refine_update(S, p, step == 0, step == S.steps - 1, smd);
        }
    }
    if (!grid_barrier(S.bar, G, S.tflag)) return;
    stamp(S, 2 + 2 * S.steps);
}

size_t solve_smem_bytes() {
    const int ldt = std::max(16 * 8 + 4, kMaxBatchD + 8);
    const size_t unit = sizeof(int) * kMaxSlab + sizeof(float) * kStages * kChunkRows * (ldt + 1) +
                        sizeof(int) * 16 + sizeof(double) * (3 * kMaxBatchD + kChunkRows);
    const size_t chol = sizeof(double) * ((size_t)kMaxBatchD * (kMaxBatchD + 1) / 2 + 2 * kMaxBatchD + 16);
    return std::max(unit, chol);
}

}  // namespace cw

// ================================================================ plan and C ABI

using namespace cw;

struct cw_batch {
    int count = 0;
    int device = 0;
    // problem data as given
    std::vector<BatchSpec> specs;
    std::vector<double*> xs;
    // sketch plan
    BatchSketchHost sk_host;
    BatchSketch sk{};
    // solve plan (host copies)
    std::vector<SolveProb> sprobs;
    std::vector<SolveUnit> units;
    std::vector<int32_t> uorder, porder;
    SolveArgs sa{};
    int steps = kMaxSteps;
    int slab = 2048;
    int ctas_per_sm = 1;
    int grid = 0;
    int graph_ok = 0;
    int graph_kernels = 0;  // kernel launches inside the graph
    int tuned = 0;
    double tune_ms = 0.0;
    // device memory
    void* mem = nullptr;       // all plan-owned device memory
    size_t mem_bytes = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

namespace {

// Bump allocator over one device allocation (offsets computed first).
struct Layout {
    size_t off = 0;
    size_t take(size_t bytes) {
        const size_t o = off;
        off += (bytes + 255) & ~(size_t)255;
        return o;
    }
};

uint64_t fnv(uint64_t h, uint64_t v) {
    for (int k = 0; k < 8; ++k) {
        h ^= (v >> (8 * k)) & 0xFF;
        h *= 1099511628211ull;
    }
    return h;
}

uint64_t shape_key(const std::vector<BatchSpec>& specs) {
    uint64_t h = 1469598103934665603ull;
    h = fnv(h, (uint64_t)specs.size());
    h = fnv(h, (uint64_t)num_sms());
    for (const BatchSpec& s : specs) {
        h = fnv(h, (uint64_t)s.n);
        h = fnv(h, (uint64_t)s.d);
        h = fnv(h, (uint64_t)s.nnz);
        h = fnv(h, (uint64_t)s.m);
    }
    return h;
}

bool cache_lookup(uint64_t key, int* slab, int* cps, int* lpr) {
    const char* path = std::getenv("CW_TUNE_CACHE");
    if (!path || !*path) return false;
    FILE* f = std::fopen(path, "r");
    if (!f) return false;
    char line[256];
    bool found = false;
    while (std::fgets(line, sizeof line, f)) {
        unsigned long long k = 0;
        int a = 0, b = 0, c = 0;
        if (std::sscanf(line, "batch %llx %d %d %d", &k, &a, &b, &c) == 4 && k == key && a > 0 && b > 0 &&
            (c == 16 || c == 32 || c == 0 || c == -8)) {
            *slab = a;
            *cps = b;
            *lpr = c;
            found = true;
        }
    }
    std::fclose(f);
    return found;
}

void cache_store(uint64_t key, int slab, int cps, int lpr) {
    const char* path = std::getenv("CW_TUNE_CACHE");
    if (!path || !*path) return;
    FILE* f = std::fopen(path, "a");
    if (!f) return;
    std::fprintf(f, "batch %llx %d %d %d\n", (unsigned long long)key, slab, cps, lpr);
    std::fclose(f);
}

// Units of `slab` bucket rows per problem, the solve descriptors and queues.
void build_units(cw_batch* B, int slab) {
    B->units.clear();
    B->sprobs.assign((size_t)B->count, SolveProb{});
    std::vector<double> cost;
    int64_t goff = 0, voff = 0;
    for (int p = 0; p < B->count; ++p) {
        const BatchSpec& s = B->specs[(size_t)p];
        SolveProb& P = B->sprobs[(size_t)p];
        P.d = (int32_t)s.d;
        P.m = (int32_t)s.m;
        P.unit0 = (int32_t)B->units.size();
        const double fill = std::min(1.0, (double)s.n / (double)s.m);
        for (int64_t r0 = 0; r0 < s.m; r0 += slab) {
            SolveUnit U;
            U.p = p;
            U.r0 = (int32_t)r0;
            U.r1 = (int32_t)std::min<int64_t>(s.m, r0 + slab);
            U.goff = goff;
            U.voff = voff;
            goff += (s.d * (s.d + 1) / 2 + 31) & ~31ll;
            voff += (s.d + 31) & ~31ll;
            B->units.push_back(U);
            cost.push_back((double)(U.r1 - U.r0) * fill * (double)(s.d * s.d + 64));
        }
        P.nunits = (int32_t)B->units.size() - P.unit0;
        P.gstride = (s.d * (s.d + 1) / 2 + 31) & ~31ll;
        P.vstride = (s.d + 31) & ~31ll;
        P.g0 = P.nunits ? B->units[(size_t)P.unit0].goff : 0;
        P.v0 = P.nunits ? B->units[(size_t)P.unit0].voff : 0;
    }
    B->uorder.resize(B->units.size());
    for (size_t u = 0; u < B->units.size(); ++u) B->uorder[u] = (int32_t)u;
    std::stable_sort(B->uorder.begin(), B->uorder.end(), [&](int32_t a, int32_t b) { return cost[a] > cost[b]; });
    B->porder.resize((size_t)B->count);
    for (int p = 0; p < B->count; ++p) B->porder[(size_t)p] = p;
    std::stable_sort(B->porder.begin(), B->porder.end(),
                     [&](int32_t a, int32_t b) { return B->specs[a].d > B->specs[b].d; });
}

// Allocates and fills all device memory of the plan for the given slab.
int build_device(cw_batch* B, int slab) {
    build_units(B, slab);
    const BatchSketchHost& H = B->sk_host;
    int64_t gsz = 0, vsz = 0;
    for (const SolveUnit& U : B->units) {
        const int64_t d = B->specs[(size_t)U.p].d;
        gsz = std::max<int64_t>(gsz, U.goff + d * (d + 1) / 2);
        vsz = std::max<int64_t>(vsz, U.voff + d);
    }
    int64_t lsz = 0;
    std::vector<int64_t> loff((size_t)B->count);
    for (int p = 0; p < B->count; ++p) {
        loff[(size_t)p] = lsz;
        const int64_t d = B->specs[(size_t)p].d;
        lsz += (d * (d + 1) / 2 + 31) & ~31ll;
    }
    int64_t sa_elems = 0, sb_elems = 0;
    for (const BatchSpec& s : B->specs) {
        sa_elems += s.m * s.d;
        sb_elems += s.m;
    }
    Layout L;
    const size_t oProbs = L.take(sizeof(BatchProb) * H.probs.size());
    const size_t oTile = L.take(sizeof(int32_t) * std::max<size_t>(1, H.tile_prob.size()));
    const size_t oChunk = L.take(sizeof(int32_t) * std::max<size_t>(1, H.chunk_prob.size()));
    const size_t oBin = L.take(sizeof(int32_t) * std::max<size_t>(1, H.bin_prob.size()));
    const size_t oBk = L.take(sizeof(int64_t) * H.bk_base.size());
    const size_t oH = L.take(sizeof(uint32_t) * std::max<int64_t>(1, H.H_elems));
    const size_t oP = L.take(sizeof(uint32_t) * std::max<int64_t>(1, H.P_elems));
    const size_t oCP = L.take(sizeof(uint32_t) * std::max<int64_t>(1, H.CP_elems));
    const size_t oRec = L.take(sizeof(int4) * std::max<int64_t>(1, H.rows));
    const size_t oR2 = L.take(sizeof(int2) * std::max<int64_t>(1, H.rows));
    const size_t oRb = L.take(sizeof(float) * std::max<int64_t>(1, H.rows));
    const size_t oBp = L.take(sizeof(int32_t) * H.bptr_elems);
    const size_t oCtr = L.take(sizeof(unsigned) * 64);
    const size_t oSA = L.take(sizeof(float) * sa_elems);
    const size_t oSb = L.take(sizeof(float) * sb_elems);
    const size_t oSP = L.take(sizeof(SolveProb) * B->sprobs.size());
    const size_t oU = L.take(sizeof(SolveUnit) * std::max<size_t>(1, B->units.size()));
    const size_t oUo = L.take(sizeof(int32_t) * std::max<size_t>(1, B->uorder.size()));
    const size_t oPo = L.take(sizeof(int32_t) * B->porder.size());
    const size_t oG = L.take(sizeof(double) * std::max<int64_t>(1, gsz));
    const size_t oV = L.take(sizeof(double) * std::max<int64_t>(1, vsz));
    const size_t oL = L.take(sizeof(double) * std::max<int64_t>(1, lsz));
    const size_t oSt = L.take(sizeof(int32_t) * B->count);
    const size_t oConv = L.take(sizeof(unsigned) * B->count);
    const size_t oStamp = L.take(sizeof(unsigned long long) * 64);
    const size_t oDprev = L.take(sizeof(double) * B->count);
    const size_t oRowl = L.take(sizeof(int32_t) * H.bptr_elems);
    const size_t oUcnt = L.take(sizeof(int32_t) * std::max<size_t>(1, B->units.size()));
    if (B->mem) {
        cudaFree(B->mem);
        B->mem = nullptr;
    }
    CW_CUDA_TRY(cudaMalloc(&B->mem, L.off));
    B->mem_bytes = L.off;
    char* base = static_cast<char*>(B->mem);
    // outputs SA / Sb: the caller's or plan-owned
    std::vector<BatchProb> probs = H.probs;
    int64_t sa_at = 0, sb_at = 0;
    for (int p = 0; p < B->count; ++p) {
        BatchSpec& s = B->specs[(size_t)p];
        float* SA = s.SA ? s.SA : reinterpret_cast<float*>(base + oSA) + sa_at;
        float* Sb = s.Sb ? s.Sb : reinterpret_cast<float*>(base + oSb) + sb_at;
        sa_at += s.m * s.d;
        sb_at += s.m;
        probs[(size_t)p].SA = SA;
        probs[(size_t)p].Sb = Sb;
        probs[(size_t)p].vec4 = (s.d % 4 == 0) && ((reinterpret_cast<uintptr_t>(SA) & 15) == 0) ? 1 : 0;
        probs[(size_t)p].skip_empty = (!s.SA && !s.Sb) ? 1 : 0;
        SolveProb& P = B->sprobs[(size_t)p];
        P.SA = SA;
        P.Sb = Sb;
        P.bptr = reinterpret_cast<int32_t*>(base + oBp) + probs[(size_t)p].bp0;
        P.x = B->xs[(size_t)p];
        P.L = reinterpret_cast<double*>(base + oL) + loff[(size_t)p];
        P.dprev = reinterpret_cast<double*>(base + oDprev) + p;
        P.rowlist = reinterpret_cast<int32_t*>(base + oRowl) + probs[(size_t)p].bp0;
        P.vec = probs[(size_t)p].vec4;
    }
    auto up = [&](size_t off, const void* src, size_t bytes) -> cudaError_t {
        if (bytes == 0) return cudaSuccess;
        return cudaMemcpy(base + off, src, bytes, cudaMemcpyHostToDevice);
    };
    CW_CUDA_TRY(up(oProbs, probs.data(), sizeof(BatchProb) * probs.size()));
    CW_CUDA_TRY(up(oTile, H.tile_prob.data(), sizeof(int32_t) * H.tile_prob.size()));
    CW_CUDA_TRY(up(oChunk, H.chunk_prob.data(), sizeof(int32_t) * H.chunk_prob.size()));
    CW_CUDA_TRY(up(oBin, H.bin_prob.data(), sizeof(int32_t) * H.bin_prob.size()));
    CW_CUDA_TRY(up(oBk, H.bk_base.data(), sizeof(int64_t) * H.bk_base.size()));
    CW_CUDA_TRY(up(oSP, B->sprobs.data(), sizeof(SolveProb) * B->sprobs.size()));
    CW_CUDA_TRY(up(oU, B->units.data(), sizeof(SolveUnit) * B->units.size()));
    CW_CUDA_TRY(up(oUo, B->uorder.data(), sizeof(int32_t) * B->uorder.size()));
    CW_CUDA_TRY(up(oPo, B->porder.data(), sizeof(int32_t) * B->porder.size()));
    CW_CUDA_TRY(cudaMemset(base + oCtr, 0, sizeof(unsigned) * 64));
    BatchSketch& K = B->sk;
    K.probs = reinterpret_cast<const BatchProb*>(base + oProbs);
    K.tile_prob = reinterpret_cast<const int32_t*>(base + oTile);
    K.chunk_prob = reinterpret_cast<const int32_t*>(base + oChunk);
    K.bin_prob = reinterpret_cast<const int32_t*>(base + oBin);
    K.bk_base = reinterpret_cast<const int64_t*>(base + oBk);
    K.H = reinterpret_cast<uint32_t*>(base + oH);
    K.P = reinterpret_cast<uint32_t*>(base + oP);
    K.CP = reinterpret_cast<uint32_t*>(base + oCP);
    K.rec = reinterpret_cast<int4*>(base + oRec);
    K.r2 = reinterpret_cast<int2*>(base + oR2);
    K.rb = reinterpret_cast<float*>(base + oRb);
    K.bptr = reinterpret_cast<int32_t*>(base + oBp);
    unsigned* ctr = reinterpret_cast<unsigned*>(base + oCtr);
    K.counter = ctr;          // [0]: apply queue
    K.status = ctr + 1;       // [1]: sketch input flags
    SolveArgs& A = B->sa;
    A.probs = reinterpret_cast<const SolveProb*>(base + oSP);
    A.units = reinterpret_cast<const SolveUnit*>(base + oU);
    A.uorder = reinterpret_cast<const int32_t*>(base + oUo);
    A.porder = reinterpret_cast<const int32_t*>(base + oPo);
    A.count = B->count;
    A.nunits = (int32_t)B->units.size();
    A.steps = B->steps;
    A.Gp = reinterpret_cast<double*>(base + oG);
    A.Vp = reinterpret_cast<double*>(base + oV);
    A.status = reinterpret_cast<int32_t*>(base + oSt);
    A.conv = reinterpret_cast<unsigned*>(base + oConv);
    A.bar = ctr + 4;          // [4..5]: barrier, [6]: timeout flag
    A.tflag = ctr + 6;
    A.qctr = ctr + 16;        // [16..16 + 2 + 2 * steps)
    A.stamps = reinterpret_cast<unsigned long long*>(base + oStamp);
    A.ucount = reinterpret_cast<int32_t*>(base + oUcnt);
    CW_CUDA_TRY(cudaMemset(A.stamps, 0, sizeof(unsigned long long) * 64));
    B->slab = slab;
    return CW_OK;
}

int solve_grid(int ctas_per_sm) {
    int per = 0;
    const size_t smem = solve_smem_bytes();
    if (cudaFuncSetAttribute(k_batch_solve, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return -1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_batch_solve, kSolveThreads, smem) != cudaSuccess)
        return -1;
    per = std::min(per, ctas_per_sm);
    if (per < 1) return -1;
    return per * num_sms();
}

// The whole batch on `stream` (no synchronisation; capturable).
int enqueue(cw_batch* B, cudaStream_t stream) {
    int st = batch_sketch_enqueue(B->sk, stream);
    if (st != CW_OK) return st;
    unsigned* ctr = B->sk.counter;
    CW_CUDA_TRY(cudaMemsetAsync(ctr + 4, 0, sizeof(unsigned) * 60, stream));
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3((unsigned)B->grid);
    cfg.blockDim = dim3(kSolveThreads);
    cfg.dynamicSmemBytes = solve_smem_bytes();
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    {
        CW_PROF("k_batch_solve", stream);
        CW_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_batch_solve, B->sa));
    }
    return CW_OK;
}

void drop_graph(cw_batch* B) {
    if (B->exec) cudaGraphExecDestroy(B->exec);
    if (B->graph) cudaGraphDestroy(B->graph);
    B->exec = nullptr;
    B->graph = nullptr;
}

// Captures enqueue() into a graph; graph_ok = 0 (direct launches) when the
// capture or instantiation is refused.
int build_graph(cw_batch* B) {
    drop_graph(B);
    B->graph_ok = 0;
    cudaStream_t s;
    CW_CUDA_TRY(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    int st = CW_OK;
    if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
        ProfSuppress quiet;  // no profiling events inside the graph
        const long long before = cw_launch_count();
        st = enqueue(B, s);
        B->graph_kernels = (int)(cw_launch_count() - before);
        cudaGraph_t g = nullptr;
        const cudaError_t e = cudaStreamEndCapture(s, &g);
        if (st == CW_OK && e == cudaSuccess && g) {
            if (cudaGraphInstantiate(&B->exec, g, 0) == cudaSuccess) {
                B->graph = g;
                B->graph_ok = 1;
            } else {
                cudaGraphDestroy(g);
            }
        } else if (g) {
            cudaGraphDestroy(g);
        }
    }
    (void)cudaGetLastError();
    cudaStreamDestroy(s);
    return st;
}

int run(cw_batch* B, cudaStream_t stream) {
    if (B->graph_ok) {
        CW_PROF("cw_batch_graph", stream);
        CW_CUDA_TRY(cudaGraphLaunch(B->exec, stream));
        for (int k = 1; k < B->graph_kernels; ++k) count_launch();  // the graph's kernels
        return CW_OK;
    }
    return enqueue(B, stream);
}

int configure(cw_batch* B, int slab, int cps, bool use_graph) {
    int st = build_device(B, slab);
    if (st != CW_OK) return st;
    B->ctas_per_sm = cps;
    B->grid = solve_grid(cps);
    if (B->grid < 1) return CW_ERR_CUDA;
    if (use_graph) return build_graph(B);
    drop_graph(B);
    B->graph_ok = 0;
    return CW_OK;
}

double time_runs(cw_batch* B, cudaStream_t s, int reps) {
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    bool ok = run(B, s) == CW_OK;  // warm-up
    cudaEventRecord(e0, s);
    for (int r = 0; ok && r < reps; ++r) ok = run(B, s) == CW_OK;
    cudaEventRecord(e1, s);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return ok ? (double)ms / reps : 1e30;
}

}  // namespace

extern "C" int cw_batch_create(const cw_batch_problem* probs, int32_t count, int32_t flags, cw_stream stream,
                               cw_batch** out) {
    if (!out) return CW_ERR_ARG;
    *out = nullptr;
    if (count < 1 || !probs) return CW_ERR_ARG;
    if (count > (1 << 20)) return CW_ERR_SHAPE;
    cw_batch* B = new cw_batch();
    B->count = count;
    cudaGetDevice(&B->device);
    B->specs.resize((size_t)count);
    B->xs.resize((size_t)count);
    for (int p = 0; p < count; ++p) {
        const cw_batch_problem& q = probs[p];
        const int64_t n = q.A.n, d = q.A.d, m = q.m;
        int st = validate_common(n, d, m);
        if (st == CW_OK && (d < 1 || d > kMaxBatchD || m < d)) st = CW_ERR_SHAPE;
        if (st == CW_OK && (q.A.nnz < 0 || q.A.nnz > 0x7FFFFFFFll)) st = CW_ERR_OVERFLOW;
        if (st == CW_OK && (!q.x || (n > 0 && (!q.A.row_ptr || !q.b || (q.A.nnz > 0 && (!q.A.col || !q.A.val))))))
            st = CW_ERR_ARG;
        if (st != CW_OK) {
            delete B;
            return st;
        }
        BatchSpec& s = B->specs[(size_t)p];
        s.n = n;
        s.d = d;
        s.nnz = q.A.nnz;
        s.m = m;
        s.seed = q.seed;
        s.row_ptr = q.A.row_ptr;
        s.col = q.A.col;
        s.val = q.A.val;
        s.b = q.b;
        s.SA = q.SA;
        s.Sb = q.Sb;
        B->xs[(size_t)p] = q.x;
    }
    int st = batch_sketch_plan(B->specs.data(), count, &B->sk_host, &B->sk);
    if (st != CW_OK) {
        delete B;
        return st;
    }
    const bool use_graph = (flags & CW_BATCH_EAGER) == 0;
    int slab = 2048, cps = 1;
    const uint64_t key = shape_key(B->specs);
    bool cached = false;
    int lpr = B->sk.lpr;
    if (flags & CW_BATCH_AUTOTUNE) cached = cache_lookup(key, &slab, &cps, &lpr);
    if (cached && !B->sk.acc_global && batch_sketch_set_lpr(&B->sk, lpr) != CW_OK) cached = false;
    if ((flags & CW_BATCH_AUTOTUNE) && !cached) {
        cudaStream_t s = (cudaStream_t)stream;
        double best = 1e30;
        int bs = slab, bc = cps;
        // lanes per row of the segmented sum first (with the default solve
        // shape), then slab x CTAs per SM
        int best_lpr = B->sk.lpr;
        if (!B->sk.acc_global) {
            double bl = 1e30;
            for (int lp : {16, 32, 0, -8}) {
                if (batch_sketch_set_lpr(&B->sk, lp) != CW_OK) continue;
                if (configure(B, slab, cps, use_graph) != CW_OK) continue;
                const double ms = time_runs(B, s, 2);
                if (ms < bl) {
                    bl = ms;
                    best_lpr = lp;
                }
            }
            batch_sketch_set_lpr(&B->sk, best_lpr);
        }
        const int slabs[] = {512, 1024, 2048, 4096};
        const int cpss[] = {1, 2};
        for (int cs : cpss) {
            for (int sl : slabs) {
                if (configure(B, sl, cs, use_graph) != CW_OK) continue;
                if (B->grid < (cs * num_sms())) continue;  // fewer CTAs per SM fit than asked
                const double ms = time_runs(B, s, 2);
                if (ms < best) {
                    best = ms;
                    bs = sl;
                    bc = cs;
                }
            }
        }
        slab = bs;
        cps = bc;
        B->tune_ms = best;
        B->tuned = 1;
        cache_store(key, slab, cps, B->sk.lpr);
    } else if (cached) {
        B->tuned = 2;
    }
    st = configure(B, slab, cps, use_graph);
    if (st != CW_OK) {
        cw_batch_destroy(B);
        return st;
    }
    *out = B;
    return CW_OK;
}

extern "C" int cw_batch_run(cw_batch* plan, cw_stream stream) {
    if (!plan) return CW_ERR_ARG;
    return run(plan, (cudaStream_t)stream);
}

extern "C" int cw_batch_finish(cw_batch* plan, cw_stream stream, int32_t* status, int32_t* fallbacks) {
    if (!plan) return CW_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<int32_t> st((size_t)plan->count);
    unsigned flags[2] = {0, 0};
    CW_CUDA_TRY(cudaMemcpyAsync(st.data(), plan->sa.status, sizeof(int32_t) * st.size(), cudaMemcpyDeviceToHost, s));
    CW_CUDA_TRY(cudaMemcpyAsync(&flags[0], plan->sa.tflag, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
    CW_CUDA_TRY(cudaMemcpyAsync(&flags[1], plan->sk.status, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
    CW_CUDA_TRY(cudaStreamSynchronize(s));
    if (flags[0]) return CW_ERR_TIMEOUT;
    if (flags[1]) return CW_ERR_ARG;
    int nfb = 0;
    int ret = CW_OK;
    for (int p = 0; p < plan->count; ++p) {
        if (st[(size_t)p] == 0) continue;
        // float64 Householder QR of this problem's SA, then R x = Q^T Sb
        const BatchSpec& sp = plan->specs[(size_t)p];
        const SolveProb& P = plan->sprobs[(size_t)p];
        if (!sp.SA && !sp.Sb) {
            // plan-owned SA / Sb hold only the non-empty rows: write them whole
            const int k = sketch_impl(kSketchCSR, sp.n, sp.d, 0, 0, sp.row_ptr, sp.col, sp.val, nullptr, sp.b,
                                      sp.m, sp.seed, const_cast<float*>(P.SA), const_cast<float*>(P.Sb), nullptr, s);
            if (k != CW_OK) {
                if (ret == CW_OK) ret = k;
                continue;
            }
        }
        double* R = nullptr;
        double* c = nullptr;
        CW_CUDA_TRY(cudaMallocAsync(&R, sizeof(double) * (size_t)(sp.d * sp.d + sp.d), s));
        c = R + sp.d * sp.d;
        int q = qr64(P.SA, sp.m, (int)sp.d, P.Sb, R, c, s);
        if (q == CW_OK) q = trsv_upper(R, (int)sp.d, c, plan->xs[(size_t)p], s);
        cudaFreeAsync(R, s);
        if (q == CW_OK) {
            st[(size_t)p] = 3;  // solved by the fallback
        } else if (q == CW_ERR_RANK) {
            st[(size_t)p] = 4;  // S_p A_p is rank deficient: x_p set to zero
            CW_CUDA_TRY(cudaMemsetAsync(plan->xs[(size_t)p], 0, sizeof(double) * (size_t)sp.d, s));
        } else if (ret == CW_OK) {
            ret = q;
        }
        ++nfb;
    }
    if (status) std::memcpy(status, st.data(), sizeof(int32_t) * st.size());
    if (fallbacks) *fallbacks = nfb;
    CW_CUDA_TRY(cudaStreamSynchronize(s));
    return ret;
}

extern "C" int cw_batch_info(const cw_batch* plan, int64_t* info) {
    if (!plan || !info) return CW_ERR_ARG;
    info[0] = plan->slab;
    info[1] = plan->ctas_per_sm;
    info[2] = plan->grid;
    info[3] = plan->graph_ok;
    info[4] = (int64_t)plan->units.size();
    info[5] = plan->tuned;
    info[6] = (int64_t)plan->mem_bytes;
    info[7] = plan->steps;
    info[8] = plan->sk.lpr;
    return CW_OK;
}

extern "C" int cw_batch_phases(const cw_batch* plan, cw_stream stream, double* ms, int32_t max) {
    if (!plan || !ms) return CW_ERR_ARG;
    const int n = 3 + 2 * plan->steps;
    unsigned long long t[64];
    CW_CUDA_TRY(cudaMemcpyAsync(t, plan->sa.stamps, sizeof(unsigned long long) * n, cudaMemcpyDeviceToHost,
                                (cudaStream_t)stream));
    CW_CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
    int k = 0;
    for (; k + 1 < n && k < max; ++k) ms[k] = t[k + 1] >= t[k] ? (double)(t[k + 1] - t[k]) * 1e-6 : 0.0;
    return k;
}

extern "C" int cw_batch_destroy(cw_batch* plan) {
    if (!plan) return CW_OK;
    drop_graph(plan);
    if (plan->mem) cudaFree(plan->mem);
    delete plan;
    return CW_OK;
}
