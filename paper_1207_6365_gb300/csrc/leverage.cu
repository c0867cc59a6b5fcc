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
#include <cuda_bf16.h>

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

// ---------------------------------------------------------------- tensor-core path
//
// The same product on the 5th-generation tensor cores (tcgen05, bf16 inputs,
// float32 accumulation in tensor memory), exact by splitting (the Ozaki
// scheme): for each 64-column chunk c of A, row i is written as
//     A_ij = 2^(E_ic - 7) * sum_s d_s(i,j) 128^-s,   s = 0..4,
// with E_ic the exponent bound of the row's largest |A_ij| in the chunk and
// integer digits |d_0| <= 128, |d_s| <= 64, and likewise each column l of M as
//     M_jl = 2^(F_cl - 7) * sum_t e_t(j,l) 128^-t.
// A digit times a digit is an integer below 2^14 and a chunk sums 64 of them,
// so every product of slices, and the sum of the g + 1 slice pairs of one
// level g = s + t, is an integer below 2^23: the tensor core adds it exactly.
// Levels g = 0..4 are kept (the first one dropped is 2^-35 of the largest
// product), each level of each chunk lands in its own accumulator
//     D_g(i,l) = sum_{s+t=g} sum_j d_s(i,j) e_t(j,l),
// and the accumulators are drained into two-word float32 sums of
//     2^(E_ic + F_cl - 14 - 7g) D_g(i,l)
// over levels and chunks (the cancellation between levels, which is where the
// conditioning of A shows, happens in those sums).  The digit slices hold
// d_s 128^-s and e_t 128^-t (still exact in bf16), so the accumulator of level
// g already carries the factor 128^-g.  Powers of two are formed in
// float32: rows whose largest entry is below 2^-90 in magnitude, or columns of
// M outside 2^+-90, would lose accuracy.

constexpr int kTcRows = 128;                       // rows per tile (MMA M)
constexpr int kTcK = 64;                           // columns of A per chunk
constexpr int kTcN = 32;                           // MMA N (k <= 32)
constexpr int kTcDig = 5;                          // digits per operand
constexpr int kTcLev = 5;                          // levels kept
static_assert(kTcDig == 5 && kTcLev == 5, "the drain sums levels 2..4 in float32 before the two-word sums");
constexpr int kTcLBO = 128;                        // bytes between core matrices along K
constexpr int kTcSBO = (kTcK / 8) * 128;           // bytes between core matrices along M / N
constexpr int kTcASlice = kTcRows * kTcK * 2;      // 16 KB per A digit slice
constexpr int kTcBSlice = kTcN * kTcK * 2;         // 4 KB per M digit slice
constexpr int kTcBChunk = kTcDig * kTcBSlice;      // 20 KB per chunk of M
constexpr int kTcRawStride = kTcK + 4;             // floats per staged row of A (conflict-free 16-byte reads)
constexpr int kTcRaw = kTcRows * kTcRawStride * 4; // bytes per staged chunk of A
constexpr size_t kTcSmem = (size_t)kTcDig * kTcASlice + 2 * (size_t)kTcRaw + 2 * (size_t)kTcBChunk +
                           3 * kTcN * sizeof(float);

// byte offset of element (r, k) in the canonical K-major layout without
// swizzle: 8 x 8 core matrices of 16-byte rows, LBO along K, SBO along M/N
__host__ __device__ __forceinline__ int tc_off(int r, int k) {
    return (r >> 3) * kTcSBO + (k >> 3) * kTcLBO + (r & 7) * 16 + (k & 7) * 2;
}

__device__ __forceinline__ uint32_t tc_smem(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor (no swizzle)
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr) {
    return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)((kTcLBO >> 4) & 0x3FFF) << 16) |
           ((uint64_t)((kTcSBO >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}

// instruction descriptor: D float32, A and B bf16, both K-major, N, M
constexpr uint32_t kTcIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kTcN >> 3) << 17) |
                              ((uint32_t)(kTcRows >> 4) << 24);

// M (float64, d x k row-major) -> per chunk c: kTcDig digit slices of the
// 32 x 64 block M[64c .., 0..31]^T in the canonical layout, and column scales
// 2^(F_cl - 7).  One thread per (chunk, column).
__global__ void k_m_digits(const double* __restrict__ M, int d, int k, int nchunk, __nv_bfloat16* __restrict__ Bd,
                           float* __restrict__ cs) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nchunk * kTcN) return;
    const int c = q / kTcN, l = q % kTcN;
    int F = -100000;
    for (int j = c * kTcK; j < min(d, (c + 1) * kTcK); ++j) {
        const double v = (l < k) ? M[(size_t)j * k + l] : 0.0;
        if (v != 0.0) {
            int e;
            frexp(v, &e);
            F = max(F, e);
        }
    }
    const bool any = F > -100000;
    if (!any) F = 0;
    cs[c * kTcN + l] = any ? ldexpf(1.f, F - 7) : 0.f;
    unsigned char* base = reinterpret_cast<unsigned char*>(Bd) + (size_t)c * kTcBChunk;
    for (int kk = 0; kk < kTcK; ++kk) {
        const int j = c * kTcK + kk;
        double x = (any && l < k && j < d) ? ldexp(M[(size_t)j * k + l], 7 - F) : 0.0;
        for (int t = 0; t < kTcDig; ++t) {
            const double dg = rint(x);
            x = (x - dg) * 128.0;
            // digit t is stored as e_t 128^-t (exact in bf16: at most 8 significant bits)
            *reinterpret_cast<__nv_bfloat16*>(base + t * kTcBSlice + tc_off(l, kk)) =
                __float2bfloat16((float)ldexp(dg, -7 * t));
        }
    }
}

struct TcLevArgs {
    unsigned* tflag;           // set when the wait for the tensor core timed out
    const float* A;
    int64_t n;
    int d;
    int64_t lda;
    int k;
    const __nv_bfloat16* Bd;   // [nchunk][kTcDig][32 x 64] canonical
    const float* cs;           // [nchunk][32]
    float* lev;
    unsigned* status;
};

constexpr int kTcWork = 256;               // two threads per row: chunk columns 0..31 / 32..63
constexpr int kTcThreads = kTcWork + 32;   // plus one warp that issues the MMAs

// Eight working warps and one that issues the MMAs.  Thread t < 256 owns row
// t % 128 of the tile and half h = t / 128 of each chunk's columns (digits of
// columns 32h ..) and of the 32 output columns (drain: warp w reads the
// tensor-memory lanes of rows 32 (w % 4) .., columns 16 (w / 4) ..).  Two
// tensor-memory accumulator sets alternate, so the MMAs of chunk q run while
// the working warps drain chunk q - 1; A and the M digits of chunk q + 1 are
// copied in (cp.async) during chunk q.  (A variant with sixteen working warps,
// double-buffered digit slices and A prefetched into registers, which also
// overlaps the digits of chunk q + 1 with the MMAs of chunk q, measured
// slower: 8.4 against 7.5 ms at n = 2^22, d = 512.)
__global__ void __launch_bounds__(kTcThreads) k_leverage_tc(TcLevArgs a) {
    extern __shared__ __align__(1024) unsigned char tsm[];
    __shared__ uint32_t tmem_base;
    __shared__ __align__(8) uint64_t mbar[2];
    __shared__ uint32_t emax_half[2][kTcRows];
    __shared__ float lev_half[2][kTcRows];
    unsigned char* sAs = tsm;                                          // kTcDig slices
    float* sRaw = reinterpret_cast<float*>(tsm + kTcDig * kTcASlice);   // 2 x [128][kTcRawStride]
    unsigned char* sB = tsm + kTcDig * kTcASlice + 2 * kTcRaw;         // 2 x kTcBChunk
    // column scales, three sets: step q's are read by its drain during step q + 1,
    // while the copies for step q + 2 land
    float* sCs = reinterpret_cast<float*>(sB + 2 * kTcBChunk);        // 3 x [32]
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const bool worker = tid < kTcWork;
    const int row_t = tid & (kTcRows - 1), half = (tid >> 7) & 1;      // tile row, column half
    const int nchunk = (a.d + kTcK - 1) / kTcK;
    const int64_t ntiles = (a.n + kTcRows - 1) / kTcRows;
    const int64_t my_tiles = ntiles > blockIdx.x ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    const int64_t nsteps = my_tiles * nchunk;

    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(tc_smem(&mbar[0])));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(tc_smem(&mbar[1])));
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;\n" ::"r"(tc_smem(&tmem_base)));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t tmem = tmem_base;
    constexpr uint32_t kTbuf = kTcLev * kTcN;   // 160 columns per accumulator set

    auto step_tile = [&](int64_t q) { return blockIdx.x + (q / nchunk) * gridDim.x; };
    // step q: warp w copies rows 16w .. 16w + 15 of the A chunk (two rows of 256
    // bytes per instruction) and a share of the chunk's M digits and scales
    auto issue = [&](int64_t q) {
        const int64_t tile = step_tile(q);
        const int c = (int)(q % nchunk);
        const int buf = (int)(q & 1);
        const int vq = lane & 15;
        const int col = c * kTcK + 4 * vq;
#pragma unroll
        for (int rr = 0; rr < 8; ++rr) {
            const int rt = warp * 16 + 2 * rr + (lane >> 4);
            const int64_t row = tile * kTcRows + rt;
            float* dst = sRaw + (size_t)buf * kTcRows * kTcRawStride + (size_t)rt * kTcRawStride + 4 * vq;
            if (row < a.n && col < a.d) cp_async16(dst, a.A + row * a.lda + col);
            else *reinterpret_cast<float4*>(dst) = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        const unsigned char* bsrc = reinterpret_cast<const unsigned char*>(a.Bd) + (size_t)c * kTcBChunk;
        unsigned char* bdst = sB + (size_t)buf * kTcBChunk;
        for (int v = tid; v < kTcBChunk / 16; v += kTcWork) cp_async16(bdst + 16 * v, bsrc + 16 * v);
        if (tid < kTcN / 4) cp_async16(sCs + (q % 3) * kTcN + 4 * tid, a.cs + (size_t)c * kTcN + 4 * tid);
    };
    auto wait_mma = [&](int64_t q) -> bool {
        const int b = (int)(q & 1);
        const uint32_t par = (uint32_t)((q >> 1) & 1);
        for (int it = 0; it < (1 << 22); ++it) {
            uint32_t done;
            asm volatile(
                "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
                : "=r"(done)
                : "r"(tc_smem(&mbar[b])), "r"(par)
                : "memory");
            if (__all_sync(0xFFFFFFFFu, done != 0)) return true;
        }
        return false;
    };

    float acc_hi[16], acc_lo[16];
#pragma unroll
    for (int l = 0; l < 16; ++l) acc_hi[l] = acc_lo[l] = 0.f;
    uint32_t emax = 7, emax_next = 7;   // this row's exponent bound: chunk being drained / being cut
    bool dead = false;
    if (nsteps > 0 && worker) issue(0);
    cp_async_commit();
    for (int64_t q = 0; q <= nsteps; ++q) {
        if (q < nsteps) {
            const int buf = (int)(q & 1);
            if (q + 1 < nsteps && worker) issue(q + 1);
            cp_async_commit();
            cp_async_wait<1>();
            __syncthreads();
            const float* raw = sRaw + (size_t)buf * kTcRows * kTcRawStride + (size_t)row_t * kTcRawStride + half * 32;
            if (worker) {
                uint32_t em = 0;
#pragma unroll
                for (int v = 0; v < 8; ++v) {
                    const float4 x = *reinterpret_cast<const float4*>(raw + 4 * v);
                    em = max(em, max(max((__float_as_uint(x.x) >> 23) & 0xFF, (__float_as_uint(x.y) >> 23) & 0xFF),
                                     max((__float_as_uint(x.z) >> 23) & 0xFF, (__float_as_uint(x.w) >> 23) & 0xFF)));
                }
                emax_half[half][row_t] = em;
            }
            __syncthreads();
            if (worker) {
                // |A_ij| < 2^E with E = emax - 126; digits of A_ij 2^(7 - E) = A_ij 2^(133 - emax)
                uint32_t e2 = max(emax_half[0][row_t], emax_half[1][row_t]);
                if (e2 < 7) e2 = 7;
                emax_next = e2;
                const float sc = __uint_as_float((260u - e2) << 23);
#pragma unroll
                for (int kq = 0; kq < 4; ++kq) {
                    const float4 x0 = *reinterpret_cast<const float4*>(raw + 8 * kq);
                    const float4 x1 = *reinterpret_cast<const float4*>(raw + 8 * kq + 4);
                    float x[8] = {x0.x * sc, x0.y * sc, x0.z * sc, x0.w * sc, x1.x * sc, x1.y * sc, x1.z * sc, x1.w * sc};
#pragma unroll
                    for (int sd = 0; sd < kTcDig; ++sd) {
                        // digit sd, kept at its weight: d_sd 128^-sd = x rounded to a multiple
                        // of 128^-sd by adding and subtracting 1.5 * 2^(23 - 7 sd) (|x| is
                        // at most 2^(6 - 7 sd) by now; float32 adds round to nearest even),
                        // and x keeps the exact remainder.  |d_sd| <= 128, so the digit is a
                        // bf16 exactly: the upper half of its float32 bits.
                        const float mg = __uint_as_float((uint32_t)(150 - 7 * sd) << 23) * 1.5f;
                        uint32_t db[8];
#pragma unroll
                        for (int u = 0; u < 8; ++u) {
                            const float dg = __fsub_rn(__fadd_rn(x[u], mg), mg);
                            x[u] = __fsub_rn(x[u], dg);
                            db[u] = __float_as_uint(dg);
                        }
                        uint4 pk;
                        pk.x = __byte_perm(db[0], db[1], 0x7632);
                        pk.y = __byte_perm(db[2], db[3], 0x7632);
                        pk.z = __byte_perm(db[4], db[5], 0x7632);
                        pk.w = __byte_perm(db[6], db[7], 0x7632);
                        *reinterpret_cast<uint4*>(sAs + sd * kTcASlice + tc_off(row_t, half * 32 + 8 * kq)) = pk;
                    }
                }
            }
            asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
            __syncthreads();
            if (tid == kTcWork) {
                asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
                const uint32_t a0 = tc_smem(sAs), b0s = tc_smem(sB + (size_t)buf * kTcBChunk);
                // The M digit slices lie one after another along N (slice t = rows 32t ..
                // 32t + 31 of one 160-row operand), so digit slice s of A times the first
                // 5 - s slices of M lands level s + t in accumulator columns 32 (s + t):
                // one MMA per (s, K-step) with N = 32 (5 - s) adds every pair of a level
                // into that level's columns.
                const uint32_t dbase = tmem + (uint32_t)buf * kTbuf;
                for (int sd = 0; sd < kTcDig; ++sd) {
                    const uint32_t nn = (uint32_t)(kTcN * (kTcLev - sd));
                    const uint32_t idesc = (kTcIdesc & ~(0x3Fu << 17)) | ((nn >> 3) << 17);
#pragma unroll
                    for (int ks = 0; ks < kTcK / 16; ++ks) {
                        const uint64_t ad = tc_desc(a0 + sd * kTcASlice + ks * 2 * kTcLBO);
                        const uint64_t bd = tc_desc(b0s + ks * 2 * kTcLBO);
                        const uint32_t accum = (sd == 0 && ks == 0) ? 0u : 1u;
                        asm volatile(
                            "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
                            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dbase + sd * kTcN),
                            "l"(ad), "l"(bd), "r"(idesc), "r"(accum));
                    }
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                                 tc_smem(&mbar[buf]))
                             : "memory");
            }
        }
        if (q >= 1) {
            // drain step q - 1 (its MMAs were waited for at the end of the previous iteration)
            const int64_t qp = q - 1;
            const int bp = (int)(qp & 1);
            const int cp = (int)(qp % nchunk);
            if (worker) {
                // level g of the chunk weighs 2^(E - 7) 2^(F_cl - 7) 128^-g
                const float rs0 = __uint_as_float((emax - 6u) << 23);   // 2^(E - 7) = 2^(emax - 133)
                const float* csb = sCs + (qp % 3) * kTcN + half * 16;
                uint32_t r[kTcLev][16];
#pragma unroll
                for (int g = 0; g < kTcLev; ++g) {
                    const uint32_t taddr = tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)bp * kTbuf +
                                           g * kTcN + half * 16;
                    asm volatile(
                        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
                        "[%16];\n"
                        : "=r"(r[g][0]), "=r"(r[g][1]), "=r"(r[g][2]), "=r"(r[g][3]), "=r"(r[g][4]), "=r"(r[g][5]),
                          "=r"(r[g][6]), "=r"(r[g][7]), "=r"(r[g][8]), "=r"(r[g][9]), "=r"(r[g][10]), "=r"(r[g][11]),
                          "=r"(r[g][12]), "=r"(r[g][13]), "=r"(r[g][14]), "=r"(r[g][15])
                        : "r"(taddr));
                }
                asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
                // both operands' digits carry their weights 128^-s, 128^-t, so level g
                // holds D_g 128^-g, exact.  Levels 0 and 1 enter the two-word sums on
                // their own; levels 2..4 (at most 2^-14 of level 0) are added in float32
                // first, an error below 2^-38 of the largest product.
#pragma unroll
                for (int l = 0; l < 16; ++l) {
                    const float sl = csb[l] * rs0;
                    const float small =
                        (__uint_as_float(r[2][l]) + __uint_as_float(r[3][l])) + __uint_as_float(r[4][l]);
                    const float terms[3] = {__uint_as_float(r[0][l]) * sl, __uint_as_float(r[1][l]) * sl, small * sl};
#pragma unroll
                    for (int g = 0; g < 3; ++g) {
                        const float term = terms[g];
                        const float t = acc_hi[l] + term;
                        const float bpv = t - acc_hi[l];
                        acc_lo[l] += (acc_hi[l] - (t - bpv)) + (term - bpv);
                        acc_hi[l] = t;
                    }
                }
                if (cp == nchunk - 1) {
                    float sum = 0.f;
#pragma unroll
                    for (int l = 0; l < 16; ++l) {
                        const float y = acc_hi[l] + acc_lo[l];
                        if (half * 16 + l < a.k) sum = fmaf(y, y, sum);
                        acc_hi[l] = acc_lo[l] = 0.f;
                    }
                    lev_half[half][row_t] = sum;
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
            __syncthreads();
            if (cp == nchunk - 1 && tid < kTcRows) {
                const int64_t row = step_tile(qp) * kTcRows + tid;
                if (row < a.n) a.lev[row] = (lev_half[0][tid] + lev_half[1][tid]) / (float)a.k;
            }
        }
        if (q < nsteps) {
            if (!wait_mma(q)) {
                if (lane == 0) {
                    flag_error(a.status, kDevTimeout);
                    atomicExch(a.tflag, 1u);
                }
                dead = true;
            }
            if (__syncthreads_or(dead)) break;
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            emax = emax_next;
        }
    }
    cp_async_wait<0>();
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;\n" ::"r"(tmem));
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
    // tensor-core path: k <= 32 and 16-byte aligned rows of A
    const bool tc = k <= kTcN && (di % 4) == 0 && (lda % 4) == 0 && ((reinterpret_cast<uintptr_t>(A) & 15) == 0);
    if (tc) {
        const int nchunk = (di + kTcK - 1) / kTcK;
        Scratch ws2(stream);
        const size_t oB = ws2.reserve((size_t)nchunk * kTcBChunk);
        const size_t oC = ws2.reserve(sizeof(float) * (size_t)nchunk * kTcN);
        const size_t oF = ws2.reserve(sizeof(unsigned));
        CW_CUDA_TRY(ws2.alloc());
        unsigned* tflag = ws2.at<unsigned>(oF);
        CW_CUDA_TRY(cudaMemsetAsync(tflag, 0, sizeof(unsigned), stream));
        {
            CW_PROF("k_m_digits", stream);
            k_m_digits<<<(nchunk * kTcN + 127) / 128, 128, 0, stream>>>(M, di, k, nchunk,
                                                                         ws2.at<__nv_bfloat16>(oB), ws2.at<float>(oC));
        }
        CW_LAUNCH_CHECK();
        if (n > 0) {
            unsigned* status = device_status_word();
            TcLevArgs ta{tflag, A, n, di, lda, k, ws2.at<__nv_bfloat16>(oB), ws2.at<float>(oC), lev, status};
            CW_CUDA_TRY(cudaFuncSetAttribute(k_leverage_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcSmem));
            const int64_t ntiles = (n + kTcRows - 1) / kTcRows;
            const int grid = (int)(ntiles < num_sms() ? ntiles : num_sms());
            {
                CW_PROF("k_leverage_tc", stream);
                k_leverage_tc<<<grid, kTcThreads, kTcSmem, stream>>>(ta);
            }
            CW_LAUNCH_CHECK();
        }
        unsigned hf = 0;
        CW_CUDA_TRY(cudaMemcpyAsync(&hf, tflag, sizeof(unsigned), cudaMemcpyDeviceToHost, stream));
        CW_CUDA_TRY(cudaStreamSynchronize(stream));
        return hf ? CW_ERR_TIMEOUT : CW_OK;
    }
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
