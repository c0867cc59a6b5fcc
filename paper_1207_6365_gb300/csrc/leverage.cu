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
// conditioning of A shows, happens in those sums).  Powers of two are formed in
// float32: rows whose largest entry is below 2^-90 in magnitude, or columns of
// M outside 2^+-90, would lose accuracy.

constexpr int kTcRows = 128;                       // rows per tile (MMA M)
constexpr int kTcK = 64;                           // columns of A per chunk
constexpr int kTcN = 32;                           // MMA N (k <= 32)
constexpr int kTcDig = 5;                          // digits per operand
constexpr int kTcLev = 5;                          // levels kept
constexpr int kTcLBO = 128;                        // bytes between core matrices along K
constexpr int kTcSBO = (kTcK / 8) * 128;           // bytes between core matrices along M / N
constexpr int kTcASlice = kTcRows * kTcK * 2;      // 16 KB per A digit slice
constexpr int kTcBSlice = kTcN * kTcK * 2;         // 4 KB per M digit slice
constexpr int kTcBChunk = kTcDig * kTcBSlice;      // 20 KB per chunk of M
constexpr int kTcRawStride = kTcK + 4;             // floats per staged row (conflict-free 16-byte reads)
constexpr int kTcRaw = kTcRows * kTcRawStride * 4; // bytes per staged chunk of A
constexpr size_t kTcSmem = (size_t)kTcDig * kTcASlice + 2 * (size_t)kTcRaw + 2 * (size_t)kTcBChunk +
                           2 * kTcN * sizeof(float);

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
            *reinterpret_cast<__nv_bfloat16*>(base + t * kTcBSlice + tc_off(l, kk)) = __float2bfloat16((float)dg);
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

__global__ void __launch_bounds__(kTcRows) k_leverage_tc(TcLevArgs a) {
    extern __shared__ __align__(1024) unsigned char tsm[];
    __shared__ uint32_t tmem_base;
    __shared__ __align__(8) uint64_t mbar;
    unsigned char* sAs = tsm;                                         // kTcDig slices
    float* sRaw = reinterpret_cast<float*>(tsm + kTcDig * kTcASlice);  // 2 x [128][kTcRawStride]
    unsigned char* sB = tsm + kTcDig * kTcASlice + 2 * kTcRaw;        // 2 x kTcBChunk
    float* sCs = reinterpret_cast<float*>(sB + 2 * kTcBChunk);       // 2 x [32]
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nchunk = (a.d + kTcK - 1) / kTcK;
    const int64_t ntiles = (a.n + kTcRows - 1) / kTcRows;
    const int64_t my_tiles = ntiles > blockIdx.x ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    const int64_t nsteps = my_tiles * nchunk;

    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(tc_smem(&mbar)));
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 256;\n" ::"r"(tc_smem(&tmem_base)));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t tmem = tmem_base;

    // step q = (tile, chunk): this thread copies its row of the A chunk and a
    // share of the chunk's M digits and scales
    auto issue = [&](int64_t q) {
        const int64_t tile = blockIdx.x + (q / nchunk) * gridDim.x;
        const int c = (int)(q % nchunk);
        const int buf = (int)(q & 1);
        const int64_t row = tile * kTcRows + tid;
        float* dst = sRaw + (size_t)buf * kTcRows * kTcRawStride + (size_t)tid * kTcRawStride;
        const float* src = a.A + row * a.lda + (int64_t)c * kTcK;
#pragma unroll
        for (int v = 0; v < kTcK / 4; ++v) {
            const int col = c * kTcK + 4 * v;
            if (row < a.n && col < a.d) cp_async16(dst + 4 * v, src + 4 * v);
            else *reinterpret_cast<float4*>(dst + 4 * v) = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        const unsigned char* bsrc = reinterpret_cast<const unsigned char*>(a.Bd) + (size_t)c * kTcBChunk;
        unsigned char* bdst = sB + (size_t)buf * kTcBChunk;
        for (int v = tid; v < kTcBChunk / 16; v += kTcRows) cp_async16(bdst + 16 * v, bsrc + 16 * v);
        if (tid < kTcN / 4) cp_async16(sCs + buf * kTcN + 4 * tid, a.cs + (size_t)c * kTcN + 4 * tid);
    };

    float acc_hi[kTcN], acc_lo[kTcN];
#pragma unroll
    for (int l = 0; l < kTcN; ++l) acc_hi[l] = acc_lo[l] = 0.f;
    bool dead = false;
    if (nsteps > 0) issue(0);
    cp_async_commit();
    for (int64_t q = 0; q < nsteps && !dead; ++q) {
        if (q + 1 < nsteps) issue(q + 1);
        cp_async_commit();
        cp_async_wait<1>();
        __syncthreads();
        const int buf = (int)(q & 1);
        const int c = (int)(q % nchunk);
        // digits of this thread's row of the chunk
        const float* raw = sRaw + (size_t)buf * kTcRows * kTcRawStride + (size_t)tid * kTcRawStride;
        uint32_t emax = 0;
#pragma unroll
        for (int v = 0; v < kTcK / 4; ++v) {
            const float4 x = *reinterpret_cast<const float4*>(raw + 4 * v);
            emax = max(emax, max(max((__float_as_uint(x.x) >> 23) & 0xFF, (__float_as_uint(x.y) >> 23) & 0xFF),
                                 max((__float_as_uint(x.z) >> 23) & 0xFF, (__float_as_uint(x.w) >> 23) & 0xFF)));
        }
        // |A_ij| < 2^E with E = emax - 126; digits of A_ij 2^(7 - E) = A_ij 2^(133 - emax)
        if (emax < 7) emax = 7;
        const float sc = __uint_as_float((260u - emax) << 23);
        for (int kq = 0; kq < kTcK / 8; ++kq) {
            float x[8];
            const float4 x0 = *reinterpret_cast<const float4*>(raw + 8 * kq);
            const float4 x1 = *reinterpret_cast<const float4*>(raw + 8 * kq + 4);
            x[0] = x0.x * sc; x[1] = x0.y * sc; x[2] = x0.z * sc; x[3] = x0.w * sc;
            x[4] = x1.x * sc; x[5] = x1.y * sc; x[6] = x1.z * sc; x[7] = x1.w * sc;
#pragma unroll
            for (int s = 0; s < kTcDig; ++s) {
                float dg[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    dg[u] = rintf(x[u]);
                    x[u] = (x[u] - dg[u]) * 128.f;
                }
                uint4 pk;
                __nv_bfloat162 b0 = __floats2bfloat162_rn(dg[0], dg[1]), b1 = __floats2bfloat162_rn(dg[2], dg[3]);
                __nv_bfloat162 b2 = __floats2bfloat162_rn(dg[4], dg[5]), b3 = __floats2bfloat162_rn(dg[6], dg[7]);
                pk.x = *reinterpret_cast<uint32_t*>(&b0);
                pk.y = *reinterpret_cast<uint32_t*>(&b1);
                pk.z = *reinterpret_cast<uint32_t*>(&b2);
                pk.w = *reinterpret_cast<uint32_t*>(&b3);
                *reinterpret_cast<uint4*>(sAs + s * kTcASlice + tc_off(tid, 8 * kq)) = pk;
            }
        }
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            const uint32_t a0 = tc_smem(sAs), b0s = tc_smem(sB + (size_t)buf * kTcBChunk);
            for (int g = 0; g < kTcLev; ++g) {
                for (int sd = 0; sd <= g; ++sd) {
                    const int td = g - sd;
                    if (sd >= kTcDig || td >= kTcDig) continue;
#pragma unroll
                    for (int ks = 0; ks < kTcK / 16; ++ks) {
                        const uint64_t ad = tc_desc(a0 + sd * kTcASlice + ks * 2 * kTcLBO);
                        const uint64_t bd = tc_desc(b0s + td * kTcBSlice + ks * 2 * kTcLBO);
                        const uint32_t accum = (sd == 0 && ks == 0) ? 0u : 1u;
                        asm volatile(
                            "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
                            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem + g * kTcN),
                            "l"(ad), "l"(bd), "r"(kTcIdesc), "r"(accum));
                    }
                }
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                             tc_smem(&mbar))
                         : "memory");
        }
        {
            const uint32_t par = (uint32_t)(q & 1);
            bool ok = false;
            for (int it = 0; it < (1 << 22); ++it) {
                uint32_t done;
                asm volatile(
                    "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
                    : "=r"(done)
                    : "r"(tc_smem(&mbar)), "r"(par)
                    : "memory");
                if (__all_sync(0xFFFFFFFFu, done != 0)) {
                    ok = true;
                    break;
                }
            }
            if (!ok) {
                if (lane == 0) {
                    flag_error(a.status, kDevTimeout);
                    atomicExch(a.tflag, 1u);
                }
                dead = true;
            }
        }
        if (__syncthreads_or(dead)) {
            dead = true;
            break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        // drain: this warp's 32 rows, 32 columns of each level accumulator
        // level g of the chunk weighs 2^(E - 7) 2^(F_cl - 7) 128^-g: column part from
        // sCs, row part rs0 = 2^(E - 7) = 2^(emax - 133), times 2^-7g
        const float rs0 = __uint_as_float((emax - 6u) << 23);
        for (int g = 0; g < kTcLev; ++g) {
            uint32_t r[32];
            const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + g * kTcN;
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
                : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                  "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                  "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
                  "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
                  "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                : "r"(taddr));
            asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
            const float rsg = rs0 * __uint_as_float((127u - 7u * (uint32_t)g) << 23);   // * 2^-7g
            const float* csb = sCs + buf * kTcN;
#pragma unroll
            for (int l = 0; l < kTcN; ++l) {
                const float term = (__uint_as_float(r[l]) * csb[l]) * rsg;
                const float t = acc_hi[l] + term;
                const float bp = t - acc_hi[l];
                acc_lo[l] += (acc_hi[l] - (t - bp)) + (term - bp);
                acc_hi[l] = t;
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
        if (c == nchunk - 1) {
            const int64_t tile = blockIdx.x + (q / nchunk) * gridDim.x;
            const int64_t row = tile * kTcRows + tid;
            float sum = 0.f;
#pragma unroll
            for (int l = 0; l < kTcN; ++l) {
                const float y = acc_hi[l] + acc_lo[l];
                if (l < a.k) sum = fmaf(y, y, sum);
                acc_hi[l] = acc_lo[l] = 0.f;
            }
            if (row < a.n) a.lev[row] = sum / (float)a.k;
        }
    }
    cp_async_wait<0>();
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 256;\n" ::"r"(tmem));
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
                k_leverage_tc<<<grid, kTcRows, kTcSmem, stream>>>(ta);
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
