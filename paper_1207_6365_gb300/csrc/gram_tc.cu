// Gram matrix SA^T SA of the sketch on the tensor cores (tcgen05, kind::tf32),
// for the LSQR preconditioner (R from its Cholesky factor, Section 7.6: any R
// with SA R^-1 orthonormal up to a constant).
//
// TF32 keeps 10 mantissa bits, so each value is split x = hi + lo with hi = x
// truncated to TF32 and lo = x - hi (exact in float32, then truncated to TF32
// by the MMA): SA^T SA ~ Hi^T Hi + Hi^T Lo + Lo^T Hi, the three products
// accumulated in float32 in tensor memory ("3xTF32"), with ~22-bit products:
// the accuracy of the CUDA-core float32 Gram it replaces.
//
// One CTA per SM owns a contiguous range of SA's rows.  Per stage of 32 rows:
// 256 threads (thread j = column j) read the staged rows, split them and write
// Hi and Lo transposed (column j of SA = row j of both MMA operands, the 32
// rows of the stage along K) in the canonical K-major no-swizzle layout (8 x 16
// byte core matrices, 128 bytes apart along K, 1024 bytes apart along M/N),
// and add SA^T Sb and Sb^T Sb on the CUDA cores; one thread issues the MMAs:
// rows 0..127 of the Gram against all columns, rows 128..dp-1 against columns
// 128..dp-1 (the lower-left block is the transpose of the upper-right), three
// products per K-step of 8.  Operands and staging are double-buffered; the
// stage's MMAs are tracked by an mbarrier (bounded waits).  Per-CTA partials
// are reduced over CTAs in a fixed order (float32 two-word sums).
#include <cstdint>

#include "cw_common.cuh"
#include "cw_internal.h"

namespace cw {

namespace {

constexpr int kGtKC = 32;                      // rows of SA per stage (MMA K: 4 steps of 8)
constexpr int kGtMaxD = 256;                   // columns handled (two M tiles)
constexpr int kGtLBO = 128;                    // bytes between core matrices along K
constexpr int kGtSBO = (kGtKC / 4) * 128;      // bytes between core matrices along M / N
constexpr int kGtTile = kGtMaxD * kGtKC * 4;   // bytes of one operand tile (Hi or Lo)
constexpr int kGtRawStride = kGtMaxD + 4;      // floats per staged row
constexpr int kGtRaw = kGtKC * kGtRawStride * 4;
constexpr int kGtWork = 256;
constexpr int kGtThreads = kGtWork + 32;       // plus the MMA-issuing warp
constexpr size_t kGtSmem = 2 * 2 * (size_t)kGtTile + 2 * (size_t)kGtRaw + 2 * kGtKC * sizeof(float);

__device__ __forceinline__ uint32_t gt_smem(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t gt_desc(uint32_t saddr) {
    return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)((kGtLBO >> 4) & 0x3FFF) << 16) |
           ((uint64_t)((kGtSBO >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}

// floats between two CTAs' partial Gram matrices: dp^2 plus one 128-byte line,
// so that the reduction's loads of one entry over all CTAs (a power-of-two
// stride otherwise) spread over the memory partitions
__host__ __device__ __forceinline__ size_t gt_pstride(int dp) { return (size_t)dp * dp + 32; }

// byte offset of (operand row r, K index k) in a tile
__device__ __forceinline__ int gt_off(int r, int k) { return (r >> 3) * kGtSBO + (k >> 2) * kGtLBO + (r & 7) * 16; }

// instruction descriptor: D float32, A and B TF32 (K-major), M = 128, N = n
__device__ __forceinline__ uint32_t gt_idesc(uint32_t n) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((n >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

struct GramTcArgs {
    const float* SA;
    const float* Sb;
    int64_t m;
    int d, dp;          // columns, padded to a multiple of 16
    int64_t rows_per;   // rows per CTA (a multiple of kGtKC)
    float* part;        // [grid] partial Gram matrices dp x dp, gt_pstride(dp) floats apart (rows 0..127: all
                        // columns; rows >= 128: columns >= 128)
    float* vpart;       // [grid][d + 1] partial SA^T Sb and Sb^T Sb
    unsigned* tflag;    // set when an MMA wait gave up
};

__global__ void __launch_bounds__(kGtThreads, 1) k_gram_tc(GramTcArgs a) {
    extern __shared__ __align__(1024) unsigned char gsm[];
    __shared__ uint32_t tmem_base;
    __shared__ __align__(8) uint64_t mbar[2];
    __shared__ int s_dead;
    unsigned char* sT = gsm;                                                  // [2 stages][Hi, Lo]
    float* sRaw = reinterpret_cast<float*>(gsm + 4 * (size_t)kGtTile);         // [2][kGtKC][kGtRawStride]
    float* sSb = sRaw + 2 * kGtKC * kGtRawStride;                             // [2][kGtKC]
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const bool worker = tid < kGtWork;
    const int dp = a.dp;
    const int64_t r0 = (int64_t)blockIdx.x * a.rows_per;
    const int64_t r1 = (r0 + a.rows_per < a.m) ? r0 + a.rows_per : a.m;
    const int nst = r1 > r0 ? (int)((r1 - r0 + kGtKC - 1) / kGtKC) : 0;

    if (tid == 0) {
        s_dead = 0;
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(gt_smem(&mbar[0])));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(gt_smem(&mbar[1])));
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;\n" ::"r"(gt_smem(&tmem_base)));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t tmem = tmem_base;

    // stage q: rows r0 + 32q .. + 31 of SA (columns 0..d-1; zeros past m and d)
    auto issue = [&](int q) {
        const int buf = q & 1;
        float* raw = sRaw + (size_t)buf * kGtKC * kGtRawStride;
        const int64_t rb = r0 + (int64_t)q * kGtKC;
        const bool vec = (a.d & 3) == 0 && ((reinterpret_cast<uintptr_t>(a.SA) & 15) == 0);
        if (vec) {
            const int q4 = dp / 4;
            for (int e = tid; e < kGtKC * q4; e += kGtWork) {
                const int i = e / q4, j = (e - i * q4) * 4;
                float* dst = raw + i * kGtRawStride + j;
                if (rb + i < r1 && j < a.d) cp_async16(dst, a.SA + (rb + i) * a.d + j);
                else *reinterpret_cast<float4*>(dst) = make_float4(0.f, 0.f, 0.f, 0.f);
            }
        } else {
            for (int e = tid; e < kGtKC * dp; e += kGtWork) {
                const int i = e / dp, j = e - i * dp;
                float* dst = raw + i * kGtRawStride + j;
                if (rb + i < r1 && j < a.d) cp_async4(dst, a.SA + (rb + i) * a.d + j);
                else *dst = 0.f;
            }
        }
        if (tid < kGtKC) {
            float* dst = sSb + buf * kGtKC + tid;
            if (a.Sb && rb + tid < r1) cp_async4(dst, a.Sb + rb + tid);
            else *dst = 0.f;
        }
    };
    auto wait_mma = [&](int q) -> bool {
        const int b = q & 1;
        const uint32_t par = (uint32_t)((q >> 1) & 1);
        for (int it = 0; it < (1 << 22); ++it) {
            uint32_t done;
            asm volatile(
                "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
                : "=r"(done)
                : "r"(gt_smem(&mbar[b])), "r"(par)
                : "memory");
            if (__all_sync(0xFFFFFFFFu, done != 0)) return true;
        }
        return false;
    };

    float cj = 0.f, ss = 0.f;
    if (nst > 0 && worker) issue(0);
    cp_async_commit();
    for (int q = 0; q < nst; ++q) {
        const int buf = q & 1;
        if (q + 1 < nst && worker) issue(q + 1);
        cp_async_commit();
        cp_async_wait<1>();
        // the operand tiles of this buffer were read by the MMAs of stage q - 2
        if (q >= 2 && worker && !wait_mma(q - 2) && lane == 0) s_dead = 1;
        __syncthreads();
        if (s_dead) break;
        if (worker) {
            const float* raw = sRaw + (size_t)buf * kGtKC * kGtRawStride;
            const float* sb = sSb + buf * kGtKC;
            unsigned char* hiT = sT + (size_t)buf * 2 * kGtTile;
            unsigned char* loT = hiT + kGtTile;
            const int j = tid;
            if (j < dp) {
#pragma unroll
                for (int k4 = 0; k4 < kGtKC / 4; ++k4) {
                    float x[4], h[4], l[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        x[u] = raw[(4 * k4 + u) * kGtRawStride + j];
                        h[u] = __uint_as_float(__float_as_uint(x[u]) & 0xFFFFE000u);
                        l[u] = __fsub_rn(x[u], h[u]);
                        cj = fmaf(x[u], sb[4 * k4 + u], cj);
                    }
                    const int off = gt_off(j, 4 * k4);
                    *reinterpret_cast<float4*>(hiT + off) = make_float4(h[0], h[1], h[2], h[3]);
                    *reinterpret_cast<float4*>(loT + off) = make_float4(l[0], l[1], l[2], l[3]);
                }
            }
            if (warp == 0) ss = fmaf(sb[lane], sb[lane], ss);
        }
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        __syncthreads();
        if (tid == kGtWork) {
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            const uint32_t hi0 = gt_smem(sT + (size_t)buf * 2 * kGtTile), lo0 = hi0 + kGtTile;
            const uint32_t n0 = (uint32_t)dp, n1 = (uint32_t)(dp > 128 ? dp - 128 : 0);
            const uint32_t t1 = (uint32_t)(16 * kGtSBO);   // operand rows 128..: 16 groups of 8
#pragma unroll
            for (int ks = 0; ks < kGtKC / 8; ++ks) {
                const uint32_t kb = (uint32_t)(ks * 2 * kGtLBO);
                // (accumulator column, A tile, B tile, N) for the three products of each block
                for (int blk = 0; blk < (n1 ? 2 : 1); ++blk) {
                    const uint32_t dcol = tmem + (blk ? 256u : 0u);
                    const uint32_t aoff = blk ? t1 : 0u, boff = blk ? t1 : 0u;
                    const uint32_t nn = blk ? n1 : n0;
                    const uint32_t idesc = gt_idesc(nn);
                    const uint64_t ah = gt_desc(hi0 + aoff + kb), al = gt_desc(lo0 + aoff + kb);
                    const uint64_t bh = gt_desc(hi0 + boff + kb), bl = gt_desc(lo0 + boff + kb);
                    const uint32_t first = (q == 0 && ks == 0) ? 0u : 1u;
                    asm volatile(
                        "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
                        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(dcol),
                        "l"(ah), "l"(bh), "r"(idesc), "r"(first));
                    asm volatile("tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, 1;\n" ::"r"(dcol), "l"(ah),
                                 "l"(bl), "r"(idesc));
                    asm volatile("tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, 1;\n" ::"r"(dcol), "l"(al),
                                 "l"(bh), "r"(idesc));
                }
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                             gt_smem(&mbar[buf]))
                         : "memory");
        }
    }
    cp_async_wait<0>();
    // the last two stages' MMAs
    if (worker && !s_dead) {
        bool ok = true;
        if (nst >= 2) ok = wait_mma(nst - 2);
        if (ok && nst >= 1) ok = wait_mma(nst - 1);
        if (!ok && lane == 0) s_dead = 1;
    }
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    if (s_dead) {
        if (tid == 0) atomicExch(a.tflag, 1u);
    } else if (worker && nst > 0) {
        // drain: warp w reads tensor-memory lanes 32 (w % 4) .. + 31 (Gram rows), half w / 4 of the columns
        const int quarter = warp & 3, half = warp >> 2;
        const int row = 32 * quarter + lane;
        float* prow = a.part + (size_t)blockIdx.x * gt_pstride(dp);
        for (int blk = 0; blk < (dp > 128 ? 2 : 1); ++blk) {
            // whole 16-column chunks (one tcgen05.ld each) split between the two halves
            const int nch = (blk ? dp - 128 : dp) / 16, h0 = (nch + 1) / 2;
            const int c0 = half ? 16 * h0 : 0, c1 = half ? 16 * nch : 16 * h0;
            for (int cb = c0; cb < c1; cb += 16) {
                uint32_t r[16];
                const uint32_t taddr = tmem + ((uint32_t)(32 * quarter) << 16) + (blk ? 256u : 0u) + (uint32_t)cb;
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
                    "[%16];\n"
                    : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                      "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                      "=r"(r[15])
                    : "r"(taddr));
                asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
                const int grow = (blk ? 128 : 0) + row, gcol = (blk ? 128 : 0) + cb;
                if (grow < dp) {
                    float* dst = prow + (size_t)grow * dp + gcol;
#pragma unroll
                    for (int u = 0; u < 16; u += 4)
                        *reinterpret_cast<float4*>(dst + u) = make_float4(
                            __uint_as_float(r[u]), __uint_as_float(r[u + 1]), __uint_as_float(r[u + 2]),
                            __uint_as_float(r[u + 3]));
                }
            }
        }
    }
    if (worker) {
        if (tid < a.d) a.vpart[(size_t)blockIdx.x * (a.d + 1) + tid] = cj;
        if (warp == 0) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xFFFFFFFFu, ss, o);
            if (lane == 0) a.vpart[(size_t)blockIdx.x * (a.d + 1) + a.d] = ss;
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;\n" ::"r"(tmem));
}

// float32 two-word sum (hi, lo) += (xh, xl): TwoSum of the high parts, the
// low parts and the rounding error carried in lo
__device__ __forceinline__ void gt_two_add(float& hi, float& lo, float xh, float xl) {
    const float t = __fadd_rn(hi, xh);
    const float bp = __fsub_rn(t, hi);
    lo = __fadd_rn(lo, __fadd_rn(__fadd_rn(__fsub_rn(hi, __fsub_rn(t, bp)), __fsub_rn(xh, bp)), xl));
    hi = t;
}

// Gm (nc x nc, symmetric, float64) = sum over CTAs of the partials.  Block
// (x, y) covers entries (ci = y, cj = 32 x + lane) with cj >= ci; warp w adds
// the partials of CTAs [w * cpw, (w + 1) * cpw) as float32 two-word sums
// (float64 arithmetic issues at 1/64 of the float32 rate on this part; two
// words carry ~44 bits, far below the 3xTF32 product error), eight loads
// issued before their adds, and warp 0 adds the eight warp sums in order:
// the result does not depend on scheduling.
__global__ void __launch_bounds__(256) k_gram_tc_reduce(const float* __restrict__ part,
                                                        const float* __restrict__ vpart, int grid, int d, int dp,
                                                        int nc, double* __restrict__ Gm, float* __restrict__ W32) {
    const int ci = blockIdx.y, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if ((int)blockIdx.x * 32 + 31 < ci) return;   // the whole block below the diagonal
    __shared__ float2 sp[8][32];
    const int cj = blockIdx.x * 32 + lane;
    const bool act = cj < nc && cj >= ci;
    const float* src = nullptr;
    size_t stride = 0;
    if (act) {
        if (cj < d) {
            src = part + (size_t)ci * dp + cj;
            stride = gt_pstride(dp);
        } else {
            src = vpart + ci;
            stride = (size_t)d + 1;
        }
    }
    const int cpw = (grid + 7) / 8, c0 = warp * cpw, c1 = min(grid, c0 + cpw);
    float hi = 0.f, lo = 0.f;
    if (act) {
        for (int c = c0; c < c1; c += 8) {
            float v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) v[u] = c + u < c1 ? __ldg(src + (size_t)(c + u) * stride) : 0.f;
#pragma unroll
            for (int u = 0; u < 8; ++u)
                if (c + u < c1) gt_two_add(hi, lo, v[u], 0.f);
        }
    }
    sp[warp][lane] = make_float2(hi, lo);
    __syncthreads();
    if (warp == 0 && act) {
        float th = sp[0][lane].x, tl = sp[0][lane].y;
#pragma unroll
        for (int w = 1; w < 8; ++w) gt_two_add(th, tl, sp[w][lane].x, sp[w][lane].y);
        const double t = (double)th + (double)tl;
        Gm[(int64_t)ci * nc + cj] = t;
        Gm[(int64_t)cj * nc + ci] = t;
        if (W32) {
            W32[(int64_t)ci * nc + cj] = (float)t;
            W32[(int64_t)cj * nc + ci] = (float)t;
        }
    }
}

}  // namespace

// [SA | Sb]^T [SA | Sb] into Gm (nc = d + 1, float64, symmetric; nc = d and
// SA^T SA alone when Sb is NULL) on the tensor cores; CW_ERR_SHAPE (nothing
// launched) when d > 256.  W32 (nullable): the same matrix rounded to float32.  With
// `tflag` (device word, zeroed by the caller) an MMA wait that gave up is
// recorded there and the call does not synchronise; without it the call
// synchronises and returns CW_ERR_TIMEOUT for that case.
int gram_tc(const float* SA, int64_t m, int d, const float* Sb, double* Gm, unsigned* tflag_ext,
            cudaStream_t stream, float* W32) {
    if (d < 1 || d > kGtMaxD || m < 1) return CW_ERR_SHAPE;
    const int dp = (d + 15) & ~15;
    int grid = num_sms();
    const int64_t stages = (m + kGtKC - 1) / kGtKC;
    if (stages < grid) grid = (int)stages;
    int64_t rows_per = (m + grid - 1) / grid;
    rows_per = (rows_per + kGtKC - 1) / kGtKC * kGtKC;
    grid = (int)((m + rows_per - 1) / rows_per);
    const int nc = d + (Sb ? 1 : 0);
    Scratch ws(stream);
    const size_t oP = ws.reserve(sizeof(float) * (size_t)grid * gt_pstride(dp));
    const size_t oV = ws.reserve(sizeof(float) * (size_t)grid * (d + 1));
    const size_t oF = ws.reserve(sizeof(unsigned) * 2);
    CW_CUDA_TRY(ws.alloc());
    unsigned* tflag = tflag_ext ? tflag_ext : ws.at<unsigned>(oF);
    if (!tflag_ext) CW_CUDA_TRY(cudaMemsetAsync(tflag, 0, sizeof(unsigned) * 2, stream));
    GramTcArgs a{SA, Sb, m, d, dp, rows_per, ws.at<float>(oP), ws.at<float>(oV), tflag};
    CW_CUDA_TRY(cudaFuncSetAttribute(k_gram_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kGtSmem));
    {
        CW_PROF("k_gram_tc", stream);
        k_gram_tc<<<grid, kGtThreads, kGtSmem, stream>>>(a);
    }
    CW_LAUNCH_CHECK();
    {
        CW_PROF("k_gram_tc_reduce", stream);
        k_gram_tc_reduce<<<dim3((unsigned)((nc + 31) / 32), (unsigned)nc), 256, 0, stream>>>(a.part, a.vpart, grid, d,
                                                                                            dp, nc, Gm, W32);
    }
    CW_LAUNCH_CHECK();
    if (tflag_ext) return CW_OK;
    unsigned h = 0;
    CW_CUDA_TRY(cudaMemcpyAsync(&h, tflag, sizeof(unsigned), cudaMemcpyDeviceToHost, stream));
    CW_CUDA_TRY(cudaStreamSynchronize(stream));
    return h ? CW_ERR_TIMEOUT : CW_OK;
}

}  // namespace cw
