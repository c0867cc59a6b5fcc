// SA = S A and Sb = S b for the sparse embedding S = Phi D (paper Section 2),
// in O(nnz(A)) (Theorem 1), as a deterministic bucketed signed segmented sum.
//
// Pipeline (one call):
//   K1  k_tile_hist     hash every row (forward differences of the two cubics)
//                       and count rows per coarse bin (bucket >> gshift) per
//                       8192-row tile.
//   S1-S3 k_scan_*       exclusive scan of the tile histograms in bin-major
//                       order -> each (tile, bin) gets its output offset.
//   K3  k_coarse_scatter stable scatter of per-row records (key, row start,
//                       row length, sigma*b) into coarse-bin order.  Rows are
//                       read coalesced here, once.
//   K4a k_fine_sort     one CTA per coarse bin (a group of G buckets): stable
//                       counting sort of the bin's records by bucket, the bin
//                       staged in shared memory (this is the permutation P of
//                       Section 5.2: rows of h^-1(1) first, then h^-1(2), ...),
//                       written as bucket-ordered {row start, length | sign}
//                       and sigma*b, with the bucket starts.
//   K4b k_apply_*       persistent warps take whole buckets from a counter and
//                       add sigma(i) A_i into the bucket's row in ascending row
//                       order (per-warp shared-memory copies summed in a fixed
//                       order); the finished SA row is written once.  No
//                       floating-point atomics: results are bitwise
//                       reproducible.
#include <algorithm>
#include <vector>
#include <cmath>

#include "cw_common.cuh"
#include "cw_internal.h"
#include "sketch_body.cuh"

namespace cw {

template <bool OUTER>
__global__ void __launch_bounds__(256) k_tile_hist(HashParams hp, int64_t i0, int64_t n, int gshift,
                                                   int nbins, uint32_t* __restrict__ H) {
    __shared__ uint32_t h[kMaxBins];
    tile_hist_body<OUTER>(hp, i0, n, gshift, nbins, blockIdx.x, H + (size_t)blockIdx.x * nbins, h);
}

__global__ void k_scan_chunk_sums(const uint32_t* __restrict__ H, int ntiles, int nbins,
                                  uint32_t* __restrict__ P) {
    scan_chunk_sums_body(H, ntiles, nbins, P, blockIdx.x * blockDim.x + threadIdx.x, blockIdx.y);
}

__global__ void __launch_bounds__(1024) k_scan_bins(uint32_t* __restrict__ P, int nchunks, int nbins,
                                                    uint32_t* __restrict__ coarse_ptr, uint32_t n) {
    __shared__ uint32_t tot[kMaxBins];
    __shared__ uint32_t wsum[32];
    scan_bins_body(P, nchunks, nbins, coarse_ptr, n, tot, wsum);
}

__global__ void k_scan_tiles(uint32_t* __restrict__ H, const uint32_t* __restrict__ P, int ntiles,
                             int nbins) {
    scan_tiles_body(H, P, ntiles, nbins, blockIdx.x * blockDim.x + threadIdx.x, blockIdx.y);
}

template <int MODE, bool HAS_B, bool OUTER>
__global__ void __launch_bounds__(256) k_coarse_scatter(HashParams hp, int64_t i0, int64_t n, int gshift,
                                                        int nbins, const uint32_t* __restrict__ O,
                                                        const int32_t* __restrict__ row_ptr,
                                                        const float* __restrict__ b, int4* __restrict__ rec,
                                                        unsigned* status) {
    extern __shared__ uint32_t sm3[];
    coarse_scatter_body<MODE, HAS_B, OUTER>(hp, i0, n, gshift, nbins, blockIdx.x, O + (size_t)blockIdx.x * nbins,
                                            row_ptr, b, rec, status, sm3);
}

template <int MODE, bool HAS_B>
__global__ void __launch_bounds__(256) k_coarse_scatter_vals(HashParams hp, int64_t i0, int64_t n, int gshift,
                                                             int nbins, const uint32_t* __restrict__ O,
                                                             const int32_t* __restrict__ row_ptr,
                                                             const float* __restrict__ b, int4* __restrict__ rec,
                                                             unsigned* status, const float* __restrict__ vals) {
    extern __shared__ uint32_t sm3[];
    coarse_scatter_body<MODE, HAS_B, false, true>(hp, i0, n, gshift, nbins, blockIdx.x,
                                                  O + (size_t)blockIdx.x * nbins, row_ptr, b, rec, status, sm3, vals);
}

template <int MODE, bool HAS_B>
__global__ void __launch_bounds__(512) k_fine_sort(const int4* __restrict__ rec, const uint32_t* __restrict__ coarse_ptr,
                                                   int64_t m, int gshift, int cap, int2* __restrict__ out2,
                                                   float* __restrict__ outb, int32_t* __restrict__ bucket_ptr) {
    extern __shared__ int4 srec[];   // [cap]
    __shared__ FineSortSmem fs;
    fine_sort_body<MODE, HAS_B>(rec, coarse_ptr, m, gshift, cap, out2, outb, bucket_ptr, blockIdx.x, srec, fs);
}

template <int LPR, int U, bool HAS_B>
__global__ void __launch_bounds__(256, 4) k_apply_csr(CsrApplyArgs a) {
    constexpr int COPIES = 32 / LPR;
    extern __shared__ __align__(16) float smacc[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int sub = lane / LPR, sl = lane % LPR;
    float* accw = a.acc_global ? nullptr : smacc + (size_t)warp * COPIES * a.dpad;
    for (;;) {
        unsigned bk = 0;
        if (lane == 0) bk = atomicAdd(a.counter, 1u);
        bk = __shfl_sync(0xFFFFFFFFu, bk, 0);
        if ((int64_t)bk >= a.m) break;
        apply_csr_bucket<LPR, U, HAS_B>(a, bk, accw, lane, sub, sl);
    }
}

template <int LPR, int U>
__global__ void __launch_bounds__(256) k_apply_csr_vals(CsrApplyArgs a) {
    constexpr int COPIES = 32 / LPR;
    extern __shared__ __align__(16) float smacc[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int sub = lane / LPR, sl = lane % LPR;
    float* accw = a.acc_global ? nullptr : smacc + (size_t)warp * COPIES * a.dpad;
    for (;;) {
        unsigned bk = 0;
        if (lane == 0) bk = atomicAdd(a.counter, 1u);
        bk = __shfl_sync(0xFFFFFFFFu, bk, 0);
        if ((int64_t)bk >= a.m) break;
        apply_csr_bucket<LPR, U, false, true>(a, bk, accw, lane, sub, sl);
    }
}

// ---------------------------------------------------------------- K4b: dense apply

struct DenseApplyArgs {
    const int2* rs;   // bucket-ordered {row | sign << 31, 0}
    const float* rb;
    const int32_t* bucket_ptr;
    const float* A;
    int64_t lda;
    float* SA;
    float* Sb;
    unsigned* counter;
    int64_t m;
    int d;
    int vec4;      // 1 when A rows and d allow 16-byte loads
    double* SA64;  // PRECISE: float64 output of the two-word sums
    const float* vals;  // VALS: the sketch's entry of row i is vals[i] (not its sign)
};

// PRECISE: each accumulator is a float32 pair (hi, lo) updated by an exact
// two-sum, so SA is exact to ~2^-48 relative and is written in float64.
__device__ __forceinline__ void two_sum_acc(float& hi, float& lo, float x) {
    const float t = hi + x;
    const float bp = t - hi;
    lo += (hi - (t - bp)) + (x - bp);
    hi = t;
}

// Each warp owns a bucket at a time; lane l holds columns {4l + 128 v .. +3}
// (vec4) or {l + 32 q + 128 v} in registers; rows are added in ascending order.
template <int NV, int U, bool HAS_B, bool PRECISE, bool VALS = false>
__global__ void __launch_bounds__(256) k_apply_dense(DenseApplyArgs a) {
    const int lane = threadIdx.x & 31;
    constexpr int COLS_PER_PASS = NV * 128;
    for (;;) {
        unsigned bk = 0;
        if (lane == 0) bk = atomicAdd(a.counter, 1u);
        bk = __shfl_sync(0xFFFFFFFFu, bk, 0);
        if ((int64_t)bk >= a.m) break;
        const int s = a.bucket_ptr[bk], e = a.bucket_ptr[bk + 1];
        float* SArow = a.SA ? a.SA + (size_t)bk * a.d : nullptr;
        float sbacc = 0.f;
        if (HAS_B) {
            for (int k0 = s; k0 < e; k0 += 32) {
                float t = (k0 + lane < e) ? __ldg(&a.rb[k0 + lane]) : 0.f;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xFFFFFFFFu, t, o);
                sbacc += t;
            }
        }
        for (int cbase = 0; cbase < a.d; cbase += COLS_PER_PASS) {
            float4 acc[NV];
            float4 accl[PRECISE ? NV : 1];
#pragma unroll
            for (int v = 0; v < NV; ++v) acc[v] = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
            for (int v = 0; v < (PRECISE ? NV : 1); ++v) accl[v] = make_float4(0.f, 0.f, 0.f, 0.f);
            for (int k0 = s; k0 < e; k0 += U) {
                float4 x[U][NV];
                uint32_t rr[U];
#pragma unroll
                for (int u = 0; u < U; ++u) rr[u] = (k0 + u < e) ? (uint32_t)__ldg(&a.rs[k0 + u].x) : 0xFFFFFFFFu;
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const bool ok = rr[u] != 0xFFFFFFFFu;
                    const float* rowp = a.A + (int64_t)(rr[u] & 0x7FFFFFFFu) * a.lda;
#pragma unroll
                    for (int v = 0; v < NV; ++v) {
                        x[u][v] = make_float4(0.f, 0.f, 0.f, 0.f);
                        if (ok) {
                            if (a.vec4) {
                                const int c = cbase + v * 128 + lane * 4;
                                if (c < a.d) x[u][v] = __ldg(reinterpret_cast<const float4*>(rowp + c));
                            } else {
                                const int c = cbase + v * 128 + lane;
                                if (c < a.d) x[u][v].x = __ldg(rowp + c);
                                if (c + 32 < a.d) x[u][v].y = __ldg(rowp + c + 32);
                                if (c + 64 < a.d) x[u][v].z = __ldg(rowp + c + 64);
                                if (c + 96 < a.d) x[u][v].w = __ldg(rowp + c + 96);
                            }
                        }
                    }
                }
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    if (rr[u] == 0xFFFFFFFFu) continue;
                    const bool neg = (rr[u] >> 31) != 0;
                    if (VALS) {
                        const float w = __ldg(a.vals + (rr[u] & 0x7FFFFFFFu));
#pragma unroll
                        for (int v = 0; v < NV; ++v) {
                            acc[v].x = fmaf(w, x[u][v].x, acc[v].x);
                            acc[v].y = fmaf(w, x[u][v].y, acc[v].y);
                            acc[v].z = fmaf(w, x[u][v].z, acc[v].z);
                            acc[v].w = fmaf(w, x[u][v].w, acc[v].w);
                        }
                        continue;
                    }
#pragma unroll
                    for (int v = 0; v < NV; ++v) {
                        if (PRECISE) {
                            const float sg = neg ? -1.f : 1.f;
                            two_sum_acc(acc[v].x, accl[v].x, sg * x[u][v].x);
                            two_sum_acc(acc[v].y, accl[v].y, sg * x[u][v].y);
                            two_sum_acc(acc[v].z, accl[v].z, sg * x[u][v].z);
                            two_sum_acc(acc[v].w, accl[v].w, sg * x[u][v].w);
                        } else if (neg) {
                            acc[v].x -= x[u][v].x; acc[v].y -= x[u][v].y;
                            acc[v].z -= x[u][v].z; acc[v].w -= x[u][v].w;
                        } else {
                            acc[v].x += x[u][v].x; acc[v].y += x[u][v].y;
                            acc[v].z += x[u][v].z; acc[v].w += x[u][v].w;
                        }
                    }
                }
            }
#pragma unroll
            for (int v = 0; v < NV; ++v) {
                const float hv[4] = {acc[v].x, acc[v].y, acc[v].z, acc[v].w};
                const float lv[4] = {PRECISE ? accl[v].x : 0.f, PRECISE ? accl[v].y : 0.f,
                                     PRECISE ? accl[v].z : 0.f, PRECISE ? accl[v].w : 0.f};
                if (PRECISE) {
                    double* row64 = a.SA64 + (size_t)bk * a.d;
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int cq = a.vec4 ? cbase + v * 128 + lane * 4 + q : cbase + v * 128 + lane + 32 * q;
                        if (cq < a.d) row64[cq] = (double)hv[q] + (double)lv[q];
                    }
                } else if (a.vec4) {
                    const int c = cbase + v * 128 + lane * 4;
                    if (c < a.d) *reinterpret_cast<float4*>(SArow + c) = acc[v];
                } else {
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int cq = cbase + v * 128 + lane + 32 * q;
                        if (cq < a.d) SArow[cq] = hv[q];
                    }
                }
            }
        }
        if (HAS_B && a.Sb && lane == 0) a.Sb[bk] = sbacc;
    }
}

// ---------------------------------------------------------------- K4b: vector only (Sx)

__global__ void __launch_bounds__(256) k_apply_vec(const float* __restrict__ rb, const int32_t* __restrict__ bucket_ptr,
                                                  int64_t m, float* __restrict__ Sx, unsigned* counter) {
    const int lane = threadIdx.x & 31;
    for (;;) {
        unsigned bk = 0;
        if (lane == 0) bk = atomicAdd(counter, 1u);
        bk = __shfl_sync(0xFFFFFFFFu, bk, 0);
        if ((int64_t)bk >= m) break;
        const int s = bucket_ptr[bk], e = bucket_ptr[bk + 1];
        float acc = 0.f;
        for (int k0 = s; k0 < e; k0 += 32) {
            float t = (k0 + lane < e) ? __ldg(&rb[k0 + lane]) : 0.f;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xFFFFFFFFu, t, o);
            acc += t;
        }
        if (lane == 0) Sx[bk] = acc;
    }
}

__global__ void k_set_last(int32_t* bucket_ptr, int64_t m, int32_t n) { bucket_ptr[m] = n; }

// mode: kModeCSR (row_ptr/col/val), kModeDense (A, lda), kModeVec (x in b).
// bucket_ptr_out: optional device array of m + 1 ints (bucket starts of the
// stable permutation); NULL uses internal scratch.  SA64 (dense only): write a
// float64 SA from two-word sums instead of the float32 SA.
int sketch_impl(int mode, int64_t n, int64_t d, int64_t lda, int64_t i0, const int32_t* row_ptr,
                const int32_t* col, const float* val, const float* A, const float* b, int64_t m,
                uint64_t seed, float* SA, float* Sb, int32_t* bucket_ptr_out, cudaStream_t stream,
                double* SA64, const SketchWorkspace* ext, const SketchLayout* lay, const float* vals,
                bool accumulate) {
    // with vals, the CSR pass forms SA only (its rb carries v_i); Sb comes
    // from a separate vector pass of the caller
    const bool has_b = b != nullptr && (mode == kModeVec || Sb != nullptr) && !(vals && mode == kModeCSR);
    if (lay && mode != kModeCSR) return CW_ERR_ARG;
    if (vals && (lay || SA64)) return CW_ERR_ARG;
    if (accumulate && (mode != kModeCSR || lay || vals || bucket_ptr_out)) return CW_ERR_ARG;
    if (n == 0 && (lay || accumulate)) return CW_OK;   // the caller zeroed the whole output / nothing to add
    if (n == 0) {
        if (SA && d > 0) CW_CUDA_TRY(cudaMemsetAsync(SA, 0, sizeof(float) * (size_t)m * (size_t)d, stream));
        if (SA64 && d > 0) CW_CUDA_TRY(cudaMemsetAsync(SA64, 0, sizeof(double) * (size_t)m * (size_t)d, stream));
        if (Sb) CW_CUDA_TRY(cudaMemsetAsync(Sb, 0, sizeof(float) * (size_t)m, stream));
        if (bucket_ptr_out) CW_CUDA_TRY(cudaMemsetAsync(bucket_ptr_out, 0, sizeof(int32_t) * (size_t)(m + 1), stream));
        return CW_OK;
    }
    SketchPlan p;
    int st = plan_sketch(mode, n, d, m, &p);
    if (st != CW_OK) return st;
    unsigned* status = ext ? ext->status : device_status_word();
    if (!status) return CW_ERR_CUDA;
    const HashParams hp = lay ? *lay->hp : make_hash_params(seed, m);

    Scratch ws = ext ? Scratch(stream, ext->base, ext->bytes) : Scratch(stream);
    const size_t oH = ws.reserve(sizeof(uint32_t) * (size_t)p.ntiles * p.nbins);
    const size_t oP = ws.reserve(sizeof(uint32_t) * (size_t)p.nchunks * p.nbins);
    const size_t oCP = ws.reserve(sizeof(uint32_t) * (size_t)(p.nbins + 1));
    const size_t oRec = ws.reserve(sizeof(int4) * (size_t)n);
    const size_t oR2 = (mode != kModeVec) ? ws.reserve(sizeof(int2) * (size_t)n) : 0;
    const bool need_rb = has_b || (vals && mode == kModeCSR);
    const size_t oRB = need_rb ? ws.reserve(sizeof(float) * (size_t)n) : 0;
    const size_t oBP = bucket_ptr_out ? 0 : ws.reserve(sizeof(int32_t) * (size_t)(m + 1));
    const size_t oCnt = ws.reserve(sizeof(unsigned) * 4);
    if (ext && ws.size() > ext->bytes) return CW_ERR_SHAPE;
    CW_CUDA_TRY(ws.alloc());
    uint32_t* H = ws.at<uint32_t>(oH);
    uint32_t* P = ws.at<uint32_t>(oP);
    uint32_t* CP = ws.at<uint32_t>(oCP);
    int4* rec = ws.at<int4>(oRec);
    int2* r2 = (mode != kModeVec) ? ws.at<int2>(oR2) : nullptr;
    float* rb = need_rb ? ws.at<float>(oRB) : nullptr;
    int32_t* bptr = bucket_ptr_out ? bucket_ptr_out : ws.at<int32_t>(oBP);
    unsigned* counter = ws.at<unsigned>(oCnt);
    CW_CUDA_TRY(cudaMemsetAsync(counter, 0, sizeof(unsigned) * 4, stream));

    {
        CW_PROF("k_tile_hist", stream);
        if (hp.outer)
            k_tile_hist<true><<<p.ntiles, 256, 0, stream>>>(hp, i0, n, p.gshift, p.nbins, H);
        else
            k_tile_hist<false><<<p.ntiles, 256, 0, stream>>>(hp, i0, n, p.gshift, p.nbins, H);
    }
    CW_LAUNCH_CHECK();
    dim3 sg((p.nbins + 255) / 256, p.nchunks);
    {
        CW_PROF("k_scan_chunk_sums", stream);
        k_scan_chunk_sums<<<sg, 256, 0, stream>>>(H, p.ntiles, p.nbins, P);
    }
    {
        CW_PROF("k_scan_bins", stream);
        k_scan_bins<<<1, 1024, 0, stream>>>(P, p.nchunks, p.nbins, CP, (uint32_t)n);
    }
    {
        CW_PROF("k_scan_tiles", stream);
        k_scan_tiles<<<sg, 256, 0, stream>>>(H, P, p.ntiles, p.nbins);
    }
    CW_LAUNCH_CHECK();

    const size_t k3smem = sizeof(uint32_t) * (size_t)kTileWarps * (p.nbins + kTileRowsPerWarp);
#define CW_K3(MODE, HB)                                                                                    \
    do {                                                                                                   \
        auto kf = k_coarse_scatter<MODE, HB, false>;                                                       \
        if (MODE == kModeCSR && hp.outer) kf = k_coarse_scatter<MODE, HB, (MODE == kModeCSR)>;             \
        CW_CUDA_TRY(set_smem(kf, k3smem));                                                                 \
        CW_PROF("k_coarse_scatter", stream);                                                               \
        kf<<<p.ntiles, 256, k3smem, stream>>>(hp, i0, n, p.gshift, p.nbins, H, row_ptr, b, rec, status);   \
    } while (0)
    // bins of up to fcap records are staged in shared memory by k_fine_sort
    const int fcap = 12 * 1024;
    const size_t k4smem = sizeof(int4) * (size_t)fcap;
#define CW_K4A(MODE, HB)                                                                                \
    do {                                                                                                \
        auto kf = k_fine_sort<MODE, HB>;                                                                \
        CW_CUDA_TRY(set_smem(kf, k4smem));                                                              \
        CW_PROF("k_fine_sort", stream);                                                                 \
        kf<<<p.nbins, 512, k4smem, stream>>>(rec, CP, m, p.gshift, fcap, r2, rb, bptr);                 \
    } while (0)
#define CW_K3V(MODE, HB)                                                                                   \
    do {                                                                                                   \
        auto kf = k_coarse_scatter_vals<MODE, HB>;                                                         \
        CW_CUDA_TRY(set_smem(kf, k3smem));                                                                 \
        CW_PROF("k_coarse_scatter", stream);                                                               \
        kf<<<p.ntiles, 256, k3smem, stream>>>(hp, i0, n, p.gshift, p.nbins, H, row_ptr, b, rec, status, vals); \
    } while (0)
    if (vals) {
        // the record's last word is v_i (CSR), v_i b_i (dense with b, vector)
        if (mode == kModeCSR) { CW_K3V(kModeCSR, false); CW_K4A(kModeCSR, true); }
        else if (mode == kModeDense && has_b) { CW_K3V(kModeDense, true); CW_K4A(kModeDense, true); }
        else if (mode == kModeDense) { CW_K3V(kModeDense, false); CW_K4A(kModeDense, false); }
        else { CW_K3V(kModeVec, true); CW_K4A(kModeVec, true); }
    } else if (mode == kModeCSR) {
        if (has_b) { CW_K3(kModeCSR, true); CW_K4A(kModeCSR, true); }
        else { CW_K3(kModeCSR, false); CW_K4A(kModeCSR, false); }
    } else if (mode == kModeDense) {
        if (has_b) { CW_K3(kModeDense, true); CW_K4A(kModeDense, true); }
        else { CW_K3(kModeDense, false); CW_K4A(kModeDense, false); }
    } else {
        CW_K3(kModeVec, true);
        CW_K4A(kModeVec, true);
    }
#undef CW_K3
#undef CW_K3V
#undef CW_K4A
    CW_LAUNCH_CHECK();
    {
        CW_PROF("k_set_last", stream);
        k_set_last<<<1, 1, 0, stream>>>(bptr, m, (int32_t)n);
    }
    CW_LAUNCH_CHECK();

    if (mode == kModeCSR) {
        const bool vec4 = (d % 4 == 0) && ((reinterpret_cast<uintptr_t>(SA) & 15) == 0);
        CsrApplyArgs a{r2, rb, bptr, col, val, SA, Sb, counter, status, m, (int)d, p.dpad, p.acc_global,
                       vec4 ? 1 : 0, lay ? lay->v : 0, lay ? lay->stride : 0, lay ? lay->off : 0,
                       lay ? lay->scale : 1.f, accumulate ? 1 : 0};
#define CW_K4C(LPR, HB)                                                   \
    do {                                                                  \
        auto kf = k_apply_csr<LPR, 8, HB>;                                \
        CW_CUDA_TRY(set_smem(kf, p.acc_smem));                            \
        const int grid = persistent_grid(kf, 256, p.acc_smem);            \
        CW_PROF("k_apply_csr", stream);                                   \
        kf<<<grid, 256, p.acc_smem, stream>>>(a);                         \
    } while (0)
#define CW_K4CV(LPR)                                                      \
    do {                                                                  \
        auto kf = k_apply_csr_vals<LPR, 8>;                               \
        CW_CUDA_TRY(set_smem(kf, p.acc_smem));                            \
        const int grid = persistent_grid(kf, 256, p.acc_smem);            \
        CW_PROF("k_apply_csr", stream);                                   \
        kf<<<grid, 256, p.acc_smem, stream>>>(a);                         \
    } while (0)
        if (vals) {
            if (p.lpr == 16) CW_K4CV(16); else CW_K4CV(32);
        } else if (p.lpr == 16) {
            if (has_b) CW_K4C(16, true); else CW_K4C(16, false);
        } else {
            if (has_b) CW_K4C(32, true); else CW_K4C(32, false);
        }
#undef CW_K4C
#undef CW_K4CV
    } else if (mode == kModeDense) {
        const bool vec4 = (lda % 4 == 0) && (d % 4 == 0) && ((reinterpret_cast<uintptr_t>(A) & 15) == 0) &&
                          (SA64 || (reinterpret_cast<uintptr_t>(SA) & 15) == 0);
        DenseApplyArgs a{r2, rb, bptr, A, lda, SA, Sb, counter, m, (int)d, vec4 ? 1 : 0, SA64, vals};
        const int nv = d <= 128 ? 1 : d <= 256 ? 2 : d <= 512 ? 4 : 8;
#define CW_K4D(NV, U, HB, PR, NAME)                                       \
    do {                                                                  \
        auto kf = k_apply_dense<NV, U, HB, PR>;                           \
        const int grid = persistent_grid(kf, 256, 0);                     \
        CW_PROF(NAME, stream);                                            \
        kf<<<grid, 256, 0, stream>>>(a);                                  \
    } while (0)
#define CW_K4DV(NV, U, HB)                                                \
    do {                                                                  \
        auto kf = k_apply_dense<NV, U, HB, false, true>;                  \
        const int grid = persistent_grid(kf, 256, 0);                     \
        CW_PROF("k_apply_dense", stream);                                 \
        kf<<<grid, 256, 0, stream>>>(a);                                  \
    } while (0)
        if (vals) {
            if (has_b) {
                if (nv == 1) CW_K4DV(1, 8, true);
                else if (nv == 2) CW_K4DV(2, 4, true);
                else if (nv == 4) CW_K4DV(4, 4, true);
                else CW_K4DV(8, 2, true);
            } else {
                if (nv == 1) CW_K4DV(1, 8, false);
                else if (nv == 2) CW_K4DV(2, 4, false);
                else if (nv == 4) CW_K4DV(4, 4, false);
                else CW_K4DV(8, 2, false);
            }
        } else if (SA64) {
            if (nv == 1) CW_K4D(1, 8, false, true, "k_apply_dense_precise");
            else if (nv == 2) CW_K4D(2, 4, false, true, "k_apply_dense_precise");
            else if (nv == 4) CW_K4D(4, 4, false, true, "k_apply_dense_precise");
            else CW_K4D(8, 2, false, true, "k_apply_dense_precise");
        } else if (has_b) {
            if (nv == 1) CW_K4D(1, 8, true, false, "k_apply_dense");
            else if (nv == 2) CW_K4D(2, 4, true, false, "k_apply_dense");
            else if (nv == 4) CW_K4D(4, 4, true, false, "k_apply_dense");
            else CW_K4D(8, 2, true, false, "k_apply_dense");
        } else {
            if (nv == 1) CW_K4D(1, 8, false, false, "k_apply_dense");
            else if (nv == 2) CW_K4D(2, 4, false, false, "k_apply_dense");
            else if (nv == 4) CW_K4D(4, 4, false, false, "k_apply_dense");
            else CW_K4D(8, 2, false, false, "k_apply_dense");
        }
#undef CW_K4D
#undef CW_K4DV
    } else {
        const int grid = persistent_grid(k_apply_vec, 256, 0);
        CW_PROF("k_apply_vec", stream);
        k_apply_vec<<<grid, 256, 0, stream>>>(rb, bptr, m, Sb, counter);
    }
    CW_LAUNCH_CHECK();
    return CW_OK;
}

int validate_common(int64_t n, int64_t d, int64_t m) {
    if (n < 0 || d < 0 || m < 1) return CW_ERR_SHAPE;
    if (n > 0x7FFFFFFFll - 1) return CW_ERR_OVERFLOW;
    if (m > (1ll << 19)) return CW_ERR_SHAPE;
    if (d > (1ll << 20)) return CW_ERR_SHAPE;
    return CW_OK;
}

}  // namespace cw

using namespace cw;

extern "C" int cw_sketch_csr_rows(const cw_csr* A, int64_t i0, const float* b, int64_t m, uint64_t seed,
                                  float* SA, float* Sb, cw_stream stream) {
    if (!A || !SA) return CW_ERR_ARG;
    int st = validate_common(A->n, A->d, m);
    if (st != CW_OK) return st;
    if (A->d < 1) return CW_ERR_SHAPE;
    if (A->nnz < 0 || A->nnz > 0x7FFFFFFFll) return CW_ERR_OVERFLOW;
    if (i0 < 0 || i0 > (1ll << 62)) return CW_ERR_OVERFLOW;
    if (A->n > 0 && (!A->row_ptr || (A->nnz > 0 && (!A->col || !A->val)))) return CW_ERR_ARG;
    return sketch_impl(kModeCSR, A->n, A->d, 0, i0, A->row_ptr, A->col, A->val, nullptr, b, m, seed, SA,
                       b ? Sb : nullptr, nullptr, stream, nullptr);
}

extern "C" int cw_sketch_csr(const cw_csr* A, const float* b, int64_t m, uint64_t seed, float* SA, float* Sb,
                             cw_stream stream) {
    return cw_sketch_csr_rows(A, 0, b, m, seed, SA, Sb, stream);
}

// Generalized sparse embedding (Section "Generalized Sparse Embedding
// Matrices"): one pass of the CSR sketch per inner sketch b = 0..kappa-1 with
// the composite bucket h(i) * v + h_b(i) over q * v buckets; bucket u of pass
// b lands in output row (u / v) * v * kappa + b * v + u % v, scaled by
// 1 / sqrt(kappa).  The passes write disjoint rows and every row of the
// q * v * kappa output is written once.
extern "C" int cw_sketch_csr_general(const cw_csr* A, const float* b, int64_t q, int64_t v, int32_t kappa,
                                     uint64_t seed, float* SA, float* Sb, cw_stream stream) {
    if (!A || !SA) return CW_ERR_ARG;
    if (q < 1 || v < 1 || kappa < 1 || kappa > 4096) return CW_ERR_SHAPE;
    if (q > (1ll << 19) || v > (1ll << 19) || q * v > (1ll << 19)) return CW_ERR_SHAPE;
    const int64_t rows = q * v * (int64_t)kappa;
    if (rows > 0x7FFFFFFFll) return CW_ERR_OVERFLOW;
    int st = validate_common(A->n, A->d, q * v);
    if (st != CW_OK) return st;
    if (A->d < 1) return CW_ERR_SHAPE;
    if (A->nnz < 0 || A->nnz > 0x7FFFFFFFll) return CW_ERR_OVERFLOW;
    if (A->n > 0 && (!A->row_ptr || (A->nnz > 0 && (!A->col || !A->val)))) return CW_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    float* sb = b ? Sb : nullptr;
    if (A->n == 0) {
        CW_CUDA_TRY(cudaMemsetAsync(SA, 0, sizeof(float) * (size_t)rows * (size_t)A->d, s));
        if (sb) CW_CUDA_TRY(cudaMemsetAsync(sb, 0, sizeof(float) * (size_t)rows, s));
        return CW_OK;
    }
    std::vector<uint64_t> seeds((size_t)kappa);
    splitmix64_after_coeffs(seed, kappa, seeds.data());
    const float scale = (float)(1.0 / std::sqrt((double)kappa));
    for (int32_t pb = 0; pb < kappa; ++pb) {
        const HashParams hp = make_general_hash_params(seed, seeds[(size_t)pb], q, v);
        const SketchLayout lay{&hp, v, v * (int64_t)kappa, (int64_t)pb * v, scale};
        st = sketch_impl(kModeCSR, A->n, A->d, 0, 0, A->row_ptr, A->col, A->val, nullptr, b, q * v, seed, SA, sb,
                         nullptr, s, nullptr, nullptr, &lay);
        if (st != CW_OK) return st;
    }
    return CW_OK;
}

extern "C" int cw_sketch_dense(const float* A, int64_t n, int64_t d, int64_t lda, const float* b, int64_t m,
                               uint64_t seed, float* SA, float* Sb, cw_stream stream) {
    if (!SA || (n > 0 && !A)) return CW_ERR_ARG;
    int st = validate_common(n, d, m);
    if (st != CW_OK) return st;
    if (d < 1 || lda < d) return CW_ERR_SHAPE;
    return sketch_impl(kModeDense, n, d, lda, 0, nullptr, nullptr, nullptr, A, b, m, seed, SA,
                       b ? Sb : nullptr, nullptr, stream, nullptr);
}

extern "C" int cw_sketch_vec(const float* x, int64_t n, int64_t m, uint64_t seed, float* Sx, cw_stream stream) {
    if (!Sx || (n > 0 && !x)) return CW_ERR_ARG;
    int st = validate_common(n, 1, m);
    if (st != CW_OK) return st;
    return sketch_impl(kModeVec, n, 0, 0, 0, nullptr, nullptr, nullptr, nullptr, x, m, seed, nullptr, Sx,
                       nullptr, stream, nullptr);
}

// ---------------------------------------------------------------- CSR structure check

namespace cw {

// One warp per row: row_ptr non-decreasing, columns in [0, d), no column twice
// in a row.  Sets bits of *bad (1: row_ptr, 2: column range, 4: duplicate).
__global__ void k_csr_check(const int32_t* __restrict__ row_ptr, const int32_t* __restrict__ col, int64_t n,
                            int64_t d, int64_t nnz, unsigned* bad) {
    const int lane = threadIdx.x & 31;
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    if (w0 == 0 && lane == 0 && (row_ptr[0] != 0 || (int64_t)row_ptr[n] != nnz)) atomicOr(bad, 1u);
    for (int64_t r = w0; r < n; r += nw) {
        const int32_t s = row_ptr[r], e = row_ptr[r + 1];
        if (e < s || s < 0 || (int64_t)e > nnz) {
            if (lane == 0) atomicOr(bad, 1u);
            continue;
        }
        for (int32_t a0 = s; a0 < e; a0 += 32) {
            const int32_t ka = a0 + lane;
            const int32_t ca = ka < e ? col[ka] : -1;
            if (ka < e && (ca < 0 || (int64_t)ca >= d)) atomicOr(bad, 2u);
            for (int32_t b0 = a0; b0 < e; b0 += 32) {
                const int32_t kb = b0 + lane;
                const int32_t cb = kb < e ? col[kb] : -2;
                for (int q = 0; q < 32; ++q) {
                    const int32_t other = __shfl_sync(0xFFFFFFFFu, cb, q);
                    const int32_t ko = b0 + q;
                    if (ka < e && ko < e && ko > ka && other == ca) atomicOr(bad, 4u);
                }
            }
        }
    }
}

}  // namespace cw

extern "C" int cw_csr_check(const cw_csr* A, cw_stream stream) {
    if (!A) return CW_ERR_ARG;
    if (A->n < 0 || A->d < 0 || A->nnz < 0) return CW_ERR_SHAPE;
    if (A->n > 0x7FFFFFFFll - 1 || A->nnz > 0x7FFFFFFFll) return CW_ERR_OVERFLOW;
    if (!A->row_ptr || (A->nnz > 0 && !A->col)) return CW_ERR_ARG;
    Scratch ws(stream);
    const size_t o = ws.reserve(sizeof(unsigned));
    CW_CUDA_TRY(ws.alloc());
    unsigned* bad = ws.at<unsigned>(o);
    CW_CUDA_TRY(cudaMemsetAsync(bad, 0, sizeof(unsigned), stream));
    const int64_t warps = A->n > 0 ? A->n : 1;
    const int64_t blocks = std::min<int64_t>((warps + 7) / 8, 65535);
    {
        CW_PROF("k_csr_check", stream);
        k_csr_check<<<(unsigned)blocks, 256, 0, stream>>>(A->row_ptr, A->col, A->n, A->d, A->nnz, bad);
    }
    CW_LAUNCH_CHECK();
    unsigned h = 0;
    CW_CUDA_TRY(cudaMemcpyAsync(&h, bad, sizeof(unsigned), cudaMemcpyDeviceToHost, stream));
    CW_CUDA_TRY(cudaStreamSynchronize(stream));
    return h ? CW_ERR_ARG : CW_OK;
}

