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
//   K4  k_apply_*       one CTA per coarse bin (a group of G buckets): stable
//                       counting sort of the group's records by bucket in
//                       shared memory (this is the permutation P of Section
//                       5.2: rows of h^-1(1) first, then h^-1(2), ...), then
//                       warps take whole buckets and add sigma(i) A_i into the
//                       bucket's row in ascending row order; the finished SA
//                       row is written once.  No global atomics, no floating
//                       point atomics: results are bitwise reproducible.
#include <algorithm>
#include <cmath>

#include "cw_common.cuh"
#include "cw_internal.h"

namespace cw {

constexpr int kTileWarps = 8;
constexpr int kTileRowsPerLane = 32;
constexpr int kTileRowsPerWarp = 32 * kTileRowsPerLane;       // 1024
constexpr int kTileRows = kTileWarps * kTileRowsPerWarp;      // 8192
constexpr int kMaxBins = 2048;
constexpr int kMaxGroupBuckets = 256;
constexpr int kScanChunk = 64;  // tiles per scan chunk

enum SketchMode { kModeCSR = 0, kModeDense = 1, kModeVec = 2 };

// ---------------------------------------------------------------- K1: tile histograms

__global__ void __launch_bounds__(256) k_tile_hist(HashParams hp, int64_t i0, int64_t n, int gshift,
                                                   int nbins, uint32_t* __restrict__ H) {
    __shared__ uint32_t h[kMaxBins];
    for (int b = threadIdx.x; b < nbins; b += blockDim.x) h[b] = 0;
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t r0 = (int64_t)blockIdx.x * kTileRows + warp * kTileRowsPerWarp + lane;
    if (r0 < n) {
        KeyWalk kw;
        kw.init(hp, (uint64_t)(i0 + r0), 32);
#pragma unroll 4
        for (int j = 0; j < kTileRowsPerLane; ++j) {
            if (r0 + 32 * j >= n) break;
            const uint32_t key = kw.key(hp);
            atomicAdd(&h[(key & 0x7FFFFFFFu) >> gshift], 1u);
            kw.step();
        }
    }
    __syncthreads();
    for (int b = threadIdx.x; b < nbins; b += blockDim.x) H[(size_t)blockIdx.x * nbins + b] = h[b];
}

// ---------------------------------------------------------------- S1-S3: scan of H (bin-major order)

// P[c][b] = sum of H[t][b] over tiles t of chunk c.
__global__ void k_scan_chunk_sums(const uint32_t* __restrict__ H, int ntiles, int nbins,
                                  uint32_t* __restrict__ P) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    const int c = blockIdx.y;
    if (b >= nbins) return;
    const int t0 = c * kScanChunk, t1 = min(ntiles, t0 + kScanChunk);
    uint32_t s = 0;
#pragma unroll 16
    for (int t = t0; t < t1; ++t) s += H[(size_t)t * nbins + b];
    P[(size_t)c * nbins + b] = s;
}

// Single CTA: per-bin totals, exclusive scan over bins (-> coarse_ptr), then
// P[c][b] becomes the offset of chunk c within bin b plus the bin's start.
__global__ void __launch_bounds__(1024) k_scan_bins(uint32_t* __restrict__ P, int nchunks, int nbins,
                                                    uint32_t* __restrict__ coarse_ptr, uint32_t n) {
    __shared__ uint32_t tot[kMaxBins];
    __shared__ uint32_t wsum[32];
    const int tid = threadIdx.x;
    for (int b = tid; b < nbins; b += blockDim.x) {
        uint32_t s = 0;
        for (int c = 0; c < nchunks; ++c) s += P[(size_t)c * nbins + b];
        tot[b] = s;
    }
    __syncthreads();
    // exclusive scan of tot[0..nbins) with 1024 threads, 2 bins per thread
    const int per = (nbins + blockDim.x - 1) / blockDim.x;
    uint32_t local = 0;
    for (int q = 0; q < per; ++q) {
        const int b = tid * per + q;
        if (b < nbins) local += tot[b];
    }
    uint32_t incl = local;
    const int lane = tid & 31, warp = tid >> 5;
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t v = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if (lane >= o) incl += v;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        uint32_t v = (lane < (int)(blockDim.x >> 5)) ? wsum[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t u = __shfl_up_sync(0xFFFFFFFFu, v, o);
            if (lane >= o) v += u;
        }
        wsum[lane] = v;
    }
    __syncthreads();
    uint32_t run = incl - local + (warp ? wsum[warp - 1] : 0);
    __syncthreads();
    for (int q = 0; q < per; ++q) {
        const int b = tid * per + q;
        if (b < nbins) {
            const uint32_t t = tot[b];
            tot[b] = run;
            run += t;
        }
    }
    __syncthreads();
    for (int b = tid; b < nbins; b += blockDim.x) {
        uint32_t off = tot[b];
        coarse_ptr[b] = off;
        for (int c = 0; c < nchunks; ++c) {
            const uint32_t t = P[(size_t)c * nbins + b];
            P[(size_t)c * nbins + b] = off;
            off += t;
        }
    }
    if (tid == 0) coarse_ptr[nbins] = n;
}

// H[t][b] <- output offset of tile t's rows of bin b (in place).
__global__ void k_scan_tiles(uint32_t* __restrict__ H, const uint32_t* __restrict__ P, int ntiles,
                             int nbins) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    const int c = blockIdx.y;
    if (b >= nbins) return;
    const int t0 = c * kScanChunk, t1 = min(ntiles, t0 + kScanChunk);
    uint32_t run = P[(size_t)c * nbins + b];
    uint32_t v[kScanChunk];
#pragma unroll
    for (int q = 0; q < kScanChunk; ++q) v[q] = (t0 + q < t1) ? H[(size_t)(t0 + q) * nbins + b] : 0u;
#pragma unroll
    for (int q = 0; q < kScanChunk; ++q) {
        if (t0 + q < t1) H[(size_t)(t0 + q) * nbins + b] = run;
        run += v[q];
    }
}

// ---------------------------------------------------------------- K3: coarse stable scatter

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned r;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(r));
    return r;
}

template <int MODE, bool HAS_B>
__global__ void __launch_bounds__(256) k_coarse_scatter(HashParams hp, int64_t i0, int64_t n, int gshift,
                                                        int nbins, const uint32_t* __restrict__ O,
                                                        const int32_t* __restrict__ row_ptr,
                                                        const float* __restrict__ b,
                                                        uint32_t* __restrict__ rkey, int32_t* __restrict__ ra,
                                                        int32_t* __restrict__ rlen, float* __restrict__ rb,
                                                        unsigned* status) {
    extern __shared__ uint32_t cnt[];  // [kTileWarps][nbins]
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int q = threadIdx.x; q < kTileWarps * nbins; q += blockDim.x) cnt[q] = 0;
    __syncthreads();

    const int64_t r0 = (int64_t)blockIdx.x * kTileRows + warp * kTileRowsPerWarp + lane;
    uint32_t keys[kTileRowsPerLane];
    {
        KeyWalk kw;
        kw.init(hp, (uint64_t)(i0 + (r0 < n ? r0 : 0)), 32);
#pragma unroll
        for (int j = 0; j < kTileRowsPerLane; ++j) {
            keys[j] = kw.key(hp);
            kw.step();
        }
    }
    uint32_t* wc = cnt + warp * nbins;
#pragma unroll
    for (int j = 0; j < kTileRowsPerLane; ++j)
        if (r0 + 32 * j < n) atomicAdd(&wc[(keys[j] & 0x7FFFFFFFu) >> gshift], 1u);
    __syncthreads();
    for (int bin = threadIdx.x; bin < nbins; bin += blockDim.x) {
        uint32_t run = O[(size_t)blockIdx.x * nbins + bin];
#pragma unroll
        for (int w = 0; w < kTileWarps; ++w) {
            const uint32_t t = cnt[w * nbins + bin];
            cnt[w * nbins + bin] = run;
            run += t;
        }
    }
    __syncthreads();

    const unsigned lt = lanemask_lt();
#pragma unroll
    for (int j0 = 0; j0 < kTileRowsPerLane; j0 += 4) {
        int32_t st[4], ln[4];
        float bv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int64_t r = r0 + 32 * (j0 + u);
            st[u] = 0;
            ln[u] = 0;
            bv[u] = 0.f;
            if (r < n) {
                if (MODE == kModeCSR) {
                    st[u] = __ldg(row_ptr + r);
                    ln[u] = __ldg(row_ptr + r + 1) - st[u];
                }
                if (HAS_B) bv[u] = __ldg(b + r);
            }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int j = j0 + u;
            const int64_t r = r0 + 32 * j;
            const bool valid = r < n;
            const unsigned am = __ballot_sync(0xFFFFFFFFu, valid);
            if (am == 0) break;
            const uint32_t key = keys[j];
            const uint32_t bin = (key & 0x7FFFFFFFu) >> gshift;
            unsigned peers = 0;
            uint32_t pos = 0;
            if (valid) {
                peers = __match_any_sync(am, bin);
                pos = wc[bin] + __popc(peers & lt);
            }
            __syncwarp();
            if (valid && (__ffs(peers) - 1) == lane) wc[bin] += __popc(peers);
            __syncwarp();
            if (valid) {
                rkey[pos] = key;
                if (MODE == kModeCSR) {
                    int32_t L = ln[u];
                    if (L < 0) {
                        flag_error(status, kDevBadRowPtr);
                        L = 0;
                    }
                    ra[pos] = st[u];
                    rlen[pos] = L;
                } else if (MODE == kModeDense) {
                    ra[pos] = (int32_t)r;
                }
                if (HAS_B) rb[pos] = (key >> 31) ? -bv[u] : bv[u];
            }
        }
    }
}

// ---------------------------------------------------------------- K4 common: in-CTA stable sort

struct GroupSort {
    uint32_t* cnt;     // [warps][G]
    uint32_t* bstart;  // [G + 1]
};

// Counts the chunk's records [c0, c1) per fine bucket for each warp's
// contiguous segment, scans, and leaves in cnt[w][fb] the first output slot of
// warp w's records of bucket fb, and in bstart[] the bucket starts (relative
// to c0).
__device__ __forceinline__ void group_count_scan(const uint32_t* __restrict__ rkey, uint32_t c0, uint32_t c1,
                                                 int G, int nwarps, GroupSort gsrt) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int q = threadIdx.x; q < nwarps * G; q += blockDim.x) gsrt.cnt[q] = 0;
    __syncthreads();
    const uint32_t len = c1 - c0;
    const uint32_t seg = ((len + nwarps - 1) / nwarps + 31) & ~31u;
    const uint32_t s0 = c0 + min(len, seg * warp), s1 = c0 + min(len, seg * (warp + 1));
    uint32_t* wc = gsrt.cnt + warp * G;
    for (uint32_t k = s0 + lane; k < s1; k += 32) atomicAdd(&wc[__ldg(rkey + k) & (G - 1)], 1u);
    __syncthreads();
    // bucket totals -> exclusive scan over buckets (G <= 256 <= blockDim)
    __shared__ uint32_t wsum[32];
    uint32_t tot = 0;
    const int b = threadIdx.x;
    if (b < G)
        for (int w = 0; w < nwarps; ++w) tot += gsrt.cnt[w * G + b];
    uint32_t incl = tot;
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t v = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if (lane >= o) incl += v;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        uint32_t v = (lane < (int)(blockDim.x >> 5)) ? wsum[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t u = __shfl_up_sync(0xFFFFFFFFu, v, o);
            if (lane >= o) v += u;
        }
        wsum[lane] = v;
    }
    __syncthreads();
    if (b < G) {
        uint32_t off = incl - tot + (warp ? wsum[warp - 1] : 0);
        gsrt.bstart[b] = off;
        for (int w = 0; w < nwarps; ++w) {
            const uint32_t t = gsrt.cnt[w * G + b];
            gsrt.cnt[w * G + b] = off;
            off += t;
        }
    }
    if (threadIdx.x == 0) gsrt.bstart[G] = len;
    __syncthreads();
}

// ---------------------------------------------------------------- K4: CSR apply

struct CsrApplyArgs {
    const uint32_t* rkey;
    const int32_t* ra;
    const int32_t* rlen;
    const float* rb;
    const uint32_t* coarse_ptr;
    const int32_t* col;
    const float* val;
    float* SA;
    float* Sb;
    int32_t* bucket_ptr;
    unsigned* status;
    int64_t m;
    int d;
    int dpad;      // accumulator row stride (floats)
    int gshift;
    int cap;       // records per chunk held in shared memory
    int acc_global;  // 1: accumulate directly in SA (large d)
};

template <int LPR, int U, bool HAS_B>
__global__ void __launch_bounds__(512) k_apply_csr(CsrApplyArgs a) {
    constexpr int COPIES = 32 / LPR;
    extern __shared__ __align__(16) uint8_t smem[];
    const int nwarps = blockDim.x >> 5;
    const int G = 1 << a.gshift;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int sub = lane / LPR, sl = lane % LPR;

    int32_t* s_start = reinterpret_cast<int32_t*>(smem);
    uint32_t* s_len = reinterpret_cast<uint32_t*>(s_start + a.cap);
    float* s_b = reinterpret_cast<float*>(s_len + a.cap);
    uint32_t* cnt = reinterpret_cast<uint32_t*>(s_b + (HAS_B ? a.cap : 0));
    uint32_t* bstart = cnt + nwarps * G;
    int* s_next = reinterpret_cast<int*>(bstart + G + 1);
    float* acc_base = reinterpret_cast<float*>(s_next + 4);
    const GroupSort gsrt{cnt, bstart};

    const int g = blockIdx.x;
    const uint32_t r0 = a.coarse_ptr[g], r1 = a.coarse_ptr[g + 1];
    const int64_t b0 = (int64_t)g << a.gshift;
    const int nb = (int)((a.m - b0) < (int64_t)G ? (a.m - b0) : (int64_t)G);
    const bool multi = (r1 - r0) > (uint32_t)a.cap;

    if (multi) {
        // bucket_ptr over the whole group first (counts only)
        group_count_scan(a.rkey, r0, r1, G, nwarps, gsrt);
        for (int q = threadIdx.x; q < nb; q += blockDim.x) a.bucket_ptr[b0 + q] = (int32_t)(r0 + bstart[q]);
        __syncthreads();
    }

    for (uint32_t c0 = r0, first = 1; first || c0 < r1; c0 += a.cap, first = 0) {
        const uint32_t c1 = min(r1, c0 + (uint32_t)a.cap);
        group_count_scan(a.rkey, c0, c1, G, nwarps, gsrt);
        if (!multi)
            for (int q = threadIdx.x; q < nb; q += blockDim.x) a.bucket_ptr[b0 + q] = (int32_t)(r0 + bstart[q]);
        // place the chunk's records, stably sorted by bucket
        {
            const uint32_t len = c1 - c0;
            const uint32_t seg = ((len + nwarps - 1) / nwarps + 31) & ~31u;
            const uint32_t s0 = c0 + min(len, seg * warp), s1 = c0 + min(len, seg * (warp + 1));
            uint32_t* wc = cnt + warp * G;
            const unsigned lt = lanemask_lt();
            for (uint32_t kb = s0; kb < s1; kb += 32) {
                const uint32_t k = kb + lane;
                const bool valid = k < s1;
                const unsigned am = __ballot_sync(0xFFFFFFFFu, valid);
                uint32_t key = 0, L = 0;
                int32_t st = 0;
                float bv = 0.f;
                if (valid) {
                    key = __ldg(a.rkey + k);
                    st = __ldg(a.ra + k);
                    L = (uint32_t)__ldg(a.rlen + k);
                    if (HAS_B) bv = __ldg(a.rb + k);
                }
                const uint32_t fb = key & (G - 1);
                unsigned peers = 0;
                uint32_t pos = 0;
                if (valid) {
                    peers = __match_any_sync(am, fb);
                    pos = wc[fb] + __popc(peers & lt);
                }
                __syncwarp();
                if (valid && (__ffs(peers) - 1) == lane) wc[fb] += __popc(peers);
                __syncwarp();
                if (valid) {
                    s_start[pos] = st;
                    s_len[pos] = L | (key & 0x80000000u);
                    if (HAS_B) s_b[pos] = bv;
                }
            }
        }
        if (threadIdx.x == 0) *s_next = 0;
        __syncthreads();

        // warps take whole buckets; sub-warp `sub` adds rows s+sub, s+sub+COPIES, ...
        float* accw = a.acc_global ? nullptr : acc_base + (size_t)warp * COPIES * a.dpad;
        for (;;) {
            int bk = 0;
            if (lane == 0) bk = atomicAdd(s_next, 1);
            bk = __shfl_sync(0xFFFFFFFFu, bk, 0);
            if (bk >= nb) break;
            const int s = (int)bstart[bk], e = (int)bstart[bk + 1];
            if (!first && s == e) continue;
            float* SArow = a.SA + (size_t)(b0 + bk) * a.d;
            float* myacc;
            if (a.acc_global) {
                // large d: this warp owns the SA row; COPIES == 1 (LPR == 32)
                myacc = SArow;
                if (first)
                    for (int c = lane; c < a.d; c += 32) SArow[c] = 0.f;
                __syncwarp();
            } else {
                for (int c = lane; c < COPIES * a.dpad; c += 32) accw[c] = 0.f;
                __syncwarp();
                myacc = accw + sub * a.dpad;
            }
            float sbacc = 0.f;
            for (int k0 = s; k0 < e; k0 += COPIES * U) {
                int st[U];
                uint32_t ln[U];
                int cc[U];
                float vv[U];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int kk = k0 + u * COPIES + sub;
                    st[u] = 0;
                    ln[u] = 0;
                    if (kk < e) {
                        st[u] = s_start[kk];
                        ln[u] = s_len[kk];
                        if (HAS_B && sl == 0) sbacc += s_b[kk];
                    }
                }
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    cc[u] = 0;
                    vv[u] = 0.f;
                    if ((uint32_t)sl < (ln[u] & 0x7FFFFFFFu)) {
                        cc[u] = __ldg(a.col + st[u] + sl);
                        vv[u] = __ldg(a.val + st[u] + sl);
                    }
                }
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const uint32_t L = ln[u] & 0x7FFFFFFFu;
                    const bool neg = (ln[u] >> 31) != 0;
                    for (uint32_t t = sl; t < L; t += LPR) {
                        int c;
                        float v;
                        if (t == (uint32_t)sl) {
                            c = cc[u];
                            v = vv[u];
                        } else {
                            c = __ldg(a.col + st[u] + t);
                            v = __ldg(a.val + st[u] + t);
                        }
                        if ((unsigned)c < (unsigned)a.d)
                            myacc[c] += neg ? -v : v;
                        else
                            flag_error(a.status, kDevBadColumn);
                    }
                    __syncwarp();
                }
            }
            __syncwarp();
            if (!a.acc_global) {
                for (int c = lane; c < a.d; c += 32) {
                    float v = accw[c];
#pragma unroll
                    for (int cp = 1; cp < COPIES; ++cp) v += accw[cp * a.dpad + c];
                    if (first)
                        SArow[c] = v;
                    else
                        SArow[c] += v;
                }
            }
            if (HAS_B && a.Sb) {
                float v = __shfl_sync(0xFFFFFFFFu, sbacc, 0);
#pragma unroll
                for (int cp = 1; cp < COPIES; ++cp) v += __shfl_sync(0xFFFFFFFFu, sbacc, cp * LPR);
                if (lane == 0) a.Sb[b0 + bk] = first ? v : a.Sb[b0 + bk] + v;
            }
            __syncwarp();
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------- K4: dense apply

struct DenseApplyArgs {
    const uint32_t* rkey;
    const int32_t* ra;
    const float* rb;
    const uint32_t* coarse_ptr;
    const float* A;
    int64_t lda;
    float* SA;
    float* Sb;
    int32_t* bucket_ptr;
    int64_t m;
    int d;
    int gshift;
    int cap;
    int vec4;      // 1 when A rows and d allow 16-byte loads
    double* SA64;  // PRECISE: float64 output of the two-word sums
};

// Each warp owns a bucket; lane l holds columns {4l + 128 v .. +3} (vec4) or
// {l + 32 v} in registers; rows are added in ascending order.
// PRECISE: each accumulator is a float32 pair (hi, lo) updated by an exact
// two-sum, so SA is exact to ~2^-48 relative and is written in float64.
__device__ __forceinline__ void two_sum_acc(float& hi, float& lo, float x) {
    const float t = hi + x;
    const float bp = t - hi;
    lo += (hi - (t - bp)) + (x - bp);
    hi = t;
}

template <int NV, int U, bool HAS_B, bool PRECISE>
__global__ void __launch_bounds__(512) k_apply_dense(DenseApplyArgs a) {
    extern __shared__ __align__(16) uint8_t smem[];
    const int nwarps = blockDim.x >> 5;
    const int G = 1 << a.gshift;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint32_t* s_row = reinterpret_cast<uint32_t*>(smem);
    float* s_b = reinterpret_cast<float*>(s_row + a.cap);
    uint32_t* cnt = reinterpret_cast<uint32_t*>(s_b + (HAS_B ? a.cap : 0));
    uint32_t* bstart = cnt + nwarps * G;
    int* s_next = reinterpret_cast<int*>(bstart + G + 1);
    const GroupSort gsrt{cnt, bstart};

    const int g = blockIdx.x;
    const uint32_t r0 = a.coarse_ptr[g], r1 = a.coarse_ptr[g + 1];
    const int64_t b0 = (int64_t)g << a.gshift;
    const int nb = (int)((a.m - b0) < (int64_t)G ? (a.m - b0) : (int64_t)G);
    const bool multi = (r1 - r0) > (uint32_t)a.cap;
    constexpr int COLS_PER_PASS = NV * 128;  // vec4 layout covers 128 columns per v

    if (multi) {
        group_count_scan(a.rkey, r0, r1, G, nwarps, gsrt);
        for (int q = threadIdx.x; q < nb; q += blockDim.x) a.bucket_ptr[b0 + q] = (int32_t)(r0 + bstart[q]);
        __syncthreads();
    }
    for (uint32_t c0 = r0, first = 1; first || c0 < r1; c0 += a.cap, first = 0) {
        const uint32_t c1 = min(r1, c0 + (uint32_t)a.cap);
        group_count_scan(a.rkey, c0, c1, G, nwarps, gsrt);
        if (!multi)
            for (int q = threadIdx.x; q < nb; q += blockDim.x) a.bucket_ptr[b0 + q] = (int32_t)(r0 + bstart[q]);
        {
            const uint32_t len = c1 - c0;
            const uint32_t seg = ((len + nwarps - 1) / nwarps + 31) & ~31u;
            const uint32_t s0 = c0 + min(len, seg * warp), s1 = c0 + min(len, seg * (warp + 1));
            uint32_t* wc = cnt + warp * G;
            const unsigned lt = lanemask_lt();
            for (uint32_t kb = s0; kb < s1; kb += 32) {
                const uint32_t k = kb + lane;
                const bool valid = k < s1;
                const unsigned am = __ballot_sync(0xFFFFFFFFu, valid);
                uint32_t key = 0;
                int32_t row = 0;
                float bv = 0.f;
                if (valid) {
                    key = __ldg(a.rkey + k);
                    row = __ldg(a.ra + k);
                    if (HAS_B) bv = __ldg(a.rb + k);
                }
                const uint32_t fb = key & (G - 1);
                unsigned peers = 0;
                uint32_t pos = 0;
                if (valid) {
                    peers = __match_any_sync(am, fb);
                    pos = wc[fb] + __popc(peers & lt);
                }
                __syncwarp();
                if (valid && (__ffs(peers) - 1) == lane) wc[fb] += __popc(peers);
                __syncwarp();
                if (valid) {
                    s_row[pos] = (uint32_t)row | (key & 0x80000000u);
                    if (HAS_B) s_b[pos] = bv;
                }
            }
        }
        if (threadIdx.x == 0) *s_next = 0;
        __syncthreads();

        for (;;) {
            int bk = 0;
            if (lane == 0) bk = atomicAdd(s_next, 1);
            bk = __shfl_sync(0xFFFFFFFFu, bk, 0);
            if (bk >= nb) break;
            const int s = (int)bstart[bk], e = (int)bstart[bk + 1];
            if (!first && s == e) continue;
            float* SArow = a.SA + (size_t)(b0 + bk) * a.d;
            float sbacc = 0.f;
            if (HAS_B && lane == 0)
                for (int k = s; k < e; ++k) sbacc += s_b[k];
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
                    for (int u = 0; u < U; ++u) rr[u] = (k0 + u < e) ? s_row[k0 + u] : 0xFFFFFFFFu;
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
                if (PRECISE) {
                    double* row64 = a.SA64 + (size_t)(b0 + bk) * a.d;
#pragma unroll
                    for (int v = 0; v < NV; ++v) {
                        const float hv[4] = {acc[v].x, acc[v].y, acc[v].z, acc[v].w};
                        const float lv[4] = {accl[v].x, accl[v].y, accl[v].z, accl[v].w};
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            const int cq = a.vec4 ? cbase + v * 128 + lane * 4 + q : cbase + v * 128 + lane + 32 * q;
                            if (cq < a.d) {
                                const double val = (double)hv[q] + (double)lv[q];
                                row64[cq] = first ? val : row64[cq] + val;
                            }
                        }
                    }
                    continue;
                }
#pragma unroll
                for (int v = 0; v < NV; ++v) {
                    if (a.vec4) {
                        const int c = cbase + v * 128 + lane * 4;
                        if (c < a.d) {
                            float4* p = reinterpret_cast<float4*>(SArow + c);
                            if (first) {
                                *p = acc[v];
                            } else {
                                float4 o = *p;
                                o.x += acc[v].x; o.y += acc[v].y; o.z += acc[v].z; o.w += acc[v].w;
                                *p = o;
                            }
                        }
                    } else {
                        const int c = cbase + v * 128 + lane;
                        const float vals[4] = {acc[v].x, acc[v].y, acc[v].z, acc[v].w};
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            const int cq = c + 32 * q;
                            if (cq < a.d) SArow[cq] = first ? vals[q] : SArow[cq] + vals[q];
                        }
                    }
                }
            }
            if (HAS_B && a.Sb && lane == 0) a.Sb[b0 + bk] = first ? sbacc : a.Sb[b0 + bk] + sbacc;
            __syncwarp();
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------- K4: vector only (Sx)

__global__ void __launch_bounds__(256) k_apply_vec(const uint32_t* __restrict__ rkey, const float* __restrict__ rb,
                                                  const uint32_t* __restrict__ coarse_ptr, int64_t m, int gshift,
                                                  int cap, float* __restrict__ Sx, int32_t* __restrict__ bucket_ptr) {
    extern __shared__ __align__(16) uint8_t smem[];
    const int nwarps = blockDim.x >> 5;
    const int G = 1 << gshift;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float* s_b = reinterpret_cast<float*>(smem);
    uint32_t* cnt = reinterpret_cast<uint32_t*>(s_b + cap);
    uint32_t* bstart = cnt + nwarps * G;
    const GroupSort gsrt{cnt, bstart};
    const int g = blockIdx.x;
    const uint32_t r0 = coarse_ptr[g], r1 = coarse_ptr[g + 1];
    const int64_t b0 = (int64_t)g << gshift;
    const int nb = (int)((m - b0) < (int64_t)G ? (m - b0) : (int64_t)G);
    const bool multi = (r1 - r0) > (uint32_t)cap;
    if (multi) {
        group_count_scan(rkey, r0, r1, G, nwarps, gsrt);
        for (int q = threadIdx.x; q < nb; q += blockDim.x) bucket_ptr[b0 + q] = (int32_t)(r0 + bstart[q]);
        __syncthreads();
    }
    for (uint32_t c0 = r0, first = 1; first || c0 < r1; c0 += cap, first = 0) {
        const uint32_t c1 = min(r1, c0 + (uint32_t)cap);
        group_count_scan(rkey, c0, c1, G, nwarps, gsrt);
        if (!multi)
            for (int q = threadIdx.x; q < nb; q += blockDim.x) bucket_ptr[b0 + q] = (int32_t)(r0 + bstart[q]);
        const uint32_t len = c1 - c0;
        const uint32_t seg = ((len + nwarps - 1) / nwarps + 31) & ~31u;
        const uint32_t s0 = c0 + min(len, seg * warp), s1 = c0 + min(len, seg * (warp + 1));
        uint32_t* wc = cnt + warp * G;
        const unsigned lt = lanemask_lt();
        for (uint32_t kb = s0; kb < s1; kb += 32) {
            const uint32_t k = kb + lane;
            const bool valid = k < s1;
            const unsigned am = __ballot_sync(0xFFFFFFFFu, valid);
            uint32_t key = valid ? __ldg(rkey + k) : 0;
            const float bv = valid ? __ldg(rb + k) : 0.f;
            const uint32_t fb = key & (G - 1);
            unsigned peers = 0;
            uint32_t pos = 0;
            if (valid) {
                peers = __match_any_sync(am, fb);
                pos = wc[fb] + __popc(peers & lt);
            }
            __syncwarp();
            if (valid && (__ffs(peers) - 1) == lane) wc[fb] += __popc(peers);
            __syncwarp();
            if (valid) s_b[pos] = bv;
        }
        __syncthreads();
        for (int q = threadIdx.x; q < nb; q += blockDim.x) {
            const int s = (int)bstart[q], e = (int)bstart[q + 1];
            if (!first && s == e) continue;
            float acc = 0.f;
            for (int k = s; k < e; ++k) acc += s_b[k];
            Sx[b0 + q] = first ? acc : Sx[b0 + q] + acc;
        }
        __syncthreads();
    }
}

__global__ void k_set_last(int32_t* bucket_ptr, int64_t m, int32_t n) { bucket_ptr[m] = n; }

// ---------------------------------------------------------------- host driver

struct SketchPlan {
    int gshift, nbins, ntiles, nchunks;
    int cap;
    int warps;
    int lpr;
    int dpad;
    int acc_global;
    size_t smem;
};

namespace {

int ilog2_ceil(uint64_t v) {
    int s = 0;
    while ((1ull << s) < v) ++s;
    return s;
}

int ilog2_floor(double v) {
    int s = 0;
    while ((double)(1ull << (s + 1)) <= v && s < 62) ++s;
    return s;
}

}  // namespace

// Chooses the group size G = 2^gshift (buckets per K4 CTA) so that at most
// kMaxBins coarse bins exist, at most kMaxGroupBuckets buckets share a CTA, and
// the expected group (n G / m rows) fills about 60% of the shared-memory record
// capacity.  Larger groups are still correct: K4 then walks them in chunks.
int plan_sketch(int mode, int64_t n, int64_t d, int64_t m, bool has_b, SketchPlan* p) {
    const size_t smem_budget = 200 * 1024;
    const int nsm = num_sms();
    p->warps = 16;
    p->acc_global = 0;
    p->lpr = 32;
    p->dpad = 0;
    size_t acc_bytes = 0;
    size_t rec_bytes = 4 + (has_b ? 4 : 0);
    if (mode == kModeCSR) {
        rec_bytes = 8 + (has_b ? 4 : 0);
        p->lpr = 16;  // two rows per warp step (two accumulator copies)
        p->dpad = (int)((d + 31) & ~31ll) + 1;  // odd stride: copies start on different banks
        acc_bytes = (size_t)p->warps * 2 * p->dpad * sizeof(float);
        if (acc_bytes > 96 * 1024) {
            p->lpr = 32;
            acc_bytes = (size_t)p->warps * p->dpad * sizeof(float);
            while (acc_bytes > 96 * 1024 && p->warps > 8) {
                p->warps /= 2;
                acc_bytes = (size_t)p->warps * p->dpad * sizeof(float);
            }
            if (acc_bytes > 96 * 1024) {  // very wide rows: accumulate in the SA row itself
                p->acc_global = 1;
                acc_bytes = 0;
                p->warps = 16;
            }
        }
    } else if (mode == kModeVec) {
        p->warps = 8;
    }
    const int threads = p->warps * 32;
    const int gmax = std::min(ilog2_floor((double)std::min(threads, kMaxGroupBuckets)), ilog2_ceil((uint64_t)m));
    const int gmin = ilog2_ceil(((uint64_t)m + kMaxBins - 1) / kMaxBins);
    if (gmin > gmax && gmin > ilog2_floor((double)std::min(threads, kMaxGroupBuckets))) return CW_ERR_SHAPE;
    const size_t fixed = acc_bytes + (size_t)p->warps * kMaxGroupBuckets * 4 + (kMaxGroupBuckets + 1) * 4 + 64;
    size_t cap_budget = (smem_budget - fixed) / rec_bytes;
    cap_budget = std::min<size_t>(cap_budget, 1u << 16) & ~size_t(31);
    const double rows_per_bucket = (double)n / (double)m;
    // largest group that fits ~60% of the record budget
    const double tgt = 0.6 * (double)cap_budget / std::max(rows_per_bucket, 1e-9);
    const int g_fit = tgt >= 1.0 ? ilog2_floor(tgt) : 0;
    // enough groups to fill the GPU several times over
    const double par = (double)m / (8.0 * nsm);
    const int g_par = par >= 1.0 ? ilog2_floor(par) : 0;
    int gs = std::min(std::min(g_fit, g_par), gmax);
    gs = std::max(gs, gmin);
    p->gshift = gs;
    p->nbins = (int)(((uint64_t)m + (1ull << gs) - 1) >> gs);
    p->ntiles = (int)((n + kTileRows - 1) / kTileRows);
    p->nchunks = (p->ntiles + kScanChunk - 1) / kScanChunk;
    const int G = 1 << gs;
    const double mean = rows_per_bucket * G;
    size_t cap = (size_t)(1.25 * mean + 8.0 * sqrt(mean) + 64.0);
    cap = (cap + 31) & ~size_t(31);
    p->cap = (int)std::min(cap, cap_budget);
    p->smem = (size_t)p->cap * rec_bytes + (size_t)p->warps * G * 4 + (size_t)(G + 1) * 4 + 16 + acc_bytes;
    return CW_OK;
}

template <class F>
static cudaError_t set_smem(F* f, size_t bytes) {
    return cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

// mode: kModeCSR (row_ptr/col/val), kModeDense (A, lda), kModeVec (x in b).
// bucket_ptr_out: optional device array of m + 1 ints (bucket starts of the
// stable permutation); NULL uses internal scratch.
int sketch_impl(int mode, int64_t n, int64_t d, int64_t lda, int64_t i0, const int32_t* row_ptr,
                const int32_t* col, const float* val, const float* A, const float* b, int64_t m,
                uint64_t seed, float* SA, float* Sb, int32_t* bucket_ptr_out, cudaStream_t stream,
                double* SA64) {
    const bool has_b = b != nullptr && (mode == kModeVec || Sb != nullptr);
    if (n == 0) {
        if (SA && d > 0) CW_CUDA_TRY(cudaMemsetAsync(SA, 0, sizeof(float) * (size_t)m * (size_t)d, stream));
        if (SA64 && d > 0) CW_CUDA_TRY(cudaMemsetAsync(SA64, 0, sizeof(double) * (size_t)m * (size_t)d, stream));
        if (Sb) CW_CUDA_TRY(cudaMemsetAsync(Sb, 0, sizeof(float) * (size_t)m, stream));
        if (bucket_ptr_out) CW_CUDA_TRY(cudaMemsetAsync(bucket_ptr_out, 0, sizeof(int32_t) * (size_t)(m + 1), stream));
        return CW_OK;
    }
    SketchPlan p;
    int st = plan_sketch(mode, n, d, m, has_b, &p);
    if (st != CW_OK) return st;
    unsigned* status = device_status_word();
    if (!status) return CW_ERR_CUDA;
    const HashParams hp = make_hash_params(seed, m);

    Scratch ws(stream);
    const size_t oH = ws.reserve(sizeof(uint32_t) * (size_t)p.ntiles * p.nbins);
    const size_t oP = ws.reserve(sizeof(uint32_t) * (size_t)p.nchunks * p.nbins);
    const size_t oCP = ws.reserve(sizeof(uint32_t) * (size_t)(p.nbins + 1));
    const size_t oKey = ws.reserve(sizeof(uint32_t) * (size_t)n);
    const size_t oA = (mode != kModeVec) ? ws.reserve(sizeof(int32_t) * (size_t)n) : 0;
    const size_t oLen = (mode == kModeCSR) ? ws.reserve(sizeof(int32_t) * (size_t)n) : 0;
    const size_t oB = has_b ? ws.reserve(sizeof(float) * (size_t)n) : 0;
    const size_t oBP = bucket_ptr_out ? 0 : ws.reserve(sizeof(int32_t) * (size_t)(m + 1));
    CW_CUDA_TRY(ws.alloc());
    uint32_t* H = ws.at<uint32_t>(oH);
    uint32_t* P = ws.at<uint32_t>(oP);
    uint32_t* CP = ws.at<uint32_t>(oCP);
    uint32_t* rkey = ws.at<uint32_t>(oKey);
    int32_t* ra = (mode != kModeVec) ? ws.at<int32_t>(oA) : nullptr;
    int32_t* rlen = (mode == kModeCSR) ? ws.at<int32_t>(oLen) : nullptr;
    float* rb = has_b ? ws.at<float>(oB) : nullptr;
    int32_t* bptr = bucket_ptr_out ? bucket_ptr_out : ws.at<int32_t>(oBP);

    {
        CW_PROF("k_tile_hist", stream);
        k_tile_hist<<<p.ntiles, 256, 0, stream>>>(hp, i0, n, p.gshift, p.nbins, H);
    }
    CW_LAUNCH_CHECK();
    dim3 sg((p.nbins + 255) / 256, p.nchunks);
    {
        CW_PROF("k_scan_chunk_sums", stream);
        k_scan_chunk_sums<<<sg, 256, 0, stream>>>(H, p.ntiles, p.nbins, P);
    }
    CW_LAUNCH_CHECK();
    {
        CW_PROF("k_scan_bins", stream);
        k_scan_bins<<<1, 1024, 0, stream>>>(P, p.nchunks, p.nbins, CP, (uint32_t)n);
    }
    CW_LAUNCH_CHECK();
    {
        CW_PROF("k_scan_tiles", stream);
        k_scan_tiles<<<sg, 256, 0, stream>>>(H, P, p.ntiles, p.nbins);
    }
    CW_LAUNCH_CHECK();

    const size_t k3smem = sizeof(uint32_t) * kTileWarps * p.nbins;
#define CW_K3(MODE, HB)                                                                             \
    do {                                                                                            \
        auto kf = k_coarse_scatter<MODE, HB>;                                                       \
        CW_CUDA_TRY(set_smem(kf, k3smem));                                                          \
        CW_PROF("k_coarse_scatter", stream);                                                        \
        kf<<<p.ntiles, 256, k3smem, stream>>>(hp, i0, n, p.gshift, p.nbins, H, row_ptr, b, rkey, ra, \
                                              rlen, rb, status);                                    \
    } while (0)
    if (mode == kModeCSR) {
        if (has_b) CW_K3(kModeCSR, true); else CW_K3(kModeCSR, false);
    } else if (mode == kModeDense) {
        if (has_b) CW_K3(kModeDense, true); else CW_K3(kModeDense, false);
    } else {
        CW_K3(kModeVec, true);
    }
#undef CW_K3
    CW_LAUNCH_CHECK();

    if (mode == kModeCSR) {
        CsrApplyArgs a{rkey, ra, rlen, rb, CP, col, val, SA, Sb, bptr, status, m, (int)d, p.dpad,
                       p.gshift, p.cap, p.acc_global};
        const int threads = p.warps * 32;
#define CW_K4C(LPR, HB)                                                   \
    do {                                                                  \
        auto kf = k_apply_csr<LPR, 8, HB>;                                \
        CW_CUDA_TRY(set_smem(kf, p.smem));                                \
        CW_PROF("k_apply_csr", stream);                                   \
        kf<<<p.nbins, threads, p.smem, stream>>>(a);                      \
    } while (0)
        if (p.lpr == 16) {
            if (has_b) CW_K4C(16, true); else CW_K4C(16, false);
        } else {
            if (has_b) CW_K4C(32, true); else CW_K4C(32, false);
        }
#undef CW_K4C
    } else if (mode == kModeDense) {
        const bool vec4 = (lda % 4 == 0) && (d % 4 == 0) && ((reinterpret_cast<uintptr_t>(A) & 15) == 0) &&
                          ((reinterpret_cast<uintptr_t>(SA) & 15) == 0);
        DenseApplyArgs a{rkey, ra, rb, CP, A, lda, SA, Sb, bptr, m, (int)d, p.gshift, p.cap, vec4 ? 1 : 0, SA64};
        const int threads = p.warps * 32;
        const int nv = d <= 128 ? 1 : d <= 256 ? 2 : d <= 512 ? 4 : 8;
#define CW_K4D(NV, U, HB)                                                 \
    do {                                                                  \
        auto kf = k_apply_dense<NV, U, HB, false>;                        \
        CW_CUDA_TRY(set_smem(kf, p.smem));                                \
        CW_PROF("k_apply_dense", stream);                                 \
        kf<<<p.nbins, threads, p.smem, stream>>>(a);                      \
    } while (0)
#define CW_K4P(NV, U)                                                     \
    do {                                                                  \
        auto kf = k_apply_dense<NV, U, false, true>;                      \
        CW_CUDA_TRY(set_smem(kf, p.smem));                                \
        CW_PROF("k_apply_dense_precise", stream);                         \
        kf<<<p.nbins, threads, p.smem, stream>>>(a);                      \
    } while (0)
        if (SA64) {
            if (nv == 1) CW_K4P(1, 8); else if (nv == 2) CW_K4P(2, 4);
            else if (nv == 4) CW_K4P(4, 4); else CW_K4P(8, 2);
        } else if (has_b) {
            if (nv == 1) CW_K4D(1, 8, true); else if (nv == 2) CW_K4D(2, 4, true);
            else if (nv == 4) CW_K4D(4, 4, true); else CW_K4D(8, 2, true);
        } else {
            if (nv == 1) CW_K4D(1, 8, false); else if (nv == 2) CW_K4D(2, 4, false);
            else if (nv == 4) CW_K4D(4, 4, false); else CW_K4D(8, 2, false);
        }
#undef CW_K4D
#undef CW_K4P
    } else {
        auto kf = k_apply_vec;
        CW_CUDA_TRY(set_smem(kf, p.smem));
        CW_PROF("k_apply_vec", stream);
        kf<<<p.nbins, p.warps * 32, p.smem, stream>>>(rkey, rb, CP, m, p.gshift, p.cap, Sb, bptr);
    }
    CW_LAUNCH_CHECK();
    {
        CW_PROF("k_set_last", stream);
        k_set_last<<<1, 1, 0, stream>>>(bptr, m, (int32_t)n);
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
