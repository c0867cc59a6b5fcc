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
#include <vector>
#include <cmath>

#include "batch.h"
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

// Histogram of one 8192-row tile (rows r of [tile * 8192, ...) < n, hashed
// with global index i0 + r) over the coarse bins, written to Hrow[0..nbins).
template <bool OUTER>
__device__ __forceinline__ void tile_hist_body(const HashParams& hp, int64_t i0, int64_t n, int gshift, int nbins,
                                               int64_t tile, uint32_t* __restrict__ Hrow, uint32_t* h) {
    for (int b = threadIdx.x; b < nbins; b += blockDim.x) h[b] = 0;
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t r0 = tile * kTileRows + warp * kTileRowsPerWarp + lane;
    if (r0 < n) {
        KeyWalkT<OUTER> kw;
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
    for (int b = threadIdx.x; b < nbins; b += blockDim.x) Hrow[b] = h[b];
}

template <bool OUTER>
__global__ void __launch_bounds__(256) k_tile_hist(HashParams hp, int64_t i0, int64_t n, int gshift,
                                                   int nbins, uint32_t* __restrict__ H) {
    __shared__ uint32_t h[kMaxBins];
    tile_hist_body<OUTER>(hp, i0, n, gshift, nbins, blockIdx.x, H + (size_t)blockIdx.x * nbins, h);
}

// ---------------------------------------------------------------- S1-S3: scan of H (bin-major order)

// P[c][b] = sum of H[t][b] over tiles t of chunk c.
__device__ __forceinline__ void scan_chunk_sums_body(const uint32_t* __restrict__ H, int ntiles, int nbins,
                                                     uint32_t* __restrict__ P, int b, int c) {
    if (b >= nbins) return;
    const int t0 = c * kScanChunk, t1 = min(ntiles, t0 + kScanChunk);
    uint32_t s = 0;
#pragma unroll 16
    for (int t = t0; t < t1; ++t) s += H[(size_t)t * nbins + b];
    P[(size_t)c * nbins + b] = s;
}

__global__ void k_scan_chunk_sums(const uint32_t* __restrict__ H, int ntiles, int nbins,
                                  uint32_t* __restrict__ P) {
    scan_chunk_sums_body(H, ntiles, nbins, P, blockIdx.x * blockDim.x + threadIdx.x, blockIdx.y);
}

// Single CTA: per-bin totals, exclusive scan over bins (-> coarse_ptr), then
// P[c][b] becomes the offset of chunk c within bin b plus the bin's start.
__device__ __forceinline__ void scan_bins_body(uint32_t* __restrict__ P, int nchunks, int nbins,
                                               uint32_t* __restrict__ coarse_ptr, uint32_t n, uint32_t* tot,
                                               uint32_t* wsum) {
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

__global__ void __launch_bounds__(1024) k_scan_bins(uint32_t* __restrict__ P, int nchunks, int nbins,
                                                    uint32_t* __restrict__ coarse_ptr, uint32_t n) {
    __shared__ uint32_t tot[kMaxBins];
    __shared__ uint32_t wsum[32];
    scan_bins_body(P, nchunks, nbins, coarse_ptr, n, tot, wsum);
}

// H[t][b] <- output offset of tile t's rows of bin b (in place).
__device__ __forceinline__ void scan_tiles_body(uint32_t* __restrict__ H, const uint32_t* __restrict__ P, int ntiles,
                                                int nbins, int b, int c) {
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

__global__ void k_scan_tiles(uint32_t* __restrict__ H, const uint32_t* __restrict__ P, int ntiles,
                             int nbins) {
    scan_tiles_body(H, P, ntiles, nbins, blockIdx.x * blockDim.x + threadIdx.x, blockIdx.y);
}

// ---------------------------------------------------------------- K3: coarse stable scatter

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned r;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(r));
    return r;
}

// Per row one 16-byte record {key, a, len, sigma*b}: a = row start (CSR) or
// the row index (dense); written in coarse-bin order, stable within a bin.
// Tile `tile` of the rows; Orow = the tile's output offsets per bin.
// VALS: the sketch's entries are the given values v_i instead of the signs:
// the record's last word is v_i (times b_i with HAS_B) and the sign is unused.
template <int MODE, bool HAS_B, bool OUTER, bool VALS = false>
__device__ __forceinline__ void coarse_scatter_body(const HashParams& hp, int64_t i0, int64_t n, int gshift,
                                                    int nbins, int64_t tile, const uint32_t* __restrict__ Orow,
                                                    const int32_t* __restrict__ row_ptr,
                                                    const float* __restrict__ b, int4* __restrict__ rec,
                                                    unsigned* status, uint32_t* sm3,
                                                    const float* __restrict__ vals = nullptr) {
    uint32_t* cnt = sm3;                                // [kTileWarps][nbins]
    uint32_t* skeys = sm3 + kTileWarps * nbins;         // [kTileWarps][kTileRowsPerWarp]
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int q = threadIdx.x; q < kTileWarps * nbins; q += blockDim.x) cnt[q] = 0;
    __syncthreads();
    const int64_t r0 = tile * kTileRows + warp * kTileRowsPerWarp + lane;
    uint32_t* wk = skeys + warp * kTileRowsPerWarp;
    uint32_t* wc = cnt + warp * nbins;
    if (r0 < n) {
        KeyWalkT<OUTER> kw;
        kw.init(hp, (uint64_t)(i0 + r0), 32);
#pragma unroll 4
        for (int j = 0; j < kTileRowsPerLane; ++j) {
            if (r0 + 32 * j >= n) break;
            const uint32_t key = kw.key(hp);
            wk[lane + 32 * j] = key;
            atomicAdd(&wc[(key & 0x7FFFFFFFu) >> gshift], 1u);
            kw.step();
        }
    }
    __syncthreads();
    for (int bin = threadIdx.x; bin < nbins; bin += blockDim.x) {
        uint32_t run = Orow[bin];
#pragma unroll
        for (int w = 0; w < kTileWarps; ++w) {
            const uint32_t t = cnt[w * nbins + bin];
            cnt[w * nbins + bin] = run;
            run += t;
        }
    }
    __syncthreads();
    const unsigned lt = lanemask_lt();
#pragma unroll 1
    for (int j0 = 0; j0 < kTileRowsPerLane; j0 += 4) {
        if (r0 - lane + 32 * j0 >= n) break;
        int32_t st[4], ln[4];
        float bv[4], wv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int64_t r = r0 + 32 * (j0 + u);
            st[u] = 0;
            ln[u] = 0;
            bv[u] = 0.f;
            wv[u] = 0.f;
            if (r < n) {
                if (MODE == kModeCSR) {
                    st[u] = __ldg(row_ptr + r);
                    ln[u] = __ldg(row_ptr + r + 1) - st[u];
                } else if (MODE == kModeDense) {
                    st[u] = (int32_t)r;
                }
                if (HAS_B) bv[u] = __ldg(b + r);
                if (VALS) wv[u] = __ldg(vals + r);
            }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int j = j0 + u;
            const int64_t r = r0 + 32 * j;
            const bool valid = r < n;
            const unsigned am = __ballot_sync(0xFFFFFFFFu, valid);
            if (am == 0) break;
            const uint32_t key = valid ? wk[lane + 32 * j] : 0u;
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
                int32_t L = ln[u];
                if (MODE == kModeCSR && L < 0) {
                    flag_error(status, kDevBadRowPtr);
                    L = 0;
                }
                const float sb = VALS ? (HAS_B ? wv[u] * bv[u] : wv[u])
                                      : (HAS_B ? ((key >> 31) ? -bv[u] : bv[u]) : 0.f);
                rec[pos] = make_int4((int)key, st[u], L, __float_as_int(sb));
            }
        }
    }
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

// ---------------------------------------------------------------- K4a: fine stable sort per group

// One CTA per coarse bin (G = 2^gshift consecutive buckets): counting sort of
// the bin's records by bucket, stable, written to the same region in bucket
// order as {a | sign << 31 (dense) or a, len | sign << 31 (CSR)} and sigma*b;
// bucket_ptr for the bin's buckets.  This is the permutation P of Section 5.2.
//
// A bin of at most `cap` records is first copied into shared memory (16-byte
// asynchronous copies, all in flight at once), so both passes over it (count,
// then scatter) read shared memory and the records cross DRAM once; larger
// bins are read from global memory twice.
struct FineSortSmem {
    uint32_t cnt[16 * kMaxGroupBuckets];
    uint32_t bstart[kMaxGroupBuckets + 1];
    uint32_t wsum[32];
};

template <int MODE, bool HAS_B>
__device__ __forceinline__ void fine_sort_body(const int4* __restrict__ rec, const uint32_t* __restrict__ coarse_ptr,
                                               int64_t m, int gshift, int cap, int2* __restrict__ out2,
                                               float* __restrict__ outb, int32_t* __restrict__ bucket_ptr, int g,
                                               int4* srec, FineSortSmem& fs) {
    uint32_t* cnt = fs.cnt;
    uint32_t* bstart = fs.bstart;
    uint32_t* wsum = fs.wsum;
    const int nwarps = blockDim.x >> 5;
    const int G = 1 << gshift;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t r0 = coarse_ptr[g], r1 = coarse_ptr[g + 1];
    const int64_t b0 = (int64_t)g << gshift;
    const int nb = (int)((m - b0) < (int64_t)G ? (m - b0) : (int64_t)G);
    for (int q = threadIdx.x; q < nwarps * G; q += blockDim.x) cnt[q] = 0;
    const uint32_t len = r1 - r0;
    const bool staged = len <= (uint32_t)cap;
    if (staged) {
        for (uint32_t k = threadIdx.x; k < len; k += blockDim.x) cp_async16(&srec[k], &rec[r0 + k]);
        cp_async_commit();
        cp_async_wait_all();
    }
    __syncthreads();
    // record k (global index) from shared memory when staged
    auto ldrec = [&](uint32_t k) -> int4 { return staged ? srec[k - r0] : __ldg(&rec[k]); };
    const uint32_t seg = ((len + nwarps - 1) / nwarps + 31) & ~31u;
    const uint32_t s0 = r0 + min(len, seg * warp), s1 = r0 + min(len, seg * (warp + 1));
    uint32_t* wc = cnt + warp * G;
#pragma unroll 4
    for (uint32_t k = s0 + lane; k < s1; k += 32) atomicAdd(&wc[(uint32_t)ldrec(k).x & (G - 1)], 1u);
    __syncthreads();
    // bucket totals -> exclusive scan (G <= blockDim)
    uint32_t tot = 0;
    const int bq = threadIdx.x;
    if (bq < G)
        for (int w = 0; w < nwarps; ++w) tot += cnt[w * G + bq];
    uint32_t incl = tot;
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t v = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if (lane >= o) incl += v;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        uint32_t v = (lane < nwarps) ? wsum[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t u = __shfl_up_sync(0xFFFFFFFFu, v, o);
            if (lane >= o) v += u;
        }
        wsum[lane] = v;
    }
    __syncthreads();
    if (bq < G) {
        uint32_t off = incl - tot + (warp ? wsum[warp - 1] : 0);
        bstart[bq] = off;
        if (bq < nb) bucket_ptr[b0 + bq] = (int32_t)(r0 + off);
        for (int w = 0; w < nwarps; ++w) {
            const uint32_t t = cnt[w * G + bq];
            cnt[w * G + bq] = off;
            off += t;
        }
    }
    __syncthreads();
    const unsigned lt = lanemask_lt();
    constexpr int PF = 4;  // records loaded ahead per lane
    for (uint32_t kb0 = s0; kb0 < s1; kb0 += 32 * PF) {
      int4 rq[PF];
#pragma unroll
      for (int u = 0; u < PF; ++u) {
          const uint32_t k = kb0 + 32 * u + lane;
          rq[u] = (k < s1) ? ldrec(k) : make_int4(0, 0, 0, 0);
      }
#pragma unroll
      for (int u = 0; u < PF; ++u) {
        const uint32_t kb = kb0 + 32 * u;
        if (kb >= s1) break;
        const uint32_t k = kb + lane;
        const bool valid = k < s1;
        const unsigned am = __ballot_sync(0xFFFFFFFFu, valid);
        const int4 r = rq[u];
        const uint32_t key = (uint32_t)r.x;
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
            const uint32_t sgn = key & 0x80000000u;
            if (MODE == kModeCSR)
                out2[r0 + pos] = make_int2(r.y, (int)((uint32_t)r.z | sgn));
            else if (MODE == kModeDense)
                out2[r0 + pos] = make_int2((int)((uint32_t)r.y | sgn), 0);
            if (HAS_B) outb[r0 + pos] = __int_as_float(r.w);
        }
      }
    }
}

template <int MODE, bool HAS_B>
__global__ void __launch_bounds__(512) k_fine_sort(const int4* __restrict__ rec, const uint32_t* __restrict__ coarse_ptr,
                                                   int64_t m, int gshift, int cap, int2* __restrict__ out2,
                                                   float* __restrict__ outb, int32_t* __restrict__ bucket_ptr) {
    extern __shared__ int4 srec[];   // [cap]
    __shared__ FineSortSmem fs;
    fine_sort_body<MODE, HAS_B>(rec, coarse_ptr, m, gshift, cap, out2, outb, bucket_ptr, blockIdx.x, srec, fs);
}

// ---------------------------------------------------------------- K4b: CSR apply

struct CsrApplyArgs {
    const int2* rs;          // bucket-ordered {row start, len | sign << 31}
    const float* rb;         // bucket-ordered sigma * b
    const int32_t* bucket_ptr;
    const int32_t* col;
    const float* val;
    float* SA;
    float* Sb;
    unsigned* counter;       // next bucket (zeroed before launch)
    unsigned* status;
    int64_t m;
    int d;
    int dpad;
    int acc_global;          // accumulate in the SA row itself (very wide rows)
    int vec4;                // SA rows 16-byte aligned and d % 4 == 0
    // output row of bucket u: (u / map_v) * map_stride + map_off + u % map_v
    // (map_v == 0: row u), values times `scale`
    int64_t map_v, map_stride, map_off;
    float scale;
};

// Persistent warps take whole buckets from a counter; sub-warp `sub` of
// COPIES = 32 / LPR adds the bucket's rows sub, sub + COPIES, ... (in order)
// into its own shared-memory copy of the SA row; the copies are summed in a
// fixed order.  No block barriers, no floating-point atomics.
// One bucket bk of a.m: its SA row (and Sb entry) from the bucket's records.
// accw: the warp's COPIES * dpad shared-memory accumulators (unused with
// acc_global).
// VALS: rb holds each row's value v_i (bucket order); rows are scaled by it
// instead of their sign, and no Sb is formed.
template <int LPR, int U, bool HAS_B, bool VALS = false>
__device__ __forceinline__ void apply_csr_bucket(const CsrApplyArgs& a, unsigned bk, float* accw, int lane, int sub, int sl) {
    constexpr int COPIES = 32 / LPR;
    {
        const int s = a.bucket_ptr[bk], e = a.bucket_ptr[bk + 1];
        const int64_t orow = a.map_v ? ((int64_t)bk / a.map_v) * a.map_stride + a.map_off + (int64_t)bk % a.map_v
                                     : (int64_t)bk;
        float* SArow = a.SA + (size_t)orow * a.d;
        float* myacc;
        if (a.acc_global) {
            for (int c = lane; c < a.d; c += 32) SArow[c] = 0.f;
            myacc = SArow;
        } else {
            for (int c = lane; c < COPIES * a.dpad; c += 32) accw[c] = 0.f;
            myacc = accw + sub * a.dpad;
        }
        __syncwarp();
        float sbacc = 0.f;
        for (int k0 = s; k0 < e; k0 += 32) {
            // records of up to 32 rows: lane l holds row k0 + l
            int2 rr = make_int2(0, 0);
            float rbv = 0.f;
            if (k0 + lane < e) {
                rr = __ldg(&a.rs[k0 + lane]);
                if (HAS_B || VALS) rbv = __ldg(&a.rb[k0 + lane]);
            }
            if (HAS_B) {
                float t = rbv;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xFFFFFFFFu, t, o);
                sbacc += t;
            }
            const int nrow = min(32, e - k0);
#pragma unroll 1
            for (int t0 = 0; t0 < 32; t0 += COPIES * U) {
                if (t0 >= nrow) break;
                int st[U];
                uint32_t ln[U];
                int cc[U];
                float vv[U];
                float wt[VALS ? U : 1];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int t = t0 + u * COPIES + sub;  // row within the 32-row chunk
                    st[u] = __shfl_sync(0xFFFFFFFFu, rr.x, t & 31);
                    ln[u] = (uint32_t)__shfl_sync(0xFFFFFFFFu, rr.y, t & 31);
                    if (VALS) wt[VALS ? u : 0] = __shfl_sync(0xFFFFFFFFu, rbv, t & 31);
                    if (t >= nrow) ln[u] = 0;
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
                    if ((uint32_t)sl < L) {
                        const int c = cc[u];
                        const float v = VALS ? wt[VALS ? u : 0] * vv[u] : (neg ? -vv[u] : vv[u]);
                        if ((unsigned)c < (unsigned)a.d)
                            myacc[c] += v;
                        else
                            flag_error(a.status, kDevBadColumn);
                    }
                    for (uint32_t t = sl + LPR; t < L; t += LPR) {  // rows longer than LPR
                        const int c = __ldg(a.col + st[u] + t);
                        const float v = __ldg(a.val + st[u] + t);
                        if ((unsigned)c < (unsigned)a.d)
                            myacc[c] += VALS ? wt[VALS ? u : 0] * v : (neg ? -v : v);
                        else
                            flag_error(a.status, kDevBadColumn);
                    }
                    __syncwarp();
                }
            }
        }
        if (!a.acc_global) {
            if (a.vec4) {
                for (int c = lane * 4; c < a.d; c += 128) {
                    float4 v = make_float4(accw[c], accw[c + 1], accw[c + 2], accw[c + 3]);
#pragma unroll
                    for (int cp = 1; cp < COPIES; ++cp) {
                        const float* o = accw + cp * a.dpad + c;
                        v.x += o[0]; v.y += o[1]; v.z += o[2]; v.w += o[3];
                    }
                    if (a.scale != 1.f) v = make_float4(v.x * a.scale, v.y * a.scale, v.z * a.scale, v.w * a.scale);
                    *reinterpret_cast<float4*>(SArow + c) = v;
                }
            } else {
                for (int c = lane; c < a.d; c += 32) {
                    float v = accw[c];
#pragma unroll
                    for (int cp = 1; cp < COPIES; ++cp) v += accw[cp * a.dpad + c];
                    SArow[c] = v * a.scale;
                }
            }
        } else if (a.scale != 1.f) {
            __syncwarp();
            for (int c = lane; c < a.d; c += 32) SArow[c] *= a.scale;
        }
        if (HAS_B && a.Sb && lane == 0) a.Sb[orow] = sbacc * a.scale;
        __syncwarp();
    }
}

template <int LPR, int U, bool HAS_B>
__global__ void __launch_bounds__(256) k_apply_csr(CsrApplyArgs a) {
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

// ---------------------------------------------------------------- batched sketch (many problems)
//
// The same stages over a table of problems: each block finds its problem from
// a block -> problem table (tiles, scan chunks, coarse bins) and runs the
// single-problem body on that problem's slice of the shared scratch arrays;
// the apply kernel's warps take buckets from one queue over all problems.

__global__ void __launch_bounds__(256) kb_tile_hist(BatchSketch B) {
    __shared__ uint32_t h[kMaxBins];
    const BatchProb& P = B.probs[B.tile_prob[blockIdx.x]];
    const int64_t lt = (int64_t)blockIdx.x - P.tile0;
    tile_hist_body<false>(P.hp, 0, P.n, P.gshift, P.nbins, lt, B.H + P.H0 + lt * P.nbins, h);
}

__global__ void kb_scan_chunk_sums(BatchSketch B) {
    const BatchProb& P = B.probs[B.chunk_prob[blockIdx.y]];
    scan_chunk_sums_body(B.H + P.H0, P.ntiles, P.nbins, B.P + P.P0, blockIdx.x * blockDim.x + threadIdx.x,
                         (int)blockIdx.y - P.chunk0);
}

__global__ void __launch_bounds__(1024) kb_scan_bins(BatchSketch B) {
    __shared__ uint32_t tot[kMaxBins];
    __shared__ uint32_t wsum[32];
    const BatchProb& P = B.probs[blockIdx.x];
    scan_bins_body(B.P + P.P0, P.nchunks, P.nbins, B.CP + P.CP0, (uint32_t)P.n, tot, wsum);
}

__global__ void kb_scan_tiles(BatchSketch B) {
    const BatchProb& P = B.probs[B.chunk_prob[blockIdx.y]];
    scan_tiles_body(B.H + P.H0, B.P + P.P0, P.ntiles, P.nbins, blockIdx.x * blockDim.x + threadIdx.x,
                    (int)blockIdx.y - P.chunk0);
}

__global__ void __launch_bounds__(256) kb_coarse_scatter(BatchSketch B) {
    extern __shared__ uint32_t sm3[];
    const BatchProb& P = B.probs[B.tile_prob[blockIdx.x]];
    const int64_t lt = (int64_t)blockIdx.x - P.tile0;
    coarse_scatter_body<kModeCSR, true, false>(P.hp, 0, P.n, P.gshift, P.nbins, lt, B.H + P.H0 + lt * P.nbins,
                                               P.row_ptr, P.b, B.rec + P.rec0, B.status, sm3);
}

// bins of up to this many rows are staged in shared memory (32 KB: several
// CTAs per SM, the batch's bins hold ~2048 rows)
constexpr int kBatchFineCap = 2048;

__global__ void __launch_bounds__(512) kb_fine_sort(BatchSketch B, int cap) {
    extern __shared__ int4 srec[];
    __shared__ FineSortSmem fs;
    const BatchProb& P = B.probs[B.bin_prob[blockIdx.x]];
    fine_sort_body<kModeCSR, true>(B.rec + P.rec0, B.CP + P.CP0, P.m, P.gshift, cap, B.r2 + P.rec0, B.rb + P.rec0,
                                   B.bptr + P.bp0, (int)blockIdx.x - P.bin0, srec, fs);
}

__global__ void kb_set_last(BatchSketch B) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < B.count) B.bptr[B.probs[p].bp0 + B.probs[p].m] = (int32_t)B.probs[p].n;
}

constexpr int kBatchApplyChunk = 16;  // buckets per queue grab (<= 32)

// Warps take kBatchApplyChunk consecutive global buckets at a time; lanes
// 0..15 look up their bucket's problem and start / end in parallel, so empty
// buckets (skipped when nobody reads their zero row) cost no dependent loads.
template <int LPR, int U>
__global__ void __launch_bounds__(256) kb_apply_csr(BatchSketch B) {
    constexpr int COPIES = 32 / LPR;
    extern __shared__ __align__(16) float smacc[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int sub = lane / LPR, sl = lane % LPR;
    float* accw = B.acc_global ? nullptr : smacc + (size_t)warp * COPIES * B.dpad;
    int cur = -1;
    CsrApplyArgs a{};
    for (;;) {
        unsigned g0 = 0;
        if (lane == 0) g0 = atomicAdd(B.counter, (unsigned)kBatchApplyChunk);
        g0 = __shfl_sync(0xFFFFFFFFu, g0, 0);
        if ((int64_t)g0 >= B.total_buckets) break;
        // lane i: bucket g0 + i -> (problem, local bucket, non-empty)
        int pi = -1, bki = 0, busy = 0;
        const int64_t gi = (int64_t)g0 + lane;
        if (lane < kBatchApplyChunk && gi < B.total_buckets) {
            int l = 0, r = B.count - 1;  // last p with bk_base[p] <= gi
            while (l < r) {
                const int mid = (l + r + 1) >> 1;
                if (B.bk_base[mid] <= gi) l = mid; else r = mid - 1;
            }
            pi = l;
            bki = (int)(gi - B.bk_base[l]);
            const BatchProb& P = B.probs[l];
            const int32_t* bp = B.bptr + P.bp0;
            busy = (!P.skip_empty || bp[bki] < bp[bki + 1]) ? 1 : 0;
        }
        unsigned todo = __ballot_sync(0xFFFFFFFFu, busy != 0);
        while (todo) {
            const int i = __ffs(todo) - 1;
            todo &= todo - 1;
            const int p = __shfl_sync(0xFFFFFFFFu, pi, i);
            const int bk = __shfl_sync(0xFFFFFFFFu, bki, i);
            if (p != cur) {
                const BatchProb& P = B.probs[p];
                cur = p;
                a.rs = B.r2 + P.rec0;
                a.rb = B.rb + P.rec0;
                a.bucket_ptr = B.bptr + P.bp0;
                a.col = P.col;
                a.val = P.val;
                a.SA = P.SA;
                a.Sb = P.Sb;
                a.status = B.status;
                a.m = P.m;
                a.d = P.d;
                a.dpad = B.acc_global ? B.dpad : (int)((P.d + 31) & ~31) + 4;  // this problem's width (<= B.dpad)
                a.acc_global = B.acc_global;
                a.vec4 = P.vec4;
                a.map_v = 0;
                a.scale = 1.f;
            }
            apply_csr_bucket<LPR, U, true>(a, (unsigned)bk, accw, lane, sub, sl);
        }
    }
}

// Range variant for batches of sparse buckets: a warp takes the buckets
// bk0 .. bk0 + nb - 1 of one problem (nb <= kBatchApplyChunk) and walks all
// their records together, a full warp per row and U = 8 rows' gathers in
// flight whatever the bucket boundaries, each row adding into its bucket's
// own shared-memory row (nb x dpad floats per warp).  Rows are added in
// ascending record order within each bucket, as in apply_csr_bucket with one
// accumulator copy; Sb entries are summed per bucket in record order.
__device__ __forceinline__ void apply_csr_range(const CsrApplyArgs& a, int bk0, int nb, int skip, float* acc,
                                                int lane) {
    constexpr int U = 8;
    // lane j < nb: start of bucket bk0 + j; lane nb: the end of the range
    const int bs = (lane <= nb) ? a.bucket_ptr[bk0 + lane] : 0;
    const int s = __shfl_sync(0xFFFFFFFFu, bs, 0), e = __shfl_sync(0xFFFFFFFFu, bs, nb);
    const int dp = a.dpad;
    for (int c = lane * 4; c < nb * dp; c += 128) *reinterpret_cast<float4*>(acc + c) = make_float4(0.f, 0.f, 0.f, 0.f);
    __syncwarp();
    for (int k0 = s; k0 < e; k0 += 32) {
        const int k = k0 + lane;
        int2 rr = make_int2(0, 0);
        int bid = 0;
        if (k < e) {
            rr = __ldg(&a.rs[k]);
            // bucket of record k: the last j with start_j <= k
#pragma unroll
            for (int j = 1; j < kBatchApplyChunk; ++j) {
                const int sj = __shfl_sync(0xFFFFFFFFu, bs, j);
                if (j < nb && sj <= k) bid = j;
            }
        } else {
#pragma unroll
            for (int j = 1; j < kBatchApplyChunk; ++j) (void)__shfl_sync(0xFFFFFFFFu, bs, j);
        }
        const int nrow = min(32, e - k0);
        for (int t0 = 0; t0 < nrow; t0 += U) {
            int st[U], bq[U];
            uint32_t ln[U];
            int cc[U];
            float vv[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int t = (t0 + u) & 31;
                st[u] = __shfl_sync(0xFFFFFFFFu, rr.x, t);
                ln[u] = (uint32_t)__shfl_sync(0xFFFFFFFFu, rr.y, t);
                bq[u] = __shfl_sync(0xFFFFFFFFu, bid, t);
                if (t0 + u >= nrow) ln[u] = 0;
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                cc[u] = 0;
                vv[u] = 0.f;
                if ((uint32_t)lane < (ln[u] & 0x7FFFFFFFu)) {
                    cc[u] = __ldg(a.col + st[u] + lane);
                    vv[u] = __ldg(a.val + st[u] + lane);
                }
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const uint32_t L = ln[u] & 0x7FFFFFFFu;
                const bool neg = (ln[u] >> 31) != 0;
                float* row = acc + bq[u] * dp;
                if ((uint32_t)lane < L) {
                    const int c = cc[u];
                    if ((unsigned)c < (unsigned)a.d) row[c] += neg ? -vv[u] : vv[u];
                    else flag_error(a.status, kDevBadColumn);
                }
                for (uint32_t t = lane + 32; t < L; t += 32) {  // rows longer than 32
                    const int c = __ldg(a.col + st[u] + t);
                    const float v = __ldg(a.val + st[u] + t);
                    if ((unsigned)c < (unsigned)a.d) row[c] += neg ? -v : v;
                    else flag_error(a.status, kDevBadColumn);
                }
                __syncwarp();
            }
        }
    }
    // Sb: lane j < nb sums bucket j's sigma * b in record order
    const int nxt = __shfl_sync(0xFFFFFFFFu, bs, (lane + 1) & 31);
    float sb = 0.f;
    if (lane < nb && a.Sb)
        for (int k = bs; k < nxt; ++k) sb += __ldg(&a.rb[k]);
    for (int j = 0; j < nb; ++j) {
        const int sj = __shfl_sync(0xFFFFFFFFu, bs, j), ej = __shfl_sync(0xFFFFFFFFu, bs, j + 1);
        if (skip && sj == ej) continue;
        float* SArow = a.SA + (size_t)(bk0 + j) * a.d;
        const float* row = acc + j * dp;
        if (a.vec4) {
            for (int c = lane * 4; c < a.d; c += 128) *reinterpret_cast<float4*>(SArow + c) = *reinterpret_cast<const float4*>(row + c);
        } else {
            for (int c = lane; c < a.d; c += 32) SArow[c] = row[c];
        }
        if (a.Sb && lane == j) a.Sb[bk0 + j] = sb;
    }
    __syncwarp();
}

// Batched segmented sum over ranges of up to kBatchApplyChunk buckets (one
// problem each; a grab that crosses a problem boundary is split).
__global__ void __launch_bounds__(256) kb_apply_csr_range(BatchSketch B) {
    extern __shared__ __align__(16) float smacc[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float* acc = smacc + (size_t)warp * kBatchApplyChunk * B.dpad;
    CsrApplyArgs a{};
    for (;;) {
        unsigned g0 = 0;
        if (lane == 0) g0 = atomicAdd(B.counter, (unsigned)kBatchApplyChunk);
        g0 = __shfl_sync(0xFFFFFFFFu, g0, 0);
        if ((int64_t)g0 >= B.total_buckets) break;
        const int64_t g1 = min((int64_t)g0 + kBatchApplyChunk, B.total_buckets);
        for (int64_t gs = g0; gs < g1;) {
            int l = 0, r = B.count - 1;  // last p with bk_base[p] <= gs
            while (l < r) {
                const int mid = (l + r + 1) >> 1;
                if (B.bk_base[mid] <= gs) l = mid; else r = mid - 1;
            }
            const BatchProb& P = B.probs[l];
            const int64_t pe = min(g1, B.bk_base[l + 1]);
            a.rs = B.r2 + P.rec0;
            a.rb = B.rb + P.rec0;
            a.bucket_ptr = B.bptr + P.bp0;
            a.col = P.col;
            a.val = P.val;
            a.SA = P.SA;
            a.Sb = P.Sb;
            a.status = B.status;
            a.m = P.m;
            a.d = P.d;
            a.dpad = (int)((P.d + 31) & ~31) + 4;
            a.vec4 = P.vec4;
            apply_csr_range(a, (int)(gs - B.bk_base[l]), (int)(pe - gs), P.skip_empty, acc, lane);
            gs = pe;
        }
    }
}

// ---------------------------------------------------------------- host driver

struct SketchPlan {
    int gshift, nbins, ntiles, nchunks;
    int lpr;        // CSR: lanes per row (16: two rows per warp step)
    int dpad;       // CSR accumulator row stride (floats)
    int acc_global; // CSR: accumulate in SA rows (very wide rows)
    size_t acc_smem;
};

namespace {

int ilog2_ceil(uint64_t v) {
    int s = 0;
    while ((1ull << s) < v) ++s;
    return s;
}

}  // namespace

// Coarse bins: about 1024 (long runs of each bin per 8192-row tile keep the
// coarse scatter's writes coalesced), more for large n so that a bin fits the
// fine sort's shared-memory stage, at most kMaxBins, at most kMaxGroupBuckets
// buckets per bin.
int plan_sketch(int mode, int64_t n, int64_t d, int64_t m, SketchPlan* p) {
    const int gmin = ilog2_ceil(((uint64_t)m + kMaxBins - 1) / kMaxBins);
    const int gmax = ilog2_ceil((uint64_t)kMaxGroupBuckets);
    if (gmin > gmax) return CW_ERR_SHAPE;
    // about 1024 bins, more (up to kMaxBins) so that a bin averages at most 8192
    // rows: k_fine_sort then stages whole bins in shared memory
    uint64_t want_bins = 1024;
    while (want_bins < (uint64_t)kMaxBins && want_bins * 8192 < (uint64_t)n) want_bins *= 2;
    int gs = ilog2_ceil(((uint64_t)m + want_bins - 1) / want_bins);
    gs = std::max(gs, gmin);
    gs = std::min(gs, gmax);
    gs = std::min(gs, ilog2_ceil((uint64_t)m));
    p->gshift = gs;
    p->nbins = (int)(((uint64_t)m + (1ull << gs) - 1) >> gs);
    p->ntiles = (int)((n + kTileRows - 1) / kTileRows);
    p->nchunks = (p->ntiles + kScanChunk - 1) / kScanChunk;
    p->lpr = 16;
    p->dpad = 0;
    p->acc_global = 0;
    p->acc_smem = 0;
    if (mode == kModeCSR) {
        p->dpad = (int)((d + 31) & ~31ll) + 4;  // copies start on different banks, rows stay 16-byte aligned
        p->acc_smem = (size_t)8 * 2 * p->dpad * sizeof(float);
        if (p->acc_smem > 96 * 1024) {
            p->lpr = 32;
            p->acc_smem = (size_t)8 * p->dpad * sizeof(float);
            if (p->acc_smem > 96 * 1024) {
                p->acc_global = 1;
                p->acc_smem = 0;
            }
        }
    }
    return CW_OK;
}

template <class F>
static cudaError_t set_smem(F* f, size_t bytes) {
    return cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <class F>
static int persistent_grid(F* f, int threads, size_t smem) {
    int per = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, f, threads, smem) != cudaSuccess || per < 1) {
        (void)cudaGetLastError();
        per = 1;
    }
    return per * num_sms();
}

// mode: kModeCSR (row_ptr/col/val), kModeDense (A, lda), kModeVec (x in b).
// bucket_ptr_out: optional device array of m + 1 ints (bucket starts of the
// stable permutation); NULL uses internal scratch.  SA64 (dense only): write a
// float64 SA from two-word sums instead of the float32 SA.
int sketch_impl(int mode, int64_t n, int64_t d, int64_t lda, int64_t i0, const int32_t* row_ptr,
                const int32_t* col, const float* val, const float* A, const float* b, int64_t m,
                uint64_t seed, float* SA, float* Sb, int32_t* bucket_ptr_out, cudaStream_t stream,
                double* SA64, const SketchWorkspace* ext, const SketchLayout* lay, const float* vals) {
    // with vals, the CSR pass forms SA only (its rb carries v_i); Sb comes
    // from a separate vector pass of the caller
    const bool has_b = b != nullptr && (mode == kModeVec || Sb != nullptr) && !(vals && mode == kModeCSR);
    if (lay && mode != kModeCSR) return CW_ERR_ARG;
    if (vals && (lay || SA64)) return CW_ERR_ARG;
    if (n == 0 && lay) return CW_OK;   // the caller zeroed the whole output
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
                       lay ? lay->scale : 1.f};
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

int batch_sketch_set_lpr(BatchSketch* dev, int lpr) {
    if (lpr != 16 && lpr != 32 && lpr != 0) return CW_ERR_ARG;
    if (lpr == 0 && dev->acc_global) return CW_ERR_ARG;
    dev->lpr = lpr;
    if (lpr == 0) {
        dev->acc_smem = (size_t)8 * kBatchApplyChunk * dev->dpad * sizeof(float);
        if (set_smem(kb_apply_csr_range, dev->acc_smem) != cudaSuccess) return CW_ERR_CUDA;
        dev->apply_grid = persistent_grid(kb_apply_csr_range, 256, dev->acc_smem);
        return CW_OK;
    }
    dev->acc_smem = dev->acc_global ? 0 : (size_t)8 * (32 / lpr) * dev->dpad * sizeof(float);
    auto kf = lpr == 16 ? kb_apply_csr<16, 8> : kb_apply_csr<32, 8>;
    if (set_smem(kf, dev->acc_smem) != cudaSuccess) return CW_ERR_CUDA;
    dev->apply_grid = persistent_grid(kf, 256, dev->acc_smem);
    return CW_OK;
}

int batch_sketch_plan(const BatchSpec* specs, int count, BatchSketchHost* host, BatchSketch* dev) {
    host->probs.assign((size_t)count, BatchProb{});
    host->tile_prob.clear();
    host->chunk_prob.clear();
    host->bin_prob.clear();
    host->bk_base.assign((size_t)count + 1, 0);
    host->H_elems = host->P_elems = host->CP_elems = host->rows = host->bptr_elems = 0;
    int32_t tiles = 0, chunks = 0, bins = 0, max_nbins = 1;
    int lpr = 16, dpad = 0, acc_global = 0;
    for (int p = 0; p < count; ++p) {
        const BatchSpec& s = specs[p];
        SketchPlan sp;
        int st = plan_sketch(kModeCSR, s.n, s.d, s.m, &sp);
        if (st != CW_OK) return st;
        // coarse bins of about 2048 rows (at most 256 buckets each): a small
        // problem gets a few bins, not the ~1024 a single large sketch uses
        {
            const uint64_t want = std::max<uint64_t>(1, ((uint64_t)s.n + 2047) / 2048);
            int gs = ilog2_ceil(((uint64_t)s.m + want - 1) / want);
            gs = std::max(gs, ilog2_ceil(((uint64_t)s.m + kMaxBins - 1) / kMaxBins));
            gs = std::min(gs, ilog2_ceil((uint64_t)kMaxGroupBuckets));
            gs = std::min(gs, ilog2_ceil((uint64_t)s.m));
            sp.gshift = gs;
            sp.nbins = (int)(((uint64_t)s.m + (1ull << gs) - 1) >> gs);
        }
        BatchProb& P = host->probs[(size_t)p];
        P.hp = make_hash_params(s.seed, s.m);
        P.n = s.n;
        P.d = (int32_t)s.d;
        P.m = (int32_t)s.m;
        P.gshift = sp.gshift;
        P.nbins = sp.nbins;
        P.ntiles = sp.ntiles;
        P.nchunks = sp.nchunks;
        P.tile0 = tiles;
        P.chunk0 = chunks;
        P.bin0 = bins;
        P.vec4 = (s.d % 4 == 0) && ((reinterpret_cast<uintptr_t>(s.SA) & 15) == 0) ? 1 : 0;
        P.H0 = host->H_elems;
        P.P0 = host->P_elems;
        P.CP0 = host->CP_elems;
        P.rec0 = host->rows;
        P.bp0 = host->bptr_elems;
        P.bk0 = host->bk_base[(size_t)p];
        P.row_ptr = s.row_ptr;
        P.col = s.col;
        P.val = s.val;
        P.b = s.b;
        P.SA = s.SA;
        P.Sb = s.Sb;
        for (int t = 0; t < sp.ntiles; ++t) host->tile_prob.push_back(p);
        for (int c = 0; c < sp.nchunks; ++c) host->chunk_prob.push_back(p);
        for (int g = 0; g < sp.nbins; ++g) host->bin_prob.push_back(p);
        tiles += sp.ntiles;
        chunks += sp.nchunks;
        bins += sp.nbins;
        max_nbins = std::max(max_nbins, sp.nbins);
        host->H_elems += (int64_t)sp.ntiles * sp.nbins;
        host->P_elems += (int64_t)sp.nchunks * sp.nbins;
        host->CP_elems += sp.nbins + 1;
        host->rows += s.n;
        host->bptr_elems += s.m + 1;
        host->bk_base[(size_t)p + 1] = host->bk_base[(size_t)p] + s.m;
        lpr = std::max(lpr, sp.lpr);
        dpad = std::max(dpad, sp.dpad);
        acc_global = std::max(acc_global, sp.acc_global);
    }
    dev->count = count;
    dev->total_tiles = tiles;
    dev->total_chunks = chunks;
    dev->total_bins = bins;
    dev->max_nbins = max_nbins;
    dev->bin_groups = (max_nbins + 255) / 256;
    dev->total_buckets = host->bk_base[(size_t)count];
    dev->dpad = dpad;
    dev->acc_global = acc_global;
    int st = batch_sketch_set_lpr(dev, lpr);
    if (st != CW_OK) return st;
    const size_t k3smem = sizeof(uint32_t) * (size_t)kTileWarps * (max_nbins + kTileRowsPerWarp);
    if (set_smem(kb_coarse_scatter, k3smem) != cudaSuccess) return CW_ERR_CUDA;
    if (set_smem(kb_fine_sort, sizeof(int4) * (size_t)kBatchFineCap) != cudaSuccess) return CW_ERR_CUDA;
    return CW_OK;
}

int batch_sketch_enqueue(const BatchSketch& B, cudaStream_t stream) {
    CW_CUDA_TRY(cudaMemsetAsync(B.counter, 0, sizeof(unsigned), stream));
    if (B.total_tiles > 0) {
        {
            CW_PROF("kb_tile_hist", stream);
            kb_tile_hist<<<B.total_tiles, 256, 0, stream>>>(B);
        }
        dim3 sg(B.bin_groups, B.total_chunks);
        {
            CW_PROF("kb_scan_chunk_sums", stream);
            kb_scan_chunk_sums<<<sg, 256, 0, stream>>>(B);
        }
        {
            CW_PROF("kb_scan_bins", stream);
            kb_scan_bins<<<B.count, 1024, 0, stream>>>(B);
        }
        {
            CW_PROF("kb_scan_tiles", stream);
            kb_scan_tiles<<<sg, 256, 0, stream>>>(B);
        }
        const size_t k3smem = sizeof(uint32_t) * (size_t)kTileWarps * (B.max_nbins + kTileRowsPerWarp);
        {
            CW_PROF("kb_coarse_scatter", stream);
            kb_coarse_scatter<<<B.total_tiles, 256, k3smem, stream>>>(B);
        }
    } else {
        // no rows anywhere: every coarse bin is empty
        CW_CUDA_TRY(cudaMemsetAsync(B.CP, 0, sizeof(uint32_t) * (size_t)(B.total_bins + B.count), stream));
    }
    CW_LAUNCH_CHECK();
    {
        CW_PROF("kb_fine_sort", stream);
        kb_fine_sort<<<B.total_bins, 512, sizeof(int4) * (size_t)kBatchFineCap, stream>>>(B, kBatchFineCap);
    }
    {
        CW_PROF("kb_set_last", stream);
        kb_set_last<<<(B.count + 255) / 256, 256, 0, stream>>>(B);
    }
    CW_LAUNCH_CHECK();
    {
        CW_PROF("kb_apply_csr", stream);
        if (B.lpr == 16)
            kb_apply_csr<16, 8><<<B.apply_grid, 256, B.acc_smem, stream>>>(B);
        else if (B.lpr == 32)
            kb_apply_csr<32, 8><<<B.apply_grid, 256, B.acc_smem, stream>>>(B);
        else
            kb_apply_csr_range<<<B.apply_grid, 256, B.acc_smem, stream>>>(B);
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
