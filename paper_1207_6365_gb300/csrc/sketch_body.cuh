// Device bodies and host planning shared by the single-problem sketch
// (sketch.cu) and the batched sketch (batch_sketch.cu): the counting sort by
// bucket (tile histograms, scans, coarse scatter, fine sort) and the CSR
// segmented sum of one bucket, each as a device function a kernel wraps.
#pragma once

#include <algorithm>

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

// ---------------------------------------------------------------- K3: coarse stable scatter

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned r;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(r));
    return r;
}

// Per row one 16-byte record {key, a, len, sigma*b}: a = row start (CSR) or
// the row index (dense); written in coarse-bin order, stable within a bin.
// Tile `tile` of the rows; Orow = the tile's output offsets per bin.  The
// tile's lines of row_ptr and b are prefetched into L2 while its rows are
// hashed, and their loads go out eight rows per lane at a time.
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
    {   // the tile's lines of row_ptr, b (and vals) into L2 while its rows are hashed
        const int64_t t0 = tile * kTileRows;
        const int rows = (n - t0) < (int64_t)kTileRows ? (int)(n - t0) : kTileRows;
        const int lines = (rows + 32) / 32;
        for (int k = threadIdx.x; k < lines; k += blockDim.x) {
            if (MODE == kModeCSR) asm volatile("prefetch.global.L2 [%0];" ::"l"(row_ptr + t0 + 32 * k));
            if (HAS_B && 32 * k < rows) asm volatile("prefetch.global.L2 [%0];" ::"l"(b + t0 + 32 * k));
            if (VALS && 32 * k < rows) asm volatile("prefetch.global.L2 [%0];" ::"l"(vals + t0 + 32 * k));
        }
    }
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
    constexpr int GR = 8;  // rows per lane whose loads are in flight together
#pragma unroll 1
    for (int j0 = 0; j0 < kTileRowsPerLane; j0 += GR) {
        if (r0 - lane + 32 * j0 >= n) break;
        int32_t st[GR], ln[GR];
        float bv[GR], wv[GR];
#pragma unroll
        for (int u = 0; u < GR; ++u) {
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
        for (int u = 0; u < GR; ++u) {
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
    int accumulate;          // add the bucket sums to SA and Sb instead of overwriting them
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
            if (!a.accumulate)
                for (int c = lane; c < a.d; c += 32) SArow[c] = 0.f;
            myacc = SArow;
        } else {
            for (int c = lane; c < COPIES * a.dpad; c += 32) accw[c] = 0.f;
            myacc = accw + sub * a.dpad;
        }
        __syncwarp();
        float sbacc = 0.f;
        // records of up to 32 rows: lane l holds row k0 + l; the next chunk's
        // records are loaded while this chunk's rows are gathered
        int2 rr_next = make_int2(0, 0);
        float rbv_next = 0.f;
        if (s + lane < e) {
            rr_next = __ldg(&a.rs[s + lane]);
            if (HAS_B || VALS) rbv_next = __ldg(&a.rb[s + lane]);
        }
        for (int k0 = s; k0 < e; k0 += 32) {
            const int2 rr = rr_next;
            const float rbv = rbv_next;
            rr_next = make_int2(0, 0);
            rbv_next = 0.f;
            if (k0 + 32 + lane < e) {
                rr_next = __ldg(&a.rs[k0 + 32 + lane]);
                if (HAS_B || VALS) rbv_next = __ldg(&a.rb[k0 + 32 + lane]);
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
                    const uint32_t L = ln[u] & 0x7FFFFFFFu;
                    if ((uint32_t)sl < L) {
                        // a row inside one 64-byte block of col and of val: fetch just
                        // that block; other rows keep the default L2 fetch (for
                        // unaligned or longer rows the 64-byte limit splits what one
                        // 128-byte fetch would bring: measured slower)
                        if ((uint32_t)(st[u] & 15) + L <= 16u) {
                            cc[u] = ld_gather(a.col + st[u] + sl);
                            vv[u] = ld_gather(a.val + st[u] + sl);
                        } else {
                            cc[u] = __ldg(a.col + st[u] + sl);
                            vv[u] = __ldg(a.val + st[u] + sl);
                        }
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
                    if (a.accumulate) {
                        const float4 o = *reinterpret_cast<const float4*>(SArow + c);
                        v = make_float4(o.x + v.x, o.y + v.y, o.z + v.z, o.w + v.w);
                    }
                    *reinterpret_cast<float4*>(SArow + c) = v;
                }
            } else {
                for (int c = lane; c < a.d; c += 32) {
                    float v = accw[c];
#pragma unroll
                    for (int cp = 1; cp < COPIES; ++cp) v += accw[cp * a.dpad + c];
                    SArow[c] = a.accumulate ? SArow[c] + v * a.scale : v * a.scale;
                }
            }
        } else if (a.scale != 1.f) {
            __syncwarp();
            for (int c = lane; c < a.d; c += 32) SArow[c] *= a.scale;
        }
        if (HAS_B && a.Sb && lane == 0) a.Sb[orow] = a.accumulate ? a.Sb[orow] + sbacc * a.scale : sbacc * a.scale;
        __syncwarp();
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

inline int ilog2_ceil(uint64_t v) {
    int s = 0;
    while ((1ull << s) < v) ++s;
    return s;
}

// Coarse bins: about 1024 (long runs of each bin per 8192-row tile keep the
// coarse scatter's writes coalesced), more for large n so that a bin fits the
// fine sort's shared-memory stage, at most kMaxBins, at most kMaxGroupBuckets
// buckets per bin.
inline int plan_sketch(int mode, int64_t n, int64_t d, int64_t m, SketchPlan* p) {
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
inline cudaError_t set_smem(F* f, size_t bytes) {
    return cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <class F>
inline int persistent_grid(F* f, int threads, size_t smem) {
    int per = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, f, threads, smem) != cudaSuccess || per < 1) {
        (void)cudaGetLastError();
        per = 1;
    }
    return per * num_sms();
}


}  // namespace cw
