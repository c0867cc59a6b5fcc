// The batched sketch: the stages of the single-problem sketch launched once
// over a table of problems (see batch.h).  Each block finds its problem from a
// block -> problem table and runs the shared stage body on that problem's
// slice of the scratch arrays.
#include <vector>

#include "batch.h"
#include "sketch_body.cuh"

namespace cw {

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
template <int NB>
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
            for (int j = 1; j < NB; ++j) {
                const int sj = __shfl_sync(0xFFFFFFFFu, bs, j);
                if (j < nb && sj <= k) bid = j;
            }
        } else {
#pragma unroll
            for (int j = 1; j < NB; ++j) (void)__shfl_sync(0xFFFFFFFFu, bs, j);
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

// Batched segmented sum over ranges of up to NB buckets (one problem each; a
// grab that crosses a problem boundary is split).  NB = 8 halves the shared
// accumulator rows per warp and is built for four CTAs per SM.
template <int NB>
__global__ void __launch_bounds__(256, NB == 8 ? 4 : 3) kb_apply_csr_range(BatchSketch B) {
    extern __shared__ __align__(16) float smacc[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float* acc = smacc + (size_t)warp * NB * B.dpad;
    CsrApplyArgs a{};
    for (;;) {
        unsigned g0 = 0;
        if (lane == 0) g0 = atomicAdd(B.counter, (unsigned)NB);
        g0 = __shfl_sync(0xFFFFFFFFu, g0, 0);
        if ((int64_t)g0 >= B.total_buckets) break;
        const int64_t g1 = min((int64_t)g0 + NB, B.total_buckets);
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
            apply_csr_range<NB>(a, (int)(gs - B.bk_base[l]), (int)(pe - gs), P.skip_empty, acc, lane);
            gs = pe;
        }
    }
}


int batch_sketch_set_lpr(BatchSketch* dev, int lpr) {
    if (lpr != 16 && lpr != 32 && lpr != 0 && lpr != -8) return CW_ERR_ARG;
    if (lpr <= 0 && dev->acc_global) return CW_ERR_ARG;
    dev->lpr = lpr;
    if (lpr <= 0) {
        const int nb = lpr == 0 ? 16 : 8;
        dev->acc_smem = (size_t)8 * nb * dev->dpad * sizeof(float);
        auto kf = lpr == 0 ? kb_apply_csr_range<16> : kb_apply_csr_range<8>;
        if (set_smem(kf, dev->acc_smem) != cudaSuccess) return CW_ERR_CUDA;
        dev->apply_grid = persistent_grid(kf, 256, dev->acc_smem);
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
            if (B.lpr == 0)
                kb_apply_csr_range<16><<<B.apply_grid, 256, B.acc_smem, stream>>>(B);
            else
                kb_apply_csr_range<8><<<B.apply_grid, 256, B.acc_smem, stream>>>(B);
    }
    CW_LAUNCH_CHECK();
    return CW_OK;
}


}  // namespace cw
