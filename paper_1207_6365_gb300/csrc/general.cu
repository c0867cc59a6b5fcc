// The generalized sparse embedding in one pass over A (paper Section
// "Generalized Sparse Embedding Matrices", "The construction"):
// S = blockdiag(B^(1), ..., B^(q)) P, where P groups the rows of A by the outer
// hash h(i) in [0, q) and B^(g) stacks kappa independent v-row sparse
// embeddings scaled by 1 / sqrt(kappa).  Row i of A therefore lands in the
// kappa output rows h(i) * v * kappa + b * v + h_b(i), b = 0..kappa-1, with
// sign sigma_b(i); S A costs O(nnz(A) kappa) arithmetic (Lemma "time") but
// needs A read only once.
//
// The rows are sorted once by h(i) (the counting sort of the plain sketch,
// records carrying the row index).  A CTA then takes an outer block g at a
// time and keeps the block's v * kappa output rows in shared memory.  Warp
// (b, j) of the CTA owns inner sketch b's buckets u with u % W == j: it walks
// the block's rows in ascending order, evaluates h_b(i) and sigma_b(i), and
// adds the rows that fall in its buckets (a half-warp per row, lane l taking
// nonzeros l, l + 16, ...; two rows of one step that fall in the same bucket
// are added one after the other).  Each output row thus receives its rows in
// ascending row order.  The kappa warps of one row read it close together in
// time, so A crosses DRAM about once.
#include <cmath>
#include <vector>

#include "cw_common.cuh"
#include "cw_internal.h"

namespace cw {

struct GeneralApplyArgs {
    const int2* rs;            // outer-block order: {row | sign << 31, 0}
    const float* rb;           // sigma_outer * b (nullable)
    const int32_t* bptr;       // q + 1 block starts
    const int32_t* row_ptr;
    const int32_t* col;
    const float* val;
    const uint64_t* coef;      // [kappa][8]: inner bucket cubic c0..c3, inner sign cubic c0..c3
    float* SA;                 // (q v kappa) x d
    float* Sb;                 // q v kappa (nullable)
    unsigned* counter;         // next outer block
    unsigned* status;
    int64_t q;
    int v, kappa, W, d, dp;    // W warps per inner sketch; dp: shared row stride
    uint64_t vinv;             // floor((2^64 - 1) / v)
    float scale;
};

__device__ __forceinline__ uint32_t mod_v(uint64_t g, uint64_t v, uint64_t vinv) {
    const uint64_t q = __umul64hi(g, vinv);
    uint64_t r = g - q * v;
    if (r >= v) r -= v;
    return (uint32_t)r;
}

template <bool HAS_B>
__global__ void __launch_bounds__(256) k_apply_general(GeneralApplyArgs a) {
    extern __shared__ __align__(16) float gacc[];   // [kappa * v][dp], then Sb [kappa * v]
    __shared__ unsigned next_block;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int half = lane >> 4, sl = lane & 15;
    const int rows_out = a.kappa * a.v;
    const int ib = warp / a.W, jw = warp % a.W;    // inner sketch, bucket residue
    const bool active = ib < a.kappa;
    float* accb = gacc + (size_t)rows_out * a.dp;
    uint64_t cb[4], cs[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        cb[k] = active ? a.coef[ib * 8 + k] : 0;
        cs[k] = active ? a.coef[ib * 8 + 4 + k] : 0;
    }
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) next_block = atomicAdd(a.counter, 1u);
        for (int i = threadIdx.x; i < rows_out * a.dp + rows_out; i += blockDim.x) gacc[i] = 0.f;
        __syncthreads();
        const unsigned g = next_block;
        if ((int64_t)g >= a.q) break;
        const int s = a.bptr[g], e = a.bptr[g + 1];
        if (active) {
            for (int k0 = s; k0 < e; k0 += 32) {
                // lane l: row k0 + l of the block, its bucket and sign in sketch ib
                int row = -1, st = 0, len = 0;
                uint32_t u = 0;
                float w = 0.f, bi = 0.f;
                if (k0 + lane < e) {
                    const int2 r = __ldg(&a.rs[k0 + lane]);
                    row = r.x & 0x7FFFFFFF;
                    const uint64_t x = (uint64_t)row;
                    u = mod_v(horner61(cb, x), (uint64_t)a.v, a.vinv);
                    w = (horner61(cs, x) & 1u) ? -1.f : 1.f;
                    if (HAS_B) {
                        const float rv = __ldg(&a.rb[k0 + lane]);
                        bi = (r.x < 0) ? -rv : rv;
                    }
                }
                const bool mine = row >= 0 && (int)(u % (uint32_t)a.W) == jw;
                const unsigned mk = __ballot_sync(0xFFFFFFFFu, mine);
                const int cnt = __popc(mk);
                if (cnt == 0) continue;
                // compact this warp's rows into lanes 0..cnt-1, in order
                const int src = __fns(mk, 0, lane + 1);
                const int srcl = lane < cnt ? src : 0;
                row = __shfl_sync(0xFFFFFFFFu, row, srcl);
                u = __shfl_sync(0xFFFFFFFFu, u, srcl);
                w = __shfl_sync(0xFFFFFFFFu, w, srcl);
                bi = __shfl_sync(0xFFFFFFFFu, bi, srcl);
                if (lane < cnt) {
                    st = __ldg(a.row_ptr + row);
                    len = __ldg(a.row_ptr + row + 1) - st;
                    if (len < 0) {
                        flag_error(a.status, kDevBadRowPtr);
                        len = 0;
                    }
                }
                constexpr int U = 4;   // two-row steps whose loads are in flight together
                for (int t0 = 0; t0 < cnt; t0 += 2 * U) {
                    int cc[U], ln[U], us[U];
                    float vv[U];
#pragma unroll
                    for (int q2 = 0; q2 < U; ++q2) {
                        const int e2 = t0 + 2 * q2 + half;
                        // every lane takes part in every shuffle (the two halves'
                        // rows may differ in validity)
                        const int sq = __shfl_sync(0xFFFFFFFFu, st, e2 & 31);
                        const int lq = __shfl_sync(0xFFFFFFFFu, len, e2 & 31);
                        ln[q2] = e2 < cnt ? lq : 0;
                        us[q2] = __shfl_sync(0xFFFFFFFFu, (int)u, e2 & 31);
                        cc[q2] = 0;
                        vv[q2] = 0.f;
                        if (sl < ln[q2]) {
                            cc[q2] = __ldg(a.col + sq + sl);
                            vv[q2] = __ldg(a.val + sq + sl);
                        }
                        ln[q2] = e2 < cnt ? ln[q2] : -1;
                    }
#pragma unroll
                    for (int q2 = 0; q2 < U; ++q2) {
                        const int e0 = t0 + 2 * q2;
                        if (e0 >= cnt) break;
                        const int e2 = e0 + half;
                        const int u0 = __shfl_sync(0xFFFFFFFFu, (int)u, e0 & 31);
                        const int u1 = __shfl_sync(0xFFFFFFFFu, (int)u, (e0 + 1) & 31);
                        const float wr = __shfl_sync(0xFFFFFFFFu, w, e2 & 31);
                        const float br = __shfl_sync(0xFFFFFFFFu, bi, e2 & 31);
                        const int sr = __shfl_sync(0xFFFFFFFFu, st, e2 & 31);
                        const bool valid = e2 < cnt;
                        float* arow = gacc + (size_t)(ib * a.v + us[q2]) * a.dp;
                        const bool serial = (e0 + 1 < cnt) && u0 == u1;
                        for (int pass = 0; pass < (serial ? 2 : 1); ++pass) {
                            if (valid && (!serial || pass == half)) {
                                if (sl < ln[q2]) {
                                    if ((unsigned)cc[q2] < (unsigned)a.d) arow[cc[q2]] += wr * vv[q2];
                                    else flag_error(a.status, kDevBadColumn);
                                }
                                for (int t = sl + 16; t < ln[q2]; t += 16) {  // rows longer than 16
                                    const int c = __ldg(a.col + sr + t);
                                    if ((unsigned)c < (unsigned)a.d) arow[c] += wr * __ldg(a.val + sr + t);
                                    else flag_error(a.status, kDevBadColumn);
                                }
                                if (HAS_B && sl == 0) accb[ib * a.v + us[q2]] += wr * br;
                            }
                            __syncwarp();
                        }
                    }
                }
            }
        }
        __syncthreads();
        // the block's kappa * v output rows: row g v kappa + b v + u
        const int64_t o0 = (int64_t)g * rows_out;
        const int nw = blockDim.x >> 5;
        for (int r = warp; r < rows_out; r += nw) {
            const float* src = gacc + (size_t)r * a.dp;
            float* dst = a.SA + (size_t)(o0 + r) * a.d;
            for (int c = lane; c < a.d; c += 32) dst[c] = src[c] * a.scale;
            if (HAS_B && a.Sb && lane == 0) a.Sb[o0 + r] = accb[r] * a.scale;
        }
    }
}

// One pass of the generalized embedding when it fits (kappa warps of at most
// 8 per CTA, the block's v kappa rows in shared memory); *done = false leaves
// the caller to the kappa-pass path.
int sketch_csr_general_onepass(const cw_csr* A, const float* b, int64_t q, int64_t v, int32_t kappa, uint64_t seed,
                               float* SA, float* Sb, cudaStream_t stream, bool* done) {
    *done = false;
    const int64_t n = A->n, d = A->d;
    if (kappa < 2 || kappa > 8 || n < 1) return CW_OK;
    const int W = 8 / kappa;
    const int dp = (int)(d % 2 == 0 ? d + 1 : d);  // odd: the rows start on different banks
    const int64_t rows_out = (int64_t)kappa * v;
    const size_t smem = sizeof(float) * (size_t)(rows_out * dp + rows_out);
    if (smem > 200 * 1024) return CW_OK;
    unsigned* status = device_status_word();
    if (!status) return CW_ERR_CUDA;
    const bool has_b = b && Sb;

    Scratch ws(stream);
    const size_t oR2 = ws.reserve(sizeof(int2) * (size_t)n);
    const size_t oRb = has_b ? ws.reserve(sizeof(float) * (size_t)n) : 0;
    const size_t oBp = ws.reserve(sizeof(int32_t) * (size_t)(q + 1));
    const size_t oCo = ws.reserve(sizeof(uint64_t) * 8 * (size_t)kappa);
    const size_t oCt = ws.reserve(sizeof(unsigned));
    CW_CUDA_TRY(ws.alloc());
    int2* r2 = ws.at<int2>(oR2);
    float* rb = has_b ? ws.at<float>(oRb) : nullptr;
    int32_t* bptr = ws.at<int32_t>(oBp);
    uint64_t* coef = ws.at<uint64_t>(oCo);
    unsigned* counter = ws.at<unsigned>(oCt);

    // inner sketch b: the bucket and sign cubics of seed_b (over v buckets)
    std::vector<uint64_t> seeds((size_t)kappa), hc(8 * (size_t)kappa);
    splitmix64_after_coeffs(seed, kappa, seeds.data());
    for (int k = 0; k < kappa; ++k) {
        const HashParams hb = make_hash_params(seeds[(size_t)k], v);
        for (int c = 0; c < 4; ++c) {
            hc[8 * (size_t)k + c] = hb.cb[c];
            hc[8 * (size_t)k + 4 + c] = hb.cs[c];
        }
    }
    CW_CUDA_TRY(cudaMemcpyAsync(coef, hc.data(), sizeof(uint64_t) * hc.size(), cudaMemcpyHostToDevice, stream));
    CW_CUDA_TRY(cudaMemsetAsync(counter, 0, sizeof(unsigned), stream));
    // rows sorted by the outer hash h(i) = the bucket cubic of `seed` over q
    const SortOut so{r2, rb, bptr};
    int st = sketch_impl(kSketchDense, n, 1, 1, 0, nullptr, nullptr, nullptr, nullptr, has_b ? b : nullptr, q, seed,
                         nullptr, nullptr, nullptr, stream, nullptr, nullptr, nullptr, nullptr, false, &so);
    if (st != CW_OK) return st;

    GeneralApplyArgs a{r2, rb, bptr, A->row_ptr, A->col, A->val, coef, SA, has_b ? Sb : nullptr, counter, status,
                       q, (int)v, (int)kappa, W, (int)d, dp, ~0ull / (uint64_t)v,
                       (float)(1.0 / std::sqrt((double)kappa))};
    auto kf = has_b ? k_apply_general<true> : k_apply_general<false>;
    CW_CUDA_TRY(cudaFuncSetAttribute(kf, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int threads = 32 * kappa * W;
    int per = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kf, threads, smem) != cudaSuccess || per < 1) {
        (void)cudaGetLastError();
        per = 1;
    }
    const int64_t grid = std::min<int64_t>((int64_t)per * num_sms(), q);
    {
        CW_PROF("k_apply_general", stream);
        kf<<<(unsigned)grid, threads, smem, stream>>>(a);
    }
    CW_LAUNCH_CHECK();
    *done = true;
    return CW_OK;
}

}  // namespace cw
