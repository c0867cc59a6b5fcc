// The fused LSQR pass: one stream over the rows of A per iteration (the
// LSQR iteration of Section 7.6 needs A M v and A^T u once each):
//     z_i = (A vhat)_i - coef * z_i          (vhat = M v, float32)
//     ||z||^2 and A^T z                      (per-CTA partials, fixed order)
// Kept apart from the rest of the solver so that its measured DRAM traffic
// stays tied to these sources alone.
#pragma once

#include <cstdint>

#include "cw_common.cuh"

namespace cw {

struct LsqrState {
    double alpha, beta, rhobar, phibar, anorm2, bnorm, s, coef, test2, rnorm;
    int iters, done, converged, pad;
};

struct PassArgs {
    const int32_t* row_ptr;
    const int32_t* col;
    const float* val;
    const float* vhat;     // d
    const float* zin;      // n (z of the previous step, or b for the first pass)
    float* zout;           // n
    float2* gpart;         // [grid][d] two-word (hi, lo) partial sums of A^T z
    double* zpart;         // [grid]
    double* bpart;         // [grid] (sum of zin^2; first pass only)
    const LsqrState* st;   // coef, done
    unsigned* status;
    int64_t n;
    int d, dpad;
    float coef_first;      // used when st == nullptr
};

constexpr int kPassBatch = 32;     // rows per warp batch (lane l holds row_ptr / z of row l)

// Streaming 16-byte loads that do not allocate in L1 (each nonzero is read
// once per pass; L1 is left to the shared-memory accumulators).
__device__ __forceinline__ int4 ld_stream_i4(const int32_t* p) {
    int4 r;
    asm volatile("ld.global.nc.L1::no_allocate.v4.s32 {%0, %1, %2, %3}, [%4];\n"
                 : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
                 : "l"(p));
    return r;
}
__device__ __forceinline__ float4 ld_stream_f4(const float* p) {
    float4 r;
    asm volatile("ld.global.nc.L1::no_allocate.v4.f32 {%0, %1, %2, %3}, [%4];\n"
                 : "=f"(r.x), "=f"(r.y), "=f"(r.z), "=f"(r.w)
                 : "l"(p));
    return r;
}

// One CTA per SM, kW warps; warp w owns a contiguous block of rows and walks
// it in batches of 32.  Shared memory holds only vhat and eight accumulator
// copies of A^T z per warp, so many warps fit on the SM; nonzeros go straight
// from global memory to registers.
//
// Quad batches (every row starts on a 4-element boundary and has a multiple
// of 4, at most 16, entries): four lanes per row, four entries per lane,
// eight rows per step; all four steps' 16-byte loads are issued before the
// first is used.  Row slot q of a step accumulates into copy q, so no two
// lanes ever update the same address in one instruction and every address is
// updated in program order: the sums are the same in every run.  A row's
// columns must be distinct (as for the sketch kernels; cw_csr_check tests it):
// a lane reads its four accumulators before writing them.
// Other batches: a half-warp per row (16 lanes, longer rows loop), four rows
// at a time, two accumulator copies.
template <int kW>
__global__ void __launch_bounds__(kW * 32, 1) k_lsqr_pass(PassArgs a) {
    extern __shared__ __align__(16) float sm[];
    if (a.st && a.st->done) return;
    constexpr int LPR = 16, HALVES = 32 / LPR, RPH = kPassBatch / HALVES, COPIES = 8;
    const float coef = a.st ? (float)a.st->coef : a.coef_first;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int sub = lane / LPR, sl = lane % LPR;
    float* vh = sm;                      // [dpad], zero past d
    float* acc = vh + a.dpad;            // [kW][COPIES][dpad]
    const bool vec16 = ((reinterpret_cast<uintptr_t>(a.col) | reinterpret_cast<uintptr_t>(a.val)) & 15) == 0;
    for (int j = threadIdx.x; j < a.dpad; j += blockDim.x) vh[j] = j < a.d ? a.vhat[j] : 0.f;
    for (int q = threadIdx.x; q < kW * COPIES * a.dpad; q += blockDim.x) acc[q] = 0.f;
    __syncthreads();
    float* myacc = acc + (size_t)(warp * COPIES + sub) * a.dpad;
    const int qd = lane >> 2, ql = lane & 3;   // quad batches: row slot, lane in quad
    float* qacc = acc + (size_t)(warp * COPIES + qd) * a.dpad;

    const int64_t nw = (int64_t)gridDim.x * kW;
    const int64_t gw = (int64_t)blockIdx.x * kW + warp;
    const int64_t per = (((a.n + nw - 1) / nw) + kPassBatch - 1) / kPassBatch * kPassBatch;
    const int64_t w0 = gw * per < a.n ? gw * per : a.n;
    const int64_t w1 = w0 + per < a.n ? w0 + per : a.n;
    const int nbatch = (int)((w1 - w0 + kPassBatch - 1) / kPassBatch);

    auto load_meta = [&](int k, int32_t& rp, int32_t& rend, float& zo) {
        rp = 0;
        rend = 0;
        zo = 0.f;
        if (k < nbatch) {
            const int64_t r0 = w0 + (int64_t)k * kPassBatch;
            const int64_t rl = (r0 + kPassBatch < w1) ? r0 + kPassBatch : w1;
            if (r0 + lane < rl) {
                rp = __ldg(a.row_ptr + r0 + lane);
                zo = __ldg(a.zin + r0 + lane);
            }
            rend = __ldg(a.row_ptr + rl);
        }
    };
    int32_t rpA, reA, rpB, reB;
    float zoA, zoB;
    load_meta(0, rpA, reA, zoA);
    float zz = 0.f, bb = 0.f;
    for (int k = 0; k < nbatch; ++k) {
        load_meta(k + 1, rpB, reB, zoB);   // next batch's rows, in flight during this one
        const int64_t r0 = w0 + (int64_t)k * kPassBatch;
        const int nrows = (int)((r0 + kPassBatch < w1 ? r0 + kPassBatch : w1) - r0);
        float zreg = 0.f;
        // every lane takes part in the shuffle and the vote (full masks)
        const int32_t nxt = __shfl_down_sync(0xFFFFFFFFu, rpA, 1);
        const int32_t myl = (lane < nrows) ? ((lane + 1 < nrows) ? nxt : reA) - rpA : 0;
        const bool okq = (lane >= nrows) || (((rpA & 3) == 0) && ((myl & 3) == 0) && myl <= 16);
        const bool quad = __all_sync(0xFFFFFFFFu, okq) && vec16;
        if (quad) {
            int4 c4[4];
            float4 v4[4];
            int lens[4];
            float zolds[4];
#pragma unroll
            for (int step = 0; step < 4; ++step) {
                const int row = step * 8 + qd;
                const int32_t rs = __shfl_sync(0xFFFFFFFFu, rpA, row);
                lens[step] = __shfl_sync(0xFFFFFFFFu, myl, row);
                zolds[step] = __shfl_sync(0xFFFFFFFFu, zoA, row);
                c4[step] = make_int4(0, 0, 0, 0);
                v4[step] = make_float4(0.f, 0.f, 0.f, 0.f);
                if (4 * ql < lens[step]) {
                    c4[step] = ld_stream_i4(a.col + rs + 4 * ql);
                    v4[step] = ld_stream_f4(a.val + rs + 4 * ql);
                }
            }
#pragma unroll
            for (int step = 0; step < 4; ++step) {
                const bool act = 4 * ql < lens[step];
                int4 c = c4[step];
                float4 v = v4[step];
                if (act) {
                    const unsigned cmax = max(max((unsigned)c.x, (unsigned)c.y), max((unsigned)c.z, (unsigned)c.w));
                    if (cmax >= (unsigned)a.d) {
                        flag_error(a.status, kDevBadColumn);
                        c = make_int4(0, 0, 0, 0);
                        v = make_float4(0.f, 0.f, 0.f, 0.f);
                    }
                }
                float p = 0.f;
                if (act) {
                    p = v.x * vh[c.x];
                    p = fmaf(v.y, vh[c.y], p);
                    p = fmaf(v.z, vh[c.z], p);
                    p = fmaf(v.w, vh[c.w], p);
                }
                p += __shfl_xor_sync(0xFFFFFFFFu, p, 1);
                p += __shfl_xor_sync(0xFFFFFFFFu, p, 2);
                const float z = p - coef * zolds[step];
                const float zt = __shfl_sync(0xFFFFFFFFu, z, (lane & 7) * 4);
                if ((lane >> 3) == step) zreg = zt;
                if (act) {
                    // a row's columns are distinct (a requirement on the input), so
                    // the four loads can all go out before the four stores
                    const float a0 = qacc[c.x], a1 = qacc[c.y], a2 = qacc[c.z], a3 = qacc[c.w];
                    qacc[c.x] = fmaf(v.x, z, a0);
                    qacc[c.y] = fmaf(v.y, z, a1);
                    qacc[c.z] = fmaf(v.z, z, a2);
                    qacc[c.w] = fmaf(v.w, z, a3);
                }
                __syncwarp();
            }
        } else {
            // RI rows of this half-warp at a time: independent dot products and
            // reductions interleave; the A^T z updates then go row by row in order
            constexpr int RI = 4;
#pragma unroll 1
            for (int t0 = 0; t0 < RPH; t0 += RI) {
                int32_t rs[RI];
                int len[RI];
                float zold[RI], p[RI];
                int c0[RI];
                float v0[RI];
#pragma unroll
                for (int u = 0; u < RI; ++u) {
                    const int row = sub * RPH + t0 + u;
                    rs[u] = __shfl_sync(0xFFFFFFFFu, rpA, row & 31);
                    len[u] = __shfl_sync(0xFFFFFFFFu, myl, row & 31);
                    zold[u] = __shfl_sync(0xFFFFFFFFu, zoA, row & 31);
                    c0[u] = 0;
                    v0[u] = 0.f;
                    if (sl < len[u]) {
                        c0[u] = __ldg(a.col + rs[u] + sl);
                        v0[u] = __ldg(a.val + rs[u] + sl);
                    }
                }
#pragma unroll
                for (int u = 0; u < RI; ++u) {
                    p[u] = 0.f;
                    if (sl < len[u]) {
                        if ((unsigned)c0[u] < (unsigned)a.d)
                            p[u] = v0[u] * vh[c0[u]];
                        else
                            flag_error(a.status, kDevBadColumn);
                    }
                    for (int q = sl + LPR; q < len[u]; q += LPR) {  // rows longer than LPR
                        const int c = __ldg(a.col + rs[u] + q);
                        const float v = __ldg(a.val + rs[u] + q);
                        if ((unsigned)c < (unsigned)a.d)
                            p[u] = fmaf(v, vh[c], p[u]);
                        else
                            flag_error(a.status, kDevBadColumn);
                    }
                }
#pragma unroll
                for (int o = LPR / 2; o > 0; o >>= 1)
#pragma unroll
                    for (int u = 0; u < RI; ++u) p[u] += __shfl_xor_sync(0xFFFFFFFFu, p[u], o);
#pragma unroll
                for (int u = 0; u < RI; ++u) {
                    const float z = p[u] - coef * zold[u];
                    if (sl == t0 + u) zreg = z;
                    if (sl < len[u] && (unsigned)c0[u] < (unsigned)a.d) myacc[c0[u]] = fmaf(v0[u], z, myacc[c0[u]]);
                    for (int q = sl + LPR; q < len[u]; q += LPR) {
                        const int c = __ldg(a.col + rs[u] + q);
                        const float v = __ldg(a.val + rs[u] + q);
                        if ((unsigned)c < (unsigned)a.d) myacc[c] = fmaf(v, z, myacc[c]);
                    }
                    __syncwarp();
                }
            }
        }
        // quad batches: lane l holds z of row l; others: lane l of half h
        // holds z of row h*RPH + l (l < RPH)
        const int myrow = quad ? lane : sub * RPH + sl;
        if ((quad || sl < RPH) && myrow < nrows) {
            a.zout[r0 + myrow] = zreg;
            zz = fmaf(zreg, zreg, zz);
        }
        if (lane < nrows) bb = fmaf(zoA, zoA, bb);
        rpA = rpB;
        reA = reB;
        zoA = zoB;
    }
    __syncthreads();
    // per-CTA partials: the accumulator copies summed in a fixed order with an
    // exact two-sum (float32 hi + lo), so no float64 pipe work per CTA
    const int NS = kW * COPIES;
    for (int j = threadIdx.x; j < a.d; j += blockDim.x) {
        float hi = 0.f, lo = 0.f;
        for (int q = 0; q < NS; ++q) {
            const float x = acc[(size_t)q * a.dpad + j];
            const float t = hi + x;
            const float bp = t - hi;
            lo += (hi - (t - bp)) + (x - bp);
            hi = t;
        }
        a.gpart[(size_t)blockIdx.x * a.d + j] = make_float2(hi, lo);
    }
    __shared__ double rz[kW], rb[kW];
    double zd = (double)zz, bd = (double)bb;
    for (int o = 16; o > 0; o >>= 1) {
        zd += __shfl_xor_sync(0xFFFFFFFFu, zd, o);
        bd += __shfl_xor_sync(0xFFFFFFFFu, bd, o);
    }
    if (lane == 0) {
        rz[warp] = zd;
        rb[warp] = bd;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0, tb = 0.0;
        for (int w = 0; w < kW; ++w) {
            t += rz[w];
            tb += rb[w];
        }
        a.zpart[blockIdx.x] = t;
        if (a.bpart) a.bpart[blockIdx.x] = tb;
    }
}

}  // namespace cw
