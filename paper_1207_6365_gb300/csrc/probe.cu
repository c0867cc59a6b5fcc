// Measurement probe (not an operation of the paper): the read throughput of
// 64-byte segments at random places of a large array, issued the way the CSR
// segmented sum issues its row gathers (a half-warp of 16 lanes per segment,
// 4 bytes a lane, 16 segments per half-warp in flight, the 64-byte L2 fetch
// size), and the same kernel on consecutive segments as its calibration.
// The bucket-ordered sum reads each row's col and val as such segments, so
// its read rate belongs beside this one rather than beside the copy rate.
#include <cstdint>

#include "cw_common.cuh"
#include "cw_internal.h"

namespace cw {

namespace {

// A 64-bit finaliser (MurmurHash3's fmix64): spreads segment indices over the
// array; its quality only has to defeat locality.
__device__ __forceinline__ uint64_t fmix64(uint64_t x) {
    x ^= x >> 33;
    x *= 0xff51afd7ed558ccdULL;
    x ^= x >> 33;
    x *= 0xc4ceb9fe1a85ec53ULL;
    x ^= x >> 33;
    return x;
}

constexpr int kProbeU = 16;  // segments in flight per half-warp

// Segment s (of nseg) reads the 16 floats at segment index f(s) & mask of a,
// f the finaliser (random) or the identity (sequential).  One float per
// thread is kept live through a store that never happens for finite data.
template <bool SEQ>
__global__ void __launch_bounds__(256) k_probe_gather64(const float* __restrict__ a, uint64_t mask, uint64_t nseg,
                                                        float* __restrict__ out) {
    const int lane = threadIdx.x & 31, sub = lane >> 4, sl = lane & 15;
    const uint64_t gw = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    float acc = 0.f;
    for (uint64_t base = gw * (2 * kProbeU); base < nseg; base += nw * (2 * kProbeU)) {
        float v[kProbeU];
#pragma unroll
        for (int u = 0; u < kProbeU; ++u) {
            const uint64_t s = base + 2 * u + sub;
            v[u] = 0.f;
            if (s < nseg) {
                const uint64_t off = ((SEQ ? s : fmix64(s)) & mask) * 16 + sl;  // < (mask + 1) * 16
                v[u] = SEQ ? __ldg(a + off) : ld_gather(a + off);
            }
        }
#pragma unroll
        for (int u = 0; u < kProbeU; ++u) acc += v[u];
    }
    if (acc != acc) out[0] = acc;
}

}  // namespace

}  // namespace cw

extern "C" int cw_probe_gather64(const float* a, int64_t nseg_total, int64_t nseg, int sequential,
                                 int ctas_per_sm, float* out, cw_stream stream) {
    using namespace cw;
    if (!a || !out) return CW_ERR_ARG;
    if (nseg_total <= 0 || (nseg_total & (nseg_total - 1)) || nseg < 0) return CW_ERR_SHAPE;
    if (nseg_total > ((int64_t)1 << 40)) return CW_ERR_OVERFLOW;
    if (ctas_per_sm < 1 || ctas_per_sm > 8) return CW_ERR_ARG;
    if (nseg == 0) return CW_OK;
    cudaStream_t st = (cudaStream_t)stream;
    const int grid = ctas_per_sm * num_sms();
    const uint64_t mask = (uint64_t)nseg_total - 1;
    if (sequential) {
        CW_PROF("k_probe_gather64", st);
        k_probe_gather64<true><<<grid, 256, 0, st>>>(a, mask, (uint64_t)nseg, out);
    } else {
        CW_PROF("k_probe_gather64", st);
        k_probe_gather64<false><<<grid, 256, 0, st>>>(a, mask, (uint64_t)nseg, out);
    }
    CW_LAUNCH_CHECK();
    return CW_OK;
}
