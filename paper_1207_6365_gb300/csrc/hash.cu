// cw_hash: the map (h, sigma) that defines S = Phi D (paper Section 2),
// evaluated with the same per-lane forward-difference walk the sketch kernels
// use (each lane owns rows base + lane + 32 j), so a bit-exact check of this
// entry point checks the keys every sketch kernel sorts by.
#include "cw_common.cuh"

namespace cw {

constexpr int kHashRowsPerLane = 32;
constexpr int kHashRowsPerWarp = 32 * kHashRowsPerLane;

__global__ void __launch_bounds__(256) k_hash(HashParams hp, int64_t i0, int64_t count,
                                              int32_t* __restrict__ bucket, int8_t* __restrict__ sign) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t r0 = warp * kHashRowsPerWarp + lane;
    if (r0 >= count) return;
    KeyWalk kw;
    kw.init(hp, (uint64_t)(i0 + r0), 32);
#pragma unroll 4
    for (int j = 0; j < kHashRowsPerLane; ++j) {
        const int64_t r = r0 + 32 * j;
        if (r >= count) break;
        const uint32_t key = kw.key(hp);
        if (bucket) bucket[r] = (int32_t)(key & 0x7FFFFFFFu);
        if (sign) sign[r] = (key >> 31) ? (int8_t)-1 : (int8_t)1;
        kw.step();
    }
}

}  // namespace cw

extern "C" int cw_hash(uint64_t seed, int64_t m, int64_t i0, int64_t count, int32_t* bucket,
                       int8_t* sign, cw_stream stream) {
    if (m < 1 || m > 0x7FFFFFFFll) return CW_ERR_SHAPE;
    if (i0 < 0 || count < 0 || i0 > (1ll << 62) - count) return CW_ERR_OVERFLOW;
    if (count == 0 || (!bucket && !sign)) return CW_OK;
    const cw::HashParams hp = cw::make_hash_params(seed, m);
    const int64_t warps = (count + cw::kHashRowsPerWarp - 1) / cw::kHashRowsPerWarp;
    const int64_t blocks = (warps + 7) / 8;
    if (blocks > 0x7FFFFFFFll) return CW_ERR_OVERFLOW;
    {
        CW_PROF("k_hash", stream);
        cw::k_hash<<<(unsigned)blocks, 256, 0, stream>>>(hp, i0, count, bucket, sign);
    }
    CW_LAUNCH_CHECK();
    return CW_OK;
}
