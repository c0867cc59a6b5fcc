// Shared device/host helpers of the sm_103a sparse-embedding library.
//
// The seeded map (h, sigma) that defines S = Phi D (paper Section 2) is
// evaluated here: two cubic polynomials over GF(p), p = 2^61 - 1, whose
// coefficients are SplitMix64 draws (Steele, Lea and Flood, 2014) masked to
// 61 bits.  Rows handled by one thread are evaluated by forward differences
// of the cubic (three modular additions per polynomial per row) after an
// initial Horner evaluation at four points.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstddef>

#include "cw.h"

namespace cw {

constexpr uint64_t kP61 = (1ull << 61) - 1;

// ---------------------------------------------------------------- host side

struct HashParams {
    uint64_t cb[4];   // bucket polynomial c0..c3
    uint64_t cs[4];   // sign polynomial c0..c3
    uint64_t m;       // number of buckets
    uint64_t minv;    // floor((2^64 - 1) / m) for the Barrett remainder
    uint32_t mmask;   // m - 1 when m is a power of two
    uint32_t pow2;    // 1 when m is a power of two
    // optional outer bucket (generalized sparse embedding): bucket = ho * m + h
    // with ho = g_outer(x) mod q from a third cubic
    uint64_t co[4];
    uint64_t q, qinv;
    uint32_t qmask, qpow2;
    uint32_t outer;
};

// SplitMix64 step as published (state advance by the golden gamma, then the
// two xor-shift-multiply rounds and a final xor-shift).
inline uint64_t splitmix64_next(uint64_t& state) {
    state += 0x9E3779B97F4A7C15ull;
    uint64_t z = state;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

inline HashParams make_hash_params(uint64_t seed, int64_t m) {
    HashParams hp;
    uint64_t st = seed;
    uint64_t c[8];
    for (int k = 0; k < 8;) {
        uint64_t v = splitmix64_next(st) & kP61;
        if (v == kP61) continue;  // p itself is not a field element; draw again
        c[k++] = v;
    }
    for (int k = 0; k < 4; ++k) {
        hp.cb[k] = c[k];
        hp.cs[k] = c[4 + k];
    }
    hp.m = (uint64_t)m;
    hp.minv = ~0ull / (uint64_t)m;
    hp.pow2 = ((uint64_t)m & ((uint64_t)m - 1)) == 0 ? 1u : 0u;
    hp.mmask = hp.pow2 ? (uint32_t)((uint64_t)m - 1) : 0u;
    for (int k = 0; k < 4; ++k) hp.co[k] = 0;
    hp.q = 1;
    hp.qinv = ~0ull;
    hp.qmask = 0;
    hp.qpow2 = 1;
    hp.outer = 0;
    return hp;
}

// The next `count` raw SplitMix64 outputs after the 8 accepted coefficient
// draws of `seed` (the seeds of the inner sketches of a generalized sparse
// embedding).
inline void splitmix64_after_coeffs(uint64_t seed, int count, uint64_t* out) {
    uint64_t st = seed;
    for (int k = 0; k < 8;) {
        if ((splitmix64_next(st) & kP61) != kP61) ++k;
    }
    for (int k = 0; k < count; ++k) out[k] = splitmix64_next(st);
}

// Inner sketch b of a generalized sparse embedding: bucket and sign cubics of
// seed_b (over v buckets), outer bucket cubic = the bucket cubic of `seed`
// (over q buckets); composite bucket h(i) * v + h_b(i) over q * v buckets.
inline HashParams make_general_hash_params(uint64_t seed, uint64_t seed_b, int64_t q, int64_t v) {
    HashParams hp = make_hash_params(seed_b, v);
    const HashParams ho = make_hash_params(seed, q);
    for (int k = 0; k < 4; ++k) hp.co[k] = ho.cb[k];
    hp.q = (uint64_t)q;
    hp.qinv = ho.minv;
    hp.qpow2 = ho.pow2;
    hp.qmask = ho.mmask;
    hp.outer = 1;
    return hp;
}

// ---------------------------------------------------------------- device field arithmetic

__device__ __forceinline__ uint64_t addmod61(uint64_t a, uint64_t b) {
    uint64_t r = a + b;  // a, b < p  =>  r < 2p < 2^62
    return r >= kP61 ? r - kP61 : r;
}

__device__ __forceinline__ uint64_t submod61(uint64_t a, uint64_t b) {
    return a >= b ? a - b : a + (kP61 - b);
}

// a * b mod p for a, b < p: the 122-bit product is split at bit 61 and the two
// halves are added (2^61 = 1 mod p), followed by one more fold.
__device__ __forceinline__ uint64_t mulmod61(uint64_t a, uint64_t b) {
    uint64_t lo = a * b;
    uint64_t hi = __umul64hi(a, b);                    // < 2^58
    uint64_t r = (lo & kP61) + ((hi << 3) | (lo >> 61));  // < 2^62
    r = (r & kP61) + (r >> 61);
    return r >= kP61 ? r - kP61 : r;
}

__device__ __forceinline__ uint64_t reduce61(uint64_t x) {
    uint64_t r = (x & kP61) + (x >> 61);
    return r >= kP61 ? r - kP61 : r;
}

__device__ __forceinline__ uint64_t horner61(const uint64_t c[4], uint64_t x) {
    x = reduce61(x);
    uint64_t acc = c[3];
    acc = addmod61(mulmod61(acc, x), c[2]);
    acc = addmod61(mulmod61(acc, x), c[1]);
    acc = addmod61(mulmod61(acc, x), c[0]);
    return acc;
}

// Cubic evaluated along x0, x0 + s, x0 + 2s, ... by forward differences.
struct CubicWalk {
    uint64_t g, d1, d2, d3;
    __device__ __forceinline__ void init(const uint64_t c[4], uint64_t x0, uint64_t s) {
        uint64_t g0 = horner61(c, x0);
        uint64_t g1 = horner61(c, x0 + s);
        uint64_t g2 = horner61(c, x0 + 2 * s);
        uint64_t g3 = horner61(c, x0 + 3 * s);
        uint64_t a1 = submod61(g1, g0), a2 = submod61(g2, g1), a3 = submod61(g3, g2);
        uint64_t b1 = submod61(a2, a1), b2 = submod61(a3, a2);
        g = g0;
        d1 = a1;
        d2 = b1;
        d3 = submod61(b2, b1);
    }
    __device__ __forceinline__ void step() {
        g = addmod61(g, d1);
        d1 = addmod61(d1, d2);
        d2 = addmod61(d2, d3);
    }
};

__device__ __forceinline__ uint32_t bucket_of(uint64_t g, const HashParams& hp) {
    if (hp.pow2) return (uint32_t)g & hp.mmask;
    uint64_t q = __umul64hi(g, hp.minv);
    uint64_t r = g - q * hp.m;
    if (r >= hp.m) r -= hp.m;
    return (uint32_t)r;
}

// key = bucket | (sign bit << 31); the sign bit is set when sigma = -1.
__device__ __forceinline__ uint32_t make_key(uint64_t gb, uint64_t gs, const HashParams& hp) {
    return bucket_of(gb, hp) | ((uint32_t)(gs & 1u) << 31);
}

__device__ __forceinline__ uint32_t outer_bucket_of(uint64_t g, const HashParams& hp) {
    if (hp.qpow2) return (uint32_t)g & hp.qmask;
    uint64_t q = __umul64hi(g, hp.qinv);
    uint64_t r = g - q * hp.q;
    if (r >= hp.q) r -= hp.q;
    return (uint32_t)r;
}

// Walks the polynomials together and yields keys; OUTER adds the outer bucket
// of a generalized embedding (hp.outer set): key bucket = ho * hp.m + h.
template <bool OUTER>
struct KeyWalkT {
    CubicWalk b, s, o;
    __device__ __forceinline__ void init(const HashParams& hp, uint64_t x0, uint64_t step) {
        b.init(hp.cb, x0, step);
        s.init(hp.cs, x0, step);
        if (OUTER) o.init(hp.co, x0, step);
    }
    __device__ __forceinline__ uint32_t key(const HashParams& hp) const {
        const uint32_t k = make_key(b.g, s.g, hp);
        if (!OUTER) return k;
        return (outer_bucket_of(o.g, hp) * (uint32_t)hp.m + (k & 0x7FFFFFFFu)) | (k & 0x80000000u);
    }
    __device__ __forceinline__ void step() {
        b.step();
        s.step();
        if (OUTER) o.step();
    }
};
using KeyWalk = KeyWalkT<false>;

// ---------------------------------------------------------------- errors and status

// Device-side sticky flag bits (one word per device).
enum : unsigned {
    kDevBadColumn = 1u,
    kDevDupColumn = 2u,
    kDevBadRowPtr = 4u,
    kDevNonFinite = 8u,
    kDevTimeout = 16u,   // a bounded device-side wait gave up
};

// Per-device status word (allocated once per device, never freed).
unsigned* device_status_word();

__device__ __forceinline__ void flag_error(unsigned* st, unsigned bit) {
    if (st) atomicOr(st, bit);
}

#define CW_CUDA_TRY(expr)                          \
    do {                                           \
        cudaError_t _e = (expr);                   \
        if (_e != cudaSuccess) {                   \
            (void)cudaGetLastError();              \
            return CW_ERR_CUDA;                    \
        }                                          \
    } while (0)

#define CW_LAUNCH_CHECK()                          \
    do {                                           \
        cudaError_t _e = cudaGetLastError();       \
        if (_e != cudaSuccess) return CW_ERR_CUDA; \
    } while (0)

// ---------------------------------------------------------------- measurement hooks

// Every kernel launch of the library sits inside a ProfScope: it counts the
// launch and, while profiling is enabled, brackets it with CUDA events recorded
// on the launching stream (durations accumulate per kernel name).
void count_launch();
class ProfScope {
  public:
    ProfScope(const char* name, cudaStream_t s);
    ~ProfScope();
    ProfScope(const ProfScope&) = delete;
    ProfScope& operator=(const ProfScope&) = delete;

  private:
    const char* name_;
    cudaStream_t s_;
    void* a_;
};

// While alive on a thread, ProfScope records no events on that thread.
class ProfSuppress {
  public:
    ProfSuppress();
    ~ProfSuppress();
    ProfSuppress(const ProfSuppress&) = delete;
    ProfSuppress& operator=(const ProfSuppress&) = delete;
};

#define CW_PROF_CAT2(a, b) a##b
#define CW_PROF_CAT(a, b) CW_PROF_CAT2(a, b)
#define CW_PROF(name, stream) ::cw::ProfScope CW_PROF_CAT(_cw_prof_scope_, __LINE__)(name, stream)

// ---------------------------------------------------------------- stream-ordered scratch

// Keeps the current device's default memory pool from returning freed memory
// to the driver at every synchronisation (its default release threshold is 0,
// which makes the next cudaMallocAsync map fresh pages).  Process-local: it
// changes this process's pool attribute only, once per device.
void keep_pool_cached();

// Scratch arena: one cudaMallocAsync on the call's stream, carved into
// 256-byte aligned pieces, released with cudaFreeAsync on the same stream.
class Scratch {
  public:
    explicit Scratch(cudaStream_t s) : s_(s) {}
    // Carve from a caller-owned buffer instead of allocating: alloc() then
    // fails with cudaErrorMemoryAllocation when the reservations exceed `bytes`.
    Scratch(cudaStream_t s, void* external, size_t bytes) : s_(s), ext_(external), ext_bytes_(bytes) {}
    ~Scratch() { release(); }
    Scratch(const Scratch&) = delete;
    Scratch& operator=(const Scratch&) = delete;

    // Reserve `bytes` (call before alloc()); returns the offset.
    size_t reserve(size_t bytes) {
        size_t off = size_;
        size_ += (bytes + 255) & ~size_t(255);
        return off;
    }
    cudaError_t alloc() {
        if (ext_) {
            if (size_ > ext_bytes_) return cudaErrorMemoryAllocation;
            base_ = ext_;
            return cudaSuccess;
        }
        if (size_ == 0) return cudaSuccess;
        keep_pool_cached();
        return cudaMallocAsync(&base_, size_, s_);
    }
    size_t size() const { return size_; }
    template <class T>
    T* at(size_t off) const {
        return reinterpret_cast<T*>(static_cast<char*>(base_) + off);
    }
    void release() {
        if (base_ && !ext_) cudaFreeAsync(base_, s_);
        base_ = nullptr;
    }

  private:
    cudaStream_t s_;
    void* base_ = nullptr;
    size_t size_ = 0;
    void* ext_ = nullptr;
    size_t ext_bytes_ = 0;
};

// ---------------------------------------------------------------- bounded grid barrier

constexpr long long kBarrierSpinLimit = 1ll << 24;  // ~1 s with 64 ns sleeps

// bar[0] = arrival count, bar[1] = generation.  Returns false (after flagging
// the status word) when the wait exceeded its limit (spin_limit polls); the
// caller must return.
static __device__ __noinline__ bool grid_barrier(unsigned* bar, unsigned nblocks, unsigned* timeout_flag,
                                                 long long spin_limit = kBarrierSpinLimit) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        ok = 1;
        __threadfence();
        const unsigned gen = atomicAdd(&bar[1], 0u);
        const unsigned arrived = atomicAdd(&bar[0], 1u) + 1u;
        if (arrived == nblocks) {
            atomicExch(&bar[0], 0u);
            __threadfence();
            atomicAdd(&bar[1], 1u);
        } else {
            long long it = 0;
            while (atomicAdd(&bar[1], 0u) == gen) {
                __nanosleep(64);
                if (++it > spin_limit) {
                    atomicExch(timeout_flag, 1u);
                    ok = 0;
                    break;
                }
            }
            if (ok && atomicAdd(timeout_flag, 0u)) ok = 0;
        }
        __threadfence();
    }
    __syncthreads();
    return ok != 0;
}

inline int num_sms() {
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 1;
}

// ---- gathers of short row segments (CSR rows visited in bucket order)
// A random 64-byte segment read with a plain load also pulls the other half
// of its 128-byte line from DRAM (measured on GB300: 2.0x the useful bytes for
// random 64-byte segments).  These loads skip L1 and limit the L2 prefetch to
// 64 bytes (1.05x); the data must not change during the kernel.  For segments
// that cross a 64-byte boundary the default fetch is faster.
__device__ __forceinline__ int ld_gather(const int32_t* p) {
    int r;
    asm("ld.global.nc.L1::no_allocate.L2::64B.s32 %0, [%1];\n" : "=r"(r) : "l"(p));
    return r;
}
__device__ __forceinline__ float ld_gather(const float* p) {
    float r;
    asm("ld.global.nc.L1::no_allocate.L2::64B.f32 %0, [%1];\n" : "=f"(r) : "l"(p));
    return r;
}

// ---- cp.async helpers (global -> shared without passing through registers)
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gmem));
}
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

}  // namespace cw
