// Status strings, version, the per-device sticky status word, and the
// measurement hooks (kernel launch counter, CUDA-event timing of named kernels).
#include <atomic>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "cw_common.cuh"

namespace cw {

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_status_mu;
unsigned* g_status[kMaxDevices] = {nullptr};
}  // namespace

unsigned* device_status_word() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return nullptr;
    std::lock_guard<std::mutex> lk(g_status_mu);
    if (!g_status[dev]) {
        unsigned* p = nullptr;
        if (cudaMalloc(&p, sizeof(unsigned)) != cudaSuccess) {
            (void)cudaGetLastError();
            return nullptr;
        }
        if (cudaMemset(p, 0, sizeof(unsigned)) != cudaSuccess) {
            (void)cudaGetLastError();
            cudaFree(p);
            return nullptr;
        }
        g_status[dev] = p;
    }
    return g_status[dev];
}

namespace {
std::mutex g_pool_mu;
bool g_pool_done[kMaxDevices] = {false};
}  // namespace

void keep_pool_cached() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        (void)cudaGetLastError();
        return;
    }
    std::lock_guard<std::mutex> lk(g_pool_mu);
    if (g_pool_done[dev]) return;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        uint64_t keep = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    (void)cudaGetLastError();
    g_pool_done[dev] = true;
}

// ---------------------------------------------------------------- measurement hooks

namespace {
std::atomic<long long> g_launches{0};
std::atomic<int> g_prof_on{0};
std::mutex g_prof_mu;
struct Pending {
    std::string name;
    cudaEvent_t a, b;
};
std::vector<Pending> g_pending;
std::vector<cudaEvent_t> g_free_events;
struct Tot {
    long long launches = 0;
    double ms = 0.0;
};
std::map<std::string, Tot> g_tot;

cudaEvent_t take_event() {
    if (!g_free_events.empty()) {
        cudaEvent_t e = g_free_events.back();
        g_free_events.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) {
        (void)cudaGetLastError();
        return nullptr;
    }
    return e;
}

void resolve_pending_locked() {
    for (auto& p : g_pending) {
        float ms = 0.f;
        if (cudaEventSynchronize(p.b) == cudaSuccess && cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
            Tot& t = g_tot[p.name];
            t.launches += 1;
            t.ms += ms;
        } else {
            (void)cudaGetLastError();
        }
        g_free_events.push_back(p.a);
        g_free_events.push_back(p.b);
    }
    g_pending.clear();
}
}  // namespace

void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

namespace {
thread_local int t_prof_suppress = 0;
}
ProfSuppress::ProfSuppress() { ++t_prof_suppress; }
ProfSuppress::~ProfSuppress() { --t_prof_suppress; }

ProfScope::ProfScope(const char* name, cudaStream_t s) : name_(name), s_(s), a_(nullptr) {
    count_launch();
    if (!g_prof_on.load(std::memory_order_relaxed) || t_prof_suppress) return;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    a_ = take_event();
    if (a_) cudaEventRecord((cudaEvent_t)a_, s_);
}

ProfScope::~ProfScope() {
    if (!a_) return;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    cudaEvent_t b = take_event();
    if (!b) return;
    cudaEventRecord(b, s_);
    g_pending.push_back(Pending{name_, (cudaEvent_t)a_, b});
}

}  // namespace cw

extern "C" {

long long cw_launch_count(void) { return cw::g_launches.load(); }

int cw_profile_enable(int enable) {
    cw::g_prof_on.store(enable ? 1 : 0);
    return CW_OK;
}

int cw_profile_reset(void) {
    std::lock_guard<std::mutex> lk(cw::g_prof_mu);
    cw::resolve_pending_locked();
    cw::g_tot.clear();
    return CW_OK;
}

int cw_profile_get(const char* kernel, long long* launches, double* total_ms) {
    if (!kernel) return CW_ERR_ARG;
    std::lock_guard<std::mutex> lk(cw::g_prof_mu);
    cw::resolve_pending_locked();
    auto it = cw::g_tot.find(kernel);
    if (launches) *launches = it == cw::g_tot.end() ? 0 : it->second.launches;
    if (total_ms) *total_ms = it == cw::g_tot.end() ? 0.0 : it->second.ms;
    return CW_OK;
}

const char* cw_status_string(int status) {
    switch (status) {
        case CW_OK: return "CW_OK";
        case CW_ERR_ARG: return "CW_ERR_ARG: invalid argument";
        case CW_ERR_SHAPE: return "CW_ERR_SHAPE: inconsistent or unsupported sizes";
        case CW_ERR_OVERFLOW: return "CW_ERR_OVERFLOW: size exceeds the index range";
        case CW_ERR_CUDA: return "CW_ERR_CUDA: CUDA runtime error";
        case CW_ERR_RANK: return "CW_ERR_RANK: numerically rank-deficient sketch";
        case CW_ERR_NOCONV: return "CW_ERR_NOCONV: LSQR did not converge";
        case CW_ERR_TIMEOUT: return "CW_ERR_TIMEOUT: bounded device wait expired";
        case CW_ERR_NONFINITE: return "CW_ERR_NONFINITE: non-finite value";
        case CW_ERR_DEVICE: return "CW_ERR_DEVICE: invalid input detected on the device";
        default: return "unknown status";
    }
}

int cw_version(void) { return 100; }

// Every block waits at a grid barrier that expects one arrival more than the
// grid has, so each wait runs out after spin_limit polls and the block returns.
__global__ void k_barrier_timeout_probe(unsigned* bar, unsigned* flag, long long spin_limit) {
    cw::grid_barrier(bar, gridDim.x + 1, flag, spin_limit);
}

int cw_selftest_barrier_timeout(int32_t blocks, int64_t spin_limit, cw_stream stream) {
    if (blocks < 1 || blocks > 1024 || spin_limit < 1 || spin_limit > (1ll << 24)) return CW_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    unsigned* w = nullptr;
    CW_CUDA_TRY(cudaMallocAsync(reinterpret_cast<void**>(&w), 4 * sizeof(unsigned), s));
    cudaError_t e = cudaMemsetAsync(w, 0, 4 * sizeof(unsigned), s);
    if (e == cudaSuccess) {
        cw::count_launch();
        k_barrier_timeout_probe<<<blocks, 32, 0, s>>>(w, w + 2, spin_limit);
        e = cudaGetLastError();
    }
    unsigned flag = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&flag, w + 2, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
    cudaFreeAsync(w, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return CW_ERR_CUDA;
    }
    return flag ? CW_ERR_TIMEOUT : CW_OK;
}

int cw_device_status(cw_stream stream) {
    unsigned* w = cw::device_status_word();
    if (!w) return CW_ERR_CUDA;
    unsigned v = 0;
    CW_CUDA_TRY(cudaStreamSynchronize(stream));
    CW_CUDA_TRY(cudaMemcpy(&v, w, sizeof(unsigned), cudaMemcpyDeviceToHost));
    if (v) CW_CUDA_TRY(cudaMemset(w, 0, sizeof(unsigned)));
    return v ? CW_ERR_DEVICE : CW_OK;
}

}  // extern "C"
