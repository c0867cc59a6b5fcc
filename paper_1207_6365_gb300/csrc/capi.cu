// Status strings, version and the per-device sticky status word.
#include <mutex>

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

}  // namespace cw

extern "C" {

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
