// cw_sketch_csr_noalloc: the CSR sketch without any device allocation.
//
// Some callers cannot allocate device memory at call time: code running under
// a custom allocator that owns all of the device's memory, real-time or
// latency-critical paths where cudaMallocAsync could block on the memory
// pool, and hosts that load this library into a process whose allocator must
// not be re-entered.  This entry point takes its scratch from one file-scope
// __device__ array instead, so it calls no cudaMalloc / cudaMallocAsync /
// cudaFree (nor any allocating library routine).
//
// The array is part of the library image: every GPU that loads the library
// holds it until the process exits.  All calls share it and it keeps the last
// call's contents; the kernels clear what must start at zero on every call.
// Calls whose work overlaps on the GPU (different streams, or the same stream
// with graph-level concurrency) race on the array and must be serialised by
// the caller.  Input errors found on the device (a column out of range, a
// decreasing row_ptr) go to a second static word that cw_noalloc_status reads
// and clears, again without allocating.
#include <mutex>

#include "cw_common.cuh"
#include "cw_internal.h"

namespace cw {

constexpr size_t kNoAllocScratchBytes = 24u << 20;  // 24 MiB

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];
static __device__ __align__(256) unsigned g_noalloc_status;

namespace {
constexpr int kNoAllocMaxDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_ptr[kNoAllocMaxDevices] = {nullptr};
unsigned* g_noalloc_status_ptr[kNoAllocMaxDevices] = {nullptr};

// Device addresses of the two arrays for the current device (set up once per
// device, with that device current).  In host code the array names are host
// stand-ins, not device addresses, so they are never passed to a kernel.
int noalloc_setup(void** scratch, unsigned** status) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNoAllocMaxDevices) {
        (void)cudaGetLastError();
        return CW_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        void* q = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess ||
            cudaGetSymbolAddress(&q, g_noalloc_status) != cudaSuccess || !p || !q) {
            (void)cudaGetLastError();
            return CW_ERR_CUDA;
        }
        g_noalloc_ptr[dev] = p;
        g_noalloc_status_ptr[dev] = static_cast<unsigned*>(q);
    }
    *scratch = g_noalloc_ptr[dev];
    *status = g_noalloc_status_ptr[dev];
    return CW_OK;
}
}  // namespace

}  // namespace cw

extern "C" int cw_sketch_csr_noalloc(const cw_csr* A, const float* b, int64_t m, uint64_t seed, float* SA,
                                     float* Sb, cw_stream stream) {
    if (!A || !SA) return CW_ERR_ARG;
    int st = cw::validate_common(A->n, A->d, m);
    if (st != CW_OK) return st;
    if (A->d < 1) return CW_ERR_SHAPE;
    if (A->nnz < 0 || A->nnz > 0x7FFFFFFFll) return CW_ERR_OVERFLOW;
    if (A->n > 0 && (!A->row_ptr || (A->nnz > 0 && (!A->col || !A->val)))) return CW_ERR_ARG;
    void* scratch = nullptr;
    unsigned* status = nullptr;
    st = cw::noalloc_setup(&scratch, &status);
    if (st != CW_OK) return st;
    const cw::SketchWorkspace ws{scratch, cw::kNoAllocScratchBytes, status};
    const cw::ProfSuppress no_events;  // no CUDA events are created inside this call
    return cw::sketch_impl(cw::kSketchCSR, A->n, A->d, 0, 0, A->row_ptr, A->col, A->val, nullptr, b, m, seed, SA,
                           b ? Sb : nullptr, nullptr, stream, nullptr, &ws);
}

extern "C" int cw_noalloc_status(cw_stream stream) {
    void* scratch = nullptr;
    unsigned* status = nullptr;
    int st = cw::noalloc_setup(&scratch, &status);
    if (st != CW_OK) return st;
    unsigned v = 0;  // host word on the stack: nothing is allocated
    cudaStream_t s = (cudaStream_t)stream;
    CW_CUDA_TRY(cudaMemcpyAsync(&v, status, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
    CW_CUDA_TRY(cudaMemsetAsync(status, 0, sizeof(unsigned), s));
    CW_CUDA_TRY(cudaStreamSynchronize(s));
    return v ? CW_ERR_DEVICE : CW_OK;
}
