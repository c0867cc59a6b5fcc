// Internal (non-exported) entry points shared between translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "cw.h"

namespace cw {

enum SketchModeId { kSketchCSR = 0, kSketchDense = 1, kSketchVec = 2 };

// Caller-provided scratch for sketch_impl (no allocation inside the call).
struct SketchWorkspace {
    void* base;        // device memory, 256-byte aligned
    size_t bytes;
    unsigned* status;  // device word for the sticky input-error flags
};

struct HashParams;

// One inner sketch of a generalized sparse embedding (CSR only): its hash
// (composite bucket over q * v buckets) and where its buckets land: bucket u
// goes to output row (u / v) * stride + off + u % v, scaled by `scale`.
struct SketchLayout {
    const HashParams* hp;
    int64_t v, stride, off;
    float scale;
};

// SA / Sb of a CSR, dense or vector input (see sketch.cu).  With `ext`, all
// scratch is carved from ext->base (CW_ERR_SHAPE when it does not fit).
// accumulate (CSR only, without lay or vals): add this call's S A and S b to
// SA and Sb instead of overwriting them (row shards of one matrix, i0 their
// first global row, summed in call order).
int sketch_impl(int mode, int64_t n, int64_t d, int64_t lda, int64_t i0, const int32_t* row_ptr,
                const int32_t* col, const float* val, const float* A, const float* b, int64_t m,
                uint64_t seed, float* SA, float* Sb, int32_t* bucket_ptr_out, cudaStream_t stream,
                double* SA64 = nullptr, const SketchWorkspace* ext = nullptr, const SketchLayout* lay = nullptr,
                const float* vals = nullptr, bool accumulate = false);
int validate_common(int64_t n, int64_t d, int64_t m);

// The preconditioned LSQR of cw_lsqr_precond (lsqr.cu); SA_in / Sb_in (device,
// the sketch of A and b with `seed`) skip its sketch step when both are given.
int lsqr_run(const cw_csr* A, const float* b, int64_t m, uint64_t seed, double rtol, int32_t max_iter, double* x,
             int32_t* iters, double* final_test, cudaStream_t stream, const float* SA_in, const float* Sb_in);

// float64 Householder QR of [SA | Sb]; synchronises.  SA64 (row-major float64)
// replaces SA when given.
int qr64(const float* SA, int64_t m, int d, const float* Sb, double* R, double* c, cudaStream_t stream,
         const double* SA64 = nullptr);
int trsv_upper(const double* R, int d, const double* rhs, double* x, cudaStream_t stream);
// x' = argmin ||SA x - Sb|| by qr64 and trsv_upper; R (nullable) receives the
// factor.  Synchronises.
int solve_from_sketch(const float* SA, const float* Sb, int64_t m, int d, double* x, double* R_out,
                      cudaStream_t stream);
int trsm_upper(const double* R, int d, const double* B, int k, double* X, cudaStream_t stream);
int tri_inverse(const double* R, int d, double* M, cudaStream_t stream);
// [SA | Sb]^T [SA | Sb] (float64, symmetric, nc = d + (Sb != NULL)) on the
// tensor cores (3xTF32); CW_ERR_SHAPE when d > 256.
// W32 (nullable) receives the same matrix rounded to float32.
int gram_tc(const float* SA, int64_t m, int d, const float* Sb, double* Gm, unsigned* tflag, cudaStream_t stream,
            float* W32 = nullptr);
// The same Gram matrix for any d <= 1024: tensor cores when d <= 256, float32
// CUDA-core tiles with float64 partials otherwise.
int gram_f64(const float* SA, int64_t m, int d, const float* Sb, double* Gm, unsigned* tflag, cudaStream_t stream,
             float* W32 = nullptr);
// Gram + Cholesky + explicit inverse in shared memory (LSQR preconditioner).
// With flags_dev NULL it synchronises and returns CW_ERR_RANK (non-positive
// pivot) or CW_ERR_TIMEOUT, *kappa_lb_host receiving R's diagonal ratio.
// With flags_dev (device, 16 bytes) it does not synchronise: flags_dev[0] =
// failed pivot, [1] = tensor-core wait gave up, float at [2] = diagonal ratio.
int gram_chol_inverse(const float* SA, int64_t m, int d, const float* Sb, double* M, float* M32T, double* c,
                      float* kappa_lb_host, cudaStream_t stream, unsigned* flags_dev = nullptr);

}  // namespace cw
