/*
 * cw.h - C ABI of the GB300 (sm_103a) sparse-embedding library.
 *
 * The library applies the sparse embedding matrix S = Phi D of Clarkson and
 * Woodruff, "Low Rank Approximation and Regression in Input Sparsity Time"
 * (Section 2): Phi is t x n with a single 1 per column, Phi[h(i), i] = 1, and
 * D = diag(sigma) holds random signs, so S has one +-1 per column and
 * SA = Phi D A is computed in O(nnz(A)) (Theorem 1).  On top of SA it solves
 * least squares by sketch-and-solve (Theorem "lin reg", with the QR solve of
 * the proof of Theorem "renRegAlg"), by LSQR preconditioned with R from the
 * QR of SA (Section 7.6, Theorem "it reg"), and it approximates leverage
 * scores as row norms of A R^-1 Pi_2 (Section 6, Theorem "icml").
 *
 * The random map.  The paper draws h uniformly and the signs independently;
 * this library fixes a seeded 4-wise independent family.  With p = 2^61 - 1
 * and the SplitMix64 stream (Steele, Lea and Flood, 2014) started at `seed`,
 * each 64-bit draw z gives a coefficient c = z & (2^61 - 1) (the value p is
 * rejected and drawn again); draws 0..3 are c0..c3 of the bucket polynomial,
 * draws 4..7 those of the sign polynomial, g(x) = c3 x^3 + c2 x^2 + c1 x + c0
 * mod p at x = the 0-based row index, and
 *     h(i) = g_bucket(i) mod m,    sigma(i) = +1 if g_sign(i) is even else -1.
 * S is unscaled (entries exactly +-1), as in the paper's definition.
 *
 * Conventions for every entry point:
 *  - Array arguments are DEVICE pointers owned by the caller unless marked
 *    "host".  Nothing is retained after the call returns (or, for
 *    asynchronous calls, after the stream reaches the call's end).
 *  - Matrices are row-major.  CSR uses int32 row_ptr[n+1] and col[nnz] and
 *    float32 val[nnz]; column indices within a row must be distinct and in
 *    [0, d); row_ptr must start at 0 and be non-decreasing.
 *  - Work is enqueued on `stream` (a cudaStream_t; NULL is the legacy default
 *    stream).  Calls without host outputs are asynchronous; calls with host
 *    outputs synchronise `stream` before returning.
 *  - Scratch memory is allocated stream-ordered (cudaMallocAsync) and freed
 *    stream-ordered before the call returns.
 *  - Arguments are validated on the host before any launch; a bad argument
 *    returns a negative status and enqueues nothing.  Violations only visible
 *    on the device (a column index out of range, a decreasing row_ptr) set a
 *    per-device sticky flag that cw_device_status() reports; cw_csr_check()
 *    validates a CSR matrix completely.
 *  - Results are deterministic: the same inputs, seed and sizes give bitwise
 *    identical outputs (fixed summation orders, no floating-point atomics).
 */
#ifndef CW_H
#define CW_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *cw_stream; /* identical to cudaStream_t */

/* Status codes returned by every entry point. */
enum {
    CW_OK = 0,
    CW_ERR_ARG = -1,       /* null pointer, bad flag, bad tolerance             */
    CW_ERR_SHAPE = -2,     /* inconsistent or unsupported sizes                 */
    CW_ERR_OVERFLOW = -3,  /* a size exceeds the library's index range          */
    CW_ERR_CUDA = -4,      /* a CUDA runtime call or launch failed              */
    CW_ERR_RANK = -5,      /* R has |R_jj| <= d * 2^-52 * max|R_ii|             */
    CW_ERR_NOCONV = -6,    /* LSQR reached max_iter without meeting its test    */
    CW_ERR_TIMEOUT = -7,   /* a bounded device wait expired                     */
    CW_ERR_NONFINITE = -8, /* NaN / Inf met where a finite value is required    */
    CW_ERR_DEVICE = -9     /* the device flagged invalid input (see above)      */
};

/* CSR matrix, n x d with nnz stored entries (all device pointers). */
typedef struct {
    int64_t n, d, nnz;
    const int32_t *row_ptr; /* n + 1 entries, row_ptr[0] = 0, row_ptr[n] = nnz */
    const int32_t *col;     /* nnz entries in [0, d), distinct within a row    */
    const float *val;       /* nnz entries                                     */
} cw_csr;

/* Human-readable name of a status code (static string, never NULL). */
const char *cw_status_string(int status);

/* Library version as major * 10000 + minor * 100 + patch. */
int cw_version(void);

/*
 * cw_device_status (a utility, no operation of the paper) - synchronise
 * `stream`, then return and clear the calling device's sticky
 * device-side flag: CW_OK, or CW_ERR_DEVICE if some kernel of this library
 * met invalid input since the last call, or CW_ERR_CUDA if the sync failed.
 */
int cw_device_status(cw_stream stream);

/*
 * cw_selftest_barrier_timeout (a test utility, no operation of the paper) -
 * runs the library's bounded grid barrier (the one its cooperative kernels
 * use) with `blocks` blocks that wait for one arrival more than the grid has,
 * so every wait gives up after spin_limit polls (about 64 ns apart) and its
 * block returns.  Returns CW_ERR_TIMEOUT, the status every timed-out
 * device-side wait of the library produces; CW_OK would mean the barrier did
 * not wait.  blocks in [1, 1024], spin_limit in [1, 2^24], else CW_ERR_ARG.
 * Synchronises `stream`; the context stays usable afterwards.
 */
int cw_selftest_barrier_timeout(int32_t blocks, int64_t spin_limit, cw_stream stream);

/*
 * cw_hash - the map (h, sigma) defining S (paper Section 2).
 * bucket[k] = h(i0 + k) in [0, m), sign[k] = sigma(i0 + k) in {+1, -1} for
 * k < count.  Requirements: m >= 1, 0 <= i0, i0 + count <= 2^62.  Either
 * output may be NULL.  Asynchronous.
 */
int cw_hash(uint64_t seed, int64_t m, int64_t i0, int64_t count, int32_t *bucket, int8_t *sign,
            cw_stream stream);

/*
 * cw_csr_check (a utility, no operation of the paper) - validate the CSR
 * structure the sketch kernels assume:
 * row_ptr[0] = 0, row_ptr[n] = nnz, row_ptr non-decreasing, every column in
 * [0, d) and no column twice within a row.  Returns CW_OK or CW_ERR_ARG.
 * The sketch kernels themselves detect out-of-range columns and decreasing
 * row_ptr (sticky device flag) but not repeated columns, which would make a
 * row's updates race.  Synchronises the stream.
 */
int cw_csr_check(const cw_csr *A, cw_stream stream);

/*
 * cw_sketch_csr - SA = S A and Sb = S b for CSR A (paper Section 2; Theorem
 * "lin reg" sketches A and b with the same S).
 * A: n x d CSR (n <= 2^31 - 1, nnz <= 2^31 - 1, 1 <= d <= 2^20).
 * b: n floats or NULL.  m: sketch rows, 1 <= m <= 2^19.
 * SA: m x d floats, row-major, fully overwritten (empty buckets give zeros).
 * Sb: m floats, overwritten; may be NULL (ignored when b is NULL).
 * Each SA entry is the float32 sum of its bucket's signed entries in a fixed
 * order.  Asynchronous.
 */
int cw_sketch_csr(const cw_csr *A, const float *b, int64_t m, uint64_t seed, float *SA,
                  float *Sb, cw_stream stream);

/*
 * cw_sketch_csr_rows - as cw_sketch_csr for a row shard: local row i of A is
 * global row i0 + i of the full matrix and is hashed with that global index,
 * so the sum over shards of their SA equals the SA of the whole matrix
 * (SA is linear in the rows of A, Section 2: the exchange step when rows are
 * spread over several devices).
 */
int cw_sketch_csr_rows(const cw_csr *A, int64_t i0, const float *b, int64_t m, uint64_t seed,
                       float *SA, float *Sb, cw_stream stream);

/*
 * cw_sketch_csr_general - SA = S A and Sb = S b for a generalized sparse
 * embedding S (paper Section "Generalized Sparse Embedding Matrices", "The
 * construction"): an outer hash h: [n] -> [q] groups the rows into q blocks;
 * block i is multiplied by B^(i), kappa independent v-row sparse embeddings
 * stacked and each scaled by 1 / sqrt(kappa) (the Kane-Nelson form of
 * Theorem "general"), so S has t = q * v * kappa rows.
 * Row i of A with outer bucket h(i) and inner bucket h_b(i), sign s_b(i), of
 * inner sketch b adds s_b(i) / sqrt(kappa) * A_i to output row
 * h(i) * v * kappa + b * v + h_b(i).
 * h is the bucket cubic of `seed` over q buckets (the same function
 * cw_hash(seed, q) returns); inner sketch b uses the bucket and sign cubics of
 * seed_b over v buckets, where seed_0, ..., seed_{kappa-1} are the next kappa
 * raw SplitMix64 outputs after the eight accepted coefficient draws of seed.
 * A: as cw_sketch_csr.  1 <= q, 1 <= v, q * v <= 2^19, 1 <= kappa <= 4096,
 * q * v * kappa <= 2^31 - 1.
 * SA: (q * v * kappa) x d floats, row-major, fully overwritten.
 * Sb: q * v * kappa floats, overwritten; may be NULL (ignored when b is NULL).
 * Runs the CSR sketch kappa times (one per inner sketch; O(nnz(A) * kappa)
 * work, as in Lemma "time"), each pass deterministic as cw_sketch_csr.
 * Asynchronous.
 */
int cw_sketch_csr_general(const cw_csr *A, const float *b, int64_t q, int64_t v, int32_t kappa,
                          uint64_t seed, float *SA, float *Sb, cw_stream stream);

/*
 * Sketches with given values at the hash positions, and their backward (the
 * derivative of SA and Sb with respect to the sketch's values).
 * S(v) has the one entry of column i at row h(i) (the map of Section 2) with
 * value v_i in place of sigma(i); v = sigma gives the sparse embedding itself.
 * SA(v)[k, :] = sum_{i: h(i) = k} v_i A_i and Sb(v)[k] = sum_{i: h(i) = k} v_i b_i.
 * v: n floats (device).  Other arguments, limits and outputs as
 * cw_sketch_csr / cw_sketch_dense (SA fully overwritten; Sb when b and Sb are
 * both given).  Sums are float32 in a fixed order.  Asynchronous.
 */
int cw_sketch_csr_values(const cw_csr *A, const float *b, int64_t m, uint64_t seed, const float *v,
                         float *SA, float *Sb, cw_stream stream);
int cw_sketch_dense_values(const float *A, int64_t n, int64_t d, int64_t lda, const float *b, int64_t m,
                           uint64_t seed, const float *v, float *SA, float *Sb, cw_stream stream);

/*
 * cw_sketch_values_backward_* - (not an operation of the paper: the derivative
 * of the values sketch above, whose positions are the map h of Section 2)
 * gv_i = dL/dv_i = <gSA[h(i), :], A_i> + gSb[h(i)] b_i
 * for a loss L with gradients gSA = dL/dSA (m x d row-major, device) and
 * gSb = dL/dSb (m, device; NULL, or b NULL, drops the second term).  gv: n
 * floats (device), fully overwritten.  One pass over the rows of A, each row
 * reading the gradient row of its bucket (float32 sum in a fixed order per
 * row; no atomics).  Limits as the forward.  Asynchronous.
 */
int cw_sketch_values_backward_csr(const cw_csr *A, const float *b, int64_t m, uint64_t seed, const float *gSA,
                                  const float *gSb, float *gv, cw_stream stream);
int cw_sketch_values_backward_dense(const float *A, int64_t n, int64_t d, int64_t lda, const float *b, int64_t m,
                                    uint64_t seed, const float *gSA, const float *gSb, float *gv,
                                    cw_stream stream);

/*
 * Batched sketch-and-solve: many independent regressions of uneven size
 * solved by one graph launch.  Problem p gives x'_p = argmin ||S_p A_p x -
 * S_p b_p|| (Theorem "lin reg"), S_p the sparse embedding of Section 2 with
 * its own m_p and seed_p (the same S_p cw_sketch_csr(A_p, b_p, m_p, seed_p)
 * applies), solved through R of a QR factorisation of S_p A_p (proof of
 * Theorem "renRegAlg").
 *
 * cw_batch_problem: A (device CSR, 1 <= d <= 128, n and nnz as for
 * cw_sketch_csr), b (device, n floats), m (d <= m <= 2^19), seed, x (device,
 * d doubles: the result), SA (device m x d floats) and Sb (device m floats):
 * where S_p A_p and S_p b_p are written, or NULL to keep them in memory the
 * plan owns.
 */
typedef struct {
    cw_csr A;
    const float *b;
    int64_t m;
    uint64_t seed;
    double *x;
    float *SA;
    float *Sb;
} cw_batch_problem;

typedef struct cw_batch cw_batch; /* opaque plan */

#define CW_BATCH_AUTOTUNE 1 /* time slab sizes and CTAs per SM on this batch */
#define CW_BATCH_EAGER 2    /* launch the kernels directly instead of a CUDA graph */

/*
 * cw_batch_create - plan a batch of `count` problems (host array; the device
 * arrays it points to must stay valid and at the same addresses for the life
 * of the plan, since the graph reads them there).  Allocates the plan's
 * device memory (scratch, and SA / Sb where NULL), uploads the descriptors and
 * captures the batch in a CUDA graph: the batched sketch (eight launches over
 * all problems) and one persistent cooperative solve kernel.  With
 * CW_BATCH_AUTOTUNE, times four segmented-sum variants (16 or 32 lanes per
 * CSR row, or 16- or 8-bucket ranges per warp),
 * then slab sizes {512, 1024, 2048, 4096} x {1, 2} CTAs per SM of the solve,
 * on the batch (running it) and keeps the fastest; the choice is
 * appended to the file named by the CW_TUNE_CACHE environment variable when
 * set, and read back from it for the same shapes.  Synchronises `stream`.
 * Errors: CW_ERR_ARG (NULL pointers), CW_ERR_SHAPE (a problem outside the
 * limits above), CW_ERR_OVERFLOW, CW_ERR_CUDA; *plan is NULL then.
 */
int cw_batch_create(const cw_batch_problem *probs, int32_t count, int32_t flags, cw_stream stream,
                    cw_batch **plan);

/* cw_batch_run - solve the whole batch once (one graph launch).  Asynchronous. */
int cw_batch_run(cw_batch *plan, cw_stream stream);

/*
 * cw_batch_finish - wait for the batch and read each problem's status into
 * `status` (host, count ints, or NULL): 0 solved in the batch, 3 re-solved by
 * the float64 Householder QR because the batch's Cholesky factor failed or
 * its refinement did not converge, 4 S_p A_p numerically rank deficient (the
 * QR found it so; x_p is set to zero).  *fallbacks (or NULL) = how many went
 * to the QR.  Returns CW_ERR_TIMEOUT if a grid barrier gave up, CW_ERR_ARG for
 * input errors the sketch kernels flagged.  Synchronises `stream`.
 */
int cw_batch_finish(cw_batch *plan, cw_stream stream, int32_t *status, int32_t *fallbacks);

/*
 * cw_batch_info - info[0..8] = slab rows, CTAs per SM, solve grid, graph in
 * use (1) or direct launches (0), work units, tuned (1 timed, 2 from the
 * cache, 0 defaults), plan device bytes, refinement steps at most, lanes per
 * CSR row of the segmented sum (16 or 32; 0 / -8: the 16- / 8-bucket range variants).
 * `info` holds 9 values.
 */
int cw_batch_info(const cw_batch *plan, int64_t *info);

/*
 * cw_batch_phases - durations (ms, from the device's global timer) of the
 * solve kernel's phases in the last completed run: [0] Gram units, [1]
 * Cholesky and x0, then for each refinement step the residual units and the
 * corrections (a converged problem skips later steps; a step with nothing to
 * do takes only its barrier).  Writes at most `max` values and returns how many
 * (2 + 2 * steps), or a negative status.  Synchronises `stream`.
 */
int cw_batch_phases(const cw_batch *plan, cw_stream stream, double *ms, int32_t max);

/* cw_batch_destroy - free the plan (NULL is allowed). */
int cw_batch_destroy(cw_batch *plan);

/*
 * cw_sketch_csr_noalloc - cw_sketch_csr for callers that cannot allocate
 * device memory during the call: code that runs under its own allocator owning
 * the device's memory, latency-critical paths where a pool allocation could
 * block, or hosts whose allocator must not be re-entered.  (Not a step of the
 * paper's method: the paper has no counterpart; it is a deployment variant.)
 * Same arguments, results and determinism as cw_sketch_csr, but every scratch
 * byte comes from one static device array of 24 MiB built into the library,
 * so this call makes no cudaMalloc / cudaMallocAsync / cudaFree call and no
 * allocating library call.  Every GPU that loads the library holds that array
 * until the process exits.
 * Limit: n * 28 (n * 24 without b) + (m + 1) * 4 bytes plus the tile
 * histograms must fit in 24 MiB (roughly n <= 850,000 rows with b for
 * m = 65536); larger problems return CW_ERR_SHAPE without launching anything.
 * The first call on each device looks up the array's device address (with
 * that device current) and caches it; make that first call before capturing
 * any stream.  All calls share the array and it keeps the previous call's
 * contents (what must start at zero is cleared by every call); calls whose
 * work can overlap on the GPU race on it and must be ordered by the caller.
 * Input errors found on the device (a column out of range, a decreasing
 * row_ptr) are kept in a separate static flag that cw_noalloc_status() reads
 * and clears; cw_device_status() does not see it.  Asynchronous.
 */
int cw_sketch_csr_noalloc(const cw_csr *A, const float *b, int64_t m, uint64_t seed, float *SA,
                          float *Sb, cw_stream stream);

/*
 * cw_noalloc_status - synchronise `stream`, then return and clear the input
 * flag that cw_sketch_csr_noalloc calls on the current device have set since
 * the last read: CW_OK, CW_ERR_DEVICE if one of them met invalid input, or
 * CW_ERR_CUDA.  Like cw_sketch_csr_noalloc it allocates nothing (the word is
 * copied into a host variable of the call), so the same callers can use it.
 * (No counterpart in the paper.)
 */
int cw_noalloc_status(cw_stream stream);

/*
 * cw_sketch_dense - SA and Sb for dense row-major A (n x d, leading dimension
 * lda >= d): the sparse embedding of Section 2 applied in O(nd) = O(nnz(A))
 * time (Theorem 1 for a dense A).  Same limits and outputs as cw_sketch_csr.
 * Asynchronous.
 */
int cw_sketch_dense(const float *A, int64_t n, int64_t d, int64_t lda, const float *b, int64_t m,
                    uint64_t seed, float *SA, float *Sb, cw_stream stream);

/* cw_sketch_vec - Sx for an n-vector x (the d = 1 case of Section 2's S A).
 * Asynchronous. */
int cw_sketch_vec(const float *x, int64_t n, int64_t m, uint64_t seed, float *Sx,
                  cw_stream stream);

/*
 * cw_gram - G = [SA | Sb]^T [SA | Sb], the Gram matrix whose Cholesky factor
 * is the R of Section 7.6's preconditioner (R^T R = (SA)^T SA).
 * SA: m x d float32 row-major (device); Sb: m float32 (device) or NULL.
 * G: (d+1) x (d+1) float64 row-major (device, caller-owned), symmetric; d x d
 * when Sb is NULL.  For d <= 256 on the tensor cores with three TF32 products
 * per pair (hi*hi + hi*lo + lo*hi), accumulated in float32 within a CTA's rows
 * and as float32 two-word sums across CTAs (fixed order: deterministic);
 * larger d on the CUDA
 * cores (float32 tiles, float64 partials).  Requires 1 <= d <= 1024, m >= 1.
 * CW_ERR_TIMEOUT if a bounded tensor-core wait gave up.  Synchronises.
 */
int cw_gram(const float *SA, int64_t m, int64_t d, const float *Sb, double *G, cw_stream stream);

/*
 * cw_qr - Householder QR of the m x d float32 matrix SA in float64 (the
 * factorisation used in the proof of Theorem "renRegAlg").
 * R: d x d row-major float64, upper triangular with a positive diagonal.
 * c: d float64, c = Q^T Sb (skipped when Sb or c is NULL).
 * Requires 1 <= d <= m, d <= 1024.  Returns CW_ERR_RANK for a numerically
 * rank-deficient SA (R still written).  Synchronises the stream.
 */
int cw_qr(const float *SA, int64_t m, int64_t d, const float *Sb, double *R, double *c,
          cw_stream stream);

/*
 * cw_solve_sketch - sketch-and-solve least squares (Theorem "lin reg"):
 * x' = argmin_x ||S A x - S b||_2 computed as R^-1 Q^T S b.
 * x: d float64 (device).  R: d x d float64 (device, upper, positive diagonal)
 * or NULL.  Requires d <= m.  Synchronises the stream.
 */
int cw_solve_sketch(const cw_csr *A, const float *b, int64_t m, uint64_t seed, double *x,
                    double *R, cw_stream stream);

/* cw_solve_sketch_dense - as cw_solve_sketch (Theorem "lin reg") for dense
 * row-major A. */
int cw_solve_sketch_dense(const float *A, int64_t n, int64_t d, int64_t lda, const float *b,
                          int64_t m, uint64_t seed, double *x, double *R, cw_stream stream);

/*
 * Training a sketch (not operations of the paper: the derivatives of its
 * sketch-and-solve, and the loss that judges it).
 *
 * cw_solve_sketched - x' = argmin ||SA x - Sb|| for an already sketched system
 * (Theorem "lin reg"), as R^-1 Q^T Sb from the float64 Householder QR of SA
 * (proof of Theorem "renRegAlg").  SA: m x d float32 row-major, Sb: m float32
 * (device).  x: d float64 (device); R: d x d float64 row-major (device) or
 * NULL.  Requires 1 <= d <= m, d <= 1024.  CW_ERR_RANK for a numerically
 * rank-deficient SA (x not written).  Synchronises.
 */
int cw_solve_sketched(const float *SA, const float *Sb, int64_t m, int64_t d, double *x, double *R,
                      cw_stream stream);

/*
 * cw_solve_sketched_backward - the gradients of a loss L(x') with respect to
 * the sketched system of cw_solve_sketched, given gx = dL/dx' (d float64,
 * device) and that call's R and x:
 *   z = R^-1 R^-T gx,  r = Sb - SA x,  gSA = r z^T - (SA z) x^T,  gSb = SA z
 * (differentiating SA^T SA x = SA^T Sb).  R may equally be cw_normal_solve's
 * factor of the same system.  gSA (m x d) and gSb (m) float32 (device), fully
 * overwritten; the row sums are float64.  Same limits as cw_solve_sketched.
 * Asynchronous.
 */
int cw_solve_sketched_backward(const float *SA, const float *Sb, int64_t m, int64_t d, const double *R,
                               const double *x, const double *gx, float *gSA, float *gSb, cw_stream stream);

/*
 * cw_normal_solve - the least-squares solution from the bordered Gram matrix
 * G = [A b]^T [A b] ((d+1) x (d+1) float64 row-major, device; what cw_gram
 * writes for A and b): the upper Cholesky factor of G is [[R, c], [0, rho]]
 * with x* = R^-1 c and rho^2 = ||A x* - b||^2.  x: d float64, r2: one
 * float64 (device); R: d x d float64 row-major, upper (R^T R = A^T A,
 * positive diagonal: the R of A's QR), or NULL.  Given cw_gram of a sketched
 * system it is the normal-equations counterpart of cw_solve_sketched.
 * CW_ERR_RANK when a pivot of A's block is not above 1e-14 of its diagonal
 * entry (outputs not written).  Requires 1 <= d <= 1024.  Synchronises.
 */
int cw_normal_solve(const double *G, int64_t d, double *x, double *r2, double *R, cw_stream stream);

/*
 * cw_excess_residual - rho^2 - 1 for rho = ||A x - b|| / ||A x* - b||:
 * loss = (x - x*)^T G_AA (x - x*) / r2 (the residual of x* is orthogonal to
 * the range of A), and gx = dloss/dx = 2 G_AA (x - x*) / r2.  G as for
 * cw_normal_solve (its leading d x d block is used), xstar and r2 from that
 * call, x: d float64.  loss: one float64; gx: d float64 or NULL (device).
 * r2 = 0 (b in the range of A) leaves the ratio undefined: loss and gx are
 * then infinite or NaN.  Requires 1 <= d <= 1024.  Asynchronous.
 */
int cw_excess_residual(const double *G, int64_t d, const double *xstar, const double *r2, const double *x,
                       double *loss, double *gx, cw_stream stream);

/*
 * cw_scale_rows - values tied per bucket: a sketch whose value at column i is
 * w_{h(i)} sigma(i) equals diag(w) S, so its sketch is the plain one with
 * row k scaled by w_k.  M[k, :] = w_k P[k, :] and y[k] = w_k Pb[k] for
 * k < ms, copied unchanged for ms <= k < m (a stacked [tied; random] sketch).
 * P, M: m x d float32 row-major; Pb, y: m float32 or both NULL; w: ms float32
 * (device).  Requires 0 <= ms <= m.  Asynchronous.
 * cw_scale_rows_backward - gw_k = <gM[k, :], P[k, :]> + gy[k] Pb[k] for
 * k < ms (float64 sums); gw: ms float32 (device), fully overwritten; Pb and
 * gy both given or both NULL.  Asynchronous.
 */
int cw_scale_rows(const float *P, const float *Pb, int64_t m, int64_t d, int64_t ms, const float *w, float *M,
                  float *y, cw_stream stream);
int cw_scale_rows_backward(const float *P, const float *Pb, int64_t ms, int64_t d, const float *gM,
                           const float *gy, float *gw, cw_stream stream);

/*
 * cw_lsqr_precond - least squares by LSQR on y -> A R^-1 y with R the
 * triangular factor of SA (R^T R = SA^T SA, the R of its QR; Section 7.6,
 * Theorem "it reg"), started at the sketch-and-solve solution, returning
 * x = R^-1 y.  R comes from a Cholesky of the Gram matrix (cw_gram's), or from
 * the float64 Householder QR of SA when that Cholesky fails or R's diagonal
 * ratio exceeds 300.
 * Stops when ||(A R^-1)^T r|| / (||A R^-1||_F ||r||) <= rtol or
 * ||r|| <= rtol (||b|| + ||A R^-1||_F ||y||) (LSQR's own estimates of the
 * norms except ||b|| and ||y||).  rtol > 0, max_iter >= 0.
 * x: d float64 (device).  iters, final_test: host (may be NULL); final_test
 * receives the last value of the first ratio.  Returns CW_ERR_NOCONV (with x
 * written) when max_iter iterations did not meet the test.  Synchronises.
 */
int cw_lsqr_precond(const cw_csr *A, const float *b, int64_t m, uint64_t seed, double rtol,
                    int32_t max_iter, double *x, int32_t *iters, double *final_test,
                    cw_stream stream);

/*
 * cw_lsqr_precond_host - cw_lsqr_precond (Section 7.6, Theorem "it reg") for A
 * and b in HOST memory: A->row_ptr, A->col, A->val, b and x are host pointers
 * (page-locked memory lets the copies run asynchronously).  The library
 * allocates the device copy, copies A in eight row chunks of about equal
 * nonzero count on a stream of its own and sketches each chunk as soon as it
 * has landed, as a row shard with its global row offset: SA = sum over the
 * chunks of S_k A_k in chunk order (Section 2's S applied block by block; the
 * float32 sums are grouped by chunk, so SA can differ from cw_sketch_csr's in
 * the last bits, deterministically).  Then the preconditioner and the LSQR
 * iterations run as in cw_lsqr_precond, and x (d float64) is copied back.
 * Requires row_ptr[0] = 0 and row_ptr[n] = nnz (CW_ERR_ARG otherwise).  Same
 * limits, statuses and stopping rule as cw_lsqr_precond.  Synchronises.
 */
int cw_lsqr_precond_host(const cw_csr *A, const float *b, int64_t m, uint64_t seed, double rtol,
                         int32_t max_iter, double *x, int32_t *iters, double *final_test,
                         cw_stream stream);

/*
 * cw_leverage - approximate leverage scores (Section 6, Theorem "icml"):
 * lev[i] = ||(A R^-1 G)_i||^2 / k, with R from the QR of SA (S with m rows
 * and `seed`) and G a d x k float64 Gaussian matrix supplied by the caller
 * (Pi_2 = G / sqrt(k)).  A: dense row-major n x d, lda >= d, d <= m.
 * lev: n floats.  Synchronises the stream.
 */
int cw_leverage(const float *A, int64_t n, int64_t d, int64_t lda, int64_t m, uint64_t seed,
                int32_t k, const double *G, float *lev, cw_stream stream);

/*
 * Measurement hooks (not part of the paper's method).
 * cw_launch_count: number of kernels this library has launched in the process.
 * cw_profile_enable: while enabled, every kernel launch of the library is
 *   bracketed by two CUDA events recorded on its launching stream.
 * cw_profile_get: launches and summed event-measured milliseconds of the named
 *   kernel (e.g. "k_lsqr_pass", "k_apply_csr") since the last reset; waits for
 *   the recorded events.  Unknown names give zero.
 * cw_profile_reset: forget all recorded durations.
 */
long long cw_launch_count(void);
int cw_profile_enable(int enable);
int cw_profile_get(const char *kernel, long long *launches, double *total_ms);
int cw_profile_reset(void);

/*
 * cw_probe_gather64 (measurement probe, not part of the paper's method): reads
 * nseg 64-byte segments of the device array a (nseg_total * 16 floats,
 * nseg_total a power of two) the way the CSR segmented sum gathers its rows
 * (16 lanes of 4 bytes per segment, 16 segments per half-warp in flight,
 * 64-byte L2 fetches), at segment indices spread over the array by a 64-bit
 * mixing function (sequential == 0) or consecutive (sequential != 0, the
 * calibration).  One launch of ctas_per_sm (1..8) CTAs of 256 threads per SM
 * on `stream`; time it with events on that stream: nseg * 64 bytes / time is
 * the segment read throughput.  out: one device float, written only if the
 * data hold a NaN.  Errors: CW_ERR_ARG (null pointer, ctas_per_sm out of
 * range), CW_ERR_SHAPE (nseg_total not a power of two, nseg < 0),
 * CW_ERR_OVERFLOW (nseg_total > 2^40), CW_ERR_CUDA.
 */
int cw_probe_gather64(const float *a, int64_t nseg_total, int64_t nseg, int sequential, int ctas_per_sm,
                      float *out, cw_stream stream);

#ifdef __cplusplus
}
#endif

#endif /* CW_H */
