// Internal structures of the batched sketch-and-solve (many independent
// regressions in one graph launch).  Shared by sketch.cu (the batched sketch
// kernels) and batch.cu (plan, solve kernels, C ABI).
#pragma once

#include <vector>

#include "cw_common.cuh"
#include "cw_internal.h"

namespace cw {

// One problem as the caller gives it (device pointers).
struct BatchSpec {
    int64_t n, d, nnz, m;
    uint64_t seed;
    const int32_t* row_ptr;
    const int32_t* col;
    const float* val;
    const float* b;
    float* SA;   // m x d output (caller's or internal)
    float* Sb;   // m output
};

// Device descriptor of one problem of the batched sketch.  Offsets are in
// elements of the shared scratch arrays.
struct BatchProb {
    HashParams hp;
    int64_t n;
    int32_t d, m;
    int32_t gshift, nbins, ntiles, nchunks;
    int32_t tile0, chunk0, bin0;  // first global tile, scan chunk and coarse bin
    int32_t vec4;                 // SA rows 16-byte aligned and d % 4 == 0
    int32_t skip_empty;           // SA / Sb plan-owned: rows of empty buckets are not written
    int64_t H0, P0, CP0;          // tile histograms, chunk sums, coarse bin starts
    int64_t rec0;                 // first row of the problem in rec / r2 / rb
    int64_t bp0;                  // bucket_ptr base (m + 1 entries per problem)
    int64_t bk0;                  // first global bucket (the apply kernel's queue)
    const int32_t* row_ptr;
    const int32_t* col;
    const float* val;
    const float* b;
    float* SA;
    float* Sb;
};

// Everything the batched sketch kernels read: descriptors, block -> problem
// tables, scratch arrays and batch-wide launch shapes.
struct BatchSketch {
    const BatchProb* probs;
    int32_t count;
    const int32_t* tile_prob;   // [total_tiles]
    const int32_t* chunk_prob;  // [total_chunks]
    const int32_t* bin_prob;    // [total_bins]
    const int64_t* bk_base;     // [count + 1], prefix sums of m
    int32_t total_tiles, total_chunks, total_bins, bin_groups, max_nbins;
    int64_t total_buckets;
    uint32_t* H;
    uint32_t* P;
    uint32_t* CP;
    int4* rec;
    int2* r2;
    float* rb;
    int32_t* bptr;
    unsigned* counter;  // apply queue, zeroed by the enqueue
    unsigned* status;
    int32_t lpr, dpad, acc_global;
    size_t acc_smem;
    int32_t apply_grid;
};

// Host side of the plan: sizes of the scratch arrays and the tables.
struct BatchSketchHost {
    std::vector<BatchProb> probs;
    std::vector<int32_t> tile_prob, chunk_prob, bin_prob;
    std::vector<int64_t> bk_base;
    int64_t H_elems = 0, P_elems = 0, CP_elems = 0, rows = 0, bptr_elems = 0;
};

// Fills `host` (descriptors with offsets, tables) and the shapes in `dev`
// for the given problems; pointers of `dev` are set by the caller.
int batch_sketch_plan(const BatchSpec* specs, int count, BatchSketchHost* host, BatchSketch* dev);
// Segmented-sum variant: lanes per CSR row (16: two rows at a time and two
// accumulator copies; 32: one row, one copy), or 0 / -8: whole 16- / 8-bucket
// ranges at a time (one accumulator row per bucket); sets the launch shape.
int batch_sketch_set_lpr(BatchSketch* dev, int lpr);
// Enqueues the batched sketch (8 launches; capturable).
int batch_sketch_enqueue(const BatchSketch& B, cudaStream_t stream);

}  // namespace cw
