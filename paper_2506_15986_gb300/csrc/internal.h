// internal.h -- host-side index object and kernel launchers of libann.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/ann.h"

struct ann_entry_model;  // learned entry selection (entry.cu)

struct ann_index {
    int device = 0;
    int num_sms = 0;
    int64_t n = 0;
    int32_t dim = 0;
    int32_t degree = 0;
    int32_t dtype = ANN_F32;
    int32_t metric = ANN_L2;
    int32_t medoid = 0;
    int32_t rowbytes = 0;  // bytes of one stored base row
    void *d_base = nullptr;
    int32_t *d_graph = nullptr;
    float *d_base_f32 = nullptr;  // optional exact copy for rerank
    int *d_status = nullptr;      // device status word (kStatus* bits)
    int *status_sink = nullptr;   // if set, kernels report here instead (hub index -> its parent)
    cudaMemPool_t pool = nullptr; // stream-ordered scratch
    ann_entry_model *model = nullptr;
    // 2-D tensor map over the base rows (4-byte elements, one row per box)
    // for TMA tensor gathers of four rows; valid when has_row_map
    CUtensorMap row_map;
    int has_row_map = 0;
};

namespace ann {

// device status bits, OR-ed into the index's status word by kernels
constexpr int kStatusCapacityBit = 1;
constexpr int kStatusTimeoutBit = 2;
constexpr int kStatusBadInputBit = 4;

int elem_size(int dtype);
// bytes of one stored base row (0 for an unknown dtype or dim < 1)
int64_t row_bytes(int dtype, int dim);

// status helpers
ann_status cuda_status(cudaError_t e);

// Scratch from the index's stream-ordered pool.
ann_status scratch_alloc(ann_index *idx, size_t bytes, cudaStream_t s, void **out);
void scratch_free(ann_index *idx, void *p, cudaStream_t s);

struct SearchLaunch {
    const void *queries;
    int qbytes;  // bytes of one query row
    int64_t nq;
    const int32_t *entries;  // nullptr = medoid
    const ann_search_params *p;
    int32_t *ids;
    void *dists;
    int32_t *stats;
    // optional caller-provided scratch: work counter (8 bytes) + spill tables
    void *scratch;
    size_t scratch_bytes;
    int max_teams;  // cap on the persistent grid (0 = occupancy-limited only)
    int64_t qdiv;   // work item i uses query row and target i / qdiv (0 = 1)
    int n_entries;  // seeds per work item in entries[] (0 = 1)
};

// Queues the beam-search kernel (search.cu).
ann_status launch_search(ann_index *idx, const SearchLaunch &L, cudaStream_t s);

// Lanes per distance when ann_search_params.team is 0: the smallest power of
// two >= 4 that leaves each lane at most four 16-byte chunks of a row.
int default_team(int rowbytes);

// log2 slots of the first global visited table when ann_search_params.
// spill_bits is 0: 40 evaluations per pool slot below 3/4 load, 12..15.
int default_spill_bits(int L);

// Scratch bytes launch_search needs for `teams` teams at the given params
// (order_items: work items of a grouped work order, 0 without one).
size_t search_scratch_bytes(int teams, int spill_bits, int64_t order_items);

// Exact k-NN (build.cu): candidates from an fp32 GEMM, exact re-scoring.
ann_status knn_exact(const void *d_base, int64_t n, int dim, int dtype, int metric, const void *d_queries,
                     int64_t nq, int k, bool exclude_self, int32_t *d_ids, void *d_dists, cudaStream_t s);

}  // namespace ann
