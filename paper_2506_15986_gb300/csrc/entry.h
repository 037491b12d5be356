// entry.h -- learned entry model held by an index, and the launchers shared by
// entry selection (entry.cu) and training (train.cu).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"
#include "tc.cuh"

struct ann_entry_model {
    int in_dim = 0;  // query dimension (= index dim)
    int H = 0;       // number of hubs
    int s = 0;       // hub-graph degree
    float *W1 = nullptr, *b1 = nullptr, *W2 = nullptr, *b2 = nullptr;  // fp32 masters
    float *E = nullptr;                      // raw hub embeddings [H][64]
    float *En = nullptr;                     // normalised [H][64]
    __nv_bfloat16 *W1t = nullptr;            // [256][in_dim]
    __nv_bfloat16 *W2t = nullptr;            // [64][256]
    __nv_bfloat16 *Eb = nullptr;             // normalised, BF16 [H][64]
    // index models only: the operands of the exhaustive entry kernel as the
    // 32 KB canonical shared-memory images its bulk copies load (W1 in
    // 64-wide k chunks, then W2, then the hubs in tiles of 256 rows)
    uint8_t *packed = nullptr;
    int32_t *hub_nodes = nullptr;            // [H] node ids
    int32_t *hub_graph = nullptr;            // [H][s]
    int32_t hub_entry = 0;
    // the hubs the hub-graph search starts from (Algorithm 1's initial node
    // set), device [ANN_MAX_SEEDS]: the caller's sample (n_hub_seeds > 0) or,
    // with n_hub_seeds = 0, hub_entry alone in slot 0
    int32_t *hub_seeds = nullptr;
    int n_hub_seeds = 0;
    ann_index *hub_index = nullptr;          // BF16 / IP index over Eb and hub_graph
};

namespace ann {

void free_model(ann_entry_model *m);
// Bytes of the packed operand images of a model (32 KB per image).
size_t packed_model_bytes(int in_dim, int H);
// BF16 copies of the weights and normalised hub embeddings, and, when
// m->packed is allocated, the packed operand images (stream-ordered).
ann_status prepare_model(ann_entry_model *m, cudaStream_t s);
ann_status build_hub_index(ann_index *idx, ann_entry_model *m, const int32_t *hub_graph, int32_t hub_entry,
                           cudaStream_t s);
ann_status launch_tower(const ann_entry_model *m, const Operand &X, int64_t nq, float *qhat,
                        __nv_bfloat16 *qhat_bf, float *z1, __nv_bfloat16 *a1, float *nrm, int *status,
                        cudaStream_t s);
// Exhaustive entry selection in one kernel: the query tower, every hub's
// score and the topm (1..8) best hubs' nodes per query (nq x topm, best
// first); qhat (optional) receives the fp32 query embeddings.
ann_status launch_entry_exhaustive(const ann_entry_model *m, const Operand &X, int64_t nq, float *qhat,
                                   int32_t *out_node, int topm, int *status, cudaStream_t s);
// Exhaustive hub scoring: the topm (1..8) best hubs per query, nq x topm
// outputs, best first.
ann_status launch_hub_argmax(const ann_entry_model *m, const Operand &Q, int64_t nq, int32_t *out_node,
                             int32_t *out_hub, float *out_score, int *status, cudaStream_t s, int topm = 1);

}  // namespace ann
