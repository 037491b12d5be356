// fusion.h -- the fusion embedding of Sec. 4.3 (Module I, Eq. fusion) for the
// topology-aware hub tower: per hub, heads attention heads of width dk,
//     F = Concat_j softmax((p WQ_j)(U WK_j)^T / sqrt(dk)) (U WV_j)  WO
// with p the hub's vector (dp) and U its T topology tokens (dU each); the
// hub row the two-tower model scores is E + F.  Forward, backward and the
// weights' gradients (summed over hubs in hub order) run in fp32.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"

namespace ann {

struct Fusion {
    int H = 0, T = 0, dU = 0, heads = 0, dk = 0, E = 0, dp = 0, dF = 64;
    float *P = nullptr, *U = nullptr;  // hub vectors [H][dp], tokens [H][T][dU]
    int64_t n_params = 0;              // WQ [dp][E] | WK [dU][E] | WV [dU][E] | WO [E][dF]
    float *params = nullptr, *grads = nullptr, *m = nullptr, *v = nullptr;
    float *Q = nullptr, *K = nullptr, *V = nullptr, *A = nullptr, *O = nullptr;  // forward cache
    float *dQ = nullptr, *dK = nullptr, *dV = nullptr;
    float *F = nullptr, *Eeff = nullptr;  // [H][dF]
    int64_t oWQ() const { return 0; }
    int64_t oWK() const { return static_cast<int64_t>(dp) * E; }
    int64_t oWV() const { return oWK() + static_cast<int64_t>(dU) * E; }
    int64_t oWO() const { return oWV() + static_cast<int64_t>(dU) * E; }
};

// allocates every buffer; weights (host or device) copied in; nullptr on failure
Fusion *fusion_create(int H, int T, int dU, int heads, int dk, int dp, const float *P, const float *U,
                      const float *WQ, const float *WK, const float *WV, const float *WO, cudaError_t &e);
void fusion_free(Fusion *f);
// F from the current weights, then Eeff = E + F
ann_status fusion_forward(Fusion *f, const float *E, cudaStream_t s);
// weights' gradients from dL/dF (= dL/dEeff), written to f->grads
ann_status fusion_backward(Fusion *f, const float *dF, cudaStream_t s);

}  // namespace ann
