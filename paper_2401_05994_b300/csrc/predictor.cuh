// Tolerance predictor and ratio-targeted compression (declarations).
#pragma once

#include "pipeline.cuh"

namespace mgb {

// y [B] = network(x [B, MGARD_NFEAT]) (mlp.cu).
mgard_status mlp_forward(const float* params, const float* x, int B, float* y, cudaStream_t st);

}  // namespace mgb
