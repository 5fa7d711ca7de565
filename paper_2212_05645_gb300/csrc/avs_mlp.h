// Learned adaptation proposer: launchers shared with the API translation unit.
#pragma once

#include <cuda_runtime.h>

#define AVS_MLP_NPARAM 4996     // W1[64][8], b1[64], W2[64][64], b2[64], W3[4][64], b3[4]
#define AVS_MLP_MAXBLK 304      // blocks of the gradient kernel (partial sums)
#define AVS_MLP_BF16_ELEMS (64 * 16 + 64 * 64 + 8 * 64 + 64 * 64 + 64 * 8)

struct avs_ctx;

namespace avs {
cudaError_t mlp_prep(avs_ctx* c);
cudaError_t mlp_forward(avs_ctx* c, int n, const float* X, float* logits);
cudaError_t mlp_grad_step(avs_ctx* c, int n, const float* X, const float* Y, float lr, float* grad_out);
cudaError_t mlp_features(avs_ctx* c, const double* Wc, const double* q, float* X);
cudaError_t mlp_labels(avs_ctx* c, const void* f, float* Y);
cudaError_t mlp_checkset(avs_ctx* c, const float* logits, float zthr, int* list, int* count);
cudaError_t mlp_misses(avs_ctx* c, const double* Mf, const double* Ms, int* count);
// threshold of the check set: keeps the top `budget` fraction of cells by dominant logit
cudaError_t mlp_calibrate(avs_ctx* c, float budget);
}  // namespace avs
