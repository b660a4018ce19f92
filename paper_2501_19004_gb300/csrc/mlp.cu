// Learned vertex-activity predictor (placeholder until the MLP kernels land).
#include "internal.h"

namespace lv {

// 8 -> 32 -> 32 -> 1 MLP: W1[32][8], b1[32], W2[32][32], b2[32], w3[32], b3.
int64_t mlp_param_count() { return 32 * 8 + 32 + 32 * 32 + 32 + 32 + 1; }

void mlp_features_init(float *, int64_t, int, cudaStream_t) {}

}  // namespace lv
