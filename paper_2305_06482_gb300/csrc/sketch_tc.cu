// Tensor-core split-precision contraction for the sketched maps (Eq. 8, random block):
//   maps_s[s][d] = sum_j S~_S[s][j] maps_rot[V + j][d].
#include "cs_internal.cuh"

namespace cs {

cs_status sketched_maps_bf16split(const float* S, const float2* mrot, int64_t D, int C, int V, int Sn, float2* out,
                                  cudaStream_t st) {
    (void)S; (void)mrot; (void)D; (void)C; (void)V; (void)Sn; (void)out; (void)st;
    set_error("CS_PREC_BF16_SPLIT is not available in this build");
    return CS_ERR_UNSUPPORTED_SIZE;
}

}  // namespace cs
