// Fused AM-QFT kernels of variant 3 (instantiated in a translation unit of
// their own so the eight variants compile in parallel).
#include "amqft_ragged_impl.cuh"

namespace amqft {
cudaError_t launch_variant_3(const FusedArgs& a, const SmallConsts& K, const FusedConfig& c, cudaStream_t st) {
  return launch_v<3>(a, K, c, st);
}
cudaError_t multipass_variant_3(const MpArgs& a, float* W0, float* W1, const SmallConsts& K, cudaStream_t st,
                                long long* nlaunch) {
  return mp_run<3>(a, W0, W1, K, st, nlaunch);
}
cudaError_t ragged_variant_3(const FusedArgs& a, const SmallConsts& K, const RaggedArgs& r, const RaggedLaunch& L,
                               cudaStream_t st, long long* nlaunch) {
  return ragged_run<3>(a, K, r, L, st, nlaunch);
}
AMQFT_BOUNDS_READER(bounds_v3)
}  // namespace amqft
