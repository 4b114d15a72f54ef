// Paired-region kernels for N = 2^15 (own translation unit: parallel build).
#include "amqft_paired_impl.cuh"

namespace amqft {
cudaError_t paired_launch_15(const void* in, void* out, const int* exp_in, int* exp_out, int dtype, long long batch,
                               int inverse, const float* ctab, const SmallConsts& K, cudaStream_t st,
                               const int* tlist, const long long* toff, const int* tcount) {
  return pr::launch_len<15>(in, out, exp_in, exp_out, dtype, batch, inverse, ctab, K, st, tlist, toff, tcount);
}
AMQFT_BOUNDS_READER(bounds_p15)
}  // namespace amqft
