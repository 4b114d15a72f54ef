// Dispatch of the paired-region kernel (amqft_paired.cuh): batched transforms
// of 2^14 .. 2^16 points, variant 4, complex64 or 16-bit storage.
#include "amqft_internal.h"

namespace amqft {

bool paired_supported(int logN, int variant, int dtype, long long batch) {
  return variant == 4 && dtype >= AMQFT_C64 && dtype <= AMQFT_CI16 && logN >= 14 && logN <= 16 &&
         batch <= 0x7fffffffLL;
}

cudaError_t paired_launch(int logN, const void* in, void* out, const int* exp_in, int* exp_out, int dtype,
                          long long batch, int inverse, const float* ctab, const SmallConsts& K, cudaStream_t st,
                          const int* tlist, const long long* toff, const int* tcount) {
  switch (logN) {
    case 14: return paired_launch_14(in, out, exp_in, exp_out, dtype, batch, inverse, ctab, K, st, tlist, toff, tcount);
    case 15: return paired_launch_15(in, out, exp_in, exp_out, dtype, batch, inverse, ctab, K, st, tlist, toff, tcount);
    case 16: return paired_launch_16(in, out, exp_in, exp_out, dtype, batch, inverse, ctab, K, st, tlist, toff, tcount);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace amqft
