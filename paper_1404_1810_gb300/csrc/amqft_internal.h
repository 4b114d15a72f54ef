// Internal declarations shared by the kernel translation units and the C ABI.
#pragma once

#include <cuda_runtime.h>

namespace amqft {

struct FusedArgs;
struct SmallConsts;

// Launch shape of the fused kernel for one transform length.
struct FusedConfig {
  int cluster;  // CTAs per transform (1: a CTA holds per_cta whole transforms)
  int per_cta;  // transforms per CTA (cluster == 1)
  int threads;  // threads per CTA
  int smem;     // dynamic shared memory bytes per CTA
  int RS;       // region stride (floats)
  int nreg;     // regions per CTA
  int tot_off;  // float offset of the scan scratch
};

FusedConfig fused_config(int logN);

cudaError_t launch_variant_1(const FusedArgs&, const SmallConsts&, const FusedConfig&, cudaStream_t);
cudaError_t launch_variant_2(const FusedArgs&, const SmallConsts&, const FusedConfig&, cudaStream_t);
cudaError_t launch_variant_3(const FusedArgs&, const SmallConsts&, const FusedConfig&, cudaStream_t);
cudaError_t launch_variant_4(const FusedArgs&, const SmallConsts&, const FusedConfig&, cudaStream_t);
cudaError_t launch_variant_5(const FusedArgs&, const SmallConsts&, const FusedConfig&, cudaStream_t);
cudaError_t launch_variant_6(const FusedArgs&, const SmallConsts&, const FusedConfig&, cudaStream_t);
cudaError_t launch_variant_7(const FusedArgs&, const SmallConsts&, const FusedConfig&, cudaStream_t);
cudaError_t launch_variant_8(const FusedArgs&, const SmallConsts&, const FusedConfig&, cudaStream_t);

}  // namespace amqft
