// Internal declarations shared by the kernel translation units and the C ABI.
#pragma once

#include <cuda_runtime.h>

#include "amqft.h"

namespace amqft {

struct FusedArgs;
struct SmallConsts;
struct MpArgs;
struct RaggedArgs;
struct RaggedLaunch;

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

FusedConfig fused_config(int logN, int variant);

cudaError_t launch_variant_1(const FusedArgs&, const SmallConsts&, const FusedConfig&, cudaStream_t);
cudaError_t launch_variant_2(const FusedArgs&, const SmallConsts&, const FusedConfig&, cudaStream_t);
cudaError_t launch_variant_3(const FusedArgs&, const SmallConsts&, const FusedConfig&, cudaStream_t);
cudaError_t launch_variant_4(const FusedArgs&, const SmallConsts&, const FusedConfig&, cudaStream_t);
cudaError_t launch_variant_5(const FusedArgs&, const SmallConsts&, const FusedConfig&, cudaStream_t);
cudaError_t launch_variant_6(const FusedArgs&, const SmallConsts&, const FusedConfig&, cudaStream_t);
cudaError_t launch_variant_7(const FusedArgs&, const SmallConsts&, const FusedConfig&, cudaStream_t);
cudaError_t launch_variant_8(const FusedArgs&, const SmallConsts&, const FusedConfig&, cudaStream_t);

// ragged batches (every length up to the plan's), all variants; the ragged and
// multi-pass sequences add the kernels they launch to *nlaunch (may be NULL)
cudaError_t ragged_variant_1(const FusedArgs&, const SmallConsts&, const RaggedArgs&, const RaggedLaunch&, cudaStream_t,
                             long long* nlaunch);
cudaError_t ragged_variant_2(const FusedArgs&, const SmallConsts&, const RaggedArgs&, const RaggedLaunch&, cudaStream_t,
                             long long* nlaunch);
cudaError_t ragged_variant_3(const FusedArgs&, const SmallConsts&, const RaggedArgs&, const RaggedLaunch&, cudaStream_t,
                             long long* nlaunch);
cudaError_t ragged_variant_4(const FusedArgs&, const SmallConsts&, const RaggedArgs&, const RaggedLaunch&, cudaStream_t,
                             long long* nlaunch);
cudaError_t ragged_variant_5(const FusedArgs&, const SmallConsts&, const RaggedArgs&, const RaggedLaunch&, cudaStream_t,
                             long long* nlaunch);
cudaError_t ragged_variant_6(const FusedArgs&, const SmallConsts&, const RaggedArgs&, const RaggedLaunch&, cudaStream_t,
                             long long* nlaunch);
cudaError_t ragged_variant_7(const FusedArgs&, const SmallConsts&, const RaggedArgs&, const RaggedLaunch&, cudaStream_t,
                             long long* nlaunch);
cudaError_t ragged_variant_8(const FusedArgs&, const SmallConsts&, const RaggedArgs&, const RaggedLaunch&, cudaStream_t,
                             long long* nlaunch);

// multi-pass path (2^17 <= N <= 2^24), every variant
cudaError_t multipass_variant_1(const MpArgs&, float*, float*, const SmallConsts&, cudaStream_t, long long* nlaunch);
cudaError_t multipass_variant_2(const MpArgs&, float*, float*, const SmallConsts&, cudaStream_t, long long* nlaunch);
cudaError_t multipass_variant_3(const MpArgs&, float*, float*, const SmallConsts&, cudaStream_t, long long* nlaunch);
cudaError_t multipass_variant_4(const MpArgs&, float*, float*, const SmallConsts&, cudaStream_t, long long* nlaunch);
cudaError_t multipass_variant_5(const MpArgs&, float*, float*, const SmallConsts&, cudaStream_t, long long* nlaunch);
cudaError_t multipass_variant_6(const MpArgs&, float*, float*, const SmallConsts&, cudaStream_t, long long* nlaunch);
cudaError_t multipass_variant_7(const MpArgs&, float*, float*, const SmallConsts&, cudaStream_t, long long* nlaunch);
cudaError_t multipass_variant_8(const MpArgs&, float*, float*, const SmallConsts&, cudaStream_t, long long* nlaunch);
// the whole multi-pass sequence of one chunk for `variant` (W0, W1: the two
// workspace buffers; nlaunch counts the kernels launched)
cudaError_t multipass_dispatch(int variant, const MpArgs& a, float* W0, float* W1, const SmallConsts& K,
                               cudaStream_t st, long long* nlaunch);

// bounds-checked build: each translation unit's failure count and first
// failure (amqft_debug.cuh), read and optionally cleared
#define AMQFT_BOUNDS_DECL(name) cudaError_t name(unsigned long long* count, unsigned long long* first, bool clear);
AMQFT_BOUNDS_DECL(bounds_v1)
AMQFT_BOUNDS_DECL(bounds_v2)
AMQFT_BOUNDS_DECL(bounds_v3)
AMQFT_BOUNDS_DECL(bounds_v4)
AMQFT_BOUNDS_DECL(bounds_v5)
AMQFT_BOUNDS_DECL(bounds_v6)
AMQFT_BOUNDS_DECL(bounds_v7)
AMQFT_BOUNDS_DECL(bounds_v8)
AMQFT_BOUNDS_DECL(bounds_p14)
AMQFT_BOUNDS_DECL(bounds_p15)
AMQFT_BOUNDS_DECL(bounds_p16)
#undef AMQFT_BOUNDS_DECL

// paired-region kernel (N = 2^14 .. 2^16, variant 4, complex64 or 16-bit
// storage, batch below 2^31): one transform per cluster of four CTAs,
// persistent over the batch; in and out 16-byte (16-bit: 8-byte) aligned
bool paired_supported(int logN, int variant, int dtype, long long batch);
// tlist / toff / tcount (all NULL: transforms 0 .. batch-1 in order): the
// ragged form, list entries t < min(*tcount, batch) at element toff[tlist[t]]
// (each 16-byte aligned)
cudaError_t paired_launch(int logN, const void* in, void* out, const int* exp_in, int* exp_out, int dtype,
                          long long batch, int inverse, const float* ctab, const SmallConsts& K, cudaStream_t st,
                          const int* tlist = nullptr, const long long* toff = nullptr, const int* tcount = nullptr);
cudaError_t paired_launch_14(const void*, void*, const int*, int*, int, long long, int, const float*, const SmallConsts&,
                             cudaStream_t, const int*, const long long*, const int*);
cudaError_t paired_launch_15(const void*, void*, const int*, int*, int, long long, int, const float*, const SmallConsts&,
                             cudaStream_t, const int*, const long long*, const int*);
cudaError_t paired_launch_16(const void*, void*, const int*, int*, int, long long, int, const float*, const SmallConsts&,
                             cudaStream_t, const int*, const long long*, const int*);

// Read-only view of a plan, for entry points defined outside the plan's
// translation unit.  Returns AMQFT_ERR_ARG for a NULL plan.
struct PlanView {
  int log2n;
  int variant;
  int dtype;
  int device;                // device the plan's constant table lives on
  const float* ctab;         // device constant table (NULL for N < 16)
  const SmallConsts* small;  // host copy of the leaf constants
};
int plan_view(amqft_plan_t plan, PlanView* v);

// Add n to the plan's count of launched kernels (amqft_plan_launches).
void add_launches(amqft_plan_t plan, long long n);

// Record the calling thread's error message (amqft_last_error) and return code.
int set_error(int code, const char* fmt, ...);
void clear_error();

}  // namespace amqft
