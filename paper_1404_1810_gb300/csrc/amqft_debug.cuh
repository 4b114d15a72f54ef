// Bounds-checked build (compile flag AMQFT_BOUNDS_CHECK; the debug library,
// built by build.build(debug=True)).  A checked access whose index falls
// outside its buffer is skipped: a store is dropped, a load returns a
// scratch word, and the failure is recorded in a device word of the
// translation unit (count, and the first failure's site and index), which the
// host reads with amqft_debug_bounds.  Nothing traps and no wait is added, so
// a kernel with a bad index finishes normally and the context stays usable.
//
// Checked: every access to a transform region (shared memory, distributed
// shared memory of the cluster kernels, the multi-pass workspace) through
// RegP / CRegP against the region's stride, the paired kernel's region and
// HBM accesses, and the HBM element indices of the loads and stores against
// the transform length.  In the release build RegP is a plain pointer and the
// checks compile to nothing.
#pragma once

#include <cuda_runtime.h>

namespace amqft {

// sites (the high 16 bits of the recorded first failure)
enum BoundsSite {
  BS_REGION = 1,   // a region word (shared, distributed shared or workspace)
  BS_HBM_IN = 2,   // an input element of a transform
  BS_HBM_OUT = 3,  // an output element of a transform
  BS_PAIRED_REG = 4,
  BS_PAIRED_HBM = 5,
};

#ifdef AMQFT_BOUNDS_CHECK

// [0] failures, [1] the first one: site << 48 | (index & 2^48 - 1)
static __device__ unsigned long long g_bounds[2];
static __device__ float g_sink[4];

__device__ __noinline__ static void bounds_fail(int site, long long idx) {
  const unsigned long long v = ((unsigned long long)(site & 0xffff) << 48) | ((unsigned long long)idx & 0xffffffffffffULL);
  if (atomicAdd(&g_bounds[0], 1ULL) == 0ULL) g_bounds[1] = v;
}

__device__ __forceinline__ bool in_bounds(long long i, long long n, int site) {
  if (i >= 0 && i < n) return true;
  bounds_fail(site, i);
  return false;
}

template <class T>
struct Chk {
  T* p;
  int n;
  __device__ __forceinline__ Chk() : p(nullptr), n(0) {}
  __device__ __forceinline__ Chk(T* q, int m) : p(q), n(m) {}
  template <class U>
  __device__ __forceinline__ Chk(const Chk<U>& o) : p(o.p), n(o.n) {}
  __device__ __forceinline__ T& operator[](int i) const {
    if (i >= 0 && i < n) return p[i];
    bounds_fail(BS_REGION, i);
    return *reinterpret_cast<T*>(g_sink);
  }
};
using RegP = Chk<float>;
using CRegP = Chk<const float>;
__device__ __forceinline__ RegP reg_ptr(float* p, int n) { return RegP(p, n); }
__device__ __forceinline__ CRegP creg_ptr(const float* p, int n) { return CRegP(p, n); }
#define AMQFT_IN_BOUNDS(i, n, site) ::amqft::in_bounds((long long)(i), (long long)(n), (site))

// host side: read (and clear) this translation unit's word
#define AMQFT_BOUNDS_READER(name)                                                          \
  cudaError_t name(unsigned long long* count, unsigned long long* first, bool clear) {      \
    unsigned long long h[2] = {0, 0};                                                      \
    cudaError_t e = cudaMemcpyFromSymbol(h, g_bounds, sizeof h);                           \
    if (e != cudaSuccess) return e;                                                        \
    *count = h[0];                                                                         \
    *first = h[1];                                                                         \
    if (clear) {                                                                           \
      const unsigned long long z[2] = {0, 0};                                              \
      e = cudaMemcpyToSymbol(g_bounds, z, sizeof z);                                       \
    }                                                                                      \
    return e;                                                                              \
  }

#else

using RegP = float*;
using CRegP = const float*;
__device__ __forceinline__ float* reg_ptr(float* p, int) { return p; }
__device__ __forceinline__ const float* creg_ptr(const float* p, int) { return p; }
#define AMQFT_IN_BOUNDS(i, n, site) true
#define AMQFT_BOUNDS_READER(name)                                                     \
  cudaError_t name(unsigned long long* count, unsigned long long* first, bool) {      \
    *count = 0;                                                                       \
    *first = 0;                                                                       \
    return cudaSuccess;                                                               \
  }

#endif

}  // namespace amqft
