// Trig constants of the tree levels (Sect. 7.1) as the kernels read them.
//
// Constant j in [0, M/8) of periodisation M (a power of two >= 16) is
// f(phi), phi = 2*pi*(2j+1)/M in (0, pi/2), with f = 2cos (variants 1, 3),
// 1/(2cos) (2, 4), 2sin (5, 7) or 1/(2sin) (6, 8).  The plan's table holds
// them level-major (M at [M/8 - 2, M/4 - 2)), rounded once from long double.
// The register leaves (M <= 128, table indices 0..29) take theirs as kernel
// arguments in every mode; the band levels (M >= 256, index >= 30) read one
// of these sources:
//
//  * TabConsts: a copy of the table from index 30 on, staged per CTA in
//    shared memory by the single-pass kernels (or the plan's table itself in
//    global memory, for the multi-pass levels above 2^13);
//  * fly_const: the "on the fly" mode, evaluated in float32 where it is
//    needed.  phi = pi * p / q with p = 2j+1 and q = M/2 is folded into
//    [0, pi/4] with integer arithmetic (cos(pi/2 - x) = sin(x)), so the
//    argument of cospif / sinpif is p'/q with p' <= q/4: exact in float32 for
//    M <= 2^26 (p' < 2^24), rounded to 24 bits above.
#pragma once

#include <cuda_runtime.h>

namespace amqft {

template <int V>
__device__ __forceinline__ float fly_const(int logM, int j) {
  const int q = 1 << (logM - 1), p = 2 * j + 1;
  const bool fold = 4 * p > q;
  const int num = fold ? (q >> 1) - p : p;
  const float t = __int2float_rn(num) * __int_as_float((127 - (logM - 1)) << 23);  // num / q, q a power of two
  float f;  // cos(phi) for variants 1-4, sin(phi) for 5-8
  if constexpr (V <= 4) f = fold ? sinpif(t) : cospif(t);
  else f = fold ? cospif(t) : sinpif(t);
  if constexpr (V == 1 || V == 3 || V == 5 || V == 7) return 2.0f * f;
  else return 1.0f / (2.0f * f);
}

// table index g (>= 0) -> the constant it holds, on the fly
template <int V>
__device__ __forceinline__ float fly_entry(int g) {
  const int lm8 = 31 - __clz(g + 2);  // log2(M/8)
  return fly_const<V>(lm8 + 3, g + 2 - (1 << lm8));
}

// Constant source of the band levels: node size Ln (= M/4) and index j.
struct TabConsts {
  const float* p;  // table entry 30 (M = 256, j = 0)
  __device__ __forceinline__ float operator()(int Ln, int j) const { return p[(Ln >> 1) - 32 + j]; }
};

template <int V>
struct FlyConsts {
  __device__ __forceinline__ float operator()(int Ln, int j) const { return fly_const<V>(33 - __clz(Ln), j); }
};

// Fill dst[0 .. n) with table entries 30 .. 30 + n: copied from the plan's
// table, or evaluated on the fly when ctab is NULL.  Threads tid, tid + nth, ...
template <int V>
__device__ __forceinline__ void stage_consts(float* dst, int n, const float* __restrict__ ctab, int tid, int nth) {
  if (ctab) {
    for (int i = tid; i < n; i += nth) dst[i] = __ldg(ctab + 30 + i);
  } else {
    for (int i = tid; i < n; i += nth) dst[i] = fly_entry<V>(30 + i);
  }
}

}  // namespace amqft
