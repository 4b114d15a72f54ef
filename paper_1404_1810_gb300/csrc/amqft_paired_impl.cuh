// Device side of the paired-region kernel (amqft_paired.cuh): the kernel,
// its synchronisation and HBM accesses, and the persistent cluster launch.
// Instantiated per transform length in amqft_paired_l{14,15,16}.cu.
#pragma once
#include "amqft_internal.h"
#include "amqft_consts.cuh"
#include "amqft_device.cuh"
#include "amqft_paired.cuh"

namespace amqft {
namespace pr {

struct DevCtx {
  int tid, rank;
  unsigned lbase;  // shared-window address of this CTA's region
#ifdef AMQFT_BOUNDS_CHECK
  // bounds of the checked build: region float2 words, and the batch in HBM
  // (gn elements of es bytes)
  int rf, es;
  const char* gin;
  const char* gout;
  long long gn;
  __device__ __forceinline__ bool reg_ok(int i, int w) const { return AMQFT_IN_BOUNDS(i, rf - (w - 1), BS_PAIRED_REG); }
  __device__ __forceinline__ bool hbm_ok(const void* p, const char* base, int w) const {
    return AMQFT_IN_BOUNDS((static_cast<const char*>(p) - base) / es, gn - (w - 1), BS_PAIRED_HBM);
  }
#define PAIRED_CHECK(cond, fallback) \
  if (!(cond)) return fallback
#else
#define PAIRED_CHECK(cond, fallback)
#endif
  // shared::cluster address of CTA q's region (mapa, recomputed at each use
  // rather than held in four registers through the whole transform)
  __device__ __forceinline__ unsigned cbase(int q) const {
    unsigned a;
    asm("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(a) : "r"(lbase), "r"(q));
    return a;
  }
  __device__ __forceinline__ void sync_warp() { __syncwarp(); }
  __device__ __forceinline__ void sync_cta() { __syncthreads(); }
  __device__ __forceinline__ void sync_cluster() { cg::this_cluster().sync(); }
  __device__ __forceinline__ float4 ldg4(const float2* p) {
    PAIRED_CHECK(hbm_ok(p, gin, 2), make_float4(0.f, 0.f, 0.f, 0.f));
    return __ldcs(reinterpret_cast<const float4*>(p));
  }
  __device__ __forceinline__ float2 ldg2(const float2* p) {
    PAIRED_CHECK(hbm_ok(p, gin, 1), make_float2(0.f, 0.f));
    return __ldcs(p);
  }
  __device__ __forceinline__ void stg4(float2* p, float4 v) {
    PAIRED_CHECK(hbm_ok(p, gout, 2), );
    __stcs(reinterpret_cast<float4*>(p), v);
  }
  __device__ __forceinline__ void stg2(float2* p, float2 v) {
    PAIRED_CHECK(hbm_ok(p, gout, 1), );
    __stcs(p, v);
  }
  // 16-bit storage: one element = a packed pair (real part in the low half)
  __device__ __forceinline__ uint2 ldg16x2(const unsigned* p) {
    PAIRED_CHECK(hbm_ok(p, gin, 2), make_uint2(0u, 0u));
    return __ldcs(reinterpret_cast<const uint2*>(p));
  }
  __device__ __forceinline__ unsigned ldg16(const unsigned* p) {
    PAIRED_CHECK(hbm_ok(p, gin, 1), 0u);
    return __ldcs(p);
  }
  __device__ __forceinline__ void stg16x2(unsigned* p, uint2 v) {
    PAIRED_CHECK(hbm_ok(p, gout, 2), );
    __stcs(reinterpret_cast<uint2*>(p), v);
  }
  __device__ __forceinline__ void stg16(unsigned* p, unsigned v) {
    PAIRED_CHECK(hbm_ok(p, gout, 1), );
    __stcs(p, v);
  }
  __device__ __forceinline__ float2 unpack16(unsigned u, int dt) {
    if (dt == 1) return make_float2(__uint_as_float(u << 16), __uint_as_float(u & 0xffff0000u));
    if (dt == 3) return make_float2((float)(short)(u & 0xffffu), (float)(short)(u >> 16));
    return make_float2(__half2float(__ushort_as_half((unsigned short)(u & 0xffffu))),
                       __half2float(__ushort_as_half((unsigned short)(u >> 16))));
  }
  __device__ __forceinline__ static unsigned i16(float v) {
    int q = __float2int_rn(v);
    q = q < -32768 ? -32768 : (q > 32767 ? 32767 : q);
    return (unsigned)(unsigned short)(short)q;
  }
  __device__ __forceinline__ unsigned pack16(float re, float im, int dt) {
    if (dt == 1)
      return (unsigned)__bfloat16_as_ushort(__float2bfloat16_rn(re)) |
             ((unsigned)__bfloat16_as_ushort(__float2bfloat16_rn(im)) << 16);
    if (dt == 3) return i16(re) | (i16(im) << 16);
    return (unsigned)__half_as_ushort(__float2half_rn(re)) | ((unsigned)__half_as_ushort(__float2half_rn(im)) << 16);
  }
  // the largest m of the CTA, for every thread
  __device__ __forceinline__ float max_cta(float m) {
    __shared__ float red[32];
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
      const float o = __shfl_xor_sync(0xffffffffu, m, d);
      m = o > m ? o : m;
    }
    if ((tid & 31) == 0) red[tid >> 5] = m;
    __syncthreads();
    float r = 0.f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) r = red[w] > r ? red[w] : r;
    __syncthreads();  // red is reused by the next transform
    return r;
  }
  __device__ __forceinline__ float2 shfl_up(float2 v, int d) {
    return make_float2(__shfl_up_sync(0xffffffffu, v.x, d), __shfl_up_sync(0xffffffffu, v.y, d));
  }
  // float2 index i of CTA q's region: the own region through the shared
  // window, the others as distributed shared memory, 32-bit addresses
  __device__ __forceinline__ void dst2(int q, int i, float2 v) {
    PAIRED_CHECK(reg_ok(i, 1), );
    if (q == rank)
      asm volatile("st.shared.v2.f32 [%0], {%1, %2};" ::"r"(lbase + 8u * (unsigned)i), "f"(v.x), "f"(v.y) : "memory");
    else
      asm volatile("st.shared::cluster.v2.f32 [%0], {%1, %2};" ::"r"(cbase(q) + 8u * (unsigned)i), "f"(v.x), "f"(v.y)
                   : "memory");
  }
  __device__ __forceinline__ float2 dld2(int q, int i) {
    PAIRED_CHECK(reg_ok(i, 1), make_float2(0.f, 0.f));
    float2 v;
    if (q == rank)
      asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(lbase + 8u * (unsigned)i) : "memory");
    else
      asm volatile("ld.shared::cluster.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(cbase(q) + 8u * (unsigned)i)
                   : "memory");
    return v;
  }
  // two float2 at index i (even): one 16-byte access
  __device__ __forceinline__ void dld4(int q, int i, float2* v) {
#ifdef AMQFT_BOUNDS_CHECK
    if (!reg_ok(i, 2)) {
      v[0] = v[1] = make_float2(0.f, 0.f);
      return;
    }
#endif
    float a, b, c, d;
    if (q == rank)
      asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(a), "=f"(b), "=f"(c), "=f"(d)
                   : "r"(lbase + 8u * (unsigned)i) : "memory");
    else
      asm volatile("ld.shared::cluster.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(a), "=f"(b), "=f"(c), "=f"(d)
                   : "r"(cbase(q) + 8u * (unsigned)i) : "memory");
    v[0] = make_float2(a, b);
    v[1] = make_float2(c, d);
  }
};

// threads per CTA and CTAs per SM of the kernel for 2^LN
__host__ __device__ constexpr int paired_tpb(int LN) { return 1 << (LN - 7); }
__host__ __device__ constexpr int paired_ctas(int LN) { return LN >= 16 ? 1 : (LN == 15 ? 2 : 4); }

template <int LN, bool INV, bool H>
__global__ void __launch_bounds__(paired_tpb(LN), paired_ctas(LN))
    paired_kernel(const void* __restrict__ in, void* __restrict__ out, const Store16 io, const TList tl,
                  long long batch, const float* __restrict__ ctab, const __grid_constant__ LeafConsts K) {
  constexpr int T = LN - 2;
  extern __shared__ __align__(16) float2 psm[];
  cg::cluster_group cl = cg::this_cluster();
  DevCtx cx;
  cx.tid = (int)threadIdx.x;
  cx.rank = (int)cl.block_rank();
  cx.lbase = (unsigned)__cvta_generic_to_shared(psm);
#ifdef AMQFT_BOUNDS_CHECK
  cx.rf = region_f2<T>();
  cx.es = H ? 4 : 8;
  cx.gin = static_cast<const char*>(in);
  cx.gout = static_cast<const char*>(out);
  cx.gn = tl.list ? (1LL << 62) / cx.es : batch << LN;  // a ragged buffer's extent is the caller's
#endif
  float* cst = reinterpret_cast<float*>(psm + region_f2<T>());
  if (!ctab) {  // constants on the fly: the same entries paired_body copies from the table
    const int ncst = (cx.rank & 1) == 0 ? (1 << T) - 32 : (1 << (T - 1)) - 32;
    for (int i = cx.tid; i < ncst; i += paired_tpb(LN)) cst[i] = fly_entry<4>(30 + i);
  }
  paired_body<LN, INV, H>(cx, in, out, &io, (int)batch, (int)(blockIdx.x >> 2), (int)(gridDim.x >> 2), psm, cst,
                          ctab, K, tl);
}

template <int LN, bool INV, bool H>
static cudaError_t launch(const void* in, void* out, const Store16& io, const TList& tl, long long batch,
                          const float* ctab, const LeafConsts& K, cudaStream_t st) {
  constexpr int T = LN - 2, SMEM = smem_bytes<T>();
  auto kern = paired_kernel<LN, INV, H>;
  // the number of clusters that fit on the device at once, queried once
  static int max_clusters[2] = {0, 0};  // per instantiation; a race only recomputes the same value
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 4;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.blockDim = dim3(paired_tpb(LN), 1, 1);
  cfg.dynamicSmemBytes = (size_t)SMEM;
  cfg.stream = st;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (max_clusters[INV] == 0) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM);
    if (e != cudaSuccess) return e;
    int n = 0;
    cfg.gridDim = dim3(4, 1, 1);
    e = cudaOccupancyMaxActiveClusters(&n, kern, &cfg);
    if (e != cudaSuccess) return e;
    if (n < 1) return cudaErrorInvalidConfiguration;
    max_clusters[INV] = n;
  }
  const long long ncl = batch < max_clusters[INV] ? batch : max_clusters[INV];
  cfg.gridDim = dim3((unsigned)(4 * ncl), 1, 1);
  return cudaLaunchKernelEx(&cfg, kern, in, out, io, tl, batch, ctab, K);
}


template <int LN>
cudaError_t launch_len(const void* in, void* out, const int* exp_in, int* exp_out, int dtype, long long batch,
                       int inverse, const float* ctab, const SmallConsts& K, cudaStream_t st, const int* tlist,
                       const long long* toff, const int* tcount) {
  LeafConsts L;
  for (int i = 0; i < 30; ++i) L.c[i] = K.c[i];
  L.cos_pi4 = K.cos_pi4;
  L.nz = -0.0f;
  const Store16 io{exp_in, exp_out, dtype};
  const TList tl{tlist, toff, tcount};
  if (dtype == 0)
    return inverse ? launch<LN, true, false>(in, out, io, tl, batch, ctab, L, st)
                   : launch<LN, false, false>(in, out, io, tl, batch, ctab, L, st);
  return inverse ? launch<LN, true, true>(in, out, io, tl, batch, ctab, L, st)
                 : launch<LN, false, true>(in, out, io, tl, batch, ctab, L, st);
}

}  // namespace pr
}  // namespace amqft
