// Ragged batches: transforms of different power-of-two lengths, each at its
// own element offset, in one stream of launches with no host synchronisation
// (so the whole sequence can be captured in a CUDA graph):
//
//   bucket    transform ids sorted into one list per log2 N (device atomics);
//             N = 1 transforms are copied here;
//   small     one persistent launch for every length up to 2^13: a CTA
//             takes a work item (up to tpc transforms of one length, the
//             same packing as the batched kernel) and runs the fused body;
//   cluster   one persistent cluster launch per length 2^14, 2^15, 2^16;
//   large     the multi-pass sequence per length above 2^16, its grids sized
//             for the plan's capacity and the actual count read on the
//             device.
#pragma once

#include "amqft_multipass_impl.cuh"

namespace amqft {

constexpr int RAGGED_CLASSES = 32;  // list slots, indexed by log2 N

struct RaggedArgs {
  const int* cnt;     // transforms per log2 N (after the bucket pass)
  const int* list;    // ids of log2 N = c at [c * cap, c * cap + cnt[c])
  long long cap;      // list capacity per class
  int* work;          // dynamic schedule counter (zero before the small launch)
  int maxlog;         // largest log2 N of the plan
  int sched;          // 0: static round robin, 1: dynamic (atomic counter)
  int order;          // 0: longest lengths first, 1: shortest first
  int ubase;          // > 0: the transforms of 2^14..2^16 whose offset is not
                      // 16-byte aligned are listed apart, as classes ubase + 0..2
                      // (the others run on the paired-region kernel)
};

__host__ __device__ constexpr int small_tot_off(int logN) {
  return ((4 * small_tpc(logN) * region_stride(logN) + 31) / 32) * 32;
}

// one work item of the small launch, compiled on its own so that its register
// allocation matches the batched kernel's
template <int V>
__device__ __noinline__ void ragged_small_item(const FusedArgs& a0, const SmallConsts& K, float* sm, int j0, int ntr,
                                               int c, const int* tlist) {
  fused_body<V, SMALL_TPB, SMALL_MAXI, 1, 0>(a0, K, sm, j0, ntr, c, region_stride(c), small_tot_off(c), tlist);
}

template <int V>
__global__ void __launch_bounds__(SMALL_TPB, 2) ragged_small_kernel(const FusedArgs a0, const __grid_constant__ SmallConsts K,
                                                           const RaggedArgs r) {
  extern __shared__ __align__(16) float sm[];
  __shared__ int s_item;
  const int cmax = r.maxlog < 13 ? r.maxlog : 13;
  int total = 0;
  for (int c = 1; c <= cmax; ++c) total += (r.cnt[c] + small_tpc(c) - 1) / small_tpc(c);
  int it = blockIdx.x;
  if (r.sched) {
    if (threadIdx.x == 0) s_item = atomicAdd(r.work, 1);
    __syncthreads();
    it = s_item;
  }
  while (it < total) {
    // work item `it` in the chosen class order
    int c = 0, w = it;
    for (int q = 0; q < cmax; ++q) {
      const int cc = r.order ? 1 + q : cmax - q;
      const int n = (r.cnt[cc] + small_tpc(cc) - 1) / small_tpc(cc);
      if (w < n) {
        c = cc;
        break;
      }
      w -= n;
    }
    const int tpc = small_tpc(c);
    const int j0 = w * tpc;
    const int left = r.cnt[c] - j0;
    ragged_small_item<V>(a0, K, sm, j0, left < tpc ? left : tpc, c, r.list + c * r.cap);
    __syncthreads();  // shared memory is reused by the next item
    if (r.sched) {
      if (threadIdx.x == 0) s_item = atomicAdd(r.work, 1);
      __syncthreads();
      it = s_item;
    } else {
      it += gridDim.x;
    }
  }
}

template <int V, int LN, int TPB = cluster_tpb(LN, Var<V>::ot)>
__global__ void __launch_bounds__(TPB, ctas_per_sm(TPB)) ragged_cluster_kernel(const FusedArgs a0, const __grid_constant__ SmallConsts K,
                                                             const RaggedArgs r, int cls) {
  extern __shared__ __align__(16) float sm[];
  const int n = r.cnt[cls];
  const int ncl = (int)(gridDim.x / 4);
  for (int j = (int)(blockIdx.x / 4); j < n; j += ncl)
    fused_body<V, TPB, cluster_maxi(LN, Var<V>::ot), 4, LN>(a0, K, sm, j, 1, LN, 0, a0.tot_off, r.list + cls * r.cap);
}

// host: launch one persistent cluster grid for length 2^LN
template <int V, int LN>
cudaError_t ragged_cluster_launch(const FusedArgs& a, const SmallConsts& K, const RaggedArgs& r, int clusters,
                                  int smem, cudaStream_t st, int cls = LN) {
  constexpr int TPB = cluster_tpb(LN, Var<V>::ot);
  auto kern = ragged_cluster_kernel<V, LN>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(4 * clusters), 1, 1);
  cfg.blockDim = dim3(TPB, 1, 1);
  cfg.dynamicSmemBytes = (size_t)smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 4;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, a, K, r, cls);
}

// Launch geometry chosen by the host (and the autotuner).
struct RaggedLaunch {
  int small_grid;          // CTAs of the small launch
  int small_smem;          // its dynamic shared memory
  int clusters[3];         // cluster grids for 2^14, 2^15, 2^16
  int cluster_smem[3];
  int cluster_tot_off[3];
};

// `nlaunch` (may be NULL) is incremented once per kernel launched.
template <int V>
cudaError_t ragged_run(const FusedArgs& a0, const SmallConsts& K, const RaggedArgs& r, const RaggedLaunch& L,
                       cudaStream_t st, long long* nlaunch) {
  cudaError_t e;
  if (r.maxlog >= 1) {
    auto kern = ragged_small_kernel<V>;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, L.small_smem);
    if (e != cudaSuccess) return e;
    kern<<<(unsigned)L.small_grid, SMALL_TPB, L.small_smem, st>>>(a0, K, r);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (nlaunch) ++*nlaunch;
  }
  FusedArgs a = a0;
  if (V == 4 && r.ubase > 0) {
    // 2^14 .. 2^16: the paired-region kernel over each length's aligned list,
    // the fused cluster kernel over the transforms listed apart
    for (int q = 0; q < 3 && 14 + q <= r.maxlog; ++q) {
      const int c = 14 + q;
      e = paired_launch(c, a0.in, a0.out, nullptr, nullptr, 0, r.cap, a0.inverse, a0.ctab, K, st, r.list + c * r.cap,
                        a0.toff, r.cnt + c);
      if (e != cudaSuccess) return e;
      if (nlaunch) ++*nlaunch;
      a.tot_off = L.cluster_tot_off[q];
      if (q == 0) e = ragged_cluster_launch<V, 14>(a, K, r, L.clusters[0], L.cluster_smem[0], st, r.ubase);
      else if (q == 1) e = ragged_cluster_launch<V, 15>(a, K, r, L.clusters[1], L.cluster_smem[1], st, r.ubase + 1);
      else e = ragged_cluster_launch<V, 16>(a, K, r, L.clusters[2], L.cluster_smem[2], st, r.ubase + 2);
      if (e != cudaSuccess) return e;
      if (nlaunch) ++*nlaunch;
    }
    return cudaSuccess;
  }
  if (r.maxlog >= 14) {
    a.tot_off = L.cluster_tot_off[0];
    e = ragged_cluster_launch<V, 14>(a, K, r, L.clusters[0], L.cluster_smem[0], st);
    if (e != cudaSuccess) return e;
    if (nlaunch) ++*nlaunch;
  }
  if (r.maxlog >= 15) {
    a.tot_off = L.cluster_tot_off[1];
    e = ragged_cluster_launch<V, 15>(a, K, r, L.clusters[1], L.cluster_smem[1], st);
    if (e != cudaSuccess) return e;
    if (nlaunch) ++*nlaunch;
  }
  if (r.maxlog >= 16) {
    a.tot_off = L.cluster_tot_off[2];
    e = ragged_cluster_launch<V, 16>(a, K, r, L.clusters[2], L.cluster_smem[2], st);
    if (e != cudaSuccess) return e;
    if (nlaunch) ++*nlaunch;
  }
  return cudaSuccess;
}

}  // namespace amqft
