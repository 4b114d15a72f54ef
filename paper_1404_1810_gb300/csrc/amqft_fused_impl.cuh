// Fused single-pass AM-QFT kernel: one HBM read and one HBM write per sample.
//
// A CTA (cluster size 1) holds `tpc` whole transforms, or a cluster of four
// CTAs holds one transform with one region per CTA (N = 2^14 .. 2^16), the
// load and store stages reaching the other CTAs' regions through
// distributed shared memory.  Stages (see amqft_device.cuh for the layout):
//   load   D_c (Sect. 3.1), D_r (Eq. qft_22-23) and, for the harmonics-first
//          variants, the first D_k of the chain; scatter into the regions.
//   trees  level-synchronous passes down the D_k / D_n trees, register
//          subtrees of LEAF values, passes back up; the chain levels.
//   store  last chain level (time-first variants), D_r^F (Eq. qft_24-25)
//          and D_c^F (Eq. qft_17-21) straight to HBM.
#pragma once
#include "amqft_bands.cuh"
#include "amqft_device.cuh"
#include "amqft_internal.h"

namespace amqft {

template <int CL>
struct Regions {
  float* sm;
  int RS;
  long long tbase;
  __device__ __forceinline__ float* get(int tau, int kind) const {
    if constexpr (CL == 1) {
      return sm + (4 * tau + kind) * RS;
    } else {
      constexpr int PER = 4 / CL;
      cg::cluster_group cl = cg::this_cluster();
      float* remote = cl.map_shared_rank(sm, kind / PER);
      return remote + (kind % PER) * RS;
    }
  }
};

__device__ __forceinline__ float2 ldz(const float2* __restrict__ p, int i, float cj) {
  float2 v = __ldcs(p + i);
  v.y *= cj;
  return v;
}

__device__ __forceinline__ void stz(float2* __restrict__ p, int i, float re, float im, float cj) {
  __stcs(p + i, make_float2(re, im * cj));
}

// Load stage for orbit item n of transform tau: samples n, N-n, N/2-n, N/2+n
// (item 0: samples 0, N/2, N/4, 3N/4).  Fetch and scatter are separate so a
// thread's four items have their global loads in flight together.
struct Fetched {
  float2 a, b, c, d;
};

__device__ __forceinline__ Fetched load_fetch(const float2* __restrict__ in, int logN, long long t, int n, float cj) {
  const int N = 1 << logN, half = N >> 1, Q = N >> 2;
  const float2* __restrict__ z = in + t * (long long)N;
  Fetched f;
  if (n == 0) {
    f.a = ldz(z, 0, cj);
    f.b = ldz(z, half, cj);
    if (N >= 4) {
      f.c = ldz(z, Q, cj);
      f.d = ldz(z, 3 * Q, cj);
    }
  } else {
    f.a = ldz(z, n, cj);
    f.b = ldz(z, N - n, cj);
    f.c = ldz(z, half - n, cj);
    f.d = ldz(z, half + n, cj);
  }
  return f;
}

template <int V, class RG>
__device__ __forceinline__ void load_scatter(const RG& rg, int logN, int tau, int n, const Fetched& f) {
  const int N = 1 << logN, half = N >> 1, Q = N >> 2, logQ = logN - 2;
  float* C1 = rg.get(tau, 0);
  float* S1 = rg.get(tau, 1);
  float* C2 = rg.get(tau, 2);
  float* S2 = rg.get(tau, 3);
  if (n == 0) {
    const float2 z0 = f.a, zh = f.b;
    if (N == 2) {
      C1[0] = z0.x; C1[1] = zh.x; C2[0] = z0.y; C2[1] = zh.y;
      return;
    }
    const float2 zq = f.c, z3 = f.d;
    const float cq1 = zq.x + z3.x, sq1 = zq.x - z3.x, cq2 = zq.y + z3.y, sq2 = zq.y - z3.y;
    if constexpr (Var<V>::ot) {
      C1[sw(half - 1)] = z0.x; C1[sw(half)] = zh.x;
      C2[sw(half - 1)] = z0.y; C2[sw(half)] = zh.y;
      C1[sw(half - 2)] = cq1; C2[sw(half - 2)] = cq2;   // pos_chain(Q, dct) = half - 2
      S1[sw(half - 2)] = sq1; S2[sw(half - 2)] = sq2;   // dst(4) base
    } else {
      C1[sw(Q)] = z0.x + zh.x; C1[sw(0)] = z0.x - zh.x;   // te(0), to(0)
      C2[sw(Q)] = z0.y + zh.y; C2[sw(0)] = z0.y - zh.y;
      C1[sw(half)] = cq1; C2[sw(half)] = cq2;           // te(Q) = dc(Q)
      S1[sw(Q - 1)] = sq1; S2[sw(Q - 1)] = sq2;         // to(Q) = ds(Q)
    }
    return;
  }
  const int m = half - n;
  const float2 za = f.a, zb = f.b, zc = f.c, zd = f.d;
  // D_r: dc(n) = x(n) + x(N-n), ds(n) = x(n) - x(N-n), for n and N/2 - n
  const float dcn1 = za.x + zb.x, dsn1 = za.x - zb.x, dcm1 = zc.x + zd.x, dsm1 = zc.x - zd.x;
  const float dcn2 = za.y + zb.y, dsn2 = za.y - zb.y, dcm2 = zc.y + zd.y, dsm2 = zc.y - zd.y;
  if constexpr (Var<V>::ot) {
    const int pcn = sw(pos_chain(n, logN, 0)), pcm = sw(pos_chain(m, logN, 0));
    const int psn = sw(pos_chain(n, logN, 1)), psm = sw(pos_chain(m, logN, 1));
    C1[pcn] = dcn1; C1[pcm] = dcm1; S1[psn] = dsn1; S1[psm] = dsm1;
    C2[pcn] = dcn2; C2[pcm] = dcm2; S2[psn] = dsn2; S2[psm] = dsm2;
  } else {
    // first D_k of the chain (M = N): te -> dct(N/2), to -> dct_to(N) bit-reversed
    const int pte = sw(Q + n), pto = sw(brev(n, logQ));
    const int ste = sw(Q + n - 1), sto = sw(brev(n - 1, logQ));
    C1[pte] = dcn1 + dcm1; C1[pto] = dcn1 - dcm1;
    C2[pte] = dcn2 + dcm2; C2[pto] = dcn2 - dcm2;
    S1[ste] = dsn1 - dsm1; S1[sto] = dsn1 + dsm1;
    S2[ste] = dsn2 - dsm2; S2[sto] = dsn2 + dsm2;
  }
}

// Store stage for orbit item k: harmonics k, N-k, N/2-k, N/2+k (item 0:
// 0, N/2, N/4, 3N/4).  Gather (shared-memory reads, remote for clusters) and
// emit (arithmetic + HBM writes) are separate so a thread's four items have
// their reads in flight together.
struct Gathered {
  float v[8];
};

template <int V, class RG>
__device__ __forceinline__ Gathered store_gather(const RG& rg, int logN, int tau, int k) {
  const int N = 1 << logN, half = N >> 1, Q = N >> 2, logQ = logN - 2;
  const float* C1 = rg.get(tau, 0);
  const float* S1 = rg.get(tau, 1);
  const float* C2 = rg.get(tau, 2);
  const float* S2 = rg.get(tau, 3);
  Gathered g;
  if (k == 0) {
    if (N == 2) {
      g.v[0] = C1[0]; g.v[1] = C1[1]; g.v[2] = C2[0]; g.v[3] = C2[1];
      return g;
    }
    if constexpr (Var<V>::ot) {
      g.v[0] = C1[sw(Q)]; g.v[1] = C1[sw(0)]; g.v[2] = C2[sw(Q)]; g.v[3] = C2[sw(0)];
      g.v[4] = C1[sw(half)]; g.v[5] = C2[sw(half)];
      g.v[6] = S1[sw(Q - 1)]; g.v[7] = S2[sw(Q - 1)];
    } else {
      g.v[0] = C1[sw(half - 1)]; g.v[1] = C1[sw(half)]; g.v[2] = C2[sw(half - 1)]; g.v[3] = C2[sw(half)];
      g.v[4] = C1[sw(half - 2)]; g.v[5] = C2[sw(half - 2)];
      g.v[6] = S1[sw(half - 2)]; g.v[7] = S2[sw(half - 2)];
    }
    return g;
  }
  const int m = half - k;
  if constexpr (Var<V>::ot) {
    const int po = sw(brev(k, logQ)), pe = sw(Q + k);
    const int qo = sw(brev(k - 1, logQ)), qe = sw(Q + k - 1);
    g.v[0] = C1[pe]; g.v[1] = C1[po]; g.v[2] = C2[pe]; g.v[3] = C2[po];
    g.v[4] = S1[qo]; g.v[5] = S1[qe]; g.v[6] = S2[qo]; g.v[7] = S2[qe];
  } else {
    const int pk = sw(pos_chain(k, logN, 0)), pm = sw(pos_chain(m, logN, 0));
    const int qk = sw(pos_chain(k, logN, 1)), qm = sw(pos_chain(m, logN, 1));
    g.v[0] = C1[pk]; g.v[1] = C1[pm]; g.v[2] = C2[pk]; g.v[3] = C2[pm];
    g.v[4] = S1[qk]; g.v[5] = S1[qm]; g.v[6] = S2[qk]; g.v[7] = S2[qm];
  }
  return g;
}

template <int V>
__device__ __forceinline__ void store_emit(float2* __restrict__ out, int logN, long long t, int k, const Gathered& g,
                                           float cj) {
  const int N = 1 << logN, half = N >> 1, Q = N >> 2;
  float2* __restrict__ z = out + t * (long long)N;
  if (k == 0) {
    if (N == 2) {
      stz(z, 0, g.v[0], g.v[2], cj);
      stz(z, 1, g.v[1], g.v[3], cj);
      return;
    }
    float c01, c02, ch1, ch2;
    if constexpr (Var<V>::ot) {
      // last D_n of the chain (M = N) at k = 0
      c01 = g.v[0] + g.v[1]; ch1 = g.v[0] - g.v[1]; c02 = g.v[2] + g.v[3]; ch2 = g.v[2] - g.v[3];
    } else {
      c01 = g.v[0]; ch1 = g.v[1]; c02 = g.v[2]; ch2 = g.v[3];
    }
    const float cq1 = g.v[4], cq2 = g.v[5], sq1 = g.v[6], sq2 = g.v[7];
    stz(z, 0, c01, c02, cj);
    stz(z, half, ch1, ch2, cj);
    stz(z, Q, cq1 + sq2, cq2 - sq1, cj);
    stz(z, 3 * Q, cq1 - sq2, cq2 + sq1, cj);
    return;
  }
  const int m = half - k;
  float ck1, ck2, cm1, cm2, sk1, sk2, sm1, sm2;
  if constexpr (Var<V>::ot) {
    // last D_n of the chain (M = N): dct S(k) = E + O, S(N/2-k) = E - O; dst S(k) = O + E, S(N/2-k) = O - E
    ck1 = g.v[0] + g.v[1]; cm1 = g.v[0] - g.v[1]; ck2 = g.v[2] + g.v[3]; cm2 = g.v[2] - g.v[3];
    sk1 = g.v[4] + g.v[5]; sm1 = g.v[4] - g.v[5]; sk2 = g.v[6] + g.v[7]; sm2 = g.v[6] - g.v[7];
  } else {
    ck1 = g.v[0]; cm1 = g.v[1]; ck2 = g.v[2]; cm2 = g.v[3];
    sk1 = g.v[4]; sm1 = g.v[5]; sk2 = g.v[6]; sm2 = g.v[7];
  }
  // D_c^F with Re R = DCT, Im R = -DST: X(k) = (C1 + S2, C2 - S1), X(N-k) = (C1 - S2, C2 + S1)
  stz(z, k, ck1 + sk2, ck2 - sk1, cj);
  stz(z, N - k, ck1 - sk2, ck2 + sk1, cj);
  stz(z, m, cm1 + sm2, cm2 - sm1, cj);
  stz(z, half + k, cm1 - sm2, cm2 + sm1, cj);
}

template <int V, int TPB, int MAXI, int CL>
__global__ void __launch_bounds__(TPB) fused_kernel(const FusedArgs a, const __grid_constant__ SmallConsts K) {
  extern __shared__ __align__(16) float sm[];
  const int logN = a.logN, N = 1 << logN, half = N >> 1;
  const int Qi = N >= 4 ? (N >> 2) : 1;   // orbit items per transform
  const int logQi = N >= 4 ? logN - 2 : 0;
  const float cj = a.inverse ? -1.f : 1.f;
  Geo g;
  g.logN = logN;
  g.half = half;
  g.RS = a.RS;
  g.sub = 0;
  Regions<CL> rg;
  rg.sm = sm;
  rg.RS = a.RS;
  int ntr;
  if constexpr (CL == 1) {
    rg.tbase = (long long)blockIdx.x * a.tpc;
    const long long left = a.batch - rg.tbase;
    ntr = left < a.tpc ? (int)left : a.tpc;
    g.nreg = 4 * ntr;
    g.gbase = 0;
  } else {
    cg::cluster_group cl = cg::this_cluster();
    rg.tbase = blockIdx.x / CL;
    ntr = 1;
    g.nreg = 4 / CL;
    g.gbase = (int)cl.block_rank() * (4 / CL);
    cl.sync();  // every CTA of the cluster is resident before remote writes
  }
  float* tot = sm + a.tot_off;
  float* wsum = tot + TPB;
  float* snap = wsum + 32;

  // ---- load ----
  // every configuration gives each thread exactly four orbit items
  {
    int n_[4], tau_[4];
    bool ok_[4];
    Fetched f_[4];
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      if constexpr (CL == 1) {
        const int w = threadIdx.x + s * TPB;
        tau_[s] = w >> logQi;
        n_[s] = w & (Qi - 1);
        ok_[s] = tau_[s] < ntr;
      } else {
        const int per = Qi / CL;
        tau_[s] = 0;
        n_[s] = (int)cg::this_cluster().block_rank() * per + threadIdx.x + s * TPB;
        ok_[s] = (int)threadIdx.x + s * TPB < per;
      }
      if (ok_[s]) f_[s] = load_fetch(a.in, a.logN, rg.tbase + tau_[s], n_[s], cj);
    }
#pragma unroll
    for (int s = 0; s < 4; ++s)
      if (ok_[s]) load_scatter<V>(rg, a.logN, tau_[s], n_[s], f_[s]);
  }
  if constexpr (CL == 1) __syncthreads();
  else cg::this_cluster().sync();

  // ---- trees and chain ----
  const int logTop = logN - 2;  // log2 of the largest tree (N/4)
  const BandPlan bp = band_plan(logN);
  if constexpr (Var<V>::ot) {
    for (int b = 0; b < bp.nb; ++b) {
      run_fold_band_r<V, TPB>(sm, g, bp.logL[b], bp.R[b], true, a.ctab);
      __syncthreads();
    }
    {
      const int nleaf = logTop >= LOG_LEAF ? ((half >> LOG_LEAF) - 1) : 0;
      const int W = g.nreg * nleaf + g.nreg;
      const Div dv(nleaf > 0 ? (unsigned)nleaf : 1u);
      for (int w = threadIdx.x; w < W; w += TPB) {
        if (w < g.nreg * nleaf) {
          const int r = (int)dv((unsigned)w), b = w - r * nleaf;
          const int p0 = b << LOG_LEAF;
          run_leaf<V>(sm + r * g.RS, p0, node_ctx_g<V>(g, p0, LOG_LEAF, ctx_of(g, r)), K);
        } else {
          const int r = w - g.nreg * nleaf;
          run_tail<V>(sm + r * g.RS, ctx_of(g, r), logN, K);
        }
      }
      __syncthreads();
    }
    if constexpr (Var<V>::scan) {
      for (int lp = LOG_LEAF + 1; lp <= logTop; ++lp) {
        pass_recurrence<V, TPB, MAXI>(sm, tot, wsum, g, lp);
        __syncthreads();
      }
    } else {
      for (int b = bp.nb - 1; b >= 0; --b) {
        run_chunk_band_r<V, TPB>(sm, snap, g, bp.logL[b], bp.R[b]);
        __syncthreads();
      }
    }
    for (int lm = LOG_LEAF + 2; lm <= logN - 1; ++lm) {
      pass_chain<V, TPB, MAXI>(sm, g, lm);
      __syncthreads();
    }
  } else {
    for (int lm = logN - 1; lm >= LOG_LEAF + 2; --lm) {
      pass_chain<V, TPB, MAXI>(sm, g, lm);
      __syncthreads();
    }
    for (int r = threadIdx.x; r < g.nreg; r += TPB) run_tail<V>(sm + r * g.RS, ctx_of(g, r), logN, K);
    __syncthreads();
    for (int lp = logTop; lp >= LOG_LEAF + 1; --lp) {
      if constexpr (Var<V>::scan) pass_recurrence<V, TPB, MAXI>(sm, tot, wsum, g, lp);
      else pass_neighbour<V, TPB, MAXI>(sm, g, lp);
      __syncthreads();
    }
    if (logTop >= LOG_LEAF) {
      const int nleaf = (half >> LOG_LEAF) - 1;
      const int W = g.nreg * nleaf;
      const Div dv((unsigned)nleaf);
      for (int w = threadIdx.x; w < W; w += TPB) {
        const int r = (int)dv((unsigned)w), b = w - r * nleaf;
        const int p0 = b << LOG_LEAF;
        run_leaf<V>(sm + r * g.RS, p0, node_ctx_g<V>(g, p0, LOG_LEAF, ctx_of(g, r)), K);
      }
      __syncthreads();
    }
    for (int b = bp.nb - 1; b >= 0; --b) {
      run_fold_band_r<V, TPB>(sm, g, bp.logL[b], bp.R[b], false, a.ctab);
      __syncthreads();
    }
  }

  // ---- store ----
  if constexpr (CL > 1) cg::this_cluster().sync();
  {
    int k_[4], tau_[4];
    bool ok_[4];
    Gathered g_[4];
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      if constexpr (CL == 1) {
        const int w = threadIdx.x + s * TPB;
        tau_[s] = w >> logQi;
        k_[s] = w & (Qi - 1);
        ok_[s] = tau_[s] < ntr;
      } else {
        const int per = Qi / CL;
        tau_[s] = 0;
        k_[s] = (int)cg::this_cluster().block_rank() * per + threadIdx.x + s * TPB;
        ok_[s] = (int)threadIdx.x + s * TPB < per;
      }
      if (ok_[s]) g_[s] = store_gather<V>(rg, a.logN, tau_[s], k_[s]);
    }
#pragma unroll
    for (int s = 0; s < 4; ++s)
      if (ok_[s]) store_emit<V>(a.out, a.logN, rg.tbase + tau_[s], k_[s], g_[s], cj);
  }
  if constexpr (CL > 1) cg::this_cluster().sync();  // keep shared memory alive for the other CTAs' reads
}

// ---------------------------------------------------------------------
// host side: configuration and launch
// ---------------------------------------------------------------------
template <int V, int TPB, int MAXI, int CL>
cudaError_t launch_cfg(const FusedArgs& a, const SmallConsts& K, long long grid, int smem,
                              cudaStream_t st) {
  auto kern = fused_kernel<V, TPB, MAXI, CL>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  if constexpr (CL == 1) {
    kern<<<(unsigned)grid, TPB, smem, st>>>(a, K);
    return cudaGetLastError();
  } else {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(grid * CL), 1, 1);
    cfg.blockDim = dim3(TPB, 1, 1);
    cfg.dynamicSmemBytes = (size_t)smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CL;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, a, K);
  }
}

template <int V>
cudaError_t launch_v(const FusedArgs& a, const SmallConsts& K, const FusedConfig& c, cudaStream_t st) {
  if (c.cluster == 1) {
    const long long grid = (a.batch + c.per_cta - 1) / c.per_cta;
    return launch_cfg<V, 512, 16, 1>(a, K, grid, c.smem, st);
  }
  switch (c.threads) {
    case 256: return launch_cfg<V, 256, 16, 4>(a, K, a.batch, c.smem, st);
    case 512: return launch_cfg<V, 512, 16, 4>(a, K, a.batch, c.smem, st);
    default: return launch_cfg<V, 1024, 16, 4>(a, K, a.batch, c.smem, st);
  }
}

}  // namespace amqft
