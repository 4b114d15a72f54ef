// Register bands: up to four consecutive tree levels per shared-memory round
// trip, computed in place (every work group writes exactly the shared-memory
// words it read), so no values are held across a barrier.  A band performs
// exactly the float32 operations of the per-level passes, in the same order
// for every output, so results are unchanged.
//
//  * fold bands (D_k + M_v time phase of the ot trees; D_n + M_v frequency
//    phase of the to trees): the values of a node that feed index i of its
//    2^R descendants form the fold orbit {i, L-1-i, L/2-1-i, L/2+i, ...};
//    the orbits of i and W-1-i (W = L/2^R) together fill exactly the two
//    descendant columns i and W-1-i, so the pair is computed in place.
//  * chunk bands (frequency phase of the ot trees for M4 / M8): the outputs
//    k in [2^R m, 2^R (m+1)) of a node need index m of every descendant plus
//    at most one neighbour (m-1 or m+1) on each path.  Consecutive m run in
//    consecutive lanes, the neighbours come by warp shuffle (and, across
//    warps, from a snapshot taken before the band), and the outputs land on
//    the same words as the inputs.
#pragma once

#include "amqft_consts.cuh"
#include "amqft_device.cuh"

namespace amqft {

constexpr int RMAX = 4;  // levels per band

// position, in the level-`lfrom` node (size L >> lfrom), of register e of the
// fold orbit of index i over R levels
template <int R>
__device__ __forceinline__ int fold_pos(int e, int lfrom, int L, int i) {
  int p = i;
#pragma unroll
  for (int l = R - 1; l >= 0; --l)
    if (l >= lfrom && ((e >> l) & 1)) p = (L >> l) - 1 - p;
  return p;
}

// context of the level-l node on the path of register e (bit l: 0 = A, 1 = B)
template <int V, int CTX>
__host__ __device__ constexpr int path_ctx(int e, int l) {
  int c = CTX;
  if (Var<V>::flip)
    for (int k = 0; k < l; ++k) c ^= (e >> k) & 1;
  return c;
}

// block of the descendant reached by register e: a DCT node keeps A in its
// first half, a DST node in its second half
template <int V, int CTX, int R>
__host__ __device__ constexpr int desc_block(int e) {
  int d = 0;
  for (int l = 0; l < R; ++l) d |= (((e >> l) & 1) ^ path_ctx<V, CTX>(e, l)) << (R - 1 - l);
  return d;
}

// ---- ot forward: D_k time phase + M_v time phase over R levels, one item --
template <int V, int R, int CTX, class CS>
__device__ __forceinline__ void fold_fwd_item(CRegP Rg, int p0, int L, int i, const CS& cs,
                                              float (&x)[1 << R]) {
  constexpr int n = 1 << R;
#pragma unroll
  for (int e = 0; e < n; ++e) x[e] = Rg[sw(p0 + fold_pos<R>(e, 0, L, i))];
#pragma unroll
  for (int l = 0; l < R; ++l) {
#pragma unroll
    for (int e = 0; e < n; ++e) {
      if ((e >> l) & 1) continue;
      const int e2 = e | (1 << l);
      const float c = cs(L >> l, fold_pos<R>(e, l + 1, L, i));
      const float u = x[e], w = x[e2];
      if (path_ctx<V, CTX>(e, l) == 0) { x[e] = u + w; x[e2] = (u - w) * c; }
      else { x[e] = u - w; x[e2] = (u + w) * c; }
    }
  }
}

template <int V, int R, int CTX, class CS>
__device__ __forceinline__ void fold_fwd_pair(RegP Rg, int p0, int L, int i, const CS& cs) {
  const int W = L >> R, i2 = W - 1 - i;
  float x[1 << R], y[1 << R];
  fold_fwd_item<V, R, CTX>(Rg, p0, L, i, cs, x);
  fold_fwd_item<V, R, CTX>(Rg, p0, L, i2, cs, y);
#pragma unroll
  for (int e = 0; e < (1 << R); ++e) {
    const int blk = p0 + desc_block<V, CTX, R>(e) * W;
    Rg[sw(blk + i)] = x[e];
    Rg[sw(blk + i2)] = y[e];
  }
}

// ---- to backward: D_n frequency phase + M_v frequency phase, one item -----
template <int V, int R, int CTX, class CS>
__device__ __forceinline__ void fold_bwd_item(CRegP Rg, int p0, int L, int i, const CS& cs,
                                              float (&x)[1 << R]) {
  constexpr int n = 1 << R;
  const int W = L >> R;
#pragma unroll
  for (int e = 0; e < n; ++e) x[e] = Rg[sw(p0 + desc_block<V, CTX, R>(e) * W + i)];
#pragma unroll
  for (int l = R - 1; l >= 0; --l) {
#pragma unroll
    for (int e = 0; e < n; ++e) {
      if ((e >> l) & 1) continue;
      const int e2 = e | (1 << l);
      const float c = cs(L >> l, fold_pos<R>(e, l + 1, L, i));
      const float E = x[e], O = x[e2] * c;
      if (path_ctx<V, CTX>(e, l) == 0) { x[e] = E + O; x[e2] = E - O; }
      else { x[e] = O + E; x[e2] = O - E; }
    }
  }
}

template <int V, int R, int CTX, class CS>
__device__ __forceinline__ void fold_bwd_pair(RegP Rg, int p0, int L, int i, const CS& cs) {
  const int W = L >> R, i2 = W - 1 - i;
  float x[1 << R], y[1 << R];
  fold_bwd_item<V, R, CTX>(Rg, p0, L, i, cs, x);
  fold_bwd_item<V, R, CTX>(Rg, p0, L, i2, cs, y);
#pragma unroll
  for (int e = 0; e < (1 << R); ++e) {
    Rg[sw(p0 + fold_pos<R>(e, 0, L, i))] = x[e];
    Rg[sw(p0 + fold_pos<R>(e, 0, L, i2))] = y[e];
  }
}

template <int V, bool FWD, int R, class CS>
__device__ __forceinline__ void fold_pair(RegP Rg, int p0, int logL, int i, int ctx, const CS& cs) {
  const int L = 1 << logL;
  if constexpr (FWD) {
    if (ctx == 0) fold_fwd_pair<V, R, 0>(Rg, p0, L, i, cs);
    else fold_fwd_pair<V, R, 1>(Rg, p0, L, i, cs);
  } else {
    if (ctx == 0) fold_bwd_pair<V, R, 0>(Rg, p0, L, i, cs);
    else fold_bwd_pair<V, R, 1>(Rg, p0, L, i, cs);
  }
}

// the trees whose roots lie inside the band: root size L >> q, R - q levels
template <int V, bool FWD, int R, int Q, class CS>
__device__ __forceinline__ void fold_bundle(RegP Rg, int half, int logL, int i, int ctx0, const CS& cs) {
  if constexpr (Q < R) {
    fold_pair<V, FWD, R - Q>(Rg, half - (2 << (logL - Q)), logL - Q, i, ctx0, cs);
    fold_bundle<V, FWD, R, Q + 1>(Rg, half, logL, i, ctx0, cs);
  }
}

// A fold band over every region of the CTA (GRID: of the whole grid, the
// regions then living in global memory).  Work groups: item pairs of the
// class-0 nodes (size L, blocks [0, half - L)), then pairs of the bundle.
template <int V, bool FWD, int R, int TPB, bool GRID = false, class CS>
__device__ __forceinline__ void run_fold_band(float* sm, const Geo& g, int logL, const CS& cs) {
  const int logW = logL - R, W2 = 1 << (logW - 1);
  const unsigned nb0 = nodes_at(g, logL);
  const unsigned per = (nb0 + (g.sub ? 0u : 1u)) << (logW - 1);  // groups per region (+ bundle)
  const unsigned total = per * (unsigned)g.nreg;
  const Div dv(per);
  const unsigned start = GRID ? blockIdx.x * TPB + threadIdx.x : threadIdx.x;
  const unsigned stride = GRID ? gridDim.x * TPB : TPB;
  for (unsigned w = start; w < total; w += stride) {
    const unsigned r = dv(w), gidx = w - r * per;
    RegP Rg = reg_ptr(sm + (long long)r * g.RS, g.RS);
    const int c0 = ctx_of(g, r);
    const unsigned b = gidx >> (logW - 1);
    const int i = (int)(gidx & (unsigned)(W2 - 1));
    if (b < nb0) {
      const int p0 = (int)(b << logL);
      fold_pair<V, FWD, R>(Rg, p0, logL, i, node_ctx_g<V>(g, p0, logL, c0), cs);
    } else {
      fold_bundle<V, FWD, R, 1>(Rg, g.half, logL, i, c0, cs);
    }
  }
}

// ---- ot backward, M4 / M8: chunk of 2^R outputs plus margins --------------
// Snapshot of the descendant values of the first (side 0) and last (side 1)
// lane of every warp-wide run of items, for the neighbours across warps.
struct Snap {
  float* buf;
  int lane;
  int run;  // index of the 32-item run of this lane
};

template <int V, int R, int CTX, int AM, int BM>
struct ChunkBwd {
  static constexpr int SZ = (1 << R) + AM + BM;
  static constexpr int NDESC = 1 << R;
  // slot: index of the first descendant of this subtree in the snapshot
  template <int SLOT, int NX>
  __device__ __forceinline__ static void run(CRegP Rg, int base, int logL, int m, const Snap& sn, int nslot,
                                             float (&out)[NX]) {
    if constexpr (R == 0) {
      const int L = 1 << logL;
      const float own = Rg[sw(base + brev(m, logL))];
      float lo_v = 0.f, hi_v = 0.f;
      if constexpr (AM > 0) {
        lo_v = __shfl_up_sync(0xffffffffu, own, 1);
        if (m == 0) lo_v = 0.f;
        else if (sn.lane == 0) lo_v = sn.buf[((sn.run - 1) * 2 + 1) * nslot + SLOT];
      }
      if constexpr (BM > 0) {
        hi_v = __shfl_down_sync(0xffffffffu, own, 1);
        if (m == L - 1) hi_v = 0.f;
        else if (sn.lane == 31) hi_v = sn.buf[((sn.run + 1) * 2 + 0) * nslot + SLOT];
      }
      static_assert(AM <= 1 && BM <= 1, "margins are at most one element");
      if constexpr (AM > 0) out[0] = lo_v;
      out[AM] = own;
      if constexpr (BM > 0) out[AM + 1] = hi_v;
    } else {
      constexpr int CB = Var<V>::flip ? 1 - CTX : CTX;
      constexpr int AAM = CTX == 0 ? 0 : AM;
      constexpr int ABM = CTX == 0 ? BM : 0;
      constexpr int BAM = V == 4 ? (CTX == 0 ? AM : 1) : (CTX == 0 ? AM + 1 : 0);
      constexpr int BBM = V == 4 ? (CTX == 0 ? 1 : BM) : (CTX == 0 ? 0 : BM + 1);
      using CA_ = ChunkBwd<V, R - 1, CTX, AAM, ABM>;
      using CB_ = ChunkBwd<V, R - 1, CB, BAM, BBM>;
      const int Lc = 1 << (logL - 1);
      float A[CA_::SZ], B[CB_::SZ];
      CA_::template run<SLOT, CA_::SZ>(Rg, CTX == 0 ? base : base + Lc, logL - 1, m, sn, nslot, A);
      CB_::template run<SLOT + (1 << (R - 1)), CB_::SZ>(Rg, CTX == 0 ? base + Lc : base, logL - 1, m, sn, nslot, B);
      const int L = 1 << logL, lo = m << R;
#pragma unroll
      for (int t = 0; t < SZ; ++t) {
        const int kk = t - AM;  // k - lo (lo is even)
        const int ii = kk >> 1;
        float v;
        if ((kk & 1) == CTX) {
          v = A[ii + AAM];
        } else if constexpr (V == 4) {
          v = CTX == 0 ? B[ii + BAM] + B[ii + 1 + BAM] : B[ii - 1 + BAM] + B[ii + BAM];
        } else {
          v = CTX == 0 ? B[ii + BAM] - B[ii - 1 + BAM] : B[ii + BAM] - B[ii + 1 + BAM];
        }
        if constexpr (AM > 0 || BM > 0) {
          const int k = lo + kk;
          out[t] = (k >= 0 && k < L) ? v : 0.f;
        } else {
          out[t] = v;
        }
      }
    }
  }
};

// descendant values of one item in snapshot order (the order of the
// ChunkBwd recursion: A subtree first, then B)
template <int V, int R, int CTX, int SLOT>
__device__ __forceinline__ void snap_item(CRegP Rg, int base, int logL, int m, float* dst) {
  if constexpr (R == 0) {
    dst[SLOT] = Rg[sw(base + brev(m, logL))];
  } else {
    constexpr int CB = Var<V>::flip ? 1 - CTX : CTX;
    const int Lc = 1 << (logL - 1);
    snap_item<V, R - 1, CTX, SLOT>(Rg, CTX == 0 ? base : base + Lc, logL - 1, m, dst);
    snap_item<V, R - 1, CB, SLOT + (1 << (R - 1))>(Rg, CTX == 0 ? base + Lc : base, logL - 1, m, dst);
  }
}

template <int V, int R, int CTX>
__device__ __forceinline__ void chunk_item(RegP Rg, int p0, int logL, int m, const Snap& sn, int nslot) {
  float out[1 << R];
  ChunkBwd<V, R, CTX, 0, 0>::template run<0, (1 << R)>(Rg, p0, logL, m, sn, nslot, out);
  const int lo = m << R;
#pragma unroll
  for (int c = 0; c < (1 << R); ++c) Rg[sw(p0 + brev(lo + c, logL))] = out[c];
}

// items of the trees rooted inside the band, same m for every tree; the
// snapshot slots of tree q follow those of the trees before it
template <int V, int R, int Q, int SLOT>
__device__ __forceinline__ void chunk_bundle(RegP Rg, int half, int logL, int m, int ctx0, const Snap& sn,
                                             int nslot, bool snap_only, float* dst) {
  if constexpr (Q < R) {
    const int p0 = half - (2 << (logL - Q));
    if (snap_only) {
      if (ctx0 == 0) snap_item<V, R - Q, 0, SLOT>(Rg, p0, logL - Q, m, dst);
      else snap_item<V, R - Q, 1, SLOT>(Rg, p0, logL - Q, m, dst);
    } else {
      Snap s2 = sn;
      s2.buf = sn.buf + SLOT;
      if (ctx0 == 0) chunk_item<V, R - Q, 0>(Rg, p0, logL - Q, m, s2, nslot);
      else chunk_item<V, R - Q, 1>(Rg, p0, logL - Q, m, s2, nslot);
    }
    chunk_bundle<V, R, Q + 1, SLOT + (1 << (R - Q))>(Rg, half, logL, m, ctx0, sn, nslot, snap_only, dst);
  }
}

// A chunk band over every region of the CTA.  Items: (class-0 node, m) and
// the bundle's m, consecutive m in consecutive lanes.  The snapshot holds, for
// every 32-item run, the first and last lane's 2^R descendant values.
template <int V, int R, int TPB>
__device__ __forceinline__ void run_chunk_band(float* sm, float* snap, const Geo& g, int logL) {
  constexpr int NSLOT = 1 << R;
  const int logW = logL - R, W = 1 << logW;
  const unsigned nb0 = nodes_at(g, logL);
  const unsigned per = (nb0 + (g.sub ? 0u : 1u)) << logW;  // items per region (W >= 32) (+ bundle)
  const unsigned total = per * (unsigned)g.nreg;
  const Div dv(per);
  const int lane = threadIdx.x & 31;
  // pass 1: snapshot of the run ends, one thread per end (entry e: run e / 2,
  // first lane for even e, last lane for odd e)
  const unsigned ends = total >> 4;
  for (unsigned e = threadIdx.x; e < ends; e += TPB) {
    const unsigned w = ((e >> 1) << 5) | ((e & 1u) ? 31u : 0u);
    const unsigned r = dv(w), it = w - r * per;
    RegP Rg = reg_ptr(sm + (long long)r * g.RS, g.RS);
    const int c0 = ctx_of(g, r);
    const unsigned b = it >> logW;
    const int m = (int)(it & (unsigned)(W - 1));
    float* dst = snap + e * NSLOT;
    if (b < nb0) {
      const int p0 = (int)(b << logL);
      if (node_ctx_g<V>(g, p0, logL, c0) == 0) snap_item<V, R, 0, 0>(Rg, p0, logL, m, dst);
      else snap_item<V, R, 1, 0>(Rg, p0, logL, m, dst);
    } else {
      Snap sn{snap, lane, 0};
      chunk_bundle<V, R, 1, 0>(Rg, g.half, logL, m, c0, sn, NSLOT, true, dst);
    }
  }
  __syncthreads();
  // pass 2: in place
  for (unsigned w = threadIdx.x; w < total; w += TPB) {
    const unsigned r = dv(w), it = w - r * per;
    RegP Rg = reg_ptr(sm + (long long)r * g.RS, g.RS);
    const int c0 = ctx_of(g, r);
    const unsigned b = it >> logW;
    const int m = (int)(it & (unsigned)(W - 1));
    Snap sn{snap, lane, (int)(w >> 5)};
    if (b < nb0) {
      const int p0 = (int)(b << logL);
      if (node_ctx_g<V>(g, p0, logL, c0) == 0) chunk_item<V, R, 0>(Rg, p0, logL, m, sn, NSLOT);
      else chunk_item<V, R, 1>(Rg, p0, logL, m, sn, NSLOT);
    } else {
      chunk_bundle<V, R, 1, 0>(Rg, g.half, logL, m, c0, sn, NSLOT, false, nullptr);
    }
  }
}

template <int V, int TPB, class CS>
__device__ __forceinline__ void run_fold_band_r(float* sm, const Geo& g, int logL, int R, bool fwd, const CS& cs) {
  if (fwd) {
    switch (R) {
      case 1: run_fold_band<V, true, 1, TPB>(sm, g, logL, cs); break;
      case 2: run_fold_band<V, true, 2, TPB>(sm, g, logL, cs); break;
      case 3: run_fold_band<V, true, 3, TPB>(sm, g, logL, cs); break;
      default: run_fold_band<V, true, 4, TPB>(sm, g, logL, cs); break;
    }
  } else {
    switch (R) {
      case 1: run_fold_band<V, false, 1, TPB>(sm, g, logL, cs); break;
      case 2: run_fold_band<V, false, 2, TPB>(sm, g, logL, cs); break;
      case 3: run_fold_band<V, false, 3, TPB>(sm, g, logL, cs); break;
      default: run_fold_band<V, false, 4, TPB>(sm, g, logL, cs); break;
    }
  }
}

template <int V, int TPB>
__device__ __forceinline__ void run_chunk_band_r(float* sm, float* snap, const Geo& g, int logL, int R) {
  switch (R) {
    case 1: run_chunk_band<V, 1, TPB>(sm, snap, g, logL); break;
    case 2: run_chunk_band<V, 2, TPB>(sm, snap, g, logL); break;
    case 3: run_chunk_band<V, 3, TPB>(sm, snap, g, logL); break;
    default: run_chunk_band<V, 4, TPB>(sm, snap, g, logL); break;
  }
}

// Band plan: pass levels (node sizes N/4 .. 2*LEAF) split into bands of at
// most RMAX levels, as even as possible, the top band first.  The multi-pass
// path uses the same split for the levels above its subproblem size.
struct BandPlan {
  int nb;
  int logL[4];  // four bands of up to RMAX levels: the 13 levels above 2^13 of N = 2^28
  int R[4];
};

__host__ __device__ __forceinline__ BandPlan band_plan(int logN, int log_bottom = LOG_LEAF) {
  BandPlan b;
  int nl = logN - 2 - log_bottom;
  int top = logN - 2;
  b.nb = 0;
  while (nl > 0 && b.nb < 4) {
    const int nbands = (nl + RMAX - 1) / RMAX;
    const int R = (nl + nbands - 1) / nbands;
    b.logL[b.nb] = top;
    b.R[b.nb] = R;
    ++b.nb;
    top -= R;
    nl -= R;
  }
  return b;
}

// snapshot floats needed by a chunk band over `values` region values of a
// CTA: items = values / 2^R, 2 run ends of 2^R values per 32 items
__host__ __device__ constexpr int snap_floats(int values) { return values / 16 + 64; }

}  // namespace amqft
