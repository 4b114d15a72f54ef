// Device code of the fused AM-QFT kernel ("A class of AM-QFT algorithms for
// power-of-two FFT", Pasquini).  One complex transform of length N = 2^logN
// is split by D_c (Sect. 3.1) and D_r (Sect. 3.2) into four real "regions"
// held in shared memory:
//     C1 = DCT-0 of Re x   S1 = DST-0 of Re x   C2 = DCT-0 of Im x   S2 = DST-0 of Im x
// (Eq. qft_0B-0C), in that order, so a region's context is (index & 1):
// 0 = DCT, 1 = DST.  Each region is laid out as the chain of its recursion:
//
//   variants 1,4,5,8 (time indices first, Sect. 6.9):
//     dct(M) = D_n -> dct(M/2) + dct_ot(M); the dct_ot(M) tree of L = M/4
//     values sits at [half - 2L, half - L) (half = N/2), the dct(2) base at
//     [half-1, half+1) (DST region: dst_ot trees down to L = 2, the dst(4)
//     base at half-2).  A tree node of size L splits by D_k (Tab. 4) into
//     children of L/2 each, the oo child going through M_v (Tab. 5-6).
//   variants 2,3,6,7 (harmonics first): dct(M) = D_k -> dct(M/2) + dct_to(M),
//     the dct_to trees at the same places, nodes split by D_n.
//
// Layout rules (they make every pass a local or in-place operation):
//   * time-domain data of an ot tree is in natural order; frequency-domain
//     data of every tree node is in bit-reversed order (S[k] at brev(k));
//     for to trees it is the other way round (time bit-reversed, frequency
//     natural).
//   * a node of DCT context keeps its A child (the e-child of D_k or D_n) in
//     its first half and its B child (the oo signal after M_v) in its second
//     half; a DST-context node swaps the two halves.  With that rule the
//     interleave of the two children's results is exactly the bit reversal.
//     For the variants that swap contexts in M_v (5-8) it also makes a
//     non-root node's context equal to the half of its parent it sits in.
//
// All arithmetic is float32 with no contraction into FMA (the library is
// built with -fmad=false): the kernel performs, for every output, the same
// operations in the same order as the paper's recursion, so variants 2, 4, 6
// and 8 are bit-identical to a float32 evaluation of the recursion.
// Variants 1, 3, 5, 7 contain first-order recurrences (M1, M3, M5, M7); on
// levels wider than a register subtree they are evaluated as chunked scans
// (sequential within a chunk, carries between chunks), which changes the
// rounding order there.
#pragma once

#include <cooperative_groups.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "amqft_debug.cuh"

namespace amqft {
namespace cg = cooperative_groups;

constexpr int LOG_LEAF = 5;
constexpr int LEAF = 1 << LOG_LEAF;  // register-resident subtree size

// Trig constants of the small periodisations M = 16 .. 4*LEAF, passed as a
// kernel parameter so register subtrees read them from the constant bank.
// Level-major layout, identical to the device table: periodisation M holds
// its M/8 constants (angle 2*pi*(2j+1)/M) at [M/8 - 2, M/4 - 2).
struct SmallConsts {
  float c[LEAF - 2];
  float cos_pi4;  // common constant of the N = 8 base cases (Sect. 7.1)
};

struct FusedArgs {
  const void* in;      // complex64, or 16-bit complex pairs (dtype)
  void* out;
  const int* exp_in;   // 16-bit input: per-transform exponents (NULL: all 0)
  int* exp_out;        // 16-bit output: per-transform exponents
  int dtype;           // 0 complex64, 1 bf16 pairs, 2 fp16 pairs
  const float* ctab;   // device constant table, level-major, N/4 - 2 floats
  long long batch;
  int logN;
  int tpc;             // transforms per CTA (cluster size 1)
  int inverse;         // 1: conj in / conj out
  int RS;              // region stride in floats
  int tot_off;         // float offset of the scan scratch in shared memory
  const int* tlist;    // transform ids by list position (NULL: the position itself)
  const long long* toff;  // element offset of each transform id (NULL: id * N)
  long long nreal;     // > 0: real input, transform t = real signals 2t and 2t+1
                       // (float32, N each, the second absent past nreal); out holds
                       // the N/2 + 1 harmonics of every signal (forward only)
  long long ntrig;     // > 0: DCT-0 / DST-0 (Eq. qft_0B-0C) of ntrig signals of each
                       // kind, transform t = signals 2t and 2t+1: regions C1 / C2 take
                       // DCT-0 inputs (in: N/2 + 1 floats each, n = 0..N/2), S1 / S2
                       // DST-0 inputs (in2: N/2 - 1 floats, n = 1..N/2-1 at [n-1]);
                       // results alike at out / out2 (a NULL pair: that kind absent)
  const float* in2;
  float* out2;
  long long nirdft;    // > 0: inverse real transform of nirdft half spectra (in:
                       // N/2 + 1 complex64 each), transform t = spectra 2t and 2t+1 as
                       // Z = X_a + i X_b; out: the real signals, N floats each
};

template <int V>
struct Var {
  static constexpr bool ot = (V == 1 || V == 4 || V == 5 || V == 8);
  static constexpr bool flip = (V >= 5);
  static constexpr bool scan = (V == 1 || V == 3 || V == 5 || V == 7);
};

// ---------------------------------------------------------------------
// small helpers
// ---------------------------------------------------------------------
__device__ __forceinline__ int sw(int p) { return p ^ ((p >> 5) & 31); }

__device__ __forceinline__ int brev(int x, int bits) {
  return bits ? (int)(__brev((unsigned)x) >> (32 - bits)) : 0;
}

__host__ __device__ constexpr int brev_c(int x, int bits) {
  int r = 0;
  for (int i = 0; i < bits; ++i) r = (r << 1) | ((x >> i) & 1);
  return r;
}

__host__ __device__ constexpr int ilog2_c(int x) { return x <= 1 ? 0 : 1 + ilog2_c(x >> 1); }

// n / d for the small operands of the pass decompositions (n * d < 2^40).
struct Div {
  unsigned d, m;
  __device__ __forceinline__ explicit Div(unsigned dd) : d(dd), m(dd > 1 ? 0xFFFFFFFFu / dd + 1u : 0u) {}
  __device__ __forceinline__ unsigned operator()(unsigned n) const {
    unsigned q = d > 1 ? __umulhi(n, m) : n;
    int r = (int)(n - q * d);
    if (r < 0) --q; else if (r >= (int)d) ++q;
    return q;
  }
};

// Shared-memory stride of one region of a transform of 2^logN: N/2 + 2
// values, padded to whole 32-float rows from N = 128 on (so the swizzle stays
// inside the region).
__host__ __device__ constexpr int region_stride(int logN) {
  return logN >= 7 ? (((1 << (logN - 1)) + 2 + 31) / 32) * 32 : (((logN >= 1 ? (1 << (logN - 1)) : 0) + 3) / 2) * 2;
}

// Launch shapes of the fused kernel, shared by every launch site and by the
// host's shared-memory sizing.  N <= 2^13: one CTA of SMALL_TPB threads holds
// 16384 region values (two CTAs per SM); 2^14..2^16: clusters of four CTAs,
// one region each.  MAXI bounds the items a thread takes in the per-level
// passes (MAXI * TPB must cover half a region).
// ot: a time-first variant (1, 4, 5, 8), whose 2^14 kernel runs 128 threads
// and four CTAs per SM (the harmonics-first variants' per-level neighbour
// passes are faster with 256 threads).
constexpr int SMALL_TPB = 256, SMALL_MAXI = 32;
__host__ __device__ constexpr bool variant_ot(int v) { return v == 1 || v == 4 || v == 5 || v == 8; }
__host__ __device__ constexpr int cluster_tpb(int logN, bool ot) {
  return logN == 16 ? 1024 : (logN == 14 && ot ? 128 : 256);
}
// items per thread that cover half a region (N/4) in the per-level passes, at least 16
__host__ __device__ constexpr int cluster_maxi(int logN, bool ot) {
  return (1 << (logN - 2)) / cluster_tpb(logN, ot) > 16 ? (1 << (logN - 2)) / cluster_tpb(logN, ot) : 16;
}
// CTAs per SM a kernel of TPB threads is compiled for (at most 128 registers a thread below 1024)
__host__ __device__ constexpr int ctas_per_sm(int tpb) { return tpb <= 128 ? 4 : (tpb <= 256 ? 2 : 1); }
static_assert(SMALL_TPB * SMALL_MAXI >= 8192, "per-level passes of the single-CTA path");
static_assert(cluster_tpb(14, true) * cluster_maxi(14, true) >= (1 << 12) &&
                  cluster_tpb(14, false) * cluster_maxi(14, false) >= (1 << 12) &&
                  cluster_tpb(15, true) * cluster_maxi(15, true) >= (1 << 13) &&
                  cluster_tpb(16, true) * cluster_maxi(16, true) >= (1 << 14),
              "per-level passes of the cluster path");

// Context (0 DCT, 1 DST) of the tree node of size 2^logLp at region position p0.
template <int V>
__device__ __forceinline__ int node_ctx(int p0, int logLp, int half, int ctx0) {
  if constexpr (!Var<V>::flip) {
    return ctx0;
  } else {
    const int d = half - p0;                       // tree t covers [half-2Lt, half-Lt)
    const int Lt = 1 << (31 - __clz(d - 1));
    if ((1 << logLp) == Lt) return ctx0;           // tree root
    return ((p0 - (half - 2 * Lt)) >> logLp) & 1;  // which half of its parent
  }
}

// Position of sample / harmonic m of a region in the chain layout (the
// selections D_n of Sect. 6.9 applied down to the base case).
__device__ __forceinline__ int pos_chain(int m, int logN, int kind) {
  const int half = 1 << (logN - 1);
  if (kind == 0) {
    if (m == 0) return half - 1;
    if (m == half) return half;
  } else if (m == (half >> 1)) {
    return half - 2;
  }
  const int t = __ffs(m) - 1;
  return half - (1 << (logN - t - 1)) + (m >> (t + 1));
}

// ---------------------------------------------------------------------
// register subtrees: the recursion of Sect. 4-6 on arrays in registers
// ---------------------------------------------------------------------
// M_v frequency phase for the ot functions (variants 1,4,5,8), Tab. 5-6.
template <int V, int CTX, int H>
__device__ __forceinline__ void mvf_ot(const float (&b)[H], float (&o)[H]) {
  if constexpr (V == 4) {
    if constexpr (CTX == 0) {
#pragma unroll
      for (int j = 0; j < H - 1; ++j) o[j] = b[j] + b[j + 1];
      o[H - 1] = b[H - 1];
    } else {
      o[0] = b[0];
#pragma unroll
      for (int j = 1; j < H; ++j) o[j] = b[j - 1] + b[j];
    }
  } else if constexpr (V == 8) {
    if constexpr (CTX == 0) {
      o[0] = b[0];
#pragma unroll
      for (int j = 1; j < H; ++j) o[j] = b[j] - b[j - 1];
    } else {
#pragma unroll
      for (int j = 0; j < H - 1; ++j) o[j] = b[j] - b[j + 1];
      o[H - 1] = b[H - 1];
    }
  } else if constexpr (V == 1) {
    if constexpr (CTX == 0) {
      o[0] = 0.5f * b[0];
#pragma unroll
      for (int j = 1; j < H; ++j) o[j] = b[j] - o[j - 1];
    } else {
      o[H - 1] = 0.5f * b[H - 1];
#pragma unroll
      for (int j = H - 2; j >= 0; --j) o[j] = b[j] - o[j + 1];
    }
  } else {  // V == 5
    if constexpr (CTX == 0) {
      o[H - 1] = 0.5f * b[H - 1];
#pragma unroll
      for (int j = H - 2; j >= 0; --j) o[j] = b[j] + o[j + 1];
    } else {
      o[0] = 0.5f * b[0];
#pragma unroll
      for (int j = 1; j < H; ++j) o[j] = b[j] + o[j - 1];
    }
  }
}

// M_v time phase for the to functions (variants 2,3,6,7), Tab. 5-6.
template <int V, int CTX, int H>
__device__ __forceinline__ void mvt_to(const float (&x)[H], float (&y)[H]) {
  if constexpr (V == 2) {
    if constexpr (CTX == 0) {
      y[0] = x[0];
#pragma unroll
      for (int i = 1; i < H; ++i) y[i] = x[i] + x[i - 1];
    } else {
      y[H - 1] = x[H - 1];
#pragma unroll
      for (int i = 0; i < H - 1; ++i) y[i] = x[i] + x[i + 1];
    }
  } else if constexpr (V == 6) {
    if constexpr (CTX == 0) {
      y[H - 1] = x[H - 1];
#pragma unroll
      for (int i = 0; i < H - 1; ++i) y[i] = x[i] - x[i + 1];
    } else {
      y[0] = x[0];
#pragma unroll
      for (int i = 1; i < H; ++i) y[i] = x[i] - x[i - 1];
    }
  } else if constexpr (V == 3) {
    if constexpr (CTX == 0) {
      y[H - 1] = x[H - 1];
#pragma unroll
      for (int i = H - 2; i >= 1; --i) y[i] = x[i] - y[i + 1];
      y[0] = 0.5f * (x[0] - y[1]);
    } else {
      y[0] = x[0];
#pragma unroll
      for (int i = 1; i <= H - 2; ++i) y[i] = x[i] - y[i - 1];
      y[H - 1] = 0.5f * (x[H - 1] - y[H - 2]);
    }
  } else {  // V == 7
    if constexpr (CTX == 0) {
      y[0] = x[0];
#pragma unroll
      for (int i = 1; i <= H - 2; ++i) y[i] = x[i] + y[i - 1];
      y[H - 1] = 0.5f * (x[H - 1] + y[H - 2]);
    } else {
      y[H - 1] = x[H - 1];
#pragma unroll
      for (int i = H - 2; i >= 1; --i) y[i] = x[i] + y[i + 1];
      y[0] = 0.5f * (x[0] + y[1]);
    }
  }
}

// dct_ot(4L) (CTX 0) or dst_ot(4L) (CTX 1): time values x[0..L) (odd n, natural)
// in, results (natural k) out.
template <int V, int L, int CTX>
__device__ __forceinline__ void ot_rec(float (&x)[L], const SmallConsts& K) {
  if constexpr (L >= 2) {
    constexpr int H = L / 2;
    float a[H], b[H];
#pragma unroll
    for (int i = 0; i < H; ++i) {
      const float u = x[i], w = x[L - 1 - i];
      float s, d;
      if constexpr (CTX == 0) { s = u + w; d = u - w; } else { s = u - w; d = u + w; }
      a[i] = s;
      if constexpr (L == 2) b[i] = d * K.cos_pi4; else b[i] = d * K.c[L / 2 - 2 + i];
    }
    ot_rec<V, H, CTX>(a, K);
    constexpr int CB = Var<V>::flip ? 1 - CTX : CTX;
    ot_rec<V, H, CB>(b, K);
    float o[H];
    if constexpr (L == 2) {
      o[0] = b[0];
    } else {
      mvf_ot<V, CTX, H>(b, o);
    }
#pragma unroll
    for (int i = 0; i < H; ++i) {
      if constexpr (CTX == 0) { x[2 * i] = a[i]; x[2 * i + 1] = o[i]; }
      else { x[2 * i] = o[i]; x[2 * i + 1] = a[i]; }
    }
  }
}

// dct_to(4L) (CTX 0) or dst_to(4L) (CTX 1): time values (natural) in, odd-k
// results (natural) out.
template <int V, int L, int CTX>
__device__ __forceinline__ void to_rec(float (&x)[L], const SmallConsts& K) {
  if constexpr (L >= 2) {
    constexpr int H = L / 2;
    float a[H], ov[H], b[H];
#pragma unroll
    for (int i = 0; i < H; ++i) {
      if constexpr (CTX == 0) { a[i] = x[2 * i]; ov[i] = x[2 * i + 1]; }
      else { a[i] = x[2 * i + 1]; ov[i] = x[2 * i]; }
    }
    if constexpr (L == 2) b[0] = ov[0] * K.cos_pi4; else mvt_to<V, CTX, H>(ov, b);
    to_rec<V, H, CTX>(a, K);
    constexpr int CB = Var<V>::flip ? 1 - CTX : CTX;
    to_rec<V, H, CB>(b, K);
#pragma unroll
    for (int j = 0; j < H; ++j) {
      float o;
      if constexpr (L == 2) o = b[j]; else o = b[j] * K.c[L / 2 - 2 + j];
      if constexpr (CTX == 0) { x[j] = a[j] + o; x[L - 1 - j] = a[j] - o; }
      else { x[j] = o + a[j]; x[L - 1 - j] = o - a[j]; }
    }
  }
}

// ---------------------------------------------------------------------
// tails: the trees smaller than LEAF plus the bottom of the chain, one
// thread per region.  TH = min(LEAF, N/2); the chain is carried up to
// TOPM = 2*TH (or to N/2 when TH = N/2).
// ---------------------------------------------------------------------
template <int SZ, int OFF, int L>
__device__ __forceinline__ void get_sub(const float (&t)[SZ], float (&x)[L]) {
#pragma unroll
  for (int e = 0; e < L; ++e) x[e] = t[OFF + e];
}
template <int SZ, int OFF, int L>
__device__ __forceinline__ void put_sub(float (&t)[SZ], const float (&x)[L]) {
#pragma unroll
  for (int e = 0; e < L; ++e) t[OFF + e] = x[e];
}

template <int V, int CTX, bool OT, int SZ, int TH, int L>
__device__ __forceinline__ void tail_trees(float (&t)[SZ], const SmallConsts& K) {
  if constexpr (L >= (CTX == 0 ? 1 : 2)) {
    float x[L];
    get_sub<SZ, TH - 2 * L, L>(t, x);
    if constexpr (OT) ot_rec<V, L, CTX>(x, K); else to_rec<V, L, CTX>(x, K);
    put_sub<SZ, TH - 2 * L, L>(t, x);
    tail_trees<V, CTX, OT, SZ, TH, L / 2>(t, K);
  }
}

// D_n backward of dct(M) (time-first variants): S from E = dct(M/2), O = dct_ot(M).
template <int SZ, int TH, int M, int TOPM>
__device__ __forceinline__ void chain_up_dct(float (&t)[SZ]) {
  if constexpr (M <= TOPM) {
    constexpr int P = TH - M / 2, Q = M / 4;
    float s[M / 2 + 1];
#pragma unroll
    for (int k = 0; k < Q; ++k) {
      const float e = t[P + Q + k], o = t[P + k];
      s[k] = e + o;
      s[M / 2 - k] = e - o;
    }
    s[Q] = t[P + 2 * Q];
#pragma unroll
    for (int k = 0; k <= M / 2; ++k) t[P + k] = s[k];
    chain_up_dct<SZ, TH, 2 * M, TOPM>(t);
  }
}

template <int SZ, int TH, int M, int TOPM>
__device__ __forceinline__ void chain_up_dst(float (&t)[SZ]) {
  if constexpr (M <= TOPM) {
    constexpr int P = TH - M / 2, Q = M / 4;
    float s[M / 2 - 1];
#pragma unroll
    for (int k = 1; k < Q; ++k) {
      const float o = t[P + k - 1], e = t[P + Q + k - 1];
      s[k - 1] = o + e;
      s[M / 2 - k - 1] = o - e;
    }
    s[Q - 1] = t[P + Q - 1];
#pragma unroll
    for (int k = 0; k < M / 2 - 1; ++k) t[P + k] = s[k];
    chain_up_dst<SZ, TH, 2 * M, TOPM>(t);
  }
}

// D_k forward of dct(M) (harmonics-first variants): te -> dct(M/2), to -> dct_to(M).
template <int SZ, int TH, int M>
__device__ __forceinline__ void chain_down_dct(float (&t)[SZ]) {
  if constexpr (M >= 4) {
    constexpr int P = TH - M / 2, Q = M / 4;
    float te[Q + 1], to[Q];
#pragma unroll
    for (int n = 0; n < Q; ++n) {
      const float a = t[P + n], b = t[P + M / 2 - n];
      te[n] = a + b;
      to[n] = a - b;
    }
    te[Q] = t[P + Q];
#pragma unroll
    for (int n = 0; n < Q; ++n) t[P + n] = to[n];
#pragma unroll
    for (int n = 0; n <= Q; ++n) t[P + Q + n] = te[n];
    chain_down_dct<SZ, TH, M / 2>(t);
  }
}

template <int SZ, int TH, int M>
__device__ __forceinline__ void chain_down_dst(float (&t)[SZ]) {
  if constexpr (M >= 8) {
    constexpr int P = TH - M / 2, Q = M / 4;
    float te[Q - 1], to[Q];
#pragma unroll
    for (int n = 1; n < Q; ++n) {
      const float a = t[P + n - 1], b = t[P + M / 2 - n - 1];
      te[n - 1] = a - b;
      to[n - 1] = a + b;
    }
    to[Q - 1] = t[P + Q - 1];
#pragma unroll
    for (int n = 0; n < Q; ++n) t[P + n] = to[n];
#pragma unroll
    for (int n = 0; n < Q - 1; ++n) t[P + Q + n] = te[n];
    chain_down_dst<SZ, TH, M / 2>(t);
  }
}

template <int V, int TH, int TOPM>
__device__ __forceinline__ void tail_dct(RegP R, int half, const SmallConsts& K) {
  constexpr int SZ = TH + 1;
  constexpr int LT = TH / 2;  // size of the top tail tree
  const int base = half - TH;
  float t[SZ];
  const bool top_brev = (TOPM == TH) && (LT >= 2);
  if constexpr (Var<V>::ot) {
#pragma unroll
    for (int e = 0; e < SZ; ++e) t[e] = R[sw(base + e)];
    tail_trees<V, 0, true, SZ, TH, LT>(t, K);
    if constexpr (TH >= 1) {
      const float a = t[TH - 1], b = t[TH];
      t[TH - 1] = a + b;
      t[TH] = a - b;
    }
    chain_up_dct<SZ, TH, 4, TOPM>(t);
    if (top_brev) {
#pragma unroll
      for (int e = 0; e < SZ; ++e) {
        const int p = (e < LT) ? brev_c(e, ilog2_c(LT)) : e;
        R[sw(base + p)] = t[e];
      }
    } else {
#pragma unroll
      for (int e = 0; e < SZ; ++e) R[sw(base + e)] = t[e];
    }
  } else {
#pragma unroll
    for (int e = 0; e < SZ; ++e) {
      const int p = (top_brev && e < LT) ? brev_c(e, ilog2_c(LT)) : e;
      t[e] = R[sw(base + p)];
    }
    chain_down_dct<SZ, TH, TOPM>(t);
    if constexpr (TH >= 1) {
      const float a = t[TH - 1], b = t[TH];
      t[TH - 1] = a + b;
      t[TH] = a - b;
    }
    tail_trees<V, 0, false, SZ, TH, LT>(t, K);
#pragma unroll
    for (int e = 0; e < SZ; ++e) R[sw(base + e)] = t[e];
  }
}

template <int V, int TH, int TOPM>
__device__ __forceinline__ void tail_dst(RegP R, int half, const SmallConsts& K) {
  if constexpr (TH >= 2) {
    constexpr int SZ = TH - 1;
    constexpr int LT = TH / 2;
    const int base = half - TH;
    const bool top_brev = (TOPM == TH) && (LT >= 2);
    float t[SZ];
    if constexpr (Var<V>::ot) {
#pragma unroll
      for (int e = 0; e < SZ; ++e) t[e] = R[sw(base + e)];
      tail_trees<V, 1, true, SZ, TH, LT>(t, K);
      chain_up_dst<SZ, TH, 8, TOPM>(t);
      if (top_brev) {
#pragma unroll
        for (int e = 0; e < SZ; ++e) {
          const int p = (e < LT) ? brev_c(e, ilog2_c(LT)) : e;
          R[sw(base + p)] = t[e];
        }
      } else {
#pragma unroll
        for (int e = 0; e < SZ; ++e) R[sw(base + e)] = t[e];
      }
    } else {
#pragma unroll
      for (int e = 0; e < SZ; ++e) {
        const int p = (top_brev && e < LT) ? brev_c(e, ilog2_c(LT)) : e;
        t[e] = R[sw(base + p)];
      }
      chain_down_dst<SZ, TH, TOPM>(t);
      tail_trees<V, 1, false, SZ, TH, LT>(t, K);
#pragma unroll
      for (int e = 0; e < SZ; ++e) R[sw(base + e)] = t[e];
    }
  }
}

template <int V>
__device__ __noinline__ void run_tail(RegP R, int ctx0, int logN, const SmallConsts& K) {
  const int half = 1 << (logN - 1);
#define AMQFT_TAIL(TH, TOPM)                                      \
  if (ctx0 == 0) tail_dct<V, TH, TOPM>(R, half, K);              \
  else tail_dst<V, TH, TOPM>(R, half, K);
  switch (logN) {
    case 1: AMQFT_TAIL(1, 1) break;
    case 2: AMQFT_TAIL(2, 2) break;
    case 3: AMQFT_TAIL(4, 4) break;
    case 4: AMQFT_TAIL(8, 8) break;
    case 5: AMQFT_TAIL(16, 16) break;
    case 6: AMQFT_TAIL(32, 32) break;
    default: AMQFT_TAIL(32, 64) break;
  }
#undef AMQFT_TAIL
}

// A register subtree of LEAF values: ot trees read time values in natural
// order and write results bit-reversed; to trees the other way round.
template <int V>
__device__ __noinline__ void run_leaf(RegP R, int p0, int ctx, const SmallConsts& K) {
  float x[LEAF];
  const int f = (p0 >> 5) & 31;  // sw() of a LEAF-aligned row
  if constexpr (Var<V>::ot) {
#pragma unroll
    for (int e = 0; e < LEAF; ++e) x[e] = R[p0 + (e ^ f)];
    if (ctx == 0) ot_rec<V, LEAF, 0>(x, K); else ot_rec<V, LEAF, 1>(x, K);
#pragma unroll
    for (int k = 0; k < LEAF; ++k) R[p0 + (brev_c(k, LOG_LEAF) ^ f)] = x[k];
  } else {
#pragma unroll
    for (int n = 0; n < LEAF; ++n) x[n] = R[p0 + (brev_c(n, LOG_LEAF) ^ f)];
    if (ctx == 0) to_rec<V, LEAF, 0>(x, K); else to_rec<V, LEAF, 1>(x, K);
#pragma unroll
    for (int k = 0; k < LEAF; ++k) R[p0 + (k ^ f)] = x[k];
  }
}

// ---------------------------------------------------------------------
// block-wide passes over all regions of the CTA (one tree level each)
// ---------------------------------------------------------------------
// Shared-memory geometry.  Region mode (sub == 0): nreg chain-layout
// regions of N/2 (+2) values.  Node mode (sub > 0): one tree node of sub
// values at [0, sub) whose root context is gbase & 1 (a subproblem of the
// multi-pass path).
struct Geo {
  int logN, half, RS, nreg, gbase, sub;
  int nreg_cap;  // regions a full CTA holds: fixes the scan chunking, so a
                 // transform's rounding does not depend on its batch neighbours
};

// Transforms per CTA of the single-CTA path (N <= 2^13): 16384 region values.
__host__ __device__ constexpr int small_tpc(int logN) { return (512 * 32) / ((1 << logN) >= 4 ? 2 * (1 << logN) : 8); }

// Constants of the band levels of a transform of 2^logN (node sizes 2^6 ..
// N/4, periodisations 256 .. N: table entries 30 .. N/4 - 3), staged per CTA
// in shared memory after the exponent slots.
__host__ __device__ constexpr int band_consts(int logN) { return logN >= 8 ? (1 << (logN - 2)) - 32 : 0; }

// context of region (or node) r: region mode, C1 S1 C2 S2 alternate DCT/DST;
// node mode, gbase is a bit mask of the nodes' root contexts
__device__ __forceinline__ int ctx_of(const Geo& g, int r) {
  return g.sub ? ((g.gbase >> r) & 1) : ((g.gbase + r) & 1);
}

// class-0 nodes of size 2^logLp: blocks [0, half - Lp) in region mode, the
// whole node range [0, sub) in node mode
__device__ __forceinline__ unsigned nodes_at(const Geo& g, int logLp) {
  return g.sub ? (unsigned)(g.sub >> logLp) : (unsigned)(g.half >> logLp) - 1u;
}

template <int V>
__device__ __forceinline__ int node_ctx_g(const Geo& g, int p0, int logLp, int ctx0) {
  if constexpr (!Var<V>::flip) {
    return ctx0;
  } else {
    if (g.sub) return (1 << logLp) == g.sub ? ctx0 : ((p0 >> logLp) & 1);
    return node_ctx<V>(p0, logLp, g.half, ctx0);
  }
}

// Neighbour form of M_v on the B half (bit-reversed order): the frequency
// phase of M4/M8 (ot variants) or the time phase of M2/M6 (to variants).
// Two phases: every thread reads, barrier, every thread writes.
template <int V, int TPB, int MAXI>
__device__ __forceinline__ void pass_neighbour(float* sm, const Geo& g, int logLp) {
  const int Lp = 1 << logLp, H = Lp >> 1, h = logLp - 1;
  const unsigned nb = nodes_at(g, logLp);
  const unsigned Wr = nb << h, W = Wr * (unsigned)g.nreg;
  const Div dv(Wr);
  float val[MAXI];
#pragma unroll
  for (int s = 0; s < MAXI; ++s) {
    const unsigned w = threadIdx.x + (unsigned)s * TPB;
    if (w < W) {
      const unsigned r = dv(w), rem = w - r * Wr;
      const int b = (int)(rem >> h), q = (int)(rem & (H - 1)), i = brev(q, h);
      CRegP R = creg_ptr(sm + r * g.RS, g.RS);
      const int p0 = b << logLp;
      const int ctx = node_ctx_g<V>(g, p0, logLp, ctx_of(g, r));
      const int base = ctx == 0 ? p0 + H : p0;
      const float bi = R[sw(base + q)];
      float o = bi;
      // which neighbour (+1 / -1) and whether it is added or subtracted
      int dir;
      bool add;
      if constexpr (V == 4) { dir = ctx == 0 ? +1 : -1; add = true; }
      else if constexpr (V == 8) { dir = ctx == 0 ? -1 : +1; add = false; }
      else if constexpr (V == 2) { dir = ctx == 0 ? -1 : +1; add = true; }
      else { dir = ctx == 0 ? +1 : -1; add = false; }  // V == 6
      const int jn = i + dir;
      if (jn >= 0 && jn < H) {
        const float bn = R[sw(base + brev(jn, h))];
        if (add) o = (dir > 0) ? (bi + bn) : (bn + bi);
        else o = bi - bn;
      }
      val[s] = o;
    }
  }
  __syncthreads();
#pragma unroll
  for (int s = 0; s < MAXI; ++s) {
    const unsigned w = threadIdx.x + (unsigned)s * TPB;
    if (w < W) {
      const unsigned r = dv(w), rem = w - r * Wr;
      const int b = (int)(rem >> h), q = (int)(rem & (H - 1));
      RegP R = reg_ptr(sm + r * g.RS, g.RS);
      const int p0 = b << logLp;
      const int ctx = node_ctx_g<V>(g, p0, logLp, ctx_of(g, r));
      const int base = ctx == 0 ? p0 + H : p0;
      R[sw(base + q)] = val[s];
    }
  }
}

// Segmented exclusive scan of tot[0..n) (segments of 2^logSL, all threads).
template <int TPB>
__device__ __forceinline__ void seg_excl_scan(float* tot, float* wsum, int n, int logSL) {
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int SL = 1 << logSL, width = SL < 32 ? SL : 32;
  const float v = (t < n) ? tot[t] : 0.f;
  float incl = v;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const float o = __shfl_up_sync(0xffffffffu, incl, d);
    if (d < width && (lane & (width - 1)) >= d) incl = incl + o;
  }
  float excl = __shfl_up_sync(0xffffffffu, incl, 1);
  if ((lane & (width - 1)) == 0) excl = 0.f;
  if (SL > 32) {
    __syncthreads();
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    if (warp == 0) {
      constexpr int NW = TPB / 32;
      const int ww = SL >> 5;  // warps per segment (<= NW)
      const float wv = (lane < NW) ? wsum[lane] : 0.f;
      float wi = wv;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const float o = __shfl_up_sync(0xffffffffu, wi, d);
        if (d < ww && (lane & (ww - 1)) >= d) wi = wi + o;
      }
      float we = __shfl_up_sync(0xffffffffu, wi, 1);
      if ((lane & (ww - 1)) == 0) we = 0.f;
      if (lane < NW) wsum[lane] = we;
    }
    __syncthreads();
    excl = excl + wsum[warp];
  }
  __syncthreads();
  if (t < n) tot[t] = excl;
  __syncthreads();
}

// Recurrence form of M_v on the B half (bit-reversed order): the frequency
// phase of M1/M5 (ot variants; the first element is halved) or the time
// phase of M3/M7 (to variants; the last element is halved).  Chunks of C
// consecutive elements are run sequentially by one thread each; the carries
// between chunks come from a segmented scan of the chunk totals.  The
// chunking follows CTPB threads (<= TPB; the rest stay idle here), so a
// kernel shape with more threads can give the same bits as one with CTPB;
// MAXI bounds the chunk length.
template <int V, int TPB, int MAXI, int CTPB = TPB>
__device__ __forceinline__ void pass_recurrence(float* sm, float* tot, float* wsum, const Geo& g, int logLp) {
  static_assert(CTPB <= TPB, "the chunking's threads");
  constexpr bool hstart = Var<V>::ot;
  constexpr bool alt = (V == 1 || V == 3);
  const int Lp = 1 << logLp, H = Lp >> 1, h = logLp - 1;
  const unsigned nb = nodes_at(g, logLp);
  const unsigned total = nb * (unsigned)H * (unsigned)g.nreg;
  const unsigned total_cap = nb * (unsigned)H * (unsigned)g.nreg_cap;
  int logC = 1;
  while (((unsigned)CTPB << logC) < total_cap) ++logC;
  const int C = 1 << logC, logSC = h - logC, SC = 1 << logSC;
  const unsigned nch = total >> logC;
  const Div dv(nb);
  const int tau = threadIdx.x;
  float l[MAXI];
  int base = 0, k = 0, kidx = 0;
  bool prefix = true;
  RegP R = reg_ptr(sm, g.RS);
  if ((unsigned)tau < nch) {
    const int seg = tau >> logSC, col = tau & (SC - 1);
    const unsigned r = dv((unsigned)seg), b = (unsigned)seg - r * nb;
    R = reg_ptr(sm + r * g.RS, g.RS);
    const int p0 = (int)(b << logLp);
    const int ctx = node_ctx_g<V>(g, p0, logLp, ctx_of(g, r));
    base = ctx == 0 ? p0 + H : p0;
    if constexpr (V == 1) prefix = ctx == 0;
    else if constexpr (V == 5) prefix = ctx == 1;
    else if constexpr (V == 3) prefix = ctx == 1;
    else prefix = ctx == 0;  // V == 7
    k = prefix ? brev(col, logSC) : SC - 1 - brev(col, logSC);
    kidx = (seg << logSC) + k;
    float prev = 0.f;
#pragma unroll
    for (int e = 0; e < MAXI; ++e) {
      if (e < C) {
        const int m = k * C + e;
        const int i = prefix ? m : H - 1 - m;
        const float xv = R[sw(base + brev(i, h))];
        float y;
        if (hstart && k == 0 && e == 0) y = 0.5f * xv;
        else y = alt ? (xv - prev) : (xv + prev);
        l[e] = y;
        prev = y;
      }
    }
    tot[kidx] = prev;
  }
  __syncthreads();
  seg_excl_scan<TPB>(tot, wsum, (int)nch, logSC);
  if ((unsigned)tau < nch) {
    const float c = tot[kidx];
#pragma unroll
    for (int e = 0; e < MAXI; ++e) {
      if (e < C) {
        const int m = k * C + e;
        const int i = prefix ? m : H - 1 - m;
        float y;
        if (alt) y = (e & 1) ? (l[e] + c) : (l[e] - c);
        else y = l[e] + c;
        if (!hstart && k == SC - 1 && e == C - 1) y = 0.5f * y;
        R[sw(base + brev(i, h))] = y;
      }
    }
  }
}

// Chain level M = 2^logM, two phases.  ot variants: D_n frequency phase
// (dct: S(k)=E(k)+O(k), S(M/2-k)=E(k)-O(k); dst analogous).  to variants:
// D_k time phase (te -> dct(M/2), to -> dct_to(M) written bit-reversed).
template <int V, int TPB, int MAXI>
__device__ __forceinline__ void pass_chain(float* sm, const Geo& g, int logM) {
  constexpr int NI = MAXI / 2 > 0 ? MAXI / 2 : 1;
  const int M = 1 << logM, logQ = logM - 2, Q = 1 << logQ, P = g.half - M / 2;
  const unsigned W = (unsigned)g.nreg << logQ;
  float v0[NI], v1[NI], v2[NI];
#pragma unroll
  for (int s = 0; s < NI; ++s) {
    const unsigned w = threadIdx.x + (unsigned)s * TPB;
    if (w < W) {
      const int r = (int)(w >> logQ), k = (int)(w & (Q - 1));
      CRegP R = creg_ptr(sm + r * g.RS, g.RS);
      const int c = ctx_of(g, r);
      if constexpr (Var<V>::ot) {
        if (c == 0) {
          const float o = R[sw(P + brev(k, logQ))], e = R[sw(P + Q + k)];
          v0[s] = e + o; v1[s] = e - o;
          if (k == 0) v2[s] = R[sw(P + 2 * Q)];
        } else if (k > 0) {
          const float o = R[sw(P + brev(k - 1, logQ))], e = R[sw(P + Q + k - 1)];
          v0[s] = o + e; v1[s] = o - e;
        }
      } else {
        if (c == 0) {
          const float a = R[sw(P + k)], b = R[sw(P + M / 2 - k)];
          v0[s] = a + b; v1[s] = a - b;
          if (k == 0) v2[s] = R[sw(P + Q)];
        } else if (k > 0) {
          const float a = R[sw(P + k - 1)], b = R[sw(P + M / 2 - k - 1)];
          v0[s] = a - b; v1[s] = a + b;
        }
      }
    }
  }
  __syncthreads();
#pragma unroll
  for (int s = 0; s < NI; ++s) {
    const unsigned w = threadIdx.x + (unsigned)s * TPB;
    if (w < W) {
      const int r = (int)(w >> logQ), k = (int)(w & (Q - 1));
      RegP R = reg_ptr(sm + r * g.RS, g.RS);
      const int c = ctx_of(g, r);
      if constexpr (Var<V>::ot) {
        if (c == 0) {
          R[sw(P + k)] = v0[s]; R[sw(P + M / 2 - k)] = v1[s];
          if (k == 0) R[sw(P + Q)] = v2[s];
        } else if (k > 0) {
          R[sw(P + k - 1)] = v0[s]; R[sw(P + M / 2 - k - 1)] = v1[s];
        }
      } else {
        if (c == 0) {
          R[sw(P + Q + k)] = v0[s]; R[sw(P + brev(k, logQ))] = v1[s];
          if (k == 0) R[sw(P + 2 * Q)] = v2[s];
        } else if (k > 0) {
          R[sw(P + Q + k - 1)] = v0[s]; R[sw(P + brev(k - 1, logQ))] = v1[s];
        }
      }
    }
  }
}

}  // namespace amqft
