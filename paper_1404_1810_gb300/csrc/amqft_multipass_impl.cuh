// Multi-pass AM-QFT for 2^17 <= N <= 2^28: the same recursion and the same
// float32 operations as the fused kernel, with the four regions of each
// transform held in a global workspace (same chain layout and swizzle).
//
//   load     D_c, D_r (and the first D_k for the harmonics-first variants),
//            scattered into the regions;
//   levels   tree levels of node size > S in bands of up to four levels per
//            pass (the fused kernel's fold and chunk bands, in place in the
//            workspace), the M2/M4/M6/M8 neighbour phase of node sizes above
//            2S two levels per gather pass, the M1/M3/M5/M7 recurrences one
//            level per three passes (chunk totals, a scan of the totals per
//            node, the chunks re-run with their carries), and chain levels of
//            periodisation > 4S two per gather pass;
//   solve    one CTA per tree node of size 2S (node mode: its two children of
//            size S and its own M_v relation) and one per region tail (the
//            trees of size <= S plus the chain up to 4S, a region of N' = 4S)
//            in shared memory, with the fused kernel's bands, register
//            subtrees and passes;
//   store    last chain level (time-first variants), D_r^F and D_c^F.
//
// The recurrence variants (1, 3, 5, 7) take the scans without any wait
// between CTAs: a level is three launches, so every carry a chunk needs has
// been written by an earlier kernel of the stream.
#pragma once

#include "amqft_bands.cuh"
#include "amqft_fused_impl.cuh"

namespace amqft {

constexpr int MP_LOG_S = 13;           // subproblem node size S = 2^13
constexpr int MP_S = 1 << MP_LOG_S;
constexpr int MP_TPB = 512;            // solve CTA: 16384 values, 32 per thread

struct MpArgs {
  const void* in;      // complex64, or 16-bit complex pairs (dtype)
  void* out;
  const int* exp_in;   // 16-bit input: per-transform exponents (NULL: all 0)
  int* exp_out;        // 16-bit output: per-transform exponents
  int dtype;
  const float* ctab;   // the plan's constant table; NULL: constants evaluated on the fly
  long long nt;       // transforms in this chunk
  long long t0;       // first transform of the chunk (for in/out)
  int logN;
  int inverse;
  long long RSg;      // region stride in the workspace (floats)
  const int* tlist;   // transform ids of chunk positions (NULL: t0 + position)
  const long long* toff;  // element offset of each transform id (NULL: id * N)
  const int* ntdev;   // transforms in this chunk, read on the device (NULL: nt); nt is then the capacity
  // special input / output forms (all 0: complex): transform id t = signals 2t, 2t + 1
  long long nreal;    // real input (in: N floats a signal), half spectra out (N/2 + 1 complex64)
  long long ntrig;    // DCT-0 / DST-0: in / out the DCT-0 signals, in2 / out2 the DST-0 ones
  long long nirdft;   // half spectra in, real signals out (inverse)
  const float* in2;
  float* out2;
};

__device__ __forceinline__ long long mp_nt(const MpArgs& a) {
  if (!a.ntdev) return a.nt;
  const long long n = (long long)*a.ntdev;  // written by an earlier kernel of the stream
  return n < a.nt ? n : a.nt;
}

// transform id of chunk position t, and the element offset of an id
__device__ __forceinline__ long long mp_id(const MpArgs& a, long long t) {
  return a.tlist ? (long long)__ldg(a.tlist + t) : a.t0 + t;
}
__device__ __forceinline__ long long mp_off(const MpArgs& a, long long id) {
  return a.toff ? __ldg(a.toff + id) : (id << a.logN);
}

struct GRegions {
  float* W;
  long long RSg;
  __device__ __forceinline__ RegP get(long long t, int kind) const {
    return reg_ptr(W + (t * 4 + kind) * RSg, (int)RSg);
  }
};

template <int V>
__global__ void mp_load_kernel(MpArgs a, float* W) {
  const int logQ = a.logN - 2;
  const long long total = mp_nt(a) << logQ;
  const float cj = a.inverse ? -1.f : 1.f;
  GRegions rg{W, a.RSg};
  for (long long w = (long long)blockIdx.x * blockDim.x + threadIdx.x; w < total; w += (long long)gridDim.x * blockDim.x) {
    const long long t = w >> logQ;
    const int n = (int)(w & ((1LL << logQ) - 1));
    const long long id = mp_id(a, t);
    if (a.ntrig > 0) {
      load_place<V>(rg, a.logN, (int)t, n,
                    load_fetch_trig(static_cast<const float*>(a.in), a.in2, a.ntrig, a.logN, id, n));
    } else {
      const Fetched f =
          a.nreal > 0 ? load_fetch_real(static_cast<const float*>(a.in), a.logN, id, a.nreal, n)
          : a.nirdft > 0 ? load_fetch_irdft(static_cast<const float2*>(a.in), a.logN, id, a.nirdft, n)
                         : load_fetch(InRef{a.in, a.exp_in, a.dtype}, a.logN, id, mp_off(a, id), n, cj);
      load_scatter<V>(rg, a.logN, (int)t, n, f);
    }
  }
}

template <int V>
__global__ void mp_store_kernel(MpArgs a, const float* W) {
  const int logQ = a.logN - 2;
  const long long total = mp_nt(a) << logQ;
  const float cj = a.inverse ? -1.f : 1.f;
  GRegions rg{const_cast<float*>(W), a.RSg};
  for (long long w = (long long)blockIdx.x * blockDim.x + threadIdx.x; w < total; w += (long long)gridDim.x * blockDim.x) {
    const long long t = w >> logQ;
    const int k = (int)(w & ((1LL << logQ) - 1));
    const Gathered g = store_gather<V>(rg, a.logN, (int)t, k);
    const long long id = mp_id(a, t);
    if (a.ntrig > 0) store_trig<V>(static_cast<float*>(a.out), a.out2, a.ntrig, a.logN, id, k, g);
    else if (a.nirdft > 0) store_irdft<V>(static_cast<float*>(a.out), a.nirdft, a.logN, id, k, g, cj);
    else if (a.nreal > 0) store_real<V>(static_cast<float2*>(a.out), a.logN, id, a.nreal, k, g);
    else store_emit<V>(static_cast<float2*>(a.out), a.logN, mp_off(a, id), k, g, cj);
  }
}

// 16-bit output, pass 1: the largest component magnitude of each transform
// of the chunk, as float bits in Mx[t] (zeroed by mp_zero_kernel)
template <int V>
__global__ void mp_max_kernel(MpArgs a, const float* W, int* Mx) {
  const int logQ = a.logN - 2;
  const long long total = mp_nt(a) << logQ;
  GRegions rg{const_cast<float*>(W), a.RSg};
  for (long long w = (long long)blockIdx.x * blockDim.x + threadIdx.x; w < total; w += (long long)gridDim.x * blockDim.x) {
    const long long t = w >> logQ;
    const int k = (int)(w & ((1LL << logQ) - 1));
    const Out4 o = emit_values<V>(a.logN, k, store_gather<V>(rg, a.logN, (int)t, k));
    const float m = out4_absmax(o);
    // a warp's 32 consecutive items belong to one transform (N/4 and the total
    // are multiples of 32, so the loop is warp-uniform): one atomic per warp.
    // Positive floats order as their bit patterns; zeros and NaN count as 0.
    const unsigned mw = __reduce_max_sync(0xffffffffu, m > 0.f ? __float_as_uint(m) : 0u);
    if ((threadIdx.x & 31) == 0 && mw != 0u) atomicMax(Mx + t, (int)mw);
  }
}

template <int V>
__global__ void mp_zero_kernel(int* Mx, long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) Mx[i] = 0;
}

// 16-bit output, pass 2: exponent per transform, outputs scaled by 2^-exp
template <int V>
__global__ void mp_store16_kernel(MpArgs a, const float* W, const int* Mx) {
  const int logQ = a.logN - 2;
  const long long total = mp_nt(a) << logQ;
  const float cj = a.inverse ? -1.f : 1.f;
  GRegions rg{const_cast<float*>(W), a.RSg};
  for (long long w = (long long)blockIdx.x * blockDim.x + threadIdx.x; w < total; w += (long long)gridDim.x * blockDim.x) {
    const long long t = w >> logQ;
    const int k = (int)(w & ((1LL << logQ) - 1));
    const Out4 o = emit_values<V>(a.logN, k, store_gather<V>(rg, a.logN, (int)t, k));
    const int e = block_exponent(__int_as_float(Mx[t]));
    const long long id = mp_id(a, t);
    store16(static_cast<unsigned*>(a.out), mp_off(a, id), o, pow2f(-e), cj, a.dtype);
    if (k == 0) a.exp_out[id] = e;
  }
}

// Region geometry of the workspace for the band kernels (every region of
// the chunk, in global memory).
__device__ __forceinline__ Geo mp_geo(const MpArgs& a) {
  Geo g;
  g.logN = a.logN;
  g.half = 1 << (a.logN - 1);
  g.RS = (int)a.RSg;
  g.nreg = (int)(4 * mp_nt(a));
  g.nreg_cap = g.nreg;
  g.gbase = 0;
  g.sub = 0;
  return g;
}

// Up to four tree levels above the subproblem size in one pass over the
// workspace: the fused kernel's fold band (D_k + M_v time phase of the ot
// trees, or D_n + M_v frequency phase of the to trees), in place.
template <int V, bool FWD, int R>
__global__ void __launch_bounds__(256) mp_fold_band_kernel(MpArgs a, float* W, int logL) {
  const Geo g = mp_geo(a);
  if (a.ctab) run_fold_band<V, FWD, R, 256, true>(W, g, logL, TabConsts{a.ctab + 30});
  else run_fold_band<V, FWD, R, 256, true>(W, g, logL, FlyConsts<V>{});
}

// Neighbour form of M_v on the B halves at node size 2^logLp (M4/M8
// frequency phase, M2/M6 time phase), gather form Win -> Wout; every other
// word is copied.
template <int V>
__global__ void mp_neighbour_kernel(MpArgs a, const float* __restrict__ Win, float* __restrict__ Wout, int logLp) {
  const int half = 1 << (a.logN - 1), Lp = 1 << logLp, H = Lp >> 1, h = logLp - 1;
  const long long total = a.RSg * 4 * mp_nt(a);
  const Div dvr((unsigned)a.RSg);  // total < 2^32 (checked by the host)
  for (long long w = (long long)blockIdx.x * blockDim.x + threadIdx.x; w < total; w += (long long)gridDim.x * blockDim.x) {
    const unsigned rq = dvr((unsigned)w);
    const long long rr = rq;
    const int ph = (int)((unsigned)w - rq * (unsigned)a.RSg);  // physical (swizzled) word
    const int p = sw(ph);                  // logical position (sw is an involution)
    CRegP R = creg_ptr(Win + rr * a.RSg, (int)a.RSg);
    float v = R[ph];
    if (p < half - Lp) {
      const int p0 = p & ~(Lp - 1), qn = p - p0;
      const int ctx = node_ctx<V>(p0, logLp, half, (int)(rr & 1));
      const int base = ctx == 0 ? p0 + H : p0;
      if (p >= base && p < base + H) {
        const int q = p - base, i = brev(q, h);
        int dir;
        bool add;
        if constexpr (V == 4) { dir = ctx == 0 ? +1 : -1; add = true; }
        else if constexpr (V == 8) { dir = ctx == 0 ? -1 : +1; add = false; }
        else if constexpr (V == 2) { dir = ctx == 0 ? -1 : +1; add = true; }
        else { dir = ctx == 0 ? +1 : -1; add = false; }
        const int jn = i + dir;
        if (jn >= 0 && jn < H) {
          const float bn = R[sw(base + brev(jn, h))];
          v = add ? ((dir > 0) ? (v + bn) : (bn + v)) : (v - bn);
        }
        (void)qn;
      }
    }
    Wout[rr * a.RSg + ph] = v;
  }
}

// Which neighbour (+1 / -1 in bit-reversed order) enters, and whether it is
// added or subtracted: M4 / M8 frequency phase, M2 / M6 time phase.
template <int V>
__device__ __forceinline__ void nb_rule(int ctx, int& dir, bool& add) {
  if constexpr (V == 4) { dir = ctx == 0 ? +1 : -1; add = true; }
  else if constexpr (V == 8) { dir = ctx == 0 ? -1 : +1; add = false; }
  else if constexpr (V == 2) { dir = ctx == 0 ? -1 : +1; add = true; }
  else { dir = ctx == 0 ? +1 : -1; add = false; }  // V == 6
}

// The neighbour form's output at position p for node size 2^logLp, from its
// input R (the value itself where p is not in a class-0 B half).
template <int V>
__device__ __forceinline__ float nb_at(CRegP R, int p, int logLp, int half, int ctx0) {
  const float v = R[sw(p)];
  const int Lp = 1 << logLp, H = Lp >> 1, h = logLp - 1;
  if (p >= half - Lp) return v;
  const int p0 = p & ~(Lp - 1);
  const int ctx = node_ctx<V>(p0, logLp, half, ctx0);
  const int base = ctx == 0 ? p0 + H : p0;
  if (p < base || p >= base + H) return v;
  const int i = brev(p - base, h);
  int dir;
  bool add;
  nb_rule<V>(ctx, dir, add);
  const int jn = i + dir;
  if (jn < 0 || jn >= H) return v;
  const float bn = R[sw(base + brev(jn, h))];
  return add ? ((dir > 0) ? (v + bn) : (bn + v)) : (v - bn);
}

// Two levels of the neighbour relation in one gather pass: node size 2^l1
// first, then 2^l2 (the time-first variants 4 / 8 climb, l2 = l1 + 1, in the
// frequency phase; the harmonics-first 2 / 6 descend, l2 = l1 - 1, in the
// time phase).  Each output of the second level takes the first level's
// outputs at its position and at its neighbour's, evaluated from Win on the
// fly: the same float32 operations as two single-level passes.
template <int V>
__global__ void mp_neighbour2_kernel(MpArgs a, const float* __restrict__ Win, float* __restrict__ Wout, int l1,
                                     int l2) {
  static_assert(!Var<V>::scan, "the neighbour form");
  const int half = 1 << (a.logN - 1), L2 = 1 << l2, H2 = L2 >> 1, h2 = l2 - 1;
  const long long total = a.RSg * 4 * mp_nt(a);
  const Div dvr((unsigned)a.RSg);  // total < 2^32 (checked by the host)
  for (long long w = (long long)blockIdx.x * blockDim.x + threadIdx.x; w < total; w += (long long)gridDim.x * blockDim.x) {
    const unsigned rq = dvr((unsigned)w);
    const long long rr = rq;
    const int ph = (int)((unsigned)w - rq * (unsigned)a.RSg);
    const int p = sw(ph);
    CRegP R = creg_ptr(Win + rr * a.RSg, (int)a.RSg);
    const int ctx0 = (int)(rr & 1);
    float v = nb_at<V>(R, p, l1, half, ctx0);
    if (p < half - L2) {
      const int p0 = p & ~(L2 - 1);
      const int ctx = node_ctx<V>(p0, l2, half, ctx0);
      const int base = ctx == 0 ? p0 + H2 : p0;
      if (p >= base && p < base + H2) {
        const int i = brev(p - base, h2);
        int dir;
        bool add;
        nb_rule<V>(ctx, dir, add);
        const int jn = i + dir;
        if (jn >= 0 && jn < H2) {
          const float bn = nb_at<V>(R, base + brev(jn, h2), l1, half, ctx0);
          v = add ? ((dir > 0) ? (v + bn) : (bn + v)) : (v - bn);
        }
      }
    }
    Wout[rr * a.RSg + ph] = v;
  }
}

// Recurrence form of M_v on the B halves at node size 2^logLp > S: the
// frequency phase of M1/M5 (ot variants, the first value halved) or the time
// phase of M3/M7 (to variants, the last value halved), Tab. 5-6.  A node's B
// half holds H = 2^(logLp-1) values in bit-reversed order; it is cut into SC
// chunks of MP_RC values consecutive in recurrence order.  Viewed as MP_RC
// rows of SC words, a chunk is one column: value e of the chunk in column col
// lies at base + brev(e) * SC + col (prefix recurrence, k = brev(col)) or at
// base + brev(MP_RC - 1 - e) * SC + col (suffix recurrence, k = SC - 1 -
// brev(col)), so the 32 columns of a warp are 32 consecutive words.
// Each recurrence y(m) = x(m) + y(m-1) (M5/M7) or x(m) - y(m-1) (M1/M3) is
// run per chunk from a zero carry; with an even chunk length the carry into
// chunk k is the plain sum of the earlier chunks' last values, added
// (alternating sign for M1/M3) when the chunk is run again.
constexpr int MP_RLOG_C = 5;
constexpr int MP_RC = 1 << MP_RLOG_C;  // values per chunk (even)

template <int V>
__device__ __forceinline__ bool rec_prefix(int ctx) {
  if constexpr (V == 1) return ctx == 0;
  else if constexpr (V == 5) return ctx == 1;
  else if constexpr (V == 3) return ctx == 1;
  else return ctx == 0;  // V == 7
}

struct RecChunk {
  RegP R;       // the region
  long long nd;  // node index over the chunk's regions
  int base;      // first position of the node's B half
  int col, k, logSC;
  bool prefix;
  __device__ __forceinline__ int pos(int e) const {
    return base + (brev(prefix ? e : MP_RC - 1 - e, MP_RLOG_C) << logSC) + col;
  }
};

// class-0 nodes of size 2^logLp per region, and the chunks of a node
__device__ __forceinline__ long long rec_nodes(const MpArgs& a, int logLp) {
  return (1LL << (a.logN - 1 - logLp)) - 1;
}

template <int V>
__device__ __forceinline__ RecChunk rec_chunk(const MpArgs& a, float* W, int logLp, long long w) {
  const int half = 1 << (a.logN - 1), H = 1 << (logLp - 1);
  RecChunk c;
  c.logSC = logLp - 1 - MP_RLOG_C;
  const int SC = 1 << c.logSC;
  const long long nb = rec_nodes(a, logLp);
  c.nd = w >> c.logSC;
  c.col = (int)(w & (SC - 1));
  const long long rr = c.nd / nb;
  const int p0 = (int)(c.nd - rr * nb) << logLp;
  const int ctx = node_ctx<V>(p0, logLp, half, (int)(rr & 1));
  c.R = reg_ptr(W + rr * a.RSg, (int)a.RSg);
  c.base = ctx == 0 ? p0 + H : p0;
  c.prefix = rec_prefix<V>(ctx);
  const int bc = brev(c.col, c.logSC);
  c.k = c.prefix ? bc : SC - 1 - bc;
  return c;
}

// pass 1: every chunk from a zero carry; T[node * SC + k] = its last value
template <int V>
__global__ void mp_rec_total_kernel(MpArgs a, float* W, float* __restrict__ T, int logLp) {
  constexpr bool hstart = Var<V>::ot;
  constexpr bool alt = (V == 1 || V == 3);
  const long long total = (4 * mp_nt(a) * rec_nodes(a, logLp)) << (logLp - 1 - MP_RLOG_C);
  for (long long w = (long long)blockIdx.x * blockDim.x + threadIdx.x; w < total; w += (long long)gridDim.x * blockDim.x) {
    const RecChunk c = rec_chunk<V>(a, W, logLp, w);
    float x[MP_RC];
#pragma unroll
    for (int e = 0; e < MP_RC; ++e) x[e] = c.R[sw(c.pos(e))];
    float prev = 0.f;
#pragma unroll
    for (int e = 0; e < MP_RC; ++e) {
      float y;
      if (hstart && c.k == 0 && e == 0) y = 0.5f * x[e];
      else y = alt ? (x[e] - prev) : (x[e] + prev);
      prev = y;
    }
    T[(c.nd << c.logSC) + c.k] = prev;
  }
}

// pass 2: exclusive prefix sum of each node's SC chunk totals (SC >= 256),
// one 256-thread CTA per node
template <int V>
__global__ void __launch_bounds__(256) mp_rec_scan_kernel(MpArgs a, float* T, int logLp) {
  __shared__ float wsum[8];
  const int logSC = logLp - 1 - MP_RLOG_C, per = (1 << logSC) >> 8;
  const long long nodes = 4 * mp_nt(a) * rec_nodes(a, logLp);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (long long nd = blockIdx.x; nd < nodes; nd += gridDim.x) {
    float* t = T + (nd << logSC) + (long long)threadIdx.x * per;
    float s = 0.f;
    for (int j = 0; j < per; ++j) s = s + t[j];
    float incl = s;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const float o = __shfl_up_sync(0xffffffffu, incl, d);
      if (lane >= d) incl = incl + o;
    }
    float run = __shfl_up_sync(0xffffffffu, incl, 1);
    if (lane == 0) run = 0.f;
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    float wp = 0.f;
    for (int j = 0; j < warp; ++j) wp = wp + wsum[j];
    run = wp + run;
    for (int j = 0; j < per; ++j) {
      const float v = t[j];
      t[j] = run;
      run = run + v;
    }
    __syncthreads();  // wsum is rewritten by the next node
  }
}

// pass 3: every chunk again, with its carry c: y = l + c (M5/M7), l -/+ c for
// even/odd e (M1/M3); the to variants halve the last value of the node
template <int V>
__global__ void mp_rec_apply_kernel(MpArgs a, float* W, const float* __restrict__ T, int logLp) {
  constexpr bool hstart = Var<V>::ot;
  constexpr bool alt = (V == 1 || V == 3);
  const long long total = (4 * mp_nt(a) * rec_nodes(a, logLp)) << (logLp - 1 - MP_RLOG_C);
  for (long long w = (long long)blockIdx.x * blockDim.x + threadIdx.x; w < total; w += (long long)gridDim.x * blockDim.x) {
    const RecChunk c = rec_chunk<V>(a, W, logLp, w);
    const int SC = 1 << c.logSC;
    const float cy = T[(c.nd << c.logSC) + c.k];
    float x[MP_RC];
#pragma unroll
    for (int e = 0; e < MP_RC; ++e) x[e] = c.R[sw(c.pos(e))];
    float prev = 0.f;
#pragma unroll
    for (int e = 0; e < MP_RC; ++e) {
      float l;
      if (hstart && c.k == 0 && e == 0) l = 0.5f * x[e];
      else l = alt ? (x[e] - prev) : (x[e] + prev);
      prev = l;
      float y;
      if (alt) y = (e & 1) ? (l + cy) : (l - cy);
      else y = l + cy;
      if (!hstart && c.k == SC - 1 && e == MP_RC - 1) y = 0.5f * y;
      c.R[sw(c.pos(e))] = y;
    }
  }
}

// One chain level of periodisation M = 2^logM, gather form: ot variants the
// D_n frequency phase, to variants the D_k time phase (Sect. 6.9).
template <int V>
__global__ void mp_chain_kernel(MpArgs a, const float* __restrict__ Win, float* __restrict__ Wout, int logM) {
  const int half = 1 << (a.logN - 1), M = 1 << logM, logQ = logM - 2, Q = 1 << logQ, P = half - M / 2;
  const long long total = a.RSg * 4 * mp_nt(a);
  const Div dvr((unsigned)a.RSg);  // total < 2^32 (checked by the host)
  for (long long w = (long long)blockIdx.x * blockDim.x + threadIdx.x; w < total; w += (long long)gridDim.x * blockDim.x) {
    const unsigned rq = dvr((unsigned)w);
    const long long rr = rq;
    const int ph = (int)((unsigned)w - rq * (unsigned)a.RSg);
    const int p = sw(ph);
    CRegP R = creg_ptr(Win + rr * a.RSg, (int)a.RSg);
    const int ctx0 = (int)(rr & 1);
    float v = R[ph];
    const int rel = p - P;
    if constexpr (Var<V>::ot) {
      if (ctx0 == 0 && rel >= 0 && rel <= M / 2) {
        if (rel == Q) {
          v = R[sw(P + 2 * Q)];
        } else {
          const int k = rel < Q ? rel : M / 2 - rel;
          const float e = R[sw(P + Q + k)], o = R[sw(P + brev(k, logQ))];
          v = rel < Q ? (e + o) : (e - o);
        }
      } else if (ctx0 == 1 && rel >= 0 && rel < M / 2 - 1) {
        const int k = rel + 1;
        if (k == Q) {
          v = R[sw(P + Q - 1)];
        } else {
          const int kk = k < Q ? k : M / 2 - k;
          const float o = R[sw(P + brev(kk - 1, logQ))], e = R[sw(P + Q + kk - 1)];
          v = k < Q ? (o + e) : (o - e);
        }
      }
    } else {
      if (ctx0 == 0 && rel >= 0 && rel <= M / 2) {
        if (rel < Q) {
          const int n = brev(rel, logQ);
          v = R[sw(P + n)] - R[sw(P + M / 2 - n)];
        } else {
          const int n = rel - Q;
          v = n < Q ? (R[sw(P + n)] + R[sw(P + M / 2 - n)]) : R[sw(P + Q)];
        }
      } else if (ctx0 == 1 && rel >= 0 && rel < M / 2 - 1) {
        if (rel < Q) {
          const int n = brev(rel, logQ) + 1;
          v = n < Q ? (R[sw(P + n - 1)] + R[sw(P + M / 2 - n - 1)]) : R[sw(P + Q - 1)];
        } else {
          const int n = rel - Q + 1;
          v = R[sw(P + n - 1)] - R[sw(P + M / 2 - n - 1)];
        }
      }
    }
    Wout[rr * a.RSg + ph] = v;
  }
}

// Two chain levels of the time-first variants in one gather pass: the D_n
// frequency phase of periodisation M = 2^logM and then of 2M.  Level 2M
// writes the whole range level M writes (its E input is level M's output),
// so each of its outputs takes its E value from level M's formula applied to
// Win on the fly (two more reads, from cache) and its O value (the 2M tree)
// from Win; every other word is copied.  Same float32 operations per output
// as the two single-level passes.
template <int V>
__device__ __forceinline__ float chain_ot_value(CRegP R, int ctx0, int P, int Q, int logQ, int M, int rel) {
  // level M's output at P + rel, from its inputs in R (rel inside its range)
  if (ctx0 == 0) {
    if (rel == Q) return R[sw(P + 2 * Q)];
    const int k = rel < Q ? rel : M / 2 - rel;
    const float e = R[sw(P + Q + k)], o = R[sw(P + brev(k, logQ))];
    return rel < Q ? (e + o) : (e - o);
  }
  const int k = rel + 1;
  if (k == Q) return R[sw(P + Q - 1)];
  const int kk = k < Q ? k : M / 2 - k;
  const float o = R[sw(P + brev(kk - 1, logQ))], e = R[sw(P + Q + kk - 1)];
  return k < Q ? (o + e) : (o - e);
}

template <int V>
__global__ void mp_chain2_kernel(MpArgs a, const float* __restrict__ Win, float* __restrict__ Wout, int logM) {
  static_assert(Var<V>::ot, "the time-first chain");
  const int half = 1 << (a.logN - 1);
  const int M = 1 << logM, logQ = logM - 2, Q = 1 << logQ, P = half - M / 2;          // level M
  const int M2 = 2 * M, logQ2 = logQ + 1, Q2 = 2 * Q, P2 = half - M;                  // level 2M
  const long long total = a.RSg * 4 * mp_nt(a);
  const Div dvr((unsigned)a.RSg);  // total < 2^32 (checked by the host)
  for (long long w = (long long)blockIdx.x * blockDim.x + threadIdx.x; w < total; w += (long long)gridDim.x * blockDim.x) {
    const unsigned rq = dvr((unsigned)w);
    const long long rr = rq;
    const int ph = (int)((unsigned)w - rq * (unsigned)a.RSg);
    const int p = sw(ph);
    CRegP R = creg_ptr(Win + rr * a.RSg, (int)a.RSg);
    const int ctx0 = (int)(rr & 1);
    float v = R[ph];
    const int rel2 = p - P2;
    if (ctx0 == 0 && rel2 >= 0 && rel2 <= M2 / 2) {
      if (rel2 == Q2) {
        v = chain_ot_value<V>(R, 0, P, Q, logQ, M, 2 * Q);  // E2(Q2): level M at its harmonic M/2
      } else {
        const int k2 = rel2 < Q2 ? rel2 : M2 / 2 - rel2;
        const float e = chain_ot_value<V>(R, 0, P, Q, logQ, M, k2), o = R[sw(P2 + brev(k2, logQ2))];
        v = rel2 < Q2 ? (e + o) : (e - o);
      }
    } else if (ctx0 == 1 && rel2 >= 0 && rel2 < M2 / 2 - 1) {
      const int k2 = rel2 + 1;
      if (k2 == Q2) {
        v = R[sw(P2 + Q2 - 1)];
      } else {
        const int kk = k2 < Q2 ? k2 : M2 / 2 - k2;
        const float o = R[sw(P2 + brev(kk - 1, logQ2))], e = chain_ot_value<V>(R, 1, P, Q, logQ, M, kk - 1);
        v = k2 < Q2 ? (o + e) : (o - e);
      }
    }
    Wout[rr * a.RSg + ph] = v;
  }
}

// The harmonics-first chain (the D_k time phase, descending): level M's
// output at P + rel from its input R (rel inside its range), and two levels
// (M, then M/2) in one gather pass.  Level M/2 rewrites exactly level M's te
// part, so each of its outputs evaluates the two level-M values it needs
// from Win on the fly; level M's to part is written from its own formula.
__device__ __forceinline__ float chain_to_value(CRegP R, int ctx0, int P, int Q, int logQ, int M, int rel) {
  if (ctx0 == 0) {
    if (rel < Q) {
      const int n = brev(rel, logQ);
      return R[sw(P + n)] - R[sw(P + M / 2 - n)];
    }
    const int n = rel - Q;
    return n < Q ? (R[sw(P + n)] + R[sw(P + M / 2 - n)]) : R[sw(P + Q)];
  }
  if (rel < Q) {
    const int n = brev(rel, logQ) + 1;
    return n < Q ? (R[sw(P + n - 1)] + R[sw(P + M / 2 - n - 1)]) : R[sw(P + Q - 1)];
  }
  const int n = rel - Q + 1;
  return R[sw(P + n - 1)] - R[sw(P + M / 2 - n - 1)];
}

template <int V>
__global__ void mp_chain2_to_kernel(MpArgs a, const float* __restrict__ Win, float* __restrict__ Wout, int logM) {
  static_assert(!Var<V>::ot, "the harmonics-first chain");
  const int half = 1 << (a.logN - 1);
  const int M = 1 << logM, logQ = logM - 2, Q = 1 << logQ, P = half - M / 2;  // level M
  const int M1 = M / 2, logQ1 = logQ - 1, Q1 = Q / 2, P1 = P + Q;            // level M/2
  const long long total = a.RSg * 4 * mp_nt(a);
  const Div dvr((unsigned)a.RSg);  // total < 2^32 (checked by the host)
  for (long long w = (long long)blockIdx.x * blockDim.x + threadIdx.x; w < total; w += (long long)gridDim.x * blockDim.x) {
    const unsigned rq = dvr((unsigned)w);
    const long long rr = rq;
    const int ph = (int)((unsigned)w - rq * (unsigned)a.RSg);
    const int p = sw(ph);
    CRegP R = creg_ptr(Win + rr * a.RSg, (int)a.RSg);
    const int ctx0 = (int)(rr & 1);
    float v = R[ph];
    const int rel = p - P;
    const bool inM = ctx0 == 0 ? (rel >= 0 && rel <= M / 2) : (rel >= 0 && rel < M / 2 - 1);
    if (inM) {
      if (rel < Q) {
        v = chain_to_value(R, ctx0, P, Q, logQ, M, rel);  // level M's to part
      } else {
        // level M/2 at P1 + r1, its input x at P1 + j being level M's output at rel Q + j
        auto in1 = [&](int j) { return chain_to_value(R, ctx0, P, Q, logQ, M, Q + j); };
        const int r1 = rel - Q;
        if (ctx0 == 0) {
          if (r1 < Q1) {
            const int n = brev(r1, logQ1);
            v = in1(n) - in1(M1 / 2 - n);
          } else {
            const int n = r1 - Q1;
            v = n < Q1 ? (in1(n) + in1(M1 / 2 - n)) : in1(Q1);
          }
        } else {
          if (r1 < Q1) {
            const int n = brev(r1, logQ1) + 1;
            v = n < Q1 ? (in1(n - 1) + in1(M1 / 2 - n - 1)) : in1(Q1 - 1);
          } else {
            const int n = r1 - Q1 + 1;
            v = in1(n - 1) - in1(M1 / 2 - n - 1);
          }
        }
        (void)P1;
      }
    }
    Wout[rr * a.RSg + ph] = v;
  }
}

// Subproblem solve.  Blocks [0, nnode/2) of each region take one tree node of
// size 2S each (node mode), the last block the region tail (region mode,
// N' = 4S).  The words are copied verbatim: S and half - 2S are multiples of
// 1024, so the swizzle of the workspace and of shared memory coincide.
template <int V, int TPB>
__global__ void __launch_bounds__(TPB) mp_solve_kernel(MpArgs a, float* W, const __grid_constant__ SmallConsts K) {
  extern __shared__ __align__(16) float sm[];
  const int half = 1 << (a.logN - 1);
  const int nnode = (half >> MP_LOG_S) - 2;  // nodes of size S in [0, half - 2S)
  const int per = nnode / 2 + 1;
  const long long rr = blockIdx.x / per;
  if (rr >= 4 * mp_nt(a)) return;  // launched for the capacity (uniform per block, before any barrier)
  const int sidx = (int)(blockIdx.x - rr * per);
  RegP R = reg_ptr(W + rr * a.RSg, (int)a.RSg);
  const int ctx0 = (int)(rr & 1);
  const int RSn = MP_S + 32;
  float* tot = sm + 2 * RSn + 64;  // scratch after the largest layout (tail: 2S + 32 words)
  float* wsum = tot + TPB;
  float* snap = wsum + 32;
  // constants of the node levels up to S (periodisations up to 4S), staged
  // from the table or evaluated on the fly; visible after the barrier that
  // ends the copy-in below
  float* cst = snap + snap_floats(2 * MP_S);
  stage_consts<V>(cst, band_consts(MP_LOG_S + 2), a.ctab, (int)threadIdx.x, TPB);
  const TabConsts cs{cst};
  Geo g;
  if (sidx < nnode / 2) {
    // node mode: the tree node of size 2S at 2S * sidx (children 2*sidx and
    // 2*sidx + 1 of size S), its levels up to and including its own M_v
    // relation (the frequency phase last for the time-first variants, the
    // time phase first for the harmonics-first ones)
    const int L2 = 2 * MP_S, P = sidx * L2;
    for (int e = threadIdx.x; e < L2; e += TPB) sm[e] = R[P + e];
    g.logN = MP_LOG_S + 3;
    g.half = L2;
    g.RS = L2;
    g.nreg = 1;
    g.nreg_cap = 1;
    g.gbase = node_ctx<V>(P, MP_LOG_S + 1, half, ctx0);
    g.sub = L2;
    __syncthreads();
    const BandPlan bp = band_plan(MP_LOG_S + 2);  // levels S .. 2*LEAF
    const int nleaf = L2 >> LOG_LEAF;
    if constexpr (Var<V>::ot) {
      for (int b = 0; b < bp.nb; ++b) {
        run_fold_band_r<V, TPB>(sm, g, bp.logL[b], bp.R[b], true, cs);
        __syncthreads();
      }
      for (int w = threadIdx.x; w < nleaf; w += TPB) {
        const int p0 = w << LOG_LEAF;
        run_leaf<V>(reg_ptr(sm, L2), p0, node_ctx_g<V>(g, p0, LOG_LEAF, ctx_of(g, 0)), K);
      }
      __syncthreads();
      if constexpr (Var<V>::scan) {
        for (int lp = LOG_LEAF + 1; lp <= MP_LOG_S + 1; ++lp) {
          pass_recurrence<V, TPB, 16>(sm, tot, wsum, g, lp);
          __syncthreads();
        }
      } else {
        for (int b = bp.nb - 1; b >= 0; --b) {
          run_chunk_band_r<V, TPB>(sm, snap, g, bp.logL[b], bp.R[b]);
          __syncthreads();
        }
        pass_neighbour<V, TPB, 16>(sm, g, MP_LOG_S + 1);
        __syncthreads();
      }
    } else {
      for (int lp = MP_LOG_S + 1; lp >= LOG_LEAF + 1; --lp) {
        if constexpr (Var<V>::scan) pass_recurrence<V, TPB, 16>(sm, tot, wsum, g, lp);
        else pass_neighbour<V, TPB, 16>(sm, g, lp);
        __syncthreads();
      }
      for (int w = threadIdx.x; w < nleaf; w += TPB) {
        const int p0 = w << LOG_LEAF;
        run_leaf<V>(reg_ptr(sm, L2), p0, node_ctx_g<V>(g, p0, LOG_LEAF, ctx_of(g, 0)), K);
      }
      __syncthreads();
      for (int b = bp.nb - 1; b >= 0; --b) {
        run_fold_band_r<V, TPB>(sm, g, bp.logL[b], bp.R[b], false, cs);
        __syncthreads();
      }
    }
    for (int e = threadIdx.x; e < L2; e += TPB) R[P + e] = sm[e];
  } else {
    // tail: region of N' = 4S at [half - 2S, RSg)
    const int base = half - 2 * MP_S;
    const int words = (int)a.RSg - base;
    for (int e = threadIdx.x; e < words; e += TPB) sm[e] = R[base + e];
    const int logNp = MP_LOG_S + 2, halfp = 2 * MP_S;
    g.logN = logNp;
    g.half = halfp;
    g.RS = words;
    g.nreg = 1;
    g.nreg_cap = 1;
    g.gbase = ctx0;
    g.sub = 0;
    __syncthreads();
    const BandPlan bp = band_plan(logNp);
    const int nleaf = (halfp >> LOG_LEAF) - 1;
    if constexpr (Var<V>::ot) {
      for (int b = 0; b < bp.nb; ++b) {
        run_fold_band_r<V, TPB>(sm, g, bp.logL[b], bp.R[b], true, cs);
        __syncthreads();
      }
      for (int w = threadIdx.x; w < nleaf + 1; w += TPB) {
        if (w < nleaf) run_leaf<V>(reg_ptr(sm, g.RS), w << LOG_LEAF, node_ctx_g<V>(g, w << LOG_LEAF, LOG_LEAF, ctx0), K);
        else run_tail<V>(reg_ptr(sm, g.RS), ctx0, logNp, K);
      }
      __syncthreads();
      if constexpr (Var<V>::scan) {
        for (int lp = LOG_LEAF + 1; lp <= logNp - 2; ++lp) {
          pass_recurrence<V, TPB, 16>(sm, tot, wsum, g, lp);
          __syncthreads();
        }
      } else {
        for (int b = bp.nb - 1; b >= 0; --b) {
          run_chunk_band_r<V, TPB>(sm, snap, g, bp.logL[b], bp.R[b]);
          __syncthreads();
        }
      }
      for (int lm = LOG_LEAF + 2; lm <= logNp; ++lm) {
        pass_chain<V, TPB, 32>(sm, g, lm);
        __syncthreads();
      }
    } else {
      for (int lm = logNp; lm >= LOG_LEAF + 2; --lm) {
        pass_chain<V, TPB, 32>(sm, g, lm);
        __syncthreads();
      }
      if (threadIdx.x == 0) run_tail<V>(reg_ptr(sm, g.RS), ctx0, logNp, K);
      __syncthreads();
      for (int lp = logNp - 2; lp >= LOG_LEAF + 1; --lp) {
        if constexpr (Var<V>::scan) pass_recurrence<V, TPB, 16>(sm, tot, wsum, g, lp);
        else pass_neighbour<V, TPB, 16>(sm, g, lp);
        __syncthreads();
      }
      for (int w = threadIdx.x; w < nleaf; w += TPB)
        run_leaf<V>(reg_ptr(sm, g.RS), w << LOG_LEAF, node_ctx_g<V>(g, w << LOG_LEAF, LOG_LEAF, ctx0), K);
      __syncthreads();
      for (int b = bp.nb - 1; b >= 0; --b) {
        run_fold_band_r<V, TPB>(sm, g, bp.logL[b], bp.R[b], false, cs);
        __syncthreads();
      }
    }
    for (int e = threadIdx.x; e < words; e += TPB) R[base + e] = sm[e];
  }
}

inline int mp_solve_smem_bytes() {
  // tail layout (2S + 32 words) is the larger one; then scan scratch,
  // snapshot and the node levels' constants
  return (2 * (MP_S + 32) + 64 + MP_TPB + 32 + snap_floats(2 * MP_S) + band_consts(MP_LOG_S + 2)) *
         (int)sizeof(float);
}

// Host side: the whole sequence for one chunk of transforms.
// `nlaunch` (may be NULL) is incremented once per kernel launched.
template <int V>
cudaError_t mp_run(const MpArgs& a0, float* W0, float* W1, const SmallConsts& K, cudaStream_t st,
                   long long* nlaunch) {
  MpArgs a = a0;
  auto launched = [&]() {
    if (nlaunch) ++*nlaunch;
    return cudaGetLastError();
  };
  const int logN = a.logN, N = 1 << logN;
  const int threads = 256;
  auto grid_for = [&](long long items) {
    long long b = (items + threads - 1) / threads;
    return (unsigned)(b < 152LL * 32 ? (b > 0 ? b : 1) : 152LL * 32);
  };
  cudaError_t e;
  float* cur = W0;
  float* oth = W1;
  const long long words = a.RSg * 4 * a.nt;
  if (words >= (1LL << 32)) return cudaErrorInvalidValue;  // the gather passes index words in 32 bits
  mp_load_kernel<V><<<grid_for(a.nt * (N / 4)), threads, 0, st>>>(a, cur);
  if ((e = launched()) != cudaSuccess) return e;
  const int smem = mp_solve_smem_bytes();
  e = cudaFuncSetAttribute(mp_solve_kernel<V, MP_TPB>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  const int half = N / 2;
  const unsigned nsolve = (unsigned)(4 * a.nt * ((half >> MP_LOG_S) / 2));  // nnode/2 + 1 per region
  // levels above the subproblem size, in bands of up to four levels
  const BandPlan bp = band_plan(logN, MP_LOG_S);
  auto fold = [&](int b, bool fwd) -> cudaError_t {
    const unsigned grid = grid_for(4 * a.nt * (half >> 2));
    switch (bp.R[b] * 2 + (fwd ? 1 : 0)) {
      case 3: mp_fold_band_kernel<V, true, 1><<<grid, threads, 0, st>>>(a, cur, bp.logL[b]); break;
      case 2: mp_fold_band_kernel<V, false, 1><<<grid, threads, 0, st>>>(a, cur, bp.logL[b]); break;
      case 5: mp_fold_band_kernel<V, true, 2><<<grid, threads, 0, st>>>(a, cur, bp.logL[b]); break;
      case 4: mp_fold_band_kernel<V, false, 2><<<grid, threads, 0, st>>>(a, cur, bp.logL[b]); break;
      case 7: mp_fold_band_kernel<V, true, 3><<<grid, threads, 0, st>>>(a, cur, bp.logL[b]); break;
      case 6: mp_fold_band_kernel<V, false, 3><<<grid, threads, 0, st>>>(a, cur, bp.logL[b]); break;
      case 9: mp_fold_band_kernel<V, true, 4><<<grid, threads, 0, st>>>(a, cur, bp.logL[b]); break;
      default: mp_fold_band_kernel<V, false, 4><<<grid, threads, 0, st>>>(a, cur, bp.logL[b]); break;
    }
    return launched();
  };
  // the M_v relation at node size 2^lp > S: the neighbour form in gather
  // form (a band would read its descendants bit-reversed, scattered across
  // sectors), or the recurrence as three in-place passes with the chunk
  // totals in the free ping-pong buffer
  auto relation = [&](int lp) -> cudaError_t {
    if constexpr (Var<V>::scan) {
      const long long nodes = 4 * a.nt * ((1LL << (logN - 1 - lp)) - 1);
      const long long chunks = nodes << (lp - 1 - MP_RLOG_C);
      mp_rec_total_kernel<V><<<grid_for(chunks), threads, 0, st>>>(a, cur, oth, lp);
      if ((e = launched()) != cudaSuccess) return e;
      mp_rec_scan_kernel<V><<<(unsigned)(nodes < 152LL * 16 ? nodes : 152LL * 16), 256, 0, st>>>(a, oth, lp);
      if ((e = launched()) != cudaSuccess) return e;
      mp_rec_apply_kernel<V><<<grid_for(chunks), threads, 0, st>>>(a, cur, oth, lp);
      return launched();
    } else {
      mp_neighbour_kernel<V><<<grid_for(words), threads, 0, st>>>(a, cur, oth, lp);
      if ((e = launched()) != cudaSuccess) return e;
      float* t = cur; cur = oth; oth = t;
      return cudaSuccess;
    }
  };
  if constexpr (Var<V>::ot) {
    for (int b = 0; b < bp.nb; ++b)
      if ((e = fold(b, true)) != cudaSuccess) return e;
    mp_solve_kernel<V, MP_TPB><<<nsolve, MP_TPB, smem, st>>>(a, cur, K);
    if ((e = launched()) != cudaSuccess) return e;
    int lp = MP_LOG_S + 2;  // 2^(S+1): in the solve
    if constexpr (!Var<V>::scan) {
      // the neighbour levels two a pass, a single one first when their count is odd
      if (lp <= logN - 2 && ((logN - 2 - lp + 1) & 1)) {
        if ((e = relation(lp)) != cudaSuccess) return e;
        ++lp;
      }
      for (; lp + 1 <= logN - 2; lp += 2) {
        mp_neighbour2_kernel<V><<<grid_for(words), threads, 0, st>>>(a, cur, oth, lp, lp + 1);
        if ((e = launched()) != cudaSuccess) return e;
        float* t = cur; cur = oth; oth = t;
      }
    } else {
      for (; lp <= logN - 2; ++lp)
        if ((e = relation(lp)) != cudaSuccess) return e;
    }
    // chain levels 2^(S+3) .. 2^(n-1): two a pass, a single one first when
    // their count is odd
    int lm = MP_LOG_S + 3;
    if (((logN - 1) - lm + 1) & 1) {
      mp_chain_kernel<V><<<grid_for(words), threads, 0, st>>>(a, cur, oth, lm);
      if ((e = launched()) != cudaSuccess) return e;
      float* t = cur; cur = oth; oth = t;
      ++lm;
    }
    for (; lm + 1 <= logN - 1; lm += 2) {
      mp_chain2_kernel<V><<<grid_for(words), threads, 0, st>>>(a, cur, oth, lm);
      if ((e = launched()) != cudaSuccess) return e;
      float* t = cur; cur = oth; oth = t;
    }
  } else {
    // chain levels 2^(n-1) .. 2^(S+3), descending, two a pass (a single one
    // first when their count is odd)
    int lm = logN - 1;
    if (((logN - 1) - (MP_LOG_S + 3) + 1) & 1) {
      mp_chain_kernel<V><<<grid_for(words), threads, 0, st>>>(a, cur, oth, lm);
      if ((e = launched()) != cudaSuccess) return e;
      float* t = cur; cur = oth; oth = t;
      --lm;
    }
    for (; lm - 1 >= MP_LOG_S + 3; lm -= 2) {
      mp_chain2_to_kernel<V><<<grid_for(words), threads, 0, st>>>(a, cur, oth, lm);
      if ((e = launched()) != cudaSuccess) return e;
      float* t = cur; cur = oth; oth = t;
    }
    int lp = logN - 2;  // down to 2^(S+2); 2^(S+1) is in the solve
    if constexpr (!Var<V>::scan) {
      if (lp >= MP_LOG_S + 2 && ((lp - (MP_LOG_S + 2) + 1) & 1)) {
        if ((e = relation(lp)) != cudaSuccess) return e;
        --lp;
      }
      for (; lp - 1 >= MP_LOG_S + 2; lp -= 2) {
        mp_neighbour2_kernel<V><<<grid_for(words), threads, 0, st>>>(a, cur, oth, lp, lp - 1);
        if ((e = launched()) != cudaSuccess) return e;
        float* t = cur; cur = oth; oth = t;
      }
    } else {
      for (; lp >= MP_LOG_S + 2; --lp)
        if ((e = relation(lp)) != cudaSuccess) return e;
    }
    mp_solve_kernel<V, MP_TPB><<<nsolve, MP_TPB, smem, st>>>(a, cur, K);
    if ((e = launched()) != cudaSuccess) return e;
    for (int b = bp.nb - 1; b >= 0; --b)
      if ((e = fold(b, false)) != cudaSuccess) return e;
  }
  if (a.dtype == 0) {
    mp_store_kernel<V><<<grid_for(a.nt * (N / 4)), threads, 0, st>>>(a, cur);
    return launched();
  }
  // 16-bit: the free ping-pong buffer holds the per-transform maxima
  int* Mx = reinterpret_cast<int*>(oth);
  mp_zero_kernel<V><<<(unsigned)((a.nt + 255) / 256), 256, 0, st>>>(Mx, a.nt);
  if ((e = launched()) != cudaSuccess) return e;
  mp_max_kernel<V><<<grid_for(a.nt * (N / 4)), threads, 0, st>>>(a, cur, Mx);
  if ((e = launched()) != cudaSuccess) return e;
  mp_store16_kernel<V><<<grid_for(a.nt * (N / 4)), threads, 0, st>>>(a, cur, Mx);
  return launched();
}

}  // namespace amqft
