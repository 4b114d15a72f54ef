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
  __device__ __forceinline__ RegP get(int tau, int kind) const {
    if constexpr (CL == 1) {
      return reg_ptr(sm + (4 * tau + kind) * RS, RS);
    } else {
      constexpr int PER = 4 / CL;
      cg::cluster_group cl = cg::this_cluster();
      float* remote = cl.map_shared_rank(sm, kind / PER);
      return reg_ptr(remote + (kind % PER) * RS, RS);
    }
  }
};

// ---- HBM elements: complex64, or 16-bit complex (a bf16 or fp16 pair, real
// part in the low half) holding value * 2^-exp with one exponent per
// transform ----
constexpr int DT_C64 = 0, DT_BF16 = 1, DT_F16 = 2, DT_I16 = 3;  // amqft_dtype

struct InRef {
  const void* p;
  const int* exp;  // per-transform exponents of 16-bit input (NULL: all 0)
  int dtype;
};

// 2^e as a float, exact (e clamped to the normal range)
__device__ __forceinline__ float pow2f(int e) {
  e = e < -126 ? -126 : (e > 127 ? 127 : e);
  return __int_as_float((127 + e) << 23);
}

__device__ __forceinline__ float2 unpack16(unsigned u, int dtype) {
  if (dtype == DT_BF16) return make_float2(__uint_as_float(u << 16), __uint_as_float(u & 0xffff0000u));
  if (dtype == DT_I16) return make_float2((float)(short)(u & 0xffffu), (float)(short)(u >> 16));
  return make_float2(__half2float(__ushort_as_half((unsigned short)(u & 0xffffu))),
                     __half2float(__ushort_as_half((unsigned short)(u >> 16))));
}

// int16: round to nearest even, saturated (a scaled output stays below 2^14)
__device__ __forceinline__ unsigned pack_i16(float v) {
  int q = __float2int_rn(v);
  q = q < -32768 ? -32768 : (q > 32767 ? 32767 : q);
  return (unsigned)(unsigned short)(short)q;
}

__device__ __forceinline__ unsigned pack16(float re, float im, int dtype) {
  if (dtype == DT_I16) return pack_i16(re) | (pack_i16(im) << 16);
  if (dtype == DT_BF16)
    return (unsigned)__bfloat16_as_ushort(__float2bfloat16_rn(re)) |
           ((unsigned)__bfloat16_as_ushort(__float2bfloat16_rn(im)) << 16);
  return (unsigned)__half_as_ushort(__float2half_rn(re)) | ((unsigned)__half_as_ushort(__float2half_rn(im)) << 16);
}

__device__ __forceinline__ float2 ldz(const float2* __restrict__ p, int i, float cj) {
  float2 v = __ldcs(p + i);
  v.y *= cj;
  return v;
}

// 16-bit element times the transform's scale 2^exp (exact)
__device__ __forceinline__ float2 ldz16(const unsigned* __restrict__ p, int i, int dtype, float s, float cj) {
  float2 v = unpack16(__ldcs(p + i), dtype);
  v.x *= s;
  v.y *= s * cj;
  return v;
}

__device__ __forceinline__ void stz(float2* __restrict__ p, int i, float re, float im, float cj) {
  __stcs(p + i, make_float2(re, im * cj));
}

// Exponent of a 16-bit output block whose largest component magnitude is m:
// the stored values are below 2^14 in magnitude (fp16 reaches 65504).
__device__ __forceinline__ int block_exponent(float m) {
  if (!(m > 0.f) || !isfinite(m)) return 0;
  int e = ((__float_as_int(m) >> 23) & 0xff) - 127;  // floor(log2 m) for normal m
  if (e < -126) e = -126;
  e -= 13;
  return e < -100 ? -100 : (e > 100 ? 100 : e);
}

// Load stage for orbit item n of transform tau: samples n, N-n, N/2-n, N/2+n
// (item 0: samples 0, N/2, N/4, 3N/4).  Fetch and scatter are separate so a
// thread's four items have their global loads in flight together.
struct Fetched {
  float2 a, b, c, d;
};

// t: transform id (indexes the exponents), off: element offset of its data
__device__ __forceinline__ Fetched load_fetch(const InRef& in, int logN, long long t, long long off, int n, float cj) {
  const int N = 1 << logN, half = N >> 1, Q = N >> 2;
  const float2* __restrict__ z = static_cast<const float2*>(in.p) + off;
  const unsigned* __restrict__ z16 = static_cast<const unsigned*>(in.p) + off;
  const bool c64 = in.dtype == DT_C64;  // the same for every thread
  const float s = (!c64 && in.exp) ? pow2f(__ldg(in.exp + t)) : 1.f;
  auto ld = [&](int i) {
    if (!AMQFT_IN_BOUNDS(i, N, BS_HBM_IN)) return make_float2(0.f, 0.f);
    return c64 ? ldz(z, i, cj) : ldz16(z16, i, in.dtype, s, cj);
  };
  Fetched f;
  if (n == 0) {
    f.a = ld(0);
    f.b = ld(half);
    if (N >= 4) {
      f.c = ld(Q);
      f.d = ld(3 * Q);
    }
  } else {
    f.a = ld(n);
    f.b = ld(N - n);
    f.c = ld(half - n);
    f.d = ld(half + n);
  }
  return f;
}

// Real input: samples n, N-n, N/2-n, N/2+n of real signals 2t (as the real
// part) and 2t+1 (as the imaginary part, zero past nreal).  The complex
// transform of a + ib then holds the DCT-0 / DST-0 of a in regions C1 / S1 and
// those of b in C2 / S2 (Sect. 3.1).
__device__ __forceinline__ Fetched load_fetch_real(const float* __restrict__ in, int logN, long long t,
                                                   long long nreal, int n) {
  const int N = 1 << logN, half = N >> 1, Q = N >> 2;
  const float* __restrict__ za = in + (2 * t) * (long long)N;
  const bool hb = 2 * t + 1 < nreal;
  const float* __restrict__ zb = za + N;
  auto ld = [&](int i) { return make_float2(__ldcs(za + i), hb ? __ldcs(zb + i) : 0.f); };
  Fetched f;
  if (n == 0) {
    f.a = ld(0);
    f.b = ld(half);
    if (N >= 4) {
      f.c = ld(Q);
      f.d = ld(3 * Q);
    }
  } else {
    f.a = ld(n);
    f.b = ld(N - n);
    f.c = ld(half - n);
    f.d = ld(half + n);
  }
  return f;
}

// Inverse real transform, orbit item n of transform t: the complex samples of
// Z = X_a + i X_b at n, N - n, N/2 - n, N/2 + n (item 0: 0, N/2, N/4, 3N/4),
// from the half spectra of signals 2t and 2t + 1 (Hermitian symmetry,
// X(N - j) = conj X(j)), conjugated (the inverse is conj F conj).
__device__ __forceinline__ Fetched load_fetch_irdft(const float2* __restrict__ in, int logN, long long t,
                                                    long long nsig, int n) {
  const int N = 1 << logN, half = N >> 1, Q = N >> 2;
  const float2* __restrict__ xa = in + (2 * t) * (long long)(half + 1);
  const float2* __restrict__ xb = xa + (half + 1);
  const bool hb = 2 * t + 1 < nsig;
  // conj(Z(j)) and conj(Z(N - j)) from X_a(j), X_b(j), 0 <= j <= N/2
  auto pair = [&](int j, float2& zj, float2& zmj) {
    const float2 A = __ldcs(xa + j), B = hb ? __ldcs(xb + j) : make_float2(0.f, 0.f);
    zj = make_float2(A.x - B.y, -(A.y + B.x));
    zmj = make_float2(A.x + B.y, -(B.x - A.y));
  };
  Fetched f;
  float2 u;
  if (n == 0) {
    pair(0, f.a, u);
    pair(half, f.b, u);
    if (N >= 4) pair(Q, f.c, f.d);
  } else {
    pair(n, f.a, f.b);
    pair(half - n, f.c, f.d);
  }
  return f;
}

// The D_r outputs of orbit item n for the two real signals of a transform
// (channel 1: the real parts, regions C1 / S1; channel 2: the imaginary
// parts, C2 / S2).  n > 0: a = dc(n), b = ds(n), c = dc(N/2-n), d = ds(N/2-n);
// n = 0: a = dc(0), b = dc(N/2), c = dc(N/4), d = ds(N/4) (N = 2: a, b only).
struct DrItem {
  float a1, b1, c1, d1, a2, b2, c2, d2;
};

// D_r (Eq. qft_22-23) on the four complex samples of item n:
// dc(n) = x(n) + x(N-n), ds(n) = x(n) - x(N-n); dc(0) = x(0), dc(N/2) = x(N/2).
__device__ __forceinline__ DrItem d_r(const Fetched& f, int N, int n) {
  DrItem r;
  if (n == 0) {
    r.a1 = f.a.x; r.b1 = f.b.x; r.a2 = f.a.y; r.b2 = f.b.y;
    if (N >= 4) {
      r.c1 = f.c.x + f.d.x; r.d1 = f.c.x - f.d.x; r.c2 = f.c.y + f.d.y; r.d2 = f.c.y - f.d.y;
    } else {
      r.c1 = r.d1 = r.c2 = r.d2 = 0.f;
    }
    return r;
  }
  r.a1 = f.a.x + f.b.x; r.b1 = f.a.x - f.b.x; r.c1 = f.c.x + f.d.x; r.d1 = f.c.x - f.d.x;
  r.a2 = f.a.y + f.b.y; r.b2 = f.a.y - f.b.y; r.c2 = f.c.y + f.d.y; r.d2 = f.c.y - f.d.y;
  return r;
}

// DCT-0 / DST-0 mode, orbit item n of transform t: the regions' inputs are
// the caller's signals themselves (no D_c, D_r).  Signals 2t (channel 1) and
// 2t + 1 (channel 2) of each kind; absent ones read as zero.
__device__ __forceinline__ DrItem load_fetch_trig(const float* __restrict__ dct, const float* __restrict__ dst,
                                                  long long ntrig, int logN, long long t, int n) {
  const int N = 1 << logN, half = N >> 1, Q = N >> 2;
  const long long s1 = 2 * t, s2 = 2 * t + 1;
  const long long c1 = s1 * (half + 1), c2 = s2 * (half + 1);  // DCT-0 input n at c + n
  const long long d1 = s1 * (half - 1) - 1, d2 = s2 * (half - 1) - 1;  // DST-0 input n at d + n
  const bool h1 = s1 < ntrig, h2 = s2 < ntrig;
  auto C = [&](bool ok, long long i) { return ok && dct ? __ldcs(dct + i) : 0.f; };
  auto S = [&](bool ok, long long i) { return ok && dst ? __ldcs(dst + i) : 0.f; };
  DrItem r;
  if (n == 0) {
    r.a1 = C(h1, c1); r.b1 = C(h1, c1 + half); r.c1 = C(h1, c1 + Q); r.d1 = S(h1, d1 + Q);
    r.a2 = C(h2, c2); r.b2 = C(h2, c2 + half); r.c2 = C(h2, c2 + Q); r.d2 = S(h2, d2 + Q);
    return r;
  }
  r.a1 = C(h1, c1 + n); r.b1 = S(h1, d1 + n); r.c1 = C(h1, c1 + half - n); r.d1 = S(h1, d1 + half - n);
  r.a2 = C(h2, c2 + n); r.b2 = S(h2, d2 + n); r.c2 = C(h2, c2 + half - n); r.d2 = S(h2, d2 + half - n);
  return r;
}

// Place item n's DCT-0 / DST-0 inputs in the four regions (chain layout; the
// harmonics-first variants also take the first D_k of the chain here).
template <int V, class RG>
__device__ __forceinline__ void load_place(const RG& rg, int logN, int tau, int n, const DrItem& r) {
  const int N = 1 << logN, half = N >> 1, Q = N >> 2, logQ = logN - 2;
  RegP C1 = rg.get(tau, 0);
  RegP S1 = rg.get(tau, 1);
  RegP C2 = rg.get(tau, 2);
  RegP S2 = rg.get(tau, 3);
  if (n == 0) {
    if (N == 2) {
      C1[0] = r.a1; C1[1] = r.b1; C2[0] = r.a2; C2[1] = r.b2;
      return;
    }
    if constexpr (Var<V>::ot) {
      C1[sw(half - 1)] = r.a1; C1[sw(half)] = r.b1;
      C2[sw(half - 1)] = r.a2; C2[sw(half)] = r.b2;
      C1[sw(half - 2)] = r.c1; C2[sw(half - 2)] = r.c2;   // pos_chain(Q, dct) = half - 2
      S1[sw(half - 2)] = r.d1; S2[sw(half - 2)] = r.d2;   // dst(4) base
    } else {
      C1[sw(Q)] = r.a1 + r.b1; C1[sw(0)] = r.a1 - r.b1;   // te(0), to(0)
      C2[sw(Q)] = r.a2 + r.b2; C2[sw(0)] = r.a2 - r.b2;
      C1[sw(half)] = r.c1; C2[sw(half)] = r.c2;           // te(Q) = dc(Q)
      S1[sw(Q - 1)] = r.d1; S2[sw(Q - 1)] = r.d2;         // to(Q) = ds(Q)
    }
    return;
  }
  const int m = half - n;
  if constexpr (Var<V>::ot) {
    const int pcn = sw(pos_chain(n, logN, 0)), pcm = sw(pos_chain(m, logN, 0));
    const int psn = sw(pos_chain(n, logN, 1)), psm = sw(pos_chain(m, logN, 1));
    C1[pcn] = r.a1; C1[pcm] = r.c1; S1[psn] = r.b1; S1[psm] = r.d1;
    C2[pcn] = r.a2; C2[pcm] = r.c2; S2[psn] = r.b2; S2[psm] = r.d2;
  } else {
    // first D_k of the chain (M = N): te -> dct(N/2), to -> dct_to(N) bit-reversed
    const int pte = sw(Q + n), pto = sw(brev(n, logQ));
    const int ste = sw(Q + n - 1), sto = sw(brev(n - 1, logQ));
    C1[pte] = r.a1 + r.c1; C1[pto] = r.a1 - r.c1;
    C2[pte] = r.a2 + r.c2; C2[pto] = r.a2 - r.c2;
    S1[ste] = r.b1 - r.d1; S1[sto] = r.b1 + r.d1;
    S2[ste] = r.b2 - r.d2; S2[sto] = r.b2 + r.d2;
  }
}

template <int V, class RG>
__device__ __forceinline__ void load_scatter(const RG& rg, int logN, int tau, int n, const Fetched& f) {
  load_place<V>(rg, logN, tau, n, d_r(f, 1 << logN, n));
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
  CRegP C1 = rg.get(tau, 0);
  CRegP S1 = rg.get(tau, 1);
  CRegP C2 = rg.get(tau, 2);
  CRegP S2 = rg.get(tau, 3);
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

// The (up to) four outputs of orbit item k: harmonics k, N-k, N/2-k, N/2+k
// (item 0: 0, N/2, N/4, 3N/4; N = 2: 0, 1).  Index -1 marks an unused slot.
struct Out4 {
  float2 v[4];
  int i[4];
};

template <int V>
__device__ __forceinline__ Out4 emit_values(int logN, int k, const Gathered& g) {
  const int N = 1 << logN, half = N >> 1, Q = N >> 2;
  Out4 o;
  if (k == 0) {
    if (N == 2) {
      o.v[0] = make_float2(g.v[0], g.v[2]); o.i[0] = 0;
      o.v[1] = make_float2(g.v[1], g.v[3]); o.i[1] = 1;
      o.i[2] = -1; o.i[3] = -1;
      o.v[2] = o.v[3] = make_float2(0.f, 0.f);
      return o;
    }
    float c01, c02, ch1, ch2;
    if constexpr (Var<V>::ot) {
      // last D_n of the chain (M = N) at k = 0
      c01 = g.v[0] + g.v[1]; ch1 = g.v[0] - g.v[1]; c02 = g.v[2] + g.v[3]; ch2 = g.v[2] - g.v[3];
    } else {
      c01 = g.v[0]; ch1 = g.v[1]; c02 = g.v[2]; ch2 = g.v[3];
    }
    const float cq1 = g.v[4], cq2 = g.v[5], sq1 = g.v[6], sq2 = g.v[7];
    o.v[0] = make_float2(c01, c02); o.i[0] = 0;
    o.v[1] = make_float2(ch1, ch2); o.i[1] = half;
    o.v[2] = make_float2(cq1 + sq2, cq2 - sq1); o.i[2] = Q;
    o.v[3] = make_float2(cq1 - sq2, cq2 + sq1); o.i[3] = 3 * Q;
    return o;
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
  o.v[0] = make_float2(ck1 + sk2, ck2 - sk1); o.i[0] = k;
  o.v[1] = make_float2(ck1 - sk2, ck2 + sk1); o.i[1] = N - k;
  o.v[2] = make_float2(cm1 + sm2, cm2 - sm1); o.i[2] = m;
  o.v[3] = make_float2(cm1 - sm2, cm2 + sm1); o.i[3] = half + k;
  return o;
}

// Real input, orbit item k: harmonics k and N/2 - k (item 0: 0, N/2, N/4)
// of both signals of the pair, R = DCT - i DST (Eq. qft_24-25), written to the
// half spectra (N/2 + 1 values each) of signals 2t and 2t+1.
template <int V>
__device__ __forceinline__ void store_real(float2* __restrict__ out, int logN, long long t, long long nreal, int k,
                                           const Gathered& g) {
  const int N = 1 << logN, half = N >> 1, Q = N >> 2;
  float2* __restrict__ ra = out + (2 * t) * (long long)(half + 1);
  float2* __restrict__ rb = ra + (half + 1);
  const bool hb = 2 * t + 1 < nreal;
  if (k == 0) {
    if (N == 2) {
      __stcs(ra, make_float2(g.v[0], 0.f));
      __stcs(ra + 1, make_float2(g.v[1], 0.f));
      if (hb) {
        __stcs(rb, make_float2(g.v[2], 0.f));
        __stcs(rb + 1, make_float2(g.v[3], 0.f));
      }
      return;
    }
    float c01, c02, ch1, ch2;
    if constexpr (Var<V>::ot) {
      c01 = g.v[0] + g.v[1]; ch1 = g.v[0] - g.v[1]; c02 = g.v[2] + g.v[3]; ch2 = g.v[2] - g.v[3];
    } else {
      c01 = g.v[0]; ch1 = g.v[1]; c02 = g.v[2]; ch2 = g.v[3];
    }
    __stcs(ra, make_float2(c01, 0.f));
    __stcs(ra + half, make_float2(ch1, 0.f));
    __stcs(ra + Q, make_float2(g.v[4], -g.v[6]));
    if (hb) {
      __stcs(rb, make_float2(c02, 0.f));
      __stcs(rb + half, make_float2(ch2, 0.f));
      __stcs(rb + Q, make_float2(g.v[5], -g.v[7]));
    }
    return;
  }
  float ck1, ck2, cm1, cm2, sk1, sk2, sm1, sm2;
  if constexpr (Var<V>::ot) {
    ck1 = g.v[0] + g.v[1]; cm1 = g.v[0] - g.v[1]; ck2 = g.v[2] + g.v[3]; cm2 = g.v[2] - g.v[3];
    sk1 = g.v[4] + g.v[5]; sm1 = g.v[4] - g.v[5]; sk2 = g.v[6] + g.v[7]; sm2 = g.v[6] - g.v[7];
  } else {
    ck1 = g.v[0]; cm1 = g.v[1]; ck2 = g.v[2]; cm2 = g.v[3];
    sk1 = g.v[4]; sm1 = g.v[5]; sk2 = g.v[6]; sm2 = g.v[7];
  }
  __stcs(ra + k, make_float2(ck1, -sk1));
  __stcs(ra + (half - k), make_float2(cm1, -sm1));
  if (hb) {
    __stcs(rb + k, make_float2(ck2, -sk2));
    __stcs(rb + (half - k), make_float2(cm2, -sm2));
  }
}

__device__ __forceinline__ float out4_absmax(const Out4& o) {
  float m = 0.f;
#pragma unroll
  for (int j = 0; j < 4; ++j)
    if (o.i[j] >= 0) m = fmaxf(m, fmaxf(fabsf(o.v[j].x), fabsf(o.v[j].y)));
  return m;
}

template <int V>
__device__ __forceinline__ void store_emit(float2* __restrict__ out, int logN, long long off, int k, const Gathered& g,
                                           float cj) {
  const Out4 o = emit_values<V>(logN, k, g);
  float2* __restrict__ z = out + off;
  const int N = 1 << logN;
  (void)N;  // the bound of the checked build
#pragma unroll
  for (int j = 0; j < 4; ++j)
    if (o.i[j] >= 0 && AMQFT_IN_BOUNDS(o.i[j], N, BS_HBM_OUT)) stz(z, o.i[j], o.v[j].x, o.v[j].y, cj);
}

// 16-bit output of one item, every value times s = 2^-exp (exact)
__device__ __forceinline__ void store16(unsigned* __restrict__ out, long long off, const Out4& o, float s, float cj,
                                        int dtype) {
  unsigned* __restrict__ z = out + off;
#pragma unroll
  for (int j = 0; j < 4; ++j)
    if (o.i[j] >= 0) __stcs(z + o.i[j], pack16(o.v[j].x * s, o.v[j].y * (s * cj), dtype));
}

// ---------------------------------------------------------------------
// chain of the time-first variants, cluster path: two levels per pass
// ---------------------------------------------------------------------
// Levels M and 2M of the D_n frequency phase (dct S(k) = E(k) + O(k),
// S(M/2-k) = E(k) - O(k); dst S(k) = O(k-1) + E(k), S(M/2-k) = O(k-1) - E(k))
// in one read / barrier / write pass: item j takes E_M(j) and O_M(j), forms
// S_M(j) and S_M(M/2-j), and combines each with the 2M tree's O_2M at the same
// harmonic, giving S_2M at j, M-j, M/2-j and M/2+j.  The float32 operations
// and their order are those of two separate levels.  FINAL (2M = N): the
// result is written in natural order, unswizzled, word k holding harmonic k
// (DST words 0 and N/2 zero), the layout the cluster store reads.
template <int V, int TPB, int LOGM, bool FINAL>
__device__ __forceinline__ void pass_chain2(RegP R, int half, int ctx) {
  constexpr int M = 1 << LOGM, Q1 = M / 4, Q2 = M / 2, L1 = LOGM - 2, L2 = LOGM - 1;
  constexpr int NI = (Q1 + 1 + TPB - 1) / TPB;
  const int P1 = half - M / 2, P2 = half - M;
  float va[NI], vb[NI], vc[NI], vd[NI];
#pragma unroll
  for (int s = 0; s < NI; ++s) {
    const int w = (int)threadIdx.x + s * TPB;
    va[s] = vb[s] = vc[s] = vd[s] = 0.f;
    if (ctx == 0 && w <= Q1) {
      const int j = w;
      float sA, sB = 0.f;
      if (j < Q1) {
        const float e = R[sw(P1 + Q1 + j)], o = R[sw(P1 + brev(j, L1))];
        sA = e + o;
        sB = e - o;
      } else {
        sA = R[sw(P1 + 2 * Q1)];
      }
      const float o2 = R[sw(P2 + brev(j, L2))];
      va[s] = sA + o2;
      vb[s] = sA - o2;
      if (j < Q1) {
        if (j > 0) {
          const float o2b = R[sw(P2 + brev(Q2 - j, L2))];
          vc[s] = sB + o2b;
          vd[s] = sB - o2b;
        } else {
          vc[s] = sB;  // S_2M(M/2) = S_M(M/2)
        }
      }
    } else if (ctx == 1 && w < Q1) {
      const int j = w + 1;
      float sA, sB = 0.f;
      if (j < Q1) {
        const float o = R[sw(P1 + brev(j - 1, L1))], e = R[sw(P1 + Q1 + j - 1)];
        sA = o + e;
        sB = o - e;
      } else {
        sA = R[sw(P1 + Q1 - 1)];  // S_M(M/4) = O_M(M/4 - 1)
      }
      const float o2 = R[sw(P2 + brev(j - 1, L2))];
      va[s] = o2 + sA;
      vb[s] = o2 - sA;
      if (j < Q1) {
        const float o2b = R[sw(P2 + brev(Q2 - j - 1, L2))];
        vc[s] = o2b + sB;
        vd[s] = o2b - sB;
      }
    }
  }
  float mid = 0.f;
  if (FINAL && ctx == 1 && threadIdx.x == 0) mid = R[sw(P2 + Q2 - 1)];  // S_N(N/4) = O_N(N/4 - 1)
  __syncthreads();
  auto put = [&](int k, float v) {
    if constexpr (FINAL) R[k] = v;
    else R[sw(P2 + (ctx == 0 ? k : k - 1))] = v;
  };
#pragma unroll
  for (int s = 0; s < NI; ++s) {
    const int w = (int)threadIdx.x + s * TPB;
    if (ctx == 0 && w <= Q1) {
      const int j = w;
      put(j, va[s]);
      put(M - j, vb[s]);
      if (j < Q1) {
        if (j > 0) {
          put(Q2 - j, vc[s]);
          put(Q2 + j, vd[s]);
        } else {
          put(Q2, vc[s]);
        }
      }
    } else if (ctx == 1 && w < Q1) {
      const int j = w + 1;
      put(j, va[s]);
      put(M - j, vb[s]);
      if (j < Q1) {
        put(Q2 - j, vc[s]);
        put(Q2 + j, vd[s]);
      }
    }
  }
  if (FINAL && ctx == 1 && threadIdx.x == 0) {
    R[Q2] = mid;
    R[0] = 0.f;
    R[2 * Q2] = 0.f;
  }
}

// Pairs of chain levels LO, LO + 1, ... below the final pair (LN - 1, LN).
template <int V, int TPB, int LN, int LO>
__device__ __forceinline__ void chain_pairs(RegP R, int half, int ctx) {
  if constexpr (LO + 1 <= LN - 2) {
    pass_chain2<V, TPB, LO, false>(R, half, ctx);
    __syncthreads();
    chain_pairs<V, TPB, LN, LO + 2>(R, half, ctx);
  }
}

// ---------------------------------------------------------------------
// store of the cluster path, in two stages
// ---------------------------------------------------------------------
// Stage 1, local: the CTA's own region is rewritten in natural frequency
// order, unswizzled (word k holds DCT/DST value k; DST words 0 and N/2 hold
// 0).  Time-first variants apply the last chain level here (D_n frequency
// phase, M = N): dct S(k) = E(k) + O(k), S(N/2-k) = E(k) - O(k), with E the
// dct(N/2) result at [Q, 2Q] and O the dct_ot(N) result in bit-reversed order
// at [0, Q); dst S(k) = O(k-1) + E(k-1), S(N/2-k) = O(k-1) - E(k-1),
// S(Q) = O(Q-1).  Harmonics-first variants only undo the chain layout.
// Every thread reads its values, then the block synchronises, then writes.
template <int V, int TPB, int LN>
__device__ __forceinline__ void region_to_natural(RegP R, int ctx) {
  constexpr int N = 1 << LN, half = N >> 1, Q = N >> 2, logQ = LN - 2;
  if constexpr (Var<V>::ot) {
    constexpr int NI = Q / TPB;
    float a[NI], b[NI];
    float mid = 0.f;
#pragma unroll
    for (int s = 0; s < NI; ++s) {
      const int j = threadIdx.x + s * TPB;
      const float o = R[sw(brev(j, logQ))];
      if (ctx == 0) {
        const float e = R[sw(Q + j)];
        a[s] = e + o;
        b[s] = e - o;
      } else if (j < Q - 1) {
        const float e = R[sw(Q + j)];
        a[s] = o + e;
        b[s] = o - e;
      } else {
        a[s] = o;  // S(Q)
        b[s] = 0.f;
      }
    }
    if (ctx == 0 && threadIdx.x == 0) mid = R[sw(half)];  // C(Q) = E(Q)
    __syncthreads();
#pragma unroll
    for (int s = 0; s < NI; ++s) {
      const int j = threadIdx.x + s * TPB;
      if (ctx == 0) {
        R[j] = a[s];
        R[half - j] = b[s];
      } else if (j < Q - 1) {
        R[j + 1] = a[s];
        R[half - j - 1] = b[s];
      } else {
        R[Q] = a[s];
      }
    }
    if (threadIdx.x == 0) {
      if (ctx == 0) {
        R[Q] = mid;
      } else {
        R[0] = 0.f;
        R[half] = 0.f;
      }
    }
  } else {
    constexpr int NI = half / TPB;
    float a[NI];
    float last = 0.f;
#pragma unroll
    for (int s = 0; s < NI; ++s) {
      const int k = threadIdx.x + s * TPB;
      a[s] = (ctx == 0 || k > 0) ? R[sw(pos_chain(k, LN, ctx))] : 0.f;
    }
    if (ctx == 0 && threadIdx.x == 0) last = R[sw(half)];  // C(N/2)
    __syncthreads();
#pragma unroll
    for (int s = 0; s < NI; ++s) R[threadIdx.x + s * TPB] = a[s];
    if (threadIdx.x == 0) R[half] = last;
  }
}

// DCT-0 / DST-0 mode, orbit item k: the regions' own results (no D_r^F,
// D_c^F) at harmonics k and N/2 - k (item 0: 0, N/2, N/4) to the DCT-0 and
// DST-0 outputs of signals 2t and 2t + 1.
template <int V>
__device__ __forceinline__ void store_trig(float* __restrict__ dct, float* __restrict__ dst, long long ntrig,
                                           int logN, long long t, int k, const Gathered& g) {
  const int N = 1 << logN, half = N >> 1, Q = N >> 2;
  const long long s1 = 2 * t, s2 = 2 * t + 1;
  const long long c1 = s1 * (half + 1), c2 = s2 * (half + 1);
  const long long d1 = s1 * (half - 1) - 1, d2 = s2 * (half - 1) - 1;
  const bool h1 = s1 < ntrig, h2 = s2 < ntrig;
  auto C = [&](bool ok, long long i, float v) { if (ok && dct) __stcs(dct + i, v); };
  auto S = [&](bool ok, long long i, float v) { if (ok && dst) __stcs(dst + i, v); };
  float ck1, ck2, cm1, cm2, sk1, sk2, sm1, sm2;
  if constexpr (Var<V>::ot) {  // last D_n of the chain (M = N)
    ck1 = g.v[0] + g.v[1]; cm1 = g.v[0] - g.v[1]; ck2 = g.v[2] + g.v[3]; cm2 = g.v[2] - g.v[3];
  } else {
    ck1 = g.v[0]; cm1 = g.v[1]; ck2 = g.v[2]; cm2 = g.v[3];
  }
  if (k == 0) {  // C(0) = ck, C(N/2) = cm, C(N/4) and S(N/4) as gathered
    C(h1, c1, ck1); C(h1, c1 + half, cm1); C(h1, c1 + Q, g.v[4]); S(h1, d1 + Q, g.v[6]);
    C(h2, c2, ck2); C(h2, c2 + half, cm2); C(h2, c2 + Q, g.v[5]); S(h2, d2 + Q, g.v[7]);
    return;
  }
  if constexpr (Var<V>::ot) {
    sk1 = g.v[4] + g.v[5]; sm1 = g.v[4] - g.v[5]; sk2 = g.v[6] + g.v[7]; sm2 = g.v[6] - g.v[7];
  } else {
    sk1 = g.v[4]; sm1 = g.v[5]; sk2 = g.v[6]; sm2 = g.v[7];
  }
  C(h1, c1 + k, ck1); C(h1, c1 + half - k, cm1); S(h1, d1 + k, sk1); S(h1, d1 + half - k, sm1);
  C(h2, c2 + k, ck2); C(h2, c2 + half - k, cm2); S(h2, d2 + k, sk2); S(h2, d2 + half - k, sm2);
}

// Inverse real transform, orbit item k: the up to four outputs of the
// complex inverse of Z = X_a + i X_b; their real parts are N x_a, their
// imaginary parts N x_b (signals 2t and 2t + 1, N floats each).
template <int V>
__device__ __forceinline__ void store_irdft(float* __restrict__ out, long long nsig, int logN, long long t, int k,
                                            const Gathered& g, float cj) {
  const int N = 1 << logN;
  float* __restrict__ xa = out + (2 * t) * (long long)N;
  float* __restrict__ xb = xa + N;
  const bool hb = 2 * t + 1 < nsig;
  const Out4 o = emit_values<V>(logN, k, g);
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    if (o.i[i] < 0) continue;
    __stcs(xa + o.i[i], o.v[i].x);
    if (hb) __stcs(xb + o.i[i], o.v[i].y * cj);
  }
}

// Stage 2, across the cluster: D_r^F (Eq. qft_24-25: Re R = DCT, Im R = -DST)
// and D_c^F (Eq. qft_17-21) for four consecutive harmonics per step, the four
// regions read as float4 through distributed shared memory:
//   X(k) = (C1 + S2, C2 - S1),  X(N-k) = (C1 - S2, C2 + S1),  k = 1..N/2-1,
//   X(0) = (C1(0), C2(0)),  X(N/2) = (C1(N/2), C2(N/2)).
// CTA r of the cluster (region r) covers k in [r N/8, (r+1) N/8).
template <int TPB, int LN>
__device__ __forceinline__ void store_natural_cluster(float* sm, const FusedArgs& a, long long t, long long off,
                                                      float cj, float* red) {
  constexpr int N = 1 << LN, half = N >> 1, PER = half / 4, NG = PER / 4 / TPB;
  static_assert(NG * 4 * TPB == PER, "four harmonics per thread and step");
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank();
  if (a.ntrig > 0) {
    // DCT-0 / DST-0 mode: each CTA writes its own region, in natural order
    const long long sig = 2 * t + (rank >> 1);
    if (sig < a.ntrig) {
      if ((rank & 1) == 0 && a.out) {
        float* __restrict__ o = static_cast<float*>(a.out) + sig * (long long)(half + 1);
        for (int k = (int)threadIdx.x; k <= half; k += TPB) __stcs(o + k, sm[k]);
      } else if ((rank & 1) == 1 && a.out2) {
        float* __restrict__ o = a.out2 + sig * (long long)(half - 1) - 1;
        for (int k = 1 + (int)threadIdx.x; k < half; k += TPB) __stcs(o + k, sm[k]);
      }
    }
    return;
  }
  if (a.nreal > 0) {
    // real input: R = DCT - i DST of each signal of the pair, harmonics 0 .. N/2
    float2* __restrict__ ra = static_cast<float2*>(a.out) + (2 * t) * (long long)(half + 1);
    float2* __restrict__ rb = ra + (half + 1);
    const bool hb = 2 * t + 1 < a.nreal;
    const float* c1 = cl.map_shared_rank(sm, 0);
    const float* s1 = cl.map_shared_rank(sm, 1);
    const float* c2 = cl.map_shared_rank(sm, 2);
    const float* s2 = cl.map_shared_rank(sm, 3);
    for (int k = rank * PER + (int)threadIdx.x; k < (rank + 1) * PER; k += TPB) {
      __stcs(ra + k, make_float2(c1[k], k == 0 ? 0.f : -s1[k]));
      if (hb) __stcs(rb + k, make_float2(c2[k], k == 0 ? 0.f : -s2[k]));
    }
    if (rank == 0 && threadIdx.x == 0) {
      __stcs(ra + half, make_float2(c1[half], 0.f));
      if (hb) __stcs(rb + half, make_float2(c2[half], 0.f));
    }
    return;
  }
  const float4* C1 = reinterpret_cast<const float4*>(cl.map_shared_rank(sm, 0));
  const float4* S1 = reinterpret_cast<const float4*>(cl.map_shared_rank(sm, 1));
  const float4* C2 = reinterpret_cast<const float4*>(cl.map_shared_rank(sm, 2));
  const float4* S2 = reinterpret_cast<const float4*>(cl.map_shared_rank(sm, 3));
  // X(k0 + i) -> f[i], X(N - k0 - i) -> b[i] (k0 = 0: b[0] = X(N/2))
  auto group = [&](int gi, float2 (&f)[4], float2 (&b)[4]) {
    const int k0 = rank * PER + 4 * ((int)threadIdx.x + gi * TPB);
    const float4 c1 = C1[k0 >> 2], s1 = S1[k0 >> 2], c2 = C2[k0 >> 2], s2 = S2[k0 >> 2];
    const float a1[4] = {c1.x, c1.y, c1.z, c1.w}, b1[4] = {s1.x, s1.y, s1.z, s1.w};
    const float a2[4] = {c2.x, c2.y, c2.z, c2.w}, b2[4] = {s2.x, s2.y, s2.z, s2.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      f[i] = make_float2(a1[i] + b2[i], a2[i] - b1[i]);
      b[i] = make_float2(a1[i] - b2[i], a2[i] + b1[i]);
    }
    if (k0 == 0) {  // X(0) = (C1(0), C2(0)); X(N/2) = (C1(N/2), C2(N/2))
      f[0] = make_float2(a1[0], a2[0]);
      b[0] = make_float2(cl.map_shared_rank(sm, 0)[half], cl.map_shared_rank(sm, 2)[half]);
    }
    return k0;
  };
  if (a.nirdft > 0) {
    // inverse real transform: Re -> signal 2t, Im -> signal 2t + 1
    float* __restrict__ xa = static_cast<float*>(a.out) + (2 * t) * (long long)N;
    float* __restrict__ xb = xa + N;
    const bool hb = 2 * t + 1 < a.nirdft;
#pragma unroll
    for (int gi = 0; gi < NG; ++gi) {
      float2 f[4], b[4];
      const int k0 = group(gi, f, b);
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int kb = k0 == 0 && i == 0 ? half : N - k0 - i;
        __stcs(xa + k0 + i, f[i].x);
        __stcs(xa + kb, b[i].x);
        if (hb) {
          __stcs(xb + k0 + i, f[i].y * cj);
          __stcs(xb + kb, b[i].y * cj);
        }
      }
    }
    return;
  }
  if (a.dtype == DT_C64) {
    float2* __restrict__ z = static_cast<float2*>(a.out) + off;
    const bool vec_ok = (reinterpret_cast<uintptr_t>(z) & 15u) == 0;  // same for every thread
#pragma unroll
    for (int gi = 0; gi < NG; ++gi) {
      float2 f[4], b[4];
      const int k0 = group(gi, f, b);
      if (vec_ok) {
        __stcs(reinterpret_cast<float4*>(z + k0), make_float4(f[0].x, f[0].y * cj, f[1].x, f[1].y * cj));
        __stcs(reinterpret_cast<float4*>(z + k0 + 2), make_float4(f[2].x, f[2].y * cj, f[3].x, f[3].y * cj));
      } else {  // out is only 8-byte aligned
#pragma unroll
        for (int i = 0; i < 4; ++i) stz(z, k0 + i, f[i].x, f[i].y, cj);
      }
#pragma unroll
      for (int i = 0; i < 4; ++i) stz(z, k0 == 0 && i == 0 ? half : N - k0 - i, b[i].x, b[i].y, cj);
    }
    return;
  }
  // 16-bit: the largest component magnitude of the transform fixes its
  // exponent; the outputs are then recomputed, scaled by 2^-exp and rounded
  float m = 0.f;
#pragma unroll
  for (int gi = 0; gi < NG; ++gi) {
    float2 f[4], b[4];
    group(gi, f, b);
#pragma unroll
    for (int i = 0; i < 4; ++i)
      m = fmaxf(m, fmaxf(fmaxf(fabsf(f[i].x), fabsf(f[i].y)), fmaxf(fabsf(b[i].x), fabsf(b[i].y))));
  }
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, d));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    float bm = 0.f;
    for (int w = 0; w < TPB / 32; ++w) bm = fmaxf(bm, red[w]);
    sm[half + 1] = bm;  // word N/2 + 1 of the region is free
  }
  cl.sync();
  float M = 0.f;
#pragma unroll
  for (int r = 0; r < 4; ++r) M = fmaxf(M, cl.map_shared_rank(sm, r)[half + 1]);
  const int e = block_exponent(M);
  const float sc = pow2f(-e), si = sc * cj;
  if (rank == 0 && threadIdx.x == 0) a.exp_out[t] = e;
  unsigned* __restrict__ z = static_cast<unsigned*>(a.out) + off;
  const bool vec_ok = (reinterpret_cast<uintptr_t>(z) & 15u) == 0;
#pragma unroll
  for (int gi = 0; gi < NG; ++gi) {
    float2 f[4], b[4];
    const int k0 = group(gi, f, b);
    unsigned u[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) u[i] = pack16(f[i].x * sc, f[i].y * si, a.dtype);
    if (vec_ok) {
      __stcs(reinterpret_cast<uint4*>(z + k0), make_uint4(u[0], u[1], u[2], u[3]));
    } else {
#pragma unroll
      for (int i = 0; i < 4; ++i) __stcs(z + k0 + i, u[i]);
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
      __stcs(z + (k0 == 0 && i == 0 ? half : N - k0 - i), pack16(b[i].x * sc, b[i].y * si, a.dtype));
  }
}

// The tree and chain stages of the fused transform on the CTA's regions (g),
// between the load and the store.  cctx: the region context on the cluster
// path (LN > 0), where the final chain pair writes natural order.
template <int V, int TPB, int MAXI, int CL, int LN>
__device__ __forceinline__ void fused_compute(float* sm, const Geo& g, const TabConsts& ctab,
                                              const SmallConsts& K, float* tot, float* wsum, float* snap, int cctx) {
  const int logN = LN > 0 ? LN : g.logN, half = 1 << (logN - 1);
  (void)tot;
  (void)wsum;
  (void)cctx;
  const int logTop = logN - 2;  // log2 of the largest tree (N/4)
  const BandPlan bp = band_plan(logN);
  // the recurrences' scan chunking of the single-CTA path follows its
  // 256-thread shape in every launch shape (a transform's bits never depend on
  // the shape that ran it)
  constexpr int RC_TPB = CL == 1 ? SMALL_TPB : TPB, RC_MAXI = CL == 1 ? SMALL_MAXI : MAXI;
  if constexpr (Var<V>::ot) {
#pragma unroll
    for (int b = 0; b < bp.nb; ++b) {
      run_fold_band_r<V, TPB>(sm, g, bp.logL[b], bp.R[b], true, ctab);
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
          run_leaf<V>(reg_ptr(sm + r * g.RS, g.RS), p0, node_ctx_g<V>(g, p0, LOG_LEAF, ctx_of(g, r)), K);
        } else {
          const int r = w - g.nreg * nleaf;
          run_tail<V>(reg_ptr(sm + r * g.RS, g.RS), ctx_of(g, r), logN, K);
        }
      }
      __syncthreads();
    }
    if constexpr (Var<V>::scan) {
      for (int lp = LOG_LEAF + 1; lp <= logTop; ++lp) {
        pass_recurrence<V, TPB, RC_MAXI, RC_TPB>(sm, tot, wsum, g, lp);
        __syncthreads();
      }
    } else {
#pragma unroll
      for (int b = bp.nb - 1; b >= 0; --b) {
        run_chunk_band_r<V, TPB>(sm, snap, g, bp.logL[b], bp.R[b]);
        __syncthreads();
      }
    }
    if constexpr (CL > 1 && LN > 0) {
      // levels 2^7 .. 2^(LN-2) in pairs (a single level first when their
      // count is odd), then the final pair (2^(LN-1), 2^LN) in natural order
      constexpr int LO = LOG_LEAF + 2;
      constexpr int LO2 = ((LN - 1 - LO) & 1) ? LO + 1 : LO;
      const int ctx = cctx;
      if constexpr (LO2 > LO) {
        pass_chain<V, TPB, MAXI>(sm, g, LO);
        __syncthreads();
      }
      chain_pairs<V, TPB, LN, LO2>(reg_ptr(sm, region_stride(LN)), half, ctx);
      pass_chain2<V, TPB, LN - 1, true>(reg_ptr(sm, region_stride(LN)), half, ctx);
    } else {
      for (int lm = LOG_LEAF + 2; lm <= logN - 1; ++lm) {
        pass_chain<V, TPB, MAXI>(sm, g, lm);
        __syncthreads();
      }
    }
  } else {
    for (int lm = logN - 1; lm >= LOG_LEAF + 2; --lm) {
      pass_chain<V, TPB, MAXI>(sm, g, lm);
      __syncthreads();
    }
    for (int r = threadIdx.x; r < g.nreg; r += TPB) run_tail<V>(reg_ptr(sm + r * g.RS, g.RS), ctx_of(g, r), logN, K);
    __syncthreads();
    for (int lp = logTop; lp >= LOG_LEAF + 1; --lp) {
      if constexpr (Var<V>::scan) pass_recurrence<V, TPB, RC_MAXI, RC_TPB>(sm, tot, wsum, g, lp);
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
        run_leaf<V>(reg_ptr(sm + r * g.RS, g.RS), p0, node_ctx_g<V>(g, p0, LOG_LEAF, ctx_of(g, r)), K);
      }
      __syncthreads();
    }
#pragma unroll
    for (int b = bp.nb - 1; b >= 0; --b) {
      run_fold_band_r<V, TPB>(sm, g, bp.logL[b], bp.R[b], false, ctab);
      __syncthreads();
    }
  }

}

// The fused transform of the CTA (cluster size 1: transforms at list
// positions [j0, j0 + ntr)) or of the cluster (list position j0).  LN > 0:
// compiled for log2 N = LN (every index computation is then resolved at
// compile time); LN == 0: a.logN at run time.
// logN_rt, RS_rt: the length and region stride when LN == 0; tot_off: float
// offset of the scan scratch; tlist: transform ids by list position (NULL:
// the position itself).  Everything else comes from a.
template <int V, int TPB, int MAXI, int CL, int LN>
__device__ __forceinline__ void fused_body(const FusedArgs& a, const SmallConsts& K, float* sm, long long j0, int ntr,
                                           int logN_rt, int RS_rt, int tot_off, const int* tlist) {
  const int logN = LN > 0 ? LN : logN_rt, N = 1 << logN, half = N >> 1;
  const int RS = LN > 0 ? region_stride(LN) : RS_rt;
  const int Qi = N >= 4 ? (N >> 2) : 1;   // orbit items per transform
  const int logQi = N >= 4 ? logN - 2 : 0;
  const float cj = a.inverse ? -1.f : 1.f;
  Geo g;
  g.logN = logN;
  g.half = half;
  g.RS = RS;
  g.sub = 0;
  Regions<CL> rg;
  rg.sm = sm;
  rg.RS = RS;
  rg.tbase = j0;
  // transform id of local transform tau, and the element offset of an id
  auto tid = [&](int tau) -> long long {
    const long long j = j0 + tau;
    return tlist ? (long long)__ldg(tlist + j) : j;
  };
  auto toff = [&](long long t) -> long long { return a.toff ? __ldg(a.toff + t) : (t << logN); };
  if constexpr (CL == 1) {
    g.nreg = 4 * ntr;
    g.nreg_cap = 4 * small_tpc(logN);
    g.gbase = 0;
  } else {
    cg::cluster_group cl = cg::this_cluster();
    g.nreg = 4 / CL;
    g.nreg_cap = 4 / CL;
    g.gbase = (int)cl.block_rank() * (4 / CL);
    cl.sync();  // every CTA of the cluster is resident (and done with the previous transform)
  }
  float* tot = sm + tot_off;
  float* wsum = tot + TPB;
  float* snap = wsum + 32;
  // the band levels' constants (table entries 30 ..), after the exponent
  // slots: copied from the plan's table, or evaluated on the fly (ctab NULL);
  // visible to the bands after the barrier that ends the load
  float* cst = snap + snap_floats(g.nreg_cap * half) + (CL == 1 ? small_tpc(logN) : 1);
  stage_consts<V>(cst, band_consts(logN), a.ctab, (int)threadIdx.x, TPB);

  // ---- load ----
  // every configuration gives each thread exactly NIT orbit items, taken in
  // rounds of U so that a round's global loads are in flight together
  constexpr int NIT = (CL > 1 && LN > 0) ? (1 << (LN - 4)) / TPB : 2048 / TPB;
  constexpr int U = NIT < 4 ? NIT : 4, NR = NIT / U;
  static_assert(NR * U == NIT, "orbit items per thread");
  // item idx of this thread for the load: (local transform, orbit item n)
  auto load_item = [&](int idx, int& tau, int& n) -> bool {
    if constexpr (CL == 1) {
      const int w = threadIdx.x + idx * TPB;
      tau = w >> logQi;
      n = w & (Qi - 1);
      return tau < ntr;
    } else {
      const int per = Qi / CL;
      tau = 0;
      n = (int)cg::this_cluster().block_rank() * per + threadIdx.x + idx * TPB;
      return (int)threadIdx.x + idx * TPB < per;
    }
  };
  if (a.ntrig > 0) {
    // DCT-0 / DST-0 inputs straight into the regions
#pragma unroll 1
    for (int rd = 0; rd < NR; ++rd) {
      int n_[U], tau_[U];
      bool ok_[U];
      DrItem r_[U];
#pragma unroll
      for (int s = 0; s < U; ++s) {
        ok_[s] = load_item(rd * U + s, tau_[s], n_[s]);
        if (ok_[s]) r_[s] = load_fetch_trig(static_cast<const float*>(a.in), a.in2, a.ntrig, logN, tid(tau_[s]), n_[s]);
      }
#pragma unroll
      for (int s = 0; s < U; ++s)
        if (ok_[s]) load_place<V>(rg, logN, tau_[s], n_[s], r_[s]);
    }
  } else {
#pragma unroll 1
    for (int rd = 0; rd < NR; ++rd) {
      int n_[U], tau_[U];
      bool ok_[U];
      Fetched f_[U];
#pragma unroll
      for (int s = 0; s < U; ++s) {
        ok_[s] = load_item(rd * U + s, tau_[s], n_[s]);
        if (ok_[s]) {
          const long long t = tid(tau_[s]);
          f_[s] = a.nreal > 0 ? load_fetch_real(static_cast<const float*>(a.in), logN, t, a.nreal, n_[s])
                  : a.nirdft > 0 ? load_fetch_irdft(static_cast<const float2*>(a.in), logN, t, a.nirdft, n_[s])
                                 : load_fetch(InRef{a.in, a.exp_in, a.dtype}, logN, t, toff(t), n_[s], cj);
        }
      }
#pragma unroll
      for (int s = 0; s < U; ++s)
        if (ok_[s]) load_scatter<V>(rg, logN, tau_[s], n_[s], f_[s]);
    }
  }
  if constexpr (CL == 1) __syncthreads();
  else cg::this_cluster().sync();

  // ---- trees and chain ----
  fused_compute<V, TPB, MAXI, CL, LN>(sm, g, TabConsts{cst}, K, tot, wsum, snap,
                                      CL > 1 ? (int)cg::this_cluster().block_rank() & 1 : 0);

  // ---- store ----
  if constexpr (CL > 1 && LN > 0) {
    // time-first variants: the final chain pair already wrote natural order
    if constexpr (!Var<V>::ot) {
      __syncthreads();
      region_to_natural<V, TPB, LN>(reg_ptr(sm, region_stride(LN)), (int)cg::this_cluster().block_rank() & 1);
    }
    cg::this_cluster().sync();
    const long long t = tid(0);
    store_natural_cluster<TPB, LN>(sm, a, t, toff(t), cj, tot);
    cg::this_cluster().sync();  // keep shared memory alive for the other CTAs' reads
    return;
  }
  if constexpr (CL > 1) cg::this_cluster().sync();
  {
    static_assert(CL == 1 || LN > 0, "the cluster path stores through store_natural_cluster");
    // item idx of this thread: (local transform, harmonic k)
    auto item = [&](int idx, int& tau, int& k) -> bool {
      if constexpr (CL == 1) {
        const int w = threadIdx.x + idx * TPB;
        tau = w >> logQi;
        k = w & (Qi - 1);
        return tau < ntr;
      } else {
        const int per = Qi / CL;
        tau = 0;
        k = (int)cg::this_cluster().block_rank() * per + threadIdx.x + idx * TPB;
        return (int)threadIdx.x + idx * TPB < per;
      }
    };
    // 16-bit: one exponent per transform from its largest component; the
    // maxima go to their own slots after the scan scratch
    int* slot = reinterpret_cast<int*>(snap + snap_floats(g.nreg_cap * half));
    const bool c64 = a.dtype == DT_C64;
    if (!c64) {
      for (int i = threadIdx.x; i < ntr; i += TPB) slot[i] = 0;
      __syncthreads();
#pragma unroll 1
      for (int rd = 0; rd < NR; ++rd) {
        int k_[U], tau_[U];
        bool ok_[U];
        Gathered g_[U];
#pragma unroll
        for (int s = 0; s < U; ++s) {
          ok_[s] = item(rd * U + s, tau_[s], k_[s]);
          if (ok_[s]) g_[s] = store_gather<V>(rg, logN, tau_[s], k_[s]);
        }
#pragma unroll
        for (int s = 0; s < U; ++s)
          if (ok_[s]) atomicMax(slot + tau_[s], __float_as_int(out4_absmax(emit_values<V>(logN, k_[s], g_[s]))));
      }
      __syncthreads();
    }
#pragma unroll 1
    for (int rd = 0; rd < NR; ++rd) {
      int k_[U], tau_[U];
      bool ok_[U];
      Gathered g_[U];
#pragma unroll
      for (int s = 0; s < U; ++s) {
        ok_[s] = item(rd * U + s, tau_[s], k_[s]);
        if (ok_[s]) g_[s] = store_gather<V>(rg, logN, tau_[s], k_[s]);
      }
#pragma unroll
      for (int s = 0; s < U; ++s) {
        if (!ok_[s]) continue;
        const long long t = tid(tau_[s]);
        if (a.ntrig > 0) {
          store_trig<V>(static_cast<float*>(a.out), a.out2, a.ntrig, logN, t, k_[s], g_[s]);
        } else if (a.nirdft > 0) {
          store_irdft<V>(static_cast<float*>(a.out), a.nirdft, logN, t, k_[s], g_[s], cj);
        } else if (a.nreal > 0) {
          store_real<V>(static_cast<float2*>(a.out), logN, t, a.nreal, k_[s], g_[s]);
        } else if (c64) {
          store_emit<V>(static_cast<float2*>(a.out), logN, toff(t), k_[s], g_[s], cj);
        } else {
          const int e = block_exponent(__int_as_float(slot[tau_[s]]));
          store16(static_cast<unsigned*>(a.out), toff(t), emit_values<V>(logN, k_[s], g_[s]), pow2f(-e), cj,
                  a.dtype);
          if (k_[s] == 0) a.exp_out[t] = e;
        }
      }
    }
  }
  if constexpr (CL > 1) cg::this_cluster().sync();  // keep shared memory alive for the other CTAs' reads
}

template <int V, int TPB, int MAXI, int CL, int LN>
__global__ void __launch_bounds__(TPB, ctas_per_sm(TPB)) fused_kernel(const FusedArgs a,
                                                                   const __grid_constant__ SmallConsts K) {
  extern __shared__ __align__(16) float sm[];
  if constexpr (CL == 1) {
    const long long j0 = (long long)blockIdx.x * a.tpc;
    const long long left = a.batch - j0;
    fused_body<V, TPB, MAXI, CL, LN>(a, K, sm, j0, left < a.tpc ? (int)left : a.tpc, a.logN, a.RS, a.tot_off,
                                     a.tlist);
  } else {
    fused_body<V, TPB, MAXI, CL, LN>(a, K, sm, (long long)(blockIdx.x / CL), 1, LN, 0, a.tot_off, a.tlist);
  }
}

// ---------------------------------------------------------------------
// host side: configuration and launch
// ---------------------------------------------------------------------
template <int V, int TPB, int MAXI, int CL, int LN>
cudaError_t launch_cfg(const FusedArgs& a, const SmallConsts& K, long long grid, int smem,
                              cudaStream_t st) {
  auto kern = fused_kernel<V, TPB, MAXI, CL, LN>;
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
    // A call that fills one CTA at most is latency-bound: 512 threads (half
    // the items per thread in every pass), one CTA per SM.  The recurrences
    // keep the 256-thread scan chunking, so the results are those of the
    // 256-thread shape and a transform's bits never depend on its batch.
    if (grid == 1)
      return launch_cfg<V, 2 * SMALL_TPB, SMALL_MAXI / 2, 1, 0>(a, K, grid, c.smem + SMALL_TPB * (int)sizeof(float),
                                                                st);
    return launch_cfg<V, SMALL_TPB, SMALL_MAXI, 1, 0>(a, K, grid, c.smem, st);
  }
  switch (a.logN) {
    case 14: return launch_cfg<V, cluster_tpb(14, Var<V>::ot), cluster_maxi(14, Var<V>::ot), 4, 14>(a, K, a.batch, c.smem, st);
    case 15: return launch_cfg<V, cluster_tpb(15, Var<V>::ot), cluster_maxi(15, Var<V>::ot), 4, 15>(a, K, a.batch, c.smem, st);
    default: return launch_cfg<V, cluster_tpb(16, Var<V>::ot), cluster_maxi(16, Var<V>::ot), 4, 16>(a, K, a.batch, c.smem, st);
  }
}

}  // namespace amqft
