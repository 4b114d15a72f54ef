// Paired-region AM-QFT kernel ("A class of AM-QFT algorithms for power-of-two
// FFT", Pasquini): one complex transform of N = 2^LN (LN = 14..16) per cluster
// of four CTAs, time-first variant 4 (Sect. 6.9: D_n chain, D_k trees, M4
// conversion of Tab. 5-6), persistent over the batch.
//
// The pairing.  D_c (Sect. 3.1) and D_r (Eq. qft_22-23) turn x = a + ib into
// the DCT-0 and DST-0 inputs of a and b.  The DCT of a and the DCT of b run
// exactly the same operations (the same holds for the two DSTs), so they
// travel as one float2 (value of a, value of b) and every butterfly is one
// sm_100+ f32x2 instruction (add / sub / mul .rn.f32x2: two IEEE float32
// operations, so the results are those of the scalar recursion).  The loaded
// pair x(n) +- x(N-n) is already that float2: D_c and D_r together cost one
// f32x2 add and one f32x2 sub per sample pair.
//
// The split.  With Q = N/4 = 2^T, the DCT region holds the dct_ot(N) tree of
// Q values (odd samples) followed by the rest of the D_n chain (Q + 1
// values); the DST region likewise (Q and Q - 1).  Cluster rank r:
//     0: DCT tree 0    1: DCT rest    2: DST tree 0    3: DST rest
// so every CTA holds 2^T float2 in shared memory (one CTA per SM at 2^16).
//
// The schedule inside a CTA (NT = 2^(T-5) threads, 32 float2 each; a warp
// owns one block of 1024 positions):
//   load     HBM -> pairs -> distributed shared memory (all four CTAs).
//   band A   the top T-10 time levels of the trees, CTA-wide: every thread
//            holds a fold orbit (the positions closed under the D_k
//            reflections of those levels) and works in registers.
//   warp     per 1024-block, warp-synchronous: five time levels (fold
//            orbit), the 32-value register leaves (the recursion itself), five
//            frequency levels (each lane holds element lane of the 32 leaves
//            and climbs in registers; the M4 neighbour of the last element of
//            a lane's chunk is read from shared memory: along the A path it
//            is an input value).
//   F-band   the top T-10 frequency levels, CTA-wide, the same way.
//   chain    rest CTAs: the D_n frequency phase (S(k) = E(k) +- O(k)) of the
//            chain levels below N, in place, four outputs per quad.
//   store    the last chain level, D_r^F (Eq. qft_24-25) and D_c^F (Eq.
//            qft_17-21), reading the four CTAs through distributed shared
//            memory, float4 stores to HBM.
// The rest CTAs' trees 1, 2, ... and the chain remainder are handled by the
// same band code with a compile-time "virtual root" rule: at every level the
// last aligned block is not a tree node (it is the chain), and its values are
// left alone.  The last warp's block holds the trees below 1024 values and
// the chain bottom (one lane runs the base cases and the chain up to dct(64)).
//
// Layout: every tree node stores its time data and its spectrum in natural
// order; the children of a node of size L occupy [0, L/2) (A: the e-child of
// D_k) and [L/2, L) (B: the oo child after M_v).  A position p is stored at
// float2 index p + 2 (p >> 5) (two pad slots per 32, so that both a lane-per-
// position and a lane-per-32-run access pattern are free of bank conflicts).
// A band reads all its values, synchronises its threads, then writes.
//
// The device code is written so that it also compiles for the host: the
// stages take the thread index and shared-memory pointers explicitly.
#pragma once

#include <stdint.h>
#include <string.h>

#if defined(__CUDACC__)
#include <cooperative_groups.h>
#include <cuda_runtime.h>
#define PR_HD __host__ __device__ __forceinline__
#else
#define PR_HD inline
#endif

namespace amqft {
namespace pr {

// ---------------------------------------------------------------------
// f32x2 arithmetic (round to nearest, never contracted)
// ---------------------------------------------------------------------
// The operations are written as PTX with an explicit rounding mode: such an
// instruction is never contracted with a neighbouring multiply into an FMA.
#if defined(__CUDA_ARCH__)
#define AMQFT_F32X2(OP, r, a, b)                                                                \
  asm("{\n\t.reg .b64 u, v, w;\n\tmov.b64 u, {%2, %3};\n\tmov.b64 v, {%4, %5};\n\t" OP \
      " w, u, v;\n\tmov.b64 {%0, %1}, w;\n\t}"                                              \
      : "=f"(r.x), "=f"(r.y)                                                                   \
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y))
#endif

PR_HD float2 add2(float2 a, float2 b) {
#if defined(__CUDA_ARCH__)
  float2 r;
  AMQFT_F32X2("add.rn.f32x2", r, a, b);
  return r;
#else
  return make_float2(a.x + b.x, a.y + b.y);
#endif
}

PR_HD float2 sub2(float2 a, float2 b) {
#if defined(__CUDA_ARCH__)
  float2 r;
  AMQFT_F32X2("sub.rn.f32x2", r, a, b);
  return r;
#else
  return make_float2(a.x - b.x, a.y - b.y);
#endif
}

// Product a * c, rounded once.  ptxas contracts an f32x2 multiply into the
// f32x2 add that consumes it even when both carry .rn, so the product is
// formed as fma(a, c, nz) with nz = -0.0 passed in at run time (a * c + (-0)
// is the rounded product, signed zeros included): an FMA with an unknown
// addend cannot be fused into anything else.
PR_HD float2 mul2(float2 a, float c, float nz) {
#if defined(__CUDA_ARCH__)
  float2 r;
  asm("{\n\t.reg .b64 u, v, z, w;\n\tmov.b64 u, {%2, %3};\n\tmov.b64 v, {%4, %4};\n\t"
      "mov.b64 z, {%5, %5};\n\tfma.rn.f32x2 w, u, v, z;\n\tmov.b64 {%0, %1}, w;\n\t}"
      : "=f"(r.x), "=f"(r.y)
      : "f"(a.x), "f"(a.y), "f"(c), "f"(nz));
  return r;
#else
  (void)nz;
  return make_float2(a.x * c, a.y * c);
#endif
}

// physical float2 index of region position p (two pad slots per 32)
PR_HD constexpr int phys(int p) { return p + ((p >> 5) << 1); }

// D_k time phase of one pair (Tab. 4) and the M4 scaling of its oo value
// (Tab. 5): DCT context A = u + w, B = (u - w) c; DST context A = u - w,
// B = (u + w) c, with c = 1 / (2 cos(2 pi (2i+1) / 4L)) for the pair
// (i, L-1-i) of a node of L values.
template <int CX>
PR_HD void bfly(float2 u, float2 w, float c, float nz, float2& A, float2& B) {
  if constexpr (CX == 0) {
    A = add2(u, w);
    B = mul2(sub2(u, w), c, nz);
  } else {
    A = sub2(u, w);
    B = mul2(add2(u, w), c, nz);
  }
}

// Constants of the leaf levels (node sizes 2..32), from the plan's table:
// node size L holds its L/2 constants at [L/2 - 2, L - 2).
struct LeafConsts {
  float c[30];
  float cos_pi4;  // node size 2 (the oo(8) base case, Sect. 7.1)
  float nz;       // -0.0, the addend of every product (see mul2)
};

// ---------------------------------------------------------------------
// register recursion: dct_ot(4L) (CX 0) / dst_ot(4L) (CX 1) on L values,
// time values in natural order in, spectrum in natural order out
// ---------------------------------------------------------------------
template <int L, int CX>
PR_HD void ot2(float2 (&x)[L], const LeafConsts& K) {
  if constexpr (L >= 2) {
    constexpr int H = L / 2;
    float2 a[H], b[H];
#pragma unroll
    for (int i = 0; i < H; ++i) bfly<CX>(x[i], x[L - 1 - i], L == 2 ? K.cos_pi4 : K.c[H - 2 + i], K.nz, a[i], b[i]);
    ot2<H, CX>(a, K);
    ot2<H, CX>(b, K);
    // M4 frequency phase: DCT o[j] = B[j] + B[j+1], o[H-1] = B[H-1];
    // DST o[0] = B[0], o[j] = B[j-1] + B[j]; then D_k^F interleaves.
    if constexpr (CX == 0) {
#pragma unroll
      for (int j = 0; j < H; ++j) {
        x[2 * j] = a[j];
        x[2 * j + 1] = (j + 1 < H) ? add2(b[j], b[j + 1]) : b[j];
      }
    } else {
#pragma unroll
      for (int j = 0; j < H; ++j) {
        x[2 * j] = (j > 0) ? add2(b[j - 1], b[j]) : b[j];
        x[2 * j + 1] = a[j];
      }
    }
  }
}

// ---------------------------------------------------------------------
// vector access of R consecutive positions p .. p+R-1 (p a multiple of R,
// R <= 32): one run inside a 32-group, contiguous in shared memory
// ---------------------------------------------------------------------
template <int R>
PR_HD void ld_run(const float2* __restrict__ sm, int p, float2* v) {
  const float2* s = sm + phys(p);
  if constexpr (R == 1) {
    v[0] = s[0];
  } else {
#pragma unroll
    for (int e = 0; e < R; e += 2) {
      const float4 q = *reinterpret_cast<const float4*>(s + e);
      v[e] = make_float2(q.x, q.y);
      v[e + 1] = make_float2(q.z, q.w);
    }
  }
}

template <int R>
PR_HD void st_run(float2* __restrict__ sm, int p, const float2* v) {
  float2* s = sm + phys(p);
  if constexpr (R == 1) {
    s[0] = v[0];
  } else {
#pragma unroll
    for (int e = 0; e < R; e += 2) *reinterpret_cast<float4*>(s + e) = make_float4(v[e].x, v[e].y, v[e + 1].x, v[e + 1].y);
  }
}

// ---------------------------------------------------------------------
// fold band: S time levels of the D_k trees below one band root of 2^M
// positions.  Thread b of 2^(M-S-RHO) holds the 32 labels (f, h, e):
//   position f 2^B0 + (h ? 2^B0 - 1 - (b R0 + e) : b R0 + e),  B0 = M - S + 1,
// f < 2^(S-1), h in {0,1}, e < R0 = 2^RHO: the orbit of its positions under
// the reflections i <-> L-1-i of every level from 2^M down to 2^B0.
// VIRT: the band root is not a tree node and at every level the last aligned
// node is not one either (it is the D_n chain): those values are left alone.
// After the band, label (f, h, e) is element b R0 + e of sub-node 2f + h
// (children of size 2^(B0-1)).
// ---------------------------------------------------------------------
template <int M, int S, int RHO>
struct Fold {
  static constexpr int B0 = M - S + 1, R0 = 1 << RHO, NF = 1 << (S - 1), NV = NF * 2 * R0;
  static constexpr int NTH = 1 << (B0 - 1 - RHO);
  PR_HD static constexpr int idx(int f, int h, int e) { return (f * 2 + h) * R0 + e; }
};

// does the last sub-node of size 2^B0 (f = NF-1) take part (not for VIRT)
template <bool VIRT, int NF>
PR_HD constexpr bool fold_f_used(int f) {
  return !(VIRT && f == NF - 1);
}

template <int M, int S, int RHO, bool VIRT>
PR_HD void fold_read(const float2* __restrict__ sm, int root, int b, float2 (&x)[Fold<M, S, RHO>::NV]) {
  using G = Fold<M, S, RHO>;
  constexpr int U = 1 << G::B0;
#pragma unroll
  for (int f = 0; f < G::NF; ++f) {
    if (!fold_f_used<VIRT, G::NF>(f)) continue;
    float2 v[G::R0];
    ld_run<G::R0>(sm, root + f * U + b * G::R0, v);
#pragma unroll
    for (int e = 0; e < G::R0; ++e) x[G::idx(f, 0, e)] = v[e];
    ld_run<G::R0>(sm, root + f * U + U - (b + 1) * G::R0, v);
#pragma unroll
    for (int e = 0; e < G::R0; ++e) x[G::idx(f, 1, e)] = v[G::R0 - 1 - e];
  }
}

// one level m of the fold band (compile-time recursion over the levels)
template <int M, int S, int RHO, int CX, bool VIRT, int m>
PR_HD void fold_level(float2 (&x)[Fold<M, S, RHO>::NV], const float* __restrict__ cst, int b, float nz) {
  using G = Fold<M, S, RHO>;
  constexpr int FB = m - G::B0;      // f bits local to a node of size 2^m
  constexpr int NN = 1 << (M - m);   // nodes of size 2^m under the band root
  constexpr int L = 1 << m;
  constexpr int U = 1 << G::B0;
  // constants of node size L at cst[L/2 - 32 + i] (the table starts at L = 64)
  const float* c0 = cst + (L / 2 - 32) + b * G::R0;
  const float* c1 = cst + (L / 2 - 32) + (U - 1) - b * G::R0;
  float2 y[G::NV];
#pragma unroll
  for (int q = 0; q < G::NV; ++q) y[q] = x[q];
#pragma unroll
  for (int f = 0; f < G::NF; ++f) {
    const int nid = f >> FB;
    if (VIRT && nid == NN - 1) continue;
    if constexpr (FB >= 1) {
      const int fl = f & ((1 << FB) - 1);
      if (fl >= (1 << (FB - 1))) continue;
      const int fh = (f & ~((1 << FB) - 1)) | ((1 << FB) - 1 - fl);
#pragma unroll
      for (int h = 0; h < 2; ++h) {
#pragma unroll
        for (int e = 0; e < G::R0; ++e) {
          const float c = h == 0 ? c0[fl * U + e] : c1[fl * U - e];
          float2 A, B;
          bfly<CX>(x[G::idx(f, h, e)], x[G::idx(fh, 1 - h, e)], c, nz, A, B);
          y[G::idx(f, h, e)] = A;
          y[G::idx(f + (1 << (FB - 1)), h, e)] = B;
        }
      }
    } else {
#pragma unroll
      for (int e = 0; e < G::R0; ++e) {
        float2 A, B;
        bfly<CX>(x[G::idx(f, 0, e)], x[G::idx(f, 1, e)], c0[e], nz, A, B);
        y[G::idx(f, 0, e)] = A;
        y[G::idx(f, 1, e)] = B;
      }
    }
  }
#pragma unroll
  for (int q = 0; q < G::NV; ++q) x[q] = y[q];
  if constexpr (m > G::B0) fold_level<M, S, RHO, CX, VIRT, m - 1>(x, cst, b, nz);
}

template <int M, int S, int RHO, int CX, bool VIRT>
PR_HD void fold_compute(float2 (&x)[Fold<M, S, RHO>::NV], const float* __restrict__ cst, int b, float nz) {
  if constexpr (VIRT) {
    if constexpr (M - 1 >= Fold<M, S, RHO>::B0) fold_level<M, S, RHO, CX, VIRT, M - 1>(x, cst, b, nz);
  } else {
    fold_level<M, S, RHO, CX, VIRT, M>(x, cst, b, nz);
  }
}

template <int M, int S, int RHO, bool VIRT>
PR_HD void fold_write(float2* __restrict__ sm, int root, int b, const float2 (&x)[Fold<M, S, RHO>::NV]) {
  using G = Fold<M, S, RHO>;
  constexpr int HU = 1 << (G::B0 - 1);
#pragma unroll
  for (int f = 0; f < G::NF; ++f) {
    if (!fold_f_used<VIRT, G::NF>(f)) continue;
#pragma unroll
    for (int h = 0; h < 2; ++h) st_run<G::R0>(sm, root + (2 * f + h) * HU + b * G::R0, &x[G::idx(f, h, 0)]);
  }
}

// ---------------------------------------------------------------------
// frequency band: S frequency levels above G = 2^S sibling nodes of 2^M0
// positions.  Thread c of NC = 2^(M0-RHO) holds chunk c (R0 = 2^RHO values)
// of every sibling; a level turns chunk c of children A = 2g and B = 2g+1 into
// chunk c (twice the size) of their parent:
//   DCT: P[2i] = A[i], P[2i+1] = B[i] + B[i+1]   (B[L/2] absent)
//   DST: P[2i] = B[i-1] + B[i], P[2i+1] = A[i]   (B[-1] absent)
// (M4 frequency phase and D_k^F, Tab. 4-5).  The neighbour outside the chunk
// is the first (DCT) / last (DST) element of the next / previous thread's
// chunk of B; B's even (DCT) / odd (DST) elements are its A child's, so that
// value is an input of the band: input node (2g+1) 2^(j-1), element
// (c+1) R0 (DCT) or c R0 - 1 (DST).
// VIRT: at every level the last node is not formed (chain); the first child
// of each such node is a finished tree root and is written out.
// ---------------------------------------------------------------------
template <int M0, int S, int RHO>
struct Freq {
  static constexpr int G = 1 << S, R0 = 1 << RHO, NV = G * R0, NC = 1 << (M0 - RHO);
};


// node gp of level j is formed (VIRT: all but the last)
template <bool VIRT, int G, int j>
PR_HD constexpr bool freq_formed(int gp) {
  return VIRT ? gp < (G >> j) - 1 : true;
}

// inputs: chunk c of every sibling (VIRT: not the last two; the next to last
// is a finished tree root, the last the chain)
template <int M0, int S, int RHO, bool VIRT>
PR_HD void freq_read(const float2* __restrict__ sm, int base, int c, float2 (&v)[Freq<M0, S, RHO>::NV]) {
  using F = Freq<M0, S, RHO>;
#pragma unroll
  for (int g = 0; g < F::G; ++g)
    if (!VIRT || g < F::G - 2) ld_run<F::R0>(sm, base + (g << M0) + c * F::R0, &v[g * F::R0]);
}

// v holds, at level j, chunk c (R0 2^j values) of node g of that level in
// slots [g R0 2^j, (g+1) R0 2^j): a node always occupies its descendants'
// slots, so a level rewrites the slots of its formed nodes in place, and a
// tree root finished below a node that is not formed (VIRT) stays put.
template <int M0, int S, int RHO, int CX, bool VIRT, int j>
PR_HD void freq_level(float2 (&v)[Freq<M0, S, RHO>::NV], const float2* __restrict__ sm, int base, int el,
                      bool has) {
  using F = Freq<M0, S, RHO>;
  constexpr int Rc = F::R0 << (j - 1);
#pragma unroll
  for (int gp = 0; gp < (F::G >> j); ++gp) {
    if (!freq_formed<VIRT, F::G, j>(gp)) continue;
    float2 h = make_float2(0.f, 0.f);
    if (has) h = sm[phys(base + (((2 * gp + 1) << (j - 1)) << M0) + el)];
    float2 P[2 * Rc];
    const int a0 = (2 * gp) * Rc, b0 = (2 * gp + 1) * Rc;
    if constexpr (CX == 0) {
#pragma unroll
      for (int i = 0; i < Rc; ++i) {
        P[2 * i] = v[a0 + i];
        if (i + 1 < Rc) P[2 * i + 1] = add2(v[b0 + i], v[b0 + i + 1]);
        else P[2 * i + 1] = has ? add2(v[b0 + i], h) : v[b0 + i];
      }
    } else {
#pragma unroll
      for (int i = 0; i < Rc; ++i) {
        if (i > 0) P[2 * i] = add2(v[b0 + i - 1], v[b0 + i]);
        else P[2 * i] = has ? add2(h, v[b0]) : v[b0];
        P[2 * i + 1] = v[a0 + i];
      }
    }
#pragma unroll
    for (int i = 0; i < 2 * Rc; ++i) v[a0 + i] = P[i];
  }
  if constexpr (j < S) freq_level<M0, S, RHO, CX, VIRT, j + 1>(v, sm, base, el, has);
}

// the levels of the band; the neighbour of a chunk's edge (its halo) is read
// here, before the band's writes
template <int M0, int S, int RHO, int CX, bool VIRT>
PR_HD void freq_compute(float2 (&v)[Freq<M0, S, RHO>::NV], const float2* __restrict__ sm, int base, int c) {
  using F = Freq<M0, S, RHO>;
  const bool has = CX == 0 ? (c + 1 < F::NC) : (c > 0);
  const int el = CX == 0 ? (c + 1) * F::R0 : c * F::R0 - 1;
  freq_level<M0, S, RHO, CX, VIRT, 1>(v, sm, base, el, has);
}

// outputs: chunk c of the band top (VIRT: of the tree roots finished at
// levels 1 .. S-1, node (G >> l) - 2 of level l)
template <int M0, int S, int RHO, bool VIRT, int l>
PR_HD void freq_write_roots(float2* __restrict__ sm, int base, int c, const float2 (&v)[Freq<M0, S, RHO>::NV]) {
  using F = Freq<M0, S, RHO>;
  constexpr int Rl = F::R0 << l, gp = (F::G >> l) - 2;
  st_run<Rl>(sm, base + (gp << (M0 + l)) + c * Rl, &v[gp * Rl]);
  if constexpr (l + 1 < S) freq_write_roots<M0, S, RHO, VIRT, l + 1>(sm, base, c, v);
}

template <int M0, int S, int RHO, bool VIRT>
PR_HD void freq_write(float2* __restrict__ sm, int base, int c, const float2 (&v)[Freq<M0, S, RHO>::NV]) {
  using F = Freq<M0, S, RHO>;
  if constexpr (!VIRT) {
    st_run<F::NV>(sm, base + c * F::NV, v);
  } else if constexpr (S >= 2) {
    freq_write_roots<M0, S, RHO, VIRT, 1>(sm, base, c, v);
  }
}

// ---------------------------------------------------------------------
// chain bottom, one thread: the trees of 16 .. 1 values (DCT) or 16 .. 2
// (DST), the base case dct(2) or dst(4), and the D_n frequency phase up to
// dct(64) / dst(64), on the 33 (DCT) or 31 (DST) positions [992, 1025) of
// the last block.  Chain level of periodisation M (Sect. 6.9):
//   DCT  S(k) = E(k) + O(k), S(M/2-k) = E(k) - O(k) (k < M/4), S(M/4) = E(M/4)
//   DST  S(k) = O(k) + E(k), S(M/2-k) = O(k) - E(k) (0 < k < M/4), S(M/4) = O(M/4)
// with O the dct_ot(M) / dst_ot(M) tree and E = dct(M/2) / dst(M/2).
// ---------------------------------------------------------------------
template <int OFF, int L, int CX, int SZ>
PR_HD void tail_tree(float2 (&t)[SZ], const LeafConsts& K) {
  float2 x[L];
#pragma unroll
  for (int e = 0; e < L; ++e) x[e] = t[OFF + e];
  ot2<L, CX>(x, K);
#pragma unroll
  for (int e = 0; e < L; ++e) t[OFF + e] = x[e];
}

template <int M, int SZ>
PR_HD void tail_chain_dct(float2 (&t)[SZ]) {
  if constexpr (M <= 64) {
    constexpr int P = 32 - M / 2, Q = M / 4;
    float2 s[M / 2 + 1];
#pragma unroll
    for (int k = 0; k < Q; ++k) {
      s[k] = add2(t[P + Q + k], t[P + k]);
      s[M / 2 - k] = sub2(t[P + Q + k], t[P + k]);
    }
    s[Q] = t[P + 2 * Q];
#pragma unroll
    for (int k = 0; k <= M / 2; ++k) t[P + k] = s[k];
    tail_chain_dct<2 * M, SZ>(t);
  }
}

template <int M, int SZ>
PR_HD void tail_chain_dst(float2 (&t)[SZ]) {
  if constexpr (M <= 64) {
    constexpr int P = 32 - M / 2, Q = M / 4;
    float2 s[M / 2 - 1];
#pragma unroll
    for (int k = 1; k < Q; ++k) {
      s[k - 1] = add2(t[P + k - 1], t[P + Q + k - 1]);
      s[M / 2 - k - 1] = sub2(t[P + k - 1], t[P + Q + k - 1]);
    }
    s[Q - 1] = t[P + Q - 1];
#pragma unroll
    for (int k = 0; k < M / 2 - 1; ++k) t[P + k] = s[k];
    tail_chain_dst<2 * M, SZ>(t);
  }
}

// blk: the block's base (float2 index of its position 0)
template <int CX>
PR_HD void run_tail(float2* __restrict__ blk, const LeafConsts& K) {
  constexpr int SZ = CX == 0 ? 33 : 31;
  float2 t[SZ];
#pragma unroll
  for (int e = 0; e < SZ; ++e) t[e] = blk[phys(992 + e)];
  tail_tree<0, 16, CX, SZ>(t, K);
  tail_tree<16, 8, CX, SZ>(t, K);
  tail_tree<24, 4, CX, SZ>(t, K);
  tail_tree<28, 2, CX, SZ>(t, K);
  if constexpr (CX == 0) {
    // dct_ot(4) of one value is a copy; dct(2): S0 = s0 + s1, S1 = s0 - s1
    const float2 a = t[31], b = t[32];
    t[31] = add2(a, b);
    t[32] = sub2(a, b);
    tail_chain_dct<4, SZ>(t);
  } else {
    tail_chain_dst<8, SZ>(t);  // dst(4): S(1) = s(1), a copy
  }
#pragma unroll
  for (int e = 0; e < SZ; ++e) blk[phys(992 + e)] = t[e];
}


// ---------------------------------------------------------------------
// chain levels of a rest CTA.  Level m's item k (H = 2^m) reads E(k), E(H-k)
// (the chain below) and the tree values O(k), O(H-k), and gives S at k,
// 2H-k, H-k, H+k, in place.  Positions: level m's tree at [P, P+H),
// P = 2^T - 2H; harmonic k of a DST spectrum sits one position lower
// (DCT d = 0, DST d = 1).
// ---------------------------------------------------------------------
// one item, in place (any k, including k = 0 and k = H/2)
template <int CX>
PR_HD void chain_item(float2* __restrict__ sm, int P, int H, int k) {
  constexpr int d = CX;
  if (CX == 0 && k == 0) {
    const float2 o = sm[phys(P)], e = sm[phys(P + H)], eH = sm[phys(P + 2 * H)];
    sm[phys(P)] = add2(e, o);
    sm[phys(P + 2 * H)] = sub2(e, o);
    sm[phys(P + H)] = eH;
    return;
  }
  if (k == 0) return;  // DST: S(H) = O(H) stays where it is
  if (2 * k == H) {
    const float2 o = sm[phys(P + k - d)], e = sm[phys(P + H + k - d)];
    sm[phys(P + k - d)] = CX == 0 ? add2(e, o) : add2(o, e);
    sm[phys(P + 2 * H - k - d)] = CX == 0 ? sub2(e, o) : sub2(o, e);
    return;
  }
  const float2 o1 = sm[phys(P + k - d)], e1 = sm[phys(P + H + k - d)];
  const float2 o2 = sm[phys(P + H - k - d)], e2 = sm[phys(P + 2 * H - k - d)];
  sm[phys(P + k - d)] = CX == 0 ? add2(e1, o1) : add2(o1, e1);
  sm[phys(P + 2 * H - k - d)] = CX == 0 ? sub2(e1, o1) : sub2(o1, e1);
  sm[phys(P + H - k - d)] = CX == 0 ? add2(e2, o2) : add2(o2, e2);
  sm[phys(P + H + k - d)] = CX == 0 ? sub2(e2, o2) : sub2(o2, e2);
}

// One chain level m on a group of NTH threads (thread tid), the chain ending at
// position TOP of sm: item k = tid + i NTH, every item's reads issued before
// its writes; item H/2 (and item 0) by thread 0.  The items of a level are
// disjoint, so a level needs no barrier inside.
template <int CX, int m, int NTH, int TOP>
PR_HD void chain_single(float2* __restrict__ sm, int tid) {
  constexpr int H = 1 << m, P = TOP - 2 * H, NI = (H / 2 + NTH - 1) / NTH, d = CX;
  float2 o1[NI], e1[NI], o2[NI], e2[NI];
#pragma unroll
  for (int i = 0; i < NI; ++i) {
    const int k = tid + i * NTH;
    if ((CX == 1 && k == 0) || k >= H / 2) {  // no DST item 0 (its positions would start at P - 1)
      o1[i] = e1[i] = o2[i] = e2[i] = make_float2(0.f, 0.f);
      continue;
    }
    o1[i] = sm[phys(P + k - d)];
    e1[i] = sm[phys(P + H + k - d)];
    o2[i] = sm[phys(P + H - k - d)];
    e2[i] = sm[phys(P + 2 * H - k - d)];
  }
  float2 eH = make_float2(0.f, 0.f);
  if (CX == 0 && tid == 0) eH = sm[phys(P + 2 * H)];
#pragma unroll
  for (int i = 0; i < NI; ++i) {
    const int k = tid + i * NTH;
    if (k >= H / 2) continue;
    if (k == 0) {
      if (CX == 0) {  // S(0) = E(0) + O(0), S(2H) = E(0) - O(0), S(H) = E(H)
        sm[phys(P)] = add2(e1[i], o1[i]);
        sm[phys(P + 2 * H)] = sub2(e1[i], o1[i]);
        sm[phys(P + H)] = eH;
      }  // DST: no item 0; S(H) = O(H) stays in place
      continue;
    }
    sm[phys(P + k - d)] = CX == 0 ? add2(e1[i], o1[i]) : add2(o1[i], e1[i]);
    sm[phys(P + 2 * H - k - d)] = CX == 0 ? sub2(e1[i], o1[i]) : sub2(o1[i], e1[i]);
    sm[phys(P + H - k - d)] = CX == 0 ? add2(e2[i], o2[i]) : add2(o2[i], e2[i]);
    sm[phys(P + H + k - d)] = CX == 0 ? sub2(e2[i], o2[i]) : sub2(o2[i], e2[i]);
  }
  if (tid == 0) chain_item<CX>(sm, P, H, H / 2);
}

// Chain levels m and m+1 in one pass.  Level m's item k (0 < k < H/2)
// gives S at k, 2H-k (the inputs of level m+1's item k) and at H-k, H+k (those
// of item H-k), so the three items form a closed orbit: its eight tree values
// and two chain values are read, and its eight outputs of level m+1 written,
// by one thread, and no other thread touches those positions.  The orbits of
// items 0 and H/2 (which meet the fixed points of the next level) are run by
// thread 0 item by item, in place.
template <int CX, int m, int NTH, int TOP>
PR_HD void chain_pair(float2* __restrict__ sm, int tid) {
  constexpr int H = 1 << m, P = TOP - 2 * H, H2 = 2 * H, P2 = TOP - 2 * H2, d = CX;
  constexpr int NI = (H / 2 + NTH - 1) / NTH;
  // one orbit at a time (its positions are its own, so no order is needed
  // between orbits; this keeps the register footprint at one orbit)
#pragma unroll
  for (int i = 0; i < NI; ++i) {
    const int k = tid + i * NTH;
    if (k == 0 || k >= H / 2) continue;
    const float2 ea = sm[phys(P + H + k - d)];      // E(k)
    const float2 eb = sm[phys(P + 2 * H - k - d)];  // E(H-k)
    const float2 oa = sm[phys(P + k - d)];          // O(k)
    const float2 ob = sm[phys(P + H - k - d)];      // O(H-k)
    const float2 p0 = sm[phys(P2 + k - d)];         // O'(k)
    const float2 p1 = sm[phys(P2 + H2 - k - d)];    // O'(2H-k)
    const float2 p2 = sm[phys(P2 + H - k - d)];     // O'(H-k)
    const float2 p3 = sm[phys(P2 + H + k - d)];     // O'(H+k)
    // level m: DCT S = E +- O, DST S = O +- E
    const float2 sk = CX == 0 ? add2(ea, oa) : add2(oa, ea);   // S(k)
    const float2 s2 = CX == 0 ? sub2(ea, oa) : sub2(oa, ea);   // S(2H-k)
    const float2 sh = CX == 0 ? add2(eb, ob) : add2(ob, eb);   // S(H-k)
    const float2 sp = CX == 0 ? sub2(eb, ob) : sub2(ob, eb);   // S(H+k)
    // level m+1, item k: E'(k) = S(k), E'(2H-k) = S(2H-k)
    sm[phys(P2 + k - d)] = CX == 0 ? add2(sk, p0) : add2(p0, sk);
    sm[phys(P2 + 2 * H2 - k - d)] = CX == 0 ? sub2(sk, p0) : sub2(p0, sk);
    sm[phys(P2 + H2 - k - d)] = CX == 0 ? add2(s2, p1) : add2(p1, s2);
    sm[phys(P2 + H2 + k - d)] = CX == 0 ? sub2(s2, p1) : sub2(p1, s2);
    // level m+1, item H-k: E'(H-k) = S(H-k), E'(H+k) = S(H+k)
    sm[phys(P2 + H - k - d)] = CX == 0 ? add2(sh, p2) : add2(p2, sh);
    sm[phys(P2 + 2 * H2 - H + k - d)] = CX == 0 ? sub2(sh, p2) : sub2(p2, sh);
    sm[phys(P2 + H + k - d)] = CX == 0 ? add2(sp, p3) : add2(p3, sp);
    sm[phys(P2 + H2 + H - k - d)] = CX == 0 ? sub2(sp, p3) : sub2(p3, sp);
  }
  if (tid == 0) {
    chain_item<CX>(sm, P, H, 0);
    chain_item<CX>(sm, P, H, H / 2);
    chain_item<CX>(sm, P2, H2, 0);
    chain_item<CX>(sm, P2, H2, H);
    chain_item<CX>(sm, P2, H2, H / 2);
  }
}

// ---------------------------------------------------------------------
// stage entry points (thread index explicit; the caller synchronises
// between the phases marked "sync")
// ---------------------------------------------------------------------
// Band A over the CTA's 2^T positions: fold band M = T, S = T - 10 levels,
// chunk 2^(15-T); VIRT for the rest CTAs (trees 1, 2, ... below a root that
// is not a node).
template <int T>
struct BandA {
  static constexpr int M = T, S = T - 10, RHO = 15 - T;
  using G = Fold<M, S, RHO>;
};

// leaf ln of the block (VIRT: lane 31 runs the chain bottom instead)
template <int CX, bool VIRT>
PR_HD void block_leaf(float2* __restrict__ blk, int ln, const LeafConsts& K) {
  if (VIRT && ln == 31) {
    run_tail<CX>(blk, K);
    return;
  }
  float2 x[32];
  ld_run<32>(blk, 32 * ln, x);
  ot2<32, CX>(x, K);
  st_run<32>(blk, 32 * ln, x);
}

// chain levels m .. T-5 inside the last block (the 32 lanes of its warp), two
// levels a pass
template <int T, int CX, int m, class Ctx>
PR_HD void block_chain(Ctx& cx, float2* __restrict__ blk, int ln) {
  if constexpr (m + 1 <= T - 5) {
    cx.sync_warp();
    chain_pair<CX, m, 32, 1024>(blk, ln);
    block_chain<T, CX, m + 2>(cx, blk, ln);
  } else if constexpr (m == T - 5) {
    cx.sync_warp();
    chain_single<CX, m, 32, 1024>(blk, ln);
  }
}

// ---------------------------------------------------------------------
// one transform, orchestrated.  Ctx supplies the thread (tid, rank), the
// synchronisation (sync_warp, sync_cta, sync_cluster) and the HBM accesses
// (ldg2, ldg4, stg2, stg4: streaming, the data is touched once).
// ---------------------------------------------------------------------
template <int T, int CX, bool VIRT, class Ctx>
PR_HD void block_stage(Ctx& cx, float2* __restrict__ blk, int ln, const float* __restrict__ cst,
                       const LeafConsts& K) {
  float2 x[32];
  fold_read<10, 5, 0, VIRT>(blk, 0, ln, x);
  fold_compute<10, 5, 0, CX, VIRT>(x, cst, ln, K.nz);
  cx.sync_warp();
  fold_write<10, 5, 0, VIRT>(blk, 0, ln, x);
  cx.sync_warp();
  block_leaf<CX, VIRT>(blk, ln, K);
  cx.sync_warp();
  freq_read<5, 5, 0, VIRT>(blk, 0, ln, x);
  freq_compute<5, 5, 0, CX, VIRT>(x, blk, 0, ln);
  cx.sync_warp();
  freq_write<5, 5, 0, VIRT>(blk, 0, ln, x);
  if constexpr (VIRT) {
    // chain levels of the trees of 32 .. 2^(T-5) values inside the block
    block_chain<T, CX, 5>(cx, blk, ln);
  }
}

// The CTA's region between the load and the store.  TOP: the tree dct_ot(N)
// (CX 0) or dst_ot(N) (CX 1) of 2^T values; otherwise the rest of the D_n
// chain: trees of 2^(T-1), 2^(T-2), ... values, the base case, and the chain
// levels up to dct(N/2) / dst(N/2).
template <int T, int CX, bool TOP, class Ctx>
PR_HD void cta_transform(Ctx& cx, float2* __restrict__ reg, const float* __restrict__ cst, const LeafConsts& K) {
  using A = BandA<T>;
  constexpr int NW = 1 << (T - 10);
  constexpr bool VA = !TOP;
  const int tid = cx.tid, ln = tid & 31, w = tid >> 5;
  {
    float2 x[32];
    fold_read<A::M, A::S, A::RHO, VA>(reg, 0, tid, x);
    fold_compute<A::M, A::S, A::RHO, CX, VA>(x, cst, tid, K.nz);
    cx.sync_cta();
    fold_write<A::M, A::S, A::RHO, VA>(reg, 0, tid, x);
  }
  cx.sync_cta();
  float2* blk = reg + phys(w << 10);
  if (TOP || w < NW - 1) block_stage<T, CX, false>(cx, blk, ln, cst, K);
  else block_stage<T, CX, true>(cx, blk, ln, cst, K);
  cx.sync_cta();
  {
    float2 v[32];
    freq_read<10, A::S, A::RHO, VA>(reg, 0, tid, v);
    freq_compute<10, A::S, A::RHO, CX, VA>(v, reg, 0, tid);
    cx.sync_cta();
    freq_write<10, A::S, A::RHO, VA>(reg, 0, tid, v);
  }
  if constexpr (!TOP) {
    // chain levels of the trees of 2^(T-4) .. 2^(T-1) values
    cx.sync_cta();
    chain_pair<CX, T - 4, (1 << (T - 5)), (1 << T)>(reg, tid);
    cx.sync_cta();
    chain_pair<CX, T - 2, (1 << (T - 5)), (1 << T)>(reg, tid);
  }
}

// region position (in its CTA) of DCT/DST sample n of an even, 0 < n < N/2:
// the rest CTA's trees hold n = 2^t (2i + 1) at Q - 2Q/2^t + i (Sect. 6.9).
template <int LN>
PR_HD int rest_pos(int n) {
  constexpr int Q = 1 << (LN - 2);
#if defined(__CUDA_ARCH__)
  const int t = __ffs(n) - 1;
#else
  const int t = __builtin_ctz((unsigned)n);
#endif
  return Q - ((2 * Q) >> t) + (n >> (t + 1));
}

// Load: D_c and D_r of samples [r N/8, (r+1) N/8) and their mirrors.  The
// pair value of sample n is (a(n) + a(N-n), b(n) + b(N-n)) for the DCT
// regions and the differences for the DST regions (Eq. qft_22-23); dc(0) =
// x(0), dc(N/2) = x(N/2).  INV: the input is conjugated (conj F conj).
// Four rounds of HBM reads per thread: a round's reads are issued together
// (load_fetch) and scattered into the four regions afterwards (load_scatter),
// and the first round of the next transform is in flight across the cluster
// barrier that ends the current one.
// The HBM form of the batch: complex64 (H = false) or 16-bit pairs (H =
// true: bfloat16, binary16 or int16, real part in the low half, the values
// times 2^exp, one exponent per transform; the Ctx converts, the arithmetic
// stays float32 and the scalings are exact powers of two).
struct Store16 {
  const int* exp_in;  // input exponents (NULL: all 0)
  int* exp_out;       // output exponents
  int dtype;          // 1 bf16, 2 fp16, 3 int16
};

// Which transforms the cluster runs: t = 0 .. batch-1 at element t * N, or
// (a ragged batch) list entries t < min(*count, batch) at element
// offset[list[t]], each 16-byte aligned, the count written by an earlier
// kernel of the stream.
struct TList {
  const int* list;
  const long long* offset;
  const int* count;
};

PR_HD float f32_from_bits(uint32_t u) {
#if defined(__CUDA_ARCH__)
  return __uint_as_float(u);
#else
  float f;
  memcpy(&f, &u, 4);
  return f;
#endif
}

// 2^e, exact (e clamped to the normal range)
PR_HD float pow2_exact(int e) {
  e = e < -126 ? -126 : (e > 127 ? 127 : e);
  return f32_from_bits((uint32_t)(127 + e) << 23);
}

// exponent of a 16-bit output transform: its largest component magnitude m
// lands in [2^13, 2^14) once scaled by 2^-e; 0 for m = 0 or not finite;
// clamped to [-100, 100]
PR_HD int block_exp(float m) {
  if (!(m > 0.f) || !(m <= 3.402823466e38f)) return 0;
  uint32_t u;
#if defined(__CUDA_ARCH__)
  u = __float_as_uint(m);
#else
  memcpy(&u, &m, 4);
#endif
  int e = (int)((u >> 23) & 0xff) - 127;  // floor(log2 m) for normal m
  if (e < -126) e = -126;
  e -= 13;
  return e < -100 ? -100 : (e > 100 ? 100 : e);
}

template <bool H>
struct LoadWords {  // one item: x(n), x(n+1) and x(N-n), x(N-n-1)
  float4 a;
  float2 m0, m1;
};
template <>
struct LoadWords<true> {
  uint2 a;
  unsigned m0, m1;
};

template <int LN, bool H = false>
struct LoadRound {
  static constexpr int NT = 1 << (LN - 7), NI = (1 << (LN - 4)) / NT / 4;  // items per round
  LoadWords<H> w[NI];
};

template <int LN, bool H, class Ctx>
PR_HD void load_fetch(Ctx& cx, const void* xin, int r, int round, LoadRound<LN, H>& R) {
  constexpr int N = 1 << LN, NT = LoadRound<LN, H>::NT, NI = LoadRound<LN, H>::NI;
#pragma unroll
  for (int i = 0; i < NI; ++i) {
    const int n = r * (N / 8) + 2 * (cx.tid + (round * NI + i) * NT);
    if constexpr (H) {
      const unsigned* x = static_cast<const unsigned*>(xin);
      R.w[i].a = cx.ldg16x2(x + n);
      R.w[i].m0 = n > 0 ? cx.ldg16(x + (N - n)) : 0u;
      R.w[i].m1 = cx.ldg16(x + (N - n - 1));
    } else {
      const float2* x = static_cast<const float2*>(xin);
      R.w[i].a = cx.ldg4(x + n);
      R.w[i].m0 = n > 0 ? cx.ldg2(x + (N - n)) : make_float2(0.f, 0.f);
      R.w[i].m1 = cx.ldg2(x + (N - n - 1));
    }
  }
}

// sample as float2, conjugated for the inverse (16-bit: times 2^exp_in)
template <bool INV, class Ctx>
PR_HD float2 sample(Ctx& cx, float2 v, float, int) {
  return make_float2(v.x, INV ? v.y * -1.f : v.y);
}
template <bool INV, class Ctx>
PR_HD float2 sample(Ctx& cx, unsigned u, float s, int dt) {
  const float2 v = cx.unpack16(u, dt);
  return make_float2(v.x * s, v.y * (INV ? s * -1.f : s));
}

template <int LN, bool INV, bool H, class Ctx>
PR_HD void load_scatter(Ctx& cx, int r, int round, const LoadRound<LN, H>& R, float s, int dt) {
  constexpr int N = 1 << LN, Q = N / 4, NT = LoadRound<LN, H>::NT, NI = LoadRound<LN, H>::NI;
#pragma unroll
  for (int i = 0; i < NI; ++i) {
    const int n = r * (N / 8) + 2 * (cx.tid + (round * NI + i) * NT);
    float2 xn, xo;
    if constexpr (H) {
      xn = sample<INV>(cx, R.w[i].a.x, s, dt);
      xo = sample<INV>(cx, R.w[i].a.y, s, dt);
    } else {
      xn = sample<INV>(cx, make_float2(R.w[i].a.x, R.w[i].a.y), s, dt);
      xo = sample<INV>(cx, make_float2(R.w[i].a.z, R.w[i].a.w), s, dt);
    }
    const float2 y0 = sample<INV>(cx, R.w[i].m0, s, dt), y1 = sample<INV>(cx, R.w[i].m1, s, dt);
    // odd sample n+1: tree 0, position n/2
    cx.dst2(0, phys(n >> 1), add2(xo, y1));
    cx.dst2(2, phys(n >> 1), sub2(xo, y1));
    if (n == 0) {
      cx.dst2(1, phys(Q - 1), xn);  // dc(0) = x(0), the first sample of dct(2)
    } else {
      const int q = rest_pos<LN>(n);
      cx.dst2(1, phys(q), add2(xn, y0));
      cx.dst2(3, phys(q), sub2(xn, y0));
    }
  }
}

// dc(N/2) = x(N/2), the second sample of dct(2) (rank 3, thread 0)
template <int LN, bool INV, bool H, class Ctx>
PR_HD void load_middle(Ctx& cx, const void* xin, int r, float s, int dt) {
  constexpr int N = 1 << LN, Q = N / 4;
  if (r == 3 && cx.tid == 0) {
    float2 h;
    if constexpr (H) h = sample<INV>(cx, cx.ldg16(static_cast<const unsigned*>(xin) + N / 2), s, dt);
    else h = sample<INV>(cx, cx.ldg2(static_cast<const float2*>(xin) + N / 2), s, dt);
    cx.dst2(1, phys(Q), h);
  }
}

// Store: the last chain level (M = N) from the four CTAs, D_r^F (R = DCT - i
// DST, Eq. qft_24-25) and D_c^F (Eq. qft_17-21):
//   X(k) = (C1 + S2, C2 - S1),  X(N-k) = (C1 - S2, C2 + S1)  at k and N/2 - k,
// harmonics k in [r Q/4, (r+1) Q/4), a pair (k, k+1) per thread and step,
// and X(N/4), X(3N/4) (rank 0).  Every read is one 16-byte run of
// distributed shared memory, consecutive lanes reading consecutive runs: the
// DST spectra hold harmonic k at position k - 1, so a thread reads positions
// k, k+1 (harmonics k+1, k+2) and takes harmonic k from the previous lane.
// INV: the output is conjugated.
// Shared memory of one CTA: the region (phys(2^T) + 1 float2, rounded up to
// an even count) and the constants of node sizes 64 .. 2^T (tree 0) or
// 64 .. 2^(T-1) (rest) as floats.
template <int T>
PR_HD constexpr int region_f2() {
  return ((phys(1 << T) + 1) + 1) & ~1;
}
template <int T>
PR_HD constexpr int smem_bytes() {
  return region_f2<T>() * 8 + ((1 << T) - 32) * 4;
}

// The outputs of this CTA's harmonics in the order of the store, handed to
// put2(i, X(i), X(i+1)) and put1(i, X(i)).
template <int LN, bool INV, class Ctx, class P2, class P1>
PR_HD void store_walk(Ctx& cx, int r, P2&& put2, P1&& put1) {
  constexpr int N = 1 << LN, Q = N / 4, NT = 1 << (LN - 7), NALL = (Q / 8) / NT;
  constexpr int NI = NALL < 2 ? NALL : 2;  // pairs in flight per thread (register budget)
  const int tid = cx.tid;
  const float cj = INV ? -1.f : 1.f;
#pragma unroll 1
  for (int g = 0; g < NALL / NI; ++g) {
    float2 oc[NI][2], ec[NI][2], os[NI][3], es[NI][3];
#pragma unroll
    for (int i = 0; i < NI; ++i) {
      const int k = r * (Q / 4) + 2 * (tid + (g * NI + i) * NT);
      cx.dld4(0, phys(k), oc[i]);
      cx.dld4(1, phys(k), ec[i]);
      cx.dld4(2, phys(k), &os[i][1]);  // harmonics k+1, k+2
      cx.dld4(3, phys(k), &es[i][1]);
    }
#pragma unroll
    for (int i = 0; i < NI; ++i) {
      const int k = r * (Q / 4) + 2 * (tid + (g * NI + i) * NT);
      float2 po = cx.shfl_up(os[i][2], 1), pe = cx.shfl_up(es[i][2], 1);
      if ((tid & 31) == 0) {  // harmonic k (position k - 1) of lane 0
        po = k > 0 ? cx.dld2(2, phys(k - 1)) : make_float2(0.f, 0.f);
        pe = k > 0 ? cx.dld2(3, phys(k - 1)) : make_float2(0.f, 0.f);
      }
      os[i][0] = po;
      es[i][0] = pe;
    }
#pragma unroll
    for (int i = 0; i < NI; ++i) {
      const int k = r * (Q / 4) + 2 * (tid + (g * NI + i) * NT);
      float2 X0[2], XM[2], XH[2], XN[2];  // X(k+j), X(N-k-j), X(N/2-k-j), X(N/2+k+j)
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        const float2 ck = add2(ec[i][j], oc[i][j]), cm = sub2(ec[i][j], oc[i][j]);
        const float2 sk = add2(os[i][j], es[i][j]), sm = sub2(os[i][j], es[i][j]);
        X0[j] = make_float2(ck.x + sk.y, (ck.y - sk.x) * cj);
        XM[j] = make_float2(ck.x - sk.y, (ck.y + sk.x) * cj);
        XH[j] = make_float2(cm.x + sm.y, (cm.y - sm.x) * cj);
        XN[j] = make_float2(cm.x - sm.y, (cm.y + sm.x) * cj);
      }
      if (k == 0) {  // X(0) = C(0), X(N/2) = C(N/2): the DST has no harmonic 0
        const float2 ck = add2(ec[i][0], oc[i][0]), cm = sub2(ec[i][0], oc[i][0]);
        X0[0] = make_float2(ck.x, ck.y * cj);
        XN[0] = make_float2(cm.x, cm.y * cj);
      }
      put2(k, X0[0], X0[1]);
      put2(N / 2 + k, XN[0], XN[1]);
      if (k > 0) {
        put1(N - k, XM[0]);
        put1(N / 2 - k, XH[0]);
      }
      put1(N - k - 1, XM[1]);
      put1(N / 2 - k - 1, XH[1]);
    }
  }
  if (r == 0 && tid == 0) {
    const float2 cq = cx.dld2(1, phys(Q)), sq = cx.dld2(2, phys(Q - 1));  // C(N/4) = E(N/4), S(N/4) = O(N/4)
    put1(Q, make_float2(cq.x + sq.y, (cq.y - sq.x) * cj));
    put1(3 * Q, make_float2(cq.x - sq.y, (cq.y + sq.x) * cj));
  }
}

PR_HD float absmax2(float m, float2 v) {
  const float a = v.x < 0.f ? -v.x : v.x, b = v.y < 0.f ? -v.y : v.y;
  m = a > m ? a : m;  // a NaN never wins (as fmaxf)
  return b > m ? b : m;
}

// Store: the last chain level (M = N) from the four CTAs, D_r^F (R = DCT - i
// DST, Eq. qft_24-25) and D_c^F (Eq. qft_17-21):
//   X(k) = (C1 + S2, C2 - S1),  X(N-k) = (C1 - S2, C2 + S1)  at k and N/2 - k,
// harmonics k in [r Q/4, (r+1) Q/4), a pair (k, k+1) per thread and step,
// and X(N/4), X(3N/4) (rank 0).  Every read is one 16-byte run of
// distributed shared memory, consecutive lanes reading consecutive runs: the
// DST spectra hold harmonic k at position k - 1, so a thread reads positions
// k, k+1 (harmonics k+1, k+2) and takes harmonic k from the previous lane.
// INV: the output is conjugated.  16-bit (H): a first walk takes the largest
// component magnitude (the CTA's through the Ctx, the cluster's through the
// spare word of each region), which fixes the transform's exponent; the
// second walk scales by 2^-exp and rounds.
template <int LN, bool INV, bool H, class Ctx>
PR_HD void store_stage(Ctx& cx, void* xo, int r, const Store16* io, long long t) {
  if constexpr (!H) {
    float2* z = static_cast<float2*>(xo);
    store_walk<LN, INV>(
        cx, r, [&](int i, float2 a, float2 b) { cx.stg4(z + i, make_float4(a.x, a.y, b.x, b.y)); },
        [&](int i, float2 a) { cx.stg2(z + i, a); });
  } else {
    constexpr int SPARE = region_f2<LN - 2>() - 1;
    float m = 0.f;
    store_walk<LN, INV>(
        cx, r, [&](int, float2 a, float2 b) { m = absmax2(absmax2(m, a), b); },
        [&](int, float2 a) { m = absmax2(m, a); });
    m = cx.max_cta(m);
    if (cx.tid == 0) cx.dst2(r, SPARE, make_float2(m, 0.f));
    cx.sync_cluster();
    float M = 0.f;
    for (int q = 0; q < 4; ++q) {
      const float v = cx.dld2(q, SPARE).x;
      M = v > M ? v : M;
    }
    const int e = block_exp(M);
    const float sc = pow2_exact(-e);
    const int dt = io->dtype;
    if (r == 0 && cx.tid == 0) io->exp_out[t] = e;
    unsigned* z = static_cast<unsigned*>(xo);
    store_walk<LN, INV>(
        cx, r,
        [&](int i, float2 a, float2 b) {
          cx.stg16x2(z + i, make_uint2(cx.pack16(a.x * sc, a.y * sc, dt), cx.pack16(b.x * sc, b.y * sc, dt)));
        },
        [&](int i, float2 a) { cx.stg16(z + i, cx.pack16(a.x * sc, a.y * sc, dt)); });
  }
}

// The cluster's work: transforms cid, cid + ncl, ... of the batch (batch below
// 2^31; the dispatch checks it).
// reg: this CTA's region; Ctx reaches CTA q's region with dst2 / dld2 / dld4
// (float2 index into the region: distributed shared memory for the others).
template <int LN, bool INV, bool H, class Ctx>
PR_HD void paired_body(Ctx& cx, const void* in, void* out, const Store16* io, int batch, int cid, int ncl,
                       float2* reg, float* __restrict__ cst, const float* __restrict__ ctab, const LeafConsts& K,
                       const TList& tl = TList{nullptr, nullptr, nullptr}) {
  constexpr int T = LN - 2, NT = 1 << (T - 5);
  constexpr long long N = 1LL << LN;
  constexpr int ES = H ? 4 : 8;  // bytes per element in HBM
  const int r = cx.rank, tid = cx.tid;
  const int ncst = (r & 1) == 0 ? (1 << T) - 32 : (1 << (T - 1)) - 32;
  if (ctab)  // else the kernel has evaluated them on the fly
    for (int i = tid; i < ncst; i += NT) cst[i] = ctab[30 + i];
  const int dt = H ? io->dtype : 0;
  if (tl.count && *tl.count < batch) batch = *tl.count;
  auto at = [&](const void* base, long long t) {
    const long long e = tl.list ? tl.offset[tl.list[t]] : t * N;
    return static_cast<const void*>(static_cast<const char*>(base) + e * ES);
  };
  // 2^exp_in of transform t (16-bit input)
  auto scale = [&](long long t) { return H && io->exp_in ? pow2_exact(io->exp_in[t]) : 1.f; };
  LoadRound<LN, H> R;
  if (cid < batch) load_fetch<LN, H>(cx, at(in, cid), r, 0, R);
  for (int t = cid; t < batch; t += ncl) {
    const void* xin = at(in, t);
    const float s = scale(t);
    cx.sync_cluster();  // the previous store has read every region
    load_scatter<LN, INV, H>(cx, r, 0, R, s, dt);
#pragma unroll
    for (int rd = 1; rd < 4; ++rd) {
      load_fetch<LN, H>(cx, xin, r, rd, R);
      load_scatter<LN, INV, H>(cx, r, rd, R, s, dt);
    }
    load_middle<LN, INV, H>(cx, xin, r, s, dt);
    cx.sync_cluster();
    switch (r) {
      case 0: cta_transform<T, 0, true>(cx, reg, cst, K); break;
      case 1: cta_transform<T, 0, false>(cx, reg, cst, K); break;
      case 2: cta_transform<T, 1, true>(cx, reg, cst, K); break;
      default: cta_transform<T, 1, false>(cx, reg, cst, K); break;
    }
    cx.sync_cluster();
    store_stage<LN, INV, H>(cx, const_cast<void*>(at(out, t)), r, io, t);
    // the next transform's first reads fly across the barrier at the loop top
    if (t + ncl < batch) load_fetch<LN, H>(cx, at(in, t + ncl), r, 0, R);
  }
  cx.sync_cluster();  // keep the regions alive for the other CTAs' reads
}

}  // namespace pr
}  // namespace amqft
