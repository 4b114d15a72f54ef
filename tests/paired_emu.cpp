// Host emulation of the paired-region kernel (amqft_paired.cuh), for the CPU
// test suite.  The kernel's stages are written against a context that
// supplies the thread index, synchronisation and memory accesses; here every
// GPU thread of one cluster of four CTAs is a std::thread, warp / CTA /
// cluster synchronisation are std::barriers, a warp shuffle goes through a
// per-warp slot array, and distributed shared memory is four host arrays.
// Built with AddressSanitizer by the test, so an index outside a region, a
// constant table or a buffer is reported on the CPU.
//
// usage: paired_emu <inverse 0|1> <batch> <in.bin> <out.bin>   (N = 2^PAIRED_LN)
#include <cuda_runtime.h>

#include <barrier>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <memory>
#include <thread>
#include <vector>

#include "amqft_paired.cuh"

using namespace amqft::pr;

namespace {

struct HostCtx {
  int tid, rank;
  std::barrier<>* bcl;
  std::barrier<>* bcta;
  std::barrier<>* bwarp;
  float2* wslot;  // the 32 shuffle slots of this thread's warp
  float2** regs;  // the four regions of the cluster
  void sync_cluster() { bcl->arrive_and_wait(); }
  void sync_cta() { bcta->arrive_and_wait(); }
  void sync_warp() { bwarp->arrive_and_wait(); }
  float4 ldg4(const float2* p) { return *reinterpret_cast<const float4*>(p); }
  float2 ldg2(const float2* p) { return *p; }
  void stg4(float2* p, float4 v) { *reinterpret_cast<float4*>(p) = v; }
  void stg2(float2* p, float2 v) { *p = v; }
  float2 shfl_up(float2 v, int d) {
    const int ln = tid & 31;
    wslot[ln] = v;
    bwarp->arrive_and_wait();
    const float2 r = ln >= d ? wslot[ln - d] : v;
    bwarp->arrive_and_wait();
    return r;
  }
  void dst2(int q, int i, float2 v) { regs[q][i] = v; }
  float2 dld2(int q, int i) { return regs[q][i]; }
  void dld4(int q, int i, float2* v) {
    v[0] = regs[q][i];
    v[1] = regs[q][i + 1];
  }
};

// trig constants of variant 4 (1 / (2 cos(2 pi (2j+1) / M))), from the exact
// turn fraction folded to [0, pi/4], in long double, rounded once: node size
// L = M/4 holds its L/2 constants at [L/2 - 2, L - 2)
long double cos_turn(long long num, long long den) {
  const long double two_pi = 6.283185307179586476925286766559005768394L;
  long long r = num % den;
  if (r < 0) r += den;
  if (2 * r > den) r = den - r;
  long double sign = 1.0L;
  if (4 * r > den) {
    r = den / 2 - r;
    sign = -1.0L;
  }
  if (8 * r > den) return sign * sinl(two_pi * (long double)(den / 4 - r) / (long double)den);
  return sign * cosl(two_pi * (long double)r / (long double)den);
}

template <int LN, bool INV>
void run(const float2* in, float2* out, long long batch) {
  constexpr int T = LN - 2, NT = 1 << (T - 5), N = 1 << LN;
  std::vector<float> ctab(N / 4 - 2);
  for (long long M = 16; M <= N; M *= 2)
    for (long long j = 0; j < M / 8; ++j) ctab[M / 8 - 2 + j] = (float)(1.0L / (2.0L * cos_turn(2 * j + 1, M)));
  LeafConsts K;
  for (int i = 0; i < 30; ++i) K.c[i] = ctab[i];
  K.cos_pi4 = (float)cos_turn(1, 8);
  K.nz = -0.0f;
  // exactly the shared memory a CTA is launched with
  std::vector<std::vector<float2>> smem(4, std::vector<float2>(smem_bytes<T>() / sizeof(float2)));
  float2* regs[4];
  for (int q = 0; q < 4; ++q) regs[q] = smem[q].data();
  std::barrier<> bcl(4 * NT);
  std::vector<std::unique_ptr<std::barrier<>>> bcta, bwarp;
  for (int q = 0; q < 4; ++q) bcta.emplace_back(new std::barrier<>(NT));
  for (int w = 0; w < 4 * NT / 32; ++w) bwarp.emplace_back(new std::barrier<>(32));
  std::vector<float2> slots(4 * NT);
  std::vector<std::thread> th;
  for (int q = 0; q < 4; ++q)
    for (int t = 0; t < NT; ++t)
      th.emplace_back([&, q, t]() {
        HostCtx cx{t, q, &bcl, bcta[q].get(), bwarp[q * (NT / 32) + t / 32].get(), &slots[(q * NT + t) & ~31], regs};
        float* cst = reinterpret_cast<float*>(regs[q] + region_f2<T>());
        paired_body<LN, INV>(cx, in, out, batch, 0, 1, regs[q], cst, ctab.data(), K);
      });
  for (auto& x : th) x.join();
}

}  // namespace

int main(int argc, char** argv) {
  if (argc != 5) return 2;
  const int inv = atoi(argv[1]);
  const long long batch = atoll(argv[2]);
  const long long N = 1LL << PAIRED_LN;
  std::vector<float2> in(N * batch), out(N * batch, make_float2(NAN, NAN));
  FILE* f = fopen(argv[3], "rb");
  if (!f || fread(in.data(), sizeof(float2), in.size(), f) != in.size()) return 3;
  fclose(f);
  if (inv) run<PAIRED_LN, true>(in.data(), out.data(), batch);
  else run<PAIRED_LN, false>(in.data(), out.data(), batch);
  f = fopen(argv[4], "wb");
  if (!f || fwrite(out.data(), sizeof(float2), out.size(), f) != out.size()) return 4;
  fclose(f);
  return 0;
}
