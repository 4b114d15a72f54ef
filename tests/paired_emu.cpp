// Host emulation of the paired-region kernel (amqft_paired.cuh), for the CPU
// test suite.  The kernel's stages are written against a context that
// supplies the thread index, synchronisation and memory accesses; here every
// GPU thread of one cluster of four CTAs is a std::thread, warp / CTA /
// cluster synchronisation are std::barriers, a warp shuffle goes through a
// per-warp slot array, and distributed shared memory is four host arrays.
// Built with AddressSanitizer by the test, so an index outside a region, a
// constant table or a buffer is reported on the CPU.
//
// usage: paired_emu <inverse 0|1> <batch> <in.bin> <out.bin> [<dtype> <exp_in.bin> <exp_out.bin>]
// (N = 2^PAIRED_LN; dtype 1 bf16, 2 fp16, 3 int16 storage, else complex64)
#include <cuda_runtime.h>

#include <barrier>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
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
  uint2 ldg16x2(const unsigned* p) { return make_uint2(p[0], p[1]); }
  unsigned ldg16(const unsigned* p) { return *p; }
  void stg16x2(unsigned* p, uint2 v) {
    p[0] = v.x;
    p[1] = v.y;
  }
  void stg16(unsigned* p, unsigned v) { *p = v; }
  // 16-bit conversions (round to nearest even), as the device's
  static float bits(uint32_t u) {
    float f;
    memcpy(&f, &u, 4);
    return f;
  }
  static uint32_t ubits(float f) {
    uint32_t u;
    memcpy(&u, &f, 4);
    return u;
  }
  static unsigned to16(float v, int dt) {
    if (dt == 1) {
      uint32_t u = ubits(v);
      if ((u & 0x7fffffffu) > 0x7f800000u) return 0x7fc0u;
      u += 0x7fffu + ((u >> 16) & 1u);
      return u >> 16;
    }
    if (dt == 3) {
      float q = std::nearbyint(v);
      q = q < -32768.f ? -32768.f : (q > 32767.f ? 32767.f : q);
      return (unsigned)(unsigned short)(short)q;
    }
    const uint32_t x = ubits(v), sign = (x >> 16) & 0x8000u, ax = x & 0x7fffffffu;
    if (ax >= 0x7f800000u) return sign | (ax > 0x7f800000u ? 0x7e00u : 0x7c00u);
    if (ax >= 0x477ff000u) return sign | 0x7c00u;  // rounds to infinity
    if (ax < 0x38800000u) return sign | (uint32_t)std::nearbyint(bits(ax) * 16777216.0f);  // subnormal
    uint32_t h = ((((ax >> 23) - 127 + 15) << 10) | ((ax & 0x7fffffu) >> 13));
    const uint32_t rem = ax & 0x1fffu;
    if (rem > 0x1000u || (rem == 0x1000u && (h & 1u))) ++h;
    return sign | h;
  }
  static float from16(unsigned h, int dt) {
    if (dt == 1) return bits(h << 16);
    if (dt == 3) return (float)(short)(unsigned short)h;
    const uint32_t sign = (h & 0x8000u) << 16, e = (h >> 10) & 31u, m = h & 1023u;
    if (e == 0) return bits(sign) + (sign ? -1.f : 1.f) * (float)m * (1.0f / 16777216.0f);
    if (e == 31) return bits(sign | 0x7f800000u | (m << 13));
    return bits(sign | ((e - 15 + 127) << 23) | (m << 13));
  }
  float2 unpack16(unsigned u, int dt) { return make_float2(from16(u & 0xffffu, dt), from16(u >> 16, dt)); }
  unsigned pack16(float re, float im, int dt) { return to16(re, dt) | (to16(im, dt) << 16); }
  float* cred;  // this CTA's max slots
  float max_cta(float m) {
    cred[tid] = m;
    bcta->arrive_and_wait();
    float r = 0.f;
    for (int i = 0; i < nth; ++i) r = cred[i] > r ? cred[i] : r;
    bcta->arrive_and_wait();
    return r;
  }
  int nth;
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

template <int LN, bool INV, bool H>
void run(const void* in, void* out, const Store16* io, long long batch, const TList& tl) {
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
  std::vector<float> red(4 * NT);
  std::vector<std::thread> th;
  for (int q = 0; q < 4; ++q)
    for (int t = 0; t < NT; ++t)
      th.emplace_back([&, q, t]() {
        HostCtx cx{t, q, &bcl, bcta[q].get(), bwarp[q * (NT / 32) + t / 32].get(), &slots[(q * NT + t) & ~31], regs};
        cx.cred = &red[q * NT];
        cx.nth = NT;
        float* cst = reinterpret_cast<float*>(regs[q] + region_f2<T>());
        paired_body<LN, INV, H>(cx, in, out, io, (int)batch, 0, 1, regs[q], cst, ctab.data(), K, tl);
      });
  for (auto& x : th) x.join();
}

}  // namespace

int main(int argc, char** argv) {
  // paired_emu <inverse> <batch> <in.bin> <out.bin> [dtype exp_in.bin exp_out.bin]
  // a negative batch -b: the b transforms through a transform list, in
  // reverse order, the count read as the kernel reads it
  if (argc != 5 && argc != 8) return 2;
  const int inv = atoi(argv[1]);
  long long batch = atoll(argv[2]);
  const bool listed = batch < 0;
  if (listed) batch = -batch;
  const long long N = 1LL << PAIRED_LN;
  const int dt = argc == 8 ? atoi(argv[5]) : 0;
  const size_t es = dt ? 4 : 8;
  std::vector<unsigned char> in(N * batch * es), out(N * batch * es, 0xff);
  FILE* f = fopen(argv[3], "rb");
  if (!f || fread(in.data(), 1, in.size(), f) != in.size()) return 3;
  fclose(f);
  std::vector<int> ein(batch, 0), eout(batch, 0);
  if (dt) {
    f = fopen(argv[6], "rb");
    if (!f || fread(ein.data(), sizeof(int), ein.size(), f) != ein.size()) return 3;
    fclose(f);
  }
  const Store16 io{ein.data(), eout.data(), dt};
  std::vector<int> list(batch);
  std::vector<long long> offs(batch);
  for (long long t = 0; t < batch; ++t) {
    list[t] = (int)(batch - 1 - t);
    offs[t] = t * N;
  }
  const int count = (int)batch;
  const TList tl = listed ? TList{list.data(), offs.data(), &count} : TList{nullptr, nullptr, nullptr};
  const long long cap = listed ? batch + 3 : batch;  // a list's capacity may exceed its count
  if (dt) {
    if (inv) run<PAIRED_LN, true, true>(in.data(), out.data(), &io, cap, tl);
    else run<PAIRED_LN, false, true>(in.data(), out.data(), &io, cap, tl);
  } else {
    if (inv) run<PAIRED_LN, true, false>(in.data(), out.data(), nullptr, cap, tl);
    else run<PAIRED_LN, false, false>(in.data(), out.data(), nullptr, cap, tl);
  }
  f = fopen(argv[4], "wb");
  if (!f || fwrite(out.data(), 1, out.size(), f) != out.size()) return 4;
  fclose(f);
  if (dt) {
    f = fopen(argv[7], "wb");
    if (!f || fwrite(eout.data(), sizeof(int), eout.size(), f) != eout.size()) return 4;
    fclose(f);
  }
  return 0;
}
