// C ABI of the AM-QFT library (include/amqft.h): plans, constant tables,
// argument checks and kernel dispatch.  No compute happens on the host
// except the trig-constant table of a plan.
#include <math.h>
#include <stdarg.h>
#include <atomic>
#include <new>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <string>
#include <thread>
#include <vector>

#include "amqft.h"
#include "amqft_ragged_impl.cuh"
#include "amqft_internal.h"

namespace amqft {

FusedConfig fused_config(int logN, int variant) {
  FusedConfig c;
  const int N = 1 << logN, half = N >> 1;
  c.RS = region_stride(logN);
  if (logN <= 13) {
    c.cluster = 1;
    c.threads = SMALL_TPB;
    // a CTA holds 16384 region values: 256 threads x 64 values, two CTAs per SM
    c.per_cta = small_tpc(logN);
    c.nreg = 4 * c.per_cta;
  } else {
    c.cluster = 4;
    c.per_cta = 1;
    c.nreg = 1;
    // 2^14, 2^15: 256 threads (two CTAs per SM); 2^16: 1024 threads, 32 values each
    c.threads = cluster_tpb(logN, variant_ot(variant));
  }
  c.tot_off = ((c.nreg * c.RS + 31) / 32) * 32;
  // scan scratch (threads + 32), snapshot, one 16-bit exponent slot per
  // transform, and the band levels' constants
  c.smem = (c.tot_off + c.threads + 32 + snap_floats(c.nreg * half) + c.per_cta + band_consts(logN)) *
           (int)sizeof(float);
  return c;
}

static cudaError_t fused_launch(int variant, const FusedArgs& a, const SmallConsts& K, const FusedConfig& c,
                                cudaStream_t st) {
  switch (variant) {
    case 1: return launch_variant_1(a, K, c, st);
    case 2: return launch_variant_2(a, K, c, st);
    case 3: return launch_variant_3(a, K, c, st);
    case 4: return launch_variant_4(a, K, c, st);
    case 5: return launch_variant_5(a, K, c, st);
    case 6: return launch_variant_6(a, K, c, st);
    case 7: return launch_variant_7(a, K, c, st);
    default: return launch_variant_8(a, K, c, st);
  }
}

static cudaError_t ragged_launch(int variant, const FusedArgs& a, const SmallConsts& K, const RaggedArgs& r,
                                 const RaggedLaunch& L, cudaStream_t st, long long* nl) {
  switch (variant) {
    case 1: return ragged_variant_1(a, K, r, L, st, nl);
    case 2: return ragged_variant_2(a, K, r, L, st, nl);
    case 3: return ragged_variant_3(a, K, r, L, st, nl);
    case 4: return ragged_variant_4(a, K, r, L, st, nl);
    case 5: return ragged_variant_5(a, K, r, L, st, nl);
    case 6: return ragged_variant_6(a, K, r, L, st, nl);
    case 7: return ragged_variant_7(a, K, r, L, st, nl);
    default: return ragged_variant_8(a, K, r, L, st, nl);
  }
}

// Bucket pass of a ragged batch: transform ids into one list per log2 N.
// ubase > 0: a transform of 2^14..2^16 whose data is not 16-byte aligned
// (offset + par odd, par = the parity of the base pointers in 8-byte words)
// goes to class ubase + (log2 N - 14) instead of its length's
__global__ void ragged_bucket_kernel(const unsigned char* __restrict__ log2n, const long long* __restrict__ off,
                                     long long count, int maxlog, long long max_points, int* cnt, int* list,
                                     long long cap, int* skipped, const float2* __restrict__ in,
                                     float2* __restrict__ out, int ubase, int par) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < count;
       i += (long long)gridDim.x * blockDim.x) {
    const int c = log2n[i];
    if (c > maxlog) {
      atomicAdd(skipped, 1);
      continue;
    }
    if (c == 0) {  // N = 1: the DFT (and its inverse) is the identity
      out[off[i]] = in[off[i]];
      continue;
    }
    const int cls = ubase > 0 && c >= 14 && c <= 16 && ((off[i] + par) & 1) ? ubase + (c - 14) : c;
    const int pos = atomicAdd(cnt + cls, 1);
    // multi-pass lengths: the workspace holds max_points >> c transforms
    const long long capc = c > AMQFT_LOG2N_FUSED_MAX && (max_points >> c) < cap ? (max_points >> c) : cap;
    if (pos >= capc) {
      atomicAdd(skipped, 1);
      continue;
    }
    list[cls * cap + pos] = (int)i;
  }
}


cudaError_t multipass_dispatch(int variant, const MpArgs& a, float* W0, float* W1, const SmallConsts& K,
                               cudaStream_t st, long long* nl) {
  switch (variant) {
    case 1: return multipass_variant_1(a, W0, W1, K, st, nl);
    case 2: return multipass_variant_2(a, W0, W1, K, st, nl);
    case 3: return multipass_variant_3(a, W0, W1, K, st, nl);
    case 4: return multipass_variant_4(a, W0, W1, K, st, nl);
    case 5: return multipass_variant_5(a, W0, W1, K, st, nl);
    case 6: return multipass_variant_6(a, W0, W1, K, st, nl);
    case 7: return multipass_variant_7(a, W0, W1, K, st, nl);
    case 8: return multipass_variant_8(a, W0, W1, K, st, nl);
    default: return cudaErrorInvalidValue;
  }
}

// N = 1: the DFT is the identity (conjugated twice for the inverse).
__global__ void copy1_kernel(const float2* __restrict__ in, float2* __restrict__ out, long long batch) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < batch) out[i] = in[i];
}

// N = 1, real input: R(0) = x(0).
__global__ void copy1_real_kernel(const float* __restrict__ in, float2* __restrict__ out, long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = make_float2(in[i], 0.f);
}

// N = 1 with 16-bit storage: the value (conjugated for the inverse) gets the
// exponent of its largest component, like every other length.
__global__ void copy1_16_kernel(const unsigned* __restrict__ in, unsigned* __restrict__ out,
                                const int* __restrict__ exp_in, int* __restrict__ exp_out, long long batch,
                                int dtype) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < batch) {
    const float s = exp_in ? pow2f(exp_in[i]) : 1.f;
    const float2 v = unpack16(in[i], dtype);
    const float re = v.x * s, im = v.y * s;
    const int e = block_exponent(fmaxf(fabsf(re), fabsf(im)));
    const float sc = pow2f(-e);
    out[i] = pack16(re * sc, im * sc, dtype);
    exp_out[i] = e;
  }
}

}  // namespace amqft

using namespace amqft;

// ---------------------------------------------------------------------
// trig constants (Sect. 7.1), computed on the host in long double from the
// exact turn fraction and rounded once to float
// ---------------------------------------------------------------------
static const long double kTwoPi = 6.283185307179586476925286766559005768394L;

// cos(2*pi*num/den), den a power of two >= 8: the angle is folded into
// [0, pi/4] with exact integer arithmetic before the libm call.
static long double cos_frac(long long num, long long den) {
  long long r = num % den;
  if (r < 0) r += den;
  if (2 * r > den) r = den - r;                  // [0, 1/2] turn
  long double sign = 1.0L;
  if (4 * r > den) { r = den / 2 - r; sign = -1.0L; }   // [0, 1/4] turn
  if (8 * r > den) return sign * sinl(kTwoPi * (long double)(den / 4 - r) / (long double)den);
  return sign * cosl(kTwoPi * (long double)r / (long double)den);
}

static long double sin_frac(long long num, long long den) { return cos_frac(den / 4 - num, den); }

// Constant of variant v at angle 2*pi*(2j+1)/M: 2cos (1,3), 1/(2cos) (2,4),
// 2sin (5,7), 1/(2sin) (6,8).
static float variant_const(int v, long long M, long long j) {
  const long long p = 2 * j + 1;
  long double c;
  switch (v) {
    case 1: case 3: c = 2.0L * cos_frac(p, M); break;
    case 2: case 4: c = 1.0L / (2.0L * cos_frac(p, M)); break;
    case 5: case 7: c = 2.0L * sin_frac(p, M); break;
    default: c = 1.0L / (2.0L * sin_frac(p, M)); break;
  }
  return (float)c;
}

// The level-major table: periodisation M = 16..N holds its M/8 constants at
// [M/8 - 2, M/4 - 2).  Long tables (N/4 - 2 = 2^26 - 2 entries at 2^28; long
// double is a software format on some hosts) are filled by several host
// threads, each entry by the same scalar function.
static void fill_range(float* h, long long lo, long long hi, int variant) {
  for (long long i = lo; i < hi; ++i) {
    long long M = 16;
    while (M / 4 - 2 <= i) M *= 2;
    h[i] = variant_const(variant, M, i - (M / 8 - 2));
  }
}

static void fill_table(float* h, long long n, int variant) {
  unsigned nt = std::thread::hardware_concurrency();
  if (nt < 1) nt = 1;
  if (nt > 64) nt = 64;
  if (n < (1LL << 16) || nt == 1) {
    fill_range(h, 0, n, variant);
    return;
  }
  std::vector<std::thread> th;
  const long long per = (n + nt - 1) / nt;
  for (unsigned t = 0; t < nt; ++t) {
    const long long lo = (long long)t * per, hi = lo + per < n ? lo + per : n;
    if (lo >= hi) break;
    try {
      th.emplace_back(fill_range, h, lo, hi, variant);
    } catch (...) {
      fill_range(h, lo, hi, variant);  // no thread: this one does the range
    }
  }
  for (auto& x : th) x.join();
}

// ---------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------
static thread_local std::string t_err;

static int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  t_err = buf;
  return code;
}

static int cuda_fail(cudaError_t e, const char* what) {
  return fail(AMQFT_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

struct amqft_plan_s {
  int log2n;
  int variant;
  int64_t batch;
  int dtype;
  int device;
  float* d_ctab;
  int const_mode;  // AMQFT_CONST_TABLE or AMQFT_CONST_FLY
  SmallConsts small;
  FusedConfig cfg;
  // multi-pass path: two ping-pong workspaces of chunk * 4 regions
  float* d_work;
  long long chunk;
  long long RSg;
  // ragged plans (amqft_plan_ragged)
  int ragged;
  int num_sms;
  long long max_count, max_points;
  int* d_rcnt;     // [0, 32) transforms per log2 N, [32] schedule counter, [33] skipped
  int* d_rlist;    // (log2n + 1) lists of max_count transform ids
  float* d_rwork;  // multi-pass workspace, shared by the lengths above 2^16 in turn
  int knob[4];     // schedule, order, small CTAs per SM, cluster grid multiplier
  // host-memory execution (amqft_exec_host): two in and two out staging
  // buffers of h_chunk transforms, copy-in / transform / copy-out streams
  long long h_chunk;
  void* h_buf[4];
  cudaStream_t h_st[3];
  cudaEvent_t h_ev[8];
  // kernels launched by the exec calls on this plan (amqft_plan_launches)
  std::atomic<long long> launches{0};
};

// workspace budget of one plan (both ping-pong buffers)
static const long long kWorkspaceBytes = 2LL << 30;

namespace amqft {

// The table the kernels read; NULL makes them evaluate the band levels'
// constants on the fly.
static const float* kernel_ctab(amqft_plan_t p) {
  return p->const_mode == AMQFT_CONST_FLY ? nullptr : p->d_ctab;
}

int plan_view(amqft_plan_t p, PlanView* v) {
  if (!p || !v) return fail(AMQFT_ERR_ARG, "plan is NULL");
  v->log2n = p->log2n;
  v->variant = p->variant;
  v->dtype = p->dtype;
  v->device = p->device;
  v->ctab = kernel_ctab(p);
  v->small = &p->small;
  return AMQFT_OK;
}

void add_launches(amqft_plan_t p, long long n) {
  if (p) p->launches += n;
}

int set_error(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  t_err = buf;
  return code;
}

void clear_error() { t_err.clear(); }

}  // namespace amqft

extern "C" {

const char* amqft_last_error(void) { return t_err.c_str(); }

const char* amqft_version(void) {
  return "amqft 0.2 (sm_103a; fused single-pass to 2^16, multi-pass to 2^24; float32 arithmetic; complex64, bf16 and "
         "fp16 storage)";
}

int amqft_plan(amqft_plan_t* out, int log2n, int variant, int64_t batch, int dtype) {
  t_err.clear();
  if (!out) return fail(AMQFT_ERR_ARG, "amqft_plan: out is NULL");
  *out = nullptr;
  if (log2n < 0 || log2n > AMQFT_LOG2N_MAX)
    return fail(AMQFT_ERR_N, "amqft_plan: log2n=%d outside [0, %d]", log2n, AMQFT_LOG2N_MAX);
  if (variant < 1 || variant > 8) return fail(AMQFT_ERR_VARIANT, "amqft_plan: variant=%d not in 1..8", variant);
  if (dtype != AMQFT_C64 && dtype != AMQFT_CBF16 && dtype != AMQFT_CF16 && dtype != AMQFT_CI16)
    return fail(AMQFT_ERR_DTYPE, "amqft_plan: dtype=%d is not AMQFT_C64, AMQFT_CBF16, AMQFT_CF16 or AMQFT_CI16",
                dtype);
  if (batch < 0) return fail(AMQFT_ERR_ARG, "amqft_plan: batch=%lld < 0", (long long)batch);
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "amqft_plan: cudaGetDevice");
  cudaDeviceProp prop;
  e = cudaGetDeviceProperties(&prop, dev);
  if (e != cudaSuccess) return cuda_fail(e, "amqft_plan: cudaGetDeviceProperties");
  if (!(prop.major == 10 && prop.minor == 3))
    return fail(AMQFT_ERR_DEVICE, "amqft_plan: device %d is sm_%d%d, this library is built for sm_103a", dev,
                prop.major, prop.minor);
  amqft_plan_s* p = new (std::nothrow) amqft_plan_s();
  if (!p) return fail(AMQFT_ERR_NOMEM, "amqft_plan: host allocation failed");
  p->log2n = log2n;
  p->variant = variant;
  p->batch = batch;
  p->dtype = dtype;
  p->device = dev;
  p->d_ctab = nullptr;
  p->const_mode = AMQFT_CONST_TABLE;
  p->d_work = nullptr;
  p->chunk = 0;
  p->RSg = 0;
  p->ragged = 0;
  p->num_sms = prop.multiProcessorCount;
  p->max_count = p->max_points = 0;
  p->d_rcnt = nullptr;
  p->d_rlist = nullptr;
  p->d_rwork = nullptr;
  p->knob[0] = 1;
  p->knob[1] = 0;
  p->knob[2] = 2;
  p->knob[3] = 1;
  p->h_chunk = 0;
  memset(p->h_buf, 0, sizeof p->h_buf);
  memset(p->h_st, 0, sizeof p->h_st);
  memset(p->h_ev, 0, sizeof p->h_ev);
  // level-major table: periodisation M = 16..N holds M/8 constants at [M/8-2, M/4-2)
  const long long N = 1LL << log2n;
  const long long ntab = N >= 16 ? N / 4 - 2 : 0;
  const long long nhost = ntab > (long long)(LEAF - 2) ? ntab : (long long)(LEAF - 2);
  float* h = (float*)calloc((size_t)nhost, sizeof(float));
  if (!h) { delete p; return fail(AMQFT_ERR_NOMEM, "amqft_plan: host allocation failed"); }
  fill_table(h, nhost, variant);
  for (int i = 0; i < LEAF - 2; ++i) p->small.c[i] = h[i];
  p->small.cos_pi4 = (float)cos_frac(1, 8);
  if (ntab > 0) {
    e = cudaMalloc(&p->d_ctab, (size_t)ntab * sizeof(float));
    if (e != cudaSuccess) { free(h); delete p; return cuda_fail(e, "amqft_plan: cudaMalloc(constant table)"); }
    e = cudaMemcpy(p->d_ctab, h, (size_t)ntab * sizeof(float), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) { free(h); cudaFree(p->d_ctab); delete p; return cuda_fail(e, "amqft_plan: cudaMemcpy"); }
  }
  free(h);
  if (log2n >= 1 && log2n <= AMQFT_LOG2N_FUSED_MAX) p->cfg = fused_config(log2n, variant);
  else memset(&p->cfg, 0, sizeof p->cfg);
  if (log2n > AMQFT_LOG2N_FUSED_MAX && batch > 0) {
    const long long half = N / 2;
    p->RSg = ((half + 2 + 31) / 32) * 32;
    const long long per_t = 2LL * 4 * p->RSg * (long long)sizeof(float);
    long long chunk = kWorkspaceBytes / per_t;
    if (chunk < 1) chunk = 1;
    if (chunk > batch) chunk = batch;
    p->chunk = chunk;
    e = cudaMalloc(&p->d_work, (size_t)(chunk * per_t));
    if (e != cudaSuccess) {
      if (p->d_ctab) cudaFree(p->d_ctab);
      delete p;
      return cuda_fail(e, "amqft_plan: cudaMalloc(workspace)");
    }
  }
  *out = p;
  return AMQFT_OK;
}

// `batch` transforms (at most the plan's batch) from in to out on stream.
static int exec_n(amqft_plan_t p, long long batch, const void* in, void* out, int inverse, const int32_t* exp_in,
                  int32_t* exp_out, void* stream) {
  const bool c64 = p->dtype == AMQFT_C64;
  if (c64 && (exp_in || exp_out)) return fail(AMQFT_ERR_DTYPE, "exponent arrays are only used with 16-bit storage");
  if (batch == 0) return AMQFT_OK;
  if (!in || !out) return fail(AMQFT_ERR_ALIGN, "in or out is NULL");
  const uintptr_t amask = c64 ? 7u : 3u;
  if (((uintptr_t)in | (uintptr_t)out) & amask)
    return fail(AMQFT_ERR_ALIGN, "in/out must be %d-byte aligned", (int)amask + 1);
  if (!c64) {
    if (!exp_out) return fail(AMQFT_ERR_ARG, "16-bit storage needs exp_out (one int32 per transform)");
    if (((uintptr_t)exp_out | (uintptr_t)exp_in) & 3u) return fail(AMQFT_ERR_ALIGN, "exponent arrays must be 4-byte aligned");
  }
  const long long N = 1LL << p->log2n;
  const uintptr_t bytes = (uintptr_t)(N * batch * (c64 ? 8 : 4));
  const uintptr_t a0 = (uintptr_t)in, b0 = (uintptr_t)out;
  // in == out is the in-place transform; any other overlap is rejected
  if (a0 != b0 && a0 < b0 + bytes && b0 < a0 + bytes)
    return fail(AMQFT_ERR_INPLACE, "in and out overlap without being equal");
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e;
  if (p->log2n > AMQFT_LOG2N_FUSED_MAX) {
    const long long per_buf = p->chunk * 4 * p->RSg;
    for (long long t0 = 0; t0 < batch; t0 += p->chunk) {
      MpArgs a = {};
      a.in = in;
      a.out = out;
      a.exp_in = exp_in;
      a.exp_out = exp_out;
      a.dtype = p->dtype;
      a.ctab = kernel_ctab(p);
      a.nt = (batch - t0) < p->chunk ? (batch - t0) : p->chunk;
      a.t0 = t0;
      a.logN = p->log2n;
      a.inverse = inverse;
      a.RSg = p->RSg;
      a.tlist = nullptr;
      a.toff = nullptr;
      a.ntdev = nullptr;
      long long nl = 0;
      e = multipass_dispatch(p->variant, a, p->d_work, p->d_work + per_buf, p->small, st, &nl);
      p->launches += nl;
      if (e != cudaSuccess) return cuda_fail(e, "multi-pass launch");
    }
    return AMQFT_OK;
  }
  if (p->log2n == 0) {
    const unsigned grid = (unsigned)((batch + 255) / 256);
    if (c64) copy1_kernel<<<grid, 256, 0, st>>>((const float2*)in, (float2*)out, batch);
    else copy1_16_kernel<<<grid, 256, 0, st>>>((const unsigned*)in, (unsigned*)out, exp_in, exp_out, batch,
                                               p->dtype);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "copy kernel launch");
    ++p->launches;
    return AMQFT_OK;
  }
  if (paired_supported(p->log2n, p->variant, p->dtype, batch) && !((a0 | b0) & (c64 ? 15u : 7u))) {
    e = paired_launch(p->log2n, in, out, exp_in, exp_out, p->dtype, batch, inverse, kernel_ctab(p), p->small, st);
    if (e != cudaSuccess) return cuda_fail(e, "paired kernel launch");
    ++p->launches;
    return AMQFT_OK;
  }
  FusedArgs a;
  memset(&a, 0, sizeof a);
  a.in = in;
  a.out = out;
  a.exp_in = exp_in;
  a.exp_out = exp_out;
  a.dtype = p->dtype;
  a.ctab = kernel_ctab(p);
  a.batch = batch;
  a.logN = p->log2n;
  a.tpc = p->cfg.per_cta;
  a.inverse = inverse;
  a.RS = p->cfg.RS;
  a.tot_off = p->cfg.tot_off;
  a.tlist = nullptr;
  a.toff = nullptr;
  a.nreal = 0;
  e = fused_launch(p->variant, a, p->small, p->cfg, st);
  if (e != cudaSuccess) return cuda_fail(e, "fused kernel launch");
  ++p->launches;
  return AMQFT_OK;
}

int amqft_exec_fwd(amqft_plan_t p, const void* in, void* out, int32_t* exp_out, void* stream) {
  t_err.clear();
  if (!p) return fail(AMQFT_ERR_ARG, "plan is NULL");
  return exec_n(p, p->batch, in, out, 0, nullptr, exp_out, stream);
}

int amqft_exec_inv(amqft_plan_t p, const void* in, const int32_t* exp_in, void* out, int32_t* exp_out,
                   void* stream) {
  t_err.clear();
  if (!p) return fail(AMQFT_ERR_ARG, "plan is NULL");
  return exec_n(p, p->batch, in, out, 1, exp_in, exp_out, stream);
}

// Special input / output forms (real input, DCT-0 / DST-0, inverse real):
// nsig signals, two per complex transform of the plan's length, on the fused
// kernels up to 2^16 and the multi-pass path above.
enum { SP_RDFT, SP_TRIG, SP_IRDFT };

static int exec_special(amqft_plan_t p, int mode, long long nsig, const void* in, void* out, const float* in2,
                        float* out2, void* stream, const char* who) {
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e;
  const long long slots = (nsig + 1) / 2;
  const int inverse = mode == SP_IRDFT ? 1 : 0;
  if (p->log2n > AMQFT_LOG2N_FUSED_MAX) {
    const long long per_buf = p->chunk * 4 * p->RSg;
    for (long long t0 = 0; t0 < slots; t0 += p->chunk) {
      MpArgs a = {};
      a.in = in;
      a.out = out;
      a.in2 = in2;
      a.out2 = out2;
      a.dtype = AMQFT_C64;
      a.ctab = kernel_ctab(p);
      a.nt = (slots - t0) < p->chunk ? (slots - t0) : p->chunk;
      a.t0 = t0;
      a.logN = p->log2n;
      a.inverse = inverse;
      a.RSg = p->RSg;
      a.nreal = mode == SP_RDFT ? nsig : 0;
      a.ntrig = mode == SP_TRIG ? nsig : 0;
      a.nirdft = mode == SP_IRDFT ? nsig : 0;
      long long nl = 0;
      e = multipass_dispatch(p->variant, a, p->d_work, p->d_work + per_buf, p->small, st, &nl);
      p->launches += nl;
      if (e != cudaSuccess) return cuda_fail(e, who);
    }
    return AMQFT_OK;
  }
  FusedArgs a;
  memset(&a, 0, sizeof a);
  a.in = in;
  a.out = out;
  a.in2 = in2;
  a.out2 = out2;
  a.dtype = AMQFT_C64;
  a.ctab = kernel_ctab(p);
  a.batch = slots;
  a.nreal = mode == SP_RDFT ? nsig : 0;
  a.ntrig = mode == SP_TRIG ? nsig : 0;
  a.nirdft = mode == SP_IRDFT ? nsig : 0;
  a.inverse = inverse;
  a.logN = p->log2n;
  a.tpc = p->cfg.per_cta;
  a.RS = p->cfg.RS;
  a.tot_off = p->cfg.tot_off;
  e = fused_launch(p->variant, a, p->small, p->cfg, st);
  if (e != cudaSuccess) return cuda_fail(e, who);
  ++p->launches;
  return AMQFT_OK;
}

static bool ranges_overlap(uintptr_t a, uintptr_t na, uintptr_t b, uintptr_t nb) {
  return a && b && na && nb && a < b + nb && b < a + na;
}

int amqft_exec_rdft(amqft_plan_t p, const float* in, void* out, void* stream) {
  t_err.clear();
  if (!p) return fail(AMQFT_ERR_ARG, "plan is NULL");
  if (p->ragged) return fail(AMQFT_ERR_ARG, "amqft_exec_rdft: not for ragged plans");
  if (p->dtype != AMQFT_C64) return fail(AMQFT_ERR_DTYPE, "amqft_exec_rdft: AMQFT_C64 plans only");
  if (p->batch == 0) return AMQFT_OK;
  if (!in || !out) return fail(AMQFT_ERR_ALIGN, "amqft_exec_rdft: in or out is NULL");
  if (((uintptr_t)in & 3u) || ((uintptr_t)out & 7u))
    return fail(AMQFT_ERR_ALIGN, "amqft_exec_rdft: in must be 4-byte and out 8-byte aligned");
  const long long N = 1LL << p->log2n;
  const uintptr_t a0 = (uintptr_t)in, b0 = (uintptr_t)out;
  const uintptr_t ia = (uintptr_t)(N * p->batch * 4), ob = (uintptr_t)((N / 2 + 1) * p->batch * 8);
  if (a0 < b0 + ob && b0 < a0 + ia) return fail(AMQFT_ERR_INPLACE, "amqft_exec_rdft: in and out overlap");
  if (p->log2n == 0) {
    copy1_real_kernel<<<(unsigned)((p->batch + 255) / 256), 256, 0, (cudaStream_t)stream>>>(in, (float2*)out,
                                                                                             p->batch);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "copy kernel launch");
    ++p->launches;
    return AMQFT_OK;
  }
  return exec_special(p, SP_RDFT, p->batch, in, out, nullptr, nullptr, stream, "amqft_exec_rdft: launch");
}

int amqft_exec_irdft(amqft_plan_t p, const void* in, float* out, void* stream) {
  t_err.clear();
  if (!p) return fail(AMQFT_ERR_ARG, "plan is NULL");
  if (p->ragged) return fail(AMQFT_ERR_ARG, "amqft_exec_irdft: not for ragged plans");
  if (p->dtype != AMQFT_C64) return fail(AMQFT_ERR_DTYPE, "amqft_exec_irdft: AMQFT_C64 plans only");
  if (p->log2n < 1) return fail(AMQFT_ERR_N, "amqft_exec_irdft: log2n=%d below 1", p->log2n);
  if (p->batch == 0) return AMQFT_OK;
  if (!in || !out) return fail(AMQFT_ERR_ALIGN, "amqft_exec_irdft: in or out is NULL");
  if (((uintptr_t)in & 7u) || ((uintptr_t)out & 3u))
    return fail(AMQFT_ERR_ALIGN, "amqft_exec_irdft: in must be 8-byte and out 4-byte aligned");
  const long long N = 1LL << p->log2n;
  if (ranges_overlap((uintptr_t)in, (uintptr_t)((N / 2 + 1) * p->batch * 8), (uintptr_t)out,
                     (uintptr_t)(N * p->batch * 4)))
    return fail(AMQFT_ERR_INPLACE, "amqft_exec_irdft: in and out overlap");
  return exec_special(p, SP_IRDFT, p->batch, in, out, nullptr, nullptr, stream, "amqft_exec_irdft: launch");
}

int amqft_exec_dct_dst(amqft_plan_t p, int64_t count, const float* dct_in, float* dct_out, const float* dst_in,
                       float* dst_out, void* stream) {
  t_err.clear();
  if (!p) return fail(AMQFT_ERR_ARG, "plan is NULL");
  if (p->ragged) return fail(AMQFT_ERR_ARG, "amqft_exec_dct_dst: not for ragged plans");
  if (p->dtype != AMQFT_C64) return fail(AMQFT_ERR_DTYPE, "amqft_exec_dct_dst: AMQFT_C64 plans only");
  if (p->log2n < 2) return fail(AMQFT_ERR_N, "amqft_exec_dct_dst: log2n=%d below 2", p->log2n);
  if (count < 0 || count > p->batch)
    return fail(AMQFT_ERR_ARG, "amqft_exec_dct_dst: count=%lld outside [0, %lld]", (long long)count,
                (long long)p->batch);
  if (!dct_in != !dct_out || !dst_in != !dst_out)
    return fail(AMQFT_ERR_ALIGN, "amqft_exec_dct_dst: give both or neither of dct_in/dct_out, dst_in/dst_out");
  if (count == 0 || (!dct_in && !dst_in)) return AMQFT_OK;
  if (((uintptr_t)dct_in | (uintptr_t)dct_out | (uintptr_t)dst_in | (uintptr_t)dst_out) & 3u)
    return fail(AMQFT_ERR_ALIGN, "amqft_exec_dct_dst: arrays must be 4-byte aligned");
  const long long half = 1LL << (p->log2n - 1);
  const uintptr_t cb = (uintptr_t)((half + 1) * count * 4), sb = (uintptr_t)((half - 1) * count * 4);
  const uintptr_t ci = (uintptr_t)dct_in, co = (uintptr_t)dct_out, si = (uintptr_t)dst_in, so = (uintptr_t)dst_out;
  // each kind may run in place; nothing else may overlap
  if ((ci != co && ranges_overlap(ci, cb, co, cb)) || (si != so && ranges_overlap(si, sb, so, sb)) ||
      ranges_overlap(ci, cb, si, sb) || ranges_overlap(ci, cb, so, sb) || ranges_overlap(co, cb, si, sb) ||
      ranges_overlap(co, cb, so, sb))
    return fail(AMQFT_ERR_INPLACE, "amqft_exec_dct_dst: arrays overlap");
  return exec_special(p, SP_TRIG, count, dct_in, dct_out, dst_in, dst_out, stream, "amqft_exec_dct_dst: launch");
}

// Host-memory execution: staging on the device, three internal streams.
static void host_release(amqft_plan_t p) {
  for (int i = 0; i < 4; ++i)
    if (p->h_buf[i]) cudaFree(p->h_buf[i]);
  for (int i = 0; i < 3; ++i)
    if (p->h_st[i]) cudaStreamDestroy(p->h_st[i]);
  for (int i = 0; i < 8; ++i)
    if (p->h_ev[i]) cudaEventDestroy(p->h_ev[i]);
  memset(p->h_buf, 0, sizeof p->h_buf);
  memset(p->h_st, 0, sizeof p->h_st);
  memset(p->h_ev, 0, sizeof p->h_ev);
  p->h_chunk = 0;
}

int amqft_exec_host(amqft_plan_t p, const void* in, void* out, int direction, int64_t chunk, void* stream) {
  t_err.clear();
  if (!p) return fail(AMQFT_ERR_ARG, "plan is NULL");
  if (p->ragged) return fail(AMQFT_ERR_ARG, "amqft_exec_host: not for ragged plans");
  if (p->dtype != AMQFT_C64) return fail(AMQFT_ERR_DTYPE, "amqft_exec_host: AMQFT_C64 plans only");
  if (direction != 0 && direction != 1) return fail(AMQFT_ERR_ARG, "amqft_exec_host: direction must be 0 or 1");
  if (chunk < 0) return fail(AMQFT_ERR_ARG, "amqft_exec_host: chunk=%lld < 0", (long long)chunk);
  if (p->batch == 0) return AMQFT_OK;
  if (!in || !out) return fail(AMQFT_ERR_ALIGN, "amqft_exec_host: in or out is NULL");
  if (((uintptr_t)in | (uintptr_t)out) & 7u) return fail(AMQFT_ERR_ALIGN, "amqft_exec_host: in/out must be 8-byte aligned");
  const long long N = 1LL << p->log2n, tbytes = N * 8;
  const uintptr_t bytes = (uintptr_t)(tbytes * p->batch), a0 = (uintptr_t)in, b0 = (uintptr_t)out;
  if (a0 != b0 && a0 < b0 + bytes && b0 < a0 + bytes)
    return fail(AMQFT_ERR_INPLACE, "amqft_exec_host: in and out overlap without being equal");
  long long C = chunk > 0 ? chunk : (64LL << 20) / tbytes;
  if (C < 1) C = 1;
  if (C > p->batch) C = p->batch;
  cudaError_t e = cudaSuccess;
  if (p->h_chunk < C) {  // first use, or a larger chunk: (re)allocate the staging
    host_release(p);
    for (int i = 0; i < 4 && e == cudaSuccess; ++i) e = cudaMalloc(&p->h_buf[i], (size_t)(C * tbytes));
    for (int i = 0; i < 3 && e == cudaSuccess; ++i) e = cudaStreamCreateWithFlags(&p->h_st[i], cudaStreamNonBlocking);
    for (int i = 0; i < 8 && e == cudaSuccess; ++i) e = cudaEventCreateWithFlags(&p->h_ev[i], cudaEventDisableTiming);
    if (e != cudaSuccess) {
      host_release(p);
      return fail(AMQFT_ERR_NOMEM, "amqft_exec_host: staging allocation failed: %s", cudaGetErrorString(e));
    }
    p->h_chunk = C;
  }
  cudaStream_t caller = (cudaStream_t)stream, s_in = p->h_st[0], s_comp = p->h_st[1], s_out = p->h_st[2];
  cudaEvent_t* ev_in = p->h_ev;        // [0, 2): copy-in of slot s done
  cudaEvent_t* ev_comp = p->h_ev + 2;  // [2, 4): transform of slot s done
  cudaEvent_t* ev_out = p->h_ev + 4;   // [4, 6): copy-out of slot s done
  cudaEvent_t ev_start = p->h_ev[6], ev_join = p->h_ev[7];
  if ((e = cudaEventRecord(ev_start, caller)) != cudaSuccess) return cuda_fail(e, "amqft_exec_host: cudaEventRecord");
  for (int i = 0; i < 3; ++i) cudaStreamWaitEvent(p->h_st[i], ev_start, 0);
  const char* hin = static_cast<const char*>(in);
  char* hout = static_cast<char*>(out);
  int slot = 0;
  for (long long t0 = 0; t0 < p->batch; t0 += C, slot ^= 1) {
    const long long c = (p->batch - t0) < C ? (p->batch - t0) : C;
    void* din = p->h_buf[slot];
    void* dout = p->h_buf[2 + slot];
    // copy in once the transform that last read this slot is done
    cudaStreamWaitEvent(s_in, ev_comp[slot], 0);
    e = cudaMemcpyAsync(din, hin + t0 * tbytes, (size_t)(c * tbytes), cudaMemcpyHostToDevice, s_in);
    if (e != cudaSuccess) return cuda_fail(e, "amqft_exec_host: copy in");
    cudaEventRecord(ev_in[slot], s_in);
    // transform once the copy in is done and the last copy out of this slot is done
    cudaStreamWaitEvent(s_comp, ev_in[slot], 0);
    cudaStreamWaitEvent(s_comp, ev_out[slot], 0);
    const int rc = exec_n(p, c, din, dout, direction, nullptr, nullptr, s_comp);
    if (rc != AMQFT_OK) return rc;
    cudaEventRecord(ev_comp[slot], s_comp);
    // copy out
    cudaStreamWaitEvent(s_out, ev_comp[slot], 0);
    e = cudaMemcpyAsync(hout + t0 * tbytes, dout, (size_t)(c * tbytes), cudaMemcpyDeviceToHost, s_out);
    if (e != cudaSuccess) return cuda_fail(e, "amqft_exec_host: copy out");
    cudaEventRecord(ev_out[slot], s_out);
  }
  // the last copy out follows every earlier operation of the call
  cudaEventRecord(ev_join, s_out);
  e = cudaStreamWaitEvent(caller, ev_join, 0);
  if (e != cudaSuccess) return cuda_fail(e, "amqft_exec_host: join");
  return AMQFT_OK;
}

int amqft_destroy(amqft_plan_t p) {
  t_err.clear();
  if (!p) return AMQFT_OK;
  if (p->d_ctab) cudaFree(p->d_ctab);
  if (p->d_work) cudaFree(p->d_work);
  if (p->d_rcnt) cudaFree(p->d_rcnt);
  if (p->d_rlist) cudaFree(p->d_rlist);
  if (p->d_rwork) cudaFree(p->d_rwork);
  host_release(p);
  delete p;
  return AMQFT_OK;
}

static long long ragged_capacity(const amqft_plan_s* p, int c) {
  const long long byp = p->max_points >> c;
  return byp < p->max_count ? byp : p->max_count;
}

static long long region_stride_g(int c) { return (((1LL << (c - 1)) + 2 + 31) / 32) * 32; }

// class index of the unaligned 2^14 list of a ragged call (0: no split, every
// 2^14..2^16 transform on the fused cluster kernels): the paired-region
// kernel runs variant 4, and needs in and out at the same 16-byte phase
static int ragged_ubase(amqft_plan_t p, const void* in, const void* out) {
  const bool same = (((uintptr_t)in ^ (uintptr_t)out) & 8u) == 0;
  return p->variant == 4 && p->log2n >= 14 && same ? p->log2n + 1 : 0;
}

int amqft_plan_ragged(amqft_plan_t* out, int max_log2n, int variant, int dtype, int64_t max_count,
                      int64_t max_points) {
  t_err.clear();
  if (!out) return fail(AMQFT_ERR_ARG, "amqft_plan_ragged: out is NULL");
  *out = nullptr;
  if (dtype != AMQFT_C64) return fail(AMQFT_ERR_DTYPE, "amqft_plan_ragged: ragged batches are AMQFT_C64 only");
  if (max_count < 1 || max_count > (1LL << 30))
    return fail(AMQFT_ERR_ARG, "amqft_plan_ragged: max_count=%lld outside [1, 2^30]", (long long)max_count);
  if (max_points < 1) return fail(AMQFT_ERR_ARG, "amqft_plan_ragged: max_points=%lld < 1", (long long)max_points);
  amqft_plan_t p = nullptr;
  int rc = amqft_plan(&p, max_log2n, variant, 0, dtype);
  if (rc != AMQFT_OK) return rc;
  p->ragged = 1;
  p->max_count = max_count;
  p->max_points = max_points;
  cudaError_t e = cudaMalloc(&p->d_rcnt, 64 * sizeof(int));
  // one list per length, and three for the unaligned transforms of 2^14..2^16
  if (e == cudaSuccess) e = cudaMalloc(&p->d_rlist, (size_t)(max_log2n + 4) * (size_t)max_count * sizeof(int));
  long long ws = 0;
  for (int c = AMQFT_LOG2N_FUSED_MAX + 1; c <= max_log2n; ++c) {
    const long long need = 2LL * ragged_capacity(p, c) * 4 * region_stride_g(c);
    if (need > ws) ws = need;
  }
  if (e == cudaSuccess && ws > 0) e = cudaMalloc(&p->d_rwork, (size_t)ws * sizeof(float));
  if (e != cudaSuccess) {
    amqft_destroy(p);
    return fail(AMQFT_ERR_NOMEM, "amqft_plan_ragged: device allocation failed: %s", cudaGetErrorString(e));
  }
  *out = p;
  return AMQFT_OK;
}

int amqft_exec_ragged(amqft_plan_t p, int64_t count, const int64_t* d_offsets, const uint8_t* d_log2n,
                      const void* in, void* out, int direction, void* stream) {
  t_err.clear();
  if (!p) return fail(AMQFT_ERR_ARG, "plan is NULL");
  if (!p->ragged) return fail(AMQFT_ERR_ARG, "amqft_exec_ragged: the plan was not made by amqft_plan_ragged");
  if (count < 0 || count > p->max_count)
    return fail(AMQFT_ERR_ARG, "amqft_exec_ragged: count=%lld outside [0, max_count=%lld]", (long long)count,
                p->max_count);
  if (direction != 0 && direction != 1) return fail(AMQFT_ERR_ARG, "amqft_exec_ragged: direction must be 0 or 1");
  if (count == 0) return AMQFT_OK;
  if (!in || !out || !d_offsets || !d_log2n) return fail(AMQFT_ERR_ALIGN, "amqft_exec_ragged: NULL pointer");
  if ((((uintptr_t)in | (uintptr_t)out | (uintptr_t)d_offsets) & 7u) != 0)
    return fail(AMQFT_ERR_ALIGN, "amqft_exec_ragged: in, out and offsets must be 8-byte aligned");
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaMemsetAsync(p->d_rcnt, 0, 64 * sizeof(int), st);
  if (e != cudaSuccess) return cuda_fail(e, "amqft_exec_ragged: cudaMemsetAsync");
  {
    long long blocks = (count + 255) / 256;
    if (blocks > 8LL * p->num_sms) blocks = 8LL * p->num_sms;
    ragged_bucket_kernel<<<(unsigned)blocks, 256, 0, st>>>(d_log2n, (const long long*)d_offsets, count, p->log2n,
                                                           p->max_points, p->d_rcnt, p->d_rlist, p->max_count,
                                                           p->d_rcnt + 33, (const float2*)in, (float2*)out,
                                                           ragged_ubase(p, in, out), (int)(((uintptr_t)in >> 3) & 1));
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "ragged bucket launch");
    ++p->launches;
  }
  FusedArgs a;
  memset(&a, 0, sizeof a);
  a.in = in;
  a.out = out;
  a.dtype = AMQFT_C64;
  a.ctab = kernel_ctab(p);
  a.inverse = direction;
  a.toff = (const long long*)d_offsets;
  RaggedArgs r;
  r.cnt = p->d_rcnt;
  r.list = p->d_rlist;
  r.cap = p->max_count;
  r.work = p->d_rcnt + 32;
  r.maxlog = p->log2n < AMQFT_LOG2N_FUSED_MAX ? p->log2n : AMQFT_LOG2N_FUSED_MAX;
  r.ubase = ragged_ubase(p, in, out);
  r.sched = p->knob[0];
  r.order = p->knob[1];
  RaggedLaunch L;
  memset(&L, 0, sizeof L);
  L.small_grid = p->num_sms * p->knob[2];
  for (int c = 1; c <= 13 && c <= r.maxlog; ++c) {
    const int tpc = small_tpc(c);
    const int sm_bytes =
        (small_tot_off(c) + SMALL_TPB + 32 + snap_floats(4 * tpc * (1 << (c - 1))) + tpc + band_consts(c)) *
        (int)sizeof(float);
    if (sm_bytes > L.small_smem) L.small_smem = sm_bytes;
  }
  for (int q = 0; q < 3; ++q) {
    const FusedConfig fc = fused_config(14 + q, p->variant);
    L.clusters[q] = (p->num_sms / 4) * p->knob[3];
    L.cluster_smem[q] = fc.smem;
    L.cluster_tot_off[q] = fc.tot_off;
  }
  long long nl = 0;
  e = ragged_launch(p->variant, a, p->small, r, L, st, &nl);
  p->launches += nl;
  if (e != cudaSuccess) return cuda_fail(e, "ragged launch");
  for (int c = AMQFT_LOG2N_FUSED_MAX + 1; c <= p->log2n; ++c) {
    const long long capc = ragged_capacity(p, c);
    if (capc < 1) continue;
    const long long RSg = region_stride_g(c);
    MpArgs m = {};
    memset(&m, 0, sizeof m);
    m.in = in;
    m.out = out;
    m.dtype = AMQFT_C64;
    m.ctab = kernel_ctab(p);
    m.nt = capc;
    m.t0 = 0;
    m.logN = c;
    m.inverse = direction;
    m.RSg = RSg;
    m.tlist = p->d_rlist + (long long)c * p->max_count;
    m.toff = (const long long*)d_offsets;
    m.ntdev = p->d_rcnt + c;
    nl = 0;
    e = multipass_dispatch(p->variant, m, p->d_rwork, p->d_rwork + capc * 4 * RSg, p->small, st, &nl);
    p->launches += nl;
    if (e != cudaSuccess) return cuda_fail(e, "ragged multi-pass launch");
  }
  return AMQFT_OK;
}

int amqft_ragged_tune(amqft_plan_t p, int knob, int value) {
  t_err.clear();
  if (!p || !p->ragged) return fail(AMQFT_ERR_ARG, "amqft_ragged_tune: not a ragged plan");
  static const int lo[4] = {0, 0, 1, 1}, hi[4] = {1, 1, 4, 4};
  if (knob < 0 || knob > 3) return fail(AMQFT_ERR_ARG, "amqft_ragged_tune: knob=%d not in 0..3", knob);
  if (value < lo[knob] || value > hi[knob])
    return fail(AMQFT_ERR_ARG, "amqft_ragged_tune: value %d for knob %d outside [%d, %d]", value, knob, lo[knob],
                hi[knob]);
  p->knob[knob] = value;
  return AMQFT_OK;
}

int amqft_ragged_skipped(amqft_plan_t p, int64_t* skipped) {
  t_err.clear();
  if (!p || !p->ragged || !skipped) return fail(AMQFT_ERR_ARG, "amqft_ragged_skipped: bad arguments");
  int v = 0;
  const cudaError_t e = cudaMemcpy(&v, p->d_rcnt + 33, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "amqft_ragged_skipped: cudaMemcpy");
  *skipped = v;
  return AMQFT_OK;
}

int64_t amqft_plan_launches(amqft_plan_t p) {
  t_err.clear();
  if (!p) return fail(AMQFT_ERR_ARG, "plan is NULL");
  return (int64_t)p->launches.load();
}

int amqft_debug_bounds(int64_t* count, uint64_t* first, int clear) {
  t_err.clear();
  using Reader = cudaError_t (*)(unsigned long long*, unsigned long long*, bool);
  static const Reader readers[] = {bounds_v1, bounds_v2, bounds_v3, bounds_v4,  bounds_v5, bounds_v6,
                                   bounds_v7, bounds_v8, bounds_p14, bounds_p15, bounds_p16};
  unsigned long long total = 0, f = 0;
  for (Reader r : readers) {
    unsigned long long c = 0, fi = 0;
    const cudaError_t e = r(&c, &fi, clear != 0);
    if (e != cudaSuccess) return cuda_fail(e, "amqft_debug_bounds");
    if (c && !total) f = fi;
    total += c;
  }
  if (count) *count = (int64_t)total;
  if (first) *first = (uint64_t)f;
#ifdef AMQFT_BOUNDS_CHECK
  return 1;
#else
  return 0;
#endif
}

int amqft_plan_set_constants(amqft_plan_t p, int mode) {
  t_err.clear();
  if (!p) return fail(AMQFT_ERR_ARG, "plan is NULL");
  if (mode != AMQFT_CONST_TABLE && mode != AMQFT_CONST_FLY)
    return fail(AMQFT_ERR_ARG, "amqft_plan_set_constants: mode=%d is not AMQFT_CONST_TABLE or AMQFT_CONST_FLY", mode);
  p->const_mode = mode;
  return AMQFT_OK;
}

int amqft_plan_get_constants(amqft_plan_t p) {
  t_err.clear();
  if (!p) return fail(AMQFT_ERR_ARG, "plan is NULL");
  return p->const_mode;
}

int amqft_plan_info(amqft_plan_t p, int* cluster, int* per_cta, int* threads, int* smem_bytes) {
  t_err.clear();
  if (!p) return fail(AMQFT_ERR_ARG, "plan is NULL");
  if (cluster) *cluster = p->cfg.cluster;
  if (per_cta) *per_cta = p->cfg.per_cta;
  if (threads) *threads = p->cfg.threads;
  if (smem_bytes) *smem_bytes = p->cfg.smem;
  return AMQFT_OK;
}

}  // extern "C"
