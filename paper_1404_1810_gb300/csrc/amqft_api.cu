// C ABI of the AM-QFT library (include/amqft.h): plans, constant tables,
// argument checks and kernel dispatch.  No compute happens on the host
// except the trig-constant table of a plan.
#include <math.h>
#include <stdarg.h>
#include <new>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <string>

#include "amqft.h"
#include "amqft_multipass_impl.cuh"
#include "amqft_internal.h"

namespace amqft {

FusedConfig fused_config(int logN) {
  FusedConfig c;
  const int N = 1 << logN, half = N >> 1;
  c.RS = region_stride(logN);
  if (logN <= 13) {
    c.cluster = 1;
    c.threads = 512;
    // a CTA holds 16384 region values: 512 threads x 32 values
    const int tpc = (512 * 32) / (N >= 4 ? 2 * N : 8);
    c.per_cta = tpc < 1 ? 1 : tpc;
    c.nreg = 4 * c.per_cta;
  } else {
    c.cluster = 4;
    c.per_cta = 1;
    c.nreg = 1;
    c.threads = half / 32;  // 32 region values per thread
  }
  c.tot_off = ((c.nreg * c.RS + 31) / 32) * 32;
  c.smem = (c.tot_off + c.threads + 32 + snap_floats(c.nreg * half)) * (int)sizeof(float);
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

static cudaError_t multipass_launch(int variant, const MpArgs& a, float* W0, float* W1, const SmallConsts& K,
                                    cudaStream_t st) {
  switch (variant) {
    case 2: return multipass_variant_2(a, W0, W1, K, st);
    case 4: return multipass_variant_4(a, W0, W1, K, st);
    case 6: return multipass_variant_6(a, W0, W1, K, st);
    default: return multipass_variant_8(a, W0, W1, K, st);
  }
}

// N = 1: the DFT is the identity (conjugated twice for the inverse).
__global__ void copy1_kernel(const float2* __restrict__ in, float2* __restrict__ out, long long batch) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < batch) out[i] = in[i];
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
  SmallConsts small;
  FusedConfig cfg;
  // multi-pass path: two ping-pong workspaces of chunk * 4 regions
  float* d_work;
  long long chunk;
  long long RSg;
};

// workspace budget of one plan (both ping-pong buffers)
static const long long kWorkspaceBytes = 2LL << 30;

namespace amqft {

int plan_view(amqft_plan_t p, PlanView* v) {
  if (!p || !v) return fail(AMQFT_ERR_ARG, "plan is NULL");
  v->log2n = p->log2n;
  v->variant = p->variant;
  v->dtype = p->dtype;
  v->device = p->device;
  v->ctab = p->d_ctab;
  v->small = &p->small;
  return AMQFT_OK;
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
  if (log2n > AMQFT_LOG2N_FUSED_MAX && (variant & 1))
    return fail(AMQFT_ERR_VARIANT,
                "amqft_plan: variant %d (a recurrence variant) is limited to log2n <= %d; "
                "variants 2, 4, 6, 8 reach %d", variant, AMQFT_LOG2N_FUSED_MAX, AMQFT_LOG2N_MAX);
  if (dtype != AMQFT_C64 && dtype != AMQFT_CBF16 && dtype != AMQFT_CF16)
    return fail(AMQFT_ERR_DTYPE, "amqft_plan: dtype=%d is not AMQFT_C64, AMQFT_CBF16 or AMQFT_CF16", dtype);
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
  p->d_work = nullptr;
  p->chunk = 0;
  p->RSg = 0;
  // level-major table: periodisation M = 16..N holds M/8 constants at [M/8-2, M/4-2)
  const long long N = 1LL << log2n;
  const long long ntab = N >= 16 ? N / 4 - 2 : 0;
  const long long nhost = ntab > (long long)(LEAF - 2) ? ntab : (long long)(LEAF - 2);
  float* h = (float*)calloc((size_t)nhost, sizeof(float));
  if (!h) { delete p; return fail(AMQFT_ERR_NOMEM, "amqft_plan: host allocation failed"); }
  for (long long M = 16; M / 8 - 2 < nhost; M *= 2)
    for (long long j = 0; j < M / 8 && M / 8 - 2 + j < nhost; ++j) h[M / 8 - 2 + j] = variant_const(variant, M, j);
  for (int i = 0; i < LEAF - 2; ++i) p->small.c[i] = h[i];
  p->small.cos_pi4 = (float)cos_frac(1, 8);
  if (ntab > 0) {
    e = cudaMalloc(&p->d_ctab, (size_t)ntab * sizeof(float));
    if (e != cudaSuccess) { free(h); delete p; return cuda_fail(e, "amqft_plan: cudaMalloc(constant table)"); }
    e = cudaMemcpy(p->d_ctab, h, (size_t)ntab * sizeof(float), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) { free(h); cudaFree(p->d_ctab); delete p; return cuda_fail(e, "amqft_plan: cudaMemcpy"); }
  }
  free(h);
  if (log2n >= 1 && log2n <= AMQFT_LOG2N_FUSED_MAX) p->cfg = fused_config(log2n);
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

static int exec(amqft_plan_t p, const void* in, void* out, int inverse, const int32_t* exp_in, int32_t* exp_out,
                void* stream) {
  t_err.clear();
  if (!p) return fail(AMQFT_ERR_ARG, "plan is NULL");
  const bool c64 = p->dtype == AMQFT_C64;
  if (c64 && (exp_in || exp_out)) return fail(AMQFT_ERR_DTYPE, "exponent arrays are only used with 16-bit storage");
  if (p->batch == 0) return AMQFT_OK;
  if (!in || !out) return fail(AMQFT_ERR_ALIGN, "in or out is NULL");
  const uintptr_t amask = c64 ? 7u : 3u;
  if (((uintptr_t)in | (uintptr_t)out) & amask)
    return fail(AMQFT_ERR_ALIGN, "in/out must be %d-byte aligned", (int)amask + 1);
  if (!c64) {
    if (!exp_out) return fail(AMQFT_ERR_ARG, "16-bit storage needs exp_out (one int32 per transform)");
    if (((uintptr_t)exp_out | (uintptr_t)exp_in) & 3u) return fail(AMQFT_ERR_ALIGN, "exponent arrays must be 4-byte aligned");
  }
  const long long N = 1LL << p->log2n;
  const uintptr_t bytes = (uintptr_t)(N * p->batch * (c64 ? 8 : 4));
  const uintptr_t a0 = (uintptr_t)in, b0 = (uintptr_t)out;
  if (a0 < b0 + bytes && b0 < a0 + bytes) return fail(AMQFT_ERR_INPLACE, "in and out overlap");
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e;
  if (p->log2n > AMQFT_LOG2N_FUSED_MAX) {
    const long long per_buf = p->chunk * 4 * p->RSg;
    for (long long t0 = 0; t0 < p->batch; t0 += p->chunk) {
      MpArgs a;
      a.in = in;
      a.out = out;
      a.exp_in = exp_in;
      a.exp_out = exp_out;
      a.dtype = p->dtype;
      a.ctab = p->d_ctab;
      a.nt = (p->batch - t0) < p->chunk ? (p->batch - t0) : p->chunk;
      a.t0 = t0;
      a.logN = p->log2n;
      a.inverse = inverse;
      a.RSg = p->RSg;
      e = multipass_launch(p->variant, a, p->d_work, p->d_work + per_buf, p->small, st);
      if (e != cudaSuccess) return cuda_fail(e, "multi-pass launch");
    }
    return AMQFT_OK;
  }
  if (p->log2n == 0) {
    const unsigned grid = (unsigned)((p->batch + 255) / 256);
    if (c64) copy1_kernel<<<grid, 256, 0, st>>>((const float2*)in, (float2*)out, p->batch);
    else copy1_16_kernel<<<grid, 256, 0, st>>>((const unsigned*)in, (unsigned*)out, exp_in, exp_out, p->batch,
                                               p->dtype);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "copy kernel launch");
    return AMQFT_OK;
  }
  FusedArgs a;
  a.in = in;
  a.out = out;
  a.exp_in = exp_in;
  a.exp_out = exp_out;
  a.dtype = p->dtype;
  a.ctab = p->d_ctab;
  a.batch = p->batch;
  a.logN = p->log2n;
  a.tpc = p->cfg.per_cta;
  a.inverse = inverse;
  a.RS = p->cfg.RS;
  a.tot_off = p->cfg.tot_off;
  e = fused_launch(p->variant, a, p->small, p->cfg, st);
  if (e != cudaSuccess) return cuda_fail(e, "fused kernel launch");
  return AMQFT_OK;
}

int amqft_exec_fwd(amqft_plan_t p, const void* in, void* out, int32_t* exp_out, void* stream) {
  return exec(p, in, out, 0, nullptr, exp_out, stream);
}

int amqft_exec_inv(amqft_plan_t p, const void* in, const int32_t* exp_in, void* out, int32_t* exp_out,
                   void* stream) {
  return exec(p, in, out, 1, exp_in, exp_out, stream);
}

int amqft_destroy(amqft_plan_t p) {
  t_err.clear();
  if (!p) return AMQFT_OK;
  if (p->d_ctab) cudaFree(p->d_ctab);
  if (p->d_work) cudaFree(p->d_work);
  delete p;
  return AMQFT_OK;
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
