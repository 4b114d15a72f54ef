/*
 * amqft: batched power-of-two complex DFT by the AM-QFT recursion
 * ("A class of AM-QFT algorithms for power-of-two FFT", Pasquini),
 * computed by hand-written CUDA kernels for sm_103a (GB300).
 *
 * The transform is the DFT of Eq. qft_0A,
 *     X(k) = sum_{n=0}^{N-1} x(n) exp(-2*pi*i*n*k/N),   N = 2^log2n,
 * computed by one of the 8 AM-QFT variants (Sect. 5-6): the D_c / D_r
 * decompositions (Sect. 3.1-3.2), the D_k / D_n separations and H_k / H_n
 * halvings (Tab. 3-4), and the odd-to-even conversion M_variant (Tab. 5-6).
 *
 * Conventions for every entry point:
 *   - Data are interleaved complex (re, im), transform-major: transform b
 *     occupies elements [b*N, (b+1)*N).  AMQFT_C64 elements are 2 x float32
 *     (8 bytes); in and out must be 8-byte aligned device pointers.
 *   - 16-bit storage (AMQFT_CBF16, AMQFT_CF16, AMQFT_CI16): an element is a
 *     pair of bfloat16, IEEE binary16 or int16 values (4 bytes, real part
 *     first), in and out 4-byte aligned; int16 is block-floating point
 *     (fixed-point mantissas with one exponent per transform, 15 bits below
 *     the largest component; the paper's fixed-point motivation, with the
 *     arithmetic kept in float32).  Transform b holds the values stored * 2^exp[b], one
 *     int32 exponent per transform in a separate device array.  Arithmetic is
 *     float32 throughout: inputs are widened and scaled exactly; each output
 *     transform gets the exponent that puts its largest component magnitude
 *     in [2^13, 2^14) (0 for an all-zero transform), is scaled by 2^-exp
 *     exactly and rounded once to nearest even (int16: to the nearest integer, ties to even).  Exponents are clamped to
 *     [-100, 100] (outside that range the scaling saturates).
 *   - in and out are owned by the caller.  in == out is the in-place
 *     transform (every entry point but amqft_exec_rdft / amqft_exec_irdft;
 *     amqft_exec_dct_dst per kind): each kernel reads a
 *     transform's whole input before it writes any of that transform's output,
 *     and no transform's output overlaps another's input, so the result is
 *     bit-identical to the out-of-place call.  Any other overlap is rejected
 *     (AMQFT_ERR_INPLACE).  The transforms up to 2^AMQFT_LOG2N_FUSED_MAX then
 *     touch one buffer: one HBM read and one write per sample, no workspace.
 *   - stream is a cudaStream_t (NULL = legacy default stream).  Calls are
 *     asynchronous on that stream and make no host synchronisation.
 *   - Return value: AMQFT_OK (0) or a negative AMQFT_ERR_* code; the
 *     message of the last error on the calling thread is amqft_last_error().
 *   - The inverse is unnormalised: inv(fwd(x)) = N * x.  Since every AM-QFT
 *     constant is real, it is computed as conj(F(conj(x))), which is also the
 *     adjoint F^H used for gradients.
 */
#ifndef AMQFT_H
#define AMQFT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define AMQFT_OK 0
#define AMQFT_ERR_N (-1)        /* log2n outside the supported range */
#define AMQFT_ERR_VARIANT (-2)  /* variant not in 1..8 */
#define AMQFT_ERR_DTYPE (-3)    /* dtype not supported by this entry point */
#define AMQFT_ERR_ALIGN (-4)    /* pointer misaligned or NULL */
#define AMQFT_ERR_INPLACE (-5)  /* in and out overlap without being equal */
#define AMQFT_ERR_CUDA (-6)     /* a CUDA call or kernel launch failed */
#define AMQFT_ERR_DEVICE (-7)   /* device is not sm_103 or lacks resources */
#define AMQFT_ERR_ARG (-8)      /* other invalid argument (NULL plan, batch < 0, ...) */
#define AMQFT_ERR_NOMEM (-9)    /* host or device allocation failed */

#define AMQFT_LOG2N_FUSED_MAX 16 /* largest log2n of the fused single-pass kernels */
#define AMQFT_LOG2N_MAX 28       /* largest log2n (multi-pass above 2^16) */

typedef enum { AMQFT_C64 = 0, AMQFT_CBF16 = 1, AMQFT_CF16 = 2, AMQFT_CI16 = 3 } amqft_dtype;

typedef struct amqft_plan_s *amqft_plan_t;

/* Create a plan for `batch` transforms of length 2^log2n with AM-QFT
 * variant `variant` (1..8, Sect. 6) and storage `dtype` (amqft_dtype).
 * The plan owns the variant's trig-constant table (Sect. 7.1: the
 * M/8 constants 2cos, 1/(2cos), 2sin or 1/(2sin) of theta*(2j+1) for every
 * periodisation M = 16..N, N/4 - 2 floats in all) on the current device.
 * Lengths up to 2^AMQFT_LOG2N_FUSED_MAX run in one fused kernel (one HBM
 * read and write per sample).  Longer transforms (every variant; the
 * recurrences of variants 1, 3, 5, 7 become chunk passes and a scan of the
 * chunk totals) run as several passes over a workspace the plan allocates:
 * two buffers of the transform's size per transform of a chunk, at most
 * 2 GiB or one transform's two buffers if larger (4 GiB at 2^28), the batch
 * processed chunk by chunk.  That workspace
 * (like the staging of amqft_exec_host) belongs to the plan, so the exec calls
 * of one plan must be ordered: one stream, or streams joined by events.  Calls
 * on different plans are independent.
 * Errors: AMQFT_ERR_N (log2n < 0 or > AMQFT_LOG2N_MAX), AMQFT_ERR_VARIANT (not in 1..8),
 * AMQFT_ERR_DTYPE (not an amqft_dtype), AMQFT_ERR_ARG (out NULL or batch < 0), AMQFT_ERR_DEVICE,
 * AMQFT_ERR_NOMEM, AMQFT_ERR_CUDA.  On error *out is set to NULL. */
int amqft_plan(amqft_plan_t *out, int log2n, int variant, int64_t batch, int dtype);

/* Forward transform of the plan's batch: out = DFT(in), Eq. qft_0A.
 * exp_out: AMQFT_C64 plans, NULL; 16-bit plans, a device array of `batch`
 * int32 that receives the output exponents (the input exponents are 0).
 * Errors: AMQFT_ERR_ARG (NULL plan; exp_out NULL for 16-bit), AMQFT_ERR_ALIGN,
 * AMQFT_ERR_INPLACE, AMQFT_ERR_DTYPE (exponents given for AMQFT_C64),
 * AMQFT_ERR_CUDA (launch failure). */
int amqft_exec_fwd(amqft_plan_t plan, const void *in, void *out, int32_t *exp_out, void *stream);

/* Unnormalised inverse / adjoint: out = conj(DFT(conj(in))) = N * IDFT(in).
 * exp_in / exp_out: NULL for AMQFT_C64; for 16-bit plans exp_in holds the
 * input exponents (NULL: all 0) and exp_out receives the output exponents.
 * Errors as amqft_exec_fwd. */
int amqft_exec_inv(amqft_plan_t plan, const void *in, const int32_t *exp_in, void *out,
                   int32_t *exp_out, void *stream);

/* Real input (forward only): `batch` real signals of N = 2^log2n float32
 * samples at in (signal j at [j*N, (j+1)*N)), their DFTs' harmonics 0 .. N/2
 * (the rest follow by conjugate symmetry) to out, N/2 + 1 complex64 values
 * per signal.  Two real signals a, b share one complex transform of a + ib:
 * its regions C1, S1 and C2, S2 (Sect. 3.1-3.2) are the DCT-0 / DST-0 of a and
 * of b, and R = DCT - i DST (Eq. qft_24-25), so the input costs 4 bytes a
 * point.  Each harmonic equals the complex transform of the signal with a zero
 * imaginary part.  Every length of the plan (the multi-pass path above
 * 2^AMQFT_LOG2N_FUSED_MAX); in 4-byte, out 8-byte aligned, not overlapping.
 * Errors: AMQFT_ERR_ARG, AMQFT_ERR_DTYPE (16-bit plans), AMQFT_ERR_ALIGN,
 * AMQFT_ERR_INPLACE, AMQFT_ERR_CUDA. */
int amqft_exec_rdft(amqft_plan_t plan, const float *in, void *out, void *stream);

/* Inverse of amqft_exec_rdft, unnormalised: `batch` half spectra at in
 * (N/2 + 1 complex64 values each, harmonics 0 .. N/2 of a real signal; the
 * imaginary parts of harmonics 0 and N/2 are taken as given) to the real
 * signals N * x at out (N float32 each).  Two spectra share one complex
 * transform: Z = X_a + i X_b with the Hermitian extension X(N - k) =
 * conj X(k), and out = conj(DFT(conj Z)) splits into N x_a (real part) and
 * N x_b (imaginary part).  log2n >= 1; in 8-byte, out 4-byte aligned, not
 * overlapping.  Errors: AMQFT_ERR_ARG, AMQFT_ERR_N, AMQFT_ERR_DTYPE,
 * AMQFT_ERR_ALIGN, AMQFT_ERR_INPLACE, AMQFT_ERR_CUDA. */
int amqft_exec_irdft(amqft_plan_t plan, const void *in, float *out, void *stream);

/* DCT-0 and DST-0 of periodisation N = 2^log2n (Eq. qft_0B-0C, theta =
 * 2 pi / N): S(k) = sum_{n=0}^{N/2} s(n) cos(theta n k), k = 0..N/2, and
 * S(k) = sum_{n=1}^{N/2-1} s(n) sin(theta n k), k = 1..N/2-1; the recursion's
 * dct(N) and dst(N) (Sect. 4-6) without D_c / D_r around them.  count
 * (<= the plan's batch) signals of each kind: DCT-0 inputs at dct_in, N/2 + 1
 * floats each (n = 0..N/2), results at dct_out alike; DST-0 inputs at
 * dst_in, N/2 - 1 floats each (n = 1..N/2-1 at [n - 1]), results at dst_out
 * alike (k at [k - 1]).  Either pair may be NULL (that kind is not
 * computed); a DCT-0 pair and a DST-0 pair of two signals each share one
 * complex transform's four regions.  Each kind may run in place (dct_in ==
 * dct_out, dst_in == dst_out); no other overlap.  log2n >= 2; arrays 4-byte
 * aligned.  Errors: AMQFT_ERR_ARG (count outside [0, batch]), AMQFT_ERR_N,
 * AMQFT_ERR_DTYPE, AMQFT_ERR_ALIGN (misaligned, or only one pointer of a
 * pair), AMQFT_ERR_INPLACE, AMQFT_ERR_CUDA. */
int amqft_exec_dct_dst(amqft_plan_t plan, int64_t count, const float *dct_in, float *dct_out,
                       const float *dst_in, float *dst_out, void *stream);

/* Transform the plan's batch from HOST memory to HOST memory: forward
 * (direction 0) or unnormalised inverse (direction 1) of `batch` complex64
 * transforms at in (read) and out (written), both host pointers, 8-byte
 * aligned, equal (in place) or not overlapping; page-locked memory lets the copies overlap the
 * transforms (pageable memory works, with synchronous copies).  The batch runs
 * in chunks of `chunk` transforms (0: about 64 MiB per chunk): each chunk is
 * copied to the device, transformed by the same kernels as amqft_exec_fwd/inv
 * and copied back, the copy-in of chunk i + 1 and the copy-out of chunk i - 1
 * overlapping the transform of chunk i on three internal streams.  The call is
 * asynchronous: `stream` is joined at the end, so out is complete once stream
 * is.  The first call (or one with a larger chunk) allocates the plan's
 * staging: two input and two output buffers of `chunk` transforms.  Calls on
 * one plan must not run concurrently from several host threads.
 * Errors: AMQFT_ERR_ARG (NULL or ragged plan, direction, chunk < 0),
 * AMQFT_ERR_DTYPE (16-bit plans), AMQFT_ERR_ALIGN, AMQFT_ERR_INPLACE,
 * AMQFT_ERR_NOMEM (staging), AMQFT_ERR_CUDA. */
int amqft_exec_host(amqft_plan_t plan, const void *in, void *out, int direction, int64_t chunk, void *stream);

/* Release the plan and everything it owns.  NULL is accepted. */
int amqft_destroy(amqft_plan_t plan);

/* Message of the last error on the calling thread ("" if none).  The string
 * stays valid until the next amqft call on the same thread. */
const char *amqft_last_error(void);

/* Library build/version string. */
const char *amqft_version(void);

/* Kernel configuration the plan selected, for tests and benchmarks:
 * cluster size (CTAs per transform, 1 when a CTA holds whole transforms),
 * transforms per CTA, threads per CTA, dynamic shared memory bytes per CTA.
 * Any out pointer may be NULL. */
int amqft_plan_info(amqft_plan_t plan, int *cluster, int *per_cta, int *threads, int *smem_bytes);

/* Number of kernels the library has launched for exec calls on this plan
 * (amqft_exec_fwd / inv / host / rdft / ragged / static) since it was made:
 * a host-side count of launches that were accepted by the CUDA runtime, for
 * benchmarks that report how many kernels a step runs.  Memsets and copies are
 * not kernels and are not counted.  Returns the count (>= 0), or
 * AMQFT_ERR_ARG for a NULL plan. */
int64_t amqft_plan_launches(amqft_plan_t plan);

/* Where the kernels take the trig constants of the tree levels of
 * periodisation M >= 256 (Sect. 7.1; the M <= 128 constants of the register
 * leaves are kernel arguments in both modes):
 *   AMQFT_CONST_TABLE (default): the plan's table, rounded once from long
 *     double; the single-pass kernels stage it per CTA in shared memory.
 *     Variants 2, 4, 6, 8 are then bit-identical to the float32 recursion.
 *   AMQFT_CONST_FLY: the "on the fly" evaluation the paper discusses (cheap
 *     for the 2cos / 2sin constants of variants 1, 3, 5, 7): each kernel
 *     computes the constants from their exact angles in float32 (cospif /
 *     sinpif after an exact fold into [0, pi/4], then 2x or 1/(2x)), staged
 *     per CTA in shared memory by the single-pass kernels and computed at
 *     each use by the multi-pass levels above 2^13.  The kernels read no
 *     table.  Results differ from table mode in the last bits of the
 *     constants (within a few ulp), so they are held to the float32
 *     tolerance rather than to bit identity.
 * The mode applies to every later exec call on the plan (all entry points).
 * Errors: AMQFT_ERR_ARG (NULL plan, unknown mode). */
#define AMQFT_CONST_TABLE 0
#define AMQFT_CONST_FLY 1
int amqft_plan_set_constants(amqft_plan_t plan, int mode);

/* The plan's constants mode, or AMQFT_ERR_ARG for a NULL plan. */
int amqft_plan_get_constants(amqft_plan_t plan);

/* Bounds checks.  The debug library (libamqft_debug.so, the same sources
 * built with AMQFT_BOUNDS_CHECK) checks every region access of the kernels
 * (shared memory, the cluster's distributed shared memory, the multi-pass
 * workspace) against the region's size, the paired kernel's region and HBM
 * accesses, and the HBM element index of every input and output against the
 * transform length.  A failing access is skipped (a load reads zero or a
 * scratch word, a store is dropped), counted, and the first one recorded as
 * (site << 48) | (index & (2^48 - 1)); nothing traps, so the kernel ends and
 * the context stays usable.  This call reads (and if `clear` is nonzero
 * resets) the record; it synchronises with the device's work through the
 * copy.  Returns 1 in the checked build, 0 in the release build (whose count
 * is always 0), or AMQFT_ERR_CUDA.  count / first may be NULL. */
int amqft_debug_bounds(int64_t *count, uint64_t *first, int clear);

/* ---------------------------------------------------------------------
 * Ragged batches: many transforms of different power-of-two lengths, each at
 * its own offset, in one call that launches a fixed sequence of kernels and
 * makes no host synchronisation (capturable in a CUDA graph once the plan
 * exists; the first call also sets kernel attributes, so make one eager call
 * before capturing).
 */

/* Plan for ragged batches of up to max_count transforms, each of length
 * 2^k with 0 <= k <= max_log2n, and at most max_points points of lengths above
 * 2^AMQFT_LOG2N_FUSED_MAX in one batch.  Owns the constant table of the longest
 * length (it holds those of every shorter length), the per-length id lists
 * ((max_log2n + 1) * max_count int32) and, when max_log2n > 16, a multi-pass
 * workspace of about 16 bytes per point of max_points.  AMQFT_C64 only.
 * Errors: as amqft_plan, plus AMQFT_ERR_ARG (max_count outside [1, 2^30],
 * max_points < 1), AMQFT_ERR_DTYPE (16-bit storage), AMQFT_ERR_NOMEM. */
int amqft_plan_ragged(amqft_plan_t *out, int max_log2n, int variant, int dtype, int64_t max_count,
                      int64_t max_points);

/* Transform `count` (<= max_count) ragged transforms: transform i has
 * 2^d_log2n[i] interleaved complex64 elements starting at element
 * d_offsets[i] of in (read) and of out (written); forward (direction 0) or
 * unnormalised inverse (direction 1).  d_offsets (int64) and d_log2n (uint8)
 * are device arrays of `count` entries; in, out and d_offsets are 8-byte
 * aligned; the transforms must not overlap each other, and in and out are
 * equal (in place) or do not overlap.
 * Transforms whose log2 N exceeds the plan's, and multi-pass transforms beyond
 * the max_points capacity, are skipped and counted (amqft_ragged_skipped).
 * Each transform gives exactly the result of amqft_exec_fwd/inv of a plan of
 * its length.  Errors: AMQFT_ERR_ARG (not a ragged plan, count outside
 * [0, max_count], direction not 0/1), AMQFT_ERR_ALIGN, AMQFT_ERR_CUDA. */
int amqft_exec_ragged(amqft_plan_t plan, int64_t count, const int64_t *d_offsets, const uint8_t *d_log2n,
                      const void *in, void *out, int direction, void *stream);

/* Launch knobs of a ragged plan, set by the autotuner: knob 0 schedule of
 * the persistent small-length launch (0 static, 1 dynamic work counter;
 * default 1), knob 1 order of its work items (0 longest lengths first, 1
 * shortest first; default 0), knob 2 its CTAs per SM (1..4; default 1),
 * knob 3 cluster grid multiplier of the 2^14..2^16 launches (1..4; default 1).
 * Errors: AMQFT_ERR_ARG. */
int amqft_ragged_tune(amqft_plan_t plan, int knob, int value);

/* Number of transforms the last amqft_exec_ragged call skipped.  Waits for
 * the device (cudaMemcpy).  Errors: AMQFT_ERR_ARG, AMQFT_ERR_CUDA. */
int amqft_ragged_skipped(amqft_plan_t plan, int64_t *skipped);

/* ---------------------------------------------------------------------
 * Allocation-free execution.  The paper has no counterpart to this entry
 * point: it runs the same multi-pass kernels as amqft_exec_fwd/inv, with
 * their workspace in a fixed device array compiled into the library instead
 * of one the plan allocates.  It serves callers that must not allocate device
 * memory when they run a transform (cudaMalloc/cudaFree may synchronise the
 * device or fail when another allocator owns the free memory) and callers
 * that cannot keep a workspace per plan.
 */
#define AMQFT_STATIC_LOG2N_MIN 17
#define AMQFT_STATIC_LOG2N_MAX 20
/* 2 transforms x 2 ping-pong buffers x 4 regions x (2^19 + 32) floats:
 * 32 MiB + 2 KiB per device, reserved when the library's module is loaded. */
#define AMQFT_STATIC_SCRATCH_FLOATS 8389120LL

/* Run `batch` transforms of the plan's length and variant: forward
 * (inverse == 0, out = DFT(in)) or unnormalised inverse (inverse != 0,
 * out = conj(DFT(conj(in)))), bit-identical to amqft_exec_fwd/inv of a plan
 * with that batch.  The plan supplies length, variant and constant table and
 * its own batch is ignored: create it with batch 0 so that it holds no
 * workspace.  in/out: device pointers to batch * 2^log2n interleaved complex
 * float32 values, owned by the caller, 8-byte aligned, equal (in place) or
 * not overlapping.  Makes no device or host allocation.  Every call looks up the scratch
 * array's address in the current context (a host-side lookup, never cached,
 * so a reset device is safe); the first call on a device may load the
 * library's module into the context, so make it before any stream capture.
 * The scratch is shared by
 * every plan on the device: calls that overlap in time (different streams, or
 * host threads without ordering) race; calls on one stream are ordered.
 * Nothing in the scratch needs to start at zero.
 * Errors: AMQFT_ERR_ARG (NULL plan, batch < 0), AMQFT_ERR_N (plan length
 * outside [2^AMQFT_STATIC_LOG2N_MIN, 2^AMQFT_STATIC_LOG2N_MAX]: shorter
 * lengths use no workspace, longer ones need more than the array holds),
 * AMQFT_ERR_DTYPE, AMQFT_ERR_ALIGN, AMQFT_ERR_INPLACE, AMQFT_ERR_DEVICE (the
 * current device is not the plan's), AMQFT_ERR_CUDA. */
int amqft_exec_static(amqft_plan_t plan, int64_t batch, const void *in, void *out, int inverse, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* AMQFT_H */
