/*
 * turbofft.h -- C ABI of a batched 1-D complex-to-complex FFT for NVIDIA
 * GB300 (sm_103a) with online two-sided algorithm-based fault tolerance.
 *
 * Method: TurboFFT (PPoPP'25).
 *   - Transform: the DFT of Sec. 2.2.1,
 *       forward  y_j = sum_n x_n exp(-2 pi i j n / N)
 *       inverse  x_j = (1/N) sum_n y_n exp(+2 pi i j n / N)
 *     computed as a Stockham FFT (Sec. 3.2), in one pass over HBM for
 *     N <= 2^13 (float32) / 2^12 (float64) and in two passes (four-step,
 *     N = N1 * N2, the kernel-level tiling of Sec. 3.1) up to N = 2^24
 *     (three passes N1 * N2 * N3 for float32 N >= 2^22; optionally one pass
 *     over a thread-block cluster for float32 2^13..2^16).
 *   - Fault tolerance: the two-sided checksum of Sec. 4.1 (Eq. 4-5) fused
 *     into the transform kernels (Sec. 4.2.2), amortised over several
 *     transactions of one thread block (Sec. 4.3), with the location
 *     encoding (1, 2, ...) of Sec. 4.1 and the delayed, batched correction
 *     of Sec. 4.1.2.  The fault model is one soft error per checksum group
 *     (Sec. 2.2.4).
 *
 * Conventions for every entry point
 *   - No call allocates or frees caller memory.  A plan owns every device
 *     and pinned-host buffer it allocates (tables, the intermediate buffer of
 *     two-pass plans unless the caller supplies one with
 *     turbofft_set_workspace, the fault-tolerance report and correction
 *     records) and frees them in turbofft_destroy.  turbofft_exec_host keeps
 *     a per-device staging area (see there).
 *   - Data layout: `batch` transforms of `n` interleaved complex values
 *     (re, im), contiguous, transform b at element offset b * n.  Element
 *     type is float (TURBOFFT_C2C_F32, 8 bytes per value) or double
 *     (TURBOFFT_C2C_F64, 16 bytes per value).
 *   - Device pointers must be 16-byte aligned device memory on the plan's
 *     device.  Out-of-place only: `in` is never written.
 *   - Status codes: every function returns TURBOFFT_SUCCESS or an error;
 *     no function aborts the process.  Launch-time CUDA errors are reported
 *     as TURBOFFT_CUDA_ERROR with the CUDA message in turbofft_last_error.
 *   - A plan is not thread-safe: calls on one plan must not overlap from
 *     several host threads.  Distinct plans are independent.
 */
#ifndef TURBOFFT_H
#define TURBOFFT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* cudaStream_t is `struct CUstream_st *`; NULL is the legacy default stream. */
struct CUstream_st;
typedef struct CUstream_st *turbofft_stream;

typedef enum {
  TURBOFFT_SUCCESS = 0,
  TURBOFFT_INVALID_VALUE = 1,     /* bad size, pointer, alignment or enum */
  TURBOFFT_UNSUPPORTED = 2,       /* valid request this library does not do (in-place) */
  TURBOFFT_ALLOC_FAILED = 3,      /* device or pinned allocation failed */
  TURBOFFT_CUDA_ERROR = 4,        /* a CUDA runtime call failed */
  TURBOFFT_FT_UNCORRECTABLE = 5,  /* the last exec saw an error it could not fix */
  TURBOFFT_TIMEOUT = 6            /* reserved: a bounded device wait expired */
} turbofft_status;

typedef enum {
  TURBOFFT_C2C_F32 = 0,           /* complex64: float re, float im */
  TURBOFFT_C2C_F64 = 1            /* complex128: double re, double im */
} turbofft_dtype;

/* direction argument of turbofft_plan_create */
#define TURBOFFT_FORWARD (-1)          /* y = W x,            W = (w^{jk}), w = e^{-2 pi i/N} */
#define TURBOFFT_INVERSE (1)           /* y = (1/N) conj(W) x  (Sec. 2.2.1 inverse) */
#define TURBOFFT_INVERSE_UNSCALED (2)  /* y = conj(W) x = W^H x, the adjoint of FORWARD */
#define TURBOFFT_FORWARD_SCALED (-2)   /* y = (1/N) W x, the adjoint of INVERSE */

typedef enum {
  TURBOFFT_FT_OFF = 0,            /* plain FFT, no checksums */
  TURBOFFT_FT_DETECT = 1,         /* checksums fused; detect and locate, report only */
  TURBOFFT_FT_CORRECT = 2,        /* detect, locate and correct in place (Sec. 4.1.2); F64
                                     two-pass plans check and correct whole transforms
                                     (one checksum pair per transform over both passes,
                                     a failing transform recomputed); others check each
                                     pass's sub-transforms in groups */
  TURBOFFT_FT_CORRECT_REGISTERS = 3, /* CORRECT, with the right-side sums accumulated in
                                        registers during the transform (the thread-level
                                        accumulation of Sec. 4.3) instead of formed from the
                                        untouched input and the stored output when a group
                                        fails its check; same results, more registers */
  TURBOFFT_FT_CORRECT_THREAD = 4  /* thread-level ABFT (Sec. 4.2.1): for lengths whose
                                     transform one thread holds whole (F32 N = 8, 16, 32;
                                     F64 N = 8, 16), each thread checks its own transform
                                     (v.x against e.y, per-transform threshold with
                                     twice the group threshold's gamma) with no
                                     block reduction and corrects a failing transform in
                                     its registers by recomputing it from the staged input.
                                     UNSUPPORTED for other lengths, other structures and
                                     ragged plans */
} turbofft_ft_mode;

typedef struct turbofft_plan turbofft_plan;

/*
 * A fault-injection site (Sec. 5.3.1 flips one bit of one value of one
 * signal).  Coordinates are the plan's own:
 *   transform  index of the transform in the batch, [0, batch)
 *   pass       kernel pass, [0, info.num_passes)
 *   stage      radix stage of that pass, [0, info.stages[pass]]: the value
 *              entering radix stage `stage` (0 = as loaded, after the input
 *              checksum is taken); stage == info.stages[pass] is the pass's
 *              output before its output checksum is taken
 *   element    [0, n): index of the value in the transform's working array
 *              at that stage.  For a two-pass plan with n = N1 * N2 the
 *              working array of pass 0 holds column n2 at elements
 *              p * N2 + n2 (p = position within the length-N1 column) and
 *              that of pass 1 holds row k1 at elements k1 * N2 + p.  A
 *              three-pass plan (n = N1 * M, M = N2 * N3) has pass 0 as a
 *              two-pass plan with N2 := M; passes 1 and 2 transform each
 *              first-pass output row k1 (length M) as a two-pass plan
 *              N2 x N3 whose working array sits at elements k1 * M + ...
 *   component  0 = real part, 1 = imaginary part
 */
typedef struct {
  int64_t transform;
  int32_t pass;
  int32_t stage;
  int64_t element;
  int32_t component;
} turbofft_site;

/* Outcome of the most recent turbofft_exec on a plan with ft_mode != OFF. */
typedef struct {
  int64_t groups_checked;   /* checksum groups verified (all passes) */
  int64_t detected;         /* groups whose checksum test failed */
  int64_t located;          /* of those, groups where one signal was identified */
  int64_t corrected;        /* signals corrected (CORRECT mode) */
  int64_t recomputed;       /* of the corrected, fixed by recomputing from the input */
  int64_t uncorrectable;    /* detected groups that could not be fixed / located */
  int64_t first_transform;  /* transform of the first located error, -1 if none */
  int32_t first_pass;       /* pass of the first detection, -1 if none */
  int32_t reserved;
  double first_residual;    /* |S1| of the first detected group */
  double first_threshold;   /* tau of that group */
  double max_clean_ratio;   /* max |S1| / tau over groups that passed */
} turbofft_report;

/* Static facts about a plan. */
typedef struct {
  int64_t n, batch;
  int32_t dtype, direction, ft_mode;
  int32_t num_passes;       /* 1, 2 or 3 */
  int64_t sub_n[3];         /* sub-transform length of each pass (n = sub_n[0] * sub_n[1] * sub_n[2],
                               unused entries 1) */
  int32_t stages[3];        /* radix stages of each pass */
  int32_t radix[3];         /* radix of the register-level butterflies of each pass */
  int32_t group_transactions; /* transactions of one thread block per checksum group */
  int32_t grid[3];          /* persistent thread blocks launched per pass */
  int32_t block[3];         /* threads per block per pass */
  int64_t workspace_bytes;  /* device memory the plan owns or will allocate;
                               float64 multi-pass plans include 16 bytes per
                               point of each column pass's length (n, and
                               n2 for the second pass of a three-pass plan)
                               for its twiddle table, twice that with fault
                               tolerance on (checksum weights) */
  int64_t scratch_bytes;    /* intermediate buffer of a two-pass plan (0 for one pass) */
  int32_t per_block[3];     /* transforms (SP) / columns / rows one block holds per transaction */
  int32_t num_members;      /* ragged plan: distinct sizes (member plans); 0 otherwise */
  int32_t autotuned;        /* 1 if launch shapes were chosen by timing (turbofft_set_autotune) */
  int32_t cluster;          /* > 0: both passes run in ONE kernel whose thread-block clusters of
                               this many blocks share each transform (one HBM round trip);
                               grid/block then describe that kernel */
  int32_t single_launch;    /* ragged plan: 1 if an exec is one launch of the persistent
                               ragged kernel, 0 if a graph of per-size kernels */
  int32_t transform_checks; /* 1: checksums over whole transforms (F64 two-pass plans with
                               DETECT / CORRECT): an exec launches the two passes, a check
                               kernel and two recompute kernels */
  int32_t tma_passes;       /* bit p set: pass p stages its input tiles with TMA copies
                               (turbofft_set_tma_staging); else 16-byte cp.async copies */
} turbofft_plan_info;

/* Duration of one kernel of the last exec (turbofft_set_profiling). */
typedef struct {
  int32_t pass;             /* kernel pass */
  int32_t is_correction;    /* 0 = transform kernel, 1 = correction kernel */
  double ms;                /* CUDA-event time on the exec's stream */
} turbofft_kernel_time;

/*
 * Create a plan on the current CUDA device.
 *   n          transform length, a power of two in [8, 2^24]
 *   batch      number of transforms, >= 1, batch * n <= 2^31 elements
 *   dtype      TURBOFFT_C2C_F32 or TURBOFFT_C2C_F64
 *   direction  TURBOFFT_FORWARD, TURBOFFT_INVERSE, TURBOFFT_INVERSE_UNSCALED or
 *              TURBOFFT_FORWARD_SCALED
 *   ft_mode    TURBOFFT_FT_OFF / _DETECT / _CORRECT
 *   plan       out: the new plan (set to NULL on failure)
 * Tables (twiddles, checksum vectors e and e^T W) are computed on the host
 * in long double / double and copied to the device here, synchronously.
 * Errors: INVALID_VALUE for any argument out of range, ALLOC_FAILED,
 * CUDA_ERROR (no device, or a copy failed).
 */
turbofft_status turbofft_plan_create(int64_t n, int64_t batch, turbofft_dtype dtype,
                                     int direction, turbofft_ft_mode ft_mode,
                                     turbofft_plan **plan);

/*
 * Same as turbofft_plan_create with the plan's structure fixed instead of
 * chosen (turbofft_plan_create uses SPLIT, or with autotuning on the faster
 * of the two by timing):
 *   TURBOFFT_STRUCTURE_SPLIT    one kernel pass for n up to the largest
 *                               single-block size (2^13 float32, 2^12
 *                               float64), two four-step passes beyond it
 *   TURBOFFT_STRUCTURE_CLUSTER  one kernel pass whose thread-block clusters
 *                               share each transform (info.cluster > 0);
 *                               TURBOFFT_UNSUPPORTED for sizes without a
 *                               cluster configuration
 *   TURBOFFT_STRUCTURE_THREE_PASS  three four-step passes N1 x N2 x N3 (the
 *                               default for float32 n >= 2^22); for n >= 2^9
 *                               where every pass has a kernel configuration,
 *                               else TURBOFFT_UNSUPPORTED
 *   TURBOFFT_STRUCTURE_FLOAT_PAIRS  F64 only, ft_mode OFF only (else
 *                               TURBOFFT_UNSUPPORTED): the SPLIT passes with
 *                               the float64 data held in registers and
 *                               shared memory as float pairs (hi + lo, 48
 *                               significand bits) and transformed with float
 *                               arithmetic instead of on the FP64 pipe
 *                               (GB300 runs FP64 at about 1/64 of its FP32
 *                               rate); the data in memory stays complex128.
 *                               Inputs must lie in [2^-74, 2^127) in
 *                               magnitude (or be zero): the float exponent
 *                               range.  No counterpart in the paper (its
 *                               GPUs run FP64 at 1/2 to 1/32 of FP32)
 * Every structure computes the same transform to the same accuracy bar.
 * Errors: as turbofft_plan_create; INVALID_VALUE for another structure.
 */
#define TURBOFFT_STRUCTURE_SPLIT 1
#define TURBOFFT_STRUCTURE_CLUSTER 2
#define TURBOFFT_STRUCTURE_THREE_PASS 3
#define TURBOFFT_STRUCTURE_FLOAT_PAIRS 4
turbofft_status turbofft_plan_create_structured(int64_t n, int64_t batch, turbofft_dtype dtype,
                                                int direction, turbofft_ft_mode ft_mode, int structure,
                                                turbofft_plan **plan);

/*
 * Ragged batch: `count` transforms of mixed power-of-two lengths in one plan
 * (a batching facility; the paper's kernels take one length per launch).
 *   sizes[i]    length of transform i, a power of two in [8, 2^24]
 *   offsets[i]  element offset of transform i in the packed buffers given
 *               to turbofft_exec; F32 offsets must be even (each transform
 *               starts on a 16-byte boundary); transforms may not overlap,
 *               gaps are allowed and never touched
 *   count       >= 1
 *   dtype, direction, ft_mode: as turbofft_plan_create; one group of
 *               equal-length transforms per distinct size may hold at most
 *               2^31 elements
 * The plan holds one member plan per distinct size (turbofft_plan_get_member_info,
 * members in ascending size order) whose kernels address their transforms
 * through a device copy of the offsets.
 *   - F32 plans whose lengths are all <= 2^16, ft_mode OFF, DETECT or
 *     CORRECT (info.single_launch = 1, unless turned off with
 *     turbofft_set_ragged_single_launch): turbofft_exec is ONE launch of a
 *     persistent kernel (cooperative: all blocks resident) whose blocks take
 *     work items, largest first, from a queue over every member's passes;
 *     a grid barrier separates the column passes of lengths >= 8192 from
 *     their row passes, and the corrections of detected groups run inside
 *     the same launch.  A barrier that waits more than about a second
 *     makes the exec fail: turbofft_get_report returns TURBOFFT_TIMEOUT.
 *   - Otherwise: ONE CUDA graph in which the members' kernels are parallel
 *     branches.
 * Either form is captured in a CUDA graph on the first exec and captured
 * again whenever `in` or `out` differ from the last captured pair (a
 * synchronous step: do not exec a ragged plan with new pointers inside a
 * stream capture of your own).  An exec with a site armed by
 * turbofft_inject runs uncaptured (the single launch carries the site; the
 * graph form queues the members' kernels directly).  The packed
 * buffers span max(offsets[i] + sizes[i]) elements.  turbofft_get_report
 * sums the members' reports, transform indices are the global ones (i), and
 * turbofft_inject takes the global transform index.  turbofft_exec_host
 * copies the whole packed span in, runs the graph and copies it out.
 * turbofft_set_workspace, turbofft_set_profiling and
 * turbofft_exec_static_scratch return TURBOFFT_UNSUPPORTED on ragged plans.
 * With autotuning on, every member is tuned on its own indexed geometry.
 * Errors: INVALID_VALUE (NULL arrays, count < 1, a bad size, a negative,
 * odd (F32) or overlapping offset), ALLOC_FAILED, CUDA_ERROR.
 */
turbofft_status turbofft_plan_create_ragged(const int64_t *sizes, const int64_t *offsets, int64_t count,
                                            turbofft_dtype dtype, int direction,
                                            turbofft_ft_mode ft_mode, turbofft_plan **plan);

/* Facts about member `index` (ascending size order) of a ragged plan;
 * INVALID_VALUE for a plan that is not ragged or an index out of range. */
turbofft_status turbofft_plan_get_member_info(const turbofft_plan *plan, int32_t index,
                                              turbofft_plan_info *info);

/*
 * Autotuning of launch shapes (process-wide switch, off by default).  When
 * on, every plan created afterwards times each registered shape of each of
 * its passes -- radix (complex values per thread), threads per transform
 * and transforms per thread block -- on its own geometry (its batch, length,
 * fault-tolerance mode and, for ragged members, offsets) and keeps the
 * fastest.  The timing runs at plan creation on temporary buffers the size
 * of the plan's data (no tuning if they cannot be allocated) and is cached
 * per process.  Results do not depend on the shape: every shape computes
 * the same transform.  Returns SUCCESS.
 */
turbofft_status turbofft_set_autotune(int enable);

/*
 * Process-wide: whether ragged plans created afterwards run as one launch of
 * the persistent ragged kernel where they can (enable = 1, the default) or
 * as a graph of per-size kernels (0).  A batching facility: the paper tunes
 * one kernel per length (Sec. 3.3).
 */
turbofft_status turbofft_set_ragged_single_launch(int enable);

/*
 * Process-wide: how F32 one- and two-pass plans created afterwards stage
 * their input tiles: mode 0 with 16-byte cp.async copies by every thread; 1
 * (the default) with TMA (tensor-memory-accelerator) copies issued by one
 * thread where they measured faster on GB300 (row passes; column passes
 * whose tile rows are S x 8 >= 64 bytes, at N1 >= 512 or with ft_mode not
 * OFF; single passes of N = 4096, of 1024 and 2048 with ft_mode not OFF,
 * of 256 and 8192 with ft_mode OFF), else cp.async; 2 with TMA wherever the
 * kernel's tile allows it.  A column tile
 * (S adjacent columns of the N1 x N2 view, Sec. 3.1's kernel-level tiling)
 * is one 2-D box of the input viewed as rows of N2 values; the tile of a
 * single pass (S whole transforms) or of a row pass (S adjacent rows) is one
 * contiguous bulk copy where the kernel keeps it unswizzled in shared memory.
 * Completion is counted on a shared-memory barrier.  The results are
 * bitwise the same either way.  Each exec encodes the tensor map of a column
 * pass's input pointer (16-byte aligned, as every exec requires); an input
 * viewed as 2^31 rows or more runs that exec with cp.async.  The wait for a
 * tile is bounded: after about a second without completion the kernel stops
 * and turbofft_get_report returns TURBOFFT_TIMEOUT (for plans with ft_mode
 * OFF that flag then stays set for the plan).  Returns SUCCESS, or
 * INVALID_VALUE for a mode outside 0..2.
 */
turbofft_status turbofft_set_tma_staging(int mode);

/*
 * Transform `in` into `out` (both device pointers, see the layout above) on
 * `stream`.  Asynchronous: returns after queueing the kernels.  in == out
 * (or overlapping buffers) returns TURBOFFT_UNSUPPORTED.  With ft_mode !=
 * OFF the checksums are verified on the device and the outcome is read with
 * turbofft_get_report.  A site armed with turbofft_inject is applied to this
 * exec and then disarmed.
 * Errors: INVALID_VALUE (NULL or misaligned pointer), UNSUPPORTED,
 * CUDA_ERROR (launch failed).
 */
turbofft_status turbofft_exec(turbofft_plan *plan, const void *in, void *out,
                              turbofft_stream stream);

/*
 * Same transform with HOST buffers: copies `host_in` to the device, runs
 * the transform and copies the result to `host_out`, pipelined in chunks of
 * the batch over three internal streams (copy in, transform, copy out)
 * ordered after `stream`, and returns when `host_out` is complete.  Host
 * buffers should be pinned (cudaHostAlloc / cudaHostRegister) for full
 * bandwidth; pageable memory works but is slower.  The device staging (five
 * chunk buffers of about 128 MiB, or one transform if larger, and the
 * streams) is shared by all plans of a device, allocated by the first call
 * and kept until the process exits; calls from several host threads on one
 * device are serialised.
 */
turbofft_status turbofft_exec_host(turbofft_plan *plan, const void *host_in, void *host_out,
                                   turbofft_stream stream);

/*
 * Arm a one-shot fault for the next exec: flip bit `bit` of the value at
 * `site` (coordinates above).  bit in [0, 31] (F32) or [0, 63] (F64).
 * Errors: INVALID_VALUE for any coordinate out of range.
 */
turbofft_status turbofft_inject(turbofft_plan *plan, turbofft_site site, int bit);

/*
 * Wait for the most recent exec on this plan and read its fault-tolerance
 * report.  Returns TURBOFFT_FT_UNCORRECTABLE (with *report filled) if that
 * exec left an error it could not correct (or, in DETECT mode, detected
 * one); SUCCESS otherwise.  With ft_mode == OFF the report is all zero.
 */
turbofft_status turbofft_get_report(turbofft_plan *plan, turbofft_report *report);

/* Fill *info with the plan's static facts. */
turbofft_status turbofft_plan_get_info(const turbofft_plan *plan, turbofft_plan_info *info);

/*
 * Scale the detection threshold tau by `factor` (> 0; 1 restores the
 * default).  For threshold studies (detection vs false-alarm rate,
 * Sec. 5.3.1); the default is calibrated for zero false alarms.
 */
turbofft_status turbofft_set_threshold_scale(turbofft_plan *plan, double factor);

/*
 * Transactions per checksum group (Sec. 4.3: a thread block verifies its
 * checksums once per `transactions` transactions; 1 = every transaction, the
 * thread-block-level scheme without amortisation).  Default 4, range
 * [1, 16]; for the ablation of the group size (overhead vs. the
 * single-error-per-group fault model).  Errors: INVALID_VALUE.
 */
turbofft_status turbofft_set_group_transactions(turbofft_plan *plan, int transactions);

/*
 * Place the intermediate buffer of a two-pass plan in caller-owned device
 * memory (`bytes` >= info.scratch_bytes, 16-byte aligned) instead of the
 * plan allocating it at its first exec.  Plans that never run at the same
 * time on the GPU may share one workspace.  The caller keeps ownership and
 * must keep it alive while the plan may run.  A one-pass plan ignores the
 * call.  Errors: INVALID_VALUE (NULL, too small, misaligned).
 */
turbofft_status turbofft_set_workspace(turbofft_plan *plan, void *workspace, size_t bytes);

/*
 * Record a CUDA event pair around every kernel of each following exec (on
 * the exec's stream) when enable != 0.  turbofft_get_kernel_times waits for
 * the last exec and returns up to `capacity` durations in launch order;
 * *count receives how many were written.
 */
turbofft_status turbofft_set_profiling(turbofft_plan *plan, int enable);
turbofft_status turbofft_get_kernel_times(turbofft_plan *plan, turbofft_kernel_time *out,
                                          int capacity, int *count);

/*
 * No counterpart in the paper: a library facility, not part of the method.
 *
 * turbofft_exec without any device allocation, for callers that create
 * their plans ahead of time but cannot call cudaMalloc (or any allocating
 * routine) when they transform -- e.g. a program whose device memory belongs
 * to another allocator that hands out no raw buffers, or one running under a
 * device-memory budget fixed at start-up.  A two-pass plan's intermediate
 * (info.scratch_bytes) is placed in a file-scope device array of
 * TURBOFFT_STATIC_SCRATCH_BYTES that the library keeps on every GPU where
 * this part of it is loaded, until the process exits; one-pass plans need
 * no intermediate.  Same results as turbofft_exec.
 *   - Plans needing more than TURBOFFT_STATIC_SCRATCH_BYTES are rejected with
 *     TURBOFFT_INVALID_VALUE (message in turbofft_last_error); nothing runs.
 *   - The first call on a device looks up the array's device address (with
 *     that device current).  Under CUDA's lazy module loading that lookup
 *     loads the part of the library that holds the array, and the 32 MiB is
 *     reserved on the device then, not when the library is opened.  So make
 *     the first call during set-up: before the device-memory budget is fixed
 *     and before any stream capture.  Later calls allocate nothing.
 *   - All calls on a device share the array: calls whose kernels may overlap
 *     on the GPU (e.g. on unordered streams) race on it.  Its contents carry
 *     over between calls and need no clearing: every element is written
 *     before it is read within one call.
 *   - in, out, stream: as turbofft_exec.
 */
#define TURBOFFT_STATIC_SCRATCH_BYTES (32u << 20)
/* The array size this library was built with (TURBOFFT_STATIC_SCRATCH_BYTES),
 * for callers that load the library without its header. */
extern const uint64_t turbofft_static_scratch_bytes;
turbofft_status turbofft_exec_static_scratch(turbofft_plan *plan, const void *in, void *out,
                                             turbofft_stream stream);

/*
 * No counterpart in the paper: a calibration call for roofline figures.
 *
 * Measured fused multiply-add rate of the current device in the arithmetic
 * of `dtype` (F32: float FMA, F64: double FMA), 2 flops per FMA: a loop of
 * independent FMA chains over every SM, timed with CUDA events on `stream`
 * for about `seconds` (0 < seconds <= 60) of launches of ~50 ms; the best
 * launch's rate is written to *tflops (TFLOP/s).  Synchronous.  The float64
 * transforms are bound by this rate on GPUs whose FP64 pipe is narrow.
 * Errors: INVALID_VALUE (bad dtype, seconds or NULL tflops), CUDA_ERROR.
 */
turbofft_status turbofft_fma_peak(turbofft_dtype dtype, double seconds, turbofft_stream stream,
                                  double *tflops);

/* Free everything the plan owns.  NULL is a no-op.  Waits for the plan's
 * outstanding work first. */
turbofft_status turbofft_destroy(turbofft_plan *plan);

/* Static, human-readable name of a status code. */
const char *turbofft_status_string(turbofft_status status);

/* Text of the last CUDA error seen by this plan ("" if none). */
const char *turbofft_last_error(const turbofft_plan *plan);

#ifdef __cplusplus
}
#endif

#endif /* TURBOFFT_H */
