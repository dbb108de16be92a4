/*
 * moa_fft.h -- C ABI of the GB300 MoA reshape-transpose FFT library
 * (libmoafft.so).
 *
 * Problem statement (Hunt, Mullin, Rosenkrantz, Raynolds, "A
 * transformation-based approach for the design of parallel/distributed
 * scientific software: the FFT", Fig. 2.1): input x in C^n with n = 2^t,
 * t >= 1; output the FFT of x.  This library computes, for exponent sign s,
 *
 *     X[k] = sum_{j=0}^{n-1} x[j] * exp(s * 2*pi*i * j*k / n),
 *
 * unnormalised in both directions (forward then inverse multiplies by n).
 * The multi-dimensional transform is the 1-D transform applied along every
 * axis (the Omega operator, Appendix B, Eq. B.6) of a row-major array (the
 * gamma ordering, Appendix A, Definition A.1); the last axis is contiguous
 * and the batch index is outermost.  Large 1-D sizes use the paper's
 * dimension lifting n = r*c (Sec. 4.2-4.8, Fig. 4.9): r-point column
 * transforms, twiddle, c-point row transforms, transposed store.
 *
 * Data: complex64, i.e. interleaved (re, im) IEEE binary32 pairs.
 *
 * Ownership and memory:
 *   - A plan is an opaque handle owned by the library.  It owns its twiddle
 *     tables, its workspace and its device status word; moa_fft_destroy
 *     frees them.  Plans are not thread-safe: one host thread at a time may
 *     use a plan.
 *   - `in` and `out` are caller-owned DEVICE pointers, 8-byte aligned
 *     (16-byte recommended), each holding at least batch * prod(n) complex64
 *     values (for a batched-uneven plan: sum(lengths)).  in == out
 *     (in-place) is allowed; any other overlap is undefined.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Execution is asynchronous on that stream: exec never
 *     synchronises, never allocates and may be captured in a CUDA graph.
 *
 * Errors: every entry point returns a moa_status_t.  Argument checks happen
 * on the host before any CUDA call, so they work without a GPU.  A kernel
 * that detects a fault on the device records it in the plan's status word;
 * read it with moa_fft_status after synchronising the stream.
 */
#ifndef MOA_FFT_H
#define MOA_FFT_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define MOA_API __attribute__((visibility("default")))
#else
#define MOA_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct moa_fft_plan_s *moa_fft_plan_t;

typedef enum {
    MOA_C64 = 0,          /* plain FP32 complex64 arithmetic */
    MOA_C64_TC_FP16 = 1,  /* complex64 I/O, radix-16 DFT blocks on FP16 tensor cores: operands split
                             hi + lo, three products, FP32 accumulate, power-of-two scaling per stage */
    MOA_C64_TC_BF16 = 2   /* complex64 I/O, radix-16 DFT blocks on BF16 tensor cores: operands split
                             hi + mid + lo, six products, FP32 accumulate */
} moa_dtype_t;

typedef enum {
    MOA_OK = 0,
    MOA_ERR_INVALID_ARG = 1,   /* NULL pointer, bad sign/dims/batch, dead plan handle */
    MOA_ERR_INVALID_SIZE = 2,  /* a length that is not a power of two >= 2 */
    MOA_ERR_UNSUPPORTED = 3,   /* valid request this build does not implement */
    MOA_ERR_ALLOC = 4,         /* device or host allocation failed */
    MOA_ERR_CUDA = 5,          /* a CUDA runtime call failed (no device, launch error) */
    MOA_ERR_TIMEOUT = 6        /* a bounded device-side wait gave up */
} moa_status_t;

/* Create a plan for `batch` transforms of shape n[0..dims-1].
 *   n      : dims lengths, each a power of two >= 2 (t >= 1, Fig. 2.1).
 *            1-D: n[0] <= 2^30 (up to 2^24 in two passes, n = r*c
 *            with r, c <= 4096; beyond, three passes, n = r1*r2*c).
 *            2-D/3-D: every n[i] <= 2^24 (an axis above 4096 is lifted
 *            L = L1*L2 inside the array, two passes for that axis, and the
 *            plan then uses a workspace of the array's size).
 *   dims   : 1, 2 or 3.
 *   batch  : >= 1; batch * prod(n) < 2^31.
 *   sign   : -1 (forward, exp(-2 pi i jk/n)) or +1.
 *   dtype  : a moa_dtype_t value.  MOA_C64: every shape above.  The two
 *            tensor-core values: 1-D with n[0] = 256 or 4096 (any batch),
 *            else MOA_ERR_UNSUPPORTED; relative L2 error <= 1e-5 per
 *            transform against the exact DFT.
 * Builds the pass sequence, generates the twiddle tables in FP64 on the
 * device (rounded once to FP32) and allocates the workspace; synchronises
 * the device once.  On failure *plan is set to NULL. */
MOA_API moa_status_t moa_fft_plan(moa_fft_plan_t *plan, const int64_t *n, int dims, int64_t batch,
                          int sign, int dtype);

/* Create a plan for `count` independent 1-D transforms of uneven lengths
 * lengths[0..count-1] (each a power of two in [2, 65536]).  Transform i
 * reads and writes the contiguous block starting at element
 * sum_{j<i} lengths[j] of `in` / `out`.  All transforms run in one
 * persistent launch fed by a device work queue.  dtype must be MOA_C64
 * (the tensor-core values give MOA_ERR_UNSUPPORTED). */
MOA_API moa_status_t moa_fft_plan_batched(moa_fft_plan_t *plan, const int64_t *lengths, int64_t count,
                                  int sign, int dtype);

/* Run the planned transform (sign as planned) from `in` to `out` on
 * `stream`.  Asynchronous; no allocation; capturable.  Stream order holds:
 * a pass may be launched as a programmatic dependent launch of the kernel
 * before it in the stream (the caller's included), so its blocks can become
 * resident while that kernel finishes, but they wait on the device for it to
 * complete before reading or writing any buffer (MOA_PDL=0 in the
 * environment turns this off). */
MOA_API moa_status_t moa_fft_exec(moa_fft_plan_t plan, const void *in, void *out, void *stream);

/* Run the adjoint of the planned transform: the unnormalised transform of
 * the opposite sign (F^H = conj(F)^T = F with -sign), on the same plan. */
MOA_API moa_status_t moa_fft_exec_adjoint(moa_fft_plan_t plan, const void *in, void *out, void *stream);

/* Run only pass `index` (0 <= index < passes, see moa_fft_plan_info) of the
 * planned transform with exponent sign `sign` (-1 or +1).  Running passes
 * 0..passes-1 in order on one stream with the same (in, out) is exactly
 * moa_fft_exec (sign = planned) or moa_fft_exec_adjoint (sign = -planned).
 * Intended for instrumentation: it lets a caller time each kernel launch
 * with CUDA events on its own stream. */
MOA_API moa_status_t moa_fft_exec_pass(moa_fft_plan_t plan, int index, int sign, const void *in, void *out,
                                       void *stream);

/* End-to-end call for host data: copies `host_in` (pinned host memory
 * recommended) to the caller's device buffer `dev_buf`, runs the transform
 * in place there and copies the result to `host_out`, all on `stream`.
 * Returns after enqueueing; synchronise the stream before reading
 * host_out. */
MOA_API moa_status_t moa_fft_exec_host(moa_fft_plan_t plan, const void *host_in, void *host_out,
                               void *dev_buf, void *stream);

/* Allocation-free 1-D transform, for callers that cannot allocate device
 * memory (a custom allocator owns all of it, or the calling path must never
 * enter the CUDA allocator).  The paper has no counterpart: this is a
 * deployment variant of moa_fft_exec with no plan.
 *   in, out : caller-owned device pointers to n complex64 values, 8-byte
 *             aligned; in == out allowed.
 *   n       : power of two, 2 <= n <= 2^20 (1,048,576).  Larger n returns
 *             MOA_ERR_UNSUPPORTED: the transform's scratch lives in a fixed
 *             8 MiB static device array.
 *   sign    : -1 or +1, as for moa_fft_plan.  stream: cudaStream_t or NULL.
 * Same kernels and results as a plan with batch 1.  Nothing is allocated:
 * the scratch and the twiddle tables (about 8.3 MiB in all) are static
 * device arrays that every GPU using this library holds until the process
 * exits.  The first call on a device sets them up (symbol lookup, twiddle
 * generation) and synchronises `stream` once: make that first call before
 * any stream capture.  All calls on a device share the arrays; calls that
 * overlap on the GPU race and must be serialised by the caller.  A kernel
 * whose bounded wait gives up records MOA_ERR_TIMEOUT in the device's status
 * word (the output is then incomplete); read it with
 * moa_fft_noalloc_status.  Each call looks up the scratch array's address
 * again (a host-side lookup) and repeats the set-up if the device's context
 * was made again since (cudaDeviceReset). */
MOA_API moa_status_t moa_fft_exec_noalloc(const void *in, void *out, int64_t n, int sign, void *stream);

/* Status word of moa_fft_exec_noalloc on the current device: MOA_OK, or the
 * first error a kernel recorded since the word was last read (for instance
 * MOA_ERR_TIMEOUT).  The paper has no counterpart.  The word is copied to
 * the host after the work already queued on `stream` (cudaStream_t or
 * NULL), then reset to MOA_OK; the call synchronises `stream` and allocates
 * nothing.  MOA_ERR_CUDA if the copy fails.  Before any transform on the
 * device it runs the same one-time set-up as moa_fft_exec_noalloc. */
MOA_API moa_status_t moa_fft_noalloc_status(void *stream);

/* Device status word of the plan (MOA_OK or the first error a kernel
 * recorded), read with a synchronous copy; the word is then reset to
 * MOA_OK. */
MOA_API moa_status_t moa_fft_status(moa_fft_plan_t plan);

/* Static, NUL-terminated description of a status code. */
MOA_API const char *moa_fft_error_string(moa_status_t status);

/* Describe the plan: number of kernel passes per exec, the r x c split of a
 * lifted 1-D transform (0 when none) and the workspace size in bytes. Any
 * output pointer may be NULL. */
MOA_API moa_status_t moa_fft_plan_info(moa_fft_plan_t plan, int *passes, int64_t *split_r,
                               int64_t *split_c, size_t *workspace_bytes);

/* What the plan chose and why: the r x c split, the tile size of the
 * generic passes and the kernels of every pass (for a batched plan, the
 * split offset of each large length), then where the choice came from
 * (defaults or environment overrides, the autotuner, or its cache), written
 * NUL-terminated into text[0..text_len-1] (truncated if needed).
 * Instrumentation, so that a benchmark can state which candidate won. */
MOA_API moa_status_t moa_fft_plan_choice(moa_fft_plan_t plan, char *text, size_t text_len);

/* Describe pass `index` of the plan (0 <= index < passes): the name of the
 * kernel it launches, written NUL-terminated into name[0..name_len-1]
 * (truncated if needed; name may be NULL when name_len is 0), and its
 * algorithmic HBM bytes per exec (complex64 elements read plus written, 8
 * bytes each).  Instrumentation for per-kernel roofline reports. */
MOA_API moa_status_t moa_fft_pass_info(moa_fft_plan_t plan, int index, char *name, size_t name_len,
                                       int64_t *bytes);

/* Host-only description of the work queue moa_fft_plan_batched builds for
 * `lengths` (default split, autotuner off; MOA_BATCH_LOG2R applies), without
 * a GPU.  The persistent blocks of the batched launch take the tasks in
 * this order (Sec. 4.3: many problems sharing the processors).
 *   lengths, count : as for moa_fft_plan_batched (same checks and codes).
 *   resident : blocks that run at once (the plan uses SMs x blocks per SM,
 *              3 x 152 on GB300); a transform's row tiles are queued about
 *              this many column tiles after its last column tile.
 *   order    : NULL or `count` entries; order[k] = index in `lengths` of the
 *              k-th transform in the plan's grouping (longest first, then
 *              input order).
 *   tasks    : 6 int32 per task, in queue order: {first, count, tile,
 *              log2 n, log2 r, kind}.  kind 0: `count` transforms of 2^log2n
 *              <= 4096 points at grouping positions first .. first+count-1,
 *              each in one block; kind 1 / 2: column / row tile `tile` of the
 *              lifted transform at position `first` (2^log2n = r*c points,
 *              r = 2^log2r, 2^(log2n - 12) tiles of each kind).  A row tile
 *              waits for all column tiles of its transform; column tiles never
 *              wait.  NULL with capacity 0 only reports *ntasks.
 *   capacity : tasks room, in tasks; ntasks receives the queue length.
 * MOA_ERR_INVALID_ARG for resident < 1, capacity below the length or a NULL
 * tasks buffer with capacity > 0. */
MOA_API moa_status_t moa_fft_batched_queue(const int64_t *lengths, int64_t count, int64_t resident,
                                           int64_t *order, int32_t *tasks, int64_t capacity,
                                           int64_t *ntasks);

/* Copy one of the plan's twiddle tables to host memory, for tests and
 * diagnostics: each entry is w_M^e = exp(-2 pi i e / M) evaluated once in
 * FP64 on the device (exact reduction e mod M, Fig. 3.8: weights computed
 * directly, not by recurrence) and rounded once to complex64.
 *   table 0: the stage table of the 2^index-point in-register transform
 *            (index 1..12, present when a pass of the plan uses it and it
 *            is not empty): for every radix stage s but the last, six rows
 *            k = 1, 2, 3, 4, 8, 12 of w_M^(u*k), u < M1 (M the stage's
 *            span, M1 = M / radix), row after row, stage after stage;
 *   table 1: lo[i] = w_n^i, i < 2^h, and
 *   table 2: hi[j] = w_n^(j * 2^h), j < n / 2^h: the two halves of the
 *            four-step twiddle w_n^e = lo[e mod 2^h] * hi[e / 2^h] of a
 *            lifted 1-D plan of length n (present when the plan lifts);
 *   table 3, 4: the stage table (layout of table 0) of the 2^index-point
 *            transform in radix schedule 1 (radix 16 with the small radix
 *            last) or 2 (radix-8 stages), present when a generic pass of
 *            the plan runs that schedule (Sec. 4.8: any factorisation of the
 *            in-register stages gives the same transform; the autotuner, or
 *            MOA_SCHED, picks one);
 *   table 5: the table of the warp-shuffle row kernel of 2^index points
 *            (index 7..9, N = 2^index, T = N/16): rows k = 1, 2, 3, 4, 8, 12
 *            of w_N^(u*k), u < T, then w_T^u, u < T.
 *   host_out : caller-owned host memory of `capacity` complex64 entries;
 *              NULL with capacity 0 only reports *entries.
 *   entries  : receives the table's length (may be NULL).
 * Synchronous.  MOA_ERR_INVALID_ARG for a dead or batched plan, a table the
 * plan does not hold, or capacity below the length. */
MOA_API moa_status_t moa_fft_plan_table(moa_fft_plan_t plan, int table, int index, void *host_out,
                                        int64_t capacity, int64_t *entries);

/* Host-only estimate of the plan moa_fft_plan would build for the same
 * request with the autotuner off (MOA_AUTOTUNE=0): the passes (the dimension
 * lifting n = r*c of Sec. 4.2 for a 1-D transform, the r x c split chosen as
 * the breakpoint of Sec. 4.8; one pass per axis, Eq. B.6, or the two-pass
 * 256^3 form for multi-D), the kernel each pass launches and the workspace
 * size, without touching the GPU and without allocating device memory.  The
 * environment overrides the plan reads (MOA_SPLIT_LOG2R, MOA_PIPE,
 * MOA_LIFT3, MOA_3D_TWO_PASS, MOA_TC_KERNEL, MOA_SCHED: radix schedule of
 * the generic passes, 0..3 as in moa_fft_plan_table) apply here too.
 *   n, dims, batch, dtype : as for moa_fft_plan (same checks, same error
 *                           codes; the sign does not change the plan).
 *   tma    : 1 = assume the driver's tensor-map encoder is present (the
 *            pipelined TMA kernels may be chosen, as on any GB300 driver),
 *            0 = assume it is absent (generic kernels only), -1 = ask the
 *            driver.
 *   passes, split_r, split_c, workspace_bytes : as moa_fft_plan_info
 *            reports them; any may be NULL.
 *   kernels: the kernel names of the passes, in order, separated by ';'
 *            (the names moa_fft_pass_info reports), NUL-terminated and
 *            truncated to kernels_len - 1 characters; may be NULL when
 *            kernels_len is 0.
 * Returns MOA_ERR_INVALID_ARG for tma outside {-1, 0, 1} or a NULL kernels
 * buffer with kernels_len > 0. */
MOA_API moa_status_t moa_fft_estimate(const int64_t *n, int dims, int64_t batch, int dtype, int tma,
                                      int *passes, int64_t *split_r, int64_t *split_c,
                                      size_t *workspace_bytes, char *kernels, size_t kernels_len);

/* Destroy a plan and free everything it owns.  NULL is a no-op (MOA_OK);
 * a handle that is not a live plan returns MOA_ERR_INVALID_ARG. */
MOA_API moa_status_t moa_fft_destroy(moa_fft_plan_t plan);

#ifdef __cplusplus
}
#endif

#endif /* MOA_FFT_H */
