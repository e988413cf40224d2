/*
 * fft3d — transpose-free 3D real-to-complex FFT and its complex-to-real
 * inverse for one NVIDIA GB300 (sm_103a).
 *
 * Method: Chatterjee, Verma & Chaudhuri, "Transpose-free Fast Fourier
 * Transform for Turbulence Simulation", arXiv:1406.5597.  Sec. 2 defines the
 * operation (a real n0 x n1 x n2 array to the complex n0 x n1 x H half
 * spectrum and back); Sec. 2.1 gives the steps (a 2D r2c per n0-plane, then a
 * 1D c2c along n0; the inverse in reverse order); Sec. 2.2 replaces the
 * transpose of step 2 by transforming the n0 axis where it lies, at its
 * natural stride.  On one GPU this library never materialises a transposed
 * copy: the n0 pass reads and writes the spectrum in place at stride
 * n1*(n2/2+1) complex elements.
 *
 * Conventions (the paper names FFTW's transforms, Sec. 3, and fixes neither
 * sign nor scaling; this library takes FFTW's):
 *   forward  X[k] = sum_j x[j] exp(-2 pi i (k0 j0/n0 + k1 j1/n1 + k2 j2/n2)),
 *            0 <= k2 < H, H = floor(n2/2) + 1;
 *   inverse  y[j] = sum_{k2=0}^{H-1} c_k2 Re(sum_{k0,k1} Y[k] exp(+2 pi i (...))),
 *            c_k2 = 1 at k2 = 0 and, for even n2 only, at the Nyquist bin
 *            k2 = n2/2; c_k2 = 2 for every other bin (for odd n2 there is no
 *            Nyquist bin, so every k2 >= 1 weighs 2); unnormalised, so
 *            c2r(r2c(x)) = n0*n1*n2 * x.  The imaginary part of the k2 = 0
 *            bin, and for even n2 of the k2 = n2/2 bin, after the n0 and n1
 *            passes, is ignored.
 *
 * Layouts: real data batch x n0 x n1 x n2 contiguous float; complex data
 * batch x n0 x n1 x H (H = floor(n2/2) + 1) contiguous interleaved float pairs
 * (float2, torch.complex64).  C row-major, n2 fastest, batch outermost.
 * All data pointers are DEVICE pointers unless a comment says otherwise.
 *
 * Ownership: the caller owns every data buffer.  A plan owns its small
 * twiddle tables and a device status word (allocated at plan time, freed by
 * fft3d_destroy); an FP32 plan whose n0 axis is 1024, 1536 or 2048 long
 * (and n1*(n2/2+1) even) also owns the scratch of the residue-split n0
 * kernel (column form 5): (C - 1) x 64 KB per SM for L = 512 C, 10 to 30 MB.
 * Large workspace, where a variant needs it, is lent by the caller through
 * fft3d_set_workspace.
 *
 * Streams: every launch goes on the stream passed in (a cudaStream_t given
 * as void*; NULL means the legacy default stream).  Nothing synchronises
 * implicitly except fft3d_plan*, fft3d_destroy and fft3d_query_device_status.
 * Calls on one plan from several host threads or streams may overlap (its
 * host-side caches are locked) unless the plan uses memory shared between
 * calls: the scratch of column form 5 or a caller workspace.  Such calls must
 * be ordered on the GPU (for instance, issued on one stream).
 *
 * Errors: functions returning int return an fft3d_status.  Argument errors
 * are found before any launch and leave the output untouched.  The status of
 * the last failing call on the calling thread is kept for fft3d_last_error.
 *
 * Tracing and environment: every pass is enclosed in an NVTX range named for
 * the pass ("row_r2c", "col_n1_fwd", "col_n0_fwd", ...; see fft3d_pass_name)
 * around its launch.  FFT3D_LOG=1 prints each plan's kernel choices and each
 * autotune result on stderr.  FFT3D_FORCE_PASSES (a test and benchmark
 * override, read at every plan creation) ORs forms into the flags of every
 * FP32 plan: a comma-separated list of "three", "generic", "fused", "cluster",
 * "transpose", "transpose_back" (the FFT3D_FLAG_* forms of the same names).
 */
#ifndef FFT3D_H
#define FFT3D_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fft3d_plan_s* fft3d_handle;

/* Arithmetic forms.  Storage is FP32 in the first three (fft3d_r2c / fft3d_c2r)
 * and FP64 in the last (fft3d_r2c_f64 / fft3d_c2r_f64). */
typedef enum {
    FFT3D_F32 = 0,            /* plain FP32 butterflies on the CUDA cores */
    FFT3D_F32_TC_BF16X3 = 1,  /* radix-16 stages as tensor-core contractions, split-BF16 (3 products) */
    FFT3D_F32_TC_F16 = 2,     /* radix-16 stages as tensor-core contractions, single-term FP16 */
    FFT3D_F64 = 3             /* FP64 data and arithmetic, runtime-length kernels (flags must be 0) */
} fft3d_dtype;

typedef enum {
    FFT3D_OK = 0,
    FFT3D_ERR_INVALID_ARG = 1,      /* NULL/overlapping pointers, bad enum, n < 1, batch < 1 */
    FFT3D_ERR_UNSUPPORTED_SIZE = 2, /* an axis or row transform longer than 4096, or a form not offered at this size */
    FFT3D_ERR_MISALIGNED = 3,       /* a data pointer not 16-byte aligned */
    FFT3D_ERR_ALLOC = 4,            /* plan-time device allocation failed */
    FFT3D_ERR_CUDA = 5,             /* a CUDA call or launch failed */
    FFT3D_ERR_TIMEOUT = 6,          /* a bounded device-side wait gave up (see fft3d_query_device_status) */
    FFT3D_ERR_NO_WORKSPACE = 7      /* the variant needs caller workspace and none was set */
} fft3d_status;

/* Plan flags for fft3d_plan_variant. */
#define FFT3D_FLAG_EXPLICIT_TRANSPOSE 0x1 /* comparator: materialise the n0<->n1 transpose (Sec. 2.1, step 2) */
#define FFT3D_FLAG_TRANSPOSE_BACK 0x2     /* with EXPLICIT_TRANSPOSE: transpose back to n0 x n1 x H */
#define FFT3D_FLAG_THREE_PASS 0x4         /* separate n2-row, n1-column and n0-column passes (the default;
                                             overrides FFT3D_FLAG_FUSED_PLANE) */
#define FFT3D_FLAG_GENERIC 0x8            /* force the runtime-length kernels (testing) */
#define FFT3D_FLAG_FUSED_PLANE 0x20       /* fuse the n2-row and n1-column passes into one persistent
                                             kernel that keeps each plane in L2 between its halves
                                             (DRAM traffic of two passes; shapes with an instantiated
                                             fused kernel only, else ignored) */
#define FFT3D_FLAG_CLUSTER_PLANE 0x40     /* fuse the n2-row and n1-column passes into one kernel that holds
                                             each plane in the distributed shared memory of a thread-block
                                             cluster (DRAM traffic of two passes; shapes with an
                                             instantiated cluster kernel only, else ignored) */
#define FFT3D_FLAG_PADDED_REAL 0x80      /* real rows padded to 2*(n2/2+1) floats (FFTW's in-place layout: the
                                             real array is batch x n0 x n1 x (n2+2) floats, the last two of
                                             each row unused); fft3d_r2c / fft3d_c2r then also accept
                                             in == out (the transform in place) */
#define FFT3D_FLAG_PRESERVE_INPUT 0x100   /* fft3d_c2r leaves its input unchanged: its first column pass writes
                                             into caller workspace (fft3d_workspace_bytes: batch*M complex)
                                             and the rest runs there */
#define FFT3D_FLAG_TEST_SKIP_ARRIVAL 0x10 /* testing only (with FUSED_PLANE): in the fused plane kernel the producers of
                                             plane 0 never report, so its consumers' bounded waits give
                                             up after about a millisecond; the call's output is then
                                             undefined and fft3d_query_device_status returns
                                             FFT3D_ERR_TIMEOUT */

/*
 * Create a plan for batch transforms of size n0 x n1 x n2 (Sec. 2).
 * Requirements: n0, n1 >= 1, n2 >= 2, no transform longer than 4096 (n0, n1
 * and the row transform length: n2/2 for even n2, n2 for odd n2),
 * H = floor(n2/2) + 1 (no Nyquist bin for odd n2), batch >= 1, and a current
 * CUDA device.  Lengths with compile-time kernels run those; other lengths whose
 * prime factors are 2, 3, 5 and 7 (and odd n2) run the runtime-radix kernels;
 * a length with any larger prime factor runs Bluestein's chirp-z form (two
 * power-of-two transforms of length M >= 2L - 1 around a pointwise product; its
 * chirp tables are computed in FP64 and take (L + 2M) x 8 bytes of device
 * memory).  Chooses the passes and the kernel shapes, computes twiddle tables in
 * FP64 on the host, rounds them to FP32 and copies them to the device.  Blocks.
 * Returns NULL on error (reason in fft3d_last_error()).
 */
fft3d_handle fft3d_plan(int n0, int n1, int n2, int dtype, int batch);

/* As fft3d_plan, with FFT3D_FLAG_* flags. */
fft3d_handle fft3d_plan_variant(int n0, int n1, int n2, int dtype, int batch, int flags);

/*
 * Forward r2c (Sec. 2; steps of Sec. 2.1 with the n0 pass of Sec. 2.2).
 * in:  batch*n0*n1*n2 floats (device), read only; batch*n0*n1*(n2+2) floats
 *      (rows padded to 2H) for FFT3D_FLAG_PADDED_REAL plans.
 * out: batch*n0*n1*H float2 (device); must not overlap in, except that a
 *      PADDED_REAL plan accepts out == in (in place, FFTW's layout).
 * For FFT3D_FLAG_EXPLICIT_TRANSPOSE plans without TRANSPOSE_BACK the result
 * is laid out batch x n1 x n0 x H ("axes 0 and 1 flipped", Sec. 2.1).
 * Both pointers 16-byte aligned.  Asynchronous on stream.
 */
int fft3d_r2c(fft3d_handle plan, const float* in, void* out, void* stream);

/*
 * Inverse c2r (Sec. 2; the forward steps in reverse order, Sec. 2.1).
 * in:  batch*n0*n1*H float2 (device); CLOBBERED (used as scratch, as FFTW's
 *      multi-dimensional c2r does) unless the plan has
 *      FFT3D_FLAG_PRESERVE_INPUT (then read only; the plan needs workspace of
 *      fft3d_workspace_bytes, which must not overlap in, else
 *      FFT3D_ERR_NO_WORKSPACE / FFT3D_ERR_INVALID_ARG).  For EXPLICIT_TRANSPOSE
 *      plans without TRANSPOSE_BACK it is read in the transposed
 *      batch x n1 x n0 x H layout.
 * out: batch*n0*n1*n2 floats (device), or batch*n0*n1*(n2+2) (rows padded to
 *      2H, the last two floats of a row untouched) for PADDED_REAL plans; must
 *      not overlap in, except that a PADDED_REAL plan without PRESERVE_INPUT
 *      accepts out == in (in place).
 * Unnormalised.  Asynchronous on stream.
 */
int fft3d_c2r(fft3d_handle plan, void* in, float* out, void* stream);

/*
 * FP64 forward r2c and inverse c2r, for FFT3D_F64 plans only (other plans, and
 * FFT3D_F64 plans passed to fft3d_r2c / fft3d_c2r, give FFT3D_ERR_INVALID_ARG).
 * Same transforms, pass sequence and layouts as fft3d_r2c / fft3d_c2r with
 * flags 0, in double precision: every pass runs the runtime-length kernels
 * (Stockham stages of radix 2..8, Bluestein for other primes) with twiddle and
 * chirp tables computed and kept in FP64.  An FFT3D_F64 plan accepts lengths up
 * to 4096, except that a length with a prime factor above 7 must be <= 2048 (its
 * Bluestein line of 4096 double2 points fills one CTA's shared memory).
 * r2c  in:  batch*n0*n1*n2 doubles (device), read only.
 *      out: batch*n0*n1*H double2 (interleaved re, im; device), must not overlap in.
 * c2r  in:  batch*n0*n1*H double2 (device), CLOBBERED (scratch, as in fft3d_c2r).
 *      out: batch*n0*n1*n2 doubles (device), must not overlap in.  Unnormalised.
 * Both pointers 16-byte aligned.  Asynchronous on stream.
 */
int fft3d_r2c_f64(fft3d_handle plan, const double* in, void* out, void* stream);
int fft3d_c2r_f64(fft3d_handle plan, void* in, double* out, void* stream);

/* Release a plan's device tables.  NULL-safe.  Blocks on the device. */
void fft3d_destroy(fft3d_handle plan);

/* Status of the last failing call on this thread (FFT3D_OK if none). */
int fft3d_last_error(void);

/* Static text for a status code. */
const char* fft3d_error_string(int status);

/*
 * Synchronise stream, then read and clear the plan's device status word.
 * Returns FFT3D_OK, FFT3D_ERR_TIMEOUT if a bounded device wait gave up, or
 * FFT3D_ERR_CUDA.
 */
int fft3d_query_device_status(fft3d_handle plan, void* stream);

/* Bytes of caller workspace the plan needs (0 when none). */
size_t fft3d_workspace_bytes(fft3d_handle plan);

/* Lend the plan a device buffer of at least fft3d_workspace_bytes(plan)
 * bytes, 256-byte aligned; the caller keeps ownership and must keep it
 * alive while work using the plan is in flight.  NULL detaches. */
int fft3d_set_workspace(fft3d_handle plan, void* dev_ptr);

/* Plan description for logs: writes a NUL-terminated text of at most len
 * bytes (host buffer) naming the passes and kernel shapes. */
int fft3d_describe(fft3d_handle plan, char* text, int len);

/* Number of kernel launches one fft3d_r2c (dir = -1) or fft3d_c2r (dir = +1)
 * call issues with this plan. */
int fft3d_launches_per_call(fft3d_handle plan, int dir);

/*
 * Per-pass timing (tracing).  While enabled, every kernel launch made by
 * fft3d_r2c / fft3d_c2r is bracketed by two CUDA events recorded on the
 * launch stream (not for use under stream capture).
 */
int fft3d_set_profiling(fft3d_handle plan, int enable);

/* Wait for the recorded events, then write per-pass totals since the last
 * read into the HOST arrays ms[i] (milliseconds) and count[i] (launches) for
 * pass ids i < n, and reset.  Pass ids are listed by fft3d_pass_name. */
int fft3d_profile_read(fft3d_handle plan, double* ms, int* count, int n);

/* Static name of pass id i ("row_r2c", "col_n1_fwd", "col_n0_fwd",
 * "col_n0_inv", "col_n1_inv", "row_c2r", "swap01", "plane_fwd", "plane_inv");
 * NULL past the last id. */
const char* fft3d_pass_name(int pass);

/* Algorithmic bytes one launch of pass id i moves with this plan: one read
 * plus one write of the data it transforms (4 bytes per real and 8 per complex
 * value).  Returns 0 for an unknown id. */
double fft3d_pass_bytes(fft3d_handle plan, int pass);

/*
 * Autotuning.  A plan's kernel shapes (columns per CTA of the n0 and n1
 * column kernels, rows per CTA of the row kernels, and the kernel form of the
 * n0 and the n1 pass) start at compiled defaults; fft3d_autotune times each
 * pass's candidates on the caller's buffers (real: batch*N floats, cplx:
 * batch*M float2; both device, contents destroyed) with CUDA events, reps
 * timed runs per candidate, and keeps the fastest.  Synchronises stream.  The
 * choices are five ints {w0, w1, rows, form0, form1} (widths/rows 0 = compiled
 * default; forms: 0 plain one-tile-per-CTA kernel, 1 TMA-fed persistent
 * kernel, 2 and 3 the first and second cluster-split kernel compiled for that
 * axis length, 4 the TMA-fed cluster split (lengths 1024, 1536, 2048: 512-row
 * TMA sub-transforms on 2, 3 or 4 CTAs; it needs an even axis stride of at
 * least 16 complex values and otherwise runs as form 0), 5 the residue split
 * through L2 (same lengths: one CTA per tile, the 512-row residues parked in
 * plan-owned scratch; on an odd axis stride, as the n1 pass with odd n2/2 + 1,
 * the odd residues read through maps started one value early), 6 (lengths
 * 1024 and 2048, odd axis stride) the TMA row-pair kernel with two columns
 * per thread and 16-byte shared and even-row global accesses (on an even
 * stride it runs as form 1), where one exists)
 * that fft3d_get_choices / fft3d_set_choices
 * read and write (host array), so a caller can cache them per GPU and shape;
 * fft3d_set_choices rejects a form the axis does not have.
 * FFT3D_F64 plans have nothing to tune: FFT3D_ERR_INVALID_ARG.
 */
int fft3d_autotune(fft3d_handle plan, float* real, void* cplx, int reps, void* stream);
int fft3d_get_choices(fft3d_handle plan, int* choices5);
int fft3d_set_choices(fft3d_handle plan, const int* choices5);

/*
 * Plane form (the 2D transform of every n0-plane, Sec. 2.1 step 1): 0 = a
 * row pass and an n1 column pass; C > 0 = one cluster plane pass that holds
 * each plane in the shared memory of a C-CTA thread-block cluster (C = 1: one
 * CTA).  fft3d_autotune (plans without FFT3D_FLAG_THREE_PASS, _GENERIC,
 * _EXPLICIT_TRANSPOSE, _FUSED_PLANE, FP32) times both forms over a whole
 * r2c + c2r, every instantiated cluster size of the shape, and keeps the
 * fastest.  fft3d_get_plane_choice returns the plan's current C (>= 0), or
 * minus the status on error.  fft3d_set_plane_choice sets it: 0 always works;
 * C > 0 needs an instantiated cluster kernel of the plan's (n2/2, n1) with that
 * cluster size (else FFT3D_ERR_UNSUPPORTED_SIZE, plan unchanged) and a plan
 * the form applies to (else FFT3D_ERR_INVALID_ARG).  Host only; set it before
 * the plan's first use in a captured graph.
 */
int fft3d_get_plane_choice(fft3d_handle plan);
int fft3d_set_plane_choice(fft3d_handle plan, int cluster);

/*
 * Grouped transforms of uneven sizes (e.g. several grids of a multi-resolution
 * run).  dims: ngroups x 3 ints (n0, n1, n2) (host); counts: fields per group
 * (host).  Group i is a plan of batch counts[i]; fft3d_group_r2c / c2r take
 * host arrays of ngroups device pointers (group i's fields contiguous, layouts
 * as for fft3d_r2c / fft3d_c2r; c2r clobbers its inputs); fft3d_group_r2c_c2r
 * runs the forward of in into mid and then the inverse of mid (clobbered)
 * into out, as one call.  On a non-default stream each kind of call is
 * captured once per operand set into a CUDA graph and replayed with a single
 * graph launch.
 *
 * Two forms.  FFT3D_GROUP_STREAMS (the default): each size's plan runs its
 * passes on an internal stream forked from and joined back into stream.
 * FFT3D_GROUP_WORK_TABLE (offered wherever it applies: FP32, even n2, every n0
 * and n1 in {64, 96, 128, 160, 192} and n2/2 in {32, 48, 64, 80, 96}): one
 * persistent kernel launch per call runs every pass of every size (a work
 * table of row / column tiles handed out in order; a tile of a size's pass
 * waits, bounded, until that size's previous pass is complete); the round trip
 * is one launch too.
 * FFT3D_GROUP_WORK_TABLE_TEST_STALL is the work table with one dependency that
 * cannot be met: its waits give up (about a second), set the timeout status
 * and end the launch -- for testing fft3d_group_query_device_status only.
 * fft3d_group_set_form returns FFT3D_ERR_INVALID_ARG for a form the group
 * cannot run.  fft3d_group_plan_at gives group i's plan (for fft3d_autotune /
 * fft3d_set_choices, which shape the streams form; tune before the first call
 * with a given operand set, since a captured graph keeps the launch shapes).
 * fft3d_group_launches: kernel launches per call (dir -1 r2c, +1 c2r, 0 the
 * round trip).  fft3d_group_query_device_status synchronises stream and
 * returns FFT3D_ERR_TIMEOUT if a bounded wait of the group gave up.
 * dtype FFT3D_F64 is not offered (FFT3D_ERR_INVALID_ARG).
 */
#define FFT3D_GROUP_STREAMS 0
#define FFT3D_GROUP_WORK_TABLE 1
#define FFT3D_GROUP_WORK_TABLE_TEST_STALL 2
typedef struct fft3d_group_s* fft3d_group_handle;
fft3d_group_handle fft3d_plan_group(const int* dims, const int* counts, int ngroups, int dtype);
fft3d_handle fft3d_group_plan_at(fft3d_group_handle group, int i);
int fft3d_group_r2c(fft3d_group_handle group, const float* const* in, void* const* out, void* stream);
int fft3d_group_c2r(fft3d_group_handle group, void* const* in, float* const* out, void* stream);
int fft3d_group_r2c_c2r(fft3d_group_handle group, const float* const* in, void* const* mid, float* const* out,
                        void* stream);
int fft3d_group_launches(fft3d_group_handle group, int dir);
int fft3d_group_set_form(fft3d_group_handle group, int form);
int fft3d_group_get_form(fft3d_group_handle group);
int fft3d_group_query_device_status(fft3d_group_handle group, void* stream);
void fft3d_group_destroy(fft3d_group_handle group);

/*
 * Pseudo-spectral nonlinear term (the quadratic term of the Tarang-type
 * solvers of Sec. 1; the paper states that FFTs take about 75% of such a
 * solver's time).  For a velocity field given by its three half spectra
 * uhat_i (i = 0, 1, 2) it computes the six dealiased product spectra
 *     N_ij = mask * r2c(u_i * u_j) / N,   u_i = c2r(uhat_i),
 *     ij in (00, 01, 02, 11, 12, 22) (in that order),
 * mask = the 2/3 rule: keep bin k iff 3|k_a| < n_a on every axis, with k_a the
 * signed wavenumber in [-n_a/2, n_a/2) (Nyquist bins always dropped).
 * Passes, batched over the fields: n0 inverse x3 (out of place into the
 * workspace), n1 inverse x3, one row kernel doing the three c2r, the six
 * products in registers and the six r2c (k2 part of the mask), n1 forward x6
 * over the columns k2 the mask keeps (k1 part), n0 forward x6 over the
 * columns (k1, k2) it keeps (k0 part and 1/N); the skipped columns are zero.
 * The three middle passes can run per chunk of planes j0 (so that a chunk's
 * operands stay in L2 between them), on one stream or alternating between
 * two (fft3d_nonlinear_set_chunking).  On a non-default stream the
 * sequence is captured once into a CUDA graph per (uhat, nhat, workspace) and
 * replayed; on the legacy default stream it is launched directly.
 * Supported when n2/2 has a warp-resident row kernel (n2/2 in 8..512 of the
 * built lengths); else fft3d_nonlinear_plan fails with UNSUPPORTED_SIZE.
 */
typedef struct fft3d_nl_s* fft3d_nl_handle;

/* Plan for n0 x n1 x n2 fields (blocks; NULL on error, see fft3d_last_error). */
fft3d_nl_handle fft3d_nonlinear_plan(int n0, int n1, int n2);

/* Caller workspace: 3 * n0 * n1 * (n2/2+1) complex64 values. */
size_t fft3d_nonlinear_workspace_bytes(fft3d_nl_handle nl);
int fft3d_nonlinear_set_workspace(fft3d_nl_handle nl, void* dev_ptr);

/* uhat: 3 contiguous half spectra (device, read only, preserved);
 * nhat: 6 contiguous half spectra (device, written); 16-byte aligned; none
 * of uhat, nhat and the workspace may overlap. */
int fft3d_nonlinear_exec(fft3d_nl_handle nl, const void* uhat, void* nhat, void* stream);

/* Plane chunking of the middle passes (n1 inverse, rows, n1 forward): planes
 * = planes j0 per chunk (0 or >= n0: one chunk, the passes over the whole
 * fields); streams = 1, or 2 to alternate the chunks between the caller's
 * stream and a second stream of the plan (graph-captured calls only; calls
 * on the legacy default stream use one stream).  Drops the captured graph;
 * INVALID_ARG for planes < 0 or streams outside 1..2.  The n1 passes of a
 * chunk take the fields as an outer batch (the plain column kernel where the
 * whole-field pass may take another form), so results can differ between
 * chunkings by rounding.  get: the current setting. */
int fft3d_nonlinear_set_chunking(fft3d_nl_handle nl, int planes, int streams);
int fft3d_nonlinear_get_chunking(fft3d_nl_handle nl, int* planes, int* streams);

/* Kernel launches per fft3d_nonlinear_exec: the kernel nodes of the captured
 * graph once a call on a stream has captured one; before that, the count the
 * plan's kernel forms give (the forward n0 pass is one launch per kept k1 block
 * where the column path takes the six fields as an outer batch, else six). */
int fft3d_nonlinear_launches(fft3d_nl_handle nl);

/* NULL-safe; blocks on the device. */
void fft3d_nonlinear_destroy(fft3d_nl_handle nl);

/*
 * One time step of the incompressible Navier-Stokes equations in a periodic
 * box [0, 2 pi)^3, pseudo-spectral (the Tarang-type solver of Sec. 1; the
 * paper names the method, the scheme below is this library's): the velocity is
 * held as three half spectra uhat_i (u_i = c2r(uhat_i)), and
 *     R_l(uhat) = mask * (-i P_lm(k) sum_j k_j N_mj - nu |k|^2 uhat_l),
 * N = the dealiased quadratic term of fft3d_nonlinear_exec, P = I - k k^T/|k|^2
 * (the pressure projection; zero at k = 0), mask = the 2/3 rule (bins outside
 * it never change).  Heun's two-stage method:
 *     u* = u + dt R(u),   u <- u + dt/2 (R(u) + R(u*)).
 * Per step: the nonlinear term twice (5 launches each) and two fused
 * elementwise stage kernels (divergence, projection, viscous term, update);
 * on a non-default stream the 12 launches are captured once into a CUDA graph
 * per (uhat, workspace, nu, dt) and replayed; on the legacy default stream they
 * are launched directly.  FP32 storage and arithmetic.  Supported shapes: as
 * fft3d_nonlinear_plan (else UNSUPPORTED_SIZE).
 */
typedef struct fft3d_ns_s* fft3d_ns_handle;

/* Plan for n0 x n1 x n2 fields (blocks; NULL on error, see fft3d_last_error). */
fft3d_ns_handle fft3d_ns_plan(int n0, int n1, int n2);

/* Caller workspace: 15 * n0 * n1 * (n2/2+1) complex64 values (u*, the Heun
 * accumulator, the six product spectra, the nonlinear term's scratch);
 * 256-byte aligned. */
size_t fft3d_ns_workspace_bytes(fft3d_ns_handle ns);
int fft3d_ns_set_workspace(fft3d_ns_handle ns, void* dev_ptr);

/* uhat: 3 contiguous half spectra (device), advanced in place by one step of
 * size dt with kinematic viscosity nu (nu >= 0, dt > 0); 16-byte aligned; must
 * not overlap the workspace. */
int fft3d_ns_step(fft3d_ns_handle ns, void* uhat, float nu, float dt, void* stream);

/* The chunking of the step's nonlinear terms (as fft3d_nonlinear_set_chunking;
 * drops the step's captured graph). */
int fft3d_ns_set_chunking(fft3d_ns_handle ns, int planes, int streams);

/* Kernel launches per fft3d_ns_step (counted as for fft3d_nonlinear_launches). */
int fft3d_ns_launches(fft3d_ns_handle ns);

/* NULL-safe; blocks on the device. */
void fft3d_ns_destroy(fft3d_ns_handle ns);

/*
 * FP64 spectral diagnostics of a half spectrum (device-side checks of a
 * transform, and the energy spectrum of a pseudo-spectral solver, Sec. 1).
 * spec:   batch*n0*n1*H float2 (device), read only, laid out as fft3d_r2c
 *         writes it for a plan without EXPLICIT_TRANSPOSE.
 * total:  batch doubles (device) or NULL: sum over the half spectrum of
 *         c_k2 |X|^2 (c_k2 = 1 at k2 = 0 and, for even n2, at k2 = n2/2;
 *         else 2), which equals
 *         n0*n1*n2 * sum_j x_j^2 when spec = r2c(x) (Parseval).
 * shells: batch*nbins doubles (device) or NULL: the same sum per integer
 *         shell b = floor(|k| + 1/2) (shell 0 holds only k = 0; shell b >= 1
 *         is (2b-1)^2 <= 4|k|^2 < (2b+1)^2), |k_a| = min(j_a, n_a - j_a),
 *         decided in integers; bins of shell >= nbins are left out.
 * 1 <= nbins <= 8192.  |X|^2 in FP32, sums in FP64, block partials summed in
 * a fixed order (deterministic).  Uses plan-owned scratch (allocated at plan
 * time for nbins up to the largest shell of the shape; a larger nbins grows
 * it, which synchronises the device).  Asynchronous on stream otherwise.
 * FFT3D_F64 plans: FFT3D_ERR_INVALID_ARG (the spectra here are float2).
 */
int fft3d_energy(fft3d_handle plan, const void* spec, double* total, double* shells, int nbins, void* stream);

/*
 * fft3d_energy for callers that cannot allocate device memory: applications
 * whose device memory is owned entirely by their own allocator or by a budget
 * fixed at start-up, or code called back from inside another library's memory
 * management, where a cudaMalloc inside a library call would fail, block, or
 * break that budget.  The paper has no counterpart; this is an interface
 * convenience of the library.
 *
 * Same inputs, outputs and definitions as fft3d_energy (spec is
 * batch*n0*n1*(n2/2+1) float2 on the device; total and shells device
 * doubles, either may be NULL, not both), but it takes the shape instead of a
 * plan and allocates nothing: its scratch is one fixed array of 2^18 doubles
 * (2 MiB) inside the library, which every GPU that loads the library holds
 * until the process exits.  A call needs batch * B * (nbins + 1) doubles of
 * it, B = min(256, ceil(n0*n1/8)); a larger call is rejected with
 * FFT3D_ERR_UNSUPPORTED_SIZE before anything is launched.
 *
 * Every call looks up the array's device address on the current device
 * (cudaGetSymbolAddress, a host-side lookup, so the address stays right after
 * anything that recreates the device's context, such as cudaDeviceReset).
 * The first call on a device is its set-up: that lookup may load the
 * library's device code there, so make the first call on each device before
 * any stream capture.  Every call on a device shares the one array, and it keeps the
 * last call's contents (each call writes all the scratch it reads, so nothing
 * needs clearing): calls that overlap on the GPU, e.g. on two streams without
 * ordering between them, race and give wrong results; order them, for
 * instance by issuing them on one stream.  Asynchronous on stream.  Reports
 * through its return value only (fft3d_last_error is not updated).
 */
int fft3d_energy_noalloc(const void* spec, int n0, int n1, int n2, int batch, double* total, double* shells,
                         int nbins, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* FFT3D_H */
