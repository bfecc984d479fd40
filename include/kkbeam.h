/*
 * kkbeam.h -- C ABI of the GB300 (sm_103a) KK beamforming library.
 *
 * KK beamforming (Khetan & Mertz, "Far-field compressive ultrasound
 * beamforming") forms a plane-wave-compounded ultrasound image in two steps:
 *   1. a far-field decomposition of each transmit angle's channel data into
 *      virtual receive plane waves, Eq. (compression), applied through the
 *      Fourier shift theorem on the analytic spectrum (Section II-F);
 *   2. image formation, Eq. (KK): every pixel interpolates each virtual
 *      plane wave's record at its (transmit + receive) delay and sums over the
 *      (transmit, receive) pairs of the chosen k-space sampling scheme
 *      (Eq. (uniform), Eq. (confocal)), with optional coherent / incoherent
 *      compounding of J groups (Eqs. (coherent), (incoherent)).
 * A delay-and-sum reference, Eq. (DAS), runs on the same plan type.
 *
 * Conventions (all calls):
 *  - Units: metres, seconds, radians.  Element l sits at (elem_x[l], 0).
 *    Image x is lateral, z is depth.  Sample n of a record is at time n/fs;
 *    a transmit plane wave passes the origin at t = 0.
 *  - Arrays are row-major, last index fastest.  Complex values are
 *    interleaved (re, im) float32 pairs ("cfloat", 8 bytes).
 *  - Ownership: the caller owns every buffer passed in (device buffers may
 *    come from any allocator).  A plan owns its look-up tables, which are
 *    immutable after creation; a plan may be used from several streams at
 *    once provided each stream has its own workspace.
 *  - Execution: every call taking a stream only enqueues work on that
 *    stream (a cudaStream_t passed as void*, NULL = legacy default stream)
 *    and returns without synchronising.  Plan creation synchronises.
 *  - Errors: no call throws.  Each returns a kk_status; on failure
 *    kk_last_error() gives a message (thread-local).  A failed call leaves
 *    the output buffers in an unspecified state and the plan unchanged.
 *  - Every enqueue call checks for launch errors before returning
 *    (KK_ERR_CUDA); errors of the asynchronous work surface at the caller's
 *    next synchronisation.
 */
#ifndef KKBEAM_H
#define KKBEAM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum kk_status {
  KK_OK = 0,
  KK_ERR_INVALID_ARG = 1, /* null pointer, size out of range, bad index */
  KK_ERR_UNSUPPORTED = 2, /* valid but not implemented (e.g. an FFT length) */
  KK_ERR_CUDA = 3,        /* a CUDA runtime call or launch failed */
  KK_ERR_OOM = 4,         /* device allocation failed at plan time */
  KK_ERR_TIMEOUT = 5,     /* a bounded device-side wait gave up */
  KK_ERR_BOUNDS = 6       /* bounds-checked build only: a kernel index fell outside
                             its buffer (the access was skipped) */
} kk_status;

typedef enum kk_rf_dtype { KK_RF_I16 = 0, KK_RF_F32 = 1 } kk_rf_dtype;

/* Operand precision of the decomposition contraction (step 1).  FFTs,
 * interpolation and summation always run in FP32. */
typedef enum kk_precision {
  KK_PREC_F32 = 0,
  KK_PREC_BF16 = 1,
  KK_PREC_F16 = 2,
  KK_PREC_F8E4M3 = 3
} kk_precision;

typedef enum kk_compound {
  KK_COMPOUND_NONE = 0,       /* I is not written */
  KK_COMPOUND_COHERENT = 1,   /* I = |sum_j B_j|^2, Eq. (coherent) */
  KK_COMPOUND_INCOHERENT = 2  /* I = sum_j |B_j|^2, Eq. (incoherent) */
} kk_compound;

typedef enum kk_aperture {
  KK_APERTURE_BOXCAR = 0,  /* 1 inside the half-width, 0 outside */
  KK_APERTURE_HANN = 1     /* (1 + cos(pi d / h)) / 2 inside, 0 outside */
} kk_aperture;

typedef enum kk_scheme {
  KK_SCHEME_SAME = 0,     /* theta_o = theta_i (Section II-C, redundant) */
  KK_SCHEME_VERNIER = 1,  /* theta_o = 2 o dtheta_i / M (Section II-C) */
  KK_SCHEME_SHIFTED = 2,  /* Eq. (uniform) with shift j */
  KK_SCHEME_CONFOCAL = 3  /* Eq. (confocal) */
} kk_scheme;

/* Pixel (ix, iz) sits at (x0 + ix*dx, z0 + iz*dz).  dz > 0, z0 >= 0. */
typedef struct kk_grid {
  int32_t nx, nz;
  double x0, dx, z0, dz;
} kk_grid;

/* Everything a plan needs.  Pointers are host pointers, read during plan
 * creation only. */
typedef struct kk_plan_desc {
  int32_t n_elem;             /* L >= 1 */
  const double *elem_x;       /* [L] lateral element positions */
  int32_t n_tx;               /* N >= 1: acquired transmit angles (rows of rf) */
  const double *tx_angles;    /* [N], |angle| < 80 deg */
  int32_t n_rx;               /* number of receive angles (KK only) */
  const double *rx_angles;    /* [n_rx], |angle| < 80 deg (KK only) */
  int32_t n_pairs;            /* P >= 1 (KK only) */
  const int32_t *pairs;       /* [P][2] = (tx index, rx index) (KK only) */
  const int32_t *group_of_pair; /* [P] in [0, n_groups); NULL = all 0 */
  int32_t n_groups;           /* J >= 1 */
  int32_t compound;           /* kk_compound */
  kk_grid grid;
  double c;                   /* speed of sound > 0 */
  double fs;                  /* sampling rate > 0 */
  int32_t n_samples;          /* T: even, T/2 in {128,256,512,768,1024,1536,2048} */
  int32_t rf_dtype;           /* kk_rf_dtype */
  int32_t precision;          /* kk_precision (KK only; DAS is FP32).  The
                                 BF16/F16/F8E4M3 forms run the decomposition
                                 contraction on tensor cores and need
                                 n_elem <= 128 and <= 256 transmits in use */
  int32_t device;             /* CUDA device ordinal the plan lives on */
  /* Apodization (the paper states Eqs. (DAS) and (KK) without it and notes
   * it folds in directly; zero-initialised fields mean none): */
  const double *pair_weight;  /* [P] weight of pair p's term in Eq. (KK)
                                 (KK only; NULL = 1).  It scales pair p's
                                 decomposed record (row p of the rf_theta
                                 that kk_decompose / kk_inverse write), so
                                 kk_beamform sums weighted terms */
  double f_number;            /* DAS receive aperture: element l reaches pixel
                                 (x, z) when |x - u_l| <= z / (2 f_number),
                                 weighted by `aperture`; <= 0 = full aperture */
  int32_t aperture;           /* kk_aperture window over that half-width */
  /* Volumetric imaging with a 2D (matrix) array, the extension Section IV
   * names (KK only; all NULL / 0 = a linear array and a 2D grid).  Element l
   * sits at (elem_x[l], elem_y[l], 0).  A plane wave with tilts (ax, ay)
   * travels along (sin ax, sin ay, sqrt(1 - sin^2 ax - sin^2 ay)) and passes
   * the origin at t = 0 (ax is tx_angles / rx_angles, ay the arrays below);
   * every used angle needs sin^2 ax + sin^2 ay < sin^2(80 deg).  The receive
   * shear of Eq. (compression) is ((xr - u_l) sx + (yr - v_l) sy) / c with
   * xr, yr the array edges that keep each term a non-negative advance.
   * Voxel (ix, iy, iz) sits at (x0 + ix dx, y0 + iy dy, z0 + iz dz); B is
   * [J][ny][nz][nx] and I [ny][nz][nx].  Set any of these to make a plan
   * volumetric. */
  const double *elem_y;       /* [L] element y positions (NULL = 0) */
  const double *tx_angles_y;  /* [N] transmit tilts ay (NULL = 0) */
  const double *rx_angles_y;  /* [n_rx] receive tilts ay (NULL = 0) */
  int32_t ny;                 /* y slices (<= 1: one slice at y0) */
  double y0, dy;              /* dy > 0 when ny > 1 */
} kk_plan_desc;

typedef struct kk_plan kk_plan;

/* Sizes a caller needs to allocate buffers for a plan. */
typedef struct kk_plan_info {
  int32_t n_elem, n_tx, n_samples, n_bins; /* L, N, T, F = T/2 */
  int32_t n_tx_used, n_rx_used;            /* transmits / receive angles in use */
  int32_t n_pairs, n_groups;               /* P, J */
  int32_t nx, nz;
  int32_t is_das;
  size_t workspace_bytes;                  /* for kk_decompose/kk_beamform/das_beamform */
  size_t rf_bytes;                         /* N*L*T*sizeof(sample) */
  size_t rf_theta_bytes;                   /* P*T*8 */
  size_t image_bytes;                      /* J*ny*nz*nx*8 (B) */
  size_t intensity_bytes;                  /* ny*nz*nx*4 (I) */
  double compression_factor;               /* L / (number of receive angles in use) */
  int32_t launches_decompose;              /* kernels one kk_decompose enqueues */
  int32_t launches_beamform;               /* kernels one kk_beamform / das_beamform enqueues */
  int32_t ny;                              /* y slices (1 for a 2D grid) */
  int32_t is_volume;                       /* a volumetric plan (2D array or y slices) */
  /* FP32 volumetric plans whose elements fill an Lx x Ly grid and whose
   * receive waves in use are every combination of Mx x-tilts and My y-tilts
   * run the element sum as two per-axis contractions (the shear delay splits
   * per axis); these are Lx, Ly, Mx, My then, all 0 for the full form */
  int32_t sep_lx, sep_ly, sep_mx, sep_my;
  /* image-formation launch shape: pixels per thread along z (tile = 32 x 4
   * gather_rows), pairs (transmits, DAS) per stage, and the number of pair
   * (element, DAS) slices whose partial images are summed after the gather */
  int32_t gather_rows, gather_stage, gather_split;
  int32_t records_trimmed;                 /* kk_plan_set_trim in force */
  size_t rf_theta_stored_bytes;            /* bytes of rf_theta one decomposition stores */
} kk_plan_info;

/*
 * KK plan.  Validates the description, sorts pairs by group, and builds on
 * the device (FP64 on the host, then stored as integer / FP32 tables):
 *   - shear phases phi[o][l] = frac(fs * delta_l(theta_o) / T) in 0.64 fixed
 *     point, delta_l(theta_o) = (x_ref - u_l) sin(theta_o) / c with x_ref the
 *     array end that makes the shear a non-negative advance (Eq. (compression));
 *   - per-pair affine delay coefficients s(ix, iz) = A ix + B iz + C in 32.32
 *     fixed point, s = fs [x sin_i + z cos_i + (x - x_ref) sin_o + z cos_o] / c
 *     (Eq. (KK) with the time origin of the sheared record at x_ref);
 *   - FFT twiddles.
 * Returns KK_ERR_INVALID_ARG / KK_ERR_UNSUPPORTED / KK_ERR_OOM / KK_ERR_CUDA.
 * On success *out owns device memory on d->device until kk_plan_destroy.
 */
kk_status kk_plan_create(kk_plan **out, const kk_plan_desc *d);

/* DAS plan (Eq. (DAS)): receive/pair/group/precision fields are ignored,
 * every transmit of rf is used, J = 1.  A volumetric description (2D array,
 * tilted transmits, ny y slices) gives the volumetric sum over elements at
 * (elem_x, elem_y) and voxels (x, y, z), full aperture only (f_number > 0:
 * KK_ERR_UNSUPPORTED), and pixel pitches fine enough for 256-sample staged
 * windows (otherwise KK_ERR_UNSUPPORTED). */
kk_status das_plan_create(kk_plan **out, const kk_plan_desc *d);

/* Frees the plan's device tables.  NULL is a no-op.  The caller must make
 * sure no work using the plan is still in flight. */
void kk_plan_destroy(kk_plan *p);

kk_status kk_plan_get_info(const kk_plan *p, kk_plan_info *info);

/*
 * Tuning of the KK image-formation kernel (no counterpart in the paper: a
 * launch-shape choice).  rows in {2, 4, 8}: pixels per thread along z, tile =
 * 32 x (4 rows) pixels; stage in {4, 8, 16}: pairs staged per batch.  Results
 * do not depend on it beyond FP32 rounding order.  Returns
 * KK_ERR_UNSUPPORTED when the grid's staged window is too long for the shape
 * (the plan keeps its previous shape).  workspace_bytes covers every shape,
 * so a workspace allocated before the call stays valid; never call it while
 * work is in flight.
 */
kk_status kk_plan_set_gather(kk_plan *p, int32_t rows, int32_t stage);

/*
 * Records trimmed to the grid's reach (no counterpart in the paper: a store
 * choice; images do not change, bit for bit).  With on = 1, kk_decompose,
 * kk_inverse and streams of the plan store of each record y_p only the
 * samples that Eq. (KK)'s interpolation can read for some pixel of the grid
 * under any image-formation launch shape (the per-pair sample range the
 * plan computes from its delay tables); the rest of rf_theta is left as it
 * was.  On the 75-transmit x 128-angle frame on a 512 x 512 grid this skips
 * about 45 % of the record stores.  Linear-array KK plans only (volumetric
 * plans: KK_ERR_UNSUPPORTED; DAS plans: KK_ERR_INVALID_ARG); on = 0 restores
 * full records.  Never call it while work is in flight.
 */
kk_status kk_plan_set_trim(kk_plan *p, int32_t on);

/*
 * Device status word of the plan's kernels: KK_OK, or KK_ERR_TIMEOUT when a
 * bounded device-side wait gave up (the kernel then abandoned its work and
 * released its resources).  Synchronises with the device, returns the word
 * in *status and resets it to KK_OK.  No counterpart in the paper.
 */
kk_status kk_plan_status(const kk_plan *p, int32_t *status);

/*
 * Check of the bounded device-side waits (no counterpart in the paper).
 * Launches one CTA of 128 threads on `stream` that waits on an mbarrier no
 * copy or thread ever signals, through the same bounded wait every pipelined
 * kernel of the library uses, with a limit of limit_ns nanoseconds (clamped
 * to [1000, 1e9]).  The wait runs out, the CTA records KK_ERR_TIMEOUT in the
 * plan's status word (read it with kk_plan_status) and returns, as a kernel
 * that lost a signal does; nothing is in flight, so the context stays usable.
 */
kk_status kk_plan_check_wait_timeout(const kk_plan *p, int64_t limit_ns, void *stream);

/*
 * Bounds-checked build (no counterpart in the paper).  The library compiled
 * with KK_DEBUG_BOUNDS checks every staged-window index of the KK and DAS
 * gathers against its pair's (channel's) window before the shared-memory
 * read; a failed check skips the read and is counted on the device.
 * kk_debug_bounds synchronises the device, returns the number of failed
 * checks since the previous call in *violations and resets it.  The
 * product build has no checks and returns KK_ERR_UNSUPPORTED.
 */
kk_status kk_debug_bounds(int64_t *violations);

/* Workspace bytes needed by kk_decompose / kk_beamform / das_beamform. */
kk_status kk_plan_workspace_size(const kk_plan *p, size_t *bytes);

/*
 * Step 1, the far-field decomposition (Eq. (compression), Section II-F):
 *   X[k][c]  = h_k sum_t rf[i][l][t] exp(-2 pi i k t / T)   (c = iu*L + l)
 *   Y[k][q]  = sum_l X[k][iu][l] exp(+2 pi i k phi[o][l])    (q = iu*Mu + ou)
 *   y[p][t]  = (1/T) sum_{k<T/2} Y[k][q(p)] exp(+2 pi i k t / T)
 * h_0 = 1, h_k = 2 (negative frequencies and the Nyquist bin dropped).
 *
 * d_rf        device [N][L][T] int16 or float32 (plan's rf_dtype)
 * d_rf_theta  device [P][T] cfloat, row p = pair p in the caller's order
 * d_workspace device, >= workspace_bytes, 256-byte aligned
 */
kk_status kk_decompose(const kk_plan *p, const void *d_rf, void *d_rf_theta,
                       void *d_workspace, void *stream);

/* Stage calls of kk_decompose, for inspection and testing.
 * d_X: [F][Nu][L] complex spectra with h_k applied: cfloat for FP32 plans,
 *      interleaved (re, im) bfloat16 for BF16 plans, float16 for F16 and
 *      F8E4M3 plans (the FP8 form rounds to e4m3 inside the contraction).
 *      The float16 spectra are stored times 2^-ceil(log2(2T)) so that RF
 *      samples of magnitude <= 32768 cannot overflow; kk_shear undoes it.
 * d_Y: [F][Nu][Mu] cfloat for every precision. */
kk_status kk_spectrum(const kk_plan *p, const void *d_rf, void *d_X, void *stream);
kk_status kk_shear(const kk_plan *p, const void *d_X, void *d_Y, void *stream);
kk_status kk_inverse(const kk_plan *p, const void *d_Y, void *d_rf_theta,
                     void *stream);

/*
 * Step 2, image formation (Eq. (KK)) and compounding:
 *   B_j(ix, iz) = sum_{p in group j} lerp(y_p, s_p(ix, iz))
 * lerp(y, s): k = floor(s), f = s - k, (1-f) y[k] + f y[k+1] when
 * 0 <= k and k+1 <= T-1, else 0.
 * d_rf_theta  device [P][T] cfloat (as written by kk_decompose)
 * d_B         device [J][nz][nx] cfloat (always written)
 * d_I         device [nz][nx] float, written when the plan's compound mode is
 *             COHERENT or INCOHERENT; may be NULL otherwise
 * d_workspace device, >= workspace_bytes
 */
kk_status kk_beamform(const kk_plan *p, const void *d_rf_theta, void *d_B,
                      float *d_I, void *d_workspace, void *stream);

/*
 * KK image formation that allocates nothing.  The paper has no counterpart:
 * this entry point exists for callers that cannot call cudaMalloc or hand
 * over a workspace -- code running inside a host framework that owns all
 * device memory through its own pool, a plugin loaded into such a process,
 * a real-time loop that must never allocate.
 *
 * Same inputs, outputs and results as kk_beamform.  The partial images of the
 * pair slices, which kk_beamform keeps in the caller's workspace, live in a
 * fixed 8 MiB device array compiled into the library; every GPU that loads
 * the library holds that array until the process exits.  A plan whose partial
 * images need more than 8 MiB (pair slices x groups x nx x nz x ny x 8 bytes,
 * ny = 1 for 2D grids; 0 when the plan uses a single slice) is rejected with
 * KK_ERR_INVALID_ARG.  Every call that needs the array looks up its device
 * address on the plan's device (a set-up step, no allocation; done per call,
 * so a re-created context is never handed a stale address): make the first
 * such call on a device before any stream capture.
 * All calls share the one array, which keeps the last call's contents (every
 * call rewrites all it reads, so nothing needs clearing); calls that overlap
 * on the GPU -- different streams, or host threads without ordering -- race
 * and must be serialised by the caller.
 */
kk_status kk_beamform_noalloc(const kk_plan *p, const void *d_rf_theta, void *d_B,
                              float *d_I, void *stream);

/*
 * DAS reference path (Eq. (DAS)): analytic signal of every channel (same FFT,
 * mask and inverse as step 1, no shear), then
 *   B(ix, iz) = sum_{i,l} lerp(y_il, fs (tau_in + |r - (u_l, 0)| / c))
 * d_rf [N][L][T], d_B [nz][nx] cfloat, d_I [nz][nx] float (|B|^2) or NULL.
 * Volumetric plans: tau_in = (x sx_i + y sy_i + z sz_i) / c with the unit
 * direction of transmit tilts (ax_i, ay_i), the receive distance to element
 * (u_l, v_l, 0), and d_B [ny][nz][nx], d_I [ny][nz][nx].
 */
kk_status das_beamform(const kk_plan *p, const void *d_rf, void *d_B,
                       float *d_I, void *d_workspace, void *stream);

/*
 * Batched form (no counterpart in the paper: a throughput form of steps 1
 * and 2 for many frames).  Frames may differ in array, record length,
 * transmit set, pair set and grid; each has its own KK plan and buffers.
 *
 * kk_batch_create builds a CUDA graph that runs every frame's decomposition
 * (frames run concurrently) and then KK image formation for all frames as
 * one persistent launch over their (frame, tile) work items, largest frames
 * first.  shape = 0 picks the image-formation launch shape by timing the
 * feasible shapes on this batch (the kernels run on the frames' buffers;
 * creation first synchronises `stream`, then works on a private stream and
 * returns when done); shape = rows * 100 + stage (rows in
 * {2, 4, 8}, stage in {4, 8, 16}) sets it.  Results match the per-frame calls
 * up to FP32 summation order.  The buffers given here are baked into the
 * graph: refill them in place between runs.  Each frame needs its own
 * workspace (frames run concurrently).  Volumetric plans may be mixed in:
 * their (frame, tile) items, tiles running over every y slice, form a
 * second list with its own persistent launch and launch shape (timed the
 * same way with shape = 0; a set shape applies to both lists), after the
 * linear-array frames' launch.
 *
 * kk_batch_run enqueues the graph on `stream`.  A batch must not run twice
 * concurrently (it owns one work counter).
 */
typedef struct kk_batch kk_batch;

typedef struct kk_batch_frame {
  const kk_plan *plan;   /* KK plan of the frame */
  const void *d_rf;      /* [N][L][T] int16 / float32 */
  void *d_rf_theta;      /* [P][T] cfloat */
  void *d_B;             /* [J][nz][nx] cfloat */
  float *d_I;            /* [nz][nx], required when the plan compounds */
  void *d_workspace;     /* >= the plan's workspace_bytes, 256-byte aligned */
} kk_batch_frame;

typedef struct kk_batch_info {
  int32_t n_frames, n_items, rows, stage, max_window, grid, graph_nodes, n_tuned;
  double pixel_pairs;      /* sum over frames of pairs x pixels (x y slices) */
  int32_t tuned_shape[16]; /* shapes timed by the autotuner (rows * 100 + stage) */
  float tuned_ms[16];      /* their image-formation times */
  /* the volumetric frames' list (all 0 without volumetric frames); the
   * fields above describe the linear-array frames' list */
  int32_t n_volume_frames, n_items_volume, rows_volume, stage_volume, max_window_volume;
} kk_batch_info;

kk_status kk_batch_create(kk_batch **out, const kk_batch_frame *frames, int32_t n_frames,
                          int32_t shape, void *stream);
kk_status kk_batch_run(kk_batch *b, void *stream);
kk_status kk_batch_get_info(const kk_batch *b, kk_batch_info *info);
void kk_batch_destroy(kk_batch *b);

/*
 * End to end from host memory: copies h_rf to the device, runs
 * kk_decompose + kk_beamform (or das_beamform for a DAS plan), copies B and
 * I back.  All on `stream`; returns after enqueueing (the caller
 * synchronises before reading h_B / h_I).  Host buffers should be pinned
 * for the copies to be asynchronous.
 * d_scratch   device, >= kk_run_host_scratch_size bytes (holds rf, rf_theta,
 *             B, I and the workspace)
 * h_I may be NULL.
 */
kk_status kk_run_host_scratch_size(const kk_plan *p, size_t *bytes);
kk_status kk_run_host(const kk_plan *p, const void *h_rf, void *h_B, float *h_I,
                      void *d_scratch, void *stream);

/*
 * Synthetic channel data on the GPU (input generation, not the method; the
 * paper has no counterpart).  rf[i][l][t] = sum_s a_s p(t/fs - tau_in - tau_out)
 * + optional white Gaussian noise, with tau_in = (x sin_i + z cos_i)/c,
 * tau_out = |(x, z) - (u_l, 0)|/c and p(t) = exp(-alpha t^2) cos(2 pi f0 t)
 * (spectrum -6 dB at f0 (1 +- bw/2), truncated at +-4 sigma), in FP32.
 * d_tx_sincos [N][2] (sin, cos) of the transmit angles; d_elem_x [L] element
 * positions (m); d_scat [n_scat][4] (x, z, amplitude, unused); noise from a
 * counter-based generator seeded by `seed`.  d_rf [N][L][T] float32.
 * Accumulation order is not fixed (shared-memory atomics): repeated calls
 * may differ in the last bits.
 */
kk_status kk_simulate_rf(int32_t n_tx, const float *d_tx_sincos, int32_t n_elem,
                         const float *d_elem_x, int32_t T, double fs, double c, double f0,
                         double bw, int32_t n_scat, const float *d_scat, double noise_sigma,
                         uint64_t seed, float *d_rf, void *stream);

/*
 * Receive angles of one scheme (pure host, FP64):
 *   o = -(M-1)/2 .. (M-1)/2 in unit steps (the paper's -floor(M/2)..floor(M/2)
 *   for odd M; half-integers for even M), dtheta = transmit spacing,
 *   SAME:     out[m] = tx_angles_sub[m] (requires M == n_tx; uses `tx`)
 *   VERNIER:  2 o dtheta / M
 *   SHIFTED:  sgn(o) dtheta (2|o|/M + j)                Eq. (uniform)
 *   CONFOCAL: sgn(o) dtheta (2|o|/M + mod(floor|o|, floor(n_tx/2)))  Eq. (confocal)
 * tx: [n_tx] transmit angles of the subset in use (SAME only; may be NULL
 * otherwise).  out_rx: [M].
 */
kk_status kk_scheme_angles(int32_t kind, int32_t n_tx, const double *tx,
                           double dtheta, int32_t M, double j, double *out_rx);

/* Thread-local message of the last failed call on this thread ("" if none). */
const char *kk_last_error(void);

/* Library version string. */
const char *kk_version(void);

#ifdef __cplusplus
}
#endif

#endif /* KKBEAM_H */
