/*
 * ewald_gb300.h -- C ABI of the GB300 spectral Ewald library for the triply
 * periodic Stokeslet sum
 *
 *     u_i = sum_j sum_{p in L Z^3} G(x_i - x_j + p) f_j,   G(r) = I/|r| + r r^T/|r|^3
 *
 * (Kosmacher, Du, Bagge, Biros, "A Performance Portable Fast Ewald Summation
 * for Stokes Flow": Sec. 2 eq. (potentials) and the Stokeslet of Sec. 2, here
 * with all three directions periodic).  The sum is evaluated by the spectral
 * Ewald method of Sec. 2 / Algorithm 1: near field (P2P) over cell lists within
 * the cutoff rc, plus far field P2G -> FFT -> CNV -> IFFT -> G2P on a uniform
 * M^3 grid, plus the self term.  Every step runs in this library's CUDA kernels
 * (cuFFT for the FFTs) on one GPU; there is no CPU fallback.
 *
 * Conventions shared by all entry points
 * --------------------------------------
 *  - Points and forces are N x 3 row-major FP64 arrays in DEVICE memory unless
 *    the entry point says HOST.  Results are written as N x 3 row-major FP64.
 *    The caller owns every array it passes; the library never frees them.
 *  - Positions may lie outside [0, L)^3: they are wrapped periodically.  A
 *    NaN or Inf coordinate is detected on the device; the apply then writes
 *    unspecified values (never out-of-bounds memory) and the next call of
 *    ewald_sync_status() returns EWALD_EINVAL.
 *  - Sources = targets = the N points.  The pair (i, i, p = 0) and exactly
 *    coincident points (|r| == 0) are skipped (Sec. 2: "the term is skipped").
 *  - The k = 0 Fourier mode is dropped (zero mean velocity, Hasimoto's
 *    convention); a net force is allowed.
 *  - Apply-type calls are asynchronous on `stream` (a cudaStream_t passed as
 *    void*; NULL = the legacy default stream) and return after launching.
 *    Host-side argument errors are returned immediately and launch nothing.
 *  - A plan is bound to the device current at ewald_plan() time and to its N;
 *    calls on one plan must not overlap in time (they share its workspace).
 *  - No call aborts the process; every call returns a status.
 */
#ifndef EWALD_GB300_H
#define EWALD_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ewald_plan_s *ewald_plan_t;

typedef enum {
    EWALD_OK = 0,
    EWALD_EINVAL = 1,      /* bad argument (N < 1, L <= 0, tol out of range, NULL, NaN input) */
    EWALD_ENOMEM = 2,      /* device or host allocation failed */
    EWALD_ECUDA = 3,       /* a CUDA runtime call failed */
    EWALD_ECUFFT = 4,      /* a cuFFT call failed */
    EWALD_ETIMEOUT = 5,    /* a bounded device wait ran out (batched / served queues) */
    EWALD_EUNSUPPORTED = 6 /* parameters outside what the kernels implement */
} ewald_status;

typedef enum {
    /* Everything in FP64 (P2P, P2G, FFT, CNV, G2P, sum). */
    EWALD_F64 = 0,
    /* P2P, P2G and G2P in FP32 with FP32 accumulation; FFT, CNV and the final
     * near + far sum in FP64 when tol < 1e-6, else FP32 FFT/CNV and FP64 sum.
     * At tol 1e-7 and below, where plain single precision does not reach
     * with margin: P2P in double-single FP32 arithmetic (down to tol 1e-9;
     * FP64 below) and P2G/G2P in double-single (8^3 tiles, 8 <= P <= 16) or
     * FP64.  Callers still pass and receive FP64 arrays. */
    EWALD_F32_BULK = 1
} ewald_dtype;

/* Method parameters (Sec. 2.4).  ewald_get_params() fills every field.  As an
 * override for ewald_plan_ex(), a field <= 0 means "choose it": the library
 * then picks it from the error estimate eq. (ese) as described at ewald_plan. */
typedef struct {
    double L;              /* box side */
    double tol;            /* requested tolerance */
    double xi;             /* Ewald splitting parameter xi (Sec. 2) */
    double rc;             /* near-field cutoff radius r_c (Sec. 2.1) */
    double cell;           /* near-field cell width L / n_c (>= rc) */
    double h;              /* grid spacing L / M */
    double est_err;        /* eq. (ese) estimate E^N + E^F + E^w for unit sum |f|^2 */
    int32_t n_c;           /* near-field cells per side */
    int32_t M;             /* grid points per side (far field) */
    int32_t P;             /* window support in grid points (Sec. 2.2) */
    int32_t poly_deg;      /* degree nu of the piecewise-polynomial window */
    int32_t tile;          /* grid tile edge T used by P2G / G2P */
    int32_t p2p_block;     /* threads per P2P block */
    int32_t near_f64;      /* 1: P2P/P2G/G2P in FP64, 0: FP32 */
    int32_t fft_f64;       /* 1: FFT/CNV in FP64, 0: FP32 */
    int64_t footprint_bytes; /* device memory owned by the plan */
    int32_t near_ds;       /* 1: P2P in double-single arithmetic (pairs of FP32 values,
                              ~44 bits) with P2G/G2P in double-single or FP64 --
                              EWALD_F32_BULK at 1e-9 <= tol <= 1e-7; 0 otherwise.
                              Read-only (not an override). */
    int32_t reserved_;     /* zero */
} ewald_params;

/* Per-stage device times (ms) of the most recent apply with timing enabled
 * (ewald_set_timing).  P2P runs on a second stream concurrently with the far
 * field, so the stages do not add up to total_ms.  In a combined apply
 * (ewald_apply_combined) p2p_ms includes the double layer's FP32 near field
 * (FP32 plans) and sum_ms its FP64 near field (the other plans); p2g_ms
 * covers the spreading of all nine components.  Plans with M in {64, 128,
 * 256} run the z transforms and the CNV in one kernel (scale_ms): with FP32
 * spectra between 2-D (y, x) transforms of each z plane (fft_ms, ifft_ms),
 * in a combined apply with the double layer's six density components
 * transformed and scaled alongside; with FP64 spectra (Stokeslet applies) in
 * double-single arithmetic, fft_ms and ifft_ms then covering the 1-D
 * transforms along x and the double-single y transforms. */
typedef struct {
    float bin_ms, p2p_ms, p2g_ms, fft_ms, scale_ms, ifft_ms, g2p_ms, sum_ms, total_ms;
} ewald_stage_timing;

/* Human-readable name of a status code (static string, never NULL). */
const char *ewald_status_string(ewald_status s);

/* Choose the method parameters for N points in a box of side L at relative
 * tolerance tol, without touching any GPU.  Rule (Sec. 2.4): each term of the
 * eq. (ese) estimate is held below tol/10 (the paper uses tol/3 for an rms
 * error; the max-norm error runs about 3x the rms one).  With M and P given:
 * xi is the largest value with E^F <= tol/10, then rc the smallest with
 * E^N <= tol/10.  Without them, M (a cuFFT-friendly multiple of 8) and rc
 * minimise a per-stage cost model subject to the same bounds, and P is the
 * smallest support with E^w <= tol/10.  M must be a multiple of 4 (the grid
 * tile).  `override` may be NULL.  Errors: EINVAL for N < 1, L <= 0,
 * tol outside [1e-12, 1e-2], NULL out; EUNSUPPORTED when an override cannot
 * be honoured (e.g. P > 16 or M < P). */
ewald_status ewald_choose_params(int64_t N, double L, double tol, ewald_dtype dtype,
                                 const ewald_params *override, ewald_params *out);

/* Create a plan: choose parameters (as ewald_choose_params), fit the
 * piecewise-polynomial window (Sec. 4, Horner form), allocate every device
 * workspace and create the cuFFT plans on the current device.  *out is set
 * only on success.  Errors: as ewald_choose_params, plus ENOMEM, ECUDA,
 * ECUFFT. */
ewald_status ewald_plan(int64_t N, double L, double tol, ewald_dtype dtype, ewald_plan_t *out);
ewald_status ewald_plan_ex(int64_t N, double L, double tol, ewald_dtype dtype,
                           const ewald_params *override, ewald_plan_t *out);

/* Release the plan and all its device memory.  NULL is ignored.  The caller
 * must make sure no work on the plan is still running. */
void ewald_destroy(ewald_plan_t plan);

/* Copy the plan's parameters into *out. */
ewald_status ewald_get_params(ewald_plan_t plan, ewald_params *out);

/* The full apply, Algorithm 1 (bin, P2P, P2G, FFT, CNV, IFFT, G2P, SUM):
 * u = (near + far - self) for positions x and forces f (device, N x 3 FP64). */
ewald_status ewald_apply(ewald_plan_t plan, const double *x, const double *f, double *u,
                         void *stream);

/* Bin new positions (cell lists and grid-tile order, Sec. 3) and keep them in
 * the plan, so that repeated applies with the same points and new forces --
 * an iterative solve -- skip the position work.  Followed by
 * ewald_apply_forces(). */
ewald_status ewald_set_positions(ewald_plan_t plan, const double *x, void *stream);

/* Apply with the positions of the last ewald_set_positions()/ewald_apply()
 * and new forces f. */
ewald_status ewald_apply_forces(ewald_plan_t plan, const double *f, double *u, void *stream);

/* Combined single and double layer apply (Sec. 2.3): u = the Stokeslet sum
 * of the forces f plus the double-layer sum over sources j and periodic
 * images of T(x_i - y_j + p) applied to q_j (x) n_j, with the stresslet
 * T_jlm(r) = -6 r_j r_l r_m / |r|^5 (u_j = sum_lm T_jlm q_l n_m; only the
 * symmetric part of q (x) n enters).  x, f, q, n: device, N x 3 row-major
 * FP64, read; u: device N x 3 FP64, written.  The double layer uses the
 * plan's xi, rc, M and P (chosen for the Stokeslet at the plan's tol); on
 * uniform points its error relative to its own size measured 2e-10 at
 * tol 1e-8 and 3e-8 at tol 1e-6 (oracle, CPU).  Near-field pairs in FP32
 * (from cell-local hi + lo coordinates) where the plan's FFTs are FP32
 * (tol >= 1e-6), else in FP64, summed in FP64; far field in the plan's grid
 * precision.
 * Double-single plans (FP32 bulk at tol <= 1e-7) spread the densities with
 * their double-single P2G onto FP64 grids and evaluate the near pairs in FP64.
 * The first call allocates the double layer's workspaces (two 3-component
 * grids and spectra, tile-order densities), all or none.  Errors: EINVAL
 * (NULL pointer), ENOMEM, ECUDA; non-finite q or n raise the device error flag
 * read by ewald_sync_status. */
ewald_status ewald_apply_combined(ewald_plan_t plan, const double *x, const double *f, const double *q,
                                  const double *n, double *u, void *stream);

/* The full apply with HOST arrays (x, f read; u written; N x 3 FP64 each).
 * Page-locked buffers (device-addressable) are read and written in place by
 * the kernels over the CPU-GPU link; pageable ones are copied through
 * plan-owned device buffers.  Synchronises `stream` before returning, so the
 * host buffers may be reused at once. */
ewald_status ewald_apply_host(ewald_plan_t plan, const double *x_host, const double *f_host,
                              double *u_host, void *stream);

/* Stage entry points (device arrays).  They share the plan's workspace.
 * ewald_near_field: u = u^N, the P2P sum of Sec. 2.1 eq. (potentials-near)
 *   over pairs with 0 < |r| <= rc, minus (4 xi/sqrt(pi)) f_j for every pair
 *   at r = 0: the far part of each pair Sec. 2 skips (the self term for
 *   j = i, coincident points otherwise), so that near + far = u.
 * ewald_far_field:  u = u^F_h, P2G -> FFT -> CNV -> IFFT -> G2P of Sec. 2.2
 *   (the self image is included; no self term is removed). */
ewald_status ewald_near_field(ewald_plan_t plan, const double *x, const double *f, double *u,
                              void *stream);
ewald_status ewald_far_field(ewald_plan_t plan, const double *x, const double *f, double *u,
                             void *stream);

/* P2G alone, eq. (p2g): writes the spread grid phi as 3 x M^3 FP64 values,
 * grid[c][iz][iy][ix] at g = h (ix, iy, iz) (device array of 3 M^3 doubles). */
ewald_status ewald_spread(ewald_plan_t plan, const double *x, const double *f, double *grid,
                          void *stream);

/* G2P alone, eq. (g2p): u(x_i) = h^3 sum_g w(x_i - g) v(g) for a caller grid v
 * in the layout of ewald_spread (device, 3 M^3 FP64, read only). */
ewald_status ewald_interp(ewald_plan_t plan, const double *x, const double *grid, double *u,
                          void *stream);

/* FFT -> CNV (eq. (sca), with the 1/M^3 of the inverse FFT folded in) -> IFFT
 * on a caller grid (3 M^3 FP64 in, 3 M^3 FP64 out; may alias). */
ewald_status ewald_fourier_convolve(ewald_plan_t plan, const double *grid_in, double *grid_out,
                                    void *stream);

/* Enable (1) or disable (0) per-stage CUDA-event timing of subsequent applies. */
ewald_status ewald_set_timing(ewald_plan_t plan, int enable);

/* Stage times of the last timed apply (synchronises on the recorded events). */
ewald_status ewald_stage_times(ewald_plan_t plan, ewald_stage_timing *out);

/* Synchronise `stream`, then report (and clear) the device-side error flag:
 * EWALD_EINVAL if an input coordinate was NaN/Inf since the last call. */
ewald_status ewald_sync_status(ewald_plan_t plan, void *stream);

/* Number of kernel launches (this library's own kernels, cuFFT excluded) that
 * one ewald_apply() issues with this plan, and the number of cuFFT executions. */
ewald_status ewald_launch_counts(ewald_plan_t plan, int32_t *kernels, int32_t *ffts);

/* Failure injection for tests (no counterpart in the paper): the nth next
 * device allocation of any plan (ewald_plan workspaces, the combined apply's
 * double-layer workspaces, the host apply's staging) fails as if the device
 * were out of memory, so the calling entry point returns EWALD_ENOMEM and
 * leaves the plan as it was before the call.  nth = 0 disarms it.  Process-
 * wide host state; nothing runs on the device.  Errors: EINVAL for nth < 0. */
ewald_status ewald_debug_fail_alloc(int32_t nth);

/* ---- Measured parameter choice and batches of boxes ----------------------
 * Sec. 2.4 leaves one free parameter once every term of eq. (ese) is held
 * below the tolerance, and picks it by minimising the modelled run time
 * T(rc) (with the GPU performance models of Sec. 5 as the better T).  Here
 * the free choice is the grid size M -- xi, rc and n_c then follow from the
 * planner's error bounds -- together with the P2G/G2P grid tile T, and T(M)
 * is measured on the device.  Every candidate meets the same error bound. */
enum { EWALD_TUNE_MODEL = 0, EWALD_TUNE_MEASURE = 1 };

/* The candidates the autotuner times for (N, L, tol, dtype), host only (no
 * GPU): first the planner's cost-model choice (= ewald_choose_params with no
 * override), then cuFFT-friendly multiples of 8 for M between 0.6x and 1.7x
 * that choice (at most 6 of them, spread over the range) with grid tile T = 8,
 * and the model's M with the other tile (T = 4), each only where the kernels
 * accept it -- and for double-single plans (EWALD_F32_BULK at tol <= 1e-7)
 * only tiles their double-single grid kernels take (T = 8), as other tiles
 * would fall back to FP64 P2G/G2P; P fixed at the planner's.  At most `cap` entries go to `cands`
 * (host array), their number to *n.
 * Errors: EINVAL for NULL pointers, cap < 1 or bad N, L, tol. */
ewald_status ewald_autotune_candidates(int64_t N, double L, double tol, ewald_dtype dtype,
                                       int32_t cap, ewald_params *cands, int32_t *n);

/* Choose the parameters for (N, L, tol, dtype).  EWALD_TUNE_MODEL: the first
 * candidate, nothing timed.  EWALD_TUNE_MEASURE: every candidate is planned
 * on the current device and timed (uniform random points of this N, one
 * warm-up apply, median of three event-timed applies); the fastest is
 * returned in *out and its median time (ms) in *ms (if ms != NULL; -1 for
 * MODEL).  Measured results are cached per (N, L, tol, dtype) for the life of
 * the process (ewald_autotune_clear empties the cache).  Candidates that do
 * not fit in memory are skipped.  Synchronises the device; not for use
 * inside stream capture.  Errors: EINVAL, ENOMEM (no candidate fits), ECUDA,
 * ECUFFT. */
ewald_status ewald_autotune(int64_t N, double L, double tol, ewald_dtype dtype, int32_t mode,
                            ewald_params *out, double *ms);
void ewald_autotune_clear(void);

/* A batch of independent boxes (own N, L, tol each; one dtype) applied with
 * one call.  Each box gets a plan with the autotuned parameters of
 * ewald_autotune(tune_mode), looked up at the half-octave representative
 * of its N (round(2^(round(2 log2 N) / 2))), so boxes of similar size share a
 * tuning.  The batch owns device buffers for every box's x, f (read) and u
 * (written), N x 3 FP64 each, reached through ewald_batch_buffers(); the
 * caller fills x and f there (any stream, ordered before the apply).
 * Boxes that share a grid size and FFT precision keep their grids side by
 * side in one batch-owned buffer (the boxes' plans use slices of it) and are
 * transformed by one batched cuFFT plan.  `nstreams` (1..64) is checked and
 * otherwise unused: every stage runs as one launch over all boxes.  Errors:
 * EINVAL for nbox < 1, NULL arrays, a bad N/L/tol entry, nstreams out of
 * range; then as ewald_plan_ex / ewald_autotune.  Nothing is left allocated
 * on failure. */
typedef struct ewald_batch_s *ewald_batch_t;
ewald_status ewald_batch_create(int32_t nbox, const int64_t *N, const double *L, const double *tol,
                                ewald_dtype dtype, int32_t tune_mode, int32_t nstreams,
                                ewald_batch_t *out);
/* Device pointers of box `box`'s x, f, u buffers (any of the outputs may be NULL). */
ewald_status ewald_batch_buffers(ewald_batch_t b, int32_t box, double **x, double **f, double **u);
ewald_status ewald_batch_get_params(ewald_batch_t b, int32_t box, ewald_params *out);
/* The plan of one box (owned by the batch; valid until ewald_batch_destroy). */
ewald_status ewald_batch_plan(ewald_batch_t b, int32_t box, ewald_plan_t *out);
/* Apply every box: u = apply(x, f) per box, as ewald_apply would give with
 * the box's plan.  The first call records the batch into one CUDA graph in
 * which every stage covers all boxes: binning (counters, keys, scans,
 * scatter), P2G and G2P (one launch per kernel instantiation: precision,
 * tile, support P), CNV, the grid copies G2P reads, the sums -- a block finds
 * its box by binary search -- the grouped FFTs, and, on a second stream, the
 * near field of all boxes as one persistent launch per P2P variant (FP32,
 * compensated FP32, double-single, FP64); every call launches that graph on
 * `stream`, asynchronously.  Calls on one batch must not overlap in time. */
ewald_status ewald_batch_apply(ewald_batch_t b, void *stream);
/* Kernel launches (this library's own kernels) and cuFFT executions in one
 * ewald_batch_apply. */
ewald_status ewald_batch_launch_counts(ewald_batch_t b, int32_t *kernels, int32_t *ffts);
void ewald_batch_destroy(ewald_batch_t b);

/* ---- Serving: a continuous-batching request loop -------------------------
 * No counterpart in the paper (it applies one suspension at a time).  A
 * request is one suspension that issues `napplies` successive applies, as
 * an iterative solve would: its positions are binned once and stay on the
 * device with the cell lists and grid order for all of them; apply t >= 1
 * uses f_t = f_{t-1} + perturb * n_t re-centred to zero mean, n_t ~ N(0, 1)
 * per component from Philox4x32-10 (Salmon et al., SC 2011) with counter
 * (i mod 2^32, i div 2^32, t, 0) for point i and key (seed mod 2^32,
 * seed div 2^32), u1, u2 from outputs 0, 1 and n_z from outputs 2, 3 as
 * (x + 1) / 2^32, Box-Muller n_x, n_y = sqrt(-2 ln u1) (cos, sin)(2 pi u2),
 * n_z = sqrt(-2 ln u3) cos(2 pi u4).  Only the last apply's velocities are
 * returned.  A scheduler thread admits queued requests while the summed
 * device footprint of the running ones (planner estimate plus request
 * buffers) stays within the budget and one of `max_active` slots is free:
 * shortest expected work first (N x napplies x a precision weight: FP32 1,
 * FP32 with FP64 FFTs 1.5, double-single 5, FP64 40), except that a request
 * queued for more than 2 s goes first (oldest first) and is not overtaken
 * while it does not fit.  Each runs on its own stream, with a CUDA stream
 * priority that falls with its expected work (log-spaced over the device's
 * priority range), so requests overlap on the GPU and the small ones'
 * kernels are scheduled first; finished ones free their room at once. */
typedef struct ewald_server_s *ewald_server_t;

typedef struct {
    int64_t N;             /* points */
    double L, tol;         /* box side, tolerance (as ewald_plan) */
    int32_t dtype;         /* ewald_dtype */
    int32_t napplies;      /* >= 1 */
    double perturb;        /* >= 0: force perturbation scale between applies */
    uint64_t seed;         /* Philox key of this request */
    const double *x_host;  /* HOST N x 3 positions; read until the request starts */
    const double *f_host;  /* HOST N x 3 forces of the first apply; read until it starts */
    double *u_host;        /* HOST N x 3: the last apply's u, written when it completes */
} ewald_request;

typedef struct {
    int64_t submitted, completed, failed, cancelled, queued, active;
    int64_t peak_footprint_bytes;  /* largest summed footprint of running requests */
    double particle_applies;       /* sum over completed requests of N * napplies */
    double p50_ms, p99_ms, mean_ms; /* arrival (submit) to completion, completed requests */
    double throughput;             /* particle_applies / (last completion - first arrival), per s */
} ewald_server_summary;

enum { EWALD_REQ_QUEUED = 0, EWALD_REQ_RUNNING = 1, EWALD_REQ_DONE = 2, EWALD_REQ_FAILED = 3,
       EWALD_REQ_CANCELLED = 4 };

/* Create a server on the current device.  hbm_budget_bytes > 0;
 * 1 <= max_active <= 256; start_paused != 0 admits nothing until
 * ewald_server_resume().  Errors: EINVAL, ENOMEM, ECUDA. */
ewald_status ewald_server_create(int64_t hbm_budget_bytes, int32_t max_active, int32_t start_paused,
                                 ewald_server_t *out);
/* Queue a request (copied; the host arrays it points to are not).  Returns at
 * once with a ticket.  Errors: EINVAL (NULL or bad fields, as ewald_plan for
 * N, L, tol), ENOMEM when the request alone exceeds the budget (never
 * admissible; nothing is queued). */
ewald_status ewald_server_submit(ewald_server_t s, const ewald_request *r, int64_t *ticket);
/* State (EWALD_REQ_*) and arrival-to-completion latency (ms; -1 until done).
 * Returns the request's failure status for a failed request. */
ewald_status ewald_server_poll(ewald_server_t s, int64_t ticket, int32_t *state, double *latency_ms);
/* Wait up to timeout_s seconds for the request to finish: EWALD_ETIMEOUT if it
 * has not (the request goes on), its failure status if it failed. */
ewald_status ewald_server_wait(ewald_server_t s, int64_t ticket, double timeout_s);
/* Cancel a request that is still queued (EINVAL once it has started). */
ewald_status ewald_server_cancel(ewald_server_t s, int64_t ticket);
ewald_status ewald_server_resume(ewald_server_t s);
ewald_status ewald_server_stats(ewald_server_t s, ewald_server_summary *out);
/* Drop the queued requests, let the running ones finish, release everything. */
void ewald_server_destroy(ewald_server_t s);

/* Host-only helpers, usable without a GPU (tests, tooling).
 * ewald_window_eval: the plan-time piecewise-polynomial fit of the Kaiser-
 *   Bessel window w_0 for support P and polynomial degree nu (Sec. 2.2 and
 *   Sec. 4): evaluates w_0(t h) at n offsets t (in grid units) into w;
 *   returns the fit's maximum error on a dense check grid in *max_err.
 * ewald_window_hat: the closed-form transform of the truncated window at n
 *   wave numbers k (for grid spacing h), as the plan uses in CNV. */
ewald_status ewald_window_eval(int32_t P, int32_t nu, int64_t n, const double *t, double *w,
                               double *max_err);
ewald_status ewald_window_hat(int32_t P, double h, int64_t n, const double *k, double *what);

/* The near field of ewald_near_field() without any device allocation.  The
 * paper has no counterpart: this entry point exists for callers that cannot
 * call cudaMalloc -- code running inside a pre-sized memory pool or a custom
 * allocator that owns the device, plugins that must leave the host
 * application's allocator alone, and paths that must not synchronise the
 * device, which cudaMalloc/cudaFree may do.  Its workspace is one fixed
 * array in device memory (about 7 MB) that every GPU loading this library
 * holds until the process exits.
 *   N      points (1 .. 32768; larger N returns EWALD_EUNSUPPORTED)
 *   prm    host struct read for L, xi, rc, near_ds (1: double-single pairs),
 *          near_f64 (with near_ds 0 -- 1: FP64 kernels, 0: FP32), tol (FP32
 *          below 1e-6 uses the compensated form) and n_c (<= 0:
 *          floor(L / rc)); n_c must be <= 16 and the cutoff may reach at most
 *          two cells (else EWALD_EUNSUPPORTED).  ewald_get_params() of a plan
 *          gives a consistent set.
 *   x, f   device, N x 3 FP64 (read); u: device, N x 3 FP64 (written): u^N as
 *          ewald_near_field() defines it.
 * The first call on a device looks up the array's address on that device;
 * make it before any stream capture.  All calls share the array and it keeps
 * the last call's contents; each call clears what must start at zero on
 * `stream`, and calls that overlap on the GPU (other streams or threads)
 * race.  A NaN or Inf coordinate makes every entry of u NaN (the call itself
 * returns before the device has looked at the data). */
ewald_status ewald_near_field_noalloc(int64_t N, const ewald_params *prm, const double *x,
                                      const double *f, double *u, void *stream);

/* Measured FMA-pipe peaks of `device` (TFLOP/s, an FMA counted as 2 flops):
 * 8 independent FP32 (then FP64) FMA chains per thread, 4 blocks of 256
 * threads per SM, the best of three timed launches after a warm-up (~10 ms of
 * device time in all).  The ALU-bound stages' roofline denominators besides
 * the peak derived from unit counts and clocks; there is no library measure
 * of these pipes.  Synchronises the device.  EWALD_ECUDA on a CUDA error. */
ewald_status ewald_probe_fma_peaks(int32_t device, double *fp32_tflops, double *fp64_tflops);

#ifdef __cplusplus
}
#endif
#endif /* EWALD_GB300_H */
