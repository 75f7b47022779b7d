/*
 * wf.h - C ABI of the GB300 Wiener-filter MAP library.
 *
 * The method (Horowitz, Seljak & Aslanyan, arXiv:1810.00503):
 *   data model d = R s + n, S diagonal in Fourier space, N diagonal in pixels
 *   (Sec. 2, eq. ddecomp); MAP field by minimising
 *   chi^2(s) = s^T S^-1 s + (d - R s)^T N^-1 (d - R s)      (Sec. 2.2, eq_chi)
 *   with its analytic gradient (eq_cost) and an L-BFGS quasi-Newton driver
 *   (Sec. 2.2); band powers from simulations (Sec. 2.4-2.5: eq. el, blmv,
 *   fisher, eq:wfmv).
 *
 * Variables.  The library works in whitened Fourier modes: the state is
 *   s_hat = U s_w, the unitary 2-D DFT of a real white field s_w, and the
 *   signal map is x = A s_w with A = U^-1 R(k) diag(sqrt P) U.  In these
 *   variables chi^2 = |s_hat|^2 + (d - x)^T W (d - x), W = mask * Ninv.
 *   The gradient returned is the full d chi^2 / d s_hat (twice the paper's g).
 *   For two channels (joint E/B shear, App. C) R(k) is the per-mode
 *   Kaiser-Squires rotation [[c, -s], [s, c]], c = (kx^2 - ky^2)/k^2,
 *   s = 2 kx ky / k^2, with s = 0 on the Nyquist row and column; one channel
 *   has R = 1.
 *
 * Layouts (row-major, C-contiguous):
 *   pixel maps   [count][C][n][n]            y (row) then x (column)
 *   spectra      [count][C][n][n/2+1]        complex (re, im) pairs, numpy
 *                                            rfft2 layout, unitary scaling
 *   mask         [n][n] uint8, 1 = observed, shared by the channels
 *   P            [C][n][n/2+1] real: variance of each unitary Fourier mode of
 *                the signal, >= 0; the kx = 0 and kx = n/2 columns must be
 *                symmetric under ky -> n - ky.
 * n is a power of two in [8, 1024]; C is 1 or 2.  The _rect calls take ny x nx
 * maps instead (each side a power of two in [8, 1024]): read [n][n] as
 * [ny][nx] and [n][n/2+1] as [ny][nx/2+1].
 *
 * Pointers.  Every array pointer is a DEVICE pointer owned by the caller,
 * unless stated otherwise; the library never frees a caller pointer nor keeps
 * it after the call returns (wf_problem_create copies what it needs).  Calls
 * are ordered on the CUDA stream passed in (NULL = legacy default stream).
 *
 * Errors.  Every call returns a wf_status; WF_OK is 0.  On failure
 * wf_last_error() returns a message for the calling thread.  Calls that launch
 * work return after enqueueing it unless documented to synchronise.
 */
#ifndef WF_H_
#define WF_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  WF_OK = 0,
  WF_EINVAL = 1,         /* bad argument: size, channel count, null pointer, negative Ninv or P */
  WF_ENONFINITE = 2,     /* a NaN or Inf in the inputs or met during a solve */
  WF_ENOMEM = 3,         /* device allocation failed */
  WF_ECUDA = 4,          /* a CUDA runtime call failed */
  WF_ENOTCONVERGED = 5,  /* iteration limit reached; outputs are still written */
  WF_ELINESEARCH = 6,    /* no decrease along the search direction */
  WF_ETIMEOUT = 7        /* a bounded device wait gave up */
} wf_status;

typedef enum { WF_FP64 = 0, WF_MIXED = 1 } wf_precision;  /* MIXED: FP32 fields, FP64 sums */
/* Step length along each L-BFGS direction p (Sec. 2.2 uses a generic L-BFGS).
 * chi^2 is quadratic, so one Hessian-vector pass q = H p gives chi^2 and its
 * slope along p in closed form: phi(a) = chi2 + a g.p + a^2 p.Hp / 2.
 *   WF_LS_EXACT: the minimiser a = -g.p / p.Hp.
 *   WF_LS_WOLFE: the strong Wolfe search of Nocedal & Wright (Alg. 3.5 with
 *     zoom, Alg. 3.6): trial a = 1, doubling, safeguarded quadratic
 *     interpolation, constants c1 and c2, run on phi. */
typedef enum { WF_LS_EXACT = 0, WF_LS_WOLFE = 1 } wf_line_search;
typedef enum { WF_F32 = 0, WF_F64 = 1 } wf_dtype;

typedef struct wf_handle wf_handle;
typedef struct wf_problem wf_problem;

/* One input map.  All pointers are device pointers, read once by
 * wf_problem_create (or wf_problem_set_data for d).  Values have the dtype
 * given to wf_problem_create. */
typedef struct {
  const void* d;               /* [C][n][n] data (0 is fine on masked pixels) */
  const unsigned char* mask;   /* [n][n] 1 = observed, 0 = masked */
  const void* Ninv;            /* [C][n][n] inverse noise variance, >= 0, finite */
  const void* P;               /* [C][n][n/2+1] signal power per mode, >= 0 */
} wf_map;

typedef struct {
  int lbfgs_m;        /* L-BFGS memory (pairs kept), 1..32; default 10 */
  int max_iter;       /* iteration limit; default 10000 */
  double gtol_rel;    /* stop when |g| <= gtol_rel |g0|; default 1e-6; 0 = off */
  double dchi2_abs;   /* stop when |chi2_k - chi2_{k-1}| < dchi2_abs (the paper's
                         Delta chi^2 rule, Sec. 3); default 0 = off */
  int refresh_every;  /* recompute the true gradient from the data every this many
                         iterations (0 = only at the start and the end); default 0 */
  int check_every;    /* iterations between host polls of the convergence flags
                         (one synchronisation each); default 16 */
  int use_graphs;     /* capture check_every iterations in one CUDA graph; default 1 */
  void* stream;       /* cudaStream_t for all work of the call; NULL = default stream */
  int line_search;    /* wf_line_search; default WF_LS_EXACT */
  int pad_;
  double c1, c2;      /* strong Wolfe constants, 0 < c1 < c2 < 1; default 1e-4, 0.9 */
  unsigned long long seed;  /* Philox key of draws made on the device (bandpower_estimate
                               with no caller-supplied fields); default 0 */
  long long spin_limit;     /* bound of every device-side wait (the TMA-fed inverse column
                               stage's copies), in SM clock cycles; 0 = default (4e9, about
                               2 s at the maximum clock).  A wait that runs out stops the maps
                               of that block with WF_ETIMEOUT; the context stays usable. */
  int inject_timeout_map;   /* diagnostic, 0 = off (default).  k > 0: the inverse column stage
                               never issues the copies of map k-1's tiles, so the bounded wait
                               runs out: exercises the timeout path without a GPU fault.  The
                               solve then uses the TMA-fed inverse column stage, untuned
                               (WF_EINVAL with a forced variant that does not). */
  int autotune;             /* 1 (default): the first solve of each shape (n, C, precision,
                               lbfgs_m, batch size) on a handle times the FFT-stage variants
                               (kernels, radix plans, tile widths) on the problem's own buffers,
                               with a full history ring, and keeps the fastest (cached in the
                               handle); 0: the built-in defaults */
  int fft_variant;          /* 0 (default): as autotune says.  Otherwise a forced variant,
                               100000 f + 10000 e + 1000 a + 100 b + 10 c + d: a = inverse column
                               stage (1 persistent, TMA-fed; 2 ping-pong; 3 in-place), b = row
                               stage (1 ping-pong; 2 in-place), c, d = column and row tiles 1, 2
                               or 4 times narrower than the widest, f, e = radix plans of the
                               ping-pong column and row passes (0: larger radices first,
                               1024 = 16 x 8 x 8; 1: ascending, 8 x 8 x 16; 2: radix 32 first
                               for lengths 512 and 1024, 32 x 32).  wf_problem_variant reports
                               the one in use: a = 1 becomes 2 on maps whose column tile is
                               wider than 128 values (few rows, many columns), which one TMA box
                               cannot hold. */
  int history;              /* 0 (default): off.  k > 0: every map keeps a device ring of its
                               last k iterations' records (k, chi2, |g|/|g0|, step, evals), the
                               convergence trace the paper plots (Sec. 3, Fig. of chi2 against
                               iteration); read with wf_solver_history.  40 k bytes per map. */
} wf_opts;

typedef struct {
  int iters;          /* L-BFGS iterations taken */
  int evals;          /* operator applications (Hessian-vector and gradient passes) */
  int status;         /* wf_status of this map */
  int fft_variant;    /* FFT-stage variant the solve ran (wf_opts.fft_variant code).  Results
                         are bitwise reproducible for a given variant (every sum runs in a
                         fixed order); with autotune the variant comes from timing and may
                         differ between runs, and variants round differently: pass this back
                         as wf_opts.fft_variant to repeat a solve bit for bit. */
  double chi2;        /* final chi^2 (true value from the data at the returned state) */
  double gnorm_rel;   /* final |g| / |g0| (true gradient) */
} wf_solve_stats;

/* Library plumbing (the calls up to wf_opts_default have no counterpart in
 * the paper; they manage devices, memory and errors for the calls that do).
 *
 * Library handle: owns the twiddle tables for the current device and charges
 * every device allocation of its problems, solvers and band-power runs to one
 * workspace.  workspace_limit: most device bytes the handle may hold at once
 * (0 = no limit); an allocation beyond it fails with WF_ENOMEM and the call
 * returns without side effects.  Create one per device and thread of use.
 * Returns WF_ECUDA if no device is usable.  wf_destroy does not free the
 * handle's problems: destroy those first. */
wf_status wf_create(wf_handle** out, size_t workspace_limit);
wf_status wf_destroy(wf_handle* h);

/* FFT-stage variant the problem's last solver start chose (wf_opts.fft_variant
 * encoding); before any start, the defaults.  Plumbing: how the transforms of
 * Sec. 2.2's objective are executed, not what they compute. */
wf_status wf_problem_variant(const wf_problem* p, int* variant);

/* Device bytes the handle holds now (twiddle tables, problems, solver state).
 * Plumbing. */
wf_status wf_workspace_used(const wf_handle* h, size_t* bytes);

/* Message for the last failing call on this thread ("" if none).  The pointer
 * stays valid until the next call from the same thread.  Plumbing. */
const char* wf_last_error(void);

/* Fill *o with the defaults listed in wf_opts (the solver settings of
 * Sec. 2.2 and Sec. 3 the paper leaves open, as listed there). */
void wf_opts_default(wf_opts* o);

/* Prepare a batch of `count` maps of one shape (n, C) for repeated use:
 * converts the inputs to the working precision, forms W = mask * Ninv and
 * sqrt(P), checks them (negative or non-finite values -> WF_EINVAL /
 * WF_ENONFINITE) and allocates the device workspace: about
 * (4 + 2 m) C n^2 values of the working type per map plus scratch.
 * maps: HOST array of `count` descriptors holding device pointers.
 * dtype: WF_F32 or WF_F64, the type of the maps' d, Ninv and P.  Every state
 * or output array of later calls (s, grad, v, hv, s0, s_out, x, x_out, z,
 * noise, d_out and the d of wf_problem_set_data) uses the WORKING type:
 * double for WF_FP64, float for WF_MIXED (complex = two of them).
 * precision: WF_FP64 computes everything in FP64; WF_MIXED keeps fields and
 * FFTs in FP32 and all reductions and L-BFGS scalars in FP64.
 * Synchronises the stream once (to read the input check).  Paper: Sec. 2
 * (data model) and Sec. 2.2 (eq_chi: the inputs of the objective). */
wf_status wf_problem_create(wf_handle* h, const wf_map* maps, int count, int n, int C,
                            int dtype, int precision, int lbfgs_m, void* stream,
                            wf_problem** out);

/* The same for rectangular maps of ny rows by nx pixels, both powers of two
 * in [8, 1024]; wf_problem_create(n) is wf_problem_create_rect(n, n).  Every
 * [n][n] array of this header is then [ny][nx] (pixel maps, x = the last
 * axis), every half-plane array [n][n/2+1] is [ny][nx/2+1], and the unitary
 * DFT carries (ny nx)^-1/2.  Pixels are square: mode (my, mx) has the
 * wavevector 2 pi (mx / nx, my / ny) / pixel, which is what the E/B rotation
 * of App. C (C = 2) is evaluated on; P and the band tables are per mode and
 * so take any convention the caller chooses.  Every call on the problem
 * takes the rectangular shape (the solver, its checkpoints and
 * wf_map_solve_many included); wf_eval_noalloc takes square maps only. */
wf_status wf_problem_create_rect(wf_handle* h, const wf_map* maps, int count, int ny, int nx, int C,
                                 int dtype, int precision, int lbfgs_m, void* stream,
                                 wf_problem** out);
/* Free a problem and its solver state (synchronises the device).  Plumbing. */
wf_status wf_problem_destroy(wf_problem* p);

/* Replace the data maps d of every map (device [count][C][n][n], working
 * type; the d of Sec. 2.1's data model); masked pixels are ignored.  Stream
 * ordered, no synchronisation. */
wf_status wf_problem_set_data(wf_problem* p, const void* d, void* stream);

/* One objective + gradient pass per map (Sec. 2.2, eq_chi and eq_cost):
 *   chi2[b] = |s_hat_b|^2 + (d_b - x_b)^T W_b (d_b - x_b)
 *   grad[b] = d chi2 / d s_hat = 2 (s_hat - sqrt P R^T U W (d - x))
 * s: device [count][C][n][n/2+1] complex of the working type (whitened modes,
 * Hermitian-consistent in the kx = 0 and kx = n/2 columns); grad: same shape,
 * written; chi2: device double [count], written; any may alias nothing else.
 * Stream ordered, no synchronisation. */
wf_status wf_eval(wf_problem* p, const void* s, void* grad, double* chi2, void* stream);

/* Band-amplitude form of the prior (Sec. 2.3, eq. pilin: S = sum_l q_l S_fid
 * restricted to band l, q_l = Theta_l / Theta_fid,l).  Scales the problem's
 * signal power by q[band(k)] on every mode (modes with band id -1 keep their
 * power); the original P is kept, so later calls replace the scale.
 * band: device int16 [C][n][n/2+1], ids < n_b; q: device double [n_b] > 0,
 * shared by all maps.  Stream ordered. */
wf_status wf_problem_set_band_scale(wf_problem* p, const int16_t* band, const double* q, int n_b,
                                    void* stream);

/* wf_eval plus the derivative of chi^2 with respect to the band amplitudes
 * q_l of Sec. 2.3 (eq. pilin), computed in the adjoint stage (Sec. 2.2,
 * eq_cost): dlogq[b][l] = d chi2_b / d log q_l
 *   = -sum over the full-plane modes k of band l of Re(conj(a_k) s_k),
 * a = sqrt(P) R^T U W (d - x) at the current scale (divide by q_l for
 * d chi2 / d q_l).  band: device int16 [C][n][n/2+1]; dlogq: device double
 * [count][n_b], written.  Other arguments as wf_eval.  Stream ordered. */
wf_status wf_eval_bands(wf_problem* p, const void* s, void* grad, double* chi2, const int16_t* band, int n_b,
                        double* dlogq, void* stream);

/* Hessian-vector product of chi^2 (twice eq_curv): hv = 2 (v + A^T W A v),
 * same layouts as wf_eval.  Stream ordered. */
wf_status wf_hess_vec(wf_problem* p, const void* v, void* hv, void* stream);

/* Signal map x = A s_w for a whitened state (the Wiener-filtered map when s is
 * the MAP, Sec. 2.2: the field s of eq_chi in pixel space; App. C for E/B):
 * s [count][C][n][n/2+1], x [count][C][n][n].  Stream ordered. */
wf_status wf_signal_map(wf_problem* p, const void* s, void* x, void* stream);

/* MAP solve of every map by L-BFGS with an exact line search (Sec. 2.2; the
 * objective is quadratic, so the step along p is -g.p / p.Hp, the point where a
 * strong-Wolfe search would stop).  Starts from s0 (device, spectrum layout) or
 * from 0 when s0 is NULL.  Writes s_out (device, spectrum layout) and, if
 * x_out is not NULL, the signal map A s_out (device, pixel layout).
 * stats: HOST array of `count` entries, written.  Returns the worst per-map
 * status (WF_ENOTCONVERGED if any map hit max_iter; outputs still written).
 * Synchronises the stream every opts->check_every iterations. */
wf_status wf_map_solve(wf_problem* p, const wf_opts* opts, const void* s0, void* s_out,
                       void* x_out, wf_solve_stats* stats);

/* MAP solve to a certified accuracy, with the state kept in FP64 (Sec. 2.2:
 * the MAP minimises eq_chi).  Certificate: the whitened half-Hessian
 * I + A^T W A has every eigenvalue >= 1, so |s - s_MAP| <= |grad chi2(s)| / 2
 * for any state s; the call stops map b once |grad chi2(s_b)| / 2 <=
 * cert_tol |s_b|, both evaluated in FP64, which bounds the relative L2 error
 * of s_b by cert_tol (to first order in cert_tol).  Rounds of iterative
 * refinement: the FP64 gradient g at the FP64 state; then the device L-BFGS
 * in the problem's working precision minimises chi2(s + delta) over delta
 * from delta = 0 (its gradient starting at g, Hessian-vector passes only),
 * and s += delta in FP64.  The first round runs to opts->gtol_rel (relative
 * to |g| at its start), later rounds only as far as the certificate needs.
 * For a WF_MIXED problem every operator pass of the rounds runs in FP32 and
 * only the outer evaluations run in FP64, on exact FP64 copies of the
 * problem's working-precision d, W and sqrt(P) (allocated on the first call,
 * about 3 C n^2 doubles per map plus the scratch).  A state kept in FP32 can
 * fail the certificate on strongly curved modes even when it is accurate
 * (its rounding alone, times curvatures up to ~1e6), hence the FP64 state.
 * opts as for wf_map_solve; refresh_every is ignored (the outer evaluations
 * are the refreshes) and opts->max_iter bounds each round.  max_rounds: 1..1000.
 * s0: working type, spectrum layout, or NULL for 0.
 * s_out: DEVICE complex double [count][C][n][n/2+1], written.
 * cert: HOST double [count] or NULL: |grad chi2(s_b)| / (2 |s_b|) at s_out.
 * stats: HOST [count] or NULL: iters and evals summed over the rounds (outer
 * evaluations included), chi2 and |g| / |g0| from the FP64 evaluations,
 * status WF_OK when certified, WF_ENOTCONVERGED when max_rounds ran out.
 * Returns the worst per-map status; synchronises. */
wf_status wf_map_solve_refined(wf_problem* p, const wf_opts* opts, double cert_tol, int max_rounds,
                               const void* s0, void* s_out, double* cert, wf_solve_stats* stats);

/* The same solve in three calls, for callers that drive the iterations
 * themselves (benchmarks, checkpoints, time-sliced serving):
 *   wf_solver_start  prepares the state at s0 (NULL = 0) with the true gradient;
 *   wf_solver_step   runs exactly n_iter more iterations on every map still
 *                    active; if n_active is not NULL it synchronises once and
 *                    stores the number of maps still iterating (HOST int);
 *   wf_solver_finish applies the last step, evaluates the true chi^2 and
 *                    gradient, writes s_out / x_out (either may be NULL) and
 *                    stats (HOST, may be NULL), and synchronises.
 * opts are copied at start; stepping is stream ordered on opts->stream.
 * Paper: Sec. 2.2 (L-BFGS minimisation of eq_chi). */
wf_status wf_solver_start(wf_problem* p, const wf_opts* opts, const void* s0);
wf_status wf_solver_step(wf_problem* p, int n_iter, int* n_active);
wf_status wf_solver_finish(wf_problem* p, void* s_out, void* x_out, wf_solve_stats* stats);

/* Checkpoint and resume of a started solve, for long solves (the paper's
 * high-accuracy CMB solves run for thousands of iterations, App. B) and for
 * time-sliced serving.  The checkpoint holds every map's L-BFGS state: the
 * state s, the gradient, the m stored pairs, the FP64 scalars and Gram
 * matrices, the iteration counters, the options and the FFT-stage variant.
 *   wf_solver_state_size  bytes of the checkpoint of p's started solve;
 *   wf_solver_export      writes it to dst (host or device memory that CUDA
 *                         can address); synchronises the solver's stream;
 *   wf_solver_import      restores it into p, which must have the same n, C,
 *                         precision and map count (WF_EINVAL otherwise) and
 *                         the same inputs (not checked: the state means
 *                         nothing for other data), replacing any solve p had;
 *                         then wf_solver_step and wf_solver_finish continue
 *                         exactly where the exported solve stood, with the
 *                         same iterates bit for bit.  stream: the stream the
 *                         resumed solve runs on; the other options are the
 *                         checkpoint's.  Synchronises stream.
 * The convergence ring (opts.history) restarts empty on import. */
wf_status wf_solver_state_size(const wf_problem* p, size_t* bytes);
wf_status wf_solver_export(wf_problem* p, void* dst, size_t bytes);
wf_status wf_solver_import(wf_problem* p, const void* src, size_t bytes, void* stream);

/* Measurement hook, no counterpart in the paper (Sec. 2.2's iteration, timed
 * kernel by kernel).  Runs n_iter more iterations of a started solve with plain
 * launches and CUDA events around each kernel on the working stream, and
 * store the average duration in milliseconds of the six kernels of an
 * iteration in ms (HOST float[6]): direction / state update / dot products,
 * inverse column stage, row stage, forward column stage, q dot products,
 * scalar step.  Synchronises after every iteration.  Not part of the method;
 * used for roofline reports. */
wf_status wf_solver_profile(wf_problem* p, int n_iter, float* ms);

/* Convergence records of the solve started last on p with opts->history = cap
 * > 0 (during the solve after a step, or after wf_solver_finish).  out: HOST
 * double [count][cap][5]; map b's records are out[b][0 .. counts[b]-1], the
 * last min(k_b, cap) iterations in order, each (k, chi2, |g|/|g0|, step length
 * alpha, operator evaluations) as tracked by the solver (chi2 from the line
 * model, |g|^2 from the dot products; the refreshes and the closing
 * evaluation are exact); the rest is NaN.  counts: HOST int [count].
 * Synchronises the solver's stream.  WF_EINVAL if no solve with a history was
 * started. */
wf_status wf_solver_history(const wf_problem* p, double* out, int* counts);

/* MAP solves of several prepared problems at once, typically one per map
 * shape of a heterogeneous batch (Sec. 2.2; the simulations of Sec. 2.5 need
 * not share a size).  Every problem is started on its own internal stream,
 * ordered after opts->stream (first gradient).  When 2 to 8 problems share
 * the precision and C and opts->fft_variant is 0, each L-BFGS iteration of
 * the whole batch is one set of seven shared launches: every launch covers
 * the blocks of every problem's own grid, each block running the
 * single-problem kernel at its place in its problem's grid, every problem on
 * the ping-pong column and row stages with radix plan 0 and its own tile
 * widths (tuned per shape when opts->autotune, else the widest: variant
 * 2111), so each map ends exactly where its problem solved alone with the
 * variant its stats report ends.  Otherwise every problem is tuned and
 * runs its own kernels, a parallel branch per problem.  opts->check_every
 * iterations are captured in one CUDA graph, so that each round of the batch
 * is one graph launch (plain launches when opts->use_graphs is 0) and one
 * read of the active counts, until every map of every problem has stopped.
 * Refreshes (opts->refresh_every) run between rounds, per problem.  ps: HOST array of np distinct problems; s_out: HOST array of np
 * device outputs (each [count][C][n][n/2+1] in its problem's working type);
 * stats: HOST array of np HOST arrays (each of its problem's count) or NULL.
 * Starts from 0.  Returns the worst status over all maps; synchronises. */
wf_status wf_map_solve_many(wf_problem* const* ps, int np, const wf_opts* opts, void* const* s_out,
                            wf_solve_stats* const* stats);

/* Data synthesis for simulations (Sec. 2.5, steps 1-2; eq. blmv):
 * d_b = mask * (A z_b + noise_b), z and noise device [count][C][n][n] of the
 * working type (z white N(0,1), noise with variance 1/Ninv), d_out the same
 * shape.  Uses each map's mask and P.  Stream ordered. */
wf_status wf_simulate_data(wf_problem* p, const void* z, const void* noise, void* d_out,
                           void* stream);

/* Band powers of the MAP fields (Sec. 2.4, eq. el):
 *   E[b][l] = 1/(2 Theta_l) sum over full-plane modes k in band l of |s_hat_k|^2
 * s: device spectra [count][C][n][n/2+1] (working type); band: device int16
 * [C][n][n/2+1] band id per half-plane mode (-1 = none), ids < n_bands;
 * theta: device double [n_bands]; E: device double [count][n_bands], written.
 * Stream ordered. */
wf_status wf_band_energy(wf_problem* p, const void* s, const int16_t* band,
                         const double* theta, int n_bands, double* E, void* stream);

/* Band table from edges in |k| (the bands of Sec. 2.4, Pi_l = 1 on the modes
 * of band l).  Mode (row j, column kx) of the half plane has the signed row
 * frequency ky = j for j < n/2 and j - n otherwise, and |k| = kscale *
 * sqrt(kx^2 + ky^2) (kscale = 1: units of the fundamental 2 pi / L; 2 pi / L
 * for physical k, or 360 / (patch side in degrees) for multipoles l).  Band
 * l = 0..n_bands-1 holds the modes with edges[l] <= |k| < edges[l+1]; other
 * modes get -1.  edges: HOST, n_bands + 1 increasing values; out: HOST
 * [C][n][n/2+1], the same table for every channel.  Host only (no device
 * work); WF_EINVAL for bad sizes or edges that do not increase. */
wf_status wf_band_table(int n, int C, const double* edges, int n_bands, double kscale, int16_t* out);
/* The same for an ny x nx map of square pixels: mode (row j, column kx) has
 * |k| = kscale * sqrt((kx N / nx)^2 + (ky N / ny)^2), N = max(ny, nx) (units
 * of the fundamental of the longer side), so kscale = 2 pi / L for a longer
 * side L; out: HOST [C][ny][nx/2+1].  Both sides even, at least 2. */
wf_status wf_band_table_rect(int ny, int nx, int C, const double* edges, int n_bands, double kscale,
                             int16_t* out);

/* Inputs of the band-power estimator.  Pointers are DEVICE pointers except
 * sim_index.  The random fields z, noise and u are either all supplied by the
 * caller (any generator, working type) or all NULL: then the call draws them
 * on the device with wf_normal_draw's generator from opts->seed.  With
 * npix = C n^2 and g the global index of a simulation (sim_index[j], or j):
 *   z of simulation g:      stream 0, deviates g npix .. (g + 1) npix - 1
 *   noise of simulation g:  stream 1, the same deviates times Ninv^-1/2 on
 *                           observed pixels (0 on masked ones)
 *   u of band l for the Fisher map reusing simulation g: stream 2, deviates
 *                           (g n_bands + l) npix .. + npix - 1
 * so a simulation's fields do not depend on how simulations are split over
 * calls or GPUs. */
typedef struct {
  int n_bands;            /* bands, ids 0 .. n_bands-1 (1..64) */
  int n_sim;              /* noise-bias simulations (>= 1; cov_E needs >= 2, else NaN) */
  int n_fd;               /* Fisher simulations per band, 0..n_sim; the j-th reuses simulation j.
                             0 (a rank of a multi-GPU run that owns no Fisher map) leaves
                             fisher, cov and theta_hat as NaN */
  int leak_split;         /* 0 = off.  L in [1, n_bands): the leakage-bias alternative of App. C
                             for the joint E/B case (C = 2), bands 0..L-1 the E bands and
                             L..n_bands-1 the B bands.  Per-band Fisher maps are made for E
                             bands only; for the B bands one Fisher map per simulation j < n_fd
                             adds the fiducial power of every B band at once, d_j + M A_B u_Bj,
                             and F[l][l] = mean_j (E_l(that map) - E_l(d_j)) / Theta_fid,l is
                             their only Fisher term.  The cross blocks F[E][B] and F[B][E] and
                             the BB off-diagonal are 0: the E-to-B leakage enters through b,
                             the mean over the simulations at the fiducial power, as the noise
                             does.  fd_bands (all < L) and trunc_bands (<= L) then concern the
                             E block, a column's interpolation staying inside it; u holds one
                             more row, u_B, after the E rows, drawn on the device as band L's
                             row.  Saves (n_bands - L - 1) n_fd solves against the full form */
  const int16_t* band;    /* [C][n][n/2+1] band id of each half-plane mode, -1 = none */
  const void* z;          /* [n_sim][C][n][n] white signal fields, N(0, 1) */
  const void* noise;      /* [n_sim][C][n][n] noise realisations with variance 1/Ninv */
  const void* u;          /* [n_R][n_fd][C][n][n] white fields for the Fisher signals: n_R = the
                             bands with Fisher maps (n_bands, n_fd_bands, or L with leak_split),
                             plus 1 with leak_split */
  const long long* sim_index;  /* HOST [n_sim] global index (>= 0) of each simulation, used by
                                  the device draws; NULL = 0 .. n_sim-1 */
  const int* fd_bands;    /* HOST [n_fd_bands] ascending band ids that get Fisher maps (NULL =
                             every band).  The other bands' Fisher columns are interpolated
                             (Sec. 3.1: the matrix is smooth and nearly translation invariant):
                             between sampled s0 < l' < s1, F[l'+o][l'] = (1-t) F[s0+o][s0] +
                             t F[s1+o][s1], t = (l'-s0)/(s1-s0), a term whose row leaves the
                             matrix dropped; beyond the first or last sampled band the nearest
                             sampled column is shifted.  u then has n_fd_bands rows. */
  int n_fd_bands;
  int trunc_bands;        /* zero F[l][l'] for l, l' < trunc_bands with |l - l'| > trunc_width */
  int trunc_width;        /* (App. C: far off-diagonal EE terms, E bands first); 0, 0 = off */
  int out_on_device;      /* 0: the wf_bandpower_out arrays are HOST arrays; 1: DEVICE arrays */
} wf_bandpower_in;

/* Outputs of the band-power estimator: HOST arrays, or DEVICE arrays when
 * in->out_on_device, written. */
typedef struct {
  double* theta_fid;      /* [n_bands] mean of P over each band's modes */
  double* E;              /* [n_bands] E_l of the data's MAP field (eq. el) */
  double* bias;           /* [n_bands] noise bias b_l (eq. blmv) */
  double* fisher;         /* [n_bands * n_bands] F[l][l'] by finite differences (eq. fisher) */
  double* cov;            /* [n_bands * n_bands] F^-1 (eq. var) */
  double* theta_hat;      /* [n_bands] Theta_fid + F^-1 (E - b) (eq. eq:wfmv) */
  double* cov_E;          /* [n_bands * n_bands] sample covariance of E over the simulations */
  double* E_maps;         /* optional (NULL = not written): [1 + n_sim + n_R * n_fd][n_bands], n_R
                             the Fisher rows of wf_bandpower_in.u,
                             E of every solved map (data, simulations, Fisher maps), for callers
                             that combine simulations from several GPUs */
} wf_bandpower_out;

/* Band powers, noise bias, Fisher matrix and covariance from simulations, for
 * one data map (Sec. 2.4-2.5; procedure of Sec. 2.5):
 *   d_j   = M (A z_j + n_j)                         noise-bias simulations
 *   d_lj  = d_j + M A_l u_lj  (j < n_fd)            Fisher simulations, A_l = A
 *           restricted to band l, Delta Theta_l = Theta_fid,l
 *   every map is solved for its MAP field in one batched L-BFGS run (opts), then
 *   E_l per map (eq. el), b = mean_j E(d_j), F[l][l'] = mean_j (E_l(d_l'j) -
 *   E_l(d_j)) / Theta_fid,l', cov = F^-1, Theta_hat = Theta_fid + F^-1 (E - b).
 * data: HOST descriptor of the data map with DEVICE pointers (its P is the
 * fiducial spectrum); n, C, dtype, precision as for wf_problem_create.
 * stats: HOST array of 1 + n_sim + n_R * n_fd entries (data, simulations,
 * Fisher maps in that order) or NULL.  Allocates its working memory and frees it
 * before returning; synchronises opts->stream.  Returns WF_ENOTCONVERGED when a
 * solve hit max_iter (outputs still written), WF_ENONFINITE if F is singular. */
wf_status bandpower_estimate(wf_handle* h, const wf_map* data, int n, int C, int dtype, int precision,
                             const wf_bandpower_in* in, const wf_opts* opts, wf_bandpower_out* out,
                             wf_solve_stats* stats);
/* The same on rectangular ny x nx maps (Sec. 2.4-2.5 as above; shapes as
 * wf_problem_create_rect; npix = C ny nx in the draw rule above). */
wf_status bandpower_estimate_rect(wf_handle* h, const wf_map* data, int ny, int nx, int C, int dtype,
                                  int precision, const wf_bandpower_in* in, const wf_opts* opts,
                                  wf_bandpower_out* out, wf_solve_stats* stats);

/* Band powers spread over several GPUs (Sec. 2.5: the simulations are
 * independent until the estimator averages them).  Each GPU runs
 * bandpower_estimate on its own simulations (sim_index keeps their random
 * fields independent of the split) and turns its per-map band energies
 * (wf_bandpower_out.E_maps, HOST [1 + n_sim + n_rows n_fd][n_bands]: data,
 * simulations, Fisher maps) into partial sums of
 * bandpower_sums_len(n_bands, n_rows) doubles:
 *   [J, J_fd, sum_j E_j (n_bands), sum_j E_j E_j^T (n_bands x n_bands),
 *    sum_{j < J_fd} (E(Fisher map of row k, j) - E_j)  (n_rows x n_bands, [k][l])]
 * n_rows: the Fisher rows of the call (the rows of wf_bandpower_in.u).
 * Partial sums of different simulations add entry by entry (one all-reduce of
 * a few KB).  Host only, no device work; bandpower_sums_len returns 0 for bad
 * sizes. */
size_t bandpower_sums_len(int n_bands, int n_rows);
wf_status bandpower_sums(const double* E_maps, int n_bands, int n_sim, int n_fd, int n_rows, double* sums);

/* The estimator from summed partial sums (eq. blmv, eq. fisher, eq:wfmv),
 * the same code bandpower_estimate ends with:
 *   b = sum E_j / J, cov_E = (sum E_j E_j^T - J b b^T) / (J - 1),
 *   F[l][l'] = (sum of Fisher row k(l') differences)_l / J_fd / Theta_fid,l',
 * the unsampled columns interpolated, the truncation and the leakage-bias
 * form applied as wf_bandpower_in describes, cov = F^-1 (Gauss-Jordan in
 * FP64), Theta_hat = Theta_fid + F^-1 (E - b).
 * rules: the wf_bandpower_in of the contributing calls; n_bands, leak_split,
 * fd_bands, n_fd_bands, trunc_bands, trunc_width and out_on_device are read,
 * the rest ignored.  sums: HOST, the summed vector (its n_rows from rules);
 * E_data, theta_fid: HOST [n_bands], the data map's band energies and the
 * fiducial band powers (E_maps row 0 and theta_fid of any contributing call).
 * out: as bandpower_estimate (E_maps not written); host arrays need no
 * device.  J_fd = 0 leaves F, cov and theta_hat NaN.  WF_ENONFINITE if F is
 * singular, WF_EINVAL for inconsistent counts in the sums. */
wf_status bandpower_combine(const double* sums, const double* E_data, const double* theta_fid,
                            const wf_bandpower_in* rules, wf_bandpower_out* out);

/* Iterated fiducial (Sec. 2.3, after eq. pilin): n_iter band-power estimates
 * with the same random fields; between two, the fiducial P moves to the
 * estimate band by band, P <- P q_l on the modes of band l with
 * q_l = Theta_hat_l / Theta_fid,l kept in [q_min, q_max] (0 < q_min <= 1 <=
 * q_max: the regularisation, no band power becomes zero or negative).  The
 * paper starts from the true spectrum with every band scaled by U[0.01, 1] and
 * finds one re-estimate enough (n_iter = 2).  data->P is the starting
 * fiducial and is not modified; P_out (DEVICE, [C][n][n/2+1] in dtype, or
 * NULL) receives the fiducial of the last estimate; theta_hat_hist (HOST
 * [n_iter][n_bands] or NULL) every estimate's Theta_hat; out and stats are
 * those of the last estimate.  Needs in->n_fd >= 1.  Synchronises. */
wf_status bandpower_iterate(wf_handle* h, const wf_map* data, int n, int C, int dtype, int precision,
                            const wf_bandpower_in* in, const wf_opts* opts, int n_iter, double q_min,
                            double q_max, void* P_out, double* theta_hat_hist, wf_bandpower_out* out,
                            wf_solve_stats* stats);
/* The same on rectangular ny x nx maps (Sec. 2.3 and 2.5 as above; shapes as
 * wf_problem_create_rect). */
wf_status bandpower_iterate_rect(wf_handle* h, const wf_map* data, int ny, int nx, int C, int dtype, int precision,
                                 const wf_bandpower_in* in, const wf_opts* opts, int n_iter, double q_min,
                                 double q_max, void* P_out, double* theta_hat_hist, wf_bandpower_out* out,
                                 wf_solve_stats* stats);

/* Standard normal deviates on the device: out[k] = deviate offset + k of
 * (seed, stream_id), k < count, in dtype WF_F32 or WF_F64 (computed in FP64).
 * Generator: Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11).  Deviate i
 * comes from block j = i / 2: counter (j mod 2^32, j div 2^32, stream_id, 0),
 * key (seed mod 2^32, seed div 2^32); output words x0..x3 give
 * u1 = (2^26 (x0 >> 5) + (x1 >> 6) + 1/2) 2^-53, u2 likewise from x2, x3, and
 * the Box-Muller pair sqrt(-2 ln u1) (cos, sin)(2 pi u2): deviate 2j is the
 * cosine, 2j + 1 the sine.  The draws of the simulations of Sec. 2.5 (white
 * fields and noise) when the caller supplies none.  out: DEVICE pointer.
 * Stream ordered; WF_EINVAL for a null output or a bad dtype. */
wf_status wf_normal_draw(unsigned long long seed, unsigned int stream_id, unsigned long long offset,
                         size_t count, int dtype, void* out, void* stream);

/* Objective + gradient pass that allocates nothing (no counterpart in the
 * paper; an interface for callers that cannot allocate device memory, for
 * example because a framework's caching allocator or a pool reserved at
 * start-up owns it, or because their real-time rules forbid allocation after
 * initialisation - wf_problem_create allocates, this call does not).
 * Computes the same chi2 and grad as wf_eval for `count` maps of one shape,
 * from inputs the caller has already prepared, all DEVICE pointers of the
 * working type (double for WF_FP64, float for WF_MIXED):
 *   s    [count][C][n][n/2+1] complex   whitened state
 *   d    [count][C][n][n]               data, finite everywhere (its value
 *                                        where w = 0 does not matter, but a NaN
 *                                        or Inf there still reaches chi2 and
 *                                        grad through 0 * Inf; zero it)
 *   w    [count][C][n][n]               mask * Ninv, >= 0
 *   P    [C][n][n/2+1]                  signal power per mode, shared by the maps
 *   chi2 double [count], grad like s    outputs
 * Scratch lives in a static device array of 16 MiB per GPU that loads the
 * library (held until the process exits).  A call whose scratch would not fit
 * (it needs about (C n^2 + C n (n/2+1)) working-type values per map plus
 * 264 KiB of twiddle tables) returns WF_EINVAL; FP32 fits up to three 1024^2
 * maps per call.
 * The first call on a device resolves the array's address, writes the
 * twiddle tables and synchronises the legacy default stream until they have
 * landed, so that the kernels of any caller stream (blocking or not) see them;
 * make that first call before any stream capture.  The address and the tables
 * are cached per device for the life of the process: cudaDeviceReset after the
 * first call is not supported.  All calls share the one array and each call overwrites what it
 * uses before reading it, so nothing needs clearing between calls, but calls
 * that overlap on the GPU (different streams, or different host threads)
 * race on it: order them on one stream.  Inputs are not checked for
 * non-finite values.  Stream ordered, no synchronisation after the first call. */
wf_status wf_eval_noalloc(const void* s, const void* d, const void* w, const void* P, int n, int C,
                          int count, int precision, double* chi2, void* grad, void* stream);

/* Objective and gradient (Sec. 2.2, eq_chi and eq_cost; E/B rotation of
 * App. C) on maps whose sides are not powers of two: ny rows by nx pixels,
 * each side in [2, 1024] with no prime factor above 7 (e.g. 360, 640, 768,
 * 1000), any parity.  The same chi2 and gradient as wf_eval, with the unitary
 * DFT carrying (ny nx)^-1/2, the rotation at the wavevector (mx / nx, my / ny)
 * of square pixels and its sine 0 on the Nyquist line of an even side, and
 * the prior |s|^2 summed over the half plane with weight 1 on column 0 (and
 * on column nx/2 when nx is even), 2 elsewhere.  With d = NULL the data term
 * takes d = 0 and grad is the Hessian-vector product 2 (I + A^T W A) s
 * (eq_curv), chi2 then s^T s + x^T W x.
 * Stateless: no problem object, no solver (wf_problem_create_rect stays for
 * powers of two, where the fused kernels, the solver and the band powers
 * run).  DEVICE pointers, working type (double for WF_FP64, float for
 * WF_MIXED; complex = two of them):
 *   s     [count][C][ny][nx/2+1] complex   half-plane spectrum of real fields
 *                                           (the kx = 0 and Nyquist columns
 *                                           Hermitian, as rfft2 gives them)
 *   d     [count][C][ny][nx] or NULL        data, finite everywhere
 *   mask  uint8 [count][ny][nx]             1 = observed
 *   Ninv  [count][C][ny][nx]                inverse noise variance, >= 0
 *   P     [C][ny][nx/2+1]                   signal power per mode, >= 0, shared
 *   grad  like s, chi2 double [count]       outputs
 * Values are not checked.  Allocates its scratch (C ny (nx/2+1) complex per
 * map plus partial sums) from the handle, synchronises the stream and frees
 * it before returning.  Kernels: Stockham transforms with radix 4, 2, 3, 5 and
 * 7 passes in shared memory, one kernel per stage (inverse column, row,
 * forward column), partial sums added in a fixed order.
 * Errors: WF_EINVAL (null pointer, s == grad, count < 1, C not 1 or 2, a side
 * outside [2, 1024] or with a prime factor above 7, unknown precision),
 * WF_ENOMEM, WF_ECUDA. */
wf_status wf_eval_any(wf_handle* h, int count, int C, int ny, int nx, int precision, const void* d,
                      const uint8_t* mask, const void* Ninv, const void* P, const void* s, void* grad,
                      double* chi2, void* stream);

/* Bounds-checked build (no counterpart in the paper; the failure handling of
 * the test plan).  A separate copy of this library compiled with
 * -DWF_DEBUG_BOUNDS checks every shared-memory tile index of the FFT stages
 * and their global spectrum, pixel and scratch accesses, and the vector
 * accesses of the streaming L-BFGS kernels, against the buffers they address.
 * A bad index is counted, the first one recorded, and the access redirected
 * to element 0 of its buffer: nothing traps and no access leaves a buffer.
 * wf_debug_bounds reads the count over the library's kernel translation units
 * and, if first is not NULL (HOST long long [4]), the first violation: unit,
 * source line, index, limit.  mode 0 reads, 1 reads and clears, 2 first runs a
 * self-test kernel that checks one index five past the end of a tile (the
 * count grows by one).  Synchronises the device.  In the normal build it sets
 * *count = 0 and returns WF_EINVAL (not a bounds-checked build). */
wf_status wf_debug_bounds(unsigned long long* count, long long* first, int mode);

/* Measured fused multiply-add throughput of the current device, in flop/s
 * (2 per FMA), for dtype WF_F32 or WF_F64: every SM's resident blocks run
 * independent FMA chains for about 40 ms.  Measurement support for the ALU
 * roofline of the FP64 path; the paper has no counterpart.  Synchronises the
 * device's work it launches (a private stream); allocates one value. */
wf_status wf_alu_peak(int dtype, double* flops_per_s);

#ifdef __cplusplus
}
#endif

#endif /* WF_H_ */
