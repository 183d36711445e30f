/*
 * msqoc.h — C ABI of the GB300 multiple-shooting quantum-optimal-control evaluator.
 *
 * One call evaluates the multiple-shooting penalty objective of Petersson, Guenther, Chung,
 * "A time-parallel multiple-shooting method for large-scale quantum optimal control"
 * (arXiv 2407.13950), Sec. 3, Eq. penalty-fcn:
 *
 *     P(alpha, W^1..W^{M-1}) = J_V(U^M(t_M)) + mu/2 sum_{m<M} ||U^m(t_m) - W^m||_F^2,
 *
 * where window m propagates U^m from U^m(t_{m-1}) = W^{m-1} (W^0 = identity embedding of the
 * essential subspace; Eqs. sch-op, sch-ic) with the implicit midpoint rule (Sec. 5) under
 * H(t) = H_s + sum_k d_k(t) a_k + conj(d_k(t)) a_k^+ (Eqs. ctrl-ham, dj-ctrl), and
 * J_V(U) = ||U||^2/E - |<V,U>_F|^2/E^2 is the generalized infidelity (Eq. mod-infid, n := E).
 * The gradient is the exact discrete adjoint of the midpoint rule (Sec. 5): Eq. grad-int
 * for alpha and Eq. dP-dW (with the factor 2 of Appendix B, Eq. dT-dW-j) for W.
 *
 * Model conventions
 *   - q subsystems, L levels each (the first `ness` essential); N = L^q rows, E = ness^q
 *     columns.  Full index i = sum_k l_k L^(q-1-k) (subsystem 0 most significant); essential
 *     column e = sum_k b_k ness^(q-1-k).
 *   - Drift: H_s = sum_k -xi_k/2 a_k^+a_k^+a_k a_k - sum_{k<l} xi_kl a_k^+a_k a_l^+a_l
 *     (transmons with self- and cross-Kerr in per-qubit rotating frames)
 *     + sum_k detune_k a_k^+ a_k + sum_{k<l} J_kl (a_l^+ a_k + a_l a_k^+) (the paper's
 *     Eq. sys-ham: detuning omega_k - omega_rot and dipole exchange).
 *   - Controls: d_k(t) = sum_f exp(i Omega_kf t) sum_s (alpha1_kfs + i alpha2_kfs) B_s(t),
 *     quadratic cardinal B-splines on knots j*dtau, dtau = T/(d1-2), spline s centred at
 *     (s - 1/2) dtau (Sec. 2 and Sec. 5: d1 = T/dtau + 2).  alpha layout [k][f][s][2],
 *     d = 2 d1 sum_k N_f(k) doubles.
 *   - Time grid: h = T/nsteps, controls evaluated at t_{n+1/2} = (n + 1/2) h, window m
 *     (1-based) owns steps [floor((m-1) nsteps/M), floor(m nsteps/M)).
 *   - Target V: N x E, column-major complex; NULL selects QFT_E on the essential rows
 *     (Sec. 5: V_jk = kappa^{jk}/sqrt(E), kappa = exp(2 pi i/E)), guard rows zero.
 *
 * Memory layouts (complex = interleaved re, im doubles)
 *   alpha     : d doubles.
 *   W         : (M-1) x E x N complex = 2 N E (M-1) doubles; W^m column c row i at
 *               2*(((m-1) E + c) N + i).  W^0 is never passed.
 *   grad_W    : same layout as W; entry (re, im) = (dP/dRe W, dP/dIm W) (real-valued
 *               formalism, Sec. 5).
 *   pen       : M-1 doubles, pen[m-1] = mu/2 ||U^m(t_m) - W^m||^2.
 *
 * Pointers: every array argument may be host or device memory (detected with
 * cudaPointerGetAttributes).  With device outputs the call is asynchronous on `stream`;
 * with any host output it synchronizes `stream` before returning.  Inputs are read during
 * the call (host) or until the stream work completes (device).  The caller owns every
 * array it passes; the library owns the device buffers it allocates for a problem.
 *
 * Errors: every function returns MSQOC_OK (0) or a negative msqoc_status; no C++ exception
 * crosses this boundary.  msqoc_last_error() copies the calling thread's last message.
 * Calls on the same problem must not overlap (they share its scratch buffers); different
 * problems may be used from different threads and streams.
 */
#ifndef MSQOC_H
#define MSQOC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t msqoc_status;

#define MSQOC_OK 0
#define MSQOC_ERR_INVALID_ARG (-1)   /* malformed description, size or pointer */
#define MSQOC_ERR_OUT_OF_MEMORY (-2) /* a device allocation failed */
#define MSQOC_ERR_NOT_ADMITTED (-3)  /* refused by a memory budget (batch/serving layer) */
#define MSQOC_ERR_CUDA (-4)          /* a CUDA runtime call failed */
#define MSQOC_ERR_TIMEOUT (-5)       /* a bounded device wait gave up (status word set) */
#define MSQOC_ERR_UNSUPPORTED (-6)   /* valid input outside what the kernels implement */
#define MSQOC_ERR_INTERNAL (-7)

/* Linear solver inside each implicit-midpoint step.
 *  MIXED: iterative refinement with FP32 inner corrections and a residual accurate to FP64
 *         round-off (formed in compensated FP32 where the step's contraction factor allows,
 *         else in FP64); the step is solved to FP64 round-off.  With one thread per fiber the
 *         state is kept as FP64 plus an FP32 carry and updated in compensated FP32 where the
 *         diagonal step |2 kappa| = h |D| <= 2^-4.5 (msqoc_selftest_carry).  Default.
 *  FP64 : diagonal-preconditioned fixed-point iteration carried out entirely in FP64. */
#define MSQOC_SOLVER_DEFAULT 0
#define MSQOC_SOLVER_FP64 1
#define MSQOC_SOLVER_MIXED 2

typedef struct msqoc_hamiltonian {
    int32_t nqubits;        /* q >= 1 */
    int32_t nlevels;        /* L >= 2, same for every subsystem */
    int32_t ness;           /* essential levels per subsystem, 1 <= ness <= L */
    const double* xi;       /* [q] self-Kerr xi_k (rad/ns); host memory */
    const double* xi_cross; /* [q*q] row-major, entry (k,l) with k<l used; NULL = 0; host */
    const double* detune;   /* [q] or NULL; host */
    const double* jx;       /* [q*q] row-major dipole exchange J_kl, (k,l) with k<l used; NULL = 0;
                               nonzero only with nlevels = 2 (else MSQOC_ERR_UNSUPPORTED); host */
} msqoc_hamiltonian;

typedef struct msqoc_controls {
    const int32_t* ncarriers; /* [q] carriers per subsystem, >= 1; host */
    const double* carriers;   /* [sum ncarriers] Omega_kf (rad/ns), subsystem-major; host */
    int32_t nsplines;         /* d1 >= 3 spline coefficients per carrier */
} msqoc_controls;

typedef struct msqoc_options {
    int32_t solver;        /* MSQOC_SOLVER_* */
    int32_t col_block;     /* columns per sweep tile (1 <= col_block <= E; col_block N/L <= 256
                              threads with one thread per fiber (384 with FIBER_LEAN), 2 col_block N/L <= 384 with
                              lane pairs, 4 col_block N/L <= 384 with lane quads; tiles run
                              along the window-major column list and may cover two windows; a
                              one-warp tile must divide E); 0 = automatic */
    int32_t ckpt_interval; /* K: forward states kept for the adjoint sweep.  1 = every midpoint
                              state (history of nsteps * E * N complex); K > 1 = the state every
                              K steps of each window, each K-step segment recomputed before its
                              adjoint sweep (one more forward sweep of work); 0 = automatic (1
                              unless that history exceeds a quarter of the device memory, then
                              64) */
    int32_t profile;       /* 1 = record CUDA events around every kernel (msqoc_kernel_times) */
    int32_t layout;        /* MSQOC_LAYOUT_*: threads per (column, fiber) of the sweep tiles */
    int32_t window_first;  /* a window range [window_first, window_last] (1-based) of the
                              M-window problem: the problem is then one shard of it (below);
                              0 and 0 = every window */
    int32_t window_last;
    int32_t steps_per_sync; /* time steps per synchronisation of a sweep tile with the midpoint
                              history in device memory: the forward stages this many steps'
                              states in shared memory and stores them with one wait, the adjoint
                              fetches this many steps per mbarrier phase (one group ahead).
                              1..8; 0 = 1.  Larger groups take more shared memory; a group that
                              does not fit is MSQOC_ERR_INVALID_ARG */
} msqoc_options;

/* Shards (window ranges).  Sec. 3 makes the windows independent given the window states: the
 * objective is a sum of window terms, window m reads W^{m-1} (its initial state) and W^m (the
 * target of its penalty), and dP/dW^m = mu (W^m - U^m(t_m)) - 2 Lambda^{m+1}(t_m) joins window
 * m's end state to window m+1's adjoint at its start (Eq. dP-dW; Sec. 4 splits the windows over
 * processes the same way).  A problem created with window_first = a, window_last = b runs only
 * windows a..b on the global time grid of the M-window problem (window m owns the steps
 * floor((m-1) N_T / M) .. floor(m N_T / M) - 1) and exchanges nothing itself:
 *   W (input)  : the window states it reads, W^k for k = max(a-1, 1) .. min(b, M-1), in the
 *                layout of W (nW = 2 N E times their count; W^0, the identity embedding, and
 *                the nonexistent W^M are never passed);
 *   P_out      : the sum of its windows' terms (pen_m for m < M, J for m = M);
 *   J_out      : J when b = M, else 0;  pen_out: pen_m for m = a .. min(b, M-1);
 *   grad_alpha : the sum of its windows' contributions (Eq. grad-int over windows a..b);
 *   grad_W     : for the same k as W, the terms of dP/dW^k it owns: mu (W^k - U^k(t_k)) when
 *                k >= a and -2 Lambda^{k+1}(t_k) when k + 1 <= b.
 * Summing P, grad_alpha and the overlapping grad_W blocks of shards that partition 1..M gives
 * the whole problem's values: two consecutive shards overlap in one window state, to which the
 * earlier shard contributes its penalty term and the later one -2 Lambda of its first window.
 * Roll-outs, roll-out estimates and batches take whole problems only (MSQOC_ERR_UNSUPPORTED). */

/* Sweep kernel families.  FIBER: one thread per fiber (the L entries of a column along the last
 * subsystem), the choice for problems whose tiles fill the GPU.  PAIR: a lane pair per fiber,
 * one thread computing the real and one the imaginary component of every complex result: half
 * the FP64 instructions per thread, so steps run faster when the tiles are too few to fill the
 * GPU (small problems, the paper's QFT cases).  QUAD: 2-level subsystems only (and at most 6
 * exchange-coupled pairs): a lane pair per entry of the fiber, four threads per fiber, a
 * quarter of its work per thread.  FIBER_LEAN: one thread per fiber like FIBER, compiled for
 * 168 registers a thread instead of 255: tiles of up to 384 threads, and two 6-warp tiles fit
 * on an SM, 12 warps whose stalls it hides better (the choice for the large 4-transmon
 * workloads); FIBER keeps the registers for problems whose tiles are few.  AUTO: chosen with
 * the column block by the library's makespan model.  A family the problem does not admit is
 * rejected (MSQOC_ERR_INVALID_ARG). */
#define MSQOC_LAYOUT_AUTO 0
#define MSQOC_LAYOUT_FIBER 1
#define MSQOC_LAYOUT_PAIR 2
#define MSQOC_LAYOUT_QUAD 3
#define MSQOC_LAYOUT_FIBER_LEAN 4

/* Kernels of one evaluation, in launch order, as indexed by msqoc_kernel_times. */
#define MSQOC_KERNEL_CONTROLS 0  /* control evaluation at the step midpoints */
#define MSQOC_KERNEL_FORWARD 1   /* forward sweep of every window */
#define MSQOC_KERNEL_TERMINAL 2  /* window terminal conditions and objective terms */
#define MSQOC_KERNEL_ADJOINT 3   /* adjoint sweep with the fused gradient quadrature */
#define MSQOC_KERNEL_FINALIZE 4  /* deterministic reductions and the W-gradient */
#define MSQOC_NKERNELS 5

typedef struct msqoc_problem msqoc_problem;

/* Create a problem: validates the description, packs the model tables (drift diagonal,
 * preconditioner, strides, spline and carrier tables, target) into device memory of the
 * current device and sizes the scratch buffers.  mu <= 0 selects mu = 2/E (Sec. 5).
 * nwindows M >= 1 (M = 1 is single shooting) and M <= nsteps.  opt may be NULL.
 * target: N x E complex column-major host array or NULL (QFT_E).  *out receives the
 * handle (NULL on failure). */
msqoc_status msqoc_create_problem(const msqoc_hamiltonian* H, const msqoc_controls* C,
                                  const double* target, double T, int64_t nsteps,
                                  int32_t nwindows, double mu, const msqoc_options* opt,
                                  msqoc_problem** out);

/* Sizes: d (control parameters), nW (doubles of the W vector, 2 N E (M-1); for a shard the
 * window states it reads) and the bytes of device memory the problem holds once a gradient has
 * been evaluated.  Any pointer may be NULL. */
msqoc_status msqoc_query(const msqoc_problem* p, int64_t* d, int64_t* nW, size_t* device_bytes);

/* Sweep layout of a problem: columns per tile, tiles (CTAs) per sweep launch, threads per
 * tile, the checkpoint interval K, the kernel family (MSQOC_LAYOUT_FIBER, _PAIR, _QUAD or
 * _FIBER_LEAN) and the steps per history synchronisation in use (after automatic
 * choices).  Any pointer may be NULL. */
msqoc_status msqoc_query_layout(const msqoc_problem* p, int32_t* col_block, int32_t* tiles,
                                int32_t* threads, int32_t* ckpt_interval, int32_t* layout,
                                int32_t* steps_per_sync);

/* Objective only (forward sweep of every window, Eq. penalty-fcn).  P_out: 1 double;
 * J_out (1 double) and pen_out (M-1 doubles; for a shard, one per penalty it owns) may be
 * NULL. */
msqoc_status msqoc_eval_objective(msqoc_problem* p, const double* alpha, const double* W,
                                  double* P_out, double* J_out, double* pen_out, void* stream);

/* Objective and gradient (forward sweep, terminal conditions Eq. terminal, discrete adjoint
 * sweep with the fused Eq. grad-int quadrature, Eq. dP-dW).  grad_alpha: d doubles;
 * grad_W: nW doubles, 2 N E (M-1) for a whole problem (may be NULL when nW = 0).  P_out may be
 * NULL. */
msqoc_status msqoc_eval_gradient(msqoc_problem* p, const double* alpha, const double* W,
                                 double* P_out, double* grad_alpha, double* grad_W, void* stream);

/* Roll-out (Sec. 5, initialisation of the window states): propagate the identity embedding
 * W^0 over the whole time grid [0, T] as one window under the controls alpha, sequentially in
 * time, and store the state at every window boundary: W_out^m = U(t_m), m = 1..M-1 (layout of
 * W).  With these window states every continuity penalty vanishes (to rounding) and the
 * objective equals the single-shooting infidelity.  This sweep cannot be parallelised over the
 * windows: it runs E / col_block tiles for all N_T steps.  W_out: host or device. */
msqoc_status msqoc_rollout(msqoc_problem* p, const double* alpha, double* W_out, void* stream);

/* Roll-out infidelity estimate (Eq. rollout-infid-est) from the problem's last evaluation
 * (objective or gradient): J + (2/sqrt(E)) sqrt(J) S + S^2/E with S = sum_m ||C^m||_F and
 * ||C^m||_F = sqrt(2 pen_m / mu), an upper bound of the infidelity of the rolled-out state
 * that needs no sequential sweep (the paper's stopping criterion).  est_out: 1 double, host
 * or device. */
msqoc_status msqoc_rollout_estimate(msqoc_problem* p, double* est_out, void* stream);

/* Regularization of the optimisation problem (Sec. 5: a Tikhonov term and a control-pulse
 * energy penalty):
 *   R = (gamma_tik / 2) ||alpha||^2 + gamma_energy * (h/T) sum_n sum_k |d_k(t_{n+1/2})|^2,
 * the time-averaged energy (1/T) int_0^T sum_k |d_k(t)|^2 dt taken with the midpoint rule on
 * the problem's time grid (the quadrature of the gradient, Eq. grad-int), and its gradient dR/dalpha
 * (d doubles, layout of alpha; may be NULL).  The paper uses gamma_tik = 1e-3/d and
 * gamma_energy = 1e-3.  Independent of W and of the problem's last evaluation (neither is
 * read or changed).  alpha, R_out, grad_alpha: host or device; the gammas must be finite and
 * >= 0 (else MSQOC_ERR_INVALID_ARG). */
msqoc_status msqoc_eval_regularization(msqoc_problem* p, const double* alpha, double gamma_tik,
                                       double gamma_energy, double* R_out, double* grad_alpha,
                                       void* stream);

/* ---- L-BFGS steps of the client optimiser (Sec. 5 minimises P + R with L-BFGS; the paper uses
 * PETSc/TAO, this library its own kernels).  The optimisation vector x has n entries; its first
 * nb entries (the control coefficients) may carry box bounds |x_i| <= lim_i (lim: nb entries,
 * NULL when nb = 0).  An entry at its bound whose gradient pushes it outward is *active*: held
 * fixed for the iteration.  The memory is a ring of cap slots (cap <= MSQOC_LBFGS_MAXMEM) of
 * pairs s_j = x_{j+1} - x_j, y_j = g_{j+1} - g_j, stored as S, Y [cap][n]; rho[slot] =
 * 1/<s, y>, yy[slot] = <y, y>; the m newest pairs are used, the newest in slot head - 1
 * (mod cap).  Every array is device memory; each call is one CTA on `stream`, asynchronous,
 * with sums in a fixed order (bitwise repeatable).  No paper counterpart beyond the choice of
 * L-BFGS. */
#define MSQOC_LBFGS_MAXMEM 64

/* Search direction d = -H pg by the two-loop recursion (pg: the gradient g with its active
 * entries zeroed; H: the limited-memory inverse Hessian with initial scaling <s,y>/<y,y> of the
 * newest pair; m = 0 gives d = -pg/||pg||), zeroed on the active set; slope_out = <pg, d>
 * (< 0 for a descent direction).  d_out: n doubles; slope_out: 1 double. */
msqoc_status msqoc_lbfgs_direction(int64_t n, int64_t nb, const double* x, const double* g,
                                   const double* lim, const double* S, const double* Y,
                                   const double* rho, const double* yy, int32_t cap, int32_t m,
                                   int32_t head, double* d_out, double* slope_out, void* stream);

/* Trial point of the projected line search: x_new = x + step d, the first nb entries clipped to
 * [-lim, lim]; dec_out = <g, x_new - x> (the first-order change of the objective). */
msqoc_status msqoc_lbfgs_trial(int64_t n, int64_t nb, const double* x, const double* d, double step,
                               const double* lim, const double* g, double* x_new, double* dec_out,
                               void* stream);

/* Memory update: s_out = x_new - x, y_out = g_new - g (n doubles each, e.g. the next ring slot
 * of S and Y), sy_yy_out = (<s, y>, <y, y>) (2 doubles). */
msqoc_status msqoc_lbfgs_update(int64_t n, const double* x, const double* x_new, const double* g,
                                const double* g_new, double* s_out, double* y_out, double* sy_yy_out,
                                void* stream);

/* Release every resource of the problem (synchronizes the device first). NULL is a no-op. */
msqoc_status msqoc_destroy_problem(msqoc_problem* p);

/* Copy the calling thread's last error message (NUL-terminated, truncated to len).
 * Returns the full message length. */
int32_t msqoc_last_error(char* buf, size_t len);

/* Device time (ms) of each kernel of the last evaluation on a problem created with
 * options.profile = 1, measured with CUDA events recorded on the evaluation's stream around
 * each launch (synchronizes on the last event).  ms[MSQOC_NKERNELS]; kernels that did not run
 * in the last evaluation report 0.  Not part of the paper's method: measurement support. */
msqoc_status msqoc_kernel_times(msqoc_problem* p, float* ms);

/* FP64 throughput of the current device, measured with a fused-multiply-add microbenchmark
 * (8 independent FMA chains per thread on every SM, best of several runs).  *tflops receives
 * FP64 TFLOP/s (an FMA counts 2 flops).  Used as the roofline denominator of the sweeps; not
 * part of the paper's method. */
msqoc_status msqoc_measure_fp64_peak(double* tflops);

/* Self-test of the sweeps' failure path (not an operation of the paper): one thread waits on
 * an mbarrier phase with the sweeps' bounded wait (a poll loop of at most `spins` try-waits,
 * 1 <= spins <= 2^18, the limit the sweeps use), after completing the phase itself when
 * arrive != 0 and otherwise on a phase that nothing completes.  Returns MSQOC_ERR_TIMEOUT when
 * the wait gave up (the device status word was set), MSQOC_OK when the phase completed;
 * *seconds_out (may be NULL) receives the launch's duration.  The device stays usable either
 * way.  Synchronizes the device. */
msqoc_status msqoc_selftest_bounded_wait(int64_t spins, int32_t arrive, double* seconds_out);

/* Self-tests of the compensated FP32 arithmetic the mixed solver uses for the gradient products
 * of Eq. grad-int and for the implicit-midpoint state update (not operations of the paper), on
 * the host (on_device = 0)
 * or on the current device (on_device != 0: device copies, a kernel, copies back; synchronizes).
 * All arrays are host arrays of n entries; -2000 <= scales <= 2000.
 *
 * msqoc_selftest_split: x_i 2^-sh as hi_i + lo_i, two floats: hi the value rounded to 24 bits
 * (ties away from zero), lo the remainder rounded to nearest; |x_i 2^-sh - hi_i - lo_i| <=
 * 2^-48 |x_i 2^-sh| for 2^-74 <= |x_i 2^-sh| < 2^127, lo_i = 0 below 2^-74, both zero below
 * 2^-126 (and for FP64 zeros and subnormals).
 *
 * msqoc_selftest_dot: *out = sum_i x_i y_i formed from the splits of x_i 2^-shx and y_i 2^-shy
 * with exact FP32 product and two-sum error terms, returned as one double scaled by
 * 2^(shx + shy); its error is about 2^-47 sum_i |x_i y_i| (plus the partial sums' magnitudes).
 *
 * msqoc_selftest_carry: n steps of the state update of the implicit midpoint rule (Sec. 5) on
 * one complex entry, U_{j+1} = R U_j + 2 d_j with R = 2P - 1, P = 1 / (1 + i kappa) the diagonal
 * preconditioner entry (P: 2 doubles, re and im; kappa = -Im P / Re P) and d_j the corrections
 * (d: n complex entries, 2n doubles, split into two floats in units 2^-sh as the solver's
 * corrections are), formed as the mixed solver forms it where |2 kappa| <= 2^-4.5: the state
 * an FP64 part u plus an FP32 carry, u' + carry' = u + carry + 2 kappa (Im b, -Re b) + 2 d_j with
 * b = P (u + carry) (R - 1 = -2 i kappa P).  u0: 2 doubles; out: the final u + carry (2 doubles).
 * -896 <= sh <= 896; Re P must lie in (1/2, 1] and (2 kappa)^2 <= 2^-9.
 *
 * Errors: MSQOC_ERR_INVALID_ARG for negative n, NULL arrays (n > 0), scales out of range or (carry
 * test) P outside the bounds; MSQOC_ERR_CUDA for a failed device step. */
msqoc_status msqoc_selftest_split(const double* x, int64_t n, int32_t sh, int32_t on_device, float* hi, float* lo);
msqoc_status msqoc_selftest_dot(const double* x, const double* y, int64_t n, int32_t shx, int32_t shy,
                                int32_t on_device, double* out);
msqoc_status msqoc_selftest_carry(const double* u0, const double* P, const double* d, int64_t n, int32_t sh,
                                  int32_t on_device, double* out);

/* ---------------------------------------------------------------------------------------
 * Batched evaluation (many problems per launch).
 *
 * Not an operation of the paper: it packs the independent evaluations of many problems (the
 * paper's method applied to many pulses at once) into few kernel launches.  Problems of one
 * shape (levels, subsystems) and solver share each sweep launch, whose CTAs take the tiles of
 * all of them, so small problems no longer leave most of the GPU idle.
 *
 * A batch refers to problems created on the current device; they must outlive it and must
 * not be evaluated on their own while a batched evaluation of them is in flight (they share
 * buffers).  flags:
 *   MSQOC_BATCH_GRADIENT: allocate every problem's history buffers now (needed by
 *                         msqoc_batch_eval_gradient);
 *   MSQOC_BATCH_GRAPH   : capture each kind of evaluation into a CUDA graph on its first use
 *                         and replay the graph afterwards (one launch per evaluation).
 * Inputs are staged per problem with msqoc_set_inputs; a batched evaluation computes every
 * problem on its staged inputs and leaves the results in the problem's output buffers, read
 * with msqoc_get_objective / msqoc_get_gradient.  All calls are stream-ordered on `stream`;
 * msqoc_get_* synchronize it (and report a device status error) when any output is host
 * memory.  A problem's numbers are the same alone and in any batch up to rounding: each
 * problem's tiles are its own, only their scheduling changes. */
#define MSQOC_BATCH_GRADIENT 1
#define MSQOC_BATCH_GRAPH 2
#define MSQOC_BATCH_SLOTS 4   /* concurrent subset evaluations (msqoc_batch_eval_subset) */

typedef struct msqoc_batch msqoc_batch;

msqoc_status msqoc_batch_create(msqoc_problem* const* problems, int32_t n, int32_t flags,
                                msqoc_batch** out);
/* Stage alpha (d doubles) and W (2 N E (M-1) doubles; NULL when M = 1) for the next batched
 * evaluation of p: stream-ordered copies from host or device arrays. */
msqoc_status msqoc_set_inputs(msqoc_problem* p, const double* alpha, const double* W, void* stream);
msqoc_status msqoc_batch_eval_objective(msqoc_batch* b, void* stream);
msqoc_status msqoc_batch_eval_gradient(msqoc_batch* b, void* stream);
/* Evaluate only the problems members[0..n-1] (indices into the batch's problem array; objective
 * or, with gradient != 0, objective and gradient) in shared launches, without a graph: the
 * continuous-batching step of a server, where the set of ready problems changes every time.
 * slot (0 <= slot < MSQOC_BATCH_SLOTS) selects the staging buffers of the subset's tile list;
 * evaluations in flight at the same time must use different slots (and, to overlap on the
 * device, different streams); a slot is reused once its previous tile list has been copied
 * (the call waits for that).  A problem must not be in two evaluations in flight. */
msqoc_status msqoc_batch_eval_subset(msqoc_batch* b, const int32_t* members, int32_t n,
                                     int32_t gradient, int32_t slot, void* stream);
/* Results of p's last batched evaluation (J_out and pen_out may be NULL; P_out may be NULL
 * for the gradient). */
msqoc_status msqoc_get_objective(msqoc_problem* p, double* P_out, double* J_out, double* pen_out,
                                 void* stream);
msqoc_status msqoc_get_gradient(msqoc_problem* p, double* P_out, double* grad_alpha,
                                double* grad_W, void* stream);
msqoc_status msqoc_batch_destroy(msqoc_batch* b);

/* ---------------------------------------------------------------------------------------
 * Objective evaluation that allocates no device memory.
 *
 * The paper has no counterpart to this entry point; it exists for callers that cannot
 * allocate device memory themselves: a plug-in inside a host application whose memory
 * manager owns the whole device heap, a process that reserved all device memory up front,
 * or a control loop that cannot afford cudaMalloc / cudaFree (cudaFree synchronizes the
 * device).  msqoc_create_problem allocates, so such callers cannot hold a problem handle.
 *
 * msqoc_eval_objective_noalloc computes the same P (and J, pen) as msqoc_create_problem
 * followed by msqoc_eval_objective with default options and the given solver, running the
 * same kernels, but every table and intermediate it needs lives in one fixed scratch array
 * of MSQOC_NOALLOC_SCRATCH_BYTES bytes that the library declares statically: each GPU that
 * loads the library holds it from module load until the process exits.  The call makes no
 * cudaMalloc, cudaFree or other allocating call.
 *
 * Arguments: the description (H, C, target, T, nsteps, nwindows, mu) as for
 * msqoc_create_problem; solver is MSQOC_SOLVER_*; alpha, W, P_out, J_out, pen_out as for
 * msqoc_eval_objective (host or device memory; J_out and pen_out may be NULL).
 * Size limit: a problem needs (16 (q + sum N_f) + 32) nsteps bytes of control tables plus
 * 32 N E M bytes of target, window and end states, plus a few KB of small tables (each
 * region rounded up to 256 bytes); one that does not fit is rejected with
 * MSQOC_ERR_INVALID_ARG before any device work, whatever kind of pointers it passes.  The
 * 4-transmon workload (N = 81, E = 16, 2 carriers each, 100000 steps, M <= 256) fits.
 * Synchronization: the call is synchronous; it returns once the results are in the outputs.
 * Set-up: every call looks up the device address of the scratch array on the current device
 * (cudaGetSymbolAddress, a host-side query; nothing is cached, so a context that was reset
 * and recreated is served at the array's new address).  Make the first call on a device
 * before any stream capture, since it may load the library's module on that device.
 * Sharing: every call on a device uses the same scratch array, which keeps the previous
 * call's contents (what must start at zero is cleared by each call).  Calls that overlap on
 * the GPU (from several host threads or streams at once) race on it and corrupt each
 * other's results: serialize them.
 */
#define MSQOC_NOALLOC_SCRATCH_BYTES (32u * 1024u * 1024u)

msqoc_status msqoc_eval_objective_noalloc(const msqoc_hamiltonian* H, const msqoc_controls* C,
                                          const double* target, double T, int64_t nsteps,
                                          int32_t nwindows, double mu, int32_t solver,
                                          const double* alpha, const double* W, double* P_out,
                                          double* J_out, double* pen_out, void* stream);

/* Sweep kernel family, tile width and steps per history synchronisation by measurement (not
 * an operation of the paper): for every admissible (family, columns per tile) pair, a problem
 * of the same description, step size and window count but only probe_steps steps per window
 * is created with it and its objective + gradient is timed (one warm-up, two timed
 * evaluations, CUDA events on the default stream); then the fastest pair is timed with 2, 4
 * and 8 steps per synchronisation (those whose history groups fit the shared memory), unless
 * opt->steps_per_sync fixes it.  *col_block, *layout and *steps_per_sync (the last two may be
 * NULL) receive the fastest (use them as msqoc_options.col_block, .layout, .steps_per_sync);
 * widths[i], layouts[i], depths[i], ms[i] (i < *n_out <= max_out; may be NULL) the candidates
 * tried and their milliseconds per evaluation.  alpha: d control coefficients (host) of a
 * typical iterate (the iteration counts of the step solver depend on the control amplitude);
 * NULL = alternating +-2 pi 0.002 rad/ns.  opt: solver, checkpoint interval, layout and steps
 * per synchronisation as for msqoc_create_problem (layout AUTO tries every family the problem
 * admits; col_block and the window range are ignored).  Allocates and frees temporary
 * problems; synchronizes the device. */
msqoc_status msqoc_autotune(const msqoc_hamiltonian* H, const msqoc_controls* C, double T,
                            int64_t nsteps, int32_t nwindows, double mu, const msqoc_options* opt,
                            const double* alpha, int32_t probe_steps, int32_t* col_block,
                            int32_t* layout, int32_t* steps_per_sync, int32_t* widths,
                            int32_t* layouts, int32_t* depths, float* ms, int32_t max_out,
                            int32_t* n_out);

/* Library version as major*10000 + minor*100 + patch. */
int32_t msqoc_version(void);

#ifdef __cplusplus
}
#endif

#endif /* MSQOC_H */
