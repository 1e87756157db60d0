/*
 * pnscan.h -- C ABI of the GB300 scan library (libpnscan.so).
 *
 * Batched phase-space scan of the conservative post-Newtonian Hamiltonian of
 * spinning compact binaries, after Ran, Liu & Zhong, "GPU accelerated
 * manifold correction method for spinning compact binaries"
 * (arXiv:1802.00147):
 *   - H = H_N + H_1PN + H_2PN + H_SO(1.5PN) + H_S1S2(2PN) [+ H_QM]      Sec. 2, Eqs. 1-5
 *   - Hamilton's equations and spin precession                          Eqs. 6-9
 *   - a fixed-step explicit Runge-Kutta step (RK4, or RK5)              Sec. 3A
 *   - manifold correction after every step: spin lengths (Eq. 10), then
 *     dual scaling p = alpha p*, r = beta r* with (alpha, beta) from E and
 *     |J| by Newton's method                                            Eqs. 11-13, Sec. 3A
 *   - fast Lyapunov indicator from two nearby trajectories with periodic
 *     renormalisation                                                   Secs. 3B-3C
 *   - gravitational-wave polarisations of the mass quadrupole field
 *     (scan_waveform)                                                   Eq. 14, Sec. 4
 *   - a learned surrogate of the FLI (mlp_*) and the adaptive scan it
 *     drives (adaptive_*); not in the paper
 *
 * Units: G = c = M = 1.  r in M, p in mu, energies in mu, t in M, spins in
 * M^2 (S_i = chi_i m_i^2 S_hat_i).  A state is 12 doubles
 * (rx, ry, rz, px, py, pz, S1x, S1y, S1z, S2x, S2y, S2z).
 *
 * Conventions shared by every entry point:
 *   - Return 0 (PNSCAN_OK) or a negative PNSCAN_ERR_* code; scan_strerror()
 *     names it.  Per-orbit failures are reported in the status array, never
 *     in the return code.
 *   - Pointers are host pointers unless scan_params.device_ptrs == 1, in
 *     which case every array argument (of scan_params and of the calls on
 *     the handle) is a device pointer on the current CUDA device.
 *   - The caller owns every input and output array; the handle owns its
 *     device buffers (allocated with scan_params.alloc_fn if given, else
 *     cudaMalloc) and frees them in scan_destroy.
 *   - Work is issued on scan_params.cuda_stream (a cudaStream_t; NULL is the
 *     legacy default stream).  scan_setup and scan_run return once the work
 *     is queued; scan_read and scan_summary synchronise the stream.
 *   - A handle is not thread-safe; use one handle per host thread.
 *
 * The library computes nothing on the CPU: there is no host fallback.
 */
#ifndef PNSCAN_H
#define PNSCAN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- return codes ---- */
#define PNSCAN_OK 0
#define PNSCAN_ERR_ARG (-1)      /* invalid argument or size */
#define PNSCAN_ERR_CUDA (-2)     /* a CUDA runtime call failed */
#define PNSCAN_ERR_OOM (-3)      /* device allocation failed */
#define PNSCAN_ERR_TIMEOUT (-4)  /* host watchdog expired waiting for the stream */
#define PNSCAN_ERR_STATE (-5)    /* call out of order (e.g. scan_run before any initial state) */
#define PNSCAN_ERR_KERNEL (-6)   /* a bounded device-side wait gave up; results of the run are invalid */
#define PNSCAN_ERR_NODEVICE (-7) /* no CUDA device */

/* ---- per-orbit status (scan_read) ---- */
#define PNSCAN_ORBIT_RUNNING 0        /* not yet at t_end of the last run (never after a completed run) */
#define PNSCAN_ORBIT_DONE 1           /* reached t_end */
#define PNSCAN_ORBIT_MERGED 2         /* |r| < r_merge */
#define PNSCAN_ORBIT_ESCAPED 3        /* |r| > r_escape */
#define PNSCAN_ORBIT_FLI_SATURATED 4  /* FLI >= fli_cap at a renormalisation */
#define PNSCAN_ORBIT_NONFINITE 5      /* a state component became Inf/NaN */

/* ---- integrator scheduling ---- */
#define PNSCAN_SCHED_AUTO 0    /* use the autotuned choice (scan_autotune); else, at block 32, PAIR for
                                  n <= 128 x SMs and STATIC for n <= 256 x SMs (every orbit in one
                                  wave of one-warp blocks); COMPACT otherwise, at 62-step tasks
                                  unless chunk_steps is set */
#define PNSCAN_SCHED_STATIC 1  /* one orbit per thread, one pass over the batch */
#define PNSCAN_SCHED_QUEUE 2   /* persistent work-queue kernel over (32-orbit group, step chunk) tasks:
                                  claimed in chunk-major order from two groups per resident warp up,
                                  below that fixed contiguous shares per warp (bit-identical results) */
#define PNSCAN_SCHED_COMPACT 3 /* the work queue over epochs of 256, 512, 1024, ... steps, the running
                                  orbits compacted into a dense list between epochs (uneven batches) */
#define PNSCAN_SCHED_PAIR 4    /* two threads per orbit (main / shadow trajectory), one pass over the
                                  batch: half an orbit's serial time per step (small batches) */

/* Per-scan configuration.  scan_params_default() fills the paper's values. */
typedef struct scan_params {
    int64_t n;               /* number of orbits (>= 0) */
    const double *beta_m;    /* [n] mass ratio m1/m2 in (0, 1] (Sec. 2); NULL: taken from each cell
                                by scan_setup (scan_run with initial states is then refused) */
    const double *kappa1;    /* [n] quadrupole-monopole multipliers; NULL = 1 (black holes) */
    const double *kappa2;    /* [n] */
    int pn_order;            /* 0: Newtonian, 1: +1PN, 2: +2PN orbital terms (default 2) */
    int use_so;              /* 1.5PN spin-orbit (default 1) */
    int use_ss;              /* 2PN S1-S2 spin-spin, Eq. 3 (default 1) */
    int use_qm;              /* spin-induced quadrupole-monopole, Eqs. 4-5 (default 0) */
    int correct;             /* correction after every step: 0 none; 1 spin lengths (Eq. 10) and dual
                                scaling (Eqs. 11-13) (default); ablations: 2 spin lengths only;
                                3 spin lengths and velocity scaling p = a p* to E0 (Sec. 1) */
    int rk_order;            /* base integrator: 4 classical RK4 (default), 5 fifth-order Runge-Kutta
                                with the Dormand-Prince (1980) weights (the paper's RK5, Sec. 3A) */
    double newton_tol;       /* Newton stop: |d alpha|, |d beta| <= tol (default 1e-10, Sec. 3A) */
    int newton_max;          /* Newton iteration cap (default 50) */
    double newton_det_min;   /* a step whose dual-scaling Jacobian has |det| <= det_min
                                (|J11 J22| + |J12 J21|) is corrected by the split scaling
                                (newton_split_min), else restores E by scaling p alone
                                (default 1e-5) */
    int newton_apply_small;  /* 1: apply a Newton step, then stop if it was within newton_tol (default);
                                0: stop before applying a step already within newton_tol (the rule
                                under which Fig. 4's tolerance dependence appears) */
    double fli_d0;           /* separation of the two trajectories (default 1e-9) */
    int fli_renorm_steps;    /* renormalise every this many steps (default 100; <= 0: never) */
    double fli_thresh;       /* FLI above this is chaotic (default 6) */
    double fli_cap;          /* stop an orbit when FLI >= cap (default 0: never) */
    double r_merge;          /* stop when |r| < r_merge (default 6; <= 0: never) */
    double r_escape;         /* stop when |r| > r_escape (default 1e3; <= 0: never) */
    int device_ptrs;         /* 1: array arguments are device pointers (default 0) */
    void *cuda_stream;       /* cudaStream_t for all work of the handle (default NULL) */
    int schedule;            /* PNSCAN_SCHED_* (default AUTO) */
    int block_size;          /* threads per block, 32..128, multiple of 32 (0: 128) */
    int chunk_steps;         /* steps per work-queue task (0: 500; 62 where AUTO picks COMPACT) */
    int epoch_steps;         /* compacting schedule: steps per epoch (0: 256, 512, 1024, ... doubling) */
    int blocks_per_sm;       /* resident blocks per SM for the queue kernel (0: occupancy maximum) */
    int register_variant;    /* RK4 queue kernel variant: 2 -- up to 255 registers/thread, 2 resident
                                128-thread blocks per SM; 3 -- 168 registers, 3 blocks, per-orbit
                                constants in shared memory; 4 -- as 2 with the RK stage and trajectory
                                loops not unrolled (smaller code, bit-identical results)
                                (0: 4, or the autotuned choice) */
    int use_graph;           /* 1: capture a queue / compact run in a CUDA graph and replay it (default 1) */
    double sync_timeout_s;   /* host watchdog for the stream wait of synchronising calls: after this
                                many seconds they return PNSCAN_ERR_TIMEOUT with the work still
                                queued (default 0: wait forever).  With host output pointers the
                                device-to-host copies themselves wait for the preceding work; the
                                bound is strict with device pointers (or pinned host memory) */
    int queue_wait_limit_ms; /* bound on a work-queue task's wait for its predecessor; on expiry the
                                kernel sets an error flag and returns, and the next synchronising
                                call reports PNSCAN_ERR_KERNEL.  0 (default): 20 s plus 2 ms per
                                step of the chunk, so that long chunks never time out while their
                                predecessor is still running.  For testing this bound, the
                                environment variable PNSCAN_TEST_STALL_GROUP=g, read by
                                scan_create, makes 32-orbit group g of the handle's queue runs
                                withhold its first chunk, so the wait of its second chunk runs
                                out */
    void *(*alloc_fn)(size_t bytes, void *ctx);  /* optional device allocator (e.g. PyTorch's) */
    void (*free_fn)(void *ptr, void *ctx);
    void *alloc_ctx;
    int radiation_reaction;  /* 1: add the leading-order 2.5PN radiation reaction a_2.5PN to dp/dt
                                (Eq. 6) and correct toward reference E and |J| carried by their
                                integral-invariant relations dE/dt = (dH/dp).a, d|J|/dt =
                                J.(r x a)/|J| (Sec. 3B, orbit 3).  Every schedule; the queue
                                kernel runs its default variant whatever register_variant
                                (default 0) */
    double rr_gauge_a;       /* gauge constants of the force, Iyer & Will (1993) family:      */
    double rr_gauge_b;       /* a = (8/5) eta u^3 [A (n.p) n - B p], A = 3 (1 + b) p^2 +
                                (23 + 6 a - 9 b) u / 3 - 5 b (n.p)^2, B = (2 + a) p^2 + (2 - a) u
                                - 3 (1 + a) (n.p)^2; (4, 5): harmonic gauge (default) */
    double newton_split_min; /* where the dual scaling is singular (newton_det_min), restore E and
                                |J| by scaling p's tangential and radial parts, p = a p_t + g p_r
                                (r kept; L = a L*, so the Jacobian is triangular), if
                                |p_r.dH/dp| > split_min (|p_t.dH/dp| + |p_r.dH/dp|) and
                                |L*.J|/|J| > split_min |L*| (near circular orbits it is as
                                ill-conditioned as the dual scaling).  In [0, 1); 0: never
                                (default 1e-3).  Not in the paper, which does not treat the
                                singular case of Eqs. 11-13 */
    double newton_cond_switch; /* where the dual scaling's relative determinant at (1, 1) is at most
                                this, the split scaling is used instead if it is better conditioned
                                (|p_r.dH/dp| / (|p_t.dH/dp| + |p_r.dH/dp|) larger, and above
                                newton_split_min).  Rounding in Eq. 13's residuals reaches the state
                                amplified by the inverse conditioning, and kicks that differ between
                                the two FLI trajectories (Sec. 3B) grow their separation by
                                themselves.  In [0, 1); 0: the dual scaling down to newton_det_min
                                (default 1e-2) */
} scan_params;

typedef struct scan_handle scan_handle;   /* opaque, library-owned */

/* Scan-level reduction (Sec. 3C scan outcome), filled by scan_summary. */
typedef struct scan_summary_t {
    int64_t n;
    int64_t n_chaotic;          /* orbits DONE or FLI_SATURATED with FLI > fli_thresh */
    int64_t status_count[6];    /* orbits per PNSCAN_ORBIT_* value */
    int64_t newton_iters;       /* Newton iterations, all orbits, both trajectories */
    int64_t n_skip;             /* corrections whose dual scaling was singular or did not converge */
    int64_t orbit_steps;        /* sum over orbits of steps taken since the initial state */
    double max_dE;              /* max |E - E0| / |E0| over DONE orbits (E0: the reference at t
                                   with radiation_reaction) */
    double max_dJ;              /* max ||J| - J0| / J0 over DONE orbits whose last step restored |J|
                                   (dual or split scaling) */
    double max_dJ_all;          /* the same over all DONE orbits */
    int64_t n_final_fallback;   /* DONE orbits whose last step fell where both the dual and the
                                   split scaling are singular (E restored by velocity scaling,
                                   |J| not) */
    double max_dS;              /* max ||S_i| - |S_i|0| / |S_i|0 over DONE orbits */
    double fli_max;             /* max(FLI, 0) over DONE orbits */
    double fli_mean;            /* mean FLI over DONE orbits */
} scan_summary_t;

/* Fill *p with the defaults listed above (n = 0, no arrays): the model and
 * method parameters of Secs. 2-3 (Newton tolerance 1e-10 of Sec. 3A, FLI
 * threshold of Sec. 3C).  Returns PNSCAN_ERR_ARG if p is NULL. */
int scan_params_default(scan_params *p);

/* Validate *p, copy the per-orbit parameters (Sec. 2: mass ratio m1/m2 <= 1,
 * quadrupole-monopole multipliers of Eqs. 4-5) to the device and allocate the
 * structure-of-arrays orbit state (about 330 bytes per orbit).  On success
 * *out receives a new handle; on failure *out is NULL.  Errors: ARG (bad
 * sizes, flags or beta_m outside (0,1]), OOM, CUDA, NODEVICE. */
int scan_create(const scan_params *p, scan_handle **out);

/* Initial conditions of a scan grid on the device (Sec. 3C).  cells is n x 9
 * row-major: (x0, pfac, theta1, phi1, theta2, phi2, beta, chi1, chi2) with
 * r = (x0, 0, 0), p = (0, pfac / sqrt(x0), 0) and
 * S_i = chi_i m_i^2 (sin th_i cos ph_i, sin th_i sin ph_i, cos th_i),
 * m1 = beta/(1+beta), m2 = 1/(1+beta).  Then computes the reference
 * integrals (E0, J0, |S_i|0) and places the shadow trajectory fli_d0 away
 * along x; resets time, FLI and status.  Errors: ARG, CUDA. */
int scan_setup(scan_handle *h, const double *cells);

/* Integrate every running orbit from its current time to t_end with step
 * h_step (number of steps = round((t_end - t) / h_step), t the handle's
 * current time).  Each step is the loop of Sec. 3A / Fig. 1 for both FLI
 * trajectories: an RK step of Eqs. 6-9, the spin lengths (Eq. 10), the dual
 * scaling (Eqs. 11-13); then the termination tests and, every
 * fli_renorm_steps, the FLI renormalisation (Secs. 3B-3C).  If initial_states (n x 12 row-major) is not NULL it first
 * replaces the state and resets as scan_setup does; if it is NULL the run
 * continues from the device-resident state (chunked runs reproduce one long
 * run exactly).  Errors: ARG (t_end < t, h_step <= 0 or too many steps),
 * STATE (no state loaded yet), CUDA, KERNEL (reported by the next
 * synchronising call). */
int scan_run(scan_handle *h, const double *initial_states, double t_end, double h_step);

/* Copy results out (synchronises the stream).  Any output pointer may be NULL.
 *   states    n x 12  main trajectory at t_stop (or t_end)
 *   integrals n x 6   (E0, E, J0, |J|, |S1|, |S2|) of the main trajectory; with
 *                     radiation_reaction, E0 and J0 are the references at t_stop
 *                     (integral-invariant relations, Sec. 3B)
 *   fli       n       FLI = sum_k log10(d_k/d0) + log10(d(t)/d0)
 *   status    n       PNSCAN_ORBIT_*
 *   t_stop    n       time at which the orbit stopped (t_end if DONE)
 * Errors: STATE, CUDA, KERNEL, TIMEOUT. */
int scan_read(scan_handle *h, double *states, double *integrals, double *fli,
              int32_t *status, double *t_stop);

/* Diagnostics of the correction (synchronises).  shadow n x 12 (the second
 * FLI trajectory, Sec. 3B), newton_iters n (Newton iterations of Eq. 13, both
 * trajectories), n_skip n (steps of either trajectory whose dual scaling was
 * singular or did not converge), last_kind n (correction of the main
 * trajectory's last step: 0 dual scaling, 3 split scaling of p's tangential
 * and radial parts (newton_split_min), 2 velocity scaling of p alone as in
 * the method Sec. 1 cites, 1 none).  Any pointer may be NULL.
 * Errors: STATE, CUDA, KERNEL, TIMEOUT. */
int scan_read_diag(scan_handle *h, double *shadow, int32_t *newton_iters, int32_t *n_skip,
                   int32_t *last_kind);

/* Scan-level reduction on the device (synchronises; *out is a host struct):
 * the chaotic count at the FLI threshold (the scan outcome of Sec. 3C), the
 * integral errors (Table 2's measure of the correction) and the status
 * histogram.  Errors: ARG, STATE, CUDA. */
int scan_summary(scan_handle *h, scan_summary_t *out);

/* Not in the paper (its launch shape is fixed, Sec. 3A).  Pick the
 * integrator schedule, block size, chunk length, blocks per SM and
 * register variant by timing candidate launches on a copy of the handle's current state for
 * `steps` steps (the state itself is left unchanged); candidates within 1 % of
 * the fastest are timed again over 4 x `steps` steps.  The choice is kept in
 * the handle and used by later scan_run calls with schedule AUTO; it is also
 * written to the optional outputs.  Errors: ARG, STATE, CUDA. */
int scan_autotune(scan_handle *h, int steps, int *schedule, int *block_size, int *chunk_steps,
                  int *blocks_per_sm, int *register_variant);

/* ---- checkpoint / resume ----
 * A checkpoint is the handle's complete orbit state: both trajectories,
 * reference integrals, FLI accumulators, times, step counters, statuses,
 * Newton counters and per-orbit parameters, with a header recording the
 * orbit count and the run configuration (term flags, correction mode,
 * Newton settings, RK order, FLI and termination settings).  Restored into
 * a handle created with the same n and configuration, the next scan_run
 * continues exactly where the checkpointed handle stood: the results are
 * bit-identical to an uninterrupted run.  Not in the paper.
 *
 * scan_checkpoint_size: bytes of a checkpoint of h (0 for a NULL handle).
 * scan_checkpoint: write it to buf, HOST memory of at least that many bytes
 *   (whatever device_ptrs says).  Synchronises.  Errors: ARG (NULL, small
 *   buffer), STATE (no state yet), CUDA.
 * scan_restore: load a checkpoint from host memory into h.  Synchronises.
 *   Errors: ARG (not a checkpoint, a different n or configuration, short
 *   buffer), CUDA. */
size_t scan_checkpoint_size(scan_handle *h);
int scan_checkpoint(scan_handle *h, void *buf, size_t bytes);
int scan_restore(scan_handle *h, const void *buf, size_t bytes);

/* Gravitational-wave polarisations of every orbit's main trajectory at its
 * current state (Eq. 14, Sec. 4): the field of the mass quadrupole moment
 * of the relative orbit (Fig. 10 uses it for orbits 2 and 4),
 *     h_ij = (4 eta / R) (v_i v_j - n_i n_j / |r|),  v = dr/dt = dH/dp (Eq. 6),
 *     h_plus = (P_i P_j - Q_i Q_j) h_ij / 2,  h_cross = (P_i Q_j + Q_i P_j) h_ij / 2,
 * in units G = c = M = 1, observer at distance R > 0 (in M) along N = P x Q.
 * P, Q: host arrays of 3 doubles, the radiation frame's unit vectors
 * orthogonal to N (the paper takes P = x, Q = y, N = z).  hplus, hcross: n
 * doubles each, host or device per device_ptrs; either may be NULL.
 * Call after scan_run to sample a waveform along the run (e.g. run to t1,
 * t2, ... and call this after each).  Synchronises.  Errors: ARG (R not
 * positive and finite, non-finite P or Q), STATE (no state), CUDA. */
int scan_waveform(scan_handle *h, double R, const double *P, const double *Q, double *hplus, double *hcross);

/* Device time of the integrator launches of the last scan_run (the elapsed
 * time that Tables 2-3 report, here from CUDA events on the handle's stream;
 * synchronises) and the number of kernels that run launched: 1 for the
 * static, paired and work-queue schedules, 2 per epoch for the compacting
 * schedule (integrator + compaction).  *ms and *launches may be NULL; 0 ms
 * if the last scan_run launched nothing.  Errors: ARG, CUDA. */
int scan_last_run_timing(scan_handle *h, double *ms, int *launches);

/* Not in the paper: the measured denominator of the integrator's FP64
 * roofline.  Time iters x 8 DFMA per thread -- 8 independent chains -- with
 * one block of 128, 256 and 512 threads on every SM, on the handle's
 * stream, and return the best achieved FP64 rate (TFLOP/s, 2 flops per
 * DFMA).  Errors: ARG, OOM, CUDA. */
int scan_fp64_peak(scan_handle *h, int iters, double *tflops);

/* ---- reduction without run-time allocation ----
 * The paper has no counterpart to this entry point; it serves callers that
 * cannot allocate device memory when they reduce a scan (a framework whose
 * caching allocator already holds the memory budget, or a loop that must
 * not allocate after start-up).
 *
 * scan_summary_noalloc computes the same reduction as scan_summary over
 * caller-owned DEVICE arrays -- typically what scan_read / scan_read_diag
 * wrote in device-pointer mode -- and fills the HOST struct *out.  It calls
 * no cudaMalloc, cudaFree or other allocating routine: its scratch is a
 * fixed array of this library in device memory (PNSCAN_NOALLOC_MAX_ORBITS /
 * 256 + 1 records of 256 bytes, 2.1 MB), present on every GPU that loads the
 * library until the process exits.
 *   n              number of orbits, 0 <= n <= PNSCAN_NOALLOC_MAX_ORBITS (else ARG)
 *   status [n], fli [n], integrals [n x 6] (E0, E, J0, |J|, |S1|, |S2|): required if n > 0
 *   spin_ref [n x 2] (|S1|0, |S2|0), newton_iters [n], n_skip [n],
 *   last_kind [n] (NULL: every last step counts as restoring |J|),
 *   t_stop [n] with h_step > 0 (orbit_steps = sum round(t_stop / h_step)): each nullable;
 *   a NULL input leaves its fields 0.
 *   fli_thresh     FLI above this counts as chaotic
 *   cuda_stream    stream to run on (cudaStream_t); the call synchronises it.
 * The first call on a device looks up the scratch address on that device
 * (the device must be current); make that first call before any stream
 * capture.  Calls share the scratch: two calls whose work overlaps on the
 * GPU race and must be serialised by the caller.  Errors: ARG, CUDA,
 * NODEVICE. */
#define PNSCAN_NOALLOC_MAX_ORBITS 2097152
int scan_summary_noalloc(int64_t n, const int32_t *status, const double *fli,
                         const double *integrals, const double *spin_ref,
                         const int32_t *newton_iters, const int32_t *n_skip,
                         const int32_t *last_kind, const double *t_stop, double h_step,
                         double fli_thresh, void *cuda_stream, scan_summary_t *out);

/* ---- surrogate network (the learned map of the adaptive scan) ----
 * Not in the paper: an ensemble of `members` networks mapping a cell's
 * (x0, theta, mass ratio, chi) to its FLI,
 *   z = (x - center) / scale, h1 = tanh(W1 z + b1), h2 = tanh(W2 h1 + b2),
 *   FLI ~ w3 . h2 + b3, 64 hidden units per layer,
 * with BF16 tensor-core operands, FP32 accumulation, FP32 master weights and
 * Adam moments (beta1 0.9, beta2 0.999, eps 1e-8).  The parameter vector of
 * a member (MLP_PARAMS floats) is W1 (64 x 4 row-major), b1, W2 (64 x 64,
 * [out][in]), b2, w3, b3.  All array arguments are DEVICE pointers; the
 * handle owns its parameters (cudaMalloc'ed at creation).  Calls run on the
 * handle's stream; mlp_train, mlp_gradient and mlp_get/set_params
 * synchronise it, mlp_predict does not. */
#define MLP_INPUTS 4
#define MLP_HIDDEN 64
#define MLP_PARAMS 4545
#define MLP_BATCH 128
typedef struct mlp_handle mlp_handle;

/* Surrogate (not in the paper).  Xavier-uniform weights from seed
 * (SplitMix64), zero biases and moments.  center/scale: host float[4], scale
 * nonzero.  members in 1..64.  Errors: ARG, OOM, CUDA, NODEVICE. */
int mlp_create(int members, uint64_t seed, const float *center, const float *scale, void *cuda_stream,
               mlp_handle **out);
/* Surrogate (not in the paper).  Copy all members' parameters out / in
 * ([members][MLP_PARAMS] floats, device); mlp_set_params also clears the
 * Adam moments.  Errors: ARG (NULL pointer), CUDA. */
int mlp_get_params(mlp_handle *h, float *params);
int mlp_set_params(mlp_handle *h, const float *params);
/* Surrogate (not in the paper).  Copy the Adam moments out: m and v, each
 * [members][MLP_PARAMS] floats (device), in the parameter layout.  Zero
 * after mlp_create and mlp_set_params.  Errors: ARG (NULL pointer), CUDA. */
int mlp_get_moments(mlp_handle *h, float *m, float *v);
/* Surrogate (not in the paper).  `steps` Adam steps of minibatch MSE
 * training on (X [n][4], y [n]).  Adam step t (counted from 1 since
 * mlp_create / mlp_set_params, across calls) draws MLP_BATCH rows with
 * replacement: row j (0 <= j < 128) of member k is
 *   X[ SM(seed ^ SM((k << 40) ^ ((t - 1) << 8) ^ j)) mod n ],
 * where SM is the SplitMix64 output function of Steele, Lea & Flood (2014)
 * applied to x + 0x9E3779B97F4A7C15 (all arithmetic modulo 2^64).  The
 * update is Adam (Kingma & Ba 2015: beta1 0.9, beta2 0.999, eps 1e-8 added
 * to the square root of the bias-corrected second moment) in FP32.
 * loss_hist [members][steps] (nullable) gets each step's loss.  Errors: ARG
 * (NULL X or y, n < 1, steps < 0, lr not positive), CUDA. */
int mlp_train(mlp_handle *h, const float *X, const float *y, int64_t n, int steps, float lr, uint64_t seed,
              float *loss_hist);
/* Surrogate (not in the paper).  Loss and gradient of every member on
 * exactly MLP_BATCH rows (X [128][4], y [128]): grad [members][MLP_PARAMS],
 * loss [members].  No update.  Errors: ARG (NULL pointer), CUDA. */
int mlp_gradient(mlp_handle *h, const float *X, const float *y, float *grad, float *loss);
/* Surrogate (not in the paper).  Ensemble mean and spread (max - min over
 * members) for X [n][4].  Errors: ARG (n < 0, NULL arrays with n > 0), CUDA. */
int mlp_predict(mlp_handle *h, const float *X, int64_t n, float *mean, float *spread);
void mlp_destroy(mlp_handle *h);

/* ---- adaptive scan: features, selection and merge ----
 * Not in the paper.  adaptive_select marks cell i when |mean_i - thr| <= band,
 * spread_i > spread_max, or mean_i is NaN; writes the marked indices in
 * ascending order to idx [n], gathers their rows of cells [n][9] (nullable)
 * into cells_out (nullable), and returns the number marked in *count (host;
 * synchronises).  workspace: device memory of adaptive_select_workspace(n)
 * bytes owned by the caller.  n <= 16,777,216.  adaptive_merge writes the
 * class map cls [n] (1 chaotic, 0 not): marked cells take the integrator's
 * result (chaotic if status is DONE or FLI_SATURATED and fli_sel > thr),
 * the others the surrogate's (mean > thr).  adaptive_features writes the
 * surrogate inputs X [n][4] = (x0, theta1, beta, chi1) of cells [n][9] as
 * float.  Device pointers throughout. */
int adaptive_features(const double *cells, int64_t n, float *X, void *cuda_stream);
size_t adaptive_select_workspace(int64_t n);
int adaptive_select(const float *mean, const float *spread, int64_t n, float thr, float band, float spread_max,
                    const double *cells, int32_t *idx, double *cells_out, int64_t *count, void *workspace,
                    void *cuda_stream);
int adaptive_merge(const float *mean, int64_t n, float thr, const int32_t *idx, int64_t count,
                   const double *fli_sel, const int32_t *status_sel, int8_t *cls, void *cuda_stream);
/* Adaptive scan (not in the paper).  The surrogate inputs X [n][4] from any
 * four fields of cells [n][9]: X[i][k] = (float) cells[i][fields[k]], fields
 * a HOST array of 4 indices in 0..8 (x0, pfac, theta1, phi1, theta2, phi2,
 * beta, chi1, chi2), e.g. (2, 4, 0, 6) for the (theta1, theta2) plane of
 * Sec. 3C, Fig. 7.  Device pointers otherwise; asynchronous on cuda_stream.
 * Errors: ARG (n < 0, a field out of range, NULL arrays with n > 0), CUDA. */
int adaptive_features_fields(const double *cells, int64_t n, const int32_t *fields, float *X,
                             void *cuda_stream);
/* Adaptive scan without a learned map (not in the paper; the comparison
 * method of the surrogate): a row-major n1 x n2 grid is estimated from its
 * coarse grid of every stride-th cell in both directions, integrated
 * beforehand: nodes (a, b) at cells (a stride, b stride), a < (n1-1)/stride+1,
 * b < (n2-1)/stride+1, with FLIs fli_nodes and statuses status_nodes
 * (row-major, device).  mean [n1 x n2] gets the FLI interpolated bilinearly
 * between the four surrounding nodes (clamped beyond the last node; a node
 * that did not finish or saturate counts as FLI 0, not chaotic), spread the
 * max - min of those four node values, as uncertainty; a cell that is a node
 * gets the node's FLI and spread 0.  Both feed adaptive_select and
 * adaptive_merge like the surrogate's mean and spread.  Asynchronous on
 * cuda_stream.  Errors: ARG (negative sizes, stride < 1, n1 or n2 > 2^20,
 * n1 n2 > 2^32, NULL arrays with a non-empty grid), CUDA. */
int adaptive_interp_grid(const double *fli_nodes, const int32_t *status_nodes, int64_t n1, int64_t n2,
                         int32_t stride, float *mean, float *spread, void *cuda_stream);

/* Library utility (not in the paper): free the handle's device buffers and
 * the handle (NULL is a no-op; no error is reported). */
void scan_destroy(scan_handle *h);

/* Library utility (not in the paper): static description of an error code
 * (an unknown code gets a generic string; never NULL, no error). */
const char *scan_strerror(int code);

/* Library utility (not in the paper): version string; static, never NULL,
 * no error; names the build's target architecture (sm_103a). */
const char *scan_version(void);

#ifdef __cplusplus
}
#endif
#endif /* PNSCAN_H */
