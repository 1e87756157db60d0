/*
 * pn_oracle.h -- plain, slow, obviously-correct FP64 CPU oracle for the
 * manifold-corrected post-Newtonian spinning-binary scan of
 * Ran, Liu & Zhong, "GPU accelerated manifold correction method for
 * spinning compact binaries" (arXiv:1802.00147).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path loads this library:
 * only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline /
 * reference leg may.  It shares no code, header, table or constant with the
 * CUDA library (paper_1802_00147_gb300/csrc); the two are written
 * independently from the paper's equations.
 *
 * Units: G = c = M = 1 (Sec. 2).  r in M, p in mu, H in mu, t in M, spins in
 * M^2 (the reading under which Eqs. 8-9 are the exact spin gradients of H and
 * J = L + S1 + S2 is conserved by Eqs. 6-7).
 *
 * State vector y[12] = (r[3], p[3], S1[3], S2[3]), FP64 (orc_real), per orbit.
 */
#ifndef PN_ORACLE_H
#define PN_ORACLE_H
#include <stdint.h>

/* The oracle's arithmetic type: FP64, or long double when built with
 * -DORC_LONG_DOUBLE (an extended-precision reference of the same plain
 * code: 64-bit significands on x86-64, 113-bit on aarch64). */
#ifdef ORC_LONG_DOUBLE
typedef long double orc_real;
#else
typedef double orc_real;
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* Per-orbit physical system (Sec. 2): mass ratio beta = m1/m2 <= 1, M = 1. */
typedef struct {
    orc_real beta, m1, m2, eta;   /* eta = mu/M = m1 m2 */
    orc_real kappa1, kappa2;      /* quadrupole-monopole multipliers (1 for black holes) */
    int pn_order;               /* 0: Newtonian, 1: +1PN, 2: +2PN orbital terms */
    int use_so, use_ss, use_qm; /* 1.5PN spin-orbit, 2PN S1S2, QM terms (Eqs. 3-5) */
} orc_sys;

/* Integration / correction / FLI configuration (one per scan). */
typedef struct {
    int pn_order, use_so, use_ss, use_qm;
    int correct;          /* correction after every step: 0 none; 1 spin lengths (Eq. 10) and dual
                             scaling (Eqs. 11-13); ablations: 2 spin lengths only; 3 spin lengths and
                             velocity scaling p = a p* to E0 (Sec. 1, Wu et al. 2007) */
    double newton_tol;    /* stop when max(|d alpha|, |d beta|) <= tol (Sec. 3A: 1e-10) */
    int newton_max;       /* iteration cap (50) */
    double det_min;       /* skip the scaling when |det| <= det_min (|J11 J22| + |J12 J21|) */
    double fli_d0;        /* initial / renormalised separation of the two trajectories */
    int fli_renorm;       /* renormalise every this many steps */
    double fli_cap;       /* stop when the FLI reaches this value (<= 0: never) */
    double r_merge;       /* stop when |r| < r_merge (<= 0: never) */
    double r_escape;      /* stop when |r| > r_escape (<= 0: never) */
    int rk_order;         /* 4: classical RK4; 5: Dormand-Prince fifth-order weights */
    int newton_apply_small; /* 1: apply a Newton step, then stop if it was within newton_tol;
                               0: stop before applying a step already within newton_tol */
    int rr;               /* 1: add the 2.5PN radiation reaction a_2.5PN to dp/dt (Eq. 6) and
                             correct toward integral-invariant reference values (Sec. 3B) */
    double rr_gauge_a, rr_gauge_b; /* gauge constants of orc_rr_accel (harmonic gauge: 4, 5) */
    double split_min;     /* use the split scaling only where |p_r.dH/dp| > split_min
                             (|p_t.dH/dp| + |p_r.dH/dp|) (<= 0: never) */
    double cond_switch;   /* where the dual scaling's relative determinant at (1, 1) is at most
                             this, the split scaling is used instead if it is better conditioned
                             (<= 0: only where the dual scaling is singular) */
} orc_config;

/* Per-orbit final status (oracle's own numbering). */
enum {
    ORC_RUNNING = 0, ORC_DONE = 1, ORC_MERGED = 2, ORC_ESCAPED = 3,
    ORC_FLI_SATURATED = 4, ORC_NONFINITE = 5
};

/* Correction outcome: dual scaling applied; singular dual scaling replaced
 * by velocity scaling of p alone; nothing converged (r*, p* kept); singular
 * dual scaling replaced by the split scaling of p's radial and tangential
 * parts (both integrals restored). */
enum { ORC_CORR_OK = 0, ORC_CORR_SKIPPED = 1, ORC_CORR_VELOCITY = 2, ORC_CORR_SPLIT = 3 };

void orc_sys_init(orc_sys *s, orc_real beta, orc_real kappa1, orc_real kappa2,
                  int pn_order, int use_so, int use_ss, int use_qm);

/* Hamiltonian pieces (Eq. 1 without 3PN and 2.5PN; Eqs. 3-5). */
orc_real orc_H_newton(const orc_sys *s, const orc_real y[12]);
orc_real orc_H_1pn(const orc_sys *s, const orc_real y[12]);
orc_real orc_H_2pn(const orc_sys *s, const orc_real y[12]);
orc_real orc_H_so(const orc_sys *s, const orc_real y[12]);
orc_real orc_H_s1s2(const orc_sys *s, const orc_real y[12]);
orc_real orc_H_qm(const orc_sys *s, const orc_real y[12]);
orc_real orc_hamiltonian(const orc_sys *s, const orc_real y[12]);

/* Analytic gradient g = (dH/dr, dH/dp, dH/dS1, dH/dS2). */
void orc_gradient(const orc_sys *s, const orc_real y[12], orc_real g[12]);

/* Equations of motion (Eqs. 6-7, conservative): dy/dt. */
void orc_rhs(const orc_sys *s, const orc_real y[12], orc_real dy[12]);

/* One classical RK4 step of size h, in place. */
void orc_rk4_step(const orc_sys *s, orc_real y[12], orc_real h);

/* One fifth-order Runge-Kutta step (Dormand-Prince 1980 tableau, fifth-order
 * weights, fixed step), in place. */
void orc_rk5_step(const orc_sys *s, orc_real y[12], orc_real h);

/* Leading-order (2.5PN) radiation-reaction acceleration a_2.5PN of Eq. 6
 * for the state y (velocity v = p at this order), in the two-parameter gauge
 * family of Iyer & Will (1993) with constants (ga, gb); (4, 5) is the
 * harmonic-gauge force of Damour & Deruelle.  The paper takes the force from
 * Levin et al. (2011) without printing it. */
void orc_rr_accel(const orc_sys *s, orc_real ga, orc_real gb, const orc_real y[12], orc_real a[3]);

/* Equations of motion with radiation reaction on the extended state
 * y14 = (r, p, S1, S2, E, |J|): Eqs. 6-7 with a_2.5PN, and the integral-
 * invariant relations dE/dt = (dH/dp).a, d|J|/dt = J.(r x a)/|J| that carry
 * the reference values of the dissipative system (Sec. 3B). */
void orc_rhs_rr(const orc_sys *s, orc_real ga, orc_real gb, const orc_real y[14], orc_real dy[14]);

/* One RK4 (rk_order 4) or fifth-order (5) step of orc_rhs_rr, in place. */
void orc_rk_step_rr(const orc_sys *s, orc_real ga, orc_real gb, int rk_order, orc_real y[14], orc_real h);

/* Integrals: out = (E, |J|, |S1|, |S2|, Jx, Jy, Jz). */
void orc_integrals(const orc_sys *s, const orc_real y[12], orc_real out[7]);

/* Manifold correction (Eqs. 10-13) toward ref = (E0, J0, |S1|0, |S2|0), in
 * place.  Returns ORC_CORR_OK (dual scaling applied), or, where the dual
 * scaling was singular (|det| <= det_min (|J11 J22| + |J12 J21|)) or did not
 * converge, or where its relative determinant at (1, 1) is at most
 * cond_switch and the split scaling is better conditioned: ORC_CORR_SPLIT
 * (p = a p_t + g p_r with r kept restored E and |J|), ORC_CORR_VELOCITY
 * (that too was singular: p alone was scaled to restore E) or
 * ORC_CORR_SKIPPED.  *iters gets the number of Newton
 * iterations of all solves; alpha_beta (nullable) gets the scale factors of
 * p and r applied (for the split scaling: a and g). */
int orc_correct(const orc_sys *s, orc_real y[12], const orc_real ref[4],
                orc_real newton_tol, int newton_max, orc_real det_min,
                int *iters, orc_real alpha_beta[2]);
/* The same with the stopping rule (apply_small as in orc_config) and the
 * correction mode (orc_config.correct: ORC_MODE_*) as parameters. */
enum { ORC_MODE_DUAL = 1, ORC_MODE_SPINS = 2, ORC_MODE_VELOCITY = 3 };
int orc_correct_rule(const orc_sys *s, orc_real y[12], const orc_real ref[4],
                     orc_real newton_tol, int newton_max, orc_real det_min, orc_real split_min,
                     orc_real cond_switch, int apply_small, int mode, int *iters, orc_real alpha_beta[2]);

/* Gravitational-wave polarisations (Eq. 14) from the mass quadrupole
 * field of the relative orbit, observer at distance R along N = P x Q:
 * out = (h_plus, h_cross). */
void orc_waveform(const orc_sys *s, const orc_real y[12], orc_real R, const orc_real P[3], const orc_real Q[3],
                  orc_real out[2]);

/* The dual-scaling Newton iterates of Eq. 13 from (1, 1) at the state y =
 * (r*, p*, S) toward ref, without stopping rule or singularity guard:
 * (alpha[k], beta[k]) after k + 1 steps, k < kmax.  Returns the number of
 * iterates written (fewer than kmax if the Jacobian became singular or not
 * finite). */
int orc_newton_trace(const orc_sys *s, const orc_real y[12], const orc_real ref[4], int kmax,
                     orc_real *alpha, orc_real *beta);

/* Initial conditions of a scan cell: cell = (x0, pfac, theta1, phi1,
 * theta2, phi2, beta, chi1, chi2).  r = (x0,0,0), p = (0, pfac/sqrt(x0), 0),
 * S_i = chi_i m_i^2 (sin th_i cos ph_i, sin th_i sin ph_i, cos th_i). */
void orc_setup_cell(const orc_real cell[9], orc_real y[12]);

/* Integrate n independent orbits for nsteps steps of size h with manifold
 * correction and FLI (two trajectories).  Arrays are AoS: y0/y_out/ys_out
 * n*12; kappa1/kappa2 nullable (1.0); outputs:
 *   integrals n*6 = (E0, E, J0, |J|, |S1|, |S2|) of the main trajectory
 *   (with cfg->rr, E0 and J0 are the reference values at the final time),
 *   fli n, status n, t_stop n, newton_iters n (sum over both trajectories),
 *   n_skip n (steps whose dual scaling was replaced by velocity scaling or
 *   skipped), last_kind n (ORC_CORR_* of the main trajectory's last step).
 * nthreads <= 0: all OpenMP threads.  Returns 0, or -1 on bad arguments. */
int orc_scan(int64_t n, const orc_real *y0, const orc_real *beta,
             const orc_real *kappa1, const orc_real *kappa2,
             const orc_config *cfg, orc_real h, int64_t nsteps,
             orc_real *y_out, orc_real *ys_out, orc_real *integrals, orc_real *fli,
             int32_t *status, orc_real *t_stop, int64_t *newton_iters,
             int32_t *n_skip, int32_t *last_kind, int nthreads);

/* Same integrator without the shadow trajectory, recording the state after
 * every `every` steps into trace[(nsteps/every) * 12] (single orbit).  With
 * cfg->rr the reference E and |J| advance with the state (not recorded), and
 * there is no termination test: stop before the orbit plunges. */
int orc_trace(const orc_real y0[12], orc_real beta, orc_real kappa1, orc_real kappa2,
              const orc_config *cfg, orc_real h, int64_t nsteps, int64_t every,
              orc_real *trace);

/* One trajectory (no FLI shadow) through nsteps steps, each followed by the
 * correction of cfg, from y0 -- like orc_trace's last row -- with every
 * operation in orc_real but the inputs and the output state in double, so
 * that a long-double build of this file can serve as an extended-precision
 * reference of the FP64 one.  Returns 0, or -1 for bad arguments. */
int orc_ext_trace(const double y0[12], double beta, double kappa1, double kappa2,
                  const orc_config *cfg, double h, int64_t nsteps, double y_out[12]);

int orc_max_threads(void);

#ifdef __cplusplus
}
#endif
#endif
