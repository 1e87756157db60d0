/*
 * pn_oracle.c -- plain, slow, obviously-correct FP64 CPU oracle.
 *
 * TEST INFRASTRUCTURE ONLY: loaded by tests/, __graft_entry__.smoke() and
 * bench.py's CPU-baseline / reference leg, never by the product path.  It
 * shares no code with the CUDA library.  Compiled with -O2
 * -ffp-contract=off: every + and * is a separately rounded IEEE operation.
 *
 * Method (arXiv:1802.00147):
 *   Sec. 2, Eq. 1      H = H_N + H_1PN + H_2PN + H_SO + H_SS   (3PN and 2.5PN off)
 *   Eqs. 3-5           spin-spin and quadrupole-monopole terms
 *   Eq. 6              dr/dt = dH/dp, dp/dt = -dH/dr          (conservative)
 *   Eqs. 7-9           dS_i/dt = Omega_i x S_i, Omega_i = dH/dS_i
 *   Sec. 2, Eq. 10     spin lengths restored after every step
 *   Eqs. 11-13         dual scaling p = alpha p*, r = beta r*, (alpha, beta)
 *                      from E and |J| by Newton's method (Sec. 3A)
 *   Sec. 3B/3C         FLI from two nearby trajectories (Wu et al. 2006)
 *   Eq. 6, Sec. 3B     optional 2.5PN radiation reaction a_2.5PN, with the
 *                      reference E and |J| carried by their integral-
 *                      invariant relations (dissipative orbit 3, Fig. 5)
 *
 * The orbital terms H_N, H_1PN, H_2PN and H_SO are not printed in the paper
 * (Sec. 2 defers to Buonanno et al. 2006); they are the standard ADM
 * expressions in reduced variables.  H_SO's coefficients are fixed by the
 * L/r^3 terms of Eqs. 8-9; H_S1S2 and H_QM carry the 1/eta that Eqs. 8-9
 * imply (spins in units of M^2).  The 1PN/2PN orbital coefficients are pinned
 * by the gauge-invariant circular-orbit energy in tests/test_oracle_pins.py.
 */
#include "pn_oracle.h"
#include <tgmath.h> /* sqrt, fabs, log10 ... of the argument's type (double or long double) */
#undef I             /* tgmath.h brings complex.h's imaginary unit; not used here */
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ---------------------------------------------------------------- vectors */
static orc_real dot3(const orc_real *a, const orc_real *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static void cross3(const orc_real *a, const orc_real *b, orc_real *c)
{
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}
static orc_real norm3(const orc_real *a) { return sqrt(dot3(a, a)); }

void orc_sys_init(orc_sys *s, orc_real beta, orc_real kappa1, orc_real kappa2,
                  int pn_order, int use_so, int use_ss, int use_qm)
{
    /* Sec. 2: m1 <= m2, beta = m1/m2, M = m1 + m2 = 1, eta = mu/M = m1 m2. */
    s->beta = beta;
    s->m1 = beta / (1.0 + beta);
    s->m2 = 1.0 / (1.0 + beta);
    s->eta = s->m1 * s->m2;
    s->kappa1 = kappa1;
    s->kappa2 = kappa2;
    s->pn_order = pn_order;
    s->use_so = use_so;
    s->use_ss = use_ss;
    s->use_qm = use_qm;
}

/* ------------------------------------------------------------ Hamiltonian */
/* H_N = p^2/2 - 1/r */
orc_real orc_H_newton(const orc_sys *s, const orc_real y[12])
{
    (void)s;
    const orc_real *r = y, *p = y + 3;
    return 0.5 * dot3(p, p) - 1.0 / norm3(r);
}

/* H_1PN = (3 eta - 1) p^4 / 8 - [(3 + eta) p^2 + eta (n.p)^2] / (2 r) + 1/(2 r^2) */
orc_real orc_H_1pn(const orc_sys *s, const orc_real y[12])
{
    const orc_real *r = y, *p = y + 3;
    orc_real eta = s->eta, rr = norm3(r), p2 = dot3(p, p), np = dot3(r, p) / rr;
    return (3.0 * eta - 1.0) * p2 * p2 / 8.0
         - ((3.0 + eta) * p2 + eta * np * np) / (2.0 * rr)
         + 1.0 / (2.0 * rr * rr);
}

/* H_2PN = (1 - 5 eta + 5 eta^2) p^6 / 16
 *       + [(5 - 20 eta - 3 eta^2) p^4 - 2 eta^2 p^2 (n.p)^2 - 3 eta^2 (n.p)^4] / (8 r)
 *       + [(5 + 8 eta) p^2 + 3 eta (n.p)^2] / (2 r^2)
 *       - (1 + 3 eta) / (4 r^3) */
orc_real orc_H_2pn(const orc_sys *s, const orc_real y[12])
{
    const orc_real *r = y, *p = y + 3;
    orc_real eta = s->eta, rr = norm3(r), p2 = dot3(p, p), np = dot3(r, p) / rr;
    return (1.0 - 5.0 * eta + 5.0 * eta * eta) * p2 * p2 * p2 / 16.0
         + ((5.0 - 20.0 * eta - 3.0 * eta * eta) * p2 * p2
            - 2.0 * eta * eta * p2 * np * np
            - 3.0 * eta * eta * np * np * np * np) / (8.0 * rr)
         + ((5.0 + 8.0 * eta) * p2 + 3.0 * eta * np * np) / (2.0 * rr * rr)
         - (1.0 + 3.0 * eta) / (4.0 * rr * rr * rr);
}

/* Spin-orbit coefficients read off the L/r^3 terms of Eqs. 8-9. */
/* Tests build a variant with a planted mistake here (-DORC_PLANTED_SO_FACTOR=...)
 * to show that the parity bounds catch it; 1.0 (exact) otherwise. */
#ifndef ORC_PLANTED_SO_FACTOR
#define ORC_PLANTED_SO_FACTOR 1.0
#endif
static orc_real g_so1(const orc_sys *s) { return ORC_PLANTED_SO_FACTOR * (2.0 + 3.0 / (2.0 * s->beta)); }
static orc_real g_so2(const orc_sys *s) { return 2.0 + 3.0 * s->beta / 2.0; }

/* H_SO = (1/r^3) L . [(2 + 3/(2 beta)) S1 + (2 + 3 beta/2) S2],  L = r x p */
orc_real orc_H_so(const orc_sys *s, const orc_real y[12])
{
    const orc_real *r = y, *p = y + 3, *S1 = y + 6, *S2 = y + 9;
    orc_real L[3], rr = norm3(r);
    cross3(r, p, L);
    return (g_so1(s) * dot3(L, S1) + g_so2(s) * dot3(L, S2)) / (rr * rr * rr);
}

/* Eq. 3 with the 1/eta of Eqs. 8-9:  H_S1S2 = [3 (S1.n)(S2.n) - S1.S2] / (eta r^3) */
orc_real orc_H_s1s2(const orc_sys *s, const orc_real y[12])
{
    const orc_real *r = y, *S1 = y + 6, *S2 = y + 9;
    orc_real rr = norm3(r), n[3] = {r[0] / rr, r[1] / rr, r[2] / rr};
    return (3.0 * dot3(S1, n) * dot3(S2, n) - dot3(S1, S2)) / (s->eta * rr * rr * rr);
}

/* Eqs. 4-5 with the 1/eta of Eqs. 8-9 and multipliers kappa_i:
 * H_QM = kappa1 [3 (S1.n)^2 - S1^2] / (2 beta eta r^3)
 *      + kappa2 beta [3 (S2.n)^2 - S2^2] / (2 eta r^3) */
orc_real orc_H_qm(const orc_sys *s, const orc_real y[12])
{
    const orc_real *r = y, *S1 = y + 6, *S2 = y + 9;
    orc_real rr = norm3(r), n[3] = {r[0] / rr, r[1] / rr, r[2] / rr};
    orc_real a1 = dot3(S1, n), a2 = dot3(S2, n), r3 = rr * rr * rr;
    return s->kappa1 * (3.0 * a1 * a1 - dot3(S1, S1)) / (2.0 * s->beta * s->eta * r3)
         + s->kappa2 * s->beta * (3.0 * a2 * a2 - dot3(S2, S2)) / (2.0 * s->eta * r3);
}

/* Eq. 1 (conservative part, 3PN not given). */
orc_real orc_hamiltonian(const orc_sys *s, const orc_real y[12])
{
    orc_real H = orc_H_newton(s, y);
    if (s->pn_order >= 1) H += orc_H_1pn(s, y);
    if (s->pn_order >= 2) H += orc_H_2pn(s, y);
    if (s->use_so) H += orc_H_so(s, y);
    if (s->use_ss) H += orc_H_s1s2(s, y);
    if (s->use_qm) H += orc_H_qm(s, y);
    return H;
}

/* --------------------------------------------------------------- gradient */
/* The orbital terms depend on (p2 = p.p, np = n.p, rr = |r|):
 *   dH/dp = 2 H_p2 p + H_np n
 *   dH/dr = H_rr n + H_np (p - np n) / rr
 * Spin terms are differentiated directly, with d(S.n)/dr = (S - (S.n) n)/rr. */
void orc_gradient(const orc_sys *s, const orc_real y[12], orc_real g[12])
{
    const orc_real *r = y, *p = y + 3, *S1 = y + 6, *S2 = y + 9;
    orc_real eta = s->eta;
    orc_real rr = norm3(r), n[3] = {r[0] / rr, r[1] / rr, r[2] / rr};
    orc_real p2 = dot3(p, p), np = dot3(n, p);
    orc_real H_p2, H_np, H_rr;
    int i;

    /* H_N */
    H_p2 = 0.5;
    H_np = 0.0;
    H_rr = 1.0 / (rr * rr);
    /* H_1PN */
    if (s->pn_order >= 1) {
        H_p2 += (3.0 * eta - 1.0) * 2.0 * p2 / 8.0 - (3.0 + eta) / (2.0 * rr);
        H_np += -eta * np / rr;
        H_rr += ((3.0 + eta) * p2 + eta * np * np) / (2.0 * rr * rr) - 1.0 / (rr * rr * rr);
    }
    /* H_2PN */
    if (s->pn_order >= 2) {
        orc_real c4 = 5.0 - 20.0 * eta - 3.0 * eta * eta;
        H_p2 += 3.0 * (1.0 - 5.0 * eta + 5.0 * eta * eta) * p2 * p2 / 16.0
              + (2.0 * c4 * p2 - 2.0 * eta * eta * np * np) / (8.0 * rr)
              + (5.0 + 8.0 * eta) / (2.0 * rr * rr);
        H_np += (-4.0 * eta * eta * p2 * np - 12.0 * eta * eta * np * np * np) / (8.0 * rr)
              + 3.0 * eta * np / (rr * rr);
        H_rr += -(c4 * p2 * p2 - 2.0 * eta * eta * p2 * np * np - 3.0 * eta * eta * np * np * np * np)
                    / (8.0 * rr * rr)
              - ((5.0 + 8.0 * eta) * p2 + 3.0 * eta * np * np) / (rr * rr * rr)
              + 3.0 * (1.0 + 3.0 * eta) / (4.0 * rr * rr * rr * rr);
    }
    for (i = 0; i < 3; i++) {
        g[i] = H_rr * n[i] + H_np * (p[i] - np * n[i]) / rr;
        g[3 + i] = 2.0 * H_p2 * p[i] + H_np * n[i];
        g[6 + i] = 0.0;
        g[9 + i] = 0.0;
    }

    if (s->use_so) {
        /* H_SO = (L . Seff) / rr^3 with L . Seff = p . (Seff x r) = r . (p x Seff) */
        orc_real Seff[3], L[3], Sxr[3], pxS[3], r3 = rr * rr * rr, g1 = g_so1(s), g2 = g_so2(s);
        for (i = 0; i < 3; i++) Seff[i] = g1 * S1[i] + g2 * S2[i];
        cross3(r, p, L);
        cross3(Seff, r, Sxr);
        cross3(p, Seff, pxS);
        orc_real LS = dot3(L, Seff);
        for (i = 0; i < 3; i++) {
            g[i] += pxS[i] / r3 - 3.0 * LS * n[i] / (r3 * rr);
            g[3 + i] += Sxr[i] / r3;
            g[6 + i] += g1 * L[i] / r3;
            g[9 + i] += g2 * L[i] / r3;
        }
    }
    if (s->use_ss) {
        orc_real a1 = dot3(S1, n), a2 = dot3(S2, n), S12 = dot3(S1, S2);
        orc_real k = 1.0 / (eta * rr * rr * rr);
        for (i = 0; i < 3; i++) {
            g[i] += -3.0 * k * (3.0 * a1 * a2 - S12) * n[i] / rr
                  + 3.0 * k * (a2 * (S1[i] - a1 * n[i]) + a1 * (S2[i] - a2 * n[i])) / rr;
            g[6 + i] += k * (3.0 * a2 * n[i] - S2[i]);
            g[9 + i] += k * (3.0 * a1 * n[i] - S1[i]);
        }
    }
    if (s->use_qm) {
        orc_real a1 = dot3(S1, n), a2 = dot3(S2, n), r3 = rr * rr * rr;
        orc_real q1 = s->kappa1 / (2.0 * s->beta * eta), q2 = s->kappa2 * s->beta / (2.0 * eta);
        orc_real Q = q1 * (3.0 * a1 * a1 - dot3(S1, S1)) + q2 * (3.0 * a2 * a2 - dot3(S2, S2));
        for (i = 0; i < 3; i++) {
            g[i] += -3.0 * Q * n[i] / (r3 * rr)
                  + (6.0 * q1 * a1 * (S1[i] - a1 * n[i]) + 6.0 * q2 * a2 * (S2[i] - a2 * n[i])) / (r3 * rr);
            g[6 + i] += q1 * (6.0 * a1 * n[i] - 2.0 * S1[i]) / r3;
            g[9 + i] += q2 * (6.0 * a2 * n[i] - 2.0 * S2[i]) / r3;
        }
    }
}

/* ------------------------------------------------------ equations of motion */
void orc_rhs(const orc_sys *s, const orc_real y[12], orc_real dy[12])
{
    orc_real g[12];
    int i;
    orc_gradient(s, y, g);
    for (i = 0; i < 3; i++) {
        dy[i] = g[3 + i];      /* Eq. 6: dr/dt = dH/dp */
        dy[3 + i] = -g[i];     /* Eq. 6: dp/dt = -dH/dr (a_2.5PN = 0) */
    }
    cross3(g + 6, y + 6, dy + 6); /* Eq. 7: dS1/dt = Omega_1 x S1 */
    cross3(g + 9, y + 9, dy + 9); /* Eq. 7: dS2/dt = Omega_2 x S2 */
}

/* Classical fourth-order Runge-Kutta step. */
void orc_rk4_step(const orc_sys *s, orc_real y[12], orc_real h)
{
    orc_real k1[12], k2[12], k3[12], k4[12], tmp[12];
    int i;
    orc_rhs(s, y, k1);
    for (i = 0; i < 12; i++) tmp[i] = y[i] + 0.5 * h * k1[i];
    orc_rhs(s, tmp, k2);
    for (i = 0; i < 12; i++) tmp[i] = y[i] + 0.5 * h * k2[i];
    orc_rhs(s, tmp, k3);
    for (i = 0; i < 12; i++) tmp[i] = y[i] + h * k3[i];
    orc_rhs(s, tmp, k4);
    for (i = 0; i < 12; i++) y[i] = y[i] + h * (k1[i] + 2.0 * k2[i] + 2.0 * k3[i] + k4[i]) / 6.0;
}

/* Fifth-order explicit Runge-Kutta step with the tableau of Dormand & Prince
 * (1980), fifth-order weights, fixed step (the paper's RK5 is not named). */
void orc_rk5_step(const orc_sys *s, orc_real y[12], orc_real h)
{
    static const orc_real a21 = 1.0 / 5.0;
    static const orc_real a31 = 3.0 / 40.0, a32 = 9.0 / 40.0;
    static const orc_real a41 = 44.0 / 45.0, a42 = -56.0 / 15.0, a43 = 32.0 / 9.0;
    static const orc_real a51 = 19372.0 / 6561.0, a52 = -25360.0 / 2187.0, a53 = 64448.0 / 6561.0,
                        a54 = -212.0 / 729.0;
    static const orc_real a61 = 9017.0 / 3168.0, a62 = -355.0 / 33.0, a63 = 46732.0 / 5247.0,
                        a64 = 49.0 / 176.0, a65 = -5103.0 / 18656.0;
    static const orc_real b1 = 35.0 / 384.0, b3 = 500.0 / 1113.0, b4 = 125.0 / 192.0,
                        b5 = -2187.0 / 6784.0, b6 = 11.0 / 84.0;
    orc_real k1[12], k2[12], k3[12], k4[12], k5[12], k6[12], t[12];
    int i;
    orc_rhs(s, y, k1);
    for (i = 0; i < 12; i++) t[i] = y[i] + h * (a21 * k1[i]);
    orc_rhs(s, t, k2);
    for (i = 0; i < 12; i++) t[i] = y[i] + h * (a31 * k1[i] + a32 * k2[i]);
    orc_rhs(s, t, k3);
    for (i = 0; i < 12; i++) t[i] = y[i] + h * (a41 * k1[i] + a42 * k2[i] + a43 * k3[i]);
    orc_rhs(s, t, k4);
    for (i = 0; i < 12; i++) t[i] = y[i] + h * (a51 * k1[i] + a52 * k2[i] + a53 * k3[i] + a54 * k4[i]);
    orc_rhs(s, t, k5);
    for (i = 0; i < 12; i++)
        t[i] = y[i] + h * (a61 * k1[i] + a62 * k2[i] + a63 * k3[i] + a64 * k4[i] + a65 * k5[i]);
    orc_rhs(s, t, k6);
    for (i = 0; i < 12; i++)
        y[i] = y[i] + h * (b1 * k1[i] + b3 * k3[i] + b4 * k4[i] + b5 * k5[i] + b6 * k6[i]);
}

/* ------------------------------------------------------ radiation reaction */
/* a_2.5PN of Eq. 6 at leading order, relative motion per unit reduced mass
 * (Iyer & Will 1993):
 *   a = (8/5) eta u^3 [A (n.v) n - B v],  u = 1/|r|, n = u r, v = p,
 *   A = 3 (1 + gb) v^2 + (23 + 6 ga - 9 gb) u / 3 - 5 gb (n.v)^2,
 *   B = (2 + ga) v^2 + (2 - ga) u - 3 (1 + ga) (n.v)^2.
 * (ga, gb) = (4, 5): A = 18 v^2 + 2u/3 - 25 (n.v)^2, B = 6 v^2 - 2u - 15 (n.v)^2,
 * the harmonic-gauge force.  For every (ga, gb) the losses of energy and
 * angular momentum averaged over a Kepler orbit are those of the quadrupole
 * formula (Peters & Mathews 1963), which the tests check. */
void orc_rr_accel(const orc_sys *s, orc_real ga, orc_real gb, const orc_real y[12], orc_real a[3])
{
    const orc_real *r = y, *v = y + 3;
    orc_real rr = norm3(r);
    orc_real u = 1.0 / rr;
    orc_real n[3], nv, v2, A, B, k;
    int i;
    for (i = 0; i < 3; i++) n[i] = r[i] / rr;
    nv = dot3(n, v);
    v2 = dot3(v, v);
    A = 3.0 * (1.0 + gb) * v2 + (23.0 + 6.0 * ga - 9.0 * gb) * u / 3.0 - 5.0 * gb * nv * nv;
    B = (2.0 + ga) * v2 + (2.0 - ga) * u - 3.0 * (1.0 + ga) * nv * nv;
    k = 8.0 / 5.0 * s->eta * u * u * u;
    for (i = 0; i < 3; i++) a[i] = k * (A * nv * n[i] - B * v[i]);
}

/* Eqs. 6-7 with a_2.5PN on y14 = (r, p, S1, S2, E, |J|).  Along the flow
 * dH/dt = (dH/dr).(dr/dt) + (dH/dp).(dp/dt) + sum_i (dH/dS_i).(dS_i/dt)
 *       = (dH/dp).a  (the conservative parts cancel, Omega_i.(Omega_i x S_i) = 0),
 * and dJ/dt = r x a (the conservative flow conserves J = L + S1 + S2), so
 * d|J|/dt = J.(r x a)/|J|: the integral-invariant relations of Sec. 3B. */
void orc_rhs_rr(const orc_sys *s, orc_real ga, orc_real gb, const orc_real y[14], orc_real dy[14])
{
    orc_real g[12], a[3], L[3], J[3], ra[3];
    int i;
    orc_gradient(s, y, g);
    orc_rr_accel(s, ga, gb, y, a);
    for (i = 0; i < 3; i++) {
        dy[i] = g[3 + i];              /* Eq. 6: dr/dt = dH/dp */
        dy[3 + i] = -g[i] + a[i];      /* Eq. 6: dp/dt = -dH/dr + a_2.5PN */
    }
    cross3(g + 6, y + 6, dy + 6);      /* Eq. 7 */
    cross3(g + 9, y + 9, dy + 9);
    dy[12] = dot3(g + 3, a);
    cross3(y, y + 3, L);
    for (i = 0; i < 3; i++) J[i] = L[i] + y[6 + i] + y[9 + i];
    cross3(y, a, ra);
    dy[13] = dot3(J, ra) / norm3(J);
}

/* The RK4 and fifth-order steps of orc_rk4_step / orc_rk5_step on the
 * 14-component system orc_rhs_rr. */
void orc_rk_step_rr(const orc_sys *s, orc_real ga, orc_real gb, int rk_order, orc_real y[14], orc_real h)
{
    int i;
    if (rk_order == 5) {
        static const orc_real a21 = 1.0 / 5.0;
        static const orc_real a31 = 3.0 / 40.0, a32 = 9.0 / 40.0;
        static const orc_real a41 = 44.0 / 45.0, a42 = -56.0 / 15.0, a43 = 32.0 / 9.0;
        static const orc_real a51 = 19372.0 / 6561.0, a52 = -25360.0 / 2187.0, a53 = 64448.0 / 6561.0,
                            a54 = -212.0 / 729.0;
        static const orc_real a61 = 9017.0 / 3168.0, a62 = -355.0 / 33.0, a63 = 46732.0 / 5247.0,
                            a64 = 49.0 / 176.0, a65 = -5103.0 / 18656.0;
        static const orc_real b1 = 35.0 / 384.0, b3 = 500.0 / 1113.0, b4 = 125.0 / 192.0,
                            b5 = -2187.0 / 6784.0, b6 = 11.0 / 84.0;
        orc_real k1[14], k2[14], k3[14], k4[14], k5[14], k6[14], t[14];
        orc_rhs_rr(s, ga, gb, y, k1);
        for (i = 0; i < 14; i++) t[i] = y[i] + h * (a21 * k1[i]);
        orc_rhs_rr(s, ga, gb, t, k2);
        for (i = 0; i < 14; i++) t[i] = y[i] + h * (a31 * k1[i] + a32 * k2[i]);
        orc_rhs_rr(s, ga, gb, t, k3);
        for (i = 0; i < 14; i++) t[i] = y[i] + h * (a41 * k1[i] + a42 * k2[i] + a43 * k3[i]);
        orc_rhs_rr(s, ga, gb, t, k4);
        for (i = 0; i < 14; i++) t[i] = y[i] + h * (a51 * k1[i] + a52 * k2[i] + a53 * k3[i] + a54 * k4[i]);
        orc_rhs_rr(s, ga, gb, t, k5);
        for (i = 0; i < 14; i++)
            t[i] = y[i] + h * (a61 * k1[i] + a62 * k2[i] + a63 * k3[i] + a64 * k4[i] + a65 * k5[i]);
        orc_rhs_rr(s, ga, gb, t, k6);
        for (i = 0; i < 14; i++)
            y[i] = y[i] + h * (b1 * k1[i] + b3 * k3[i] + b4 * k4[i] + b5 * k5[i] + b6 * k6[i]);
    } else {
        orc_real k1[14], k2[14], k3[14], k4[14], tmp[14];
        orc_rhs_rr(s, ga, gb, y, k1);
        for (i = 0; i < 14; i++) tmp[i] = y[i] + 0.5 * h * k1[i];
        orc_rhs_rr(s, ga, gb, tmp, k2);
        for (i = 0; i < 14; i++) tmp[i] = y[i] + 0.5 * h * k2[i];
        orc_rhs_rr(s, ga, gb, tmp, k3);
        for (i = 0; i < 14; i++) tmp[i] = y[i] + h * k3[i];
        orc_rhs_rr(s, ga, gb, tmp, k4);
        for (i = 0; i < 14; i++) y[i] = y[i] + h * (k1[i] + 2.0 * k2[i] + 2.0 * k3[i] + k4[i]) / 6.0;
    }
}

/* --------------------------------------------------------------- integrals */
void orc_integrals(const orc_sys *s, const orc_real y[12], orc_real out[7])
{
    orc_real L[3], J[3];
    int i;
    cross3(y, y + 3, L);
    for (i = 0; i < 3; i++) J[i] = L[i] + y[6 + i] + y[9 + i]; /* J = L + S1 + S2 */
    out[0] = orc_hamiltonian(s, y);
    out[1] = norm3(J);
    out[2] = norm3(y + 6);
    out[3] = norm3(y + 9);
    out[4] = J[0];
    out[5] = J[1];
    out[6] = J[2];
}

/* ------------------------------------------------------ gravitational waves */
/* Eq. 14 with the field of the mass quadrupole moment (Sec. 4, Fig. 10): at
 * distance R (in M) along N, with the relative velocity v = dr/dt = dH/dp
 * (Eq. 6) and n = r/|r|,
 *     h_ij = (4 eta / R) (v_i v_j - n_i n_j / |r|),
 *     h_plus  = (P_i P_j - Q_i Q_j) h_ij / 2,
 *     h_cross = (P_i Q_j + Q_i P_j) h_ij / 2,
 * P, Q the unit vectors of the radiation frame orthogonal to N (the
 * contraction with them takes the transverse-traceless part). */
void orc_waveform(const orc_sys *s, const orc_real y[12], orc_real R, const orc_real P[3], const orc_real Q[3],
                  orc_real out[2])
{
    orc_real g[12], h[3][3], r, hp = 0.0, hc = 0.0;
    int i, j;
    orc_gradient(s, y, g);                 /* g[3..5] = dH/dp = dr/dt */
    r = norm3(y);
    for (i = 0; i < 3; i++)
        for (j = 0; j < 3; j++)
            h[i][j] = 4.0 * s->eta / R * (g[3 + i] * g[3 + j] - (y[i] / r) * (y[j] / r) / r);
    for (i = 0; i < 3; i++)
        for (j = 0; j < 3; j++) {
            hp += 0.5 * (P[i] * P[j] - Q[i] * Q[j]) * h[i][j];
            hc += 0.5 * (P[i] * Q[j] + Q[i] * P[j]) * h[i][j];
        }
    out[0] = hp;
    out[1] = hc;
}

/* ------------------------------------------------------ manifold correction */
int orc_correct(const orc_sys *s, orc_real y[12], const orc_real ref[4],
                orc_real newton_tol, int newton_max, orc_real det_min,
                int *iters, orc_real alpha_beta[2])
{
    return orc_correct_rule(s, y, ref, newton_tol, newton_max, det_min, 0.0, 0.0, 1, ORC_MODE_DUAL, iters,
                            alpha_beta);
}

/* One Newton step of Eq. 13 at (alpha, beta): F = (H(beta r*, alpha p*, S)
 * - E0, |J(beta r*, alpha p*, S)| - J0) and its Jacobian in (alpha, beta).
 * y holds (r*, p*, S); returns 0 and the step (da, db) to subtract, or -1
 * where the dual scaling is singular (|det| <= det_min (|J11 J22| + |J12 J21|))
 * or not finite. */
static int dual_newton_step(const orc_sys *s, const orc_real y[12], const orc_real ref[4], orc_real alpha,
                            orc_real beta, orc_real det_min, orc_real *da, orc_real *db)
{
    orc_real yb[12], g[12], rs[3], ps[3];
    orc_real J[3], rxp[3], rsxp[3], rxps[3], Jn, F1, F2, A, B, C, D, det;
    int i;
    memcpy(yb, y, sizeof(yb));
    for (i = 0; i < 3; i++) {
        rs[i] = y[i];
        ps[i] = y[3 + i];
        yb[i] = beta * rs[i];
        yb[3 + i] = alpha * ps[i];
    }
    F1 = orc_hamiltonian(s, yb) - ref[0];
    cross3(yb, yb + 3, rxp);
    for (i = 0; i < 3; i++) J[i] = rxp[i] + yb[6 + i] + yb[9 + i];
    Jn = norm3(J);
    F2 = Jn - ref[1];
    orc_gradient(s, yb, g);
    A = dot3(g + 3, ps);           /* dF1/dalpha = dH/dp . p* */
    B = dot3(g, rs);               /* dF1/dbeta  = dH/dr . r* */
    cross3(yb, ps, rsxp);          /* d(r x p)/dalpha = (beta r*) x p* */
    cross3(rs, yb + 3, rxps);      /* d(r x p)/dbeta  = r* x (alpha p*) */
    C = dot3(J, rsxp) / Jn;        /* dF2/dalpha */
    D = dot3(J, rxps) / Jn;        /* dF2/dbeta */
    det = A * D - B * C;
    /* The dual scaling is singular where alpha p*.dH/dp = beta r*.dH/dr
     * (twice per orbit); there rounding noise in F would be amplified by
     * 1/det.  Below det_min relative cancellation the dual scaling is not
     * used for this step (the paper does not treat this case). */
    if (!(fabs(det) > det_min * (fabs(A * D) + fabs(B * C))) || !isfinite(det)) return -1;
    *da = (F1 * D - B * F2) / det;
    *db = (A * F2 - C * F1) / det;
    return 0;
}

/* One Newton step of the split scaling at (a, g): p = a p_t + g p_r, r = r*,
 * with p_r = (n.p*) n and p_t = p* - p_r the radial and tangential parts of
 * p* (n the unit vector along r*).  Since r* x p_r = 0, L = a (r* x p_t) =
 * a L*, so |J|
 * depends on a alone and the Jacobian of F = (H - E0, |J| - J0) in (a, g),
 *   [ p_t.dH/dp   p_r.dH/dp ]
 *   [ L*.J/|J|    0         ],
 * is triangular.  It is singular where the radial part vanishes (turning
 * points, circular orbits) or L*.J = 0; -1 is returned there, below det_min
 * of the row or column it is compared with, or if not finite. */
static int split_newton_step(const orc_sys *s, const orc_real y[12], const orc_real ref[4],
                             const orc_real pt[3], const orc_real pr[3], orc_real a, orc_real g,
                             orc_real split_min, orc_real *da, orc_real *dg)
{
    orc_real yb[12], grad[12], J[3], L[3], Ls[3], Jn, F1, F2, A, B, C;
    int i;
    memcpy(yb, y, sizeof(yb));
    for (i = 0; i < 3; i++) yb[3 + i] = a * pt[i] + g * pr[i];
    F1 = orc_hamiltonian(s, yb) - ref[0];
    cross3(yb, yb + 3, L);
    for (i = 0; i < 3; i++) J[i] = L[i] + yb[6 + i] + yb[9 + i];
    Jn = norm3(J);
    F2 = Jn - ref[1];
    orc_gradient(s, yb, grad);
    A = dot3(grad + 3, pt);          /* dF1/da */
    B = dot3(grad + 3, pr);          /* dF1/dg */
    cross3(yb, pt, Ls);              /* dL/da = r* x p_t = L* */
    C = dot3(J, Ls) / Jn;            /* dF2/da; dF2/dg = 0 */
    if (!(fabs(B) > split_min * (fabs(A) + fabs(B))) || !(fabs(C) > split_min * norm3(Ls)) ||
        !isfinite(A) || !isfinite(B) || !isfinite(C))
        return -1;
    *da = F2 / C;
    *dg = (F1 - A * (*da)) / B;
    return 0;
}

int orc_newton_trace(const orc_sys *s, const orc_real y[12], const orc_real ref[4], int kmax,
                     orc_real *alpha, orc_real *beta)
{
    orc_real a = 1.0, b = 1.0, da, db;
    int k;
    for (k = 0; k < kmax; k++) {
        if (dual_newton_step(s, y, ref, a, b, 0.0, &da, &db)) break;
        a = a - da;
        b = b - db;
        alpha[k] = a;
        beta[k] = b;
    }
    return k;
}

/* Conditioning of the two scalings at the unscaled point y = (r*, p*, S):
 * the dual scaling's relative determinant |A - B| / (|A| + |B|), with
 * A = p*.dH/dp and B = r*.dH/dr (its two |J| derivatives are equal there);
 * and the split scaling's |p_r.dH/dp| / (|p_t.dH/dp| + |p_r.dH/dp|), or 0
 * where its |J| row is degenerate (|L*.J|/|J| <= split_min |L*|). */
static void conditioning(const orc_sys *s, const orc_real y[12], orc_real split_min, orc_real *c_dual,
                         orc_real *c_split)
{
    orc_real g[12], pr[3], pt[3], L[3], J[3], A, B, As, Bs, rn, np_;
    int i;
    orc_gradient(s, y, g);
    A = dot3(g + 3, y + 3);
    B = dot3(g, y);
    *c_dual = fabs(A - B) / (fabs(A) + fabs(B));
    rn = norm3(y);
    np_ = dot3(y, y + 3) / rn;
    for (i = 0; i < 3; i++) {
        pr[i] = np_ * (y[i] / rn);
        pt[i] = y[3 + i] - pr[i];
    }
    As = dot3(g + 3, pt);
    Bs = dot3(g + 3, pr);
    cross3(y, y + 3, L);
    for (i = 0; i < 3; i++) J[i] = L[i] + y[6 + i] + y[9 + i];
    *c_split = fabs(Bs) / (fabs(As) + fabs(Bs));
    if (!(fabs(dot3(J, L)) / norm3(J) > split_min * norm3(L))) *c_split = 0.0;
    if (!isfinite(*c_dual)) *c_dual = 0.0;
    if (!isfinite(*c_split)) *c_split = 0.0;
}

int orc_correct_rule(const orc_sys *s, orc_real y[12], const orc_real ref[4],
                     orc_real newton_tol, int newton_max, orc_real det_min, orc_real split_min,
                     orc_real cond_switch, int apply_small, int mode, int *iters, orc_real alpha_beta[2])
{
    orc_real rs[3], ps[3], yb[12];
    orc_real alpha = 1.0, beta = 1.0;
    int it = 0, i, converged = 0, prefer_split = 0;

    /* Eq. 10: restore both spin lengths (skipped for a zero-length spin). */
    for (i = 0; i < 2; i++) {
        orc_real *S = y + 6 + 3 * i, len = norm3(S);
        if (ref[2 + i] > 0.0 && len > 0.0) {
            S[0] = S[0] * (ref[2 + i] / len);
            S[1] = S[1] * (ref[2 + i] / len);
            S[2] = S[2] * (ref[2 + i] / len);
        }
    }

    if (mode == ORC_MODE_SPINS) {          /* ablation: Eq. 10 alone */
        if (iters) *iters = 0;
        if (alpha_beta) {
            alpha_beta[0] = 1.0;
            alpha_beta[1] = 1.0;
        }
        return ORC_CORR_SKIPPED;
    }

    /* Eqs. 11-13: p = alpha p*, r = beta r*; the two conditions
     * H(beta r*, alpha p*, S) = E0 and |J(beta r*, alpha p*, S)| = J0 make the
     * least-squares function of Eq. 12 vanish; Newton from (1, 1). */
    for (i = 0; i < 3; i++) {
        rs[i] = y[i];
        ps[i] = y[3 + i];
    }
    memcpy(yb, y, sizeof(yb));
    /* mode ORC_MODE_VELOCITY (ablation): no dual scaling, straight to the
     * velocity scaling below */
    /* In the dual scaling's ill-conditioned band (relative determinant at
     * most cond_switch) the split scaling is used instead where it is better
     * conditioned: rounding in F reaches the correction amplified by the
     * inverse conditioning, and kicks that differ between the two FLI
     * trajectories would masquerade as divergence. */
    if (mode == ORC_MODE_DUAL && cond_switch > 0.0 && split_min > 0.0) {
        orc_real cd, cs;
        conditioning(s, y, split_min, &cd, &cs);
        if (cd <= cond_switch && cs > cd && cs > split_min) prefer_split = 1;
    }
    for (it = 1; mode == ORC_MODE_DUAL && !prefer_split && it <= newton_max; it++) {
        orc_real da, db;
        if (dual_newton_step(s, y, ref, alpha, beta, det_min, &da, &db)) break;
        /* stopping rule: apply the step and then test it (default), or stop
         * before applying a step already within the tolerance */
        if (!apply_small && fabs(da) <= newton_tol && fabs(db) <= newton_tol) {
            converged = 1;
            break;
        }
        alpha = alpha - da;
        beta = beta - db;
        if (!isfinite(alpha) || !isfinite(beta)) break;
        if (fabs(da) <= newton_tol && fabs(db) <= newton_tol) {
            converged = 1;
            break;
        }
    }
    if (mode != ORC_MODE_DUAL || prefer_split) it = 0;
    if (it > newton_max) it = newton_max;
    if (converged) {
        for (i = 0; i < 3; i++) {
            y[i] = beta * rs[i];
            y[3 + i] = alpha * ps[i];
        }
        if (iters) *iters = it;
        if (alpha_beta) {
            alpha_beta[0] = alpha;
            alpha_beta[1] = beta;
        }
        return ORC_CORR_OK;
    }
    /* Singular (or non-converged) dual scaling: both integrals by the split
     * scaling p = a p_t + g p_r (r* kept), 2x2 Newton on (a, g) from (1, 1)
     * with the same stopping rule.  The dual scaling is singular where
     * p*.dH/dp = r*.dH/dr (for a Kepler ellipse at r = a, where
     * |p_r| / |p| = e), away from the turning points where this one is. */
    if (mode == ORC_MODE_DUAL && split_min > 0.0) {
        orc_real pt[3], pr[3], rn = norm3(rs), np_ = dot3(rs, ps) / rn, a = 1.0, g = 1.0;
        int k, ok = 0;
        for (i = 0; i < 3; i++) {
            pr[i] = np_ * (rs[i] / rn);
            pt[i] = ps[i] - pr[i];
        }
        for (k = 1; k <= newton_max; k++) {
            orc_real da, dg;
            if (split_newton_step(s, y, ref, pt, pr, a, g, split_min, &da, &dg)) break;
            if (!apply_small && fabs(da) <= newton_tol && fabs(dg) <= newton_tol) {
                ok = 1;
                break;
            }
            a = a - da;
            g = g - dg;
            if (!isfinite(a) || !isfinite(g)) break;
            if (fabs(da) <= newton_tol && fabs(dg) <= newton_tol) {
                ok = 1;
                break;
            }
        }
        if (k > newton_max) k = newton_max;
        if (ok) {
            for (i = 0; i < 3; i++) y[3 + i] = a * pt[i] + g * pr[i];
            if (iters) *iters = it + k;
            if (alpha_beta) {
                alpha_beta[0] = a;
                alpha_beta[1] = g;
            }
            return ORC_CORR_SPLIT;
        }
        it += k;
    }
    /* Both singular (or non-converged): restore the energy alone by
     * velocity scaling, p = a p*, H(r*, a p*, S) = E0, Newton in a from 1
     * (the momentum-scaling correction of Sec. 1, Wu et al. 2007).  |J| is
     * left to the next step. */
    {
        orc_real a = 1.0, g2[12];
        int k, ok = 0;
        memcpy(yb, y, sizeof(yb));
        for (k = 1; k <= newton_max; k++) {
            orc_real F, A, da;
            for (i = 0; i < 3; i++) yb[3 + i] = a * ps[i];
            F = orc_hamiltonian(s, yb) - ref[0];
            orc_gradient(s, yb, g2);
            A = dot3(g2 + 3, ps);             /* dH/da = dH/dp . p* */
            da = F / A;
            if (!isfinite(da)) break;
            if (!apply_small && fabs(da) <= newton_tol) {
                ok = 1;
                break;
            }
            a = a - da;
            if (fabs(da) <= newton_tol) {
                ok = 1;
                break;
            }
        }
        if (k > newton_max) k = newton_max;
        if (iters) *iters = it + k;
        if (alpha_beta) {
            alpha_beta[0] = ok ? a : 1.0;
            alpha_beta[1] = 1.0;
        }
        if (!ok) return ORC_CORR_SKIPPED;  /* keep the spin-corrected r*, p* */
        for (i = 0; i < 3; i++) y[3 + i] = a * ps[i];
        return ORC_CORR_VELOCITY;
    }
}

/* ------------------------------------------------------------ cell set-up */
void orc_setup_cell(const orc_real cell[9], orc_real y[12])
{
    orc_real x0 = cell[0], pfac = cell[1];
    orc_real beta = cell[6], m1 = beta / (1.0 + beta), m2 = 1.0 / (1.0 + beta);
    orc_real s1 = cell[7] * m1 * m1, s2 = cell[8] * m2 * m2;
    y[0] = x0;
    y[1] = 0.0;
    y[2] = 0.0;
    y[3] = 0.0;
    y[4] = pfac / sqrt(x0); /* fraction of the Newtonian circular momentum */
    y[5] = 0.0;
    y[6] = s1 * sin(cell[2]) * cos(cell[3]);
    y[7] = s1 * sin(cell[2]) * sin(cell[3]);
    y[8] = s1 * cos(cell[2]);
    y[9] = s2 * sin(cell[4]) * cos(cell[5]);
    y[10] = s2 * sin(cell[4]) * sin(cell[5]);
    y[11] = s2 * cos(cell[4]);
}

/* ------------------------------------------------------------- integrator */
static void reference_integrals(const orc_sys *s, const orc_real y[12], orc_real ref[4])
{
    orc_real I[7];
    orc_integrals(s, y, I);
    ref[0] = I[0];
    ref[1] = I[1];
    ref[2] = I[2];
    ref[3] = I[3];
}

static int all_finite(const orc_real y[12])
{
    int i;
    for (i = 0; i < 12; i++)
        if (!isfinite(y[i])) return 0;
    return 1;
}

static orc_real distance12(const orc_real a[12], const orc_real b[12])
{
    orc_real d2 = 0.0;
    int i;
    for (i = 0; i < 12; i++) d2 += (b[i] - a[i]) * (b[i] - a[i]);
    return sqrt(d2);
}

/* One integration step of a trajectory.  Without radiation reaction the
 * reference integrals stay fixed; with it, ref[0] = E and ref[1] = |J|
 * advance with the state by their integral-invariant relations. */
static void step(const orc_config *cfg, const orc_sys *s, orc_real y[12], orc_real ref[4], orc_real h)
{
    if (cfg->rr) {
        orc_real y14[14];
        memcpy(y14, y, 12 * sizeof(orc_real));
        y14[12] = ref[0];
        y14[13] = ref[1];
        orc_rk_step_rr(s, cfg->rr_gauge_a, cfg->rr_gauge_b, cfg->rk_order, y14, h);
        memcpy(y, y14, 12 * sizeof(orc_real));
        ref[0] = y14[12];
        ref[1] = y14[13];
    } else if (cfg->rk_order == 5) {
        orc_rk5_step(s, y, h);
    } else {
        orc_rk4_step(s, y, h);
    }
}

static void integrate_one(const orc_config *cfg, const orc_sys *s, const orc_real y0[12],
                          orc_real h, int64_t nsteps, orc_real y[12], orc_real ys[12],
                          orc_real integ[6], orc_real *fli_out, int32_t *status_out,
                          orc_real *t_stop_out, int64_t *iters_out, int32_t *skip_out,
                          int32_t *last_kind_out)
{
    orc_real ref[4], refs[4], acc = 0.0, d0 = cfg->fli_d0;
    int64_t k, iters = 0;
    int32_t st = ORC_DONE, skips = 0, last_kind = ORC_CORR_OK;
    orc_real t_stop = (orc_real)nsteps * h;

    memcpy(y, y0, 12 * sizeof(orc_real));
    memcpy(ys, y0, 12 * sizeof(orc_real));
    ys[0] = ys[0] + d0; /* shadow displaced by d0 along x */
    reference_integrals(s, y, ref);
    reference_integrals(s, ys, refs);

    for (k = 1; k <= nsteps; k++) {
        int it = 0;
        step(cfg, s, y, ref, h);
        if (cfg->correct) {
            last_kind = orc_correct_rule(s, y, ref, cfg->newton_tol, cfg->newton_max, cfg->det_min,
                                         cfg->split_min, cfg->cond_switch, cfg->newton_apply_small, cfg->correct, &it, 0);
            if (last_kind != ORC_CORR_OK) skips++;
            iters += it;
        }
        step(cfg, s, ys, refs, h);
        if (cfg->correct) {
            if (orc_correct_rule(s, ys, refs, cfg->newton_tol, cfg->newton_max, cfg->det_min,
                                 cfg->split_min, cfg->cond_switch, cfg->newton_apply_small, cfg->correct, &it, 0))
                skips++;
            iters += it;
        }
        /* termination tests on the main trajectory */
        if (!all_finite(y) || !all_finite(ys)) { st = ORC_NONFINITE; t_stop = (orc_real)k * h; break; }
        {
            orc_real rr = norm3(y);
            if (cfg->r_merge > 0.0 && rr < cfg->r_merge) { st = ORC_MERGED; t_stop = (orc_real)k * h; break; }
            if (cfg->r_escape > 0.0 && rr > cfg->r_escape) { st = ORC_ESCAPED; t_stop = (orc_real)k * h; break; }
        }
        /* FLI renormalisation every fli_renorm steps */
        if (cfg->fli_renorm > 0 && k % cfg->fli_renorm == 0) {
            orc_real d = distance12(y, ys);
            int i;
            acc += log10(d / d0);
            for (i = 0; i < 12; i++) ys[i] = y[i] + (d0 / d) * (ys[i] - y[i]);
            reference_integrals(s, ys, refs); /* the shadow keeps its own integrals */
            if (cfg->fli_cap > 0.0 && acc >= cfg->fli_cap) { st = ORC_FLI_SATURATED; t_stop = (orc_real)k * h; break; }
        }
    }
    {
        orc_real I[7];
        orc_integrals(s, y, I);
        integ[0] = ref[0];
        integ[1] = I[0];
        integ[2] = ref[1];
        integ[3] = I[1];
        integ[4] = I[2];
        integ[5] = I[3];
    }
    *fli_out = acc + log10(distance12(y, ys) / d0);
    *status_out = st;
    *t_stop_out = t_stop;
    *iters_out = iters;
    *skip_out = skips;
    *last_kind_out = last_kind;
}

int orc_scan(int64_t n, const orc_real *y0, const orc_real *beta,
             const orc_real *kappa1, const orc_real *kappa2,
             const orc_config *cfg, orc_real h, int64_t nsteps,
             orc_real *y_out, orc_real *ys_out, orc_real *integrals, orc_real *fli,
             int32_t *status, orc_real *t_stop, int64_t *newton_iters,
             int32_t *n_skip, int32_t *last_kind, int nthreads)
{
    int64_t i;
    if (n < 0 || nsteps < 0 || !y0 || !beta || !cfg || !y_out || !ys_out || !integrals ||
        !fli || !status || !t_stop || !newton_iters || !n_skip || !last_kind)
        return -1;
#ifdef _OPENMP
    if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads)
#endif
    for (i = 0; i < n; i++) {
        orc_sys s;
        orc_sys_init(&s, beta[i], kappa1 ? kappa1[i] : 1.0, kappa2 ? kappa2[i] : 1.0,
                     cfg->pn_order, cfg->use_so, cfg->use_ss, cfg->use_qm);
        integrate_one(cfg, &s, y0 + 12 * i, h, nsteps, y_out + 12 * i, ys_out + 12 * i,
                      integrals + 6 * i, fli + i, status + i, t_stop + i, newton_iters + i,
                      n_skip + i, last_kind + i);
    }
    (void)nthreads;
    return 0;
}

int orc_trace(const orc_real y0[12], orc_real beta, orc_real kappa1, orc_real kappa2,
              const orc_config *cfg, orc_real h, int64_t nsteps, int64_t every,
              orc_real *trace)
{
    orc_sys s;
    orc_real y[12], ref[4];
    int64_t k, m = 0;
    if (every <= 0 || !trace) return -1;
    orc_sys_init(&s, beta, kappa1, kappa2, cfg->pn_order, cfg->use_so, cfg->use_ss, cfg->use_qm);
    memcpy(y, y0, sizeof(y));
    reference_integrals(&s, y, ref);
    for (k = 1; k <= nsteps; k++) {
        int it;
        step(cfg, &s, y, ref, h);
        if (cfg->correct)
            orc_correct_rule(&s, y, ref, cfg->newton_tol, cfg->newton_max, cfg->det_min,
                             cfg->split_min, cfg->cond_switch, cfg->newton_apply_small, cfg->correct, &it, 0);
        if (k % every == 0) {
            memcpy(trace + 12 * m, y, sizeof(y));
            m++;
        }
    }
    return 0;
}

int orc_ext_trace(const double y0[12], double beta, double kappa1, double kappa2,
                  const orc_config *cfg, double h, int64_t nsteps, double y_out[12])
{
    orc_sys s;
    orc_real y[12], ref[4];
    int64_t k;
    int i;
    if (!y0 || !cfg || !y_out || nsteps < 0) return -1;
    orc_sys_init(&s, beta, kappa1, kappa2, cfg->pn_order, cfg->use_so, cfg->use_ss, cfg->use_qm);
    for (i = 0; i < 12; i++) y[i] = y0[i];
    reference_integrals(&s, y, ref);
    for (k = 1; k <= nsteps; k++) {
        int it;
        step(cfg, &s, y, ref, h);
        if (cfg->correct)
            orc_correct_rule(&s, y, ref, cfg->newton_tol, cfg->newton_max, cfg->det_min,
                             cfg->split_min, cfg->cond_switch, cfg->newton_apply_small, cfg->correct, &it, 0);
    }
    for (i = 0; i < 12; i++) y_out[i] = (double)y[i];
    return 0;
}

int orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
