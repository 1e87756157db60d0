// pn_device.cuh -- FP64 device arithmetic of the manifold-corrected PN scan
// (arXiv:1802.00147): Hamiltonian and equations of motion (Sec. 2, Eqs. 1-9),
// fixed-step RK4 and fifth-order Runge-Kutta steps, the manifold correction
// (Eqs. 10-13) and its ablation modes; the optional 2.5PN radiation
// reaction of Eq. 6 with the integral-invariant reference values of Sec. 3B.
//
// Everything here runs in the registers of the thread that owns an orbit (or,
// in the paired kernel, one of its two trajectories).  On GB300 the
// FP64 pipe retires two DFMA per SM per clock, so these routines are written
// to minimise FP64 instructions: every product-sum is an fma, per-orbit
// constants are pre-multiplied once, and the Newton solve of Eq. 13 evaluates
// H at the scaled point from monomials in (alpha, 1/beta) instead of
// re-evaluating the Hamiltonian.
//
// Units: G = c = M = 1; r in M, p in mu, H in mu, t in M, spins in M^2
// (the reading under which Eqs. 8-9 are the exact spin gradients of H).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace pnscan {

// ------------------------------------------------------------------ state
struct Vec12 {
    double r[3], p[3], s1[3], s2[3];
};

// Per-orbit constants derived from (beta, kappa1, kappa2) and the term flags.
// Orbital Hamiltonian H_O(p2, np, u), u = 1/|r|, np = n.p (Sec. 2):
//   H_N   = p2/2 - u
//   H_1PN = a1 p2^2 + u (b1 p2 + b2 np^2) + h1 u^2
//   H_2PN = a2 p2^3 + u (c1 p2^2 + c2 p2 np^2 + c3 np^4) + u^2 (d1 p2 + d2 np^2) + e1 u^3
// a1 = (3 eta - 1)/8, b1 = -(3 + eta)/2, b2 = -eta/2, h1 = 1/2,
// a2 = (1 - 5 eta + 5 eta^2)/16, c1 = (5 - 20 eta - 3 eta^2)/8, c2 = -eta^2/4,
// c3 = -3 eta^2/8, d1 = (5 + 8 eta)/2, d2 = 3 eta/2, e1 = -(1 + 3 eta)/4.
// Spin terms: H_SO = u^3 L.(g1 S1 + g2 S2), g1 = 2 + 3/(2 beta), g2 = 2 + 3 beta/2
// (Eqs. 8-9); H_S1S2 = ieta u^3 [3 (S1.n)(S2.n) - S1.S2] (Eq. 3 with the 1/eta
// of Eqs. 8-9); H_QM = u^3 [q1 (3 (S1.n)^2 - S1^2) + q2 (3 (S2.n)^2 - S2^2)],
// q1 = kappa1/(2 beta eta), q2 = kappa2 beta/(2 eta) (Eqs. 4-5).
enum CoefIdx : int {
    // value of H (integrals, Newton monomials)
    K_A1, K_B1, K_B2, K_H1, K_A2, K_C1, K_C2, K_C3, K_D1, K_D2, K_E1,
    K_G1, K_G2, K_IETA, K_Q1, K_Q2,
    // derivative polynomials, pre-multiplied
    K_A1X4, K_A2X6, K_C1X4, K_C2X2, K_D1X2, K_B1X2,   // 2 dH/dp2
    K_B2X2, K_C3X4, K_D2X2,                          // W = H_np / np
    K_H1X2, K_E1X3,                                  // dH/du
    K_IETA3, K_IETA15, K_Q1X6, K_Q2X6, K_Q1X15, K_Q2X15, K_Q1X3, K_Q2X3,
    NCOEF
};

// Per-orbit constants held in registers.
struct Coef {
    double v[NCOEF];
    __host__ __device__ double operator[](int k) const { return v[k]; }
};

// Per-orbit constants held in shared memory, one plane per constant across
// the block's threads (consecutive threads, consecutive doubles): read on
// use, so they cost no registers between uses.
struct CoefShared {
    const volatile double* p;   // &plane[0][threadIdx.x]
    int stride;                 // threads per block
    __device__ double operator[](int k) const { return p[k * stride]; }
};

struct Flags {
    int pn_order;          // 0, 1, 2
    int use_so, use_ss, use_qm;
};

__host__ __device__ inline Coef make_coef(double beta, double kappa1, double kappa2, Flags f)
{
    Coef c;
    double* v = c.v;
    const double eta = beta / ((1.0 + beta) * (1.0 + beta));
    const double pn1 = f.pn_order >= 1 ? 1.0 : 0.0;
    const double pn2 = f.pn_order >= 2 ? 1.0 : 0.0;
    v[K_A1] = pn1 * (3.0 * eta - 1.0) / 8.0;
    v[K_B1] = pn1 * -(3.0 + eta) / 2.0;
    v[K_B2] = pn1 * -eta / 2.0;
    v[K_H1] = pn1 * 0.5;
    v[K_A2] = pn2 * (1.0 - 5.0 * eta + 5.0 * eta * eta) / 16.0;
    v[K_C1] = pn2 * (5.0 - 20.0 * eta - 3.0 * eta * eta) / 8.0;
    v[K_C2] = pn2 * -(eta * eta) / 4.0;
    v[K_C3] = pn2 * -3.0 * eta * eta / 8.0;
    v[K_D1] = pn2 * (5.0 + 8.0 * eta) / 2.0;
    v[K_D2] = pn2 * 3.0 * eta / 2.0;
    v[K_E1] = pn2 * -(1.0 + 3.0 * eta) / 4.0;
    v[K_G1] = f.use_so ? 2.0 + 3.0 / (2.0 * beta) : 0.0;
    v[K_G2] = f.use_so ? 2.0 + 1.5 * beta : 0.0;
    v[K_IETA] = f.use_ss ? 1.0 / eta : 0.0;
    v[K_Q1] = f.use_qm ? kappa1 / (2.0 * beta * eta) : 0.0;
    v[K_Q2] = f.use_qm ? kappa2 * beta / (2.0 * eta) : 0.0;
    // 2 dH/dp2 = 1 + 4 a1 p2 + 2 b1 u + 6 a2 p2^2 + u (4 c1 p2 + 2 c2 np^2) + 2 d1 u^2
    v[K_A1X4] = 4.0 * v[K_A1];
    v[K_A2X6] = 6.0 * v[K_A2];
    v[K_C1X4] = 4.0 * v[K_C1];
    v[K_C2X2] = 2.0 * v[K_C2];
    v[K_D1X2] = 2.0 * v[K_D1];
    v[K_B1X2] = 2.0 * v[K_B1];
    // W = H_np / np = u (2 b2 + 2 c2 p2 + 4 c3 np^2 + 2 d2 u)
    v[K_B2X2] = 2.0 * v[K_B2];
    v[K_C3X4] = 4.0 * v[K_C3];
    v[K_D2X2] = 2.0 * v[K_D2];
    // dH/du = -1 + p2 (b1 + c1 p2 + c2 np^2) + np^2 (b2 + c3 np^2)
    //         + u (2 h1 + 2 d1 p2 + 2 d2 np^2 + 3 e1 u)
    v[K_H1X2] = 2.0 * v[K_H1];
    v[K_E1X3] = 3.0 * v[K_E1];
    v[K_IETA3] = 3.0 * v[K_IETA];
    v[K_IETA15] = 15.0 * v[K_IETA];
    v[K_Q1X6] = 6.0 * v[K_Q1];
    v[K_Q2X6] = 6.0 * v[K_Q2];
    v[K_Q1X15] = 15.0 * v[K_Q1];
    v[K_Q2X15] = 15.0 * v[K_Q2];
    v[K_Q1X3] = 3.0 * v[K_Q1];
    v[K_Q2X3] = 3.0 * v[K_Q2];
    return c;
}

__device__ __forceinline__ double dot3(const double* a, const double* b)
{
    return fma(a[0], b[0], fma(a[1], b[1], a[2] * b[2]));
}

// ------------------------------------------------------- equations of motion
// dy/dt = (dH/dp, -dH/dr, Omega_1 x S1, Omega_2 x S2)  (Eqs. 6-7, a_2.5PN = 0)
// With n = u r, np = u (r.p), H_np = np W and E = u^3 Seff:
//   dH/dp = 2 H_p2 p + (np W u) r + E x r
//   dH/dr = u np W p - u^2 (u H_u + np^2 W) r + p x E - 3 u^2 (L.E) r
//           + spin-spin / QM parts (see below)
//
// rhs_u takes u = 1/|r| = rsqrt(r.r) from the caller (so that the caller can
// start it early); rhs computes it.
template <bool QM, class C>
__device__ __forceinline__ void rhs_u(const C& c, const Vec12& y, double u, Vec12& dy)
{
    const double* r = y.r;
    const double* p = y.p;
    const double* S1 = y.s1;
    const double* S2 = y.s2;

    const double u2 = u * u;
    const double u3 = u2 * u;
    const double u5 = u3 * u2;
    const double rp = dot3(r, p);
    const double p2 = dot3(p, p);
    const double np = rp * u;
    const double np2 = np * np;
    const double a1s = dot3(S1, r);     // (S1.n) / u
    const double a2s = dot3(S2, r);
    const double S12 = dot3(S1, S2);

    // L = r x p; E = u^3 Seff = G1 S1 + G2 S2 with G_i = u^3 g_i (Seff = g1 S1 + g2 S2)
    const double L0 = fma(r[1], p[2], -r[2] * p[1]);
    const double L1 = fma(r[2], p[0], -r[0] * p[2]);
    const double L2 = fma(r[0], p[1], -r[1] * p[0]);
    const double G1 = u3 * c[K_G1], G2 = u3 * c[K_G2];
    const double E0 = fma(G1, S1[0], G2 * S2[0]);
    const double E1 = fma(G1, S1[1], G2 * S2[1]);
    const double E2 = fma(G1, S1[2], G2 * S2[2]);
    const double LE = fma(L0, E0, fma(L1, E1, L2 * E2));                     // u^3 L.Seff

    // orbital partial derivatives
    const double tq = fma(c[K_C2], np2, c[K_B1]);                                 // b1 + c2 np^2
    const double Hp2x2 = fma(fma(c[K_A2X6], p2, c[K_A1X4]), p2, 1.0)
                       + u * fma(c[K_D1X2], u, fma(c[K_C1X4], p2, fma(c[K_C2X2], np2, c[K_B1X2])));
    const double W = u * fma(c[K_D2X2], u, fma(c[K_C2X2], p2, fma(c[K_C3X4], np2, c[K_B2X2])));
    const double Hu = fma(fma(c[K_C1], p2, tq), p2, -1.0) + np2 * fma(c[K_C3], np2, c[K_B2])
                    + u * fma(c[K_E1X3], u, fma(c[K_D1X2], p2, fma(c[K_D2X2], np2, c[K_H1X2])));
    const double cr = np * W * u;                                            // H_np u

    // spin-spin and QM scalars:
    //   V1 = u^5 (3 ieta a2s + 6 q1 a1s),  V2 = u^5 (3 ieta a1s + 6 q2 a2s)
    //   Ar = u^2 (u H_u + np^2 W + 3 u^3 L.Seff)
    //      + u^5 [15 u^2 (ieta a1s a2s + q1 a1s^2 + q2 a2s^2) - 3 ieta S12 - 3 (q1 S11 + q2 S22)]
    double V1, V2, Ass;   // Ass: the u^5 [...] spin part of Ar
    if (QM) {
        const double T1 = fma(c[K_Q1X6], a1s, c[K_IETA3] * a2s);
        const double T2 = fma(c[K_Q2X6], a2s, c[K_IETA3] * a1s);
        const double Q = fma(c[K_Q1X15] * a1s, a1s, fma(c[K_Q2X15] * a2s, a2s, c[K_IETA15] * (a1s * a2s)));
        const double K = fma(-c[K_Q1X3], dot3(S1, S1), fma(-c[K_Q2X3], dot3(S2, S2), -c[K_IETA3] * S12));
        V1 = u5 * T1;
        V2 = u5 * T2;
        Ass = u5 * fma(Q, u2, K);
    } else {
        // common factor w = 3 ieta u^5:  V1 = w a2s, V2 = w a1s, Ass = w (5 u^2 a1s a2s - S12)
        const double w = u5 * c[K_IETA3];
        V1 = w * a2s;
        V2 = w * a1s;
        Ass = w * fma(a1s * a2s, 5.0 * u2, -S12);
    }
    const double Ar = fma(u2, fma(3.0, LE, fma(np2, W, u * Hu)), Ass);

    // dr/dt = Hp2x2 p + cr r + E x r
    const double X0 = fma(E1, r[2], -E2 * r[1]);
    const double X1 = fma(E2, r[0], -E0 * r[2]);
    const double X2 = fma(E0, r[1], -E1 * r[0]);
    dy.r[0] = fma(Hp2x2, p[0], fma(cr, r[0], X0));
    dy.r[1] = fma(Hp2x2, p[1], fma(cr, r[1], X1));
    dy.r[2] = fma(Hp2x2, p[2], fma(cr, r[2], X2));

    // dp/dt = -cr p + Ar r - V1 S1 - V2 S2 - p x E
    const double Y0 = fma(p[1], E2, -p[2] * E1);
    const double Y1 = fma(p[2], E0, -p[0] * E2);
    const double Y2 = fma(p[0], E1, -p[1] * E0);
    dy.p[0] = fma(-cr, p[0], fma(Ar, r[0], fma(-V1, S1[0], fma(-V2, S2[0], -Y0))));
    dy.p[1] = fma(-cr, p[1], fma(Ar, r[1], fma(-V1, S1[1], fma(-V2, S2[1], -Y1))));
    dy.p[2] = fma(-cr, p[2], fma(Ar, r[2], fma(-V1, S1[2], fma(-V2, S2[2], -Y2))));

    // dS1/dt = (u^3 g1 L + V1 r - u^3 ieta S2) x S1, and 1 <-> 2 (Eqs. 7-9)
    const double I3 = u3 * c[K_IETA];
    const double O10 = fma(G1, L0, fma(V1, r[0], -I3 * S2[0]));
    const double O11 = fma(G1, L1, fma(V1, r[1], -I3 * S2[1]));
    const double O12 = fma(G1, L2, fma(V1, r[2], -I3 * S2[2]));
    dy.s1[0] = fma(O11, S1[2], -O12 * S1[1]);
    dy.s1[1] = fma(O12, S1[0], -O10 * S1[2]);
    dy.s1[2] = fma(O10, S1[1], -O11 * S1[0]);
    const double O20 = fma(G2, L0, fma(V2, r[0], -I3 * S1[0]));
    const double O21 = fma(G2, L1, fma(V2, r[1], -I3 * S1[1]));
    const double O22 = fma(G2, L2, fma(V2, r[2], -I3 * S1[2]));
    dy.s2[0] = fma(O21, S2[2], -O22 * S2[1]);
    dy.s2[1] = fma(O22, S2[0], -O20 * S2[2]);
    dy.s2[2] = fma(O20, S2[1], -O21 * S2[0]);
}

template <bool QM, class C>
__device__ __forceinline__ void rhs(const C& c, const Vec12& y, Vec12& dy)
{
    rhs_u<QM, C>(c, y, rsqrt(dot3(y.r, y.r)), dy);
}

// ------------------------------------------------------------ Hamiltonian
template <bool QM, class C>
__device__ __forceinline__ double hamiltonian(const C& c, const Vec12& y)
{
    const double rr2 = dot3(y.r, y.r);
    const double u = rsqrt(rr2);
    const double p2 = dot3(y.p, y.p);
    const double np = dot3(y.r, y.p) * u;
    const double np2 = np * np;
    const double L0 = fma(y.r[1], y.p[2], -y.r[2] * y.p[1]);
    const double L1 = fma(y.r[2], y.p[0], -y.r[0] * y.p[2]);
    const double L2 = fma(y.r[0], y.p[1], -y.r[1] * y.p[0]);
    const double LS1 = fma(L0, y.s1[0], fma(L1, y.s1[1], L2 * y.s1[2]));
    const double LS2 = fma(L0, y.s2[0], fma(L1, y.s2[1], L2 * y.s2[2]));
    const double a1 = dot3(y.s1, y.r) * u, a2 = dot3(y.s2, y.r) * u;
    const double u3 = u * u * u;
    double Hp = fma(fma(c[K_A2], p2, c[K_A1]), p2, 0.5) * p2;                         // p2/2 + a1 p2^2 + a2 p2^3
    double Hu1 = fma(c[K_B1], p2, c[K_B2] * np2) + p2 * fma(c[K_C1], p2, c[K_C2] * np2) + c[K_C3] * np2 * np2 - 1.0;
    double Hu2 = fma(c[K_D1], p2, fma(c[K_D2], np2, c[K_H1]));
    double Hu3 = c[K_E1] + c[K_IETA] * fma(3.0 * a1, a2, -dot3(y.s1, y.s2));
    if (QM)
        Hu3 += c[K_Q1] * fma(3.0 * a1, a1, -dot3(y.s1, y.s1)) + c[K_Q2] * fma(3.0 * a2, a2, -dot3(y.s2, y.s2));
    const double Hso = u3 * fma(c[K_G1], LS1, c[K_G2] * LS2);
    return Hp + u * fma(u, fma(u, Hu3, Hu2), Hu1) + Hso;
}

// |J|, J = L + S1 + S2
__device__ __forceinline__ double jnorm(const Vec12& y)
{
    const double J0 = fma(y.r[1], y.p[2], -y.r[2] * y.p[1]) + y.s1[0] + y.s2[0];
    const double J1 = fma(y.r[2], y.p[0], -y.r[0] * y.p[2]) + y.s1[1] + y.s2[1];
    const double J2 = fma(y.r[0], y.p[1], -y.r[1] * y.p[0]) + y.s1[2] + y.s2[2];
    return sqrt(fma(J0, J0, fma(J1, J1, J2 * J2)));
}

// Reference integrals of one trajectory: E0, J0, |S1|0, |S2|0 (Eq. 12).
struct Ref {
    double E, J, S1, S2;
};

template <bool QM, class C>
__device__ __forceinline__ Ref integrals(const C& c, const Vec12& y)
{
    Ref R;
    R.E = hamiltonian<QM>(c, y);
    R.J = jnorm(y);
    R.S1 = sqrt(dot3(y.s1, y.s1));
    R.S2 = sqrt(dot3(y.s2, y.s2));
    return R;
}

// ------------------------------------------------------------------- RK4
template <bool QM, class C>
__device__ __forceinline__ void rk4_step(const C& c, Vec12& y, double h)
{
    const double h2 = 0.5 * h, h3 = h * (1.0 / 3.0), h6 = h * (1.0 / 6.0);
    Vec12 k, st, acc;
    double* yv = &y.r[0];
    double* kv = &k.r[0];
    double* sv = &st.r[0];
    double* av = &acc.r[0];
    rhs<QM>(c, y, k);
#pragma unroll
    for (int i = 0; i < 12; i++) {
        av[i] = fma(h6, kv[i], yv[i]);
        sv[i] = fma(h2, kv[i], yv[i]);
    }
    rhs<QM>(c, st, k);
#pragma unroll
    for (int i = 0; i < 12; i++) {
        av[i] = fma(h3, kv[i], av[i]);
        sv[i] = fma(h2, kv[i], yv[i]);
    }
    rhs<QM>(c, st, k);
#pragma unroll
    for (int i = 0; i < 12; i++) {
        av[i] = fma(h3, kv[i], av[i]);
        sv[i] = fma(h, kv[i], yv[i]);
    }
    rhs<QM>(c, st, k);
#pragma unroll
    for (int i = 0; i < 12; i++) yv[i] = fma(h6, kv[i], av[i]);
}

// The same RK4 step with the four stages in a loop that is not unrolled, so
// the equations of motion are compiled once instead of four times (smaller
// code, same arithmetic in the same order: results are bit-identical).
template <bool QM, class C>
__device__ __forceinline__ void rk4_step_rolled(const C& c, Vec12& y, double h)
{
    const double h2 = 0.5 * h, h3 = h * (1.0 / 3.0), h6 = h * (1.0 / 6.0);
    Vec12 k, st = y, acc = y;
    const double* yv = &y.r[0];
    const double* kv = &k.r[0];
    double* sv = &st.r[0];
    double* av = &acc.r[0];
    double u = rsqrt(dot3(y.r, y.r));
#pragma unroll 1
    for (int j = 0; j < 4; j++) {
        rhs_u<QM>(c, st, u, k);
        // next stage state first, and its 1/|r| started before the
        // accumulator update that does not depend on it
        if (j < 3) {
            const double a = j == 2 ? h : h2;
#pragma unroll
            for (int i = 0; i < 12; i++) sv[i] = fma(a, kv[i], yv[i]);
            u = rsqrt(dot3(st.r, st.r));
        }
        const double w = (j == 0 || j == 3) ? h6 : h3;
        // stage 0: acc = y + h/6 k1 (acc starts as y)
#pragma unroll
        for (int i = 0; i < 12; i++) av[i] = fma(w, kv[i], av[i]);
    }
    y = acc;
}

// Fifth-order Runge-Kutta step, Dormand & Prince (1980) tableau with the
// fifth-order weights (b7 = 0, so six derivative evaluations).  The stage
// derivatives go to shared memory (kst: 6 x 12 planes of `stride` doubles,
// this thread's column) so the registers hold only y and the stage state.
template <bool QM, class C>
__device__ __forceinline__ void rk5_step(const C& c, Vec12& y, double h, double* kst, int stride)
{
    const double a21 = 1.0 / 5.0;
    const double a31 = 3.0 / 40.0, a32 = 9.0 / 40.0;
    const double a41 = 44.0 / 45.0, a42 = -56.0 / 15.0, a43 = 32.0 / 9.0;
    const double a51 = 19372.0 / 6561.0, a52 = -25360.0 / 2187.0, a53 = 64448.0 / 6561.0, a54 = -212.0 / 729.0;
    const double a61 = 9017.0 / 3168.0, a62 = -355.0 / 33.0, a63 = 46732.0 / 5247.0, a64 = 49.0 / 176.0,
                 a65 = -5103.0 / 18656.0;
    const double b1 = 35.0 / 384.0, b3 = 500.0 / 1113.0, b4 = 125.0 / 192.0, b5 = -2187.0 / 6784.0,
                 b6 = 11.0 / 84.0;
    const double A[6][5] = {{0, 0, 0, 0, 0},
                            {a21, 0, 0, 0, 0},
                            {a31, a32, 0, 0, 0},
                            {a41, a42, a43, 0, 0},
                            {a51, a52, a53, a54, 0},
                            {a61, a62, a63, a64, a65}};
    const double B[6] = {b1, 0.0, b3, b4, b5, b6};
    double* yv = &y.r[0];
    Vec12 st, k;
    double* sv = &st.r[0];
    double* kv = &k.r[0];
#pragma unroll
    for (int j = 0; j < 6; j++) {
        if (j == 0) {
            rhs<QM, C>(c, y, k);
        } else {
#pragma unroll
            for (int i = 0; i < 12; i++) {
                double acc = yv[i];
#pragma unroll
                for (int m = 0; m < 5; m++)
                    if (m < j && A[j][m] != 0.0) acc = fma(h * A[j][m], kst[(m * 12 + i) * stride], acc);
                sv[i] = acc;
            }
            rhs<QM, C>(c, st, k);
        }
#pragma unroll
        for (int i = 0; i < 12; i++) kst[(j * 12 + i) * stride] = kv[i];
    }
#pragma unroll
    for (int i = 0; i < 12; i++) {
        double acc = yv[i];
#pragma unroll
        for (int m = 0; m < 6; m++)
            if (B[m] != 0.0) acc = fma(h * B[m], kst[(m * 12 + i) * stride], acc);
        yv[i] = acc;
    }
}

// Tableau of rk5_step scaled by the step: hab[5 j + m] = h a_{j+1, m+1}
// (j = 1..5, m < j) and hab[30 + m] = h b_{m+1}.
__device__ __forceinline__ void rk5_scaled_tableau(double h, double* hab)
{
    const double A[6][5] = {{0, 0, 0, 0, 0},
                            {1.0 / 5.0, 0, 0, 0, 0},
                            {3.0 / 40.0, 9.0 / 40.0, 0, 0, 0},
                            {44.0 / 45.0, -56.0 / 15.0, 32.0 / 9.0, 0, 0},
                            {19372.0 / 6561.0, -25360.0 / 2187.0, 64448.0 / 6561.0, -212.0 / 729.0, 0},
                            {9017.0 / 3168.0, -355.0 / 33.0, 46732.0 / 5247.0, 49.0 / 176.0, -5103.0 / 18656.0}};
    const double B[6] = {35.0 / 384.0, 0.0, 500.0 / 1113.0, 125.0 / 192.0, -2187.0 / 6784.0, 11.0 / 84.0};
#pragma unroll
    for (int j = 0; j < 6; j++)
#pragma unroll
        for (int m = 0; m < 5; m++) hab[5 * j + m] = h * A[j][m];
#pragma unroll
    for (int m = 0; m < 6; m++) hab[30 + m] = h * B[m];
}

// rk5_step with the stage loops not unrolled (one compiled copy of the
// equations of motion); hab from rk5_scaled_tableau.  Same products and
// sums in the same order as rk5_step: bit-identical results.
template <bool QM, class C>
__device__ __forceinline__ void rk5_step_rolled(const C& c, Vec12& y, const double* hab, double* kst, int stride)
{
    double* yv = &y.r[0];
    Vec12 st = y, k;
    double* sv = &st.r[0];
    const double* kv = &k.r[0];
#pragma unroll 1
    for (int j = 0; j < 6; j++) {
        if (j > 0) {
            st = y;
#pragma unroll 1
            for (int m = 0; m < j; m++) {
                const double a = hab[5 * j + m];
#pragma unroll
                for (int i = 0; i < 12; i++) sv[i] = fma(a, kst[(m * 12 + i) * stride], sv[i]);
            }
        }
        rhs<QM, C>(c, st, k);
#pragma unroll
        for (int i = 0; i < 12; i++) kst[(j * 12 + i) * stride] = kv[i];
    }
#pragma unroll 1
    for (int m = 0; m < 6; m++) {
        if (m == 1) continue;                        // b2 = 0
        const double b = hab[30 + m];
#pragma unroll
        for (int i = 0; i < 12; i++) yv[i] = fma(b, kst[(m * 12 + i) * stride], yv[i]);
    }
}

// ------------------------------------------------------ radiation reaction
// Leading-order (2.5PN) radiation-reaction acceleration a_2.5PN of Eq. 6, in
// the gauge family of Iyer & Will (1993), velocity v = p at this order:
//   a = (8/5) eta u^3 [A (n.p) n - B p]
//   A = 3 (1 + gb) p^2 + (23 + 6 ga - 9 gb) u / 3 - 5 gb (n.p)^2
//   B = (2 + ga) p^2 + (2 - ga) u - 3 (1 + ga) (n.p)^2
// ((ga, gb) = (4, 5): the harmonic-gauge force).  With rp = r.p:
//   a = sr r + sp p,  sr = (8/5) eta u^5 A rp,  sp = -(8/5) eta u^3 B.
// The reference values of the dissipative system follow the integral-
// invariant relations (Sec. 3B): dE/dt = (dH/dp).a = (dr/dt).a and, since
// r x a = sp L, d|J|/dt = J.(r x a)/|J| = sp (J.L)/|J|.
struct RRCoef {
    double A0, A1, A2;   // A = A0 p^2 + A1 u + A2 (n.p)^2
    double B0, B1, B2;   // B = B0 p^2 + B1 u + B2 (n.p)^2
};

__host__ __device__ inline RRCoef make_rr_coef(double ga, double gb)
{
    RRCoef g;
    g.A0 = 3.0 * (1.0 + gb);
    g.A1 = (23.0 + 6.0 * ga - 9.0 * gb) / 3.0;
    g.A2 = -5.0 * gb;
    g.B0 = 2.0 + ga;
    g.B1 = 2.0 - ga;
    g.B2 = -3.0 * (1.0 + ga);
    return g;
}

// Eqs. 6-7 with a_2.5PN: dy, and dE/dt, d|J|/dt of the reference values.
// k8eta = (8/5) eta of the orbit.
template <bool QM, class C>
__device__ __forceinline__ void rhs_rr(const C& c, const RRCoef& g, double k8eta, const Vec12& y, double u,
                                       Vec12& dy, double& dE, double& dJ)
{
    rhs_u<QM, C>(c, y, u, dy);
    const double rp = dot3(y.r, y.p);
    const double p2 = dot3(y.p, y.p);
    const double u2 = u * u;
    const double np2 = rp * rp * u2;
    const double A = fma(g.A0, p2, fma(g.A1, u, g.A2 * np2));
    const double B = fma(g.B0, p2, fma(g.B1, u, g.B2 * np2));
    const double ku3 = k8eta * u2 * u;
    const double sr = ku3 * u2 * A * rp;
    const double sp = -ku3 * B;
    double a[3];
#pragma unroll
    for (int i = 0; i < 3; i++) {
        a[i] = fma(sr, y.r[i], sp * y.p[i]);
        dy.p[i] += a[i];
    }
    dE = dot3(dy.r, a);
    const double L0 = fma(y.r[1], y.p[2], -y.r[2] * y.p[1]);
    const double L1 = fma(y.r[2], y.p[0], -y.r[0] * y.p[2]);
    const double L2 = fma(y.r[0], y.p[1], -y.r[1] * y.p[0]);
    const double J0 = L0 + y.s1[0] + y.s2[0];
    const double J1 = L1 + y.s1[1] + y.s2[1];
    const double J2 = L2 + y.s1[2] + y.s2[2];
    const double JL = fma(J0, L0, fma(J1, L1, J2 * L2));
    dJ = sp * JL * rsqrt(fma(J0, J0, fma(J1, J1, J2 * J2)));
}

// RK4 step of rhs_rr (stage loop rolled, as rk4_step_rolled).  The reference
// values ref.E, ref.J advance with the state; the equations of motion do not
// depend on them, so they need no stage values.
template <bool QM, class C>
__device__ __forceinline__ void rk4_step_rr(const C& c, const RRCoef& g, double k8eta, Vec12& y, Ref& ref, double h)
{
    const double h2 = 0.5 * h, h3 = h * (1.0 / 3.0), h6 = h * (1.0 / 6.0);
    Vec12 k, st = y, acc = y;
    const double* yv = &y.r[0];
    const double* kv = &k.r[0];
    double* sv = &st.r[0];
    double* av = &acc.r[0];
    double eA = ref.E, jA = ref.J;
    double u = rsqrt(dot3(y.r, y.r));
#pragma unroll 1
    for (int j = 0; j < 4; j++) {
        double dE, dJ;
        rhs_rr<QM>(c, g, k8eta, st, u, k, dE, dJ);
        if (j < 3) {
            const double a = j == 2 ? h : h2;
#pragma unroll
            for (int i = 0; i < 12; i++) sv[i] = fma(a, kv[i], yv[i]);
            u = rsqrt(dot3(st.r, st.r));
        }
        const double w = (j == 0 || j == 3) ? h6 : h3;
#pragma unroll
        for (int i = 0; i < 12; i++) av[i] = fma(w, kv[i], av[i]);
        eA = fma(w, dE, eA);
        jA = fma(w, dJ, jA);
    }
    y = acc;
    ref.E = eA;
    ref.J = jA;
}

// Fifth-order step of rhs_rr (as rk5_step_rolled); the reference values take
// the fifth-order weights stage by stage.
template <bool QM, class C>
__device__ __forceinline__ void rk5_step_rr(const C& c, const RRCoef& g, double k8eta, Vec12& y, Ref& ref,
                                            const double* hab, double* kst, int stride)
{
    double* yv = &y.r[0];
    Vec12 st = y, k;
    double* sv = &st.r[0];
    const double* kv = &k.r[0];
#pragma unroll 1
    for (int j = 0; j < 6; j++) {
        if (j > 0) {
            st = y;
#pragma unroll 1
            for (int m = 0; m < j; m++) {
                const double a = hab[5 * j + m];
#pragma unroll
                for (int i = 0; i < 12; i++) sv[i] = fma(a, kst[(m * 12 + i) * stride], sv[i]);
            }
        }
        double dE, dJ;
        rhs_rr<QM, C>(c, g, k8eta, st, rsqrt(dot3(st.r, st.r)), k, dE, dJ);
        ref.E = fma(hab[30 + j], dE, ref.E);
        ref.J = fma(hab[30 + j], dJ, ref.J);
#pragma unroll
        for (int i = 0; i < 12; i++) kst[(j * 12 + i) * stride] = kv[i];
    }
#pragma unroll 1
    for (int m = 0; m < 6; m++) {
        if (m == 1) continue;                        // b2 = 0
        const double b = hab[30 + m];
#pragma unroll
        for (int i = 0; i < 12; i++) yv[i] = fma(b, kst[(m * 12 + i) * stride], yv[i]);
    }
}

// ------------------------------------------------------ manifold correction
enum CorrKind : int { CORR_DUAL = 0, CORR_NONE = 1, CORR_VELOCITY = 2, CORR_SPLIT = 3 };

struct NewtonCfg {
    double tol;       // stop when |d alpha| <= tol and |d beta| <= tol (Sec. 3A: 1e-10)
    int max_iter;     // iteration cap
    double det_min;   // relative-determinant guard of the singular scaling
    int apply_small;  // 1: apply a step, then stop if it was within tol; 0: stop before applying it
    int mode;         // CORR_MODE_*: what the correction restores
    double split_min; // conditioning guard of the split scaling (<= 0: not used)
    double cond_switch; // dual scaling's relative determinant below which the better-conditioned
                        // of the dual and split scalings is used (<= 0: dual down to det_min)
};

// Correction modes: spin lengths and dual scaling (Eqs. 10-13); ablations:
// spin lengths only (Eq. 10), or spin lengths and velocity scaling p = a p*
// to E0 (the single-factor correction of Sec. 1, Wu et al. 2007).
enum CorrMode : int { CORR_MODE_DUAL = 1, CORR_MODE_SPINS = 2, CORR_MODE_VELOCITY = 3 };

// Eq. 10, then Eqs. 11-13: p = alpha p*, r = beta r* with (alpha, beta) from
// H(beta r*, alpha p*, S) = E0 and |J(beta r*, alpha p*, S)| = J0 by Newton's
// method from (1, 1).  Returns the number of Newton iterations; *kind is
// CORR_DUAL when the dual scaling was applied; where it was singular (or did
// not converge) CORR_SPLIT when the split scaling of p's tangential and
// radial parts restored both integrals, CORR_VELOCITY when that was singular
// too and E was restored by scaling p alone, and CORR_NONE when nothing
// converged.
//
// With u = 1/beta, every term of H at the scaled point is a monomial in
// (alpha, u):  H(alpha, u) = alpha^2 (A2 + alpha^2 (A4 + alpha^2 A6))
//   + u (B0 + alpha^2 (B2 + alpha^2 B4)) + u^2 (C0 + alpha^2 C2 + alpha E1) + u^3 D0
// whose coefficients are evaluated once at (r*, p*, S); and
// |J|^2 = k^2 L*.L* + 2 k L*.S + S.S with k = alpha beta, S = S1 + S2.
template <bool QM, class C>
__device__ __forceinline__ int correct(const C& c, Vec12& y, const Ref& ref,
                                       const NewtonCfg& nc, int* kind)
{
    // Eq. 10: spin lengths
    {
        const double l1 = dot3(y.s1, y.s1), l2 = dot3(y.s2, y.s2);
        if (ref.S1 > 0.0 && l1 > 0.0) {
            const double f = ref.S1 * rsqrt(l1);
            y.s1[0] *= f; y.s1[1] *= f; y.s1[2] *= f;
        }
        if (ref.S2 > 0.0 && l2 > 0.0) {
            const double f = ref.S2 * rsqrt(l2);
            y.s2[0] *= f; y.s2[1] *= f; y.s2[2] *= f;
        }
    }
    if (nc.mode == CORR_MODE_SPINS) {
        *kind = CORR_NONE;
        return 0;
    }
    // monomial coefficients at (r*, p*, S)
    const double R = rsqrt(dot3(y.r, y.r));
    const double P2 = dot3(y.p, y.p);
    const double NP = dot3(y.r, y.p) * R;
    const double NP2 = NP * NP;
    const double L0 = fma(y.r[1], y.p[2], -y.r[2] * y.p[1]);
    const double L1 = fma(y.r[2], y.p[0], -y.r[0] * y.p[2]);
    const double L2 = fma(y.r[0], y.p[1], -y.r[1] * y.p[0]);
    const double Sx = y.s1[0] + y.s2[0], Sy = y.s1[1] + y.s2[1], Sz = y.s1[2] + y.s2[2];
    const double LL = fma(L0, L0, fma(L1, L1, L2 * L2));
    const double LJ = fma(L0, Sx, fma(L1, Sy, L2 * Sz));
    const double SSq = fma(Sx, Sx, fma(Sy, Sy, Sz * Sz));
    const double LSe = c[K_G1] * fma(L0, y.s1[0], fma(L1, y.s1[1], L2 * y.s1[2]))
                     + c[K_G2] * fma(L0, y.s2[0], fma(L1, y.s2[1], L2 * y.s2[2]));
    const double a1 = dot3(y.s1, y.r) * R, a2 = dot3(y.s2, y.r) * R;
    const double R2 = R * R, R3 = R2 * R;
    const double A2 = 0.5 * P2;
    const double A4 = c[K_A1] * P2 * P2;
    const double A6 = c[K_A2] * P2 * P2 * P2;
    const double B0 = -R;
    const double B2 = R * fma(c[K_B1], P2, c[K_B2] * NP2);
    const double B4 = R * fma(P2, fma(c[K_C1], P2, c[K_C2] * NP2), c[K_C3] * NP2 * NP2);
    const double C0 = c[K_H1] * R2;
    const double C2 = R2 * fma(c[K_D1], P2, c[K_D2] * NP2);
    const double E1 = R3 * LSe;
    double Dq = fma(c[K_IETA], fma(3.0 * a1, a2, -dot3(y.s1, y.s2)), c[K_E1]);
    if (QM)
        Dq += c[K_Q1] * fma(3.0 * a1, a1, -dot3(y.s1, y.s1)) + c[K_Q2] * fma(3.0 * a2, a2, -dot3(y.s2, y.s2));
    const double D0 = R3 * Dq;
    const double A4x2 = 2.0 * A4, A6x3 = 3.0 * A6, B4x2 = 2.0 * B4, D0x3 = 3.0 * D0, LJx2 = 2.0 * LJ;

    double al = 1.0, be = 1.0;
    int it = 0;
    bool conv = false, stop = false;
    // split scaling state (below): factors of p's tangential and radial parts,
    // iterations done, converged
    double sa = 1.0, sg = 1.0;
    int ks = 0;
    bool sok = false;
    // First iteration at alpha = beta = 1 (u = 1, k = 1): the monomial sums
    // need no powers and no reciprocal; there dF2/dalpha = dF2/dbeta = dJ and
    // dH/dbeta = -dH/du, so det = dJ (Ha + Hu).
    if (nc.mode != CORR_MODE_DUAL) {
        stop = true;   // velocity-scaling mode: no dual scaling
    } else {
        ++it;
        const double Pb = B0 + B2 + B4, Pc = C0 + C2 + E1;
        const double H = (A2 + A4 + A6) + Pb + Pc + D0;
        const double Ha = fma(2.0, (A2 + A4x2 + A6x3) + (B2 + B4x2) + C2, E1);
        const double Hu = fma(2.0, Pc, Pb + D0x3);
        const double Jn2 = LL + LJx2 + SSq;
        const double rJ = rsqrt(Jn2);
        const double dJ = (LL + LJ) * rJ;
        const double F1 = H - ref.E;
        const double F2 = fma(Jn2, rJ, -ref.J);
        const double p1 = Ha * dJ, p2 = -Hu * dJ;
        const double det = p1 - p2;
        // In the dual scaling's ill-conditioned band the split scaling below is
        // used instead where it is better conditioned: its relative
        // conditioning at (1, 1) is |H_g| / (|H_a| + |H_g|), with
        // H_a = p_t.dH/dp and H_g = p_r.dH/dp from the split polynomial's
        // derivatives at q = P2, w = NP2 (P2 = 2 A2 exactly).
        bool prefer_split = false;
        if (nc.cond_switch > 0.0 && nc.split_min > 0.0 && fabs(det) <= nc.cond_switch * (fabs(p1) + fabs(p2))) {
            const double P2s = 2.0 * A2, Rr = -B0;
            const double Hq1 = fma(P2s, fma(3.0 * c[K_A2], P2s, 2.0 * c[K_A1]), fma(Rr * Rr, c[K_D1], 0.5))
                             + Rr * fma(2.0 * c[K_C1], P2s, fma(c[K_C2], NP2, c[K_B1]));
            const double Hw1 = Rr * fma(c[K_C2], P2s, fma(2.0 * c[K_C3], NP2, c[K_B2])) + Rr * Rr * c[K_D2];
            const double As = fma(2.0 * (P2s - NP2), Hq1, E1);
            const double Bs = 2.0 * NP2 * (Hq1 + Hw1);
            prefer_split = fabs(Bs) * (fabs(p1) + fabs(p2)) > fabs(det) * (fabs(As) + fabs(Bs)) &&
                           fabs(Bs) > nc.split_min * (fabs(As) + fabs(Bs)) &&
                           dJ * dJ > (nc.split_min * nc.split_min) * LL;       // |dJ| > split_min |L*|
            if (prefer_split) {
                // the split scaling's first Newton step at (1, 1): H, F and the
                // |J| derivative are the dual scaling's at its own (1, 1)
                ks = 1;
                const double rd = __drcp_rn(dJ * Bs);
                const double da = F2 * Bs * rd;
                const double dg = fma(F1, dJ, -As * F2) * rd;
                const bool small = fabs(da) <= nc.tol && fabs(dg) <= nc.tol;
                if (!(small && !nc.apply_small)) {
                    sa -= da;
                    sg -= dg;
                }
                sok = small;
            }
        }
        if (prefer_split) {
            it = 0;
            stop = true;   // straight to the split scaling
        } else if (fabs(det) > nc.det_min * (fabs(p1) + fabs(p2))) {
            const double rd = __drcp_rn(det);
            const double da = fma(F1, dJ, Hu * F2) * rd;
            const double db = fma(Ha, F2, -dJ * F1) * rd;
            const bool small = fabs(da) <= nc.tol && fabs(db) <= nc.tol;
            if (small && !nc.apply_small) {
                conv = true;
            } else {
                al -= da;
                be -= db;
                if (small) conv = true;
                else if (!(fabs(al) < 1e300) || !(fabs(be) < 1e300)) stop = true;   // diverged
            }
        } else {
            stop = true;   // singular: straight to velocity scaling
        }
    }
    while (!conv && !stop && it < nc.max_iter) {
        ++it;
        const double u = __drcp_rn(be);
        const double a2s = al * al;
        const double Pa = fma(a2s, fma(a2s, A6, A4), A2);
        const double Pb = fma(a2s, fma(a2s, B4, B2), B0);
        const double Pc = fma(a2s, C2, fma(al, E1, C0));
        const double H = fma(a2s, Pa, u * fma(u, fma(u, D0, Pc), Pb));
        const double Ha = fma(2.0 * al, fma(a2s, fma(a2s, A6x3, A4x2), A2)
                                        + u * fma(u, C2, fma(a2s, B4x2, B2)), u * u * E1);
        const double Hu = fma(u, fma(u, D0x3, 2.0 * Pc), Pb);
        const double Hb = -(u * u) * Hu;
        const double k = al * be;
        const double Jn2 = fma(k, fma(k, LL, LJx2), SSq);
        const double rJ = rsqrt(Jn2);
        const double dJ = fma(k, LL, LJ) * rJ;
        const double Ja = be * dJ, Jb = al * dJ;
        const double F1 = H - ref.E;
        const double F2 = fma(Jn2, rJ, -ref.J);
        const double p1 = Ha * Jb, p2 = Hb * Ja;
        const double det = p1 - p2;
        if (!(fabs(det) > nc.det_min * (fabs(p1) + fabs(p2)))) break;   // singular (or NaN)
        const double rd = __drcp_rn(det);
        const double da = fma(F1, Jb, -Hb * F2) * rd;
        const double db = fma(Ha, F2, -Ja * F1) * rd;
        const bool small = fabs(da) <= nc.tol && fabs(db) <= nc.tol;
        if (small && !nc.apply_small) { conv = true; break; }
        al -= da;
        be -= db;
        if (small) { conv = true; break; }
        if (!(fabs(al) < 1e300) || !(fabs(be) < 1e300)) break;
    }
    if (conv) {
        y.r[0] *= be; y.r[1] *= be; y.r[2] *= be;
        y.p[0] *= al; y.p[1] *= al; y.p[2] *= al;
        *kind = CORR_DUAL;
        return it;
    }
    // Singular (or non-converged) dual scaling -- for a Kepler ellipse at
    // r = a, where |p_r| / |p| = e: restore both integrals by the split
    // scaling p = a p_t + g p_r of p*'s tangential and radial parts, r = r*.
    // There L = a L*, and with q = p^2 = a^2 Pt2 + g^2 NP2, w = (n.p)^2 =
    // g^2 NP2 every term of H is a polynomial in (q, w, a):
    //   H = q (1/2 + q (A1 + q A2)) + R (q (B1 + C1 q + C2 w) + w (B2 + C3 w))
    //       + R^2 (D1 q + D2 w) + a E1 + (B0 + C0 + D0),
    // and |J|^2 = a^2 LL + 2 a LJ + SSq.  Newton on (a, g) from (1, 1); the
    // Jacobian [[H_a, H_g], [J_a, 0]] is triangular.  It is used only where
    // |H_g| > split_min (|H_a| + |H_g|) and |J_a| > split_min |L*| (compared
    // as squares): near a
    // circular orbit E and |J| cannot be moved independently, and it is as
    // ill-conditioned as the dual scaling.  State quantities are recomputed
    // from (r*, p*), which are still unchanged here.
    if (nc.mode == CORR_MODE_DUAL && nc.split_min > 0.0) {
        const double Rr = -B0;
        const double NPs = dot3(y.r, y.p) * Rr;
        const double NP2s = NPs * NPs;
        const double Pt2 = dot3(y.p, y.p) - NP2s;
        const double RR2 = Rr * Rr;
        const double hq0 = fma(Rr, c[K_B1], fma(RR2, c[K_D1], 0.5));    // dH/dq at q = w = 0
        const double hw0 = fma(Rr, c[K_B2], RR2 * c[K_D2]);             // dH/dw at q = w = 0
        const double Hc = (B0 + C0) + D0;
        const double smin2LL = (nc.split_min * nc.split_min) * LL;     // (split_min |L*|)^2
        while (!sok && ks < nc.max_iter) {
            ++ks;
            const double w = sg * sg * NP2s;
            const double q = fma(sa * sa, Pt2, w);
            const double H = fma(q, fma(q, fma(q, c[K_A2], c[K_A1]), 0.5),
                                 fma(Rr, fma(q, fma(c[K_C1], q, fma(c[K_C2], w, c[K_B1])),
                                             w * fma(c[K_C3], w, c[K_B2])),
                                     fma(RR2, fma(c[K_D1], q, c[K_D2] * w), fma(sa, E1, Hc))));
            const double Hq = fma(q, fma(3.0 * c[K_A2], q, 2.0 * c[K_A1]), hq0)
                            + Rr * fma(2.0 * c[K_C1], q, c[K_C2] * w);
            const double Hw = fma(Rr, fma(c[K_C2], q, 2.0 * c[K_C3] * w), hw0);
            const double Ha = fma(2.0 * sa * Pt2, Hq, E1);
            const double Hg = 2.0 * sg * NP2s * (Hq + Hw);
            const double Jn2 = fma(sa, fma(sa, LL, LJx2), SSq);
            const double rJ = rsqrt(Jn2);
            const double Ja = fma(sa, LL, LJ) * rJ;
            if (!(fabs(Hg) > nc.split_min * (fabs(Ha) + fabs(Hg))) || !(Ja * Ja > smin2LL))
                break;   // ill-conditioned (or NaN)
            const double F1 = H - ref.E;
            const double F2 = fma(Jn2, rJ, -ref.J);
            // triangular Jacobian [[Ha, Hg], [Ja, 0]]: da = F2 / Ja,
            // dg = (F1 - Ha da) / Hg, with one reciprocal of Ja Hg
            const double rd = __drcp_rn(Ja * Hg);
            const double da = F2 * Hg * rd;
            const double dg = fma(F1, Ja, -Ha * F2) * rd;
            const bool small = fabs(da) <= nc.tol && fabs(dg) <= nc.tol;
            if (small && !nc.apply_small) { sok = true; break; }
            sa -= da;
            sg -= dg;
            if (small) { sok = true; break; }
            if (!(fabs(sa) < 1e300) || !(fabs(sg) < 1e300)) break;
        }
        if (sok) {
            // p = a (p* - p_r) + g p_r = a p* + (g - a) p_r, p_r = (n.p*) n = (NPs Rr) r*
            const double f = (sg - sa) * (NPs * Rr);
#pragma unroll
            for (int i = 0; i < 3; i++) y.p[i] = fma(sa, y.p[i], f * y.r[i]);
            *kind = CORR_SPLIT;
            return it + ks;
        }
    }
    // Both singular (or non-converged): restore E alone by velocity scaling,
    // p = a p*, H(r*, a p*, S) = E0 (Newton in a from 1), i.e. the monomial
    // form at 1/beta = 1.  |J| is left to the next step.
    double a = 1.0;
    int k = 0;
    bool ok = false;
    const double Bsum = B0 + C0 + D0;
    while (k < nc.max_iter) {
        ++k;
        const double a2s = a * a;
        const double H = fma(a2s, fma(a2s, fma(a2s, A6, A4), A2) + fma(a2s, B4, B2) + C2, fma(a, E1, Bsum));
        const double Ha = fma(2.0 * a, fma(a2s, fma(a2s, A6x3, A4x2), A2) + fma(a2s, B4x2, B2) + C2, E1);
        const double da = (H - ref.E) / Ha;
        if (!(fabs(da) <= 1.7976931348623157e308)) break;
        if (!nc.apply_small && fabs(da) <= nc.tol) { ok = true; break; }
        a -= da;
        if (fabs(da) <= nc.tol) { ok = true; break; }
    }
    if (ok) {
        y.p[0] *= a; y.p[1] *= a; y.p[2] *= a;
    }
    *kind = ok ? CORR_VELOCITY : CORR_NONE;
    return it + ks + k;
}

}  // namespace pnscan
