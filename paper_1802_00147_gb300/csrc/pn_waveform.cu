// pn_waveform.cu -- gravitational-wave polarisations (Eq. 14) of the scan's
// orbits from the field of the mass quadrupole moment (Sec. 4, Fig. 10).
//
// For the relative orbit at distance R (in M) along N, with the coordinate
// velocity v = dr/dt = dH/dp (Eq. 6), n = r/|r| and eta = m1 m2:
//     h_ij    = (4 eta / R) (v_i v_j - n_i n_j / |r|)
//     h_plus  = (P_i P_j - Q_i Q_j) h_ij / 2 = (2 eta / R) [(v.P)^2 - (v.Q)^2 - ((n.P)^2 - (n.Q)^2) / |r|]
//     h_cross = (P_i Q_j + Q_i P_j) h_ij / 2 = (4 eta / R) [(v.P)(v.Q) - (n.P)(n.Q) / |r|]
// P, Q: the radiation frame's unit vectors orthogonal to N.
#include <cuda_runtime.h>

#include "pn_device.cuh"
#include "pn_waveform.cuh"

namespace pnscan {

struct Frame {
    double P[3], Q[3];
};

template <bool QM>
__global__ void k_waveform(DevState S, RunCfg rc, double R, Frame f, double* hp, double* hc)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= S.n) return;
    const double beta = S.beta[i];
    const Coef c = make_coef(beta, S.kappa1[i], S.kappa2[i], rc.flags);
    Vec12 y, dy;
    double* yv = &y.r[0];
#pragma unroll
    for (int k = 0; k < 12; k++) yv[k] = S.y[k * S.ld + i];
    rhs<QM, Coef>(c, y, dy);
    const double eta = beta / ((1.0 + beta) * (1.0 + beta));
    const double u = rsqrt(dot3(y.r, y.r));
    const double vP = dot3(dy.r, f.P), vQ = dot3(dy.r, f.Q);
    const double nP = dot3(y.r, f.P) * u, nQ = dot3(y.r, f.Q) * u;
    const double k = 4.0 * eta / R;
    if (hp) hp[i] = 0.5 * k * fma(vP, vP, -vQ * vQ) - 0.5 * k * fma(nP, nP, -nQ * nQ) * u;
    if (hc) hc[i] = k * fma(vP, vQ, -nP * nQ * u);
}

cudaError_t launch_waveform(DevState S, RunCfg rc, double R, const double P[3], const double Q[3], double* hp,
                            double* hc, cudaStream_t st)
{
    if (S.n == 0 || (!hp && !hc)) return cudaSuccess;
    Frame f;
    for (int k = 0; k < 3; k++) {
        f.P[k] = P[k];
        f.Q[k] = Q[k];
    }
    const unsigned grid = (unsigned)((S.n + 127) / 128);
    if (rc.flags.use_qm) k_waveform<true><<<grid, 128, 0, st>>>(S, rc, R, f, hp, hc);
    else k_waveform<false><<<grid, 128, 0, st>>>(S, rc, R, f, hp, hc);
    return cudaGetLastError();
}

}  // namespace pnscan
