// pn_waveform.cuh -- gravitational-wave polarisations of the scan's orbits
// (arXiv:1802.00147, Eq. 14, Sec. 4).
#pragma once
#include <cuda_runtime.h>

#include "pn_kernels.cuh"

namespace pnscan {

// h_plus / h_cross of every orbit's main trajectory at its current state,
// observer at distance R along N = P x Q.  hp, hc: device arrays of S.n
// doubles, either may be null.
cudaError_t launch_waveform(DevState S, RunCfg rc, double R, const double P[3], const double Q[3], double* hp,
                            double* hc, cudaStream_t st);

}  // namespace pnscan
