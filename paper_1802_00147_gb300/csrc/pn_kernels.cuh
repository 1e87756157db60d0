// pn_kernels.cuh -- device state layout and kernel launch interface of the
// scan library (internal to the library; the public boundary is
// include/pnscan.h).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "pn_device.cuh"

namespace pnscan {

enum OrbitStatus : int32_t {
    ORBIT_RUNNING = 0,
    ORBIT_DONE = 1,
    ORBIT_MERGED = 2,
    ORBIT_ESCAPED = 3,
    ORBIT_FLI_SATURATED = 4,
    ORBIT_NONFINITE = 5,
};

// Structure-of-arrays orbit state in HBM.  Plane k of an [m][n] array starts
// at base + k * n; a warp reads 32 consecutive orbits of one plane at a time.
struct DevState {
    int64_t n;             // orbits
    int64_t ld;            // plane stride (n rounded up to a multiple of 32)
    double* y;             // [12][n] main trajectory (r, p, S1, S2)
    double* ys;            // [12][n] shadow trajectory
    double* ref;           // [8][n]  E0, J0, |S1|0, |S2|0 of main, then of shadow (with
                           //         radiation reaction E and J are the values at t)
    double* fli_acc;       // [n]     sum of log10(d_k / d0) over renormalisations
    double* t;             // [n]     time reached
    int32_t* nstep;        // [n]     steps taken since the initial state
    int32_t* status;       // [n]     OrbitStatus
    int32_t* newton_iters; // [n]     Newton iterations, both trajectories
    int32_t* n_skip;       // [n]     corrections without the dual scaling
    int32_t* last_kind;    // [n]     CorrKind of the main trajectory's last step
    double* beta;          // [n]     m1/m2
    double* kappa1;        // [n]
    double* kappa2;        // [n]
    double* out;           // [5][n]  E, |J|, |S1|, |S2|, FLI (written by finalize)
    int32_t* order;        // [n]     compacting schedule: running orbits, densely
    int32_t* order_next;   // [n]     the next epoch's list
};

struct RunCfg {
    Flags flags;
    NewtonCfg newton;
    int correct;           // apply the manifold correction each step
    int rk_order;          // 4: classical RK4; 5: Dormand-Prince fifth order
    int rr;                // 2.5PN radiation reaction
    RRCoef rrc;            // its gauge constants
    double h;              // step size
    double d0;             // FLI separation
    int renorm;            // renormalise every `renorm` steps (<= 0: never)
    double fli_cap;        // stop at FLI >= cap (<= 0: never)
    double rmerge2;        // stop at |r|^2 < rmerge2 (<= 0: never)
    double rescape2;       // stop at |r|^2 > rescape2 (<= 0: never)
    int32_t nstep_base;    // nstep of every running orbit when the run (or epoch) started
    int32_t nsteps;        // steps in this run (or epoch)
    int32_t final_step;    // nstep at which an orbit is DONE (end of the whole run)
    int first_epoch;       // 1: orbits left DONE by an earlier run may continue
    unsigned long long wait_limit_ns;  // bound on a queue task's wait for its predecessor
    int stall_group;       // test hook: this group never publishes chunk 0 (-1: off)
};

// Work-queue state of the persistent integrator (device memory, 256-byte
// aligned): next task counter, error flag, then one progress counter per
// 32-orbit group.
struct QueueState {
    unsigned long long* next;   // [1]
    int* error;                 // [1] nonzero: a bounded wait gave up
    int* group_done;            // [groups] chunks finished per group
    int* count;                 // [2] compacting schedule: orbits in order / order_next
};

// Dynamic shared memory of the integrators for the RK5 stage derivatives
// (6 x 12 doubles per thread).
inline size_t rk5_smem_bytes(int block) { return (size_t)6 * 12 * block * sizeof(double); }

struct Summary {                // scan-level reduction (device layout)
    unsigned long long n_chaotic;
    unsigned long long status_count[8];
    unsigned long long newton_iters;
    unsigned long long n_skip;
    unsigned long long steps;
    unsigned long long max_dE_bits;   // non-negative doubles as ordered integers
    unsigned long long max_dJ_bits;       // over DONE orbits whose last step was dual-scaled
    unsigned long long max_dJ_all_bits;   // over all DONE orbits
    unsigned long long n_final_fallback;  // DONE orbits whose last step was not dual-scaled
    unsigned long long max_dS_bits;
    unsigned long long fli_max_bits;
    double fli_sum;
};

// ---- launchers (return cudaError_t of the launch) ----
cudaError_t launch_setup_cells(const double* cells_aos, int64_t n, DevState S, int beta_from_cells,
                               cudaStream_t st);
cudaError_t launch_load_states(const double* states_aos, int64_t n, DevState S, cudaStream_t st);
cudaError_t launch_init(DevState S, RunCfg rc, cudaStream_t st);
// One orbit per thread.
cudaError_t launch_integrate_static(DevState S, RunCfg rc, int block, cudaStream_t st);
// Two lanes per orbit (main / shadow trajectory), one pass over the batch.
cudaError_t launch_integrate_pair(DevState S, RunCfg rc, int block, cudaStream_t st);
// minb: variant of the queue kernel: 2 -- two resident 128-thread blocks per
// SM, per-orbit constants in registers (up to 255 per thread); 3 -- three,
// constants in shared memory (168 registers); 4 -- as 2 with the RK stage
// and trajectory loops rolled (the default; with radiation reaction the
// only variant, whatever minb)
int queue_blocks_per_sm(int block, bool qm, int minb, int rk_order, bool rr);
cudaError_t launch_integrate_queue(DevState S, RunCfg rc, QueueState q, int block, int grid,
                                   int chunk, int minb, int use_order, cudaStream_t st);
// Compacting schedule: order_next <- running orbits of order (or of all
// orbits when from_all), count[1] <- their number; then swap is up to the caller.
cudaError_t launch_compact(DevState S, QueueState q, int from_all, int first_epoch, cudaStream_t st);
cudaError_t launch_finalize(DevState S, RunCfg rc, cudaStream_t st);
cudaError_t launch_reduce(DevState S, double fli_thresh, Summary* out, cudaStream_t st);
cudaError_t launch_gather(DevState S, double* states_aos, double* shadow_aos, double* integ_aos,
                          cudaStream_t st);
cudaError_t launch_fp64_probe(double* out, int blocks, int threads, int iters, cudaStream_t st);

}  // namespace pnscan
