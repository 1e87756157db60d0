// pn_kernels.cu -- kernels of the batched manifold-corrected PN scan
// (arXiv:1802.00147, Secs. 2-3).  One orbit per thread (a lane pair per
// orbit in the paired kernel); the state of both trajectories lives in
// registers for a whole run (or a whole chunk of the persistent work-queue
// kernel) and HBM is touched only at entry and exit.
#include <cmath>

#include "pn_kernels.cuh"

namespace pnscan {

// --------------------------------------------------------------- helpers
__device__ __forceinline__ bool finite12(const Vec12& a)
{
    const double* v = &a.r[0];
    int bad = 0;
#pragma unroll
    for (int i = 0; i < 12; i++) bad |= ((__double2hiint(v[i]) & 0x7ff00000) == 0x7ff00000);
    return !bad;
}

template <bool CG>
__device__ __forceinline__ double ld(const double* p)
{
    if (CG) return __ldcg(p);
    return *p;
}

template <bool CG>
__device__ __forceinline__ int32_t ldi(const int32_t* p)
{
    if (CG) return __ldcg(p);
    return *p;
}

template <bool CG>
__device__ __forceinline__ void load12(const double* base, int64_t n, int64_t i, Vec12& v)
{
    double* d = &v.r[0];
#pragma unroll
    for (int k = 0; k < 12; k++) d[k] = ld<CG>(base + k * n + i);
}

__device__ __forceinline__ void store12(double* base, int64_t n, int64_t i, const Vec12& v)
{
    const double* d = &v.r[0];
#pragma unroll
    for (int k = 0; k < 12; k++) base[k * n + i] = d[k];
}

// Everything one orbit carries between kernel invocations.
struct Orbit {
    Vec12 y, ys;
    Ref ref, refs;
    double acc, t;
    int32_t nstep, status, iters, skips, last_kind;
};

template <bool CG>
__device__ __forceinline__ void load_orbit(const DevState& S, int64_t i, Orbit& o)
{
    const int64_t n = S.ld;
    load12<CG>(S.y, n, i, o.y);
    load12<CG>(S.ys, n, i, o.ys);
    o.ref.E = ld<CG>(S.ref + 0 * n + i);
    o.ref.J = ld<CG>(S.ref + 1 * n + i);
    o.ref.S1 = ld<CG>(S.ref + 2 * n + i);
    o.ref.S2 = ld<CG>(S.ref + 3 * n + i);
    o.refs.E = ld<CG>(S.ref + 4 * n + i);
    o.refs.J = ld<CG>(S.ref + 5 * n + i);
    o.refs.S1 = ld<CG>(S.ref + 6 * n + i);
    o.refs.S2 = ld<CG>(S.ref + 7 * n + i);
    o.acc = ld<CG>(S.fli_acc + i);
    o.t = ld<CG>(S.t + i);
    o.nstep = ldi<CG>(S.nstep + i);
    o.iters = ldi<CG>(S.newton_iters + i);
    o.skips = ldi<CG>(S.n_skip + i);
    o.last_kind = ldi<CG>(S.last_kind + i);
}

__device__ __forceinline__ void store_orbit(const DevState& S, int64_t i, const Orbit& o)
{
    const int64_t n = S.ld;
    store12(S.y, n, i, o.y);
    store12(S.ys, n, i, o.ys);
    S.ref[4 * n + i] = o.refs.E;
    S.ref[5 * n + i] = o.refs.J;
    S.ref[6 * n + i] = o.refs.S1;
    S.ref[7 * n + i] = o.refs.S2;
    S.fli_acc[i] = o.acc;
    S.t[i] = o.t;
    S.nstep[i] = o.nstep;
    S.status[i] = o.status;
    S.newton_iters[i] = o.iters;
    S.n_skip[i] = o.skips;
    S.last_kind[i] = o.last_kind;
}

template <bool CG>
__device__ __forceinline__ Coef load_coef(const DevState& S, int64_t i, const Flags& f)
{
    return make_coef(ld<CG>(S.beta + i), ld<CG>(S.kappa1 + i), ld<CG>(S.kappa2 + i), f);
}

// Advance one orbit (both trajectories) until nstep == step_end or it stops.
// One step: RK4 and manifold correction of the main trajectory, the same for
// the shadow, termination tests, and every `renorm` steps the FLI
// renormalisation (acc += log10(d/d0), shadow pulled back to distance d0 and
// given its own reference integrals).
//
// ROLLED: the two trajectories and the RK stages run in loops that are not
// unrolled -- one compiled copy of the equations of motion and of the
// correction instead of eight (RK4) or twelve (RK5) and two; the trajectories
// are swapped in registers between the passes.  Same operations in the same
// order.  hab: the step-scaled RK5 tableau (RK5 only).
//
// RR: the steps include the 2.5PN radiation reaction and advance the
// reference E and |J| of each trajectory with it (rolled form only); k8eta =
// (8/5) eta of the orbit.
template <class T>
__device__ __forceinline__ void swap_regs(T& a, T& b)
{
    const T t = a;
    a = b;
    b = t;
}

template <bool QM, int RK, class C, bool ROLLED = false, bool RR = false>
__device__ __forceinline__ void advance(const RunCfg& rc, const C& c, Orbit& o, int32_t step_end,
                                        const double* hab = nullptr, double k8eta = 0.0)
{
    static_assert(!RR || ROLLED, "radiation reaction runs in the rolled form");
    extern __shared__ double kst_dyn[];      // RK5 stage derivatives (rk_order 5 only)
    double* kst = kst_dyn + threadIdx.x;
    const int kstride = (int)blockDim.x;
    const double t0 = o.t;
    const int32_t n0 = o.nstep;
    while (o.nstep < step_end) {
        if (ROLLED) {
#pragma unroll 1
            for (int tr = 0; tr < 2; tr++) {
                if (RR) {
                    if (RK == 5) rk5_step_rr<QM, C>(c, rc.rrc, k8eta, o.y, o.ref, hab, kst, kstride);
                    else rk4_step_rr<QM, C>(c, rc.rrc, k8eta, o.y, o.ref, rc.h);
                } else if (RK == 5) {
                    rk5_step_rolled<QM, C>(c, o.y, hab, kst, kstride);
                } else {
                    rk4_step_rolled<QM, C>(c, o.y, rc.h);
                }
                if (rc.correct) {
                    int kind;
                    o.iters += correct<QM, C>(c, o.y, o.ref, rc.newton, &kind);
                    o.skips += kind != CORR_DUAL;
                    if (tr == 0) o.last_kind = kind;
                }
                swap_regs(o.y, o.ys);
                swap_regs(o.ref, o.refs);
            }
        } else {
        if (RK == 5) rk5_step<QM, C>(c, o.y, rc.h, kst, kstride);
        else rk4_step<QM, C>(c, o.y, rc.h);
        if (rc.correct) {
            int kind;
            o.iters += correct<QM, C>(c, o.y, o.ref, rc.newton, &kind);
            o.skips += kind != CORR_DUAL;
            o.last_kind = kind;
        }
        if (RK == 5) rk5_step<QM, C>(c, o.ys, rc.h, kst, kstride);
        else rk4_step<QM, C>(c, o.ys, rc.h);
        if (rc.correct) {
            int kind;
            o.iters += correct<QM, C>(c, o.ys, o.refs, rc.newton, &kind);
            o.skips += kind != CORR_DUAL;
        }
        }
        o.nstep++;
        if (!finite12(o.y) || !finite12(o.ys)) { o.status = ORBIT_NONFINITE; break; }
        const double rr2 = dot3(o.y.r, o.y.r);
        if (rc.rmerge2 > 0.0 && rr2 < rc.rmerge2) { o.status = ORBIT_MERGED; break; }
        if (rc.rescape2 > 0.0 && rr2 > rc.rescape2) { o.status = ORBIT_ESCAPED; break; }
        if (rc.renorm > 0 && (o.nstep % rc.renorm) == 0) {
            double dv[12];
            const double* a = &o.y.r[0];
            double* b = &o.ys.r[0];
            double d2 = 0.0;
#pragma unroll
            for (int k = 0; k < 12; k++) {
                dv[k] = b[k] - a[k];
                d2 = fma(dv[k], dv[k], d2);
            }
            const double d = sqrt(d2);
            o.acc += log10(d / rc.d0);
            const double f = rc.d0 / d;
#pragma unroll
            for (int k = 0; k < 12; k++) b[k] = fma(f, dv[k], a[k]);
            o.refs = integrals<QM, C>(c, o.ys);
            if (rc.fli_cap > 0.0 && o.acc >= rc.fli_cap) { o.status = ORBIT_FLI_SATURATED; break; }
        }
    }
    o.t = t0 + (double)(o.nstep - n0) * rc.h;
}

// ------------------------------------------------------------------ set-up
// Initial conditions of a scan cell (x0, pfac, theta1, phi1, theta2, phi2,
// beta, chi1, chi2): r = (x0, 0, 0), p = (0, pfac / sqrt(x0), 0),
// S_i = chi_i m_i^2 (sin th_i cos ph_i, sin th_i sin ph_i, cos th_i).
__global__ void k_setup_cells(const double* __restrict__ cells, int64_t n, DevState S, int beta_from_cells)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double* c = cells + 9 * i;
    const double x0 = c[0], beta = c[6];
    if (beta_from_cells) S.beta[i] = beta;
    const double m1 = beta / (1.0 + beta), m2 = 1.0 / (1.0 + beta);
    const double s1 = c[7] * m1 * m1, s2 = c[8] * m2 * m2;
    double st1, ct1, sp1, cp1, st2, ct2, sp2, cp2;
    sincos(c[2], &st1, &ct1);
    sincos(c[3], &sp1, &cp1);
    sincos(c[4], &st2, &ct2);
    sincos(c[5], &sp2, &cp2);
    Vec12 y;
    y.r[0] = x0; y.r[1] = 0.0; y.r[2] = 0.0;
    y.p[0] = 0.0; y.p[1] = c[1] / sqrt(x0); y.p[2] = 0.0;
    y.s1[0] = s1 * st1 * cp1; y.s1[1] = s1 * st1 * sp1; y.s1[2] = s1 * ct1;
    y.s2[0] = s2 * st2 * cp2; y.s2[1] = s2 * st2 * sp2; y.s2[2] = s2 * ct2;
    store12(S.y, S.ld, i, y);
}

__global__ void k_load_states(const double* __restrict__ states, int64_t n, DevState S)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    Vec12 y;
    double* d = &y.r[0];
#pragma unroll
    for (int k = 0; k < 12; k++) d[k] = states[12 * i + k];
    store12(S.y, S.ld, i, y);
}

// Reference integrals (E0, J0, |S_i|0) of both trajectories; the shadow
// starts d0 away along x.
template <bool QM>
__global__ void k_init(DevState S, RunCfg rc)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= S.n) return;
    const Coef c = load_coef<false>(S, i, rc.flags);
    Vec12 y, ys;
    load12<false>(S.y, S.ld, i, y);
    ys = y;
    ys.r[0] = ys.r[0] + rc.d0;
    const Ref a = integrals<QM, Coef>(c, y), b = integrals<QM, Coef>(c, ys);
    store12(S.ys, S.ld, i, ys);
    const int64_t n = S.ld;
    S.ref[0 * n + i] = a.E; S.ref[1 * n + i] = a.J; S.ref[2 * n + i] = a.S1; S.ref[3 * n + i] = a.S2;
    S.ref[4 * n + i] = b.E; S.ref[5 * n + i] = b.J; S.ref[6 * n + i] = b.S1; S.ref[7 * n + i] = b.S2;
    S.fli_acc[i] = 0.0;
    S.t[i] = 0.0;
    S.nstep[i] = 0;
    S.status[i] = finite12(y) ? ORBIT_RUNNING : ORBIT_NONFINITE;
    S.newton_iters[i] = 0;
    S.n_skip[i] = 0;
    S.last_kind[i] = CORR_DUAL;
}

// ----------------------------------------------------- static integrator
// One orbit per thread for the whole run; stage and trajectory loops rolled
// (one compiled copy of the equations of motion, as in the queue kernel's
// default variant).  RR: with the 2.5PN radiation reaction; the main
// trajectory's reference E and |J| then change and are stored back.
template <bool QM, int RK, bool RR = false>
__global__ void __launch_bounds__(128) k_integrate_static(DevState S, RunCfg rc)
{
    __shared__ double hab[RK == 5 ? 36 : 1];
    if (RK == 5) {
        if (threadIdx.x == 0) rk5_scaled_tableau(rc.h, hab);
        __syncthreads();
    }
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= S.n) return;
    const int32_t st = S.status[i];
    if (st != ORBIT_RUNNING && st != ORBIT_DONE) return;
    Orbit o;
    load_orbit<false>(S, i, o);
    o.status = ORBIT_RUNNING;
    const Coef c = load_coef<false>(S, i, rc.flags);
    const int32_t end = rc.nstep_base + rc.nsteps;
    double k8eta = 0.0;
    if (RR) {
        const double beta = S.beta[i];
        k8eta = 1.6 * (beta / ((1.0 + beta) * (1.0 + beta)));
    }
    advance<QM, RK, Coef, true, RR>(rc, c, o, end, hab, k8eta);
    if (o.status == ORBIT_RUNNING && o.nstep == rc.final_step) o.status = ORBIT_DONE;
    store_orbit(S, i, o);
    if (RR) {
        S.ref[0 * S.ld + i] = o.ref.E;
        S.ref[1 * S.ld + i] = o.ref.J;
    }
}

// ------------------------------------------------ paired static integrator
// Two lanes per orbit: the even lane of a pair integrates the main
// trajectory, the odd lane the shadow.  Each lane issues half of an orbit's
// instructions per step, so a batch too small to fill the SM sub-partitions
// finishes in about half the time.  The lanes exchange data only where the
// method couples the trajectories: the termination tests after each step
// (non-finite either side; merger / escape on the main trajectory) and the
// FLI renormalisation every `renorm` steps (the shadow lane needs the main
// state; the main lane the new distance).  Shuffles are masked to the pair,
// whose lanes always take the same branches.  The operations and their order
// per trajectory are those of advance(): results are bit-identical.
template <bool QM, int RK, bool RR = false>
__global__ void __launch_bounds__(128) k_integrate_pair(DevState S, RunCfg rc)
{
    __shared__ double hab[RK == 5 ? 36 : 1];
    if (RK == 5) {
        if (threadIdx.x == 0) rk5_scaled_tableau(rc.h, hab);
        __syncthreads();
    }
    extern __shared__ double kst_dyn[];          // RK5 stage derivatives (rk_order 5 only)
    double* kst = kst_dyn + threadIdx.x;
    const int kstride = (int)blockDim.x;
    const int64_t gt = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t i = gt >> 1;                   // both lanes of a pair share i
    const bool shadow = (gt & 1) != 0;
    const unsigned lane = threadIdx.x & 31u;
    const unsigned pair = 3u << (lane & ~1u);
    const int main_lane = (int)(lane & ~1u), shadow_lane = (int)(lane | 1u);
    if (i >= S.n) return;
    const int32_t st0 = S.status[i];
    if (st0 != ORBIT_RUNNING && st0 != ORBIT_DONE) return;
    const int64_t n = S.ld;
    const Coef c = load_coef<false>(S, i, rc.flags);
    Vec12 y;
    load12<false>(shadow ? S.ys : S.y, n, i, y);
    const int rb = shadow ? 4 : 0;
    Ref ref;
    ref.E = S.ref[(rb + 0) * n + i];
    ref.J = S.ref[(rb + 1) * n + i];
    ref.S1 = S.ref[(rb + 2) * n + i];
    ref.S2 = S.ref[(rb + 3) * n + i];
    double k8eta = 0.0;
    if (RR) {
        const double beta = S.beta[i];
        k8eta = 1.6 * (beta / ((1.0 + beta) * (1.0 + beta)));
    }
    double acc = S.fli_acc[i];
    const double t0 = S.t[i];
    const int32_t n0 = S.nstep[i];
    int32_t nstep = n0, iters = 0, skips = 0, last_kind = S.last_kind[i];
    int32_t status = ORBIT_RUNNING;
    const int32_t step_end = rc.nstep_base + rc.nsteps;
    double* yv = &y.r[0];
    while (nstep < step_end) {
        if (RR) {
            if (RK == 5) rk5_step_rr<QM, Coef>(c, rc.rrc, k8eta, y, ref, hab, kst, kstride);
            else rk4_step_rr<QM, Coef>(c, rc.rrc, k8eta, y, ref, rc.h);
        } else if (RK == 5) {
            rk5_step_rolled<QM, Coef>(c, y, hab, kst, kstride);
        } else {
            rk4_step_rolled<QM, Coef>(c, y, rc.h);
        }
        if (rc.correct) {
            int kind;
            iters += correct<QM, Coef>(c, y, ref, rc.newton, &kind);
            skips += kind != CORR_DUAL;
            if (!shadow) last_kind = kind;
        }
        nstep++;
        const int fin = finite12(y) ? 1 : 0;
        if (!(fin & __shfl_xor_sync(pair, fin, 1))) { status = ORBIT_NONFINITE; break; }
        int code = 0;
        if (!shadow) {
            const double rr2 = dot3(y.r, y.r);
            if (rc.rmerge2 > 0.0 && rr2 < rc.rmerge2) code = ORBIT_MERGED;
            else if (rc.rescape2 > 0.0 && rr2 > rc.rescape2) code = ORBIT_ESCAPED;
        }
        code = __shfl_sync(pair, code, main_lane);
        if (code) { status = code; break; }
        if (rc.renorm > 0 && (nstep % rc.renorm) == 0) {
            double a[12];
#pragma unroll
            for (int k = 0; k < 12; k++) a[k] = __shfl_sync(pair, yv[k], main_lane);
            double d = 0.0;
            if (shadow) {
                double dv[12];
                double d2 = 0.0;
#pragma unroll
                for (int k = 0; k < 12; k++) {
                    dv[k] = yv[k] - a[k];
                    d2 = fma(dv[k], dv[k], d2);
                }
                d = sqrt(d2);
                const double f = rc.d0 / d;
#pragma unroll
                for (int k = 0; k < 12; k++) yv[k] = fma(f, dv[k], a[k]);
                ref = integrals<QM, Coef>(c, y);
            }
            d = __shfl_sync(pair, d, shadow_lane);
            int sat = 0;
            if (!shadow) {
                acc += log10(d / rc.d0);
                sat = rc.fli_cap > 0.0 && acc >= rc.fli_cap;
            }
            if (__shfl_sync(pair, sat, main_lane)) { status = ORBIT_FLI_SATURATED; break; }
        }
    }
    if (status == ORBIT_RUNNING && nstep == rc.final_step) status = ORBIT_DONE;
    const int32_t it_pair = iters + __shfl_xor_sync(pair, iters, 1);
    const int32_t sk_pair = skips + __shfl_xor_sync(pair, skips, 1);
    if (shadow) {
        store12(S.ys, n, i, y);
        S.ref[4 * n + i] = ref.E;
        S.ref[5 * n + i] = ref.J;
        S.ref[6 * n + i] = ref.S1;
        S.ref[7 * n + i] = ref.S2;
    } else {
        store12(S.y, n, i, y);
        if (RR) {
            S.ref[0 * n + i] = ref.E;
            S.ref[1 * n + i] = ref.J;
        }
        S.fli_acc[i] = acc;
        S.t[i] = t0 + (double)(nstep - n0) * rc.h;
        S.nstep[i] = nstep;
        S.status[i] = status;
        S.newton_iters[i] += it_pair;
        S.n_skip[i] += sk_pair;
        S.last_kind[i] = last_kind;
    }
}

// ------------------------------------------- persistent work-queue integrator
// Tasks are (chunk c, group g): advance the 32 orbits of group g (one warp)
// through steps [c K, (c+1) K) of the run; task (c, g) waits for (c-1, g).
// How the W resident warps get their tasks depends on the G groups:
// - G >= 2W: warps claim tasks from one atomic counter in chunk-major order,
//   so every group advances chunk by chunk and the load balances itself.  A
//   group's next chunk is claimed about G / W task times after its previous
//   one, so with G >= 2W the claiming warp rarely finds it unfinished.
// - G < 2W: that claim order would make warps wait on their predecessors'
//   chunks.  Instead the G x (chunks) units, taken group by group, are cut
//   into min(G, W) contiguous shares of equal size (to one unit), one per
//   warp (McNaughton's wrap-around rule), unless the run is one chunk long
//   (then no task waits, and claims balance the whole groups).  A group cut between the end of
//   warp w's share and the start of warp w + 1's runs its first chunks first
//   on warp w and its last chunks last on warp w + 1, which is after them
//   whenever every share is at least one group long (G >= W); for G < W each
//   warp runs one whole group.  Equal task times then leave no warp waiting;
//   otherwise warp w + 1 waits only on chunks that warp w runs first, and
//   the grid is sized so that every warp is resident.
// Either way an orbit's steps and their arithmetic are the same, so results
// are bit-identical.  Every wait is bounded in time (rc.wait_limit_ns,
// global timer); on expiry the kernel sets the error flag and all warps
// return.
__device__ __forceinline__ int ld_acquire(const int* p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release(int* p, int v)
{
    asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ unsigned long long globaltimer_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// One task: advance group g through chunk c (after waiting for chunk c - 1),
// then publish the group's progress.  Returns false when the kernel must stop
// (a wait ran out).
template <bool QM, bool SMEM, int RK, bool ROLLED, bool RR>
__device__ __forceinline__ bool queue_task(const DevState& S, const RunCfg& rc, const QueueState& q, int chunk,
                                           int use_order, long long nslots, long long c, long long g, int lane,
                                           double* scoef, const double* hab)
{
    int ok = 1;
    if (c > 0 && lane == 0) {
        const unsigned long long t0 = globaltimer_ns();
        while (ld_acquire(q.group_done + g) < c) {
            if (globaltimer_ns() - t0 > rc.wait_limit_ns) {
                atomicExch(q.error, 1);
                ok = 0;
                break;
            }
            __nanosleep(200);
        }
    }
    ok = __shfl_sync(0xffffffffu, ok, 0);
    if (!ok) return false;
    const int64_t slot = g * 32 + lane;
    if (slot < nslots) {
        const int64_t i = use_order ? (int64_t)__ldcg(S.order + slot) : slot;
        const int32_t st = __ldcg(S.status + i);
        if (st == ORBIT_RUNNING || (c == 0 && rc.first_epoch && st == ORBIT_DONE)) {
            Orbit o;
            load_orbit<true>(S, i, o);
            o.status = ORBIT_RUNNING;
            const long long e = (c + 1) * (long long)chunk;
            const int32_t end = rc.nstep_base + (int32_t)(e < rc.nsteps ? e : rc.nsteps);
            if (SMEM) {
                const Coef cf = load_coef<true>(S, i, rc.flags);
                volatile double* mine = scoef + threadIdx.x;
#pragma unroll
                for (int k = 0; k < NCOEF; k++) mine[k * (int)blockDim.x] = cf.v[k];
                const CoefShared cs{mine, (int)blockDim.x};
                advance<QM, RK, CoefShared, ROLLED>(rc, cs, o, end, hab);
            } else {
                const Coef cf = load_coef<true>(S, i, rc.flags);
                double k8eta = 0.0;
                if (RR) {
                    const double beta = __ldcg(S.beta + i);
                    k8eta = 1.6 * (beta / ((1.0 + beta) * (1.0 + beta)));
                }
                advance<QM, RK, Coef, ROLLED, RR>(rc, cf, o, end, hab, k8eta);
            }
            if (o.status == ORBIT_RUNNING && o.nstep == rc.final_step) o.status = ORBIT_DONE;
            store_orbit(S, i, o);
            if (RR) {
                S.ref[0 * S.ld + i] = o.ref.E;
                S.ref[1 * S.ld + i] = o.ref.J;
            }
        }
    }
    __threadfence();
    __syncwarp();
    if (lane == 0 && !(c == 0 && g == rc.stall_group)) st_release(q.group_done + g, (int)(c + 1));
    return true;
}

// SMEM: keep the per-orbit constants in shared memory (one plane per constant)
// instead of registers, which is what lets MINB = 3 blocks fit without spills.
template <bool QM, int MINB, bool SMEM, int RK, bool ROLLED = false, bool RR = false>
__global__ void __launch_bounds__(128, MINB) k_integrate_queue(DevState S, RunCfg rc, QueueState q, int chunk,
                                                                int use_order)
{
    static_assert(!RR || (ROLLED && !SMEM), "radiation reaction: rolled variant with register constants");
    __shared__ double scoef[SMEM ? NCOEF * 128 : 1];
    __shared__ double hab[(RK == 5 && ROLLED) ? 36 : 1];
    if (RK == 5 && ROLLED) {
        if (threadIdx.x == 0) rk5_scaled_tableau(rc.h, hab);
        __syncthreads();
    }
    const int lane = threadIdx.x & 31;
    // compacting schedule: slot s of the dense list holds orbit order[s]
    const long long nslots = use_order ? (long long)__ldcg(q.count) : S.n;
    const long long groups = (nslots + 31) / 32;
    const long long nchunks = (rc.nsteps + chunk - 1) / chunk;
    const long long units = groups * nchunks;
    const long long nwarps = (long long)gridDim.x * (blockDim.x >> 5);
    const long long wshare = groups < nwarps ? groups : nwarps;
    // claims when there are at least two groups per warp, or when the run is one
    // chunk (no task waits; whole-group shares could not balance)
    if (groups >= 2 * nwarps || nchunks == 1) {
        for (;;) {
            unsigned long long task = 0;
            if (lane == 0) task = (*(volatile int*)q.error) ? (unsigned long long)units : atomicAdd(q.next, 1ull);
            task = __shfl_sync(0xffffffffu, task, 0);
            if (task >= (unsigned long long)units) break;
            const long long c = (long long)(task / (unsigned long long)groups);
            const long long g = (long long)(task % (unsigned long long)groups);
            if (!queue_task<QM, SMEM, RK, ROLLED, RR>(S, rc, q, chunk, use_order, nslots, c, g, lane, scoef, hab))
                break;
        }
        return;
    }
    // static share: units [u0, u1) of the group-major order u = g nchunks + c (a
    // balanced cut: every share has floor or ceil of units / wshare units, so at
    // least nchunks when G >= W), run as the first pe chunks of the last group
    // (if it is cut at u1), the whole groups, then the last ps chunks of the
    // first group (if it is cut at u0)
    const long long gw = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (gw >= wshare) return;
    const long long u0 = gw * units / wshare, u1 = (gw + 1) * units / wshare, len = u1 - u0;
    if (len <= 0) return;
    const long long gA = u0 / nchunks, cA = u0 % nchunks, gB = (u1 - 1) / nchunks;
    const long long cBend = (u1 - 1) % nchunks + 1;
    const long long pe = (gA < gB && cBend < nchunks) ? cBend : 0;
    const long long ps = (gA < gB && cA > 0) ? nchunks - cA : 0;
    for (long long k = 0; k < len; k++) {
        int stop = 0;
        if (lane == 0) stop = *(volatile int*)q.error;
        stop = __shfl_sync(0xffffffffu, stop, 0);
        if (stop) break;
        long long c, g;
        if (k < pe) {
            g = gB;
            c = k;
        } else if (k < len - ps) {
            const long long u = u0 + ps + (k - pe);
            g = u / nchunks;
            c = u % nchunks;
        } else {
            g = gA;
            c = cA + (k - (len - ps));
        }
        if (!queue_task<QM, SMEM, RK, ROLLED, RR>(S, rc, q, chunk, use_order, nslots, c, g, lane, scoef, hab))
            break;
    }
}

// ------------------------------------------------------------- compaction
// Running orbits of the current list (or of all orbits) appended to the next
// list with one warp-aggregated atomic per warp; the order within the list
// does not matter, since an orbit's arithmetic does not depend on its slot.
__global__ void k_compact(DevState S, QueueState q, int from_all, int first_epoch)
{
    const long long nslots = from_all ? S.n : (long long)__ldcg(q.count);
    const long long slot = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    bool keep = false;
    int32_t i = 0;
    if (slot < nslots) {
        i = from_all ? (int32_t)slot : __ldcg(S.order + slot);
        const int32_t st = __ldcg(S.status + i);
        keep = st == ORBIT_RUNNING || (first_epoch && st == ORBIT_DONE);
    }
    const unsigned m = __ballot_sync(0xffffffffu, keep);
    int base = 0;
    if (lane == 0 && m) base = atomicAdd(q.count + 1, __popc(m));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (keep) S.order_next[base + __popc(m & ((1u << lane) - 1u))] = i;
}

// --------------------------------------------------------------- finalize
// Integrals of the main trajectory and FLI(t) = acc + log10(d(t)/d0).
template <bool QM>
__global__ void k_finalize(DevState S, RunCfg rc)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= S.n) return;
    const Coef c = load_coef<false>(S, i, rc.flags);
    Vec12 y, ys;
    load12<false>(S.y, S.ld, i, y);
    load12<false>(S.ys, S.ld, i, ys);
    const Ref I = integrals<QM, Coef>(c, y);
    const double* a = &y.r[0];
    const double* b = &ys.r[0];
    double d2 = 0.0;
#pragma unroll
    for (int k = 0; k < 12; k++) d2 = fma(b[k] - a[k], b[k] - a[k], d2);
    const int64_t n = S.ld;
    S.out[0 * n + i] = I.E;
    S.out[1 * n + i] = I.J;
    S.out[2 * n + i] = I.S1;
    S.out[3 * n + i] = I.S2;
    S.out[4 * n + i] = S.fli_acc[i] + log10(sqrt(d2) / rc.d0);
}

// ----------------------------------------------------------- scan summary
__device__ __forceinline__ unsigned long long dbits(double x)
{
    return (unsigned long long)__double_as_longlong(x);
}

__global__ void k_reduce(DevState S, double thr, Summary* out)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    unsigned long long chaotic = 0, iters = 0, skips = 0, steps = 0, fallback = 0;
    double dE = 0.0, dJ = 0.0, dJall = 0.0, dS = 0.0, fmx = -1e300, fsum = 0.0;
    int32_t st = -1;
    if (i < S.n) {
        const int64_t n = S.ld;
        st = S.status[i];
        const double fli = S.out[4 * n + i];
        iters = (unsigned long long)S.newton_iters[i];
        skips = (unsigned long long)S.n_skip[i];
        steps = (unsigned long long)S.nstep[i];
        if (st == ORBIT_DONE || st == ORBIT_FLI_SATURATED) chaotic = fli > thr;
        if (st == ORBIT_DONE) {
            dE = fabs((S.out[0 * n + i] - S.ref[0 * n + i]) / S.ref[0 * n + i]);
            dJall = fabs((S.out[1 * n + i] - S.ref[1 * n + i]) / S.ref[1 * n + i]);
            if (!(dJall == dJall)) dJall = 1e300;
            if (S.last_kind[i] == CORR_DUAL || S.last_kind[i] == CORR_SPLIT) dJ = dJall;
            else fallback = 1;
            const double s1 = S.ref[2 * n + i], s2 = S.ref[3 * n + i];
            if (s1 > 0.0) dS = fmax(dS, fabs(S.out[2 * n + i] - s1) / s1);
            if (s2 > 0.0) dS = fmax(dS, fabs(S.out[3 * n + i] - s2) / s2);
            fmx = fli;
            fsum = fli;
        }
        if (!(dE == dE)) dE = 1e300;
        if (!(dJ == dJ)) dJ = 1e300;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        chaotic += __shfl_down_sync(0xffffffffu, chaotic, off);
        iters += __shfl_down_sync(0xffffffffu, iters, off);
        skips += __shfl_down_sync(0xffffffffu, skips, off);
        steps += __shfl_down_sync(0xffffffffu, steps, off);
        fallback += __shfl_down_sync(0xffffffffu, fallback, off);
        dJall = fmax(dJall, __shfl_down_sync(0xffffffffu, dJall, off));
        dE = fmax(dE, __shfl_down_sync(0xffffffffu, dE, off));
        dJ = fmax(dJ, __shfl_down_sync(0xffffffffu, dJ, off));
        dS = fmax(dS, __shfl_down_sync(0xffffffffu, dS, off));
        fmx = fmax(fmx, __shfl_down_sync(0xffffffffu, fmx, off));
        fsum += __shfl_down_sync(0xffffffffu, fsum, off);
    }
    // status histogram: one ballot per status value
#pragma unroll
    for (int s = 0; s < 6; s++) {
        const unsigned m = __ballot_sync(0xffffffffu, st == s);
        if (lane == 0 && m) atomicAdd(&out->status_count[s], (unsigned long long)__popc(m));
    }
    if (lane == 0) {
        if (chaotic) atomicAdd(&out->n_chaotic, chaotic);
        atomicAdd(&out->newton_iters, iters);
        atomicAdd(&out->n_skip, skips);
        atomicAdd(&out->steps, steps);
        atomicMax(&out->max_dE_bits, dbits(dE));
        atomicMax(&out->max_dJ_bits, dbits(dJ));
        atomicMax(&out->max_dJ_all_bits, dbits(dJall));
        if (fallback) atomicAdd(&out->n_final_fallback, fallback);
        atomicMax(&out->max_dS_bits, dbits(dS));
        if (fmx > -1e300) atomicMax(&out->fli_max_bits, dbits(fmx > 0.0 ? fmx : 0.0));
        atomicAdd(&out->fli_sum, fsum);
    }
}

// ------------------------------------------------------------------ gather
__global__ void k_gather(DevState S, double* states, double* shadow, double* integ)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= S.n) return;
    const int64_t n = S.ld;
    if (states) {
#pragma unroll
        for (int k = 0; k < 12; k++) states[12 * i + k] = S.y[k * n + i];
    }
    if (shadow) {
#pragma unroll
        for (int k = 0; k < 12; k++) shadow[12 * i + k] = S.ys[k * n + i];
    }
    if (integ) {   // E0, E, J0, |J|, |S1|, |S2|
        integ[6 * i + 0] = S.ref[0 * n + i];
        integ[6 * i + 1] = S.out[0 * n + i];
        integ[6 * i + 2] = S.ref[1 * n + i];
        integ[6 * i + 3] = S.out[1 * n + i];
        integ[6 * i + 4] = S.out[2 * n + i];
        integ[6 * i + 5] = S.out[3 * n + i];
    }
}

// ----------------------------------------------------------- FP64 probe
// Independent dependent DFMA chains; measures the FP64 pipe's throughput.
// 8 independent DFMA chains per thread, unrolled by 4: 32 DFMA per loop
// trip, so loop overhead and dependency latency do not limit the rate.
__global__ void k_fp64_probe(double* out, int iters)
{
    double x[8];
#pragma unroll
    for (int k = 0; k < 8; k++) x[k] = threadIdx.x * 1e-3 + k;
    const double a = 0.9999999, b = 1e-7;
#pragma unroll 4
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int k = 0; k < 8; k++) x[k] = fma(x[k], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < 8; k++) s += x[k];
    out[blockIdx.x * (int64_t)blockDim.x + threadIdx.x] = s;
}

// -------------------------------------------------------------- launchers
static inline unsigned grid_for(int64_t n, int block) { return (unsigned)((n + block - 1) / block); }

cudaError_t launch_setup_cells(const double* cells, int64_t n, DevState S, int beta_from_cells, cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    k_setup_cells<<<grid_for(n, 256), 256, 0, st>>>(cells, n, S, beta_from_cells);
    return cudaGetLastError();
}

cudaError_t launch_load_states(const double* states, int64_t n, DevState S, cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    k_load_states<<<grid_for(n, 256), 256, 0, st>>>(states, n, S);
    return cudaGetLastError();
}

cudaError_t launch_init(DevState S, RunCfg rc, cudaStream_t st)
{
    if (S.n == 0) return cudaSuccess;
    if (rc.flags.use_qm) k_init<true><<<grid_for(S.n, 128), 128, 0, st>>>(S, rc);
    else k_init<false><<<grid_for(S.n, 128), 128, 0, st>>>(S, rc);
    return cudaGetLastError();
}

template <int RK, bool RR>
static void launch_static(DevState S, RunCfg rc, int block, cudaStream_t st)
{
    const size_t sm = RK == 5 ? rk5_smem_bytes(block) : 0;
    if (sm > 48 * 1024) {
        cudaFuncSetAttribute(k_integrate_static<true, RK, RR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        cudaFuncSetAttribute(k_integrate_static<false, RK, RR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    }
    if (rc.flags.use_qm) k_integrate_static<true, RK, RR><<<grid_for(S.n, block), block, sm, st>>>(S, rc);
    else k_integrate_static<false, RK, RR><<<grid_for(S.n, block), block, sm, st>>>(S, rc);
}

template <int RK, bool RR>
static void launch_pair(DevState S, RunCfg rc, int block, cudaStream_t st)
{
    const size_t sm = RK == 5 ? rk5_smem_bytes(block) : 0;
    if (sm > 48 * 1024) {
        cudaFuncSetAttribute(k_integrate_pair<true, RK, RR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        cudaFuncSetAttribute(k_integrate_pair<false, RK, RR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    }
    const unsigned grid = grid_for(2 * S.n, block);
    if (rc.flags.use_qm) k_integrate_pair<true, RK, RR><<<grid, block, sm, st>>>(S, rc);
    else k_integrate_pair<false, RK, RR><<<grid, block, sm, st>>>(S, rc);
}

cudaError_t launch_integrate_pair(DevState S, RunCfg rc, int block, cudaStream_t st)
{
    if (S.n == 0 || rc.nsteps <= 0) return cudaSuccess;
    if (block <= 0 || block > 128 || block % 32) return cudaErrorInvalidValue;
    if (rc.rr) {
        if (rc.rk_order == 5) launch_pair<5, true>(S, rc, block, st);
        else launch_pair<4, true>(S, rc, block, st);
    } else {
        if (rc.rk_order == 5) launch_pair<5, false>(S, rc, block, st);
        else launch_pair<4, false>(S, rc, block, st);
    }
    return cudaGetLastError();
}

cudaError_t launch_integrate_static(DevState S, RunCfg rc, int block, cudaStream_t st)
{
    if (S.n == 0 || rc.nsteps <= 0) return cudaSuccess;
    if (block <= 0 || block > 128 || block % 32) return cudaErrorInvalidValue;
    if (rc.rr) {
        if (rc.rk_order == 5) launch_static<5, true>(S, rc, block, st);
        else launch_static<4, true>(S, rc, block, st);
    } else {
        if (rc.rk_order == 5) launch_static<5, false>(S, rc, block, st);
        else launch_static<4, false>(S, rc, block, st);
    }
    return cudaGetLastError();
}

template <int MINB, bool SMEM, int RK, bool ROLLED = false, bool RR = false>
static int occupancy_queue(int block, bool qm)
{
    const size_t sm = RK == 5 ? rk5_smem_bytes(block) : 0;
    int nb = 0;
    if (sm > 48 * 1024) {
        cudaFuncSetAttribute(k_integrate_queue<true, MINB, SMEM, RK, ROLLED, RR>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        cudaFuncSetAttribute(k_integrate_queue<false, MINB, SMEM, RK, ROLLED, RR>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    }
    if (qm) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_integrate_queue<true, MINB, SMEM, RK, ROLLED, RR>, block, sm);
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_integrate_queue<false, MINB, SMEM, RK, ROLLED, RR>, block, sm);
    return nb;
}

// Compiled variants (the `minb` code): RK4 with the per-orbit constants in
// registers, 2 blocks per SM (2); in shared memory, 3 blocks per SM (3); in
// registers with the stage and trajectory loops rolled (4).  RK5 with the
// constants in registers, loops unrolled (2, 3) or rolled (4).
int queue_blocks_per_sm(int block, bool qm, int minb, int rk_order, bool rr)
{
    if (rr) return rk_order == 5 ? occupancy_queue<2, false, 5, true, true>(block, qm)
                                 : occupancy_queue<2, false, 4, true, true>(block, qm);
    if (rk_order == 5)
        return minb == 4 ? occupancy_queue<2, false, 5, true>(block, qm) : occupancy_queue<2, false, 5>(block, qm);
    if (minb == 3) return occupancy_queue<3, true, 4, true>(block, qm);
    if (minb == 4) return occupancy_queue<2, false, 4, true>(block, qm);
    return occupancy_queue<2, false, 4>(block, qm);
}

template <int MINB, bool SMEM, int RK, bool ROLLED = false, bool RR = false>
static void launch_queue(DevState S, RunCfg rc, QueueState q, int block, int grid, int chunk, int use_order,
                         cudaStream_t st)
{
    const size_t sm = RK == 5 ? rk5_smem_bytes(block) : 0;
    if (rc.flags.use_qm)
        k_integrate_queue<true, MINB, SMEM, RK, ROLLED, RR><<<grid, block, sm, st>>>(S, rc, q, chunk, use_order);
    else
        k_integrate_queue<false, MINB, SMEM, RK, ROLLED, RR><<<grid, block, sm, st>>>(S, rc, q, chunk, use_order);
}

cudaError_t launch_integrate_queue(DevState S, RunCfg rc, QueueState q, int block, int grid,
                                   int chunk, int minb, int use_order, cudaStream_t st)
{
    if (S.n == 0 || rc.nsteps <= 0) return cudaSuccess;
    if (block <= 0 || block > 128 || block % 32 || grid <= 0 || chunk <= 0) return cudaErrorInvalidValue;
    // radiation reaction: the default (rolled) variant, whatever minb
    if (rc.rr && rc.rk_order == 5) launch_queue<2, false, 5, true, true>(S, rc, q, block, grid, chunk, use_order, st);
    else if (rc.rr) launch_queue<2, false, 4, true, true>(S, rc, q, block, grid, chunk, use_order, st);
    else if (rc.rk_order == 5 && minb == 4) launch_queue<2, false, 5, true>(S, rc, q, block, grid, chunk, use_order, st);
    else if (rc.rk_order == 5) launch_queue<2, false, 5>(S, rc, q, block, grid, chunk, use_order, st);
    else if (minb == 3) launch_queue<3, true, 4, true>(S, rc, q, block, grid, chunk, use_order, st);
    else if (minb == 4) launch_queue<2, false, 4, true>(S, rc, q, block, grid, chunk, use_order, st);
    else launch_queue<2, false, 4>(S, rc, q, block, grid, chunk, use_order, st);
    return cudaGetLastError();
}

cudaError_t launch_compact(DevState S, QueueState q, int from_all, int first_epoch, cudaStream_t st)
{
    if (S.n == 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(q.count + 1, 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
    k_compact<<<grid_for(S.n, 256), 256, 0, st>>>(S, q, from_all, first_epoch);
    return cudaGetLastError();
}

cudaError_t launch_finalize(DevState S, RunCfg rc, cudaStream_t st)
{
    if (S.n == 0) return cudaSuccess;
    if (rc.flags.use_qm) k_finalize<true><<<grid_for(S.n, 128), 128, 0, st>>>(S, rc);
    else k_finalize<false><<<grid_for(S.n, 128), 128, 0, st>>>(S, rc);
    return cudaGetLastError();
}

cudaError_t launch_reduce(DevState S, double thr, Summary* out, cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(out, 0, sizeof(Summary), st);
    if (e != cudaSuccess || S.n == 0) return e;
    k_reduce<<<grid_for(S.n, 256), 256, 0, st>>>(S, thr, out);
    return cudaGetLastError();
}

cudaError_t launch_gather(DevState S, double* states, double* shadow, double* integ, cudaStream_t st)
{
    if (S.n == 0) return cudaSuccess;
    k_gather<<<grid_for(S.n, 256), 256, 0, st>>>(S, states, shadow, integ);
    return cudaGetLastError();
}

cudaError_t launch_fp64_probe(double* out, int blocks, int threads, int iters, cudaStream_t st)
{
    k_fp64_probe<<<blocks, threads, 0, st>>>(out, iters);
    return cudaGetLastError();
}

}  // namespace pnscan
