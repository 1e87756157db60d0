// pn_noalloc.cu -- scan_summary_noalloc: the scan-level reduction over
// caller-owned device arrays, with its scratch in a fixed device array of
// this library instead of memory allocated at run time.
//
// Who needs it: callers that cannot call cudaMalloc (or any allocating
// routine) when they reduce a scan -- a framework whose caching allocator
// already holds the device memory budget, so that a further cudaMalloc
// would fail or force the framework to release its cache, or a host process
// that forbids run-time allocation after start-up in its latency-critical
// loop.  They pass their own input arrays and a host output struct; the
// library touches no device memory it did not reserve when it was loaded.
// The call waits for its stream to finish (it copies the result into the
// host struct).
//
// Scratch: g_scratch below, kNoallocBlocks + 1 partial records of 256 bytes
// (2.1 MB), reserved on every GPU that loads the library, until the process
// exits.  Every call shares it and leaves the last call's contents behind;
// each call overwrites every record it reads, so nothing has to start at
// zero.  Two calls whose kernels overlap on the GPU (different streams, or
// different host threads) race on it and must be serialised by the caller.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <mutex>

#include "../../include/pnscan.h"

namespace {

constexpr int kNoallocBlock = 256;
constexpr int kNoallocBlocks = PNSCAN_NOALLOC_MAX_ORBITS / kNoallocBlock;   // 8192
constexpr int kMaxDevices = 64;

// One block's partial result (and, at index kNoallocBlocks, the total).
struct __align__(256) NoallocPartial {
    unsigned long long status_count[6];
    unsigned long long n_chaotic, newton_iters, n_skip, steps, n_final_fallback, n_done;
    double max_dE, max_dJ, max_dJ_all, max_dS, fli_max, fli_sum;
};

static __device__ __align__(256) NoallocPartial g_scratch[kNoallocBlocks + 1];

std::mutex g_setup_mutex;
NoallocPartial* g_scratch_ptr[kMaxDevices] = {};

struct Inputs {
    long long n;
    const int32_t* status;
    const double* fli;
    const double* integ;      // n x 6: E0, E, J0, |J|, |S1|, |S2|
    const double* spin_ref;   // n x 2 or null
    const int32_t* iters;     // or null
    const int32_t* skips;     // or null
    const int32_t* last_kind; // or null
    const double* t_stop;     // or null
    double inv_h;
    double thr;
};

__device__ __forceinline__ double warp_max(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
    return v;
}
__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ unsigned long long warp_sum(unsigned long long v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Reduce one NoallocPartial per thread to thread 0 of the block (256 threads).
__device__ void block_reduce(NoallocPartial& p, NoallocPartial* sh)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int k = 0; k < 6; k++) p.status_count[k] = warp_sum(p.status_count[k]);
    p.n_chaotic = warp_sum(p.n_chaotic);
    p.newton_iters = warp_sum(p.newton_iters);
    p.n_skip = warp_sum(p.n_skip);
    p.steps = warp_sum(p.steps);
    p.n_final_fallback = warp_sum(p.n_final_fallback);
    p.n_done = warp_sum(p.n_done);
    p.max_dE = warp_max(p.max_dE);
    p.max_dJ = warp_max(p.max_dJ);
    p.max_dJ_all = warp_max(p.max_dJ_all);
    p.max_dS = warp_max(p.max_dS);
    p.fli_max = warp_max(p.fli_max);
    p.fli_sum = warp_sum(p.fli_sum);
    if (lane == 0) sh[warp] = p;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < kNoallocBlock / 32; w++) {
            const NoallocPartial& q = sh[w];
            for (int k = 0; k < 6; k++) p.status_count[k] += q.status_count[k];
            p.n_chaotic += q.n_chaotic;
            p.newton_iters += q.newton_iters;
            p.n_skip += q.n_skip;
            p.steps += q.steps;
            p.n_final_fallback += q.n_final_fallback;
            p.n_done += q.n_done;
            p.max_dE = fmax(p.max_dE, q.max_dE);
            p.max_dJ = fmax(p.max_dJ, q.max_dJ);
            p.max_dJ_all = fmax(p.max_dJ_all, q.max_dJ_all);
            p.max_dS = fmax(p.max_dS, q.max_dS);
            p.fli_max = fmax(p.fli_max, q.fli_max);
            p.fli_sum += q.fli_sum;
        }
    }
}

__device__ __forceinline__ void clear(NoallocPartial& p)
{
    for (int k = 0; k < 6; k++) p.status_count[k] = 0;
    p.n_chaotic = p.newton_iters = p.n_skip = p.steps = p.n_final_fallback = p.n_done = 0;
    p.max_dE = p.max_dJ = p.max_dJ_all = p.max_dS = 0.0;
    p.fli_max = 0.0;
    p.fli_sum = 0.0;
}

// Pass 1: one partial per block, written in full to scratch[blockIdx.x].
__global__ void __launch_bounds__(kNoallocBlock) k_noalloc_partials(Inputs in, NoallocPartial* scratch)
{
    __shared__ NoallocPartial sh[kNoallocBlock / 32];
    NoallocPartial p;
    clear(p);
    const long long i = blockIdx.x * (long long)kNoallocBlock + threadIdx.x;
    if (i < in.n) {
        const int st = in.status[i];
        if (st >= 0 && st < 6) p.status_count[st] = 1;
        const double f = in.fli[i];
        if (in.iters) p.newton_iters = (unsigned long long)in.iters[i];
        if (in.skips) p.n_skip = (unsigned long long)in.skips[i];
        if (in.t_stop) p.steps = (unsigned long long)llrint(in.t_stop[i] * in.inv_h);
        if (st == PNSCAN_ORBIT_DONE || st == PNSCAN_ORBIT_FLI_SATURATED) p.n_chaotic = f > in.thr;
        if (st == PNSCAN_ORBIT_DONE) {
            const double* I = in.integ + 6 * i;
            double dE = fabs((I[1] - I[0]) / I[0]);
            double dJ = fabs((I[3] - I[2]) / I[2]);
            if (!(dE == dE)) dE = 1e300;
            if (!(dJ == dJ)) dJ = 1e300;
            p.max_dE = dE;
            p.max_dJ_all = dJ;
            // last step dual-scaled (0) or split-scaled (3): |J| was restored
            if (!in.last_kind || in.last_kind[i] == 0 || in.last_kind[i] == 3) p.max_dJ = dJ;
            else p.n_final_fallback = 1;
            if (in.spin_ref) {
                const double s1 = in.spin_ref[2 * i], s2 = in.spin_ref[2 * i + 1];
                if (s1 > 0.0) p.max_dS = fmax(p.max_dS, fabs(I[4] - s1) / s1);
                if (s2 > 0.0) p.max_dS = fmax(p.max_dS, fabs(I[5] - s2) / s2);
            }
            p.fli_max = f > 0.0 ? f : 0.0;
            p.fli_sum = f;
            p.n_done = 1;
        }
    }
    block_reduce(p, sh);
    if (threadIdx.x == 0) scratch[blockIdx.x] = p;
}

// Pass 2: one block folds the nblocks partials into scratch[kNoallocBlocks].
__global__ void __launch_bounds__(kNoallocBlock) k_noalloc_total(int nblocks, NoallocPartial* scratch)
{
    __shared__ NoallocPartial sh[kNoallocBlock / 32];
    NoallocPartial p;
    clear(p);
    for (int b = threadIdx.x; b < nblocks; b += kNoallocBlock) {
        const NoallocPartial& q = scratch[b];
        for (int k = 0; k < 6; k++) p.status_count[k] += q.status_count[k];
        p.n_chaotic += q.n_chaotic;
        p.newton_iters += q.newton_iters;
        p.n_skip += q.n_skip;
        p.steps += q.steps;
        p.n_final_fallback += q.n_final_fallback;
        p.n_done += q.n_done;
        p.max_dE = fmax(p.max_dE, q.max_dE);
        p.max_dJ = fmax(p.max_dJ, q.max_dJ);
        p.max_dJ_all = fmax(p.max_dJ_all, q.max_dJ_all);
        p.max_dS = fmax(p.max_dS, q.max_dS);
        p.fli_max = fmax(p.fli_max, q.fli_max);
        p.fli_sum += q.fli_sum;
    }
    block_reduce(p, sh);
    if (threadIdx.x == 0) scratch[kNoallocBlocks] = p;
}

// Device address of g_scratch on the current device, looked up once per
// device (with that device current) and cached.
int scratch_for_current_device(NoallocPartial** out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return PNSCAN_ERR_NODEVICE;
    }
    if (dev < 0 || dev >= kMaxDevices) return PNSCAN_ERR_ARG;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
        NoallocPartial* ptr = nullptr;
        const cudaError_t e = cudaGetSymbolAddress((void**)&ptr, g_scratch);
        if (e != cudaSuccess || !ptr) {
            cudaGetLastError();
            return PNSCAN_ERR_CUDA;
        }
        g_scratch_ptr[dev] = ptr;
    }
    *out = g_scratch_ptr[dev];
    return PNSCAN_OK;
}

}  // namespace

extern "C" int scan_summary_noalloc(int64_t n, const int32_t* status, const double* fli,
                                    const double* integrals, const double* spin_ref,
                                    const int32_t* newton_iters, const int32_t* n_skip,
                                    const int32_t* last_kind, const double* t_stop, double h_step,
                                    double fli_thresh, void* cuda_stream, scan_summary_t* out)
{
    if (!out || n < 0) return PNSCAN_ERR_ARG;
    if (n > PNSCAN_NOALLOC_MAX_ORBITS) return PNSCAN_ERR_ARG;   // beyond the fixed scratch
    if (n > 0 && (!status || !fli || !integrals)) return PNSCAN_ERR_ARG;
    if (t_stop && !(h_step > 0.0)) return PNSCAN_ERR_ARG;
    NoallocPartial* scratch = nullptr;
    int r = scratch_for_current_device(&scratch);
    if (r != PNSCAN_OK) return r;
    std::memset(out, 0, sizeof(*out));
    out->n = n;
    if (n == 0) return PNSCAN_OK;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    Inputs in{(long long)n, status, fli, integrals, spin_ref, newton_iters, n_skip, last_kind,
              t_stop, t_stop ? 1.0 / h_step : 0.0, fli_thresh};
    const int nblocks = (int)((n + kNoallocBlock - 1) / kNoallocBlock);
    k_noalloc_partials<<<nblocks, kNoallocBlock, 0, st>>>(in, scratch);
    k_noalloc_total<<<1, kNoallocBlock, 0, st>>>(nblocks, scratch);
    if (cudaGetLastError() != cudaSuccess) return PNSCAN_ERR_CUDA;
    NoallocPartial total;
    if (cudaMemcpyAsync(&total, scratch + kNoallocBlocks, sizeof(total), cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return PNSCAN_ERR_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return PNSCAN_ERR_CUDA;
    out->n_chaotic = (int64_t)total.n_chaotic;
    for (int k = 0; k < 6; k++) out->status_count[k] = (int64_t)total.status_count[k];
    out->newton_iters = (int64_t)total.newton_iters;
    out->n_skip = (int64_t)total.n_skip;
    out->orbit_steps = (int64_t)total.steps;
    out->max_dE = total.max_dE;
    out->max_dJ = total.max_dJ;
    out->max_dJ_all = total.max_dJ_all;
    out->n_final_fallback = (int64_t)total.n_final_fallback;
    out->max_dS = total.max_dS;
    out->fli_max = total.fli_max;
    out->fli_mean = total.n_done ? total.fli_sum / (double)total.n_done : 0.0;
    return PNSCAN_OK;
}
