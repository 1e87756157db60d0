// pn_capi.cu -- implementation of the C ABI declared in include/pnscan.h:
// handle lifecycle, host <-> device staging, integrator scheduling (static
// or persistent work queue, optionally replayed from a captured CUDA graph),
// the launch-shape autotuner, the host watchdog and timing.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>
#include <thread>
#include <vector>

#include "../../include/pnscan.h"
#include "pn_kernels.cuh"
#include "pn_waveform.cuh"

using namespace pnscan;

struct scan_handle {
    scan_params p;            // copy; array pointers are not retained
    int device = 0;
    int num_sms = 0;
    cudaStream_t stream = nullptr;     // caller's stream
    cudaStream_t cap_stream = nullptr; // private stream used for graph capture
    DevState S{};
    void* state_block = nullptr;
    size_t state_bytes = 0;
    void* queue_block = nullptr;       // QueueState storage
    size_t queue_bytes = 0;
    QueueState q{};
    Summary* dsum = nullptr;
    double* staging = nullptr;         // n x 12 device staging for host I/O
    bool loaded = false;
    bool beta_from_cells = false;      // beta_m was NULL: scan_setup takes beta from the cells
    double t_now = 0.0;
    int32_t nstep_now = 0;
    RunCfg base{};
    // launch shape (tuned or from params)
    int sched = PNSCAN_SCHED_QUEUE;
    int block = 128;
    int chunk = 500;
    int bps = 0;
    int minb = 2;                      // register-budget variant of the queue kernel
    bool tuned = false;
    // timing of the last run
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    int last_launches = 0;             // kernels launched by the last scan_run
    int glaunches = 0;                 // kernels in the captured graph
    bool timed = false;
    // CUDA graph of the queue run
    cudaGraphExec_t gexec = nullptr;
    RunCfg gcfg{};
    int gshape[5] = {0, 0, 0, 0, 0};
};

namespace {

const char* kVersion = "pnscan 0.1 (sm_103a, FP64)";

int cuda_err(cudaError_t e) { return e == cudaSuccess ? PNSCAN_OK : (e == cudaErrorMemoryAllocation ? PNSCAN_ERR_OOM : PNSCAN_ERR_CUDA); }

void* dev_alloc(scan_handle* h, size_t bytes)
{
    if (bytes == 0) bytes = 256;
    if (h->p.alloc_fn) return h->p.alloc_fn(bytes, h->p.alloc_ctx);
    void* ptr = nullptr;
    if (cudaMalloc(&ptr, bytes) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return ptr;
}

void dev_free(scan_handle* h, void* ptr)
{
    if (!ptr) return;
    if (h->p.free_fn) h->p.free_fn(ptr, h->p.alloc_ctx);
    else cudaFree(ptr);
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// Carve the structure-of-arrays state out of one allocation.
size_t layout_state(DevState& S, char* base, int64_t n)
{
    const int64_t ld = (n + 31) / 32 * 32;
    size_t off = 0;
    auto take = [&](size_t bytes) { char* p = base ? base + off : nullptr; off = align256(off + bytes); return p; };
    S.n = n;
    S.ld = ld;
    S.y = (double*)take(sizeof(double) * 12 * ld);
    S.ys = (double*)take(sizeof(double) * 12 * ld);
    S.ref = (double*)take(sizeof(double) * 8 * ld);
    S.fli_acc = (double*)take(sizeof(double) * ld);
    S.t = (double*)take(sizeof(double) * ld);
    S.nstep = (int32_t*)take(sizeof(int32_t) * ld);
    S.status = (int32_t*)take(sizeof(int32_t) * ld);
    S.newton_iters = (int32_t*)take(sizeof(int32_t) * ld);
    S.n_skip = (int32_t*)take(sizeof(int32_t) * ld);
    S.last_kind = (int32_t*)take(sizeof(int32_t) * ld);
    S.beta = (double*)take(sizeof(double) * ld);
    S.kappa1 = (double*)take(sizeof(double) * ld);
    S.kappa2 = (double*)take(sizeof(double) * ld);
    S.out = (double*)take(sizeof(double) * 5 * ld);
    S.order = (int32_t*)take(sizeof(int32_t) * ld);
    S.order_next = (int32_t*)take(sizeof(int32_t) * ld);
    return off;
}

int sync(scan_handle* h)
{
    if (h->p.sync_timeout_s > 0.0) {
        const auto t0 = std::chrono::steady_clock::now();
        for (;;) {
            cudaError_t e = cudaStreamQuery(h->stream);
            if (e == cudaSuccess) break;
            if (e != cudaErrorNotReady) return cuda_err(e);
            const double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
            if (el > h->p.sync_timeout_s) return PNSCAN_ERR_TIMEOUT;
            std::this_thread::sleep_for(std::chrono::microseconds(200));
        }
    } else {
        cudaError_t e = cudaStreamSynchronize(h->stream);
        if (e != cudaSuccess) return cuda_err(e);
    }
    // a bounded device-side wait of the work queue that gave up?
    int err = 0;
    cudaError_t e = cudaMemcpy(&err, h->q.error, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_err(e);
    return err ? PNSCAN_ERR_KERNEL : PNSCAN_OK;
}

RunCfg make_run(const scan_handle* h, double h_step, int32_t nsteps)
{
    RunCfg rc = h->base;
    rc.h = h_step;
    rc.nstep_base = h->nstep_now;
    rc.nsteps = nsteps;
    rc.final_step = h->nstep_now + nsteps;
    rc.first_epoch = 1;
    return rc;
}

// Copy an array argument to the device staging buffer (or use it in place).
int stage_in(scan_handle* h, const double* src, size_t count, const double** dev)
{
    if (h->p.device_ptrs) {
        *dev = src;
        return PNSCAN_OK;
    }
    cudaError_t e = cudaMemcpyAsync(h->staging, src, count * sizeof(double), cudaMemcpyHostToDevice, h->stream);
    *dev = h->staging;
    return cuda_err(e);
}

int begin_state(scan_handle* h)
{
    RunCfg rc = make_run(h, 1.0, 0);
    int rc_ = cuda_err(launch_init(h->S, rc, h->stream));
    if (rc_ != PNSCAN_OK) return rc_;
    h->loaded = true;
    h->t_now = 0.0;
    h->nstep_now = 0;
    return PNSCAN_OK;
}

int reset_queue(scan_handle* h, cudaStream_t st)
{
    return cuda_err(cudaMemsetAsync(h->queue_block, 0, h->queue_bytes, st));
}

int queue_grid(scan_handle* h, int block, int bps, int minb)
{
    int occ = queue_blocks_per_sm(block, h->base.flags.use_qm != 0, minb, h->base.rk_order, h->base.rr != 0);
    if (occ <= 0) occ = 1;
    if (bps <= 0 || bps > occ) bps = occ;
    return h->num_sms * bps;
}

// Launch the integrator for one run on stream st (no timing).
// Epoch lengths of the compacting schedule: `fixed` steps each, or (fixed =
// 0) 256, 512, 1024, ... steps; the last one cut to the run's end, so orbits
// that stop early leave the dense list soon after they stop.
std::vector<int32_t> epoch_lengths(int32_t nsteps, int32_t fixed)
{
    std::vector<int32_t> e;
    int32_t len = fixed > 0 ? fixed : 256, done = 0;
    while (done < nsteps) {
        const int32_t l = len < nsteps - done ? len : nsteps - done;
        e.push_back(l);
        done += l;
        if (fixed <= 0 && len < (1 << 30) / 2) len *= 2;
    }
    return e;
}

// Kernels launched by one run of the schedule (integrator and compaction;
// queue resets are memsets): *launches, if not null.
int launch_run(scan_handle* h, const RunCfg& rc_in, int sched, int block, int chunk, int bps, int minb,
               const DevState& S, cudaStream_t st, int* launches = nullptr)
{
    // default bound on a task's wait for its predecessor: 20 s plus 2 ms per
    // step of the chunk (a step takes ~0.06 ms for a warp alone on its SM
    // sub-partition, ~0.5 ms with 8 warps sharing it)
    RunCfg rc = rc_in;
    if (rc.wait_limit_ns == 0) rc.wait_limit_ns = 20000000000ull + (unsigned long long)chunk * 2000000ull;
    int dummy = 0;
    int& nl = launches ? *launches : dummy;
    nl = 0;
    if (sched == PNSCAN_SCHED_STATIC) {
        nl = 1;
        return cuda_err(launch_integrate_static(S, rc, block, st));
    }
    if (sched == PNSCAN_SCHED_PAIR) {
        nl = 1;
        return cuda_err(launch_integrate_pair(S, rc, block, st));
    }
    const int grid = queue_grid(h, block, bps, minb);
    if (sched == PNSCAN_SCHED_QUEUE) {
        int r = reset_queue(h, st);
        if (r != PNSCAN_OK) return r;
        nl = 1;
        return cuda_err(launch_integrate_queue(S, rc, h->q, block, grid, chunk, minb, 0, st));
    }
    // PNSCAN_SCHED_COMPACT: epochs over a dense list of the running orbits
    DevState E = S;
    nl = 1;
    int r = cuda_err(launch_compact(E, h->q, 1, 1, st));
    if (r == PNSCAN_OK) r = cuda_err(cudaMemcpyAsync(h->q.count, h->q.count + 1, sizeof(int), cudaMemcpyDeviceToDevice, st));
    std::swap(E.order, E.order_next);
    int32_t offset = 0;
    const std::vector<int32_t> lens = epoch_lengths(rc.nsteps, h->p.epoch_steps);
    for (size_t k = 0; k < lens.size() && r == PNSCAN_OK; k++) {
        RunCfg erc = rc;
        erc.nstep_base = rc.nstep_base + offset;
        erc.nsteps = lens[k];
        erc.first_epoch = k == 0;
        r = reset_queue(h, st);
        if (r == PNSCAN_OK) r = cuda_err(launch_integrate_queue(E, erc, h->q, block, grid, chunk, minb, 1, st));
        ++nl;
        offset += lens[k];
        if (r == PNSCAN_OK && k + 1 < lens.size()) {
            ++nl;
            r = cuda_err(launch_compact(E, h->q, 0, 0, st));
            if (r == PNSCAN_OK)
                r = cuda_err(cudaMemcpyAsync(h->q.count, h->q.count + 1, sizeof(int), cudaMemcpyDeviceToDevice, st));
            std::swap(E.order, E.order_next);
        }
    }
    return r;
}

bool same_run(const RunCfg& a, const RunCfg& b)
{
    return a.flags.pn_order == b.flags.pn_order && a.flags.use_so == b.flags.use_so &&
           a.flags.use_ss == b.flags.use_ss && a.flags.use_qm == b.flags.use_qm &&
           a.newton.tol == b.newton.tol && a.newton.max_iter == b.newton.max_iter &&
           a.newton.det_min == b.newton.det_min && a.newton.apply_small == b.newton.apply_small &&
           a.newton.mode == b.newton.mode && a.newton.split_min == b.newton.split_min &&
           a.newton.cond_switch == b.newton.cond_switch &&
           a.correct == b.correct && a.rk_order == b.rk_order && a.h == b.h &&
           a.d0 == b.d0 && a.renorm == b.renorm && a.fli_cap == b.fli_cap &&
           a.rmerge2 == b.rmerge2 && a.rescape2 == b.rescape2 && a.nstep_base == b.nstep_base &&
           a.nsteps == b.nsteps && a.wait_limit_ns == b.wait_limit_ns && a.stall_group == b.stall_group &&
           a.final_step == b.final_step && a.first_epoch == b.first_epoch;
}

int run_graph(scan_handle* h, const RunCfg& rc)
{
    const int shape[5] = {h->sched, h->block, h->chunk, h->bps, h->minb};
    if (!h->gexec || !same_run(h->gcfg, rc) || std::memcmp(h->gshape, shape, sizeof(shape)) != 0) {
        if (h->gexec) {
            cudaGraphExecDestroy(h->gexec);
            h->gexec = nullptr;
        }
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return cuda_err(e);
        int r = launch_run(h, rc, h->sched, h->block, h->chunk, h->bps, h->minb, h->S, h->cap_stream,
                           &h->glaunches);
        e = cudaStreamEndCapture(h->cap_stream, &g);
        if (r != PNSCAN_OK) {
            if (g) cudaGraphDestroy(g);
            return r;
        }
        if (e != cudaSuccess) return cuda_err(e);
        e = cudaGraphInstantiate(&h->gexec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return cuda_err(e);
        h->gcfg = rc;
        std::memcpy(h->gshape, shape, sizeof(shape));
    }
    h->last_launches = h->glaunches;
    return cuda_err(cudaGraphLaunch(h->gexec, h->stream));
}

}  // namespace

extern "C" {

int scan_params_default(scan_params* p)
{
    if (!p) return PNSCAN_ERR_ARG;
    std::memset(p, 0, sizeof(*p));
    p->pn_order = 2;
    p->use_so = 1;
    p->use_ss = 1;
    p->use_qm = 0;
    p->correct = 1;
    p->rk_order = 4;
    p->newton_tol = 1e-10;
    p->newton_max = 50;
    p->newton_det_min = 1e-5;
    p->newton_split_min = 1e-3;
    p->newton_cond_switch = 1e-2;
    p->newton_apply_small = 1;
    p->fli_d0 = 1e-9;
    p->fli_renorm_steps = 100;
    p->fli_thresh = 6.0;
    p->fli_cap = 0.0;
    p->r_merge = 6.0;
    p->r_escape = 1e3;
    p->schedule = PNSCAN_SCHED_AUTO;
    p->use_graph = 1;
    p->queue_wait_limit_ms = 0;
    p->radiation_reaction = 0;
    p->rr_gauge_a = 4.0;
    p->rr_gauge_b = 5.0;
    return PNSCAN_OK;
}

int scan_create(const scan_params* p, scan_handle** out)
{
    if (!out) return PNSCAN_ERR_ARG;
    *out = nullptr;
    if (!p || p->n < 0 || p->n > (int64_t)1 << 31) return PNSCAN_ERR_ARG;
    if (p->pn_order < 0 || p->pn_order > 2) return PNSCAN_ERR_ARG;
    if (!(p->newton_tol > 0.0) || p->newton_max < 1 || p->newton_max > 1000 || !(p->newton_det_min >= 0.0) ||
        !(p->newton_split_min >= 0.0) || !(p->newton_split_min < 1.0) || !(p->newton_cond_switch >= 0.0) ||
        !(p->newton_cond_switch < 1.0))
        return PNSCAN_ERR_ARG;
    if (!(p->fli_d0 > 0.0)) return PNSCAN_ERR_ARG;
    if (p->block_size && (p->block_size < 32 || p->block_size > 128 || p->block_size % 32)) return PNSCAN_ERR_ARG;
    if (p->chunk_steps < 0 || p->blocks_per_sm < 0 || p->queue_wait_limit_ms < 0 || p->epoch_steps < 0)
        return PNSCAN_ERR_ARG;
    if (p->register_variant != 0 && (p->register_variant < 2 || p->register_variant > 4)) return PNSCAN_ERR_ARG;
    if (p->rk_order != 0 && p->rk_order != 4 && p->rk_order != 5) return PNSCAN_ERR_ARG;
    if (p->schedule < 0 || p->schedule > 4) return PNSCAN_ERR_ARG;
    if (p->correct < 0 || p->correct > 3) return PNSCAN_ERR_ARG;
    if ((p->alloc_fn == nullptr) != (p->free_fn == nullptr)) return PNSCAN_ERR_ARG;
    if (p->radiation_reaction != 0 && p->radiation_reaction != 1) return PNSCAN_ERR_ARG;
    if (p->radiation_reaction && (!std::isfinite(p->rr_gauge_a) || !std::isfinite(p->rr_gauge_b)))
        return PNSCAN_ERR_ARG;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return PNSCAN_ERR_NODEVICE;
    }
    // beta must lie in (0, 1] (m1 <= m2, Sec. 2)
    const int64_t n = p->n;
    if (!p->device_ptrs && n > 0 && p->beta_m) {
        for (int64_t i = 0; i < n; i++)
            if (!(p->beta_m[i] > 0.0 && p->beta_m[i] <= 1.0)) return PNSCAN_ERR_ARG;
    }

    scan_handle* h = new (std::nothrow) scan_handle();
    if (!h) return PNSCAN_ERR_OOM;
    h->p = *p;
    h->beta_from_cells = p->beta_m == nullptr;
    h->p.beta_m = h->p.kappa1 = h->p.kappa2 = nullptr;
    h->stream = (cudaStream_t)p->cuda_stream;
    cudaGetDevice(&h->device);
    cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device);
    int r = PNSCAN_OK;
    auto fail = [&](int code) { scan_destroy(h); return code; };

    h->state_bytes = layout_state(h->S, nullptr, n);
    h->state_block = dev_alloc(h, h->state_bytes);
    if (!h->state_block) return fail(PNSCAN_ERR_OOM);
    layout_state(h->S, (char*)h->state_block, n);

    const int64_t groups = (n + 31) / 32;
    h->queue_bytes = align256(sizeof(unsigned long long)) + align256(sizeof(int)) + align256(sizeof(int) * (groups + 1));
    h->queue_block = dev_alloc(h, h->queue_bytes + align256(2 * sizeof(int)) + align256(sizeof(Summary)));
    if (!h->queue_block) return fail(PNSCAN_ERR_OOM);
    {
        char* b = (char*)h->queue_block;
        h->q.next = (unsigned long long*)b;
        h->q.error = (int*)(b + align256(sizeof(unsigned long long)));
        h->q.group_done = (int*)(b + align256(sizeof(unsigned long long)) + align256(sizeof(int)));
        h->q.count = (int*)(b + h->queue_bytes);
        h->dsum = (Summary*)(b + h->queue_bytes + align256(2 * sizeof(int)));
    }
    if (!p->device_ptrs) {
        h->staging = (double*)dev_alloc(h, sizeof(double) * 12 * (size_t)(n > 0 ? n : 1));
        if (!h->staging) return fail(PNSCAN_ERR_OOM);
    }
    if (cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreate(&h->ev0) != cudaSuccess || cudaEventCreate(&h->ev1) != cudaSuccess)
        return fail(PNSCAN_ERR_CUDA);
    r = reset_queue(h, h->stream);
    if (r != PNSCAN_OK) return fail(r);

    // per-orbit physical parameters
    if (n > 0) {
        const cudaMemcpyKind kind = p->device_ptrs ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
        if (p->beta_m && cudaMemcpyAsync(h->S.beta, p->beta_m, sizeof(double) * n, kind, h->stream) != cudaSuccess)
            return fail(PNSCAN_ERR_CUDA);
        for (int k = 0; k < 2; k++) {
            const double* src = k == 0 ? p->kappa1 : p->kappa2;
            double* dst = k == 0 ? h->S.kappa1 : h->S.kappa2;
            if (src) {
                if (cudaMemcpyAsync(dst, src, sizeof(double) * n, kind, h->stream) != cudaSuccess)
                    return fail(PNSCAN_ERR_CUDA);
            } else {
                std::vector<double> ones((size_t)n, 1.0);
                if (cudaMemcpyAsync(dst, ones.data(), sizeof(double) * n, cudaMemcpyHostToDevice, h->stream) != cudaSuccess ||
                    cudaStreamSynchronize(h->stream) != cudaSuccess)
                    return fail(PNSCAN_ERR_CUDA);
            }
        }
    }
    // per-run constants
    RunCfg& b = h->base;
    b.flags.pn_order = p->pn_order;
    b.flags.use_so = p->use_so != 0;
    b.flags.use_ss = p->use_ss != 0;
    b.flags.use_qm = p->use_qm != 0;
    b.newton.tol = p->newton_tol;
    b.newton.max_iter = p->newton_max;
    b.newton.det_min = p->newton_det_min;
    b.newton.split_min = p->newton_split_min;
    b.newton.cond_switch = p->newton_cond_switch;
    b.newton.apply_small = p->newton_apply_small != 0;
    b.newton.mode = p->correct;
    b.correct = p->correct != 0;
    b.rk_order = p->rk_order == 5 ? 5 : 4;
    b.d0 = p->fli_d0;
    b.renorm = p->fli_renorm_steps;
    b.fli_cap = p->fli_cap;
    b.rmerge2 = p->r_merge > 0.0 ? p->r_merge * p->r_merge : 0.0;
    b.rescape2 = p->r_escape > 0.0 ? p->r_escape * p->r_escape : 0.0;
    b.wait_limit_ns = (unsigned long long)p->queue_wait_limit_ms * 1000000ull;   // 0: set per launch
    // test switch of the bounded queue wait (documented with queue_wait_limit_ms)
    b.stall_group = -1;
    if (const char* env = std::getenv("PNSCAN_TEST_STALL_GROUP")) {
        char* end = nullptr;
        const long g = std::strtol(env, &end, 10);
        if (end != env && *end == '\0' && g >= 0 && g < (1L << 30)) b.stall_group = (int)g;
    }
    b.rr = p->radiation_reaction;
    b.rrc = make_rr_coef(p->rr_gauge_a, p->rr_gauge_b);
    // AUTO beyond one resident wave: the compacting schedule at 62-step tasks.
    // Measured (GB300, against the plain work queue at 500): the uneven 1e5
    // batch 2.95e8 against 1.67e8 orbit-steps/s, a 65,536-orbit QM subset
    // (mergers spread over the run) 2.73e8 against 2.38e8, a 51,700-cell
    // batch without cuts the same, the 314 x 314 scan 0.7 % slower.
    const bool auto_sched = p->schedule == PNSCAN_SCHED_AUTO;
    h->sched = auto_sched ? PNSCAN_SCHED_COMPACT : p->schedule;
    h->block = p->block_size ? p->block_size : 128;
    // AUTO with few orbits.  Chained work-queue tasks would share SM
    // sub-partitions and take up to twice one orbit's serial time, so:
    // - n <= 128 x SMs (one warp of 32 orbits per sub-partition): the paired
    //   kernel in one-warp blocks, each warp issuing half of an orbit's
    //   instructions per step (2,048-16,384 orbits: 1.2-2x faster than static);
    // - n <= 256 x SMs (every orbit in one resident wave of one-warp blocks;
    //   the integrators use <= 255 registers per thread, so at least 8 warps
    //   per SM are resident): the static kernel in one-warp blocks.
    if (p->schedule == PNSCAN_SCHED_AUTO && n <= (int64_t)32 * 8 * h->num_sms) {
        h->sched = n <= (int64_t)32 * 4 * h->num_sms ? PNSCAN_SCHED_PAIR : PNSCAN_SCHED_STATIC;
        if (!p->block_size) h->block = 32;
    }
    h->chunk = p->chunk_steps ? p->chunk_steps : (auto_sched && h->sched == PNSCAN_SCHED_COMPACT ? 62 : 500);
    h->bps = p->blocks_per_sm;
    h->minb = p->register_variant >= 2 ? p->register_variant : 4;
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) return fail(PNSCAN_ERR_CUDA);
    *out = h;
    return PNSCAN_OK;
}

int scan_setup(scan_handle* h, const double* cells)
{
    if (!h || (!cells && h->S.n > 0)) return PNSCAN_ERR_ARG;
    const double* d = nullptr;
    int r = PNSCAN_OK;
    if (h->S.n > 0) {
        r = stage_in(h, cells, (size_t)h->S.n * 9, &d);
        if (r != PNSCAN_OK) return r;
        r = cuda_err(launch_setup_cells(d, h->S.n, h->S, h->beta_from_cells ? 1 : 0, h->stream));
        if (r != PNSCAN_OK) return r;
    }
    return begin_state(h);
}

int scan_run(scan_handle* h, const double* initial_states, double t_end, double h_step)
{
    if (!h || !(h_step > 0.0) || !std::isfinite(t_end)) return PNSCAN_ERR_ARG;
    int r = PNSCAN_OK;
    if (initial_states) {
        if (h->beta_from_cells) return PNSCAN_ERR_STATE;   // beta comes only with scan_setup's cells
        if (h->S.n > 0) {
            const double* d = nullptr;
            r = stage_in(h, initial_states, (size_t)h->S.n * 12, &d);
            if (r != PNSCAN_OK) return r;
            r = cuda_err(launch_load_states(d, h->S.n, h->S, h->stream));
            if (r != PNSCAN_OK) return r;
        }
        r = begin_state(h);
        if (r != PNSCAN_OK) return r;
    }
    if (!h->loaded) return PNSCAN_ERR_STATE;
    const double span = t_end - h->t_now;
    if (span < -1e-9 * std::fabs(h_step)) return PNSCAN_ERR_ARG;
    const double steps_d = std::nearbyint(span / h_step);
    if (steps_d < 0.0 || steps_d + h->nstep_now > 2.0e9) return PNSCAN_ERR_ARG;
    const int32_t nsteps = (int32_t)steps_d;
    h->timed = false;
    h->last_launches = 0;
    if (nsteps > 0 && h->S.n > 0) {
        const RunCfg rc = make_run(h, h_step, nsteps);
        if (cudaEventRecord(h->ev0, h->stream) != cudaSuccess) return PNSCAN_ERR_CUDA;
        if (h->sched != PNSCAN_SCHED_STATIC && h->sched != PNSCAN_SCHED_PAIR && h->p.use_graph) r = run_graph(h, rc);
        else r = launch_run(h, rc, h->sched, h->block, h->chunk, h->bps, h->minb, h->S, h->stream,
                            &h->last_launches);
        if (r != PNSCAN_OK) return r;
        if (cudaEventRecord(h->ev1, h->stream) != cudaSuccess) return PNSCAN_ERR_CUDA;
        h->timed = true;
    }
    h->t_now = h->t_now + nsteps * h_step;
    h->nstep_now += nsteps;
    return PNSCAN_OK;
}

int scan_read(scan_handle* h, double* states, double* integrals, double* fli, int32_t* status, double* t_stop)
{
    if (!h) return PNSCAN_ERR_ARG;
    if (!h->loaded) return PNSCAN_ERR_STATE;
    const int64_t n = h->S.n;
    int r = PNSCAN_OK;
    if (n > 0) {
        const RunCfg rc = make_run(h, 1.0, 0);
        r = cuda_err(launch_finalize(h->S, rc, h->stream));
        if (r != PNSCAN_OK) return r;
        const cudaMemcpyKind d2x = h->p.device_ptrs ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
        // AoS outputs go through the staging buffer when host pointers are used
        struct { double* dst; int which; size_t per; } aos[2] = {{states, 0, 12}, {integrals, 2, 6}};
        for (auto& a : aos) {
            if (!a.dst) continue;
            double* dd = h->p.device_ptrs ? a.dst : h->staging;
            r = cuda_err(launch_gather(h->S, a.which == 0 ? dd : nullptr, nullptr, a.which == 2 ? dd : nullptr, h->stream));
            if (r != PNSCAN_OK) return r;
            if (!h->p.device_ptrs) {
                r = cuda_err(cudaMemcpyAsync(a.dst, h->staging, sizeof(double) * a.per * n, d2x, h->stream));
                if (r != PNSCAN_OK) return r;
            }
        }
        if (fli && cudaMemcpyAsync(fli, h->S.out + 4 * h->S.ld, sizeof(double) * n, d2x, h->stream) != cudaSuccess)
            return PNSCAN_ERR_CUDA;
        if (status && cudaMemcpyAsync(status, h->S.status, sizeof(int32_t) * n, d2x, h->stream) != cudaSuccess)
            return PNSCAN_ERR_CUDA;
        if (t_stop && cudaMemcpyAsync(t_stop, h->S.t, sizeof(double) * n, d2x, h->stream) != cudaSuccess)
            return PNSCAN_ERR_CUDA;
    }
    return sync(h);
}

int scan_read_diag(scan_handle* h, double* shadow, int32_t* newton_iters, int32_t* n_skip,
                   int32_t* last_kind)
{
    if (!h) return PNSCAN_ERR_ARG;
    if (!h->loaded) return PNSCAN_ERR_STATE;
    const int64_t n = h->S.n;
    if (n > 0) {
        const cudaMemcpyKind d2x = h->p.device_ptrs ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
        if (shadow) {
            double* dd = h->p.device_ptrs ? shadow : h->staging;
            int r = cuda_err(launch_gather(h->S, nullptr, dd, nullptr, h->stream));
            if (r != PNSCAN_OK) return r;
            if (!h->p.device_ptrs &&
                cudaMemcpyAsync(shadow, h->staging, sizeof(double) * 12 * n, d2x, h->stream) != cudaSuccess)
                return PNSCAN_ERR_CUDA;
        }
        if (newton_iters &&
            cudaMemcpyAsync(newton_iters, h->S.newton_iters, sizeof(int32_t) * n, d2x, h->stream) != cudaSuccess)
            return PNSCAN_ERR_CUDA;
        if (n_skip && cudaMemcpyAsync(n_skip, h->S.n_skip, sizeof(int32_t) * n, d2x, h->stream) != cudaSuccess)
            return PNSCAN_ERR_CUDA;
        if (last_kind &&
            cudaMemcpyAsync(last_kind, h->S.last_kind, sizeof(int32_t) * n, d2x, h->stream) != cudaSuccess)
            return PNSCAN_ERR_CUDA;
    }
    return sync(h);
}

int scan_summary(scan_handle* h, scan_summary_t* out)
{
    if (!h || !out) return PNSCAN_ERR_ARG;
    if (!h->loaded) return PNSCAN_ERR_STATE;
    const RunCfg rc = make_run(h, 1.0, 0);
    int r = cuda_err(launch_finalize(h->S, rc, h->stream));
    if (r != PNSCAN_OK) return r;
    r = cuda_err(launch_reduce(h->S, h->p.fli_thresh, h->dsum, h->stream));
    if (r != PNSCAN_OK) return r;
    Summary s;
    if (cudaMemcpyAsync(&s, h->dsum, sizeof(Summary), cudaMemcpyDeviceToHost, h->stream) != cudaSuccess)
        return PNSCAN_ERR_CUDA;
    r = sync(h);
    if (r != PNSCAN_OK) return r;
    auto bits = [](unsigned long long b) { double d; std::memcpy(&d, &b, sizeof(d)); return d; };
    std::memset(out, 0, sizeof(*out));
    out->n = h->S.n;
    out->n_chaotic = (int64_t)s.n_chaotic;
    for (int k = 0; k < 6; k++) out->status_count[k] = (int64_t)s.status_count[k];
    out->newton_iters = (int64_t)s.newton_iters;
    out->n_skip = (int64_t)s.n_skip;
    out->orbit_steps = (int64_t)s.steps;
    out->max_dE = bits(s.max_dE_bits);
    out->max_dJ = bits(s.max_dJ_bits);
    out->max_dJ_all = bits(s.max_dJ_all_bits);
    out->n_final_fallback = (int64_t)s.n_final_fallback;
    out->max_dS = bits(s.max_dS_bits);
    out->fli_max = bits(s.fli_max_bits);
    out->fli_mean = s.status_count[PNSCAN_ORBIT_DONE] ? s.fli_sum / (double)s.status_count[PNSCAN_ORBIT_DONE] : 0.0;
    return PNSCAN_OK;
}

int scan_autotune(scan_handle* h, int steps, int* schedule, int* block_size, int* chunk_steps, int* blocks_per_sm,
                  int* register_variant)
{
    if (!h || steps <= 0) return PNSCAN_ERR_ARG;
    if (!h->loaded) return PNSCAN_ERR_STATE;
    int r = PNSCAN_OK;
    if (h->S.n > 0) {
        // scratch copy of the state: candidates run on it, the handle's state is untouched
        DevState T{};
        const size_t bytes = layout_state(T, nullptr, h->S.n);
        void* blk = dev_alloc(h, bytes);
        if (!blk) return PNSCAN_ERR_OOM;
        layout_state(T, (char*)blk, h->S.n);
        struct Cand { int sched, block, chunk, bps, minb; };
        std::vector<Cand> cands;
        for (int blk_sz : {32, 64, 128}) cands.push_back({PNSCAN_SCHED_STATIC, blk_sz, 0, 0, 2});
        // radiation reaction: one (rolled) queue variant
        const bool rr = h->base.rr != 0;
        for (int blk_sz : {32, 64}) cands.push_back({PNSCAN_SCHED_PAIR, blk_sz, 0, 0, 2});
        for (int ch : {steps / 32, steps / 16, steps / 8})
            if (ch >= 1) cands.push_back({PNSCAN_SCHED_COMPACT, 128, ch, 0, 4});
        if (!rr && steps / 16 >= 1) cands.push_back({PNSCAN_SCHED_COMPACT, 128, steps / 16, 0, 2});
        for (int minb : {2, 3, 4})
            for (int ch : {steps / 16, steps / 8, steps / 4}) {
                if (ch < 1 || (rr && minb != 4)) continue;
                cands.push_back({PNSCAN_SCHED_QUEUE, 128, ch, 0, minb});
                if (minb == 2) cands.push_back({PNSCAN_SCHED_QUEUE, 128, ch, 1, minb});
                if (minb == 3) cands.push_back({PNSCAN_SCHED_QUEUE, 64, ch, 0, minb});
            }
        double best = 1e300;
        Cand bestc = cands[0];
        cudaEvent_t e0, e1;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        // time one candidate over `n` steps on a fresh copy of the state
        auto time_cand = [&](const Cand& c, const RunCfg& rcn, float* ms) -> int {
            if (cudaMemcpyAsync(blk, h->state_block, bytes, cudaMemcpyDeviceToDevice, h->stream) != cudaSuccess)
                return PNSCAN_ERR_CUDA;
            cudaEventRecord(e0, h->stream);
            int rr2 = launch_run(h, rcn, c.sched, c.block, c.chunk, c.bps, c.minb, T, h->stream);
            cudaEventRecord(e1, h->stream);
            if (rr2 != PNSCAN_OK) return rr2;
            rr2 = sync(h);
            if (rr2 != PNSCAN_OK) return rr2;
            cudaEventElapsedTime(ms, e0, e1);
            return PNSCAN_OK;
        };
        const RunCfg rc = make_run(h, 1.0, steps);
        std::vector<float> times;
        for (const Cand& c : cands) {
            float ms = 0.f;
            r = time_cand(c, rc, &ms);
            if (r != PNSCAN_OK) break;
            times.push_back(ms);
            if (ms < best) {
                best = ms;
                bestc = c;
            }
        }
        // Shapes within 1 % of the best are re-timed over four times the trial:
        // what separates them (e.g. compacting against plain work queue, whose
        // order flips between 2,000 and 8,000 steps of the 314 x 314 scan) is
        // often below a short trial's resolution.
        if (r == PNSCAN_OK && steps <= (1 << 28)) {
            std::vector<Cand> close;
            for (size_t k = 0; k < times.size(); k++)
                if (times[k] <= 1.01 * best) close.push_back(cands[k]);
            if (close.size() > 1) {
                const RunCfg rc4 = make_run(h, 1.0, 4 * steps);
                double best4 = 1e300;
                for (const Cand& c : close) {
                    float ms = 0.f;
                    r = time_cand(c, rc4, &ms);
                    if (r != PNSCAN_OK) break;
                    if (ms < best4) {
                        best4 = ms;
                        bestc = c;
                    }
                }
            }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        dev_free(h, blk);
        if (r != PNSCAN_OK) return r;
        h->sched = bestc.sched;
        h->block = bestc.block;
        // the tuned chunk length (in steps) is kept for longer runs too: more
        // chunks per group only shorten the tail (the static and paired
        // schedules have no chunks and keep the previous setting)
        h->chunk = (bestc.sched != PNSCAN_SCHED_STATIC && bestc.sched != PNSCAN_SCHED_PAIR) ? bestc.chunk : h->chunk;
        h->bps = bestc.bps;
        h->minb = bestc.minb;
        h->tuned = true;
    }
    if (schedule) *schedule = h->sched;
    if (block_size) *block_size = h->block;
    if (chunk_steps) *chunk_steps = h->chunk;
    if (blocks_per_sm) *blocks_per_sm = h->bps;
    if (register_variant) *register_variant = h->minb;
    return PNSCAN_OK;
}

// Checkpoint: a header with the run configuration and the handle's time and
// step counters, then the whole device state block (both trajectories,
// reference integrals, FLI accumulators, times, step counters, statuses,
// Newton counters, per-orbit parameters).
struct CheckpointHeader {
    char magic[8];
    int64_t n;
    uint64_t state_bytes;
    double t_now;
    int64_t nstep_now;
    Flags flags;
    int newton_max, newton_apply_small, newton_mode, correct, rk_order, renorm;
    double newton_tol, newton_det_min, d0, fli_cap, rmerge2, rescape2;
    int rr;
    RRCoef rrc;
    double newton_split_min, newton_cond_switch;
};

static const char kCheckpointMagic[8] = {'P', 'N', 'S', 'C', 'A', 'N', '0', '2'};

static void fill_header(const scan_handle* h, CheckpointHeader& c)
{
    std::memset(&c, 0, sizeof(c));
    std::memcpy(c.magic, kCheckpointMagic, sizeof(c.magic));
    c.n = h->S.n;
    c.state_bytes = h->state_bytes;
    c.t_now = h->t_now;
    c.nstep_now = h->nstep_now;
    const RunCfg& b = h->base;
    c.flags = b.flags;
    c.newton_max = b.newton.max_iter;
    c.newton_apply_small = b.newton.apply_small;
    c.newton_mode = b.newton.mode;
    c.correct = b.correct;
    c.rk_order = b.rk_order;
    c.renorm = b.renorm;
    c.newton_tol = b.newton.tol;
    c.newton_det_min = b.newton.det_min;
    c.newton_split_min = b.newton.split_min;
    c.newton_cond_switch = b.newton.cond_switch;
    c.d0 = b.d0;
    c.fli_cap = b.fli_cap;
    c.rmerge2 = b.rmerge2;
    c.rescape2 = b.rescape2;
    c.rr = b.rr;
    c.rrc = b.rrc;
}

size_t scan_checkpoint_size(scan_handle* h)
{
    return h ? sizeof(CheckpointHeader) + h->state_bytes : 0;
}

int scan_checkpoint(scan_handle* h, void* buf, size_t bytes)
{
    if (!h || !buf || bytes < scan_checkpoint_size(h)) return PNSCAN_ERR_ARG;
    if (!h->loaded) return PNSCAN_ERR_STATE;
    CheckpointHeader c;
    fill_header(h, c);
    std::memcpy(buf, &c, sizeof(c));
    char* dst = (char*)buf + sizeof(c);
    if (h->state_bytes &&
        cudaMemcpyAsync(dst, h->state_block, h->state_bytes, cudaMemcpyDeviceToHost, h->stream) != cudaSuccess)
        return PNSCAN_ERR_CUDA;
    return sync(h);
}

int scan_restore(scan_handle* h, const void* buf, size_t bytes)
{
    if (!h || !buf || bytes < sizeof(CheckpointHeader)) return PNSCAN_ERR_ARG;
    CheckpointHeader c, mine;
    std::memcpy(&c, buf, sizeof(c));
    fill_header(h, mine);
    // the checkpoint must come from a handle with the same orbits and physics
    mine.t_now = c.t_now;
    mine.nstep_now = c.nstep_now;
    if (std::memcmp(&c, &mine, sizeof(c)) != 0 || bytes < sizeof(c) + c.state_bytes) return PNSCAN_ERR_ARG;
    const char* src = (const char*)buf + sizeof(c);
    if (h->state_bytes &&
        cudaMemcpyAsync(h->state_block, src, h->state_bytes, cudaMemcpyHostToDevice, h->stream) != cudaSuccess)
        return PNSCAN_ERR_CUDA;
    const int r = sync(h);
    if (r != PNSCAN_OK) return r;
    h->t_now = c.t_now;
    h->nstep_now = (int32_t)c.nstep_now;
    h->loaded = true;
    return PNSCAN_OK;
}

int scan_waveform(scan_handle* h, double R, const double* P, const double* Q, double* hplus, double* hcross)
{
    if (!h || !P || !Q || !(R > 0.0) || !std::isfinite(R)) return PNSCAN_ERR_ARG;
    for (int k = 0; k < 3; k++)
        if (!std::isfinite(P[k]) || !std::isfinite(Q[k])) return PNSCAN_ERR_ARG;
    if (!h->loaded) return PNSCAN_ERR_STATE;
    const int64_t n = h->S.n;
    if (n == 0 || (!hplus && !hcross)) return PNSCAN_OK;
    const RunCfg rc = make_run(h, 1.0, 0);
    const bool dev = h->p.device_ptrs != 0;
    double* dp = hplus ? (dev ? hplus : h->staging) : nullptr;
    double* dc = hcross ? (dev ? hcross : h->staging + n) : nullptr;
    int r = cuda_err(launch_waveform(h->S, rc, R, P, Q, dp, dc, h->stream));
    if (r != PNSCAN_OK) return r;
    if (!dev) {
        if (hplus && cudaMemcpyAsync(hplus, dp, sizeof(double) * n, cudaMemcpyDeviceToHost, h->stream) != cudaSuccess)
            return PNSCAN_ERR_CUDA;
        if (hcross && cudaMemcpyAsync(hcross, dc, sizeof(double) * n, cudaMemcpyDeviceToHost, h->stream) != cudaSuccess)
            return PNSCAN_ERR_CUDA;
    }
    return sync(h);
}

int scan_last_run_timing(scan_handle* h, double* ms, int* launches)
{
    if (!h) return PNSCAN_ERR_ARG;
    float t = 0.f;
    if (h->timed) {
        if (cudaEventSynchronize(h->ev1) != cudaSuccess) return PNSCAN_ERR_CUDA;
        if (cudaEventElapsedTime(&t, h->ev0, h->ev1) != cudaSuccess) return PNSCAN_ERR_CUDA;
    }
    if (ms) *ms = t;
    if (launches) *launches = h->last_launches;
    return PNSCAN_OK;
}

int scan_fp64_peak(scan_handle* h, int iters, double* tflops)
{
    if (!h || !tflops || iters <= 0) return PNSCAN_ERR_ARG;
    // one block per SM of 4, 8 and 16 warps (one, two and four per
    // sub-partition); the best of the three is reported
    const int threads_list[3] = {128, 256, 512}, blocks = h->num_sms;
    double* buf = (double*)dev_alloc(h, sizeof(double) * 512 * blocks);
    if (!buf) return PNSCAN_ERR_OOM;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    int r = PNSCAN_OK;
    double best = 0.0;
    for (int t = 0; t < 3 && r == PNSCAN_OK; t++) {
        const int threads = threads_list[t];
        r = cuda_err(launch_fp64_probe(buf, blocks, threads, iters / 10 + 1, h->stream));   // warm-up
        cudaEventRecord(e0, h->stream);
        if (r == PNSCAN_OK) r = cuda_err(launch_fp64_probe(buf, blocks, threads, iters, h->stream));
        cudaEventRecord(e1, h->stream);
        if (r == PNSCAN_OK) r = cuda_err(cudaEventSynchronize(e1));
        float ms = 0.f;
        if (r == PNSCAN_OK) cudaEventElapsedTime(&ms, e0, e1);
        if (r == PNSCAN_OK && ms > 0.f) {
            const double tf = 2.0 * 8.0 * (double)iters * threads * blocks / (ms * 1e-3) / 1e12;
            if (tf > best) best = tf;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    dev_free(h, buf);
    if (r != PNSCAN_OK) return r;
    *tflops = best;
    return PNSCAN_OK;
}

void scan_destroy(scan_handle* h)
{
    if (!h) return;
    if (h->stream || h->cap_stream) cudaStreamSynchronize(h->stream);
    if (h->gexec) cudaGraphExecDestroy(h->gexec);
    if (h->ev0) cudaEventDestroy(h->ev0);
    if (h->ev1) cudaEventDestroy(h->ev1);
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    dev_free(h, h->staging);
    dev_free(h, h->queue_block);
    dev_free(h, h->state_block);
    delete h;
}

const char* scan_strerror(int code)
{
    switch (code) {
    case PNSCAN_OK: return "ok";
    case PNSCAN_ERR_ARG: return "invalid argument";
    case PNSCAN_ERR_CUDA: return "CUDA runtime error";
    case PNSCAN_ERR_OOM: return "device allocation failed";
    case PNSCAN_ERR_TIMEOUT: return "host watchdog expired";
    case PNSCAN_ERR_STATE: return "call out of order (no state loaded)";
    case PNSCAN_ERR_KERNEL: return "device-side bounded wait gave up";
    case PNSCAN_ERR_NODEVICE: return "no CUDA device";
    default: return "unknown error";
    }
}

const char* scan_version(void) { return kVersion; }

}  // extern "C"
