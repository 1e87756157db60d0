// mlp_kernels.cu -- the scan surrogate and the adaptive scan's cell selection.
//
// Surrogate: an ensemble of K small networks mapping a scan cell's four
// parameters (x0, theta, mass ratio, chi) to its FLI,
//     h1 = tanh(W1 z + b1), h2 = tanh(W2 h1 + b2), y = w3 . h2 + b3,
// z the normalised inputs, 64 hidden units per layer.  BF16 operands with
// FP32 accumulation on the tensor cores (mma.sync m16n8k16) for the
// 64 x 64 contractions, FP32 master weights and Adam moments.  Training is one
// persistent CTA per member that runs every minibatch step (forward, backward,
// Adam) without leaving the kernel.  Minibatch rows are drawn with
// replacement by SplitMix64 (Steele, Lea & Flood 2014) of (seed, member,
// step, row).
//
// Selection: cells whose ensemble mean lies within `band` of the FLI
// threshold, or whose ensemble spread (max - min) exceeds `spread_max`, are
// compacted in index order (per-block counts, one scan, ordered writes) and
// their scan parameters gathered for the integrator.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "mlp_kernels.cuh"

namespace pnscan {
namespace mlp {

// ------------------------------------------------------------ constants
constexpr int TILE = 128;        // rows (cells or samples) per CTA
constexpr int LDB = NH + 8;      // padded bf16 row stride
constexpr int LDF = NH + 1;      // padded fp32 row stride

struct Smem {
    float W1[NH * NIN];
    float b1[NH];
    float b2[NH];
    float w3[NH];
    float b3;
    float z[TILE][NIN];
    float t[TILE];
    float d3[TILE];
    float err2[TILE];
    float H1f[TILE][LDF];
    float H2f[TILE][LDF];
    float D1f[TILE][LDF];
    float grad[NPARAM];
    __nv_bfloat16 W2b[NH][LDB];
    __nv_bfloat16 H1b[TILE][LDB];
    __nv_bfloat16 D2b[TILE][LDB];
};

size_t smem_bytes() { return sizeof(Smem); }

// Training keeps the member's fp32 master weights in shared memory for the
// whole run (the Adam moments live in registers) and reduces per-warp sums
// of the batch's squared errors and output errors.
struct TrainSmem {
    Smem s;
    float P[NPARAM];        // fp32 master weights of this member
    float err_part[TILE / 32];
    float d3_part[TILE / 32];
    float red_out[2][2][NH];           // output-layer / b2 gradient partials over two row halves
    float red_in[2][NIN + 1][NH];      // first-layer gradient partials over two row halves
};

size_t smem_train_bytes() { return sizeof(TrainSmem); }

constexpr int PER_THREAD = (NPARAM + TILE - 1) / TILE;   // parameters per thread in the Adam update

__device__ __forceinline__ uint64_t splitmix64(uint64_t x)
{
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}

__device__ __forceinline__ uint32_t pack2(__nv_bfloat16 lo, __nv_bfloat16 hi)
{
    return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

// A fragment of mma.m16n8k16 (row-major 16 x 16) from element (r, c) at
// base[(row0 + r) * sr + (k0 + c) * sc].
__device__ __forceinline__ void load_a(uint32_t a[4], const __nv_bfloat16* base, int sr, int sc, int row0,
                                       int k0, int lane)
{
    const int g = lane >> 2, q = lane & 3;
    auto el = [&](int r, int c) { return base[(row0 + r) * sr + (k0 + c) * sc]; };
    a[0] = pack2(el(g, 2 * q), el(g, 2 * q + 1));
    a[1] = pack2(el(g + 8, 2 * q), el(g + 8, 2 * q + 1));
    a[2] = pack2(el(g, 2 * q + 8), el(g, 2 * q + 9));
    a[3] = pack2(el(g + 8, 2 * q + 8), el(g + 8, 2 * q + 9));
}

// B fragment (16 x 8, "col") from element (k, n) at base[(k0 + k) * sk + (n0 + n) * sn].
__device__ __forceinline__ void load_b(uint32_t b[2], const __nv_bfloat16* base, int sk, int sn, int k0,
                                       int n0, int lane)
{
    const int g = lane >> 2, q = lane & 3;
    auto el = [&](int k, int n) { return base[(k0 + k) * sk + (n0 + n) * sn]; };
    b[0] = pack2(el(2 * q, g), el(2 * q + 1, g));
    b[1] = pack2(el(2 * q + 8, g), el(2 * q + 9, g));
}

__device__ __forceinline__ void mma16816(float c[4], const uint32_t a[4], const uint32_t b[2])
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// Positions of accumulator element i of a 16 x 8 tile for this lane.
__device__ __forceinline__ int c_row(int lane, int i) { return (lane >> 2) + (i >= 2 ? 8 : 0); }
__device__ __forceinline__ int c_col(int lane, int i) { return 2 * (lane & 3) + (i & 1); }

// Parameters of one member from global (fp32) into shared memory.
__device__ void load_params(Smem& s, const float* p)
{
    for (int i = threadIdx.x; i < NPARAM; i += blockDim.x) {
        const float v = p[i];
        if (i < OFF_B1) s.W1[i] = v;
        else if (i < OFF_W2) s.b1[i - OFF_B1] = v;
        else if (i < OFF_B2) {
            const int j = i - OFF_W2;
            s.W2b[j / NH][j % NH] = __float2bfloat16_rn(v);
        } else if (i < OFF_W3) s.b2[i - OFF_B2] = v;
        else if (i < OFF_B3) s.w3[i - OFF_W3] = v;
        else s.b3 = v;
    }
}

// Forward pass of the TILE rows held in s.z; fills H1f, H1b, H2f.  Row r's
// output is returned to thread r.
__device__ float forward_tile(Smem& s)
{
    const int r = threadIdx.x, lane = r & 31, warp = r >> 5;
    // layer 1 (K = 4): plain FP32
    for (int j = 0; j < NH; j++) {
        float a = s.b1[j];
#pragma unroll
        for (int i = 0; i < NIN; i++) a = fmaf(s.W1[j * NIN + i], s.z[r][i], a);
        const float h = tanhf(a);
        s.H1f[r][j] = h;
        s.H1b[r][j] = __float2bfloat16_rn(h);
    }
    __syncthreads();
    // layer 2: Z2[t][n] = sum_k H1[t][k] W2[n][k]; warp owns rows [32 warp, 32 warp + 32)
    float acc[2][8][4];
#pragma unroll
    for (int mt = 0; mt < 2; mt++)
#pragma unroll
        for (int nt = 0; nt < 8; nt++)
#pragma unroll
            for (int i = 0; i < 4; i++) acc[mt][nt][i] = 0.f;
#pragma unroll
    for (int kk = 0; kk < NH / 16; kk++) {
        uint32_t a[2][4];
#pragma unroll
        for (int mt = 0; mt < 2; mt++) load_a(a[mt], &s.H1b[0][0], LDB, 1, 32 * warp + 16 * mt, 16 * kk, lane);
#pragma unroll
        for (int nt = 0; nt < 8; nt++) {
            uint32_t b[2];
            load_b(b, &s.W2b[0][0], 1, LDB, 16 * kk, 8 * nt, lane);
#pragma unroll
            for (int mt = 0; mt < 2; mt++) mma16816(acc[mt][nt], a[mt], b);
        }
    }
#pragma unroll
    for (int mt = 0; mt < 2; mt++)
#pragma unroll
        for (int nt = 0; nt < 8; nt++)
#pragma unroll
            for (int i = 0; i < 4; i++) {
                const int row = 32 * warp + 16 * mt + c_row(lane, i), col = 8 * nt + c_col(lane, i);
                s.H2f[row][col] = tanhf(acc[mt][nt][i] + s.b2[col]);
            }
    __syncthreads();
    float y = s.b3;
    for (int n = 0; n < NH; n++) y = fmaf(s.w3[n], s.H2f[r][n], y);
    return y;
}

// ------------------------------------------------------------- training
__device__ __forceinline__ float warp_sum(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__global__ void __launch_bounds__(TILE) k_mlp_train(TrainArgs A)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TrainSmem& ts = *reinterpret_cast<TrainSmem*>(smem_raw);
    Smem& s = ts.s;
    const int member = blockIdx.x;
    const int r = threadIdx.x, lane = r & 31, warp = r >> 5;
    float* P = A.params + (size_t)member * NPARAM;
    float* M = A.adam_m + (size_t)member * NPARAM;
    float* V = A.adam_v + (size_t)member * NPARAM;
    const int nsteps = A.mode == 1 ? 1 : A.steps;

    // master weights to shared memory, this thread's Adam moments to registers
    // (parameter i = r + TILE k)
    float m_reg[PER_THREAD], v_reg[PER_THREAD];
#pragma unroll
    for (int k = 0; k < PER_THREAD; k++) {
        const int i = r + TILE * k;
        if (i < NPARAM) {
            ts.P[i] = P[i];
            m_reg[k] = M[i];
            v_reg[k] = V[i];
        }
    }
    __syncthreads();

    for (int step = 0; step < nsteps; step++) {
        load_params(s, ts.P);
        // minibatch rows
        long long idx;
        if (A.mode == 1) idx = r < A.N ? r : 0;
        else {
            const uint64_t h = splitmix64(A.seed ^ splitmix64(((uint64_t)member << 40) ^ ((uint64_t)(A.step0 + step) << 8) ^ (uint64_t)r));
            idx = (long long)(h % (uint64_t)A.N);
        }
#pragma unroll
        for (int i = 0; i < NIN; i++) s.z[r][i] = (A.X[idx * NIN + i] - A.center[i]) / A.scale[i];
        s.t[r] = A.Y[idx];
        __syncthreads();
        const float y = forward_tile(s);
        const float e = y - s.t[r];
        const float d3 = 2.f * e / (float)TILE;
        s.d3[r] = d3;
        s.err2[r] = e * e;
        {
            const float pe = warp_sum(e * e), pd = warp_sum(d3);
            if (lane == 0) {
                ts.err_part[warp] = pe;
                ts.d3_part[warp] = pd;
            }
        }
        for (int n = 0; n < NH; n++) {
            const float h2 = s.H2f[r][n];
            s.D2b[r][n] = __float2bfloat16_rn(d3 * s.w3[n] * (1.f - h2 * h2));
        }
        __syncthreads();
        // output layer and b2 gradients (reductions over the batch): thread r
        // sums unit r % NH over half r / NH of the rows; halves combined below
        {
            static_assert(TILE == 2 * NH, "two row halves per hidden unit");
            const int u = r % NH, half = r / NH;
            float gw3 = 0.f, gb2 = 0.f;
            for (int t = half * (TILE / 2); t < (half + 1) * (TILE / 2); t++) {
                gw3 = fmaf(s.d3[t], s.H2f[t][u], gw3);
                gb2 += __bfloat162float(s.D2b[t][u]);
            }
            ts.red_out[half][0][u] = gw3;
            ts.red_out[half][1][u] = gb2;
        }
        // gW2[n][k] = sum_t D2[t][n] H1[t][k]: M = 64 (n), N = 64 (k), K = 128 (t); warp owns n-rows [16 warp, +16)
        {
            float acc[8][4];
#pragma unroll
            for (int nt = 0; nt < 8; nt++)
#pragma unroll
                for (int i = 0; i < 4; i++) acc[nt][i] = 0.f;
#pragma unroll
            for (int kk = 0; kk < TILE / 16; kk++) {
                uint32_t a[4];
                load_a(a, &s.D2b[0][0], 1, LDB, 16 * warp, 16 * kk, lane);     // (n, t) -> D2b[t][n]
#pragma unroll
                for (int nt = 0; nt < 8; nt++) {
                    uint32_t b[2];
                    load_b(b, &s.H1b[0][0], LDB, 1, 16 * kk, 8 * nt, lane);    // (t, k) -> H1b[t][k]
                    mma16816(acc[nt], a, b);
                }
            }
#pragma unroll
            for (int nt = 0; nt < 8; nt++)
#pragma unroll
                for (int i = 0; i < 4; i++) {
                    const int n = 16 * warp + c_row(lane, i), k = 8 * nt + c_col(lane, i);
                    s.grad[OFF_W2 + n * NH + k] = acc[nt][i];
                }
        }
        // D1[t][k] = (sum_n D2[t][n] W2[n][k]) (1 - H1[t][k]^2): M = 128, N = 64, K = 64
        {
            float acc[2][8][4];
#pragma unroll
            for (int mt = 0; mt < 2; mt++)
#pragma unroll
                for (int nt = 0; nt < 8; nt++)
#pragma unroll
                    for (int i = 0; i < 4; i++) acc[mt][nt][i] = 0.f;
#pragma unroll
            for (int kk = 0; kk < NH / 16; kk++) {
                uint32_t a[2][4];
#pragma unroll
                for (int mt = 0; mt < 2; mt++) load_a(a[mt], &s.D2b[0][0], LDB, 1, 32 * warp + 16 * mt, 16 * kk, lane);
#pragma unroll
                for (int nt = 0; nt < 8; nt++) {
                    uint32_t b[2];
                    load_b(b, &s.W2b[0][0], LDB, 1, 16 * kk, 8 * nt, lane);    // (n, k) -> W2b[n][k]
#pragma unroll
                    for (int mt = 0; mt < 2; mt++) mma16816(acc[mt][nt], a[mt], b);
                }
            }
#pragma unroll
            for (int mt = 0; mt < 2; mt++)
#pragma unroll
                for (int nt = 0; nt < 8; nt++)
#pragma unroll
                    for (int i = 0; i < 4; i++) {
                        const int row = 32 * warp + 16 * mt + c_row(lane, i), col = 8 * nt + c_col(lane, i);
                        const float h1 = s.H1f[row][col];
                        s.D1f[row][col] = acc[mt][nt][i] * (1.f - h1 * h1);
                    }
        }
        __syncthreads();
        // first-layer gradients: gW1[j][i] = sum_t D1[t][j] z[t][i], gb1[j] = sum_t D1[t][j];
        // thread r sums unit r % NH over half r / NH of the rows
        {
            const int j = r % NH, half = r / NH;
            float g[NIN + 1];
#pragma unroll
            for (int i = 0; i <= NIN; i++) g[i] = 0.f;
            for (int t = half * (TILE / 2); t < (half + 1) * (TILE / 2); t++) {
                const float d = s.D1f[t][j];
#pragma unroll
                for (int i = 0; i < NIN; i++) g[i] = fmaf(d, s.z[t][i], g[i]);
                g[NIN] += d;
            }
#pragma unroll
            for (int i = 0; i <= NIN; i++) ts.red_in[half][i][j] = g[i];
        }
        __syncthreads();
        // combine the two row halves
        if (r < NH) {
            s.grad[OFF_W3 + r] = ts.red_out[0][0][r] + ts.red_out[1][0][r];
            s.grad[OFF_B2 + r] = ts.red_out[0][1][r] + ts.red_out[1][1][r];
#pragma unroll
            for (int i = 0; i < NIN; i++) s.grad[OFF_W1 + r * NIN + i] = ts.red_in[0][i][r] + ts.red_in[1][i][r];
            s.grad[OFF_B1 + r] = ts.red_in[0][NIN][r] + ts.red_in[1][NIN][r];
        } else if (r == NH) {
            float gb3 = 0.f;
#pragma unroll
            for (int w = 0; w < TILE / 32; w++) gb3 += ts.d3_part[w];
            s.grad[OFF_B3] = gb3;
        }
        __syncthreads();
        if (A.mode == 1) {
            for (int i = r; i < NPARAM; i += TILE) A.grad_out[(size_t)member * NPARAM + i] = s.grad[i];
            if (r == 0) {
                float l = 0.f;
#pragma unroll
                for (int w = 0; w < TILE / 32; w++) l += ts.err_part[w];
                A.loss_out[member] = l / (float)TILE;
            }
            return;
        }
        // Adam (Kingma & Ba 2015), bias-corrected moments
        const int tstep = A.step0 + step + 1;
        const float c1 = 1.f - powf(0.9f, (float)tstep), c2 = 1.f - powf(0.999f, (float)tstep);
#pragma unroll
        for (int k = 0; k < PER_THREAD; k++) {
            const int i = r + TILE * k;
            if (i < NPARAM) {
                const float g = s.grad[i];
                const float m = 0.9f * m_reg[k] + 0.1f * g;
                const float v = 0.999f * v_reg[k] + 0.001f * g * g;
                m_reg[k] = m;
                v_reg[k] = v;
                ts.P[i] = ts.P[i] - A.lr * (m / c1) / (sqrtf(v / c2) + 1e-8f);
            }
        }
        if (A.loss_hist && r == 0) {
            float l = 0.f;
#pragma unroll
            for (int w = 0; w < TILE / 32; w++) l += ts.err_part[w];
            A.loss_hist[(size_t)member * A.steps + step] = l / (float)TILE;
        }
        __syncthreads();
    }
    // the trained weights and moments back to the handle
#pragma unroll
    for (int k = 0; k < PER_THREAD; k++) {
        const int i = r + TILE * k;
        if (i < NPARAM) {
            P[i] = ts.P[i];
            M[i] = m_reg[k];
            V[i] = v_reg[k];
        }
    }
}

// ------------------------------------------------------------ inference
__global__ void __launch_bounds__(TILE) k_mlp_predict(PredictArgs A)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Smem& s = *reinterpret_cast<Smem*>(smem_raw);
    const int r = threadIdx.x;
    const long long cell = (long long)blockIdx.x * TILE + r;
    const long long c = cell < A.N ? cell : A.N - 1;
    float sum = 0.f, lo = 3.4e38f, hi = -3.4e38f;
    for (int k = 0; k < A.members; k++) {
        load_params(s, A.params + (size_t)k * NPARAM);
#pragma unroll
        for (int i = 0; i < NIN; i++) s.z[r][i] = (A.X[c * NIN + i] - A.center[i]) / A.scale[i];
        __syncthreads();
        const float y = forward_tile(s);
        sum += y;
        lo = fminf(lo, y);
        hi = fmaxf(hi, y);
        __syncthreads();
    }
    if (cell < A.N) {
        A.mean[cell] = sum / (float)A.members;
        A.spread[cell] = hi - lo;
    }
}

// --------------------------------------------------------- initialisation
// Xavier-uniform weights (bound sqrt(6 / (fan_in + fan_out))), zero biases,
// zero Adam moments.
__global__ void k_mlp_init(float* params, float* m, float* v, int members, uint64_t seed)
{
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= (long long)members * NPARAM) return;
    const int j = (int)(i % NPARAM);
    const int member = (int)(i / NPARAM);
    float bound = 0.f;
    if (j < OFF_B1) bound = sqrtf(6.f / (NIN + NH));
    else if (j >= OFF_W2 && j < OFF_B2) bound = sqrtf(6.f / (NH + NH));
    else if (j >= OFF_W3 && j < OFF_B3) bound = sqrtf(6.f / (NH + 1));
    const uint64_t h = splitmix64(seed ^ splitmix64(((uint64_t)member << 32) ^ (uint64_t)j));
    const float u = (float)((h >> 40) * (1.0 / 16777216.0));            // [0, 1)
    params[i] = bound * (2.f * u - 1.f);
    m[i] = 0.f;
    v[i] = 0.f;
}

// ------------------------------------------------------------- selection
__device__ __forceinline__ bool selected(const SelectArgs& A, long long i)
{
    const float mu = A.mean[i];
    return fabsf(mu - A.thr) <= A.band || A.spread[i] > A.spread_max || !(mu == mu);
}

__global__ void k_select_count(SelectArgs A, int* block_counts)
{
    __shared__ int warp_counts[8];
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const bool f = i < A.N && selected(A, i);
    const unsigned m = __ballot_sync(0xffffffffu, f);
    if ((threadIdx.x & 31) == 0) warp_counts[threadIdx.x >> 5] = __popc(m);
    __syncthreads();
    if (threadIdx.x == 0) {
        int c = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) c += warp_counts[w];
        block_counts[blockIdx.x] = c;
    }
}

// Exclusive scan of the block counts by one block (nblocks <= SELECT_MAX_BLOCKS).
__global__ void k_select_scan(int* block_counts, int nblocks, long long* total)
{
    __shared__ int part[1024];
    const int t = threadIdx.x;
    const int per = (nblocks + 1023) / 1024;
    int sum = 0;
    for (int b = t * per; b < (t + 1) * per && b < nblocks; b++) sum += block_counts[b];
    part[t] = sum;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {
        const int v = t >= off ? part[t - off] : 0;
        __syncthreads();
        part[t] += v;
        __syncthreads();
    }
    int run = t > 0 ? part[t - 1] : 0;
    for (int b = t * per; b < (t + 1) * per && b < nblocks; b++) {
        const int c = block_counts[b];
        block_counts[b] = run;
        run += c;
    }
    if (t == 1023) *total = part[1023];
}

__global__ void k_select_write(SelectArgs A, const int* block_offsets)
{
    __shared__ int warp_off[8];
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const bool f = i < A.N && selected(A, i);
    const unsigned m = __ballot_sync(0xffffffffu, f);
    if (lane == 0) warp_off[warp] = __popc(m);
    __syncthreads();
    if (threadIdx.x == 0) {
        int run = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) {
            const int c = warp_off[w];
            warp_off[w] = run;
            run += c;
        }
    }
    __syncthreads();
    if (f) {
        const long long pos = block_offsets[blockIdx.x] + warp_off[warp] + __popc(m & ((1u << lane) - 1u));
        A.idx[pos] = (int32_t)i;
        if (A.cells && A.cells_out) {
#pragma unroll
            for (int k = 0; k < 9; k++) A.cells_out[pos * 9 + k] = A.cells[i * 9 + k];
        }
    }
}

// Class map: a selected cell takes the integrator's result (chaotic if it
// reached t_end or saturated with FLI > thr), any other cell the surrogate's
// mean (chaotic if > thr).  cls: 1 chaotic, 0 not.
__global__ void k_merge(MergeArgs A)
{
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < A.N) A.cls[i] = A.mean[i] > A.thr ? 1 : 0;
}

__global__ void k_merge_selected(MergeArgs A)
{
    const long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (j >= A.count) return;
    const int st = A.status[j];
    const bool chaotic = (st == 1 || st == 4) && A.fli[j] > A.thr;
    A.cls[A.idx[j]] = chaotic ? 1 : 0;
}

// Surrogate inputs of scan cells: (x0, theta1, beta, chi1) as float.
__global__ void k_features(const double* cells, long long n, float* X)
{
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    X[4 * i + 0] = (float)cells[9 * i + 0];
    X[4 * i + 1] = (float)cells[9 * i + 2];
    X[4 * i + 2] = (float)cells[9 * i + 6];
    X[4 * i + 3] = (float)cells[9 * i + 7];
}

// Features from any four of a cell's nine fields.
__global__ void k_features_fields(const double* cells, long long n, FieldSel f, float* X)
{
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
#pragma unroll
    for (int k = 0; k < NIN; k++) X[NIN * i + k] = (float)cells[9 * i + f.field[k]];
}

// No-learning map of a row-major n1 x n2 grid from an integrated coarse grid
// of every stride-th cell in both directions (nc1 x nc2 nodes, node (a, b) at
// cell (a stride, b stride)): the FLI interpolated bilinearly between the
// four surrounding nodes (clamped beyond the last node), and the spread of
// those four values (max - min) as the uncertainty.  A node counts with its
// FLI when it finished (DONE) or saturated, else as 0 (not chaotic).  A cell
// that is itself a node takes the node's FLI and spread 0.
__global__ void k_interp_grid(InterpArgs A)
{
    const long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (c >= A.n1 * A.n2) return;
    const long long i = c / A.n2, j = c % A.n2;
    const long long a0 = i / A.stride, b0 = j / A.stride;
    const long long a1 = a0 + 1 < A.nc1 ? a0 + 1 : a0, b1 = b0 + 1 < A.nc2 ? b0 + 1 : b0;
    const float wa = a1 > a0 ? (float)(i - a0 * A.stride) / (float)A.stride : 0.f;
    const float wb = b1 > b0 ? (float)(j - b0 * A.stride) / (float)A.stride : 0.f;
    auto node = [&](long long a, long long b) {
        const long long k = a * A.nc2 + b;
        const int st = A.status[k];
        return (st == 1 || st == 4) ? (float)A.fli[k] : 0.f;
    };
    const float v00 = node(a0, b0), v01 = node(a0, b1), v10 = node(a1, b0), v11 = node(a1, b1);
    const float lo = fminf(fminf(v00, v01), fminf(v10, v11)), hi = fmaxf(fmaxf(v00, v01), fmaxf(v10, v11));
    const bool is_node = (i % A.stride == 0) && (j % A.stride == 0);
    const float top = fmaf(wb, v01 - v00, v00), bot = fmaf(wb, v11 - v10, v10);
    A.mean[c] = is_node ? v00 : fmaf(wa, bot - top, top);
    A.spread[c] = is_node ? 0.f : hi - lo;
}

// -------------------------------------------------------------- launchers
cudaError_t launch_features_fields(const double* cells, long long n, FieldSel f, float* X, cudaStream_t st)
{
    if (n > 0) k_features_fields<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(cells, n, f, X);
    return cudaGetLastError();
}

cudaError_t launch_interp_grid(const InterpArgs& A, cudaStream_t st)
{
    const long long n = A.n1 * A.n2;
    if (n > 0) k_interp_grid<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(A);
    return cudaGetLastError();
}

cudaError_t launch_features(const double* cells, long long n, float* X, cudaStream_t st)
{
    if (n > 0) k_features<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(cells, n, X);
    return cudaGetLastError();
}

cudaError_t launch_init(float* params, float* m, float* v, int members, uint64_t seed, cudaStream_t st)
{
    const long long n = (long long)members * NPARAM;
    k_mlp_init<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(params, m, v, members, seed);
    return cudaGetLastError();
}

cudaError_t launch_train(const TrainArgs& A, int members, cudaStream_t st)
{
    const size_t sm = smem_train_bytes();
    cudaError_t e = cudaFuncSetAttribute(k_mlp_train, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    k_mlp_train<<<members, TILE, sm, st>>>(A);
    return cudaGetLastError();
}

cudaError_t launch_predict(const PredictArgs& A, cudaStream_t st)
{
    if (A.N == 0) return cudaSuccess;
    const size_t sm = smem_bytes();
    cudaError_t e = cudaFuncSetAttribute(k_mlp_predict, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    k_mlp_predict<<<(unsigned)((A.N + TILE - 1) / TILE), TILE, sm, st>>>(A);
    return cudaGetLastError();
}

size_t select_workspace_bytes(long long n)
{
    const long long nb = (n + 255) / 256;
    return (size_t)((nb + 1) * sizeof(int) + 2 * sizeof(long long) + 256);
}

cudaError_t launch_select(const SelectArgs& A, void* ws, long long* d_total, cudaStream_t st)
{
    const long long nb = (A.N + 255) / 256;
    if (nb > SELECT_MAX_BLOCKS) return cudaErrorInvalidValue;
    int* counts = (int*)ws;
    if (A.N == 0) return cudaMemsetAsync(d_total, 0, sizeof(long long), st);
    k_select_count<<<(unsigned)nb, 256, 0, st>>>(A, counts);
    k_select_scan<<<1, 1024, 0, st>>>(counts, (int)nb, d_total);
    k_select_write<<<(unsigned)nb, 256, 0, st>>>(A, counts);
    return cudaGetLastError();
}

cudaError_t launch_merge(const MergeArgs& A, cudaStream_t st)
{
    if (A.N > 0) k_merge<<<(unsigned)((A.N + 255) / 256), 256, 0, st>>>(A);
    if (A.count > 0) k_merge_selected<<<(unsigned)((A.count + 255) / 256), 256, 0, st>>>(A);
    return cudaGetLastError();
}

}  // namespace mlp
}  // namespace pnscan
