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
constexpr int LDT = NH + 8;      // fp32 row stride of the training arrays written from MMA fragments
                                 // (8-byte pairs of a half-warp land in distinct banks)

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

// Training: one CTA of NT threads (8 warps, two per SM sub-partition) per
// member.  The member's fp32 master weights stay in shared memory for the
// whole run, with a bfloat16 copy of W2 that the Adam update refreshes; the
// Adam moments live in registers.  The output layer is folded into the
// epilogue of the second layer's contraction (row sums by warp shuffles), so
// the second hidden layer never goes to shared memory.
constexpr int NT = 256;
constexpr int NWT = NT / 32;

struct TrainSmem {
    float P[NPARAM];                   // fp32 master weights of this member
    alignas(16) float gW2[NH][LDT];    // gradient of W2, [n][k]
    float gout[2][NH];                 // gradients of w3 and b2
    float z[TILE][NIN];
    float t[TILE];
    alignas(16) float H1f[TILE][LDT];
    alignas(16) float D1f[TILE][LDT];
    alignas(16) __nv_bfloat16 W2b[NH][LDB];   // 16-byte aligned rows for ldmatrix
    alignas(16) __nv_bfloat16 H1b[TILE][LDB];
    alignas(16) __nv_bfloat16 D2b[TILE][LDB];
    float red_out[NWT][2][NH];         // per-warp partials of the w3 and b2 gradients
    float red_in[4][NIN + 1][NH];      // first-layer gradient partials over four row quarters
    float err_part[NWT];
    float d3_part[NWT];
    float gb3, loss;
};

size_t smem_train_bytes() { return sizeof(TrainSmem); }

constexpr int PER_THREAD = (NPARAM + NT - 1) / NT;   // parameters per thread in the Adam update

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

// The same fragments by ldmatrix (four 8 x 8 b16 matrices per instruction,
// one 16-byte row address per lane; rows must be 16-byte aligned).  `ld` is
// the row stride of the shared array in elements.
__device__ __forceinline__ void ldsm_x4(uint32_t r[4], const __nv_bfloat16* p)
{
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]) : "r"(a));
}

__device__ __forceinline__ void ldsm_x4_t(uint32_t r[4], const __nv_bfloat16* p)
{
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]) : "r"(a));
}

// A fragment of the 16 x 16 tile at (m0, k0) of A stored [m][k] (k contiguous).
__device__ __forceinline__ void ldsm_a(uint32_t a[4], const __nv_bfloat16* S, int ld, int m0, int k0, int lane)
{
    const int mi = lane >> 3, rr = lane & 7;
    ldsm_x4(a, S + (m0 + rr + 8 * (mi & 1)) * ld + k0 + 8 * (mi >> 1));
}

// A fragment of the tile at (m0, k0) of A stored transposed, S[k][m] (m contiguous).
__device__ __forceinline__ void ldsm_a_t(uint32_t a[4], const __nv_bfloat16* S, int ld, int m0, int k0, int lane)
{
    const int mi = lane >> 3, rr = lane & 7;
    ldsm_x4_t(a, S + (k0 + rr + 8 * (mi >> 1)) * ld + m0 + 8 * (mi & 1));
}

// B fragments of two adjacent 16 x 8 tiles at (k0, n0) and (k0, n0 + 8) of B
// stored S[n][k] (k contiguous): b[0..1] the first tile, b[2..3] the second.
__device__ __forceinline__ void ldsm_b2(uint32_t b[4], const __nv_bfloat16* S, int ld, int k0, int n0, int lane)
{
    const int mi = lane >> 3, rr = lane & 7;
    ldsm_x4(b, S + (n0 + rr + 8 * (mi >> 1)) * ld + k0 + 8 * (mi & 1));
}

// The same for B stored S[k][n] (n contiguous).
__device__ __forceinline__ void ldsm_b2_t(uint32_t b[4], const __nv_bfloat16* S, int ld, int k0, int n0, int lane)
{
    const int mi = lane >> 3, rr = lane & 7;
    ldsm_x4_t(b, S + (k0 + rr + 8 * (mi & 1)) * ld + n0 + 8 * (mi >> 1));
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

// Row of minibatch slot r at Adam step `step` of this launch: SplitMix64 of
// (seed, member, step0 + step, r) modulo N (mode 0); rows 0..TILE-1 in
// order (mode 1, clamped to row 0 past N).
__device__ __forceinline__ long long batch_row(const TrainArgs& A, int member, int step, int r)
{
    if (A.mode == 1) return r < A.N ? r : 0;
    const uint64_t h = splitmix64(A.seed ^ splitmix64(((uint64_t)member << 40) ^ ((uint64_t)(A.step0 + step) << 8) ^ (uint64_t)r));
    return (long long)(h % (uint64_t)A.N);
}

// Gradient of parameter i once a step's reductions are complete: the
// first layer's from its four row-quarter partials, the rest as stored.
__device__ __forceinline__ float grad_at(const TrainSmem& ts, int i)
{
    if (i < OFF_W2) {
        const int j = i < OFF_B1 ? i / NIN : i - OFF_B1;
        const int c = i < OFF_B1 ? i % NIN : NIN;
        return ((ts.red_in[0][c][j] + ts.red_in[1][c][j]) + ts.red_in[2][c][j]) + ts.red_in[3][c][j];
    }
    if (i < OFF_B2) return ts.gW2[(i - OFF_W2) / NH][(i - OFF_W2) % NH];
    if (i < OFF_W3) return ts.gout[1][i - OFF_B2];
    if (i < OFF_B3) return ts.gout[0][i - OFF_W3];
    return ts.gb3;
}

__global__ void __launch_bounds__(NT) k_mlp_train(TrainArgs A)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TrainSmem& ts = *reinterpret_cast<TrainSmem*>(smem_raw);
    const int member = blockIdx.x;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int g = lane >> 2, q = lane & 3;
    float* P = A.params + (size_t)member * NPARAM;
    float* M = A.adam_m + (size_t)member * NPARAM;
    float* V = A.adam_v + (size_t)member * NPARAM;
    const int nsteps = A.mode == 1 ? 1 : A.steps;
    const float* W1 = ts.P + OFF_W1;
    const float* b1 = ts.P + OFF_B1;
    const float* b2 = ts.P + OFF_B2;
    const float* w3 = ts.P + OFF_W3;

    // master weights (and the bfloat16 W2) to shared memory, this thread's
    // Adam moments to registers (parameter i = tid + NT k)
    float m_reg[PER_THREAD], v_reg[PER_THREAD];
#pragma unroll
    for (int k = 0; k < PER_THREAD; k++) {
        const int i = tid + NT * k;
        if (i < NPARAM) {
            const float p = P[i];
            ts.P[i] = p;
            if (i >= OFF_W2 && i < OFF_B2) ts.W2b[(i - OFF_W2) / NH][(i - OFF_W2) % NH] = __float2bfloat16_rn(p);
            m_reg[k] = M[i];
            v_reg[k] = V[i];
        }
    }
    // the first minibatch row of slot tid; later rows are fetched one step ahead
    float xr[NIN], yr = 0.f;
    if (tid < TILE) {
        const long long idx = batch_row(A, member, 0, tid);
#pragma unroll
        for (int i = 0; i < NIN; i++) xr[i] = A.X[idx * NIN + i];
        yr = A.Y[idx];
    }

    for (int step = 0; step < nsteps; step++) {
        // (1) this step's rows to shared memory, the next step's loads issued
        if (tid < TILE) {
#pragma unroll
            for (int i = 0; i < NIN; i++) ts.z[tid][i] = (xr[i] - A.center[i]) / A.scale[i];
            ts.t[tid] = yr;
            if (step + 1 < nsteps) {
                const long long idx = batch_row(A, member, step + 1, tid);
#pragma unroll
                for (int i = 0; i < NIN; i++) xr[i] = A.X[idx * NIN + i];
                yr = A.Y[idx];
            }
        }
        __syncthreads();
        // (2) layer 1 (K = 4, plain FP32): lane <-> hidden unit, warp <-> 32 rows
        {
            const int j = lane + 32 * (warp & 1);
            float wj[NIN];
#pragma unroll
            for (int i = 0; i < NIN; i++) wj[i] = W1[j * NIN + i];
            const float bj = b1[j];
            const int row0 = 32 * (warp >> 1);
            for (int row = row0; row < row0 + 32; row++) {
                float a = bj;
#pragma unroll
                for (int i = 0; i < NIN; i++) a = fmaf(wj[i], ts.z[row][i], a);
                const float h = tanhf(a);
                ts.H1f[row][j] = h;
                ts.H1b[row][j] = __float2bfloat16_rn(h);
            }
        }
        __syncthreads();
        // (3) layer 2 and the output: Z2[t][n] = sum_k H1[t][k] W2[n][k], warp
        // owns rows [16 warp, +16); h2 = tanh(Z2 + b2) stays in registers
        {
            const int R0 = 16 * warp;
            float acc[8][4];
#pragma unroll
            for (int nt = 0; nt < 8; nt++)
#pragma unroll
                for (int i = 0; i < 4; i++) acc[nt][i] = 0.f;
#pragma unroll
            for (int kk = 0; kk < NH / 16; kk++) {
                uint32_t a[4];
                ldsm_a(a, &ts.H1b[0][0], LDB, R0, 16 * kk, lane);
#pragma unroll
                for (int nt = 0; nt < 8; nt += 2) {
                    uint32_t b[4];
                    ldsm_b2(b, &ts.W2b[0][0], LDB, 16 * kk, 8 * nt, lane);     // (k, n) -> W2b[n][k]
                    mma16816(acc[nt], a, b);
                    mma16816(acc[nt + 1], a, b + 2);
                }
            }
            // elements i = 0, 1 are row R0 + g, i = 2, 3 row R0 + g + 8; columns 8 nt + 2 q + (i & 1)
            float ya = 0.f, yb = 0.f;
#pragma unroll
            for (int nt = 0; nt < 8; nt++)
#pragma unroll
                for (int i = 0; i < 4; i++) {
                    const int col = 8 * nt + c_col(lane, i);
                    const float h = tanhf(acc[nt][i] + b2[col]);
                    acc[nt][i] = h;
                    if (i < 2) ya = fmaf(w3[col], h, ya);
                    else yb = fmaf(w3[col], h, yb);
                }
            ya += __shfl_xor_sync(0xffffffffu, ya, 1);
            ya += __shfl_xor_sync(0xffffffffu, ya, 2);
            yb += __shfl_xor_sync(0xffffffffu, yb, 1);
            yb += __shfl_xor_sync(0xffffffffu, yb, 2);
            const float b3 = ts.P[OFF_B3];
            const float ea = (ya + b3) - ts.t[R0 + g], eb = (yb + b3) - ts.t[R0 + g + 8];
            const float d3a = 2.f * ea / (float)TILE, d3b = 2.f * eb / (float)TILE;
            // output-layer error through tanh: D2 = d3 w3 (1 - h2^2), rounded to bfloat16
            // for the two contractions below; w3 and b2 gradient partials over the warp's rows
            float pw[8][2], pb[8][2];
#pragma unroll
            for (int nt = 0; nt < 8; nt++) {
                const int c0 = 8 * nt + 2 * q;
                const float ha0 = acc[nt][0], ha1 = acc[nt][1], hb0 = acc[nt][2], hb1 = acc[nt][3];
                const __nv_bfloat16 da0 = __float2bfloat16_rn(d3a * w3[c0] * (1.f - ha0 * ha0));
                const __nv_bfloat16 da1 = __float2bfloat16_rn(d3a * w3[c0 + 1] * (1.f - ha1 * ha1));
                const __nv_bfloat16 db0 = __float2bfloat16_rn(d3b * w3[c0] * (1.f - hb0 * hb0));
                const __nv_bfloat16 db1 = __float2bfloat16_rn(d3b * w3[c0 + 1] * (1.f - hb1 * hb1));
                *reinterpret_cast<uint32_t*>(&ts.D2b[R0 + g][c0]) = pack2(da0, da1);
                *reinterpret_cast<uint32_t*>(&ts.D2b[R0 + g + 8][c0]) = pack2(db0, db1);
                pw[nt][0] = fmaf(d3b, hb0, d3a * ha0);
                pw[nt][1] = fmaf(d3b, hb1, d3a * ha1);
                pb[nt][0] = __bfloat162float(da0) + __bfloat162float(db0);
                pb[nt][1] = __bfloat162float(da1) + __bfloat162float(db1);
            }
            // sums over the warp's 8 row pairs (lanes of equal q) by recursive
            // halving: at lane-mask bit b the lane keeps the half of its 2^(3-b) x 2
            // partials selected by bit b of g and adds its partner's; afterwards it
            // holds the sums of partial index c = 2 nt + j with c >> 1 =
            // 4 (g & 1) + 2 ((g >> 1) & 1) + ((g >> 2) & 1)
            float* vw = &pw[0][0];
            float* vb = &pb[0][0];
#pragma unroll
            for (int lvl = 0, half = 8; lvl < 3; lvl++, half >>= 1) {
                const bool hi = (g >> lvl) & 1;
#pragma unroll
                for (int i = 0; i < half; i++) {
                    const float sw = __shfl_xor_sync(0xffffffffu, hi ? vw[i] : vw[i + half], 4 << lvl);
                    const float sb = __shfl_xor_sync(0xffffffffu, hi ? vb[i] : vb[i + half], 4 << lvl);
                    vw[i] = (hi ? vw[i + half] : vw[i]) + sw;
                    vb[i] = (hi ? vb[i + half] : vb[i]) + sb;
                }
            }
            {
                const int nt = 4 * (g & 1) + 2 * ((g >> 1) & 1) + ((g >> 2) & 1);
#pragma unroll
                for (int j = 0; j < 2; j++) {
                    ts.red_out[warp][0][8 * nt + 2 * q + j] = vw[j];
                    ts.red_out[warp][1][8 * nt + 2 * q + j] = vb[j];
                }
            }
            const float le = warp_sum(q == 0 ? fmaf(ea, ea, eb * eb) : 0.f);
            const float ld = warp_sum(q == 0 ? d3a + d3b : 0.f);
            if (lane == 0) {
                ts.err_part[warp] = le;
                ts.d3_part[warp] = ld;
            }
        }
        __syncthreads();
        // (4) gW2[n][k] = sum_t D2[t][n] H1[t][k] (M = 64 n, N = 64 k, K = 128 t; warp owns
        // n-rows [16 (warp & 3), +16) and k-columns [32 (warp >> 2), +32)), then
        // D1[t][k] = (sum_n D2[t][n] W2[n][k]) (1 - H1[t][k]^2) (M = 128 t, N = 64 k, K = 64 n;
        // warp owns rows [16 warp, +16))
        {
            const int n0 = 16 * (warp & 3), nt0 = 4 * (warp >> 2);
            float acc[4][4];
#pragma unroll
            for (int nt = 0; nt < 4; nt++)
#pragma unroll
                for (int i = 0; i < 4; i++) acc[nt][i] = 0.f;
#pragma unroll
            for (int kk = 0; kk < TILE / 16; kk++) {
                uint32_t a[4];
                ldsm_a_t(a, &ts.D2b[0][0], LDB, n0, 16 * kk, lane);              // (n, t) -> D2b[t][n]
#pragma unroll
                for (int nt = 0; nt < 4; nt += 2) {
                    uint32_t b[4];
                    ldsm_b2_t(b, &ts.H1b[0][0], LDB, 16 * kk, 8 * (nt0 + nt), lane);   // (t, k) -> H1b[t][k]
                    mma16816(acc[nt], a, b);
                    mma16816(acc[nt + 1], a, b + 2);
                }
            }
            // accumulator pairs (i, i + 1) are adjacent columns of one row
#pragma unroll
            for (int nt = 0; nt < 4; nt++)
#pragma unroll
                for (int i = 0; i < 4; i += 2)
                    *reinterpret_cast<float2*>(&ts.gW2[n0 + c_row(lane, i)][8 * (nt0 + nt) + c_col(lane, i)]) =
                        make_float2(acc[nt][i], acc[nt][i + 1]);
        }
        {
            const int R0 = 16 * warp;
            float acc[8][4];
#pragma unroll
            for (int nt = 0; nt < 8; nt++)
#pragma unroll
                for (int i = 0; i < 4; i++) acc[nt][i] = 0.f;
#pragma unroll
            for (int kk = 0; kk < NH / 16; kk++) {
                uint32_t a[4];
                ldsm_a(a, &ts.D2b[0][0], LDB, R0, 16 * kk, lane);
#pragma unroll
                for (int nt = 0; nt < 8; nt += 2) {
                    uint32_t b[4];
                    ldsm_b2_t(b, &ts.W2b[0][0], LDB, 16 * kk, 8 * nt, lane);   // (n, k) -> W2b[n][k]
                    mma16816(acc[nt], a, b);
                    mma16816(acc[nt + 1], a, b + 2);
                }
            }
#pragma unroll
            for (int nt = 0; nt < 8; nt++)
#pragma unroll
                for (int i = 0; i < 4; i += 2) {
                    const int row = R0 + c_row(lane, i), col = 8 * nt + c_col(lane, i);
                    const float2 h1 = *reinterpret_cast<const float2*>(&ts.H1f[row][col]);
                    *reinterpret_cast<float2*>(&ts.D1f[row][col]) =
                        make_float2(acc[nt][i] * (1.f - h1.x * h1.x), acc[nt][i + 1] * (1.f - h1.y * h1.y));
                }
        }
        // w3 and b2 gradients over the warps' partials; b3 and the loss
        if (tid < 2 * NH) {
            const int col = tid & (NH - 1), which = tid >> 6;
            float s = 0.f;
#pragma unroll
            for (int w = 0; w < NWT; w++) s += ts.red_out[w][which][col];
            ts.gout[which][col] = s;
        } else if (tid == 2 * NH) {
            float gb3 = 0.f, l = 0.f;
#pragma unroll
            for (int w = 0; w < NWT; w++) {
                gb3 += ts.d3_part[w];
                l += ts.err_part[w];
            }
            ts.gb3 = gb3;
            ts.loss = l / (float)TILE;
        }
        __syncthreads();
        // (5) first-layer gradients: gW1[j][i] = sum_t D1[t][j] z[t][i], gb1[j] = sum_t D1[t][j];
        // thread sums unit tid % 64 over row quarter tid / 64
        {
            const int j = tid & (NH - 1), quarter = tid >> 6;
            float gz[NIN + 1];
#pragma unroll
            for (int i = 0; i <= NIN; i++) gz[i] = 0.f;
            for (int t = quarter * (TILE / 4); t < (quarter + 1) * (TILE / 4); t++) {
                const float d = ts.D1f[t][j];
#pragma unroll
                for (int i = 0; i < NIN; i++) gz[i] = fmaf(d, ts.z[t][i], gz[i]);
                gz[NIN] += d;
            }
#pragma unroll
            for (int i = 0; i <= NIN; i++) ts.red_in[quarter][i][j] = gz[i];
        }
        __syncthreads();
        if (A.mode == 1) {
            for (int i = tid; i < NPARAM; i += NT) A.grad_out[(size_t)member * NPARAM + i] = grad_at(ts, i);
            if (tid == 0) A.loss_out[member] = ts.loss;
            return;
        }
        // (6) Adam (Kingma & Ba 2015), bias-corrected moments; the bfloat16 W2
        // follows its master weight.  The next step's first shared-memory
        // reads of P and W2b come after its first barrier.
        const int tstep = A.step0 + step + 1;
        // (the bias corrections' reciprocals once per step)
        const float ic1 = 1.f / (1.f - powf(0.9f, (float)tstep)), ic2 = 1.f / (1.f - powf(0.999f, (float)tstep));
#pragma unroll
        for (int k = 0; k < PER_THREAD; k++) {
            const int i = tid + NT * k;
            if (i < NPARAM) {
                const float gr = grad_at(ts, i);
                const float m = 0.9f * m_reg[k] + 0.1f * gr;
                const float v = 0.999f * v_reg[k] + 0.001f * gr * gr;
                m_reg[k] = m;
                v_reg[k] = v;
                const float p = ts.P[i] - A.lr * (m * ic1) / (sqrtf(v * ic2) + 1e-8f);
                ts.P[i] = p;
                if (i >= OFF_W2 && i < OFF_B2) ts.W2b[(i - OFF_W2) / NH][(i - OFF_W2) % NH] = __float2bfloat16_rn(p);
            }
        }
        if (A.loss_hist && tid == 0) A.loss_hist[(size_t)member * A.steps + step] = ts.loss;
    }
    __syncthreads();
    // the trained weights and moments back to the handle
#pragma unroll
    for (int k = 0; k < PER_THREAD; k++) {
        const int i = tid + NT * k;
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
    k_mlp_train<<<members, NT, sm, st>>>(A);
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
