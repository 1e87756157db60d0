// mlp_kernels.cuh -- launch interface of the surrogate and selection kernels
// (internal to the library; the public boundary is include/pnscan.h).
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace pnscan {
namespace mlp {

constexpr int NIN = 4;
constexpr int NH = 64;
// parameter vector: W1 (64 x 4), b1 (64), W2 (64 x 64, [out][in]), b2 (64), w3 (64), b3
constexpr int OFF_W1 = 0;
constexpr int OFF_B1 = OFF_W1 + NH * NIN;
constexpr int OFF_W2 = OFF_B1 + NH;
constexpr int OFF_B2 = OFF_W2 + NH * NH;
constexpr int OFF_W3 = OFF_B2 + NH;
constexpr int OFF_B3 = OFF_W3 + NH;
constexpr int NPARAM = OFF_B3 + 1;
constexpr int BATCH = 128;
constexpr long long SELECT_MAX_BLOCKS = 65536;

struct TrainArgs {
    float* params;        // [members][NPARAM] fp32 master weights
    float* adam_m;        // [members][NPARAM]
    float* adam_v;        // [members][NPARAM]
    const float* X;       // [N][4] raw cell parameters
    const float* Y;       // [N] targets (FLI)
    long long N;
    int steps;
    int step0;            // Adam steps already taken (bias correction)
    float lr;
    uint64_t seed;
    float center[NIN], scale[NIN];
    float* loss_hist;     // [members][steps] or null
    int mode;             // 0: train; 1: gradient of rows 0..BATCH-1, no update
    float* grad_out;      // mode 1: [members][NPARAM]
    float* loss_out;      // mode 1: [members]
};

struct PredictArgs {
    const float* params;  // [members][NPARAM]
    int members;
    const float* X;       // [N][4]
    long long N;
    float center[NIN], scale[NIN];
    float* mean;          // [N]
    float* spread;        // [N] max - min over members
};

struct SelectArgs {
    const float* mean;
    const float* spread;
    long long N;
    float thr, band, spread_max;
    const double* cells;  // [N][9] or null
    int32_t* idx;         // [N] selected cell indices, ascending
    double* cells_out;    // [N][9] gathered cells or null
};

struct MergeArgs {
    const float* mean;
    long long N;
    float thr;
    const int32_t* idx;
    long long count;
    const double* fli;    // [count] integrator FLI of the selected cells
    const int32_t* status;// [count]
    int8_t* cls;          // [N]
};

size_t smem_bytes();
size_t select_workspace_bytes(long long n);
cudaError_t launch_init(float* params, float* m, float* v, int members, uint64_t seed, cudaStream_t st);
cudaError_t launch_train(const TrainArgs& A, int members, cudaStream_t st);
cudaError_t launch_predict(const PredictArgs& A, cudaStream_t st);
cudaError_t launch_select(const SelectArgs& A, void* ws, long long* d_total, cudaStream_t st);
cudaError_t launch_merge(const MergeArgs& A, cudaStream_t st);
cudaError_t launch_features(const double* cells, long long n, float* X, cudaStream_t st);

struct FieldSel {
    int field[NIN];   // cell field (0..8) of each input
};
cudaError_t launch_features_fields(const double* cells, long long n, FieldSel f, float* X, cudaStream_t st);

struct InterpArgs {
    const double* fli;      // [nc1][nc2] node FLIs
    const int32_t* status;  // [nc1][nc2] node statuses
    long long nc1, nc2, stride, n1, n2;
    float* mean;            // [n1][n2]
    float* spread;          // [n1][n2]
};
cudaError_t launch_interp_grid(const InterpArgs& A, cudaStream_t st);

}  // namespace mlp
}  // namespace pnscan
