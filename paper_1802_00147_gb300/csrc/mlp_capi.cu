// mlp_capi.cu -- C ABI of the scan surrogate (mlp_*) and of the adaptive
// scan's selection and merge (adaptive_*), declared in include/pnscan.h.
#include <cuda_runtime.h>

#include <cstring>
#include <new>

#include "../../include/pnscan.h"
#include "mlp_kernels.cuh"

using namespace pnscan::mlp;

struct mlp_handle {
    int members = 0;
    cudaStream_t stream = nullptr;
    float* params = nullptr;   // [members][NPARAM], then adam_m, adam_v in the same block
    float* adam_m = nullptr;
    float* adam_v = nullptr;
    int adam_steps = 0;
    float center[NIN], scale[NIN];
};

static_assert(NPARAM == MLP_PARAMS, "parameter layout");

extern "C" {

int mlp_create(int members, uint64_t seed, const float* center, const float* scale, void* cuda_stream,
               mlp_handle** out)
{
    if (!out) return PNSCAN_ERR_ARG;
    *out = nullptr;
    if (members < 1 || members > 64 || !center || !scale) return PNSCAN_ERR_ARG;
    for (int i = 0; i < NIN; i++)
        if (!(scale[i] != 0.0f)) return PNSCAN_ERR_ARG;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return PNSCAN_ERR_NODEVICE;
    }
    mlp_handle* h = new (std::nothrow) mlp_handle();
    if (!h) return PNSCAN_ERR_OOM;
    h->members = members;
    h->stream = (cudaStream_t)cuda_stream;
    std::memcpy(h->center, center, sizeof(h->center));
    std::memcpy(h->scale, scale, sizeof(h->scale));
    const size_t n = (size_t)members * NPARAM;
    if (cudaMalloc(&h->params, 3 * n * sizeof(float)) != cudaSuccess) {
        cudaGetLastError();
        delete h;
        return PNSCAN_ERR_OOM;
    }
    h->adam_m = h->params + n;
    h->adam_v = h->params + 2 * n;
    if (launch_init(h->params, h->adam_m, h->adam_v, members, seed, h->stream) != cudaSuccess ||
        cudaStreamSynchronize(h->stream) != cudaSuccess) {
        mlp_destroy(h);
        return PNSCAN_ERR_CUDA;
    }
    *out = h;
    return PNSCAN_OK;
}

int mlp_get_params(mlp_handle* h, float* params)
{
    if (!h || !params) return PNSCAN_ERR_ARG;
    if (cudaMemcpyAsync(params, h->params, sizeof(float) * h->members * NPARAM, cudaMemcpyDeviceToDevice,
                        h->stream) != cudaSuccess)
        return PNSCAN_ERR_CUDA;
    return cudaStreamSynchronize(h->stream) == cudaSuccess ? PNSCAN_OK : PNSCAN_ERR_CUDA;
}

int mlp_get_moments(mlp_handle* h, float* m, float* v)
{
    if (!h || !m || !v) return PNSCAN_ERR_ARG;
    const size_t bytes = sizeof(float) * h->members * NPARAM;
    if (cudaMemcpyAsync(m, h->adam_m, bytes, cudaMemcpyDeviceToDevice, h->stream) != cudaSuccess ||
        cudaMemcpyAsync(v, h->adam_v, bytes, cudaMemcpyDeviceToDevice, h->stream) != cudaSuccess)
        return PNSCAN_ERR_CUDA;
    return cudaStreamSynchronize(h->stream) == cudaSuccess ? PNSCAN_OK : PNSCAN_ERR_CUDA;
}

int mlp_set_params(mlp_handle* h, const float* params)
{
    if (!h || !params) return PNSCAN_ERR_ARG;
    const size_t bytes = sizeof(float) * h->members * NPARAM;
    if (cudaMemcpyAsync(h->params, params, bytes, cudaMemcpyDeviceToDevice, h->stream) != cudaSuccess ||
        cudaMemsetAsync(h->adam_m, 0, 2 * bytes, h->stream) != cudaSuccess)
        return PNSCAN_ERR_CUDA;
    h->adam_steps = 0;
    return cudaStreamSynchronize(h->stream) == cudaSuccess ? PNSCAN_OK : PNSCAN_ERR_CUDA;
}

static TrainArgs train_args(mlp_handle* h)
{
    TrainArgs A{};
    A.params = h->params;
    A.adam_m = h->adam_m;
    A.adam_v = h->adam_v;
    std::memcpy(A.center, h->center, sizeof(A.center));
    std::memcpy(A.scale, h->scale, sizeof(A.scale));
    return A;
}

int mlp_train(mlp_handle* h, const float* X, const float* y, int64_t n, int steps, float lr, uint64_t seed,
              float* loss_hist)
{
    if (!h || !X || !y || n < 1 || steps < 0 || !(lr > 0.0f)) return PNSCAN_ERR_ARG;
    if (steps == 0) return PNSCAN_OK;
    TrainArgs A = train_args(h);
    A.X = X;
    A.Y = y;
    A.N = n;
    A.steps = steps;
    A.step0 = h->adam_steps;
    A.lr = lr;
    A.seed = seed;
    A.loss_hist = loss_hist;
    A.mode = 0;
    if (launch_train(A, h->members, h->stream) != cudaSuccess) return PNSCAN_ERR_CUDA;
    h->adam_steps += steps;
    return cudaStreamSynchronize(h->stream) == cudaSuccess ? PNSCAN_OK : PNSCAN_ERR_CUDA;
}

int mlp_gradient(mlp_handle* h, const float* X, const float* y, float* grad, float* loss)
{
    if (!h || !X || !y || !grad || !loss) return PNSCAN_ERR_ARG;
    TrainArgs A = train_args(h);
    A.X = X;
    A.Y = y;
    A.N = BATCH;
    A.steps = 1;
    A.mode = 1;
    A.grad_out = grad;
    A.loss_out = loss;
    if (launch_train(A, h->members, h->stream) != cudaSuccess) return PNSCAN_ERR_CUDA;
    return cudaStreamSynchronize(h->stream) == cudaSuccess ? PNSCAN_OK : PNSCAN_ERR_CUDA;
}

int mlp_predict(mlp_handle* h, const float* X, int64_t n, float* mean, float* spread)
{
    if (!h || n < 0 || (n > 0 && (!X || !mean || !spread))) return PNSCAN_ERR_ARG;
    PredictArgs A{};
    A.params = h->params;
    A.members = h->members;
    A.X = X;
    A.N = n;
    std::memcpy(A.center, h->center, sizeof(A.center));
    std::memcpy(A.scale, h->scale, sizeof(A.scale));
    A.mean = mean;
    A.spread = spread;
    if (launch_predict(A, h->stream) != cudaSuccess) return PNSCAN_ERR_CUDA;
    return PNSCAN_OK;
}

void mlp_destroy(mlp_handle* h)
{
    if (!h) return;
    cudaStreamSynchronize(h->stream);
    if (h->params) cudaFree(h->params);
    delete h;
}

size_t adaptive_select_workspace(int64_t n) { return n < 0 ? 0 : select_workspace_bytes(n); }

int adaptive_features(const double* cells, int64_t n, float* X, void* cuda_stream)
{
    if (n < 0 || (n > 0 && (!cells || !X))) return PNSCAN_ERR_ARG;
    return launch_features(cells, n, X, (cudaStream_t)cuda_stream) == cudaSuccess ? PNSCAN_OK : PNSCAN_ERR_CUDA;
}

int adaptive_features_fields(const double* cells, int64_t n, const int32_t* fields, float* X, void* cuda_stream)
{
    if (n < 0 || !fields || (n > 0 && (!cells || !X))) return PNSCAN_ERR_ARG;
    FieldSel f{};
    for (int k = 0; k < NIN; k++) {
        if (fields[k] < 0 || fields[k] > 8) return PNSCAN_ERR_ARG;
        f.field[k] = fields[k];
    }
    return launch_features_fields(cells, n, f, X, (cudaStream_t)cuda_stream) == cudaSuccess ? PNSCAN_OK
                                                                                            : PNSCAN_ERR_CUDA;
}

int adaptive_interp_grid(const double* fli_nodes, const int32_t* status_nodes, int64_t n1, int64_t n2,
                         int32_t stride, float* mean, float* spread, void* cuda_stream)
{
    if (n1 < 0 || n2 < 0 || stride < 1) return PNSCAN_ERR_ARG;
    if (n1 > 0 && n2 > 0 && (!fli_nodes || !status_nodes || !mean || !spread)) return PNSCAN_ERR_ARG;
    if (n1 > (int64_t)1 << 20 || n2 > (int64_t)1 << 20 || n1 * n2 > (int64_t)1 << 32) return PNSCAN_ERR_ARG;
    InterpArgs A{fli_nodes, status_nodes, n1 > 0 ? (n1 - 1) / stride + 1 : 0, n2 > 0 ? (n2 - 1) / stride + 1 : 0,
                 stride, n1, n2, mean, spread};
    return launch_interp_grid(A, (cudaStream_t)cuda_stream) == cudaSuccess ? PNSCAN_OK : PNSCAN_ERR_CUDA;
}

int adaptive_select(const float* mean, const float* spread, int64_t n, float thr, float band, float spread_max,
                    const double* cells, int32_t* idx, double* cells_out, int64_t* count, void* workspace,
                    void* cuda_stream)
{
    if (n < 0 || !count || (n > 0 && (!mean || !spread || !idx || !workspace))) return PNSCAN_ERR_ARG;
    if ((n + 255) / 256 > SELECT_MAX_BLOCKS) return PNSCAN_ERR_ARG;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    SelectArgs A{mean, spread, (long long)n, thr, band, spread_max, cells, idx, cells_out};
    const long long nb = (n + 255) / 256;
    long long* d_total = (long long*)((char*)workspace + ((nb + 1) * sizeof(int) + 7) / 8 * 8);
    if (launch_select(A, workspace, d_total, st) != cudaSuccess) return PNSCAN_ERR_CUDA;
    long long total = 0;
    if (cudaMemcpyAsync(&total, d_total, sizeof(total), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return PNSCAN_ERR_CUDA;
    *count = total;
    return PNSCAN_OK;
}

int adaptive_merge(const float* mean, int64_t n, float thr, const int32_t* idx, int64_t count,
                   const double* fli_sel, const int32_t* status_sel, int8_t* cls, void* cuda_stream)
{
    if (n < 0 || count < 0 || count > n || (n > 0 && (!mean || !cls)) ||
        (count > 0 && (!idx || !fli_sel || !status_sel)))
        return PNSCAN_ERR_ARG;
    MergeArgs A{mean, (long long)n, thr, idx, (long long)count, fli_sel, status_sel, cls};
    return launch_merge(A, (cudaStream_t)cuda_stream) == cudaSuccess ? PNSCAN_OK : PNSCAN_ERR_CUDA;
}

}  // extern "C"
