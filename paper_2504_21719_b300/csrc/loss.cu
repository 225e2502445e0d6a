// Small kernels around the tracer: the dB-MSE loss of the differentiable
// workload with its gradient, the gradient hand-off, and record filling.
#include "common.cuh"

namespace rmsbr {
namespace {

constexpr float LN10 = 2.302585092994046f;

__device__ __forceinline__ double block_sum(double v, double* sh) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(FULL_MASK, v, o);
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sh[w];
    __syncthreads();
    return s;
}

// acc[0] += sum over valid cells of (10 log10 C - 10 log10 T)^2, acc[1] += |V|
__global__ void k_db_pass1(const float* __restrict__ m, const float* __restrict__ t, int64_t n, float floor_lin,
                           double* acc) {
    __shared__ double sh[32];
    double s = 0.0, c = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float a = m[i], b = t[i];
        if (a > floor_lin && b > floor_lin) {
            const float d = 10.0f * (log10f(a) - log10f(b));
            s += (double)d * d;
            c += 1.0;
        }
    }
    s = block_sum(s, sh);
    c = block_sum(c, sh);
    if (threadIdx.x == 0) {
        atomicAdd(&acc[0], s);
        atomicAdd(&acc[1], c);
    }
}

// dL/dC_i = (2 / |V|) d_i * 10 / (ln 10 C_i) on V, 0 elsewhere
__global__ void k_db_pass2(const float* __restrict__ m, const float* __restrict__ t, int64_t n, float floor_lin,
                           const double* __restrict__ acc, float* loss, float* dLdC, int64_t* valid) {
    const double V = acc[1];
    const float inv = V > 0.0 ? (float)(2.0 / V) : 0.0f;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float a = m[i], b = t[i];
        float g = 0.0f;
        if (a > floor_lin && b > floor_lin) {
            const float d = 10.0f * (log10f(a) - log10f(b));
            g = inv * d * 10.0f / (LN10 * a);
        }
        dLdC[i] = g;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if (loss) loss[0] = V > 0.0 ? (float)(acc[0] / V) : 0.0f;
        if (valid) valid[0] = (int64_t)V;
    }
}

__global__ void k_grad_out(const double* __restrict__ g, int nm, int ntx, float* d_eps, float* d_sigma,
                           float* d_tx) {
    const int i = threadIdx.x;
    if (i < nm) {
        if (d_eps) d_eps[i] += (float)g[i];
        if (d_sigma) d_sigma[i] += (float)g[RM_MAX_MATERIALS + i];
    }
    if (d_tx && i < 3 * ntx) d_tx[i] += (float)g[2 * RM_MAX_MATERIALS + i];
}

__global__ void k_fill_record(rm_segment_record* r, unsigned long long n) {
    for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (unsigned long long)gridDim.x * blockDim.x)
        r[i] = rm_segment_record{-2, NO_CELL, NO_CELL, -1};
}

__global__ void k_map_to_f32(const double* __restrict__ m64, float* __restrict__ m, unsigned long long n) {
    for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (unsigned long long)gridDim.x * blockDim.x)
        m[i] = (float)m64[i];
}

}  // namespace

cudaError_t launch_map_to_f32(const double* m64, float* m, unsigned long long n, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    const unsigned long long b = (n + 255) / 256;
    k_map_to_f32<<<(unsigned)(b < 8192 ? b : 8192), 256, 0, s>>>(m64, m, n);
    return cudaGetLastError();
}

cudaError_t launch_db_mse(const float* maps, const float* target, int64_t n, float floor_lin, double* acc,
                          float* loss, float* dLdC, int64_t* valid, cudaStream_t s) {
    const int grid = (int)((n + 255) / 256 < 1184 ? (n + 255) / 256 : 1184);
    const int g = grid > 0 ? grid : 1;
    k_db_pass1<<<g, 256, 0, s>>>(maps, target, n, floor_lin, acc);
    k_db_pass2<<<g, 256, 0, s>>>(maps, target, n, floor_lin, acc, loss, dLdC, valid);
    return cudaGetLastError();
}

cudaError_t launch_grad_out(const double* grad, int nm, int ntx, float* d_eps, float* d_sigma, float* d_tx,
                            cudaStream_t s) {
    k_grad_out<<<1, 3 * RM_MAX_TX, 0, s>>>(grad, nm, ntx, d_eps, d_sigma, d_tx);
    return cudaGetLastError();
}

cudaError_t launch_fill_record(rm_segment_record* rec, unsigned long long n, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    const unsigned long long b = (n + 255) / 256;
    k_fill_record<<<(unsigned)(b < 4096 ? b : 4096), 256, 0, s>>>(rec, n);
    return cudaGetLastError();
}

}  // namespace rmsbr
