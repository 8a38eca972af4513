// Diagnostic: measured fused multiply-add issue rate of the current device,
// the denominator of the ALU roofline of the force kernels.
#include <cuda_runtime.h>

#include "fire2.h"
#include "fire2_math.cuh"

namespace {

// Eight independent FMA chains per thread keep the FMA pipe busy without
// memory traffic; the final sum is stored so nothing is optimised away.
template <typename T>
__global__ void k_fma_chains(T* out, int iters, T a, T b) {
    T x0 = T(threadIdx.x) * T(1e-3), x1 = x0 + T(1), x2 = x0 + T(2), x3 = x0 + T(3);
    T x4 = x0 + T(4), x5 = x0 + T(5), x6 = x0 + T(6), x7 = x0 + T(7);
    for (int i = 0; i < iters; ++i) {
        x0 = fma(x0, a, b); x1 = fma(x1, a, b); x2 = fma(x2, a, b); x3 = fma(x3, a, b);
        x4 = fma(x4, a, b); x5 = fma(x5, a, b); x6 = fma(x6, a, b); x7 = fma(x7, a, b);
    }
    out[blockIdx.x * blockDim.x + threadIdx.x] = ((x0 + x1) + (x2 + x3)) + ((x4 + x5) + (x6 + x7));
}

template <typename T>
cudaError_t time_fma(int sms, int iters, double* ms) {
    const int blocks = sms * 8, threads = 256;
    T* out = nullptr;
    cudaError_t e = cudaMalloc(&out, sizeof(T) * blocks * threads);
    if (e != cudaSuccess) return e;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    k_fma_chains<T><<<blocks, threads>>>(out, iters, T(0.999999), T(1e-6));
    cudaEventRecord(e0);
    k_fma_chains<T><<<blocks, threads>>>(out, iters, T(0.999999), T(1e-6));
    cudaEventRecord(e1);
    e = cudaEventSynchronize(e1);
    float f = 0.f;
    cudaEventElapsedTime(&f, e0, e1);
    *ms = f;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    if (e == cudaSuccess) e = cudaGetLastError();
    return e;
}

__global__ void k_exp_tang(int64_t n, const double* x, double* out, const double* table,
                           fire2::ExpC c) {
    __shared__ double tbl[fire2::kExpTableSize];
    for (int t = threadIdx.x; t < fire2::kExpTableSize; t += blockDim.x) tbl[t] = table[t];
    __syncthreads();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = fire2::exp_tang(x[i], c, tbl);
}

}  // namespace

extern "C" fire_status fire_diag_exp(int64_t n, const double* d_x, double* d_out, void* stream) {
    if (n < 0 || (n > 0 && (!d_x || !d_out))) return FIRE_ERR_ARG;
    if (n == 0) return FIRE_OK;
    double host_table[fire2::kExpTableSize];
    const fire2::ExpC c = fire2::make_exp_constants(host_table);
    double* d_table = nullptr;
    if (cudaMalloc(&d_table, sizeof host_table) != cudaSuccess) return FIRE_ERR_NOMEM;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemcpyAsync(d_table, host_table, sizeof host_table, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
        k_exp_tang<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, d_x, d_out, d_table, c);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(d_table);
    return e == cudaSuccess ? FIRE_OK : FIRE_ERR_CUDA;
}

extern "C" fire_status fire_diag_fma_peak(int32_t which, double* flops_per_s) {
    if (!flops_per_s || (which != 0 && which != 1)) return FIRE_ERR_ARG;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return FIRE_ERR_CUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return FIRE_ERR_CUDA;
    int iters = which == 0 ? 2000 : 20000;
    double ms = 0.0;
    for (int pass = 0; pass < 2; ++pass) {
        cudaError_t e = which == 0 ? time_fma<double>(sms, iters, &ms) : time_fma<float>(sms, iters, &ms);
        if (e != cudaSuccess) return FIRE_ERR_CUDA;
        if (pass == 0 && ms > 0.0) {
            // aim for ~100 ms in the measured pass
            double scale = 100.0 / ms;
            iters = (int)(iters * (scale > 1000.0 ? 1000.0 : (scale < 1.0 ? 1.0 : scale)));
        }
    }
    const double fmas = (double)sms * 8 * 256 * 8 * (double)iters;
    *flops_per_s = 2.0 * fmas / (ms * 1e-3);
    return FIRE_OK;
}
