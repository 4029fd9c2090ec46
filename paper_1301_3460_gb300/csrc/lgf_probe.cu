// lgf_probe_fma: the FMA rate of this GPU in FP64 or FP32, the arithmetic peak
// that the FP64 kernels of the gauge fixing are measured against (their bound is
// the FP64 pipe, not memory).  Instrumentation; not a step of the method.
//
// Each thread runs 16 independent FMA chains of n_iter steps on values that stay
// bounded (x <- x * a + b with |a| < 1), so the pipe sees no dependency stalls,
// and writes one value so the work cannot be dropped.  The grid fills every SM
// several times over.
#include <cuda_runtime.h>

#include "../../include/lgf.h"
#include "lgf_common.cuh"

namespace {

template <typename T> __global__ void __launch_bounds__(256) k_fma_probe(int n_iter, T a, T b, T* out)
{
    T x[16];
#pragma unroll
    for (int k = 0; k < 16; k++) x[k] = (T)(threadIdx.x + k) * (T)1e-3;
    for (int i = 0; i < n_iter; i++) {
#pragma unroll
        for (int k = 0; k < 16; k++) x[k] = fma(x[k], a, b);
    }
    T s = 0;
#pragma unroll
    for (int k = 0; k < 16; k++) s += x[k];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename T> int probe(int n_iter, double* gflops, double* ms_out)
{
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return LGF_ERR_CUDA;
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return LGF_ERR_CUDA;
    const int blocks = nsm * 8, threads = 256;
    T* out = nullptr;
    if (cudaMalloc((void**)&out, (size_t)blocks * threads * sizeof(T)) != cudaSuccess) return LGF_ERR_CUDA;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    k_fma_probe<T><<<blocks, threads>>>(n_iter / 10 + 1, (T)0.999, (T)1e-4, out);  // warm-up
    cudaEventRecord(e0);
    k_fma_probe<T><<<blocks, threads>>>(n_iter, (T)0.999, (T)1e-4, out);
    cudaEventRecord(e1);
    const cudaError_t e = cudaEventSynchronize(e1);
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    if (e != cudaSuccess || cudaGetLastError() != cudaSuccess) return LGF_ERR_CUDA;
    const double flops = 2.0 * 16.0 * (double)n_iter * blocks * threads;
    *gflops = flops / (ms * 1e-3) / 1e9;
    if (ms_out) *ms_out = ms;
    return LGF_OK;
}

__global__ void k_check_conversions(const double* __restrict__ d_in, float* __restrict__ f_out,
                                    const float* __restrict__ f_in, double* __restrict__ d_out, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    f_out[i] = lgf::d2f_int(d_in[i]);
    d_out[i] = lgf::f2d_int(f_in[i]);
}

}  // namespace

extern "C" int lgf_check_conversions(const double* d_in, float* f_out, const float* f_in, double* d_out, int n)
{
    if (n < 0 || (n > 0 && (!d_in || !f_out || !f_in || !d_out))) return LGF_ERR_ARG;
    if (n == 0) return LGF_OK;
    k_check_conversions<<<(n + 255) / 256, 256>>>(d_in, f_out, f_in, d_out, n);
    if (cudaGetLastError() != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) return LGF_ERR_CUDA;
    return LGF_OK;
}

extern "C" int lgf_probe_fma(int precision, int n_iter, double* gflops, double* ms)
{
    if (!gflops || n_iter < 1 || (precision != 64 && precision != 32)) return LGF_ERR_ARG;
    return precision == 64 ? probe<double>(n_iter, gflops, ms) : probe<float>(n_iter, gflops, ms);
}
