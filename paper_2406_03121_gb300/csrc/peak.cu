// CUDA-core FMA throughput microbenchmark (diagnostic): independent FMA chains per thread, timed
// with CUDA events on the given stream.  Used as the roofline denominator of the ALU-bound kernels.
#include "mess_internal.h"

namespace {

template <typename R>
__global__ void k_fma_chain(R* __restrict__ out, int iters, R a, R b)
{
    R x0 = (R)threadIdx.x, x1 = x0 + R(1), x2 = x0 + R(2), x3 = x0 + R(3);
    R x4 = x0 + R(4), x5 = x0 + R(5), x6 = x0 + R(6), x7 = x0 + R(7);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            x0 = x0 * a + b; x1 = x1 * a + b; x2 = x2 * a + b; x3 = x3 * a + b;
            x4 = x4 * a + b; x5 = x5 * a + b; x6 = x6 * a + b; x7 = x7 * a + b;
        }
    }
    const R s = ((x0 + x1) + (x2 + x3)) + ((x4 + x5) + (x6 + x7));
    if (s == R(-12345.678)) out[blockIdx.x * blockDim.x + threadIdx.x] = s;   // keeps the chains live
}

template <typename R>
cudaError_t time_fma(int iters, cudaStream_t s, double* tflops)
{
    int dev = 0, nsm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const int T = 256, B = nsm * 8;
    R* out = nullptr;
    e = cudaMalloc((void**)&out, sizeof(R) * (size_t)T * B);
    if (e != cudaSuccess) return e;
    cudaEvent_t t0, t1;
    cudaEventCreate(&t0);
    cudaEventCreate(&t1);
    k_fma_chain<R><<<B, T, 0, s>>>(out, iters / 4, R(0.999999), R(1e-7));   // warm-up
    cudaEventRecord(t0, s);
    k_fma_chain<R><<<B, T, 0, s>>>(out, iters, R(0.999999), R(1e-7));
    cudaEventRecord(t1, s);
    e = cudaEventSynchronize(t1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t0, t1);
    if (e == cudaSuccess) e = cudaGetLastError();
    const double flops = 2.0 * 8.0 * 16.0 * (double)iters * T * B;
    *tflops = flops / (ms * 1e-3) / 1e12;
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    cudaFree(out);
    return e;
}

}  // namespace

extern "C" mess_status mess_fma_peak(double* fp32_tflops, double* fp64_tflops, void* stream)
{
    if (!fp32_tflops || !fp64_tflops) { mess_set_error("null argument"); return MESS_EINVAL; }
    cudaStream_t s = (cudaStream_t)stream;
    MESS_CUDA_TRY(time_fma<float>(4096, s, fp32_tflops));
    MESS_CUDA_TRY(time_fma<double>(256, s, fp64_tflops));
    return MESS_OK;
}
