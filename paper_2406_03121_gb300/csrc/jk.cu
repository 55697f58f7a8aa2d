// Finishing step of the J/K build: J = 2 (Jacc + Jacc^T), K = Kacc + Kacc^T, in place.
#include "mess_internal.h"

namespace {

__global__ void k_symmetrise_jk(double* __restrict__ J, double* __restrict__ K, int n)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long npairs = (long long)n * (n + 1) / 2;
    if (t >= npairs) return;
    // t -> (i, j), i >= j, row-major lower triangle
    int i = (int)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
    while ((long long)i * (i + 1) / 2 > t) --i;
    while ((long long)(i + 1) * (i + 2) / 2 <= t) ++i;
    const int j = (int)(t - (long long)i * (i + 1) / 2);
    const size_t ij = (size_t)i * n + j, ji = (size_t)j * n + i;
    const double js = 2.0 * (J[ij] + J[ji]);
    const double ks = K[ij] + K[ji];
    J[ij] = js; J[ji] = js;
    K[ij] = ks; K[ji] = ks;
}

}  // namespace

cudaError_t mess_launch_symmetrise_jk(double* J, double* K, int n, cudaStream_t s)
{
    const long long np = (long long)n * (n + 1) / 2;
    const int T = 256;
    k_symmetrise_jk<<<(unsigned)((np + T - 1) / T), T, 0, s>>>(J, K, n);
    return cudaGetLastError();
}
