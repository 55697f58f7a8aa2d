// Finishing step of the J/K build: J = 2 (Jacc + Jacc^T), K = Kacc + Kacc^T, in place, for every
// molecule block of the packed matrices.
#include <algorithm>

#include "mess_internal.h"

namespace {

__global__ void k_symmetrise_jk(double* __restrict__ J, double* __restrict__ K, const long long* __restrict__ mbase,
                                const int* __restrict__ mn)
{
    const int m = blockIdx.y;
    const int n = mn[m];
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long npairs = (long long)n * (n + 1) / 2;
    if (t >= npairs) return;
    // t -> (i, j), i >= j, row-major lower triangle
    int i = (int)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
    while ((long long)i * (i + 1) / 2 > t) --i;
    while ((long long)(i + 1) * (i + 2) / 2 <= t) ++i;
    const int j = (int)(t - (long long)i * (i + 1) / 2);
    double* Jm = J + mbase[m];
    double* Km = K + mbase[m];
    const size_t ij = (size_t)i * n + j, ji = (size_t)j * n + i;
    const double js = 2.0 * (Jm[ij] + Jm[ji]);
    const double ks = Km[ij] + Km[ji];
    Jm[ij] = js; Jm[ji] = js;
    Km[ij] = ks; Km[ji] = ks;
}

// Copies of D read by the reduced-precision J/K kernels: FP32 (round to nearest) and double-float
// (hi = D rounded to FP32, lo = the remainder rounded to FP32).  Either output may be null.
__global__ void k_convert_density(const double* __restrict__ D, float* __restrict__ D32, float2* __restrict__ Ddf,
                                  long long count)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (long long)gridDim.x * blockDim.x) {
        const double v = D[i];
        const float hi = __double2float_rn(v);
        if (D32) D32[i] = hi;
        if (Ddf) Ddf[i] = make_float2(hi, __double2float_rn(v - (double)hi));
    }
}

}  // namespace

cudaError_t mess_launch_convert_density(const double* D, float* D32, float2* Ddf, long long count, cudaStream_t s)
{
    if (count <= 0 || (!D32 && !Ddf)) return cudaSuccess;
    const int T = 256;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const long long blocks = std::min<long long>((count + T - 1) / T, 4LL * std::max(1, sms));
    k_convert_density<<<(unsigned)blocks, T, 0, s>>>(D, D32, Ddf, count);
    return cudaGetLastError();
}

cudaError_t mess_launch_symmetrise_jk(const mess_basis* b, double* J, double* K, cudaStream_t s)
{
    const long long np = (long long)b->max_nbf * (b->max_nbf + 1) / 2;
    const int T = 256;
    dim3 grid((unsigned)((np + T - 1) / T), (unsigned)b->nmol);
    k_symmetrise_jk<<<grid, T, 0, s>>>(J, K, b->d_mol_base.p, b->d_mol_n.p);
    return cudaGetLastError();
}
