// Finishing step of the J/K build: J = 2 (Jacc + Jacc^T), K = Kacc + Kacc^T, in place, for every
// molecule block of the packed matrices.
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

}  // namespace

cudaError_t mess_launch_symmetrise_jk(const mess_basis* b, double* J, double* K, cudaStream_t s)
{
    const long long np = (long long)b->max_nbf * (b->max_nbf + 1) / 2;
    const int T = 256;
    dim3 grid((unsigned)((np + T - 1) / T), (unsigned)b->nmol);
    k_symmetrise_jk<<<grid, T, 0, s>>>(J, K, b->d_mol_base.p, b->d_mol_n.p);
    return cudaGetLastError();
}
