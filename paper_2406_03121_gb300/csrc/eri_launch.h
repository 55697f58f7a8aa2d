// Host-side launch interface of the generated per-class ERI kernels.
#pragma once
#include <cuda_runtime.h>

#include "df32.cuh"
#include "eri_classes.h"
#include "mess_device.h"

template <typename R> struct PairTable;

enum { MESS_KIND_JK = 0, MESS_KIND_STORE = 1, MESS_KIND_SCHWARZ = 2 };
// kernel modes: FP64; FP32 recursion with FP64 Boys at small T; FP32 recursion with FP32 Boys;
// double-float (FP32 pairs) recursion and Boys
enum { MESS_MODE_FP64 = 0, MESS_MODE_MIXED = 1, MESS_MODE_FP32 = 2, MESS_MODE_DF32 = 3 };

struct ClassLaunchArgs {
    int kind;                    // MESS_KIND_*
    int mode;                    // MESS_MODE_* (JK only)
    int G;                       // JK: lanes per shell quartet (1, 4 or 8)
    int team;                    // JK: 1 = one warp per shell quartet (level-scheduled program)
    BinLaunch bin;               // JK / STORE
    const int* pairs;            // SCHWARZ: pair ids of one diagonal class
    int npairs;
    const PairTable<double>* P64_ptr;
    const PairTable<float>* P32_ptr;
    const PairTable<df32>* Pdf_ptr;
    const double* D;             // device, n x n
    const float* D32;            // D rounded to FP32 (FP32 kernels)
    const float2* Ddf;           // D as double-float hi, lo (double-float kernels)
    double* J;                   // device, n x n accumulators
    double* K;
    double* out;                 // STORE: n^4 tensor; SCHWARZ: Q per pair
    int n;
    cudaStream_t stream;
};

template <typename R> inline const typename DElem<R>::T* dmat(const ClassLaunchArgs& a);
template <> inline const double* dmat<double>(const ClassLaunchArgs& a) { return a.D; }
template <> inline const float* dmat<float>(const ClassLaunchArgs& a) { return a.D32; }
template <> inline const float2* dmat<df32>(const ClassLaunchArgs& a) { return a.Ddf; }

typedef cudaError_t (*mess_class_launcher)(const ClassLaunchArgs&);
extern const mess_class_launcher MESS_CLASS_LAUNCHERS[MESS_NUM_QCLASS];

// Launch of a warp-per-quartet kernel with its dynamic shared memory (opt-in above 48 KB, set
// once per kernel).
template <typename R, int BMODE, typename Kern>
cudaError_t mess_team_launch(Kern kern, dim3 grid, size_t smem, const ClassLaunchArgs& a, const PairTable<R>& P,
                             int* configured /* per kernel: 0 until the attribute is set on this device */)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!configured[dev]) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        configured[dev] = 1;
    }
    kern<<<grid, 32 * MESS_TEAM_WARPS, smem, a.stream>>>(a.bin, P, dmat<R>(a), a.J, a.K, a.n);
    return cudaGetLastError();
}
