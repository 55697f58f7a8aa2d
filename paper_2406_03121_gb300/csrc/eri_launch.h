// Host-side launch interface of the generated per-class ERI kernels.
#pragma once
#include <cuda_runtime.h>

#include "eri_classes.h"
#include "mess_device.h"

template <typename R> struct PairTable;

enum { MESS_KIND_JK = 0, MESS_KIND_STORE = 1, MESS_KIND_SCHWARZ = 2 };
// kernel modes: FP64; FP32 recursion with FP64 Boys at small T; FP32 recursion with FP32 Boys
enum { MESS_MODE_FP64 = 0, MESS_MODE_MIXED = 1, MESS_MODE_FP32 = 2 };

struct ClassLaunchArgs {
    int kind;                    // MESS_KIND_*
    int mode;                    // MESS_MODE_* (JK only)
    BinLaunch bin;               // JK / STORE
    const int* pairs;            // SCHWARZ: pair ids of one diagonal class
    int npairs;
    const PairTable<double>* P64_ptr;
    const PairTable<float>* P32_ptr;
    const double* D;             // device, n x n
    double* J;                   // device, n x n accumulators
    double* K;
    double* out;                 // STORE: n^4 tensor; SCHWARZ: Q per pair
    int n;
    cudaStream_t stream;
};

typedef cudaError_t (*mess_class_launcher)(const ClassLaunchArgs&);
extern const mess_class_launcher MESS_CLASS_LAUNCHERS[MESS_NUM_QCLASS];
