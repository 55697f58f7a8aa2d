// Internal host-side state of the library (C++; never crosses the C ABI).
#pragma once
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "../../include/mess.h"
#include "eri_common.cuh"
#include "eri_launch.h"
#include "mess_device.h"

void mess_set_error(const char* fmt, ...);

#define MESS_CUDA_TRY(expr)                                                                      \
    do {                                                                                          \
        cudaError_t e_ = (expr);                                                                  \
        if (e_ != cudaSuccess) {                                                                  \
            mess_set_error("%s failed: %s (%s:%d)", #expr, cudaGetErrorString(e_), __FILE__, __LINE__); \
            return e_ == cudaErrorMemoryAllocation ? MESS_ENOMEM : MESS_ECUDA;                    \
        }                                                                                         \
    } while (0)

// A device allocation owned by the basis.
template <typename T> struct DevBuf {
    T* p = nullptr;
    size_t n = 0;
    cudaError_t alloc(size_t count)
    {
        free();
        n = count;
        if (count == 0) return cudaSuccess;
        return cudaMalloc((void**)&p, count * sizeof(T));
    }
    cudaError_t upload(const std::vector<T>& h)
    {
        cudaError_t e = alloc(h.size());
        if (e != cudaSuccess || h.empty()) return e;
        return cudaMemcpy(p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice);
    }
    void free()
    {
        if (p) cudaFree(p);
        p = nullptr;
        n = 0;
    }
};

struct HostShell {
    int l, K, atom, f0;
    double R[3];
    std::vector<double> alpha, coef;   // coef: contraction x primitive norm (x^l component) x contraction norm
};

// Quartet bins of one (schwarz_tau, fp64_tau) setting: per class, an FP64 part and an FP32 part.
struct BinPart {
    int qclass;
    int fp64;              // 1: evaluated in FP64
    int G;                 // lanes per shell quartet (primitive loop split across G lanes)
    int bra_off, nbra;     // into the concatenated bra / kbeg / offs arrays
    int ket_list;          // pair class of the ket list
    long long total;       // shell quartets
    long long fn_quartets; // unique function quartets
    long long prim_quartets;
    size_t offs_off;       // into offs
};

struct BinSet {
    double tau = -1.0, tau64 = -1.0;
    int split = -1;        // whether an FP64 / FP32 split was requested
    std::vector<BinPart> parts;
    DevBuf<int> bra, kbeg;
    DevBuf<long long> offs;
};

struct mess_basis {
    int natom = 0, nbf = 0, nelec = 0;
    std::vector<int> Z;
    std::vector<double> xyz;
    std::vector<HostShell> shells;
    std::vector<double> fscale;     // per function: component normalisation relative to x^l

    // canonical shell pairs (A, B): l_A > l_B, or l_A == l_B and A >= B
    int npair = 0;
    std::vector<int> pair_a, pair_b, pair_class, pp_off, pp_n;
    std::vector<double> Q;          // Schwarz factor per pair
    std::vector<int> class_list[MESS_NUM_PCLASS];   // pair ids sorted by Q descending
    DevBuf<int> d_class_list[MESS_NUM_PCLASS];

    DevBuf<PrimPairRec<double>> d_pp64;
    DevBuf<PrimPairRec<float>> d_pp32;
    DevBuf<int> d_pp_off, d_pp_n, d_fa, d_fb, d_same;
    DevBuf<double> d_AB, d_Q, d_Ccen;
    DevBuf<double> d_boys64;
    DevBuf<float> d_boys32;
    DevBuf<int> d_Z;
    DevBuf<double> d_xyz;
    DevBuf<int> d_shell_l, d_shell_K, d_shell_f0, d_shell_poff;
    DevBuf<double> d_shell_R, d_shell_alpha, d_shell_coef, d_fscale;
    DevBuf<int> d_pair_a, d_pair_b;

    PairTable<double> P64;
    PairTable<float> P32;
    BinSet bins;
};

// one-electron integrals on the device (one_e.cu)
cudaError_t mess_launch_one_e(const mess_basis* b, double* dS, double* dT, double* dV, cudaStream_t s);
// J/K helpers (jk.cu)
cudaError_t mess_launch_symmetrise_jk(double* J, double* K, int n, cudaStream_t s);
// Boys tables (boys_table.cu): rows x MESS_BOYS_NCOL
void mess_boys_table(std::vector<double>& tab);
// bins (host.cu)
mess_status mess_ensure_bins(mess_basis* b, double tau, double tau64, int split);
