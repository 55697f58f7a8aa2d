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

// Phase timing of the host-driven calls, for users who want to see where a call spends its time:
// with MESS_TIMING=1 in the environment, every mark() synchronises the given stream and prints the
// host wall time since the previous mark to stderr ("[mess] <label>: <ms> ms").  Off by default:
// then mark() does nothing (no synchronisation).
struct PhaseTimer {
    bool on;
    cudaStream_t s;
    double t;
    explicit PhaseTimer(cudaStream_t stream);
    void mark(const char* label);
};

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
    int l, K, atom, f0;    // f0: global first function (across the molecules of a batch)
    int fl;                // first function within its molecule
    int mol;               // molecule index
    double R[3];
    std::vector<double> alpha, coef;   // coef: contraction x primitive norm (x^l component) x contraction norm
};

// Quartet bins of one (schwarz_tau, fp64_tau) setting: per class, an FP64 part and an FP32 part.
struct BinPart {
    int qclass;
    int fp64;              // 1: evaluated in FP64
    int G;                 // lanes per shell quartet (primitive loop split across G lanes)
    int team;              // 1: one warp per shell quartet, 2: one block (MESS_TEAM_WARPS warps) per quartet,
                           // 3: one block per quartet whose warps split the primitive quartets
    int mode = -1;         // kernel arithmetic (MESS_MODE_*) chosen by the autotuner; -1: from the options
    int tuned = 0;         // 1: G / team / mode were picked by timing the candidates
    int bra_off, nbra;     // into the concatenated bra / kbeg / offs arrays
    int ket_list;          // pair class of the ket list
    long long total;       // shell quartets
    long long fn_quartets; // unique function quartets
    long long prim_quartets;
    size_t offs_off;       // into offs
    size_t seg_off;        // into seg: bra index of every 32nd quartet of the part
};

struct BinSet {
    double tau = -1.0, tau64 = -1.0;
    int split = -1;        // whether an FP64 / FP32 split was requested
    long long active_version = -1;
    long long generation = 0;   // incremented on every rebuild (cached graphs refer to one generation)
    std::vector<BinPart> parts;
    DevBuf<int> bra, kbeg;
    DevBuf<long long> offs;
    DevBuf<int> seg;
};

// An instantiated CUDA graph of one J/K build: the bins' generation, the options that select
// kernels and the D / J / K buffers it was captured with.
struct JKGraph {
    long long bins_gen = -1;
    int prec = 0, boys_fp64 = 0, split_df32 = 0;
    const double* D = nullptr;
    double* J = nullptr;
    double* K = nullptr;
    cudaGraphExec_t exec = nullptr;
    int failed = 0;            // capture or instantiation failed once: launch directly
    mess_jk_info info{};
};

// Exchange-correlation quadrature of a basis (built on first use, kept with the basis): grid points
// and weights (Becke-partitioned), and every basis function's value and gradient at its molecule's
// points ([npts_m][n_m] blocks per molecule; gradients as three such blocks).
struct XcState {
    bool ready = false;
    long long npts = 0, ao = 0, mol_npts_max = 0;
    DevBuf<double> pts, w, phi, dphi, vrho, vgrad, Exc;
    DevBuf<int> atom, mol, fbase, shell_off, shell_n, shell_fl;
    DevBuf<long long> pbase, aobase;
};

// A basis of one molecule, or (internally) of a batch of molecules: shells, pairs and quartets
// never couple two molecules, and every n x n matrix of a molecule m is the block
// [mol_base[m], mol_base[m] + n_m^2) of a packed array (row-major, row stride n_m).
struct mess_basis {
    int natom = 0, nbf = 0, nelec = 0;     // totals over the molecules
    int nmol = 1, max_nbf = 0;
    long long packed = 0;                   // sum over molecules of n_m^2
    std::vector<int> Z;
    std::vector<double> xyz;
    std::vector<HostShell> shells;
    std::vector<double> fscale;     // per function: component normalisation relative to x^l
    std::vector<int> f_local;       // per function: index within its molecule
    std::vector<int> mol_nbf, mol_nelec, mol_atom_off, mol_atom_n, mol_shell_off, mol_shell_n;
    std::vector<long long> mol_base;
    std::vector<unsigned char> active;      // per molecule: included in J/K builds
    long long active_version = 0;

    // canonical shell pairs (A, B) within a molecule: l_A > l_B, or l_A == l_B and A >= B
    int npair = 0;
    std::vector<int> pair_a, pair_b, pair_class, pp_off, pp_n, pair_mol;
    std::vector<double> Q;          // Schwarz factor per pair
    // pair lists per (pair class c, primitive-count group g) at index c * MESS_NGROUP + g: pair ids,
    // per molecule sorted by Q descending, with nmol + 1 segment offsets
    std::vector<int> class_list[MESS_NUM_PCLASS * MESS_NGROUP];
    std::vector<int> class_seg[MESS_NUM_PCLASS * MESS_NGROUP];
    DevBuf<int> d_class_list[MESS_NUM_PCLASS * MESS_NGROUP];
    DevBuf<KetRec> d_ketrec[MESS_NUM_PCLASS * MESS_NGROUP];   // the lists' pair records, list order
    std::vector<KetRec> pair_rec;                             // per pair
    DevBuf<KetRec> d_pair_rec;

    DevBuf<PrimPairRec<double>> d_pp64;
    DevBuf<PrimPairRec<float>> d_pp32;
    DevBuf<int> d_pp_off, d_pp_n, d_fa, d_fb, d_same;
    DevBuf<double> d_AB, d_Q, d_Ccen;
    DevBuf<float> d_Qf;            // Schwarz factor per pair in FP32 (density screening)
    DevBuf<float> d_ABf, d_Cf;
    DevBuf<double> d_boys64;
    DevBuf<float> d_boys32;
    DevBuf<float4> d_boys32v;
    DevBuf<int> d_Z;
    DevBuf<double> d_xyz;
    DevBuf<int> d_shell_l, d_shell_K, d_shell_f0, d_shell_poff;
    DevBuf<double> d_shell_R, d_shell_alpha, d_shell_coef, d_fscale;
    DevBuf<int> d_pair_a, d_pair_b, d_pair_mol, d_mol_n, d_mol_atom_off, d_mol_atom_n, d_f_local;
    DevBuf<long long> d_mol_base;

    PairTable<double> P64;
    PairTable<float> P32;
    PairTable<df32> Pdf;
    DevBuf<PrimPairRec<df32>> d_ppdf;
    DevBuf<float2> d_boysdf;
    BinSet bins;
    // reduced-precision copies of the density of the J/K build in flight (allocated with the bins);
    // a build waits on dconv_free (recorded when the previous build's kernels are done) before
    // overwriting them
    DevBuf<float> d_D32;
    DevBuf<float2> d_Ddf;
    cudaEvent_t dconv_free = nullptr;
    std::vector<JKGraph> graphs;   // J/K graphs of repeated builds (at most 4, oldest dropped first)
    DevBuf<double> d_stage;        // D, J, K of the host-buffer J/K build (kept for repeated calls)
    XcState xc;                    // exchange-correlation grid (Kohn-Sham functionals)
    bool gpu_ready = false;        // pair tables and Schwarz factors built (on first use of the basis)
};

// the basis's device data (primitive-pair tables, records, Schwarz factors, class lists), built on
// the first call that needs them; a basis used only inside batches never builds its own (host.cu)
mess_status mess_basis_gpu(mess_basis* b);

// one-electron integrals on the device (one_e.cu)
cudaError_t mess_launch_one_e(const mess_basis* b, double* dS, double* dT, double* dV, cudaStream_t s);
// J/K helpers (jk.cu)
cudaError_t mess_launch_symmetrise_jk(const mess_basis* b, double* J, double* K, cudaStream_t s);
// FP32 and double-float copies of the packed density (either output may be null)
cudaError_t mess_launch_convert_density(const double* D, float* D32, float2* Ddf, long long count, cudaStream_t s);
// Boys tables (boys_table.cu): rows x MESS_BOYS_NCOL
// F_0..F_{NF-1} and exp(-T) at T_k = k * dt, k < nrow (row-major, MESS_BOYS_NCOL columns)
void mess_boys_table(std::vector<double>& tab, int nrow, double dt);
// bins (host.cu)
mess_status mess_ensure_bins(mess_basis* b, double tau, double tau64, int split);
// derivative basis (host.cu) of a single-molecule basis whose shells have l < MESS_LMAX: the shells of b
// (same order, so its functions come first), then for every shell k a raised shell raised[k] (l + 1,
// coefficients 2 alpha_i c_i) and for l > 0 a lowered shell lowered[k] (l - 1, coefficients c_i), -1 if
// none; the derivative of a function of shell k with respect to its centre combines the two
mess_status mess_derivative_basis(const mess_basis* b, mess_basis** out, std::vector<int>& raised,
                                  std::vector<int>& lowered);
// batches (host.cu): one basis over several molecules (copies of the given bases' shells)
mess_status mess_batch_basis(int nmol, const mess_basis* const* bases, mess_basis** out);
void mess_free_basis(mess_basis* b);
// one single-atom molecule (at the origin) per distinct element of b; elements[e] = Z of molecule e
mess_status mess_atoms_basis(const mess_basis* b, std::vector<int>& elements, mess_basis** out);
// A host-only copy of a single-molecule basis with one atom (its nucleus and its shells) moved by dx
// bohr along axis (0 x, 1 y, 2 z); its device data are built on first use like any basis's.
mess_status mess_displaced_basis(const mess_basis* b, int atom, int axis, double dx, mess_basis** out);
// batched SCF on an internal batch basis, final densities into dD (device, packed) (scf.cu)
mess_status mess_scf_batch_density(mess_basis* b, const mess_scf_opts* opts, mess_scf_result* res, double* dD);
// exchange-correlation (xc.cu): the grid and basis-function values of b (once), then for a packed
// density dD the matrix dV (packed, overwritten) and E_xc per molecule (dExc, overwritten) of
// functional kind 1 (LDA) or 2 (PBE); on stream s, no allocation after the first call
mess_status mess_xc_prepare(mess_basis* b, cudaStream_t s);
mess_status mess_xc_eval(mess_basis* b, int kind, const double* dD, double* dV, double* dExc, cudaStream_t s);
void mess_free_xc(mess_basis* b);
// learned guess: predicted D0 of every molecule of b (device, packed) (mlp.cu)
mess_status mess_mlp_guess_device(const mess_mlp* m, const mess_basis* b, double* dD0, cudaStream_t s);
// whether the quartet bins for these options are built (a J/K build with them would not allocate);
// MESS_EINVAL for invalid options (checked first)
mess_status mess_jk_bins_ready(const mess_basis* b, const mess_jk_opts* opts, bool* ready);
// J/K on packed device matrices of (possibly batched) bases (host.cu)
mess_status mess_jk_packed(mess_basis* b, const double* dD, double* dJ, double* dK, const mess_jk_opts* opts,
                           mess_jk_info* info, bool graphs = true);
void mess_free_jk_graphs(mess_basis* b);
// the quartet bins for these options, built if missing (may allocate; not under stream capture)
mess_status mess_jk_ensure_bins(mess_basis* b, const mess_jk_opts* opts);
// the launches of one J/K build on opts->cuda_stream and nothing else: no allocation, no event
// shared with other builds and no cached graph, so that a caller's stream capture can record them.
// The bins for the options must already exist (MESS_EINVAL otherwise).  The caller orders builds
// on one basis (they share its reduced-precision density copies).
mess_status mess_jk_enqueue_only(mess_basis* b, const double* dD, double* dJ, double* dK, const mess_jk_opts* opts);
