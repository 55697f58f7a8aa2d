// Plain-data layouts shared by the host code and the kernels (no torch types anywhere).
#pragma once
#include <stdint.h>

// Boys-function grid: rows k = 0..MESS_BOYS_NROW-1 at T_k = k * MESS_BOYS_DT; columns n = 0..NF-1
// hold F_n(T_k) and column NF holds exp(-T_k).
#define MESS_BOYS_DT 0.1
#define MESS_BOYS_INV_DT 10.0
#define MESS_BOYS_TMAX64 36.0     // FP64 small-T branch below this (Taylor order 7)
#define MESS_BOYS_TMAX32 30.0     // FP32 small-T branch below this (Taylor order 4)
#define MESS_BOYS_NF 16
#define MESS_BOYS_NCOL (MESS_BOYS_NF + 1)
#define MESS_BOYS_NROW 362
#define MESS_BOYS_NL 9            // orders L = 0..8 of the FP32 Taylor rows (L = la+lb+lc+ld <= 8)
// FP32 rows: T_k = k * MESS_BOYS32_DT with a step that FP32 holds exactly (1/16: T_k - T is then
// formed with one rounding; a step of 0.1 or 0.05 rounded to FP32 shifts x by up to 5e-7 at the far
// end of the grid, a one-signed error of up to 1e-7 in F_L); F_L, F_L+1, F_L+2 and exp(-T_k) in one
// 16-byte row (Taylor order 4, F_L+3 and F_L+4 from the upward recursion); rows up to T = MESS_BOYS_TMAX32.
#define MESS_BOYS32_DT 0.0625
#define MESS_BOYS32_INV_DT 16.0
#define MESS_BOYS32_NROW 482

#define MESS_PRIM_EPS 1e-18       // primitive pairs below this weight bound are left out (build_pairs)

#define MESS_LMAX 2               // s, p, Cartesian d
#define MESS_NUM_PCLASS 6         // pair classes (la,lb): ss ps pp ds dp dd
#define MESS_NGROUP 3             // primitive-pair count groups: <= 3, 4..12, >= 13
#define MESS_TEAM_WARPS 4         // warps (one shell quartet each) per block of the large-class kernels

// One primitive pair: zeta, PAx, PAy, PAz (P - A, P the Gaussian product centre), K, 1/(2 zeta), and
// two padding slots: 32 bytes in FP32 (one sector per record), 64 in FP64 and double-float.
template <typename R> struct alignas(32) PrimPairRec { R v[8]; };

// Everything a J/K kernel reads about the ket pair of a quartet, in one 112-byte record (seven 16-byte
// loads at most; the arithmetic reads only the ones it needs).  Stored per pair (pair order) and per
// class list (list order, so that the consecutive kets of consecutive lanes are adjacent).
//   [0]   pp_off, pp_n, fa | fb << 16 (first functions within the molecule), same | mol << 1
//   [16]  C (centre of the pair's first shell) and A - B, FP64
//   [64]  C as FP32 hi[3], lo[3]; A - B in FP32; the pair id
struct alignas(16) KetRec {
    int pp_off, pp_n, fab, flags;
    double C[3], AB[3];
    float Cf[6], ABf[3];
    int pair;
};

// One launch over a class bin (a contiguous range of quartets of one angular class).
struct BinLaunch {
    const int* bra;          // [nbra] pair ids, Q descending
    const int* ket;          // ket list (pair ids, Q descending)
    const KetRec* ketrec;    // the ket list's records, same order
    const long long* offs;   // [nbra + 1] exclusive prefix of ket counts
    const int* kbeg;         // [nbra] first ket index of each bra
    const int* seg;          // [ceil(total / 32)] bra of quartet 32 k (narrows the bra search)
    int nbra;
    long long total;
};
