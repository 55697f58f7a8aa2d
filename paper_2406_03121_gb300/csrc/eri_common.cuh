// Device-side building blocks shared by the generated per-class ERI code and the kernels:
// primitive-pair tables, the Boys function F_m(T), and J/K accumulation helpers.
#pragma once
#include <type_traits>
#include <cuda_runtime.h>
#include <stdint.h>

#include "df32.cuh"
#include "mess_device.h"

// ------------------------------------------------------------------------------------------
// Primitive-pair record (Gaussian product theorem): for primitives alpha on A, beta on B,
//   zeta = alpha + beta,  P = (alpha A + beta B)/zeta,  PA = P - A,
//   K = sqrt(2) pi^{5/4} c_a c_b exp(-alpha beta/zeta |AB|^2) / zeta   (so that K_ab K_cd / sqrt(zeta+eta)
//       is the 2 pi^{5/2}/(zeta eta sqrt(zeta+eta)) prefactor of [00|00]^(m)),
//   oo2z = 1/(2 zeta).
// ------------------------------------------------------------------------------------------
template <typename R> struct PrimPair { R zeta, PAx, PAy, PAz, K, oo2z; };

template <typename R> struct PairTable;

// Conversions between FP64 and FP32 done on the integer ALU: on this GPU the FP64 pipe (which also
// executes F2F / I2F conversions) runs at 1/64 of the FP32 rate, so FP32 kernels avoid it entirely,
// including in rarely taken branches (the compiler predicates them, and a predicated-off FP64-pipe
// instruction still issues).  d2f: round to nearest with ties away from zero, results below 2^-126
// flush to signed zero, overflow and infinities give signed infinity, NaN stays NaN.  f2d: exact; FP32 subnormals flush to zero.
__device__ __forceinline__ float d2f_alu(double d)
{
    const unsigned long long o = (unsigned long long)__double_as_longlong(d);
    const unsigned long long b = o + (1ull << 28);
    const unsigned ohi = (unsigned)(o >> 32);
    const unsigned sign = ohi & 0x80000000u;
    const unsigned hi = (unsigned)(b >> 32);
    const int fe = (int)((hi >> 20) & 0x7ffu) - 896;
    const unsigned mant = (unsigned)((b >> 29) & 0x7fffffu);
    unsigned bits = sign | ((unsigned)fe << 23) | mant;
    bits = fe <= 0 ? sign : bits;
    bits = fe >= 255 ? (sign | 0x7f800000u) : bits;
    bits = ((ohi >> 20) & 0x7ffu) == 0x7ffu ? (sign | 0x7f800000u | ((o << 12) ? 0x400000u : 0u)) : bits;
    return __uint_as_float(bits);
}

__device__ __forceinline__ double f2d_alu(float f)
{
    const unsigned u = __float_as_uint(f);
    const unsigned e = (u >> 23) & 0xffu;
    const unsigned m = u & 0x7fffffu;
    const unsigned sign = u & 0x80000000u;
    unsigned hi = sign | ((e + 896u) << 20) | (m >> 3);
    hi = e == 0u ? sign : hi;
    hi = e == 0xffu ? (sign | 0x7ff00000u | (m >> 3)) : hi;
    const unsigned lo = (e == 0u) ? 0u : (m << 29);
    return __hiloint2double((int)hi, (int)lo);
}

// small non-negative integer to float without I2F: 2^23 + k as bits, minus 2^23 (0 <= k < 2^22)
__device__ __forceinline__ float int_to_f32_alu(int k) { return __int_as_float(0x4B000000 | k) - 8388608.0f; }

template <typename R> __device__ __forceinline__ R small_int(int k);
template <> __device__ __forceinline__ double small_int<double>(int k) { return (double)k; }
template <> __device__ __forceinline__ float small_int<float>(int k) { return int_to_f32_alu(k); }
template <> __device__ __forceinline__ df32 small_int<df32>(int k) { return df32(int_to_f32_alu(k), 0.f); }

// a generated per-integral scale (double with float hi / lo copies) in R
template <typename R> __device__ __forceinline__ R gen_scale(const double* d, const float* hi, const float* lo, int k);
template <> __device__ __forceinline__ double gen_scale<double>(const double* d, const float*, const float*, int k) { return __ldg(d + k); }
template <> __device__ __forceinline__ float gen_scale<float>(const double*, const float* hi, const float*, int k) { return __ldg(hi + k); }
template <> __device__ __forceinline__ df32 gen_scale<df32>(const double*, const float* hi, const float* lo, int k)
{ return df32(__ldg(hi + k), __ldg(lo + k)); }

// double -> double-float: hi rounded to nearest, lo the rounded remainder (one FP64 subtraction)
__device__ __forceinline__ df32::df32(double v)
{
    hi = d2f_alu(v);
    lo = d2f_alu(v - f2d_alu(hi));
}

// density elements: the FP32 and double-float kernels read copies of D converted once per build
__device__ __forceinline__ double ldD(const double* p) { return __ldg(p); }
__device__ __forceinline__ float ldD(const float* p) { return __ldg(p); }
__device__ __forceinline__ df32 ldD(const float2* p) { const float2 v = __ldg(p); return df32(v.x, v.y); }
__device__ __forceinline__ double to_f64(double v) { return v; }
__device__ __forceinline__ double to_f64(float v) { return f2d_alu(v); }
__device__ __forceinline__ double to_f64(df32 v) { return f2d_alu(v.hi) + f2d_alu(v.lo); }

template <typename R> struct PairTable {
    const PrimPairRec<R>* __restrict__ pp;   // [npp]
    const int* __restrict__ pp_off;          // [npair]
    const int* __restrict__ pp_n;            // [npair]
    const double* __restrict__ AB;           // [npair][3]  A - B
    const int* __restrict__ fa;              // [npair] first function of A
    const int* __restrict__ fb;              // [npair] first function of B
    const int* __restrict__ same;            // [npair] 1 if A == B (same shell)
    const double* __restrict__ C;            // [npair][3] centre of the pair's first shell A
    const float* __restrict__ Cf;            // [npair][6] the same as FP32 hi[3], lo[3] (C = hi + lo)
    const float* __restrict__ ABf;           // [npair][3] A - B in FP32
    const int* __restrict__ mol;             // [npair] molecule of the pair (batched bases)
    const long long* __restrict__ mbase;     // [nmol] offset of the molecule's n x n block (packed matrices)
    const int* __restrict__ mn;              // [nmol] basis functions of the molecule (row stride)
    const double* __restrict__ boys64;       // Boys grid, FP64
    const float* __restrict__ boys32;        // Boys grid, FP32
    const float4* __restrict__ boys32v;      // FP32 rows per order L: [L][row] {F_L, F_L+1, F_L+2, exp(-T_k)}
    const float2* __restrict__ boysdf;       // Boys grid, double-float (hi, lo)
    // per molecule: 0 = left the computation (a converged molecule of a batched SCF): its quartets
    // are skipped by the J/K kernels.  Null: every molecule takes part.
    const unsigned char* __restrict__ active = nullptr;
    // Density-weighted screening of a build (null dmax: none): a shell quartet is skipped when
    // Q_ab Q_cd max(dmax_ab, dmax_cd) < dtau, with dmax_p the largest |D_mn| over the rows m of the
    // two shells of pair p.  Every density element a quartet's J/K terms read lies in one of those
    // rows, so each skipped contribution is below dtau (the incremental Fock builds of an SCF, whose
    // density changes shrink as it converges).
    const KetRec* __restrict__ rec = nullptr;   // per pair (pair order)
    const float* __restrict__ Qf = nullptr;     // Schwarz factor per pair (FP32)
    const float* __restrict__ dmax = nullptr;
    float dtau = 0.f;

    __device__ __forceinline__ bool live(int pair) const { return !active || __ldg(active + __ldg(mol + pair)) != 0; }
    __device__ __forceinline__ bool dens_ok(int bp, int kp) const
    {
        return !dmax || __ldg(Qf + bp) * __ldg(Qf + kp) * fmaxf(__ldg(dmax + bp), __ldg(dmax + kp)) >= dtau;
    }

    __device__ __forceinline__ PrimPair<R> load(int i) const
    {
        const PrimPairRec<R>& r = pp[i];
        PrimPair<R> o;
        o.zeta = r.v[0]; o.PAx = r.v[1]; o.PAy = r.v[2]; o.PAz = r.v[3];
        o.K = r.v[4]; o.oo2z = r.v[5];
        return o;
    }
};

// A - C between the first shells of two pairs, and A - B of one pair, in R.  FP32 forms the
// difference from hi/lo parts, so it is accurate relative to |A - C|, not to |A|.
__device__ __forceinline__ double pair_ac(const PairTable<double>& P, int bp, int kp, int x)
{
    return P.C[3 * bp + x] - P.C[3 * kp + x];
}
__device__ __forceinline__ float pair_ac(const PairTable<float>& P, int bp, int kp, int x)
{
    return (__ldg(P.Cf + 6 * bp + x) - __ldg(P.Cf + 6 * kp + x)) + (__ldg(P.Cf + 6 * bp + 3 + x) - __ldg(P.Cf + 6 * kp + 3 + x));
}
__device__ __forceinline__ df32 pair_ac(const PairTable<df32>& P, int bp, int kp, int x)
{
    const df32 h = df_two_sum(__ldg(P.Cf + 6 * bp + x), -__ldg(P.Cf + 6 * kp + x));
    const df32 l = df_two_sum(__ldg(P.Cf + 6 * bp + 3 + x), -__ldg(P.Cf + 6 * kp + 3 + x));
    return h + l;
}
__device__ __forceinline__ double pair_ab(const PairTable<double>& P, int p, int x) { return P.AB[3 * p + x]; }
__device__ __forceinline__ df32 pair_ab(const PairTable<df32>& P, int p, int x) { return df32(P.AB[3 * p + x]); }
__device__ __forceinline__ float pair_ab(const PairTable<float>& P, int p, int x) { return __ldg(P.ABf + 3 * p + x); }

// The ket side of a quartet as the recursion needs it: its primitive range, A - C (bra first centre
// minus ket first centre, formed as in pair_ac) and C - D, from the ket's record.
template <typename R> struct KetView {
    int k0, nk;
    R AC[3], CD[3];
};

__device__ __forceinline__ int4 ket_hdr(const KetRec* r) { return __ldg(reinterpret_cast<const int4*>(r)); }

__device__ __forceinline__ KetView<double> ket_view(const PairTable<double>& P, int bp, const KetRec* r, int4 h)
{
    KetView<double> v;
    v.k0 = h.x;
    v.nk = h.y;
    const double2 c01 = __ldg(reinterpret_cast<const double2*>(r) + 1);
    const double2 c2a0 = __ldg(reinterpret_cast<const double2*>(r) + 2);
    const double2 a12 = __ldg(reinterpret_cast<const double2*>(r) + 3);
    v.AC[0] = __ldg(P.C + 3 * bp) - c01.x;
    v.AC[1] = __ldg(P.C + 3 * bp + 1) - c01.y;
    v.AC[2] = __ldg(P.C + 3 * bp + 2) - c2a0.x;
    v.CD[0] = c2a0.y; v.CD[1] = a12.x; v.CD[2] = a12.y;
    return v;
}
__device__ __forceinline__ KetView<float> ket_view(const PairTable<float>& P, int bp, const KetRec* r, int4 h)
{
    KetView<float> v;
    v.k0 = h.x;
    v.nk = h.y;
    const float4 f0 = __ldg(reinterpret_cast<const float4*>(r) + 4);   // Cf hi x y z, lo x
    const float4 f1 = __ldg(reinterpret_cast<const float4*>(r) + 5);   // lo y z, ABf x y
    const float4 f2 = __ldg(reinterpret_cast<const float4*>(r) + 6);   // ABf z, pair
    const float* cb = P.Cf + 6 * bp;
    v.AC[0] = (__ldg(cb) - f0.x) + (__ldg(cb + 3) - f0.w);
    v.AC[1] = (__ldg(cb + 1) - f0.y) + (__ldg(cb + 4) - f1.x);
    v.AC[2] = (__ldg(cb + 2) - f0.z) + (__ldg(cb + 5) - f1.y);
    v.CD[0] = f1.z; v.CD[1] = f1.w; v.CD[2] = f2.x;
    return v;
}
__device__ __forceinline__ KetView<df32> ket_view(const PairTable<df32>& P, int bp, const KetRec* r, int4 h)
{
    KetView<df32> v;
    v.k0 = h.x;
    v.nk = h.y;
    const float4 f0 = __ldg(reinterpret_cast<const float4*>(r) + 4);
    const float4 f1 = __ldg(reinterpret_cast<const float4*>(r) + 5);
    const float* cb = P.Cf + 6 * bp;
    const float kh[3] = {f0.x, f0.y, f0.z}, kl[3] = {f0.w, f1.x, f1.y};
#pragma unroll
    for (int x = 0; x < 3; ++x) {
        const df32 hi = df_two_sum(__ldg(cb + x), -kh[x]);
        const df32 lo = df_two_sum(__ldg(cb + 3 + x), -kl[x]);
        v.AC[x] = hi + lo;
    }
    const double2 c2a0 = __ldg(reinterpret_cast<const double2*>(r) + 2);
    const double2 a12 = __ldg(reinterpret_cast<const double2*>(r) + 3);
    v.CD[0] = df32(c2a0.y); v.CD[1] = df32(a12.x); v.CD[2] = df32(a12.y);
    return v;
}
__device__ __forceinline__ int ket_pair(const KetRec* r) { return __ldg(&r->pair); }

// ------------------------------------------------------------------------------------------
// Boys function F_m(T) = int_0^1 t^{2m} exp(-T t^2) dt, m = 0..L.
// Grid tables tab[k][n] = F_n(k dT) for n = 0..MESS_BOYS_NF-1 and tab[k][MESS_BOYS_NF] = exp(-k dT).
//   small T: Taylor expansion about the nearest grid point, F_n(T) = sum_j F_{n+j}(T_k) (-x)^j / j!,
//            x = T - T_k (|x| <= dT/2), for the highest order L, then the stable downward recursion
//            F_{m-1} = (2 T F_m + exp(-T)) / (2m - 1);
//   large T: F_0 = (1/2) sqrt(pi/T) (erf(sqrt T) = 1 to working precision there) and the upward
//            recursion F_{m+1} = ((2m+1) F_m - exp(-T)) / (2T), stable for large T.
// BMODE 0: everything in FP64.  BMODE 1: FP64 for T < MESS_BOYS_TMAX64 (small-T Taylor + downward
// recursion), FP32 asymptote above it.  BMODE 2: everything in FP32.
// ------------------------------------------------------------------------------------------
template <int L> __device__ __forceinline__ void boys_small_f64(double T, double* F, const double* __restrict__ c_boys64)
{
    const int k = __double2int_rn(T * MESS_BOYS_INV_DT);
    const double x = (double)k * MESS_BOYS_DT - T;      // = -(T - T_k)
    const double* row = c_boys64 + (size_t)k * MESS_BOYS_NCOL;
    if (L == 0) {
        double s = __ldg(row + 7);
#pragma unroll
        for (int j = 7; j >= 1; --j) s = __ldg(row + j - 1) + s * x * (1.0 / j);
        F[0] = s;
        return;
    }
    double s = __ldg(row + L + 7);
#pragma unroll
    for (int j = 7; j >= 1; --j) s = __ldg(row + L + j - 1) + s * x * (1.0 / j);
    F[L] = s;
    // exp(-T) = exp(-T_k) * exp(x), exp(x) by its Taylor series (|x| <= 0.05)
    double ex = 1.0 + x * (1.0 + x * (1.0 / 2 + x * (1.0 / 6 + x * (1.0 / 24 + x * (1.0 / 120
                + x * (1.0 / 720 + x * (1.0 / 5040 + x * (1.0 / 40320))))))));
    const double e = __ldg(row + MESS_BOYS_NF) * ex;
    const double t2 = 2.0 * T;
#pragma unroll
    for (int m = L; m >= 1; --m) F[m - 1] = (t2 * F[m] + e) * (1.0 / (2 * m - 1));
}

template <int L> __device__ __forceinline__ void boys_large_f64(double T, double* F)
{
    const double rt = rsqrt(T);
    F[0] = 0.886226925452758014 * rt;   // sqrt(pi)/2 / sqrt(T)
    if (L > 0) {
        const double e = exp(-T);
        const double h = 0.5 * rt * rt;
#pragma unroll
        for (int m = 0; m < L; ++m) F[m + 1] = ((2 * m + 1) * F[m] - e) * h;
    }
}

template <int L> __device__ __forceinline__ void boys_small_f32(float T, float* F, const float4* __restrict__ tabv)
{
    // nearest grid index without F2I / I2F conversions (those issue on the slow FP64 pipe): adding
    // 1.5 * 2^23 rounds T / dT to an integer held in the low mantissa bits (0 <= T / dT < 2^22)
    const float r = fmaf(T, (float)MESS_BOYS32_INV_DT, 12582912.0f);
    const int k = __float_as_int(r) - 0x4B400000;
    const float kf = r - 12582912.0f;                  // k as a float, exactly
    const float x = kf * (float)MESS_BOYS32_DT - T;    // T_k - T (T_k exact), |x| <= 1/32
    // One 16-byte row: F_L, F_L+1, F_L+2 and exp(-T_k), each rounded once from the FP64 grid.
    // F_L+3 and F_L+4 at T_k for the third- and fourth-order terms (at most 5e-6 and 4e-8 of F_L,
    // so a few correct digits suffice; the fourth is kept because dropping it would bias every FP32
    // integral with one sign) come from the upward recursion F_m+1 = ((2m+1) F_m - exp(-T_k)) / (2 T_k),
    // F_m(0) = 1/(2m+1) at the first grid point.
    const float4 a = __ldg(tabv + (size_t)L * MESS_BOYS32_NROW + k);
    const float ek = a.w;
    float f3, f4;
    if (k > 0) {
        const float h = __fdividef(0.5f * (float)MESS_BOYS32_INV_DT, kf);   // 1 / (2 T_k)
        f3 = ((float)(2 * L + 5) * a.z - ek) * h;
        f4 = ((float)(2 * L + 7) * f3 - ek) * h;
    } else {
        f3 = 1.0f / (float)(2 * L + 7);
        f4 = 1.0f / (float)(2 * L + 9);
    }
    float s = f4;
    s = f3 + s * x * 0.25f;
    s = a.z + s * x * (1.0f / 3);
    s = a.y + s * x * 0.5f;
    s = a.x + s * x;
    F[L] = s;
    if (L == 0) return;
    // exp(-T) = exp(-T_k) exp(x), exp(x) to fourth order (|x| <= 1/32: the next term is below 2e-9)
    const float e = ek * (1.0f + x * (1.0f + x * (0.5f + x * (1.0f / 6 + x * (1.0f / 24)))));
    const float t2 = 2.0f * T;
#pragma unroll
    for (int m = L; m >= 1; --m) F[m - 1] = (t2 * F[m] + e) * (1.0f / (2 * m - 1));
}

template <int L> __device__ __forceinline__ void boys_large_f32(float T, float* F)
{
    const float rt = rsqrtf(T);
    F[0] = 0.886226925f * rt;
    if (L > 0) {
        const float e = __expf(-T);
        const float h = 0.5f * rt * rt;
#pragma unroll
        for (int m = 0; m < L; ++m) F[m + 1] = ((2 * m + 1) * F[m] - e) * h;
    }
}

// double-float Boys: the same grid expansion and recursions in df32 arithmetic (grid in hi/lo
// pairs); above the grid F_0 = sqrt(pi)/2 T^-1/2 and the upward recursion, whose exp(-T) term
// (below 3e-16 there) is taken in FP32.
__device__ __forceinline__ df32 df_inv_int(int j)   // 1/j as double-float
{
    const float h = 1.0f / (float)j;
    return df32(h, fmaf(-h, (float)j, 1.0f) / (float)j);
}

template <int L> __device__ __forceinline__ void boys_small_df(df32 T, df32* F, const float2* __restrict__ tab)
{
    const float r = fmaf(T.hi, (float)MESS_BOYS_INV_DT, 12582912.0f);
    const int k = __float_as_int(r) - 0x4B400000;
    const df32 dt(0.1f, -1.490116119384765625e-9f);   // 0.1 = hi + lo to 48 bits
    const df32 x = df32(k) * dt - T;                  // T_k - T
    const float2* row = tab + (size_t)k * MESS_BOYS_NCOL;
    const float2 t7 = __ldg(row + L + 7);
    df32 s(t7.x, t7.y);
#pragma unroll
    for (int j = 7; j >= 1; --j) {
        const float2 tj = __ldg(row + L + j - 1);
        s = df32(tj.x, tj.y) + s * x * df_inv_int(j);
    }
    F[L] = s;
    if (L == 0) return;
    df32 ex = df32(1.0f, 0.f);
#pragma unroll
    for (int j = 9; j >= 1; --j) ex = df32(1.0f, 0.f) + x * df_inv_int(j) * ex;
    const float2 te = __ldg(row + MESS_BOYS_NF);
    const df32 e = df32(te.x, te.y) * ex;
    const df32 t2 = T + T;
#pragma unroll
    for (int m = L; m >= 1; --m) F[m - 1] = (t2 * F[m] + e) * df_inv_int(2 * m - 1);
}

template <int L> __device__ __forceinline__ void boys_large_df(df32 T, df32* F)
{
    const df32 rt = df32(1.0f, 0.f) / df_sqrt(T);
    F[0] = df32(0.8862269520759583f, -2.6623199644859596e-08f) * rt;   // sqrt(pi)/2 = 0.88622692545275801 as hi + lo
    if (L > 0) {
        const df32 e(__expf(-T.hi), 0.f);
        const df32 h = df32(0.5f, 0.f) / T;
#pragma unroll
        for (int m = 0; m < L; ++m) F[m + 1] = (df32(2 * m + 1) * F[m] - e) * h;
    }
}

template <typename R> struct PairTable;
template <typename R, int L, int BMODE>
__device__ __forceinline__ void boys_eval(R T, R* F, const PairTable<R>& P);

template <> __device__ __forceinline__ void boys_eval<double, 0, 0>(double T, double* F, const PairTable<double>& P)
{ if (T < MESS_BOYS_TMAX64) boys_small_f64<0>(T, F, P.boys64); else boys_large_f64<0>(T, F); }

#define MESS_BOYS_SPECIALISE(LL)                                                                  \
    template <> __device__ __forceinline__ void boys_eval<double, LL, 0>(double T, double* F,     \
                                                                        const PairTable<double>& P) \
    { if (T < MESS_BOYS_TMAX64) boys_small_f64<LL>(T, F, P.boys64); else boys_large_f64<LL>(T, F); } \
    template <> __device__ __forceinline__ void boys_eval<float, LL, 1>(float T, float* F,        \
                                                                       const PairTable<float>& P) \
    {                                                                                             \
        if (T < (float)MESS_BOYS_TMAX64) {                                                        \
            double Fd[LL + 1];                                                                    \
            boys_small_f64<LL>((double)T, Fd, P.boys64);                                          \
            _Pragma("unroll") for (int m = 0; m <= LL; ++m) F[m] = (float)Fd[m];                  \
        } else {                                                                                  \
            boys_large_f32<LL>(T, F);                                                             \
        }                                                                                         \
    }                                                                                             \
    template <> __device__ __forceinline__ void boys_eval<float, LL, 2>(float T, float* F,        \
                                                                       const PairTable<float>& P) \
    { if (T < (float)MESS_BOYS_TMAX32) boys_small_f32<LL>(T, F, P.boys32v); else boys_large_f32<LL>(T, F); } \
    template <> __device__ __forceinline__ void boys_eval<df32, LL, 3>(df32 T, df32* F,           \
                                                                      const PairTable<df32>& P)   \
    { if (T < MESS_BOYS_TMAX64) boys_small_df<LL>(T, F, P.boysdf); else boys_large_df<LL>(T, F); }

MESS_BOYS_SPECIALISE(1)
MESS_BOYS_SPECIALISE(2)
MESS_BOYS_SPECIALISE(3)
MESS_BOYS_SPECIALISE(4)
MESS_BOYS_SPECIALISE(5)
MESS_BOYS_SPECIALISE(6)
MESS_BOYS_SPECIALISE(7)
MESS_BOYS_SPECIALISE(8)

template <> __device__ __forceinline__ void boys_eval<float, 0, 1>(float T, float* F, const PairTable<float>& P)
{
    if (T < (float)MESS_BOYS_TMAX64) { double Fd[1]; boys_small_f64<0>((double)T, Fd, P.boys64); F[0] = (float)Fd[0]; }
    else boys_large_f32<0>(T, F);
}
template <> __device__ __forceinline__ void boys_eval<float, 0, 2>(float T, float* F, const PairTable<float>& P)
{ if (T < (float)MESS_BOYS_TMAX32) boys_small_f32<0>(T, F, P.boys32v); else boys_large_f32<0>(T, F); }
template <> __device__ __forceinline__ void boys_eval<df32, 0, 3>(df32 T, df32* F, const PairTable<df32>& P)
{ if (T < MESS_BOYS_TMAX64) boys_small_df<0>(T, F, P.boysdf); else boys_large_df<0>(T, F); }

// 1/(zeta + eta) and its square root (the prefactor's 1/sqrt(zeta + eta)).  FP32: one reciprocal
// square root (a few ulp, within the FP32 path's rounding) instead of a division and a square root.
__device__ __forceinline__ void recip_and_sqrt(double s, double& rz, double& sq) { rz = 1.0 / s; sq = sqrt(rz); }
__device__ __forceinline__ void recip_and_sqrt(float s, float& rz, float& sq) { sq = rsqrtf(s); rz = sq * sq; }
__device__ __forceinline__ void recip_and_sqrt(df32 s, df32& rz, df32& sq) { rz = df32(1.0f, 0.f) / s; sq = df_sqrt(rz); }

// primitive loops of the straight-line FP32 kernels run two primitive quartets per iteration (more
// independent loads in flight); FP64 and double-float keep one (register pressure)
template <typename R> struct PrimUnroll { static constexpr int value = 1; };
template <> struct PrimUnroll<float> { static constexpr int value = 2; };


// ------------------------------------------------------------------------------------------
// J/K accumulation.  For a unique shell quartet (ab|cd) (pair ab >= pair cd, a >= b, c >= d by
// the canonical pair order) with degeneracy weight s = (1/2)^{[a=b] + [c=d] + [ab=cd]}:
//   Jacc_ab += s sum_cd I D_cd,   Jacc_cd += s sum_ab I D_ab,
//   Kacc_ac += s sum_bd I D_bd,   Kacc_ad += s sum_bc I D_bc,
//   Kacc_bc += s sum_ad I D_ad,   Kacc_bd += s sum_ac I D_ac,
// and afterwards J = 2 (Jacc + Jacc^T), K = Kacc + Kacc^T.  This visits each of the 8 index
// permutations of every function quartet exactly once for a symmetric D.
// ------------------------------------------------------------------------------------------
template <typename R> struct DigestCtx {
    const typename DElem<R>::T* __restrict__ D;
    double* __restrict__ J;
    double* __restrict__ K;
    int n;
    int fa, fb, fc, fd;
    bool warp_reduce_ab;   // all 32 lanes share the bra pair: reduce J_ab across the warp first
};

__device__ __forceinline__ float shfl_xor(float v, int o) { return __shfl_xor_sync(0xffffffffu, v, o); }
__device__ __forceinline__ double shfl_xor(double v, int o) { return __shfl_xor_sync(0xffffffffu, v, o); }
__device__ __forceinline__ df32 shfl_xor(df32 v, int o) { return df_shfl_xor(v, o); }

// sum over aligned groups of G consecutive lanes (G a power of two); every lane of the warp takes part
template <int G, typename R> __device__ __forceinline__ R group_sum(R v)
{
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) v += shfl_xor(v, o);
    return v;
}

template <typename R> __device__ __forceinline__ R warp_sum(R v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += shfl_xor(v, o);
    return v;
}

template <typename R>
__device__ __forceinline__ void jk_add(double* __restrict__ M, size_t idx, R v, bool warp_reduce)
{
    if (warp_reduce) {
        v = warp_sum(v);
        if ((threadIdx.x & 31) == 0) atomicAdd(M + idx, to_f64(v));
    } else {
        if (v != R(0)) atomicAdd(M + idx, to_f64(v));
    }
}

// ------------------------------------------------------------------------------------------
// Work decomposition of one class bin: bra pairs i (sorted by Q descending), each with a
// contiguous ket range [kbeg[i], kbeg[i] + offs[i+1] - offs[i]) of the ket list.  A flat quartet
// index q maps to (i, j) by a binary search over offs.
// ------------------------------------------------------------------------------------------
// bra of flat quartet q: the largest i with offs[i] <= q, searched between the bras of quartets
// 32 floor(q / 32) and 32 (floor(q / 32) + 1) (a few steps instead of a search over all bras)
__device__ __forceinline__ int find_bra(const BinLaunch& b, long long q)
{
    const long long k = q >> 5;
    int lo = __ldg(b.seg + k);
    int hi = ((k + 1) << 5) < b.total ? __ldg(b.seg + k + 1) : b.nbra - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(b.offs + mid) <= q) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ bool warp_uniform_int(int v)
{
    const int v0 = __shfl_sync(0xffffffffu, v, 0);
    return __all_sync(0xffffffffu, v == v0);
}

#define MESS_THREADS 128

// JK kernel of one class: G consecutive lanes per shell quartet of the bin (G = 1: one thread).
#define MESS_DEFINE_CLASS_KERNELS(TAG, NA, NB, NC, ND)                                             \
    template <typename R, int BMODE, int G>                                                         \
    __global__ void __launch_bounds__(MESS_THREADS)                                                 \
    k_jk_##TAG(const BinLaunch b, const PairTable<R> P, const typename DElem<R>::T* __restrict__ D,            \
               double* __restrict__ J, double* __restrict__ K, int n)                               \
    {                                                                                               \
        const long long t0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;                     \
        const long long q0 = t0 / G;                                                                \
        const int g = (int)(t0 % G);                                                                \
        const bool valid = q0 < b.total;                                                            \
        const long long q = valid ? q0 : b.total - 1;                                               \
        const int i = find_bra(b, q);                                                  \
        const int j = __ldg(b.kbeg + i) + (int)(q - __ldg(b.offs + i));                            \
        const int bp = __ldg(b.bra + i);                                                            \
        const KetRec* kr = b.ketrec + j;                                                            \
        const int4 kh = ket_hdr(kr);                                                                \
        const int kp = ket_pair(kr);                                                                \
        /* quartets past the end or of a molecule that has left: no work; a warp without any    */ \
        /* quartet to do leaves (lanes of a group share the quartet, so groups leave together)  */ \
        const bool live = valid && P.live(bp) && P.dens_ok(bp, kp);                                 \
        if (__all_sync(0xffffffffu, !live)) return;                                                 \
        R I[(NA) * (NB) * (NC) * (ND)];                                                             \
        eri_##TAG<R, BMODE, G>(P, bp, ket_view(P, bp, kr, kh), g, I, live);                        \
        DigestCtx<R> c;                                                                              \
        {                                                                                           \
            const int m_ = __ldg(P.mol + bp);                                                       \
            const long long o_ = __ldg(P.mbase + m_);                                               \
            c.D = D + o_; c.J = J + o_; c.K = K + o_; c.n = __ldg(P.mn + m_);                       \
        }                                                                                           \
        (void)n;                                                                                    \
        c.fa = __ldg(P.fa + bp); c.fb = __ldg(P.fb + bp);                                           \
        c.fc = kh.z & 0xffff; c.fd = kh.z >> 16;                                                    \
        R s = live ? R(1) : R(0);                                                                   \
        if (__ldg(P.same + bp)) s *= R(0.5);                                                        \
        if (kh.w & 1) s *= R(0.5);                                                                  \
        if (bp == kp) s *= R(0.5);                                                                  \
        if (G == 1) {                                                                               \
            c.warp_reduce_ab = warp_uniform_int(bp);                                                \
            digest_##TAG<R>(I, c, s);                                                               \
        } else if (g == 0) {                                                                        \
            c.warp_reduce_ab = false;                                                               \
            digest_##TAG<R>(I, c, s);                                                               \
        }                                                                                           \
    }                                                                                               \
    /* every integral of the bin written to a dense n^4 tensor, all 8 index permutations */         \
    __global__ void __launch_bounds__(MESS_THREADS)                                                 \
    k_store_##TAG(const BinLaunch b, const PairTable<double> P, double* __restrict__ G, int n)      \
    {                                                                                               \
        const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;                      \
        if (q >= b.total) return;                                                                   \
        const int i = find_bra(b, q);                                                  \
        const int j = b.kbeg[i] + (int)(q - b.offs[i]);                                             \
        const int bp = b.bra[i], kp = b.ket[j];                                                     \
        double I[(NA) * (NB) * (NC) * (ND)];                                                        \
        eri_##TAG<double, 0, 1>(P, bp, ket_view(P, bp, P.rec + kp, ket_hdr(P.rec + kp)), 0, I);     \
        const int fa = P.fa[bp], fb = P.fb[bp], fc = P.fa[kp], fd = P.fb[kp];                       \
        const size_t nn = (size_t)n;                                                                \
        for (int ia = 0; ia < (NA); ++ia)                                                           \
            for (int ib = 0; ib < (NB); ++ib)                                                       \
                for (int ic = 0; ic < (NC); ++ic)                                                   \
                    for (int id = 0; id < (ND); ++id) {                                             \
                        const double v = I[((ia * (NB) + ib) * (NC) + ic) * (ND) + id];             \
                        const size_t a = fa + ia, bb = fb + ib, c = fc + ic, d = fd + id;           \
                        G[((a * nn + bb) * nn + c) * nn + d] = v;                                   \
                        G[((bb * nn + a) * nn + c) * nn + d] = v;                                   \
                        G[((a * nn + bb) * nn + d) * nn + c] = v;                                   \
                        G[((bb * nn + a) * nn + d) * nn + c] = v;                                   \
                        G[((c * nn + d) * nn + a) * nn + bb] = v;                                   \
                        G[((d * nn + c) * nn + a) * nn + bb] = v;                                   \
                        G[((c * nn + d) * nn + bb) * nn + a] = v;                                   \
                        G[((d * nn + c) * nn + bb) * nn + a] = v;                                   \
                    }                                                                               \
    }

// Schwarz factors Q_ab = sqrt(max_{m in a, n in b} |(mn|mn)|) for a list of pairs of one class.
#define MESS_DEFINE_SCHWARZ_KERNEL(TAG, NA, NB)                                                    \
    __global__ void __launch_bounds__(MESS_THREADS)                                                 \
    k_schwarz_##TAG(const int* __restrict__ pairs, int npairs, const PairTable<double> P,           \
                    double* __restrict__ Q)                                                         \
    {                                                                                               \
        const int t = blockIdx.x * blockDim.x + threadIdx.x;                                        \
        if (t >= npairs) return;                                                                    \
        const int p = pairs[t];                                                                     \
        double I[(NA) * (NB) * (NA) * (NB)];                                                        \
        eri_##TAG<double, 0, 1>(P, p, ket_view(P, p, P.rec + p, ket_hdr(P.rec + p)), 0, I);         \
        double m = 0.0;                                                                             \
        for (int ia = 0; ia < (NA); ++ia)                                                           \
            for (int ib = 0; ib < (NB); ++ib)                                                       \
                m = fmax(m, fabs(I[((ia * (NB) + ib) * (NA) + ia) * (NB) + ib]));                   \
        Q[p] = sqrt(m);                                                                             \
    }

// ------------------------------------------------------------------------------------------
// Op-program evaluation of one shell quartet (large angular classes).  The program is the same
// VRR / HRR sequence as the straight-line code, with values packed into NV / NH slots:
//   VRR op (uint4): x = kind | dir<<2 | m1<<4 | m2<<8 | target<<16, y = s1 | s2<<16,
//                   z = s3 | s4<<16, w = s5
//     kind 0: V[t] = F[s1] (base [00|00]^(m), prefactor included)
//     kind 1: V[t] = PA_d V[s1] + WP_d V[s2] + m1/(2 zeta) (V[s3] - rho/zeta V[s4])
//     kind 2: V[t] = QC_d V[s1] + WQ_d V[s2] + m1/(2 eta) (V[s3] - rho/eta V[s4])
//                    + m2/(2(zeta+eta)) V[s5]
//     kind 3: H[s1] += V[t]  (contraction into [e0|f0])
//   HRR op (uint2): x = target | dir<<16 | side<<18, y = s1 | s2<<16:
//     H[t] = H[s1] + X_d H[s2],  X = A - B (side 0) or C - D (side 1)
//   I[k] = fscale[k] * H[fslot[k]]  (per-component normalisation)
// Every thread runs the same op sequence, so the kind / direction branches are warp-uniform.
// ------------------------------------------------------------------------------------------
template <typename R> __device__ __forceinline__ R pick3(int d, R x, R y, R z)
{
    return d == 0 ? x : (d == 1 ? y : z);
}

template <typename R, int BMODE, int L, int NV, int NH, int NACC, int NVOPS, int NHOPS, int NINT>
__device__ __forceinline__ void eri_program(const PairTable<R>& P, int bp, const KetView<R>& kv,
                                            const uint4* __restrict__ vprog, const uint2* __restrict__ hprog,
                                            const int* __restrict__ fslot, const double* __restrict__ fscale,
                                            const float* __restrict__ fscale_hi, const float* __restrict__ fscale_lo,
                                            R* I, bool live)
{
    R V[NV];
    R H[NH];
#pragma unroll 1
    for (int k = 0; k < NACC; ++k) H[k] = R(0);
    const int b0 = P.pp_off[bp], b1 = b0 + (live ? P.pp_n[bp] : 0);
    const int k0 = kv.k0, k1 = k0 + kv.nk;
    const R ACx = kv.AC[0], ACy = kv.AC[1], ACz = kv.AC[2];
    // ket primitives outside (per-lane records read once), bra primitives inside (the same for the warp)
#pragma unroll 1
    for (int ik = k0; ik < (live ? k1 : k0); ++ik) {
        const PrimPair<R> pk = P.load(ik);
#pragma unroll 1
        for (int ib = b0; ib < b1; ++ib) {
            const PrimPair<R> pb = P.load(ib);
            R rz, srz;
            recip_and_sqrt(pb.zeta + pk.zeta, rz, srz);
            const R roz = pk.zeta * rz, roe = pb.zeta * rz, oo2ze = R(0.5) * rz;
            const R PQx = pb.PAx - pk.PAx + ACx, PQy = pb.PAy - pk.PAy + ACy, PQz = pb.PAz - pk.PAz + ACz;
            const R WPx = -roz * PQx, WPy = -roz * PQy, WPz = -roz * PQz;
            const R WQx = roe * PQx, WQy = roe * PQy, WQz = roe * PQz;
            const R T = pb.zeta * roz * (PQx * PQx + PQy * PQy + PQz * PQz);
            const R pref = pb.K * pk.K * srz;
            R F[L + 1];
            boys_eval<R, L, BMODE>(T, F, P);
#pragma unroll
            for (int m = 0; m <= L; ++m) F[m] *= pref;
#pragma unroll 1
            for (int o = 0; o < NVOPS; ++o) {
                const uint4 w = __ldg(vprog + o);
                const int kind = w.x & 3, d = (w.x >> 2) & 3;
                const int m1 = (w.x >> 4) & 15, m2 = (w.x >> 8) & 15, t = w.x >> 16;
                const int s1 = w.y & 0xffff, s2 = w.y >> 16;
                if (kind == 0) {
                    R f = F[0];
#pragma unroll
                    for (int m = 1; m <= L; ++m) f = (s1 == m) ? F[m] : f;
                    V[t] = f;
                } else if (kind == 3) {
                    H[s1] += V[t];
                } else {
                    R v;
                    if (kind == 1) {
                        v = pick3(d, pb.PAx, pb.PAy, pb.PAz) * V[s1] + pick3(d, WPx, WPy, WPz) * V[s2];
                        if (m1) v += small_int<R>(m1) * pb.oo2z * (V[w.z & 0xffff] - roz * V[w.z >> 16]);
                    } else {
                        v = pick3(d, pk.PAx, pk.PAy, pk.PAz) * V[s1] + pick3(d, WQx, WQy, WQz) * V[s2];
                        if (m1) v += small_int<R>(m1) * pk.oo2z * (V[w.z & 0xffff] - roe * V[w.z >> 16]);
                        if (m2) v += small_int<R>(m2) * oo2ze * V[w.w];
                    }
                    V[t] = v;
                }
            }
        }
    }
    const R ABx = pair_ab(P, bp, 0), ABy = pair_ab(P, bp, 1), ABz = pair_ab(P, bp, 2);
    const R CDx = kv.CD[0], CDy = kv.CD[1], CDz = kv.CD[2];
#pragma unroll 1
    for (int o = 0; o < NHOPS; ++o) {
        const uint2 w = __ldg(hprog + o);
        const int t = w.x & 0xffff, d = (w.x >> 16) & 3, side = (w.x >> 18) & 1;
        const R X = side ? pick3(d, CDx, CDy, CDz) : pick3(d, ABx, ABy, ABz);
        H[t] = H[w.y & 0xffff] + X * H[w.y >> 16];
    }
#pragma unroll 1
    for (int k = 0; k < NINT; ++k) I[k] = gen_scale<R>(fscale, fscale_hi, fscale_lo, k) * H[__ldg(fslot + k)];
}


// ------------------------------------------------------------------------------------------
// Warp-per-quartet J/K kernel for the large classes: the 32 lanes of a warp run the independent
// ops of one dependency level of the level-scheduled program in parallel (values in shared
// memory, __syncwarp between levels), then split the digestion outputs between them.
// ------------------------------------------------------------------------------------------

// TW threads share one shell quartet: 32 (a warp, MESS_TEAM_WARPS quartets per block) or
// 32 * MESS_TEAM_WARPS (the whole block on one quartet, for parts with very few quartets)
template <int TW> __device__ __forceinline__ void team_sync()
{
    if (TW == 32) __syncwarp();
    else __syncthreads();
}

// PS (with TW = the block): the block's warps split the quartet's primitive quartets, each warp
// accumulating into its own copy of the contracted values, summed before the HRR.
template <typename R, int BMODE, int TW, int PS, int L, int NVI, int NH, int NACC, int NVL, int NHL, int NINT,
          int NA, int NB, int NC, int ND>
__device__ __forceinline__ void jk_team_body(const BinLaunch& b, const PairTable<R>& P, const typename DElem<R>::T* __restrict__ D,
                                             double* __restrict__ J, double* __restrict__ K, int n,
                                             const uint4* __restrict__ vprog, const int* __restrict__ vlev,
                                             const uint2* __restrict__ hprog, const int* __restrict__ hlev,
                                             const int* __restrict__ fslot, const double* __restrict__ fscale,
                                             const float* __restrict__ fscale_hi, const float* __restrict__ fscale_lo,
                                             R* __restrict__ sm)
{
    static_assert(TW == 32 || TW == 32 * MESS_TEAM_WARPS, "a warp or the whole block per quartet");
    static_assert(!PS || TW == 32 * MESS_TEAM_WARPS, "the primitive split spans the block");
    constexpr int TP = PS ? 32 : TW;                // threads of one primitive-loop group
    const int slot = threadIdx.x / TW, lane = threadIdx.x % TW;
    const long long q = (long long)blockIdx.x * (32 * MESS_TEAM_WARPS / TW) + slot;
    if (q >= b.total) return;                       // the quartet's threads leave together
    const int pslot = PS ? (int)(threadIdx.x >> 5) : slot, plane = threadIdx.x % TP;
    R* V = sm + (size_t)slot * (NVI + NH);
    R* H = V + NVI;
    R* Vp = sm + (size_t)pslot * (NVI + NH);        // the group's own values and contracted sums
    R* Hp = Vp + NVI;
    const int i = find_bra(b, q);
    const int j = __ldg(b.kbeg + i) + (int)(q - __ldg(b.offs + i));
    const int bp = __ldg(b.bra + i);
    const KetRec* kr = b.ketrec + j;
    const int4 kh = ket_hdr(kr);
    const int kp = ket_pair(kr);
    if (!P.live(bp) || !P.dens_ok(bp, kp)) return;   // the quartet's threads leave together
    const KetView<R> kv = ket_view(P, bp, kr, kh);
    for (int k = plane; k < NACC; k += TP) Hp[k] = R(0);
    team_sync<TP>();
    const int b0 = P.pp_off[bp], nbp = P.pp_n[bp];
    const int k0 = kv.k0, nkp = kv.nk;
    const R ACx = kv.AC[0], ACy = kv.AC[1], ACz = kv.AC[2];
#pragma unroll 1
    for (int ip = PS ? pslot : 0; ip < nbp * nkp; ip += PS ? MESS_TEAM_WARPS : 1) {
        const int ib = b0 + ip / nkp, ik = k0 + ip % nkp;
        const PrimPair<R> pb = P.load(ib);
        {
            const PrimPair<R> pk = P.load(ik);
            R rz, srz;
            recip_and_sqrt(pb.zeta + pk.zeta, rz, srz);
            const R roz = pk.zeta * rz, roe = pb.zeta * rz, oo2ze = R(0.5) * rz;
            const R PQx = pb.PAx - pk.PAx + ACx, PQy = pb.PAy - pk.PAy + ACy, PQz = pb.PAz - pk.PAz + ACz;
            const R WPx = -roz * PQx, WPy = -roz * PQy, WPz = -roz * PQz;
            const R WQx = roe * PQx, WQy = roe * PQy, WQz = roe * PQz;
            const R T = pb.zeta * roz * (PQx * PQx + PQy * PQy + PQz * PQz);
            const R pref = pb.K * pk.K * srz;
            R F[L + 1];
            boys_eval<R, L, BMODE>(T, F, P);
#pragma unroll
            for (int m = 0; m <= L; ++m) F[m] *= pref;
#pragma unroll 1
            for (int lv = 0; lv < NVL; ++lv) {
                const int oend = __ldg(vlev + lv + 1);
#pragma unroll 1
                for (int o = __ldg(vlev + lv) + plane; o < oend; o += TP) {
                    const uint4 w = __ldg(vprog + o);
                    const int kind = w.x & 3, d = (w.x >> 2) & 3;
                    const int m1 = (w.x >> 4) & 15, m2 = (w.x >> 8) & 15, t = w.x >> 16;
                    const int s1 = w.y & 0xffff, s2 = w.y >> 16;
                    if (kind == 0) {
                        R f = F[0];
#pragma unroll
                        for (int m = 1; m <= L; ++m) f = (s1 == m) ? F[m] : f;
                        Vp[t] = f;
                    } else if (kind == 3) {
                        Hp[s1] += Vp[t];
                    } else if (kind == 1) {
                        R v = pick3(d, pb.PAx, pb.PAy, pb.PAz) * Vp[s1] + pick3(d, WPx, WPy, WPz) * Vp[s2];
                        if (m1) v += small_int<R>(m1) * pb.oo2z * (Vp[w.z & 0xffff] - roz * Vp[w.z >> 16]);
                        Vp[t] = v;
                    } else {
                        R v = pick3(d, pk.PAx, pk.PAy, pk.PAz) * Vp[s1] + pick3(d, WQx, WQy, WQz) * Vp[s2];
                        if (m1) v += small_int<R>(m1) * pk.oo2z * (Vp[w.z & 0xffff] - roe * Vp[w.z >> 16]);
                        if (m2) v += small_int<R>(m2) * oo2ze * Vp[w.w];
                        Vp[t] = v;
                    }
                }
                team_sync<TP>();
            }
        }
    }
    if (PS) {
        __syncthreads();
        for (int k = threadIdx.x; k < NACC; k += TW) {
            R acc = H[k];
#pragma unroll
            for (int w = 1; w < MESS_TEAM_WARPS; ++w) acc += sm[(size_t)w * (NVI + NH) + NVI + k];
            H[k] = acc;
        }
        __syncthreads();
    }
    const R ABx = pair_ab(P, bp, 0), ABy = pair_ab(P, bp, 1), ABz = pair_ab(P, bp, 2);
    const R CDx = kv.CD[0], CDy = kv.CD[1], CDz = kv.CD[2];
#pragma unroll 1
    for (int lv = 0; lv < NHL; ++lv) {
        const int oend = __ldg(hlev + lv + 1);
#pragma unroll 1
        for (int o = __ldg(hlev + lv) + lane; o < oend; o += TW) {
            const uint2 w = __ldg(hprog + o);
            const int t = w.x & 0xffff, d = (w.x >> 16) & 3, side = (w.x >> 18) & 1;
            const R X = side ? pick3(d, CDx, CDy, CDz) : pick3(d, ABx, ABy, ABz);
            H[t] = H[w.y & 0xffff] + X * H[w.y >> 16];
        }
        team_sync<TW>();
    }
    for (int k = lane; k < NINT; k += TW) V[k] = gen_scale<R>(fscale, fscale_hi, fscale_lo, k) * H[__ldg(fslot + k)];
    team_sync<TW>();
    const R* I = V;
    R s = R(1);
    if (__ldg(P.same + bp)) s *= R(0.5);
    if (kh.w & 1) s *= R(0.5);
    if (bp == kp) s *= R(0.5);
    const int fa = __ldg(P.fa + bp), fb = __ldg(P.fb + bp), fc = kh.z & 0xffff, fd = kh.z >> 16;
    const int mol_ = __ldg(P.mol + bp);
    const long long off_ = __ldg(P.mbase + mol_);
    D += off_;
    J += off_;
    K += off_;
    const size_t nn = (size_t)__ldg(P.mn + mol_);
    (void)n;
#define MESS_I(a_, b_, c_, d_) I[(((a_) * NB + (b_)) * NC + (c_)) * ND + (d_)]
    for (int o = lane; o < NA * NB; o += TW) {          // J_ab = sum_cd I D_cd
        const int a = o / NB, bb = o % NB;
        R t = R(0);
        for (int c = 0; c < NC; ++c)
            for (int d = 0; d < ND; ++d) t += MESS_I(a, bb, c, d) * ldD(D + (fc + c) * nn + fd + d);
        atomicAdd(J + (fa + a) * nn + fb + bb, to_f64(s * t));
    }
    for (int o = lane; o < NC * ND; o += TW) {          // J_cd = sum_ab I D_ab
        const int c = o / ND, d = o % ND;
        R t = R(0);
        for (int a = 0; a < NA; ++a)
            for (int bb = 0; bb < NB; ++bb) t += MESS_I(a, bb, c, d) * ldD(D + (fa + a) * nn + fb + bb);
        atomicAdd(J + (fc + c) * nn + fd + d, to_f64(s * t));
    }
    for (int o = lane; o < NA * NC; o += TW) {          // K_ac = sum_bd I D_bd
        const int a = o / NC, c = o % NC;
        R t = R(0);
        for (int bb = 0; bb < NB; ++bb)
            for (int d = 0; d < ND; ++d) t += MESS_I(a, bb, c, d) * ldD(D + (fb + bb) * nn + fd + d);
        atomicAdd(K + (fa + a) * nn + fc + c, to_f64(s * t));
    }
    for (int o = lane; o < NA * ND; o += TW) {          // K_ad = sum_bc I D_bc
        const int a = o / ND, d = o % ND;
        R t = R(0);
        for (int bb = 0; bb < NB; ++bb)
            for (int c = 0; c < NC; ++c) t += MESS_I(a, bb, c, d) * ldD(D + (fb + bb) * nn + fc + c);
        atomicAdd(K + (fa + a) * nn + fd + d, to_f64(s * t));
    }
    for (int o = lane; o < NB * NC; o += TW) {          // K_bc = sum_ad I D_ad
        const int bb = o / NC, c = o % NC;
        R t = R(0);
        for (int a = 0; a < NA; ++a)
            for (int d = 0; d < ND; ++d) t += MESS_I(a, bb, c, d) * ldD(D + (fa + a) * nn + fd + d);
        atomicAdd(K + (fb + bb) * nn + fc + c, to_f64(s * t));
    }
    for (int o = lane; o < NB * ND; o += TW) {          // K_bd = sum_ac I D_ac
        const int bb = o / ND, d = o % ND;
        R t = R(0);
        for (int a = 0; a < NA; ++a)
            for (int c = 0; c < NC; ++c) t += MESS_I(a, bb, c, d) * ldD(D + (fa + a) * nn + fc + c);
        atomicAdd(K + (fb + bb) * nn + fd + d, to_f64(s * t));
    }
#undef MESS_I
}

#define MESS_DEFINE_TEAM_KERNEL_IMPL(TAG, ...)                                                      \
    template <typename R> constexpr size_t team_smem_##TAG()                                        \
    {                                                                                               \
        return team_smem_bytes<R, __VA_ARGS__>();                                                   \
    }                                                                                               \
    template <typename R, int BMODE, int TW, int PS>                                                \
    __global__ void __launch_bounds__(32 * MESS_TEAM_WARPS)                                         \
    k_jk_team_##TAG(const BinLaunch b, const PairTable<R> P, const typename DElem<R>::T* __restrict__ D,          \
                    double* __restrict__ J, double* __restrict__ K, int n)                          \
    {                                                                                               \
        extern __shared__ __align__(16) unsigned char mess_team_smem[];                             \
        jk_team_body<R, BMODE, TW, PS, __VA_ARGS__>(b, P, D, J, K, n, MESS_TEAM_PROG_##TAG,         \
                                            reinterpret_cast<R*>(mess_team_smem));                  \
    }
#define MESS_DEFINE_TEAM_KERNEL(TAG) MESS_DEFINE_TEAM_KERNEL_IMPL(TAG, MESS_TEAM_ARGS_##TAG)

template <typename R, int L, int NVI, int NH, int NACC, int NVL, int NHL, int NINT, int NA, int NB, int NC, int ND>
constexpr size_t team_smem_bytes()
{
    return (size_t)MESS_TEAM_WARPS * (NVI + NH) * sizeof(R);
}
