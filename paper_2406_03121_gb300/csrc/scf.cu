// Self-consistent-field solution of the Roothaan equation F(C) C = S C eps (paper Eq. 2, Sec. 3),
// closed shell, on the device, for one molecule or a batch of molecules (the paper's vmap over
// conformers, Sec. 5.2).  Every molecule m owns the n_m x n_m block [base_m, base_m + n_m^2) of each
// packed array.  One iteration:
//   J, K from D (integral-direct, the J/K kernels);  F = H + J - K/2;  E = 1/2 sum D (H + F);
//   e = F D S - S D F;  Pulay DIIS on e;  F' = X^T F X (X = S^-1/2, Loewdin);
//   F' = V eps V^T (cyclic Jacobi, one thread block per molecule);  C = X V;  D = 2 C_occ C_occ^T.
// A molecule is converged when |dE| < conv_E and max|e| < conv_comm; converged molecules leave the
// J/K builds and every other kernel of the loop.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "mess_internal.h"

namespace {

struct Layout {
    const long long* base;   // [nmol]
    const int* n;            // [nmol]
    const int* nocc;         // [nmol] orbitals with a non-zero occupation
    const unsigned char* active;   // [nmol]
    const double* occ;       // occupation of orbital k of molecule m at occ[obase[m] + k] (energy order)
    const long long* obase;  // [nmol]
};

__device__ __forceinline__ double block_sum(double v, double* red)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = (blockDim.x + 31) >> 5;
    __syncthreads();
    if (l == 0) red[w] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x < 32) {
        t = (l < nw) ? red[l] : 0.0;
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    }
    if (threadIdx.x == 0) red[0] = t;
    __syncthreads();
    const double r = red[0];
    __syncthreads();
    return r;
}

__device__ __forceinline__ double block_max(double v, double* red)
{
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = (blockDim.x + 31) >> 5;
    __syncthreads();
    if (l == 0) red[w] = v;
    __syncthreads();
    double t = -INFINITY;
    if (threadIdx.x < 32) {
        t = (l < nw) ? red[l] : -INFINITY;
        for (int o = 16; o > 0; o >>= 1) t = fmax(t, __shfl_xor_sync(0xffffffffu, t, o));
    }
    if (threadIdx.x == 0) red[0] = t;
    __syncthreads();
    const double r = red[0];
    __syncthreads();
    return r;
}

// out = a*X + b*Y + c*Z elementwise on each active molecule block (grid.y = molecule)
__global__ void k_axpbypcz(double* out, double a, const double* X, double bb, const double* Y, double c,
                           const double* Z, Layout L)   // out may alias X (elementwise)
{
    const int m = blockIdx.y;
    if (!L.active[m]) return;
    const long long nn = (long long)L.n[m] * L.n[m], o = L.base[m];
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nn; i += (long long)gridDim.x * blockDim.x) {
        double v = a * X[o + i];
        if (Y) v += bb * Y[o + i];
        if (Z) v += c * Z[o + i];
        out[o + i] = v;
    }
}

// E_m = 1/2 sum D (H + F)
__global__ void k_energy(const double* __restrict__ D, const double* __restrict__ H, const double* __restrict__ F,
                         Layout L, double* __restrict__ E)
{
    __shared__ double red[32];
    const int m = blockIdx.x;
    if (!L.active[m]) return;
    const long long nn = (long long)L.n[m] * L.n[m], o = L.base[m];
    double s = 0.0;
    for (long long i = threadIdx.x; i < nn; i += blockDim.x) s += D[o + i] * (H[o + i] + F[o + i]);
    s = block_sum(s, red);
    if (threadIdx.x == 0) E[m] = 0.5 * s;
}

// Kohn-Sham: E_m = sum D (H + J/2) + E_xc,m
__global__ void k_energy_ks(const double* __restrict__ D, const double* __restrict__ H, const double* __restrict__ J,
                            const double* __restrict__ Exc, Layout L, double* __restrict__ E)
{
    __shared__ double red[32];
    const int m = blockIdx.x;
    if (!L.active[m]) return;
    const long long nn = (long long)L.n[m] * L.n[m], o = L.base[m];
    double s = 0.0;
    for (long long i = threadIdx.x; i < nn; i += blockDim.x) s += D[o + i] * (H[o + i] + 0.5 * J[o + i]);
    s = block_sum(s, red);
    if (threadIdx.x == 0) E[m] = s + Exc[m];
}

// C = alpha * A op(B) + beta * C per molecule; A is n x k (row stride n), op(B) k x n; k = n (kmode 0)
// or the occupied orbitals (kmode 1, column kk of A weighted by its occupation: C diag(occ) C^T).
// 16 x 16 output tiles staged through shared memory.
template <bool TRANSA, bool TRANSB>
__global__ void k_gemm(const double* __restrict__ A, const double* __restrict__ B, double* __restrict__ C,
                       Layout L, int kmode, double alpha, double beta)
{
    __shared__ double As[16][17], Bs[16][17];
    const int m = blockIdx.z;
    if (!L.active[m]) return;
    const int n = L.n[m];
    const int k = kmode ? L.nocc[m] : n;
    const int r0 = blockIdx.y * 16, c0 = blockIdx.x * 16;
    if (r0 >= n || c0 >= n) return;
    const long long o = L.base[m];
    const int ty = threadIdx.y, tx = threadIdx.x;
    double acc = 0.0;
    for (int k0 = 0; k0 < k; k0 += 16) {
        if (TRANSA) {
            const int ar = k0 + ty, ac = r0 + tx;      // A^T[i][kk] = A[kk][i]
            As[tx][ty] = (ar < k && ac < n) ? A[o + (long long)ar * n + ac] : 0.0;
        } else {
            const int ar = r0 + ty, ac = k0 + tx;
            double w = 1.0;
            if (kmode && ac < k) w = L.occ[L.obase[m] + ac];
            As[ty][tx] = (ar < n && ac < k) ? w * A[o + (long long)ar * n + ac] : 0.0;
        }
        if (TRANSB) {
            const int br = c0 + ty, bc = k0 + tx;      // B[j][kk]
            Bs[tx][ty] = (br < n && bc < k) ? B[o + (long long)br * n + bc] : 0.0;
        } else {
            const int br = k0 + ty, bc = c0 + tx;      // B[kk][j]
            Bs[ty][tx] = (br < k && bc < n) ? B[o + (long long)br * n + bc] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) acc += As[ty][kk] * Bs[kk][tx];
        __syncthreads();
    }
    const int r = r0 + ty, cc = c0 + tx;
    if (r < n && cc < n) {
        const long long idx = o + (long long)r * n + cc;
        C[idx] = alpha * acc + (beta != 0.0 ? beta * C[idx] : 0.0);
    }
}

// e = W - W^T (W = F D S, so W^T = S D F) and max |e| per molecule
__global__ void k_commutator(const double* __restrict__ W, double* __restrict__ e, Layout L, double* __restrict__ emax)
{
    __shared__ double red[32];
    const int m = blockIdx.x;
    if (!L.active[m]) return;
    const int n = L.n[m];
    const long long o = L.base[m];
    double mx = 0.0;
    for (long long t = threadIdx.x; t < (long long)n * n; t += blockDim.x) {
        const int i = (int)(t / n), j = (int)(t % n);
        const double v = W[o + (long long)i * n + j] - W[o + (long long)j * n + i];
        e[o + t] = v;
        mx = fmax(mx, fabs(v));
    }
    mx = block_max(mx, red);
    if (threadIdx.x == 0) emax[m] = mx;
}

// Pulay DIIS: store (F, e) in history slot `slot`, update the error inner products and replace F by
// the extrapolation sum_i c_i F_i with sum_i c_i = 1 minimising |sum_i c_i e_i|.
// The slot of this iteration's (F, e) and the number of stored pairs follow from the iteration
// number it (device state[0], 1-based): slot (it - 1) mod nmax, min(it, nmax) stored.
__global__ void k_diis(double* __restrict__ Fh, double* __restrict__ eh, long long hstride, double* __restrict__ F,
                       const double* __restrict__ e, Layout L, const int* __restrict__ state, int nmax,
                       double* __restrict__ Bm)
{
    __shared__ double red[32];
    __shared__ double coef[16];
    __shared__ int ok;
    const int m = blockIdx.x;
    if (!L.active[m]) return;
    const int it = state[0];
    const int slot = (it - 1) % nmax, nstored = min(it, nmax);
    const long long nn = (long long)L.n[m] * L.n[m], o = L.base[m];
    for (long long t = threadIdx.x; t < nn; t += blockDim.x) {
        Fh[slot * hstride + o + t] = F[o + t];
        eh[slot * hstride + o + t] = e[o + t];
    }
    __syncthreads();
    double* B = Bm + (size_t)m * nmax * nmax;
    for (int i = 0; i < nstored; ++i) {
        double s = 0.0;
        for (long long t = threadIdx.x; t < nn; t += blockDim.x) s += eh[i * hstride + o + t] * eh[slot * hstride + o + t];
        s = block_sum(s, red);
        if (threadIdx.x == 0) { B[i * nmax + slot] = s; B[slot * nmax + i] = s; }
    }
    __syncthreads();
    if (nstored < 2) return;
    if (threadIdx.x == 0) {
        // augmented system [B 1; 1 0][c; lambda] = [0; 1], Gaussian elimination with partial pivoting
        const int k = nstored + 1;
        double M[17][18];
        double scale = 0.0;
        for (int i = 0; i < nstored; ++i) scale = fmax(scale, fabs(B[i * nmax + i]));
        if (!(scale > 0.0)) scale = 1.0;
        for (int i = 0; i < k; ++i)
            for (int j = 0; j <= k; ++j) M[i][j] = 0.0;
        for (int i = 0; i < nstored; ++i) {
            for (int j = 0; j < nstored; ++j) M[i][j] = B[i * nmax + j] / scale;
            M[i][nstored] = 1.0;
            M[nstored][i] = 1.0;
        }
        M[nstored][k] = 1.0;
        ok = 1;
        for (int c = 0; c < k; ++c) {
            int piv = c;
            for (int r = c + 1; r < k; ++r) if (fabs(M[r][c]) > fabs(M[piv][c])) piv = r;
            if (fabs(M[piv][c]) < 1e-300) { ok = 0; break; }
            if (piv != c)
                for (int j = 0; j <= k; ++j) { const double t = M[c][j]; M[c][j] = M[piv][j]; M[piv][j] = t; }
            for (int r = 0; r < k; ++r) {
                if (r == c) continue;
                const double f = M[r][c] / M[c][c];
                for (int j = c; j <= k; ++j) M[r][j] -= f * M[c][j];
            }
        }
        for (int i = 0; i < nstored && ok; ++i) coef[i] = M[i][k] / M[i][i];
    }
    __syncthreads();
    if (!ok) return;   // singular subspace: keep the plain Fock matrix
    for (long long t = threadIdx.x; t < nn; t += blockDim.x) {
        double v = 0.0;
        for (int i = 0; i < nstored; ++i) v += coef[i] * Fh[i * hstride + o + t];
        F[o + t] = v;
    }
}

// Device state of the SCF loop: state[0] iteration number (1-based once an iteration starts),
// state[1] molecules still iterating, state[2] 1 + the first molecule with a non-finite energy
// (0: none).  One thread advances the iteration counter.
__global__ void k_iter_begin(int* state) { state[0] += 1; }

// Input of this iteration's J/K build: the change of the density since the previous build (J and K
// are linear in D, so J(D_k) = J(D_{k-1}) + J(D_k - D_{k-1})), or the whole density every
// full_every iterations, when the accumulated J, K restart from zero.  Dprev <- D.
__global__ void k_delta(const double* __restrict__ D, double* __restrict__ Dprev, double* __restrict__ W,
                        double* __restrict__ Jt, double* __restrict__ Kt, Layout L, const int* __restrict__ state,
                        int full_every)
{
    const int m = blockIdx.y;
    if (!L.active[m]) return;
    const bool full = (state[0] - 1) % full_every == 0;
    const long long nn = (long long)L.n[m] * L.n[m], o = L.base[m];
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nn; i += (long long)gridDim.x * blockDim.x) {
        const double d = D[o + i];
        W[o + i] = full ? d : d - Dprev[o + i];
        Dprev[o + i] = d;
        if (full) { Jt[o + i] = 0.0; Kt[o + i] = 0.0; }
    }
}

// Largest |W_mn| of every row m of each active molecule's block, at the row's global function index
// (rowmax[fbase[mol] + m]); inactive molecules' rows are 0.
__global__ void k_rowmax(const double* __restrict__ W, Layout L, const int* __restrict__ fbase,
                         float* __restrict__ rowmax)
{
    const int m = blockIdx.y;
    const int n = L.n[m];
    const long long o = L.base[m];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double mx = 0.0;
        if (L.active[m])
            for (int j = 0; j < n; ++j) mx = fmax(mx, fabs(W[o + (long long)i * n + j]));
        rowmax[fbase[m] + i] = nextafterf((float)mx, INFINITY);   // rounded up: still a bound
    }
}

// dmax of every shell pair: the largest row maximum over the functions of its two shells
__global__ void k_pairmax(const float* __restrict__ rowmax, const int* __restrict__ pair_a,
                          const int* __restrict__ pair_b, const int* __restrict__ shell_f0,
                          const int* __restrict__ shell_l, float* __restrict__ dmax, int npair)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= npair) return;
    float mx = 0.f;
    for (int s = 0; s < 2; ++s) {
        const int sh = s ? pair_b[p] : pair_a[p];
        const int f0 = shell_f0[sh], l = shell_l[sh];
        for (int k = 0; k < (l + 1) * (l + 2) / 2; ++k) mx = fmaxf(mx, rowmax[f0 + k]);
    }
    dmax[p] = mx;
}

// Convergence test of every molecule still iterating (|dE| < conv_E and max|FDS - SDF| < conv_comm
// from the second iteration on): a converged molecule records its iteration count and energy and
// leaves (active = 0); a non-finite energy or error stops the molecule and is reported.
__global__ void k_converge(const double* __restrict__ E, const double* __restrict__ emax, double* __restrict__ Eold,
                           int* __restrict__ iters, int* __restrict__ conv, double* __restrict__ Efin,
                           unsigned char* __restrict__ active, int* __restrict__ state, int nmol, double conv_E,
                           double conv_comm)
{
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= nmol || !active[m]) return;
    const int it = state[0];
    const double e = E[m], x = emax[m];
    iters[m] = it;
    if (!isfinite(e) || !isfinite(x)) {
        atomicCAS(state + 2, 0, m + 1);
        active[m] = 0;
        atomicSub(state + 1, 1);
        return;
    }
    if (it > 1 && fabs(e - Eold[m]) < conv_E && x < conv_comm) {
        conv[m] = 1;
        Efin[m] = e;
        active[m] = 0;
        atomicSub(state + 1, 1);
    }
    Eold[m] = e;
}

// Element arithmetic of the Jacobi eigensolver: FP64, or double-float (hi + lo FP32 pairs, about
// 48 significant bits) for the reduced-precision SCF, where the eigensolver then runs on the FP32
// units instead of the FP64 pipe (1/64 of their rate on this GPU).
__device__ __forceinline__ void jac_set(double& x, double v) { x = v; }
__device__ __forceinline__ void jac_set(df32& x, double v) { x = df32(v); }
__device__ __forceinline__ double jac_get(double x) { return x; }
__device__ __forceinline__ double jac_get(df32 x) { return f2d_alu(x.hi) + f2d_alu(x.lo); }
__device__ __forceinline__ double jac_lead(double x) { return x; }            // for tests and sums
__device__ __forceinline__ double jac_lead(df32 x) { return f2d_alu(x.hi); }
__device__ __forceinline__ bool jac_iszero(double x) { return x == 0.0; }
__device__ __forceinline__ bool jac_iszero(df32 x) { return x.hi == 0.f; }
__device__ __forceinline__ double jac_sqrt(double x) { return sqrt(x); }
__device__ __forceinline__ df32 jac_sqrt(df32 x) { return df_sqrt(x); }
__device__ __forceinline__ double jac_abs(double x) { return fabs(x); }
__device__ __forceinline__ df32 jac_abs(df32 x) { return x.hi < 0.f ? -x : x; }
template <typename T> __device__ __forceinline__ T jac_one();
template <> __device__ __forceinline__ double jac_one<double>() { return 1.0; }
template <> __device__ __forceinline__ df32 jac_one<df32>() { return df32(1.0f, 0.f); }
template <typename T> __device__ __forceinline__ T jac_zero();
template <> __device__ __forceinline__ double jac_zero<double>() { return 0.0; }
template <> __device__ __forceinline__ df32 jac_zero<df32>() { return df32(0.f, 0.f); }
// a rotation is skipped when |a_pq| <= JacEps::skip sqrt(|a_pp a_qq|); the sweeps stop when the
// off-diagonal Frobenius norm squared is below JacEps::off of the whole (relative round-off level)
template <typename T> struct JacEps;
template <> struct JacEps<double> { static constexpr double skip = 1e-15, off = 1e-28; };
template <> struct JacEps<df32> { static constexpr double skip = 1e-13, off = 1e-25; };

// Cyclic Jacobi eigensolver of the symmetric n x n block of each molecule, one thread block per
// molecule, rotations in parallel over disjoint index pairs (round-robin "circle" schedule).  The
// rotation of (p, q) uses tau = (a_qq - a_pp)/(2 a_pq), t = sign(tau)/(|tau| + sqrt(1 + tau^2)),
// c = 1/sqrt(1 + t^2), s = t c, and A <- J^T A J, V <- V J.  Eigenvalues ascending in eps, the
// matching eigenvectors as the columns of Vout.  The matrix (element type T, 8 bytes) lives in
// shared memory when it fits, otherwise in the global workspace Wk.  The eigenvectors accumulate
// transposed in the global workspace Vt (row k = eigenvector k), so that the update of V's columns
// p, q runs along contiguous rows.  Each warp takes whole rows (lanes along the row): no index
// division anywhere in the sweeps.
template <typename T>
__global__ void __launch_bounds__(512) k_jacobi(const double* __restrict__ Ain, T* __restrict__ Vt_ws,
                                                double* __restrict__ Vout, double* __restrict__ eps,
                                                const long long* __restrict__ ebase, Layout L, int use_smem,
                                                T* __restrict__ Wk, int max_sweeps, int* __restrict__ sweeps_out)
{
    extern __shared__ __align__(16) unsigned char jsm_raw[];
    __shared__ double red[32];
    __shared__ int pp_[128], qq_[128];
    __shared__ T cc_[128], ss_[128];
    __shared__ int rotated;
    const int m = blockIdx.x;
    if (!L.active[m]) return;
    const int n = L.n[m];
    const long long o = L.base[m];
    T* A = use_smem ? reinterpret_cast<T*>(jsm_raw) : Wk + o;
    T* Vt = Vt_ws + o;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarp = blockDim.x >> 5;
    const int npad = n + (n & 1), half = npad / 2, rounds = npad - 1;
    const T one = jac_one<T>(), zero = jac_zero<T>();
    double nrm = 0.0;
    for (int i = warp; i < n; i += nwarp)
        for (int j = lane; j < n; j += 32) {
            jac_set(A[i * n + j], Ain[o + (long long)i * n + j]);
            Vt[i * n + j] = (i == j) ? one : zero;
            const double a = jac_lead(A[i * n + j]);
            nrm += a * a;
        }
    nrm = block_sum(nrm, red);   // (synchronises the block)
    int sweep = 0;
    for (; sweep < max_sweeps; ++sweep) {
        double off = 0.0;
        for (int i = warp; i < n; i += nwarp)
            for (int j = lane; j < n; j += 32) {
                const double a = jac_lead(A[i * n + j]);
                if (i != j) off += a * a;
            }
        off = block_sum(off, red);
        if (off <= JacEps<T>::off * nrm || off == 0.0) break;
        if (threadIdx.x == 0) rotated = 0;
        __syncthreads();
        for (int r = 0; r < rounds; ++r) {
            for (int k = threadIdx.x; k < half; k += blockDim.x) {
                int a, b2;
                if (k == 0) { a = rounds; b2 = r; }
                else { a = (r + k) % rounds; b2 = (r - k + rounds) % rounds; }
                const int p = min(a, b2), q = max(a, b2);
                T c = one, s = zero;
                if (q < n) {
                    const T apq = A[p * n + q];
                    const T app = A[p * n + p], aqq = A[q * n + q];
                    const double lpq = fabs(jac_lead(apq));
                    // rotate unless a_pq is negligible against the diagonal (round-off level)
                    if (lpq > 1e-300 && lpq > JacEps<T>::skip * sqrt(fabs(jac_lead(app)) * fabs(jac_lead(aqq)))) {
                        const T tau = (aqq - app) / (apq + apq);
                        T t;
                        if (fabs(jac_lead(tau)) > 1e15) {
                            t = one / (tau + tau);   // t -> 1/(2 tau); tau^2 would overflow FP32
                        } else {
                            const T den = jac_abs(tau) + jac_sqrt(one + tau * tau);
                            t = (jac_lead(tau) >= 0.0 ? one : -one) / den;
                        }
                        c = one / jac_sqrt(one + t * t);
                        s = t * c;
                        rotated = 1;
                    }
                }
                pp_[k] = p; qq_[k] = q; cc_[k] = c; ss_[k] = s;
            }
            __syncthreads();
            // rows p, q:  row_p <- c row_p - s row_q,  row_q <- s row_p + c row_q  (a warp per pair)
            for (int k = warp; k < half; k += nwarp) {
                const int p = pp_[k], q = qq_[k];
                if (q >= n || jac_iszero(ss_[k])) continue;
                const T c = cc_[k], s = ss_[k];
                for (int j = lane; j < n; j += 32) {
                    const T x = A[p * n + j], y = A[q * n + j];
                    A[p * n + j] = c * x - s * y;
                    A[q * n + j] = s * x + c * y;
                }
            }
            __syncthreads();
            // columns p, q of A; rows p, q of V^T
            for (int k = warp; k < half; k += nwarp) {
                const int p = pp_[k], q = qq_[k];
                if (q >= n || jac_iszero(ss_[k])) continue;
                const T c = cc_[k], s = ss_[k];
                for (int i = lane; i < n; i += 32) {
                    const T x = A[i * n + p], y = A[i * n + q];
                    A[i * n + p] = c * x - s * y;
                    A[i * n + q] = s * x + c * y;
                    const T vx = Vt[p * n + i], vy = Vt[q * n + i];
                    Vt[p * n + i] = c * vx - s * vy;
                    Vt[q * n + i] = s * vx + c * vy;
                }
            }
            __syncthreads();
        }
        if (!rotated) break;
        __syncthreads();
    }
    // eigenvalues ascending (rank by counting), eigenvectors (rows of V^T) into the columns of Vout
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const double ai = jac_get(A[i * n + i]);
        int rank = 0;
        for (int j = 0; j < n; ++j) {
            const double aj = jac_get(A[j * n + j]);
            rank += (aj < ai) || (aj == ai && j < i);
        }
        eps[ebase[m] + rank] = ai;
        for (int r = 0; r < n; ++r) Vout[o + (long long)r * n + rank] = jac_get(Vt[i * n + r]);
    }
    if (threadIdx.x == 0 && sweeps_out) sweeps_out[m] = sweep;
}

// W = U diag(s^-1/2) (columns of the eigenvectors of S scaled); smin per molecule
__global__ void k_scale_cols(const double* __restrict__ U, const double* __restrict__ s,
                             const long long* __restrict__ ebase, double* __restrict__ W, Layout L,
                             double* __restrict__ smin)
{
    __shared__ double red[32];
    const int m = blockIdx.x;
    if (!L.active[m]) return;
    const int n = L.n[m];
    const long long o = L.base[m];
    for (long long t = threadIdx.x; t < (long long)n * n; t += blockDim.x) {
        const int j = (int)(t % n);
        const double ev = s[ebase[m] + j];
        W[o + t] = ev > 0.0 ? U[o + t] / sqrt(ev) : 0.0;
    }
    double mn = 1e300;
    for (int j = threadIdx.x; j < n; j += blockDim.x) mn = fmin(mn, s[ebase[m] + j]);
    mn = -block_max(-mn, red);
    if (threadIdx.x == 0) smin[m] = mn;
}

template <typename T> struct Dev {
    T* p = nullptr;
    cudaError_t alloc(size_t n) { return cudaMalloc((void**)&p, std::max<size_t>(n, 1) * sizeof(T)); }
    ~Dev() { if (p) cudaFree(p); }
};

struct StreamGuard {
    cudaStream_t s = nullptr;
    ~StreamGuard()
    {
        if (s) { cudaStreamSynchronize(s); cudaStreamDestroy(s); }
    }
};

struct SCFState {
    mess_basis* b;
    cudaStream_t s;
    int nmol, maxn;
    long long P;
    Dev<double> S, H, X, F, D, J, K, V, C, W1, W2, e, eps, E, emax, smin, Bm, Fh, eh, Wk;
    Dev<double> Vprev, Dprev, Jt, Kt;   // warm-start eigenvectors, previous density, accumulated J / K
    Dev<double> Eold, Efin;             // per molecule: previous energy, energy at convergence
    Dev<int> state, iters, conv;        // loop state (see k_iter_begin), per molecule iterations / converged
    bool warm = false;
    Dev<long long> base, ebase;
    Dev<double> occ;
    Dev<int> n, nocc, sweeps;
    Dev<unsigned char> active;
    int use_smem;
    size_t jac_smem;
    // eigensolver arithmetic: FP64 (the FP64 path) or double-float (reduced precision), for the
    // Fock matrices and the overlap matrix of the orthogonaliser alike
    bool fock_fp64 = true;
    Layout L;
    StreamGuard sg;   // the private stream: last member, so it is drained before the buffers are freed
};

cudaError_t gemm(SCFState& st, bool transB, const double* A, const double* B, double* C, int kmode, double alpha,
                 bool transA = false)
{
    dim3 blk(16, 16), grid((st.maxn + 15) / 16, (st.maxn + 15) / 16, st.nmol);
    if (transA) k_gemm<true, false><<<grid, blk, 0, st.s>>>(A, B, C, st.L, kmode, alpha, 0.0);
    else if (transB) k_gemm<false, true><<<grid, blk, 0, st.s>>>(A, B, C, st.L, kmode, alpha, 0.0);
    else k_gemm<false, false><<<grid, blk, 0, st.s>>>(A, B, C, st.L, kmode, alpha, 0.0);
    return cudaGetLastError();
}

// The dynamic shared memory the Jacobi kernel may use: the attribute is per kernel, not per call,
// so it is set again after anything that may have changed it (a nested SCF of atomic densities).
cudaError_t jacobi_prepare(SCFState& st)
{
    if (!st.use_smem) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(k_jacobi<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)st.jac_smem);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_jacobi<df32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)st.jac_smem);
}

// Eigen-decomposition of the packed symmetric blocks A (eigenvectors to Vout, eigenvalues to eps).
// fp64: FP64 arithmetic; otherwise double-float (the reduced-precision SCF's Fock matrices).  The
// workspaces W2 and Wk hold 8-byte elements of either type.
cudaError_t jacobi(SCFState& st, const double* A, double* Vout, bool fp64 = true)
{
    if (fp64)
        k_jacobi<double><<<st.nmol, 512, st.jac_smem, st.s>>>(A, st.W2.p, Vout, st.eps.p, st.ebase.p, st.L,
                                                              st.use_smem, st.Wk.p, 40, st.sweeps.p);
    else
        k_jacobi<df32><<<st.nmol, 512, st.jac_smem, st.s>>>(A, reinterpret_cast<df32*>(st.W2.p), Vout, st.eps.p,
                                                            st.ebase.p, st.L, st.use_smem,
                                                            reinterpret_cast<df32*>(st.Wk.p), 40, st.sweeps.p);
    return cudaGetLastError();
}

// D = 2 C_occ C_occ^T from a Fock matrix (F' = X F X -> eigenvectors V -> C = X V).  After the
// first call the eigensolver starts from the previous eigenvectors: it diagonalises
// Vprev^T F' Vprev, which is nearly diagonal once the SCF settles, and V = Vprev V_rel.
cudaError_t density_from_fock(SCFState& st, const double* Fin)
{
    cudaError_t e;
    if ((e = gemm(st, false, st.X.p, Fin, st.W1.p, 0, 1.0)) != cudaSuccess) return e;   // X F
    if ((e = gemm(st, false, st.W1.p, st.X.p, st.V.p, 0, 1.0)) != cudaSuccess) return e; // F' = X F X
    if (st.warm) {
        if ((e = gemm(st, false, st.V.p, st.Vprev.p, st.W1.p, 0, 1.0)) != cudaSuccess) return e;          // F' Vprev
        if ((e = gemm(st, false, st.Vprev.p, st.W1.p, st.V.p, 0, 1.0, true)) != cudaSuccess) return e;    // Vprev^T F' Vprev
        if ((e = jacobi(st, st.V.p, st.W1.p, st.fock_fp64)) != cudaSuccess) return e;                     // V_rel -> W1
        if ((e = gemm(st, false, st.Vprev.p, st.W1.p, st.V.p, 0, 1.0)) != cudaSuccess) return e;          // V = Vprev V_rel
    } else {
        if ((e = jacobi(st, st.V.p, st.W1.p, st.fock_fp64)) != cudaSuccess) return e;       // V -> W1
        if ((e = cudaMemcpyAsync(st.V.p, st.W1.p, sizeof(double) * st.P, cudaMemcpyDeviceToDevice, st.s)) != cudaSuccess) return e;
        st.warm = true;
    }
    if ((e = cudaMemcpyAsync(st.Vprev.p, st.V.p, sizeof(double) * st.P, cudaMemcpyDeviceToDevice, st.s)) != cudaSuccess) return e;
    if ((e = gemm(st, false, st.X.p, st.V.p, st.C.p, 0, 1.0)) != cudaSuccess) return e;  // C = X V
    return gemm(st, true, st.C.p, st.C.p, st.D.p, 1, 1.0);                             // D = C diag(occ) C^T
}

// Block-diagonal superposition of atomic densities: atom a of molecule m (functions [f, f + na) of
// the molecule) receives the density block of its element (molecule e of the atomic batch).
__global__ void k_assemble_blocks(double* __restrict__ D, const long long* __restrict__ mbase, const int* __restrict__ mn,
                                  const int* __restrict__ amol, const int* __restrict__ af, const int* __restrict__ an,
                                  const int* __restrict__ ael, const double* __restrict__ Dat,
                                  const long long* __restrict__ ebase, int natom)
{
    const int a = blockIdx.x;
    if (a >= natom) return;
    const int m = amol[a], f = af[a], na = an[a];
    const long long o = mbase[m], eo = ebase[ael[a]];
    const int n = mn[m];
    for (int t = threadIdx.x; t < na * na; t += blockDim.x) {
        const int i = t / na, j = t % na;
        D[o + (long long)(f + i) * n + f + j] = Dat[eo + (long long)i * na + j];
    }
}

// occupations of the orbitals (energy order) of one neutral atom, spherically averaged: 1s, 2s
// doubly occupied, the 2p electrons spread evenly over the three 2p orbitals (reading C10)
static std::vector<double> atomic_occupation(int Z)
{
    std::vector<double> o;
    if (Z <= 2) { o.push_back((double)Z); return o; }
    o.push_back(2.0);
    if (Z <= 4) { o.push_back((double)(Z - 2)); return o; }
    o.push_back(2.0);
    for (int k = 0; k < 3; ++k) o.push_back((Z - 4) / 3.0);
    return o;
}

mess_status scf_run(mess_basis* b, const mess_scf_opts* opts, mess_scf_result* res, double* D_out, bool D_out_device,
                    const std::vector<std::vector<double>>* occ_in = nullptr);

// Superposition of atomic densities: an SCF of every distinct element as an isolated atom with
// spherically averaged fractional occupation, then the block-diagonal D0 of each molecule.
static mess_status sad_density(mess_basis* b, const mess_scf_opts& o, double* D0, cudaStream_t s)
{
    std::vector<int> elements;
    mess_basis* atoms = nullptr;
    mess_status st = mess_atoms_basis(b, elements, &atoms);
    if (st != MESS_OK) return st;
    std::vector<std::vector<double>> occ;
    for (int z : elements) occ.push_back(atomic_occupation(z));
    mess_scf_opts ao = o;
    ao.guess = MESS_GUESS_CORE;
    ao.prec = MESS_FP64;
    ao.max_iter = 200;
    std::vector<mess_scf_result> ares(elements.size());
    DevBuf<double> Dat;
    cudaError_t e = Dat.alloc((size_t)atoms->packed);
    if (e != cudaSuccess) { mess_free_basis(atoms); delete atoms; mess_set_error("SAD: allocation failed"); return MESS_ENOMEM; }
    st = scf_run(atoms, &ao, ares.data(), Dat.p, true, &occ);
    if (st != MESS_OK && st != MESS_ENOCONV) { Dat.free(); mess_free_basis(atoms); delete atoms; return st; }
    // per atom of b: molecule, first local function, function count, element index in `elements`
    std::vector<int> amol(b->natom), af(b->natom, -1), an(b->natom, 0), ael(b->natom);
    for (const HostShell& sh : b->shells) {
        if (af[sh.atom] < 0) af[sh.atom] = sh.fl;
        an[sh.atom] += (sh.l + 1) * (sh.l + 2) / 2;
        amol[sh.atom] = sh.mol;
    }
    for (int a = 0; a < b->natom; ++a)
        ael[a] = (int)(std::find(elements.begin(), elements.end(), b->Z[a]) - elements.begin());
    DevBuf<int> d_amol, d_af, d_an, d_ael;
    if (d_amol.upload(amol) != cudaSuccess || d_af.upload(af) != cudaSuccess || d_an.upload(an) != cudaSuccess ||
        d_ael.upload(ael) != cudaSuccess) {
        Dat.free(); mess_free_basis(atoms); delete atoms;
        mess_set_error("SAD: upload failed");
        return MESS_ECUDA;
    }
    e = cudaMemsetAsync(D0, 0, sizeof(double) * b->packed, s);
    if (e == cudaSuccess) {
        k_assemble_blocks<<<b->natom, 128, 0, s>>>(D0, b->d_mol_base.p, b->d_mol_n.p, d_amol.p, d_af.p, d_an.p,
                                                   d_ael.p, Dat.p, atoms->d_mol_base.p, b->natom);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    Dat.free(); d_amol.free(); d_af.free(); d_an.free(); d_ael.free();
    mess_free_basis(atoms);
    delete atoms;
    if (e != cudaSuccess) { mess_set_error("SAD assembly: %s", cudaGetErrorString(e)); return MESS_ECUDA; }
    return MESS_OK;
}

// Set-up shared by the SCF and the direct minimisation: the private stream (ordered after the
// caller's), per-molecule layout and occupations (closed shell: N_e / 2 doubly occupied orbitals, or
// the given fractional occupations), every packed work matrix, the one-electron matrices S and
// H = T + V, and the Loewdin orthogonaliser X = S^-1/2 (MESS_ENUMERIC if S is nearly singular).
static mess_status scf_setup(SCFState& st, mess_basis* b, cudaStream_t caller, int diis_n,
                             const std::vector<std::vector<double>>* occ_in, bool fp64_eig)
{
    st.b = b;
    st.fock_fp64 = fp64_eig;
    // The SCF runs on a private non-blocking stream (a CUDA graph cannot be captured on the legacy
    // default stream), ordered after the caller's stream; the call synchronises it before returning.
    {
        cudaEvent_t ready = nullptr;
        MESS_CUDA_TRY(cudaStreamCreateWithFlags(&st.sg.s, cudaStreamNonBlocking));
        MESS_CUDA_TRY(cudaEventCreateWithFlags(&ready, cudaEventDisableTiming));
        cudaError_t e = cudaEventRecord(ready, caller);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(st.sg.s, ready, 0);
        cudaEventDestroy(ready);
        MESS_CUDA_TRY(e);
    }
    st.s = st.sg.s;
    st.nmol = b->nmol;
    st.maxn = b->max_nbf;
    st.P = b->packed;
    std::vector<int> nocc(b->nmol);
    std::vector<long long> ebase(b->nmol);
    long long etot = 0;
    for (int m = 0; m < b->nmol; ++m) {
        if (!occ_in && b->mol_nelec[m] % 2) {
            mess_set_error("molecule %d: odd electron count %d", m, b->mol_nelec[m]);
            return MESS_EINVAL;
        }
        ebase[m] = etot;
        etot += b->mol_nbf[m];
    }
    std::vector<double> occ_h((size_t)etot, 0.0);
    for (int m = 0; m < b->nmol; ++m) {
        if (occ_in) {
            const std::vector<double>& w = (*occ_in)[m];
            if ((int)w.size() > b->mol_nbf[m]) { mess_set_error("molecule %d: too many occupied orbitals", m); return MESS_EINVAL; }
            for (size_t k = 0; k < w.size(); ++k) occ_h[ebase[m] + k] = w[k];
            nocc[m] = (int)w.size();
        } else {
            nocc[m] = b->mol_nelec[m] / 2;
            for (int k = 0; k < nocc[m]; ++k) occ_h[ebase[m] + k] = 2.0;
        }
    }
    const size_t P = (size_t)st.P;
    for (Dev<double>* d : {&st.S, &st.H, &st.X, &st.F, &st.D, &st.J, &st.K, &st.V, &st.C, &st.W1, &st.W2, &st.e,
                           &st.Vprev, &st.Dprev, &st.Jt, &st.Kt})
        MESS_CUDA_TRY(d->alloc(P));
    MESS_CUDA_TRY(st.Fh.alloc(P * diis_n));
    MESS_CUDA_TRY(st.eh.alloc(P * diis_n));
    MESS_CUDA_TRY(st.eps.alloc(etot));
    MESS_CUDA_TRY(st.occ.alloc(etot));
    MESS_CUDA_TRY(cudaMemcpy(st.occ.p, occ_h.data(), sizeof(double) * etot, cudaMemcpyHostToDevice));
    MESS_CUDA_TRY(st.E.alloc(b->nmol));
    MESS_CUDA_TRY(st.emax.alloc(b->nmol));
    MESS_CUDA_TRY(st.smin.alloc(b->nmol));
    MESS_CUDA_TRY(st.Bm.alloc((size_t)b->nmol * diis_n * diis_n));
    MESS_CUDA_TRY(st.base.alloc(b->nmol));
    MESS_CUDA_TRY(st.ebase.alloc(b->nmol));
    MESS_CUDA_TRY(st.n.alloc(b->nmol));
    MESS_CUDA_TRY(st.nocc.alloc(b->nmol));
    MESS_CUDA_TRY(st.sweeps.alloc(b->nmol));
    MESS_CUDA_TRY(st.active.alloc(b->nmol));
    MESS_CUDA_TRY(cudaMemcpy(st.base.p, b->mol_base.data(), sizeof(long long) * b->nmol, cudaMemcpyHostToDevice));
    MESS_CUDA_TRY(cudaMemcpy(st.ebase.p, ebase.data(), sizeof(long long) * b->nmol, cudaMemcpyHostToDevice));
    MESS_CUDA_TRY(cudaMemcpy(st.n.p, b->mol_nbf.data(), sizeof(int) * b->nmol, cudaMemcpyHostToDevice));
    MESS_CUDA_TRY(cudaMemcpy(st.nocc.p, nocc.data(), sizeof(int) * b->nmol, cudaMemcpyHostToDevice));
    {
        std::vector<unsigned char> act(b->nmol, 1);
        MESS_CUDA_TRY(cudaMemcpy(st.active.p, act.data(), b->nmol, cudaMemcpyHostToDevice));
    }
    st.L = Layout{st.base.p, st.n.p, st.nocc.p, st.active.p, st.occ.p, st.ebase.p};
    // Jacobi matrix in shared memory when it fits
    const size_t need = (size_t)st.maxn * st.maxn * sizeof(double);
    int dev = 0, smax = 0;
    MESS_CUDA_TRY(cudaGetDevice(&dev));
    MESS_CUDA_TRY(cudaDeviceGetAttribute(&smax, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    st.use_smem = need + 4096 <= (size_t)smax - 8192 ? 1 : 0;
    st.jac_smem = st.use_smem ? need : 0;
    if (!st.use_smem) MESS_CUDA_TRY(st.Wk.alloc(P));
    for (int m = 0; m < b->nmol; ++m) b->active[m] = 1;
    b->active_version++;

    // one-electron matrices, Loewdin X = S^-1/2
    MESS_CUDA_TRY(mess_launch_one_e(b, st.S.p, st.W1.p, st.W2.p, st.s));            // S, T, V
    const dim3 eg(64, b->nmol);
    k_axpbypcz<<<eg, 256, 0, st.s>>>(st.H.p, 1.0, st.W1.p, 1.0, st.W2.p, 0.0, nullptr, st.L);   // H = T + V
    MESS_CUDA_TRY(cudaGetLastError());
    MESS_CUDA_TRY(jacobi_prepare(st));
    MESS_CUDA_TRY(jacobi(st, st.S.p, st.V.p, st.fock_fp64));                          // S = U s U^T
    k_scale_cols<<<b->nmol, 256, 0, st.s>>>(st.V.p, st.eps.p, st.ebase.p, st.W1.p, st.L, st.smin.p);
    MESS_CUDA_TRY(cudaGetLastError());
    MESS_CUDA_TRY(gemm(st, true, st.W1.p, st.V.p, st.X.p, 0, 1.0));                 // X = U s^-1/2 U^T
    std::vector<double> hmin(b->nmol);
    MESS_CUDA_TRY(cudaMemcpyAsync(hmin.data(), st.smin.p, sizeof(double) * b->nmol, cudaMemcpyDeviceToHost, st.s));
    MESS_CUDA_TRY(cudaStreamSynchronize(st.s));
    for (int m = 0; m < b->nmol; ++m)
        if (!(hmin[m] > 1e-7)) { mess_set_error("molecule %d: overlap matrix nearly singular (%g)", m, hmin[m]); return MESS_ENUMERIC; }

    return MESS_OK;
}

mess_status scf_run(mess_basis* b, const mess_scf_opts* opts, mess_scf_result* res, double* D_out, bool D_out_device,
                    const std::vector<std::vector<double>>* occ_in)
{
    mess_scf_opts o{};
    if (opts) o = *opts;
    const int max_iter = o.max_iter > 0 ? o.max_iter : 100;
    const double conv_E = o.conv_E > 0 ? o.conv_E : 1e-10;
    const double conv_comm = o.conv_comm > 0 ? o.conv_comm : 1e-8;
    const int diis_n = std::min(o.diis_n > 0 ? o.diis_n : 8, 16);
    if (o.guess != MESS_GUESS_CORE && o.guess != MESS_GUESS_SAD && o.guess != MESS_GUESS_MLP) {
        mess_set_error("mess_scf: unknown initial guess %d", o.guess);
        return MESS_EINVAL;
    }
    if (b->max_nbf > 256) {
        mess_set_error("mess_scf: %d basis functions; the on-device eigensolver handles n <= 256", b->max_nbf);
        return MESS_ENOTIMPL;
    }
    SCFState st;
    PhaseTimer tm((cudaStream_t)o.cuda_stream);
    mess_status su = scf_setup(st, b, (cudaStream_t)o.cuda_stream, diis_n, occ_in, o.prec == MESS_FP64);
    if (su != MESS_OK) return su;
    tm.s = st.s;
    tm.mark(occ_in ? "scf (atoms): set-up" : "scf: set-up (pairs, one-electron matrices, orthogonaliser)");
    const size_t P = (size_t)st.P;
    const dim3 eg(64, b->nmol);
    std::vector<unsigned char> act(b->nmol, 1);

    // initial density: core Hamiltonian (eigenvectors of X H X), or the superposition of atomic densities
    st.warm = false;
    if (o.guess == MESS_GUESS_SAD && !occ_in) {
        mess_status gs = sad_density(b, o, st.D.p, st.s);
        if (gs != MESS_OK) return gs;
    } else if (o.guess == MESS_GUESS_MLP && !occ_in) {
        if (!o.mlp_weights) { mess_set_error("MESS_GUESS_MLP needs opts->mlp_weights"); return MESS_EINVAL; }
        mess_mlp* net = nullptr;
        mess_status gs = mess_mlp_load(o.mlp_weights, &net);
        if (gs != MESS_OK) return gs;
        gs = mess_mlp_guess_device(net, b, st.D.p, st.s);
        mess_mlp_destroy(net);
        if (gs != MESS_OK) return gs;
    } else {
        MESS_CUDA_TRY(density_from_fock(st, st.H.p));
    }
    MESS_CUDA_TRY(jacobi_prepare(st));   // a nested SCF of the atomic densities may have changed it
    tm.mark(occ_in ? "scf (atoms): initial density" : "scf: initial density");

    std::vector<double> Enuc(b->nmol), E(b->nmol);
    std::vector<int> iters(b->nmol, 0), conv(b->nmol, 0);
    for (int m = 0; m < b->nmol; ++m) {
        double e = 0.0;
        const int a0 = b->mol_atom_off[m], na = b->mol_atom_n[m];
        for (int a = a0; a < a0 + na; ++a)
            for (int c = a0; c < a; ++c) {
                double r2 = 0.0;
                for (int x = 0; x < 3; ++x) { const double d = b->xyz[3 * a + x] - b->xyz[3 * c + x]; r2 += d * d; }
                e += (double)b->Z[a] * b->Z[c] / sqrt(r2);
            }
        Enuc[m] = e;
    }
    mess_jk_opts jo{};
    jo.prec = o.prec;
    jo.schwarz_tau = o.schwarz_tau;
    jo.fp64_tau = o.fp64_tau;
    jo.boys_fp64 = o.boys_fp64;
    jo.split_df32 = o.split_df32;
    jo.cuda_stream = st.s;
    mess_status status = MESS_OK;
    // Iterations.  Every decision inside one iteration - which molecules still take part, a full or
    // an incremental Fock build, the DIIS slot - is read from device state, so the launches of one
    // iteration are the same every time: they are captured once into a CUDA graph and replayed.  The
    // host reads a status word (molecules left, errors) one iteration behind the GPU, and rebuilds
    // the quartet bins (then the graph) when fewer than half of the molecules they cover are left.
    // Incremental Fock builds: J(D_k) = J(D_{k-1}) + J(D_k - D_{k-1}) (J, K linear in D); the
    // reduced-precision error of each build then scales with |D_k - D_{k-1}|, which shrinks as the
    // SCF converges; a full build every full_every iterations resets the accumulation.
    const int full_every = 12;
    MESS_CUDA_TRY(st.Eold.alloc(b->nmol));
    MESS_CUDA_TRY(st.Efin.alloc(b->nmol));
    MESS_CUDA_TRY(st.iters.alloc(b->nmol));
    MESS_CUDA_TRY(st.conv.alloc(b->nmol));
    MESS_CUDA_TRY(st.state.alloc(4));
    {
        const int s0[4] = {0, b->nmol, 0, 0};
        MESS_CUDA_TRY(cudaMemcpyAsync(st.state.p, s0, sizeof(s0), cudaMemcpyHostToDevice, st.s));
        MESS_CUDA_TRY(cudaMemsetAsync(st.iters.p, 0, sizeof(int) * b->nmol, st.s));
        MESS_CUDA_TRY(cudaMemsetAsync(st.conv.p, 0, sizeof(int) * b->nmol, st.s));
        MESS_CUDA_TRY(cudaMemsetAsync(st.Eold.p, 0, sizeof(double) * b->nmol, st.s));
        MESS_CUDA_TRY(cudaStreamSynchronize(st.s));   // s0 is a stack array
    }
    {
        mess_status js = mess_jk_ensure_bins(b, &jo);
        if (js != MESS_OK) return js;
    }
    tm.mark("scf: quartet bins");
    // Kohn-Sham functionals: the grid and basis-function values (once per basis), E_xc and V_xc buffers
    Dev<double> Vxc, Exc;
    if (o.xc) {
        if (o.xc != 1 && o.xc != 2) { mess_set_error("mess_scf: unknown functional %d", o.xc); return MESS_EINVAL; }
        MESS_CUDA_TRY(Vxc.alloc(P));
        MESS_CUDA_TRY(Exc.alloc(b->nmol));
        mess_status xs = mess_xc_prepare(b, st.s);
        if (xs != MESS_OK) return xs;
    }
    // F = H + J - K/2 (Hartree-Fock) or H + J + V_xc (Kohn-Sham) from the accumulated J, K, and its energy
    auto fock_energy = [&]() -> mess_status {
        if (o.xc) {
            mess_status xs = mess_xc_eval(b, o.xc, st.D.p, Vxc.p, Exc.p, st.s);
            if (xs != MESS_OK) return xs;
            k_axpbypcz<<<eg, 256, 0, st.s>>>(st.F.p, 1.0, st.H.p, 1.0, st.Jt.p, 1.0, Vxc.p, st.L);
            k_energy_ks<<<b->nmol, 256, 0, st.s>>>(st.D.p, st.H.p, st.Jt.p, Exc.p, st.L, st.E.p);
        } else {
            k_axpbypcz<<<eg, 256, 0, st.s>>>(st.F.p, 1.0, st.H.p, 1.0, st.Jt.p, -0.5, st.Kt.p, st.L);
            k_energy<<<b->nmol, 256, 0, st.s>>>(st.D.p, st.H.p, st.F.p, st.L, st.E.p);
        }
        MESS_CUDA_TRY(cudaGetLastError());
        return MESS_OK;
    };
    // the J/K kernels skip the quartets of molecules that have left (device flags) and, with a
    // screening threshold, the quartets whose contribution from this iteration's density change
    // stays below it (density-weighted screening of the incremental builds)
    const bool dscreen = o.dens_tau > 0.0;
    Dev<float> rowmax, dmax;
    Dev<int> fbase;
    if (dscreen) {
        MESS_CUDA_TRY(rowmax.alloc((size_t)b->nbf));
        MESS_CUDA_TRY(dmax.alloc((size_t)std::max(1, b->npair)));
        std::vector<int> fb(b->nmol, 0);
        for (int m = 1; m < b->nmol; ++m) fb[m] = fb[m - 1] + b->mol_nbf[m - 1];
        MESS_CUDA_TRY(fbase.alloc(b->nmol));
        MESS_CUDA_TRY(cudaMemcpy(fbase.p, fb.data(), sizeof(int) * b->nmol, cudaMemcpyHostToDevice));
    }
    struct ScreenReset {
        mess_basis* b;
        void off()
        {
            for (auto* P : {&b->P64.active, &b->P32.active, &b->Pdf.active}) *P = nullptr;
            b->P64.dmax = nullptr; b->P32.dmax = nullptr; b->Pdf.dmax = nullptr;
        }
        ~ScreenReset() { off(); }
    } screen_reset{b};
    b->P64.active = b->P32.active = b->Pdf.active = st.active.p;
    if (dscreen) {
        b->P64.dmax = b->P32.dmax = b->Pdf.dmax = dmax.p;
        b->P64.dtau = b->P32.dtau = b->Pdf.dtau = (float)o.dens_tau;
    }
    auto iteration = [&]() -> mess_status {
        k_iter_begin<<<1, 1, 0, st.s>>>(st.state.p);
        k_delta<<<eg, 256, 0, st.s>>>(st.D.p, st.Dprev.p, st.W1.p, st.Jt.p, st.Kt.p, st.L, st.state.p, full_every);
        MESS_CUDA_TRY(cudaGetLastError());
        if (dscreen) {
            k_rowmax<<<dim3((st.maxn + 127) / 128, b->nmol), 128, 0, st.s>>>(st.W1.p, st.L, fbase.p, rowmax.p);
            k_pairmax<<<(b->npair + 255) / 256, 256, 0, st.s>>>(rowmax.p, b->d_pair_a.p, b->d_pair_b.p,
                                                                   b->d_shell_f0.p, b->d_shell_l.p, dmax.p, b->npair);
            MESS_CUDA_TRY(cudaGetLastError());
        }
        mess_status js = mess_jk_enqueue_only(b, st.W1.p, st.J.p, st.K.p, &jo);
        if (js != MESS_OK) return js;
        k_axpbypcz<<<eg, 256, 0, st.s>>>(st.Jt.p, 1.0, st.Jt.p, 1.0, st.J.p, 0.0, nullptr, st.L);
        k_axpbypcz<<<eg, 256, 0, st.s>>>(st.Kt.p, 1.0, st.Kt.p, 1.0, st.K.p, 0.0, nullptr, st.L);
        const mess_status fe = fock_energy();
        if (fe != MESS_OK) return fe;
        MESS_CUDA_TRY(gemm(st, false, st.F.p, st.D.p, st.W1.p, 0, 1.0));   // F D
        MESS_CUDA_TRY(gemm(st, false, st.W1.p, st.S.p, st.W2.p, 0, 1.0));  // F D S
        k_commutator<<<b->nmol, 256, 0, st.s>>>(st.W2.p, st.e.p, st.L, st.emax.p);
        k_converge<<<(b->nmol + 127) / 128, 128, 0, st.s>>>(st.E.p, st.emax.p, st.Eold.p, st.iters.p, st.conv.p,
                                                             st.Efin.p, st.active.p, st.state.p, b->nmol, conv_E,
                                                             conv_comm);
        // DIIS extrapolation of F, then the new density (molecules that just converged are skipped)
        k_diis<<<b->nmol, 256, 0, st.s>>>(st.Fh.p, st.eh.p, (long long)P, st.F.p, st.e.p, st.L, st.state.p, diis_n,
                                          st.Bm.p);
        MESS_CUDA_TRY(cudaGetLastError());
        MESS_CUDA_TRY(density_from_fock(st, st.F.p));
        return MESS_OK;
    };
    cudaGraphExec_t gexec = nullptr;
    struct GraphGuard {
        cudaGraphExec_t* g;
        ~GraphGuard() { if (*g) cudaGraphExecDestroy(*g); }
    } graph_guard{&gexec};
    bool use_graph = true;
    auto capture = [&]() {
        if (gexec) { cudaGraphExecDestroy(gexec); gexec = nullptr; }
        cudaGraph_t g = nullptr;
        if (cudaStreamBeginCapture(st.s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) { use_graph = false; return; }
        const mess_status r = iteration();
        const cudaError_t e = cudaStreamEndCapture(st.s, &g);
        if (r == MESS_OK && e == cudaSuccess && g && cudaGraphInstantiate(&gexec, g, 0) != cudaSuccess) gexec = nullptr;
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();            // a failed capture leaves nothing sticky: iterate without a graph
        if (!gexec) use_graph = false;
    };
    // status of iteration k is copied into hstat[k % 2] (page-locked), then event hev[k % 2]
    struct HostStatus {
        int* h = nullptr;
        cudaEvent_t ev[2] = {nullptr, nullptr};
        ~HostStatus()
        {
            if (h) cudaFreeHost(h);
            for (auto e : ev) if (e) cudaEventDestroy(e);
        }
    } hs;
    MESS_CUDA_TRY(cudaHostAlloc((void**)&hs.h, 8 * sizeof(int), cudaHostAllocDefault));
    for (auto& e : hs.ev) MESS_CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    int remaining = b->nmol, bins_cover = b->nmol, err_mol = 0;
    for (auto& a : act) a = 1;
    for (int it = 1; it <= max_iter; ++it) {
        if (use_graph && it >= 2 && !gexec) capture();
        if (gexec) MESS_CUDA_TRY(cudaGraphLaunch(gexec, st.s));
        else {
            const mess_status r = iteration();
            if (r != MESS_OK) return r;
        }
        MESS_CUDA_TRY(cudaMemcpyAsync(hs.h + 4 * (it % 2), st.state.p, 4 * sizeof(int), cudaMemcpyDeviceToHost, st.s));
        MESS_CUDA_TRY(cudaEventRecord(hs.ev[it % 2], st.s));
        // the previous iteration's status, while this one runs (the first iteration waits for itself)
        const int k = it >= 2 ? it - 1 : it;
        MESS_CUDA_TRY(cudaEventSynchronize(hs.ev[k % 2]));
        remaining = hs.h[4 * (k % 2) + 1];
        err_mol = hs.h[4 * (k % 2) + 2];
        if (tm.on) {
            char lbl[96];
            snprintf(lbl, sizeof lbl, "scf: iteration %d (%d molecules left after iteration %d)", it, remaining, k);
            tm.mark(lbl);
        }
        if (err_mol) break;
        if (remaining == 0) break;
        if (remaining * 2 < bins_cover && it < max_iter) {
            // rebuild the bins over the molecules still iterating (and the graph with them)
            MESS_CUDA_TRY(cudaStreamSynchronize(st.s));
            MESS_CUDA_TRY(cudaMemcpy(act.data(), st.active.p, b->nmol, cudaMemcpyDeviceToHost));
            remaining = 0;
            for (int m = 0; m < b->nmol; ++m) { b->active[m] = act[m]; remaining += act[m] ? 1 : 0; }
            if (remaining == 0) break;
            b->active_version++;
            mess_status js = mess_jk_ensure_bins(b, &jo);
            if (js != MESS_OK) return js;
            bins_cover = remaining;
            if (gexec) { cudaGraphExecDestroy(gexec); gexec = nullptr; }
            tm.mark("scf: quartet bins rebuilt");
        }
    }
    MESS_CUDA_TRY(cudaStreamSynchronize(st.s));
    if (err_mol) {
        mess_set_error("molecule %d: non-finite energy or error during the SCF", err_mol - 1);
        return MESS_ENUMERIC;
    }
    {
        int sfinal[4];
        MESS_CUDA_TRY(cudaMemcpy(sfinal, st.state.p, sizeof(sfinal), cudaMemcpyDeviceToHost));
        if (sfinal[2]) {
            mess_set_error("molecule %d: non-finite energy or error during the SCF", sfinal[2] - 1);
            return MESS_ENUMERIC;
        }
    }
    std::vector<double> Ef(b->nmol);
    MESS_CUDA_TRY(cudaMemcpy(iters.data(), st.iters.p, sizeof(int) * b->nmol, cudaMemcpyDeviceToHost));
    MESS_CUDA_TRY(cudaMemcpy(conv.data(), st.conv.p, sizeof(int) * b->nmol, cudaMemcpyDeviceToHost));
    MESS_CUDA_TRY(cudaMemcpy(Ef.data(), st.Efin.p, sizeof(double) * b->nmol, cudaMemcpyDeviceToHost));
    MESS_CUDA_TRY(cudaMemcpy(E.data(), st.E.p, sizeof(double) * b->nmol, cudaMemcpyDeviceToHost));
    for (int m = 0; m < b->nmol; ++m) {
        if (!conv[m] || !res) continue;
        res[m].E_elec = Ef[m];
        res[m].E_nuc = Enuc[m];
        res[m].E_total = Ef[m] + Enuc[m];
        res[m].E_iter = res[m].E_total;
        res[m].iterations = iters[m];
        res[m].converged = 1;
    }
    for (int m = 0; m < b->nmol; ++m) {
        if (conv[m]) continue;
        status = MESS_ENOCONV;
        if (res) {
            res[m].E_elec = E[m];
            res[m].E_nuc = Enuc[m];
            res[m].E_total = E[m] + Enuc[m];
            res[m].E_iter = res[m].E_total;
            res[m].iterations = iters[m];
            res[m].converged = 0;
        }
    }
    if (o.prec != MESS_FP64 && !occ_in) {
        // Reported energy of the reduced-precision forms: E at the final density from one full Fock
        // build in which the quartets above a ten times lower split threshold (MESS_MIXED; every
        // quartet for MESS_FP32) run in FP64-class arithmetic (double-float if split_df32, else
        // FP64).  Most of the integrals' rounding then leaves the energy, and the density's own
        // deviation from the FP64 solution enters it only at second order (E is stationary there).
        screen_reset.off();            // the energy's build: Schwarz screening only, every molecule
        for (int m = 0; m < b->nmol; ++m) { act[m] = 1; b->active[m] = 1; }
        b->active_version++;
        MESS_CUDA_TRY(cudaMemcpyAsync(st.active.p, act.data(), b->nmol, cudaMemcpyHostToDevice, st.s));
        mess_jk_opts jf = jo;
        jf.prec = MESS_MIXED;
        // ten times more of the largest quartets in FP64-class arithmetic than in the iterations
        const double it_tau = o.prec == MESS_MIXED ? (o.fp64_tau > 0.0 ? o.fp64_tau : MESS_DEFAULT_FP64_TAU) : 0.0;
        jf.fp64_tau = it_tau > 0.0 ? 0.1 * it_tau : 1e-300;
        mess_status js = mess_jk_packed(b, st.D.p, st.Jt.p, st.Kt.p, &jf, nullptr);
        if (js != MESS_OK) return js;
        js = fock_energy();
        if (js != MESS_OK) return js;
        MESS_CUDA_TRY(cudaMemcpyAsync(E.data(), st.E.p, sizeof(double) * b->nmol, cudaMemcpyDeviceToHost, st.s));
        MESS_CUDA_TRY(cudaStreamSynchronize(st.s));
        tm.mark("scf: final energy (bins and build)");
        for (int m = 0; m < b->nmol; ++m) {
            if (!std::isfinite(E[m])) { mess_set_error("molecule %d: non-finite final energy", m); return MESS_ENUMERIC; }
            if (res) {
                res[m].E_elec = E[m];
                res[m].E_total = E[m] + Enuc[m];
            }
        }
    }
    if (status == MESS_ENOCONV) mess_set_error("SCF did not converge within %d iterations", max_iter);
    if (D_out) {
        if (D_out_device) MESS_CUDA_TRY(cudaMemcpyAsync(D_out, st.D.p, sizeof(double) * P, cudaMemcpyDeviceToDevice, st.s));
        else MESS_CUDA_TRY(cudaMemcpyAsync(D_out, st.D.p, sizeof(double) * P, cudaMemcpyDeviceToHost, st.s));
    }
    MESS_CUDA_TRY(cudaStreamSynchronize(st.s));
    for (int m = 0; m < b->nmol; ++m) b->active[m] = 1;
    b->active_version++;
    return status;
}

// ------------------------------------------------------------------------------------------------
// Direct minimisation of the energy functional (paper Sec. 3: min E(C) subject to C^T S C = 1;
// Sec. 5.1 / 5.2: Adam on unconstrained parameters, the constraint built in by a QR decomposition).
// Per molecule, parameters Z (n x n):
//   Z = Q R (Householder),  C = X Q (X = S^-1/2),  D = 2 C_occ C_occ^T,  F = H + J(D) - K(D)/2,
//   E = 1/2 sum D (H + F) + E_nuc;
//   dE/dC_occ = 4 F C_occ (other columns 0),  G = X^T dE/dC,
//   dE/dZ = Q tril(Q^T G - G^T Q, -1) R^-T   (Q^T dQ is skew and dR R^-1 upper triangular, so a
//   perturbation of Z moves Q by Q times the strictly lower part of Q^T dZ R^-1 minus its transpose);
//   Adam: m = b1 m + (1 - b1) g, v = b2 v + (1 - b2) g^2, Z -= lr m_hat / (sqrt(v_hat) + eps).
// ------------------------------------------------------------------------------------------------

// Householder QR of each molecule's Z: R (upper triangular, in place of a copy of Z), the unit
// reflectors in the columns of Vh, and Q = H_0 H_1 ... H_{n-2} formed explicitly.  One block per
// molecule.  singular[m] = 1 if a diagonal element of R is zero.
__global__ void k_qr(const double* __restrict__ Z, double* __restrict__ Q, double* __restrict__ R,
                     double* __restrict__ Vh, Layout L, int* __restrict__ singular)
{
    __shared__ double red[32];
    const int m = blockIdx.x;
    if (!L.active[m]) return;
    const int n = L.n[m];
    const long long o = L.base[m];
    double* A = R + o;
    double* V = Vh + o;
    double* Qm = Q + o;
    for (long long t = threadIdx.x; t < (long long)n * n; t += blockDim.x) { A[t] = Z[o + t]; V[t] = 0.0; }
    __syncthreads();
    for (int k = 0; k < n - 1; ++k) {
        double ss = 0.0;
        for (int i = k + threadIdx.x; i < n; i += blockDim.x) ss += A[(long long)i * n + k] * A[(long long)i * n + k];
        ss = block_sum(ss, red);
        const double x0 = A[(long long)k * n + k];
        const double nrm = sqrt(ss);
        const double alpha = x0 >= 0.0 ? -nrm : nrm;      // R_kk; the sign avoids cancellation in x0 - alpha
        const double vn2 = 2.0 * nrm * (nrm + fabs(x0));  // |x - alpha e_k|^2
        if (vn2 > 0.0) {
            const double inv = 1.0 / sqrt(vn2);
            for (int i = k + threadIdx.x; i < n; i += blockDim.x)
                V[(long long)i * n + k] = (i == k ? x0 - alpha : A[(long long)i * n + k]) * inv;
        }
        __syncthreads();
        if (vn2 > 0.0) {
            for (int j = k + threadIdx.x; j < n; j += blockDim.x) {
                double d = 0.0;
                for (int i = k; i < n; ++i) d += V[(long long)i * n + k] * A[(long long)i * n + j];
                d *= 2.0;
                for (int i = k; i < n; ++i) A[(long long)i * n + j] -= d * V[(long long)i * n + k];
            }
        }
        __syncthreads();
    }
    int sing = 0;
    for (long long t = threadIdx.x; t < (long long)n * n; t += blockDim.x) {
        const int i = (int)(t / n), j = (int)(t % n);
        if (i > j) A[t] = 0.0;
        if (i == j && A[t] == 0.0) sing = 1;
        Qm[t] = i == j ? 1.0 : 0.0;
    }
    if (sing) singular[m] = 1;
    __syncthreads();
    for (int k = n - 2; k >= 0; --k) {
        for (int j = threadIdx.x; j < n; j += blockDim.x) {
            double d = 0.0;
            for (int i = k; i < n; ++i) d += V[(long long)i * n + k] * Qm[(long long)i * n + j];
            d *= 2.0;
            for (int i = k; i < n; ++i) Qm[(long long)i * n + j] -= d * V[(long long)i * n + k];
        }
        __syncthreads();
    }
}

// G = scale * W on the occupied columns (j < nocc), 0 on the others
__global__ void k_occ_cols(const double* __restrict__ W, double* __restrict__ G, Layout L, double scale)
{
    const int m = blockIdx.y;
    if (!L.active[m]) return;
    const int n = L.n[m], no = L.nocc[m];
    const long long o = L.base[m];
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < (long long)n * n;
         t += (long long)gridDim.x * blockDim.x)
        G[o + t] = (t % n) < no ? scale * W[o + t] : 0.0;
}

// B = tril(A - A^T, -1)
__global__ void k_skew_lower(const double* __restrict__ A, double* __restrict__ B, Layout L)
{
    const int m = blockIdx.y;
    if (!L.active[m]) return;
    const int n = L.n[m];
    const long long o = L.base[m];
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < (long long)n * n;
         t += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(t / n), j = (int)(t % n);
        B[o + t] = i > j ? A[o + t] - A[o + (long long)j * n + i] : 0.0;
    }
}

// X R^T = W for X (R upper triangular): row by row, back substitution over the columns; one
// thread per row, one block per molecule.  gmax[m] = max |X|.
__global__ void k_solve_rt(const double* __restrict__ W, const double* __restrict__ R, double* __restrict__ X,
                           Layout L, double* __restrict__ gmax)
{
    __shared__ double red[32];
    const int m = blockIdx.x;
    if (!L.active[m]) return;
    const int n = L.n[m];
    const long long o = L.base[m];
    double mx = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const double* w = W + o + (long long)i * n;
        double* x = X + o + (long long)i * n;
        for (int j = n - 1; j >= 0; --j) {
            double t = w[j];
            for (int k = j + 1; k < n; ++k) t -= x[k] * R[o + (long long)j * n + k];
            x[j] = t / R[o + (long long)j * n + j];
            mx = fmax(mx, fabs(x[j]));
        }
    }
    mx = block_max(mx, red);
    if (threadIdx.x == 0) gmax[m] = mx;
}

// one Adam step on every element of Z (c1 = 1 - b1^t, c2 = 1 - b2^t)
__global__ void k_adam(double* __restrict__ Z, const double* __restrict__ G, double* __restrict__ Mm,
                       double* __restrict__ Vv, Layout L, double lr, double b1, double b2, double eps, double c1,
                       double c2)
{
    const int m = blockIdx.y;
    if (!L.active[m]) return;
    const long long nn = (long long)L.n[m] * L.n[m], o = L.base[m];
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < nn; t += (long long)gridDim.x * blockDim.x) {
        const double g = G[o + t];
        const double mm = b1 * Mm[o + t] + (1.0 - b1) * g;
        const double vv = b2 * Vv[o + t] + (1.0 - b2) * g * g;
        Mm[o + t] = mm;
        Vv[o + t] = vv;
        Z[o + t] -= lr * (mm / c1) / (sqrt(vv / c2) + eps);
    }
}

// trace[step * nmol + m] = E_elec[m] + E_nuc[m]
__global__ void k_trace(const double* __restrict__ E, const double* __restrict__ Enuc, double* __restrict__ trace,
                        int nmol)
{
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m < nmol) trace[m] = E[m] + Enuc[m];
}

// Z = identity in every molecule's block
__global__ void k_identity(double* __restrict__ Z, Layout L)
{
    const int m = blockIdx.y;
    const int n = L.n[m];
    const long long o = L.base[m];
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < (long long)n * n;
         t += (long long)gridDim.x * blockDim.x)
        Z[o + t] = (t / n) == (t % n) ? 1.0 : 0.0;
}

mess_status min_run(mess_basis* b, const mess_min_opts* opts, mess_scf_result* res, double* trace_out)
{
    mess_min_opts o{};
    if (opts) o = *opts;
    const int steps = o.steps > 0 ? o.steps : 200;
    const double lr = o.lr > 0 ? o.lr : 0.1, b1 = o.beta1 > 0 ? o.beta1 : 0.9, b2 = o.beta2 > 0 ? o.beta2 : 0.999;
    const double eps = o.eps > 0 ? o.eps : 1e-8, gtol = o.grad_tol > 0 ? o.grad_tol : 1e-5;
    if (!(lr < 1e3) || !(b1 < 1.0) || !(b2 < 1.0)) { mess_set_error("mess_minimise: bad Adam parameters"); return MESS_EINVAL; }
    if (b->max_nbf > 256) {
        mess_set_error("mess_minimise: %d basis functions; the set-up eigensolver handles n <= 256", b->max_nbf);
        return MESS_ENOTIMPL;
    }
    SCFState st;
    mess_status su = scf_setup(st, b, (cudaStream_t)o.cuda_stream, 1, nullptr, o.prec == MESS_FP64);
    if (su != MESS_OK) return su;
    const size_t P = (size_t)st.P;
    const int nmol = b->nmol;
    const dim3 eg(64, nmol);
    Dev<double> Z, Q, R, Vh, G, Mm, Vv, Enuc_d, trace, gmax;
    Dev<int> singular;
    for (Dev<double>* d : {&Z, &Q, &R, &Vh, &G, &Mm, &Vv}) MESS_CUDA_TRY(d->alloc(P));
    MESS_CUDA_TRY(Enuc_d.alloc(nmol));
    MESS_CUDA_TRY(gmax.alloc(nmol));
    MESS_CUDA_TRY(trace.alloc((size_t)(steps + 1) * nmol));
    MESS_CUDA_TRY(singular.alloc(nmol));
    Dev<double> Vxc, Exc;
    if (o.xc) {
        if (o.xc != 1 && o.xc != 2) { mess_set_error("mess_minimise: unknown functional %d", o.xc); return MESS_EINVAL; }
        MESS_CUDA_TRY(Vxc.alloc(P));
        MESS_CUDA_TRY(Exc.alloc(nmol));
        mess_status xs = mess_xc_prepare(b, st.s);
        if (xs != MESS_OK) return xs;
    }
    std::vector<double> Enuc(nmol);
    for (int m = 0; m < nmol; ++m) {
        double e = 0.0;
        const int a0 = b->mol_atom_off[m], na = b->mol_atom_n[m];
        for (int a = a0; a < a0 + na; ++a)
            for (int c = a0; c < a; ++c) {
                double r2 = 0.0;
                for (int x = 0; x < 3; ++x) { const double d = b->xyz[3 * a + x] - b->xyz[3 * c + x]; r2 += d * d; }
                e += (double)b->Z[a] * b->Z[c] / sqrt(r2);
            }
        Enuc[m] = e;
    }
    MESS_CUDA_TRY(cudaMemcpyAsync(Enuc_d.p, Enuc.data(), sizeof(double) * nmol, cudaMemcpyHostToDevice, st.s));
    MESS_CUDA_TRY(cudaMemsetAsync(Mm.p, 0, sizeof(double) * P, st.s));
    MESS_CUDA_TRY(cudaMemsetAsync(Vv.p, 0, sizeof(double) * P, st.s));
    MESS_CUDA_TRY(cudaMemsetAsync(singular.p, 0, sizeof(int) * nmol, st.s));
    k_identity<<<eg, 256, 0, st.s>>>(Z.p, st.L);                  // the paper's start: Z = 1
    MESS_CUDA_TRY(cudaGetLastError());
    mess_jk_opts jo{};
    jo.prec = o.prec;
    jo.schwarz_tau = o.schwarz_tau;
    jo.fp64_tau = o.fp64_tau;
    jo.boys_fp64 = o.boys_fp64;
    jo.split_df32 = o.split_df32;
    jo.cuda_stream = st.s;
    // E(Z) on every molecule (trace row `row`), and with grad = true dE/dZ into G
    auto energy = [&](int row, bool grad) -> mess_status {
        k_qr<<<nmol, 256, 0, st.s>>>(Z.p, Q.p, R.p, Vh.p, st.L, singular.p);
        MESS_CUDA_TRY(cudaGetLastError());
        MESS_CUDA_TRY(gemm(st, false, st.X.p, Q.p, st.C.p, 0, 1.0));        // C = X Q
        MESS_CUDA_TRY(gemm(st, true, st.C.p, st.C.p, st.D.p, 1, 1.0));      // D = C diag(occ) C^T
        mess_status js = mess_jk_packed(b, st.D.p, st.J.p, st.K.p, &jo, nullptr);
        if (js != MESS_OK) return js;
        if (o.xc) {                                                          // F = H + J + V_xc (Kohn-Sham)
            js = mess_xc_eval(b, o.xc, st.D.p, Vxc.p, Exc.p, st.s);
            if (js != MESS_OK) return js;
            k_axpbypcz<<<eg, 256, 0, st.s>>>(st.F.p, 1.0, st.H.p, 1.0, st.J.p, 1.0, Vxc.p, st.L);
            k_energy_ks<<<nmol, 256, 0, st.s>>>(st.D.p, st.H.p, st.J.p, Exc.p, st.L, st.E.p);
        } else {                                                             // F = H + J - K/2
            k_axpbypcz<<<eg, 256, 0, st.s>>>(st.F.p, 1.0, st.H.p, 1.0, st.J.p, -0.5, st.K.p, st.L);
            k_energy<<<nmol, 256, 0, st.s>>>(st.D.p, st.H.p, st.F.p, st.L, st.E.p);
        }
        k_trace<<<(nmol + 127) / 128, 128, 0, st.s>>>(st.E.p, Enuc_d.p, trace.p + (size_t)row * nmol, nmol);
        MESS_CUDA_TRY(cudaGetLastError());
        if (!grad) return MESS_OK;
        MESS_CUDA_TRY(gemm(st, false, st.F.p, st.C.p, st.W1.p, 0, 1.0));    // F C
        k_occ_cols<<<eg, 256, 0, st.s>>>(st.W1.p, st.W2.p, st.L, 4.0);     // dE/dC = 4 F C_occ
        MESS_CUDA_TRY(cudaGetLastError());
        MESS_CUDA_TRY(gemm(st, false, st.X.p, st.W2.p, st.W1.p, 0, 1.0));   // G = X^T dE/dC (X symmetric)
        MESS_CUDA_TRY(gemm(st, false, Q.p, st.W1.p, st.W2.p, 0, 1.0, true)); // A = Q^T G
        k_skew_lower<<<eg, 256, 0, st.s>>>(st.W2.p, st.W1.p, st.L);          // B = tril(A - A^T, -1)
        MESS_CUDA_TRY(cudaGetLastError());
        MESS_CUDA_TRY(gemm(st, false, Q.p, st.W1.p, st.W2.p, 0, 1.0));      // Q B
        k_solve_rt<<<nmol, 128, 0, st.s>>>(st.W2.p, R.p, G.p, st.L, gmax.p); // dE/dZ = Q B R^-T
        MESS_CUDA_TRY(cudaGetLastError());
        return MESS_OK;
    };
    double c1 = 1.0, c2 = 1.0;
    for (int t = 1; t <= steps; ++t) {
        mess_status r = energy(t - 1, true);
        if (r != MESS_OK) return r;
        c1 *= b1;
        c2 *= b2;
        k_adam<<<eg, 256, 0, st.s>>>(Z.p, G.p, Mm.p, Vv.p, st.L, lr, b1, b2, eps, 1.0 - c1, 1.0 - c2);
        MESS_CUDA_TRY(cudaGetLastError());
    }
    mess_status r = energy(steps, true);     // the energy (and gradient size) at the final parameters
    if (r != MESS_OK) return r;
    std::vector<double> tr((size_t)(steps + 1) * nmol), gm(nmol);
    std::vector<int> sing(nmol);
    MESS_CUDA_TRY(cudaMemcpyAsync(tr.data(), trace.p, sizeof(double) * tr.size(), cudaMemcpyDeviceToHost, st.s));
    MESS_CUDA_TRY(cudaMemcpyAsync(gm.data(), gmax.p, sizeof(double) * nmol, cudaMemcpyDeviceToHost, st.s));
    MESS_CUDA_TRY(cudaMemcpyAsync(sing.data(), singular.p, sizeof(int) * nmol, cudaMemcpyDeviceToHost, st.s));
    MESS_CUDA_TRY(cudaStreamSynchronize(st.s));
    mess_status status = MESS_OK;
    for (int m = 0; m < nmol; ++m) {
        const double E = tr[(size_t)steps * nmol + m];
        if (sing[m] || !std::isfinite(E)) {
            mess_set_error("molecule %d: %s", m, sing[m] ? "the parameters became singular (a zero diagonal of R)"
                                                         : "non-finite energy");
            return MESS_ENUMERIC;
        }
        const bool conv = gm[m] < gtol;
        if (!conv) status = MESS_ENOCONV;
        if (res) {
            res[m].E_total = E;
            res[m].E_nuc = Enuc[m];
            res[m].E_elec = E - Enuc[m];
            res[m].E_iter = E;
            res[m].iterations = steps;
            res[m].converged = conv ? 1 : 0;
        }
    }
    if (trace_out) memcpy(trace_out, tr.data(), sizeof(double) * (size_t)steps * nmol);
    for (int m = 0; m < nmol; ++m) b->active[m] = 1;
    if (status == MESS_ENOCONV)
        mess_set_error("mess_minimise: the largest |dE/dZ| after %d steps is above %g for some molecule", steps, gtol);
    return status;
}

}  // namespace

mess_status mess_scf_batch_density(mess_basis* b, const mess_scf_opts* opts, mess_scf_result* res, double* dD)
{
    return scf_run(b, opts, res, dD, true);
}

extern "C" mess_status mess_scf(const mess_basis* bc, const mess_scf_opts* opts, mess_scf_result* res, double* D_out)
{
    mess_basis* b = const_cast<mess_basis*>(bc);
    if (!b || !res) { mess_set_error("null argument"); return MESS_EINVAL; }
    { const mess_status gs = mess_basis_gpu(b); if (gs != MESS_OK) return gs; }
    return scf_run(b, opts, res, D_out, false);
}

extern "C" mess_status mess_scf_batch(int nmol, mess_basis* const* bases, const mess_scf_opts* opts, mess_scf_result* res)
{
    if (nmol <= 0 || !bases || !res) { mess_set_error("bad batch arguments"); return MESS_EINVAL; }
    mess_basis* batch = nullptr;
    PhaseTimer tm(opts ? (cudaStream_t)opts->cuda_stream : nullptr);
    mess_status st = mess_batch_basis(nmol, bases, &batch);
    if (st != MESS_OK) return st;
    tm.mark("scf batch: batched basis");
    st = scf_run(batch, opts, res, nullptr, false);
    mess_free_basis(batch);
    delete batch;
    return st;
}

extern "C" mess_status mess_minimise(const mess_basis* bc, const mess_min_opts* opts, mess_scf_result* res,
                                     double* trace)
{
    mess_basis* b = const_cast<mess_basis*>(bc);
    if (!b || !res) { mess_set_error("null argument"); return MESS_EINVAL; }
    { const mess_status gs = mess_basis_gpu(b); if (gs != MESS_OK) return gs; }
    return min_run(b, opts, res, trace);
}

extern "C" mess_status mess_minimise_batch(int nmol, mess_basis* const* bases, const mess_min_opts* opts,
                                           mess_scf_result* res, double* trace)
{
    if (nmol <= 0 || !bases || !res) { mess_set_error("bad batch arguments"); return MESS_EINVAL; }
    mess_basis* batch = nullptr;
    mess_status st = mess_batch_basis(nmol, bases, &batch);
    if (st != MESS_OK) return st;
    st = min_run(batch, opts, res, trace);
    mess_free_basis(batch);
    delete batch;
    return st;
}
