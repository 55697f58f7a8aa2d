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
__global__ void k_diis(double* __restrict__ Fh, double* __restrict__ eh, long long hstride, double* __restrict__ F,
                       const double* __restrict__ e, Layout L, int slot, int nstored, int nmax,
                       double* __restrict__ Bm)
{
    __shared__ double red[32];
    __shared__ double coef[16];
    __shared__ int ok;
    const int m = blockIdx.x;
    if (!L.active[m]) return;
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

// Cyclic Jacobi eigensolver of the symmetric n x n block of each molecule, one thread block per
// molecule, rotations in parallel over disjoint index pairs (round-robin "circle" schedule).  The
// rotation of (p, q) uses tau = (a_qq - a_pp)/(2 a_pq), t = sign(tau)/(|tau| + sqrt(1 + tau^2)),
// c = 1/sqrt(1 + t^2), s = t c, and A <- J^T A J, V <- V J.  Eigenvalues ascending in eps, the
// matching eigenvectors as the columns of Vout.  The matrix lives in shared memory when it fits,
// otherwise in the global workspace Wk.
__global__ void k_jacobi(const double* __restrict__ Ain, double* __restrict__ V, double* __restrict__ Vout,
                         double* __restrict__ eps, const long long* __restrict__ ebase, Layout L, int use_smem,
                         double* __restrict__ Wk, int max_sweeps, int* __restrict__ sweeps_out)
{
    extern __shared__ __align__(16) double jsm[];
    __shared__ double red[32];
    __shared__ int pp_[128], qq_[128];
    __shared__ double cc_[128], ss_[128];
    __shared__ int rotated;
    const int m = blockIdx.x;
    if (!L.active[m]) return;
    const int n = L.n[m];
    const long long o = L.base[m];
    double* A = use_smem ? jsm : Wk + o;
    const int npad = n + (n & 1), half = npad / 2, rounds = npad - 1;
    for (long long t = threadIdx.x; t < (long long)n * n; t += blockDim.x) {
        A[t] = Ain[o + t];
        const int i = (int)(t / n), j = (int)(t % n);
        V[o + t] = (i == j) ? 1.0 : 0.0;
    }
    __syncthreads();
    double nrm = 0.0;
    for (long long t = threadIdx.x; t < (long long)n * n; t += blockDim.x) nrm += A[t] * A[t];
    nrm = block_sum(nrm, red);
    int sweep = 0;
    for (; sweep < max_sweeps; ++sweep) {
        double off = 0.0;
        for (long long t = threadIdx.x; t < (long long)n * n; t += blockDim.x) {
            const int i = (int)(t / n), j = (int)(t % n);
            if (i != j) off += A[t] * A[t];
        }
        off = block_sum(off, red);
        if (off <= 1e-28 * nrm || off == 0.0) break;
        if (threadIdx.x == 0) rotated = 0;
        __syncthreads();
        for (int r = 0; r < rounds; ++r) {
            for (int k = threadIdx.x; k < half; k += blockDim.x) {
                int a, b2;
                if (k == 0) { a = rounds; b2 = r; }
                else { a = (r + k) % rounds; b2 = (r - k + rounds) % rounds; }
                const int p = min(a, b2), q = max(a, b2);
                double c = 1.0, s = 0.0;
                if (q < n) {
                    const double apq = A[(long long)p * n + q];
                    const double app = A[(long long)p * n + p], aqq = A[(long long)q * n + q];
                    // rotate unless a_pq is negligible against the diagonal (round-off level)
                    if (fabs(apq) > 1e-300 && fabs(apq) > 1e-15 * sqrt(fabs(app) * fabs(aqq))) {
                        const double tau = (aqq - app) / (2.0 * apq);
                        const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                        c = 1.0 / sqrt(1.0 + t * t);
                        s = t * c;
                        rotated = 1;
                    }
                }
                pp_[k] = p; qq_[k] = q; cc_[k] = c; ss_[k] = s;
            }
            __syncthreads();
            // rows p, q:  row_p <- c row_p - s row_q,  row_q <- s row_p + c row_q
            for (long long t = threadIdx.x; t < (long long)half * n; t += blockDim.x) {
                const int k = (int)(t / n), j = (int)(t % n);
                const int p = pp_[k], q = qq_[k];
                if (q >= n || ss_[k] == 0.0) continue;
                const double c = cc_[k], s = ss_[k];
                const double x = A[(long long)p * n + j], y = A[(long long)q * n + j];
                A[(long long)p * n + j] = c * x - s * y;
                A[(long long)q * n + j] = s * x + c * y;
            }
            __syncthreads();
            // columns p, q of A and of V
            for (long long t = threadIdx.x; t < (long long)half * n; t += blockDim.x) {
                const int k = (int)(t / n), i = (int)(t % n);
                const int p = pp_[k], q = qq_[k];
                if (q >= n || ss_[k] == 0.0) continue;
                const double c = cc_[k], s = ss_[k];
                const double x = A[(long long)i * n + p], y = A[(long long)i * n + q];
                A[(long long)i * n + p] = c * x - s * y;
                A[(long long)i * n + q] = s * x + c * y;
                const double vx = V[o + (long long)i * n + p], vy = V[o + (long long)i * n + q];
                V[o + (long long)i * n + p] = c * vx - s * vy;
                V[o + (long long)i * n + q] = s * vx + c * vy;
            }
            __syncthreads();
        }
        if (!rotated) break;
        __syncthreads();
    }
    // eigenvalues ascending (rank by counting), eigenvectors permuted into Vout
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const double ai = A[(long long)i * n + i];
        int rank = 0;
        for (int j = 0; j < n; ++j) {
            const double aj = A[(long long)j * n + j];
            rank += (aj < ai) || (aj == ai && j < i);
        }
        eps[ebase[m] + rank] = ai;
        for (int r = 0; r < n; ++r) Vout[o + (long long)r * n + rank] = V[o + (long long)r * n + i];
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

struct SCFState {
    mess_basis* b;
    cudaStream_t s;
    int nmol, maxn;
    long long P;
    Dev<double> S, H, X, F, D, J, K, V, C, W1, W2, e, eps, E, emax, smin, Bm, Fh, eh, Wk;
    Dev<double> Vprev, Dprev, Jt, Kt;   // warm-start eigenvectors, previous density, accumulated J / K
    bool warm = false;
    Dev<long long> base, ebase;
    Dev<double> occ;
    Dev<int> n, nocc, sweeps;
    Dev<unsigned char> active;
    int use_smem;
    size_t jac_smem;
    Layout L;
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

cudaError_t jacobi(SCFState& st, const double* A, double* Vout)
{
    // the attribute is per kernel, not per call: a nested SCF (atomic densities) may have lowered it
    if (st.use_smem) {
        cudaError_t e = cudaFuncSetAttribute(k_jacobi, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)st.jac_smem);
        if (e != cudaSuccess) return e;
    }
    k_jacobi<<<st.nmol, 512, st.jac_smem, st.s>>>(A, st.W2.p, Vout, st.eps.p, st.ebase.p, st.L, st.use_smem,
                                                  st.Wk.p, 40, st.sweeps.p);
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
        if ((e = jacobi(st, st.V.p, st.W1.p)) != cudaSuccess) return e;                                   // V_rel -> W1
        if ((e = gemm(st, false, st.Vprev.p, st.W1.p, st.V.p, 0, 1.0)) != cudaSuccess) return e;          // V = Vprev V_rel
    } else {
        if ((e = jacobi(st, st.V.p, st.W1.p)) != cudaSuccess) return e;                      // V -> W1
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
    st.b = b;
    st.s = (cudaStream_t)o.cuda_stream;
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
    std::vector<unsigned char> act(b->nmol, 1);
    MESS_CUDA_TRY(cudaMemcpy(st.active.p, act.data(), b->nmol, cudaMemcpyHostToDevice));
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
    MESS_CUDA_TRY(jacobi(st, st.S.p, st.V.p));                                        // S = U s U^T
    k_scale_cols<<<b->nmol, 256, 0, st.s>>>(st.V.p, st.eps.p, st.ebase.p, st.W1.p, st.L, st.smin.p);
    MESS_CUDA_TRY(cudaGetLastError());
    MESS_CUDA_TRY(gemm(st, true, st.W1.p, st.V.p, st.X.p, 0, 1.0));                 // X = U s^-1/2 U^T
    std::vector<double> hmin(b->nmol);
    MESS_CUDA_TRY(cudaMemcpyAsync(hmin.data(), st.smin.p, sizeof(double) * b->nmol, cudaMemcpyDeviceToHost, st.s));
    MESS_CUDA_TRY(cudaStreamSynchronize(st.s));
    for (int m = 0; m < b->nmol; ++m)
        if (!(hmin[m] > 1e-7)) { mess_set_error("molecule %d: overlap matrix nearly singular (%g)", m, hmin[m]); return MESS_ENUMERIC; }

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

    std::vector<double> Enuc(b->nmol), E(b->nmol), Eold(b->nmol, 0.0), em(b->nmol);
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
    int nstored = 0, slot = 0, remaining = b->nmol;
    mess_status status = MESS_OK;
    // Incremental Fock builds: J(D_k) = J(D_{k-1}) + J(D_k - D_{k-1}) (J, K linear in D).  The
    // reduced-precision error of each build then scales with |D_k - D_{k-1}|, which shrinks as
    // the SCF converges; a full build every `full_every` iterations resets the accumulation.
    const int full_every = 12;
    for (int it = 1; it <= max_iter && remaining > 0; ++it) {
        const bool full = (it - 1) % full_every == 0;
        if (full) {
            mess_status js = mess_jk_packed(b, st.D.p, st.Jt.p, st.Kt.p, &jo, nullptr);
            if (js != MESS_OK) return js;
        } else {
            k_axpbypcz<<<eg, 256, 0, st.s>>>(st.W1.p, 1.0, st.D.p, -1.0, st.Dprev.p, 0.0, nullptr, st.L);   // dD
            MESS_CUDA_TRY(cudaGetLastError());
            mess_status js = mess_jk_packed(b, st.W1.p, st.J.p, st.K.p, &jo, nullptr);
            if (js != MESS_OK) return js;
            k_axpbypcz<<<eg, 256, 0, st.s>>>(st.Jt.p, 1.0, st.Jt.p, 1.0, st.J.p, 0.0, nullptr, st.L);
            k_axpbypcz<<<eg, 256, 0, st.s>>>(st.Kt.p, 1.0, st.Kt.p, 1.0, st.K.p, 0.0, nullptr, st.L);
        }
        MESS_CUDA_TRY(cudaMemcpyAsync(st.Dprev.p, st.D.p, sizeof(double) * P, cudaMemcpyDeviceToDevice, st.s));
        k_axpbypcz<<<eg, 256, 0, st.s>>>(st.F.p, 1.0, st.H.p, 1.0, st.Jt.p, -0.5, st.Kt.p, st.L);   // F = H + J - K/2
        k_energy<<<b->nmol, 256, 0, st.s>>>(st.D.p, st.H.p, st.F.p, st.L, st.E.p);
        MESS_CUDA_TRY(cudaGetLastError());
        MESS_CUDA_TRY(gemm(st, false, st.F.p, st.D.p, st.W1.p, 0, 1.0));   // F D
        MESS_CUDA_TRY(gemm(st, false, st.W1.p, st.S.p, st.W2.p, 0, 1.0));  // F D S
        k_commutator<<<b->nmol, 256, 0, st.s>>>(st.W2.p, st.e.p, st.L, st.emax.p);
        MESS_CUDA_TRY(cudaGetLastError());
        MESS_CUDA_TRY(cudaMemcpyAsync(E.data(), st.E.p, sizeof(double) * b->nmol, cudaMemcpyDeviceToHost, st.s));
        MESS_CUDA_TRY(cudaMemcpyAsync(em.data(), st.emax.p, sizeof(double) * b->nmol, cudaMemcpyDeviceToHost, st.s));
        MESS_CUDA_TRY(cudaStreamSynchronize(st.s));
        bool changed = false;
        for (int m = 0; m < b->nmol; ++m) {
            if (!act[m]) continue;
            if (!std::isfinite(E[m]) || !std::isfinite(em[m])) {
                mess_set_error("molecule %d: non-finite energy or error at iteration %d", m, it);
                return MESS_ENUMERIC;
            }
            iters[m] = it;
            if (it > 1 && fabs(E[m] - Eold[m]) < conv_E && em[m] < conv_comm) {
                conv[m] = 1;
                act[m] = 0;
                changed = true;
                --remaining;
                if (res) {
                    res[m].E_elec = E[m];
                    res[m].E_nuc = Enuc[m];
                    res[m].E_total = E[m] + Enuc[m];
                    res[m].E_iter = res[m].E_total;
                    res[m].iterations = it;
                    res[m].converged = 1;
                }
            }
            Eold[m] = E[m];
        }
        if (remaining == 0) break;
        if (changed) {
            MESS_CUDA_TRY(cudaMemcpyAsync(st.active.p, act.data(), b->nmol, cudaMemcpyHostToDevice, st.s));
            for (int m = 0; m < b->nmol; ++m) b->active[m] = act[m];
            b->active_version++;
        }
        // DIIS extrapolation of F, then the new density
        nstored = std::min(nstored + 1, diis_n);
        k_diis<<<b->nmol, 256, 0, st.s>>>(st.Fh.p, st.eh.p, (long long)P, st.F.p, st.e.p, st.L, slot, nstored, diis_n, st.Bm.p);
        MESS_CUDA_TRY(cudaGetLastError());
        slot = (slot + 1) % diis_n;
        MESS_CUDA_TRY(density_from_fock(st, st.F.p));
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
        // Reported energy of the reduced-precision forms: E at the final density with one Fock build
        // in which every quartet runs in FP64-class arithmetic (double-float if split_df32, else
        // FP64).  The integrals' rounding then no longer enters the energy, and the density's own
        // deviation from the FP64 solution enters it only at second order (E is stationary there).
        for (int m = 0; m < b->nmol; ++m) { act[m] = 1; b->active[m] = 1; }
        b->active_version++;
        MESS_CUDA_TRY(cudaMemcpyAsync(st.active.p, act.data(), b->nmol, cudaMemcpyHostToDevice, st.s));
        mess_jk_opts jf = jo;
        jf.prec = MESS_MIXED;
        jf.fp64_tau = 1e-300;          // every quartet above the split threshold
        mess_status js = mess_jk_packed(b, st.D.p, st.Jt.p, st.Kt.p, &jf, nullptr);
        if (js != MESS_OK) return js;
        k_axpbypcz<<<eg, 256, 0, st.s>>>(st.F.p, 1.0, st.H.p, 1.0, st.Jt.p, -0.5, st.Kt.p, st.L);
        k_energy<<<b->nmol, 256, 0, st.s>>>(st.D.p, st.H.p, st.F.p, st.L, st.E.p);
        MESS_CUDA_TRY(cudaGetLastError());
        MESS_CUDA_TRY(cudaMemcpyAsync(E.data(), st.E.p, sizeof(double) * b->nmol, cudaMemcpyDeviceToHost, st.s));
        MESS_CUDA_TRY(cudaStreamSynchronize(st.s));
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

}  // namespace

mess_status mess_scf_batch_density(mess_basis* b, const mess_scf_opts* opts, mess_scf_result* res, double* dD)
{
    return scf_run(b, opts, res, dD, true);
}

extern "C" mess_status mess_scf(const mess_basis* bc, const mess_scf_opts* opts, mess_scf_result* res, double* D_out)
{
    mess_basis* b = const_cast<mess_basis*>(bc);
    if (!b || !res) { mess_set_error("null argument"); return MESS_EINVAL; }
    return scf_run(b, opts, res, D_out, false);
}

extern "C" mess_status mess_scf_batch(int nmol, mess_basis* const* bases, const mess_scf_opts* opts, mess_scf_result* res)
{
    if (nmol <= 0 || !bases || !res) { mess_set_error("bad batch arguments"); return MESS_EINVAL; }
    mess_basis* batch = nullptr;
    mess_status st = mess_batch_basis(nmol, bases, &batch);
    if (st != MESS_OK) return st;
    st = scf_run(batch, opts, res, nullptr, false);
    mess_free_basis(batch);
    delete batch;
    return st;
}
