// Learned SCF initial guess: a multilayer perceptron that maps atom-pair descriptors to blocks of the
// converged closed-shell density (minimal basis: one s function on H, s s' p_x p_y p_z on C / N / O),
// trained on densities the SCF itself produces.  The network is 112 -> 256 -> 256 -> 25 with SiLU,
// BF16 inputs and weights, FP32 accumulation (tensor-core mma.sync m16n8k16), FP32 master weights
// and Adam (the optimiser the paper uses for its energy minimisations, Sec. 5).
//
// Descriptor of the ordered atom pair (i, j) of one molecule (112 floats):
//   [0, 4)    one-hot element of i (H, C, N, O)      [4, 8)  one-hot element of j
//   [8]       1 if i == j
//   [9, 41)   Gaussian radial basis of r_ij: exp(-2 (r - mu_k)^2), mu_k = 10 k / 31 bohr
//   [41, 73)  environment of i: 1/4 sum_{k != i} of the radial basis of r_ik
//   [73, 105) environment of j
//   [105,112) zero padding
// Target / output: the 5 x 5 density block D_ij in the pair frame (rows: functions of i, columns:
// functions of j, order s, s', x', y', z'), masked to the functions the atoms carry.  For i != j the
// frame has z' along R_j - R_i; for i == j the block is the rotation average (s part kept, s-p
// zero, p-p = trace / 3 times the identity).  The predicted blocks are rotated back, assembled and
// symmetrised into D0; the SCF's first diagonalisation then makes it idempotent.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include <cuda_bf16.h>

#include "mess_internal.h"

namespace {

constexpr int DIN = MESS_MLP_DIN, WID = MESS_MLP_WIDTH, DOUT = MESS_MLP_DOUT, DOUT_PAD = 32;
constexpr int MLP_MAX_SPLIT = 64;    // K slices of the split gradient GEMMs and column sums
constexpr int NRBF = 32;

struct MlpParams {   // offsets into the flat parameter vector
    static constexpr int W1 = 0, B1 = W1 + DIN * WID, W2 = B1 + WID, B2 = W2 + WID * WID, W3 = B2 + WID,
                         B3 = W3 + WID * DOUT_PAD, N = B3 + DOUT_PAD;
};

// ------------------------------------------------------------------------------------ descriptors
struct AtomArgs {
    const double* xyz;     // [natom][3]
    const int* Z;
    const int* amol;       // molecule of atom
    const int* afn;        // first local function of the atom
    const int* anf;        // functions of the atom (1 or 5)
    const int* mat0;       // [nmol] first atom of the molecule
    const int* mnat;       // [nmol] atoms of the molecule
    const long long* mrow; // [nmol] first descriptor row of the molecule
    const long long* mbase;
    const int* mn;
};

__device__ int elem_index(int z) { return z == 1 ? 0 : (z == 6 ? 1 : (z == 7 ? 2 : 3)); }

__device__ void pair_frame(const double* ri, const double* rj, double R[3][3])
{
    double z[3] = {rj[0] - ri[0], rj[1] - ri[1], rj[2] - ri[2]};
    const double r = sqrt(z[0] * z[0] + z[1] * z[1] + z[2] * z[2]);
    for (int k = 0; k < 3; ++k) z[k] /= r;
    // x' = normalise(z' x e) with e the lab axis least aligned with z'
    int a = 0;
    for (int k = 1; k < 3; ++k) if (fabs(z[k]) < fabs(z[a])) a = k;
    double e[3] = {0, 0, 0};
    e[a] = 1.0;
    double x[3] = {z[1] * e[2] - z[2] * e[1], z[2] * e[0] - z[0] * e[2], z[0] * e[1] - z[1] * e[0]};
    const double xn = sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
    for (int k = 0; k < 3; ++k) x[k] /= xn;
    const double y[3] = {z[1] * x[2] - z[2] * x[1], z[2] * x[0] - z[0] * x[2], z[0] * x[1] - z[1] * x[0]};
    for (int k = 0; k < 3; ++k) { R[0][k] = x[k]; R[1][k] = y[k]; R[2][k] = z[k]; }
}

// T5 = diag(1, 1, R) acting on the 5 functions (s, s', p_x, p_y, p_z) of a heavy atom; [1] for H
__device__ double tmat(int nf, const double R[3][3], int a, int b)
{
    if (nf == 1) return (a == 0 && b == 0) ? 1.0 : 0.0;
    if (a < 2 || b < 2) return a == b ? 1.0 : 0.0;
    return R[a - 2][b - 2];
}

// one row per ordered atom pair: descriptor (float), and with D the pair-frame target + mask
__global__ void k_features(AtomArgs A, int nmol, float* __restrict__ X, float* __restrict__ T, float* __restrict__ M,
                           const double* __restrict__ D)
{
    const int m = blockIdx.y;
    const int na = A.mnat[m], a0 = A.mat0[m];
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= na * na) return;
    const int i = a0 + t / na, j = a0 + t % na;
    const long long row = A.mrow[m] + t;
    float* x = X + row * DIN;
    for (int k = 0; k < DIN; ++k) x[k] = 0.f;
    x[elem_index(A.Z[i])] = 1.f;
    x[4 + elem_index(A.Z[j])] = 1.f;
    x[8] = (i == j) ? 1.f : 0.f;
    const double* ri = A.xyz + 3 * i;
    const double* rj = A.xyz + 3 * j;
    const double dx = rj[0] - ri[0], dy = rj[1] - ri[1], dz = rj[2] - ri[2];
    const double r = sqrt(dx * dx + dy * dy + dz * dz);
    for (int k = 0; k < NRBF; ++k) {
        const double mu = 10.0 * k / (NRBF - 1);
        x[9 + k] = (float)exp(-2.0 * (r - mu) * (r - mu));
    }
    for (int c = a0; c < a0 + na; ++c) {
        const double* rc = A.xyz + 3 * c;
        if (c != i) {
            const double ex = rc[0] - ri[0], ey = rc[1] - ri[1], ez = rc[2] - ri[2];
            const double rr = sqrt(ex * ex + ey * ey + ez * ez);
            for (int k = 0; k < NRBF; ++k) {
                const double mu = 10.0 * k / (NRBF - 1);
                x[41 + k] += (float)(0.25 * exp(-2.0 * (rr - mu) * (rr - mu)));
            }
        }
        if (c != j) {
            const double ex = rc[0] - rj[0], ey = rc[1] - rj[1], ez = rc[2] - rj[2];
            const double rr = sqrt(ex * ex + ey * ey + ez * ez);
            for (int k = 0; k < NRBF; ++k) {
                const double mu = 10.0 * k / (NRBF - 1);
                x[73 + k] += (float)(0.25 * exp(-2.0 * (rr - mu) * (rr - mu)));
            }
        }
    }
    if (!T) return;
    const int ni = A.anf[i], nj = A.anf[j];
    const int fi = A.afn[i], fj = A.afn[j];
    const int n = A.mn[m];
    const double* Dm = D + A.mbase[m];
    float* tt = T + row * DOUT;
    float* mm = M + row * DOUT;
    for (int k = 0; k < DOUT; ++k) { tt[k] = 0.f; mm[k] = 0.f; }
    if (i == j) {
        // rotation average of the atomic block
        double ptr = 0.0;
        if (ni == 5) for (int k = 2; k < 5; ++k) ptr += Dm[(size_t)(fi + k) * n + fi + k];
        for (int a = 0; a < ni; ++a)
            for (int b = 0; b < ni; ++b) {
                double v;
                if (a < 2 && b < 2) v = Dm[(size_t)(fi + a) * n + fi + b];
                else if (a >= 2 && b >= 2) v = (a == b) ? ptr / 3.0 : 0.0;
                else v = 0.0;
                tt[a * 5 + b] = (float)v;
                mm[a * 5 + b] = 1.f;
            }
        return;
    }
    double R[3][3];
    pair_frame(ri, rj, R);
    // D_pair = T_i D_lab T_j^T
    for (int a = 0; a < ni; ++a)
        for (int b = 0; b < nj; ++b) {
            double v = 0.0;
            for (int p = 0; p < ni; ++p) {
                const double tap = tmat(ni, R, a, p);
                if (tap == 0.0) continue;
                for (int q = 0; q < nj; ++q) {
                    const double tbq = tmat(nj, R, b, q);
                    if (tbq == 0.0) continue;
                    v += tap * Dm[(size_t)(fi + p) * n + fj + q] * tbq;
                }
            }
            tt[a * 5 + b] = (float)v;
            mm[a * 5 + b] = 1.f;
        }
}

// predicted pair-frame blocks -> lab-frame D0 blocks (D0 = T_i^T Y T_j), then symmetrised elsewhere
__global__ void k_assemble_guess(AtomArgs A, const float* __restrict__ Y, double* __restrict__ D0)
{
    const int m = blockIdx.y;
    const int na = A.mnat[m], a0 = A.mat0[m];
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= na * na) return;
    const int i = a0 + t / na, j = a0 + t % na;
    const float* y = Y + (A.mrow[m] + t) * DOUT_PAD;
    const int ni = A.anf[i], nj = A.anf[j], fi = A.afn[i], fj = A.afn[j], n = A.mn[m];
    double* Dm = D0 + A.mbase[m];
    if (i == j) {
        for (int a = 0; a < ni; ++a)
            for (int b = 0; b < ni; ++b) {
                double v = 0.0;
                if (a < 2 && b < 2) v = y[a * 5 + b];
                else if (a >= 2 && b >= 2 && a == b) v = (y[10 + 2] + y[15 + 3] + y[20 + 4]) / 3.0;
                Dm[(size_t)(fi + a) * n + fi + b] = v;
            }
        return;
    }
    double R[3][3];
    pair_frame(A.xyz + 3 * i, A.xyz + 3 * j, R);
    for (int p = 0; p < ni; ++p)
        for (int q = 0; q < nj; ++q) {
            double v = 0.0;
            for (int a = 0; a < ni; ++a) {
                const double tap = tmat(ni, R, a, p);
                if (tap == 0.0) continue;
                for (int b = 0; b < nj; ++b) {
                    const double tbq = tmat(nj, R, b, q);
                    if (tbq != 0.0) v += tap * (double)y[a * 5 + b] * tbq;
                }
            }
            Dm[(size_t)(fi + p) * n + fj + q] = v;
        }
}

__global__ void k_symmetrise(double* __restrict__ D, const long long* __restrict__ mbase, const int* __restrict__ mn)
{
    const int m = blockIdx.y;
    const int n = mn[m];
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n * n) return;
    const int i = t / n, j = t % n;
    if (j >= i) return;
    double* Dm = D + mbase[m];
    const double v = 0.5 * (Dm[(size_t)i * n + j] + Dm[(size_t)j * n + i]);
    Dm[(size_t)i * n + j] = v;
    Dm[(size_t)j * n + i] = v;
}

// ------------------------------------------------------------------------------------ BF16 GEMM
// C[m][n] (op)= sum_k A(m, k) B(k, n), A(m, k) = A[m * sam + k * sak], B(k, n) = B[k * sbk + n * sbn]
// (BF16), FP32 accumulation on tensor cores (mma.sync m16n8k16).  64 x 64 block tile, 4 warps of
// 32 x 32, K step 16.  gridDim.z splits K: slice z then stores its partial sums to part + z * pstride
// (same layout as C), and k_sum_parts adds the slices in order z = 0, 1, ... (no atomics: training is
// reproducible run to run).  Epilogue: + bias[n]; store FP32 to C (ldc) and optionally SiLU(C) as
// BF16 to Abf (ldc).
struct GemmArgs {
    const __nv_bfloat16* A;
    long long sam, sak;
    const __nv_bfloat16* B;
    long long sbk, sbn;
    float* C;
    long long ldc;
    const float* bias;
    __nv_bfloat16* act;     // SiLU(C + bias) as BF16 (nullable)
    int M, N, K;
    float* part;            // split K: per-slice partial sums (no epilogue); null: one slice
    long long pstride;      // elements between slices of part
};

__device__ __forceinline__ unsigned pack2(__nv_bfloat16 lo, __nv_bfloat16 hi)
{
    return (unsigned)__bfloat16_as_ushort(lo) | ((unsigned)__bfloat16_as_ushort(hi) << 16);
}

__global__ void __launch_bounds__(128) k_gemm_bf16(GemmArgs g)
{
    __shared__ __nv_bfloat16 As[64][16 + 8];
    __shared__ __nv_bfloat16 Bs[16][64 + 8];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
    const int m0 = blockIdx.y * 64, n0 = blockIdx.x * 64;
    const int kchunk = (g.K + gridDim.z - 1) / gridDim.z;
    const int kbeg = blockIdx.z * kchunk, kend = min(g.K, kbeg + kchunk);
    float acc[2][4][4];
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[a][b][c] = 0.f;
    const __nv_bfloat16 zero = __float2bfloat16(0.f);
    for (int k0 = kbeg; k0 < kend; k0 += 16) {
        for (int t = threadIdx.x; t < 64 * 16; t += 128) {
            const int r = t / 16, c = t % 16;
            const int gm = m0 + r, gk = k0 + c;
            As[r][c] = (gm < g.M && gk < kend) ? g.A[(long long)gm * g.sam + (long long)gk * g.sak] : zero;
        }
        for (int t = threadIdx.x; t < 16 * 64; t += 128) {
            const int r = t / 64, c = t % 64;
            const int gk = k0 + r, gn = n0 + c;
            Bs[r][c] = (gk < kend && gn < g.N) ? g.B[(long long)gk * g.sbk + (long long)gn * g.sbn] : zero;
        }
        __syncthreads();
        const int gid = lane >> 2, tig = lane & 3;
#pragma unroll
        for (int a = 0; a < 2; ++a) {
            const int rb = wm + 16 * a;
            unsigned af[4];
            af[0] = pack2(As[rb + gid][tig * 2], As[rb + gid][tig * 2 + 1]);
            af[1] = pack2(As[rb + gid + 8][tig * 2], As[rb + gid + 8][tig * 2 + 1]);
            af[2] = pack2(As[rb + gid][tig * 2 + 8], As[rb + gid][tig * 2 + 9]);
            af[3] = pack2(As[rb + gid + 8][tig * 2 + 8], As[rb + gid + 8][tig * 2 + 9]);
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                const int cb = wn + 8 * b;
                unsigned bf[2];
                bf[0] = pack2(Bs[tig * 2][cb + gid], Bs[tig * 2 + 1][cb + gid]);
                bf[1] = pack2(Bs[tig * 2 + 8][cb + gid], Bs[tig * 2 + 9][cb + gid]);
                float* c = acc[a][b];
                asm volatile(
                    "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                    "{%0,%1,%2,%3};\n"
                    : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
                    : "r"(af[0]), "r"(af[1]), "r"(af[2]), "r"(af[3]), "r"(bf[0]), "r"(bf[1]));
            }
        }
        __syncthreads();
    }
    const int gid = lane >> 2, tig = lane & 3;
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b)
#pragma unroll
            for (int h = 0; h < 4; ++h) {
                const int r = m0 + wm + 16 * a + gid + (h >= 2 ? 8 : 0);
                const int c = n0 + wn + 8 * b + tig * 2 + (h & 1);
                if (r >= g.M || c >= g.N) continue;
                float v = acc[a][b][h];
                if (g.part) { g.part[blockIdx.z * g.pstride + (long long)r * g.ldc + c] = v; continue; }
                float* dst = g.C + (long long)r * g.ldc + c;
                if (g.bias) v += g.bias[c];
                *dst = v;
                if (g.act) g.act[(long long)r * g.ldc + c] = __float2bfloat16(v / (1.f + __expf(-v)));
            }
}

// ------------------------------------------------------------------------------------ elementwise
__global__ void k_to_bf16(const float* __restrict__ x, __nv_bfloat16* __restrict__ y, long long n)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        y[i] = __float2bfloat16(x[i]);
}

// masked mean squared error over the DOUT outputs; dY (BF16, DOUT_PAD columns) = d loss / d Y
__global__ void k_loss(const float* __restrict__ Y, const float* __restrict__ T, const float* __restrict__ M,
                       long long rows, double inv_count, double* __restrict__ loss, __nv_bfloat16* __restrict__ dY)
{
    double s = 0.0;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < rows * DOUT_PAD;
         t += (long long)gridDim.x * blockDim.x) {
        const long long r = t / DOUT_PAD;
        const int c = (int)(t % DOUT_PAD);
        float g = 0.f;
        if (c < DOUT) {
            const float mk = M[r * DOUT + c];
            const float d = Y[r * DOUT_PAD + c] - T[r * DOUT + c];
            s += (double)(mk * d * d);
            g = (float)(2.0 * inv_count) * mk * d;
        }
        dY[t] = __float2bfloat16(g);
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(loss, s * inv_count);
}

// dZ = dA * silu'(Z) as BF16, silu'(z) = s(z) (1 + z (1 - s(z))), s the logistic function
__global__ void k_silu_back(const float* __restrict__ dA, const float* __restrict__ Z, __nv_bfloat16* __restrict__ dZ,
                            long long n)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float z = Z[i];
        const float sg = 1.f / (1.f + __expf(-z));
        dZ[i] = __float2bfloat16(dA[i] * sg * (1.f + z * (1.f - sg)));
    }
}

// out[i] = sum over slices z = 0 .. nz-1 (in that order) of part[z * pstride + i], for the M x N
// entries i = r * ld + c
__global__ void k_sum_parts(const float* __restrict__ part, int nz, long long pstride, int M, int N, long long ld,
                            float* __restrict__ out)
{
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < (long long)M * N;
         t += (long long)gridDim.x * blockDim.x) {
        const long long i = (t / N) * ld + t % N;
        float s = 0.f;
        for (int z = 0; z < nz; ++z) s += part[z * pstride + i];
        out[i] = s;
    }
}

// column sums of a BF16 rows x cols matrix: block (x, y) sums the rows y, y + gridDim.y, ... of its 32
// columns (its warps' shares added in warp order) into part[y * cols + c]; k_sum_parts then adds the
// gridDim.y slices in order (no atomics)
__global__ void k_colsum(const __nv_bfloat16* __restrict__ X, long long rows, int cols, float* __restrict__ part)
{
    __shared__ float ws[32][33];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int c = blockIdx.x * 32 + lane;
    float s = 0.f;
    if (c < cols)
        for (long long r = (long long)blockIdx.y * nw + w; r < rows; r += (long long)gridDim.y * nw)
            s += __bfloat162float(X[r * cols + c]);
    ws[w][lane] = s;
    __syncthreads();
    if (w == 0 && c < cols) {
        float t = 0.f;
        for (int k = 0; k < nw; ++k) t += ws[k][lane];
        part[(long long)blockIdx.y * cols + c] = t;
    }
}

__global__ void k_adam(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m1, float* __restrict__ m2,
                       int n, float lr, float b1, float b2, float eps, float c1, float c2)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    m1[i] = b1 * m1[i] + (1.f - b1) * gi;
    m2[i] = b2 * m2[i] + (1.f - b2) * gi * gi;
    w[i] -= lr * (m1[i] / c1) / (sqrtf(m2[i] / c2) + eps);
}

__global__ void k_gather_rows(const float* __restrict__ src, const long long* __restrict__ idx, long long n, int cols,
                              float* __restrict__ dst)
{
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n * cols; t += (long long)gridDim.x * blockDim.x)
        dst[t] = src[idx[t / cols] * cols + t % cols];
}

}  // namespace

// ------------------------------------------------------------------------------------ host side
struct mess_mlp {
    DevBuf<float> w, g, m1, m2;                 // master weights, gradient, Adam moments
    DevBuf<__nv_bfloat16> wb;                   // BF16 copy for the forward / backward GEMMs
    long long step = 0;
    // activations of the current batch
    long long cap = 0;
    DevBuf<__nv_bfloat16> xb, a1, a2, dyb, dz2, dz1;
    DevBuf<float> z1, z2, y, da2, da1;
    DevBuf<double> loss;
    DevBuf<float> part;                         // per-slice partial sums of the gradient reductions
};

namespace {

cudaError_t ensure_cap(mess_mlp* m, long long rows)
{
    if (rows <= m->cap) return cudaSuccess;
    cudaError_t e;
    if ((e = m->xb.alloc(rows * DIN)) != cudaSuccess) return e;
    if ((e = m->a1.alloc(rows * WID)) != cudaSuccess) return e;
    if ((e = m->a2.alloc(rows * WID)) != cudaSuccess) return e;
    if ((e = m->dyb.alloc(rows * DOUT_PAD)) != cudaSuccess) return e;
    if ((e = m->dz2.alloc(rows * WID)) != cudaSuccess) return e;
    if ((e = m->dz1.alloc(rows * WID)) != cudaSuccess) return e;
    if ((e = m->z1.alloc(rows * WID)) != cudaSuccess) return e;
    if ((e = m->z2.alloc(rows * WID)) != cudaSuccess) return e;
    if ((e = m->y.alloc(rows * DOUT_PAD)) != cudaSuccess) return e;
    if ((e = m->da2.alloc(rows * WID)) != cudaSuccess) return e;
    if ((e = m->da1.alloc(rows * WID)) != cudaSuccess) return e;
    if (!m->part.p) {
        const long long most = std::max<long long>({(long long)WID * WID, (long long)DIN * WID, (long long)WID * DOUT_PAD});
        if ((e = m->part.alloc(MLP_MAX_SPLIT * most)) != cudaSuccess) return e;
    }
    m->cap = rows;
    return cudaSuccess;
}

unsigned grid1(long long n) { return (unsigned)std::min<long long>((n + 255) / 256, 65535LL * 8); }

cudaError_t gemm(const __nv_bfloat16* A, long long sam, long long sak, const __nv_bfloat16* B, long long sbk,
                 long long sbn, float* C, long long ldc, int M, int N, int K, const float* bias,
                 __nv_bfloat16* act, int splitk, cudaStream_t s, float* part = nullptr)
{
    // split K only into a workspace of MLP_MAX_SPLIT slices of M x ldc (no epilogue then)
    if (splitk > 1 && (!part || splitk > MLP_MAX_SPLIT || bias || act)) return cudaErrorInvalidValue;
    const long long pstride = (long long)M * ldc;
    GemmArgs g{A, sam, sak, B, sbk, sbn, C, ldc, bias, act, M, N, K, splitk > 1 ? part : nullptr, pstride};
    dim3 grid((N + 63) / 64, (M + 63) / 64, splitk);
    k_gemm_bf16<<<grid, 128, 0, s>>>(g);
    if (splitk > 1) k_sum_parts<<<grid1((long long)M * N), 256, 0, s>>>(part, splitk, pstride, M, N, ldc, C);
    return cudaGetLastError();
}


// forward of `rows` rows whose FP32 descriptors are in X (device); output Y (rows x 32, FP32)
cudaError_t forward(mess_mlp* m, const float* X, long long rows, cudaStream_t s)
{
    cudaError_t e;
    if ((e = ensure_cap(m, rows)) != cudaSuccess) return e;
    const __nv_bfloat16* wb = m->wb.p;
    k_to_bf16<<<grid1(rows * DIN), 256, 0, s>>>(X, m->xb.p, rows * DIN);
    const float* w = m->w.p;
    if ((e = gemm(m->xb.p, DIN, 1, wb + MlpParams::W1, WID, 1, m->z1.p, WID, (int)rows, WID, DIN,
                  w + MlpParams::B1, m->a1.p, 1, s)) != cudaSuccess) return e;
    if ((e = gemm(m->a1.p, WID, 1, wb + MlpParams::W2, WID, 1, m->z2.p, WID, (int)rows, WID, WID,
                  w + MlpParams::B2, m->a2.p, 1, s)) != cudaSuccess) return e;
    return gemm(m->a2.p, WID, 1, wb + MlpParams::W3, DOUT_PAD, 1, m->y.p, DOUT_PAD, (int)rows, DOUT_PAD, WID,
                w + MlpParams::B3, nullptr, 1, s);
}

// loss and gradient (into m->g) of the rows forward() just processed
cudaError_t backward(mess_mlp* m, const float* T, const float* M, long long rows, double count, cudaStream_t s)
{
    cudaError_t e;
    if ((e = cudaMemsetAsync(m->g.p, 0, sizeof(float) * MlpParams::N, s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(m->loss.p, 0, sizeof(double), s)) != cudaSuccess) return e;
    k_loss<<<grid1(rows * DOUT_PAD), 256, 0, s>>>(m->y.p, T, M, rows, 1.0 / std::max(1.0, count), m->loss.p, m->dyb.p);
    const __nv_bfloat16* wb = m->wb.p;
    float* g = m->g.p;
    const int split = (int)std::min<long long>(MLP_MAX_SPLIT, std::max<long long>(1, rows / 4096));
    float* part = m->part.p;
    auto colsum = [&](const __nv_bfloat16* X, int cols, float* out) {
        k_colsum<<<dim3((cols + 31) / 32, MLP_MAX_SPLIT), 256, 0, s>>>(X, rows, cols, part);
        k_sum_parts<<<grid1(cols), 256, 0, s>>>(part, MLP_MAX_SPLIT, cols, 1, cols, cols, out);
    };
    // layer 3: dW3 = A2^T dY, db3 = sum dY, dA2 = dY W3^T
    if ((e = gemm(m->a2.p, 1, WID, m->dyb.p, DOUT_PAD, 1, g + MlpParams::W3, DOUT_PAD, WID, DOUT_PAD, (int)rows,
                  nullptr, nullptr, split, s, part)) != cudaSuccess) return e;
    colsum(m->dyb.p, DOUT_PAD, g + MlpParams::B3);
    if ((e = gemm(m->dyb.p, DOUT_PAD, 1, wb + MlpParams::W3, 1, DOUT_PAD, m->da2.p, WID, (int)rows, WID, DOUT_PAD,
                  nullptr, nullptr, 1, s)) != cudaSuccess) return e;
    k_silu_back<<<grid1(rows * WID), 256, 0, s>>>(m->da2.p, m->z2.p, m->dz2.p, rows * WID);
    // layer 2
    if ((e = gemm(m->a1.p, 1, WID, m->dz2.p, WID, 1, g + MlpParams::W2, WID, WID, WID, (int)rows,
                  nullptr, nullptr, split, s, part)) != cudaSuccess) return e;
    colsum(m->dz2.p, WID, g + MlpParams::B2);
    if ((e = gemm(m->dz2.p, WID, 1, wb + MlpParams::W2, 1, WID, m->da1.p, WID, (int)rows, WID, WID,
                  nullptr, nullptr, 1, s)) != cudaSuccess) return e;
    k_silu_back<<<grid1(rows * WID), 256, 0, s>>>(m->da1.p, m->z1.p, m->dz1.p, rows * WID);
    // layer 1
    if ((e = gemm(m->xb.p, 1, DIN, m->dz1.p, WID, 1, g + MlpParams::W1, WID, DIN, WID, (int)rows,
                  nullptr, nullptr, split, s, part)) != cudaSuccess) return e;
    colsum(m->dz1.p, WID, g + MlpParams::B1);
    return cudaGetLastError();
}

cudaError_t refresh_bf16(mess_mlp* m, cudaStream_t s)
{
    k_to_bf16<<<grid1(MlpParams::N), 256, 0, s>>>(m->w.p, m->wb.p, MlpParams::N);
    return cudaGetLastError();
}

// atom tables of a (batch) basis for the descriptor / assembly kernels; rows = sum natom_m^2
struct AtomTables {
    DevBuf<int> amol, afn, anf, mat0, mnat;
    DevBuf<long long> mrow;
    long long rows = 0;
    AtomArgs args(const mess_basis* b) const
    {
        return AtomArgs{b->d_xyz.p, b->d_Z.p, amol.p, afn.p, anf.p, mat0.p, mnat.p, mrow.p, b->d_mol_base.p, b->d_mol_n.p};
    }
};

mess_status atom_tables(const mess_basis* b, AtomTables& t)
{
    std::vector<int> amol(b->natom), afn(b->natom, -1), anf(b->natom, 0);
    for (const HostShell& sh : b->shells) {
        if (afn[sh.atom] < 0) afn[sh.atom] = sh.fl;
        anf[sh.atom] += (sh.l + 1) * (sh.l + 2) / 2;
        amol[sh.atom] = sh.mol;
        if (sh.l > 1) { mess_set_error("learned guess: minimal s/p basis only (found l = %d)", sh.l); return MESS_EINVAL; }
    }
    for (int a = 0; a < b->natom; ++a) {
        const int z = b->Z[a];
        const bool ok = (z == 1 && anf[a] == 1) || ((z == 6 || z == 7 || z == 8) && anf[a] == 5);
        if (!ok) {
            mess_set_error("learned guess: atom %d (Z = %d) carries %d functions; it needs a minimal basis "
                           "(1 on H, 5 on C / N / O)", a, z, anf[a]);
            return MESS_EINVAL;
        }
    }
    std::vector<long long> mrow(b->nmol);
    long long r = 0;
    for (int m = 0; m < b->nmol; ++m) {
        mrow[m] = r;
        r += (long long)b->mol_atom_n[m] * b->mol_atom_n[m];
    }
    t.rows = r;
    if (t.amol.upload(amol) != cudaSuccess || t.afn.upload(afn) != cudaSuccess || t.anf.upload(anf) != cudaSuccess ||
        t.mat0.upload(b->mol_atom_off) != cudaSuccess || t.mnat.upload(b->mol_atom_n) != cudaSuccess ||
        t.mrow.upload(mrow) != cudaSuccess) {
        mess_set_error("learned guess: upload failed");
        return MESS_ECUDA;
    }
    return MESS_OK;
}

int max_atoms(const mess_basis* b)
{
    int mx = 0;
    for (int v : b->mol_atom_n) mx = std::max(mx, v);
    return mx;
}

mess_status init_params(mess_mlp* m, unsigned long long seed)
{
    // uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) weights from a splitmix64 stream, zero biases
    std::vector<float> h(MlpParams::N, 0.f);
    unsigned long long x = seed ? seed : 0x9E3779B97F4A7C15ull;
    auto next = [&]() {
        x += 0x9E3779B97F4A7C15ull;
        unsigned long long z = x;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return (double)((z ^ (z >> 31)) >> 11) * (1.0 / 9007199254740992.0);
    };
    auto fill = [&](int off, int fan_in, int rows, int cols, int valid_cols) {
        const double a = 1.0 / sqrt((double)fan_in);
        for (int r = 0; r < rows; ++r)
            for (int c = 0; c < cols; ++c) h[off + r * cols + c] = c < valid_cols ? (float)((2.0 * next() - 1.0) * a) : 0.f;
    };
    fill(MlpParams::W1, DIN, DIN, WID, WID);
    fill(MlpParams::W2, WID, WID, WID, WID);
    fill(MlpParams::W3, WID, WID, DOUT_PAD, DOUT);
    if (m->w.upload(h) != cudaSuccess || m->g.alloc(MlpParams::N) != cudaSuccess || m->m1.alloc(MlpParams::N) != cudaSuccess ||
        m->m2.alloc(MlpParams::N) != cudaSuccess || m->wb.alloc(MlpParams::N) != cudaSuccess ||
        m->loss.alloc(1) != cudaSuccess) {
        mess_set_error("mlp: allocation failed");
        return MESS_ENOMEM;
    }
    cudaMemset(m->m1.p, 0, sizeof(float) * MlpParams::N);
    cudaMemset(m->m2.p, 0, sizeof(float) * MlpParams::N);
    if (refresh_bf16(m, 0) != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) {
        mess_set_error("mlp: initialisation failed");
        return MESS_ECUDA;
    }
    return MESS_OK;
}

void free_mlp(mess_mlp* m)
{
    for (DevBuf<float>* d : {&m->w, &m->g, &m->m1, &m->m2, &m->z1, &m->z2, &m->y, &m->da2, &m->da1}) d->free();
    for (DevBuf<__nv_bfloat16>* d : {&m->wb, &m->xb, &m->a1, &m->a2, &m->dyb, &m->dz2, &m->dz1}) d->free();
    m->loss.free();
}

// the rows' descriptors of a basis into X (device, rows x DIN); with D (device, packed) also targets
mess_status features(const mess_basis* b, const AtomTables& t, const double* dD, float* X, float* T, float* M, cudaStream_t s)
{
    const int mx = max_atoms(b);
    dim3 grid((mx * mx + 127) / 128, b->nmol);
    k_features<<<grid, 128, 0, s>>>(t.args(b), b->nmol, X, T, M, dD);
    MESS_CUDA_TRY(cudaGetLastError());
    return MESS_OK;
}

}  // namespace

// predicted D0 (device, packed layout of b) from the network
mess_status mess_mlp_guess_device(const mess_mlp* mc, const mess_basis* b, double* dD0, cudaStream_t s)
{
    mess_mlp* m = const_cast<mess_mlp*>(mc);
    AtomTables t;
    mess_status st = atom_tables(b, t);
    if (st != MESS_OK) return st;
    DevBuf<float> X;
    MESS_CUDA_TRY(X.alloc(t.rows * DIN));
    st = features(b, t, nullptr, X.p, nullptr, nullptr, s);
    if (st != MESS_OK) return st;
    MESS_CUDA_TRY(forward(m, X.p, t.rows, s));
    MESS_CUDA_TRY(cudaMemsetAsync(dD0, 0, sizeof(double) * b->packed, s));
    const int mx = max_atoms(b);
    k_assemble_guess<<<dim3((mx * mx + 127) / 128, b->nmol), 128, 0, s>>>(t.args(b), m->y.p, dD0);
    MESS_CUDA_TRY(cudaGetLastError());
    k_symmetrise<<<dim3((b->max_nbf * b->max_nbf + 255) / 256, b->nmol), 256, 0, s>>>(dD0, b->d_mol_base.p, b->d_mol_n.p);
    MESS_CUDA_TRY(cudaGetLastError());
    MESS_CUDA_TRY(cudaStreamSynchronize(s));
    return MESS_OK;
}

extern "C" int mess_mlp_num_params(void) { return MlpParams::N; }

extern "C" mess_status mess_mlp_create(unsigned long long seed, mess_mlp** out)
{
    if (!out) { mess_set_error("out is NULL"); return MESS_EINVAL; }
    mess_mlp* m = new (std::nothrow) mess_mlp();
    if (!m) { mess_set_error("host allocation failed"); return MESS_ENOMEM; }
    mess_status st = init_params(m, seed);
    if (st != MESS_OK) { free_mlp(m); delete m; return st; }
    *out = m;
    return MESS_OK;
}

extern "C" void mess_mlp_destroy(mess_mlp* m)
{
    if (!m) return;
    free_mlp(m);
    delete m;
}

extern "C" mess_status mess_mlp_get_params(const mess_mlp* m, float* host)
{
    if (!m || !host) { mess_set_error("null argument"); return MESS_EINVAL; }
    MESS_CUDA_TRY(cudaMemcpy(host, m->w.p, sizeof(float) * MlpParams::N, cudaMemcpyDeviceToHost));
    return MESS_OK;
}

extern "C" mess_status mess_mlp_set_params(mess_mlp* m, const float* host)
{
    if (!m || !host) { mess_set_error("null argument"); return MESS_EINVAL; }
    MESS_CUDA_TRY(cudaMemcpy(m->w.p, host, sizeof(float) * MlpParams::N, cudaMemcpyHostToDevice));
    MESS_CUDA_TRY(refresh_bf16(m, 0));
    MESS_CUDA_TRY(cudaDeviceSynchronize());
    return MESS_OK;
}

extern "C" mess_status mess_mlp_save(const mess_mlp* m, const char* path)
{
    if (!m || !path) { mess_set_error("null argument"); return MESS_EINVAL; }
    std::vector<float> h(MlpParams::N);
    MESS_CUDA_TRY(cudaMemcpy(h.data(), m->w.p, sizeof(float) * h.size(), cudaMemcpyDeviceToHost));
    FILE* f = fopen(path, "wb");
    if (!f) { mess_set_error("cannot write %s", path); return MESS_EINVAL; }
    const char magic[8] = {'M', 'E', 'S', 'S', 'M', 'L', 'P', '1'};
    const int dims[4] = {DIN, WID, DOUT, MlpParams::N};
    bool ok = fwrite(magic, 1, 8, f) == 8 && fwrite(dims, sizeof(int), 4, f) == 4 &&
              fwrite(h.data(), sizeof(float), h.size(), f) == h.size();
    ok = (fclose(f) == 0) && ok;
    if (!ok) { mess_set_error("writing %s failed", path); return MESS_EINVAL; }
    return MESS_OK;
}

extern "C" mess_status mess_mlp_load(const char* path, mess_mlp** out)
{
    if (!path || !out) { mess_set_error("null argument"); return MESS_EINVAL; }
    FILE* f = fopen(path, "rb");
    if (!f) { mess_set_error("cannot open weight file %s", path); return MESS_EINVAL; }
    char magic[8];
    int dims[4];
    std::vector<float> h(MlpParams::N);
    bool ok = fread(magic, 1, 8, f) == 8 && memcmp(magic, "MESSMLP1", 8) == 0 && fread(dims, sizeof(int), 4, f) == 4 &&
              dims[0] == DIN && dims[1] == WID && dims[2] == DOUT && dims[3] == MlpParams::N &&
              fread(h.data(), sizeof(float), h.size(), f) == h.size();
    fclose(f);
    if (!ok) { mess_set_error("%s is not a weight file of this network", path); return MESS_EINVAL; }
    mess_mlp* m = nullptr;
    mess_status st = mess_mlp_create(1, &m);
    if (st != MESS_OK) return st;
    st = mess_mlp_set_params(m, h.data());
    if (st != MESS_OK) { mess_mlp_destroy(m); return st; }
    *out = m;
    return MESS_OK;
}

extern "C" mess_status mess_mlp_features(const mess_basis* b, const double* D, float* X, float* T, float* M, long long* nrows)
{
    if (!b || !nrows) { mess_set_error("null argument"); return MESS_EINVAL; }
    if (b->nmol != 1) { mess_set_error("single-molecule bases only"); return MESS_EINVAL; }
    { const mess_status gs = mess_basis_gpu(const_cast<mess_basis*>(b)); if (gs != MESS_OK) return gs; }
    AtomTables t;
    mess_status st = atom_tables(b, t);
    if (st != MESS_OK) return st;
    *nrows = t.rows;
    if (!X) return MESS_OK;
    if (D && (!T || !M)) { mess_set_error("targets need T and M"); return MESS_EINVAL; }
    DevBuf<float> dX, dT, dM;
    DevBuf<double> dD;
    MESS_CUDA_TRY(dX.alloc(t.rows * DIN));
    if (D) {
        MESS_CUDA_TRY(dT.alloc(t.rows * DOUT));
        MESS_CUDA_TRY(dM.alloc(t.rows * DOUT));
        MESS_CUDA_TRY(dD.alloc(b->packed));
        MESS_CUDA_TRY(cudaMemcpy(dD.p, D, sizeof(double) * b->packed, cudaMemcpyHostToDevice));
    }
    st = features(b, t, D ? dD.p : nullptr, dX.p, D ? dT.p : nullptr, D ? dM.p : nullptr, 0);
    if (st != MESS_OK) return st;
    MESS_CUDA_TRY(cudaDeviceSynchronize());
    MESS_CUDA_TRY(cudaMemcpy(X, dX.p, sizeof(float) * t.rows * DIN, cudaMemcpyDeviceToHost));
    if (D) {
        MESS_CUDA_TRY(cudaMemcpy(T, dT.p, sizeof(float) * t.rows * DOUT, cudaMemcpyDeviceToHost));
        MESS_CUDA_TRY(cudaMemcpy(M, dM.p, sizeof(float) * t.rows * DOUT, cudaMemcpyDeviceToHost));
    }
    return MESS_OK;
}

extern "C" mess_status mess_mlp_loss_grad(mess_mlp* m, long long nrows, const float* X, const float* T, const float* M,
                                          double* loss, float* grad)
{
    if (!m || !X || !T || !M || nrows <= 0) { mess_set_error("bad arguments"); return MESS_EINVAL; }
    DevBuf<float> dX, dT, dM;
    MESS_CUDA_TRY(dX.alloc(nrows * DIN));
    MESS_CUDA_TRY(dT.alloc(nrows * DOUT));
    MESS_CUDA_TRY(dM.alloc(nrows * DOUT));
    MESS_CUDA_TRY(cudaMemcpy(dX.p, X, sizeof(float) * nrows * DIN, cudaMemcpyHostToDevice));
    MESS_CUDA_TRY(cudaMemcpy(dT.p, T, sizeof(float) * nrows * DOUT, cudaMemcpyHostToDevice));
    MESS_CUDA_TRY(cudaMemcpy(dM.p, M, sizeof(float) * nrows * DOUT, cudaMemcpyHostToDevice));
    double count = 0.0;
    for (long long i = 0; i < nrows * DOUT; ++i) count += M[i];
    MESS_CUDA_TRY(forward(m, dX.p, nrows, 0));
    MESS_CUDA_TRY(backward(m, dT.p, dM.p, nrows, count, 0));
    MESS_CUDA_TRY(cudaDeviceSynchronize());
    if (loss) MESS_CUDA_TRY(cudaMemcpy(loss, m->loss.p, sizeof(double), cudaMemcpyDeviceToHost));
    if (grad) MESS_CUDA_TRY(cudaMemcpy(grad, m->g.p, sizeof(float) * MlpParams::N, cudaMemcpyDeviceToHost));
    return MESS_OK;
}

// Training set = the converged densities of the given molecules (batched device SCF), every
// ordered atom pair one row; Adam over shuffled mini-batches of batch_rows rows.
extern "C" mess_status mess_mlp_train(mess_mlp* m, int nmol, mess_basis* const* bases, const mess_scf_opts* scf,
                                      int epochs, int batch_rows, double lr, double* loss_out)
{
    if (!m || nmol <= 0 || !bases || epochs <= 0 || batch_rows <= 0 || !(lr > 0)) {
        mess_set_error("bad training arguments");
        return MESS_EINVAL;
    }
    mess_basis* batch = nullptr;
    mess_status st = mess_batch_basis(nmol, bases, &batch);
    if (st != MESS_OK) return st;
    struct Guard { mess_basis* b; ~Guard() { mess_free_basis(b); delete b; } } guard{batch};
    AtomTables t;
    if ((st = atom_tables(batch, t)) != MESS_OK) return st;
    DevBuf<double> dD;
    MESS_CUDA_TRY(dD.alloc(batch->packed));
    std::vector<mess_scf_result> res(nmol);
    st = mess_scf_batch_density(batch, scf, res.data(), dD.p);
    if (st != MESS_OK && st != MESS_ENOCONV) return st;
    DevBuf<float> X, T, M, Xb, Tb, Mb;
    DevBuf<long long> idx;
    const long long rows = t.rows;
    MESS_CUDA_TRY(X.alloc(rows * DIN));
    MESS_CUDA_TRY(T.alloc(rows * DOUT));
    MESS_CUDA_TRY(M.alloc(rows * DOUT));
    if ((st = features(batch, t, dD.p, X.p, T.p, M.p, 0)) != MESS_OK) return st;
    const long long br = std::min<long long>(batch_rows, rows);
    MESS_CUDA_TRY(Xb.alloc(br * DIN));
    MESS_CUDA_TRY(Tb.alloc(br * DOUT));
    MESS_CUDA_TRY(Mb.alloc(br * DOUT));
    MESS_CUDA_TRY(idx.alloc(rows));
    std::vector<float> hM(rows * DOUT);
    MESS_CUDA_TRY(cudaMemcpy(hM.data(), M.p, sizeof(float) * hM.size(), cudaMemcpyDeviceToHost));
    std::vector<long long> perm(rows);
    for (long long i = 0; i < rows; ++i) perm[i] = i;
    unsigned long long rs = 0x243F6A8885A308D3ull;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    // step size: half-cosine decay from lr to 0 over the run (the last epochs average out the
    // mini-batch noise that a constant step leaves in the weights)
    const long long steps_per_epoch = rows / br, total_steps = std::max(1LL, steps_per_epoch * epochs);
    long long step = 0;
    for (int ep = 0; ep < epochs; ++ep) {
        for (long long i = rows - 1; i > 0; --i) {   // Fisher-Yates with an xorshift stream
            rs ^= rs << 13; rs ^= rs >> 7; rs ^= rs << 17;
            std::swap(perm[i], perm[rs % (unsigned long long)(i + 1)]);
        }
        MESS_CUDA_TRY(cudaMemcpy(idx.p, perm.data(), sizeof(long long) * rows, cudaMemcpyHostToDevice));
        double ep_loss = 0.0;
        long long nb = 0;
        for (long long r0 = 0; r0 + br <= rows; r0 += br, ++nb) {
            k_gather_rows<<<grid1(br * DIN), 256>>>(X.p, idx.p + r0, br, DIN, Xb.p);
            k_gather_rows<<<grid1(br * DOUT), 256>>>(T.p, idx.p + r0, br, DOUT, Tb.p);
            k_gather_rows<<<grid1(br * DOUT), 256>>>(M.p, idx.p + r0, br, DOUT, Mb.p);
            double count = 0.0;
            for (long long i = r0; i < r0 + br; ++i)
                for (int c = 0; c < DOUT; ++c) count += hM[perm[i] * DOUT + c];
            MESS_CUDA_TRY(forward(m, Xb.p, br, 0));
            MESS_CUDA_TRY(backward(m, Tb.p, Mb.p, br, count, 0));
            m->step++;
            const float c1 = 1.f - powf(b1, (float)m->step), c2 = 1.f - powf(b2, (float)m->step);
            const double lr_t = lr * 0.5 * (1.0 + cos(M_PI * (double)step / (double)total_steps));
            ++step;
            k_adam<<<(MlpParams::N + 255) / 256, 256>>>(m->w.p, m->g.p, m->m1.p, m->m2.p, MlpParams::N, (float)lr_t, b1,
                                                      b2, eps, c1, c2);
            MESS_CUDA_TRY(refresh_bf16(m, 0));
            double l = 0.0;
            MESS_CUDA_TRY(cudaMemcpy(&l, m->loss.p, sizeof(double), cudaMemcpyDeviceToHost));
            ep_loss += l;
        }
        if (loss_out) loss_out[ep] = nb ? ep_loss / nb : 0.0;
    }
    MESS_CUDA_TRY(cudaDeviceSynchronize());
    return MESS_OK;
}

extern "C" mess_status mess_mlp_predict(const mess_mlp* m, const mess_basis* b, double* D0)
{
    if (!m || !b || !D0) { mess_set_error("null argument"); return MESS_EINVAL; }
    if (b->nmol != 1) { mess_set_error("single-molecule bases only"); return MESS_EINVAL; }
    { const mess_status gs = mess_basis_gpu(const_cast<mess_basis*>(b)); if (gs != MESS_OK) return gs; }
    DevBuf<double> d;
    MESS_CUDA_TRY(d.alloc(b->packed));
    mess_status st = mess_mlp_guess_device(m, b, d.p, 0);
    if (st != MESS_OK) return st;
    MESS_CUDA_TRY(cudaMemcpy(D0, d.p, sizeof(double) * b->packed, cudaMemcpyDeviceToHost));
    return MESS_OK;
}
