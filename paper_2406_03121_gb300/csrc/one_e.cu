// One-electron integrals S, T, V over contracted Cartesian shells (Obara-Saika recursions), FP64.
//   overlap (1-D):  s_{i+1,j} = X_PA s_ij + (i s_{i-1,j} + j s_{i,j-1}) / (2p),
//                   s_{i,j+1} = X_PB s_ij + (i s_{i-1,j} + j s_{i,j-1}) / (2p),  s_00 = 1
//   kinetic:        T = 1/2 <grad a | grad b>, with d/dx (x_A^i e^{-a x_A^2}) = i x_A^{i-1} - 2a x_A^{i+1}
//   nuclear:        [e|0]^(m) by the VRR
//                   [e+1_i|0]^(m) = PA_i [e|0]^(m) - PC_i [e|0]^(m+1)
//                                   + e_i/(2p) ([e-1_i|0]^(m) - [e-1_i|0]^(m+1)),
//                   [0|0]^(m) = 2 pi/p exp(-ab/p |AB|^2) F_m(p |PC|^2), then the HRR
//                   (a|b+1_i) = (a+1_i|b) + AB_i (a|b).
// One thread per canonical shell pair writes both (m, n) and (n, m) blocks.
#include <math.h>

#include "mess_internal.h"

namespace {

constexpr int LMAX = MESS_LMAX;
constexpr int LAB = 2 * LMAX;                    // highest |e| in the nuclear VRR
constexpr int NCE = (LAB + 1) * (LAB + 2) * (LAB + 3) / 6;   // Cartesian triples with |e| <= LAB

__device__ __forceinline__ int cart_index(int lx, int ly, int lz)
{
    const int L = lx + ly + lz;
    return L * (L + 1) * (L + 2) / 6 + (L - lx) * (L - lx + 1) / 2 + lz;
}

__device__ void boys_f64_all(int L, double T, double* F, const double* __restrict__ tab)
{
    if (T < MESS_BOYS_TMAX64) {
        const int k = __double2int_rn(T * MESS_BOYS_INV_DT);
        const double x = (double)k * MESS_BOYS_DT - T;
        const double* row = tab + (size_t)k * MESS_BOYS_NCOL;
        for (int m = 0; m <= L; ++m) {
            double s = row[m + 7];
            for (int j = 7; j >= 1; --j) s = row[m + j - 1] + s * x / j;
            F[m] = s;
        }
    } else {
        const double rt = rsqrt(T), e = exp(-T);
        F[0] = 0.886226925452758014 * rt;
        for (int m = 0; m < L; ++m) F[m + 1] = ((2 * m + 1) * F[m] - e) * 0.5 / T;
    }
}

struct ShellArgs {
    const int *l, *K, *f0, *poff;
    const double *R, *alpha, *coef, *fscale;
    const int* Z;
    const double* xyz;
    const int* pair_mol;          // molecule of each pair
    const int* atom_off;          // [nmol] first atom of the molecule
    const int* atom_n;            // [nmol] atoms of the molecule
    const long long* mbase;       // [nmol] offset of the molecule's block in the packed matrices
    const int* mn;                // [nmol] basis functions of the molecule
    const int* fglob;             // [nbf] global function index -> offset within its molecule's basis
    const double* boys;
};

__global__ void k_one_e(const int* __restrict__ pa, const int* __restrict__ pb, int npair, ShellArgs s,
                        double* __restrict__ S, double* __restrict__ T, double* __restrict__ V, int n)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= npair) return;
    const int A = pa[t], B = pb[t];
    const int la = s.l[A], lb = s.l[B];
    const int na = (la + 1) * (la + 2) / 2, nb = (lb + 1) * (lb + 2) / 2;
    double Sab[6][6], Tab[6][6], Vab[6][6];
    for (int i = 0; i < 6; ++i)
        for (int j = 0; j < 6; ++j) Sab[i][j] = Tab[i][j] = Vab[i][j] = 0.0;
    const double Ax = s.R[3 * A], Ay = s.R[3 * A + 1], Az = s.R[3 * A + 2];
    const double Bx = s.R[3 * B], By = s.R[3 * B + 1], Bz = s.R[3 * B + 2];
    const double AB[3] = {Ax - Bx, Ay - By, Az - Bz};
    const double ab2 = AB[0] * AB[0] + AB[1] * AB[1] + AB[2] * AB[2];
    for (int ia = 0; ia < s.K[A]; ++ia) {
        for (int ib = 0; ib < s.K[B]; ++ib) {
            const double a = s.alpha[s.poff[A] + ia], b = s.alpha[s.poff[B] + ib];
            const double c = s.coef[s.poff[A] + ia] * s.coef[s.poff[B] + ib];
            const double p = a + b, o2p = 0.5 / p;
            const double P[3] = {(a * Ax + b * Bx) / p, (a * Ay + b * By) / p, (a * Az + b * Bz) / p};
            const double PA[3] = {P[0] - Ax, P[1] - Ay, P[2] - Az};
            const double PB[3] = {P[0] - Bx, P[1] - By, P[2] - Bz};
            const double Eab = exp(-a * b / p * ab2);
            // 1-D overlaps s[x][i][j], i <= la+1, j <= lb+1
            double s1[3][LMAX + 2][LMAX + 2];
            for (int x = 0; x < 3; ++x) {
                for (int i = 0; i <= la + 1; ++i)
                    for (int j = 0; j <= lb + 1; ++j) {
                        double v;
                        if (i == 0 && j == 0) v = 1.0;
                        else if (i > 0) {
                            v = PA[x] * s1[x][i - 1][j];
                            if (i > 1) v += (i - 1) * o2p * s1[x][i - 2][j];
                            if (j > 0) v += j * o2p * s1[x][i - 1][j - 1];
                        } else {
                            v = PB[x] * s1[x][0][j - 1];
                            if (j > 1) v += (j - 1) * o2p * s1[x][0][j - 2];
                        }
                        s1[x][i][j] = v;
                    }
            }
            const double s00 = c * pow(M_PI / p, 1.5) * Eab;
            // nuclear attraction VRR over all nuclei
            double Ve[NCE];
            for (int k = 0; k < NCE; ++k) Ve[k] = 0.0;
            const int Lab = la + lb;
            const int mol = s.pair_mol[t];
            for (int C = s.atom_off[mol]; C < s.atom_off[mol] + s.atom_n[mol]; ++C) {
                const double PC[3] = {P[0] - s.xyz[3 * C], P[1] - s.xyz[3 * C + 1], P[2] - s.xyz[3 * C + 2]};
                double F[LAB + 1];
                boys_f64_all(Lab, p * (PC[0] * PC[0] + PC[1] * PC[1] + PC[2] * PC[2]), F, s.boys);
                double th[NCE][LAB + 1];
                const double pre = -(double)s.Z[C] * 2.0 * M_PI / p * Eab * c;
                for (int m = 0; m <= Lab; ++m) th[0][m] = pre * F[m];
                for (int L = 1; L <= Lab; ++L)
                    for (int lx = L; lx >= 0; --lx)
                        for (int ly = L - lx; ly >= 0; --ly) {
                            const int lz = L - lx - ly;
                            const int e[3] = {lx, ly, lz};
                            int d = 0;
                            for (int x = 1; x < 3; ++x) if (e[x] > e[d]) d = x;
                            int e1[3] = {lx, ly, lz};
                            e1[d] -= 1;
                            const int i1 = cart_index(e1[0], e1[1], e1[2]);
                            const int it = cart_index(lx, ly, lz);
                            for (int m = 0; m <= Lab - L; ++m) {
                                double v = PA[d] * th[i1][m] - PC[d] * th[i1][m + 1];
                                if (e1[d] > 0) {
                                    int e2[3] = {e1[0], e1[1], e1[2]};
                                    e2[d] -= 1;
                                    const int i2 = cart_index(e2[0], e2[1], e2[2]);
                                    v += e1[d] * o2p * (th[i2][m] - th[i2][m + 1]);
                                }
                                th[it][m] = v;
                            }
                        }
                for (int k = 0; k < cart_index(0, 0, Lab) + 1; ++k) Ve[k] += th[k][0];
            }
            // assemble the (a|b) blocks; nuclear via HRR (a|b+1_i) = (a+1_i|b) + AB_i (a|b)
            int ca = 0;
            for (int ax = la; ax >= 0; --ax)
                for (int ay = la - ax; ay >= 0; --ay, ++ca) {
                    const int az = la - ax - ay;
                    const int av[3] = {ax, ay, az};
                    int cb = 0;
                    for (int bx = lb; bx >= 0; --bx)
                        for (int by = lb - bx; by >= 0; --by, ++cb) {
                            const int bz = lb - bx - by;
                            const int bv[3] = {bx, by, bz};
                            double sx[3], dx[3];
                            for (int x = 0; x < 3; ++x) {
                                const int i = av[x], j = bv[x];
                                sx[x] = s1[x][i][j];
                                double g = 4.0 * a * b * s1[x][i + 1][j + 1];
                                if (i > 0) g -= 2.0 * b * i * s1[x][i - 1][j + 1];
                                if (j > 0) g -= 2.0 * a * j * s1[x][i + 1][j - 1];
                                if (i > 0 && j > 0) g += (double)i * j * s1[x][i - 1][j - 1];
                                dx[x] = g;
                            }
                            Sab[ca][cb] += s00 * sx[0] * sx[1] * sx[2];
                            Tab[ca][cb] += 0.5 * s00 * (dx[0] * sx[1] * sx[2] + sx[0] * dx[1] * sx[2] + sx[0] * sx[1] * dx[2]);
                            // HRR: expand b as sum over binomial shifts onto a
                            double v = 0.0;
                            for (int tx = 0; tx <= bx; ++tx)
                                for (int ty = 0; ty <= by; ++ty)
                                    for (int tz = 0; tz <= bz; ++tz) {
                                        // (a|b) = sum_t C(b,t) AB^{b-t} (a+t|0)
                                        double coef = 1.0;
                                        const int tv[3] = {tx, ty, tz};
                                        for (int x = 0; x < 3; ++x) {
                                            double bin = 1.0;
                                            for (int k = 0; k < tv[x]; ++k) bin = bin * (bv[x] - k) / (k + 1);
                                            coef *= bin * pow(AB[x], bv[x] - tv[x]);
                                        }
                                        v += coef * Ve[cart_index(ax + tx, ay + ty, az + tz)];
                                    }
                            Vab[ca][cb] += v;
                        }
                }
        }
    }
    const int fa = s.f0[A], fb = s.f0[B];       // global function indices (fscale)
    const int mol = s.pair_mol[t];
    const int nm = s.mn[mol];
    const long long base = s.mbase[mol];
    const int la0 = s.fglob[fa], lb0 = s.fglob[fb];   // offsets within the molecule
    (void)n;
    for (int i = 0; i < na; ++i)
        for (int j = 0; j < nb; ++j) {
            const double sc = s.fscale[fa + i] * s.fscale[fb + j];
            const size_t ij = base + (size_t)(la0 + i) * nm + lb0 + j, ji = base + (size_t)(lb0 + j) * nm + la0 + i;
            if (S) { S[ij] = sc * Sab[i][j]; S[ji] = sc * Sab[i][j]; }
            if (T) { T[ij] = sc * Tab[i][j]; T[ji] = sc * Tab[i][j]; }
            if (V) { V[ij] = sc * Vab[i][j]; V[ji] = sc * Vab[i][j]; }
        }
}

}  // namespace

cudaError_t mess_launch_one_e(const mess_basis* b, double* dS, double* dT, double* dV, cudaStream_t st)
{
    ShellArgs s;
    s.l = b->d_shell_l.p; s.K = b->d_shell_K.p; s.f0 = b->d_shell_f0.p; s.poff = b->d_shell_poff.p;
    s.R = b->d_shell_R.p; s.alpha = b->d_shell_alpha.p; s.coef = b->d_shell_coef.p; s.fscale = b->d_fscale.p;
    s.Z = b->d_Z.p; s.xyz = b->d_xyz.p; s.boys = b->d_boys64.p;
    s.pair_mol = b->d_pair_mol.p; s.atom_off = b->d_mol_atom_off.p; s.atom_n = b->d_mol_atom_n.p;
    s.mbase = b->d_mol_base.p; s.mn = b->d_mol_n.p; s.fglob = b->d_f_local.p;
    const int T = 64;
    k_one_e<<<(b->npair + T - 1) / T, T, 0, st>>>(b->d_pair_a.p, b->d_pair_b.p, b->npair, s, dS, dT, dV, b->nbf);
    return cudaGetLastError();
}
