// Exchange-correlation part of the Kohn-Sham energy functional (paper Sec. 5.1: the Hamiltonian's
// xc_method "lda" or "pbe"): the density of a closed-shell density matrix on a molecular quadrature
// grid, the functional's energy and its matrix V_xc,mn = dE_xc / dD_mn.
//
// Grid (per atom, then Becke's fuzzy-cell partition between the atoms of each molecule):
//   radial: Gauss-Chebyshev of the second kind, x_i = cos(i pi / (N + 1)), i = 1..N, weight
//           pi / (N + 1) sin^2(i pi / (N + 1)) / sqrt(1 - x_i^2), mapped by r = R (1 + x) / (1 - x)
//           (Jacobian 2 R / (1 - x)^2, times r^2); R = 0.35 angstrom for H (its Bragg-Slater
//           radius), half the Bragg-Slater radius otherwise (C 0.35, N 0.325, O 0.30 angstrom);
//           N = 50 for H, 75 otherwise;
//   angular: Gauss-Legendre nodes in cos(theta) (16) times 32 equally spaced phi, weight
//           w_theta * 2 pi / 32;
//   partition: w_A(r) = P_A(r) / sum_B P_B(r), P_A = prod_{B != A} s(mu_AB), mu_AB = (|r - R_A| -
//           |r - R_B|) / |R_A - R_B|, s(mu) = (1 - f(f(f(mu)))) / 2, f(mu) = 3/2 mu - 1/2 mu^3.
// Functionals (closed shell): LDA = Slater exchange + Perdew-Wang 1992 correlation; PBE (Perdew,
// Burke & Ernzerhof 1996) on top of the same PW92 correlation.  Derivatives are written out
// analytically below.
#include <math.h>

#include <algorithm>
#include <vector>

#include "mess_internal.h"

namespace {

constexpr double kAngstrom = 1.0 / 0.52917721092;
constexpr int kNTheta = 16, kNPhi = 32;
constexpr double kRhoMin = 1e-14;   // points with less density carry no exchange-correlation energy

double radius_of(int Z)
{
    switch (Z) {
    case 1: return 0.35;
    case 6: return 0.35;
    case 7: return 0.325;
    case 8: return 0.30;
    default: return 0.35;
    }
}

// Gauss-Legendre nodes and weights on [-1, 1]: Newton's method on P_n from the Chebyshev guesses
// cos(pi (i + 3/4) / (n + 1/2)), P_n and P_n' by the three-term recurrence.
void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w)
{
    x.assign(n, 0.0);
    w.assign(n, 0.0);
    for (int i = 0; i < n; ++i) {
        double z = cos(M_PI * (i + 0.75) / (n + 0.5)), dp = 0.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            const double dz = p1 / dp;
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        x[n - 1 - i] = z;
        w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

// ------------------------------------------------------------------------------------------ kernels
struct GridArgs {
    const double* pts;       // [npts][3]
    double* w;               // [npts] radial x angular weight, times the partition after k_becke
    const int* atom;         // [npts] global atom index of the point's atomic grid
    const int* mol;          // [npts]
    const long long* pbase;  // [nmol + 1] first point of each molecule
    const int* atom_off;     // [nmol] first atom of each molecule
    const int* atom_n;       // [nmol]
    const double* xyz;       // [natom][3]
    long long npts;
};

__global__ void k_becke(GridArgs g)
{
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= g.npts) return;
    const int m = g.mol[p], a0 = g.atom_off[m], na = g.atom_n[m], own = g.atom[p];
    if (na == 1) return;
    const double x = g.pts[3 * p], y = g.pts[3 * p + 1], z = g.pts[3 * p + 2];
    double sum = 0.0, mine = 0.0;
    for (int A = a0; A < a0 + na; ++A) {
        const double* RA = g.xyz + 3 * A;
        const double dA = sqrt((x - RA[0]) * (x - RA[0]) + (y - RA[1]) * (y - RA[1]) + (z - RA[2]) * (z - RA[2]));
        double P = 1.0;
        for (int B = a0; B < a0 + na; ++B) {
            if (B == A) continue;
            const double* RB = g.xyz + 3 * B;
            const double dB = sqrt((x - RB[0]) * (x - RB[0]) + (y - RB[1]) * (y - RB[1]) + (z - RB[2]) * (z - RB[2]));
            const double RAB = sqrt((RA[0] - RB[0]) * (RA[0] - RB[0]) + (RA[1] - RB[1]) * (RA[1] - RB[1]) +
                                    (RA[2] - RB[2]) * (RA[2] - RB[2]));
            double f = (dA - dB) / RAB;
            for (int k = 0; k < 3; ++k) f = 1.5 * f - 0.5 * f * f * f;
            P *= 0.5 * (1.0 - f);
        }
        sum += P;
        if (A == own) mine = P;
    }
    g.w[p] *= sum > 0.0 ? mine / sum : 0.0;
}

struct AoArgs {
    const double* pts;
    const int* mol;
    long long npts;
    const int* shell_off;    // [nmol] first shell of the molecule
    const int* shell_n;      // [nmol]
    const int* shell_l;
    const int* shell_K;
    const int* shell_poff;   // first primitive of the shell
    const int* shell_fl;     // first function of the shell within its molecule
    const double* shell_R;   // [nshell][3]
    const double* alpha;
    const double* coef;
    const double* fscale;    // per global function: component normalisation
    const int* fbase;        // [nmol] global index of the molecule's first function
    const long long* pbase;  // [nmol + 1]
    const long long* aobase; // [nmol] offset of the molecule's [npts_m][n_m] block
    const int* mn;           // [nmol] functions of the molecule
    double* phi;             // values
    double* dphi;            // gradients: three blocks [3][npts_m][n_m] from 3 * aobase[m]
};

// value and gradient of every basis function of the point's molecule at the point
__global__ void k_ao(AoArgs a)
{
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= a.npts) return;
    const int m = a.mol[p], n = a.mn[m];
    const long long lp = p - a.pbase[m], np_ = a.pbase[m + 1] - a.pbase[m];
    double* ph = a.phi + a.aobase[m] + lp * n;
    double* dx = a.dphi + 3 * a.aobase[m] + lp * n;
    double* dy = dx + np_ * n;
    double* dz = dy + np_ * n;
    const double x = a.pts[3 * p], y = a.pts[3 * p + 1], z = a.pts[3 * p + 2];
    for (int s = a.shell_off[m]; s < a.shell_off[m] + a.shell_n[m]; ++s) {
        const double X = x - a.shell_R[3 * s], Y = y - a.shell_R[3 * s + 1], Z = z - a.shell_R[3 * s + 2];
        const double r2 = X * X + Y * Y + Z * Z;
        double g = 0.0, gd = 0.0;   // sum c e^{-a r^2}, sum -2 a c e^{-a r^2}
        for (int k = 0; k < a.shell_K[s]; ++k) {
            const double al = a.alpha[a.shell_poff[s] + k];
            const double e = a.coef[a.shell_poff[s] + k] * exp(-al * r2);
            g += e;
            gd -= 2.0 * al * e;
        }
        const int l = a.shell_l[s], f0 = a.shell_fl[s];
        int k = 0;
        for (int lx = l; lx >= 0; --lx)
            for (int ly = l - lx; ly >= 0; --ly, ++k) {
                const int lz = l - lx - ly;
                const double px = lx == 0 ? 1.0 : (lx == 1 ? X : X * X);
                const double py = ly == 0 ? 1.0 : (ly == 1 ? Y : Y * Y);
                const double pz = lz == 0 ? 1.0 : (lz == 1 ? Z : Z * Z);
                const double dpx = lx == 0 ? 0.0 : (lx == 1 ? 1.0 : 2.0 * X);
                const double dpy = ly == 0 ? 0.0 : (ly == 1 ? 1.0 : 2.0 * Y);
                const double dpz = lz == 0 ? 0.0 : (lz == 1 ? 1.0 : 2.0 * Z);
                const double sc = a.fscale[a.fbase[m] + f0 + k];
                const double poly = px * py * pz;
                ph[f0 + k] = sc * poly * g;
                dx[f0 + k] = sc * (dpx * py * pz * g + poly * gd * X);
                dy[f0 + k] = sc * (px * dpy * pz * g + poly * gd * Y);
                dz[f0 + k] = sc * (px * py * dpz * g + poly * gd * Z);
            }
    }
}

// Perdew-Wang 1992 correlation energy per electron (closed shell) and its derivative in rs
__device__ __forceinline__ void pw92(double rs, double& ec, double& dec)
{
    const double A = 0.031091, a1 = 0.21370, b1 = 7.5957, b2 = 3.5876, b3 = 1.6382, b4 = 0.49294;
    const double srs = sqrt(rs);
    const double Q = 2.0 * A * (b1 * srs + b2 * rs + b3 * rs * srs + b4 * rs * rs);
    const double dQ = 2.0 * A * (0.5 * b1 / srs + b2 + 1.5 * b3 * srs + 2.0 * b4 * rs);
    const double L = log1p(1.0 / Q);
    ec = -2.0 * A * (1.0 + a1 * rs) * L;
    dec = -2.0 * A * a1 * L + 2.0 * A * (1.0 + a1 * rs) * dQ / (Q * (Q + 1.0));
}

struct FuncArgs {
    const double* phi;
    const double* dphi;
    const double* D;         // packed density
    const long long* mbase;  // [nmol] offset of the molecule's n x n block
    const int* mol;
    const long long* pbase;
    const long long* aobase;
    const int* mn;
    const double* w;
    long long npts;
    int kind;                // 1 LDA, 2 PBE
    double* vrho;            // [npts] w * d e / d rho
    double* vgrad;           // [npts][3] w * 2 d e / d sigma * grad rho (PBE)
    double* Exc;             // [nmol] accumulated
};

// density, its gradient, and the functional at every point; E_xc accumulated per molecule
__global__ void k_functional(FuncArgs f)
{
    __shared__ double red[32];
    __shared__ int mols[2];
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    double e = 0.0;
    int m = -1;
    if (p < f.npts) {
        m = f.mol[p];
        const int n = f.mn[m];
        const long long lp = p - f.pbase[m], np_ = f.pbase[m + 1] - f.pbase[m];
        const double* ph = f.phi + f.aobase[m] + lp * n;
        const double* dx = f.dphi + 3 * f.aobase[m] + lp * n;
        const double* dy = dx + np_ * n;
        const double* dz = dy + np_ * n;
        const double* D = f.D + f.mbase[m];
        double rho = 0.0, gx = 0.0, gy = 0.0, gz = 0.0;
        for (int i = 0; i < n; ++i) {
            double t = 0.0;
            for (int j = 0; j < n; ++j) t += D[(long long)i * n + j] * ph[j];
            rho += t * ph[i];
            gx += 2.0 * t * dx[i];
            gy += 2.0 * t * dy[i];
            gz += 2.0 * t * dz[i];
        }
        double vr = 0.0, vs = 0.0;
        if (rho > kRhoMin) {
            const double c13 = cbrt(rho);
            const double cx = 0.7385587663820224;    // (3/4)(3/pi)^(1/3)
            const double ex = -cx * rho * c13;
            const double vx = -(4.0 / 3.0) * cx * c13;
            const double rs = 0.6203504908994001 / c13;   // (3/(4 pi))^(1/3) rho^(-1/3)
            double ec, dec;
            pw92(rs, ec, dec);
            const double drs = -rs / (3.0 * rho);
            if (f.kind == 1) {
                e = ex + rho * ec;
                vr = vx + ec + rho * dec * drs;
            } else {
                const double sigma = gx * gx + gy * gy + gz * gz;
                const double kF = 3.0936677262801355 * c13;            // (3 pi^2 rho)^(1/3)
                const double kappa = 0.804, beta = 0.06672455060314922;
                const double mu = beta * M_PI * M_PI / 3.0, gamma = (1.0 - M_LN2) / (M_PI * M_PI);
                // exchange: ex F(s^2), s^2 = sigma / (2 kF rho)^2 (d s^2 / d rho = -8/3 s^2 / rho)
                const double s2 = sigma / (4.0 * kF * kF * rho * rho);
                const double den = 1.0 + mu * s2 / kappa;
                const double F = 1.0 + kappa - kappa / den;
                const double dF = mu / (den * den);
                const double exg = ex * F;
                const double dex_drho = vx * F + ex * dF * (-8.0 / 3.0) * s2 / rho;
                const double dex_dsig = ex * dF / (4.0 * kF * kF * rho * rho);
                // correlation: rho (ec + H), u = t^2 = sigma pi / (16 kF rho^2) (d u / d rho = -7/3 u / rho)
                const double u = sigma * M_PI / (16.0 * kF * rho * rho);
                const double E = exp(-ec / gamma);
                const double bg = beta / gamma;
                const double A = bg / (E - 1.0);
                const double dA_dec = A * A * E / beta;
                const double au = A * u;
                const double M = 1.0 + au + au * au;
                const double y = bg * u * (1.0 + au) / M;
                const double H = gamma * log1p(y);
                const double dH_dy = gamma / (1.0 + y);
                const double dy_du = bg * (1.0 + 2.0 * au) / (M * M);
                const double dy_dA = -bg * u * u * u * A * (2.0 + au) / (M * M);
                const double dec_drho = dec * drs;
                const double dH_drho = dH_dy * (dy_dA * dA_dec * dec_drho + dy_du * (-7.0 / 3.0) * u / rho);
                e = exg + rho * (ec + H);
                vr = dex_drho + ec + H + rho * (dec_drho + dH_drho);
                vs = dex_dsig + rho * dH_dy * dy_du * M_PI / (16.0 * kF * rho * rho);
            }
        }
        const double w = f.w[p];
        e *= w;
        f.vrho[p] = w * vr;
        if (f.kind == 2) {
            f.vgrad[3 * p] = w * 2.0 * vs * gx;
            f.vgrad[3 * p + 1] = w * 2.0 * vs * gy;
            f.vgrad[3 * p + 2] = w * 2.0 * vs * gz;
        }
    }
    // block sum per molecule (a block holds points of at most two molecules in practice; the general
    // case falls back to one atomic per point)
    if (threadIdx.x == 0) { mols[0] = m; mols[1] = 0; }
    __syncthreads();
    if (m >= 0 && m != mols[0]) atomicExch(&mols[1], 1);
    __syncthreads();
    if (mols[1]) {
        if (m >= 0 && e != 0.0) atomicAdd(f.Exc + m, e);
        return;
    }
    for (int o = 16; o > 0; o >>= 1) e += __shfl_xor_sync(0xffffffffu, e, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = e;
    __syncthreads();
    if (threadIdx.x < 32) {
        double t = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (threadIdx.x == 0 && mols[0] >= 0) atomicAdd(f.Exc + mols[0], t);
    }
}

struct VxcArgs {
    const double* phi;
    const double* dphi;
    const double* vrho;
    const double* vgrad;
    const long long* pbase;
    const long long* aobase;
    const long long* mbase;
    const int* mn;
    int kind;
    int chunk;               // points per block
    double* V;               // packed, accumulated
};

// V_mn += sum over a chunk of the molecule's points of a_m phi_n + phi_m a_n, a = (1/2) w v_rho phi +
// w 2 v_sigma grad rho . grad phi (vgrad holds w 2 v_sigma grad rho); grid (chunks, nmol)
__global__ void k_vxc(VxcArgs v)
{
    const int m = blockIdx.y;
    const int n = v.mn[m];
    const long long np_ = v.pbase[m + 1] - v.pbase[m];
    const long long p0 = (long long)blockIdx.x * v.chunk;
    if (p0 >= np_) return;
    const long long p1 = min(np_, p0 + v.chunk);
    const double* ph = v.phi + v.aobase[m];
    const double* dx = v.dphi + 3 * v.aobase[m];
    const double* dy = dx + np_ * n;
    const double* dz = dy + np_ * n;
    const long long gp = v.pbase[m];
    for (int t = threadIdx.x; t < n * n; t += blockDim.x) {
        const int i = t / n, j = t % n;
        if (j < i) continue;
        double s = 0.0;
        for (long long p = p0; p < p1; ++p) {
            const double fi = ph[p * n + i], fj = ph[p * n + j];
            double ai = 0.5 * v.vrho[gp + p] * fi, aj = 0.5 * v.vrho[gp + p] * fj;
            if (v.kind == 2) {
                const double* g = v.vgrad + 3 * (gp + p);
                ai += g[0] * dx[p * n + i] + g[1] * dy[p * n + i] + g[2] * dz[p * n + i];
                aj += g[0] * dx[p * n + j] + g[1] * dy[p * n + j] + g[2] * dz[p * n + j];
            }
            s += ai * fj + fi * aj;
        }
        atomicAdd(v.V + v.mbase[m] + (long long)i * n + j, s);
        if (i != j) atomicAdd(v.V + v.mbase[m] + (long long)j * n + i, s);
    }
}

}  // namespace

// ------------------------------------------------------------------------------------------ host
void mess_free_xc(mess_basis* b)
{
    XcState& x = b->xc;
    x.pts.free(); x.w.free(); x.atom.free(); x.mol.free(); x.pbase.free(); x.phi.free(); x.dphi.free();
    x.aobase.free(); x.vrho.free(); x.vgrad.free(); x.fbase.free(); x.shell_off.free(); x.shell_n.free();
    x.shell_fl.free(); x.Exc.free();
    x.npts = 0;
    x.ready = false;
}

mess_status mess_xc_prepare(mess_basis* b, cudaStream_t s)
{
    XcState& X = b->xc;
    if (X.ready) return MESS_OK;
    std::vector<double> pts, w;
    std::vector<int> atom, mol;
    std::vector<long long> pbase(1, 0), aobase;
    std::vector<double> ct, wt;
    gauss_legendre(kNTheta, ct, wt);
    long long ao = 0;
    for (int m = 0; m < b->nmol; ++m) {
        const long long start = (long long)w.size();
        for (int A = b->mol_atom_off[m]; A < b->mol_atom_off[m] + b->mol_atom_n[m]; ++A) {
            const int Z = b->Z[A];
            const int nr = Z == 1 ? 50 : 75;
            const double R = radius_of(Z) * kAngstrom;
            for (int i = 1; i <= nr; ++i) {
                const double th = i * M_PI / (nr + 1);
                const double xr = cos(th);
                const double wx = M_PI / (nr + 1) * sin(th) * sin(th) / sqrt(1.0 - xr * xr);
                const double r = R * (1.0 + xr) / (1.0 - xr);
                const double wr = wx * r * r * 2.0 * R / ((1.0 - xr) * (1.0 - xr));
                for (int t = 0; t < kNTheta; ++t) {
                    const double st = sqrt(1.0 - ct[t] * ct[t]);
                    for (int k = 0; k < kNPhi; ++k) {
                        const double ph = 2.0 * M_PI * k / kNPhi;
                        pts.push_back(b->xyz[3 * A] + r * st * cos(ph));
                        pts.push_back(b->xyz[3 * A + 1] + r * st * sin(ph));
                        pts.push_back(b->xyz[3 * A + 2] + r * ct[t]);
                        w.push_back(wr * wt[t] * 2.0 * M_PI / kNPhi);
                        atom.push_back(A);
                        mol.push_back(m);
                    }
                }
            }
        }
        pbase.push_back((long long)w.size());
        aobase.push_back(ao);
        ao += ((long long)w.size() - start) * b->mol_nbf[m];
    }
    std::vector<int> fbase(b->nmol, 0), shell_fl;
    for (int m = 1; m < b->nmol; ++m) fbase[m] = fbase[m - 1] + b->mol_nbf[m - 1];
    for (const HostShell& sh : b->shells) shell_fl.push_back(sh.fl);
    X.npts = (long long)w.size();
    X.ao = ao;
    X.mol_npts_max = 0;
    for (int m = 0; m < b->nmol; ++m) X.mol_npts_max = std::max(X.mol_npts_max, pbase[m + 1] - pbase[m]);
    MESS_CUDA_TRY(X.pts.upload(pts));
    MESS_CUDA_TRY(X.w.upload(w));
    MESS_CUDA_TRY(X.atom.upload(atom));
    MESS_CUDA_TRY(X.mol.upload(mol));
    MESS_CUDA_TRY(X.pbase.upload(pbase));
    MESS_CUDA_TRY(X.aobase.upload(aobase));
    MESS_CUDA_TRY(X.fbase.upload(fbase));
    MESS_CUDA_TRY(X.shell_off.upload(b->mol_shell_off));
    MESS_CUDA_TRY(X.shell_n.upload(b->mol_shell_n));
    MESS_CUDA_TRY(X.shell_fl.upload(shell_fl));
    MESS_CUDA_TRY(X.phi.alloc((size_t)ao));
    MESS_CUDA_TRY(X.dphi.alloc((size_t)ao * 3));
    MESS_CUDA_TRY(X.vrho.alloc((size_t)X.npts));
    MESS_CUDA_TRY(X.vgrad.alloc((size_t)X.npts * 3));
    MESS_CUDA_TRY(X.Exc.alloc((size_t)b->nmol));
    const int T = 256;
    const unsigned blocks = (unsigned)((X.npts + T - 1) / T);
    GridArgs g{X.pts.p, X.w.p, X.atom.p, X.mol.p, X.pbase.p, b->d_mol_atom_off.p, b->d_mol_atom_n.p, b->d_xyz.p, X.npts};
    k_becke<<<blocks, T, 0, s>>>(g);
    MESS_CUDA_TRY(cudaGetLastError());
    AoArgs a{X.pts.p, X.mol.p, X.npts, X.shell_off.p, X.shell_n.p, b->d_shell_l.p, b->d_shell_K.p, b->d_shell_poff.p,
             X.shell_fl.p, b->d_shell_R.p, b->d_shell_alpha.p, b->d_shell_coef.p, b->d_fscale.p, X.fbase.p, X.pbase.p,
             X.aobase.p, b->d_mol_n.p, X.phi.p, X.dphi.p};
    k_ao<<<blocks, T, 0, s>>>(a);
    MESS_CUDA_TRY(cudaGetLastError());
    X.ready = true;
    return MESS_OK;
}

mess_status mess_xc_eval(mess_basis* b, int kind, const double* dD, double* dV, double* dExc, cudaStream_t s)
{
    if (kind != 1 && kind != 2) { mess_set_error("exchange-correlation: unknown functional %d", kind); return MESS_EINVAL; }
    XcState& X = b->xc;
    if (!X.ready) { mess_set_error("exchange-correlation grid not prepared"); return MESS_EINVAL; }
    MESS_CUDA_TRY(cudaMemsetAsync(dExc, 0, sizeof(double) * b->nmol, s));
    MESS_CUDA_TRY(cudaMemsetAsync(dV, 0, sizeof(double) * b->packed, s));
    const int T = 256;
    const unsigned blocks = (unsigned)((X.npts + T - 1) / T);
    FuncArgs f{X.phi.p, X.dphi.p, dD, b->d_mol_base.p, X.mol.p, X.pbase.p, X.aobase.p, b->d_mol_n.p, X.w.p, X.npts,
               kind, X.vrho.p, X.vgrad.p, dExc};
    k_functional<<<blocks, T, 0, s>>>(f);
    MESS_CUDA_TRY(cudaGetLastError());
    const int chunk = 2048;   // points per block of the V_xc reduction; the largest molecule grid sets the grid
    VxcArgs v{X.phi.p, X.dphi.p, X.vrho.p, X.vgrad.p, X.pbase.p, X.aobase.p, b->d_mol_base.p, b->d_mol_n.p, kind, chunk, dV};
    dim3 grid((unsigned)((X.mol_npts_max + chunk - 1) / chunk), (unsigned)b->nmol);
    k_vxc<<<grid, 256, 0, s>>>(v);
    MESS_CUDA_TRY(cudaGetLastError());
    return MESS_OK;
}

extern "C" mess_status mess_xc(const mess_basis* bc, int xc, const double* D, double* Exc, double* V, long long* npts)
{
    mess_basis* b = const_cast<mess_basis*>(bc);
    if (!b || !D) { mess_set_error("null argument"); return MESS_EINVAL; }
    if (xc != 1 && xc != 2) { mess_set_error("mess_xc: functional must be 1 (LDA) or 2 (PBE)"); return MESS_EINVAL; }
    { const mess_status gs = mess_basis_gpu(b); if (gs != MESS_OK) return gs; }
    mess_status st = mess_xc_prepare(b, 0);
    if (st != MESS_OK) return st;
    const size_t nn = (size_t)b->packed;
    DevBuf<double> d;
    MESS_CUDA_TRY(d.alloc(2 * nn + b->nmol));
    cudaError_t e = cudaMemcpy(d.p, D, nn * sizeof(double), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        st = mess_xc_eval(b, xc, d.p, d.p + nn, d.p + 2 * nn, 0);
        if (st == MESS_OK) {
            e = cudaDeviceSynchronize();
            if (e == cudaSuccess && V) e = cudaMemcpy(V, d.p + nn, nn * sizeof(double), cudaMemcpyDeviceToHost);
            if (e == cudaSuccess && Exc) e = cudaMemcpy(Exc, d.p + 2 * nn, b->nmol * sizeof(double), cudaMemcpyDeviceToHost);
        }
    }
    d.free();
    if (st != MESS_OK) return st;
    if (e != cudaSuccess) { mess_set_error("mess_xc: %s", cudaGetErrorString(e)); return MESS_ECUDA; }
    if (npts) *npts = b->xc.npts;
    return MESS_OK;
}
