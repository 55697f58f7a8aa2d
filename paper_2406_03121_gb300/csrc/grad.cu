// Nuclear gradient of the closed-shell Hartree-Fock energy (the derivative the paper obtains by
// automatic differentiation of E(P) + nuclear_energy, Sec. 1 and 4; here written out analytically).
//
// For a converged density D (W = D F D / 2 the energy-weighted density) and atom A, direction x:
//   dE/dA_x = sum_{m on A} sum_n [ 2 D_mn (d m|h|n) + D_mn (2 J'_mn - K'_mn) - 2 W_mn (d m|n) ]
//             - 2 sum_{m, n} D_mn (d m|V_A|n) + dE_nuc/dA_x,
//   J'_mn = sum_ls (d m n|l s) D_ls,  K'_mn = sum_ls (d m l|n s) D_ls,
// where d m is the derivative of basis function m with respect to its own centre, h = T + V and V_A
// the attraction of nucleus A (its operator derivative follows from translational invariance:
// d/dC <m|V_C|n> = -<d m|V_C|n> - <m|V_C|d n>).  For a Cartesian Gaussian component
// x^i y^j z^k exp(-a r^2), d/dA_x = 2a x^(i+1)(...) - i x^(i-1)(...): every d m is a combination of one
// function of a "raised" shell (l + 1, coefficients 2 a c) and one of a "lowered" shell (l - 1), so one
// pass of the one-electron kernels and one J/K build over the basis extended by those shells give every
// derivative integral above.  Shells up to p (derivatives up to d, the kernels' highest shell).
#include <math.h>

#include <vector>

#include "mess_internal.h"

namespace {

// sqrt((2L-1)!! / ((2i-1)!!(2j-1)!!(2k-1)!!)): the per-component factor of unit-norm Cartesian functions
double comp_scale(int i, int j, int k)
{
    auto df = [](int n) { double r = 1.0; while (n > 1) { r *= n; n -= 2; } return r; };
    return sqrt(df(2 * (i + j + k) - 1) / (df(2 * i - 1) * df(2 * j - 1) * df(2 * k - 1)));
}

// index of component (i, j, k) within its shell (x^i y^j z^k, i descending then j descending)
int comp_index(int i, int j, int k)
{
    const int L = i + j + k;
    int idx = 0;
    for (int lx = L; lx >= 0; --lx)
        for (int ly = L - lx; ly >= 0; --ly, ++idx)
            if (lx == i && ly == j && L - lx - ly == k) return idx;
    return -1;
}

struct GradArgs {
    int n, ne, natom;
    const double* D;        // n x n
    const double* W;        // n x n
    const double* Se;       // ne x ne (extended basis)
    const double* He;       // ne x ne, T + V
    const double* Je;       // ne x ne
    const double* Ke;       // ne x ne
    const double* VA;       // natom x ne x ne, attraction of one nucleus each
    const int* fatom;       // [n] atom of each function
    const int* ridx;        // [n][3] raised extended function of d m / d x (or -1)
    const double* rc;       // [n][3] its coefficient
    const int* lidx;        // [n][3] lowered extended function (or -1)
    const double* lc;       // [n][3]
    double* grad;           // natom x 3 (electronic part)
};

__device__ __forceinline__ double dmat(const double* X, int ne, int r, double rcoef, int l, double lcoef, int col)
{
    double v = 0.0;
    if (r >= 0) v += rcoef * X[(long long)r * ne + col];
    if (l >= 0) v += lcoef * X[(long long)l * ne + col];
    return v;
}

// one block per (atom, direction)
__global__ void k_grad(GradArgs g)
{
    __shared__ double red[32];
    const int A = blockIdx.x, x = blockIdx.y;
    const int n = g.n, ne = g.ne;
    const double* VA = g.VA + (long long)A * ne * ne;
    double s = 0.0;
    for (long long t = threadIdx.x; t < (long long)n * n; t += blockDim.x) {
        const int m = (int)(t / n), nu = (int)(t % n);
        const int r = g.ridx[3 * m + x], l = g.lidx[3 * m + x];
        const double rc = g.rc[3 * m + x], lc = g.lc[3 * m + x];
        const double Dmn = g.D[t];
        if (g.fatom[m] == A) {
            s += 2.0 * Dmn * dmat(g.He, ne, r, rc, l, lc, nu);
            s += Dmn * (2.0 * dmat(g.Je, ne, r, rc, l, lc, nu) - dmat(g.Ke, ne, r, rc, l, lc, nu));
            s -= 2.0 * g.W[t] * dmat(g.Se, ne, r, rc, l, lc, nu);
        }
        s -= 2.0 * Dmn * dmat(VA, ne, r, rc, l, lc, nu);
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        double t = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (threadIdx.x == 0) g.grad[3 * A + x] = t;
    }
}

// C = A + B elementwise
__global__ void k_add(const double* __restrict__ A, const double* __restrict__ B, double* __restrict__ C, long long count)
{
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < count; t += (long long)gridDim.x * blockDim.x)
        C[t] = A[t] + B[t];
}

// D_e = D in the leading n x n block of an ne x ne matrix, zero elsewhere
__global__ void k_embed(const double* __restrict__ D, int n, double* __restrict__ De, int ne)
{
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < (long long)ne * ne;
         t += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(t / ne), j = (int)(t % ne);
        De[t] = (i < n && j < n) ? D[(long long)i * n + j] : 0.0;
    }
}

// W = D F D / 2 with F = T + V + J - K/2 read from the leading block of the extended matrices
__global__ void k_energy_weighted(const double* __restrict__ D, const double* __restrict__ He,
                                  const double* __restrict__ Je, const double* __restrict__ Ke, int n, int ne,
                                  double* __restrict__ W)
{
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (long long)n * n) return;
    const int i = (int)(t / n), j = (int)(t % n);
    double s = 0.0;
    for (int k = 0; k < n; ++k) {
        double u = 0.0;
        for (int l = 0; l < n; ++l) {
            const long long kl = (long long)k * ne + l;
            u += (He[kl] + Je[kl] - 0.5 * Ke[kl]) * D[(long long)l * n + j];
        }
        s += D[(long long)i * n + k] * u;
    }
    W[t] = 0.5 * s;
}

}  // namespace

// step of the central differences of the numerical gradient, bohr
#define MESS_GRAD_STEP 1e-3

extern "C" mess_status mess_gradient_numerical(const mess_basis* bc, const mess_scf_opts* opts,
                                               mess_scf_result* res, double* grad)
{
    mess_basis* b = const_cast<mess_basis*>(bc);
    if (!b || !grad) { mess_set_error("null argument"); return MESS_EINVAL; }
    if (b->nmol != 1) { mess_set_error("mess_gradient_numerical: single-molecule bases only"); return MESS_EINVAL; }
    mess_scf_opts o{};
    if (opts) o = *opts;
    mess_scf_result r{};
    mess_status st = mess_scf(b, &o, &r, nullptr);
    if (res) *res = r;
    if (st != MESS_OK) return st;
    // the 12 natom displaced geometries R + k h e_(atom, axis), k = 2, 1, -1, -2, as one batch
    const int na = b->natom;
    const double h = MESS_GRAD_STEP;
    const int ks[4] = {2, 1, -1, -2};
    std::vector<mess_basis*> disp;
    disp.reserve((size_t)12 * na);
    struct FreeAll {
        std::vector<mess_basis*>& v;
        ~FreeAll() { for (mess_basis* d : v) { mess_free_basis(d); delete d; } }
    } free_all{disp};
    for (int a = 0; a < na; ++a)
        for (int x = 0; x < 3; ++x)
            for (int k : ks) {
                mess_basis* d = nullptr;
                st = mess_displaced_basis(b, a, x, k * h, &d);
                if (st != MESS_OK) return st;
                disp.push_back(d);
            }
    // the differences resolve 1e-9 hartree/bohr only with FP64 energies: the displaced SCFs run in
    // FP64 whatever opts->prec
    mess_scf_opts od = o;
    od.prec = MESS_FP64;
    std::vector<mess_scf_result> rr(disp.size());
    st = mess_scf_batch((int)disp.size(), disp.data(), &od, rr.data());
    if (st != MESS_OK) return st;
    for (int a = 0; a < na; ++a)
        for (int x = 0; x < 3; ++x) {
            const mess_scf_result* e = rr.data() + 4 * (3 * a + x);
            const double g = (-e[0].E_total + 8.0 * e[1].E_total - 8.0 * e[2].E_total + e[3].E_total) / (12.0 * h);
            if (!std::isfinite(g)) { mess_set_error("mess_gradient_numerical: non-finite gradient"); return MESS_ENUMERIC; }
            grad[3 * a + x] = g;
        }
    return MESS_OK;
}

extern "C" mess_status mess_gradient(const mess_basis* bc, const mess_scf_opts* opts, mess_scf_result* res,
                                     double* grad)
{
    mess_basis* b = const_cast<mess_basis*>(bc);
    if (!b || !grad) { mess_set_error("null argument"); return MESS_EINVAL; }
    if (b->nmol != 1) { mess_set_error("mess_gradient: single-molecule bases only"); return MESS_EINVAL; }
    mess_scf_opts o{};
    if (opts) o = *opts;
    // the analytic form covers Hartree-Fock with shells up to p (the derivative of a d shell needs f
    // functions); otherwise the numerical form
    bool analytic = o.xc == 0;
    for (const HostShell& s : b->shells)
        if (s.l + 1 > MESS_LMAX) analytic = false;
    if (!analytic) return mess_gradient_numerical(bc, opts, res, grad);
    const int n = b->nbf, na = b->natom;
    std::vector<double> Dh((size_t)n * n);
    mess_scf_result r{};
    mess_status st = mess_scf(b, &o, &r, Dh.data());
    if (res) *res = r;
    if (st != MESS_OK) return st;

    mess_basis* e = nullptr;
    std::vector<int> raised, lowered;
    st = mess_derivative_basis(b, &e, raised, lowered);
    if (st != MESS_OK) return st;
    struct Free { mess_basis* e; ~Free() { mess_free_basis(e); delete e; } } free_e{e};
    const int ne = e->nbf;
    const size_t nn = (size_t)n * n, ee = (size_t)ne * ne;
    // derivative map: d m / d x = rc * (raised function) + lc * (lowered function)
    std::vector<int> fatom(n), ridx(3 * n, -1), lidx(3 * n, -1);
    std::vector<double> rcv(3 * n, 0.0), lcv(3 * n, 0.0);
    for (int k = 0; k < (int)b->shells.size(); ++k) {
        const HostShell& s = b->shells[k];
        int c = 0;
        for (int i = s.l; i >= 0; --i)
            for (int j = s.l - i; j >= 0; --j, ++c) {
                const int kk = s.l - i - j;
                const int m = s.fl + c;
                fatom[m] = s.atom;
                const int cc[3] = {i, j, kk};
                for (int x = 0; x < 3; ++x) {
                    int up[3] = {cc[0], cc[1], cc[2]};
                    up[x] += 1;
                    const HostShell& rs = e->shells[raised[k]];
                    ridx[3 * m + x] = rs.fl + comp_index(up[0], up[1], up[2]);
                    rcv[3 * m + x] = comp_scale(i, j, kk) / comp_scale(up[0], up[1], up[2]);
                    if (cc[x] > 0) {
                        int dn[3] = {cc[0], cc[1], cc[2]};
                        dn[x] -= 1;
                        const HostShell& ls = e->shells[lowered[k]];
                        lidx[3 * m + x] = ls.fl + comp_index(dn[0], dn[1], dn[2]);
                        lcv[3 * m + x] = -cc[x] * comp_scale(i, j, kk) / comp_scale(dn[0], dn[1], dn[2]);
                    }
                }
            }
    }
    DevBuf<double> dD, dW, De, Se, Te, Ve, He, Je, Ke, VA, dg, drc, dlc;
    DevBuf<int> dfatom, dridx, dlidx;
    MESS_CUDA_TRY(dD.upload(Dh));
    MESS_CUDA_TRY(dW.alloc(nn));
    for (DevBuf<double>* d : {&De, &Se, &Te, &Ve, &He, &Je, &Ke}) MESS_CUDA_TRY(d->alloc(ee));
    MESS_CUDA_TRY(VA.alloc(ee * na));
    MESS_CUDA_TRY(dg.alloc(3 * (size_t)na));
    MESS_CUDA_TRY(drc.upload(rcv));
    MESS_CUDA_TRY(dlc.upload(lcv));
    MESS_CUDA_TRY(dfatom.upload(fatom));
    MESS_CUDA_TRY(dridx.upload(ridx));
    MESS_CUDA_TRY(dlidx.upload(lidx));
    cudaStream_t s = (cudaStream_t)o.cuda_stream;
    // one-electron integrals over the extended basis: S, T, V (all nuclei), then V of each nucleus alone
    MESS_CUDA_TRY(mess_launch_one_e(e, Se.p, Te.p, Ve.p, s));
    std::vector<int> Zm(na, 0);
    for (int A = 0; A < na; ++A) {
        for (int B = 0; B < na; ++B) Zm[B] = B == A ? b->Z[A] : 0;
        MESS_CUDA_TRY(cudaMemcpyAsync(e->d_Z.p, Zm.data(), sizeof(int) * na, cudaMemcpyHostToDevice, s));
        MESS_CUDA_TRY(mess_launch_one_e(e, nullptr, nullptr, VA.p + ee * A, s));
        MESS_CUDA_TRY(cudaStreamSynchronize(s));   // Zm is reused
    }
    // J, K over the extended basis from D embedded in it (FP64, no screening)
    k_embed<<<64, 256, 0, s>>>(dD.p, n, De.p, ne);
    MESS_CUDA_TRY(cudaGetLastError());
    mess_jk_opts jo{};
    jo.prec = MESS_FP64;
    jo.cuda_stream = s;
    st = mess_jk_packed(e, De.p, Je.p, Ke.p, &jo, nullptr, false);
    if (st != MESS_OK) return st;
    k_add<<<64, 256, 0, s>>>(Te.p, Ve.p, He.p, (long long)ee);   // He = T + V over the extended basis
    MESS_CUDA_TRY(cudaGetLastError());
    k_energy_weighted<<<(unsigned)((nn + 127) / 128), 128, 0, s>>>(dD.p, He.p, Je.p, Ke.p, n, ne, dW.p);
    MESS_CUDA_TRY(cudaGetLastError());
    GradArgs g{n, ne, na, dD.p, dW.p, Se.p, He.p, Je.p, Ke.p, VA.p, dfatom.p, dridx.p, drc.p, dlidx.p, dlc.p, dg.p};
    k_grad<<<dim3(na, 3), 256, 0, s>>>(g);
    MESS_CUDA_TRY(cudaGetLastError());
    std::vector<double> gh(3 * (size_t)na);
    MESS_CUDA_TRY(cudaMemcpyAsync(gh.data(), dg.p, sizeof(double) * gh.size(), cudaMemcpyDeviceToHost, s));
    MESS_CUDA_TRY(cudaStreamSynchronize(s));
    // nuclear repulsion: d/dA sum_{B<C} Z_B Z_C / R_BC = -sum_{B != A} Z_A Z_B (R_A - R_B) / R_AB^3
    for (int A = 0; A < na; ++A)
        for (int B = 0; B < na; ++B) {
            if (B == A) continue;
            double d[3], r2 = 0.0;
            for (int x = 0; x < 3; ++x) { d[x] = b->xyz[3 * A + x] - b->xyz[3 * B + x]; r2 += d[x] * d[x]; }
            const double r3 = r2 * sqrt(r2);
            for (int x = 0; x < 3; ++x) gh[3 * A + x] -= (double)b->Z[A] * b->Z[B] * d[x] / r3;
        }
    for (size_t i = 0; i < gh.size(); ++i) {
        if (!std::isfinite(gh[i])) { mess_set_error("mess_gradient: non-finite gradient"); return MESS_ENUMERIC; }
        grad[i] = gh[i];
    }
    return MESS_OK;
}
