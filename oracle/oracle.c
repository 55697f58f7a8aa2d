/*
 * Plain FP64 CPU oracle for the Gaussian-integral, J/K and energy path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the package smoke check and the benchmark's CPU
 * baseline may load this library.  It shares no code, table or constant generator with the
 * CUDA library, and it is deliberately written for clarity, not speed.
 *
 * Method (the closed-form Gaussian integral expressions the paper cites, Taketa, Huzinaga and
 * O-ohata 1966, in the Hermite-Gaussian form of McMurchie and Davidson 1978): every integral
 * is evaluated one contracted Cartesian function at a time, one primitive at a time,
 *   - overlap     S = (pi/p)^{3/2} K_ab E^x_0 E^y_0 E^z_0                         (Sec. 3, S_mu_nu)
 *   - kinetic     T = -1/2 <a|nabla^2|b> from overlaps of shifted powers
 *   - nuclear     V = -sum_C Z_C 2 pi/p K_ab sum_tuv E_t E_u E_v R_tuv(p, P-C)
 *   - repulsion  (ab|cd) = 2 pi^{5/2}/(p q sqrt(p+q)) K_ab K_cd
 *                    sum_tuv E^ab_tuv sum_t'u'v' (-1)^{t'+u'+v'} E^cd_t'u'v' R_{t+t',u+u',v+v'}(alpha, P-Q)
 * where E are the Hermite expansion coefficients of a 1-D Gaussian product, R the Hermite
 * Coulomb integrals built from the Boys function F_n.  J and K are the plain sums
 *   J_mn = sum_ls (mn|ls) D_ls,   K_mn = sum_ls (ml|ns) D_ls
 * which the Fock matrix F = H + J - K/2 of the Hartree-Fock ("hfx") energy functional H(P) needs.
 *
 * parity: pinned (see the oracle tests: Boys closed forms, quadrature, textbook integrals).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define LMAX_FN 2           /* highest Cartesian power sum per function (d) */
#define LSUM_MAX (4 * LMAX_FN + 4)   /* room for kinetic shifts and R recursion */

/* ------------------------------------------------------------------------------------------ */
/* Boys function F_n(T) = int_0^1 t^{2n} exp(-T t^2) dt.                                        */
/* T < 50: the positive series F_n(T) = exp(-T) sum_i (2T)^i / ((2n+1)(2n+3)...(2n+2i+1)),      */
/* summed in double with Kahan compensation (every term is positive, so the compensated sum is   */
/* accurate to a few units in the last place); T >= 50: F_0 from erf and the upward recursion     */
/* F_{n+1} = ((2n+1) F_n - exp(-T)) / (2T), which is stable for large T.                          */
/* ------------------------------------------------------------------------------------------ */
void oracle_boys(int nmax, double T, double *F)
{
    if (T < 50.0) {
        double eT = exp(-T);
        for (int n = 0; n <= nmax; ++n) {
            double term = 1.0 / (double)(2 * n + 1);
            double sum = term, comp = 0.0;
            for (int i = 1; i < 4000; ++i) {
                term *= 2.0 * T / (double)(2 * n + 2 * i + 1);
                double y = term - comp;
                double t = sum + y;
                comp = (t - sum) - y;
                sum = t;
                if (term < 1e-20 * sum) break;
            }
            F[n] = eT * sum;
        }
    } else {
        double e = exp(-T);
        F[0] = 0.5 * sqrt(M_PI / T) * erf(sqrt(T));
        for (int n = 0; n < nmax; ++n) F[n + 1] = ((2 * n + 1) * F[n] - e) / (2.0 * T);
    }
}

/* ------------------------------------------------------------------------------------------ */
/* Hermite expansion coefficients E^{ij}_t of the 1-D product x_A^i x_B^j exp(-a x_A^2 - b x_B^2) */
/* (the exponential prefactor exp(-ab/p X_AB^2) is kept outside, so E^{00}_0 = 1):                */
/*   E^{i+1,j}_t = E^{ij}_{t-1}/(2p) + X_PA E^{ij}_t + (t+1) E^{ij}_{t+1}                           */
/*   E^{i,j+1}_t = E^{ij}_{t-1}/(2p) + X_PB E^{ij}_t + (t+1) E^{ij}_{t+1}                           */
/* E is filled for all i <= imax, j <= jmax, t <= i+j.                                            */
/* ------------------------------------------------------------------------------------------ */
#define EDIM 8
typedef struct { double v[EDIM][EDIM][2 * EDIM]; } etab;

static void hermite_E(int imax, int jmax, double p, double XPA, double XPB, etab *E)
{
    memset(E, 0, sizeof(*E));
    E->v[0][0][0] = 1.0;
    double h = 0.5 / p;
    for (int i = 0; i <= imax; ++i) {
        for (int j = 0; j <= jmax; ++j) {
            if (i == 0 && j == 0) continue;
            if (i > 0) {          /* raise i from (i-1, j) */
                for (int t = 0; t <= i + j; ++t) {
                    double s = XPA * E->v[i - 1][j][t];
                    if (t > 0) s += h * E->v[i - 1][j][t - 1];
                    if (t + 1 <= i - 1 + j) s += (t + 1) * E->v[i - 1][j][t + 1];
                    E->v[i][j][t] = s;
                }
            } else {              /* raise j from (0, j-1) */
                for (int t = 0; t <= j; ++t) {
                    double s = XPB * E->v[0][j - 1][t];
                    if (t > 0) s += h * E->v[0][j - 1][t - 1];
                    if (t + 1 <= j - 1) s += (t + 1) * E->v[0][j - 1][t + 1];
                    E->v[0][j][t] = s;
                }
            }
        }
    }
}

/* ------------------------------------------------------------------------------------------ */
/* Hermite Coulomb integrals R_tuv(alpha, X) for t+u+v <= L:                                      */
/*   R^n_000 = (-2 alpha)^n F_n(alpha |X|^2)                                                       */
/*   R^n_{t+1,u,v} = t R^{n+1}_{t-1,u,v} + X_x R^{n+1}_{t,u,v}   (same for u with X_y, v with X_z)  */
/* ------------------------------------------------------------------------------------------ */
#define RDIM (LSUM_MAX + 1)
typedef struct { double v[RDIM][RDIM][RDIM]; } rtab;

static void hermite_R(int L, double alpha, const double X[3], rtab *R)
{
    double T = alpha * (X[0] * X[0] + X[1] * X[1] + X[2] * X[2]);
    double F[RDIM + 1];
    oracle_boys(L, T, F);
    /* two layers: cur holds R^n, nxt holds R^{n+1}; n runs from L down to 0 */
    static __thread double layer[2][RDIM][RDIM][RDIM];
    double (*nxt)[RDIM][RDIM] = layer[0];
    double (*cur)[RDIM][RDIM] = layer[1];
    double f = 1.0;
    double R000[RDIM + 1];
    for (int n = 0; n <= L; ++n) { R000[n] = f * F[n]; f *= -2.0 * alpha; }
    for (int n = L; n >= 0; --n) {
        int top = L - n;
        for (int t = 0; t <= top; ++t)
            for (int u = 0; u + t <= top; ++u)
                for (int v = 0; v + u + t <= top; ++v) {
                    double r;
                    if (t == 0 && u == 0 && v == 0) r = R000[n];
                    else if (t > 0) r = (t > 1 ? (t - 1) * nxt[t - 2][u][v] : 0.0) + X[0] * nxt[t - 1][u][v];
                    else if (u > 0) r = (u > 1 ? (u - 1) * nxt[t][u - 2][v] : 0.0) + X[1] * nxt[t][u - 1][v];
                    else            r = (v > 1 ? (v - 1) * nxt[t][u][v - 2] : 0.0) + X[2] * nxt[t][u][v - 1];
                    cur[t][u][v] = r;
                }
        double (*tmp)[RDIM][RDIM] = nxt; nxt = cur; cur = tmp;
    }
    /* after the last swap nxt holds R^0 */
    for (int t = 0; t <= L; ++t)
        for (int u = 0; u + t <= L; ++u)
            for (int v = 0; v + u + t <= L; ++v)
                R->v[t][u][v] = nxt[t][u][v];
}

/* ------------------------------------------------------------------------------------------ */
/* Basis functions as handed in by the Python side: one contracted Cartesian function each.   */
/* ------------------------------------------------------------------------------------------ */
typedef struct {
    int nfn;
    const double *center;   /* [nfn][3] */
    const int *lmn;         /* [nfn][3] */
    const int *nprim;       /* [nfn] */
    const int *poff;        /* [nfn] offset into exps/coefs */
    const double *exps;
    const double *coefs;    /* contraction coefficient x primitive norm x contraction norm */
} fnset;

static void mkset(fnset *s, int nfn, const double *c, const int *lmn, const int *np,
                  const int *po, const double *ex, const double *co)
{
    s->nfn = nfn; s->center = c; s->lmn = lmn; s->nprim = np; s->poff = po; s->exps = ex; s->coefs = co;
}

/* primitive pair: exponent sum, centre P, prefactor exp(-ab/p |AB|^2) and its E tables */
typedef struct { double p, P[3], K; etab E[3]; } ppair;

static void make_ppair(double a, const double *A, int ia[3], double b, const double *B, int ib[3],
                       int extra_j, ppair *pp)
{
    double p = a + b, mu = a * b / p, ab2 = 0.0;
    pp->p = p;
    for (int x = 0; x < 3; ++x) {
        pp->P[x] = (a * A[x] + b * B[x]) / p;
        ab2 += (A[x] - B[x]) * (A[x] - B[x]);
    }
    pp->K = exp(-mu * ab2);
    for (int x = 0; x < 3; ++x)
        hermite_E(ia[x], ib[x] + extra_j, p, pp->P[x] - A[x], pp->P[x] - B[x], &pp->E[x]);
}

/* ---------------------------------- one-electron integrals ---------------------------------- */
static double prim_overlap(const ppair *pp, const int ia[3], const int ib[3])
{
    double s = pow(M_PI / pp->p, 1.5) * pp->K;
    for (int x = 0; x < 3; ++x) s *= pp->E[x].v[ia[x]][ib[x]][0];
    return s;
}

/* 1-D overlap of x^i and x^j (without the exponential prefactor) */
static double s1d(const ppair *pp, int x, int i, int j)
{
    if (j < 0) return 0.0;
    return pp->E[x].v[i][j][0] * sqrt(M_PI / pp->p);
}

static double prim_kinetic(const ppair *pp, double b, const int ia[3], const int ib[3])
{
    double S[3], Tk[3];
    for (int x = 0; x < 3; ++x) {
        int i = ia[x], j = ib[x];
        S[x] = s1d(pp, x, i, j);
        /* -1/2 d^2/dx^2 acting on x^j exp(-b x^2) */
        Tk[x] = -0.5 * (j * (j - 1) * s1d(pp, x, i, j - 2) - 2.0 * b * (2 * j + 1) * s1d(pp, x, i, j)
                        + 4.0 * b * b * s1d(pp, x, i, j + 2));
    }
    return pp->K * (Tk[0] * S[1] * S[2] + S[0] * Tk[1] * S[2] + S[0] * S[1] * Tk[2]);
}

static double prim_nuclear(const ppair *pp, const int ia[3], const int ib[3], int natom,
                           const int *Z, const double *xyz)
{
    int L = ia[0] + ib[0] + ia[1] + ib[1] + ia[2] + ib[2];
    double total = 0.0;
    rtab R;
    for (int c = 0; c < natom; ++c) {
        double X[3] = {pp->P[0] - xyz[3 * c], pp->P[1] - xyz[3 * c + 1], pp->P[2] - xyz[3 * c + 2]};
        hermite_R(L, pp->p, X, &R);
        double s = 0.0;
        for (int t = 0; t <= ia[0] + ib[0]; ++t)
            for (int u = 0; u <= ia[1] + ib[1]; ++u)
                for (int v = 0; v <= ia[2] + ib[2]; ++v)
                    s += pp->E[0].v[ia[0]][ib[0]][t] * pp->E[1].v[ia[1]][ib[1]][u]
                         * pp->E[2].v[ia[2]][ib[2]][v] * R.v[t][u][v];
        total += -Z[c] * 2.0 * M_PI / pp->p * pp->K * s;
    }
    return total;
}

/* S, T, V for every function pair (full n x n, row-major). */
void oracle_one_e(int nfn, const double *center, const int *lmn, const int *nprim, const int *poff,
                  const double *exps, const double *coefs, int natom, const int *Z, const double *xyz,
                  double *S, double *T, double *V)
{
    fnset f;
    mkset(&f, nfn, center, lmn, nprim, poff, exps, coefs);
#pragma omp parallel for schedule(dynamic)
    for (int m = 0; m < nfn; ++m) {
        for (int n = 0; n < nfn; ++n) {
            int ia[3] = {f.lmn[3 * m], f.lmn[3 * m + 1], f.lmn[3 * m + 2]};
            int ib[3] = {f.lmn[3 * n], f.lmn[3 * n + 1], f.lmn[3 * n + 2]};
            double s = 0.0, t = 0.0, v = 0.0;
            for (int i = 0; i < f.nprim[m]; ++i) {
                for (int j = 0; j < f.nprim[n]; ++j) {
                    double a = f.exps[f.poff[m] + i], b = f.exps[f.poff[n] + j];
                    double c = f.coefs[f.poff[m] + i] * f.coefs[f.poff[n] + j];
                    ppair pp;
                    make_ppair(a, &f.center[3 * m], ia, b, &f.center[3 * n], ib, 2, &pp);
                    s += c * prim_overlap(&pp, ia, ib);
                    t += c * prim_kinetic(&pp, b, ia, ib);
                    v += c * prim_nuclear(&pp, ia, ib, natom, Z, xyz);
                }
            }
            if (S) S[m * nfn + n] = s;
            if (T) T[m * nfn + n] = t;
            if (V) V[m * nfn + n] = v;
        }
    }
}

/* ------------------------------- electron repulsion integrals ------------------------------- */
static double eri_fn(const fnset *f, int m, int n, int l, int s)
{
    int ia[3], ib[3], ic[3], id[3];
    for (int x = 0; x < 3; ++x) {
        ia[x] = f->lmn[3 * m + x]; ib[x] = f->lmn[3 * n + x];
        ic[x] = f->lmn[3 * l + x]; id[x] = f->lmn[3 * s + x];
    }
    int Lab[3], Lcd[3], L = 0;
    for (int x = 0; x < 3; ++x) { Lab[x] = ia[x] + ib[x]; Lcd[x] = ic[x] + id[x]; L += Lab[x] + Lcd[x]; }
    const double pi52 = 2.0 * pow(M_PI, 2.5);
    double total = 0.0;
    for (int i = 0; i < f->nprim[m]; ++i)
    for (int j = 0; j < f->nprim[n]; ++j) {
        ppair bra;
        make_ppair(f->exps[f->poff[m] + i], &f->center[3 * m], ia,
                   f->exps[f->poff[n] + j], &f->center[3 * n], ib, 0, &bra);
        double cab = f->coefs[f->poff[m] + i] * f->coefs[f->poff[n] + j];
        for (int k = 0; k < f->nprim[l]; ++k)
        for (int q = 0; q < f->nprim[s]; ++q) {
            ppair ket;
            make_ppair(f->exps[f->poff[l] + k], &f->center[3 * l], ic,
                       f->exps[f->poff[s] + q], &f->center[3 * s], id, 0, &ket);
            double ccd = f->coefs[f->poff[l] + k] * f->coefs[f->poff[s] + q];
            double p = bra.p, qq = ket.p, alpha = p * qq / (p + qq);
            double X[3] = {bra.P[0] - ket.P[0], bra.P[1] - ket.P[1], bra.P[2] - ket.P[2]};
            rtab R;
            hermite_R(L, alpha, X, &R);
            double sum = 0.0;
            for (int t = 0; t <= Lab[0]; ++t)
            for (int u = 0; u <= Lab[1]; ++u)
            for (int v = 0; v <= Lab[2]; ++v) {
                double eab = bra.E[0].v[ia[0]][ib[0]][t] * bra.E[1].v[ia[1]][ib[1]][u]
                             * bra.E[2].v[ia[2]][ib[2]][v];
                if (eab == 0.0) continue;
                double inner = 0.0;
                for (int tt = 0; tt <= Lcd[0]; ++tt)
                for (int uu = 0; uu <= Lcd[1]; ++uu)
                for (int vv = 0; vv <= Lcd[2]; ++vv) {
                    double ecd = ket.E[0].v[ic[0]][id[0]][tt] * ket.E[1].v[ic[1]][id[1]][uu]
                                 * ket.E[2].v[ic[2]][id[2]][vv];
                    double sign = ((tt + uu + vv) & 1) ? -1.0 : 1.0;
                    inner += sign * ecd * R.v[t + tt][u + uu][v + vv];
                }
                sum += eab * inner;
            }
            total += cab * ccd * pi52 / (p * qq * sqrt(p + qq)) * bra.K * ket.K * sum;
        }
    }
    return total;
}

/* one contracted integral (mn|ls) */
double oracle_eri(int nfn, const double *center, const int *lmn, const int *nprim, const int *poff,
                  const double *exps, const double *coefs, int m, int n, int l, int s)
{
    fnset f;
    mkset(&f, nfn, center, lmn, nprim, poff, exps, coefs);
    return eri_fn(&f, m, n, l, s);
}

/* full n^4 tensor, no symmetry used (small cases only) */
void oracle_eri_tensor(int nfn, const double *center, const int *lmn, const int *nprim,
                       const int *poff, const double *exps, const double *coefs, double *out)
{
    fnset f;
    mkset(&f, nfn, center, lmn, nprim, poff, exps, coefs);
    long n = nfn;
#pragma omp parallel for collapse(2) schedule(dynamic)
    for (int m = 0; m < nfn; ++m)
        for (int a = 0; a < nfn; ++a)
            for (int l = 0; l < nfn; ++l)
                for (int s = 0; s < nfn; ++s)
                    out[((m * n + a) * n + l) * n + s] = eri_fn(&f, m, a, l, s);
}

/* Schwarz factor per shell pair: Q_AB = sqrt(max_{m in A, n in B} |(mn|mn)|).
 * shell[] gives the shell index of each function; Q is nshell x nshell. */
void oracle_schwarz(int nfn, const double *center, const int *lmn, const int *nprim,
                    const int *poff, const double *exps, const double *coefs,
                    const int *shell, int nshell, double *Q)
{
    fnset f;
    mkset(&f, nfn, center, lmn, nprim, poff, exps, coefs);
    for (int i = 0; i < nshell * nshell; ++i) Q[i] = 0.0;
    double *diag = (double *)malloc(sizeof(double) * (size_t)nfn * nfn);
#pragma omp parallel for collapse(2) schedule(dynamic)
    for (int m = 0; m < nfn; ++m)
        for (int n = 0; n < nfn; ++n)
            diag[m * nfn + n] = fabs(eri_fn(&f, m, n, m, n));
    for (int m = 0; m < nfn; ++m)
        for (int n = 0; n < nfn; ++n) {
            int A = shell[m], B = shell[n];
            double q = sqrt(diag[m * nfn + n]);
            if (q > Q[A * nshell + B]) Q[A * nshell + B] = q;
        }
    free(diag);
}

static int keep_quartet(const int *shell, int nshell, const double *Q, double tau, int m, int n,
                        int l, int s)
{
    if (tau <= 0.0 || !Q) return 1;
    double qab = Q[shell[m] * nshell + shell[n]], qcd = Q[shell[l] * nshell + shell[s]];
    return qab * qcd >= tau;
}

/* J and K by the definition, every (m, n, l, s) visited: J_mn = sum (mn|ls) D_ls, K_mn = sum (ml|ns) D_ls.
 * Quartets whose shell quartet fails Q_ab Q_cd >= tau are dropped (tau <= 0: nothing dropped). */
void oracle_jk_brute(int nfn, const double *center, const int *lmn, const int *nprim,
                     const int *poff, const double *exps, const double *coefs,
                     const int *shell, int nshell, const double *Q, double tau,
                     const double *D, double *J, double *K)
{
    fnset f;
    mkset(&f, nfn, center, lmn, nprim, poff, exps, coefs);
    int n = nfn;
#pragma omp parallel for schedule(dynamic)
    for (int m = 0; m < n; ++m) {
        for (int a = 0; a < n; ++a) {
            double j = 0.0, k = 0.0;
            for (int l = 0; l < n; ++l)
                for (int s = 0; s < n; ++s) {
                    if (keep_quartet(shell, nshell, Q, tau, m, a, l, s))
                        j += eri_fn(&f, m, a, l, s) * D[l * n + s];
                    if (keep_quartet(shell, nshell, Q, tau, m, l, a, s))
                        k += eri_fn(&f, m, l, a, s) * D[l * n + s];
                }
            J[m * n + a] = j;
            K[m * n + a] = k;
        }
    }
}

/* J and K from the unique quartets m>=n, l>=s, (mn)>=(ls): every distinct index permutation of a
 * unique quartet under the 8-fold symmetry (mn|ls)=(nm|ls)=(mn|sl)=(ls|mn)=... is added once. */
void oracle_jk_sym(int nfn, const double *center, const int *lmn, const int *nprim,
                   const int *poff, const double *exps, const double *coefs,
                   const int *shell, int nshell, const double *Q, double tau,
                   const double *D, double *J, double *K)
{
    fnset f;
    mkset(&f, nfn, center, lmn, nprim, poff, exps, coefs);
    int n = nfn;
    size_t nn = (size_t)n * n;
    memset(J, 0, sizeof(double) * nn);
    memset(K, 0, sizeof(double) * nn);
#pragma omp parallel
    {
        double *Jt = (double *)calloc(nn, sizeof(double));
        double *Kt = (double *)calloc(nn, sizeof(double));
#pragma omp for schedule(dynamic)
        for (int m = 0; m < n; ++m)
            for (int a = 0; a <= m; ++a) {
                int mn = m * (m + 1) / 2 + a;
                for (int l = 0; l < n; ++l)
                    for (int s = 0; s <= l; ++s) {
                        int ls = l * (l + 1) / 2 + s;
                        if (ls > mn) continue;
                        if (!keep_quartet(shell, nshell, Q, tau, m, a, l, s)) continue;
                        double v = eri_fn(&f, m, a, l, s);
                        int perm[8][4] = {{m, a, l, s}, {a, m, l, s}, {m, a, s, l}, {a, m, s, l},
                                          {l, s, m, a}, {s, l, m, a}, {l, s, a, m}, {s, l, a, m}};
                        for (int i = 0; i < 8; ++i) {
                            int dup = 0;
                            for (int k2 = 0; k2 < i; ++k2)
                                if (perm[k2][0] == perm[i][0] && perm[k2][1] == perm[i][1] &&
                                    perm[k2][2] == perm[i][2] && perm[k2][3] == perm[i][3]) dup = 1;
                            if (dup) continue;
                            int p0 = perm[i][0], p1 = perm[i][1], p2 = perm[i][2], p3 = perm[i][3];
                            Jt[p0 * n + p1] += v * D[p2 * n + p3];
                            Kt[p0 * n + p2] += v * D[p1 * n + p3];
                        }
                    }
            }
#pragma omp critical
        {
            for (size_t i = 0; i < nn; ++i) { J[i] += Jt[i]; K[i] += Kt[i]; }
        }
        free(Jt);
        free(Kt);
    }
}

/* Selected elements J_mn and K_mn by the definition (for spot checks of large cases). */
void oracle_jk_elements(int nfn, const double *center, const int *lmn, const int *nprim,
                        const int *poff, const double *exps, const double *coefs,
                        const int *shell, int nshell, const double *Q, double tau,
                        const double *D, int nsel, const int *rows, const int *cols,
                        double *Jsel, double *Ksel)
{
    fnset f;
    mkset(&f, nfn, center, lmn, nprim, poff, exps, coefs);
    int n = nfn;
#pragma omp parallel for schedule(dynamic)
    for (int e = 0; e < nsel; ++e) {
        int m = rows[e], a = cols[e];
        double j = 0.0, k = 0.0;
        for (int l = 0; l < n; ++l)
            for (int s = 0; s < n; ++s) {
                if (keep_quartet(shell, nshell, Q, tau, m, a, l, s))
                    j += eri_fn(&f, m, a, l, s) * D[l * n + s];
                if (keep_quartet(shell, nshell, Q, tau, m, l, a, s))
                    k += eri_fn(&f, m, l, a, s) * D[l * n + s];
            }
        Jsel[e] = j;
        Ksel[e] = k;
    }
}

/* Threads of the OpenMP loops (n <= 0: the runtime's default).  Scheduling only: the sums of
 * every loop above are the same whatever the thread count. */
void oracle_set_num_threads(int n)
{
#ifdef _OPENMP
    if (n <= 0) n = omp_get_num_procs();
    omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int oracle_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
