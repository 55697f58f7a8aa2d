/*
 * mess.h - C ABI of the GB300 Gaussian-basis Hartree-Fock hot path.
 *
 * The calls follow the problem statement of MESS (Helal & Fitzgibbon, arXiv 2406.03121):
 *   Structure(Z, positions) -> basisset(mol, name) -> one-electron integrals, the Coulomb / exchange
 *   contraction of the repulsion integrals with a density, the energy functional H(P) +
 *   nuclear_energy, and the self-consistent-field solution of the Roothaan equation.
 *
 * Conventions (all calls):
 *   - Units: bohr and hartree.  Atomic numbers are ints; coordinates natom x 3 row-major doubles.
 *   - Basis functions are contracted Cartesian Gaussians (paper Sec. 3, Eq. 1): per atom in input
 *     order, per shell in basis-file order, per Cartesian component in the order
 *     x^l y^m z^n with l descending then m descending (p: x y z; d: xx xy xz yy yz zz).  Every
 *     function is normalised on its own (S_mm = 1).  n = mess_basis_nbf().
 *   - Matrices are n x n row-major doubles.  D is the total closed-shell density 2 C_occ C_occ^T.
 *   - J_mn = sum_ls (mn|ls) D_ls and K_mn = sum_ls (ml|ns) D_ls (Hartree-Fock exchange, the
 *     paper's xc_method="hfx"); the Fock matrix is F = H + J - K/2 and the electronic energy
 *     E_elec = 1/2 sum D (H + F) (the paper's H(P), Sec. 5.1).
 *   - Ownership: every output buffer is caller-owned.  mess_basis is library-owned (create/destroy).
 *     Host-buffer calls copy through internal device buffers and synchronise before returning.
 *   - Errors: every call returns a mess_status; no exception crosses the ABI.  mess_last_error()
 *     returns a message for the calling thread's most recent failure.
 *   - Threads: calls on distinct bases are independent.  A mess_basis may be shared by calls that do
 *     not overlap in time on the host (it caches screening bins); device-pointer calls on the same
 *     basis may overlap on the GPU (their builds take turns with the basis's reduced-precision
 *     density copies).
 *   - Environment: MESS_JK_STREAMS (8..64, default 16), read once per device, sets how many
 *     streams the parts of one J/K build are spread over.
 */
#ifndef MESS_H
#define MESS_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mess_basis mess_basis; /* opaque, library-owned */

typedef enum {
    MESS_OK = 0,
    MESS_EINVAL = -1,     /* bad argument (null pointer, size, unknown element, malformed file) */
    MESS_ENOMEM = -2,     /* device or host allocation failed */
    MESS_ECUDA = -3,      /* CUDA runtime error (message in mess_last_error) */
    MESS_ENOCONV = -4,    /* SCF did not converge within max_iter (result holds the last iterate) */
    MESS_ENUMERIC = -5,   /* non-finite value detected */
    MESS_ETIMEOUT = -6,   /* a bounded device wait gave up */
    MESS_ENOTIMPL = -7    /* feature not available */
} mess_status;

typedef enum {
    MESS_FP64 = 0,  /* all recursion arithmetic in FP64 */
    MESS_MIXED = 1, /* FP32 recursion and FP32 per-quartet digestion; the shell quartets with
                       Q_ab Q_cd >= fp64_tau (the largest integrals) in FP64; FP64 J/K accumulation */
    MESS_FP32 = 2   /* FP32 recursion for every quartet; FP64 J/K accumulation */
} mess_precision;

/* Default MESS_MIXED split: quartets with Q_ab Q_cd >= 3e-2 run in FP64. */
#define MESS_DEFAULT_FP64_TAU 3e-2

/* J/K build options.  Zero-initialised opts mean FP64, no screening, default stream. */
typedef struct {
    mess_precision prec;
    double schwarz_tau; /* drop shell quartets with Q_ab Q_cd < schwarz_tau (0: keep all) */
    double fp64_tau;    /* MESS_MIXED: quartets with Q_ab Q_cd >= fp64_tau run in FP64;
                           0 selects MESS_DEFAULT_FP64_TAU, < 0 runs every quartet in FP32 */
    int boys_fp64;      /* MESS_MIXED / MESS_FP32: 1 evaluates the Boys function of the FP32 quartets
                           in FP64 for T < 36 (Taylor grid + downward recursion), 0 in FP32 */
    int split_df32;     /* MESS_MIXED: 1 evaluates the quartets above fp64_tau in double-float
                           arithmetic (pairs of FP32 values, about 48 bits, on the FP32 units: on this
                           GPU several times faster than FP64) instead of FP64; 0 in FP64 */
    void* cuda_stream;  /* cudaStream_t for the device-pointer calls (NULL: default stream) */
} mess_jk_opts;

/* Work done by one J/K build (after screening). */
typedef struct {
    long long shell_quartets;        /* unique shell quartets evaluated */
    long long function_quartets;     /* unique Cartesian function quartets evaluated */
    long long shell_quartets_fp64;   /* of which evaluated in FP64 */
    long long primitive_quartets;    /* primitive quartets evaluated */
    long long kernel_launches;       /* kernels launched by the call */
} mess_jk_info;

/* Initial density of the SCF: eigenvectors of the core Hamiltonian; superposition of spherically
 * averaged atomic densities (an SCF of each element's atom with fractional 2p occupation); or the
 * learned guess (mess_mlp_* below).  The converged energy does not depend on the choice. */
typedef enum { MESS_GUESS_CORE = 0, MESS_GUESS_SAD = 1, MESS_GUESS_MLP = 2 } mess_guess;

typedef struct {
    mess_precision prec;  /* precision of the J/K builds */
    int guess;            /* mess_guess */
    int max_iter;         /* default 100 when <= 0 */
    double conv_E;        /* |dE| threshold, default 1e-10 when <= 0 */
    double conv_comm;     /* max|FDS - SDF| threshold, default 1e-8 when <= 0 */
    int diis_n;           /* DIIS subspace size, default 8 when <= 0 */
    double schwarz_tau;   /* screening threshold for the J/K builds */
    double fp64_tau;      /* MESS_MIXED split, see mess_jk_opts */
    int boys_fp64;        /* see mess_jk_opts */
    int split_df32;       /* see mess_jk_opts */
    const char* mlp_weights; /* MESS_GUESS_MLP: weight file of mess_mlp_save (unused otherwise) */
    void* cuda_stream;
    double dens_tau;      /* density-weighted screening of the incremental Fock builds: a shell quartet is
                             skipped when Q_ab Q_cd times the largest change of the density in the rows of
                             its shells is below dens_tau (0: off, the default).  Each skipped contribution
                             is below dens_tau, but they change from one iteration to the next: values
                             above about 1e-13 can hold the commutator above conv_comm */
    int xc;               /* energy functional: 0 Hartree-Fock (xc_method "hfx"), 1 LDA (Slater exchange +
                             Perdew-Wang 1992 correlation), 2 PBE; see mess_xc for the grid */
} mess_scf_opts;

typedef struct {
    double E_total, E_elec, E_nuc;
    int iterations, converged;
    double E_iter;   /* total energy of the last iteration's own J/K build: with MESS_MIXED / MESS_FP32
                        the reduced-precision energy, before the final full-precision evaluation that
                        sets E_total; with MESS_FP64 equal to E_total */
} mess_scf_result;

/* Build the contracted Cartesian basis of a structure (paper Sec. 3 LCAO basis; Sec. 5.1 basisset)
 * from a basis data file: "element <sym>" lines followed by shells "<S|P|D|SP> <nprim>" and nprim
 * lines "exponent coefficient(s)".  Computes on the GPU the primitive-pair tables (Gaussian product
 * theorem) and the Schwarz factors Q_ab = sqrt(max |(mn|mn)|) of every shell pair - on the first call
 * that computes on this basis alone (a basis used only inside batches never builds its own), so CUDA
 * errors of that step are reported by that call.
 * Z: natom ints; xyz_bohr: natom*3 doubles.  *out receives a new basis (free with mess_basis_destroy).
 * Errors: MESS_EINVAL (unknown element, unreadable or malformed file, natom <= 0), MESS_ENOMEM,
 * MESS_ECUDA. */
mess_status mess_basis_create(int natom, const int* Z, const double* xyz_bohr, const char* basis_file,
                              mess_basis** out);
int mess_basis_nbf(const mess_basis* b);      /* number of basis functions n (-1 if b is NULL) */
int mess_basis_nshell(const mess_basis* b);   /* number of shells */
int mess_basis_nelectron(const mess_basis* b);/* sum of Z */
void mess_basis_destroy(mess_basis* b);       /* NULL is accepted */

/* Overlap S_mn = <phi_m|phi_n> (paper Eq. 3), kinetic T_mn = <phi_m|-1/2 nabla^2|phi_n>, nuclear
 * attraction V_mn = -sum_C Z_C <phi_m|1/|r-C||phi_n> (the "closed-form expressions for all the
 * relevant integrals", Sec. 3).  Output: caller-owned host n*n doubles. */
mess_status mess_overlap(const mess_basis* b, double* S);
mess_status mess_kinetic(const mess_basis* b, double* T);
mess_status mess_nuclear(const mess_basis* b, double* V);
/* The same three on device pointers (each n*n doubles, any may be NULL), on cuda_stream. */
mess_status mess_one_e_device(const mess_basis* b, double* dS, double* dT, double* dV, void* cuda_stream);

/* sum_{A<B} Z_A Z_B / R_AB (the paper's nuclear_energy, Sec. 5.1).  NaN if b is NULL. */
double mess_nuclear_repulsion(const mess_basis* b);

/* Integral-direct Coulomb and exchange matrices of a symmetric density (Sec. 3 / 5.1 "hfx"):
 * J_mn = sum_ls (mn|ls) D_ls, K_mn = sum_ls (ml|ns) D_ls, over the unique shell quartets that pass
 * Schwarz screening, with the 8-fold permutational symmetry.  D, J, K: host n*n doubles
 * (caller-owned).  opts may be NULL (FP64, no screening).  info may be NULL.  The first call on a
 * basis allocates a device staging buffer of 3 n^2 doubles kept with the basis (freed by
 * mess_basis_destroy); the call synchronises opts->cuda_stream before returning.
 * Errors: MESS_EINVAL, MESS_ENOMEM, MESS_ECUDA. */
mess_status mess_jk_build(const mess_basis* b, const double* D, double* J, double* K,
                          const mess_jk_opts* opts, mess_jk_info* info);
/* Same on caller-owned device buffers (n*n doubles each), enqueued on opts->cuda_stream; returns
 * after enqueueing (no synchronisation).  dD must not alias dJ or dK. */
mess_status mess_jk_build_device(const mess_basis* b, const double* dD, double* dJ, double* dK,
                                 const mess_jk_opts* opts, mess_jk_info* info);

/* mess_jk_build without any device allocation (the paper has no counterpart: this is a library
 * service).  For callers that cannot let a library call cudaMalloc / cudaFree: programs whose
 * device memory belongs to their own pool or arena, latency-critical loops that cannot absorb
 * cudaFree's implicit synchronisation, processes running with the device already full.  D, J, K
 * are staged in one fixed device array inside the library (3 x 256 x 256 doubles, 1.5 MiB per GPU,
 * held until the process exits) instead of freshly allocated buffers; results equal mess_jk_build's.
 * Limits: single-molecule bases with n <= 256 (larger n: MESS_EINVAL with a message); the quartet
 * bins for these opts must already exist - a prior mess_jk_build / mess_jk_build_device call with
 * the same opts builds them, otherwise MESS_EINVAL (invalid opts: MESS_EINVAL with their own message).
 * That prior allocating call also creates, with the bins, the basis's FP32 / double-float copies of
 * the density that MESS_MIXED and MESS_FP32 builds read; this call reuses them and allocates none.
 * A mess_scf on the same basis changes which molecules the bins cover and so invalidates them: the
 * next static call returns MESS_EINVAL until another allocating build with these opts has run.
 * Every return after the first copy has been enqueued (errors included) synchronises
 * opts->cuda_stream first, so the array is free when the call returns.  The first call on each device looks up the
 * array's device address (cudaGetSymbolAddress, with that device current), so make that first call
 * before any stream capture.  All calls share the array and it keeps the last call's contents:
 * calls that overlap on the GPU race on it - serialise them. */
mess_status mess_jk_build_static(const mess_basis* b, const double* D, double* J, double* K,
                                 const mess_jk_opts* opts, mess_jk_info* info);

/* Every repulsion integral (mn|ls) in FP64 as a dense n^4 host tensor (index ((m*n+n')*n+l)*n+s).
 * For small bases only (n <= 64).  Errors: MESS_EINVAL (n > 64), MESS_ENOMEM, MESS_ECUDA. */
mess_status mess_eri_tensor(const mess_basis* b, double* G);

/* Schwarz factor of every shell pair as an nshell x nshell host matrix (symmetric). */
mess_status mess_schwarz(const mess_basis* b, double* Q);

/* Exchange-correlation energy and matrix of a density on the library's molecular grid (paper Sec. 5.1,
 * xc_method "lda" / "pbe"; Kohn-Sham 1965).  Grid per atom: radial Gauss-Chebyshev (second kind) mapped
 * by r = R (1 + x) / (1 - x) (R = 0.35 angstrom for H, half the Bragg-Slater radius otherwise: C 0.35,
 * N 0.325, O 0.30), 50 points for H and 75 otherwise, times 16 Gauss-Legendre cos(theta) x 32 phi;
 * Becke's fuzzy-cell partition between atoms.  xc: 1 LDA (Slater exchange, Perdew-Wang 1992
 * correlation), 2 PBE.  D: host n x n (closed-shell total density); Exc (nullable): E_xc; V (nullable):
 * host n x n, V_mn = dE_xc/dD_mn = sum_g w_g [v_rho phi_m phi_n + 2 v_sigma grad rho . grad(phi_m phi_n)];
 * npts (nullable): grid points.  The grid and the basis functions' values are built on the first call
 * and kept with the basis.  Errors: MESS_EINVAL, MESS_ENOMEM, MESS_ECUDA. */
mess_status mess_xc(const mess_basis* b, int xc, const double* D, double* Exc, double* V, long long* npts);

/* Closed-shell Roothaan SCF (paper Eq. 2, Sec. 3): Loewdin orthogonalisation, core-Hamiltonian
 * guess, Pulay DIIS on FDS - SDF, converged when |dE| < conv_E and max|FDS - SDF| < conv_comm.
 * Runs entirely on the GPU: one-electron integrals, Loewdin X (Jacobi eigensolver), the J/K builds of
 * mess_jk_build_device with opts->prec / schwarz_tau / fp64_tau, F = H + J - K/2, DIIS, the
 * diagonalisation of X^T F X (one thread block per molecule, cyclic Jacobi: FP64 for MESS_FP64,
 * double-float - about 48 significant bits, on the FP32 units - for MESS_MIXED / MESS_FP32) and
 * D = 2 C_occ C_occ^T; the overlap matrix of X in the same arithmetic.
 * With prec MESS_MIXED / MESS_FP32 the iterations use the reduced-precision builds and the reported
 * energy E_total is that of the final density from one full build in which the quartets above a ten
 * times lower split threshold (MESS_MIXED; every quartet for MESS_FP32) run in double-float
 * (split_df32) or FP64: most of the integrals' rounding leaves the energy, and the density's residual
 * error enters it only at second order.  E_iter is the iterations' own energy.
 * With opts->xc = 1 or 2 it is the Kohn-Sham SCF of that functional: F = H + J + V_xc and E_elec =
 * tr(D H) + 1/2 tr(D J) + E_xc (the exchange matrix K is not used).
 * D_out (nullable): host n*n final density.  Errors: MESS_ENOCONV (res holds the last iterate),
 * MESS_EINVAL (odd electron count, MESS_GUESS_MLP without weights), MESS_ENOTIMPL (n > 256),
 * MESS_ENOMEM, MESS_ECUDA, MESS_ENUMERIC (singular overlap, non-finite energy). */
mess_status mess_scf(const mess_basis* b, const mess_scf_opts* opts, mess_scf_result* res, double* D_out);

/* Nuclear gradient dE/dR of the closed-shell Hartree-Fock energy at the SCF solution (the paper
 * differentiates E(P) + nuclear_energy automatically, Secs. 1 and 4; here the analytic expression):
 * runs mess_scf with opts (prec as there; the derivative integrals are FP64), then
 *   dE/dA_x = sum_{m on A, n} [2 D_mn (dm|h|n) + D_mn (2 J'_mn - K'_mn) - 2 W_mn (dm|n)]
 *             - 2 sum_{m,n} D_mn (dm|V_A|n) + dE_nuc/dA_x,
 * dm the derivative of basis function m with respect to its own centre, J'_mn = sum_ls (dm n|l s) D_ls,
 * K'_mn = sum_ls (dm l|n s) D_ls, W = D F D / 2, V_A the attraction of nucleus A.  That analytic form
 * covers single-molecule bases with shells up to p (STO-3G, 6-31G) and xc = 0.  For bases with d
 * shells (whose derivatives need f functions) or xc != 0 this call returns the numerical form of
 * mess_gradient_numerical instead.  grad: natom x 3 doubles (hartree/bohr); res (nullable): the SCF
 * result.  Errors: as mess_scf; MESS_EINVAL (batch bases). */
mess_status mess_gradient(const mess_basis* b, const mess_scf_opts* opts, mess_scf_result* res, double* grad);

/* Nuclear gradient as the derivative of the SCF energy taken numerically (the paper differentiates
 * the energy, Secs. 1 and 4): runs mess_scf with opts for res, then one batched SCF (mess_scf_batch,
 * the paper's batching over conformations, Sec. 5.2) of the 12 natom geometries with one atom moved
 * by k h along one axis, k = 2, 1, -1, -2, h = 1e-3 bohr, in FP64 whatever opts->prec (the other
 * options as given: converge tightly, e.g. conv_E 1e-12 and conv_comm 1e-10, for gradients good to
 * 1e-8), and the fourth-order central difference
 *   dE/dR = [-E(R + 2h) + 8 E(R + h) - 8 E(R - h) + E(R - 2h)] / (12 h)
 * (truncation error of order h^4).  Any shells, Hartree-Fock or Kohn-Sham (opts->xc).  Single-molecule
 * bases of at most 256 functions.  grad: natom x 3 doubles (hartree/bohr); res (nullable): the SCF
 * result at R.  Errors: as mess_scf and mess_scf_batch; MESS_EINVAL (batch bases). */
mess_status mess_gradient_numerical(const mess_basis* b, const mess_scf_opts* opts, mess_scf_result* res,
                                    double* grad);

/* Batched SCF over many molecules (the paper's vmap over conformers, Sec. 5.2): every molecule of
 * bases[0..nmol) (single-molecule bases, any sizes) in the same kernel launches - the J/K kernels
 * take quartets of all molecules from one set of bins; Fock, DIIS, Jacobi and the density run one
 * block per molecule; converged molecules drop out.  res: nmol entries (caller-owned).
 * Errors: as mess_scf; MESS_ENOCONV if any molecule did not converge. */
mess_status mess_scf_batch(int nmol, mess_basis* const* bases, const mess_scf_opts* opts, mess_scf_result* res);

/* Direct minimisation of the energy functional (paper Sec. 3: E(C) minimised subject to the
 * orthonormality C^T S C = 1, Eqs. 4-5; Sec. 5.1 and 5.2: first-order optimisation with Adam, the
 * constraint built in by a QR decomposition).  Per molecule the unconstrained parameters are an n x n
 * matrix Z, starting from the identity: Z = Q R (Householder), C = X Q with X = S^-1/2, D =
 * 2 C_occ C_occ^T, E(Z) = 1/2 sum D (H + F) + E_nuc with F = H + J(D) - K(D)/2 from the J/K build
 * (prec, schwarz_tau, fp64_tau, boys_fp64, split_df32 as in mess_jk_opts), and dE/dZ = Q
 * tril(Q^T G - G^T Q, -1) R^-T with G = X (4 F C_occ | 0).  Adam: m = b1 m + (1 - b1) g, v = b2 v +
 * (1 - b2) g^2, Z -= lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps). */
typedef struct {
    mess_precision prec;
    int steps;            /* Adam steps, default 200 when <= 0 */
    double lr;            /* default 0.1 when <= 0 */
    double beta1, beta2;  /* defaults 0.9, 0.999 when <= 0 */
    double eps;           /* default 1e-8 when <= 0 */
    double grad_tol;      /* converged when max |dE/dZ| at the final Z is below it; default 1e-5 */
    double schwarz_tau;
    double fp64_tau;
    int boys_fp64;
    int split_df32;
    void* cuda_stream;
    int xc;               /* 0 Hartree-Fock, 1 LDA, 2 PBE (as mess_scf_opts) */
} mess_min_opts;

/* One molecule; res->E_total etc. at the final Z, res->iterations = steps, res->converged as above.
 * trace (nullable): steps doubles, the total energy at the parameters of each step (before its
 * update).  Errors: MESS_ENOCONV (the gradient criterion failed; results still filled), MESS_EINVAL,
 * MESS_ENOTIMPL (n > 256), MESS_ENUMERIC (singular R or a non-finite energy), MESS_ENOMEM, MESS_ECUDA. */
mess_status mess_minimise(const mess_basis* b, const mess_min_opts* opts, mess_scf_result* res, double* trace);
/* The same over every molecule of bases[0..nmol) at once (the paper's batch over conformations,
 * Sec. 5.2: one set of launches per step for the whole batch; the loss is the sum of the molecules'
 * energies, so each molecule follows its own Adam trajectory).  res: nmol entries; trace (nullable):
 * steps x nmol doubles, row t holding every molecule's energy at step t. */
mess_status mess_minimise_batch(int nmol, mess_basis* const* bases, const mess_min_opts* opts, mess_scf_result* res,
                                double* trace);

/* One kernel launch of a profiled J/K build. */
typedef struct {
    int qclass;                  /* shell-quartet class index (la lb | lc ld), see mess_jk_class_info */
    int la, lb, lc, ld;
    int fp64;                    /* 1: FP64 kernel, 0: FP32 kernel */
    long long shell_quartets, primitive_quartets, function_quartets;
    double flops;                /* algorithmic flops of the launch (op counts of the recursion, Boys,
                                    contraction, HRR and digestion; an FMA counts as 2) */
    double ms;                   /* launch duration, CUDA events on opts->cuda_stream */
    int G;                       /* lanes per shell quartet (primitive loop split over G lanes) */
    int team;                    /* 1: one warp per shell quartet (level-scheduled recursion), 2: one
                                    block of 4 warps per quartet, 3: one block per quartet whose warps
                                    split its primitive quartets, 0: G lanes per quartet */
    int mode;                    /* arithmetic: 0 FP64, 1 FP32 + FP64 Boys, 2 FP32, 3 double-float */
} mess_jk_part;

/* Diagnostic: the J/K build of mess_jk_build_device with a CUDA event pair around every kernel
 * launch; synchronises opts->cuda_stream and fills parts[0..*nparts) (at most max_parts).
 * Errors: as mess_jk_build_device, MESS_EINVAL if max_parts is too small. */
mess_status mess_jk_profile(const mess_basis* b, const double* dD, double* dJ, double* dK,
                            const mess_jk_opts* opts, mess_jk_part* parts, int max_parts, int* nparts);

/* The kernel choice of the quartet bins for these options (the paper has no counterpart), so that one
 * process's autotuning can be reused by another (a profiling run, whose own timings the profiler
 * distorts): 4 ints per bin part - quartet class, G, team, arithmetic (0 FP64, 1 FP32 + FP64 Boys,
 * 2 FP32, 3 double-float).  get: *nparts = number of parts; table (nullable) receives them if
 * max_parts suffices (else MESS_EINVAL).  set: nparts must equal the parts of the same basis and
 * options, and every entry must be a kernel that exists for its part (else MESS_EINVAL, nothing
 * changed).  No GPU work. */
mess_status mess_jk_get_tuning(const mess_basis* b, const mess_jk_opts* opts, int* table, int max_parts, int* nparts);
mess_status mess_jk_set_tuning(const mess_basis* b, const mess_jk_opts* opts, const int* table, int nparts);

/* Diagnostic: the Boys-function grid the J/K kernels expand around (Sec. 3's closed-form integrals
 * need F_m(T)): row k holds F_0..F_15(T_k) and exp(-T_k) at T_k = k * *dT (0.1).  Host-only, no GPU.
 * *nrows, *ncols, *dT (each nullable) receive the shape and spacing; out (nullable) receives
 * nrows * ncols doubles row-major if max_values suffices, else MESS_EINVAL. */
mess_status mess_boys_grid(double* out, int max_values, int* nrows, int* ncols, double* dT);

/* Diagnostic (not part of the paper's method): marks the start (on != 0) or end of the region a
 * kernel profiler started with profiling off at launch (ncu --profile-from-start off) records, so
 * that set-up work (autotuning, warm-up) stays out of a capture.  Errors: MESS_ECUDA. */
mess_status mess_profiler_range(int on);

/* Manual kernel choice for the quartet bins of these options (the paper has no counterpart), e.g. to
 * test every kernel variant against the oracle: every part of a straight-line class runs with G lanes
 * per quartet (1, 4, 8 or 32), or one warp (team = 1), one block of 4 warps (team = 2) or one block
 * whose warps split the primitive quartets (team = 3) per quartet if the class has those kernels;
 * parts of the op-program classes run one warp or block per quartet if team != 0, else one thread
 * per quartet.
 * split_mode: -1 keeps the arithmetic of the split parts, 0 = FP64, 3 = double-float (needs
 * prec MESS_MIXED and split_df32).  Kept until the bins are rebuilt for other options or the
 * autotuner runs.  *nchanged (nullable): parts whose kernel changed.  No GPU work.
 * Errors: MESS_EINVAL (bad arguments). */
mess_status mess_jk_set_variant(const mess_basis* b, const mess_jk_opts* opts, int G, int team, int split_mode,
                                int* nchanged);

/* Kernel autotuner for the quartet bins of these options (the paper has no counterpart: its kernels
 * come from a tracing compiler).  Each bin part (one shell-quartet class x primitive-count group x
 * precision) can be computed by several kernels: G = 1, 4, 8 or 32 lanes per quartet, one warp per
 * quartet, one block of 4 warps per quartet (sharing each recursion level, or splitting the
 * primitive quartets), and for the split (large-integral) parts FP64 or
 * double-float arithmetic when opts->split_df32 allows it.  Each candidate runs on host density D
 * (nbf x nbf): one untimed launch, then reps timings (clamped to 1..50) of 8 copies launched together
 * on the library's streams, forked from and joined to opts->cuda_stream - the parts of a build run
 * concurrently, so a variant is charged for the share of the GPU it takes as well as for its
 * latency - and the fastest is kept for later builds with the same options; results are unchanged to
 * round-off.  The choice is dropped when the bins are rebuilt for other options.  *nchanged
 * (nullable): parts whose kernel changed.  Allocates 3 nbf^2 doubles of device scratch for the call
 * and synchronises the stream.  Errors: as mess_jk_build. */
mess_status mess_jk_autotune(const mess_basis* b, const double* D, const mess_jk_opts* opts, int reps, int* nchanged);

/* Diagnostic (not part of the paper's method): measured CUDA-core FMA throughput of this GPU in
 * TFLOP/s (2 flops per FMA), FP32 and FP64, from independent FMA chains timed with CUDA events on
 * cuda_stream.  Used as the roofline denominator of the ALU-bound integral kernels. */
mess_status mess_fma_peak(double* fp32_tflops, double* fp64_tflops, void* cuda_stream);

/* ---------------------------------------------------------------------------------------------
 * Learned initial density (an addition to the paper's method; the paper motivates combining ML
 * models with the SCF, Sec. 1, and uses Adam, Sec. 5).  A multilayer perceptron 112 -> 256 -> 256 -> 25 (SiLU)
 * maps descriptors of an ordered atom pair (element one-hots, a Gaussian radial basis of the pair
 * distance, radial environments of both atoms) to the 5 x 5 density block of the pair in a frame
 * with z along the pair axis (minimal basis: 1 function on H, s s' p on C / N / O, e.g. STO-3G).
 * BF16 inputs and weights, FP32 accumulation on tensor cores, FP32 master weights, Adam.
 * Parameter vector layout (floats): W1[112][256], b1[256], W2[256][256], b2[256], W3[256][32]
 * (columns 25..31 unused), b3[32].
 * ------------------------------------------------------------------------------------------- */
#define MESS_MLP_DIN 112
#define MESS_MLP_WIDTH 256
#define MESS_MLP_DOUT 25
typedef struct mess_mlp mess_mlp;   /* opaque, library-owned */

int mess_mlp_num_params(void);
/* New network with weights uniform in +-1/sqrt(fan_in) from a seeded splitmix64 stream, zero biases. */
mess_status mess_mlp_create(unsigned long long seed, mess_mlp** out);
void mess_mlp_destroy(mess_mlp* m);
mess_status mess_mlp_get_params(const mess_mlp* m, float* params /* mess_mlp_num_params() */);
mess_status mess_mlp_set_params(mess_mlp* m, const float* params);
/* Binary weight file: "MESSMLP1", 4 ints (112, 256, 25, num_params), the FP32 parameters. */
mess_status mess_mlp_save(const mess_mlp* m, const char* path);
mess_status mess_mlp_load(const char* path, mess_mlp** out);
/* Descriptors of all ordered atom pairs of one molecule (rows = natom^2, row i*natom + j), and with a
 * density D (host n*n) the pair-frame targets T and masks M (rows x 25).  X/T/M may be NULL to query
 * *nrows only.  Errors: MESS_EINVAL for a basis that is not minimal (see above). */
mess_status mess_mlp_features(const mess_basis* b, const double* D, float* X, float* T, float* M, long long* nrows);
/* One forward + backward pass over host rows: masked mean squared error and its gradient
 * (mess_mlp_num_params() floats).  For gradient checks. */
mess_status mess_mlp_loss_grad(mess_mlp* m, long long nrows, const float* X, const float* T, const float* M,
                               double* loss, float* grad);
/* Train on the converged densities of bases[0..nmol) (batched device SCF with opts scf), every
 * ordered atom pair one row, Adam (beta 0.9 / 0.999) over shuffled batches of batch_rows rows for
 * `epochs` epochs, the step size decaying from lr to 0 along a half cosine over all the steps;
 * loss_out (nullable, epochs doubles) receives each epoch's mean loss. */
mess_status mess_mlp_train(mess_mlp* m, int nmol, mess_basis* const* bases, const mess_scf_opts* scf, int epochs,
                           int batch_rows, double lr, double* loss_out);
/* The network's density D0 (host n*n, symmetrised, before any diagonalisation) for one molecule. */
mess_status mess_mlp_predict(const mess_mlp* m, const mess_basis* b, double* D0);

/* Message for the calling thread's most recent failure ("" if none).  Valid until the next call. */
const char* mess_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* MESS_H */
