"""Plain FP64 CPU oracle for the Gaussian-integral / J-K / SCF path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg
of ``bench.py`` may import this package.  It shares no code with the CUDA library: it has its own
basis-file reader, its own normalisation, its own integral code (``oracle.c``, the closed-form
Hermite-Gaussian expressions of Taketa, Huzinaga and O-ohata / McMurchie and Davidson) and its
own SCF.  It never imports the product package and the product never imports it.

What it computes (paper, Sec. 3 "Electronic Structure Theory in a Nutshell"):
  * the LCAO basis of contracted Cartesian Gaussians (Eq. 1) read from a basis-set data file,
  * S_mn = <phi_m|phi_n> (Eq. 3), T and V (the "closed-form expressions for all the relevant
    integrals"), the repulsion integrals (mn|ls),
  * J_mn = sum_ls (mn|ls) D_ls and K_mn = sum_ls (ml|ns) D_ls (Hartree-Fock exchange,
    ``xc_method="hfx"`` in Sec. 5.1),
  * the Roothaan equation F(C) C = S C eps (Eq. 2) solved by self-consistent-field iteration
    (Sec. 3), F = H + J - K/2, E_elec = 1/2 tr D (H + F), plus the nuclear repulsion
    ``nuclear_energy`` of Sec. 5.1.

Readings where the paper is silent (each listed with its reason in the design notes):
  * Cartesian d (6 components, order xx, xy, xz, yy, yz, zz); every contracted function is
    normalised to <phi|phi> = 1 on its own.
  * D is the total closed-shell density 2 C_occ C_occ^T.
  * SCF: Loewdin X = S^-1/2, core-Hamiltonian guess, Pulay DIIS on FDS - SDF with 8 vectors,
    converged when |dE| < 1e-10 and max|FDS - SDF| < 1e-8.
  * Screening: a shell quartet is dropped iff Q_ab Q_cd < tau, Q_ab = sqrt(max |(mn|mn)|).

parity: pinned by tests/test_oracle_*.py (Boys closed forms and quadrature, textbook
minimal-basis H2 and HeH+ integrals and energies, brute-force quadrature of every integral
class, permutational symmetry, Schwarz inequality, idempotency and trace invariants).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_SYMBOL_Z = {"H": 1, "He": 2, "Li": 3, "Be": 4, "B": 5, "C": 6, "N": 7, "O": 8, "F": 9}
_Z_SYMBOL = {v: k for k, v in _SYMBOL_Z.items()}
_L_OF = {"S": 0, "P": 1, "D": 2}


def build(force: bool = False) -> str:
    """Compile ``oracle.c`` with gcc (OpenMP) into ``liboracle.so`` next to it."""
    src = os.path.join(_HERE, "oracle.c")
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(src):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", src, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB_PATH)
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        fn_args = [ctypes.c_int, dp, ip, ip, ip, dp, dp]
        L.oracle_boys.argtypes = [ctypes.c_int, ctypes.c_double, dp]
        L.oracle_one_e.argtypes = fn_args + [ctypes.c_int, ip, dp, dp, dp, dp]
        L.oracle_eri.argtypes = fn_args + [ctypes.c_int] * 4
        L.oracle_eri.restype = ctypes.c_double
        L.oracle_eri_tensor.argtypes = fn_args + [dp]
        L.oracle_schwarz.argtypes = fn_args + [ip, ctypes.c_int, dp]
        jk_args = fn_args + [ip, ctypes.c_int, dp, ctypes.c_double, dp, dp, dp]
        L.oracle_jk_brute.argtypes = jk_args
        L.oracle_jk_sym.argtypes = jk_args
        L.oracle_jk_elements.argtypes = fn_args + [ip, ctypes.c_int, dp, ctypes.c_double, dp,
                                                   ctypes.c_int, ip, ip, dp, dp]
        L.oracle_num_threads.restype = ctypes.c_int
        L.oracle_set_num_threads.argtypes = [ctypes.c_int]
        _lib = L
    return _lib


def _d(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _i(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def num_threads() -> int:
    return int(lib().oracle_num_threads())


def set_num_threads(n: int) -> None:
    """Threads of the oracle's OpenMP loops (n <= 0: every processor)."""
    lib().oracle_set_num_threads(int(n))


# ----------------------------------------------------------------------------- Boys function
def boys(nmax: int, T: float) -> np.ndarray:
    """F_n(T) for n = 0..nmax (compensated positive series / erf + upward recursion)."""
    out = np.zeros(nmax + 1)
    lib().oracle_boys(int(nmax), float(T), _d(out))
    return out


# ----------------------------------------------------------------------------- basis set
def read_basis_file(path: str) -> dict:
    """Element symbol -> list of shells (l, exponents, coefficients); SP shells are split."""
    out: dict = {}
    cur = None
    lines = [ln.split("#")[0].strip() for ln in open(path)]
    lines = [ln for ln in lines if ln]
    i = 0
    while i < len(lines):
        tok = lines[i].split()
        if tok[0] == "element":
            cur = out.setdefault(tok[1], [])
            i += 1
            continue
        kind, nprim = tok[0].upper(), int(tok[1])
        rows = [list(map(float, lines[i + 1 + k].split())) for k in range(nprim)]
        exps = [r[0] for r in rows]
        if kind == "SP":
            cur.append((0, exps, [r[1] for r in rows]))
            cur.append((1, exps, [r[2] for r in rows]))
        else:
            cur.append((_L_OF[kind], exps, [r[1] for r in rows]))
        i += 1 + nprim
    return out


def cartesian_components(l: int):
    """Cartesian power triples of angular momentum l in the order x..., e.g. xx xy xz yy yz zz."""
    comps = []
    for lx in range(l, -1, -1):
        for ly in range(l - lx, -1, -1):
            comps.append((lx, ly, l - lx - ly))
    return comps


def _dfact(k: int) -> int:
    r = 1
    while k > 1:
        r *= k
        k -= 2
    return r


def primitive_norm(alpha: float, lmn) -> float:
    """N(alpha, l, m, n) making one Cartesian Gaussian primitive of unit norm."""
    l, m, n = lmn
    L = l + m + n
    return ((2 * alpha / math.pi) ** 0.75 * (4 * alpha) ** (L / 2)
            / math.sqrt(_dfact(2 * l - 1) * _dfact(2 * m - 1) * _dfact(2 * n - 1)))


@dataclass
class Basis:
    """One row per contracted Cartesian function (atom order, then shell order, then component)."""
    nfn: int
    center: np.ndarray   # [nfn, 3]
    lmn: np.ndarray      # [nfn, 3] int32
    nprim: np.ndarray    # [nfn] int32
    poff: np.ndarray     # [nfn] int32
    exps: np.ndarray     # [sum nprim]
    coefs: np.ndarray    # [sum nprim], normalised
    shell: np.ndarray    # [nfn] int32 shell index
    nshell: int
    atom: np.ndarray     # [nfn] int32 atom index
    Z: np.ndarray
    xyz: np.ndarray

    def args(self):
        return (int(self.nfn), _d(self.center), _i(self.lmn), _i(self.nprim), _i(self.poff),
                _d(self.exps), _d(self.coefs))


def make_basis(Z, xyz, basis_file: str, scale_exponents=None) -> Basis:
    """Expand atoms into contracted Cartesian functions; each normalised so S_mm = 1."""
    Z = np.asarray(Z, dtype=np.int32)
    xyz = np.ascontiguousarray(np.asarray(xyz, dtype=np.float64).reshape(-1, 3))
    data = read_basis_file(basis_file)
    center, lmn, nprim, poff, exps, coefs, shell, atom = [], [], [], [], [], [], [], []
    nsh = 0
    for a, z in enumerate(Z):
        sym = _Z_SYMBOL[int(z)]
        if sym not in data:
            raise ValueError(f"element {sym} missing from {basis_file}")
        for (l, ex, co) in data[sym]:
            if scale_exponents is not None:
                ex = [e * scale_exponents[a] for e in ex]
            for comp in cartesian_components(l):
                center.append(xyz[a])
                lmn.append(comp)
                nprim.append(len(ex))
                poff.append(len(exps))
                for e, c in zip(ex, co):
                    exps.append(e)
                    coefs.append(c * primitive_norm(e, comp))
                shell.append(nsh)
                atom.append(a)
            nsh += 1
    b = Basis(len(lmn), np.ascontiguousarray(np.array(center, dtype=np.float64)),
              np.ascontiguousarray(np.array(lmn, dtype=np.int32)),
              np.array(nprim, dtype=np.int32), np.array(poff, dtype=np.int32),
              np.array(exps, dtype=np.float64), np.array(coefs, dtype=np.float64),
              np.array(shell, dtype=np.int32), nsh, np.array(atom, dtype=np.int32), Z, xyz)
    # renormalise every contracted function by its own self-overlap
    S = overlap(b)
    for m in range(b.nfn):
        sl = slice(b.poff[m], b.poff[m] + b.nprim[m])
        b.coefs[sl] /= math.sqrt(S[m, m])
    return b


def basis_for(mol, basis_file: str) -> Basis:
    return make_basis(mol.Z, mol.xyz, basis_file)


# ----------------------------------------------------------------------------- integrals
def one_e(b: Basis):
    n = b.nfn
    S, T, V = np.zeros((n, n)), np.zeros((n, n)), np.zeros((n, n))
    Z = np.ascontiguousarray(b.Z, dtype=np.int32)
    lib().oracle_one_e(*b.args(), int(len(Z)), _i(Z), _d(b.xyz), _d(S), _d(T), _d(V))
    return S, T, V


def overlap(b: Basis):
    n = b.nfn
    S = np.zeros((n, n))
    Z = np.ascontiguousarray(b.Z, dtype=np.int32)
    null = ctypes.POINTER(ctypes.c_double)()
    lib().oracle_one_e(*b.args(), 0, _i(Z), _d(b.xyz), _d(S), null, null)
    return S


def eri(b: Basis, m: int, n: int, l: int, s: int) -> float:
    return float(lib().oracle_eri(*b.args(), m, n, l, s))


def eri_tensor(b: Basis) -> np.ndarray:
    n = b.nfn
    out = np.zeros((n, n, n, n))
    lib().oracle_eri_tensor(*b.args(), _d(out))
    return out


def schwarz(b: Basis) -> np.ndarray:
    """Q[A, B] = sqrt(max_{m in A, n in B} |(mn|mn)|) over shells."""
    Q = np.zeros((b.nshell, b.nshell))
    lib().oracle_schwarz(*b.args(), _i(b.shell), int(b.nshell), _d(Q))
    return Q


def jk(b: Basis, D: np.ndarray, tau: float = 0.0, method: str = "sym", Q=None):
    """J and K of a symmetric density D; quartets with Q_ab Q_cd < tau dropped (tau > 0)."""
    n = b.nfn
    D = np.ascontiguousarray(D, dtype=np.float64)
    J, K = np.zeros((n, n)), np.zeros((n, n))
    if tau > 0.0 and Q is None:
        Q = schwarz(b)
    Qa = np.ascontiguousarray(Q if Q is not None else np.zeros((b.nshell, b.nshell)))
    fn = {"sym": lib().oracle_jk_sym, "brute": lib().oracle_jk_brute}[method]
    fn(*b.args(), _i(b.shell), int(b.nshell), _d(Qa), float(tau), _d(D), _d(J), _d(K))
    return J, K


def jk_elements(b: Basis, D: np.ndarray, rows, cols, tau: float = 0.0, Q=None):
    """J_mn, K_mn for the listed (m, n) only, each by its defining sum over all (l, s)."""
    D = np.ascontiguousarray(D, dtype=np.float64)
    rows = np.ascontiguousarray(rows, dtype=np.int32)
    cols = np.ascontiguousarray(cols, dtype=np.int32)
    Js, Ks = np.zeros(len(rows)), np.zeros(len(rows))
    if tau > 0.0 and Q is None:
        Q = schwarz(b)
    Qa = np.ascontiguousarray(Q if Q is not None else np.zeros((b.nshell, b.nshell)))
    lib().oracle_jk_elements(*b.args(), _i(b.shell), int(b.nshell), _d(Qa), float(tau), _d(D),
                             int(len(rows)), _i(rows), _i(cols), _d(Js), _d(Ks))
    return Js, Ks


def nuclear_repulsion(Z, xyz) -> float:
    """sum_{A<B} Z_A Z_B / |R_A - R_B| (the paper's ``nuclear_energy``)."""
    Z = np.asarray(Z, dtype=np.float64)
    xyz = np.asarray(xyz, dtype=np.float64).reshape(-1, 3)
    e = 0.0
    for a in range(len(Z)):
        for c in range(a):
            e += Z[a] * Z[c] / float(np.linalg.norm(xyz[a] - xyz[c]))
    return e


# ----------------------------------------------------------------------------- energy / SCF
def fock(H, J, K):
    """F = H + J - K/2 for the closed-shell density D (Hartree-Fock exchange)."""
    return H + J - 0.5 * K


def electronic_energy(D, H, F) -> float:
    """E_elec = 1/2 sum_mn D_mn (H_mn + F_mn)."""
    return 0.5 * float(np.sum(D * (H + F)))


def density_from_fock(F, X, nocc):
    """Solve F C = S C eps through the orthonormal basis X: D = 2 C_occ C_occ^T, C = X C'."""
    Fp = X.T @ F @ X
    eps, Cp = np.linalg.eigh(Fp)
    C = X @ Cp
    Cocc = C[:, :nocc]
    return 2.0 * Cocc @ Cocc.T, eps, C


def loewdin(S):
    s, U = np.linalg.eigh(S)
    if s.min() < 1e-7:
        raise ValueError("overlap matrix nearly singular")
    return U @ np.diag(s ** -0.5) @ U.T


@dataclass
class SCFResult:
    E_total: float
    E_elec: float
    E_nuc: float
    iterations: int
    converged: bool
    D: np.ndarray
    eps: np.ndarray
    history: list


def scf(b: Basis, nelectron: int | None = None, max_iter: int = 100, conv_E: float = 1e-10,
        conv_comm: float = 1e-8, diis_n: int = 8, tau: float = 0.0, D0=None) -> SCFResult:
    """Closed-shell Roothaan SCF (Eq. 2) to self-consistency."""
    nel = int(np.sum(b.Z)) if nelectron is None else nelectron
    if nel % 2:
        raise ValueError("closed-shell SCF needs an even electron count")
    nocc = nel // 2
    S, T, V = one_e(b)
    H = T + V
    X = loewdin(S)
    Enuc = nuclear_repulsion(b.Z, b.xyz)
    Q = schwarz(b) if tau > 0 else None
    D = density_from_fock(H, X, nocc)[0] if D0 is None else D0
    Fs, es, hist = [], [], []
    E_old = None
    converged = False
    eps = None
    it = 0
    for it in range(1, max_iter + 1):
        J, K = jk(b, D, tau=tau, Q=Q)
        F = fock(H, J, K)
        E = electronic_energy(D, H, F)
        err = F @ D @ S - S @ D @ F
        emax = float(np.abs(err).max())
        hist.append((E + Enuc, emax))
        if E_old is not None and abs(E - E_old) < conv_E and emax < conv_comm:
            converged = True
            break
        E_old = E
        Fs.append(F)
        es.append(err)
        if len(Fs) > diis_n:
            Fs.pop(0)
            es.pop(0)
        if len(Fs) >= 2:
            m = len(Fs)
            B = np.empty((m + 1, m + 1))
            B[-1, :] = -1.0
            B[:, -1] = -1.0
            B[-1, -1] = 0.0
            for i in range(m):
                for j in range(m):
                    B[i, j] = float(np.sum(es[i] * es[j]))
            rhs = np.zeros(m + 1)
            rhs[-1] = -1.0
            c = np.linalg.solve(B, rhs)[:m]
            F = sum(ci * Fi for ci, Fi in zip(c, Fs))
        D, eps, _ = density_from_fock(F, X, nocc)
    return SCFResult(E + Enuc, E, Enuc, it, converged, D, eps, hist)
