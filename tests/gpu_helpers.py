"""Input preparation shared by the full-size GPU tests (no oracle arithmetic here).

converged_density: a converged closed-shell density of a basis too large for the library's
on-device SCF (its Jacobi eigensolver takes n <= 256), from Roothaan iterations with Pulay DIIS in
numpy around the library's FP64 J/K build.  It is an input for the precision comparisons (the
FP64 J/K build it uses is itself held to the oracle by the sampled-element tests).

sample_pairs: (row, col) index pairs of J / K chosen to cover given function kinds.
"""
import numpy as np


def converged_density(g, schwarz_tau=1e-10, iters=60, conv_E=1e-9, conv_comm=1e-7):
    S, H = g.overlap(), g.kinetic() + g.nuclear()
    s, U = np.linalg.eigh(S)
    X = U @ np.diag(s ** -0.5) @ U.T
    nocc = g.nelectron // 2

    def dens(F):
        _, C = np.linalg.eigh(X.T @ F @ X)
        C = X @ C
        return 2.0 * C[:, :nocc] @ C[:, :nocc].T

    D, Fs, es, E_old = dens(H), [], [], 0.0
    for _ in range(iters):
        J, K, _ = g.jk(D, prec="fp64", schwarz_tau=schwarz_tau)
        F = H + J - 0.5 * K
        E = 0.5 * float(np.sum(D * (H + F)))
        err = F @ D @ S - S @ D @ F
        if abs(E - E_old) < conv_E and np.abs(err).max() < conv_comm:
            return D
        E_old = E
        Fs, es = (Fs + [F])[-8:], (es + [err])[-8:]
        if len(Fs) >= 2:
            k = len(Fs)
            B = -np.ones((k + 1, k + 1))
            B[-1, -1] = 0.0
            for i in range(k):
                for j in range(k):
                    B[i, j] = float(np.sum(es[i] * es[j]))
            c = np.linalg.solve(B, np.r_[np.zeros(k), -1.0])[:k]
            F = sum(ci * Fi for ci, Fi in zip(c, Fs))
        D = dens(F)
    raise RuntimeError("Roothaan iterations did not converge")


def function_kinds(o):
    """Per function of an oracle basis: (atomic number of its atom, angular momentum)."""
    Z = np.asarray(o.Z)[np.asarray(o.atom)]
    l = np.asarray(o.lmn).sum(axis=1)
    return Z, l


def sample_pairs(o, rng, per_kind, n_random):
    """(rows, cols): per_kind pairs of each kind - O-d with O-d (different functions), O-s with H-s,
    diagonal elements of every kind of function (O s, O p, O d, H s) - plus n_random uniform pairs."""
    Z, l = function_kinds(o)
    od = np.flatnonzero((Z == 8) & (l == 2))
    os_ = np.flatnonzero((Z == 8) & (l == 0))
    op = np.flatnonzero((Z == 8) & (l == 1))
    hs = np.flatnonzero(Z == 1)
    rows, cols = [], []
    for _ in range(per_kind):
        a, b = rng.choice(od, 2, replace=False)
        rows.append(a); cols.append(b)
        rows.append(rng.choice(os_)); cols.append(rng.choice(hs))
    diag = [rng.choice(x) for x in (os_, op, od, hs) for _ in range(max(1, per_kind // 4))]
    rows += diag
    cols += diag
    n = o.nfn
    rows += list(rng.integers(0, n, n_random))
    cols += list(rng.integers(0, n, n_random))
    return np.array(rows, dtype=np.int64), np.array(cols, dtype=np.int64)
