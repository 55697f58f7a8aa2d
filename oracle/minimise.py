"""Oracle of the direct energy minimisation (paper Sec. 3, the constrained minimisation of E(C)
subject to C^T S C = 1, and Sec. 5.1 / 5.2, its solution with the Adam optimiser).

TEST INFRASTRUCTURE ONLY (same rules as the rest of ``oracle/``): plain numpy in FP64, with the
oracle's own integrals and J/K.  Nothing on the library's product path imports it.

The unconstrained parameters are an n x n matrix Z.  The orthonormality constraint (Eq. 4) is
built in by a QR decomposition: Z = Q R, C = X Q with X = S^-1/2 (the Loewdin orthogonaliser of
the SCF), so C^T S C = Q^T X S X Q = 1 for every Z.  The density is D = 2 C_occ C_occ^T (the first
N_e / 2 columns) and the energy E(Z) = 1/2 sum D (H + F) + E_nuc with F = H + J(D) - K(D)/2 (the
Hartree-Fock energy functional H(P) plus the nuclear energy).

Gradient (written out from the chain rule; E depends on Z only through the first N_e / 2 columns
of Q, whatever sign convention the QR uses):
  dE/dD = F  =>  dE/dC_occ = 4 F C_occ (zero for the other columns),  G = dE/dQ = X^T dE/dC;
  for Z = Q R with Q square orthogonal, a perturbation gives Q^T dZ R^-1 = Omega + dR R^-1 with
  Omega = Q^T dQ skew and dR R^-1 upper triangular, so Omega is the strictly lower part of
  Q^T dZ R^-1 minus its transpose; pairing with G gives
      dE/dZ = Q tril(Q^T G - G^T Q, -1) R^-T.
Adam (Kingma & Ba 2014): m = b1 m + (1 - b1) g, v = b2 v + (1 - b2) g^2,
  Z -= lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps), elementwise, t = 1, 2, ...

parity: pinned by tests/test_oracle_minimise.py (the gradient against central finite differences of
E(Z); the energy of Z = the SCF eigenvectors equal to the SCF energy; Adam's minimum equal to the
SCF energy; C^T S C = 1).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import jk, loewdin, nuclear_repulsion, one_e


@dataclass
class Problem:
    H: np.ndarray
    S: np.ndarray
    X: np.ndarray
    nocc: int
    E_nuc: float
    basis: object


def problem(b) -> Problem:
    S, T, V = one_e(b)
    nel = int(np.sum(b.Z))
    if nel % 2:
        raise ValueError("closed-shell minimisation needs an even electron count")
    return Problem(T + V, S, loewdin(S), nel // 2, nuclear_repulsion(b.Z, b.xyz), b)


def orthonormalise(p: Problem, Z):
    Q, R = np.linalg.qr(Z)
    return p.X @ Q, Q, R


def energy(p: Problem, Z) -> float:
    C, _, _ = orthonormalise(p, Z)
    Co = C[:, :p.nocc]
    D = 2.0 * Co @ Co.T
    J, K = jk(p.basis, D)
    F = p.H + J - 0.5 * K
    return 0.5 * float(np.sum(D * (p.H + F))) + p.E_nuc


def energy_and_grad(p: Problem, Z):
    C, Q, R = orthonormalise(p, Z)
    Co = C[:, :p.nocc]
    D = 2.0 * Co @ Co.T
    J, K = jk(p.basis, D)
    F = p.H + J - 0.5 * K
    E = 0.5 * float(np.sum(D * (p.H + F))) + p.E_nuc
    dC = np.zeros_like(C)
    dC[:, :p.nocc] = 4.0 * F @ Co
    G = p.X.T @ dC
    A = Q.T @ G
    B = np.tril(A - A.T, -1)
    dZ = np.linalg.solve(R, (Q @ B).T).T        # (Q B) R^-T
    return E, dZ


def adam(p: Problem, steps: int, lr: float = 0.1, b1: float = 0.9, b2: float = 0.999, eps: float = 1e-8,
         Z0=None):
    """Adam on E(Z) from Z0 (default the identity, the paper's start); returns (Z, energies per step,
    the energy at the final Z)."""
    n = p.H.shape[0]
    Z = np.eye(n) if Z0 is None else np.array(Z0, dtype=np.float64)
    m = np.zeros_like(Z)
    v = np.zeros_like(Z)
    trace = []
    for t in range(1, steps + 1):
        E, g = energy_and_grad(p, Z)
        trace.append(E)
        m = b1 * m + (1.0 - b1) * g
        v = b2 * v + (1.0 - b2) * g * g
        Z = Z - lr * (m / (1.0 - b1 ** t)) / (np.sqrt(v / (1.0 - b2 ** t)) + eps)
    return Z, np.array(trace), energy(p, Z)
