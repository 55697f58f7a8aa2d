"""Oracle of the nuclear gradient: dE/dR of the oracle's Hartree-Fock energy by its definition, a
derivative, taken numerically.

TEST INFRASTRUCTURE ONLY (same rules as the rest of ``oracle/``).  Each component is the fourth-order
central difference [-E(R + 2h) + 8 E(R + h) - 8 E(R - h) + E(R - 2h)] / (12 h) of the total energy of
the oracle's SCF converged tightly (max |FDS - SDF| < 1e-10, so the energy is exact to far below the
difference's resolution: it is stationary in the density), with h = 1e-3 bohr (truncation error of
order h^4 times the fifth derivative, below 1e-10).

parity: pinned by tests/test_oracle_gradient.py (translational and rotational invariance of the
forces; the mirror symmetry of a symmetric molecule's forces; agreement of two step sizes).
"""
from __future__ import annotations

import numpy as np

from . import make_basis, scf


def total_energy(Z, xyz, basis_file):
    r = scf(make_basis(Z, xyz, basis_file), conv_E=1e-13, conv_comm=1e-10, max_iter=200)
    if not r.converged:
        raise RuntimeError("SCF did not converge")
    return r.E_total


def fd_gradient(Z, xyz, basis_file, h=1e-3):
    xyz = np.asarray(xyz, dtype=np.float64).reshape(-1, 3)
    g = np.zeros_like(xyz)
    for a in range(len(xyz)):
        for x in range(3):
            e = []
            for k in (2, 1, -1, -2):
                p = xyz.copy()
                p[a, x] += k * h
                e.append(total_energy(Z, p, basis_file))
            g[a, x] = (-e[0] + 8.0 * e[1] - 8.0 * e[2] + e[3]) / (12.0 * h)
    return g
