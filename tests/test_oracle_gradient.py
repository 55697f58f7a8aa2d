"""Pins for the finite-difference gradient oracle (CPU only)."""
import numpy as np
import pytest

import mess_inputs as mi
from oracle import gradient as og


def test_invariances_and_step_size():
    mol = mi.h2o()
    xyz = mol.xyz + np.random.default_rng(3).normal(scale=0.05, size=mol.xyz.shape)
    path = mi.basis_path("sto-3g")
    g = og.fd_gradient(mol.Z, xyz, path)
    # translations: the forces sum to zero; rotations: no net torque
    assert np.abs(g.sum(axis=0)).max() < 1e-8
    torque = np.cross(xyz - xyz.mean(axis=0), g).sum(axis=0)
    assert np.abs(torque).max() < 1e-8
    g2 = og.fd_gradient(mol.Z, xyz, path, h=2e-3)
    assert np.abs(g - g2).max() < 1e-8


def test_mirror_symmetry():
    """H2O in its C2v frame (plane xz, axis z): the H forces mirror each other in x, the O force lies on z."""
    mol = mi.h2o()
    g = og.fd_gradient(mol.Z, mol.xyz, mi.basis_path("sto-3g"))
    assert abs(g[0, 0]) < 1e-9 and abs(g[0, 1]) < 1e-9
    assert g[1, 0] == pytest.approx(-g[2, 0], abs=1e-9)
    assert g[1, 2] == pytest.approx(g[2, 2], abs=1e-9)
