"""Pins for the direct-minimisation oracle (CPU only): its gradient, its energy functional and its
minimum, each against something other than itself."""
import numpy as np
import pytest

import mess_inputs as mi
from oracle import minimise as om


@pytest.fixture(scope="module")
def h2o(oracle_mod):
    b = oracle_mod.basis_for(mi.h2o(), mi.basis_path("sto-3g"))
    return b, om.problem(b), oracle_mod.scf(b)


def test_gradient_matches_finite_differences(h2o):
    _, p, _ = h2o
    n = p.H.shape[0]
    rng = np.random.default_rng(11)
    Z = np.eye(n) + 0.2 * rng.normal(size=(n, n))
    _, g = om.energy_and_grad(p, Z)
    h = 1e-5
    for i, j in [(0, 0), (3, 1), (6, 4), (2, 2), (5, 0)]:
        e = np.zeros_like(Z)
        e[i, j] = h
        fd = (om.energy(p, Z + e) - om.energy(p, Z - e)) / (2 * h)
        assert g[i, j] == pytest.approx(fd, rel=1e-6, abs=1e-8)
    # columns beyond the occupied ones do not enter the energy
    assert np.all(g[:, p.nocc:] == 0.0)


def test_orthonormality_and_scf_stationary_point(h2o, oracle_mod):
    b, p, ref = h2o
    rng = np.random.default_rng(3)
    C, _, _ = om.orthonormalise(p, rng.normal(size=p.H.shape))
    np.testing.assert_allclose(C.T @ p.S @ C, np.eye(p.H.shape[0]), atol=1e-12)
    # Z = the SCF's orthonormal-basis eigenvectors reproduces the SCF energy, and is stationary
    J, K = oracle_mod.jk(b, ref.D)
    F = p.H + J - 0.5 * K
    _, Cp = np.linalg.eigh(p.X.T @ F @ p.X)
    E, g = om.energy_and_grad(p, Cp)
    assert E == pytest.approx(ref.E_total, abs=1e-10)
    assert np.abs(g).max() < 1e-6


def test_adam_reaches_the_scf_energy(h2o, oracle_mod):
    """The paper's loop (Adam, learning rate 0.1, from Z = 1) on H2 (128 steps, as in its batched
    example) and H2O / STO-3G (200 steps, as in its single-molecule example) ends at the SCF energy."""
    _, p, ref = h2o
    _, trace, E = om.adam(p, 200)
    assert abs(E - ref.E_total) < 1e-8
    assert trace[0] > trace[-1]
    b2 = oracle_mod.basis_for(mi.h2(1.4), mi.basis_path("sto-3g"))
    _, _, E2 = om.adam(om.problem(b2), 128)
    assert abs(E2 - oracle_mod.scf(b2).E_total) < 1e-6
