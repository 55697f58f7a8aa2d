"""Pins for the oracle's J/K and SCF: textbook energies, invariants, brute force vs symmetry."""
import json
import math
import os

import numpy as np
import pytest

import mess_inputs as mi

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "szabo_ostlund_minimal_basis.json")
TEXTBOOK = os.path.join(os.path.dirname(__file__), "golden", "szabo_ostlund_hf_energies.json")


def test_jk_symmetric_loop_equals_definition(oracle_mod):
    for mol, basis in ((mi.h2o(), "sto-3g"), (mi.alkane(2, np.random.default_rng(5)), "sto-3g"),
                       (mi.water_cluster(2, 9.0, 11), "6-31gs")):
        b = oracle_mod.basis_for(mol, mi.basis_path(basis))
        D = mi.random_symmetric_density(b.nfn, 3)
        Js, Ks = oracle_mod.jk(b, D, method="sym")
        Jb, Kb = oracle_mod.jk(b, D, method="brute")
        assert np.abs(Js - Jb).max() < 1e-12
        assert np.abs(Ks - Kb).max() < 1e-12
        assert np.abs(Js - Js.T).max() < 1e-12 and np.abs(Ks - Ks.T).max() < 1e-12
        # Coulomb energy of a positive semidefinite density is non-negative
        assert 0.5 * np.sum(D * Js) > 0.0
        # exchange is bounded by Coulomb for a PSD density: tr(DK) <= tr(DJ)
        assert np.sum(D * Ks) <= np.sum(D * Js) + 1e-12


def test_jk_elements_match_full(oracle_mod):
    b = oracle_mod.basis_for(mi.water_cluster(2, 9.0, 11), mi.basis_path("6-31gs"))
    D = mi.random_symmetric_density(b.nfn, 4)
    J, K = oracle_mod.jk(b, D)
    rows, cols = np.array([0, 5, 17, 30, 37]), np.array([0, 9, 3, 31, 12])
    Js, Ks = oracle_mod.jk_elements(b, D, rows, cols)
    assert np.allclose(Js, J[rows, cols], atol=1e-12)
    assert np.allclose(Ks, K[rows, cols], atol=1e-12)


def test_screening_rule(oracle_mod):
    """Screened J/K differ from the unscreened sums by no more than the dropped bound allows."""
    b = oracle_mod.basis_for(mi.water_cluster(3, 16.0, 13), mi.basis_path("sto-3g"))
    D = mi.random_symmetric_density(b.nfn, 5)
    Q = oracle_mod.schwarz(b)
    J0, K0 = oracle_mod.jk(b, D)
    tau = 1e-6
    J1, K1 = oracle_mod.jk(b, D, tau=tau, Q=Q)
    dropped = np.sum((np.outer(Q.ravel(), Q.ravel()) < tau))
    assert dropped > 0
    bound = tau * np.abs(D).max() * b.nfn ** 2
    assert np.abs(J1 - J0).max() <= bound and np.abs(K1 - K0).max() <= bound
    # Schwarz: every |(mn|ls)| <= Q_ab Q_cd
    for q in [(0, 1, 5, 6), (2, 7, 9, 12), (3, 3, 20, 8)]:
        sh = b.shell[list(q)]
        assert abs(oracle_mod.eri(b, *q)) <= Q[sh[0], sh[1]] * Q[sh[2], sh[3]] * (1 + 1e-12)


def test_szabo_ostlund_h2_scf(oracle_mod):
    g = json.load(open(GOLDEN))["h2"]
    b = oracle_mod.basis_for(mi.h2(g["R_bohr"]), mi.basis_path("sto-3g"))
    r = oracle_mod.scf(b)
    assert r.converged
    tol = g["tol"]
    assert r.eps[0] == pytest.approx(g["eps1"], abs=tol)
    assert r.eps[1] == pytest.approx(g["eps2"], abs=tol)
    assert r.E_elec == pytest.approx(g["E_elec"], abs=tol)
    assert r.E_total == pytest.approx(g["E_total"], abs=tol)


def test_szabo_ostlund_heh_plus_scf(oracle_mod, tmp_path):
    g = json.load(open(GOLDEN))
    h, z = g["heh_plus"], g["sto1g_zeta1_expansion"]
    lines = []
    for sym, zeta in (("He", h["zeta_He"]), ("H", h["zeta_H"])):
        lines += [f"element {sym}", "S 3"]
        lines += [f"{e * zeta ** 2:.10f} {c}" for e, c in zip(z["exponents"], z["coefficients"])]
    path = tmp_path / "heh.basis"
    path.write_text("\n".join(lines) + "\n")
    b = oracle_mod.make_basis([2, 1], [[0, 0, 0], [h["R_bohr"], 0, 0]], str(path))
    r = oracle_mod.scf(b, nelectron=2)
    assert r.converged
    assert r.E_elec == pytest.approx(h["E_elec"], abs=h["tol_energy"])
    assert r.E_total == pytest.approx(h["E_total"], abs=h["tol_energy"])


def _ch4():
    d = 2.050 / math.sqrt(3.0)
    xyz = [[0, 0, 0], [d, d, d], [d, -d, -d], [-d, d, -d], [-d, -d, d]]
    return mi.Molecule("ch4", np.array([6, 1, 1, 1, 1], dtype=np.int32), np.array(xyz, dtype=float))


@pytest.mark.parametrize("key", ["h2o_sto-3g", "h2o_6-31gs", "ch4_sto-3g", "ch4_6-31gs"])
def test_textbook_hf_energies(oracle_mod, key):
    g = json.load(open(TEXTBOOK))
    mol = mi.h2o() if key.startswith("h2o") else _ch4()
    b = oracle_mod.basis_for(mol, mi.basis_path(key.split("_")[1]))
    r = oracle_mod.scf(b)
    assert r.converged
    assert r.E_total == pytest.approx(g[key], abs=g["tol"])


def test_scf_invariants_h2o_631gs(oracle_mod):
    mol = mi.h2o()
    b = oracle_mod.basis_for(mol, mi.basis_path("6-31gs"))
    r = oracle_mod.scf(b)
    S = oracle_mod.overlap(b)
    assert r.converged and r.iterations < 40
    assert np.trace(r.D @ S) == pytest.approx(10.0, abs=1e-10)
    assert np.abs(r.D @ S @ r.D - 2.0 * r.D).max() < 1e-8
    # rotation + translation invariance exercises every Cartesian d component
    rng = np.random.default_rng(3)
    q = rng.standard_normal(4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    R = np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
                  [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
                  [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)]])
    b2 = oracle_mod.make_basis(mol.Z, mol.xyz @ R.T + np.array([1.0, 2.0, -0.5]), mi.basis_path("6-31gs"))
    r2 = oracle_mod.scf(b2)
    assert r2.E_total == pytest.approx(r.E_total, abs=1e-9)
    # scaling one basis function leaves the energy unchanged (absorbed into C)
    b3 = oracle_mod.basis_for(mol, mi.basis_path("6-31gs"))
    b3.coefs[b3.poff[10]:b3.poff[10] + b3.nprim[10]] *= 1.7
    r3 = oracle_mod.scf(b3)
    assert r3.E_total == pytest.approx(r.E_total, abs=1e-9)


def test_scf_guess_independence(oracle_mod):
    b = oracle_mod.basis_for(mi.h2o(), mi.basis_path("sto-3g"))
    r1 = oracle_mod.scf(b)
    D0 = mi.random_symmetric_density(b.nfn, 9, nocc=5)
    r2 = oracle_mod.scf(b, D0=D0)
    assert r1.converged and r2.converged
    assert r2.E_total == pytest.approx(r1.E_total, abs=1e-9)


def test_h2_dissociation_limit(oracle_mod):
    """Minimal-basis RHF H2 dissociates to 2 h_11 + (11|11)/2 (one sigma_g orbital, cross terms
    vanishing), approached as -1/(2R): at large R the neutral atoms' Coulomb terms cancel except half
    of the inter-atomic electron repulsion.  h_11 = T_11 + V^(1)_11 and (11|11) from the printed
    STO-3G values (zeta = 1.24): 2 (0.7600 - 1.2266) + 0.7746 / 2 = -0.5459."""
    gold = json.load(open(GOLDEN))["h2"]
    limit = 2.0 * (gold["T11"] + gold["V1_11"]) + 0.5 * gold["eri_1111"]
    for R in (10.0, 20.0):
        o = oracle_mod.basis_for(mi.h2(R), mi.basis_path("sto-3g"))
        r = oracle_mod.scf(o)
        assert r.converged
        assert r.E_total + 0.5 / R == pytest.approx(limit, abs=3e-4)
