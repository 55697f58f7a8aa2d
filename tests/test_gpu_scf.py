"""Device SCF (mess_scf / mess_scf_batch through the C ABI) against the oracle's SCF."""
import json
import os

import numpy as np
import pytest

import mess_inputs as mi

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "szabo_ostlund_minimal_basis.json")


def _pair(mess, oracle, mol, basis):
    path = mi.basis_path(basis)
    return mess.Basis.from_molecule(mol, path), oracle.basis_for(mol, path)


@pytest.mark.parametrize("name,mol,basis", [
    ("h2", mi.h2(1.4), "sto-3g"),
    ("h2o_sto3g", mi.h2o(), "sto-3g"),
    ("h2o_631gs", mi.h2o(), "6-31gs"),
    ("propane_sto3g", mi.alkane(3, np.random.default_rng(21)), "sto-3g"),
    ("water2_631gs", mi.water_cluster(2, 9.0, 11), "6-31gs"),
], ids=lambda x: x if isinstance(x, str) else "")
def test_scf_fp64_matches_oracle(mess, oracle_mod, name, mol, basis):
    g, o = _pair(mess, oracle_mod, mol, basis)
    r = g.scf(prec="fp64")
    ref = oracle_mod.scf(o)
    assert r["status"] == mess.MESS_OK and r["converged"] == 1
    assert abs(r["E_total"] - ref.E_total) <= 1e-8
    assert abs(r["E_nuc"] - ref.E_nuc) <= 1e-12
    assert np.abs(r["D"] - ref.D).max() <= 1e-5
    S = oracle_mod.overlap(o)
    assert np.trace(r["D"] @ S) == pytest.approx(mol.nelectron, abs=1e-8)
    assert np.abs(r["D"] @ S @ r["D"] - 2 * r["D"]).max() < 1e-6


def test_scf_szabo_ostlund_h2(mess):
    g = json.load(open(GOLDEN))["h2"]
    b = mess.Basis.from_molecule(mi.h2(g["R_bohr"]), mi.basis_path("sto-3g"))
    r = b.scf()
    assert r["E_total"] == pytest.approx(g["E_total"], abs=g["tol"])
    assert r["E_elec"] == pytest.approx(g["E_elec"], abs=g["tol"])


def test_scf_mixed_precision_energy(mess, oracle_mod):
    mol = mi.water_cluster(2, 9.0, 11)
    g, o = _pair(mess, oracle_mod, mol, "6-31gs")
    ref = oracle_mod.scf(o)
    r = g.scf(prec="mixed", schwarz_tau=1e-10)
    assert r["converged"] == 1
    assert abs(r["E_total"] - ref.E_total) <= 1e-6


def test_scf_batch_matches_individual(mess, oracle_mod):
    rng = np.random.default_rng(77)
    mols = [mi.alkane(n, rng) for n in (1, 2, 3, 1, 4)] + [mi.h2(r) for r in (0.9, 1.4, 3.0)]
    bases = [mess.Basis.from_molecule(m, mi.basis_path("sto-3g")) for m in mols]
    res, st = mess.scf_batch(bases, prec="fp64")
    assert st == mess.MESS_OK
    for m, r in zip(mols, res):
        ref = oracle_mod.scf(oracle_mod.basis_for(m, mi.basis_path("sto-3g")))
        assert r["converged"] == 1
        assert abs(r["E_total"] - ref.E_total) <= 1e-8


def test_scf_errors(mess):
    oh = mi.Molecule("oh", np.array([8, 1], dtype=np.int32), np.array([[0, 0, 0], [1.8, 0, 0]], dtype=float))
    b = mess.Basis.from_molecule(oh, mi.basis_path("sto-3g"))
    with pytest.raises(mess.MessError) as e:
        b.scf()
    assert e.value.status == mess.MESS_EINVAL
    h2o = mess.Basis.from_molecule(mi.h2o(), mi.basis_path("sto-3g"))
    r = h2o.scf(max_iter=2)
    assert r["status"] == mess.MESS_ENOCONV and r["converged"] == 0


def test_sad_guess_same_energy(mess, oracle_mod):
    for mol, basis in ((mi.h2o(), "6-31gs"), (mi.alkane(4, np.random.default_rng(9)), "sto-3g")):
        g = mess.Basis.from_molecule(mol, mi.basis_path(basis))
        rc = g.scf(guess=mess.MESS_GUESS_CORE)
        rs = g.scf(guess=mess.MESS_GUESS_SAD)
        assert rc["converged"] == 1 and rs["converged"] == 1
        assert abs(rs["E_total"] - rc["E_total"]) <= 1e-8
        assert rs["iterations"] <= rc["iterations"] + 1
