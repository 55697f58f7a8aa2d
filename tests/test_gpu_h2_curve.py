"""The batched H2 dissociation curve in Hartree-Fock form (the paper's batching over conformations,
Sec. 5.2): 64 H2 molecules with bond lengths linspace(0.6, 10) bohr, STO-3G, all in one batched
device SCF, each total energy against the oracle's SCF of the same molecule."""
import numpy as np
import pytest

import mess_inputs as mi

pytestmark = pytest.mark.gpu

RS = np.linspace(0.6, 10.0, 64)


@pytest.fixture(scope="module")
def curve(mess, oracle_mod):
    path = mi.basis_path("sto-3g")
    mols = [mi.h2(float(r)) for r in RS]
    bases = [mess.Basis.from_molecule(m, path) for m in mols]
    ref = [oracle_mod.scf(oracle_mod.basis_for(m, path)) for m in mols]
    assert all(r.converged for r in ref)
    return bases, np.array([r.E_total for r in ref])


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-8), ("mixed", 1e-6)])
def test_batched_h2_curve_matches_oracle(mess, curve, prec, tol):
    bases, Eref = curve
    res, st = mess.scf_batch(bases, prec=prec, split_df32=(prec == "mixed"))
    assert st == mess.MESS_OK
    E = np.array([r["E_total"] for r in res])
    assert all(r["converged"] == 1 for r in res)
    assert np.abs(E - Eref).max() <= tol, np.abs(E - Eref).max()
    # the curve's shape: repulsive wall at 0.6 bohr, a single minimum near 1.35 bohr, and the
    # minimal-basis RHF approach to dissociation from below the limit (E increases monotonically)
    k = int(np.argmin(E))
    assert 1.2 < RS[k] < 1.5
    assert np.all(np.diff(E[:k + 1]) < 0) and np.all(np.diff(E[k:]) > 0)
