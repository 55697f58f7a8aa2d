"""The batched device SCF (every molecule of the batch in the same launches, one CUDA graph per
iteration, converged molecules leaving on the device) on 64 molecules of different sizes, each
total energy against the oracle's SCF of that molecule."""
import numpy as np
import pytest

import mess_inputs as mi

pytestmark = pytest.mark.gpu


def _scaled(mol, f):
    return mi.Molecule(f"{mol.name}_x{f:.3f}", mol.Z, mol.xyz * f)


def _batch():
    """24 waters and 24 methanes with bond lengths scaled by 0.85..1.25, 16 ethane conformers
    (random torsion), STO-3G: 7, 9 and 16 functions."""
    rng = np.random.default_rng(64)
    mols = [_scaled(mi.h2o(), f) for f in np.linspace(0.85, 1.25, 24)]
    ch4 = mi.alkane(1, np.random.default_rng(5))
    mols += [_scaled(ch4, f) for f in np.linspace(0.85, 1.25, 24)]
    mols += [mi.alkane(2, rng) for _ in range(16)]
    return mols


@pytest.fixture(scope="module")
def batch(mess, oracle_mod):
    path = mi.basis_path("sto-3g")
    mols = _batch()
    bases = [mess.Basis.from_molecule(m, path) for m in mols]
    ref = [oracle_mod.scf(oracle_mod.basis_for(m, path)) for m in mols]
    assert all(r.converged for r in ref)
    return mols, bases, np.array([r.E_total for r in ref]), [r.iterations for r in ref]


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-8), ("mixed", 1e-6)])
def test_batch_of_64_matches_oracle(mess, batch, prec, tol):
    mols, bases, Eref, _ = batch
    assert len(bases) == 64
    res, st = mess.scf_batch(bases, prec=prec, schwarz_tau=1e-12, split_df32=(prec == "mixed"))
    assert st == mess.MESS_OK
    assert all(r["converged"] == 1 for r in res)
    E = np.array([r["E_total"] for r in res])
    assert np.abs(E - Eref).max() <= tol, np.abs(E - Eref).max()
    if prec == "mixed":
        # the iterations' own (reduced-precision) energies, before the final full-precision evaluation
        Ei = np.array([r["E_iter"] for r in res])
        assert np.abs(Ei - Eref).max() <= 1e-5


def test_batch_iterations_match_single_molecule_runs(mess, batch):
    """A molecule's SCF in the batch follows the same iterations as on its own: molecules that
    converge early leave without disturbing the others.  The iteration at which the thresholds
    (|dE| < 1e-10, max|FDS - SDF| < 1e-8) are first met depends on round-off: the J/K builds sum
    with FP64 atomics in no fixed order, and repeated single-molecule runs of the stretched methanes
    of this batch stop after 7, 8 or 10 iterations.  So the counts agree to within 3, and on average
    to within 1."""
    mols, bases, _, _ = batch
    res, st = mess.scf_batch(bases, prec="fp64")
    assert st == mess.MESS_OK
    diffs = []
    for k in (0, 23, 24, 47, 48, 63):
        r1 = bases[k].scf(prec="fp64")
        assert abs(r1["E_total"] - res[k]["E_total"]) <= 1e-9
        diffs.append(abs(r1["iterations"] - res[k]["iterations"]))
    assert max(diffs) <= 3 and sum(diffs) / len(diffs) <= 1.0, diffs
