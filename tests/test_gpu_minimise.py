"""Direct energy minimisation on the device (QR-orthonormalised parameters, Adam; the paper's
Sec. 5.1 single-molecule loop and Sec. 5.2 batch over conformations) against the oracle's
minimiser step by step and against the oracle's SCF energy at the end."""
import numpy as np
import pytest

import mess_inputs as mi
from oracle import minimise as om

pytestmark = pytest.mark.gpu


def test_single_molecule_reaches_the_oracle_minimum(mess, oracle_mod):
    """H2O / STO-3G, 200 Adam steps with learning rate 0.1 from Z = 1 (FP64 J/K).  The starting energy
    and the final energy are unique and equal the oracle's (and the final one the SCF energy).  The path
    in between is not unique: gradient components that vanish by the molecule's symmetry come out as
    rounding noise of either sign, and Adam's first steps (m / sqrt(v) = sign g) turn that noise into
    steps of +-lr, differently on each side; the energy must still fall to the minimum."""
    path = mi.basis_path("sto-3g")
    g = mess.Basis.from_molecule(mi.h2o(), path)
    o = oracle_mod.basis_for(mi.h2o(), path)
    r, trace, st = g.minimise(prec="fp64", steps=200, lr=0.1, grad_tol=1e-3)
    _, tref, Eref = om.adam(om.problem(o), 200)
    assert abs(trace[0] - tref[0]) <= 1e-10
    assert trace[-1] < trace[0] and abs(trace[-1] - Eref) <= 1e-8
    assert abs(r["E_total"] - Eref) <= 1e-8
    assert abs(r["E_total"] - oracle_mod.scf(o).E_total) <= 1e-8
    assert st == mess.MESS_OK and r["converged"] == 1


def test_batched_h2_curve_by_minimisation(mess, oracle_mod):
    """The paper's batched example in Hartree-Fock form: 64 H2 molecules, bond lengths
    linspace(0.6, 10) bohr, STO-3G, one Adam loop of 128 steps (learning rate 0.1, Z = 1) over the
    whole batch; each molecule's trajectory equals the oracle's for that molecule alone (H2 has no
    gradient component that vanishes only up to rounding: the ones that vanish are exact zeros)."""
    path = mi.basis_path("sto-3g")
    rs = np.linspace(0.6, 10.0, 64)
    mols = [mi.h2(float(r)) for r in rs]
    bases = [mess.Basis.from_molecule(m, path) for m in mols]
    res, trace, st = mess.minimise_batch(bases, prec="fp64", steps=128, lr=0.1)
    assert trace.shape == (128, 64)
    for k in range(0, 64, 7):
        o = oracle_mod.basis_for(mols[k], path)
        _, tref, Eref = om.adam(om.problem(o), 128)
        assert np.abs(trace[:, k] - tref).max() <= 1e-8
        assert abs(res[k]["E_total"] - Eref) <= 1e-8
        assert abs(res[k]["E_total"] - oracle_mod.scf(o).E_total) <= 1e-6
    E = np.array([r["E_total"] for r in res])
    k = int(np.argmin(E))
    assert 1.2 < rs[k] < 1.5
