"""Nuclear gradient of the Hartree-Fock energy on the GPU (analytic, and numerical from one batched SCF
of the displaced geometries) against the oracle's numerical derivative of its own SCF energy
(hartree/bohr), on distorted geometries."""
import numpy as np
import pytest

import mess_inputs as mi
from oracle import gradient as og

pytestmark = pytest.mark.gpu


def _distorted(mol, seed, scale=0.1):
    return mi.Molecule(mol.name + "_d", mol.Z, mol.xyz + np.random.default_rng(seed).normal(scale=scale, size=mol.xyz.shape))


@pytest.mark.parametrize("name,mol,basis", [
    ("h2o_sto3g", _distorted(mi.h2o(), 1), "sto-3g"),
    ("h2o_631g", _distorted(mi.h2o(), 2), "6-31g"),
    ("ch4_sto3g", _distorted(mi.alkane(1, np.random.default_rng(4)), 3), "sto-3g"),
], ids=lambda x: x if isinstance(x, str) else "")
def test_gradient_matches_the_oracle(mess, name, mol, basis):
    path = mi.basis_path(basis)
    g = mess.Basis.from_molecule(mol, path)
    r, grad = g.gradient(prec="fp64", conv_E=1e-12, conv_comm=1e-10)
    assert r["converged"] == 1
    ref = og.fd_gradient(mol.Z, mol.xyz, path)
    print(name, "max |dG| =", np.abs(grad - ref).max())
    assert np.abs(grad - ref).max() <= 1e-6
    assert np.abs(grad.sum(axis=0)).max() <= 1e-8


def test_gradient_with_d_shells_matches_the_oracle(mess):
    """H2O in 6-31G* (d shells on O): mess_gradient takes the numerical form, one batched FP64 SCF of
    the 36 displaced geometries, against the oracle's numerical derivative of its own SCF energy."""
    mol = _distorted(mi.h2o(), 5)
    path = mi.basis_path("6-31gs")
    g = mess.Basis.from_molecule(mol, path)
    r, grad = g.gradient(prec="fp64", conv_E=1e-12, conv_comm=1e-10)
    assert r["converged"] == 1
    ref = og.fd_gradient(mol.Z, mol.xyz, path)
    print("h2o_631gs max |dG| =", np.abs(grad - ref).max())
    assert np.abs(grad - ref).max() <= 1e-6
    assert np.abs(grad.sum(axis=0)).max() <= 1e-6


def test_numerical_gradient_matches_the_analytic_one(mess):
    """The numerical form against the analytic one on a basis both cover (CH4, 6-31G), both on the GPU:
    the two share no step beyond the SCF."""
    mol = _distorted(mi.alkane(1, np.random.default_rng(6)), 7)
    g = mess.Basis.from_molecule(mol, mi.basis_path("6-31g"))
    kw = dict(prec="fp64", conv_E=1e-12, conv_comm=1e-10)
    ra, ga = g.gradient(**kw)
    rn, gn = g.gradient(numerical=True, **kw)
    assert ra["converged"] == 1 and rn["converged"] == 1
    assert abs(ra["E_total"] - rn["E_total"]) <= 1e-9
    print("ch4_631g max |numerical - analytic| =", np.abs(gn - ga).max())
    assert np.abs(gn - ga).max() <= 1e-7


def test_kohn_sham_gradient_matches_the_oracle(mess, oracle_mod):
    """LDA on a distorted H2O in STO-3G: mess_gradient takes the numerical form (one batched Kohn-Sham
    SCF of the 36 displaced geometries, each on its own atom-centred grid), against the fourth-order
    central difference of the oracle's Kohn-Sham energy on its own grid."""
    from oracle import dft
    mol = _distorted(mi.h2o(), 8)
    path = mi.basis_path("sto-3g")
    g = mess.Basis.from_molecule(mol, path)
    r, grad = g.gradient(prec="fp64", xc="lda", conv_E=1e-12, conv_comm=1e-10)
    assert r["converged"] == 1
    h = 1e-3
    ref = np.zeros_like(mol.xyz)
    for a in range(len(mol.Z)):
        for x in range(3):
            e = []
            for k in (2, 1, -1, -2):
                p = mol.xyz.copy()
                p[a, x] += k * h
                e.append(dft.ks_scf(oracle_mod.make_basis(mol.Z, p, path), "lda", conv_E=1e-12, conv_comm=1e-10)[0])
            ref[a, x] = (-e[0] + 8.0 * e[1] - 8.0 * e[2] + e[3]) / (12.0 * h)
    print("h2o_sto3g_lda max |dG| =", np.abs(grad - ref).max())
    assert np.abs(grad - ref).max() <= 1e-6
