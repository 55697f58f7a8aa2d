"""Learned-guess network on the GPU (through the C ABI) against the oracle, and what it gains."""
import numpy as np
import pytest

import mess_inputs as mi
from oracle import mlp as om

pytestmark = pytest.mark.gpu


def _atom_funcs(o):
    out = []
    for a in range(len(o.Z)):
        idx = np.nonzero(o.atom == a)[0]
        out.append((int(idx[0]), len(idx)))
    return out


@pytest.fixture(scope="module")
def propane(oracle_mod):
    mol = mi.alkane(3, np.random.default_rng(21))
    o = oracle_mod.basis_for(mol, mi.basis_path("sto-3g"))
    r = oracle_mod.scf(o)
    return mol, o, r.D


def test_features_and_targets_match_oracle(mess, propane):
    mol, o, D = propane
    g = mess.Basis.from_molecule(mol, mi.basis_path("sto-3g"))
    X, T, M = mess.mlp_features(g, D)
    Xr = om.descriptors(mol.Z, mol.xyz)
    Tr, Mr = om.targets(mol.Z, mol.xyz, _atom_funcs(o), D)
    assert np.abs(X - Xr).max() < 2e-6
    assert np.array_equal(M, Mr.astype(np.float32))
    assert np.abs(T - Tr).max() < 2e-6


def test_loss_and_gradient_match_oracle(mess, propane):
    mol, o, D = propane
    g = mess.Basis.from_molecule(mol, mi.basis_path("sto-3g"))
    X, T, M = mess.mlp_features(g, D)
    p = om.random_params(7).astype(np.float32)
    net = mess.MLP(seed=1)
    net.set_params(p)
    loss, grad = net.loss_grad(X, T, M)
    lr, gr = om.loss_grad(p.astype(np.float64), X.astype(np.float64), T.astype(np.float64), M.astype(np.float64))
    assert loss == pytest.approx(lr, rel=2e-3)
    assert np.linalg.norm(grad - gr) <= 2e-2 * np.linalg.norm(gr)
    # each layer's weight gradient separately
    offs = [0, om.DIN * om.WID, om.DIN * om.WID + om.WID, om.DIN * om.WID + om.WID + om.WID * om.WID]
    for a, b in zip(offs[:-1], offs[1:]):
        assert np.linalg.norm(grad[a:b] - gr[a:b]) <= 3e-2 * np.linalg.norm(gr[a:b]) + 1e-12


def test_training_gains_over_the_plain_guesses(mess, tmp_path):
    train = mi.alkane_batch(48, 1, 4, 2004)
    test = mi.alkane_batch(4, 5, 6, 2005)
    bases = [mess.Basis.from_molecule(m, mi.basis_path("sto-3g")) for m in train]
    net = mess.MLP(seed=3)
    losses = net.train(bases, epochs=40, batch_rows=512, lr=2e-3, prec="fp64")
    assert losses[-1] < 0.25 * losses[0]
    w = str(tmp_path / "guess.bin")
    net.save(w)
    its = {"core": [], "sad": [], "mlp": []}
    for m in test:
        b = mess.Basis.from_molecule(m, mi.basis_path("sto-3g"))
        rc = b.scf(guess=mess.MESS_GUESS_CORE)
        rs = b.scf(guess=mess.MESS_GUESS_SAD)
        rm = b.scf(guess=mess.MESS_GUESS_MLP, mlp_weights=w)
        for r in (rc, rs, rm):
            assert r["converged"] == 1
        assert abs(rm["E_total"] - rc["E_total"]) < 1e-8 and abs(rs["E_total"] - rc["E_total"]) < 1e-8
        its["core"].append(rc["iterations"])
        its["sad"].append(rs["iterations"])
        its["mlp"].append(rm["iterations"])
    print("mean SCF iterations", {k: float(np.mean(v)) for k, v in its.items()})
    assert np.mean(its["mlp"]) < np.mean(its["core"])
    assert np.mean(its["sad"]) < np.mean(its["core"])


def test_mlp_guess_rejects_non_minimal_basis(mess, tmp_path):
    net = mess.MLP(seed=1)
    w = str(tmp_path / "w.bin")
    net.save(w)
    b = mess.Basis.from_molecule(mi.h2o(), mi.basis_path("6-31gs"))
    with pytest.raises(mess.MessError):
        b.scf(guess=mess.MESS_GUESS_MLP, mlp_weights=w)
