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
    """Trained on converged densities of small alkanes (n = 1..6), the learned guess is checked on
    unseen longer ones (n = 7..8): its energy error after one diagonalisation of its Fock matrix must
    be below that of the SAD guess (and far below the core-Hamiltonian guess's), it must converge in
    fewer iterations than the core-Hamiltonian guess, and every guess reaches the same energy."""
    sto = mi.basis_path("sto-3g")
    train = [mess.Basis.from_molecule(m, sto) for m in mi.alkane_batch(400, 1, 6, 2004)]
    test = [mess.Basis.from_molecule(m, sto) for m in mi.alkane_batch(16, 7, 8, 2005)]
    net = mess.MLP(seed=3)
    losses = net.train(train, epochs=100, batch_rows=2048, lr=5e-3, prec="mixed", split_df32=True)
    assert losses[-1] < 0.25 * losses[0]
    w = str(tmp_path / "guess.bin")
    net.save(w)
    guesses = {"core": dict(guess=mess.MESS_GUESS_CORE), "sad": dict(guess=mess.MESS_GUESS_SAD),
               "mlp": dict(guess=mess.MESS_GUESS_MLP, mlp_weights=w)}
    final, its, de1 = {}, {}, {}
    for name, kw in guesses.items():
        res, st = mess.scf_batch(test, prec="fp64", **kw)
        assert st == mess.MESS_OK
        first, _ = mess.scf_batch(test, prec="fp64", max_iter=2, **kw)
        final[name] = np.array([r["E_total"] for r in res])
        its[name] = float(np.mean([r["iterations"] for r in res]))
        de1[name] = float(np.mean([f["E_total"] - r["E_total"] for f, r in zip(first, res)]))
    print("mean SCF iterations", its, "mean energy error after one diagonalisation", de1)
    for name in ("sad", "mlp"):
        assert np.abs(final[name] - final["core"]).max() < 1e-8
    assert de1["mlp"] < de1["sad"] < de1["core"]
    assert its["mlp"] < its["core"]


def test_mlp_guess_rejects_non_minimal_basis(mess, tmp_path):
    net = mess.MLP(seed=1)
    w = str(tmp_path / "w.bin")
    net.save(w)
    b = mess.Basis.from_molecule(mi.h2o(), mi.basis_path("6-31gs"))
    with pytest.raises(mess.MessError):
        b.scf(guess=mess.MESS_GUESS_MLP, mlp_weights=w)
