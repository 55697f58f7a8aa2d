"""Pins for the oracle of the learned-guess network (CPU only)."""
import numpy as np
import pytest

import mess_inputs as mi
from oracle import mlp as om


def test_finite_difference_gradient():
    rng = np.random.default_rng(3)
    rows = 24
    X = rng.normal(size=(rows, om.DIN)) * 0.5
    T = rng.normal(size=(rows, om.DOUT))
    M = (rng.random((rows, om.DOUT)) < 0.7).astype(float)
    p = om.random_params(5)
    _, g = om.loss_grad(p, X, T, M, bf16_mode=False)
    W3_off = om.DIN * om.WID + om.WID + om.WID * om.WID + om.WID
    idx = [0, 17, om.DIN * om.WID + 3, om.DIN * om.WID + om.WID + 1000, W3_off + 7, len(p) - om.DOUT_PAD + 2]
    h = 1e-6
    for k in idx:
        e = np.zeros_like(p)
        e[k] = h
        lp, _ = om.loss_grad(p + e, X, T, M, bf16_mode=False)
        lm, _ = om.loss_grad(p - e, X, T, M, bf16_mode=False)
        fd = (lp - lm) / (2 * h)
        assert g[k] == pytest.approx(fd, rel=1e-5, abs=1e-9)
    # unused output columns get no gradient
    W3 = g[W3_off:W3_off + om.WID * om.DOUT_PAD].reshape(om.WID, om.DOUT_PAD)
    assert np.all(W3[:, om.DOUT:] == 0.0)


def test_bf16_rounding():
    assert om.bf16(1.0) == 1.0
    assert om.bf16(1.0 + 2 ** -9) == 1.0                     # tie to even
    assert om.bf16(1.0 + 3 * 2 ** -9) == 1.0 + 2 ** -7       # 1.0117 -> 1.015625
    assert abs(om.bf16(np.pi) - np.pi) < 2 ** -7 * np.pi


def test_descriptor_closed_forms_and_frames():
    mol = mi.h2(1.4)
    X = om.descriptors(mol.Z, mol.xyz)
    assert X.shape == (4, om.DIN)
    mu = 10.0 * np.arange(32) / 31
    # off-diagonal pair: radial basis of r = 1.4; environment of each H = 1/4 of the same
    np.testing.assert_allclose(X[1, 9:41], np.exp(-2.0 * (1.4 - mu) ** 2), rtol=1e-14)
    np.testing.assert_allclose(X[1, 41:73], 0.25 * np.exp(-2.0 * (1.4 - mu) ** 2), rtol=1e-14)
    assert X[0, 8] == 1.0 and X[1, 8] == 0.0 and X[0, 0] == 1.0 and X[0, 4] == 1.0
    R = om.pair_frame([0.3, -1.0, 2.0], [1.1, 0.5, -0.7])
    np.testing.assert_allclose(R @ R.T, np.eye(3), atol=1e-14)
    assert np.linalg.det(R) == pytest.approx(1.0)


def test_targets_invert():
    """A lab-frame block rotated into the pair frame and back is unchanged."""
    rng = np.random.default_rng(1)
    D = rng.normal(size=(10, 10))
    D = D + D.T
    Z = [6, 6]
    xyz = np.array([[0.0, 0.0, 0.0], [1.3, -0.4, 2.1]])
    T, M = om.targets(Z, xyz, [(0, 5), (5, 5)], D)
    R = om.pair_frame(xyz[0], xyz[1])
    Tm = om._tmat(5, R)
    back = Tm.T @ T[1].reshape(5, 5) @ Tm
    np.testing.assert_allclose(back, D[0:5, 5:10], atol=1e-12)
    assert M.sum() == 4 * 25
