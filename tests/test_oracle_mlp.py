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


def _hand_network():
    """Weights zero except W1[0,0] = 1, W2[0,0] = 4/3, W3[0,0] = 4/3 and the bias b3[1] = 1/2."""
    W1 = np.zeros((om.DIN, om.WID))
    W2 = np.zeros((om.WID, om.WID))
    W3 = np.zeros((om.WID, om.DOUT_PAD))
    b1, b2, b3 = np.zeros(om.WID), np.zeros(om.WID), np.zeros(om.DOUT_PAD)
    W1[0, 0], W2[0, 0], W3[0, 0], b3[1] = 1.0, 4.0 / 3.0, 4.0 / 3.0, 0.5
    return np.concatenate([W1.ravel(), b1, W2.ravel(), b2, W3.ravel(), b3])


def test_forward_and_loss_of_a_hand_set_network():
    """Worked by hand: SiLU(z) = z / (1 + exp(-z)), so SiLU(ln 3) = (3/4) ln 3 and SiLU(0) = 0.
    Row 0 has x_0 = ln 3: layer 1 gives (3/4) ln 3, layer 2 (x 4/3) gives SiLU(ln 3) = (3/4) ln 3
    again, the output (x 4/3) is y_0 = ln 3, y_1 = b3[1] = 1/2 and every other output 0.  Row 1 has
    x = 0: y_0 = 0, y_1 = 1/2.  With targets (0, -1/2, 2) in row 0 (mask on outputs 0..2) and 1/2 in
    row 1 (mask on output 1 only) the squared errors are (ln 3)^2, 1, 4 and 0 over a mask count of
    4, so the loss is ((ln 3)^2 + 5) / 4; dL/dW3[0,0] = (2/4) (ln 3) (3/4) ln 3 = (3/8)(ln 3)^2."""
    ln3 = np.log(3.0)
    X = np.zeros((2, om.DIN))
    X[0, 0] = ln3
    T = np.zeros((2, om.DOUT))
    M = np.zeros((2, om.DOUT))
    T[0, :3] = [0.0, -0.5, 2.0]
    M[0, :3] = 1.0
    T[1, 1] = 0.5
    M[1, 1] = 1.0
    p = _hand_network()
    loss, g = om.loss_grad(p, X, T, M, bf16_mode=False)
    assert loss == pytest.approx((ln3 ** 2 + 5.0) / 4.0, rel=1e-14)
    W3_off = om.DIN * om.WID + om.WID + om.WID * om.WID + om.WID
    assert g[W3_off] == pytest.approx(3.0 / 8.0 * ln3 ** 2, rel=1e-14)
    # dL/db3[1] = (2/4) * (1/2 - (-1/2)) for row 0 + 0 for row 1 = 1/2
    assert g[W3_off + om.WID * om.DOUT_PAD + 1] == pytest.approx(0.5, rel=1e-14)


def _cube_rotations():
    """The 24 proper rotations of the cube: signed permutation matrices of determinant +1."""
    import itertools
    out = []
    for perm in itertools.permutations(range(3)):
        for signs in itertools.product((1.0, -1.0), repeat=3):
            R = np.zeros((3, 3))
            for i, (j, s) in enumerate(zip(perm, signs)):
                R[i, j] = s
            if np.linalg.det(R) > 0:
                out.append(R)
    assert len(out) == 24
    return out


def test_atomic_block_target_is_the_rotation_average():
    """The i == j target of a 5-function atom (s, s', p) is its density block averaged over
    rotations: the s/s' block unchanged, the s-p blocks averaging to zero, the p block to
    tr(D_pp)/3 times the identity.  Checked against the explicit average over the cube's 24 rotations
    (a group acting irreducibly on vectors, so the average is exact for these blocks)."""
    rng = np.random.default_rng(9)
    A = rng.normal(size=(5, 5))
    blk = A + A.T
    D = np.zeros((6, 6))
    D[:5, :5] = blk
    D[5, 5] = 0.7
    Z = [8, 1]
    xyz = np.array([[0.0, 0.0, 0.0], [0.3, 1.1, -0.8]])
    Tt, M = om.targets(Z, xyz, [(0, 5), (5, 1)], D)
    avg = np.zeros((5, 5))
    rots = _cube_rotations()
    for R in rots:
        Tm = np.eye(5)
        Tm[2:, 2:] = R
        avg += Tm @ blk @ Tm.T
    avg /= len(rots)
    np.testing.assert_allclose(Tt[0].reshape(5, 5), avg, atol=1e-14)
    assert M[0].sum() == 25
    # a one-function atom keeps its element
    assert Tt[3, 0] == pytest.approx(0.7) and M[3].sum() == 1
