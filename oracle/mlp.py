"""Oracle of the learned-guess network: descriptors, pair-frame targets, forward and backward.

TEST INFRASTRUCTURE ONLY (same rules as the rest of ``oracle/``).  Plain numpy in FP64, written
from the definitions (the library header states them): descriptor of the ordered atom pair (i, j),
a 112 -> 256 -> 256 -> 25 perceptron with SiLU activations, masked mean squared error.  With
``bf16=True`` the values the GPU kernels round to BF16 (inputs, weights, activations fed to the next
product, back-propagated products) are rounded the same way, so the GPU's FP32 accumulation can be
compared with exact FP64 sums; with ``bf16=False`` it is the exact-arithmetic network used by the
finite-difference pin.

parity: pinned by tests/test_oracle_mlp.py (the loss and two gradient entries of a hand-set network
worked out by hand; central finite differences of the loss; descriptor closed forms for a diatomic;
frame orthonormality; the atomic target block equal to the average over the cube's rotations).
"""
from __future__ import annotations

import math

import numpy as np

DIN, WID, DOUT, DOUT_PAD, NRBF = 112, 256, 25, 32, 32
_ELEM = {1: 0, 6: 1, 7: 2, 8: 3}


def bf16(x):
    """Round to the nearest BF16 value (ties to even), returned as float64."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def rbf(r):
    mu = 10.0 * np.arange(NRBF) / (NRBF - 1)
    return np.exp(-2.0 * (r - mu) ** 2)


def pair_frame(ri, rj):
    """Rows x', y', z': z' along rj - ri, x' = normalise(z' x e) with e the least aligned lab axis."""
    z = (np.asarray(rj) - np.asarray(ri)) / np.linalg.norm(np.asarray(rj) - np.asarray(ri))
    a = int(np.argmin(np.abs(z)))
    e = np.zeros(3)
    e[a] = 1.0
    x = np.cross(z, e)
    x /= np.linalg.norm(x)
    y = np.cross(z, x)
    return np.array([x, y, z])


def descriptors(Z, xyz):
    """Rows i * natom + j: one-hots, i == j flag, radial basis of r_ij, environments of i and j."""
    Z = np.asarray(Z)
    xyz = np.asarray(xyz, dtype=np.float64).reshape(-1, 3)
    na = len(Z)
    X = np.zeros((na * na, DIN))
    env = np.zeros((na, NRBF))
    for i in range(na):
        for k in range(na):
            if k != i:
                env[i] += 0.25 * rbf(np.linalg.norm(xyz[k] - xyz[i]))
    for i in range(na):
        for j in range(na):
            row = X[i * na + j]
            row[_ELEM[int(Z[i])]] = 1.0
            row[4 + _ELEM[int(Z[j])]] = 1.0
            row[8] = 1.0 if i == j else 0.0
            row[9:41] = rbf(np.linalg.norm(xyz[j] - xyz[i]))
            row[41:73] = env[i]
            row[73:105] = env[j]
    return X


def _tmat(nf, R):
    if nf == 1:
        return np.ones((1, 1))
    T = np.eye(5)
    T[2:, 2:] = R
    return T


def targets(Z, xyz, atom_funcs, D):
    """Pair-frame density blocks T_i D_ij T_j^T (i != j) and rotation-averaged atomic blocks."""
    Z = np.asarray(Z)
    xyz = np.asarray(xyz, dtype=np.float64).reshape(-1, 3)
    na = len(Z)
    T = np.zeros((na * na, DOUT))
    M = np.zeros((na * na, DOUT))
    for i in range(na):
        fi, ni = atom_funcs[i]
        for j in range(na):
            fj, nj = atom_funcs[j]
            blk = D[fi:fi + ni, fj:fj + nj]
            if i == j:
                b = np.zeros((ni, ni))
                b[:min(ni, 2), :min(ni, 2)] = blk[:min(ni, 2), :min(ni, 2)]
                if ni == 5:
                    b[2:, 2:] = np.eye(3) * np.trace(blk[2:, 2:]) / 3.0
            else:
                R = pair_frame(xyz[i], xyz[j])
                b = _tmat(ni, R) @ blk @ _tmat(nj, R).T
            out = np.zeros((5, 5))
            mk = np.zeros((5, 5))
            out[:ni, :nj] = b
            mk[:ni, :nj] = 1.0
            T[i * na + j] = out.ravel()
            M[i * na + j] = mk.ravel()
    return T, M


def unpack(p):
    p = np.asarray(p, dtype=np.float64)
    o = 0
    W1 = p[o:o + DIN * WID].reshape(DIN, WID); o += DIN * WID
    b1 = p[o:o + WID]; o += WID
    W2 = p[o:o + WID * WID].reshape(WID, WID); o += WID * WID
    b2 = p[o:o + WID]; o += WID
    W3 = p[o:o + WID * DOUT_PAD].reshape(WID, DOUT_PAD); o += WID * DOUT_PAD
    b3 = p[o:o + DOUT_PAD]; o += DOUT_PAD
    return W1, b1, W2, b2, W3, b3


def silu(z):
    return z / (1.0 + np.exp(-z))


def dsilu(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def loss_grad(p, X, T, M, bf16_mode=True):
    """Masked mean squared error of the network and its gradient (flat, same layout as p)."""
    r = bf16 if bf16_mode else (lambda v: np.asarray(v, dtype=np.float64))
    W1, b1, W2, b2, W3, b3 = unpack(p)
    Xb, W1b, W2b, W3b = r(X), r(W1), r(W2), r(W3)
    Z1 = Xb @ W1b + b1
    A1 = r(silu(Z1))
    Z2 = A1 @ W2b + b2
    A2 = r(silu(Z2))
    Y = A2 @ W3b + b3
    count = float(np.sum(M))
    diff = Y[:, :DOUT] - T
    loss = float(np.sum(M * diff * diff)) / count
    dY = np.zeros_like(Y)
    dY[:, :DOUT] = 2.0 * M * diff / count
    dY = r(dY)
    gW3 = A2.T @ dY
    gb3 = dY.sum(axis=0)
    dZ2 = r((dY @ W3b.T) * dsilu(Z2))
    gW2 = A1.T @ dZ2
    gb2 = dZ2.sum(axis=0)
    dZ1 = r((dZ2 @ W2b.T) * dsilu(Z1))
    gW1 = Xb.T @ dZ1
    gb1 = dZ1.sum(axis=0)
    g = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3.ravel(), gb3])
    return loss, g


def random_params(seed, scale=1.0):
    rng = np.random.default_rng(seed)
    W1 = rng.uniform(-1, 1, (DIN, WID)) / math.sqrt(DIN) * scale
    W2 = rng.uniform(-1, 1, (WID, WID)) / math.sqrt(WID) * scale
    W3 = rng.uniform(-1, 1, (WID, DOUT_PAD)) / math.sqrt(WID) * scale
    W3[:, DOUT:] = 0.0
    return np.concatenate([W1.ravel(), rng.normal(0, 0.1, WID), W2.ravel(), rng.normal(0, 0.1, WID),
                           W3.ravel(), rng.normal(0, 0.1, DOUT_PAD)])
