"""Small helpers shared by the oracle tests (no integral arithmetic)."""
import numpy as np


def prim_basis(oracle, prims):
    """An oracle basis of single unnormalised primitives (coefficient 1): prims = [(alpha, A, lmn)]."""
    n = len(prims)
    return oracle.Basis(
        n,
        np.ascontiguousarray([p[1] for p in prims], dtype=np.float64),
        np.ascontiguousarray([p[2] for p in prims], dtype=np.int32),
        np.ones(n, np.int32), np.arange(n, dtype=np.int32),
        np.array([p[0] for p in prims], dtype=np.float64), np.ones(n),
        np.arange(n, dtype=np.int32), n, np.zeros(n, np.int32),
        np.array([1], np.int32), np.zeros((1, 3)))


def function_primitives(b, m):
    """The primitives of contracted function m of an oracle basis: [(coef, (alpha, A, lmn))]."""
    out = []
    for k in range(b.nprim[m]):
        out.append((b.coefs[b.poff[m] + k],
                    (b.exps[b.poff[m] + k], b.center[m], tuple(int(v) for v in b.lmn[m]))))
    return out
