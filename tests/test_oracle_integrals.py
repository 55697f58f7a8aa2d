"""Pins for the oracle's one- and two-electron integrals (independent of its closed forms)."""
import itertools
import json
import math
import os

import numpy as np
import pytest

import mess_inputs as mi
import quadrature as Q
from oracle_helpers import function_primitives, prim_basis

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "szabo_ostlund_minimal_basis.json")


def _lmn_of(l, rng):
    comps = [(lx, ly, l - lx - ly) for lx in range(l, -1, -1) for ly in range(l - lx, -1, -1)]
    return comps[rng.integers(len(comps))]


def _random_prims(rng, ls):
    return [(float(rng.uniform(0.3, 2.5)), rng.normal(scale=0.8, size=3), _lmn_of(l, rng)) for l in ls]


def test_self_overlap_is_one_for_every_cartesian_component(oracle_mod):
    for name in ("sto-3g", "6-31gs"):
        b = oracle_mod.basis_for(mi.h2o(), mi.basis_path(name))
        S = oracle_mod.overlap(b)
        assert np.allclose(np.diag(S), 1.0, atol=1e-13)


def test_h2o_function_counts(oracle_mod):
    assert oracle_mod.basis_for(mi.h2o(), mi.basis_path("sto-3g")).nfn == 7
    assert oracle_mod.basis_for(mi.h2o(), mi.basis_path("6-31gs")).nfn == 19
    assert oracle_mod.basis_for(mi.water_cluster(8, 12.0, 2002), mi.basis_path("6-31gs")).nfn == 152


@pytest.mark.parametrize("seed", range(6))
def test_one_electron_vs_quadrature(oracle_mod, seed):
    rng = np.random.default_rng(100 + seed)
    prims = _random_prims(rng, [0, 1, 2, 2, 1])
    b = prim_basis(oracle_mod, prims)
    S, T, _ = oracle_mod.one_e(b)
    for i, j in itertools.product(range(len(prims)), repeat=2):
        assert S[i, j] == pytest.approx(Q.overlap(prims[i], prims[j]), rel=1e-12, abs=1e-15)
        assert T[i, j] == pytest.approx(Q.kinetic(prims[i], prims[j]), rel=1e-11, abs=1e-14)


@pytest.mark.parametrize("seed", range(4))
def test_nuclear_attraction_vs_quadrature(oracle_mod, seed):
    rng = np.random.default_rng(200 + seed)
    prims = _random_prims(rng, [0, 1, 2])
    charges = [(3, rng.normal(size=3)), (1, rng.normal(size=3))]
    b = prim_basis(oracle_mod, prims)
    b.Z = np.array([c[0] for c in charges], dtype=np.int32)
    b.xyz = np.ascontiguousarray([c[1] for c in charges])
    _, _, V = oracle_mod.one_e(b)
    for i, j in itertools.product(range(3), repeat=2):
        ref = -sum(z * Q.nuclear(prims[i], prims[j], c) for z, c in charges)
        assert V[i, j] == pytest.approx(ref, rel=1e-11, abs=1e-14)


# every (la lb | lc ld) class up to (dd|dd), one random quartet each
_CLASSES = [c for c in itertools.product(range(3), repeat=4)]


@pytest.mark.parametrize("cls", _CLASSES)
def test_eri_primitive_vs_quadrature(oracle_mod, cls):
    rng = np.random.default_rng(1000 + sum(v * 3 ** i for i, v in enumerate(cls)))
    prims = _random_prims(rng, cls)
    b = prim_basis(oracle_mod, prims)
    ref = Q.eri(*prims)
    val = oracle_mod.eri(b, 0, 1, 2, 3)
    assert val == pytest.approx(ref, rel=1e-11, abs=1e-15)


def test_contracted_eri_vs_quadrature(oracle_mod):
    """A contracted O 1s (6 primitives) / d / p quartet of real 6-31G* water functions."""
    b = oracle_mod.basis_for(mi.h2o(), mi.basis_path("6-31gs"))
    # functions: O 1s = 0, O 2s = 1, O 2p = 2..4, O 3s = 5, O 3p = 6..8, O d = 9..14, H...
    for quartet in [(0, 9, 2, 15), (10, 9, 13, 17), (0, 0, 0, 0)]:
        ref = 0.0
        for terms in itertools.product(*[function_primitives(b, m) for m in quartet]):
            c = math.prod(t[0] for t in terms)
            ref += c * Q.eri(*[t[1] for t in terms])
        assert oracle_mod.eri(b, *quartet) == pytest.approx(ref, rel=1e-11, abs=1e-14)


def test_ssss_closed_form(oracle_mod):
    rng = np.random.default_rng(7)
    for _ in range(5):
        prims = _random_prims(rng, [0, 0, 0, 0])
        (a, A, _), (bb, B, _), (c, C, _), (d, Dd, _) = prims
        p, q = a + bb, c + d
        P, Qc = (a * A + bb * B) / p, (c * C + d * Dd) / q
        Kab = math.exp(-a * bb / p * np.sum((A - B) ** 2))
        Kcd = math.exp(-c * d / q * np.sum((C - Dd) ** 2))
        T = p * q / (p + q) * float(np.sum((P - Qc) ** 2))
        F0 = 0.5 * math.sqrt(math.pi / T) * math.erf(math.sqrt(T))
        ref = 2 * math.pi ** 2.5 / (p * q * math.sqrt(p + q)) * Kab * Kcd * F0
        val = oracle_mod.eri(prim_basis(oracle_mod, prims), 0, 1, 2, 3)
        assert val == pytest.approx(ref, rel=1e-13)


def test_szabo_ostlund_h2_integrals(oracle_mod):
    g = json.load(open(GOLDEN))["h2"]
    b = oracle_mod.basis_for(mi.h2(g["R_bohr"]), mi.basis_path("sto-3g"))
    S, T, V = oracle_mod.one_e(b)
    tol = g["tol"]
    assert S[0, 1] == pytest.approx(g["S12"], abs=tol)
    assert T[0, 0] == pytest.approx(g["T11"], abs=tol)
    assert T[0, 1] == pytest.approx(g["T12"], abs=tol)
    # V of the book is per nucleus; by symmetry V_11(total) = V1_11 + V1_22
    assert V[0, 0] == pytest.approx(g["V1_11"] + g["V1_22"], abs=2 * tol)
    assert V[0, 1] == pytest.approx(2 * g["V1_12"], abs=2 * tol)
    H = T + V
    assert H[0, 0] == pytest.approx(g["Hcore11"], abs=tol)
    assert H[0, 1] == pytest.approx(g["Hcore12"], abs=tol)
    assert oracle_mod.eri(b, 0, 0, 0, 0) == pytest.approx(g["eri_1111"], abs=tol)
    assert oracle_mod.eri(b, 0, 0, 1, 1) == pytest.approx(g["eri_1122"], abs=tol)
    assert oracle_mod.eri(b, 1, 0, 0, 0) == pytest.approx(g["eri_2111"], abs=tol)
    assert oracle_mod.eri(b, 1, 0, 1, 0) == pytest.approx(g["eri_2121"], abs=tol)


def test_heh_plus_overlap(oracle_mod, tmp_path):
    g = json.load(open(GOLDEN))
    h, z = g["heh_plus"], g["sto1g_zeta1_expansion"]
    path = tmp_path / "heh.basis"
    lines = []
    for sym, zeta in (("He", h["zeta_He"]), ("H", h["zeta_H"])):
        lines += [f"element {sym}", "S 3"]
        lines += [f"{e * zeta ** 2:.10f} {c}" for e, c in zip(z["exponents"], z["coefficients"])]
    path.write_text("\n".join(lines) + "\n")
    b = oracle_mod.make_basis([2, 1], [[0, 0, 0], [h["R_bohr"], 0, 0]], str(path))
    assert oracle_mod.overlap(b)[0, 1] == pytest.approx(h["S12"], abs=h["tol_S"])


def test_eri_tensor_symmetry_schwarz_and_psd(oracle_mod):
    b = oracle_mod.basis_for(mi.h2o(), mi.basis_path("sto-3g"))
    G = oracle_mod.eri_tensor(b)
    n = b.nfn
    for perm in [(1, 0, 2, 3), (0, 1, 3, 2), (2, 3, 0, 1), (3, 2, 1, 0)]:
        assert np.allclose(G, G.transpose(perm), atol=1e-14)
    diag = np.einsum("ijij->ij", G)
    bound = np.sqrt(np.abs(diag)[:, :, None, None] * np.abs(diag)[None, None, :, :])
    assert np.all(np.abs(G) <= bound + 1e-14)
    M = G.reshape(n * n, n * n)
    assert np.linalg.eigvalsh(M).min() > -1e-12
    # 406 distinct values up to 8-fold symmetry for 7 functions
    uniq = {tuple(sorted([tuple(sorted((i, j))), tuple(sorted((k, l)))]))
            for i, j, k, l in itertools.product(range(n), repeat=4)}
    assert len(uniq) == 406


def test_translation_invariance(oracle_mod):
    mol = mi.h2o()
    b0 = oracle_mod.basis_for(mol, mi.basis_path("6-31gs"))
    b1 = oracle_mod.make_basis(mol.Z, mol.xyz + np.array([0.7, -1.3, 2.2]), mi.basis_path("6-31gs"))
    for q in [(0, 9, 2, 15), (10, 9, 13, 17), (14, 11, 12, 16)]:
        assert oracle_mod.eri(b0, *q) == pytest.approx(oracle_mod.eri(b1, *q), rel=1e-12, abs=1e-15)
