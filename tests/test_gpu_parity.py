"""GPU path (through the C ABI) against the FP64 CPU oracle on the same seeded inputs."""
import numpy as np
import pytest

import mess_inputs as mi

pytestmark = pytest.mark.gpu


def _cases():
    return [
        ("h2o_sto3g", mi.h2o(), "sto-3g"),
        ("h2o_631gs", mi.h2o(), "6-31gs"),
        ("water2_631gs", mi.water_cluster(2, 9.0, 11), "6-31gs"),
        ("propane_sto3g", mi.alkane(3, np.random.default_rng(21)), "sto-3g"),
        ("ch4_631g", mi.alkane(1, np.random.default_rng(4)), "6-31g"),
    ]


CASES = _cases()
IDS = [c[0] for c in CASES]


def _pair(mess, oracle, mol, basis):
    path = mi.basis_path(basis)
    return mess.Basis.from_molecule(mol, path), oracle.basis_for(mol, path)


@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_one_electron_parity(mess, oracle_mod, case):
    _, mol, basis = case
    g, o = _pair(mess, oracle_mod, mol, basis)
    assert g.nbf == o.nfn
    S, T, V = oracle_mod.one_e(o)
    assert np.abs(g.overlap() - S).max() < 1e-12
    assert np.abs(g.kinetic() - T).max() < 1e-11
    assert np.abs(g.nuclear() - V).max() < 1e-11
    assert g.nuclear_repulsion() == pytest.approx(oracle_mod.nuclear_repulsion(mol.Z, mol.xyz), rel=1e-15)


@pytest.mark.parametrize("case", [CASES[0], CASES[1], CASES[4]], ids=[IDS[0], IDS[1], IDS[4]])
def test_eri_tensor_parity_every_class(mess, oracle_mod, case):
    """Every integral of the basis (s, p, Cartesian d: all 21 shell-quartet classes for 6-31G*)."""
    _, mol, basis = case
    g, o = _pair(mess, oracle_mod, mol, basis)
    G = g.eri_tensor()
    ref = oracle_mod.eri_tensor(o)
    assert np.abs(G - ref).max() < 1e-12 * max(1.0, np.abs(ref).max())


@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_schwarz_parity(mess, oracle_mod, case):
    _, mol, basis = case
    g, o = _pair(mess, oracle_mod, mol, basis)
    assert np.abs(g.schwarz() - oracle_mod.schwarz(o)).max() < 1e-12


@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_jk_fp64_parity(mess, oracle_mod, case):
    _, mol, basis = case
    g, o = _pair(mess, oracle_mod, mol, basis)
    D = mi.random_symmetric_density(g.nbf, 17)
    J, K, info = g.jk(D, prec="fp64")
    Jr, Kr = oracle_mod.jk(o, D)
    assert np.abs(J - Jr).max() <= 1e-8
    assert np.abs(K - Kr).max() <= 1e-8
    n = g.nbf
    assert info["function_quartets"] == (n * (n + 1) // 2) * (n * (n + 1) // 2 + 1) // 2


def test_jk_screened_parity(mess, oracle_mod):
    mol = mi.water_cluster(4, 18.0, 5)
    g, o = _pair(mess, oracle_mod, mol, "sto-3g")
    D = mi.random_symmetric_density(g.nbf, 23)
    Q = oracle_mod.schwarz(o)
    for tau in (1e-10, 1e-6):
        J, K, info = g.jk(D, prec="fp64", schwarz_tau=tau)
        Jr, Kr = oracle_mod.jk(o, D, tau=tau, Q=Q)
        assert np.abs(J - Jr).max() <= 1e-8
        assert np.abs(K - Kr).max() <= 1e-8
    full = g.jk(D, prec="fp64")[2]
    assert info["shell_quartets"] < full["shell_quartets"]


def _two_electron_energy(D, J, K):
    return 0.5 * float(np.sum(D * (J - 0.5 * K)))


@pytest.fixture(scope="module")
def water2_scf(oracle_mod):
    mol = mi.water_cluster(2, 9.0, 11)
    o = oracle_mod.basis_for(mol, mi.basis_path("6-31gs"))
    r = oracle_mod.scf(o)
    assert r.converged
    J, K = oracle_mod.jk(o, r.D)
    return mol, r.D, J, K


@pytest.mark.parametrize("prec,fp64_tau,boys64,df32,tol", [
    ("mixed", 0.0, False, False, 1e-6),    # default split (Q_ab Q_cd >= 3e-2 in FP64): the reduced-precision bar
    ("mixed", 0.0, False, True, 1e-6),     # the same split in double-float
    ("mixed", 1e-3, True, False, 1e-6),
    ("mixed", -1.0, False, False, 2e-5),   # no FP64 quartets at all: reported, not held to the bar
    ("fp32", 0.0, False, False, 2e-5),
])
def test_jk_reduced_precision_energy(mess, water2_scf, prec, fp64_tau, boys64, df32, tol):
    mol, D, Jr, Kr = water2_scf
    g = mess.Basis.from_molecule(mol, mi.basis_path("6-31gs"))
    J, K, info = g.jk(D, prec=prec, fp64_tau=fp64_tau, boys_fp64=boys64, split_df32=df32)
    dE = abs(_two_electron_energy(D, J, K) - _two_electron_energy(D, Jr, Kr))
    assert dE <= tol, dE
    assert np.abs(J - Jr).max() < 1e-4 and np.abs(K - Kr).max() < 1e-4
    if prec == "mixed" and fp64_tau >= 0:
        assert 0 < info["shell_quartets_fp64"] < info["shell_quartets"]
    else:
        assert info["shell_quartets_fp64"] == 0


@pytest.mark.parametrize("case", [CASES[1], CASES[2], CASES[3]], ids=[IDS[1], IDS[2], IDS[3]])
def test_jk_double_float_every_quartet(mess, oracle_mod, case):
    """Every quartet above a vanishing split threshold runs in double-float: FP64-class results."""
    _, mol, basis = case
    g, o = _pair(mess, oracle_mod, mol, basis)
    D = mi.random_symmetric_density(g.nbf, 29)
    J, K, info = g.jk(D, prec="mixed", fp64_tau=1e-300, split_df32=True)
    assert info["shell_quartets_fp64"] == info["shell_quartets"]
    Jr, Kr = oracle_mod.jk(o, D)
    assert np.abs(J - Jr).max() <= 1e-8
    assert np.abs(K - Kr).max() <= 1e-8


def test_jk_device_matches_host(mess):
    import torch
    mol = mi.water_cluster(2, 9.0, 11)
    g = mess.Basis.from_molecule(mol, mi.basis_path("6-31gs"))
    D = mi.random_symmetric_density(g.nbf, 3)
    J, K, _ = g.jk(D)
    dD = torch.from_numpy(D).cuda()
    dJ = torch.empty_like(dD)
    dK = torch.empty_like(dD)
    s = torch.cuda.current_stream()
    g.jk_device(dD, dJ, dK, stream=s)
    torch.cuda.synchronize()
    assert np.abs(dJ.cpu().numpy() - J).max() == 0.0 or np.abs(dJ.cpu().numpy() - J).max() < 1e-12
    assert np.abs(dK.cpu().numpy() - K).max() < 1e-12


@pytest.mark.parametrize("opts", [dict(prec="fp64"), dict(prec="mixed", split_df32=True), dict(prec="fp32")],
                         ids=["fp64", "mixed_df32", "fp32"])
def test_jk_device_repeated_builds(mess, opts):
    """Repeated device builds on the same buffers (replayed as one captured graph from the third call)
    follow the density's current contents and match one-off host-buffer builds."""
    import torch
    mol = mi.water_cluster(2, 9.0, 11)
    g = mess.Basis.from_molecule(mol, mi.basis_path("6-31gs"))
    Ds = [mi.random_symmetric_density(g.nbf, 40 + k) for k in range(2)]
    ref = [g.jk(D, **opts)[:2] for D in Ds]
    dD = torch.zeros((g.nbf, g.nbf), dtype=torch.float64, device="cuda")
    dJ, dK = torch.empty_like(dD), torch.empty_like(dD)
    s = torch.cuda.current_stream()
    for it in range(6):
        k = it % 2
        dD.copy_(torch.from_numpy(Ds[k]))
        info = g.jk_device(dD, dJ, dK, stream=s, **opts)
        torch.cuda.synchronize()
        assert info["function_quartets"] > 0
        assert np.abs(dJ.cpu().numpy() - ref[k][0]).max() < 1e-11
        assert np.abs(dK.cpu().numpy() - ref[k][1]).max() < 1e-11


@pytest.mark.parametrize("prec,df32", [("fp64", False), ("mixed", True), ("fp32", False)])
def test_jk_autotuned_kernels(mess, oracle_mod, water2_scf, prec, df32):
    """After the autotuner has picked a kernel per bin part, the build still matches the oracle
    (FP64: every element to 1e-8; reduced precision: the energy bar), and the profile reports
    only variants that exist."""
    import torch
    mol, D, Jr, Kr = water2_scf
    g = mess.Basis.from_molecule(mol, mi.basis_path("6-31gs"))
    kw = dict(prec=prec, split_df32=df32)
    changed = g.jk_autotune(D, reps=2, **kw)
    assert changed >= 0
    J, K, info = g.jk(D, **kw)
    e = lambda J, K: 0.5 * float(np.sum(D * (J - 0.5 * K)))  # noqa: E731
    if prec == "fp64":
        assert np.abs(J - Jr).max() <= 1e-8 and np.abs(K - Kr).max() <= 1e-8
    else:
        assert abs(e(J, K) - e(Jr, Kr)) <= (1e-6 if prec == "mixed" else 2e-5)
    dD = torch.from_numpy(D).cuda()
    dJ, dK = torch.empty_like(dD), torch.empty_like(dD)
    parts = g.jk_profile(dD, dJ, dK, **kw)
    assert len(parts) == info["kernel_launches"] - 1 - (prec != "fp64")
    for p in parts:
        assert p["G"] in (1, 4, 8, 32) and p["team"] in (0, 1, 2, 3)
        assert p["mode"] in ((0, 3) if p["fp64"] and df32 else (0,) if p["fp64"] else (2,))
        assert not (p["team"] and p["G"] != 1)
    assert np.abs(dJ.cpu().numpy() - J).max() < 1e-9


def test_jk_tuning_save_restore(mess):
    """A kernel choice read from one basis restores on another basis of the same molecule, and
    entries that name a kernel the part does not have are refused without changing anything."""
    mol = mi.water_cluster(2, 9.0, 11)
    kw = dict(prec="mixed", split_df32=True)
    g1 = mess.Basis.from_molecule(mol, mi.basis_path("6-31gs"))
    g2 = mess.Basis.from_molecule(mol, mi.basis_path("6-31gs"))
    g1.jk_set_variant(G=32, team=0, split_mode=0, **kw)
    t1 = g1.jk_tuning(**kw)
    assert {r[1] for r in t1} <= {1, 32}
    g2.jk_set_tuning(t1, **kw)
    assert g2.jk_tuning(**kw) == t1
    before = g2.jk_tuning(**kw)
    bad = [list(r) for r in t1]
    bad[0][1] = 3
    with pytest.raises(mess.MessError):
        g2.jk_set_tuning(bad, **kw)
    with pytest.raises(mess.MessError):
        g2.jk_set_tuning(t1[:-1], **kw)
    assert g2.jk_tuning(**kw) == before
    D = mi.random_symmetric_density(g1.nbf, 5)
    J1, K1, _ = g1.jk(D, **kw)
    J2, K2, _ = g2.jk(D, **kw)
    assert np.abs(J1 - J2).max() < 1e-11 and np.abs(K1 - K2).max() < 1e-11


VARIANTS = [(1, 0), (4, 0), (8, 0), (32, 0), (1, 1), (1, 2), (1, 3)]


@pytest.mark.parametrize("G,team", VARIANTS, ids=[f"G{g}_team{t}" for g, t in VARIANTS])
def test_jk_every_kernel_variant(mess, oracle_mod, G, team):
    """Each kernel variant (lanes per quartet, warp or block per quartet) on every class of a water dimer in
    6-31G*: FP64, and double-float on every quartet, against the oracle to 1e-8; FP32 on every
    quartet within the reduced-precision energy tolerance of the unsplit form."""
    mol = mi.water_cluster(2, 9.0, 11)
    g, o = _pair(mess, oracle_mod, mol, "6-31gs")
    D = mi.random_symmetric_density(g.nbf, 31)
    Jr, Kr = oracle_mod.jk(o, D)
    e = lambda J, K: 0.5 * float(np.sum(D * (J - 0.5 * K)))  # noqa: E731
    for kw, split_mode, tol in ((dict(prec="fp64"), -1, 1e-8),
                                (dict(prec="mixed", fp64_tau=1e-300, split_df32=True), 3, 1e-8),
                                (dict(prec="mixed", fp64_tau=1e-300, split_df32=True), 0, 1e-8),
                                (dict(prec="mixed", fp64_tau=-1.0), -1, None)):
        g.jk_set_variant(G=G, team=team, split_mode=split_mode, **kw)
        J, K, info = g.jk(D, **kw)
        if tol is not None:
            assert np.abs(J - Jr).max() <= tol, (kw, split_mode)
            assert np.abs(K - Kr).max() <= tol, (kw, split_mode)
        else:
            assert abs(e(J, K) - e(Jr, Kr)) <= 2e-5


def test_single_atom_and_errors(mess, oracle_mod, tmp_path):
    he = mi.Molecule("he", np.array([2], dtype=np.int32), np.zeros((1, 3)))
    g, o = _pair(mess, oracle_mod, he, "sto-3g")
    D = np.array([[1.7]])
    J, K, info = g.jk(D)
    ref = oracle_mod.eri(o, 0, 0, 0, 0) * 1.7
    assert J[0, 0] == pytest.approx(ref, rel=1e-13) and K[0, 0] == pytest.approx(ref, rel=1e-13)
    assert info["shell_quartets"] == 1
    with pytest.raises(mess.MessError):
        mess.Basis([11], [[0, 0, 0]], mi.basis_path("sto-3g"))
    with pytest.raises(mess.MessError):
        mess.Basis([1], [[0, 0, 0]], str(tmp_path / "missing.basis"))
    bad = tmp_path / "bad.basis"
    bad.write_text("element H\nS 2\n 1.0 1.0\n")
    with pytest.raises(mess.MessError):
        mess.Basis([1], [[0, 0, 0]], str(bad))
