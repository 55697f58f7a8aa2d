"""Pins for the Kohn-Sham oracle (CPU only): the grid, the functionals and the Kohn-Sham energy,
each against something other than the oracle itself."""
import math

import numpy as np
import pytest
from scipy.optimize import minimize

import mess_inputs as mi
import oracle
from oracle import dft


def test_slater_exchange_of_the_hydrogen_atom():
    """rho = exp(-2r)/pi: int rho^(4/3) = (27/64) pi^(-1/3), so E_x = -(81/256) 3^(1/3) pi^(-2/3)."""
    pts, w = dft.atomic_grid(1)
    r = np.linalg.norm(pts, axis=1)
    rho = np.exp(-2.0 * r) / np.pi
    assert np.sum(w * rho) == pytest.approx(1.0, abs=1e-8)
    Ex = float(np.sum(w * dft.slater_exchange(rho)))
    assert Ex == pytest.approx(-(81.0 / 256.0) * 3 ** (1 / 3) * math.pi ** (-2 / 3), abs=1e-7)


def _single_gaussian(alpha):
    """One normalised s Gaussian on an atom at the origin (unit contraction of a single primitive)."""
    n = 1
    N = (2 * alpha / math.pi) ** 0.75
    return oracle.Basis(n, np.zeros((1, 3)), np.zeros((1, 3), dtype=np.int32), np.ones(1, dtype=np.int32),
                        np.zeros(1, dtype=np.int32), np.array([alpha]), np.array([N]), np.zeros(1, dtype=np.int32),
                        1, np.zeros(1, dtype=np.int32), np.array([2], dtype=np.int32), np.zeros((1, 3)))


def test_slater_exchange_of_a_gaussian_pair_density():
    """Two electrons in phi = (2a/pi)^(3/4) exp(-a r^2): rho = 2 phi^2, and
    int rho^(4/3) = 2^(4/3) (2a/pi)^2 (3 pi / (8 a))^(3/2)."""
    a = 0.8
    b = _single_gaussian(a)
    pts, w = dft.atomic_grid(8)
    phi, _ = dft.ao_values(b, pts)
    rho = 2.0 * phi[:, 0] ** 2
    assert np.sum(w * rho) == pytest.approx(2.0, abs=1e-8)
    closed = 2 ** (4 / 3) * (2 * a / math.pi) ** 2 * (3 * math.pi / (8 * a)) ** 1.5
    Ex = float(np.sum(w * dft.slater_exchange(rho)))
    assert Ex == pytest.approx(-0.75 * (3 / math.pi) ** (1 / 3) * closed, rel=1e-8)


def test_molecular_grid_integrates_the_overlap(oracle_mod):
    """The Becke-partitioned grid reproduces the analytic overlap matrix (AO values and cell weights)."""
    o = oracle_mod.basis_for(mi.h2o(), mi.basis_path("6-31gs"))
    pts, w = dft.molecular_grid(o.Z, o.xyz)
    phi, dphi = dft.ao_values(o, pts)
    S = oracle_mod.overlap(o)
    assert np.abs(phi.T @ (w[:, None] * phi) - S).max() < 1e-6
    # kinetic energy from the gradients: T_mn = 1/2 int grad phi_m . grad phi_n
    T = 0.5 * np.einsum("p,pmx,pnx->mn", w, dphi, dphi)
    Tref = oracle_mod.one_e(o)[1]
    assert np.abs(T - Tref).max() < 1e-6 * np.abs(Tref).max()


def test_pw92_high_density_coefficient():
    """The uniform-gas correlation energy grows like A ln rs at high density, A = (1 - ln 2) / pi^2
    (Gell-Mann and Brueckner); PW92's parameter A = 0.031091 carries it."""
    rs = np.array([1e-7, 1e-6])
    rho = 3.0 / (4.0 * math.pi * rs ** 3)
    ec = dft.pw92_correlation(rho)
    slope = (ec[1] - ec[0]) / math.log(rs[1] / rs[0])
    assert slope == pytest.approx((1 - math.log(2)) / math.pi ** 2, rel=2e-3)


def test_pbe_limits():
    rho = np.array([1e-3, 0.1, 2.0])
    # zero gradient: PBE is LDA
    np.testing.assert_allclose(dft.energy_density("pbe", rho, np.zeros(3)), dft.energy_density("lda", rho, np.zeros(3)),
                               rtol=1e-14)
    # very large reduced gradient: the exchange enhancement saturates at 1 + kappa
    kf = (3 * math.pi ** 2 * rho) ** (1 / 3)
    sigma = (2 * kf * rho * 1e4) ** 2
    ex_lda = dft.slater_exchange(rho)
    e = dft.energy_density("pbe", rho, sigma)
    ec_pbe = e - ex_lda * (1 + dft.PBE_KAPPA)
    assert np.all(np.abs(ec_pbe) < np.abs(ex_lda) * 1e-2 + 1.0 * rho)


@pytest.mark.parametrize("kind", ["lda", "pbe"])
def test_complex_step_derivatives(kind):
    rho = np.array([1e-4, 0.03, 0.5, 3.0])
    sigma = np.array([1e-8, 1e-3, 0.2, 4.0])
    _, er, es = dft.derivatives(kind, rho, sigma)
    for i in range(4):
        h = 1e-6 * rho[i]
        fd = (dft.energy_density(kind, rho[i] + h, sigma[i]) - dft.energy_density(kind, rho[i] - h, sigma[i])) / (2 * h)
        assert er[i] == pytest.approx(fd, rel=1e-6)
        if kind == "pbe":
            h = 1e-6 * sigma[i]
            fd = (dft.energy_density(kind, rho[i], sigma[i] + h) - dft.energy_density(kind, rho[i], sigma[i] - h)) / (2 * h)
            assert es[i] == pytest.approx(fd, rel=1e-5)


@pytest.mark.parametrize("kind,mol", [("lda", "h2"), ("pbe", "h2o")])
def test_kohn_sham_scf_is_the_energy_minimum(oracle_mod, kind, mol):
    """The Kohn-Sham SCF (which uses V_xc) converges to the minimum of the energy functional found by
    a quasi-Newton search over orthonormal orbitals that evaluates energies only (finite-difference
    gradients, no V_xc): a wrong potential would stop the SCF elsewhere."""
    m = mi.h2(1.4) if mol == "h2" else mi.h2o()
    b = oracle_mod.basis_for(m, mi.basis_path("sto-3g"))
    E_scf, D_scf, _ = dft.ks_scf(b, kind)
    S = oracle_mod.overlap(b)
    X = oracle_mod.loewdin(S)
    nocc = int(np.sum(b.Z)) // 2
    n = b.nfn
    grid = dft.molecular_grid(b.Z, b.xyz)
    ao = dft.ao_values(b, grid[0])
    # occupied orbitals = core-Hamiltonian occupied + virtual x K, orthonormalised by QR (in the
    # orthonormal basis X); the (n - nocc) x nocc entries of K are the parameters
    S_, T_, V_ = oracle_mod.one_e(b)
    _, Cp = np.linalg.eigh(X.T @ (T_ + V_) @ X)
    occ, vir = Cp[:, :nocc], Cp[:, nocc:]
    z0 = np.zeros((n - nocc) * nocc)

    def energy(z):
        Q, _ = np.linalg.qr(occ + vir @ z.reshape(n - nocc, nocc))
        C = X @ Q
        return dft.ks_energy(b, kind, 2.0 * C @ C.T, grid=grid, ao=ao)

    r = minimize(energy, z0, method="BFGS", options={"gtol": 1e-7, "eps": 1e-7})
    assert r.fun == pytest.approx(E_scf, abs=2e-7)
    assert E_scf <= r.fun + 1e-9
