"""Oracle of the Kohn-Sham energy functional (paper Sec. 5.1: Hamiltonian(basis, xc_method="lda" or
"pbe"), the exchange-correlation energy of the density on a quadrature grid).

TEST INFRASTRUCTURE ONLY (same rules as the rest of ``oracle/``): plain numpy in FP64, its own grid,
its own basis-function values and its own functional formulas.  Nothing on the library's product
path imports it.

Readings (the paper names the functionals, not their parametrisation or the grid):
  * LDA = Slater exchange + Perdew-Wang 1992 correlation (closed shell, zeta = 0).
    e_x = -(3/4)(3/pi)^(1/3) rho^(4/3);  eps_c(rs) = -2A(1 + a1 rs) ln(1 + 1/(2A(b1 rs^1/2 + b2 rs
    + b3 rs^3/2 + b4 rs^2))), rs = (3/(4 pi rho))^(1/3), A = 0.031091, a1 = 0.21370, b1 = 7.5957,
    b2 = 3.5876, b3 = 1.6382, b4 = 0.49294.
  * PBE (Perdew, Burke & Ernzerhof 1996), closed shell: exchange e_x^LDA F_x(s), F_x = 1 + kappa -
    kappa / (1 + mu s^2 / kappa), s = |grad rho| / (2 k_F rho), k_F = (3 pi^2 rho)^(1/3), kappa = 0.804,
    mu = beta pi^2 / 3; correlation rho (eps_c^PW92 + H), H = gamma ln(1 + (beta/gamma) t^2 (1 + A t^2)
    / (1 + A t^2 + A^2 t^4)), A = (beta/gamma) / (exp(-eps_c/gamma) - 1), t = |grad rho| / (2 k_s rho),
    k_s = sqrt(4 k_F / pi), beta = 0.06672455060314922, gamma = (1 - ln 2) / pi^2.
  * Grid: one atomic grid per atom, weighted by Becke's fuzzy-cell partition (Becke 1988: cell
    function s(mu) = (1 - f(f(f(mu)))) / 2, f(mu) = 3/2 mu - 1/2 mu^3, no size adjustment).
    Radial: Gauss-Chebyshev of the second kind, x_i = cos(i pi / (N + 1)), mapped by r = R (1 + x) /
    (1 - x) with R = the Bragg-Slater radius (H) or half of it (other elements): H 0.35, C 0.35,
    N 0.325, O 0.30 angstrom; N = 50 (H) or 75 points.  Angular: Gauss-Legendre in cos(theta)
    (16 points) times 32 equally spaced phi (exact for spherical harmonics up to degree 31).
  * The functional derivatives (v_rho = d e / d rho, v_sigma = d e / d sigma, sigma = |grad rho|^2)
    by complex-step differentiation of the energy density (exact to rounding, no derivation).
  * Kohn-Sham energy: E = tr(D H) + 1/2 tr(D J) + E_xc + E_nuc; Fock matrix F = H + J + V_xc with
    V_xc,mn = sum_g w_g [v_rho phi_m phi_n + 2 v_sigma grad rho . grad(phi_m phi_n)].

parity: pinned by tests/test_oracle_dft.py (the Slater exchange energy of the hydrogen-atom density
and of a Gaussian density against their closed forms; the grid integrating the electron count and
the overlap matrix; PBE reducing to LDA exchange at zero gradient; the complex-step derivatives
against central differences; the Kohn-Sham SCF energy equal to the minimum found by direct
minimisation of the same energy functional, which never uses V_xc).
"""
from __future__ import annotations

import math

import numpy as np

from . import jk, loewdin, nuclear_repulsion, one_e

ANGSTROM = 1.0 / 0.52917721092
BRAGG_HALF = {1: 0.35, 6: 0.35, 7: 0.325, 8: 0.30}       # angstrom: H full, others half
N_RADIAL = {1: 50}
N_RADIAL_DEFAULT = 75
N_THETA, N_PHI = 16, 32

PW_A, PW_A1, PW_B1, PW_B2, PW_B3, PW_B4 = 0.031091, 0.21370, 7.5957, 3.5876, 1.6382, 0.49294
PBE_KAPPA = 0.804
PBE_BETA = 0.06672455060314922
PBE_MU = PBE_BETA * math.pi ** 2 / 3.0
PBE_GAMMA = (1.0 - math.log(2.0)) / math.pi ** 2


# ----------------------------------------------------------------------------- grid
def atomic_grid(Z: int):
    """Points (relative to the atom) and weights of one atom's radial x angular grid."""
    nr = N_RADIAL.get(int(Z), N_RADIAL_DEFAULT)
    R = BRAGG_HALF[int(Z)] * ANGSTROM
    i = np.arange(1, nr + 1)
    x = np.cos(i * np.pi / (nr + 1))
    wx = np.pi / (nr + 1) * np.sin(i * np.pi / (nr + 1)) ** 2
    r = R * (1 + x) / (1 - x)
    wr = wx / np.sqrt(1 - x * x) * r * r * 2 * R / (1 - x) ** 2
    ct, wt = np.polynomial.legendre.leggauss(N_THETA)
    phi = 2 * np.pi * np.arange(N_PHI) / N_PHI
    st = np.sqrt(1 - ct * ct)
    dirs = np.array([[s * math.cos(p), s * math.sin(p), c] for c, s in zip(ct, st) for p in phi])
    wa = np.array([w * 2 * np.pi / N_PHI for w in wt for _ in phi])
    pts = (r[:, None, None] * dirs[None, :, :]).reshape(-1, 3)
    w = (wr[:, None] * wa[None, :]).reshape(-1)
    return pts, w


def becke_weights(pts, xyz, owner):
    """Fuzzy-cell weight of atom `owner` at each point."""
    xyz = np.asarray(xyz, dtype=np.float64).reshape(-1, 3)
    na = len(xyz)
    d = np.linalg.norm(pts[:, None, :] - xyz[None, :, :], axis=2)       # [npts, natom]
    P = np.ones((len(pts), na))
    for a in range(na):
        for b in range(na):
            if a == b:
                continue
            mu = (d[:, a] - d[:, b]) / np.linalg.norm(xyz[a] - xyz[b])
            f = mu
            for _ in range(3):
                f = 1.5 * f - 0.5 * f ** 3
            P[:, a] *= 0.5 * (1.0 - f)
    return P[:, owner] / P.sum(axis=1)


def molecular_grid(Z, xyz):
    xyz = np.asarray(xyz, dtype=np.float64).reshape(-1, 3)
    P, W = [], []
    for a, z in enumerate(Z):
        p, w = atomic_grid(int(z))
        p = p + xyz[a]
        P.append(p)
        W.append(w * (becke_weights(p, xyz, a) if len(Z) > 1 else 1.0))
    return np.concatenate(P), np.concatenate(W)


# ----------------------------------------------------------------------------- basis functions
def ao_values(b, pts):
    """phi_m(r) and grad phi_m(r) of every contracted Cartesian function at the points: [npts, n] and
    [npts, n, 3]."""
    n = b.nfn
    phi = np.zeros((len(pts), n))
    dphi = np.zeros((len(pts), n, 3))
    for m in range(n):
        d = pts - b.center[m]
        l = b.lmn[m]
        r2 = np.sum(d * d, axis=1)
        g = np.zeros(len(pts))
        gd = np.zeros(len(pts))             # sum_k c_k (-2 a_k) exp(-a_k r^2)
        for k in range(b.nprim[m]):
            a = b.exps[b.poff[m] + k]
            c = b.coefs[b.poff[m] + k]
            e = c * np.exp(-a * r2)
            g += e
            gd += -2.0 * a * e
        poly = d[:, 0] ** l[0] * d[:, 1] ** l[1] * d[:, 2] ** l[2]
        phi[:, m] = poly * g
        for x in range(3):
            dl = list(l)
            dpoly = np.zeros(len(pts))
            if l[x] > 0:
                dl[x] -= 1
                dpoly = l[x] * d[:, 0] ** dl[0] * d[:, 1] ** dl[1] * d[:, 2] ** dl[2]
            dphi[:, m, x] = dpoly * g + poly * gd * d[:, x]
    return phi, dphi


# ----------------------------------------------------------------------------- functionals
def _pw92(rs):
    den = 2.0 * PW_A * (PW_B1 * np.sqrt(rs) + PW_B2 * rs + PW_B3 * rs ** 1.5 + PW_B4 * rs * rs)
    return -2.0 * PW_A * (1.0 + PW_A1 * rs) * np.log(1.0 + 1.0 / den)


def slater_exchange(rho):
    """Local exchange energy per volume of the uniform gas, -(3/4)(3/pi)^(1/3) rho^(4/3)."""
    return -0.75 * (3.0 / np.pi) ** (1.0 / 3.0) * rho ** (4.0 / 3.0)


def pw92_correlation(rho):
    """Correlation energy per electron of the uniform gas (Perdew-Wang 1992, closed shell)."""
    return _pw92((3.0 / (4.0 * np.pi * rho)) ** (1.0 / 3.0))


def energy_density(kind, rho, sigma):
    """Exchange-correlation energy per volume, e(rho, sigma) (complex arguments allowed)."""
    ex = slater_exchange(rho)
    ec = pw92_correlation(rho)
    if kind == "lda":
        return ex + rho * ec
    kf = (3.0 * np.pi ** 2 * rho) ** (1.0 / 3.0)
    s2 = sigma / (2.0 * kf * rho) ** 2
    fx = 1.0 + PBE_KAPPA - PBE_KAPPA / (1.0 + PBE_MU * s2 / PBE_KAPPA)
    ks = np.sqrt(4.0 * kf / np.pi)
    t2 = sigma / (2.0 * ks * rho) ** 2
    A = (PBE_BETA / PBE_GAMMA) / (np.exp(-ec / PBE_GAMMA) - 1.0)
    at2 = A * t2
    H = PBE_GAMMA * np.log(1.0 + PBE_BETA / PBE_GAMMA * t2 * (1.0 + at2) / (1.0 + at2 + at2 * at2))
    return ex * fx + rho * (ec + H)


def derivatives(kind, rho, sigma, h=1e-30):
    """e, d e / d rho, d e / d sigma by complex steps (rho > 0)."""
    e = energy_density(kind, rho, sigma)
    er = np.imag(energy_density(kind, rho + 1j * h * rho, sigma)) / (h * rho)
    if kind == "lda":
        return e, er, np.zeros_like(rho)
    es = np.imag(energy_density(kind, rho, sigma + 1j * h * np.maximum(sigma, 1e-300))) / (h * np.maximum(sigma, 1e-300))
    return e, er, es


RHO_MIN = 1e-14      # points with less density carry no exchange-correlation energy


def xc(b, D, pts, w, kind, ao=None):
    """E_xc and V_xc of the density D on the grid."""
    phi, dphi = ao if ao is not None else ao_values(b, pts)
    T = phi @ D
    rho = np.sum(T * phi, axis=1)
    grad = 2.0 * np.einsum("pm,pmx->px", T, dphi)
    sigma = np.sum(grad * grad, axis=1)
    ok = rho > RHO_MIN
    e = np.zeros_like(rho)
    vr = np.zeros_like(rho)
    vs = np.zeros_like(rho)
    e[ok], vr[ok], vs[ok] = derivatives(kind, rho[ok], sigma[ok])
    E = float(np.sum(w * e))
    a = w[:, None] * (0.5 * vr[:, None] * phi + 2.0 * vs[:, None] * np.einsum("px,pmx->pm", grad, dphi))
    V = phi.T @ a
    return E, V + V.T


# ----------------------------------------------------------------------------- Kohn-Sham SCF
def ks_scf(b, kind, max_iter=100, conv_E=1e-10, conv_comm=1e-8, diis_n=8):
    """Closed-shell Kohn-Sham SCF on the oracle's grid; returns (E_total, D, iterations)."""
    nel = int(np.sum(b.Z))
    nocc = nel // 2
    S, T, V = one_e(b)
    H = T + V
    X = loewdin(S)
    Enuc = nuclear_repulsion(b.Z, b.xyz)
    pts, w = molecular_grid(b.Z, b.xyz)
    ao = ao_values(b, pts)

    def dens(F):
        _, C = np.linalg.eigh(X.T @ F @ X)
        C = X @ C
        return 2.0 * C[:, :nocc] @ C[:, :nocc].T

    D = dens(H)
    Fs, es = [], []
    E_old = None
    for it in range(1, max_iter + 1):
        J, _ = jk(b, D)
        Exc, Vxc = xc(b, D, pts, w, kind, ao)
        F = H + J + Vxc
        E = float(np.sum(D * H)) + 0.5 * float(np.sum(D * J)) + Exc
        err = F @ D @ S - S @ D @ F
        if E_old is not None and abs(E - E_old) < conv_E and np.abs(err).max() < conv_comm:
            return E + Enuc, D, it
        E_old = E
        Fs = (Fs + [F])[-diis_n:]
        es = (es + [err])[-diis_n:]
        if len(Fs) >= 2:
            k = len(Fs)
            B = -np.ones((k + 1, k + 1))
            B[-1, -1] = 0.0
            for i in range(k):
                for j in range(k):
                    B[i, j] = float(np.sum(es[i] * es[j]))
            c = np.linalg.solve(B, np.r_[np.zeros(k), -1.0])[:k]
            F = sum(ci * Fi for ci, Fi in zip(c, Fs))
        D = dens(F)
    raise RuntimeError("Kohn-Sham SCF did not converge")


def ks_energy(b, kind, D, grid=None, ao=None):
    """E_total of a density D (no Fock matrix involved)."""
    S, T, V = one_e(b)
    H = T + V
    pts, w = grid if grid is not None else molecular_grid(b.Z, b.xyz)
    J, _ = jk(b, D)
    Exc, _ = xc(b, D, pts, w, kind, ao)
    return float(np.sum(D * H)) + 0.5 * float(np.sum(D * J)) + Exc + nuclear_repulsion(b.Z, b.xyz)
