"""Seeded molecular geometries (bohr) and seeded random matrices.  No integral arithmetic here."""
from __future__ import annotations

import math
import os
from dataclasses import dataclass

import numpy as np

ATOMIC_NUMBER = {"H": 1, "He": 2, "C": 6, "N": 7, "O": 8}
SYMBOL = {v: k for k, v in ATOMIC_NUMBER.items()}

_BASIS_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "basis")

# Water internal geometry: O-H 1.809 bohr, H-O-H 104.52 degrees.
R_OH = 1.809
HOH_DEG = 104.52
# Alkane internal geometry: C-C 1.54 A, C-H 1.09 A (in bohr), tetrahedral angles.
R_CC = 2.910
R_CH = 2.060
TETRA_DEG = 109.4712206  # arccos(-1/3)


def basis_path(name: str) -> str:
    """Path of a basis data file: ``sto-3g``, ``6-31g`` or ``6-31gs`` (6-31G*)."""
    key = name.lower().replace("*", "s")
    path = os.path.join(_BASIS_DIR, key + ".basis")
    if not os.path.exists(path):
        raise FileNotFoundError(f"no basis data file for {name!r} ({path})")
    return path


@dataclass
class Molecule:
    name: str
    Z: np.ndarray    # int32 [natom]
    xyz: np.ndarray  # float64 [natom, 3], bohr

    @property
    def natom(self) -> int:
        return int(self.Z.shape[0])

    @property
    def nelectron(self) -> int:
        return int(self.Z.sum())


def _mol(name, symbols, xyz) -> Molecule:
    Z = np.array([ATOMIC_NUMBER[s] for s in symbols], dtype=np.int32)
    return Molecule(name, Z, np.ascontiguousarray(np.asarray(xyz, dtype=np.float64).reshape(-1, 3)))


def _water_frame():
    half = math.radians(HOH_DEG / 2.0)
    return np.array([[0.0, 0.0, 0.0],
                     [R_OH * math.sin(half), 0.0, R_OH * math.cos(half)],
                     [-R_OH * math.sin(half), 0.0, R_OH * math.cos(half)]])


def h2o() -> Molecule:
    """One water: O at the origin, both H in the xz plane."""
    return _mol("h2o", ["O", "H", "H"], _water_frame())


def h2(r: float) -> Molecule:
    """H2 with bond length r (bohr) along x."""
    return _mol(f"h2_{r:.4f}", ["H", "H"], [[0.0, 0.0, 0.0], [r, 0.0, 0.0]])


def _random_rotation(rng: np.random.Generator) -> np.ndarray:
    """Rotation matrix uniform on SO(3): unit quaternion from four standard normals."""
    q = rng.standard_normal(4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
        [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
        [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)],
    ])


def water_cluster(n: int, box: float, seed: int, min_oo: float = 5.0,
                  max_tries: int = 20000) -> Molecule:
    """n rigid waters; orientations uniform on SO(3); O uniform in [0, box]^3.

    Waters are placed one after another; a candidate O position is redrawn until it lies at
    least ``min_oo`` bohr from every O already placed (the whole cluster restarts if a water
    cannot be placed within ``max_tries`` draws).
    """
    rng = np.random.default_rng(seed)
    frame = _water_frame()
    for _restart in range(100):
        oxygens = []
        atoms = []
        ok = True
        for _ in range(n):
            R = _random_rotation(rng)
            for _t in range(max_tries):
                o = rng.random(3) * box
                if all(np.linalg.norm(o - p) >= min_oo for p in oxygens):
                    break
            else:
                ok = False
                break
            oxygens.append(o)
            atoms.append(frame @ R.T + o)
        if ok:
            xyz = np.concatenate(atoms, axis=0)
            return _mol(f"water{n}_seed{seed}", ["O", "H", "H"] * n, xyz)
    raise RuntimeError("could not place the water cluster")


def _unit(v):
    return v / np.linalg.norm(v)


def _place(a, b, c, r, theta, phi):
    """Atom d bonded to c with |cd| = r, angle b-c-d = theta, torsion a-b-c-d = phi."""
    bc = _unit(c - b)
    nrm = _unit(np.cross(b - a, bc))
    m = np.cross(nrm, bc)
    d2 = np.array([-r * math.cos(theta), r * math.sin(theta) * math.cos(phi),
                   r * math.sin(theta) * math.sin(phi)])
    return c + d2[0] * bc + d2[1] * m + d2[2] * nrm


def _perp_basis(u):
    t = np.array([1.0, 0.0, 0.0]) if abs(u[0]) < 0.9 else np.array([0.0, 1.0, 0.0])
    e1 = _unit(np.cross(u, t))
    e2 = np.cross(u, e1)
    return e1, e2


def _alkane_once(n: int, rng: np.random.Generator):
    th = math.radians(TETRA_DEG)
    carbons = []
    if n == 1:
        carbons.append(np.zeros(3))
    else:
        carbons.append(np.zeros(3))
        carbons.append(np.array([R_CC, 0.0, 0.0]))
        if n >= 3:
            c2 = carbons[1]
            carbons.append(c2 + R_CC * np.array([-math.cos(th), math.sin(th), 0.0]))
        for k in range(3, n):
            phi = rng.random() * 2.0 * math.pi
            carbons.append(_place(carbons[k - 3], carbons[k - 2], carbons[k - 1], R_CC, th, phi))
    hydrogens = []
    bonds = [(i, i + 1) for i in range(n - 1)]
    for i, c in enumerate(carbons):
        nbr = [carbons[j] for j in (i - 1, i + 1) if 0 <= j < n]
        dirs = []
        if len(nbr) == 0:
            t = np.array([[1, 1, 1], [1, -1, -1], [-1, 1, -1], [-1, -1, 1]], dtype=float) / math.sqrt(3)
            dirs = list(t)
        elif len(nbr) == 1:
            u1 = _unit(nbr[0] - c)
            e1, e2 = _perp_basis(u1)
            phi0 = rng.random() * 2.0 * math.pi
            for k in range(3):
                ph = phi0 + 2.0 * math.pi * k / 3.0
                dirs.append(math.cos(th) * u1 + math.sin(th) * (math.cos(ph) * e1 + math.sin(ph) * e2))
        else:
            u1, u2 = _unit(nbr[0] - c), _unit(nbr[1] - c)
            bis = -_unit(u1 + u2)
            nrm = _unit(np.cross(u1, u2))
            half = th / 2.0
            dirs = [math.cos(half) * bis + math.sin(half) * nrm,
                    math.cos(half) * bis - math.sin(half) * nrm]
        for d in dirs:
            bonds.append((i, n + len(hydrogens)))
            hydrogens.append(c + R_CH * d)
    xyz = np.array(carbons + hydrogens)
    return xyz, bonds


def alkane(n: int, rng: np.random.Generator, min_nonbonded: float = 2.0) -> Molecule:
    """Linear alkane C_nH_(2n+2); all torsions are redrawn while any non-bonded pair < 2.0 bohr."""
    for _ in range(1000):
        xyz, bonds = _alkane_once(n, rng)
        bonded = set(bonds) | {(j, i) for i, j in bonds}
        d = np.linalg.norm(xyz[:, None, :] - xyz[None, :, :], axis=-1)
        clash = False
        na = xyz.shape[0]
        for i in range(na):
            for j in range(i + 1, na):
                if (i, j) not in bonded and d[i, j] < min_nonbonded:
                    clash = True
                    break
            if clash:
                break
        if not clash:
            R = _random_rotation(rng)
            return _mol(f"C{n}H{2 * n + 2}", ["C"] * n + ["H"] * (2 * n + 2), xyz @ R.T)
    raise RuntimeError("could not build a clash-free alkane")


def alkane_batch(count: int, nmin: int, nmax: int, seed: int) -> list:
    """``count`` alkanes, chain length n uniform on {nmin..nmax}, one seeded stream."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        n = int(rng.integers(nmin, nmax + 1))
        out.append(alkane(n, rng))
    return out


def random_symmetric_density(n: int, seed: int, nocc: int | None = None) -> np.ndarray:
    """Seeded symmetric positive semidefinite n x n matrix 2 X X^T, X ~ N(0, 1/n) of shape n x nocc."""
    rng = np.random.default_rng(seed)
    nocc = max(1, n // 4) if nocc is None else nocc
    X = rng.standard_normal((n, nocc)) / math.sqrt(n)
    D = 2.0 * X @ X.T
    return np.ascontiguousarray(0.5 * (D + D.T))
