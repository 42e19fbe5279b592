"""Seeded synthetic inputs for the DF-J/K build: molecules, basis sets, C_occ.

This module holds no integral or J/K arithmetic; the CUDA library and the
oracle both consume what it produces.  The paper benchmarks 13 molecules of
20-168 atoms with def2-TZVPP / def2-universal-JKFIT (Sec. "Dataset and
Performance" and the dataset appendix); neither the molecules nor those basis
files are available here, so synthetic molecules of the same size range with
even-tempered Cartesian bases stand in for them.

Recipe (every draw from ``numpy.random.default_rng``):
  * water (3 atoms): O at the origin, H at (+-1.43, 1.11, 0) bohr, each
    coordinate jittered by U(-0.05, 0.05), seed 1001.  Orbital basis per atom:
    s shells 0.15*3^k (k=0..2) and one p shell 0.8, each a 2-primitive
    contraction whose second exponent is 2.5x the first; aux per atom:
    s 0.2*2.5^k (k=0..3) and p 0.5, 1.5, uncontracted.  nao=18, naux=30.
  * N-atom molecules: N atoms uniform in a cube of side (N/0.01)^(1/3) bohr by
    rejection sampling to a minimum separation of 1.8 bohr.  Orbital basis per
    atom: s 0.15*3^k (k=0..2), p 0.8*3^k (k=0,1), d 1.0, each 2-primitive
    (x2.5); aux per atom: s 0.2*2.5^k (k=0..5), p 0.5*2.5^k (k=0..3),
    d 0.6*2.5^k (k=0..2), uncontracted.  nao=15N, naux=36N.
  * contraction coefficients: U(0.2, 1.0), seed 2000, one draw per shell
    template (every atom carries the same basis, like one element).
  * C_occ: N(0,1) entries, seed 3000+mol_id, made orthonormal in the overlap
    metric by ``orthonormalize``; nocc = round(0.2 nao) unless given.
"""

from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class Shell:
    atom: int
    l: int
    exps: np.ndarray
    coefs: np.ndarray  # coefficients of unnormalised primitives


@dataclass
class Basis:
    shells: list = field(default_factory=list)

    @property
    def nfunc(self) -> int:
        return sum((s.l + 1) * (s.l + 2) // 2 for s in self.shells)


@dataclass
class Molecule:
    coords: np.ndarray  # natom x 3, bohr
    orb: Basis
    aux: Basis
    name: str = ""

    @property
    def natom(self) -> int:
        return int(self.coords.shape[0])

    @property
    def nao(self) -> int:
        return self.orb.nfunc

    @property
    def naux(self) -> int:
        return self.aux.nfunc


# (l, first exponent) templates; orbital shells are 2-primitive (x2.5).
ORB_WATER = [(0, 0.15), (0, 0.45), (0, 1.35), (1, 0.8)]
AUX_WATER = [(0, 0.2 * 2.5**k) for k in range(4)] + [(1, 0.5), (1, 1.5)]
ORB_STD = [(0, 0.15 * 3**k) for k in range(3)] + [(1, 0.8 * 3**k) for k in range(2)] + [(2, 1.0)]
AUX_STD = (
    [(0, 0.2 * 2.5**k) for k in range(6)]
    + [(1, 0.5 * 2.5**k) for k in range(4)]
    + [(2, 0.6 * 2.5**k) for k in range(3)]
)
COEF_SEED = 2000


def _orb_coefs(template, seed=COEF_SEED):
    rng = np.random.default_rng(seed)
    return [rng.uniform(0.2, 1.0, size=2) for _ in template]


def make_basis(natom: int, template, contracted: bool, seed=COEF_SEED) -> Basis:
    coefs = _orb_coefs(template, seed) if contracted else None
    shells = []
    for a in range(natom):
        for t, (l, e) in enumerate(template):
            if contracted:
                shells.append(Shell(a, l, np.array([e, 2.5 * e]), coefs[t].copy()))
            else:
                shells.append(Shell(a, l, np.array([e]), np.array([1.0])))
    return Basis(shells)


def water(seed: int = 1001) -> Molecule:
    rng = np.random.default_rng(seed)
    xyz = np.array([[0.0, 0.0, 0.0], [1.43, 1.11, 0.0], [-1.43, 1.11, 0.0]])
    xyz = xyz + rng.uniform(-0.05, 0.05, size=xyz.shape)
    return Molecule(xyz, make_basis(3, ORB_WATER, True), make_basis(3, AUX_WATER, False), "water")


def random_geometry(natom: int, seed: int, density: float = 0.01, min_sep: float = 1.8):
    rng = np.random.default_rng(seed)
    side = (natom / density) ** (1.0 / 3.0)
    pts = []
    tries = 0
    while len(pts) < natom:
        tries += 1
        if tries > 1000000:
            raise RuntimeError("rejection sampling did not converge")
        x = rng.uniform(0.0, side, size=3)
        if all(np.sum((x - q) ** 2) >= min_sep * min_sep for q in pts):
            pts.append(x)
    return np.array(pts)


def molecule(natom: int, seed: int) -> Molecule:
    """N-atom molecule with the standard per-atom bases (nao=15N, naux=36N)."""
    xyz = random_geometry(natom, seed)
    return Molecule(
        xyz, make_basis(natom, ORB_STD, True), make_basis(natom, AUX_STD, False), f"mol{natom}"
    )


def c_occ_raw(nao: int, nocc: int, seed: int) -> np.ndarray:
    return np.random.default_rng(seed).standard_normal((nao, nocc))


def default_nocc(nao: int) -> int:
    return int(round(0.2 * nao))


def orthonormalize(C0: np.ndarray, S: np.ndarray) -> np.ndarray:
    """Loewdin: C = C0 (C0^T S C0)^(-1/2), so that C^T S C = 1."""
    M = C0.T @ S @ C0
    w, U = np.linalg.eigh(M)
    return C0 @ ((U / np.sqrt(w)) @ U.T)


def batch_atom_counts(n: int = 256, lo: int = 5, hi: int = 80, seed: int = 4000) -> np.ndarray:
    """Atom counts for a batch of molecules, uniform integers in [lo, hi]."""
    return np.random.default_rng(seed).integers(lo, hi + 1, size=n)


def poisson_arrivals(rate: float, n: int, seed: int) -> np.ndarray:
    """Arrival times (s) of a Poisson stream."""
    return np.cumsum(np.random.default_rng(seed).exponential(1.0 / rate, size=n))


def serve_atom_counts(n: int, lo: int = 5, hi: int = 150, seed: int = 6000) -> np.ndarray:
    """Log-uniform atom counts in [lo, hi]."""
    rng = np.random.default_rng(seed)
    return np.round(np.exp(rng.uniform(np.log(lo), np.log(hi), size=n))).astype(int)
