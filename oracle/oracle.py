"""Plain FP64 CPU oracle for the density-fitted Coulomb/exchange (DF-J/K) build.

TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the benchmark's
CPU-baseline leg may import this module.  It shares no code with the CUDA
library: the integrals come from ``dfjk_oracle.c`` (Obara-Saika recursion), the
dense steps from NumPy/SciPy FP64 LAPACK/BLAS, in the order of the method:

  O3  V = (P|Q)                                   2-centre metric
  O4  T = (P|mu nu), every ordered pair, unscreened
  O5  L = chol(V), lower, positive diagonal
  O6  B = L^-1 T                                  whitened 3-centre tensor
  O7  D = C C^T
  O8  rho = B vec(D);  J = B^T rho
  O9  X_P = B_P C;     K = sum_P X_P X_P^T
  O10 E_J = Tr(D J)/2, E_K = Tr(D K)/2
  O11 dE_J/dR, dE_K/dR at fixed D: central differences of O3-O10 with the
      shells moved with their atoms (the definition of the derivative)

The paper (Introduction, contribution 1) says only that density fitting first
evaluates 3-centre integrals and then reduces to tensor contractions; it prints
no formula, so these steps are the textbook definition of density-fitted J and
K with a Coulomb metric, written out directly.  The accuracy passage of the
section on PySCF compatibility attributes the larger deviations to an
ill-conditioned fitting system and is the paper's only remark on the linear
solve; this oracle uses a Cholesky factor with no pivoting and no eigenvalue
cut-off.
"""

from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np
import scipy.linalg

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle_dfjk.so")
_SRC = os.path.join(_HERE, "dfjk_oracle.c")
_lib_handle = None


def build(force: bool = False) -> str:
    """Compile the C part of the oracle with the host gcc (OpenMP)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        subprocess.check_call(
            ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", _SO, _SRC, "-lm"]
        )
    return _SO


def _lib():
    global _lib_handle
    if _lib_handle is None:
        build()
        lib = ctypes.CDLL(_SO)
        i32p = ctypes.POINTER(ctypes.c_int)
        f64p = ctypes.POINTER(ctypes.c_double)
        shell_args = [ctypes.c_int, i32p, i32p, i32p, i32p, f64p, f64p]
        lib.oracle_boys.argtypes = [ctypes.c_int, ctypes.c_double, f64p]
        lib.oracle_boys.restype = None
        lib.oracle_overlap.argtypes = shell_args + [f64p, f64p]
        lib.oracle_metric.argtypes = shell_args + [f64p, f64p]
        lib.oracle_three_center.argtypes = (
            shell_args + shell_args + [f64p, ctypes.c_int, ctypes.c_int, ctypes.c_int, f64p]
        )
        lib.oracle_three_center_triples.argtypes = (
            shell_args
            + shell_args
            + [f64p, ctypes.c_int, i32p, ctypes.POINTER(ctypes.c_longlong), f64p]
        )
        lib.oracle_num_threads.argtypes = []
        _lib_handle = lib
    return _lib_handle


def num_threads() -> int:
    """OpenMP threads the C part uses."""
    return int(_lib().oracle_num_threads())


def _ptr(a, t):
    return a.ctypes.data_as(ctypes.POINTER(t))


def ncart(l: int) -> int:
    return (l + 1) * (l + 2) // 2


def cart_powers(l: int):
    """Cartesian components of angular momentum l: x,y,z / xx,xy,xz,yy,yz,zz."""
    out = []
    for i in range(l, -1, -1):
        for j in range(l - i, -1, -1):
            out.append((i, j, l - i - j))
    return out


class _Flat:
    """Flat C arrays for a basis given as an object with ``.shells`` (each with
    ``atom``, ``l``, ``exps``, ``coefs``)."""

    def __init__(self, basis):
        shells = list(basis.shells)
        self.n = len(shells)
        self.atom = np.array([s.atom for s in shells], dtype=np.int32)
        self.l = np.array([s.l for s in shells], dtype=np.int32)
        self.nprim = np.array([len(s.exps) for s in shells], dtype=np.int32)
        self.off = np.zeros(self.n, dtype=np.int32)
        if self.n:
            self.off[1:] = np.cumsum(self.nprim)[:-1]
        self.exps = np.ascontiguousarray(np.concatenate([np.asarray(s.exps, float) for s in shells]))
        self.coefs = np.ascontiguousarray(
            np.concatenate([np.asarray(s.coefs, float) for s in shells])
        )
        self.nfunc = int(sum(ncart(int(l)) for l in self.l))
        self.func_off = np.zeros(self.n + 1, dtype=np.int64)
        self.func_off[1:] = np.cumsum([ncart(int(l)) for l in self.l])

    def args(self):
        i32 = ctypes.c_int
        return [
            self.n,
            _ptr(self.atom, i32),
            _ptr(self.l, i32),
            _ptr(self.nprim, i32),
            _ptr(self.off, i32),
            _ptr(self.exps, ctypes.c_double),
            _ptr(self.coefs, ctypes.c_double),
        ]


def boys(mmax: int, T: float) -> np.ndarray:
    """F_0..F_mmax at T (series for T <= 30, erf + upward recursion above)."""
    F = np.zeros(mmax + 1)
    _lib().oracle_boys(int(mmax), float(T), _ptr(F, ctypes.c_double))
    return F


def overlap(basis, coords) -> np.ndarray:
    """S[mu][nu], normalised Cartesian contracted Gaussians."""
    f = _Flat(basis)
    xyz = np.ascontiguousarray(coords, dtype=float)
    S = np.zeros((f.nfunc, f.nfunc))
    rc = _lib().oracle_overlap(*f.args(), _ptr(xyz, ctypes.c_double), _ptr(S, ctypes.c_double))
    if rc:
        raise ValueError(f"oracle_overlap failed ({rc})")
    return S


def metric(aux, coords) -> np.ndarray:
    """V[P][Q] = (P|Q) (step O3)."""
    f = _Flat(aux)
    xyz = np.ascontiguousarray(coords, dtype=float)
    V = np.zeros((f.nfunc, f.nfunc))
    rc = _lib().oracle_metric(*f.args(), _ptr(xyz, ctypes.c_double), _ptr(V, ctypes.c_double))
    if rc:
        raise ValueError(f"oracle_metric failed ({rc})")
    return V


def three_center(basis, aux, coords, sym: bool = False, aux_shells=None) -> np.ndarray:
    """T[P][mu][nu] = (P|mu nu) (step O4), optionally for a range of aux shells."""
    fo, fa = _Flat(basis), _Flat(aux)
    s0, s1 = (0, fa.n) if aux_shells is None else aux_shells
    p0, p1 = int(fa.func_off[s0]), int(fa.func_off[s1])
    xyz = np.ascontiguousarray(coords, dtype=float)
    T = np.zeros((p1 - p0, fo.nfunc, fo.nfunc))
    rc = _lib().oracle_three_center(
        *fo.args(), *fa.args(), _ptr(xyz, ctypes.c_double), int(s0), int(s1), int(bool(sym)),
        _ptr(T, ctypes.c_double)
    )
    if rc:
        raise ValueError(f"oracle_three_center failed ({rc})")
    return T


def three_center_triples(basis, aux, coords, triples) -> list:
    """Blocks (P|a b)[ca][cb][cc] for explicit shell triples (a, b, P-shell)."""
    fo, fa = _Flat(basis), _Flat(aux)
    trip = np.ascontiguousarray(np.asarray(triples, dtype=np.int32).reshape(-1, 3))
    sizes = [
        ncart(int(fo.l[a])) * ncart(int(fo.l[b])) * ncart(int(fa.l[c])) for a, b, c in trip
    ]
    offs = np.zeros(len(sizes), dtype=np.int64)
    if sizes:
        offs[1:] = np.cumsum(sizes)[:-1]
    out = np.zeros(int(sum(sizes)))
    xyz = np.ascontiguousarray(coords, dtype=float)
    rc = _lib().oracle_three_center_triples(
        *fo.args(), *fa.args(), _ptr(xyz, ctypes.c_double), len(trip),
        _ptr(trip, ctypes.c_int), _ptr(offs, ctypes.c_longlong), _ptr(out, ctypes.c_double)
    )
    if rc:
        raise ValueError(f"oracle_three_center_triples failed ({rc})")
    blocks = []
    for (a, b, c), o, n in zip(trip, offs, sizes):
        shape = (ncart(int(fo.l[a])), ncart(int(fo.l[b])), ncart(int(fa.l[c])))
        blocks.append(out[o : o + n].reshape(shape))
    return blocks


def whiten(V: np.ndarray, T: np.ndarray, how: str = "cholesky"):
    """Steps O5-O6: B = L^-1 T with V = L L^T (or B = V^-1/2 T for the check
    that J and K do not depend on the choice of whitening)."""
    naux = V.shape[0]
    T2 = T.reshape(naux, -1)
    if how == "cholesky":
        L = scipy.linalg.cholesky(V, lower=True)
        return L, scipy.linalg.solve_triangular(L, T2, lower=True).reshape(T.shape)
    if how == "eigh":
        w, U = np.linalg.eigh(V)
        W = (U / np.sqrt(w)) @ U.T
        return W, (W @ T2).reshape(T.shape)
    raise ValueError(how)


def jk_from_B(B: np.ndarray, C: np.ndarray):
    """Steps O7-O10 from the whitened tensor B[P][mu][nu] and C[mu][i]."""
    naux, nao, _ = B.shape
    D = C @ C.T
    B2 = B.reshape(naux, nao * nao)
    rho = B2 @ D.ravel()
    J = (rho @ B2).reshape(nao, nao)
    X = np.matmul(B, C)  # X[P][mu][i] = (B_P C)[mu][i]
    Xr = X.transpose(1, 0, 2).reshape(nao, -1)
    K = Xr @ Xr.T
    return dict(D=D, rho=rho, J=J, K=K, X=X, E_J=0.5 * np.sum(D * J), E_K=0.5 * np.sum(D * K))


def dfjk(basis, aux, coords, C, how: str = "cholesky", T=None, V=None):
    """The whole oracle, O3-O10.  Returns a dict with V, T, L, B, rho, J, K, E_J, E_K."""
    V = metric(aux, coords) if V is None else V
    T = three_center(basis, aux, coords) if T is None else T
    L, B = whiten(V, T, how)
    out = jk_from_B(B, np.asarray(C, float))
    out.update(V=V, T=T, L=L, B=B)
    return out


def energies_second_way(T, V, B, C):
    """Step O11.  E_J' = u^T d / 2 with u_P = sum T[P,mu,nu] D[mu,nu] and the
    fitted coefficients d = V^-1 u (LU solve, no Cholesky);
    E_K' = sum_P ||C^T B_P C||_F^2 / 2."""
    naux = V.shape[0]
    D = C @ C.T
    u = T.reshape(naux, -1) @ D.ravel()
    d = np.linalg.solve(V, u)
    M = np.einsum("mi,Pmn,nj->Pij", C, B, C, optimize=True)
    return 0.5 * float(u @ d), 0.5 * float(np.sum(M * M))



def dfjk_uks(B: np.ndarray, C_a: np.ndarray, C_b: np.ndarray):
    """Spin-unrestricted J/K from the whitened tensor B (the unrestricted row of
    the paper's functionality table): D_a = C_a C_a^T, D_b = C_b C_b^T, J from
    the total density D_a + D_b (J is linear in D), K per spin, and
    E_J = Tr((D_a + D_b) J)/2, E_K,s = Tr(D_s K_s)/2.  C_b may have no columns."""
    naux, nao, _ = B.shape
    B2 = B.reshape(naux, nao * nao)
    D_a = C_a @ C_a.T
    D_b = C_b @ C_b.T
    D = D_a + D_b
    rho = B2 @ D.ravel()
    J = (rho @ B2).reshape(nao, nao)

    def exchange(C):
        X = np.matmul(B, C).transpose(1, 0, 2).reshape(nao, -1)
        return X @ X.T

    K_a, K_b = exchange(C_a), exchange(C_b)
    return dict(D=D, J=J, K_a=K_a, K_b=K_b, E_J=0.5 * np.sum(D * J),
                E_K_a=0.5 * np.sum(D_a * K_a), E_K_b=0.5 * np.sum(D_b * K_b))


def jk_from_density(B: np.ndarray, D: np.ndarray):
    """J and K from a symmetric density D (not necessarily C C^T): the same
    definitions as steps O8-O10 with D given directly, K = sum_P B_P D B_P."""
    naux, nao, _ = B.shape
    B2 = B.reshape(naux, nao * nao)
    J = ((B2 @ D.ravel()) @ B2).reshape(nao, nao)
    K = np.einsum("Pml,ls,Psn->mn", B, D, B, optimize=True)
    return dict(J=J, K=K, E_J=0.5 * np.sum(D * J), E_K=0.5 * np.sum(D * K))


def coulomb_energy_geometry(basis, aux, coords, D):
    """Energy side of the gradient module the paper benchmarks next to SCF and
    Hessians (section "Speedup of SCF, Gradient, and Hessian Calculations").
    E_J = u^T V^-1 u / 2 with u_P = sum (P|mu nu) D_mu nu at the given atom
    positions (the shells move with their atoms; D is held fixed in the AO
    basis).  LU solve, no Cholesky."""
    V = metric(aux, coords)
    T = three_center(basis, aux, coords)
    u = T.reshape(V.shape[0], -1) @ D.ravel()
    return 0.5 * float(u @ np.linalg.solve(V, u))


def exchange_energy_geometry(basis, aux, coords, D):
    """E_K = sum_P Tr(D B_P D B_P) / 2 at the given atom positions, D held
    fixed, B = L^-1 T (steps O3-O6, O10 with K = sum_P B_P D B_P).  The
    algebraically equal sum_PQ (V^-1)_PQ Tr(D T_P D T_Q) / 2 through a solve
    with V loses ~1e-8 to cancellation when V is ill-conditioned (cond ~1e8
    at six atoms), which finite differences turn into ~1e-5 errors."""
    return energies_geometry(basis, aux, coords, D)[1]


def energies_geometry(basis, aux, coords, D):
    """(E_J, E_K) at the given atom positions from one metric and one set of
    3-centre integrals: E_J = u^T V^-1 u / 2 (LU solve), E_K through
    B = L^-1 T as in exchange_energy_geometry."""
    V = metric(aux, coords)
    T = three_center(basis, aux, coords)
    u = T.reshape(V.shape[0], -1) @ D.ravel()
    e_j = 0.5 * float(u @ np.linalg.solve(V, u))
    L = np.linalg.cholesky(V)
    B = scipy.linalg.solve_triangular(L, T.reshape(V.shape[0], -1), lower=True).reshape(T.shape)
    A = np.matmul(D, B)  # D B_P for every P
    e_k = 0.5 * float(np.sum(A * A.transpose(0, 2, 1)))  # sum_P Tr(D B_P D B_P)
    return e_j, e_k


def gradient_fd(energy, coords, h: float = 2e-3):
    """O11 (the gradients of the section "Speedup of SCF, Gradient, and
    Hessian Calculations", which the paper reports but does not derive):
    d energy(coords)/dR for every atom and direction by central differences
    with Richardson extrapolation (steps h and h/2, error O(h^4)): the
    derivative taken from its definition, for checking an analytic gradient."""
    coords = np.asarray(coords, float)
    g = np.zeros_like(coords)
    for a in range(coords.shape[0]):
        for x in range(3):
            d = []
            for step in (h, h / 2):
                cp, cm = coords.copy(), coords.copy()
                cp[a, x] += step
                cm[a, x] -= step
                d.append((energy(cp) - energy(cm)) / (2 * step))
            g[a, x] = (4 * d[1] - d[0]) / 3
    return g


def coulomb_gradient_fd(basis, aux, coords, D, h: float = 2e-3):
    """dE_J/dR at fixed D by Richardson-extrapolated central differences."""
    return gradient_fd(lambda c: coulomb_energy_geometry(basis, aux, c, D), coords, h)


def exchange_gradient_fd(basis, aux, coords, D, h: float = 2e-3):
    """dE_K/dR at fixed D by Richardson-extrapolated central differences."""
    return gradient_fd(lambda c: exchange_energy_geometry(basis, aux, c, D), coords, h)
