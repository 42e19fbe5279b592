"""Pins for the oracle's J/K steps: symmetry, positivity, energies two ways,
invariance under aux rescaling, under the choice of whitening and under the
orthonormalisation of C_occ (J and K depend on C only through D = C C^T)."""
import json
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2404_09452_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "water_dfjk.json")


def system(name):
    m = I.water() if name == "water" else I.molecule(4, seed=1004)
    nocc = 5 if name == "water" else I.default_nocc(m.nao)
    S = O.overlap(m.orb, m.coords)
    C = I.orthonormalize(I.c_occ_raw(m.nao, nocc, 3000), S)
    T = O.three_center(m.orb, m.aux, m.coords)
    V = O.metric(m.aux, m.coords)
    return m, S, C, T, V


@pytest.fixture(scope="module", params=["water", "mol4"])
def sys_(request):
    m, S, C, T, V = system(request.param)
    return m, S, C, T, V, O.dfjk(m.orb, m.aux, m.coords, C, T=T, V=V)


def test_c_orthonormal(sys_):
    _, S, C, *_ = sys_
    assert np.max(np.abs(C.T @ S @ C - np.eye(C.shape[1]))) < 1e-12


def test_J_K_symmetric_and_K_psd(sys_):
    r = sys_[5]
    J, K = r["J"], r["K"]
    assert np.max(np.abs(J - J.T)) < 1e-13 * np.abs(J).max()
    assert np.max(np.abs(K - K.T)) < 1e-13 * np.abs(K).max()
    assert np.linalg.eigvalsh(K).min() > -1e-12 * np.abs(K).max()


def test_energies_two_ways(sys_):
    m, S, C, T, V, r = sys_
    ej2, ek2 = O.energies_second_way(T, V, r["B"], C)
    assert r["E_J"] == pytest.approx(ej2, rel=1e-12)
    assert r["E_K"] == pytest.approx(ek2, rel=1e-12)
    assert r["E_J"] > 0 and r["E_K"] > 0
    # E_J = rho.rho / 2 with rho = B vec(D)
    assert r["E_J"] == pytest.approx(0.5 * r["rho"] @ r["rho"], rel=1e-12)


def test_whitening_choice_invariance(sys_):
    m, S, C, T, V, r = sys_
    r2 = O.dfjk(m.orb, m.aux, m.coords, C, how="eigh", T=T, V=V)
    assert np.max(np.abs(r2["J"] - r["J"])) < 1e-11 * np.abs(r["J"]).max()
    assert np.max(np.abs(r2["K"] - r["K"])) < 1e-11 * np.abs(r["K"]).max()


def test_aux_rescaling_invariance(sys_):
    m, S, C, T, V, r = sys_
    s = np.random.default_rng(1).uniform(0.3, 3.0, size=V.shape[0])
    r2 = O.dfjk(m.orb, m.aux, m.coords, C, T=T * s[:, None, None], V=V * np.outer(s, s))
    assert np.max(np.abs(r2["J"] - r["J"])) < 1e-11 * np.abs(r["J"]).max()
    assert np.max(np.abs(r2["K"] - r["K"])) < 1e-11 * np.abs(r["K"]).max()


def test_depends_on_C_only_through_D(sys_):
    m, S, C, T, V, r = sys_
    nocc = C.shape[1]
    U, _ = np.linalg.qr(np.random.default_rng(2).standard_normal((nocc, nocc)))
    r2 = O.dfjk(m.orb, m.aux, m.coords, C @ U, T=T, V=V)
    assert np.max(np.abs(r2["K"] - r["K"])) < 1e-11 * np.abs(r["K"]).max()
    # Cholesky (Gram-Schmidt) orthonormalisation of the same raw C0
    C0 = I.c_occ_raw(m.nao, nocc, 3000)
    R = np.linalg.cholesky(C0.T @ S @ C0).T
    r3 = O.dfjk(m.orb, m.aux, m.coords, np.linalg.solve(R.T, C0.T).T, T=T, V=V)
    assert np.max(np.abs(r3["J"] - r["J"])) < 1e-11 * np.abs(r["J"]).max()
    assert np.max(np.abs(r3["K"] - r["K"])) < 1e-11 * np.abs(r["K"]).max()


def test_exact_limit_complete_aux():
    """With one centre and an aux set that spans every orbital product exactly
    (products of s Gaussians are s Gaussians), density fitting is exact:
    E_J equals the 4-centre (ii|jj) energy computed from the closed form."""
    a1, a2 = 0.5, 1.3
    orb = I.Basis([I.Shell(0, 0, np.array([a1]), np.array([1.0])), I.Shell(0, 0, np.array([a2]), np.array([1.0]))])
    aux = I.Basis([I.Shell(0, 0, np.array([e]), np.array([1.0])) for e in (2 * a1, a1 + a2, 2 * a2)])
    xyz = np.zeros((1, 3))
    S = O.overlap(orb, xyz)
    C = I.orthonormalize(np.array([[1.0], [0.4]]), S)
    r = O.dfjk(orb, aux, xyz, C)
    # exact (ab|cd) for s primitives at one centre: 2 pi^2.5/(p q sqrt(p+q))
    ex = np.array([a1, a2])
    nrm = (2 * ex / np.pi) ** 0.75
    D = C @ C.T
    E = 0.0
    for i in range(2):
        for j in range(2):
            for k in range(2):
                for l in range(2):
                    p, q = ex[i] + ex[j], ex[k] + ex[l]
                    v = 2 * np.pi**2.5 / (p * q * np.sqrt(p + q)) * nrm[i] * nrm[j] * nrm[k] * nrm[l]
                    E += 0.5 * D[i, j] * D[k, l] * v
    assert r["E_J"] == pytest.approx(E, rel=1e-12)
    assert r["E_K"] == pytest.approx(E, rel=1e-12)  # one orbital: K = J


def test_water_golden():
    """Stored values written by tests/golden/make_golden.py from this oracle;
    they catch any later drift of the oracle's arithmetic."""
    g = json.load(open(GOLDEN))
    m, S, C, T, V = system("water")
    r = O.dfjk(m.orb, m.aux, m.coords, C, T=T, V=V)
    assert r["E_J"] == pytest.approx(g["E_J"], rel=1e-13)
    assert r["E_K"] == pytest.approx(g["E_K"], rel=1e-13)
    assert np.allclose(r["J"], np.array(g["J"]), rtol=0, atol=1e-13)
    assert np.allclose(r["K"], np.array(g["K"]), rtol=0, atol=1e-13)


# ---- spin-unrestricted densities (two occupied sets) -------------------------------


def test_uks_one_electron_has_no_two_electron_energy(sys_):
    """A single occupied spin orbital: the Coulomb self-energy equals its
    exchange self-energy (both are sum_P (c^T B_P c)^2 / 2), so the
    two-electron energy vanishes — also within density fitting."""
    _, _, C, _, _, r = sys_
    u = O.dfjk_uks(r["B"], C[:, :1], C[:, :0])
    assert abs(u["E_J"] - u["E_K_a"]) < 1e-13 * abs(u["E_J"]) and u["E_K_b"] == 0.0
    assert np.max(np.abs(u["K_b"])) == 0.0


def test_uks_closed_shell_limit(sys_):
    """C_a = C_b = C: J doubles, each K is the restricted one, E_J is 4x."""
    _, _, C, _, _, r = sys_
    u = O.dfjk_uks(r["B"], C, C)
    assert np.max(np.abs(u["J"] - 2 * r["J"])) < 1e-12 * np.abs(r["J"]).max()
    assert np.max(np.abs(u["K_a"] - r["K"])) < 1e-13 * np.abs(r["K"]).max()
    assert np.array_equal(u["K_a"], u["K_b"])
    assert abs(u["E_J"] - 4 * r["E_J"]) < 1e-12 * abs(r["E_J"])


def test_uks_coulomb_from_fitted_coefficients(sys_):
    """E_J of the total density through the fitted coefficients d = V^-1 u of
    u_P = sum (P|mu nu)(D_a + D_b)_mu nu (LU solve, no Cholesky, no B), and the
    exchange energies as sum_P ||C_s^T B_P C_s||^2 / 2."""
    _, _, C, T, V, r = sys_
    nb = max(1, C.shape[1] - 2)
    Ca, Cb = C, C[:, ::-1][:, :nb].copy()
    u = O.dfjk_uks(r["B"], Ca, Cb)
    naux = V.shape[0]
    ut = T.reshape(naux, -1) @ (Ca @ Ca.T + Cb @ Cb.T).ravel()
    assert abs(u["E_J"] - 0.5 * ut @ np.linalg.solve(V, ut)) < 1e-10 * abs(u["E_J"])
    for Cs, key in ((Ca, "E_K_a"), (Cb, "E_K_b")):
        M = np.einsum("mi,Pmn,nj->Pij", Cs, r["B"], Cs, optimize=True)
        assert abs(u[key] - 0.5 * np.sum(M * M)) < 1e-12 * abs(u[key])


# ---- J and K from a density -------------------------------------------------------


def test_density_path_equals_orbital_path(sys_):
    """D = C C^T: the density route (K = sum_P B_P D B_P) equals the orbital
    route (K = sum_P (B_P C)(B_P C)^T), which never forms D B_P."""
    _, _, C, _, _, r = sys_
    d = O.jk_from_density(r["B"], C @ C.T)
    assert np.max(np.abs(d["J"] - r["J"])) < 1e-12 * np.abs(r["J"]).max()
    assert np.max(np.abs(d["K"] - r["K"])) < 1e-12 * np.abs(r["K"]).max()
    assert abs(d["E_K"] - r["E_K"]) < 1e-12 * abs(r["E_K"])


def test_density_path_is_linear_and_signed(sys_):
    """J and K are linear in D; for D = D1 - D2 (not positive semidefinite) the
    result is the difference of the two orbital builds."""
    _, _, C, _, _, r = sys_
    n = C.shape[1]
    C1, C2 = C[:, : (n + 1) // 2], C[:, (n + 1) // 2 :]
    d = O.jk_from_density(r["B"], C1 @ C1.T - C2 @ C2.T)
    r1, r2 = O.jk_from_B(r["B"], C1), O.jk_from_B(r["B"], C2)
    assert np.max(np.abs(d["J"] - (r1["J"] - r2["J"]))) < 1e-12 * np.abs(r["J"]).max()
    assert np.max(np.abs(d["K"] - (r1["K"] - r2["K"]))) < 1e-12 * np.abs(r["K"]).max()
