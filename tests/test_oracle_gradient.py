"""Pins for the oracle's Coulomb gradient by finite differences: the energy
it differentiates equals the oracle's E_J, translations leave the energy
unchanged (the gradients sum to zero), and the extrapolated difference
agrees with a finer plain central difference."""
import numpy as np

from oracle import oracle as O
from paper_2404_09452_gb300 import inputs as I


def _water():
    m = I.water()
    S = O.overlap(m.orb, m.coords)
    C = I.orthonormalize(I.c_occ_raw(m.nao, 5, 3000), S)
    return m, C @ C.T, C


def test_energy_matches_oracle_e_j():
    m, D, C = _water()
    r = O.dfjk(m.orb, m.aux, m.coords, C)
    assert abs(O.coulomb_energy_geometry(m.orb, m.aux, m.coords, D) - r["E_J"]) < 1e-11 * abs(r["E_J"])


def test_gradient_sums_to_zero_and_converges():
    m, D, _ = _water()
    g = O.coulomb_gradient_fd(m.orb, m.aux, m.coords, D)
    assert np.max(np.abs(g.sum(axis=0))) < 1e-7 * np.abs(g).max()
    # one component by a plain central difference with a small step
    a, x, h = 1, 2, 2e-4
    cp, cm = m.coords.copy(), m.coords.copy()
    cp[a, x] += h
    cm[a, x] -= h
    fd = (O.coulomb_energy_geometry(m.orb, m.aux, cp, D) - O.coulomb_energy_geometry(m.orb, m.aux, cm, D)) / (2 * h)
    assert abs(fd - g[a, x]) < 1e-6 * max(1.0, abs(g[a, x]))


def test_exchange_energy_matches_oracle_e_k():
    m, D, C = _water()
    r = O.dfjk(m.orb, m.aux, m.coords, C)
    assert abs(O.exchange_energy_geometry(m.orb, m.aux, m.coords, D) - r["E_K"]) < 1e-11 * abs(r["E_K"])


def test_exchange_gradient_sums_to_zero_and_converges():
    m, D, _ = _water()
    g = O.exchange_gradient_fd(m.orb, m.aux, m.coords, D)
    assert np.abs(g).max() > 1e-3
    assert np.max(np.abs(g.sum(axis=0))) < 1e-7 * np.abs(g).max()
    a, x, h = 0, 0, 2e-4
    cp, cm = m.coords.copy(), m.coords.copy()
    cp[a, x] += h
    cm[a, x] -= h
    fd = (O.exchange_energy_geometry(m.orb, m.aux, cp, D) - O.exchange_energy_geometry(m.orb, m.aux, cm, D)) / (2 * h)
    assert abs(fd - g[a, x]) < 1e-6 * max(1.0, abs(g[a, x]))


def test_one_occupied_orbital_exchange_is_coulomb():
    """With one occupied orbital (D = c c^T, rank one) Tr(D T_P D T_Q) = u_P u_Q,
    so E_K = E_J at every geometry and the two gradients coincide."""
    m = I.water()
    S = O.overlap(m.orb, m.coords)
    C = I.orthonormalize(I.c_occ_raw(m.nao, 1, 3002), S)
    D = C @ C.T
    gj = O.coulomb_gradient_fd(m.orb, m.aux, m.coords, D)
    gk = O.exchange_gradient_fd(m.orb, m.aux, m.coords, D)
    assert np.max(np.abs(gj - gk)) < 1e-9 * max(1.0, np.abs(gj).max())


def test_exchange_gradient_step_independent():
    """Roundoff in the energy would show as a step-size dependence of the
    extrapolated difference (it grows like 1/h); truncation shrinks like h^4."""
    m = I.molecule(4, seed=1004)
    S = O.overlap(m.orb, m.coords)
    C = I.orthonormalize(I.c_occ_raw(m.nao, I.default_nocc(m.nao), 3000), S)
    D = C @ C.T
    g1 = O.exchange_gradient_fd(m.orb, m.aux, m.coords, D, h=2e-3)
    g2 = O.exchange_gradient_fd(m.orb, m.aux, m.coords, D, h=5e-4)
    assert np.max(np.abs(g1 - g2)) < 1e-8 * max(1.0, np.abs(g1).max())
