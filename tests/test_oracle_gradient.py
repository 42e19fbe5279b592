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


def _ssc_and_grad(xa, XA, xb, XB, g, C):
    """(ab|c) for normalised s primitives and its derivatives with respect to
    A, B and C, written out from the closed form
    (ab|c) = N 2 pi^2.5 / (p g sqrt(p + g)) K_ab F_0(x), x = p g / (p + g) |P - C|^2,
    with dF_0/dx = -F_1 and F_1 = (F_0 - e^-x) / (2x)."""
    import math
    p = xa + xb
    P = (xa * XA + xb * XB) / p
    AB = XA - XB
    K = math.exp(-xa * xb / p * AB @ AB)
    rho = p * g / (p + g)
    PC = P - C
    x = rho * PC @ PC
    F0 = 0.5 * math.sqrt(math.pi / x) * math.erf(math.sqrt(x))
    F1 = (F0 - math.exp(-x)) / (2 * x)
    N = (2 * xa / math.pi) ** 0.75 * (2 * xb / math.pi) ** 0.75 * (2 * g / math.pi) ** 0.75
    pref = N * 2 * math.pi**2.5 / (p * g * math.sqrt(p + g))
    dK_dA = K * (-2 * xa * xb / p) * AB
    dx_dP = 2 * rho * PC
    dA = pref * (dK_dA * F0 - K * F1 * dx_dP * (xa / p))
    dB = pref * (-dK_dA * F0 - K * F1 * dx_dP * (xb / p))
    dC = pref * (K * F1 * dx_dP)
    return pref * K * F0, dA, dB, dC


def test_coulomb_gradient_closed_form():
    """Two s orbitals and one s aux function on three atoms: V = (c|c) does
    not move, so E_J = u^2 / (2V) and dE_J/dR = (u / V) du/dR with u written
    from the closed-form (ab|c) above; the finite-difference oracle agrees."""
    import math
    A, B, Cc = np.array([0.1, -0.4, 0.3]), np.array([1.2, 0.5, -0.7]), np.array([-0.9, 1.4, 2.2])
    a, b, g = 0.7, 1.9, 0.45
    coords = np.array([A, B, Cc])
    orb = I.Basis([I.Shell(0, 0, np.array([a]), np.array([1.0])), I.Shell(1, 0, np.array([b]), np.array([1.0]))])
    aux = I.Basis([I.Shell(2, 0, np.array([g]), np.array([1.0]))])
    D = np.array([[0.9, -0.35], [-0.35, 0.6]])
    V = 2 * math.pi**2.5 / (g * g * math.sqrt(2 * g)) * (2 * g / math.pi) ** 1.5  # (c|c)
    u, gA, gB, gC = 0.0, np.zeros(3), np.zeros(3), np.zeros(3)
    for (i, xi, Xi), (j, xj, Xj) in (((0, a, A), (0, a, A)), ((0, a, A), (1, b, B)), ((1, b, B), (1, b, B))):
        w = D[i, j] * (1.0 if i == j else 2.0)
        val, dX, dY, dC = _ssc_and_grad(xi, Xi, xj, Xj, g, Cc)
        u += w * val
        for atom, d in ((i, dX), (j, dY)):
            (gA if atom == 0 else gB)[:] += w * d
        gC += w * dC
    ref = (u / V) * np.array([gA, gB, gC])
    assert abs(O.coulomb_energy_geometry(orb, aux, coords, D) - 0.5 * u * u / V) < 1e-13 * u * u / V
    g_fd = O.coulomb_gradient_fd(orb, aux, coords, D)
    assert np.max(np.abs(g_fd - ref)) < 1e-9 * np.abs(ref).max(), (g_fd, ref)


def test_exchange_gradient_closed_form():
    """Same three-atom system: with one aux function E_K = Tr(D T D T) / (2V)
    for the 2 x 2 matrix T_ab = (ab|c), so dE_K/dR = Tr(D dT/dR D T) / V."""
    import math
    A, B, Cc = np.array([0.1, -0.4, 0.3]), np.array([1.2, 0.5, -0.7]), np.array([-0.9, 1.4, 2.2])
    a, b, g = 0.7, 1.9, 0.45
    coords = np.array([A, B, Cc])
    orb = I.Basis([I.Shell(0, 0, np.array([a]), np.array([1.0])), I.Shell(1, 0, np.array([b]), np.array([1.0]))])
    aux = I.Basis([I.Shell(2, 0, np.array([g]), np.array([1.0]))])
    D = np.array([[0.9, -0.35], [-0.35, 0.6]])
    V = 2 * math.pi**2.5 / (g * g * math.sqrt(2 * g)) * (2 * g / math.pi) ** 1.5
    ex, X = (a, b), (A, B)
    T = np.zeros((2, 2))
    dT = np.zeros((3, 3, 2, 2))  # [atom][direction][mu][nu]
    for i in range(2):
        for j in range(2):
            val, dX, dY, dC = _ssc_and_grad(ex[i], X[i], ex[j], X[j], g, Cc)
            T[i, j] = val
            dT[i, :, i, j] += dX
            dT[j, :, i, j] += dY
            dT[2, :, i, j] += dC
    DT = D @ T
    assert abs(O.exchange_energy_geometry(orb, aux, coords, D) - 0.5 * np.trace(DT @ DT) / V) < 1e-13
    ref = np.array([[np.trace(D @ dT[k, x] @ DT) / V for x in range(3)] for k in range(3)])
    g_fd = O.exchange_gradient_fd(orb, aux, coords, D)
    assert np.max(np.abs(g_fd - ref)) < 1e-9 * np.abs(ref).max(), (g_fd, ref)
