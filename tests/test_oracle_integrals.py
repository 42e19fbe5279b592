"""Pins for the oracle's Gaussian integrals: brute-force quadrature for every
class up to (dd|d), closed forms, symmetry, invariance and the far-field limit.

A dropped or mis-signed term in the Obara-Saika recursion, a wrong HRR index
or a wrong normalisation changes at least one of these by far more than the
tolerances used here."""
import math

import numpy as np
import pytest

import quadrature as Q
from oracle import oracle as O
from paper_2404_09452_gb300 import inputs as I


def pin_system():
    """Three centres, shells of every l on each, random exponents/coefs."""
    rng = np.random.default_rng(11)
    coords = rng.uniform(-1.3, 1.3, size=(3, 3))
    orb, aux = [], []
    for l in range(3):
        a = rng.uniform(0.3, 1.5)
        orb.append(I.Shell(l % 3, l, np.array([a, 2.5 * a]), rng.uniform(0.2, 1.0, 2)))
        orb.append(I.Shell((l + 1) % 3, l, np.array([1.3 * a, 3.25 * a]), rng.uniform(0.2, 1.0, 2)))
        aux.append(I.Shell((l + 2) % 3, l, np.array([rng.uniform(0.4, 2.0)]), np.array([1.0])))
    return coords, I.Basis(orb), I.Basis(aux)


def offsets(basis):
    return np.cumsum([0] + [O.ncart(s.l) for s in basis.shells])


@pytest.fixture(scope="module")
def pin():
    coords, orb, aux = pin_system()
    return coords, orb, aux, O.three_center(orb, aux, coords), O.metric(aux, coords)


def test_three_center_vs_quadrature(pin):
    coords, orb, aux, T, _ = pin
    oo, oa = offsets(orb), offsets(aux)
    seen = set()
    for ia, sa in enumerate(orb.shells):
        for ib, sb in enumerate(orb.shells):
            for ic, sc in enumerate(aux.shells):
                cls = (sa.l, sb.l, sc.l)
                if cls in seen:
                    continue
                seen.add(cls)
                comps = [
                    (ca, cb, cc)
                    for ca in range(O.ncart(sa.l))
                    for cb in range(O.ncart(sb.l))
                    for cc in range(O.ncart(sc.l))
                ]
                for ca, cb, cc in (comps[0], comps[len(comps) // 2], comps[-1]):
                    pa, pb, pc = (
                        O.cart_powers(sa.l)[ca],
                        O.cart_powers(sb.l)[cb],
                        O.cart_powers(sc.l)[cc],
                    )
                    ref = Q.contracted_3c(
                        sa, coords[sa.atom], pa, sb, coords[sb.atom], pb, sc, coords[sc.atom], pc, 300
                    )
                    got = T[oa[ic] + cc, oo[ia] + ca, oo[ib] + cb]
                    assert abs(got - ref) < 1e-11 * max(1.0, abs(ref)), (cls, pa, pb, pc, got, ref)
    assert len(seen) == 27


def test_metric_vs_quadrature(pin):
    coords, _, aux, _, V = pin
    oa = offsets(aux)
    for ip, sp in enumerate(aux.shells):
        for iq, sq in enumerate(aux.shells):
            for cp in {0, O.ncart(sp.l) - 1}:
                for cq in {0, O.ncart(sq.l) // 2}:
                    pp, pq = O.cart_powers(sp.l)[cp], O.cart_powers(sq.l)[cq]
                    ref = Q.contracted_2c(sp, coords[sp.atom], pp, sq, coords[sq.atom], pq, 300)
                    assert abs(V[oa[ip] + cp, oa[iq] + cq] - ref) < 1e-11 * max(1.0, abs(ref))


def _n_s(a):
    return (2 * a / math.pi) ** 0.75


def test_ss_s_closed_form():
    """(ab|c) = 2 pi^2.5 / (p g sqrt(p+g)) K_ab F_0(pg/(p+g) |PC|^2) for s primitives."""
    A, B, C = np.array([0.1, -0.4, 0.3]), np.array([1.2, 0.5, -0.7]), np.array([-0.9, 1.4, 2.2])
    a, b, g = 0.7, 1.9, 0.45
    coords = np.array([A, B, C])
    orb = I.Basis([I.Shell(0, 0, np.array([a]), np.array([1.0])), I.Shell(1, 0, np.array([b]), np.array([1.0]))])
    aux = I.Basis([I.Shell(2, 0, np.array([g]), np.array([1.0]))])
    T = O.three_center(orb, aux, coords)
    p = a + b
    P = (a * A + b * B) / p
    K = math.exp(-a * b / p * np.sum((A - B) ** 2))
    x = p * g / (p + g) * np.sum((P - C) ** 2)
    F0 = 0.5 * math.sqrt(math.pi / x) * math.erf(math.sqrt(x))
    ref = 2 * math.pi**2.5 / (p * g * math.sqrt(p + g)) * K * F0 * _n_s(a) * _n_s(b) * _n_s(g)
    assert T[0, 0, 1] == pytest.approx(ref, rel=1e-14)
    assert T[0, 1, 0] == pytest.approx(ref, rel=1e-14)


def test_s_s_closed_form():
    A, C = np.array([0.3, 0.2, -0.5]), np.array([-1.1, 0.8, 0.9])
    a, g = 0.6, 2.3
    aux = I.Basis([I.Shell(0, 0, np.array([a]), np.array([1.0])), I.Shell(1, 0, np.array([g]), np.array([1.0]))])
    V = O.metric(aux, np.array([A, C]))
    x = a * g / (a + g) * np.sum((A - C) ** 2)
    F0 = 0.5 * math.sqrt(math.pi / x) * math.erf(math.sqrt(x))
    ref = 2 * math.pi**2.5 / (a * g * math.sqrt(a + g)) * F0 * _n_s(a) * _n_s(g)
    assert V[0, 1] == pytest.approx(ref, rel=1e-14)


def test_overlap_unit_diagonal_and_pd():
    m = I.molecule(4, seed=5)
    S = O.overlap(m.orb, m.coords)
    assert np.max(np.abs(np.diag(S) - 1.0)) < 1e-14
    assert np.max(np.abs(S - S.T)) < 1e-15
    assert np.linalg.eigvalsh(S).min() > 0


def test_overlap_ss_closed_form():
    A, B = np.array([0.0, 0.0, 0.0]), np.array([0.4, -0.3, 1.1])
    a, b = 0.9, 0.35
    orb = I.Basis([I.Shell(0, 0, np.array([a]), np.array([1.0])), I.Shell(1, 0, np.array([b]), np.array([1.0]))])
    S = O.overlap(orb, np.array([A, B]))
    p = a + b
    ref = (math.pi / p) ** 1.5 * math.exp(-a * b / p * np.sum((A - B) ** 2)) * _n_s(a) * _n_s(b)
    assert S[0, 1] == pytest.approx(ref, rel=1e-14)


def test_pair_symmetry_two_evaluations(pin):
    _, _, _, T, _ = pin
    assert np.max(np.abs(T - T.transpose(0, 2, 1))) < 1e-14 * max(1.0, np.abs(T).max())
    m = I.water()
    Tw = O.three_center(m.orb, m.aux, m.coords)
    assert np.max(np.abs(Tw - Tw.transpose(0, 2, 1))) < 1e-13


def test_sym_option_matches_full(pin):
    coords, orb, aux, T, _ = pin
    Ts = O.three_center(orb, aux, coords, sym=True)
    assert np.max(np.abs(Ts - T)) < 1e-14


def test_triples_entry_matches_full(pin):
    coords, orb, aux, T, _ = pin
    oo, oa = offsets(orb), offsets(aux)
    trip = [(0, 5, 2), (3, 1, 0), (4, 4, 1)]
    for (a, b, c), blk in zip(trip, O.three_center_triples(orb, aux, coords, trip)):
        ref = T[oa[c] : oa[c + 1], oo[a] : oo[a + 1], oo[b] : oo[b + 1]].transpose(1, 2, 0)
        assert np.array_equal(blk, ref)


def test_metric_symmetric_positive_definite(pin):
    _, _, _, _, V = pin
    assert np.max(np.abs(V - V.T)) < 1e-14 * np.abs(V).max()
    assert np.linalg.eigvalsh(V).min() > 0
    m = I.molecule(3, seed=9)
    Vm = O.metric(m.aux, m.coords)
    assert np.linalg.eigvalsh(Vm).min() > 0


def test_translation_invariance(pin):
    coords, orb, aux, T, V = pin
    shift = np.array([3.7, -12.25, 0.6])
    T2 = O.three_center(orb, aux, coords + shift)
    V2 = O.metric(aux, coords + shift)
    S1, S2 = O.overlap(orb, coords), O.overlap(orb, coords + shift)
    assert np.max(np.abs(T2 - T)) < 1e-13
    assert np.max(np.abs(V2 - V)) < 1e-13
    assert np.max(np.abs(S2 - S1)) < 1e-14


def _swap_xy_perm(basis):
    """AO permutation induced by exchanging the x and y axes."""
    perm = []
    off = 0
    for s in basis.shells:
        pw = O.cart_powers(s.l)
        for i, j, k in pw:
            perm.append(off + pw.index((j, i, k)))
        off += len(pw)
    return np.array(perm)


def test_axis_swap_covariance(pin):
    coords, orb, aux, T, V = pin
    sw = coords[:, [1, 0, 2]]
    T2 = O.three_center(orb, aux, sw)
    V2 = O.metric(aux, sw)
    po, pa = _swap_xy_perm(orb), _swap_xy_perm(aux)
    assert np.max(np.abs(T2 - T[np.ix_(pa, po, po)])) < 1e-13
    assert np.max(np.abs(V2 - V[np.ix_(pa, pa)])) < 1e-13


def test_far_field_monopole_limit():
    """An s aux function at distance R from a compact pair: (P|mu nu) ->
    S_mu_nu N_P (pi/g)^1.5 / R, with the error falling like 1/R (dipole)."""
    rng = np.random.default_rng(3)
    A, B = np.array([0.0, 0.0, 0.0]), np.array([0.5, 0.2, -0.3])
    orb = I.Basis(
        [I.Shell(0, 1, np.array([0.8, 2.0]), rng.uniform(0.2, 1, 2)),
         I.Shell(1, 2, np.array([1.1, 2.75]), rng.uniform(0.2, 1, 2))]
    )
    g = 0.9
    aux = I.Basis([I.Shell(2, 0, np.array([g]), np.array([1.0]))])
    direction = np.array([0.3, -0.5, 0.81])
    direction /= np.linalg.norm(direction)
    errs = []
    for R in (40.0, 80.0, 160.0):
        coords = np.array([A, B, R * direction])
        T = O.three_center(orb, aux, coords)[0]
        S = O.overlap(orb, coords[:2])
        mono = S * _n_s(g) * (math.pi / g) ** 1.5 / R
        errs.append(np.max(np.abs(T - mono)) / np.max(np.abs(mono)))
    assert errs[0] < 0.05
    assert errs[1] == pytest.approx(errs[0] / 2, rel=0.1)
    assert errs[2] == pytest.approx(errs[1] / 2, rel=0.1)
