"""GPU parity of the CUDA DF-J/K path against the FP64 CPU oracle, called
through the C ABI.  Tolerances: the accuracy bar (|dE| <= 1e-6 Eh,
max|dJ|, max|dK| <= 1e-7) is asserted everywhere; the FP64 path additionally
must stay within 1e-9 of the oracle (FP64 rounding differences only)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2404_09452_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2404_09452_gb300 import dfjk  # noqa: E402

E_TOL, JK_TOL, FP64_TOL = 1e-6, 1e-7, 1e-9


def pin_system():
    rng = np.random.default_rng(11)
    coords = rng.uniform(-1.3, 1.3, size=(3, 3))
    orb, aux = [], []
    for l in range(3):
        a = rng.uniform(0.3, 1.5)
        orb.append(I.Shell(l % 3, l, np.array([a, 2.5 * a]), rng.uniform(0.2, 1.0, 2)))
        orb.append(I.Shell((l + 1) % 3, l, np.array([1.3 * a, 3.25 * a]), rng.uniform(0.2, 1.0, 2)))
        aux.append(I.Shell((l + 2) % 3, l, np.array([rng.uniform(0.4, 2.0)]), np.array([1.0])))
        aux.append(I.Shell(l % 3, l, np.array([rng.uniform(0.4, 2.0)]), np.array([1.0])))
    return I.Molecule(coords, I.Basis(orb), I.Basis(aux), "pin")


SYSTEMS = {
    "water": lambda: (I.water(), 5),
    "pin": lambda: (pin_system(), 4),
    "mol4": lambda: (I.molecule(4, seed=1004), None),
    "mol12": lambda: (I.molecule(12, seed=1012), None),
}


@pytest.fixture(scope="module", params=list(SYSTEMS))
def case(request):
    m, nocc = SYSTEMS[request.param]()
    nocc = nocc or I.default_nocc(m.nao)
    S = O.overlap(m.orb, m.coords)
    C = I.orthonormalize(I.c_occ_raw(m.nao, nocc, 3000), S)
    ref = O.dfjk(m.orb, m.aux, m.coords, C)
    ref["S"] = S
    h = dfjk.Handle(m)
    yield request.param, m, C, ref, h
    h.close()


def test_boys_device_vs_oracle():
    T = np.concatenate([[0.0, 1e-12], np.logspace(-8, np.log10(300.0), 400), [39.95, 40.0, 40.05]])
    F = dfjk.boys(8, torch.from_numpy(T).cuda()).cpu().numpy()
    for i, t in enumerate(T):
        ref = O.boys(8, t)
        np.testing.assert_allclose(F[i], ref, rtol=2e-14, atol=0)


def test_overlap(case):
    _, m, _, ref, h = case
    S = h.overlap().cpu().numpy()
    assert np.max(np.abs(S - ref["S"])) < 1e-13


def test_metric(case):
    _, m, _, ref, h = case
    V = h.metric().cpu().numpy()
    assert np.max(np.abs(V - ref["V"])) < 1e-12 * max(1.0, np.abs(ref["V"]).max())


def test_three_center(case):
    _, m, _, ref, h = case
    T = h.three_center().cpu().numpy()
    # screened pairs (threshold 1e-12) may differ by the Schwarz bound
    assert np.max(np.abs(T - ref["T"])) < 1e-11


def test_cholesky_and_B(case):
    """The Cholesky factor is pinned by its backward error, which does not depend
    on conditioning; its forward error is bounded by 32 cond(V) u max|L| (the
    metric of these molecules has cond up to ~1e8, so two correct FP64
    factorisations legitimately differ by ~1e-9)."""
    _, m, _, ref, h = case
    u = np.finfo(float).eps / 2
    V, T = ref["V"], ref["T"]
    kappa = np.linalg.cond(V)
    L = h.cholesky().cpu().numpy()
    assert np.array_equal(L, np.tril(L)) and np.all(np.diag(L) > 0)
    assert np.max(np.abs(L @ L.T - V)) < 1e-13 * np.abs(V).max()
    assert np.max(np.abs(L - ref["L"])) < 32 * kappa * u * np.abs(ref["L"]).max()
    B = h.B().cpu().numpy()
    naux = V.shape[0]
    resid = L @ B.reshape(naux, -1) - T.reshape(naux, -1)
    assert np.max(np.abs(resid)) < 1e-11 * max(1.0, np.abs(T).max())
    assert np.max(np.abs(B - ref["B"])) < 32 * kappa * u * max(1.0, np.abs(ref["B"]).max())


def test_jk_energies(case):
    name, m, C, ref, h = case
    J, K, EJ, EK = h.build(torch.from_numpy(C).cuda())
    J, K = J[0].cpu().numpy(), K[0].cpu().numpy()
    dJ, dK = np.max(np.abs(J - ref["J"])), np.max(np.abs(K - ref["K"]))
    dEJ, dEK = abs(EJ[0] - ref["E_J"]), abs(EK[0] - ref["E_K"])
    assert dJ <= JK_TOL and dK <= JK_TOL and dEJ <= E_TOL and dEK <= E_TOL
    assert dJ <= FP64_TOL and dK <= FP64_TOL, (name, dJ, dK)
    assert dEJ <= FP64_TOL * max(1, abs(ref["E_J"])) and dEK <= FP64_TOL * max(1, abs(ref["E_K"]))
    assert np.array_equal(J, J.T) and np.array_equal(K, K.T)


def test_two_sets_and_repeat_is_bitwise(case):
    name, m, C, ref, h = case
    C2 = np.stack([C, C[:, ::-1].copy()])
    J, K, EJ, EK = h.build(torch.from_numpy(C2).cuda())
    J1, K1, EJ1, EK1 = h.build(torch.from_numpy(C).cuda())
    # a reversed column order of C leaves D, J, K unchanged mathematically
    assert np.max(np.abs(J[1].cpu().numpy() - ref["J"])) < FP64_TOL
    assert np.max(np.abs(K[1].cpu().numpy() - ref["K"])) < FP64_TOL
    # same input, same handle: bitwise identical (fixed reduction order)
    assert torch.equal(J[0], J1[0]) and torch.equal(K[0], K1[0])
    assert EJ[0] == EJ1[0] and EK[0] == EK1[0]


def test_evict_and_recompute():
    m = I.molecule(4, seed=1004)
    S = O.overlap(m.orb, m.coords)
    C = torch.from_numpy(I.orthonormalize(I.c_occ_raw(m.nao, 12, 3000), S)).cuda()
    h = dfjk.Handle(m)
    J0, K0, EJ0, EK0 = h.build(C)
    J0, K0 = J0.clone(), K0.clone()
    h.evict()
    J1, K1, EJ1, EK1 = h.build(C)
    assert torch.equal(J0, J1) and torch.equal(K0, K1) and EJ0[0] == EJ1[0]
    h.close()


def test_single_atom_and_nocc_one():
    m = I.molecule(1, seed=7)
    S = O.overlap(m.orb, m.coords)
    C = I.orthonormalize(I.c_occ_raw(m.nao, 1, 3000), S)
    ref = O.dfjk(m.orb, m.aux, m.coords, C)
    h = dfjk.Handle(m)
    J, K, EJ, EK = h.build(torch.from_numpy(C).cuda())
    assert np.max(np.abs(J[0].cpu().numpy() - ref["J"])) < FP64_TOL
    assert np.max(np.abs(K[0].cpu().numpy() - ref["K"])) < FP64_TOL
    h.close()


def test_errors_are_reported_not_raised_on_device():
    m = I.water()
    bad = I.Molecule(m.coords, I.Basis(m.orb.shells + [I.Shell(0, 3, np.array([1.0]), np.array([1.0]))]), m.aux)
    with pytest.raises(dfjk.DfjkError) as e:
        dfjk.Handle(bad)
    assert e.value.code == 2  # DFJK_ERR_UNSUPPORTED
    bad = I.Molecule(m.coords, I.Basis([I.Shell(5, 0, np.array([1.0]), np.array([1.0]))]), m.aux)
    with pytest.raises(dfjk.DfjkError) as e:
        dfjk.Handle(bad)
    assert e.value.code == 1  # DFJK_ERR_ARG
    bad = I.Molecule(m.coords, I.Basis([I.Shell(0, 0, np.array([-1.0]), np.array([1.0]))]), m.aux)
    with pytest.raises(dfjk.DfjkError):
        dfjk.Handle(bad)


def test_singular_metric_reports_not_pd():
    m = I.water()
    aux = I.Basis(m.aux.shells + [m.aux.shells[0]])  # duplicated aux shell: V singular
    with pytest.raises(dfjk.DfjkError) as e:
        dfjk.Handle(I.Molecule(m.coords, m.orb, aux))
    assert e.value.code == 3  # DFJK_ERR_NOT_PD
    # the context stays usable afterwards
    h = dfjk.Handle(m)
    h.close()


def test_budget_rejects_setup():
    m = I.molecule(4, seed=1004)
    with pytest.raises(dfjk.DfjkError) as e:
        dfjk.Handle(m, hbm_budget_bytes=1024)
    assert e.value.code == 5  # DFJK_ERR_BUDGET


def test_screening_drops_only_negligible_pairs():
    """A sparse molecule: the Schwarz-dropped pairs carry oracle integrals
    below the threshold, and kept/dropped J, K match the unscreened oracle."""
    xyz = np.array([[0.0, 0.0, 0.0], [0.0, 0.0, 30.0], [0.0, 30.0, 0.0]])
    m0 = I.molecule(3, seed=3)
    m = I.Molecule(xyz, m0.orb, m0.aux)
    h = dfjk.Handle(m)
    mask = h.pair_mask().cpu().numpy()
    assert 0 < mask.sum() < mask.size
    T = O.three_center(m.orb, m.aux, m.coords)
    off = np.cumsum([0] + [(s.l + 1) * (s.l + 2) // 2 for s in m.orb.shells])
    for a in range(len(m.orb.shells)):
        for b in range(len(m.orb.shells)):
            if not mask[a, b]:
                assert np.abs(T[:, off[a]:off[a + 1], off[b]:off[b + 1]]).max() < 1e-12
    S = O.overlap(m.orb, m.coords)
    C = I.orthonormalize(I.c_occ_raw(m.nao, 9, 3000), S)
    ref = O.dfjk(m.orb, m.aux, m.coords, C, T=T)
    J, K, EJ, EK = h.build(torch.from_numpy(C).cuda())
    assert np.max(np.abs(J[0].cpu().numpy() - ref["J"])) < 1e-10
    assert np.max(np.abs(K[0].cpu().numpy() - ref["K"])) < 1e-10
    h.close()
