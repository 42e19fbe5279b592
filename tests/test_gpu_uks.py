"""Spin-unrestricted build (dfjk_build_uks) against the oracle: J of the total
density, K per spin, E = [E_J, E_K alpha, E_K beta]; FP64 and mixed paths."""
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


def _case(name):
    if name == "water+":  # a doublet cation: 5 alpha, 4 beta electrons
        m, na, nb = I.water(), 5, 4
    else:
        m = I.molecule(12, seed=1012)
        na = I.default_nocc(m.nao)
        nb = na - 3
    S = O.overlap(m.orb, m.coords)
    Ca = I.orthonormalize(I.c_occ_raw(m.nao, na, 3000), S)
    Cb = I.orthonormalize(I.c_occ_raw(m.nao, nb, 3001), S)
    r = O.dfjk(m.orb, m.aux, m.coords, Ca)
    return m, Ca, Cb, O.dfjk_uks(r["B"], Ca, Cb)


@pytest.mark.parametrize("name", ["water+", "mol12"])
@pytest.mark.parametrize("precision", [dfjk.DFJK_FP64, dfjk.DFJK_MIXED])
def test_uks_vs_oracle(name, precision):
    m, Ca, Cb, ref = _case(name)
    h = dfjk.Handle(m, precision=precision)
    J, Ka, Kb, E = h.build_uks(torch.from_numpy(Ca).cuda(), torch.from_numpy(Cb).cuda())
    h.close()
    tol = FP64_TOL if precision == dfjk.DFJK_FP64 else JK_TOL
    assert np.max(np.abs(J.cpu().numpy() - ref["J"])) < tol
    assert np.max(np.abs(Ka.cpu().numpy() - ref["K_a"])) < tol
    assert np.max(np.abs(Kb.cpu().numpy() - ref["K_b"])) < tol
    etol = FP64_TOL * 10 if precision == dfjk.DFJK_FP64 else E_TOL
    for got, key in zip(E, ("E_J", "E_K_a", "E_K_b")):
        assert abs(got - ref[key]) < etol * max(1.0, abs(ref[key])), key


@pytest.mark.parametrize("precision", [dfjk.DFJK_FP64, dfjk.DFJK_MIXED])
def test_uks_closed_shell_limit_is_bitwise(precision):
    """C_a = C_b = C: K_a = K_b = K (same kernels, same order), J = 2 J and
    E_J = 4 E_J exactly (scaling by powers of two commutes with rounding)."""
    m = I.molecule(4, seed=1004)
    S = O.overlap(m.orb, m.coords)
    C = torch.from_numpy(I.orthonormalize(I.c_occ_raw(m.nao, I.default_nocc(m.nao), 3000), S)).cuda()
    h = dfjk.Handle(m, precision=precision)
    J0, K0, EJ0, EK0 = h.build(C)
    J0, K0 = J0[0].clone(), K0[0].clone()
    J, Ka, Kb, E = h.build_uks(C, C, energies_on_device=True)
    torch.cuda.synchronize()
    h.close()
    assert torch.equal(J, 2 * J0) and torch.equal(Ka, K0) and torch.equal(Kb, K0)
    E = E.cpu().numpy()
    assert E[0] == 4 * EJ0[0] and E[1] == EK0[0] and E[2] == EK0[0]


@pytest.mark.parametrize("precision", [dfjk.DFJK_FP64, dfjk.DFJK_MIXED])
def test_uks_one_electron(precision):
    """nocc_b = 0 and one alpha electron: K_b = 0 and the Coulomb
    self-energy equals the exchange self-energy."""
    m = I.molecule(4, seed=1004)
    S = O.overlap(m.orb, m.coords)
    Ca = torch.from_numpy(I.orthonormalize(I.c_occ_raw(m.nao, 1, 3000), S)).cuda()
    Cb = torch.empty((m.nao, 0), dtype=torch.float64, device="cuda")
    h = dfjk.Handle(m, precision=precision)
    J, Ka, Kb, E = h.build_uks(Ca, Cb)
    h.close()
    assert torch.count_nonzero(Kb).item() == 0 and E[2] == 0.0
    assert abs(E[0] - E[1]) < (1e-12 if precision == dfjk.DFJK_FP64 else 1e-8) * abs(E[0])


def test_uks_rejects_bad_counts():
    m = I.water()
    h = dfjk.Handle(m)
    Ca = torch.zeros((m.nao, 3), dtype=torch.float64, device="cuda")
    Cb = torch.zeros((m.nao, 4), dtype=torch.float64, device="cuda")
    with pytest.raises(dfjk.DfjkError) as e:
        h.build_uks(Ca, Cb)  # nocc_b > nocc_a
    assert e.value.code == 1
    h.close()
