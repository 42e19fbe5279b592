"""dfjk_build_density: J and K from a symmetric density (FP64 pipe) against
the oracle, for D = C C^T (also against dfjk_build) and for a density that is
not positive semidefinite."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2404_09452_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2404_09452_gb300 import dfjk  # noqa: E402

FP64_TOL = 1e-9


@pytest.mark.parametrize("precision", [dfjk.DFJK_FP64, dfjk.DFJK_MIXED])
def test_density_build_vs_oracle(precision):
    m = I.molecule(12, seed=1012)
    S = O.overlap(m.orb, m.coords)
    C = I.orthonormalize(I.c_occ_raw(m.nao, I.default_nocc(m.nao), 3000), S)
    ref = O.dfjk(m.orb, m.aux, m.coords, C)
    n = C.shape[1]
    C1, C2 = C[:, : n // 2], C[:, n // 2 :]
    Dm = C1 @ C1.T - 0.5 * C2 @ C2.T  # not positive semidefinite
    refm = O.jk_from_density(ref["B"], Dm)
    h = dfjk.Handle(m, precision=precision)
    D = torch.from_numpy(np.stack([C @ C.T, Dm])).cuda()
    J, K, EJ, EK = h.build_density(D)
    Jc, Kc, EJc, EKc = h.build(torch.from_numpy(C).cuda())
    h.close()
    J, K = J.cpu().numpy(), K.cpu().numpy()
    # the density route is FP64 whatever the handle's precision; B is FP64 in
    # both, with the mixed handle's small-pair integrals in FP32 (about 1e-9)
    t = FP64_TOL if precision == dfjk.DFJK_FP64 else 1e-8
    assert np.max(np.abs(J[0] - ref["J"])) < t and np.max(np.abs(K[0] - ref["K"])) < t
    assert np.max(np.abs(J[1] - refm["J"])) < t and np.max(np.abs(K[1] - refm["K"])) < t
    assert abs(EJ[1] - refm["E_J"]) < 10 * t and abs(EK[1] - refm["E_K"]) < 10 * t
    assert np.array_equal(K[0], K[0].T) and np.array_equal(J[1], J[1].T)
    # and agrees with the orbital build of the same handle
    tol = FP64_TOL if precision == dfjk.DFJK_FP64 else 1e-7
    assert np.max(np.abs(K[0] - Kc[0].cpu().numpy())) < tol
    assert abs(EK[0] - EKc[0]) < 10 * tol
