"""Schwarz-guided FP32 integrals: kept shell pairs whose bound
sqrt(max(ab|ab)) max_P sqrt((P|P)) is below the threshold are evaluated on the
FP32 pipe.  Every integral of such a pair is below the bound; the FP32 error
is at most ~3e-4 of the bound (measured: cancellation between Hermite terms of
tight d-d pairs a few bohr apart), so the whitened J, K and energies move by
about 1e-10 (threshold 1e-6) to 2e-9 (1e-5, the mixed default)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2404_09452_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2404_09452_gb300 import dfjk  # noqa: E402


def _c(m, h):
    return torch.from_numpy(dfjk.orthonormal_c_occ(h, I.c_occ_raw(m.nao, I.default_nocc(m.nao), 3000))).cuda()


@pytest.mark.parametrize("thr", [1e-6, 1e-5])
def test_fp32_pairs_error_is_a_fraction_of_the_threshold(thr):
    m = I.molecule(20, seed=1020)
    h64 = dfjk.Handle(m, precision=dfjk.DFJK_FP64, fp32_pair_thresh=0.0)
    h32 = dfjk.Handle(m, precision=dfjk.DFJK_FP64, fp32_pair_thresh=thr)
    assert h64.npair_fp32 == 0 and 0 < h32.npair_fp32 < h32.npair_kept and h32.fp32_pair_thresh == thr
    T64, T32 = h64.three_center(), h32.three_center()
    dT = (T64 - T32).abs().max().item()
    assert 0 < dT <= 1e-3 * thr, dT
    C = _c(m, h64)
    J64, K64, EJ64, EK64 = h64.build(C)
    J32, K32, EJ32, EK32 = h32.build(C)
    tol = 1e-9 if thr <= 1e-6 else 1e-8
    assert (J64 - J32).abs().max().item() < tol and (K64 - K32).abs().max().item() < tol
    assert abs(EJ64[0] - EJ32[0]) < 10 * tol * max(1.0, abs(EJ64[0]))
    assert abs(EK64[0] - EK32[0]) < 10 * tol * max(1.0, abs(EK64[0]))
    h64.close()
    h32.close()


def test_defaults_per_precision():
    m = I.molecule(12, seed=1012)
    h = dfjk.Handle(m, precision=dfjk.DFJK_FP64)
    assert h.npair_fp32 == 0 and h.fp32_pair_thresh == 0.0
    h.close()
    h = dfjk.Handle(m, precision=dfjk.DFJK_MIXED)
    assert h.fp32_pair_thresh == 1e-5 and h.npair_fp32 > 0
    h.close()


def test_mixed_with_fp32_pairs_vs_oracle():
    m = I.molecule(12, seed=1012)
    S = O.overlap(m.orb, m.coords)
    C = I.orthonormalize(I.c_occ_raw(m.nao, I.default_nocc(m.nao), 3000), S)
    ref = O.dfjk(m.orb, m.aux, m.coords, C)
    h = dfjk.Handle(m, precision=dfjk.DFJK_MIXED)
    J, K, EJ, EK = h.build(torch.from_numpy(C).cuda())
    h.close()
    assert np.max(np.abs(J[0].cpu().numpy() - ref["J"])) < 1e-8
    assert np.max(np.abs(K[0].cpu().numpy() - ref["K"])) < 1e-8
    assert abs(EJ[0] - ref["E_J"]) < 1e-7 and abs(EK[0] - ref["E_K"]) < 1e-7
