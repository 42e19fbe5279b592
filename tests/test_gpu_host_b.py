"""B kept in pinned host memory (mapped into the device address space; the
kernels read and write it in place): the same kernels run on the same values,
so J, K and the energies are bitwise those of the device-resident build."""
import pytest

from paper_2404_09452_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2404_09452_gb300 import dfjk  # noqa: E402


@pytest.mark.parametrize("precision", [dfjk.DFJK_FP64, dfjk.DFJK_MIXED])
def test_host_resident_b_is_bitwise_equal(precision):
    m = I.molecule(12, seed=1012)
    hd = dfjk.Handle(m, precision=precision)
    hh = dfjk.Handle(m, precision=precision, b_on_host=True)
    assert hh.device_bytes < hd.device_bytes
    assert hh.lean == (precision == dfjk.DFJK_MIXED)
    C = torch.from_numpy(dfjk.orthonormal_c_occ(hd, I.c_occ_raw(m.nao, I.default_nocc(m.nao), 3000))).cuda()
    Jd, Kd, EJd, EKd = hd.build(C)
    Jh, Kh, EJh, EKh = hh.build(C)
    assert torch.equal(Jd, Jh) and torch.equal(Kd, Kh)
    assert EJd[0] == EJh[0] and EKd[0] == EKh[0]
    assert torch.equal(hd.B(), hh.B())
    hd.close()
    hh.close()
