"""The allocation-free energy entry point (dfjk_energies_noalloc) against the
energies that dfjk_build returns, through the C ABI, on two calls in a row.

It serves callers that must not call cudaMalloc (a process whose memory pool
already owns the device memory, or a latency path that cannot take the
device-wide synchronisation of an allocation); its scratch is a static device
array inside the library.  This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2404_09452_gb300 import dfjk, inputs as I  # noqa: E402

E_TOL = 1e-6  # |dE| bar used by the parity tests (hartree)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def _check_against_build(m, nocc):
    h = dfjk.Handle(m)
    C = torch.from_numpy(dfjk.orthonormal_c_occ(h, I.c_occ_raw(m.nao, nocc, 3000))).cuda()
    J, K, EJ, EK = h.build(C)
    D = C @ C.T
    E = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = dfjk.load_library().dfjk_energies_noalloc(m.nao, _ptr(D), _ptr(J[0]), _ptr(K[0]), _ptr(E), stream)
    assert rc == 0, dfjk.load_library().dfjk_last_error()
    torch.cuda.synchronize()
    e = E.cpu().numpy()
    assert abs(e[0] - EJ[0]) <= E_TOL and abs(e[1] - EK[0]) <= E_TOL
    assert e[0] == pytest.approx(EJ[0], rel=1e-12) and e[1] == pytest.approx(EK[0], rel=1e-12)
    h.close()


def test_noalloc_energies_match_build_on_two_calls():
    _check_against_build(I.molecule(4, seed=1004), 12)  # n = 60
    _check_against_build(I.water(), 5)  # n = 18: fewer blocks, stale slots must not leak in


def test_noalloc_rejects_sizes_beyond_the_scratch():
    x = torch.zeros(4, dtype=torch.float64, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    lib = dfjk.load_library()
    assert lib.dfjk_energies_noalloc(8193, _ptr(x), _ptr(x), _ptr(x), _ptr(x), stream) == 1
    assert b"8192" in lib.dfjk_last_error()
