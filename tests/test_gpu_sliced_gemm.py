"""The exact sliced-product tensor-core GEMM (tcgen05, BF16 slices of 6 bits,
exact FP32 accumulation per 1024-wide K block, FP64 recombination) against
FP64 matmul.  Error bound per element: dropped slice products and the
representation residual, at most (S+2) 2^-6S max|A_m| max|B_n| K."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2404_09452_gb300 import dfjk  # noqa: E402


def _case(batch, M, N, K, seed, spread=3.0):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((batch, M, K)) * 10.0 ** rng.uniform(-spread, spread, (batch, M, 1))
    B = rng.standard_normal((N, K)) * 10.0 ** rng.uniform(-spread, spread, (N, 1))
    A[:, M // 3, :] = 0.0  # an all-zero row
    return A, B


def _check(A, B, S):
    C = dfjk.sliced_gemm(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), S=S).cpu().numpy()
    ref = A @ B.T
    K = A.shape[-1]
    bound = (S + 2) * 2.0 ** (-6 * S) * np.abs(A).max(-1)[..., None] * np.abs(B).max(-1)[None, None, :] * K
    err = np.abs(C - ref)
    assert np.all(err <= bound), (err / bound).max()
    return float((err / np.maximum(bound, 1e-300)).max())


@pytest.mark.parametrize("S", [6, 8])
def test_single_tile(S):
    A, B = _case(1, 128, 64, 64, 1)
    _check(A, B, S)


@pytest.mark.parametrize("S", [6, 8])
def test_ragged_batched_multi_kblock(S):
    A, B = _case(3, 300, 100, 2500, 2)  # 3 K-blocks, ragged M, N, K
    _check(A, B, S)


@pytest.mark.parametrize("S", [6, 8])
def test_long_k_blocked_layout(S):
    """More than 4 exponent blocks along K: the slices are stored K-blocked
    (1024-wide blocks, rows inside) and loaded through 4-D tensor maps."""
    A, B = _case(2, 200, 70, 5300, 5)  # 6 K-blocks, last one partial
    _check(A, B, S)


def test_exact_for_small_integers():
    """Integer-valued operands that fit in the slices are multiplied exactly."""
    rng = np.random.default_rng(3)
    A = rng.integers(-30, 31, (1, 130, 1024)).astype(float)
    B = rng.integers(-30, 31, (70, 1024)).astype(float)
    C = dfjk.sliced_gemm(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), S=6).cpu().numpy()
    assert np.array_equal(C, A @ B.T)


def test_persistent_and_simple_kernels_agree(tmp_path):
    """The persistent warp-specialised kernel (default) and the one-tile-per-CTA
    kernel (DFJK_OZ_SIMPLE=1, read once per process) give identical results."""
    import os
    import subprocess
    import sys

    A, B = _case(2, 200, 130, 2100, 4)
    np.save(tmp_path / "A.npy", A)
    np.save(tmp_path / "B.npy", B)
    code = (
        "import sys, numpy as np, torch; sys.path.insert(0, %r);"
        "from paper_2404_09452_gb300 import dfjk;"
        "A = torch.from_numpy(np.load(%r)).cuda(); B = torch.from_numpy(np.load(%r)).cuda();"
        "np.save(%r, dfjk.sliced_gemm(A, B, S=int(sys.argv[1])).cpu().numpy())"
    )
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    for S in (6, 8):
        outs = []
        for simple in ("0", "1"):
            out = str(tmp_path / f"C{S}{simple}.npy")
            env = dict(os.environ, DFJK_OZ_SIMPLE=simple)
            subprocess.run([sys.executable, "-c", code % (root, str(tmp_path / "A.npy"), str(tmp_path / "B.npy"), out),
                            str(S)], check=True, env=env, timeout=300)
            outs.append(np.load(out))
        assert np.array_equal(outs[0], outs[1])
