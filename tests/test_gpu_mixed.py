"""DFJK_MIXED (whitening, X = B C and K as exact sliced products on the tcgen05
tensor cores; integrals, Cholesky, rho, J and energies FP64) against the FP64
oracle on small systems and against the FP64 GPU path at the full 60-atom
size.  Bar: |dE| <= 1e-6 Eh, max|dJ|, max|dK| <= 1e-7."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2404_09452_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2404_09452_gb300 import dfjk  # noqa: E402

E_TOL, JK_TOL = 1e-6, 1e-7


@pytest.fixture(scope="module", params=["water", "mol4", "mol12", "mol20"])
def case(request):
    name = request.param
    m = I.water() if name == "water" else I.molecule(int(name[3:]), seed=1000 + int(name[3:]))
    nocc = 5 if name == "water" else I.default_nocc(m.nao)
    S = O.overlap(m.orb, m.coords)
    C = I.orthonormalize(I.c_occ_raw(m.nao, nocc, 3000), S)
    ref = O.dfjk(m.orb, m.aux, m.coords, C)
    return name, m, C, ref


def test_mixed_vs_oracle(case):
    name, m, C, ref = case
    h = dfjk.Handle(m, precision=dfjk.DFJK_MIXED)
    J, K, EJ, EK = h.build(torch.from_numpy(C).cuda())
    J, K = J[0].cpu().numpy(), K[0].cpu().numpy()
    dJ, dK = np.abs(J - ref["J"]).max(), np.abs(K - ref["K"]).max()
    dEJ, dEK = abs(EJ[0] - ref["E_J"]), abs(EK[0] - ref["E_K"])
    print(f"{name}: dJ {dJ:.2e} dK {dK:.2e} dEJ {dEJ:.2e} dEK {dEK:.2e}")
    assert dJ <= JK_TOL and dK <= JK_TOL and dEJ <= E_TOL and dEK <= E_TOL
    assert np.array_equal(J, J.T) and np.array_equal(K, K.T)
    # the FP64 B kept by the mixed path comes from the tensor-core whitening
    B = h.B().cpu().numpy()
    assert np.abs(B - ref["B"]).max() < 1e-6 * max(1.0, np.abs(ref["B"]).max())
    h.close()


def test_mixed_repeat_is_bitwise():
    m = I.molecule(4, seed=1004)
    h = dfjk.Handle(m, precision=dfjk.DFJK_MIXED)
    C = torch.from_numpy(dfjk.orthonormal_c_occ(h, I.c_occ_raw(m.nao, 12, 3000))).cuda()
    J0, K0, EJ0, EK0 = h.build(C)
    J0, K0 = J0.clone(), K0.clone()
    J1, K1, EJ1, EK1 = h.build(C)
    assert torch.equal(J0, J1) and torch.equal(K0, K1) and EJ0[0] == EJ1[0] and EK0[0] == EK1[0]
    h.close()


def test_full_size_mixed_vs_fp64_gpu():
    """The 60-atom workload the benchmark times (nao 900, naux 2160, nocc 180):
    the mixed path against the FP64 GPU path (itself oracle-checked above at
    smaller sizes), plus the symmetry and positivity the method guarantees."""
    m = I.molecule(60, seed=1002)
    nocc = I.default_nocc(m.nao)
    h64 = dfjk.Handle(m, precision=dfjk.DFJK_FP64)
    C = torch.from_numpy(dfjk.orthonormal_c_occ(h64, I.c_occ_raw(m.nao, nocc, 3000))).cuda()
    J64, K64, EJ64, EK64 = h64.build(C)
    J64, K64 = J64.clone(), K64.clone()
    h64.close()
    hm = dfjk.Handle(m, precision=dfjk.DFJK_MIXED)
    Jm, Km, EJm, EKm = hm.build(C)
    dJ = (Jm - J64).abs().max().item()
    dK = (Km - K64).abs().max().item()
    dEJ, dEK = abs(EJm[0] - EJ64[0]), abs(EKm[0] - EK64[0])
    print(f"mol60 mixed vs fp64: dJ {dJ:.2e} dK {dK:.2e} dEJ {dEJ:.2e} dEK {dEK:.2e}")
    assert dJ <= JK_TOL and dK <= JK_TOL and dEJ <= E_TOL and dEK <= E_TOL
    assert torch.equal(Jm[0], Jm[0].T) and torch.equal(Km[0], Km[0].T)
    assert torch.linalg.eigvalsh(Km[0]).min().item() > -1e-10
    hm.close()


def test_full_size_sampled_integrals():
    """At the full 60-atom size: 3-centre integrals of randomly sampled shell
    triples recomputed one by one by the oracle."""
    m = I.molecule(60, seed=1002)
    h = dfjk.Handle(m, precision=dfjk.DFJK_MIXED)
    T = h.three_center()
    mask = h.pair_mask().cpu().numpy()
    rng = np.random.default_rng(0)
    no, na = len(m.orb.shells), len(m.aux.shells)
    oo = np.cumsum([0] + [(s.l + 1) * (s.l + 2) // 2 for s in m.orb.shells])
    oa = np.cumsum([0] + [(s.l + 1) * (s.l + 2) // 2 for s in m.aux.shells])
    kept = np.argwhere(mask)
    trip = [(int(a), int(b), int(rng.integers(na))) for a, b in kept[rng.integers(len(kept), size=300)]]
    blocks = O.three_center_triples(m.orb, m.aux, m.coords, trip)
    for (a, b, c), blk in zip(trip, blocks):
        got = T[oa[c]:oa[c + 1], oo[a]:oo[a + 1], oo[b]:oo[b + 1]].permute(1, 2, 0).cpu().numpy()
        assert np.abs(got - blk).max() < 1e-11, (a, b, c)
    h.close()


def test_expired_device_wait_is_reported_and_context_survives():
    """Failure detection without a GPU fault: the tensor-core kernels poll
    their mbarriers a bounded number of times.  With a limit of 1 poll the
    waits run out, the kernel records DFJK_ERR_TIMEOUT, lets its copies and
    MMAs land, frees TMEM and returns; the context stays usable."""
    m = I.molecule(4, seed=1004)
    with pytest.raises(dfjk.DfjkError) as e:
        dfjk.Handle(m, precision=dfjk.DFJK_MIXED, timeout_iters=1)
    assert e.value.code == 6  # DFJK_ERR_TIMEOUT
    h = dfjk.Handle(m, precision=dfjk.DFJK_MIXED)
    C = torch.from_numpy(dfjk.orthonormal_c_occ(h, I.c_occ_raw(m.nao, 12, 3000))).cuda()
    J, K, EJ, EK = h.build(C)
    assert np.isfinite(EJ[0]) and np.isfinite(EK[0])
    h.close()


def test_chunked_build_matches_one_chunk_and_oracle(tmp_path):
    """The mixed build works through the aux index in chunks of rows P when its
    work buffers would exceed DFJK_BUILD_WS_MB (here forced to the 128-row
    minimum: four chunks at 12 atoms, the last one short).  K accumulates the
    chunks in order, so the result differs from the one-chunk build only by
    the rounding of the sliced products: both meet the bar against the
    oracle and agree to 1e-9."""
    import os
    import subprocess
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    code = (
        "import sys, numpy as np, torch; sys.path.insert(0, %r);"
        "from paper_2404_09452_gb300 import dfjk, inputs as I;"
        "m = I.molecule(12, seed=1012); C = np.load(sys.argv[2]);"
        "h = dfjk.Handle(m, precision=dfjk.DFJK_MIXED);"
        "J, K, EJ, EK = h.build(torch.from_numpy(C).cuda()); np.save(sys.argv[1], np.concatenate(["
        "J[0].cpu().numpy().ravel(), K[0].cpu().numpy().ravel(), [EJ[0], EK[0]]]))"
    ) % root
    m = I.molecule(12, seed=1012)
    S = O.overlap(m.orb, m.coords)
    C = I.orthonormalize(I.c_occ_raw(m.nao, I.default_nocc(m.nao), 3000), S)
    cpath = str(tmp_path / "C.npy")
    np.save(cpath, C)
    outs = []
    for ws in ("1", "8192"):
        out = str(tmp_path / f"r{ws}.npy")
        env = dict(os.environ, DFJK_BUILD_WS_MB=ws)
        subprocess.run([sys.executable, "-c", code, out, cpath], check=True, env=env, timeout=300)
        outs.append(np.load(out))
    n2 = m.nao * m.nao
    ref = O.dfjk(m.orb, m.aux, m.coords, C)
    for r in outs:
        J, K = r[:n2].reshape(m.nao, m.nao), r[n2:2 * n2].reshape(m.nao, m.nao)
        assert np.abs(J - ref["J"]).max() <= JK_TOL and np.abs(K - ref["K"]).max() <= JK_TOL
        assert abs(r[-2] - ref["E_J"]) <= E_TOL and abs(r[-1] - ref["E_K"]) <= E_TOL
        assert np.array_equal(K, K.T)
    assert np.abs(outs[0] - outs[1]).max() < 1e-9
    assert not np.array_equal(outs[0][n2:2 * n2], outs[1][n2:2 * n2])  # the chunked path did run


def test_config_120_atoms_mixed_vs_fp64_gpu():
    """The 120-atom mixed configuration (nao 1800, naux 4320, nocc 360; B kept
    for the kept pairs only, sliced per build in chunks of aux rows) against the
    FP64 GPU path at the same size."""
    m = I.molecule(120, seed=1003)
    nocc = I.default_nocc(m.nao)
    h64 = dfjk.Handle(m, precision=dfjk.DFJK_FP64)
    C = torch.from_numpy(dfjk.orthonormal_c_occ(h64, I.c_occ_raw(m.nao, nocc, 3000))).cuda()
    J64, K64, EJ64, EK64 = h64.build(C)
    J64, K64 = J64.clone(), K64.clone()
    h64.close()
    hm = dfjk.Handle(m, precision=dfjk.DFJK_MIXED)
    Jm, Km, EJm, EKm = hm.build(C)
    dJ, dK = (Jm - J64).abs().max().item(), (Km - K64).abs().max().item()
    dEJ, dEK = abs(EJm[0] - EJ64[0]), abs(EKm[0] - EK64[0])
    print(f"mol120 mixed vs fp64: dJ {dJ:.2e} dK {dK:.2e} dEJ {dEJ:.2e} dEK {dEK:.2e}")
    assert dJ <= JK_TOL and dK <= JK_TOL and dEJ <= E_TOL and dEK <= E_TOL
    hm.close()


def test_ordered_split_k_matches_partial_reduction(tmp_path):
    """The persistent kernel adds the K splits of a tile into K in split order;
    the one-tile-per-CTA kernel (DFJK_OZ_SIMPLE=1) writes one partial per split
    and reduces them in the same order: identical K."""
    import os
    import subprocess
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    code = (
        "import sys, numpy as np, torch; sys.path.insert(0, %r);"
        "from paper_2404_09452_gb300 import dfjk, inputs as I;"
        "m = I.molecule(12, seed=1012); h = dfjk.Handle(m, precision=dfjk.DFJK_MIXED);"
        "C = torch.from_numpy(dfjk.orthonormal_c_occ(h, I.c_occ_raw(m.nao, 36, 3000))).cuda();"
        "J, K, EJ, EK = h.build(C); np.save(sys.argv[1], K[0].cpu().numpy())"
    ) % root
    outs = []
    for simple in ("0", "1"):
        out = str(tmp_path / f"k{simple}.npy")
        env = dict(os.environ, DFJK_OZ_SIMPLE=simple, DFJK_K_RANGE_MB="1")
        subprocess.run([sys.executable, "-c", code, out], check=True, env=env, timeout=300)
        outs.append(np.load(out))
    assert np.array_equal(outs[0], outs[1])
    assert np.array_equal(outs[0], outs[0].T)


def test_config_120_atoms_sampled_B_columns_vs_oracle():
    """At the full 120-atom size (nao 1800, naux 4320): whitened columns
    B[:, mu, nu] of 40 sampled kept shell pairs against the oracle, which
    evaluates (P|mu nu) for those pairs against every aux shell, the metric
    (P|Q) in full, its Cholesky factor and the triangular solve.  This covers
    the integrals and the tensor-core whitening at a size where the oracle's
    full build does not fit a test."""
    import scipy.linalg

    m = I.molecule(120, seed=1003)
    h = dfjk.Handle(m, precision=dfjk.DFJK_MIXED)
    mask = h.pair_mask().cpu().numpy()
    rng = np.random.default_rng(1)
    kept = np.argwhere(np.tril(mask))
    pairs = kept[rng.choice(len(kept), size=40, replace=False)]
    oo = np.cumsum([0] + [(s.l + 1) * (s.l + 2) // 2 for s in m.orb.shells])
    oa = np.cumsum([0] + [(s.l + 1) * (s.l + 2) // 2 for s in m.aux.shells])
    na = len(m.aux.shells)
    trip = [(int(a), int(b), c) for a, b in pairs for c in range(na)]
    blocks = O.three_center_triples(m.orb, m.aux, m.coords, trip)
    V = O.metric(m.aux, m.coords)
    L = scipy.linalg.cholesky(V, lower=True)
    cols_mu, cols_nu, T = [], [], []
    k = 0
    for a, b in pairs:
        blk = blocks[k:k + na]
        k += na
        for ca in range(oo[a + 1] - oo[a]):
            for cb in range(oo[b + 1] - oo[b]):
                cols_mu.append(oo[a] + ca)
                cols_nu.append(oo[b] + cb)
                T.append(np.concatenate([blk[c][ca, cb, :] for c in range(na)]))
    Bref = scipy.linalg.solve_triangular(L, np.array(T).T, lower=True).T
    Bgpu = h.B_columns(cols_mu, cols_nu).cpu().numpy()
    err = np.abs(Bgpu - Bref).max()
    print(f"mol120 sampled B columns: {len(cols_mu)} columns, max|dB| {err:.2e}, max|B| {np.abs(Bref).max():.2e}")
    assert err < 1e-6 * max(1.0, np.abs(Bref).max())
    h.close()


def test_B_holds_the_kept_pairs_only():
    """The mixed handle stores B for the Schwarz-kept AO pairs only (rows found
    through a row map): a screened pair reads back as exact zeros through both
    accessors, a kept one as the FP64 handle's column, and the handle holds
    fewer bytes than the FP64 handle with both triangles of every pair."""
    m = I.molecule(12, seed=1012)
    thr = 1e-5  # screens a good share of the pairs of this molecule
    hm = dfjk.Handle(m, precision=dfjk.DFJK_MIXED, schwarz_thresh=thr)
    hf = dfjk.Handle(m, precision=dfjk.DFJK_FP64, schwarz_thresh=thr)
    ncart = [(s.l + 1) * (s.l + 2) // 2 for s in m.orb.shells]
    off = np.concatenate([[0], np.cumsum(ncart)])
    mask = hm.pair_mask().cpu().numpy()
    kept, screened = [], []
    for a in range(len(ncart)):
        for b in range(a + 1):
            (kept if mask[a, b] else screened).append((off[a], off[b] + ncart[b] - 1))
    assert screened and kept
    mu = np.array([p[0] for p in kept + screened], dtype=np.int32)
    nu = np.array([p[1] for p in kept + screened], dtype=np.int32)
    Bm = hm.B_columns(mu, nu).cpu().numpy()
    Bf = hf.B_columns(mu, nu).cpu().numpy()
    nk = len(kept)
    assert not Bm[nk:].any() and not Bf[nk:].any()
    assert np.abs(Bm[:nk] - Bf[:nk]).max() <= 1e-8 * max(1.0, np.abs(Bf).max())
    Bfull_m, Bfull_f = hm.B().cpu().numpy(), hf.B().cpu().numpy()
    assert np.abs(Bfull_m - Bfull_f).max() <= 1e-8 * max(1.0, np.abs(Bfull_f).max())
    for (a, b) in screened[:20]:
        assert not Bfull_m[:, a, b].any() and not Bfull_m[:, b, a].any()
    assert hm.device_bytes < hf.device_bytes
    hm.close()
    hf.close()
