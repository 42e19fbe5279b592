"""Batching (many molecules of uneven size, waves under a memory budget, one
multi-stream build call per wave) and serving (continuous admission, LRU
residency with evict-and-recompute, overlapping builds): every result must be
the same alone and in the mix.  The kernels use a fixed reduction order per
molecule, so "the same" is bitwise here."""
import numpy as np
import pytest

from paper_2404_09452_gb300 import inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2404_09452_gb300 import batch, dfjk, serve  # noqa: E402


def _mols(counts, seed0=7000):
    return [I.molecule(int(n), seed=seed0 + i) for i, n in enumerate(counts)]


def _alone(m, C, precision):
    h = dfjk.Handle(m, precision=precision)
    J, K, EJ, EK = h.build(C)
    out = (J[0].clone(), K[0].clone(), float(EJ[0]), float(EK[0]))
    h.close()
    return out


def _c(m, k, seed=3000):
    h = dfjk.Handle(m)
    C = torch.from_numpy(dfjk.orthonormal_c_occ(h, I.c_occ_raw(m.nao, I.default_nocc(m.nao), seed + k))).cuda()
    h.close()
    return C


@pytest.mark.parametrize("precision", [dfjk.DFJK_FP64, dfjk.DFJK_MIXED])
def test_batch_equals_alone(precision):
    mols = _mols([2, 7, 3, 5, 1, 4])
    Cs = [_c(m, i) for i, m in enumerate(mols)]
    # a budget that forces several waves
    budget = int(1.2 * max(batch.resident_bytes(m.nao, m.naux, C.shape[1], precision) for m, C in zip(mols, Cs)))
    E, res, st = batch.run_batch(mols, Cs, precision=precision, budget_bytes=budget, workers=3,
                                 nstreams=4, keep_results=True)
    assert st["waves"] > 1
    for i, (m, C) in enumerate(zip(mols, Cs)):
        J, K, EJ, EK = _alone(m, C, precision)
        assert E[i, 0] == EJ and E[i, 1] == EK
        assert torch.equal(res[i][0], J) and torch.equal(res[i][1], K)


def test_build_batch_matches_sequential_builds():
    mols = _mols([3, 6, 2])
    hs = [dfjk.Handle(m, precision=dfjk.DFJK_MIXED) for m in mols]
    Cs = [_c(m, i) for i, m in enumerate(mols)]
    seq = []
    for h, C in zip(hs, Cs):
        J, K, EJ, EK = h.build(C)
        seq.append((J[0].clone(), K[0].clone(), EJ[0], EK[0]))
    Js, Ks, E = dfjk.build_batch(hs, Cs, nstreams=3)
    torch.cuda.synchronize()
    for k in range(3):
        assert torch.equal(Js[k], seq[k][0]) and torch.equal(Ks[k], seq[k][1])
        assert E[0, k].item() == seq[k][2] and E[1, k].item() == seq[k][3]
    for h in hs:
        h.close()


def test_serving_same_alone_and_in_mix():
    mols = _mols([3, 5, 2, 6, 4], seed0=7100)
    prec = dfjk.DFJK_MIXED
    cache = {}

    def c_of(mid, k):
        key = (mid, k % 3)
        if key not in cache:
            cache[key] = _c(mols[mid], 100 * mid + key[1])
        return cache[key]

    reqs = serve.make_stream(mols, 40, rate=2000.0, repeat=0.7, seed=5001, c_of=c_of)
    # budget for about two molecules at a time: forces evictions and recompute
    budget = int(1.5 * max(batch.resident_bytes(m.nao, m.naux, I.default_nocc(m.nao), prec) for m in mols))
    srv = serve.Server(mols, precision=prec, budget_bytes=budget, slots=4, keep_outputs=True)
    srv.run(reqs)
    srv.close()
    s = srv.stats.summary()
    assert s["requests"] == 40 and s["p99_ms"] >= s["p50_ms"] > 0
    assert srv.stats.evictions > 0 and srv.stats.misses > len(set(r.mol_id for r in reqs)) - 1
    alone = {}
    for r in reqs:
        key = (r.mol_id, id(r.C))
        if key not in alone:
            alone[key] = _alone(mols[r.mol_id], r.C, prec)
        J, K, EJ, EK = alone[key]
        assert r.E == (EJ, EK)
        assert torch.equal(r.J, J) and torch.equal(r.K, K)
