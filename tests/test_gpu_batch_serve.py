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


def test_build_batch_captured_in_a_cuda_graph():
    """Once every handle has been built at its nocc (work buffers exist), a
    dfjk_build_batch call records into a CUDA graph: the replay gives the
    direct call's results bitwise, and replaying after new orbitals are
    copied into the same input buffers (an SCF iteration) gives the direct
    build of those orbitals."""
    mols = _mols([3, 6, 2, 5], seed0=7200)
    hs = [dfjk.Handle(m, precision=dfjk.DFJK_MIXED) for m in mols]
    C0 = [_c(m, i) for i, m in enumerate(mols)]
    C1 = [_c(m, 10 + i) for i, m in enumerate(mols)]
    Cs = [c.clone() for c in C0]
    Js = [torch.empty((h.nao, h.nao), dtype=torch.float64, device="cuda") for h in hs]
    Ks = [torch.empty_like(j) for j in Js]
    E = torch.empty((2, len(hs)), dtype=torch.float64, device="cuda")
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        dfjk.build_batch(hs, Cs, Js=Js, Ks=Ks, E=E, nstreams=3, stream=s)  # buffers exist from here
    s.synchronize()
    ref0 = [(j.clone(), k.clone()) for j, k in zip(Js, Ks)], E.clone()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        dfjk.build_batch(hs, Cs, Js=Js, Ks=Ks, E=E, nstreams=3, stream=s)
    for j, k in zip(Js, Ks):
        j.zero_()
        k.zero_()
    g.replay()
    torch.cuda.synchronize()
    for (j0, k0), j, k in zip(ref0[0], Js, Ks):
        assert torch.equal(j0, j) and torch.equal(k0, k)
    assert torch.equal(ref0[1], E)
    for c, c1 in zip(Cs, C1):
        c.copy_(c1)
    g.replay()
    torch.cuda.synchronize()
    for h, c1, j, k, i in zip(hs, C1, Js, Ks, range(len(hs))):
        J, K, EJ, EK = h.build(c1)
        assert torch.equal(J[0], j) and torch.equal(K[0], k)
        assert E[0, i].item() == EJ[0] and E[1, i].item() == EK[0]
    for h in hs:
        h.close()


def test_batch_with_a_60_atom_molecule_matches_the_oracle():
    """A multi-wave batch whose largest member is the 60-atom workload
    molecule (mixed path: B of the kept pairs, built in four aux-row chunks): that
    member's J, K and energies against the FP64 CPU oracle at full size, and
    a small member against the oracle too."""
    from oracle import oracle as O

    big = I.molecule(60, seed=1002)
    mols = [I.molecule(5, seed=7300), big, I.molecule(9, seed=7301)]
    Cs, Cnp = [], []
    for i, m in enumerate(mols):
        C = I.orthonormalize(I.c_occ_raw(m.nao, I.default_nocc(m.nao), 3100 + i), O.overlap(m.orb, m.coords))
        Cnp.append(C)
        Cs.append(torch.from_numpy(C).cuda())
    prec = dfjk.DFJK_MIXED
    # the 60-atom molecule fits alone, not with the first small one: three waves
    small = batch.resident_bytes(mols[0].nao, mols[0].naux, Cs[0].shape[1], prec)
    budget = batch.resident_bytes(big.nao, big.naux, Cs[1].shape[1], prec) + small // 2
    E, res, st = batch.run_batch(mols, Cs, precision=prec, budget_bytes=budget, workers=2, nstreams=2,
                                 keep_results=True)
    assert st["waves"] > 1
    for i in (1, 2):
        ref = O.dfjk(mols[i].orb, mols[i].aux, mols[i].coords, Cnp[i])
        J, K = res[i][0].cpu().numpy(), res[i][1].cpu().numpy()
        dJ, dK = np.abs(J - ref["J"]).max(), np.abs(K - ref["K"]).max()
        print(f"batch member {mols[i].natom} atoms vs oracle: dJ {dJ:.2e} dK {dK:.2e} "
              f"dEJ {abs(E[i, 0] - ref['E_J']):.2e} dEK {abs(E[i, 1] - ref['E_K']):.2e}")
        assert dJ <= 1e-7 and dK <= 1e-7
        assert abs(E[i, 0] - ref["E_J"]) <= 1e-6 and abs(E[i, 1] - ref["E_K"]) <= 1e-6
        del ref
