"""Host logic of the continuous-batching server with asynchronous admission,
on CPU: fake streams, events and handles stand in for the GPU (a setup sleeps
on the worker thread; a build completes after a fixed time).  Checks that
every request is served (no stall, no livelock), that hits are admitted while
a miss sets up, that a molecule is never built while its setup runs or two
builds of it overlap, and that the residency accounting ends balanced."""
import collections
import contextlib
import threading
import time
import types

import numpy as np

from paper_2404_09452_gb300 import serve


class _Stream:
    dur = 0.0

    def synchronize(self):
        pass


class _Event:
    def __init__(self, log):
        self.log = log
        self.t_done = None

    def record(self, s):
        self.t_done = time.perf_counter() + s.dur

    def query(self):
        return time.perf_counter() >= self.t_done


def _fake_torch(log):
    cuda = types.SimpleNamespace(
        Stream=_Stream,
        stream=lambda s: contextlib.nullcontext(),
        Event=lambda: _Event(log),
        current_device=lambda: 0,
        set_device=lambda d: None,
    )
    return types.SimpleNamespace(cuda=cuda)


class _Mol:
    def __init__(self, natom):
        self.natom = natom
        self.nao = 15 * natom
        self.naux = 36 * natom


class _Scalar(float):
    def item(self):
        return float(self)


def _make_handle_cls(log, lock):
    class Handle:
        def __init__(self, mol, precision=None, stream=None):
            with lock:
                log["setups"] += 1
                log["setting_up"].add(id(mol))
            time.sleep(2e-4 * mol.natom)  # setup time grows with size
            with lock:
                log["setting_up"].discard(id(mol))
            self.mol = mol
            self.building = False

        def build(self, C, stream=None, energies_on_device=True):
            mid = id(self.mol)
            with lock:
                assert mid not in log["setting_up"], "built during its own setup"
                log["builds"] += 1
            stream.dur = 1e-5 * self.mol.natom
            e = [_Scalar(self.mol.natom), _Scalar(0.5 * self.mol.natom)]
            return None, None, e, e[1:]

        def close(self):
            pass

    return Handle


def test_async_server_serves_every_request():
    log = {"setups": 0, "builds": 0, "setting_up": set()}
    lock = threading.Lock()
    rng = np.random.default_rng(3)
    mols = [_Mol(int(n)) for n in np.round(np.exp(rng.uniform(np.log(5), np.log(150), size=60)))]
    C = types.SimpleNamespace(shape=(0, 8))
    reqs = serve.make_stream(mols, 400, rate=4000.0, repeat=0.7, seed=11, c_of=lambda mid, k: C)
    budget = 3 * 150 ** 2  # room for a few molecules at a time: evictions and recompute
    srv = serve.Server(mols, budget_bytes=budget, slots=4, setup_workers=2,
                       backend=(_fake_torch(log), _make_handle_cls(log, lock), lambda nao, naux, nocc, p: nao * nao // 15))
    done = {}

    def run():
        srv.run(reqs)
        done["ok"] = True

    th = threading.Thread(target=run, daemon=True)
    th.start()
    th.join(timeout=120)
    assert done.get("ok"), "the server did not finish"
    st = srv.stats.summary()
    srv.close()
    assert st["requests"] == 400 and st["failed"] == 0
    assert all(r.done >= r.arrival for r in reqs)
    assert all(r.E == (float(mols[r.mol_id].natom), 0.5 * mols[r.mol_id].natom) for r in reqs)
    assert log["builds"] == 400 and log["setups"] == st["misses"] > len(set(r.mol_id for r in reqs))
    assert st["evictions"] > 0
    assert srv.lru.used == 0 and not srv.busy


def test_hits_are_admitted_while_a_miss_sets_up():
    """A slow setup of a large new molecule does not hold up builds of a
    resident one: those finish while the setup is still running."""
    log = {"setups": 0, "builds": 0, "setting_up": set()}
    lock = threading.Lock()
    mols = [_Mol(5), _Mol(3000)]  # the second takes 0.6 s to set up
    C = types.SimpleNamespace(shape=(0, 8))
    reqs = [serve.Request(0, 0.0, 0, C), serve.Request(1, 0.01, 1, C)] + [
        serve.Request(2 + i, 0.02 + 0.01 * i, 0, C) for i in range(20)]
    srv = serve.Server(mols, budget_bytes=1 << 40, slots=2, setup_workers=1,
                       backend=(_fake_torch(log), _make_handle_cls(log, lock), lambda *a: 1))
    srv.run(reqs)
    srv.close()
    big = reqs[1]
    hits_done = [r.done for r in reqs if r.mol_id == 0 and r.rid >= 2]
    assert max(hits_done) < big.done  # every hit finished before the miss


def test_setup_recharges_the_actual_bytes():
    """A miss reserves the bound from the molecule's sizes; after the setup the
    molecule is charged its actual bytes, so that two molecules whose bounds
    do not fit the budget together (60 + 60 > 100) stay resident together
    (30 + 60, then 30 + 30)."""
    C = types.SimpleNamespace(shape=(0, 8))
    mols = [_Mol(5), _Mol(6)]
    # alternating requests of two molecules
    reqs = [serve.Request(i, 0.001 * i, i % 2, C) for i in range(40)]

    def run(actual):
        log = {"setups": 0, "builds": 0, "setting_up": set()}
        lock = threading.Lock()
        backend = (_fake_torch(log), _make_handle_cls(log, lock), lambda *a: 60)
        if actual is not None:
            backend = backend + (actual,)
        srv = serve.Server(mols, budget_bytes=100, slots=2, setup_workers=1, backend=backend)
        srv.run([serve.Request(r.rid, r.arrival, r.mol_id, C) for r in reqs])
        st = srv.stats.summary()
        used = srv.lru.used
        srv.close()
        assert st["requests"] == 40 and st["failed"] == 0
        return st["misses"], used

    misses, used = run(lambda h, mol, nocc, p: 30)
    assert misses == 2 and used == 60  # both resident, charged 30 each
    misses_bound, _ = run(None)
    assert misses_bound > 2  # charged the bound, they evict each other


def test_a_larger_nocc_raises_the_charge():
    """A later request with more occupied orbitals (a larger build work
    buffer) raises its molecule's charge."""
    log = {"setups": 0, "builds": 0, "setting_up": set()}
    lock = threading.Lock()
    mols = [_Mol(5)]
    small, large = types.SimpleNamespace(shape=(0, 8)), types.SimpleNamespace(shape=(0, 16))
    reqs = [serve.Request(0, 0.0, 0, small), serve.Request(1, 0.01, 0, large)]
    charged = []

    def actual(h, mol, nocc, p):
        charged.append(nocc)
        return 10 * nocc

    srv = serve.Server(mols, budget_bytes=10 ** 6, slots=1, setup_workers=1,
                       backend=(_fake_torch(log), _make_handle_cls(log, lock), lambda *a: 1000, actual))
    srv.run(reqs)
    used = srv.lru.used
    srv.close()
    assert charged == [8, 16] and used == 160 and log["setups"] == 1
