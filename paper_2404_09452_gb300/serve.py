"""Continuous-batching DF-J/K server (SCF-iteration pattern).

Requests (molecule, C_occ) arrive as a stream.  The server keeps each
molecule's whitened tensor B resident under a device-memory budget (LRU order;
a miss evicts the least recently used idle molecules and recomputes B with
`dfjk_setup` on a worker thread, while other requests keep being admitted).
Requests that arrive while others are on the GPU are admitted as soon as a
build slot and their molecule are free: each build runs on one of `slots`
CUDA streams, so builds of different molecules overlap on the device.
Builds of the same molecule are serialised (its work buffers are shared).
Latency is measured from arrival to the host observing completion of the
build's event.  The paper's SCF loop (Sec. "Improved Compatibility with
PySCF", the `kernel()` call) repeats J/K builds for one molecule with new
orbitals; the ~70 % repeat rate of the request stream models that.
"""

from __future__ import annotations

import collections
import time
from dataclasses import dataclass, field

import numpy as np

from . import dfjk
from .batch import resident_bytes


def setup_bytes(h, mol, nocc: int, precision: int) -> int:
    """Device bytes a set-up molecule holds from now on: its handle's resident
    data (dfjk_query) plus the work buffers of a build at nocc."""
    return int(h.device_bytes + dfjk.estimate_bytes(mol.nao, mol.naux, nocc, precision)["build_ws"])


@dataclass
class Request:
    rid: int
    arrival: float  # seconds from the start of the run
    mol_id: int
    C: object  # device tensor [nao, nocc]
    done: float = -1.0
    error: str = ""  # set when the request could not be served (its setup failed)
    E: tuple = ()
    J: object = None
    K: object = None


class Residency:
    """LRU residency under a byte budget.  Each resident molecule is charged
    the bytes it was admitted with, and exactly that is returned when it is
    evicted."""

    def __init__(self, budget: int):
        self.budget = budget
        self.bytes = collections.OrderedDict()  # mol_id -> bytes (LRU order)
        self.used = 0

    def touch(self, mol_id) -> bool:
        if mol_id in self.bytes:
            self.bytes.move_to_end(mol_id)
            return True
        return False

    def admit(self, mol_id, need: int, busy) -> tuple:
        """Makes room for `need` bytes by evicting least recently used molecules
        that are not in `busy`.  Returns (admitted, evicted ids).  A molecule
        larger than the whole budget is admitted alone once nothing else is
        resident (it cannot be served otherwise)."""
        evicted = []
        while self.used + need > self.budget and self.bytes:
            victim = next((k for k in self.bytes if k not in busy), None)
            if victim is None:
                return False, evicted  # everything resident is in flight: wait
            self.used -= self.bytes.pop(victim)
            evicted.append(victim)
        self.bytes[mol_id] = need
        self.used += need
        return True, evicted

    def drop(self, mol_id):
        if mol_id in self.bytes:
            self.used -= self.bytes.pop(mol_id)

    def resize(self, mol_id, need: int):
        """Charges a resident molecule `need` bytes instead of its current charge
        (after its setup, when its actual size is known)."""
        if mol_id in self.bytes:
            self.used += need - self.bytes[mol_id]
            self.bytes[mol_id] = need


@dataclass
class Stats:
    latencies: list = field(default_factory=list)
    misses: int = 0
    evictions: int = 0
    failed: int = 0
    seconds: float = 0.0

    def summary(self):
        lat = np.array(self.latencies) * 1e3
        return {
            "requests": len(lat),
            "p50_ms": float(np.percentile(lat, 50)) if len(lat) else None,
            "p99_ms": float(np.percentile(lat, 99)) if len(lat) else None,
            "builds_per_s": len(lat) / self.seconds if self.seconds else None,
            "misses": self.misses,
            "evictions": self.evictions,
            "failed": self.failed,
        }


class Server:
    """Continuous batching with asynchronous admission: a request whose
    molecule is resident and idle starts its build on a free slot at once; a
    miss reserves the molecule's bytes (evicting idle molecules in LRU order)
    and runs its setup on a worker thread with a stream of its own, so that
    hits keep being admitted and completions keep being retired while the
    setup runs.  The reservation is the library's bound from the molecule's
    sizes alone (every AO pair kept); once the setup is done the molecule is
    charged what its handle holds (only the Schwarz-kept pairs of B) plus the
    build's work buffers.  Builds of one molecule are serialised (its work
    buffers are shared)."""

    def __init__(self, mols, precision=dfjk.DFJK_MIXED, budget_bytes=150 << 30, slots=8,
                 keep_outputs=False, setup_workers=2, backend=None):
        """`backend`: (torch, handle class, bytes function[, set-up bytes
        function]) to use instead of torch, dfjk.Handle, resident_bytes and
        setup_bytes (host-logic tests on CPU)."""
        import threading
        from concurrent.futures import ThreadPoolExecutor

        if backend is None:
            import torch

            backend = (torch, dfjk.Handle, resident_bytes, setup_bytes)
        torch, self._handle_cls, self._bytes_fn = backend[:3]
        self._actual_fn = backend[3] if len(backend) > 3 else None
        self.torch = torch
        self.mols = mols
        self.precision = precision
        self.budget = budget_bytes
        self.keep = keep_outputs
        self.resident = {}  # mol_id -> Handle (set up, ready)
        self.nocc_of = {}  # mol_id -> the largest nocc it is charged for
        self.setting_up = {}  # mol_id -> Future of its Handle
        self.lru = Residency(budget_bytes)
        self.busy = set()  # mol_ids with a build or a setup in flight
        self.streams = [torch.cuda.Stream() for _ in range(slots)]
        self.free_slots = list(range(slots))
        self.stats = Stats()
        self._local = threading.local()
        self._pool = ThreadPoolExecutor(max_workers=max(1, setup_workers))
        self.device = torch.cuda.current_device()

    def _bytes(self, mol_id, nocc):
        m = self.mols[mol_id]
        return self._bytes_fn(m.nao, m.naux, nocc, self.precision)

    def _setup(self, mol_id):
        torch = self.torch
        if not hasattr(self._local, "stream"):
            torch.cuda.set_device(self.device)
            self._local.stream = torch.cuda.Stream()
        s = self._local.stream
        with torch.cuda.stream(s):
            h = self._handle_cls(self.mols[mol_id], precision=self.precision, stream=s)
        s.synchronize()
        return h

    def _start_setup(self, mol_id, nocc, keep) -> bool:
        """Reserves the molecule's bytes and starts its setup; False when the
        budget cannot be met now (every resident molecule is busy or needed
        by an older waiting request: `keep`)."""
        ok, evicted = self.lru.admit(mol_id, self._bytes(mol_id, nocc), self.busy | keep)
        for v in evicted:
            self.resident.pop(v).close()
            self.stats.evictions += 1
        if not ok:
            return False
        self.busy.add(mol_id)
        self.nocc_of[mol_id] = nocc
        self.setting_up[mol_id] = (self._pool.submit(self._setup, mol_id), nocc)
        self.stats.misses += 1
        return True

    def run(self, requests):
        torch = self.torch
        pending = collections.deque(sorted(requests, key=lambda r: r.arrival))
        waiting = collections.deque()
        inflight = []  # (request, slot, event, outputs)
        t0 = time.perf_counter()
        while pending or waiting or inflight or self.setting_up:
            now = time.perf_counter() - t0
            while pending and pending[0].arrival <= now:
                waiting.append(pending.popleft())
            progressed = False
            # setups that finished: their molecules become resident and idle
            for mid, (fut, nocc) in list(self.setting_up.items()):
                if fut.done():
                    del self.setting_up[mid]
                    self.busy.discard(mid)
                    progressed = True
                    try:
                        h = self.resident[mid] = fut.result()
                        if self._actual_fn is not None:
                            actual = self._actual_fn(h, self.mols[mid], nocc, self.precision)
                            if actual < self.lru.bytes.get(mid, 0):
                                self.lru.resize(mid, actual)
                    except dfjk.DfjkError as e:
                        # the molecule cannot be set up (device memory, budget):
                        # its waiting requests fail, its reservation is returned
                        self.lru.drop(mid)
                        for req in [r for r in waiting if r.mol_id == mid]:
                            req.error = str(e)
                            req.done = time.perf_counter() - t0
                            waiting.remove(req)
                            self.stats.failed += 1
            # admission, oldest waiting request first: a hit builds at once on a
            # free slot; requests whose molecule is busy (a build or a setup in
            # flight) wait.  Misses start their setups in arrival order: once
            # one cannot be admitted, younger misses wait too (they would take
            # the memory it waits for), and a miss never evicts a molecule an
            # older waiting request needs -- without these two rules a setup
            # could evict a molecule whose own setup had just finished, before
            # its request was built, and setups would chase each other forever
            started, keep, miss_blocked = set(), set(), False
            for req in list(waiting):
                mid = req.mol_id
                if mid in self.busy or mid in started:
                    keep.add(mid)
                    continue
                if self.lru.touch(mid):
                    keep.add(mid)
                    if not self.free_slots:
                        continue
                    h = self.resident[mid]
                    nocc = int(req.C.shape[1])
                    if nocc > self.nocc_of.get(mid, 0):
                        # a larger build work buffer: charge it (later
                        # admissions evict to make room)
                        self.nocc_of[mid] = nocc
                        grown = (self._actual_fn(h, self.mols[mid], nocc, self.precision)
                                 if self._actual_fn is not None else self._bytes(mid, nocc))
                        if grown > self.lru.bytes.get(mid, 0):
                            self.lru.resize(mid, grown)
                    slot = self.free_slots.pop()
                    s = self.streams[slot]
                    with torch.cuda.stream(s):
                        J, K, EJ, EK = h.build(req.C, stream=s, energies_on_device=True)
                        ev = torch.cuda.Event()
                        ev.record(s)
                    self.busy.add(mid)
                    inflight.append((req, slot, ev, (J, K, EJ, EK)))
                    waiting.remove(req)
                    progressed = True
                elif not miss_blocked:
                    if self._start_setup(mid, int(req.C.shape[1]), keep):
                        started.add(mid)
                        progressed = True
                    else:
                        miss_blocked = True
                    keep.add(mid)
            still = []
            for req, slot, ev, out in inflight:
                if ev.query():
                    req.done = time.perf_counter() - t0
                    J, K, EJ, EK = out
                    req.E = (float(EJ[0].item()), float(EK[0].item()))
                    if self.keep:
                        req.J, req.K = J[0], K[0]
                    self.stats.latencies.append(req.done - req.arrival)
                    self.busy.discard(req.mol_id)
                    self.free_slots.append(slot)
                    progressed = True
                else:
                    still.append((req, slot, ev, out))
            inflight = still
            if not progressed:
                if inflight or self.setting_up:
                    time.sleep(20e-6)
                elif pending and not waiting:
                    time.sleep(max(0.0, min(1e-3, pending[0].arrival - (time.perf_counter() - t0))))
                elif waiting:
                    # nothing in flight, so nothing is busy: admission cannot fail
                    raise RuntimeError("serving stalled: a waiting request could not be admitted")
        self.stats.seconds = time.perf_counter() - t0
        return requests

    def close(self):
        for fut, _ in self.setting_up.values():
            try:
                fut.result().close()
            except dfjk.DfjkError:
                pass
        self.setting_up.clear()
        self._pool.shutdown(wait=True)
        for h in self.resident.values():
            h.close()
        self.resident.clear()
        self.nocc_of.clear()
        self.lru = Residency(self.budget)


def make_stream(mols, nreq, rate, repeat=0.7, seed=5000, c_of=None, active=None):
    """Poisson arrivals; with probability `repeat` a request repeats a molecule
    whose SCF is in progress (new C_occ), otherwise it introduces the next
    molecule of the pool.  `active`: how many molecules are in SCF at once
    (the last `active` introduced; None = every molecule introduced so far).
    `c_of(mol_id, k)` returns the device C_occ of the k-th request of that
    molecule."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, size=nreq))
    seen, nxt, out, count = [], 0, [], collections.Counter()
    for i in range(nreq):
        live = seen if active is None else seen[-active:]
        if live and (rng.random() < repeat or nxt >= len(mols)):
            mid = live[int(rng.integers(len(live)))]
        else:
            mid = nxt
            seen.append(mid)
            nxt += 1
        out.append(Request(i, float(t[i]), mid, c_of(mid, count[mid])))
        count[mid] += 1
    return out
