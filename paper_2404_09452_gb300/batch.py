"""Batched DF-J/K over many molecules of uneven size.

The paper runs one molecule per GPU job; this driver processes a list of
molecules (e.g. 256 with 5-80 atoms) on one GPU: molecules are grouped into
waves whose resident data fit a device-memory budget; within a wave the
setups run concurrently from worker threads (each with its own CUDA stream;
the C ABI releases the GIL), then one `dfjk_build_batch` call builds every
handle of the wave over several streams, and the wave is released.
"""

from __future__ import annotations

import threading
import time
from concurrent.futures import ThreadPoolExecutor

from . import dfjk


def resident_bytes(nao: int, naux: int, nocc: int, precision: int) -> int:
    """Device bytes one molecule holds while set up and built, as the library
    states them (dfjk_estimate_bytes) from its sizes alone: its resident data
    (B -- in the mixed path bounded by every mu >= nu pair, of which the setup
    keeps the Schwarz-significant ones, both triangles in the FP64 path -- and
    the metric, its Cholesky factor and inverse) plus the larger of the
    build's work buffers and the setup's transient peak."""
    e = dfjk.estimate_bytes(nao, naux, nocc, precision)
    return int(e["resident"] + max(e["build_ws"], e["setup_ws"]))


def make_waves(sizes, budget: int):
    """Greedy waves in the given order: indices whose summed bytes fit the budget
    (a molecule larger than the budget gets a wave of its own)."""
    waves, cur, used = [], [], 0
    for i, b in enumerate(sizes):
        if cur and used + b > budget:
            waves.append(cur)
            cur, used = [], 0
        cur.append(i)
        used += b
    if cur:
        waves.append(cur)
    return waves


def run_batch(mols, Cs, precision=dfjk.DFJK_MIXED, budget_bytes=150 << 30, workers=4, nstreams=8,
              keep_results=False, tune_table=None):
    """Setup + build for every molecule.  `Cs` are device tensors [nao_i, nocc_i];
    `tune_table`: launch shapes from the autotuner (tune.py), or None.
    Returns (energies [n, 2] numpy, results or None, stats dict)."""
    import numpy as np
    import torch

    n = len(mols)
    sizes = [resident_bytes(m.nao, m.naux, int(C.shape[1]), precision) for m, C in zip(mols, Cs)]
    waves = make_waves(sizes, budget_bytes)
    energies = np.zeros((n, 2))
    results = [None] * n if keep_results else None
    local = threading.local()

    def setup(i):
        if not hasattr(local, "stream"):
            local.stream = torch.cuda.Stream()
        with torch.cuda.stream(local.stream):
            h = dfjk.Handle(mols[i], precision=precision, stream=local.stream, tune_table=tune_table)
        local.stream.synchronize()
        return h

    t0 = time.perf_counter()
    with ThreadPoolExecutor(max_workers=max(1, workers)) as ex:
        for wave in waves:
            # biggest first inside a wave so the long setups start early
            order = sorted(wave, key=lambda i: -sizes[i])
            handles = dict(zip(order, ex.map(setup, order)))
            hs = [handles[i] for i in wave]
            torch.cuda.current_stream().synchronize()
            Js, Ks, E = dfjk.build_batch(hs, [Cs[i] for i in wave], nstreams=nstreams)
            torch.cuda.current_stream().synchronize()
            e = E.cpu().numpy()
            for k, i in enumerate(wave):
                energies[i] = e[:, k]
                if keep_results:
                    results[i] = (Js[k].clone(), Ks[k].clone())
            for h in hs:
                h.close()
    dt = time.perf_counter() - t0
    return energies, results, {"seconds": dt, "waves": len(waves), "builds_per_s": n / dt}
