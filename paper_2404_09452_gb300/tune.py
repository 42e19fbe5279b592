"""Autotuner of the launch shapes that do not change what the build
computes: rows per block of the slicing kernels (T, C and X slices; the
per-build slices of B), the K GEMM's split-K range and the mixed
build's work-buffer cap (which sets the aux-row chunk).

For each range of nao it times setup + build of a representative synthetic
molecule (the workload generator's atoms, nao = 15 per atom) on this GPU with
CUDA events, choosing one parameter at a time (coordinate descent from the
defaults, one pass), and writes a table that `dfjk_setup` reads through the
`tune_table` option or the DFJK_TUNE_TABLE environment variable:

    nao_lo nao_hi slice_rows pslice_rows k_range_mb build_ws_mb  # ms

The slicing choices leave every result bitwise equal; the K range and the
work-buffer cap regroup FP64 sums of exact slice products, so J and K move by
rounding only (checked here against the default shapes).
"""

from __future__ import annotations

import os
import statistics
import tempfile

from . import dfjk, inputs

# nao ranges (15 AOs per atom) and the atom count that represents each
BUCKETS = [(0, 150, 6), (150, 300, 14), (300, 600, 30), (600, 1200, 60), (1200, 2400, 110)]
CHOICES = {
    "slice_rows": [16, 8, 32],
    "pslice_rows": [4, 8, 16],
    "k_range_mb": [64, 32, 128],
    "build_ws_mb": [8192, 4096],
}
PARAMS = ["slice_rows", "pslice_rows", "k_range_mb", "build_ws_mb"]


def _write(path, rows):
    with open(path, "w") as f:
        f.write("# nao_lo nao_hi slice_rows pslice_rows k_range_mb build_ws_mb  # setup+build ms\n")
        for r in rows:
            f.write("%d %d %d %d %d %d  # %.3f\n" % tuple(r))


def _time(mol, C, table, reps, precision):
    import torch

    ms = []
    out = None
    for i in range(reps + 1):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        h = dfjk.Handle(mol, precision=precision, tune_table=table)
        J, K, EJ, EK = h.build(C)
        e1.record()
        torch.cuda.synchronize()
        if i > 0:
            ms.append(e0.elapsed_time(e1))
        out = (J[0].clone(), K[0].clone())
        h.close()
    return statistics.median(ms), out


def tune(path: str, buckets=BUCKETS, reps: int = 3, precision: int = dfjk.DFJK_MIXED, log=None) -> list:
    """Times the candidates on the current GPU and writes the table to
    `path`.  Returns its rows [nao_lo, nao_hi, choices..., ms]."""
    import torch

    rows = []
    tmp = tempfile.NamedTemporaryFile("w", suffix=".tune", delete=False)
    tmp.close()
    try:
        for lo, hi, natom in buckets:
            mol = inputs.molecule(natom, seed=8000 + natom)
            h = dfjk.Handle(mol, precision=dfjk.DFJK_FP64)
            C = torch.from_numpy(dfjk.orthonormal_c_occ(
                h, inputs.c_occ_raw(mol.nao, inputs.default_nocc(mol.nao), 3000))).cuda()
            h.close()
            best = {p: CHOICES[p][0] for p in PARAMS}

            def run(choice):
                _write(tmp.name, [[0, 1 << 30] + [choice[p] for p in PARAMS] + [0.0]])
                return _time(mol, C, tmp.name, reps, precision)

            best_ms, ref = run(best)
            for p in PARAMS:
                for v in CHOICES[p][1:]:
                    cand = dict(best, **{p: v})
                    ms, out = run(cand)
                    dJ = (out[0] - ref[0]).abs().max().item()
                    dK = (out[1] - ref[1]).abs().max().item()
                    if max(dJ, dK) > 1e-9:
                        raise RuntimeError(f"tuning choice {cand} changed J/K by {max(dJ, dK):.2e}")
                    if log:
                        log(f"nao [{lo},{hi}) {cand}: {ms:.3f} ms (best {best_ms:.3f})")
                    if ms < best_ms:
                        best, best_ms = cand, ms
            rows.append([lo, hi] + [best[p] for p in PARAMS] + [best_ms])
        _write(path, rows)
    finally:
        os.unlink(tmp.name)
    return rows
