#!/usr/bin/env python
"""DF-J/K benchmark: one step = the whole hot path (shell pairs, metric,
Cholesky, 3-centre integrals, whitening, X = B C, K, rho and J, energies) for
one synthetic molecule, through the C ABI.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp64|mixed]
                  [--workload mol60|mol120|water] [--impl ours|reference]

Prints one JSON line on rank 0.  `value` is whole-job builds/s with inputs
resident in HBM (device time, CUDA events, max over ranks); `e2e` is the same
metric through the public API with pinned host buffers and the host<->device
copies inside the timed region.  For N > 1 (torchrun) every rank runs its own
molecule (independent units, no data-path collective): weak scaling.
--impl reference times one complete FP64 CPU oracle build of the same
molecule, split into --steps consecutive pieces (rank 0 only).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time
import types

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "DF-J/K builds/s & TFLOP/s vs plain FP64 GPU at |ΔE|≤1e-6 Eh; p50/p99 latency"
UNIT = "builds/s"
WORKLOADS = {
    "mol60": dict(natom=60, seed=1002, note="60 atoms uniform in a cube at 0.01 atoms/bohr^3, "
                  "nao 900, naux 2160, nocc 180, Schwarz 1e-12"),
    "mol120": dict(natom=120, seed=1003, note="120 atoms, nao 1800, naux 4320, nocc 360"),
    "mol20": dict(natom=20, seed=1020, note="20 atoms, nao 300, naux 720, nocc 60 (profiling size)"),
    "water": dict(natom=0, seed=1001, note="3-atom water, nao 18, naux 30, nocc 5"),
}
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "traffic_mol60.md")
ERI_COUNTS_FILE = os.path.join(ROOT, "profiles", "eri3c_mol20.md")
PAIR_CLASSES = [(0, 0), (1, 0), (1, 1), (2, 0), (2, 1), (2, 2)]


def eri_flops_per_triple():
    """FP64 and FP32 flops per primitive triple of each 3-centre integral
    kernel, {(LA, LB, LC, "fp64"|"fp32"): (dflop, sflop)}: the ncu instruction
    counts of one capture (DFMA x2 + DMUL + DADD; FFMA x2 + FFMA2 x4 + FMUL +
    FADD) divided by the primitive triples that launch processed, both
    recorded in profiles/eri3c_mol20.md; empty when the kernel source
    (csrc/md.cuh) changed since the capture."""
    import hashlib

    src = os.path.join(ROOT, "paper_2404_09452_gb300", "csrc", "md.cuh")
    if not os.path.exists(ERI_COUNTS_FILE) or not os.path.exists(src):
        return {}
    sha = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    out = {}
    for line in open(ERI_COUNTS_FILE):
        f = line.split()
        # eri3c-count <LA> <LB> <LC> <fp64|fp32> <primitive triples> <dflop> <sflop> <sha16 of md.cuh>
        if len(f) == 9 and f[0] == "eri3c-count" and f[8] == sha and int(f[5]) > 0:
            n = float(f[5])
            out[(int(f[1]), int(f[2]), int(f[3]), f[4])] = (float(f[6]) / n, float(f[7]) / n)
    return out


def eri_roofline(h, m, ms64, ms32, fp64_peak, fp32_peak):
    """Roofline of the 3-centre integral phase (FP64-ALU bound): counted
    flops of the step's primitive triples per precision, divided by the
    phase's CUDA-event time, against the measured FMA rates."""
    per = eri_flops_per_triple()
    if not per:
        return None
    naux_prims = [sum(len(sh.exps) for sh in m.aux.shells if sh.l == lc) for lc in range(3)]
    f64 = f32_s = f32_d = 0.0
    trip64 = trip32 = 0
    for c, (la, lb) in enumerate(PAIR_CLASSES):
        for lc in range(3):
            t64 = h.prim_pairs_fp64[c] * naux_prims[lc]
            t32 = h.prim_pairs_fp32[c] * naux_prims[lc]
            trip64 += t64
            trip32 += t32
            d, _ = per.get((la, lb, lc, "fp64"), (0.0, 0.0))
            d32, s32 = per.get((la, lb, lc, "fp32"), (0.0, 0.0))
            f64 += t64 * d
            f32_d += t32 * d32
            f32_s += t32 * s32
    out = {"bound": "alu", "unit": "TFLOP/s", "primitive_triples_fp64": trip64,
           "primitive_triples_fp32": trip32, "flop_source": "ncu instruction counts per primitive triple "
           "(profiles/eri3c_mol20.md)"}
    if ms64:
        a = f64 / (ms64 / 1e3) / 1e12
        out["fp64"] = {"flops": f64, "ms": ms64, "achieved": a, "peak": fp64_peak, "frac": a / fp64_peak,
                       "peak_source": "dfjk_fma_rate(64), measured in this run"}
    if ms32:
        a = f32_s / (ms32 / 1e3) / 1e12
        out["fp32"] = {"flops": f32_s, "fp64_flops": f32_d, "ms": ms32, "achieved": a, "peak": fp32_peak,
                       "frac": a / fp32_peak, "peak_source": "dfjk_fma_rate(32), measured in this run"}
    return out


def gemm_source_sha() -> str:
    """sha256 of the tensor-core GEMM's source: csrc/ozaki.cu from its
    '// ---- GEMM' section marker to the end (the kernels, their tensor maps and
    launch code; the slicing kernels come before the marker)."""
    import hashlib

    src = os.path.join(ROOT, "paper_2404_09452_gb300", "csrc", "ozaki.cu")
    if not os.path.exists(src):
        return ""
    text = open(src, "rb").read()
    at = text.find(b"// ---- GEMM")
    return hashlib.sha256(text[at:] if at >= 0 else text).hexdigest()


def recorded_traffic(key: str, workload: str):
    """DRAM bytes (read + write) per launch of the tensor-core GEMM `key`, from the
    ncu capture summarised in profiles/traffic_mol60.md, or None when there is
    no capture for this workload or the GEMM source changed since (the summary
    records gemm_source_sha() at capture time)."""
    if not os.path.exists(TRAFFIC_FILE):
        return None
    sha = gemm_source_sha()
    for line in open(TRAFFIC_FILE):
        f = line.split()
        # traffic-per-launch <kernel> <workload> <bytes> <gemm_source_sha()>
        if len(f) == 5 and f[0] == "traffic-per-launch" and f[1] == key and f[2] == workload and f[4] == sha:
            return int(f[3])
    return None


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["fp64", "mixed"])
    ap.add_argument("--fp64-steps", type=int, default=2,
                    help="mixed runs: steps of the plain FP64 path timed alongside (0: skip)")
    ap.add_argument("--workload", default="mol60", choices=list(WORKLOADS) + ["batch", "serve", "gradient"])
    ap.add_argument("--grad-mol", default="mol60", choices=list(WORKLOADS),
                    help="molecule of --workload gradient")
    ap.add_argument("--batch-n", type=int, default=256)
    ap.add_argument("--autotune", action="store_true",
                    help="batch: run the autotuner (tune.py) first and use its table")
    ap.add_argument("--tune-table", default=None, help="tuning table to use (or to write with --autotune)")
    ap.add_argument("--compare-fp64", action="store_true",
                    help="batch/serve: also time the plain FP64 per-molecule path")
    ap.add_argument("--serve-rates", default="10,20,50,100,200,500")
    ap.add_argument("--serve-requests", type=int, default=2000, help="measured requests per rate")
    ap.add_argument("--serve-warmup", type=int, default=200, help="requests before the measured ones")
    ap.add_argument("--serve-max-atoms", type=int, default=150)
    ap.add_argument("--serve-slots", type=int, default=8)
    ap.add_argument("--serve-active", type=int, default=8,
                    help="molecules in SCF at once: repeats are drawn from the last this many introduced")
    ap.add_argument("--serve-fp64-rates", default="10,50")
    ap.add_argument("--serve-fp64-requests", type=int, default=100)
    ap.add_argument("--e2e-steps", type=int, default=-1,
                    help="steps of the end-to-end timing (-1: the same as --steps)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--b-on-host", action="store_true",
                    help="keep B in pinned host memory, read in place by the kernels")
    ap.add_argument("--fp32-pair-thresh", type=float, default=-1.0,
                    help="Schwarz bound below which shell pairs' integrals run in FP32 "
                         "(-1: the precision's default, 0: all FP64)")
    return ap.parse_args()


def make_molecule(name):
    from paper_2404_09452_gb300 import inputs as I

    w = WORKLOADS[name]
    if w["natom"] == 0:
        return I.water(), 5
    m = I.molecule(w["natom"], seed=w["seed"])
    return m, I.default_nocc(m.nao)


def algorithmic_flops(nao, naux, nocc, ncol):
    """Flops of each dense phase as the method defines them (not as tiled):
    whitening a triangular solve per kept AO pair, X = B_P C for every P,
    K on one triangle, rho and J on the mu >= nu rows."""
    return {
        "whiten": float(ncol) * naux * (naux + 1),
        "X=BC": 2.0 * naux * nao * nao * nocc,
        "K": float(naux) * nocc * nao * (nao + 1),
        "rho+J": 2.0 * 2.0 * naux * nao * (nao + 1) / 2 + 2.0 * nao * nao * nocc,
    }


def algorithmic_bytes(nao, naux, nocc, ncol):
    """Bytes each tensor-core GEMM must move once per step (operand slices read
    once, outputs written once): whitening reads the 8 BF16 slices of T and of
    L^-1 and writes B (one FP64 row per kept column); X reads the 6 slices of
    B (every mu, nu) and C and writes X; K reads the 6 slices of X and writes
    one FP64 triangle."""
    npad = (naux + 63) // 64 * 64
    return {
        "whiten": 16.0 * ncol * npad + 16.0 * npad * npad + 8.0 * ncol * npad,
        "X=BC": 12.0 * nao * nao * npad + 12.0 * nao * nocc + 8.0 * nao * npad * nocc,
        "K": 12.0 * nao * npad * nocc + 8.0 * nao * (nao + 1) / 2,
    }


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=5)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for n, v in zip(names, parts[3:7]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "samples": len(sm),
                "reasons": sorted(reasons)}


# ---- CPU baseline: one complete oracle build, in pieces ---------------------------------

def oracle_pieces(m, C, nsteps):
    """One complete FP64 CPU oracle build (steps O3-O10) of molecule `m` with
    orbitals C, as `nsteps` consecutive pieces, each a call of the oracle's
    own functions on the real inputs: the metric and the 3-centre integrals
    for consecutive ranges of aux shells (sym=True, the oracle's mirrored
    evaluation of mu >= nu pairs), then the whitening (Cholesky + triangular
    solve), then J, K and the energies.  Running all pieces in order is
    exactly one build; nothing is extrapolated.  Returns (pieces, state,
    kinds): callables, the dict they fill, and "setup"/"build" per piece."""
    import numpy as np

    from oracle import oracle as O

    na = len(m.aux.shells)
    nt = max(1, nsteps - 2) if nsteps >= 3 else 1
    bounds = np.linspace(0, na, nt + 1).astype(int)
    st = {"T": []}

    def t_piece(i):
        def f():
            if i == 0:
                st["V"] = O.metric(m.aux, m.coords)
            st["T"].append(O.three_center(m.orb, m.aux, m.coords, sym=True,
                                          aux_shells=(int(bounds[i]), int(bounds[i + 1]))))
        return f

    def whiten():
        T = np.concatenate(st.pop("T"), axis=0)
        st["L"], st["B"] = O.whiten(st["V"], T)

    def jk():
        st["out"] = O.jk_from_B(st.pop("B"), C)

    pieces = [t_piece(i) for i in range(nt)] + [whiten, jk]
    kinds = ["setup"] * (nt + 1) + ["build"]
    if nsteps == 2:  # [metric + integrals] [whitening + J/K]
        pieces = [pieces[0], lambda: (whiten(), jk())]
        kinds = ["setup", "setup+build"]
    elif nsteps == 1:
        pieces = [lambda: (t_piece(0)(), whiten(), jk())]
        kinds = ["setup+build"]
    return pieces, st, kinds


def oracle_build_timed(m, C, nsteps, nwarm=0):
    """Times oracle_pieces piece by piece (after `nwarm` untimed pieces of
    another build's integrals).  Returns (seconds per piece, kinds, state)."""
    if nwarm:
        wp, _, _ = oracle_pieces(m, C, max(3, nwarm + 2))
        for f in wp[:nwarm]:
            f()
    pieces, st, kinds = oracle_pieces(m, C, nsteps)
    secs = []
    for f in pieces:
        t0 = time.perf_counter()
        f()
        secs.append(time.perf_counter() - t0)
    return secs, kinds, st


def oracle_c_occ(m, nocc, seed):
    """C_occ of the workload for the CPU arm: orthonormal in the oracle's own
    overlap (the GPU arm uses the library's; the two agree to rounding)."""
    from oracle import oracle as O
    from paper_2404_09452_gb300 import inputs as I

    return I.orthonormalize(I.c_occ_raw(m.nao, nocc, seed), O.overlap(m.orb, m.coords))


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle import oracle as O

    m, nocc = make_molecule(args.workload)
    C = oracle_c_occ(m, nocc, 3000)
    secs, kinds, st = oracle_build_timed(m, C, args.steps, nwarm=args.warmup)
    total = sum(secs)
    value = 1.0 / total
    split = "setup+build" not in kinds  # with fewer than 3 steps a piece holds both
    setup_s = sum(t for t, k in zip(secs, kinds) if k == "setup") if split else None
    build_s = sum(t for t, k in zip(secs, kinds) if k == "build") if split else None
    desc = (f"one complete oracle build (metric, 3-centre integrals of every aux shell with sym=True, "
            f"Cholesky + triangular solve, J/K/energies) of the {m.natom}-atom workload on the real inputs, "
            f"in {len(secs)} consecutive pieces (one per step); value = 1 / total seconds")
    out = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / len(secs),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": args.workload, "note": WORKLOADS[args.workload]["note"]},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": O.num_threads(), "kind": "oracle",
                         "sample": desc, "setup_s": setup_s, "build_s": build_s,
                         "E_J": float(st["out"]["E_J"]), "E_K": float(st["out"]["E_K"])},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out), flush=True)


# ---- our arm -------------------------------------------------------------------------------

def run_ours(args):
    import numpy as np
    import torch

    from paper_2404_09452_gb300 import dfjk, dist as D, inputs as I

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    prec = dfjk.DFJK_MIXED if args.precision == "mixed" else dfjk.DFJK_FP64
    m, nocc = make_molecule(args.workload)

    # input preparation (outside any timed region): C_occ orthonormal in the
    # overlap metric the library computes; kept-pair columns for the flop count
    h0 = dfjk.Handle(m, precision=prec, fp32_pair_thresh=args.fp32_pair_thresh, b_on_host=args.b_on_host)
    fp32_pairs = {"thresh": h0.fp32_pair_thresh, "fp32_shell_pairs": h0.npair_fp32,
                  "kept_shell_pairs": h0.npair_kept}
    nslab, lean = h0.nslab, h0.lean
    pair_work = types.SimpleNamespace(prim_pairs_fp64=h0.prim_pairs_fp64, prim_pairs_fp32=h0.prim_pairs_fp32)
    S = h0.overlap().cpu().numpy()
    Cnp = I.orthonormalize(I.c_occ_raw(m.nao, nocc, 3000 + rank), S)
    mask = h0.pair_mask().cpu().numpy()
    nc = [(s.l + 1) * (s.l + 2) // 2 for s in m.orb.shells]
    ncol = sum(nc[a] * nc[b] for a in range(len(nc)) for b in range(a + 1) if mask[a, b])
    ncol -= sum(nc[a] * (nc[a] - 1) // 2 for a in range(len(nc)) if mask[a, a])
    h0.close()
    C = torch.from_numpy(Cnp).cuda()
    J = torch.empty((1, m.nao, m.nao), dtype=torch.float64, device="cuda")
    K = torch.empty_like(J)
    stream = torch.cuda.current_stream()

    chunks = [0, 0]  # aux-row chunks of the mixed build: rows, count

    def step():
        h = dfjk.Handle(m, precision=prec, fp32_pair_thresh=args.fp32_pair_thresh, b_on_host=args.b_on_host)
        _, _, EJ, EK = h.build(C, J=J, K=K)
        chunks[:] = h.build_chunks()
        h.close()
        return EJ[0], EK[0]

    # FP64 / FP32 FMA throughput of this GPU (the integral kernels' roofline)
    fp64_peak, fp32_peak = dfjk.fma_rate(64), dfjk.fma_rate(32)
    for _ in range(args.warmup):
        energies = step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    sampler.start()
    dfjk.phase_times()
    dfjk.set_timing(True)
    n0 = dfjk.launch_count()
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    evs[0].record(stream)
    for i in range(args.steps):
        energies = step()
        evs[i + 1].record(stream)
    torch.cuda.synchronize()
    launches = dfjk.launch_count() - n0
    dfjk.set_timing(False)
    phases = dfjk.phase_times()
    clocks = sampler.stop()
    if dist:
        dist.barrier()
    total_ms = evs[0].elapsed_time(evs[-1])
    step_ms = [evs[i].elapsed_time(evs[i + 1]) for i in range(args.steps)]
    total_ms = D.max_over_ranks(total_ms, device="cuda")
    value = world * args.steps / (total_ms / 1e3)

    # e2e: public API, pinned host C in, J/K/energies out, copies timed
    Ch = torch.from_numpy(Cnp).pin_memory()
    Jh = torch.empty((1, m.nao, m.nao), dtype=torch.float64).pin_memory()
    Kh = torch.empty_like(Jh).pin_memory()
    h2d = Ch.numel() * 8 + 8 * (m.coords.size + sum(2 * len(s.exps) for s in m.orb.shells + m.aux.shells))
    d2h = 2 * m.nao * m.nao * 8 + 16
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    e2e_steps = args.steps if args.e2e_steps < 0 else args.e2e_steps
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        Cd = Ch.to("cuda", non_blocking=True)
        h = dfjk.Handle(m, precision=prec, fp32_pair_thresh=args.fp32_pair_thresh, b_on_host=args.b_on_host)
        Jd, Kd, EJ, EK = h.build(Cd)
        Jh.copy_(Jd, non_blocking=True)
        Kh.copy_(Kd, non_blocking=True)
        torch.cuda.synchronize()
        h.close()
    e2e_s = D.max_over_ranks(time.perf_counter() - t0, device="cuda")
    e2e_value = world * e2e_steps / e2e_s if e2e_steps > 0 else None

    # the plain FP64 GPU path on the same input, same clocks: builds/s and the
    # energy deviation of the timed path from it
    fp64_cmp = None
    if prec != dfjk.DFJK_FP64 and args.fp64_steps > 0:
        def step64():
            h = dfjk.Handle(m, precision=dfjk.DFJK_FP64)
            J64, K64, EJ, EK = h.build(C)
            h.close()
            return J64, K64, EJ[0], EK[0]

        J64, K64, ej64, ek64 = step64()
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for _ in range(args.fp64_steps):
            step64()
        ev1.record(stream)
        torch.cuda.synchronize()
        ms64 = ev0.elapsed_time(ev1) / args.fp64_steps
        hm = dfjk.Handle(m, precision=prec, fp32_pair_thresh=args.fp32_pair_thresh, b_on_host=args.b_on_host)
        Jm, Km, ejm, ekm = hm.build(C)
        fp64_cmp = {"fp64_builds_per_s": 1e3 / ms64, "fp64_ms_per_step": ms64,
                    "dE_J_vs_fp64": abs(float(ejm[0]) - float(ej64)),
                    "dE_K_vs_fp64": abs(float(ekm[0]) - float(ek64)),
                    "max_dJ_vs_fp64": float((Jm[0] - J64[0]).abs().max()),
                    "max_dK_vs_fp64": float((Km[0] - K64[0]).abs().max())}
        hm.close()

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return

    flops = algorithmic_flops(m.nao, m.naux, nocc, ncol)
    per_step = {k: v / args.steps for k, v in phases.items()}
    step_flops = sum(flops.values())
    fp64 = prec == dfjk.DFJK_FP64
    peaks = {}
    if os.path.exists(PEAKS_FILE):
        peaks = json.load(open(PEAKS_FILE))
    bf16_sust = float(peaks.get("bf16_tflops_sustained", 1700.0))
    if fp64:
        dom = max(flops, key=lambda k: per_step.get(k, 0.0))
        dom_ms = per_step[dom]
        achieved = flops[dom] / (dom_ms / 1e3) / 1e12
        roof = {"kernel": dom, "bound": "alu", "achieved": achieved, "unit": "TFLOP/s",
                "peak": fp64_peak,
                "peak_source": "dfjk_fma_rate(64): FP64 FMA chains on every SM, measured in this run",
                "traffic": None, "algorithmic_flops_per_launch": flops[dom], "ms_per_launch": dom_ms,
                "launches_per_step": 1}
    else:
        # tensor-core GEMM launches alone; products = exact slice products per
        # FP64-equivalent multiply-add (S (S+1) / 2 with S = 8 or 6 slices)
        tc = {"whiten": ("tc:whiten", 36), "X=BC": ("tc:X=BC", 21), "K": ("tc:K", 21)}
        dom = max(tc, key=lambda k: per_step.get(tc[k][0], 0.0))
        key, prods = tc[dom]
        # launches per step: whitening one per T slab, X and K one per aux chunk
        nl = nslab if dom == "whiten" else max(1, chunks[1])
        dom_ms = per_step[key] / nl
        achieved = flops[dom] / nl / (dom_ms / 1e3) / 1e12
        roof = {"kernel": "oz_gemm_kernel (" + dom + ")", "bound": "tensor", "achieved": achieved,
                "unit": "TFLOP/s", "peak": bf16_sust / prods,
                "peak_source": f"measured sustained BF16 dense {bf16_sust} TFLOP/s of measured "
                               f"(MEASURED_PEAKS.json) / {prods} exact slice products",
                "tensor_pipe_tflops": achieved * prods, "traffic": recorded_traffic(dom, args.workload),
                "algorithmic_flops_per_launch": flops[dom] / nl, "ms_per_launch": dom_ms,
                "algorithmic_bytes_per_launch": algorithmic_bytes(m.nao, m.naux, nocc, ncol)[dom] / nl,
                "launches_per_step": nl}
    roof["frac"] = roof["achieved"] / roof["peak"]
    # per-row units of the measurement table: a4 as shell triples/s and
    # integrals/s, a8 (rho from X, then J over the rows of B: the kept
    # columns in the mixed path, the mu >= nu rows in FP64) as GB/s
    triples = int(fp32_pairs["kept_shell_pairs"]) * len(m.aux.shells)
    n_int = int(ncol) * int(m.naux)
    eri_ms = per_step.get("eri3c", 0.0) + per_step.get("eri3c32", 0.0)
    np_pad = (m.naux + 63) // 64 * 64
    b_rows = m.nao * (m.nao + 1) // 2 if fp64 else int(ncol)
    j_bytes = (b_rows * np_pad + m.nao * np_pad * nocc) * 8
    j_ms = per_step.get("rho+J", 0.0)
    units = {"a4_integrals": {"shell_triples": triples, "integrals": n_int, "ms": eri_ms,
                              "shell_triples_per_s": triples / (eri_ms / 1e3) if eri_ms else None,
                              "integrals_per_s": n_int / (eri_ms / 1e3) if eri_ms else None},
             "a8_rho_J": {"bytes": j_bytes, "ms": j_ms,
                          "GB_per_s": j_bytes / (j_ms / 1e3) / 1e9 if j_ms else None,
                          "note": "side stream, beside the K GEMM"}}
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if fp64 else "bf16 (exact 6-bit slices, fp32 accumulate) + f64",
        "data": "synthetic",
        "config": {"workload": args.workload, "note": WORKLOADS[args.workload]["note"],
                   "natom": m.natom, "nao": m.nao, "naux": m.naux, "nocc": nocc,
                   "kept_ao_pairs": ncol, "precision": args.precision, "fp32_integrals": fp32_pairs,
                   "t_slabs": nslab, "memory_lean": lean, "b_on_host": bool(args.b_on_host),
                   "l2": "working set > L2 (B alone is GBs), no flush needed",
                   "parallelism": f"replicas x{world}"},
        "tflops": step_flops / (total_ms / args.steps / 1e3) / 1e12,
        "p50_ms": statistics.median(step_ms), "p99_ms": max(step_ms) if len(step_ms) < 100 else
        sorted(step_ms)[int(0.99 * len(step_ms))],
        "phase_ms": per_step, "E_J": float(energies[0]), "E_K": float(energies[1]),
        "roofline": roof,
        "units": units,
        "roofline_a4": eri_roofline(pair_work, m, per_step.get("eri3c", 0.0), per_step.get("eri3c32", 0.0),
                                    fp64_peak, fp32_peak),
        "fma_peaks_tflops": {"fp64": fp64_peak, "fp32": fp32_peak},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h)},
        "gpu_launches": int(launches),
        "clocks": clocks,
    }
    if fp64_cmp:
        out.update(fp64_cmp)
        out["vs_fp64"] = value / fp64_cmp["fp64_builds_per_s"]
    if world == 1 and not args.no_cpu_baseline:
        from oracle import oracle as O

        secs, kinds, st = oracle_build_timed(m, oracle_c_occ(m, nocc, 3000), 3)
        out["cpu_baseline"] = {
            "value": 1.0 / sum(secs), "unit": UNIT, "cores": O.num_threads(), "kind": "oracle",
            "sample": f"one complete oracle build of the {m.natom}-atom workload (metric, 3-centre integrals "
                      f"sym=True, Cholesky + triangular solve, J/K/energies) on the real inputs, timed "
                      f"once; value = 1 / seconds",
            "setup_s": secs[0] + secs[1], "build_s": secs[2],
            "dE_J_vs_timed_path": abs(float(st["out"]["E_J"]) - float(energies[0])),
            "dE_K_vs_timed_path": abs(float(st["out"]["E_K"]) - float(energies[1]))}
    print(json.dumps(out), flush=True)
    if dist:
        dist.destroy_process_group()


def _orthonormal_cs(mols, seed0):
    import torch

    from paper_2404_09452_gb300 import dfjk, inputs as I

    out = []
    for i, m in enumerate(mols):
        S = dfjk.overlap_matrix(m).cpu().numpy()
        C = I.orthonormalize(I.c_occ_raw(m.nao, I.default_nocc(m.nao), seed0 + i), S)
        out.append(torch.from_numpy(C).cuda())
    return out


def run_batch_mode(args):
    """Batching: a batch of uneven molecules (atom counts uniform in [5, 80],
    seed 4000), each set up and built once per step; waves under a 150 GB
    budget, concurrent setups, one multi-stream build call per wave."""
    import torch

    from paper_2404_09452_gb300 import batch, dfjk, inputs as I

    counts = I.batch_atom_counts(n=args.batch_n)
    mols = [I.molecule(int(n), seed=4100 + i) for i, n in enumerate(counts)]
    Cs = _orthonormal_cs(mols, 3000)
    prec = dfjk.DFJK_MIXED if args.precision == "mixed" else dfjk.DFJK_FP64
    table, tune_rows, tune_s = args.tune_table, None, None
    if args.autotune:  # the project's autotuner picks the launch shapes on this GPU first
        from paper_2404_09452_gb300 import tune

        table = table or os.path.join(ROOT, "_build", "dfjk_tune.txt")
        os.makedirs(os.path.dirname(table), exist_ok=True)
        t0 = time.perf_counter()
        tune_rows = tune.tune(table, precision=prec)
        tune_s = time.perf_counter() - t0
    for _ in range(args.warmup):
        batch.run_batch(mols, Cs, precision=prec, tune_table=table)
    torch.cuda.synchronize()
    n0 = dfjk.launch_count()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        E, _, st = batch.run_batch(mols, Cs, precision=prec, tune_table=table)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    out = {"metric": "DF-J/K builds/s, batch of uneven molecules (setup + build each)",
           "value": len(mols) * args.steps / dt, "unit": UNIT, "n_gpus": 1, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True,
           "scaling": "weak", "dtype": "f64" if prec == dfjk.DFJK_FP64 else "f64+bf16-sliced",
           "data": "synthetic",
           "config": {"workload": f"batch of {len(mols)} molecules, atoms uniform in [5, 80] (seed 4000)",
                      "atoms_total": int(sum(counts)), "waves": st["waves"], "precision": args.precision,
                      "budget_bytes": 150 << 30, "tune_table": table, "tuned": tune_rows,
                      "tuning_s": tune_s},
           "gpu_launches": int(dfjk.launch_count() - n0)}
    if args.compare_fp64:
        t0 = time.perf_counter()
        for m, C in zip(mols, Cs):
            h = dfjk.Handle(m, precision=dfjk.DFJK_FP64)
            h.build(C)
            h.close()
        torch.cuda.synchronize()
        out["fp64_sequential_builds_per_s"] = len(mols) / (time.perf_counter() - t0)
        out["vs_fp64_sequential"] = out["value"] / out["fp64_sequential_builds_per_s"]
    print(json.dumps(out), flush=True)


def run_gradient_mode(args):
    """Nuclear gradient of E_J - E_K / 2 at fixed D = C C^T (derivative 3c and
    2c integrals, FP64), after the setup; also the Coulomb-only gradient."""
    import torch

    from paper_2404_09452_gb300 import dfjk

    m, nocc = make_molecule(args.grad_mol)
    C = _orthonormal_cs([m], 3000)[0][:, :nocc].contiguous()
    prec = dfjk.DFJK_MIXED if args.precision == "mixed" else dfjk.DFJK_FP64
    h = dfjk.Handle(m, precision=prec)
    res = {}
    for name, ck in (("jk", -0.5), ("j", 0.0)):
        for _ in range(args.warmup):
            h.jk_gradient(C, 1.0, ck)
        torch.cuda.synchronize()
        n0 = dfjk.launch_count()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.steps):
            g = h.jk_gradient(C, 1.0, ck)
        e1.record()
        torch.cuda.synchronize()
        res[name] = (e0.elapsed_time(e1) / args.steps, (dfjk.launch_count() - n0) // args.steps)
    h.close()
    out = {"metric": "DF J/K nuclear gradients/s (after setup)", "value": 1e3 / res["jk"][0],
           "unit": "gradients/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": res["jk"][0], "higher_is_better": True, "scaling": "weak", "dtype": "f64",
           "data": "synthetic",
           "config": {"workload": WORKLOADS[args.grad_mol]["note"], "energy": "E_J - E_K/2",
                      "handle_precision": args.precision},
           "ms_coulomb_only": res["j"][0], "gpu_launches": int(res["jk"][1]),
           "max_abs_grad": float(g.abs().max())}
    print(json.dumps(out), flush=True)


def run_serve_mode(args):
    """Serving: Poisson requests for molecules with atom counts log-uniform in
    [5, serve-max-atoms]; with probability 0.7 a request repeats a molecule
    already requested (new C_occ: an SCF-iteration pattern), otherwise it
    brings the next molecule of the pool; 150 GB residency budget with LRU
    eviction and recompute.  Per arrival rate: p50/p99 latency and builds/s
    over the requests after the warm-up ones, for the mixed path and (on a
    shorter stream) the plain FP64 path with the same slots."""
    import torch

    from paper_2404_09452_gb300 import dfjk, inputs as I, serve

    nreq, nwarm = args.serve_requests, args.serve_warmup
    total = nreq + nwarm
    npool = int(0.3 * total * 1.2) + 8  # new molecules are ~30 % of the requests
    counts = I.serve_atom_counts(npool, hi=args.serve_max_atoms)
    pool = [I.molecule(int(n), seed=6100 + i) for i, n in enumerate(counts)]
    t_prep = time.perf_counter()
    Cbase = _orthonormal_cs(pool, 3100)
    t_prep = time.perf_counter() - t_prep
    # four orbital sets per molecule (an SCF-like sequence of new C_occ)
    rng_sets = {}

    def c_of(mid, k):
        key = (mid, k % 4)
        if key not in rng_sets:
            C = Cbase[mid]
            Q, _ = torch.linalg.qr(torch.randn(C.shape[1], C.shape[1], dtype=torch.float64,
                                               generator=torch.Generator().manual_seed(97 * mid + key[1])))
            rng_sets[key] = (C @ Q.cuda()).contiguous()
        return rng_sets[key]

    def measure(prec, rate, n, warm, slots):
        reqs = serve.make_stream(pool, n + warm, rate, repeat=0.7, seed=5000 + int(rate), c_of=c_of,
                                 active=args.serve_active)
        srv = serve.Server(pool, precision=prec, budget_bytes=150 << 30, slots=slots)
        srv.run(reqs)
        st = srv.stats
        srv.close()
        meas = [r for r in reqs[warm:] if not r.error]
        lat = np.array([r.done - r.arrival for r in meas]) * 1e3
        span = max(r.done for r in meas) - min(r.arrival for r in reqs[warm:])
        sizes = [pool[r.mol_id].natom for r in reqs[warm:]]
        return {"rate": rate, "requests": len(meas), "warmup_requests": warm,
                "failed": sum(1 for r in reqs[warm:] if r.error),
                "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                "builds_per_s": len(meas) / span, "misses": st.misses, "evictions": st.evictions,
                "distinct_molecules": len(set(r.mol_id for r in reqs)),
                "atoms_median": float(np.median(sizes)), "atoms_max": int(max(sizes)), "slots": slots}

    import numpy as np

    rates = [float(r) for r in args.serve_rates.split(",")]
    rows = []
    for rate in rates:
        row = measure(dfjk.DFJK_MIXED, rate, nreq, nwarm, args.serve_slots)
        row["precision"] = "mixed"
        rows.append(row)
        print(json.dumps(row), file=sys.stderr, flush=True)
    if args.compare_fp64:
        for rate in [float(r) for r in args.serve_fp64_rates.split(",")]:
            row = measure(dfjk.DFJK_FP64, rate, args.serve_fp64_requests, max(1, args.serve_fp64_requests // 10),
                          args.serve_slots)
            row["precision"] = "fp64"
            rows.append(row)
            print(json.dumps(row), file=sys.stderr, flush=True)
    best = max(r["builds_per_s"] for r in rows if r["precision"] == "mixed")
    out = {"metric": "DF-J/K serving: builds/s and p50/p99 latency under Poisson arrivals",
           "value": best, "unit": UNIT, "n_gpus": 1, "higher_is_better": True, "scaling": "weak",
           "dtype": "f64+bf16-sliced", "data": "synthetic",
           "config": {"workload": f"Poisson requests, molecules with atoms log-uniform in [5, {args.serve_max_atoms}] "
                                  f"(pool of {len(pool)}), 70% repeats of one of the {args.serve_active} molecules "
                                  f"in SCF (the last introduced), {nreq} requests per "
                                  f"rate after {nwarm} warm-up requests, 150 GB residency budget, "
                                  f"{args.serve_slots} build slots",
                      "input_prep_s": t_prep},
           "rates": rows}
    print(json.dumps(out), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batch":
        run_batch_mode(args)
    elif args.workload == "serve":
        run_serve_mode(args)
    elif args.workload == "gradient":
        run_gradient_mode(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
