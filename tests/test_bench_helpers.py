"""Host logic of bench.py's measurement fields (no GPU): the recorded DRAM
traffic and integral flop counts are used only while the source they were
captured with is unchanged, and the algorithmic work formulas count what the
build computes."""
import hashlib
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import bench  # noqa: E402


def test_recorded_traffic_needs_the_capture_time_gemm_source(tmp_path, monkeypatch):
    sha = bench.gemm_source_sha()
    assert len(sha) == 64
    f = tmp_path / "traffic.md"
    f.write_text(f"traffic-per-launch X=BC mol60 123 {sha}\n"
                 f"traffic-per-launch K mol60 456 {'0' * 64}\n")
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(f))
    assert bench.recorded_traffic("X=BC", "mol60") == 123
    assert bench.recorded_traffic("X=BC", "mol120") is None  # another workload
    assert bench.recorded_traffic("K", "mol60") is None  # another source


def test_gemm_source_sha_covers_the_gemm_section_only():
    src = os.path.join(bench.ROOT, "paper_2404_09452_gb300", "csrc", "ozaki.cu")
    text = open(src, "rb").read()
    at = text.find(b"// ---- GEMM")
    assert at > 0 and text.find(b"oz_slice_sym_kernel") < at < text.find(b"oz_gemm_ws_kernel")
    assert bench.gemm_source_sha() == hashlib.sha256(text[at:]).hexdigest()


def test_eri_counts_need_the_capture_time_kernel_source(tmp_path, monkeypatch):
    src = os.path.join(bench.ROOT, "paper_2404_09452_gb300", "csrc", "md.cuh")
    sha16 = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    f = tmp_path / "eri.md"
    f.write_text(f"eri3c-count 2 2 2 fp64 100 5000 0 {sha16}\n"
                 f"eri3c-count 1 0 0 fp32 10 20 300 {'f' * 16}\n")
    monkeypatch.setattr(bench, "ERI_COUNTS_FILE", str(f))
    per = bench.eri_flops_per_triple()
    assert per == {(2, 2, 2, "fp64"): (50.0, 0.0)}


def test_algorithmic_work_formulas():
    nao, naux, nocc, ncol = 4, 6, 2, 7
    fl = bench.algorithmic_flops(nao, naux, nocc, ncol)
    assert fl["whiten"] == ncol * naux * (naux + 1)          # triangular L^-1 times T
    assert fl["X=BC"] == 2 * naux * nao * nao * nocc
    assert fl["K"] == naux * nocc * nao * (nao + 1)          # one triangle of K
    by = bench.algorithmic_bytes(nao, naux, nocc, ncol)
    npad = 64
    assert by["whiten"] == 16 * ncol * npad + 16 * npad * npad + 8 * ncol * npad
    assert by["X=BC"] == 12 * nao * nao * npad + 12 * nao * nocc + 8 * nao * npad * nocc
