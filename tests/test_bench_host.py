"""Host-side accounting of the benchmark: the algorithmic byte counts that
the reported GB/s divide by, and the gating of the recorded ncu traffic on
the kernel source it was measured on.  No GPU is needed."""

import os
import shutil

import bench


def test_iteration_bytes_from_the_fused_passes():
    """One fused BiCGStab iteration: two SpMVs (values, columns, row pointers,
    x read once, y written once) plus the vector traffic of F1..F5 (16 bytes
    per complex128 element read or written)."""
    n, nnz = 618401, 9181729
    vec = 16 * n
    passes = {
        "F1 p = r + beta (p - omega v)": 3 * vec + vec,   # read r, p, v; write p
        "F2 epilogue <rh, v>": vec,                       # read rh (v is the SpMV output)
        "F3 s = r - alpha v": 2 * vec + vec,              # read r, v; write s
        "F4 epilogue <t, s>, <t, t>": 0,                  # s is the SpMV input
        "F5 x, r update": 5 * vec + 2 * vec,              # read x, p, s, t, rh; write x, r
    }
    two_spmv = 2 * (bench.spmv_bytes(n, nnz) - 4)
    assert bench.iter_bytes(n, nnz) == two_spmv + sum(passes.values())


def test_spmv_bytes_counts_each_array_once():
    n, nnz = 5, 11
    # val 16 + col 4 per entry, rowptr 4 (n + 1), x 16 read, y 16 written
    assert bench.spmv_bytes(n, nnz) == 16 * nnz + 4 * nnz + 4 * (n + 1) + 16 * n + 16 * n


def test_solve_bytes_is_start_plus_iterations_plus_finish():
    n, nnz = 1000, 7000
    s0 = bench.solve_bytes(n, nnz, 0)
    for k in (1, 7, 1000):
        assert bench.solve_bytes(n, nnz, k) - s0 == k * bench.iter_bytes(n, nnz)
    # start: x0 copy, r = b - A x (one SpMV, b read, r/rh/p/v written);
    # finish: the true-residual SpMV, b read, copy-out
    assert s0 == 32 * n + bench.spmv_bytes(n, nnz) + 16 * n + 64 * n + bench.spmv_bytes(n, nnz) + 48 * n


def _fake_root(tmp_path, sha):
    csrc = tmp_path / "paper_2112_06465_gb300" / "csrc"
    csrc.mkdir(parents=True)
    src = os.path.join(bench.ROOT, "paper_2112_06465_gb300", "csrc")
    for f in ("spmv.cuh", "hz_internal.cuh", "arith.cuh", "spmv.cu"):
        shutil.copy(os.path.join(src, f), csrc / f)
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "spmv_ffb_c2_traffic.txt").write_text(
        "# comment: 1\ndram_bytes_per_launch: 123456\nkernel_source_sha: %s\n" % sha)
    return str(tmp_path)


def test_recorded_traffic_only_for_the_measured_source(tmp_path, monkeypatch):
    root = _fake_root(tmp_path, "0" * 16)
    monkeypatch.setattr(bench, "ROOT", root)
    current = bench.kernel_source_sha()
    assert bench.recorded_traffic("spmv_ffb_c2_traffic.txt") is None               # another kernel source
    (tmp_path / "profiles" / "spmv_ffb_c2_traffic.txt").write_text(
        "dram_bytes_per_launch: 123456\nkernel_source_sha: %s\n" % current)
    assert bench.recorded_traffic("spmv_ffb_c2_traffic.txt") == 123456.0
    with open(os.path.join(root, "paper_2112_06465_gb300", "csrc", "spmv.cu"), "a") as f:
        f.write("\n// edited\n")
    assert bench.kernel_source_sha() != current          # any edit invalidates it
    assert bench.recorded_traffic("spmv_ffb_c2_traffic.txt") is None


def test_peaks_fall_back_when_unmeasured(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.peaks() == (bench.FALLBACK_HBM_GBS, "fallback")
    (tmp_path / "MEASURED_PEAKS.json").write_text('{"hbm_gbs": 6774.6}')
    assert bench.peaks() == (6774.6, "measured")
