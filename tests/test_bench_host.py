"""Host-side logic of bench.py that needs no GPU: the kernel hash that keys the
committed ncu summaries, the traffic lookup per (storage, lattice), workload
names and the FP64 roofline constants."""
import os
import re
import shutil

import pytest

import bench


def test_kernel_hash_ignores_comments_and_whitespace(tmp_path, monkeypatch):
    src = os.path.join(bench.ROOT, "paper_1202_6130_gb300", "csrc")
    fake_root = tmp_path / "root"
    dst = fake_root / "paper_1202_6130_gb300" / "csrc"
    dst.mkdir(parents=True)
    for f in bench.KERNEL_SOURCES:
        shutil.copy(os.path.join(src, f), dst / f)
    monkeypatch.setattr(bench, "ROOT", str(fake_root))
    h0 = bench.kernel_hash()
    assert h0 == bench.kernel_hash() and re.fullmatch(r"[0-9a-f]{16}", h0)
    p = dst / "step_kernel.cuh"
    text = p.read_text()
    p.write_text("// a new comment line\n" + text.replace("\n", "\n\n", 3) + "\n/* block */\n")
    assert bench.kernel_hash() == h0
    p.write_text(text.replace("__syncthreads();", "__syncthreads(); __syncthreads();", 1))
    assert bench.kernel_hash() != h0


def test_traffic_comes_only_from_a_summary_of_the_current_kernels():
    # every committed full-size summary resolves for its own storage and lattice
    for st, q in (("fp32", 9), ("fp16s", 9), ("bf16s", 9), ("fp32", 21), ("fp16s", 21)):
        path = os.path.join(bench.ROOT, "profiles", f"step_{st}_d2q{q}_8192x4096.txt")
        assert os.path.exists(path), path
        text = open(path).read()
        h = re.search(r"kernel_hash:\s*([0-9a-f]+)", text).group(1)
        t = bench.ncu_traffic(st, q)
        if h == bench.kernel_hash():
            assert t is not None and t > 2 * q * bench.BYTES[st] * 8192 * 4096 * 0.9
        else:
            assert t is None
    assert bench.ncu_traffic("fp64", 9) is None          # no full-size FP64 summary


def test_workload_names_and_fp64_constants():
    assert bench.workload_name(8192, 4096, 9) == bench.WORKLOAD
    n21 = bench.workload_name(1024, 512, 21)
    assert n21.startswith("1024x512 D2Q21") and "D2Q9" not in n21
    # executed FP64 flops per node grow with the velocity set; the DFMA peak of
    # a GB300 (152 SMs at 2.07 GHz) is its nominal 1.25 TFLOP/s
    assert bench.FP64_FLOPS_PER_NODE[21] > bench.FP64_FLOPS_PER_NODE[9] > 0
    peak = 152 * bench.FP64_DFMA_PER_SM_CLK * 2 * 2.07e9 / 1e12
    assert peak == pytest.approx(1.25, rel=0.02)


def test_all_cores_baseline_runs_the_oracle_in_spawned_processes():
    r = bench.cpu_baseline_all_cores(lattice=9, rows=4, seconds=0.2)
    assert r["kind"] == "oracle" and r["unit"] == "MLUPS"
    assert r["cores"] == max(1, min(64, os.cpu_count() or 1))
    assert r["value"] > 0 and str(r["cores"]) in r["sample"]
