"""The benchmark's JSON contract and the per-unit work its roofline divides by.

CPU: the algorithmic work per unit (butterflies of the exact-integer matvec, flops of the FP64 FFT matvec and
of one COCG iteration) written out from the transforms' definitions.
GPU: one small run of the bench's own arm prints exactly one JSON line with every key of the contract.
"""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_ntt_butterflies_per_row():
    # 4 primes x (forward + inverse) radix-2 NTT of the embedding length L (the smallest power of
    # two >= 2M, at least 4): L/2 butterflies per stage, log2 L stages
    assert bench.ntt_butterflies(8191, 1) == 4 * 2 * 8192 * 14
    assert bench.ntt_butterflies(8191, 1024) == 1024 * 4 * 2 * 8192 * 14
    assert bench.ntt_butterflies(1, 1) == 4 * 2 * 2 * 2
    assert bench.ntt_butterflies(4097, 1) == 4 * 2 * 8192 * 14  # 2M = 8194 -> L = 16384


def test_fft64_matvec_flops_per_row():
    # real FFT convolution of length L = 16384: two complex FFTs of L/2 (5 n log2 n each), 20 flops per
    # half-length point for the real split / merge and spectrum product, 5 flops per point of the BDF band
    n = 8192
    assert bench.matvec_flops(8191, 1) == pytest.approx(2 * 5 * n * np.log2(n) + 20 * n + 5 * 8191)


@pytest.mark.parametrize("inner,strang_ffts,pre_ffts", [("strang", 2, 2), ("strang", 4, 4), ("tau", 4, 2)])
def test_cocg_flops(inner, strang_ffts, pre_ffts):
    # per iteration: the Toeplitz product (2 FFTs of L) + one preconditioner solve + 40 flops per point;
    # each system also applies the preconditioner once before its first iteration
    L = 16384
    f = 5 * L * np.log2(L)
    iters, n_apply, nsys = 37, 3, 5
    want = iters * (2 * f + pre_ffts * f + 40 * 8191) + n_apply * nsys * pre_ffts * f
    assert bench.cocg_flops(8191, inner, iters, n_apply, nsys, strang_ffts=strang_ffts) == pytest.approx(want)


@pytest.mark.gpu
def test_bench_json_contract_small_run():
    M, Nt = 255, 32
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--M", str(M), "--Nt", str(Nt), "--steps", "1",
           "--warmup", "3", "--no-cpu-baseline"]
    out = subprocess.run(cmd, capture_output=True, text=True, timeout=900, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-3000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, out.stdout[-3000:]
    rec = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "roofline", "e2e", "clocks", "gpu_launches"):
        assert k in rec, k
    assert rec["n_gpus"] == 1 and rec["steps"] == 1 and rec["warmup"] == 3
    assert rec["value"] > 0 and rec["ms_per_step"] > 0 and rec["higher_is_better"] is True
    assert rec["scaling"] == "weak" and rec["data"] == "synthetic" and rec["gpu_launches"] > 0
    assert rec["value"] == pytest.approx(M * Nt / (rec["ms_per_step"] * 1e-3), rel=1e-6)
    roof = rec["roofline"]
    for k in ("bound", "achieved", "peak", "unit", "frac", "traffic"):
        assert k in roof, k
    assert roof["peak"] > 0 and roof["frac"] == pytest.approx(roof["achieved"] / roof["peak"])
    e2e = rec["e2e"]
    assert e2e["value"] > 0 and e2e["unit"] == rec["unit"]
    assert e2e["h2d_bytes_per_step"] == M * Nt * 8 and e2e["d2h_bytes_per_step"] == M * Nt * 8
    assert "sm_mhz" in rec["clocks"] and "reasons" in rec["clocks"]
    cfg = rec["config"]
    assert "workload" in cfg and cfg["M"] == M and cfg["Nt"] == Nt
    assert cfg["true_rel_res_max"] <= 1e-10
