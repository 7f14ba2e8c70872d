"""Host-side helpers of bench.py: the nvidia-smi clock summary, the
algorithmic-bytes model of the refinement kernel, the backward error of the
bench lines and the recipe of the 512-system batch (CPU only)."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_clock_summary_reads_one_device(tmp_path):
    p = tmp_path / "clocks.csv"
    p.write_text(
        "0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active\n"
        "1, 1500, 2070, 300.0, 0x0, Active, Not Active, Not Active, Not Active\n"
        "0, 2070, 2070, 950.2, 0x4, Not Active, Not Active, Not Active, Active\n"
        "0, 1980, 2070, 1001.0, 0x0, Not Active, Not Active, Not Active, Not Active\n"
        "garbage line\n")
    s = bench.ClockSampler(str(p)).summary(0)
    assert s == dict(sm_mhz=2070.0, sm_max_mhz=2070.0, reasons=["sw_power_cap"], samples=3)
    s1 = bench.ClockSampler(str(p)).summary(1)
    assert s1["reasons"] == ["hw_slowdown"] and s1["samples"] == 1
    assert bench.ClockSampler(str(tmp_path / "missing.csv")).summary(0) is None


def test_ir_kernel_bytes_hand_example():
    # n = 2, nnz(A) = 3, nnz(P) = 4, one refinement step with one Arnoldi iteration,
    # all vectors 4-byte: rowptr 24 B; SpMV A 24 + 24 + 8 + 8 = 64; SpMV P 32 + 24 + 8 = 64;
    # residual 36 + 24 + 16 + 8 + 8 = 92 (twice: the step's and the final stop test);
    # z = P r 32 + 24 + 8 + 8 = 72; MGS 8 + 16 = 24; d = V y 8 + 16 = 24
    assert bench.ir_kernel_bytes(2, 3, 4, [1]) == 92 + 92 + 72 + 64 + 64 + 24 + 24
    # bytes grow with every Arnoldi iteration by the two products plus (j + 3) basis vectors
    b1 = bench.ir_kernel_bytes(10, 30, 40, [3])
    b2 = bench.ir_kernel_bytes(10, 30, 40, [4])
    spmv = (30 * 8 + 11 * 8 + 10 * 8) + (40 * 8 + 11 * 8 + 10 * 4)
    assert b2 - b1 == spmv + (3 + 1) * 10 * 4 + 2 * 10 * 4 + 10 * 4


def test_ir_kernel_bytes_scale_with_the_precisions():
    # half-precision u_g and u_p (2 bytes) against single (4): every vector and matrix-value
    # term halves, the column indices and row pointers do not
    n, na, npp, its = 1000, 7000, 25000, [30, 20]
    b4 = bench.ir_kernel_bytes(n, na, npp, its, s_u=4, s_g=4, s_p=4)
    b2 = bench.ir_kernel_bytes(n, na, npp, its, s_u=4, s_g=2, s_p=2)
    b8 = bench.ir_kernel_bytes(n, na, npp, its, s_u=4, s_g=8, s_p=8)
    assert b2 < b4 < b8
    assert b8 - b4 == 2 * (b4 - b2)  # linear in the element size


def test_labels_name_the_grid():
    m, w = bench.labels(64)
    assert m == bench.METRIC and w == bench.WORKLOAD
    m, w = bench.labels(32)
    assert "32^3" in m and "64^3" not in m and "n=32768" in w


def test_backward_error_definition():
    import numpy as np
    import scipy.sparse as sp
    from paper_2202_10204_gb300 import synth
    A = synth.random_sparse(50, 6, seed=3)
    M = synth.to_scipy(A).toarray()
    b = np.random.default_rng(1).normal(size=50)
    # x = 0 leaves the whole of b: ||b|| / ||b|| = 1
    assert bench.backward_error(A, b, np.zeros(50)) == 1.0
    # an exactly representable solution of a diagonal system has no residual
    D = synth._to_csr(sp.diags(np.full(8, 2.0)))
    assert bench.backward_error(D, np.full(8, 3.0), np.full(8, 1.5)) == 0.0
    # the normwise formula with dense numpy, and invariance under power-of-two scaling
    x = np.linalg.solve(M, b) + 1e-6
    ref = np.max(np.abs(b - M @ x)) / (np.max(np.abs(M).sum(axis=1)) * np.max(np.abs(x)) + np.max(np.abs(b)))
    assert abs(bench.backward_error(A, b, x) - ref) <= 1e-12 * ref
    assert bench.backward_error(A, 8.0 * b, 8.0 * x) == bench.backward_error(A, b, x)


def test_batched_512_recipe():
    # 512 systems, n log-uniform in [2e3, 5e4] (2D grids rounded to a square), even ones the
    # 5-point convection-diffusion stencil, odd ones 8-16 nonzeros in every column; seeded
    import numpy as np
    from paper_2202_10204_gb300 import synth
    batch = bench.batched_512_systems(synth)
    assert len(batch) == 512
    ns = np.array([len(A[0]) - 1 for A, _ in batch])
    assert ns.min() >= 1900 and ns.max() <= 50000 and ns.sum() == 8336131
    for i, (A, b) in enumerate(batch):
        n = len(A[0]) - 1
        assert len(b) == n
        if i % 2 == 0:
            N = int(round(np.sqrt(n)))
            assert N * N == n and len(A[1]) == 5 * n - 4 * N
        elif i % 64 == 1:  # column counts of a sample of the random systems
            per_col = np.bincount(A[1], minlength=n)
            assert per_col.min() == per_col.max() and 8 <= per_col[0] <= 16


def test_reference_arm_line_contract():
    # the reference arm times the oracle (CPU): one JSON line with the contract's keys, the
    # same metric labels as the main arm for the grid, a cpu_baseline describing the run and
    # an e2e object with no host-device copies; other ranks exit 0 without work
    import json
    import subprocess
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--grid", "10", "--steps", "2",
           "--warmup", "3"]
    out = subprocess.run(cmd, capture_output=True, text=True, check=True, cwd=ROOT, timeout=600).stdout
    lines = [l for l in out.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "impl", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["steps"] == 2 and d["warmup"] == 3 and d["higher_is_better"] is True
    assert (d["metric"], d["config"]["workload"]) == bench.labels(10) and d["config"]["n"] == 1000
    assert d["value"] > 0 and abs(d["ms_per_step"] * d["steps"] / 1000.0 - 1.0 / d["value"]) < 1e-9 / d["value"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1 and cb["sample"]
    assert d["e2e"] == dict(value=d["value"], unit=d["unit"], h2d_bytes_per_step=0, d2h_bytes_per_step=0)
    env = dict(os.environ, RANK="1", WORLD_SIZE="2")
    r = subprocess.run(cmd, capture_output=True, text=True, cwd=ROOT, env=env, timeout=600)
    assert r.returncode == 0 and not [l for l in r.stdout.splitlines() if l.startswith("{")]
