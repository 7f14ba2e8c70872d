"""Host-side helpers of bench.py: the nvidia-smi clock summary and the
algorithmic-bytes model of the refinement kernel (CPU only)."""
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
