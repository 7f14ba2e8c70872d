"""Benchmark: SPAI-GMRES-IR solves/s on the 64^3 convection-diffusion system.

Workload (one "step" = one full solve: SPAI build on A^T D with pattern(A^2)
plus the whole refinement loop): 3D 7-point convection-diffusion on a 64^3
grid (n = 262144, 1,810,432 nonzeros), per-cell coefficients lognormal(0,1),
Peclet 50 upwind; precisions (u_f,u,u_g,u_p,u_r) = (half, single, single,
single, double); tau = 1e-4; b = A x_true with x_true ~ N(0,1).  Inputs are
seeded and synthetic.  The GMRES solves orthogonalise by modified
Gram-Schmidt in its one-reduction form (ir_opts.orth = 2: MGS in exact
arithmetic, one grid-wide reduction per Arnoldi iteration); the same workload
with the MGS exchange rounds (orth 0) and with CGS2 (orth 1) is reported
beside it, and so is the all-FP64 form of the method.

N > 1 (torchrun): every rank solves its own copy (independent replicas, weak
scaling); no collective is on the data path.

``--impl reference`` times the CPU oracle (the only reference that exists for
this method) on the same 64^3 system: one full oracle solve, split into K
bounded steps (SPAI column slices, then the refinement), on all host cores
(OpenMP over the SPAI columns; the refinement is serial).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "SPAI-GMRES-IR solves/s (64^3 conv-diff, (half,single,single,single,double))"
UNIT = "solves/s"
WORKLOAD = "3D 7-point convection-diffusion 64^3, n=262144, lognormal(0,1) cells, Peclet 50, SPAI pattern(A^2)"


def labels(grid):
    """METRIC and WORKLOAD for a grid^3 run (the defaults at 64^3; other grids only for profiling)."""
    if grid == 64:
        return METRIC, WORKLOAD
    return (METRIC.replace("64^3", "%d^3" % grid),
            WORKLOAD.replace("64^3, n=262144", "%d^3, n=%d" % (grid, grid ** 3)))


TUPLE = dict(uf="half", u="single", ug="single", up="single", ur="double")
FP64 = dict(uf="double", u="double", ug="double", up="double", ur="double")
TAU = 1e-4
MAX_FILL = 25
ORTH = 2  # the headline's Arnoldi: MGS in its one-reduction form


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--grid", type=int, default=64, help="grid points per dimension")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cgs2", action="store_true")
    p.add_argument("--no-extra", action="store_true", help="skip the double-precision, adaptive and serving lines")
    p.add_argument("--sweep", action="store_true",
                   help="instead of the bench line: the eps trade-off of adaptive SPAI against fixed patterns "
                        "and no preconditioner (one JSON line)")
    p.add_argument("--case", default=None, choices=["batched_spai", "half_krylov"],
                   help="instead of the bench line, one run of a single case for profiling: batched_spai = "
                        "two spai_build_batch calls on the 512 systems of the batched line, the first tuning; "
                        "half_krylov = three solves of the grid^3 system with u_g = u_p = half (one JSON line)")
    return p.parse_args()


def batched_512_systems(synth):
    """The 512 systems of the batched line: n log-uniform in [2e3, 5e4], even ones 2D
    convection-diffusion (Peclet U(0, 50)), odd ones random sparse with 8-16 nonzeros per column
    and row/column scaling 10^U(1,3); returns [(A, b)]."""
    rng = np.random.default_rng(4)
    R = 512
    ns = np.exp(rng.uniform(np.log(2e3), np.log(5e4), size=R))
    batch = []
    for i in range(R):
        if i % 2 == 0:
            N = max(8, int(round(np.sqrt(ns[i]))))
            A2 = synth.conv_diff_2d(N, float(rng.uniform(0.0, 50.0)), 1.0, 0.1, seed=1000 + i)
        else:
            A2 = synth.random_sparse(int(ns[i]), int(rng.integers(8, 17)), seed=2000 + i,
                                     log10_scale=float(rng.uniform(1.0, 3.0)))
        b2, _ = synth.rhs(A2, seed=3000 + i)
        batch.append((A2, b2))
    return batch


def run_case(args):
    """One run of a single case (for ncu), printing one JSON line."""
    import paper_2202_10204_gb300 as S
    from paper_2202_10204_gb300 import synth
    if args.case == "half_krylov":
        import torch
        A, b, x_true = synth.cfg_large_3d(N=args.grid)
        ctx = S.Context(0)
        dev = torch.device("cuda:0")
        Ad = tuple(torch.from_numpy(a).to(dev) for a in A)
        bd = torch.from_numpy(b).to(dev)
        so = S.make_spai_opts(init=2, max_fill=MAX_FILL, uf=TUPLE["uf"], eps=0.3)
        io = S.make_ir_opts(tau=1e-2, orth=2, ir_max_steps=30, **dict(TUPLE, ug="half", up="half"))
        P, _ = S.spai_build(ctx, Ad, so)
        sts = []
        for _ in range(3):
            xd = torch.zeros_like(bd)
            sts.append(S.gmres_ir_solve(ctx, Ad, bd, xd, P=P, opts=io))
        torch.cuda.synchronize()
        n, nnz = len(b), len(A[1])
        out = dict(case=args.case, n=n, its=sts[-1]["its"], steps=sts[-1]["steps"],
                   ms_kernel=[s_["ms_kernel"] for s_ in sts],
                   algorithmic_bytes=ir_kernel_bytes(n, nnz, sts[-1]["nnz_P"], sts[-1]["its"], s_u=4, s_g=2, s_p=2))
        P.free()
        ctx.close()
        print(json.dumps(out))
        return 0
    if args.case == "batched_spai":
        batch = batched_512_systems(synth)
        ctx = S.Context(0)
        so = S.make_spai_opts(init=1, max_fill=30, uf="single")
        # the first build also tunes the shared-memory tiles (spai_tune_get); the second is timed
        Ps, sts = S.spai_build_batch(ctx, [A for A, _ in batch], so)
        first_ms = sts[0]["ms"]
        for P in Ps:
            P.free()
        Ps, sts = S.spai_build_batch(ctx, [A for A, _ in batch], so, per_column=True)
        nI = np.concatenate([st["nI"] for st in sts])
        out = dict(case=args.case, columns=int(len(nI)), first_ms=first_ms, ms=sts[0]["ms"], ms_kernel=sts[0]["ms_kernel"],
                   tuned={b: S.tune_get(0, "single", b) for b in range(2, 14)},
                   launches=sts[0]["launches"],
                   shadow_rows={"1-32": int(np.sum(nI <= 32)), "33-64": int(np.sum((nI > 32) & (nI <= 64))),
                                "65-256": int(np.sum((nI > 64) & (nI <= 256))), "257-512": int(np.sum(nI > 256))})
        for P in Ps:
            P.free()
        ctx.close()
        print(json.dumps(out))
    return 0


def nproc():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


# ---------------------------------------------------------------- oracle arm

def oracle_solve_split(grid, parts, threads=0):
    """One full oracle SPAI-GMRES-IR solve of the grid^3 system, in `parts` pieces:
    the SPAI columns in parts-1 slices, then the assembly and the refinement.
    Returns the list of piece durations (s), the refinement result and the
    number of threads the SPAI used."""
    import oracle as O
    from paper_2202_10204_gb300 import synth
    A, b, x = synth.cfg_large_3d(N=grid)
    n = len(A[0]) - 1
    th = O.set_threads(threads)
    F = MAX_FILL
    pieces = max(1, parts - 1)
    bounds = np.linspace(0, n, pieces + 1).astype(np.int64)
    Jcnt = np.zeros(n, dtype=np.int32)
    Jidx = np.full((n, F), -1, dtype=np.int32)
    mbar = np.zeros((n, F))
    d = None
    times = []
    for i in range(pieces):
        cols = np.arange(bounds[i], bounds[i + 1], dtype=np.int32)
        t0 = time.perf_counter()
        if len(cols):
            S = O.spai(A, init=O.PAT_A2, max_fill=F, uf=TUPLE["uf"], eps=0.3, cols=cols)
            Jcnt[cols] = S["Jcnt"][cols]
            Jidx[cols] = S["Jidx"][cols]
            mbar[cols] = S["mbar"][cols]
            d = S["d"]
        times.append(time.perf_counter() - t0)
    t0 = time.perf_counter()
    Sfull = dict(n=n, max_fill=F, d=d, Jcnt=Jcnt, Jidx=Jidx, mbar=mbar)
    P = O.assemble_P(Sfull, TUPLE["up"], TUPLE["uf"])
    R = O.gmres_ir(A, b, P, tau=TAU, orth=ORTH, **TUPLE)
    times.append(time.perf_counter() - t0)
    if parts == 1:
        times = [sum(times)]
    return times, R, th


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle as O
    O.build()
    # warm-up: the same code path on a small system (untimed)
    for _ in range(args.warmup):
        oracle_solve_split(12, 2)
    K = max(1, args.steps)
    times, R, th = oracle_solve_split(args.grid, K)
    tot = float(sum(times))
    value = 1.0 / tot  # exactly one full solve over the K steps
    n_full = args.grid ** 3
    sample = ("one full oracle SPAI-GMRES-IR solve of the %d^3 system (n=%d) split into %d steps: SPAI columns in %d "
              "slices on %d threads (OpenMP), then assembly and the serial refinement (%s iterations); value = 1 / "
              "total time" % (args.grid, n_full, K, max(1, K - 1), th, list(map(int, R["its"]))))
    metric, workload = labels(args.grid)
    line = dict(metric=metric, value=value, unit=UNIT, n_gpus=args.gpus, steps=K, warmup=args.warmup,
                ms_per_step=1000 * tot / K, higher_is_better=True, scaling="weak", vs_baseline=None,
                dtype="f64 (u_f half, u single, u_g/u_p single, u_r double, simulated)", data="synthetic",
                impl="reference",
                config=dict(workload=workload, n=n_full, tuple=TUPLE, tau=TAU, orth=ORTH),
                cpu_baseline=dict(value=value, unit=UNIT, cores=th, kind="oracle", sample=sample,
                                  nproc=nproc()),
                e2e=dict(value=value, unit=UNIT, h2d_bytes_per_step=0, d2h_bytes_per_step=0))
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------- clocks

class ClockSampler:
    def __init__(self, path):
        self.path = path
        self.proc = None

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "--query-gpu=" + q, "--format=csv,noheader,nounits",
                                          "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self, device_index=0):
        try:
            rows = [l.split(",") for l in open(self.path).read().strip().splitlines()]
        except Exception:
            return None
        rows = [[c.strip() for c in r] for r in rows if len(r) >= 9 and r[0].strip() == str(device_index)]
        if not rows:
            return None
        sm = [float(r[1]) for r in rows]
        mx = float(rows[0][2])
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for i, nm in enumerate(names):
                if r[5 + i].lower().startswith("active"):
                    reasons.add(nm)
        return dict(sm_mhz=float(np.median(sm)), sm_max_mhz=mx, reasons=sorted(reasons), samples=len(rows))


# ---------------------------------------------------------------- algorithmic bytes

# DRAM bytes (read + write) of one k_ir launch (one-reduction MGS) on the 64^3 workload, from one
# ncu capture of the current kernel build (dram__bytes_read.sum + dram__bytes_write.sum, one pass,
# a timed launch): 4.24 GB read + 0.22 GB written against 13.6 GB algorithmic; A, P and the
# recent basis vectors are served from L2.
K_IR_DRAM_BYTES_64CUBE = 4.464e9


def ir_kernel_bytes(n, nnz_a, nnz_p, its, s_u=4, s_g=4, s_p=4):
    """Algorithmic HBM bytes of one refinement-kernel launch: every matrix and
    vector the method reads or writes, counted once per use.

    Per Arnoldi iteration j: SpMV A (values in u_p + int32 cols + int64 rowptr,
    read v, write t), SpMV P (same, read t), MGS (read V(:,0..j) once, write
    v_{j+1} and the published w).  Per refinement step: residual (A in fp64,
    b, x, r), z = P r, correction d = V y (read V(:,0..k-1), x in and out).
    The final residual evaluation is included.
    """
    rp = (n + 1) * 8
    spmv_a = nnz_a * (s_p + 4) + rp + n * s_g + n * s_p
    spmv_p = nnz_p * (s_p + 4) + rp + n * s_p
    resid = nnz_a * (8 + 4) + rp + n * 8 + n * s_u + n * s_u
    total = resid  # the last residual (the stop test)
    for k in its:
        total += resid + nnz_p * (s_p + 4) + rp + n * s_u + n * s_g
        for j in range(k):
            total += spmv_a + spmv_p + (j + 1) * n * s_g + 2 * n * s_g
        total += k * n * s_g + 2 * n * s_u
    return total


# ---------------------------------------------------------------- multi-rank aggregation

def max_over_ranks(value, dist=None, device="cpu"):
    """Largest value over all ranks (the slowest rank's time); identity at N = 1."""
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    if dist is not None and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world, steps, max_ms):
    """Whole-job solves/s: every rank solves `steps` systems; time is the slowest rank's."""
    return world * steps / (max_ms / 1000.0)


# ---------------------------------------------------------------- other workloads (reported beside the headline)

def backward_error(A, b, x):
    """Normwise backward error max|b - A x| / (||A||_inf max|x| + max|b|) in float64."""
    import scipy.sparse as sp
    rp, ci, va = A
    n = len(rp) - 1
    M = sp.csr_matrix((va, ci, rp), shape=(n, n))
    r = b - M @ x
    return float(np.max(np.abs(r)) / (abs(M).sum(axis=1).max() * np.max(np.abs(x)) + np.max(np.abs(b))))


def serve_stream(S, dev, reqs, arrivals, so, io, budget=120 << 30):
    """Submit reqs[i] = (A, b) at arrivals[i] (seconds) to a serving context and poll
    until all are done; returns (latencies in ms = completion - arrival, makespan s,
    largest backward error of the solutions)."""
    sctx = S.Context(dev.index or 0, hbm_budget=budget)
    # warm the workers and kernels
    t = S.solver_submit(sctx, reqs[0][0], reqs[0][1], so, io)
    while S.solver_poll(sctx, t) is None:
        time.sleep(0.001)
    R = len(reqs)
    pending = {}
    lat = [None] * R
    xs = [None] * R
    t0 = time.perf_counter()
    nxt = 0
    while nxt < R or pending:
        now = time.perf_counter() - t0
        while nxt < R and arrivals[nxt] <= now:
            pending[nxt] = S.solver_submit(sctx, reqs[nxt][0], reqs[nxt][1], so, io)
            nxt += 1
        for i in list(pending):
            xs[i] = np.zeros(len(reqs[i][1]))
            stt = S.solver_poll(sctx, pending[i], xs[i])
            if stt is not None:
                lat[i] = (time.perf_counter() - t0) - arrivals[i]
                del pending[i]
        time.sleep(0.0002)
    makespan = time.perf_counter() - t0
    sctx.close()
    nbe = max(backward_error(A, b, xs[i]) for i, (A, b) in enumerate(reqs))
    return np.array(lat) * 1000.0, makespan, nbe


def extra_workloads(S, synth, torch, dev):
    """Five secondary lines, each bounded to a few seconds:
    * u = double: the 32x32 2D system with (single, double, double, double, quad), the
      configuration whose backward error must reach 1e-15;
    * right: the 64^3 workload with the right SPAI (A P ~ I) and right-preconditioned GMRES;
    * adaptive: Grote-Huckle SPAI from the identity on a 100,000-column random nonsymmetric
      matrix (16 nonzeros per column, row/column scaling 1e6), eps 0.5, beta 8, fill cap 30,
      u_f single, then the solve with (single, double, double, double, quad);
    * serving: Poisson streams at 10, 30, 100, 300, 1000 and 2000 requests/s of 3D systems
      (n log-uniform in [1e3, 1e6]) into a context with a 120 GB admission budget, in the
      mixed tuple and in the all-FP64 form; latency = completion - arrival;
    * batched: 512 independent systems (half 2D convection-diffusion, half random sparse,
      n log-uniform in [2e3, 5e4]): spai_build_batch and gmres_ir_solve_batch (refinements in shared
      cooperative launches), beside the same systems submitted at once to the serving queue."""
    import numpy as np
    out = {}
    stream = torch.cuda.current_stream()
    ctx = S.Context(dev.index or 0, stream=stream)
    # ---- u = double
    A, b, xt = synth.cfg_small_2d()
    Ad = tuple(torch.from_numpy(a).to(dev) for a in A)
    bd = torch.from_numpy(b).to(dev)
    xd = torch.zeros_like(bd)
    so = S.make_spai_opts(init=1, max_fill=30, uf="single")
    io = S.make_ir_opts(uf="single", u="double", ug="double", up="double", ur="quad", tau=1e-4)
    for _ in range(3):
        S.gmres_ir_solve(ctx, Ad, bd, xd, sopts=so, opts=io)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 20
    e0.record(stream)
    for _ in range(reps):
        st = S.gmres_ir_solve(ctx, Ad, bd, xd, sopts=so, opts=io)
    e1.record(stream)
    torch.cuda.synchronize()
    Ms = synth.to_scipy(A)
    x = xd.cpu().numpy()
    nbe = float(np.max(np.abs(b - Ms @ x)) / (abs(Ms).sum(axis=1).max() * np.max(np.abs(x)) + np.max(np.abs(b))))
    out["double_2d"] = dict(workload="2D conv-diff 32x32 (n=1024), Peclet 10, pattern(A), "
                                     "(single,double,double,double,quad), tau 1e-4",
                            solves_per_s=reps / (e0.elapsed_time(e1) / 1000.0), backward_error=nbe,
                            its=st["its"], steps=st["steps"])
    # ---- right preconditioning on the 64^3 workload (SPAI with A P ~ I, GMRES on A P)
    A, b, xt = synth.cfg_large_3d(N=64)
    Ad = tuple(torch.from_numpy(a).to(dev) for a in A)
    bd = torch.from_numpy(b).to(dev)
    xd = torch.zeros_like(bd)
    so = S.make_spai_opts(init=2, max_fill=25, uf="half", eps=0.3, side=S.SIDE_RIGHT)
    io = S.make_ir_opts(uf="half", u="single", ug="single", up="single", ur="double", tau=1e-4, side=S.SIDE_RIGHT,
                        orth=ORTH)
    for _ in range(2):
        S.gmres_ir_solve(ctx, Ad, bd, xd, sopts=so, opts=io)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 5
    e0.record(stream)
    for _ in range(reps):
        st = S.gmres_ir_solve(ctx, Ad, bd, xd, sopts=so, opts=io)
    e1.record(stream)
    torch.cuda.synchronize()
    Ms = synth.to_scipy(A)
    x = xd.cpu().numpy()
    nbe = float(np.max(np.abs(b - Ms @ x)) / (abs(Ms).sum(axis=1).max() * np.max(np.abs(x)) + np.max(np.abs(b))))
    out["right_64cube"] = dict(workload="the 64^3 workload with the right SPAI (A P ~ I) and right-preconditioned "
                                        "GMRES (one-reduction MGS); spai_build + solve per step, device inputs",
                               solves_per_s=reps / (e0.elapsed_time(e1) / 1000.0), its=st["its"], steps=st["steps"],
                               backward_error=nbe, ms_spai=st["ms_spai"], ms_ir=st["ms_ir"])
    # ---- adaptive
    A = synth.random_sparse(100_000, 16, seed=6, log10_scale=6.0)
    b, xt = synth.rhs(A, seed=7)
    Ad = tuple(torch.from_numpy(a).to(dev) for a in A)
    bd = torch.from_numpy(b).to(dev)
    xd = torch.zeros_like(bd)
    so = S.make_spai_opts(init=0, adaptive=True, eps=0.5, beta=8, max_fill=30, uf="single")
    io = S.make_ir_opts(uf="single", u="double", ug="double", up="double", ur="quad", tau=1e-8, orth=ORTH)
    io0 = S.make_ir_opts(uf="single", u="double", ug="double", up="double", ur="quad", tau=1e-8, orth=0)
    P, sst = S.spai_build(ctx, Ad, so)
    P.free()
    P, sst = S.spai_build(ctx, Ad, so)
    torch.cuda.synchronize()
    st = S.gmres_ir_solve(ctx, Ad, bd, xd, P=P, opts=io)
    x = xd.cpu().numpy()
    Ms = synth.to_scipy(A)
    nbe = float(np.max(np.abs(b - Ms @ x)) / (abs(Ms).sum(axis=1).max() * np.max(np.abs(x)) + np.max(np.abs(b))))
    st0 = S.gmres_ir_solve(ctx, Ad, bd, xd, P=P, opts=io0)  # the textbook MGS rounds, for context
    out["adaptive_100k"] = dict(workload="random nonsymmetric n=100000, 16 nnz/col, scaling 1e6; adaptive "
                                          "SPAI eps 0.5, beta 8, cap 30, u_f single; (single,double,double,double,quad), "
                                          "tau 1e-8, one-reduction MGS (ir_ms_mgs_rounds: the textbook MGS)",
                                spai_ms=sst["ms"], spai_cols_per_s=100_000 / (sst["ms"] / 1000.0),
                                nnz_P=sst["nnz_P"], cols_converged=sst["cols_converged"],
                                cols_fillcap=sst["cols_fillcap"], ir_ms=st["ms_ir"], its=st["its"],
                                steps=st["steps"], backward_error=nbe, ir_ms_mgs_rounds=st0["ms_ir"],
                                its_mgs_rounds=st0["its"])
    P.free()
    ctx.close()
    # ---- serving: Poisson streams at 10..2000 requests/s of 3D systems with n log-uniform in
    # [1e3, 1e6], the mixed tuple and the all-FP64 form, 120 GB admission budget
    rng = np.random.default_rng(5)
    pool = []
    for i, N in enumerate(np.round(np.exp(rng.uniform(np.log(10), np.log(100), size=32))).astype(int)):
        A3 = synth.conv_diff_3d(int(N), 50.0, seed=100 + i)
        b3, _ = synth.rhs(A3, seed=200 + i)
        pool.append((A3, b3))
    so = S.make_spai_opts(init=2, max_fill=25, uf="half", eps=0.3)
    io = S.make_ir_opts(uf="half", u="single", ug="single", up="double", ur="double", tau=1e-4, orth=2)
    so64 = S.make_spai_opts(init=2, max_fill=25, uf="double", eps=0.3)
    io64 = S.make_ir_opts(uf="double", u="double", ug="double", up="double", ur="double", tau=1e-4, orth=2)
    sweep = []
    for rate in (10.0, 30.0, 100.0, 300.0, 1000.0, 2000.0):
        R = int(min(96, max(16, 2.0 * rate)))
        arrivals = np.cumsum(rng.exponential(1.0 / rate, size=R))
        reqs = [pool[int(j)] for j in rng.integers(0, len(pool), size=R)]
        lat, makespan, nbe = serve_stream(S, dev, reqs, arrivals, so, io)
        lat64, makespan64, nbe64 = serve_stream(S, dev, reqs, arrivals, so64, io64)
        sweep.append(dict(rate=rate, requests=R, sum_n=int(sum(len(b3) for _, b3 in reqs)),
                          solves_per_s=R / makespan, p50_ms=float(np.percentile(lat, 50)),
                          p99_ms=float(np.percentile(lat, 99)), backward_error_max=nbe,
                          fp64=dict(solves_per_s=R / makespan64, p50_ms=float(np.percentile(lat64, 50)),
                                    p99_ms=float(np.percentile(lat64, 99)), backward_error_max=nbe64),
                          mixed_over_fp64=makespan64 / makespan))
    out["serving"] = dict(workload="Poisson streams at 10..2000 requests/s (16..96 requests each), 3D conv-diff "
                                   "(Peclet 50, lognormal coefficients) grids 10^3..100^3 (n log-uniform in "
                                   "[1e3, 1e6], 32 distinct systems), pattern(A^2) cap 25, one-reduction MGS, "
                                   "(half,single,single,double,double) against (double x5), budget 120 GB, "
                                   "host inputs; latency = completion - arrival",
                          sweep=sweep)
    out["fp64_serving"] = dict(workload="the serving sweep's streams in the all-FP64 form (double x5)",
                               sweep=[dict(rate=w["rate"], solves_per_s=w["fp64"]["solves_per_s"],
                                           p50_ms=w["fp64"]["p50_ms"], p99_ms=w["fp64"]["p99_ms"],
                                           backward_error_max=w["fp64"]["backward_error_max"],
                                           mixed_over_fp64=w["mixed_over_fp64"]) for w in sweep])
    # ---- batched: 512 independent systems through the queue at once
    batch = batched_512_systems(synth)
    R = len(batch)
    so = S.make_spai_opts(init=1, max_fill=30, uf="single")
    io = S.make_ir_opts(uf="single", u="double", ug="single", up="single", ur="double", tau=1e-4, orth=ORTH)
    # warm-up build of the whole batch (untimed): the first build with enough columns per bin
    # also times the tile shapes (the tuner, whose choice the process keeps), a one-time cost
    # reported apart as first_build_s
    wctx = S.Context(dev.index or 0)
    torch.cuda.synchronize()
    tw = time.perf_counter()
    Ps, _ = S.spai_build_batch(wctx, [A2 for A2, _ in batch], so)
    first_build_s = time.perf_counter() - tw
    for P_ in Ps:
        P_.free()
    wctx.close()
    bctx = S.Context(dev.index or 0, hbm_budget=120 << 30)
    t = S.solver_submit(bctx, batch[0][0], batch[0][1], so, io)
    while S.solver_poll(bctx, t) is None:
        time.sleep(0.001)
    t0 = time.perf_counter()
    tickets = [S.solver_submit(bctx, A2, b2, so, io) for A2, b2 in batch]
    done, conv, its = {}, 0, 0
    while len(done) < R:
        for i, tk in enumerate(tickets):
            if i in done:
                continue
            stt = S.solver_poll(bctx, tk, np.zeros(len(batch[i][1])))
            if stt is not None:
                done[i] = time.perf_counter() - t0
                conv += int(stt["flags"] & 1)
                its += stt["total_its"]
        time.sleep(0.0005)
    makespan = time.perf_counter() - t0
    bctx.close()
    sum_n = int(sum(len(a[0]) - 1 for a, _ in batch))
    queue = dict(solves_per_s=R / makespan, makespan_s=makespan, converged=conv, total_its=its,
                 p50_ms=float(np.percentile(list(done.values()), 50) * 1000.0),
                 p99_ms=float(np.percentile(list(done.values()), 99) * 1000.0))
    # the same systems through spai_build_batch (concurrent builds) and gmres_ir_solve_batch (all
    # refinements in shared cooperative launches); host inputs and outputs, copies timed
    bctx = S.Context(dev.index or 0)
    Pw, _ = S.spai_build(bctx, batch[0][0], so)
    S.gmres_ir_solve_batch(bctx, [batch[0][0]], [batch[0][1]], [np.zeros(len(batch[0][1]))], [Pw], io)
    Pw.free()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    Ps, _ = S.spai_build_batch(bctx, [A2 for A2, _ in batch], so)
    t1 = time.perf_counter()
    xs = [np.zeros(len(b2)) for _, b2 in batch]
    sts, status = S.gmres_ir_solve_batch(bctx, [A2 for A2, _ in batch], [b2 for _, b2 in batch], xs, Ps, io)
    t2 = time.perf_counter()
    for P_ in Ps:
        P_.free()
    bctx.close()
    batch_api = dict(solves_per_s=R / (t2 - t0), makespan_s=t2 - t0, spai_s=t1 - t0, refinement_s=t2 - t1,
                     first_build_s=first_build_s,
                     spai_cols_per_s=sum(len(b2) for _, b2 in batch) / (t1 - t0),
                     refinement_launches=int(sts[0]["launches"]), converged=int(sum(int(st_["flags"] & 1) for st_ in sts)),
                     total_its=int(sum(st_["total_its"] for st_ in sts)),
                     backward_error_max=max(backward_error(A2, b2, x2) for (A2, b2), x2 in zip(batch, xs)))
    # the same systems in the all-FP64 form (every precision double)
    so64 = S.make_spai_opts(init=1, max_fill=30, uf="double")
    io64 = S.make_ir_opts(uf="double", u="double", ug="double", up="double", ur="double", tau=1e-4, orth=ORTH)
    bctx = S.Context(dev.index or 0)
    Ps, _ = S.spai_build_batch(bctx, [A2 for A2, _ in batch], so64)  # warm-up (tuner at u_f = double)
    for P_ in Ps:
        P_.free()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    Ps, _ = S.spai_build_batch(bctx, [A2 for A2, _ in batch], so64)
    t1 = time.perf_counter()
    xs = [np.zeros(len(b2)) for _, b2 in batch]
    sts64, _ = S.gmres_ir_solve_batch(bctx, [A2 for A2, _ in batch], [b2 for _, b2 in batch], xs, Ps, io64)
    t2 = time.perf_counter()
    for P_ in Ps:
        P_.free()
    bctx.close()
    fp64_batch = dict(solves_per_s=R / (t2 - t0), makespan_s=t2 - t0, spai_s=t1 - t0, refinement_s=t2 - t1,
                      converged=int(sum(int(st_["flags"] & 1) for st_ in sts64)),
                      total_its=int(sum(st_["total_its"] for st_ in sts64)),
                      backward_error_max=max(backward_error(A2, b2, x2) for (A2, b2), x2 in zip(batch, xs)),
                      mixed_over_fp64=(R / batch_api["makespan_s"]) / (R / (t2 - t0)))
    out["batched_512"] = dict(workload="512 systems, n log-uniform in [2e3, 5e4]: even = 2D conv-diff (Peclet "
                                       "U(0,50)), odd = random sparse 8-16 nnz/col with row/column scaling "
                                       "10^U(1,3) (cond_1 ~1e2-5e3); pattern(A), (single,double,single,single,double), tau 1e-4, "
                                       "one-reduction MGS, "
                                       "host inputs; value = gmres_ir_solve_batch path, serving_queue = all submitted to the queue at once",
                              systems=R, solves_per_s=batch_api["solves_per_s"],
                              cols_per_s=sum_n / batch_api["makespan_s"], sum_n=sum_n,
                              batch_api=batch_api, serving_queue=queue, fp64_batch_api=fp64_batch)
    out["fp64_batched"] = dict(workload="the 512 systems of batched_512 in the all-FP64 form (double x5), "
                                        "spai_build_batch + gmres_ir_solve_batch", **fp64_batch)
    return out


def run_sweep(args):
    """The paper's trade-off between the SPAI stopping tolerance eps, the fill of P and the GMRES
    iterations (its Section 5 discussion and figures), on two synthetic stand-ins: adaptive SPAI
    from the identity for eps in 0.1..0.9 against the fixed patterns pattern(A), pattern(A^2) and
    against no preconditioner.  Per run: nnz(P)/n, the refinement steps and GMRES iterations, the
    final backward error, SPAI and refinement milliseconds (CUDA events of the library)."""
    import numpy as np
    import torch

    import paper_2202_10204_gb300 as S
    from paper_2202_10204_gb300 import synth
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream()
    ctx = S.Context(0, stream=stream)
    cases = [
        ("3D conv-diff 32^3 (n=32768), Peclet 50, (half,single,single,single,double), tau 1e-4",
         synth.conv_diff_3d(32, 50.0, seed=3), dict(uf="half", u="single", ug="single", up="single", ur="double",
                                                    tau=1e-4), "half"),
        ("random nonsymmetric n=20000, 12 nnz/col, scaling 1e3, (single,double,single,single,double), tau 1e-4",
         synth.random_sparse(20000, 12, seed=31, log10_scale=3.0),
         dict(uf="single", u="double", ug="single", up="single", ur="double", tau=1e-4), "single"),
    ]
    out = []
    for name, A, io_kw, uf in cases:
        b, xt = synth.rhs(A, seed=5)
        n = len(A[0]) - 1
        Ad = tuple(torch.from_numpy(a).to(dev) for a in A)
        bd = torch.from_numpy(b).to(dev)
        io = S.make_ir_opts(**io_kw)
        Ms = synth.to_scipy(A)
        runs = []
        configs = [("none", None)]
        configs += [("pattern(A)", S.make_spai_opts(init=1, max_fill=30, uf=uf))]
        configs += [("pattern(A^2)", S.make_spai_opts(init=2, max_fill=30, uf=uf))]
        for eps in (0.1, 0.2, 0.3, 0.4, 0.5, 0.6, 0.7, 0.8, 0.9):
            configs.append(("adaptive eps=%.1f" % eps,
                            S.make_spai_opts(init=0, adaptive=True, eps=eps, beta=8, max_fill=30, uf=uf)))
        for label, so in configs:
            P, sst = (None, None)
            if so is not None:
                P, sst = S.spai_build(ctx, Ad, so)
            xd = torch.zeros_like(bd)
            st = S.gmres_ir_solve(ctx, Ad, bd, xd, P=P, opts=io)
            x = xd.cpu().numpy()
            nbe = float(np.max(np.abs(b - Ms @ x)) / (abs(Ms).sum(axis=1).max() * np.max(np.abs(x)) + np.max(np.abs(b))))
            runs.append(dict(precond=label, nnz_P_per_n=(sst["nnz_P"] / n) if sst else 0.0,
                             cols_converged=sst["cols_converged"] if sst else None,
                             steps=st["steps"], its=st["its"], total_its=st["total_its"], backward_error=nbe,
                             spai_ms=sst["ms"] if sst else 0.0, ir_ms=st["ms_ir"]))
            if P is not None:
                P.free()
        out.append(dict(workload=name, n=n, runs=runs))
    ctx.close()
    print(json.dumps(dict(sweep="eps trade-off", data="synthetic", cases=out)))
    return 0


# ---------------------------------------------------------------- GPU arm

def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.case:
        return run_case(args)
    if args.sweep:
        return run_sweep(args)
    import torch
    import torch.distributed as dist

    import paper_2202_10204_gb300 as S
    from paper_2202_10204_gb300 import synth

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()

    A, b, x_true = synth.cfg_large_3d(N=args.grid)
    n = len(A[0]) - 1
    nnz = len(A[1])
    Ad = tuple(torch.from_numpy(a).to(dev) for a in A)
    bd = torch.from_numpy(b).to(dev)
    xd = torch.zeros_like(bd)
    ctx = S.Context(local, stream=stream)
    so = S.make_spai_opts(init=2, max_fill=MAX_FILL, uf=TUPLE["uf"], eps=0.3)
    io = S.make_ir_opts(tau=TAU, orth=ORTH, **TUPLE)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)

    def step():
        P, sst = S.spai_build(ctx, Ad, so)
        st = S.gmres_ir_solve(ctx, Ad, bd, xd, P=P, opts=io)
        P.free()
        st["ms_spai"] = sst["ms"]
        st["ms_spai_kernel"] = sst["ms_kernel"]
        st["launches"] += sst["launches"]
        return st

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    stats = []
    # nvidia-smi samples during the timed steps; BENCH_CLOCKS_DIR keeps the raw file
    clk_dir = os.environ.get("BENCH_CLOCKS_DIR") or tempfile.gettempdir()
    clk_path = os.path.join(clk_dir, "clocks_rank%d.csv" % rank)
    os.makedirs(clk_dir, exist_ok=True)
    with ClockSampler(clk_path) as cs:
        time.sleep(0.3)
        for i in range(args.steps):
            flush.zero_()  # L2 flush between timed steps (outside the events)
            ev[i][0].record(stream)
            stats.append(step())
            ev[i][1].record(stream)
        torch.cuda.synchronize()
    per = [e0.elapsed_time(e1) for e0, e1 in ev]
    tot_ms = float(sum(per))
    if world > 1:
        dist.barrier()
    tot_max = max_over_ranks(tot_ms, dist if world > 1 else None, dev)
    value = job_throughput(world, args.steps, tot_max)

    # correctness of the timed solves (the metric counts solves meeting the accuracy bar)
    x = xd.cpu().numpy()
    Ms = synth.to_scipy(A)
    nbe = float(np.max(np.abs(b - Ms @ x)) / (abs(Ms).sum(axis=1).max() * np.max(np.abs(x)) + np.max(np.abs(b))))
    fe = float(np.max(np.abs(x - x_true)) / np.max(np.abs(x_true)))
    last = stats[-1]

    # dominant kernel roofline: the persistent refinement kernel (HBM-bound)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    peak_src = "measured" if "hbm_gbs" in peaks else "fallback"
    ir_ms = [s["ms_kernel"] for s in stats]
    ir_bytes = [ir_kernel_bytes(n, nnz, s["nnz_P"], s["its"]) for s in stats]
    achieved = float(np.mean([b_ / (m / 1000.0) for b_, m in zip(ir_bytes, ir_ms)]) / 1e9)
    spai_ms = float(np.mean([s["ms_spai"] for s in stats]))
    launches = int(sum(s["launches"] for s in stats))
    lat = np.array(per)

    # end to end through the public API with pinned host buffers
    e2e = None
    if not args.no_e2e:
        Ah = tuple(torch.from_numpy(a).pin_memory() for a in A)
        bh = torch.from_numpy(b).pin_memory()
        xh = torch.zeros_like(bh).pin_memory()
        S.gmres_ir_solve(ctx, Ah, bh, xh, sopts=so, opts=io)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        ke = max(1, min(args.steps, 5))
        # each solve timed on its own, the L2 flushed between them (outside the events), as
        # for the device-resident steps
        ev_e = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(ke)]
        for i in range(ke):
            flush.zero_()
            ev_e[i][0].record(stream)
            S.gmres_ir_solve(ctx, Ah, bh, xh, sopts=so, opts=io)
            ev_e[i][1].record(stream)
        torch.cuda.synchronize()
        te = max_over_ranks(sum(a_.elapsed_time(b_) for a_, b_ in ev_e), dist if world > 1 else None, dev)
        h2d = sum(a.numel() * a.element_size() for a in Ah) + bh.numel() * 8
        e2e = dict(value=job_throughput(world, ke, te), unit=UNIT, h2d_bytes_per_step=int(h2d),
                   d2h_bytes_per_step=int(n * 8 + 4 * 2), steps=ke, l2="flushed between solves")

    # the other Arnoldi options on the same workload: MGS with one exchange round per
    # projection (orth 0, the library's default), and classical Gram-Schmidt twice (orth 1);
    # then the all-FP64 form of the method (every precision double) on the same inputs
    variants = {}
    q_row = int(np.max(np.diff(A[0])))
    # u_g = u_p = half (half storage, binary32 arithmetic; tau ~ sqrt(u_half)) beside them
    half_k = dict(TUPLE, ug="half", up="half")
    for name, orth, tup, stol, tau2 in (("arnoldi_mgs_rounds", 0, TUPLE, 0.0, TAU), ("arnoldi_cgs2", 1, TUPLE, 0.0, TAU),
                                        ("fp64_64cube", ORTH, FP64, 0.0, TAU),
                                        ("fp64_64cube_mixed_stop", ORTH, FP64, q_row * 2.0 ** -24, TAU),
                                        ("half_krylov_64cube", 2, half_k, 0.0, 1e-2)):
        if args.no_cgs2:
            break
        io2 = S.make_ir_opts(tau=tau2, orth=orth, stop_tol=stol, ir_max_steps=30, **tup)
        so2 = so if tup["uf"] == TUPLE["uf"] else S.make_spai_opts(init=2, max_fill=MAX_FILL, uf=tup["uf"], eps=0.3)

        def step2():
            P, sst = S.spai_build(ctx, Ad, so2)
            st = S.gmres_ir_solve(ctx, Ad, bd, xd, P=P, opts=io2)
            P.free()
            st["ms_spai"] = sst["ms"]
            return st

        for _ in range(max(1, args.warmup)):
            step2()
        torch.cuda.synchronize()
        ev2 = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        st2 = []
        for i in range(args.steps):
            flush.zero_()
            ev2[i][0].record(stream)
            st2.append(step2())
            ev2[i][1].record(stream)
        torch.cuda.synchronize()
        t2 = max_over_ranks(sum(e0.elapsed_time(e1) for e0, e1 in ev2), dist if world > 1 else None, dev)
        x2 = xd.cpu().numpy()
        nbe2 = float(np.max(np.abs(b - Ms @ x2)) / (abs(Ms).sum(axis=1).max() * np.max(np.abs(x2)) + np.max(np.abs(b))))
        kms = [s["ms_kernel"] for s in st2]
        nb = {"half": 2, "single": 4, "double": 8}
        sz = dict(s_u=nb[tup["u"]], s_g=nb[tup["ug"]], s_p=nb[tup["up"]])
        kbytes = [ir_kernel_bytes(n, nnz, s["nnz_P"], s["its"], **sz) for s in st2]
        ach = float(np.mean([b_ / (m / 1000.0) for b_, m in zip(kbytes, kms)]) / 1e9)
        variants[name] = dict(value=job_throughput(world, args.steps, t2), unit=UNIT, ms_per_step=t2 / args.steps,
                              ir_kernel_ms=float(np.mean(kms)), its=st2[-1]["its"], steps=st2[-1]["steps"],
                              backward_error=nbe2, tuple=tup, orth=orth, tau=tau2,
                              roofline=dict(kernel="k_ir (orth=%d)" % orth, bound="hbm", achieved=ach,
                                            peak=hbm_peak, unit="GB/s", frac=ach / hbm_peak,
                                            algorithmic_bytes_per_launch=float(np.mean(kbytes))))
    if "fp64_64cube" in variants:
        variants["fp64_64cube"]["workload"] = ("the 64^3 workload with every precision double (the all-FP64 form), "
                                               "same pattern, eps, tau and Arnoldi; stop at q u_double")
        variants["fp64_64cube"]["mixed_over_fp64"] = value / variants["fp64_64cube"]["value"]
        variants["fp64_64cube_mixed_stop"]["workload"] = ("the all-FP64 form stopped at the mixed form's backward-error "
                                                          "tolerance q u_single (the same accuracy target)")
        variants["fp64_64cube_mixed_stop"]["mixed_over_fp64"] = value / variants["fp64_64cube_mixed_stop"]["value"]
    if "half_krylov_64cube" in variants:
        variants["half_krylov_64cube"]["workload"] = (
            "the 64^3 workload with u_g = u_p = half (Krylov vectors and the SELL copies of A and P in half, "
            "binary32 arithmetic, residual scaled by a power of two), tau 1e-2, one-reduction MGS; stop at q u_single")
        variants["half_krylov_64cube"]["over_headline"] = variants["half_krylov_64cube"]["value"] / value

    extra = {}
    if world == 1 and not args.no_extra:
        extra = extra_workloads(S, synth, torch, dev)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        try:
            import oracle as O
            O.build()
            # one full oracle solve of this very system on all host cores (OpenMP over the
            # SPAI columns; the refinement is serial)
            times, R, th = oracle_solve_split(args.grid, 1)
            # one thread: the SPAI columns/s on a sample of 8192 columns of the same matrix
            O.set_threads(1)
            cols = np.sort(np.random.default_rng(0).choice(n, size=min(n, 8192), replace=False)).astype(np.int32)
            t0 = time.perf_counter()
            O.spai(A, init=O.PAT_A2, max_fill=MAX_FILL, uf=TUPLE["uf"], eps=0.3, cols=cols)
            t1 = time.perf_counter()
            O.set_threads(0)
            cpu = dict(value=1.0 / times[0], unit=UNIT, cores=th, kind="oracle", nproc=nproc(),
                       sample="one full oracle solve of this %d^3 system (n=%d) on %d threads (OpenMP over the SPAI "
                              "columns, serial refinement): %.1f s, %s iterations" %
                              (args.grid, n, th, times[0], list(map(int, R["its"]))),
                       one_thread_spai_cols_per_s=len(cols) / (t1 - t0),
                       one_thread_sample="SPAI of 8192 sampled columns of the same matrix on 1 thread")
        except Exception as e:  # the baseline is reported, never required
            cpu = dict(value=None, unit=UNIT, cores=0, kind="oracle", sample="failed: %s" % e)

    clocks = cs.summary(local)
    if rank == 0:
        line = dict(
            metric=labels(args.grid)[0], value=value, unit=UNIT, n_gpus=world, steps=args.steps, warmup=args.warmup,
            ms_per_step=tot_max / args.steps, higher_is_better=True, scaling="weak", vs_baseline=None,
            dtype="f16/f32 (u_f half; u, u_g, u_p single; u_r double)", data="synthetic",
            config=dict(workload=labels(args.grid)[1], n=n, nnz=nnz, nnz_P=int(last["nnz_P"]), tuple=TUPLE, tau=TAU,
                        max_fill=MAX_FILL, orth=ORTH, arnoldi="modified Gram-Schmidt, one-reduction form",
                        l2="flushed between timed steps (256 MiB write)",
                        parallelism="replicas" if world > 1 else "single GPU"),
            latency_ms=dict(p50=float(np.percentile(lat, 50)), p99=float(np.percentile(lat, 99))),
            spai_cols_per_s=n / (spai_ms / 1000.0),
            phases_ms=dict(spai_build=spai_ms, spai_column_kernel=float(np.mean([s["ms_spai_kernel"] for s in stats])),
                           ir_total=float(np.mean([s["ms_ir"] for s in stats])),
                           ir_kernel=float(np.mean(ir_ms))),
            ir=dict(steps=last["steps"], its=last["its"], total_its=last["total_its"], grid=last["grid"],
                    backward_error=nbe, forward_error=fe, nbe_trace=last["nbe"]),
            roofline=dict(kernel="k_ir (persistent refinement kernel, orth=%d)" % ORTH, bound="hbm", achieved=achieved,
                          peak=hbm_peak, unit="GB/s", frac=achieved / hbm_peak,
                          traffic=K_IR_DRAM_BYTES_64CUBE if args.grid == 64 else None,
                          peak_source=peak_src, algorithmic_bytes_per_launch=float(np.mean(ir_bytes))),
            gpu_launches=launches,
            **variants,
            **extra,
            clocks=clocks,
            e2e=e2e,
            cpu_baseline=cpu,
        )
        print(json.dumps(line))
    ctx.close()
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
