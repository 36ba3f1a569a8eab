"""CQRRPT benchmark on GB300: one step = one full CQRRPT factorisation (sketch,
QRCP of the sketch, rank, M^pre TRSM, Gram, Cholesky, Q TRSM, TRMM) of the
plain-FP64 rank-deficient workload m = 131072, n = 1024, planted rank 800
(singular values 1 -> 1e-6 geometric, zero after, plus 1e-15 Gaussian noise;
SASO d = 1.25 n = 1280 with 8 nonzeros per column; tol 1e-9).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  `value` is factorisations/s over all ranks
with A resident in HBM; `e2e` is the same metric through the public API with
host buffers (pinned host -> device copy of A, device -> host copy of Q, R,
J, k every step), measured through cqrrpt_host_pipeline_d, whose copies
overlap the factorisations of neighbouring steps.  Under torchrun each rank
factors its own independent problem (the factorisations do not exchange
data): weak scaling, no collective on the data path.  At N = 1 the line also
carries `configs`: the small (4096 x 64) latency case, the mixed-precision
case (2^20 x 512), the 512-problem batch and a shortened serving run,
measured in the same run (--configs none leaves them out).
`--impl reference` times the CPU oracle on the full headline workload, one
of its eight phases per step (OracleSteps).
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402
import torch  # noqa: E402

import workloads as W  # noqa: E402

# FP64 peak of GB300 for an ALU-bound FP64 kernel: 152 SMs x 2 DFMA/clk x
# 2 flop x 2.070 GHz (nominal 1.25 TFLOP/s at the maximum SM clock).
FP64_PEAK_GFLOPS = 152 * 2 * 2 * 2.070
# measured dense bf16 peak of the GB300s (cuBLAS, burst)
BF16_PEAK_TFLOPS = 1968.7
# DRAM bytes of one trsm_rut_kernel launch of the headline factorisation
# (m = 131072, n = 1024, k = 800): dram__bytes_read.sum + dram__bytes_write.sum
# = 10.452 GB + 0.834 GB from one ncu capture of this bench command (one-pass
# metrics, lines 4 and 7 alike; profiles/ncu_trsm_traffic_m131072_n1024.md).
# Valid for that size and the kernel as captured; None otherwise.
TRSM_DRAM_BYTES_HEADLINE = 10.451892e9 + 0.834476e9


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--rows", type=int, default=131072, help="m of the workload")
    p.add_argument("--workload", default="single",
                   choices=["single", "small", "batched", "mixed", "serve", "dense", "panels",
                            "srrqr", "sharded", "sweep"],
                   help="single: the rank-800 131072 x 1024 problem (headline); small: the "
                        "4096 x 64 cond-1e8 problem (latency per factorisation); batched: 512 "
                        "uneven problems in one batched pass; mixed: 1048576 x 512, cond 1e10, "
                        "split-BF16 modes against FP64; serve: a Poisson stream of mixed-size "
                        "requests through the continuous-batching server; dense: the "
                        "headline matrix with a dense Gaussian operator instead of the SASO; "
                        "panels: the headline matrix streamed from pinned host memory in row "
                        "panels; srrqr: the headline matrix with the strong rank-revealing "
                        "exchanges on the sketch; sharded: one (ranks x --rows) x 1024 "
                        "matrix partitioned by rows over the torchrun ranks; sweep: Gaussian "
                        "--rows x n, n = 512 .. 4096 (the paper's speed experiment), FP64 "
                        "and split-BF16")
    p.add_argument("--configs", default="all", choices=["all", "none"],
                   help="single workload, N = 1: also measure the small, mixed, batched and "
                        "serving workloads in the same run (all) or only the headline (none)")
    p.add_argument("--batch", type=int, default=512)
    p.add_argument("--requests", type=int, default=600, help="serve: requests in the open loop")
    p.add_argument("--pool", type=int, default=32, help="serve: distinct matrices")
    p.add_argument("--lanes", type=int, default=3, help="serve: server lanes (units in flight)")
    p.add_argument("--load", type=float, default=0.7,
                   help="serve: offered rate as a fraction of the closed-loop capacity")
    return p.parse_args()


# --------------------------------------------------------------- distributed
def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        dist.init_process_group(backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world, device="cpu"):
    """Max of a float over all ranks (the slowest rank sets the step time)."""
    if world == 1:
        return float(x)
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def rank_workload(w, rank):
    """Rank r's own problem of the same shape: matrix and S seeds shifted by
    r (rank 0 keeps the published seeds), so ranks factor independent inputs."""
    if rank == 0:
        return w
    import dataclasses
    return dataclasses.replace(w, seed=w.seed + 7919 * rank,
                               sketch_seed=w.sketch_seed + 7919 * rank)


def rank_batch(count, rank):
    """Rank r's own batch of `count` uneven problems (independent seeds)."""
    return W.batch_uneven(count=count, seed=W.BASE_SEED + 3 + 104729 * rank)


# --------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ["clocks.sm", "clocks.max.sm", "power.draw", "clocks_event_reasons.active",
              "clocks_event_reasons.hw_slowdown", "clocks_event_reasons.hw_thermal_slowdown",
              "clocks_event_reasons.sw_thermal_slowdown", "clocks_event_reasons.sw_power_cap"]

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + ",".join(self.FIELDS),
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < len(self.FIELDS):
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------- reference arm
def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo), or None."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return None


def cpu_threads():
    """Threads the oracle's OpenMP loops use (OMP_NUM_THREADS, else every
    core the process may run on)."""
    env = os.environ.get("OMP_NUM_THREADS")
    if env and env.isdigit():
        return int(env)
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count()


ORACLE_PHASES = ["sketch", "qrcp", "rank", "trsm_pre", "gram", "cholesky", "trsm_q", "trmm"]


class OracleSteps:
    """The oracle's CQRRPT (Alg. 1 + Alg. 2) cut into its eight public phase
    calls, made in the order oracle_cqrrpt makes them: the sketch (line 1),
    the QRCP (2), the rank rule (3), M^pre (4), the Gram (5), the Cholesky
    with Remark 4 and the second rank stage (6), Q (7), R (8).  run(i) makes
    phase i; after phase 7 `result` holds (Q, R, J, k) of one factorisation
    and the next run(0) starts another."""

    def __init__(self, M, gamma, nnz, tol, seed):
        import oracle
        self.o = oracle
        self.M, self.gamma, self.nnz, self.tol, self.seed = M, gamma, nnz, tol, seed
        self.result = None

    def run(self, i):
        o, st = self.o, self
        m, n = st.M.shape
        if i == 0:
            st.d = o.sketch_dim(n, st.gamma)
            st.Msk, st.status = o.sketch(st.M, st.d, st.nnz, st.seed)
            st.k = 0
        elif i == 1:
            if st.status == 0:
                st.Rsk, st.J = o.qrcp(st.Msk)[:2]
        elif i == 2:
            if st.status == 0:
                st.stage2 = not (st.tol > 0.0)
                st.k = o.rank_stage1(st.Rsk) if st.stage2 else o.rank_tol(st.Rsk, st.tol)
        elif i == 3:
            if st.status == 0 and st.k > 0:
                st.X = o.trsm_rut(st.M, st.Rsk[:st.k, :st.k], st.J)
        elif i == 4:
            if st.status == 0 and st.k > 0:
                st.G = o.gram(st.X)
        elif i == 5:
            if st.status == 0 and st.k > 0:
                st.Rpre, fail = o.potrf_upper(st.G)
                kc = fail if fail >= 0 else st.k
                if st.stage2 and kc > 0:
                    kc = o.rank_stage2(kc, st.Rpre)
                st.k = kc
        elif i == 6:
            if st.status == 0 and st.k > 0:
                st.Q = o.trsm_rut(st.X, st.Rpre[:st.k, :st.k])
        elif i == 7:
            if st.status == 0 and st.k > 0:
                R = o.trmm_upper(st.Rpre[:st.k, :st.k], st.Rsk[:st.k, :])
                st.result = (st.Q, R, st.J, st.k)
            else:
                st.result = (None, None, getattr(st, "J", None), 0)
            st.X = st.G = None


def run_reference(args, world, rank):
    """The oracle, as it stands, on the full headline workload (m = 131072,
    n = 1024, planted rank 800), on the host cores.  Step i makes phase
    i mod 8 of a factorisation (OracleSteps), so a factorisation spans eight
    consecutive steps and the whole --warmup + --steps run stays within a few
    minutes; value = 1 / (sum over the eight phases of the mean time of that
    phase in the timed steps): factorisations/s of the full workload, no
    extrapolation."""
    if rank != 0:
        return
    w = W.single_large(m=args.rows)
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    A = np.asfortranarray(W.planted(w.m, w.n, w.sv, w.seed, w.noise, dev).cpu().numpy())
    steps = OracleSteps(A, w.gamma, w.nnz, w.tol, w.sketch_seed)
    phase_ms = {p: [] for p in ORACLE_PHASES}
    step_ms = []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        steps.run(i % 8)
        dt = (time.perf_counter() - t0) * 1e3
        if i >= args.warmup:
            step_ms.append(dt)
            phase_ms[ORACLE_PHASES[i % 8]].append(dt)
    if all(phase_ms.values()):
        fact_ms = sum(statistics.mean(v) for v in phase_ms.values())
        how = "1 / sum of the eight phases' mean times"
    else:  # fewer than eight timed steps: steps / 8 factorisations over the time
        fact_ms = sum(step_ms) * 8.0 / len(step_ms)
        how = "(steps / 8) factorisations over the timed seconds"
    value = 1e3 / fact_ms
    threads = cpu_threads()
    sample = ("the full workload (%d x %d); step i makes phase i mod 8 (%s) of the oracle's "
              "factorisation, so 8 consecutive steps are one factorisation; value = %s"
              % (w.m, w.n, ", ".join(ORACLE_PHASES), how))
    line = {"metric": "cqrrpt_factorizations_per_s", "value": value, "unit": "factorizations/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": statistics.mean(step_ms), "ms_per_factorization": fact_ms,
            "phase_ms": {p: (statistics.mean(v) if v else None) for p, v in phase_ms.items()},
            "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": config_of(w),
            "cpu_baseline": {"value": value, "unit": "factorizations/s", "cores": threads,
                             "cpu_model": cpu_model(), "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "factorizations/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def config_of(w):
    return {"workload": w.name, "m": w.m, "n": w.n, "d": w.d, "nnz_per_col": w.nnz,
            "gamma": w.gamma, "tol": w.tol, "planted_rank": w.rank, "precision": "fp64",
            "l2": "inputs larger than L2 (A = %.2f GiB > 129 MB), no flush" % (w.m * w.n * 8 / 2**30)}


def cqrrpt_flops(m, n, d, k, s):
    """Sec. 2.1 count (GEQP3 on the sketch) at the actual k, plus the sketch's
    m*s*n additions."""
    return (2.0 * m * k * k + m * k * (k + 1) + 4.0 * d * n * k - 2.0 * k * k * (d + n)
            + 5.0 * k ** 3 / 3.0 + float(m) * s * n)


def run_small(args, world, rank, local, C):
    """The small full-rank problem (m = 4096, n = 64, sv 1 -> 1e-8 log-spaced,
    SASO d = 128 with 4 nonzeros per column, tol 1e-12): a launch-bound
    factorisation.  Latency per call two ways: device span of each call
    between CUDA events on its stream (calls queued back to back), and host
    wall time of a synchronous call (k read back), p50 / p99 over the calls;
    throughput of back-to-back calls.  Parity: bit-identical to the oracle."""
    import oracle
    w = rank_workload(W.single_small(), rank)
    m, n = w.m, w.n
    A = w.matrix("cuda")
    h = C.Handle(local)
    Q = C.colmajor_empty(m, n)
    R = C.colmajor_empty(n, n)
    J = torch.empty(n, dtype=torch.int64, device="cuda")
    stream = torch.cuda.current_stream()

    def call(sync):
        return C.cqrrpt(A, w.gamma, w.nnz, w.tol, w.sketch_seed, out=(Q, R, J), handle=h,
                        stream=stream, sync=sync)

    for _ in range(max(3, args.warmup)):
        res = call(True)
    assert res.status == 0 and res.k == n
    calls = max(200, args.steps)
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    barrier(world)
    torch.cuda.synchronize()
    launches0 = C.kernel_launches()
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(2 * calls)]
    t0 = time.perf_counter()
    for i in range(calls):
        evs[2 * i].record(stream)
        call(False)
        evs[2 * i + 1].record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    launches = C.kernel_launches() - launches0
    dev_us = [evs[2 * i].elapsed_time(evs[2 * i + 1]) * 1e3 for i in range(calls)]
    host_us = []
    for _ in range(calls):
        t1 = time.perf_counter()
        call(True)
        host_us.append((time.perf_counter() - t1) * 1e6)
    clk = clocks.stop()
    st, k = h.last_status()
    assert st == 0 and k == n
    wall = max_over_ranks(wall, world)
    value = world * calls / wall
    ref = oracle.cqrrpt(np.asfortranarray(A.cpu().numpy()), w.gamma, w.nnz, w.tol, w.sketch_seed)
    same = (ref.k == k and np.array_equal(ref.J, J.cpu().numpy())
            and np.array_equal(ref.Q.view(np.uint64),
                               np.asfortranarray(Q[:, :k].cpu().numpy()).view(np.uint64))
            and np.array_equal(ref.R.view(np.uint64),
                               np.asfortranarray(R[:k].cpu().numpy()).view(np.uint64)))
    flops = cqrrpt_flops(m, n, w.d, n, w.nnz)
    h.close()
    return {"metric": "cqrrpt_factorizations_per_s", "value": value, "unit": "factorizations/s",
            "n_gpus": world, "steps": calls, "warmup": max(3, args.warmup),
            "ms_per_step": wall * 1e3 / calls, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w.name, "m": m, "n": n, "d": w.d, "nnz_per_col": w.nnz,
                       "gamma": w.gamma, "tol": w.tol, "precision": "fp64",
                       "l2": "A = 2 MiB is L2-resident between calls (latency case), no flush"},
            "latency_us": {"device_p50": float(np.percentile(dev_us, 50)),
                           "device_p99": float(np.percentile(dev_us, 99)),
                           "host_sync_p50": float(np.percentile(host_us, 50)),
                           "host_sync_p99": float(np.percentile(host_us, 99))},
            "gflops_algorithmic": value * flops / 1e9,
            "fp64_fraction": value * flops / 1e9 / FP64_PEAK_GFLOPS,
            "parity_vs_oracle": "bit-identical J, k, Q, R" if same else "MISMATCH",
            "gpu_launches": int(launches), "clocks": clk}


def run_sharded(args, world, rank, local, C):
    """The row-partitioned form (Sec. 2.1) across the torchrun ranks: one
    m x 1024 problem with m = world x --rows (each rank holds --rows rows,
    planted rank 800 as the headline workload), the sketch and the Gram
    summed over the ranks in rank order (ordered_scan: NCCL send / receive
    and broadcast of d x n and n x n doubles; gloo through host copies).
    One step = one factorisation of the whole matrix by all ranks; weak
    scaling (fixed rows per rank).  Rank 0 checks its rows of Q and the whole
    R, J, k against cqrrpt_d on the whole matrix (N = 1: the same call)."""
    import torch.distributed as dist
    w = W.single_large(m=args.rows * world)
    rows = args.rows
    r0 = rank * rows
    A_full = w.matrix("cuda")
    A = C.colmajor(A_full[r0:r0 + rows])
    ref = None
    if rank == 0:
        ref = C.cqrrpt(A_full, w.gamma, w.nnz, w.tol, w.sketch_seed)
        ref = (ref.k, ref.J.clone(), ref.Q[:rows].clone(), ref.R.clone())
    del A_full
    torch.cuda.empty_cache()
    h = C.Handle(local)
    group = None

    def step():
        return C.cqrrpt_sharded(A, w.m, r0, w.gamma, w.nnz, w.tol, w.sketch_seed, group=group,
                                handle=h)

    for _ in range(args.warmup):
        res = step()
    assert res.status == 0
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    barrier(world)
    torch.cuda.synchronize()
    launches0 = C.kernel_launches()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        res = step()
    torch.cuda.synchronize()
    elapsed = time.perf_counter() - t0
    barrier(world)
    launches = C.kernel_launches() - launches0
    clk = clocks.stop()
    elapsed = max_over_ranks(elapsed, world, "cuda")
    value = args.steps / elapsed
    parity = None
    if rank == 0:
        k, J, Q, R = ref
        parity = ("bit-identical to cqrrpt_d on the whole matrix (rank 0's rows of Q, R, J, k)"
                  if res.k == k and torch.equal(res.J, J) and torch.equal(res.Qbuf[:, :k], Q)
                  and torch.equal(res.Rbuf[:k], R) else "MISMATCH")
    d = w.d
    return {"metric": "cqrrpt_factorizations_per_s", "value": value,
            "unit": "factorizations/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": elapsed * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "cqrrpt_fp64_row_partitioned_m%d_n%d_rank800" % (w.m, w.n),
                       "m": w.m, "rows_per_rank": rows, "n": w.n, "d": d,
                       "nnz_per_col": w.nnz, "tol": w.tol,
                       "parallelism": "rows over %d ranks" % world,
                       "l2": "inputs larger than L2, no flush"},
            "gflops_2mn2": value * 2.0 * w.m * w.n * w.n / 1e9,
            "communication_bytes_per_rank": 8 * (d * w.n + w.n * w.n) * (2 if world > 1 else 0),
            "parity": parity, "gpu_launches": int(launches), "clocks": clk}


def run_batched(args, world, rank, local, C):
    """512 independent problems (m ~ U[4096, 65536], n ~ U[32, 256], rank ~
    U[n/2, n]) factored by one batched pass (one graph launch) per step."""
    ws = rank_batch(args.batch, rank)
    mats = [w.matrix("cuda") for w in ws]
    outs = [(C.colmajor_empty(w.m, w.n), C.colmajor_empty(w.n, w.n),
             torch.empty(w.n, dtype=torch.int64, device="cuda")) for w in ws]
    tols = [w.tol for w in ws]
    seeds = [w.sketch_seed for w in ws]
    h = C.Handle(local)
    stream = torch.cuda.current_stream()

    def step(sync):
        return C.cqrrpt_batched(mats, 1.25, 4, tols, seeds, outs=outs, handle=h, stream=stream,
                                sync=sync)

    # the first warm-up step runs the autotuner (tile shapes per width bucket)
    res, kd, sd, tune_us = C.cqrrpt_batched(mats, 1.25, 4, tols, seeds, outs=outs, handle=h,
                                            stream=stream, autotune=True)
    tuned = C.get_batch_tuning(handle=h)
    for _ in range(max(0, args.warmup - 1)):
        res, kd, sd = step(True)
    ks = [r.k for r in res]
    assert all(r.status == 0 for r in res), [r.status for r in res]
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    barrier(world)
    torch.cuda.synchronize()
    launches0 = C.kernel_launches()
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    evs[0].record(stream)
    for i in range(args.steps):
        step(False)
        evs[i + 1].record(stream)
    torch.cuda.synchronize()
    barrier(world)
    launches = C.kernel_launches() - launches0
    clk = clocks.stop()
    step_ms = [evs[i].elapsed_time(evs[i + 1]) for i in range(args.steps)]
    elapsed = max_over_ranks(sum(step_ms), world, "cuda")
    ms_per_step = elapsed / args.steps
    value = world * len(ws) * args.steps / (elapsed / 1e3)
    flops = sum(cqrrpt_flops(w.m, w.n, w.d, k, w.nnz) for w, k in zip(ws, ks))
    achieved = flops / (ms_per_step * 1e-3) / 1e9
    line = {"metric": "cqrrpt_factorizations_per_s", "value": value, "unit": "factorizations/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "cqrrpt_fp64_batched%d_m4096-65536_n32-256" % len(ws),
                       "batch": len(ws), "sum_m": sum(w.m for w in ws),
                       "sum_2mn2": sum(2.0 * w.m * w.n * w.n for w in ws),
                       "gamma": 1.25, "nnz_per_col": 4, "precision": "fp64",
                       "launch": "one CUDA graph of per-phase batched kernels per step",
                       "autotuned": {"trsm_jb": tuned[0], "gram_tile": tuned[1],
                                     "bucket": "min((n-1)//32, 15)",
                                     "times_us": {str(b): v for b, v in tune_us.items()}},
                       "l2": "inputs larger than L2 (sum of A = %.1f GB), no flush"
                             % (sum(w.m * w.n * 8 for w in ws) / 1e9)},
            "gflops_2mn2": value * sum(2.0 * w.m * w.n * w.n for w in ws) / len(ws) / 1e9,
            "gflops_algorithmic": achieved * world,
            "latency_ms": {"p50": float(np.percentile(step_ms, 50)),
                           "p99": float(np.percentile(step_ms, 99))},
            "roofline": {"kernel": "whole batched pass", "bound": "alu", "achieved": achieved,
                         "peak": FP64_PEAK_GFLOPS, "unit": "GFLOP/s",
                         "frac": achieved / FP64_PEAK_GFLOPS, "traffic": None},
            "gpu_launches": int(launches), "clocks": clk}
    # ---- the same batch in the split-BF16 mode (lines 4, 5, 7 as batched
    # tensor-core products): time, and J / k / accuracy against FP64
    split = None
    try:
        outs_s = [(C.colmajor_empty(w.m, w.n), C.colmajor_empty(w.n, w.n),
                   torch.empty(w.n, dtype=torch.int64, device="cuda")) for w in ws]
        for _ in range(2):
            res_s, _, _ = C.cqrrpt_batched(mats, 1.25, 4, tols, seeds, precision=C.SPLITBF16,
                                           outs=outs_s, handle=h, stream=stream)
        ms_s = []
        for _ in range(max(1, args.steps)):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            res_s, _, _ = C.cqrrpt_batched(mats, 1.25, 4, tols, seeds, precision=C.SPLITBF16,
                                           outs=outs_s, handle=h, stream=stream)
            e1.record(stream)
            torch.cuda.synchronize()
            ms_s.append(e0.elapsed_time(e1))
        same_jk = all(a.k == b.k and torch.equal(a.J, b.J) for a, b in zip(res, res_s))
        worst_recon, worst_orth = 0.0, 0.0
        for i in list(range(0, len(ws), max(1, len(ws) // 8)))[:8]:
            r = res_s[i]
            if r.k:
                AJ = mats[i][:, r.J]
                worst_recon = max(worst_recon, (torch.linalg.norm(AJ - r.Q @ r.R)
                                                / torch.linalg.norm(mats[i])).item())
                worst_orth = max(worst_orth, torch.linalg.matrix_norm(
                    r.Q.t() @ r.Q - torch.eye(r.k, dtype=torch.float64, device="cuda"),
                    ord=2).item())
        split = {"ms_per_batch": statistics.median(ms_s),
                 "factorizations_per_s": len(ws) / (statistics.median(ms_s) / 1e3),
                 "speedup_vs_fp64": ms_per_step / statistics.median(ms_s),
                 "J_and_k_equal_fp64": bool(same_jk),
                 "worst_recon_rel_F_sampled": worst_recon, "worst_orth_2_sampled": worst_orth,
                 "note": "wall time of the call: includes its two host waits for k"}
        del outs_s, res_s
    except Exception as ex:  # reported, not hidden
        split = {"error": str(ex)}
    line["splitbf16_same_batch"] = split

    if rank == 0 and world == 1:
        import oracle
        # parity and CPU baseline on a sample of 8 problems
        sample = list(range(0, len(ws), max(1, len(ws) // 8)))[:8]
        t_cpu, f_cpu, same = 0.0, 0.0, True
        for i in sample:
            w = ws[i]
            A = np.asfortranarray(mats[i].cpu().numpy())
            t0 = time.perf_counter()
            ref = oracle.cqrrpt(A, 1.25, 4, w.tol, w.sketch_seed)
            t_cpu += time.perf_counter() - t0
            f_cpu += cqrrpt_flops(w.m, w.n, w.d, ref.k, w.nnz)
            r = res[i]
            same &= (ref.k == r.k and np.array_equal(ref.J, r.J.cpu().numpy())
                     and np.array_equal(ref.Q.view(np.uint64),
                                        np.asfortranarray(r.Q.cpu().numpy()).view(np.uint64))
                     and np.array_equal(ref.R.view(np.uint64),
                                        np.asfortranarray(r.R.cpu().numpy()).view(np.uint64)))
        cpu_batch_s = t_cpu * flops / f_cpu
        line["cpu_baseline"] = {"value": len(ws) / cpu_batch_s, "unit": "factorizations/s",
                                "cores": os.cpu_count(), "kind": "oracle",
                                "sample": "%d of the %d problems (%.1f s), extrapolated to the "
                                          "batch by the Sec. 2.1 flop count" % (len(sample), len(ws), t_cpu)}
        line["parity_vs_oracle"] = ("bit-identical J, k, Q, R on %d sampled problems" % len(sample)
                                    if same else "MISMATCH")
    return line


def run_mixed(args, world, rank, local, C):
    """m = 2^20, n = 512, cond 1e10 (log-spaced), gamma 1.25, 4 nnz/col,
    tol 1e-12: the split-BF16 modes (lines 4, 5, 7 on the tensor cores,
    with and without a second Cholesky-QR pass) timed against the FP64
    mode on the same inputs; accuracy of each against the FP64 result (which
    is bit-identical to the oracle)."""
    w = rank_workload(W.mixed_tall(m=args.rows if args.rows != 131072 else (1 << 20)), rank)
    A = w.matrix("cuda")
    m, n = w.m, w.n
    h = C.Handle(local)
    stream = torch.cuda.current_stream()
    out = {}
    results = {}
    clocks = ClockSampler(local)
    clocks.start()
    for prec, name in [(C.FP64, "fp64"), (C.SPLITBF16, "splitbf16"),
                       (C.SPLITBF16_CHOLQR2, "splitbf16_cholqr2")]:
        Q = C.colmajor_empty(m, n)
        R = C.colmajor_empty(n, n)
        J = torch.empty(n, dtype=torch.int64, device="cuda")
        for _ in range(max(1, args.warmup)):
            res = C.cqrrpt(A, w.gamma, w.nnz, w.tol, w.sketch_seed, precision=prec, out=(Q, R, J),
                           handle=h, stream=stream)
        torch.cuda.synchronize()
        steps = args.steps if prec != C.FP64 else max(1, min(args.steps, 3))
        ms = []
        for _ in range(steps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            res = C.cqrrpt(A, w.gamma, w.nnz, w.tol, w.sketch_seed, precision=prec, out=(Q, R, J),
                           handle=h, stream=stream)
            e1.record(stream)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        k = res.k
        AJ = A[:, J]
        recon = (torch.linalg.norm(AJ - Q[:, :k] @ R[:k]) / torch.linalg.norm(A)).item()
        orth = torch.linalg.matrix_norm(Q[:, :k].t() @ Q[:, :k] - torch.eye(k, dtype=torch.float64,
                                                                           device="cuda"),
                                        ord=2).item()
        del AJ
        results[name] = (Q, R, J, k)
        out[name] = {"ms": statistics.median(ms), "factorizations_per_s": 1e3 / statistics.median(ms),
                     "k": k, "recon_rel_F": recon, "orth_2": orth}
    # Sec. 1.3's randomized CholeskyQR (no pivoting) on the same full-rank
    # matrix, in FP64: time and accuracy beside CQRRPT's
    try:
        Qr, Rr, Jr = C.colmajor_empty(m, n), C.colmajor_empty(n, n), torch.empty(
            n, dtype=torch.int64, device="cuda")
        rr = C.rcholqr(A, w.gamma, w.nnz, w.sketch_seed, out=(Qr, Rr, Jr), handle=h, stream=stream)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        rr = C.rcholqr(A, w.gamma, w.nnz, w.sketch_seed, out=(Qr, Rr, Jr), handle=h, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        kr = rr.k
        out["fp64_rcholqr"] = {
            "ms": e0.elapsed_time(e1), "k": kr,
            "recon_rel_F": (torch.linalg.norm(A - Qr[:, :kr] @ Rr[:kr]) / torch.linalg.norm(A)).item(),
            "orth_2": torch.linalg.matrix_norm(Qr[:, :kr].t() @ Qr[:, :kr] - torch.eye(
                kr, dtype=torch.float64, device="cuda"), ord=2).item(),
            "note": "unpivoted (Sec. 1.3): J is the identity"}
        del Qr, Rr, Jr
    except Exception as ex:  # reported, not hidden
        out["fp64_rcholqr"] = {"error": str(ex)}
    clk = clocks.stop()
    Rf = results["fp64"][1][: results["fp64"][3]]
    for name in ("splitbf16", "splitbf16_cholqr2"):
        Rs = results[name][1][: results[name][3]]
        out[name]["R_rel_diff_vs_fp64"] = (torch.linalg.norm(Rs - Rf) / torch.linalg.norm(Rf)).item()
        out[name]["J_equal_fp64"] = bool(torch.equal(results[name][2], results["fp64"][2]))
        out[name]["speedup_vs_fp64"] = out["fp64"]["ms"] / out[name]["ms"]
    best = out["splitbf16"]
    line = {"metric": "cqrrpt_factorizations_per_s", "value": best["factorizations_per_s"],
            "unit": "factorizations/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": best["ms"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "bf16 digits -> f32 (exact) -> f64",
            "data": "synthetic",
            "config": {"workload": w.name, "m": m, "n": n, "d": w.d, "nnz_per_col": w.nnz,
                       "gamma": w.gamma, "tol": w.tol, "cond": 1e10,
                       "l2": "inputs larger than L2 (A = %.1f GiB), no flush" % (m * n * 8 / 2**30)},
            "gflops_2mn2": best["factorizations_per_s"] * 2.0 * m * n * n / 1e9,
            "modes": out, "clocks": clk,
            "note": "FP64 mode is bit-identical to the oracle (tests); differences are vs that"}
    return line


def run_dense(args, world, rank, local, C):
    """The headline matrix (m = 131072, n = 1024, planted rank 800, tol 1e-9)
    sketched by a dense Gaussian operator (Sec. 2.3.1: iid N(0, 1/d),
    d = 1280, drawn once on the device, resident) instead of the SASO: in FP64
    (bit-identical to the oracle, tests), and in split-BF16, where the sketch
    too runs on the tensor cores.  The sketch is 2 d m n flops; its time and
    roofline fraction are reported beside the SASO run of the same matrix."""
    w = rank_workload(W.single_large(m=args.rows), rank)
    m, n, d = w.m, w.n, w.d
    A = w.matrix("cuda")
    S = W.gaussian_operator(d, m, w.sketch_seed, "cuda")
    h = C.Handle(local)
    stream = torch.cuda.current_stream()
    Q = C.colmajor_empty(m, n)
    R = C.colmajor_empty(n, n)
    J = torch.empty(n, dtype=torch.int64, device="cuda")
    steps = max(1, min(args.steps, 3))
    out = {}

    def timed(call):
        for _ in range(max(1, args.warmup)):
            call()
        torch.cuda.synchronize()
        h.set_profiling(True)
        ms, sk = [], []
        for _ in range(steps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            call()
            e1.record(stream)
            sk.append(h.phase_times()["sketch"])
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        h.set_profiling(False)
        st, k = h.last_status()
        assert st == 0, st
        return statistics.median(ms), statistics.median(sk), k

    for prec, name in [(C.FP64, "fp64"), (C.SPLITBF16, "splitbf16")]:
        t, tsk, k = timed(lambda: C.cqrrpt_dense(A, S, w.tol, precision=prec, out=(Q, R, J),
                                                 handle=h, stream=stream, sync=False))
        AJ = A[:, J]
        recon = (torch.linalg.norm(AJ - Q[:, :k] @ R[:k]) / torch.linalg.norm(A)).item()
        del AJ
        orth = torch.linalg.matrix_norm(Q[:, :k].t() @ Q[:, :k] - torch.eye(
            k, dtype=torch.float64, device="cuda"), ord=2).item()
        sk_flops = 2.0 * d * m * n
        out[name] = {"ms": t, "factorizations_per_s": 1e3 / t, "k": k, "sketch_ms": tsk,
                     "recon_rel_F": recon, "orth_2": orth}
        if prec == C.FP64:
            out[name]["sketch_roofline"] = {
                "kernel": "sketch_dense_partial_kernel", "bound": "alu",
                "achieved": sk_flops / (tsk * 1e-3) / 1e9, "peak": FP64_PEAK_GFLOPS,
                "unit": "GFLOP/s", "frac": sk_flops / (tsk * 1e-3) / 1e9 / FP64_PEAK_GFLOPS,
                "algorithmic_flops_per_launch": sk_flops}
        else:
            # split-BF16 sketch: 36 digit-pair products of the d x m x n shape
            # (plus transpose and splits) against the measured bf16 peak
            tc = 36.0 * sk_flops / (tsk * 1e-3) / 1e12
            out[name]["sketch_roofline"] = {
                "kernel": "sketch (transpose, splits, oz_tc_kernel, combine)", "bound": "tensor",
                "achieved": tc, "peak": BF16_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": tc / BF16_PEAK_TFLOPS,
                "fp64_equivalent_gflops": sk_flops / (tsk * 1e-3) / 1e9,
                "algorithmic_flops_per_launch": 36.0 * sk_flops}
    t, tsk, k = timed(lambda: C.cqrrpt(A, w.gamma, w.nnz, w.tol, w.sketch_seed, out=(Q, R, J),
                                       handle=h, stream=stream, sync=False))
    out["saso_fp64"] = {"ms": t, "sketch_ms": tsk, "k": k}
    best = out["fp64"]
    line = {"metric": "cqrrpt_factorizations_per_s", "value": best["factorizations_per_s"],
            "unit": "factorizations/s", "n_gpus": world, "steps": steps,
            "warmup": args.warmup, "ms_per_step": best["ms"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": w.name + "_gaussian_operator", "m": m, "n": n, "d": d,
                       "operator": "dense Gaussian N(0, 1/d)", "tol": w.tol,
                       "l2": "inputs larger than L2 (A %.1f GiB, S %.1f GiB), no flush"
                             % (m * n * 8 / 2**30, d * m * 8 / 2**30)},
            "modes": out,
            "note": "S is drawn once before timing (not timed); FP64 mode bit-identical to "
                    "the oracle (tests)"}
    return line


def run_panels(args, world, rank, local, C):
    """The headline matrix (m = 131072, n = 1024, planted rank 800) held in
    pinned host memory and factored over row panels (cqrrpt_panels_host_d:
    three passes over the panels, two device slots, copies on their own
    streams), against the device-resident cqrrpt_d on the same matrix.  The
    timed region includes every host<->device copy (M twice, M^pre out and
    back, Q out)."""
    w = rank_workload(W.single_large(m=args.rows), rank)
    m, n = w.m, w.n
    Ad = w.matrix("cuda")
    A = torch.empty((n, m), dtype=torch.float64, pin_memory=True).t()
    A.copy_(Ad)
    Qh = torch.empty((n, m), dtype=torch.float64, pin_memory=True).t()
    Rh = C.colmajor_empty(n, n, "cpu")
    Jh = torch.empty(n, dtype=torch.int64)
    h = C.Handle(local)
    steps = max(1, min(args.steps, 3))
    out = {}
    for P in (16384, 65536):
        for _ in range(max(1, args.warmup)):
            Q, R, J, k, st = C.cqrrpt_panels(A, w.gamma, w.nnz, w.tol, w.sketch_seed,
                                             panel_rows=P, out=(Qh, Rh, Jh), handle=h)
        ms = []
        for _ in range(steps):
            t0 = time.perf_counter()
            Q, R, J, k, st = C.cqrrpt_panels(A, w.gamma, w.nnz, w.tol, w.sketch_seed,
                                             panel_rows=P, out=(Qh, Rh, Jh), handle=h)
            ms.append((time.perf_counter() - t0) * 1e3)
        assert st == 0, st
        out["panel_rows_%d" % P] = {"ms": statistics.median(ms), "k": k,
                                    "factorizations_per_s": 1e3 / statistics.median(ms),
                                    "device_bytes_panels": 4 * P * n * 8}
    res = C.cqrrpt(Ad, w.gamma, w.nnz, w.tol, w.sketch_seed, handle=h)
    ms = []
    for _ in range(steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        res = C.cqrrpt(Ad, w.gamma, w.nnz, w.tol, w.sketch_seed, handle=h)
        ms.append((time.perf_counter() - t0) * 1e3)
    out["device_resident_ms"] = statistics.median(ms)
    same = bool(torch.equal(res.J.cpu(), Jh) and torch.equal(res.Q.cpu(), Q)
                and torch.equal(res.R.cpu(), R))
    best = min((v for v in out.values() if isinstance(v, dict)), key=lambda v: v["ms"])
    line = {"metric": "cqrrpt_factorizations_per_s", "value": best["factorizations_per_s"],
            "unit": "factorizations/s", "n_gpus": world, "steps": steps,
            "warmup": args.warmup, "ms_per_step": best["ms"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w.name + "_host_row_panels", "m": m, "n": n, "d": w.d,
                       "nnz_per_col": w.nnz, "tol": w.tol,
                       "h2d_bytes_per_step": 2 * m * n * 8 + m * k * 8,
                       "d2h_bytes_per_step": 2 * m * k * 8 + k * n * 8 + n * 8},
            "modes": out, "equal_to_device_resident_bits": same,
            "note": "wall clock of the whole call (host copies included)"}
    return line


def run_srrqr(args, world, rank, local, C):
    """The headline matrix (m = 131072, n = 1024, planted rank 800) with the
    strong rank-revealing exchanges of Sec. 2.2 after the rank rule
    (cqrrpt_srrqr_d, f = 2 as the paper names, and f = 1.05), against
    cqrrpt_d on the same matrix.  Wall clock of the whole call (the
    exchange loop waits on the host once per step)."""
    w = rank_workload(W.single_large(m=args.rows), rank)
    m, n = w.m, w.n
    A = w.matrix("cuda")
    h = C.Handle(local)
    Q = C.colmajor_empty(m, n)
    R = C.colmajor_empty(n, n)
    J = torch.empty(n, dtype=torch.int64, device="cuda")
    steps = max(1, min(args.steps, 3))
    out = {}

    def wall(call):
        for _ in range(max(1, args.warmup)):
            r = call()
        ms = []
        for _ in range(steps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            r = call()
            torch.cuda.synchronize()
            ms.append((time.perf_counter() - t0) * 1e3)
        return statistics.median(ms), r

    t, res = wall(lambda: C.cqrrpt(A, w.gamma, w.nnz, w.tol, w.sketch_seed, out=(Q, R, J),
                                   handle=h))
    out["cqrrpt_fp64_ms"] = t
    J0 = J.clone()
    for f in (2.0, 1.05):
        t, (res, sw) = wall(lambda: C.cqrrpt_srrqr(A, w.gamma, w.nnz, w.tol, w.sketch_seed, f=f,
                                                   out=(Q, R, J), handle=h))
        k = res.k
        recon = (torch.linalg.norm(A[:, J] - Q[:, :k] @ R[:k]) / torch.linalg.norm(A)).item()
        orth = torch.linalg.matrix_norm(Q[:, :k].t() @ Q[:, :k] - torch.eye(
            k, dtype=torch.float64, device="cuda"), ord=2).item()
        out["f_%g" % f] = {"ms": t, "k": k, "exchanges": sw, "recon_rel_F": recon,
                           "orth_2": orth, "J_equal_cqrrpt": bool(torch.equal(J, J0))}
    best = out["f_2"]
    line = {"metric": "cqrrpt_factorizations_per_s", "value": 1e3 / best["ms"],
            "unit": "factorizations/s", "n_gpus": world, "steps": steps,
            "warmup": args.warmup, "ms_per_step": best["ms"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w.name + "_strong_rrqr", "m": m, "n": n, "d": w.d,
                       "nnz_per_col": w.nnz, "tol": w.tol},
            "modes": out, "note": "wall clock per call; bit-identical to the oracle (tests)"}
    return line


def run_serve(args, world, rank, local, C):
    """Continuous-batching server under a Poisson stream.  Requests are drawn
    from a pool of `--pool` matrices of the serving mix (m = 2^U[12,20],
    n = 2^U[4,9], cond 10^U[2,12], 30% planted rank with 1e-15 noise); each
    request has its own sketch seed and precision (FP64 or split-BF16, 50/50).
    First the closed-loop capacity (every request queued at once), then the
    open loop at `--load` x capacity; latency is arrival -> results in the
    request's host buffers (host copies included), measured by the server."""
    import oracle
    rng = np.random.default_rng(W.BASE_SEED + 5)
    pool = W.serving_requests(args.pool)
    hosts, outs = [], []
    for w, _ in pool:
        A = w.matrix("cuda")
        Ah = torch.empty((w.n, w.m), dtype=torch.float64, pin_memory=True).t()
        Ah.copy_(A)
        del A
        hosts.append(Ah)
        # one output set per pool entry, shared by its non-sampled requests
        # (their results are not read; sampled requests get their own)
        outs.append((torch.empty((w.n, w.m), dtype=torch.float64, pin_memory=True).t(),
                     torch.empty((w.n, w.n), dtype=torch.float64, pin_memory=True).t(),
                     torch.empty(w.n, dtype=torch.int64, pin_memory=True)))
    torch.cuda.synchronize()
    h = C.Handle(local)
    srv = C.Server(hbm_budget_bytes=120 << 30, max_inflight=64, handle=h, lanes=args.lanes)

    def make(count, seed_base):
        reqs = []
        for i in range(count):
            e = int(rng.integers(len(pool)))
            prec = C.SPLITBF16 if rng.random() < 0.5 else C.FP64
            reqs.append((e, prec, seed_base + i))
        return reqs

    def submit(req, out=None):
        e, prec, seed = req
        w = pool[e][0]
        return srv.submit(hosts[e], w.tol, seed, precision=prec, out=out or outs[e])

    # warm-up: every pool entry once in each precision (sizes the workspace)
    for e in range(len(pool)):
        for prec in (C.FP64, C.SPLITBF16):
            submit((e, prec, 7))
    srv.drain(timeout_us=600_000_000)
    assert srv.stats()["completed"] == 2 * len(pool)
    # each pool entry alone on the idle server, in each precision: the
    # latency a request has without any other in flight (host copies included)
    alone = {}
    for e in range(len(pool)):
        for prec in (C.FP64, C.SPLITBF16):
            t = submit((e, prec, 8))
            srv.drain(timeout_us=600_000_000)
            alone[(e, prec)] = srv.poll(t)[1].latency_us / 1e3
    largest = max(alone, key=alone.get)

    # closed loop: capacity
    cap_reqs = make(max(len(pool), args.requests // 2), 10**7)
    t0 = time.perf_counter()
    tk = [submit(r) for r in cap_reqs]
    srv.drain(timeout_us=600_000_000)
    cap_s = time.perf_counter() - t0
    for t in tk:
        assert srv.poll(t) is not None
    capacity = len(cap_reqs) / cap_s

    # open loop: Poisson arrivals at load x capacity
    rate = args.load * capacity
    reqs = make(args.requests, 2 * 10**7)
    gaps = rng.exponential(1.0 / rate, size=len(reqs))
    # parity sample: the four smallest FP64 requests and two split-BF16 ones
    order = sorted(range(len(reqs)), key=lambda i: pool[reqs[i][0]][0].m * pool[reqs[i][0]][0].n)
    sample = [i for i in order if reqs[i][1] == C.FP64][:4] + \
             [i for i in order if reqs[i][1] != C.FP64][:2]
    own = {}
    for i in sample:
        w = pool[reqs[i][0]][0]
        own[i] = (torch.empty((w.n, w.m), dtype=torch.float64, pin_memory=True).t(),
                  torch.empty((w.n, w.n), dtype=torch.float64, pin_memory=True).t(),
                  torch.empty(w.n, dtype=torch.int64, pin_memory=True))
    tickets = [None] * len(reqs)
    results = {}
    stats0 = srv.stats()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    launches0 = C.kernel_launches()

    def feeder():
        t_next = time.perf_counter()
        for i, r in enumerate(reqs):
            t_next += gaps[i]
            dt = t_next - time.perf_counter()
            if dt > 0:
                time.sleep(dt)
            tickets[i] = submit(r, own.get(i))

    th = threading.Thread(target=feeder)
    t_start = time.perf_counter()
    th.start()
    pending = set(range(len(reqs)))
    t_last = t_start
    while pending:
        for i in list(pending):
            if tickets[i] is None:
                continue
            got = srv.poll(tickets[i])
            if got is not None:
                fac, res = got
                results[i] = res
                if i in own:
                    own[i] = (fac.Q.numpy()[:, :res.k].copy(), fac.R.numpy()[:res.k].copy(),
                              fac.J.numpy().copy(), res.k, res.status)
                pending.discard(i)
                t_last = time.perf_counter()
        time.sleep(0.0002)
    th.join()
    wall = t_last - t_start
    launches = C.kernel_launches() - launches0
    clk = clocks.stop()
    stats = srv.stats()
    srv.close()

    lat = np.array([results[i].latency_us for i in range(len(reqs))]) / 1e3
    que = np.array([results[i].queue_us for i in range(len(reqs))]) / 1e3
    isfp = np.array([reqs[i][1] == C.FP64 for i in range(len(reqs))])
    assert all(results[i].status in (0, 1) for i in range(len(reqs)))
    ws = [pool[r[0]][0] for r in reqs]
    ks = [results[i].k for i in range(len(reqs))]
    throughput = len(reqs) / wall
    flops = sum(cqrrpt_flops(w.m, w.n, w.d, k, w.nnz) for w, k in zip(ws, ks))
    h2d = statistics.mean(w.m * w.n * 8 for w in ws)
    d2h = statistics.mean(w.m * k * 8 + k * w.n * 8 + w.n * 8 + 8 for w, k in zip(ws, ks))

    # parity: sampled FP64 requests bit-identical to the oracle; split-BF16
    # ones: same J and k as the oracle, FP64-level residuals
    par = []
    for i in sample:
        Qs, Rs, Js, k, st = own[i]
        w = pool[reqs[i][0]][0]
        A = np.asfortranarray(hosts[reqs[i][0]].numpy())
        ref = oracle.cqrrpt(A, w.gamma, w.nnz, w.tol, reqs[i][2])
        ok = ref.k == k and np.array_equal(ref.J, Js)
        if reqs[i][1] == C.FP64:
            ok = ok and np.array_equal(ref.Q.view(np.uint64), np.asfortranarray(Qs).view(np.uint64)) \
                and np.array_equal(ref.R.view(np.uint64), np.asfortranarray(Rs).view(np.uint64))
        else:
            AJ = A[:, Js]
            rec = np.linalg.norm(AJ - Qs @ Rs) / np.linalg.norm(A)
            orth = np.linalg.norm(Qs.T @ Qs - np.eye(k), 2)
            ok = ok and rec <= 1e-12 and orth <= 1e-12
        par.append(bool(ok))

    def pct(a):
        return {"p50": float(np.percentile(a, 50)), "p99": float(np.percentile(a, 99)),
                "mean": float(a.mean())} if len(a) else None

    line = {"metric": "cqrrpt_requests_per_s", "value": throughput, "unit": "requests/s",
            "n_gpus": world, "steps": len(reqs), "warmup": 2 * len(pool),
            "ms_per_step": wall * 1e3 / len(reqs), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64 / bf16 digits -> f64", "data": "synthetic",
            "config": {"workload": "cqrrpt_serving_poisson_%dreq_pool%d_m2^12-2^20_n16-512_"
                                   "cond1e2-1e12" % (len(reqs), len(pool)),
                       "sample": "%d requests (of the 20000-request mix) drawn from %d distinct "
                                 "matrices of the mix, each with its own S seed and precision"
                                 % (len(reqs), len(pool)),
                       "requests": len(reqs), "pool_matrices": len(pool),
                       "mean_A_bytes": h2d, "hbm_budget_bytes": 120 << 30, "max_inflight": 64,
                       "offered_rate_per_s": rate, "load": args.load,
                       "precision_mix": "fp64 / splitbf16 50/50",
                       "l2": "inputs copied from host per request (mean %.0f MB), no flush"
                             % (h2d / 1e6)},
            "capacity_requests_per_s": capacity,
            "latency_ms": {"all": pct(lat), "fp64": pct(lat[isfp]), "splitbf16": pct(lat[~isfp]),
                           "queue": pct(que)},
            "standalone_ms": {"largest": alone[largest],
                              "largest_request": {"m": pool[largest[0]][0].m,
                                                  "n": pool[largest[0]][0].n,
                                                  "precision": "fp64" if largest[1] == C.FP64
                                                  else "splitbf16"},
                              "p99_over_largest": float(np.percentile(lat, 99)) / alone[largest],
                              "mean_over_requests": float(np.mean(
                                  [alone[(r[0], r[1])] for r in reqs])),
                              "note": "each pool entry run alone on the idle server (host "
                                      "copies included) before the open loop"},
            "gflops_algorithmic": flops / wall / 1e9,
            "gflops_2mn2": sum(2.0 * w.m * w.n * w.n for w in ws) / wall / 1e9,
            "units": stats["waves"] - stats0["waves"],
            "single_route_units": stats["single_units"] - stats0["single_units"],
            "batched_waves": stats["batched_units"] - stats0["batched_units"],
            "mean_wave_size": ((stats["batched_requests"] - stats0["batched_requests"])
                               / max(1, stats["batched_units"] - stats0["batched_units"])),
            "lanes": stats["lanes"], "max_units_in_flight": stats["max_busy_lanes"],
            "e2e": {"value": throughput, "unit": "requests/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h,
                    "note": "the serving loop is end to end: pinned host in, host out"},
            "parity_vs_oracle": ("%d/%d sampled requests match (fp64 bit-identical, split-BF16 "
                                 "same J/k and residuals <= 1e-12)" % (sum(par), len(par))),
            "gpu_launches": int(launches), "clocks": clk}
    return line


def run_sweep(args, world, rank, local, C):
    """The paper's speed experiment (Sec. 5.2): iid Gaussian --rows x n
    matrices, n = 512, 1024, 2048, 4096, gamma 1.25, 4 nonzeros per column,
    tol 1e-12 (full rank); per n one warm-up and --steps timed
    factorisations (at most 3) in FP64 (with the per-phase split) and in
    split-BF16.  The rate is the paper's canonical one, 2 m n^2 / time."""
    m = args.rows
    steps = max(1, min(args.steps, 3))
    stream = torch.cuda.current_stream()
    h = C.Handle(local)
    per_n = {}
    clocks = ClockSampler(local)
    clocks.start()
    t_wall = time.perf_counter()
    for n in (512, 1024, 2048, 4096):
        A = W.gaussian(m, n, W.BASE_SEED + 40 + n, "cuda")
        Q = C.colmajor_empty(m, n, A.device)
        R = C.colmajor_empty(n, n, A.device)
        J = torch.empty(n, dtype=torch.int64, device=A.device)
        rec = {}
        for prec, name in ((C.FP64, "fp64"), (C.SPLITBF16, "splitbf16")):
            res = C.cqrrpt(A, 1.25, 4, 1e-12, 7, precision=prec, out=(Q, R, J), handle=h,
                           stream=stream)
            assert res.status == 0 and res.k == n, (res.status, res.k)
            h.set_profiling(prec == C.FP64)
            ts, qr = [], []
            for _ in range(steps):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                C.cqrrpt(A, 1.25, 4, 1e-12, 7, precision=prec, out=(Q, R, J), handle=h,
                         stream=stream)
                e1.record(stream)
                torch.cuda.synchronize()
                ts.append(e0.elapsed_time(e1))
                if prec == C.FP64:
                    qr.append(h.phase_times()["qrcp"])
            h.set_profiling(False)
            ms = statistics.median(ts)
            rec[name] = {"ms": ms, "gflops_2mn2": 2.0 * m * n * n / (ms * 1e6), "k": res.k}
            if qr:
                rec[name]["qrcp_ms"] = statistics.median(qr)
                rec[name]["qrcp_share"] = statistics.median(qr) / ms
        rec["splitbf16"]["speedup_vs_fp64"] = rec["fp64"]["ms"] / rec["splitbf16"]["ms"]
        per_n[str(n)] = rec
        del A, Q, R, J
        torch.cuda.empty_cache()
    wall = time.perf_counter() - t_wall
    clk = clocks.stop()
    top = per_n["2048"]["fp64"]
    return {"metric": "cqrrpt_gflops_canonical", "value": top["gflops_2mn2"],
            "unit": "GFLOP/s (2mn^2 / time)", "n_gpus": world, "steps": steps, "warmup": 1,
            "ms_per_step": top["ms"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64 / bf16 digits -> f64", "data": "synthetic",
            "config": {"workload": "cqrrpt_sweep_gaussian_m%d_n512-4096" % m, "m": m,
                       "n": [512, 1024, 2048, 4096], "gamma": 1.25, "nnz_per_col": 4,
                       "tol": 1e-12, "value_is": "FP64 at n = 2048",
                       "l2": "inputs larger than L2, no flush"},
            "per_n": per_n, "clocks": clk, "wall_s": wall}


# --------------------------------------------------------------- our arm
def main():
    args = parse()
    world, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, world, rank)
        barrier(world)
        return
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU (the library has no CPU path)")
    torch.cuda.set_device(local)
    import paper_2311_08316_gb300 as C
    from paper_2311_08316_gb300 import build as cbuild
    cbuild.build()
    others = {"batched": run_batched, "mixed": run_mixed, "serve": run_serve,
              "dense": run_dense, "panels": run_panels, "srrqr": run_srrqr,
              "small": run_small, "sharded": run_sharded, "sweep": run_sweep}
    if args.workload in others:
        line = others[args.workload](args, world, rank, local, C)
        if rank == 0:
            print(json.dumps(line), flush=True)
        barrier(world)
        return

    w = rank_workload(W.single_large(m=args.rows), rank)
    m, n = w.m, w.n
    A = w.matrix("cuda")
    h = C.Handle(local)
    h.reserve(C.workspace_size(m, n, w.gamma, w.nnz))
    Q = C.colmajor_empty(m, n)
    R = C.colmajor_empty(n, n)
    J = torch.empty(n, dtype=torch.int64, device="cuda")
    stream = torch.cuda.current_stream()

    def step(sync):
        return C.cqrrpt(A, w.gamma, w.nnz, w.tol, w.sketch_seed, out=(Q, R, J), handle=h,
                        stream=stream, sync=sync)

    res = None
    for _ in range(args.warmup):
        res = step(True)
    assert res is not None and res.status == 0, res.status if res else None
    k = res.k

    # ---- timed region: A resident in HBM
    h.set_profiling(True)
    phases = {p: [] for p in C.PHASES}
    step_ms = []
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    barrier(world)
    torch.cuda.synchronize()
    launches0 = C.kernel_launches()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        step(False)
        pt = h.phase_times()        # waits for this step's last phase event
        for p, v in pt.items():
            phases[p].append(v)
        step_ms.append(sum(pt.values()))
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    elapsed_ms = ev0.elapsed_time(ev1)
    launches = C.kernel_launches() - launches0
    clk = clocks.stop()
    h.set_profiling(False)
    st, k2 = h.last_status()
    assert st == 0 and k2 == k

    elapsed_ms = max_over_ranks(elapsed_ms, world, "cuda")
    ms_per_step = elapsed_ms / args.steps
    value = world * args.steps / (elapsed_ms / 1e3)

    # ---- roofline of the dominant kernel (trsm_rut_kernel: lines 4 and 7)
    trsm_ms = (statistics.mean(phases["trsm_pre"]) + statistics.mean(phases["trsm_q"])) / 2
    trsm_flops = float(m) * k * k          # k^2/2 fma per row, 2 flop each
    achieved = trsm_flops / (trsm_ms * 1e-3) / 1e9
    try:
        probe_gflops, _ = C.probe_fp64_gflops(local)
    except Exception:
        probe_gflops = None
    roof = {"kernel": "trsm_rut_kernel", "bound": "alu", "achieved": achieved,
            "peak": FP64_PEAK_GFLOPS, "unit": "GFLOP/s", "frac": achieved / FP64_PEAK_GFLOPS,
            "peak_probe_measured": probe_gflops,
            "frac_of_probe": (achieved / probe_gflops) if probe_gflops else None,
            "traffic": TRSM_DRAM_BYTES_HEADLINE if (m, n, k) == (131072, 1024, 800) else None,
            "algorithmic_flops_per_launch": trsm_flops,
            "launch_ms": trsm_ms,
            "peak_note": "FP64 ALU: 152 SM x 2 DFMA/clk x 2 flop x 2.07 GHz (derived, nominal)"}
    alg_flops = (2.0 * m * k * k + m * k * (k + 1) + 4.0 * w.d * n * k - 2.0 * k * k * (w.d + n)
                 + 5.0 * k ** 3 / 3.0)   # paper's count (Sec. 2.1), plus sketch adds below
    alg_flops += float(m) * w.nnz * n
    phase_share = {p: statistics.mean(v) / (ms_per_step) for p, v in phases.items()}

    # ---- the same input in the split-BF16 mode (lines 4, 5, 7 on the
    # tensor cores): time and accuracy next to the FP64 result
    split = None
    try:
        Qs = C.colmajor_empty(m, n)
        Rs = C.colmajor_empty(n, n)
        Js = torch.empty(n, dtype=torch.int64, device="cuda")
        rs = C.cqrrpt(A, w.gamma, w.nnz, w.tol, w.sketch_seed, precision=C.SPLITBF16,
                      out=(Qs, Rs, Js), handle=h, stream=stream)
        ms_s = []
        for _ in range(3):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            rs = C.cqrrpt(A, w.gamma, w.nnz, w.tol, w.sketch_seed, precision=C.SPLITBF16,
                          out=(Qs, Rs, Js), handle=h, stream=stream)
            e1.record(stream)
            torch.cuda.synchronize()
            ms_s.append(e0.elapsed_time(e1))
        ks = rs.k
        recon = (torch.linalg.norm(A[:, Js] - Qs[:, :ks] @ Rs[:ks]) / torch.linalg.norm(A)).item()
        orth = torch.linalg.matrix_norm(Qs[:, :ks].t() @ Qs[:, :ks]
                                        - torch.eye(ks, dtype=torch.float64, device="cuda"),
                                        ord=2).item()
        split = {"ms": statistics.median(ms_s), "factorizations_per_s": 1e3 / statistics.median(ms_s),
                 "speedup_vs_fp64": ms_per_step / statistics.median(ms_s), "k": ks,
                 "J_equal_fp64": bool(torch.equal(Js, J)), "recon_rel_F": recon, "orth_2": orth}
        del Qs, Rs, Js
    except Exception as ex:  # reported, not hidden
        split = {"error": str(ex)}

    # ---- the implicit Q (Alg. 2 without line 7): the factorisation returns
    # M^pre and R^pre; Q X and Q^T Y are applied to 16 right-hand sides
    implicit = None
    try:
        Ap = C.colmajor_empty(m, n)
        Rp = C.colmajor_empty(n, n)
        Ri = C.colmajor_empty(n, n)
        Ji = torch.empty(n, dtype=torch.int64, device="cuda")
        imp = C.cqrrpt_implicit(A, w.gamma, w.nnz, w.tol, w.sketch_seed, out=(Ap, Rp, Ri, Ji),
                                handle=h, stream=stream)
        Xr = torch.randn(16, imp.k, dtype=torch.float64, device="cuda").t()
        Yr = torch.randn(16, m, dtype=torch.float64, device="cuda").t()
        ms_i, ms_q, ms_qt = [], [], []
        for _ in range(3):
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
            ev[0].record(stream)
            imp = C.cqrrpt_implicit(A, w.gamma, w.nnz, w.tol, w.sketch_seed, out=(Ap, Rp, Ri, Ji),
                                    handle=h, stream=stream)
            ev[1].record(stream)
            yq = imp.apply_q(Xr, stream=stream)
            ev[2].record(stream)
            zq = imp.apply_qt(Yr, stream=stream)
            ev[3].record(stream)
            torch.cuda.synchronize()
            ms_i.append(ev[0].elapsed_time(ev[1]))
            ms_q.append(ev[1].elapsed_time(ev[2]))
            ms_qt.append(ev[2].elapsed_time(ev[3]))
        implicit = {"ms": statistics.median(ms_i),
                    "factorizations_per_s": 1e3 / statistics.median(ms_i),
                    "speedup_vs_explicit_q": ms_per_step / statistics.median(ms_i),
                    "k": imp.k, "R_and_J_equal_explicit": bool(torch.equal(Ri[:k], R[:k])
                                                               and torch.equal(Ji, J)),
                    "apply_q_16rhs_ms": statistics.median(ms_q),
                    "apply_qt_16rhs_ms": statistics.median(ms_qt),
                    "apply_q_vs_explicit_max_abs": (yq - Q[:, :k] @ Xr).abs().max().item()}
        del Ap, Rp, Ri, Ji, Xr, Yr, yq, zq
    except Exception as ex:  # reported, not hidden
        implicit = {"error": str(ex)}

    # ---- e2e through the public API with host buffers
    A_host = torch.empty((n, m), dtype=torch.float64, pin_memory=True).t()
    A_host.copy_(A)
    Qh = torch.empty((n, m), dtype=torch.float64, pin_memory=True).t()
    Rh = torch.empty((n, n), dtype=torch.float64, pin_memory=True).t()
    Jh = torch.empty(n, dtype=torch.int64, pin_memory=True)
    del A
    Ad = C.colmajor_empty(m, n)
    e2e_ms = []
    for i in range(args.warmup + args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        out = C.cqrrpt_from_host(A_host, w.gamma, w.nnz, w.tol, w.sketch_seed, out_host=(Qh, Rh, Jh),
                                 device_buffers=(Ad, Q, R, J), handle=h, stream=stream)
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            e2e_ms.append(dt * 1e3)
    assert out.k == k
    one_call_step = max_over_ranks(statistics.mean(e2e_ms), world)
    # the host pipeline: copies in, factorisations and copies out overlap;
    # every step still copies its A in and its Q, R, J out (two output
    # buffer sets, used in turn)
    outs = [(Qh, Rh, Jh)] + [(torch.empty((n, m), dtype=torch.float64, pin_memory=True).t(),
                              torch.empty((n, n), dtype=torch.float64, pin_memory=True).t(),
                              torch.empty(n, dtype=torch.int64, pin_memory=True))]
    C.cqrrpt_host_pipeline([A_host] * max(args.warmup, 2), w.gamma, w.nnz, w.tol,
                           [w.sketch_seed] * max(args.warmup, 2),
                           outs_host=[outs[i % 2] for i in range(max(args.warmup, 2))],
                           handle=h, stream=stream)
    torch.cuda.synchronize()
    barrier(world)
    t0 = time.perf_counter()
    pres = C.cqrrpt_host_pipeline([A_host] * args.steps, w.gamma, w.nnz, w.tol,
                                  [w.sketch_seed] * args.steps,
                                  outs_host=[outs[i % 2] for i in range(args.steps)],
                                  handle=h, stream=stream)
    torch.cuda.synchronize()
    e2e_step = max_over_ranks((time.perf_counter() - t0) * 1e3 / args.steps, world)
    assert all(r.k == k and r.status == 0 for r in pres)
    h2d = m * n * 8
    d2h = m * k * 8 + k * n * 8 + n * 8

    line = {"metric": "cqrrpt_factorizations_per_s", "value": value, "unit": "factorizations/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": config_of(w),
            "k": k,
            "gflops_2mn2": value * 2.0 * m * n * n / 1e9,
            "gflops_geqrf_basis": value * (2.0 * m * n * n - 2.0 * n ** 3 / 3.0) / 1e9,
            "gflops_algorithmic": value * alg_flops / 1e9,
            "latency_ms": {"p50": float(np.percentile(step_ms, 50)),
                           "p99": float(np.percentile(step_ms, 99))},
            "phase_share": phase_share,
            "roofline": roof,
            "e2e": {"value": world * 1e3 / e2e_step, "unit": "factorizations/s",
                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "ms_per_step": e2e_step, "api": "cqrrpt_host_pipeline_d",
                    "one_call_per_matrix_ms_per_step": one_call_step},
            "gpu_launches": int(launches),
            "clocks": clk,
            "splitbf16_same_input": split,
            "implicit_q": implicit}

    # ---- CPU baseline: the oracle on the full workload (rank 0, N = 1 only)
    if rank == 0 and world == 1:
        import oracle
        Ahost = np.asfortranarray(A_host.numpy())
        t0 = time.perf_counter()
        ref = oracle.cqrrpt(Ahost, w.gamma, w.nnz, w.tol, w.sketch_seed)
        t = time.perf_counter() - t0
        same = (ref.k == out.k and np.array_equal(ref.J, Jh.numpy())
                and np.array_equal(ref.Q.view(np.uint64),
                                   np.asfortranarray(Qh[:, :k].numpy()).view(np.uint64))
                and np.array_equal(ref.R.view(np.uint64),
                                   np.asfortranarray(Rh[:k, :].numpy()).view(np.uint64)))
        line["cpu_baseline"] = {"value": 1.0 / t, "unit": "factorizations/s",
                                "cores": cpu_threads(), "cpu_model": cpu_model(),
                                "kind": "oracle",
                                "sample": "the full workload, one factorisation (%.1f s)" % t}
        line["parity_vs_oracle"] = "bit-identical J, k, Q, R" if same else "MISMATCH"
        del Ahost, ref

    # ---- the other workloads, measured in the same run (N = 1 only): the
    # small latency case, the mixed-precision case, the batched case and a
    # shortened serving run; each with its own clocks and parity check
    if world == 1 and args.configs == "all":
        import argparse as _ap
        h.close()
        del A_host, Qh, Rh, Jh, Ad, Q, R, J, outs, pres, out
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
        subs = {}
        plan = [("small_m4096_n64", run_small, dict(steps=200, warmup=3)),
                ("mixed_m1048576_n512", run_mixed, dict(steps=5, warmup=1, rows=131072)),
                ("batched_512", run_batched, dict(steps=3, warmup=2, batch=512)),
                ("serving_poisson", run_serve, dict(steps=1, warmup=0, requests=200, pool=32,
                                                    load=0.7))]
        for name, fn, over in plan:
            sub = _ap.Namespace(**vars(args))
            for key, v in over.items():
                setattr(sub, key, v)
            t0 = time.perf_counter()
            try:
                rec = fn(sub, world, rank, local, C)
            except Exception as ex:  # reported, not hidden
                rec = {"error": "%s: %s" % (type(ex).__name__, ex)}
            rec["wall_s"] = time.perf_counter() - t0
            subs[name] = rec
            torch.cuda.synchronize()
            torch.cuda.empty_cache()
        line["configs"] = subs
    if rank == 0:
        print(json.dumps(line), flush=True)
    barrier(world)


if __name__ == "__main__":
    main()
