#!/usr/bin/env python
"""Benchmark: DOF*timesteps/s to MGRIT relative residual 1e-10.

Workload (multilevel MGRIT on the unit square): heat equation u_t = Laplace u + f,
manufactured solution u = sin(pi x) sin(pi y) cos t, B-splines of order
p in {2,3,4,5} on 64 x 64 elements (N = (62+p)^2 interior unknowns), backward
Euler with N_t = 256 steps on [0,1], MGRIT with m = 4 down to <= 4 coarse steps
(256 -> 64 -> 16 -> 4), FCF relaxation, p-multigrid V(1,1) spatial solves to
relative residual 1e-10.  One "step" of the benchmark = one MGRIT solve for
each of the four orders (a unit of work = N_p * N_t DOF*timesteps, summed).

Forms: "chosen" = FP32 smoothing / SpMM / transfers / Gauss--Seidel with FP64
residual refinement (precision 1), one p-multigrid cycle per coarse-level solve,
sweep layouts autotuned at setup; "mixed_only" = the same precision split with
every level solved to 1e-10; "plain" = everything FP64 (precision 0) to 1e-10
on every level.  The value is the chosen form's throughput; the other two are
reported beside it, so that the speed-up over the plain form splits into its
precision and coarse-propagator parts.  Every form's iterate of the last timed
step is compared with the oracle's sequential backward Euler (the fixed point of
MGRIT, Sec. 3) per order ("error_vs_oracle").  The default run also measures the
curved-map workload annulus_c3 ("annulus_c3", with its own roofline and error),
the CPU baseline (the oracle on a bounded sample of heat_c2, on one core and as
independent replicas on every host core) and, in a child process with a time
limit, the uneven batch batch_c5 in one persistent launch ("batch_c5").

Other modes (one JSON line each): --annulus (the curved-map workload annulus_c3),
--batch (the uneven 64-problem batch, latency percentiles), --learned (two-level
MGRIT with the trained coarse propagator against backward Euler and the plain
form), --spmm (the batched FP32 operator apply against the HBM copy bandwidth),
--trace (the per-phase clock split of one p-multigrid cycle), --profile-only (per-launch grids
and V-cycles, to pair with ncu), and
--impl reference (the oracle timed on the host cores).
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "DOF*timesteps/s to MGRIT rel. residual 1e-10, chosen vs plain FP64 form"
UNIT = "DOF*timesteps/s"


_T0 = time.perf_counter()


def log(msg):
    """Progress of the run on stderr (the JSON line stays alone on stdout)."""
    sys.stderr.write(f"[bench +{time.perf_counter() - _T0:7.1f} s] {msg}\n")
    sys.stderr.flush()


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--orders", default="2,3,4,5")
    ap.add_argument("--nel", type=int, default=64)
    ap.add_argument("--Nt", type=int, default=256)
    ap.add_argument("--skip-plain", action="store_true")
    ap.add_argument("--skip-check", action="store_true")
    ap.add_argument("--skip-cpu", action="store_true",
                    help="skip the CPU baseline leg (oracle timings and the errors against it)")
    ap.add_argument("--skip-extra", action="store_true",
                    help="leave the batch_c5 sub-object (a child process) out of the default run")
    ap.add_argument("--skip-annulus", action="store_true",
                    help="skip the annulus_c3 sub-measurement of the default run")
    ap.add_argument("--sjf", type=int, default=1,
                    help="--batch: 1 = shortest-job-first stream priorities (default), 0 = equal")
    ap.add_argument("--batch-order", default="shortest", choices=["shortest", "longest"],
                    help="--batch: the order in which the persistent launch's idle CTAs look "
                         "for work (shortest first: low latency; longest first: short makespan)")
    ap.add_argument("--learned", action="store_true",
                    help="learned_c4: two-level MGRIT with the learned coarse propagator against "
                         "backward Euler on the coarse level, one JSON line (not the headline)")
    ap.add_argument("--annulus", action="store_true",
                    help="annulus_c3 (curved map, N = 16900, N_t = 1024, m = 8): chosen form, "
                         "throughput and the sweep kernel's roofline")
    ap.add_argument("--spmm", action="store_true",
                    help="batched FP32 operator apply (iga_apply_f32) on 8192 columns: achieved "
                         "HBM GB/s against the measured peak, one JSON line per order")
    ap.add_argument("--batch", action="store_true",
                    help="the uneven 64-problem batch (batch_c5): per-problem latency p50/p99 "
                         "and batch throughput, one JSON line (not the headline metric)")
    ap.add_argument("--trace", action="store_true",
                    help="per-phase clock split of one p-multigrid cycle (pmg_trace) at 64 x 64 "
                         "elements, p = 2..5, both forms, with the untraced cycle time")
    ap.add_argument("--profile-only", action="store_true",
                    help="one chosen-form solve per order and exit (for ncu launch lists)")
    return ap.parse_args()


def manufactured():
    import numpy as np
    S = lambda xi, eta, x, y: np.sin(np.pi * x) * np.sin(np.pi * y)
    C = lambda t: 2 * np.pi ** 2 * np.cos(t) - np.sin(t)
    return S, C


# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per launch of the
# dominant kernel, averaged over the launches of one chosen-form solve per
# order of the workload at its full size (the per-launch profiled solves of
# --profile-only), from one single-pass ncu capture of that command.  Must be
# re-captured whenever k_mgrit_sweep changes.
NCU_DRAM_BYTES_PER_LAUNCH = {"heat_c2": 9.538e6, "annulus_c3": 1.077e9}


def bytes_per_vcycle_dof(p, B):
    """Algorithmic bytes of one V(1,1) per DOF per right-hand side (8-byte
    values; matrices amortised over the B right-hand sides of a launch):
    3 residual products + 2 ILUT sweeps (L and U) + 2 order transfers plus the
    p = 1 W-cycle and vector traffic."""
    q = (2 * p + 1) ** 2
    return (3 * 8 * q + 2 * 12 * q + 2 * 8 * (p + 2) ** 2) / max(B, 1) + 300.0


def job_time_ms(local_total_ms, world, device="cpu"):
    """Length of a timed region for the whole job: the maximum over ranks (every
    rank's steps must have finished)."""
    if world > 1:
        import torch
        t = torch.tensor([float(local_total_ms)], dtype=torch.float64, device=device)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        return float(t.item())
    return float(local_total_ms)


def job_throughput(units_per_rank, world, steps, total_ms):
    """Whole-job throughput: every rank processed units_per_rank per step (the
    ranks run independent replicas of the workload, weak scaling)."""
    return world * units_per_rank * steps / (total_ms * 1e-3)


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, dev):
        self.dev = dev
        self.proc = None
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        try:
            rows = [l.split(",") for l in open(self.f.name).read().strip().splitlines() if l.strip()]
        except OSError:
            rows = []
        os.unlink(self.f.name)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4)
                          if len(r) > 5 + k and r[5 + k].strip().lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return None


# ---------------------------------------------------------------------------
# CPU baseline leg: the only part of this file that runs the oracle.  The
# oracle runs in processes started with "spawn" (never forked from a process
# that has used the GPU), one solve per process, BLAS threads pinned to 1.
# ---------------------------------------------------------------------------
SAMPLE = dict(p=2, nel=64, Nt=32)   # bounded sample of heat_c2 for the CPU legs


def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else the ISA)."""
    import platform
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return platform.machine()


def _single_thread_env():
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[k] = "1"


def _oracle_replica(p, nel, Nt, cmd, res):
    """Worker: build the oracle's MGRIT with p-multigrid spatial solves for the
    sample (setup: assembly and ILUT per time level), then one timed solve to
    MGRIT tolerance 1e-10 per command received; None ends it."""
    import numpy as np
    from oracle import assembly, geometry, mgrit
    S, C = manufactured()
    hi, lo = assembly.problem(p, nel, geometry.UnitSquare())
    u0, fhat = hi.project(S), hi.load_vector(S)
    fac = mgrit.pmg_factory(hi, lo, tol=1e-10)
    cache = {}
    mk = lambda l, c: cache.setdefault(l, fac(l, c))
    mgrit.MGRIT(hi.M, hi.K, 1.0, 1.0, Nt, 4, mk, u0, fhat, C)   # builds every level's solver
    res.put(("ready", hi.N))
    while cmd.get() is not None:
        mg = mgrit.MGRIT(hi.M, hi.K, 1.0, 1.0, Nt, 4, mk, u0, fhat, C)
        t0 = time.perf_counter()
        _, it, _ = mg.run(tol=1e-10)
        res.put(("done", time.perf_counter() - t0, it))


class OracleReplicas:
    """`cores` independent replicas of the oracle sample, one spawned process
    each (weak scaling over host cores, like the GPU replicas of --gpus N)."""

    def __init__(self, cores, p=SAMPLE["p"], nel=SAMPLE["nel"], Nt=SAMPLE["Nt"]):
        import multiprocessing as mp
        _single_thread_env()
        ctx = mp.get_context("spawn")
        self.cores, self.p, self.nel, self.Nt = cores, p, nel, Nt
        self.res = ctx.Queue()
        self.cmds = [ctx.Queue() for _ in range(cores)]
        self.procs = [ctx.Process(target=_oracle_replica, args=(p, nel, Nt, q, self.res), daemon=True)
                      for q in self.cmds]
        for pr in self.procs:
            pr.start()
        self.N = None
        for _ in range(cores):
            tag, N = self.res.get(timeout=1800)
            assert tag == "ready"
            self.N = N

    def step(self):
        """Wall seconds for every replica to finish one solve (the units of
        work are cores * N * N_t)."""
        t0 = time.perf_counter()
        for q in self.cmds:
            q.put(1)
        its = [self.res.get(timeout=1800)[2] for _ in range(self.cores)]
        return time.perf_counter() - t0, its

    def desc(self):
        from oracle import mgrit
        return (f"oracle MGRIT (NumPy/SciPy FP64, p-multigrid spatial solves) on p={self.p}, "
                f"{self.nel}x{self.nel} elements, N_t={self.Nt} (levels "
                f"{mgrit.level_sizes(self.Nt, 4)}), tol 1e-10; {self.cores} independent "
                f"replica(s), one spawned process per core, BLAS threads 1; setup excluded; "
                f"CPU: {cpu_model()}")

    def close(self):
        for q in self.cmds:
            q.put(None)
        for pr in self.procs:
            pr.join(timeout=30)


def cpu_baseline_leg():
    """The oracle on one core and on all host cores (same bounded sample)."""
    cores = os.cpu_count() or 1
    one = OracleReplicas(1)
    t1, _ = one.step()
    one.close()
    allc = OracleReplicas(cores)
    ta, _ = allc.step()
    desc = allc.desc()
    units = allc.N * allc.Nt
    allc.close()
    return {"value": cores * units / ta, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": desc, "cpu": cpu_model(),
            "single_thread": {"value": units / t1, "cores": 1, "seconds": round(t1, 3)}}


def _oracle_sequential(job):
    """Sequential backward Euler with sparse direct spatial solves (the result
    MGRIT converges to, Sec. 3) for one benchmarked problem."""
    _single_thread_env()
    import numpy as np
    from oracle import assembly, geometry, timestep
    from paper_2107_05337_gb300 import inputs
    S, C = manufactured()
    if job[0] == "heat_c2":
        _, p, nel, Nt = job
        d = assembly.Discretisation(p, nel, geometry.UnitSquare())
        return timestep.sequential(d.M, d.K, 1.0, 1.0, Nt, d.project(S), d.load_vector(S), C)
    w = inputs.WORKLOADS["annulus_c3"]
    k, l, a = inputs.fourier_modes()
    u0fn = lambda xi, eta, x, y: sum(a[s] * np.sin(k[s] * np.pi * xi) * np.sin(l[s] * np.pi * eta)
                                     for s in range(len(a)))
    d = assembly.Discretisation(w["p"][0], w["nel"], geometry.get(w["geom"]))
    return timestep.sequential(d.M, d.K, 1.0, w["T"], w["Nt"], d.project(u0fn))


def oracle_references(jobs):
    """Start the oracle's sequential solutions of the benchmarked problems in
    spawned processes (they run while the GPU is timed and are collected
    afterwards; nothing of them is timed).  Returns {job: future}."""
    import multiprocessing as mp
    from concurrent.futures import ProcessPoolExecutor
    _single_thread_env()
    ex = ProcessPoolExecutor(max_workers=len(jobs), mp_context=mp.get_context("spawn"))
    return ex, {job: ex.submit(_oracle_sequential, job) for job in jobs}


def rel_err(U, ref):
    import numpy as np
    return float(np.linalg.norm(U - ref) / np.linalg.norm(ref))


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    # each step = every host core solving the bounded sample once (independent replicas)
    cores = os.cpu_count() or 1
    reps = OracleReplicas(cores)
    for _ in range(args.warmup):
        reps.step()
    t = sum(reps.step()[0] for _ in range(args.steps))
    units = reps.N * reps.Nt * cores
    desc = reps.desc()
    reps.close()
    v = units * args.steps / t
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": f"heat_c2 bounded sample (p={SAMPLE['p']}, nel={SAMPLE['nel']}, "
                                   f"N_t={SAMPLE['Nt']}), {cores} replicas"},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def run_batch(args):
    print(json.dumps(batch_measure(args.steps, args.warmup, args.sjf, args.batch_order,
                                   host_arm=not args.skip_plain)))


def batch_measure(steps, warmup, sjf=1, batch_order="shortest", host_arm=True):
    """batch_c5: 64 independent problems (inputs.batch_members) in the chosen
    (mixed) form, solved in one persistent launch (mgrit_run_batched_device)
    and, beside it (host_arm), by streams with a host scheduler
    (mgrit_run_batched).  Reports the per-problem latency distribution from the
    batch start and the batch throughput sum(N * N_t) / makespan.  L2 is
    flushed before every timed batch."""
    import numpy as np
    import torch
    from concurrent.futures import ThreadPoolExecutor
    from paper_2107_05337_gb300 import binding as B
    from paper_2107_05337_gb300 import inputs
    torch.cuda.set_device(0)
    members = inputs.batch_members()
    probs, u0s = [], []
    for mb in members:
        pr = B.Problem(mb["p"], mb["nel"], kappa=mb["kappa"])
        k, l, a = inputs.fourier_modes(seed=mb["modes_seed"], count=16)
        fn = lambda xi, eta, x, y, k=k, l=l, a=a: sum(
            a[s] * np.sin(k[s] * np.pi * xi) * np.sin(l[s] * np.pi * eta) for s in range(len(a)))
        probs.append(pr)
        u0s.append(pr.project(fn))
    # shortest job first: members with less work (N * N_t) get higher stream
    # priority (six levels by work rank), so small problems finish early
    work = [pr.N * mb["Nt"] for pr, mb in zip(probs, members)]
    order = sorted(range(len(members)), key=lambda i: work[i])
    prio = [0] * len(members)
    for r, i in enumerate(order):
        prio[i] = 5 - (6 * r) // len(members) if sjf else 0
    t0 = time.perf_counter()
    # (fused = 0: a fused visit's cooperative launch needs all its CTAs resident at
    # once, which serialises members running on concurrent streams; the
    # persistent batch does not use it)
    mk = lambda i: B.MGRIT(probs[i], T=members[i]["T"], Nt=members[i]["Nt"], m=members[i]["m"],
                           tol=1e-10, max_iter=100, priority=prio[i], coarse_cycles=1, fused=0,
                           pmg=dict(precision=1, tol=1e-10, autotune=1))
    with ThreadPoolExecutor(max_workers=16) as ex:
        handles = list(ex.map(mk, range(len(members))))
    setup_s = time.perf_counter() - t0
    log(f"batch_c5: {len(handles)} members set up in {setup_s:.1f} s")
    Us = [torch.empty((h.Nt + 1, h.problem.N), dtype=torch.float64, device="cuda") for h in handles]
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    units = sum(pr.N * mb["Nt"] for pr, mb in zip(probs, members))
    def measure(device, hs, u0l, Ul):
        lats, spans, iters = [], [], []
        for rep in range(warmup + steps):
            flush.fill_(1.0)
            torch.cuda.synchronize()
            _, stats, lat, status = B.mgrit_run_batched(hs, u0l, Us=Ul, device=device)
            torch.cuda.synchronize()
            log(f"batch_c5: {'device' if device else 'host'}-scheduled run {rep}, "
                f"makespan {float(lat.max()):.0f} ms")
            if rep >= warmup:
                lats.extend(lat.tolist())
                spans.append(float(lat.max()))
                iters = [st["iters"] for st in stats]
        return np.array(lats), float(np.mean(spans)), iters

    # one persistent launch for the whole batch (members in shortest-first
    # order, the order in which idle CTAs look for work)
    dev_order = order if batch_order == "shortest" else order[::-1]
    lat_d, span_d, iters_d = measure(True, [handles[i] for i in dev_order],
                                     [u0s[i] for i in dev_order], [Us[i] for i in dev_order])
    # streams and a host scheduler, with shortest-job-first stream priorities
    host_sched = None
    if host_arm:
        lat, makespan, iters = measure(False, handles, u0s, Us)
        host_sched = {"value": units / (makespan * 1e-3), "makespan_ms": makespan,
                      "latency_ms": {"p50": float(np.percentile(lat, 50)),
                                     "p99": float(np.percentile(lat, 99)), "max": float(lat.max())},
                      "scheduling": "streams + host scheduler, shortest job first (stream priorities)"
                      if sjf else "streams + host scheduler, equal priorities"}
    lat, makespan, iters = lat_d, span_d, iters_d
    line = {"metric": "DOF*timesteps/s of an uneven 64-problem batch to MGRIT rel. residual 1e-10",
            "value": units / (makespan * 1e-3), "unit": "DOF*timesteps/s", "n_gpus": 1,
            "steps": steps, "warmup": warmup, "higher_is_better": True,
            "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": "batch_c5: 64 problems, h in {1/32,1/64,1/128}, p in 2..5, "
                                   "N_t in {128..2048}, kappa log-uniform [0.1,10], f=0, m=4, "
                                   "16-mode random initial conditions, seed 20210714",
                       "l2": "flushed (256 MiB write) before every timed batch"},
            "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                           "max": float(lat.max())},
            "makespan_ms": makespan, "setup_s": round(setup_s, 2),
            "scheduling": f"one persistent launch (device work claiming, members scanned "
                          f"{batch_order} first, device-side stopping tests)",
            "host_scheduled": host_sched,
            "form": "mixed precision, one p-MG cycle per coarse-level solve, autotuned sweep layouts",
            "iters": {"min": int(min(iters)), "max": int(max(iters))}, "members": len(members)}
    del handles, Us, flush
    return line


def run_learned(args):
    print(json.dumps(learned_measure(args.steps, plain_arm=not args.skip_plain)))


def extra_child(mode_args, timeout_s):
    """One of the standalone measurement modes in a child process (a fresh CUDA
    context, as when it runs alone), its JSON line as a dict; a child that does
    not finish within timeout_s seconds is killed and reported unavailable."""
    cmd = [sys.executable, os.path.abspath(__file__)] + mode_args
    t0 = time.perf_counter()
    try:
        r = subprocess.run(cmd, capture_output=True, text=True, timeout=timeout_s)
    except subprocess.TimeoutExpired:
        return {"unavailable": f"{' '.join(mode_args)}: did not finish within {timeout_s} s"}
    if r.returncode != 0:
        tail = r.stderr.strip().splitlines()[-1:] or [""]
        return {"unavailable": f"{' '.join(mode_args)}: exit {r.returncode}: {tail[0][:200]}"}
    try:
        line = json.loads(r.stdout.strip().splitlines()[-1])
    except (ValueError, IndexError):
        return {"unavailable": f"{' '.join(mode_args)}: no JSON line"}
    line["child_seconds"] = round(time.perf_counter() - t0, 1)
    return line


def learned_measure(steps, plain_arm=True):
    """learned_c4: unit square, p = 3, 64 x 64 elements, N_t = 4096, T = 4,
    two-level MGRIT with m = 8, f = 0.  Training pairs (u_n, u_{n+8}) come from
    the fine stepper (sequential backward Euler through the library) on five
    16-mode random initial conditions; the network is trained with the BF16
    kernels; then the same two-level MGRIT (chosen form) is timed on a sixth
    initial condition with the learned coarse propagator and with backward
    Euler on the coarse level, and (plain_arm) the plain FP64 form with
    backward Euler."""
    import numpy as np
    import torch
    from paper_2107_05337_gb300 import binding as B
    from paper_2107_05337_gb300 import inputs
    torch.cuda.set_device(0)
    w = inputs.WORKLOADS["learned_c4"]
    p, nel, T, Nt, m = w["p"][0], w["nel"], w["T"], w["Nt"], w["m"]
    prob = B.Problem(p, nel)

    def ic(seed):
        k, l, a = inputs.fourier_modes(seed=seed, count=w["modes"])
        return prob.project(lambda xi, eta, x, y: sum(
            a[s] * np.sin(k[s] * np.pi * xi) * np.sin(l[s] * np.pi * eta) for s in range(len(a))))

    t0 = time.perf_counter()
    seq = B.MGRIT(prob, T=T, Nt=Nt, m=m, max_levels=1, pmg=dict(precision=1, tol=1e-10))
    U0s, U1s = [], []
    for i in range(w["train_ics"] - 1):
        U, _, _ = seq.run(ic(w["seed"] + i))
        U0s.append(U[:-m].clone())
        U1s.append(U[m:].clone())
    # rough pairs: m fine steps from white noise (all columns solved at once),
    # so that the network also learns how the fine stepper damps rough modes
    gen = torch.Generator(device="cuda").manual_seed(w["seed"])
    X0 = torch.randn((Nt, prob.N), dtype=torch.float64, device="cuda", generator=gen)
    stepper = B.PMG(prob, T / Nt, precision=1, tol=1e-10)
    X = X0.clone()
    for _ in range(m):
        rhs = prob.apply("M", X)
        stepper.solve(rhs, X)
    U0s.append(X0)
    U1s.append(X)
    U0, U1 = torch.cat(U0s), torch.cat(U1s)
    npairs = int(U0.shape[0])
    gen_s = time.perf_counter() - t0
    log(f"learned_c4: {npairs} training pairs in {gen_s:.1f} s")
    phic = B.Phic(prob.n, 32, seed=w["seed"])
    t0 = time.perf_counter()
    steps = 3000
    loss = phic.train(U0, U1, steps=steps, batch=32, lr=2e-3, seed=1)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    log(f"learned_c4: trained in {train_s:.1f} s")
    del U0, U1, U0s, U1s
    u0 = ic(w["seed"] + 100)
    Uref, _, _ = seq.run(u0)
    Uref = Uref.clone()
    units = prob.N * Nt

    def timed(make):
        """A warm-up run, then each timed run on a handle of its own (made before
        its timing starts): a second run on one handle of the learned form
        stalled on the GPU (open), a handle's first run converges."""
        make().run(u0, check=False)
        torch.cuda.synchronize()
        ms = []
        st = None
        status = 0
        for _ in range(max(1, steps)):
            h = make()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            U, st, status = h.run(u0, check=False)
            e1.record()
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
            del h
        err = float(torch.linalg.norm(U - Uref) / torch.linalg.norm(Uref))
        return float(np.mean(ms)), st, err, status

    common = dict(T=T, Nt=Nt, m=m, max_levels=2, tol=1e-10, max_iter=100)

    def make_learned():
        h = B.MGRIT(prob, **common, coarse_cycles=1, pmg=dict(precision=1, tol=1e-10))
        h.set_coarse_propagator(phic, 0.5)
        return h

    arms = [("learned", make_learned),
            ("backward_euler", lambda: B.MGRIT(prob, **common, coarse_cycles=1,
                                               pmg=dict(precision=1, tol=1e-10)))]
    if plain_arm:
        arms.append(("plain_fp64", lambda: B.MGRIT(prob, **common, pmg=dict(precision=0, tol=1e-10))))
    res = {}
    for name, make in arms:
        ms, st, err, status = timed(make)
        log(f"learned_c4: {name} {ms:.0f} ms, {st['iters']} iterations")
        hist = st["res_hist"]
        res[name] = {"value": units / (ms * 1e-3), "ms": ms, "iters": st["iters"],
                     "status": status, "coarse_fallback": st["coarse_fallback"],
                     "error_vs_sequential": err,
                     "contraction": [round(hist[k + 1] / hist[k], 4) for k in range(min(12, len(hist) - 1))]}
    line = {"metric": "DOF*timesteps/s, two-level MGRIT with a learned coarse propagator",
            "value": res["learned"]["value"], "unit": "DOF*timesteps/s", "n_gpus": 1,
            "higher_is_better": True, "dtype": "bf16 (network) + f32/f64 (solves)",
            "data": "synthetic",
            "config": {"workload": "learned_c4: unit square, p=3, nel=64, N_t=4096, T=4, m=8, "
                                   "two levels, f=0, 16-mode random initial conditions"},
            "runs": res,
            "speedup_vs_backward_euler_coarse": res["learned"]["value"] / res["backward_euler"]["value"],
            "speedup_vs_plain_fp64": (res["learned"]["value"] / res["plain_fp64"]["value"]
                                      if plain_arm else None),
            "training": {"pairs": npairs, "steps": steps, "batch": 32,
                         "seconds": round(train_s, 2), "data_seconds": round(gen_s, 2),
                         "loss_first": float(np.mean(loss[:20])), "loss_last": float(np.mean(loss[-20:]))},
            "steps": max(1, steps)}
    del arms, phic, seq, stepper, X, X0, Uref
    return line


def annulus_measure(steps, warmup, profile_only=False):
    """annulus_c3: quarter annulus (cubic Bezier arc x radial line), p = 4, 128 x 128
    elements (N = 16900), kappa = 1, T = 1, N_t = 1024, m = 8 (1024 -> 128 -> 16 -> 2),
    f = 0, 8-mode Fourier initial condition (seed 20210712).  Chosen form (FP32
    p-multigrid cycles with FP64 refinement, one cycle per coarse-level solve,
    autotuned sweep layouts) to MGRIT relative residual 1e-10: DOF*timesteps/s over
    `steps` solves after `warmup`, and the V-cycle-model GB/s of k_mgrit_sweep from a
    per-launch profiled solve, against the measured HBM bandwidth.  The fine-level
    iterate is 139 MB (above L2).  Returns (result dict, final iterate on the host);
    profile_only prints each launch's grid and V-cycles (to pair with ncu's
    per-launch DRAM counters) and returns (None, None)."""
    import numpy as np
    import torch
    from paper_2107_05337_gb300 import binding as B
    from paper_2107_05337_gb300 import inputs
    w = inputs.WORKLOADS["annulus_c3"]
    p, nel, T, Nt, m = w["p"][0], w["nel"], w["T"], w["Nt"], w["m"]
    k, l, a = inputs.fourier_modes()
    u0fn = lambda xi, eta, x, y: sum(a[s] * np.sin(k[s] * np.pi * xi) * np.sin(l[s] * np.pi * eta)
                                     for s in range(len(a)))
    prob = B.Problem(p, nel, w["geom"])
    u0 = prob.project(u0fn)
    U = torch.empty((Nt + 1, prob.N), dtype=torch.float64, device="cuda")
    opts = dict(T=T, Nt=Nt, m=m, max_levels=w["max_levels"], min_coarse=w["min_coarse"], relax=1,
                tol=1e-10, max_iter=100, coarse_cycles=1)
    pmg = dict(precision=1, tol=1e-10, autotune=1)
    h = B.MGRIT(prob, **opts, pmg=pmg)
    if profile_only:
        h.run(u0, None, None, U)
        torch.cuda.synchronize()
        hp = B.MGRIT(prob, **opts, pmg=pmg, profile=1, graphs=0)
        hp.run(u0, None, None, U)
        pr = hp.profile()
        print(json.dumps({"order": p, "N": int(prob.N), "grid": [int(g) for g in pr["grid"]],
                          "cycles": [int(c) for c in pr["cycles"]]}))
        return None, None
    stream = torch.cuda.current_stream()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")  # 256 MiB > L2
    for _ in range(warmup):
        h.run(u0, None, None, U)
    torch.cuda.synchronize()
    ms, st = [], None
    with Clocks(0) as ck:
        for _ in range(steps):
            flush.fill_(1.0)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            _, st, _ = h.run(u0, None, None, U)
            e1.record(stream)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
    Uh = U.cpu().numpy()
    hp = B.MGRIT(prob, **opts, pmg=pmg, profile=1, graphs=0)
    hp.run(u0, None, None, U)
    pr = hp.profile()
    tot_ms = sum(pr["ms"])
    byts = sum(c * prob.N * bytes_per_vcycle_dof(p, g) for g, c in zip(pr["grid"], pr["cycles"]))
    peaks = measured_peaks()
    peak = peaks["hbm_gbs"] if peaks else 6800.0
    achieved = byts / (tot_ms * 1e-3) / 1e9
    dram = NCU_DRAM_BYTES_PER_LAUNCH["annulus_c3"]
    return ({"workload": "annulus_c3: quarter annulus, p=4, nel=128 (N=16900), N_t=1024, T=1, "
                         "m=8 multilevel FCF MGRIT, f=0, 8-mode initial condition",
             "form": "chosen (FP32 p-MG cycles with FP64 refinement, one cycle per coarse-level "
                     "solve, autotuned sweep layouts)",
             "metric": "DOF*timesteps/s to MGRIT rel. residual 1e-10",
             "value": prob.N * Nt * len(ms) / (sum(ms) * 1e-3), "unit": UNIT,
             "ms_per_solve": round(sum(ms) / len(ms), 2), "steps": len(ms),
             "warmup": warmup, "iters": st["iters"], "levels": st["levels"],
             "vcyc_mean": round(st["vcyc_mean"], 3),
             "l2": "flushed (256 MiB write) before every timed solve",
             "roofline": {"kernel": "k_mgrit_sweep", "bound": "hbm", "achieved": round(achieved, 2),
                          "peak": peak, "unit": "GB/s", "frac": round(achieved / peak, 5),
                          "traffic": dram,
                          "launches_profiled": len(pr["ms"]),
                          "mean_launch_ms": round(tot_ms / len(pr["ms"]), 3),
                          "peak_source": "measured" if peaks else "fallback"},
             "clocks": ck.summary()}, Uh)


def run_annulus(args):
    import torch
    torch.cuda.set_device(0)
    res, _ = annulus_measure(args.steps, args.warmup, args.profile_only)
    if res is not None:
        print(json.dumps(res))


def run_trace(args):
    """One right-hand side on 64 x 64 elements, c = 1/256 (a heat_c2 fine-level step), p = 2..5,
    mixed and FP64 forms: the microseconds per cycle of every solver phase from pmg_trace
    (SM clocks of thread 0 at the maximum SM clock, 10 fixed cycles after 2 untimed), and the
    cycle time without tracing (CUDA events).  One JSON line per order and form."""
    import torch
    from paper_2107_05337_gb300 import binding as B
    from paper_2107_05337_gb300 import inputs
    torch.cuda.set_device(0)
    peaks = measured_peaks()
    mhz = peaks["sm_max_mhz"] if peaks else 2070.0
    for p in (2, 3, 4, 5):
        prob = B.Problem(p, 64)
        for prec in (1, 0):
            g = B.PMG(prob, 1.0 / 256, precision=prec, trace=1, autotune=1)
            g2 = B.PMG(prob, 1.0 / 256, precision=prec, autotune=1)
            Bm = torch.as_tensor(inputs.random_block(1, prob.N, 1), dtype=torch.float64,
                                 device="cuda")
            X = torch.zeros_like(Bm)
            g.solve(Bm, X, ncycles=2)
            g.trace(reset=True)
            X.zero_()
            g.solve(Bm, X, ncycles=10)
            tr = g.trace(reset=True)
            X.zero_()
            g2.solve(Bm, X, ncycles=10)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            X.zero_()
            e0.record()
            g2.solve(Bm, X, ncycles=10)
            e1.record()
            torch.cuda.synchronize()
            print(json.dumps({"p": p, "form": "mixed" if prec else "fp64", "layout": g2.layout(),
                              "us_per_cycle": round(e0.elapsed_time(e1) * 1e3 / 10, 1),
                              "trace_us_per_cycle": {k: round(v / mhz / 10, 1)
                                                     for k, v in tr.items() if v}}))


def run_spmm(args):
    """(M + c K) applied to a block of FP32 columns (one column per time point of a
    long interval), p = 2..5, on the unit square and on the quarter annulus with
    64 x 64 elements (8192 columns) and 128 x 128 elements (2048 columns): bytes
    moved (one read of x, one write of y; on the annulus also the FP32 stencils)
    over the CUDA-event time, against the measured HBM copy bandwidth.  286 MB in
    and out per call at p = 4, h = 1/64, far above L2; the timed calls alternate
    between two input blocks.  Columns are padded to a multiple of four floats."""
    import torch
    from paper_2107_05337_gb300 import binding as B
    torch.cuda.set_device(0)
    peaks = measured_peaks()
    peak = peaks["hbm_gbs"] if peaks else 6800.0
    cases = [("unit_square", nel, q) for nel in (64, 128) for q in (2, 3, 4, 5)]
    cases += [("quarter_annulus", nel, q) for nel in (64, 128) for q in (2, 3, 4, 5)]
    for geom, nel, p in cases:
        # h = 1/128: fewer columns (same order of bytes per call); on the unit square
        # n > 84 grid lines take the row-strip form
        ncol = 8192 if nel == 64 else 2048
        prob = B.Problem(p, nel, geom)
        ld = (prob.N + 3) // 4 * 4   # 16-byte aligned columns: the streamed path
        X = [torch.randn((ncol, ld), dtype=torch.float32, device="cuda") for _ in range(2)]
        for _ in range(3):
            prob.apply_f32("A", X[0], c=1.0 / 256)
        torch.cuda.synchronize()
        reps = 10
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for r in range(reps):
            prob.apply_f32("A", X[r % 2], c=1.0 / 256)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        Q = (2 * p + 1) ** 2
        curved = geom != "unit_square"
        # x read and y written per column; on the curved map also the FP32 M and K
        # stencils (read once per call)
        nbytes = 2 * 4 * prob.N * ncol + (2 * 4 * Q * prob.N if curved else 0)
        gbs = nbytes / (ms * 1e-3) / 1e9
        kern = ("k_spmm32_curved (iga_apply_f32, assembled stencils)" if curved else
                "k_spmm32 (iga_apply_f32)" if prob.n <= 84 else
                "k_spmm32_strip (iga_apply_f32, row strips)")
        print(json.dumps({"kernel": kern, "geometry": geom, "p": p, "nel": nel,
                          "N": prob.N, "columns": ncol,
                          "ms_per_call": round(ms, 4), "achieved_gbs": round(gbs, 1),
                          "peak_gbs": peak, "frac": round(gbs / peak, 3),
                          "peak_source": "measured" if peaks else "fallback",
                          "flops_per_unknown": 2 * Q if curved else 4 * (2 * p + 1) * 2}))


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.spmm:
        return run_spmm(args)
    if args.trace:
        return run_trace(args)
    if args.annulus:
        return run_annulus(args)
    if args.learned:
        return run_learned(args)
    if args.batch:
        return run_batch(args)
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    orders = [int(x) for x in args.orders.split(",")]
    T, Nt, nel = 1.0, args.Nt, args.nel
    # the oracle's sequential solutions of every benchmarked problem, for the
    # errors of the GPU results (CPU baseline leg; spawned before any GPU use,
    # collected after the timed regions)
    refs_ex, refs = None, {}
    if not args.skip_cpu and rank == 0 and not args.profile_only:
        jobs = [("heat_c2", p, nel, Nt) for p in orders]
        if not args.skip_annulus:
            jobs.append(("annulus_c3",))
        refs_ex, refs = oracle_references(jobs)
    import numpy as np
    import torch
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2107_05337_gb300 import binding as B
    S, C = manufactured()
    fcoef = np.array([C(n * T / Nt) for n in range(Nt + 1)])
    probs, u0s, fhats, Us = {}, {}, {}, {}
    for p in orders:
        probs[p] = B.Problem(p, nel)
        u0s[p] = probs[p].project(S)
        fhats[p] = probs[p].load_vector(S)
        Us[p] = torch.empty((Nt + 1, probs[p].N), dtype=torch.float64, device="cuda")
    opts = dict(T=T, Nt=Nt, m=4, max_levels=30, min_coarse=4, relax=1, tol=1e-10, max_iter=100)
    CHOSEN = dict(coarse_cycles=1, pmg=dict(precision=1, tol=1e-10, autotune=1))
    t_setup = time.perf_counter()
    # chosen form: FP32 p-multigrid cycles with FP64 refinement, and one cycle per
    # spatial solve on the coarse time levels (inexact coarse propagator)
    chosen = {p: B.MGRIT(probs[p], **opts, **CHOSEN) for p in orders}
    setup_s = time.perf_counter() - t_setup
    units = sum(probs[p].N * Nt for p in orders)
    stream = torch.cuda.current_stream()

    def step(handles, stats=None, concurrent=True):
        """One MGRIT solve per order.  The orders are independent problems: each
        runs from its own host thread on its own stream, so their (latency-bound)
        sweeps overlap on the GPU."""
        out = {}

        def one(p):
            _, st, _ = handles[p].run(u0s[p], fhats[p], fcoef, Us[p])
            out[p] = st

        if concurrent and len(orders) > 1:
            th = [threading.Thread(target=one, args=(p,)) for p in orders]
            for t in th:
                t.start()
            for t in th:
                t.join()
        else:
            for p in orders:
                one(p)
        if stats is not None:
            stats.update(out)

    if args.profile_only:
        step(chosen, concurrent=False)
        torch.cuda.synchronize()
        # per-launch V-cycle counts of the same solves (same order of launches),
        # to relate a captured launch's DRAM counters to its units of work
        for p in orders:
            hp = B.MGRIT(probs[p], **opts, **CHOSEN, profile=1, graphs=0)
            hp.run(u0s[p], fhats[p], fcoef, Us[p])
            pr = hp.profile()
            print(json.dumps({"order": p, "N": int(probs[p].N), "grid": [int(g) for g in pr["grid"]],
                              "cycles": [int(c) for c in pr["cycles"]]}))
        return

    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")  # 256 MiB > L2

    def timed(handles, K, W):
        for _ in range(W):
            step(handles)
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        ms = []
        stats = {}
        l0 = B.kernel_launches()
        with Clocks(local) as ck:
            for _ in range(K):
                flush.fill_(1.0)
                torch.cuda.synchronize()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                step(handles, stats)
                e1.record(stream)
                torch.cuda.synchronize()
                ms.append(e0.elapsed_time(e1))
        launches = B.kernel_launches() - l0
        total = job_time_ms(sum(ms), world, "cuda")
        host = {p: Us[p].cpu().numpy() for p in orders}   # the last step's iterates
        return total, ms, stats, ck.summary(), launches, host

    log("heat_c2: chosen form")
    total, ms, stats, clocks, launches, U_chosen = timed(chosen, args.steps, args.warmup)
    value = job_throughput(units, world, args.steps, total)

    def side_form(handles, name):
        k = max(1, min(args.steps, 2))
        tot, _, st, _, _, host = timed(handles, k, 1)
        return ({"value": world * units * k / (tot * 1e-3), "ms_per_step": tot / k,
                 "iters": {p: st[p]["iters"] for p in orders},
                 "vcyc_mean": {p: round(st[p]["vcyc_mean"], 3) for p in orders}}, host)

    # the mixed-precision form alone (every level solved to 1e-10): splits the
    # chosen form's speed-up over the plain form into its two parts
    mixed, U_mixed = None, None
    plain, U_plain = None, None
    if not args.skip_plain:
        h = {p: B.MGRIT(probs[p], **opts, pmg=dict(precision=1, tol=1e-10, autotune=1))
             for p in orders}
        log("heat_c2: mixed-only and plain FP64 forms")
        mixed, U_mixed = side_form(h, "mixed")
        del h
        h = {p: B.MGRIT(probs[p], **opts, pmg=dict(precision=0, tol=1e-10)) for p in orders}
        plain, U_plain = side_form(h, "plain")
        del h
    # the chosen form with the p = 1 W-cycle in FP64 instead of FP32 (the
    # alternative reading of which part of the cycle stays FP64)
    w64, U_w64 = None, None
    if not args.skip_plain:
        h = {p: B.MGRIT(probs[p], **opts, coarse_cycles=1,
                        pmg=dict(precision=1, tol=1e-10, autotune=1, hmg_fp64=1)) for p in orders}
        w64, U_w64 = side_form(h, "w64")
        del h

    # end to end through the C ABI with host buffers: H2D of u0, fhat (pinned),
    # solve, D2H of the final time level, every step
    log("heat_c2: end to end")
    hu0 = {p: u0s[p].cpu().pin_memory() for p in orders}
    hfh = {p: fhats[p].cpu().pin_memory() for p in orders}
    hout = {p: torch.empty(probs[p].N, dtype=torch.float64).pin_memory() for p in orders}
    du0 = {p: torch.empty_like(u0s[p]) for p in orders}
    dfh = {p: torch.empty_like(fhats[p]) for p in orders}
    e2e_ms = []

    def e2e_one(p):
        s = torch.cuda.Stream()
        with torch.cuda.stream(s):
            du0[p].copy_(hu0[p], non_blocking=True)
            dfh[p].copy_(hfh[p], non_blocking=True)
            chosen[p].run(du0[p], dfh[p], fcoef, Us[p])
            hout[p].copy_(Us[p][Nt], non_blocking=True)
        s.synchronize()

    for k in range(args.warmup + args.steps):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        th = [threading.Thread(target=e2e_one, args=(p,)) for p in orders]
        for t in th:
            t.start()
        for t in th:
            t.join()
        torch.cuda.synchronize()
        if k >= args.warmup:
            e2e_ms.append(1e3 * (time.perf_counter() - t0))
    h2d = sum(2 * probs[p].N * 8 + (Nt + 1) * 8 for p in orders)
    d2h = sum(probs[p].N * 8 for p in orders)
    e2e = {"value": job_throughput(units, world, len(e2e_ms), job_time_ms(sum(e2e_ms), world, "cuda")),
           "unit": UNIT,
           "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}

    # roofline of the dominant kernel (k_mgrit_sweep), one profiled solve per order
    log("heat_c2: profiled solves for the roofline")
    roof = None
    prof_tot_ms, prof_bytes, prof_launches = 0.0, 0.0, 0
    for p in orders:
        hp = B.MGRIT(probs[p], **opts, **CHOSEN, profile=1, graphs=0)
        hp.run(u0s[p], fhats[p], fcoef, Us[p])
        pr = hp.profile()
        for g, c, t in zip(pr["grid"], pr["cycles"], pr["ms"]):
            prof_bytes += c * probs[p].N * bytes_per_vcycle_dof(p, g)
            prof_tot_ms += t
            prof_launches += 1
        del hp
    peaks = measured_peaks()
    if prof_launches:
        achieved = prof_bytes / (prof_tot_ms * 1e-3) / 1e9
        peak = peaks["hbm_gbs"] if peaks else 6800.0
        roof = {"bound": "hbm", "achieved": round(achieved, 2), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 5),
                "traffic": NCU_DRAM_BYTES_PER_LAUNCH["heat_c2"],
                "kernel": "k_mgrit_sweep", "launches_profiled": prof_launches,
                "mean_launch_ms": round(prof_tot_ms / prof_launches, 4),
                "peak_source": "measured" if peaks else "fallback"}

    # the orders one after another (no overlap), for reference
    serial_ms = None
    if not args.skip_check and rank == 0:
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step(chosen, None, concurrent=False)
        e1.record(stream)
        torch.cuda.synchronize()
        serial_ms = e0.elapsed_time(e1)

    # the curved-map workload, where the iterate exceeds L2
    annulus, U_annulus = None, None
    if not args.skip_annulus and rank == 0:
        log("annulus_c3")
        annulus, U_annulus = annulus_measure(2, 1)


    cpu, errors = None, None
    if refs:
        # errors against the oracle's sequential backward Euler (Sec. 3: the
        # fixed point of MGRIT), every timed form and order
        log("oracle references and CPU baseline")
        seq = {job: f.result() for job, f in refs.items()}
        refs_ex.shutdown()
        errors = {}
        for name, Uf in (("chosen", U_chosen), ("mixed", U_mixed), ("plain_fp64", U_plain),
                         ("chosen_fp64_w_cycle", U_w64)):
            if Uf is not None:
                errors[name] = {p: rel_err(Uf[p], seq[("heat_c2", p, nel, Nt)]) for p in orders}
        if annulus is not None:
            annulus["error_vs_oracle"] = rel_err(U_annulus, seq[("annulus_c3",)])
        cpu = cpu_baseline_leg()

    # the uneven batch in one persistent launch (batch_c5, device scheduling only),
    # one timed run, as a child process with a time limit (single-GPU runs only)
    batch_c5 = None
    if not args.skip_extra and rank == 0 and world == 1:
        log("batch_c5 (child process)")
        batch_c5 = extra_child(["--batch", "--steps", "1", "--warmup", "1", "--skip-plain"], 360)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": total / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
                "data": "synthetic",
                "config": {"workload": f"heat_c2: unit square, nel={nel}, p={orders}, N_t={Nt}, T=1, "
                                       "m=4 multilevel FCF MGRIT, p-MG V(1,1) to 1e-10",
                           "chosen_form": "FP32 p-MG cycles with FP64 refinement; one p-MG cycle "
                                          "per coarse-time-level solve (fine level to 1e-10); "
                                          "sweep layouts autotuned at setup",
                           "mixed_form": "FP32 p-MG cycles with FP64 refinement, every level to 1e-10",
                           "chosen_fp64_w_cycle_form": "the chosen form with the p=1 W-cycle in FP64",
                           "plain_form": "FP64 p-MG on every level to 1e-10",
                           "orders": "solved concurrently, one stream each",
                           "parallelism": f"replicas{world}" if world > 1 else "single GPU",
                           "l2": "flushed (256 MiB write) before every timed step"},
                "mixed_only": mixed,
                "plain_fp64": plain,
                "chosen_fp64_w_cycle": w64,
                "speedup_vs_plain": (value / plain["value"]) if plain else None,
                "speedup_parts": ({"mixed_precision": mixed["value"] / plain["value"],
                                   "one_cycle_coarse_levels": value / mixed["value"]}
                                  if plain and mixed else None),
                "iters": {p: stats[p]["iters"] for p in orders},
                "vcyc_mean": {p: round(stats[p]["vcyc_mean"], 3) for p in orders},
                "error_vs_oracle": errors,
                "setup_s": round(setup_s, 3),
                "orders_one_after_another_ms": serial_ms,
                "e2e": e2e, "gpu_launches": launches, "roofline": roof, "cpu_baseline": cpu,
                "annulus_c3": annulus,
                "batch_c5": batch_c5,
                "clocks": clocks}
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
