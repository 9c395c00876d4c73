#!/usr/bin/env python
"""Benchmark of the LB IMEX-TR hot path on GB300 (one JSON line on stdout).

Workload: 3D LB at scale, 128^3 grid, cubic box side 4*pi*sqrt(2), tau = -0.05,
gamma = 0.3, phi0 ~ N(0, 0.05^2) mean-removed (seeded), mixed precision (float FFTs,
diagonals and pointwise updates; double reductions).

A step is a batch of `--batch` Hessian-vector products H v = P[F^{-1} Lambda F v +
F''(phi) v] over a rotating pool of distinct (phi, v, Hv) triples whose total size is
three times the 129 MB L2, so every product reads its inputs from HBM.  `value` is
products per second over the timed steps with inputs resident in HBM; `e2e` is the same
metric through the C ABI with the inputs copied from pinned host memory and the results
copied back inside the timed region.  The FP64 path and 256^3 are reported beside it.

--impl reference times the FP64 CPU oracle (the reference arm of this build) on a
bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Hessian-vector products/s & TR iters/s at 128³, mixed vs FP64 GPU; HBM GB/s"
UNIT = "HVP/s"
L2_BYTES = 129 * 1024 * 1024

# ncu DRAM traffic per launch of a kernel class, with the hash of the kernel sources it
# was captured from (a traffic figure is reported only while those sources match).
TRAFFIC = {
    # k_hvp_fused<float> (the whole 128^3 product, one launch): ncu dram__bytes_read.sum +
    # dram__bytes_write.sum of one cold launch (profiles/hvp_fused_128cubed_mixed_ncu_full.md)
    "xfwd": (16845312 + 0, "be4b96ca632d7443"),
}


# the sources that define the HVP kernels (their DRAM traffic is keyed to these)
HVP_KERNEL_SOURCES = ("common.cuh", "fft_core.cuh", "reduce.cuh", "passes.cuh", "hvp3d.cuh")


def csrc_hash() -> str:
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2603_03933_gb300", "csrc")
    for name in HVP_KERNEL_SOURCES:
        with open(os.path.join(d, name), "rb") as f:
            h.update(name.encode())
            h.update(f.read())
    return h.hexdigest()[:16]


def measured_peaks() -> dict:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return {"hbm_gbs": float(d["hbm_gbs"]), "source": "measured"}
    return {"hbm_gbs": 6800.0, "source": "fallback"}


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.proc = None
        self.idx = gpu_index
        # the raw samples go to LB_CLOCKS_DIR (default: the system temporary directory)
        self.path = os.path.join(os.environ.get("LB_CLOCKS_DIR", tempfile.gettempdir()),
                                 f"clocks_bench_{gpu_index}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self) -> dict | None:
        if self.proc is None:
            return None
        time.sleep(0.2)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    mx = max(mx, float(parts[2]))
                except ValueError:
                    continue
                for n, v in zip(names, parts[5:9]):
                    if v.lower() == "active":
                        reasons.add(n)
        if not sm:
            return None
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup(n_gpus: int):
    import torch
    rank, world = int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, world: int, device: str = "cuda") -> float:
    """The largest of the ranks' values (the job's time is its slowest rank's)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, seconds_max: float, world: int) -> float:
    """Units processed by all ranks per second of the slowest rank (weak scaling: every
    replica processes the same number of units)."""
    return units_per_rank * world / seconds_max


def shard(n_items: int, rank: int, world: int) -> list:
    """Items of an independent batch (e.g. sweep instances) owned by `rank`: round-robin,
    disjoint across ranks and covering all items."""
    return list(range(rank, n_items, world))


def _oracle_worker(M: int, seconds: float, seed: int, barrier, queue):
    """One host core: FP64 oracle Hessian-vector products for `seconds` after all workers
    are ready; puts (products, elapsed seconds), or an error text, on the queue."""
    try:
        import numpy as np
        from oracle import lb as olb
        from paper_2603_03933_gb300 import inputs
        w = inputs.config_3d_scale(M)
        p = olb.Problem.from_workload(w)
        v = inputs.remove_mean(np.random.default_rng(seed).standard_normal(w.shape))
        barrier.wait(timeout=300)
        done, t0 = 0, time.perf_counter()
        while True:
            olb.hessvec(p, w.phi0, v)
            done += 1
            el = time.perf_counter() - t0
            if el >= seconds or done >= 50:
                break
        queue.put((done, el))
    except Exception as ex:  # reported by the parent
        queue.put(f"{type(ex).__name__}: {ex}")


def oracle_hvp_rate(M: int, seconds: float = 12.0, workers: int = 0) -> dict:
    """The FP64 CPU oracle's Hessian-vector products on the same workload, one process per
    host core (spawned, so safe after CUDA has started), all timed together over a bounded
    sample; the rate is the sum of the processes' rates."""
    import multiprocessing as mp
    if workers <= 0:
        try:
            workers = len(os.sched_getaffinity(0))      # the cores this process may run on
        except (AttributeError, OSError):
            workers = os.cpu_count() or 1
    n = max(1, min(workers, 32))
    ctx = mp.get_context("spawn")
    barrier, queue = ctx.Barrier(n), ctx.Queue()
    procs = [ctx.Process(target=_oracle_worker, args=(M, seconds, 77 + i, barrier, queue)) for i in range(n)]
    for pr in procs:
        pr.start()
    res = []
    try:
        for _ in procs:
            res.append(queue.get(timeout=seconds + 400))
    except Exception as ex:  # a worker died without reporting
        res.append(f"no result: {type(ex).__name__}")
    bad = [r for r in res if isinstance(r, str)]
    if bad:
        barrier.abort()
    for pr in procs:
        pr.join(timeout=30)
        if pr.is_alive():
            pr.terminate()
            pr.join()
    if bad:
        return {"error": bad[0], "kind": "oracle", "cores": n}
    done = sum(d for d, _ in res)
    el = max(e for _, e in res)
    return {"value": sum(d / e for d, e in res), "unit": UNIT, "cores": n, "kind": "oracle",
            "sample": f"{done} FP64 oracle Hessian-vector products at {M}^3 on {n} processes "
                      f"(~{el:.1f} s each, numpy, 1 thread per process)"}


def run_reference(args, rank: int):
    """The oracle as it stands: each step is one FP64 Hessian-vector product at --size."""
    if rank != 0:
        return
    import numpy as np
    from oracle import lb as olb
    from paper_2603_03933_gb300 import inputs
    w = inputs.config_3d_scale(args.size)
    p = olb.Problem.from_workload(w)
    vs = [inputs.gaussian_field(w.shape, 1.0, 2000 + i) for i in range(2)]
    for i in range(args.warmup):
        olb.hessvec(p, w.phi0, vs[i % 2])
    t0 = time.perf_counter()
    for i in range(args.steps):
        olb.hessvec(p, w.phi0, vs[i % 2])
    total = time.perf_counter() - t0
    value = args.steps / total
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": f"3D LB at scale {args.size}^3 (tau -0.05, gamma 0.3, box 4*pi*sqrt(2))",
                       "step": "1 Hessian-vector product of the FP64 CPU oracle", "l2": "n/a (CPU)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"{args.steps} oracle Hessian-vector products at {args.size}^3 "
                                       "(numpy, 1 thread)"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def hvp_pool(lbtr, ctx, w, M, dtype, count, device):
    import torch
    from paper_2603_03933_gb300 import inputs
    pool = []
    for i in range(count):
        phi = torch.tensor(w.phi0 if i == 0 else inputs.gaussian_field(w.shape, 0.05, 1000 + i),
                           dtype=dtype, device=device)
        v = torch.tensor(inputs.gaussian_field(w.shape, 1.0, 2000 + i), dtype=dtype, device=device)
        pool.append((phi, v, torch.empty_like(v)))
    return pool


def time_hvp(lbtr, ctx, pool, batch, steps, warmup, world):
    """Per-step device time (s) of `batch` products cycling through the pool."""
    import torch
    s = torch.cuda.current_stream()
    k = 0

    def step():
        nonlocal k
        for _ in range(batch):
            phi, v, hv = pool[k % len(pool)]
            lbtr.lb_hessvec(ctx, phi, v, hv, stream=s)
            k += 1

    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    barrier(world)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s)
    for _ in range(steps):
        step()
    e1.record(s)
    torch.cuda.synchronize()
    barrier(world)
    return e0.elapsed_time(e1) / 1000.0


def time_tr(lbtr, w, prec: str, outer: int, persistent: bool = True) -> dict:
    """Outer IMEX-TR iterations per second on the workload from its initial field.

    Both precisions solve every subproblem to the same relative residual (1e-6 of
    ||g||) so the comparison is at equal inner accuracy.  `persistent`: the one-launch
    inner loop where the library has it (128^3 mixed), else per-iteration launches."""
    import torch
    ctx = lbtr.lb_create_from_array_box(w.shape, w.box, w.xi, w.tau, w.gamma,
                                        lbtr.LB_MIXED if prec == "mixed" else lbtr.LB_FP64)
    lbtr.lb_set_persistent_subproblem(ctx, persistent)
    o = lbtr.default_tr_opts()
    o.eps = 1e-8
    o.sub.eps_sub = 0.0
    o.sub.rel_tol = 1e-6
    o.sub.max_iter = 20000
    o.sub.check_every = 256
    # warm-up: one short outer iteration
    phi = torch.tensor(w.phi0, dtype=torch.float64, device="cuda")
    o.max_outer = 1
    lbtr.lb_imex_tr_solve(ctx, phi, opts=o, raise_on_noconv=False)
    phi = torch.tensor(w.phi0, dtype=torch.float64, device="cuda")
    o.max_outer = outer
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    info = lbtr.lb_imex_tr_solve(ctx, phi, opts=o, raise_on_noconv=False)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    n_out = max(1, info["outer"])
    out = {"outer_iters": n_out, "seconds": dt, "tr_iters_per_s": n_out / dt,
           "inner_iters": info["inner"], "inner_iters_per_s": info["inner"] / dt,
           "energy": info["energy"], "gmax": info["gmax"], "sub_rel_tol": 1e-6,
           "sub_stalled": info["sub_stalled"], "sub_capped": info["sub_capped"],
           "sub_worst_rel_res": info["sub_worst_rel_res"],
           "inner_loop": ("one launch per subproblem" if lbtr.lb_persistent_subproblem_available(ctx)
                          else "launches per inner iteration"),
           # an inner iteration must at least read phi and g and read and write the iterate:
           # 16 N bytes in float, 32 N in double (the one-launch form keeps them in L2)
           "inner_alg_bytes": (16 if prec == "mixed" else 32) * w.n_points,
           "inner_alg_gbs": (16 if prec == "mixed" else 32) * w.n_points * info["inner"] / dt / 1e9,
           "note": "outer iterations from the initial field, not a solve"}
    # per-kernel-class breakdown of one more outer iteration (CUDA events per launch)
    phi = torch.tensor(w.phi0, dtype=torch.float64, device="cuda")
    o.max_outer = 1
    lbtr.lb_profile_enable(ctx, True)
    info1 = lbtr.lb_imex_tr_solve(ctx, phi, opts=o, raise_on_noconv=False)
    prof = lbtr.lb_profile_read(ctx)
    lbtr.lb_profile_enable(ctx, False)
    n1 = max(1, info1["inner"])
    out["profiled_outer_iteration"] = {"inner_iters": n1, "classes": {
        k: {"total_ms": v[0], "launches": v[1], "us_per_inner_iter": 1e3 * v[0] / n1} for k, v in prof.items() if v[1] > 0}}
    return out


def time_tr_solve_bcc64(lbtr, prec: str) -> dict:
    """A whole IMEX-TR solve of the 3D BCC workload (64^3, box 4 pi sqrt(2), tau -0.1,
    gamma 0.2) to max|g| < 1e-8 with the second-order test lambda_min >= -1e-8, inner
    iterations to a residual below 1e-4 ||g|| (at most 2000): the same accuracy in both
    precisions.  The oracle's solve with the same settings, when stored, gives the energy
    the result is compared with."""
    import torch
    from paper_2603_03933_gb300 import inputs
    w = inputs.config_3d_bcc(64)
    ctx = lbtr.lb_create_from_array_box(w.shape, w.box, w.xi, w.tau, w.gamma,
                                        lbtr.LB_MIXED if prec == "mixed" else lbtr.LB_FP64)
    o = lbtr.default_tr_opts()
    o.eps, o.tol2, o.second_order = 1e-8, 1e-8, 1
    o.sub.eps_sub, o.sub.rel_tol, o.sub.max_iter, o.sub.check_every = 0.0, 1e-4, 2000, 256
    o.max_outer = 1                                       # warm-up
    phi = torch.tensor(w.phi0, dtype=torch.float64, device="cuda")
    lbtr.lb_imex_tr_solve(ctx, phi, opts=o, raise_on_noconv=False)
    o.max_outer = 200
    phi = torch.tensor(w.phi0, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    info = lbtr.lb_imex_tr_solve(ctx, phi, opts=o, raise_on_noconv=False)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    out = {"status": info["status"], "seconds_to_solution": dt, "outer_iters": info["outer"],
           "tr_iters_per_s": info["outer"] / dt, "inner_iters": info["inner"],
           "inner_per_outer": info["inner"] / max(1, info["outer"]),
           "energy": info["energy"], "gmax": info["gmax"], "lambda_min": info["lambda_min"],
           "sub_stalled": info["sub_stalled"], "sub_capped": info["sub_capped"],
           "sub_worst_rel_res": info["sub_worst_rel_res"]}
    gold = os.path.join(ROOT, "tests", "golden", "oracle_solves.json")
    if os.path.exists(gold):
        with open(gold) as f:
            ref = json.load(f).get("3d_64_bcc_rel")
        if ref:
            out["oracle_energy"] = ref["energy"]
            out["energy_minus_oracle"] = info["energy"] - ref["energy"]
    return out


def time_sweep(lbtr, rank: int, world: int, n_instances: int, replays: int = 20) -> dict:
    """The batched 2D sweep (256 instances, M in {64..512}, mixed): every instance's
    Hessian-vector product in one persistent launch with device-side task queues
    (lb_batch_hessvec, recorded as a CUDA graph), its launch shape chosen by the library's
    tuner (lb_batch_tune, whose table is reported), timed over `replays` replays with CUDA
    events after 3 warm-up replays; instances are sharded across ranks."""
    import torch
    from paper_2603_03933_gb300 import inputs
    ws = [inputs.batched_sweep(n_instances)[i] for i in shard(n_instances, rank, world)]
    probs = [(w.dim, w.shape[0], list(w.box)[::-1], w.xi, w.tau, w.gamma) for w in ws]
    t0 = time.perf_counter()
    batch = lbtr.lb_batch_create(probs, lbtr.LB_MIXED)
    setup_s = time.perf_counter() - t0
    phis = [torch.tensor(w.phi0, dtype=torch.float32, device="cuda") for w in ws]
    vs = [torch.tensor(inputs.gaussian_field(w.shape, 1.0, 5000 + i), dtype=torch.float32, device="cuda")
          for i, w in enumerate(ws)]
    hvs = [torch.empty_like(v) for v in vs]
    s = torch.cuda.current_stream()
    tuning = lbtr.lb_batch_tune(batch, phis, vs, hvs, replays=10, stream=s)
    fields = lbtr.BatchFields(batch, phis, vs, hvs)         # pointers marshalled once
    for _ in range(3):
        lbtr.lb_batch_hessvec(batch, fields, stream=s)
    torch.cuda.synchronize()
    barrier(world)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s)
    for _ in range(replays):
        lbtr.lb_batch_hessvec(batch, fields, stream=s)
    e1.record(s)
    torch.cuda.synchronize()
    barrier(world)
    dt = max_over_ranks(e0.elapsed_time(e1) / 1000.0, world)
    npts = sum(w.n_points for w in ws)
    sizes = {}
    for w in ws:
        sizes[w.shape[0]] = sizes.get(w.shape[0], 0) + 1
    return {"workload": f"{n_instances} 2D instances, M in {{64,128,256,512}} (seed 5), mixed; one CUDA graph "
                        "per replay: grouped launches or one persistent launch with device-side task "
                        "queues, whichever the library's tuner measured faster (table in 'tuning')",
            "tuning": tuning,
            "value": whole_job_rate(len(ws) * replays, dt, world), "unit": "instance-HVP/s",
            "alg_gbs": whole_job_rate(12.0 * npts * replays, dt, world) / 1e9,
            "us_per_replay": 1e6 * dt / replays, "instances_per_rank": len(ws), "sizes": sizes,
            "setup_s": setup_s,
            # the tuned strategy: one persistent kernel per replay (and a memset of its queue
            # heads), or three grouped launches per grid size up to 256^2 and three launches
            # for each 512^2 instance (a graph branch: no batched line kernel at that size)
            "gpu_launches": (replays if tuning["candidates"][tuning["chosen"]]["strategy"] == "persistent"
                             else replays * (3 * sum(1 for m in sizes if int(m) <= 256) +
                                             3 * sum(c for m, c in sizes.items() if int(m) > 256)))}


def time_sweep_solve(lbtr, rank: int, world: int, n_instances: int, threads: int = 16) -> dict:
    """Whole IMEX-TR solves of a sweep (2D instances of the batched sweep's recipe, M in
    {64, 128}, mixed, eps 1e-8) through lb_batch_tr_solve on `threads` host threads; wall
    clock of the one call, instances sharded across ranks, max over ranks."""
    import torch
    from paper_2603_03933_gb300 import inputs
    ws = [inputs.batched_sweep(n_instances, seed=5, sizes=(64, 128))[i] for i in shard(n_instances, rank, world)]
    probs = [(w.dim, w.shape[0], list(w.box)[::-1], w.xi, w.tau, w.gamma) for w in ws]
    batch = lbtr.lb_batch_create(probs, lbtr.LB_MIXED)
    o = lbtr.default_tr_opts()
    o.eps, o.max_outer = 1e-8, 300
    phis = [torch.tensor(w.phi0, dtype=torch.float64, device="cuda") for w in ws]
    torch.cuda.synchronize()
    barrier(world)
    t0 = time.perf_counter()
    infos = lbtr.lb_batch_tr_solve(batch, phis, opts=o, nthreads=threads, raise_on_error=False)
    torch.cuda.synchronize()
    dt = max_over_ranks(time.perf_counter() - t0, world)
    return {"workload": f"{n_instances} 2D instances, M in {{64,128}} (seed 5), mixed, IMEX-TR to "
                        f"max|g| < 1e-8 with the second-order test; {threads} host threads, one call",
            "value": whole_job_rate(len(ws), dt, world), "unit": "instances/s", "seconds": dt,
            "instances_per_rank": len(ws), "converged": sum(1 for i in infos if i["status"] == 0),
            "outer_iters": sum(i["outer"] for i in infos), "inner_iters": sum(i["inner"] for i in infos)}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="lbtr", choices=["lbtr", "reference"])
    ap.add_argument("--size", type=int, default=128)
    ap.add_argument("--batch", type=int, default=32)
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--only-hvp", action="store_true",
                    help="time only the mixed HVP at --size (small runs for profilers)")
    ap.add_argument("--pool", type=int, default=0, help="override the number of (phi, v, Hv) triples")
    ap.add_argument("--tr-outer", type=int, default=4, help="outer IMEX-TR iterations timed per precision")
    ap.add_argument("--sweep-instances", type=int, default=256,
                    help="instances of the batched 2D sweep timed as one CUDA graph (0: skip)")
    ap.add_argument("--sweep-solve-instances", type=int, default=16,
                    help="instances of the sweep solved whole by lb_batch_tr_solve (0: skip)")
    ap.add_argument("--no-solve", action="store_true", help="skip the whole 64^3 BCC solves")
    ap.add_argument("--inner-launches", action="store_true",
                    help="with --profile-sub: run the inner loop as per-iteration launches, not one launch")
    ap.add_argument("--profile-sub", type=int, default=0,
                    help="profile this many IMEX inner iterations per precision and exit")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    if args.impl == "reference":
        rank = int(os.environ.get("RANK", "0"))
        run_reference(args, rank)
        return

    import torch
    from paper_2603_03933_gb300 import inputs, lbtr
    lbtr.load()
    rank, world, local = dist_setup(args.gpus)
    dev = torch.device("cuda", torch.cuda.current_device())
    M = args.size
    w = inputs.config_3d_scale(M)
    field_bytes = 4 * w.n_points
    npool = args.pool if args.pool > 0 else max(4, math.ceil(3 * L2_BYTES / (3 * field_bytes)))

    ctx = lbtr.lb_create_from_array_box(w.shape, w.box, w.xi, w.tau, w.gamma, lbtr.LB_MIXED)
    pool = hvp_pool(lbtr, ctx, w, M, torch.float32, npool, dev)

    # ---- timed region: value --------------------------------------------------
    clocks = ClockSampler(local)
    clocks.start()
    dt = time_hvp(lbtr, ctx, pool, args.batch, args.steps, args.warmup, world)
    clk = clocks.stop()
    dt = max_over_ranks(dt, world)
    hvps = args.batch * args.steps * world
    value = whole_job_rate(args.batch * args.steps, dt, world)

    if args.profile_sub > 0:
        # per-kernel-class times of a fixed number of IMEX inner iterations (Algorithm 3)
        res = {}
        for prec in ("mixed", "fp64"):
            c = ctx if prec == "mixed" else lbtr.lb_create_from_array_box(w.shape, w.box, w.xi, w.tau, w.gamma,
                                                                          lbtr.LB_FP64)
            lbtr.lb_set_persistent_subproblem(c, not args.inner_launches)
            dt_ = torch.float32 if prec == "mixed" else torch.float64
            phi_t = torch.tensor(w.phi0, dtype=dt_, device=dev)
            g_t = torch.empty_like(phi_t)
            lbtr.lb_energy_grad(c, phi_t, g_t)
            d_t = torch.empty_like(phi_t)
            o = lbtr.default_sub_opts()
            o.eps_sub = 0.0
            o.rel_tol = 0.0
            o.max_iter = args.profile_sub
            o.check_every = args.profile_sub
            lbtr.lb_tr_subproblem(c, phi_t, g_t, 1.0, d_t, opts=o, raise_on_noconv=False)
            lbtr.lb_profile_enable(c, True)
            t0 = time.perf_counter()
            info = lbtr.lb_tr_subproblem(c, phi_t, g_t, 1.0, d_t, opts=o, raise_on_noconv=False)
            wall = time.perf_counter() - t0
            prof = lbtr.lb_profile_read(c)
            lbtr.lb_profile_enable(c, False)
            n1 = max(1, info["iterations"])
            res[prec] = {"iterations": n1, "wall_us_per_iter": 1e6 * wall / n1,
                         "classes": {k: {"launches": v[1], "us_per_iter": 1e3 * v[0] / n1}
                                     for k, v in prof.items() if v[1] > 0}}
        print(json.dumps({"mode": "profile-sub", "size": M, **res}), flush=True)
        return

    if args.only_hvp:
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": value, "unit": UNIT, "mode": "only-hvp",
                              "size": M, "pool": npool, "us_per_hvp": dt / (args.batch * args.steps * world) * 1e6}),
                  flush=True)
        return

    # ---- per-kernel live timing (CUDA events on the launching stream) -----------
    lbtr.lb_profile_enable(ctx, True)
    time_hvp(lbtr, ctx, pool, args.batch, max(3, args.steps // 4), 1, 1)
    prof = lbtr.lb_profile_read(ctx)
    lbtr.lb_profile_enable(ctx, False)
    peaks = measured_peaks()
    dom = max(prof, key=lambda k: prof[k][0])
    ms, nl, by = prof[dom]
    achieved = (by / nl) / (ms / nl / 1e3) / 1e9
    tr = TRAFFIC.get(dom)
    traffic = tr[0] if (tr and tr[0] is not None and tr[1] == csrc_hash()) else None
    # headline: the whole Hessian-vector product against its algorithmic bytes (read v and
    # phi, write Hv: 12 N bytes in float), timed over the timed region above
    hvp_time = dt / (args.batch * args.steps)
    hvp_alg = 3 * field_bytes
    hvp_gbs = hvp_alg / hvp_time / 1e9
    traffic_hvp = (sum(TRAFFIC[k][0] for k in TRAFFIC)
                   if all(TRAFFIC[k][0] is not None and TRAFFIC[k][1] == csrc_hash() for k in TRAFFIC) else None)
    roofline = {"bound": "hbm", "kernel": "hvp: " + " + ".join(k for k in prof if prof[k][1] > 0),
                "achieved": hvp_gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": hvp_gbs / peaks["hbm_gbs"], "traffic": traffic_hvp, "peak_source": peaks["source"],
                "alg_bytes_per_hvp": hvp_alg, "us_per_hvp": hvp_time * 1e6,
                "dominant": {"kernel": dom, "achieved": achieved, "frac": achieved / peaks["hbm_gbs"],
                             "traffic": traffic},
                "per_kernel": {k: {"launches": v[1], "avg_us": 1e3 * v[0] / v[1],
                                   "alg_gbs": (v[2] / v[1]) / (v[0] / v[1] / 1e3) / 1e9,
                                   "share": v[0] / sum(x[0] for x in prof.values())}
                               for k, v in prof.items() if v[1] > 0}}

    # ---- FP64 path at the same size -------------------------------------------
    ctx64 = lbtr.lb_create_from_array_box(w.shape, w.box, w.xi, w.tau, w.gamma, lbtr.LB_FP64)
    pool64 = [(a.double(), b.double(), c.double()) for a, b, c in pool[: max(2, npool // 2)]]
    dt64 = time_hvp(lbtr, ctx64, pool64, 4, 3, 1, 1)
    fp64 = {"value": 12 / dt64, "unit": UNIT, "us_per_hvp": dt64 / 12 * 1e6}
    # the FP64 path is bound by FP64 arithmetic: algorithmic flops of one HVP (a real 3D
    # FFT each way, 2.5 N log2 N each, plus ~10 N pointwise) against the FP64 FMA rate
    # measured on this GPU by the library's FMA-loop probe
    try:
        nn = float(w.n_points)
        flops64 = 5.0 * nn * math.log2(nn) + 10.0 * nn
        ach64 = flops64 / (dt64 / 12) / 1e12
        peak64 = lbtr.lb_measure_fp64_rate()
        fp64["roofline"] = {"bound": "alu", "achieved": ach64, "peak": peak64, "unit": "TFLOP/s",
                            "frac": ach64 / peak64, "flops_per_hvp": flops64,
                            "peak_source": "measured: FP64 FMA loop (lb_measure_fp64_rate), this run"}
    except Exception as ex:  # report, do not hide
        fp64["roofline"] = {"error": str(ex)}
    del pool64, ctx64

    # ---- e2e: host buffers, copies inside the timed region ----------------------
    # through the library's host-buffer entry (lb_hessvec_host): phi and the batch's v in
    # page-locked host memory, the products' Hv back to host memory, the copies overlapped
    # with the products inside the library
    s = torch.cuda.current_stream()
    nb = args.batch
    phi_h = pool[0][0].cpu().pin_memory()
    v_h = [pool[i % npool][1].cpu().pin_memory() for i in range(nb)]
    out_h = [torch.empty(w.shape, dtype=torch.float32).pin_memory() for _ in range(nb)]

    def e2e_step():
        lbtr.lb_hessvec_host(ctx, phi_h, v_h, out_h, stream=s)

    e2e_steps = max(3, args.steps // 4)
    for _ in range(args.warmup):
        e2e_step()
    torch.cuda.synchronize()
    barrier(world)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s)
    for _ in range(e2e_steps):
        e2e_step()
    e1.record(s)
    torch.cuda.synchronize()
    barrier(world)
    dte = max_over_ranks(e0.elapsed_time(e1) / 1000.0, world)
    e2e = {"value": nb * e2e_steps * world / dte, "unit": UNIT,
           "h2d_bytes_per_step": (1 + nb) * field_bytes, "d2h_bytes_per_step": nb * field_bytes,
           "api": "lb_hessvec_host (C ABI, page-locked host fields, copies overlapped with the products)"}
    # the copies alone: one field in and one out at once on two streams, repeated (the bound
    # of a product whose input and output cross the host link)
    try:
        sa, sb = torch.cuda.Stream(), torch.cuda.Stream()
        dst_d, src_d = torch.empty_like(pool[0][1]), pool[0][1]

        def copies():
            with torch.cuda.stream(sa):
                dst_d.copy_(v_h[0], non_blocking=True)
            with torch.cuda.stream(sb):
                out_h[0].copy_(src_d, non_blocking=True)

        for _ in range(3):
            copies()
        torch.cuda.synchronize()
        reps = 16
        t0 = time.perf_counter()
        for _ in range(reps):
            copies()
        torch.cuda.synchronize()
        tc = (time.perf_counter() - t0) / reps
        e2e["copy_bound"] = {"gbs_bidirectional": 2 * field_bytes / tc / 1e9, "hvp_per_s": 1.0 / tc,
                             "frac": e2e["value"] / world * tc}
    except Exception as ex:  # report, do not hide
        e2e["copy_bound"] = {"error": str(ex)}

    # ---- 256^3 at the same settings (context, not the headline) ------------------
    big = None
    if M == 128 and world == 1:
        try:
            w2 = inputs.config_3d_scale(256)
            ctx2 = lbtr.lb_create_from_array_box(w2.shape, w2.box, w2.xi, w2.tau, w2.gamma, lbtr.LB_MIXED)
            pool2 = []
            for i in range(4):
                pool2.append((torch.tensor(w2.phi0, dtype=torch.float32, device=dev),
                              torch.tensor(inputs.gaussian_field(w2.shape, 1.0, 3000 + i), dtype=torch.float32,
                                           device=dev),
                              torch.empty(w2.shape, dtype=torch.float32, device=dev)))
            d2 = time_hvp(lbtr, ctx2, pool2, 8, 4, 1, 1)
            big = {"value": 32 / d2, "unit": UNIT, "us_per_hvp": d2 / 32 * 1e6,
                   "alg_gbs": 3 * 4 * w2.n_points / (d2 / 32) / 1e9}
            del pool2, ctx2
        except Exception as ex:  # report, do not hide
            big = {"error": str(ex)}

    # ---- TR iterations (Algorithm 1 outer steps, whole path a1-a9) -------------
    tr = {}
    if args.tr_outer > 0:
        for prec in ("mixed", "fp64"):
            tr[prec] = time_tr(lbtr, w, prec, args.tr_outer if prec == "mixed" else max(1, args.tr_outer // 2))
        # the same mixed outer iterations with the inner loop as per-iteration launches
        tr["mixed_per_iteration_launches"] = time_tr(lbtr, w, "mixed", args.tr_outer, persistent=False)
        tr["mixed_per_iteration_launches"].pop("profiled_outer_iteration", None)
        tr["inner_speedup_one_launch"] = (tr["mixed"]["inner_iters_per_s"] /
                                          tr["mixed_per_iteration_launches"]["inner_iters_per_s"])
        for k in ("mixed", "fp64", "mixed_per_iteration_launches"):
            tr[k]["inner_frac_of_hbm"] = tr[k]["inner_alg_gbs"] / peaks["hbm_gbs"]
    # ---- lambda_min at 128^3 (the second-order test of an SP-II, §1) ------------
    lam128 = None
    if args.tr_outer > 0:
        lam128 = {"workload": "the 128^3 scale field (initial phi), Lanczos to a Ritz residual below 1e-8 "
                              "(at most 300 steps), default options"}
        for prec in ("mixed", "fp64"):
            try:
                c = lbtr.lb_create_from_array_box(w.shape, w.box, w.xi, w.tau, w.gamma,
                                                  lbtr.LB_MIXED if prec == "mixed" else lbtr.LB_FP64)
                ph = torch.tensor(w.phi0, dtype=torch.float32 if prec == "mixed" else torch.float64, device=dev)
                lbtr.lb_lambda_min(c, ph, raise_on_noconv=False)          # warm-up
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                r = lbtr.lb_lambda_min(c, ph, raise_on_noconv=False)
                torch.cuda.synchronize()
                el = time.perf_counter() - t0
                lam128[prec] = {"lambda_min": r["lambda_min"], "steps": r["steps"], "converged": r["converged"],
                                "ritz_residual": r["residual"], "seconds": el,
                                "ms_per_step": 1e3 * el / max(1, r["steps"])}
                del c, ph
            except Exception as ex:  # report, do not hide
                lam128[prec] = {"error": str(ex)}
    tr_solve = None
    if not args.no_solve:
        try:
            tr_solve = {"workload": "3D BCC 64^3 (tau -0.1, gamma 0.2), to max|g| < 1e-8 and lambda_min >= -1e-8, "
                                    "inner residual < 1e-4 ||g|| (<= 2000 iterations), both precisions"}
            for prec in ("mixed", "fp64"):
                tr_solve[prec] = time_tr_solve_bcc64(lbtr, prec)
            tr_solve["time_ratio_fp64_over_mixed"] = (tr_solve["fp64"]["seconds_to_solution"] /
                                                      tr_solve["mixed"]["seconds_to_solution"])
        except Exception as ex:  # report, do not hide
            tr_solve = {"error": str(ex)}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = oracle_hvp_rate(M)
        # the other grid sizes of the scale workload, shorter samples (context)
        if M == 128 and "value" in cpu:
            cpu["other_sizes"] = {}
            for m2, secs in ((64, 4.0), (256, 6.0)):
                try:
                    r2 = oracle_hvp_rate(m2, seconds=secs)
                except Exception as ex:  # report, do not hide
                    r2 = {"error": str(ex)}
                cpu["other_sizes"][f"{m2}^3"] = ({"value": r2["value"], "unit": UNIT, "cores": r2["cores"],
                                                  "sample": r2["sample"]} if "value" in r2 else r2)

    # kernels per HVP: one cooperative launch at 128^3 (float); x/y plane pass, z line pass,
    # inverse plane pass at 32^3-64^3; else x rows, the three line passes in one cooperative
    # launch, inverse x rows
    launches_per_hvp = 1 if M == 128 else 3
    sweep = time_sweep(lbtr, rank, world, args.sweep_instances) if args.sweep_instances > 0 else None
    sweep_solve = None
    if args.sweep_solve_instances > 0:
        try:
            sweep_solve = time_sweep_solve(lbtr, rank, world, args.sweep_solve_instances)
        except Exception as ex:  # report, do not hide
            sweep_solve = {"error": str(ex)}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1000.0 * dt / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64 (mixed)", "data": "synthetic",
        "config": {"workload": f"3D LB at scale {M}^3, mixed precision (tau -0.05, gamma 0.3, "
                               f"box 4*pi*sqrt(2), phi0 ~ N(0, 0.05^2))",
                   "step": f"{args.batch} Hessian-vector products", "pool_triples": npool,
                   "l2": "inputs larger than L2 (rotating pool of 3x L2)", "parallelism": f"replicas x{world}"},
        "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": clk,
        "gpu_launches": launches_per_hvp * args.batch * args.steps,
        "fp64": fp64, "size_256": big, "tr": tr, "lambda_min_128": lam128, "tr_solve": tr_solve, "sweep": sweep,
        "sweep_solve": sweep_solve,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
