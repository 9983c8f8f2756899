"""Benchmark: 2D-2V SLAR steps/s and sampled entries/s on the 2D-2V weak Landau workload
(64 points per dimension, tree ((x1,x2),(v1,v2)), rank cap 32, eps 1e-5, dt 0.2), with the
implicit LoMaC correction.  Headline: the precision-split path (FP32 entry evaluation; FP64
moments, truncation, LoMaC and Newton) with the block-circulant preconditioner of the
Newton-Krylov solve and block cross approximation (two fibres per step).  Beside it, on the
same steps: the plain FP64 path (the paper's unpreconditioned JFNK, one fibre per step), the
preconditioned FP64 path, FP32 entries with one fibre per step and with the learned JFNK warm
start (network trained in the same run, untimed, on samples of seeded weak-Landau runs that
the solver generates), each form's electric-energy history compared with an FP64 run
truncated 100 times more tightly; the 1D-1V weak Landau workload in microseconds per step.
The line ends with a compact summary of the forms.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--precision fp32|fp64] [--solver precond|plain|learned] [--workload NAME]

One JSON line on rank 0.  Multi-GPU runs are independent replicas (the method has no
data-parallel exchange): value = steps of all ranks / max-over-ranks time.
The reference arm (--impl reference) times the FP64 CPU oracle on the host cores.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "2D2V SLAR steps/s"
UNIT = "steps/s"
FP32_PEAK_TFLOPS = 148 * 128 * 2 * 2.032e9 / 1e12   # 148 SMs x 128 FP32 lanes x FMA x 2032 MHz
FP64_PEAK_TFLOPS = 1.25                              # nominal B300 FP64 (recipe table)
# DRAM bytes (read + write) per launch of the entry evaluator on this workload, by entry
# precision, from an ncu capture (cold cache); None where no capture of the current kernel
# exists
EVAL_TRAFFIC_BYTES = {"fp32": 295542.0, "fp64": None}
EVAL_TRAFFIC_SOURCE = ("ncu dram__bytes_read.sum + dram__bytes_write.sum, mean over 26 launches of "
                       "k_sl_eval_dev<float> in the warm-up steps of this workload (block cross "
                       "approximation b = 2; cold cache under ncu)")


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--precision", default="fp32", choices=["fp32", "fp64", "bf16x3", "bf16x6"],
                   help="entry precision of the headline run (bf16x3: 2D2V workloads, "
                        "--profile-step only)")
    p.add_argument("--workload", default="landau_2d2v")
    p.add_argument("--fp64-steps", type=int, default=None,
                   help="steps of the comparison forms (default: --steps, the same steps as the headline)")
    p.add_argument("--solver", default="precond", choices=["learned", "precond", "plain"])
    p.add_argument("--aca-block", type=int, default=2,
                   help="fibres per cross-approximation step of the headline form (1: partial "
                        "pivoting; 2..8: block cross approximation)")
    p.add_argument("--block-forms", default="2,4,8",
                   help="block sizes timed as extra forms of the headline precision and solver")
    p.add_argument("--c1-steps", type=int, default=200,
                   help="steps of the 1D-1V weak Landau workload timed in microseconds per step "
                        "(0 skips it)")
    p.add_argument("--train-runs", type=int, default=8)
    p.add_argument("--train-steps", type=int, default=40)
    p.add_argument("--train-iters", type=int, default=1500)
    p.add_argument("--large-steps", type=int, default=3,
                   help="timed steps of the 128^4 configurations (0 skips them)")
    p.add_argument("--c5-steps", type=int, default=8,
                   help="BDF3 steps of the 128^4 strong-Landau learned / precond / plain comparison (0: skip)")
    p.add_argument("--ensemble-runs", type=int, default=64)
    p.add_argument("--ensemble-steps", type=int, default=3)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--profile-eval", default=None, choices=["fp64", "fp32", "bf16x3", "bf16x6"],
                   help="evaluator microbenchmark: one warm-up and one measured sl_eval launch on "
                        "a random 2D2V HT (--eval-rank, --eval-n points per dimension, "
                        "--eval-entries tuples), for ncu captures of the evaluator kernels")
    p.add_argument("--eval-rank", type=int, default=64)
    p.add_argument("--eval-n", type=int, default=128)
    p.add_argument("--eval-entries", type=int, default=65536)
    p.add_argument("--oracle-timing", action="store_true",
                   help="time the FP64 oracle (1 BDF3 step after 2 start-up steps) and print it")
    p.add_argument("--profile-step", action="store_true",
                   help="profiling configuration: init, 3 steps, then one BDF3 step with every "
                        "kernel launched individually; prints the launch counts for ncu -s/-c")
    return p.parse_args()


def workload_config(w, precision, solver="plain"):
    return {"workload": f"{w.name}: 2D-2V weak Landau damping, alpha {w.alpha}, k {w.k}, "
                        f"{w.N[0]} pts/dim, x in [0,4pi)^2, v in [-6,6]^2, tree ((x1,x2),(v1,v2)), "
                        f"rank cap {w.rank_cap}, eps {w.eps}, dt {w.dt}, LoMaC with BDF3 (DIRK3 start-up), "
                        f"Newton tol {w.newton_tol}",
            "entries_precision": precision, "rest_precision": "fp64",
            "newton_krylov": {"plain": "JFNK from U(F*), unpreconditioned GMRES (the paper)",
                              "precond": "block-circulant right preconditioner",
                              "learned": "network guess and per-point block on top of the "
                                         "block-circulant preconditioner; plain JFNK fallback"}[solver],
            "timed_steps": "BDF3 steps after the DIRK3 start-up (in warm-up)",
            "l2": "flushed between timed steps (256 MiB write, outside the step events)",
            "global_batch": 1, "parallelism": "replicas"}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons during the timed region."""

    def __init__(self, index):
        self.index = index
        self.samples = []
        self.proc = None

    def start(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except FileNotFoundError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.samples.append([x.strip() for x in line.split(",")])

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.3)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm = [float(s[1]) for s in self.samples if len(s) >= 9 and s[1].replace(".", "").isdigit()]
        mx = [float(s[2]) for s in self.samples if len(s) >= 9 and s[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for s in self.samples if len(s) >= 9
                          for i in range(4) if s[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(self.samples)}


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def cpu_threads():
    try:
        from threadpoolctl import threadpool_info
        n = max((i.get("num_threads", 1) for i in threadpool_info()), default=1)
        return int(n)
    except Exception:
        return os.cpu_count() or 1


def max_over_ranks(x, world, device):
    """The slowest rank's value of x (all ranks get it); x itself on one rank."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(world, steps, max_ms):
    """Whole-job throughput of independent replicas: the steps of all ranks over the slowest
    rank's timed region."""
    return world * steps / (max_ms / 1000.0)


def oracle_steps(w, n_warm, n_timed):
    """Time the FP64 oracle: n_warm untimed steps (DIRK3 start-up), then n_timed steps."""
    from oracle import sl, stepper
    from paper_2606_29027_b300 import inputs
    g = sl.PhaseGrid(w.dx, w.dv, w.N, w.lo, w.hi)
    prm = stepper.Params(eps=w.eps, cap=w.rank_cap, newton_tol=w.newton_tol)
    st = stepper.init_state(inputs.initial_factors(w), g, prm)
    for _ in range(n_warm):
        stepper.sl_step(st, w.dt, g, prm)
    t0 = time.perf_counter()
    ent = 0
    for _ in range(n_timed):
        ent += stepper.sl_step(st, w.dt, g, prm).entries
    dt = time.perf_counter() - t0
    return n_timed / dt, ent / dt, dt


def oracle_single_thread(workload):
    """The same oracle timing in a child process whose BLAS / OpenMP pools have one thread
    (the variables must be set before numpy loads).  Returns steps/s or None."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    try:
        r = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-timing", "--workload", workload],
                           env=env, capture_output=True, text=True, timeout=600)
        return float(json.loads(r.stdout.strip().splitlines()[-1])["steps_per_s"])
    except (subprocess.SubprocessError, ValueError, IndexError, KeyError):
        return None


def run_reference(args, w):
    world, rank, _ = dist_setup(args)
    if rank != 0:
        return
    n_warm = max(2, min(args.warmup, 3))
    n_timed = max(1, min(args.steps, 6))
    sps, eps_, dt = oracle_steps(w, n_warm, n_timed)
    cores = cpu_threads()
    sample = (f"{n_timed} oracle BDF3 steps of {w.name} after {n_warm} untimed start-up steps, "
              f"{dt:.1f} s")
    line = {"impl": "reference", "metric": METRIC, "value": sps, "unit": UNIT, "n_gpus": args.gpus,
            "steps": n_timed, "warmup": n_warm, "ms_per_step": 1000.0 / sps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(w, "fp64"),
            "entries_per_s": eps_,
            "cpu_baseline": {"value": sps, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": sps, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def time_steps(ctx, w, K, flush, stream):
    import torch
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    stats = []
    with torch.cuda.stream(stream):
        for i in range(K):
            ev[i][0].record(stream)
            s = ctx.step(w.dt)
            ev[i][1].record(stream)
            stats.append(s)
            flush.zero_()
    torch.cuda.synchronize()
    ms = [a.elapsed_time(b) for a, b in ev]
    return ms, stats


def run_ours(args, w):
    import torch
    from paper_2606_29027_b300 import inputs, slar

    world, rank, local = dist_setup(args)
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    stream = torch.cuda.Stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    fac = inputs.initial_factors(w)

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    net = None
    train_info = None
    if args.train_iters > 0:
        # untimed: samples from seeded weak-Landau runs (alpha ~ U[0.005, 0.05], k ~ U[0.4,
        # 0.6]; the benchmark run itself, alpha 0.01 and k 0.5, is not among them), then Adam
        from paper_2606_29027_b300 import warmstart
        tt0 = time.perf_counter()
        fam = warmstart.training_family("weak_landau", w.N[0], args.train_runs, seed=7 + rank)
        with torch.cuda.stream(stream):
            samples = warmstart.generate_samples(fam, args.train_steps, 4, seed=7 + rank)
            n0, n1 = warmstart.spatial_shape(w)
            net = slar.Net(w.dv + 2, n0, n1, max_batch=16, stream=stream)
            net.set_params(warmstart.init_params(w.dv + 2, 7))
            L0 = warmstart.mean_loss(net, samples, 4)
            warmstart.train(net, samples, 4, args.train_iters, 16, 2e-3, seed=1)
            L1 = warmstart.mean_loss(net, samples, 4)
        torch.cuda.synchronize()
        train_info = {"samples": int(samples.shape[0]), "runs": args.train_runs,
                      "steps_per_run": args.train_steps, "adam_iters": args.train_iters,
                      "loss_initial": L0, "loss_final": L1,
                      "seconds": time.perf_counter() - tt0,
                      "family": "2D2V weak Landau, alpha ~ U[0.005,0.05], k ~ U[0.4,0.6], seed 7"}
        del samples
    if args.solver == "learned" and net is None:
        raise SystemExit("--solver learned needs the trained network (--train-iters > 0)")

    def make(precision, profile, profile_eval=False, solver=None, wl=None, block=None):
        solver = args.solver if solver is None else solver
        cfg = slar.make_config(wl or w, precision=precision, profile=profile, profile_eval=profile_eval,
                               solver=solver, aca_block=args.aca_block if block is None else block)
        c = slar.Context(cfg, stream=stream)
        if solver == "learned":
            c.attach_net(net)
        return c

    def eval_roofline(precision, solver=None, steps=3):
        # separate pass: events around every evaluator launch (cross approximation launched
        # step by step instead of as a graph); same kernels, same workload
        cp = make(precision, True, True, solver=solver)
        with torch.cuda.stream(stream):
            cp.init_ht(fac)
            for _ in range(3):
                cp.step(w.dt)
        barrier()
        _, stp = time_steps(cp, w, steps, flush, stream)
        em = sum(s.eval_ms for s in stp)
        ef = sum(s.eval_flop for s in stp)
        nl = sum(s.entries for s in stp)
        del cp
        return em, ef, nl

    # ---- device-resident timed run (headline form) ----
    # an untimed pass of the same form and steps first: the evaluator's tile autotuner keeps
    # its choices per process and rank bucket, so the timed run does not tune inside its steps
    pre = make(args.precision, True)
    with torch.cuda.stream(stream):
        pre.init_ht(fac)
        for _ in range(max(3, args.warmup) + args.steps):
            pre.step(w.dt)
    del pre
    barrier()
    ctx = make(args.precision, True)
    with torch.cuda.stream(stream):
        ctx.init_ht(fac)
        warm_stats = [ctx.step(w.dt) for _ in range(max(3, args.warmup))]
    barrier()
    clk = ClockSampler(local)
    clk.start()
    l0 = slar.launch_count()
    barrier()
    t0 = time.perf_counter()
    ms, stats = time_steps(ctx, w, args.steps, flush, stream)
    barrier()
    wall = time.perf_counter() - t0
    launches = slar.launch_count() - l0
    clocks = clk.stop()
    tot_ms = max_over_ranks(float(sum(ms)), world, "cuda")
    value = job_value(world, args.steps, tot_ms)
    entries = sum(s.entries for s in stats)
    eval_ms, eval_flop, eval_entries = eval_roofline(args.precision)
    converged = all(s.converged for s in stats)
    phase_names = ["cross_approx", "truncation", "fields_moments", "lomac_closure", "newton_krylov", "diagnostics"]
    phases = {nm: sum(s.phase_ms[i] for s in stats) / args.steps for i, nm in enumerate(phase_names)}
    del ctx

    # ---- the other forms on the same steps ----
    def short_run(precision, solver, K, eps=None, cap=None, block=1):
        if eps is None:
            cc = make(precision, True, solver=solver, block=block)
        else:
            cfg = slar.make_config(w, precision=precision, profile=True, solver=solver)
            cfg.eps, cfg.rank_cap = eps, cap
            cc = slar.Context(cfg, stream=stream)
        with torch.cuda.stream(stream):
            cc.init_ht(fac)
            warm = [cc.step(w.dt) for _ in range(max(3, args.warmup))]
        barrier()
        msk, stk = time_steps(cc, w, K, flush, stream)
        del cc
        return msk, warm + stk

    def summary(msk, stk, K):
        tk = float(sum(msk))
        return {"value": K / (tk / 1000.0), "unit": UNIT, "ms_per_step": tk / K,
                "entries_per_s": sum(s.entries for s in stk[-K:]) / (tk / 1000.0),
                "newton_per_step": float(np.mean([s.newton for s in stk[-K:]])),
                "krylov_per_step": float(np.mean([s.krylov for s in stk[-K:]])),
                "g_evals_per_step": float(np.mean([s.g_evals for s in stk[-K:]])),
                "guess_used_steps": int(sum(s.guess_used for s in stk[-K:])),
                "launches_per_step": float(np.mean([s.launches for s in stk[-K:]])),
                "phase_ms_per_step": {nm: sum(s.phase_ms[i] for s in stk[-K:]) / K
                                      for i, nm in enumerate(phase_names)}}

    head_key = f"{args.precision}_{args.solver}" + (f"_b{args.aca_block}" if args.aca_block > 1 else "")
    forms = {}
    W_hist = {head_key: np.array([s.field_energy for s in (warm_stats + stats)])}
    Kh = args.steps
    forms[head_key] = summary(ms, warm_stats + stats, Kh)
    K = args.steps if args.fp64_steps is None else args.fp64_steps
    acc = None
    if K > 0:
        wanted = [("fp64", "plain", 1), ("fp64", "precond", args.aca_block), ("fp32", "precond", 1)]
        wanted += [("fp32", "learned", 1)] if net is not None else []
        wanted += [(args.precision, args.solver, int(b)) for b in args.block_forms.split(",") if b and int(b) > 1]
        if args.aca_block > 1:
            wanted.append((args.precision, args.solver, 1))
        for prec, solver, blk in wanted:
            key = f"{prec}_{solver}" + (f"_b{blk}" if blk > 1 else "")
            if key == head_key or key in forms:
                continue
            msk, stk = short_run(prec, solver, K, block=blk)
            forms[key] = summary(msk, stk, K)
            W_hist[key] = np.array([s.field_energy for s in stk])
        em64, ef64, _ = eval_roofline("fp64", "plain", 2)
        forms["fp64_plain"]["eval_tflops"] = ef64 / max(em64, 1e-9) / 1e9
        # accuracy: electric-energy history W(t) of each form against an FP64 run truncated
        # 100 times more tightly (rank cap 64), on the same steps
        _, stref = short_run("fp64", "plain", K, eps=w.eps / 100.0, cap=64)
        Wref = np.array([s.field_energy for s in stref])
        n = min([len(Wref)] + [len(v) for v in W_hist.values()])
        scale = np.max(np.abs(Wref[:n]))
        acc = {"steps_compared": n, "reference": f"FP64 plain, eps {w.eps / 100.0:g}, rank cap 64",
               "measure": "max over steps of |W - W_ref| / max |W_ref|",
               "note": "weak Landau perturbs f by alpha = 0.01, so a truncation error eps ||f|| is "
                       "eps / alpha relative to the field: the eps-1e-5 method itself is accurate "
                       "to about 1e-3 in W"}
        for key, Wk in W_hist.items():
            forms[key]["W_err"] = float(np.max(np.abs(Wk[:n] - Wref[:n])) / scale)
            if "fp64_plain" in W_hist:
                forms[key]["W_diff_vs_fp64_plain"] = float(np.max(np.abs(Wk[:n] - W_hist["fp64_plain"][:n])) / scale)

    # ---- the 1D-1V weak Landau workload (64 x 128, cap 16, eps 1e-6, dt 0.1): FP64, the
    # paper's JFNK; latency-bound, so microseconds per step ----
    c1 = None
    if args.c1_steps > 0:
        w1 = inputs.landau_1d1v()
        c1c = make("fp64", True, solver="plain", wl=w1)
        with torch.cuda.stream(stream):
            c1c.init_ht(inputs.initial_factors(w1))
            for _ in range(2):
                c1c.step(w1.dt)
        barrier()
        ms1, st1 = time_steps(c1c, w1, args.c1_steps - 2, flush, stream)
        c1 = {"workload": "landau_1d1v_64x128: alpha 0.01, k 0.5, cap 16, eps 1e-6, dt 0.1, FP64, plain JFNK; "
                          f"BDF3 steps 3..{args.c1_steps} (after the 2 DIRK3 steps)",
              "us_per_step": 1000.0 * float(np.mean(ms1)), "us_per_step_median": 1000.0 * float(np.median(ms1)),
              "launches_per_step": float(np.mean([s.launches for s in st1])),
              "W_last": st1[-1].field_energy, "converged": all(s.converged for s in st1)}
        del c1c

    # ---- the 128^4 configurations (strong Landau, two-stream, and the 2D-2V bump-on-tail
    # example of Sec. 4.2 at its eps 1e-4 and a CFL-5 step): FP32 SIMT entries vs BF16x3 and
    # BF16x6 tensor-core entries ----
    large = None
    if args.large_steps > 0:
        large = {}
        for wname in ("strong_landau_2d2v", "two_stream_2d2v", "bump_on_tail_2d2v"):
            wl = inputs.workload_by_name(wname)
            res = {}
            for prec in ("fp32", "bf16x3", "bf16x6"):
                cl = slar.Context(slar.make_config(wl, precision=prec, solver="precond", profile=True), stream=stream)
                with torch.cuda.stream(stream):
                    cl.init_ht(inputs.initial_factors(wl))
                    for _ in range(3):
                        cl.step(wl.dt)
                barrier()
                msl, stl = time_steps(cl, wl, args.large_steps, flush, stream)
                tl = float(sum(msl))
                res[prec] = {"value": args.large_steps / (tl / 1000.0), "unit": UNIT,
                             "ms_per_step": tl / args.large_steps,
                             "entries_per_s": sum(x.entries for x in stl) / (tl / 1000.0),
                             "phase_ms_per_step": {nm: sum(x.phase_ms[i] for x in stl) / args.large_steps
                                                   for i, nm in enumerate(phase_names)},
                             "ranks_last": list(stl[-1].ranks), "W_last": stl[-1].field_energy}
                del cl
            res["speedup_bf16x3"] = res["bf16x3"]["value"] / res["fp32"]["value"]
            res["speedup_bf16x6"] = res["bf16x6"]["value"] / res["fp32"]["value"]
            res["workload"] = (f"{wl.name}: alpha {wl.alpha}, k {wl.k}, rank cap {wl.rank_cap}, eps {wl.eps}, "
                               f"dt {wl.dt}; block-circulant preconditioner; {args.large_steps} BDF3 steps "
                               f"after the DIRK3 start-up")
            large[wname] = res

    # ---- the 2D-2V strong Landau configuration with the learned warm start: the network
    # trained (untimed, offline) on solver-generated samples of seeded strong-Landau runs at
    # 128^4 (alpha ~ U[0.3, 0.6], k ~ U[0.4, 0.6], seed 7; weights shipped with the package),
    # on the held-out run alpha 0.5, k 0.5; learned vs preconditioner alone vs the paper's
    # plain JFNK, FP32 entries, the same Newton tolerance ----
    c5 = None
    if args.c5_steps > 0:
        from paper_2606_29027_b300 import warmstart
        wpath = os.path.join(ROOT, "paper_2606_29027_b300", "weights", "warmstart_strong_landau_128.npy")
        held = inputs.landau_2d2v(n=128, alpha=0.5, k=0.5, cap=64, dt=0.2)
        c5 = {"workload": "2D2V strong Landau alpha 0.5, k 0.5, 128^4, v in [-6,6]^2, rank cap 64, eps 1e-5, "
                          f"dt 0.2; {args.c5_steps} BDF3 steps after the DIRK3 start-up; FP32 entries",
              "network": json.load(open(wpath.replace(".npy", ".json"))) if os.path.exists(wpath) else None}
        for solver in ("learned", "precond", "plain"):
            if solver == "learned" and not os.path.exists(wpath):
                continue
            cc = slar.Context(slar.make_config(held, precision="fp32", solver=solver, profile=True), stream=stream)
            net5 = None
            if solver == "learned":
                net5 = slar.Net(4, 128, 128, max_batch=1, stream=stream)
                net5.set_params(warmstart.load_params(wpath))
                cc.attach_net(net5)
            with torch.cuda.stream(stream):
                cc.init_ht(inputs.initial_factors(held))
                for _ in range(2):
                    cc.step(held.dt)
            barrier()
            ms5, st5 = time_steps(cc, held, args.c5_steps, flush, stream)
            t5 = float(sum(ms5))
            c5[solver] = {"value": args.c5_steps / (t5 / 1000.0), "unit": UNIT, "ms_per_step": t5 / args.c5_steps,
                          "newton_per_step": float(np.mean([x.newton for x in st5])),
                          "krylov_per_step": float(np.mean([x.krylov for x in st5])),
                          "g_evals_per_step": float(np.mean([x.g_evals for x in st5])),
                          "jfnk_ms_per_step": float(np.mean([x.phase_ms[4] for x in st5])),
                          "guess_used_steps": int(sum(x.guess_used for x in st5)),
                          "fallback_steps": int(sum(x.fallback for x in st5)),
                          "rank_capped_steps": int(sum(1 for x in st5 if x.rank_capped)),
                          "W_last": st5[-1].field_energy}
            del cc
            if net5 is not None:
                net5.close()

    # ---- ensemble of uneven runs (1D1V/2D2V Landau/two-stream, 32-128 points per
    # dimension, rank caps 8-48), concurrent on private streams vs one after another ----
    ensemble = None
    if args.ensemble_runs > 0:
        ews = inputs.ensemble(n_runs=args.ensemble_runs)
        ectx = []
        for ew in ews:
            ec = slar.Context(slar.make_config(ew, precision="fp32", solver="precond", own_stream=True))
            ec.init_ht(inputs.initial_factors(ew))
            ectx.append(ec)
        torch.cuda.synchronize()
        edts = [ew.dt for ew in ews]
        for _ in range(max(3, args.warmup)):
            slar.ensemble_step(ectx, edts, threads=16)
        torch.cuda.synchronize()
        ens = {}
        for label, thr in (("concurrent", 16), ("sequential", 1)):
            t0 = time.perf_counter()
            for _ in range(args.ensemble_steps):
                est = slar.ensemble_step(ectx, edts, threads=thr)
            torch.cuda.synchronize()
            ens[label] = len(ews) * args.ensemble_steps / (time.perf_counter() - t0)
        ensemble = {"metric": "run-steps/s", "runs": len(ews), "steps": args.ensemble_steps,
                    "concurrent": ens["concurrent"], "sequential": ens["sequential"],
                    "speedup": ens["concurrent"] / ens["sequential"],
                    "threads": 16, "converged": all(s.converged for s in est),
                    "tiles_chosen": sorted({s.eval_tile for s in est}),
                    "workload": "64 seeded runs (PCG64 seed 20261202): 1D1V/2D2V x Landau/"
                                "two-stream round-robin, alpha ~ U[0.001,0.5], k ~ U[0.2,0.6], "
                                "N per dim in {32,64,128}, caps ~ U{8..48}, eps 1e-5, dt 0.1, "
                                "FP32 entries, block-circulant preconditioner, after the DIRK3 "
                                "start-up; host wall clock around each ensemble step"}
        for ec in ectx:
            ec.close()
        del ectx

    # ---- end to end through the C ABI with host buffers (headline form) ----
    e2e_steps = max(3, args.warmup) + min(args.steps, 10)
    ctx_e = make(args.precision, False)
    U_host = torch.empty((w.dv + 2, ctx_e.NX), dtype=torch.float64, pin_memory=True)
    U_dev = torch.empty((w.dv + 2, ctx_e.NX), dtype=torch.float64, device="cuda")
    h2d = sum(sum(np.asarray(f).nbytes for f in term) for term in fac)
    barrier()
    t0 = time.perf_counter()
    with torch.cuda.stream(stream):
        ctx_e.init_ht(fac)                       # host factors -> device
        for _ in range(e2e_steps):
            ctx_e.step(w.dt)                     # stats returned to host
            ctx_e.get_conserved(U_dev)
            U_host.copy_(U_dev, non_blocking=True)
        stream.synchronize()
    e2e_t = time.perf_counter() - t0
    e2e = {"value": e2e_steps / e2e_t, "unit": UNIT, "h2d_bytes_per_step": h2d / e2e_steps,
           "d2h_bytes_per_step": U_host.numel() * 8 + 200,
           "note": "fresh context: init_ht upload of the host initial data, DIRK3 start-up and "
                   "BDF3 steps, each step's U^{n+1} and stats read back to host"}

    if rank != 0:
        return
    with torch.cuda.stream(stream):
        peak32 = max(slar.fma_peak(False, stream=stream) for _ in range(3))
        peak64 = max(slar.fma_peak(True, stream=stream) for _ in range(3))
    peak = peak32 if args.precision == "fp32" else peak64
    # where the arithmetic dominates: the same evaluators at rank 64 on one 65536-entry launch
    bf16, bf16_src = bf16_peak_tflops()
    eval64 = {"workload": "random HT, all six ranks 64, 2D2V 128^4, 65536 random tuples, RK3 feet; "
                          "median of 3 launches after one warm-up",
              "flop_per_entry": 2 * (3 * 4 * 64 + 2 * 64 ** 3 + 64 * 64) + 60}
    for prec, pk, src in (("fp32", peak32, "measured FP32 FMA peak (this run)"),
                          ("bf16x3", bf16 / 3.0, bf16_src + " / 3 (three BF16 products per K-step)"),
                          ("bf16x6", bf16 / 6.0, bf16_src + " / 6 (six BF16 products per K-step)")):
        ms64, tf64 = eval_launch(prec, 64, 128, 65536, reps=3)
        eval64[prec] = {"kernel": "k_sl_eval<float> (GEMM contraction)" if prec == "fp32"
                        else f"k_sl_eval_tc (tcgen05, {prec.upper()})",
                        "ms": ms64, "tflops": tf64, "peak_tflops": pk, "frac": tf64 / pk, "peak_source": src}
    achieved = eval_flop / max(eval_ms, 1e-9) / 1e9          # TFLOP/s
    traffic = EVAL_TRAFFIC_BYTES.get(args.precision)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": max(3, args.warmup), "ms_per_step": tot_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp32": "f32", "fp64": "f64", "bf16x3": "bf16x3", "bf16x6": "bf16x6"}[args.precision], "data": "synthetic",
            "config": workload_config(w, args.precision, args.solver),
            "entries_per_s": entries / (tot_ms / 1000.0) * world,
            "entries_per_step": entries / args.steps,
            "converged": converged,
            "ranks_last": list(stats[-1].ranks),
            "forms": forms,
            "accuracy": acc,
            "warm_start_training": train_info,
            "ensemble": ensemble,
            "large_128": large,
            "c5_strong_landau_learned": c5,
            "newton_per_step": float(np.mean([s.newton for s in stats])),
            "krylov_per_step": float(np.mean([s.krylov for s in stats])),
            "roofline": {"kernel": f"k_sl_eval_dev<{'double' if args.precision == 'fp64' else 'float'}> "
                                   "(SL entry evaluator)", "bound": "alu",
                         "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak,
                         "traffic": traffic,
                         "traffic_source": EVAL_TRAFFIC_SOURCE if traffic is not None else None,
                         "peak_source": "measured in this run: FMA-chain kernel (slar_fma_peak), "
                                        "best of 3; derived FP32 148 SMs x 128 lanes x 2 x 2032 MHz = "
                                        f"{FP32_PEAK_TFLOPS:.1f}, nominal FP64 {FP64_PEAK_TFLOPS}",
                         "measured_fp32_tflops": peak32, "measured_fp64_tflops": peak64,
                         "eval_share_of_step": (eval_ms / 3.0) / (tot_ms / args.steps),
                         "method": "separate profiled pass of 3 steps: CUDA events around each "
                                   "evaluator launch on the library stream; algorithmic flops "
                                   "2(3 sum r_mu + r0 r1 r12 + r2 r3 r34 + r12 r34) + 60 per entry",
                         "eval_ms_per_step": eval_ms / 3.0},
            "eval_rank64": eval64,
            "phase_ms_per_step": phases,
            "gpu_launches": launches, "wall_s": wall, "clocks": clocks, "e2e": e2e,
            "c1_landau_1d1v": c1}
    if not args.no_cpu_baseline and world == 1:
        sps, eps_, dt = oracle_steps(w, 2, 1)
        cores = cpu_threads()
        sps1 = oracle_single_thread(args.workload)
        line["cpu_baseline"] = {"value": sps, "unit": UNIT, "cores": cores, "kind": "oracle",
                                "sample": f"1 oracle BDF3 step of {w.name} after 2 untimed DIRK3 "
                                          f"start-up steps ({dt:.1f} s); entries/s {eps_:.3g}",
                                "single_thread": sps1}
    # compact summary last, so that it stays in a short tail of the output
    line["summary"] = {
        "headline": f"{head_key}: {value:.1f} steps/s, W_err {forms[head_key].get('W_err', float('nan')):.1e}",
        "forms_steps_per_s": {k: round(v["value"], 2) for k, v in forms.items()},
        "forms_W_err": {k: v.get("W_err") for k, v in forms.items()},
        "forms_launches_per_step": {k: round(v["launches_per_step"], 1) for k, v in forms.items()},
        "learned_guess_used_steps": forms.get("fp32_learned", {}).get("guess_used_steps"),
        "c1_us_per_step": c1["us_per_step"] if c1 else None,
        "c5_g_evals_per_step": ({k: round(v["g_evals_per_step"], 1) for k, v in c5.items()
                                 if isinstance(v, dict) and "g_evals_per_step" in v} if c5 else None),
        "cpu_single_thread_steps_per_s": line.get("cpu_baseline", {}).get("single_thread"),
        "roofline_frac": achieved / peak}
    print(json.dumps(line), flush=True)


def profile_step(args, w):
    import torch
    from paper_2606_29027_b300 import inputs, slar
    # autotuner off: launch counts (ncu -s / -c) must not depend on timings
    ctx = slar.Context(slar.make_config(w, precision=args.precision, profile_eval=True, solver=args.solver,
                                        autotune=False, aca_block=args.aca_block))
    if args.solver == "learned":
        # untrained parameters: the same kernels and launch structure as the trained network
        from paper_2606_29027_b300 import warmstart
        n0, n1 = warmstart.spatial_shape(w)
        net = slar.Net(w.dv + 2, n0, n1, max_batch=1)
        net.set_params(warmstart.init_params(w.dv + 2, 7))
        ctx.attach_net(net)
    ctx.init_ht(inputs.initial_factors(w))
    for _ in range(3):
        ctx.step(w.dt)
    torch.cuda.synchronize()
    l0 = slar.launch_count()
    s = ctx.step(w.dt)
    torch.cuda.synchronize()
    print("WARM_LAUNCHES", l0, "STEP_LAUNCHES", slar.launch_count() - l0, json.dumps(s.to_dict()),
          flush=True)


def eval_launch(precision, r, n, entries, reps=1):
    """Time one entry-evaluator launch (CUDA events on the current stream, after one warm-up;
    median of reps) on a random 2D2V HT with all six ranks r, n points per dimension and
    `entries` random tuples (RK3 feet).  Returns (ms, algorithmic TFLOP/s)."""
    import torch
    from paper_2606_29027_b300 import inputs, slar
    N = (n, n, n, n)
    L = 4 * math.pi
    cfg = slar.make_config(dx=2, dv=2, N=N, lo=(0, 0, -6, -6), hi=(L, L, 6, 6), eps=1e-6, rank_cap=64,
                           precision=precision)
    ctx = slar.Context(cfg)
    h = inputs.random_ht(N, (r,) * 6, seed=5)
    ctx.import_ht(U=h.U, Broot=h.Broot, B12=np.transpose(h.B12, (2, 0, 1)), B34=np.transpose(h.B34, (2, 0, 1)))
    E = torch.as_tensor(inputs.random_field(N[:2], 2, 0.6, seed=4), device="cuda")
    idx = torch.as_tensor(inputs.random_tuples(N, entries, seed=7), device="cuda")
    out = torch.zeros(entries, dtype=torch.float64, device="cuda")
    ctx.sl_eval(1.1, E, idx, out)
    torch.cuda.synchronize()
    times = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        ctx.sl_eval(1.1, E, idx, out)
        b.record()
        torch.cuda.synchronize()
        times.append(a.elapsed_time(b))
    ctx.close()
    ms = statistics.median(times)
    flop = (2 * (3 * 4 * r + 2 * r ** 3 + r * r) + 60) * entries
    return ms, flop / ms / 1e9


def bf16_peak_tflops():
    """Dense BF16 burst peak from MEASURED_PEAKS.json when present, else the fallback figure."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["bf16_tflops"]), "MEASURED_PEAKS.json bf16_tflops (burst)"
    except (OSError, KeyError, ValueError):
        return 1800.0, "fallback 1.8 PFLOP/s bf16 burst (no MEASURED_PEAKS.json)"


def profile_eval(args):
    """Time the entry evaluator alone (CUDA events, one launch after one warm-up)."""
    ms, tflops = eval_launch(args.profile_eval, args.eval_rank, args.eval_n, args.eval_entries)
    print(json.dumps({"profile_eval": args.profile_eval, "rank": args.eval_rank, "n": args.eval_n,
                      "entries": args.eval_entries, "ms": ms, "tflops": tflops}), flush=True)


def main():
    args = parse()
    if args.profile_eval:
        profile_eval(args)
        return
    from paper_2606_29027_b300 import inputs
    w = inputs.workload_by_name(args.workload)
    if args.oracle_timing:
        sps, eps_, dt = oracle_steps(w, 2, 1)
        print(json.dumps({"steps_per_s": sps, "entries_per_s": eps_, "seconds": dt}), flush=True)
        return
    if args.profile_step:
        profile_step(args, w)
        return
    if args.precision in ("bf16x3", "bf16x6"):
        raise SystemExit(f"--precision {args.precision} is for --profile-step; the benchmark reports the "
                         "tensor-core splits in its 128^4 and eval_rank64 sections")
    if args.impl == "reference":
        run_reference(args, w)
    else:
        run_ours(args, w)


if __name__ == "__main__":
    main()
