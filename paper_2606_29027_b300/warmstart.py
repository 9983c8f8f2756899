"""Training data and training loop of the learned JFNK warm start (include/slar.h, section
"Learned JFNK warm start").  Orchestration only: the solver steps, the sample recording,
the network's forward/backward passes and the Adam updates all run in libslar.so's kernels;
this module chooses which samples form each mini-batch and keeps the tensors.

    samples = generate_samples(workloads, steps=200, n_probes=4, seed=7)
    net = slar.Net(m, n0, n1)
    train(net, samples, n_probes=4, iters=3000, batch=16, lr=2e-3, seed=1)
    save_params(net, path)
"""
from __future__ import annotations

import math
import os
import time
from typing import Iterable, List, Optional

import numpy as np

from . import inputs, slar

HERE = os.path.dirname(os.path.abspath(__file__))
WEIGHTS = os.path.join(HERE, "weights")
HIDDEN = 32


def spatial_shape(w: inputs.Workload):
    return (w.N[0], w.N[1]) if w.dx == 2 else (w.N[0], 1)


def init_params(m: int, seed: int, hidden: int = HIDDEN) -> np.ndarray:
    """Uniform(+-1/sqrt(fan_in)) weights, zero biases, last layer scaled by 0.1 (so the first
    guesses stay near U* and the block near the identity)."""
    rng = np.random.default_rng(seed)
    shapes = [(hidden, 2 * m), (hidden, hidden), (hidden, hidden), (m + m * m, hidden)]
    parts = []
    for l, (co, ci) in enumerate(shapes):
        a = 1.0 / math.sqrt(ci * 9) * (0.1 if l == len(shapes) - 1 else 1.0)
        parts += [rng.uniform(-a, a, size=co * ci * 9), np.zeros(co)]
    return np.concatenate(parts).astype(np.float32)


def run_solver(w: inputs.Workload, steps: int, precision: str = "fp32", solver: str = "precond",
               net: Optional["slar.Net"] = None, record=None, n_probes: int = 4, seed: int = 0,
               skip: int = 2):
    """Advance a fresh context `steps` steps; with `record` (a float32 CUDA tensor of shape
    [steps - skip, sample_floats]) the BDF3 steps from `skip` on write their training
    samples.  Returns the per-step stats dicts."""
    cfg = slar.make_config(w, precision=precision, solver=solver)
    ctx = slar.Context(cfg)
    if net is not None:
        ctx.attach_net(net)
    ctx.init_ht(inputs.initial_factors(w))
    out = []
    for s in range(steps):
        if record is not None and s >= skip:
            ctx.set_record(record[s - skip], n_probes, seed)
        st = ctx.step(w.dt)
        out.append(st.to_dict())
    ctx.close()
    return out


def generate_samples(workloads: Iterable[inputs.Workload], steps: int, n_probes: int, seed: int,
                     precision: str = "fp32", skip: int = 2):
    """Samples of the BDF3 steps of each workload (steps - skip per run), stacked in one
    float32 CUDA tensor [n_samples, sample_floats]."""
    import torch
    ws = list(workloads)
    w0 = ws[0]
    m = w0.dv + 2
    nx = int(np.prod(spatial_shape(w0)))
    L = slar.sample_floats(m, nx, n_probes)
    per = steps - skip
    buf = torch.empty((len(ws) * per, L), dtype=torch.float32, device="cuda")
    for r, w in enumerate(ws):
        if spatial_shape(w) != spatial_shape(w0) or w.dv != w0.dv:
            raise ValueError("all workloads must share the spatial grid")
        run_solver(w, steps, precision=precision, record=buf[r * per:(r + 1) * per], n_probes=n_probes,
                   seed=seed + 1000003 * r, skip=skip)
    torch.cuda.synchronize()
    return buf


def train(net: "slar.Net", samples, n_probes: int, iters: int, batch: int, lr: float, seed: int,
          log_every: int = 0, lr_final: Optional[float] = None) -> List[float]:
    """Adam on mini-batches drawn without replacement within each epoch (host RNG), with a
    cosine decay from lr to lr_final.  Returns the losses that were read back."""
    import torch
    n = samples.shape[0]
    batch = min(batch, n, net.max_batch)
    rng = np.random.default_rng(seed)
    order = rng.permutation(n)
    pos = 0
    losses = []
    lr_final = lr * 0.05 if lr_final is None else lr_final
    for it in range(iters):
        if pos + batch > n:
            order = rng.permutation(n)
            pos = 0
        idx = torch.from_numpy(order[pos:pos + batch].astype(np.int32)).to("cuda")
        pos += batch
        frac = it / max(1, iters - 1)
        lr_t = lr_final + 0.5 * (lr - lr_final) * (1.0 + math.cos(math.pi * frac))
        want = bool(log_every) and (it % log_every == 0 or it == iters - 1)
        L = net.train_step(samples, n_probes, idx, lr_t, want_loss=want)
        if want:
            losses.append(L)
    return losses


def mean_loss(net: "slar.Net", samples, n_probes: int) -> float:
    import torch
    n = samples.shape[0]
    tot = 0.0
    for a in range(0, n, net.max_batch):
        idx = torch.arange(a, min(n, a + net.max_batch), dtype=torch.int32, device="cuda")
        tot += net.loss_grad(samples, n_probes, idx) * idx.shape[0]
    return tot / n


def save_params(net: "slar.Net", path: str, meta: Optional[dict] = None):
    os.makedirs(os.path.dirname(path), exist_ok=True)
    np.save(path, net.get_params())
    if meta is not None:
        import json
        with open(path.replace(".npy", ".json"), "w") as f:
            json.dump(meta, f, indent=1, sort_keys=True)


def load_params(path: str) -> np.ndarray:
    return np.load(path).astype(np.float32)


def training_family(kind: str, n: int, runs: int, seed: int):
    """Seeded training workloads: kind "strong_landau" draws alpha ~ U[0.3, 0.6],
    k ~ U[0.4, 0.6] (rank cap 64 at n = 128); kind "weak_landau" draws alpha ~ U[0.005, 0.05],
    k ~ U[0.4, 0.6] with the 64^4 benchmark settings (cap 32, eps 1e-5, dt 0.2)."""
    rng = np.random.default_rng(seed)
    ws = []
    for _ in range(runs):
        k = float(rng.uniform(0.4, 0.6))
        if kind == "strong_landau":
            a = float(rng.uniform(0.3, 0.6))
            ws.append(inputs.landau_2d2v(n=n, alpha=a, k=k, cap=64 if n >= 128 else 16, dt=0.2))
        elif kind == "weak_landau":
            a = float(rng.uniform(0.005, 0.05))
            ws.append(inputs.landau_2d2v(n=n, alpha=a, k=k, cap=32 if n >= 64 else 16, dt=0.2))
        else:
            raise ValueError(kind)
    return ws


def main():
    """Generate samples from a seeded workload family, train, and save the parameters:
        python -m paper_2606_29027_b300.warmstart strong_landau 128 10 200
    """
    import argparse
    import torch
    ap = argparse.ArgumentParser()
    ap.add_argument("kind")
    ap.add_argument("n", type=int)
    ap.add_argument("runs", type=int)
    ap.add_argument("steps", type=int)
    ap.add_argument("--probes", type=int, default=4)
    ap.add_argument("--iters", type=int, default=4000)
    ap.add_argument("--batch", type=int, default=16)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--seed", type=int, default=7)
    ap.add_argument("--out", default=None)
    a = ap.parse_args()
    t0 = time.time()
    ws = training_family(a.kind, a.n, a.runs, a.seed)
    samples = generate_samples(ws, a.steps, a.probes, a.seed)
    t1 = time.time()
    w0 = ws[0]
    n0, n1 = spatial_shape(w0)
    net = slar.Net(w0.dv + 2, n0, n1, hidden=HIDDEN, max_batch=a.batch)
    net.set_params(init_params(w0.dv + 2, a.seed))
    L0 = mean_loss(net, samples, a.probes)
    losses = train(net, samples, a.probes, a.iters, a.batch, a.lr, a.seed, log_every=500)
    L1 = mean_loss(net, samples, a.probes)
    torch.cuda.synchronize()
    t2 = time.time()
    out = a.out or os.path.join(WEIGHTS, f"warmstart_{a.kind}_{a.n}.npy")
    meta = dict(kind=a.kind, n=a.n, runs=a.runs, steps=a.steps, samples=int(samples.shape[0]),
                probes=a.probes, iters=a.iters, batch=a.batch, lr=a.lr, seed=a.seed,
                loss_initial=L0, loss_final=L1, loss_log=losses, gen_s=t1 - t0, train_s=t2 - t1)
    save_params(net, out, meta)
    print(meta)


if __name__ == "__main__":
    main()
