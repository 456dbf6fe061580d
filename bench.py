"""Benchmark of the efunc hot path on GB300.

One step = one fitting iteration on a fresh batch of J = 2^22 (x, y, z, SDF)
rows at R = 32 (32^3 x 13 parameters): cell sort, fused forward + L1 loss
gradient + backward (gradient scatter), Adam.  The batch pool (3 batches of
64 MiB, 192 MiB > the 129 MB L2) is resident in HBM before the timed region;
consecutive steps use different batches.

Printed JSON line (rank 0):
  value           query-points/s over all ranks (J * steps * ranks / time)
  roofline        the fused forward/backward kernel against the FP32 pipe
                  (ALU bound): algorithmic FP32 operations per launch /
                  average launch time from CUDA events on its stream
  e2e             the same metric through efunc_fit with the batches in
                  pinned host memory: every step copies its batch to the
                  device and reads the (loss, MAE) pair back
  cpu_baseline    the FP64 oracle on the host cores, on a sample
  clocks          nvidia-smi samples taken during the timed region

``--impl reference`` times the FP64 oracle (the only reference available) on
the same workload, a bounded sample per step.

Multi-GPU: replicas only.  Under torchrun every rank fits its own batch pool
on its own GPU; no collective touches the data path.
"""
from __future__ import annotations

import argparse
import json
import math
import multiprocessing as mp
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

R_DEFAULT = 32
J_DEFAULT = 1 << 22
N_BATCHES = 3
LR = 1e-3
# Algorithmic FP32 operations per (query, centre) of the fused fit step:
# forward 12 per key (difference 3, squared distance 3, scale 1, value 3,
# two accumulations 2), backward 18 for the grid key and 21 for the offset
# key (recomputed difference, distance, exponent, weight times dL/dO, value,
# residual, and the 5 / 8 gradient sums).  In an interior (full 4x4x4)
# window the grid keys sit on the lattice, so their forward needs 7 (the
# squared distance from per-axis terms formed once per query: 24 operations).
OPS_PER_CENTRE = 12 + 12 + 18 + 21
OPS_PER_CENTRE_FULL = 7 + 12 + 18 + 21
OPS_PER_QUERY_FULL_SETUP = 24
EX2_PER_CENTRE = 4
# The fit step with the Eikonal term (backward through dO/dq), per (query,
# centre), adds to the counts above: a second forward pass forming dO/dq
# and V = sum w beta (q - key), 24 per key (difference 3, squared distance 3,
# exponent 1, value 3, w beta 2, 2 beta w (O - f) 3, dO/dq 6, V 3); and in the
# backward the derivative of u . dO/dq, 23 per grid key (u.r 3, u.t 1, u.d 3,
# h 1, w (u.t - T) 2, (h - H) - dlt T 2, 7 sums, log-scale term 4) and 8 more
# for an offset key (its 6 position sums and 2 products).  Per-query terms
# (residual, u, H, T) are left out.
EIK_GV_PER_KEY = 24
EIK_BWD_GRID_EXTRA = 23
EIK_BWD_OFFSET_EXTRA = 23 + 8
EIK_EXTRA_PER_CENTRE = 2 * EIK_GV_PER_KEY + EIK_BWD_GRID_EXTRA + EIK_BWD_OFFSET_EXTRA
FP32_LANES_PER_SM = 128
# steps of one whole fit: 2000 at 32^3 x 2^22 queries, 100 at 16^3 x 65,536
# (fits/s = 1 / (steps x time per step))
FIT_STEPS_32 = 2000
FIT_STEPS_16 = 100
# plain fits to the MAE target: held-out points (half uniform, half near the
# surface), the target of the metric, and the steps between evaluations
HELDOUT = 1 << 20
TARGET_MAE = 1e-3
TARGET_CHUNK = 50
# batched fit: shapes fitted together
BATCH_SHAPES = 256
# learned warm start: encoder batch (shapes per step); multiply-adds per
# voxel of one training step's tensor-core convolutions at the real channel
# counts: forward L2 27*32*64, L3 27*64*128, L4 128*13; the same again for
# the weight gradients and for the input gradients
WARM_BATCH = 16
ENC_MACS_PER_VOXEL = 3 * (27 * 32 * 64 + 27 * 64 * 128 + 128 * 13)
ENC_PROFILE_STEPS = 5
# FP32-pipe operations of one (centre, point) pair of the mean-shift
# initialisation: 3 differences, 3 for the squared norm, 1 scale, 1 compare,
# 1 exponent difference, 1 add to Z, 3 FMAs into S (the ex2 runs on the MUFU)
MEAN_SHIFT_OPS_PER_PAIR = 13
WORKLOAD = "C2 plain fit: 32^3x13 FP32 grid, 2^22 queries/step (50% uniform, 50% surface+N(0,0.01^2)), " \
           "union of 8 random primitives, L1 loss, Adam lr 1e-3"


def kernel_source_hash() -> str:
    """SHA-256 of the fused kernel's sources with comments and blank lines
    removed, so that the hash follows the code, not its prose."""
    import hashlib
    import re
    h = hashlib.sha256()
    for f in ("paper_2505_21319_gb300/csrc/fused.cu", "paper_2505_21319_gb300/csrc/common.cuh"):
        src = open(os.path.join(ROOT, f)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        lines = [ln.rstrip() for ln in src.splitlines() if ln.strip()]
        h.update("\n".join(lines).encode())
    return h.hexdigest()


def fused_traffic():
    """DRAM bytes per fused launch from the committed ncu summary, or None when
    the kernel's code changed since that capture."""
    import re
    try:
        txt = open(os.path.join(ROOT, "profiles", "fused_fit_32cubed_2p22.md")).read()
    except OSError:
        return None
    sha = re.search(r"source_sha256:\s*([0-9a-f]{64})", txt)
    tb = re.search(r"traffic_bytes_per_launch:\s*(\d+)", txt)
    if not sha or not tb or sha.group(1) != kernel_source_hash():
        return None
    return int(tb.group(1))


def json_safe(x):
    """x with every non-finite float replaced by None (strict JSON)."""
    if isinstance(x, dict):
        return {k: json_safe(v) for k, v in x.items()}
    if isinstance(x, (list, tuple)):
        return [json_safe(v) for v in x]
    if isinstance(x, float) and not math.isfinite(x):
        return None
    return x


def max_over_ranks(x: float, device=None) -> float:
    """Max of a per-rank scalar over all ranks (identity without a process group)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def algorithmic_ops(q: np.ndarray, R: int) -> float:
    """Exact algorithmic FP32 operations of one fused fit launch over the batch q."""
    nc = centres_per_query(q, R)
    full = nc == 64
    return float(full.sum()) * (64 * OPS_PER_CENTRE_FULL + OPS_PER_QUERY_FULL_SETUP) + \
        float(nc[~full].sum()) * OPS_PER_CENTRE


def eikonal_algorithmic_ops(q: np.ndarray, R: int) -> float:
    """Exact algorithmic FP32 operations of one fused fit launch with the
    Eikonal term: the plain fit's count plus the second-order terms of every
    (query, centre) pair."""
    return algorithmic_ops(q, R) + float(centres_per_query(q, R).sum()) * EIK_EXTRA_PER_CENTRE


def variant_ops_per_key(deg: int, learn: int, offset: bool) -> int:
    """Algorithmic FP32 operations of one (query, key) pair of a variant's
    fused fit: forward (squared distance 6, exponent 1, monomials, polynomial
    nv - 1, sums 2) plus backward (distance 6, exponent 1, upstream 1,
    monomials, nv accumulations; the value f, f - O and the log-scale term
    when the scale is learnt or the key moves; 3 offset terms and, for degree
    >= 2, the polynomial's gradient and its 3 accumulations for offset keys).
    Degree 1 with both key sets reproduces the default model's 12 + 18 / 21."""
    nv = [1, 4, 10, 20][deg]
    mono = [0, 0, 6, 16][deg]
    fwd = 6 + 1 + mono + (nv - 1) + 2
    bwd = 6 + 1 + 1 + mono + nv
    if learn or offset:
        bwd += (nv - 1) + 3
    if offset:
        bwd += 3 + ([0, 0, 9, 30][deg] + 3 if deg >= 2 else 0)
    return fwd + bwd


def variant_algorithmic_ops(q: np.ndarray, R: int, sets: int, deg: int, learn: int) -> float:
    per_centre = sum(variant_ops_per_key(deg, learn, s == 2) for s in (1, 2) if sets & s)
    return float(centres_per_query(q, R).sum()) * per_centre


def centres_per_query(q: np.ndarray, R: int) -> np.ndarray:
    """Window size (number of centres) of every query, from the FP32 window rule."""
    u = (q[:, :3] + np.float32(1)) * np.float32(R * 0.5) - np.float32(0.5)
    c = np.floor(np.clip(u, np.float32(-1), np.float32(R - 1))).astype(np.int64)
    n = np.minimum(c + 2, R - 1) - np.maximum(c - 1, 0) + 1
    return n.prod(axis=1)


class ClockSampler:
    """nvidia-smi samples of one GPU while the timed region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            time.sleep(0.3)
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        rows = []
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                rows.append((float(parts[0]), float(parts[1]), parts[4:8]))
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = np.array([r[0] for r in rows])
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i, v in enumerate(r[2]) if v.lower().startswith("active")})
        load = sm[sm >= 0.5 * sm.max()] if sm.max() > 0 else sm
        return {"sm_mhz": float(np.median(load)), "sm_max_mhz": float(rows[0][1]), "reasons": reasons,
                "samples": len(rows)}


# ------------------------------------------------------------ CPU baseline

def _oracle_chunk(args):
    params, qo, R, lb = args
    import oracle
    O, _ = oracle.forward(params, qo, R, 2, lb)
    gO, L, mae = oracle.loss_grad(O, qo[:, 3], oracle.L1)
    gO *= len(O)   # the chunk's share of dL/dO; rescaled by the caller
    grad = oracle.backward(params, qo, gO, R, 2, lb)
    return grad, float(np.abs(O - qo[:, 3]).sum())


def oracle_step(pool, params, qo, R, lb, cores):
    """Oracle fit step on qo: forward, L1 gradient, backward (split over the
    pool's processes), Adam on the full grid."""
    import oracle
    chunks = np.array_split(qo.astype(np.float64), cores)
    res = pool.map(_oracle_chunk, [(params, c, R, lb) for c in chunks if len(c)])
    grad = sum(r[0] for r in res) / len(qo)
    return grad


def cpu_baseline(qo: np.ndarray, R: int, lb: float, seconds: float = 12.0):
    import oracle
    oracle.build()
    cores = os.cpu_count() or 1
    ctx = mp.get_context("spawn")
    params = __import__("paper_2505_21319_gb300.synth", fromlist=["synth"]).init_params(R, 0).astype(np.float64)
    m = np.zeros_like(params)
    v = np.zeros_like(params)
    with ctx.Pool(cores) as pool:
        n = 512 * cores
        t0 = time.perf_counter()
        oracle_step(pool, params, qo[:n], R, lb, cores)
        dt = time.perf_counter() - t0
        n = int(min(len(qo), max(n, n * seconds / max(dt, 1e-3))))
        t0 = time.perf_counter()
        grad = oracle_step(pool, params, qo[:n], R, lb, cores)
        oracle.adam(params, grad, m, v, 1, lr=LR)
        dt = time.perf_counter() - t0
    # the same step single-threaded, on a sample of about two seconds
    n1 = int(min(len(qo), max(256, (n / dt) / cores * 2.0)))
    t0 = time.perf_counter()
    O, _ = oracle.forward(params, qo[:n1], R, 2, lb)
    gO, _, _ = oracle.loss_grad(O, qo[:n1, 3].astype(np.float64), oracle.L1)
    grad1 = oracle.backward(params, qo[:n1], gO, R, 2, lb)
    oracle.adam(params, grad1, m, v, 2, lr=LR)
    dt1 = time.perf_counter() - t0
    return {"value": n / dt, "unit": "query-pts/s", "cores": cores, "kind": "oracle",
            "sample": f"one fit step (forward, L1 gradient, backward, Adam) on the first {n} queries of the "
                      f"2^22 batch at 32^3, FP64, {cores} spawn processes",
            "single_thread": {"value": n1 / dt1, "unit": "query-pts/s", "sample": f"the first {n1} queries"}}


# ------------------------------------------------------------------ main

def make_pool(R, J, n_batches, rank):
    from paper_2505_21319_gb300 import synth
    shape = synth.random_union(0)
    return np.concatenate([synth.sample_batch(shape, J, seed=1000 * rank + b) for b in range(n_batches)])


def run_reference(args, ws, rank):
    if rank != 0:
        return 0
    import oracle
    from paper_2505_21319_gb300 import synth
    oracle.build()
    R = R_DEFAULT
    lb = float(np.float32(oracle.default_log_beta0(R)))
    cores = os.cpu_count() or 1
    ctx = mp.get_context("spawn")
    params = synth.init_params(R, 0).astype(np.float64)
    m = np.zeros_like(params)
    v = np.zeros_like(params)
    qo = synth.sample_batch(synth.random_union(0), 1 << 18, seed=0)
    budget = float(args.reference_seconds)   # seconds for warm-up + timed steps
    with ctx.Pool(cores) as pool:
        n = 256 * cores
        t0 = time.perf_counter()
        oracle_step(pool, params, qo[:n], R, lb, cores)
        per_q = (time.perf_counter() - t0) / n
        S = int(max(64, min(len(qo), budget / max(1, args.steps + args.warmup) / per_q)))
        step = 0
        for _ in range(args.warmup):
            step += 1
            g = oracle_step(pool, params, qo[(step * S) % (len(qo) - S):][:S], R, lb, cores)
            params, m, v = oracle.adam(params, g, m, v, step, lr=LR)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            step += 1
            g = oracle_step(pool, params, qo[(step * S) % (len(qo) - S):][:S], R, lb, cores)
            params, m, v = oracle.adam(params, g, m, v, step, lr=LR)
        dt = time.perf_counter() - t0
    value = S * args.steps / dt
    sample = f"{S} queries of the 32^3 workload per step (bounded sample), FP64 oracle over {cores} processes"
    print(json.dumps({
        "impl": "reference", "metric": "fwd+bwd query-pts/s @32^3x13", "value": value, "unit": "query-pts/s",
        "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD + " (oracle on a bounded sample per step)", "R": R, "J_per_step": S},
        "cpu_baseline": {"value": value, "unit": "query-pts/s", "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "query-pts/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)
    return 0


def algorithmic_ops_torch(q, R: int) -> float:
    """algorithmic_ops for a device tensor of rows (the same FP32 window rule)."""
    import torch
    u = (q[:, :3] + 1.0) * (R * 0.5) - 0.5
    c = torch.floor(torch.clamp(u, -1.0, float(R - 1))).to(torch.int64)
    n = (torch.clamp(c + 2, max=R - 1) - torch.clamp(c - 1, min=0) + 1).prod(dim=1)
    full = n == 64
    return float(full.sum().item()) * (64 * OPS_PER_CENTRE_FULL + OPS_PER_QUERY_FULL_SETUP) + \
        float(n[~full].sum().item()) * OPS_PER_CENTRE


def bench_batched(api, dev, stream, rank, steps, peak, ws=1):
    """Many shapes fitted together (efunc_fit_batched): 256 unions of 4-16
    random primitives, grid resolution drawn from {16, 32, 64}, queries per
    shape log-uniform in [2^14, 2^20]; two batches per shape drawn on the
    device; the launch configuration chosen by efunc_tune_batched; the
    steps replayed from a CUDA graph (one period = two steps)."""
    import torch
    from paper_2505_21319_gb300 import synth
    g = synth.rng(7000 + rank)
    S = BATCH_SHAPES
    Rs = [int(x) for x in g.choice([16, 32, 64], size=S)]
    Js = [int(round(2.0 ** x)) for x in g.uniform(14.0, 20.0, size=S)]
    prims = [int(x) for x in g.integers(4, 17, size=S)]
    t0 = time.perf_counter()
    shapes = [synth.random_union(8000 + 1000 * rank + s, n_prims=prims[s]) for s in range(S)]
    b = api.Batch(Rs, Js, device=dev)
    qo = torch.cat([synth.sample_batch_torch(shapes[s], Js[s], seed=(rank * 2 + k) * 100003 + s, device=dev)
                    for k in range(2) for s in range(S)])
    params = torch.cat([torch.from_numpy(synth.init_params(R, seed=s).reshape(-1)) for s, R in enumerate(Rs)]).to(dev)
    m, v = torch.zeros_like(params), torch.zeros_like(params)
    torch.cuda.synchronize(dev)
    gen_s = time.perf_counter() - t0
    # default configuration, a few steps issued one by one
    d0, d1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    b.fit(params, m, v, qo, steps=2, n_batches=2, lr=LR, graph=False)
    d0.record(stream)
    b.fit(params, m, v, qo, steps=4, n_batches=2, lr=LR, graph=False)
    d1.record(stream)
    torch.cuda.synchronize(dev)
    default_ms = d0.elapsed_time(d1) / 4
    tuning, tuned_ms = b.tune(params, m, v, qo, n_batches=2, trial_steps=3)
    params = torch.cat([torch.from_numpy(synth.init_params(R, seed=s).reshape(-1)) for s, R in enumerate(Rs)]).to(dev)
    # the fused kernel's launch time (profiled steps issued one by one)
    b.fit(params, m, v, qo, steps=3, n_batches=2, lr=LR, graph=False)
    torch.cuda.synchronize(dev)
    api.profile_reset()
    api.profile(True)
    b.fit(params, m, v, qo, steps=4, n_batches=2, step0=3, lr=LR, graph=False)
    torch.cuda.synchronize(dev)
    api.profile(False)
    fk_ms, fk_n = api.profile_read("batched")
    fk = fk_ms / max(1, fk_n)
    # timed: the whole graph-replayed loop
    params = torch.cat([torch.from_numpy(synth.init_params(R, seed=s).reshape(-1)) for s, R in enumerate(Rs)]).to(dev)
    m.zero_()
    v.zero_()
    stats = torch.zeros(steps * S * 2, device=dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    e0.record(stream)
    b.fit(params, m, v, qo, steps=steps, n_batches=2, stats=stats, lr=LR, graph=True)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms = max_over_ranks(e0.elapsed_time(e1) / steps, dev)
    st = stats.view(steps, S, 2)
    ops = 0.0
    for k in range(2):
        for s in range(S):
            lo = k * b.n_queries + b.query_offsets[s]
            ops += algorithmic_ops_torch(qo[lo:lo + Js[s]], Rs[s])
    ops /= 2
    ach = ops / (fk * 1e-3) / 1e12
    return {"shapes": S, "grids": {str(R): Rs.count(R) for R in (16, 32, 64)}, "queries_per_step": b.n_queries,
            "params": b.n_params, "steps": steps, "ms_per_step": ms,
            "value": b.n_queries * ws / (ms * 1e-3), "unit": "query-pts/s",
            "fits_per_s": S * ws / (steps * ms * 1e-3), "fits_unit": f"shapes per second ({steps}-step fits)",
            "tuning": tuning, "tuned_ms_per_step": tuned_ms, "default_ms_per_step": default_ms,
            "fused_ms": fk, "ops_per_launch": ops, "achieved": ach, "peak": peak, "unit_roofline": "T FP32 op/s",
            "frac": ach / peak,
            "mae_first": float(st[0, :, 1].mean()), "mae_last": float(st[-1, :, 1].mean()),
            "generation_s": gen_s, "graph": "one period of 2 steps captured, replayed",
            "timing": "CUDA events around the whole efunc_fit_batched call (capture and instantiation included)"}


def bench_warm_start(dev, rank, n_train, n_eval, train_steps, epochs, eval_steps, ws=1):
    """The learned warm start against the plain initialisation: plain batched
    fits of n_train random shapes (32^3, 2^16 queries per step, train_steps
    steps) give the encoder's training pairs; the encoder is trained for
    `epochs`; n_eval held-out shapes are then fitted (32^3, 2^17 queries per
    step) from the N(0, 1e-3) initialisation and from the encoder's
    prediction, the held-out MAE of every shape (2^15 points, half uniform,
    half near the surface) tracked every 25 steps.  A shape's target is MAE
    1e-3, or the plain fit's final MAE where the plain fit does not reach
    1e-3; each arm reports the steps and seconds until its shapes reach their
    targets (the warm arm's seconds include the encoder's prediction)."""
    import torch
    from paper_2505_21319_gb300 import synth
    from paper_2505_21319_gb300 import warmstart as W
    t0 = time.perf_counter()
    train = W.random_shapes(200000 + 10000 * rank, n_train)
    tp, fit_s = W.fit_plain(train, J=1 << 16, steps=train_steps, seed=11, device=dev)
    sdf = W.sdf_grids(train, dev)
    w, losses, enc_s = W.train_encoder(sdf, tp, epochs=epochs, batch=WARM_BATCH, lr=1e-3, seed=rank)
    # the tensor-core convolutions of a training step against the bf16 peak:
    # algorithmic flops (real channel counts; the kernels pad L2's 32 input
    # channels to 64) over their CUDA-event time
    from paper_2505_21319_gb300 import api
    enc = api.Encoder(WARM_BATCH, dev)
    idx = torch.arange(WARM_BATCH, device=dev)
    sd, tg = sdf[idx].contiguous(), tp[idx].contiguous()
    for _ in range(3):
        enc.train_step(w, sd, tg)
    torch.cuda.synchronize(dev)
    api.profile_reset()
    api.profile(True)
    for _ in range(ENC_PROFILE_STEPS):
        enc.train_step(w, sd, tg)
    torch.cuda.synchronize(dev)
    api.profile(False)
    conv_ms = sum(api.profile_read(k)[0] for k in ("enc_conv", "enc_wgrad")) / ENC_PROFILE_STEPS
    aux_ms = api.profile_read("enc_aux")[0] / ENC_PROFILE_STEPS
    V = WARM_BATCH * 32 ** 3
    flops = 2.0 * V * ENC_MACS_PER_VOXEL
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        bf16_peak, peak_from = float(peaks["bf16_tflops"]), "measured cuBLAS bf16 burst (MEASURED_PEAKS.json)"
    except (OSError, ValueError, KeyError):
        bf16_peak, peak_from = 1900.0, "fallback 1.9 PFLOP/s bf16"
    enc_roof = {"bound": "tensor", "achieved": flops / (conv_ms * 1e-3) / 1e12, "peak": bf16_peak,
                "unit": "TFLOP/s", "frac": flops / (conv_ms * 1e-3) / 1e12 / bf16_peak, "peak_from": peak_from,
                "flops_per_step": flops, "tc_ms_per_step": conv_ms, "other_ms_per_step": aux_ms,
                "batch": WARM_BATCH, "kernels": "conv_fwd_kernel (forward, dgrad) + conv_wgrad_kernel"}
    ev = W.random_shapes(300000 + 10000 * rank, n_eval)
    held = W.heldout_rows(ev, 1 << 15, seed=99, device=dev)
    pred, pred_s = W.predict(w, W.sdf_grids(ev, dev), batch=WARM_BATCH)
    init = torch.cat([torch.from_numpy(synth.init_params(W.R, seed=i).reshape(1, -1)) for i in range(n_eval)]).to(dev)
    arms = {}
    for name, p0 in (("plain", init), ("warm", pred)):
        st, mae, sec = W.fit_curves(ev, p0, J=1 << 17, max_steps=eval_steps, every=25, seed=5, held=held)
        arms[name] = (st, mae, sec)
    st_p, mae_p, _ = arms["plain"]
    target = np.where(mae_p.min(0) <= 1e-3, 1e-3, mae_p[-1])
    out = {"train_shapes": n_train, "train_fit_steps": train_steps, "train_fit_s": fit_s, "encoder_epochs": epochs,
           "encoder_train_s": enc_s, "encoder_loss_first": losses[0], "encoder_loss_last": losses[-1],
           "eval_shapes": n_eval, "eval_steps": eval_steps, "predict_s": pred_s,
           "target_rule": "per shape: 1e-3, or the plain fit's final held-out MAE where 1e-3 is not reached",
           "shapes_reaching_1e-3_plain": int((mae_p.min(0) <= 1e-3).sum()), "encoder_roofline": enc_roof}
    def finite(x):
        return float(x) if np.isfinite(x) else None   # JSON has no inf / nan

    for name, (st, mae, sec) in arms.items():
        steps = W.steps_to(st, mae, target)
        reached = np.isfinite(steps)
        sec_per_step = float(sec[-1] / st[-1])
        extra = pred_s if name == "warm" else 0.0
        # steps until half / 90 % / all of the shapes reached their targets
        # (inf where that many never did within eval_steps)
        q = {k: float(np.quantile(steps, f, method="higher")) for k, f in (("p50", 0.5), ("p90", 0.9), ("all", 1.0))}
        out[name] = {"mae_median_start": float(np.median(mae[0])), "mae_median_final": float(np.median(mae[-1])),
                     "mae_median_at_step": {str(int(s_)): float(np.median(mae[i])) for i, s_ in enumerate(st)
                                            if int(s_) in (100, 250, 500, 1000, 1500)},
                     "shapes_reached": int(reached.sum()), "steps_to_target": {k: finite(v) for k, v in q.items()},
                     "seconds_per_step": sec_per_step,
                     "wall_s_to_target": {k: finite(v * sec_per_step + extra) for k, v in q.items()},
                     "fits_per_s_half": (0.5 * n_eval * ws / (q["p50"] * sec_per_step + extra))
                     if np.isfinite(q["p50"]) else None}
    sp, sw = out["plain"]["steps_to_target"]["p50"], out["warm"]["steps_to_target"]["p50"]
    out["median_step_ratio"] = sp / sw if sp and sw else None
    out["fits_per_s_note"] = "fits_per_s_half: half of the shapes at their targets over the seconds that took"
    out["total_s"] = time.perf_counter() - t0
    return out


def fit_to_target(api, dev, stream, R, J, pool, held, rank, max_steps, chunk, target, ws=1, params0=None):
    """A plain fit from the N(0, 1e-3) initialisation (or params0) in chunks of
    ``chunk`` steps, the held-out MAE (volume, near-surface, and the two
    together) after every chunk.  Returns the MAE curve, the first step count
    at which the joint held-out MAE is <= target (if any), the fit's own
    CUDA-event seconds up to there, and fits/s = 1 / those seconds."""
    import torch
    from paper_2505_21319_gb300 import synth
    p = params0.clone() if params0 is not None else torch.from_numpy(synth.init_params(R, seed=rank)).to(dev)
    m, v = torch.zeros_like(p), torch.zeros_like(p)
    wsb = api.Workspace(dev)
    nb = pool.shape[0] // J

    def heldout():
        outs = {k: api.efunc_eval_loss(p, q, ws=wsb) for k, q in held.items()}
        mae = {k: float(o[1]) for k, o in outs.items()}
        mae["all"] = (mae["volume"] + mae["near"]) / 2.0   # equal halves
        return mae

    curve = [{"step": 0, "seconds": 0.0, **heldout()}]
    secs, step, reached = 0.0, 0, None
    while step < max_steps:
        n = min(chunk, max_steps - step)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(dev)
        e0.record(stream)
        api.efunc_fit(p, m, v, pool, steps=n, J=J, n_batches=nb, step0=step, lr=LR, ws=wsb)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        secs += e0.elapsed_time(e1) * 1e-3
        step += n
        mae = heldout()
        curve.append({"step": step, "seconds": secs, **mae})
        if reached is None and mae["all"] <= target:
            reached = {"steps": step, "seconds": secs}
    final = curve[-1]
    tgt, how = target, f"held-out MAE <= {target:g}"
    if reached is None:   # the plain fit's final MAE stands in for the target
        tgt, how = final["all"], "the plain fit's final held-out MAE (1e-3 not reached)"
        reached = {"steps": final["step"], "seconds": final["seconds"]}
    out = {"R": R, "J_per_step": J, "target": tgt, "target_rule": how, "steps_to_target": reached["steps"],
           "seconds_to_target": reached["seconds"], "fits_per_s": ws / reached["seconds"],
           "final_mae": {k: final[k] for k in ("volume", "near", "all")}, "steps": final["step"],
           "seconds_per_step": final["seconds"] / max(1, final["step"]), "chunk": chunk,
           "heldout_points": {k: int(q.shape[0]) for k, q in held.items()}, "curve": curve,
           "timing": "CUDA events around each chunk's efunc_fit; held-out evaluation between chunks not timed"}
    out["summary"] = (f"MAE {final['all']:.3e} after {final['step']} steps (volume {final['volume']:.3e}, "
                      f"near {final['near']:.3e}); target {tgt:.3e} at step {reached['steps']}, "
                      f"{reached['seconds']:.3f} s")
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--e2e-steps", type=int, default=200)
    ap.add_argument("--eikonal-steps", type=int, default=100)
    ap.add_argument("--mean-shift-reps", type=int, default=20)
    ap.add_argument("--variant-steps", type=int, default=50)
    ap.add_argument("--cosine-steps", type=int, default=50)
    ap.add_argument("--isolated-steps", type=int, default=50)
    ap.add_argument("--graph-steps", type=int, default=500)
    ap.add_argument("--large-steps", type=int, default=20)
    ap.add_argument("--warm-train-shapes", type=int, default=512,
                    help="shapes fitted to train the warm-start encoder (0 skips the warm-start comparison)")
    ap.add_argument("--warm-eval-shapes", type=int, default=64)
    ap.add_argument("--warm-train-steps", type=int, default=800)
    ap.add_argument("--warm-epochs", type=int, default=30)
    ap.add_argument("--warm-eval-steps", type=int, default=1500)
    ap.add_argument("--batched-steps", type=int, default=300,
                    help="steps of the batched fit of 256 shapes (0 skips it)")
    ap.add_argument("--target-steps", type=int, default=2000,
                    help="steps of the plain fits to the MAE target (0 skips them)")
    ap.add_argument("--dense-reps", type=int, default=5,
                    help="efunc_forward calls over a 256^3 lattice of points (0 skips the dense query)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--reference-seconds", type=float, default=150.0,
                    help="--impl reference: seconds of oracle work over warm-up and timed steps")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be at least 3")
    ws, rank, local = dist_env()
    if args.impl == "reference":
        return run_reference(args, ws, rank)

    import torch
    import torch.distributed as dist
    from paper_2505_21319_gb300 import api

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if ws > 1:
        dist.init_process_group("nccl", device_id=dev)

    R, J = R_DEFAULT, J_DEFAULT
    lb = api.default_log_beta0(R)
    t0 = time.perf_counter()
    pool_np = make_pool(R, J, N_BATCHES, rank)
    log(f"[bench] rank {rank}: batch pool {pool_np.shape} generated in {time.perf_counter() - t0:.1f}s")
    cpu_line = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu_line = cpu_baseline(pool_np[:J], R, float(np.float32(lb)))
        log(f"[bench] cpu baseline {cpu_line['value']:.3e} q/s")

    from paper_2505_21319_gb300 import synth
    n = R ** 3 * 13
    pool = torch.from_numpy(pool_np).to(dev)
    params = torch.from_numpy(synth.init_params(R, seed=rank)).to(dev)
    m = torch.zeros(n, device=dev)
    v = torch.zeros(n, device=dev)
    ws_buf = api.Workspace(dev)
    stats_w = torch.zeros(2 * args.warmup, device=dev)
    stats = torch.zeros(2 * args.steps, device=dev)
    stream = torch.cuda.current_stream(dev)

    api.efunc_fit(params, m, v, pool, steps=args.warmup, J=J, n_batches=N_BATCHES, stats=stats_w, lr=LR,
                  ws=ws_buf)
    torch.cuda.synchronize(dev)

    # ---- timed region: K fit steps, device-resident inputs
    api.profile_reset()
    api.profile(True)
    launches0 = api.launch_count()
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        if ws > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)
        start.record(stream)
        api.efunc_fit(params, m, v, pool, steps=args.steps, J=J, n_batches=N_BATCHES, step0=args.warmup,
                      stats=stats, lr=LR, ws=ws_buf)
        end.record(stream)
        torch.cuda.synchronize(dev)
        if ws > 1:
            dist.barrier()
    launches = api.launch_count() - launches0
    api.profile(False)
    ms = start.elapsed_time(end) / args.steps
    fused_ms, fused_n = api.profile_read("fused_fit")
    kernel_ms = {k: api.profile_read(k)[0] / max(1, api.profile_read(k)[1])
                 for k in ("bin", "scan_reduce", "scan_top", "scan_emit", "scatter", "pack_keys", "fused_fit", "adam")}
    ms = max_over_ranks(ms, dev)
    value = J * ws / (ms * 1e-3)
    st = stats.view(-1, 2).cpu().numpy()

    # ---- roofline of the fused kernel (ALU bound)
    ops_per_launch = sum(algorithmic_ops(pool_np[b * J:(b + 1) * J], R) for b in range(N_BATCHES)) / N_BATCHES
    props = torch.cuda.get_device_properties(dev)
    sm_max = 2070.0
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        sm_max = float(peaks.get("sm_max_mhz", sm_max))
    except (OSError, ValueError):
        pass
    peak = props.multi_processor_count * FP32_LANES_PER_SM * sm_max * 1e6 / 1e12   # T FP32 ops/s
    avg_fused = fused_ms / max(1, fused_n)
    achieved = ops_per_launch / (avg_fused * 1e-3) / 1e12
    clocks = clk.summary()

    # ---- the fused kernel alone: the same fit with the sort in line (no
    # sort of the next batch beside it), for the kernel's own roofline
    iso = None
    if args.isolated_steps > 0:
        api.profile_reset()
        api.profile(True)
        api.efunc_fit(params, m, v, pool, steps=args.isolated_steps, J=J, n_batches=N_BATCHES, step0=4 * 10 ** 6,
                      lr=LR, ws=ws_buf, pipelined=False)
        torch.cuda.synchronize(dev)
        api.profile(False)
        im, icnt = api.profile_read("fused_fit")
        iavg = im / max(1, icnt)
        iach = ops_per_launch / (iavg * 1e-3) / 1e12
        iso = {"avg_launch_ms": iavg, "achieved": iach, "frac": iach / peak, "steps": args.isolated_steps,
               "note": "fused kernel of the same fit with the batch sorted in line: nothing runs beside it"}
        # the memory-bound kernels of the same in-line run against the measured copy bandwidth:
        # algorithmic bytes per launch (bin: query row read + rank written; scatter: row and
        # rank read, row written; adam: p, g, m, v read and p, m, v, g written)
        try:
            hbm = float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"])
            hbm_from = "measured copy bandwidth"
        except (OSError, ValueError, KeyError):
            hbm, hbm_from = 6800.0, "fallback"
        n_par = R ** 3 * 13
        for kname, nbytes in (("bin", J * 20), ("scatter", J * 36), ("adam", n_par * 32)):
            km, kc = api.profile_read(kname)
            kavg = km / max(1, kc)
            gbs = nbytes / (kavg * 1e-3) / 1e9
            iso.setdefault("memory_bound", {})[kname] = {
                "avg_launch_ms": kavg, "bytes": nbytes, "achieved": gbs, "peak": hbm, "unit": "GB/s",
                "frac": gbs / hbm, "peak_from": hbm_from}

    # ---- the same fit with the Eikonal term (NEXT-1: second-order fused
    # backward through dO/dq), timed the same way on a shorter run
    eik = None
    if args.eikonal_steps > 0:
        api.efunc_fit(params, m, v, pool, steps=3, J=J, n_batches=N_BATCHES, step0=5 * 10 ** 6, lr=LR, ws=ws_buf,
                      eikonal_weight=0.1)
        torch.cuda.synchronize(dev)
        api.profile_reset()
        api.profile(True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        api.efunc_fit(params, m, v, pool, steps=args.eikonal_steps, J=J, n_batches=N_BATCHES, step0=6 * 10 ** 6,
                      lr=LR, ws=ws_buf, eikonal_weight=0.1)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        api.profile(False)
        ems = max_over_ranks(e0.elapsed_time(e1) / args.eikonal_steps, dev)
        fm, fn = api.profile_read("fused_fit")
        eops = sum(eikonal_algorithmic_ops(pool_np[b * J:(b + 1) * J], R) for b in range(N_BATCHES)) / N_BATCHES
        eavg = fm / max(1, fn)
        each = eops / (eavg * 1e-3) / 1e12
        eik = {"value": J * ws / (ems * 1e-3), "unit": "query-pts/s", "ms_per_step": ems,
               "fused_ms": eavg, "achieved": each, "peak": peak, "unit_roofline": "T FP32 op/s",
               "frac": each / peak, "ops_per_launch": eops, "steps": args.eikonal_steps, "eikonal_weight": 0.1}

    # ---- the largest configuration, 64^3 x 13 with 2^24 queries per step
    # (one 256 MiB batch, larger than L2: the three 2^22 batches of the pool
    # and a fourth drawn the same way), same fit and roofline accounting
    large = None
    if args.large_steps > 0:
        RL, JL = 64, 1 << 24
        big_np = np.concatenate([pool_np, synth.sample_batch(synth.random_union(0), J, seed=1000 * rank + N_BATCHES)])
        assert big_np.shape[0] == JL
        big = torch.from_numpy(big_np).to(dev)
        lp = torch.from_numpy(synth.init_params(RL, seed=rank)).to(dev)
        lm, lv = torch.zeros_like(lp), torch.zeros_like(lp)
        lws = api.Workspace(dev)
        api.efunc_fit(lp, lm, lv, big, steps=3, J=JL, lr=LR, ws=lws)
        torch.cuda.synchronize(dev)
        api.profile_reset()
        api.profile(True)
        l0, l1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        if ws > 1:
            dist.barrier()
        l0.record(stream)
        api.efunc_fit(lp, lm, lv, big, steps=args.large_steps, J=JL, step0=3, lr=LR, ws=lws)
        l1.record(stream)
        torch.cuda.synchronize(dev)
        api.profile(False)
        lms = max_over_ranks(l0.elapsed_time(l1) / args.large_steps, dev)
        fm, fn = api.profile_read("fused_fit")
        lavg = fm / max(1, fn)
        lops = algorithmic_ops(big_np, RL)
        lach = lops / (lavg * 1e-3) / 1e12
        large = {"R": RL, "J_per_step": JL, "value": JL * ws / (lms * 1e-3), "unit": "query-pts/s",
                 "ms_per_step": lms, "fused_ms": lavg, "achieved": lach, "peak": peak,
                 "unit_roofline": "T FP32 op/s", "frac": lach / peak, "ops_per_launch": lops,
                 "steps": args.large_steps, "l2": "one 256 MiB batch, larger than L2"}
        del big, big_np, lp, lm, lv, lws

    # ---- mean-shift offset initialisation (Sec. 3.3): R^3 centres x 16384
    # surface points, 13 FP32-pipe operations and one ex2 per pair
    ms_init = None
    if args.mean_shift_reps > 0:
        n_pts = 16384
        pts = torch.from_numpy(synth.surface_points(synth.random_union(0), n_pts, synth.rng(77))
                               .astype(np.float32)).to(dev)
        scratch = params.clone()
        for _ in range(3):
            api.efunc_mean_shift_init(scratch, pts)
        torch.cuda.synchronize(dev)
        api.profile_reset()
        api.profile(True)
        for _ in range(args.mean_shift_reps):
            api.efunc_mean_shift_init(scratch, pts)
        torch.cuda.synchronize(dev)
        api.profile(False)
        mt, mn = api.profile_read("mean_shift")
        mms = mt / max(1, mn)
        pairs = R ** 3 * n_pts
        ms_ach = pairs * MEAN_SHIFT_OPS_PER_PAIR / (mms * 1e-3) / 1e12
        ms_init = {"ms": mms, "pairs_per_s": pairs / (mms * 1e-3), "R": R, "points": n_pts, "bandwidth": 100.0,
                   "achieved": ms_ach, "peak": peak, "unit": "T FP32 op/s", "frac": ms_ach / peak,
                   "ops_per_pair": MEAN_SHIFT_OPS_PER_PAIR}
        del scratch, pts

    # ---- dense query (inference): efunc_forward over a 256^3 lattice of points
    # filling the domain, on the fitted grid (sort, key pack, forward, outputs
    # in the lattice's order).  The paper's timing discussion after Table
    # tab:memory_time quotes about 5 s for such a 256^3 query with global
    # support on unstated hardware: context, not a comparable figure.
    dense = None
    if args.dense_reps > 0:
        n_ax = 256
        ax = (torch.arange(n_ax, device=dev, dtype=torch.float32) + 0.5) * (2.0 / n_ax) - 1.0
        lat = torch.stack(torch.meshgrid(ax, ax, ax, indexing="ij"), dim=-1).reshape(-1, 3).contiguous()
        api.efunc_forward(params, lat)
        torch.cuda.synchronize(dev)
        d0 = torch.cuda.Event(enable_timing=True)
        d1 = torch.cuda.Event(enable_timing=True)
        d0.record(stream)
        for _ in range(args.dense_reps):
            api.efunc_forward(params, lat)
        d1.record(stream)
        torch.cuda.synchronize(dev)
        dms = d0.elapsed_time(d1) / args.dense_reps
        dense = {"points": int(lat.shape[0]), "R": R, "ms": dms, "pts_per_s": lat.shape[0] / (dms * 1e-3),
                 "timing": "CUDA events around efunc_forward calls (sort, key pack, forward, outputs in lattice order)",
                 "paper": "about 5 s for a 256^3 dense query with global support, hardware not stated (context)"}
        del lat

    # ---- ablation variants of Table tab:ablation: the same fit (sort, pack,
    # fused forward + L1 + backward, Adam) with each configuration's layout
    variants = None
    if args.variant_steps > 0:
        variants = {}
        for name in ("G-6", "G-7", "G-8", "Full-1"):
            var = api.VARIANTS[name]
            ch = api.variant_channels(name)
            vp = torch.from_numpy((synth.rng(rank).standard_normal(R ** 3 * ch) * 1e-3).astype(np.float32)).to(dev)
            vm, vv = torch.zeros_like(vp), torch.zeros_like(vp)
            vws = api.VariantWorkspace(dev)
            api.efunc_variant_fit(name, vp, vm, vv, pool, steps=3, J=J, n_batches=N_BATCHES, lr=LR, ws=vws)
            torch.cuda.synchronize(dev)
            api.profile_reset()
            api.profile(True)
            v0, v1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            v0.record(stream)
            api.efunc_variant_fit(name, vp, vm, vv, pool, steps=args.variant_steps, J=J, n_batches=N_BATCHES,
                                  step0=3, lr=LR, ws=vws)
            v1.record(stream)
            torch.cuda.synchronize(dev)
            api.profile(False)
            vms = max_over_ranks(v0.elapsed_time(v1) / args.variant_steps, dev)
            fm, fn = api.profile_read("variant_fit")
            kms = fm / max(1, fn)
            vops = sum(variant_algorithmic_ops(pool_np[b * J:(b + 1) * J], R, *var) for b in range(N_BATCHES)) / N_BATCHES
            vach = vops / (kms * 1e-3) / 1e12
            variants[name] = {"variant": list(var), "channels": ch, "value": J * ws / (vms * 1e-3),
                              "unit": "query-pts/s", "ms_per_step": vms, "fit_kernel_ms": kms,
                              "achieved": vach, "peak": peak, "unit_roofline": "T FP32 op/s", "frac": vach / peak,
                              "ops_per_launch": vops, "steps": args.variant_steps}
            del vp, vm, vv, vws

    # ---- cosine-series decomposition (Sec. 4.4): B bands of 16^3 Config-G-6
    # grids, the paper's resolution, fitted on the same batches
    cosine = None
    if args.cosine_steps > 0:
        cosine = {}
        Rc = 16
        for Bc in (1, 4, 8):
            cp = torch.from_numpy((synth.rng(rank).standard_normal(Bc * Rc ** 3 * 5) * 1e-3).astype(np.float32)).to(dev)
            cm, cv = torch.zeros_like(cp), torch.zeros_like(cp)
            cws = api.CosineWorkspace(dev)
            api.efunc_cosine_fit(Bc, cp, cm, cv, pool, steps=3, J=J, n_batches=N_BATCHES, lr=LR, ws=cws)
            torch.cuda.synchronize(dev)
            api.profile_reset()
            api.profile(True)
            c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            c0.record(stream)
            api.efunc_cosine_fit(Bc, cp, cm, cv, pool, steps=args.cosine_steps, J=J, n_batches=N_BATCHES, step0=3,
                                 lr=LR, ws=cws)
            c1.record(stream)
            torch.cuda.synchronize(dev)
            api.profile(False)
            cms = max_over_ranks(c0.elapsed_time(c1) / args.cosine_steps, dev)
            fm, fn = api.profile_read("cosine_fit")
            kms = fm / max(1, fn)
            cops = Bc * sum(variant_algorithmic_ops(pool_np[b * J:(b + 1) * J], Rc, 1, 1, 1)
                            for b in range(N_BATCHES)) / N_BATCHES
            cach = cops / (kms * 1e-3) / 1e12
            cosine[f"B={Bc}"] = {"bands": Bc, "R": Rc, "value": J * ws / (cms * 1e-3), "unit": "query-pts/s",
                                 "ms_per_step": cms, "fit_kernel_ms": kms, "achieved": cach, "peak": peak,
                                 "unit_roofline": "T FP32 op/s", "frac": cach / peak, "ops_per_launch": cops,
                                 "steps": args.cosine_steps}
            del cp, cm, cv, cws

    # ---- the fit replayed from a CUDA graph (efunc_fit_graph): the same
    # 32^3 x 2^22 workload, and the small 16^3 x 65,536-query configuration
    # (1 MiB batches, L2-resident) whose steps are shorter than the host's
    # time to launch them one by one; the stream-issued fit beside it
    graph_fit = None
    if args.graph_steps > 0:
        def timed_fit(p_, m_, v_, pool_, Jg, steps, step0, graph, wsp):
            g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            if ws > 1:
                dist.barrier()
            torch.cuda.synchronize(dev)
            g0.record(stream)
            api.efunc_fit(p_, m_, v_, pool_, steps=steps, J=Jg, n_batches=N_BATCHES, step0=step0, lr=LR, ws=wsp,
                          graph=graph)
            g1.record(stream)
            torch.cuda.synchronize(dev)
            return max_over_ranks(g0.elapsed_time(g1) / steps, dev)

        api.efunc_fit(params, m, v, pool, steps=3, J=J, n_batches=N_BATCHES, step0=7 * 10 ** 6, lr=LR, ws=ws_buf,
                      graph=True)
        gms = timed_fit(params, m, v, pool, J, args.graph_steps, 8 * 10 ** 6, True, ws_buf)
        Rs, Js = 16, 65536
        small = torch.from_numpy(make_pool(Rs, Js, N_BATCHES, rank)).to(dev)
        sp = torch.from_numpy(synth.init_params(Rs, seed=rank)).to(dev)
        sm_, sv_ = torch.zeros_like(sp), torch.zeros_like(sp)
        sws = api.Workspace(dev)
        small_ms = {}
        for graph in (False, True):
            api.efunc_fit(sp, sm_, sv_, small, steps=6, J=Js, n_batches=N_BATCHES, lr=LR, ws=sws, graph=graph)
            small_ms[graph] = timed_fit(sp, sm_, sv_, small, Js, 4 * args.graph_steps, 100, graph, sws)
        graph_fit = {
            "32^3 x 2^22": {"value": J * ws / (gms * 1e-3), "unit": "query-pts/s", "ms_per_step": gms,
                            "stream_ms_per_step": ms, "steps": args.graph_steps},
            "16^3 x 65536": {"value": Js * ws / (small_ms[True] * 1e-3), "unit": "query-pts/s",
                             "fits_per_s": 1e3 / (FIT_STEPS_16 * small_ms[True]) * ws, "steps_per_fit": FIT_STEPS_16,
                             "ms_per_step": small_ms[True], "stream_value": Js * ws / (small_ms[False] * 1e-3),
                             "stream_ms_per_step": small_ms[False], "steps": 4 * args.graph_steps,
                             "l2": "1 MiB batches: L2-resident"},
            "note": "CUDA events around the whole call: graph capture and instantiation included"}
        del small, sp, sm_, sv_, sws

    # ---- plain fits to an MAE target (the plain half of the metric): the
    # fit runs in chunks of steps (CUDA events around each chunk's
    # efunc_fit); between chunks efunc_eval_loss evaluates the held-out MAE
    # on the device (not timed): 2^19 uniform + 2^19 near-surface points
    # drawn apart from the training pool, the paper's volume / near-surface
    # split of its AE metrics (Sec. 4.1)
    to_target = None
    if args.target_steps > 0:
        to_target = {}
        for cname, (Rt, Jt, shape_t, seed_t) in (("C2 32^3 union of 8", (R, J, synth.random_union(0), 0)),
                                                 ("C1 16^3 sphere", (16, 65536, synth.sphere(0.5), 1))):
            if Rt == R and Jt == J:
                pool_t = pool
            else:
                pool_t = torch.from_numpy(np.concatenate([synth.sample_batch(shape_t, Jt, seed=500 + b)
                                                          for b in range(N_BATCHES)])).to(dev)
            held = {k: torch.from_numpy(synth.sample_batch(shape_t, HELDOUT // 2, seed=900 + seed_t, near_frac=f))
                    .to(dev) for k, f in (("volume", 0.0), ("near", 1.0))}
            to_target[cname] = fit_to_target(api, dev, stream, Rt, Jt, pool_t, held, rank, args.target_steps,
                                             TARGET_CHUNK, TARGET_MAE, ws)
            log(f"[bench] {cname}: {to_target[cname]['summary']}")
            del pool_t, held

    # ---- batched fit of many shapes of uneven size (efunc_fit_batched)
    batched = None
    if args.batched_steps > 0:
        batched = bench_batched(api, dev, stream, rank, args.batched_steps, peak, ws)
        log(f"[bench] batched: {batched['ms_per_step']:.3f} ms/step, {batched['value']:.3e} q/s, "
            f"frac {batched['frac']:.3f}, tuning {batched['tuning']}")

    # ---- learned warm start (encoder) against the plain initialisation
    warm = None
    if args.warm_train_shapes > 0:
        warm = bench_warm_start(dev, rank, args.warm_train_shapes, args.warm_eval_shapes, args.warm_train_steps,
                                args.warm_epochs, args.warm_eval_steps, ws)
        log(f"[bench] warm start: plain {warm['plain']['steps_to_target']['p50']} / warm "
            f"{warm['warm']['steps_to_target']['p50']} median steps to target, {warm['total_s']:.0f} s")

    # ---- end to end through the C ABI with host buffers: the batch pool in
    # pinned host memory, every step copies its 64 MiB batch to the device
    # (overlapped with the previous step's compute by the library) and copies
    # its (loss, MAE) pair back to pinned host memory
    e2e = None
    if args.e2e_steps > 0:
        host_pool = torch.from_numpy(pool_np).pin_memory()
        host_stats = torch.zeros(2 * args.e2e_steps, dtype=torch.float32).pin_memory()
        api.efunc_fit(params, m, v, host_pool, steps=3, J=J, n_batches=N_BATCHES, step0=10 ** 6,
                      stats=host_stats, lr=LR, ws=ws_buf)
        torch.cuda.synchronize(dev)
        if ws > 1:
            dist.barrier()
        t0 = time.perf_counter()
        api.efunc_fit(params, m, v, host_pool, steps=args.e2e_steps, J=J, n_batches=N_BATCHES, step0=2 * 10 ** 6,
                      stats=host_stats, lr=LR, ws=ws_buf)   # returns after the last statistics reached the host
        dt = time.perf_counter() - t0
        dt = max_over_ranks(dt, dev)
        e2e = {"value": J * ws * args.e2e_steps / dt, "unit": "query-pts/s", "h2d_bytes_per_step": J * 16,
               "d2h_bytes_per_step": 8, "steps": args.e2e_steps}

    if rank == 0:
        line = {
            "metric": "fwd+bwd query-pts/s @32^3x13",
            "value": value,
            "unit": "query-pts/s",
            "n_gpus": ws,
            "steps": args.steps,
            "warmup": args.warmup,
            "ms_per_step": ms,
            "higher_is_better": True,
            "scaling": "weak",
            "vs_baseline": None,
            "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "R": R, "J_per_step": J, "batches": N_BATCHES,
                       "l2": "inputs larger than L2: 3 batches x 64 MiB cycle, 192 MiB > 129 MB",
                       "parallelism": "replicas" if ws > 1 else "single GPU"},
            "roofline": {"bound": "alu", "kernel": "fused_fit", "achieved": achieved, "peak": peak,
                         "unit": "T FP32 op/s", "frac": achieved / peak, "traffic": fused_traffic(),
                         "ops_per_launch": ops_per_launch, "avg_launch_ms": avg_fused,
                         "peak_from": f"{props.multi_processor_count} SMs x 128 FP32 lanes x {sm_max:.0f} MHz",
                         "co_running": "the sort of the next batch runs beside the fused kernel (pipelined fit)",
                         "isolated": iso},
            "kernel_ms": kernel_ms,
            "e2e": e2e,
            "eikonal_fit": eik,
            "mean_shift_init": ms_init,
            "dense_query_256cubed": dense,
            "variants": variants,
            "cosine_series": cosine,
            "graph_fit": graph_fit,
            "fit_64cubed_2p24": large,
            "cpu_baseline": cpu_line,
            "clocks": clocks,
            "gpu_launches": launches,
            "fits_to_target": to_target,
            "batched_fit": batched,
            "warm_start": warm,
            "fit": {"steps_total": args.warmup + args.steps, "loss_first_timed": float(st[0, 0]),
                    "mae_first_timed": float(st[0, 1]), "mae_last": float(st[-1, 1]),
                    "fits_per_s": 1e3 / (FIT_STEPS_32 * ms) * ws, "steps_per_fit": FIT_STEPS_32},
        }
        print(json.dumps(json_safe(line), allow_nan=False), flush=True)
    if ws > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
