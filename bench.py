#!/usr/bin/env python3
"""Benchmark of the PageRank hot path on GB300 (one JSON line on stdout).

Default (``--workload headline``): the paper's sweeps as batched solves
against the plain per-instance GPU solver, the composite of three workloads
(synthetic, seeded; stand-ins for the paper's SuiteSparse graphs):

* ``sweep330`` — the 10k-vertex Erdos-Renyi graph (100,000 unique edges, 5 %
  dangling), alpha 0.50..1.00 step .05 x tau 1e-1..1e-10 x {L1, L2, Linf} =
  330 instances, max 500 iterations; learned start, precision chosen by the
  planner (Sections 2-4: the alpha sweep, the tau sweep, the norm comparison).
* ``multi64`` — 64 R-MAT graphs of scale 12 + (i mod 9), edge factor 16,
  alpha 0.85, tau 1e-10, L1, one batch.
* ``evalsweep`` — the learned start's evaluation graphs, unseen in training:
  R-MAT scale 22 (seed 3022) and 24 (seed 3024) and a directed configuration
  model with N = 8,000,000 (Zipf 2.1 in/out degrees, mean 12; seed 3008), each
  swept over alpha 0.50..0.95 x tau 1e-1..1e-10 x {L1, L2, Linf} (300
  instances per graph), learned start, planner-chosen precision.

A step solves the three workloads once each as batches (``pr_solve_batch``
through the binding's ``PreparedBatch``: each workload's instances are
marshalled once, before timing) with the graphs resident in HBM; ``value`` is
their instances per second. The
plain per-instance solver (every instance alone through ``pr_solve``, one
launch per iteration and a host read of the stop flag) is timed on the same
resident graphs; the per-workload ratios and their geometric mean (GM-RATIO,
Section 1) are reported with and without trajectory sharing. ``roofline`` is
the one-column gather kernel on R-MAT scale 22 (seed 22; alpha 0.85, tau
{1e-6, 1e-10} x {L1, L2, Linf}), measured in the same run. ``e2e`` repeats the
composite through the C ABI from pinned host arrays (graph creation, solve,
results to the host). ``cpu_baseline`` is the CPU oracle on a bounded sample,
on all host cores and on one.

Single workloads (``--workload rmat22`` and others below) keep the same line
for one workload. ``--impl reference`` times the CPU oracle instead.
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
from dataclasses import dataclass, field
from pathlib import Path

ROOT = Path(__file__).resolve().parent
sys.path.insert(0, str(ROOT))

METRIC = "sweep solves/s and GTEPS (%HBM roofline), batched+warm vs plain, ≤10τ/(1−α) L1 err"
HEADLINE = ("sweep330", "multi64", "evalsweep")
SINGLE = ("rmat22", "rmat21", "sweep330", "sweep330warm", "multi64", "rmat24mixed", "learned", "road24", "evalsweep")
ALPHAS_SWEEP = [round(0.5 + 0.05 * i, 2) for i in range(11)]      # 0.50 .. 1.00
ALPHAS_TRAIN = [round(0.5 + 0.05 * i, 2) for i in range(10)]      # 0.50 .. 0.95
TAUS_SWEEP = [10.0 ** -k for k in range(1, 11)]                    # 1e-1 .. 1e-10


def kernel_traffic_ratio():
    """DRAM traffic / algorithmic bytes of the gather kernel from the ncu
    capture summarised in profiles/, valid only while the kernel sources hash
    to the value recorded there (else None)."""
    import hashlib
    import re
    prof = ROOT / "profiles" / "pr_gather_hub1_kernel_rmat-s21.md"
    if not prof.exists():
        return None, None
    text = prof.read_text()
    m_hash = re.search(r"first 16 hex\): `([0-9a-f]{16})`", text)
    m_ratio = re.search(r"\| traffic / algorithmic \| ([0-9.]+) \|", text)
    csrc = ROOT / "paper_2108_02997_gb300" / "csrc"
    h = hashlib.sha256(b"".join((csrc / f).read_bytes() for f in ("pr_kernels.cuh", "pr_internal.cuh", "df64.cuh")))
    if not (m_hash and m_ratio) or h.hexdigest()[:16] != m_hash.group(1):
        return None, None
    return float(m_ratio.group(1)), ("scaled: one ncu capture at R-MAT scale 21 "
                                     "(profiles/pr_gather_hub1_kernel_rmat-s21.md), traffic/algorithmic bytes "
                                     "times this launch's algorithmic bytes")


def peaks():
    p = ROOT / "MEASURED_PEAKS.json"
    if p.exists():
        d = json.loads(p.read_text())
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# --------------------------------------------------------------------------- workloads

@dataclass
class Workload:
    name: str
    graphs: list
    specs: list                 # (graph index, alpha, tau, norm, max_iter)
    desc: str
    precision: str = "df64"     # batched arm
    learned: bool = False       # the learned warm start takes part (trained before timing)
    start: str = "uniform"      # batched arm's start: uniform, learned, or auto (learned where it pays)
    dgs: list = field(default_factory=list)
    outs: list = field(default_factory=list)


def sweep_specs(gis, alphas):
    return [(gi, a, t, nm, 500) for gi in gis for a in alphas for t in TAUS_SWEEP for nm in (1, 2, 3)]


def make_workload(name, gg, rank=0) -> Workload:
    """Graphs and instances of one workload. Rank r > 0 of a multi-GPU run gets
    graphs of the same shape from its own seeds (weak scaling: every rank
    solves a full batch of its own)."""
    from paper_2108_02997_gb300.dist import rank_seed
    s = lambda seed: rank_seed(seed, rank)
    if name in ("rmat22", "rmat21"):
        scale = int(name[4:])
        g = gg.rmat(scale, 16, seed=s(scale))
        specs = [(0, 0.85, t, nm, 500) for t in (1e-6, 1e-10) for nm in (1, 2, 3)]
        return Workload(name, [g], specs, f"rmat-s{scale} ef16 seed{scale}, alpha .85, tau {{1e-6,1e-10}} x {{L1,L2,Linf}}")
    if name == "sweep330":
        g = gg.erdos_renyi_10k(seed=s(1))
        return Workload(name, [g], sweep_specs([0], ALPHAS_SWEEP),
                        ("er-10k (100k edges, 5% dangling), 11 alpha x 10 tau x 3 norms; planner-chosen start "
                         "(learned where it pays) and precision"),
                        precision="auto", learned=True, start="auto")
    if name == "sweep330warm":
        g = gg.erdos_renyi_10k(seed=s(1))
        return Workload(name, [g], sweep_specs([0], ALPHAS_SWEEP),
                        "er-10k, 11 alpha x 10 tau x 3 norms; learned start, fp32->df64", precision="mixed",
                        learned=True, start="learned")
    if name == "multi64":
        gs = [gg.rmat(12 + (i % 9), 16, seed=s(1000 + i)) for i in range(64)]
        specs = [(i, 0.85, 1e-10, 1, 500) for i in range(64)]
        return Workload(name, gs, specs, "64 rmat graphs scale 12..20 ef16, alpha .85, tau 1e-10, L1",
                        precision="auto")
    if name == "evalsweep":
        gs = [gg.rmat(22, 16, seed=s(3022)), gg.rmat(24, 16, seed=s(3024)), gg.config_model(8_000_000, seed=s(3008))]
        return Workload(name, gs, sweep_specs(range(3), ALPHAS_TRAIN),
                        ("unseen rmat-s22 (seed 3022), rmat-s24 (seed 3024), config model N=8M (seed 3008); "
                         "10 alpha x 10 tau x 3 norms each; planner-chosen start (learned where it pays) and precision"),
                        precision="auto", learned=True, start="auto")
    if name == "rmat24mixed":
        g = gg.rmat(24, 16, seed=s(24))
        specs = [(0, a, 1e-10, 3, 500) for a in (0.85, 0.95)]
        return Workload(name, [g], specs, "rmat-s24 ef16 seed24, alpha {.85,.95}, Linf, tau 1e-10, fp32->df64",
                        precision="mixed")
    if name == "road24":
        g = gg.road_grid(4096, 4096, seed=s(7))
        specs = [(0, 0.85, t, nm, 500) for t in (1e-6, 1e-10) for nm in (1, 2, 3)]
        return Workload(name, [g], specs, ("road-like lattice 4096 x 4096 (links kept .8, one-way .2), alpha .85, "
                                           "tau {1e-6,1e-10} x {L1,L2,Linf}"))
    if name == "learned":
        gs = [gg.rmat(22, 16, seed=s(3022)), gg.rmat(24, 16, seed=s(3024)), gg.config_model(8_000_000, seed=s(3008))]
        specs = [(i, a, 1e-10, 1, 500) for i in range(len(gs)) for a in (0.5, 0.6, 0.7, 0.8, 0.85, 0.9, 0.95)]
        return Workload(name, gs, specs, ("unseen rmat-s22, rmat-s24, config model N=8M; 7 alpha x tau 1e-10 L1; "
                                          "learned start, fp32->df64"), precision="mixed", learned=True, start="learned")
    raise SystemExit(f"unknown workload {name}")


def train_warm_start(B, gg, torch, sptr, epochs=30, lr=3e-3):
    """Training of the learned warm start: 32 seeded R-MAT graphs of
    scale 16 + (i mod 5), alpha 0.50..0.95; targets are this library's own
    solves at tau 1e-12. Returns (mlp, graphs to keep alive, report)."""
    t0 = time.perf_counter()
    sets, keep = [], []
    for i in range(32):
        g = gg.rmat(16 + (i % 5), 16, seed=2000 + i)
        dg = B.Graph.from_csr(g)
        keep.append(dg)
        xs = [B.Instance(dg, a, 1e-12, 1, 2000, out=torch.empty(g.n, dtype=torch.float64, device="cuda"))
              for a in ALPHAS_TRAIN]
        B.pr_solve_batch(xs, outputs_on_device=True, stream=sptr)
        sets += [(dg, x.alpha, x.out) for x in xs]
    t1 = time.perf_counter()
    mlp = B.MLP(B.init_mlp_params(seed=17))
    loss0, _ = mlp.loss_grad(*sets[0])
    loss = mlp.train(sets, epochs=epochs, lr=lr, stream=sptr)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    return mlp, keep, {"train_sets": len(sets), "epochs": epochs, "lr": lr, "loss_first_set_initial": loss0,
                       "loss_final_mean": loss, "target_solves_s": round(t1 - t0, 2), "train_s": round(t2 - t1, 2)}


# --------------------------------------------------------------------------- clocks

class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "20"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            # sampling is live before the timed region starts
            t0 = time.time()
            while not self.lines and time.time() - t0 < 3.0 and self.proc.poll() is None:
                time.sleep(0.005)
            self.lines.clear()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, val in zip(names, f[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------------------- distributed

def dist_init(n_gpus):
    from paper_2108_02997_gb300 import dist
    return dist.init("cuda")


def barrier(world):
    from paper_2108_02997_gb300 import dist
    dist.barrier(world, "cuda")


def max_over_ranks(x, world):
    from paper_2108_02997_gb300 import dist
    return dist.max_over_ranks(x, world, "cuda")


# --------------------------------------------------------------------------- helpers of our arm

def gm(v):
    v = [float(x) for x in v]
    return math.exp(sum(math.log(x) for x in v) / len(v))


def trajectories(w):
    """(graph, alpha) -> instance indices: the iterate sequences the instances share."""
    out = {}
    for k, (gi, a, t, nm, mi) in enumerate(w.specs):
        out.setdefault((gi, a), []).append(k)
    return out


def sweep_report(B, torch, w, last, mlp, sptr):
    """Outputs of an alpha x tau x norm sweep on one graph beyond its timing
    (untimed): per alpha, the L1 distance of its ranks (tau 1e-10, L1) to the
    alpha = 0.85 ranks and its iteration count relative to alpha = 0.85 (the
    comparisons of Section 2); the same instances solved in FP32 throughout,
    giving per norm the largest tau at which an alpha < 1 instance ran into the
    500 cap (the stalls Section 4 describes); and the tau 1e-10 L1 column of
    every alpha started from the uniform vector, from the learned start, and
    from the previous alpha's answer (alpha continuation), in one batch each."""
    dg = w.dgs[0]
    ks = {a: [k for k, (gi, a2, t, nm, mi) in enumerate(w.specs) if a2 == a and t == 1e-10 and nm == 1][0]
          for a in ALPHAS_SWEEP}
    ref = w.outs[ks[0.85]]
    l1 = [float((w.outs[ks[a]] - ref).abs().sum()) for a in ALPHAS_SWEEP]
    ratio = [last[ks[a]].iters / last[ks[0.85]].iters for a in ALPHAS_SWEEP]
    xs = [B.Instance(w.dgs[gi], a, t, nm, mi) for gi, a, t, nm, mi in w.specs]
    B.pr_solve_batch(xs, precision="fp32", stream=sptr)
    stall = {}
    for nm, name in ((1, "L1"), (2, "L2"), (3, "Linf")):
        hit = [t for (gi, a, t, n2, mi), x in zip(w.specs, xs) if n2 == nm and a < 1.0 and not x.converged]
        stall[name] = max(hit) if hit else None
    starts = {}
    for mode, kw in (("uniform", {}), ("learned", {"init": "learned", "mlp": mlp}), ("continuation", {"init": "chain"})):
        ys = [B.Instance(dg, a, 1e-10, 1, 500) for a in ALPHAS_SWEEP]
        B.pr_solve_batch(ys, stream=sptr, **kw)
        starts[mode] = [y.iters for y in ys]
    its = {nm: [x.iters for (gi, a, t, n2, mi), x in zip(w.specs, last) if a == 0.85 and n2 == nm] for nm in (1, 2, 3)}
    norm_gm = {name: gm(its[nm]) / gm(its[1]) for nm, name in ((1, "L1"), (2, "L2"), (3, "Linf"))}
    return {"alpha": ALPHAS_SWEEP, "l1_vs_alpha_085": l1, "iterations_vs_alpha_085": ratio,
            "tau_sweep_iteration_gm_ratio_alpha_085": norm_gm,
            "fp32_largest_tau_hitting_cap": stall,
            "fp32_stalls_road_lattice": fp32_stalls(B, sptr),
            "start_iterations_tau_1e-10_L1": starts,
            "start_iterations_total": {k: sum(v) for k, v in starts.items()}}


def fp32_stalls(B, sptr):
    """The sensitivity stalls of Section 4 on a slow-mixing input: a road-like
    lattice of 300 x 400 vertices (seed 7), alpha 0.85, tau 1e-4 .. 1e-12 x
    {L1, L2, Linf}, in FP32 and in DF64; per norm the largest tau at which the
    solve ran into the 500 cap (None: none did)."""
    from paper_2108_02997_gb300 import graphgen as gg
    g = gg.road_grid(300, 400, seed=7)
    taus = [10.0 ** -k for k in range(4, 13)]
    out = {"graph": "road-like lattice 300 x 400 (seed 7), alpha .85"}
    with B.Graph.from_csr(g) as dg:
        for prec in ("fp32", "df64"):
            xs = [B.Instance(dg, 0.85, t, nm, 500) for t in taus for nm in (1, 2, 3)]
            B.pr_solve_batch(xs, precision=prec, stream=sptr)
            out[prec] = {name: max([x.tol for x in xs if x.norm == nm and x.iters >= 500], default=None)
                         for nm, name in ((1, "L1"), (2, "L2"), (3, "Linf"))}
    return out


def cuda_ms(torch, stream, fn):
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    r = fn()
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1), r


# --------------------------------------------------------------------------- our arm

def run_ours(args, world, rank, local):
    import numpy as np
    import torch

    from paper_2108_02997_gb300 import binding as B
    from paper_2108_02997_gb300 import graphgen as gg

    torch.cuda.set_device(local)
    B.lib()
    stream = torch.cuda.current_stream()
    sptr = int(stream.cuda_stream)
    names = HEADLINE if args.workload == "headline" else (args.workload,)
    wls = [make_workload(n, gg, rank) for n in names]
    for w in wls:
        w.dgs = [B.Graph.from_csr(g) for g in w.graphs]
        w.outs = [torch.empty(w.graphs[gi].n, dtype=torch.float64, device="cuda") for gi, *_ in w.specs]
    mlp, train = None, None
    if any(w.learned for w in wls):
        mlp, _train_keep, train = train_warm_start(B, gg, torch, sptr)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    # every workload's instances marshalled once (PreparedBatch), solved once
    # per call into the same device outputs; the timed arm and the comparison
    # arms below (no sharing, fixed starts) all go through these
    prepared = {w.name: B.PreparedBatch([B.Instance(w.dgs[gi], a, t, nm, mi, out=w.outs[k])
                                         for k, (gi, a, t, nm, mi) in enumerate(w.specs)], outputs_on_device=True)
                for w in wls}

    def solve(w, share=True, init=None):
        pb = prepared[w.name]
        kw = {"init": init, "mlp": mlp} if init in ("learned", "auto") else {}
        pb.solve(precision=w.precision, stream=sptr, share=share, loop=args.loop, **kw)
        return pb

    def timed_avg(fn):
        # L2 flushed before each run, as before each step of the timed arm;
        # runs under 100 ms are repeated three times and averaged
        out = []
        while True:
            flush.zero_()
            ms, r = cuda_ms(torch, stream, fn)
            out.append(ms)
            if len(out) >= (3 if out[0] < 100.0 else 1):
                return sum(out) / len(out), r

    def batched(w):
        pb = prepared[w.name]
        kw = {"init": w.start, "mlp": mlp} if w.start != "uniform" else {}
        pb.solve(precision=w.precision, stream=sptr, loop=args.loop, **kw)
        return pb

    for _ in range(args.warmup):
        flush.zero_()
        for w in wls:
            batched(w)
    torch.cuda.synchronize()
    learned_cols = {}
    for w in wls:
        batched(w)
        learned_cols[w.name] = B.pr_last_solve_stats()["learned_columns"]
    per_w = {w.name: [] for w in wls}
    launches = 0
    last = {}
    barrier(world)
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        for _ in range(args.steps):
            flush.zero_()                      # L2 flushed between steps (outside the timed regions)
            for w in wls:
                ms, _ = cuda_ms(torch, stream, lambda w=w: batched(w))
                per_w[w.name].append(ms)
                launches += B.pr_last_solve_stats()["launches"]
        torch.cuda.synchronize()
    barrier(world)
    clocks = clk.summary()
    for w in wls:
        last[w.name] = prepared[w.name].fill()
    ms_w = {n: sum(v) / len(v) for n, v in per_w.items()}
    ms_step = sum(ms_w.values())
    ms_step_max = max_over_ranks(ms_step, world)
    solves = sum(len(w.specs) for w in wls)
    value = world * solves * 1000.0 / ms_step_max
    # ---- per workload: the plain per-instance solver, the batch without
    # trajectory sharing, the learned start's net effect
    records = {}
    for w in wls:
        xs = last[w.name]
        rec = {"instances": len(w.specs), "graphs": len(w.graphs), "edges": sum(g.nnz for g in w.graphs),
               "trajectories": len(trajectories(w)), "batched_ms": ms_w[w.name],
               "batched": {"precision": w.precision, "start": w.start,
                           "learned_start_columns": learned_cols[w.name]},
               "iterations_total": sum(x.iters for x in xs),
               "converged": sum(1 for x in xs if x.converged)}
        # edges traversed: each trajectory's graph times its last tap's iterations
        tr = trajectories(w)
        rec["gteps_trajectories"] = sum(w.graphs[gi].nnz * max(xs[k].iters for k in ks)
                                        for (gi, a), ks in tr.items()) / (ms_w[w.name] * 1e-3) / 1e9
        if not args.no_plain:
            t_plain = 0.0
            for k, (gi, a, t, nm, mi) in enumerate(w.specs):
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                B.pr_solve(w.dgs[gi], a, t, nm, mi, out=w.outs[k], loop="host", stream=sptr, precision="df64")
                torch.cuda.synchronize()
                t_plain += time.perf_counter() - t0
            rec["plain_ms"] = t_plain * 1000.0
            rec["ratio"] = rec["plain_ms"] / rec["batched_ms"]
            ms_ns, _ = timed_avg(lambda w=w: solve(w, share=False, init=w.start))
            rec["batched_no_share_ms"] = ms_ns
            rec["ratio_no_share"] = rec["plain_ms"] / ms_ns
        if w.learned:
            # both fixed starts: what the learned start saves net of its own
            # cost (features, network, softmax)
            ms_u, pb = timed_avg(lambda w=w: solve(w))
            it_u = int(pb.iters.sum())
            ms_l, pb = timed_avg(lambda w=w: solve(w, init="learned"))
            it_l = int(pb.iters.sum())
            rec["uniform_start"] = {"batched_ms": ms_u, "iterations_total": it_u}
            rec["learned_start"] = {"batched_ms": ms_l, "iterations_total": it_l,
                                    "saves_iterations": it_u - it_l, "net_ms_saved": ms_u - ms_l}
            rec["mlp_gain"] = mlp.gain()[0]
            # the start's own cost: features once per graph, network and softmax per alpha
            ws = []
            for dg in w.dgs:
                buf = torch.empty(dg.n, dtype=torch.float64, device="cuda")
                mlp.warm_start(dg, 0.85, out=buf, stream=sptr)
                ms1, _ = cuda_ms(torch, stream, lambda dg=dg, buf=buf: mlp.warm_start(dg, 0.85, out=buf, stream=sptr))
                ws.append({"n": dg.n, "ms": ms1})
            rec["warm_start_ms_per_call"] = ws
        if w.name.startswith("sweep330"):
            rec["sweep_report"] = sweep_report(B, torch, w, xs, mlp, sptr)
        records[w.name] = rec
    gm_ratio = gm_ratio_ns = None
    if not args.no_plain:
        gm_ratio = gm([records[n]["ratio"] for n in records])
        gm_ratio_ns = gm([records[n]["ratio_no_share"] for n in records])
    # ---- roofline: the one-column gather kernel at R-MAT scale 22, one launch
    # per iteration, each launch bracketed by CUDA events on the solve's stream
    roofline = roofline_s22(B, gg, torch, sptr, rank, wls if args.workload == "rmat22" else None)
    # ---- e2e: through the C ABI from pinned host arrays, every step: graph
    # creation (host CSR to the device), the batched solves, per-instance
    # results and each trajectory's answer (its last stopping rule) to the host
    e2e = None if args.no_e2e else run_e2e(B, torch, wls, mlp, sptr, args, world)
    # ---- CPU baseline: the oracle on the host cores, bounded samples
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline(wls, args.cpu_seconds)
    precisions = sorted({w.precision for w in wls})
    line = {
        "metric": METRIC,
        "value": value,
        "unit": "solves/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms_step_max,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "df64 (f32x2); f32 -> df64 where the planner picks mixed precision"
        if "auto" in precisions or "mixed" in precisions else "df64 (f32x2)",
        "data": "synthetic (seeded generators; paper's SuiteSparse graphs unavailable)",
        "config": {"workload": " + ".join(w.name for w in wls) if len(wls) > 1 else wls[0].desc,
                   "workloads": {w.name: w.desc for w in wls},
                   "instances": solves, "graphs": sum(len(w.graphs) for w in wls),
                   "edges": sum(sum(g.nnz for g in w.graphs) for w in wls),
                   "parallelism": f"instance batches x{world} (one per rank, no collective)",
                   "l2": "L2 flushed (256 MB write) before every step"},
        "workloads": records,
        "gm_ratio": gm_ratio,
        "gm_ratio_no_share": gm_ratio_ns,
        "gm_ratio_what": ("geometric mean over the workloads of (plain per-instance time) / (batched time); "
                          "plain = every instance alone through pr_solve, df64, uniform start, one launch per "
                          "iteration and a host read of the stop flag"),
        "learned_training": train,
        "roofline": roofline,
        "e2e": e2e,
        "cpu_baseline": cpu,
        "clocks": clocks,
        "gpu_launches": launches,
    }
    if rank == 0:
        print(json.dumps(line))
    for w in wls:
        for d in w.dgs:
            d.close()


def roofline_s22(B, gg, torch, sptr, rank, have):
    """The gather kernel's and the whole pass's achieved bandwidth on R-MAT
    scale 22 against the measured copy bandwidth. Algorithmic bytes per
    one-column pass (the method's data): offsets 4(N+1), in-edge indices 4E,
    each source's contribution once 8 N_src, previous ranks 8N, new ranks 8N,
    out-degrees 4N; of these the gather kernel moves the first three."""
    if have is not None:
        w = have[0]
    else:
        w = make_workload("rmat22", gg, rank)
        w.dgs = [B.Graph.from_csr(w.graphs[0])]
        w.outs = [torch.empty(w.graphs[0].n, dtype=torch.float64, device="cuda") for _ in w.specs]
    g, dg = w.graphs[0], w.dgs[0]
    hbm, peak_kind = peaks()
    xs = [B.Instance(dg, a, t, nm, mi, out=w.outs[k]) for k, (gi, a, t, nm, mi) in enumerate(w.specs)]
    B.pr_solve_batch(xs, outputs_on_device=True, stream=sptr, loop="host")
    st = B.pr_last_solve_stats()
    n_src = int((g.outdeg > 0).sum())
    b_pass = 4.0 * (g.n + 1) + 4.0 * g.nnz + 8.0 * n_src + 8.0 * g.n + 8.0 * g.n + 4.0 * g.n
    b_gather = 4.0 * (g.n + 1) + 4.0 * g.nnz + 8.0 * n_src
    passes = max(st["passes"], 1)
    pass_us = st["kernel_ms"] / passes * 1e3
    gather_us = st["gather_ms"] / passes * 1e3
    ach = b_gather / (gather_us * 1e-6) / 1e9
    ratio, tsrc = kernel_traffic_ratio()
    if have is None:
        dg.close()
    ceiling = gather_ceiling(g, b_gather, gather_us)
    return {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm,
            "ceiling": ceiling,
            "traffic": ratio * b_gather if ratio else None, "traffic_source": tsrc,
            "kernel": "pr_gather_hub1_kernel<df64> (gather half of a one-column pass)",
            "workload": "rmat-s22 ef16 seed22 (N 4,194,304, E %d), alpha .85, tau {1e-6,1e-10} x {L1,L2,Linf}, df64"
                        % g.nnz,
            "avg_launch_us": gather_us, "algorithmic_bytes_per_launch": b_gather, "launches": passes,
            "peak_source": peak_kind, "frac_of": "measured copy bandwidth" if peak_kind == "measured" else "fallback",
            "pass": {"avg_pass_us": pass_us, "algorithmic_bytes_per_pass": b_pass,
                     "achieved": b_pass / (pass_us * 1e-6) / 1e9, "frac": b_pass / (pass_us * 1e-6) / 1e9 / hbm,
                     "update_kernel_us": st["update_ms"] / passes * 1e3}}


def gather_ceiling(g, b_gather, gather_us, hub_values=12288):
    """What the GPU's memory system allows this gather (libprceiling.so, CUDA
    probes over the same relabelled in-edge stream, no row sums): the index
    stream alone, every gather through L1/L2, the same with the hub table in
    shared memory, and uniform random gathers over a table of N values."""
    import ctypes as C

    import numpy as np

    from paper_2108_02997_gb300 import _build
    L = C.CDLL(str(_build.build_ceiling()))
    L.prc_gather_ceiling.argtypes = [C.c_int32, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p]
    L.prc_gather_ceiling.restype = C.c_int
    off = np.ascontiguousarray(g.offsets, np.int32)
    src = np.ascontiguousarray(g.sources, np.int32)
    od = np.ascontiguousarray(g.outdeg, np.int32)
    us = np.zeros(4, np.float64)
    rc = L.prc_gather_ceiling(g.n, g.nnz, off.ctypes.data, src.ctypes.data, od.ctypes.data, hub_values, us.ctypes.data)
    if rc != 0:
        return {"error": f"probe returned {rc}"}
    best = min(us[1], us[2])
    return {"index_stream_us": us[0], "gathers_us": us[1], "gathers_hub_us": us[2], "hub_values": hub_values,
            "uniform_random_us": us[3], "gathers_per_s": g.nnz / (us[1] * 1e-6),
            "gathers_hub_per_s": g.nnz / (us[2] * 1e-6), "uniform_random_gathers_per_s": g.nnz / (us[3] * 1e-6),
            "ceiling_frac_of_peak": b_gather / (best * 1e-6) / 1e9 / peaks()[0],
            "kernel_vs_ceiling": best / gather_us,
            "what": ("edge-parallel probes over the same relabelled in-edge stream, eight gathers per thread in "
                     "flight, values folded by XOR (no row sums): the fastest the memory system serves these "
                     "random 8-byte reads; kernel_vs_ceiling = probe time / gather kernel time")}


def run_e2e(B, torch, wls, mlp, sptr, args, world):
    import numpy as np
    pinned = []
    for w in wls:
        pinned.append([(torch.from_numpy(g.offsets).pin_memory().numpy(), torch.from_numpy(g.sources).pin_memory().numpy(),
                        torch.from_numpy(g.outdeg).pin_memory().numpy()) for g in w.graphs])
    # each trajectory's answer at its last stopping rule (the last instance of the trajectory)
    picks = []
    for w in wls:
        picks.append([ks[-1] for ks in trajectories(w).values()])
    host = [[torch.empty(w.graphs[w.specs[k][0]].n, dtype=torch.float64).pin_memory() for k in pk]
            for w, pk in zip(wls, picks)]
    h2d = sum(a.nbytes + b.nbytes + c.nbytes for pw in pinned for a, b, c in pw)
    d2h = sum(h.numel() * 8 for hw in host for h in hw) + sum(len(w.specs) * 24 for w in wls)
    reps = min(args.steps, 5)
    et = []
    for i in range(1 + reps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for w, pw, pk, hw in zip(wls, pinned, picks, host):
            hg = [B.Graph(*p) for p in pw]
            xs = [B.Instance(hg[gi], a, t, nm, mi, out=w.outs[k]) for k, (gi, a, t, nm, mi) in enumerate(w.specs)]
            kw = {"init": w.start, "mlp": mlp} if w.start != "uniform" else {}
            B.pr_solve_batch(xs, precision=w.precision, outputs_on_device=True, stream=sptr, **kw)
            for k, h in zip(pk, hw):
                h.copy_(w.outs[k], non_blocking=True)
            torch.cuda.synchronize()
            for h in hg:
                h.close()
        t1 = time.perf_counter()
        if i >= 1:
            et.append((t1 - t0) * 1000.0)
    e2e_ms = max_over_ranks(sum(et) / len(et), world)
    solves = sum(len(w.specs) for w in wls)
    return {"value": world * solves * 1000.0 / e2e_ms, "unit": "solves/s", "ms_per_step": e2e_ms,
            "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "steps": reps,
            "what": ("graph creation from pinned host CSR arrays, pr_solve_batch, every instance's iterations/"
                     "error and each trajectory's final ranks to pinned host memory")}


def oracle_sample(graphs, specs, budget_s, cores):
    """Time the CPU oracle on a workload within about budget_s seconds.

    Instances sharing (graph, alpha) are one trajectory read at several stopping
    rules (oracle.pagerank_taps). Trajectories are solved in workload order for
    real while the estimated cost fits the budget; the rest are costed as
    (iterations) x (measured time of one oracle update on that graph), with
    iterations from Section 1's estimate round(log10 tau / log10 alpha)."""
    import numpy as np

    from oracle import oracle as orc
    t_upd = {}
    for gi in sorted({s[0] for s in specs}):
        g = graphs[gi]
        r = np.full(g.n, 1.0 / g.n)
        t0 = time.perf_counter()
        r, _ = orc.step(g, 0.85, r, threads=cores)
        orc.norms(r, r)
        t_upd[gi] = time.perf_counter() - t0
    groups = {}
    for k, (gi, a, t, nm, mi) in enumerate(specs):
        groups.setdefault((gi, a), []).append(k)
    spent, solved, modeled = 0.0, 0, 0.0
    for (gi, a), ks in groups.items():
        taps = [(specs[k][2], specs[k][3], specs[k][4]) for k in ks]
        est = max(min(mi, orc.estimate_iterations(t, a) if 0 < a < 1 else mi) for t, nm, mi in taps)
        if spent + t_upd[gi] * est <= budget_s:
            t0 = time.perf_counter()
            orc.pagerank_taps(graphs[gi], a, taps, threads=cores)
            spent += time.perf_counter() - t0
            solved += len(ks)
        else:
            for t, nm, mi in taps:
                it = min(mi, orc.estimate_iterations(t, a)) if 0 < a < 1 else mi
                modeled += t_upd[gi] * max(it, 1)
    total_time = spent + modeled
    kind = "measured" if modeled == 0 else ("mixed" if solved else "extrapolated")
    return {"time_s": total_time, "solved": solved, "spent_s": spent, "kind": kind}


def cpu_baseline(wls, seconds):
    """The oracle as it stands on a bounded sample of every workload, on all
    host cores and on one (the paper's program is single-threaded)."""
    from oracle import oracle as orc
    out = {}
    for cores in (orc.default_threads(), 1):
        t_all, parts = 0.0, []
        for w in wls:
            r = oracle_sample(w.graphs, w.specs, seconds / len(wls), cores)
            t_all += r["time_s"]
            parts.append(f"{w.name}: {r['solved']} of {len(w.specs)} solved ({r['spent_s']:.1f}s), rest {r['kind']}")
        out[cores] = (sum(len(w.specs) for w in wls) / t_all, "; ".join(parts))
    allc = orc.default_threads()
    return {"value": out[allc][0], "unit": "solves/s", "cores": allc, "kind": "oracle",
            "sample": out[allc][1] + " (unsolved instances costed as Section 1's estimated iterations x measured "
                                     "update time)",
            "single_thread": {"value": out[1][0], "unit": "solves/s", "cores": 1, "sample": out[1][1]}}


# --------------------------------------------------------------------------- reference arm

def run_reference(args, world, rank):
    """The oracle, as it stands, on the host cores; rank 0 only."""
    if rank != 0:
        return
    from oracle import oracle as orc
    from paper_2108_02997_gb300 import graphgen as gg
    orc.build()
    names = HEADLINE if args.workload == "headline" else (args.workload,)
    wls = [make_workload(n, gg) for n in names]
    cores = orc.default_threads()
    budget = max(1.0, args.ref_seconds)
    w0 = wls[0]
    for _ in range(args.warmup):
        oracle_sample(w0.graphs, w0.specs[:1], 0.2, cores)
    vals, samples = [], []
    for _ in range(args.steps):
        t, parts = 0.0, []
        for w in wls:
            r = oracle_sample(w.graphs, w.specs, budget / len(wls), cores)
            t += r["time_s"]
            parts.append(f"{w.name}: {r['solved']} of {len(w.specs)} solved, rest {r['kind']}")
        vals.append(sum(len(w.specs) for w in wls) / t)
        samples.append("; ".join(parts))
    v = statistics.mean(vals)
    solves = sum(len(w.specs) for w in wls)
    line = {"metric": METRIC, "value": v, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": solves / v * 1000.0, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": " + ".join(w.name for w in wls) if len(wls) > 1 else wls[0].desc,
                       "instances": solves, "graphs": sum(len(w.graphs) for w in wls)},
            "impl": "reference",
            "cpu_baseline": {"kind": "oracle", "cores": cores, "value": v, "unit": "solves/s",
                             "sample": samples[-1] + " (unsolved instances costed as Section 1's estimated "
                                                     "iterations x measured update time)"},
            "e2e": {"value": v, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="headline", choices=("headline",) + SINGLE)
    ap.add_argument("--loop", default="auto", choices=["auto", "graph", "persistent", "host"],
                    help="loop of the timed solves (auto: persistent passes where they apply, else the CUDA "
                         "graph's while-loop; host: one launch per iteration)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-plain", action="store_true", help="skip the plain per-instance GPU solver comparison")
    ap.add_argument("--cpu-seconds", type=float, default=20.0, help="oracle budget of the cpu_baseline sample")
    ap.add_argument("--ref-seconds", type=float, default=6.0, help="oracle budget per step of --impl reference")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args, int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")))
        return
    world, rank, local = dist_init(args.gpus)
    run_ours(args, world, rank, local)
    from paper_2108_02997_gb300 import dist
    dist.finish(world)


if __name__ == "__main__":
    main()
