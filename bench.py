#!/usr/bin/env python3
"""Benchmark of the PageRank hot path on GB300 (one JSON line on stdout).

Workloads (synthetic, seeded; stand-ins for the paper's SuiteSparse graphs):

* ``rmat22`` (default) — R-MAT scale 22 (N = 4,194,304; 67,108,864 sampled
  edges; a/b/c/d = .57/.19/.19/.05; ids permuted; self-loops and duplicates
  removed), alpha = 0.85, tau in {1e-6, 1e-10} x {L1, L2, Linf}: 6 instances
  solved as one batch (one shared iterate sequence, six stopping rules).
* ``sweep330`` — the 10k-vertex Erdos-Renyi graph, alpha 0.50..1.00 step .05
  x tau 1e-1..1e-10 x {L1, L2, Linf} = 330 instances, max 500 iterations.
* ``multi64`` — 64 R-MAT graphs of scale 12 + (i mod 9), edge factor 16,
  alpha 0.85, tau 1e-10, L1, one batch.
* ``rmat24mixed`` — R-MAT scale 24, alpha in {0.85, 0.95}, Linf, tau 1e-10,
  FP32 phase to 1e-6 then DF64 refinement.

A step is one solve of the whole workload with the graph resident in HBM
(``value``); ``e2e`` repeats it through the public C ABI from pinned host
arrays (graph creation, solve, ranks back to the host) every step.
``--impl reference`` times the CPU oracle on the host cores instead.
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
from pathlib import Path

ROOT = Path(__file__).resolve().parent
sys.path.insert(0, str(ROOT))

METRIC = "sweep solves/s and GTEPS (%HBM roofline), batched+warm vs plain, ≤10τ/(1−α) L1 err"


def kernel_traffic_ratio():
    """DRAM traffic / algorithmic bytes of the iteration kernel from the ncu
    capture summarised in profiles/, valid only while the kernel sources hash
    to the value recorded there (else None)."""
    import hashlib
    import re
    prof = ROOT / "profiles" / "pr_iter_kernel-gather_rmat-s21.md"
    if not prof.exists():
        return None, None
    text = prof.read_text()
    m_hash = re.search(r"first 16 hex\): `([0-9a-f]{16})`", text)
    m_ratio = re.search(r"\| traffic / algorithmic \| ([0-9.]+) \|", text)
    csrc = ROOT / "paper_2108_02997_gb300" / "csrc"
    h = hashlib.sha256(b"".join((csrc / f).read_bytes() for f in ("pr_kernels.cuh", "pr_internal.cuh", "df64.cuh")))
    if not (m_hash and m_ratio) or h.hexdigest()[:16] != m_hash.group(1):
        return None, None
    return float(m_ratio.group(1)), "ncu capture at rmat-s21 (profiles/pr_iter_kernel-gather_rmat-s21.md), scaled by algorithmic bytes"


def peaks():
    p = ROOT / "MEASURED_PEAKS.json"
    if p.exists():
        d = json.loads(p.read_text())
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# --------------------------------------------------------------------------- workloads

def make_workload(name, gg, rank=0):
    """(graphs, instance specs [(graph index, alpha, tau, norm, max_iter)], precision, description).
    Rank r > 0 of a multi-GPU run gets graphs of the same shape from its own
    seeds (weak scaling: every rank solves a full batch of its own)."""
    from paper_2108_02997_gb300.dist import rank_seed
    s = lambda seed: rank_seed(seed, rank)
    if name in ("rmat22", "rmat21"):
        scale = int(name[4:])
        g = gg.rmat(scale, 16, seed=s(scale))
        specs = [(0, 0.85, t, nm, 500) for t in (1e-6, 1e-10) for nm in (1, 2, 3)]
        return [g], specs, "df64", f"rmat-s{scale} ef16 seed{scale}, alpha .85, tau {{1e-6,1e-10}} x {{L1,L2,Linf}}"
    if name == "sweep330":
        g = gg.erdos_renyi_10k(seed=s(1))
        alphas = [round(0.5 + 0.05 * i, 2) for i in range(11)]
        specs = [(0, a, 10.0 ** -k, nm, 500) for a in alphas for k in range(1, 11) for nm in (1, 2, 3)]
        return [g], specs, "df64", "er-10k (100k edges, 5% dangling), 11 alpha x 10 tau x 3 norms"
    if name == "multi64":
        gs = [gg.rmat(12 + (i % 9), 16, seed=s(1000 + i)) for i in range(64)]
        specs = [(i, 0.85, 1e-10, 1, 500) for i in range(64)]
        return gs, specs, "df64", "64 rmat graphs scale 12..20 ef16, alpha .85, tau 1e-10, L1"
    if name == "rmat24mixed":
        g = gg.rmat(24, 16, seed=s(24))
        specs = [(0, a, 1e-10, 3, 500) for a in (0.85, 0.95)]
        return [g], specs, "mixed", "rmat-s24 ef16 seed24, alpha {.85,.95}, Linf, tau 1e-10, fp32->df64"
    if name == "sweep330warm":
        g = gg.erdos_renyi_10k(seed=s(1))
        alphas = [round(0.5 + 0.05 * i, 2) for i in range(11)]
        specs = [(0, a, 10.0 ** -k, nm, 500) for a in alphas for k in range(1, 11) for nm in (1, 2, 3)]
        return [g], specs, "mixed", ("er-10k, 11 alpha x 10 tau x 3 norms; learned start, fp32->df64 "
                                     "(the batched mixed-precision warm-started sweep)")
    if name == "road24":
        g = gg.road_grid(4096, 4096, seed=s(7))
        specs = [(0, 0.85, t, nm, 500) for t in (1e-6, 1e-10) for nm in (1, 2, 3)]
        return [g], specs, "df64", ("road-like lattice 4096 x 4096 (links kept .8, one-way .2), alpha .85, "
                                    "tau {1e-6,1e-10} x {L1,L2,Linf}")
    if name == "learned":
        gs = [gg.rmat(22, 16, seed=s(3022)), gg.rmat(24, 16, seed=s(3024)), gg.config_model(8_000_000, seed=s(3008))]
        alphas = (0.5, 0.6, 0.7, 0.8, 0.85, 0.9, 0.95)
        specs = [(i, a, 1e-10, 1, 500) for i in range(len(gs)) for a in alphas]
        return gs, specs, "mixed", ("unseen rmat-s22 (seed 3022), rmat-s24 (seed 3024), config model N=8M "
                                    "(seed 3008); 7 alpha x tau 1e-10 L1; learned start, fp32->df64")
    raise SystemExit(f"unknown workload {name}")


def train_warm_start(B, gg, torch, sptr, epochs=30, lr=3e-3):
    """Training of the learned warm start: 32 seeded R-MAT graphs of
    scale 16 + (i mod 5), alpha 0.50..0.95; targets are this library's own
    solves at tau 1e-12. Returns (mlp, report)."""
    alphas = [round(0.5 + 0.05 * i, 2) for i in range(10)]
    t0 = time.perf_counter()
    sets, keep = [], []
    for i in range(32):
        g = gg.rmat(16 + (i % 5), 16, seed=2000 + i)
        dg = B.Graph.from_csr(g)
        keep.append(dg)
        xs = [B.Instance(dg, a, 1e-12, 1, 2000, out=torch.empty(g.n, dtype=torch.float64, device="cuda"))
              for a in alphas]
        B.pr_solve_batch(xs, outputs_on_device=True, stream=sptr)
        sets += [(dg, x.alpha, x.out) for x in xs]
    t1 = time.perf_counter()
    mlp = B.MLP(B.init_mlp_params(seed=17))
    loss0, _ = mlp.loss_grad(*sets[0])
    loss = mlp.train(sets, epochs=epochs, lr=lr, stream=sptr)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    return mlp, keep, {"train_sets": len(sets), "epochs": epochs, "lr": lr, "loss_first_set_initial": loss0,
                       "loss_final_mean": loss, "target_solves_s": t1 - t0, "train_s": t2 - t1}


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

def sweep_report(B, torch, dgs, specs, last, outs, sptr):
    """Outputs of the alpha x tau x norm sweep beyond its timing (untimed):
    per alpha, the L1 distance of its ranks (tau 1e-10, L1) to the alpha = 0.85
    ranks and its iteration count relative to alpha = 0.85 (the comparisons of
    Section 2); and the same 330 instances solved in FP32 throughout, giving per
    norm the largest tau at which an alpha < 1 instance ran into the 500 cap
    (the stalls Section 4 describes)."""
    ref_k = [k for k, (gi, a, t, nm, mi) in enumerate(specs) if a == 0.85 and t == 1e-10 and nm == 1][0]
    alphas, l1, ratio = [], [], []
    for k, (gi, a, t, nm, mi) in enumerate(specs):
        if t == 1e-10 and nm == 1:
            alphas.append(a)
            l1.append(float((outs[k] - outs[ref_k]).abs().sum()))
            ratio.append(last[k].iters / last[ref_k].iters)
    xs = [B.Instance(dgs[gi], a, t, nm, mi) for gi, a, t, nm, mi in specs]
    B.pr_solve_batch(xs, precision="fp32", stream=sptr)
    stall = {}
    for nm, name in ((1, "L1"), (2, "L2"), (3, "Linf")):
        hit = [t for (gi, a, t, n2, mi), x in zip(specs, xs) if n2 == nm and a < 1.0 and not x.converged]
        stall[name] = max(hit) if hit else None
    # alpha continuation (tau 1e-10, L1, df64): each alpha starts from the
    # previous alpha's ranks instead of 1/N
    uni, cont, prev = [], [], None
    for a in alphas:
        r_u = B.pr_solve(dgs[0], a, 1e-10, 1, 500, out=torch.empty(dgs[0].n, dtype=torch.float64, device="cuda"))
        uni.append(r_u.iters)
        out = torch.empty(dgs[0].n, dtype=torch.float64, device="cuda")
        r_c = B.pr_solve(dgs[0], a, 1e-10, 1, 500, out=out, init=prev) if prev is not None else r_u
        cont.append(r_c.iters)
        prev = out if prev is not None else r_u.ranks
    # the paper's norm comparison over the tau sweep at alpha 0.85: geometric
    # mean over tau of iterations, each norm relative to L1 (Section 4)
    def gm(v):
        v = [float(x) for x in v]
        return math.exp(sum(math.log(x) for x in v) / len(v))
    its = {nm: [x.iters for (gi, a, t, n2, mi), x in zip(specs, last) if a == 0.85 and n2 == nm] for nm in (1, 2, 3)}
    norm_gm = {name: gm(its[nm]) / gm(its[1]) for nm, name in ((1, "L1"), (2, "L2"), (3, "Linf"))}
    return {"alpha": alphas, "l1_vs_alpha_085": l1, "iterations_vs_alpha_085": ratio,
            "tau_sweep_iteration_gm_ratio_alpha_085": norm_gm,
            "fp32_largest_tau_hitting_cap": stall,
            "continuation": {"iterations_uniform": uni, "iterations_from_previous_alpha": cont,
                             "saved": sum(uni) - sum(cont)}}


def dist_init(n_gpus):
    from paper_2108_02997_gb300 import dist
    return dist.init("cuda")


def barrier(world):
    from paper_2108_02997_gb300 import dist
    dist.barrier(world, "cuda")


def max_over_ranks(x, world):
    from paper_2108_02997_gb300 import dist
    return dist.max_over_ranks(x, world, "cuda")


# --------------------------------------------------------------------------- our arm

def run_ours(args, world, rank, local):
    import numpy as np
    import torch

    from paper_2108_02997_gb300 import binding as B
    from paper_2108_02997_gb300 import graphgen as gg

    torch.cuda.set_device(local)
    B.lib()
    graphs, specs, precision, desc = make_workload(args.workload, gg, rank)
    dgs = [B.Graph.from_csr(g) for g in graphs]
    outs = [torch.empty(graphs[gi].n, dtype=torch.float64, device="cuda") for gi, *_ in specs]
    stream = torch.cuda.current_stream()
    sptr = int(stream.cuda_stream)
    mlp, learned = None, None
    if args.workload in ("learned", "sweep330warm"):
        mlp, _train_keep, learned = train_warm_start(B, gg, torch, sptr)
    init_kw = {"init": "learned", "mlp": mlp} if mlp is not None else {}
    total_edges = sum(g.nnz for g in graphs)
    l2_bytes = sum(4 * (g.n + 1) + 4 * g.nnz + 24 * g.n for g in graphs)
    inputs_large = l2_bytes > 2 * 129e6
    flush = None if inputs_large else torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    def insts():
        return [B.Instance(dgs[gi], a, t, nm, mi, out=outs[k]) for k, (gi, a, t, nm, mi) in enumerate(specs)]

    def step():
        xs = insts()
        B.pr_solve_batch(xs, precision=precision, outputs_on_device=True, stream=sptr, loop=args.loop, **init_kw)
        return xs

    for _ in range(args.warmup):
        if flush is not None:
            flush.zero_()
        last = step()
    torch.cuda.synchronize()
    launches = 0
    times = []
    barrier(world)
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        for _ in range(args.steps):
            if flush is not None:
                flush.zero_()
            ev0.record(stream)
            last = step()
            ev1.record(stream)
            ev1.synchronize()
            times.append(ev0.elapsed_time(ev1))
            launches += B.pr_last_solve_stats()["launches"]
        torch.cuda.synchronize()
    barrier(world)
    ms_step = sum(times) / len(times)
    ms_step_max = max_over_ranks(ms_step, world)
    solves = len(specs)
    value = world * solves * 1000.0 / ms_step_max
    inst_iters = [x.iters for x in last]
    edges_inst = sum(graphs[gi].nnz * x.iters for (gi, *_), x in zip(specs, last))
    # ---- roofline pass: the same solves with one launch per iteration, each
    # launch bracketed by CUDA events on the launching stream
    hbm, peak_kind = peaks()
    k_ms, k_launches, bytes_per_launch = 0.0, 0, 0.0
    g_ms, g_bytes = 0.0, 0.0
    for gi, g in enumerate(graphs):
        sel = [k for k, s in enumerate(specs) if s[0] == gi]
        xs = [B.Instance(dgs[gi], specs[k][1], specs[k][2], specs[k][3], specs[k][4], out=outs[k]) for k in sel]
        B.pr_solve_batch(xs, precision=precision, outputs_on_device=True, stream=sptr, loop="host", **init_kw)
        st = B.pr_last_solve_stats()
        n_src = int((g.outdeg > 0).sum())
        # one pass, one column: offsets, indices, gathered contributions (each
        # source once), previous ranks, new ranks, out-degrees
        b = 4.0 * (g.n + 1) + 4.0 * g.nnz + 8.0 * n_src + 8.0 * g.n + 8.0 * g.n + 4.0 * g.n
        # its gather kernel: offsets, indices, gathered contributions, row sums written
        bg = 4.0 * (g.n + 1) + 4.0 * g.nnz + 8.0 * n_src + 8.0 * g.n
        passes = st["passes"]
        k_ms += st["kernel_ms"]
        k_launches += passes
        bytes_per_launch += b * passes
        if st["gather_ms"] > 0:
            g_ms += st["gather_ms"]
            g_bytes += bg * passes
    avg_launch_ms = k_ms / max(k_launches, 1)
    bytes_avg = bytes_per_launch / max(k_launches, 1)
    achieved = bytes_avg / (avg_launch_ms * 1e-3) / 1e9
    pass_roofline = {"achieved": achieved, "frac": achieved / hbm, "avg_pass_us": avg_launch_ms * 1e3,
                     "algorithmic_bytes_per_pass": bytes_avg, "unit": "GB/s"}
    if g_ms > 0:
        # the dominant kernel is the gather kernel of the split passes
        kernel_name = "pr_iter_kernel (gather half of a one-column pass)"
        avg_kernel_ms = g_ms / max(k_launches, 1)
        kernel_bytes = g_bytes / max(k_launches, 1)
    else:
        kernel_name = "pr_iter_kernel (whole pass)"
        avg_kernel_ms = avg_launch_ms
        kernel_bytes = bytes_avg
    kernel_achieved = kernel_bytes / (avg_kernel_ms * 1e-3) / 1e9
    gteps_device = total_edges * (k_launches / max(len(graphs), 1)) / (ms_step * 1e-3) / 1e9
    if learned is not None:
        # iterations from the uniform start, same batched mixed-precision sweep
        xs_u = [B.Instance(dgs[gi], a, t, nm, mi, out=outs[k]) for k, (gi, a, t, nm, mi) in enumerate(specs)]
        B.pr_solve_batch(xs_u, precision=precision, outputs_on_device=True, stream=sptr)
        learned["iterations_uniform"] = [x.iters for x in xs_u]
        learned["iterations_learned"] = inst_iters
        learned["iterations_saved_total"] = sum(x.iters for x in xs_u) - sum(inst_iters)
        # cost of the start itself: features + MLP + softmax, per graph (CUDA events)
        ws = []
        for gi, dg in enumerate(dgs):
            buf = torch.empty(dg.n, dtype=torch.float64, device="cuda")
            mlp.warm_start(dg, 0.85, out=buf, stream=sptr)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            mlp.warm_start(dg, 0.85, out=buf, stream=sptr)
            e1.record(stream)
            e1.synchronize()
            ws.append({"n": dg.n, "ms": e0.elapsed_time(e1)})
        learned["warm_start_ms"] = ws
        if precision != "df64":
            # the same comparison with df64 throughout (no FP32 phase)
            its = {}
            for mode, kw in (("uniform", {}), ("learned", init_kw)):
                xs_d = [B.Instance(dgs[gi], a, t, nm, mi, out=outs[k]) for k, (gi, a, t, nm, mi) in enumerate(specs)]
                B.pr_solve_batch(xs_d, precision="df64", outputs_on_device=True, stream=sptr, **kw)
                its[mode] = [x.iters for x in xs_d]
            learned["df64"] = {"iterations_uniform": its["uniform"], "iterations_learned": its["learned"],
                               "iterations_saved_total": sum(its["uniform"]) - sum(its["learned"])}
    sweep = sweep_report(B, torch, dgs, specs, last, outs, sptr) if args.workload.startswith("sweep330") else None
    # ---- plain per-instance GPU solver on the same resident graphs: every
    # instance alone through pr_solve, one launch per iteration and a host read
    # of the stop flag after each (the baseline the batched path is measured against)
    plain = None
    if not args.no_plain:
        t_plain = 0.0
        for k, (gi, a, t, nm, mi) in enumerate(specs):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            B.pr_solve(dgs[gi], a, t, nm, mi, out=outs[k], loop="host", stream=sptr,
                       precision="df64" if precision == "mixed" else precision)
            torch.cuda.synchronize()
            t_plain += time.perf_counter() - t0
        plain = {"solves_per_s": solves / t_plain, "ms_per_step": t_plain * 1000.0,
                 "what": "each instance alone, pr_solve with one launch per iteration and a host read of the stop flag",
                 "speedup_of_value": (solves * 1000.0 / ms_step) / (solves / t_plain)}
    # ---- e2e: graph creation from pinned host arrays + solve + ranks to host, every step
    e2e = None
    if not args.no_e2e:
        pinned = []
        for g in graphs:
            off = torch.from_numpy(g.offsets).pin_memory().numpy()
            src = torch.from_numpy(g.sources).pin_memory().numpy()
            od = torch.from_numpy(g.outdeg).pin_memory().numpy()
            pinned.append((off, src, od))
        host_outs = [torch.empty(graphs[gi].n, dtype=torch.float64).pin_memory().numpy() for gi, *_ in specs]
        h2d = sum(a.nbytes + b.nbytes + c.nbytes for a, b, c in pinned)
        d2h = sum(o.nbytes for o in host_outs)
        et = []
        for i in range(args.warmup + args.steps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            hg = [B.Graph(*p) for p in pinned]
            xs = [B.Instance(hg[gi], a, t, nm, mi, out=host_outs[k]) for k, (gi, a, t, nm, mi) in enumerate(specs)]
            B.pr_solve_batch(xs, precision=precision, stream=sptr)
            for h in hg:
                h.close()
            t1 = time.perf_counter()
            if i >= args.warmup:
                et.append((t1 - t0) * 1000.0)
        e2e_ms = max_over_ranks(sum(et) / len(et), world)
        e2e = {"value": world * solves * 1000.0 / e2e_ms, "unit": "solves/s", "ms_per_step": e2e_ms,
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}
    # ---- CPU baseline: the oracle on the host cores, bounded sample
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline(graphs, specs, inst_iters, args.cpu_seconds)
    clocks = clk.summary()
    ratio, tsrc = kernel_traffic_ratio()
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
        "dtype": {"df64": "df64 (f32x2)", "mixed": "f32 -> df64", "fp64": "f64", "fp32": "f32"}[precision],
        "data": "synthetic (seeded generators; paper's SuiteSparse graphs unavailable)",
        "config": {"workload": desc, "instances": solves, "graphs": len(graphs),
                   "edges": total_edges, "parallelism": f"instance batches x{world} (one per rank, no collective)",
                   "l2": "inputs larger than L2" if inputs_large else "L2 flushed (256 MB write) between steps"},
        "iterations": inst_iters,
        "gteps_instances": edges_inst / (ms_step * 1e-3) / 1e9,
        "gteps_device": gteps_device,
        "roofline": {"bound": "hbm", "achieved": kernel_achieved, "peak": hbm, "unit": "GB/s",
                     "frac": kernel_achieved / hbm,
                     "traffic": (ratio * kernel_bytes) if ratio and precision == "df64" else None,
                     "traffic_source": tsrc if ratio and precision == "df64" else None,
                     "kernel": kernel_name, "avg_launch_us": avg_kernel_ms * 1e3,
                     "algorithmic_bytes_per_launch": kernel_bytes, "peak_source": peak_kind,
                     "pass": pass_roofline},
        "e2e": e2e,
        "plain_gpu": plain,
        "learned_start": learned,
        "sweep_report": sweep,
        "cpu_baseline": cpu,
        "clocks": clocks,
        "gpu_launches": launches,
    }
    if rank == 0:
        print(json.dumps(line))
    for d in dgs:
        d.close()


def oracle_sample(graphs, specs, budget_s, cores):
    """Time the CPU oracle on the workload within about budget_s seconds.

    Instances sharing (graph, alpha) are one trajectory read at several stopping
    rules (oracle.pagerank_taps). Trajectories are solved in workload order for
    real while the estimated cost fits the budget; the rest are costed as
    (iterations) x (measured time of one oracle update on that graph), with
    iterations from the first solved trajectory of the same graph when there
    is one, else Section 1's estimate round(log10 tau / log10 alpha)."""
    import numpy as np

    from oracle import oracle as orc
    t_upd = {}
    for gi, g in enumerate(graphs):
        r = np.full(g.n, 1.0 / g.n)
        t0 = time.perf_counter()
        r, _ = orc.step(g, 0.85, r, threads=cores)
        orc.norms(r, r)
        t_upd[gi] = time.perf_counter() - t0
    groups = {}
    for k, (gi, a, t, nm, mi) in enumerate(specs):
        groups.setdefault((gi, a), []).append(k)
    spent, solved, modeled = 0.0, 0, 0.0
    iters_seen = {}
    for (gi, a), ks in groups.items():
        taps = [(specs[k][2], specs[k][3], specs[k][4]) for k in ks]
        est = max(min(mi, orc.estimate_iterations(t, a) if 0 < a < 1 else mi) for t, nm, mi in taps)
        if spent + t_upd[gi] * est <= budget_s:
            t0 = time.perf_counter()
            res = orc.pagerank_taps(graphs[gi], a, taps, threads=cores)
            spent += time.perf_counter() - t0
            solved += len(ks)
            iters_seen[(gi, a)] = [x.iters for x in res]
        else:
            for t, nm, mi in taps:
                it = min(mi, orc.estimate_iterations(t, a)) if 0 < a < 1 else mi
                modeled += t_upd[gi] * max(it, 1)
    total_time = spent + modeled
    value = len(specs) / total_time
    kind = "measured" if modeled == 0 else ("mixed" if solved else "extrapolated")
    sample = (f"{solved} of {len(specs)} instances solved by the oracle ({spent:.1f}s); "
              f"{len(specs) - solved} costed as estimated iterations x measured update time ({kind})")
    return {"value": value, "unit": "solves/s", "cores": cores, "kind": "oracle", "sample": sample}


def cpu_baseline(graphs, specs, inst_iters, seconds):
    from oracle import oracle as orc
    return oracle_sample(graphs, specs, seconds, orc.default_threads())


# --------------------------------------------------------------------------- reference arm

def run_reference(args, world, rank):
    """The oracle, as it stands, on the host cores; rank 0 only."""
    if rank != 0:
        return
    from oracle import oracle as orc
    from paper_2108_02997_gb300 import graphgen as gg
    orc.build()
    graphs, specs, precision, desc = make_workload(args.workload, gg)
    cores = orc.default_threads()
    budget = max(5.0, args.cpu_seconds)
    for _ in range(args.warmup):
        oracle_sample(graphs, specs[:1], 1.0, cores)
    vals = [oracle_sample(graphs, specs, budget, cores) for _ in range(args.steps)]
    v = statistics.mean(x["value"] for x in vals)
    line = {"metric": METRIC, "value": v, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": len(specs) / v * 1000.0, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": desc, "instances": len(specs), "graphs": len(graphs)},
            "impl": "reference",
            "cpu_baseline": {"kind": "oracle", "cores": cores, "value": v, "unit": "solves/s",
                             "sample": vals[-1]["sample"]},
            "e2e": {"value": v, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="rmat22",
                    choices=["rmat22", "rmat21", "sweep330", "sweep330warm", "multi64", "rmat24mixed", "learned",
                             "road24"])
    ap.add_argument("--loop", default="graph", choices=["graph", "host"],
                    help="device loop of the timed solves (host: one launch per iteration)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-plain", action="store_true", help="skip the plain per-instance GPU solver comparison")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
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
