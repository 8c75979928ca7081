"""Benchmark of the coupled LB-IB time step on GB300.

Workload (default): the 4096^2 FP32 tissue -- periodic, tau 0.6, 9,801
64-vertex cells of radius 15 on a jittered 100x100 grid, one D2Q5 species
with sources in a seeded 10% of the cells -- the largest configuration that
fits one GPU; one benchmark step = one coupled time step (labels, vertex
forces, spreading, fused lattice update, interpolation and vertex update).
The 1024^2 walled tissue with two species is the named workload c2.

Printed JSON line (rank 0):
  value       MLUPS = lattice nodes x steps / device time of the K timed steps
              (all ranks' nodes for N > 1, max time over ranks), inputs
              resident in HBM, the steps advanced by lbib_advance (ordinary
              steps replayed from the library's CUDA graphs; the output
              fields of the last step are not written inside the timed
              region);
  roofline    the lattice-update kernel: algorithmic population bytes per
              launch / its mean launch time (CUDA events on the context
              stream, from a profiled pass of the same steps) against the
              measured HBM copy peak; traffic (ncu DRAM bytes per launch,
              recorded for the current kernel source) with its own fraction
              of the peak beside it;
  e2e         MLUPS through the public C ABI from host buffers: every step
              uploads the per-cell pressure and source flags from pinned host
              memory, advances one step and reads the vertex positions and
              cell areas back to pinned host memory (the lattice fields stay
              on the device), the readback of each step running beside the
              next step (lbib_get_cells_async, waited on once the next step
              is enqueued; every readback ends inside the timed region);
  cpu_baseline the FP64 oracle on the host cores on a bounded sample.

Other workloads (--workload): c2 (the 1024^2 tissue, no-slip walls in y,
tau 0.8, 400 hexagonally packed 100-vertex cells, two reacting species);
c3-fp16, c3-fp64 (the default tissue with FP16-shifted / FP64 storage);
c3-precision (that tissue with all three storages, errors against FP64);
nn (the neural operator's training step and forward pass, TFLOP/s);
c4 (64 independent tissues in one persistent launch); c5 (the learned warm
start of the steady morphogen solve, warm vs cold); turing (the
Schnakenberg system on a static cellular domain of 1024^2, receptor confined
to its cell); c2-junctions (the default tissue with cell junctions renewed
every 10 steps); c2-growth (the default tissue growing under the area
controller, pressure nodes along the walls); case1 / case2 (the mass-source
growth studies: a cell grown by a point source / doubling its area under a
uniform source, at four refinements); case4 (the immersed-
boundary leakage study: area loss under constant membrane tension at four
refinements and its order of convergence).

--impl reference times the FP64 oracle (the reference arm of this build)
on the same workload and metric.
"""
from __future__ import annotations

import argparse
import ctypes
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import lbib_inputs as li  # noqa: E402

METRIC = "coupled LB-IB MLUPS and % HBM peak; time-to-steady morphogen (warm vs cold) at resid 1e-6"
UNIT = "MLUPS"
L2_BYTES = 129 * 1024 * 1024


def alg_bytes_per_node(precision: str, n_species: int) -> int:
    """Populations read once and written once per node and step."""
    b = {"fp64": 8, "fp32": 4, "fp16": 2}[precision]
    return 2 * 9 * b + 2 * 5 * n_species * b


def workload(name: str, c3_n: int = 4096):
    if name == "c2":
        return li.config2(), "fp32"
    if name == "c3-fp32":
        return li.config3(n=c3_n), "fp32"
    if name == "c3-fp16":
        return li.config3(n=c3_n), "fp16"
    if name == "c3-fp64":
        return li.config3(n=c3_n), "fp64"
    if name == "c4":
        return li.config4(), "fp32"
    if name == "turing":
        return li.turing(), "fp32"
    if name == "c2-junctions":
        return li.config2_junctions(), "fp32"
    if name == "c2-growth":
        return li.config2_growth(), "fp32"
    raise SystemExit(f"unknown workload {name}")


def prepare(sim, w):
    """Workload extras beyond the cells: static domains, initial species."""
    if getattr(w, "domains", None) is not None:
        sim.set_domains(w.domains)
    if getattr(w, "phi0", None) is not None:
        for s in range(w.params.n_species):
            sim.set_species(s, w.phi0[s])
    if getattr(w, "mass_rate", None) is not None or getattr(w, "target_area", None) is not None:
        sim.set_mass_sources(getattr(w, "mass_rate", None), getattr(w, "target_area", None))
    if getattr(w, "pressure_mask", None) is not None:
        sim.set_pressure_nodes(w.pressure_mask)


def workload_config(w, precision, extra=None):
    p = w.params
    cfg = {
        "workload": w.name,
        "lattice": [p.nx, p.ny],
        "bc_y": "walls" if p.bc_y else "periodic",
        "tau": p.tau,
        "cells": w.tissue.n_cells,
        "vertices": w.tissue.n_vertices,
        "species": p.n_species,
        "storage": precision,
        "vertex_precision": "fp64",
        "seed": w.seed,
    }
    if extra:
        cfg.update(extra)
    return cfg


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi samples of one GPU during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int, period_ms: int = 100):
        self.rows = []
        self.proc = None
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(gpu_index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", str(period_ms)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[5 + i] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


# ------------------------------------------------------------------ helpers
def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def lattice_kernel_hash() -> str:
    h = hashlib.sha256()
    for f in ("lattice.cu", "lattice_kernel.cuh", "lattice_node.cuh", "lbib_internal.cuh"):
        h.update(open(os.path.join(ROOT, "paper_1503_06726_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def ensemble_kernel_hash() -> str:
    h = hashlib.sha256()
    for f in ("ensemble.cu", "ib_cell.cuh", "lattice_node.cuh", "lbib_internal.cuh"):
        h.update(open(os.path.join(ROOT, "paper_1503_06726_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def recorded_traffic(workload_name: str, key: str = "dram_bytes_per_launch", sha=None):
    """DRAM bytes per launch (or per step) from the committed ncu summary, if
    it was taken on the current kernel source."""
    path = os.path.join(ROOT, "profiles", "lattice_kernel_traffic.json")
    try:
        d = json.load(open(path))
        e = d.get(workload_name)
        if e and e.get("kernel_sha") == (sha or lattice_kernel_hash()):
            return float(e[key])
    except Exception:
        pass
    return None


def fp64_flops_per_node(n_species: int, forcing: int) -> int:
    """FP64 operations of the collision of one node as written (add, sub,
    mul and reciprocal count 1, fma 2): force 2, moments 26, common even
    part 18, four direction pairs 72, each species 25 + 2 S; the paper's
    forcing term instead of Guo's drops 4 + 5 + 4 x 3."""
    f = 2 + 26 + 18 + 72 + n_species * (25 + 2 * n_species)
    if forcing == 1:
        f -= 4 + 5 + 12
    return f


def max_over_ranks(x: float, dist, device) -> float:
    """The largest x over the ranks of the process group (x itself without
    one): every rank's time counts, the job ends with its slowest rank."""
    if not dist:
        return float(x)
    import torch
    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_mlups(world: int, nodes: int, steps: int, seconds: float) -> float:
    """Whole-job throughput of `world` independent replicas of `nodes`
    lattice nodes each, all advanced `steps` steps in `seconds` (the max over
    ranks)."""
    return world * nodes * steps / seconds / 1e6


def oracle_sample(w, target_s: float, max_steps: int, threads: int | None = None):
    """Time the FP64 oracle on the workload: whole coupled steps until
    target_s of CPU time or max_steps.  Returns (mlups, steps, seconds, cores)."""
    import oracle
    oracle.build()
    if threads:
        oracle.set_threads(threads)
    cores = oracle.max_threads()
    p, T = w.params, w.tissue
    f, g = oracle.equilibrium_state(p)
    phi0, dom = getattr(w, "phi0", None), getattr(w, "domains", None)
    if phi0 is not None:  # species at equilibrium of the initial fields
        W5 = [1 / 3] + [1 / 6] * 4
        g = np.concatenate([np.stack([W5[q] * phi0[s] for q in range(5)])
                            for s in range(p.n_species)])
    xy = T.xy.copy()
    # the oracle renews junction partners at the start of every call: call it
    # once per renewal period so that it renews exactly as often as the GPU
    chunk = p.junction_period if (p.junction_period > 0 and T.n_cells > 0) else 1
    steps, t0 = 0, time.perf_counter()
    while steps < max_steps:
        r = oracle.run(p, T, chunk, f=f, g=g, xy=xy, dom=dom,
                       mass_rate=getattr(w, "mass_rate", None),
                       target_area=getattr(w, "target_area", None),
                       pmask=getattr(w, "pressure_mask", None))
        f, g, xy = r.f, r.g, r.xy
        steps += chunk
        if time.perf_counter() - t0 >= target_s:
            break
    dt = time.perf_counter() - t0
    return p.nx * p.ny * steps / dt / 1e6, steps, dt, cores


# ------------------------------------------------------------------ arms
def run_ensemble(args, rank, world, dist):
    """64 independent tissues of uneven sizes advanced together, by one
    persistent cooperative launch per step call or by the split schedule of
    two launches per step (either replayed from a CUDA graph; the autotuner
    picks the schedule unless --ens-schedule names one)."""
    import torch
    from paper_1503_06726_gb300 import lbib

    lbib.load()
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    ws = li.config4()
    N = sum(w.params.nx * w.params.ny for w in ws)
    ens = lbib.Ensemble([w.params for w in ws], [w.tissue for w in ws], device=dev)
    tune = ens.tune_cached(f"c4-{len(ws)}-{N}", trial_steps=10)
    forced = {"persistent": lbib.LBIB_ENS_PERSISTENT, "split": lbib.LBIB_ENS_SPLIT,
              "split_wide": lbib.LBIB_ENS_SPLIT_WIDE}.get(args.ens_schedule)
    if forced is not None:
        ens.schedule(forced)
    sched = ens.schedule()
    split = sched != lbib.LBIB_ENS_PERSISTENT
    warmup = max(args.warmup, 4)
    ens.step(warmup)
    ens.status()
    torch.cuda.synchronize()
    stream = ens.stream
    clocks = ClockSampler(dev.index if dev.index is not None else 0) if rank == 0 else None
    time.sleep(0.3 if clocks else 0)
    if dist:
        dist.barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    ens.step(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ens.status()
    if dist:
        dist.barrier()
    ms = e0.elapsed_time(e1)
    clk = clocks.stop() if clocks else None
    ms = max_over_ranks(ms, dist, dev)
    value = replica_mlups(world, N, args.steps, ms * 1e-3)
    bpn = alg_bytes_per_node("fp32", ws[0].params.n_species)
    achieved = bpn * N * args.steps / (ms * 1e-3) / 1e9
    peak, peak_kind = peaks()
    # end to end: per step, per-cell parameters of every tissue up from pinned
    # host memory, one ensemble step, cell areas of every tissue back
    L = lbib.load()
    vp = ctypes.c_void_p
    pins = []
    for w in ws:
        pp = torch.empty(w.tissue.n_cells, dtype=torch.float64).pin_memory()
        pp.numpy()[:] = w.tissue.pressure
        aa = torch.empty(w.tissue.n_cells, dtype=torch.float64).pin_memory()
        pins.append((pp, aa))
    e2e_steps = max(1, min(args.e2e_steps, 100))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        for t, (pp, aa) in enumerate(pins):
            rc = L.lbib_set_cell_params(ens.ctx[t], vp(pp.data_ptr()), None)
            if rc:
                raise RuntimeError(lbib.lbib_last_error(ens.ctx[t]))
        ens.step(1)
        for t, (pp, aa) in enumerate(pins):
            rc = L.lbib_get_fields(ens.ctx[t], lbib.LBIB_AREA, None, None, None, None, None,
                                   vp(aa.data_ptr()), None, None, None)
            if rc:
                raise RuntimeError(lbib.lbib_last_error(ens.ctx[t]))
    t_e2e = max_over_ranks(time.perf_counter() - t0, dist, dev)
    cells = sum(w.tissue.n_cells for w in ws)
    e2e = {"value": replica_mlups(world, N, e2e_steps, t_e2e), "unit": UNIT,
           "h2d_bytes_per_step": cells * 8, "d2h_bytes_per_step": cells * 8,
           "steps": e2e_steps,
           "api": "per tissue lbib_set_cell_params, lbib_ensemble_step(1), per tissue "
                  "lbib_get_fields(AREA)"}
    info = ens.config()
    ens.close()
    if rank != 0:
        return None
    return {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded tissue generator)",
        "config": {"workload": f"c4_ensemble_{len(ws)}_tissues", "nodes": N,
                   "sides": [w.params.nx for w in ws], "cells": cells,
                   "storage": "fp32", "vertex_precision": "fp64",
                   "l2": f"inputs larger than L2: {2 * bpn * N / 2**20:.0f} MiB of populations",
                   "launch": ("split schedule: one lattice launch over every tissue and one IB "
                              "launch over every cell per step, programmatic, one graph per "
                              "step call" + (" (wide lattice kernel)"
                                             if sched == lbib.LBIB_ENS_SPLIT_WIDE else "")
                              if split else "one persistent cooperative kernel per step call"),
                   "schedule": {0: "persistent", 1: "split", 2: "split_wide"}[sched],
                   "graph": info["graph"], "grid": None if split else info["grid"],
                   "tuned": tune},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak,
                     "traffic": (lambda t: t * args.steps if t is not None else None)(
                         recorded_traffic("c4-split-per-step" if split else "c4-per-step",
                                          "dram_bytes_per_step", ensemble_kernel_hash())),
                     "kernel": ("ens_lattice_kernel + ens_ib_kernel (whole steps: every launch "
                                "of the step call)" if split else
                                "ensemble_kernel (whole persistent launch: lattice + IB phases)"),
                     "alg_bytes_per_node": bpn, "peak_kind": f"{peak_kind} hbm_gbs (copy)"},
        "e2e": e2e, "gpu_launches": 2 * args.steps + 1 if split else 1, "clocks": clk,
        "cpu_baseline": None,
    }


def warm_start_sample(args, dev):
    """The second half of the metric at a bounded size: train the neural
    operator on --ws-train cold-solved 256^2 tissues for --ws-epochs epochs and
    compare warm vs cold time to r <= 1e-6 on --ws-test held-out seeds.  The
    full-size run (20k pairs, 1k seeds) is --workload c5."""
    import torch
    from paper_1503_06726_gb300 import lbib, warmstart as wsm
    H = 256
    t0 = time.perf_counter()
    data = wsm.make_dataset([li.steady_tissue(s, n=H) for s in range(5, 5 + args.ws_train)],
                            H, H, batch=256)
    net = lbib.NeuralOperator(16, H, H, device=dev)
    layers = net.layers()
    shapes = [(f"layer{i}", ci, co) for i, (ci, co) in enumerate(layers[:-1])]
    shapes.append(("out",) + tuple(layers[-1]))
    net.set_params(li.nop_init_params(5, shapes))
    losses = wsm.train(net, data, epochs=args.ws_epochs, batch=16, lr=1e-3, lr_end=5e-5)
    del data
    rows = wsm.evaluate(net, [li.steady_tissue(s, n=H) for s in range(1000, 1000 + args.ws_test)],
                        H, H)
    net.close()
    torch.cuda.synchronize()
    summ = wsm.summarize(rows)
    summ.update({"train_pairs": args.ws_train, "epochs": args.ws_epochs,
                 "loss_first_epoch": losses[0], "loss_last_epoch": losses[-1],
                 "seconds": time.perf_counter() - t0,
                 "note": "bounded sample; --workload c5 is the full 20k-pair / 1k-seed run"})
    return summ


def run_warmstart(args, rank, world, dist):
    """256^2 steady morphogen solves: the neural operator is trained on pairs
    the LB solver generates (cold solves of --c5-train random tissues), then
    on --c5-test held-out seeds each tissue is solved to r <= 1e-6 from a cold
    start and from the network's prediction (inference included)."""
    import torch
    from paper_1503_06726_gb300 import lbib, warmstart as wsm

    lbib.load()
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    H = 256
    t0 = time.perf_counter()
    train_items = [li.steady_tissue(s, n=H) for s in range(5, 5 + args.c5_train)]
    data = wsm.make_dataset(train_items, H, H, batch=256)
    t_data = time.perf_counter() - t0
    net = lbib.NeuralOperator(args.c5_batch, H, H, device=dev)
    layers = net.layers()
    shapes = [(f"layer{i}", ci, co) for i, (ci, co) in enumerate(layers[:-1])]
    shapes.append(("out",) + tuple(layers[-1]))
    net.set_params(li.nop_init_params(5, shapes))
    n_params = net.n_params
    t0 = time.perf_counter()
    losses = wsm.train(net, data, epochs=args.c5_epochs, batch=args.c5_batch, lr=1e-3,
                       lr_end=5e-5)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    del data
    test_items = [li.steady_tissue(s, n=H) for s in range(1000, 1000 + args.c5_test)]
    rows = wsm.evaluate(net, test_items, H, H)
    summ = wsm.summarize(rows)
    n_train_steps = args.c5_epochs * (args.c5_train // args.c5_batch)
    train_flop = 3 * 9.7e9 * args.c5_batch * n_train_steps
    net.close()
    if rank != 0:
        return None
    return {
        "metric": "time-to-steady morphogen (warm vs cold) at resid 1e-6",
        "value": summ["warm_ms_mean"], "unit": "ms per tissue (warm start, inference included)",
        "higher_is_better": False, "n_gpus": world, "steps": summ["n"], "warmup": 0,
        "ms_per_step": summ["warm_ms_mean"], "scaling": "weak", "vs_baseline": None,
        "dtype": "bf16 network, f32 relaxation", "data": "synthetic (seeded tissue generator)",
        "config": {"workload": "c5_warm_start_256x256", "train_pairs": args.c5_train,
                   "test_seeds": args.c5_test, "epochs": args.c5_epochs,
                   "batch": args.c5_batch, "params": n_params},
        "warm_vs_cold": summ,
        "training": {"data_seconds": t_data, "train_seconds": t_train,
                     "loss_first_epoch": losses[0], "loss_last_epoch": losses[-1],
                     "approx_tflops": train_flop / t_train / 1e12},
        "cpu_baseline": None,
    }


def nn_conv_flops(layers, H, W, N):
    """Algorithmic FLOPs of the U-Net's 3x3 convolutions per sample batch:
    forward 2 * 9 * Ci * Co * pixels per layer (canonical channels), the
    data gradient the same except for the input layer, the weight gradient
    the same.  Layers in the network's order: encoder levels 0..5 (two each),
    decoder levels 4..0 (two each), the output layer at level 0."""
    levels = [l for l in range(6) for _ in range(2)] + \
        [l for l in range(4, -1, -1) for _ in range(2)] + [0]
    fwd = [2 * 9 * ci * co * (H >> l) * (W >> l) * N for (ci, co), l in zip(layers, levels)]
    return sum(fwd), sum(fwd) + sum(fwd[1:]) + sum(fwd)


def run_nn(args, rank, world, dist):
    """The neural operator alone: training steps (forward, loss, backward,
    Adam) and forward passes of the six-level U-Net on 256^2 batches of 16,
    inputs resident on the device, timed with CUDA events on the network's
    stream; throughput = the convolutions' algorithmic FLOPs per second
    against the measured BF16 tensor peak."""
    import torch
    from paper_1503_06726_gb300 import lbib

    lbib.load()
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    B, H = args.c5_batch, 256
    net = lbib.NeuralOperator(B, H, H, device=dev)
    layers = net.layers()
    shapes = [(f"layer{i}", ci, co) for i, (ci, co) in enumerate(layers[:-1])]
    shapes.append(("out",) + tuple(layers[-1]))
    net.set_params(li.nop_init_params(5, shapes))
    g = torch.Generator(device="cpu").manual_seed(3)
    mask = (torch.rand((B, H, H), generator=g) < 0.6).to(torch.uint8).to(dev)
    src = (torch.rand((B, H, H), generator=g) < 0.1).to(torch.uint8).to(dev)
    phi = torch.rand((B, H, H), generator=g).to(dev)
    D = np.full(B, 0.1)
    k = np.full(B, 1e-3)
    r = np.full(B, 1e-3)
    fwd_flop, train_flop = nn_conv_flops(layers, H, H, B)
    st = net.stream
    for _ in range(max(args.warmup, 3)):
        net.train_step(mask, src, D, k, r, phi, lr=1e-4)
    torch.cuda.synchronize()
    clocks = ClockSampler(dev.index if dev.index is not None else 0) if rank == 0 else None
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    n = max(1, args.steps)
    e0.record(st)
    for _ in range(n):
        net.train_step(mask, src, D, k, r, phi, lr=1e-4)
    e1.record(st)
    torch.cuda.synchronize()
    t_train = e0.elapsed_time(e1) / n
    out = torch.empty((B, H, H), dtype=torch.float32, device=dev)
    e0.record(st)
    for _ in range(n):
        net.forward(mask, src, D, k, r, out=out)
    e1.record(st)
    torch.cuda.synchronize()
    t_fwd = e0.elapsed_time(e1) / n
    clk = clocks.stop() if clocks else None
    net.close()
    if rank != 0:
        return None
    peak = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))).get("bf16_tflops", 1900.0)
    tf_train = train_flop / (t_train * 1e-3) / 1e12
    tf_fwd = fwd_flop / (t_fwd * 1e-3) / 1e12
    return {
        "metric": "neural-operator training throughput (3x3 convolutions)",
        "value": tf_train, "unit": "TFLOP/s", "higher_is_better": True, "n_gpus": world,
        "steps": n, "warmup": max(args.warmup, 3), "ms_per_step": t_train, "scaling": "weak",
        "vs_baseline": None, "dtype": "bf16 (fp32 accumulation)", "data": "synthetic",
        "config": {"workload": f"nn_unet_{H}x{H}_batch{B}", "params": net.n_params,
                   "layers": layers},
        "training_step_ms": t_train, "forward_ms": t_fwd,
        "roofline": {"bound": "tensor", "achieved": tf_train, "peak": peak, "unit": "TFLOP/s",
                     "frac": tf_train / peak, "forward_tflops": tf_fwd,
                     "forward_frac": tf_fwd / peak,
                     "alg_flop_per_step": train_flop, "alg_flop_per_forward": fwd_flop,
                     "peak_kind": "measured bf16_tflops (burst)",
                     "note": "whole steps: the numerator counts the convolutions only, the "
                             "time includes the elementwise layers and the host's input "
                             "staging of every call"},
        "clocks": clk, "cpu_baseline": None,
    }


def run_precision(args, rank, world, dist):
    """The 4096^2 precision sweep: the same tissue advanced --prec-steps
    steps with FP64, FP32 and FP16-shifted population storage; velocity,
    concentration and vertex errors of the FP32/FP16 runs against the FP64
    run (the FP64 GPU path matches the FP64 oracle to 1e-10), and the per-cell
    area drift of every run."""
    import torch
    from paper_1503_06726_gb300 import lbib

    lbib.load()
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    w = li.config3()
    p, T = w.params, w.tissue
    n = args.prec_steps
    which = lbib.LBIB_U | lbib.LBIB_PHI | lbib.LBIB_X | lbib.LBIB_AREA | lbib.LBIB_ID
    res, secs = {}, {}
    area0 = None
    for name, prec in (("fp64", lbib.LBIB_FP64), ("fp32", lbib.LBIB_FP32),
                       ("fp16", lbib.LBIB_FP16)):
        sim = lbib.Simulation(p, prec, T.n_vertices, T.n_cells, device=dev)
        sim.set_cells(T)
        if area0 is None:
            area0 = sim.fields(lbib.LBIB_AREA)["area"]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sim.step(n)
        torch.cuda.synchronize()
        secs[name] = time.perf_counter() - t0
        res[name] = sim.fields(which)
        sim.close()
        del sim
        torch.cuda.empty_cache()
    ref = res["fp64"]
    umax = max(np.abs(ref["ux"]).max(), np.abs(ref["uy"]).max())
    pmax = np.abs(ref["phi"]).max()
    # nodes at least three nodes from any membrane (uniform 7x7 label block):
    # away from the source cells' edges, whose source bits flip between runs
    # when a node centre lies within the vertex-position error of an edge
    lab = ref["id"]
    away = np.ones_like(lab, bool)
    for dy in range(-3, 4):
        for dx in range(-3, 4):
            away &= np.roll(np.roll(lab, dy, 0), dx, 1) == lab

    def errs(r):
        du = max(np.abs(r["ux"] - ref["ux"]).max(), np.abs(r["uy"] - ref["uy"]).max())
        dp = np.abs(r["phi"] - ref["phi"])[0]
        return {"u_rel_linf": float(du / umax),
                "phi_rel_linf": float(dp.max() / pmax),
                "phi_rel_linf_away_from_membranes": float(dp[away].max() / pmax),
                "labels_differ_at_end": int((r["id"] != ref["id"]).sum()),
                "x_abs_linf_lu": float(np.abs(r["xy"] - ref["xy"]).max()),
                "area_rel_linf_vs_fp64": float(np.abs(r["area"] - ref["area"]).max() /
                                               np.abs(ref["area"]).max())}

    # the same tissue scaled to 512^2, against the FP64 oracle itself (it
    # runs the 2000 steps in about a minute on the host cores)
    ws = li.config3(n=512)
    import oracle
    oracle.build()
    t0 = time.perf_counter()
    oref = oracle.run(ws.params, ws.tissue, n)
    osec = time.perf_counter() - t0
    oerr = {}
    for name, prec in (("fp32", lbib.LBIB_FP32), ("fp16", lbib.LBIB_FP16)):
        sim = lbib.Simulation(ws.params, prec, ws.tissue.n_vertices, ws.tissue.n_cells,
                              device=dev)
        sim.set_cells(ws.tissue)
        sim.step(n)
        r = sim.fields(which)
        sim.close()
        ou = max(np.abs(oref.ux).max(), np.abs(oref.uy).max())
        oerr[name] = {
            "u_rel_linf": float(max(np.abs(r["ux"] - oref.ux).max(),
                                    np.abs(r["uy"] - oref.uy).max()) / ou),
            "phi_rel_linf": float(np.abs(r["phi"] - oref.phi).max() / np.abs(oref.phi).max()),
            "x_abs_linf_lu": float(np.abs(r["xy"] - oref.xy).max())}

    def drift(r):
        d = (r["area"] - area0) / area0
        return {"mean": float(d.mean()), "max_abs": float(np.abs(d).max())}

    if rank != 0:
        return None
    return {
        "metric": "precision-path error vs FP64 storage after the stated steps",
        "value": errs(res["fp32"])["u_rel_linf"], "unit": "relative L-inf of u (FP32 storage)",
        "higher_is_better": False, "n_gpus": world, "steps": n, "warmup": 0,
        "ms_per_step": secs["fp32"] * 1e3 / n, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 arithmetic; f64/f32/f16-shifted storage",
        "data": "synthetic (seeded tissue generator)",
        "config": workload_config(w, "fp64/fp32/fp16"),
        "errors_vs_fp64": {"fp32": errs(res["fp32"]), "fp16": errs(res["fp16"])},
        "errors_vs_oracle_512sq": dict(oerr, workload=ws.name, steps=n,
                                       oracle_seconds=osec),
        "area_drift": {k: drift(v) for k, v in res.items()},
        "field_scale": {"u_max": float(umax), "phi_max": float(pmax)},
        "seconds": secs,
        "cpu_baseline": None,
    }


def run_case4(args, rank, world, dist):
    """The immersed-boundary leakage study (validation Case IV): relative area
    loss of a circular cell under constant membrane tension at four lattice
    refinements, and the observed order of convergence."""
    import math
    import torch
    from paper_1503_06726_gb300 import lbib

    lbib.load()
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    levels, nodes_steps, t_gpu = [], 0, 0.0
    for k in range(4):
        w = li.case4(k, args.case4_max_length)
        T = w.tissue
        sim = lbib.Simulation(w.params, lbib.LBIB_FP32, T.n_vertices, T.n_cells, device=dev)
        sim.set_cells(T)
        sim.step(1)
        a0 = float(sim.fields(lbib.LBIB_AREA)["area"][0])
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sim.step(w.n_steps - 1)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        a1 = float(sim.fields(lbib.LBIB_AREA)["area"][0])
        sim.close()
        nodes_steps += w.params.nx * w.params.ny * (w.n_steps - 1)
        t_gpu += dt
        levels.append({"lattice": w.params.nx, "diameter": 10 * 2 ** k, "vertices": T.n_vertices,
                       "steps": w.n_steps, "tension_lb": w.params.tension,
                       "area_loss_rel": (a0 - a1) / a0, "seconds": dt})
    loss = [lv["area_loss_rel"] for lv in levels]
    orders = [math.log2(loss[k] / loss[k + 1]) for k in range(3)]
    if rank != 0:
        return None
    return {
        "metric": "IB leakage: observed order of the relative area loss (validation Case IV)",
        "value": orders[-1], "unit": "order (two finest lattices)", "n_gpus": world,
        "steps": sum(lv["steps"] for lv in levels), "warmup": 1,
        "ms_per_step": None, "higher_is_better": None, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic (one circular cell, no random input)",
        "config": {"workload": "case4_dia10-80_lattice100-800", "max_length": args.case4_max_length,
                   "bc": "periodic (the study's outflow boundary is out of scope)"},
        "orders": orders, "levels": levels,
        "paper": {"order": "about 1", "two_finest": 0.9891},
        "mlups": nodes_steps / t_gpu / 1e6,
    }


def run_growth_study(args, rank, world, dist, case: int):
    """Validation Case I (point source at the cell centre, A(T) = A0 + q T)
    or Case II (uniform per-node source ln 2 / T, A(T) = 2 A0): relative area
    error at four lattice refinements and the observed order of convergence."""
    import math
    import torch
    from paper_1503_06726_gb300 import lbib

    lbib.load()
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    levels, nodes_steps, t_gpu = [], 0, 0.0
    for k in range(4):
        w = li.case1(k) if case == 1 else li.case2(k)
        T = w.tissue
        sim = lbib.Simulation(w.params, lbib.LBIB_FP32, T.n_vertices, T.n_cells, device=dev)
        sim.set_cells(T)
        if case == 1:
            sim.set_node_sources(w.node_source)
        else:
            sim.set_mass_sources(w.mass_rate)
        sim.set_pressure_nodes(w.pressure_mask)
        a0 = float(sim.fields(lbib.LBIB_AREA)["area"][0])
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sim.step(w.n_steps)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        a1 = float(sim.fields(lbib.LBIB_AREA)["area"][0])
        sim.close()
        nodes_steps += w.params.nx * w.params.ny * w.n_steps
        t_gpu += dt
        if case == 1:
            q = float(w.node_source.sum())
            expect = (a0 + q * w.n_steps) / a0
        else:
            q = float(w.mass_rate[0])
            expect = math.exp(q * w.n_steps)
        levels.append({"lattice": w.params.nx, "diameter": 10 * 2 ** k, "vertices": T.n_vertices,
                       "steps": w.n_steps, "source_lb": q, "area_ratio": a1 / a0,
                       "expected": expect, "area_err_rel": a1 / a0 / expect - 1.0,
                       "seconds": dt})
    err = [abs(lv["area_err_rel"]) for lv in levels]
    orders = [math.log2(err[k] / err[k + 1]) for k in range(3)]
    if rank != 0:
        return None
    what = ("point mass source" if case == 1 else "uniform mass source")
    paper = ({"order": "about 1 (text); fitted slope -1.80 (figure)", "fitted_slope": -1.80}
             if case == 1 else {"order": "about 1 (area, finer grids)", "fitted_slope": -0.99})
    return {
        "metric": f"{what} growth: observed order of the relative area error "
                  f"(validation Case {'I' if case == 1 else 'II'})",
        "value": orders[-1], "unit": "order (two finest lattices)", "n_gpus": world,
        "steps": sum(lv["steps"] for lv in levels), "warmup": 0,
        "ms_per_step": None, "higher_is_better": None, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic (one circular cell, no random input)",
        "config": {"workload": f"case{case}_dia10-80_lattice100-800",
                   "bc": "periodic with pressure nodes at rho0 on the seam (the study's outflow "
                         "boundary is out of scope)"},
        "orders": orders, "levels": levels, "paper": paper,
        "mlups": nodes_steps / t_gpu / 1e6,
    }


def run_gb300(args, rank, world, dist):
    if args.workload == "case4":
        return run_case4(args, rank, world, dist)
    if args.workload in ("case1", "case2"):
        return run_growth_study(args, rank, world, dist, int(args.workload[-1]))
    if args.workload == "c3-precision":
        return run_precision(args, rank, world, dist)
    if args.workload == "c4":
        return run_ensemble(args, rank, world, dist)
    if args.workload == "c5":
        return run_warmstart(args, rank, world, dist)
    if args.workload == "nn":
        return run_nn(args, rank, world, dist)
    import torch
    from paper_1503_06726_gb300 import lbib

    lbib.load()
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    w, prec = workload(args.workload, args.c3_n)
    p, T = w.params, w.tissue
    N = p.nx * p.ny
    sim = lbib.Simulation(p, lbib.PRECISIONS[prec], T.n_vertices, T.n_cells, device=dev)
    sim.set_cells(T)
    prepare(sim, w)
    # FP16 storage: nodes per lattice thread (the pair or the quad update
    # where the width allows it)
    npt = 1
    if prec == "fp16":
        sim.set_lattice_variant(args.fp16_npt)
        npt = args.fp16_npt or 2
        if p.nx % npt:
            npt = 2 if p.nx % 2 == 0 else 1
    stream = sim.stream
    # warm-up: 4 + 5 steps capture and instantiate the two-step graphs of
    # both buffer parities (ordinary and final chunks) before the timed region
    warmup = max(args.warmup, 9)
    sim.advance(4)
    sim.advance(5)
    if warmup > 9:
        sim.advance(warmup - 9)
    torch.cuda.synchronize()

    clocks = ClockSampler(dev.index if dev.index is not None else 0) if rank == 0 else None
    time.sleep(0.3 if clocks else 0)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    sim.advance(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ms = e0.elapsed_time(e1)
    clk = clocks.stop() if clocks else None
    ms = max_over_ranks(ms, dist, dev)
    ms_per_step = ms / args.steps
    value = replica_mlups(world, N, args.steps, ms * 1e-3)

    # profiled pass: the same steps, every launch bracketed by events
    n_prof = max(10, min(args.steps, 400))
    lat_ms, ib_ms = sim.step_profiled(n_prof)
    lat_avg = lat_ms / n_prof
    bpn = alg_bytes_per_node(prec, p.n_species)
    alg_bytes = bpn * N
    achieved = alg_bytes / (lat_avg * 1e-3) / 1e9
    peak, peak_kind = peaks()
    sh = sim.fields(lbib.LBIB_U)  # raises on non-finite state
    assert np.isfinite(sh["ux"]).all()

    # end-to-end through the C ABI with pinned host buffers
    e2e_steps = max(1, min(args.e2e_steps, args.steps))
    pin_p = torch.empty(T.n_cells, dtype=torch.float64).pin_memory()
    pin_s = torch.empty(T.n_cells, dtype=torch.uint8).pin_memory()
    pin_p.numpy()[:] = T.pressure
    pin_s.numpy()[:] = T.src_flag
    # two host buffers: step k's readback lands in one while the host reads
    # step k - 1's from the other
    outs = [(torch.empty((T.n_vertices, 2), dtype=torch.float64).pin_memory(),
             torch.empty(T.n_cells, dtype=torch.float64).pin_memory()) for _ in range(2)]
    L = lbib.load()
    vp = ctypes.c_void_p
    which = lbib.LBIB_X | lbib.LBIB_AREA
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    for k in range(e2e_steps):
        rc = L.lbib_set_cell_params(sim.ctx, vp(pin_p.data_ptr()), vp(pin_s.data_ptr()))
        # the step as the timed loop runs it (no output fields: the caller
        # reads back vertex positions and areas, which every step has)
        rc = rc or L.lbib_advance(sim.ctx, 1)
        # the previous step's positions and areas (their copy ran beside this
        # step's prep and lattice update), then this step's readback
        rc = rc or L.lbib_wait_readback(sim.ctx)
        xy_k, area_k = outs[k % 2]
        rc = rc or L.lbib_get_cells_async(sim.ctx, which, vp(xy_k.data_ptr()),
                                          vp(area_k.data_ptr()))
        if rc:
            raise RuntimeError(lbib.lbib_last_error(sim.ctx))
    if L.lbib_wait_readback(sim.ctx):
        raise RuntimeError(lbib.lbib_last_error(sim.ctx))
    t_e2e = max_over_ranks(time.perf_counter() - t0, dist, dev)
    assert np.isfinite(outs[(e2e_steps - 1) % 2][0].numpy()).all()
    e2e = {"value": replica_mlups(world, N, e2e_steps, t_e2e), "unit": UNIT,
           "h2d_bytes_per_step": T.n_cells * 9, "d2h_bytes_per_step": T.n_vertices * 16 + T.n_cells * 8,
           "steps": e2e_steps,
           "api": "lbib_set_cell_params + lbib_advance(1) + lbib_get_cells_async(X|AREA) per "
                  "step, each readback waited on (lbib_wait_readback) after the next step is "
                  "enqueued",
           "note": "per step the cells' pressures and source flags go up and the vertex "
                   "positions and cell areas come back; the lattice fields stay on the device"}
    sim.close()

    if rank != 0:
        return None
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        mlups, steps, dt, cores = oracle_sample(w, args.cpu_seconds, 60)
        cpu = {"value": mlups, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"{steps} coupled FP64 steps of {w.name} from rest ({dt:.1f} s)"}
    # both population buffers (= the algorithmic bytes of one launch) plus the
    # force, velocity and label planes
    ws = alg_bytes + N * (2 * 4 * (2 if prec == "fp64" else 1) * 2 + 4)
    warm = None
    if world == 1 and not args.no_warm_start:
        warm = warm_start_sample(args, dev)
    traffic = recorded_traffic(args.workload + ("-quad" if npt == 4 else ""))
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "traffic": traffic,
            "dram_frac": (traffic / (lat_avg * 1e-3) / 1e9 / peak) if traffic else None,
            "kernel": {4: "lattice_quad_kernel (four nodes per thread)",
                       2: "lattice_pair_kernel (two nodes per thread)"}.get(npt, "lattice_kernel"),
            "alg_bytes_per_launch": alg_bytes,
            "alg_bytes_per_node": bpn, "launch_ms": lat_avg,
            "peak_kind": f"{peak_kind} hbm_gbs (copy)",
            "ib_launch_ms": ib_ms / (n_prof + 1)}
    jp = p.junction_period if T.n_cells > 0 else 0
    if jp > 0:
        # with junctions the IB time per step is a move, a prep and the
        # partner renewal every jp steps
        roof.pop("ib_launch_ms")
        roof["ib_ms_per_step"] = ib_ms / n_prof
    if prec == "fp64":
        # GB300's FP64 rate, not HBM, bounds this kernel: report it against the
        # FP64 peak (nominal 1.25 TFLOP/s = 152 SMs x 2.07 GHz x 2 FP64 FMA per
        # SM per clock x 2), with the HBM figures kept beside it
        fpn = fp64_flops_per_node(p.n_species, p.forcing)
        gflops = fpn * N / (lat_avg * 1e-3) / 1e9
        roof = dict(roof, bound="alu", achieved=gflops, peak=1250.0, unit="GFLOP/s",
                    frac=gflops / 1250.0, alg_flops_per_node=fpn,
                    peak_kind="nominal FP64 (no measured FP64 peak on this pool)",
                    hbm={"achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak})
    launches = 2 * args.steps + 1
    if jp > 0:
        # lattice, move and prep per step (the first prep before the loop, none
        # after the last step), four kernels per renewal (count, scan, fill,
        # search), one renewal at every step count in [warmup, warmup + steps)
        # that is a multiple of jp
        renewals = len([n for n in range(warmup, warmup + args.steps) if n % jp == 0])
        launches = 3 * args.steps + 4 * renewals
    rec = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32" if prec != "fp64" else "f64",
        "data": "synthetic (seeded tissue generator)",
        "config": workload_config(w, prec, {
            "l2": f"inputs larger than L2: {ws / 2**20:.0f} MiB working set > 129 MiB L2, no flush",
            "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
            "graph": ("direct launches (steps with junctions are not graphed)" if jp > 0
                      else "two-step CUDA graph chunks")}),
        "roofline": roof,
        "e2e": e2e,
        "warm_start": warm,
        "gpu_launches": launches,
        "clocks": clk,
        "cpu_baseline": cpu,
    }
    return rec


def run_reference(args, rank, world):
    if rank != 0:
        return None
    w, prec = workload(args.workload, args.c3_n)
    p = w.params
    # bounded sample: at most a minute of whole coupled oracle steps
    max_steps = max(1, args.steps)
    _, wsteps, _, _ = oracle_sample(w, 1e9, max(1, min(args.warmup, 3)))
    mlups, steps, dt, cores = oracle_sample(w, args.ref_seconds, max_steps)
    return {
        "impl": "reference", "metric": METRIC, "value": mlups, "unit": UNIT, "n_gpus": world,
        "steps": steps, "warmup": wsteps, "ms_per_step": dt / steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded tissue generator)",
        "config": workload_config(w, "fp64", {"implementation": "FP64 CPU oracle (plain C)"}),
        "cpu_baseline": {"value": mlups, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{steps} coupled FP64 steps of {w.name} from rest "
                                   f"(bounded to {args.ref_seconds:.0f} s of {args.steps} asked)"},
        "e2e": {"value": mlups, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5000)
    ap.add_argument("--warmup", type=int, default=100)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="c3-fp32")
    ap.add_argument("--e2e-steps", type=int, default=500)
    ap.add_argument("--ens-schedule", default="tuned",
                    choices=["tuned", "persistent", "split", "split_wide"],
                    help="c4: the ensemble's schedule (tuned: the autotuner's choice)")
    ap.add_argument("--fp16-npt", type=int, default=0, choices=[0, 1, 2, 4],
                    help="FP16 storage: lattice nodes per thread (0: the library's choice)")
    ap.add_argument("--c3-n", type=int, default=4096,
                    help="side of the c3 tissue (4096: the configuration; smaller for profiling)")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--ref-seconds", type=float, default=60.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-warm-start", action="store_true")
    ap.add_argument("--ws-train", type=int, default=2000)
    ap.add_argument("--ws-epochs", type=int, default=4)
    ap.add_argument("--ws-test", type=int, default=64)
    ap.add_argument("--c5-train", type=int, default=20000)
    ap.add_argument("--c5-test", type=int, default=1000)
    ap.add_argument("--c5-epochs", type=int, default=8)
    ap.add_argument("--c5-batch", type=int, default=16)
    ap.add_argument("--prec-steps", type=int, default=2000)
    ap.add_argument("--case4-max-length", type=float, default=0.5)
    args = ap.parse_args()
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    dist = None
    if args.impl == "reference":
        rec = run_reference(args, rank, world)
    else:
        if world > 1:
            import torch
            import torch.distributed as tdist
            torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
            tdist.init_process_group("nccl")
            dist = tdist
        rec = run_gb300(args, rank, world, dist)
        if dist:
            dist.barrier()
            dist.destroy_process_group()
    if rec is not None:
        print(json.dumps(rec), flush=True)


if __name__ == "__main__":
    main()
