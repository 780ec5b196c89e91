"""Benchmark of the per-step vehicle update on GB300.

One benchmark step = one simulated day of the regional workload: a planar
road network at the paper's single-GPU scale (about 224k nodes / 548k
directed edges) with 2.82M trips (gravity OD from 1,500 zones, AM/PM
departure peaks, free-flow shortest-path routes), dt = 0.5 s, simulated from
step 0 until every trip has arrived, with network and trips resident in HBM.
The metric is vehicle-steps per second (sum over steps of the vehicles on the
network, divided by the time).

Printed as one JSON line by rank 0, with:
  roofline      the dominant kernel (step_p1) against the measured HBM copy
                bandwidth, from CUDA events around every launch in one extra
                day run with per-kernel timing on;
  cpu_baseline  the CPU oracle (single thread) on a bounded sample of the
                same workload;
  e2e           the same metric through the public API from host buffers
                (network and trip upload, the run, trip and link-statistics
                download inside the timed region);
  clocks        nvidia-smi samples taken during the timed region.

`--impl reference` times the CPU oracle on the bounded sample instead.
`--gpus N` under torchrun runs N independent replicas (one per GPU).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

BYTES_PER_VEH_STEP_P1 = 64  # 24 state read + 8 state write + 16 edge record + 16 lane-map window
DAY_STEPS = 172_800
# bounded CPU sample: the trips departing in a few minutes from 07:30 (five
# for the regional day, two for the 9.01M-trip day, about 10-30 s of oracle work)
SAMPLE_START = 7 * 7200 + 3600
SAMPLE_STEPS_BY_WORKLOAD = {"large": 240}


def sample_window(workload: str) -> tuple[int, int]:
    return SAMPLE_START, SAMPLE_START + SAMPLE_STEPS_BY_WORKLOAD.get(workload, 600)


def sample_label(workload: str) -> str:
    k0, k1 = sample_window(workload)
    clock = lambda k: f"{int(k * 0.5) // 3600:02d}:{int(k * 0.5) // 60 % 60:02d}"
    return f"{clock(k0)}-{clock(k1)}"
SAMPLE_STEPS = 1200


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--workload", default="regional",
                    choices=["regional", "regional-small", "grid", "large", "batch64", "assignment", "paths", "surrogate",
                             "onchip"])
    ap.add_argument("--repeats", type=int, default=1,
                    help="assignment workload: alternate the two arms this many times and report the spread")
    ap.add_argument("--iterations", type=int, default=40,
                    help="assignment workload: MSA iterations at most per arm (each stops at the 1%% gap)")
    ap.add_argument("--assignment-scale", default="paper", choices=["paper", "small", "tiny"],
                    help="assignment workload: the 2.82M-trip regional day (paper) or the reduced cases")
    ap.add_argument("--paths", default="gpu", choices=["gpu", "host"],
                    help="assignment workload: where the time-dependent shortest paths are searched")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--day-profile", type=int, default=0, metavar="STEPS",
                    help="time the day in windows of STEPS steps (CUDA-synchronised wall time per window, vehicles "
                         "on the network) and print one JSON line per window, then exit")
    ap.add_argument("--profile-window", type=int, default=0,
                    help="run to 08:00, then profile this many directly launched steps (for ncu) and exit")
    ap.add_argument("--no-sort", action="store_true",
                    help="compact the vehicle slots without sorting them by lane-map cell (LPSIM_F_NO_SORT)")
    return ap.parse_args()


def load_workload(name: str):
    import workloads as W
    if name == "regional":
        net, dem = W.regional_day(seed=2, n_trips=2_820_000)
        label = "regional-224k-nodes-2.82M-trips-24h"
    elif name == "large":
        net, dem = W.regional_day(seed=3, n_trips=9_010_000, scale="large")
        label = "regional-1M-nodes-9.01M-trips-24h"
    elif name == "regional-small":
        # the regional generator at reduced scale (the small case for full
        # profiler captures: a few hundred MB on the device)
        net, dem = W.assignment_case(scale="small")
        label = "regional-27k-nodes-340k-trips-24h"
    else:
        net, dem = W.grid_day(seed=1)
        label = "grid-8x8-2000-trips"
    return net, dem, label


def sample_workload(net, dem, workload: str = "regional"):
    """Bounded CPU sample of the same workload: the trips departing in a
    few-minute window of the morning peak, simulated for 10 minutes."""
    import workloads as W
    k0, k1 = sample_window(workload)
    keep = (dem["depart_step"] >= k0) & (dem["depart_step"] < k1)
    sub = W.subset_trips(dem, keep)
    sub["depart_step"] = (sub["depart_step"] - k0).astype(np.uint32)
    return sub


def run_oracle_sample(net, sub, params):
    import oracle as O
    o = O.Oracle(net, params)
    o.load_demand(sub)
    t0 = time.perf_counter()
    r = o.run(SAMPLE_STEPS)
    dt = time.perf_counter() - t0
    o.close()
    return r["veh_steps"], dt


class ClockSampler:
    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.lines = []
        self.proc = None

    def __enter__(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.gpu)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
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
            self.t.join(timeout=2)

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
            except ValueError:
                continue
            for nm, val in zip(names, f[4:8]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def ncu_traffic():
    """DRAM bytes per launch of step_p1 from the committed ncu summary, if it
    was taken on the current kernel source."""
    import hashlib
    summ = os.path.join(ROOT, "profiles", "step_p1_regional_peak.json")
    src = os.path.join(ROOT, "paper_2406_08496_gb300", "csrc", "step_kernels.cu")
    if not os.path.exists(summ):
        return None
    with open(summ) as f:
        d = json.load(f)
    with open(src, "rb") as f:
        h = hashlib.sha1(f.read()).hexdigest()[:12]
    if d.get("source_sha1") != h:
        return None
    return d


def l2_note(net, dem) -> str:
    """What the timed region reads, against the 129 MB L2: the route array
    and the three rotating lane maps (each lane row padded to 16 bytes)."""
    cells = np.maximum(1, np.ceil(np.asarray(net["edge_len"], np.float64))).astype(np.int64)
    rows = ((cells + 15) // 16 * 16) * np.asarray(net["edge_lanes"], np.int64)
    map_gb = float(rows.sum() + 16) / 1e9
    route_gb = float(np.asarray(dem["route_edges"]).size * 4) / 1e9
    return (f"inputs larger than L2 (129 MB): routes {route_gb:.2f} GB, lane maps 3 x {map_gb:.3f} GB; "
            "no flush between steps")


def whole_job(ms: float, units: float, dist, device: str):
    """The whole job over N ranks: the longest rank's timed span (max) and
    the units every rank processed (sum); value = units / span.  One rank
    (dist None) returns its own pair."""
    if dist is None:
        return float(ms), float(units)
    import torch
    t = torch.tensor([float(ms)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    v = torch.tensor([float(units)], device=device, dtype=torch.float64)
    dist.all_reduce(v, op=dist.ReduceOp.SUM)
    return float(t.item()), float(v.item())


def reference_arm(args, rank, world):
    if rank != 0:
        return
    net, dem, label = load_workload(args.workload)
    sub = sample_workload(net, dem, args.workload)
    params = dict(bin_steps=1800, n_bins=0)
    for _ in range(args.warmup):
        run_oracle_sample(net, sub, params)
    vs_tot, t_tot = 0, 0.0
    for _ in range(args.steps):
        vs, dt = run_oracle_sample(net, sub, params)
        vs_tot += vs
        t_tot += dt
    value = vs_tot / t_tot
    sample = (f"{len(sub['depart_step'])} trips departing {sample_label(args.workload)} of the {label} workload, "
              f"{SAMPLE_STEPS} steps from 07:30, full network")
    line = {"impl": "reference", "metric": "veh-steps/s", "value": value, "unit": "veh-steps/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_tot / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": label, "sample": sample},
            "cpu_baseline": {"value": value, "unit": "veh-steps/s", "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "veh-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def batch_arm(args, L, torch, rank, world, local, dist=None):
    """64 independent scenarios of uneven size (grid and planar networks of
    1k-50k nodes, 10k-400k trips, each with its own seed) advanced by one
    launch of each step kernel per step; the launch configuration comes from
    the autotuner.  One benchmark step = the whole 2-hour horizon of all
    scenarios."""
    import workloads as W
    sc = W.batch_scenarios(64, base_seed=100)
    nets = [n for n, _, _ in sc]
    dems = [d for _, d, _ in sc]
    seeds = [s for _, _, s in sc]
    params = dict(bin_steps=1800, n_bins=4)
    sim = L.BatchSimulation(nets, params)
    sim.load_demand(dems, seeds)
    tune = sim.autotune(1536)
    horizon = 4 * 3600 * 2  # 4 simulated hours: the 2-hour departure window plus the tail
    for _ in range(args.warmup):
        sim.reset()
        sim.run(horizon)
    stream = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    vs = 0
    launches0 = sim.counters()["launches"]
    def barrier():
        torch.cuda.synchronize()
        if dist:
            dist.barrier()

    with ClockSampler(local) as clk:
        barrier()
        ev0.record(stream)
        for _ in range(args.steps):
            sim.reset()
            r = sim.run(horizon)
            vs += r["veh_steps"]
        ev1.record(stream)
        barrier()
    ms, vs = whole_job(ev0.elapsed_time(ev1), vs, dist, "cuda")
    if rank != 0:
        return
    trips = int(sum(len(d["depart_step"]) for d in dems))
    out = {"metric": "veh-steps/s", "value": vs / (ms / 1e3), "unit": "veh-steps/s", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": "batch-64-scenarios", "scenarios": 64, "trips": trips,
                      "edges": int(sum(n["n_edges"] for n in nets)), "horizon_steps": horizon,
                      "parallelism": f"replicas x{world}", "tuned": tune},
           "clocks": clk.summary(), "gpu_launches": int(sim.counters()["launches"] - launches0)}
    print(json.dumps(out), flush=True)


def surrogate_rows(torch) -> int:
    """Rows per surrogate batch at the large scales: eight 128-row tiles per
    SM (155,648 on 152 SMs), so the fused forward's persistent CTAs each run
    four pairs of tiles and none idles while others finish a last tile."""
    n_sm = torch.cuda.get_device_properties(0).multi_processor_count
    return 128 * 8 * n_sm


def assignment_arm(args, L, torch):
    """Plain and surrogate-assisted MSA on the regional day (the 224k-node
    network and its 2.82M trips; --assignment-scale picks a reduced case),
    each run until the relative gap reaches 1% or for --iterations
    iterations; every gap is measured by a full simulation and both arms use
    the same routing code (--paths).  value = the surrogate arm's wall time to
    the 1% gap (null if not reached); both arms' times to 2%, 1.5% and 1%."""
    import workloads as W
    from paper_2406_08496_gb300.assignment import msa
    net, dem = W.assignment_case(scale=args.assignment_scale)
    iters = args.iterations
    res = {}
    runs = {"plain": [], "surrogate": []}
    for rep in range(max(1, args.repeats)):
        for mode in ("plain", "surrogate"):
            r = msa(net, dem, mode, iterations=iters, target_gap=0.01, paths=args.paths,
                    surrogate_batch=surrogate_rows(torch) if args.assignment_scale == "paper" else 8192)
            runs[mode].append(r)
    for mode in ("plain", "surrogate"):
        r = runs[mode][-1]
        hist = [(h["wall_s"], h["gap"]) for h in r["history"] if h["gap"] is not None]

        def hit(th):
            return next((t for t, g in hist if g <= th), None)
        sims = [h for h in r["history"] if h["kind"] == "simulation"]
        res[mode] = {"time_to_1pct_gap_s": hit(0.01), "time_to_1.5pct_gap_s": hit(0.015),
                     "time_to_2pct_gap_s": hit(0.02), "final_gap": r["final_gap"], "wall_s": r["wall_s"],
                     "iterations": len(r["history"]), "gaps": [round(g, 5) for _, g in hist],
                     "gap_wall_s": [round(t, 2) for t, _ in hist],
                     "sim_s_mean": float(np.mean([h["sim_s"] for h in sims])) if sims else None,
                     "paths_s_mean": float(np.mean([h["paths_s"] for h in sims])) if sims else None,
                     "train_s_mean": (float(np.mean([h["train_s"] for h in sims if "train_s" in h]))
                                      if any("train_s" in h for h in sims) else None),
                     "surrogate_iter_s_mean": (float(np.mean([h["iter_s"] for h in r["history"]
                                                              if h["kind"] == "surrogate"]))
                                               if any(h["kind"] == "surrogate" for h in r["history"]) else None),
                     "time_to_1pct_gap_s_runs": [x["time_to_target_s"] for x in runs[mode]]}
    trips = int(len(dem["depart_step"]))
    label = {"paper": "assignment-224k-nodes-2.82M-trips", "small": "assignment-27k-nodes-340k-trips",
             "tiny": "assignment-3k-nodes-30k-trips"}[args.assignment_scale]
    def median(v):
        v = [x for x in v if x is not None]
        return float(np.median(v)) if v else None
    out = {"metric": "time-to-1%-gap", "value": median(res["surrogate"]["time_to_1pct_gap_s_runs"]), "unit": "s",
           "higher_is_better": False, "n_gpus": 1, "steps": iters, "warmup": 0, "dtype": "f32+bf16",
           "data": "synthetic", "vs_baseline": None,
           "config": {"workload": label, "nodes": net["n_nodes"], "edges": net["n_edges"], "trips": trips,
                      "reroute_fraction": 0.1, "selection": "random", "paths": args.paths,
                      "full_simulation": "every iteration (plain), every 2nd (surrogate)"},
           "plain_time_to_1pct_gap_s": median(res["plain"]["time_to_1pct_gap_s_runs"]),
           "repeats": max(1, args.repeats), "arms": res}
    print(json.dumps(out), flush=True)


def paths_arm(args):
    """Time-dependent shortest paths of every trip of the assignment case
    (one tree per origin and 30-minute departure period) under the link
    times of one simulation of its free-flow routes, per pass: the GPU
    search (one warp per tree) or the host search (--paths host)."""
    import workloads as W
    import paper_2406_08496_gb300 as L
    from paper_2406_08496_gb300.assignment import Assignment
    net, dem = W.assignment_case(scale=args.assignment_scale)
    A = Assignment(net, dem, seed=0)
    sim = L.Simulation(net, dict(bin_steps=1800, n_bins=96))
    sim.load_demand(A.routes())
    sim.run(300_000)
    ls = sim.link_stats()
    sim.close()
    tt, _ = A.link_times(ls["tt_sum"], ls["tt_cnt"])
    search = A.shortest_paths_gpu if args.paths == "gpu" else A.shortest_paths
    for _ in range(args.warmup):
        search(tt, 1800, 3600)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        search(tt, 1800, 3600)
    dt = (time.perf_counter() - t0) / args.steps
    groups = len(np.unique(dem["orig"].astype(np.uint64) * 1000 + dem["depart_step"] // 3600))
    out = {"metric": "shortest-path pass", "value": dt, "unit": "s", "higher_is_better": False, "n_gpus": 1,
           "steps": args.steps, "warmup": args.warmup, "dtype": "u32 ms", "data": "synthetic", "vs_baseline": None,
           "config": {"workload": f"assignment-paths-{args.assignment_scale}", "nodes": net["n_nodes"],
                      "edges": net["n_edges"], "trips": int(len(dem["depart_step"])), "trees": int(groups),
                      "paths": args.paths, "period_steps": 3600}}
    print(json.dumps(out), flush=True)


def onchip_arm(args):
    """The lane maps on chip (the paper's shared-memory direction, Sec. 5):
    a 4x4 grid (48 two-lane 400 m links, 38 KB of lane map) whose five maps
    fit the light-load kernel's shared memory, 1,200 trips over 30 minutes
    run to completion in light-load chunks, timed with the maps in shared
    memory (LPSIM_F_SHARED_MAPS) and, alternately, in global memory; same
    results either way (tested).  value = vehicle-steps/s with the maps on
    chip."""
    import paper_2406_08496_gb300 as L
    import torch
    import workloads as W
    L.use_torch_allocator()
    st = torch.cuda.Stream()
    torch.cuda.set_stream(st)
    net = W.grid_network(4, 4)
    dem = W.route(net, W.uniform_demand(net, 1200, 5))
    base = dict(bin_steps=1800, n_bins=4)
    sims = {"shared": L.Simulation(net, dict(base, flags=8)), "global": L.Simulation(net, dict(base))}
    for s in sims.values():
        s.load_demand(dem)
    res = {k: [] for k in sims}
    veh = {}
    for rep in range(max(args.warmup, 1) + max(args.steps, 1)):
        for name, s in sims.items():
            s.reset()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(st)
            r = s.run(200_000)
            e1.record(st)
            torch.cuda.synchronize()
            veh[name] = (r["veh_steps"], r["steps"])
            if rep >= max(args.warmup, 1):
                res[name].append(e0.elapsed_time(e1))
    ms = {k: float(np.median(v)) for k, v in res.items()}
    out = {"metric": "veh-steps/s", "value": veh["shared"][0] / (ms["shared"] / 1e3), "unit": "veh-steps/s",
           "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms["shared"],
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": "grid-4x4-1200-trips-lane-maps-on-chip", "edges": int(net["n_edges"]),
                      "trips": 1200, "sim_steps": veh["shared"][1], "step": "the demand run to completion"},
           "global_maps": {"value": veh["global"][0] / (ms["global"] / 1e3), "ms_per_run": ms["global"]},
           "speedup_on_chip": ms["global"] / ms["shared"],
           "us_per_sim_step": {k: 1e3 * ms[k] / veh[k][1] for k in ms}}
    print(json.dumps(out), flush=True)


def surrogate_arm(args):
    """The surrogate MLP's tensor-core kernels on device-resident batches:
    the inference forward (one persistent kernel: three BF16 layers and the
    head, activations kept in shared and tensor memory) and a training
    forward + backward (one GEMM launch per layer and gradient, fused
    epilogues), as TFLOP/s against the measured BF16 peak."""
    import paper_2406_08496_gb300 as L
    with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
        peaks = json.load(f)
    import torch
    rows = surrogate_rows(torch)
    s = L.Surrogate(n_features=11, batch=rows, seed=0)
    t = s.time(max(args.steps, 10))
    # the method's own multiply-adds per row: 11 real inputs (the zero
    # padding of the input columns is not the method's work)
    mac_fwd = 11 * 256 + 256 * 256 * 2 + 256
    flop_fwd = 2.0 * rows * mac_fwd
    # training: the forward, the weight gradients (as many MACs as the forward)
    # and the input gradients of layers 3 and 2 (layer 1 needs none)
    flop_train = 2.0 * rows * (2 * mac_fwd + 2 * 256 * 256 + 256)
    fwd = flop_fwd / (t["forward_ms"] / 1e3) / 1e12
    trn = flop_train / (t["train_ms"] / 1e3) / 1e12
    peak = float(peaks["bf16_tflops"])
    out = {"metric": "surrogate forward TFLOP/s", "value": fwd, "unit": "TFLOP/s", "n_gpus": 1, "steps": args.steps,
           "warmup": 1, "ms_per_step": t["forward_ms"], "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
           "config": {"workload": f"surrogate-mlp-{rows}-rows", "layers": "64-256-256-256-1", "rows": rows},
           "roofline": {"bound": "tensor", "achieved": fwd, "peak": peak, "unit": "TFLOP/s", "frac": fwd / peak,
                        "traffic": None, "kernel": "mlp_forward_fused",
                        "peak_source": "MEASURED_PEAKS.json bf16_tflops (measured)"},
           "train": {"ms_per_batch": t["train_ms"], "tflops": trn, "frac": trn / peak}}
    print(json.dumps(out), flush=True)


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        reference_arm(args, rank, world)
        return

    import torch
    import paper_2406_08496_gb300 as L

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    L.build()
    L.use_torch_allocator()
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    if args.workload == "batch64":
        batch_arm(args, L, torch, rank, world, local, dist)
        if dist:
            dist.barrier()
            dist.destroy_process_group()
        return
    if args.workload == "assignment":
        assignment_arm(args, L, torch)
        return
    if args.workload == "paths":
        paths_arm(args)
        return
    if args.workload == "surrogate":
        surrogate_arm(args)
        return
    if args.workload == "onchip":
        onchip_arm(args)
        return

    net, dem, label = load_workload(args.workload)
    n_bins = 96 if args.workload != "grid" else 4
    params = dict(bin_steps=1800, n_bins=n_bins)
    if args.no_sort:
        params["flags"] = 1
    sim = L.Simulation(net, params)
    sim.load_demand(dem)

    if args.day_profile:
        sim.step(3840)  # warm-up: graph capture and caches
        torch.cuda.synchronize()
        sim.reset()
        dep = np.sort(dem["depart_step"])
        while True:
            c0 = sim.counters()
            t0 = time.perf_counter()
            sim.step(args.day_profile)
            torch.cuda.synchronize()
            ms = (time.perf_counter() - t0) * 1e3
            c1 = sim.counters()
            print(json.dumps({"k": c0["k"], "steps": args.day_profile, "ms": ms,
                              "us_per_step": ms * 1e3 / args.day_profile, "active_start": c0["active"],
                              "slots_start": c0["slots"],
                              "veh_steps_per_step": (c1["veh_steps"] - c0["veh_steps"]) / args.day_profile,
                              "departures_due": int(np.searchsorted(dep, c0["k"] + args.day_profile)) - c0["arrived"]}),
                  flush=True)
            if c1["arrived"] >= len(dep):
                return
    if args.profile_window:
        sim.step(8 * 7200)  # to 08:00
        torch.cuda.synchronize()
        torch.cuda.cudart().cudaProfilerStart()
        sim.step(args.profile_window)
        torch.cuda.synchronize()
        torch.cuda.cudart().cudaProfilerStop()
        c = sim.counters()
        print(json.dumps({"profile_window": args.profile_window, "k": c["k"], "active": c["active"]}))
        return

    def day():
        sim.reset()
        return sim.run(DAY_STEPS + 100_000)

    for _ in range(args.warmup):
        day()

    def barrier():
        torch.cuda.synchronize()
        if dist:
            dist.barrier()

    launches0 = sim.counters()["launches"]
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    veh_steps = 0
    steps_per_day = []
    with ClockSampler(local) as clk:
        barrier()
        ev0.record(stream)
        for _ in range(args.steps):
            r = day()
            veh_steps += r["veh_steps"]
            steps_per_day.append(r["steps"])
        ev1.record(stream)
        barrier()
    ms = ev0.elapsed_time(ev1)
    launches = sim.counters()["launches"] - launches0
    t_max, vs_all = whole_job(ms, veh_steps, dist, "cuda")
    value = vs_all / (t_max / 1e3)

    out = None
    if rank == 0:
        # roofline of the dominant kernel: one more day with the kernels
        # stamping their own device spans (graphs, programmatic dependent
        # launch and light-load chunks as in the timed days), bracketed by
        # CUDA events on the library's stream
        sim.set_kernel_timing(True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        rr = day()
        e1.record(stream)
        torch.cuda.synchronize()
        day_ms = e0.elapsed_time(e1)
        kt = sim.kernel_times()
        sim.set_kernel_timing(False)
        p1 = kt["step_p1"]
        if p1["ms"] <= 0 or p1["launches"] == 0:
            raise RuntimeError(f"no step_p1 launch was timed: {kt}")
        achieved = BYTES_PER_VEH_STEP_P1 * p1["veh_steps"] / (p1["ms"] / 1e3) / 1e9
        peak, peak_src = measured_peaks()
        tr = ncu_traffic()
        roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                    # ncu DRAM bytes per vehicle-step of a morning-peak launch, scaled to this
                    # run's average launch (traffic grows with the vehicles processed)
                    "traffic": (tr["dram_bytes_per_veh_step"] * p1["veh_steps"] / max(1, p1["launches"])
                                if tr else None),
                    "kernel": "step_p1", "bytes_per_veh_step": BYTES_PER_VEH_STEP_P1,
                    "avg_launch_us": p1["ms"] * 1e3 / max(1, p1["launches"]),
                    "avg_veh_per_launch": p1["veh_steps"] / max(1, p1["launches"]),
                    "launches": p1["launches"], "veh_steps": p1["veh_steps"],
                    "timing": "device spans stamped by the kernels (first block start to last block end, "
                              "%globaltimer) over one extra day run as timed; CUDA events around that day",
                    "day_ms_events": day_ms,
                    "kernel_ms": {k: v["ms"] for k, v in kt.items()},
                    "kernel_launches": {k: v["launches"] for k, v in kt.items()},
                    "kernel_share_of_day": {k: v["ms"] / day_ms for k, v in kt.items()},
                    "peak_source": f"MEASURED_PEAKS.json hbm_gbs ({peak_src})",
                    "traffic_source": ("profiles/step_p1_regional_peak.json: " + tr["captured_launch"]) if tr else
                    "stale or missing ncu summary"}
        # the same at the morning peak (the hour the roofline target is about):
        # the graph chunk that holds 08:00
        peak_window = None
        if args.workload in ("regional", "large"):
            cw = int(L.DEFAULT_PARAMS["chunk_steps"])
            kw0 = (8 * 7200) // cw * cw

            def clock(k):
                sec = int(k * 0.5)
                return f"{sec // 3600:02d}:{sec // 60 % 60:02d}:{sec % 60:02d}"
            sim.reset()
            sim.step(kw0)
            sim.set_kernel_timing(True)
            torch.cuda.synchronize()
            e0.record(stream)
            sim.step(cw)
            e1.record(stream)
            torch.cuda.synchronize()
            win_ms = e0.elapsed_time(e1)
            kw = sim.kernel_times()
            sim.set_kernel_timing(False)
            pw = kw["step_p1"]
            if pw["ms"] > 0 and pw["launches"]:
                ach = BYTES_PER_VEH_STEP_P1 * pw["veh_steps"] / (pw["ms"] / 1e3) / 1e9
                per_launch_s = pw["ms"] / 1e3 / pw["launches"]
                dram = tr["dram_bytes_per_veh_step"] * pw["veh_steps"] / pw["launches"] if tr else None
                peak_window = {"window": f"steps {kw0:,}-{kw0 + cw - 1:,} ({clock(kw0)}-{clock(kw0 + cw)})",
                               "achieved": ach, "frac": ach / peak, "unit": "GB/s",
                               "avg_launch_us": per_launch_s * 1e6,
                               "avg_veh_per_launch": pw["veh_steps"] / pw["launches"],
                               "window_ms_events": win_ms,
                               "kernel_share_of_window": {k: v["ms"] / win_ms for k, v in kw.items()},
                               "dram_gbs": dram / per_launch_s / 1e9 if dram else None,
                               "dram_frac": dram / per_launch_s / 1e9 / peak if dram else None,
                               "dram_source": "ncu DRAM bytes per vehicle-step of step_p1 launches at 08:00 "
                                              "(profiles/step_p1_regional_peak.json) x this window's vehicles "
                                              "per launch / live span"}
            roofline["peak_window"] = peak_window
        cpu = None
        if not args.no_cpu_baseline and world == 1:
            sub = sample_workload(net, dem, args.workload)
            vs, dt = run_oracle_sample(net, sub, dict(bin_steps=1800, n_bins=0))
            cpu = {"value": vs / dt, "unit": "veh-steps/s", "cores": 1, "kind": "oracle",
                   "sample": f"{len(sub['depart_step'])} trips departing {sample_label(args.workload)} of the same day, "
                             f"{SAMPLE_STEPS} steps from 07:30 on the full network ({vs} veh-steps, {dt:.1f} s)",
                   "host_cpus": os.cpu_count()}
        e2e = None
        if not args.no_e2e:
            e2e = end_to_end(L, torch, net, dem, params)
        clocks = clk.summary()
        out = {"metric": "veh-steps/s", "value": value, "unit": "veh-steps/s", "n_gpus": world,
               "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_max / args.steps,
               "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
               "data": "synthetic",
               "config": {"workload": label, "nodes": net["n_nodes"], "edges": net["n_edges"],
                          "trips": int(len(dem["depart_step"])), "dt_s": 0.5,
                          "sim_steps_per_day": int(np.mean(steps_per_day)),
                          "step": "one simulated day from step 0 until every trip has arrived",
                          "parallelism": f"replicas x{world}",
                          "l2": l2_note(net, dem)},
               "wall_per_sim_day_s": t_max / args.steps / 1e3,
               "pct_hbm_peak": roofline["frac"],
               "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks,
               "gpu_launches": int(launches)}
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    if out is not None:
        print(json.dumps(out), flush=True)


def end_to_end(L, torch, net, dem, params):
    """One day through the public API from host buffers: network and trip
    upload, the run, trips and link statistics back to the host."""
    net_bytes = sum(int(np.asarray(net[k]).nbytes) for k in
                    ("edge_src", "edge_dst", "edge_len", "edge_lanes", "edge_vmax", "node_green"))
    if net.get("edge_approach_rank") is not None:
        net_bytes += int(net["edge_approach_rank"].nbytes)
    dem_bytes = int(dem["depart_step"].nbytes + dem["route_off"].nbytes + dem["route_edges"].nbytes)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    sim = L.Simulation(net, params)
    sim.load_demand(dem)
    r = sim.run(DAY_STEPS + 100_000)
    trips = sim.trips()
    ls = sim.link_stats()
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    d2h = int(trips["depart"].nbytes + trips["arrive"].nbytes + sum(v.nbytes for v in ls.values()))
    sim.close()
    return {"value": r["veh_steps"] / dt, "unit": "veh-steps/s", "h2d_bytes_per_step": net_bytes + dem_bytes,
            "d2h_bytes_per_step": d2h, "seconds": dt}


if __name__ == "__main__":
    main()
