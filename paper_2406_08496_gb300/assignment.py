"""Traffic assignment around the simulator: the method of successive
averages with time-dependent shortest paths, plain or surrogate-assisted.

Binding of include/lpsim_assign.h plus the iteration driver.  All arithmetic
runs in the library: simulations, the surrogate and (by default) the
time-dependent shortest paths on the GPU; gaps, loading and features in the
host engine (C++ threads); this module only sequences the calls.
"""
from __future__ import annotations

import ctypes
import os
import time

import numpy as np

from . import Simulation, Surrogate, _check, _p, load_library

N_FEATURES = 11


def _lib():
    lib = load_library()
    if not getattr(lib, "_assign_ready", False):
        P = ctypes.c_void_p
        lib.lpsim_assign_create.argtypes = [ctypes.POINTER(P), ctypes.c_uint32, ctypes.c_uint32, P, P, P, P, P,
                                            ctypes.c_uint64, P, P, P, P, P, ctypes.c_float, ctypes.c_uint64]
        lib.lpsim_assign_shortest_paths.argtypes = [P, P, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32,
                                                    ctypes.c_uint32, P]
        lib.lpsim_assign_shortest_paths_gpu.argtypes = [P, P, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32, P]
        lib.lpsim_assign_gap.argtypes = [P, P, P, P, P]
        lib.lpsim_assign_reroute.argtypes = [P, ctypes.c_double, ctypes.c_uint32, P]
        lib.lpsim_assign_route_excess.argtypes = [P, P, ctypes.c_uint32, ctypes.c_uint32]
        lib.lpsim_assign_reroute_worst.argtypes = [P, ctypes.c_double, ctypes.c_double, P]
        lib.lpsim_assign_route_length.argtypes = [P]
        lib.lpsim_assign_route_length.restype = ctypes.c_uint64
        lib.lpsim_assign_get_routes.argtypes = [P, P, P, ctypes.c_uint64]
        lib.lpsim_assign_load.argtypes = [P, P, ctypes.c_uint32, ctypes.c_uint32, P]
        lib.lpsim_assign_load_gpu.argtypes = [P, P, ctypes.c_uint32, ctypes.c_uint32, P]
        lib.lpsim_assign_features.argtypes = [P, ctypes.c_uint32, P, P, P, P, P, ctypes.c_uint32]
        lib.lpsim_assign_features_rows.argtypes = [P, ctypes.c_uint32, P, P, P, P, ctypes.c_uint64, P, P,
                                                   ctypes.c_uint32]
        lib.lpsim_assign_link_times.argtypes = [P, ctypes.c_uint32, P, P, P, P]
        lib.lpsim_assign_times_from_ratio.argtypes = [P, ctypes.c_uint32, P, P]
        lib.lpsim_assign_destroy.argtypes = [P]
        lib.lpsim_assign_destroy.restype = None
        lib._assign_ready = True
    return lib


class Assignment:
    """Routes of a trip table and the assignment engine's state."""

    def __init__(self, net: dict, dem: dict, dt: float = 0.5, seed: int = 0):
        self.lib = _lib()
        self.net = net
        self.n_edges = int(net["n_edges"])
        self.dep = np.ascontiguousarray(dem["depart_step"], dtype=np.uint32)
        self.n = len(self.dep)
        arrs = [np.ascontiguousarray(net[k]) for k in ("edge_src", "edge_dst")]
        self._keep = [np.ascontiguousarray(net["edge_src"], dtype=np.uint32),
                      np.ascontiguousarray(net["edge_dst"], dtype=np.uint32),
                      np.ascontiguousarray(net["edge_len"], dtype=np.float32),
                      np.ascontiguousarray(net["edge_lanes"], dtype=np.uint8),
                      np.ascontiguousarray(net["edge_vmax"], dtype=np.float32),
                      np.ascontiguousarray(dem["orig"], dtype=np.uint32),
                      np.ascontiguousarray(dem["dest"], dtype=np.uint32), self.dep,
                      np.ascontiguousarray(dem["route_off"], dtype=np.uint64),
                      np.ascontiguousarray(dem["route_edges"], dtype=np.uint32)]
        del arrs
        k = self._keep
        h = ctypes.c_void_p()
        _check(self.lib, self.lib.lpsim_assign_create(ctypes.byref(h), int(net["n_nodes"]), self.n_edges, _p(k[0]),
                                                      _p(k[1]), _p(k[2]), _p(k[3]), _p(k[4]), self.n, _p(k[5]),
                                                      _p(k[6]), _p(k[7]), _p(k[8]), _p(k[9]), dt, seed))
        self.h = h

    def shortest_paths(self, tt: np.ndarray, bin_steps: int, period_steps: int, n_threads: int | None = None):
        tt = np.ascontiguousarray(tt, dtype=np.float32)
        tsp = np.empty(self.n, np.float32)
        nt = n_threads or (os.cpu_count() or 1)
        _check(self.lib, self.lib.lpsim_assign_shortest_paths(self.h, _p(tt), tt.shape[1], bin_steps, period_steps,
                                                              nt, _p(tsp)))
        return tsp

    def shortest_paths_gpu(self, tt: np.ndarray, bin_steps: int, period_steps: int):
        """The same trees searched on the GPU (identical routes and times)."""
        tt = np.ascontiguousarray(tt, dtype=np.float32)
        tsp = np.empty(self.n, np.float32)
        _check(self.lib, self.lib.lpsim_assign_shortest_paths_gpu(self.h, _p(tt), tt.shape[1], bin_steps,
                                                                  period_steps, _p(tsp)))
        return tsp

    def gap(self, depart_actual: np.ndarray, arrive_step: np.ndarray):
        d = np.ascontiguousarray(depart_actual, dtype=np.uint32)
        a = np.ascontiguousarray(arrive_step, dtype=np.uint32)
        rg = ctypes.c_double()
        used = ctypes.c_uint64()
        _check(self.lib, self.lib.lpsim_assign_gap(self.h, _p(d), _p(a), ctypes.byref(rg), ctypes.byref(used)))
        return rg.value, used.value

    def reroute(self, fraction: float, iteration: int) -> int:
        n = ctypes.c_uint64()
        _check(self.lib, self.lib.lpsim_assign_reroute(self.h, fraction, iteration, ctypes.byref(n)))
        return n.value

    def route_excess(self, tt: np.ndarray, bin_steps: int) -> None:
        tt = np.ascontiguousarray(tt, dtype=np.float32)
        _check(self.lib, self.lib.lpsim_assign_route_excess(self.h, _p(tt), tt.shape[1], bin_steps))

    def reroute_worst(self, fraction: float, min_rel_excess: float = 0.0) -> int:
        n = ctypes.c_uint64()
        _check(self.lib, self.lib.lpsim_assign_reroute_worst(self.h, fraction, min_rel_excess, ctypes.byref(n)))
        return n.value

    def routes(self) -> dict:
        total = int(self.lib.lpsim_assign_route_length(self.h))
        off = np.empty(self.n + 1, np.uint64)
        edges = np.empty(max(1, total), np.uint32)
        _check(self.lib, self.lib.lpsim_assign_get_routes(self.h, _p(off), _p(edges), edges.size))
        return {"depart_step": self.dep, "route_off": off, "route_edges": edges[:total]}

    def load(self, tt: np.ndarray, bin_steps: int) -> np.ndarray:
        tt = np.ascontiguousarray(tt, dtype=np.float32)
        inflow = np.empty(tt.shape, np.uint32)
        _check(self.lib, self.lib.lpsim_assign_load(self.h, _p(tt), tt.shape[1], bin_steps, _p(inflow)))
        return inflow

    def load_gpu(self, tt: np.ndarray, bin_steps: int) -> np.ndarray:
        """The same inflow counts, the routes walked on the GPU."""
        tt = np.ascontiguousarray(tt, dtype=np.float32)
        inflow = np.empty(tt.shape, np.uint32)
        _check(self.lib, self.lib.lpsim_assign_load_gpu(self.h, _p(tt), tt.shape[1], bin_steps, _p(inflow)))
        return inflow

    def features(self, inflow: np.ndarray, occ: np.ndarray, prev_log_ratio: np.ndarray,
                 prev_inflow: np.ndarray, rows: np.ndarray | None = None) -> np.ndarray:
        """Surrogate inputs of every (edge, bin) cell, edge-major, or of the
        listed cells (rows: indices edge * n_bins + bin) in that order."""
        inflow = np.ascontiguousarray(inflow, dtype=np.uint32)
        occ = np.ascontiguousarray(occ, dtype=np.uint32)
        plr = np.ascontiguousarray(prev_log_ratio, dtype=np.float32)
        pin = np.ascontiguousarray(prev_inflow, dtype=np.uint32)
        if rows is not None:
            rows = np.ascontiguousarray(rows, dtype=np.uint64)
            X = np.empty((len(rows), N_FEATURES), np.float32)
            _check(self.lib, self.lib.lpsim_assign_features_rows(self.h, inflow.shape[1], _p(inflow), _p(occ), _p(plr),
                                                                 _p(pin), len(rows), _p(rows), _p(X), N_FEATURES))
            return X
        X = np.empty((inflow.shape[0] * inflow.shape[1], N_FEATURES), np.float32)
        _check(self.lib, self.lib.lpsim_assign_features(self.h, inflow.shape[1], _p(inflow), _p(occ), _p(plr),
                                                        _p(pin), _p(X), N_FEATURES))
        return X

    def link_times(self, tt_sum: np.ndarray, tt_cnt: np.ndarray):
        s = np.ascontiguousarray(tt_sum, dtype=np.uint32)
        c = np.ascontiguousarray(tt_cnt, dtype=np.uint32)
        tt = np.empty(s.shape, np.float32)
        lr = np.empty(s.shape, np.float32)
        _check(self.lib, self.lib.lpsim_assign_link_times(self.h, s.shape[1], _p(s), _p(c), _p(tt), _p(lr)))
        return tt, lr

    def times_from_ratio(self, y: np.ndarray, n_bins: int) -> np.ndarray:
        y = np.ascontiguousarray(y, dtype=np.float32)
        tt = np.empty((self.n_edges, n_bins), np.float32)
        _check(self.lib, self.lib.lpsim_assign_times_from_ratio(self.h, n_bins, _p(y), _p(tt)))
        return tt

    def close(self):
        if getattr(self, "h", None):
            self.lib.lpsim_assign_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def msa(net: dict, dem: dict, mode: str = "plain", iterations: int = 10, fraction: float = 0.1,
        target_gap: float = 0.01, sim_params: dict | None = None, bin_steps: int = 1800, n_bins: int = 96,
        period_steps: int = 3600, max_steps: int = 300_000, surrogate_steps: int = 400, surrogate_batch: int = 8192,
        seed: int = 0, select: str = "random", min_rel_excess: float = 0.0, paths: str = "gpu", log=None) -> dict:
    """Method of successive averages.  plain: every iteration simulates the
    current routes, measures the relative gap and moves `fraction` of the
    trips to their time-dependent shortest paths under the simulated link
    times.  surrogate: even iterations do the same (and train the surrogate
    on every simulation's link statistics so far); odd iterations skip the
    simulation, predict the link times of the current routes with the
    surrogate (inflows from loading the routes with the last simulated
    times) and re-route under the prediction.  The surrogate predicts the
    change of each (link, bin) log travel-time ratio from the last
    simulation (taken as 0 where that simulation did not measure the cell),
    and it is trained on exactly the inputs a prediction sees: each
    simulation's routes loaded under the previous simulation's link times,
    with the previous simulation's occupancy, ratios and inflows.  Every reported gap is
    measured by a full simulation.  select: which trips move -- "random"
    (each trip with probability fraction, seeded) or "worst" (the fraction
    with the largest relative excess of their route over the shortest path
    under the iteration's link times, measured or predicted; only trips more
    than min_rel_excess worse than their shortest path).  paths: where the
    time-dependent shortest paths are searched -- "gpu" (one warp per tree)
    or "host" (Dijkstra on the host threads); both give the same routes and
    times.  Returns the iteration history and the wall time to reach
    target_gap (None if never reached)."""
    assert mode in ("plain", "surrogate") and select in ("worst", "random") and paths in ("gpu", "host")

    def move(it):
        return A.reroute_worst(fraction, min_rel_excess) if select == "worst" else A.reroute(fraction, it)

    params = dict(bin_steps=bin_steps, n_bins=n_bins)
    params.update(sim_params or {})
    A = Assignment(net, dem, dt=0.5, seed=seed)
    search = A.shortest_paths_gpu if paths == "gpu" else A.shortest_paths
    mlp = Surrogate(n_features=N_FEATURES, batch=surrogate_batch, seed=seed) if mode == "surrogate" else None
    hist = []
    t_start = time.perf_counter()
    t_hit = None
    tt_last = occ_last = lr_last = in_last = None
    for it in range(iterations):
        full = mode == "plain" or it % 2 == 0
        t0 = time.perf_counter()
        if full:
            routes = A.routes()
            sim = Simulation(net, params)
            vid = sim.load_demand(routes).astype(np.int64)
            run = sim.run(max_steps)
            ls = sim.link_stats()
            tr = sim.trips()
            sim.close()
            t_sim = time.perf_counter() - t0
            tt, logratio = A.link_times(ls["tt_sum"], ls["tt_cnt"])
            search(tt, bin_steps, period_steps)
            rg, used = A.gap(tr["depart"][vid], tr["arrive"][vid])
            if select == "worst":
                # rank trips by their route's excess under the measured link
                # times (as the surrogate iterations do under predicted ones)
                A.route_excess(tt, bin_steps)
            now = time.perf_counter() - t_start
            rec = dict(iteration=it, kind="simulation", gap=rg, trips_used=used, veh_steps=run["veh_steps"],
                       wall_s=now, iter_s=time.perf_counter() - t0, sim_s=t_sim,
                       paths_s=time.perf_counter() - t0 - t_sim)
            if rg <= target_gap and t_hit is None:
                t_hit = now
            if mlp is not None:
                # training pair (previous simulation -> this one; this one
                # itself at first): the inputs a prediction from the previous
                # simulation sees for these routes, and the change of the log
                # ratios it should predict
                t1 = time.perf_counter()
                first = lr_last is None
                ref_tt, ref_occ = (tt, ls["occ"]) if first else (tt_last, occ_last)
                ref_lr, ref_in = (logratio, ls["inflow"]) if first else (lr_last, in_last)
                loaded = A.load_gpu(ref_tt, bin_steps) if paths == "gpu" else A.load(ref_tt, bin_steps)
                # samples: cells crossed at least twice (a measured ratio)
                rows = np.flatnonzero(ls["tt_cnt"].reshape(-1) >= 2)
                dy = logratio.reshape(-1)[rows] - np.nan_to_num(ref_lr.reshape(-1)[rows], nan=0.0)
                # every simulation's samples join the model's device-resident pool
                mlp.pool_add(A.features(loaded, ref_occ, ref_lr, ref_in, rows=rows), dy)
                losses = mlp.train_pool(surrogate_steps, lr=1e-3, seed=seed + it)
                rec["train_s"] = time.perf_counter() - t1
                rec["surrogate_loss"] = float(losses[-20:].mean())
                rec["surrogate_samples"] = mlp.pool_size()
            tt_last, occ_last, lr_last, in_last = tt, ls["occ"], logratio, ls["inflow"]
            if t_hit is not None:
                hist.append(rec)
                if log:
                    log(rec)
                break
            rec["rerouted"] = move(it)
        else:
            inflow = A.load_gpu(tt_last, bin_steps) if paths == "gpu" else A.load(tt_last, bin_steps)
            X = A.features(inflow, occ_last, lr_last, in_last)
            y = mlp.forward(X) + np.nan_to_num(lr_last, nan=0.0).reshape(-1)
            tt_pred = A.times_from_ratio(y, n_bins)
            search(tt_pred, bin_steps, period_steps)
            if select == "worst":
                A.route_excess(tt_pred, bin_steps)
            rec = dict(iteration=it, kind="surrogate", gap=None, wall_s=time.perf_counter() - t_start,
                       iter_s=time.perf_counter() - t0)
            rec["rerouted"] = move(it)
        hist.append(rec)
        if log:
            log(rec)
    A.close()
    return {"mode": mode, "history": hist, "time_to_target_s": t_hit,
            "final_gap": next((h["gap"] for h in reversed(hist) if h["gap"] is not None), None),
            "wall_s": time.perf_counter() - t_start}
