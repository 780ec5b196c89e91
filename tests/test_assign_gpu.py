"""The assignment loop on the GPU: plain MSA and surrogate-assisted MSA on a
small regional case; every gap is measured by a full simulation; the
trained surrogate predicts link times better than the method without it."""
from __future__ import annotations

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import paper_2406_08496_gb300 as L
    L.build()
    L.load_library()
    L.use_torch_allocator()


@pytest.fixture(scope="module")
def case():
    return W.assignment_case(scale="tiny")


def _tables(net, n_bins, seed, spread=0.8):
    """Link-time tables around free flow, each (edge, bin) scaled by its own
    random factor -- times fall as well as rise between bins, so the FIFO
    rule (holding an entry back to a later bin) is exercised."""
    rng = np.random.default_rng(seed)
    ff = (net["edge_len"] / net["edge_vmax"]).astype(np.float64)[:, None]
    return (ff * np.exp(rng.uniform(0.0, spread, (net["n_edges"], n_bins)))).astype(np.float32)


def _paths(A, search, tt, bin_steps, period_steps):
    tsp = search(tt, bin_steps, period_steps)
    A.reroute(1.0, 0)  # every trip takes its candidate: the routes are the paths
    return tsp, A.routes()


@pytest.mark.parametrize("scale,period_steps,seed", [("tiny", 3600, 1), ("tiny", 600, 2), ("tiny", 36000, 3),
                                                     ("small", 3600, 4)])
def test_gpu_paths_equal_host_paths(scale, period_steps, seed):
    """The GPU search (one warp per tree, label-correcting rounds on packed
    (arrival, edge) labels) returns the host Dijkstra's routes and times bit
    for bit: the earliest arrival, ties to the lower entering edge id."""
    from paper_2406_08496_gb300.assignment import Assignment
    net, dem = W.assignment_case(scale=scale)
    tt = _tables(net, 96, seed)
    host = Assignment(net, dem, seed=seed)
    gpu = Assignment(net, dem, seed=seed)
    th, rh = _paths(host, host.shortest_paths, tt, 1800, period_steps)
    tg, rg = _paths(gpu, gpu.shortest_paths_gpu, tt, 1800, period_steps)
    assert np.array_equal(th.view(np.uint32), tg.view(np.uint32))
    assert np.array_equal(rh["route_off"], rg["route_off"])
    assert np.array_equal(rh["route_edges"], rg["route_edges"])
    # a second call on the same engine reuses its device state
    tt2 = _tables(net, 96, seed + 10)
    th2 = host.shortest_paths(tt2, 1800, period_steps)
    tg2 = gpu.shortest_paths_gpu(tt2, 1800, period_steps)
    assert np.array_equal(th2.view(np.uint32), tg2.view(np.uint32))
    host.close()
    gpu.close()


@pytest.mark.parametrize("scale", ["tiny", "small"])
def test_gpu_load_equals_host_load(scale):
    """Inflow per (edge, bin) of the current routes walked on the GPU equals
    the host walk, count for count, before and after a re-routing."""
    from paper_2406_08496_gb300.assignment import Assignment
    net, dem = W.assignment_case(scale=scale)
    tt = _tables(net, 96, 7)
    A = Assignment(net, dem, seed=2)
    assert np.array_equal(A.load(tt, 1800), A.load_gpu(tt, 1800))
    A.shortest_paths_gpu(tt, 1800, 3600)
    A.reroute(0.3, 1)
    tt2 = _tables(net, 96, 8)
    ref = A.load(tt2, 1800)
    assert ref.sum() > 0
    assert np.array_equal(ref, A.load_gpu(tt2, 1800))
    A.close()


def test_gpu_paths_match_brute_force():
    """On a five-edge diamond, every trip's GPU route is an earliest-arrival
    path among all simple paths, from the middle of its period, and its time
    is that path's from the trip's own departure."""
    from test_assign_cpu import _all_paths, _arrival, _diamond
    from paper_2406_08496_gb300.assignment import Assignment
    net, edges = _diamond()
    rng = np.random.default_rng(5)
    n_bins, bin_steps, dt, period = 6, 20, 0.5, 10
    bin_s = bin_steps * dt
    dep = np.array([0, 13, 31, 55, 70], np.uint32)
    for _ in range(20):
        tt = rng.uniform(1.0, 30.0, (6, n_bins)).astype(np.float32)
        dem = {"orig": np.zeros(5, np.uint32), "dest": np.full(5, 3, np.uint32), "depart_step": dep,
               "route_off": np.arange(0, 11, 2, dtype=np.uint64), "route_edges": np.array([0, 1] * 5, np.uint32)}
        a = Assignment(net, dem, dt=dt, seed=3)
        tsp = a.shortest_paths_gpu(tt, bin_steps, period)
        a.reroute(1.0, 0)
        routes = a.routes()
        for j in range(5):
            t0 = ((dep[j] // period) + 0.5) * period * dt
            best = min(_arrival(p, t0, tt, bin_s) for p in _all_paths(edges, 0, 3))
            r = list(routes["route_edges"][int(routes["route_off"][j]):int(routes["route_off"][j + 1])])
            assert _arrival(r, t0, tt, bin_s) == best
            tj = float(dep[j]) * dt
            assert abs(tsp[j] - (_arrival(r, tj, tt, bin_s) - tj)) < 1e-3
        a.close()


def test_msa_plain_reduces_gap(case):
    from paper_2406_08496_gb300.assignment import msa
    net, dem = case
    r = msa(net, dem, "plain", iterations=4, target_gap=0.0)
    gaps = [h["gap"] for h in r["history"]]
    assert all(g is not None and np.isfinite(g) for g in gaps)
    assert gaps[-1] < gaps[0]
    assert all(h["trips_used"] == len(dem["depart_step"]) for h in r["history"])


def test_msa_surrogate_runs_and_is_judged_by_simulation(case):
    from paper_2406_08496_gb300.assignment import msa
    net, dem = case
    r = msa(net, dem, "surrogate", iterations=5, target_gap=0.0, surrogate_batch=2048, surrogate_steps=300)
    kinds = [h["kind"] for h in r["history"]]
    assert kinds == ["simulation", "surrogate", "simulation", "surrogate", "simulation"]
    sims = [h for h in r["history"] if h["kind"] == "simulation"]
    assert all(np.isfinite(h["gap"]) for h in sims)
    assert all(np.isfinite(h["surrogate_loss"]) for h in sims)
    assert sims[-1]["gap"] < sims[0]["gap"]


def test_surrogate_beats_free_flow_and_stale_times(case):
    """Train on one simulation of the routes, then predict the link times of
    a second simulation after 30% of the trips moved to new paths; compare
    the errors (seconds, over measured (link, bin) cells) with the free-flow
    times and with the first simulation's times."""
    from paper_2406_08496_gb300 import Simulation, Surrogate
    from paper_2406_08496_gb300.assignment import Assignment
    net, dem = case
    params = dict(bin_steps=1800, n_bins=96)
    A = Assignment(net, dem, seed=1)

    def simulate():
        s = Simulation(net, params)
        s.load_demand(A.routes())
        s.run(300_000)
        ls = s.link_stats()
        s.close()
        return ls

    # three simulations, 20% of the trips re-routed between them; train on
    # the pairs (sim0 -> sim0) and (sim0 -> sim1), predict sim2 from sim1
    ls, tt, lr = [], [], []
    for k in range(3):
        ls.append(simulate())
        a, b = A.link_times(ls[-1]["tt_sum"], ls[-1]["tt_cnt"])
        tt.append(a)
        lr.append(b)
        if k < 2:
            A.shortest_paths(a, 1800, 3600)
            A.reroute(0.2, k)
    mlp = Surrogate(n_features=11, batch=2048, seed=3)
    Xs, ts = [], []
    for ref, k in ((0, 0), (0, 1)):
        X = A.features(ls[k]["inflow"], ls[k]["occ"], lr[ref], ls[ref]["inflow"])
        ok = (ls[k]["tt_cnt"].reshape(-1) >= 2) & np.isfinite(lr[k].reshape(-1))
        Xs.append(X[ok])
        ts.append(lr[k].reshape(-1)[ok])
    mlp.train(np.concatenate(Xs), np.concatenate(ts), steps=1500, lr=1e-3, seed=4)
    inflow = A.load(tt[1], 1800)
    tt_pred = A.times_from_ratio(mlp.forward(A.features(inflow, ls[1]["occ"], lr[1], ls[1]["inflow"])), 96)
    ff = np.repeat((net["edge_len"] / net["edge_vmax"])[:, None], 96, axis=1)
    w = ls[2]["tt_cnt"].reshape(-1).astype(np.float64)
    ok2 = w > 0
    # per-vehicle error: cells weighted by the vehicles that crossed them
    err = lambda p: float(np.average(np.abs(p.reshape(-1)[ok2] - tt[2].reshape(-1)[ok2]), weights=w[ok2]))
    e_sur, e_ff, e_stale = err(tt_pred), err(ff), err(tt[1])
    print(f"link-time error per vehicle (s): surrogate {e_sur:.3f}, free flow {e_ff:.3f}, "
          f"previous simulation {e_stale:.3f}")
    assert e_sur < 0.5 * e_ff
    assert e_sur < 1.5 * e_stale
