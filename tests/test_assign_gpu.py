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
