"""Batched scenarios, snapshot/restore and the autotuner on the GPU.

Each scenario of a batch must equal the oracle run of that scenario alone,
bit for bit; a restored snapshot must replay identically; the tuned launch
configuration must not change any result."""
from __future__ import annotations

import numpy as np
import pytest

import oracle as O
import workloads as W
from simutil import assert_outputs_equal, assert_state_equal

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import paper_2406_08496_gb300 as L
    L.build()
    L.load_library()
    L.use_torch_allocator()


@pytest.fixture(scope="module")
def scenarios():
    return W.batch_scenarios(6, base_seed=7, min_nodes=200, max_nodes=2500, min_trips=500, max_trips=5000,
                             horizon_h=0.5)


def _compare_scenario(g, vids_b, off, s, o, vid_o, n_bins):
    so, sg = o.state(), g.state()
    idx_b = vids_b[s].astype(np.int64)
    idx_o = vid_o.astype(np.int64)
    for key in ("status", "lane", "ridx"):
        assert np.array_equal(sg[key][idx_b], so[key][idx_o]), (s, key)
    act = so["status"][idx_o] == 1
    assert np.array_equal(sg["edge"][idx_b][act] - off["edge"][s], so["edge"][idx_o][act].astype(np.int64)), s
    for key in ("x", "v"):
        assert np.array_equal(sg[key][idx_b].view(np.uint32), so[key][idx_o].view(np.uint32)), (s, key)
    tg, to = g.trips(), o.trips()
    assert np.array_equal(tg["arrive"][idx_b], to["arrive"][idx_o]), s
    assert np.array_equal(tg["depart"][idx_b], to["depart"][idx_o]), s
    lg, lo = g.link_stats(), o.link_stats()
    e0, e1 = off["edge"][s], off["edge"][s + 1]
    for key in ("entries", "exits", "tt_steps"):
        assert np.array_equal(lg[key][e0:e1], lo[key]), (s, key)
    if n_bins:
        for key in ("inflow", "tt_sum", "tt_cnt", "occ"):
            assert np.array_equal(lg[key][e0:e1], lo[key]), (s, key)
    c0, c1 = off["cell"][s], off["cell"][s + 1]
    assert np.array_equal(g.lane_map()[c0:c1], o.lane_map()), s


@pytest.mark.parametrize("gpu_params,extra", [({}, {}), (dict(block_size=128, blocks_per_sm=2, sort_period=32), {}),
                                               ({}, dict(dlc_prob=0.3, dlc_gain=3.0, eps_amp=1.0))])
def test_batch_equals_each_scenario_alone(scenarios, gpu_params, extra):
    """Each scenario of a batch bit for bit equal to the oracle's run of it
    alone: in two launch configurations, and with the discretionary lane
    change on (its draws keyed by the scenario's own seed and ids)."""
    from paper_2406_08496_gb300 import BatchSimulation
    params = dict(bin_steps=300, n_bins=8, x0=80.0, **extra)
    nets = [n for n, _, _ in scenarios]
    dems = [d for _, d, _ in scenarios]
    seeds = [s for _, _, s in scenarios]
    g = BatchSimulation(nets, dict(params, **gpu_params))
    vids = g.load_demand(dems, seeds)
    off = g.offsets()
    assert off["trip"][-1] == sum(len(d["depart_step"]) for d in dems)
    g.step(2400)
    lane_changes = 0
    for s, (net, dem, seed) in enumerate(scenarios):
        o = O.Oracle(net, dict(params, seed=seed))
        vid_o = o.load_demand(dem)
        o.step(2400)
        lane_changes += o.counters()["lane_changes"]
        _compare_scenario(g, vids, off, s, o, vid_o, params["n_bins"])
    assert lane_changes > 0


def test_snapshot_restore_replays_identically(grid_day):
    from paper_2406_08496_gb300 import Simulation
    net, dem = grid_day
    g = Simulation(net, dict(bin_steps=600, n_bins=6))
    g.load_demand(dem)
    g.step(700)
    g.snapshot()
    g.step(900)
    s1, t1, l1, m1 = g.state(), g.trips(), g.link_stats(), g.lane_map()
    g.restore()
    g.step(400)
    g.step(500)
    assert_state_equal(s1, g.state())
    assert np.array_equal(t1["arrive"], g.trips()["arrive"])
    assert np.array_equal(l1["occ"], g.link_stats()["occ"])
    assert np.array_equal(m1, g.lane_map())


def test_autotuned_configuration_keeps_results(grid_day):
    from paper_2406_08496_gb300 import Simulation
    net, dem = grid_day
    o = O.Oracle(net, {})
    o.load_demand(dem)
    g = Simulation(net, {})
    g.load_demand(dem)
    g.step(768)
    o.step(768)
    res = g.autotune(768)
    assert res["n_tried"] >= 20 and res["best_ms"] <= res["default_ms"] * 1.0001
    assert_state_equal(o.state(), g.state(), "after tuning")  # left at the starting state
    g.step(2000)
    o.step(2000)
    assert_outputs_equal(o, g)
