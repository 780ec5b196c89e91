"""Parity at the full regional size (the 2.82M-trip day on 224k nodes) and at
the large size (the 9.01M-trip day on 1.01M nodes), in the launch
configuration the benchmark times (default block size, blocks per SM, sort
period and graph chunk; no debug flags).

* A sample the oracle can finish: every trip of the 2.82M-trip day that
  departs in a five-minute window of the morning peak, simulated alone on the
  full 224k-node network for 1,536 steps (one graph chunk).  Every output is
  compared bit for bit.
* The same for the 9.01M-trip day (departures 07:30-07:33).
* Each whole day on the GPU, checked through properties that hold at any size:
  every trip departs no earlier than planned and arrives; each trip's travel
  time is at least its route length at the network's top speed; every edge
  was left as often as it was entered, and entered once per route position;
  traversal steps are at least one per exit; the lane map ends empty.
"""
from __future__ import annotations

import math

import numpy as np
import pytest

import oracle as O
from simutil import assert_outputs_equal

pytestmark = pytest.mark.gpu

PEAK_WINDOW = (7 * 7200 + 3600, 7 * 7200 + 3600 + 600)  # departures 07:30-07:35 (dt = 0.5 s)
WINDOW_STEPS = 1536  # one graph chunk of the default length
DAY_STEPS = 172_800


@pytest.fixture(scope="module")
def regional():
    import workloads as W
    return W.regional_day(seed=2, n_trips=2_820_000)


@pytest.fixture(scope="module")
def large():
    import workloads as W
    return W.regional_day(seed=3, n_trips=9_010_000, scale="large")


def test_regional_peak_window_matches_oracle(regional):
    peak_window_matches_oracle(regional, PEAK_WINDOW, min_trips=10_000)


def test_large_peak_window_matches_oracle(large):
    """The 9.01M-trip day: its 07:30-07:33 departures on the full 1.01M-node
    network for one graph chunk, bit for bit."""
    net, dem = large
    assert net["n_nodes"] > 1_000_000 and len(dem["depart_step"]) == 9_010_000
    peak_window_matches_oracle(large, (PEAK_WINDOW[0], PEAK_WINDOW[0] + 360), min_trips=20_000)


def peak_window_matches_oracle(workload, window, min_trips):
    import workloads as W
    from paper_2406_08496_gb300 import Simulation
    net, dem = workload
    keep = (dem["depart_step"] >= window[0]) & (dem["depart_step"] < window[1])
    sub = W.subset_trips(dem, keep)
    sub["depart_step"] = (sub["depart_step"] - window[0]).astype(np.uint32)
    assert len(sub["depart_step"]) > min_trips
    params = dict(bin_steps=1800, n_bins=2)
    o = O.Oracle(net, params)
    vo = o.load_demand(sub)
    g = Simulation(net, params)
    vg = g.load_demand(sub)
    assert np.array_equal(vo, vg)
    o.step(WINDOW_STEPS)
    g.step(WINDOW_STEPS)
    assert_outputs_equal(o, g, n_bins=2, where=f"peak window of {net['n_nodes']} nodes")
    co, cg = o.counters(), g.counters()
    for key in ("veh_steps", "arrived", "active", "waiting", "lane_changes"):
        assert co[key] == cg[key], (key, co[key], cg[key])
    assert cg["lane_changes"] > 0 and cg["arrived"] > 0


def test_regional_day_properties(regional):
    day_properties(regional)


def test_large_day_properties(large):
    day_properties(large)


def day_properties(workload):
    from paper_2406_08496_gb300 import Simulation
    net, dem = workload
    n = len(dem["depart_step"])
    g = Simulation(net, dict(bin_steps=1800, n_bins=96))
    vid = g.load_demand(dem)
    r = g.run(DAY_STEPS + 100_000)
    assert r["arrived"] == n and r["active"] == 0 and r["waiting"] == 0
    tr = g.trips()
    # per vehicle id: planned departure step and route
    order = np.empty(n, np.int64)
    order[vid] = np.arange(n)
    dep_plan = dem["depart_step"][order]
    assert np.all(tr["depart"] >= dep_plan)
    assert np.all(tr["arrive"] > tr["depart"])
    off = dem["route_off"]
    edges = dem["route_edges"]
    cells = np.maximum(1, np.ceil(net["edge_len"].astype(np.float64))).astype(np.int64)
    route_cells = np.add.reduceat(cells[edges], off[:-1].astype(np.int64))
    # no speed exceeds the top speed limit (IDM never accelerates past v0 and
    # decelerates above it; 0.1% slack for rounding); every step advances at
    # most vmax * dt, and the whole route length has to be covered
    vmax = float(np.max(net["edge_vmax"])) * 1.001
    min_steps = np.floor(route_cells[order] / (vmax * 0.5))
    assert np.all(tr["arrive"] - tr["depart"] >= min_steps)
    ls = g.link_stats()
    assert np.array_equal(ls["entries"], ls["exits"])
    expect = np.bincount(edges, minlength=net["n_edges"]).astype(np.uint64)
    assert np.array_equal(ls["entries"], expect)
    assert np.all(ls["tt_steps"] >= ls["exits"])
    assert int(ls["inflow"].sum()) == int(ls["entries"].sum())
    assert int(ls["tt_cnt"].sum()) == int(ls["exits"].sum())
    assert np.all(g.lane_map() == 255)
    assert math.isfinite(r["wall_ms"])
