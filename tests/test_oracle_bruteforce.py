"""Brute force on tiny inputs: the oracle against an independent restatement
(tests/bruteforce_sim.py: vehicle records instead of a lane map) on a few
hundred seeded tiny scenarios -- 7 edges with a merge, a diverge and two
possibly signalised nodes, 1-3 lanes, edges shorter than one step's travel,
1-5 vehicles departing in steps 0..4.  Trajectories must agree bit for bit
at every step."""
from __future__ import annotations

import numpy as np
import pytest

import oracle as O
from bruteforce_sim import BruteForce
from netutil import make_demand, make_net, routes_of

# nodes 0..6; e0 0->1, e1 1->2, e2 1->3, e3 2->4, e4 3->4, e5 5->1, e6 4->6
TOPO = [(0, 1), (1, 2), (1, 3), (2, 4), (3, 4), (5, 1), (4, 6)]
ROUTES = [[0, 1, 3, 6], [0, 2, 4, 6], [5, 1, 3], [5, 2], [1, 3, 6], [0], [2, 4], [5, 2, 4, 6], [0, 1]]


def scenario(seed):
    rng = np.random.default_rng(seed)
    lens = rng.choice([2.5, 6.0, 9.0, 14.0, 23.0, 40.0, 71.0], size=len(TOPO))
    lanes = rng.integers(1, 4, size=len(TOPO))
    vmax = rng.choice([3.0, 5.5, 13.9, 20.0], size=len(TOPO))
    edges = [(a, b, float(l), int(n), float(v)) for (a, b), l, n, v in zip(TOPO, lens, lanes, vmax)]
    green = {1: int(rng.choice([0, 2, 5])), 4: int(rng.choice([0, 3, 7]))}
    ranks = None
    if rng.random() < 0.3:
        ranks = [0] * len(TOPO)
        ranks[5] = 1  # node 1: e0 phase 0, e5 phase 1; node 4: e3, e4 share phase 0
    net = make_net(7, edges, green=green, approach_rank=ranks)
    nveh = int(rng.integers(1, 6))
    trips = [(int(rng.integers(0, 5)), ROUTES[int(rng.integers(len(ROUTES)))]) for _ in range(nveh)]
    params = dict(x0=float(rng.choice([100.0, 15.0])), seed=int(rng.integers(1, 1 << 40)),
                  eps_amp=float(rng.choice([0.0, 0.0, 1.5])), bin_steps=0, n_bins=0)
    return net, trips, params


# vehicle types of the typed scenarios: a car, a truck (slower to start, longer
# standstill gap, top speed 12 m/s) and a bike (top speed 4.5 m/s)
TYPES = [dict(a=1.0, b=1.5, s0=2.0, T=1.5, vmax=254.0), dict(a=0.6, b=1.2, s0=4.0, T=2.0, vmax=12.0),
         dict(a=0.8, b=1.0, s0=1.0, T=1.0, vmax=4.5)]


def scenario_overtaking(seed, busy=False):
    """Long multi-lane edges in a chain with a diverge, a slow vehicle
    departing first and faster ones behind it: the case the discretionary
    rule is for.  busy: 10-17 vehicles departing about one a step, so the
    lanes fill and mandatory changes toward the diverge meet traffic."""
    rng = np.random.default_rng(seed)
    topo = [(0, 1), (1, 2), (1, 3), (2, 4)]
    lens = rng.choice([60.0, 120.0, 250.0], size=len(topo))
    lanes = rng.integers(2, 4, size=len(topo))
    vmax = rng.choice([13.9, 20.0], size=len(topo))
    edges = [(a, b, float(l), int(n), float(v)) for (a, b), l, n, v in zip(topo, lens, lanes, vmax)]
    net = make_net(5, edges, green={1: int(rng.choice([0, 20]))})
    routes = [[0, 1, 3], [0, 2], [0, 1], [0]]
    nveh = int(rng.integers(10, 18)) if busy else int(rng.integers(3, 8))
    spacing = 1 if busy else 2
    trips = [(int(spacing * q + rng.integers(0, 3)), routes[int(rng.integers(len(routes)))]) for q in range(nveh)]
    params = dict(x0=float(rng.choice([100.0, 30.0])), seed=int(rng.integers(1, 1 << 40)),
                  eps_amp=float(rng.choice([0.0, 1.5])), bin_steps=0, n_bins=0)
    vt = np.concatenate([[2], rng.integers(0, len(TYPES), nveh - 1)]).astype(np.uint8)  # a bike first
    return net, trips, params, vt


def compare(seed, steps=70, typed=False, dlc=False, overtaking=False, busy=False):
    if overtaking:
        net, trips, params, vt = scenario_overtaking(seed, busy)
    else:
        net, trips, params = scenario(seed)
    if dlc:
        # discretionary lane changes (an extension of the paper's mandatory rule)
        rng = np.random.default_rng(seed + 11)
        params.update(dlc_prob=float(rng.choice([0.3, 1.0])), dlc_gain=float(rng.choice([0.0, 3.0, 8.0])))
    dem = make_demand(trips)
    types = None
    if typed or overtaking:
        types = TYPES
        dem["vtype"] = (vt if overtaking else
                        np.random.default_rng(seed + 7).integers(0, len(TYPES), len(trips)).astype(np.uint8))
    o = O.Oracle(net, params, vehicle_types=types)
    vid = o.load_demand(dem)
    bf = BruteForce(net, dict(O.DEFAULT_PARAMS, **params), vehicle_types=types)
    bf.load(dem["depart_step"], routes_of(dem), dem.get("vtype"))
    assert bf.vid == vid.tolist()
    for k in range(steps):
        a = o.state()
        b = bf.state()
        for key in ("status", "edge", "lane", "ridx"):
            assert np.array_equal(a[key], b[key]), (seed, k, key, a[key], b[key])
        for key in ("x", "v"):
            assert np.array_equal(a[key].view(np.uint32), b[key].view(np.uint32)), (seed, k, key, a[key], b[key])
        o.step(1)
        bf.step()
    tr = o.trips()
    assert tr["depart"].tolist() == [w["dep_act"] for w in bf.veh]
    assert tr["arrive"].tolist() == [w["arr"] for w in bf.veh]
    return o.counters()


@pytest.mark.parametrize("block", range(8))
def test_bruteforce_tiny(block):
    changes = crossings = 0
    for seed in range(block * 40, block * 40 + 40):
        c = compare(seed)
        changes += c["lane_changes"]
        crossings += c["arrived"]
    assert crossings > 0


@pytest.mark.parametrize("block", range(2))
def test_bruteforce_tiny_vehicle_types(block):
    """The same family with each vehicle a car, a truck or a bike (Algorithm 1
    State: vehicle type; multimodal traffic, Sec. 5)."""
    for seed in range(1000 + block * 40, 1000 + block * 40 + 40):
        compare(seed, typed=True)


@pytest.mark.parametrize("block", range(2))
def test_bruteforce_tiny_discretionary_lane_changes(block):
    """Discretionary lane changes on, in the typed family and in a family of
    long multi-lane edges with a bike departing ahead of cars and trucks:
    trajectories agree bit for bit, and the rule fires (more lane changes
    than the same overtaking scenarios with it off)."""
    on = off = 0
    for seed in range(2000 + block * 40, 2000 + block * 40 + 40):
        compare(seed, typed=True, dlc=True)
        on += compare(seed, steps=120, dlc=True, overtaking=True)["lane_changes"]
        off += compare(seed, steps=120, overtaking=True)["lane_changes"]
    assert on > off


def test_bruteforce_busy_lanes():
    """Ten to seventeen vehicles a scenario on the long multi-lane family,
    the lanes filling, with the mandatory rule alone and with the
    discretionary rule on: bit for bit at every step, and the mandatory
    changes toward the diverge happen in traffic (over a hundred of them in
    sixty scenarios)."""
    changes = 0
    for seed in range(3000, 3060):
        changes += compare(seed, steps=150, overtaking=True, busy=True)["lane_changes"]
        compare(seed, steps=150, overtaking=True, busy=True, dlc=True)
    assert changes > 100


def test_bruteforce_exercises_lane_changes_and_conflicts():
    """The scenario family reaches the rarer branches: accepted lane changes,
    entry conflicts and red holds."""
    lane_changes = 0
    for seed in range(320):
        lane_changes += compare(seed, steps=70)["lane_changes"]
    assert lane_changes > 0
