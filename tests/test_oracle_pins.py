"""Pins of the CPU oracle against what the paper and the mathematics fix.

Closed forms (IDM against Treiber's formula in double precision, free-flow
arrival, signal wait, departure headway, saturation discharge, no-crash
standstill gap), the paper's lane-map worked example, and invariants
(conservation, one vehicle per cell, FIFO on single-lane links, no backward
motion, speed bounds, link-statistics bookkeeping).
"""
from __future__ import annotations

import math
import os

import numpy as np
import pytest

import oracle as O
from bruteforce_sim import splitmix64_mix, unit24
from netutil import make_demand, make_net

F = np.float32
NOVAL = 0xFFFFFFFF
P0 = dict(O.DEFAULT_PARAMS)
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def run_oracle(net, trips, steps, **params):
    o = O.Oracle(net, params)
    o.load_demand(make_demand(trips))
    o.step(steps)
    return o


# ---------------------------------------------------------------------------- IDM

def idm_double(v, vf, s, v0, a, b, s0, T, dt):
    """Intelligent Driver Model (Treiber, Hennecke, Helbing 2000), delta = 4,
    evaluated in double precision, one explicit Euler step of length dt."""
    s_star = s0 + max(0.0, v * T + v * (v - vf) / (2.0 * math.sqrt(a * b)))
    acc = a * (1.0 - (v / v0) ** 4 - (s_star / s) ** 2)
    return max(0.0, v + acc * dt), acc


@pytest.mark.parametrize("v0", [11.1, 13.9, 30.0])
def test_idm_matches_double_closed_form(v0):
    p = P0
    worst = 0.0
    for v in [0.0, 0.5, 5.5, 13.9, 22.0, 30.0]:
        for vf in [0.0, 3.0, 14.0, 29.0]:
            for s in [0.4, 1.0, 3.7, 9.5, 18.0, 40.0, 75.0]:
                got = O.idm_speed(v, vf, s, v0)
                want, acc = idm_double(v, vf, s, v0, p["a"], p["b"], p["s0"], p["T"], p["dt"])
                # a few binary32 roundings of terms as large as |acc*dt|
                tol = 16 * 2.0 ** -24 * (abs(v) + abs(acc) * p["dt"] + p["a"] * p["dt"]) + 1e-7
                assert abs(got - want) <= tol, (v, vf, s, v0, got, want)
                worst = max(worst, abs(got - want))
    assert worst < 1e-2


def test_idm_free_road_limit():
    """s -> infinity: acceleration a*(1 - (v/v0)^4)."""
    p = P0
    for v in [0.0, 4.0, 10.0, 13.9]:
        got = O.idm_speed(v, v, 1e7, 13.9)
        want = v + p["a"] * (1 - (v / 13.9) ** 4) * p["dt"]
        assert abs(got - want) < 1e-5


def test_idm_catches_dropped_terms():
    """The closed form distinguishes the approach-rate term and the exponent:
    variants with either changed disagree with the oracle by far more than
    the tolerance used above."""
    p = P0
    v, vf, s, v0 = 13.9, 3.0, 20.0, 13.9
    got = O.idm_speed(v, vf, s, v0)
    no_dv, _ = idm_double(v, v, s, v0, p["a"], p["b"], p["s0"], p["T"], p["dt"])
    assert abs(got - no_dv) > 0.5
    s_star = p["s0"] + v * p["T"] + v * (v - vf) / (2 * math.sqrt(p["a"] * p["b"]))
    delta2 = max(0.0, v + p["a"] * (1 - (v / 8.0) ** 2 - (s_star / s) ** 2) * p["dt"])
    assert abs(O.idm_speed(v, vf, s, 8.0) - delta2) > 0.1


# ---------------------------------------------------------------- lane-map example

def _golden(name):
    out = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                k, v = line.split()
                out[k] = int(v)
    return out


def test_lane_map_worked_example():
    g = _golden("lane_map_example.txt")
    net = make_net(2, [(0, 1, float(g["edge_len_m"]), g["lanes"], 5.0)])
    o = O.Oracle(net)
    o.load_demand(make_demand([(0, [0])]))
    m = o.lane_map()
    assert m.size == g["cells"]
    assert np.all(m == g["empty"])
    o.step(1)
    m = o.lane_map()
    # the departed vehicle sits in cell 0 of lane 0 (target lane of a final edge) at speed 0
    assert m[0] == 0 and np.count_nonzero(m != g["empty"]) == 1
    o.step(1)
    m = o.lane_map()
    st = o.state()
    assert st["status"][0] == 1 and st["x"][0] == F(2.5)  # 5 m/s * 0.5 s
    assert m[2] == 5 and np.count_nonzero(m != 255) == 1


def test_speed_byte_saturates_at_254():
    g = _golden("lane_map_example.txt")
    net = make_net(2, [(0, 1, 2000.0, 1, 254.0)])
    o = O.Oracle(net, dict(dt=0.01))
    o.load_demand(make_demand([(0, [0])]))
    o.step(2)
    m = o.lane_map()
    occ = m[m != 255]
    assert occ.tolist() == [g["max_speed_byte"]]


# -------------------------------------------------------------------- free flow

def test_free_flow_arrival_closed_form():
    # chain 0 -> 1 -> 2 -> 3, all nodes uncontrolled; v0*dt = 7, 3, 6.95 m
    net = make_net(4, [(0, 1, 100.0, 1, 14.0), (1, 2, 37.0, 2, 6.0), (2, 3, 400.0, 2, 13.9)])
    kd = 3
    o = run_oracle(net, [(kd, [0, 1, 2])], 0)
    o.step(kd + 1)
    st = o.state()
    assert st["status"][0] == 1 and st["x"][0] == 0.0
    xs = []
    for _ in range(14):
        o.step(1)
        xs.append(float(o.state()["x"][0]))
    assert xs == [7.0 * j for j in range(1, 15)]  # exact multiples on the first edge
    o.step(500)
    tr = o.trips()
    # ceil(100/7) = 15, ceil(37/3) = 13, 57*6.95 < 400 <= 58*6.95
    assert tr["depart"][0] == kd + 1
    assert tr["arrive"][0] == kd + 1 + 15 + 13 + 58


def test_free_flow_grid_link_is_58_steps():
    """Config-1 link: 400 m at 13.9 m/s, dt = 0.5 s: 58 steps per link."""
    net = make_net(3, [(0, 1, 400.0, 2, 13.9), (1, 2, 400.0, 2, 13.9)])
    o = run_oracle(net, [(0, [0, 1])], 200)
    assert o.trips()["arrive"][0] == 0 + 1 + 58 + 58


# ---------------------------------------------------------------------- signals

def _signal_net(G, approach_rank=None):
    # e0: 0->1 (50 m, 7 m/step: reaches the stop line on its 8th step)
    # e1: 1->2 (21 m, 3 steps); e2: 3->1, e3: 4->1 extra approaches
    return make_net(5, [(0, 1, 50.0, 1, 14.0), (1, 2, 21.0, 1, 14.0), (3, 1, 30.0, 1, 14.0),
                        (4, 1, 30.0, 1, 14.0)], green={1: G}, approach_rank=approach_rank)


@pytest.mark.parametrize("kd", [0, 5, 11, 12, 30, 51, 52, 70])
def test_signal_wait_closed_form(kd):
    G = 20
    o = run_oracle(_signal_net(G), [(kd, [0, 1])], kd + 200)
    k_reach = kd + 8
    phases = 3  # approaches e0, e2, e3 ranked 0, 1, 2 by edge id
    k_cross = next(k for k in range(k_reach, k_reach + 200) if (k // G) % phases == 0)
    assert o.trips()["arrive"][0] == k_cross + 3 + 1


@pytest.mark.parametrize("kd", [0, 12, 25, 33])
def test_two_phase_signal_closed_form(kd):
    """Explicit ranks: e0 and e3 share phase 1, e2 has phase 0 -> 2 phases."""
    G = 20
    o = run_oracle(_signal_net(G, approach_rank=[1, 0, 0, 1]), [(kd, [0, 1])], kd + 200)
    k_reach = kd + 8
    k_cross = next(k for k in range(k_reach, k_reach + 200) if (k // G) % 2 == 1)
    assert o.trips()["arrive"][0] == k_cross + 3 + 1


# ------------------------------------------------------------------ departures

@pytest.mark.parametrize("lanes,gap", [(1, 2), (2, 1), (3, 1)])
def test_departure_headway(lanes, gap):
    """Vehicles queued on one first edge leave one per step when another lane's
    first cell is free, else one every two steps (cell 0 must be empty in the
    step-k map, and a vehicle placed there leaves it the next step)."""
    net = make_net(2, [(0, 1, 500.0, lanes, 10.0)])
    n = 8
    o = run_oracle(net, [(0, [0]) for _ in range(n)], 40)
    dep = o.trips()["depart"]
    assert dep.tolist() == [1 + gap * j for j in range(n)]


def test_departure_respects_depart_step_and_order():
    net = make_net(2, [(0, 1, 500.0, 1, 10.0)])
    # input order is not departure order: ids follow a stable sort by step
    trips = [(9, [0]), (2, [0]), (2, [0]), (0, [0])]
    o = O.Oracle(net)
    vid = o.load_demand(make_demand(trips))
    assert vid.tolist() == [3, 1, 2, 0]
    o.step(30)
    dep = o.trips()["depart"]
    assert dep.tolist() == [1, 3, 5, 10]


# --------------------------------------------------------- saturation discharge

def test_saturation_discharge_one_every_two_steps():
    """A standing single-lane queue discharging into an empty single-lane
    link on green: one crossing every 2 steps, ceil(G/2) per green."""
    G = 60
    # e0: 0->1 queue link (600 m), e1: 1->2 long exit, e2: 3->1 cross street
    net = make_net(4, [(0, 1, 600.0, 1, 10.0), (1, 2, 2000.0, 1, 10.0), (3, 1, 50.0, 1, 10.0)],
                   green={1: G})
    n = 200
    o = run_oracle(net, [(0, [0, 1]) for _ in range(n)], 0)
    exits_per_step = []
    for k in range(840):
        before = int(o.link_stats()["exits"][0])
        o.step(1)
        exits_per_step.append(int(o.link_stats()["exits"][0]) - before)
    # e0 is green in [0,60), [120,180), ...; look at full greens with a long queue
    for start in (480, 600, 720):
        window = exits_per_step[start:start + G]
        assert sum(window) == math.ceil(G / 2), (start, window)
        assert window == [1, 0] * (G // 2)
        assert sum(exits_per_step[start + G:start + 2 * G]) == 0  # red


# ----------------------------------------------------------------- no-crash gap

def test_standstill_gap_is_s0():
    """A vehicle catching up with a vehicle stopped at a red stop line ends at
    exactly c_f - s0 with speed 0, and never beyond it."""
    # e0: 0->1 (200 m, 1 lane) ends at a signal whose phase (rank 1) stays
    # red for the first 10,000 steps
    net2 = make_net(4, [(0, 1, 200.0, 1, 14.0), (1, 2, 50.0, 1, 14.0), (3, 1, 30.0, 1, 14.0)],
                    green={1: 10_000}, approach_rank=[1, 0, 0])
    o = run_oracle(net2, [(0, [0, 1]), (10, [0, 1])], 0)
    xs = []
    for _ in range(150):
        o.step(1)
        st = o.state()
        xs.append((float(st["x"][0]), float(st["x"][1]), float(st["v"][1])))
    x0, x1, v1 = xs[-1]
    assert x0 == 199.0  # L - 1 at the stop line
    assert x1 == 197.0 and v1 == 0.0  # c_f - s0
    assert all(b <= 197.0 for _, b, _ in xs)


def test_follower_inside_d_front_uses_idm():
    """Leader parked 10 m ahead of a follower doing 13.9 m/s: 10 <= 2*dt*v, so
    the follower's new speed is the IDM speed, not the speed limit."""
    net = make_net(4, [(0, 1, 300.0, 1, 13.9), (1, 2, 50.0, 1, 13.9), (3, 1, 30.0, 1, 13.9)],
                   green={1: 10_000}, approach_rank=[1, 0, 0])
    o = run_oracle(net, [(0, [0, 1]), (30, [0, 1])], 0)
    seen_idm = False
    prev = None
    for _ in range(120):
        st = o.state()
        m = o.lane_map()
        if st["status"][1] == 1 and st["status"][0] == 1:
            x1, v1 = F(st["x"][1]), F(st["v"][1])
            cf = int(st["x"][0])
            s = F(F(cf) - x1)
            prev = (x1, v1, cf, s, F(m[cf]))
        o.step(1)
        st2 = o.state()
        if prev is not None and prev[3] <= F(F(2.0 * 0.5) * prev[1]) and prev[1] > 0:
            want = F(O.idm_speed(float(prev[1]), float(prev[4]), float(prev[3]), 13.9))
            xn = F(prev[0] + F(want * F(0.5)))
            if xn <= F(F(prev[2]) - F(2.0)):
                assert F(st2["v"][1]) == want
                seen_idm = True
        prev = None
    assert seen_idm


# --------------------------------------------------------------- lane changing

def test_lane_change_draw_matches_splitmix64():
    """u = top 24 bits of SplitMix64 / 2^24: reference values of the published
    output function for a few inputs, computed here with Python integers."""
    # SplitMix64 with state increment 0x9E3779B97F4A7C15 from seed 0 gives, as
    # its first output, mix(0x9E3779B97F4A7C15) = 0xE220A8397B1DCDAF
    assert splitmix64_mix(0x9E3779B97F4A7C15) == 0xE220A8397B1DCDAF
    assert 0.0 <= unit24(splitmix64_mix(12345)) < 1.0


def _lane_change_trace(seed, eps_amp=0.0):
    import workloads as W
    net = W.planar_network(24, 24, seed=seed)
    dem = W.route(net, W.gravity_demand(net, 2500, seed + 7, zones_x=4, zones_y=4, access_per_zone=3,
                                        beta_m=1500.0, peaks_h=(0.04, 0.08), peak_sigma_h=0.04))
    params = dict(seed=seed * 11 + 3, eps_amp=eps_amp)
    o = O.Oracle(net, params)
    o.load_demand(dem)
    return net, dem, o, dict(O.DEFAULT_PARAMS, **params)


@pytest.mark.parametrize("seed,eps_amp", [(5, 0.0), (6, 1.5)])
def test_lane_change_rule(seed, eps_amp):
    """Every accepted lane change follows the rule: intent drawn with
    probability 1 - x_rem/x0, direction toward the target lane, upward moves
    on odd steps only, critical gaps met in the step-k map, x' >= 1 cell; and
    an intender that met the gaps but stayed had its target cell reserved."""
    net, dem, o, p = _lane_change_trace(seed, eps_amp)
    off = dem["route_off"].astype(np.int64)
    vid = np.argsort(np.argsort(dem["depart_step"], kind="stable"), kind="stable")
    routes = {}
    for j in range(len(dem["depart_step"])):
        routes[int(vid[j])] = dem["route_edges"][off[j]:off[j + 1]]
    ne = net["n_edges"]
    ncell = np.maximum(1, np.ceil(net["edge_len"].astype(np.float32))).astype(np.int64)
    lanes = net["edge_lanes"].astype(np.int64)
    moff = np.concatenate([[0], np.cumsum(ncell * lanes)])
    out_rank = np.zeros(ne, np.int64)
    n_out = np.bincount(net["edge_src"], minlength=net["n_nodes"])
    for node in range(net["n_nodes"]):
        es = np.nonzero(net["edge_src"] == node)[0]
        out_rank[es] = np.arange(len(es))
    changes = stays = 0
    for k in range(600):
        st0, m0 = o.state(), o.lane_map()
        o.step(1)
        st1, m1 = o.state(), o.lane_map()
        for i in np.nonzero((st0["status"] == 1) & (st1["status"] == 1) & (st0["edge"] == st1["edge"]))[0]:
            e = int(st0["edge"][i])
            r = int(st0["ridx"][i])
            route = routes[int(i)]
            if lanes[e] == 1 or r == len(route) - 1:
                assert st1["lane"][i] == st0["lane"][i]
                continue
            if int(st1["x"][i]) == ncell[e] - 1 and st1["v"][i] == 0:
                # held at the stop line: reached the edge end, so no lane change
                assert st1["lane"][i] == st0["lane"][i]
                continue
            nxt = int(route[r + 1])
            tl = out_rank[nxt] * lanes[e] // n_out[net["edge_dst"][e]]
            ln = int(st0["lane"][i])
            x, xn, vn = F(st0["x"][i]), F(st1["x"][i]), F(st1["v"][i])
            intent = False
            if tl != ln:
                d = 1 if tl > ln else -1
                if (d > 0) == (k % 2 == 1):
                    L = F(ncell[e])
                    xrem = F(L - x)
                    mprob = F(0) if xrem >= F(p["x0"]) else F(F(1) - F(xrem / F(p["x0"])))
                    h = splitmix64_mix(p["seed"] ^ ((int(i) * 0x9E3779B97F4A7C15) & (2**64 - 1))
                                       ^ ((k * 0xD1B54A32D192ED03) & (2**64 - 1)))
                    intent = bool(unit24(h) < mprob)
            changed = int(st1["lane"][i]) != ln
            if not intent:
                assert not changed
                continue
            ln2 = ln + d
            row = m0[moff[e] + ln2 * ncell[e]: moff[e] + (ln2 + 1) * ncell[e]]
            c0 = int(x)
            ahead = [c for c in range(c0, min(c0 + 64, ncell[e])) if row[c] != 255]
            behind = [c for c in range(max(0, c0 - 64), c0) if row[c] != 255]
            eps_a = eps_b = F(0)
            if p["eps_amp"] > 0:
                ea = unit24(splitmix64_mix(h ^ 0x632BE59BD9B4E019))
                eb = unit24(splitmix64_mix(h ^ 0x8CB92BA72F3D8DD7))
                eps_a = F(F(p["eps_amp"]) * F(F(F(2) * ea) - F(1)))
                eps_b = F(F(p["eps_amp"]) * F(F(F(2) * eb) - F(1)))
            ok = True
            if ahead:
                ca = ahead[0]
                G = F(F(F(p["g_a"]) + max(F(0), F(F(F(p["alpha_i"]) * vn) - F(F(p["alpha_a"]) * F(row[ca]))))) + eps_a)
                ok &= bool(F(F(ca) - xn) >= G)
            if behind:
                cb = behind[-1]
                G = F(F(F(p["g_b"]) + max(F(0), F(F(F(p["alpha_b"]) * F(row[cb])) - F(F(p["alpha_i"]) * vn)))) + eps_b)
                ok &= bool(F(xn - F(cb)) >= G)
            ok &= int(xn) >= 1
            if changed:
                assert int(st1["lane"][i]) == ln2 and ok
                changes += 1
            elif ok:
                # stayed although the gaps were fine: the target cell was reserved
                c = int(xn)
                occ2 = m1[moff[e] + ln2 * ncell[e] + c] != 255
                ln3 = ln2 + d
                occ3 = 0 <= ln3 < lanes[e] and m1[moff[e] + ln3 * ncell[e] + c] != 255
                assert occ2 or occ3
                stays += 1
    assert changes > 20


# ------------------------------------------------------------------ invariants

def _invariant_run(net, dem, steps, params=None, every=1):
    o = O.Oracle(net, params or {})
    o.load_demand(dem)
    n = len(dem["depart_step"])
    ncell = np.maximum(1, np.ceil(net["edge_len"].astype(np.float32))).astype(np.int64)
    lanes = net["edge_lanes"].astype(np.int64)
    moff = np.concatenate([[0], np.cumsum(ncell * lanes)])
    prev = o.state()
    fifo_in, fifo_out = {}, {}
    for k in range(steps):
        o.step(1)
        st = o.state()
        c = o.counters()
        act = st["status"] == 1
        assert c["active"] == act.sum()
        assert c["waiting"] + c["active"] + c["arrived"] == n
        assert (st["status"] == 2).sum() == c["arrived"]
        # the lane map holds exactly the active vehicles, each at its speed byte
        if k % every == 0:
            m = o.lane_map()
            e, ln, x, v = st["edge"][act], st["lane"][act].astype(np.int64), st["x"][act], st["v"][act]
            idx = moff[e] + ln * ncell[e] + x.astype(np.int64)
            assert len(np.unique(idx)) == len(idx)
            assert np.count_nonzero(m != 255) == len(idx)
            assert np.all(m[idx] == np.minimum(v, 254).astype(np.uint8))
            assert np.all(x >= 0) and np.all(x < ncell[e])
            # a vehicle entering an edge keeps the speed it crossed at, so the
            # bound is the fastest speed limit of the network
            assert np.all(v >= 0) and np.all(v <= net["edge_vmax"].max())
            ls = o.link_stats()
            on_edge = np.bincount(e, minlength=net["n_edges"])
            assert np.all(ls["entries"].astype(np.int64) - ls["exits"].astype(np.int64) == on_edge)
        # no backward motion on the same edge
        same = (prev["status"] == 1) & act & (prev["edge"] == st["edge"])
        assert np.all(st["x"][same] >= prev["x"][same])
        # FIFO bookkeeping on single-lane edges
        moved = (prev["status"] == 1) & ((st["status"] == 2) | (prev["edge"] != st["edge"]))
        for i in np.nonzero(moved)[0]:
            e0 = int(prev["edge"][i])
            if lanes[e0] == 1:
                fifo_out.setdefault(e0, []).append(int(i))
        entered = act & ((prev["status"] != 1) | (prev["edge"] != st["edge"]))
        for i in np.nonzero(entered)[0]:
            e1 = int(st["edge"][i])
            if lanes[e1] == 1:
                fifo_in.setdefault(e1, []).append(int(i))
        prev = st
    for e0, outs in fifo_out.items():
        assert outs == fifo_in.get(e0, [])[:len(outs)], e0
    return o


def test_invariants_grid(grid_day):
    net, dem = grid_day
    o = _invariant_run(net, dem, 900, every=7)
    assert o.counters()["arrived"] > 100


def test_invariants_planar_single_lane_fifo():
    import workloads as W
    net = W.planar_network(30, 30, seed=9)
    dem = W.route(net, W.gravity_demand(net, 3000, 19, zones_x=5, zones_y=5, access_per_zone=3,
                                        beta_m=2000.0, peaks_h=(0.04, 0.08), peak_sigma_h=0.04))
    o = _invariant_run(net, dem, 1200, every=5)
    c = o.counters()
    assert c["arrived"] > 500 and c["lane_changes"] > 10


def test_link_stats_bins():
    """Binned inflow equals per-edge entries; traversal sums by entry bin add
    up to the per-edge totals; occupancy samples count the vehicles on the
    edge at the first step of each bin."""
    import workloads as W
    net, dem = W.grid_day(seed=4, n_trips=800)
    bs, nb = 300, 20
    o = O.Oracle(net, dict(bin_steps=bs, n_bins=nb))
    o.load_demand(dem)
    occ_expected = np.zeros((net["n_edges"], nb), np.int64)
    for b in range(nb):
        st = o.state()
        act = st["status"] == 1
        occ_expected[:, b] = np.bincount(st["edge"][act], minlength=net["n_edges"])
        o.step(bs)
    ls = o.link_stats()
    # bins cover steps [0, 6000): every entry happens at k+1 <= 6000, the
    # last one at 6000 falls outside, so allow for that
    assert np.all(ls["inflow"].sum(axis=1) <= ls["entries"])
    assert ls["inflow"].sum() >= ls["entries"].sum() - 50
    assert np.array_equal(ls["tt_sum"].sum(axis=1).astype(np.uint64), ls["tt_steps"])
    assert np.array_equal(ls["tt_cnt"].sum(axis=1).astype(np.uint64), ls["exits"])
    assert np.array_equal(ls["occ"].astype(np.int64), occ_expected)


def test_rejects_bad_input():
    net = make_net(3, [(0, 1, 100.0, 1, 10.0), (1, 2, 100.0, 1, 10.0)])
    o = O.Oracle(net)
    with pytest.raises(O.OracleError):
        o.load_demand(make_demand([(0, [1, 0])]))  # not contiguous
    with pytest.raises(O.OracleError):
        O.Oracle(make_net(2, [(0, 1, 100.0, 5, 10.0)]))  # 5 lanes
    with pytest.raises(O.OracleError):
        O.Oracle(make_net(2, [(0, 1, 100.0, 1, 300.0)]))  # speed above 254 m/s


def test_entry_conflict_lowest_id_wins():
    """Two vehicles reach an uncontrolled merge in the same step and ask for
    the same single lane: the lower id enters, the other waits at the stop
    line and enters two steps later (the first cell is still taken in the
    next step's map)."""
    # e0: 0->1 and e1: 2->1, both 14 m at 7 m/step (stop line reached on the 2nd step); e2: 1->3 exit
    net = make_net(4, [(0, 1, 14.0, 1, 14.0), (2, 1, 14.0, 1, 14.0), (1, 3, 700.0, 1, 14.0)])
    for first, second in (([1, 2], [0, 2]), ([0, 2], [1, 2])):
        o = O.Oracle(net)
        o.load_demand(make_demand([(0, first), (0, second)]))
        entered = {}
        for k in range(12):
            o.step(1)
            st = o.state()
            for i in (0, 1):
                if st["edge"][i] == 2 and i not in entered:
                    entered[i] = k
        # both depart at step 0 (different first edges), reach x' >= 14 in step 2
        assert entered == {0: 2, 1: 4}


def test_ring_of_one_cell_edges_gridlocks():
    """Four one-cell single-lane edges in a ring, one vehicle departing onto
    each at step 0: from step 1 on every vehicle reaches the end of its edge
    (v0 dt = 2.5 m >= 1 m) and asks for cell 0 of the next edge, which the
    vehicle ahead holds in the step-k map, so no lane is free and it holds at
    x = max(x, L - 1) = 0 with v = 0.  The state is a fixed point: nothing
    enters, leaves or moves, and each step adds four vehicle-steps."""
    net = make_net(4, [(0, 1, 1.0, 1, 5.0), (1, 2, 1.0, 1, 5.0), (2, 3, 1.0, 1, 5.0), (3, 0, 1.0, 1, 5.0)])
    trips = [(j // 4, [(j % 4 + q) % 4 for q in range(10)]) for j in range(16)]
    o = O.Oracle(net)
    o.load_demand(make_demand(trips))
    o.step(1)
    s1, m1 = o.state(), o.lane_map().copy()
    assert np.array_equal(m1, np.zeros(4, np.uint8))
    assert int((s1["status"] == 1).sum()) == 4
    for k in (2, 50, 3001):
        o.step(k - o.counters()["k"])
        c = o.counters()
        assert c == {"k": k, "veh_steps": 4 * (k - 1), "arrived": 0, "active": 4, "waiting": 12,
                     "lane_changes": 0}, c
        s = o.state()
        for key in ("status", "edge", "lane", "ridx", "x", "v"):
            assert np.array_equal(s[key], s1[key]), key
        assert np.array_equal(o.lane_map(), m1)
    ls = o.link_stats()
    assert np.array_equal(ls["entries"], np.ones(4, np.uint64)) and not ls["exits"].any()


# ----------------------------------------------------------------- vehicle types

TRUCK = dict(a=0.6, b=1.2, s0=4.0, T=2.0, vmax=10.0)  # top speed 10 m/s: 5 m per step, exactly
CAR = dict(a=1.0, b=1.5, s0=2.0, T=1.5, vmax=254.0)


def test_type_top_speed_free_flow_closed_form():
    """A lone vehicle's free-flow speed is the lower of the edge limit and its
    type's top speed (Algorithm 1: v <- v_free; vehicle type V): on 14 m/s
    edges a car covers 7 m per step and a 10 m/s truck 5 m, so they arrive
    after k_d + 1 + sum ceil(len / 7) and k_d + 1 + sum ceil(len / 5) steps;
    on a 6 m/s edge both are held to the limit (3 m per step)."""
    net = make_net(4, [(0, 1, 100.0, 1, 14.0), (1, 2, 37.0, 2, 6.0), (2, 3, 143.0, 1, 14.0)])
    o = O.Oracle(net, vehicle_types=[CAR, TRUCK])
    dem = make_demand([(2, [0, 1, 2]), (2, [0, 1, 2])])
    dem["vtype"] = np.array([0, 1], np.uint8)
    vid = o.load_demand(dem)
    o.step(400)
    tr = o.trips()
    car, truck = int(vid[0]), int(vid[1])
    assert tr["depart"][car] == 3  # ids by input order: the car enters first
    assert tr["arrive"][car] == 3 + math.ceil(100 / 7) + math.ceil(37 / 3) + math.ceil(143 / 7)
    # the truck enters two steps later (one departure every two steps from one lane)
    assert tr["depart"][truck] == 5
    assert tr["arrive"][truck] == 5 + math.ceil(100 / 5) + math.ceil(37 / 3) + math.ceil(143 / 5)


def test_type_standstill_gap():
    """Behind a vehicle stopped at a red stop line, a follower stops at
    c_f - s0 of its own type: 2 m for a car, 4 m for a truck."""
    net = make_net(4, [(0, 1, 200.0, 1, 14.0), (1, 2, 50.0, 1, 14.0), (3, 1, 30.0, 1, 14.0)],
                   green={1: 10_000}, approach_rank=[1, 0, 0])
    for ty, gap in ((0, 2.0), (1, 4.0)):
        o = O.Oracle(net, vehicle_types=[CAR, TRUCK])
        dem = make_demand([(0, [0, 1]), (10, [0, 1])])
        dem["vtype"] = np.array([0, ty], np.uint8)
        o.load_demand(dem)
        o.step(200)
        st = o.state()
        assert st["x"][0] == 199.0 and st["x"][1] == 199.0 - gap and st["v"][1] == 0.0


BIKE = dict(a=0.8, b=1.0, s0=1.0, T=1.0, vmax=4.5)


def test_type_idm_matches_double_closed_form():
    """A truck departing right behind a car on a long 10 m/s single-lane edge
    closes in on it: whenever the car is within d_front and the no-crash
    clamp does not bind, the truck's new speed is the IDM speed of the
    truck's own parameters (a, b, s0, T; free-flow speed min(edge limit,
    truck top speed)), within FP32 rounding of Treiber's formula in double
    precision."""
    net = make_net(3, [(0, 1, 1500.0, 1, 10.0), (1, 2, 50.0, 1, 10.0)])
    o = O.Oracle(net, vehicle_types=[CAR, TRUCK, BIKE])
    dem = make_demand([(0, [0, 1]), (0, [0, 1])])
    dem["vtype"] = np.array([0, 1], np.uint8)
    o.load_demand(dem)
    positive = 0
    for _ in range(600):
        st = o.state()
        o.step(1)
        nx = o.state()
        if not (st["status"][0] == 1 and st["status"][1] == 1 and st["edge"][0] == 0 and st["edge"][1] == 0):
            continue
        x1, v1 = float(st["x"][1]), float(st["v"][1])
        cf = int(st["x"][0])
        s = cf - x1
        vf = float(min(int(st["v"][0]), 254))  # the leader's speed byte
        if not (0 < s <= 2 * 0.5 * v1):
            continue
        want, _ = idm_double(v1, vf, s, 10.0, TRUCK["a"], TRUCK["b"], TRUCK["s0"], TRUCK["T"], 0.5)
        if x1 + want * 0.5 > cf - TRUCK["s0"]:
            continue  # the clamp binds
        assert abs(float(nx["v"][1]) - want) <= 1e-5 * max(1.0, want), (v1, vf, s, nx["v"][1], want)
        positive += want > 0
    assert positive > 0


def test_discretionary_lane_change_lets_a_car_pass_a_bike():
    """Discretionary lane change (an extension: the paper defines only the
    mandatory change): on a 1 km two-lane edge a bike (top speed 4.5 m/s)
    departs first and a car follows in the same lane.  With the rule off the
    car cannot pass (no mandatory change on its last edge) and arrives after
    the bike; with it on, the first odd step at which the bike holds it below
    its free speed (the bike slower than that speed, an empty lane above)
    moves it up one lane, and it arrives first."""
    types = [dict(a=1.0, b=1.5, s0=2.0, T=1.5, vmax=254.0), dict(a=0.8, b=1.0, s0=1.0, T=1.0, vmax=4.5)]
    net = make_net(2, [(0, 1, 1000.0, 2, 20.0)])
    dem = make_demand([(0, [0]), (4, [0])])
    dem["vtype"] = np.array([1, 0], np.uint8)
    arrive, lanes_seen = {}, {}
    for dlc in (0.0, 1.0):
        o = O.Oracle(net, dict(bin_steps=0, n_bins=0, dlc_prob=dlc, dlc_gain=5.0), vehicle_types=types)
        o.load_demand(dem)
        seen = set()
        for _ in range(600):
            o.step(1)
            st = o.state()
            if st["status"][1] == 1:
                seen.add(int(st["lane"][1]))
        arrive[dlc] = o.trips()["arrive"].tolist()
        lanes_seen[dlc] = seen
    bike, car = 0, 1
    assert arrive[0.0][car] > arrive[0.0][bike] and lanes_seen[0.0] == {0}
    assert arrive[1.0][car] < arrive[1.0][bike] and lanes_seen[1.0] == {0, 1}
