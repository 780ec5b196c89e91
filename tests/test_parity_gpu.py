"""GPU library against the CPU oracle, element by element, bit for bit, on
the same seeded inputs (IEEE binary32 state, integer statistics)."""
from __future__ import annotations

import numpy as np
import pytest

import workloads as W
from netutil import make_demand, make_net
from simutil import assert_outputs_equal, assert_state_equal, lockstep

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import paper_2406_08496_gb300 as L
    L.build()
    L.load_library()
    L.use_torch_allocator()


def test_grid_day_every_step(grid_day):
    """8x8 signalised grid, 2,000 trips over 30 min, 3,600 steps."""
    net, dem = grid_day
    lockstep(net, dem, dict(bin_steps=300, n_bins=12), 3600, check_every=25)


def test_grid_day_first_steps_each_step(grid_day):
    net, dem = grid_day
    lockstep(net, dem, {}, 400, check_every=1)


@pytest.mark.parametrize("gpu_params", [
    dict(block_size=128, blocks_per_sm=1, sort_period=1, chunk_steps=6),
    dict(block_size=512, blocks_per_sm=2, sort_period=7, chunk_steps=42),
    dict(block_size=256, blocks_per_sm=8, sort_period=32, flags=1),
    dict(block_size=256, blocks_per_sm=4, sort_period=128, chunk_steps=768),
])
def test_launch_configuration_invariance(grid_day, gpu_params):
    """Results do not depend on block size, grid size, sort period, sorting
    or graph chunking."""
    net, dem = grid_day
    lockstep(net, dem, dict(bin_steps=600, n_bins=6), 2000, check_every=250, gpu_params=gpu_params)


def test_small_regional_with_lane_changes():
    net = W.planar_network(40, 40, seed=21)
    dem = W.route(net, W.gravity_demand(net, 12000, 22, zones_x=6, zones_y=6, access_per_zone=3,
                                        beta_m=2500.0, peaks_h=(0.1, 0.25), peak_sigma_h=0.1))
    o, g = lockstep(net, dem, dict(bin_steps=450, n_bins=8, seed=99), 3000, check_every=100)
    assert o.counters()["lane_changes"] > 100


def test_random_gap_components():
    net = W.planar_network(32, 32, seed=8)
    dem = W.route(net, W.gravity_demand(net, 6000, 9, zones_x=4, zones_y=4, access_per_zone=2,
                                        beta_m=2000.0, peaks_h=(0.05, 0.15), peak_sigma_h=0.05))
    lockstep(net, dem, dict(eps_amp=1.5, x0=60.0, seed=7), 1500, check_every=50)


def test_tiny_scenarios():
    """The brute-force scenario family (merge, diverge, two signals, edges
    shorter than one step, 1-5 vehicles) on the GPU."""
    from test_oracle_bruteforce import scenario
    for seed in range(0, 120):
        net, trips, params = scenario(seed)
        lockstep(net, make_demand(trips), params, 70, check_every=1)


TYPES = [dict(a=1.0, b=1.5, s0=2.0, T=1.5, vmax=254.0), dict(a=0.6, b=1.2, s0=4.0, T=2.0, vmax=12.0),
         dict(a=0.8, b=1.0, s0=1.0, T=1.0, vmax=4.5)]


def _typed(dem, seed, weights=(0.7, 0.2, 0.1)):
    out = dict(dem)
    rng = np.random.default_rng(seed)
    out["vtype"] = rng.choice(len(TYPES), size=len(dem["depart_step"]), p=weights).astype(np.uint8)
    return out


def test_vehicle_types_grid_day(grid_day):
    """Cars, trucks and bikes (Algorithm 1 State: vehicle type; multimodal
    traffic, Sec. 5) on the 8x8 grid day, every 10 steps bit for bit."""
    net, dem = grid_day
    lockstep(net, _typed(dem, 3), dict(bin_steps=300, n_bins=12), 3600, check_every=10, vehicle_types=TYPES)


def test_vehicle_types_small_regional_with_lane_changes():
    net = W.planar_network(40, 40, seed=21)
    dem = W.route(net, W.gravity_demand(net, 12000, 22, zones_x=6, zones_y=6, access_per_zone=3,
                                        beta_m=2500.0, peaks_h=(0.1, 0.25), peak_sigma_h=0.1))
    o, g = lockstep(net, _typed(dem, 4), dict(bin_steps=450, n_bins=8, seed=99), 3000, check_every=100,
                    vehicle_types=TYPES)
    assert o.counters()["lane_changes"] > 100


def test_vehicle_types_tiny_scenarios():
    from test_oracle_bruteforce import TYPES as BF_TYPES
    from test_oracle_bruteforce import scenario
    for seed in range(1000, 1060):
        net, trips, params = scenario(seed)
        dem = make_demand(trips)
        dem["vtype"] = np.random.default_rng(seed + 7).integers(0, len(BF_TYPES), len(trips)).astype(np.uint8)
        lockstep(net, dem, params, 70, check_every=1, vehicle_types=BF_TYPES)


def test_discretionary_lane_changes_small_regional():
    """Discretionary lane changes on (an extension of the paper's mandatory
    rule) with cars, trucks and bikes on the small planar network, with
    random gap components: bit for bit every 100 steps, and the rule adds
    lane changes over the same run with it off."""
    net = W.planar_network(40, 40, seed=21)
    dem = W.route(net, W.gravity_demand(net, 12000, 22, zones_x=6, zones_y=6, access_per_zone=3,
                                        beta_m=2500.0, peaks_h=(0.1, 0.25), peak_sigma_h=0.1))
    base = dict(bin_steps=450, n_bins=8, seed=99, eps_amp=1.0)
    o, g = lockstep(net, _typed(dem, 4), dict(base, dlc_prob=0.3, dlc_gain=3.0), 3000, check_every=100,
                    vehicle_types=TYPES)
    o2, _ = lockstep(net, _typed(dem, 4), base, 3000, check_every=3000, vehicle_types=TYPES)
    assert o.counters()["lane_changes"] > o2.counters()["lane_changes"] + 100


@pytest.mark.parametrize("chunked", [False, True])
def test_discretionary_lane_changes_tiny_overtaking(chunked):
    """The brute force's overtaking family (long multi-lane edges, a bike
    departing ahead of cars and trucks) with the rule on: step by step in
    the grid-wide kernels, and in 24-step graph chunks, which these few
    trips run in the single-block light-load kernel."""
    from test_oracle_bruteforce import TYPES as BF_TYPES
    from test_oracle_bruteforce import scenario_overtaking
    for seed in range(2000, 2030):
        net, trips, params, vt = scenario_overtaking(seed)
        dem = make_demand(trips)
        dem["vtype"] = vt
        params.update(dlc_prob=1.0 if seed % 2 else 0.3, dlc_gain=float(seed % 3) * 4.0)
        if chunked:
            lockstep(net, dem, params, 120, check_every=24, vehicle_types=BF_TYPES,
                     gpu_params=dict(sort_period=6, chunk_steps=24))
        else:
            lockstep(net, dem, params, 120, check_every=1, vehicle_types=BF_TYPES, gpu_params=dict(flags=4))


def test_busy_lanes_tiny():
    """The brute force's busy family (10-17 vehicles on long multi-lane edges
    with a diverge), the mandatory rule alone and with the discretionary one,
    every step."""
    from test_oracle_bruteforce import TYPES as BF_TYPES
    from test_oracle_bruteforce import scenario_overtaking
    for seed in range(3000, 3020):
        for dlc in (0.0, 1.0):
            net, trips, params, vt = scenario_overtaking(seed, busy=True)
            dem = make_demand(trips)
            dem["vtype"] = vt
            params.update(dlc_prob=dlc, dlc_gain=3.0)
            lockstep(net, dem, params, 150, check_every=1, vehicle_types=BF_TYPES, gpu_params=dict(flags=4))


def test_edge_cases():
    # one-cell edges, 4 lanes, single-edge routes, far-future departure, a
    # queue of 30 vehicles released at once onto a one-lane edge
    net = make_net(5, [(0, 1, 0.4, 4, 13.9), (1, 2, 1.0, 1, 30.0), (2, 3, 250.0, 2, 5.5), (3, 4, 3.0, 4, 254.0),
                       (4, 0, 33.3, 3, 11.1)], green={2: 4, 3: 1})
    trips = [(0, [0, 1, 2, 3, 4]) for _ in range(30)] + [(5, [2]), (1000, [4, 0]), (3, [1, 2, 3])]
    lockstep(net, make_demand(trips), dict(bin_steps=50, n_bins=30), 1200, check_every=1)


def test_run_until_done_matches_oracle(grid_day):
    import oracle as O
    from paper_2406_08496_gb300 import Simulation
    net, dem = grid_day
    o = O.Oracle(net, {})
    o.load_demand(dem)
    g = Simulation(net, {})
    g.load_demand(dem)
    ro = o.run(20000)
    rg = g.run(20000)
    for key in ("steps", "veh_steps", "arrived", "active", "waiting", "k"):
        assert ro[key] == rg[key], (key, ro[key], rg[key])
    assert_outputs_equal(o, g)


def test_reset_replays_identically(grid_day):
    from paper_2406_08496_gb300 import Simulation
    net, dem = grid_day
    g = Simulation(net, dict(bin_steps=600, n_bins=6))
    g.load_demand(dem)
    g.step(1500)
    s1, t1, l1 = g.state(), g.trips(), g.link_stats()
    g.reset()
    g.step(700)
    g.step(800)
    assert_state_equal(s1, g.state())
    assert np.array_equal(t1["arrive"], g.trips()["arrive"])
    assert np.array_equal(l1["inflow"], g.link_stats()["inflow"])


@pytest.mark.parametrize("chunk_steps", [384, 42])
def test_idle_hours_match_oracle(grid_day, chunk_steps):
    """Two waves of departures eight simulated hours apart: the network
    empties between them (the library jumps over the idle steps) and every
    output still matches the oracle, which steps through all of them; so do
    runs that stop inside the idle stretch and resume."""
    import oracle as O
    import workloads as Wk
    from paper_2406_08496_gb300 import Simulation
    net, dem = grid_day
    keep = np.zeros(len(dem["depart_step"]), bool)
    keep[::4] = True
    sub = Wk.subset_trips(dem, keep)
    dep = sub["depart_step"].astype(np.int64)
    dep[1::2] += 8 * 7200
    sub["depart_step"] = dep.astype(np.uint32)
    params = dict(bin_steps=3600, n_bins=20)
    o = O.Oracle(net, params)
    o.load_demand(sub)
    g = Simulation(net, dict(params, chunk_steps=chunk_steps))
    g.load_demand(sub)
    for n in (9000, 20000, 10000):  # the second call starts and ends inside the idle stretch
        o.step(n)
        g.step(n)
        assert_state_equal(o.state(), g.state(), f"after {n}")
    ro = o.run(40000)
    rg = g.run(40000)
    for key in ("steps", "veh_steps", "arrived", "active", "waiting", "k"):
        assert ro[key] == rg[key], (key, ro[key], rg[key])
    assert_outputs_equal(o, g, n_bins=20)


@pytest.mark.parametrize("flags", [0, 8])
def test_lane_maps_on_chip_match_oracle(flags):
    """A 4x4 grid (38 KB of lane map): the light-load kernel keeps all five
    lane maps in its shared memory for each chunk (flags 8 =
    LPSIM_F_SHARED_MAPS) or in global memory (flags 0); both match the oracle bit for bit
    at every chunk boundary, in the outputs and with lane changes on (the
    discretionary rule too), and the maps read back equal."""
    import oracle as O
    from paper_2406_08496_gb300 import Simulation
    net = W.grid_network(4, 4)
    dem = W.route(net, W.uniform_demand(net, 1200, 5))
    params = dict(bin_steps=600, n_bins=8, dlc_prob=0.3, dlc_gain=3.0, eps_amp=1.0)
    o = O.Oracle(net, params)
    o.load_demand(dem)
    g = Simulation(net, dict(params, flags=flags | 2))
    g.load_demand(dem)
    for _ in range(3):
        o.step(1536)
        g.step(1536)
        assert_state_equal(o.state(), g.state(), f"step {o.counters()['k']}")
        assert np.array_equal(o.lane_map(), g.lane_map())
    ro, rg = o.run(20000), g.run(20000)
    for key in ("steps", "veh_steps", "arrived", "active", "waiting", "k"):
        assert ro[key] == rg[key], (key, ro[key], rg[key])
    assert_outputs_equal(o, g, n_bins=8)
    co, cg = o.counters(), g.counters()
    assert co["lane_changes"] == cg["lane_changes"] and co["lane_changes"] > 0
    assert g.counters()["light_chunks"] >= 3


@pytest.mark.parametrize("flags", [0, 4])
def test_light_load_chunks_match_oracle(grid_day, flags):
    """A quarter of the grid day's trips: at most 1,536 trips are ever due
    and not yet arrived, so every graph chunk runs in the single-block
    light-load kernel (flags 0) or in the grid-wide kernels (flags 4 =
    LPSIM_F_NO_LIGHT); both match the oracle bit for bit at every chunk
    boundary and at the end."""
    import oracle as O
    import workloads as Wk
    from paper_2406_08496_gb300 import Simulation
    net, dem = grid_day
    keep = np.zeros(len(dem["depart_step"]), bool)
    keep[::4] = True
    sub = Wk.subset_trips(dem, keep)
    params = dict(bin_steps=600, n_bins=8)
    o = O.Oracle(net, params)
    o.load_demand(sub)
    g = Simulation(net, dict(params, flags=flags))
    g.load_demand(sub)
    for _ in range(2):
        o.step(1536)  # one graph chunk at the default chunk length
        g.step(1536)
        assert_state_equal(o.state(), g.state(), f"step {o.counters()['k']}")
    ro = o.run(20000)
    rg = g.run(20000)
    for key in ("steps", "veh_steps", "arrived", "active", "waiting", "k"):
        assert ro[key] == rg[key], (key, ro[key], rg[key])
    assert_outputs_equal(o, g, n_bins=8)
    co, cg = o.counters(), g.counters()
    assert co["lane_changes"] == cg["lane_changes"]


def test_light_and_grid_wide_chunks_alternate():
    """8,000 trips on a 12x12 grid: the chunks switch between the grid-wide
    kernels and the light-load block as the network fills and drains; every
    output matches the oracle."""
    import oracle as O
    from paper_2406_08496_gb300 import Simulation
    net = W.grid_network(12, 12)
    dem = W.route(net, W.uniform_demand(net, 8000, 11, t_max_s=3600.0))
    params = dict(bin_steps=1200, n_bins=12)
    o = O.Oracle(net, params)
    o.load_demand(dem)
    g = Simulation(net, params)
    g.load_demand(dem)
    for _ in range(6):
        o.step(1536)
        g.step(1536)
        assert_state_equal(o.state(), g.state(), f"step {o.counters()['k']}")
    ro = o.run(60000)
    rg = g.run(60000)
    for key in ("steps", "veh_steps", "arrived", "active", "waiting", "k"):
        assert ro[key] == rg[key], (key, ro[key], rg[key])
    assert_outputs_equal(o, g, n_bins=12)


def test_light_kernel_lists_beyond_its_stages():
    """Every chunk in the light-load block (light_trips far above the trip
    count) while 6,000 trips leave a 12x12 grid within two minutes: hundreds
    of departure requests and crossing requests per step, more than the
    block's shared-memory stages hold, so the overflow through the global
    lists is exercised; every output matches the oracle."""
    import oracle as O
    from paper_2406_08496_gb300 import Simulation
    net = W.grid_network(12, 12)
    dem = W.route(net, W.uniform_demand(net, 6000, 13, t_max_s=120.0))
    params = dict(bin_steps=600, n_bins=6)
    o = O.Oracle(net, params)
    o.load_demand(dem)
    g = Simulation(net, dict(params, light_trips=10**9))
    g.load_demand(dem)
    for _ in range(2):
        o.step(1536)  # one light-load chunk each
        g.step(1536)
        assert_state_equal(o.state(), g.state(), f"step {o.counters()['k']}")
    ro = o.run(60000)
    rg = g.run(60000)
    for key in ("steps", "veh_steps", "arrived", "active", "waiting", "k"):
        assert ro[key] == rg[key], (key, ro[key], rg[key])
    assert_outputs_equal(o, g, n_bins=6)
    assert o.counters()["lane_changes"] == g.counters()["lane_changes"]


@pytest.mark.parametrize("seed,eps_amp", [(2, 6.0), (5, 10.0)])
@pytest.mark.parametrize("flags", [0, 4])
def test_stop_line_intents_beside_losing_crossers(seed, eps_amp, flags):
    """Short three-lane edges (60 m), 20-step greens and wide random gap
    components: lane-change intents that end on a stop-line cell pass the gap
    test (a dozen per run), and in each of these two runs one of them aims
    at the cell where a crosser of the target lane, losing its entry claim in
    the same step, is held.  step_p2 decides such an intent alongside the
    crossings from the target lane's crossing request and its claim; the
    run matches the oracle, which decides it after placing the holds.  With
    flags 4 no chunk runs in the light-load block."""
    import oracle as O
    from paper_2406_08496_gb300 import Simulation
    net = W.grid_network(8, 8, spacing=60.0, lanes=3, vmax=13.9, green_steps=20)
    dem = W.route(net, W.uniform_demand(net, 5000, seed, t_max_s=200.0))
    params = dict(bin_steps=600, n_bins=2, eps_amp=eps_amp)
    o = O.Oracle(net, params)
    o.load_demand(dem)
    g = Simulation(net, dict(params, flags=flags))
    g.load_demand(dem)
    o.step(768)
    g.step(768)
    assert_state_equal(o.state(), g.state(), f"step {o.counters()['k']}")
    ro = o.run(40000)
    rg = g.run(40000)
    for key in ("steps", "veh_steps", "arrived", "active", "waiting", "k"):
        assert ro[key] == rg[key], (key, ro[key], rg[key])
    assert_outputs_equal(o, g, n_bins=2)
    assert o.counters()["lane_changes"] == g.counters()["lane_changes"]


@pytest.mark.parametrize("flags", [4, 0])
def test_kernel_timing_direct_and_graph_steps(grid_day, flags):
    """Per-kernel span timing over direct steps and graph chunks alike (with
    and without light-load chunks), every launch accounted for, the spans
    summing to no more than the wall time, and the results unchanged."""
    import time

    import torch
    from paper_2406_08496_gb300 import Simulation
    net, dem = grid_day
    g = Simulation(net, dict(flags=flags))
    g.load_demand(dem)
    g.set_kernel_timing(True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    g.step(5)      # direct steps (not at a chunk boundary afterwards)
    g.step(1531)   # direct steps up to the chunk boundary (default chunk: 1,536 steps)
    g.step(3072)   # two graph chunks (or light-load chunks)
    torch.cuda.synchronize()
    wall_ms = (time.perf_counter() - t0) * 1e3
    kt = g.kernel_times()
    g.set_kernel_timing(False)
    vs = g.counters()["veh_steps"]
    n_light = kt["step_small"]["launches"]
    assert kt["step_p1"]["launches"] + 1536 * n_light == 4608, kt
    assert kt["step_p2"]["launches"] == kt["step_p1"]["launches"]
    # compaction every 256 steps, and once at the end of each light-load chunk
    assert kt["compact_sort"]["launches"] == (4608 - 1536 * n_light) // 256 + n_light, kt
    assert kt["step_p1"]["ms"] > 0 and kt["step_p2"]["ms"] > 0
    assert sum(v["ms"] for v in kt.values()) <= wall_ms
    if flags == 4:
        assert n_light == 0 and kt["step_p1"]["veh_steps"] == vs
    else:
        assert n_light > 0 and 0 < kt["step_p1"]["veh_steps"] < vs
    ref = Simulation(net, {})
    ref.load_demand(dem)
    ref.step(4608)
    assert_state_equal(ref.state(), g.state(), "timing on vs off")
