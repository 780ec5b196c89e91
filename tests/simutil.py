"""Helpers shared by the GPU tests: run the oracle and the GPU library side
by side on the same seeded inputs and compare their outputs."""
from __future__ import annotations

import numpy as np

import oracle as O

STATE_KEYS = ("status", "edge", "lane", "ridx")


def assert_state_equal(a: dict, b: dict, where: str = "") -> None:
    for key in STATE_KEYS:
        if not np.array_equal(a[key], b[key]):
            bad = np.nonzero(a[key] != b[key])[0][:5]
            raise AssertionError(f"{where} {key} differs at ids {bad}: {a[key][bad]} vs {b[key][bad]}")
    for key in ("x", "v"):
        ab, bb = a[key].view(np.uint32), b[key].view(np.uint32)
        if not np.array_equal(ab, bb):
            bad = np.nonzero(ab != bb)[0][:5]
            raise AssertionError(f"{where} {key} differs at ids {bad}: {a[key][bad]} vs {b[key][bad]}")


def assert_outputs_equal(o, g, n_bins: int = 0, where: str = "") -> None:
    assert_state_equal(o.state(), g.state(), where)
    to, tg = o.trips(), g.trips()
    assert np.array_equal(to["depart"], tg["depart"]), where + " depart steps differ"
    assert np.array_equal(to["arrive"], tg["arrive"]), where + " arrival steps differ"
    lo, lg = o.link_stats(), g.link_stats()
    for key in ("entries", "exits", "tt_steps"):
        assert np.array_equal(lo[key], lg[key]), f"{where} link {key} differ"
    if n_bins:
        for key in ("inflow", "tt_sum", "tt_cnt", "occ"):
            assert np.array_equal(lo[key], lg[key]), f"{where} binned {key} differ"
    assert np.array_equal(o.lane_map(), g.lane_map()), where + " lane maps differ"


def lockstep(net: dict, dem: dict, params: dict, steps: int, check_every: int = 1, gpu_params: dict | None = None,
             vehicle_types: list | None = None):
    """Run oracle and GPU for `steps` steps, comparing state every
    `check_every` steps and all outputs at the end (vehicle_types: the
    types the demand's "vtype" array names, if any)."""
    from paper_2406_08496_gb300 import Simulation
    o = O.Oracle(net, params, vehicle_types=vehicle_types)
    vo = o.load_demand(dem)
    gp = dict(params, **(gpu_params or {}))
    gp["flags"] = gp.get("flags", 0) | 2  # LPSIM_F_CHECK_CELLS: every lane-map write must find an empty cell
    g = Simulation(net, gp, vehicle_types=vehicle_types)
    vg = g.load_demand(dem)
    assert np.array_equal(vo, vg)
    done = 0
    while done < steps:
        n = min(check_every, steps - done)
        o.step(n)
        g.step(n)
        done += n
        assert_state_equal(o.state(), g.state(), f"step {done}")
    assert_outputs_equal(o, g, int(params.get("n_bins", 0)), f"after {steps} steps")
    co, cg = o.counters(), g.counters()
    for key in ("veh_steps", "arrived", "active", "waiting", "lane_changes"):
        assert co[key] == cg[key], (key, co[key], cg[key])
    return o, g
