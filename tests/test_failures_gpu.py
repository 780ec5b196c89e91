"""Failure paths of the library, made on the host (no GPU fault, trap or hang):
a gridlocked network the run loop must report, device allocations that fail
at every point of the set-up, and a demand with no trips at all.

* Gridlock: four one-cell single-lane edges in a ring, one vehicle departing
  onto each at step 0.  From step 1 every vehicle asks for cell 0 of the next
  edge, which the vehicle ahead holds, so none can ever cross (the oracle pin
  `test_ring_of_one_cell_edges_gridlocks` fixes this).  The detector is a
  host check of the device counters after each graph chunk: no kernel waits
  on anything.
* Out of memory: an allocator callback that returns NULL on its N-th call,
  for every N the set-up makes; each must fail with LPSIM_E_OOM and leave no
  device allocation behind once the context is destroyed.
* Empty demand: a network with zero trips steps and runs like the oracle.
"""
from __future__ import annotations

import ctypes

import numpy as np
import pytest

import oracle as O
from netutil import make_demand, make_net
from simutil import assert_outputs_equal

pytestmark = pytest.mark.gpu

E_OOM = -2
E_GRIDLOCK = -6


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import paper_2406_08496_gb300 as L
    L.build()
    L.load_library()
    L.use_torch_allocator()
    yield
    L.use_torch_allocator()


def ring():
    net = make_net(4, [(0, 1, 1.0, 1, 5.0), (1, 2, 1.0, 1, 5.0), (2, 3, 1.0, 1, 5.0), (3, 0, 1.0, 1, 5.0)])
    trips = [(j // 4, [(j % 4 + q) % 4 for q in range(10)]) for j in range(16)]
    return net, make_demand(trips)


def test_gridlock_is_reported_and_state_matches_oracle():
    from paper_2406_08496_gb300 import LpsimError, Simulation
    net, dem = ring()
    g = Simulation(net, dict(gridlock_steps=500))
    g.load_demand(dem)
    with pytest.raises(LpsimError) as ei:
        g.run(20_000)
    assert ei.value.code == E_GRIDLOCK, str(ei.value)
    assert "no vehicle crossed, departed or arrived" in str(ei.value)
    c = g.counters()
    # detected at the first chunk boundary 500 or more steps after the last
    # departure (step 0); the state is the oracle's at that step
    assert 500 <= c["k"] <= 500 + 2 * 1536, c
    assert c["active"] == 4 and c["waiting"] == 12 and c["arrived"] == 0
    o = O.Oracle(net, {})
    o.load_demand(dem)
    o.step(c["k"])
    assert_outputs_equal(o, g, where="gridlocked ring")
    assert o.counters()["veh_steps"] == c["veh_steps"]
    g.close()


def test_gridlock_detector_off_runs_to_max_steps():
    from paper_2406_08496_gb300 import Simulation
    net, dem = ring()
    g = Simulation(net, dict(gridlock_steps=0))
    g.load_demand(dem)
    r = g.run(4000)
    assert r["steps"] == 4000 and r["arrived"] == 0 and r["active"] == 4
    g.close()


class _FailingAllocator:
    """Allocator callbacks that forward to cudaMalloc / cudaFree through
    torch, except that call number `fail_at` returns NULL."""

    def __init__(self, fail_at: int):
        import torch
        self.torch = torch
        self.fail_at = fail_at
        self.calls = 0
        self.live = {}

    def alloc(self, size, user):
        self.calls += 1
        if self.calls == self.fail_at:
            return None
        t = self.torch.empty(int(size), dtype=self.torch.uint8, device="cuda")
        self.live[t.data_ptr()] = t
        return t.data_ptr()

    def free(self, ptr, user):
        self.live.pop(int(ptr))


def _install(lib, fa):
    import paper_2406_08496_gb300 as L
    cbs = (L.ALLOC_T(fa.alloc), L.FREE_T(fa.free))
    assert lib.lpsim_set_allocator(cbs[0], cbs[1], None) == 0
    return cbs


def test_every_failing_allocation_gives_oom_and_frees_everything():
    import paper_2406_08496_gb300 as L
    import workloads as W
    lib = L.load_library()
    net, dem = W.grid_day(seed=2, n_trips=200)
    # how many allocations a full set-up makes
    fa = _FailingAllocator(fail_at=0)
    cbs = _install(lib, fa)
    s = L.Simulation(net, dict(bin_steps=100, n_bins=4))
    s.load_demand(dem)
    s.step(50)
    s.state()
    s.link_stats()
    total = fa.calls
    s.close()
    assert not fa.live, "destroy left allocations behind"
    assert total > 20
    failed_at = []
    for n in range(1, total + 1):
        fa = _FailingAllocator(fail_at=n)
        cbs = _install(lib, fa)
        err = None
        s = None
        try:
            s = L.Simulation(net, dict(bin_steps=100, n_bins=4))
            s.load_demand(dem)
            s.step(50)
            s.state()
            s.link_stats()
        except L.LpsimError as e:
            err = e
        if s is not None:
            s.close()
        assert err is not None, f"allocation {n} failed but no call reported it"
        assert err.code == E_OOM, (n, str(err))
        assert not fa.live, f"allocation {n} failed: {len(fa.live)} allocations left after destroy"
        failed_at.append(n)
    assert len(failed_at) == total
    del cbs
    L.use_torch_allocator()


def test_empty_demand_matches_oracle():
    import workloads as W
    from paper_2406_08496_gb300 import Simulation
    net, _ = W.grid_day(seed=1, n_trips=10)
    empty = {"depart_step": np.zeros(0, np.uint32), "route_off": np.zeros(1, np.uint64),
             "route_edges": np.zeros(0, np.uint32)}
    params = dict(bin_steps=100, n_bins=4)
    g = Simulation(net, params)
    assert len(g.load_demand(empty)) == 0
    r = g.run(5000)
    assert r["steps"] == 0 and r["veh_steps"] == 0 and r["arrived"] == 0
    g.step(2000)
    o = O.Oracle(net, params)
    o.load_demand(empty)
    o.step(2000)
    c = g.counters()
    assert c["k"] == 2000 and c["veh_steps"] == 0 and c["active"] == 0 and c["waiting"] == 0
    assert_outputs_equal(o, g, n_bins=4, where="empty demand")
    assert np.all(g.lane_map() == 255)
    g.close()
