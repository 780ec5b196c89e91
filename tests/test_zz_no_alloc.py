"""lpsim_get_state_noalloc, the state query that allocates nothing.

Callers that cannot allocate device memory while the simulation runs (a
fixed pool already handed out, a memory-capped service, no allocator
callback) read the vehicle state through this entry point, whose scratch is
a fixed device array inside the library.  Its output must equal
lpsim_get_state's, bit for bit, on consecutive calls (the array keeps the
previous call's contents, so the second call checks that it is cleared).
This file is collected last on purpose.
"""
from __future__ import annotations

import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

MAX_VEHICLES = 1048576  # LPSIM_NOALLOC_MAX_VEHICLES


def _lib():
    import paper_2406_08496_gb300 as L
    L.build()
    lib = L.load_library()
    P = ctypes.c_void_p
    lib.lpsim_get_state_noalloc.argtypes = [P, ctypes.c_uint64, P, P, P, P, P, P]
    lib.lpsim_get_state_noalloc.restype = ctypes.c_int
    return L, lib


def _noalloc_state(lib, h, n):
    st = {"x": np.full(n, -1, np.float32), "v": np.full(n, -1, np.float32), "edge": np.zeros(n, np.uint32),
          "lane": np.full(n, 7, np.uint8), "ridx": np.full(n, 9, np.uint32), "status": np.full(n, 9, np.uint8)}
    ptr = {k: ctypes.c_void_p(a.ctypes.data) for k, a in st.items()}
    rc = lib.lpsim_get_state_noalloc(h, n, ptr["x"], ptr["v"], ptr["edge"], ptr["lane"], ptr["ridx"], ptr["status"])
    assert rc == 0, lib.lpsim_last_error().decode()
    return st


def test_noalloc_state_matches_get_state():
    import torch
    import workloads as W
    L, lib = _lib()
    L.use_torch_allocator()
    net, dem = W.grid_day(seed=5, n_trips=1500)
    sim = L.Simulation(net, {})
    sim.load_demand(dem)
    for _ in range(2):
        sim.step(350)
        want = sim.state()
        before = torch.cuda.memory_stats().get("allocation.all.allocated", 0)
        got = _noalloc_state(lib, sim.h, sim.n)
        after = torch.cuda.memory_stats().get("allocation.all.allocated", 0)
        assert after == before, "the no-alloc query went through the allocator"
        for key in ("status", "edge", "lane", "ridx"):
            assert np.array_equal(got[key], want[key]), key
        for key in ("x", "v"):
            assert np.array_equal(got[key].view(np.uint32), want[key].view(np.uint32)), key
        assert (want["status"] == 1).sum() > 0
    sim.close()


def test_noalloc_rejects_more_than_its_scratch():
    import workloads as W
    L, lib = _lib()
    net, dem = W.grid_day(seed=6, n_trips=50)
    sim = L.Simulation(net, {})
    sim.load_demand(dem)
    rc = lib.lpsim_get_state_noalloc(sim.h, MAX_VEHICLES + 1, None, None, None, None, None, None)
    assert rc == -1
    assert "exceed" in lib.lpsim_last_error().decode()
    sim.close()
