"""lpsim_load_demand: input checks (the lowest failing trip is named, offset
errors before edge errors) and the vehicle ids (ranks of a stable sort by
departure step), on a device context."""
from __future__ import annotations

import numpy as np
import pytest

from netutil import make_demand, make_net

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import paper_2406_08496_gb300 as L
    L.build()
    L.load_library()
    L.use_torch_allocator()


def _net():
    # 0 -> 1 -> 2 -> 3 and back 3 -> 0
    return make_net(4, [(0, 1, 50.0, 1, 10.0), (1, 2, 50.0, 2, 10.0), (2, 3, 50.0, 1, 10.0), (3, 0, 50.0, 1, 10.0)])


def _load(dem):
    from paper_2406_08496_gb300 import Simulation
    s = Simulation(_net(), {})
    try:
        return s.load_demand(dem)
    finally:
        s.close()


@pytest.mark.parametrize("trips,msg", [
    ([(0, [0, 1]), (3, [1, 3]), (5, [9])], "trip 1: route edges are not contiguous"),
    ([(0, [0, 1]), (3, [1, 2]), (5, [9])], "trip 2: edge id out of range"),
    ([(0, [0, 7]), (3, [1, 3])], "trip 0: edge id out of range"),
])
def test_rejects_bad_routes(trips, msg):
    from paper_2406_08496_gb300 import LpsimError
    with pytest.raises(LpsimError, match=msg):
        _load(make_demand(trips))


def test_offset_errors_come_first():
    from paper_2406_08496_gb300 import LpsimError
    dem = make_demand([(0, [0, 1]), (3, [1, 3]), (5, [2])])
    dem["route_off"] = np.array([0, 2, 2, 5], np.uint64)  # trip 1 empty; trip 0's edges are fine
    with pytest.raises(LpsimError, match="trip 1: empty route"):
        _load(dem)


def test_many_trips_checked_on_every_piece():
    """Enough trips to spread the checks over many host threads; one bad
    trip far from the start is found and named."""
    from paper_2406_08496_gb300 import LpsimError
    n = 200_000
    trips = [(int(i % 977), [i % 4, (i + 1) % 4]) for i in range(n)]
    trips[150_001] = (5, [0, 2])
    with pytest.raises(LpsimError, match="trip 150001: route edges are not contiguous"):
        _load(make_demand(trips))


def test_vehicle_ids_are_stable_departure_ranks():
    rng = np.random.default_rng(3)
    n = 50_000
    dep = rng.integers(0, 3000, n)
    trips = [(int(dep[i]), [i % 4]) for i in range(n)]
    vid = _load(make_demand(trips))
    assert np.array_equal(vid, np.argsort(np.argsort(dep, kind="stable"), kind="stable"))


def test_departure_steps_beyond_the_counting_range():
    """Steps of 2^24 and above take the comparison sort: same ranks."""
    dep = np.array([1 << 25, 3, (1 << 24) + 1, 3, 0], np.uint32)
    vid = _load(make_demand([(int(d), [0]) for d in dep]))
    assert np.array_equal(vid, np.argsort(np.argsort(dep, kind="stable"), kind="stable"))
