"""Seeded synthetic inputs: road networks, trip tables and routes.

This module is shared by the CPU oracle tests and the GPU path.  It holds
none of the simulation's arithmetic: it only draws networks and demand of
the shape the paper simulates (Sec. 4: a regional network of 224,223 nodes
and 549,008 edges; 2.82M to 9.01M car trips with AM/PM peaks) and routes
every trip along a free-flow shortest path, which the method takes as given
("the route path ... from the input demand data after the routing",
Sec. 3.1, Vehicle Data Information).

Every generator is a pure function of its arguments and seed.
"""
from __future__ import annotations

import ctypes
import hashlib
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB = None
_LIB_LOCK = threading.Lock()

# Road classes of the planar generator: (lanes, speed limit m/s).
ROAD_CLASSES = {
    "local": (1, 11.1),
    "collector": (2, 15.6),
    "arterial": (3, 22.2),
    "highway": (4, 30.0),
}


def _build_lib() -> str:
    src = os.path.join(_HERE, "route.c")
    with open(src, "rb") as f:
        tag = hashlib.sha1(f.read()).hexdigest()[:12]
    out = os.path.join(_HERE, f"_libwlroute_{tag}.so")
    if not os.path.exists(out):
        tmp = out + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-shared", "-fPIC", "-pthread", "-o", tmp, src])
        os.replace(tmp, out)
    return out


def _lib():
    global _LIB
    with _LIB_LOCK:
        if _LIB is None:
            lib = ctypes.CDLL(_build_lib())
            lib.wl_route.restype = ctypes.c_void_p
            lib.wl_route.argtypes = [ctypes.c_uint32, ctypes.c_uint32, ctypes.c_void_p, ctypes.c_void_p,
                                     ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p, ctypes.c_void_p,
                                     ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
            lib.wl_route_total.restype = ctypes.c_uint64
            lib.wl_route_total.argtypes = [ctypes.c_void_p]
            lib.wl_route_copy.restype = None
            lib.wl_route_copy.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
            lib.wl_route_free.restype = None
            lib.wl_route_free.argtypes = [ctypes.c_void_p]
            _LIB = lib
    return _LIB


def build() -> None:
    """Compile the routing helper (host C, no GPU)."""
    _lib()


def _ptr(a: np.ndarray) -> ctypes.c_void_p:
    return ctypes.c_void_p(a.ctypes.data)


# --------------------------------------------------------------------------------------
# networks
# --------------------------------------------------------------------------------------

def _finish_network(node_x, node_y, src, dst, length, lanes, vmax, cls_nonlocal, green_steps):
    n_nodes = len(node_x)
    n_in = np.bincount(dst, minlength=n_nodes)
    nonlocal_in = np.bincount(dst, weights=cls_nonlocal.astype(np.float64), minlength=n_nodes)
    return {
        "n_nodes": int(n_nodes),
        "n_edges": int(len(src)),
        "node_x": np.ascontiguousarray(node_x, dtype=np.float32),
        "node_y": np.ascontiguousarray(node_y, dtype=np.float32),
        "edge_src": np.ascontiguousarray(src, dtype=np.uint32),
        "edge_dst": np.ascontiguousarray(dst, dtype=np.uint32),
        "edge_len": np.ascontiguousarray(length, dtype=np.float32),
        "edge_lanes": np.ascontiguousarray(lanes, dtype=np.uint8),
        "edge_vmax": np.ascontiguousarray(vmax, dtype=np.float32),
        "_n_in": n_in,
        "_nonlocal_in": nonlocal_in,
        "node_green": None,
        "_green_steps": green_steps,
    }


def grid_network(rows: int = 8, cols: int = 8, spacing: float = 400.0, lanes: int = 2,
                 vmax: float = 13.9, green_steps: int = 60) -> dict:
    """Bidirectional grid.  Nodes with >= 3 approaches are signalised with
    `green_steps` per approach; the others are uncontrolled."""
    src, dst = [], []
    for r in range(rows):
        for c in range(cols):
            u = r * cols + c
            for dr, dc in ((-1, 0), (0, 1), (1, 0), (0, -1)):
                rr, cc = r + dr, c + dc
                if 0 <= rr < rows and 0 <= cc < cols:
                    src.append(u)
                    dst.append(rr * cols + cc)
    src = np.array(src, dtype=np.uint32)
    dst = np.array(dst, dtype=np.uint32)
    n_nodes = rows * cols
    node_x = (np.arange(n_nodes) % cols) * spacing
    node_y = (np.arange(n_nodes) // cols) * spacing
    m = len(src)
    net = _finish_network(node_x, node_y, src, dst, np.full(m, spacing), np.full(m, lanes),
                          np.full(m, vmax), np.zeros(m, dtype=bool), green_steps)
    net["node_green"] = np.where(net["_n_in"] >= 3, green_steps, 0).astype(np.uint32)
    return net


def _line_class(idx: np.ndarray) -> np.ndarray:
    """Road class of a lattice line by its index: 0 local, 1 collector, 2 arterial, 3 highway."""
    cls = np.zeros(idx.shape, dtype=np.int64)
    cls[idx % 4 == 0] = 1
    cls[idx % 10 == 0] = 2
    cls[idx % 40 == 0] = 3
    return cls


def planar_network(rows: int, cols: int, seed: int, spacing: float = 150.0, jitter: float = 0.3,
                   local_keep: float = 0.32, diag_p: float = 0.02, len_median: float = 150.0,
                   len_sigma: float = 0.6, green_steps: int = 60) -> dict:
    """Jittered planar lattice with road classes by line, random deletion of
    local links, sparse local diagonals, lognormal link lengths, restricted to
    its largest connected component (all links are two-way, so this is also
    the largest strongly connected component)."""
    from scipy.sparse import coo_matrix
    from scipy.sparse.csgraph import connected_components

    rng = np.random.default_rng(seed)
    n = rows * cols
    r_of = np.arange(n) // cols
    c_of = np.arange(n) % cols
    x = c_of * spacing + rng.uniform(-jitter, jitter, n) * spacing
    y = r_of * spacing + rng.uniform(-jitter, jitter, n) * spacing
    # horizontal links (r,c)-(r,c+1), class by row; vertical (r,c)-(r+1,c), class by column
    hr, hc = np.meshgrid(np.arange(rows), np.arange(cols - 1), indexing="ij")
    h_u = (hr * cols + hc).ravel()
    h_v = h_u + 1
    h_cls = _line_class(hr.ravel())
    vr, vc = np.meshgrid(np.arange(rows - 1), np.arange(cols), indexing="ij")
    v_u = (vr * cols + vc).ravel()
    v_v = v_u + cols
    v_cls = _line_class(vc.ravel())
    u = np.concatenate([h_u, v_u])
    v = np.concatenate([h_v, v_v])
    cls = np.concatenate([h_cls, v_cls])
    keep = (cls > 0) | (rng.random(len(u)) < local_keep)
    u, v, cls = u[keep], v[keep], cls[keep]
    # diagonals: at most one per lattice cell, so the graph stays planar
    dr, dc = np.meshgrid(np.arange(rows - 1), np.arange(cols - 1), indexing="ij")
    dr, dc = dr.ravel(), dc.ravel()
    has = rng.random(len(dr)) < diag_p
    flip = rng.random(len(dr)) < 0.5
    dr, dc, flip = dr[has], dc[has], flip[has]
    d_u = np.where(flip, dr * cols + dc + 1, dr * cols + dc)
    d_v = np.where(flip, (dr + 1) * cols + dc, (dr + 1) * cols + dc + 1)
    u = np.concatenate([u, d_u])
    v = np.concatenate([v, d_v])
    cls = np.concatenate([cls, np.zeros(len(d_u), dtype=np.int64)])
    length = np.exp(np.log(len_median) + len_sigma * rng.standard_normal(len(u)))
    length = np.clip(length, 10.0, 2000.0)
    # largest connected component
    g = coo_matrix((np.ones(len(u)), (u, v)), shape=(n, n))
    _, lab = connected_components(g, directed=False)
    big = np.argmax(np.bincount(lab))
    alive = lab == big
    new_id = np.full(n, -1, dtype=np.int64)
    new_id[alive] = np.arange(int(alive.sum()))
    ok = alive[u]
    u, v, cls, length = new_id[u[ok]], new_id[v[ok]], cls[ok], length[ok]
    # two directed edges per link, ordered by (src, dst)
    src = np.concatenate([u, v])
    dst = np.concatenate([v, u])
    cls2 = np.concatenate([cls, cls])
    len2 = np.concatenate([length, length])
    order = np.lexsort((dst, src))
    src, dst, cls2, len2 = src[order], dst[order], cls2[order], len2[order]
    lane_tab = np.array([ROAD_CLASSES[k][0] for k in ("local", "collector", "arterial", "highway")])
    vmax_tab = np.array([ROAD_CLASSES[k][1] for k in ("local", "collector", "arterial", "highway")])
    net = _finish_network(x[alive], y[alive], src, dst, len2, lane_tab[cls2], vmax_tab[cls2],
                          cls2 > 0, green_steps)
    # signals where non-local roads meet (>= 3 non-local approaches); local
    # side streets joining a major road stay uncontrolled
    net["node_green"] = np.where(net["_nonlocal_in"] >= 3, green_steps, 0).astype(np.uint32)
    # two-phase signals: approaches arriving along x share one phase, along y
    # the other; a node whose approaches all run one way has a single phase
    nx, ny = net["node_x"].astype(np.float64), net["node_y"].astype(np.float64)
    along_y = (np.abs(ny[dst] - ny[src]) > np.abs(nx[dst] - nx[src])).astype(np.int64)
    has_x = np.bincount(dst, weights=(1 - along_y), minlength=net["n_nodes"]) > 0
    rank = np.where(has_x[dst], along_y, 0)
    net["edge_approach_rank"] = rank.astype(np.uint8)
    net["edge_class"] = cls2.astype(np.uint8)
    return net


def regional_network(seed: int = 2, scale: str = "paper") -> dict:
    """Planar network at the paper's single-GPU regional scale
    (about 224k nodes / 549k directed edges) or the large variant
    (about 1M nodes / 2.5M edges)."""
    if scale == "paper":
        return planar_network(515, 515, seed)
    if scale == "large":
        return planar_network(1095, 1095, seed)
    raise ValueError(scale)


# --------------------------------------------------------------------------------------
# demand
# --------------------------------------------------------------------------------------

def _depart_steps(t_seconds: np.ndarray, dt: float) -> np.ndarray:
    return np.ceil(t_seconds / dt).astype(np.uint32)


def uniform_demand(net: dict, n_trips: int, seed: int, t_max_s: float = 1800.0, dt: float = 0.5) -> dict:
    """Origins and destinations uniform over nodes (o != d), departures
    uniform over [0, t_max_s)."""
    rng = np.random.default_rng(seed)
    n = net["n_nodes"]
    o = rng.integers(0, n, n_trips)
    d = rng.integers(0, n - 1, n_trips)
    d = np.where(d >= o, d + 1, d)
    t = rng.uniform(0.0, t_max_s, n_trips)
    return {"orig": o.astype(np.uint32), "dest": d.astype(np.uint32), "depart_step": _depart_steps(t, dt)}


def gravity_demand(net: dict, n_trips: int, seed: int, zones_x: int = 50, zones_y: int = 30,
                   access_per_zone: int = 4, beta_m: float = 8000.0, pop_sigma: float = 1.0,
                   peaks_h=(8.0, 17.5), peak_sigma_h: float = 0.75, day_s: float = 86400.0,
                   dt: float = 0.5) -> dict:
    """Gravity OD between zones: P(o,d) ~ pop_o * pop_d * exp(-dist/beta),
    o != d; each zone exposes `access_per_zone` nodes drawn uniformly from
    the nodes inside it (trips start and end there); departures are a 50/50
    mixture of two normal peaks truncated to [0, day_s)."""
    rng = np.random.default_rng(seed)
    x, y = net["node_x"].astype(np.float64), net["node_y"].astype(np.float64)
    x0, x1, y0, y1 = x.min(), x.max() + 1e-3, y.min(), y.max() + 1e-3
    zx = np.minimum(((x - x0) / (x1 - x0) * zones_x).astype(np.int64), zones_x - 1)
    zy = np.minimum(((y - y0) / (y1 - y0) * zones_y).astype(np.int64), zones_y - 1)
    zone = zy * zones_x + zx
    nz = zones_x * zones_y
    order = np.argsort(zone, kind="stable")
    counts = np.bincount(zone, minlength=nz)
    starts = np.concatenate([[0], np.cumsum(counts)])
    access = np.full((nz, access_per_zone), -1, dtype=np.int64)
    for z in range(nz):
        members = order[starts[z]:starts[z + 1]]
        if len(members) == 0:
            continue
        k = min(access_per_zone, len(members))
        pick = rng.choice(members, size=k, replace=False)
        access[z, :k] = pick
        access[z, k:] = pick[rng.integers(0, k, access_per_zone - k)]
    pop = np.exp(pop_sigma * rng.standard_normal(nz))
    pop[counts == 0] = 0.0
    cx = (np.arange(nz) % zones_x + 0.5) * (x1 - x0) / zones_x
    cy = (np.arange(nz) // zones_x + 0.5) * (y1 - y0) / zones_y
    dist = np.hypot(cx[:, None] - cx[None, :], cy[:, None] - cy[None, :])
    w = pop[:, None] * pop[None, :] * np.exp(-dist / beta_m)
    np.fill_diagonal(w, 0.0)
    w = w.ravel()
    w /= w.sum()
    pair = rng.choice(nz * nz, size=n_trips, p=w)
    zo, zd = pair // nz, pair % nz
    o = access[zo, rng.integers(0, access_per_zone, n_trips)]
    d = access[zd, rng.integers(0, access_per_zone, n_trips)]
    which = rng.random(n_trips) < 0.5
    t = np.where(which, peaks_h[0], peaks_h[1]) * 3600.0 + rng.standard_normal(n_trips) * peak_sigma_h * 3600.0
    bad = (t < 0) | (t >= day_s)
    while bad.any():
        m = int(bad.sum())
        w2 = rng.random(m) < 0.5
        t[bad] = np.where(w2, peaks_h[0], peaks_h[1]) * 3600.0 + rng.standard_normal(m) * peak_sigma_h * 3600.0
        bad = (t < 0) | (t >= day_s)
    return {"orig": o.astype(np.uint32), "dest": d.astype(np.uint32), "depart_step": _depart_steps(t, dt)}


def route(net: dict, demand: dict, n_threads: int | None = None) -> dict:
    """Free-flow shortest path (integer milliseconds, ties to the lower edge
    id) for every trip.  Returns demand plus route_off (u64, n+1) and
    route_edges (u32)."""
    lib = _lib()
    cost = np.maximum(1, np.rint(net["edge_len"].astype(np.float64) /
                                 net["edge_vmax"].astype(np.float64) * 1000.0)).astype(np.int64)
    o = np.ascontiguousarray(demand["orig"], dtype=np.uint32)
    d = np.ascontiguousarray(demand["dest"], dtype=np.uint32)
    st = ctypes.c_int(0)
    nt = n_threads or max(1, os.cpu_count() or 1)
    h = lib.wl_route(net["n_nodes"], net["n_edges"], _ptr(net["edge_src"]), _ptr(net["edge_dst"]),
                     _ptr(cost), len(o), _ptr(o), _ptr(d), nt, ctypes.byref(st))
    if not h:
        raise ValueError(f"routing failed (status {st.value})")
    try:
        total = lib.wl_route_total(h)
        off = np.empty(len(o) + 1, dtype=np.uint64)
        edges = np.empty(max(1, total), dtype=np.uint32)
        lib.wl_route_copy(h, _ptr(off), _ptr(edges))
    finally:
        lib.wl_route_free(h)
    if st.value != 0:
        raise ValueError("some trips have no route (origin == destination or unreachable)")
    out = dict(demand)
    out["route_off"] = off
    out["route_edges"] = edges[:total]
    return out


# --------------------------------------------------------------------------------------
# named workloads
# --------------------------------------------------------------------------------------

def grid_day(seed: int = 1, n_trips: int = 2000) -> tuple[dict, dict]:
    """8x8 grid, 224 directed 400 m links, 2 lanes, 13.9 m/s, 30 s green per
    approach; trips between uniform random nodes departing over 30 min."""
    net = grid_network()
    dem = route(net, uniform_demand(net, n_trips, seed))
    return net, dem


def regional_day(seed: int = 2, n_trips: int = 2_820_000, scale: str = "paper") -> tuple[dict, dict]:
    """Regional planar network and a 24 h gravity demand with AM/PM peaks.
    The zone grid grows with the network's area (50 x 30 zones at the
    paper's scale, 107 x 64 on the large network), so each zone -- and each
    access node -- keeps about the same size and load."""
    net = regional_network(seed, scale)
    zx, zy = (50, 30) if scale == "paper" else (107, 64)
    dem = route(net, gravity_demand(net, n_trips, seed + 1000, zones_x=zx, zones_y=zy))
    return net, dem


def subset_trips(dem: dict, keep: np.ndarray) -> dict:
    """Trips selected by a boolean mask, routes repacked."""
    idx = np.nonzero(keep)[0]
    off = dem["route_off"]
    lens = (off[idx + 1] - off[idx]).astype(np.uint64)
    new_off = np.zeros(len(idx) + 1, dtype=np.uint64)
    new_off[1:] = np.cumsum(lens)
    parts = [dem["route_edges"][int(off[i]):int(off[i + 1])] for i in idx]
    edges = np.concatenate(parts) if parts else np.zeros(0, dtype=np.uint32)
    out = {k: (v[idx] if isinstance(v, np.ndarray) and len(v) == len(dem["depart_step"]) else v)
           for k, v in dem.items() if k not in ("route_off", "route_edges")}
    out["route_off"] = new_off
    out["route_edges"] = edges.astype(np.uint32)
    return out


def batch_scenarios(n_scen: int = 64, base_seed: int = 100, min_nodes: int = 1000, max_nodes: int = 50_000,
                    trips_per_node: float = 8.0, min_trips: int = 10_000, max_trips: int = 400_000,
                    horizon_h: float = 2.0, dt: float = 0.5) -> list:
    """Independent scenarios of uneven size for batched runs: grid or planar
    networks of log-uniform node count, demand scaled by U(0.5, 1.5), each
    with its own seed.  Departures peak twice inside `horizon_h` hours.
    Returns a list of (network, routed demand, seed)."""
    out = []
    for s in range(n_scen):
        seed = base_seed + s
        rng = np.random.default_rng(seed)
        nodes = int(np.exp(rng.uniform(np.log(min_nodes), np.log(max_nodes))))
        scale = rng.uniform(0.5, 1.5)
        if rng.random() < 0.5:
            side = max(3, int(round(np.sqrt(nodes))))
            net = grid_network(side, side, spacing=250.0)
        else:
            side = max(6, int(round(np.sqrt(nodes / 0.84))))
            net = planar_network(side, side, seed)
        n_trips = int(np.clip(net["n_nodes"] * trips_per_node * scale, min_trips, max_trips))
        zx = max(2, side // 10)
        zy = max(2, side // 17)
        extent = float(max(net["node_x"].max() - net["node_x"].min(), net["node_y"].max() - net["node_y"].min()))
        dem = gravity_demand(net, n_trips, seed + 5000, zones_x=zx, zones_y=zy, access_per_zone=4,
                             beta_m=max(500.0, extent / 6.0), peaks_h=(0.3 * horizon_h, 0.6 * horizon_h),
                             peak_sigma_h=0.12 * horizon_h, day_s=horizon_h * 3600.0, dt=dt)
        out.append((net, route(net, dem), seed))
    return out


def assignment_case(seed: int = 5, scale: str = "small") -> tuple[dict, dict]:
    """Regional network and day demand for the assignment loop: "paper" is
    the 224k-node network with the 2.82M-trip day (regional_day, seed 2);
    "small" and "tiny" are the regional generator at reduced scale (~27k
    nodes / ~340k trips -- the same trips per node -- and ~3k / 30k)."""
    if scale == "paper":
        return regional_day(seed=2, n_trips=2_820_000)
    sizes = {"small": (180, 340_000, 12, 8), "tiny": (60, 30_000, 5, 3)}
    side, n_trips, zx, zy = sizes[scale]
    net = planar_network(side, side, seed)
    extent = float(net["node_x"].max() - net["node_x"].min())
    dem = gravity_demand(net, n_trips, seed + 1000, zones_x=zx, zones_y=zy, access_per_zone=4,
                         beta_m=extent / 9.0)
    return net, route(net, dem)
