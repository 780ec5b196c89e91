"""Tiny hand-built networks and trip tables for the oracle pins."""
from __future__ import annotations

import numpy as np


def make_net(n_nodes, edges, green=None, approach_rank=None):
    """edges: list of (src, dst, length_m, lanes, vmax)."""
    g = np.zeros(n_nodes, np.uint32)
    for node, steps in (green or {}).items():
        g[node] = steps
    net = {
        "n_nodes": n_nodes,
        "n_edges": len(edges),
        "edge_src": np.array([e[0] for e in edges], np.uint32),
        "edge_dst": np.array([e[1] for e in edges], np.uint32),
        "edge_len": np.array([e[2] for e in edges], np.float32),
        "edge_lanes": np.array([e[3] for e in edges], np.uint8),
        "edge_vmax": np.array([e[4] for e in edges], np.float32),
        "node_green": g,
    }
    if approach_rank is not None:
        net["edge_approach_rank"] = np.array(approach_rank, np.uint8)
    return net


def make_demand(trips):
    """trips: list of (depart_step, [edge ids])."""
    dep = np.array([t[0] for t in trips], np.uint32)
    off = np.zeros(len(trips) + 1, np.uint64)
    off[1:] = np.cumsum([len(t[1]) for t in trips])
    edges = np.array([e for t in trips for e in t[1]], np.uint32)
    return {"depart_step": dep, "route_off": off, "route_edges": edges}


def routes_of(dem):
    off = dem["route_off"].astype(np.int64)
    return [list(dem["route_edges"][off[j]:off[j + 1]]) for j in range(len(off) - 1)]
