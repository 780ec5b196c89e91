"""CPU oracle of the per-step vehicle update (Algorithm 1 of arXiv 2406.08496).

TEST INFRASTRUCTURE ONLY.  The tests, the smoke check and the benchmark's
CPU-baseline leg load this module; the GPU library never does.  It shares no
code with the GPU path: its own C source (lpsim_oracle.c), its own header,
its own parameter struct and its own ctypes binding.

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
_LOCK = threading.Lock()

# The paper lists the IDM / lane-change symbols (Table 3) without values; these
# are the readings used throughout (dt from the workloads; IDM a, b, s0, T;
# lane-change horizon x0; critical-gap constants).
DEFAULT_PARAMS = dict(dt=0.5, a=1.0, b=1.5, s0=2.0, T=1.5, x0=100.0, g_a=2.0, g_b=2.0,
                      alpha_i=1.0, alpha_a=1.0, alpha_b=1.0, eps_amp=0.0, seed=12345,
                      bin_steps=1800, n_bins=0, dlc_prob=0.0, dlc_gain=5.0)


class OrcParams(ctypes.Structure):
    _fields_ = [("dt", ctypes.c_float), ("a", ctypes.c_float), ("b", ctypes.c_float),
                ("s0", ctypes.c_float), ("T", ctypes.c_float), ("x0", ctypes.c_float),
                ("g_a", ctypes.c_float), ("g_b", ctypes.c_float), ("alpha_i", ctypes.c_float),
                ("alpha_a", ctypes.c_float), ("alpha_b", ctypes.c_float), ("eps_amp", ctypes.c_float),
                ("seed", ctypes.c_uint64), ("bin_steps", ctypes.c_uint32), ("n_bins", ctypes.c_uint32),
                ("dlc_prob", ctypes.c_float), ("dlc_gain", ctypes.c_float)]


class OrcVehicleType(ctypes.Structure):
    _fields_ = [(n, ctypes.c_float) for n in ("a", "b", "s0", "T", "vmax")]


def build() -> str:
    src = os.path.join(_HERE, "lpsim_oracle.c")
    hdr = os.path.join(_HERE, "lpsim_oracle.h")
    h = hashlib.sha1()
    for f in (src, hdr):
        with open(f, "rb") as fh:
            h.update(fh.read())
    out = os.path.join(_HERE, f"_liblpsim_oracle_{h.hexdigest()[:12]}.so")
    if not os.path.exists(out):
        tmp = out + f".tmp{os.getpid()}"
        # -ffp-contract=off: no fused multiply-add (gcc contracts by default on aarch64)
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
                               "-shared", "-fPIC", "-o", tmp, src, "-lm"])
        os.replace(tmp, out)
    return out


def _lib():
    global _LIB
    with _LOCK:
        if _LIB is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            lib.orc_create.argtypes = [ctypes.POINTER(P), ctypes.c_uint32, ctypes.c_uint32, P, P, P, P, P, P, P,
                                       ctypes.POINTER(OrcParams)]
            lib.orc_load_demand.argtypes = [P, ctypes.c_uint64, P, P, P, P]
            lib.orc_load_demand_typed.argtypes = [P, ctypes.c_uint64, P, P, P, P, P]
            lib.orc_set_vehicle_types.argtypes = [P, ctypes.c_uint32, P]
            lib.orc_step.argtypes = [P, ctypes.c_uint32]
            lib.orc_run.argtypes = [P, ctypes.c_uint32, P]
            lib.orc_get_state.argtypes = [P, P, P, P, P, P, P]
            lib.orc_get_trips.argtypes = [P, P, P]
            lib.orc_lane_map_size.argtypes = [P]
            lib.orc_lane_map_size.restype = ctypes.c_uint64
            lib.orc_get_lane_map.argtypes = [P, P]
            lib.orc_link_stats.argtypes = [P, P, P, P, P, P]
            lib.orc_counters.argtypes = [P, P]
            lib.orc_idm_speed.argtypes = [ctypes.POINTER(OrcParams), ctypes.c_float, ctypes.c_float,
                                          ctypes.c_float, ctypes.c_float]
            lib.orc_idm_speed.restype = ctypes.c_float
            lib.orc_destroy.argtypes = [P]
            lib.orc_destroy.restype = None
            _LIB = lib
    return _LIB


def _p(a):
    return None if a is None else ctypes.c_void_p(a.ctypes.data)


def make_params(**over) -> OrcParams:
    d = dict(DEFAULT_PARAMS)
    d.update(over)
    return OrcParams(**d)


class OracleError(RuntimeError):
    pass


def _check(rc: int, what: str) -> None:
    if rc != 0:
        raise OracleError(f"{what} failed with status {rc}")


def idm_speed(v: float, vf: float, s: float, v0: float, **params) -> float:
    p = make_params(**params)
    return float(_lib().orc_idm_speed(ctypes.byref(p), v, vf, s, v0))


class Oracle:
    """One simulation on the CPU oracle."""

    def __init__(self, net: dict, params: dict | None = None, vehicle_types: list | None = None):
        """vehicle_types (optional): per type a dict of a, b, s0, T and vmax;
        trips then name their type in the demand's "vtype" array."""
        self.lib = _lib()
        self.params = dict(DEFAULT_PARAMS)
        if params:
            self.params.update(params)
        self._p = OrcParams(**self.params)
        self.net = {k: np.ascontiguousarray(net[k]) for k in
                    ("edge_src", "edge_dst", "edge_len", "edge_lanes", "edge_vmax", "node_green")}
        self.n_edges = int(net["n_edges"])
        self.n_bins = int(self.params["n_bins"])
        arank = net.get("edge_approach_rank")
        self._arank = None if arank is None else np.ascontiguousarray(arank, dtype=np.uint8)
        h = ctypes.c_void_p()
        n = self.net
        _check(self.lib.orc_create(ctypes.byref(h), int(net["n_nodes"]), self.n_edges,
                                   _p(n["edge_src"]), _p(n["edge_dst"]), _p(n["edge_len"]), _p(n["edge_lanes"]),
                                   _p(n["edge_vmax"]), _p(n["node_green"]), _p(self._arank),
                                   ctypes.byref(self._p)), "orc_create")
        self.h = h
        self.n = 0
        if vehicle_types:
            arr = (OrcVehicleType * len(vehicle_types))(*[OrcVehicleType(**t) for t in vehicle_types])
            _check(self.lib.orc_set_vehicle_types(self.h, len(vehicle_types), ctypes.cast(arr, ctypes.c_void_p)),
                   "orc_set_vehicle_types")

    def load_demand(self, dem: dict) -> np.ndarray:
        dep = np.ascontiguousarray(dem["depart_step"], dtype=np.uint32)
        off = np.ascontiguousarray(dem["route_off"], dtype=np.uint64)
        edges = np.ascontiguousarray(dem["route_edges"], dtype=np.uint32)
        if edges.size == 0:
            edges = np.zeros(1, dtype=np.uint32)
        vt = dem.get("vtype")
        vt = None if vt is None else np.ascontiguousarray(vt, dtype=np.uint8)
        vid = np.empty(len(dep), dtype=np.uint32)
        _check(self.lib.orc_load_demand_typed(self.h, len(dep), _p(dep), _p(off), _p(edges), _p(vt), _p(vid)),
               "orc_load_demand")
        self.n = len(dep)
        return vid

    def step(self, n_steps: int = 1) -> None:
        _check(self.lib.orc_step(self.h, n_steps), "orc_step")

    def run(self, max_steps: int) -> dict:
        out = np.zeros(6, dtype=np.uint64)
        _check(self.lib.orc_run(self.h, max_steps, _p(out)), "orc_run")
        return dict(zip(("steps", "veh_steps", "arrived", "active", "waiting", "k"), map(int, out)))

    def counters(self) -> dict:
        out = np.zeros(6, dtype=np.uint64)
        _check(self.lib.orc_counters(self.h, _p(out)), "orc_counters")
        return dict(zip(("k", "veh_steps", "arrived", "active", "waiting", "lane_changes"), map(int, out)))

    def state(self) -> dict:
        n = self.n
        st = {"x": np.empty(n, np.float32), "v": np.empty(n, np.float32), "edge": np.empty(n, np.uint32),
              "lane": np.empty(n, np.uint8), "ridx": np.empty(n, np.uint32), "status": np.empty(n, np.uint8)}
        _check(self.lib.orc_get_state(self.h, *(_p(st[k]) for k in ("x", "v", "edge", "lane", "ridx", "status"))),
               "orc_get_state")
        return st

    def trips(self) -> dict:
        d = np.empty(self.n, np.uint32)
        a = np.empty(self.n, np.uint32)
        _check(self.lib.orc_get_trips(self.h, _p(d), _p(a)), "orc_get_trips")
        return {"depart": d, "arrive": a}

    def lane_map(self) -> np.ndarray:
        m = np.empty(int(self.lib.orc_lane_map_size(self.h)), np.uint8)
        _check(self.lib.orc_get_lane_map(self.h, _p(m)), "orc_get_lane_map")
        return m

    def link_stats(self) -> dict:
        ne, nb = self.n_edges, self.n_bins
        pe = np.empty((ne, 3), np.uint64)
        bins = {k: np.empty((ne, max(nb, 0)), np.uint32) for k in ("inflow", "tt_sum", "tt_cnt", "occ")}
        _check(self.lib.orc_link_stats(self.h, _p(pe), *(_p(bins[k]) for k in ("inflow", "tt_sum", "tt_cnt", "occ"))),
               "orc_link_stats")
        out = {"entries": pe[:, 0].copy(), "exits": pe[:, 1].copy(), "tt_steps": pe[:, 2].copy()}
        out.update(bins)
        return out

    def close(self) -> None:
        if getattr(self, "h", None):
            self.lib.orc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
