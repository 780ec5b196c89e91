"""GB300-native per-step microsimulation of arXiv 2406.08496 (LPSim).

Thin Python binding of the C ABI in include/lpsim.h (liblpsim.so, hand-written
sm_103a CUDA).  This module only marshals arguments: every step of the
simulation runs in the library's kernels.  PyTorch, when present, supplies
device memory (caching allocator) and the stream.  There is no CPU fallback:
importing the binding without the compiled library raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from ._build import LIB as _LIB_PATH
from ._build import build as _build_lib

__all__ = ["Simulation", "LpsimError", "DEFAULT_PARAMS", "build", "load_library", "EXPORTED"]

# Model readings (Table 3 lists the symbols without values): dt from the
# workloads; IDM a, b, s0, T; lane-change horizon x0; critical-gap constants.
DEFAULT_PARAMS = dict(dt=0.5, a=1.0, b=1.5, s0=2.0, T=1.5, x0=100.0, g_a=2.0, g_b=2.0,
                      alpha_i=1.0, alpha_a=1.0, alpha_b=1.0, eps_amp=0.0, seed=12345,
                      bin_steps=1800, n_bins=0, sort_period=256, block_size=256, blocks_per_sm=4,
                      chunk_steps=1536, gridlock_steps=0, flags=0, light_trips=0, dlc_prob=0.0, dlc_gain=5.0)
FLAG_NO_SORT = 1

EXPORTED = ["lpsim_last_error", "lpsim_version", "lpsim_set_allocator", "lpsim_load_network",
            "lpsim_load_demand", "lpsim_load_demand_typed", "lpsim_set_vehicle_types", "lpsim_step", "lpsim_run", "lpsim_reset", "lpsim_link_stats",
            "lpsim_get_trips", "lpsim_get_state", "lpsim_lane_map_size", "lpsim_get_lane_map",
            "lpsim_get_counters", "lpsim_set_kernel_timing", "lpsim_get_kernel_times", "lpsim_get_state_noalloc",
            "lpsim_load_network_batch", "lpsim_load_demand_batch", "lpsim_batch_offsets", "lpsim_snapshot",
            "lpsim_restore", "lpsim_autotune", "lpsim_set_config", "lpsim_destroy",
            "lpsim_mlp_create", "lpsim_mlp_set_params", "lpsim_mlp_get_params", "lpsim_mlp_forward",
            "lpsim_mlp_grad", "lpsim_mlp_train", "lpsim_mlp_apply_grads", "lpsim_mlp_pool_add",
            "lpsim_mlp_pool_clear", "lpsim_mlp_pool_size", "lpsim_mlp_train_pool", "lpsim_mlp_gemm_test", "lpsim_mlp_time", "lpsim_mlp_gelu_eval",
            "lpsim_mlp_destroy",
            "lpsim_assign_create", "lpsim_assign_shortest_paths", "lpsim_assign_shortest_paths_gpu", "lpsim_assign_gap", "lpsim_assign_reroute",
            "lpsim_assign_route_excess", "lpsim_assign_reroute_worst", "lpsim_assign_route_length",
            "lpsim_assign_get_routes", "lpsim_assign_load", "lpsim_assign_load_gpu", "lpsim_assign_features", "lpsim_assign_features_rows", "lpsim_assign_link_times", "lpsim_assign_times_from_ratio", "lpsim_assign_destroy"]

STATUS = {0: "LPSIM_OK", -1: "LPSIM_E_INVALID_ARG", -2: "LPSIM_E_OOM", -3: "LPSIM_E_CUDA", -4: "LPSIM_E_STATE",
          -5: "LPSIM_E_TIMEOUT", -6: "LPSIM_E_GRIDLOCK", -7: "LPSIM_E_INVARIANT"}


class Params(ctypes.Structure):
    _fields_ = [(n, ctypes.c_float) for n in ("dt", "a", "b", "s0", "T", "x0", "g_a", "g_b", "alpha_i",
                                              "alpha_a", "alpha_b", "eps_amp")] + \
               [("seed", ctypes.c_uint64)] + \
               [(n, ctypes.c_uint32) for n in ("bin_steps", "n_bins", "sort_period", "block_size",
                                               "blocks_per_sm", "chunk_steps", "gridlock_steps", "flags",
                                               "light_trips")] + \
               [(n, ctypes.c_float) for n in ("dlc_prob", "dlc_gain")]


class Network(ctypes.Structure):
    _fields_ = [("n_nodes", ctypes.c_uint32), ("n_edges", ctypes.c_uint32),
                ("edge_src", ctypes.c_void_p), ("edge_dst", ctypes.c_void_p), ("edge_len_m", ctypes.c_void_p),
                ("edge_lanes", ctypes.c_void_p), ("edge_vmax", ctypes.c_void_p),
                ("node_green_steps", ctypes.c_void_p), ("edge_approach_rank", ctypes.c_void_p)]


class RunResult(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint64) for n in ("steps", "veh_steps", "arrived", "active", "waiting", "k")] + \
               [("wall_ms", ctypes.c_double)]


class LinkStat(ctypes.Structure):
    _fields_ = [("entries", ctypes.c_uint64), ("exits", ctypes.c_uint64), ("tt_steps", ctypes.c_uint64)]


class Counters(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint64) for n in ("k", "veh_steps", "arrived", "active", "waiting", "lane_changes",
                                               "slots", "launches", "light_chunks")]


class TuneResult(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint32) for n in ("block_size", "blocks_per_sm", "sort_period", "chunk_steps")] + \
               [("best_ms", ctypes.c_double), ("default_ms", ctypes.c_double), ("n_tried", ctypes.c_uint32)]


class VehicleType(ctypes.Structure):
    _fields_ = [(n, ctypes.c_float) for n in ("a", "b", "s0", "T", "vmax")]


class KernelTimes(ctypes.Structure):
    _fields_ = [("ms", ctypes.c_double * 4), ("launches", ctypes.c_uint64 * 4), ("p1_veh_steps", ctypes.c_uint64)]


class LpsimError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


_lib = None
_alloc_cbs = None  # keeps the ctypes callbacks alive
ALLOC_T = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_T = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)


def build(force: bool = False) -> str:
    """Compile liblpsim.so for sm_103a (nvcc; works without a GPU)."""
    return _build_lib(force=force)


def load_library(path: str | None = None):
    """Load liblpsim.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or _LIB_PATH
    if not os.path.exists(p):
        raise ImportError(f"liblpsim.so not found at {p}: run paper_2406_08496_gb300.build() first "
                          "(the simulation has no CPU fallback)")
    lib = ctypes.CDLL(p)
    P = ctypes.c_void_p
    lib.lpsim_last_error.restype = ctypes.c_char_p
    lib.lpsim_version.restype = ctypes.c_char_p
    lib.lpsim_set_allocator.argtypes = [ALLOC_T, FREE_T, P]
    lib.lpsim_load_network.argtypes = [ctypes.POINTER(P), ctypes.POINTER(Network), ctypes.POINTER(Params), P]
    lib.lpsim_load_demand.argtypes = [P, ctypes.c_uint64, P, P, P, P]
    lib.lpsim_load_demand_typed.argtypes = [P, ctypes.c_uint64, P, P, P, P, P]
    lib.lpsim_set_vehicle_types.argtypes = [P, ctypes.c_uint32, P]
    lib.lpsim_step.argtypes = [P, ctypes.c_uint32]
    lib.lpsim_run.argtypes = [P, ctypes.c_uint32, ctypes.POINTER(RunResult)]
    lib.lpsim_reset.argtypes = [P]
    lib.lpsim_link_stats.argtypes = [P, P, ctypes.c_uint64, P, P, P, P, ctypes.c_uint32]
    lib.lpsim_get_trips.argtypes = [P, ctypes.c_uint64, P, P]
    lib.lpsim_get_state.argtypes = [P, ctypes.c_uint64, P, P, P, P, P, P]
    lib.lpsim_lane_map_size.argtypes = [P]
    lib.lpsim_lane_map_size.restype = ctypes.c_uint64
    lib.lpsim_get_lane_map.argtypes = [P, P, ctypes.c_uint64]
    lib.lpsim_get_counters.argtypes = [P, ctypes.POINTER(Counters)]
    lib.lpsim_set_kernel_timing.argtypes = [P, ctypes.c_int]
    lib.lpsim_get_kernel_times.argtypes = [P, ctypes.POINTER(KernelTimes)]
    lib.lpsim_get_state_noalloc.argtypes = [P, ctypes.c_uint64, P, P, P, P, P, P]
    lib.lpsim_load_network_batch.argtypes = [ctypes.POINTER(P), ctypes.c_uint32, P, ctypes.POINTER(Params), P]
    lib.lpsim_load_demand_batch.argtypes = [P, ctypes.c_uint32, P, P, P, P, P, P]
    lib.lpsim_batch_offsets.argtypes = [P, ctypes.c_uint32, P, P, P, P]
    lib.lpsim_snapshot.argtypes = [P]
    lib.lpsim_restore.argtypes = [P]
    lib.lpsim_autotune.argtypes = [P, ctypes.c_uint32, ctypes.POINTER(TuneResult)]
    lib.lpsim_set_config.argtypes = [P, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32]
    lib.lpsim_destroy.argtypes = [P]
    lib.lpsim_destroy.restype = None
    lib.lpsim_mlp_create.argtypes = [ctypes.POINTER(P), ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint64, P]
    lib.lpsim_mlp_set_params.argtypes = [P, P]
    lib.lpsim_mlp_get_params.argtypes = [P, P]
    lib.lpsim_mlp_forward.argtypes = [P, ctypes.c_uint64, P, P]
    lib.lpsim_mlp_grad.argtypes = [P, ctypes.c_uint64, P, P, P, P]
    lib.lpsim_mlp_train.argtypes = [P, ctypes.c_uint64, P, P, ctypes.c_uint32, ctypes.c_float, ctypes.c_uint64, P]
    lib.lpsim_mlp_apply_grads.argtypes = [P, P, ctypes.c_float]
    lib.lpsim_mlp_pool_add.argtypes = [P, ctypes.c_uint64, P, P]
    lib.lpsim_mlp_pool_clear.argtypes = [P]
    lib.lpsim_mlp_pool_size.argtypes = [P]
    lib.lpsim_mlp_pool_size.restype = ctypes.c_uint64
    lib.lpsim_mlp_train_pool.argtypes = [P, ctypes.c_uint32, ctypes.c_float, ctypes.c_uint64, P]
    lib.lpsim_mlp_gemm_test.argtypes = [ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32, P, P, P]
    lib.lpsim_mlp_time.argtypes = [P, ctypes.c_uint32, P, P]
    lib.lpsim_mlp_gelu_eval.argtypes = [ctypes.c_uint64, P, P, P]
    lib.lpsim_mlp_destroy.argtypes = [P]
    lib.lpsim_mlp_destroy.restype = None
    _lib = lib
    return lib


def _p(a):
    return None if a is None else ctypes.c_void_p(a.ctypes.data)


def _check(lib, rc: int) -> None:
    if rc != 0:
        raise LpsimError(rc, lib.lpsim_last_error().decode(errors="replace"))


def use_torch_allocator() -> bool:
    """Route the library's device allocations through PyTorch's caching
    allocator (contexts created afterwards).  Returns False without CUDA."""
    global _alloc_cbs
    lib = load_library()
    try:
        import torch
    except ImportError:
        return False
    if not torch.cuda.is_available():
        return False

    def _alloc(size, user):
        try:
            return int(torch.cuda.caching_allocator_alloc(int(size), stream=torch.cuda.current_stream()))
        except Exception:
            return None

    def _free(ptr, user):
        torch.cuda.caching_allocator_delete(int(ptr))

    cbs = (ALLOC_T(_alloc), FREE_T(_free))
    _check(lib, lib.lpsim_set_allocator(cbs[0], cbs[1], None))
    _alloc_cbs = cbs
    return True


def _current_stream():
    """torch's current stream, or None for the library's own stream (the
    legacy default stream cannot be captured into a CUDA graph)."""
    try:
        import torch
        if torch.cuda.is_available():
            h = torch.cuda.current_stream().cuda_stream
            return ctypes.c_void_p(h) if h else None
    except ImportError:
        pass
    return None


def _net_arrays(net: dict) -> dict:
    out = {
        "edge_src": np.ascontiguousarray(net["edge_src"], dtype=np.uint32),
        "edge_dst": np.ascontiguousarray(net["edge_dst"], dtype=np.uint32),
        "edge_len": np.ascontiguousarray(net["edge_len"], dtype=np.float32),
        "edge_lanes": np.ascontiguousarray(net["edge_lanes"], dtype=np.uint8),
        "edge_vmax": np.ascontiguousarray(net["edge_vmax"], dtype=np.float32),
        "node_green": np.ascontiguousarray(net["node_green"], dtype=np.uint32),
    }
    ar = net.get("edge_approach_rank")
    out["edge_approach_rank"] = None if ar is None else np.ascontiguousarray(ar, dtype=np.uint8)
    return out


def _net_desc(net: dict, n: dict) -> Network:
    return Network(int(net["n_nodes"]), int(net["n_edges"]), _p(n["edge_src"]), _p(n["edge_dst"]), _p(n["edge_len"]),
                   _p(n["edge_lanes"]), _p(n["edge_vmax"]), _p(n["node_green"]), _p(n["edge_approach_rank"]))


class Simulation:
    """One network + demand on the GPU library.

    net: dict with n_nodes, n_edges, edge_src, edge_dst, edge_len, edge_lanes,
    edge_vmax, node_green and optionally edge_approach_rank (numpy arrays).
    """

    def __init__(self, net: dict, params: dict | None = None, stream=None, vehicle_types: list | None = None):
        """vehicle_types (optional): per type a dict of a, b, s0, T and vmax;
        trips then name their type in the demand's "vtype" array."""
        self.lib = load_library()
        self.params = dict(DEFAULT_PARAMS)
        if params:
            self.params.update(params)
        self._p = Params(**self.params)
        self._net = {
            "edge_src": np.ascontiguousarray(net["edge_src"], dtype=np.uint32),
            "edge_dst": np.ascontiguousarray(net["edge_dst"], dtype=np.uint32),
            "edge_len": np.ascontiguousarray(net["edge_len"], dtype=np.float32),
            "edge_lanes": np.ascontiguousarray(net["edge_lanes"], dtype=np.uint8),
            "edge_vmax": np.ascontiguousarray(net["edge_vmax"], dtype=np.float32),
            "node_green": np.ascontiguousarray(net["node_green"], dtype=np.uint32),
        }
        ar = net.get("edge_approach_rank")
        self._net["edge_approach_rank"] = None if ar is None else np.ascontiguousarray(ar, dtype=np.uint8)
        n = self._net
        self.n_edges = int(net["n_edges"])
        self.n_bins = int(self.params["n_bins"])
        desc = Network(int(net["n_nodes"]), self.n_edges, _p(n["edge_src"]), _p(n["edge_dst"]), _p(n["edge_len"]),
                       _p(n["edge_lanes"]), _p(n["edge_vmax"]), _p(n["node_green"]), _p(n["edge_approach_rank"]))
        h = ctypes.c_void_p()
        st = stream if stream is not None else _current_stream()
        _check(self.lib, self.lib.lpsim_load_network(ctypes.byref(h), ctypes.byref(desc), ctypes.byref(self._p), st))
        self.h = h
        self.n = 0
        if vehicle_types:
            arr = (VehicleType * len(vehicle_types))(*[VehicleType(**t) for t in vehicle_types])
            _check(self.lib, self.lib.lpsim_set_vehicle_types(self.h, len(vehicle_types),
                                                              ctypes.cast(arr, ctypes.c_void_p)))

    def load_demand(self, dem: dict) -> np.ndarray:
        dep = np.ascontiguousarray(dem["depart_step"], dtype=np.uint32)
        off = np.ascontiguousarray(dem["route_off"], dtype=np.uint64)
        edges = np.ascontiguousarray(dem["route_edges"], dtype=np.uint32)
        vt = dem.get("vtype")
        vt = None if vt is None else np.ascontiguousarray(vt, dtype=np.uint8)
        vid = np.empty(len(dep), dtype=np.uint32)
        _check(self.lib, self.lib.lpsim_load_demand_typed(self.h, len(dep), _p(dep), _p(off), _p(edges), _p(vt),
                                                          _p(vid)))
        self.n = len(dep)
        return vid

    def step(self, n_steps: int = 1) -> None:
        _check(self.lib, self.lib.lpsim_step(self.h, n_steps))

    def run(self, max_steps: int) -> dict:
        r = RunResult()
        _check(self.lib, self.lib.lpsim_run(self.h, max_steps, ctypes.byref(r)))
        return {f: getattr(r, f) for f, _ in RunResult._fields_}

    def reset(self) -> None:
        _check(self.lib, self.lib.lpsim_reset(self.h))

    def counters(self) -> dict:
        c = Counters()
        _check(self.lib, self.lib.lpsim_get_counters(self.h, ctypes.byref(c)))
        return {f: getattr(c, f) for f, _ in Counters._fields_}

    def state(self) -> dict:
        n = self.n
        st = {"x": np.empty(n, np.float32), "v": np.empty(n, np.float32), "edge": np.empty(n, np.uint32),
              "lane": np.empty(n, np.uint8), "ridx": np.empty(n, np.uint32), "status": np.empty(n, np.uint8)}
        _check(self.lib, self.lib.lpsim_get_state(self.h, n, *(_p(st[k]) for k in
                                                              ("x", "v", "edge", "lane", "ridx", "status"))))
        return st

    def trips(self) -> dict:
        d = np.empty(self.n, np.uint32)
        a = np.empty(self.n, np.uint32)
        _check(self.lib, self.lib.lpsim_get_trips(self.h, self.n, _p(d), _p(a)))
        return {"depart": d, "arrive": a}

    def lane_map(self) -> np.ndarray:
        m = np.empty(int(self.lib.lpsim_lane_map_size(self.h)), np.uint8)
        _check(self.lib, self.lib.lpsim_get_lane_map(self.h, _p(m), m.size))
        return m

    def link_stats(self) -> dict:
        ne, nb = self.n_edges, self.n_bins
        pe = np.empty((ne, 3), np.uint64)
        bins = {k: np.empty((ne, nb), np.uint32) for k in ("inflow", "tt_sum", "tt_cnt", "occ")}
        _check(self.lib, self.lib.lpsim_link_stats(self.h, _p(pe), ne, *(_p(bins[k]) for k in
                                                                         ("inflow", "tt_sum", "tt_cnt", "occ")), nb))
        out = {"entries": pe[:, 0].copy(), "exits": pe[:, 1].copy(), "tt_steps": pe[:, 2].copy()}
        out.update(bins)
        return out

    def set_kernel_timing(self, on: bool) -> None:
        _check(self.lib, self.lib.lpsim_set_kernel_timing(self.h, 1 if on else 0))

    def kernel_times(self) -> dict:
        """Summed device spans per kernel since timing was switched on, and
        the vehicle-steps the step_p1 launches handled."""
        t = KernelTimes()
        _check(self.lib, self.lib.lpsim_get_kernel_times(self.h, ctypes.byref(t)))
        names = ("step_p1", "step_p2", "compact_sort", "step_small")
        out = {k: {"ms": float(t.ms[i]), "launches": int(t.launches[i])} for i, k in enumerate(names)}
        out["step_p1"]["veh_steps"] = int(t.p1_veh_steps)
        return out

    def snapshot(self) -> None:
        _check(self.lib, self.lib.lpsim_snapshot(self.h))

    def restore(self) -> None:
        _check(self.lib, self.lib.lpsim_restore(self.h))

    def autotune(self, window_steps: int) -> dict:
        r = TuneResult()
        _check(self.lib, self.lib.lpsim_autotune(self.h, window_steps, ctypes.byref(r)))
        return {f: getattr(r, f) for f, _ in TuneResult._fields_}

    def set_config(self, block_size: int, blocks_per_sm: int, sort_period: int, chunk_steps: int) -> None:
        _check(self.lib, self.lib.lpsim_set_config(self.h, block_size, blocks_per_sm, sort_period, chunk_steps))

    def close(self) -> None:
        if getattr(self, "h", None):
            self.lib.lpsim_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class BatchSimulation(Simulation):
    """Many independent scenarios in one context (one launch per step kernel
    advances them all); each scenario's results equal simulating it alone."""

    def __init__(self, nets: list, params: dict | None = None, stream=None):
        self.lib = load_library()
        self.params = dict(DEFAULT_PARAMS)
        if params:
            self.params.update(params)
        self._p = Params(**self.params)
        self._nets = [_net_arrays(n) for n in nets]
        descs = (Network * len(nets))(*[_net_desc(n, a) for n, a in zip(nets, self._nets)])
        h = ctypes.c_void_p()
        st = stream if stream is not None else _current_stream()
        _check(self.lib, self.lib.lpsim_load_network_batch(ctypes.byref(h), len(nets), ctypes.cast(descs, ctypes.c_void_p),
                                                           ctypes.byref(self._p), st))
        self.h = h
        self.n_scen = len(nets)
        self.n_edges = int(sum(int(n["n_edges"]) for n in nets))
        self.n_bins = int(self.params["n_bins"])
        self.n = 0

    def load_demand(self, dems: list, seeds=None) -> list:
        ns = self.n_scen
        keep = []
        dep_p = (ctypes.c_void_p * ns)()
        off_p = (ctypes.c_void_p * ns)()
        edg_p = (ctypes.c_void_p * ns)()
        counts = np.array([len(d["depart_step"]) for d in dems], np.uint64)
        for i, d in enumerate(dems):
            a = np.ascontiguousarray(d["depart_step"], dtype=np.uint32)
            b = np.ascontiguousarray(d["route_off"], dtype=np.uint64)
            c = np.ascontiguousarray(d["route_edges"], dtype=np.uint32)
            keep += [a, b, c]
            dep_p[i], off_p[i], edg_p[i] = a.ctypes.data, b.ctypes.data, c.ctypes.data
        sd = None if seeds is None else np.ascontiguousarray(seeds, dtype=np.uint64)
        total = int(counts.sum())
        vid = np.empty(total, np.uint32)
        _check(self.lib, self.lib.lpsim_load_demand_batch(self.h, ns, _p(counts), ctypes.cast(dep_p, ctypes.c_void_p),
                                                          ctypes.cast(off_p, ctypes.c_void_p),
                                                          ctypes.cast(edg_p, ctypes.c_void_p), _p(sd), _p(vid)))
        self.n = total
        splits = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
        return [vid[splits[i]:splits[i + 1]] for i in range(ns)]

    def offsets(self) -> dict:
        ns = self.n_scen
        arr = {k: np.zeros(ns + 1, np.uint64) for k in ("node", "edge", "cell", "trip")}
        _check(self.lib, self.lib.lpsim_batch_offsets(self.h, ns, *(_p(arr[k]) for k in ("node", "edge", "cell", "trip"))))
        return {k: v.astype(np.int64) for k, v in arr.items()}


PARAM_SHAPES = [(256, 64), (256,), (256, 256), (256,), (256, 256), (256,), (1, 256), (1,)]
PARAM_NAMES = ["W1", "b1", "W2", "b2", "W3", "b3", "W4", "b4"]


def gemm_bf16(A: np.ndarray, B: np.ndarray) -> np.ndarray:
    """D = A . B^T on the tensor-core GEMM kernel; A, B are uint16 BF16 bit
    patterns (M x K and N x K)."""
    lib = load_library()
    A = np.ascontiguousarray(A, dtype=np.uint16)
    B = np.ascontiguousarray(B, dtype=np.uint16)
    M, K = A.shape
    N = B.shape[0]
    D = np.empty((M, N), np.float32)
    _check(lib, lib.lpsim_mlp_gemm_test(M, N, K, _p(A), _p(B), _p(D)))
    return D


def gelu_eval(z: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """GELU(z) and GELU'(z) as the surrogate's epilogues compute them."""
    lib = load_library()
    z = np.ascontiguousarray(z, dtype=np.float32)
    g = np.empty_like(z)
    dg = np.empty_like(z)
    _check(lib, lib.lpsim_mlp_gelu_eval(z.size, _p(z), _p(g), _p(dg)))
    return g, dg


class Surrogate:
    """The link-travel-time MLP on the GPU (include/lpsim_surrogate.h)."""

    def __init__(self, n_features: int = 9, batch: int = 8192, seed: int = 0, stream=None):
        self.lib = load_library()
        self.nf = n_features
        self.batch = batch
        h = ctypes.c_void_p()
        st = stream if stream is not None else _current_stream()
        _check(self.lib, self.lib.lpsim_mlp_create(ctypes.byref(h), n_features, batch, seed, st))
        self.h = h

    def set_params(self, params: dict) -> None:
        arrs = [np.ascontiguousarray(params[k], dtype=np.float32).reshape(s) for k, s in zip(PARAM_NAMES, PARAM_SHAPES)]
        ptrs = (ctypes.c_void_p * 8)(*[a.ctypes.data for a in arrs])
        _check(self.lib, self.lib.lpsim_mlp_set_params(self.h, ctypes.cast(ptrs, ctypes.c_void_p)))

    def get_params(self) -> dict:
        arrs = [np.empty(s, np.float32) for s in PARAM_SHAPES]
        ptrs = (ctypes.c_void_p * 8)(*[a.ctypes.data for a in arrs])
        _check(self.lib, self.lib.lpsim_mlp_get_params(self.h, ctypes.cast(ptrs, ctypes.c_void_p)))
        return dict(zip(PARAM_NAMES, arrs))

    def forward(self, X: np.ndarray) -> np.ndarray:
        X = np.ascontiguousarray(X, dtype=np.float32)
        y = np.empty(len(X), np.float32)
        _check(self.lib, self.lib.lpsim_mlp_forward(self.h, len(X), _p(X), _p(y)))
        return y

    def grad(self, X: np.ndarray, t: np.ndarray):
        X = np.ascontiguousarray(X, dtype=np.float32)
        t = np.ascontiguousarray(t, dtype=np.float32)
        arrs = [np.empty(s, np.float32) for s in PARAM_SHAPES]
        ptrs = (ctypes.c_void_p * 8)(*[a.ctypes.data for a in arrs])
        loss = ctypes.c_float()
        _check(self.lib, self.lib.lpsim_mlp_grad(self.h, len(X), _p(X), _p(t), ctypes.byref(loss),
                                                 ctypes.cast(ptrs, ctypes.c_void_p)))
        return float(loss.value), dict(zip(PARAM_NAMES, arrs))

    def train(self, X: np.ndarray, t: np.ndarray, steps: int, lr: float = 1e-3, seed: int = 0) -> np.ndarray:
        X = np.ascontiguousarray(X, dtype=np.float32)
        t = np.ascontiguousarray(t, dtype=np.float32)
        losses = np.empty(steps, np.float32)
        _check(self.lib, self.lib.lpsim_mlp_train(self.h, len(X), _p(X), _p(t), steps, lr, seed, _p(losses)))
        return losses

    def pool_add(self, X: np.ndarray, t: np.ndarray) -> None:
        """Append training samples to the model's device-resident pool."""
        X = np.ascontiguousarray(X, dtype=np.float32)
        t = np.ascontiguousarray(t, dtype=np.float32)
        _check(self.lib, self.lib.lpsim_mlp_pool_add(self.h, len(X), _p(X), _p(t)))

    def pool_clear(self) -> None:
        _check(self.lib, self.lib.lpsim_mlp_pool_clear(self.h))

    def pool_size(self) -> int:
        return int(self.lib.lpsim_mlp_pool_size(self.h))

    def train_pool(self, steps: int, lr: float = 1e-3, seed: int = 0) -> np.ndarray:
        """Adam steps on minibatches of shuffled passes over the pool."""
        losses = np.empty(steps, np.float32)
        _check(self.lib, self.lib.lpsim_mlp_train_pool(self.h, steps, lr, seed, _p(losses)))
        return losses

    def apply_grads(self, grads: dict, lr: float) -> None:
        """One Adam step with the given gradients (the update train applies)."""
        arrs = [np.ascontiguousarray(grads[k], dtype=np.float32).reshape(s) for k, s in zip(PARAM_NAMES, PARAM_SHAPES)]
        ptrs = (ctypes.c_void_p * 8)(*[a.ctypes.data for a in arrs])
        _check(self.lib, self.lib.lpsim_mlp_apply_grads(self.h, ctypes.cast(ptrs, ctypes.c_void_p), lr))

    def time(self, iters: int = 20) -> dict:
        f = ctypes.c_double()
        t = ctypes.c_double()
        _check(self.lib, self.lib.lpsim_mlp_time(self.h, iters, ctypes.byref(f), ctypes.byref(t)))
        return {"forward_ms": f.value, "train_ms": t.value}

    def close(self) -> None:
        if getattr(self, "h", None):
            self.lib.lpsim_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
