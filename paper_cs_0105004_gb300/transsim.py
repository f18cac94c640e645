"""Python binding of the C ABI in include/transsim.h (argument marshalling only).

Every step of the simulation runs in the CUDA library ``libtranssim.so``;
this module converts numpy arrays and torch streams to the plain pointers
and handles the ABI takes.  There is no fallback: if the library is missing
or no CUDA device is present the calls raise.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libtranssim.so")

STATS_FIELDS = ("step", "active", "buffered", "waiting", "arrived", "lane_changes", "transfers", "inserted",
                "sum_v", "vehicle_updates", "state_hash", "moving")
STATS_DTYPE = np.dtype([(f, np.uint64) for f in STATS_FIELDS])

TS_OK, TS_ERR_INVALID, TS_ERR_OOM, TS_ERR_CUDA, TS_ERR_TIMEOUT, TS_ERR_STATE, TS_ERR_DEVICE_CHECK = range(7)
STEP_AUTO, STEP_FUSED, STEP_SPLIT = range(3)
_NAMES = {1: "INVALID", 2: "OOM", 3: "CUDA", 4: "TIMEOUT", 5: "STATE", 6: "DEVICE_CHECK"}

u32p = ctypes.POINTER(ctypes.c_uint32)
u64p = ctypes.POINTER(ctypes.c_uint64)
i32p = ctypes.POINTER(ctypes.c_int32)
i8p = ctypes.POINTER(ctypes.c_int8)
u8p = ctypes.POINTER(ctypes.c_uint8)


class TsError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"TS_ERR_{_NAMES.get(code, code)}: {msg}")
        self.code = code


class Params(ctypes.Structure):
    _fields_ = [("vmax", ctypes.c_uint32), ("p_threshold", ctypes.c_uint32), ("seed", ctypes.c_uint64),
                ("lane_change", ctypes.c_uint32), ("debug_checks", ctypes.c_uint32)]


class NetworkDesc(ctypes.Structure):
    _fields_ = [("n_nodes", ctypes.c_uint32), ("n_links", ctypes.c_uint32), ("link_from", u32p),
                ("link_to", u32p), ("link_cells", u32p), ("link_lanes", u32p), ("link_ring", u8p),
                ("link_signal", u32p), ("turn_lanes", u8p), ("link_yield", u8p)]


class Stats(ctypes.Structure):
    _fields_ = [(f, ctypes.c_uint64) for f in STATS_FIELDS]


TOTALS_FIELDS = ("steps", "vehicle_updates", "lane_changes", "transfers", "inserted", "arrived", "last_state_hash",
                 "moving", "active")


class Totals(ctypes.Structure):
    _fields_ = [(f, ctypes.c_uint64) for f in TOTALS_FIELDS]


class State(ctypes.Structure):
    _fields_ = [("cell_id", i32p), ("cell_v", i8p), ("buf_id", i32p), ("buf_v", i8p), ("cursor", u32p),
                ("dep_head", u32p), ("step", ctypes.c_uint64), ("arrived", ctypes.c_uint64),
                ("inserted", ctypes.c_uint64)]


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)


class Allocator(ctypes.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("user", ctypes.c_void_p)]


# The C ABI: name -> (restype, argtypes)
_API = {
    "ts_create_network": (ctypes.c_int, [ctypes.POINTER(NetworkDesc), ctypes.POINTER(Params),
                                         ctypes.POINTER(Allocator), ctypes.POINTER(ctypes.c_void_p)]),
    "ts_load_vehicles": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint32, u32p, u32p, u32p]),
    "ts_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint32, ctypes.c_void_p]),
    "ts_reset": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "ts_step_timed": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint32, ctypes.c_void_p, ctypes.c_void_p,
                                     ctypes.c_void_p]),
    "ts_read_stats": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(Stats), ctypes.c_uint32]),
    "ts_read_stats_range": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_void_p,
                                           ctypes.c_uint32]),
    "ts_read_totals": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(Totals), ctypes.c_uint32]),
    "ts_state_sizes": (ctypes.c_int, [ctypes.c_void_p, u64p, u32p, u32p, u32p]),
    "ts_read_state": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(State), ctypes.c_uint32]),
    "ts_write_state": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(State)]),
    "ts_footprint_bytes": (ctypes.c_size_t, [ctypes.POINTER(NetworkDesc), ctypes.c_uint32, ctypes.c_uint64]),
    "ts_last_error": (ctypes.c_char_p, []),
    "ts_destroy": (None, [ctypes.c_void_p]),
    "ts_batch_create": (ctypes.c_int, [ctypes.c_uint32, ctypes.POINTER(ctypes.c_void_p)]),
    "ts_batch_add": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint64]),
    "ts_batch_add_many": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p), ctypes.c_uint32,
                                         ctypes.c_uint64]),
    "ts_batch_remove": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "ts_batch_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint32, ctypes.c_void_p]),
    "ts_batch_sync": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint32]),
    "ts_batch_reset": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p]),
    "ts_ctx_step": (ctypes.c_int, [ctypes.c_void_p, u64p]),
    "ts_batch_destroy": (None, [ctypes.c_void_p]),
    "ts_set_tile_words": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint32]),
    "ts_set_step_mode": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint32]),
    "ts_save_state": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(ctypes.c_size_t),
                                     ctypes.c_uint32]),
    "ts_load_state": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t]),
    "ts_tile_words": (ctypes.c_uint32, [ctypes.c_void_p]),
    "ts_read_link_times": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint32]),
    "ts_batch_set_step_mode": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint32]),
    "ts_launches_per_step": (ctypes.c_uint32, []),
    "ts_philox_words": (ctypes.c_int, [ctypes.c_uint32, u32p, u32p, ctypes.c_uint64, u32p]),
    "ts_set_load_balance": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint32]),
    "ts_set_kernel_timing": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint32]),
    "ts_set_link_grid": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint32]),
    "ts_batch_set_link_grid": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint32]),
    "ts_read_kernel_times": (ctypes.c_int, [ctypes.c_void_p, u64p, ctypes.c_uint32, ctypes.c_uint32]),
    "ts_ring_step_noalloc": (ctypes.c_int, [ctypes.c_uint32, ctypes.c_uint32, ctypes.POINTER(Params), ctypes.c_uint64,
                                            ctypes.c_uint32] + [ctypes.c_void_p] * 8),
}

_lib = None


def lib():
    """Loads libtranssim.so (built in-tree by __graft_entry__.build())."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build the CUDA library first "
                               "(python -c 'import __graft_entry__ as g; g.build()')")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _API.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def exported_symbols():
    return list(_API)


def philox_words(step, vehicle_id, seed: int) -> np.ndarray:
    """Word 0 of Philox-4x32-10 for counters (step[i], vehicle_id[i], 0, 0)
    and the seed's key, computed by the library's step-kernel draw."""
    c0 = np.ascontiguousarray(step, np.uint32)
    c1 = np.ascontiguousarray(vehicle_id, np.uint32)
    out = np.zeros(c0.size, np.uint32)
    _check(lib().ts_philox_words(c0.size, _p(c0, ctypes.c_uint32), _p(c1, ctypes.c_uint32), int(seed),
                                 _p(out, ctypes.c_uint32)))
    return out


def _check(rc):
    if rc != TS_OK:
        raise TsError(rc, lib().ts_last_error().decode(errors="replace"))


def _p(a, t):
    return a.ctypes.data_as(ctypes.POINTER(t))


def _stream_handle(stream) -> Optional[int]:
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


class _NetArrays:
    def __init__(self, net):
        self.lf = np.ascontiguousarray(net.link_from, np.uint32)
        self.lt = np.ascontiguousarray(net.link_to, np.uint32)
        self.lc = np.ascontiguousarray(net.link_cells, np.uint32)
        self.ll = np.ascontiguousarray(net.link_lanes, np.uint32)
        self.lr = np.ascontiguousarray(net.link_ring, np.uint8)
        sig = getattr(net, "link_signal", None)
        self.ls = None if sig is None else np.ascontiguousarray(sig, np.uint32).reshape(-1)
        turn = getattr(net, "turn_lanes", None)
        self.tl = None if turn is None else np.ascontiguousarray(turn, np.uint8).reshape(-1)
        ly = getattr(net, "link_yield", None)
        self.ly = None if ly is None else np.ascontiguousarray(ly, np.uint8).reshape(-1)
        self.desc = NetworkDesc(net.n_nodes, net.n_links, _p(self.lf, ctypes.c_uint32), _p(self.lt, ctypes.c_uint32),
                                _p(self.lc, ctypes.c_uint32), _p(self.ll, ctypes.c_uint32), _p(self.lr, ctypes.c_uint8),
                                _p(self.ls, ctypes.c_uint32) if self.ls is not None else None,
                                _p(self.tl, ctypes.c_uint8) if self.tl is not None else None,
                                _p(self.ly, ctypes.c_uint8) if self.ly is not None else None)


def footprint_bytes(scenario) -> int:
    na = _NetArrays(scenario.net)
    return int(lib().ts_footprint_bytes(ctypes.byref(na.desc), scenario.demand.n,
                                        int(scenario.demand.route_offsets[-1])))


def _torch_allocator():
    import torch

    # all contexts allocate on the calling thread's current stream, so blocks
    # freed by finished jobs are reused by the next ones
    def _alloc(nbytes, stream, user):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes))
        except Exception:
            return None

    def _free(ptr, nbytes, stream, user):
        torch.cuda.caching_allocator_delete(int(ptr))

    fa, ff = ALLOC_FN(_alloc), FREE_FN(_free)
    return Allocator(fa, ff, None), (fa, ff)


class Simulation:
    """One scenario on the current CUDA device (wraps a ts_ctx)."""

    def __init__(self, scenario, use_torch_allocator: bool = False, tile_words: Optional[int] = None):
        L = lib()
        self.scenario = scenario
        net, dem = scenario.net, scenario.demand
        self._net = _NetArrays(net)
        params = Params(scenario.vmax, scenario.p_threshold, scenario.seed, scenario.lane_change, 0)
        self._alloc_keep = None
        alloc = None
        if use_torch_allocator:
            a, keep = _torch_allocator()
            self._alloc_keep = (a, keep)
            alloc = ctypes.byref(a)
        h = ctypes.c_void_p()
        _check(L.ts_create_network(ctypes.byref(self._net.desc), ctypes.byref(params), alloc, ctypes.byref(h)))
        self.h = h
        if tile_words is not None:
            _check(L.ts_set_tile_words(self.h, tile_words))
        dep = np.ascontiguousarray(dem.depart_step, np.uint32)
        off = np.ascontiguousarray(dem.route_offsets, np.uint32)
        links = np.ascontiguousarray(dem.route_links, np.uint32)
        rc = L.ts_load_vehicles(self.h, dem.n, _p(dep, ctypes.c_uint32), _p(off, ctypes.c_uint32),
                                _p(links, ctypes.c_uint32))
        if rc != TS_OK:
            msg = L.ts_last_error().decode(errors="replace")
            L.ts_destroy(self.h)
            self.h = None
            raise TsError(rc, msg)
        cells, lanes, veh, nl = ctypes.c_uint64(), ctypes.c_uint32(), ctypes.c_uint32(), ctypes.c_uint32()
        _check(L.ts_state_sizes(self.h, ctypes.byref(cells), ctypes.byref(lanes), ctypes.byref(veh), ctypes.byref(nl)))
        self.n_lane_cells, self.n_lanes, self.n_veh, self.n_links = cells.value, lanes.value, veh.value, nl.value
        if scenario.init is not None:
            self.write_state(scenario.init)

    def close(self):
        if getattr(self, "h", None):
            lib().ts_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_load_balance(self, every_steps: int, vehicles_per_tile: int = 1024):
        _check(lib().ts_set_load_balance(self.h, every_steps, vehicles_per_tile))

    def set_tile_words(self, words: int):
        _check(lib().ts_set_tile_words(self.h, words))

    @property
    def tile_words(self) -> int:
        return int(lib().ts_tile_words(self.h))

    def save(self, timeout_ms: int = 600000) -> bytes:
        """A checkpoint of the current state (ts_save_state)."""
        n = ctypes.c_size_t(0)
        _check(lib().ts_save_state(self.h, None, ctypes.byref(n), timeout_ms))
        buf = ctypes.create_string_buffer(n.value)
        _check(lib().ts_save_state(self.h, buf, ctypes.byref(n), timeout_ms))
        return buf.raw[:n.value]

    def load(self, checkpoint: bytes):
        """Replaces the state by a checkpoint from save() (ts_load_state)."""
        _check(lib().ts_load_state(self.h, ctypes.c_char_p(checkpoint), len(checkpoint)))

    def link_times(self, timeout_ms: int = 600000):
        """Per-link travel-time sums and counts of completed traversals (uint64 arrays)."""
        tsum = np.zeros(self.n_links, np.uint64)
        tcnt = np.zeros(self.n_links, np.uint64)
        _check(lib().ts_read_link_times(self.h, tsum.ctypes.data_as(ctypes.c_void_p),
                                        tcnt.ctypes.data_as(ctypes.c_void_p), timeout_ms))
        return tsum, tcnt

    def set_link_grid(self, blocks_per_sm: int):
        """Link-kernel blocks per SM (0: every resident block); results do not depend on it."""
        _check(lib().ts_set_link_grid(self.h, blocks_per_sm))

    def set_kernel_timing(self, on: bool):
        """Launches of later ts_step calls record their spans inside the graphs."""
        _check(lib().ts_set_kernel_timing(self.h, 1 if on else 0))

    def kernel_times(self, reset: bool = False, timeout_ms: int = 600000) -> dict:
        """Summed in-graph durations: link/node kernel seconds and launch counts."""
        out = np.zeros(4, np.uint64)
        _check(lib().ts_read_kernel_times(self.h, _p(out, ctypes.c_uint64), 1 if reset else 0, timeout_ms))
        return {"link_s": int(out[0]) * 1e-9, "link_launches": int(out[1]),
                "node_s": int(out[2]) * 1e-9, "node_launches": int(out[3])}

    def set_step_mode(self, mode: int):
        """STEP_AUTO, STEP_FUSED or STEP_SPLIT; results do not depend on it."""
        _check(lib().ts_set_step_mode(self.h, mode))

    def step(self, n: int, stream=None):
        s = _stream_handle(stream)
        _check(lib().ts_step(self.h, n, ctypes.c_void_p(s) if s else None))

    def reset(self, stream=None):
        s = _stream_handle(stream)
        _check(lib().ts_reset(self.h, ctypes.c_void_p(s) if s else None))

    def step_timed(self, n: int, stream=None):
        """Runs n steps with a CUDA event around every kernel; returns the
        per-step durations (ms) of the link kernel and the node kernel."""
        s = _stream_handle(stream)
        a = np.zeros(n, np.float32)
        b = np.zeros(n, np.float32)
        _check(lib().ts_step_timed(self.h, n, ctypes.c_void_p(s) if s else None, a.ctypes.data_as(ctypes.c_void_p),
                                   b.ctypes.data_as(ctypes.c_void_p)))
        return a, b

    def stats(self, timeout_ms: int = 600000) -> dict:
        st = Stats()
        _check(lib().ts_read_stats(self.h, ctypes.byref(st), timeout_ms))
        return {f: getattr(st, f) for f in STATS_FIELDS}

    def totals(self, timeout_ms: int = 600000) -> dict:
        t = Totals()
        _check(lib().ts_read_totals(self.h, ctypes.byref(t), timeout_ms))
        return {f: getattr(t, f) for f in TOTALS_FIELDS}

    def stats_range(self, first: int, n: int, timeout_ms: int = 600000) -> np.ndarray:
        out = np.zeros(n, STATS_DTYPE)
        _check(lib().ts_read_stats_range(self.h, first, n, out.ctypes.data_as(ctypes.c_void_p), timeout_ms))
        return out

    def current_step(self) -> int:
        s = ctypes.c_uint64()
        _check(lib().ts_ctx_step(self.h, ctypes.byref(s)))
        return s.value

    def read_state(self, timeout_ms: int = 600000) -> dict:
        s = dict(cell_id=np.empty(self.n_lane_cells, np.int32), cell_v=np.empty(self.n_lane_cells, np.int8),
                 buf_id=np.empty(self.n_lanes, np.int32), buf_v=np.empty(self.n_lanes, np.int8),
                 cursor=np.empty(self.n_veh, np.uint32), dep_head=np.empty(self.n_links, np.uint32))
        st = State(_p(s["cell_id"], ctypes.c_int32), _p(s["cell_v"], ctypes.c_int8), _p(s["buf_id"], ctypes.c_int32),
                   _p(s["buf_v"], ctypes.c_int8), _p(s["cursor"], ctypes.c_uint32), _p(s["dep_head"], ctypes.c_uint32),
                   0, 0, 0)
        _check(lib().ts_read_state(self.h, ctypes.byref(st), timeout_ms))
        s["step"], s["arrived"], s["inserted"] = st.step, st.arrived, st.inserted
        return s

    def write_state(self, init):
        a = [np.ascontiguousarray(init.cell_id, np.int32), np.ascontiguousarray(init.cell_v, np.int8),
             np.ascontiguousarray(init.buf_id, np.int32), np.ascontiguousarray(init.buf_v, np.int8),
             np.ascontiguousarray(init.cursor, np.uint32), np.ascontiguousarray(init.dep_head, np.uint32)]
        st = State(_p(a[0], ctypes.c_int32), _p(a[1], ctypes.c_int8), _p(a[2], ctypes.c_int32), _p(a[3], ctypes.c_int8),
                   _p(a[4], ctypes.c_uint32), _p(a[5], ctypes.c_uint32), init.step, init.arrived, init.inserted)
        _check(lib().ts_write_state(self.h, ctypes.byref(st)))


class Batch:
    """Many scenarios advanced by the same kernel launches (wraps a ts_batch)."""

    def __init__(self, capacity: int):
        h = ctypes.c_void_p()
        _check(lib().ts_batch_create(capacity, ctypes.byref(h)))
        self.h = h

    def add(self, sim: Simulation, target_step: int):
        _check(lib().ts_batch_add(self.h, sim.h, target_step))

    def add_many(self, sims, target_step: int):
        arr = (ctypes.c_void_p * len(sims))(*[s.h.value for s in sims])
        _check(lib().ts_batch_add_many(self.h, arr, len(sims), target_step))

    def remove(self, sim: Simulation):
        _check(lib().ts_batch_remove(self.h, sim.h))

    def step(self, n: int, stream):
        s = _stream_handle(stream)
        _check(lib().ts_batch_step(self.h, n, ctypes.c_void_p(s)))

    def set_step_mode(self, mode: int):
        _check(lib().ts_batch_set_step_mode(self.h, mode))

    def set_link_grid(self, blocks_per_sm: int):
        _check(lib().ts_batch_set_link_grid(self.h, blocks_per_sm))

    def sync(self, timeout_ms: int = 600000):
        _check(lib().ts_batch_sync(self.h, timeout_ms))

    def reset(self, target_step: int, stream):
        s = _stream_handle(stream)
        _check(lib().ts_batch_reset(self.h, target_step, ctypes.c_void_p(s)))

    def close(self):
        if getattr(self, "h", None):
            lib().ts_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def launches_per_step() -> int:
    return int(lib().ts_launches_per_step())
