"""Plain CPU oracle of the TRANSIMS cellular-automaton step (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library never loads it.
The arithmetic lives in ``oracle.c`` (plain C, single thread); this module
compiles it with gcc and wraps it with ctypes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "oracle.c")
LIB = os.path.join(HERE, "liboracle.so")

STATS_FIELDS = ("step", "active", "buffered", "waiting", "arrived", "lane_changes", "transfers",
                "inserted", "sum_v", "vehicle_updates", "state_hash", "moving")
STATS_DTYPE = np.dtype([(f, np.uint64) for f in STATS_FIELDS])


def build(force: bool = False) -> str:
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        tmp = LIB + f".tmp{os.getpid()}"
        subprocess.run(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", SRC, "-o", tmp], check=True)
        os.replace(tmp, LIB)
    return LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = bind(build())
    return _lib


def bind(path: str):
    """Loads a build of oracle.c from `path` and declares its functions."""
    L = ctypes.CDLL(path)
    P = ctypes.POINTER
    u32p, u64p, i32p, i8p, u8p = P(ctypes.c_uint32), P(ctypes.c_uint64), P(ctypes.c_int32), P(ctypes.c_int8), P(ctypes.c_uint8)
    L.oracle_create.restype = ctypes.c_void_p
    L.oracle_create.argtypes = [ctypes.c_uint32, ctypes.c_uint32, u32p, u32p, u32p, u32p, u8p, u32p, u8p, u8p,
                                ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_uint32]
    L.oracle_destroy.argtypes = [ctypes.c_void_p]
    L.oracle_load_vehicles.restype = ctypes.c_int
    L.oracle_load_vehicles.argtypes = [ctypes.c_void_p, ctypes.c_uint32, u32p, u32p, u32p]
    L.oracle_step.restype = ctypes.c_int
    L.oracle_step.argtypes = [ctypes.c_void_p, ctypes.c_uint32, ctypes.c_void_p]
    L.oracle_n_cells.restype = ctypes.c_uint64
    L.oracle_n_cells.argtypes = [ctypes.c_void_p]
    L.oracle_n_lanes.restype = ctypes.c_uint32
    L.oracle_n_lanes.argtypes = [ctypes.c_void_p]
    L.oracle_get_state.argtypes = [ctypes.c_void_p, i32p, i8p, i32p, i8p, u32p, u32p, u64p]
    L.oracle_set_state.restype = ctypes.c_int
    L.oracle_set_state.argtypes = [ctypes.c_void_p, i32p, i8p, i32p, i8p, u32p, u32p, u64p]
    L.oracle_philox4x32_10.argtypes = [u32p, u32p, u32p]
    L.oracle_splitmix64.restype = ctypes.c_uint64
    L.oracle_splitmix64.argtypes = [ctypes.c_uint64]
    L.oracle_vehicle_term.restype = ctypes.c_uint64
    L.oracle_vehicle_term.argtypes = [ctypes.c_uint32] * 5
    L.oracle_link_times.argtypes = [ctypes.c_void_p, u64p, u64p]
    return L


def _p(a, t):
    return a.ctypes.data_as(ctypes.POINTER(t))


def philox4x32_10(ctr, key):
    c = np.ascontiguousarray(ctr, np.uint32)
    k = np.ascontiguousarray(key, np.uint32)
    out = np.zeros(4, np.uint32)
    lib().oracle_philox4x32_10(_p(c, ctypes.c_uint32), _p(k, ctypes.c_uint32), _p(out, ctypes.c_uint32))
    return out


def splitmix64(z: int) -> int:
    return int(lib().oracle_splitmix64(z))


def vehicle_term(id_, link, lane, cell, v) -> int:
    return int(lib().oracle_vehicle_term(id_, link, lane, cell, v))


class Oracle:
    """One scenario simulated by the plain C oracle."""

    def __init__(self, scenario):
        net, dem = scenario.net, scenario.demand
        L = lib()
        self._keep = [np.ascontiguousarray(a, np.uint32) for a in
                      (net.link_from, net.link_to, net.link_cells, net.link_lanes)]
        ring = np.ascontiguousarray(net.link_ring, np.uint8)
        sig = getattr(net, "link_signal", None)
        self._sig = None if sig is None else np.ascontiguousarray(sig, np.uint32).reshape(-1)
        turn = getattr(net, "turn_lanes", None)
        self._turn = None if turn is None else np.ascontiguousarray(turn, np.uint8).reshape(-1)
        ga = getattr(net, "link_yield", None)
        self._yield = None if ga is None else np.ascontiguousarray(ga, np.uint8).reshape(-1)
        self.h = L.oracle_create(net.n_nodes, net.n_links, *[_p(a, ctypes.c_uint32) for a in self._keep],
                                 _p(ring, ctypes.c_uint8),
                                 _p(self._sig, ctypes.c_uint32) if self._sig is not None else None,
                                 _p(self._turn, ctypes.c_uint8) if self._turn is not None else None,
                                 _p(self._yield, ctypes.c_uint8) if self._yield is not None else None,
                                 scenario.vmax, scenario.p_threshold, scenario.seed, scenario.lane_change)
        if not self.h:
            raise ValueError("oracle rejected the network")
        dep = np.ascontiguousarray(dem.depart_step, np.uint32)
        off = np.ascontiguousarray(dem.route_offsets, np.uint32)
        links = np.ascontiguousarray(dem.route_links, np.uint32)
        if L.oracle_load_vehicles(self.h, dem.n, _p(dep, ctypes.c_uint32), _p(off, ctypes.c_uint32),
                                  _p(links, ctypes.c_uint32)) != 0:
            raise ValueError("oracle rejected the vehicles")
        self.n_links = net.n_links
        self.n_veh = dem.n
        self.n_cells = int(L.oracle_n_cells(self.h))
        self.n_lanes = int(L.oracle_n_lanes(self.h))
        if scenario.init is not None:
            self.set_state(scenario.init)

    def close(self):
        if self.h:
            lib().oracle_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, n: int) -> np.ndarray:
        out = np.zeros(n, STATS_DTYPE)
        lib().oracle_step(self.h, n, out.ctypes.data_as(ctypes.c_void_p))
        return out

    def get_state(self) -> dict:
        s = dict(cell_id=np.empty(self.n_cells, np.int32), cell_v=np.empty(self.n_cells, np.int8),
                 buf_id=np.empty(self.n_lanes, np.int32), buf_v=np.empty(self.n_lanes, np.int8),
                 cursor=np.empty(self.n_veh, np.uint32), dep_head=np.empty(self.n_links, np.uint32))
        sc = np.zeros(3, np.uint64)
        lib().oracle_get_state(self.h, _p(s["cell_id"], ctypes.c_int32), _p(s["cell_v"], ctypes.c_int8),
                               _p(s["buf_id"], ctypes.c_int32), _p(s["buf_v"], ctypes.c_int8),
                               _p(s["cursor"], ctypes.c_uint32), _p(s["dep_head"], ctypes.c_uint32),
                               _p(sc, ctypes.c_uint64))
        s["step"], s["arrived"], s["inserted"] = int(sc[0]), int(sc[1]), int(sc[2])
        return s

    def set_state(self, init):
        a = [np.ascontiguousarray(init.cell_id, np.int32), np.ascontiguousarray(init.cell_v, np.int8),
             np.ascontiguousarray(init.buf_id, np.int32), np.ascontiguousarray(init.buf_v, np.int8),
             np.ascontiguousarray(init.cursor, np.uint32), np.ascontiguousarray(init.dep_head, np.uint32)]
        sc = np.array([init.step, init.arrived, init.inserted], np.uint64)
        rc = lib().oracle_set_state(self.h, _p(a[0], ctypes.c_int32), _p(a[1], ctypes.c_int8),
                                    _p(a[2], ctypes.c_int32), _p(a[3], ctypes.c_int8),
                                    _p(a[4], ctypes.c_uint32), _p(a[5], ctypes.c_uint32), _p(sc, ctypes.c_uint64))
        if rc != 0:
            raise ValueError("oracle rejected the state")

    def link_times(self):
        """Per-link travel-time sums and counts of completed traversals."""
        tsum = np.zeros(self.n_links, np.uint64)
        tcnt = np.zeros(self.n_links, np.uint64)
        lib().oracle_link_times(self.h, _p(tsum, ctypes.c_uint64), _p(tcnt, ctypes.c_uint64))
        return tsum, tcnt
