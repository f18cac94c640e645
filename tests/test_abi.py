"""The C-ABI library loads on a machine without a GPU and exports every
entry point that include/transsim.h declares; calls fail loudly without a
device instead of falling back to the CPU."""
import os
import re

import pytest

from paper_cs_0105004_gb300 import transsim as T

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(ts_[a-z_0-9]+)\s*\(", src))
    return names


def test_library_exports_every_declared_symbol():
    L = T.lib()
    declared = _declared()
    assert len(declared) >= 20
    for name in sorted(declared):
        assert hasattr(L, name), name
    assert declared == set(T.exported_symbols())


def test_no_silent_fallback_without_device():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_cs_0105004_gb300.inputs import networks as N
    with pytest.raises(T.TsError):
        T.Simulation(N.small_grid_scenario(2, 1, 10, 5, 5, 5))


def test_footprint_grows_with_network():
    from paper_cs_0105004_gb300.inputs import networks as N
    a = T.footprint_bytes(N.small_grid_scenario(3, 1, 10, 10, 10, 10))
    b = T.footprint_bytes(N.small_grid_scenario(5, 2, 60, 100, 10, 10))
    assert 0 < a < b


def test_footprint_counts_the_intersection_tables():
    # turn lanes add one byte per route entry and per traveller; yield
    # approaches add nine bytes per link-end buffer (gap and lane tail)
    from paper_cs_0105004_gb300.inputs import networks as N
    plain = N.small_grid_scenario(4, 3, 20, 300, 100, 10, gen_seed=3)
    turns = N.small_grid_scenario(4, 3, 20, 300, 100, 10, gen_seed=3, turns=True)
    both = N.small_grid_scenario(4, 3, 20, 300, 100, 10, gen_seed=3, turns=True, yield_gap=5)
    a, b, c = (T.footprint_bytes(s) for s in (plain, turns, both))
    route_len = int(plain.demand.route_offsets[-1])
    assert b - a == route_len + plain.demand.n
    assert c - b == 9 * plain.net.n_lanes
