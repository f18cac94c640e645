"""ts_ring_step_noalloc: stepping a ring road held in the caller's own device
buffers, for callers that cannot let the library allocate GPU memory.

Checks, through the C ABI, that two calls in a row give exactly the same
statistics and final state as the allocating path (ts_create_network +
ts_write_state + ts_step) on the same ring; all step arithmetic is integer,
so the comparison is exact.  Collected last on purpose (file name).
"""
import ctypes

import numpy as np
import pytest

from paper_cs_0105004_gb300 import transsim as T
from paper_cs_0105004_gb300.inputs import networks as N

pytestmark = pytest.mark.gpu


def _to_layout(init, cells, lanes):
    nw = cells // 32 * lanes
    occ = np.zeros(nw, np.uint32)
    vel = np.zeros(nw * 32, np.int8)
    vid = np.zeros(nw * 32, np.uint32)
    for k in range(lanes):
        for x in np.nonzero(init.cell_id[k * cells:(k + 1) * cells] >= 0)[0]:
            w = (x // 32) * lanes + k
            occ[w] |= np.uint32(1 << (x % 32))
            vel[w * 32 + x % 32] = init.cell_v[k * cells + x]
            vid[w * 32 + x % 32] = init.cell_id[k * cells + x]
    return occ, vel, vid


def _from_layout(occ, vel, vid, cells, lanes):
    cell_id = np.full(cells * lanes, -1, np.int32)
    cell_v = np.zeros(cells * lanes, np.int8)
    for w in np.nonzero(occ)[0]:
        j, k = divmod(int(w), lanes)
        m = int(occ[w])
        for i in range(32):
            if m >> i & 1:
                cell_id[k * cells + 32 * j + i] = vid[w * 32 + i]
                cell_v[k * cells + 32 * j + i] = vel[w * 32 + i]
    return cell_id, cell_v


@pytest.mark.parametrize("cells,lanes,rho", [(320, 1, 0.25), (9984, 3, 0.3)])
def test_noalloc_ring_matches_allocating_path_on_two_calls(cells, lanes, rho):
    import torch

    net = N.ring_network(cells, lanes)
    dem, init = N.ring_initial_state(net, int(rho * cells * lanes), "random", 0, np.random.default_rng(cells + lanes))
    sc = N.Scenario("ring", net, dem, 0, 9, 5, N.P_THRESHOLD_0_2, 1, init)
    calls = (150, 250)

    ref = T.Simulation(sc)
    ref_stats = []
    first = 0
    for n in calls:
        ref.step(n)
        ref_stats.append(ref.stats_range(first, n))
        first += n
    ref_state = ref.read_state()
    ref.close()

    dev = torch.device("cuda", 0)
    occ, vel, vid = _to_layout(init, cells, lanes)
    nw = occ.size
    b_occ = [torch.zeros(nw, dtype=torch.int32, device=dev) for _ in range(2)]
    b_vel = [torch.zeros(nw * 32, dtype=torch.int8, device=dev) for _ in range(2)]
    b_vid = [torch.zeros(nw * 32, dtype=torch.int32, device=dev) for _ in range(2)]
    b_occ[0].copy_(torch.from_numpy(occ.view(np.int32)))
    b_vel[0].copy_(torch.from_numpy(vel))
    b_vid[0].copy_(torch.from_numpy(vid.view(np.int32)))
    params = T.Params(sc.vmax, sc.p_threshold, sc.seed, sc.lane_change, 0)
    stream = torch.cuda.current_stream(dev)
    first = 0
    for n, want in zip(calls, ref_stats):
        out = torch.zeros((n, len(T.STATS_FIELDS)), dtype=torch.int64, device=dev)
        ptrs = [b_occ[0], b_occ[1], b_vel[0], b_vel[1], b_vid[0], b_vid[1], out]
        rc = T.lib().ts_ring_step_noalloc(cells, lanes, ctypes.byref(params), first, n,
                                          *[ctypes.c_void_p(p.data_ptr()) for p in ptrs],
                                          ctypes.c_void_p(stream.cuda_stream))
        assert rc == T.TS_OK, T.lib().ts_last_error().decode()
        torch.cuda.synchronize()
        got = out.cpu().numpy().view(np.uint64).reshape(n, len(T.STATS_FIELDS))
        for c, f in enumerate(T.STATS_FIELDS):
            assert np.array_equal(got[:, c], want[f]), (first, f)
        first += n
    cur = first & 1
    cell_id, cell_v = _from_layout(b_occ[cur].cpu().numpy().view(np.uint32), b_vel[cur].cpu().numpy(),
                                   b_vid[cur].cpu().numpy().view(np.uint32), cells, lanes)
    assert np.array_equal(cell_id, ref_state["cell_id"])
    assert np.array_equal(cell_v, ref_state["cell_v"])


def test_noalloc_rejects_sizes_beyond_its_limits():
    params = T.Params(5, 0, 1, 1, 0)
    dummy = [ctypes.c_void_p(16)] * 7
    for cells, lanes, n in ((33, 1, 10), (1 << 18, 1, 10), (64, 5, 10), (64, 1, 2000)):
        rc = T.lib().ts_ring_step_noalloc(cells, lanes, ctypes.byref(params), 0, n, *dummy, None)
        assert rc == T.TS_ERR_INVALID
