"""A second, deliberately naive restatement of the step rules (test only).

It exists to pin the C oracle on tiny inputs: a slip in either (a dropped
term, a wrong index or sign) shows up as a state mismatch.  It keeps the
state as dictionaries keyed by position and re-derives everything from the
rules of Sec. 3 (car following, lane changing, signals, lane changing for
plan following, gap acceptance at unprotected turns) and Sec. 4 (sub-step
order, entry from parking), with the same readings of the points the paper
leaves open as the oracle documents.  It has its own Philox-4x32-10.
"""
from __future__ import annotations

MASK32 = 0xFFFFFFFF


def philox(ctr, key):
    """Philox-4x32-10 (Salmon et al., SC'11)."""
    x = list(ctr)
    k0, k1 = key
    for _ in range(10):
        p0 = 0xD2511F53 * x[0]
        p1 = 0xCD9E8D57 * x[2]
        x = [((p1 >> 32) ^ x[1] ^ k0) & MASK32, p1 & MASK32, ((p0 >> 32) ^ x[3] ^ k1) & MASK32, p0 & MASK32]
        k0 = (k0 + 0x9E3779B9) & MASK32
        k1 = (k1 + 0xBB67AE85) & MASK32
    return x


class Brute:
    def __init__(self, sc):
        net, dem = sc.net, sc.demand
        self.vmax, self.p, self.seed, self.lc = sc.vmax, sc.p_threshold, sc.seed, sc.lane_change
        self.cells = [int(c) for c in net.link_cells]
        self.lanes = [int(c) for c in net.link_lanes]
        self.ring = [bool(r) for r in net.link_ring]
        self.frm = [int(c) for c in net.link_from]
        self.to = [int(c) for c in net.link_to]
        self.n_nodes = net.n_nodes
        # turn lanes: (link, next link) -> set of lanes; the table lists, per
        # link, the links leaving its end node in ascending id
        self.turn = None
        if getattr(net, "turn_lanes", None) is not None:
            self.turn = {}
            j = 0
            for l in range(len(self.cells)):
                if self.ring[l]:
                    continue
                for m in sorted(m for m in range(len(self.cells)) if self.frm[m] == self.to[l] and not self.ring[m]):
                    self.turn[(l, m)] = {k for k in range(self.lanes[l]) if int(net.turn_lanes[j]) >> k & 1}
                    j += 1
        sig = getattr(net, "link_signal", None)
        self.sig = None if sig is None else [tuple(int(x) for x in row) for row in sig]
        ga = getattr(net, "link_yield", None)
        self.gap_accept = [0] * len(self.cells) if ga is None else [int(g) for g in ga]
        off = [int(c) for c in dem.route_offsets]
        self.routes = [[int(x) for x in dem.route_links[off[i]:off[i + 1]]] for i in range(dem.n)]
        self.depart = [int(x) for x in dem.depart_step]
        self.occ = {}      # (link, lane, x) -> id
        self.buf = {}      # (link, lane) -> id
        self.v = {}
        self.cur = {}
        self.arrived = 0
        self.queue = {}
        for i in sorted(range(dem.n), key=lambda i: (self.depart[i], i)):
            self.queue.setdefault(self.routes[i][0], []).append(i)
        self.done_ids = set()
        self.t = 0
        if sc.init is not None:
            self._load(sc.init, net)

    def _load(self, init, net):
        lb = net.lane_base(); cb = net.lane_cell_base()
        for l in range(len(self.cells)):
            for k in range(self.lanes[l]):
                ln = lb[l] + k
                for x in range(self.cells[l]):
                    i = int(init.cell_id[cb[ln] + x])
                    if i >= 0:
                        self.occ[(l, k, x)] = i; self.v[i] = int(init.cell_v[cb[ln] + x])
                if init.buf_id[ln] >= 0:
                    i = int(init.buf_id[ln]); self.buf[(l, k)] = i; self.v[i] = int(init.buf_v[ln])
        for i, c in enumerate(init.cursor):
            self.cur[i] = int(c)
        for l, q in self.queue.items():
            h = int(init.dep_head[l])
            for i in q[:h]:
                self.done_ids.add(i)
            self.queue[l] = q[h:]
        self.t = init.step
        self.arrived = init.arrived

    def last(self, i):
        return self.cur[i] == len(self.routes[i]) - 1

    def allowed(self, i, l):
        if self.turn is None or self.last(i):
            return set(range(self.lanes[l]))
        return self.turn[(l, self.routes[i][self.cur[i] + 1])]

    def green(self, l):
        if self.sig is None or self.sig[l][0] == 0:
            return True
        cycle, green, offset = self.sig[l]
        return (self.t + offset) % cycle < green

    def gap(self, occ, buf, l, k, x, i):
        L = self.cells[l]
        g = 0
        while g < self.vmax:
            y = x + g + 1
            if y >= L and not self.ring[l]:
                if ((l, k) not in buf or self.last(i)) and k in self.allowed(i, l) and self.green(l):
                    g += 1
                return min(g, self.vmax)
            if (l, k, y % L) in occ:
                return g
            g += 1
        return g

    def step(self):
        t = self.t
        d = 1 if t % 2 == 0 else -1
        vmax = self.vmax
        old = dict(self.occ)
        buf0 = dict(self.buf)
        lc = 0
        moves = []
        if self.lc:
            for (l, k, x), i in old.items():
                kt = k + d
                if not (0 <= kt < self.lanes[l]):
                    continue
                go = self.gap(old, buf0, l, k, x, i)
                gt = self.gap(old, buf0, l, kt, x, i)
                ok = self.allowed(i, l)
                need_lane = k not in ok and any((j - k) * d > 0 for j in ok)
                faster = go < min(self.v[i] + 1, vmax) and gt > go and kt in ok
                if not (need_lane or faster):
                    continue
                L = self.cells[l]
                back = vmax
                if need_lane and not self.ring[l]:
                    back = min(vmax, L - 1 - x)
                behind = range(x - back, x + 1) if self.ring[l] else range(max(0, x - back), x + 1)
                if any((l, kt, y % L) in old for y in behind):
                    continue
                moves.append(((l, k, x), (l, kt, x), i))
        mid = dict(old)
        for a, b, i in moves:
            del mid[a]
        for a, b, i in moves:
            mid[b] = i
        lc = len(moves)
        new = {}
        upd = 0
        for (l, k, x), i in mid.items():
            upd += 1
            v = min(self.v[i] + 1, vmax)
            v = min(v, self.gap(mid, buf0, l, k, x, i))
            if v > 0 and philox([t & MASK32, i, 0, 0], [self.seed & MASK32, self.seed >> 32])[0] < self.p:
                v -= 1
            self.v[i] = v
            L = self.cells[l]
            nx = x + v
            if self.ring[l]:
                nx %= L
            if nx < L:
                assert (l, k, nx) not in new
                new[(l, k, nx)] = i
            elif self.last(i):
                self.arrived += 1
            else:
                assert (l, k) not in self.buf
                self.buf[(l, k)] = i
        transfers = 0
        for n in range(self.n_nodes):
            inc = sorted((l for l in range(len(self.cells)) if self.to[l] == n and not self.ring[l]),
                         key=lambda l: (self.gap_accept[l] > 0, l))
            # the gap on the priority approaches, judged after the moves
            def clear(G):
                for p in inc:
                    if self.gap_accept[p] == 0:
                        L = self.cells[p]
                        if any((p, k, x) in new for k in range(self.lanes[p]) for x in range(max(1, L - G), L)):
                            return False
                return True
            for l in inc:
                for k in range(self.lanes[l]):
                    if (l, k) not in self.buf:
                        continue
                    if self.gap_accept[l] and not clear(self.gap_accept[l]):
                        continue
                    i = self.buf[(l, k)]
                    m = self.routes[i][self.cur[i] + 1]
                    p = min(k, self.lanes[m] - 1)
                    for q in [p] + [q for q in range(self.lanes[m]) if q != p]:
                        if (m, q, 0) not in new:
                            new[(m, q, 0)] = i
                            del self.buf[(l, k)]
                            self.cur[i] += 1
                            transfers += 1
                            break
        inserted = 0
        for m in range(len(self.cells)):
            q = self.queue.get(m, [])
            while q and self.depart[q[0]] <= t:
                free = [lane for lane in range(self.lanes[m]) if (m, lane, 0) not in new]
                if not free:
                    break
                i = q.pop(0)
                new[(m, free[0], 0)] = i
                self.v[i] = 0
                self.cur[i] = 0
                self.done_ids.add(i)
                inserted += 1
        self.occ = new
        self.t = t + 1
        waiting = sum(1 for m, q in self.queue.items() for i in q if self.depart[i] <= t)
        return dict(step=t, active=len(new), buffered=len(self.buf), waiting=waiting, arrived=self.arrived,
                    lane_changes=lc, transfers=transfers, inserted=inserted,
                    sum_v=sum(self.v[i] for i in new.values()), vehicle_updates=upd,
                    moving=sum(1 for i in new.values() if self.v[i] > 0))

    def state(self, net):
        import numpy as np
        lb = net.lane_base(); cb = net.lane_cell_base()
        cell_id = np.full(net.n_lane_cells, -1, np.int32)
        cell_v = np.zeros(net.n_lane_cells, np.int8)
        for (l, k, x), i in self.occ.items():
            cell_id[cb[lb[l] + k] + x] = i
            cell_v[cb[lb[l] + k] + x] = self.v[i]
        buf_id = np.full(net.n_lanes, -1, np.int32)
        buf_v = np.zeros(net.n_lanes, np.int8)
        for (l, k), i in self.buf.items():
            buf_id[lb[l] + k] = i
            buf_v[lb[l] + k] = self.v[i]
        return cell_id, cell_v, buf_id, buf_v
