// Step kernels of the TRANSIMS cellular automaton for sm_103a.
//
// One time step (Sec. 3 and Sec. 4 of Nagel & Rickert) is two launches:
//
//   link_kernel  lane change (sub-step 1), velocity update and move
//                (sub-step 2) of every vehicle on every lane.  It reads the
//                state of step t (set t&1) and writes the cells of step t+1
//                (set (t+1)&1); a vehicle reaching its link end enters the
//                lane's link-end buffer, or leaves on its last link.
//   node_kernel  node transfer: for every link m, the buffered vehicles at
//                m's upstream node whose next link is m, in fixed priority
//                order (incoming link id, then lane), move to cell 0 of m;
//                then departures from parking enter m.
// (Fused steps fold the node transfer of step t-1 into the link kernel of
// step t and run the node kernel once per chunk.)  turn_link_kernel and
// turn_node_kernel are the same bodies with the intersection rules a network
// may add (turn lanes for plan-following lane changes, yield approaches for
// gap acceptance); signals need no other instance.  Once per captured chunk
// of steps, advance_kernel closes the chunk's statistics and moves the step
// counter; inside a chunk the step index of a launch is the chunk base plus
// the launch's position.
//
// The paper's split-link boundary exchange (Sec. 4: each CPU sends the
// first five cells of its half of a split link to the other) becomes a
// one-column halo here: a block owns a tile of 32-cell columns and
// re-computes the lane-change decisions of the vehicles in the neighbouring
// column that can influence its own cells instead of exchanging them.
// Inside a tile, occupancy, moving and location words are staged in shared
// memory.  Stopped vehicles whose next cell stays occupied are handled 32 at
// a time with bit operations and never touch their payload; the others are
// compacted into a list, one thread per vehicle, so the cost follows the
// number of vehicles that move or may move.  Gaps come from a 64-bit window
// of two occupancy words and one find-first-set.
#include "internal.h"

namespace tsim {

// ------------------------------------------------------------------ arithmetic

// Philox-4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), word 0 of the output.
__device__ __forceinline__ uint32_t philox_word0(uint32_t c0, uint32_t c1, uint32_t k0, uint32_t k1) {
    uint32_t c2 = 0u, c3 = 0u;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c0, hi0 = __umulhi(0xD2511F53u, c0);
        const uint32_t lo1 = 0xCD9E8D57u * c2, hi1 = __umulhi(0xCD9E8D57u, c2);
        const uint32_t n0 = hi1 ^ c1 ^ k0;
        const uint32_t n2 = hi0 ^ c3 ^ k1;
        c1 = lo1;
        c3 = lo0;
        c0 = n0;
        c2 = n2;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c0;
}

#ifdef TS_PHASE_TIMING
// Measurement builds only: stamp(phase, first) calls placed by hand at the
// phase boundaries of link_step record %globaltimer for the first tile of
// every link_kernel block of the last launch and sum each phase's time over
// all tiles of warp 0 of every block (the source carries no calls; without
// TS_PHASE_TIMING stamp() is empty).
constexpr int kPhases = 10;
constexpr int kPhaseBlocks = 4096;
__device__ unsigned long long g_phase[kPhases][kPhaseBlocks];
// and the time spent in each phase summed over all tiles of all blocks
__device__ unsigned long long g_phase_sum[kPhases];
static __shared__ unsigned long long s_phase_last;
__device__ __forceinline__ void stamp(int ph, bool first) {
    if (threadIdx.x == 0) {
        unsigned long long t;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
        if (first && blockIdx.x < kPhaseBlocks) g_phase[ph][blockIdx.x] = t;
        if (ph > 0) atomicAdd(&g_phase_sum[ph], t - s_phase_last);
        s_phase_last = t;
    }
}
#else
__device__ __forceinline__ void stamp(int, bool) {}
#endif

// Kernel spans (ts_set_kernel_timing): with a span buffer, thread 0 of every
// block of a link or node launch at chunk position pos lowers the launch's
// start to the time its wait for the previous kernel returned (so spans of
// consecutive launches do not overlap under programmatic dependent launch)
// and raises its end to its exit time, on the %globaltimer clock; the
// chunk-closing kernel turns them into sums.
// span layout: [kChunk][kind: 0 link, 1 node][start, end], then per kind
// {sum of durations in ns, launches}.
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ void span_mark(unsigned long long *span, uint32_t pos, int kind, bool enter) {
    if (span != nullptr && threadIdx.x == 0 && pos < kChunk) {
        unsigned long long *s = span + (pos * 2u + (uint32_t)kind) * 2u;
        if (enter) atomicMin(s, global_ns());
        else atomicMax(s + 1, global_ns());
    }
}

// Programmatic dependent launch: a kernel lets the next one in its stream
// launch at once, and waits for its predecessor only before touching state.
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

__device__ __forceinline__ StatRec *stat_rec(const ScenDev &D, unsigned long long t) {
    return D.stats + (size_t)(t & (kStatsRing - 1)) * D.n_sub + (blockIdx.x & (D.n_sub - 1));
}

// Sum of NF per-thread counters over the block, added to base[field[f]] once.
template <int NF, int NT>
__device__ __forceinline__ void block_flush(unsigned long long (&acc)[NF], unsigned long long *base,
                                            const int (&field)[NF], unsigned long long (*red)[NF]) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int f = 0; f < NF; ++f) {
        unsigned long long v = acc[f];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) red[warp][f] = v;
        acc[f] = 0;
    }
    __syncthreads();
    if (threadIdx.x < NF) {
        unsigned long long s = 0;
#pragma unroll
        for (int w = 0; w < NT / 32; ++w) s += red[w][threadIdx.x];
        if (s) atomicAdd(base + field[threadIdx.x], s);
    }
    __syncthreads();
}

// ------------------------------------------------------------------ node transfer

// Free lanes of link m at cell 0 (bit k set: cell 0 of lane k is empty in
// occ); the lanes' words are loaded together.
__device__ __forceinline__ uint32_t free_cell0(const uint32_t *__restrict__ occ, const uint4 &nd) {
    const uint32_t lanes = (nd.z >> 8) & 0xFFu;
    uint32_t o[kMaxLanes];
#pragma unroll
    for (int k = 0; k < kMaxLanes; ++k) o[k] = (uint32_t)k < lanes ? occ[nd.y + k] : 1u;
    uint32_t f = 0u;
#pragma unroll
    for (int k = 0; k < kMaxLanes; ++k) f |= ((o[k] & 1u) ^ 1u) << k;
    return f;
}

constexpr int kSlotPrefetch = 8;  // buffers of a node loaded together before resolving

// Loads the first kSlotPrefetch buffers of a node's slot group together.
__device__ __forceinline__ void prefetch_slots(const uint4 *__restrict__ slots, uint32_t slot_lo, uint32_t cnt,
                                               uint4 (&pre)[kSlotPrefetch]) {
#pragma unroll
    for (int s = 0; s < kSlotPrefetch; ++s)
        pre[s] = (uint32_t)s < cnt ? slots[slot_lo + s] : make_uint4(kSlotEmpty, 0u, 0u, 0u);
}

// Gap acceptance at unprotected turns (Sec. 3): true iff none of the
// node's first `prio` slots (the lanes of its priority approaches, from
// slot_lo) has a vehicle in cells max(1, cells - G) .. cells - 1 of its lane
// in occ (the state after the step's moves; cell 0, which transfers write,
// never counts).  G <= 31: at most the last two columns of a lane.
__device__ __forceinline__ bool priority_gap_clear(const uint2 *__restrict__ slot_tail, const uint32_t *__restrict__ occ,
                                                uint32_t slot_lo, uint32_t prio, uint32_t G) {
    for (uint32_t s = 0; s < prio; ++s) {
        const uint2 tl = slot_tail[slot_lo + s];
        const uint32_t L = tl.y & 0xFFFFFFu, lanes = (tl.y >> 24) & 7u;
        const uint32_t lo = L > G ? L - G : 1u;
        if (lo >= L) continue;
        const uint32_t jl = (L - 1u) >> 5, jf = lo >> 5;
        for (uint32_t j = jf; j <= jl; ++j) {
            const uint32_t a = j == jf ? (lo & 31u) : 0u;
            const uint32_t b = j == jl ? ((L - 1u) & 31u) : 31u;
            const uint32_t mask = (0xFFFFFFFFu >> (31u - b)) & (0xFFFFFFFFu << a);
            if (occ[tl.x - (jl - j) * lanes] & mask) return false;
        }
    }
    return true;
}

// Node transfer into link m at the end of a step (Sec. 3): the buffered
// vehicles at m's upstream node whose next link is m, in slot (priority)
// order, each take cell 0 of the preferred lane min(k, lanes(m)-1) if it is
// free, else of the lowest free lane, else stay buffered.  The node's slot
// group is [slot_lo, slot_lo + cnt), its first buffers prefetched in pre;
// free_mask from free_cell0 (after the step's moves).  Calls
// place(slot index, slot, lane) for every placement and returns the lanes
// still free (for departures).  Any number of threads may evaluate the same
// m on the same inputs and get the same placements.  TURNS: with slot_gap,
// a vehicle of a yield approach also needs the gap on the node's `prio`
// priority slots in occ (priority_gap_clear).
template <bool TURNS, class F>
__device__ __forceinline__ uint32_t resolve_prefetched(const uint4 (&pre)[kSlotPrefetch],
                                                       const uint4 *__restrict__ slots, uint32_t slot_lo,
                                                       uint32_t cnt, uint32_t m, uint32_t lanes, uint32_t free_mask,
                                                       const uint8_t *__restrict__ slot_gap,
                                                       const uint2 *__restrict__ slot_tail,
                                                       const uint32_t *__restrict__ occ, uint32_t prio, F &&place) {
    auto visit = [&](const uint4 &x, uint32_t si) {
        if (x.x == kSlotEmpty || x.y != m || !free_mask) return;
        if constexpr (TURNS) {
            if (slot_gap) {
                const uint32_t G = slot_gap[si];
                if (G && !priority_gap_clear(slot_tail, occ, slot_lo, prio, G)) return;
            }
        }
        const uint32_t ks = (x.w >> 8) & 3u;
        const uint32_t pref = ks < lanes - 1u ? ks : lanes - 1u;
        uint32_t qn;
        if ((free_mask >> pref) & 1u) {
            qn = pref;
        } else {
            const uint32_t rest = free_mask & ~(1u << pref);
            if (!rest) return;
            qn = (uint32_t)(__ffs(rest) - 1);
        }
        free_mask &= ~(1u << qn);
        place(si, x, qn);
    };
#pragma unroll
    for (int s = 0; s < kSlotPrefetch; ++s) visit(pre[s], slot_lo + (uint32_t)s);
    for (uint32_t s = kSlotPrefetch; s < cnt && free_mask; ++s) visit(slots[slot_lo + s], slot_lo + s);
    return free_mask;
}

// The same for link m with nd = nd_info[m] (first slot of its upstream node,
// word of its column 0, slot count | lanes << 8 | priority slots << 16).
template <bool TURNS, class F>
__device__ __forceinline__ uint32_t resolve_transfers(const uint4 *__restrict__ slots, const uint4 &nd, uint32_t m,
                                                      uint32_t free_mask, const ScenDev &D,
                                                      const uint32_t *__restrict__ occ, F &&place) {
    // the gap tables are read once, before any placement's stores
    const uint8_t *slot_gap = TURNS ? D.slot_gap : nullptr;
    const uint2 *slot_tail = TURNS ? D.slot_tail : nullptr;
    uint4 pre[kSlotPrefetch];
    prefetch_slots(slots, nd.x, nd.z & 0xFFu, pre);
    return resolve_prefetched<TURNS>(pre, slots, nd.x, nd.z & 0xFFu, m, (nd.z >> 8) & 0xFFu, free_mask, slot_gap,
                                     slot_tail, occ, (nd.z >> 16) & 0xFFu, place);
}

// Departures from parking onto link m after the transfers: the head of m's
// queue enters the lowest free lane with v = 0 while lanes are free and its
// departure step has come.  The head's departure step is kept beside the
// head index, so a link with nothing due costs one load.  Calls
// insert(queue entry, lane, queue index).  hd = dep_head[m], loaded by the
// caller.
template <class F>
__device__ __forceinline__ void run_departures_from(const ScenDev &D, const uint4 &nd, uint32_t m, uint32_t t,
                                                    const uint2 hd, uint32_t free_mask, F &&insert) {
    if (hd.y > t || !free_mask) return;  // y = ~0 once the queue is empty
    const uint32_t dep_end = nd.w;
    uint32_t h = hd.x, next;
    do {
        const uint32_t qn = (uint32_t)(__ffs(free_mask) - 1);
        free_mask &= ~(1u << qn);
        const uint32_t idw = D.dep_ids[h];
        const uint32_t qi = h;
        ++h;
        next = h < dep_end ? D.dep_steps[h] : 0xFFFFFFFFu;
        insert(idw, qn, qi);
    } while (next <= t && free_mask);
    D.dep_head[m] = make_uint2(h, next);
}

template <class F>
__device__ __forceinline__ void run_departures(const ScenDev &D, const uint4 &nd, uint32_t m, uint32_t t,
                                               uint32_t free_mask, F &&insert) {
    run_departures_from(D, nd, m, t, D.dep_head[m], free_mask, insert);
}

// ------------------------------------------------------------------ link kernel
//
// A warp advances one warp tile at a time: up to 30 consecutive columns of
// one scenario in col_info order (link-major, then column j).  Every lane
// owns one slot of the warp's shared-memory rows: lanes 1..n the tile's
// columns, lane 0 the column left of the first one (left halo) and lane
// n + 1 the column right of the last one (right halo), the halos present
// only where such a neighbour exists outside the tile.  A lane handles all
// lanes of its column.  The phases of a tile are separated by __syncwarp,
// never by a block barrier, so every warp runs its own chain of dependent
// loads.  The host builds the tiles so that a ring of at most 30 columns
// lies inside one tile (longer rings get tiles of their own), and so that a
// link's last column is never separated from the column before it when it
// holds at most 2*vmax cells: the cells of a halo that the tile looks at
// are then never within vmax cells of a link end, and the vehicle that
// enters a link-end buffer is handled by the warp that owns the buffer.

constexpr int kSlots = 32;  // slot = lane
constexpr int kRowWords = kMaxLanes * kSlots;
constexpr int kCodes = 256;  // listed vehicles per round of a warp
constexpr uint32_t kNoSlot = 0xFFFFFFFFu;

// How much of a warp's next tile is copied in while it works on the current
// one: 0 nothing, 1 its descriptor and column records, 2 also its columns'
// words of step t.
constexpr int kPrefetch = 0;

struct WarpSmem {
    uint4 pf_ci[kPrefetch >= 1 ? kSlots : 1], pf_ca[kPrefetch >= 1 ? kSlots : 1];
    uint32_t pf_o[kPrefetch >= 2 ? kRowWords : 1], pf_m[kPrefetch >= 2 ? kRowWords : 1],
        pf_l[kPrefetch >= 2 ? kRowWords : 1];
    uint2 pf_td;
    uint32_t o0[kRowWords];  // occupancy of step t (cell 0 placements of fused transfers or-ed in)
    uint32_t m0[kRowWords];  // v > 0 at step t
    uint32_t l0[kRowWords];  // which payload buffer holds each vehicle at step t
    uint32_t mv[kRowWords];  // vehicles that changed INTO the word's lane
    uint32_t o1[kRowWords];  // occupancy after the lane-change sub-step
    uint32_t no[kRowWords];  // step t+1 (tile columns only)
    uint32_t nm[kRowWords];
    uint32_t nl[kRowWords];
    uint32_t cw[kSlots];     // word of lane 0 of the slot's column, kNoSlot if the slot is empty
    uint32_t cx0[kSlots];    // first cell of the column within its link
    uint32_t ccells[kSlots];
    uint32_t clink[kSlots];
    uint32_t cnear[kSlots];  // cells within vmax of the link end (non-periodic links)
    uint32_t cbpos[kSlots];  // first link-end buffer of the link
    int8_t cleft[kSlots], cright[kSlots];  // neighbour slots, -1: none
    uint8_t clanes[kSlots], cring[kSlots], ckind[kSlots];  // ckind: 0 tile column, 1 left halo, 2 right halo
    uint8_t cexit[kSlots];   // lanes whose link-end buffer is free in this step (near columns)
    uint8_t cgreen[kSlots];  // the light at the link end is green in this step (1 without a signal)
    uint16_t code[kCodes];
};

template <int NW>
struct LinkSmem {
    WarpSmem w[NW];
    unsigned long long red[NW][8];
    unsigned long long *rec[NW];
    unsigned long long red2[NW][7];
    unsigned long long *rec2[NW];
};

__device__ __forceinline__ int wi(int k, int s) { return k * kSlots + s; }

// Asynchronous global-to-shared copies (no registers involved); a lane's
// copies are complete after cp_async_wait_all, other lanes' after that and
// a __syncwarp.
__device__ __forceinline__ void cp_async(void *smem, const void *gmem, int bytes) {
    const uint32_t s = (uint32_t)__cvta_generic_to_shared(smem);
    if (bytes == 16) asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem) : "memory");
    else if (bytes == 8) asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(s), "l"(gmem) : "memory");
    else asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// The column of slot `lane` in a tile of n columns from its record ci (the
// halo lanes pass the record of the column next to theirs): word of lane 0,
// column j, neighbour slots, and whether the slot holds a column at all.
struct ColGeo {
    uint32_t cw, j;
    int left, right;
    bool exists;
};
__device__ __forceinline__ ColGeo col_geometry(const uint4 &ci, int lane, int n) {
    const bool core = lane >= 1 && lane <= n, lh = lane == 0, rh = lane == n + 1;
    const uint32_t lanes = (ci.z >> 20) & 7u, ring = (ci.z >> 23) & 1u, ncl = (ci.w + 31u) >> 5;
    ColGeo g{ci.x, ci.z & 0xFFFFFu, -1, -1, core};
    if (core) {
        if (g.j > 0u) g.left = lane - 1;  // lane - 1 = 0: the left halo
        else if (ring) g.left = lane + (int)ncl - 1 <= n ? lane + (int)ncl - 1 : 0;
        if (g.j + 1u < ncl) g.right = lane + 1;  // lane + 1 = n + 1: the right halo
        else if (ring) g.right = lane - (int)g.j >= 1 ? lane - (int)g.j : n + 1;
    } else if (lh) {
        // left of the first column: its column j - 1, or the ring's last
        // column when the ring does not fit the tile
        if (g.j > 0u) {
            g.exists = true;
            g.j -= 1u;
            g.cw -= lanes;
        } else if (ring && ncl > (uint32_t)n) {
            g.exists = true;
            g.j = ncl - 1u;
            g.cw += (ncl - 1u) * lanes;
        }
        g.right = 1;
    } else if (rh) {
        if (g.j + 1u < ncl) {
            g.exists = true;
            g.j += 1u;
            g.cw += lanes;
        } else if (ring && g.j + 1u > (uint32_t)n) {
            g.exists = true;
            g.cw -= g.j * lanes;
            g.j = 0u;
        }
        g.left = n;
    }
    return g;
}

__device__ __forceinline__ uint32_t gap_ahead(const uint32_t *O, const WarpSmem &S, int s, int k, int i,
                                              uint32_t dist, uint32_t open, uint32_t vmax) {
    const uint32_t w0 = O[wi(k, s)];
    const int r = S.cright[s];
    const uint32_t w1 = r >= 0 ? O[wi(k, r)] : 0u;
    const unsigned long long win = (((unsigned long long)w1 << 32) | w0) >> (i + 1);
    uint32_t g = win ? (uint32_t)(__ffsll((long long)win) - 1) : 64u;
    if (g > dist) g = dist + open;
    return g < vmax ? g : vmax;
}

__device__ __forceinline__ bool room_behind(const uint32_t *O, const WarpSmem &S, int s, int k, int i,
                                            uint32_t back) {
    const int l = S.cleft[s];
    const unsigned long long w = ((unsigned long long)O[wi(k, s)] << 32) | (l >= 0 ? O[wi(k, l)] : 0u);
    const unsigned long long mask = ((2ull << back) - 1ull) << (32 + i - (int)back);
    return (w & mask) == 0ull;
}

// Bit x: cell x+1 of the same lane is occupied (bit 0 of the next column for x = 31).
__device__ __forceinline__ uint32_t ahead_mask(const uint32_t *O, const WarpSmem &S, int s, int k) {
    const int r = S.cright[s];
    return (O[wi(k, s)] >> 1) | ((r >= 0 ? O[wi(k, r)] : 0u) << 31);
}

// Vehicles a tile decides lane changes for: all of its own columns, the last
// vmax cells of the left halo (they can move into the tile) and the first
// vmax cells of the right halo (their changes shape the cells the tile's
// last column looks ahead into).
__device__ __forceinline__ uint32_t lc_mask(uint32_t kind, uint32_t vmax) {
    return kind == 0 ? 0xFFFFFFFFu : (kind == 1 ? ~((1u << (32 - vmax)) - 1u) : ((1u << vmax) - 1u));
}

// Vehicles a tile moves: its own columns and the last vmax cells of the left halo.
__device__ __forceinline__ uint32_t move_mask(uint32_t kind, uint32_t vmax) {
    return kind == 0 ? 0xFFFFFFFFu : (kind == 1 ? ~((1u << (32 - vmax)) - 1u) : 0u);
}

__device__ __forceinline__ uint32_t near_mask(uint32_t ring, uint32_t cells, uint32_t x0, uint32_t vmax) {
    if (ring) return 0u;
    const int thr = (int)cells - 1 - (int)vmax - (int)x0;  // first cell within vmax of the end
    return thr <= 0 ? 0xFFFFFFFFu : (thr >= 32 ? 0u : ~((1u << thr) - 1u));
}

// Runs `proc(code)` for every set bit of the lanes' word masks m[k] (word
// (k, slot) of the lane's own slot), the warp's lanes sharing the work:
// rounds of at most kCodes listed vehicles go through the warp's code list.
template <class F>
__device__ __forceinline__ void warp_list(WarpSmem &S, uint32_t (&m)[kMaxLanes], int slot, F &&proc) {
    const int lane = threadIdx.x & 31;
    for (;;) {
        uint32_t cnt = 0u;
#pragma unroll
        for (int q = 0; q < kMaxLanes; ++q) cnt += (uint32_t)__popc(m[q]);
        uint32_t inc = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += y;
        }
        const uint32_t total = __shfl_sync(0xffffffffu, inc, 31);
        if (total == 0u) break;
        uint32_t pos = inc - cnt;
#pragma unroll
        for (int q = 0; q < kMaxLanes; ++q) {
            while (m[q] && pos < (uint32_t)kCodes) {
                const int b = __ffs(m[q]) - 1;
                m[q] &= m[q] - 1u;
                S.code[pos++] = (uint16_t)((wi(q, slot) << 5) | b);
            }
        }
        __syncwarp();
        const uint32_t nproc = total < (uint32_t)kCodes ? total : (uint32_t)kCodes;
        for (uint32_t e = (uint32_t)lane; e < nproc; e += 32u) proc((uint32_t)S.code[e]);
        __syncwarp();
    }
}

// The same with each vehicle's step split in two: addr(code, pa, pb) gives
// the global 32-bit words its step needs (its step-t payload, which no
// thread writes during the step; nullptr: not needed) and proc(code, wa, wb)
// completes it from their values.  (Measured on the 200,000-link network:
// loading two vehicles' payload into registers before processing either,
// 55.6 vs 47.4 us per launch; copying all of a lane's payload words of a
// round into shared memory first, 47.2-48.5 vs 46.4 us.)
template <class A, class F>
__device__ __forceinline__ void warp_list2(WarpSmem &S, uint32_t (&m)[kMaxLanes], int slot, A &&addr, F &&proc) {
    const int lane = threadIdx.x & 31;
    for (;;) {
        uint32_t cnt = 0u;
#pragma unroll
        for (int q = 0; q < kMaxLanes; ++q) cnt += (uint32_t)__popc(m[q]);
        uint32_t inc = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += y;
        }
        const uint32_t total = __shfl_sync(0xffffffffu, inc, 31);
        if (total == 0u) break;
        uint32_t pos = inc - cnt;
#pragma unroll
        for (int q = 0; q < kMaxLanes; ++q) {
            while (m[q] && pos < (uint32_t)kCodes) {
                const int b = __ffs(m[q]) - 1;
                m[q] &= m[q] - 1u;
                S.code[pos++] = (uint16_t)((wi(q, slot) << 5) | b);
            }
        }
        __syncwarp();
        const uint32_t nproc = total < (uint32_t)kCodes ? total : (uint32_t)kCodes;
        for (uint32_t e = (uint32_t)lane; e < nproc; e += 32u) {
            const uint32_t c = S.code[e];
            const uint32_t *pa = nullptr, *pb = nullptr;
            addr(c, pa, pb);
            proc(c, pa ? *pa : 0u, pb ? *pb : 0u);
        }
        __syncwarp();
    }
}

// The aligned 32-bit word holding byte p of an int8 array (whose length is
// a multiple of 4), and the byte's value from that word.
__device__ __forceinline__ const uint32_t *byte_word(const int8_t *a, size_t p) {
    return reinterpret_cast<const uint32_t *>(a + (p & ~(size_t)3));
}
__device__ __forceinline__ uint32_t word_byte(uint32_t w, uint32_t p) { return (w >> (8u * (p & 3u))) & 0xFFu; }

// Sum over the warp, then lane f adds field f's sum at rec + field[f].
template <int NF>
__device__ __forceinline__ void warp_flush(unsigned long long (&acc)[NF], unsigned long long *rec,
                                           const int (&field)[NF]) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int f = 0; f < NF; ++f) {
        unsigned long long v = acc[f];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == f && v) atomicAdd(rec + field[f], v);
        acc[f] = 0ull;
    }
}

// At the end of the launch: the warps' sums of one record go out with one
// atomic per field per block; a warp whose record differs from warp 0's
// adds its own.
template <int NW, int NF>
__device__ __forceinline__ void block_end_flush(unsigned long long (&acc)[NF], unsigned long long *rec,
                                                unsigned long long (*red)[NF], unsigned long long **recs,
                                                const int (&field)[NF]) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int f = 0; f < NF; ++f) {
        unsigned long long v = acc[f];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) red[warp][f] = v;
        acc[f] = 0ull;
    }
    if (lane == 0) recs[warp] = rec;
    __syncthreads();
    if (threadIdx.x < NF) {
        const int f = threadIdx.x;
        unsigned long long s = 0ull;
        unsigned long long *r0 = recs[0];
        for (int w = 0; w < NW; ++w) {
            if (recs[w] == nullptr) continue;
            if (r0 == nullptr) r0 = recs[w];
            if (recs[w] == r0) s += red[w][f];
            else if (red[w][f]) atomicAdd(recs[w] + field[f], red[w][f]);
        }
        if (r0 && s) atomicAdd(r0 + field[f], s);
    }
}

// Node transfers and departures into link l (whose column 0 this lane owns)
// at the end of step t-1, for fused steps.  Returns the lanes of l whose
// cell 0 received a vehicle (moving: with v > 0); acc2 gets the counts of
// the previous step's record (transfers, insertions, changes of active,
// buffered, sum of v, digest, moving).
template <bool TURNS>
__device__ __forceinline__ uint32_t xfer_into_link(const ScenDev &D, uint32_t t, const uint4 *__restrict__ sc,
                                                   const uint32_t *__restrict__ oc, uint32_t l, uint32_t &moving,
                                                   unsigned long long (&acc2)[7]) {
    const uint4 nd = D.nd_info[l];
    uint32_t placed = 0u;
    moving = 0u;
    int8_t *vel = D.vel[0];    // cell 0 was empty: its payload goes
    uint32_t *vid = D.vid[0];  // to buffer 0 (location bit 0)
    uint32_t fr = resolve_transfers<TURNS>(sc, nd, l, free_cell0(oc, nd), D, oc, [&](uint32_t, const uint4 &x,
                                                                                    uint32_t qn) {
        const uint32_t id = x.x & kIdMask, v = x.w & (TURNS ? 0xFu : 0xFFu), ks = (x.w >> 8) & 3u;
        placed |= 1u << qn;
        if (v) moving |= 1u << qn;
        const size_t pc = (size_t)(nd.y + qn) * 32u;
        vel[pc] = (int8_t)(TURNS ? (x.w & 0xFFu) : v);
        vid[pc] = x.x;  // id with the last-link flag of l
        atomicAdd(&D.veh[id].x, 1u);
        atomicAdd(&D.link_time[x.z], kLinkTimeOne + (t - 1u));
        atomicAdd(&D.link_time[l], 0ull - (unsigned long long)(t - 1u));
        D.enter_step[id] = t - 1u;
        acc2[0] += 1;
        acc2[2] += 1;
        acc2[3] -= 1;
        acc2[4] += v;
        acc2[5] += vehicle_term(id, l, qn, 0u, v) - vehicle_term(id, x.z, ks, x.w >> 10, v);
        acc2[6] += v ? 1u : 0u;
    });
    run_departures(D, nd, l, t - 1u, fr, [&](uint32_t idw, uint32_t qn, uint32_t qi) {
        placed |= 1u << qn;
        const size_t pc = (size_t)(nd.y + qn) * 32u;
        vel[pc] = (TURNS && D.dep_turn) ? (int8_t)(D.dep_turn[qi] << 4) : (int8_t)0;
        vid[pc] = idw;
        atomicAdd(&D.link_time[l], 0ull - (unsigned long long)(t - 1u));
        D.enter_step[idw & kIdMask] = t - 1u;
        acc2[1] += 1;
        acc2[2] += 1;
        acc2[5] += vehicle_term(idw & kIdMask, l, qn, 0u, 0u);
    });
    return placed;
}

// Whether the buffer idx holding x is emptied by the node transfer of step
// t-1 (the same resolution as the warp owning x's next link computes).
template <bool TURNS>
__device__ __forceinline__ bool buffer_emptied(const ScenDev &D, const uint4 *__restrict__ sc,
                                               const uint32_t *__restrict__ oc, const uint4 &x, uint32_t idx) {
    bool empty = false;
    const uint4 nd = D.nd_info[x.y];
    resolve_transfers<TURNS>(sc, nd, x.y, free_cell0(oc, nd), D, oc,
                             [&](uint32_t si, const uint4 &, uint32_t) { empty |= si == idx; });
    return empty;
}

// The fused-step work of one lane, out of line so that its registers stay
// out of the step: with first, the transfers and departures into the lane's
// link (column 0) ending step t-1; with end, the link's lane-end buffers for
// step t (empty, emptied by a transfer of step t-1, or still holding their
// vehicle) copied into the next set.  Returns the free buffers (end) and
// writes the cell-0 placements.
template <bool TURNS>
__device__ __noinline__ uint32_t fused_link_work(const ScenDev &D, uint32_t t, int cur, uint32_t link,
                                                 uint32_t bpos, uint32_t lanes, bool first, bool end,
                                                 uint32_t &placed, uint32_t &moving,
                                                 unsigned long long (&acc2)[7]) {
    const uint4 *__restrict__ sc = D.slots[cur];
    uint4 *__restrict__ sn = D.slots[cur ^ 1];
    const uint32_t *__restrict__ oc = D.occ[cur];
    placed = 0u;
    moving = 0u;
    if (first) placed = xfer_into_link<TURNS>(D, t, sc, oc, link, moving, acc2);
    uint32_t open = 0u;
    if (end) {
        for (uint32_t k = 0; k < lanes; ++k) {
            const uint4 x = sc[bpos + k];
            const bool empty = x.x == kSlotEmpty || buffer_emptied<TURNS>(D, sc, oc, x, bpos + k);
            if (empty) open |= 1u << k;
            sn[bpos + k] = empty ? make_uint4(kSlotEmpty, kSlotEmpty, kSlotEmpty, kSlotEmpty) : x;
        }
    }
    return open;
}

// One launch of the link kernel (body of link_kernel and turn_link_kernel)
// for NW warps per block.  XFER (fused steps): the launch first completes the
// node transfers and departures of the previous step, the tiles of a link's
// first and last columns resolving them.  TURNS: the intersection rules of Sec. 3 a network
// may carry: plan-following lane changes (every velocity byte carries the
// lanes A of its link from which the vehicle may take its next turn) and gap
// acceptance at unprotected turns (in the node transfers).  VM: 0, or the
// vmax every scenario of the launch has, as a compile-time constant (the
// masks, gap windows and loops over the vmax cells behind or ahead of a
// vehicle then fold into fixed bit operations).
template <int NW, bool TURNS, bool XFER, int VM>
__device__ __forceinline__ void link_step(LinkSmem<NW> &SB, const ScenDev *__restrict__ table,
                                          const uint2 *__restrict__ tiles, const uint32_t *__restrict__ n_tiles_p,
                                          uint32_t pos, unsigned long long *span, uint32_t *tile_ctr) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    WarpSmem &S = SB.w[warp];
    const uint32_t n_tiles = *n_tiles_p;  // changes only between graph launches
    // statistics: updates, lane changes, arrivals, the changes of active,
    // buffered, sum of velocities and digest, and the moving vehicles
    static constexpr int kField[8] = {kUpdates, kLaneChanges, kArrived, kDActive, kDBuffered, kDSumV, kDHash,
                                      kMoving};
    static constexpr int kField2[7] = {kTransfers, kInserted, kDActive, kDBuffered, kDSumV, kDHash, kMoving};
    uint32_t acc[7] = {0u, 0u, 0u, 0u, 0u, 0u, 0u};  // counts (per warp and step far below 2^31), signed changes
    unsigned long long acc_hash = 0ull;
    unsigned long long acc2[7] = {0ull, 0ull, 0ull, 0ull, 0ull, 0ull, 0ull};
    unsigned long long *cur_rec = nullptr, *cur_rec2 = nullptr;
    auto widen = [&](unsigned long long (&v)[8]) {
        v[0] = acc[0];
        v[1] = acc[1];
        v[2] = acc[2];
        v[3] = (unsigned long long)(long long)(int)acc[3];
        v[4] = (unsigned long long)(long long)(int)acc[4];
        v[5] = (unsigned long long)(long long)(int)acc[5];
        v[6] = acc_hash;
        v[7] = acc[6];
#pragma unroll
        for (int f = 0; f < 7; ++f) acc[f] = 0u;
        acc_hash = 0ull;
    };
    bool waited = false;
    const uint32_t nwarps = gridDim.x * (uint32_t)NW;
    const int s = lane;  // this lane's slot
    // what the prefetch area holds for the tile about to start: its
    // descriptor, its column records, its columns' words of step t
    bool pf_td = false, pf_geo = false, pf_state = false;
    // a warp's first two tiles are given by its index (warp, warp + nwarps);
    // after them, with a claim counter for this chunk position and more than
    // two tiles per warp, it takes the next unclaimed tile (claimed while its
    // second or later tile runs, when the warps no longer start together, so
    // warps whose tiles ran short take more), else every nwarps-th
    uint32_t *const ctr = tile_ctr != nullptr && n_tiles > 2u * nwarps ? tile_ctr + pos : nullptr;
    uint32_t claim = 0u;
    for (uint32_t tile = blockIdx.x * (uint32_t)NW + (uint32_t)warp; tile < n_tiles;
         tile = ctr != nullptr && tile >= nwarps ? 2u * nwarps + __shfl_sync(0xffffffffu, claim, 0) : tile + nwarps) {
        if (ctr != nullptr && tile >= nwarps && lane == 0) claim = atomicAdd(ctr, 1u);
        // the next kernel may launch once every block has begun its last
        // round of tiles (warp 0 has the most tiles of its block): launched
        // earlier, its waiting blocks would hold registers and shared memory
        // this launch still needs
        if (warp == 0 && tile + nwarps >= n_tiles) pdl_trigger();
        if (pf_td) {
            cp_async_wait_all();
            __syncwarp();
        }
        const uint2 td = pf_td ? S.pf_td : tiles[tile];
        const bool geo_ready = pf_geo, state_ready = pf_state;
        pf_td = pf_geo = pf_state = false;
        const ScenDev &D = table[td.x & 0xFFFFFFu];
        if (D.ctrl == nullptr) continue;
        if (VM != 0 && D.vmax != (uint32_t)VM) {
            if (lane == 0) atomicOr(&D.ctrl->error, kErrInstance);
            continue;
        }
        const int n = (int)(td.x >> 24) + 1;
        const uint32_t cb = td.y;
        const uint32_t vmax = VM != 0 ? (uint32_t)VM : D.vmax;

        // ---------------- geometry (static data: read before waiting).  The
        // halo lanes read the column next to theirs and step to their own.
        const bool core = lane >= 1 && lane <= n, lh = lane == 0, rh = lane == n + 1;
        uint4 ci = make_uint4(0u, 0u, 0u, 0u), ca = make_uint4(0u, 0u, 0u, 0u);
        if (core || lh || rh)
            ci = geo_ready ? S.pf_ci[lane]
                           : D.col_info[core ? cb + (uint32_t)lane - 1u : (lh ? cb : cb + (uint32_t)n - 1u)];
        if (core) ca = geo_ready ? S.pf_ca[lane] : D.col_aux[cb + (uint32_t)lane - 1u];
        const ColGeo geo = col_geometry(ci, lane, n);
        const uint32_t cw = geo.cw, j = geo.j;
        const int left = geo.left, right = geo.right;
        const bool exists = geo.exists;
        const uint32_t link = ci.y, lanes = (ci.z >> 20) & 7u, ring = (ci.z >> 23) & 1u, cells = ci.w;
        const uint32_t ncl = (cells + 31u) >> 5;
        const uint32_t kind = core ? 0u : (lh ? 1u : 2u);
        const uint32_t near = exists ? near_mask(ring, cells, 32u * j, vmax) : 0u;
        // the link's last cell, when it lies in this column
        const uint32_t endb = (exists && !ring && cells - 1u - 32u * j < 32u) ? 1u << (cells - 1u - 32u * j) : 0u;
        const bool first = core && !ring && j == 0u, end = core && !ring && j + 1u == ncl;
        const uint32_t bpos = ca.x;
        S.cw[s] = exists ? cw : kNoSlot;
        S.cx0[s] = 32u * j;
        S.ccells[s] = cells;
        S.clink[s] = link;
        S.cnear[s] = near;
        S.cbpos[s] = bpos;
        S.cleft[s] = (int8_t)left;
        S.cright[s] = (int8_t)right;
        S.clanes[s] = (uint8_t)(exists ? lanes : 0u);
        S.cring[s] = (uint8_t)ring;
        S.ckind[s] = (uint8_t)kind;
        S.cexit[s] = 0;
        S.cgreen[s] = 1;
        // The step base and target change only between captured chunks (the
        // chunk-closing kernel has finished before a chunk's first launch), so
        // they may be read before waiting for the previous kernel.
        const unsigned long long step = D.ctrl->base + pos;
        const bool active = step < D.ctrl->target;
        __syncwarp();
        if (!active) continue;
        if (!waited) {
            pdl_wait();
            waited = true;
            if (warp == 0) span_mark(span, pos, 0, true);  // the predecessor has completed: the work starts
        }
        unsigned long long *rec = reinterpret_cast<unsigned long long *>(stat_rec(D, step));
        if (rec != cur_rec) {
            if (cur_rec) {
                unsigned long long v[8];
                widen(v);
                warp_flush<8>(v, cur_rec, kField);
            }
            cur_rec = rec;
        }
        constexpr bool do_xfer = XFER;
        if constexpr (do_xfer) {
            unsigned long long *rec2 = reinterpret_cast<unsigned long long *>(stat_rec(D, step - 1ull));
            if (rec2 != cur_rec2) {
                if (cur_rec2) warp_flush<7>(acc2, cur_rec2, kField2);
                cur_rec2 = rec2;
            }
        }
        const uint32_t t = (uint32_t)step;
        const int cur = (int)(step & 1ull), nxt = cur ^ 1;
        const int d = (t & 1u) ? -1 : 1;
        // prefetch, stage 1: the next tile's descriptor
        const uint32_t tile_n = tile + nwarps;
        if (kPrefetch >= 1 && tile_n < n_tiles) {
            if (lane == 0) cp_async(&S.pf_td, &tiles[tile_n], 8);
            pf_td = true;
        }

        // ---------------- state of step t: every load before any store
        uint32_t o[kMaxLanes], mo[kMaxLanes], lo[kMaxLanes];
#pragma unroll
        for (int k = 0; k < kMaxLanes; ++k) {
            const bool w = exists && (uint32_t)k < lanes;
            const bool pre = kPrefetch >= 2 && state_ready;
            o[k] = w ? (pre ? S.pf_o[wi(k, s)] : D.occ[cur][cw + (uint32_t)k]) : 0u;
            mo[k] = w ? (pre ? S.pf_m[wi(k, s)] : D.mov[cur][cw + (uint32_t)k]) : 0u;
            lo[k] = w ? (pre ? S.pf_l[wi(k, s)] : D.loc[cur][cw + (uint32_t)k]) : 0u;
        }
        uint4 own[kMaxLanes];
        const bool plain_end = end && !do_xfer;
#pragma unroll
        for (int k = 0; k < kMaxLanes; ++k)
            own[k] = plain_end && (uint32_t)k < lanes ? D.slots[cur][bpos + (uint32_t)k]
                                                      : make_uint4(kSlotEmpty, 0u, 0u, 0u);
        uint32_t placed = 0u, moving = 0u, open = 0u;
        bool fused_done = false;
        if constexpr (XFER) {
            if (first || end) {
                open = fused_link_work<TURNS>(D, t, cur, link, bpos, lanes, first, end, placed, moving, acc2);
                fused_done = true;
            }
        }
        if (!fused_done && end) {
            // l's lane-end buffers for step t: empty (the node pass of step
            // t-1 has emptied transferred ones) or still holding their vehicle
#pragma unroll
            for (int k = 0; k < kMaxLanes; ++k) {
                if ((uint32_t)k >= lanes) break;
                const bool empty = own[k].x == kSlotEmpty;
                if (empty) open |= 1u << k;
                D.slots[nxt][bpos + (uint32_t)k] =
                    empty ? make_uint4(kSlotEmpty, kSlotEmpty, kSlotEmpty, kSlotEmpty) : own[k];
            }
        }
        uint32_t upd = 0u;
#pragma unroll
        for (int k = 0; k < kMaxLanes; ++k) {
            if (!exists || (uint32_t)k >= lanes) continue;
            const uint32_t ok = o[k] | ((placed >> k) & 1u);
            S.o0[wi(k, s)] = ok;
            S.m0[wi(k, s)] = mo[k] | ((moving >> k) & 1u);
            S.l0[wi(k, s)] = lo[k];
            S.mv[wi(k, s)] = 0u;
            S.no[wi(k, s)] = 0u;
            S.nm[wi(k, s)] = 0u;
            S.nl[wi(k, s)] = 0u;
            upd += (uint32_t)__popc(ok);
        }
        if (core) acc[0] += upd;  // vehicle updates
        if (end) {
            // the light at the link end (Sec. 3): while red, a virtual
            // vehicle of maximum velocity zero stands at every lane end
            const uint32_t cycle = ca.y & 0xFFFFu, green = ca.y >> 16;
            const uint8_t gr = (uint8_t)(cycle == 0u || (t + ca.z) % cycle < green);
            S.cexit[s] = (uint8_t)open;
            S.cgreen[s] = gr;
            if (lane > 1 && j > 0u) {  // the column before it (same link), a column of this tile
                S.cexit[s - 1] = (uint8_t)open;
                S.cgreen[s - 1] = gr;
            }
        }
        // the cells of a halo that the tile looks at are never within vmax
        // cells of a link end; a tile built otherwise is flagged
        if (!core && exists && (near & lc_mask(kind, vmax))) atomicOr(&D.ctrl->error, kErrGeometry);
        const uint32_t kmax = __reduce_max_sync(0xffffffffu, exists ? lanes : 0u);
        __syncwarp();
        if (!__any_sync(0xffffffffu, upd != 0u)) {
            // no vehicle in the tile or its halos: the next state's words are empty
            if (core) {
#pragma unroll
                for (int k = 0; k < kMaxLanes; ++k) {
                    if ((uint32_t)k >= lanes) break;
                    const uint32_t g = cw + (uint32_t)k;
                    D.occ[nxt][g] = 0u;
                    D.mov[nxt][g] = 0u;
                    D.loc[nxt][g] = 0u;
                }
            }
            continue;
        }
        const int8_t *__restrict__ vel0 = D.vel[0];
        const int8_t *__restrict__ vel1 = D.vel[1];
        const uint32_t *__restrict__ vid0 = D.vid[0];
        const uint32_t *__restrict__ vid1 = D.vid[1];

        // ---------------- sub-step 1: lane changes, decided on the state of step t.
        // A vehicle with v = 0 and an occupied cell ahead always has a reason to
        // change (its gap 0 is below min(v+1, vmax) = 1); it changes iff the
        // target cell and the vmax cells behind it are empty and the target
        // lane's next cell is free.  That is decided here for whole words.  A
        // vehicle with v = 0 and a free cell ahead has no reason to change.
        // Both hold within vmax of a link end too: the gaps compared are 0 and
        // whether the next cell of the target lane (inside the link) is free,
        // neither of which looks past the end.  Moving vehicles and a vehicle
        // in a link's last cell (whose gaps do: the end's state, its last-link
        // flag) are decided one by one.
        if (D.lane_change != 0u) {
            uint32_t lst[kMaxLanes] = {0u, 0u, 0u, 0u};
#pragma unroll
            for (int k = 0; k < kMaxLanes; ++k) {
                if ((uint32_t)k >= kmax) break;
                const int kt = k + d;
                if (!exists || (uint32_t)k >= lanes || kt < 0 || kt >= (int)lanes) continue;
                const uint32_t oc = S.o0[wi(k, s)] & lc_mask(kind, vmax);
                if (!oc) continue;
                if (TURNS) {
                    // the allowed lanes are in the payload: every vehicle
                    // whose target cell is free is decided one by one
                    lst[k] = oc & ~S.o0[wi(kt, s)];
                } else {
                    const uint32_t tw = S.o0[wi(kt, s)];
                    const unsigned long long tt =
                        ((unsigned long long)tw << 32) | (left >= 0 ? S.o0[wi(kt, left)] : 0u);
                    uint32_t behind = 0u;
                    for (uint32_t b = 1; b <= vmax; ++b) behind |= (uint32_t)(tt >> (32 - b));
                    const uint32_t okm = ahead_mask(S.o0, S, s, k) & ~tw & ~behind & ~ahead_mask(S.o0, S, s, kt);
                    const uint32_t lcv0 = oc & ~S.m0[wi(k, s)] & ~endb & okm;
                    if (lcv0) {
                        S.mv[wi(kt, s)] |= lcv0;  // this lane's own slot
                        if (core) acc[1] += (uint32_t)__popc(lcv0);
                    }
                    // a vehicle with vmax free cells ahead, more than vmax
                    // cells before the end, has a gap of vmax: no reason
                    const unsigned long long ow =
                        ((unsigned long long)(right >= 0 ? S.o0[wi(k, right)] : 0u) << 32) | S.o0[wi(k, s)];
                    uint32_t busy_ahead = 0u;
                    for (uint32_t b = 1; b <= vmax; ++b) busy_ahead |= (uint32_t)(ow >> b);
                    lst[k] = oc & ((S.m0[wi(k, s)] & (busy_ahead | near)) | endb);
                }
            }
            __syncwarp();
            // payload at step t (velocity byte; the id only within vmax
            // cells of the link end, for its last-link flag)
            auto lcaddr = [&](uint32_t code, const uint32_t *&pv, const uint32_t *&pid) {
                const int ww = (int)(code >> 5), i = (int)(code & 31u);
                const int k = ww / kSlots, c = ww - k * kSlots, kt = k + d;
                if ((S.o0[wi(kt, c)] >> i) & 1u) return;  // target cell taken: not needed
                const size_t p = (size_t)(S.cw[c] + (uint32_t)k) * 32u + (uint32_t)i;
                const bool b1 = (S.l0[ww] >> i) & 1u;
                pv = byte_word(b1 ? vel1 : vel0, p);
                if ((S.cnear[c] >> i) & 1u) pid = (b1 ? vid1 : vid0) + p;
            };
            warp_list2(S, lst, s, lcaddr, [&](uint32_t code, uint32_t vword, uint32_t idw) {
                const int ww = (int)(code >> 5), i = (int)(code & 31u);
                const uint32_t byte = word_byte(vword, (uint32_t)i);
                const int k = ww / kSlots, c = ww - k * kSlots, kt = k + d;
                if ((S.o0[wi(kt, c)] >> i) & 1u) return;  // target cell taken
                const uint32_t ringc = S.cring[c];
                const uint32_t x = S.cx0[c] + (uint32_t)i;
                const uint32_t dist = ringc ? 0xFFFFu : S.ccells[c] - 1u - x;
                uint32_t v;
                uint32_t al = 0xFu;  // lanes it may leave the link from
                if constexpr (TURNS) {
                    v = byte & 0xFu;
                    if (byte >> 4) al = byte >> 4;
                } else {
                    v = byte;
                }
                if constexpr (TURNS) {
                    if (!((al >> k) & 1u)) {
                        // outside its allowed lanes: a reason to change when
                        // one of them lies on the side d points to; the gap
                        // accepted behind the target cell shrinks from vmax to
                        // 0 over the link's last vmax cells
                        const uint32_t side = d > 0 ? al & ~((2u << k) - 1u) : al & ((1u << k) - 1u);
                        if (side && room_behind(S.o0, S, c, kt, i, dist < vmax ? dist : vmax)) {
                            atomicOr(&S.mv[wi(kt, c)], 1u << i);
                            if (S.ckind[c] == 0) acc[1] += 1;
                        }
                        return;
                    }
                    // the speed reason applies only into an allowed lane (and
                    // then both lanes are allowed: the gaps below need no
                    // closed link end)
                    if (!((al >> kt) & 1u)) return;
                }
                const uint32_t last = idw >> 31;  // 0 outside the near cells
                const uint32_t want = v + 1u < vmax ? v + 1u : vmax;
                const uint32_t ex = S.cexit[c], gr = S.cgreen[c];
                const uint32_t g_own = gap_ahead(S.o0, S, c, k, i, dist, (((ex >> k) & 1u) | last) & gr, vmax);
                if (g_own >= want) return;
                const uint32_t g_tgt = gap_ahead(S.o0, S, c, kt, i, dist, (((ex >> kt) & 1u) | last) & gr, vmax);
                if (g_tgt > g_own && room_behind(S.o0, S, c, kt, i, vmax)) {
                    atomicOr(&S.mv[wi(kt, c)], 1u << i);
                    if (S.ckind[c] == 0) acc[1] += 1;
                }
            });
        }
        __syncwarp();
        // prefetch, stage 2: the next tile's column records (when it is a
        // tile of the same scenario: the same step and state buffers)
        if (pf_td) {
            cp_async_wait_all();
            __syncwarp();
            const uint2 tn = S.pf_td;
            if ((tn.x & 0xFFFFFFu) == (td.x & 0xFFFFFFu)) {
                const int nn = (int)(tn.x >> 24) + 1;
                const bool cn = lane >= 1 && lane <= nn, ln = lane == 0, rn = lane == nn + 1;
                if (cn || ln || rn)
                    cp_async(&S.pf_ci[lane],
                             &D.col_info[cn ? tn.y + (uint32_t)lane - 1u : (ln ? tn.y : tn.y + (uint32_t)nn - 1u)], 16);
                if (cn) cp_async(&S.pf_ca[lane], &D.col_aux[tn.y + (uint32_t)lane - 1u], 16);
                pf_geo = true;
            }
        }

        // ---------------- sub-step 2: velocity update and move.  A vehicle with
        // v = 0, an occupied cell ahead and no lane change keeps v = 0 and its
        // cell (its gap is 0 wherever it stands, link end or not): its bits are
        // copied, its payload stays.
        {
            uint32_t lst[kMaxLanes] = {0u, 0u, 0u, 0u};
#pragma unroll
            for (int k = 0; k < kMaxLanes; ++k) {
                if ((uint32_t)k >= kmax) break;
                if (!exists || (uint32_t)k >= lanes) continue;
                // the words after the lane-change sub-step, from the step-t
                // words and the lane-change marks (mv: vehicles that changed
                // into a word's lane; those leaving lane k went to k + d)
                const int kf = k + d, kb = k - d;
                const bool has_f = kf >= 0 && kf < (int)lanes, has_b = kb >= 0 && kb < (int)lanes;
                const uint32_t arriving = S.mv[wi(k, s)];
                const uint32_t leaving = has_f ? S.mv[wi(kf, s)] : 0u;
                const uint32_t o1 = (S.o0[wi(k, s)] & ~leaving) | arriving;
                const uint32_t src_mov = (arriving && has_b) ? S.m0[wi(kb, s)] : 0u;
                const uint32_t m1 = (S.m0[wi(k, s)] & ~leaving) | (src_mov & arriving);
                S.o1[wi(k, s)] = o1;
                const uint32_t o1r =
                    right >= 0 ? (S.o0[wi(k, right)] & ~(has_f ? S.mv[wi(kf, right)] : 0u)) | S.mv[wi(k, right)] : 0u;
                const uint32_t free_ahead = ~((o1 >> 1) | (o1r << 31));
                const uint32_t busy = m1 | free_ahead | arriving;
                lst[k] = o1 & busy & move_mask(kind, vmax);
                if (core) {
                    const uint32_t inert = o1 & ~busy;
                    S.no[wi(k, s)] = inert;
                    S.nl[wi(k, s)] = inert & S.l0[wi(k, s)];
                }
            }
            __syncwarp();
            // prefetch, stage 3: the next tile's words of step t (read-only
            // during the step)
            if (kPrefetch >= 2 && pf_geo) {
                cp_async_wait_all();
                __syncwarp();
                const int nn = (int)(S.pf_td.x >> 24) + 1;
                if (lane <= nn + 1) {
                    const uint4 cin = S.pf_ci[lane];
                    const ColGeo gn = col_geometry(cin, lane, nn);
                    const uint32_t ln = (cin.z >> 20) & 7u;
                    if (gn.exists)
                        for (uint32_t k = 0; k < ln; ++k) {
                            cp_async(&S.pf_o[wi((int)k, lane)], &D.occ[cur][gn.cw + k], 4);
                            cp_async(&S.pf_m[wi((int)k, lane)], &D.mov[cur][gn.cw + k], 4);
                            cp_async(&S.pf_l[wi((int)k, lane)], &D.loc[cur][gn.cw + k], 4);
                        }
                }
                pf_state = true;
            }
            int8_t *__restrict__ velw0 = D.vel[0];
            int8_t *__restrict__ velw1 = D.vel[1];
            uint32_t *__restrict__ vidw0 = D.vid[0];
            uint32_t *__restrict__ vidw1 = D.vid[1];
            const uint32_t key0 = D.seed_lo, key1 = D.seed_hi, pthr = D.p_threshold;
            // payload from where the vehicle was at step t; no thread of
            // this step writes a buffer that a step-t occupant is read from
            auto vaddr = [&](uint32_t code, const uint32_t *&pid, const uint32_t *&pv) {
                const int ww = (int)(code >> 5), i = (int)(code & 31u);
                const int k = ww / kSlots, c = ww - k * kSlots;
                const int ks = ((S.mv[ww] >> i) & 1u) ? k - d : k;  // lane at step t
                const size_t ps = (size_t)(S.cw[c] + (uint32_t)ks) * 32u + (uint32_t)i;
                const bool sb1 = (S.l0[wi(ks, c)] >> i) & 1u;
                pid = (sb1 ? vid1 : vid0) + ps;
                pv = byte_word(sb1 ? vel1 : vel0, ps);
            };
            warp_list2(S, lst, s, vaddr, [&](uint32_t code, uint32_t idw, uint32_t vword) {
                const int ww = (int)(code >> 5), i = (int)(code & 31u);
                const uint32_t byte = word_byte(vword, (uint32_t)i);
                const int k = ww / kSlots, c = ww - k * kSlots;
                const int ks = ((S.mv[ww] >> i) & 1u) ? k - d : k;  // lane at step t
                uint32_t v0, al = 0u;  // al: allowed lanes of the next turn (0: any)
                if constexpr (TURNS) {
                    v0 = byte & 0xFu;
                    al = byte >> 4;
                } else {
                    v0 = byte;
                }
                const uint32_t id = idw & kIdMask, last = idw >> 31;
                const uint32_t ringc = S.cring[c];
                const uint32_t x = S.cx0[c] + (uint32_t)i;
                const uint32_t cellsc = S.ccells[c];
                const uint32_t dist = ringc ? 0xFFFFu : cellsc - 1u - x;
                uint32_t v = v0 + 1u < vmax ? v0 + 1u : vmax;  // (i) accelerate
                uint32_t open = (((S.cexit[c] >> k) & 1u) | last) & S.cgreen[c];
                if constexpr (TURNS) {
                    if (al && !((al >> k) & 1u)) open = 0u;  // the next turn is not taken from lane k
                }
                const uint32_t g = gap_ahead(S.o1, S, c, k, i, dist, open, vmax);
                if (v > g) v = g;                                                 // (ii) gap
                if (v > 0u && philox_word0(t, id, key0, key1) < pthr) v -= 1u;  // (iii) random
                const bool core = S.ckind[c] == 0;
                const uint32_t lid = S.clink[c];
                // the tile whose column held the vehicle at step t accounts for it
                const unsigned long long old_term = core ? vehicle_term(id, lid, (uint32_t)ks, x, v0) : 0ull;
                if (!ringc && x + v >= cellsc) {
                    // reaches the link end: only from a near column, which is
                    // always a column of this tile
                    if (!core) {
                        atomicOr(&D.ctrl->error, kErrGeometry);
                    } else if (last) {
                        acc[2] += 1;  // leaves to parking
                        acc[3] -= 1;
                        // travel time: + the exit step here, - the entry step at entry
                        atomicAdd(&D.link_time[lid], kLinkTimeOne + t);
                        D.enter_step[id] = kNotOnLink;
                        acc[5] -= v0;
                        acc_hash -= old_term;
                    } else {
                        const uint2 ve = D.veh[id];
                        if (ve.x + 1u >= ve.y) {
                            atomicOr(&D.ctrl->error, kErrRoute);
                        } else {
                            const uint32_t m = D.route_links[ve.x + 1u];
                            const uint32_t fl = (ve.x + 2u == ve.y) ? kLastLinkBit : 0u;
                            if (!((S.cexit[c] >> k) & 1u)) atomicOr(&D.ctrl->error, kErrSlotTaken);
                            uint32_t vb = v;  // with the allowed lanes of the turn after m
                            if constexpr (TURNS) {
                                if (D.route_turn) vb |= (uint32_t)D.route_turn[ve.x + 1u] << 4;
                            }
                            D.slots[nxt][S.cbpos[c] + (uint32_t)k] =
                                make_uint4(id | fl, m, lid, vb | ((uint32_t)k << 8) | (cellsc << 10));
                            acc[3] -= 1;
                            acc[4] += 1;
                            acc[5] -= v0;
                            acc_hash += vehicle_term(id, lid, (uint32_t)k, cellsc, v) - old_term;
                        }
                    }
                } else {
                    int ni = i + (int)v;
                    int dc = c;
                    if (ni >= 32) {
                        dc = S.cright[c];
                        ni -= 32;
                    }
                    if (dc < 0) {
                        atomicOr(&D.ctrl->error, kErrGeometry);
                    } else {
                        if (core) {
                            acc[5] += v - v0;
                            acc[6] += v ? 1u : 0u;
                            acc_hash += vehicle_term(id, lid, (uint32_t)k, S.cx0[dc] + (uint32_t)ni, v) - old_term;
                        }
                        if (S.ckind[dc] == 0) {
                            const int dw = wi(k, dc);
                            const uint32_t bit = 1u << ni;
                            // write the payload buffer that no reader of this step uses
                            const bool b1 = (S.o0[dw] & bit) ? !(S.l0[dw] & bit) : false;
                            const size_t pd = (size_t)(S.cw[dc] + (uint32_t)k) * 32u + (uint32_t)ni;
                            const int8_t vb = (int8_t)(TURNS ? (v | (al << 4)) : v);
                            if (b1) {
                                velw1[pd] = vb;
                                vidw1[pd] = idw;
                                atomicOr(&S.nl[dw], bit);
                            } else {
                                velw0[pd] = vb;
                                vidw0[pd] = idw;
                            }
                            const uint32_t old = atomicOr(&S.no[dw], bit);
                            if (old & bit) atomicOr(&D.ctrl->error, kErrCellTaken);
                            if (v) atomicOr(&S.nm[dw], bit);
                        }
                    }
                }
            });
        }

        // ---------------- the state of step t+1 of this lane's column
        if (core) {
#pragma unroll
            for (int k = 0; k < kMaxLanes; ++k) {
                if ((uint32_t)k >= lanes) break;
                const uint32_t g = cw + (uint32_t)k;
                D.occ[nxt][g] = S.no[wi(k, s)];
                D.mov[nxt][g] = S.nm[wi(k, s)];
                D.loc[nxt][g] = S.nl[wi(k, s)];
            }
        }
        __syncwarp();
    }
    {
        unsigned long long v[8];
        widen(v);
        block_end_flush<NW, 8>(v, cur_rec, SB.red, SB.rec, kField);
        if constexpr (XFER) {
            __syncthreads();
            block_end_flush<NW, 7>(acc2, cur_rec2, SB.red2, SB.rec2, kField2);
        }
    }
    pdl_trigger();  // blocks without tiles
    span_mark(span, pos, 0, false);
}

constexpr int kLinkWarps = kLinkWarpsPerBlock;
constexpr int kLinkBlock = kLinkWarps * 32;

template <bool XFER, int VM>
__global__ void __launch_bounds__(kLinkBlock, 6)
    link_kernel(const ScenDev *__restrict__ table, const uint2 *__restrict__ tiles,
                const uint32_t *__restrict__ n_tiles_p, uint32_t pos, unsigned long long *span,
                uint32_t *tile_ctr) {
    __shared__ LinkSmem<kLinkWarps> S;
    link_step<kLinkWarps, false, XFER, VM>(S, table, tiles, n_tiles_p, pos, span, tile_ctr);
}

// The same with the intersection rules (scenarios with turn lanes or yield
// approaches).
template <bool XFER, int VM>
__global__ void __launch_bounds__(kLinkBlock, 6)
    turn_link_kernel(const ScenDev *__restrict__ table, const uint2 *__restrict__ tiles,
                     const uint32_t *__restrict__ n_tiles_p, uint32_t pos, unsigned long long *span,
                     uint32_t *tile_ctr) {
    __shared__ LinkSmem<kLinkWarps> S;
    link_step<kLinkWarps, true, XFER, VM>(S, table, tiles, n_tiles_p, pos, span, tile_ctr);
}

// ------------------------------------------------------------------ node kernel
//
// One thread per link m, NT links per block.  Before resolving, each warp
// stages the link-end buffers of the upstream nodes of its 32 links (and,
// with yield approaches, their lane-tail records) into shared memory with
// one flattened load, so no thread walks a long slot list through dependent
// global loads; a thread whose node's buffers do not fit the warp's stage
// reads them from global memory.  Warps synchronise only among their own
// lanes.

constexpr int kStageSlots = 256;  // staged buffers per warp

template <int NT, bool TAILS>
struct NodeSmem {
    uint32_t off[NT / 32][33];  // first staged entry of each lane's node buffers; [32]: the warp's total
    uint32_t lo[NT / 32][32];   // first buffer of each lane's upstream node
    uint4 stage[NT / 32][kStageSlots];
    uint2 tail[NT / 32][TAILS ? kStageSlots : 1];
    unsigned long long red[NT / 32][7];
};

// Gap acceptance with the node's staged tail records (x word of the lane's
// last column, y cells | lanes << 24 | acceptance gap << 27): true iff no
// priority lane of the node has a vehicle in its cells max(1, L - G) .. L - 1
// in occ.  All tail words are loaded before any test.
__device__ __forceinline__ bool gap_clear_staged(const uint2 *tails, const uint32_t *__restrict__ occ, uint32_t prio,
                                                 uint32_t G) {
    uint32_t hit = 0u;
#pragma unroll 4
    for (uint32_t s = 0; s < prio; ++s) {
        const uint2 tl = tails[s];
        const uint32_t L = tl.y & 0xFFFFFFu, lanes = (tl.y >> 24) & 7u;
        const uint32_t lo = L > G ? L - G : 1u;
        if (lo >= L) continue;
        const uint32_t jl = (L - 1u) >> 5, jf = lo >> 5;  // G <= 31: at most two columns
        const uint32_t b = (L - 1u) & 31u;
        const uint32_t a = jf == jl ? (lo & 31u) : 0u;
        hit |= occ[tl.x] & (0xFFFFFFFFu >> (31u - b)) & (0xFFFFFFFFu << a);
        if (jf < jl) hit |= occ[tl.x - lanes] & (0xFFFFFFFFu << (lo & 31u));
    }
    return hit == 0u;
}

// Node transfer into link m from staged buffers st[0..cnt) of its upstream
// node (global indices slot_lo ..): the same placements as
// resolve_transfers.
template <bool TURNS, class F>
__device__ __forceinline__ uint32_t resolve_staged(const uint4 *st, const uint2 *tails, uint32_t slot_lo, uint32_t cnt,
                                                   uint32_t m, uint32_t lanes, uint32_t free_mask,
                                                   const uint32_t *__restrict__ occ, uint32_t prio, F &&place) {
    for (uint32_t s = 0; s < cnt && free_mask; ++s) {
        const uint4 x = st[s];
        if (x.x == kSlotEmpty || x.y != m) continue;
        if constexpr (TURNS) {
            if (tails) {
                const uint32_t G = tails[s].y >> 27;
                if (G && !gap_clear_staged(tails, occ, prio, G)) continue;
            }
        }
        const uint32_t ks = (x.w >> 8) & 3u;
        const uint32_t pref = ks < lanes - 1u ? ks : lanes - 1u;
        uint32_t qn;
        if ((free_mask >> pref) & 1u) {
            qn = pref;
        } else {
            const uint32_t rest = free_mask & ~(1u << pref);
            if (!rest) continue;
            qn = (uint32_t)(__ffs(rest) - 1);
        }
        free_mask &= ~(1u << qn);
        place(slot_lo + s, x, qn);
    }
    return free_mask;
}

// Node transfer into link m reading its upstream node's buffers from global
// memory one by one (for nodes whose buffers do not fit a warp's stage): the
// same placements as resolve_staged.
template <bool TURNS, class F>
__device__ __forceinline__ uint32_t resolve_global(const uint4 *slots, uint32_t slot_lo, uint32_t cnt, uint32_t m,
                                                   uint32_t lanes, uint32_t free_mask, const ScenDev &D,
                                                   const uint32_t *__restrict__ occ, uint32_t prio, F &&place) {
    for (uint32_t s = 0; s < cnt && free_mask; ++s) {
        const uint4 x = slots[slot_lo + s];
        if (x.x == kSlotEmpty || x.y != m) continue;
        if constexpr (TURNS) {
            if (D.slot_gap) {
                const uint32_t G = D.slot_gap[slot_lo + s];
                if (G && !priority_gap_clear(D.slot_tail, occ, slot_lo, prio, G)) continue;
            }
        }
        const uint32_t ks = (x.w >> 8) & 3u;
        const uint32_t pref = ks < lanes - 1u ? ks : lanes - 1u;
        uint32_t qn;
        if ((free_mask >> pref) & 1u) {
            qn = pref;
        } else {
            const uint32_t rest = free_mask & ~(1u << pref);
            if (!rest) continue;
            qn = (uint32_t)(__ffs(rest) - 1);
        }
        free_mask &= ~(1u << qn);
        place(slot_lo + s, x, qn);
    }
    return free_mask;
}

// The step of a node pass at chunk position pos: per step (split steps) the
// step itself if the scenario runs it; at a chunk's end (fused steps) the last
// step the scenario ran in the chunk.  Returns false if there is none.
__device__ __forceinline__ bool node_step(const ScenDev &D, uint32_t pos, bool chunk_end, unsigned long long &step) {
    const unsigned long long base = D.ctrl->base, target = D.ctrl->target;
    if (target <= base) return false;
    step = base + pos;
    if (step >= target) {
        if (!chunk_end) return false;
        step = target - 1ull;
    }
    return true;
}

// One node pass (body of node_kernel and turn_node_kernel): node transfers
// and departures into every link m at the end of the step, on the state
// after that step's moves.  acc gets the transfers, insertions and the
// changes of active, buffered, sum of velocities, digest, and the moving
// vehicles placed.  TURNS: velocity bytes and buffer words carry the allowed
// lanes of the next turn, and transfers from yield approaches wait for the
// gap.
template <int NT, bool TURNS>
__device__ __forceinline__ void node_pass(NodeSmem<NT, TURNS> &S, const ScenDev *__restrict__ table,
                                          const uint4 *__restrict__ tiles, const uint32_t *__restrict__ n_tiles_p,
                                          uint32_t pos, uint32_t chunk_end, unsigned long long *span) {
    const uint32_t n_tiles = *n_tiles_p;
    static constexpr int kField[7] = {kTransfers, kInserted, kDActive, kDBuffered, kDSumV, kDHash, kMoving};
    unsigned long long acc[7] = {0, 0, 0, 0, 0, 0, 0};
    unsigned long long *cur_rec = nullptr;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    bool waited = false;
    for (uint32_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        if (tile + gridDim.x >= n_tiles) pdl_trigger();  // the block's last tile (see link_step)
        const uint4 td = tiles[tile];
        const ScenDev &D = table[td.x];
        if (D.ctrl == nullptr) continue;
        const uint32_t m = td.y + threadIdx.x;
        const bool has = m < td.z;
        const uint4 nd = has ? D.nd_info[m] : make_uint4(0u, 0u, 0u, 0u);  // static
        // base and target are constant within a captured chunk
        unsigned long long step;
        if (!node_step(D, pos, chunk_end != 0u, step)) continue;
        // staging offsets: exclusive scan of the buffer counts over the warp
        const uint32_t cnt = nd.z & 0xFFu;
        uint32_t inc = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += y;
        }
        const uint32_t off = inc - cnt;
        S.off[warp][lane] = off;
        S.lo[warp][lane] = nd.x;
        if (lane == 31) S.off[warp][32] = inc;
        __syncwarp();
        if (!waited) {
            pdl_wait();
            waited = true;
            if (threadIdx.x == 0) span_mark(span, pos, 1, true);
        }
        const int nxt = (int)((step + 1ull) & 1ull);
        uint32_t *occ = D.occ[nxt];
        uint32_t *mov = D.mov[nxt];
        uint4 *slots = D.slots[nxt];
        // this thread's inputs (m's cells 0 and queue head) with the staged loads
        const uint2 hd = has ? D.dep_head[m] : make_uint2(0u, 0xFFFFFFFFu);
        // m's column-0 words (this thread is their only writer in the pass):
        // loaded once, changed bits written once at the end
        const uint32_t mlanes = (nd.z >> 8) & 0xFFu;
        uint32_t o4[kMaxLanes], m4[kMaxLanes];
        uint32_t free0 = 0u;
#pragma unroll
        for (int k = 0; k < kMaxLanes; ++k) {
            const bool w = has && (uint32_t)k < mlanes;
            o4[k] = w ? occ[nd.y + (uint32_t)k] : 1u;
            m4[k] = w ? mov[nd.y + (uint32_t)k] : 0u;
            free0 |= ((o4[k] & 1u) ^ 1u) << k;
        }
        uint32_t placed = 0u, moved = 0u;
        const uint32_t total = S.off[warp][32];
        const uint32_t lim = total < (uint32_t)kStageSlots ? total : (uint32_t)kStageSlots;
        const bool tails = TURNS && D.slot_tail != nullptr;
        // every copy is issued before any is waited for (one round trip)
        for (uint32_t e = (uint32_t)lane; e < lim; e += 32u) {
            // owner: the last lane whose range starts at or before e
            uint32_t i = 0u;
#pragma unroll
            for (uint32_t h = 16; h > 0; h >>= 1)
                if (S.off[warp][i + h] <= e) i += h;
            const uint32_t si = S.lo[warp][i] + (e - S.off[warp][i]);
            cp_async(&S.stage[warp][e], &slots[si], 16);
            if constexpr (TURNS) {
                if (tails) cp_async(&S.tail[warp][e], &D.slot_tail[si], 8);
            }
        }
        cp_async_wait_all();
        __syncwarp();
        unsigned long long *rec = reinterpret_cast<unsigned long long *>(stat_rec(D, step));
        if (rec != cur_rec) {
            if (cur_rec) block_flush<7, NT>(acc, cur_rec, kField, S.red);
            cur_rec = rec;
        }
        if (has) {
            int8_t *vel = D.vel[0];   // a vehicle placed in an empty cell 0 keeps its
            uint32_t *vid = D.vid[0];  // payload in buffer 0 (location bit 0)
            auto place = [&](uint32_t si, const uint4 &x, uint32_t qn) {
                const uint32_t id = x.x & kIdMask, v = x.w & (TURNS ? 0xFu : 0xFFu), ks = (x.w >> 8) & 3u;
                const uint32_t w = nd.y + qn;  // column 0 of lane qn
                placed |= 1u << qn;
                if (v) moved |= 1u << qn;
                vel[(size_t)w * 32u] = (int8_t)(TURNS ? (x.w & 0xFFu) : v);
                vid[(size_t)w * 32u] = x.x;  // id with the last-link flag of m
                atomicAdd(&D.veh[id].x, 1u);
                slots[si].x = kSlotEmpty;
                // travel times: + the exit step on the link left, - the entry step on m
                atomicAdd(&D.link_time[x.z], kLinkTimeOne + step);
                atomicAdd(&D.link_time[m], 0ull - step);
                D.enter_step[id] = (uint32_t)step;
                acc[0] += 1;
                acc[2] += 1;
                acc[3] -= 1;
                acc[4] += v;
                acc[5] += vehicle_term(id, m, qn, 0u, v) - vehicle_term(id, x.z, ks, x.w >> 10, v);
                acc[6] += v ? 1u : 0u;
            };
            const uint32_t lanes = (nd.z >> 8) & 0xFFu, prio = (nd.z >> 16) & 0xFFu;
            uint32_t fr;
            if (off + cnt <= (uint32_t)kStageSlots)
                fr = resolve_staged<TURNS>(S.stage[warp] + off, tails ? S.tail[warp] + off : nullptr, nd.x, cnt, m,
                                           lanes, free0, occ, prio, place);
            else  // a node whose buffers do not fit the stage: straight from global memory
                fr = resolve_global<TURNS>(slots, nd.x, cnt, m, lanes, free0, D, occ, prio, place);
            run_departures_from(D, nd, m, (uint32_t)step, hd, fr, [&](uint32_t idw, uint32_t qn, uint32_t qi) {
                const uint32_t w = nd.y + qn;
                placed |= 1u << qn;
                vel[(size_t)w * 32u] = (TURNS && D.dep_turn) ? (int8_t)(D.dep_turn[qi] << 4) : (int8_t)0;
                vid[(size_t)w * 32u] = idw;
                atomicAdd(&D.link_time[m], 0ull - step);
                D.enter_step[idw & kIdMask] = (uint32_t)step;
                acc[1] += 1;
                acc[2] += 1;
                acc[5] += vehicle_term(idw & kIdMask, m, qn, 0u, 0u);
            });
#pragma unroll
            for (int k = 0; k < kMaxLanes; ++k) {
                if ((placed >> k) & 1u) occ[nd.y + (uint32_t)k] = o4[k] | 1u;
                if ((moved >> k) & 1u) mov[nd.y + (uint32_t)k] = m4[k] | 1u;
            }
        }
        __syncwarp();  // the stage is rewritten by the next tile
    }
    if (cur_rec) block_flush<7, NT>(acc, cur_rec, kField, S.red);
    pdl_trigger();
    span_mark(span, pos, 1, false);
}

__global__ void __launch_bounds__(kNodeThreads) node_kernel(const ScenDev *__restrict__ table,
                                                            const uint4 *__restrict__ tiles,
                                                            const uint32_t *__restrict__ n_tiles_p, uint32_t pos,
                                                            uint32_t chunk_end, unsigned long long *span) {
    __shared__ NodeSmem<kNodeThreads, false> S;
    node_pass<kNodeThreads, false>(S, table, tiles, n_tiles_p, pos, chunk_end, span);
}

// The same for scenarios with turn lanes or yield approaches.
__global__ void __launch_bounds__(kNodeThreads) turn_node_kernel(const ScenDev *__restrict__ table,
                                                                 const uint4 *__restrict__ tiles,
                                                                 const uint32_t *__restrict__ n_tiles_p, uint32_t pos,
                                                                 uint32_t chunk_end, unsigned long long *span) {
    __shared__ NodeSmem<kNodeThreads, true> S;
    node_pass<kNodeThreads, true>(S, table, tiles, n_tiles_p, pos, chunk_end, span);
}

// ------------------------------------------------------------------ load balancing

// Re-tiling from the occupancy (the counterpart of feeding measured load
// back into the partition): one warp per static tile counts the vehicles of
// each of its columns in the current state and cuts the tile greedily where
// the running count would exceed vt, at the positions cut_ok allows (bit t: a
// cut before column t keeps the tiling rules); the sub-tiles go to out, in
// any order, and count (zero before the launch) becomes their number.
// Re-tiling weight of a moving vehicle against a standing one: a standing
// vehicle with an occupied cell ahead is advanced with whole-word bit
// operations, a moving one goes through the per-vehicle lists.
#ifndef TS_MOVING_WEIGHT
#define TS_MOVING_WEIGHT 8
#endif
constexpr uint32_t kMovingWeight = TS_MOVING_WEIGHT;

__global__ void __launch_bounds__(128) retile_kernel(const ScenDev *__restrict__ table, const uint2 *__restrict__ base,
                                                     const uint32_t *__restrict__ cut_ok, uint32_t n_base, uint32_t vt,
                                                     uint2 *__restrict__ out, uint32_t *__restrict__ count) {
    const int lane = threadIdx.x & 31;
    const uint32_t wpb = blockDim.x / 32u, nw = gridDim.x * wpb;
    for (uint32_t b = blockIdx.x * wpb + (threadIdx.x >> 5); b < n_base; b += nw) {
        const uint2 td = base[b];
        const uint32_t scen = td.x & 0xFFFFFFu;
        const int n = (int)(td.x >> 24) + 1;
        const ScenDev &D = table[scen];
        uint32_t cnt = 0u;
        if (lane < n && D.ctrl != nullptr) {
            const uint4 ci = D.col_info[td.y + (uint32_t)lane];
            const uint32_t lanes = (ci.z >> 20) & 7u;
            const uint32_t *occ = D.occ[D.ctrl->base & 1ull];
            const uint32_t *mov = D.mov[D.ctrl->base & 1ull];
            for (uint32_t k = 0; k < lanes; ++k)
                cnt += (uint32_t)__popc(occ[ci.x + k]) + (kMovingWeight - 1u) * (uint32_t)__popc(mov[ci.x + k]);
        }
        const uint32_t ok = cut_ok[b];
        uint32_t cuts = 0u, sum = __shfl_sync(0xffffffffu, cnt, 0);
        for (int t = 1; t < 32; ++t) {
            const uint32_t c = __shfl_sync(0xffffffffu, cnt, t);
            if (t >= n) continue;
            if (sum + c > vt && ((ok >> t) & 1u)) {
                cuts |= 1u << t;
                sum = c;
            } else {
                sum += c;
            }
        }
        const uint32_t starts = cuts | 1u;
        uint32_t at = 0u;
        if (lane == 0) at = atomicAdd(count, (uint32_t)__popc(starts));
        at = __shfl_sync(0xffffffffu, at, 0);
        if (lane < n && ((starts >> lane) & 1u)) {
            const uint32_t later = starts & ~((2u << lane) - 1u);
            const int end = later ? __ffs((int)later) - 1 : n;
            const uint32_t rank = (uint32_t)__popc(starts & ((1u << lane) - 1u));
            out[at + rank] = make_uint2(scen | ((uint32_t)(end - lane - 1) << 24), td.y + (uint32_t)lane);
        }
    }
}

void launch_retile(const ScenDev *table, const uint2 *base, const uint32_t *cut_ok, uint32_t n_base, uint32_t vt,
                   uint2 *out, uint32_t *count, cudaStream_t s) {
    const uint32_t blocks = (n_base + 3u) / 4u;
    const int grid = blocks == 0u ? 1 : (blocks > 4096u ? 4096 : (int)blocks);
    retile_kernel<<<grid, 128, 0, s>>>(table, base, cut_ok, n_base, vt, out, count);
}

// ------------------------------------------------------------------ link travel times

// link_time holds, per link, the exit steps of completed traversals minus
// the entry steps of every traversal begun (plus the count of completed ones
// times kLinkTimeOne); adding back the entry steps of the vehicles still on
// each link (in a cell or its buffer) leaves the travel times of the
// completed ones.  out starts as a copy of link_time.
__global__ void link_time_fix_kernel(const ScenDev D, uint32_t n_veh, unsigned long long *out) {
    for (uint32_t id = blockIdx.x * blockDim.x + threadIdx.x; id < n_veh; id += gridDim.x * blockDim.x) {
        const uint32_t s = D.enter_step[id];
        if (s == kNotOnLink) continue;
        atomicAdd(out + D.route_links[D.veh[id].x], (unsigned long long)s);
    }
}

void launch_link_time_fix(const ScenDev &sd, uint32_t n_veh, unsigned long long *out, cudaStream_t s) {
    const uint32_t blocks = (n_veh + 255u) / 256u;
    const int grid = blocks == 0u ? 1 : (blocks > 4096u ? 4096 : (int)blocks);
    link_time_fix_kernel<<<grid, 256, 0, s>>>(sd, n_veh, out);
}

// ------------------------------------------------------------------ chunk close

// One block per scenario: sums the statistics of the g steps just run,
// moves the step counter and clears the records of the next chunk.
__global__ void __launch_bounds__(128) advance_kernel(const ScenDev *__restrict__ table, uint32_t g_max,
                                                      unsigned long long *span, uint32_t *tile_ctr) {
    pdl_wait();
    // the next chunk's tile claims start from zero
    if (tile_ctr != nullptr && blockIdx.x == 0 && threadIdx.x < kChunk) tile_ctr[threadIdx.x] = 0u;
    if (span != nullptr && blockIdx.x == 0 && threadIdx.x < 2) {
        // the chunk's launches of one kind: durations into the sums, spans reset
        const uint32_t kind = threadIdx.x;
        unsigned long long *acc = span + kChunk * 4u + kind * 2u;
        for (uint32_t p = 0; p < g_max; ++p) {
            unsigned long long *s = span + (p * 2u + kind) * 2u;
            if (s[1] > s[0]) {
                acc[0] += s[1] - s[0];
                acc[1] += 1ull;
            }
            s[0] = ~0ull;
            s[1] = 0ull;
        }
    }
    const ScenDev &D = table[blockIdx.x];
    Ctrl *c = D.ctrl;
    if (c == nullptr) return;
    constexpr int NF = kStatFields;
    __shared__ unsigned long long red[4][NF];
    __shared__ unsigned long long s_base;
    __shared__ unsigned long long s_dact[kChunk];  // change of the vehicles in cells, per step of the chunk
    const unsigned long long base = c->base, target = c->target;
    const uint32_t g = base < target ? (uint32_t)min((unsigned long long)g_max, target - base) : 0u;
    const uint32_t nsub = D.n_sub;
    // sums of every field of the StatRec over the g steps just run
    unsigned long long a[NF] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (uint32_t r = threadIdx.x; r < g * nsub; r += blockDim.x) {
        const unsigned long long t = base + r / nsub;
        const unsigned long long *R =
            reinterpret_cast<const unsigned long long *>(&D.stats[(size_t)(t & (kStatsRing - 1)) * nsub + r % nsub]);
#pragma unroll
        for (int f = 0; f < NF; ++f) a[f] += R[f];
    }
    // per step: the change of the vehicles in cells, summed over its sub-records
    if (threadIdx.x < g) {
        unsigned long long s = 0;
        for (uint32_t u = 0; u < nsub; ++u)
            s += D.stats[(size_t)((base + threadIdx.x) & (kStatsRing - 1)) * nsub + u].d_active;
        s_dact[threadIdx.x] = s;
    }
#pragma unroll
    for (int f = 0; f < NF; ++f) {
        unsigned long long v = a[f];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5][f] = v;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long sm[NF] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
        for (int w = 0; w < 4; ++w)
            for (int f = 0; f < NF; ++f) sm[f] += red[w][f];
        if (g) {
            c->tot_updates += sm[kUpdates];
            c->tot_lane_changes += sm[kLaneChanges];
            c->tot_transfers += sm[kTransfers];
            c->tot_moving += sm[kMoving];
            // vehicles in cells after each step of the chunk, summed
            unsigned long long act = c->active, sum_act = 0;
            for (uint32_t r = 0; r < g; ++r) {
                act += s_dact[r];
                sum_act += act;
            }
            c->tot_active += sum_act;
            c->arrived += sm[kArrived];
            c->inserted += sm[kInserted];
            c->active += sm[kDActive];
            c->buffered += sm[kDBuffered];
            c->sum_v += sm[kDSumV];
            c->hash += sm[kDHash];
            c->steps_run += g;
            c->base = base + g;
        }
        s_base = base + g;
    }
    __syncthreads();
    if (g == 0) return;
    // clear the records of the next chunk
    const unsigned long long nb = s_base;
    const uint32_t per = nsub * (uint32_t)(sizeof(StatRec) / 8);
    for (uint32_t u = threadIdx.x; u < kChunk * per; u += blockDim.x) {
        const unsigned long long t = nb + u / per;
        unsigned long long *z = reinterpret_cast<unsigned long long *>(D.stats + (size_t)(t & (kStatsRing - 1)) * nsub);
        z[u % per] = 0ull;
    }
}

__global__ void set_target_kernel(Ctrl *ctrl, unsigned long long target) { ctrl->target = target; }

// Word 0 of Philox-4x32-10 for counters (c0[i], c1[i], 0, 0), as the link
// kernel draws it (ts_philox_words).
__global__ void philox_words_kernel(const uint32_t *__restrict__ c0, const uint32_t *__restrict__ c1, uint32_t k0,
                                    uint32_t k1, uint32_t n, uint32_t *__restrict__ out) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        out[i] = philox_word0(c0[i], c1[i], k0, k1);
}

void launch_philox_words(const uint32_t *c0, const uint32_t *c1, uint32_t k0, uint32_t k1, uint32_t n,
                         uint32_t *out, cudaStream_t s) {
    const uint32_t blocks = (n + 255u) / 256u;
    const int grid = blocks == 0u ? 1 : (blocks > 4096u ? 4096 : (int)blocks);
    philox_words_kernel<<<grid, 256, 0, s>>>(c0, c1, k0, k1, n, out);
}

template <typename... KArgs, typename... Args>
static void launch_pdl(void (*kernel)(KArgs...), int grid, int threads, bool pdl, cudaStream_t s, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(threads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    cudaLaunchKernelEx(&cfg, kernel, args...);
}

static void (*link_instance(bool turns, bool xfer, bool vmax5))(const ScenDev *, const uint2 *, const uint32_t *,
                                                                 uint32_t, unsigned long long *, uint32_t *) {
    if (vmax5) {
        if (turns) return xfer ? turn_link_kernel<true, 5> : turn_link_kernel<false, 5>;
        return xfer ? link_kernel<true, 5> : link_kernel<false, 5>;
    }
    if (turns) return xfer ? turn_link_kernel<true, 0> : turn_link_kernel<false, 0>;
    return xfer ? link_kernel<true, 0> : link_kernel<false, 0>;
}

void launch_link_kernel(const ScenDev *table, const uint2 *tiles, const uint32_t *n_tiles, uint32_t i, int grid,
                        cudaStream_t s, bool pdl, bool xfer, bool turns, unsigned long long *span, bool vmax5,
                        uint32_t *tile_ctr) {
    launch_pdl(link_instance(turns, xfer, vmax5), grid, kLinkBlock, pdl, s, table, tiles, n_tiles, i, span,
               tile_ctr);
}

void launch_node_kernel(const ScenDev *table, const uint4 *tiles, const uint32_t *n_tiles, uint32_t i, int grid,
                        cudaStream_t s, bool pdl, bool chunk_end, bool turns, unsigned long long *span) {
    launch_pdl(turns ? turn_node_kernel : node_kernel, grid, kNodeThreads, pdl, s, table, tiles, n_tiles, i,
               chunk_end ? 1u : 0u, span);
}

void launch_advance_kernel(const ScenDev *table, uint32_t n_scen, uint32_t g, cudaStream_t s, bool pdl,
                           unsigned long long *span, uint32_t *tile_ctr) {
    launch_pdl(advance_kernel, (int)n_scen, 128, pdl, s, table, g, span, tile_ctr);
}

void launch_set_target(Ctrl *ctrl, unsigned long long target, cudaStream_t s) {
    set_target_kernel<<<1, 1, 0, s>>>(ctrl, target);
}

static int resident_blocks(const void *fn, int threads) {
    int dev = 0, n = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, threads, 0);
    return (n > 0 ? n : 1) * (sms > 0 ? sms : 1);
}

#ifdef TS_PHASE_TIMING
extern "C" int ts_debug_phase_times(unsigned long long *out, int n_blocks) {
    if (n_blocks > kPhaseBlocks) n_blocks = kPhaseBlocks;
    for (int p = 0; p < kPhases; ++p)
        if (cudaMemcpyFromSymbol(out + (size_t)p * n_blocks, g_phase, sizeof(unsigned long long) * n_blocks,
                                 sizeof(unsigned long long) * kPhaseBlocks * p) != cudaSuccess)
            return -1;
    return n_blocks;
}
extern "C" int ts_debug_phase_sums(unsigned long long *out, int reset) {
    if (reset) {
        unsigned long long z[kPhases] = {};
        return cudaMemcpyToSymbol(g_phase_sum, z, sizeof(z)) == cudaSuccess ? 0 : -1;
    }
    return cudaMemcpyFromSymbol(out, g_phase_sum, sizeof(unsigned long long) * kPhases) == cudaSuccess ? 0 : -1;
}
#endif

// Shared-memory share of the unified L1/shared storage the kernels ask for,
// in percent of the maximum (228 KB); the rest stays L1, which holds the
// payload lines a tile's lane-change phase loads and its velocity phase
// reads again.  Measured on GB300 (config 2, link kernel per launch): 60 %
// 46.4-47.0 us, 56 % 51.8, 100 % 48.3, 70 % 56.4, 50 % 49.8, 40 % 67.6.
constexpr int kLinkCarveout = 60;
constexpr int kNodeCarveout = 50;

int max_link_blocks(bool turns) {
    // six blocks of four warps per SM (80 registers a thread: fewer spills
    // than at 64 with eight blocks, measured faster on the 20,024- and
    // 200,000-link networks) need the largest shared-memory share of L1
    for (int x = 0; x < 4; ++x)
        cudaFuncSetAttribute((const void *)link_instance(turns, (x & 1) != 0, (x & 2) != 0),
                             cudaFuncAttributePreferredSharedMemoryCarveout, kLinkCarveout);
    return resident_blocks((const void *)link_instance(turns, false, false), kLinkBlock);
}
int max_node_blocks(bool turns) {
    const void *fn = turns ? (const void *)turn_node_kernel : (const void *)node_kernel;
    cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, kNodeCarveout);
    return resident_blocks(fn, kNodeThreads);
}

}  // namespace tsim
