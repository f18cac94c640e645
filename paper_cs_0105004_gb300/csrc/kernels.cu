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
// Debug builds only: %globaltimer stamps at the phase boundaries of the first
// tile of every link_kernel block of the last launch.
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
// [launch position * 3 + kernel kind][first block entry, last block exit]
__device__ unsigned long long g_span[128][2];
__device__ __forceinline__ void span_mark(int slot, bool enter) {
    if (threadIdx.x == 0 && slot < 128) {
        unsigned long long t;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
        if (enter) atomicMin(&g_span[slot][0], t);
        else atomicMax(&g_span[slot][1], t);
    }
}
#else
__device__ __forceinline__ void stamp(int, bool) {}
__device__ __forceinline__ void span_mark(int, bool) {}
#endif

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
        const uint32_t L = tl.y & 0xFFFFFFu, lanes = tl.y >> 24;
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

constexpr int kCols = kTileMaxCols + 2;

// Shared memory of one link-kernel block for tiles of at most TW occupancy
// words (core + a merged tail column + a halo column on each side).
template <int TW>
struct LinkSmem {
    static constexpr int kWords = TW + 4 + 2 * kMaxLanes;
    static constexpr int kList = kWords * 32;  // every cell of a tile can hold a vehicle
    uint32_t occ0[kWords];  // step t: occupancy, v > 0, payload buffer  // step t: occupancy, v > 0, payload buffer
    uint32_t mov0[kWords];
    uint32_t loc0[kWords];
    uint32_t mv[kWords];    // vehicles that changed INTO the word's lane
    uint32_t occ1[kWords];  // after the lane-change sub-step
    uint32_t mov1[kWords];
    uint32_t oocc[kWords];  // step t+1 (core words)
    uint32_t omov[kWords];
    uint32_t oloc[kWords];
    uint32_t gw[kWords];    // global word index of each local word
    uint8_t wcol[kWords], wlane[kWords];
    uint16_t cw[kCols];             // local word of lane 0 of each column
    uint32_t cx0[kCols];            // first cell of the column within its link
    uint32_t cnear[kCols];          // cells within vmax of a (non-periodic) link end
    int16_t right[kCols], left[kCols];
    uint8_t clink[kCols], ckind[kCols];  // ckind: 0 core, 1 left halo, 2 right halo
    uint32_t lcells[kTileMaxCols], lid[kTileMaxCols], lbpos[kTileMaxCols];
    uint8_t llanes[kTileMaxCols], lring[kTileMaxCols], lexit[kTileMaxCols];  // lexit: lanes whose buffer is empty
    uint8_t lend[kTileMaxCols];       // the link's end (and its buffers) is in this tile
    uint8_t lgreen[kTileMaxCols];     // the light at the link's end is green in this step (1 without a signal)
    uint2 lsig[kTileMaxCols];         // its signal: cycle | green << 16, offset
    uint16_t lcw0[kTileMaxCols];      // local word of column 0 if the link starts in this tile, else 0xFFFF
    uint32_t nlist[2];                // vehicles in the lane-change list and in the velocity list
    uint16_t code[kList];             // (local word << 5) | bit
    unsigned long long red[kLinkThreads / 32][8];  // per warp (at most kLinkThreads threads)
    unsigned long long xacc[7];       // node-transfer counts of the current previous-step record
    int ncols, nwords, ncore_words, nlinks;
};

template <class SM>
__device__ __forceinline__ uint32_t gap_ahead(const uint32_t *O, const SM &S, int c, int k, int i,
                                              uint32_t dist, uint32_t open, uint32_t vmax) {
    const uint32_t w0 = O[S.cw[c] + k];
    const int r = S.right[c];
    const uint32_t w1 = r >= 0 ? O[S.cw[r] + k] : 0u;
    const unsigned long long win = (((unsigned long long)w1 << 32) | w0) >> (i + 1);
    uint32_t g = win ? (uint32_t)(__ffsll((long long)win) - 1) : 64u;
    if (g > dist) g = dist + open;
    return g < vmax ? g : vmax;
}

template <class SM>
__device__ __forceinline__ bool room_behind(const uint32_t *O, const SM &S, int c, int k, int i,
                                            uint32_t vmax) {
    const int l = S.left[c];
    const unsigned long long back = ((unsigned long long)O[S.cw[c] + k] << 32) | (l >= 0 ? O[S.cw[l] + k] : 0u);
    const unsigned long long mask = ((2ull << vmax) - 1ull) << (32 + i - (int)vmax);
    return (back & mask) == 0ull;
}

// Bit x of the result: cell x+1 of the same lane is occupied (next word's bit
// 0 for x = 31).
template <class SM>
__device__ __forceinline__ uint32_t ahead_mask(const uint32_t *O, const SM &S, int c, int k) {
    const int r = S.right[c];
    return (O[S.cw[c] + k] >> 1) | ((r >= 0 ? O[S.cw[r] + k] : 0u) << 31);
}

// Vehicles a tile must look at for lane changes: every one in its core
// columns, the last vmax cells of a left halo column (they can move into the
// core) and the first vmax cells of a right halo column (their lane changes
// shape the cells the core vehicles look ahead into).
__device__ __forceinline__ uint32_t lc_mask(uint8_t kind, uint32_t vmax) {
    return kind == 0 ? 0xFFFFFFFFu : (kind == 1 ? ~((1u << (32 - vmax)) - 1u) : ((1u << vmax) - 1u));
}

// Vehicles a tile moves: its core, and the last vmax cells of a left halo.
__device__ __forceinline__ uint32_t move_mask(uint8_t kind, uint32_t vmax) {
    return kind == 0 ? 0xFFFFFFFFu : (kind == 1 ? ~((1u << (32 - vmax)) - 1u) : 0u);
}

// Appends the set bits of m (word w) to the block's vehicle list; one thread
// per word, one shared-memory reservation per warp.
template <class SM>
__device__ __forceinline__ void list_append(SM &S, uint32_t &count, int w, uint32_t m) {
    const int lane = threadIdx.x & 31;
    const uint32_t cnt = (uint32_t)__popc(m);
    uint32_t inc = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    uint32_t base = 0u;
    if (lane == 31 && inc) base = atomicAdd(&count, inc);
    base = __shfl_sync(0xffffffffu, base, 31);
    uint32_t r = base + inc - cnt;
    while (m) {
        const int b = __ffs(m) - 1;
        m &= m - 1;
        S.code[r++] = (uint16_t)((w << 5) | b);
    }
}

// Node transfers and departures into link l = S.lid[q] (which starts in this
// tile) at the end of step t-1, for fused steps.  Returns the vehicles
// placed on l.
template <bool TURNS, class SM>
__device__ __forceinline__ uint32_t xfer_into_link(SM &S, const ScenDev &D, int q, uint32_t t,
                                                   const uint4 *__restrict__ sc, const uint32_t *__restrict__ oc,
                                                   uint32_t l) {
    const uint4 nd = D.nd_info[l];
    uint32_t placed = 0u, moving = 0u;
    unsigned long long acc2[7] = {0, 0, 0, 0, 0, 0, 0};
    int8_t *vel = D.vel[0];  // cell 0 was empty: its payload goes
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
    const uint32_t n_placed = (uint32_t)__popc(placed);  // they are updated in step t
    if (placed)
        for (int f = 0; f < 7; ++f)
            if (acc2[f]) atomicAdd(&S.xacc[f], acc2[f]);
    for (uint32_t m = placed; m; m &= m - 1u) {
        const uint32_t qn = (uint32_t)(__ffs(m) - 1);
        atomicOr(&S.occ0[S.lcw0[q] + qn], 1u);
        if ((moving >> qn) & 1u) atomicOr(&S.mov0[S.lcw0[q] + qn], 1u);
    }
    return n_placed;
}

// Whether the buffer idx holding x is emptied by the node transfer of step
// t-1 (the same resolution as the tile of x's next link computes).
template <bool TURNS>
__device__ __forceinline__ void buffer_emptied(const ScenDev &D, const uint4 *__restrict__ sc,
                                               const uint32_t *__restrict__ oc, const uint4 &x, uint32_t idx,
                                               bool &empty) {
    const uint4 nd = D.nd_info[x.y];
    resolve_transfers<TURNS>(sc, nd, x.y, free_cell0(oc, nd), D, oc,
                             [&](uint32_t si, const uint4 &, uint32_t) { empty |= si == idx; });
}

// The intersection-rule versions out of line, so that their registers stay
// out of link_buffers_phase.
template <class SM>
__device__ __noinline__ uint32_t xfer_into_link_turns(SM &S, const ScenDev &D, int q, uint32_t t,
                                                      const uint4 *__restrict__ sc, const uint32_t *__restrict__ oc,
                                                      uint32_t l) {
    return xfer_into_link<true>(S, D, q, t, sc, oc, l);
}
__device__ __noinline__ bool buffer_emptied_turns(const ScenDev &D, const uint4 *__restrict__ sc,
                                                  const uint32_t *__restrict__ oc, uint4 x, uint32_t idx) {
    bool empty = false;
    buffer_emptied<true>(D, sc, oc, x, idx, empty);
    return empty;
}

// The link thread of link q (index in the tile): with do_xfer, completes the
// node transfers and departures into q (if q starts in this tile) at the end
// of step t-1; then sets up q's lane-end buffers for step t (if q ends in this
// tile).  Returns the vehicles placed on q.  Out of line, so that its
// registers do not weigh on the rest of the step.  TURNS: velocity bytes and
// buffer words carry the allowed lanes of the next turn, and transfers from
// yield approaches wait for the gap.
template <bool TURNS, class SM>
__device__ __noinline__ uint32_t link_buffers_phase(SM &S, const ScenDev &D, int q, int cur, uint32_t t,
                                                    bool do_xfer) {
    const int nxt = cur ^ 1;
    uint32_t n_placed = 0u;
    const uint4 *__restrict__ sc = D.slots[cur];
    uint4 *__restrict__ sn = D.slots[nxt];
    const uint32_t *__restrict__ oc = D.occ[cur];
    const uint32_t l = S.lid[q];
    if (do_xfer && S.lcw0[q] != 0xFFFFu) {
        // transfers and departures into l at the end of step t-1
        if constexpr (TURNS)
            n_placed = xfer_into_link_turns(S, D, q, t, sc, oc, l);
        else
            n_placed = xfer_into_link<false>(S, D, q, t, sc, oc, l);
    }
    uint32_t open = 0u;
    if (S.lend[q]) {
        // l's lane-end buffers for step t: empty, or emptied by a
        // transfer of step t-1 (the same resolution as the tile of
        // the next link computes), or still holding their vehicle
        const uint32_t nl = S.llanes[q], b0 = S.lbpos[q];
        uint4 own[kMaxLanes];
#pragma unroll
        for (int k = 0; k < kMaxLanes; ++k)
            own[k] = (uint32_t)k < nl ? sc[b0 + k] : make_uint4(kSlotEmpty, 0u, 0u, 0u);
#pragma unroll
        for (uint32_t k = 0; k < (uint32_t)kMaxLanes; ++k) {
            if (k >= nl) break;
            const uint32_t idx = b0 + k;
            const uint4 x = own[k];
            bool empty = x.x == kSlotEmpty;
            if (!empty && do_xfer) {
                if constexpr (TURNS)
                    empty = buffer_emptied_turns(D, sc, oc, x, idx);
                else
                    buffer_emptied<false>(D, sc, oc, x, idx, empty);
            }
            if (empty) open |= 1u << k;
            sn[idx] = empty ? make_uint4(kSlotEmpty, kSlotEmpty, kSlotEmpty, kSlotEmpty) : x;
        }
    }
    S.lexit[q] = (uint8_t)open;
    // the light at the link end (Sec. 3): while red, a virtual vehicle of
    // maximum velocity zero stands at every lane end
    const uint2 sg = S.lsig[q];
    const uint32_t cycle = sg.x & 0xFFFFu, green = sg.x >> 16;
    S.lgreen[q] = (uint8_t)(cycle == 0u || (t + sg.y) % cycle < green);
    return n_placed;
}

// Threads of a link-kernel block for tiles of at most TW words: one per word
// of the default tile (halos included), or 256 for the large tiles; as many
// blocks per SM as 64 registers per thread allow.
template <int TW>
struct LinkLaunch {
    static constexpr int kThreads = TW <= kDefaultTileWords ? kSmallTileThreads : kLinkThreads;
    static constexpr int kMinBlocks = 65536 / (kThreads * 64);
};

// One launch of the link kernel (body of link_kernel and turn_link_kernel).
// TURNS: the intersection rules of Sec. 3 a network may carry: plan-following
// lane changes (every velocity byte carries the lanes A of its link from
// which the vehicle may take its next turn) and gap acceptance at
// unprotected turns (in the node transfers).
template <int TW, bool TURNS>
__device__ __forceinline__ void link_step(LinkSmem<TW> &S, const ScenDev *__restrict__ table,
                                          const LinkTile *__restrict__ tiles, const uint32_t *__restrict__ n_tiles_p,
                                          uint32_t pos, uint32_t xfer) {
    const uint32_t n_tiles = *n_tiles_p;  // changes only between graph launches
    // statistics of the block: updates, lane changes, arrivals, and the changes
    // of active, buffered, sum of velocities and digest
    static constexpr int kField[8] = {kUpdates, kLaneChanges, kArrived, kDActive, kDBuffered, kDSumV, kDHash,
                                      kMoving};
    // counts in 32 bits (per block and step they stay far below 2^31; the
    // changes are signed), the digest change in 64
    uint32_t acc[7] = {0u, 0u, 0u, 0u, 0u, 0u, 0u};
    unsigned long long acc_hash = 0ull;
    auto flush_acc = [&](unsigned long long *rec) {
        unsigned long long v[8] = {acc[0], acc[1], acc[2], (unsigned long long)(long long)(int)acc[3],
                                   (unsigned long long)(long long)(int)acc[4],
                                   (unsigned long long)(long long)(int)acc[5], acc_hash, acc[6]};
        block_flush<8, LinkLaunch<TW>::kThreads>(v, rec, kField, S.red);
#pragma unroll
        for (int f = 0; f < 7; ++f) acc[f] = 0u;
        acc_hash = 0ull;
    };
    unsigned long long *cur_rec = nullptr;
    // with xfer set, the launch first completes the node transfers and
    // departures of the previous step (whose record gets these counts):
    // transfers, insertions and the changes of active, buffered, sum of v, digest
    static constexpr int kField2[7] = {kTransfers, kInserted, kDActive, kDBuffered, kDSumV, kDHash, kMoving};
    unsigned long long *cur_rec2 = nullptr;
    if (threadIdx.x < 7) S.xacc[threadIdx.x] = 0ull;  // ordered by the first tile's barrier
    auto flush_xacc = [&]() {
        if (threadIdx.x < 7 && S.xacc[threadIdx.x]) {
            atomicAdd(cur_rec2 + kField2[threadIdx.x], S.xacc[threadIdx.x]);
            S.xacc[threadIdx.x] = 0ull;
        }
        __syncthreads();
    };
    pdl_trigger();
    span_mark((int)pos * 3, true);
    bool waited = false;
    bool first = true;
    stamp(0, true);
    for (uint32_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        const LinkTile td = tiles[tile];
        const ScenDev &D = table[td.a.x];
        if (D.ctrl == nullptr) continue;
        stamp(1, first);
        const uint32_t vmax = D.vmax;

        // ---------------- tile geometry (static data: read before waiting)
        const bool partial = (td.a.z & kPartial) != 0u;
        auto near_mask = [&](uint32_t ring, uint32_t cells, uint32_t x0) -> uint32_t {
            if (ring) return 0u;
            const int thr = (int)cells - 1 - (int)vmax - (int)x0;  // first cell within vmax of the end
            return thr <= 0 ? 0xFFFFFFFFu : (thr >= 32 ? 0u : ~((1u << thr) - 1u));
        };
        if (!partial) {
            const int nl = (int)td.a.z;
            const uint32_t wb = td.b.x;
            const int nw = (int)(td.b.y - td.b.x);
            for (int q = threadIdx.x; q < nl; q += blockDim.x) {
                const uint4 li = D.lk_info[td.a.y + q];
                S.lcells[q] = li.y;
                S.llanes[q] = (uint8_t)(li.z & 0xFFu);
                S.lring[q] = (uint8_t)((li.z >> 8) & 1u);
                S.lid[q] = td.a.y + q;
                S.lbpos[q] = li.w;
                const int ncol = (int)((li.y + 31u) >> 5), c0 = (int)((li.z >> 16) & 0xFFu);
                const uint32_t lanes = li.z & 0xFFu, ring = (li.z >> 8) & 1u;
                S.lend[q] = (uint8_t)(ring ^ 1u);
                S.lcw0[q] = ring ? (uint16_t)0xFFFFu : (uint16_t)(li.x - wb);
                S.lsig[q] = D.sig_info ? D.sig_info[td.a.y + q] : make_uint2(0u, 0u);
                for (int j = 0; j < ncol; ++j) {
                    const int c = c0 + j;
                    const uint32_t lw = li.x - wb + (uint32_t)j * lanes;
                    S.cw[c] = (uint16_t)lw;
                    S.cx0[c] = 32u * (uint32_t)j;
                    S.cnear[c] = near_mask(ring, li.y, 32u * (uint32_t)j);
                    S.clink[c] = (uint8_t)q;
                    S.ckind[c] = 0;
                    S.right[c] = (int16_t)(j + 1 < ncol ? c + 1 : (ring ? c0 : -1));
                    S.left[c] = (int16_t)(j > 0 ? c - 1 : (ring ? c0 + ncol - 1 : -1));
                    for (uint32_t k = 0; k < lanes; ++k) {
                        S.wcol[lw + k] = (uint8_t)c;
                        S.wlane[lw + k] = (uint8_t)k;
                    }
                }
                if (q == nl - 1) S.ncols = c0 + ncol;
            }
            for (int w = threadIdx.x; w < nw; w += blockDim.x) {
                S.gw[w] = wb + w;
                S.occ0[w] = 0u;
                S.mov0[w] = 0u;
                S.mv[w] = 0u;
                S.oocc[w] = 0u;
                S.omov[w] = 0u;
                S.oloc[w] = 0u;
            }
            if (threadIdx.x == 0) {
                S.nwords = nw;
                S.ncore_words = nw;
                S.nlinks = nl;
            }
        } else {
            const uint32_t l = td.a.y, wbase = td.b.x, cells = td.b.y;
            const uint32_t lanes = td.b.z & 0xFFu, ring = (td.b.z >> 8) & 1u;
            const int ncol = (int)((cells + 31u) >> 5);
            const int j0 = (int)(td.a.z & ~kPartial), j1 = (int)td.a.w;
            const int ncore = j1 - j0;
            const bool has_l = j0 > 0 || ring, has_r = j1 < ncol || ring;
            const int hl = has_l ? ncore : -1;
            const int hr = has_r ? ncore + (has_l ? 1 : 0) : -1;
            const int ncols = ncore + (has_l ? 1 : 0) + (has_r ? 1 : 0);
            for (int c = threadIdx.x; c < ncols; c += blockDim.x) {
                int j;
                uint8_t kind;
                int16_t rr, ll;
                if (c < ncore) {
                    j = j0 + c;
                    kind = 0;
                    rr = (int16_t)(c + 1 < ncore ? c + 1 : hr);
                    ll = (int16_t)(c > 0 ? c - 1 : hl);
                } else if (c == hl) {
                    j = j0 > 0 ? j0 - 1 : ncol - 1;
                    kind = 1;
                    rr = 0;
                    ll = -1;
                } else {
                    j = j1 < ncol ? j1 : 0;
                    kind = 2;
                    rr = -1;
                    ll = (int16_t)(ncore - 1);
                }
                const uint32_t lw = (uint32_t)c * lanes;
                S.cw[c] = (uint16_t)lw;
                S.cx0[c] = 32u * (uint32_t)j;
                S.cnear[c] = near_mask(ring, cells, 32u * (uint32_t)j);
                S.clink[c] = 0;
                S.ckind[c] = kind;
                S.right[c] = rr;
                S.left[c] = ll;
                for (uint32_t k = 0; k < lanes; ++k) {
                    S.gw[lw + k] = wbase + (uint32_t)j * lanes + k;
                    S.occ0[lw + k] = 0u;
                    S.mov0[lw + k] = 0u;
                    S.mv[lw + k] = 0u;
                    S.oocc[lw + k] = 0u;
                    S.omov[lw + k] = 0u;
                    S.oloc[lw + k] = 0u;
                    S.wcol[lw + k] = (uint8_t)c;
                    S.wlane[lw + k] = (uint8_t)k;
                }
            }
            if (threadIdx.x == 0) {
                S.lcells[0] = cells;
                S.llanes[0] = (uint8_t)lanes;
                S.lring[0] = (uint8_t)ring;
                S.lid[0] = l;
                S.lbpos[0] = td.b.w;
                S.lend[0] = (uint8_t)((!ring && j1 == ncol) ? 1u : 0u);
                S.lcw0[0] = (!ring && j0 == 0) ? (uint16_t)0u : (uint16_t)0xFFFFu;
                S.lsig[0] = D.sig_info ? D.sig_info[l] : make_uint2(0u, 0u);
                S.ncols = ncols;
                S.nwords = ncols * (int)lanes;
                S.ncore_words = ncore * (int)lanes;
                S.nlinks = 1;
            }
        }
        // The step base and target change only between captured chunks (the
        // chunk-closing kernel has finished before a chunk's first launch), so
        // they may be read before waiting for the previous kernel.
        const unsigned long long step = D.ctrl->base + pos;
        const bool active = step < D.ctrl->target;
        if (threadIdx.x == 0) {
            S.nlist[0] = 0u;
            S.nlist[1] = 0u;
        }
        __syncthreads();
        stamp(2, first);
        if (!active) continue;
        if (!waited) {
            pdl_wait();
            waited = true;
        }
        stamp(3, first);
        unsigned long long *rec = reinterpret_cast<unsigned long long *>(stat_rec(D, step));
        if (rec != cur_rec) {
            if (cur_rec) flush_acc(cur_rec);
            cur_rec = rec;
        }
        const uint32_t t = (uint32_t)step;
        const int cur = (int)(step & 1ull), nxt = cur ^ 1;
        const int d = (t & 1u) ? -1 : 1;
        const int nwords = S.nwords, ncore_words = S.ncore_words;
        // word phases: one thread per occupancy word, looping when a tile has
        // more words than the block has threads

        // with xfer, memory holds the state after the moves of step t-1 and
        // the node transfers of t-1 are completed here, before step t
        const bool do_xfer = xfer != 0u;
        if (do_xfer) {
            unsigned long long *rec2 = reinterpret_cast<unsigned long long *>(stat_rec(D, step - 1ull));
            if (rec2 != cur_rec2) {
                if (cur_rec2) flush_xacc();
                cur_rec2 = rec2;
            }
        }

        // ---------------- state of step t (occ0/mov0 start at zero: the word
        // loads and the placements of the node transfers are or-ed in)
        for (int w = threadIdx.x; w < nwords; w += LinkLaunch<TW>::kThreads) {
            const uint32_t g = S.gw[w];
            const uint32_t o = D.occ[cur][g];
            if (o) {
                atomicOr(&S.occ0[w], o);
                atomicOr(&S.mov0[w], D.mov[cur][g]);
            }
            S.loc0[w] = o ? D.loc[cur][g] : 0u;
            if (S.ckind[S.wcol[w]] == 0) acc[0] += (uint32_t)__popc(o);  // vehicle updates
        }
        {
            // link threads, counted down from the last thread
            const int q = LinkLaunch<TW>::kThreads - 1 - (int)threadIdx.x;
            if (q < S.nlinks) acc[0] += link_buffers_phase<TURNS>(S, D, q, cur, t, do_xfer);
        }
        __syncthreads();
        stamp(4, first);
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
        // Moving vehicles and vehicles near a link end are decided one by one.
        const bool lc_on = D.lane_change != 0u;
        if (lc_on) {
            for (int wb = 0; wb < nwords; wb += LinkLaunch<TW>::kThreads) {  // uniform per warp (list_append)
            const int w = wb + (int)threadIdx.x;
            uint32_t listed = 0u;
            if (w < nwords) {
                const int c = S.wcol[w], k = S.wlane[w], kt = k + d;
                const int q = S.clink[c];
                if (kt >= 0 && kt < (int)S.llanes[q]) {
                    const uint32_t o = S.occ0[w] & lc_mask(S.ckind[c], vmax);
                    if (TURNS && o) {
                        // the allowed lanes are in the payload: every vehicle
                        // whose target cell is free is decided one by one
                        listed = o & ~S.occ0[S.cw[c] + kt];
                    } else if (o) {
                        const uint32_t near = S.cnear[c];
                        const uint32_t tw = S.occ0[S.cw[c] + kt];
                        const int lf = S.left[c];
                        const unsigned long long tt =
                            ((unsigned long long)tw << 32) | (lf >= 0 ? S.occ0[S.cw[lf] + kt] : 0u);
                        uint32_t behind = 0u;
                        for (uint32_t j = 1; j <= vmax; ++j) behind |= (uint32_t)(tt >> (32 - j));
                        const uint32_t ok = ahead_mask(S.occ0, S, c, k) & ~tw & ~behind & ~ahead_mask(S.occ0, S, c, kt);
                        const uint32_t lcv0 = o & ~S.mov0[w] & ~near & ok;
                        if (lcv0) {
                            atomicOr(&S.mv[S.cw[c] + kt], lcv0);
                            if (S.ckind[c] == 0) acc[1] += (uint32_t)__popc(lcv0);
                        }
                        listed = o & (S.mov0[w] | near);
                    }
                }
            }
            list_append(S, S.nlist[0], w, listed);
            }
            __syncthreads();
            const uint32_t total = S.nlist[0];
            for (uint32_t e = threadIdx.x; e < total; e += blockDim.x) {
                const uint32_t code = S.code[e];
                const int ww = code >> 5, i = code & 31;
                const int c = S.wcol[ww], k = S.wlane[ww], kt = k + d;
                if ((S.occ0[S.cw[c] + kt] >> i) & 1u) continue;  // target cell taken
                const int q = S.clink[c];
                const uint32_t ring = S.lring[q];
                const uint32_t x = S.cx0[c] + (uint32_t)i;
                const uint32_t dist = ring ? 0xFFFFu : S.lcells[q] - 1u - x;
                // payload at step t; the last-link flag matters only within
                // vmax cells of the link end
                const size_t p = (size_t)S.gw[ww] * 32u + (uint32_t)i;
                const bool b1 = (S.loc0[ww] >> i) & 1u;
                uint32_t v;
                uint32_t al = 0xFu;  // lanes it may leave the link from
                if constexpr (TURNS) {
                    const uint32_t byte = (uint32_t)(uint8_t)(b1 ? vel1[p] : vel0[p]);
                    v = byte & 0xFu;
                    if (byte >> 4) al = byte >> 4;
                } else {
                    v = (uint32_t)(b1 ? vel1[p] : vel0[p]);
                }
                if constexpr (TURNS) {
                    if (!((al >> k) & 1u)) {
                        // outside its allowed lanes: a reason to change when
                        // one of them lies on the side d points to; the gap
                        // accepted behind the target cell shrinks from vmax to
                        // 0 over the link's last vmax cells
                        const uint32_t side = d > 0 ? al & ~((2u << k) - 1u) : al & ((1u << k) - 1u);
                        if (side && room_behind(S.occ0, S, c, kt, i, dist < vmax ? dist : vmax)) {
                            atomicOr(&S.mv[S.cw[c] + kt], 1u << i);
                            if (S.ckind[c] == 0) acc[1] += 1;
                        }
                        continue;
                    }
                    // the speed reason applies only into an allowed lane (and
                    // then both lanes are allowed: the gaps below need no
                    // closed link end)
                    if (!((al >> kt) & 1u)) continue;
                }
                const uint32_t last = ((S.cnear[c] >> i) & 1u) ? (b1 ? vid1[p] : vid0[p]) >> 31 : 0u;
                const uint32_t want = v + 1u < vmax ? v + 1u : vmax;
                const uint32_t g_own =
                    gap_ahead(S.occ0, S, c, k, i, dist, (((S.lexit[q] >> k) & 1u) | last) & S.lgreen[q], vmax);
                if (g_own >= want) continue;
                const uint32_t g_tgt =
                    gap_ahead(S.occ0, S, c, kt, i, dist, (((S.lexit[q] >> kt) & 1u) | last) & S.lgreen[q], vmax);
                if (g_tgt > g_own && room_behind(S.occ0, S, c, kt, i, vmax)) {
                    atomicOr(&S.mv[S.cw[c] + kt], 1u << i);
                    if (S.ckind[c] == 0) acc[1] += 1;
                }
            }
        }
        __syncthreads();
        stamp(5, first);

        // ---------------- sub-step 2: velocity update and move.  A vehicle with
        // v = 0, an occupied cell ahead, no lane change and far from the link
        // end keeps v = 0 and its cell: its bits are copied, its payload stays.
        {
            for (int wb = 0; wb < nwords; wb += LinkLaunch<TW>::kThreads) {  // uniform per warp (list_append)
            const int w = wb + (int)threadIdx.x;
            uint32_t listed = 0u;
            if (w < nwords) {
                const int c = S.wcol[w], k = S.wlane[w];
                const uint8_t kind = S.ckind[c];
                // the words after the lane-change sub-step, from the step-t
                // words and the lane-change marks (mv: vehicles that changed
                // into a word's lane; those leaving lane k went to k + d)
                const int lanes = S.llanes[S.clink[c]];
                const int kf = k + d, kb = k - d;
                const bool has_f = kf >= 0 && kf < lanes, has_b = kb >= 0 && kb < lanes;
                const uint32_t arriving = S.mv[w];
                const uint32_t leaving = has_f ? S.mv[S.cw[c] + kf] : 0u;
                const uint32_t o1 = (S.occ0[w] & ~leaving) | arriving;
                const uint32_t src_mov = (arriving && has_b) ? S.mov0[S.cw[c] + kb] : 0u;
                const uint32_t m1 = (S.mov0[w] & ~leaving) | (src_mov & arriving);
                S.occ1[w] = o1;
                S.mov1[w] = m1;
                const int r = S.right[c];
                const uint32_t o1r =
                    r >= 0 ? (S.occ0[S.cw[r] + k] & ~(has_f ? S.mv[S.cw[r] + kf] : 0u)) | S.mv[S.cw[r] + k] : 0u;
                const uint32_t free_ahead = ~((o1 >> 1) | (o1r << 31));
                const uint32_t busy = m1 | free_ahead | S.cnear[c] | arriving;
                listed = o1 & busy & move_mask(kind, vmax);
                if (kind == 0) {
                    const uint32_t inert = o1 & ~busy;
                    if (inert) {
                        atomicOr(&S.oocc[w], inert);
                        atomicOr(&S.oloc[w], inert & S.loc0[w]);
                    }
                }
            }
            list_append(S, S.nlist[1], w, listed);
            }
            __syncthreads();
            const uint32_t total = S.nlist[1];
            int8_t *__restrict__ velw0 = D.vel[0];
            int8_t *__restrict__ velw1 = D.vel[1];
            uint32_t *__restrict__ vidw0 = D.vid[0];
            uint32_t *__restrict__ vidw1 = D.vid[1];
            const uint32_t key0 = D.seed_lo, key1 = D.seed_hi, pthr = D.p_threshold;
            for (uint32_t e = threadIdx.x; e < total; e += blockDim.x) {
                const uint32_t code = S.code[e];
                const int ww = code >> 5, i = code & 31;
                const int c = S.wcol[ww];
                const int k = S.wlane[ww];
                const int ks = ((S.mv[ww] >> i) & 1u) ? k - d : k;  // lane at step t
                // payload from where the vehicle was at step t; no thread of
                // this step writes a buffer that a step-t occupant is read from
                const int sw = S.cw[c] + ks;
                const size_t ps = (size_t)S.gw[sw] * 32u + (uint32_t)i;
                const bool sb1 = (S.loc0[sw] >> i) & 1u;
                const uint32_t idw = sb1 ? vid1[ps] : vid0[ps];
                uint32_t v0, al = 0u;  // al: allowed lanes of the next turn (0: any)
                if constexpr (TURNS) {
                    const uint32_t byte = (uint32_t)(uint8_t)(sb1 ? vel1[ps] : vel0[ps]);
                    v0 = byte & 0xFu;
                    al = byte >> 4;
                } else {
                    v0 = (uint32_t)(sb1 ? vel1[ps] : vel0[ps]);
                }
                const int q = S.clink[c];
                const uint32_t id = idw & kIdMask, last = idw >> 31;
                const uint32_t ring = S.lring[q];
                const uint32_t x = S.cx0[c] + (uint32_t)i;
                const uint32_t dist = ring ? 0xFFFFu : S.lcells[q] - 1u - x;
                uint32_t v = v0 + 1u < vmax ? v0 + 1u : vmax;  // (i) accelerate
                uint32_t open = (((S.lexit[q] >> k) & 1u) | last) & S.lgreen[q];
                if constexpr (TURNS) {
                    if (al && !((al >> k) & 1u)) open = 0u;  // the next turn is not taken from lane k
                }
                const uint32_t g = gap_ahead(S.occ1, S, c, k, i, dist, open, vmax);
                if (v > g) v = g;                                                 // (ii) gap
                if (v > 0u && philox_word0(t, id, key0, key1) < pthr) v -= 1u;  // (iii) random
                const bool core = S.ckind[c] == 0;
                const uint32_t lid = S.lid[q];
                // the tile whose core held the vehicle at step t accounts for it
                const unsigned long long old_term = core ? vehicle_term(id, lid, (uint32_t)ks, x, v0) : 0ull;
                if (!ring && x + v >= S.lcells[q]) {
                    // reaches the link end; a split leaves more than 2*vmax cells
                    // after it, so such a vehicle is always in this tile's core
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
                            if (!((S.lexit[q] >> k) & 1u)) atomicOr(&D.ctrl->error, kErrSlotTaken);
                            uint32_t vb = v;  // with the allowed lanes of the turn after m
                            if constexpr (TURNS) {
                                if (D.route_turn) vb |= (uint32_t)D.route_turn[ve.x + 1u] << 4;
                            }
                            D.slots[nxt][S.lbpos[q] + (uint32_t)k] =
                                make_uint4(id | fl, m, lid, vb | ((uint32_t)k << 8) | (S.lcells[q] << 10));
                            acc[3] -= 1;
                            acc[4] += 1;
                            acc[5] -= v0;
                            acc_hash += vehicle_term(id, lid, (uint32_t)k, S.lcells[q], v) - old_term;
                        }
                    }
                } else {
                    int ni = i + (int)v;
                    int dc = c;
                    if (ni >= 32) {
                        dc = S.right[c];
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
                            const int dw = S.cw[dc] + k;
                            const uint32_t bit = 1u << ni;
                            // write the payload buffer that no reader of this step uses
                            const bool b1 = (S.occ0[dw] & bit) ? !(S.loc0[dw] & bit) : false;
                            const size_t pd = (size_t)S.gw[dw] * 32u + (uint32_t)ni;
                            const int8_t vb = (int8_t)(TURNS ? (v | (al << 4)) : v);
                            if (b1) {
                                velw1[pd] = vb;
                                vidw1[pd] = idw;
                                atomicOr(&S.oloc[dw], bit);
                            } else {
                                velw0[pd] = vb;
                                vidw0[pd] = idw;
                            }
                            const uint32_t old = atomicOr(&S.oocc[dw], bit);
                            if (old & bit) atomicOr(&D.ctrl->error, kErrCellTaken);
                            if (v) atomicOr(&S.omov[dw], bit);
                        }
                    }
                }
            }
        }
        __syncthreads();
        stamp(6, first);

        // ---------------- write the state of step t+1 and the buffer states
        for (int w = threadIdx.x; w < ncore_words; w += LinkLaunch<TW>::kThreads) {
            const uint32_t g = S.gw[w];
            D.occ[nxt][g] = S.oocc[w];
            D.mov[nxt][g] = S.omov[w];
            D.loc[nxt][g] = S.oloc[w];
        }
        __syncthreads();
        stamp(7, first);
        first = false;
    }
    if (cur_rec) flush_acc(cur_rec);
    if (cur_rec2) flush_xacc();
    stamp(9, true);
    span_mark((int)pos * 3, false);
}

template <int TW>
__global__ void __launch_bounds__(LinkLaunch<TW>::kThreads, LinkLaunch<TW>::kMinBlocks)
    link_kernel(const ScenDev *__restrict__ table, const LinkTile *__restrict__ tiles,
                const uint32_t *__restrict__ n_tiles_p, uint32_t pos, uint32_t xfer) {
    __shared__ LinkSmem<TW> S;
    link_step<TW, false>(S, table, tiles, n_tiles_p, pos, xfer);
}

// The same with the intersection rules (scenarios with turn lanes or yield
// approaches).
template <int TW>
__global__ void __launch_bounds__(LinkLaunch<TW>::kThreads, LinkLaunch<TW>::kMinBlocks)
    turn_link_kernel(const ScenDev *__restrict__ table, const LinkTile *__restrict__ tiles,
                     const uint32_t *__restrict__ n_tiles_p, uint32_t pos, uint32_t xfer) {
    __shared__ LinkSmem<TW> S;
    link_step<TW, true>(S, table, tiles, n_tiles_p, pos, xfer);
}

// ------------------------------------------------------------------ node kernel

// Node transfers and departures into link m (nd = nd_info[m]) at the end of
// step `step`, on the state after that step's moves; acc gets the transfers,
// insertions and the changes of active, buffered, sum of velocities, digest.
// TURNS: velocity bytes and buffer words carry the allowed lanes of the next
// turn, and transfers from yield approaches wait for the gap.
template <bool TURNS>
__device__ __forceinline__ void node_link(const ScenDev &D, uint32_t m, const uint4 &nd, unsigned long long step,
                                          unsigned long long (&acc)[7]) {
    const int nxt = (int)((step + 1ull) & 1ull);
    uint32_t *occ = D.occ[nxt];
    uint32_t *mov = D.mov[nxt];
    uint4 *slots = D.slots[nxt];
    int8_t *vel = D.vel[0];   // a vehicle placed in an empty cell 0 keeps its
    uint32_t *vid = D.vid[0];  // payload in buffer 0 (location bit 0)
    // slots with next link m, the cells 0 of m and m's queue head are
    // written by this thread only; the head is loaded with the node's buffers
    // and m's cells 0, not after the transfers
    const uint2 hd = D.dep_head[m];
    const uint32_t fr = resolve_transfers<TURNS>(slots, nd, m, free_cell0(occ, nd), D, occ,
                                                 [&](uint32_t si, const uint4 &x, uint32_t qn) {
        const uint32_t id = x.x & kIdMask, v = x.w & (TURNS ? 0xFu : 0xFFu), ks = (x.w >> 8) & 3u;
        const uint32_t w = nd.y + qn;  // column 0 of lane qn
        occ[w] |= 1u;
        if (v) mov[w] |= 1u;
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
    });
    run_departures_from(D, nd, m, (uint32_t)step, hd, fr, [&](uint32_t idw, uint32_t qn, uint32_t qi) {
        const uint32_t w = nd.y + qn;
        occ[w] |= 1u;
        vel[(size_t)w * 32u] = (TURNS && D.dep_turn) ? (int8_t)(D.dep_turn[qi] << 4) : (int8_t)0;
        vid[(size_t)w * 32u] = idw;
        atomicAdd(&D.link_time[m], 0ull - step);
        D.enter_step[idw & kIdMask] = (uint32_t)step;
        acc[1] += 1;
        acc[2] += 1;
        acc[5] += vehicle_term(idw & kIdMask, m, qn, 0u, 0u);
    });
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

// One node pass, one thread per link m (body of node_kernel and
// turn_node_kernel).
template <bool TURNS>
__device__ __forceinline__ void node_pass(unsigned long long (*red)[7], const ScenDev *__restrict__ table,
                                          const uint4 *__restrict__ tiles, const uint32_t *__restrict__ n_tiles_p,
                                          uint32_t pos, uint32_t chunk_end) {
    const uint32_t n_tiles = *n_tiles_p;
    // transfers, insertions and the changes of active, buffered, sum of velocities, digest
    static constexpr int kField[7] = {kTransfers, kInserted, kDActive, kDBuffered, kDSumV, kDHash, kMoving};
    unsigned long long acc[7] = {0, 0, 0, 0, 0, 0, 0};
    unsigned long long *cur_rec = nullptr;
    pdl_trigger();
    span_mark((int)pos * 3 + 1, true);
    bool waited = false;
    for (uint32_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        const uint4 td = tiles[tile];
        const ScenDev &D = table[td.x];
        if (D.ctrl == nullptr) continue;
        const uint32_t m = td.y + threadIdx.x;
        const uint4 nd = m < td.z ? D.nd_info[m] : make_uint4(0u, 0u, 0u, 0u);  // static
        // base and target are constant within a captured chunk
        unsigned long long step;
        if (!node_step(D, pos, chunk_end != 0u, step)) continue;
        if (!waited) {
            pdl_wait();
            waited = true;
        }
        unsigned long long *rec = reinterpret_cast<unsigned long long *>(stat_rec(D, step));
        if (rec != cur_rec) {
            if (cur_rec) block_flush<7, kNodeThreads>(acc, cur_rec, kField, red);
            cur_rec = rec;
        }
        if (m < td.z) node_link<TURNS>(D, m, nd, step, acc);
    }
    if (cur_rec) block_flush<7, kNodeThreads>(acc, cur_rec, kField, red);
    span_mark((int)pos * 3 + 1, false);
}

__global__ void __launch_bounds__(kNodeThreads) node_kernel(const ScenDev *__restrict__ table,
                                                            const uint4 *__restrict__ tiles,
                                                            const uint32_t *__restrict__ n_tiles_p, uint32_t pos,
                                                            uint32_t chunk_end) {
    __shared__ unsigned long long red[kNodeThreads / 32][7];
    node_pass<false>(red, table, tiles, n_tiles_p, pos, chunk_end);
}

// The same for scenarios with turn lanes or yield approaches.
__global__ void __launch_bounds__(kNodeThreads) turn_node_kernel(const ScenDev *__restrict__ table,
                                                                 const uint4 *__restrict__ tiles,
                                                                 const uint32_t *__restrict__ n_tiles_p, uint32_t pos,
                                                                 uint32_t chunk_end) {
    __shared__ unsigned long long red[kNodeThreads / 32][7];
    node_pass<true>(red, table, tiles, n_tiles_p, pos, chunk_end);
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
__global__ void __launch_bounds__(128) advance_kernel(const ScenDev *__restrict__ table, uint32_t g_max) {
    span_mark((int)g_max * 3 + 2, true);
    pdl_wait();
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
    span_mark((int)g_max * 3 + 2, false);
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

template <int TW>
static void (*link_instance(bool turns))(const ScenDev *, const LinkTile *, const uint32_t *, uint32_t, uint32_t) {
    return turns ? turn_link_kernel<TW> : link_kernel<TW>;
}

void launch_link_kernel(const ScenDev *table, const LinkTile *tiles, const uint32_t *n_tiles, uint32_t i, int grid,
                        cudaStream_t s, bool pdl, bool xfer, uint32_t tile_cap, bool turns) {
    if (tile_cap <= (uint32_t)kDefaultTileWords)
        launch_pdl(link_instance<kDefaultTileWords>(turns), grid, LinkLaunch<kDefaultTileWords>::kThreads, pdl, s,
                   table, tiles, n_tiles, i, xfer ? 1u : 0u);
    else
        launch_pdl(link_instance<kTileWords>(turns), grid, LinkLaunch<kTileWords>::kThreads, pdl, s, table, tiles,
                   n_tiles, i, xfer ? 1u : 0u);
}

void launch_node_kernel(const ScenDev *table, const uint4 *tiles, const uint32_t *n_tiles, uint32_t i, int grid,
                        cudaStream_t s, bool pdl, bool chunk_end, bool turns) {
    launch_pdl(turns ? turn_node_kernel : node_kernel, grid, kNodeThreads, pdl, s, table, tiles, n_tiles, i,
               chunk_end ? 1u : 0u);
}

void launch_advance_kernel(const ScenDev *table, uint32_t n_scen, uint32_t g, cudaStream_t s, bool pdl) {
    launch_pdl(advance_kernel, (int)n_scen, 128, pdl, s, table, g);
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
extern "C" int ts_debug_spans(unsigned long long *out, int reset) {
    if (reset) {
        unsigned long long init[128][2];
        for (int i = 0; i < 128; ++i) {
            init[i][0] = ~0ull;
            init[i][1] = 0ull;
        }
        return cudaMemcpyToSymbol(g_span, init, sizeof(init)) == cudaSuccess ? 0 : -1;
    }
    return cudaMemcpyFromSymbol(out, g_span, sizeof(unsigned long long) * 256) == cudaSuccess ? 0 : -1;
}
#endif

int max_link_blocks(uint32_t tile_cap, bool turns) {
    if (tile_cap <= (uint32_t)kDefaultTileWords) {
        // five blocks of the default instance need more shared memory than
        // the smallest L1/shared splits give
        const void *fn = (const void *)link_instance<kDefaultTileWords>(turns);
        cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, 50);
        return resident_blocks(fn, LinkLaunch<kDefaultTileWords>::kThreads);
    }
    // the large-tile instance needs more shared memory per block than the
    // default L1/shared split leaves for four blocks; the largest shared
    // share measured fastest on GB300 (config 3: 3.3e10 vs 2.4e10
    // vehicle-updates/s with the default split)
    const void *fn = (const void *)link_instance<kTileWords>(turns);
    cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, (int)cudaSharedmemCarveoutMaxShared);
    return resident_blocks(fn, LinkLaunch<kTileWords>::kThreads);
}
int max_node_blocks(bool turns) {
    return resident_blocks(turns ? (const void *)turn_node_kernel : (const void *)node_kernel, kNodeThreads);
}

}  // namespace tsim
