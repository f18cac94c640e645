// Step kernels of the TRANSIMS cellular automaton for sm_103a.
//
// One time step (Sec. 3 and Sec. 4 of Nagel & Rickert) is two launches:
//
//   link_kernel  lane change (sub-step 1), velocity update and move
//                (sub-step 2) of every vehicle on every lane, reading the
//                state of step t (buffer t&1) and writing the cells of step
//                t+1 (buffer (t+1)&1); vehicles reaching a link end enter the
//                lane's link-end buffer or arrive.
//   node_kernel  node transfer from the link-end buffers to cell 0 of the
//                next link in fixed priority order, then departures from
//                parking; the last block to finish closes the step's
//                statistics and advances the step counter.
//
// The paper's split-link boundary exchange (Sec. 4: the first five cells of
// each half are sent to the other CPU) becomes a one-column halo here: a
// block owns a tile of 32-cell columns and re-computes the lane-change
// decisions of the vehicles in the neighbouring column that can influence
// its own cells, instead of exchanging them.  Work inside a tile is one
// thread per vehicle: occupancy words are staged in shared memory and the
// vehicles are compacted into a list, so the cost follows the number of
// vehicles, not the number of cells.  Gaps come from a 64-bit funnel of two
// occupancy words and one find-first-set.
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

// splitmix64 output function (Steele, Lea, Flood 2014).
__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
    z += 0x9e3779b97f4a7c15ull;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ unsigned long long vehicle_term(uint32_t id, uint32_t link, uint32_t lane, uint32_t cell,
                                                           uint32_t v) {
    const unsigned long long a = ((unsigned long long)id << 32) | link;
    const unsigned long long b = ((unsigned long long)cell << 16) | ((unsigned long long)lane << 8) | v;
    return mix64(a ^ mix64(b));
}

// Sum of NF per-thread counters over the block, added to dst[f] once.
template <int NF, int NT>
__device__ __forceinline__ void block_flush(unsigned long long (&acc)[NF], unsigned long long *const (&dst)[NF],
                                            unsigned long long (*red)[NF]) {
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
        if (s) atomicAdd(dst[threadIdx.x], s);
    }
    __syncthreads();
}

// Exclusive prefix sum of a[0..m) in place (m <= 3 * blockDim.x); returns the total.
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t *a, int m, uint32_t *s_warp) {
    constexpr int PER = 3;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5, nw = blockDim.x >> 5;
    uint32_t v[PER], sum = 0;
#pragma unroll
    for (int q = 0; q < PER; ++q) {
        const int i = t * PER + q;
        v[q] = i < m ? a[i] : 0u;
        sum += v[q];
    }
    uint32_t inc = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) s_warp[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = lane < nw ? s_warp[lane] : 0u;
        uint32_t wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += y;
        }
        if (lane < nw) s_warp[lane] = wi - w;  // exclusive warp offsets
        if (lane == nw - 1) s_warp[31] = wi;     // total
    }
    __syncthreads();
    uint32_t run = s_warp[warp] + inc - sum;
#pragma unroll
    for (int q = 0; q < PER; ++q) {
        const int i = t * PER + q;
        if (i < m) a[i] = run;
        run += v[q];
    }
    const uint32_t total = s_warp[31];
    __syncthreads();
    return total;
}

// ------------------------------------------------------------------ link kernel

struct LinkSmem {
    uint32_t occ0[kTileSlots][kMaxLanes];  // state of step t
    uint32_t mv[kTileSlots][kMaxLanes];    // vehicles that changed INTO this lane
    uint32_t occ1[kTileSlots][kMaxLanes];  // after the lane-change sub-step
    uint32_t out[kTileSlots][kMaxLanes];   // step t+1, core columns only
    uint32_t cword[kTileSlots];            // word index of lane 0 of the column
    uint32_t cx0[kTileSlots];              // first cell of the column within its link
    int16_t right[kTileSlots], left[kTileSlots];
    uint8_t clink[kTileSlots], cncell[kTileSlots], clast[kTileSlots], ckind[kTileSlots];
    uint32_t lcells[kMaxTileCols], lbpos[kMaxTileCols], lid[kMaxTileCols], lcol0[kMaxTileCols];
    uint32_t lwbase[kMaxTileCols];
    uint8_t llanes[kMaxTileCols], lring[kMaxTileCols], lopen[kMaxTileCols];
    uint32_t wpre[kTileSlots * kMaxLanes + 4];
    uint16_t list[kListCap];
    uint32_t warp_tmp[32];
    unsigned long long red[kLinkThreads / 32][6];
    int ncore, ncols, nlinks;
};

__device__ __forceinline__ uint32_t gap_ahead(const uint32_t (*O)[kMaxLanes], const int16_t *right, int c, int k,
                                              int i, uint32_t dist, uint32_t open, uint32_t vmax) {
    const uint32_t w0 = O[c][k];
    const int r = right[c];
    const uint32_t w1 = r >= 0 ? O[r][k] : 0u;
    const unsigned long long win = (((unsigned long long)w1 << 32) | w0) >> (i + 1);
    uint32_t g = win ? (uint32_t)(__ffsll((long long)win) - 1) : 64u;
    if (g > dist) g = dist + open;
    return g < vmax ? g : vmax;
}

__device__ __forceinline__ bool room_behind(const uint32_t (*O)[kMaxLanes], const int16_t *left, int c, int k, int i,
                                            uint32_t vmax) {
    const int l = left[c];
    const unsigned long long back = ((unsigned long long)O[c][k] << 32) | (l >= 0 ? O[l][k] : 0u);
    const unsigned long long mask = ((2ull << vmax) - 1ull) << (32 + i - (int)vmax);
    return (back & mask) == 0ull;
}

__device__ __forceinline__ uint32_t lc_mask(uint8_t kind, uint32_t vmax) {
    // core: all; left halo: the last vmax cells; right halo: the first vmax cells
    return kind == 0 ? 0xFFFFFFFFu : (kind == 1 ? ~((1u << (32 - vmax)) - 1u) : ((1u << vmax) - 1u));
}

__device__ __forceinline__ uint32_t mv_mask(uint8_t kind, uint32_t vmax) {
    return kind == 0 ? 0xFFFFFFFFu : (kind == 1 ? ~((1u << (32 - vmax)) - 1u) : 0u);
}

// Fills list[] with the vehicles of rank [base, base+kListCap) among the set
// bits of masked words (word w = column w>>2, lane w&3); wpre holds the
// exclusive prefix of the per-word counts.
template <typename MaskFn>
__device__ __forceinline__ void fill_list(LinkSmem &S, int nwords, uint32_t base, MaskFn maskof) {
    for (int w = threadIdx.x; w < nwords; w += blockDim.x) {
        uint32_t m = maskof(w);
        if (!m) continue;
        const uint32_t r0 = S.wpre[w];
        const uint32_t cnt = __popc(m);
        if (r0 + cnt <= base || r0 >= base + kListCap) continue;
        uint32_t r = r0;
        while (m) {
            const int b = __ffs(m) - 1;
            m &= m - 1;
            if (r >= base && r < base + kListCap) S.list[r - base] = (uint16_t)((w << 5) | b);
            ++r;
        }
    }
}

__global__ void __launch_bounds__(kLinkThreads) link_kernel(const ScenDev *__restrict__ table,
                                                            const uint4 *__restrict__ tiles,
                                                            const WorldDev *__restrict__ wd) {
    __shared__ LinkSmem S;
    // per-thread counters: lane_changes, vehicle_updates, active, sum_v, state_hash, arrived_step
    unsigned long long acc[6] = {0, 0, 0, 0, 0, 0};
    StatRec *cur_rec = nullptr;
    const uint32_t n_tiles = wd->n_link_tiles;

    for (uint32_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        const uint4 td = tiles[tile];
        const ScenDev &D = table[td.x];
        const Ctrl *ctrl = D.ctrl;
        if (ctrl == nullptr) continue;
        const unsigned long long step = ctrl->step;
        if (step >= ctrl->target) continue;
        StatRec *rec = D.stats + (step & (kStatsRing - 1));
        if (rec != cur_rec) {
            if (cur_rec) {
                unsigned long long *const dst[6] = {&cur_rec->lane_changes, &cur_rec->vehicle_updates,
                                                    &cur_rec->active, &cur_rec->sum_v, &cur_rec->state_hash,
                                                    &cur_rec->arrived_step};
                block_flush<6, kLinkThreads>(acc, dst, S.red);
            }
            cur_rec = rec;
        }
        const uint32_t t = (uint32_t)step;
        const int cur = (int)(step & 1ull), nxt = cur ^ 1;
        const uint32_t vmax = D.vmax;
        const int d = (t & 1u) ? -1 : 1;
        const uint32_t *__restrict__ occ_in = D.occ[cur];
        const int8_t *__restrict__ vel_in = D.vel[cur];
        const uint32_t *__restrict__ vid_in = D.vid[cur];

        // ---------------- tile geometry
        const bool partial = (td.z & kPartial) != 0u;
        if (!partial) {
            const int nl = (int)td.z;
            for (int q = threadIdx.x; q < nl; q += blockDim.x) {
                const uint4 li = D.link_info[td.y + q];
                S.lcells[q] = li.y;
                S.llanes[q] = (uint8_t)(li.z & 0xFFu);
                S.lring[q] = (uint8_t)((li.z >> 8) & 1u);
                S.lbpos[q] = li.w;
                S.lid[q] = td.y + q;
                S.lwbase[q] = li.x;
                S.lcol0[q] = (li.y + 31u) >> 5;
            }
            __syncthreads();
            const uint32_t ncore = block_exclusive_scan(S.lcol0, nl, S.warp_tmp);
            for (int q = threadIdx.x; q < nl; q += blockDim.x) {
                const uint32_t cells = S.lcells[q], lanes = S.llanes[q], ring = S.lring[q];
                const int ncol = (int)((cells + 31u) >> 5), c0 = (int)S.lcol0[q];
                for (int j = 0; j < ncol; ++j) {
                    const int c = c0 + j;
                    S.cword[c] = S.lwbase[q] + (uint32_t)j * lanes;
                    S.cx0[c] = 32u * (uint32_t)j;
                    S.clink[c] = (uint8_t)q;
                    S.cncell[c] = (uint8_t)min(32u, cells - 32u * (uint32_t)j);
                    S.clast[c] = (uint8_t)(!ring && j == ncol - 1);
                    S.ckind[c] = 0;
                    S.right[c] = (int16_t)(j + 1 < ncol ? c + 1 : (ring ? c0 : -1));
                    S.left[c] = (int16_t)(j > 0 ? c - 1 : (ring ? c0 + ncol - 1 : -1));
                }
                uint8_t open = 0;
                if (!ring) {
                    const uint32_t *sx = reinterpret_cast<const uint32_t *>(D.slots + S.lbpos[q]);
                    for (uint32_t k = 0; k < lanes; ++k) open |= (uint8_t)((sx[4 * k] == kSlotEmpty) << k);
                }
                S.lopen[q] = open;
            }
            if (threadIdx.x == 0) { S.ncore = (int)ncore; S.ncols = (int)ncore; S.nlinks = nl; }
        } else {
            if (threadIdx.x == 0) {
                const uint4 li = D.link_info[td.y];
                const uint32_t cells = li.y, lanes = li.z & 0xFFu, ring = (li.z >> 8) & 1u;
                const int ncol = (int)((cells + 31u) >> 5);
                const int j0 = (int)(td.z & ~kPartial), j1 = (int)td.w;
                S.lcells[0] = cells; S.llanes[0] = (uint8_t)lanes; S.lring[0] = (uint8_t)ring;
                S.lbpos[0] = li.w; S.lid[0] = td.y; S.lwbase[0] = li.x;
                uint8_t open = 0;
                if (!ring && j1 == ncol) {
                    const uint32_t *sx = reinterpret_cast<const uint32_t *>(D.slots + li.w);
                    for (uint32_t k = 0; k < lanes; ++k) open |= (uint8_t)((sx[4 * k] == kSlotEmpty) << k);
                }
                S.lopen[0] = open;
                const int ncore = j1 - j0;
                const bool has_l = j0 > 0 || ring;
                const bool has_r = j1 < ncol || ring;
                int nc = ncore;
                const int hl = has_l ? nc++ : -1;
                const int hr = has_r ? nc++ : -1;
                for (int c = 0; c < ncore; ++c) {
                    const int j = j0 + c;
                    S.cword[c] = li.x + (uint32_t)j * lanes;
                    S.cx0[c] = 32u * (uint32_t)j;
                    S.clink[c] = 0;
                    S.cncell[c] = (uint8_t)min(32u, cells - 32u * (uint32_t)j);
                    S.clast[c] = (uint8_t)(!ring && j == ncol - 1);
                    S.ckind[c] = 0;
                    S.right[c] = (int16_t)(c + 1 < ncore ? c + 1 : hr);
                    S.left[c] = (int16_t)(c > 0 ? c - 1 : hl);
                }
                if (hl >= 0) {
                    const int j = j0 > 0 ? j0 - 1 : ncol - 1;
                    S.cword[hl] = li.x + (uint32_t)j * lanes;
                    S.cx0[hl] = 32u * (uint32_t)j;
                    S.clink[hl] = 0;
                    S.cncell[hl] = (uint8_t)min(32u, cells - 32u * (uint32_t)j);
                    S.clast[hl] = 0;
                    S.ckind[hl] = 1;
                    S.right[hl] = 0;
                    S.left[hl] = -1;
                }
                if (hr >= 0) {
                    const int j = j1 < ncol ? j1 : 0;
                    S.cword[hr] = li.x + (uint32_t)j * lanes;
                    S.cx0[hr] = 32u * (uint32_t)j;
                    S.clink[hr] = 0;
                    S.cncell[hr] = (uint8_t)min(32u, cells - 32u * (uint32_t)j);
                    S.clast[hr] = 0;
                    S.ckind[hr] = 2;
                    S.right[hr] = -1;
                    S.left[hr] = (int16_t)(ncore - 1);
                }
                S.ncore = ncore; S.ncols = nc; S.nlinks = 1;
            }
        }
        __syncthreads();
        const int ncore = S.ncore, ncols = S.ncols;
        const int nwords = ncols * kMaxLanes;

        // ---------------- stage occupancy of step t
        for (int w = threadIdx.x; w < nwords; w += blockDim.x) {
            const int c = w >> 2, k = w & 3;
            const uint32_t lanes = S.llanes[S.clink[c]];
            S.occ0[c][k] = k < (int)lanes ? occ_in[S.cword[c] + k] : 0u;
            S.mv[c][k] = 0u;
            S.out[c][k] = 0u;
        }
        __syncthreads();

        // ---------------- sub-step 1: lane changes on the state of step t
        const bool lc_on = D.lane_change != 0u;
        if (lc_on) {
            auto lcword = [&](int w) -> uint32_t {
                const int c = w >> 2, k = w & 3, kt = k + d;
                const int lanes = S.llanes[S.clink[c]];
                if (k >= lanes || kt < 0 || kt >= lanes) return 0u;
                return S.occ0[c][k] & lc_mask(S.ckind[c], vmax);
            };
            for (int w = threadIdx.x; w < nwords; w += blockDim.x) S.wpre[w] = __popc(lcword(w));
            __syncthreads();
            const uint32_t total = block_exclusive_scan(S.wpre, nwords, S.warp_tmp);
            for (uint32_t base = 0; base < total; base += kListCap) {
                fill_list(S, nwords, base, lcword);
                __syncthreads();
                const uint32_t n = min((uint32_t)kListCap, total - base);
                for (uint32_t e = threadIdx.x; e < n; e += blockDim.x) {
                    const uint32_t code = S.list[e];
                    const int i = code & 31, w = code >> 5, c = w >> 2, k = w & 3, kt = k + d;
                    const int q = S.clink[c];
                    const uint32_t ring = S.lring[q];
                    const uint32_t x = S.cx0[c] + (uint32_t)i;
                    const uint32_t dist = ring ? 0xFFFFu : S.lcells[q] - 1u - x;
                    const size_t p = (size_t)(S.cword[c] + (uint32_t)k) * 32u + (uint32_t)i;
                    const uint32_t v = (uint32_t)vel_in[p];
                    uint32_t last = 0u;
                    if (dist < vmax) last = vid_in[p] >> 31;
                    const uint32_t open_own = ((S.lopen[q] >> k) & 1u) | last;
                    const uint32_t open_tgt = ((S.lopen[q] >> kt) & 1u) | last;
                    const uint32_t g_own = gap_ahead(S.occ0, S.right, c, k, i, dist, open_own, vmax);
                    const uint32_t want = v + 1u < vmax ? v + 1u : vmax;
                    if (g_own < want) {
                        const uint32_t g_tgt = gap_ahead(S.occ0, S.right, c, kt, i, dist, open_tgt, vmax);
                        if (g_tgt > g_own && room_behind(S.occ0, S.left, c, kt, i, vmax)) {
                            atomicOr(&S.mv[c][kt], 1u << i);
                            if (S.ckind[c] == 0) acc[0] += 1;
                        }
                    }
                }
                __syncthreads();
            }
            for (int w = threadIdx.x; w < nwords; w += blockDim.x) {
                const int c = w >> 2, k = w & 3, kf = k + d;
                const uint32_t leaving = (kf >= 0 && kf < kMaxLanes) ? S.mv[c][kf] : 0u;
                S.occ1[c][k] = (S.occ0[c][k] & ~leaving) | S.mv[c][k];
            }
        } else {
            for (int w = threadIdx.x; w < nwords; w += blockDim.x) S.occ1[w >> 2][w & 3] = S.occ0[w >> 2][w & 3];
        }
        __syncthreads();

        // ---------------- sub-step 2: velocity update and move
        {
            auto mvword = [&](int w) -> uint32_t {
                const int c = w >> 2, k = w & 3;
                return S.occ1[c][k] & mv_mask(S.ckind[c], vmax);
            };
            for (int w = threadIdx.x; w < nwords; w += blockDim.x) S.wpre[w] = __popc(mvword(w));
            __syncthreads();
            const uint32_t total = block_exclusive_scan(S.wpre, nwords, S.warp_tmp);
            int8_t *__restrict__ vel_out = D.vel[nxt];
            uint32_t *__restrict__ vid_out = D.vid[nxt];
            const uint32_t key0 = D.seed_lo, key1 = D.seed_hi, pthr = D.p_threshold;
            for (uint32_t base = 0; base < total; base += kListCap) {
                fill_list(S, nwords, base, mvword);
                __syncthreads();
                const uint32_t n = min((uint32_t)kListCap, total - base);
                for (uint32_t e = threadIdx.x; e < n; e += blockDim.x) {
                    const uint32_t code = S.list[e];
                    const int i = code & 31, w = code >> 5, c = w >> 2, k = w & 3;
                    const int q = S.clink[c];
                    const int ks = (lc_on && ((S.mv[c][k] >> i) & 1u)) ? k - d : k;
                    const size_t p = (size_t)(S.cword[c] + (uint32_t)ks) * 32u + (uint32_t)i;
                    const uint32_t v0 = (uint32_t)vel_in[p];
                    const uint32_t idw = vid_in[p];
                    const uint32_t id = idw & kIdMask, last = idw >> 31;
                    const uint32_t ring = S.lring[q];
                    const uint32_t x = S.cx0[c] + (uint32_t)i;
                    const uint32_t dist = ring ? 0xFFFFu : S.lcells[q] - 1u - x;
                    const uint32_t open = ((S.lopen[q] >> k) & 1u) | last;
                    uint32_t v = v0 + 1u < vmax ? v0 + 1u : vmax;                            // (i)
                    const uint32_t g = gap_ahead(S.occ1, S.right, c, k, i, dist, open, vmax);
                    if (v > g) v = g;                                                         // (ii)
                    if (v > 0u && philox_word0(t, id, key0, key1) < pthr) v -= 1u;           // (iii)
                    const bool core = S.ckind[c] == 0;
                    if (core) acc[1] += 1;
                    int ni = i + (int)v;
                    if (!ring && x + v >= S.lcells[q]) {
                        // reaches the link end (only possible for a vehicle owned by
                        // this tile: a split leaves more than 2*vmax cells after it)
                        if (!core) {
                            atomicOr(&D.ctrl->error, kErrCellTaken);
                        } else if (last) {
                            acc[5] += 1;  // leaves to parking
                        } else {
                            const uint32_t s = S.lbpos[q] + (uint32_t)k;
                            const uint2 ve = D.veh[id];
                            if (ve.x + 1u >= ve.y) {
                                atomicOr(&D.ctrl->error, kErrRoute);
                            } else {
                                const uint32_t m = D.route_links[ve.x + 1u];
                                const uint32_t fl = (ve.x + 2u == ve.y) ? kLastLinkBit : 0u;
                                uint32_t *sx = reinterpret_cast<uint32_t *>(D.slots + s);
                                if (*sx != kSlotEmpty) atomicOr(&D.ctrl->error, kErrSlotTaken);
                                D.slots[s] = make_uint4(id | fl, m, S.lid[q], v | ((uint32_t)k << 8));
                            }
                        }
                    } else {
                        int dc = c;
                        if (ni >= 32) { dc = S.right[c]; ni -= 32; }
                        if (dc < 0) {
                            atomicOr(&D.ctrl->error, kErrCellTaken);
                        } else if (S.ckind[dc] == 0) {
                            const size_t pd = (size_t)(S.cword[dc] + (uint32_t)k) * 32u + (uint32_t)ni;
                            vel_out[pd] = (int8_t)v;
                            vid_out[pd] = idw;
                            const uint32_t old = atomicOr(&S.out[dc][k], 1u << ni);
                            if (old & (1u << ni)) atomicOr(&D.ctrl->error, kErrCellTaken);
                            acc[2] += 1;
                            acc[3] += v;
                            acc[4] += vehicle_term(id, S.lid[q], (uint32_t)k, S.cx0[dc] + (uint32_t)ni, v);
                        }
                    }
                }
                __syncthreads();
            }
        }

        // ---------------- write the occupancy of step t+1 for the core columns
        {
            uint32_t *__restrict__ occ_out = D.occ[nxt];
            for (int w = threadIdx.x; w < ncore * kMaxLanes; w += blockDim.x) {
                const int c = w >> 2, k = w & 3;
                if (k < (int)S.llanes[S.clink[c]]) occ_out[S.cword[c] + k] = S.out[c][k];
            }
        }
        __syncthreads();
    }
    if (cur_rec) {
        unsigned long long *const dst[6] = {&cur_rec->lane_changes, &cur_rec->vehicle_updates, &cur_rec->active,
                                            &cur_rec->sum_v, &cur_rec->state_hash, &cur_rec->arrived_step};
        block_flush<6, kLinkThreads>(acc, dst, S.red);
    }
}

// ------------------------------------------------------------------ node kernel

__global__ void __launch_bounds__(kNodeThreads) node_kernel(const ScenDev *__restrict__ table,
                                                            const uint4 *__restrict__ tiles, WorldDev *wd) {
    __shared__ unsigned long long red[kNodeThreads / 32][6];
    __shared__ bool am_last;
    // transfers, inserted, buffered, active, sum_v, state_hash
    unsigned long long acc[6] = {0, 0, 0, 0, 0, 0};
    StatRec *cur_rec = nullptr;
    const uint32_t n_tiles = wd->n_node_tiles;
    for (uint32_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        const uint4 td = tiles[tile];
        const ScenDev &D = table[td.x];
        if (D.ctrl == nullptr) continue;
        const unsigned long long step = D.ctrl->step;
        if (step >= D.ctrl->target) continue;
        StatRec *rec = D.stats + (step & (kStatsRing - 1));
        if (rec != cur_rec) {
            if (cur_rec) {
                unsigned long long *const dst[6] = {&cur_rec->transfers, &cur_rec->inserted, &cur_rec->buffered,
                                                    &cur_rec->active, &cur_rec->sum_v, &cur_rec->state_hash};
                block_flush<6, kNodeThreads>(acc, dst, red);
            }
            cur_rec = rec;
        }
        const uint32_t t = (uint32_t)step;
        const int nxt = (int)((step + 1ull) & 1ull);
        uint32_t *occ = D.occ[nxt];
        int8_t *vel = D.vel[nxt];
        uint32_t *vid = D.vid[nxt];
        const uint32_t n = td.y + threadIdx.x;
        if (n < td.z) {
            // node transfer, priority = slot order (incoming link id, then lane)
            const uint32_t s_end = D.node_in_off[n + 1];
            for (uint32_t s = D.node_in_off[n]; s < s_end; ++s) {
                const uint4 sl = D.slots[s];
                if (sl.x == kSlotEmpty) continue;
                const uint32_t id = sl.x & kIdMask, m = sl.y, l = sl.z;
                const uint32_t v = sl.w & 0xFFu, ks = (sl.w >> 8) & 0xFFu;
                const uint4 mi = D.link_info[m];
                const uint32_t lanes = mi.z & 0xFFu;
                const uint32_t pref = ks < lanes - 1u ? ks : lanes - 1u;
                bool placed = false;
                for (uint32_t tr = 0; tr < lanes; ++tr) {
                    const uint32_t qn = tr == 0 ? pref : (tr - 1u < pref ? tr - 1u : tr);
                    const uint32_t w = mi.x + qn;  // column 0, lane qn
                    const uint32_t o = occ[w];
                    if (!(o & 1u)) {
                        occ[w] = o | 1u;
                        vel[(size_t)w * 32u] = (int8_t)v;
                        vid[(size_t)w * 32u] = sl.x;  // id with the last-link flag of the next link
                        D.veh[id].x += 1u;
                        D.slots[s].x = kSlotEmpty;
                        acc[0] += 1; acc[3] += 1; acc[4] += v;
                        acc[5] += vehicle_term(id, m, qn, 0u, v);
                        placed = true;
                        break;
                    }
                }
                if (!placed) {
                    acc[2] += 1;
                    acc[5] += vehicle_term(id, l, ks, D.link_info[l].y, v);
                }
            }
            // departures from parking onto the links leaving this node
            const uint32_t a_end = D.node_out_off[n + 1];
            for (uint32_t a = D.node_out_off[n]; a < a_end; ++a) {
                const uint32_t m = D.node_out_link[a];
                uint32_t h = D.dep_head[m];
                const uint32_t e = D.dep_off[m + 1];
                if (h >= e || D.dep_steps[h] > t) continue;
                const uint4 mi = D.link_info[m];
                const uint32_t lanes = mi.z & 0xFFu;
                while (h < e && D.dep_steps[h] <= t) {
                    uint32_t qn = 0;
                    for (; qn < lanes; ++qn)
                        if (!(occ[mi.x + qn] & 1u)) break;
                    if (qn == lanes) break;
                    const uint32_t id = D.dep_ids[h];
                    const uint2 ve = D.veh[id];
                    const uint32_t w = mi.x + qn;
                    occ[w] |= 1u;
                    vel[(size_t)w * 32u] = 0;
                    vid[(size_t)w * 32u] = id | ((ve.x + 1u == ve.y) ? kLastLinkBit : 0u);
                    acc[1] += 1; acc[3] += 1;
                    acc[5] += vehicle_term(id, m, qn, 0u, 0u);
                    ++h;
                }
                D.dep_head[m] = h;
            }
        }
    }
    if (cur_rec) {
        unsigned long long *const dst[6] = {&cur_rec->transfers, &cur_rec->inserted, &cur_rec->buffered,
                                            &cur_rec->active, &cur_rec->sum_v, &cur_rec->state_hash};
        block_flush<6, kNodeThreads>(acc, dst, red);
    }
    // The last block to finish closes the step of every active scenario.
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned int tk = atomicAdd(&wd->ticket, 1u);
        am_last = (tk == gridDim.x - 1u);
    }
    __syncthreads();
    if (!am_last) return;
    __threadfence();
    const uint32_t n_scen = wd->n_scen;
    for (uint32_t s = threadIdx.x; s < n_scen; s += blockDim.x) {
        const ScenDev &D = table[s];
        Ctrl *c = D.ctrl;
        if (c == nullptr) continue;
        const unsigned long long step = __ldcg(&c->step);
        if (step >= __ldcg(&c->target)) continue;
        StatRec *r = D.stats + (step & (kStatsRing - 1));
        const unsigned long long arrived = __ldcg(&c->arrived) + __ldcg(&r->arrived_step);
        const unsigned long long inserted = __ldcg(&c->inserted) + __ldcg(&r->inserted);
        unsigned long long departed = 0;
        if (D.n_dep_steps) departed = D.departed_upto[step < D.n_dep_steps ? step : D.n_dep_steps - 1];
        r->step = step;
        r->arrived = arrived;
        r->waiting = departed - inserted;
        c->arrived = arrived;
        c->inserted = inserted;
        StatRec *nr = D.stats + ((step + 1ull) & (kStatsRing - 1));
        unsigned long long *z = reinterpret_cast<unsigned long long *>(nr);
        for (int f = 0; f < (int)(sizeof(StatRec) / 8); ++f) z[f] = 0ull;
        c->step = step + 1ull;
    }
    if (threadIdx.x == 0) wd->ticket = 0u;
}

__global__ void set_target_kernel(Ctrl *ctrl, unsigned long long target) { ctrl->target = target; }

void launch_link_kernel(const ScenDev *table, const uint4 *tiles, WorldDev *wd, int grid, cudaStream_t s) {
    link_kernel<<<grid, kLinkThreads, 0, s>>>(table, tiles, wd);
}

void launch_node_kernel(const ScenDev *table, const uint4 *tiles, WorldDev *wd, int grid, cudaStream_t s) {
    node_kernel<<<grid, kNodeThreads, 0, s>>>(table, tiles, wd);
}

void launch_set_target(Ctrl *ctrl, unsigned long long target, cudaStream_t s) {
    set_target_kernel<<<1, 1, 0, s>>>(ctrl, target);
}

static int blocks_per_sm(const void *fn, int threads) {
    int dev = 0, n = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, threads, 0);
    return (n > 0 ? n : 1) * (sms > 0 ? sms : 1);
}

int max_link_blocks() { return blocks_per_sm((const void *)link_kernel, kLinkThreads); }
int max_node_blocks() { return blocks_per_sm((const void *)node_kernel, kNodeThreads); }

}  // namespace tsim
