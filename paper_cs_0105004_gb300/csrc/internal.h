// Device-side layout shared by the step kernels and the host API.
//
// Data layout of one scenario in HBM (all arrays owned by its ts_ctx):
//   * A lane of link l is stored as ceil(cells/32) 32-cell columns.  Word
//     (l, column j, lane k) is word index wbase[l] + j*lanes[l] + k, so the
//     lanes of one column are adjacent and a link's columns are contiguous
//     (link-major, lane-interleaved).  Bit i of that word is cell 32j+i.
//   * occ[2][n_words]: occupancy bitmasks, double-buffered by step parity
//     (the state at step t lives in occ[t&1]); mov[2][n_words]: bit set when
//     the vehicle in that cell has v > 0; loc[2][n_words]: which of the two
//     payload buffers holds the vehicle's velocity and id.
//   * vel[2][32*n_words] (int8) and vid[2][32*n_words] (uint32): the two
//     payload buffers, velocity and vehicle id of the cell with the same bit
//     index; vid bit 31 marks a vehicle driving the last link of its route.
//     A vehicle that stays where it is with v = 0 keeps its payload where it
//     is; a vehicle that moves or changes speed writes the buffer that no
//     reader of the step can be using (the other one than the cell's current
//     occupant's).  Payload of empty cells is never read.  With a turn table
//     (plan-following lane changes) the velocity byte is v | A << 4, A the
//     lanes of the current link from which the vehicle may take its next
//     turn (0: any lane).
//   * slots[2][n_slots]: one link-end buffer per lane, grouped by the node
//     the link ends at, in intersection priority order (priority approaches
//     before yield approaches, then link id, then lane):
//     x = id | next-link-is-last << 31 (0xffffffff = empty), y = next link,
//     z = current link, w = v | A << 4 | lane << 8 | current link cells << 10
//     (A: the allowed lanes on the next link, as in the velocity byte).
//     Double-buffered by step parity like the cells: a step reads
//     slots[t&1] (which every tile may read to resolve node transfers) and
//     each tile writes its own links' buffers into slots[(t+1)&1].
//   * veh[n_vehicles]: {absolute index of the current route entry, end of the
//     vehicle's route}; enter_step[n_vehicles]: the step at whose end it
//     entered its current link (departure or node transfer), kNotOnLink
//     before departure and after arrival.
//   * link_time[n_links]: per link, in one 64-bit word updated by one
//     atomic per event, the number of completed traversals times 2^40 plus
//     the exit steps of completed traversals minus the entry steps of all
//     traversals begun (mod 2^64); ts_read_link_times adds back the entry
//     steps of the vehicles still on each link, which leaves count << 40 |
//     travel-time sum, the input of re-planning between relaxation
//     iterations.  Neither the entry nor the exit reads any per-vehicle
//     value.  Between resets a link's sum stays below 2^40 and its count
//     below 2^24.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace tsim {

constexpr int kMaxLanes = 4;
constexpr int kMaxVmax = 15;
constexpr uint32_t kSlotEmpty = 0xFFFFFFFFu;
constexpr uint32_t kLastLinkBit = 0x80000000u;
constexpr uint32_t kIdMask = 0x7FFFFFFFu;
constexpr uint32_t kMaxCells = 1u << 22;      // cells per link (buffer digest packs 22 bits)
constexpr int kTileWords = 256;               // tile_words setting: at most
constexpr int kDefaultTileWords = 128;        // default: occupancy words (columns x lanes) per warp tile
constexpr int kWarpTileCols = 30;             // columns per warp tile (lanes 1..30; lanes 0, 31: halos)
constexpr int kLinkWarpsPerBlock = 4;         // warps of one link-kernel block
constexpr int kNodeThreads = 128;
constexpr uint32_t kStatsRing = 4096;         // steps of statistics kept on the device
constexpr uint32_t kChunk = 32;               // steps per captured graph
constexpr uint32_t kNoLink = 0xFFFFFFFFu;
constexpr uint32_t kNotOnLink = 0xFFFFFFFFu;  // enter_step of a vehicle not (or no longer) on the network
constexpr unsigned long long kLinkTimeOne = 1ull << 40;  // one completed traversal in link_time

struct Ctrl {
    unsigned long long base;      // steps completed (first step of the next chunk)
    unsigned long long target;    // run while step < target
    // values of the state at `base` (statistics of earlier steps are rebuilt
    // from these and the per-step changes)
    unsigned long long arrived;   // cumulative arrivals
    unsigned long long inserted;  // cumulative departures inserted
    unsigned long long active;    // vehicles in cells
    unsigned long long buffered;  // vehicles in link-end buffers
    unsigned long long sum_v;     // sum of velocities of vehicles in cells
    unsigned long long hash;      // state digest
    unsigned long long tot_updates, tot_lane_changes, tot_transfers;  // since the last reset
    unsigned long long tot_moving, tot_active;  // per-step counts summed since the last reset
    unsigned long long steps_run;
    unsigned int error;  // device-check flags (bitwise or)
    unsigned int pad;
};

// error flags
constexpr unsigned kErrCellTaken = 1u;  // two vehicles for one cell
constexpr unsigned kErrSlotTaken = 2u;  // buffer entry into an occupied buffer
constexpr unsigned kErrRoute = 4u;      // route cursor past the route end
constexpr unsigned kErrGeometry = 8u;   // a vehicle left the tile geometry
constexpr unsigned kErrInstance = 16u;  // a tile's scenario does not fit the kernel instance launched

// One statistics sub-record per step; n_sub of them per step, each on its own
// 128-byte line, so that block flushes spread over L2 slices.  Counts of the
// step, and the changes (modulo 2^64) of the state's running values.
struct StatRec {
    unsigned long long vehicle_updates, lane_changes, transfers, inserted, arrived, d_active, d_buffered, d_sum_v,
        d_hash, moving;
    unsigned long long pad[6];
};
enum StatField {
    kUpdates = 0, kLaneChanges, kTransfers, kInserted, kArrived, kDActive, kDBuffered, kDSumV, kDHash, kMoving,
    kStatFields
};
static_assert(sizeof(StatRec) == 128, "StatRec is one line");

struct ScenDev {
    const uint4 *lk_info;         // x wbase, y cells, z lanes | ring << 8, w slot base
    const uint4 *col_info;        // per column (link-major, then j): x word of lane 0, y link,
                                  // z j | lanes << 20 | ring << 23, w link cells
    const uint4 *col_aux;         // per column: x first link-end buffer of its link, y z its signal, w 0
    uint32_t n_cols;
    const uint4 *nd_info;         // per link m: x first slot of from(m), y wbase, z slot count | lanes << 8 |
                                  // priority slots << 16, w dep end
    const uint2 *sig_info;        // per link: signal cycle | green << 16, offset (nullptr: no signals)
    uint32_t *occ[2];
    uint32_t *mov[2];
    uint32_t *loc[2];
    int8_t *vel[2];
    uint32_t *vid[2];
    uint4 *slots[2];
    uint2 *veh;
    uint32_t *enter_step;         // [n_vehicles] step at whose end the vehicle entered its current link
    unsigned long long *link_time;  // [n_links] traversal count << 40 | travel-time sum (before correction)
    const uint32_t *route_links;
    const uint32_t *dep_ids;      // id | last-link flag << 31, queue order
    const uint32_t *dep_steps;
    uint2 *dep_head;              // [n_links] absolute queue index of the head, its departure step (~0: none left)
    Ctrl *ctrl;                   // nullptr marks an unused table entry
    StatRec *stats;               // [kStatsRing * n_sub]
    uint32_t n_sub;               // sub-records per step (power of two)
    uint32_t vmax, p_threshold, seed_lo, seed_hi, lane_change;
    uint32_t n_links;
    // turn table (nullptr: none): per route entry, the lanes of that link from
    // which the turn onto the route's next link may be taken (bit k = lane k;
    // 0 = any lane, and on the route's last entry); per departure-queue entry,
    // the same for the traveller's first link
    const uint8_t *route_turn;
    const uint8_t *dep_turn;
    // gap acceptance (nullptr: none): per slot the acceptance gap G of its
    // link (0: a priority approach), and {word of the lane's last column,
    // link cells | lanes << 24 | acceptance gap << 27}; a node's priority slots come first, their
    // count in nd_info z bits 16..23
    const uint8_t *slot_gap;
    const uint2 *slot_tail;
};

// warp tile (uint2): x = scenario | (columns - 1) << 24, y = first column;
// up to 32 consecutive columns of the scenario's col_info order
// node tile: {scen, first link, end link, 0}

// pdl: launch with programmatic stream serialization (overlaps this launch
// with the tail of the previous kernel in the stream)
// n_tiles points to the tile count in device memory; it may change between
// graph launches (load balancing) without a new capture
// xfer: the launch first completes the node transfers and departures of the
// previous step (the step at position i-1 of the chunk); without it, the
// previous step must have been completed by node_kernel
// turns: some scenario of the table has turn lanes (plan-following lane
// changes) or yield approaches (gap acceptance); picks the instances that
// apply those rules
// span: kernel-span buffer (nullptr: no timing), see kSpanWords
// grid: blocks of kLinkWarpsPerBlock warps; each warp takes the tiles warp,
// warp + all warps, ... or, with tile_ctr (kChunk counters, one per chunk
// position, zero at the chunk's start) and more than two tiles per warp,
// after its first two 2 * all warps + the next value it claims from
// tile_ctr[i]
// vmax5: every scenario of the table has vmax = 5 (the paper's value): picks
// the instances compiled for that constant (a scenario that does not is
// flagged, not stepped)
void launch_link_kernel(const ScenDev *table, const uint2 *tiles, const uint32_t *n_tiles, uint32_t i, int grid,
                        cudaStream_t s, bool pdl, bool xfer, bool turns, unsigned long long *span = nullptr,
                        bool vmax5 = false, uint32_t *tile_ctr = nullptr);
// chunk_end: the pass completes the last step each scenario ran in the
// chunk (after fused steps); else step i of the chunk only
void launch_node_kernel(const ScenDev *table, const uint4 *tiles, const uint32_t *n_tiles, uint32_t i, int grid,
                        cudaStream_t s, bool pdl, bool chunk_end, bool turns, unsigned long long *span = nullptr);
// tile_ctr: the link kernels' claim counters (kChunk), zeroed for the next chunk
void launch_advance_kernel(const ScenDev *table, uint32_t n_scen, uint32_t g, cudaStream_t s, bool pdl,
                           unsigned long long *span = nullptr, uint32_t *tile_ctr = nullptr);
// Kernel-span buffer: per chunk position and kind (link, node) the launch's
// first block entry and last block exit on %globaltimer, then per kind the
// sum of launch durations (ns) and the launch count.
constexpr uint32_t kSpanWords = kChunk * 4u + 4u;
void launch_set_target(Ctrl *ctrl, unsigned long long target, cudaStream_t s);
// Re-tiling on the device: the n_base static tiles of base, cut where
// cut_ok[b] allows so that a tile holds at most vt vehicles of the current
// state, written to out; *count (zeroed by the caller) becomes the tile count.
void launch_retile(const ScenDev *table, const uint2 *base, const uint32_t *cut_ok, uint32_t n_base, uint32_t vt,
                   uint2 *out, uint32_t *count, cudaStream_t s);
// adds the entry steps of vehicles on the network to out (a copy of link_time)
void launch_link_time_fix(const ScenDev &sd, uint32_t n_veh, unsigned long long *out, cudaStream_t s);
// out[i] = word 0 of Philox-4x32-10, counter (c0[i], c1[i], 0, 0), key
// (k0, k1): the slowdown draw of the link kernel (device arrays of n)
void launch_philox_words(const uint32_t *c0, const uint32_t *c1, uint32_t k0, uint32_t k1, uint32_t n,
                         uint32_t *out, cudaStream_t s);
int max_link_blocks(bool turns);
int max_node_blocks(bool turns);
// Sets the thread-local message returned by ts_last_error.
void set_last_error(const char *msg);

// splitmix64 output function (Steele, Lea, Flood 2014).
__host__ __device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
    z += 0x9e3779b97f4a7c15ull;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

// Digest term of one vehicle: the state digest is the sum (mod 2^64) of this
// over all vehicles in cells and buffers (a buffered vehicle has cell = link
// cells).
__host__ __device__ __forceinline__ unsigned long long vehicle_term(uint32_t id, uint32_t link, uint32_t lane,
                                                                    uint32_t cell, uint32_t v) {
    const unsigned long long a = ((unsigned long long)id << 32) | link;
    const unsigned long long b = ((unsigned long long)cell << 16) | ((unsigned long long)lane << 8) | v;
    return mix64(a ^ mix64(b));
}

}  // namespace tsim
