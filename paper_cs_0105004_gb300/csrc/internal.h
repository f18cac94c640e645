// Device-side layout shared by the step kernels and the host API.
//
// Data layout of one scenario in HBM (all arrays owned by its ts_ctx):
//   * A lane of link l is stored as ceil(cells/32) 32-cell columns.  Word
//     (l, column j, lane k) is word index wbase[l] + j*lanes[l] + k, so the
//     lanes of one column are adjacent and a link's columns are contiguous
//     (link-major, lane-interleaved).  Bit i of that word is cell 32j+i.
//   * occ[2][n_words]: occupancy bitmasks, double-buffered by step parity
//     (state at step t lives in buffer t&1).
//   * vel[2][32*n_words] (int8) and vid[2][32*n_words] (uint32): velocity and
//     vehicle id of the cell with the same bit index; vid bit 31 marks a
//     vehicle driving the last link of its route.  Payload of empty cells is
//     never read.
//   * slots[n_slots]: one link-end buffer per lane, grouped by the node the
//     link ends at (node_in_off), in priority order (link id, then lane).
//     x = id | last-link-next flag << 31 (0xffffffff = empty), y = next link,
//     z = current link, w = v | lane << 8.
//   * veh[n_vehicles]: {absolute index of the current route entry, end of the
//     vehicle's route}.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace tsim {

constexpr int kMaxLanes = 4;
constexpr int kMaxVmax = 15;
constexpr uint32_t kSlotEmpty = 0xFFFFFFFFu;
constexpr uint32_t kLastLinkBit = 0x80000000u;
constexpr uint32_t kIdMask = 0x7FFFFFFFu;
constexpr int kMaxTileCols = 129;          // columns of a link tile (128 + one merged tail column)
constexpr int kTileSlots = kMaxTileCols + 2;  // plus a halo column on each side
constexpr int kLinkThreads = 256;
constexpr int kNodeThreads = 128;
constexpr int kListCap = 4096;             // vehicles staged per round in shared memory
constexpr uint32_t kStatsRing = 4096;      // per-step statistics kept on the device
constexpr uint32_t kNoNode = 0xFFFFFFFFu;

struct Ctrl {
    unsigned long long step;      // next step to run
    unsigned long long target;    // run while step < target
    unsigned long long arrived;   // cumulative arrivals
    unsigned long long inserted;  // cumulative departures inserted
    unsigned int error;           // device-check flags (bitwise or)
    unsigned int pad;
};

// error flags
constexpr unsigned kErrCellTaken = 1u;   // two vehicles for one cell
constexpr unsigned kErrSlotTaken = 2u;   // buffer entry into an occupied buffer
constexpr unsigned kErrRoute = 4u;       // route cursor past the route end
constexpr unsigned kErrListCap = 8u;     // internal: list round bookkeeping

struct StatRec {
    unsigned long long step, active, buffered, waiting, arrived, lane_changes, transfers, inserted, sum_v,
        vehicle_updates, state_hash, arrived_step;
};

struct ScenDev {
    const uint4 *link_info;       // x wbase, y cells, z lanes | ring << 8, w first slot (bpos)
    const uint32_t *node_in_off;  // [n_nodes_total + 1] slot ranges per node
    const uint32_t *node_out_off; // [n_nodes_total + 1]
    const uint32_t *node_out_link;
    uint32_t *occ[2];
    int8_t *vel[2];
    uint32_t *vid[2];
    uint4 *slots;
    uint2 *veh;
    const uint32_t *route_links;
    const uint32_t *dep_off;      // [n_links + 1]
    const uint32_t *dep_ids;
    const uint32_t *dep_steps;
    uint32_t *dep_head;           // [n_links] absolute queue index
    const uint32_t *departed_upto;
    uint32_t n_dep_steps;
    Ctrl *ctrl;                   // nullptr marks an unused table entry
    StatRec *stats;               // [kStatsRing]
    uint32_t vmax, p_threshold, seed_lo, seed_hi, lane_change;
    uint32_t n_links, n_nodes_total;
};

struct WorldDev {
    unsigned int ticket;
    unsigned int n_link_tiles;
    unsigned int n_node_tiles;
    unsigned int n_scen;
};

// link tile: x scenario slot, y first link, z link count (whole links) or
// kPartial | first column (one link), w end column (partial tiles)
constexpr uint32_t kPartial = 0x80000000u;

void launch_link_kernel(const ScenDev *table, const uint4 *tiles, WorldDev *wd, int grid, cudaStream_t s);
void launch_node_kernel(const ScenDev *table, const uint4 *tiles, WorldDev *wd, int grid, cudaStream_t s);
void launch_set_target(Ctrl *ctrl, unsigned long long target, cudaStream_t s);
int max_link_blocks();
int max_node_blocks();

}  // namespace tsim
