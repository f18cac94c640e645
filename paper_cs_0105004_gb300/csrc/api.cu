// Host side of the C ABI declared in include/transsim.h: input validation,
// device layout, CUDA-graph stepping, batching and state conversion.
#include <algorithm>
#include <chrono>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "internal.h"
#include "transsim.h"

using namespace tsim;

namespace {

thread_local std::string g_err;

ts_status fail(ts_status s, const std::string &msg) {
    g_err = msg;
    return s;
}

ts_status cuda_fail(cudaError_t e, const char *what) {
    return fail(TS_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define CK(call)                                            \
    do {                                                    \
        cudaError_t e_ = (call);                            \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
    } while (0)

// Polls an event until it completes or the deadline passes.
ts_status wait_event(cudaEvent_t ev, uint32_t timeout_ms) {
    const auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        const cudaError_t e = cudaEventQuery(ev);
        if (e == cudaSuccess) return TS_OK;
        if (e != cudaErrorNotReady) return cuda_fail(e, "cudaEventQuery");
        const auto ms =
            std::chrono::duration_cast<std::chrono::milliseconds>(std::chrono::steady_clock::now() - t0).count();
        if ((uint64_t)ms >= timeout_ms) return fail(TS_ERR_TIMEOUT, "timed out waiting for the device");
        std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
}

// Waits (at most timeout_ms) for the work queued on s so far.
constexpr uint32_t kHostWaitMs = 300000;  // internal waits of the library's own calls
ts_status sync_stream(cudaStream_t s, uint32_t timeout_ms = kHostWaitMs) {
    cudaEvent_t ev;
    CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    cudaError_t e = cudaEventRecord(ev, s);
    ts_status st = e == cudaSuccess ? wait_event(ev, timeout_ms) : cuda_fail(e, "cudaEventRecord");
    cudaEventDestroy(ev);
    return st;
}

}  // namespace

void tsim::set_last_error(const char *msg) { g_err = msg; }


// ------------------------------------------------------------------ world (scenarios stepped together)

struct World {
    int device = 0;
    cudaStream_t cap_stream = nullptr;  // used only for graph capture
    uint32_t capacity = 0;
    std::vector<ts_ctx *> members;      // slot -> context
    ScenDev *d_table = nullptr;
    uint2 *d_link_tiles = nullptr;
    uint4 *d_node_tiles = nullptr;
    uint32_t *d_counts = nullptr;  // [0] link tiles, [1] node tiles, read by the kernels; then the link
                                   // kernels' tile claim counters, one per chunk position
    size_t link_cap = 0, node_cap = 0;
    uint32_t n_link_tiles = 0, n_node_tiles = 0;
    int grid_l = 1, grid_n = 1, grid_cap = 0;
    bool turns = false;  // some member has turn lanes or yield approaches (picks the turn instances)
    bool vmax5 = false;  // every member has vmax = 5 (picks the instances compiled for it)
    uint32_t mode = TS_STEP_AUTO;  // fused or split steps (ts_set_step_mode)
    uint32_t link_blocks_per_sm = 0;  // cap on the link kernel's grid per SM (0: every resident block)
    std::map<uint32_t, cudaGraphExec_t> graphs;  // by chunk length | fused << 16
    unsigned long long *d_span = nullptr;  // kernel spans (kSpanWords), allocated on first use
    bool timing = false;                   // launches record their spans (ts_set_kernel_timing)
    bool fused() const;
    ~World();
    ts_status init(uint32_t cap);
    ts_status rebuild();
    ts_status run(uint32_t n, cudaStream_t s);
    void drop_graphs();
};

struct ts_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    cudaEvent_t ev = nullptr;
    ts_allocator alloc{};
    bool has_alloc = false;
    ts_params params{};
    // network (host copies)
    uint32_t n_nodes = 0, n_links = 0, n_ring = 0;
    std::vector<uint32_t> from, to, cells, lanes, ncols, wbase, bpos, lane_base, col_base;
    std::vector<uint32_t> sig_cycle_green, sig_offset;  // per link: cycle | green << 16, offset (0: no signal)
    std::vector<uint8_t> ring;
    std::vector<uint64_t> cell_base;
    std::vector<uint32_t> node_in_off;
    // turn table (plan-following lane changes): per link, entries for the
    // links leaving its end node (out_link[out_off[n]..], ascending id)
    bool has_turn = false;
    std::vector<uint8_t> turn;
    std::vector<uint8_t> gap_accept;       // acceptance gap per link (empty: every approach has priority)
    std::vector<uint32_t> node_prio;       // per node: slots of its priority approaches (they come first)
    std::vector<uint32_t> turn_off, out_off, out_link;
    uint32_t n_words = 0, n_slots = 0, n_lanes = 0;
    uint64_t n_lane_cells = 0;
    uint32_t tile_words = kDefaultTileWords;
    std::vector<uint2> link_tiles;     // warp tiles (scenario index 0)
    std::vector<uint32_t> tile_cuts;   // per tile: bit t set = it may be cut before its column t
    uint32_t n_cols = 0;
    uint2 *d_base_tiles = nullptr;     // the static tiles and their cut masks, for re-tiling on the device
    uint32_t *d_cut_ok = nullptr;
    size_t base_cap = 0;
    std::vector<uint4> node_tiles;
    uint32_t n_sub = 1;                // statistics sub-records per step (fixed at creation)
    uint32_t tile_vehicles = 1024;     // vehicle budget per tile when re-tiling from occupancy
    uint32_t retile_every = 0;         // steps between load-balancing passes (0 = static tiles)
    uint32_t step_mode = TS_STEP_AUTO; // for the context's own world
    uint32_t link_blocks_per_sm = 0;   // for the context's own world (ts_set_link_grid)
    // vehicles
    bool loaded = false;
    uint32_t n_veh = 0;
    std::vector<uint32_t> route_off, depart, depart_sorted, dep_off, dep_ids;
    std::vector<uint32_t> route_links;  // host copy, fetched from the device when ts_write_state needs it
    std::vector<uint8_t> route_turn;    // allowed lanes of the turn after each route entry (with a turn table)
    // device
    ScenDev sd{};
    uint4 *d_lk_info = nullptr;
    uint2 *d_veh0 = nullptr;           // route starts, for resets
    unsigned long long *d_lt_tmp = nullptr;  // scratch of ts_read_link_times
    uint2 *d_dep_head0 = nullptr;      // queue starts, for resets
    std::vector<std::pair<void *, size_t>> allocs, veh_allocs;
    World *own = nullptr;
    ts_batch *batch = nullptr;
    uint64_t host_step = 0;
    bool sticky = false;

    void *dalloc(size_t bytes) {
        if (bytes == 0) bytes = 16;
        void *p = nullptr;
        if (has_alloc) {
            p = alloc.alloc(bytes, (void *)stream, alloc.user);
        } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
            cudaGetLastError();
            p = nullptr;
        }
        return p;
    }
    void dfree(void *p, size_t bytes) {
        if (!p) return;
        if (has_alloc) alloc.free(p, bytes, (void *)stream, alloc.user);
        else cudaFree(p);
    }
};

struct ts_batch {
    World w;
    cudaEvent_t ev = nullptr;
};

World::~World() {
    drop_graphs();
    if (d_span) cudaFree(d_span);
    if (d_table) cudaFree(d_table);
    if (d_counts) cudaFree(d_counts);
    if (d_link_tiles) cudaFree(d_link_tiles);
    if (d_node_tiles) cudaFree(d_node_tiles);
    if (cap_stream) cudaStreamDestroy(cap_stream);
}

void World::drop_graphs() {
    for (auto &g : graphs) cudaGraphExecDestroy(g.second);
    graphs.clear();
}

ts_status World::init(uint32_t cap) {
    capacity = cap;
    members.assign(cap, nullptr);
    CK(cudaGetDevice(&device));
    CK(cudaStreamCreateWithFlags(&cap_stream, cudaStreamNonBlocking));
    CK(cudaMalloc(&d_table, sizeof(ScenDev) * cap));
    CK(cudaMemset(d_table, 0, sizeof(ScenDev) * cap));
    CK(cudaMalloc(&d_counts, (2 + kChunk) * sizeof(uint32_t)));
    CK(cudaMemset(d_counts, 0, (2 + kChunk) * sizeof(uint32_t)));
    return TS_OK;
}

// Re-uploads the scenario table, the concatenated tile lists and their
// counts (synchronous; callers make sure no work of this world is in
// flight).  Captured graphs stay valid unless a tile array has to grow.
ts_status World::rebuild() {
    std::vector<ScenDev> table(capacity);
    std::vector<uint2> lt;
    std::vector<uint4> nt;
    for (uint32_t s = 0; s < capacity; ++s) {
        memset(&table[s], 0, sizeof(ScenDev));
        ts_ctx *c = members[s];
        if (!c) continue;
        table[s] = c->sd;
        for (uint2 t : c->link_tiles) {
            t.x |= s;
            lt.push_back(t);
        }
        for (uint4 t : c->node_tiles) {
            t.x = s;
            nt.push_back(t);
        }
    }
    CK(cudaMemcpy(d_table, table.data(), sizeof(ScenDev) * capacity, cudaMemcpyHostToDevice));
    // room for re-tiling on the device: at most one tile per column
    size_t need = lt.size();
    bool lb = false;
    for (ts_ctx *c : members)
        if (c && c->retile_every) {
            need = std::max<size_t>(need, c->n_cols);
            lb = true;
        }
    if (need > link_cap) {
        drop_graphs();
        if (d_link_tiles) cudaFree(d_link_tiles);
        d_link_tiles = nullptr;
        link_cap = std::max<size_t>(2 * need, need + 1024);
        CK(cudaMalloc(&d_link_tiles, sizeof(uint2) * link_cap));
    }
    if (nt.size() > node_cap) {
        drop_graphs();
        if (d_node_tiles) cudaFree(d_node_tiles);
        d_node_tiles = nullptr;
        node_cap = std::max<size_t>(nt.size(), 2 * node_cap);
        CK(cudaMalloc(&d_node_tiles, sizeof(uint4) * node_cap));
    }
    if (!lt.empty()) CK(cudaMemcpy(d_link_tiles, lt.data(), sizeof(uint2) * lt.size(), cudaMemcpyHostToDevice));
    if (!nt.empty()) CK(cudaMemcpy(d_node_tiles, nt.data(), sizeof(uint4) * nt.size(), cudaMemcpyHostToDevice));
    n_link_tiles = (uint32_t)lt.size();
    n_node_tiles = (uint32_t)nt.size();
    const uint32_t counts[2] = {n_link_tiles, n_node_tiles};
    CK(cudaMemcpy(d_counts, counts, sizeof(counts), cudaMemcpyHostToDevice));
    // persistent grids: at most the resident blocks, and room for the tile
    // count to double through load balancing before warps loop over tiles
    bool pl = false, v5 = true;
    for (ts_ctx *c : members)
        if (c) {
            pl = pl || c->sd.route_turn != nullptr || c->sd.slot_gap != nullptr;
            v5 = v5 && c->sd.vmax == 5u;
        }
    if (pl != turns || v5 != vmax5) {
        drop_graphs();
        turns = pl;
        vmax5 = v5;
    }
    // re-tiling changes the tile count on the device: then the grid is every
    // resident block
    const int want = lb ? (1 << 30) : (int)((2ull * n_link_tiles + kLinkWarpsPerBlock - 1) / kLinkWarpsPerBlock);
    int cap = max_link_blocks(turns);
    if (link_blocks_per_sm) {
        int sms = 0;
        CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
        cap = std::min(cap, (int)link_blocks_per_sm * std::max(sms, 1));
    }
    const int gl = std::max(1, std::min<int>(want, cap));
    const int gn = std::max(1, std::min<int>((int)n_node_tiles, max_node_blocks(turns)));
    if (gl > grid_l || gn != grid_n || gl < grid_l / 2 || cap != grid_cap) {
        drop_graphs();
        grid_l = gl;
        grid_n = gn;
        grid_cap = cap;
    }
    return TS_OK;
}

// Fused steps (one launch per step) save the node kernel's launch but make
// every tile with an occupied lane-end buffer resolve that buffer's node
// transfer itself (two to three dependent memory round trips before the
// step can start).  Measured on GB300, that costs more than the launch it
// saves as soon as buffers are in use (config 1: 16.8 us per step split,
// 18.3 fused; an empty network: 9.4 us fused, 12.4 split), so AUTO splits.
bool World::fused() const { return mode == TS_STEP_FUSED; }

// Enqueues n steps of every active member on stream s, as CUDA graphs of up
// to kChunk steps.  Fused: one link kernel per step, each but the first also
// completing the node transfers of the step before it, and the node kernel
// for the chunk's last step.  Split: a link and a node kernel per step.
// Then the chunk-closing kernel.
ts_status World::run(uint32_t n, cudaStream_t s) {
    const bool fu = fused();
    while (n > 0) {
        const uint32_t g = std::min(n, kChunk);
        const uint32_t key = g | (fu ? 1u << 16 : 0u);
        auto it = graphs.find(key);
        if (it == graphs.end()) {
            cudaGraph_t graph;
            CK(cudaStreamBeginCapture(cap_stream, cudaStreamCaptureModeThreadLocal));
            unsigned long long *sp = timing ? d_span : nullptr;
            for (uint32_t i = 0; i < g; ++i) {
                launch_link_kernel(d_table, d_link_tiles, d_counts, i, grid_l, cap_stream, i > 0, fu && i > 0,
                                   turns, sp, vmax5, d_counts + 2);
                if (!fu || i + 1 == g)
                    launch_node_kernel(d_table, d_node_tiles, d_counts + 1, i, grid_n, cap_stream, true, fu, turns,
                                       sp);
            }
            launch_advance_kernel(d_table, capacity, g, cap_stream, true, sp, d_counts + 2);
            CK(cudaStreamEndCapture(cap_stream, &graph));
            cudaGraphExec_t exec;
            const cudaError_t e = cudaGraphInstantiate(&exec, graph, 0);
            cudaGraphDestroy(graph);
            if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
            it = graphs.emplace(key, exec).first;
        }
        CK(cudaGraphLaunch(it->second, s));
        n -= g;
    }
    return TS_OK;
}

// ------------------------------------------------------------------ helpers

namespace {

ts_status check_ctx(ts_ctx *c) {
    if (!c) return fail(TS_ERR_INVALID, "null context");
    if (c->sticky) return fail(TS_ERR_CUDA, "context is in an error state");
    if (cudaSetDevice(c->device) != cudaSuccess) return cuda_fail(cudaGetLastError(), "cudaSetDevice");
    return TS_OK;
}

void free_list(ts_ctx *c, std::vector<std::pair<void *, size_t>> &lst) {
    for (auto &a : lst) c->dfree(a.first, a.second);
    lst.clear();
}

template <typename T>
T *alloc_in(ts_ctx *c, std::vector<std::pair<void *, size_t>> &lst, size_t count, bool &ok) {
    const size_t bytes = sizeof(T) * std::max<size_t>(count, 1);
    void *p = c->dalloc(bytes);
    if (p) lst.emplace_back(p, bytes);
    else ok = false;
    return reinterpret_cast<T *>(p);
}

// Reads the control block (after the context's work is complete).
ts_status read_ctrl(ts_ctx *c, Ctrl *out) {
    CK(cudaMemcpyAsync(out, c->sd.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, c->stream));
    const ts_status sw = sync_stream(c->stream);
    if (sw != TS_OK) return sw;
    if (out->error) {
        c->sticky = true;
        char buf[96];
        snprintf(buf, sizeof(buf), "device consistency check failed (flags 0x%x)", out->error);
        return fail(TS_ERR_DEVICE_CHECK, buf);
    }
    return TS_OK;
}

ts_status wait_ctx(ts_ctx *c, uint32_t timeout_ms) {
    const ts_status s = wait_event(c->ev, timeout_ms);
    if (s == TS_ERR_CUDA) c->sticky = true;
    return s;
}

// Warp tiles: runs of at most 32 consecutive columns (link-major, then
// column j) holding at most tile_words occupancy words (columns times
// lanes).  A ring of at most 32 columns (and tile_words words) lies inside
// one tile; a longer ring gets tiles of its own.  The last column of a link
// is never separated from the one before it when it holds at most 2*vmax
// cells, so the cells of a halo that a tile looks at are never within vmax
// cells of a link end, and vehicles near a link end and its buffers are in
// one tile.  Re-tiling from the occupancy (on the device) cuts these tiles
// further where tile_cuts allows.  Results do not depend on the tiling.
void build_tiles(ts_ctx *c) {
    const uint32_t TW = std::max<uint32_t>(c->tile_words, 2u * (uint32_t)kMaxLanes), vmax = c->params.vmax;
    const uint32_t MC = (uint32_t)kWarpTileCols;
    c->link_tiles.clear();
    uint32_t start = 0, n = 0, words = 0;
    auto flush = [&]() {
        if (n) c->link_tiles.push_back(make_uint2((n - 1u) << 24, start));
        n = words = 0;
    };
    auto add = [&](uint32_t col, uint32_t w) {
        if (n == 0) start = col;
        ++n;
        words += w;
    };
    for (uint32_t l = 0; l < c->n_links; ++l) {
        const uint32_t nc = c->ncols[l], lanes = c->lanes[l], c0 = c->col_base[l];
        if (c->ring[l]) {
            if (nc <= MC && nc * lanes <= TW) {
                if (n + nc > MC || words + nc * lanes > TW) flush();
                if (n == 0) start = c0;
                n += nc;
                words += nc * lanes;
                continue;
            }
            flush();
            for (uint32_t j = 0; j < nc; ++j) {
                if (n > 0 && (n + 1 > MC || words + lanes > TW)) flush();
                add(c0 + j, lanes);
            }
            flush();
            continue;
        }
        const bool short_tail = nc >= 2 && c->cells[l] - 32u * (nc - 1u) <= 2u * vmax;
        for (uint32_t j = 0; j < nc; ++j) {
            if (n > 0 && (n + 1 > MC || words + lanes > TW)) {
                if (short_tail && j == nc - 1u && start + n - 1u == c0 + j - 1u) {
                    // the short last column goes with the one before it
                    if (n >= 2) {
                        --n;
                        words -= lanes;
                        flush();
                        add(c0 + j - 1u, lanes);
                    }  // else the tile is that column alone: it takes the last one too
                } else {
                    flush();
                }
            }
            add(c0 + j, lanes);
        }
    }
    flush();
    // where a tile may be cut by re-tiling: not before a short last column,
    // not inside a ring that starts after the tile's first column
    c->tile_cuts.assign(c->link_tiles.size(), 0u);
    {
        uint32_t l = 0;
        for (size_t i = 0; i < c->link_tiles.size(); ++i) {
            const uint2 t = c->link_tiles[i];
            const uint32_t n = (t.x >> 24) + 1u;
            uint32_t ok = 0u;
            for (uint32_t k = 0; k < n; ++k) {
                const uint32_t col = t.y + k;
                while (c->col_base[l + 1] <= col) ++l;
                const uint32_t j = col - c->col_base[l], nc = c->ncols[l];
                bool allow = k > 0;
                if (c->ring[l] && j > 0 && k > j) allow = false;
                if (!c->ring[l] && j + 1 == nc && j >= 1 && c->cells[l] - 32u * j <= 2u * vmax) allow = false;
                if (allow) ok |= 1u << k;
            }
            c->tile_cuts[i] = ok;
        }
    }
    c->node_tiles.clear();
    for (uint32_t m = 0; m < c->n_links; m += kNodeThreads)
        c->node_tiles.push_back(make_uint4(0u, m, std::min(c->n_links, m + (uint32_t)kNodeThreads), 0u));
}

ts_status upload_lk_info(ts_ctx *c) {
    std::vector<uint4> li(c->n_links);
    for (uint32_t l = 0; l < c->n_links; ++l)
        li[l] = make_uint4(c->wbase[l], c->cells[l], c->lanes[l] | ((uint32_t)c->ring[l] << 8), c->bpos[l]);
    CK(cudaMemcpy(c->d_lk_info, li.data(), sizeof(uint4) * c->n_links, cudaMemcpyHostToDevice));
    // per column: word of lane 0, link, j | lanes << 20 | ring << 23, cells;
    // and its link's first link-end buffer and signal
    std::vector<uint4> ci(std::max<uint32_t>(c->n_cols, 1u)), ca(ci.size(), make_uint4(0u, 0u, 0u, 0u));
    for (uint32_t l = 0; l < c->n_links; ++l)
        for (uint32_t j = 0; j < c->ncols[l]; ++j) {
            ci[c->col_base[l] + j] = make_uint4(c->wbase[l] + j * c->lanes[l], l,
                                                j | (c->lanes[l] << 20) | ((uint32_t)c->ring[l] << 23), c->cells[l]);
            ca[c->col_base[l] + j] = make_uint4(c->bpos[l], c->sig_cycle_green[l], c->sig_offset[l], 0u);
        }
    CK(cudaMemcpy(const_cast<uint4 *>(c->sd.col_info), ci.data(), sizeof(uint4) * ci.size(), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(const_cast<uint4 *>(c->sd.col_aux), ca.data(), sizeof(uint4) * ca.size(), cudaMemcpyHostToDevice));
    return TS_OK;
}

ts_status validate_desc(const ts_network_desc *d, const ts_params *p) {
    if (!d || !p) return fail(TS_ERR_INVALID, "null descriptor");
    if (p->vmax < 1 || p->vmax > (uint32_t)kMaxVmax) return fail(TS_ERR_INVALID, "vmax must be 1..15");
    if (d->n_links == 0) return fail(TS_ERR_INVALID, "network has no links");
    if (!d->link_cells || !d->link_lanes || !d->link_from || !d->link_to) return fail(TS_ERR_INVALID, "null link array");
    for (uint32_t l = 0; l < d->n_links; ++l) {
        const bool ring = d->link_ring && d->link_ring[l];
        if (d->link_lanes[l] < 1 || d->link_lanes[l] > (uint32_t)kMaxLanes) return fail(TS_ERR_INVALID, "lanes must be 1..4");
        if (d->link_cells[l] < 1 || d->link_cells[l] >= kMaxCells) return fail(TS_ERR_INVALID, "cells must be 1..2^22-1");
        if (ring) {
            if (d->link_cells[l] % 32u != 0u) return fail(TS_ERR_INVALID, "ring length must be a multiple of 32 cells");
        } else if (d->link_from[l] >= d->n_nodes || d->link_to[l] >= d->n_nodes) {
            return fail(TS_ERR_INVALID, "link node id out of range");
        }
        if (d->link_yield && d->link_yield[l] > 31u)
            return fail(TS_ERR_INVALID, "an acceptance gap must be 0..31 cells");
        if (d->link_signal) {
            const uint32_t cycle = d->link_signal[3 * l], green = d->link_signal[3 * l + 1];
            const uint32_t offset = d->link_signal[3 * l + 2];
            if (cycle >= 65536u || green >= 65536u || offset >= 65536u || (cycle && green > cycle))
                return fail(TS_ERR_INVALID, "signal cycle, green and offset must be below 2^16, green <= cycle");
        }
    }
    return TS_OK;
}

// Zeroes the statistics ring and sets the control block.
ts_status reset_ctrl(ts_ctx *c, uint64_t step, uint64_t arrived, uint64_t inserted, cudaStream_t s,
                     uint64_t active = 0, uint64_t buffered = 0, uint64_t sum_v = 0, uint64_t hash = 0) {
    Ctrl h{};
    h.base = step;
    h.target = step;
    h.arrived = arrived;
    h.inserted = inserted;
    h.active = active;
    h.buffered = buffered;
    h.sum_v = sum_v;
    h.hash = hash;
    CK(cudaMemcpyAsync(c->sd.ctrl, &h, sizeof(Ctrl), cudaMemcpyHostToDevice, s));
    CK(cudaMemsetAsync(c->sd.stats, 0, sizeof(StatRec) * kStatsRing * c->n_sub, s));
    const ts_status sw = sync_stream(s);
    if (sw != TS_OK) return sw;
    c->host_step = step;
    return TS_OK;
}

uint64_t departed_upto(const ts_ctx *c, uint64_t t) {
    return (uint64_t)(std::upper_bound(c->depart_sorted.begin(), c->depart_sorted.end(), t) - c->depart_sorted.begin());
}

}  // namespace

// ------------------------------------------------------------------ C ABI

extern "C" {

const char *ts_last_error(void) { return g_err.c_str(); }

uint32_t ts_launches_per_step(void) { return 1u; }

ts_status ts_philox_words(uint32_t n, const uint32_t *host_step, const uint32_t *host_id, uint64_t seed,
                          uint32_t *host_out) {
    if (n == 0) return TS_OK;
    if (!host_step || !host_id || !host_out) return fail(TS_ERR_INVALID, "null array");
    uint32_t *d = nullptr;
    const size_t bytes = 4ull * n;
    if (cudaMalloc(&d, 3 * bytes) != cudaSuccess) {
        cudaGetLastError();
        return fail(TS_ERR_OOM, "device allocation failed");
    }
    cudaError_t e = cudaMemcpy(d, host_step, bytes, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(d + n, host_id, bytes, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        launch_philox_words(d, d + n, (uint32_t)(seed & 0xFFFFFFFFull), (uint32_t)(seed >> 32), n, d + 2ull * n,
                            nullptr);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(host_out, d + 2ull * n, bytes, cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) return cuda_fail(e, "ts_philox_words");
    return TS_OK;
}

size_t ts_footprint_bytes(const ts_network_desc *d, uint32_t n_vehicles, uint64_t route_len) {
    if (!d) return 0;
    uint64_t words = 0, slots = 0;
    for (uint32_t l = 0; l < d->n_links; ++l) {
        const bool ring = d->link_ring && d->link_ring[l];
        words += (uint64_t)((d->link_cells[l] + 31u) / 32u) * d->link_lanes[l];
        if (!ring) slots += d->link_lanes[l];
    }
    size_t b = 0;
    b += 16ull * d->n_links * 2;                              // lk_info, nd_info
    if (d->link_signal) b += 8ull * d->n_links;              // signals
    b += words * (4 + 4 + 4 + 32 + 128) * 2;                  // occupancy, v>0, location, velocity, id (x2)
    b += 16ull * slots * 2 + 8ull * n_vehicles * 2 + 4ull * route_len;  // buffers (x2), vehicles, routes
    b += 8ull * n_vehicles + 8ull * d->n_links * 2;           // departure queue, heads (+ reset copy)
    b += 4ull * n_vehicles + 16ull * d->n_links;              // link entry steps, link times (+ scratch)
    b += sizeof(Ctrl) + sizeof(StatRec) * kStatsRing * 8;
    if (d->turn_lanes) b += route_len + n_vehicles;             // allowed lanes per route entry and departure
    if (d->link_yield) b += 9ull * slots;                       // acceptance gap and lane tail per buffer
    return b;
}

ts_status ts_create_network(const ts_network_desc *desc, const ts_params *params, const ts_allocator *allocator,
                            ts_ctx **out) {
    if (!out) return fail(TS_ERR_INVALID, "null output");
    *out = nullptr;
    ts_status st = validate_desc(desc, params);
    if (st != TS_OK) return st;
    std::unique_ptr<ts_ctx> c(new (std::nothrow) ts_ctx());
    if (!c) return fail(TS_ERR_OOM, "host allocation failed");
    CK(cudaGetDevice(&c->device));
    CK(cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking));
    CK(cudaEventCreateWithFlags(&c->ev, cudaEventDisableTiming));
    CK(cudaEventRecord(c->ev, c->stream));
    if (allocator && allocator->alloc && allocator->free) {
        c->alloc = *allocator;
        c->has_alloc = true;
    }
    c->params = *params;
    const uint32_t L = desc->n_links;
    c->n_nodes = desc->n_nodes;
    c->n_links = L;
    c->from.assign(desc->link_from, desc->link_from + L);
    c->to.assign(desc->link_to, desc->link_to + L);
    c->cells.assign(desc->link_cells, desc->link_cells + L);
    c->lanes.assign(desc->link_lanes, desc->link_lanes + L);
    c->ring.assign(L, 0);
    if (desc->link_ring)
        for (uint32_t l = 0; l < L; ++l) c->ring[l] = desc->link_ring[l] ? 1 : 0;
    for (uint32_t l = 0; l < L; ++l) c->n_ring += c->ring[l];
    // words, lanes, canonical cells
    c->ncols.resize(L);
    c->wbase.resize(L);
    c->col_base.resize(L + 1);
    c->lane_base.resize(L + 1);
    uint64_t w = 0;
    c->lane_base[0] = 0;
    for (uint32_t l = 0; l < L; ++l) {
        c->ncols[l] = (c->cells[l] + 31u) / 32u;
        c->wbase[l] = (uint32_t)w;
        c->col_base[l + 1] = c->col_base[l] + c->ncols[l];
        w += (uint64_t)c->ncols[l] * c->lanes[l];
        c->lane_base[l + 1] = c->lane_base[l] + c->lanes[l];
    }
    if (w >= (1ull << 31) / 32ull) return fail(TS_ERR_INVALID, "network too large");
    c->n_words = (uint32_t)w;
    c->n_cols = c->col_base[L];
    c->n_lanes = c->lane_base[L];
    c->cell_base.resize(c->n_lanes + 1);
    c->cell_base[0] = 0;
    for (uint32_t l = 0; l < L; ++l)
        for (uint32_t k = 0; k < c->lanes[l]; ++k) {
            const uint32_t ln = c->lane_base[l] + k;
            c->cell_base[ln + 1] = c->cell_base[ln] + c->cells[l];
        }
    c->n_lane_cells = c->cell_base[c->n_lanes];
    // link-end buffers grouped by the node the link ends at, priority order
    c->node_in_off.assign(c->n_nodes + 1, 0);
    for (uint32_t l = 0; l < L; ++l)
        if (!c->ring[l]) c->node_in_off[c->to[l] + 1] += c->lanes[l];
    for (uint32_t n = 0; n < c->n_nodes; ++n) c->node_in_off[n + 1] += c->node_in_off[n];
    c->n_slots = c->node_in_off[c->n_nodes];
    if (desc->link_yield) c->gap_accept.assign(desc->link_yield, desc->link_yield + L);
    auto yields = [&](uint32_t l) { return !c->gap_accept.empty() && c->gap_accept[l] > 0; };
    // a node's buffers: its priority approaches, then its yield approaches,
    // each in ascending link id
    c->bpos.assign(L, 0);
    c->node_prio.assign(c->n_nodes, 0);
    {
        std::vector<uint32_t> fill(c->node_in_off.begin(), c->node_in_off.end() - 1);
        for (int pass = 0; pass < 2; ++pass)
            for (uint32_t l = 0; l < L; ++l)
                if (!c->ring[l] && yields(l) == (pass == 1)) {
                    c->bpos[l] = fill[c->to[l]];
                    fill[c->to[l]] += c->lanes[l];
                    if (pass == 0) c->node_prio[c->to[l]] += c->lanes[l];
                }
    }
    for (uint32_t n = 0; n < c->n_nodes; ++n)
        if (c->node_in_off[n + 1] - c->node_in_off[n] > 255u)
            return fail(TS_ERR_INVALID, "more than 255 lanes end at one node");
    // links leaving every node (ascending id) and the turn table
    c->out_off.assign(c->n_nodes + 1, 0);
    for (uint32_t l = 0; l < L; ++l)
        if (!c->ring[l]) c->out_off[c->from[l] + 1]++;
    for (uint32_t n = 0; n < c->n_nodes; ++n) c->out_off[n + 1] += c->out_off[n];
    c->out_link.resize(c->out_off[c->n_nodes]);
    {
        std::vector<uint32_t> fill(c->out_off.begin(), c->out_off.end() - 1);
        for (uint32_t l = 0; l < L; ++l)
            if (!c->ring[l]) c->out_link[fill[c->from[l]]++] = l;
    }
    c->turn_off.assign(L + 1, 0);
    for (uint32_t l = 0; l < L; ++l)
        c->turn_off[l + 1] = c->turn_off[l] + (c->ring[l] ? 0u : c->out_off[c->to[l] + 1] - c->out_off[c->to[l]]);
    if (desc->turn_lanes) {
        c->has_turn = true;
        c->turn.assign(desc->turn_lanes, desc->turn_lanes + c->turn_off[L]);
        for (uint32_t l = 0; l < L; ++l)
            for (uint32_t j = c->turn_off[l]; j < c->turn_off[l + 1]; ++j)
                if (c->turn[j] == 0 || (c->turn[j] >> c->lanes[l]) != 0)
                    return fail(TS_ERR_INVALID, "a turn needs at least one lane of its link, and only lanes it has");
    }
    build_tiles(c.get());
    c->n_sub = c->link_tiles.size() >= 64 ? 8u : 1u;  // small networks keep one sub-record per step
    // device arrays of the network
    bool ok = true;
    auto &A = c->allocs;
    c->d_lk_info = alloc_in<uint4>(c.get(), A, L, ok);
    uint4 *col_info = alloc_in<uint4>(c.get(), A, c->n_cols, ok);
    uint4 *col_aux = alloc_in<uint4>(c.get(), A, c->n_cols, ok);
    uint4 *nd_info = alloc_in<uint4>(c.get(), A, L, ok);
    uint2 *sig_info = desc->link_signal ? alloc_in<uint2>(c.get(), A, L, ok) : nullptr;
    uint8_t *slot_gap = desc->link_yield ? alloc_in<uint8_t>(c.get(), A, c->n_slots, ok) : nullptr;
    uint2 *slot_tail = desc->link_yield ? alloc_in<uint2>(c.get(), A, c->n_slots, ok) : nullptr;
    uint32_t *occ0 = alloc_in<uint32_t>(c.get(), A, c->n_words, ok);
    uint32_t *occ1 = alloc_in<uint32_t>(c.get(), A, c->n_words, ok);
    uint32_t *mov0 = alloc_in<uint32_t>(c.get(), A, c->n_words, ok);
    uint32_t *mov1 = alloc_in<uint32_t>(c.get(), A, c->n_words, ok);
    uint32_t *loc0 = alloc_in<uint32_t>(c.get(), A, c->n_words, ok);
    uint32_t *loc1 = alloc_in<uint32_t>(c.get(), A, c->n_words, ok);
    int8_t *vel0 = alloc_in<int8_t>(c.get(), A, (size_t)c->n_words * 32, ok);
    int8_t *vel1 = alloc_in<int8_t>(c.get(), A, (size_t)c->n_words * 32, ok);
    uint32_t *vid0 = alloc_in<uint32_t>(c.get(), A, (size_t)c->n_words * 32, ok);
    uint32_t *vid1 = alloc_in<uint32_t>(c.get(), A, (size_t)c->n_words * 32, ok);
    uint4 *slots0 = alloc_in<uint4>(c.get(), A, c->n_slots, ok);
    uint4 *slots1 = alloc_in<uint4>(c.get(), A, c->n_slots, ok);
    unsigned long long *lt = alloc_in<unsigned long long>(c.get(), A, 2ull * L, ok);  // link times, scratch
    Ctrl *ctrl = alloc_in<Ctrl>(c.get(), A, 1, ok);
    StatRec *stats = alloc_in<StatRec>(c.get(), A, (size_t)kStatsRing * c->n_sub, ok);
    if (!ok) {
        free_list(c.get(), A);
        return fail(TS_ERR_OOM, "device allocation failed");
    }
    ScenDev &sd = c->sd;
    sd.lk_info = c->d_lk_info;
    sd.col_info = col_info;
    sd.col_aux = col_aux;
    sd.n_cols = c->n_cols;
    sd.nd_info = nd_info;
    sd.sig_info = sig_info;
    sd.slot_gap = slot_gap;
    sd.slot_tail = slot_tail;
    sd.occ[0] = occ0;
    sd.occ[1] = occ1;
    sd.mov[0] = mov0;
    sd.mov[1] = mov1;
    sd.loc[0] = loc0;
    sd.loc[1] = loc1;
    sd.vel[0] = vel0;
    sd.vel[1] = vel1;
    sd.vid[0] = vid0;
    sd.vid[1] = vid1;
    sd.slots[0] = slots0;
    sd.slots[1] = slots1;
    sd.link_time = lt;
    c->d_lt_tmp = lt + L;
    sd.ctrl = ctrl;
    sd.stats = stats;
    sd.vmax = params->vmax;
    sd.p_threshold = params->p_threshold;
    sd.seed_lo = (uint32_t)(params->seed & 0xFFFFFFFFull);
    sd.seed_hi = (uint32_t)(params->seed >> 32);
    sd.lane_change = params->lane_change ? 1u : 0u;
    sd.n_links = L;
    sd.n_sub = c->n_sub;
    c->sig_cycle_green.assign(L, 0u);
    c->sig_offset.assign(L, 0u);
    if (desc->link_signal)
        for (uint32_t l = 0; l < L; ++l) {
            c->sig_cycle_green[l] = desc->link_signal[3 * l] | (desc->link_signal[3 * l + 1] << 16);
            c->sig_offset[l] = desc->link_signal[3 * l + 2];
        }
    st = upload_lk_info(c.get());
    if (st != TS_OK) return st;
    for (uint32_t *p : {occ0, occ1, mov0, mov1, loc0, loc1}) CK(cudaMemset(p, 0, 4ull * c->n_words));
    if (sig_info) {
        std::vector<uint2> sg(L);
        for (uint32_t l = 0; l < L; ++l)
            sg[l] = make_uint2(desc->link_signal[3 * l] | (desc->link_signal[3 * l + 1] << 16), desc->link_signal[3 * l + 2]);
        CK(cudaMemcpy(sig_info, sg.data(), sizeof(uint2) * L, cudaMemcpyHostToDevice));
    }
    if (slot_gap && c->n_slots) {
        // per buffer: its link's acceptance gap, and its lane's last column
        std::vector<uint8_t> sg(c->n_slots);
        std::vector<uint2> tl(c->n_slots);
        for (uint32_t l = 0; l < L; ++l)
            if (!c->ring[l])
                for (uint32_t k = 0; k < c->lanes[l]; ++k) {
                    sg[c->bpos[l] + k] = c->gap_accept[l];
                    tl[c->bpos[l] + k] = make_uint2(c->wbase[l] + (c->ncols[l] - 1u) * c->lanes[l] + k,
                                                    c->cells[l] | (c->lanes[l] << 24) |
                                                        ((uint32_t)c->gap_accept[l] << 27));
                }
        CK(cudaMemcpy(slot_gap, sg.data(), c->n_slots, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(slot_tail, tl.data(), sizeof(uint2) * c->n_slots, cudaMemcpyHostToDevice));
    }
    CK(cudaMemset(slots0, 0xFF, 16ull * std::max<uint32_t>(c->n_slots, 1)));
    CK(cudaMemset(slots1, 0xFF, 16ull * std::max<uint32_t>(c->n_slots, 1)));
    CK(cudaMemset(lt, 0, 16ull * L));
    CK(cudaMemset(ctrl, 0, sizeof(Ctrl)));
    CK(cudaMemset(stats, 0, sizeof(StatRec) * kStatsRing * c->n_sub));
    *out = c.release();
    return TS_OK;
}

// Departure-queue head of link l at absolute queue index h: {h, departure
// step of entry h, or ~0 when the queue is exhausted}.
static uint2 queue_head(const ts_ctx *c, uint32_t l, uint32_t h) {
    return make_uint2(h, h < c->dep_off[l + 1] ? c->depart[c->dep_ids[h]] : 0xFFFFFFFFu);
}

// Host-to-device copy of a large pageable buffer: host threads fill two
// pinned staging buffers in turn while the copy engine drains the other, so
// the transfer is not limited by one thread's pageable staging.  The staging
// buffers are allocated on first use and kept for the process; without
// them (allocation refused) the copy is a plain cudaMemcpy.
static ts_status upload_large(void *dst, const void *src, size_t bytes, cudaStream_t s) {
    constexpr size_t kStage = 128ull << 20;
    static std::mutex mu;
    static void *stage[2] = {nullptr, nullptr};
    if (bytes < 2 * kStage) {
        CK(cudaMemcpy(dst, src, bytes, cudaMemcpyHostToDevice));
        return TS_OK;
    }
    std::lock_guard<std::mutex> lock(mu);
    for (int i = 0; i < 2; ++i)
        if (!stage[i] && cudaHostAlloc(&stage[i], kStage, cudaHostAllocPortable) != cudaSuccess) {
            cudaGetLastError();
            stage[i] = nullptr;
        }
    if (!stage[0] || !stage[1]) {
        CK(cudaMemcpy(dst, src, bytes, cudaMemcpyHostToDevice));
        return TS_OK;
    }
    cudaEvent_t done[2];
    CK(cudaEventCreateWithFlags(&done[0], cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&done[1], cudaEventDisableTiming));
    const unsigned hw = std::thread::hardware_concurrency();
    const size_t nt = std::max<size_t>(1, std::min<size_t>(hw ? hw : 1u, 16u));
    const char *from = static_cast<const char *>(src);
    char *to = static_cast<char *>(dst);
    cudaError_t e = cudaSuccess;
    int buf = 0;
    for (size_t off = 0; off < bytes && e == cudaSuccess; off += kStage, buf ^= 1) {
        const size_t n = std::min(kStage, bytes - off);
        if (off >= 2 * kStage) {  // this buffer's previous copy, bounded
            const ts_status sw = wait_event(done[buf], kHostWaitMs);
            if (sw != TS_OK) {
                cudaEventDestroy(done[0]);
                cudaEventDestroy(done[1]);
                return sw;
            }
        }
        char *st = static_cast<char *>(stage[buf]);
        std::vector<std::thread> pool;
        for (size_t t = 1; t < nt; ++t)
            pool.emplace_back([=] { memcpy(st + n * t / nt, from + off + n * t / nt, n * (t + 1) / nt - n * t / nt); });
        memcpy(st, from + off, n / nt);
        for (auto &th : pool) th.join();
        e = cudaMemcpyAsync(to + off, st, n, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaEventRecord(done[buf], s);
    }
    const ts_status sw = e == cudaSuccess ? sync_stream(s) : TS_OK;
    cudaEventDestroy(done[0]);
    cudaEventDestroy(done[1]);
    if (e != cudaSuccess) return cuda_fail(e, "route upload");
    return sw;
}

// Allowed lanes of the turn after route entry j (of a route ending before
// entry b): the turn-table entry of (links[j], links[j + 1]); 0 (any lane)
// on the last entry and where every lane of the link serves the turn.
static uint8_t turn_after(const ts_ctx *c, const uint32_t *links, uint32_t j, uint32_t b) {
    if (j + 1 >= b) return 0;
    const uint32_t l = links[j], m = links[j + 1], n = c->to[l];
    for (uint32_t r = c->out_off[n]; r < c->out_off[n + 1]; ++r)
        if (c->out_link[r] == m) {
            const uint8_t a = c->turn[c->turn_off[l] + (r - c->out_off[n])];
            return a == (uint8_t)((1u << c->lanes[l]) - 1u) ? (uint8_t)0 : a;
        }
    return 0;  // not reached for a connected route
}

static ts_status upload_vehicles(ts_ctx *c, const uint32_t *links) {
    free_list(c, c->veh_allocs);
    auto &A = c->veh_allocs;
    const uint32_t n = c->n_veh, L = c->n_links;
    const uint64_t total = c->route_off[n];
    bool ok = true;
    uint2 *veh = alloc_in<uint2>(c, A, n, ok);
    c->d_veh0 = alloc_in<uint2>(c, A, n, ok);
    uint32_t *enter = alloc_in<uint32_t>(c, A, n, ok);
    uint32_t *routes = alloc_in<uint32_t>(c, A, total, ok);
    uint32_t *dep_ids = alloc_in<uint32_t>(c, A, n, ok);
    uint32_t *dep_steps = alloc_in<uint32_t>(c, A, n, ok);
    uint2 *dep_head = alloc_in<uint2>(c, A, L, ok);
    c->d_dep_head0 = alloc_in<uint2>(c, A, L, ok);
    uint8_t *route_turn = c->has_turn ? alloc_in<uint8_t>(c, A, total, ok) : nullptr;
    uint8_t *dep_turn = c->has_turn ? alloc_in<uint8_t>(c, A, n, ok) : nullptr;
    if (!ok) {
        free_list(c, A);
        return fail(TS_ERR_OOM, "device allocation failed");
    }
    std::vector<uint2> hv(n);
    for (uint32_t i = 0; i < n; ++i) hv[i] = make_uint2(c->route_off[i], c->route_off[i + 1]);
    std::vector<uint32_t> ids(n), steps(n);
    for (uint32_t q = 0; q < n; ++q) {
        const uint32_t id = c->dep_ids[q];
        steps[q] = c->depart[id];
        ids[q] = id | (c->route_off[id + 1] - c->route_off[id] == 1 ? kLastLinkBit : 0u);
    }
    // per link: first slot of its upstream node, word of its column 0, slot
    // count, lanes and end of its departure queue
    std::vector<uint4> nd(L);
    for (uint32_t m = 0; m < L; ++m) {
        uint32_t lo = 0, cnt = 0, prio = 0;
        if (!c->ring[m]) {
            lo = c->node_in_off[c->from[m]];
            cnt = c->node_in_off[c->from[m] + 1] - lo;
            prio = c->node_prio[c->from[m]];
        }
        nd[m] = make_uint4(lo, c->wbase[m], cnt | (c->lanes[m] << 8) | (prio << 16), c->dep_off[m + 1]);
    }
    if (n) {
        CK(cudaMemcpy(veh, hv.data(), 8ull * n, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(c->d_veh0, hv.data(), 8ull * n, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(dep_ids, ids.data(), 4ull * n, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(dep_steps, steps.data(), 4ull * n, cudaMemcpyHostToDevice));
    }
    if (total) {
        const ts_status su = upload_large(routes, links, 4ull * total, c->stream);
        if (su != TS_OK) return su;
    }
    if (c->has_turn && total) {
        const ts_status su = upload_large(route_turn, c->route_turn.data(), total, c->stream);
        if (su != TS_OK) return su;
        std::vector<uint8_t> dt(n);
        for (uint32_t q = 0; q < n; ++q) dt[q] = c->route_turn[c->route_off[c->dep_ids[q]]];
        if (n) CK(cudaMemcpy(dep_turn, dt.data(), n, cudaMemcpyHostToDevice));
    }
    CK(cudaMemcpy(const_cast<uint4 *>(c->sd.nd_info), nd.data(), sizeof(uint4) * L, cudaMemcpyHostToDevice));
    std::vector<uint2> heads(L);
    for (uint32_t l = 0; l < L; ++l) heads[l] = queue_head(c, l, c->dep_off[l]);
    CK(cudaMemcpy(dep_head, heads.data(), 8ull * L, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(c->d_dep_head0, heads.data(), 8ull * L, cudaMemcpyHostToDevice));
    ScenDev &sd = c->sd;
    sd.veh = veh;
    sd.enter_step = enter;
    if (n) CK(cudaMemset(enter, 0xFF, 4ull * n));  // nobody on the network
    sd.route_links = routes;
    sd.dep_ids = dep_ids;
    sd.dep_steps = dep_steps;
    sd.dep_head = dep_head;
    sd.route_turn = route_turn;
    sd.dep_turn = dep_turn;
    return TS_OK;
}

// Device-side return to the empty network at step 0.
static ts_status reset_device_state(ts_ctx *c, cudaStream_t s) {
    ScenDev &sd = c->sd;
    for (int b = 0; b < 2; ++b) {
        CK(cudaMemsetAsync(sd.occ[b], 0, 4ull * c->n_words, s));
        CK(cudaMemsetAsync(sd.mov[b], 0, 4ull * c->n_words, s));
        CK(cudaMemsetAsync(sd.loc[b], 0, 4ull * c->n_words, s));
    }
    for (int b = 0; b < 2; ++b) CK(cudaMemsetAsync(sd.slots[b], 0xFF, 16ull * std::max<uint32_t>(c->n_slots, 1), s));
    CK(cudaMemsetAsync(sd.link_time, 0, 8ull * c->n_links, s));
    if (c->n_veh) CK(cudaMemsetAsync(sd.enter_step, 0xFF, 4ull * c->n_veh, s));  // nobody on the network
    if (c->n_veh) CK(cudaMemcpyAsync(sd.veh, c->d_veh0, 8ull * c->n_veh, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(sd.dep_head, c->d_dep_head0, 8ull * c->n_links, cudaMemcpyDeviceToDevice, s));
    CK(cudaMemsetAsync(sd.ctrl, 0, sizeof(Ctrl), s));
    CK(cudaMemsetAsync(sd.stats, 0, sizeof(StatRec) * kStatsRing * c->n_sub, s));
    return TS_OK;
}

static ts_status upload_base_tiles(ts_ctx *c);

static ts_status ensure_own_world(ts_ctx *c) {
    if (!c->own) {
        c->own = new (std::nothrow) World();
        if (!c->own) return fail(TS_ERR_OOM, "host allocation failed");
        const ts_status s = c->own->init(1);
        if (s != TS_OK) return s;
    }
    c->own->members[0] = c;
    c->own->mode = c->step_mode;
    c->own->link_blocks_per_sm = c->link_blocks_per_sm;
    return c->own->rebuild();
}

ts_status ts_load_vehicles(ts_ctx *c, uint32_t n, const uint32_t *dep, const uint32_t *off, const uint32_t *links) {
    ts_status st = check_ctx(c);
    if (st != TS_OK) return st;
    if (c->loaded) return fail(TS_ERR_STATE, "vehicles already loaded");
    if (n >= 0x7FFFFFFEu) return fail(TS_ERR_INVALID, "too many vehicles");
    if (n && (!dep || !off || !links)) return fail(TS_ERR_INVALID, "null vehicle array");
    std::vector<uint32_t> ro(off, off + n + 1);
    if (ro[0] != 0) return fail(TS_ERR_INVALID, "route offsets must start at 0");
    for (uint32_t i = 0; i < n; ++i)
        if (ro[i + 1] <= ro[i]) return fail(TS_ERR_INVALID, "empty or decreasing route");
    // every route entry, on host threads: link in range, connected to the
    // next entry, a ring link only as a whole route
    {
        const unsigned hw = std::thread::hardware_concurrency();
        const uint32_t nt = std::max(1u, std::min(hw ? hw : 1u, 16u));
        std::vector<int> bad(nt, 0);
        auto check = [&](uint32_t t) {
            for (uint32_t i = (uint32_t)((uint64_t)n * t / nt); i < (uint32_t)((uint64_t)n * (t + 1) / nt); ++i) {
                const uint32_t a = ro[i], b = ro[i + 1];
                for (uint32_t j = a; j < b; ++j) {
                    const uint32_t l = links[j];
                    if (l >= c->n_links) { bad[t] = 1; return; }
                    if (c->ring[l] && b - a != 1) { bad[t] = 2; return; }
                    if (j + 1 < b && (links[j + 1] >= c->n_links || c->to[l] != c->from[links[j + 1]])) {
                        bad[t] = 3;
                        return;
                    }
                }
            }
        };
        std::vector<std::thread> pool;
        for (uint32_t t = 1; t < nt; ++t) pool.emplace_back(check, t);
        check(0);
        for (auto &th : pool) th.join();
        for (int b : bad) {
            if (b == 1) return fail(TS_ERR_INVALID, "route link out of range");
            if (b == 2) return fail(TS_ERR_INVALID, "a ring link must be the whole route");
            if (b == 3) return fail(TS_ERR_INVALID, "route is not connected");
        }
    }
    c->n_veh = n;
    c->route_off = std::move(ro);
    c->route_links.clear();
    c->route_turn.clear();
    if (c->has_turn) {
        // the allowed lanes of every route entry's turn, on host threads
        c->route_turn.resize(c->route_off[n]);
        const unsigned hw = std::thread::hardware_concurrency();
        const uint32_t nt = std::max(1u, std::min(hw ? hw : 1u, 16u));
        auto fill = [&](uint32_t t) {
            for (uint32_t i = (uint32_t)((uint64_t)n * t / nt); i < (uint32_t)((uint64_t)n * (t + 1) / nt); ++i)
                for (uint32_t j = c->route_off[i]; j < c->route_off[i + 1]; ++j)
                    c->route_turn[j] = turn_after(c, links, j, c->route_off[i + 1]);
        };
        std::vector<std::thread> pool;
        for (uint32_t t = 1; t < nt; ++t) pool.emplace_back(fill, t);
        fill(0);
        for (auto &th : pool) th.join();
    }
    c->depart.assign(dep, dep + n);
    c->depart_sorted = c->depart;
    std::sort(c->depart_sorted.begin(), c->depart_sorted.end());
    // departure queues: per first link, ordered by (departure step, id)
    c->dep_off.assign(c->n_links + 1, 0);
    for (uint32_t i = 0; i < n; ++i) c->dep_off[links[c->route_off[i]] + 1]++;
    for (uint32_t l = 0; l < c->n_links; ++l) c->dep_off[l + 1] += c->dep_off[l];
    c->dep_ids.resize(n);
    {
        std::vector<uint32_t> fill(c->dep_off.begin(), c->dep_off.end() - 1);
        for (uint32_t i = 0; i < n; ++i) c->dep_ids[fill[links[c->route_off[i]]]++] = i;
        for (uint32_t l = 0; l < c->n_links; ++l)
            std::stable_sort(c->dep_ids.begin() + c->dep_off[l], c->dep_ids.begin() + c->dep_off[l + 1],
                             [&](uint32_t a, uint32_t b) { return c->depart[a] < c->depart[b]; });
    }
    st = upload_vehicles(c, links);
    if (st != TS_OK) return st;
    st = reset_device_state(c, c->stream);
    if (st != TS_OK) return st;
    st = sync_stream(c->stream);
    if (st != TS_OK) return st;
    c->host_step = 0;
    c->loaded = true;
    CK(cudaEventRecord(c->ev, c->stream));
    return TS_OK;  // the single-scenario launch set is built on first use
}

ts_status ts_set_tile_words(ts_ctx *c, uint32_t words) {
    ts_status st = check_ctx(c);
    if (st != TS_OK) return st;
    if (words < 8 || words > (uint32_t)kTileWords) return fail(TS_ERR_INVALID, "tile words must be 8..256");
    if (c->batch) return fail(TS_ERR_STATE, "context is in a batch");
    st = wait_ctx(c, 60000);
    if (st != TS_OK) return st;
    c->tile_words = words;
    build_tiles(c);
    if (c->retile_every) {
        st = upload_base_tiles(c);
        if (st != TS_OK) return st;
    }
    if (c->own) return ensure_own_world(c);
    return TS_OK;
}

uint32_t ts_tile_words(const ts_ctx *c) { return c ? c->tile_words : 0u; }

ts_status ts_set_step_mode(ts_ctx *c, uint32_t mode) {
    ts_status st = check_ctx(c);
    if (st != TS_OK) return st;
    if (mode > TS_STEP_SPLIT) return fail(TS_ERR_INVALID, "unknown step mode");
    if (c->batch) return fail(TS_ERR_STATE, "context is in a batch");
    c->step_mode = mode;
    if (c->own) c->own->mode = mode;
    return TS_OK;
}

ts_status ts_set_link_grid(ts_ctx *c, uint32_t blocks_per_sm) {
    ts_status st = check_ctx(c);
    if (st != TS_OK) return st;
    if (blocks_per_sm > 64) return fail(TS_ERR_INVALID, "at most 64 blocks per SM");
    if (c->batch) return fail(TS_ERR_STATE, "context is in a batch");
    st = wait_ctx(c, 60000);
    if (st != TS_OK) return st;
    c->link_blocks_per_sm = blocks_per_sm;
    if (c->own) return ensure_own_world(c);
    return TS_OK;
}

ts_status ts_batch_set_link_grid(ts_batch *b, uint32_t blocks_per_sm) {
    if (!b) return fail(TS_ERR_INVALID, "null batch");
    if (blocks_per_sm > 64) return fail(TS_ERR_INVALID, "at most 64 blocks per SM");
    ts_status st = wait_event(b->ev, 60000);  // the graphs may be rebuilt
    if (st != TS_OK) return st;
    b->w.link_blocks_per_sm = blocks_per_sm;
    return b->w.rebuild();
}

ts_status ts_batch_set_step_mode(ts_batch *b, uint32_t mode) {
    if (!b) return fail(TS_ERR_INVALID, "null batch");
    if (mode > TS_STEP_SPLIT) return fail(TS_ERR_INVALID, "unknown step mode");
    b->w.mode = mode;
    return TS_OK;
}

// The static tiles and their cut masks in device memory, for re-tiling.
static ts_status upload_base_tiles(ts_ctx *c) {
    const size_t n = c->link_tiles.size();
    if (n > c->base_cap) {
        if (c->d_base_tiles) cudaFree(c->d_base_tiles);
        if (c->d_cut_ok) cudaFree(c->d_cut_ok);
        c->d_base_tiles = nullptr;
        c->d_cut_ok = nullptr;
        c->base_cap = 0;
        CK(cudaMalloc(&c->d_base_tiles, sizeof(uint2) * n));
        CK(cudaMalloc(&c->d_cut_ok, sizeof(uint32_t) * n));
        c->base_cap = n;
    }
    if (n) {
        CK(cudaMemcpy(c->d_base_tiles, c->link_tiles.data(), sizeof(uint2) * n, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(c->d_cut_ok, c->tile_cuts.data(), sizeof(uint32_t) * n, cudaMemcpyHostToDevice));
    }
    return TS_OK;
}

// Load balancing between chunks, enqueued on the stream like the steps: the
// tiles are rebuilt on the device from the current occupancy so that no tile
// carries more than tile_vehicles vehicles; the captured graphs read the
// new tile count from device memory.
static ts_status retile_async(ts_ctx *c, cudaStream_t s) {
    World *w = c->own;
    CK(cudaMemsetAsync(w->d_counts, 0, sizeof(uint32_t), s));
    launch_retile(w->d_table, c->d_base_tiles, c->d_cut_ok, (uint32_t)c->link_tiles.size(),
                  c->tile_vehicles ? c->tile_vehicles : 0xFFFFFFFFu, w->d_link_tiles, w->d_counts, s);
    CK(cudaGetLastError());
    return TS_OK;
}

ts_status ts_step(ts_ctx *c, uint32_t n_steps, void *cuda_stream) {
    ts_status st = check_ctx(c);
    if (st != TS_OK) return st;
    if (!c->loaded) return fail(TS_ERR_STATE, "no vehicles loaded");
    if (c->batch) return fail(TS_ERR_STATE, "context is stepped by its batch");
    if (n_steps == 0) return TS_OK;
    cudaStream_t s = cuda_stream ? (cudaStream_t)cuda_stream : c->stream;
    if (!c->own) {
        st = ensure_own_world(c);
        if (st != TS_OK) return st;
    }
    const uint64_t start = c->host_step;
    c->host_step += n_steps;
    launch_set_target(c->sd.ctrl, c->host_step, s);
    CK(cudaGetLastError());
    const uint64_t R = c->retile_every;
    uint64_t done = 0;
    while (done < n_steps) {
        uint64_t seg = n_steps - done;
        if (R) seg = std::min<uint64_t>(seg, ((start + done) / R + 1) * R - (start + done));
        st = c->own->run((uint32_t)seg, s);
        if (st != TS_OK) {
            c->sticky = true;
            return st;
        }
        done += seg;
        if (R && done < n_steps && (start + done) % R == 0) {
            st = retile_async(c, s);
            if (st != TS_OK) {
                c->sticky = true;
                return st;
            }
        }
    }
    CK(cudaEventRecord(c->ev, s));
    return TS_OK;
}

ts_status ts_set_kernel_timing(ts_ctx *c, uint32_t on) {
    ts_status st = check_ctx(c);
    if (st != TS_OK) return st;
    if (c->batch) return fail(TS_ERR_STATE, "context is stepped by its batch");
    if (!c->loaded) return fail(TS_ERR_STATE, "no vehicles loaded");
    if (!c->own) {
        st = ensure_own_world(c);
        if (st != TS_OK) return st;
    }
    st = wait_ctx(c, 60000);
    if (st != TS_OK) return st;
    World *w = c->own;
    if (on && !w->d_span) {
        CK(cudaMalloc(&w->d_span, sizeof(unsigned long long) * kSpanWords));
        std::vector<unsigned long long> init(kSpanWords, 0ull);
        for (uint32_t i = 0; i < kChunk * 2u; ++i) init[2u * i] = ~0ull;  // starts: none yet
        CK(cudaMemcpy(w->d_span, init.data(), sizeof(unsigned long long) * kSpanWords, cudaMemcpyHostToDevice));
    }
    if ((on != 0) != w->timing) {
        w->drop_graphs();  // the launches' span argument is part of the captured graphs
        w->timing = on != 0;
    }
    return TS_OK;
}

ts_status ts_read_kernel_times(ts_ctx *c, uint64_t *out, uint32_t reset, uint32_t timeout_ms) {
    ts_status st = check_ctx(c);
    if (st != TS_OK) return st;
    if (!out) return fail(TS_ERR_INVALID, "null output");
    st = wait_ctx(c, timeout_ms);
    if (st != TS_OK) return st;
    if (!c->own || !c->own->d_span) {
        for (int i = 0; i < 4; ++i) out[i] = 0;
        return TS_OK;
    }
    unsigned long long *acc = c->own->d_span + kChunk * 4u;
    CK(cudaMemcpy(out, acc, 4 * sizeof(unsigned long long), cudaMemcpyDeviceToHost));
    if (reset) CK(cudaMemset(acc, 0, 4 * sizeof(unsigned long long)));
    return TS_OK;
}

ts_status ts_set_load_balance(ts_ctx *c, uint32_t every_steps, uint32_t vehicles_per_tile) {
    ts_status st = check_ctx(c);
    if (st != TS_OK) return st;
    if (every_steps && every_steps < kChunk) return fail(TS_ERR_INVALID, "load balancing at most every 32 steps");
    if (vehicles_per_tile && vehicles_per_tile < 32) return fail(TS_ERR_INVALID, "vehicle budget below 32");
    if (c->batch) return fail(TS_ERR_STATE, "context is in a batch");
    st = wait_ctx(c, 60000);  // the tile arrays are rewritten below
    if (st != TS_OK) return st;
    c->retile_every = every_steps;
    c->tile_vehicles = vehicles_per_tile;
    if (every_steps) {
        st = upload_base_tiles(c);
        if (st != TS_OK) return st;
    }
    if (c->own) return ensure_own_world(c);
    return TS_OK;
}

ts_status ts_reset(ts_ctx *c, void *cuda_stream) {
    ts_status st = check_ctx(c);
    if (st != TS_OK) return st;
    if (!c->loaded) return fail(TS_ERR_STATE, "no vehicles loaded");
    if (c->batch) return fail(TS_ERR_STATE, "context is stepped by its batch");
    cudaStream_t s = cuda_stream ? (cudaStream_t)cuda_stream : c->stream;
    st = reset_device_state(c, s);
    if (st != TS_OK) return st;
    CK(cudaEventRecord(c->ev, s));
    c->host_step = 0;
    return TS_OK;
}

ts_status ts_step_timed(ts_ctx *c, uint32_t n_steps, void *cuda_stream, float *link_ms, float *node_ms) {
    ts_status st = check_ctx(c);
    if (st != TS_OK) return st;
    if (!c->loaded) return fail(TS_ERR_STATE, "no vehicles loaded");
    if (c->batch) return fail(TS_ERR_STATE, "context is stepped by its batch");
    if (!link_ms || !node_ms) return fail(TS_ERR_INVALID, "null output");
    if (n_steps == 0) return TS_OK;
    cudaStream_t s = cuda_stream ? (cudaStream_t)cuda_stream : c->stream;
    if (!c->own) {
        st = ensure_own_world(c);
        if (st != TS_OK) return st;
    }
    World *w = c->own;
    std::vector<cudaEvent_t> ev(3ull * n_steps);
    size_t made = 0;
    ts_status rs = TS_OK;
    for (; made < ev.size(); ++made)
        if (cudaEventCreate(&ev[made]) != cudaSuccess) {
            rs = cuda_fail(cudaGetLastError(), "cudaEventCreate");
            break;
        }
    if (rs == TS_OK) {
        c->host_step += n_steps;
        launch_set_target(c->sd.ctrl, c->host_step, s);
        for (uint32_t b = 0; b < n_steps && rs == TS_OK; b += kChunk) {
            const uint32_t g = std::min(kChunk, n_steps - b);
            // the launch sequence of a captured chunk, with events around
            // every kernel (fused: node time is 0 but for the chunk's last step)
            const bool fu = w->fused();
            for (uint32_t i = 0; i < g; ++i) {
                const size_t e = 3ull * (b + i);
                cudaEventRecord(ev[e], s);
                launch_link_kernel(w->d_table, w->d_link_tiles, w->d_counts, i, w->grid_l, s, false, fu && i > 0,
                                   w->turns, nullptr, w->vmax5, w->d_counts + 2);
                cudaEventRecord(ev[e + 1], s);
                if (!fu || i + 1 == g)
                    launch_node_kernel(w->d_table, w->d_node_tiles, w->d_counts + 1, i, w->grid_n, s, false, fu,
                                       w->turns);
                cudaEventRecord(ev[e + 2], s);
            }
            launch_advance_kernel(w->d_table, w->capacity, g, s, false, nullptr, w->d_counts + 2);
            const cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) rs = cuda_fail(e, "kernel launch");
        }
    }
    if (rs == TS_OK) {
        rs = wait_event(ev[3ull * n_steps - 1], kHostWaitMs);
    }
    for (uint32_t i = 0; i < n_steps && rs == TS_OK; ++i) {
        cudaEventElapsedTime(&link_ms[i], ev[3ull * i], ev[3ull * i + 1]);
        cudaEventElapsedTime(&node_ms[i], ev[3ull * i + 1], ev[3ull * i + 2]);
    }
    for (size_t i = 0; i < made; ++i) cudaEventDestroy(ev[i]);
    if (rs != TS_OK) {
        c->sticky = true;
        return rs;
    }
    CK(cudaEventRecord(c->ev, s));
    return TS_OK;
}

ts_status ts_read_stats_range(ts_ctx *c, uint64_t first, uint32_t n, ts_stats *out, uint32_t timeout_ms) {
    ts_status st = check_ctx(c);
    if (st != TS_OK) return st;
    if (!out && n) return fail(TS_ERR_INVALID, "null output");
    st = wait_ctx(c, timeout_ms);
    if (st != TS_OK) return st;
    Ctrl h;
    st = read_ctrl(c, &h);
    if (st != TS_OK) return st;
    if (n == 0) return TS_OK;
    // the ring keeps the last kStatsRing - kChunk completed steps
    if (first + n > h.base || h.base - first > kStatsRing - kChunk || first < h.base - h.steps_run)
        return fail(TS_ERR_STATE, "requested steps are not available");
    const uint32_t nsub = c->n_sub;
    std::vector<StatRec> ring((size_t)kStatsRing * nsub);
    CK(cudaMemcpy(ring.data(), c->sd.stats, sizeof(StatRec) * ring.size(), cudaMemcpyDeviceToHost));
    auto sum = [&](uint64_t t, int f) {
        unsigned long long s = 0;
        for (uint32_t u = 0; u < nsub; ++u) {
            const unsigned long long *r =
                reinterpret_cast<const unsigned long long *>(&ring[(size_t)(t & (kStatsRing - 1)) * nsub + u]);
            s += r[f];
        }
        return (uint64_t)s;
    };
    // running values after step t, counted back from the values at the base
    uint64_t arr = h.arrived, ins = h.inserted, act = h.active, buf = h.buffered, sv = h.sum_v, hs = h.hash;
    auto back = [&](uint64_t t) {
        arr -= sum(t, kArrived);
        ins -= sum(t, kInserted);
        act -= sum(t, kDActive);
        buf -= sum(t, kDBuffered);
        sv -= sum(t, kDSumV);
        hs -= sum(t, kDHash);
    };
    for (uint64_t t = h.base - 1; t + 1 > first + n; --t) back(t);
    for (uint32_t i = n; i-- > 0;) {
        const uint64_t t = first + i;
        ts_stats &o = out[i];
        o.step = t;
        o.active = act;
        o.buffered = buf;
        o.lane_changes = sum(t, kLaneChanges);
        o.transfers = sum(t, kTransfers);
        o.inserted = sum(t, kInserted);
        o.sum_v = sv;
        o.vehicle_updates = sum(t, kUpdates);
        o.moving = sum(t, kMoving);
        o.state_hash = hs;
        o.arrived = arr;
        o.waiting = departed_upto(c, t) - ins;
        back(t);
    }
    return TS_OK;
}

ts_status ts_read_stats(ts_ctx *c, ts_stats *out, uint32_t timeout_ms) {
    ts_status st = check_ctx(c);
    if (st != TS_OK) return st;
    if (!out) return fail(TS_ERR_INVALID, "null output");
    st = wait_ctx(c, timeout_ms);
    if (st != TS_OK) return st;
    Ctrl h;
    st = read_ctrl(c, &h);
    if (st != TS_OK) return st;
    if (h.steps_run == 0) return fail(TS_ERR_STATE, "no step has completed");
    return ts_read_stats_range(c, h.base - 1, 1, out, timeout_ms);
}

ts_status ts_read_totals(ts_ctx *c, ts_totals *out, uint32_t timeout_ms) {
    ts_status st = check_ctx(c);
    if (st != TS_OK) return st;
    if (!out) return fail(TS_ERR_INVALID, "null output");
    st = wait_ctx(c, timeout_ms);
    if (st != TS_OK) return st;
    Ctrl h;
    st = read_ctrl(c, &h);
    if (st != TS_OK) return st;
    out->steps = h.steps_run;
    out->vehicle_updates = h.tot_updates;
    out->lane_changes = h.tot_lane_changes;
    out->transfers = h.tot_transfers;
    out->inserted = h.inserted;
    out->arrived = h.arrived;
    out->last_state_hash = h.hash;
    out->moving = h.tot_moving;
    out->active = h.tot_active;
    return TS_OK;
}

ts_status ts_read_link_times(ts_ctx *c, uint64_t *sum, uint64_t *count, uint32_t timeout_ms) {
    ts_status st = check_ctx(c);
    if (st != TS_OK) return st;
    if (!sum || !count) return fail(TS_ERR_INVALID, "null output");
    st = wait_ctx(c, timeout_ms);
    if (st != TS_OK) return st;
    Ctrl h;
    st = read_ctrl(c, &h);  // reports device consistency failures
    if (st != TS_OK) return st;
    CK(cudaMemcpyAsync(c->d_lt_tmp, c->sd.link_time, 8ull * c->n_links, cudaMemcpyDeviceToDevice, c->stream));
    if (c->n_veh) launch_link_time_fix(c->sd, c->n_veh, c->d_lt_tmp, c->stream);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(sum, c->d_lt_tmp, 8ull * c->n_links, cudaMemcpyDeviceToHost, c->stream));
    st = sync_stream(c->stream, timeout_ms);
    if (st != TS_OK) return st;
    for (uint32_t l = 0; l < c->n_links; ++l) {
        count[l] = sum[l] >> 40;
        sum[l] &= kLinkTimeOne - 1ull;
    }
    return TS_OK;
}

ts_status ts_state_sizes(const ts_ctx *c, uint64_t *cells, uint32_t *lanes, uint32_t *veh, uint32_t *links) {
    if (!c) return fail(TS_ERR_INVALID, "null context");
    if (cells) *cells = c->n_lane_cells;
    if (lanes) *lanes = c->n_lanes;
    if (veh) *veh = c->n_veh;
    if (links) *links = c->n_links;
    return TS_OK;
}

ts_status ts_read_state(ts_ctx *c, ts_state *o, uint32_t timeout_ms) {
    ts_status st = check_ctx(c);
    if (st != TS_OK) return st;
    if (!c->loaded) return fail(TS_ERR_STATE, "no vehicles loaded");
    if (!o || !o->cell_id || !o->cell_v || !o->buf_id || !o->buf_v || !o->cursor || !o->dep_head)
        return fail(TS_ERR_INVALID, "null state array");
    st = wait_ctx(c, timeout_ms);
    if (st != TS_OK) return st;
    Ctrl h;
    st = read_ctrl(c, &h);
    if (st != TS_OK) return st;
    const int cur = (int)(h.base & 1ull);
    const size_t nw = c->n_words;
    std::vector<uint32_t> occ(nw), loc(nw), vid0(nw * 32), vid1(nw * 32);
    std::vector<uint2> head(c->n_links);
    std::vector<int8_t> vel0(nw * 32), vel1(nw * 32);
    std::vector<uint4> slots(c->n_slots);
    std::vector<uint2> veh(c->n_veh);
    CK(cudaMemcpy(occ.data(), c->sd.occ[cur], 4 * nw, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(loc.data(), c->sd.loc[cur], 4 * nw, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(vel0.data(), c->sd.vel[0], nw * 32, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(vel1.data(), c->sd.vel[1], nw * 32, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(vid0.data(), c->sd.vid[0], 4 * nw * 32, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(vid1.data(), c->sd.vid[1], 4 * nw * 32, cudaMemcpyDeviceToHost));
    if (c->n_slots) CK(cudaMemcpy(slots.data(), c->sd.slots[cur], 16ull * c->n_slots, cudaMemcpyDeviceToHost));
    if (c->n_veh) CK(cudaMemcpy(veh.data(), c->sd.veh, 8ull * c->n_veh, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(head.data(), c->sd.dep_head, 8ull * c->n_links, cudaMemcpyDeviceToHost));
    for (uint64_t i = 0; i < c->n_lane_cells; ++i) {
        o->cell_id[i] = -1;
        o->cell_v[i] = 0;
    }
    for (uint32_t i = 0; i < c->n_lanes; ++i) {
        o->buf_id[i] = -1;
        o->buf_v[i] = 0;
    }
    for (uint32_t l = 0; l < c->n_links; ++l) {
        const uint32_t nl = c->lanes[l];
        for (uint32_t j = 0; j < c->ncols[l]; ++j)
            for (uint32_t k = 0; k < nl; ++k) {
                const size_t w = (size_t)c->wbase[l] + (size_t)j * nl + k;
                uint32_t m = occ[w];
                while (m) {
                    const int b = __builtin_ctz(m);
                    m &= m - 1;
                    const uint64_t x = 32ull * j + (uint64_t)b;
                    if (x >= c->cells[l]) return fail(TS_ERR_DEVICE_CHECK, "occupancy bit past the link end");
                    const uint64_t ci = c->cell_base[c->lane_base[l] + k] + x;
                    const bool b1 = (loc[w] >> b) & 1u;
                    o->cell_id[ci] = (int32_t)((b1 ? vid1 : vid0)[w * 32 + b] & kIdMask);
                    o->cell_v[ci] = (int8_t)((b1 ? vel1 : vel0)[w * 32 + b] & 0x0F);  // v (not the allowed lanes)
                }
            }
        if (!c->ring[l])
            for (uint32_t k = 0; k < nl; ++k) {
                const uint4 s = slots[c->bpos[l] + k];
                if (s.x == kSlotEmpty) continue;
                o->buf_id[c->lane_base[l] + k] = (int32_t)(s.x & kIdMask);
                o->buf_v[c->lane_base[l] + k] = (int8_t)(s.w & 0x0Fu);
            }
    }
    for (uint32_t i = 0; i < c->n_veh; ++i) o->cursor[i] = veh[i].x - c->route_off[i];
    for (uint32_t l = 0; l < c->n_links; ++l) o->dep_head[l] = head[l].x - c->dep_off[l];
    o->step = h.base;
    o->arrived = h.arrived;
    o->inserted = h.inserted;
    return TS_OK;
}

ts_status ts_write_state(ts_ctx *c, const ts_state *in) {
    ts_status st = check_ctx(c);
    if (st != TS_OK) return st;
    if (!c->loaded) return fail(TS_ERR_STATE, "no vehicles loaded");
    if (c->batch) return fail(TS_ERR_STATE, "context is in a batch");
    if (!in || !in->cell_id || !in->cell_v || !in->buf_id || !in->buf_v || !in->cursor || !in->dep_head)
        return fail(TS_ERR_INVALID, "null state array");
    st = wait_ctx(c, 60000);
    if (st != TS_OK) return st;
    if (c->route_links.size() != c->route_off[c->n_veh]) {  // host copy of the routes, once
        c->route_links.resize(c->route_off[c->n_veh]);
        if (!c->route_links.empty())
            CK(cudaMemcpy(c->route_links.data(), c->sd.route_links, 4ull * c->route_links.size(),
                          cudaMemcpyDeviceToHost));
    }
    const uint32_t vmax = c->params.vmax;
    const size_t nw = c->n_words;
    std::vector<uint32_t> occ(nw, 0), mov(nw, 0), vid(nw * 32, 0);
    uint64_t n_active = 0, n_buffered = 0, sum_v = 0, hash = 0;
    std::vector<int8_t> vel(nw * 32, 0);
    std::vector<uint4> slots(c->n_slots, make_uint4(kSlotEmpty, 0, 0, 0));
    std::vector<uint8_t> seen(c->n_veh, 0);
    std::vector<uint32_t> head(c->n_links);
    for (uint32_t i = 0; i < c->n_veh; ++i)
        if (in->cursor[i] >= c->route_off[i + 1] - c->route_off[i]) return fail(TS_ERR_INVALID, "cursor past route end");
    auto on_route = [&](int32_t id, uint32_t l) { return c->route_links[c->route_off[id] + in->cursor[id]] == l; };
    for (uint32_t l = 0; l < c->n_links; ++l) {
        const uint32_t nl = c->lanes[l];
        for (uint32_t k = 0; k < nl; ++k) {
            const uint64_t cb = c->cell_base[c->lane_base[l] + k];
            for (uint32_t x = 0; x < c->cells[l]; ++x) {
                const int32_t id = in->cell_id[cb + x];
                if (id < 0) continue;
                if ((uint32_t)id >= c->n_veh || seen[id]) return fail(TS_ERR_INVALID, "bad or repeated vehicle id");
                if (!on_route(id, l)) return fail(TS_ERR_INVALID, "vehicle not on the link its cursor names");
                const int8_t v = in->cell_v[cb + x];
                if (v < 0 || (uint32_t)v > vmax) return fail(TS_ERR_INVALID, "velocity out of range");
                seen[id] = 1;
                const size_t w = (size_t)c->wbase[l] + (size_t)(x / 32) * nl + k;
                occ[w] |= 1u << (x % 32);
                if (v) mov[w] |= 1u << (x % 32);
                const uint32_t al = c->has_turn ? c->route_turn[c->route_off[id] + in->cursor[id]] : 0u;
                vel[w * 32 + x % 32] = (int8_t)((uint32_t)v | (al << 4));
                const bool last = in->cursor[id] + 1 == c->route_off[id + 1] - c->route_off[id];
                vid[w * 32 + x % 32] = (uint32_t)id | (last ? kLastLinkBit : 0u);
                ++n_active;
                sum_v += (uint64_t)v;
                hash += vehicle_term((uint32_t)id, l, k, x, (uint32_t)v);
            }
            const int32_t b = in->buf_id[c->lane_base[l] + k];
            if (b >= 0) {
                if (c->ring[l]) return fail(TS_ERR_INVALID, "ring links have no link-end buffer");
                if ((uint32_t)b >= c->n_veh || seen[b]) return fail(TS_ERR_INVALID, "bad or repeated vehicle id");
                if (!on_route(b, l)) return fail(TS_ERR_INVALID, "vehicle not on the link its cursor names");
                const uint32_t len = c->route_off[b + 1] - c->route_off[b];
                if (in->cursor[b] + 1 >= len) return fail(TS_ERR_INVALID, "buffered vehicle on its last link");
                const int8_t v = in->buf_v[c->lane_base[l] + k];
                if (v < 0 || (uint32_t)v > vmax) return fail(TS_ERR_INVALID, "velocity out of range");
                seen[b] = 1;
                const uint32_t p = c->route_off[b] + in->cursor[b];
                const uint32_t fl = (in->cursor[b] + 2 == len) ? kLastLinkBit : 0u;
                const uint32_t al = c->has_turn ? c->route_turn[p + 1] : 0u;
                slots[c->bpos[l] + k] = make_uint4((uint32_t)b | fl, c->route_links[p + 1], l,
                                                   (uint32_t)v | (al << 4) | (k << 8) | (c->cells[l] << 10));
                ++n_buffered;
                hash += vehicle_term((uint32_t)b, l, k, c->cells[l], (uint32_t)v);
            }
        }
    }
    // vehicles on the network must already have left their departure queue
    for (uint32_t l = 0; l < c->n_links; ++l) {
        const uint32_t len = c->dep_off[l + 1] - c->dep_off[l];
        if (in->dep_head[l] > len) return fail(TS_ERR_INVALID, "dep_head beyond queue");
        head[l] = c->dep_off[l] + in->dep_head[l];
        for (uint32_t q = head[l]; q < c->dep_off[l + 1]; ++q)
            if (seen[c->dep_ids[q]]) return fail(TS_ERR_INVALID, "vehicle on the network is still queued");
    }
    std::vector<uint2> veh(c->n_veh);
    for (uint32_t i = 0; i < c->n_veh; ++i) veh[i] = make_uint2(c->route_off[i] + in->cursor[i], c->route_off[i + 1]);
    const int cur = (int)(in->step & 1ull);
    ScenDev &sd = c->sd;
    for (int b = 0; b < 2; ++b) {
        CK(cudaMemset(sd.occ[b], 0, 4 * nw));
        CK(cudaMemset(sd.mov[b], 0, 4 * nw));
        CK(cudaMemset(sd.loc[b], 0, 4 * nw));  // all payload in buffer 0
    }
    CK(cudaMemcpy(sd.occ[cur], occ.data(), 4 * nw, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(sd.mov[cur], mov.data(), 4 * nw, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(sd.vel[0], vel.data(), nw * 32, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(sd.vid[0], vid.data(), 4 * nw * 32, cudaMemcpyHostToDevice));
    if (c->n_slots) {
        CK(cudaMemset(sd.slots[cur ^ 1], 0xFF, 16ull * c->n_slots));
        CK(cudaMemcpy(sd.slots[cur], slots.data(), 16ull * c->n_slots, cudaMemcpyHostToDevice));
    }
    if (c->n_veh) {
        CK(cudaMemcpy(sd.veh, veh.data(), 8ull * c->n_veh, cudaMemcpyHostToDevice));
        // travel times restart: vehicles on the network count from the state's
        // step (entered then: - step on their link's sum)
        std::vector<uint32_t> enter(c->n_veh, kNotOnLink);
        std::vector<unsigned long long> lts(c->n_links, 0ull);
        for (uint32_t i = 0; i < c->n_veh; ++i)
            if (seen[i]) {
                enter[i] = (uint32_t)in->step;
                lts[c->route_links[veh[i].x]] -= in->step;
            }
        CK(cudaMemcpy(sd.enter_step, enter.data(), 4ull * c->n_veh, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(sd.link_time, lts.data(), 8ull * c->n_links, cudaMemcpyHostToDevice));
    } else {
        CK(cudaMemset(sd.link_time, 0, 8ull * c->n_links));
    }
    std::vector<uint2> heads(c->n_links);
    for (uint32_t l = 0; l < c->n_links; ++l) heads[l] = queue_head(c, l, head[l]);
    CK(cudaMemcpy(sd.dep_head, heads.data(), 8ull * c->n_links, cudaMemcpyHostToDevice));
    st = reset_ctrl(c, in->step, in->arrived, in->inserted, c->stream, n_active, n_buffered, sum_v, hash);
    if (st != TS_OK) return st;
    CK(cudaEventRecord(c->ev, c->stream));
    return TS_OK;
}

namespace {
struct CkptHeader {
    char magic[4];
    uint32_t format;
    uint64_t n_lane_cells;
    uint32_t n_lanes, n_veh, n_links, pad;
    uint64_t step, arrived, inserted;
    uint64_t reserved;
};
static_assert(sizeof(CkptHeader) == 64, "checkpoint header is 64 bytes");

size_t ckpt_bytes(const ts_ctx *c) {
    return sizeof(CkptHeader) + 4ull * c->n_lane_cells + 4ull * c->n_lanes + 4ull * c->n_veh +
           4ull * c->n_links + c->n_lane_cells + c->n_lanes;
}

// The arrays behind the header: the 4-byte ones first, then the 1-byte ones.
ts_state ckpt_view(const ts_ctx *c, unsigned char *base) {
    ts_state s{};
    unsigned char *p = base + sizeof(CkptHeader);
    s.cell_id = reinterpret_cast<int32_t *>(p);
    p += 4ull * c->n_lane_cells;
    s.buf_id = reinterpret_cast<int32_t *>(p);
    p += 4ull * c->n_lanes;
    s.cursor = reinterpret_cast<uint32_t *>(p);
    p += 4ull * c->n_veh;
    s.dep_head = reinterpret_cast<uint32_t *>(p);
    p += 4ull * c->n_links;
    s.cell_v = reinterpret_cast<int8_t *>(p);
    p += c->n_lane_cells;
    s.buf_v = reinterpret_cast<int8_t *>(p);
    return s;
}
}  // namespace

ts_status ts_save_state(ts_ctx *c, void *host, size_t *bytes, uint32_t timeout_ms) {
    if (!c || !bytes) return fail(TS_ERR_INVALID, "null argument");
    const size_t need = ckpt_bytes(c);
    if (!host) {
        *bytes = need;
        return TS_OK;
    }
    if (*bytes < need) return fail(TS_ERR_INVALID, "checkpoint buffer too small");
    unsigned char *base = static_cast<unsigned char *>(host);
    ts_state s = ckpt_view(c, base);
    const ts_status st = ts_read_state(c, &s, timeout_ms);
    if (st != TS_OK) return st;
    CkptHeader h{};
    memcpy(h.magic, "TSCK", 4);
    h.format = 1;
    h.n_lane_cells = c->n_lane_cells;
    h.n_lanes = c->n_lanes;
    h.n_veh = c->n_veh;
    h.n_links = c->n_links;
    h.step = s.step;
    h.arrived = s.arrived;
    h.inserted = s.inserted;
    memcpy(base, &h, sizeof(h));
    *bytes = need;
    return TS_OK;
}

ts_status ts_load_state(ts_ctx *c, const void *host, size_t bytes) {
    if (!c || !host) return fail(TS_ERR_INVALID, "null argument");
    CkptHeader h;
    if (bytes < sizeof(h)) return fail(TS_ERR_INVALID, "checkpoint too short");
    memcpy(&h, host, sizeof(h));
    if (memcmp(h.magic, "TSCK", 4) != 0 || h.format != 1) return fail(TS_ERR_INVALID, "not a checkpoint of format 1");
    if (h.n_lane_cells != c->n_lane_cells || h.n_lanes != c->n_lanes || h.n_veh != c->n_veh ||
        h.n_links != c->n_links || bytes < ckpt_bytes(c))
        return fail(TS_ERR_INVALID, "checkpoint of another network or vehicle set");
    ts_state s = ckpt_view(c, const_cast<unsigned char *>(static_cast<const unsigned char *>(host)));
    s.step = h.step;
    s.arrived = h.arrived;
    s.inserted = h.inserted;
    return ts_write_state(c, &s);
}

void ts_destroy(ts_ctx *c) {
    if (!c) return;
    cudaSetDevice(c->device);
    if (c->ev) cudaEventSynchronize(c->ev);
    if (c->stream) cudaStreamSynchronize(c->stream);
    delete c->own;
    if (c->d_base_tiles) cudaFree(c->d_base_tiles);
    if (c->d_cut_ok) cudaFree(c->d_cut_ok);
    free_list(c, c->veh_allocs);
    free_list(c, c->allocs);
    if (c->ev) cudaEventDestroy(c->ev);
    if (c->stream) cudaStreamDestroy(c->stream);
    delete c;
}

// ------------------------------------------------------------------ batching

ts_status ts_batch_create(uint32_t capacity, ts_batch **out) {
    if (!out || capacity == 0) return fail(TS_ERR_INVALID, "bad batch arguments");
    *out = nullptr;
    ts_batch *b = new (std::nothrow) ts_batch();
    if (!b) return fail(TS_ERR_OOM, "host allocation failed");
    ts_status st = b->w.init(capacity);
    if (st != TS_OK) {
        delete b;
        return st;
    }
    if (cudaEventCreateWithFlags(&b->ev, cudaEventDisableTiming) != cudaSuccess) {
        delete b;
        return cuda_fail(cudaGetLastError(), "cudaEventCreate");
    }
    cudaEventRecord(b->ev, b->w.cap_stream);
    *out = b;
    return TS_OK;
}

ts_status ts_batch_add_many(ts_batch *b, ts_ctx *const *ctxs, uint32_t n, uint64_t target_step) {
    if (!b || (n && !ctxs)) return fail(TS_ERR_INVALID, "null batch or contexts");
    ts_status st = wait_event(b->ev, 60000);  // the table is rewritten below
    if (st != TS_OK) return st;
    uint32_t free_slots = 0;
    for (ts_ctx *m : b->w.members) free_slots += m == nullptr;
    if (n > free_slots) return fail(TS_ERR_STATE, "batch is full");
    for (uint32_t i = 0; i < n; ++i) {
        ts_ctx *c = ctxs[i];
        st = check_ctx(c);
        if (st != TS_OK) return st;
        if (!c->loaded) return fail(TS_ERR_STATE, "no vehicles loaded");
        if (c->batch) return fail(TS_ERR_STATE, "context already in a batch");
        for (uint32_t j = 0; j < i; ++j)
            if (ctxs[j] == c) return fail(TS_ERR_INVALID, "context listed twice");
    }
    for (uint32_t i = 0; i < n; ++i) {
        ts_ctx *c = ctxs[i];
        st = wait_ctx(c, 60000);
        if (st != TS_OK) return st;
        CK(cudaMemcpy(&c->sd.ctrl->target, &target_step, sizeof(target_step), cudaMemcpyHostToDevice));
        uint32_t slot = 0;
        while (b->w.members[slot]) ++slot;
        b->w.members[slot] = c;
        c->batch = b;
    }
    return b->w.rebuild();
}

ts_status ts_batch_add(ts_batch *b, ts_ctx *c, uint64_t target_step) { return ts_batch_add_many(b, &c, 1, target_step); }

ts_status ts_batch_remove(ts_batch *b, ts_ctx *c) {
    if (!b || !c || c->batch != b) return fail(TS_ERR_INVALID, "context is not in this batch");
    ts_status st = wait_event(b->ev, 60000);
    if (st != TS_OK) return st;
    for (uint32_t s = 0; s < b->w.capacity; ++s)
        if (b->w.members[s] == c) b->w.members[s] = nullptr;
    c->batch = nullptr;
    Ctrl h;
    st = read_ctrl(c, &h);
    if (st != TS_OK) return st;
    c->host_step = h.base;
    return b->w.rebuild();
}

ts_status ts_batch_step(ts_batch *b, uint32_t n_steps, void *cuda_stream) {
    if (!b) return fail(TS_ERR_INVALID, "null batch");
    if (n_steps == 0) return TS_OK;
    CK(cudaSetDevice(b->w.device));
    cudaStream_t s = (cudaStream_t)cuda_stream;
    if (!s || s == b->w.cap_stream) return fail(TS_ERR_INVALID, "pass a stream to ts_batch_step");
    ts_status st = b->w.run(n_steps, s);
    if (st != TS_OK) return st;
    CK(cudaEventRecord(b->ev, s));
    for (ts_ctx *c : b->w.members)
        if (c) CK(cudaEventRecord(c->ev, s));
    return TS_OK;
}

ts_status ts_batch_reset(ts_batch *b, uint64_t target_step, void *cuda_stream) {
    if (!b) return fail(TS_ERR_INVALID, "null batch");
    CK(cudaSetDevice(b->w.device));
    cudaStream_t s = (cudaStream_t)cuda_stream;
    if (!s || s == b->w.cap_stream) return fail(TS_ERR_INVALID, "pass a stream to ts_batch_reset");
    for (ts_ctx *c : b->w.members) {
        if (!c) continue;
        if (c->sticky) return fail(TS_ERR_CUDA, "a member is in an error state");
        ts_status st = reset_device_state(c, s);
        if (st != TS_OK) return st;
        launch_set_target(c->sd.ctrl, target_step, s);
        c->host_step = 0;
    }
    CK(cudaGetLastError());
    CK(cudaEventRecord(b->ev, s));
    for (ts_ctx *c : b->w.members)
        if (c) CK(cudaEventRecord(c->ev, s));
    return TS_OK;
}

ts_status ts_batch_sync(ts_batch *b, uint32_t timeout_ms) {
    if (!b) return fail(TS_ERR_INVALID, "null batch");
    return wait_event(b->ev, timeout_ms);
}

ts_status ts_ctx_step(ts_ctx *c, uint64_t *step) {
    ts_status st = check_ctx(c);
    if (st != TS_OK) return st;
    if (!step) return fail(TS_ERR_INVALID, "null output");
    st = wait_ctx(c, 60000);
    if (st != TS_OK) return st;
    Ctrl h;
    st = read_ctrl(c, &h);
    if (st != TS_OK) return st;
    *step = h.base;
    return TS_OK;
}

void ts_batch_destroy(ts_batch *b) {
    if (!b) return;
    cudaSetDevice(b->w.device);
    if (b->ev) {
        cudaEventSynchronize(b->ev);
        cudaEventDestroy(b->ev);
    }
    for (ts_ctx *c : b->w.members)
        if (c) c->batch = nullptr;
    delete b;
}

}  // extern "C"
