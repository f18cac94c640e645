/* transsim.h -- C ABI of the GB300 TRANSIMS cellular-automaton step library.
 *
 * One time step of the TRANSIMS micro-simulation (Nagel & Rickert,
 * "Parallel implementation of the TRANSIMS micro-simulation"):
 *   1. lane change, a sideways move decided on the start-of-step state
 *      (Sec. 3: two sub-time-steps per step, lane changes first; symmetric
 *      rules made of a reason to change and a gap check);
 *   2. velocity update: accelerate by one up to vmax, limit to the free
 *      cells ahead (interaction range vmax = 5 cells, Sec. 3 and Sec. 4),
 *      random slowdown by one with probability p (Sec. 3 rule (iii));
 *   3. move: every vehicle hops v cells at once (Sec. 3); a vehicle that
 *      reaches the end of its link enters that lane's one-vehicle link-end
 *      buffer, or leaves to parking on the last link of its route (Sec. 4);
 *   4. node transfer: buffered vehicles move to cell 0 of the next link of
 *      their route in a fixed intersection priority (ascending incoming link
 *      id, then lane), then travellers whose departure time has come enter
 *      cell 0 of their first link from parking (Sec. 4).
 * The readings the paper leaves open are fixed as follows: lane-change
 * direction +1 on even steps and -1 on odd steps; a vehicle changes when
 * its own gap is below min(v+1, vmax) and the target lane's gap is larger,
 * and the target cell plus the vmax cells behind it are empty; at a link end
 * the gap counts one extra cell when the lane's buffer is empty or the link
 * is the vehicle's last; a transferred vehicle keeps its velocity and tries
 * the lane with its current index (capped to the next link's lanes) first,
 * then the others ascending; departures enter with velocity 0 in the first
 * free lane, in (departure step, id) order.
 * Options of the network (ts_network_desc): fixed-time signals at link
 * ends, turn lanes (plan-following lane changes) and yield approaches (gap
 * acceptance at unprotected turns), the intersection rules of Sec. 3; a
 * network without them runs exactly the rules above.
 * Randomness: vehicle `id` slows down at step t iff word 0 of
 * Philox-4x32-10 with counter (t, id, 0, 0) and key (seed & 0xffffffff,
 * seed >> 32) is below p_threshold, so results do not depend on the
 * parallel schedule and are bit-identical to a sequential implementation.
 *
 * Conventions for every call:
 *   - Every call returns ts_status.  TS_OK is 0.  Nothing aborts or throws
 *     across this boundary.  ts_last_error() gives a thread-local message.
 *   - After TS_ERR_CUDA or TS_ERR_DEVICE_CHECK a context is unusable
 *     ("sticky") except for ts_destroy.
 *   - Pointers named host_* or passed in descriptor structs are HOST
 *     pointers; the library deep-copies them before returning, so the
 *     caller may free them at once.  Device memory is owned by the context.
 *   - A context is used by one host thread at a time.
 *   - cuda_stream arguments are cudaStream_t values passed as void*; NULL
 *     means the context's own stream.  Stepping is asynchronous on that
 *     stream; read calls synchronise with a bounded wait.
 */
#ifndef TRANSSIM_H
#define TRANSSIM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ts_ctx ts_ctx;
typedef struct ts_batch ts_batch;

typedef enum {
    TS_OK = 0,
    TS_ERR_INVALID = 1,      /* bad argument or malformed network / routes / state */
    TS_ERR_OOM = 2,          /* device allocation failed                            */
    TS_ERR_CUDA = 3,         /* a CUDA runtime call failed (sticky)                 */
    TS_ERR_TIMEOUT = 4,      /* a bounded wait ran out; the work may still finish   */
    TS_ERR_STATE = 5,        /* call not valid in the current state                 */
    TS_ERR_DEVICE_CHECK = 6  /* a kernel found an impossible state (sticky)         */
} ts_status;

/* Driving-rule parameters (Sec. 3).  vmax in cells per 1 s step, 1..15
 * (5 = 135 km/h with 7.5 m cells).  p_threshold = floor(p * 2^32): the
 * random slowdown fires when the 32-bit Philox word is below it.
 * lane_change = 0 disables sub-step 1.  debug_checks is reserved (the
 * device-side consistency checks are always on). */
typedef struct {
    uint32_t vmax;
    uint32_t p_threshold;
    uint64_t seed;
    uint32_t lane_change;
    uint32_t debug_checks;
} ts_params;

/* Road network: directed links between nodes.  Link l runs from node
 * link_from[l] to node link_to[l], has link_cells[l] cells of 7.5 m
 * (1 .. 2^22 - 1) and link_lanes[l] lanes (1..4).  link_ring may be NULL; a
 * link with link_ring[l] = 1 is a periodic circle road (Sec. 5) with no
 * nodes: its from/to are ignored, it must not appear in a multi-link route,
 * and its cell count must be a multiple of 32.  Intersection priority is
 * ascending incoming link id, then lane. */
typedef struct {
    uint32_t n_nodes, n_links;
    const uint32_t *link_from, *link_to, *link_cells, *link_lanes;
    const uint8_t *link_ring;
    /* Optional (NULL: no signals): [3 * n_links] = per link (cycle, green,
     * offset), all below 2^16, green <= cycle.  A signal at the end of link l
     * (Sec. 3: a virtual vehicle of maximum velocity zero at the end of every
     * lane while the light is red): the lane ends are green at step t iff
     * (t + offset) mod cycle < green; cycle 0 = no signal.  While red, the
     * gap to the lane end counts no extra cell and no vehicle reaches the end
     * (neither the link-end buffer nor parking); a vehicle already in the
     * buffer crosses the node as usual. */
    const uint32_t *link_signal;
    /* Optional (NULL: any lane serves every turn): turn lanes for
     * plan-following lane changes (Sec. 3: a driver who turns at the end of
     * the link needs the right lane, and accepts a smaller gap to get there
     * the closer the intersection is).  For every non-ring link l in id
     * order, one byte per non-ring link m leaving node link_to[l], in
     * ascending id of m: bit k set = lane k of l may be used to continue
     * onto m.  Each byte must be non-zero and name only lanes l has
     * (TS_ERR_INVALID otherwise).  A vehicle's allowed lanes are those of
     * the turn onto the next link of its route (every lane on its last
     * link).  With a table: the extra cell at the link end is open only
     * from an allowed lane (from any other lane the end is closed, as at a
     * red light); a vehicle outside its allowed lanes has a reason to
     * change lanes when an allowed lane lies on the side the step's
     * direction points to, and then needs the target cell and the
     * min(vmax, cells left to the link's last cell) cells behind it empty;
     * the faster-lane reason applies only into an allowed lane. */
    const uint8_t *turn_lanes;
    /* Optional (NULL: every approach has priority): gap acceptance at
     * unprotected turns (Sec. 3: the car from the non-priority street needs
     * a large enough gap on the priority street).  [n_links] acceptance gap
     * G in cells, 0..31 (TS_ERR_INVALID above): 0 = link l's end is a
     * priority approach, G > 0 = a yield approach.  A vehicle in a link-end
     * buffer of a yield approach crosses only while every priority approach
     * of the same node has no vehicle in its last G cells on any lane
     * (cells max(1, cells - G) .. cells - 1, judged after the step's moves
     * and before any transfer); it still needs a free cell 0.  A node serves
     * its priority approaches first, then its yield approaches, each in
     * ascending link id and lane. */
    const uint8_t *link_yield;
} ts_network_desc;

/* Statistics of the state after step `step` (0-based).  active: vehicles
 * in cells; buffered: vehicles in link-end buffers; waiting: departure time
 * reached but not yet on a link; arrived: cumulative arrivals; lane_changes,
 * transfers (buffer -> next link), inserted (from parking): counts within
 * this step; sum_v: sum of velocities of vehicles in cells; vehicle_updates:
 * vehicles that went through the velocity update this step; moving:
 * vehicles in cells with v > 0 after the step (one standing in a jam has
 * v = 0, so moving / active is the share of traffic that flows);
 * state_hash: sum
 * modulo 2^64 over vehicles on links of splitmix64(A ^ splitmix64(B)),
 * A = id << 32 | link, B = cell << 16 | lane << 8 | v, with cell = link
 * length for a buffered vehicle (splitmix64 as published by Steele, Lea and
 * Flood, 2014). */
typedef struct {
    uint64_t step, active, buffered, waiting, arrived, lane_changes, transfers, inserted, sum_v,
        vehicle_updates, state_hash, moving;
} ts_stats;

/* Totals since the last ts_load_vehicles / ts_reset / ts_write_state:
 * steps run, vehicle updates, lane changes and transfers summed over those
 * steps; inserted and arrived are the cumulative counts of the state;
 * last_state_hash is the digest after the last step; moving and active are
 * the per-step counts of ts_stats summed over those steps. */
typedef struct {
    uint64_t steps, vehicle_updates, lane_changes, transfers, inserted, arrived, last_state_hash, moving, active;
} ts_totals;

/* Optional device-memory provider (for example a framework's caching
 * allocator).  alloc returns device memory of at least `bytes` bytes, 256-byte
 * aligned, or NULL; free releases it.  stream is the context stream. */
typedef struct {
    void *(*alloc)(size_t bytes, void *stream, void *user);
    void (*free)(void *ptr, size_t bytes, void *stream, void *user);
    void *user;
} ts_allocator;

/* Canonical host-side state, used to read a state out, to start from a
 * given state (ring experiments, checkpoints) and for parity checks.
 * cell_id/cell_v: one entry per lane-cell in (link, lane, cell) order,
 * -1 = empty.  buf_id/buf_v: one entry per lane in (link, lane) order.
 * cursor: index of each vehicle's current link within its route.
 * dep_head: per link, how many entries of its departure queue (ordered by
 * departure step, then id) have entered the network.  Sizes come from
 * ts_state_sizes.  All pointers are host pointers owned by the caller. */
typedef struct {
    int32_t *cell_id;
    int8_t *cell_v;
    int32_t *buf_id;
    int8_t *buf_v;
    uint32_t *cursor;
    uint32_t *dep_head;
    uint64_t step, arrived, inserted;
} ts_state;

/* Builds the device layout of one network on the current CUDA device.
 * desc arrays are host pointers, deep-copied.  allocator may be NULL
 * (cudaMalloc).  On success *out owns all device memory.  Errors:
 * TS_ERR_INVALID (lanes outside 1..4, too-short link, bad node id, ring
 * length not a multiple of 32, vmax outside 1..15), TS_ERR_OOM, TS_ERR_CUDA. */
ts_status ts_create_network(const ts_network_desc *desc, const ts_params *params,
                            const ts_allocator *allocator, ts_ctx **out);

/* Loads n travellers (once per context): host_depart_step[n],
 * host_route_offsets[n+1] (route i = host_route_links[offsets[i] ..
 * offsets[i+1])), each route a connected, non-empty list of link ids (Sec. 1:
 * plans come precomputed from the route-choice module).  Resets the state to
 * the empty network at step 0.  TS_ERR_INVALID on a malformed route or n
 * above 2^31-2. */
ts_status ts_load_vehicles(ts_ctx *ctx, uint32_t n, const uint32_t *host_depart_step,
                           const uint32_t *host_route_offsets, const uint32_t *host_route_links);

/* Enqueues n_steps time steps on cuda_stream (asynchronous; captured CUDA
 * graphs of the per-step kernels). */
ts_status ts_step(ts_ctx *ctx, uint32_t n_steps, void *cuda_stream);

/* Enqueues a return to the empty network at step 0 (all travellers back
 * in their departure queues) on cuda_stream, without host transfers. */
ts_status ts_reset(ts_ctx *ctx, void *cuda_stream);

/* Runs n_steps steps with plain launches (no graph) and a CUDA event around
 * each kernel; waits for them and writes the per-step durations of the
 * link kernel and the node kernel to host arrays link_ms[n], node_ms[n].
 * For measurement only. */
ts_status ts_step_timed(ts_ctx *ctx, uint32_t n_steps, void *cuda_stream, float *host_link_ms,
                        float *host_node_ms);

/* Waits (at most timeout_ms) for the context's queued work, then returns
 * the statistics of the last completed step.  TS_ERR_STATE before the first
 * step, TS_ERR_TIMEOUT if the wait runs out. */
ts_status ts_read_stats(ts_ctx *ctx, ts_stats *out, uint32_t timeout_ms);

/* Like ts_read_stats for steps first_step .. first_step+n-1 (the context
 * keeps the last 4096 steps).  TS_ERR_STATE if a step is not available. */
ts_status ts_read_stats_range(ts_ctx *ctx, uint64_t first_step, uint32_t n, ts_stats *out,
                              uint32_t timeout_ms);

/* Waits (bounded) and returns the run totals (see ts_totals). */
ts_status ts_read_totals(ts_ctx *ctx, ts_totals *out, uint32_t timeout_ms);

/* Number of lane-cells, lanes, vehicles and links of the canonical state. */
ts_status ts_state_sizes(const ts_ctx *ctx, uint64_t *n_lane_cells, uint32_t *n_lanes,
                         uint32_t *n_vehicles, uint32_t *n_links);

/* Copies the current state into caller-owned host arrays (bounded wait). */
ts_status ts_read_state(ts_ctx *ctx, ts_state *out, uint32_t timeout_ms);

/* Replaces the current state by a caller-given canonical state (host
 * arrays).  TS_ERR_INVALID if ids repeat, a vehicle sits on a link its
 * cursor does not name, or a velocity is outside 0..vmax. */
ts_status ts_write_state(ts_ctx *ctx, const ts_state *in);

/* Checkpoints as one byte buffer: the canonical state (ts_state) behind a
 * 64-byte header (magic "TSCK", format 1, the four sizes, step, arrived,
 * inserted).  ts_save_state with host == NULL sets *bytes to the size
 * needed; otherwise it fills host (*bytes must be at least that size) after
 * a bounded wait.  ts_load_state replaces the state like ts_write_state and
 * returns TS_ERR_INVALID for a buffer of another format or network. */
ts_status ts_save_state(ts_ctx *ctx, void *host, size_t *bytes, uint32_t timeout_ms);
ts_status ts_load_state(ts_ctx *ctx, const void *host, size_t bytes);

/* Device bytes a context would hold for a network of this shape with
 * n_vehicles travellers and route_len route entries in total (admission
 * control for the job server). */
size_t ts_footprint_bytes(const ts_network_desc *desc, uint32_t n_vehicles, uint64_t route_len);

/* Thread-local description of the last error. */
const char *ts_last_error(void);

/* The random draw of the velocity update (Sec. 3 rule (iii)) as the step
 * kernels make it: host_out[i] = word 0 of Philox-4x32-10 (Salmon, Moraes,
 * Dror, Shaw, SC'11) with counter (host_step[i], host_id[i], 0, 0) and key
 * (seed & 0xffffffff, seed >> 32); vehicle host_id[i] slows down at step
 * host_step[i] iff that word is below p_threshold.  For reproducing or
 * auditing draws.  Host arrays of n entries; runs on the current device and
 * returns when host_out is written.  TS_ERR_INVALID for a null array,
 * TS_ERR_OOM, TS_ERR_CUDA. */
ts_status ts_philox_words(uint32_t n, const uint32_t *host_step, const uint32_t *host_id, uint64_t seed,
                          uint32_t *host_out);

/* Frees the context and its device memory.  It first waits, without a
 * deadline, for the work queued on its stream (that work uses the memory it
 * frees); call ts_read_stats with a deadline first to bound the wait. */
void ts_destroy(ts_ctx *ctx);

/* ---- batching: many independent scenarios advanced by the same kernels.
 * A batch references contexts (it does not own them).  Every member
 * advances by one step per batch step until it reaches its own target step
 * (set by ts_batch_add / ts_batch_set_target); members that reached their
 * target are skipped.  Membership changes take effect at the next
 * ts_batch_step and need no re-capture. */
ts_status ts_batch_create(uint32_t capacity, ts_batch **out);
ts_status ts_batch_add(ts_batch *b, ts_ctx *ctx, uint64_t target_step);
/* Adds n contexts at once (one table rebuild). */
ts_status ts_batch_add_many(ts_batch *b, ts_ctx *const *ctxs, uint32_t n, uint64_t target_step);
ts_status ts_batch_remove(ts_batch *b, ts_ctx *ctx);
ts_status ts_batch_step(ts_batch *b, uint32_t n_steps, void *cuda_stream);
/* Enqueues, on cuda_stream, a return of every member to the empty network
 * at step 0 with the new target step; no host transfers, no rebuild. */
ts_status ts_batch_reset(ts_batch *b, uint64_t target_step, void *cuda_stream);
/* Waits (bounded) for the batch's queued work. */
ts_status ts_batch_sync(ts_batch *b, uint32_t timeout_ms);
/* Current step of a member (after ts_batch_sync). */
ts_status ts_ctx_step(ts_ctx *ctx, uint64_t *step);
/* Frees the batch (not its members); waits, without a deadline, for the
 * batch's queued work first (ts_batch_sync bounds that wait). */
void ts_batch_destroy(ts_batch *b);

/* Kernel launch shape: at most this many occupancy words (32-cell columns
 * times lanes) per warp tile, 8..256 (default 128); a warp tile also holds
 * at most 32 columns, so values from 128 up give the same tiles.  Results
 * do not depend on it.  ts_tile_words returns the current value. */
ts_status ts_set_tile_words(ts_ctx *ctx, uint32_t words);
uint32_t ts_tile_words(const ts_ctx *ctx);

/* Kernel launch shape: the link kernel's grid, at most blocks_per_sm
 * blocks (of four independent warps, each taking one warp tile at a time)
 * per SM, 1..64; 0 (default) = every block that can be resident, so each
 * warp takes about tiles / (resident warps) tiles in turn.  Results do not
 * depend on it.  Waits (bounded) for queued work; the graphs are captured
 * again.  TS_ERR_STATE for a context in a batch (set the batch's). */
ts_status ts_set_link_grid(ts_ctx *ctx, uint32_t blocks_per_sm);
ts_status ts_batch_set_link_grid(ts_batch *b, uint32_t blocks_per_sm);

/* Advances a periodic ring road held in caller-owned device buffers by
 * n_steps steps, without allocating any device memory.  The paper has no
 * counterpart to this call: it exists for callers that cannot let a
 * library allocate GPU memory (a framework that owns all device memory
 * through its own pool, a plugin given fixed buffers).  It runs the same
 * step kernel as ts_step on one ring link of `cells` cells (a multiple of
 * 32, at most 131072) and `lanes` lanes (1..4); n_steps at most 1024.
 * Layout of the caller's buffers, W = cells/32 * lanes words: dev_occ0/1
 * [W] uint32 occupancy words, word (column j, lane k) = j*lanes + k, bit i =
 * cell 32j+i; dev_vel0/1 [32*W] int8 velocities and dev_vid0/1 [32*W]
 * uint32 vehicle ids at word*32 + bit; ids must be below 2^31 (bit 31 is
 * the kernels' last-link flag: an id with it set is not checked and gives
 * undefined movement and statistics).  The state of step
 * first_step is read from buffer set (first_step & 1) and the state after
 * the last step is written to set ((first_step + n_steps) & 1); the other
 * set is overwritten.  dev_stats_out [n_steps] (device memory) receives the
 * statistics of steps first_step .. first_step+n_steps-1 (buffered, waiting,
 * arrived, transfers and inserted are 0 on a ring).  Asynchronous on
 * cuda_stream; device consistency flags are not reported by this call.
 * Scratch: a fixed array of about 900 KB in device memory, held by every
 * device that loads the library until the process exits.  All calls share
 * it, so calls that overlap on the GPU (other streams, other threads) race;
 * each call rewrites and clears what it uses.  The first call on a device
 * looks up the array's device address (cudaGetSymbolAddress), so make that
 * first call before any stream capture.  Returns TS_ERR_INVALID for sizes
 * beyond the limits above, TS_ERR_CUDA if a copy or launch fails. */
ts_status ts_ring_step_noalloc(uint32_t cells, uint32_t lanes, const ts_params *params, uint64_t first_step,
                               uint32_t n_steps, uint32_t *dev_occ0, uint32_t *dev_occ1, int8_t *dev_vel0,
                               int8_t *dev_vel1, uint32_t *dev_vid0, uint32_t *dev_vid1, ts_stats *dev_stats_out,
                               void *cuda_stream);

/* Step launch mode.  FUSED: one link-kernel launch per step, each also
 * completing the node transfers of the step before it (every tile resolves
 * the transfers that concern its own links; a node kernel completes the last
 * step of each chunk of up to 32 steps).  SPLIT: a link kernel and a node
 * kernel per step.  AUTO (default) is SPLIT: resolving an occupied buffer's
 * transfer inside the link kernel lengthens the step more than the saved
 * launch shortens it, except on nearly empty networks, where FUSED is
 * faster.  Results do not depend on the mode. */
enum { TS_STEP_AUTO = 0, TS_STEP_FUSED = 1, TS_STEP_SPLIT = 2 };
ts_status ts_set_step_mode(ts_ctx *ctx, uint32_t mode);
ts_status ts_batch_set_step_mode(ts_batch *b, uint32_t mode);

/* Load balancing (the counterpart of feeding measured per-link load back
 * into the partition): every `every_steps` steps of a ts_step call
 * (0 = never; otherwise at least 32) the link tiles are rebuilt from the
 * current occupancy so that a tile's load stays within `vehicles_per_tile`,
 * a moving vehicle counting 8 and a standing one 1 (standing vehicles are
 * mostly advanced 32 cells at a time, moving ones one by one) (0 = no
 * budget, else at least 32; a single column is never cut, so a tile may
 * exceed the budget by one column's load).  Each pass is a kernel enqueued on the step's
 * stream, so ts_step stays asynchronous.  Waits (bounded) for the context's
 * queued work; TS_ERR_STATE for a context in a batch.  Results do not
 * depend on it. */
ts_status ts_set_load_balance(ts_ctx *ctx, uint32_t every_steps, uint32_t vehicles_per_tile);

/* Kernel timing inside the captured step graphs, for measurement.  With
 * timing on, every link-kernel and node-kernel launch of ts_step records
 * when its work started (the first of its blocks past the wait for the
 * previous kernel) and ended (the last block's exit) on the GPU's global
 * nanosecond timer, and each chunk's closing kernel adds the durations up on
 * the device, so the kernels run exactly as in the untimed graphs apart
 * from two timer reads per block.  ts_set_kernel_timing waits (bounded) for
 * queued work and re-captures the graphs on its next ts_step.
 * ts_read_kernel_times waits (at most timeout_ms) and writes host_out[4] =
 * {link-kernel nanoseconds, link-kernel launches, node-kernel nanoseconds,
 * node-kernel launches} summed since timing was first switched on or last
 * reset (reset != 0 clears the sums after reading).  TS_ERR_STATE for a
 * context in a batch. */
ts_status ts_set_kernel_timing(ts_ctx *ctx, uint32_t on);
ts_status ts_read_kernel_times(ts_ctx *ctx, uint64_t *host_out, uint32_t reset, uint32_t timeout_ms);

/* Per-link travel times of completed link traversals since the last
 * ts_load_vehicles / ts_reset / ts_write_state: sum[l] = sum over vehicles
 * that left link l of (the step at whose end they left it by a node
 * transfer, or the step in which they arrived, minus the step at whose end
 * they entered it by a departure or a transfer), count[l] = their number.
 * Vehicles written by ts_write_state count from the state's step.  These
 * are the link costs that the re-planning between relaxation iterations
 * (Sec. 1) feeds back into the routes.  sum and count: host arrays of
 * n_links entries.  Between resets a link's sum must stay below 2^40 and
 * its count below 2^24 (the device keeps both in one 64-bit word).  Waits
 * for the context's queued work (at most timeout_ms; TS_ERR_TIMEOUT after
 * that). */
ts_status ts_read_link_times(ts_ctx *ctx, uint64_t *sum, uint64_t *count, uint32_t timeout_ms);

/* Number of kernel launches one time step enqueues in FUSED mode (1: the
 * link kernel, which also completes the node transfers of the step before
 * it; SPLIT mode adds the node kernel: 2).  On top, every chunk of up to 32
 * steps adds the chunk-closing kernel and, in FUSED mode, the node kernel
 * of its last step, and every ts_step call one launch (its target step). */
uint32_t ts_launches_per_step(void);

#ifdef __cplusplus
}
#endif
#endif
