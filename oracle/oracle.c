/* Plain CPU oracle of the TRANSIMS cellular-automaton time step.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header, table or constant with the CUDA library; it is written to be read
 * against the paper, not to be fast.
 *
 * Nagel & Rickert, "Parallel implementation of the TRANSIMS
 * micro-simulation", Sec. 3 (driving logic) and Sec. 4 (update order):
 *   - the road is a row of 7.5 m cells, each empty or holding one vehicle;
 *     vehicles move by hopping, one time step is 1 s (Sec. 3);
 *   - car following: (i) accelerate by one up to vmax, (ii) no faster than
 *     the free cells ahead allow (constant time headway), (iii) sometimes
 *     one slower at random (Sec. 3);
 *   - every step has two sub-steps: sideways lane changes first, then
 *     velocity update and forward motion (Sec. 3; Sec. 4's per-step order
 *     "change lanes, exchange, compute speed and move, exchange");
 *   - lane changes are symmetric: a reason to change (the other lane is
 *     faster) plus a check that the gap allows getting in (Sec. 3);
 *   - the interaction range on a link is 5 cells (Sec. 4);
 *   - vehicles enter from parking and leave to parking (Sec. 4) and follow
 *     precomputed routes (Sec. 1).
 * Where the paper leaves a detail open, this file takes one fixed reading
 * (velocity order accelerate/limit/slow down; lane-change direction +1 on
 * even steps and -1 on odd steps; gap to the link end counts one extra cell
 * when the lane's one-vehicle link-end buffer is free or the link is the
 * vehicle's last; fixed intersection priority by ascending incoming link id,
 * then lane; departures enter cell 0 of their first link with velocity 0).
 *
 * Randomness: the slowdown draw of vehicle `id` at step t is word 0 of
 * Philox-4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) with counter
 * (t, id, 0, 0) and key (seed low 32 bits, seed high 32 bits); the vehicle
 * slows down iff that word is below p_threshold.
 *
 * State digest: sum over vehicles on links of
 * splitmix64(A ^ splitmix64(B)) modulo 2^64, A = id<<32 | link,
 * B = cell<<16 | lane<<8 | v (a vehicle in a link-end buffer has cell =
 * link length); splitmix64 is the finaliser published by Steele, Lea and
 * Flood (OOPSLA 2014) applied to z + 0x9e3779b97f4a7c15.
 *
 * Traffic signals (Sec. 3): while the light at the end of link l is red, a
 * virtual vehicle of maximum velocity zero stands at the end of each of
 * its lanes, so the gap there counts no extra cell and no vehicle reaches
 * the end; l's lanes are green at step t iff (t + offset) mod cycle < green
 * (cycle 0: no signal).  A vehicle already in the link-end buffer crosses.
 *
 * Lane changing for plan following (Sec. 3: a driver who must turn at the
 * end of the link needs the right lane for it, and the gap such a driver
 * accepts shrinks as the intersection comes closer).  An optional turn
 * table lists, for every link l and every link m leaving l's end node
 * (ascending link id), the lanes of l from which a vehicle may continue
 * onto m (bit k = lane k).  A vehicle's allowed lanes are those of the turn
 * to the next link of its route (all lanes on its last link, or without a
 * table).  Readings: the extra cell at the link end is open only from an
 * allowed lane (from any other lane the end is closed, as at a red light);
 * a vehicle outside its allowed lanes has a reason to change when an
 * allowed lane lies on the side the step's direction points to, and then
 * needs the target cell and only the min(vmax, dist) cells behind it
 * empty, dist = cells between it and the link's last cell; the speed reason
 * applies only into an allowed lane.
 *
 * Gap acceptance at unprotected turns (Sec. 3: a car from the non-priority
 * street needs a large enough gap on the priority street).  An optional
 * per-link acceptance gap G (0: a priority approach, 1..31: a yield
 * approach): a vehicle in the link-end buffer of a yield approach crosses
 * only while every priority approach of the same node has no vehicle in
 * its last G cells (not counting its cell 0) on any lane, in the state
 * after the step's moves and before any transfer; it still needs a free
 * cell 0.  A node serves its priority approaches first, then its yield
 * approaches, each in ascending link id and lane.
 *
 * Link travel times (the input of the re-planning step of the relaxation
 * iterations, Sec. 1): a vehicle that enters a link at the end of step t0
 * (a departure or a node transfer) and leaves it at the end of step t1 (a
 * node transfer to its next link) or arrives during step t1 adds t1 - t0 to
 * that link's travel-time sum and 1 to its count.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define NONE_NODE 0xFFFFFFFFu

typedef struct {
    uint64_t step, active, buffered, waiting, arrived, lane_changes, transfers, inserted,
        sum_v, vehicle_updates, state_hash, moving;
} oracle_stats;

typedef struct oracle {
    /* network */
    uint32_t n_nodes, n_links, n_lanes;
    uint64_t n_cells;
    uint32_t *from, *to, *cells, *lanes;
    uint8_t *ring;
    uint32_t *sig;        /* [3 * n_links] signal cycle, green, offset (all 0: none) */
    uint8_t *turn;        /* turn table (NULL: every lane for every turn)  */
    uint32_t *turn_off;   /* first turn-table entry of each link          */
    uint32_t *out_off, *out_link; /* per node: outgoing links, ascending id */
    uint8_t *gap_accept;  /* [n_links] acceptance gap G of a yield approach, 0: priority */
    uint64_t t_now;       /* step being computed (for the signals)        */
    uint32_t *lane_base;  /* first canonical lane of each link            */
    uint32_t *lane_link;  /* link of each canonical lane                  */
    uint64_t *cell_base;  /* first canonical cell of each canonical lane  */
    uint32_t *in_off, *in_lane; /* per node: incoming lanes, priority order */
    /* parameters */
    uint32_t vmax, p_threshold, lane_change;
    uint64_t seed;
    /* vehicles */
    uint32_t n_veh;
    uint32_t *depart, *route_off, *route;
    uint32_t *q_off, *q_id; /* per link: departure queue sorted by (depart, id) */
    /* state */
    int32_t *cell;       /* [n_cells] vehicle id or -1 */
    int32_t *buf;        /* [n_lanes] vehicle id in the link-end buffer or -1 */
    int32_t *vel;        /* [n_veh] */
    uint32_t *cursor;    /* [n_veh] index of the current link in the route */
    uint8_t *status;     /* [n_veh] 0 not yet on the network, 1 on a link, 2 arrived */
    uint32_t *dep_head;  /* [n_links] queue entries already inserted */
    uint64_t step, arrived, inserted;
    uint32_t *t_enter;   /* [n_veh] step at whose end the vehicle entered its current link */
    uint64_t *lt_sum, *lt_cnt; /* [n_links] travel-time sums and counts of completed traversals */
    /* scratch copies of the cell array */
    int32_t *s_start, *s_lc;
    int32_t *buf_start;
} oracle;

/* ------------------------------------------------------------ Philox-4x32-10 */
/* Multipliers and Weyl key increments as published by Salmon et al. (2011). */
static void philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; round++) {
        uint64_t p0 = (uint64_t)M0 * c0;
        uint64_t p1 = (uint64_t)M1 * c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        c0 = hi1 ^ c1 ^ k0;
        c1 = lo1;
        c2 = hi0 ^ c3 ^ k1;
        c3 = lo0;
        k0 += W0;
        k1 += W1;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

void oracle_philox4x32_10(const uint32_t *ctr, const uint32_t *key, uint32_t *out) {
    philox4x32_10(ctr, key, out);
}

static uint64_t splitmix64(uint64_t z) {
    z += 0x9e3779b97f4a7c15ull;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

uint64_t oracle_splitmix64(uint64_t z) { return splitmix64(z); }

static uint64_t vehicle_term(uint32_t id, uint32_t link, uint32_t lane, uint32_t cell, uint32_t v) {
    uint64_t a = ((uint64_t)id << 32) | link;
    uint64_t b = ((uint64_t)cell << 16) | ((uint64_t)lane << 8) | v;
    return splitmix64(a ^ splitmix64(b));
}

uint64_t oracle_vehicle_term(uint32_t id, uint32_t link, uint32_t lane, uint32_t cell, uint32_t v) {
    return vehicle_term(id, link, lane, cell, v);
}

/* ------------------------------------------------------------ helpers */
static uint64_t cell_index(const oracle *o, uint32_t l, uint32_t k, uint32_t x) {
    return o->cell_base[o->lane_base[l] + k] + x;
}

static int is_last_link(const oracle *o, int32_t id) {
    return o->cursor[id] + 1 == o->route_off[id + 1] - o->route_off[id];
}

/* Lanes of the vehicle's current link from which it may continue onto the
 * next link of its route: bit k = lane k. */
static uint32_t allowed_lanes(const oracle *o, int32_t id) {
    uint32_t l = o->route[o->route_off[id] + o->cursor[id]];
    uint32_t all = (1u << o->lanes[l]) - 1u;
    if (!o->turn || is_last_link(o, id)) return all;
    uint32_t m = o->route[o->route_off[id] + o->cursor[id] + 1];
    uint32_t n = o->to[l];
    for (uint32_t j = o->out_off[n]; j < o->out_off[n + 1]; j++)
        if (o->out_link[j] == m) return o->turn[o->turn_off[l] + (j - o->out_off[n])];
    abort(); /* the route is not connected: rejected when loaded */
}

static int is_green(const oracle *o, uint32_t l) {
    uint32_t cycle = o->sig[3 * l], green = o->sig[3 * l + 1], offset = o->sig[3 * l + 2];
    if (cycle == 0) return 1;
    return (o->t_now + offset) % cycle < green;
}

/* Free cells ahead of (l,k,x) in state S, at most vmax (Sec. 3 rule (ii);
 * Sec. 4: interaction range 5 cells).  There is no look-ahead across a
 * node; at the link end the gap counts one more cell when the light there
 * is green, the lane's link-end buffer is free or this is the vehicle's
 * last link, and the lane is one of the vehicle's allowed lanes. */
static uint32_t gap_ahead(const oracle *o, const int32_t *S, const int32_t *buf, uint32_t l, uint32_t k,
                          uint32_t x, int32_t id) {
    uint32_t L = o->cells[l];
    for (uint32_t i = 1; i <= o->vmax; i++) {
        uint32_t y = x + i;
        if (y >= L) {
            if (o->ring[l]) {
                y -= L;
            } else {
                uint32_t open = is_green(o, l) && ((buf[o->lane_base[l] + k] < 0) || is_last_link(o, id)) &&
                                ((allowed_lanes(o, id) >> k) & 1u);
                uint32_t g = i - 1 + open;
                return g < o->vmax ? g : o->vmax;
            }
        }
        if (S[cell_index(o, l, k, y)] >= 0) return i - 1;
    }
    return o->vmax;
}

/* Safety check of a lane change into (l,k,x): the target cell and the
 * `back` cells behind it must be empty (on a non-periodic link only the
 * cells that exist behind x). */
static int room_to_get_in(const oracle *o, const int32_t *S, uint32_t l, uint32_t k, uint32_t x, uint32_t back) {
    uint32_t L = o->cells[l];
    if (S[cell_index(o, l, k, x)] >= 0) return 0;
    for (uint32_t i = 1; i <= back; i++) {
        uint32_t y;
        if (i > x) {
            if (!o->ring[l]) break;
            y = x + L - i;
        } else {
            y = x - i;
        }
        if (S[cell_index(o, l, k, y)] >= 0) return 0;
    }
    return 1;
}

/* ------------------------------------------------------------ construction */
void oracle_destroy(oracle *o) {
    if (!o) return;
    free(o->from); free(o->to); free(o->cells); free(o->lanes); free(o->ring); free(o->sig);
    free(o->turn); free(o->turn_off); free(o->out_off); free(o->out_link); free(o->gap_accept);
    free(o->lane_base); free(o->lane_link); free(o->cell_base); free(o->in_off); free(o->in_lane);
    free(o->depart); free(o->route_off); free(o->route); free(o->q_off); free(o->q_id);
    free(o->cell); free(o->buf); free(o->vel); free(o->cursor); free(o->status); free(o->dep_head);
    free(o->t_enter); free(o->lt_sum); free(o->lt_cnt);
    free(o->s_start); free(o->s_lc); free(o->buf_start);
    free(o);
}

/* Returns NULL on invalid input or out of memory. */
oracle *oracle_create(uint32_t n_nodes, uint32_t n_links, const uint32_t *from, const uint32_t *to,
                      const uint32_t *cells, const uint32_t *lanes, const uint8_t *ring, const uint32_t *signal,
                      const uint8_t *turn, const uint8_t *gap_accept, uint32_t vmax, uint32_t p_threshold,
                      uint64_t seed, uint32_t lane_change) {
    if (vmax < 1 || n_links == 0) return NULL;
    oracle *o = (oracle *)calloc(1, sizeof(oracle));
    if (!o) return NULL;
    o->n_nodes = n_nodes; o->n_links = n_links;
    o->vmax = vmax; o->p_threshold = p_threshold; o->seed = seed; o->lane_change = lane_change;
    o->from = (uint32_t *)malloc(4ull * n_links); o->to = (uint32_t *)malloc(4ull * n_links);
    o->cells = (uint32_t *)malloc(4ull * n_links); o->lanes = (uint32_t *)malloc(4ull * n_links);
    o->ring = (uint8_t *)calloc(n_links, 1);
    o->sig = (uint32_t *)calloc(3ull * n_links, 4);
    o->gap_accept = (uint8_t *)calloc(n_links, 1);
    o->lane_base = (uint32_t *)malloc(4ull * (n_links + 1));
    if (!o->from || !o->to || !o->cells || !o->lanes || !o->ring || !o->sig || !o->gap_accept || !o->lane_base)
        goto fail;
    if (gap_accept) {
        memcpy(o->gap_accept, gap_accept, n_links);
        for (uint32_t l = 0; l < n_links; l++)
            if (o->gap_accept[l] > 31) goto fail;
    }
    if (signal) {
        memcpy(o->sig, signal, 12ull * n_links);
        for (uint32_t l = 0; l < n_links; l++)
            if (o->sig[3 * l] && o->sig[3 * l + 1] > o->sig[3 * l]) goto fail;
    }
    memcpy(o->from, from, 4ull * n_links); memcpy(o->to, to, 4ull * n_links);
    memcpy(o->cells, cells, 4ull * n_links); memcpy(o->lanes, lanes, 4ull * n_links);
    if (ring) memcpy(o->ring, ring, n_links);
    o->lane_base[0] = 0;
    for (uint32_t l = 0; l < n_links; l++) {
        if (lanes[l] < 1 || cells[l] < 1) goto fail;
        if (o->ring[l]) {
            if (cells[l] <= vmax) goto fail;
        } else if (from[l] >= n_nodes || to[l] >= n_nodes) {
            goto fail;
        }
        o->lane_base[l + 1] = o->lane_base[l] + lanes[l];
    }
    o->n_lanes = o->lane_base[n_links];
    o->cell_base = (uint64_t *)malloc(8ull * (o->n_lanes + 1));
    o->lane_link = (uint32_t *)malloc(4ull * (o->n_lanes ? o->n_lanes : 1));
    if (!o->cell_base || !o->lane_link) goto fail;
    for (uint32_t l = 0; l < n_links; l++)
        for (uint32_t k = 0; k < lanes[l]; k++) o->lane_link[o->lane_base[l] + k] = l;
    o->cell_base[0] = 0;
    for (uint32_t l = 0; l < n_links; l++)
        for (uint32_t k = 0; k < lanes[l]; k++) {
            uint32_t ln = o->lane_base[l] + k;
            o->cell_base[ln + 1] = o->cell_base[ln] + cells[l];
        }
    o->n_cells = o->cell_base[o->n_lanes];
    /* incoming lanes of every node: priority approaches, then yield
     * approaches, each in ascending link id, lanes ascending */
    o->in_off = (uint32_t *)calloc((size_t)n_nodes + 1, 4);
    o->in_lane = (uint32_t *)malloc(4ull * (o->n_lanes ? o->n_lanes : 1));
    if (!o->in_off || !o->in_lane) goto fail;
    for (uint32_t l = 0; l < n_links; l++)
        if (!o->ring[l]) o->in_off[to[l] + 1] += lanes[l];
    for (uint32_t n = 0; n < n_nodes; n++) o->in_off[n + 1] += o->in_off[n];
    {
        uint32_t *fill = (uint32_t *)malloc(4ull * (n_nodes + 1));
        if (!fill) goto fail;
        memcpy(fill, o->in_off, 4ull * (n_nodes + 1));
        for (int yield = 0; yield < 2; yield++)
            for (uint32_t l = 0; l < n_links; l++)
                if (!o->ring[l] && (o->gap_accept[l] > 0) == yield)
                    for (uint32_t k = 0; k < lanes[l]; k++) o->in_lane[fill[to[l]]++] = o->lane_base[l] + k;
        free(fill);
    }
    /* outgoing links of every node, ascending id, and the turn table */
    o->out_off = (uint32_t *)calloc((size_t)n_nodes + 1, 4);
    o->out_link = (uint32_t *)malloc(4ull * n_links);
    o->turn_off = (uint32_t *)malloc(4ull * (n_links + 1));
    if (!o->out_off || !o->out_link || !o->turn_off) goto fail;
    for (uint32_t l = 0; l < n_links; l++)
        if (!o->ring[l]) o->out_off[from[l] + 1]++;
    for (uint32_t n = 0; n < n_nodes; n++) o->out_off[n + 1] += o->out_off[n];
    {
        uint32_t *fill = (uint32_t *)malloc(4ull * (n_nodes + 1));
        if (!fill) goto fail;
        memcpy(fill, o->out_off, 4ull * (n_nodes + 1));
        for (uint32_t l = 0; l < n_links; l++)
            if (!o->ring[l]) o->out_link[fill[from[l]]++] = l;
        free(fill);
    }
    o->turn_off[0] = 0;
    for (uint32_t l = 0; l < n_links; l++)
        o->turn_off[l + 1] = o->turn_off[l] + (o->ring[l] ? 0 : o->out_off[to[l] + 1] - o->out_off[to[l]]);
    if (turn) {
        o->turn = (uint8_t *)malloc(o->turn_off[n_links] ? o->turn_off[n_links] : 1);
        if (!o->turn) goto fail;
        memcpy(o->turn, turn, o->turn_off[n_links]);
        for (uint32_t l = 0; l < n_links; l++)
            for (uint32_t j = o->turn_off[l]; j < o->turn_off[l + 1]; j++)
                if (o->turn[j] == 0 || o->turn[j] >> lanes[l]) goto fail; /* no lane, or a lane l lacks */
    }
    o->cell = (int32_t *)malloc(4ull * o->n_cells);
    o->s_start = (int32_t *)malloc(4ull * o->n_cells);
    o->s_lc = (int32_t *)malloc(4ull * o->n_cells);
    o->buf = (int32_t *)malloc(4ull * o->n_lanes);
    o->buf_start = (int32_t *)malloc(4ull * o->n_lanes);
    o->dep_head = (uint32_t *)calloc(n_links, 4);
    o->lt_sum = (uint64_t *)calloc(n_links, 8);
    o->lt_cnt = (uint64_t *)calloc(n_links, 8);
    if (!o->cell || !o->s_start || !o->s_lc || !o->buf || !o->buf_start || !o->dep_head || !o->lt_sum || !o->lt_cnt)
        goto fail;
    for (uint64_t i = 0; i < o->n_cells; i++) o->cell[i] = -1;
    for (uint32_t i = 0; i < o->n_lanes; i++) o->buf[i] = -1;
    return o;
fail:
    oracle_destroy(o);
    return NULL;
}

/* Loads n travellers: departure step and route (list of links).  Each
 * route must be a connected path; a route on a periodic link has exactly
 * that one link.  Returns 0, or -1 on invalid input / out of memory. */
int oracle_load_vehicles(oracle *o, uint32_t n, const uint32_t *depart, const uint32_t *route_off,
                         const uint32_t *route) {
    uint64_t total = route_off[n];
    o->n_veh = n;
    o->depart = (uint32_t *)malloc(4ull * (n ? n : 1));
    o->route_off = (uint32_t *)malloc(4ull * (n + 1));
    o->route = (uint32_t *)malloc(4ull * (total ? total : 1));
    o->vel = (int32_t *)calloc(n ? n : 1, 4);
    o->cursor = (uint32_t *)calloc(n ? n : 1, 4);
    o->t_enter = (uint32_t *)calloc(n ? n : 1, 4);
    o->status = (uint8_t *)calloc(n ? n : 1, 1);
    o->q_off = (uint32_t *)calloc((size_t)o->n_links + 1, 4);
    o->q_id = (uint32_t *)malloc(4ull * (n ? n : 1));
    if (!o->depart || !o->route_off || !o->route || !o->vel || !o->cursor || !o->t_enter || !o->status ||
        !o->q_off || !o->q_id)
        return -1;
    memcpy(o->depart, depart, 4ull * n);
    memcpy(o->route_off, route_off, 4ull * (n + 1));
    memcpy(o->route, route, 4ull * total);
    for (uint32_t i = 0; i < n; i++) {
        uint32_t a = route_off[i], b = route_off[i + 1];
        if (b <= a) return -1;
        for (uint32_t j = a; j < b; j++) {
            if (route[j] >= o->n_links) return -1;
            if (o->ring[route[j]] && b - a != 1) return -1;
            if (j + 1 < b && o->to[route[j]] != o->from[route[j + 1]]) return -1;
        }
        o->q_off[route[a] + 1]++;
    }
    for (uint32_t l = 0; l < o->n_links; l++) o->q_off[l + 1] += o->q_off[l];
    /* insertion sort per link would be slow; a counting fill then a plain
     * per-link sort by (depart, id) */
    uint32_t *fill = (uint32_t *)malloc(4ull * (o->n_links + 1));
    if (!fill) return -1;
    memcpy(fill, o->q_off, 4ull * (o->n_links + 1));
    for (uint32_t i = 0; i < n; i++) o->q_id[fill[route[route_off[i]]]++] = i;
    free(fill);
    for (uint32_t l = 0; l < o->n_links; l++) {
        uint32_t a = o->q_off[l], b = o->q_off[l + 1];
        /* ids are already ascending within the link; a stable sort by depart
         * gives (depart, id) order */
        uint32_t len = b - a;
        if (len < 2) continue;
        uint32_t *tmp = (uint32_t *)malloc(4ull * len);
        if (!tmp) return -1;
        /* merge sort (stable) */
        for (uint32_t width = 1; width < len; width *= 2) {
            for (uint32_t lo = 0; lo < len; lo += 2 * width) {
                uint32_t mid = lo + width < len ? lo + width : len;
                uint32_t hi = lo + 2 * width < len ? lo + 2 * width : len;
                uint32_t i = lo, j = mid, k = lo;
                while (i < mid && j < hi)
                    tmp[k++] = (o->depart[o->q_id[a + j]] < o->depart[o->q_id[a + i]]) ? o->q_id[a + j++] : o->q_id[a + i++];
                while (i < mid) tmp[k++] = o->q_id[a + i++];
                while (j < hi) tmp[k++] = o->q_id[a + j++];
            }
            memcpy(o->q_id + a, tmp, 4ull * len);
        }
        free(tmp);
    }
    return 0;
}

/* Gap acceptance: may a vehicle leave yield approach l (gap G) at node n?
 * Every priority approach p of n must have its cells max(1, L_p - G) ..
 * L_p - 1 empty on every lane in the cell state S. */
static int priority_gap_clear(const oracle *o, const int32_t *S, uint32_t n, uint32_t l) {
    uint32_t G = o->gap_accept[l];
    for (uint32_t p = 0; p < o->n_links; p++) {
        if (o->ring[p] || o->to[p] != n || o->gap_accept[p] != 0) continue;
        uint32_t L = o->cells[p];
        uint32_t lo = L > G ? L - G : 1;
        for (uint32_t k = 0; k < o->lanes[p]; k++)
            for (uint32_t x = lo; x < L; x++)
                if (S[cell_index(o, p, k, x)] >= 0) return 0;
    }
    return 1;
}

/* ------------------------------------------------------------ one time step */
static void step_once(oracle *o, oracle_stats *st) {
    const uint64_t t = o->step;
    const int d = (t % 2 == 0) ? +1 : -1;
    o->t_now = t;
    const uint32_t vmax = o->vmax;
    memset(st, 0, sizeof(*st));

    /* Sub-step 1: lane changes, all decided on the start-of-step state S_t
     * and applied simultaneously.  Every mover goes the same way d and its
     * target cell is empty in S_t, so no two movers meet. */
    memcpy(o->s_start, o->cell, 4ull * o->n_cells);
    memcpy(o->s_lc, o->cell, 4ull * o->n_cells);
    memcpy(o->buf_start, o->buf, 4ull * o->n_lanes);
    if (o->lane_change) {
        for (uint32_t l = 0; l < o->n_links; l++) {
            for (uint32_t k = 0; k < o->lanes[l]; k++) {
                int kt = (int)k + d;
                if (kt < 0 || kt >= (int)o->lanes[l]) continue;
                for (uint32_t x = 0; x < o->cells[l]; x++) {
                    int32_t id = o->s_start[cell_index(o, l, k, x)];
                    if (id < 0) continue;
                    uint32_t v = (uint32_t)o->vel[id];
                    uint32_t g_own = gap_ahead(o, o->s_start, o->buf_start, l, k, x, id);
                    uint32_t g_tgt = gap_ahead(o, o->s_start, o->buf_start, l, (uint32_t)kt, x, id);
                    uint32_t want_v = v + 1 < vmax ? v + 1 : vmax;
                    /* plan following: outside the allowed lanes, with one of
                     * them on the side d points to */
                    uint32_t allowed = allowed_lanes(o, id);
                    int toward = 0;
                    for (uint32_t j = 0; j < o->lanes[l]; j++)
                        if (((allowed >> j) & 1u) && ((int)j - (int)k) * d > 0) toward = 1;
                    int plan = !((allowed >> k) & 1u) && toward;
                    /* the faster lane, if it is an allowed one */
                    int faster = g_own < want_v && g_tgt > g_own && ((allowed >> kt) & 1u);
                    /* the gap accepted behind: vmax cells, shrinking to 0 over
                     * the last vmax cells for a plan-following change */
                    uint32_t back = vmax;
                    if (plan && !o->ring[l] && o->cells[l] - 1 - x < back) back = o->cells[l] - 1 - x;
                    if ((plan || faster) && room_to_get_in(o, o->s_start, l, (uint32_t)kt, x, back)) {
                        o->s_lc[cell_index(o, l, k, x)] = -1;
                        o->s_lc[cell_index(o, l, (uint32_t)kt, x)] = id;
                        st->lane_changes++;
                    }
                }
            }
        }
    }

    /* Sub-step 2: velocity update on the post-lane-change state, then all
     * vehicles move at once.  Rules (i)-(iii) of Sec. 3 in that order. */
    for (uint64_t i = 0; i < o->n_cells; i++) o->cell[i] = -1;
    const uint32_t key[2] = {(uint32_t)o->seed, (uint32_t)(o->seed >> 32)};
    for (uint32_t l = 0; l < o->n_links; l++) {
        uint32_t L = o->cells[l];
        for (uint32_t k = 0; k < o->lanes[l]; k++) {
            for (uint32_t x = 0; x < L; x++) {
                int32_t id = o->s_lc[cell_index(o, l, k, x)];
                if (id < 0) continue;
                st->vehicle_updates++;
                uint32_t v = (uint32_t)o->vel[id] + 1;           /* (i) accelerate */
                if (v > vmax) v = vmax;
                uint32_t g = gap_ahead(o, o->s_lc, o->buf_start, l, k, x, id);
                if (v > g) v = g;                                /* (ii) headway   */
                if (v > 0) {                                     /* (iii) random   */
                    uint32_t ctr[4] = {(uint32_t)t, (uint32_t)id, 0u, 0u}, r[4];
                    philox4x32_10(ctr, key, r);
                    if (r[0] < o->p_threshold) v -= 1;
                }
                o->vel[id] = (int32_t)v;
                uint32_t nx = x + v;
                if (o->ring[l] && nx >= L) nx -= L;
                if (nx < L) {
                    uint64_t c = cell_index(o, l, k, nx);
                    if (o->cell[c] >= 0) abort(); /* two vehicles in one cell: a rule bug */
                    o->cell[c] = id;
                } else if (is_last_link(o, id)) {
                    o->status[id] = 2;                           /* to parking     */
                    o->arrived++;
                    o->lt_sum[l] += t - o->t_enter[id];
                    o->lt_cnt[l]++;
                } else {
                    uint32_t ln = o->lane_base[l] + k;
                    if (o->buf[ln] >= 0) abort();
                    o->buf[ln] = id;
                }
            }
        }
    }

    /* Node transfer: at every node, buffered vehicles in priority order
     * (priority approaches before yield approaches, then incoming link id
     * ascending, then lane) move to cell 0 of their next link, trying the
     * lane with the same index (or the highest one) first, then the other
     * lanes ascending.  A vehicle keeps its velocity; one that finds no free
     * cell 0, or leaves a yield approach while the priority approaches lack
     * the gap, stays in its buffer.  (The gap is judged on cells 1 and up,
     * which transfers never write: it is the state after the moves.) */
    for (uint32_t n = 0; n < o->n_nodes; n++) {
        for (uint32_t s = o->in_off[n]; s < o->in_off[n + 1]; s++) {
            uint32_t ln = o->in_lane[s];
            int32_t id = o->buf[ln];
            if (id < 0) continue;
            uint32_t l = o->lane_link[ln];
            uint32_t k = ln - o->lane_base[l];
            if (o->gap_accept[l] && !priority_gap_clear(o, o->cell, n, l)) continue;
            uint32_t m = o->route[o->route_off[id] + o->cursor[id] + 1];
            uint32_t nl = o->lanes[m];
            uint32_t pref = k < nl - 1 ? k : nl - 1;
            for (uint32_t tr = 0; tr < nl; tr++) {
                uint32_t q;
                if (tr == 0) q = pref;
                else q = (tr - 1 < pref) ? tr - 1 : tr;   /* remaining lanes ascending */
                uint64_t c = cell_index(o, m, q, 0);
                if (o->cell[c] < 0) {
                    o->cell[c] = id;
                    o->buf[ln] = -1;
                    o->cursor[id]++;
                    st->transfers++;
                    o->lt_sum[l] += t - o->t_enter[id];
                    o->lt_cnt[l]++;
                    o->t_enter[id] = (uint32_t)t;
                    break;
                }
            }
        }
    }

    /* Departures (entering from parking): per link, travellers whose
     * departure step has come, in (departure step, id) order, take the first
     * lane (ascending) whose cell 0 is free, with velocity 0, until the head
     * of the queue finds no free cell. */
    for (uint32_t m = 0; m < o->n_links; m++) {
        while (o->q_off[m] + o->dep_head[m] < o->q_off[m + 1]) {
            uint32_t id = o->q_id[o->q_off[m] + o->dep_head[m]];
            if (o->depart[id] > t) break;
            int placed = 0;
            for (uint32_t q = 0; q < o->lanes[m]; q++) {
                uint64_t c = cell_index(o, m, q, 0);
                if (o->cell[c] < 0) {
                    o->cell[c] = (int32_t)id;
                    o->vel[id] = 0;
                    o->cursor[id] = 0;
                    o->status[id] = 1;
                    o->t_enter[id] = (uint32_t)t;
                    placed = 1;
                    break;
                }
            }
            if (!placed) break;
            o->dep_head[m]++;
            o->inserted++;
            st->inserted++;
        }
    }

    /* Statistics of the state after step t. */
    st->step = t;
    st->arrived = o->arrived;
    for (uint32_t l = 0; l < o->n_links; l++) {
        for (uint32_t k = 0; k < o->lanes[l]; k++) {
            for (uint32_t x = 0; x < o->cells[l]; x++) {
                int32_t id = o->cell[cell_index(o, l, k, x)];
                if (id < 0) continue;
                st->active++;
                st->sum_v += (uint64_t)o->vel[id];
                if (o->vel[id] > 0) st->moving++;   /* in a cell and not standing */
                st->state_hash += vehicle_term((uint32_t)id, l, k, x, (uint32_t)o->vel[id]);
            }
            int32_t b = o->buf[o->lane_base[l] + k];
            if (b >= 0) {
                st->buffered++;
                st->state_hash += vehicle_term((uint32_t)b, l, k, o->cells[l], (uint32_t)o->vel[b]);
            }
        }
    }
    for (uint32_t i = 0; i < o->n_veh; i++)
        if (o->status[i] == 0 && o->depart[i] <= t) st->waiting++;
    o->step = t + 1;
}

/* Runs n steps; writes one stats record per step if out != NULL. */
int oracle_step(oracle *o, uint32_t n, oracle_stats *out) {
    oracle_stats st;
    for (uint32_t i = 0; i < n; i++) {
        step_once(o, &st);
        if (out) out[i] = st;
    }
    return 0;
}

/* ------------------------------------------------------------ canonical state */
uint64_t oracle_n_cells(const oracle *o) { return o->n_cells; }
uint32_t oracle_n_lanes(const oracle *o) { return o->n_lanes; }

/* Canonical state: cell_id/cell_v per lane-cell (link, lane, cell order;
 * -1 = empty), buf_id/buf_v per lane, cursor per vehicle, dep_head per
 * link, and scalars[0..2] = step, arrived, inserted. */
void oracle_get_state(const oracle *o, int32_t *cell_id, int8_t *cell_v, int32_t *buf_id, int8_t *buf_v,
                      uint32_t *cursor, uint32_t *dep_head, uint64_t *scalars) {
    for (uint64_t i = 0; i < o->n_cells; i++) {
        cell_id[i] = o->cell[i];
        cell_v[i] = o->cell[i] >= 0 ? (int8_t)o->vel[o->cell[i]] : 0;
    }
    for (uint32_t i = 0; i < o->n_lanes; i++) {
        buf_id[i] = o->buf[i];
        buf_v[i] = o->buf[i] >= 0 ? (int8_t)o->vel[o->buf[i]] : 0;
    }
    memcpy(cursor, o->cursor, 4ull * o->n_veh);
    memcpy(dep_head, o->dep_head, 4ull * o->n_links);
    scalars[0] = o->step; scalars[1] = o->arrived; scalars[2] = o->inserted;
}

/* Replaces the state.  A vehicle counts as on the network when it sits in a
 * cell or buffer, as arrived when its queue entry is below dep_head but it
 * is not on the network, and as not yet departed otherwise.  Returns -1 if
 * an id is out of range or appears twice. */
int oracle_set_state(oracle *o, const int32_t *cell_id, const int8_t *cell_v, const int32_t *buf_id,
                     const int8_t *buf_v, const uint32_t *cursor, const uint32_t *dep_head,
                     const uint64_t *scalars) {
    memset(o->status, 0, o->n_veh ? o->n_veh : 1);
    for (uint64_t i = 0; i < o->n_cells; i++) {
        int32_t id = cell_id[i];
        o->cell[i] = id;
        if (id < 0) continue;
        if ((uint32_t)id >= o->n_veh || o->status[id]) return -1;
        o->status[id] = 1;
        o->vel[id] = cell_v[i];
    }
    for (uint32_t i = 0; i < o->n_lanes; i++) {
        int32_t id = buf_id[i];
        o->buf[i] = id;
        if (id < 0) continue;
        if ((uint32_t)id >= o->n_veh || o->status[id]) return -1;
        o->status[id] = 1;
        o->vel[id] = buf_v[i];
    }
    memcpy(o->cursor, cursor, 4ull * o->n_veh);
    memcpy(o->dep_head, dep_head, 4ull * o->n_links);
    for (uint32_t m = 0; m < o->n_links; m++)
        for (uint32_t q = 0; q < dep_head[m] && o->q_off[m] + q < o->q_off[m + 1]; q++) {
            uint32_t id = o->q_id[o->q_off[m] + q];
            if (o->status[id] == 0) o->status[id] = 2;
        }
    o->step = scalars[0]; o->arrived = scalars[1]; o->inserted = scalars[2];
    /* travel times restart: vehicles on the network count from the state's step */
    for (uint32_t i = 0; i < o->n_veh; i++) o->t_enter[i] = (uint32_t)o->step;
    memset(o->lt_sum, 0, 8ull * o->n_links);
    memset(o->lt_cnt, 0, 8ull * o->n_links);
    return 0;
}

/* Travel-time sums and counts per link since creation or the last
 * set_state. */
void oracle_link_times(const oracle *o, uint64_t *sum, uint64_t *cnt) {
    memcpy(sum, o->lt_sum, 8ull * o->n_links);
    memcpy(cnt, o->lt_cnt, 8ull * o->n_links);
}
