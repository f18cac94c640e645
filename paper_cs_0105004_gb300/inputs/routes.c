/* Shortest-path route builder for synthetic trip demand (input generation).
 *
 * The micro-simulation takes each traveller's plan as a precomputed route:
 * the sequence of links from origin node to destination node (Sec. 1, the
 * "modal and route choice" module produces these plans; the router itself is
 * not part of the simulated step).  This file only builds such inputs.
 *
 * Route rule: Dijkstra on link length in cells; among equally short paths the
 * predecessor of every node is the tight predecessor with the smallest node
 * id.  That rule makes the tree unique, so the result does not depend on the
 * heap's pop order or on the number of threads.
 *
 * Work is split over distinct origins with POSIX threads; each origin's routes
 * go to a private buffer and are stitched together in trip order at the end.
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    uint32_t n_nodes, n_links;
    const uint32_t *from, *to, *w;
    uint32_t *adj_off, *adj_link; /* out-links per node (CSR) */
    uint64_t n_trips;
    const uint32_t *orig, *dest;
    const uint64_t *order;        /* trip indices sorted by origin */
    const uint64_t *grp_off;      /* group g = order[grp_off[g] .. grp_off[g+1]) */
    uint64_t n_groups;
    uint32_t *out_len;            /* per trip */
    uint32_t **grp_buf;           /* per group, concatenated routes of its trips */
    volatile int error;
    uint64_t next_group;
    pthread_mutex_t lock;
} job_t;

typedef struct { uint64_t d; uint32_t v; } hitem;

static void heap_push(hitem *h, uint64_t *n, hitem it) {
    uint64_t i = (*n)++;
    while (i > 0) {
        uint64_t p = (i - 1) / 2;
        if (h[p].d < it.d || (h[p].d == it.d && h[p].v <= it.v)) break;
        h[i] = h[p];
        i = p;
    }
    h[i] = it;
}

static hitem heap_pop(hitem *h, uint64_t *n) {
    hitem top = h[0];
    hitem last = h[--(*n)];
    uint64_t i = 0;
    for (;;) {
        uint64_t c = 2 * i + 1;
        if (c >= *n) break;
        if (c + 1 < *n && (h[c + 1].d < h[c].d || (h[c + 1].d == h[c].d && h[c + 1].v < h[c].v))) c++;
        if (last.d < h[c].d || (last.d == h[c].d && last.v <= h[c].v)) break;
        h[i] = h[c];
        i = c;
    }
    if (*n > 0) h[i] = last;
    return top;
}

static void *worker(void *arg) {
    job_t *J = (job_t *)arg;
    uint32_t N = J->n_nodes;
    uint64_t *dist = (uint64_t *)malloc(sizeof(uint64_t) * N);
    uint32_t *pred_link = (uint32_t *)malloc(sizeof(uint32_t) * N);
    uint32_t *hops = (uint32_t *)malloc(sizeof(uint32_t) * N);
    uint8_t *done = (uint8_t *)malloc(N);
    uint64_t cap = (uint64_t)J->n_links + N + 16;
    hitem *heap = (hitem *)malloc(sizeof(hitem) * cap);
    if (!dist || !pred_link || !hops || !done || !heap) { J->error = 1; goto out; }
    for (;;) {
        pthread_mutex_lock(&J->lock);
        uint64_t g = J->next_group++;
        pthread_mutex_unlock(&J->lock);
        if (g >= J->n_groups || J->error) break;
        uint64_t t0 = J->grp_off[g], t1 = J->grp_off[g + 1];
        uint32_t src = J->orig[J->order[t0]];
        for (uint32_t i = 0; i < N; i++) { dist[i] = UINT64_MAX; pred_link[i] = UINT32_MAX; done[i] = 0; }
        uint64_t hn = 0;
        dist[src] = 0; hops[src] = 0;
        heap_push(heap, &hn, (hitem){0, src});
        while (hn > 0) {
            hitem it = heap_pop(heap, &hn);
            uint32_t u = it.v;
            if (done[u] || it.d != dist[u]) continue;
            done[u] = 1;
            if (u != src) hops[u] = hops[J->from[pred_link[u]]] + 1;
            for (uint32_t a = J->adj_off[u]; a < J->adj_off[u + 1]; a++) {
                uint32_t l = J->adj_link[a];
                uint32_t v = J->to[l];
                uint64_t nd = dist[u] + J->w[l];
                if (nd < dist[v]) {
                    dist[v] = nd; pred_link[v] = l;
                    if (hn >= cap) { J->error = 2; goto out; }
                    heap_push(heap, &hn, (hitem){nd, v});
                } else if (nd == dist[v] && !done[v] && u < J->from[pred_link[v]]) {
                    pred_link[v] = l;
                }
            }
        }
        uint64_t total = 0;
        for (uint64_t q = t0; q < t1; q++) {
            uint32_t d = J->dest[J->order[q]];
            if (dist[d] == UINT64_MAX || d == src) { J->error = 3; goto out; }
            total += hops[d];
        }
        uint32_t *buf = (uint32_t *)malloc(sizeof(uint32_t) * (total ? total : 1));
        if (!buf) { J->error = 1; goto out; }
        uint64_t pos = 0;
        for (uint64_t q = t0; q < t1; q++) {
            uint64_t trip = J->order[q];
            uint32_t d = J->dest[trip];
            uint32_t h = hops[d];
            J->out_len[trip] = h;
            uint32_t v = d;
            for (uint32_t s = h; s > 0; s--) {
                uint32_t l = pred_link[v];
                buf[pos + s - 1] = l;
                v = J->from[l];
            }
            pos += h;
        }
        J->grp_buf[g] = buf;
    }
out:
    free(dist); free(pred_link); free(hops); free(done); free(heap);
    return NULL;
}

/* Builds routes for n_trips trips.  order/grp_off group the trips by origin
 * (trip order[grp_off[g]..grp_off[g+1]) share one origin).  On success writes
 * out_off[n_trips+1] (route offsets, trip order) and returns a malloc'd array
 * of route links through *out_links (free with routes_free).  Returns 0 on
 * success, 1 out of memory, 3 unreachable or origin == destination. */
int routes_build(uint32_t n_nodes, uint32_t n_links, const uint32_t *from, const uint32_t *to,
                 const uint32_t *w, uint64_t n_trips, const uint32_t *orig, const uint32_t *dest,
                 const uint64_t *order, const uint64_t *grp_off, uint64_t n_groups,
                 uint64_t *out_off, uint32_t **out_links, int n_threads) {
    job_t J;
    memset(&J, 0, sizeof(J));
    J.n_nodes = n_nodes; J.n_links = n_links; J.from = from; J.to = to; J.w = w;
    J.n_trips = n_trips; J.orig = orig; J.dest = dest; J.order = order; J.grp_off = grp_off;
    J.n_groups = n_groups;
    J.adj_off = (uint32_t *)calloc((size_t)n_nodes + 1, sizeof(uint32_t));
    J.adj_link = (uint32_t *)malloc(sizeof(uint32_t) * (n_links ? n_links : 1));
    J.out_len = (uint32_t *)calloc(n_trips ? n_trips : 1, sizeof(uint32_t));
    J.grp_buf = (uint32_t **)calloc(n_groups ? n_groups : 1, sizeof(uint32_t *));
    int rc = 0;
    if (!J.adj_off || !J.adj_link || !J.out_len || !J.grp_buf) { rc = 1; goto done; }
    for (uint32_t l = 0; l < n_links; l++) J.adj_off[from[l] + 1]++;
    for (uint32_t i = 0; i < n_nodes; i++) J.adj_off[i + 1] += J.adj_off[i];
    {
        uint32_t *fill = (uint32_t *)malloc(sizeof(uint32_t) * ((size_t)n_nodes + 1));
        if (!fill) { rc = 1; goto done; }
        memcpy(fill, J.adj_off, sizeof(uint32_t) * ((size_t)n_nodes + 1));
        for (uint32_t l = 0; l < n_links; l++) J.adj_link[fill[from[l]]++] = l;
        free(fill);
    }
    pthread_mutex_init(&J.lock, NULL);
    if (n_threads < 1) n_threads = 1;
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * n_threads);
    for (int i = 0; i < n_threads; i++) pthread_create(&th[i], NULL, worker, &J);
    for (int i = 0; i < n_threads; i++) pthread_join(th[i], NULL);
    free(th);
    pthread_mutex_destroy(&J.lock);
    if (J.error) { rc = J.error == 3 ? 3 : 1; goto done; }
    out_off[0] = 0;
    for (uint64_t t = 0; t < n_trips; t++) out_off[t + 1] = out_off[t] + J.out_len[t];
    {
        uint64_t total = out_off[n_trips];
        uint32_t *links = (uint32_t *)malloc(sizeof(uint32_t) * (total ? total : 1));
        if (!links) { rc = 1; goto done; }
        for (uint64_t g = 0; g < n_groups; g++) {
            uint64_t pos = 0;
            for (uint64_t q = grp_off[g]; q < grp_off[g + 1]; q++) {
                uint64_t trip = order[q];
                memcpy(links + out_off[trip], J.grp_buf[g] + pos, sizeof(uint32_t) * J.out_len[trip]);
                pos += J.out_len[trip];
            }
        }
        *out_links = links;
    }
done:
    if (J.grp_buf) for (uint64_t g = 0; g < n_groups; g++) free(J.grp_buf[g]);
    free(J.grp_buf); free(J.out_len); free(J.adj_off); free(J.adj_link);
    return rc;
}

void routes_free(uint32_t *p) { free(p); }
