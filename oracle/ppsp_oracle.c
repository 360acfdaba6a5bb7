/*
 * CPU oracle for exact point-to-point shortest paths.  TEST INFRASTRUCTURE ONLY:
 * the tests, the smoke check and the benchmark's CPU-baseline leg call it; the
 * library's query path never does.  It shares no code with the CUDA path.
 *
 * What it computes.  The paper's PPSP algorithms (Alg. 2 with the ET, A*, BiDS
 * and BiD-A* plug-ins of Table 2, and Multi-BiDS for batches, Sec. 4.2) return
 * exactly the shortest-path distance d(s,t) (Theorem 3.3 for BiDS, Theorem 3.4
 * for BiD-A*, on any stepping schedule).  The oracle is therefore the plain
 * definition of d(s,t): textbook binary-heap Dijkstra from s, stopped when t is
 * settled, with 64-bit unsigned sums.  Weights are non-negative integers
 * (paper Sec. 2 "Notations": w: E -> R+, here uint32).  Unreachable = UINT64_MAX.
 *
 * Also here: full single-source Dijkstra (with parent pointers, for paths and
 * multi-target checks) and Floyd-Warshall for brute-force checks on tiny graphs.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_INF UINT64_MAX

typedef struct {
    uint64_t key;
    uint32_t v;
} item_t;

typedef struct {
    item_t* a;
    uint64_t size, cap;
} heap_t;

static int heap_push(heap_t* h, uint64_t key, uint32_t v) {
    if (h->size == h->cap) {
        uint64_t nc = h->cap ? 2 * h->cap : 1024;
        item_t* na = (item_t*)realloc(h->a, nc * sizeof(item_t));
        if (!na) return -1;
        h->a = na;
        h->cap = nc;
    }
    uint64_t i = h->size++;
    while (i > 0) {
        uint64_t p = (i - 1) / 2;
        if (h->a[p].key <= key) break;
        h->a[i] = h->a[p];
        i = p;
    }
    h->a[i].key = key;
    h->a[i].v = v;
    return 0;
}

static item_t heap_pop(heap_t* h) {
    item_t top = h->a[0];
    item_t last = h->a[--h->size];
    uint64_t i = 0;
    for (;;) {
        uint64_t l = 2 * i + 1;
        if (l >= h->size) break;
        uint64_t c = l;
        if (l + 1 < h->size && h->a[l + 1].key < h->a[l].key) c = l + 1;
        if (h->a[c].key >= last.key) break;
        h->a[i] = h->a[c];
        i = c;
    }
    if (h->size > 0) h->a[i] = last;
    return top;
}

static uint64_t add_sat(uint64_t a, uint64_t b) {
    uint64_t s = a + b;
    return s < a ? ORACLE_INF : s;
}

/*
 * Dijkstra from s over the CSR (off[n+1], tgt[m], w[m]).  Stops when `stop`
 * (if < n) is settled.  dist[n] receives tentative distances (exact for settled
 * vertices); parent[n] (nullable) the predecessor on a shortest path
 * (UINT32_MAX for s and unreached vertices).  *edges_scanned (nullable) counts
 * adjacency entries examined.  Returns 0, or -1 on allocation failure.
 */
static int dijkstra_core(uint64_t n, const uint64_t* off, const uint32_t* tgt, const uint32_t* w,
                         uint32_t s, uint64_t stop, uint64_t* dist, uint32_t* parent,
                         uint64_t* edges_scanned) {
    heap_t h = {0, 0, 0};
    uint64_t scanned = 0;
    for (uint64_t i = 0; i < n; ++i) dist[i] = ORACLE_INF;
    if (parent)
        for (uint64_t i = 0; i < n; ++i) parent[i] = UINT32_MAX;
    dist[s] = 0;
    if (heap_push(&h, 0, s)) return -1;
    while (h.size > 0) {
        item_t it = heap_pop(&h);
        if (it.key != dist[it.v]) continue; /* stale entry */
        if ((uint64_t)it.v == stop) break;
        for (uint64_t e = off[it.v]; e < off[it.v + 1]; ++e) {
            ++scanned;
            uint32_t v = tgt[e];
            uint64_t nd = add_sat(it.key, (uint64_t)w[e]);
            if (nd < dist[v]) {
                dist[v] = nd;
                if (parent) parent[v] = it.v;
                if (heap_push(&h, nd, v)) {
                    free(h.a);
                    return -1;
                }
            }
        }
    }
    free(h.a);
    if (edges_scanned) *edges_scanned = scanned;
    return 0;
}

/* d(s,t), or UINT64_MAX if t is unreachable.  Returns UINT64_MAX-1 on OOM. */
uint64_t oracle_dijkstra_pair(uint64_t n, const uint64_t* off, const uint32_t* tgt, const uint32_t* w,
                              uint32_t s, uint32_t t, uint64_t* edges_scanned) {
    uint64_t* dist = (uint64_t*)malloc(n * sizeof(uint64_t));
    if (!dist) return ORACLE_INF - 1;
    if (dijkstra_core(n, off, tgt, w, s, t, dist, NULL, edges_scanned)) {
        free(dist);
        return ORACLE_INF - 1;
    }
    uint64_t d = dist[t];
    free(dist);
    return d;
}

/* Full single-source distances (and optional parents).  Returns 0 or -1. */
int oracle_sssp(uint64_t n, const uint64_t* off, const uint32_t* tgt, const uint32_t* w, uint32_t s,
                uint64_t* dist_out, uint32_t* parent_out) {
    return dijkstra_core(n, off, tgt, w, s, n, dist_out, parent_out, NULL);
}

/*
 * d(s,t) and one shortest path s..t written to path[0..len).  Returns the
 * distance; *path_len = number of vertices (0 if unreachable).  If the path
 * needs more than cap entries, *path_len holds the needed length and nothing
 * beyond cap is written.
 */
uint64_t oracle_dijkstra_path(uint64_t n, const uint64_t* off, const uint32_t* tgt, const uint32_t* w,
                              uint32_t s, uint32_t t, uint32_t* path, uint64_t cap, uint64_t* path_len) {
    uint64_t* dist = (uint64_t*)malloc(n * sizeof(uint64_t));
    uint32_t* par = (uint32_t*)malloc(n * sizeof(uint32_t));
    *path_len = 0;
    if (!dist || !par || dijkstra_core(n, off, tgt, w, s, t, dist, par, NULL)) {
        free(dist);
        free(par);
        return ORACLE_INF - 1;
    }
    uint64_t d = dist[t];
    if (d != ORACLE_INF) {
        uint64_t len = 1;
        for (uint32_t v = t; v != s; v = par[v]) ++len;
        *path_len = len;
        if (len <= cap) {
            uint64_t i = len;
            for (uint32_t v = t;; v = par[v]) {
                path[--i] = v;
                if (v == s) break;
            }
        }
    }
    free(dist);
    free(par);
    return d;
}

/* All-pairs distances d[i*n+j] by Floyd-Warshall over the CSR (tiny n only). */
void oracle_floyd_warshall(uint64_t n, const uint64_t* off, const uint32_t* tgt, const uint32_t* w,
                           uint64_t* d) {
    for (uint64_t i = 0; i < n * n; ++i) d[i] = ORACLE_INF;
    for (uint64_t i = 0; i < n; ++i) d[i * n + i] = 0;
    for (uint64_t u = 0; u < n; ++u)
        for (uint64_t e = off[u]; e < off[u + 1]; ++e) {
            uint64_t v = tgt[e];
            if ((uint64_t)w[e] < d[u * n + v]) d[u * n + v] = w[e];
        }
    for (uint64_t k = 0; k < n; ++k)
        for (uint64_t i = 0; i < n; ++i) {
            uint64_t dik = d[i * n + k];
            if (dik == ORACLE_INF) continue;
            for (uint64_t j = 0; j < n; ++j) {
                uint64_t dkj = d[k * n + j];
                if (dkj == ORACLE_INF) continue;
                uint64_t s = dik + dkj;
                if (s < d[i * n + j]) d[i * n + j] = s;
            }
        }
}

/* Pairs answered one by one: out[q] = d(pairs[2q], pairs[2q+1]). */
int oracle_pairs(uint64_t n, const uint64_t* off, const uint32_t* tgt, const uint32_t* w,
                 const uint32_t* pairs, uint64_t k, uint64_t* out, uint64_t* edges_scanned) {
    uint64_t total = 0;
    for (uint64_t q = 0; q < k; ++q) {
        uint64_t sc = 0;
        out[q] = oracle_dijkstra_pair(n, off, tgt, w, pairs[2 * q], pairs[2 * q + 1], &sc);
        if (out[q] == ORACLE_INF - 1) return -1;
        total += sc;
    }
    if (edges_scanned) *edges_scanned = total;
    return 0;
}
