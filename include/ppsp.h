/*
 * ppsp.h -- C ABI of the GB300 point-to-point shortest-path (PPSP) library.
 *
 * The library answers exact s-t distance queries on a device-resident CSR graph
 * with the paper's stepping-style PPSP framework (Alg. 2): a frontier is
 * processed in steps under an advancing threshold (Alg. 1, Delta*-stepping,
 * Sec. 2), with the Init / Prune / UpdateDistance plug-ins of Table 2 for
 * early termination (ET, Sec. 3.2), A* (Sec. 3.3), bidirectional search (BiDS,
 * Sec. 3.4, Theorem 3.3) and bidirectional A* (BiD-A*, Sec. 3.5, Theorem 3.4),
 * and batches of queries organised as a query graph (Sec. 4.1) and searched
 * with Multi-BiDS (Sec. 4.2) or single-source searches from a vertex cover
 * (Sec. 4.3), on undirected or directed graphs (Sec. 4.4).  All arithmetic on
 * distances is integer, so results are exact.  The paper defines no
 * programming interface; names and layouts here are this library's own.
 *
 * Conventions for every entry point:
 *  - Every function returns a ppsp_status; nothing aborts or throws across the
 *    ABI.  A device-side failure (a bounded wait that ran out, a distance that
 *    does not fit the chosen width) comes back as a status, and the library
 *    stays usable afterwards.
 *  - "host" pointers are ordinary CPU memory owned by the caller and only read
 *    or written during the call.  "device" pointers are CUDA global memory on
 *    the graph's device, owned by the caller.
 *  - Unreachable targets have distance PPSP_INF (UINT64_MAX) and a path
 *    length of 0.
 *  - A graph object may be used from one host thread at a time.
 */
#ifndef PPSP_H
#define PPSP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PPSP_INF UINT64_MAX

typedef struct ppsp_graph ppsp_graph;
typedef struct ppsp_plan ppsp_plan;

typedef enum {
    PPSP_OK = 0,
    PPSP_ERR_INVALID_ARG = 1,      /* null pointer, id >= n, bad option value */
    PPSP_ERR_BAD_GRAPH = 2,        /* malformed CSR, asymmetric "undirected" graph */
    PPSP_ERR_OOM = 3,              /* device or host allocation failed */
    PPSP_ERR_CUDA = 4,             /* a CUDA runtime call failed (no device, launch error) */
    PPSP_ERR_TIMEOUT = 5,          /* a bounded device-side wait ran out of iterations */
    PPSP_ERR_NO_COORDS = 6,        /* A* mode on a graph created without coordinates */
    PPSP_ERR_BUFFER_TOO_SMALL = 7, /* a path did not fit; the needed length is reported */
    PPSP_ERR_OVERFLOW = 8,         /* a distance does not fit 32 bits (use dist_bits = 64) */
    PPSP_ERR_UNSUPPORTED = 9       /* valid request outside what this build supports */
} ppsp_status;

/* Search plug-ins (Table 2). */
enum {
    PPSP_BIDS = 0,     /* bidirectional search, prune 2*d >= mu (Sec. 3.4)            */
    PPSP_BIDASTAR = 1, /* bidirectional A*, average potential h_F = -h_B (Sec. 3.5)   */
    PPSP_ET = 2,       /* one-directional with early termination, prune d >= mu       */
    PPSP_ASTAR = 3     /* one-directional A*, prune d + h_t(v) >= mu (Sec. 3.3)       */
};

/* Graph flags. */
enum { PPSP_UNDIRECTED = 1u, PPSP_KEEP_VERTEX_ORDER = 2u };

/* Frontier representation policy (App. B "Sparse-Dense Optimization").
 * AUTO: a group run by one CTA keeps its frontier as Delta*-stepping buckets
 * in shared memory (overflow and far-ahead entries in the slot); a group run
 * by several CTAs uses a queue while the frontier is small and a bitmap once
 * it exceeds (searches * n) / dense_den entries.  SPARSE / DENSE force the
 * queue / bitmap for every group. */
enum { PPSP_FRONTIER_AUTO = 0, PPSP_FRONTIER_SPARSE = 1, PPSP_FRONTIER_DENSE = 2 };

/* Layout of the per-search tentative-distance arrays of one batch group. */
enum { PPSP_LAYOUT_AUTO = 0, PPSP_LAYOUT_INTERLEAVED = 1, PPSP_LAYOUT_STACKED = 2 };

/* How a batch is executed (Sec. 4.2, Sec. 4.3 and the batch baselines of Sec. 6). */
enum {
    PPSP_BATCH_MULTI = 0,      /* Multi-BiDS: one search per query-graph vertex, shared  */
    PPSP_BATCH_PLAIN_STAR = 1, /* Plain*: every query its own pair of searches, all at once */
    PPSP_BATCH_PLAIN = 2,      /* Plain: one query at a time, each on one team of team_ctas
                                  CTAs (default: the whole GPU)                           */
    PPSP_BATCH_SSSP = 3,       /* Plain-SSSP (Sec. 4.3): a single-source search from every
                                  query source; answers read from its distances          */
    PPSP_BATCH_VC = 4,         /* VC-SSSP (Sec. 4.3): single-source searches only from a
                                  vertex cover of G_q (exact up to 32 vertices per
                                  component, greedy above; directed graphs: a minimum
                                  bipartite cover, targets searching backward).  For both
                                  SSSP strategies a search stops once every one of its
                                  targets is settled (no remaining key below the largest
                                  target distance, the multi-target form of ET's prune) */
    PPSP_BATCH_AUTO = 5        /* per connected component of G_q: an isolated pair runs as
                                  a pair; with BiD-A* potentials a star runs as one SSSP
                                  search from its centre and any other component as
                                  independent pairs (Plain*); without potentials a
                                  component with a vertex cover of at most a quarter of
                                  its vertices runs as VC-SSSP, any other as Multi-BiDS,
                                  except on graphs of average degree >= 8 (the social
                                  shape), where every component runs as VC-SSSP.
                                  ET / A*: sources with 4 or more targets run one
                                  multi-target search                                   */
};

/*
 * Query options.  Call ppsp_options_init() first; it fills in the defaults
 * noted beside each field.  Options never change answers, only speed
 * (Theorems 3.3 and 3.4 hold for any stepping schedule), except mode, which
 * selects the plug-in, and dist_bits, which bounds representable distances.
 */
typedef struct {
    int32_t mode;            /* PPSP_BIDS (default) ... PPSP_ASTAR                         */
    int32_t dist_bits;       /* 32 (default) or 64: width of tentative distances in HBM     */
    uint64_t delta;          /* stepping increment Delta >= 1; 0 = auto (learned model if
                                attached to the graph, else mean edge weight)               */
    int32_t frontier;        /* PPSP_FRONTIER_* (default AUTO)                              */
    int32_t layout;          /* PPSP_LAYOUT_* (default AUTO)                                */
    int32_t batch_strategy;  /* PPSP_BATCH_* (default MULTI)                                */
    int32_t block_threads;   /* 256, 512 or 1024 threads per CTA; 0 = auto: 1024 when every
                                team is one CTA (the bucketed path), else 512              */
    int32_t team_ctas;       /* CTAs cooperating on one small group (pair); 0 = auto        */
    int32_t big_team_ctas;   /* CTAs cooperating on one multi-search group; 0 = auto        */
    uint32_t dense_den;      /* frontier goes dense above (searches * n) / dense_den; 0=auto */
    int32_t want_paths;      /* 1: also return one shortest path per query (weights >= 1)   */
    int32_t max_ctas;        /* cap on resident CTAs used (0 = all that fit)               */
    uint64_t spin_limit;     /* iterations of a device-side wait before PPSP_ERR_TIMEOUT;
                                0 = default (about a few seconds)                          */
    void* stream;            /* cudaStream_t to run on; NULL = the legacy default stream    */
    uint32_t debug_flags;    /* test hooks, 0 in normal use (PPSP_DEBUG_*)                  */
    uint32_t cuda_graph;     /* plans: 1 = capture the launches of ppsp_plan_run into a CUDA
                                graph on a non-NULL stream and replay it (default 0)         */
    uint32_t stepping_rho;   /* GetDist variant (Sec. 2: Delta*-stepping, rho-stepping and
                                Bellman-Ford are all stepping algorithms).  0 (default):
                                one Delta-bucket per step.  rho > 0: a step of a one-CTA
                                group takes consecutive non-empty buckets until they hold
                                at least rho entries (with Delta small this approaches
                                rho-stepping, which extracts the rho smallest keys; with
                                Delta huge every step takes the whole frontier, which is
                                Bellman-Ford).  Groups on several CTAs ignore it.            */
    uint32_t memo_potential; /* 1: heuristic memoization (Sec. 5): the A* potential term of
                                an entry is computed from the coordinates once per group and
                                read back from a per-slot array afterwards (4 more bytes per
                                distance entry of a slot); 0 (default): recomputed each time */
    uint32_t pull_push;      /* 1: bidirectional relaxation (App. B) on the queue / bitmap
                                path of undirected graphs: before an extracted vertex pushes,
                                it pulls min over its neighbours x of d(x) + w(x, u); groups
                                on one CTA and directed graphs ignore it.  Default 0         */
    uint32_t ring_entries;   /* groups on one CTA: shared-memory entries per Delta-bucket of
                                the frontier ring (32 buckets), 1..256; 0 = default (64).
                                Larger buckets stay out of the global overflow region; a
                                smaller ring leaves more of the SM's L1 to the graph        */
    uint32_t multi_potential;/* BiD-A* Multi-BiDS groups: 1 = every shared search prunes with
                                the smallest partner potential against mumax (multi-target
                                A*, an extension: Sec. 4.4 leaves it open); 0 (default) =
                                shared searches run without a potential (plain Multi-BiDS)  */
    uint32_t reserved[1];
} ppsp_options;

/* Test hook: device barriers wait for one arrival that never comes, so every
 * multi-CTA wait runs out and the call returns PPSP_ERR_TIMEOUT. */
#define PPSP_DEBUG_BARRIER_NEVER_RELEASES 1u

/* Work counters of one call (paper Sec. 6 measures time; these feed GTEPS and
 * the algorithmic-bytes roofline). */
typedef struct {
    uint64_t extracted;   /* frontier entries taken and not pruned (X)           */
    uint64_t edges;       /* adjacency entries scanned (E)                        */
    uint64_t relaxed;     /* WriteMin relaxations that lowered a distance (R); on
                             the one-CTA path: lower than the value read just
                             before, a concurrent smaller write aside            */
    uint64_t pushed;      /* frontier insertions (P)                              */
    uint64_t rounds;      /* stepping rounds summed over groups                   */
    uint64_t groups;      /* searched groups (pairs or query-graph components)    */
    uint64_t searches;    /* single-source searches                               */
    uint64_t touched;     /* tentative distances that left infinity               */
    uint64_t dense_rounds;/* rounds whose frontier was a bitmap                   */
    uint64_t reserved[7];
} ppsp_counters;

/* Graph properties computed at creation. */
typedef struct {
    uint64_t n, m;
    uint64_t w_min, w_max;
    double w_mean, w_std;
    uint64_t deg_max;
    double potential_scale;   /* c of the A* potential (0 if no coordinates)            */
    int32_t potential_shift;  /* fixed-point bits F of the potential coordinates        */
    int32_t has_coords;
    int32_t undirected;
    int32_t has_zero_weight;
    uint64_t device_bytes;    /* device memory held by the graph (CSR + coordinates)    */
} ppsp_graph_info;

/* Fill *o with defaults.  Never fails for a non-null o. */
void ppsp_options_init(ppsp_options* o);

/* Static string for a status code. */
const char* ppsp_status_string(ppsp_status s);

/* Text of the last CUDA failure seen by the calling thread ("" if none);
 * valid until the thread's next library call. */
const char* ppsp_last_error_detail(void);

/*
 * Create a device-resident graph from a host CSR (paper Sec. 2: G = (V, E, w),
 * w: E -> R+, here non-negative uint32).
 *   n        number of vertices, 1 <= n < 2^32 - 1
 *   m        number of adjacency entries (an undirected edge counts twice), m < 2^32
 *   offsets  host uint64[n+1], offsets[0] = 0, non-decreasing, offsets[n] = m
 *   targets  host uint32[m], every id < n
 *   weights  host uint32[m]
 *   coords   host float[2n] (x, y per vertex) or NULL; needed by the A* modes.
 *            With coordinates the library also keeps the adjacency as 16-byte
 *            records (target, weight, integer potential coordinates of the
 *            target: another 16m bytes, 32m for a directed graph), which the
 *            searches with a potential read instead of gathering the
 *            target's coordinates separately
 *   flags    PPSP_UNDIRECTED: the CSR is symmetric with equal weights both ways
 *            (validated; the bidirectional modes search backwards on the same CSR).
 *            Without it the graph is directed: the library also keeps its
 *            transpose on the device (another 4(n+1) + 8m bytes), and a query's
 *            target searches in-edges (Sec. 4.4: searches forward from sources,
 *            backward from targets; Multi-BiDS groups pair them bipartitely).
 *            VC-SSSP covers the bipartite query graph (Konig).
 *            PPSP_KEEP_VERTEX_ORDER: keep the caller's vertex order on the
 *            device.  By default a graph with coordinates is stored in the
 *            order of a Hilbert curve over its coordinates, so that vertices
 *            near each other in the plane share cache lines of the
 *            adjacency, potential and distance arrays (a search's frontier
 *            is a compact region).  The renumbering is internal: every call
 *            takes and returns the caller's vertex ids (pairs, paths,
 *            potential coordinates), and distances do not depend on it.
 * Inputs are copied; the caller may free them after the call.  On success
 * *out owns device memory until ppsp_graph_destroy.
 * Errors: INVALID_ARG (null pointers, n or m out of range), BAD_GRAPH
 * (malformed or asymmetric CSR), OOM, CUDA.
 */
ppsp_status ppsp_graph_create(uint64_t n, uint64_t m, const uint64_t* offsets,
                              const uint32_t* targets, const uint32_t* weights,
                              const float* coords, uint32_t flags, ppsp_graph** out);

/* Free the graph and every buffer the library allocated for it.  NULL is a no-op. */
void ppsp_graph_destroy(ppsp_graph* g);

/* Copy the graph's properties into *out (host). */
ppsp_status ppsp_graph_get_info(const ppsp_graph* g, ppsp_graph_info* out);

/*
 * One query d(s, t) with the plug-in of opt->mode (NULL opt = defaults), on
 * the whole GPU ("Plain" execution of one query, Sec. 4.2).
 *   dist_out  host uint64, receives d(s, t) or PPSP_INF
 *   path_buf  host uint32[path_cap] or NULL; with opt->want_paths it receives
 *             one shortest path s..t (s == t gives [s])
 *   path_len  host uint64 or NULL; receives the number of vertices of the path
 *             (0 if unreachable), also when the path did not fit (then the
 *             status is BUFFER_TOO_SMALL and dist_out is still valid)
 * Errors: INVALID_ARG (s or t >= n, bad options), NO_COORDS, UNSUPPORTED
 * (paths on a graph with zero-weight edges), OOM, CUDA, TIMEOUT, OVERFLOW.
 */
ppsp_status ppsp_query(ppsp_graph* g, uint32_t s, uint32_t t, const ppsp_options* opt,
                       uint64_t* dist_out, uint32_t* path_buf, uint64_t path_cap,
                       uint64_t* path_len);

/*
 * A batch of k queries (Sec. 4): pairs is host uint32[2k] (s0, t0, s1, t1, ...).
 * The batch is turned into a query graph G_q (Sec. 4.1; repeated and reversed
 * pairs collapse to one query edge) and run with opt->batch_strategy.
 *   dists_out     host uint64[k], answer of each pair in input order
 *   paths_buf     host uint32 buffer or NULL (needs opt->want_paths)
 *   path_offsets  host uint64[k+1] or NULL: query q may use
 *                 paths_buf[path_offsets[q] .. path_offsets[q+1])
 *   path_lens     host uint64[k] or NULL: vertices on each path (needed length
 *                 if it did not fit; then the call returns BUFFER_TOO_SMALL)
 *   counters      host ppsp_counters or NULL: work done by the call
 * k = 0 is valid and does nothing.  Errors as ppsp_query, and UNSUPPORTED
 * for paths with the SSSP strategies or for a multi-search group whose
 * distance arrays would need 2^32 entries or more (use smaller groups:
 * PPSP_BATCH_PLAIN_STAR or a smaller batch).
 */
ppsp_status ppsp_batch(ppsp_graph* g, const uint32_t* pairs, uint64_t k, const ppsp_options* opt,
                       uint64_t* dists_out, uint32_t* paths_buf, const uint64_t* path_offsets,
                       uint64_t* path_lens, ppsp_counters* counters);

/*
 * Split form of ppsp_batch for callers that keep results in device memory and
 * replay the same batch shape: ppsp_plan_create does the host-side work (query
 * graph, groups, schedule, device descriptors, search memory), ppsp_plan_run
 * launches the searches on opt->stream and writes d_dists_out (device
 * uint64[k], input order) before the stream's next work; ppsp_plan_sync waits
 * for the stream and returns the run's device status and counters.  With
 * opt->cuda_graph = 1 and a non-NULL stream, the first run for a given
 * d_dists_out captures the run's launches into a CUDA graph and every run
 * replays it (if the driver refuses the capture, runs launch directly).  A
 * plan keeps device memory until ppsp_plan_destroy and belongs to its graph:
 * destroy every plan of a graph before the graph (ppsp_plan_destroy takes the
 * graph's lock).
 * Its descriptor memory comes from the device's stream-ordered pool on
 * opt->stream (creating or destroying a plan never synchronises other
 * streams), so that stream must outlive the plan; ppsp_plan_destroy waits for
 * the plan's own work on it.  Paths are not available through plans (use
 * ppsp_batch).
 */
ppsp_status ppsp_plan_create(ppsp_graph* g, const uint32_t* pairs, uint64_t k,
                             const ppsp_options* opt, ppsp_plan** out);
ppsp_status ppsp_plan_run(ppsp_plan* p, uint64_t* d_dists_out);
ppsp_status ppsp_plan_sync(ppsp_plan* p, ppsp_counters* counters);
void ppsp_plan_destroy(ppsp_plan* p);

/*
 * A* potential of the graph (Sec. 3.3; consistency, Fact 3.1).  The library
 * stores integer potential coordinates P(v) = floor(p(v) * c * 2^F + 0.5)
 * (float64 arithmetic, c and F in ppsp_graph_info) chosen at creation so that
 * |P(u) - P(v)|^2 <= (2^F * w(u,v))^2 on every edge; the potential is
 * h_x(v) = floor(|P(v) - P(x)| / 2^F), computed exactly in integers.
 *   ppsp_potential_coords: host int64[2n] receives P (x, y per vertex).
 *   ppsp_potential_eval:   evaluates h_anchor(v) on the device for the host
 *                          uint32 vertices[count], into host int64 out[count].
 * Errors: NO_COORDS, INVALID_ARG, CUDA.
 */
ppsp_status ppsp_potential_coords(const ppsp_graph* g, int64_t* out);
ppsp_status ppsp_potential_eval(ppsp_graph* g, uint32_t anchor, const uint32_t* vertices,
                                uint64_t count, int64_t* out);

/*
 * Features of each group of a plan, as the stepping-increment model sees them:
 * out[12 * g + f] = log2(1 + raw_f) for f = heuristic s-t distance (mean over
 * the group's queries, 0 without coordinates), deg(s), deg(t) (for groups of
 * more than two searches: mean and max degree), mean/std/min/max edge weight,
 * n, m, |V_q|, |E_q| of the group and its mean query-graph degree.
 *   out     host float[12 * cap] or NULL (then only *ngroups is written)
 * Errors: INVALID_ARG, BUFFER_TOO_SMALL (cap < number of groups).
 */
ppsp_status ppsp_plan_features(const ppsp_plan* p, float* out, uint64_t cap, uint64_t* ngroups);

/*
 * Device time of every group in the plan's last run (ns between the group's
 * Init and the end of its tidy step, on the team that ran it); waits for the
 * plan's stream.  out_ns host uint64[cap] or NULL (then only *ngroups).
 * Used to label the stepping-increment sweep.  Errors: INVALID_ARG (never
 * run), BUFFER_TOO_SMALL, CUDA.
 */
ppsp_status ppsp_plan_group_times(ppsp_plan* p, uint64_t* out_ns, uint64_t cap, uint64_t* ngroups);

/*
 * Device memory of a plan (host outputs, each nullable):
 *   slot_bytes   search memory of its teams (one slot per team: distances,
 *                frontier bitmaps and queues, touched list, bucket overflow);
 *                slots come from the graph's pool and go back to it when the
 *                plan is destroyed
 *   teams        number of teams, that is of slots held
 *   other_bytes  descriptors, per-query state and path buffers of the plan
 * Errors: INVALID_ARG.
 */
ppsp_status ppsp_plan_device_bytes(const ppsp_plan* p, uint64_t* slot_bytes, uint64_t* teams,
                                   uint64_t* other_bytes);

/*
 * Device bytes of the slot one team of a batch allocates for groups of
 * `searches` searches (2 for a BiDS pair, 1 for an SSSP-based or
 * one-directional search, up to 64 for a Multi-BiDS group) with the given
 * distance width (32 or 64) and frontier policy: the larger of the two
 * sizes a team can take (a team that spans the plan's whole grid keeps a
 * touched list for every entry of the range, a smaller team a quarter of it
 * plus 4,096).  A batch plan holds one slot per team, and at most as many
 * teams as groups, so admission control can bound a batch's search memory
 * before creating its plan (host only, no device work).
 * Errors: INVALID_ARG.
 */
ppsp_status ppsp_slot_bytes(const ppsp_graph* g, uint32_t searches, int32_t dist_bits, int32_t frontier,
                            uint64_t* out);

/* 1 if the plan's last run replayed a captured CUDA graph, else 0. */
ppsp_status ppsp_plan_uses_graph(const ppsp_plan* p, int32_t* out);

/*
 * The device vertex order ppsp_graph_create gives a graph with these
 * coordinates (host only, no graph, no device work): vertices sorted by their
 * position along a Hilbert curve over a 2^16 x 2^16 lattice spanning the
 * bounding square of the coordinates (ties by id).
 *   coords    host float[2n], (x, y) per vertex
 *   perm_out  host uint32[n], caller-owned: perm_out[v] = device id of v
 * Errors: INVALID_ARG (null pointers, n = 0 or n >= 2^32), UNSUPPORTED
 * (non-finite coordinates: the graph keeps the caller's order).
 */
ppsp_status ppsp_vertex_order(uint64_t n, const float* coords, uint32_t* perm_out);

/* Source selection of the SSSP-based batch strategies (Sec. 4.3), host only
 * (no device work, usable without a GPU).
 *   pairs      host array of k (s, t) vertex-id pairs (uint32, row-major k x 2)
 *   strategy   PPSP_BATCH_SSSP (a forward search from the source of each
 *              query) or PPSP_BATCH_VC (a search from an endpoint in a vertex
 *              cover of the query graph)
 *   flags      PPSP_UNDIRECTED for an undirected graph: the cover is minimum by
 *              exhaustive branch and bound for components of at most 32
 *              vertices, greedy by uncovered degree above; 0 for a directed
 *              graph: the query graph is bipartite (sources, targets) and the
 *              cover is minimum (maximum matching and Konig's theorem), a
 *              target in it searching backward
 *   src_out    host array of k: the vertex whose single-source search answers
 *              pair q, 0xFFFFFFFF for s == t (no search); caller-owned
 *   dir_out    host array of k or NULL: 0 = the search follows out-edges,
 *              1 = in-edges (a backward search from the query's target)
 *   n_sources  number of distinct (vertex, direction) searches the plan runs
 * This is exactly the selection ppsp_plan_create makes for these strategies.
 * Vertex ids are not range-checked (no graph). Errors: PPSP_ERR_INVALID_ARG for
 * null pointers or another strategy. */
ppsp_status ppsp_batch_sources(const uint32_t* pairs, uint64_t k, int32_t strategy, uint32_t flags,
                               uint32_t* src_out, uint32_t* dir_out, uint64_t* n_sources);

/*
 * Learned stepping increment.  The paper tunes Delta of Delta*-stepping by
 * doubling it until the time stops improving (Sec. 6.1); Delta changes only
 * the schedule, never an answer (Theorems 3.3/3.4).  This library predicts it
 * per group with a 12 -> 64 -> 64 -> 1 MLP (ReLU; bf16 weights, fp32
 * accumulation): y = log2(Delta / Delta_default), Delta_default = mean edge
 * weight, Delta = round(Delta_default * 2^clamp(y, -8, 6)), at least 1.
 * Parameter vector: PPSP_MLP_PARAMS floats, in order mean[12], std[12]
 * (input standardisation, std > 0), W1[64][12], b1[64], W2[64][64], b2[64],
 * W3[64], b3[1].  A model lives on the device until destroyed.
 *   create:     copies params (host).  Errors: INVALID_ARG (std <= 0), OOM, CUDA.
 *   get_params: host float[PPSP_MLP_PARAMS] receives the fp32 master copy.
 *   predict:    host feats[12 * count] -> host out[count] (y per sample).
 *   grad:       gradient of mean((y - labels)^2) w.r.t. every parameter
 *               (zero for mean/std) into host grad_out[PPSP_MLP_PARAMS];
 *               *loss_out (nullable) = that mean.
 *   train:      `epochs` full-batch Adam steps (beta 0.9/0.999, eps 1e-8) at
 *               learning rate lr; *loss_out (nullable) = loss before the last step.
 *   graph_set_delta_model: plans of mode `mode` created afterwards with
 *               delta = 0 use the model (borrowed: keep it alive while such
 *               plans run; NULL detaches).
 */
#define PPSP_MLP_FEATURES 12
#define PPSP_MLP_PARAMS 5081
typedef struct ppsp_delta_model ppsp_delta_model;
ppsp_status ppsp_delta_model_create(const float* params, ppsp_delta_model** out);
void ppsp_delta_model_destroy(ppsp_delta_model* m);
ppsp_status ppsp_delta_model_get_params(const ppsp_delta_model* m, float* out);
ppsp_status ppsp_delta_model_predict(ppsp_delta_model* m, const float* feats, uint64_t count, float* out);
ppsp_status ppsp_delta_model_grad(ppsp_delta_model* m, const float* feats, const float* labels, uint64_t count,
                                  float* grad_out, float* loss_out);
ppsp_status ppsp_delta_model_train(ppsp_delta_model* m, const float* feats, const float* labels, uint64_t count,
                                   uint32_t epochs, float lr, float* loss_out);
ppsp_status ppsp_graph_set_delta_model(ppsp_graph* g, int32_t mode, ppsp_delta_model* m);

/*
 * Allocation-free single query.  The paper has no counterpart: this entry
 * point exists for callers that cannot allocate device memory (code running
 * inside a memory pool it does not own, a serving process under a strict
 * no-allocation policy, or a moment where cudaMalloc's implicit device
 * synchronisation is not acceptable).  It answers one BiDS query (Sec. 3.4)
 * without calling cudaMalloc, cudaFree or any allocating routine: all scratch
 * lives in one fixed device array inside the library (about 13 MB, kept by
 * every GPU that loads the library until the process exits).
 *   d_offsets   device uint32[n+1], CSR offsets (4-byte aligned)
 *   d_edges     device uint32[2m], (target, weight) per adjacency entry,
 *               8-byte aligned; the CSR must be symmetric (undirected)
 *   n, m        1 <= n <= PPSP_NOALLOC_MAX_N, m < 2^32
 *   s, t        query endpoints (< n)
 *   delta       stepping increment, 0 = mean edge weight (computed on the device)
 *   d_dist_out  device uint64[1]: d(s, t) or PPSP_INF, written on `stream`
 *   stream      cudaStream_t or NULL
 * The call waits for its stream before returning the status.  All calls share
 * the one array: calls that overlap on the GPU race and must not be issued.
 * The first call on a device resolves the array's address and initialises it.
 * Errors: INVALID_ARG (null
 * pointers, n above the limit, ids >= n, d_offsets not 4-byte aligned,
 * d_edges or d_dist_out not 8-byte aligned), UNSUPPORTED (a device on which
 * fewer than two engine CTAs fit), CUDA, TIMEOUT, OVERFLOW.
 */
#define PPSP_NOALLOC_MAX_N (1u << 20)
ppsp_status ppsp_query_noalloc(const uint32_t* d_offsets, const uint32_t* d_edges, uint32_t n, uint64_t m,
                               uint32_t s, uint32_t t, uint64_t delta, uint64_t* d_dist_out, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* PPSP_H */
