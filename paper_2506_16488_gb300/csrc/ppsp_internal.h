// Internal declarations of the GB300 PPSP library (not part of the C ABI).
//
// Execution model.  A batch is a set of *groups*; a group is a set of k
// single-source *searches* that share answers through *query edges* (a query
// graph component, paper Sec. 4.1; a BiDS query is a group of two searches and
// one query edge, Table 2).  One persistent cooperative kernel runs all groups.
// Its CTAs are partitioned into *teams*; a team takes groups from its queue and
// runs each to completion with the stepping loop of Alg. 2, synchronising its
// CTAs once per step.  Every team owns a *slot*: the tentative-distance arrays,
// the two frontier bitmaps, the two frontier queues and the touched list of the
// group it is running.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/ppsp.h"

namespace ppsp {

typedef uint32_t u32;
typedef uint64_t u64;
typedef int64_t i64;

constexpr u64 INF64 = ~0ull;
constexpr u32 INF32 = ~0u;
constexpr u32 NONE = ~0u;
constexpr int KMAX = 64;          // searches per group (query-graph vertices)
constexpr int MAX_QUEUES = 2;     // group queues: 0 = multi-search groups, 1 = pairs/singles

// Group modes (plug-ins of Table 2).
enum : u32 {
    GM_BIDIR = 0,    // BiDS / BiD-A* / Multi-BiDS: searches joined by query edges
    GM_ET = 1,       // one-directional, early termination at target
    GM_ASTAR = 2,    // one-directional A*
    GM_SSSP = 3      // no target, no pruning (full single-source distances)
};

// Device error word bits.
enum : u32 { ERRB_TIMEOUT = 1u, ERRB_OVERFLOW = 2u, ERRB_INTERNAL = 4u };

struct GraphDev {
    const u32* off;       // [n+1]
    const uint2* edges;   // [m] (target, weight)
    const u32* off_t;     // [n+1] transpose (in-edges); the same arrays as off / edges when undirected
    const uint2* edges_t; // [m] (source, weight)
    const int2* pc;       // [n] integer potential coordinates, or null
    // graphs with coordinates: the adjacency again as 16-byte records
    // (target, weight, P(target).x, P(target).y), so that a relaxation gets
    // the target's potential coordinates with its edge instead of a second,
    // random load; null otherwise
    const int4* edges_pc;
    const int4* edges_t_pc;
    u32 n;
    u32 pot_shift;        // F: h = isqrt(d2 >> 2F)
    u32 m;                // adjacency entries (bounds of checked builds)
    u32 pad;
};

struct SearchDev {
    u32 src;              // q_i
    u32 pbeg, pcnt;       // partners[pbeg .. pbeg+pcnt)
    u32 pot;              // 1: bidirectional A* potential rho_i(v) = h_{pot_b}(v) - h_{src}(v);
                          // 2: multi-target form min_j h_{q_j}(v) - h_{src}(v) over the partners j
    u32 pot_b;            // partner vertex of the potential
    u32 dir;              // 0: searches out-edges (from a source); 1: in-edges (back from a target)
    u32 pad;
    i64 key_off;          // added to keys so the source's key is 0
};

struct PartnerDev {
    u32 j;                // local index of the partner search in the group
    u32 qe;               // global query-edge index
};

struct QEdgeDev {
    u32 a, b;             // local search indices (a == b for one-directional groups)
};

struct GroupDev {
    u32 sbeg, scnt;       // searches[sbeg .. sbeg+scnt)
    u32 qbeg, qcnt;       // query edges
    u32 mode;             // GM_*
    u32 target;           // ET / A*: target vertex
    u32 layout;           // PPSP_LAYOUT_INTERLEAVED or PPSP_LAYOUT_STACKED
    u32 kshift;           // interleaved: flat = (v << kshift) | i
    u64 delta;            // stepping increment
};

// Per-slot step state, triple buffered by step index (cur, next, reset).
struct StepState {
    u64 minkey;           // min key inserted into this step's frontier
    u32 count;            // distinct entries in this step's frontier (queue tail when sparse)
    u32 tile;             // dynamic tile counter while the step is processed
    u32 overflow;         // queue overflowed: step must be processed from the bitmap
    u32 cnt_dir[2];       // entries per direction (two-search groups)
    u32 pad;
    u64 bmax;             // largest prune bound of the group, taken before the step's barrier
};

struct SlotState {
    StepState s[3];
    u32 touched_n;
    u32 touched_overflow;
    u32 pad[2];
};

struct SlotDev {
    void* dist;           // tentative distances, flat_cap entries of DistT
    u32* bm[2];           // frontier bitmaps, flat_cap bits each
    u32* q[2];            // frontier queues (one-CTA teams: far lists), qcap entries each
    void* fd[2];          // one-CTA teams: distance stored with each far-list entry
    u32* of;              // one-CTA teams: bucket overflow (flat index), ocap entries
    void* od;             //   and the stored distances
    u32 ocap;             //   split evenly between the ring's buckets
    u32* touched;         // flat indices that left infinity, tcap entries
    u32* memo;            // memoized potential terms (flat_cap entries, 0 = unset), or null
    SlotState* st;
    u64 flat_cap;         // k_cap * n
    u32 qcap, tcap;
};

struct TeamState {
    u32 bar_count;
    u32 bar_gen;
    u32 group;
    u32 pad[29];          // one 128-byte line per team
};

struct EngineCounters {
    unsigned long long extracted, edges, relaxed, pushed, rounds, groups, searches, touched,
        dense_rounds;
};

struct EngineArgs {
    GraphDev g;
    const GroupDev* groups;
    const SearchDev* searches;
    const PartnerDev* partners;
    const QEdgeDev* qedges;
    u64* mu;              // [num_qedges]
    u64* mumax;           // [num_searches]
    // teams
    const u32* cta_team;  // [grid] team of each CTA
    const u32* team_first;// [teams] first CTA
    const u32* team_size; // [teams]
    const u32* team_queue;// [teams] group queue
    TeamState* tstate;    // [teams]
    SlotDev* slots;       // [teams]
    const u32* queue_items[MAX_QUEUES];
    u32 queue_len[MAX_QUEUES];
    u32* queue_head;      // [MAX_QUEUES] claim counters
    // options
    u32 dense_den;        // dense when count > flat_size / dense_den (0 = never)
    u32 frontier;         // PPSP_FRONTIER_*
    u32 rho;              // one-CTA path: a step takes buckets until it holds >= rho entries (0 = one)
    u32 memo;             // memoize potential terms in the slot (Sec. 5)
    u32 pull;             // queue / bitmap path: pull before push (App. B), undirected graphs
    u32 ring_cap;         // one-CTA path: shared-memory entries per bucket (1 .. 256)
    u32 debug;
    u64 spin_limit;
    u32* err;
    EngineCounters* counters;
    u64* group_ns;        // [groups] device time of each group, or null
    // optional paths (null path_buf = distances only)
    u32* meet;            // [num_qedges] meeting vertex, NONE-initialised per run
    u32* path_buf;        // concatenated per-query-edge path buffers
    const u64* path_off;  // [num_qedges + 1] buffer offsets (capacity = difference)
    u64* path_len;        // [num_qedges] vertices on the path (needed length)
};

// ---- host helpers shared between translation units ----
#define PPSP_CUDA_TRY(expr)                                          \
    do {                                                              \
        cudaError_t e__ = (expr);                                     \
        if (e__ != cudaSuccess) {                                     \
            ppsp::set_last_cuda_error(e__, #expr, __FILE__, __LINE__); \
            return e__ == cudaErrorMemoryAllocation ? PPSP_ERR_OOM : PPSP_ERR_CUDA; \
        }                                                             \
    } while (0)

void set_last_cuda_error(cudaError_t e, const char* what, const char* file, int line);
// Detail text for an internal device error (the error word).
void set_last_device_error(u32 err);
// Detail text for an internal host-side inconsistency (printf format).
void set_last_internal_error(const char* fmt, ...);

// Launch the persistent engine.  dist_bits selects the distance width.
ppsp_status launch_engine(const EngineArgs& a, int dist_bits, int block_threads, u32 grid,
                          cudaStream_t stream, bool local_only = false);

// Max resident CTAs of the engine for a block size / distance width (of the
// one-CTA instance when local_only).
// ring_cap: shared-memory entries per bucket of the one-CTA frontier.
constexpr u32 RING_CAP_DEFAULT = 64;
ppsp_status engine_occupancy(int dist_bits, int block_threads, int* blocks_per_sm, int* sms,
                             bool local_only = false, u32 ring_cap = RING_CAP_DEFAULT);

// Evaluate potentials h_anchor(v) on the device.
ppsp_status launch_potential_eval(const GraphDev& g, u32 anchor, const u32* d_verts, u64 count,
                                  i64* d_out, cudaStream_t stream);

// Result scatter out[q] = (map[q] == NONE) ? 0 : mu[map[q]].
ppsp_status launch_scatter(const u32* d_map, const u64* d_mu, u64 k, u64* d_out, cudaStream_t s);

}  // namespace ppsp
