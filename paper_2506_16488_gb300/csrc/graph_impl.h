// Host-side objects behind the opaque ppsp_graph / ppsp_plan handles.
#pragma once

#include <map>
#include <memory>
#include <mutex>
#include <tuple>
#include <vector>

#include "ppsp_internal.h"

namespace ppsp {

// One team's search memory (device).  Invariant between uses: every tentative
// distance is infinity, both bitmaps are zero.
struct Slot {
    void* base = nullptr;   // single allocation
    size_t bytes = 0;
    SlotDev dev{};
    int dist_bits = 32;
    u64 flat_cap = 0;
    bool busy = false;
    bool dirty = false;  // a failed run may have left it unclean: scrub before its next use
};

struct SlotKey {
    int dist_bits;
    u64 flat_cap;
    u32 qcap, tcap;
    bool memo;  // holds the memoized-potential array
    bool operator<(const SlotKey& o) const {
        return std::tie(dist_bits, flat_cap, qcap, tcap, memo) <
               std::tie(o.dist_bits, o.flat_cap, o.qcap, o.tcap, o.memo);
    }
};

}  // namespace ppsp

struct ppsp_graph {
    int device = 0;
    uint64_t n = 0, m = 0;
    ppsp::u32* d_off = nullptr;
    uint2* d_edges = nullptr;
    int4* d_edges_pc = nullptr;    // (target, weight, P(target)) when the graph has coordinates
    int4* d_edges_t_pc = nullptr;  // the same for the transpose of a directed graph
    ppsp::u32* d_off_t = nullptr;  // transpose of a directed graph (null when undirected)
    uint2* d_edges_t = nullptr;
    int2* d_pc = nullptr;
    std::vector<int64_t> pc_host;  // 2n potential coordinates
    double pot_scale = 0.0;
    int pot_shift = 0;
    ppsp_graph_info info{};
    std::vector<uint64_t> deg;     // host copy of degrees (features, schedules)
    // internal vertex order: perm[caller id] = device id, inv[device id] =
    // caller id (both empty when the caller's order is kept)
    std::vector<ppsp::u32> perm, inv;
    // slot pool
    std::multimap<ppsp::SlotKey, std::unique_ptr<ppsp::Slot>> pool;
    std::mutex mu;
    // scratch for small transfers (potential eval)
    ppsp::u32* d_scratch_u32 = nullptr;
    int64_t* d_scratch_i64 = nullptr;
    uint64_t scratch_cap = 0;
    // learned stepping-increment models, one per plug-in (borrowed)
    ppsp_delta_model* delta_model[4] = {nullptr, nullptr, nullptr, nullptr};

    ppsp::GraphDev dev() const {
        ppsp::GraphDev g;
        g.off = d_off;
        g.edges = d_edges;
        g.off_t = d_off_t ? d_off_t : d_off;
        g.edges_t = d_edges_t ? d_edges_t : d_edges;
        g.pc = d_pc;
        g.edges_pc = d_edges_pc;
        g.edges_t_pc = d_edges_t_pc ? d_edges_t_pc : d_edges_pc;
        g.n = (ppsp::u32)n;
        g.pot_shift = (ppsp::u32)pot_shift;
        g.m = (ppsp::u32)m;
        g.pad = 0;
        return g;
    }
};

namespace ppsp {

// Capacities of the slot of a team whose groups span `range` flat entries
// (searches x n): frontier queues, touched list (a whole-GPU team never
// overflows its touched list).
struct SlotCaps {
    u64 flat_cap;
    u32 qcap, tcap;
};
SlotCaps slot_caps(u64 range, int frontier, bool whole_gpu);
// Device bytes of a freshly allocated slot with these capacities (memo: with
// the memoized-potential array).
u64 slot_alloc_bytes(int dist_bits, u64 flat_cap, u32 qcap, u32 tcap, bool memo = false);

// Borrow a slot with at least the requested capacities (allocating if needed;
// a new slot is initialised on `stream`, the stream of the plan that takes it).
ppsp_status slot_acquire(ppsp_graph* g, int dist_bits, u64 flat_cap, u32 qcap, u32 tcap, bool memo,
                         cudaStream_t stream, Slot** out);
void slot_release(ppsp_graph* g, Slot* s);
// Restore the clean invariant of a slot a failed run used, on the stream of
// the plan that uses it next (other plans' slots are left alone).
ppsp_status slot_scrub(Slot* s, cudaStream_t stream);

// Exact floor(sqrt(x)) on the host.
u64 isqrt_host(u64 x);
i64 pot_h_host(const ppsp_graph* g, u32 x, u32 v);

}  // namespace ppsp
