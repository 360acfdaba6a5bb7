// Batch planning: query graph (Sec. 4.1), groups, team schedule, launches.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <functional>
#include <numeric>
#include <unordered_map>
#include <unordered_set>

#include "graph_impl.h"
#include "mlp_internal.h"

using namespace ppsp;

struct ppsp_plan {
    ppsp_graph* g = nullptr;
    ppsp_options opt{};
    cudaStream_t stream = nullptr;
    u64 k = 0;
    int dist_bits = 32;
    int block = 512;
    bool local_only = false;           // every team is one CTA on the bucketed path
    bool memo = false;                 // slots keep memoized potential terms (Sec. 5)
    u32 grid = 0;
    std::vector<GroupDev> groups;
    std::vector<SearchDev> searches;
    std::vector<PartnerDev> partners;
    std::vector<QEdgeDev> qedges;
    std::vector<u32> map;              // input query -> global query edge, NONE for s == t
    std::vector<std::pair<u32, u32>> qedge_ends;  // global query edge -> (s, t) vertices
    std::vector<u32> team_first, team_size, team_queue, cta_team;
    std::vector<u32> queue_items[MAX_QUEUES];
    std::vector<Slot*> slots;
    void* d_arena = nullptr;
    size_t arena_bytes = 0;
    char* d_runstate = nullptr;
    size_t runstate_bytes = 0;
    u32* d_map = nullptr;
    EngineArgs args{};
    bool launched = false;
    // learned Delta: per-group features (log2(1 + raw)) and the model used
    std::vector<float> feats;
    float* d_feats = nullptr;
    ppsp_delta_model* model = nullptr;
    u64 delta_default = 1;
    // paths (ppsp_query / ppsp_batch with want_paths)
    bool paths = false;
    std::vector<u64> path_off;  // [qedges + 1]
    void* d_paths = nullptr;    // path buffer, offsets, lengths, meeting vertices
    u32* d_meet = nullptr;
    // CUDA-graph replay of plan_run (per output pointer)
    cudaGraphExec_t gexec = nullptr;
    u64* gexec_out = nullptr;
    bool graph_failed = false;
    bool last_used_graph = false;
};

namespace {

struct UF {
    std::vector<u32> p;
    explicit UF(u32 n) : p(n) { std::iota(p.begin(), p.end(), 0u); }
    u32 find(u32 x) {
        while (p[x] != x) x = p[x] = p[p[x]];
        return x;
    }
    void join(u32 a, u32 b) {
        a = find(a);
        b = find(b);
        if (a != b) p[std::max(a, b)] = std::min(a, b);
    }
};

// Minimum vertex cover of a graph of at most 32 vertices given as adjacency
// bit masks, by branch and bound: take the vertex v of largest uncovered
// degree and branch on "v in the cover" / "all uncovered neighbours of v in
// the cover"; a greedy maximal matching of the uncovered edges bounds the
// rest from below (every matching edge needs its own cover vertex), and once
// no vertex has two uncovered edges the remaining edges form a matching.
void vc_exact(const std::vector<u32>& adj, u32 cover, u32 size, u32& best_size, u32& best) {
    if (size >= best_size) return;
    const u32 nv = (u32)adj.size();
    u32 v = 0, maxd = 0;
    for (u32 u = 0; u < nv; ++u) {
        if (cover >> u & 1u) continue;
        const u32 d = (u32)__builtin_popcount(adj[u] & ~cover);
        if (d > maxd) {
            maxd = d;
            v = u;
        }
    }
    if (maxd <= 1) {
        u32 c = cover, sz = size;
        for (u32 u = 0; u < nv; ++u)
            if (!(c >> u & 1u) && (adj[u] & ~c)) {
                c |= 1u << u;
                ++sz;
            }
        if (sz < best_size) {
            best_size = sz;
            best = c;
        }
        return;
    }
    u32 m = cover, lb = 0;
    for (u32 u = 0; u < nv; ++u) {
        if (m >> u & 1u) continue;
        const u32 w = adj[u] & ~m;
        if (w) {
            m |= (1u << u) | (w & (0u - w));
            ++lb;
        }
    }
    if (size + lb >= best_size) return;
    vc_exact(adj, cover | (1u << v), size + 1, best_size, best);
    const u32 nb = adj[v] & ~cover;
    vc_exact(adj, cover | nb, size + (u32)__builtin_popcount(nb), best_size, best);
}

// Vertex cover of the query graph (Sec. 4.3): exact for components of at most
// 32 vertices, greedy by uncovered degree otherwise.  Returns in[v] for the
// local vertex ids 0..nv-1.
std::vector<char> vertex_cover(u32 nv, const std::vector<std::pair<u32, u32>>& E) {
    std::vector<u32> comp(nv);
    std::iota(comp.begin(), comp.end(), 0u);
    std::function<u32(u32)> find = [&](u32 x) { return comp[x] == x ? x : comp[x] = find(comp[x]); };
    for (auto& e : E) comp[find(e.first)] = find(e.second);
    std::unordered_map<u32, std::vector<u32>> cv;
    std::unordered_map<u32, std::vector<std::pair<u32, u32>>> ce;
    for (u32 v = 0; v < nv; ++v) cv[find(v)].push_back(v);
    for (auto& e : E) ce[find(e.first)].push_back(e);
    std::vector<char> in(nv, 0);
    for (auto& kv : cv) {
        auto& verts = kv.second;
        auto& edges = ce[kv.first];
        if (edges.empty()) continue;
        if (verts.size() <= 32) {
            std::unordered_map<u32, u32> loc;
            for (u32 i = 0; i < verts.size(); ++i) loc[verts[i]] = i;
            std::vector<u32> adj(verts.size(), 0u);
            for (auto& e : edges) {
                const u32 x = loc[e.first], y = loc[e.second];
                adj[x] |= 1u << y;
                adj[y] |= 1u << x;
            }
            u32 best = (verts.size() == 32) ? ~0u : ((1u << verts.size()) - 1u), best_size = (u32)verts.size();
            vc_exact(adj, 0u, 0, best_size, best);
            for (u32 i = 0; i < verts.size(); ++i) in[verts[i]] = (char)(best >> i & 1u);
        } else {
            std::vector<char> covered(edges.size(), 0);
            size_t left = edges.size();
            while (left) {
                std::unordered_map<u32, u32> deg;
                for (size_t k = 0; k < edges.size(); ++k)
                    if (!covered[k]) {
                        ++deg[edges[k].first];
                        ++deg[edges[k].second];
                    }
                u32 pick = 0, pd = 0;
                for (auto& d : deg)
                    if (d.second > pd || (d.second == pd && d.first < pick)) {
                        pick = d.first;
                        pd = d.second;
                    }
                in[pick] = 1;
                for (size_t k = 0; k < edges.size(); ++k)
                    if (!covered[k] && (edges[k].first == pick || edges[k].second == pick)) {
                        covered[k] = 1;
                        --left;
                    }
            }
        }
    }
    return in;
}

// Minimum vertex cover of a bipartite graph (left 0..nl-1, right
// 0..nr-1): a maximum matching by augmenting paths, then Konig's
// construction (left vertices not reachable by alternating paths from free
// left vertices, right vertices reachable).  Returns cover flags.
void bipartite_cover(u32 nl, u32 nr, const std::vector<std::pair<u32, u32>>& E, std::vector<char>& inl,
                     std::vector<char>& inr) {
    std::vector<std::vector<u32>> adjl(nl);
    for (auto& e : E) adjl[e.first].push_back(e.second);
    std::vector<u32> ml(nl, NONE), mr(nr, NONE);
    std::vector<u32> seen(nr, NONE);
    // iterative augmenting-path search from left vertex r0 (stamp = r0)
    auto augment = [&](u32 r0) {
        std::vector<std::pair<u32, u32>> st;  // (left vertex, next edge index)
        std::vector<u32> via;                 // right vertex taken from each frame
        st.emplace_back(r0, 0);
        while (!st.empty()) {
            auto& [x, k] = st.back();
            if (k == adjl[x].size()) {
                st.pop_back();
                if (!via.empty()) via.pop_back();
                continue;
            }
            const u32 y = adjl[x][k++];
            if (seen[y] == r0) continue;
            seen[y] = r0;
            if (mr[y] == NONE) {
                // flip the path: frames hold left vertices, via the right ones
                via.push_back(y);
                for (size_t f = st.size(); f-- > 0;) {
                    const u32 lx = st[f].first, ry = via[f];
                    ml[lx] = ry;
                    mr[ry] = lx;
                }
                return true;
            }
            via.push_back(y);
            st.emplace_back(mr[y], 0);
        }
        return false;
    };
    for (u32 x = 0; x < nl; ++x) augment(x);
    // alternating reachability from free left vertices
    std::vector<char> zl(nl, 0), zr(nr, 0);
    std::vector<u32> queue;
    for (u32 x = 0; x < nl; ++x)
        if (ml[x] == NONE) {
            zl[x] = 1;
            queue.push_back(x);
        }
    for (size_t h = 0; h < queue.size(); ++h) {
        const u32 x = queue[h];
        for (u32 y : adjl[x])
            if (!zr[y] && ml[x] != y) {
                zr[y] = 1;
                const u32 x2 = mr[y];
                if (x2 != NONE && !zl[x2]) {
                    zl[x2] = 1;
                    queue.push_back(x2);
                }
            }
    }
    inl.assign(nl, 0);
    inr.assign(nr, 0);
    for (u32 x = 0; x < nl; ++x) inl[x] = zl[x] ? 0 : 1;
    for (u32 y = 0; y < nr; ++y) inr[y] = zr[y] ? 1 : 0;
}

// Search that answers each query (s, t) of an SSSP-based batch (Sec. 4.3),
// as (vertex, direction): Plain-SSSP searches forward from s; VC-SSSP from an
// endpoint in a vertex cover of G_q: on an undirected graph (direction 0)
// exact up to 32 vertices per component and greedy above; on a directed
// graph G_q is bipartite (sources, targets: Sec. 4.4) and its minimum cover
// comes from a maximum matching (Konig); a target in the cover searches
// backward (direction 1) over the transpose.
struct SrcDir {
    u32 v;
    u32 dir;
};
std::vector<SrcDir> sssp_sources(int strategy, bool directed, const std::vector<std::pair<u32, u32>>& uq) {
    const u32 U = (u32)uq.size();
    std::vector<SrcDir> src(U);
    if (strategy != PPSP_BATCH_VC) {
        for (u32 u = 0; u < U; ++u) src[u] = {uq[u].first, 0};
        return src;
    }
    if (directed) {
        std::unordered_map<u32, u32> lid, rid;
        std::vector<std::pair<u32, u32>> E(U);
        for (u32 u = 0; u < U; ++u)
            E[u] = {lid.emplace(uq[u].first, (u32)lid.size()).first->second,
                    rid.emplace(uq[u].second, (u32)rid.size()).first->second};
        std::vector<char> inl, inr;
        bipartite_cover((u32)lid.size(), (u32)rid.size(), E, inl, inr);
        for (u32 u = 0; u < U; ++u)
            src[u] = inl[E[u].first] ? SrcDir{uq[u].first, 0} : SrcDir{uq[u].second, 1};
        return src;
    }
    std::unordered_map<u32, u32> vid;
    std::vector<u32> verts;
    auto get = [&](u32 v) {
        auto it = vid.find(v);
        if (it != vid.end()) return it->second;
        vid.emplace(v, (u32)verts.size());
        verts.push_back(v);
        return (u32)verts.size() - 1;
    };
    std::vector<std::pair<u32, u32>> le(U);
    for (u32 u = 0; u < U; ++u) le[u] = {get(uq[u].first), get(uq[u].second)};
    const std::vector<char> in = vertex_cover((u32)verts.size(), le);
    for (u32 u = 0; u < U; ++u) src[u] = {in[le[u].first] ? uq[u].first : uq[u].second, 0};
    return src;
}

// AUTO strategy: smallest number of targets that makes a source's queries
// one multi-target search (ET / A* modes).
constexpr u32 AUTO_MIN_TARGETS = 4;

// AUTO strategy, per connected component of G_q with nv vertices, ne edges
// and a vertex cover of `cover` vertices.  With BiD-A* potentials a pair
// search settles far fewer vertices than an unpruned or shared search (the
// potential is only exact for isolated pairs, so shared searches lose it):
// components run as independent pairs unless one vertex covers the whole
// component (a star), whose one search from the centre answers every query.
// Without potentials, a cover of at most a quarter of the vertices runs as
// VC-SSSP (stars, forks), the rest as Multi-BiDS (Sec. 4.2 / 4.3).  On a
// dense low-diameter graph (average degree at least AUTO_DENSE_DEG, the
// social-graph shape) every component, an isolated pair too, runs as
// VC-SSSP: there a search that stops at its last target beats the
// bidirectional searches (measured on RMAT-22: 1.6 s against 3.7 s for the
// same batch, Sec. 4.3 notes the same trend for social graphs).
constexpr double AUTO_DENSE_DEG = 8.0;
int auto_component(bool pot_pairs, bool dense, u32 nv, u32 ne, u32 cover) {
    if (pot_pairs) return (cover == 1 && ne >= AUTO_MIN_TARGETS) ? PPSP_BATCH_VC : PPSP_BATCH_PLAIN_STAR;
    if (dense) return PPSP_BATCH_VC;
    return (4u * cover <= nv) ? PPSP_BATCH_VC : PPSP_BATCH_MULTI;
}

u32 ceil_log2(u32 x) {
    u32 s = 0;
    while ((1u << s) < x) ++s;
    return s;
}

ppsp_status check_options(const ppsp_graph* g, const ppsp_options& o) {
    if (o.mode < PPSP_BIDS || o.mode > PPSP_ASTAR) return PPSP_ERR_INVALID_ARG;
    if (o.dist_bits != 32 && o.dist_bits != 64) return PPSP_ERR_INVALID_ARG;
    if (o.block_threads != 0 && o.block_threads != 256 && o.block_threads != 512 && o.block_threads != 1024)
        return PPSP_ERR_INVALID_ARG;
    if (o.frontier < PPSP_FRONTIER_AUTO || o.frontier > PPSP_FRONTIER_DENSE) return PPSP_ERR_INVALID_ARG;
    if (o.layout < PPSP_LAYOUT_AUTO || o.layout > PPSP_LAYOUT_STACKED) return PPSP_ERR_INVALID_ARG;
    if (o.batch_strategy < PPSP_BATCH_MULTI || o.batch_strategy > PPSP_BATCH_AUTO) return PPSP_ERR_INVALID_ARG;
    if ((o.batch_strategy == PPSP_BATCH_SSSP || o.batch_strategy == PPSP_BATCH_VC) && o.want_paths)
        return PPSP_ERR_UNSUPPORTED;
    if (o.team_ctas < 0 || o.big_team_ctas < 0 || o.max_ctas < 0) return PPSP_ERR_INVALID_ARG;
    if (o.ring_entries > 256) return PPSP_ERR_INVALID_ARG;
    const bool astar = o.mode == PPSP_BIDASTAR || o.mode == PPSP_ASTAR;
    if (astar && !g->info.has_coords) return PPSP_ERR_NO_COORDS;
    const bool bidir = o.mode == PPSP_BIDS || o.mode == PPSP_BIDASTAR;
    return PPSP_OK;
}

}  // namespace

static void plan_free_partial(ppsp_plan* P) {
    // a new slot may still be initialising on the plan's stream
    cudaStreamSynchronize(P->stream);
    for (Slot* x : P->slots) slot_release(P->g, x);
    P->slots.clear();
    // stream-ordered frees: no device-wide synchronisation, so plans on other
    // streams keep running (the serving loop closes plans while others run)
    if (P->d_arena) cudaFreeAsync(P->d_arena, P->stream);
    if (P->d_paths) cudaFreeAsync(P->d_paths, P->stream);
    P->d_arena = nullptr;
    P->d_paths = nullptr;
    cudaGetLastError();
}

// Build everything from host pairs.  Separated so ppsp_query can reuse it.
static ppsp_status plan_create_impl(ppsp_graph* g, const uint32_t* pairs, uint64_t k, const ppsp_options* opt_in,
                                    bool single_query, ppsp_plan** out, const u64* path_caps = nullptr) {
    ppsp_options o;
    if (opt_in)
        o = *opt_in;
    else
        ppsp_options_init(&o);
    ppsp_status st = check_options(g, o);
    if (st != PPSP_OK) return st;
    if (k && !pairs) return PPSP_ERR_INVALID_ARG;
    if (o.want_paths && (!path_caps || g->info.has_zero_weight)) return PPSP_ERR_UNSUPPORTED;
    const u64 n = g->n;
    for (u64 q = 0; q < 2 * k; ++q)
        if (pairs[q] >= n) return PPSP_ERR_INVALID_ARG;
    // the graph's device order (caller ids in, device ids from here on)
    std::vector<u32> pairs_dev;
    if (!g->perm.empty()) {
        pairs_dev.resize(2 * k);
        for (u64 q = 0; q < 2 * k; ++q) pairs_dev[q] = g->perm[pairs[q]];
        pairs = pairs_dev.data();
    }

    auto P = std::make_unique<ppsp_plan>();
    P->g = g;
    P->opt = o;
    P->k = k;
    P->stream = (cudaStream_t)o.stream;
    P->dist_bits = o.dist_bits;
    const bool bidir = o.mode == PPSP_BIDS || o.mode == PPSP_BIDASTAR;
    P->memo = o.memo_potential && g->info.has_coords && (o.mode == PPSP_BIDASTAR || o.mode == PPSP_ASTAR);
    const u64 delta = o.delta ? o.delta : std::max<u64>(1, (u64)std::llround(g->info.w_mean));
    const int strategy = single_query ? PPSP_BATCH_PLAIN : o.batch_strategy;

    // ---- unique query edges ----
    P->map.assign(k, NONE);
    std::unordered_map<u64, u32> qe_id;
    std::vector<std::pair<u32, u32>> uq;  // unique queries (s, t)
    for (u64 q = 0; q < k; ++q) {
        u32 s = pairs[2 * q], t = pairs[2 * q + 1];
        if (s == t) continue;  // d(s, s) = 0, no search
        // Plain-SSSP searches from every query's own source (ordered pairs)
        const bool unordered = g->info.undirected && ((bidir && strategy != PPSP_BATCH_SSSP) ||
                                                      strategy == PPSP_BATCH_VC || strategy == PPSP_BATCH_AUTO);
        u64 key = unordered ? (((u64)std::min(s, t) << 32) | std::max(s, t)) : (((u64)s << 32) | t);
        auto it = qe_id.find(key);
        if (it == qe_id.end()) {
            it = qe_id.emplace(key, (u32)uq.size()).first;
            uq.emplace_back(s, t);
        }
        P->map[q] = it->second;  // provisional: unique-query index, renumbered below
    }
    const u32 U = (u32)uq.size();

    // ---- groups ----
    // Each group: list of vertices (searches) and list of unique-query indices.
    std::vector<std::vector<u32>> gverts, gqueries;
    std::vector<char> gsssp;                // group is one SSSP-based search (Sec. 4.3)
    // directed graphs: a query's source searches out-edges (direction 0), its
    // target in-edges (direction 1); on undirected graphs every search is 0
    const bool directed = !g->info.undirected;
    std::vector<std::vector<unsigned char>> gdirs;
    std::vector<SrcDir> sssp_src(U, SrcDir{NONE, 0});  // SSSP groups: the search answering each query
    // one SSSP group per distinct source of the queries in `qs`
    auto add_sssp_groups = [&](const std::vector<u32>& qs) {
        std::unordered_map<u64, u32> gid;
        for (u32 u : qs) {
            const u64 key = ((u64)sssp_src[u].v << 1) | sssp_src[u].dir;
            auto it = gid.find(key);
            if (it == gid.end()) {
                it = gid.emplace(key, (u32)gverts.size()).first;
                gverts.push_back({sssp_src[u].v});
                gdirs.push_back({(unsigned char)sssp_src[u].dir});
                gqueries.push_back({});
                gsssp.push_back(1);
            }
            gqueries[it->second].push_back(u);
        }
    };
    auto add_single = [&](u32 u) {
        if (bidir) {
            gverts.push_back({uq[u].first, uq[u].second});
            gdirs.push_back({0, (unsigned char)(directed ? 1 : 0)});
        } else {
            gverts.push_back({uq[u].first});
            gdirs.push_back({0});
        }
        gqueries.push_back({u});
        gsssp.push_back(0);
    };
    if (strategy == PPSP_BATCH_SSSP || strategy == PPSP_BATCH_VC) {
        // Sec. 4.3: one single-source search per selected source
        sssp_src = sssp_sources(strategy, directed, uq);
        std::vector<u32> all(U);
        std::iota(all.begin(), all.end(), 0u);
        add_sssp_groups(all);
    } else if (strategy == PPSP_BATCH_AUTO && !bidir) {
        // one search per target, except sources with several targets, which
        // get one search that stops when all of them are settled
        std::unordered_map<u32, u32> per_src;
        for (u32 u = 0; u < U; ++u) ++per_src[uq[u].first];
        std::vector<u32> multi_t;
        for (u32 u = 0; u < U; ++u) {
            if (per_src[uq[u].first] >= AUTO_MIN_TARGETS && !o.want_paths) {
                sssp_src[u] = {uq[u].first, 0};
                multi_t.push_back(u);
            } else {
                add_single(u);
            }
        }
        add_sssp_groups(multi_t);
    } else if (!bidir || (strategy != PPSP_BATCH_MULTI && strategy != PPSP_BATCH_AUTO)) {
        for (u32 u = 0; u < U; ++u) add_single(u);
    } else {
        // Multi-BiDS: V_q = distinct endpoints, components of G_q (Sec. 4.2).
        // On a directed graph V_q holds (vertex, role) pairs: a source searches
        // forward, a target backward, so G_q is bipartite (Sec. 4.4).
        std::unordered_map<u64, u32> vid;
        std::vector<u32> verts;
        std::vector<unsigned char> vrole;
        auto get = [&](u32 v, unsigned char role) {
            const u64 key = directed ? (((u64)v << 1) | role) : (u64)v;
            auto it = vid.find(key);
            if (it != vid.end()) return it->second;
            vid.emplace(key, (u32)verts.size());
            verts.push_back(v);
            vrole.push_back(directed ? role : 0);
            return (u32)verts.size() - 1;
        };
        std::vector<std::pair<u32, u32>> le(U);
        for (u32 u = 0; u < U; ++u) le[u] = {get(uq[u].first, 0), get(uq[u].second, 1)};
        UF uf((u32)verts.size());
        for (auto& e : le) uf.join(e.first, e.second);
        std::unordered_map<u32, std::vector<u32>> comp_edges;
        std::vector<u32> comp_order;
        for (u32 u = 0; u < U; ++u) {
            u32 r = uf.find(le[u].first);
            auto it = comp_edges.find(r);
            if (it == comp_edges.end()) {
                comp_order.push_back(r);
                it = comp_edges.emplace(r, std::vector<u32>()).first;
            }
            it->second.push_back(u);
        }
        const bool pot_pairs = o.mode == PPSP_BIDASTAR && g->info.has_coords;
        const bool dense = g->info.m >= AUTO_DENSE_DEG * (double)g->info.n;
        for (u32 r : comp_order) {
            const std::vector<u32>& ce = comp_edges[r];
            if (strategy == PPSP_BATCH_AUTO && (ce.size() > 1 || (dense && !pot_pairs && !o.want_paths))) {
                // the cheaper of Multi-BiDS, VC-SSSP and Plain* for this component
                std::unordered_map<u32, u32> cl;
                std::vector<std::pair<u32, u32>> cle;
                for (u32 u : ce) {
                    const u32 a = cl.emplace(le[u].first, (u32)cl.size()).first->second;
                    const u32 b = cl.emplace(le[u].second, (u32)cl.size()).first->second;
                    cle.emplace_back(a, b);
                }
                const std::vector<char> in = vertex_cover((u32)cl.size(), cle);
                u32 cover = 0;
                for (char x : in) cover += x ? 1u : 0u;
                int pick = auto_component(pot_pairs, dense, (u32)cl.size(), (u32)ce.size(), cover);
                if (pick == PPSP_BATCH_VC && o.want_paths)  // SSSP groups record no paths
                    pick = pot_pairs ? PPSP_BATCH_PLAIN_STAR : PPSP_BATCH_MULTI;
                if (pick == PPSP_BATCH_VC) {
                    // on a directed graph the component is bipartite ((vertex,
                    // role) pairs): a target in the cover searches backward
                    for (u32 j = 0; j < ce.size(); ++j)
                        sssp_src[ce[j]] = in[cle[j].first] ? SrcDir{uq[ce[j]].first, 0}
                                                           : SrcDir{uq[ce[j]].second, directed ? 1u : 0u};
                    add_sssp_groups(ce);
                    continue;
                }
                if (pick == PPSP_BATCH_PLAIN_STAR) {
                    for (u32 u : ce) add_single(u);
                    continue;
                }
            }
            // split components with more than KMAX vertices into sub-groups
            std::vector<u32> cur_v, cur_q;
            std::vector<unsigned char> cur_d;
            std::unordered_map<u32, u32> in_cur;
            for (u32 u : comp_edges[r]) {
                u32 a = le[u].first, b = le[u].second;
                u32 need = (in_cur.count(a) ? 0 : 1) + (in_cur.count(b) ? 0 : 1);
                if (cur_v.size() + need > (size_t)KMAX) {
                    gverts.push_back(cur_v);
                    gdirs.push_back(cur_d);
                    gqueries.push_back(cur_q);
                    gsssp.push_back(0);
                    cur_v.clear();
                    cur_d.clear();
                    cur_q.clear();
                    in_cur.clear();
                }
                for (u32 x : {a, b})
                    if (!in_cur.count(x)) {
                        in_cur.emplace(x, (u32)cur_v.size());
                        cur_v.push_back(verts[x]);
                        cur_d.push_back(vrole[x]);
                    }
                cur_q.push_back(u);
            }
            gverts.push_back(cur_v);
            gdirs.push_back(cur_d);
            gqueries.push_back(cur_q);
            gsssp.push_back(0);
        }
    }

    // ---- descriptors ----
    const u32 NG = (u32)gverts.size();
    std::vector<u32> uq_to_qe(U, NONE);
    std::vector<double> gwork(NG, 1.0);
    for (u32 gi = 0; gi < NG; ++gi) {
        GroupDev G{};
        const auto& V = gverts[gi];
        const auto& Q = gqueries[gi];
        G.sbeg = (u32)P->searches.size();
        G.scnt = (u32)V.size();
        G.qbeg = (u32)P->qedges.size();
        G.qcnt = (u32)Q.size();
        G.delta = delta;
        const bool sssp = gsssp[gi] != 0;
        if (sssp) {
            G.mode = GM_SSSP;
            G.target = NONE;
        } else if (bidir) {
            G.mode = GM_BIDIR;
            G.target = NONE;
        } else {
            G.mode = (o.mode == PPSP_ASTAR) ? GM_ASTAR : GM_ET;
            G.target = uq[Q[0]].second;
        }
        if (G.scnt <= 2) {
            G.layout = PPSP_LAYOUT_INTERLEAVED;
            G.kshift = (G.scnt == 2) ? 1 : 0;
        } else {
            G.layout = (o.layout == PPSP_LAYOUT_STACKED) ? PPSP_LAYOUT_STACKED : PPSP_LAYOUT_INTERLEAVED;
            G.kshift = ceil_log2(G.scnt);
        }
        const u64 range = G.layout == PPSP_LAYOUT_INTERLEAVED ? (n << G.kshift) : (u64)G.scnt * n;
        if (range >= 0xFFFFFFFFull) return PPSP_ERR_UNSUPPORTED;
        const auto& Dv = gdirs[gi];
        std::unordered_map<u64, u32> local;  // (vertex, direction) -> search
        auto lkey = [](u32 v, unsigned char d) { return ((u64)v << 1) | d; };
        for (u32 i = 0; i < G.scnt; ++i) local.emplace(lkey(V[i], Dv[i]), i);
        const unsigned char tdir = directed ? 1 : 0;  // direction of a query's target search
        std::vector<std::vector<PartnerDev>> plist(G.scnt);
        std::vector<i64> hmax(G.scnt, 0);
        double work = 0.0;
        for (u32 qi = 0; qi < G.qcnt; ++qi) {
            u32 u = Q[qi];
            u32 qe = G.qbeg + qi;
            uq_to_qe[u] = qe;
            QEdgeDev e;
            if (sssp) {
                // one search; b holds the query's other endpoint (a vertex id)
                e.a = 0;
                e.b = (uq[u].first == sssp_src[u].v && sssp_src[u].dir == 0) ? uq[u].second : uq[u].first;
            } else {
                e.a = local[lkey(uq[u].first, 0)];
                e.b = bidir ? local[lkey(uq[u].second, tdir)] : e.a;
            }
            P->qedges.push_back(e);
            P->qedge_ends.emplace_back(uq[u].first, uq[u].second);
            if (bidir && !sssp) {
                plist[e.a].push_back(PartnerDev{e.b, qe});
                plist[e.b].push_back(PartnerDev{e.a, qe});
            }
            i64 h = g->info.has_coords ? pot_h_host(g, uq[u].first, uq[u].second) : 1;
            hmax[e.a] = std::max(hmax[e.a], h);
            if (!sssp) hmax[e.b] = std::max(hmax[e.b], h);
        }
        for (u32 i = 0; i < G.scnt; ++i) {
            SearchDev s{};
            s.src = V[i];
            s.dir = Dv[i];
            s.pbeg = (u32)P->partners.size();
            s.pcnt = (u32)plist[i].size();
            for (auto& pd : plist[i]) P->partners.push_back(pd);
            s.pot = 0;
            s.pot_b = V[i];
            s.key_off = 0;
            if (sssp) {
                // no pruning, no potential
            } else if (o.mode == PPSP_BIDASTAR && G.scnt == 2) {
                // Sec. 3.5 for an isolated pair: rho_i = h_partner - h_self, so the
                // two searches use exactly opposite potentials (h_F = -h_B, which
                // Theorem 3.4 relies on).
                s.pot = 1;
                s.pot_b = V[plist[i][0].j];
                s.key_off = -pot_h_host(g, s.pot_b, s.src);
            } else if (o.mode == PPSP_BIDASTAR && o.multi_potential && g->info.has_coords && !plist[i].empty()) {
                // a shared search cannot hold the opposite of every partner's
                // potential at once.  By default it runs without one (plain
                // Multi-BiDS); with multi_potential it takes the smallest
                // partner potential (multi-target A*), so that for every query
                // (i, j) it prunes no more than the pair's BiD-A* rule would;
                // the key is shifted so that the source's key is 0
                s.pot = 2;
                i64 hmin = INT64_MAX;
                for (const PartnerDev& pd : plist[i]) hmin = std::min(hmin, pot_h_host(g, V[pd.j], s.src));
                s.key_off = -hmin;
            } else if (o.mode == PPSP_ASTAR && !sssp) {
                s.pot_b = G.target;
                s.key_off = -pot_h_host(g, G.target, s.src);
            }
            P->searches.push_back(s);
            // estimated settled area: a disc of radius hmax / 2 per search of a
            // pruned bidirectional group, of radius hmax for an SSSP group
            work += (double)(hmax[i] + 1) * (double)(hmax[i] + 1) / (sssp ? 1.0 : 4.0);
        }
        gwork[gi] = work;
        P->groups.push_back(G);
    }
    for (u64 q = 0; q < k; ++q)
        if (P->map[q] != NONE) P->map[q] = uq_to_qe[P->map[q]];

    // ---- features of the learned stepping increment (per group) ----
    // raw: heuristic distance, deg(s), deg(t), w mean/std/min/max, n, m,
    // |V_q|, |E_q|, mean query-graph degree; the model sees log2(1 + raw).
    P->delta_default = delta;
    P->feats.assign((size_t)NG * 12, 0.f);
    for (u32 gi = 0; gi < NG; ++gi) {
        const GroupDev& G = P->groups[gi];
        double hsum = 0.0;
        for (u32 qi = 0; qi < G.qcnt; ++qi) {
            auto ends = P->qedge_ends[G.qbeg + qi];
            if (g->info.has_coords) hsum += (double)pot_h_host(g, ends.first, ends.second);
        }
        double dmean = 0.0, dmax = 0.0;
        for (u32 i = 0; i < G.scnt; ++i) {
            double d = (double)g->deg[P->searches[G.sbeg + i].src];
            dmean += d / G.scnt;
            dmax = std::max(dmax, d);
        }
        double ds = (double)g->deg[P->searches[G.sbeg].src];
        double dt = G.scnt >= 2 ? (double)g->deg[P->searches[G.sbeg + 1].src]
                                : (G.target != NONE ? (double)g->deg[G.target] : 0.0);
        if (G.scnt > 2) {
            ds = dmean;
            dt = dmax;
        }
        const double raw[12] = {hsum / std::max<u32>(1, G.qcnt), ds, dt, g->info.w_mean, g->info.w_std,
                                (double)g->info.w_min, (double)g->info.w_max, (double)g->n, (double)g->m,
                                (double)G.scnt, (double)G.qcnt, 2.0 * G.qcnt / std::max<u32>(1, G.scnt)};
        for (int f = 0; f < 12; ++f) P->feats[(size_t)gi * 12 + f] = (float)std::log2(1.0 + std::max(0.0, raw[f]));
    }
    // the models were trained on pair and Multi-BiDS groups: the inference
    // kernel leaves SSSP groups at the default increment
    if (o.delta == 0 && g->delta_model[o.mode] != nullptr) P->model = g->delta_model[o.mode];

    // ---- launch shape ----
    int block = o.block_threads ? o.block_threads : 512;
    int bpsm = 0, sms = 0;
    const u32 ring_cap = o.ring_entries ? o.ring_entries : RING_CAP_DEFAULT;
    st = engine_occupancy(o.dist_bits, block, &bpsm, &sms, false, ring_cap);
    if (st != PPSP_OK) return st;
    if (bpsm < 1) return PPSP_ERR_UNSUPPORTED;
    u32 grid = (u32)(bpsm * sms);
    if (o.max_ctas > 0) grid = std::min<u32>(grid, (u32)o.max_ctas);
    P->block = block;

    // ---- teams and queues ----
    std::vector<u32> big, small;
    for (u32 gi = 0; gi < NG; ++gi) (P->groups[gi].scnt > 2 ? big : small).push_back(gi);
    auto by_work = [&](u32 a, u32 b) { return gwork[a] > gwork[b]; };
    std::stable_sort(big.begin(), big.end(), by_work);
    std::stable_sort(small.begin(), small.end(), by_work);
    struct TeamSpec {
        u32 size, queue;
    };
    // teams for `grid` resident CTAs; returns the CTAs they use
    auto build_teams = [&](u32 grid_in, std::vector<TeamSpec>& teams) -> u32 {
        teams.clear();
        u32 g_used = grid_in;
        if (strategy == PPSP_BATCH_PLAIN) {
            // one query (group) at a time on the whole GPU
            u32 ts = o.team_ctas ? std::min<u32>(grid_in, (u32)o.team_ctas) : grid_in;
            g_used = ts;
            teams.push_back({ts, 1});
            P->queue_items[0].clear();
            P->queue_items[1] = big;
            P->queue_items[1].insert(P->queue_items[1].end(), small.begin(), small.end());
        } else {
            double wb = 0, ws = 0;
            for (u32 gi : big) wb += gwork[gi];
            for (u32 gi : small) ws += gwork[gi];
            u32 g_big = 0;
            if (!big.empty() && small.empty())
                g_big = grid_in;
            else if (!big.empty())
                g_big = std::min<u32>(grid_in - 1, std::max<u32>(1, (u32)std::llround(grid_in * wb / (wb + ws))));
            u32 tb = 0, nbt = 0;
            if (g_big) {
                nbt = std::min<u32>((u32)big.size(), g_big);
                tb = o.big_team_ctas ? std::min<u32>((u32)o.big_team_ctas, g_big) : g_big / nbt;
                nbt = std::max<u32>(1, std::min<u32>(g_big / tb, (u32)big.size()));
                for (u32 t = 0; t < nbt; ++t) teams.push_back({tb, 0});
            }
            u32 g_small = grid_in - nbt * tb;
            if (!small.empty() && g_small > 0) {
                // fewer groups than CTAs: give each group a team of several CTAs
                u32 ts_auto = 1;
                while (ts_auto * 2 <= 32 && (u64)ts_auto * 2 * small.size() <= g_small) ts_auto *= 2;
                u32 ts = o.team_ctas ? std::min<u32>((u32)o.team_ctas, g_small) : ts_auto;
                // no more teams than groups: an idle team would still hold a slot
                u32 nst = std::max<u32>(1, std::min<u32>(g_small / ts, (u32)small.size()));
                for (u32 t = 0; t < nst; ++t) teams.push_back({ts, 1});
                g_small = nst * ts;
            } else {
                g_small = 0;
            }
            g_used = nbt * tb + g_small;
            P->queue_items[0] = big;
            P->queue_items[1] = small;
        }
        if (teams.empty() || g_used == 0) {
            teams.assign(1, {1, 1});
            g_used = 1;
        }
        return g_used;
    };
    auto all_single = [](const std::vector<TeamSpec>& teams) {
        bool one = !teams.empty();
        for (auto& tm : teams) one = one && tm.size == 1;
        return one;
    };
    std::vector<TeamSpec> teams;
    const u32 grid_max = grid;  // resident CTAs of the general kernel
    grid = build_teams(grid_max, teams);

    // ---- block size ----
    // Every team of one CTA runs the bucketed shared-memory path, in the
    // kernel instance without the queue / bitmap path (fewer registers):
    // by default one CTA of 1,024 threads per SM (one group per CTA then
    // finishes sooner: on the road benchmark the longest query drops from 34
    // to 25 ms and the batch from 38.3 to 36.8 ms); block_threads = 512 or
    // 256 gives two or four CTAs per SM, each running its own group.  Teams
    // of several CTAs keep 512 threads (128 registers, no spills on the queue
    // path).  The barrier test hook needs the team barrier, so not with it.
    if (o.frontier == PPSP_FRONTIER_AUTO && o.debug_flags == 0 && all_single(teams)) {
        const int lb = o.block_threads ? o.block_threads : 1024;
        int lbpsm = 0, lsms = 0;
        if (engine_occupancy(o.dist_bits, lb, &lbpsm, &lsms, true, ring_cap) == PPSP_OK && lbpsm >= 1) {
            u32 lgrid = (u32)(lbpsm * lsms);
            if (o.max_ctas > 0) lgrid = std::min<u32>(lgrid, (u32)o.max_ctas);
            if (lgrid >= grid) {
                std::vector<TeamSpec> t2;
                const u32 g2 = build_teams(lgrid, t2);
                if (all_single(t2)) {
                    teams.swap(t2);
                    grid = g2;
                } else {
                    // the first layout (all single), rebuilt from the same
                    // input so that its queues are restored with it
                    grid = build_teams(grid_max, teams);
                }
                P->block = lb;
                P->local_only = true;
            }
        }
    }
    P->grid = grid;
    u32 first = 0;
    for (u32 t = 0; t < teams.size(); ++t) {
        P->team_first.push_back(first);
        P->team_size.push_back(teams[t].size);
        P->team_queue.push_back(teams[t].queue);
        for (u32 c = 0; c < teams[t].size; ++c) P->cta_team.push_back(t);
        first += teams[t].size;
    }
    // every launched CTA belongs to exactly one team (a CTA without one would
    // read past the team tables)
    if (first != grid || grid == 0) {
        set_last_internal_error("team layout covers %u CTAs of a grid of %u", first, grid);
        return PPSP_ERR_CUDA;
    }

    // ---- slots ----
    u64 range_q[MAX_QUEUES] = {0, 0};
    for (u32 qd = 0; qd < MAX_QUEUES; ++qd)
        for (u32 gi : P->queue_items[qd]) {
            const GroupDev& G = P->groups[gi];
            u64 range = G.layout == PPSP_LAYOUT_INTERLEAVED ? (n << G.kshift) : (u64)G.scnt * n;
            range_q[qd] = std::max(range_q[qd], range);
        }
    for (u32 t = 0; t < teams.size(); ++t) {
        const SlotCaps sc = slot_caps(range_q[teams[t].queue], o.frontier, teams[t].size == grid);
        Slot* s = nullptr;
        st = slot_acquire(g, o.dist_bits, sc.flat_cap, sc.qcap, sc.tcap, P->memo, P->stream, &s);
        if (st != PPSP_OK) {
            cudaStreamSynchronize(P->stream);  // new slots may still be initialising
            cudaGetLastError();
            for (Slot* x : P->slots) slot_release(g, x);
            return st;
        }
        P->slots.push_back(s);
    }

    // ---- device arena ----
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const u32 NT = (u32)teams.size();
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o2 = off;
        off += al(std::max<size_t>(bytes, 1));
        return o2;
    };
    size_t o_groups = take(P->groups.size() * sizeof(GroupDev));
    size_t o_search = take(P->searches.size() * sizeof(SearchDev));
    size_t o_part = take(P->partners.size() * sizeof(PartnerDev));
    size_t o_qe = take(P->qedges.size() * sizeof(QEdgeDev));
    size_t o_ctat = take(P->cta_team.size() * 4);
    size_t o_tf = take(NT * 4), o_tsz = take(NT * 4), o_tq = take(NT * 4);
    size_t o_slots = take(NT * sizeof(SlotDev));
    size_t o_q0 = take(P->queue_items[0].size() * 4), o_q1 = take(P->queue_items[1].size() * 4);
    size_t o_map = take(k * 4);
    size_t o_feat = take(P->feats.size() * 4);
    size_t static_bytes = off;
    size_t o_mu = take(P->qedges.size() * 8);
    size_t o_mumax = take(P->searches.size() * 8);
    size_t o_run = off;
    size_t o_qh = take(MAX_QUEUES * 4);
    size_t o_ts = take(NT * sizeof(TeamState));
    size_t o_err = take(4);
    size_t o_cnt = take(sizeof(EngineCounters));
    size_t o_gns = take(P->groups.size() * 8);
    P->runstate_bytes = off - o_run;
    P->arena_bytes = off;
    cudaError_t ce = cudaMallocAsync(&P->d_arena, P->arena_bytes, P->stream);
    if (ce != cudaSuccess) {
        cudaGetLastError();
        cudaStreamSynchronize(P->stream);  // new slots may still be initialising
        cudaGetLastError();
        for (Slot* x : P->slots) slot_release(g, x);
        return ce == cudaErrorMemoryAllocation ? PPSP_ERR_OOM : PPSP_ERR_CUDA;
    }
    char* base = (char*)P->d_arena;
    std::vector<char> h(static_bytes, 0);
    auto put = [&](size_t o2, const void* src, size_t bytes) {
        if (bytes) memcpy(h.data() + o2, src, bytes);
    };
    put(o_groups, P->groups.data(), P->groups.size() * sizeof(GroupDev));
    put(o_search, P->searches.data(), P->searches.size() * sizeof(SearchDev));
    put(o_part, P->partners.data(), P->partners.size() * sizeof(PartnerDev));
    put(o_qe, P->qedges.data(), P->qedges.size() * sizeof(QEdgeDev));
    put(o_ctat, P->cta_team.data(), P->cta_team.size() * 4);
    put(o_tf, P->team_first.data(), NT * 4);
    put(o_tsz, P->team_size.data(), NT * 4);
    put(o_tq, P->team_queue.data(), NT * 4);
    std::vector<SlotDev> sd(NT);
    for (u32 t = 0; t < NT; ++t) sd[t] = P->slots[t]->dev;
    put(o_slots, sd.data(), NT * sizeof(SlotDev));
    put(o_q0, P->queue_items[0].data(), P->queue_items[0].size() * 4);
    put(o_q1, P->queue_items[1].data(), P->queue_items[1].size() * 4);
    put(o_map, P->map.data(), k * 4);
    put(o_feat, P->feats.data(), P->feats.size() * 4);
    // pageable source: staged before the call returns, so h may go out of scope
    ce = cudaMemcpyAsync(base, h.data(), static_bytes, cudaMemcpyHostToDevice, P->stream);
    if (ce != cudaSuccess) {
        cudaGetLastError();
        plan_free_partial(P.get());
        return PPSP_ERR_CUDA;
    }

    EngineArgs& a = P->args;
    a.g = g->dev();
    a.groups = (const GroupDev*)(base + o_groups);
    a.searches = (const SearchDev*)(base + o_search);
    a.partners = (const PartnerDev*)(base + o_part);
    a.qedges = (const QEdgeDev*)(base + o_qe);
    a.mu = (u64*)(base + o_mu);
    a.mumax = (u64*)(base + o_mumax);
    a.cta_team = (const u32*)(base + o_ctat);
    a.team_first = (const u32*)(base + o_tf);
    a.team_size = (const u32*)(base + o_tsz);
    a.team_queue = (const u32*)(base + o_tq);
    a.tstate = (TeamState*)(base + o_ts);
    a.slots = (SlotDev*)(base + o_slots);
    a.queue_items[0] = (const u32*)(base + o_q0);
    a.queue_items[1] = (const u32*)(base + o_q1);
    a.queue_len[0] = (u32)P->queue_items[0].size();
    a.queue_len[1] = (u32)P->queue_items[1].size();
    a.queue_head = (u32*)(base + o_qh);
    a.dense_den = o.dense_den ? o.dense_den : 16u;
    a.frontier = (u32)o.frontier;
    a.rho = o.stepping_rho;
    a.memo = P->memo ? 1u : 0u;
    a.ring_cap = ring_cap;
    a.pull = (o.pull_push && g->info.undirected) ? 1u : 0u;
    a.debug = o.debug_flags;
    a.spin_limit = o.spin_limit ? o.spin_limit : (1ull << 26);
    a.err = (u32*)(base + o_err);
    a.counters = (EngineCounters*)(base + o_cnt);
    a.group_ns = (u64*)(base + o_gns);
    P->d_runstate = base + o_run;
    P->d_map = (u32*)(base + o_map);
    P->d_feats = (float*)(base + o_feat);
    if (o.want_paths) {
        const u64 NQ = P->qedges.size();
        std::vector<u64> cap(NQ, 0);
        for (u64 q = 0; q < k; ++q)
            if (P->map[q] != NONE) cap[P->map[q]] = std::max(cap[P->map[q]], path_caps[q]);
        P->path_off.assign(NQ + 1, 0);
        for (u64 e = 0; e < NQ; ++e) P->path_off[e + 1] = P->path_off[e] + cap[e];
        const size_t b_buf = ((P->path_off[NQ] * 4) + 255) & ~(size_t)255;
        const size_t b_off = ((NQ + 1) * 8 + 255) & ~(size_t)255;
        const size_t b_len = (NQ * 8 + 255) & ~(size_t)255;
        const size_t b_meet = (NQ * 4 + 255) & ~(size_t)255;
        ce = cudaMallocAsync(&P->d_paths, std::max<size_t>(256, b_buf + b_off + b_len + b_meet), P->stream);
        if (ce != cudaSuccess) {
            cudaGetLastError();
            plan_free_partial(P.get());
            return ce == cudaErrorMemoryAllocation ? PPSP_ERR_OOM : PPSP_ERR_CUDA;
        }
        char* pb = (char*)P->d_paths;
        a.path_buf = (u32*)pb;
        a.path_off = (const u64*)(pb + b_buf);
        a.path_len = (u64*)(pb + b_buf + b_off);
        P->d_meet = (u32*)(pb + b_buf + b_off + b_len);
        a.meet = P->d_meet;
        ce = cudaMemcpyAsync((void*)a.path_off, P->path_off.data(), (NQ + 1) * 8, cudaMemcpyHostToDevice,
                             P->stream);
        if (ce != cudaSuccess) {
            cudaGetLastError();
            plan_free_partial(P.get());
            return PPSP_ERR_CUDA;
        }
        P->paths = true;
    }
    *out = P.release();
    return PPSP_OK;
}

static void plan_free(ppsp_plan* P) {
    if (!P) return;
    if (P->stream)
        cudaStreamSynchronize(P->stream);
    else
        cudaDeviceSynchronize();
    for (Slot* s : P->slots) slot_release(P->g, s);
    if (P->gexec) cudaGraphExecDestroy(P->gexec);
    if (P->d_arena) cudaFreeAsync(P->d_arena, P->stream);
    if (P->d_paths) cudaFreeAsync(P->d_paths, P->stream);
    cudaGetLastError();
    delete P;
}

static ppsp_status plan_launch_direct(ppsp_plan* P, u64* d_out);

// Capture the launches of one run into a CUDA graph (once per output pointer)
// and replay it; any capture failure falls back to direct launches.
static ppsp_status plan_launch(ppsp_plan* P, u64* d_out) {
    P->last_used_graph = false;
    bool dirty = false;
    for (const Slot* s : P->slots) dirty = dirty || s->dirty;
    if (!P->opt.cuda_graph || P->stream == nullptr || P->graph_failed || dirty)
        return plan_launch_direct(P, d_out);
    if (P->gexec == nullptr || P->gexec_out != d_out) {
        if (P->gexec) {
            cudaGraphExecDestroy(P->gexec);
            P->gexec = nullptr;
        }
        cudaGraph_t graph = nullptr;
        if (cudaStreamBeginCapture(P->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
            cudaGetLastError();
            P->graph_failed = true;
            return plan_launch_direct(P, d_out);
        }
        ppsp_status st = plan_launch_direct(P, d_out);
        cudaError_t ce = cudaStreamEndCapture(P->stream, &graph);
        if (st != PPSP_OK || ce != cudaSuccess || graph == nullptr) {
            cudaGetLastError();
            if (graph) cudaGraphDestroy(graph);
            P->graph_failed = true;
            return plan_launch_direct(P, d_out);
        }
        ce = cudaGraphInstantiate(&P->gexec, graph, 0);
        cudaGraphDestroy(graph);
        if (ce != cudaSuccess) {
            cudaGetLastError();
            P->gexec = nullptr;
            P->graph_failed = true;
            return plan_launch_direct(P, d_out);
        }
        P->gexec_out = d_out;
    }
    PPSP_CUDA_TRY(cudaGraphLaunch(P->gexec, P->stream));
    P->launched = true;
    P->last_used_graph = true;
    return PPSP_OK;
}

static ppsp_status plan_launch_direct(ppsp_plan* P, u64* d_out) {
    for (Slot* s : P->slots) {
        ppsp_status st = slot_scrub(s, P->stream);
        if (st != PPSP_OK) return st;
    }
    ppsp_status st = PPSP_OK;
    PPSP_CUDA_TRY(cudaMemsetAsync(P->d_runstate, 0, P->runstate_bytes, P->stream));
    if (P->paths && !P->qedges.empty())
        PPSP_CUDA_TRY(cudaMemsetAsync(P->d_meet, 0xFF, P->qedges.size() * 4, P->stream));
    if (P->model && !P->groups.empty()) {
        // learned Delta per group, written into the device group descriptors
        st = mlp_launch_infer(P->model, P->d_feats, P->groups.size(), nullptr, const_cast<GroupDev*>(P->args.groups),
                              P->delta_default, P->stream);
        if (st != PPSP_OK) return st;
    }
    if (!P->groups.empty()) {
        st = launch_engine(P->args, P->dist_bits, P->block, P->grid, P->stream, P->local_only);
        if (st != PPSP_OK) return st;
    }
    if (d_out) {
        st = launch_scatter(P->d_map, P->args.mu, P->k, d_out, P->stream);
        if (st != PPSP_OK) return st;
    }
    P->launched = true;
    return PPSP_OK;
}

static ppsp_status plan_wait(ppsp_plan* P, ppsp_counters* counters) {
    if (P->stream) {
        PPSP_CUDA_TRY(cudaStreamSynchronize(P->stream));
    } else {
        PPSP_CUDA_TRY(cudaDeviceSynchronize());
    }
    u32 err = 0;
    EngineCounters ec{};
    PPSP_CUDA_TRY(cudaMemcpyAsync(&err, P->args.err, 4, cudaMemcpyDeviceToHost, P->stream));
    PPSP_CUDA_TRY(cudaMemcpyAsync(&ec, P->args.counters, sizeof(ec), cudaMemcpyDeviceToHost, P->stream));
    PPSP_CUDA_TRY(cudaStreamSynchronize(P->stream));
    if (counters) {
        memset(counters, 0, sizeof(*counters));
        counters->extracted = ec.extracted;
        counters->edges = ec.edges;
        counters->relaxed = ec.relaxed;
        counters->pushed = ec.pushed;
        counters->rounds = ec.rounds;
        counters->groups = ec.groups;
        counters->searches = ec.searches;
        counters->touched = ec.touched;
        counters->dense_rounds = ec.dense_rounds;
    }
    if (err) {
        for (Slot* s : P->slots) s->dirty = true;
        if (err & ERRB_OVERFLOW) return PPSP_ERR_OVERFLOW;
        if (err & ERRB_TIMEOUT) return PPSP_ERR_TIMEOUT;
        set_last_device_error(err);
        return PPSP_ERR_CUDA;
    }
    return PPSP_OK;
}

extern "C" {

ppsp_status ppsp_plan_create(ppsp_graph* g, const uint32_t* pairs, uint64_t k, const ppsp_options* opt,
                             ppsp_plan** out) {
    if (!g || !out) return PPSP_ERR_INVALID_ARG;
    *out = nullptr;
    std::lock_guard<std::mutex> lk(g->mu);
    return plan_create_impl(g, pairs, k, opt, false, out);
}

ppsp_status ppsp_plan_run(ppsp_plan* p, uint64_t* d_dists_out) {
    if (!p) return PPSP_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(p->g->mu);
    return plan_launch(p, d_dists_out);
}

ppsp_status ppsp_plan_sync(ppsp_plan* p, ppsp_counters* counters) {
    if (!p) return PPSP_ERR_INVALID_ARG;
    if (!p->launched) return PPSP_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(p->g->mu);
    return plan_wait(p, counters);
}

ppsp_status ppsp_plan_features(const ppsp_plan* p, float* out, uint64_t cap, uint64_t* ngroups) {
    if (!p || !ngroups) return PPSP_ERR_INVALID_ARG;
    *ngroups = p->groups.size();
    if (out) {
        if (cap < p->groups.size()) return PPSP_ERR_BUFFER_TOO_SMALL;
        memcpy(out, p->feats.data(), p->feats.size() * 4);
    }
    return PPSP_OK;
}

ppsp_status ppsp_plan_group_times(ppsp_plan* p, uint64_t* out_ns, uint64_t cap, uint64_t* ngroups) {
    if (!p || !ngroups) return PPSP_ERR_INVALID_ARG;
    *ngroups = p->groups.size();
    if (!out_ns) return PPSP_OK;
    if (cap < p->groups.size()) return PPSP_ERR_BUFFER_TOO_SMALL;
    if (!p->launched) return PPSP_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(p->g->mu);
    if (p->stream) {
        PPSP_CUDA_TRY(cudaStreamSynchronize(p->stream));
    } else {
        PPSP_CUDA_TRY(cudaDeviceSynchronize());
    }
    if (!p->groups.empty())
        PPSP_CUDA_TRY(cudaMemcpy(out_ns, p->args.group_ns, p->groups.size() * 8, cudaMemcpyDeviceToHost));
    return PPSP_OK;
}

ppsp_status ppsp_batch_sources(const uint32_t* pairs, uint64_t k, int32_t strategy, uint32_t flags,
                               uint32_t* src_out, uint32_t* dir_out, uint64_t* n_sources) {
    if ((k && !pairs) || (k && !src_out) || !n_sources) return PPSP_ERR_INVALID_ARG;
    if (strategy != PPSP_BATCH_SSSP && strategy != PPSP_BATCH_VC) return PPSP_ERR_INVALID_ARG;
    // the same deduplication as the plan: unordered pairs for VC-SSSP on an
    // undirected graph, ordered pairs otherwise
    const bool directed = !(flags & PPSP_UNDIRECTED);
    const bool unordered = !directed && strategy == PPSP_BATCH_VC;
    std::unordered_map<u64, u32> qe_id;
    std::vector<std::pair<u32, u32>> uq;
    std::vector<u32> map(k, NONE);
    for (u64 q = 0; q < k; ++q) {
        const u32 s = pairs[2 * q], t = pairs[2 * q + 1];
        if (s == t) continue;
        const u64 key = unordered ? (((u64)std::min(s, t) << 32) | std::max(s, t)) : (((u64)s << 32) | t);
        auto it = qe_id.find(key);
        if (it == qe_id.end()) {
            it = qe_id.emplace(key, (u32)uq.size()).first;
            uq.emplace_back(s, t);
        }
        map[q] = it->second;
    }
    const std::vector<SrcDir> src = sssp_sources(strategy, directed, uq);
    std::unordered_set<u64> distinct;
    for (const SrcDir& x : src) distinct.insert(((u64)x.v << 1) | x.dir);
    for (u64 q = 0; q < k; ++q) {
        src_out[q] = (map[q] == NONE) ? NONE : src[map[q]].v;
        if (dir_out) dir_out[q] = (map[q] == NONE) ? 0u : src[map[q]].dir;
    }
    *n_sources = distinct.size();
    return PPSP_OK;
}

ppsp_status ppsp_plan_device_bytes(const ppsp_plan* p, uint64_t* slot_bytes, uint64_t* teams,
                                   uint64_t* other_bytes) {
    if (!p) return PPSP_ERR_INVALID_ARG;
    u64 sb = 0;
    for (const Slot* s : p->slots) sb += s->bytes;
    u64 ob = p->arena_bytes;
    if (p->d_paths) {
        const u64 NQ = p->qedges.size();
        auto al = [](u64 x) { return (x + 255) & ~255ull; };
        ob += std::max<u64>(256, al(p->path_off[NQ] * 4) + al((NQ + 1) * 8) + al(NQ * 8) + al(NQ * 4));
    }
    if (slot_bytes) *slot_bytes = sb;
    if (teams) *teams = p->slots.size();
    if (other_bytes) *other_bytes = ob;
    return PPSP_OK;
}

ppsp_status ppsp_slot_bytes(const ppsp_graph* g, uint32_t searches, int32_t dist_bits, int32_t frontier,
                            uint64_t* out) {
    if (!g || !out || searches == 0 || searches > (u32)KMAX) return PPSP_ERR_INVALID_ARG;
    if (dist_bits != 32 && dist_bits != 64) return PPSP_ERR_INVALID_ARG;
    if (frontier < PPSP_FRONTIER_AUTO || frontier > PPSP_FRONTIER_DENSE) return PPSP_ERR_INVALID_ARG;
    // the plan's layouts: a group of k searches spans n * 2^ceil(log2 k)
    // interleaved entries (k entries per vertex for pairs and singles)
    const u64 range = (u64)g->n << ceil_log2(searches);
    // the larger touched list of a team that spans the whole grid
    const SlotCaps sc = slot_caps(range, frontier, true);
    *out = slot_alloc_bytes(dist_bits, sc.flat_cap, sc.qcap, sc.tcap);
    return PPSP_OK;
}

ppsp_status ppsp_plan_uses_graph(const ppsp_plan* p, int32_t* out) {
    if (!p || !out) return PPSP_ERR_INVALID_ARG;
    *out = p->last_used_graph ? 1 : 0;
    return PPSP_OK;
}

void ppsp_plan_destroy(ppsp_plan* p) {
    if (!p) return;
    ppsp_graph* g = p->g;
    std::lock_guard<std::mutex> lk(g->mu);
    plan_free(p);
}

struct HostPaths {
    uint32_t* buf = nullptr;          // caller's path buffer
    const uint64_t* offsets = nullptr;  // per query [k+1] (batch), or null (single query)
    uint64_t single_cap = 0;          // single query: capacity
    uint64_t* lens = nullptr;         // per query needed lengths
};

static ppsp_status run_host(ppsp_graph* g, const uint32_t* pairs, uint64_t k, const ppsp_options* opt,
                            bool single, uint64_t* dists_out, ppsp_counters* counters, const HostPaths* hp) {
    ppsp_plan* P = nullptr;
    std::vector<u64> caps;
    if (hp) {
        caps.resize(k);
        for (u64 q = 0; q < k; ++q) caps[q] = hp->offsets ? hp->offsets[q + 1] - hp->offsets[q] : hp->single_cap;
    }
    ppsp_status st = plan_create_impl(g, pairs, k, opt, single, &P, hp ? caps.data() : nullptr);
    if (st != PPSP_OK) return st;
    u64* d_out = nullptr;
    cudaError_t ce = cudaMallocAsync((void**)&d_out, std::max<u64>(1, k) * 8, P->stream);
    if (ce != cudaSuccess) {
        cudaGetLastError();
        plan_free(P);
        return ce == cudaErrorMemoryAllocation ? PPSP_ERR_OOM : PPSP_ERR_CUDA;
    }
    st = plan_launch(P, d_out);
    if (st == PPSP_OK) st = plan_wait(P, counters);
    if (st == PPSP_OK && k) {
        ce = cudaMemcpyAsync(dists_out, d_out, k * 8, cudaMemcpyDeviceToHost, P->stream);
        if (ce == cudaSuccess) ce = cudaStreamSynchronize(P->stream);
        if (ce != cudaSuccess) {
            cudaGetLastError();
            st = PPSP_ERR_CUDA;
        }
    }
    if (st == PPSP_OK && hp && P->paths) {
        // device paths are per query edge, oriented from its first to its
        // second endpoint; copy (or reverse) them into each query's slice
        const u64 NQ = P->qedges.size();
        std::vector<u64> plen(NQ, 0);
        std::vector<u32> pbuf(P->path_off[NQ]);
        if (NQ) {
            ce = cudaMemcpyAsync(plen.data(), P->args.path_len, NQ * 8, cudaMemcpyDeviceToHost, P->stream);
            if (ce == cudaSuccess && !pbuf.empty())
                ce = cudaMemcpyAsync(pbuf.data(), P->args.path_buf, pbuf.size() * 4, cudaMemcpyDeviceToHost,
                                     P->stream);
            if (ce == cudaSuccess) ce = cudaStreamSynchronize(P->stream);
            if (ce != cudaSuccess) {
                cudaGetLastError();
                st = PPSP_ERR_CUDA;
            }
        }
        bool small = false;
        for (u64 q = 0; q < k && st == PPSP_OK; ++q) {
            const u32 s = pairs[2 * q], t = pairs[2 * q + 1];
            uint32_t* dst = hp->buf + (hp->offsets ? hp->offsets[q] : 0);
            const u64 cap = caps[q];
            u64 len = 0;
            if (s == t) {
                len = 1;
                if (cap >= 1 && hp->buf) dst[0] = s;
            } else if (dists_out[q] != PPSP_INF) {
                const u32 qe = P->map[q];
                len = plen[qe];
                if (len <= cap && len <= P->path_off[qe + 1] - P->path_off[qe] && hp->buf) {
                    // device ids back to the caller's
                    const u32* src = pbuf.data() + P->path_off[qe];
                    const u32 s_dev = g->perm.empty() ? s : g->perm[s];
                    const bool fwd = (P->qedge_ends[qe].first == s_dev);
                    for (u64 x = 0; x < len; ++x) {
                        const u32 y = fwd ? src[x] : src[len - 1 - x];
                        dst[x] = g->inv.empty() ? y : g->inv[y];
                    }
                } else {
                    small = true;
                }
            }
            if (hp->lens) hp->lens[q] = len;
        }
        if (st == PPSP_OK && small) st = PPSP_ERR_BUFFER_TOO_SMALL;
    }
    cudaFreeAsync(d_out, P->stream);
    plan_free(P);
    return st;
}

ppsp_status ppsp_query(ppsp_graph* g, uint32_t s, uint32_t t, const ppsp_options* opt, uint64_t* dist_out,
                       uint32_t* path_buf, uint64_t path_cap, uint64_t* path_len) {
    if (!g || !dist_out) return PPSP_ERR_INVALID_ARG;
    if (path_len) *path_len = 0;
    uint32_t pr[2] = {s, t};
    std::lock_guard<std::mutex> lk(g->mu);
    if (opt && opt->want_paths) {
        if (path_cap && !path_buf) return PPSP_ERR_INVALID_ARG;
        HostPaths hp;
        hp.buf = path_buf;
        hp.single_cap = path_cap;
        hp.lens = path_len;
        return run_host(g, pr, 1, opt, true, dist_out, nullptr, &hp);
    }
    return run_host(g, pr, 1, opt, true, dist_out, nullptr, nullptr);
}

ppsp_status ppsp_batch(ppsp_graph* g, const uint32_t* pairs, uint64_t k, const ppsp_options* opt,
                       uint64_t* dists_out, uint32_t* paths_buf, const uint64_t* path_offsets, uint64_t* path_lens,
                       ppsp_counters* counters) {
    if (!g || (k && (!pairs || !dists_out))) return PPSP_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(g->mu);
    if (opt && opt->want_paths) {
        if (k && (!path_offsets || !paths_buf)) return PPSP_ERR_INVALID_ARG;
        for (u64 q = 0; q < k; ++q)
            if (path_offsets[q + 1] < path_offsets[q]) return PPSP_ERR_INVALID_ARG;
        HostPaths hp;
        hp.buf = paths_buf;
        hp.offsets = path_offsets;
        hp.lens = path_lens;
        return run_host(g, pairs, k, opt, false, dists_out, counters, &hp);
    }
    return run_host(g, pairs, k, opt, false, dists_out, counters, nullptr);
}

}  // extern "C"
