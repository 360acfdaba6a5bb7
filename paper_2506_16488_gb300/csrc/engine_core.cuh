// Persistent PPSP search engine for sm_103a (device code and launch templates;
// engine_{u32,u64}{,_local}.cu instantiate it for each distance width and for
// the one-CTA or general kernel, so the four families compile in parallel).
//
// One cooperative launch runs every group of a batch.  Each team of CTAs loops:
// claim a group, Init (Table 2), then steps of Alg. 2 until the frontier is
// empty, then tidy its slot.  A step is
//   theta <- GetDist(F)            Delta*-stepping threshold (Sec. 2), empty
//                                  buckets skipped
//   for <u,i> in F.Extract(theta)  keys <= theta; the rest stay in F
//     UpdateDistance(<u,i>)        (see "correctness of mu" below)
//     if not Prune(<u,i>):
//       for v in N(u): if WriteMin(delta_i[v], delta_i[u] + w(u,v)):
//         UpdateDistance(<v,i>); if not Prune(<v,i>): F.Add(<v,i>)
// with one team barrier per step.  The frontier of the next step is a bitmap
// over flat (vertex, search) indices (dedup: an entry is added once), plus a
// queue of the newly set indices while the frontier is small ("sparse"); a
// large frontier is processed by scanning the bitmap ("dense"), App. B.
//
// Keys and prune values per plug-in (Table 2), with integer arithmetic:
//   BiDS        key = 2 d,                       prune 2 d >= mu   (mu/2 test doubled)
//   BiD-A*      key = 2 d + rho_i(v) - rho_i(q_i), prune 2 d + rho_i(v) >= mu,
//               rho_i(v) = h_{q_j}(v) - h_{q_i}(v)  (= 2 h_F for the forward search,
//               2 h_B for the backward one: h_F = (h_t - h_s)/2 = -h_B, Sec. 3.5)
//   Multi-BiDS  key = 2 d,                       prune 2 d >= mumax[i]  (Sec. 4.2)
//   Multi-BiDS with A* (the multi-target extension; Sec. 4.4 leaves it open)
//               key = 2 d + phi_i(v) - phi_i(q_i), prune 2 d + phi_i(v) >= mumax[i],
//               phi_i(v) = min_j h_{q_j}(v) - h_{q_i}(v) over the partners j of i:
//               for every query (i, j) each side prunes only where the pair's
//               BiD-A* rule would (min_j h <= h_j, mumax[i] >= mu[i, j])
//   ET          key = d,                         prune d >= mu, update when v = t
//   A*          key = d + h_t(v) - h_t(s),       prune d + h_t(v) >= mu
// The threshold step is 2 Delta on doubled keys and Delta otherwise.
//
// Correctness of mu.  Theorems 3.3/3.4 need, for the two ends x of some edge on
// a shortest path, that mu is updated after both delta_i[x] and delta_j[x] hold
// their final values.  The update at a successful WriteMin reads the other
// search's value; when the two final writes race inside one step neither reader
// may see the other's write.  The extraction-time update closes that gap: steps
// are separated by a barrier with device-scope fences, and if both copies were
// pruned on insertion then 2(delta_i + delta_j) >= mu_i + mu_j >= 2 mu, so x
// cannot improve mu; otherwise one copy is extracted in a later step and its
// update reads both final values.
#pragma once

#include <cooperative_groups.h>

#include <atomic>

#include "ppsp_internal.h"

namespace cg = cooperative_groups;

namespace ppsp {

// ----------------------------------------------------------------------------
// device helpers
// ----------------------------------------------------------------------------
template <typename D>
struct DT;
template <>
struct DT<u32> {
    static constexpr u64 INF = 0xFFFFFFFFull;
    static constexpr u64 MAXV = 0xFFFFFFFEull;
};
template <>
struct DT<u64> {
    static constexpr u64 INF = ~0ull;
    static constexpr u64 MAXV = (1ull << 61);
};

__device__ __forceinline__ u64 ld_dist(const u32* p) { return (u64)__ldcg(p); }
__device__ __forceinline__ u64 ld_dist(const u64* p) {
    return (u64)__ldcg(reinterpret_cast<const unsigned long long*>(p));
}
__device__ __forceinline__ u64 amin_dist(u32* p, u64 v) { return (u64)atomicMin(p, (u32)v); }
__device__ __forceinline__ u64 amin_dist(u64* p, u64 v) {
    return (u64)atomicMin(reinterpret_cast<unsigned long long*>(p), (unsigned long long)v);
}
__device__ __forceinline__ void st_dist(u32* p, u64 v) { *p = (u32)v; }
__device__ __forceinline__ void st_dist(u64* p, u64 v) { *p = v; }

__device__ __forceinline__ u64 ldcg64(const u64* p) {
    return (u64)__ldcg(reinterpret_cast<const unsigned long long*>(p));
}
__device__ __forceinline__ u64 amin64(u64* p, u64 v) {
    return (u64)atomicMin(reinterpret_cast<unsigned long long*>(p), (unsigned long long)v);
}
__device__ __forceinline__ u32 ld_volatile(const u32* p) { return *reinterpret_cast<const volatile u32*>(p); }
__device__ __forceinline__ u64 global_ns() {
    u64 t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Exact floor(sqrt(x)) for x < 2^62: a floating-point estimate, then integer
// correction.  Below 2^48 the float32 estimate is within 1 of the result
// (relative error about 2^-24 on a value below 2^24); above, float64.
__device__ __forceinline__ u64 isqrt_u64(u64 x) {
    if (x < (1ull << 48)) {
        // result below 2^24: 32-bit candidate, 32 x 32 -> 64-bit checks
        u32 r = (u32)sqrtf((float)x);
        while ((u64)r * r > x) --r;
        while ((u64)(r + 1) * (r + 1) <= x) ++r;
        return r;
    }
    u64 r = (u64)sqrt((double)x);
    while (r * r > x) --r;
    while ((r + 1) * (r + 1) <= x) ++r;
    return r;
}

// h_x(v) = floor(|P(v) - P(x)| / 2^F)  (integer potential, Sec. 3.3).
__device__ __forceinline__ i64 pot_h(int2 px, int2 pv, u32 shift) {
    i64 dx = (i64)pv.x - (i64)px.x;
    i64 dy = (i64)pv.y - (i64)px.y;
    u64 d2 = (u64)(dx * dx) + (u64)(dy * dy);
    return (i64)isqrt_u64(d2 >> (2 * shift));
}

__device__ __forceinline__ u32 agg_inc(u32* ctr) {
    cg::coalesced_group g = cg::coalesced_threads();
    u32 base = 0;
    if (g.thread_rank() == 0) base = atomicAdd(ctr, (u32)g.size());
    base = g.shfl(base, 0);
    return base + g.thread_rank();
}

// ----------------------------------------------------------------------------
// team barrier: bounded spin, device-scope release/acquire
// ----------------------------------------------------------------------------
struct TeamCtx {
    u32 team, rank, size;
    TeamState* ts;
    bool global_bar;  // size > 1 or a test hook forces the global path
    u32 expect;       // arrivals that release the barrier
};

static __device__ bool team_sync(const TeamCtx& tc, const EngineArgs& a, u32* s_flag) {
    __syncthreads();
    if (!tc.global_bar) return true;
    if (threadIdx.x == 0) {
        u32 ok = 1;
        u32 gen = ld_volatile(&tc.ts->bar_gen);
        __threadfence();
        u32 arrived = atomicAdd(&tc.ts->bar_count, 1u);
        if (arrived == tc.expect - 1) {
            tc.ts->bar_count = 0;
            __threadfence();
            atomicAdd(&tc.ts->bar_gen, 1u);
        } else {
            u64 it = 0;
            while (ld_volatile(&tc.ts->bar_gen) == gen) {
                if (ld_volatile(a.err) != 0) {  // another CTA failed: leave
                    ok = 0;
                    break;
                }
                if (++it > a.spin_limit) {
                    atomicOr(a.err, ERRB_TIMEOUT);
                    ok = 0;
                    break;
                }
                __nanosleep(32);
            }
        }
        __threadfence();
        *s_flag = ok;
    }
    __syncthreads();
    return *s_flag != 0;
}

// ----------------------------------------------------------------------------
// shared memory
// ----------------------------------------------------------------------------
constexpr u32 QSTAGE = 1024;  // staged frontier appends per CTA and tile
constexpr u32 TSTAGE = 512;   // staged touched-list appends per CTA and tile
constexpr u32 PCAP = 1024;    // partner entries of a group cached in shared memory

constexpr u32 LR_NB = 32;  // buckets in the one-CTA ring

// Edges of a tile up to OWN_MULT * B find their entry in a shared-memory
// owner table instead of a binary search over the degree prefix sums, when no
// entry of the tile has more than OWN_MAXDEG edges (so that filling the table
// costs each thread a few stores).
constexpr u32 OWN_MULT = 4;
constexpr u32 OWN_MAXDEG = 32;

template <int B>
struct Smem {
    // tile of frontier entries
    u32 flat[B];
    u32 beg[B];
    u32 pre[B];
    unsigned short own[OWN_MULT * B];  // entry of each edge of the tile (see OWN_MULT)
    u32 own_off;                       // a tile entry has more than OWN_MAXDEG edges (set by the scan)
    u64 d[B];
    unsigned char si[B];
    u32 wsum[B / 32];
    u32 wbig[B / 32];
    // staging of appends
    u32 qbuf[QSTAGE];
    u32 tbuf[TSTAGE];
    u32 qn, tn, qbase, tbase;
    // group cache
    u32 src[KMAX];
    u32 pbeg[KMAX];
    u32 pcnt[KMAX];
    u32 pot[KMAX];
    u32 sdir[KMAX];  // 0: out-edges (off / edges), 1: in-edges (off_t / edges_t)
    int2 pa[KMAX];
    int2 pb[KMAX];
    i64 key_off[KMAX];
    u64 bound[KMAX];
    PartnerDev pcache[PCAP];
    u32 pcached, pot_any;
    // one-CTA bucketed frontier (run_local)
    u64 lstep, lcur, llate;
    u64 lfirst;         // first bucket of the step (lcur is its last; more than one with rho)
    u32 lpre[LR_NB];    // entries in buckets cur + 1 .. cur + j of the ring (lpre[0] = 0)
    u32 lj0, ljl;       // the step's buckets, relative to the previous step's last bucket
    u64 lfar_min[2];
    u32 lfar_n[2];
    u32 lfar_fb, lfar_tgt, lspill, tov;
    u32 lrecov, lidle;  // spill recovered since the last processed bucket; decisions without one
    u32 lfar_after;     // far-list entries right after the last re-bucketing
    // entries a warp with many edges hands to the whole CTA (process_local)
    u32 fbeg[B];
    u32 fdeg[B];
    u64 fdd[B];
    unsigned char fsi[B];
    u32 ndefer;
    // step scalars
    u64 minkey_in, minkey_acc;
    u32 count, overflow, dir0, dir1, tile, flag, total, nitems, cert;
    u32 cnt_dir[2];
    u32 group;
    u64 mu0;
#ifdef PPSP_PHASE_CLOCKS
    u64 ph_t, ph_acc[16];  // thread 0's clock at the last mark; cycles per phase
#endif
};

// Opt-in profiling of the one-CTA path (-DPPSP_PHASE_CLOCKS): thread 0 adds
// the SM cycles since its previous mark to phase k; the totals of all CTAs
// are summed in g_phase_clk and read with ppsp_debug_phase_clocks.  Off in
// normal builds (the macros expand to nothing).
#ifdef PPSP_PHASE_CLOCKS
// one copy per translation unit; the 32-bit instances report theirs
static __device__ unsigned long long g_phase_clk[16];
#define PH_START(sm)                                    \
    do {                                                \
        if (threadIdx.x == 0) (sm).ph_t = clock64();    \
    } while (0)
#define PH_MARK(sm, k)                                  \
    do {                                                \
        if (threadIdx.x == 0) {                         \
            const u64 now_ = clock64();                 \
            (sm).ph_acc[k] += now_ - (sm).ph_t;         \
            (sm).ph_t = now_;                           \
        }                                               \
    } while (0)
#else
#define PH_START(sm) \
    do {             \
    } while (0)
#define PH_MARK(sm, k) \
    do {               \
    } while (0)
#endif

template <int B>
__device__ __forceinline__ u32 block_excl_scan(u32 x, Smem<B>& sm, u32* total, bool big = false) {
    const u32 lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    u32 incl = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        u32 y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= (u32)o) incl += y;
    }
    const u32 wbig = __any_sync(0xffffffffu, big) ? 1u : 0u;
    if (lane == 31) {
        sm.wsum[wid] = incl;
        sm.wbig[wid] = wbig;
    }
    __syncthreads();
    if (wid == 0) {
        u32 s = (lane < B / 32) ? sm.wsum[lane] : 0;
        u32 si = s;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            u32 y = __shfl_up_sync(0xffffffffu, si, o);
            if (lane >= (u32)o) si += y;
        }
        if (lane < B / 32) sm.wsum[lane] = si - s;  // exclusive warp offsets
        if (lane == B / 32 - 1) sm.total = si;
        // some entry of the tile has more edges than the owner table handles
        const bool any = __any_sync(0xffffffffu, lane < B / 32 && sm.wbig[lane] != 0);
        if (lane == 0) sm.own_off = any ? 1u : 0u;
    }
    __syncthreads();
    *total = sm.total;
    return sm.wsum[wid] + incl - x;
}

// After the degree scan (before its closing barrier): thread t records itself
// as the owner of its edges excl .. excl + deg - 1 that fall in the table.
template <int B>
__device__ __forceinline__ void write_owner(Smem<B>& sm, u32 t, u32 excl, u32 deg) {
    if (deg > OWN_MAXDEG) return;  // the tile falls back to the binary search
    const u32 end = min(excl + deg, OWN_MULT * (u32)B);
    for (u32 e = excl; e < end; ++e) sm.own[e] = (unsigned short)t;
}

// Entry of edge e of the tile: the owner table, or the largest j with
// pre[j] <= e.
template <int B>
__device__ __forceinline__ u32 edge_owner(const Smem<B>& sm, u32 e, u32 cnt) {
    if (e < OWN_MULT * (u32)B && !sm.own_off) return sm.own[e];
    u32 lo = 0, hi = cnt;
    while (hi - lo > 1) {
        const u32 mid = (lo + hi) >> 1;
        if (sm.pre[mid] <= e) lo = mid; else hi = mid;
    }
    return lo;
}

// CSR rows a search follows: out-edges from a source, in-edges back from a
// target (the same arrays for an undirected graph).
template <int B>
__device__ __forceinline__ const u32* rows(const EngineArgs& a, const Smem<B>& sm, u32 i) {
    return sm.sdir[i] ? a.g.off_t : a.g.off;
}
template <int B>
__device__ __forceinline__ const uint2* adj(const EngineArgs& a, const Smem<B>& sm, u32 i) {
    return sm.sdir[i] ? a.g.edges_t : a.g.edges;
}
// The same rows as 16-byte records carrying P(target) (graphs with
// coordinates, searches with a potential).
template <int B>
__device__ __forceinline__ const int4* adj16(const EngineArgs& a, const Smem<B>& sm, u32 i) {
    return sm.sdir[i] ? a.g.edges_t_pc : a.g.edges_pc;
}

// ----------------------------------------------------------------------------
// per-group context
// ----------------------------------------------------------------------------
template <typename D>
struct GCtx {
    GroupDev G;
    D* dist;
    u32* bm_cur;
    u32* bm_nxt;
    u32* q_nxt;
    StepState* S_nxt;
    SlotDev slot;
    u64 theta;
    bool dense_nxt;
    bool pair;        // two searches, interleaved: both distances of v share 2*W bytes
    u32 n;
    // per-thread counters
    u32 c_x, c_e, c_r, c_p, c_t;  // this group's counts (flushed at its end)
    // one-CTA path: this thread's net change of the per-direction entry
    // counts, added to the shared counts once per tile (flush_dir)
    int dc0, dc1;
    u32* err;         // the device error word (checked builds)
    bool adj16;       // relaxations read 16-byte edge records with P(target)
    // heuristic memoization (Sec. 5): the potential term of each entry,
    // stored as term + 2^31 (0 = not evaluated yet), indexed by vertex for
    // pair groups (the two searches' terms are opposite) and by flat index
    // otherwise; null when off
    u32* memo;
};

// Checked builds (-DPPSP_BOUNDS_CHECK): an index read from memory that falls
// outside its array records ERRB_INTERNAL with the site number in bits 8..15
// of the error word, and the access is skipped; normal builds compile the
// checks out.
#ifdef PPSP_BOUNDS_CHECK
__device__ __forceinline__ bool bad_index(const EngineArgs& a, bool ok, u32 site) {
    if (!ok) atomicOr(a.err, ERRB_INTERNAL | (site << 8));
    return !ok;
}
#else
__device__ __forceinline__ bool bad_index(const EngineArgs&, bool, u32) { return false; }
#endif

__device__ __forceinline__ u32 flat_range_of(const GroupDev& G, u32 n) {
    return G.layout == PPSP_LAYOUT_INTERLEAVED ? (n << G.kshift) : G.scnt * n;
}

__device__ __forceinline__ u32 flat_of(const GroupDev& G, u32 n, u32 v, u32 i) {
    return G.layout == PPSP_LAYOUT_INTERLEAVED ? ((v << G.kshift) | i) : (i * n + v);
}
__device__ __forceinline__ void decode_flat(const GroupDev& G, u32 n, u32 f, u32& v, u32& i) {
    if (G.layout == PPSP_LAYOUT_INTERLEAVED) {
        v = f >> G.kshift;
        i = f & ((1u << G.kshift) - 1u);
    } else {
        i = f / n;
        v = f - i * n;
    }
}

// Potential of <v, i>, in two halves so that its load overlaps the
// distance loads: pot_prefetch issues the load (P(v), or the memoized term),
// pot_resolve evaluates.  With memoization a term is computed from P(v) once
// per group and read back afterwards (Sec. 5: memoize h on first use).
struct PotPre {
    int2 pv;
    u32 mw;
};

// Potential coordinates that came with an edge record (no load).
__device__ __forceinline__ PotPre pot_given(int2 q) {
    PotPre p;
    p.pv = q;
    p.mw = 0;
    return p;
}

template <typename D, int B>
__device__ __forceinline__ PotPre pot_prefetch(const EngineArgs& a, const GCtx<D>& c, const Smem<B>& sm, u32 v,
                                               u32 f) {
    PotPre p;
    p.pv = make_int2(0, 0);
    p.mw = 0;
    if (sm.pot_any) {
        if (c.memo)
            p.mw = __ldcg(c.memo + (c.pair ? v : f));
        else
            p.pv = __ldg(a.g.pc + v);
    }
    return p;
}

template <int B>
__device__ __forceinline__ i64 pot_term(const EngineArgs& a, const GroupDev& G, const Smem<B>& sm, u32 i, int2 pv2);

template <typename D, int B>
__device__ __forceinline__ i64 pot_resolve(const EngineArgs& a, const GCtx<D>& c, const Smem<B>& sm, u32 i, u32 v,
                                           u32 f, const PotPre& p) {
    if (!sm.pot_any) return 0;
    if (!c.memo) return pot_term<B>(a, c.G, sm, i, p.pv);
    const bool neg = c.pair && i;  // a pair stores search 0's term
    i64 r;
    if (p.mw != 0) {
        r = (i64)p.mw - (1ll << 31);
    } else {
        r = pot_term<B>(a, c.G, sm, c.pair ? 0u : i, __ldg(a.g.pc + v));
        c.memo[c.pair ? v : f] = (u32)(r + (1ll << 31));
    }
    return neg ? -r : r;
}

// Both tentative distances of vertex v in a pair group, one 2W-byte load.
__device__ __forceinline__ void ld_pair(const u32* d, u32 v, u64& x0, u64& x1) {
    uint2 p = __ldcg(reinterpret_cast<const uint2*>(d) + v);
    x0 = p.x;
    x1 = p.y;
}
__device__ __forceinline__ void ld_pair(const u64* d, u32 v, u64& x0, u64& x1) {
    ulonglong2 p = __ldcg(reinterpret_cast<const ulonglong2*>(d) + v);
    x0 = p.x;
    x1 = p.y;
}

template <int B>
__device__ __forceinline__ PartnerDev partner(const EngineArgs& a, const Smem<B>& sm, u32 i, u32 p);

// Multi-target potential of search i (Multi-BiDS with A*): the smallest
// h_{q_j}(v) over the partners j of search i.  floor(sqrt(floor(x / 4^F)))
// grows with x, so the minimum is taken over the squared fixed-point
// distances and only one square root is evaluated.
template <int B>
__device__ __forceinline__ i64 pot_min_partner(const EngineArgs& a, const Smem<B>& sm, u32 i, int2 pv2) {
    u64 best = ~0ull;
    const u32 pc = sm.pcnt[i];
    for (u32 p = 0; p < pc; ++p) {
        const int2 q = sm.pa[partner<B>(a, sm, i, p).j];
        const i64 dx = (i64)pv2.x - (i64)q.x, dy = (i64)pv2.y - (i64)q.y;
        const u64 d2 = (u64)(dx * dx) + (u64)(dy * dy);
        best = d2 < best ? d2 : best;
    }
    return pc ? (i64)isqrt_u64(best >> (2 * a.g.pot_shift)) : 0;
}

// Potential part of the key and prune value of <v, i> (Table 2): rho_i(v)
// for BiD-A*, phi_i(v) for multi-target A*, h_t(v) for A*, 0 otherwise;
// pv2 = P(v).
template <int B>
__device__ __forceinline__ i64 pot_term(const EngineArgs& a, const GroupDev& G, const Smem<B>& sm, u32 i, int2 pv2) {
    if (G.mode == GM_BIDIR) {
        const u32 pk = sm.pot[i];
        if (pk == 1) return pot_h(sm.pb[i], pv2, a.g.pot_shift) - pot_h(sm.pa[i], pv2, a.g.pot_shift);
        if (pk == 2) return pot_min_partner<B>(a, sm, i, pv2) - pot_h(sm.pa[i], pv2, a.g.pot_shift);
        return 0;
    }
    if (G.mode == GM_ASTAR) return pot_h(sm.pb[0], pv2, a.g.pot_shift);
    return 0;
}

// key and prune value of <v, i> at tentative distance d, given its potential term
template <int B>
__device__ __forceinline__ void key_of(const GroupDev& G, const Smem<B>& sm, u32 i, i64 term, u64 d, i64& key,
                                       i64& pv) {
    if (G.mode == GM_BIDIR) {
        pv = 2 * (i64)d + term;
        key = pv + sm.key_off[i];
    } else if (G.mode == GM_ASTAR) {
        pv = (i64)d + term;
        key = pv + sm.key_off[0];
    } else {
        pv = (i64)d;
        key = (i64)d;
    }
    if (key < 0) key = 0;
}

__device__ __forceinline__ bool pruned(i64 pv, u64 bound) {
    return bound != INF64 && pv >= 0 && (u64)pv >= bound;
}

template <int B>
__device__ __forceinline__ PartnerDev partner(const EngineArgs& a, const Smem<B>& sm, u32 i, u32 p) {
    return sm.pcached ? sm.pcache[sm.pbeg[i] + p] : a.partners[sm.pbeg[i] + p];
}

// mu[qe] <- min(mu[qe], s); on improvement refresh mumax of both ends (Table 2,
// Multi-PPSP: WriteMin(mumax[i], max_j mu[<q_i, q_j>])).
template <int B>
__device__ __forceinline__ void try_mu(const EngineArgs& a, const GroupDev& G, Smem<B>& sm,
                                       u32 qe, u64 s) {
    if (G.qcnt <= 1 || G.mode != GM_BIDIR) {
        // one query edge: the prune bound of every search is mu itself.  The
        // shared-memory mirror is never below mu (exact for one-CTA teams,
        // refreshed from mu every tile otherwise), so s >= mirror cannot
        // improve mu; otherwise lower the mirror and write mu without
        // waiting for the old value (s is the length of a real s-t path).
        if (s >= sm.bound[0]) return;
        atomicMin(reinterpret_cast<unsigned long long*>(&sm.bound[0]), (unsigned long long)s);
        if (G.scnt == 2) atomicMin(reinterpret_cast<unsigned long long*>(&sm.bound[1]), (unsigned long long)s);
        atomicMin(reinterpret_cast<unsigned long long*>(a.mu + qe), (unsigned long long)s);
        return;
    }
    if (s >= ldcg64(a.mu + qe)) return;
    u64 old = amin64(a.mu + qe, s);
    if (s >= old) return;
    QEdgeDev e = a.qedges[qe];
    u32 ends[2] = {e.a, e.b};
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        u32 x = ends[k];
        u64 m = 0;
        for (u32 p = 0; p < sm.pcnt[x]; ++p) {
            u64 mv = ldcg64(a.mu + partner(a, sm, x, p).qe);
            m = mv > m ? mv : m;
        }
        amin64(a.mumax + G.sbeg + x, m);
        atomicMin(reinterpret_cast<unsigned long long*>(&sm.bound[x]), (unsigned long long)m);
    }
}

// UpdateDistance for <v, i> at distance d (bidirectional family, generic groups)
template <typename D, int B>
__device__ __forceinline__ void update_bidir(const EngineArgs& a, GCtx<D>& c, Smem<B>& sm,
                                             u32 v, u32 i, u64 d) {
    const u32 pc = sm.pcnt[i];
    for (u32 p = 0; p < pc; ++p) {
        PartnerDev pd = partner(a, sm, i, p);
        u64 o = ld_dist(c.dist + flat_of(c.G, c.n, v, pd.j));
        if (o != DT<D>::INF) try_mu(a, c.G, sm, pd.qe, d + o);
    }
}

// F.Add(<v, i>): dedup through the next-step bitmap; new entries are staged
// in shared memory and appended to the global queue once per tile.
template <typename D, int B>
__device__ __forceinline__ void insert(const EngineArgs& a, GCtx<D>& c, Smem<B>& sm, u32 f, u32 i,
                                       i64 key) {
    const u32 bit = 1u << (f & 31u);
    u32 old = atomicOr(c.bm_nxt + (f >> 5), bit);
    if (!(old & bit)) {
        ++c.c_p;
        if (c.G.scnt == 2) atomicAdd(&sm.cnt_dir[i], 1u);
        u32 s = atomicAdd(&sm.qn, 1u);
        if (s < QSTAGE) {
            sm.qbuf[s] = f;
        } else {  // staging full: append directly
            u32 pos = agg_inc(&c.S_nxt->count);
            if (!c.dense_nxt) {
                if (pos < c.slot.qcap)
                    c.q_nxt[pos] = f;
                else
                    c.S_nxt->overflow = 1u;
            }
        }
    }
    atomicMin(reinterpret_cast<unsigned long long*>(&sm.minkey_acc), (unsigned long long)key);
}

template <typename D, int B>
__device__ __forceinline__ void touch(GCtx<D>& c, Smem<B>& sm, u32 f) {
    ++c.c_t;
    u32 s = atomicAdd(&sm.tn, 1u);
    if (s < TSTAGE) {
        sm.tbuf[s] = f;
    } else {
        u32 pos = agg_inc(&c.slot.st->touched_n);
        if (pos < c.slot.tcap)
            c.slot.touched[pos] = f;
        else
            c.slot.st->touched_overflow = 1u;
    }
}

// Write the staged frontier and touched entries of this tile to global memory:
// one atomicAdd per CTA for each list, then coalesced stores.
template <typename D, int B>
__device__ __forceinline__ void flush_stage(GCtx<D>& c, Smem<B>& sm) {
    const u32 t = threadIdx.x;
    __syncthreads();
    const u32 nq = min(sm.qn, (u32)QSTAGE), nt = min(sm.tn, (u32)TSTAGE);
    if (t == 0) {
        sm.qbase = nq ? atomicAdd(&c.S_nxt->count, nq) : 0u;
        sm.tbase = nt ? atomicAdd(&c.slot.st->touched_n, nt) : 0u;
    }
    __syncthreads();
    if (!c.dense_nxt) {
        for (u32 k = t; k < nq; k += B) {
            const u32 pos = sm.qbase + k;
            if (pos < c.slot.qcap)
                c.q_nxt[pos] = sm.qbuf[k];
            else
                c.S_nxt->overflow = 1u;
        }
    }
    for (u32 k = t; k < nt; k += B) {
        const u32 pos = sm.tbase + k;
        if (pos < c.slot.tcap)
            c.slot.touched[pos] = sm.tbuf[k];
        else
            c.slot.st->touched_overflow = 1u;
    }
    __syncthreads();
    if (t == 0) {
        sm.qn = 0;
        sm.tn = 0;
    }
    __syncthreads();
}

// prune, then F.Add for a successful relaxation of <v2, i> to nd
template <typename D, int B>
__device__ __forceinline__ void after_relax(const EngineArgs& a, GCtx<D>& c, Smem<B>& sm, u32 f2,
                                            u32 i, u32 v2, const PotPre& pp, u64 nd) {
    i64 key, pv;
    key_of<B>(c.G, sm, i, pot_resolve<D, B>(a, c, sm, i, v2, f2, pp), nd, key, pv);
    if (pruned(pv, sm.bound[i])) return;
    insert<D, B>(a, c, sm, f2, i, key);
}

template <typename D, int B>
__device__ __forceinline__ void relax(const EngineArgs& a, GCtx<D>& c, Smem<B>& sm, u32 i, u64 d,
                                      uint2 ew, int2 q) {
    const u32 v2 = ew.x;
    const u64 nd = d + (u64)ew.y;
    if (bad_index(a, v2 < c.n, 4)) return;
    // prefetch, overlaps the distance load (or P(v2) came with the edge)
    const PotPre pp = c.adj16 ? pot_given(q)
                              : pot_prefetch<D, B>(a, c, sm, v2, c.pair ? ((v2 << 1) | i) : flat_of(c.G, c.n, v2, i));
    if (nd > DT<D>::MAXV) {
        atomicOr(a.err, ERRB_OVERFLOW);
        return;
    }
    if (c.pair) {
        u64 x0, x1;
        ld_pair(c.dist, v2, x0, x1);
        const u64 own = i ? x1 : x0, oth = i ? x0 : x1;
        if (nd >= own) return;
        const u32 f2 = (v2 << 1) | i;
        const u64 old = amin_dist(c.dist + f2, nd);
        if (nd >= old) return;
        ++c.c_r;
        if (old == DT<D>::INF) touch<D, B>(c, sm, f2);
        if (oth != DT<D>::INF) try_mu(a, c.G, sm, c.G.qbeg, nd + oth);
        after_relax<D, B>(a, c, sm, f2, i, v2, pp, nd);
        return;
    }
    const u32 f2 = flat_of(c.G, c.n, v2, i);
    if (nd >= ld_dist(c.dist + f2)) return;
    const u64 old = amin_dist(c.dist + f2, nd);
    if (nd >= old) return;
    ++c.c_r;
    if (old == DT<D>::INF) touch<D, B>(c, sm, f2);
    if (c.G.mode == GM_BIDIR) {
        update_bidir<D, B>(a, c, sm, v2, i, nd);
    } else if (c.G.mode != GM_SSSP && v2 == c.G.target) {
        try_mu(a, c.G, sm, c.G.qbeg, nd);
    }
    after_relax<D, B>(a, c, sm, f2, i, v2, pp, nd);
}

// Process sm.flat[0 .. cnt): extract, update, prune, then relax all edges of
// the survivors with a load-balanced sweep (consecutive threads read
// consecutive adjacency entries, 8 bytes each: target and weight).
template <typename D, int B>
__device__ void process_items(const EngineArgs& a, GCtx<D>& c, Smem<B>& sm, u32 cnt, bool sparse_src,
                              u32* bm_cur) {
    const u32 t = threadIdx.x;
    // refresh prune bounds for this tile
    if (t < c.G.scnt) {
        u64 b;
        if (c.G.mode == GM_BIDIR)
            b = (c.G.qcnt == 1) ? ldcg64(a.mu + c.G.qbeg) : ldcg64(a.mumax + c.G.sbeg + t);
        else if (c.G.mode == GM_SSSP)
            b = sm.bound[t];  // set from the round's target snapshot
        else
            b = ldcg64(a.mu + c.G.qbeg);
        sm.bound[t] = b;
    }
    __syncthreads();
    u32 deg = 0;
    u32 xf = 0, xv = 0, xi = 0;  // the survivor this thread extracted (pull-then-push)
    u64 xd = DT<D>::INF, xoth = DT<D>::INF;
    bool valid = t < cnt;
    if (valid) {
        u32 v, i;
        decode_flat(c.G, c.n, sm.flat[t], v, i);
        if (!(sm.flat[t] < flat_range_of(c.G, c.n) && v < c.n && i < c.G.scnt)) {
            // an entry of another layout (no search of this group): an
            // internal error, reported instead of reading past the group's
            // descriptors
            atomicOr(a.err, ERRB_INTERNAL | (5u << 8));
            valid = false;
        }
    }
    if (valid) {
        const u32 f = sm.flat[t];
        u32 v, i;
        decode_flat(c.G, c.n, f, v, i);
        // independent loads issued together: offsets, potential coordinates, distances
        const u32* off = rows<B>(a, sm, i);
        const u32 b0 = __ldg(off + v);
        const u32 b1 = __ldg(off + v + 1);
        const PotPre pp = pot_prefetch<D, B>(a, c, sm, v, f);
        if (sparse_src) atomicAnd(bm_cur + (f >> 5), ~(1u << (f & 31u)));
        u64 d, oth = DT<D>::INF;
        if (c.pair) {
            u64 x0, x1;
            ld_pair(c.dist, v, x0, x1);
            d = i ? x1 : x0;
            oth = i ? x0 : x1;
        } else {
            d = ld_dist(c.dist + f);
        }
        if (d != DT<D>::INF) {
            i64 key, pv;
            key_of<B>(c.G, sm, i, pot_resolve<D, B>(a, c, sm, i, v, f, pp), d, key, pv);
            if ((u64)key > c.theta) {
                insert<D, B>(a, c, sm, f, i, key);  // stays in F
            } else {
                if (c.pair) {
                    if (oth != DT<D>::INF) try_mu(a, c.G, sm, c.G.qbeg, d + oth);
                } else if (c.G.mode == GM_BIDIR) {
                    update_bidir<D, B>(a, c, sm, v, i, d);
                }
                if (!pruned(pv, sm.bound[i])) {
                    deg = b1 - b0;
                    sm.beg[t] = b0;
                    sm.si[t] = (unsigned char)i;
                    sm.d[t] = d;
                    ++c.c_x;
                    xf = f;
                    xv = v;
                    xi = i;
                    xd = d;
                    xoth = oth;
                }
            }
        }
    }
    u32 total;
    u32 excl = block_excl_scan<B>(deg, sm, &total, deg > OWN_MAXDEG);
    sm.pre[t] = (t < cnt) ? excl : total;
    if (deg) write_owner<B>(sm, t, excl, deg);
    __syncthreads();
    if (a.pull && a.g.off == a.g.off_t) {
        // App. B, bidirectional relaxation: before pushing from u, pull
        // d(u) <- min(d(u), d(x) + w(x, u)) over its neighbours x (the same
        // adjacency on an undirected graph); every candidate is the length of
        // a real path, so d stays an upper bound
        for (u32 e = t; e < total; e += B) {
            const u32 lo = edge_owner<B>(sm, e, cnt);
            const u32 si = sm.si[lo];
            const uint2 ew = __ldg(adj<B>(a, sm, si) + sm.beg[lo] + (e - sm.pre[lo]));
            ++c.c_e;
            const u64 dx = ld_dist(c.dist + flat_of(c.G, c.n, ew.x, si));
            if (dx != DT<D>::INF && dx + ew.y < sm.d[lo])
                atomicMin(reinterpret_cast<unsigned long long*>(&sm.d[lo]), (unsigned long long)(dx + ew.y));
        }
        __syncthreads();
        if (deg && sm.d[t] < xd) {
            const u64 nd = sm.d[t];  // <= xd <= the largest representable distance
            amin_dist(c.dist + xf, nd);
            ++c.c_r;
            if (c.pair) {
                if (xoth != DT<D>::INF) try_mu(a, c.G, sm, c.G.qbeg, nd + xoth);
            } else if (c.G.mode == GM_BIDIR) {
                update_bidir<D, B>(a, c, sm, xv, xi, nd);
            } else if (c.G.mode != GM_SSSP && xv == c.G.target) {
                try_mu(a, c.G, sm, c.G.qbeg, nd);
            }
        }
    }
    for (u32 e = t; e < total; e += B) {
        const u32 lo = edge_owner<B>(sm, e, cnt);
        const u32 edge = sm.beg[lo] + (e - sm.pre[lo]);
        if (bad_index(a, lo < cnt && edge < a.g.m, 7)) continue;
        uint2 ew;
        int2 q = make_int2(0, 0);
        if (c.adj16) {
            const int4 r = __ldg(adj16<B>(a, sm, sm.si[lo]) + edge);
            ew = make_uint2((u32)r.x, (u32)r.y);
            q = make_int2(r.z, r.w);
        } else {
            ew = __ldg(adj<B>(a, sm, sm.si[lo]) + edge);
        }
        ++c.c_e;
        relax<D, B>(a, c, sm, sm.si[lo], sm.d[lo], ew, q);
    }
    flush_stage<D, B>(c, sm);
}

// ----------------------------------------------------------------------------
// one-CTA teams: bucketed frontier in shared memory
// ----------------------------------------------------------------------------
// Delta*-stepping with buckets.  An entry <v, i> is stored with the distance it
// was inserted with, in the bucket of the step whose threshold first covers its
// key: bucket b = ceil(key / step), i.e. it is extracted at theta = b * step
// (keys at or below the current threshold go to the next step).  Waiting
// entries are therefore never re-read.  A later, smaller distance inserts a new
// entry; the old one is recognised as stale at extraction (the stored distance
// no longer matches) and dropped.  The ring holds the next LR_NB - 1 steps in
// shared memory; entries further ahead go to a far list in the slot (re-bucketed
// when the ring's window reaches them); an entry that finds its bucket or the
// far list full sets its bit in the slot's spill bitmap and is recovered from
// its current distance when nothing else is left.
// Shared-memory entries per bucket: chosen per plan (a small ring leaves more
// of the SM's L1 to the adjacency and offsets; a large one keeps big buckets
// out of the global overflow region), at most RING_CAP_MAX.
constexpr u32 RING_CAP_MAX = 256;
template <typename D>
struct LR {
    static constexpr u32 NB = LR_NB;  // buckets in the ring
    static constexpr size_t bytes(u32 cap) { return (size_t)NB * cap * (4 + sizeof(D)) + NB * 4; }
};

template <typename D, int B>
struct LocalView {
    u32* rf;  // [NB * cap] flat index
    D* rd;    // [NB * cap] distance at insertion
    u32* rn;  // [NB] entries per bucket
    u32 cap;  // shared-memory entries per bucket
};

template <typename D, int B>
__device__ __forceinline__ LocalView<D, B> local_view(Smem<B>& sm, u32 cap) {
    unsigned char* p = reinterpret_cast<unsigned char*>(&sm) + ((sizeof(Smem<B>) + 15) & ~(size_t)15);
    LocalView<D, B> L;
    L.rd = reinterpret_cast<D*>(p);
    L.rf = reinterpret_cast<u32*>(p + (size_t)LR<D>::NB * cap * sizeof(D));
    L.rn = L.rf + LR<D>::NB * cap;
    L.cap = cap;
    return L;
}

template <typename D, int B>
__device__ __forceinline__ void insert_local(GCtx<D>& c, Smem<B>& sm, const LocalView<D, B>& L, u32 f, u32 i,
                                             i64 key, u64 d) {
#ifdef PPSP_BOUNDS_CHECK
    if (f >= flat_range_of(c.G, c.n)) {
        atomicOr(c.err, ERRB_INTERNAL | (9u << 8));
        return;
    }
#endif
    const u64 step = sm.lstep;
    // b = ceil(key / step), in 32 bits when both fit (the common case)
    u64 b;
    if ((((u64)key | step) >> 32) == 0)
        b = key == 0 ? 0 : (u64)(((u32)key - 1u) / (u32)step + 1u);
    else
        b = ((u64)key + step - 1) / step;
    const u64 cur = sm.lcur;
    if (b <= cur) {
        // already under the threshold: due at the next step; remember the key
        // (the bucket's lower bound (b - 1) * step does not hold for it)
        b = cur + 1;
        atomicMin(reinterpret_cast<unsigned long long*>(&sm.llate), (unsigned long long)key);
    }
    bool stored = false;
    // ring slots of the buckets of this step are not reused until it ends
    if (b < sm.lfirst + LR<D>::NB) {
        const u32 s = (u32)(b % LR<D>::NB);
        // one shared-memory atomic per bucket per warp
        cg::coalesced_group peers = cg::labeled_partition(cg::coalesced_threads(), (int)s);
        u32 pos = 0;
        if (peers.thread_rank() == 0) pos = atomicAdd(&L.rn[s], (u32)peers.size());
        pos = peers.shfl(pos, 0) + peers.thread_rank();
        if (pos < L.cap) {
            L.rf[s * L.cap + pos] = f;
            L.rd[s * L.cap + pos] = (D)d;
            stored = true;
        } else {
            // the bucket continues in its global overflow region
            const u32 ob = c.slot.ocap / LR<D>::NB, p2 = pos - L.cap;
            if (p2 < ob) {
                c.slot.of[s * ob + p2] = f;
                reinterpret_cast<D*>(c.slot.od)[s * ob + p2] = (D)d;
                stored = true;
            }
        }
    } else {
        const u32 fb = sm.lfar_tgt;
        const u32 pos = agg_inc(&sm.lfar_n[fb]);
        if (pos < c.slot.qcap) {
            c.slot.q[fb][pos] = f;
            reinterpret_cast<D*>(c.slot.fd[fb])[pos] = (D)d;
            atomicMin(reinterpret_cast<unsigned long long*>(&sm.lfar_min[fb]), (unsigned long long)b);
            stored = true;
        }
    }
    if (!stored) {
        const u32 bit = 1u << (f & 31u);
        if (atomicOr(c.slot.bm[0] + (f >> 5), bit) & bit) return;  // already spilled
        sm.lspill = 1;
    }
    ++c.c_p;
    if (i) ++c.dc1; else ++c.dc0;
}

// Add the warp's net per-direction entry counts to the shared counts (all
// threads of the CTA call this, converged, before a barrier).
template <typename D, int B>
__device__ __forceinline__ void flush_dir(GCtx<D>& c, Smem<B>& sm) {
    if (c.G.scnt == 2) {
        const u32 s0 = __reduce_add_sync(0xffffffffu, (u32)c.dc0);
        const u32 s1 = __reduce_add_sync(0xffffffffu, (u32)c.dc1);
        if ((threadIdx.x & 31) == 0) {
            if (s0) atomicAdd(&sm.cnt_dir[0], s0);
            if (s1) atomicAdd(&sm.cnt_dir[1], s1);
        }
    }
    c.dc0 = c.dc1 = 0;
}

template <typename D, int B>
__device__ __forceinline__ void touch_local(GCtx<D>& c, Smem<B>& sm, u32 f) {
    ++c.c_t;
    const u32 pos = agg_inc(&sm.tn);
    if (pos < c.slot.tcap)
        c.slot.touched[pos] = f;
    else
        sm.tov = 1;
}

template <typename D, int B>
__device__ __forceinline__ void relax_local(const EngineArgs& a, GCtx<D>& c, Smem<B>& sm, const LocalView<D, B>& L,
                                            u32 i, u64 d, uint2 ew, int2 q) {
    const u32 v2 = ew.x;
    const u64 nd = d + (u64)ew.y;
    if (bad_index(a, v2 < c.n, 4)) return;
    const u32 f2 = c.pair ? ((v2 << 1) | i) : flat_of(c.G, c.n, v2, i);
    const PotPre pp = c.adj16 ? pot_given(q) : pot_prefetch<D, B>(a, c, sm, v2, f2);
    if (nd > DT<D>::MAXV) {
        atomicOr(a.err, ERRB_OVERFLOW);
        return;
    }
    if (c.pair) {
        u64 x0, x1;
        ld_pair(c.dist, v2, x0, x1);
        const u64 own = i ? x1 : x0, oth = i ? x0 : x1;
        if (nd >= own) return;
        const u64 old = amin_dist(c.dist + f2, nd);
        if (nd >= old) return;
        ++c.c_r;
        if (old == DT<D>::INF) touch_local<D, B>(c, sm, f2);
        if (oth != DT<D>::INF) try_mu(a, c.G, sm, c.G.qbeg, nd + oth);
    } else {
        if (nd >= ld_dist(c.dist + f2)) return;
        const u64 old = amin_dist(c.dist + f2, nd);
        if (nd >= old) return;
        ++c.c_r;
        if (old == DT<D>::INF) touch_local<D, B>(c, sm, f2);
        if (c.G.mode == GM_BIDIR)
            update_bidir<D, B>(a, c, sm, v2, i, nd);
        else if (c.G.mode != GM_SSSP && v2 == c.G.target)
            try_mu(a, c.G, sm, c.G.qbeg, nd);
    }
    i64 key, pv;
    key_of<B>(c.G, sm, i, pot_resolve<D, B>(a, c, sm, i, v2, f2, pp), nd, key, pv);
    if (pruned(pv, sm.bound[i])) return;
    insert_local<D, B>(c, sm, L, f2, i, key, nd);
}

// SSSP-based groups (Sec. 4.3): the largest tentative distance of the
// group's targets, or INF while one of them is unreached.  Called by one full
// warp.  Every entry that remains with a key at least this large cannot lower
// any target, so it is both the prune bound and the stop certificate of the
// search (the multi-target form of ET, Sec. 3.2).
template <typename D, int B>
__device__ __forceinline__ u64 sssp_target_max(const EngineArgs& a, const GCtx<D>& c, const Smem<B>& sm) {
    const u32 lane = threadIdx.x & 31u;
    u64 m = 0;
    bool all = true;
    for (u32 q = lane; q < c.G.qcnt; q += 32) {
        const u32 tv = sm.pcached ? sm.pcache[q].j : a.qedges[c.G.qbeg + q].b;
        const u64 d = ld_dist(c.dist + flat_of(c.G, c.n, tv, 0));
        all = all && d != DT<D>::INF;
        m = d > m ? d : m;
    }
    all = __all_sync(0xffffffffu, all);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const u64 y = __shfl_xor_sync(0xffffffffu, m, o);
        m = y > m ? y : m;
    }
    return (all && c.G.qcnt > 0) ? m : INF64;
}

// Entries of a bucket step are spread over the warps: thread (warp w, lane l)
// takes entry l * (B / 32) + w, so that a step of few entries gives every warp
// a share and each warp can expand its own entries' edges.  (Packing the
// entries into fewer warps, about 16 per warp, was measured 3-6% slower on
// the 2048^2 road batch: each busy warp's extraction and expansion take
// longer.)
template <int B>
__device__ __forceinline__ u32 spread_index(u32 t) {
    return (t & 31u) * (u32)(B / 32) + (t >> 5);
}

// A warp expands its own entries' edges while no warp holds more than this
// many; otherwise the CTA shares the edges (degree scan and owner table).
constexpr u32 WARP_EDGES_MAX = 256;

// One relaxation of a pair group without waiting for the old distance: the
// pair just read decides success (a concurrent smaller write only leaves a
// stale entry behind, which extraction drops).  In parts, so that a lane
// can issue the loads of two edges before it waits for either and a warp can
// pack its successes: pair_issue loads both distances of v2 (and its
// potential unless the edge record carried it), pair_try tests and writes
// the distance, pair_success does the rest.
template <typename D>
struct PairLd {
    u64 x0, x1;
    PotPre pp;
};

template <typename D, int B>
__device__ __forceinline__ PairLd<D> pair_issue(const EngineArgs& a, const GCtx<D>& c, const Smem<B>& sm, u32 v2,
                                                int2 q) {
    PairLd<D> r;
    // pair: the term is indexed by vertex; with 16-byte records P(v2) came with the edge
    r.pp = c.adj16 ? pot_given(q) : pot_prefetch<D, B>(a, c, sm, v2, 0);
    ld_pair(c.dist, v2, r.x0, r.x1);
    return r;
}

// The cheap half of a pair relaxation: overflow check, the success test
// against the distance just read, and the WriteMin (not waited for).  On
// success returns true with the flat index, the other search's distance and
// whether the entry left infinity.
template <typename D, int B>
__device__ __forceinline__ bool pair_try(const EngineArgs& a, GCtx<D>& c, u32 i, u32 v2, u64 nd, const PairLd<D>& r,
                                         u32& f2, u64& oth, bool& fresh) {
    if (nd > DT<D>::MAXV) {
        atomicOr(a.err, ERRB_OVERFLOW);
        return false;
    }
    const u64 own = i ? r.x1 : r.x0;
    if (nd >= own) return false;
    oth = i ? r.x0 : r.x1;
    f2 = (v2 << 1) | i;
    fresh = own == DT<D>::INF;
    amin_dist(c.dist + f2, nd);
    return true;
}

// The rest of a successful pair relaxation: touched list, mu, key, prune,
// insertion.
template <typename D, int B>
__device__ __forceinline__ void pair_success(const EngineArgs& a, GCtx<D>& c, Smem<B>& sm, const LocalView<D, B>& L,
                                             u32 f2, u64 nd, u64 oth, bool fresh, const PotPre& pp) {
    const u32 i = f2 & 1u, v2 = f2 >> 1;
    ++c.c_r;
    if (fresh) touch_local<D, B>(c, sm, f2);
    if (oth != DT<D>::INF) try_mu(a, c.G, sm, c.G.qbeg, nd + oth);
    i64 key, pv;
    key_of<B>(c.G, sm, i, pot_resolve<D, B>(a, c, sm, i, v2, f2, pp), nd, key, pv);
    if (pruned(pv, sm.bound[i])) return;
    insert_local<D, B>(c, sm, L, f2, i, key, nd);
}

// Position of the k-th (from 0) set bit of m, for k < popc(m).
__device__ __forceinline__ u32 nth_set_bit(u32 m, u32 k) {
    u32 pos = 0;
#pragma unroll
    for (u32 step = 16; step > 0; step >>= 1)
        if ((u32)__popc(m & ((1u << (pos + step)) - 1u)) <= k) pos += step;
    return pos;
}

__device__ __forceinline__ u64 shfl_u64(u64 x, u32 src) {
    const u32 lo = __shfl_sync(0xffffffffu, (u32)x, src), hi = __shfl_sync(0xffffffffu, (u32)(x >> 32), src);
    return ((u64)hi << 32) | lo;
}

// Owner of edge j of a warp's expansion (the first lane whose inclusive
// degree prefix exceeds j) and that edge: its adjacency index, search and the
// owner's distance.  Called by the full warp; valid only for j < wtot.
struct WarpEdge {
    u32 edge, si;
    u64 d;
};

__device__ __forceinline__ WarpEdge warp_edge(u32 j, u32 incl, u32 xb0, u32 xex, u32 xsi, u64 xd) {
    u32 o = 0;
#pragma unroll
    for (int step = 16; step > 0; step >>= 1) {
        const u32 x = __shfl_sync(0xffffffffu, incl, o + step - 1);
        if (x <= j) o += step;
    }
    WarpEdge w;
    w.edge = __shfl_sync(0xffffffffu, xb0, o) + (j - __shfl_sync(0xffffffffu, xex, o));
    w.si = __shfl_sync(0xffffffffu, xsi, o);
    const u32 dl = __shfl_sync(0xffffffffu, (u32)xd, o);
    const u32 dh = __shfl_sync(0xffffffffu, (u32)(xd >> 32), o);
    w.d = ((u64)dh << 32) | dl;
    return w;
}

// Relax up to two edges of this thread (edge index and search, the owner's
// distance): both adjacency loads, then for pair groups both distance loads,
// are issued before the first update waits on memory.  Called by full warps
// (a warp-uniform number of times): pair groups pack the warp's successful
// relaxations with ballots and shuffles.
template <typename D, int B>
__device__ __forceinline__ void relax_two(const EngineArgs& a, GCtx<D>& c, Smem<B>& sm, const LocalView<D, B>& L,
                                          bool va, u32 sa, u32 ga, u64 da, bool vb, u32 sb, u32 gb, u64 db) {
    uint2 ea = make_uint2(0, 0), eb = make_uint2(0, 0);
    int2 qa = make_int2(0, 0), qb = make_int2(0, 0);
    if (c.adj16) {
        if (va) {
            const int4 r = __ldg(adj16<B>(a, sm, sa) + ga);
            ea = make_uint2((u32)r.x, (u32)r.y);
            qa = make_int2(r.z, r.w);
        }
        if (vb) {
            const int4 r = __ldg(adj16<B>(a, sm, sb) + gb);
            eb = make_uint2((u32)r.x, (u32)r.y);
            qb = make_int2(r.z, r.w);
        }
    } else {
        if (va) ea = __ldg(adj<B>(a, sm, sa) + ga);
        if (vb) eb = __ldg(adj<B>(a, sm, sb) + gb);
    }
    c.c_e += (va ? 1u : 0u) + (vb ? 1u : 0u);
    if (c.pair) {
        const bool pa = va && !bad_index(a, ea.x < c.n, 4);
        const bool pb = vb && !bad_index(a, eb.x < c.n, 4);
        PairLd<D> ra{}, rb{};
        if (pa) ra = pair_issue<D, B>(a, c, sm, ea.x, qa);
        if (pb) rb = pair_issue<D, B>(a, c, sm, eb.x, qb);
        // the success tests and WriteMins of both edges, then the warp's
        // successes (about 40% of its edges) packed into as few passes of
        // the heavier rest as they fill: one pass instead of one per edge
        u32 fa = 0, fb = 0;
        u64 nda = da + (u64)ea.y, ndb = db + (u64)eb.y, otha = 0, othb = 0;
        bool fra = false, frb = false;
        const bool oka = pa && pair_try<D, B>(a, c, sa, ea.x, nda, ra, fa, otha, fra);
        const bool okb = pb && pair_try<D, B>(a, c, sb, eb.x, ndb, rb, fb, othb, frb);
        const u32 lane = threadIdx.x & 31u;
        const u32 ma = __ballot_sync(0xffffffffu, oka), mb = __ballot_sync(0xffffffffu, okb);
        const u32 na = __popc(ma), ntot = na + __popc(mb);
        for (u32 k0 = 0; k0 < ntot; k0 += 32) {
            const u32 k = k0 + lane;
            const bool has = k < ntot, from_a = k < na;
            const u32 src = has ? (from_a ? nth_set_bit(ma, k) : nth_set_bit(mb, k - na)) : 0u;
            const u32 f_a = __shfl_sync(0xffffffffu, fa, src), f_b = __shfl_sync(0xffffffffu, fb, src);
            const u64 nd_a = shfl_u64(nda, src), nd_b = shfl_u64(ndb, src);
            const u64 ot_a = shfl_u64(otha, src), ot_b = shfl_u64(othb, src);
            const u32 fl = __shfl_sync(0xffffffffu, (fra ? 1u : 0u) | (frb ? 2u : 0u), src);
            PotPre pp;
            const int px_a = __shfl_sync(0xffffffffu, ra.pp.pv.x, src), px_b = __shfl_sync(0xffffffffu, rb.pp.pv.x, src);
            const int py_a = __shfl_sync(0xffffffffu, ra.pp.pv.y, src), py_b = __shfl_sync(0xffffffffu, rb.pp.pv.y, src);
            const u32 mw_a = __shfl_sync(0xffffffffu, ra.pp.mw, src), mw_b = __shfl_sync(0xffffffffu, rb.pp.mw, src);
            pp.pv = from_a ? make_int2(px_a, py_a) : make_int2(px_b, py_b);
            pp.mw = from_a ? mw_a : mw_b;
            if (has)
                pair_success<D, B>(a, c, sm, L, from_a ? f_a : f_b, from_a ? nd_a : nd_b, from_a ? ot_a : ot_b,
                                   (fl & (from_a ? 1u : 2u)) != 0, pp);
        }
    } else {
        if (va) relax_local<D, B>(a, c, sm, L, sa, da, ea, qa);
        if (vb) relax_local<D, B>(a, c, sm, L, sb, db, eb, qb);
    }
}

// mode 0: entries of the current bucket (extract), spread over the warps
// (spread_index); mode 1: far-list or spill entries in threads 0 .. cnt - 1
// (re-bucket, nothing is expanded).  sm.flat / sm.d hold each thread's entry.
template <typename D, int B>
__device__ void process_local(const EngineArgs& a, GCtx<D>& c, Smem<B>& sm, const LocalView<D, B>& L, u32 cnt,
                              int mode) {
    const u32 t = threadIdx.x;
    u32 deg = 0;
    u32 xb0 = 0, xsi = 0;  // the survivor's first edge and search
    u64 xd = 0;            // and its distance
    if ((mode == 0 ? spread_index<B>(t) : t) < cnt) {
        const u32 f = sm.flat[t];
        const u64 dins = sm.d[t];  // stored distance (INF: recover from the current one)
        u32 v, i;
        decode_flat(c.G, c.n, f, v, i);
        // an entry of another layout (no search of this group): an internal
        // error, reported instead of reading past the group's descriptors
        const bool bad = !(f < flat_range_of(c.G, c.n) && v < c.n && i < c.G.scnt);
        if (bad) {
            atomicOr(a.err, ERRB_INTERNAL | (2u << 8));
            v = 0;
            i = 0;
        }
        const u32* off = rows<B>(a, sm, i);
        const u32 b0 = __ldg(off + v);
        const u32 b1 = (mode == 0) ? __ldg(off + v + 1) : b0;
        const PotPre pp = pot_prefetch<D, B>(a, c, sm, v, f);
        u64 d, oth = DT<D>::INF;
        if (c.pair) {
            u64 x0, x1;
            ld_pair(c.dist, v, x0, x1);
            d = i ? x1 : x0;
            oth = i ? x0 : x1;
        } else {
            d = ld_dist(c.dist + f);
        }
        if (i) --c.dc1; else --c.dc0;  // the stored entry is consumed
        if (!bad && d != DT<D>::INF && (dins == DT<D>::INF || d == dins)) {
            i64 key, pv;
            key_of<B>(c.G, sm, i, pot_resolve<D, B>(a, c, sm, i, v, f, pp), d, key, pv);
            if (mode == 1) {
                insert_local<D, B>(c, sm, L, f, i, key, d);  // into the ring window or back to far
            } else {
                if (c.pair) {
                    if (oth != DT<D>::INF) try_mu(a, c.G, sm, c.G.qbeg, d + oth);
                } else if (c.G.mode == GM_BIDIR) {
                    update_bidir<D, B>(a, c, sm, v, i, d);
                }
                if (!pruned(pv, sm.bound[i])) {
                    deg = b1 - b0;
                    xb0 = b0;
                    xsi = i;
                    xd = d;
                    ++c.c_x;
                }
            }
        }
    }
    if (mode == 1) {
        flush_dir<D, B>(c, sm);
        __syncthreads();
        return;
    }
    PH_MARK(sm, 1);  // staging + extraction of thread 0's entry
    // each warp's edges: prefix sums of its lanes' degrees
    const u32 lane = t & 31u;
    u32 incl = deg;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const u32 y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= (u32)o) incl += y;
    }
    const u32 wtot = __shfl_sync(0xffffffffu, incl, 31);
    const bool many = wtot > WARP_EDGES_MAX;
    if (!many) {
        // the warp expands its own entries' edges, two per lane in flight:
        // both edge loads, then both distance loads, before the first
        // update waits on memory
        const u32 xex = incl - deg;
        for (u32 j0 = 0; j0 < wtot; j0 += 64) {
            const u32 ja = j0 + lane, jb = j0 + 32 + lane;
            const WarpEdge wa = warp_edge(ja, incl, xb0, xex, xsi, xd);
            const WarpEdge wb = warp_edge(jb, incl, xb0, xex, xsi, xd);
            const bool va = ja < wtot && !bad_index(a, wa.edge < a.g.m && wa.si < c.G.scnt, 3);
            const bool vb = jb < wtot && !bad_index(a, wb.edge < a.g.m && wb.si < c.G.scnt, 3);
            relax_two<D, B>(a, c, sm, L, va, wa.si, wa.edge, wa.d, vb, wb.si, wb.edge, wb.d);
        }
    } else if (deg) {
        // a warp with many edges (high-degree vertices) hands its entries to
        // the whole CTA, after the step's closing barrier
        const u32 k = atomicAdd(&sm.ndefer, 1u);  // < B: one entry per thread
        sm.fbeg[k] = xb0;
        sm.fsi[k] = (unsigned char)xsi;
        sm.fdd[k] = xd;
        sm.fdeg[k] = deg;
    }
    PH_MARK(sm, 3);  // thread 0's relaxations
    flush_dir<D, B>(c, sm);
    if (!__syncthreads_or(many)) {
        PH_MARK(sm, 4);  // wait for the slowest relaxation
        return;
    }
    // the deferred entries (threads 0 .. nd - 1): degree scan, owner table,
    // then the CTA relaxes their edges together
    const u32 nd = sm.ndefer;
    const u32 fdeg = t < nd ? sm.fdeg[t] : 0u;
    u32 total;
    const u32 excl = block_excl_scan<B>(fdeg, sm, &total, fdeg > OWN_MAXDEG);
    sm.pre[t] = excl;  // threads past the deferred entries hold the total
    if (fdeg) write_owner<B>(sm, t, excl, fdeg);
    if (t == 0) sm.ndefer = 0;  // every thread read it before the scan's barriers
    __syncthreads();
    // warp-uniform trip count: relax_two packs a warp's successes with shuffles
    for (u32 w0 = t & ~31u; w0 < total; w0 += 2 * B) {
        const u32 ea = w0 + (t & 31u), eb = ea + B;
        u32 la = 0, lb = 0, ga = 0, gb = 0;
        bool va = ea < total, vb = eb < total;
        if (va) {
            la = edge_owner<B>(sm, ea, nd);
            ga = sm.fbeg[la] + (ea - sm.pre[la]);
            va = !bad_index(a, la < nd && ga < a.g.m && sm.fsi[la] < c.G.scnt, 6);
        }
        if (vb) {
            lb = edge_owner<B>(sm, eb, nd);
            gb = sm.fbeg[lb] + (eb - sm.pre[lb]);
            vb = !bad_index(a, lb < nd && gb < a.g.m && sm.fsi[lb] < c.G.scnt, 6);
        }
        relax_two<D, B>(a, c, sm, L, va, va ? sm.fsi[la] : 0u, ga, va ? sm.fdd[la] : 0ull, vb,
                        vb ? sm.fsi[lb] : 0u, gb, vb ? sm.fdd[lb] : 0ull);
    }
    flush_dir<D, B>(c, sm);
    __syncthreads();
    PH_MARK(sm, 4);  // wait for the slowest relaxation
}

// Re-bucket every entry of the far list `fb` (relative to the current bucket);
// survivors beyond the ring window go to the other far list.
template <typename D, int B>
__device__ void redistribute_far(const EngineArgs& a, GCtx<D>& c, Smem<B>& sm, const LocalView<D, B>& L) {
    const u32 t = threadIdx.x;
    const u32 fb = sm.lfar_fb, nb = fb ^ 1u;
    const u32 n = min(sm.lfar_n[fb], c.slot.qcap);
    if (t == 0) {
        sm.lfar_tgt = nb;
        sm.lfar_n[nb] = 0;
        sm.lfar_min[nb] = INF64;
    }
    __syncthreads();
    for (u32 base = 0; base < n; base += B) {
        const u32 cnt = min((u32)B, n - base);
        if (t < cnt) {
            sm.flat[t] = __ldcg(c.slot.q[fb] + base + t);
            sm.d[t] = (u64)__ldcg(reinterpret_cast<const D*>(c.slot.fd[fb]) + base + t);
        }
        __syncthreads();
        process_local<D, B>(a, c, sm, L, cnt, 1);
    }
    if (t == 0) {
        sm.lfar_fb = nb;
        sm.lfar_n[fb] = 0;
        sm.lfar_min[fb] = INF64;
        sm.lfar_after = sm.lfar_n[nb];
    }
    __syncthreads();
}

// Recover spilled entries (their bits in the slot's spill bitmap) from their
// current distances.
template <typename D, int B>
__device__ void recover_spill(const EngineArgs& a, GCtx<D>& c, Smem<B>& sm, const LocalView<D, B>& L,
                              u32 nwords) {
    const u32 t = threadIdx.x;
    if (t == 0) sm.lspill = 0;
    __syncthreads();
    for (u32 wb = 0; wb < nwords; wb += B) {
        const u32 w = wb + t;
        u32 bits = 0;
        if (w < nwords) {
            bits = __ldcg(c.slot.bm[0] + w);
            if (bits) c.slot.bm[0][w] = 0u;
        }
        u32 total;
        u32 idx = block_excl_scan<B>(__popc(bits), sm, &total);
        for (u32 base = 0; base < total; base += B) {
            while (bits && idx < base + B) {
                const u32 bb = __ffs(bits) - 1;
                bits &= bits - 1;
                sm.flat[idx - base] = (w << 5) | bb;
                sm.d[idx - base] = DT<D>::INF;
                ++idx;
            }
            __syncthreads();
            process_local<D, B>(a, c, sm, L, min((u32)B, total - base), 1);
        }
    }
}

// The stepping loop of one group on one CTA.  Returns the number of steps.
template <typename D, int B>
__device__ u64 run_local(const EngineArgs& a, GCtx<D>& c, Smem<B>& sm, u32 nwords) {
    const u32 t = threadIdx.x;
    const LocalView<D, B> L = local_view<D, B>(sm, a.ring_cap);
    const GroupDev& G = c.G;
    for (u32 k = t; k < LR<D>::NB; k += B) L.rn[k] = 0;
    if (t == 0) {
        sm.lstep = (G.mode == GM_BIDIR) ? 2 * G.delta : G.delta;
        sm.lcur = 0;
        sm.lfirst = 0;
        sm.lfar_fb = 0;
        sm.lfar_tgt = 0;
        sm.lfar_n[0] = sm.lfar_n[1] = 0;
        sm.lfar_min[0] = sm.lfar_min[1] = INF64;
        sm.lspill = 0;
        sm.llate = INF64;
        sm.lrecov = 0;
        sm.lidle = 0;
        sm.lfar_after = 0;
        sm.ndefer = 0;
        sm.cnt_dir[0] = sm.cnt_dir[1] = 0;
    }
    __syncthreads();
    // Init: the sources (key 0) go to the first step
    c.dc0 = c.dc1 = 0;
    if (t < G.scnt) insert_local<D, B>(c, sm, L, flat_of(G, c.n, sm.src[t], t), t, 0, 0);
    flush_dir<D, B>(c, sm);
#ifdef PPSP_PHASE_CLOCKS
    if (t < 16) sm.ph_acc[t] = 0;
#endif
    __syncthreads();
    PH_START(sm);
    u64 rounds = 0;
    for (;;) {
        // choose the next bucket (warp 0 finds the first non-empty bucket of
        // the ring, thread 0 decides), moving far entries into the window when
        // they are due soon or the ring is empty
        u64 rb = INF64;
        if (G.mode == GM_SSSP && t >= 32 && t < 64) {
            const u64 m = sssp_target_max<D, B>(a, c, sm);
            if (t == 32 && m < sm.bound[0]) sm.bound[0] = m;  // only thread 32 writes it here
        }
        if (t < 32) {
            const u64 cur = sm.lcur;
            const u32 ob = c.slot.ocap / LR<D>::NB;
            u32 cnt = 0;
            if (t >= 1 && t < LR<D>::NB) cnt = min(L.rn[(u32)((cur + t) % LR<D>::NB)], L.cap + ob);
            const u32 mask = __ballot_sync(0xffffffffu, cnt != 0);
            if (mask) rb = cur + (u32)(__ffs(mask) - 1);
            u32 incl = cnt;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const u32 y = __shfl_up_sync(0xffffffffu, incl, o);
                if (t >= (u32)o) incl += y;
            }
            sm.lpre[t] = incl;  // entries in buckets cur + 1 .. cur + t
            __syncwarp();
        }
        if (t == 0) {
            sm.flag = 0;  // 0 = process lcur, 1 = redistribute, 2 = recover, 3 = done
            const u64 cur = sm.lcur;
            const u32 fb = sm.lfar_fb;
            const u64 fm = sm.lfar_n[fb] ? sm.lfar_min[fb] : INF64;
            bool stop = false;
            if (G.scnt == 2 && G.mode == GM_BIDIR && sm.bound[0] == INF64 &&
                (sm.cnt_dir[0] == 0 || sm.cnt_dir[1] == 0))
                stop = true;  // App. B: one side ran dry before mu was set
            // mu certificate: every stored entry has key > (next bucket - 1) * step,
            // and a prune value >= its key; once that reaches the largest prune
            // bound of the group, every remaining entry would be pruned.
            const u64 nextb = rb < fm ? rb : fm;
            if (!stop && !sm.lspill && nextb != INF64) {
                u64 bmax = 0;
                for (u32 i = 0; i < G.scnt; ++i) bmax = sm.bound[i] > bmax ? sm.bound[i] : bmax;
                u64 lb = (nextb - 1) * sm.lstep + 1;  // keys in buckets >= nextb
                if (nextb == cur + 1 && sm.llate < lb) lb = sm.llate;
                if (bmax != INF64 && bmax > 0 && lb >= bmax) stop = true;
            }
            if (stop) {
                sm.flag = 3;
            } else if (sm.lspill && (!sm.lrecov || (rb == INF64 && fm == INF64))) {
                // recover spilled entries before they fall behind, at most once
                // between two processed buckets (re-spilled entries wait for
                // the bucket in front of them to be processed first)
                sm.flag = 2;
            } else if (fm != INF64 && (fm <= rb || fm < cur + LR<D>::NB / 2 ||
                                       (sm.lfar_n[fb] > c.slot.qcap / 2 && sm.lfar_n[fb] > 2 * sm.lfar_after))) {
                // far entries due soon, an empty ring, or a far list filling up
                // with stale entries (re-bucketing drops them)
                if (fm <= rb && fm > cur + 1) sm.lcur = sm.lfirst = fm - 1;
                sm.flag = 1;
            } else if (rb != INF64) {
                // the step takes bucket rb, and with rho the following ones
                // while the entries before them number fewer than rho (never a
                // bucket the far list reaches)
                const u32 j0 = (u32)(rb - cur);
                u32 jl = j0;
                if (a.rho) {
                    const u32 base = sm.lpre[j0 - 1];
                    for (u32 j = j0 + 1; j < LR<D>::NB; ++j) {
                        if (sm.lpre[j - 1] - base >= a.rho || cur + j >= fm) break;
                        if (sm.lpre[j] != sm.lpre[j - 1]) jl = j;
                    }
                }
                sm.lj0 = j0;
                sm.ljl = jl;
                sm.lfirst = rb;
                sm.lcur = cur + jl;
            } else if (sm.lspill) {
                sm.flag = 2;
            } else {
                sm.flag = 3;
            }
        }
        if (t == 0) {
            // a bounded number of decisions without processing a bucket: the
            // ring always gains entries from a redistribution or a recovery,
            // so this only trips on an internal error, never on valid input
            sm.lidle = (sm.flag == 1 || sm.flag == 2) ? sm.lidle + 1 : 0;
            if (sm.lidle > 4096) {
                atomicOr(a.err, ERRB_INTERNAL);
                sm.flag = 3;
            }
            if (sm.flag == 2) sm.lrecov = 1;
            if (sm.flag == 0) {
                sm.lrecov = 0;
                sm.llate = INF64;  // late entries of this bucket's processing
            }
        }
        __syncthreads();
        // every path below passes a barrier before thread 0 writes the flag
        // again (a chosen bucket is never empty)
        const u32 what = sm.flag;
        PH_MARK(sm, 0);  // decision
        if (what == 3) break;
        if (what == 1) {
            redistribute_far<D, B>(a, c, sm, L);
            PH_MARK(sm, 5);
            continue;
        }
        if (what == 2) {
            recover_spill<D, B>(a, c, sm, L, nwords);
            PH_MARK(sm, 6);
            continue;
        }
        // process buckets lfirst .. lcur (theta = lcur * step) as one list:
        // bucket cur0 + j holds entries lpre[j - 1] .. lpre[j] - 1 of the
        // ring window counted from the previous step's last bucket cur0
        ++rounds;
        const u32 j0 = sm.lj0, jl = sm.ljl;
        const u64 cur0 = sm.lfirst - j0;
        const u32 ob = c.slot.ocap / LR<D>::NB;
        const u32 pbase = sm.lpre[j0 - 1];
        const u32 n = sm.lpre[jl] - pbase;
        for (u32 base = 0; base < n; base += B) {
            const u32 cnt = min((u32)B, n - base);
            if (spread_index<B>(t) < cnt) {
                const u32 e = base + spread_index<B>(t);
                u32 j = j0;
                while (sm.lpre[j] - pbase <= e) ++j;  // at most jl (e < n)
                const u32 k = e - (sm.lpre[j - 1] - pbase);
                const u32 s = (u32)((cur0 + j) % LR<D>::NB);
                if (bad_index(a, k < L.cap + ob, 1)) {
                    sm.flat[t] = 0;
                    sm.d[t] = 0;
                } else if (k < L.cap) {
                    sm.flat[t] = L.rf[s * L.cap + k];
                    sm.d[t] = (u64)L.rd[s * L.cap + k];
                } else {
                    sm.flat[t] = __ldcg(c.slot.of + s * ob + (k - L.cap));
                    sm.d[t] = (u64)__ldcg(reinterpret_cast<const D*>(c.slot.od) + s * ob + (k - L.cap));
                }
            }
            // no barrier: thread t reads only its own staged entry before the
            // block scan inside process_local
            process_local<D, B>(a, c, sm, L, cnt, 0);
        }
        // the buckets receive nothing while they are processed (insertions go
        // to later buckets); the trailing barrier of process_local has been
        // passed by every thread, and only thread 0 reads rn next
        if (t == 0) {
            for (u32 j = j0; j <= jl; ++j) L.rn[(u32)((cur0 + j) % LR<D>::NB)] = 0;
            sm.lfirst = sm.lcur;  // the insertion window starts after this step
        }
    }
#ifdef PPSP_PHASE_CLOCKS
    if (t < 16) atomicAdd(&g_phase_clk[t], (unsigned long long)sm.ph_acc[t]);
#endif
    // entries left behind by the disconnected exit: clear the ring and spills
    if (sm.lspill) {
        for (u32 w = t; w < nwords; w += B) c.slot.bm[0][w] = 0u;
    }
#ifdef PPSP_BOUNDS_CHECK
    __syncthreads();
    for (u32 w = t; w < nwords; w += B)
        if (__ldcg(c.slot.bm[0] + w)) atomicOr(a.err, ERRB_INTERNAL | (21u << 8));
#endif
    __syncthreads();
    return rounds;
}

// ----------------------------------------------------------------------------
// paths: meeting vertex, then a warp walks tight edges back to each source
// ----------------------------------------------------------------------------
// Walk from x0 towards the source of search i along edges (u, x) with
// delta_i[u] + w(u, x) = delta_i[x] (smallest u first), writing x0, ..., q_i to
// out[start ..] while below cap.  Weights are >= 1, so delta_i strictly
// decreases along the walk; every such u has an exact delta_i because x does.
template <typename D, int B>
__device__ u64 walk_back(const EngineArgs& a, GCtx<D>& c, const Smem<B>& sm, u32 x0, u32 i, u32* out,
                         u64 cap, u64 start) {
    const u32 lane = threadIdx.x & 31;
    u32 x = x0;
    u64 idx = start;
    if (lane == 0 && idx < cap) out[idx] = x;
    ++idx;
    for (u32 steps = 0; x != sm.src[i]; ++steps) {
        if (steps > c.n) {  // cannot happen with positive weights; never loop forever
            if (lane == 0) atomicOr(a.err, ERRB_INTERNAL);
            break;
        }
        // the tight edges into x of a forward search are in-edges, those of
        // a backward search (distances to its target) out-edges
        const u64 dx = ld_dist(c.dist + flat_of(c.G, c.n, x, i));
        const u32* off = sm.sdir[i] ? a.g.off : a.g.off_t;
        const uint2* edges = sm.sdir[i] ? a.g.edges : a.g.edges_t;
        const u32 b0 = __ldg(off + x), b1 = __ldg(off + x + 1);
        u32 best = NONE;
        for (u32 e = b0 + lane; e < b1; e += 32) {
            const uint2 ew = __ldg(edges + e);
            const u64 du = ld_dist(c.dist + flat_of(c.G, c.n, ew.x, i));
            if (du != DT<D>::INF && du + ew.y == dx && ew.x < best) best = ew.x;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) best = min(best, __shfl_xor_sync(0xffffffffu, best, o));
        if (best == NONE) {
            if (lane == 0) atomicOr(a.err, ERRB_INTERNAL);
            break;
        }
        x = best;
        if (lane == 0 && idx < cap) out[idx] = x;
        ++idx;
    }
    return idx - start;
}

template <typename D, int B>
__device__ bool find_paths(const EngineArgs& a, const TeamCtx& tc, GCtx<D>& c, Smem<B>& sm, u32 flat_range) {
    const GroupDev& G = c.G;
    const u32 t = threadIdx.x;
    if (G.mode == GM_BIDIR) {
        // meeting vertex of each query edge: smallest v with delta_a[v] + delta_b[v] = mu
        const u32 tn = ld_volatile(&c.slot.st->touched_n);
        const bool tov = ld_volatile(&c.slot.st->touched_overflow) != 0;
        const u32 lim = tov ? flat_range : min(tn, c.slot.tcap);
        for (u32 k = tc.rank * B + t; k < lim; k += tc.size * B) {
            const u32 f = tov ? k : __ldcg(c.slot.touched + k);
            u32 v, i;
            decode_flat(G, c.n, f, v, i);
            if (i >= G.scnt) continue;
            const u64 di = ld_dist(c.dist + f);
            if (di == DT<D>::INF) continue;
            for (u32 p = 0; p < sm.pcnt[i]; ++p) {
                const PartnerDev pd = partner(a, sm, i, p);
                if (pd.j < i) continue;  // each query edge from its lower-index end
                const u64 dj = ld_dist(c.dist + flat_of(G, c.n, v, pd.j));
                if (dj != DT<D>::INF && di + dj == ldcg64(a.mu + pd.qe)) atomicMin(a.meet + pd.qe, v);
            }
        }
    } else if (tc.rank == 0 && t == 0) {
        a.meet[G.qbeg] = G.target;
    }
    if (!team_sync(tc, a, &sm.flag)) return false;
    const u32 warps = B / 32, lane = t & 31, wid = t >> 5;
    for (u32 q = tc.rank * warps + wid; q < G.qcnt; q += tc.size * warps) {
        const u32 qe = G.qbeg + q;
        const u64 mu = ldcg64(a.mu + qe);
        u64 len = 0;
        if (mu != INF64) {
            const QEdgeDev e = a.qedges[qe];
            const u32 m = ld_volatile(a.meet + qe);
            const u64 cap = a.path_off[qe + 1] - a.path_off[qe];
            u32* out = a.path_buf + a.path_off[qe];
            if (m == NONE) {
                if (lane == 0) atomicOr(a.err, ERRB_INTERNAL);
            } else {
                // q_a .. m: walk m -> q_a, then reverse in place
                const u64 na = walk_back<D, B>(a, c, sm, m, e.a, out, cap, 0);
                if (na <= cap) {
                    for (u64 k = lane; k < na / 2; k += 32) {
                        const u32 x = out[k];
                        out[k] = out[na - 1 - k];
                        out[na - 1 - k] = x;
                    }
                }
                __syncwarp();
                len = na;
                if (G.mode == GM_BIDIR) {
                    // m .. q_b along delta_b (m itself already written)
                    const u64 nb = walk_back<D, B>(a, c, sm, m, e.b, out, cap, na - 1);
                    len = na + nb - 1;
                }
            }
        }
        if (lane == 0) a.path_len[qe] = len;
    }
    return team_sync(tc, a, &sm.flag);
}

// ----------------------------------------------------------------------------
// one group
// ----------------------------------------------------------------------------
// LOCAL: every team is one CTA on the bucketed path (the host guarantees it),
// so the queue / bitmap path is compiled out and the kernel needs fewer
// registers.
template <typename D, int B, bool LOCAL>
__device__ bool run_group(const EngineArgs& a, const TeamCtx& tc, const SlotDev& slot, u32 gi,
                          Smem<B>& sm) {
    const u32 t = threadIdx.x;
    GCtx<D> c;
    c.G = a.groups[gi];
    c.slot = slot;
    c.dist = reinterpret_cast<D*>(slot.dist);
    c.n = a.g.n;
    c.c_x = c.c_e = c.c_r = c.c_p = c.c_t = 0;
    const GroupDev& G = c.G;
    StepState* S = slot.st->s;
    const u64 t_start = (a.group_ns && tc.rank == 0 && t == 0) ? global_ns() : 0;

    // group cache
    c.pair = (G.mode == GM_BIDIR && G.scnt == 2 && G.layout == PPSP_LAYOUT_INTERLEAVED && G.kshift == 1);
    c.memo = (a.memo && a.g.pc != nullptr) ? slot.memo : nullptr;
    c.err = a.err;
    c.adj16 = false;
    if (t == 0) {
        const SearchDev s0 = a.searches[G.sbeg];
        const SearchDev sl = a.searches[G.sbeg + G.scnt - 1];
        const u32 np = sl.pbeg + sl.pcnt - s0.pbeg;
        sm.pcached = (np <= PCAP) ? 1u : 0u;
        sm.pot_any = (G.mode == GM_ASTAR) ? 1u : 0u;
        sm.qn = 0;
        sm.tn = 0;
    }
    __syncthreads();
    if (t < G.scnt) {
        SearchDev s = a.searches[G.sbeg + t];
        const u32 p0 = a.searches[G.sbeg].pbeg;
        sm.src[t] = s.src;
        sm.pbeg[t] = sm.pcached ? s.pbeg - p0 : s.pbeg;
        sm.pcnt[t] = s.pcnt;
        sm.pot[t] = s.pot;
        sm.sdir[t] = s.dir;
        sm.key_off[t] = s.key_off;
        if (s.pot) atomicOr(&sm.pot_any, 1u);
        if (a.g.pc != nullptr) {
            sm.pa[t] = a.g.pc[s.src];
            sm.pb[t] = a.g.pc[s.pot_b];
        }
    }
    if (G.mode == GM_SSSP) {
        // SSSP groups have no partners: the cache holds the targets instead
        if (t == 0) sm.pcached = (G.qcnt <= PCAP) ? 1u : 0u;
        __syncthreads();
        if (sm.pcached)
            for (u32 k = t; k < G.qcnt; k += B) sm.pcache[k] = PartnerDev{a.qedges[G.qbeg + k].b, G.qbeg + k};
    } else if (sm.pcached) {
        const SearchDev s0 = a.searches[G.sbeg];
        const SearchDev sl = a.searches[G.sbeg + G.scnt - 1];
        const u32 np = sl.pbeg + sl.pcnt - s0.pbeg;
        for (u32 k = t; k < np; k += B) sm.pcache[k] = a.partners[s0.pbeg + k];
    }
    __syncthreads();
    // with a potential (and no memo), relaxations take P(target) from
    // 16-byte edge records when the graph has them
    c.adj16 = a.g.edges_pc != nullptr && sm.pot_any != 0 && c.memo == nullptr;

    // Init (Table 2): delta_i[q_i] = 0 and <q_i, i> in F for every search;
    // mu = inf (0 when both ends coincide).
    // one-CTA teams keep the frontier in shared memory (run_local); the
    // policies SPARSE and DENSE force the global queue / bitmap path
    const bool local = (tc.size == 1) && (a.frontier == PPSP_FRONTIER_AUTO) && !tc.global_bar;
    if (LOCAL && !local) {  // the host chose the local-only kernel for a plan it cannot run
        if (t == 0) atomicOr(a.err, ERRB_INTERNAL);
        return false;
    }
    if (!LOCAL && !local) {
        // the queue / bitmap path reads its two bitmaps as the frontier and as
        // the dedup of the next one: they start empty over the group's range
        // whatever an earlier group that used the slot left behind (a word
        // of another layout decodes to another search)
        const u32 nwg = (flat_range_of(G, c.n) + 31u) >> 5;
#ifdef PPSP_BOUNDS_CHECK
        for (u32 w = tc.rank * B + t; w < nwg; w += tc.size * B)
            if (__ldcg(slot.bm[0] + w) | __ldcg(slot.bm[1] + w)) atomicOr(a.err, ERRB_INTERNAL | (20u << 8));
#endif
        for (u32 w = tc.rank * B + t; w < nwg; w += tc.size * B) {
            slot.bm[0][w] = 0u;
            slot.bm[1][w] = 0u;
        }
        if (!team_sync(tc, a, &sm.flag)) return false;
    }
    if (tc.rank == 0) {
        if (t < G.scnt) {
            const u32 f = flat_of(G, c.n, sm.src[t], t);
            st_dist(c.dist + f, 0);
            if (!local) {
                atomicOr(slot.bm[0] + (f >> 5), 1u << (f & 31u));
                slot.q[0][t] = f;
            }
            slot.touched[t] = f;
        }
        for (u32 q = t; q < G.qcnt; q += B) {
            QEdgeDev e = a.qedges[G.qbeg + q];
            u64 m;
            if (G.mode == GM_BIDIR)
                m = (sm.src[e.a] == sm.src[e.b]) ? 0 : INF64;
            else if (G.mode == GM_SSSP)
                m = INF64;
            else
                m = (sm.src[0] == G.target) ? 0 : INF64;
            a.mu[G.qbeg + q] = m;
        }
        if (t == 0) {
            S[0].count = G.scnt;
            S[0].minkey = 0;
            S[0].tile = 0;
            S[0].overflow = 0;
            S[0].cnt_dir[0] = 1;
            S[0].cnt_dir[1] = G.scnt == 2 ? 1 : 0;
            S[0].bmax = INF64;
            S[1].bmax = INF64;
            S[1].count = 0;
            S[1].minkey = INF64;
            S[1].tile = 0;
            S[1].overflow = 0;
            S[1].cnt_dir[0] = S[1].cnt_dir[1] = 0;
            slot.st->touched_n = G.scnt;
            slot.st->touched_overflow = 0;
        }
        __syncthreads();
        if (t < G.scnt && G.mode == GM_BIDIR) {
            u64 m = 0;
            for (u32 p = 0; p < sm.pcnt[t]; ++p) {
                u64 mv = a.mu[partner(a, sm, t, p).qe];
                m = mv > m ? mv : m;
            }
            a.mumax[G.sbeg + t] = (sm.pcnt[t] == 0) ? INF64 : m;
        }
    }
    if (!team_sync(tc, a, &sm.flag)) return false;

    const u64 step = (G.mode == GM_BIDIR) ? 2 * G.delta : G.delta;
    const u32 flat_range = (G.layout == PPSP_LAYOUT_INTERLEAVED) ? (c.n << G.kshift) : G.scnt * c.n;
    const u32 nwords = (flat_range + 31u) >> 5;
    u64 dense_thresh = (a.dense_den == 0) ? ~0ull : (u64)flat_range / a.dense_den;
    c.theta = 0;
    bool dense_cur = (a.frontier == PPSP_FRONTIER_DENSE);
    u32 r = 0;
    u64 rounds = 0, dense_rounds = 0;
    u32 exit_count = 0, exit_bcur = 0;
    bool exit_dense = false;
    // prune bounds (the shared-memory mirror one-CTA teams read)
    if (t < G.scnt) {
        u64 b;
        if (G.mode == GM_BIDIR)
            b = (G.qcnt == 1) ? ldcg64(a.mu + G.qbeg) : ldcg64(a.mumax + G.sbeg + t);
        else if (G.mode == GM_SSSP)
            b = INF64;
        else
            b = ldcg64(a.mu + G.qbeg);
        sm.bound[t] = b;
    }
    if (local) {
        if (t == 0) {
            sm.tn = G.scnt;  // touched entries so far: the sources
            sm.tov = 0;
        }
        __syncthreads();
        rounds = run_local<D, B>(a, c, sm, nwords);
        if (t == 0) {
            slot.st->touched_n = sm.tn;
            slot.st->touched_overflow = sm.tov;
            sm.tn = 0;
        }
        __syncthreads();
    }
    for (; !LOCAL && !local; ++r) {
        const u32 cur = r % 3, nxt = (r + 1) % 3, old = (r + 2) % 3;
        const u32 bcur = r & 1u, bnxt = bcur ^ 1u;
        if (t == 0) {
            sm.count = ld_volatile(&S[cur].count);
            sm.overflow = ld_volatile(&S[cur].overflow);
            sm.minkey_in = ldcg64(&S[cur].minkey);
            sm.dir0 = ld_volatile(&S[cur].cnt_dir[0]);
            sm.dir1 = ld_volatile(&S[cur].cnt_dir[1]);
            sm.mu0 = ldcg64(a.mu + G.qbeg);
            const u64 bm = ldcg64(&S[cur].bmax);
            sm.cert = (u32)(bm <= sm.minkey_in);
            if (G.mode == GM_SSSP && bm < sm.bound[0]) sm.bound[0] = bm;
        }
        __syncthreads();
        const u32 count = sm.count;
        const u64 minkey = sm.minkey_in;
        dense_cur = dense_cur || sm.overflow != 0;
        // mu certificate: every entry's prune value >= its key >= minkey >= the
        // largest bound (snapshotted by the team leader before the barrier)
        bool stop = (count == 0) || (sm.cert != 0);
        // App. B: a two-search group whose one side ran dry before mu was ever
        // set is disconnected.
        if (!stop && G.mode == GM_BIDIR && G.scnt == 2 && sm.mu0 == INF64 &&
            (sm.dir0 == 0 || sm.dir1 == 0))
            stop = true;
        if (stop) {
            exit_count = count;
            exit_bcur = bcur;
            exit_dense = dense_cur;
            break;
        }
        // GetDist: next multiple of the step, at least one step further and
        // not below the smallest key in F.
        {
            u64 want = c.theta + step;
            u64 rk = (minkey / step) * step;
            if (rk < minkey) rk += step;
            c.theta = want > rk ? want : rk;
        }
        c.dense_nxt = (a.frontier == PPSP_FRONTIER_DENSE) ||
                      (a.frontier == PPSP_FRONTIER_AUTO && (u64)count > dense_thresh);
        c.bm_cur = slot.bm[bcur];
        c.bm_nxt = slot.bm[bnxt];
        c.q_nxt = slot.q[bnxt];
        c.S_nxt = &S[nxt];
        if (tc.rank == 0 && t == 0) {
            S[old].count = 0;
            S[old].minkey = INF64;
            S[old].tile = 0;
            S[old].overflow = 0;
            S[old].cnt_dir[0] = S[old].cnt_dir[1] = 0;
            S[old].bmax = INF64;
        }
        if (t == 0) {
            sm.minkey_acc = INF64;
            sm.cnt_dir[0] = sm.cnt_dir[1] = 0;
        }
        __syncthreads();
        ++rounds;
        if (dense_cur) ++dense_rounds;

        if (!dense_cur) {
            const u32 nt = (count + B - 1) / B;
            u32 local = tc.rank;
            for (;;) {
                if (t == 0) sm.tile = tc.size == 1 ? local : atomicAdd(&S[cur].tile, 1u);
                __syncthreads();
                const u32 tile = sm.tile;
                __syncthreads();
                if (tile >= nt) break;
                local += tc.size;
                const u32 base = tile * B;
                const u32 cnt = min((u32)B, count - base);
                if (t < cnt) sm.flat[t] = __ldcg(slot.q[bcur] + base + t);
                __syncthreads();
                process_items<D, B>(a, c, sm, cnt, true, c.bm_cur);
            }
        } else {
            const u32 nt = (nwords + B - 1) / B;
            u32 local = tc.rank;
            for (;;) {
                if (t == 0) sm.tile = tc.size == 1 ? local : atomicAdd(&S[cur].tile, 1u);
                __syncthreads();
                const u32 tile = sm.tile;
                __syncthreads();
                if (tile >= nt) break;
                local += tc.size;
                const u32 w = tile * B + t;
                u32 bits = 0;
                if (w < nwords) {
                    bits = __ldcg(c.bm_cur + w);
                    if (bits) c.bm_cur[w] = 0u;
                }
                u32 total;
                u32 idx = block_excl_scan<B>(__popc(bits), sm, &total);
                for (u32 base = 0; base < total; base += B) {
                    while (bits && idx < base + B) {
                        const u32 b = __ffs(bits) - 1;
                        bits &= bits - 1;
                        sm.flat[idx - base] = (w << 5) | b;
                        ++idx;
                    }
                    __syncthreads();
                    process_items<D, B>(a, c, sm, min((u32)B, total - base), false, c.bm_cur);
                }
            }
        }
        // flush per-CTA step results
        __syncthreads();
        if (G.mode == GM_SSSP && tc.rank == 0 && t < 32) {
            const u64 m = sssp_target_max<D, B>(a, c, sm);
            if (t == 0) S[nxt].bmax = (m == 0) ? INF64 : m;
        } else if (t == 0 && tc.rank == 0) {
            u64 bmax = 0;
            for (u32 i = 0; i < G.scnt && bmax != INF64; ++i) {
                u64 b;
                if (G.mode == GM_BIDIR)
                    b = (G.qcnt == 1) ? ldcg64(a.mu + G.qbeg) : ldcg64(a.mumax + G.sbeg + i);
                else if (G.mode == GM_SSSP)
                    b = INF64;
                else
                    b = ldcg64(a.mu + G.qbeg);
                bmax = b > bmax ? b : bmax;
            }
            S[nxt].bmax = (bmax == 0) ? INF64 : bmax;
        }
        if (t == 0) {
            if (sm.minkey_acc != INF64)
                amin64(&S[nxt].minkey, sm.minkey_acc);
            if (sm.cnt_dir[0]) atomicAdd(&S[nxt].cnt_dir[0], sm.cnt_dir[0]);
            if (sm.cnt_dir[1]) atomicAdd(&S[nxt].cnt_dir[1], sm.cnt_dir[1]);
        }
        if (!team_sync(tc, a, &sm.flag)) return false;
        dense_cur = c.dense_nxt;
    }

    // ---- SSSP-based batches (Sec. 4.3): every query of the group reads its
    // other endpoint's final distance from the single search ----
    if (G.mode == GM_SSSP && G.qcnt > 0) {
        for (u32 q = tc.rank * B + t; q < G.qcnt; q += tc.size * B) {
            const QEdgeDev e = a.qedges[G.qbeg + q];
            const u64 d = ld_dist(c.dist + flat_of(G, c.n, e.b, 0));
            a.mu[G.qbeg + q] = (d == DT<D>::INF) ? INF64 : d;
        }
        if (!team_sync(tc, a, &sm.flag)) return false;
    }

    // ---- paths (optional), before the distances are reset ----
    if (a.path_buf != nullptr && !find_paths<D, B>(a, tc, c, sm, flat_range)) return false;

    // ---- tidy the slot ----
    if (exit_count > 0) {
        // the frontier was abandoned (disconnected exit): clear its bits
        u32* bm = slot.bm[exit_bcur];
        if (exit_dense) {
            for (u32 w = tc.rank * B + t; w < nwords; w += tc.size * B) bm[w] = 0u;
        } else {
            const u32 q_n = min(exit_count, slot.qcap);
            for (u32 k = tc.rank * B + t; k < q_n; k += tc.size * B) bm[__ldcg(slot.q[exit_bcur] + k) >> 5] = 0u;
        }
    }
    {
        // memoized terms exist only for touched entries (a term is evaluated
        // for an extracted entry or after a successful relaxation)
        const u32 tn = ld_volatile(&slot.st->touched_n);
        const u32 tov = ld_volatile(&slot.st->touched_overflow);
        if (tov) {
            for (u32 f = tc.rank * B + t; f < flat_range; f += tc.size * B) {
                st_dist(c.dist + f, DT<D>::INF);
                if (c.memo) c.memo[c.pair ? (f >> 1) : f] = 0u;
            }
        } else {
            for (u32 k = tc.rank * B + t; k < tn; k += tc.size * B) {
                const u32 f = __ldcg(slot.touched + k);
                if (bad_index(a, f < flat_range && k < slot.tcap, 8)) continue;
                st_dist(c.dist + f, DT<D>::INF);
                if (c.memo) c.memo[c.pair ? (f >> 1) : f] = 0u;
            }
        }
    }
    // this group's counts, one atomic per warp and counter (order of
    // EngineCounters: extracted, edges, relaxed, pushed, rounds, groups,
    // searches, touched, dense_rounds)
    if (a.counters) {
        unsigned long long* cp = &a.counters->extracted;
        const u32 mine[5] = {c.c_x, c.c_e, c.c_r, c.c_p, c.c_t};
        const int at[5] = {0, 1, 2, 3, 7};
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            u64 x = mine[k];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
            if ((t & 31u) == 0 && x) atomicAdd(cp + at[k], (unsigned long long)x);
        }
        if (t == 0 && tc.rank == 0) {
            atomicAdd(cp + 4, (unsigned long long)rounds);
            atomicAdd(cp + 5, 1ull);
            atomicAdd(cp + 6, (unsigned long long)G.scnt);
            if (dense_rounds) atomicAdd(cp + 8, (unsigned long long)dense_rounds);
        }
    }
    if (a.group_ns && t == 0 && tc.rank == 0) a.group_ns[gi] = global_ns() - t_start;
    return team_sync(tc, a, &sm.flag);
}

template <typename D, int B>
constexpr size_t engine_smem_bytes(u32 ring_cap) {
    return ((sizeof(Smem<B>) + 15) & ~(size_t)15) + LR<D>::bytes(ring_cap);
}

// Threads per SM the engine is compiled to keep resident (register budget):
// 512 gives one 512-thread CTA per SM up to 128 registers per thread (the
// two-way relaxation keeps its loads in registers instead of spilling); a
// 1,024-thread CTA gets 64.
#ifndef PPSP_ENGINE_SM_THREADS
#define PPSP_ENGINE_SM_THREADS 512
#endif

// The one-CTA (LOCAL) instances keep 1,024 threads per SM resident: one
// CTA of 1,024, two of 512 or four of 256 (64 registers per thread); each
// CTA runs its own group, so smaller CTAs run more groups side by side.
template <int B, bool LOCAL>
struct EngineMinBlocks {
    static constexpr int value = LOCAL ? 1024 / B : ((PPSP_ENGINE_SM_THREADS / B) > 0 ? PPSP_ENGINE_SM_THREADS / B : 1);
};

template <typename D, int B, bool LOCAL>
__global__ void __launch_bounds__(B, (EngineMinBlocks<B, LOCAL>::value))
    engine_kernel(EngineArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Smem<B>& sm = *reinterpret_cast<Smem<B>*>(smem_raw);
    TeamCtx tc;
    tc.team = a.cta_team[blockIdx.x];
    tc.rank = blockIdx.x - a.team_first[tc.team];
    tc.size = a.team_size[tc.team];
    tc.ts = a.tstate + tc.team;
    if (tc.rank >= tc.size) {  // a CTA outside its team's range: the host's team tables disagree with the grid
        if (threadIdx.x == 0) atomicOr(a.err, ERRB_INTERNAL);
        return;
    }
    const bool never = (a.debug & PPSP_DEBUG_BARRIER_NEVER_RELEASES) != 0;
    tc.global_bar = tc.size > 1 || never;
    tc.expect = tc.size + (never ? 1u : 0u);
    const u32 qid = a.team_queue[tc.team];
    const SlotDev slot = a.slots[tc.team];
    for (;;) {
        if (threadIdx.x == 0) {
            if (tc.rank == 0) {
                u32 idx = atomicAdd(a.queue_head + qid, 1u);
                u32 g = idx < a.queue_len[qid] ? a.queue_items[qid][idx] : NONE;
                if (tc.global_bar) tc.ts->group = g;
                sm.group = g;
            }
        }
        if (!team_sync(tc, a, &sm.flag)) break;
        if (tc.global_bar && threadIdx.x == 0) sm.group = ld_volatile(&tc.ts->group);
        __syncthreads();
        const u32 gi = sm.group;
        if (!team_sync(tc, a, &sm.flag)) break;  // everyone has read ts->group
        if (gi == NONE) break;
        if (!run_group<D, B, LOCAL>(a, tc, slot, gi, sm)) break;
    }
}

// ----------------------------------------------------------------------------
// host side
// ----------------------------------------------------------------------------
// The dynamic shared-memory limit is an attribute of the function on the
// current device: it is set once per instantiation and device.
constexpr int SMEM_ATTR_DEVICES = 64;
template <typename D, int B, bool LOCAL>
static ppsp_status set_smem_attr() {
    static std::atomic<bool> done[SMEM_ATTR_DEVICES];
    int dev = 0;
    PPSP_CUDA_TRY(cudaGetDevice(&dev));
    if (dev >= 0 && dev < SMEM_ATTR_DEVICES && done[dev].load(std::memory_order_acquire)) return PPSP_OK;
    PPSP_CUDA_TRY(cudaFuncSetAttribute(engine_kernel<D, B, LOCAL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)engine_smem_bytes<D, B>(RING_CAP_MAX)));
    if (dev >= 0 && dev < SMEM_ATTR_DEVICES) done[dev].store(true, std::memory_order_release);
    return PPSP_OK;
}

template <typename D, int B, bool LOCAL>
static ppsp_status launch_t(const EngineArgs& a, u32 grid, cudaStream_t stream) {
    ppsp_status st = set_smem_attr<D, B, LOCAL>();
    if (st != PPSP_OK) return st;
    EngineArgs args = a;
    void* params[] = {&args};
    PPSP_CUDA_TRY(cudaLaunchCooperativeKernel((const void*)engine_kernel<D, B, LOCAL>, dim3(grid), dim3(B),
                                              params, engine_smem_bytes<D, B>(a.ring_cap), stream));
    return PPSP_OK;
}

// The three block sizes of one (distance width, LOCAL) instance family.
template <typename D, bool LOCAL>
static ppsp_status launch_family(const EngineArgs& a, int block_threads, u32 grid, cudaStream_t stream) {
    if (a.ring_cap < 1 || a.ring_cap > RING_CAP_MAX) return PPSP_ERR_INVALID_ARG;
    if (block_threads == 256) return launch_t<D, 256, LOCAL>(a, grid, stream);
    if (block_threads == 512) return launch_t<D, 512, LOCAL>(a, grid, stream);
    if (block_threads == 1024) return launch_t<D, 1024, LOCAL>(a, grid, stream);
    return PPSP_ERR_INVALID_ARG;
}

template <typename D, int B, bool LOCAL>
static ppsp_status occ_t(int* bpsm, u32 ring_cap) {
    ppsp_status st = set_smem_attr<D, B, LOCAL>();
    if (st != PPSP_OK) return st;
    PPSP_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(bpsm, engine_kernel<D, B, LOCAL>, B,
                                                                engine_smem_bytes<D, B>(ring_cap)));
    return PPSP_OK;
}

template <typename D, bool LOCAL>
static ppsp_status occ_family(int block_threads, u32 ring_cap, int* bpsm) {
    if (ring_cap < 1 || ring_cap > RING_CAP_MAX) return PPSP_ERR_INVALID_ARG;
    if (block_threads == 256) return occ_t<D, 256, LOCAL>(bpsm, ring_cap);
    if (block_threads == 512) return occ_t<D, 512, LOCAL>(bpsm, ring_cap);
    if (block_threads == 1024) return occ_t<D, 1024, LOCAL>(bpsm, ring_cap);
    return PPSP_ERR_INVALID_ARG;
}

}  // namespace ppsp
