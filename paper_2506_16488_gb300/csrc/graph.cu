// Graph creation, validation, A* potential, slot pool, small ABI helpers.
#include <cstdarg>
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <thread>

#include "graph_impl.h"

namespace ppsp {

static thread_local char g_last_error[512] = {0};

void set_last_cuda_error(cudaError_t e, const char* what, const char* file, int line) {
    snprintf(g_last_error, sizeof(g_last_error), "%s failed: %s (%s:%d)", what, cudaGetErrorString(e), file,
             line);
}

void set_last_device_error(u32 err) {
    snprintf(g_last_error, sizeof(g_last_error), "device error word 0x%x (internal error, site %u)", err,
             (err >> 8) & 0xFFu);
}

void set_last_internal_error(const char* fmt, ...) {
    char msg[400];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(msg, sizeof(msg), fmt, ap);
    va_end(ap);
    snprintf(g_last_error, sizeof(g_last_error), "internal error: %s", msg);
}

u64 isqrt_host(u64 x) {
    // bitwise integer square root: exact floor(sqrt(x))
    u64 r = 0, bit = 1ull << 62;
    while (bit > x) bit >>= 2;
    while (bit != 0) {
        if (x >= r + bit) {
            x -= r + bit;
            r = (r >> 1) + bit;
        } else {
            r >>= 1;
        }
        bit >>= 2;
    }
    return r;
}

i64 pot_h_host(const ppsp_graph* g, u32 x, u32 v) {
    if (g->pc_host.empty()) return 0;
    i64 dx = g->pc_host[2 * (u64)v] - g->pc_host[2 * (u64)x];
    i64 dy = g->pc_host[2 * (u64)v + 1] - g->pc_host[2 * (u64)x + 1];
    u64 d2 = (u64)(dx * dx) + (u64)(dy * dy);
    return (i64)isqrt_host(d2 >> (2 * g->pot_shift));
}

template <typename F>
static void parallel_for(u64 n, F f) {
    unsigned nt = std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
    if (n < (1u << 16)) nt = 1;
    std::vector<std::thread> th;
    for (unsigned k = 0; k < nt; ++k)
        th.emplace_back([=, &f]() {
            u64 lo = n * k / nt, hi = n * (k + 1) / nt;
            f(lo, hi, k);
        });
    for (auto& t : th) t.join();
}

// The certified integer potential (Sec. 3.3, Fact 3.1): choose c and F, round
// P(v) = floor(p(v) * c * 2^F + 0.5), and check |P(u)-P(v)|^2 <= (2^F w)^2 on
// every edge in exact integer arithmetic; shrink c until the check passes.
static void build_potential(ppsp_graph* g, const u64* off, const u32* tgt, const u32* w, const float* xy) {
    const u64 n = g->n;
    double cmax = INFINITY;
    double amax = 0.0;
    bool zero_block = false;
    u64 wmin_pos = ~0ull;
    for (u64 v = 0; v < n; ++v) {
        amax = std::max(amax, (double)std::fabs(xy[2 * v]));
        amax = std::max(amax, (double)std::fabs(xy[2 * v + 1]));
    }
    for (u64 u = 0; u < n; ++u)
        for (u64 e = off[u]; e < off[u + 1]; ++e) {
            u64 v = tgt[e];
            double dx = (double)xy[2 * u] - (double)xy[2 * v];
            double dy = (double)xy[2 * u + 1] - (double)xy[2 * v + 1];
            double l = std::sqrt(dx * dx + dy * dy);
            if (l > 0.0) {
                if (w[e] == 0) zero_block = true;
                cmax = std::min(cmax, (double)w[e] / l);
                wmin_pos = std::min<u64>(wmin_pos, w[e]);
            }
        }
    g->pc_host.assign(2 * n, 0);
    if (zero_block || !std::isfinite(cmax) || cmax <= 0.0 || amax == 0.0) {
        g->pot_scale = 0.0;
        g->pot_shift = 0;
        return;
    }
    int F = 8;
    while (F > 0 && amax * cmax * std::ldexp(1.0, F) >= std::ldexp(1.0, 30)) --F;
    if (amax * cmax * std::ldexp(1.0, F) >= std::ldexp(1.0, 30)) {
        g->pot_scale = 0.0;
        g->pot_shift = 0;
        return;
    }
    double eps = 2.0 / (std::ldexp(1.0, F) * (double)std::max<u64>(1, wmin_pos));
    for (int attempt = 0; attempt < 40; ++attempt, eps *= 2.0) {
        double c = cmax * (1.0 - eps);
        if (c <= 0.0) break;
        const double s = std::ldexp(1.0, F) * c;
        for (u64 v = 0; v < 2 * n; ++v) g->pc_host[v] = (int64_t)std::floor((double)xy[v] * s + 0.5);
        std::atomic<bool> ok(true);
        const int64_t* P = g->pc_host.data();
        parallel_for(n, [&](u64 lo, u64 hi, unsigned) {
            for (u64 u = lo; u < hi && ok.load(std::memory_order_relaxed); ++u)
                for (u64 e = off[u]; e < off[u + 1]; ++e) {
                    u64 v = tgt[e];
                    __int128 dx = P[2 * u] - P[2 * v], dy = P[2 * u + 1] - P[2 * v + 1];
                    __int128 lhs = dx * dx + dy * dy;
                    __int128 rw = ((__int128)w[e]) << F;
                    if (lhs > rw * rw) {
                        ok = false;
                        break;
                    }
                }
        });
        if (ok) {
            g->pot_scale = c;
            g->pot_shift = F;
            return;
        }
    }
    std::fill(g->pc_host.begin(), g->pc_host.end(), 0);
    g->pot_scale = 0.0;
    g->pot_shift = 0;
}

static bool check_symmetric(u64 n, const u64* off, const u32* tgt, const u32* w) {
    const u64 m = off[n];
    std::vector<u64> key(m);
    parallel_for(n, [&](u64 lo, u64 hi, unsigned) {
        for (u64 u = lo; u < hi; ++u) {
            for (u64 e = off[u]; e < off[u + 1]; ++e) key[e] = ((u64)tgt[e] << 32) | w[e];
            std::sort(key.begin() + off[u], key.begin() + off[u + 1]);
        }
    });
    std::atomic<bool> ok(true);
    parallel_for(n, [&](u64 lo, u64 hi, unsigned) {
        for (u64 u = lo; u < hi && ok.load(std::memory_order_relaxed); ++u)
            for (u64 e = off[u]; e < off[u + 1]; ++e) {
                u64 v = tgt[e];
                u64 want = (u << 32) | w[e];
                if (!std::binary_search(key.begin() + off[v], key.begin() + off[v + 1], want)) {
                    ok = false;
                    break;
                }
            }
    });
    return ok;
}

// Position of the point (x, y) of a 2^bits x 2^bits lattice along the
// Hilbert curve that fills it: at each scale the quadrant adds its rank in
// the curve's visiting order (lower-left, upper-left, upper-right,
// lower-right for the unrotated curve) times the quadrant's size, and the
// point is rotated or reflected into the orientation the curve has inside
// that quadrant.
static u64 hilbert_rank(u32 x, u32 y, u32 bits) {
    const u32 side = 1u << bits;
    u64 d = 0;
    for (u32 q = side >> 1; q > 0; q >>= 1) {
        const u32 rx = (x & q) ? 1u : 0u, ry = (y & q) ? 1u : 0u;
        d += (u64)q * q * ((3u * rx) ^ ry);
        if (ry == 0) {
            if (rx == 1) {
                x = side - 1 - x;
                y = side - 1 - y;
            }
            const u32 tmp = x;
            x = y;
            y = tmp;
        }
    }
    return d;
}

// Device order of a graph with coordinates: vertices sorted by the Hilbert
// rank of their coordinates on a 2^16 x 2^16 lattice over the bounding
// square (ties by id).  Returns false (order kept) for non-finite
// coordinates.  perm[v] = device id of caller vertex v; inv = its inverse.
static bool locality_order(u64 n, const float* xy, std::vector<u32>& perm, std::vector<u32>& inv) {
    double xmin = INFINITY, ymin = INFINITY, xmax = -INFINITY, ymax = -INFINITY;
    for (u64 v = 0; v < n; ++v) {
        const double x = xy[2 * v], y = xy[2 * v + 1];
        if (!std::isfinite(x) || !std::isfinite(y)) return false;
        xmin = std::min(xmin, x);
        xmax = std::max(xmax, x);
        ymin = std::min(ymin, y);
        ymax = std::max(ymax, y);
    }
    const double span = std::max(xmax - xmin, ymax - ymin);
    const double scale = span > 0.0 ? 65535.0 / span : 0.0;
    std::vector<u64> key(n);
    for (u64 v = 0; v < n; ++v) {
        const u32 qx = (u32)std::min(65535.0, std::max(0.0, ((double)xy[2 * v] - xmin) * scale));
        const u32 qy = (u32)std::min(65535.0, std::max(0.0, ((double)xy[2 * v + 1] - ymin) * scale));
        key[v] = (hilbert_rank(qx, qy, 16) << 32) | v;  // the rank is below 2^32
    }
    std::sort(key.begin(), key.end());
    perm.resize(n);
    inv.resize(n);
    for (u64 i = 0; i < n; ++i) {
        const u32 v = (u32)(key[i] & 0xFFFFFFFFull);
        inv[i] = v;
        perm[v] = (u32)i;
    }
    return true;
}

SlotCaps slot_caps(u64 range, int frontier, bool whole_gpu) {
    u64 fc = std::max<u64>(range, 64);
    fc = (fc + 63) & ~63ull;
    SlotCaps c;
    c.flat_cap = fc;
    c.qcap = (frontier == PPSP_FRONTIER_SPARSE) ? (u32)fc : (u32)std::min<u64>(fc, fc / 8 + 4096);
    c.tcap = whole_gpu ? (u32)fc : (u32)std::min<u64>(fc, fc / 4 + 4096);
    return c;
}

namespace {
struct SlotLayout {
    u64 ocap, b_dist, b_bm, b_q, b_fd, b_t, b_st, b_of, b_od, b_memo, total;
};
SlotLayout slot_layout(int dist_bits, u64 flat_cap, u32 qcap, u32 tcap, bool memo) {
    const u64 W = dist_bits / 8;
    const u64 words = (flat_cap + 31) / 32;
    auto al = [](u64 x) { return (x + 255) & ~255ull; };
    SlotLayout L;
    L.ocap = std::max<u64>(32 * 256, flat_cap / 4) / 32 * 32;
    L.b_dist = al(flat_cap * W);
    L.b_bm = al(words * 4);
    L.b_q = al((u64)qcap * 4);
    L.b_fd = al((u64)qcap * W);
    L.b_t = al((u64)tcap * 4);
    L.b_st = al(sizeof(SlotState));
    L.b_of = al(L.ocap * 4);
    L.b_od = al(L.ocap * W);
    L.b_memo = memo ? al(flat_cap * 4) : 0;
    L.total = L.b_dist + 2 * L.b_bm + 2 * L.b_q + 2 * L.b_fd + L.b_t + L.b_st + L.b_of + L.b_od + L.b_memo;
    return L;
}
}  // namespace

u64 slot_alloc_bytes(int dist_bits, u64 flat_cap, u32 qcap, u32 tcap, bool memo) {
    return slot_layout(dist_bits, flat_cap, qcap, tcap, memo).total;
}

ppsp_status slot_acquire(ppsp_graph* g, int dist_bits, u64 flat_cap, u32 qcap, u32 tcap, bool memo,
                         cudaStream_t stream, Slot** out) {
    SlotKey key{dist_bits, flat_cap, qcap, tcap, memo};
    for (auto it = g->pool.lower_bound(key); it != g->pool.end(); ++it) {
        Slot* s = it->second.get();
        if (!s->busy && it->first.dist_bits == dist_bits && it->first.flat_cap >= flat_cap &&
            it->first.qcap >= qcap && it->first.tcap >= tcap && it->first.flat_cap <= 2 * flat_cap + 4096 &&
            (it->first.memo || !memo)) {
            s->busy = true;
            *out = s;
            return PPSP_OK;
        }
    }
    auto s = std::make_unique<Slot>();
    const SlotLayout L = slot_layout(dist_bits, flat_cap, qcap, tcap, memo);
    const u64 ocap = L.ocap, b_dist = L.b_dist, b_bm = L.b_bm, b_q = L.b_q, b_fd = L.b_fd, b_t = L.b_t,
              b_st = L.b_st, b_of = L.b_of, b_od = L.b_od;
    s->bytes = L.total;
    cudaError_t e = cudaMalloc(&s->base, s->bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return e == cudaErrorMemoryAllocation ? PPSP_ERR_OOM : PPSP_ERR_CUDA;
    }
    char* p = (char*)s->base;
    s->dev.dist = p;
    p += b_dist;
    s->dev.bm[0] = (u32*)p;
    p += b_bm;
    s->dev.bm[1] = (u32*)p;
    p += b_bm;
    s->dev.q[0] = (u32*)p;
    p += b_q;
    s->dev.q[1] = (u32*)p;
    p += b_q;
    s->dev.fd[0] = p;
    p += b_fd;
    s->dev.fd[1] = p;
    p += b_fd;
    s->dev.of = (u32*)p;
    p += b_of;
    s->dev.od = p;
    p += b_od;
    s->dev.ocap = (u32)ocap;
    s->dev.touched = (u32*)p;
    p += b_t;
    s->dev.st = (SlotState*)p;
    p += b_st;
    s->dev.memo = memo ? (u32*)p : nullptr;
    s->dev.flat_cap = flat_cap;
    s->dev.qcap = qcap;
    s->dev.tcap = tcap;
    s->dist_bits = dist_bits;
    s->flat_cap = flat_cap;
    // clean invariant: distances infinite (all-ones bytes), bitmaps zero.
    // Written on the stream of the plan that takes the slot, so the writes
    // are ordered before its searches (a plain cudaMemset runs on the legacy
    // default stream, which a non-blocking stream does not wait for).
    PPSP_CUDA_TRY(cudaMemsetAsync(s->dev.dist, 0xFF, b_dist, stream));
    PPSP_CUDA_TRY(cudaMemsetAsync(s->dev.bm[0], 0, 2 * b_bm, stream));
    PPSP_CUDA_TRY(cudaMemsetAsync(s->dev.st, 0, b_st, stream));
    if (memo) PPSP_CUDA_TRY(cudaMemsetAsync(s->dev.memo, 0, L.b_memo, stream));  // 0 = no term memoized
    s->busy = true;
    *out = s.get();
    g->pool.emplace(key, std::move(s));
    return PPSP_OK;
}

void slot_release(ppsp_graph* g, Slot* s) {
    (void)g;
    if (s) s->busy = false;
}

ppsp_status slot_scrub(Slot* s, cudaStream_t stream) {
    if (!s->dirty) return PPSP_OK;
    const u64 W = s->dist_bits / 8;
    const u64 words = (s->flat_cap + 31) / 32;
    PPSP_CUDA_TRY(cudaMemsetAsync(s->dev.dist, 0xFF, s->flat_cap * W, stream));
    PPSP_CUDA_TRY(cudaMemsetAsync(s->dev.bm[0], 0, words * 4, stream));
    PPSP_CUDA_TRY(cudaMemsetAsync(s->dev.bm[1], 0, words * 4, stream));
    PPSP_CUDA_TRY(cudaMemsetAsync(s->dev.st, 0, sizeof(SlotState), stream));
    if (s->dev.memo) PPSP_CUDA_TRY(cudaMemsetAsync(s->dev.memo, 0, s->flat_cap * 4, stream));
    s->dirty = false;
    return PPSP_OK;
}

}  // namespace ppsp

using namespace ppsp;

extern "C" {

void ppsp_options_init(ppsp_options* o) {
    if (!o) return;
    memset(o, 0, sizeof(*o));
    o->mode = PPSP_BIDS;
    o->dist_bits = 32;
    o->frontier = PPSP_FRONTIER_AUTO;
    o->layout = PPSP_LAYOUT_AUTO;
    o->batch_strategy = PPSP_BATCH_MULTI;
}

const char* ppsp_status_string(ppsp_status s) {
    switch (s) {
        case PPSP_OK: return "ok";
        case PPSP_ERR_INVALID_ARG: return "invalid argument";
        case PPSP_ERR_BAD_GRAPH: return "malformed graph";
        case PPSP_ERR_OOM: return "out of memory";
        case PPSP_ERR_CUDA: return "CUDA error";
        case PPSP_ERR_TIMEOUT: return "device wait timed out";
        case PPSP_ERR_NO_COORDS: return "graph has no coordinates";
        case PPSP_ERR_BUFFER_TOO_SMALL: return "buffer too small";
        case PPSP_ERR_OVERFLOW: return "distance overflows the distance width";
        case PPSP_ERR_UNSUPPORTED: return "unsupported request";
    }
    return "unknown status";
}

const char* ppsp_last_error_detail(void) { return g_last_error; }

ppsp_status ppsp_graph_create(uint64_t n, uint64_t m, const uint64_t* offsets, const uint32_t* targets,
                              const uint32_t* weights, const float* coords, uint32_t flags,
                              ppsp_graph** out) {
    if (!out || !offsets || (m > 0 && (!targets || !weights))) return PPSP_ERR_INVALID_ARG;
    *out = nullptr;
    if (n == 0 || n >= 0xFFFFFFFFull || m >= 0xFFFFFFFFull) return PPSP_ERR_INVALID_ARG;
    if (offsets[0] != 0 || offsets[n] != m) return PPSP_ERR_BAD_GRAPH;
    for (u64 v = 0; v < n; ++v)
        if (offsets[v + 1] < offsets[v]) return PPSP_ERR_BAD_GRAPH;
    for (u64 e = 0; e < m; ++e)
        if (targets[e] >= n) return PPSP_ERR_BAD_GRAPH;
    if ((flags & PPSP_UNDIRECTED) && !check_symmetric(n, offsets, targets, weights)) return PPSP_ERR_BAD_GRAPH;

    auto g = std::make_unique<ppsp_graph>();
    g->n = n;
    g->m = m;
    // device order: along a Hilbert curve over the coordinates, so that a
    // search's compact frontier region maps to few cache lines; the arrays
    // below are renumbered copies and every call maps ids at the boundary
    std::vector<u64> off_r;
    std::vector<u32> tgt_r, w_r;
    std::vector<float> xy_r;
    if (coords && !(flags & PPSP_KEEP_VERTEX_ORDER) && n > 1 && locality_order(n, coords, g->perm, g->inv)) {
        off_r.resize(n + 1);
        tgt_r.resize(m);
        w_r.resize(m);
        xy_r.resize(2 * n);
        off_r[0] = 0;
        for (u64 i = 0; i < n; ++i) {
            const u64 v = g->inv[i];
            u64 o = off_r[i];
            for (u64 e = offsets[v]; e < offsets[v + 1]; ++e, ++o) {
                tgt_r[o] = g->perm[targets[e]];
                w_r[o] = weights[e];
            }
            off_r[i + 1] = o;
            xy_r[2 * i] = coords[2 * v];
            xy_r[2 * i + 1] = coords[2 * v + 1];
        }
        offsets = off_r.data();
        targets = tgt_r.data();
        weights = w_r.data();
        coords = xy_r.data();
    }
    ppsp_graph_info& info = g->info;
    info.n = n;
    info.m = m;
    info.undirected = (flags & PPSP_UNDIRECTED) ? 1 : 0;
    info.has_coords = coords ? 1 : 0;
    u64 wmin = ~0ull, wmax = 0;
    double sum = 0, sum2 = 0;
    for (u64 e = 0; e < m; ++e) {
        u64 x = weights[e];
        wmin = std::min(wmin, x);
        wmax = std::max(wmax, x);
        sum += (double)x;
        sum2 += (double)x * (double)x;
        if (x == 0) info.has_zero_weight = 1;
    }
    info.w_min = m ? wmin : 0;
    info.w_max = wmax;
    info.w_mean = m ? sum / (double)m : 0.0;
    info.w_std = m ? std::sqrt(std::max(0.0, sum2 / (double)m - info.w_mean * info.w_mean)) : 0.0;
    g->deg.resize(n);
    u64 dmax = 0;
    for (u64 v = 0; v < n; ++v) {
        g->deg[v] = offsets[v + 1] - offsets[v];
        dmax = std::max(dmax, g->deg[v]);
    }
    info.deg_max = dmax;
    if (coords) build_potential(g.get(), offsets, targets, weights, coords);
    info.potential_scale = g->pot_scale;
    info.potential_shift = g->pot_shift;

    // device copies
    std::vector<u32> off32(n + 1);
    for (u64 v = 0; v <= n; ++v) off32[v] = (u32)offsets[v];
    std::vector<uint2> ed(m);
    for (u64 e = 0; e < m; ++e) ed[e] = make_uint2(targets[e], weights[e]);
    cudaError_t ce;
    if ((ce = cudaGetDevice(&g->device)) != cudaSuccess) {
        set_last_cuda_error(ce, "cudaGetDevice", __FILE__, __LINE__);
        cudaGetLastError();
        return PPSP_ERR_CUDA;
    }
    {
        // plans take their descriptor arenas from the device's stream-ordered
        // pool; keep up to 1 GiB of freed pool memory mapped between plans
        // instead of returning it at every synchronisation (this process only)
        cudaMemPool_t pool;
        if (cudaDeviceGetDefaultMemPool(&pool, g->device) == cudaSuccess) {
            uint64_t keep = 1ull << 30;
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        }
        cudaGetLastError();
    }
    auto fail = [&](cudaError_t e, const char* what) {
        set_last_cuda_error(e, what, __FILE__, __LINE__);
        cudaGetLastError();
        cudaFree(g->d_off);
        cudaFree(g->d_edges);
        cudaFree(g->d_off_t);
        cudaFree(g->d_edges_t);
        cudaFree(g->d_pc);
        cudaFree(g->d_edges_pc);
        cudaFree(g->d_edges_t_pc);
        return e == cudaErrorMemoryAllocation ? PPSP_ERR_OOM : PPSP_ERR_CUDA;
    };
    if ((ce = cudaMalloc(&g->d_off, (n + 1) * 4)) != cudaSuccess) return fail(ce, "cudaMalloc(off)");
    if ((ce = cudaMalloc(&g->d_edges, std::max<u64>(1, m) * 8)) != cudaSuccess) return fail(ce, "cudaMalloc(edges)");
    if ((ce = cudaMemcpy(g->d_off, off32.data(), (n + 1) * 4, cudaMemcpyHostToDevice)) != cudaSuccess)
        return fail(ce, "cudaMemcpy(off)");
    if (m && (ce = cudaMemcpy(g->d_edges, ed.data(), m * 8, cudaMemcpyHostToDevice)) != cudaSuccess)
        return fail(ce, "cudaMemcpy(edges)");
    info.device_bytes = (n + 1) * 4 + m * 8;
    std::vector<uint2> edt;  // transpose records (directed graphs)
    if (!info.undirected) {
        // transpose (in-edges, each row sorted by source): backward searches
        // from a target and path walks of forward searches follow it
        std::vector<u32> offt(n + 1, 0);
        for (u64 e = 0; e < m; ++e) ++offt[targets[e] + 1];
        for (u64 v = 0; v < n; ++v) offt[v + 1] += offt[v];
        std::vector<u32> fill(offt.begin(), offt.end() - 1);
        edt.resize(m);
        for (u64 u = 0; u < n; ++u)
            for (u64 e = offsets[u]; e < offsets[u + 1]; ++e) edt[fill[targets[e]]++] = make_uint2((u32)u, weights[e]);
        if ((ce = cudaMalloc(&g->d_off_t, (n + 1) * 4)) != cudaSuccess) return fail(ce, "cudaMalloc(off_t)");
        if ((ce = cudaMalloc(&g->d_edges_t, std::max<u64>(1, m) * 8)) != cudaSuccess)
            return fail(ce, "cudaMalloc(edges_t)");
        if ((ce = cudaMemcpy(g->d_off_t, offt.data(), (n + 1) * 4, cudaMemcpyHostToDevice)) != cudaSuccess)
            return fail(ce, "cudaMemcpy(off_t)");
        if (m && (ce = cudaMemcpy(g->d_edges_t, edt.data(), m * 8, cudaMemcpyHostToDevice)) != cudaSuccess)
            return fail(ce, "cudaMemcpy(edges_t)");
        info.device_bytes += (n + 1) * 4 + m * 8;
    }
    if (coords && g->pot_scale > 0.0) {
        std::vector<int2> pc(n);
        for (u64 v = 0; v < n; ++v) pc[v] = make_int2((int)g->pc_host[2 * v], (int)g->pc_host[2 * v + 1]);
        if ((ce = cudaMalloc(&g->d_pc, n * 8)) != cudaSuccess) return fail(ce, "cudaMalloc(pc)");
        if ((ce = cudaMemcpy(g->d_pc, pc.data(), n * 8, cudaMemcpyHostToDevice)) != cudaSuccess)
            return fail(ce, "cudaMemcpy(pc)");
        info.device_bytes += n * 8;
    } else if (coords) {
        // coordinates given but no positive scale exists: the potential is 0
        std::vector<int2> pc(n, make_int2(0, 0));
        if ((ce = cudaMalloc(&g->d_pc, n * 8)) != cudaSuccess) return fail(ce, "cudaMalloc(pc)");
        if ((ce = cudaMemcpy(g->d_pc, pc.data(), n * 8, cudaMemcpyHostToDevice)) != cudaSuccess)
            return fail(ce, "cudaMemcpy(pc)");
        info.device_bytes += n * 8;
    }
    if (coords) {
        // the adjacency again as (target, weight, P(target)): a relaxation's
        // potential coordinates arrive with its edge record
        const bool scaled = g->pot_scale > 0.0;
        auto rec = [&](u32 v, u32 w) {
            return make_int4((int)v, (int)w, scaled ? (int)g->pc_host[2 * (u64)v] : 0,
                             scaled ? (int)g->pc_host[2 * (u64)v + 1] : 0);
        };
        std::vector<int4> e16(std::max<u64>(1, m));
        for (u64 e = 0; e < m; ++e) e16[e] = rec(targets[e], weights[e]);
        if ((ce = cudaMalloc(&g->d_edges_pc, std::max<u64>(1, m) * 16)) != cudaSuccess)
            return fail(ce, "cudaMalloc(edges_pc)");
        if (m && (ce = cudaMemcpy(g->d_edges_pc, e16.data(), m * 16, cudaMemcpyHostToDevice)) != cudaSuccess)
            return fail(ce, "cudaMemcpy(edges_pc)");
        info.device_bytes += m * 16;
        if (!info.undirected) {
            for (u64 e = 0; e < m; ++e) e16[e] = rec(edt[e].x, edt[e].y);
            if ((ce = cudaMalloc(&g->d_edges_t_pc, std::max<u64>(1, m) * 16)) != cudaSuccess)
                return fail(ce, "cudaMalloc(edges_t_pc)");
            if (m && (ce = cudaMemcpy(g->d_edges_t_pc, e16.data(), m * 16, cudaMemcpyHostToDevice)) != cudaSuccess)
                return fail(ce, "cudaMemcpy(edges_t_pc)");
            info.device_bytes += m * 16;
        }
    }
    *out = g.release();
    return PPSP_OK;
}

void ppsp_graph_destroy(ppsp_graph* g) {
    if (!g) return;
    cudaDeviceSynchronize();
    for (auto& kv : g->pool) cudaFree(kv.second->base);
    g->pool.clear();
    cudaFree(g->d_off);
    cudaFree(g->d_edges);
    cudaFree(g->d_off_t);
    cudaFree(g->d_edges_t);
    cudaFree(g->d_pc);
    cudaFree(g->d_edges_pc);
    cudaFree(g->d_edges_t_pc);
    cudaFree(g->d_scratch_u32);
    cudaFree(g->d_scratch_i64);
    cudaGetLastError();
    delete g;
}

ppsp_status ppsp_vertex_order(uint64_t n, const float* coords, uint32_t* perm_out) {
    if (!coords || !perm_out || n == 0 || n >= 0xFFFFFFFFull) return PPSP_ERR_INVALID_ARG;
    if (n == 1) {
        perm_out[0] = 0;
        return PPSP_OK;
    }
    std::vector<u32> perm, inv;
    if (!locality_order(n, coords, perm, inv)) return PPSP_ERR_UNSUPPORTED;
    memcpy(perm_out, perm.data(), n * sizeof(u32));
    return PPSP_OK;
}

ppsp_status ppsp_graph_get_info(const ppsp_graph* g, ppsp_graph_info* out) {
    if (!g || !out) return PPSP_ERR_INVALID_ARG;
    *out = g->info;
    return PPSP_OK;
}

ppsp_status ppsp_potential_coords(const ppsp_graph* g, int64_t* out) {
    if (!g || !out) return PPSP_ERR_INVALID_ARG;
    if (!g->info.has_coords) return PPSP_ERR_NO_COORDS;
    if (g->perm.empty()) {
        memcpy(out, g->pc_host.data(), 2 * g->n * sizeof(int64_t));
    } else {
        for (u64 v = 0; v < g->n; ++v) {  // caller order
            out[2 * v] = g->pc_host[2 * (u64)g->perm[v]];
            out[2 * v + 1] = g->pc_host[2 * (u64)g->perm[v] + 1];
        }
    }
    return PPSP_OK;
}

ppsp_status ppsp_potential_eval(ppsp_graph* g, uint32_t anchor, const uint32_t* vertices, uint64_t count,
                                int64_t* out) {
    if (!g || (count && (!vertices || !out))) return PPSP_ERR_INVALID_ARG;
    if (!g->info.has_coords) return PPSP_ERR_NO_COORDS;
    if (anchor >= g->n) return PPSP_ERR_INVALID_ARG;
    if (count == 0) return PPSP_OK;
    std::lock_guard<std::mutex> lk(g->mu);
    if (count > g->scratch_cap) {
        cudaFree(g->d_scratch_u32);
        cudaFree(g->d_scratch_i64);
        g->d_scratch_u32 = nullptr;
        g->d_scratch_i64 = nullptr;
        g->scratch_cap = 0;
        PPSP_CUDA_TRY(cudaMalloc(&g->d_scratch_u32, count * 4));
        PPSP_CUDA_TRY(cudaMalloc(&g->d_scratch_i64, count * 8));
        g->scratch_cap = count;
    }
    std::vector<u32> mapped;
    if (!g->perm.empty()) {  // device ids (an id out of range stays out of range: the kernel answers -1)
        mapped.resize(count);
        for (u64 k = 0; k < count; ++k) mapped[k] = vertices[k] < g->n ? g->perm[vertices[k]] : vertices[k];
        vertices = mapped.data();
        anchor = g->perm[anchor];
    }
    PPSP_CUDA_TRY(cudaMemcpy(g->d_scratch_u32, vertices, count * 4, cudaMemcpyHostToDevice));
    ppsp_status st = launch_potential_eval(g->dev(), anchor, g->d_scratch_u32, count, g->d_scratch_i64, 0);
    if (st != PPSP_OK) return st;
    PPSP_CUDA_TRY(cudaMemcpy(out, g->d_scratch_i64, count * 8, cudaMemcpyDeviceToHost));
    return PPSP_OK;
}

}  // extern "C"
