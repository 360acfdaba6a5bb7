// Allocation-free single BiDS query, for callers that cannot allocate device
// memory: code running inside a memory pool they do not own, under a strict
// no-allocation policy in a serving process, or where cudaMalloc would
// synchronise the device at a bad moment.  The caller passes the graph and the
// output in device memory it already has; every piece of scratch the search
// needs lives in one file-scope device array of fixed size.
//
// Limits and sharing rules:
//  * the array holds the state of one query on graphs of at most
//    PPSP_NOALLOC_MAX_N vertices (about 13 MB, held by every GPU that loads
//    the library until the process exits);
//  * every call uses the same array; calls that overlap on the GPU (from two
//    streams or two host threads) race and must not be issued;
//  * the first call on a device resolves the array's device address
//    (cudaGetSymbolAddress) and fills it;
//  * the search leaves the array clean (distances infinite, bitmaps zero), and
//    the per-call state is cleared at the start of every call.
#include <algorithm>
#include <mutex>

#include "graph_impl.h"

namespace ppsp {

namespace {

constexpr u32 NA_MAX_N = PPSP_NOALLOC_MAX_N;
constexpr u32 NA_FLAT = 2 * NA_MAX_N;          // two searches, interleaved
constexpr u32 NA_WORDS = NA_FLAT / 32;
constexpr u32 NA_QCAP = NA_FLAT / 8 + 4096;
constexpr u32 NA_TCAP = NA_FLAT / 4 + 4096;     // overflow falls back to a full reset
constexpr u32 NA_MAX_CTAS = 4096;

// byte offsets inside the scratch array (256-aligned)
constexpr size_t al(size_t x) { return (x + 255) & ~(size_t)255; }
constexpr size_t O_DIST = 0;
constexpr size_t O_BM0 = O_DIST + al((size_t)NA_FLAT * 4);
constexpr size_t O_BM1 = O_BM0 + al((size_t)NA_WORDS * 4);
constexpr size_t O_Q0 = O_BM1 + al((size_t)NA_WORDS * 4);
constexpr size_t O_Q1 = O_Q0 + al((size_t)NA_QCAP * 4);
constexpr size_t O_TOUCH = O_Q1 + al((size_t)NA_QCAP * 4);
constexpr size_t O_SLOTST = O_TOUCH + al((size_t)NA_TCAP * 4);
constexpr size_t O_GROUP = O_SLOTST + al(sizeof(SlotState));
constexpr size_t O_SEARCH = O_GROUP + al(sizeof(GroupDev));
constexpr size_t O_PART = O_SEARCH + al(2 * sizeof(SearchDev));
constexpr size_t O_QEDGE = O_PART + al(2 * sizeof(PartnerDev));
constexpr size_t O_MU = O_QEDGE + al(sizeof(QEdgeDev));
constexpr size_t O_MUMAX = O_MU + al(8);
constexpr size_t O_CTAT = O_MUMAX + al(2 * 8);
constexpr size_t O_TEAM = O_CTAT + al((size_t)NA_MAX_CTAS * 4);  // first, size, queue
constexpr size_t O_SLOTDEV = O_TEAM + al(3 * 4);
constexpr size_t O_QITEMS = O_SLOTDEV + al(sizeof(SlotDev));
constexpr size_t O_MAP = O_QITEMS + al(4);
constexpr size_t O_RUN = O_MAP + al(4);                         // cleared every call:
constexpr size_t O_QHEAD = O_RUN;                                 //   queue heads
constexpr size_t O_TSTATE = O_QHEAD + al(MAX_QUEUES * 4);         //   team state
constexpr size_t O_ERR = O_TSTATE + al(sizeof(TeamState));        //   error word
constexpr size_t O_CNT = O_ERR + al(4);                           //   counters
constexpr size_t O_WSUM = O_CNT + al(sizeof(EngineCounters));     //   weight sum
constexpr size_t O_END = O_WSUM + al(8);
constexpr size_t RUN_BYTES = O_END - O_RUN;
constexpr size_t NA_BYTES = O_END;

}  // namespace

static __device__ __align__(256) unsigned char g_noalloc_scratch[NA_BYTES];

namespace {

std::mutex g_na_mu;
constexpr int NA_MAX_DEV = 64;
unsigned char* g_na_addr[NA_MAX_DEV] = {nullptr};
bool g_na_dirty[NA_MAX_DEV] = {false};

// Restore the clean state: distances infinite, bitmaps, queues heads and
// slot state zero.
__global__ void na_fill_kernel(unsigned char* base) {
    u32* dist = reinterpret_cast<u32*>(base + O_DIST);
    u32* bm0 = reinterpret_cast<u32*>(base + O_BM0);
    u32* bm1 = reinterpret_cast<u32*>(base + O_BM1);
    for (u32 k = blockIdx.x * blockDim.x + threadIdx.x; k < NA_FLAT; k += gridDim.x * blockDim.x) dist[k] = ~0u;
    for (u32 k = blockIdx.x * blockDim.x + threadIdx.x; k < NA_WORDS; k += gridDim.x * blockDim.x) {
        bm0[k] = 0u;
        bm1[k] = 0u;
    }
    u32* st = reinterpret_cast<u32*>(base + O_SLOTST);
    for (u32 k = blockIdx.x * blockDim.x + threadIdx.x; k < sizeof(SlotState) / 4; k += gridDim.x * blockDim.x)
        st[k] = 0u;
}

// Sum of all edge weights (for the default Delta), into the scratch.
__global__ void na_weight_sum_kernel(const uint2* edges, u64 m, unsigned char* base) {
    u64 s = 0;
    for (u64 e = (u64)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += (u64)gridDim.x * blockDim.x) s += edges[e].y;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0 && s) atomicAdd(reinterpret_cast<unsigned long long*>(base + O_WSUM), s);
}

// Descriptors of one BiDS pair group run by one team of `grid` CTAs.
__global__ void na_setup_kernel(unsigned char* base, u32 s, u32 t, u64 m, u64 delta, u32 grid) {
    const u32 k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < grid) reinterpret_cast<u32*>(base + O_CTAT)[k] = 0u;
    if (k != 0) return;
    u64 d = delta;
    if (d == 0) {
        const u64 sum = *reinterpret_cast<const u64*>(base + O_WSUM);
        d = m ? (2 * sum + m) / (2 * m) : 1;  // round(sum / m)
        if (d == 0) d = 1;
    }
    GroupDev* G = reinterpret_cast<GroupDev*>(base + O_GROUP);
    G->sbeg = 0;
    G->scnt = 2;
    G->qbeg = 0;
    G->qcnt = 1;
    G->mode = GM_BIDIR;
    G->target = NONE;
    G->layout = PPSP_LAYOUT_INTERLEAVED;
    G->kshift = 1;
    G->delta = d;
    SearchDev* S = reinterpret_cast<SearchDev*>(base + O_SEARCH);
    S[0] = SearchDev{s, 0, 1, 0, s, 0, 0, 0};
    S[1] = SearchDev{t, 1, 1, 0, t, 1, 0, 0};
    PartnerDev* P = reinterpret_cast<PartnerDev*>(base + O_PART);
    P[0] = PartnerDev{1, 0};
    P[1] = PartnerDev{0, 0};
    *reinterpret_cast<QEdgeDev*>(base + O_QEDGE) = QEdgeDev{0, 1};
    u32* team = reinterpret_cast<u32*>(base + O_TEAM);
    team[0] = 0;      // first CTA
    team[1] = grid;   // size
    team[2] = 1;      // queue
    SlotDev* sd = reinterpret_cast<SlotDev*>(base + O_SLOTDEV);
    sd->dist = base + O_DIST;
    sd->bm[0] = reinterpret_cast<u32*>(base + O_BM0);
    sd->bm[1] = reinterpret_cast<u32*>(base + O_BM1);
    sd->q[0] = reinterpret_cast<u32*>(base + O_Q0);
    sd->q[1] = reinterpret_cast<u32*>(base + O_Q1);
    sd->touched = reinterpret_cast<u32*>(base + O_TOUCH);
    sd->memo = nullptr;
    sd->st = reinterpret_cast<SlotState*>(base + O_SLOTST);
    sd->flat_cap = NA_FLAT;
    sd->qcap = NA_QCAP;
    sd->tcap = NA_TCAP;
    *reinterpret_cast<u32*>(base + O_QITEMS) = 0u;         // the one group
    *reinterpret_cast<u32*>(base + O_MAP) = (s == t) ? NONE : 0u;
}

}  // namespace

}  // namespace ppsp

using namespace ppsp;

extern "C" ppsp_status ppsp_query_noalloc(const uint32_t* d_offsets, const uint32_t* d_edges, uint32_t n,
                                          uint64_t m, uint32_t s, uint32_t t, uint64_t delta,
                                          uint64_t* d_dist_out, void* stream) {
    if (!d_offsets || (m && !d_edges) || !d_dist_out) return PPSP_ERR_INVALID_ARG;
    if (n == 0 || n > NA_MAX_N || m >= 0xFFFFFFFFull || s >= n || t >= n) return PPSP_ERR_INVALID_ARG;
    // the kernels read offsets as 4-byte words, adjacency records as 8-byte
    // pairs and write the answer as one 8-byte word: a misaligned pointer
    // would fault on the device, so it is refused here
    if (((uintptr_t)d_offsets & 3u) || ((uintptr_t)d_edges & 7u) || ((uintptr_t)d_dist_out & 7u))
        return PPSP_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    std::lock_guard<std::mutex> lk(g_na_mu);
    int dev = 0;
    PPSP_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= NA_MAX_DEV) return PPSP_ERR_UNSUPPORTED;
    if (g_na_addr[dev] == nullptr) {
        // once per device: the array's device address (the host-side name is
        // only a stand-in), then the clean state
        void* p = nullptr;
        PPSP_CUDA_TRY(cudaGetSymbolAddress(&p, g_noalloc_scratch));
        if (p == nullptr) return PPSP_ERR_CUDA;
        g_na_addr[dev] = static_cast<unsigned char*>(p);
        g_na_dirty[dev] = true;
    }
    unsigned char* base = g_na_addr[dev];
    if (g_na_dirty[dev]) {
        na_fill_kernel<<<256, 256, 0, st>>>(base);
        PPSP_CUDA_TRY(cudaGetLastError());
        g_na_dirty[dev] = false;
    }
    int bpsm = 0, sms = 0;
    ppsp_status rs = engine_occupancy(32, 512, &bpsm, &sms);
    if (rs != PPSP_OK) return rs;
    u32 grid = (u32)std::min<long long>((long long)bpsm * sms, NA_MAX_CTAS);
    // the one team must span at least two CTAs: a one-CTA team would take the
    // bucketed path, whose overflow and far lists this scratch does not hold
    if (grid < 2) return PPSP_ERR_UNSUPPORTED;

    PPSP_CUDA_TRY(cudaMemsetAsync(base + O_RUN, 0, RUN_BYTES, st));
    if (delta == 0 && m) {
        na_weight_sum_kernel<<<152, 256, 0, st>>>(reinterpret_cast<const uint2*>(d_edges), m, base);
        PPSP_CUDA_TRY(cudaGetLastError());
    }
    na_setup_kernel<<<(grid + 255) / 256, 256, 0, st>>>(base, s, t, m, delta, grid);
    PPSP_CUDA_TRY(cudaGetLastError());

    EngineArgs a{};
    a.g.off = d_offsets;
    a.g.edges = reinterpret_cast<const uint2*>(d_edges);
    a.g.off_t = a.g.off;  // symmetric CSR: the transpose is the graph itself
    a.g.edges_t = a.g.edges;
    a.g.pc = nullptr;
    a.g.n = n;
    a.g.pot_shift = 0;
    a.g.m = (u32)m;
    a.groups = reinterpret_cast<const GroupDev*>(base + O_GROUP);
    a.searches = reinterpret_cast<const SearchDev*>(base + O_SEARCH);
    a.partners = reinterpret_cast<const PartnerDev*>(base + O_PART);
    a.qedges = reinterpret_cast<const QEdgeDev*>(base + O_QEDGE);
    a.mu = reinterpret_cast<u64*>(base + O_MU);
    a.mumax = reinterpret_cast<u64*>(base + O_MUMAX);
    a.cta_team = reinterpret_cast<const u32*>(base + O_CTAT);
    a.team_first = reinterpret_cast<const u32*>(base + O_TEAM);
    a.team_size = reinterpret_cast<const u32*>(base + O_TEAM) + 1;
    a.team_queue = reinterpret_cast<const u32*>(base + O_TEAM) + 2;
    a.tstate = reinterpret_cast<TeamState*>(base + O_TSTATE);
    a.slots = reinterpret_cast<SlotDev*>(base + O_SLOTDEV);
    a.queue_items[0] = reinterpret_cast<const u32*>(base + O_QITEMS);
    a.queue_items[1] = reinterpret_cast<const u32*>(base + O_QITEMS);
    a.queue_len[0] = 0;
    a.queue_len[1] = (s == t) ? 0u : 1u;
    a.queue_head = reinterpret_cast<u32*>(base + O_QHEAD);
    a.dense_den = 16;
    a.ring_cap = RING_CAP_DEFAULT;
    a.frontier = PPSP_FRONTIER_AUTO;
    a.debug = 0;
    a.spin_limit = 1ull << 26;
    a.err = reinterpret_cast<u32*>(base + O_ERR);
    a.counters = reinterpret_cast<EngineCounters*>(base + O_CNT);
    a.group_ns = nullptr;
    rs = launch_engine(a, 32, 512, grid, st);
    if (rs != PPSP_OK) {
        g_na_dirty[dev] = true;
        return rs;
    }
    rs = launch_scatter(reinterpret_cast<const u32*>(base + O_MAP), a.mu, 1, d_dist_out, st);
    if (rs != PPSP_OK) {
        g_na_dirty[dev] = true;  // the engine may have run: scrub before the next call
        return rs;
    }
    u32 err = 0;
    PPSP_CUDA_TRY(cudaMemcpyAsync(&err, base + O_ERR, 4, cudaMemcpyDeviceToHost, st));
    PPSP_CUDA_TRY(cudaStreamSynchronize(st));
    if (err) {
        g_na_dirty[dev] = true;
        if (err & ERRB_OVERFLOW) return PPSP_ERR_OVERFLOW;
        if (err & ERRB_TIMEOUT) return PPSP_ERR_TIMEOUT;
        return PPSP_ERR_CUDA;
    }
    return PPSP_OK;
}
