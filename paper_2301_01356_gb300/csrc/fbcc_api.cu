// libfbcc C ABI: workspace management, the per-solve driver (optionally replayed
// from a captured CUDA graph) and format validation.
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <mutex>
#include <vector>
#include <new>

#include "fbcc_internal.cuh"

using namespace fbcc;

namespace {

thread_local char g_cuda_err[256] = "";

fbcc_status cuda_fail(cudaError_t e, const char *where)
{
    snprintf(g_cuda_err, sizeof(g_cuda_err), "%s: %s", where, cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? FBCC_E_OOM : FBCC_E_CUDA;
}

#define API_CK(x, where)                                   \
    do {                                                   \
        cudaError_t e_ = (x);                              \
        if (e_ != cudaSuccess) return cuda_fail(e_, where); \
    } while (0)

constexpr int kMinStride = 8;

struct GraphKey {
    const void *off, *adj, *edge_bcc, *bcc_head, *is_ap, *is_bridge;
    const void *vtx_base, *arc_base, *bstats;
    int64_t n, m;
    int offsets_64, G;
    fbcc_config cfg;
    bool operator==(const GraphKey &o) const { return memcmp(this, &o, sizeof(*this)) == 0; }
};

// Lays out every workspace array in one allocation (256-byte aligned pieces).
struct Carver {
    char *base;
    size_t used = 0;
    template <typename T>
    T *take(int64_t count)
    {
        size_t at = (used + 255) & ~size_t(255);
        used = at + size_t(count > 0 ? count : 1) * sizeof(T);
        return base ? reinterpret_cast<T *>(base + at) : nullptr;
    }
};

size_t batch_stage_bytes(int64_t N, int64_t Z, int32_t G);

int64_t st_levels_for(int64_t tiles)
{
    int64_t l = 1;
    while ((1ll << l) <= tiles) ++l;
    return l;
}

size_t carve(Dev &d, char *base, int64_t N, int64_t Z)
{
    if (N < 1) N = 1;
    if (Z < 1) Z = 1;
    Carver c{base};
    d.n_max = N;
    d.nnz_max = Z;
    // level-1 rulers: a head per tour (a tour spans >= 2 vertices) plus one per stride
    d.ruler_max = N / 2 + ceil_div(2 * N, kMinStride) + 2;
    d.rmq_tiles_max = ceil_div(N, kRmqTile);
    d.st_levels = st_levels_for(d.rmq_tiles_max);
    const int64_t words = ceil_div(Z, 32) + 1;
    int64_t scan_items = 2 * N + 1;
    if (words + 1 > scan_items) scan_items = words + 1;
    // arrays that live through the whole solve
    d.err = c.take<int>(4);
    d.counters = c.take<long long>(16);
    d.scan_status = c.take<uint64_t>(ceil_div(scan_items, kTile) + 2);
    d.stats = c.take<fbcc_stats>(1);
    d.uf = c.take<int32_t>(N);
    d.tile_v = c.take<int32_t>(ceil_div(Z, kWTile) + 2);
    d.fp = c.take<int2>(N);
    d.parc = c.take<int32_t>(N);
    d.lastp = c.take<int32_t>(N);
    d.dirb = c.take<uint8_t>(ceil_div(Z, 8) + 8);
    d.bigb = c.take<uint32_t>(ceil_div(N, 32) + 2);
    d.ord = c.take<int32_t>(N);
    d.porig = c.take<int32_t>(N);
    d.w1 = c.take<int32_t>(N);
    d.w2 = c.take<int32_t>(N);
    // First-CC and rooting scratch; the later phases reuse the same bytes
    const size_t shared_from = c.used;
    d.te_u = c.take<int32_t>(N);
    d.te_v = c.take<int32_t>(N);
    d.te_a = c.take<int32_t>(N);
    d.hub_cap = Z / kHubMinDeg + 1 < kHubCap ? Z / kHubMinDeg + 1 : kHubCap;
    d.hubidx = c.take<int32_t>(N);            // (set by First-CC: not in the local-first list's space)
    d.hubvert = c.take<int32_t>(d.hub_cap);
    const size_t xl_from = c.used;
    d.te2_u = c.take<int32_t>(N);
    d.te2_v = c.take<int32_t>(N);
    d.te2_a = c.take<int32_t>(N);
    d.lhead = c.take<int32_t>(N);
    d.nxt = c.take<int32_t>(2 * N);
    d.rhead = c.take<uint8_t>(d.ruler_max);
    d.link = c.take<int2>(2 * N);
    d.relem = c.take<int32_t>(d.ruler_max);
    d.rlen = c.take<int32_t>(d.ruler_max);
    d.rnx1 = c.take<int32_t>(d.ruler_max);
    d.sd1 = c.take<int32_t>(d.ruler_max);
    {
        // level k holds the heads of the multi-node lists of level k-1 (at most the
        // stride samples of level k-2) plus one node in kStride2 of level k-1
        int64_t below = d.ruler_max, below2 = ceil_div(2 * N, kMinStride);
        for (int k = 0; k < kRankLevels; ++k) {
            RankLevel &v = d.lv[k];
            v.cap = below2 + ceil_div(below, kStride2) + 2;
            v.l = c.take<int2>(below);
            v.relem = c.take<int32_t>(v.cap);
            v.owner = c.take<int32_t>(below);
            v.offs = c.take<int32_t>(below);
            v.next = c.take<int32_t>(v.cap);
            v.w = c.take<int32_t>(v.cap);
            v.head = c.take<uint8_t>(v.cap);
            v.sd = c.take<int32_t>(v.cap);
            below2 = ceil_div(below, kStride2);
            below = v.cap;
        }
        d.top_tmp_cap = below;
        for (int i = 0; i < 4; ++i) d.top_tmp[i] = c.take<int32_t>(below);
    }
    d.csize = c.take<int32_t>(N + 1);
    d.vbase = c.take<int32_t>(N + 1);
    d.rec = c.take<int2>(2 * N);
    d.hubhead = c.take<int32_t>(d.hub_cap * kHubSub);
    d.hubnext = c.take<int32_t>(d.hub_cap * kHubSub);
    size_t rooting_end = c.used;
    {
        const size_t at = (xl_from + 255) & ~size_t(255);
        // First-CC's scratch in this space (LDD: three arrays of N ids and a byte per
        // vertex, counters and at least a few hundred list entries) always fits
        const size_t ldd_min = 13 * (size_t)N + 16384;
        if (rooting_end - at < ldd_min) rooting_end = c.used = at + ldd_min;
        d.xl = base ? reinterpret_cast<int2 *>(base + at) : nullptr;
        d.xl_cap = (int64_t)((rooting_end - at) / sizeof(int2));
    }
    // tagging, Last-CC and output scratch (alive only after rooting has finished)
    c.used = shared_from;
    d.pmm = c.take<int2>(N);
    d.tmin = c.take<int32_t>(d.st_levels * d.rmq_tiles_max);
    d.tmax = c.take<int32_t>(d.st_levels * d.rmq_tiles_max);
    d.vbits = c.take<uint8_t>(N);
    d.low = c.take<int32_t>(N);
    d.high = c.take<int32_t>(N);
    d.lp = c.take<int32_t>(N);
    d.ext = c.take<uint8_t>(N);
    d.qlist = c.take<int32_t>(N);
    d.first4 = c.take<int32_t>(N);
    d.fl = c.take<int2>(N);
    d.cr = c.take<int2>(N);
    d.lab = c.take<int32_t>(N);
    d.smin = c.take<int32_t>(N);
    d.nh = c.take<int32_t>(N);
    d.key = c.take<unsigned long long>(N);
    d.scanv = c.take<uint8_t>(N);
    d.klist_cap = N + ceil_div(Z, kKeyChunk) + 2;
    d.klist = c.take<int2>(d.klist_cap);
    d.kmin = c.take<int32_t>(N);
    d.key_bits = c.take<uint32_t>(words);
    d.key_pre = c.take<int32_t>(words + 1);
    d.rank = c.take<int32_t>(N);
    d.word = c.take<int32_t>(N);
    d.hoff = c.take<int32_t>(N + 1);
    d.hfill = c.take<int32_t>(N);
    d.hlist = c.take<int32_t>(N);
    if (c.used < rooting_end) c.used = rooting_end;
    return c.used + 256;
}

}  // namespace

struct fbcc_workspace {
    Dev d;
    void *slab = nullptr;
    size_t bytes = 0;
    fbcc_config cfg;
    cudaStream_t cap = nullptr;        // private stream used for graph capture
    cudaGraphExec_t exec = nullptr;
    GraphKey key;
    bool have_key = false;
    // staging buffers of fbcc_solve_host (allocated on first use)
    void *stage = nullptr;
    size_t stage_bytes = 0;
    // global offsets/adjacency and per-graph bases of fbcc_solve_batch (first use)
    void *bstage = nullptr;
    size_t bstage_bytes = 0;
    bool caller_mem = false;   // slab and batch staging are the caller's memory (fbcc_workspace_create_in)
    Prof prof;             // per-kernel events of profiled solves
    int64_t last_n = -1;   // vertices of the last solve (-1: none yet)
    bool qindex = false;   // the query index of the last solve has been enqueued
};

static fbcc_config default_config()
{
    fbcc_config c;
    c.ruler_stride = 16;
    c.cc_sample = 0;
    c.grid_ctas = 0;
    c.use_graph = 1;
    c.profile = 0;
    c.chase_chains = 1;
    c.cc_local = 0;
    c.lcc_sample = 0;
    c.rank_variant = 0;
    c.cc_order = 0;
    c.hub_deg = 0;
    c.cc_ldd = 0;
    return c;
}

static int device_grid(const fbcc_config &c)
{
    if (c.grid_ctas > 0) return c.grid_ctas;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return (sms > 0 ? sms : 1) * (c.grid_ctas < 0 ? -c.grid_ctas : 8);
}

extern "C" {

size_t fbcc_workspace_bytes(int64_t n, int64_t nnz)
{
    Dev d;
    return carve(d, nullptr, n, nnz);
}

fbcc_status fbcc_workspace_create(int64_t n_max, int64_t nnz_max, fbcc_workspace **ws)
{
    if (!ws || n_max < 0 || nnz_max < 0 || n_max >= (1ll << 30) || nnz_max >= (1ll << 40)) return FBCC_E_INVALID;
    *ws = nullptr;
    fbcc_workspace *w = new (std::nothrow) fbcc_workspace();
    if (!w) return FBCC_E_OOM;
    w->cfg = default_config();
    w->bytes = carve(w->d, nullptr, n_max, nnz_max);
    cudaError_t e = cudaMalloc(&w->slab, w->bytes);
    if (e != cudaSuccess) {
        delete w;
        return cuda_fail(e, "cudaMalloc(workspace)");
    }
    carve(w->d, static_cast<char *>(w->slab), n_max, nnz_max);
    e = prepare_rooting();
    if (e != cudaSuccess) {
        cudaFree(w->slab);
        delete w;
        return cuda_fail(e, "cudaFuncSetAttribute");
    }
    *ws = w;
    return FBCC_OK;
}

fbcc_status fbcc_workspace_create_in(void *mem, size_t bytes, int64_t n_max, int64_t nnz_max, int32_t max_graphs,
                                     fbcc_workspace **ws)
{
    if (!ws) return FBCC_E_INVALID;
    *ws = nullptr;
    if (!mem || ((uintptr_t)mem & 255) || n_max < 0 || nnz_max < 0 || n_max >= (1ll << 30) ||
        nnz_max >= (1ll << 40) || max_graphs < 0)
        return FBCC_E_INVALID;
    Dev probe;
    // carve() reports the slab's last byte plus 256: the staging starts 256-aligned
    // below that, and the total never exceeds fbcc_batch_workspace_bytes
    const size_t wb = carve(probe, nullptr, n_max, nnz_max) & ~size_t(255);
    const size_t bb = max_graphs > 0 ? batch_stage_bytes(n_max, nnz_max, max_graphs) : 0;
    if (bytes < wb + bb) return FBCC_E_WORKSPACE;
    fbcc_workspace *w = new (std::nothrow) fbcc_workspace();
    if (!w) return FBCC_E_OOM;
    w->cfg = default_config();
    w->caller_mem = true;
    w->slab = mem;
    w->bytes = wb;
    carve(w->d, static_cast<char *>(mem), n_max, nnz_max);
    if (bb) {
        w->bstage = static_cast<char *>(mem) + wb;
        w->bstage_bytes = bb;
    }
    const cudaError_t e = prepare_rooting();
    if (e != cudaSuccess) {
        delete w;
        return cuda_fail(e, "cudaFuncSetAttribute");
    }
    *ws = w;
    return FBCC_OK;
}

void fbcc_workspace_destroy(fbcc_workspace *ws)
{
    if (!ws) return;
    if (!ws->caller_mem) cudaDeviceSynchronize();
    if (ws->exec) cudaGraphExecDestroy(ws->exec);
    if (ws->cap) cudaStreamDestroy(ws->cap);
    if (ws->prof.ready)
        for (int i = 0; i <= kProfMax; ++i) cudaEventDestroy(ws->prof.ev[i]);
    if (!ws->caller_mem) {
        cudaFree(ws->slab);
        cudaFree(ws->stage);
        cudaFree(ws->bstage);
    }
    delete ws;
}

fbcc_status fbcc_workspace_configure(fbcc_workspace *ws, const fbcc_config *cfg)
{
    if (!ws) return FBCC_E_INVALID;
    fbcc_config c = default_config();
    if (cfg) {
        if (cfg->ruler_stride) {
            if (cfg->ruler_stride < kMinStride || (cfg->ruler_stride & (cfg->ruler_stride - 1))) return FBCC_E_INVALID;
            c.ruler_stride = cfg->ruler_stride;
        }
        if (cfg->cc_sample < 0 || cfg->grid_ctas < -64) return FBCC_E_INVALID;
        c.cc_sample = cfg->cc_sample;
        c.grid_ctas = cfg->grid_ctas;
        if (cfg->use_graph) c.use_graph = cfg->use_graph;
        c.profile = cfg->profile > 0;
        if (cfg->cc_local) {
            if (cfg->cc_local < 1024 || cfg->cc_local > 16384 || (cfg->cc_local & (cfg->cc_local - 1)))
                return FBCC_E_INVALID;
            cudaError_t e = prepare_cc_local(cfg->cc_local);
            if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute");
            c.cc_local = cfg->cc_local;
        }
        if (cfg->lcc_sample < 0 || cfg->lcc_sample > 4) return FBCC_E_INVALID;
        c.lcc_sample = cfg->lcc_sample;
        if (cfg->rank_variant < 0 || cfg->rank_variant > 1) return FBCC_E_INVALID;
        c.rank_variant = cfg->rank_variant;
        if (cfg->cc_order < 0 || cfg->cc_order > 1) return FBCC_E_INVALID;
        c.cc_order = cfg->cc_order;
        if (cfg->hub_deg < -1 || (cfg->hub_deg > 0 && cfg->hub_deg < kHubMinDeg)) return FBCC_E_INVALID;
        c.hub_deg = cfg->hub_deg;
        if (cfg->cc_ldd < 0 || cfg->cc_ldd > 64) return FBCC_E_INVALID;
        c.cc_ldd = cfg->cc_ldd;
        if (cfg->chase_chains) {
            if (cfg->chase_chains != 1 && cfg->chase_chains != 2 && cfg->chase_chains != 4) return FBCC_E_INVALID;
            c.chase_chains = cfg->chase_chains;
        }
    }
    ws->cfg = c;
    return FBCC_OK;
}

const char *fbcc_status_string(fbcc_status s)
{
    switch (s) {
    case FBCC_OK: return "ok";
    case FBCC_E_INVALID: return "invalid argument";
    case FBCC_E_NOT_SIMPLE: return "graph is not a simple symmetric sorted CSR";
    case FBCC_E_OOM: return "out of device memory";
    case FBCC_E_CUDA: return "CUDA runtime error";
    case FBCC_E_ITER_LIMIT: return "a bounded device loop reached its iteration cap";
    case FBCC_E_WORKSPACE: return "graph exceeds the workspace size";
    }
    return "unknown status";
}

const char *fbcc_last_cuda_error(void) { return g_cuda_err; }

}  // extern "C"

// ---------------------------------------------------------------------------
// The solve itself
// ---------------------------------------------------------------------------
namespace {

__global__ void k_finish(const int *err, fbcc_stats *stats)
{
    stats->device_status = !*err ? FBCC_OK : (*err & kErrIndex) ? FBCC_E_INVALID : FBCC_E_ITER_LIMIT;
}

// Batch input: global int64 offsets and global neighbour ids from the packed
// per-graph local CSR (one thread per vertex; its list is translated in place).
__global__ void k_batch_globalize(int32_t G, const int64_t *__restrict__ vtx_base,
                                  const int64_t *__restrict__ arc_base, const int32_t *__restrict__ loff,
                                  const int32_t *__restrict__ ladj, int64_t n, int64_t *goff, int32_t *gadj)
{
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        const int32_t g = graph_of(vtx_base, G, v);
        const int64_t vb = vtx_base[g], ab = arc_base[g];
        const int64_t b = ab + loff[v];
        const int64_t e = (v + 1 < vtx_base[g + 1]) ? ab + loff[v + 1] : arc_base[g + 1];
        goff[v] = b;
        for (int64_t a = b; a < e; ++a) gadj[a] = ladj[a] + (int32_t)vb;
        if (v == n - 1) goff[n] = arc_base[G];
    }
}

template <typename OffT>
cudaError_t enqueue_solve(fbcc_workspace *ws, const OffT *off, const int32_t *adj, int64_t n, int64_t m,
                          int32_t *edge_bcc, int32_t *bcc_head, uint8_t *is_ap, uint8_t *is_bridge, cudaStream_t s,
                          const Batch &B = Batch(), const TvScratch *tv = nullptr)
{
    const Dev &d = ws->d;
    const int64_t nnz = 2 * m;
    Launch L{s, device_grid(ws->cfg)};
    if (ws->cfg.profile) {
        L.prof = &ws->prof;
        ws->prof.count = 0;
        cudaEventRecord(ws->prof.ev[0], s);
    }
    const bool vec = ((uintptr_t)adj & 15) == 0;
    cudaError_t e;
#define CK(x) do { e = (x); if (e != cudaSuccess) return e; } while (0)
    CK(cudaMemsetAsync(d.err, 0, sizeof(int), s));
    CK(cudaMemsetAsync(d.stats, 0, sizeof(fbcc_stats), s));
    if (n > 0) {
        const int hub_deg = ws->cfg.hub_deg == 0 ? kHubDeg : ws->cfg.hub_deg;   // -1: no hubs
        CK(launch_first_cc<OffT>(d, off, adj, n, nnz, ws->cfg.cc_sample, ws->cfg.cc_local, ws->cfg.cc_ldd,
                                 hub_deg, vec, L));
        CK(launch_rooting<OffT>(d, off, adj, n, nnz, ws->cfg.ruler_stride, ws->cfg.chase_chains,
                                ws->cfg.rank_variant, ws->cfg.cc_order, hub_deg > 0, L));
        CK(launch_tagging<OffT>(d, off, adj, n, nnz, vec, ws->cfg.profile != 0, L));
        if (tv) CK(launch_tv_connect<OffT>(d, off, adj, n, nnz, *tv, vec, L));
        else CK(launch_last_cc<OffT>(d, off, adj, n, nnz, ws->cfg.lcc_sample, vec, L));
        CK(launch_outputs<OffT>(d, off, adj, n, nnz, vec, hub_deg > 0, edge_bcc, bcc_head, is_ap, is_bridge, B,
                                L));
    }
    k_finish<<<1, 1, 0, s>>>(d.err, d.stats);
    L.mark("k_finish");
#undef CK
    return cudaGetLastError();
}

fbcc_status check_args(const void *off, const int32_t *adj, int64_t n, int64_t m, const void *edge_bcc,
                       const void *bcc_head, const void *is_ap, const void *is_bridge, fbcc_workspace *ws)
{
    if (!ws || n < 0 || m < 0) return FBCC_E_INVALID;
    if (n >= (1ll << 30)) return FBCC_E_INVALID;
    if (n > ws->d.n_max || m > ws->d.nnz_max / 2) return FBCC_E_WORKSPACE;
    if (m > 0 && n < 2) return FBCC_E_INVALID;
    if (n > 0 && (!off || !is_ap || !bcc_head)) return FBCC_E_INVALID;
    if (m > 0 && (!adj || !edge_bcc || !is_bridge)) return FBCC_E_INVALID;
    return FBCC_OK;
}

fbcc_status solve_device(const void *off, int offsets_64, const int32_t *adj, int64_t n, int64_t m,
                         int32_t *edge_bcc, int32_t *bcc_head, uint8_t *is_ap, uint8_t *is_bridge, fbcc_stats *stats,
                         fbcc_workspace *ws, cudaStream_t s, const Batch &B = Batch(),
                         const int32_t *loff = nullptr, const int32_t *ladj = nullptr)
{
    // A batch first translates its packed local CSR into global ids (in the graph too).
    auto enqueue = [&](cudaStream_t q) -> cudaError_t {
        if (B.G > 0 && n > 0) {
            k_batch_globalize<<<device_grid(ws->cfg), kThreads, 0, q>>>(B.G, B.vtx_base, B.arc_base, loff, ladj, n,
                                                                         (int64_t *)off, (int32_t *)adj);
            // (in a profiled solve this kernel's time is folded into the first phase's first mark)
            cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) return e;
        }
        return offsets_64
            ? enqueue_solve<int64_t>(ws, (const int64_t *)off, adj, n, m, edge_bcc, bcc_head, is_ap, is_bridge, q, B)
            : enqueue_solve<int32_t>(ws, (const int32_t *)off, adj, n, m, edge_bcc, bcc_head, is_ap, is_bridge, q, B);
    };
    ws->last_n = n;
    ws->qindex = false;
    if (ws->cfg.profile && !ws->prof.ready) {
        for (int i = 0; i <= kProfMax; ++i) API_CK(cudaEventCreate(&ws->prof.ev[i]), "cudaEventCreate");
        ws->prof.ready = true;
    }
    if (ws->cfg.use_graph > 0 && !ws->cfg.profile) {
        GraphKey k;
        memset(&k, 0, sizeof(k));
        k.off = off; k.adj = adj; k.edge_bcc = edge_bcc; k.bcc_head = bcc_head; k.is_ap = is_ap;
        k.is_bridge = is_bridge; k.n = n; k.m = m; k.offsets_64 = offsets_64; k.cfg = ws->cfg;
        k.vtx_base = B.vtx_base; k.arc_base = loff; k.bstats = B.stats; k.G = B.G;
        if (B.G > 0) k.adj = ladj;
        if (!ws->have_key || !(ws->key == k)) {
            if (ws->exec) {
                cudaGraphExecDestroy(ws->exec);
                ws->exec = nullptr;
            }
            ws->have_key = false;
            if (!ws->cap) API_CK(cudaStreamCreateWithFlags(&ws->cap, cudaStreamNonBlocking), "cudaStreamCreate");
            API_CK(cudaStreamBeginCapture(ws->cap, cudaStreamCaptureModeThreadLocal), "cudaStreamBeginCapture");
            cudaError_t e = enqueue(ws->cap);
            cudaGraph_t g = nullptr;
            cudaError_t e2 = cudaStreamEndCapture(ws->cap, &g);
            if (e != cudaSuccess) {
                if (g) cudaGraphDestroy(g);
                return cuda_fail(e, "enqueue (capture)");
            }
            API_CK(e2, "cudaStreamEndCapture");
            e = cudaGraphInstantiate(&ws->exec, g, 0);
            cudaGraphDestroy(g);
            API_CK(e, "cudaGraphInstantiate");
            ws->key = k;
            ws->have_key = true;
        }
        API_CK(cudaGraphLaunch(ws->exec, s), "cudaGraphLaunch");
    } else {
        API_CK(enqueue(s), "enqueue");
    }
    if (stats) API_CK(cudaMemcpyAsync(stats, ws->d.stats, sizeof(fbcc_stats), cudaMemcpyDeviceToHost, s), "stats copy");
    return FBCC_OK;
}

size_t batch_stage_bytes(int64_t N, int64_t Z, int32_t G)
{
    Carver c{nullptr};
    c.take<int64_t>(N + 1);
    c.take<int32_t>(Z);
    c.take<int64_t>((int64_t)G + 1);
    return c.used + 256;
}

}  // namespace

extern "C" {

size_t fbcc_tv_scratch_bytes(int64_t n, int64_t nnz)
{
    return tv_scratch_bytes(n < 0 ? 0 : n, nnz < 0 ? 0 : nnz);
}

fbcc_status fbcc_solve_tv(const void *csr_offsets, int offsets_64, const int32_t *csr_adj, int64_t n, int64_t m,
                          int32_t *edge_bcc, int32_t *bcc_head, uint8_t *is_ap, uint8_t *is_bridge,
                          fbcc_stats *stats, void *scratch, size_t scratch_bytes, fbcc_workspace *ws, void *stream)
{
    fbcc_status st = check_args(csr_offsets, csr_adj, n, m, edge_bcc, bcc_head, is_ap, is_bridge, ws);
    if (st != FBCC_OK) return st;
    if (n + 2 * m >= INT32_MAX) return FBCC_E_INVALID;   // skeleton vertices are 32-bit ids
    if (!scratch || ((uintptr_t)scratch & 255)) return FBCC_E_INVALID;
    if (scratch_bytes < tv_scratch_bytes(n, 2 * m)) return FBCC_E_WORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    ws->last_n = n;
    ws->qindex = false;
    if (ws->cfg.profile && !ws->prof.ready) {
        for (int i = 0; i <= kProfMax; ++i) API_CK(cudaEventCreate(&ws->prof.ev[i]), "cudaEventCreate");
        ws->prof.ready = true;
    }
    const TvScratch tv{scratch, scratch_bytes};
    API_CK(offsets_64 ? enqueue_solve<int64_t>(ws, (const int64_t *)csr_offsets, csr_adj, n, m, edge_bcc, bcc_head,
                                               is_ap, is_bridge, s, Batch(), &tv)
                      : enqueue_solve<int32_t>(ws, (const int32_t *)csr_offsets, csr_adj, n, m, edge_bcc, bcc_head,
                                               is_ap, is_bridge, s, Batch(), &tv),
           "enqueue (Tarjan-Vishkin)");
    if (stats) API_CK(cudaMemcpyAsync(stats, ws->d.stats, sizeof(fbcc_stats), cudaMemcpyDeviceToHost, s), "stats copy");
    return FBCC_OK;
}

fbcc_status fbcc_solve(const void *csr_offsets, int offsets_64, const int32_t *csr_adj, int64_t n, int64_t m,
                       int32_t *edge_bcc, int32_t *bcc_head, uint8_t *is_ap, uint8_t *is_bridge, fbcc_stats *stats,
                       fbcc_workspace *ws, void *stream)
{
    fbcc_status st = check_args(csr_offsets, csr_adj, n, m, edge_bcc, bcc_head, is_ap, is_bridge, ws);
    if (st != FBCC_OK) return st;
    return solve_device(csr_offsets, offsets_64, csr_adj, n, m, edge_bcc, bcc_head, is_ap, is_bridge, stats, ws,
                        (cudaStream_t)stream);
}

}  // extern "C"

namespace {

// The host entry points: inputs copied into the workspace's staging buffers,
// the solve, the outputs copied back; `wait` synchronises and trims bcc_head to
// n_bcc entries.
fbcc_status solve_host(const void *csr_offsets, int offsets_64, const int32_t *csr_adj, int64_t n, int64_t m,
                       int32_t *edge_bcc, int32_t *bcc_head, uint8_t *is_ap, uint8_t *is_bridge, fbcc_stats *stats,
                       fbcc_workspace *ws, cudaStream_t s, bool wait)
{
    fbcc_status st = check_args(csr_offsets, csr_adj, n, m, edge_bcc, bcc_head, is_ap, is_bridge, ws);
    if (st != FBCC_OK) return st;
    if (ws->caller_mem) return FBCC_E_INVALID;   // its staging would be an allocation
    const int64_t N = ws->d.n_max, Z = ws->d.nnz_max;
    if (!ws->stage) {
        ws->stage_bytes = size_t(N + 1) * 8 + size_t(Z) * 4 + size_t(Z) * 4 + size_t(N) * 4 + size_t(N) + size_t(Z) + 5 * 256;
        API_CK(cudaMalloc(&ws->stage, ws->stage_bytes), "cudaMalloc(staging)");
    }
    Carver c{static_cast<char *>(ws->stage)};
    void *d_off = c.take<int64_t>(N + 1);
    int32_t *d_adj = c.take<int32_t>(Z);
    int32_t *d_eb = c.take<int32_t>(Z);
    int32_t *d_bh = c.take<int32_t>(N);
    uint8_t *d_ap = c.take<uint8_t>(N);
    uint8_t *d_br = c.take<uint8_t>(Z);
    const int64_t nnz = 2 * m;
    const size_t ob = size_t(n + 1) * (offsets_64 ? 8 : 4);
    if (n > 0) API_CK(cudaMemcpyAsync(d_off, csr_offsets, ob, cudaMemcpyHostToDevice, s), "H2D offsets");
    if (nnz > 0) API_CK(cudaMemcpyAsync(d_adj, csr_adj, nnz * 4, cudaMemcpyHostToDevice, s), "H2D adj");
    fbcc_stats hs;
    st = solve_device(d_off, offsets_64, d_adj, n, m, d_eb, d_bh, d_ap, d_br, wait ? &hs : stats, ws, s);
    if (st != FBCC_OK) return st;
    if (nnz > 0) {
        API_CK(cudaMemcpyAsync(edge_bcc, d_eb, nnz * 4, cudaMemcpyDeviceToHost, s), "D2H edge_bcc");
        API_CK(cudaMemcpyAsync(is_bridge, d_br, nnz, cudaMemcpyDeviceToHost, s), "D2H is_bridge");
    }
    if (n > 0) API_CK(cudaMemcpyAsync(is_ap, d_ap, n, cudaMemcpyDeviceToHost, s), "D2H is_ap");
    if (!wait) {
        if (n > 0) API_CK(cudaMemcpyAsync(bcc_head, d_bh, n * 4, cudaMemcpyDeviceToHost, s), "D2H bcc_head");
        return FBCC_OK;
    }
    API_CK(cudaStreamSynchronize(s), "cudaStreamSynchronize");
    if (hs.n_bcc > 0)
        API_CK(cudaMemcpy(bcc_head, d_bh, hs.n_bcc * 4, cudaMemcpyDeviceToHost), "D2H bcc_head");
    if (stats) *stats = hs;
    return FBCC_OK;
}

}  // namespace

extern "C" fbcc_status fbcc_solve_host(const void *csr_offsets, int offsets_64, const int32_t *csr_adj, int64_t n,
                                       int64_t m, int32_t *edge_bcc, int32_t *bcc_head, uint8_t *is_ap,
                                       uint8_t *is_bridge, fbcc_stats *stats, fbcc_workspace *ws, void *stream)
{
    return solve_host(csr_offsets, offsets_64, csr_adj, n, m, edge_bcc, bcc_head, is_ap, is_bridge, stats, ws,
                      (cudaStream_t)stream, true);
}

extern "C" fbcc_status fbcc_solve_host_async(const void *csr_offsets, int offsets_64, const int32_t *csr_adj,
                                             int64_t n, int64_t m, int32_t *edge_bcc, int32_t *bcc_head,
                                             uint8_t *is_ap, uint8_t *is_bridge, fbcc_stats *stats,
                                             fbcc_workspace *ws, void *stream)
{
    return solve_host(csr_offsets, offsets_64, csr_adj, n, m, edge_bcc, bcc_head, is_ap, is_bridge, stats, ws,
                      (cudaStream_t)stream, false);
}

// ---------------------------------------------------------------------------
// Validation (warp per vertex)
// ---------------------------------------------------------------------------
namespace {

template <typename OffT>
__global__ void k_validate(const OffT *__restrict__ off, const int32_t *__restrict__ adj, int64_t n, int64_t nnz,
                           int *bad)
{
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x / 32);
    for (int64_t v = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / 32; v < n; v += warps) {
        const int64_t b = off[v], e = off[v + 1];
        if (lane == 0 && (e < b || b < 0 || e > nnz)) atomicOr(bad, 1);
        if (e < b || b < 0 || e > nnz) continue;
        for (int64_t a = b + lane; a < e; a += 32) {
            const int32_t w = adj[a];
            if (w < 0 || w >= n) { atomicOr(bad, 1); continue; }
            if (w == v || (a > b && adj[a - 1] >= w)) { atomicOr(bad, 2); continue; }
            int64_t lo = off[w], hi = off[w + 1];
            if (lo < 0 || hi > nnz || hi < lo) { atomicOr(bad, 1); continue; }
            while (lo < hi) {
                int64_t mid = (lo + hi) >> 1;
                if (adj[mid] < v) lo = mid + 1; else hi = mid;
            }
            if (lo >= off[w + 1] || adj[lo] != v) atomicOr(bad, 2);
        }
    }
}

}  // namespace

extern "C" fbcc_status fbcc_validate(const void *csr_offsets, int offsets_64, const int32_t *csr_adj, int64_t n,
                                     int64_t m, fbcc_workspace *ws, void *stream)
{
    if (!ws || n < 0 || m < 0 || (n > 0 && !csr_offsets) || (m > 0 && !csr_adj)) return FBCC_E_INVALID;
    if (n > ws->d.n_max || m > ws->d.nnz_max / 2) return FBCC_E_WORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    int64_t ends[2] = {0, 0};
    if (n == 0) return m == 0 ? FBCC_OK : FBCC_E_INVALID;
    if (offsets_64) {
        API_CK(cudaMemcpyAsync(&ends[0], csr_offsets, 8, cudaMemcpyDeviceToHost, s), "D2H");
        API_CK(cudaMemcpyAsync(&ends[1], (const int64_t *)csr_offsets + n, 8, cudaMemcpyDeviceToHost, s), "D2H");
    } else {
        int32_t e32[2] = {0, 0};
        API_CK(cudaMemcpyAsync(&e32[0], csr_offsets, 4, cudaMemcpyDeviceToHost, s), "D2H");
        API_CK(cudaMemcpyAsync(&e32[1], (const int32_t *)csr_offsets + n, 4, cudaMemcpyDeviceToHost, s), "D2H");
        API_CK(cudaStreamSynchronize(s), "sync");
        ends[0] = e32[0];
        ends[1] = e32[1];
    }
    API_CK(cudaStreamSynchronize(s), "sync");
    if (ends[0] != 0 || ends[1] != 2 * m) return FBCC_E_INVALID;
    API_CK(cudaMemsetAsync(ws->d.err, 0, sizeof(int), s), "memset");
    const int grid = device_grid(ws->cfg);
    if (offsets_64)
        k_validate<int64_t><<<grid, kThreads, 0, s>>>((const int64_t *)csr_offsets, csr_adj, n, 2 * m, ws->d.err);
    else
        k_validate<int32_t><<<grid, kThreads, 0, s>>>((const int32_t *)csr_offsets, csr_adj, n, 2 * m, ws->d.err);
    API_CK(cudaGetLastError(), "k_validate");
    int bad = 0;
    API_CK(cudaMemcpyAsync(&bad, ws->d.err, sizeof(int), cudaMemcpyDeviceToHost, s), "D2H");
    API_CK(cudaStreamSynchronize(s), "sync");
    if (bad & 1) return FBCC_E_INVALID;
    if (bad & 2) return FBCC_E_NOT_SIMPLE;
    return FBCC_OK;
}

// ---------------------------------------------------------------------------
// Batched solve
// ---------------------------------------------------------------------------
extern "C" size_t fbcc_batch_workspace_bytes(int64_t n_total, int64_t nnz_total, int32_t n_graphs)
{
    return fbcc_workspace_bytes(n_total, nnz_total) + batch_stage_bytes(n_total, nnz_total, n_graphs);
}

extern "C" fbcc_status fbcc_solve_batch(int32_t n_graphs, const int64_t *vtx_base, const int64_t *arc_base,
                                        const int64_t *host_vtx_base, const int64_t *host_arc_base,
                                        const int32_t *local_off, const int32_t *local_adj, int32_t *edge_bcc,
                                        int32_t *bcc_head, uint8_t *is_ap, uint8_t *is_bridge, fbcc_stats *stats,
                                        fbcc_workspace *ws, void *stream)
{
    if (!ws || n_graphs < 1 || !vtx_base || !arc_base || !host_vtx_base || !host_arc_base || !stats)
        return FBCC_E_INVALID;
    const int64_t n = host_vtx_base[n_graphs], nnz = host_arc_base[n_graphs];
    if (host_vtx_base[0] != 0 || host_arc_base[0] != 0 || nnz % 2) return FBCC_E_INVALID;
    for (int32_t g = 0; g < n_graphs; ++g)
        if (host_vtx_base[g + 1] < host_vtx_base[g] || host_arc_base[g + 1] < host_arc_base[g] ||
            (host_arc_base[g + 1] - host_arc_base[g]) % 2)
            return FBCC_E_INVALID;
    fbcc_status st = check_args(host_vtx_base, local_adj, n, nnz / 2, edge_bcc, bcc_head, is_ap, is_bridge, ws);
    if (st != FBCC_OK) return st;
    if (n > 0 && !local_off) return FBCC_E_INVALID;
    const size_t need = batch_stage_bytes(ws->d.n_max, ws->d.nnz_max, n_graphs);
    if (ws->bstage_bytes < need) {
        if (ws->caller_mem) return FBCC_E_WORKSPACE;   // more graphs than the memory was carved for
        cudaStreamSynchronize((cudaStream_t)stream);
        cudaFree(ws->bstage);
        ws->bstage = nullptr;
        ws->bstage_bytes = 0;
        ws->have_key = false;
        API_CK(cudaMalloc(&ws->bstage, need), "cudaMalloc(batch staging)");
        ws->bstage_bytes = need;
    }
    Carver c{static_cast<char *>(ws->bstage)};
    int64_t *goff = c.take<int64_t>(ws->d.n_max + 1);
    int32_t *gadj = c.take<int32_t>(ws->d.nnz_max);
    Batch B;
    B.G = n_graphs;
    B.vtx_base = vtx_base;
    B.arc_base = arc_base;
    B.bcc_base = c.take<int64_t>((int64_t)n_graphs + 1);
    B.stats = stats;
    return solve_device(goff, 1, gadj, n, nnz / 2, edge_bcc, bcc_head, is_ap, is_bridge, nullptr, ws,
                        (cudaStream_t)stream, B, local_off, local_adj);
}

extern "C" int32_t fbcc_profile_count(const fbcc_workspace *ws) { return ws ? ws->prof.count : 0; }

extern "C" fbcc_status fbcc_profile_get(const fbcc_workspace *ws, int32_t i, const char **name, float *ms)
{
    if (!ws || !ws->prof.ready || i < 0 || i >= ws->prof.count || !name || !ms) return FBCC_E_INVALID;
    API_CK(cudaEventSynchronize(ws->prof.ev[i + 1]), "cudaEventSynchronize");
    API_CK(cudaEventElapsedTime(ms, ws->prof.ev[i], ws->prof.ev[i + 1]), "cudaEventElapsedTime");
    *name = ws->prof.names[i];
    return FBCC_OK;
}

extern "C" fbcc_status fbcc_debug_read(const fbcc_workspace *ws, const char *name, void *host_dst, int64_t count)
{
    if (!ws || !name || !host_dst || count < 0) return FBCC_E_INVALID;
    const Dev &d = ws->d;
    if (!strcmp(name, "dirb")) {   // one bit per arc, bytes
        if (count > ceil_div(d.nnz_max, 8)) return FBCC_E_INVALID;
        API_CK(cudaDeviceSynchronize(), "cudaDeviceSynchronize");
        API_CK(cudaMemcpy(host_dst, d.dirb, size_t(count), cudaMemcpyDeviceToHost), "debug copy");
        return FBCC_OK;
    }
    if (count > d.n_max) return FBCC_E_INVALID;
    const void *src = nullptr;
    size_t elem = 4;
    const bool f = !strcmp(name, "first"), pa = !strcmp(name, "parent"), la = !strcmp(name, "last");
    if (f || pa || la) {
        // by vertex, from fp = {first, parent}; last[v] = lastp[first[v]]
        std::vector<int2> fp(size_t(count) + 1);
        std::vector<int32_t> lastp;
        API_CK(cudaDeviceSynchronize(), "cudaDeviceSynchronize");
        API_CK(cudaMemcpy(fp.data(), d.fp, size_t(count) * sizeof(int2), cudaMemcpyDeviceToHost), "debug copy");
        if (la) {
            lastp.resize(size_t(count) + 1);
            API_CK(cudaMemcpy(lastp.data(), d.lastp, size_t(count) * sizeof(int32_t), cudaMemcpyDeviceToHost),
                   "debug copy");
        }
        int32_t *out = static_cast<int32_t *>(host_dst);
        for (int64_t v = 0; v < count; ++v) {
            const int32_t fv = fp[size_t(v)].x;
            if (f) out[v] = fv;
            else if (pa) out[v] = fp[size_t(v)].y;
            else out[v] = fv >= 0 && fv < count ? lastp[size_t(fv)] : -1;
        }
        return FBCC_OK;
    }
    if (!strcmp(name, "label")) src = d.lab;
    else if (!strcmp(name, "w1")) src = d.w1;
    else if (!strcmp(name, "w2")) src = d.w2;
    else if (!strcmp(name, "low")) src = d.low;
    else if (!strcmp(name, "high")) src = d.high;
    else if (!strcmp(name, "ord")) src = d.ord;
    else if (!strcmp(name, "porig")) src = d.porig;
    else if (!strcmp(name, "err")) { src = d.err; if (count > 1) return FBCC_E_INVALID; }
    else if (!strcmp(name, "sampled")) { src = d.counters + 8; if (count > 4) return FBCC_E_INVALID; }
    else if (!strcmp(name, "vbits")) { src = d.vbits; elem = 1; }
    else return FBCC_E_INVALID;
    API_CK(cudaDeviceSynchronize(), "cudaDeviceSynchronize");
    API_CK(cudaMemcpy(host_dst, src, size_t(count) * elem, cudaMemcpyDeviceToHost), "debug copy");
    return FBCC_OK;
}

// ---------------------------------------------------------------------------
// Biconnectivity queries over the last solve (section 3.4's representation)
// ---------------------------------------------------------------------------
namespace {

fbcc_status query_ready(fbcc_workspace *ws, cudaStream_t s)
{
    if (!ws || ws->last_n < 0) return FBCC_E_INVALID;
    if (!ws->qindex) {
        API_CK(launch_query_index(ws->d, ws->last_n, s), "query index");
        ws->qindex = true;
    }
    return FBCC_OK;
}

}  // namespace

extern "C" fbcc_status fbcc_query_biconnected(fbcc_workspace *ws, const int32_t *u, const int32_t *v, int64_t q,
                                              int32_t *bcc, void *stream)
{
    if (q < 0 || (q > 0 && (!u || !v || !bcc))) return FBCC_E_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    fbcc_status st = query_ready(ws, s);
    if (st != FBCC_OK) return st;
    API_CK(launch_query_pairs(ws->d, ws->last_n, u, v, q, bcc, device_grid(ws->cfg), s), "k_qpairs");
    return FBCC_OK;
}

extern "C" fbcc_status fbcc_query_bcc_count(fbcc_workspace *ws, const int32_t *v, int64_t q, int64_t *out_off,
                                            void *stream)
{
    if (q < 0 || !out_off || (q > 0 && !v)) return FBCC_E_INVALID;
    if (ws && q > 2 * ws->d.n_max) return FBCC_E_WORKSPACE;
    cudaStream_t s = (cudaStream_t)stream;
    fbcc_status st = query_ready(ws, s);
    if (st != FBCC_OK) return st;
    API_CK(launch_query_count(ws->d, ws->last_n, v, q, out_off, device_grid(ws->cfg), s), "k_qcount_scan");
    return FBCC_OK;
}

extern "C" fbcc_status fbcc_query_bccs_of(fbcc_workspace *ws, const int32_t *v, int64_t q, const int64_t *out_off,
                                          int32_t *out, void *stream)
{
    if (q < 0 || (q > 0 && (!v || !out_off || !out))) return FBCC_E_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    fbcc_status st = query_ready(ws, s);
    if (st != FBCC_OK) return st;
    API_CK(launch_query_list(ws->d, ws->last_n, v, q, out_off, out, device_grid(ws->cfg), s), "k_qlist");
    return FBCC_OK;
}

// ---------------------------------------------------------------------------
// Solve with no allocation at all: the workspace lives in a fixed device array.
//
// For callers that must not allocate device memory themselves or through us:
// code running under an allocator or memory pool that forbids cudaMalloc,
// plugin hosts that own every byte of device memory, latency-critical paths
// where an allocation's implicit synchronisation is not acceptable. They pass
// their inputs and outputs; the scratch is kNoAllocBytes of static device memory
// that every GPU loading this library keeps until the process exits.
// ---------------------------------------------------------------------------
namespace {

constexpr int64_t kNoAllocMaxN = 1 << 15;     // vertices
constexpr int64_t kNoAllocMaxNnz = 1 << 18;   // arcs (2m)
constexpr size_t kNoAllocBytes = size_t(12) << 20;
constexpr int kNoAllocMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// The device address of g_noalloc_scratch differs per device and per context (a
// cudaDeviceReset destroys the primary context, and the module is loaded again
// into the next one), so it is cached per device together with the id of the
// context it was looked up in, and looked up again when that id changes.
struct NoAllocSlot {
    unsigned long long ctx_id;
    char *base;
};
std::mutex g_noalloc_mu;
NoAllocSlot g_noalloc_slot[kNoAllocMaxDevices];

typedef int (*CtxGetCurrentFn)(void **);
typedef int (*CtxGetIdFn)(void *, unsigned long long *);

// Id of the context current on this thread (0 when the driver cannot tell).
unsigned long long current_ctx_id()
{
    static CtxGetCurrentFn get_cur = nullptr;
    static CtxGetIdFn get_id = nullptr;
    static bool looked = false;
    if (!looked) {
        cudaDriverEntryPointQueryResult q1, q2;
        void *f1 = nullptr, *f2 = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) == cudaSuccess &&
            q1 == cudaDriverEntryPointSuccess)
            get_cur = reinterpret_cast<CtxGetCurrentFn>(f1);
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) == cudaSuccess &&
            q2 == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<CtxGetIdFn>(f2);
        looked = true;
    }
    void *ctx = nullptr;
    unsigned long long id = 0;
    if (get_cur && get_id && get_cur(&ctx) == 0 && ctx && get_id(ctx, &id) == 0) return id;
    return 0;
}

}  // namespace

extern "C" fbcc_status fbcc_solve_noalloc(const void *csr_offsets, int offsets_64, const int32_t *csr_adj,
                                          int64_t n, int64_t m, int32_t *edge_bcc, int32_t *bcc_head,
                                          uint8_t *is_ap, uint8_t *is_bridge, fbcc_stats *stats_dev, void *stream)
{
    if (n < 0 || m < 0) return FBCC_E_INVALID;
    if (n > kNoAllocMaxN || m > kNoAllocMaxNnz / 2) return FBCC_E_WORKSPACE;
    int dev = 0;
    API_CK(cudaGetDevice(&dev), "cudaGetDevice");
    if (dev < 0 || dev >= kNoAllocMaxDevices) return FBCC_E_INVALID;
    API_CK(cudaSetDevice(dev), "cudaSetDevice");   // makes the device's primary context current
    char *base = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_noalloc_mu);
        const unsigned long long id = current_ctx_id();
        NoAllocSlot &sl = g_noalloc_slot[dev];
        if (!sl.base || id == 0 || sl.ctx_id != id) {
            // host code may not use g_noalloc_scratch as an address: ask the runtime
            // for the device address of this device's copy in the current context
            void *p = nullptr;
            API_CK(cudaGetSymbolAddress(&p, g_noalloc_scratch), "cudaGetSymbolAddress");
            sl.base = static_cast<char *>(p);
            sl.ctx_id = id;
        }
        base = sl.base;
    }
    API_CK(prepare_rooting(), "cudaFuncSetAttribute");
    fbcc_workspace ws;  // host-side view only: no allocation, no stream, no graph
    ws.cfg = default_config();
    ws.cfg.use_graph = -1;
    if (carve(ws.d, nullptr, kNoAllocMaxN, kNoAllocMaxNnz) > kNoAllocBytes) return FBCC_E_WORKSPACE;
    carve(ws.d, base, kNoAllocMaxN, kNoAllocMaxNnz);
    fbcc_status st = check_args(csr_offsets, csr_adj, n, m, edge_bcc, bcc_head, is_ap, is_bridge, &ws);
    if (st != FBCC_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = offsets_64
        ? enqueue_solve<int64_t>(&ws, (const int64_t *)csr_offsets, csr_adj, n, m, edge_bcc, bcc_head, is_ap,
                                 is_bridge, s)
        : enqueue_solve<int32_t>(&ws, (const int32_t *)csr_offsets, csr_adj, n, m, edge_bcc, bcc_head, is_ap,
                                 is_bridge, s);
    API_CK(e, "enqueue (no-alloc)");
    if (stats_dev)
        API_CK(cudaMemcpyAsync(stats_dev, ws.d.stats, sizeof(fbcc_stats), cudaMemcpyDeviceToDevice, s),
               "stats copy");
    return FBCC_OK;
}
