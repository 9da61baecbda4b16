// Biconnectivity queries over the space-efficient BCC representation (section
// 3.4): after a solve every non-root vertex v has a label l[v] (its class's top
// vertex), and each label's BCC is its class plus one head, the parent of the top
// (section 4.2). So
//  - u and v (u != v) lie in a common BCC iff l[u] = l[v] (both non-root), or u is
//    the head of l[v], or v the head of l[u]; two BCCs share at most one vertex, so
//    that BCC is unique, and its canonical index is the rank of the label;
//  - the BCCs of v are its own label's (v non-root) and those of the labels it
//    heads. A per-head list of the labels' ranks is built once per solve (a scan of
//    the per-vertex head counts and a fill), on the stream of the first query.
// Everything reads the workspace's arrays of the last solve: labels, the {first,
// parent} pairs, the label ranks and the head counts.
#include "fbcc_internal.cuh"

namespace fbcc {

namespace {

// Exclusive prefix of the head counts: hoff[v] = labels headed by vertices < v.
__global__ void __launch_bounds__(kThreads) k_qindex_scan(int64_t n, const int32_t *__restrict__ nh, int32_t *hoff,
                                                          long long *ticket, uint64_t *status, int *err)
{
    const int64_t ntiles = (n + 1 + kTile - 1) / kTile;
    while (true) {
        const int64_t t = scan_ticket(ticket);
        if (t >= ntiles) return;
        long long v[kItems];
        const int64_t i0 = t * kTile + (int64_t)threadIdx.x * kItems;
#pragma unroll
        for (int j = 0; j < kItems; ++j) v[j] = i0 + j < n ? nh[i0 + j] : 0;
        scan_tile_exclusive(v, t, status, err);
#pragma unroll
        for (int j = 0; j < kItems; ++j)
            if (i0 + j <= n) hoff[i0 + j] = (int32_t)v[j];
    }
}

// Every label's rank into its head's list (in no particular order).
__global__ void __launch_bounds__(kThreads) k_qindex_fill(int64_t n, const int2 *__restrict__ fp,
                                                          const int32_t *__restrict__ lab,
                                                          const int32_t *__restrict__ rank,
                                                          const int32_t *__restrict__ hoff, int32_t *hfill,
                                                          int32_t *hlist, int *err)
{
    for (int64_t l = blockIdx.x * (int64_t)kThreads + threadIdx.x; l < n; l += (int64_t)gridDim.x * kThreads) {
        const int32_t h = fp[l].y;
        if (h < 0 || lab[l] != l || !in_range(h, n, err)) continue;
        const int32_t s = atomicAdd(hfill + h, 1);
        const int64_t at = (int64_t)hoff[h] + s;
        if (at < hoff[h + 1]) hlist[at] = rank[l];
        else atomicOr(err, kErrIndex);
    }
}

// Common BCC of every pair, or -1 (no common BCC, u == v, or an id out of range).
__global__ void __launch_bounds__(kThreads) k_qpairs(int64_t q, const int32_t *__restrict__ qu,
                                                     const int32_t *__restrict__ qv, int64_t n,
                                                     const int2 *__restrict__ fp, const int32_t *__restrict__ lab,
                                                     const int32_t *__restrict__ rank, int32_t *out)
{
    for (int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x; i < q; i += (int64_t)gridDim.x * kThreads) {
        const int32_t u = qu[i], v = qv[i];
        int32_t r = -1;
        if (u != v && (uint32_t)u < (uint64_t)n && (uint32_t)v < (uint64_t)n) {
            const int32_t lu = fp[u].y >= 0 ? lab[u] : -1, lv = fp[v].y >= 0 ? lab[v] : -1;
            if (lu >= 0 && lu == lv) r = rank[lu];
            else if (lv >= 0 && fp[lv].y == u) r = rank[lv];
            else if (lu >= 0 && fp[lu].y == v) r = rank[lu];
        }
        out[i] = r;
    }
}

__device__ __forceinline__ int32_t bcc_count_of(int32_t v, int64_t n, const int2 *__restrict__ fp,
                                                const int32_t *__restrict__ hoff)
{
    if ((uint32_t)v >= (uint64_t)n) return 0;
    return (fp[v].y >= 0 ? 1 : 0) + (hoff[v + 1] - hoff[v]);
}

// out_off[i] = BCCs of the queried vertices before i; out_off[q] = their total.
__global__ void __launch_bounds__(kThreads) k_qcount_scan(int64_t q, const int32_t *__restrict__ qv, int64_t n,
                                                          const int2 *__restrict__ fp,
                                                          const int32_t *__restrict__ hoff, int64_t *out_off,
                                                          long long *ticket, uint64_t *status, int *err)
{
    const int64_t ntiles = (q + 1 + kTile - 1) / kTile;
    while (true) {
        const int64_t t = scan_ticket(ticket);
        if (t >= ntiles) return;
        long long v[kItems];
        const int64_t i0 = t * kTile + (int64_t)threadIdx.x * kItems;
#pragma unroll
        for (int j = 0; j < kItems; ++j) v[j] = i0 + j < q ? bcc_count_of(qv[i0 + j], n, fp, hoff) : 0;
        scan_tile_exclusive(v, t, status, err);
#pragma unroll
        for (int j = 0; j < kItems; ++j)
            if (i0 + j <= q) out_off[i0 + j] = v[j];
    }
}

// The BCCs of every queried vertex at out[out_off[i] ..]: its own label's first,
// then the labels it heads. A warp takes 32 queries, one per lane; lists longer
// than kShortList are then copied by the whole warp, one at a time.
constexpr int kShortList = 16;

__global__ void __launch_bounds__(kThreads) k_qlist(int64_t q, const int32_t *__restrict__ qv, int64_t n,
                                                    const int2 *__restrict__ fp, const int32_t *__restrict__ lab,
                                                    const int32_t *__restrict__ rank,
                                                    const int32_t *__restrict__ hoff,
                                                    const int32_t *__restrict__ hlist,
                                                    const int64_t *__restrict__ out_off, int32_t *out)
{
    const int lane = threadIdx.x & 31;
    const int64_t q_pad = (q + 31) & ~31ll;
    for (int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x; i < q_pad; i += (int64_t)gridDim.x * kThreads) {
        int32_t v = -1, hb = 0, he = 0;
        int64_t o = 0;
        if (i < q) {
            v = qv[i];
            if ((uint32_t)v < (uint64_t)n) {
                o = out_off[i];
                if (fp[v].y >= 0) out[o++] = rank[lab[v]];
                hb = hoff[v];
                he = hoff[v + 1];
            }
        }
        const bool lng = he - hb > kShortList;
        if (!lng)
            for (int32_t k = hb; k < he; ++k) out[o++] = hlist[k];
        unsigned todo = __ballot_sync(0xffffffffu, lng);
        while (todo) {
            const int src = __ffs(todo) - 1;
            todo &= todo - 1;
            const int32_t b = __shfl_sync(0xffffffffu, hb, src), e = __shfl_sync(0xffffffffu, he, src);
            const int64_t oo = __shfl_sync(0xffffffffu, o, src);
            for (int32_t k = b + lane; k < e; k += 32) out[oo + (k - b)] = hlist[k];
        }
    }
}

}  // namespace

cudaError_t launch_query_index(const Dev &d, int64_t n, cudaStream_t s)
{
    Launch L{s, 0};
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    L.grid = (sms > 0 ? sms : 1) * 8;
    const int64_t ntiles = (n + 1 + kTile - 1) / kTile;
    cudaError_t e = cudaMemsetAsync(d.counters, 0, sizeof(long long), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(d.scan_status, 0, ntiles * sizeof(uint64_t), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(d.hfill, 0, (n > 0 ? n : 1) * sizeof(int32_t), s);
    if (e != cudaSuccess) return e;
    k_qindex_scan<<<grid_for(L, ntiles), kThreads, 0, s>>>(n, d.nh, d.hoff, d.counters, d.scan_status, d.err);
    k_qindex_fill<<<grid_for(L, ceil_div(n, kThreads)), kThreads, 0, s>>>(n, d.fp, d.lab, d.rank, d.hoff, d.hfill,
                                                                          d.hlist, d.err);
    return cudaGetLastError();
}

cudaError_t launch_query_pairs(const Dev &d, int64_t n, const int32_t *u, const int32_t *v, int64_t q, int32_t *out,
                               int grid, cudaStream_t s)
{
    if (q <= 0) return cudaSuccess;
    const int64_t want = ceil_div(q, kThreads);
    k_qpairs<<<(int)(want < grid ? want : grid), kThreads, 0, s>>>(q, u, v, n, d.fp, d.lab, d.rank, out);
    return cudaGetLastError();
}

cudaError_t launch_query_count(const Dev &d, int64_t n, const int32_t *v, int64_t q, int64_t *out_off, int grid,
                               cudaStream_t s)
{
    const int64_t ntiles = (q + 1 + kTile - 1) / kTile;
    cudaError_t e = cudaMemsetAsync(d.counters, 0, sizeof(long long), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(d.scan_status, 0, ntiles * sizeof(uint64_t), s);
    if (e != cudaSuccess) return e;
    k_qcount_scan<<<(int)(ntiles < grid ? ntiles : grid), kThreads, 0, s>>>(q, v, n, d.fp, d.hoff, out_off,
                                                                             d.counters, d.scan_status, d.err);
    return cudaGetLastError();
}

cudaError_t launch_query_list(const Dev &d, int64_t n, const int32_t *v, int64_t q, const int64_t *out_off,
                              int32_t *out, int grid, cudaStream_t s)
{
    if (q <= 0) return cudaSuccess;
    const int64_t want = ceil_div(q, kThreads);
    k_qlist<<<(int)(want < grid ? want : grid), kThreads, 0, s>>>(q, v, n, d.fp, d.lab, d.rank, d.hoff, d.hlist,
                                                                   out_off, out);
    return cudaGetLastError();
}

}  // namespace fbcc
