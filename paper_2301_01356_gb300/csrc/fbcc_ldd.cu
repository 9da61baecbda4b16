// First-CC by low-diameter decomposition and union-find (section 5,
// "Connectivity": an LDD of the graph before union-find, after Miller, Peng and
// Xu's exponential-shift clustering).
//
// Every vertex v draws a shift delta_v ~ Exp(beta) and wakes at round
// start_v = D - floor(delta_v) (0 when delta_v >= D; beta = 1 / inv_beta and
// D = ceil(inv_beta * ln n), at most kLddMaxRounds). Round r:
//  - the vertices woken at r that no cluster has reached become centres of their
//    own clusters;
//  - the frontier (the vertices reached in round r - 1 and the centres of round r)
//    goes through its lists: an unreached neighbour joins the frontier vertex's
//    cluster (one CAS decides it), and the edge that reached it is a forest edge,
//    recorded at the reached vertex's slot with its arc's CSR position; a
//    neighbour in another cluster puts the edge on the list of edges between
//    clusters.
// Every vertex is reached or woken by round D, so D + 1 rounds finish the
// clusters, each spanned by the tree of the edges that reached its vertices.
// Union-find over the centres then takes the edges between clusters (a hook of
// centre r records its edge at r's slot, which no reaching edge uses); when the
// list outgrew its space, a full hook pass over all arcs follows instead. Last,
// every component's root moves to its smallest vertex, where the tours start.
//
// Layout of the scratch (the rooting step's space, free during First-CC): two
// frontier queues of n ids, the wake rounds (one byte per vertex), the vertices
// bucketed by wake round, the per-round counters, the chunk queue of long lists
// and the list of edges between clusters.
#include "fbcc_internal.cuh"

#include <math.h>

namespace fbcc {

constexpr int kLddMaxRounds = 63;

// SplitMix64 (Steele, Lea and Flood, 2014): output k of the stream seeded with seed.
__device__ __forceinline__ uint64_t splitmix64_at(uint64_t seed, uint64_t k)
{
    uint64_t z = seed + (k + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Wake rounds, the count of vertices waking in each round (a histogram in shared
// memory per CTA), and the centres of round 0 (their queue is q0).
__global__ void __launch_bounds__(kThreads) k_ldd_init(int64_t n, int inv_beta, int D, uint64_t seed,
                                                       int32_t *cluster, uint8_t *start, int32_t *q0,
                                                       long long *cnt0, long long *bcount)
{
    __shared__ int32_t hist[kLddMaxRounds + 1];
    if (threadIdx.x <= D) hist[threadIdx.x] = 0;
    __syncthreads();
    const int64_t n_pad = (n + 31) & ~31ll;
    for (int64_t v = blockIdx.x * (int64_t)kThreads + threadIdx.x; v < n_pad; v += (int64_t)gridDim.x * kThreads) {
        bool centre = false;
        if (v < n) {
            const uint64_t z = splitmix64_at(seed, (uint64_t)v);
            const float u = (float)((z >> 40) + 1) * 0x1.0p-24f;   // uniform on (0, 1]
            const float shift = -logf(u) * (float)inv_beta;       // Exp(1 / inv_beta)
            const int s = shift >= (float)D ? 0 : D - (int)shift;
            start[v] = (uint8_t)s;
            atomicAdd(hist + s, 1);
            centre = s == 0;
            cluster[v] = centre ? (int32_t)v : -1;
        }
        warp_append<int32_t>(q0, cnt0, n, centre, (int32_t)v);
    }
    __syncthreads();
    if (threadIdx.x <= D && hist[threadIdx.x])
        atomicAdd((unsigned long long *)(bcount + threadIdx.x), (unsigned long long)hist[threadIdx.x]);
}

// The vertices waking in rounds 1..D, bucketed by round (a counting sort: each
// CTA counts a tile in shared memory and reserves its slots in each bucket with
// one atomic per round), so that a round's centres are read from their bucket
// rather than found by a scan of every vertex. bstart[r] = the bucket's start.
__global__ void __launch_bounds__(kThreads) k_ldd_fill(int64_t n, int D, const uint8_t *__restrict__ start,
                                                       const long long *__restrict__ bcount, long long *bfill,
                                                       long long *bstart, int32_t *bucket)
{
    constexpr int kPer = 8;
    __shared__ long long base[kLddMaxRounds + 1], sbase[kLddMaxRounds + 1];
    __shared__ int32_t scount[kLddMaxRounds + 1];
    if (threadIdx.x == 0) {
        long long run = 0;
        for (int r = 0; r <= D; ++r) {
            base[r] = run;
            run += r ? bcount[r] : 0;   // round 0's centres are queued already
        }
    }
    __syncthreads();
    if (blockIdx.x == 0 && threadIdx.x <= D) bstart[threadIdx.x] = base[threadIdx.x];
    for (int64_t v0 = (int64_t)blockIdx.x * kThreads * kPer; v0 < n; v0 += (int64_t)gridDim.x * kThreads * kPer) {
        if (threadIdx.x <= D) scount[threadIdx.x] = 0;
        __syncthreads();
        int s[kPer];
        int32_t loc[kPer];
#pragma unroll
        for (int k = 0; k < kPer; ++k) {
            const int64_t v = v0 + k * kThreads + threadIdx.x;
            s[k] = v < n ? start[v] : 0;
            loc[k] = s[k] > 0 ? atomicAdd(scount + s[k], 1) : 0;
        }
        __syncthreads();
        if (threadIdx.x > 0 && threadIdx.x <= D && scount[threadIdx.x])
            sbase[threadIdx.x] = base[threadIdx.x] + (long long)atomicAdd((unsigned long long *)(bfill + threadIdx.x),
                                                                        (unsigned long long)scount[threadIdx.x]);
        __syncthreads();
#pragma unroll
        for (int k = 0; k < kPer; ++k)
            if (s[k] > 0) bucket[sbase[s[k]] + loc[k]] = (int32_t)(v0 + k * kThreads + threadIdx.x);
        __syncthreads();   // before the counts are reset
    }
}

// One arc per lane (the whole warp calls): u -> w at CSR position a, u in cluster cu.
__device__ __forceinline__ void ldd_arc(const int32_t *__restrict__ adj, int32_t *cluster, int32_t *te_u,
                                        int32_t *te_v, int32_t *te_a, bool valid, int32_t u, int32_t cu, int64_t a,
                                        int32_t *qn, long long *cnt_n, int64_t n, int2 *xl, int64_t xl_cap,
                                        long long *xl_n)
{
    bool reached = false, cross = false;
    int32_t w = 0;
    if (valid) {
        w = adj[a];
        int32_t c = cluster[w];   // a set cluster never changes; a stale -1 only costs the CAS
        if (c < 0) {
            c = atomicCAS(cluster + w, -1, cu);
            reached = c < 0;
        }
        if (reached) tree_edge(te_u, te_v, te_a, w, u, w, a);
        else cross = c != cu;
    }
    warp_append<int32_t>(qn, cnt_n, n, reached, w);
    warp_append<int2>(xl, xl_n, xl_cap, cross, make_int2(u, w));
}

// The frontier of one round. A warp takes 32 queue entries: lists above kRestLong
// arcs go to the chunk queue, the others are concatenated and gone through 32
// arcs at a time, each lane finding its arc's list by a search of the warp's
// prefix sums of list lengths.
template <typename OffT>
__global__ void __launch_bounds__(kThreads) k_ldd_expand(const OffT *__restrict__ off,
                                                         const int32_t *__restrict__ adj, int64_t n,
                                                         const int32_t *__restrict__ qc,
                                                         const long long *__restrict__ cnt_c, int32_t *qn,
                                                         long long *cnt_n, int32_t *cluster, int32_t *te_u,
                                                         int32_t *te_v, int32_t *te_a, int2 *cq, int64_t cq_cap,
                                                         long long *cq_n, int2 *xl, int64_t xl_cap,
                                                         long long *xl_n)
{
    const int lane = threadIdx.x & 31;
    const int64_t cnt = *cnt_c < n ? *cnt_c : n;
    const int64_t warps = (int64_t)gridDim.x * (kThreads / 32);
    for (int64_t i0 = ((blockIdx.x * (int64_t)kThreads + threadIdx.x) >> 5) * 32; i0 < cnt; i0 += warps * 32) {
        const int64_t i = i0 + lane;
        int32_t u = 0, cu = 0;
        int64_t b = 0, len = 0;
        if (i < cnt) {
            u = qc[i];
            cu = cluster[u];
            b = off[u];
            len = (int64_t)off[u + 1] - b;
        }
        // the long lists, one at a time, to the chunk queue (or kept by the warp)
        unsigned lng = __ballot_sync(0xffffffffu, len > kRestLong);
        while (lng) {
            const int src = __ffs(lng) - 1;
            lng &= lng - 1;
            const int32_t uu = __shfl_sync(0xffffffffu, u, src), cc = __shfl_sync(0xffffffffu, cu, src);
            const int64_t bb = __shfl_sync(0xffffffffu, b, src), ll = __shfl_sync(0xffffffffu, len, src);
            if (rest_queue(cq, cq_cap, cq_n, uu, ll, lane)) continue;
            for (int64_t a0 = bb; a0 < bb + ll; a0 += 32)
                ldd_arc(adj, cluster, te_u, te_v, te_a, a0 + lane < bb + ll, uu, cc, a0 + lane, qn, cnt_n, n, xl,
                        xl_cap, xl_n);
        }
        if (len > kRestLong) len = 0;
        // inclusive prefix sums of the remaining lengths
        int32_t inc = (int32_t)len;
        for (int o = 1; o < 32; o <<= 1) {
            const int32_t y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += y;
        }
        const int32_t total = __shfl_sync(0xffffffffu, inc, 31);
        for (int32_t k0 = 0; k0 < total; k0 += 32) {
            const int32_t k = k0 + lane;
            // the first lane whose prefix exceeds k owns arc k
            int j = 0;
            for (int step = 16; step > 0; step >>= 1) {
                const int32_t p = __shfl_sync(0xffffffffu, inc, j + step - 1);
                if (p <= k) j += step;
            }
            j = j < 31 ? j : 31;
            const int32_t pj = __shfl_sync(0xffffffffu, inc, j), lj = __shfl_sync(0xffffffffu, (int32_t)len, j);
            const int32_t uj = __shfl_sync(0xffffffffu, u, j), cj = __shfl_sync(0xffffffffu, cu, j);
            const int64_t bj = __shfl_sync(0xffffffffu, b, j);
            ldd_arc(adj, cluster, te_u, te_v, te_a, k < total, uj, cj, bj + (k - (pj - lj)), qn, cnt_n, n, xl,
                    xl_cap, xl_n);
        }
    }
}

// The chunks of the round's long lists (a warp per chunk), then the centres of
// the next round: woken vertices that no cluster has reached (one CAS decides
// against a chunk reaching them at the same time).
template <typename OffT>
__global__ void __launch_bounds__(kThreads) k_ldd_chunks(const OffT *__restrict__ off,
                                                         const int32_t *__restrict__ adj, int64_t n,
                                                         const int2 *__restrict__ cq, int64_t cq_cap,
                                                         const long long *__restrict__ cq_n, int32_t *qn,
                                                         long long *cnt_n, int32_t *cluster, int32_t *te_u,
                                                         int32_t *te_v, int32_t *te_a, int2 *xl, int64_t xl_cap,
                                                         long long *xl_n, const int32_t *__restrict__ bucket,
                                                         const long long *__restrict__ bstart,
                                                         const long long *__restrict__ bcount, int next_round)
{
    const int lane = threadIdx.x & 31;
    const int64_t nq = *cq_n < cq_cap ? *cq_n : cq_cap;
    const int64_t warps = (int64_t)gridDim.x * (kThreads / 32);
    for (int64_t i = (blockIdx.x * (int64_t)kThreads + threadIdx.x) >> 5; i < nq; i += warps) {
        const int2 q = cq[i];
        if (q.x < 0) continue;
        const int32_t cu = cluster[q.x];
        const int64_t b = (int64_t)off[q.x] + (int64_t)q.y * kRestChunk, end = off[q.x + 1];
        const int64_t e = b + kRestChunk < end ? b + kRestChunk : end;
        for (int64_t a0 = b; a0 < e; a0 += 32)
            ldd_arc(adj, cluster, te_u, te_v, te_a, a0 + lane < e, q.x, cu, a0 + lane, qn, cnt_n, n, xl, xl_cap,
                    xl_n);
    }
    if (next_round < 0) return;
    const long long b0 = bstart[next_round], nb = bcount[next_round];
    const int64_t nb_pad = (nb + 31) & ~31ll;
    for (int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x; i < nb_pad; i += (int64_t)gridDim.x * kThreads) {
        const int32_t v = i < nb ? bucket[b0 + i] : -1;
        const bool centre = v >= 0 && cluster[v] < 0 && atomicCAS(cluster + v, -1, v) < 0;
        warp_append<int32_t>(qn, cnt_n, n, centre, v);
    }
}

// Union-find over the edges between clusters (every vertex points at its centre,
// and a centre at itself); flag[1] = 1 when the list held them all, else the full
// hook pass that follows (k_cc_hook) goes over every arc.
__global__ void __launch_bounds__(kThreads) k_ldd_unite(const int2 *__restrict__ xl, int64_t xl_cap,
                                                        const long long *__restrict__ xl_n, int32_t *uf,
                                                        int32_t *te_u, int32_t *te_v, int32_t *te_a, int32_t *flag,
                                                        int *err)
{
    const long long cnt = *xl_n;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        flag[0] = 0;
        flag[1] = cnt <= xl_cap;
    }
    const int64_t m = cnt < xl_cap ? cnt : xl_cap;
    for (int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x; i < m; i += (int64_t)gridDim.x * kThreads) {
        const int2 e = xl[i];
        const int32_t r = uf_unite(uf, e.x, e.y, err);
        if (r >= 0) tree_edge(te_u, te_v, te_a, r, e.x, e.y, -1);
    }
}

// The smallest vertex of every component (uf flattened: every vertex names its
// root); lanes with the same root reduce first, and a read of the current
// minimum filters most of the remaining atomics.
__global__ void __launch_bounds__(kThreads) k_ldd_minroot(int64_t n, const int32_t *__restrict__ uf, int32_t *cmin)
{
    const int64_t n_pad = (n + 31) & ~31ll;
    for (int64_t v = blockIdx.x * (int64_t)kThreads + threadIdx.x; v < n_pad; v += (int64_t)gridDim.x * kThreads) {
        const int32_t r = v < n ? uf[v] : -1;
        const unsigned peers = __match_any_sync(0xffffffffu, r);
        const int32_t m = (int32_t)__reduce_min_sync(peers, v < n ? (unsigned)v : 0xffffffffu);
        if (r >= 0 && (int)(threadIdx.x & 31) == __ffs(peers) - 1 && m < cmin[r]) atomicMin(cmin + r, m);
    }
}

// Every vertex then names its component's smallest vertex (which names itself).
__global__ void __launch_bounds__(kThreads) k_ldd_reroot(int64_t n, int32_t *uf, const int32_t *__restrict__ cmin)
{
    for (int64_t v = blockIdx.x * (int64_t)kThreads + threadIdx.x; v < n; v += (int64_t)gridDim.x * kThreads)
        uf[v] = cmin[uf[v]];
}

int ldd_rounds(int64_t n, int inv_beta)
{
    const double d = ceil((double)inv_beta * log((double)(n > 2 ? n : 2)));
    return d < kLddMaxRounds ? (int)d : kLddMaxRounds;
}

template <typename OffT>
cudaError_t launch_ldd_forest(const Dev &d, const OffT *off, const int32_t *adj, int64_t n, int64_t nnz,
                              int inv_beta, int32_t *te_a, int32_t *flag, const Launch &L)
{
    const int D = ldd_rounds(n, inv_beta);
    const int gv = grid_for(L, ceil_div(n, kThreads));
    // the scratch, carved from the local-first list's space (the rooting step's),
    // which holds far more than the queues, the buckets and the wake rounds (13 bytes
// per vertex)
    char *p = reinterpret_cast<char *>(d.xl);
    const size_t room = (size_t)d.xl_cap * sizeof(int2);
    size_t used = 0;
    auto take = [&](size_t bytes) {
        char *q = p + used;
        used += (bytes + 255) & ~size_t(255);
        return q;
    };
    int32_t *q[2] = {reinterpret_cast<int32_t *>(take(n * sizeof(int32_t))),
                     reinterpret_cast<int32_t *>(take(n * sizeof(int32_t)))};
    uint8_t *start = reinterpret_cast<uint8_t *>(take(n));
    int32_t *bucket = reinterpret_cast<int32_t *>(take(n * sizeof(int32_t)));
    // cnt[r]: the frontier of round r; cqn[r]: the chunks of round r; xln: edges
    // between clusters; bcount/bfill/bstart: the buckets of wake rounds
    const size_t ncnt = 5 * (kLddMaxRounds + 2) + 1;
    long long *cnt = reinterpret_cast<long long *>(take(ncnt * sizeof(long long)));
    long long *cqn = cnt + kLddMaxRounds + 2, *bcount = cqn + kLddMaxRounds + 2;
    long long *bfill = bcount + kLddMaxRounds + 2, *bstart = bfill + kLddMaxRounds + 2;
    long long *xln = bstart + kLddMaxRounds + 2;
    if (used + 512 * sizeof(int2) > room) return cudaErrorInvalidValue;   // (cannot happen: see carve)
    // the chunk queue takes up to a quarter of what is left (a full queue leaves a
    // list to its warp), the list of edges between clusters the rest
    const int64_t left = (int64_t)((room - used) / sizeof(int2)) - 256;
    const int64_t cq_want = ceil_div(nnz, kRestChunk) + ceil_div(n, kRestLong) + 64;
    const int64_t cq_cap = cq_want < left / 4 ? cq_want : left / 4;
    int2 *cq = reinterpret_cast<int2 *>(take((size_t)cq_cap * sizeof(int2)));
    int2 *xl = reinterpret_cast<int2 *>(p + used);
    const int64_t xl_cap = (int64_t)((room - used) / sizeof(int2));
    cudaError_t e = cudaMemsetAsync(cnt, 0, ncnt * sizeof(long long), L.s);
    if (e != cudaSuccess) return e;
    k_ldd_init<<<gv, kThreads, 0, L.s>>>(n, inv_beta, D, 0x5eed1dd5eed1dd5ull, d.uf, start, q[0], cnt, bcount);
    L.mark("k_ldd_init");
    k_ldd_fill<<<grid_for(L, ceil_div(n, kThreads * 8)), kThreads, 0, L.s>>>(n, D, start, bcount, bfill, bstart,
                                                                             bucket);
    L.mark("k_ldd_fill");
    for (int r = 0; r <= D; ++r) {
        k_ldd_expand<OffT><<<gv, kThreads, 0, L.s>>>(off, adj, n, q[r & 1], cnt + r, q[(r + 1) & 1], cnt + r + 1,
                                                     d.uf, d.te_u, d.te_v, te_a, cq, cq_cap, cqn + r, xl, xl_cap,
                                                     xln);
        L.mark("k_ldd_expand");
        k_ldd_chunks<OffT><<<gv, kThreads, 0, L.s>>>(off, adj, n, cq, cq_cap, cqn + r, q[(r + 1) & 1],
                                                     cnt + r + 1, d.uf, d.te_u, d.te_v, te_a, xl, xl_cap, xln, bucket,
                                                     bstart, bcount, r < D ? r + 1 : -1);
        L.mark("k_ldd_chunks");
    }
    k_ldd_unite<<<gv, kThreads, 0, L.s>>>(xl, xl_cap, xln, d.uf, d.te_u, d.te_v, te_a, flag, d.err);
    L.mark("k_ldd_unite");
    return cudaGetLastError();
}

cudaError_t launch_ldd_reroot(const Dev &d, int64_t n, const Launch &L)
{
    const int gv = grid_for(L, ceil_div(n, kThreads));
    int32_t *cmin = reinterpret_cast<int32_t *>(d.xl);   // the first frontier queue, free by now
    cudaError_t e = cudaMemsetAsync(cmin, 0x7f, n * sizeof(int32_t), L.s);
    if (e != cudaSuccess) return e;
    k_ldd_minroot<<<gv, kThreads, 0, L.s>>>(n, d.uf, cmin);
    L.mark("k_ldd_minroot");
    k_ldd_reroot<<<gv, kThreads, 0, L.s>>>(n, d.uf, cmin);
    L.mark("k_ldd_reroot");
    return cudaGetLastError();
}

template cudaError_t launch_ldd_forest<int32_t>(const Dev &, const int32_t *, const int32_t *, int64_t, int64_t,
                                                int, int32_t *, int32_t *, const Launch &);
template cudaError_t launch_ldd_forest<int64_t>(const Dev &, const int64_t *, const int32_t *, int64_t, int64_t,
                                                int, int32_t *, int32_t *, const Launch &);

}  // namespace fbcc
