// First-CC and Last-CC (Algorithm 1, steps 1 and 4; section 5, "Connectivity").
//
// Both steps are connectivity by CAS union-find: every union hooks the larger root
// under the smaller one (so a component's root is its smallest vertex, which is
// also the root the spanning tree is later rooted at), finds use path halving.
// First-CC records, for each successful hook, the edge that caused it: those
// n - #CC edges form a spanning forest F (section 5, "Spanning Forest": the forest
// is a by-product of CC). Last-CC runs the same union-find on the skeleton G'
// (plain tree edges and cross edges) without materialising it: the plain tree
// edges are united in the low/high kernel (tagging), and this file's arc pass
// unites the cross edges, skipping tree and back edges by the tags.
#include "fbcc_internal.cuh"

namespace fbcc {

// tile_v[t] = source of arc t*kWTile; tile_v[ntiles] = source of the last arc.
// Also resets the union-find and the tree-edge record, finds the hubs (hub_deg >
// 0: a vertex of at least hub_deg arcs gets a hub slot while slots last, a warp's
// hubs taking consecutive slots with one atomic; rooting uses them to split their
// forest-arc lists), and the largest degree, by which rooting decides how to
// aggregate its list pushes (each warp's maximum over its vertices, with one
// atomic when it beats the value read from L2).
template <typename OffT>
__global__ void __launch_bounds__(kThreads) k_cc_init(const OffT *__restrict__ off, int64_t n, int64_t nnz,
                                                      int32_t *tile_v, int64_t ntiles, int32_t *uf,
                                                      int32_t *te_u, int hub_deg, int32_t *hubidx,
                                                      int32_t *hubvert, int64_t hub_cap, long long *nhub,
                                                      int32_t *maxdeg)
{
    int64_t top = 0;
    const int lane = threadIdx.x & 31;
    const int64_t n_pad = (n + 31) & ~31ll;
    for (int64_t v = blockIdx.x * (int64_t)kThreads + threadIdx.x; v < n_pad; v += (int64_t)gridDim.x * kThreads) {
        int64_t b = 0, e = 0;
        if (v < n) {
            uf[v] = (int32_t)v;
            te_u[v] = -1;
            b = off[v];
            e = off[v + 1];
            top = e - b > top ? e - b : top;
            if (e > b) {
                for (int64_t t = (b + kWTile - 1) / kWTile; t * kWTile < e; ++t) tile_v[t] = (int32_t)v;
                if (b <= nnz - 1 && nnz - 1 < e) tile_v[ntiles] = (int32_t)v;
            }
        }
        if (hub_deg > 0) {
            const bool hub = v < n && e - b >= hub_deg;
            const unsigned m = __ballot_sync(0xffffffffu, hub);
            long long k0 = 0;
            if (m && lane == 0) k0 = (long long)atomicAdd((unsigned long long *)nhub, (unsigned long long)__popc(m));
            k0 = __shfl_sync(0xffffffffu, k0, 0);
            int32_t id = -1;
            if (hub) {
                const long long k = k0 + __popc(m & ((1u << lane) - 1u));
                if (k < hub_cap) {
                    id = (int32_t)k;
                    hubvert[id] = (int32_t)v;
                }
            }
            if (v < n) hubidx[v] = id;
        }
    }
    const unsigned t = __reduce_max_sync(0xffffffffu, (unsigned)(top < INT32_MAX ? top : INT32_MAX));
    if (lane == 0 && (int32_t)t > __ldcg(maxdeg)) atomicMax(maxdeg, (int32_t)t);
}

// Hook every edge u-v (from its arc with u < v). A successful CAS hooks root r
// and records u-v as the tree edge owned by r.
template <typename OffT>
__global__ void __launch_bounds__(kThreads) k_cc_hook(const OffT *__restrict__ off, const int32_t *__restrict__ adj,
                                                      int64_t nnz, const int32_t *__restrict__ tile_v, int64_t ntiles,
                                                      int32_t *uf, int32_t *te_u, int32_t *te_v, int32_t *te_a, int *err,
                                                      bool vec, const int32_t *__restrict__ sampled)
{
    if (sampled && sampled[1]) return;   // after a strong sample the by-vertex pass runs instead
    __shared__ OffT win[kCtaWin];
    ArcTile<OffT> at;
    const int64_t nct = (ntiles + kWarpsPerCta - 1) / kWarpsPerCta;
    for (int64_t t = blockIdx.x; t < nct; t += gridDim.x) {
        arc_cta_tile_sources(off, nnz, tile_v, ntiles, t, win, at);
        if (!at.cnt) continue;
        int32_t d[kItems];
        arc_tile_targets(adj, at.a0, at.cnt, vec, d);
        int32_t cur = -1, rs = -1;   // the source, and where its finds start (its set's root, or near it)
#pragma unroll
        for (int j = 0; j < kItems; ++j) {
            if (j >= at.cnt || at.src[j] >= d[j]) continue;
            if (at.src[j] != cur) {
                cur = at.src[j];
                rs = cur;
            }
            int32_t r = uf_unite(uf, rs, d[j], err);
            if (r >= 0) tree_edge(te_u, te_v, te_a, r, cur, d[j], at.a0 + j);
        }
    }
}

// Sampling pre-pass: hook each vertex's first `k` neighbours (vertex-parallel).
template <typename OffT>
__global__ void __launch_bounds__(kThreads) k_cc_sample(const OffT *__restrict__ off, const int32_t *__restrict__ adj,
                                                        int64_t n, int k, int32_t *uf, int32_t *te_u, int32_t *te_v,
                                                        int32_t *te_a, int *err)
{
    for (int64_t v = blockIdx.x * (int64_t)kThreads + threadIdx.x; v < n; v += (int64_t)gridDim.x * kThreads) {
        int64_t b = off[v], e = off[v + 1];
        for (int64_t a = b; a < e && a < b + k; ++a) {
            int32_t w = adj[a];
            int32_t r = uf_unite(uf, (int32_t)v, w, err);
            if (r >= 0) tree_edge(te_u, te_v, te_a, r, (int32_t)v, w, a);
        }
    }
}

// Membership of the sampled largest component, as a bitmap taken before the full
// pass: the component's root can change during the pass (a component with a
// smaller id joins it), and a test against the live root would then stop skipping.
__global__ void __launch_bounds__(kThreads) k_mark_big(const int32_t *__restrict__ uf, int64_t n,
                                                       const int32_t *__restrict__ big, uint32_t *bigb)
{
    if (!big[1]) return;   // a weak sample: nothing is skipped (see pick_big)
    const int32_t root = big[0];
    const int64_t n_pad = (n + 31) & ~31ll;
    for (int64_t v = blockIdx.x * (int64_t)kThreads + threadIdx.x; v < n_pad; v += (int64_t)gridDim.x * kThreads) {
        const unsigned m = __ballot_sync(0xffffffffu, v < n && uf[v] == root);
        if ((threadIdx.x & 31) == 0) bigb[v >> 5] = m;
    }
}

// The full pass after sampling, by vertex: only vertices outside the sampled
// component (membership frozen in a bitmap before the pass, see k_mark_big) hook
// their arcs, in both directions (an edge from a skipped vertex is seen from its
// other end, unless both ends are in the sampled component, where it cannot join
// anything new). A lane takes a list of up to kRestShort arcs alone; longer lists
// are then hooked by the whole warp, one list at a time, and a list above
// kRestLong arcs (a hub left outside the sample) is cut into chunks of kRestChunk
// arcs that a second launch spreads over the whole grid, so that no warp walks a
// hub's list alone. Where sampling gathered nearly every vertex, this touches the
// offsets and the bitmap and little else.
constexpr int kRestShort = 32;
template <typename OffT>
__global__ void __launch_bounds__(kThreads) k_cc_hook_rest(const OffT *__restrict__ off,
                                                           const int32_t *__restrict__ adj, int64_t n, int32_t *uf,
                                                           int32_t *te_u, int32_t *te_v, int32_t *te_a,
                                                           const uint32_t *__restrict__ bigb, int2 *lq, int64_t lq_cap,
                                                           long long *lq_n, const int32_t *__restrict__ sampled,
                                                           int *err)
{
    if (!sampled[1]) return;   // a weak sample: the tiled full pass runs instead
    const int lane = threadIdx.x & 31;
    const int64_t n_pad = (n + 31) & ~31ll;
    for (int64_t v = blockIdx.x * (int64_t)kThreads + threadIdx.x; v < n_pad; v += (int64_t)gridDim.x * kThreads) {
        int64_t b = 0, e = 0;
        if (v < n && !test_bit(bigb, v)) {
            b = off[v];
            e = off[v + 1];
        }
        const bool lng = e - b > kRestShort;
        if (!lng) {
            for (int64_t a = b; a < e; ++a) {
                const int32_t w = adj[a];
                const int32_t r = uf_unite(uf, (int32_t)v, w, err);
                if (r >= 0) tree_edge(te_u, te_v, te_a, r, (int32_t)v, w, a);
            }
        }
        unsigned todo = __ballot_sync(0xffffffffu, lng);
        while (todo) {
            const int src = __ffs(todo) - 1;
            todo &= todo - 1;
            const int32_t u = (int32_t)__shfl_sync(0xffffffffu, v, src);
            const int64_t bb = __shfl_sync(0xffffffffu, b, src), ee = __shfl_sync(0xffffffffu, e, src);
            if (ee - bb > kRestLong && rest_queue(lq, lq_cap, lq_n, u, ee - bb, lane)) continue;
            for (int64_t a = bb + lane; a < ee; a += 32) {
                const int32_t w = adj[a];
                const int32_t r = uf_unite(uf, u, w, err);
                if (r >= 0) tree_edge(te_u, te_v, te_a, r, u, w, a);
            }
        }
    }
}

// The queued chunks of long lists, a warp per chunk.
template <typename OffT>
__global__ void __launch_bounds__(kThreads) k_cc_hook_chunks(const OffT *__restrict__ off,
                                                             const int32_t *__restrict__ adj,
                                                             const int2 *__restrict__ lq, int64_t lq_cap,
                                                             const long long *__restrict__ lq_n, int32_t *uf,
                                                             int32_t *te_u, int32_t *te_v, int32_t *te_a,
                                                             const int32_t *__restrict__ sampled, int *err)
{
    if (!sampled[1]) return;
    const int lane = threadIdx.x & 31;
    const int64_t nq = *lq_n < lq_cap ? *lq_n : lq_cap;
    const int64_t warps = (int64_t)gridDim.x * (kThreads / 32);
    for (int64_t i = (blockIdx.x * (int64_t)kThreads + threadIdx.x) >> 5; i < nq; i += warps) {
        const int2 q = lq[i];
        if (q.x < 0) continue;
        const int64_t b = off[q.x] + (int64_t)q.y * kRestChunk, end = off[q.x + 1];
        const int64_t e = b + kRestChunk < end ? b + kRestChunk : end;
        for (int64_t a = b + lane; a < e; a += 32) {
            const int32_t w = adj[a];
            const int32_t r = uf_unite(uf, q.x, w, err);
            if (r >= 0) tree_edge(te_u, te_v, te_a, r, q.x, w, a);
        }
    }
}

// Flatten every set to its root. Only roots are ever stored, so concurrent
// threads cannot leave a vertex pointing at a non-root (see uf_root).
__global__ void __launch_bounds__(kThreads) k_uf_compress(int32_t *uf, int64_t n)
{
    const int64_t n_pad = (n + 31) & ~31ll;
    for (int64_t v = blockIdx.x * (int64_t)kThreads + threadIdx.x; v < n_pad; v += (int64_t)gridDim.x * kThreads)
        uf_flatten_warp(uf, v, v < n);
}

// The component that a sample left largest, by a vote of the sources of a fixed
// sample of arcs (tile_v: the source of every kWTile-th arc), so that a vertex
// weighs as much as its list, the work that skipping it saves. A single CTA
// writes big[0] = the winning root (-1: none) and big[1] = whether it holds at
// least half of the votes: below that the by-vertex pass would go through most
// arcs anyway, slower than the tiled full pass, which then runs instead. `cand`
// maps a vertex to its vote (-1: none).
template <typename Cand>
__device__ __forceinline__ void pick_big(const int32_t *__restrict__ tile_v, int64_t ntiles, Cand cand_of,
                                         int32_t *big)
{
    __shared__ int32_t cand[kThreads];
    __shared__ int32_t cnt[kThreads];
    const int64_t t = (int64_t)threadIdx.x * ntiles / kThreads;
    cand[threadIdx.x] = cand_of(tile_v[t]);
    __syncthreads();
    int c = 0, votes = 0;
    for (int i = 0; i < kThreads; ++i) {
        c += cand[i] == cand[threadIdx.x];
        votes += cand[i] >= 0;
    }
    cnt[threadIdx.x] = cand[threadIdx.x] >= 0 ? c : 0;
    __syncthreads();
    if (threadIdx.x == 0) {
        int best = 0;
        for (int i = 1; i < kThreads; ++i)
            if (cnt[i] > cnt[best]) best = i;
        big[0] = cand[best];
        big[1] = cand[best] >= 0 && 2 * cnt[best] >= votes;
    }
}

__global__ void __launch_bounds__(kThreads) k_cc_pick_big(int32_t *uf, const int32_t *__restrict__ tile_v,
                                                          int64_t ntiles, int32_t *big)
{
    pick_big(tile_v, ntiles, [&](int32_t v) { return uf_find(uf, v); }, big);
}

// Local-first variant: each CTA owns a range of V consecutive vertex ids and
// unites the edges inside the range in shared memory (graphs whose ids follow
// their geometry, such as grids or meshes, keep most edges inside a range); the
// range's sets then enter the global union-find flattened.
//
// Edges between ranges (u < w) are gathered into a list on the way, and one
// launch hooks them all. (Hooking every boundary at once can hang a component
// that crosses R ranges in a chain of up to R roots; the finds walk such chains
// through L1 and halve them, and measured faster than hooking the boundaries in
// the level order of a merge tree, one launch per level.) When the list outgrows
// its space the global pass falls back to one full arc scan.
constexpr int kLocalThreads = 512;

// Local union-find in shared memory with 16-bit parents (range-local ids < 2^15).
__device__ __forceinline__ int32_t sm_find(uint16_t *par, int32_t v)
{
    while (true) {
        int32_t p = par[v];
        if (p == v) return v;
        int32_t gp = par[p];
        if (gp == p) return p;
        par[v] = (uint16_t)gp;
        v = gp;
    }
}

template <typename OffT>
__global__ void __launch_bounds__(kLocalThreads) k_cc_local(const OffT *__restrict__ off,
                                                            const int32_t *__restrict__ adj, int64_t n, int64_t nnz,
                                                            int V, int32_t *uf, int32_t *te_u, int32_t *te_v,
                                                            int32_t *te_a,
                                                            int2 *xl, int64_t xl_cap, long long *nxl, int *err,
                                                            bool vec)
{
    extern __shared__ __align__(16) unsigned char smem[];
    uint32_t *woff = reinterpret_cast<uint32_t *>(smem);                   // V+1 offsets, relative to the range
    uint16_t *par = reinterpret_cast<uint16_t *>(smem + (size_t)(V + 1) * 4 + 12);
    const int lane = threadIdx.x & 31;
    const int64_t nranges = (n + V - 1) / V;
    for (int64_t g = blockIdx.x; g < nranges; g += gridDim.x) {
        const int64_t v0 = g * V;
        const int cnt = (int)((n - v0) < V ? (n - v0) : V);
        const int64_t a_beg = off[v0], a_end = off[v0 + cnt];
        if (a_end - a_beg > (int64_t)0x7fffffff) {   // relative offsets are 32-bit
            if (threadIdx.x == 0) atomicOr(err, kErrIndex);
            continue;
        }
        __syncthreads();
        for (int i = threadIdx.x; i <= cnt; i += kLocalThreads) {
            woff[i] = (uint32_t)(off[v0 + i] - a_beg);
            if (i < cnt) par[i] = (uint16_t)i;
        }
        __syncthreads();
        // runs of kItems arcs aligned to kItems in the global arc order (two 16-byte
        // loads each); the range's arcs are [a_beg, a_end), relative [0, span)
        const int64_t a_al = a_beg & ~(int64_t)(kItems - 1);
        const int span = (int)(a_end - a_beg);
        const int64_t rounds = (a_end - a_al + (int64_t)kLocalThreads * kItems - 1) / ((int64_t)kLocalThreads * kItems);
        // every lane runs every round (warp-wide reservation of the list slots below)
        for (int64_t rd = 0; rd < rounds; ++rd) {
            const int64_t a0 = a_al + (rd * kLocalThreads + threadIdx.x) * kItems;
            const int r0 = (int)(a0 - a_beg);          // relative; the first run may start below 0
            int32_t dw[kItems], su[kItems];
            uint32_t xmask = 0;   // arcs to a later range
            if (r0 < span) {
                if (vec && a0 + kItems <= nnz) {
                    const int4 x = __ldcs(reinterpret_cast<const int4 *>(adj + a0));
                    const int4 y = __ldcs(reinterpret_cast<const int4 *>(adj + a0) + 1);
                    dw[0] = x.x; dw[1] = x.y; dw[2] = x.z; dw[3] = x.w;
                    dw[4] = y.x; dw[5] = y.y; dw[6] = y.z; dw[7] = y.w;
                } else {
#pragma unroll
                    for (int j = 0; j < kItems; ++j) dw[j] = a0 + j < nnz ? __ldcs(adj + a0 + j) : 0;
                }
                const uint32_t rs = r0 > 0 ? (uint32_t)r0 : 0u;
                int lo = 0, hi = cnt - 1;   // the vertex whose list holds the run's first arc
                while (lo < hi) {
                    int mid = (lo + hi + 1) >> 1;
                    if (woff[mid] <= rs) lo = mid; else hi = mid - 1;
                }
#pragma unroll
                for (int j = 0; j < kItems; ++j) {
                    const int r = r0 + j;
                    su[j] = -1;
                    if (r < 0 || r >= span) continue;
                    while (woff[lo + 1] <= (uint32_t)r) ++lo;
                    const int64_t lw = (int64_t)dw[j] - v0;
                    if (lw <= lo) continue;                  // each edge once, from its smaller end
                    su[j] = lo;
                    if (lw >= cnt) xmask |= 1u << j;         // to a later range: the global pass
                }
            }
            // reserve list slots: one atomic per warp and round with such arcs
            const int xc = __popc(xmask);
            int xpre = xc;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, xpre, o);
                if (lane >= o) xpre += y;
            }
            long long xb = 0;
            const int xtot = __shfl_sync(0xffffffffu, xpre, 31);
            if (lane == 31 && xtot) xb = (long long)atomicAdd((unsigned long long *)nxl, (unsigned long long)xtot);
            xb = __shfl_sync(0xffffffffu, xb, 31) + (xpre - xc);
            if (r0 >= span) continue;
#pragma unroll
            for (int j = 0; j < kItems; ++j) {
                if (su[j] < 0) continue;
                if ((xmask >> j) & 1u) {
                    if (xb < xl_cap) xl[xb] = make_int2((int32_t)(v0 + su[j]), dw[j]);
                    ++xb;
                    continue;
                }
                const int32_t lw = (int32_t)(dw[j] - v0);
                int32_t ru = sm_find(par, su[j]), rv = sm_find(par, lw);
                for (int it = 0; it < kUniteCap && ru != rv; ++it) {
                    const int32_t h = ru > rv ? ru : rv, l = ru > rv ? rv : ru;
                    const int32_t old = atomicCAS(par + h, (unsigned short)h, (unsigned short)l);
                    if (old == h) {
                        tree_edge(te_u, te_v, te_a, (int32_t)(v0 + h), (int32_t)(v0 + su[j]), dw[j], a0 + j);
                        ru = rv;   // joined
                        break;
                    }
                    ru = sm_find(par, old);
                    rv = sm_find(par, l);
                }
                if (ru != rv) atomicOr(err, kErrUnite);   // the cap ended the retries: the union is lost
            }
        }
        __syncthreads();
        for (int i = threadIdx.x; i < cnt; i += kLocalThreads) {
            int32_t r = i;
            while (par[r] != r) r = par[r];
            uf[v0 + i] = (int32_t)(v0 + r);
        }
    }
}

// Global hooks of the gathered edges; when the list did not fit, every edge
// between ranges is hooked from a full arc scan instead.
template <typename OffT>
__global__ void __launch_bounds__(kThreads) k_cc_hook_cross(const OffT *__restrict__ off,
                                                            const int32_t *__restrict__ adj, int64_t nnz,
                                                            const int32_t *__restrict__ tile_v, int64_t ntiles, int V,
                                                            const int2 *__restrict__ xl, int64_t xl_cap,
                                                            const long long *__restrict__ nxl, int32_t *uf,
                                                            int32_t *te_u, int32_t *te_v, int32_t *te_a, int *err,
                                                            bool vec)
{
    const long long nx = *nxl;
    if (nx <= xl_cap) {
        for (int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x; i < nx; i += (int64_t)gridDim.x * kThreads) {
            const int2 e = xl[i];
            const int32_t r = uf_unite(uf, e.x, e.y, err);
            if (r >= 0) tree_edge(te_u, te_v, te_a, r, e.x, e.y, -1);   // (the list keeps no positions)
        }
        return;
    }
    __shared__ OffT win[kCtaWin];
    ArcTile<OffT> at;
    const int64_t nct = (ntiles + kWarpsPerCta - 1) / kWarpsPerCta;
    for (int64_t t = blockIdx.x; t < nct; t += gridDim.x) {
        arc_cta_tile_sources(off, nnz, tile_v, ntiles, t, win, at);
        if (!at.cnt) continue;
        int32_t d[kItems];
        arc_tile_targets(adj, at.a0, at.cnt, vec, d);
#pragma unroll
        for (int j = 0; j < kItems; ++j) {
            if (j >= at.cnt || at.src[j] >= d[j] || at.src[j] / V == d[j] / V) continue;
            int32_t r = uf_unite(uf, at.src[j], d[j], err);
            if (r >= 0) tree_edge(te_u, te_v, te_a, r, at.src[j], d[j], at.a0 + j);
        }
    }
}

size_t cc_local_smem(int V, bool off64)
{
    (void)off64;
    return (size_t)(V + 1) * 4 + 12 + (size_t)V * 2;
}

cudaError_t prepare_cc_local(int V)
{
    cudaError_t e = cudaFuncSetAttribute(k_cc_local<int32_t>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)cc_local_smem(V, false));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_cc_local<int64_t>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)cc_local_smem(V, true));
    return e;
}

template <typename OffT>
cudaError_t launch_first_cc(const Dev &d, const OffT *off, const int32_t *adj, int64_t n, int64_t nnz,
                            int cc_sample, int cc_local, int cc_ldd, int hub_deg, bool vec, const Launch &L)
{
    const int64_t ntiles = ceil_div(nnz, kWTile);
    const int gv = grid_for(L, ceil_div(n, kThreads));
    const int ga = grid_for(L, ceil_div(ntiles, kWarpsPerCta));
    long long *nhub = d.counters + 14;
    const cudaError_t e0 = cudaMemsetAsync(nhub, 0, sizeof(long long), L.s);
    if (e0 != cudaSuccess) return e0;
    // the tree edges' CSR positions are kept only where hubs are in use (their keys read them)
    int32_t *te_a = hub_deg > 0 ? d.te_a : nullptr;
    int32_t *maxdeg = reinterpret_cast<int32_t *>(d.counters + 5);
    const cudaError_t e1 = cudaMemsetAsync(maxdeg, 0, sizeof(int32_t), L.s);
    if (e1 != cudaSuccess) return e1;
    k_cc_init<OffT><<<gv, kThreads, 0, L.s>>>(off, n, nnz, d.tile_v, ntiles, d.uf, d.te_u, hub_deg, d.hubidx,
                                              d.hubvert, d.hub_cap, nhub, maxdeg);
    L.mark("k_cc_init");
    if (nnz > 0) {
        if (cc_local > 0) {
            const int64_t nr = ceil_div(n, cc_local);
            const int gl = (int)(nr < L.grid ? nr : L.grid);
            long long *nxl = d.counters + 4;
            const cudaError_t e = cudaMemsetAsync(nxl, 0, sizeof(long long), L.s);
            if (e != cudaSuccess) return e;
            k_cc_local<OffT><<<gl, kLocalThreads, cc_local_smem(cc_local, sizeof(OffT) == 8), L.s>>>(
                off, adj, n, nnz, cc_local, d.uf, d.te_u, d.te_v, te_a, d.xl, d.xl_cap, nxl, d.err, vec);
            L.mark("k_cc_local");
            k_cc_hook_cross<OffT><<<ga, kThreads, 0, L.s>>>(off, adj, nnz, d.tile_v, ntiles, cc_local, d.xl,
                                                           d.xl_cap, nxl, d.uf, d.te_u, d.te_v, te_a, d.err, vec);
            L.mark("k_cc_hook_cross");
        } else if (cc_ldd > 0) {
            int32_t *flag = reinterpret_cast<int32_t *>(d.counters + 8);
            const cudaError_t e = launch_ldd_forest<OffT>(d, off, adj, n, nnz, cc_ldd, te_a, flag, L);
            if (e != cudaSuccess) return e;
            // when the list of edges between clusters overflowed, every arc as without
            // LDD; otherwise it returns at once
            k_cc_hook<OffT><<<ga, kThreads, 0, L.s>>>(off, adj, nnz, d.tile_v, ntiles, d.uf, d.te_u, d.te_v,
                                                     te_a, d.err, vec, flag);
            L.mark("k_cc_hook");
        } else if (cc_sample > 0) {
            int32_t *big = reinterpret_cast<int32_t *>(d.counters + 8);
            k_cc_sample<OffT><<<gv, kThreads, 0, L.s>>>(off, adj, n, cc_sample, d.uf, d.te_u, d.te_v, te_a,
                                                        d.err);
            L.mark("k_cc_sample");
            k_uf_compress<<<gv, kThreads, 0, L.s>>>(d.uf, n);
            L.mark("k_uf_compress");
            k_cc_pick_big<<<1, kThreads, 0, L.s>>>(d.uf, d.tile_v, ntiles, big);
            L.mark("k_cc_pick_big");
            k_mark_big<<<gv, kThreads, 0, L.s>>>(d.uf, n, big, d.bigb);
            L.mark("k_mark_big");
            // the long lists' chunks go to the local-first list's space (unused here)
            long long *nlq = d.counters + 15;
            const cudaError_t e = cudaMemsetAsync(nlq, 0, sizeof(long long), L.s);
            if (e != cudaSuccess) return e;
            k_cc_hook_rest<OffT><<<gv, kThreads, 0, L.s>>>(off, adj, n, d.uf, d.te_u, d.te_v, te_a, d.bigb, d.xl,
                                                           d.xl_cap, nlq, big, d.err);
            L.mark("k_cc_hook_rest");
            k_cc_hook_chunks<OffT><<<gv, kThreads, 0, L.s>>>(off, adj, d.xl, d.xl_cap, nlq, d.uf, d.te_u, d.te_v,
                                                             te_a, big, d.err);
            L.mark("k_cc_hook_chunks");
            // after a weak sample (see pick_big) the tiled pass; otherwise it returns at once
            k_cc_hook<OffT><<<ga, kThreads, 0, L.s>>>(off, adj, nnz, d.tile_v, ntiles, d.uf, d.te_u, d.te_v,
                                                     te_a, d.err, vec, big);
            L.mark("k_cc_hook");
        } else {
            k_cc_hook<OffT><<<ga, kThreads, 0, L.s>>>(off, adj, nnz, d.tile_v, ntiles, d.uf, d.te_u, d.te_v,
                                                     te_a, d.err, vec, nullptr);
            L.mark("k_cc_hook");
        }
    }
    k_uf_compress<<<gv, kThreads, 0, L.s>>>(d.uf, n);
    L.mark("k_uf_compress");
    if (nnz > 0 && cc_local <= 0 && cc_ldd > 0) return launch_ldd_reroot(d, n, L);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Last-CC (Algorithm 1, step 4) on the skeleton G' = plain tree edges + cross
// edges, by preorder number.
//  1. plain components: the low/high kernel left lp[p] = parent position for a
//     plain edge, flattened inside each 1024-position tile; positions referenced
//     from another tile (ext) are compacted and resolved by a halving walk and a
//     read-only flatten;
//  2. cross edges: union-find over the plain components' roots (hook the larger
//     position under the smaller); an arc u->w with first[w] > first[u] (its
//     direction bit) that is not a tree arc to a child is a back edge iff
//     first[w] <= last[u] (u an ancestor of w; Algorithm 1, Back), a cross edge
//     otherwise, and a tree arc to a child always passes as a back edge there;
//     arcs with first[w] < first[u] are left to the reverse arc;
//  3. every position's final root, the smallest vertex id of each component and
//     the label of every vertex: the id of its component's top vertex.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads) k_ext_compact(int64_t n, const uint8_t *__restrict__ ext, int32_t *qlist,
                                                          long long *nq)
{
    // kTile positions per CTA step (kItems per thread, striped), one atomic per step
    __shared__ int32_t warp_cnt[kThreads / 32];
    __shared__ long long block_base;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int64_t p0 = blockIdx.x * (int64_t)kTile; p0 < n; p0 += (int64_t)gridDim.x * kTile) {
        uint32_t on = 0;
#pragma unroll
        for (int k = 0; k < kItems; ++k) {
            const int64_t p = p0 + k * kThreads + threadIdx.x;
            if (p < n && ext[p]) on |= 1u << k;
        }
        const int mine = __popc(on);
        int inc = mine;
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += y;
        }
        if (lane == 31) warp_cnt[wid] = inc;
        __syncthreads();
        if (threadIdx.x == 0) {
            int32_t t = 0;
            for (int w = 0; w < kThreads / 32; ++w) t += warp_cnt[w];
            block_base = t ? (long long)atomicAdd((unsigned long long *)nq, (unsigned long long)t) : 0;
        }
        __syncthreads();
        long long q = block_base + inc - mine;
        for (int w = 0; w < wid; ++w) q += warp_cnt[w];
        __syncthreads();
#pragma unroll
        for (int k = 0; k < kItems; ++k)
            if ((on >> k) & 1u) qlist[q++] = (int32_t)(p0 + k * kThreads + threadIdx.x);
    }
}

// Cross-tile positions resolved to their plain roots in two passes, the way the
// union-find is flattened: first a walk with path halving from every listed
// position (every store writes an ancestor, so the pointer forest stays valid and
// the chains shrink for every later walker), then a read-only walk that stores
// each listed position's root (a halving store from another thread can then no
// longer overwrite a root with a non-root).
__global__ void __launch_bounds__(kThreads) k_ext_halve(const long long *__restrict__ nq_p,
                                                        const int32_t *__restrict__ qlist, int32_t *lp)
{
    const int64_t nq = *nq_p;
    for (int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x; i < nq; i += (int64_t)gridDim.x * kThreads)
        (void)uf_find(lp, qlist[i]);
}

__global__ void __launch_bounds__(kThreads) k_ext_finish(const long long *__restrict__ nq_p,
                                                         const int32_t *__restrict__ qlist, int32_t *lp)
{
    const int64_t nq = *nq_p;
    for (int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x; i < nq; i += (int64_t)gridDim.x * kThreads) {
        const int32_t q = qlist[i];
        lp[q] = uf_root(lp, q);
    }
}

__device__ __forceinline__ int32_t plain_root(const int32_t *lp, int64_t p)
{
    const int32_t t = lp[p];
    return t < (p & ~(int64_t)(kRmqTile - 1)) ? lp[t] : t;
}

// Per vertex {first, plain-component root} for the cross-edge passes (one 8-byte
// gather gives both), and a fresh union-find.
__global__ void __launch_bounds__(kThreads) k_plain_label(int64_t n, const int32_t *__restrict__ lp,
                                                          const int32_t *__restrict__ ord, int2 *cr, int32_t *uf)
{
    // kPer positions per thread and step, each round of their loads issued together
    constexpr int kPer = 4;
    const int64_t T = (int64_t)gridDim.x * kThreads;
    for (int64_t p0 = blockIdx.x * (int64_t)kThreads + threadIdx.x; p0 < n; p0 += T * kPer) {
        int32_t o[kPer], t[kPer];
#pragma unroll
        for (int k = 0; k < kPer; ++k) {
            const int64_t p = p0 + k * T;
            if (p >= n) continue;
            o[k] = ord[p];
            t[k] = lp[p];
        }
#pragma unroll
        for (int k = 0; k < kPer; ++k) {
            const int64_t p = p0 + k * T;
            if (p >= n) continue;
            if (t[k] < (p & ~(int64_t)(kRmqTile - 1))) t[k] = lp[t[k]];   // plain_root
        }
#pragma unroll
        for (int k = 0; k < kPer; ++k) {
            const int64_t p = p0 + k * T;
            if (p >= n) continue;
            cr[o[k]] = make_int2((int32_t)p, t[k]);
            uf[p] = (int32_t)p;
        }
    }
}

// Cross edges from their earlier endpoint: arc u->w with w later in preorder (its
// direction bit) is a cross edge iff first[w] > last[u], i.e. w lies after T_u;
// a tree arc to a child and a back edge to a descendant both fail that test, and
// arcs to earlier vertices are left to the reverse arc, so only half of the arcs
// gather anything.
template <typename OffT>
__global__ void __launch_bounds__(kThreads) k_last_cc_cross(const OffT *__restrict__ off, const int32_t *__restrict__ adj,
                                                            int64_t nnz, const int32_t *__restrict__ tile_v,
                                                            int64_t ntiles, const int2 *__restrict__ cr,
                                                            const int32_t *__restrict__ lastp,
                                                            const uint8_t *__restrict__ dirb, int32_t *uf, int *err,
                                                            bool vec, const int32_t *__restrict__ sampled)
{
    if (sampled && sampled[1]) return;   // after a strong sample the by-vertex pass runs instead
    __shared__ OffT win[kCtaWin];
    ArcTile<OffT> at;
    const int64_t nct = (ntiles + kWarpsPerCta - 1) / kWarpsPerCta;
    for (int64_t t = blockIdx.x; t < nct; t += gridDim.x) {
        arc_cta_tile_sources(off, nnz, tile_v, ntiles, t, win, at);
        if (!at.cnt) continue;
        const uint32_t bits = __ldg(dirb + (at.a0 >> 3));
        if (!bits) continue;
        int32_t d[kItems];
        arc_tile_targets(adj, at.a0, at.cnt, vec, d);
        int32_t cur = -1, lastu = 0, ru = -1;
        int2 cs = make_int2(0, 0);
#pragma unroll
        for (int j = 0; j < kItems; ++j) {
            if (j >= at.cnt || !((bits >> j) & 1u)) continue;
            if (at.src[j] != cur) {
                cur = at.src[j];
                cs = __ldg(cr + cur);
                lastu = __ldg(lastp + cs.x);
                ru = -1;
            }
            const int2 cd = __ldg(cr + d[j]);
            if (cd.y == cs.y || cd.x <= lastu) continue;
            if (ru < 0) ru = uf_find(uf, cs.y);
            const int32_t rv = uf_find(uf, cd.y);
            if (rv == ru) continue;
            uf_unite(uf, ru, rv, err);
            ru = -1;
        }
    }
}

// Sampling variant of the cross-edge pass (the Afforest idea applied to G'):
// first the first K arcs of every vertex are tested and their cross edges united,
// then the component holding most sampled positions is found, and a pass by
// vertex goes through the arcs of every vertex outside it (membership fixed
// before that pass, see k_mark_big). A skipped vertex's edges are still seen from
// their other ends, so here cross edges are tested from both ends: towards a later
// vertex w as above, and towards an earlier one iff first[u] > last[w] (u after
// T_w; a parent arc and a back edge to an ancestor fail it).
__device__ __forceinline__ bool cross_from(int32_t fu, int32_t lastu, int32_t fw, bool later,
                                           const int32_t *__restrict__ lastp)
{
    return later ? fw > lastu : fu > __ldg(lastp + fw);
}

// One vertex per thread: its first K arcs other than the tree arc to its parent
// (which is never a cross edge, and under sampled hooking is usually the first
// arc), their gathers issued together before the unions (a tree root has no
// cross edges and is passed over).
template <typename OffT, int K>
__global__ void __launch_bounds__(kThreads) k_lcc_sample(const OffT *__restrict__ off, const int32_t *__restrict__ adj,
                                                         int64_t n, const int2 *__restrict__ fp,
                                                         const int2 *__restrict__ cr, const int32_t *__restrict__ lastp,
                                                         const uint8_t *__restrict__ dirb, int32_t *uf, int *err)
{
    for (int64_t v = blockIdx.x * (int64_t)kThreads + threadIdx.x; v < n; v += (int64_t)gridDim.x * kThreads) {
        const int32_t par = fp[v].y;
        if (par < 0) continue;
        const int64_t b = off[v];
        const int64_t deg = off[v + 1] - b;
        const int cntl = deg < K + 1 ? (int)deg : K + 1;
        const int2 cs = cr[v];
        int32_t wl[K + 1];
#pragma unroll
        for (int j = 0; j <= K; ++j) wl[j] = j < cntl ? adj[b + j] : -1;
        int sk = K;   // the parent arc's index among the first K arcs, else K
#pragma unroll
        for (int j = K - 1; j >= 0; --j)
            if (wl[j] == par) sk = j;
        const int32_t lastu = __ldg(lastp + cs.x);
        int2 cd[K];
        bool later[K], ok[K];
#pragma unroll
        for (int i = 0; i < K; ++i) {
            const int idx = i < sk ? i : i + 1;
            ok[i] = idx < cntl;
            cd[i] = ok[i] ? __ldg(cr + wl[idx]) : cs;
            later[i] = ok[i] && dir_bit(dirb, b + idx);
        }
#pragma unroll
        for (int i = 0; i < K; ++i) {
            if (!ok[i] || cd[i].y == cs.y || !cross_from(cs.x, lastu, cd[i].x, later[i], lastp)) continue;
            uf_unite(uf, cs.y, cd[i].y, err);
        }
    }
}

// Flatten the union-find over positions (roots only, see uf_root).
__global__ void __launch_bounds__(kThreads) k_pos_compress(int32_t *uf, int64_t n)
{
    const int64_t n_pad = (n + 31) & ~31ll;
    for (int64_t p = blockIdx.x * (int64_t)kThreads + threadIdx.x; p < n_pad; p += (int64_t)gridDim.x * kThreads)
        uf_flatten_warp(uf, p, p < n);
}

// The full cross-edge pass after sampling, by vertex: a vertex whose plain root
// is outside the sampled component tests all its arcs, in both directions; a lane
// takes a list of up to kRestShort arcs alone, longer lists are then tested by the
// whole warp, one list at a time, and lists above kRestLong arcs go to the chunk
// queue (see rest_queue). Where sampling gathered nearly every vertex, this reads
// fp, cr and the bitmap and little else.
__device__ __forceinline__ void cross_unite_warp(const int32_t *__restrict__ adj, const int2 *__restrict__ cr,
                                                 const int32_t *__restrict__ lastp, const uint8_t *__restrict__ dirb,
                                                 int32_t *uf, int *err, int32_t fu, int32_t ru, int32_t lu,
                                                 int64_t b, int64_t e, int lane)
{
    for (int64_t a = b + lane; a < e; a += 32) {
        const int2 cd = __ldg(cr + adj[a]);
        if (cd.y == ru || !cross_from(fu, lu, cd.x, dir_bit(dirb, a), lastp)) continue;
        uf_unite(uf, ru, cd.y, err);
    }
}

template <typename OffT>
__global__ void __launch_bounds__(kThreads) k_last_cc_cross_rest(const OffT *__restrict__ off,
                                                                 const int32_t *__restrict__ adj, int64_t n,
                                                                 const int2 *__restrict__ fp,
                                                                 const int2 *__restrict__ cr,
                                                                 const int32_t *__restrict__ lastp,
                                                                 const uint8_t *__restrict__ dirb, int32_t *uf,
                                                                 const uint32_t *__restrict__ bigb, int2 *lq,
                                                                 int64_t lq_cap, long long *lq_n,
                                                                 const int32_t *__restrict__ sampled, int *err)
{
    if (!sampled[1]) return;   // a weak sample: the tiled full pass runs instead
    const int lane = threadIdx.x & 31;
    const int64_t n_pad = (n + 31) & ~31ll;
    for (int64_t v = blockIdx.x * (int64_t)kThreads + threadIdx.x; v < n_pad; v += (int64_t)gridDim.x * kThreads) {
        int64_t b = 0, e = 0;
        int2 cs = make_int2(0, 0);
        int32_t lastu = 0;
        if (v < n && fp[v].y >= 0) {
            cs = cr[v];
            if (!test_bit(bigb, cs.y)) {
                b = off[v];
                e = off[v + 1];
                lastu = __ldg(lastp + cs.x);
            }
        }
        const bool lng = e - b > kRestShort;
        if (!lng) {
            for (int64_t a = b; a < e; ++a) {
                const int2 cd = __ldg(cr + adj[a]);
                if (cd.y == cs.y || !cross_from(cs.x, lastu, cd.x, dir_bit(dirb, a), lastp)) continue;
                uf_unite(uf, cs.y, cd.y, err);
            }
        }
        unsigned todo = __ballot_sync(0xffffffffu, lng);
        while (todo) {
            const int src = __ffs(todo) - 1;
            todo &= todo - 1;
            const int64_t bb = __shfl_sync(0xffffffffu, b, src), ee = __shfl_sync(0xffffffffu, e, src);
            if (ee - bb > kRestLong &&
                rest_queue(lq, lq_cap, lq_n, (int32_t)__shfl_sync(0xffffffffu, v, src), ee - bb, lane))
                continue;
            cross_unite_warp(adj, cr, lastp, dirb, uf, err, __shfl_sync(0xffffffffu, cs.x, src),
                             __shfl_sync(0xffffffffu, cs.y, src), __shfl_sync(0xffffffffu, lastu, src), bb, ee, lane);
        }
    }
}

// The queued chunks of long lists, a warp per chunk.
template <typename OffT>
__global__ void __launch_bounds__(kThreads) k_last_cc_cross_chunks(const OffT *__restrict__ off,
                                                                   const int32_t *__restrict__ adj,
                                                                   const int2 *__restrict__ cr,
                                                                   const int32_t *__restrict__ lastp,
                                                                   const uint8_t *__restrict__ dirb,
                                                                   const int2 *__restrict__ lq, int64_t lq_cap,
                                                                   const long long *__restrict__ lq_n, int32_t *uf,
                                                                   const int32_t *__restrict__ sampled, int *err)
{
    if (!sampled[1]) return;
    const int lane = threadIdx.x & 31;
    const int64_t nq = *lq_n < lq_cap ? *lq_n : lq_cap;
    const int64_t warps = (int64_t)gridDim.x * (kThreads / 32);
    for (int64_t i = (blockIdx.x * (int64_t)kThreads + threadIdx.x) >> 5; i < nq; i += warps) {
        const int2 q = lq[i];
        if (q.x < 0) continue;
        const int2 cs = cr[q.x];
        const int64_t b = off[q.x] + (int64_t)q.y * kRestChunk, end = off[q.x + 1];
        cross_unite_warp(adj, cr, lastp, dirb, uf, err, cs.x, cs.y, __ldg(lastp + cs.x), b,
                         b + kRestChunk < end ? b + kRestChunk : end, lane);
    }
}

// The same vote in Last-CC: an arc's source votes for the union-find root of its
// plain component (a tree root, alone in its plain component with no cross edge,
// does not vote).
__global__ void __launch_bounds__(kThreads) k_pos_pick_big(int32_t *uf, const int32_t *__restrict__ tile_v,
                                                           int64_t ntiles, const int2 *__restrict__ fp,
                                                           const int2 *__restrict__ cr, int32_t *big)
{
    pick_big(tile_v, ntiles, [&](int32_t v) { return fp[v].y >= 0 ? uf_find(uf, cr[v].y) : -1; }, big);
}

// Final labels. Every position's skeleton component root r (its top vertex has
// position r), the label of its vertex (the top vertex's id; roots are their own
// label), and the smallest vertex id of every class (lanes with the same root
// reduce first, and a read of the current minimum, stale values only costing an
// extra atomic, filters most of the remaining atomics).
// A top vertex t heads nothing itself: its BCC is its class plus the head p(t)
// (the tree edge above a top is a fence, so p(t) lies outside the class;
// Algorithm 1's head loop stores p(v) for every v whose parent has another label,
// and all of one label's writers agree, t among them). So the labels are counted
// here and each adds one to the count of labels its head heads (articulation
// points and root heads need it). The labels go to their own array: the
// union-find over positions is still being read.
__global__ void __launch_bounds__(kThreads) k_final_label(int64_t n, const int32_t *__restrict__ lp,
                                                          const int32_t *__restrict__ uf,
                                                          const int32_t *__restrict__ ord,
                                                          const int32_t *__restrict__ porig, int32_t *lab,
                                                          int32_t *smin, int32_t *nh, fbcc_stats *stats, int *err)
{
    long long c = 0;
    const int64_t n_pad = (n + 31) & ~31ll;
    for (int64_t p = blockIdx.x * (int64_t)kThreads + threadIdx.x; p < n_pad; p += (int64_t)gridDim.x * kThreads) {
        int32_t r = -1, v = INT32_MAX, l = -1;
        if (p < n) {
            const int32_t u = ord[p], x = porig[p];
            if (x < 0) {
                lab[u] = u;
            } else {
                r = uf_root(uf, plain_root(lp, p));
                l = ord[r];
                lab[u] = l;
                v = u;
                if (r == p) {
                    if (in_range(x, n, err)) atomicAdd(nh + x, 1);
                    ++c;
                }
            }
        }
        const unsigned peers = __match_any_sync(0xffffffffu, r);
        const int32_t m = (int32_t)__reduce_min_sync(peers, (unsigned)v);
        if (r >= 0 && (threadIdx.x & 31) == __ffs(peers) - 1 && in_range(l, n, err) && m < smin[l])
            atomicMin(smin + l, m);
    }
    block_count((long long *)&stats->n_bcc, c);
}

template <typename OffT>
cudaError_t launch_last_cc(const Dev &d, const OffT *off, const int32_t *adj, int64_t n, int64_t nnz,
                           int lcc_sample, bool vec, const Launch &L)
{
    cudaError_t e;
#define CK(x) do { e = (x); if (e != cudaSuccess) return e; } while (0)
    const int64_t ntiles = ceil_div(nnz, kWTile);
    const int gv = grid_for(L, ceil_div(n, kThreads));
    long long *nq = d.counters + 2;
    CK(cudaMemsetAsync(nq, 0, sizeof(long long), L.s));
    k_ext_compact<<<grid_for(L, ceil_div(n, kTile)), kThreads, 0, L.s>>>(n, d.ext, d.qlist, nq);
    L.mark("k_ext_compact");
    k_ext_halve<<<gv, kThreads, 0, L.s>>>(nq, d.qlist, d.lp);
    L.mark("k_ext_halve");
    k_ext_finish<<<gv, kThreads, 0, L.s>>>(nq, d.qlist, d.lp);
    L.mark("k_ext_finish");
    k_plain_label<<<gv, kThreads, 0, L.s>>>(n, d.lp, d.ord, d.cr, d.uf);
    L.mark("k_plain_label");
    if (nnz > 0 && lcc_sample > 0) {
        int32_t *big = reinterpret_cast<int32_t *>(d.counters + 9);
        switch (lcc_sample) {
        case 1: k_lcc_sample<OffT, 1><<<gv, kThreads, 0, L.s>>>(off, adj, n, d.fp, d.cr, d.lastp, d.dirb, d.uf, d.err); break;
        case 2: k_lcc_sample<OffT, 2><<<gv, kThreads, 0, L.s>>>(off, adj, n, d.fp, d.cr, d.lastp, d.dirb, d.uf, d.err); break;
        case 3: k_lcc_sample<OffT, 3><<<gv, kThreads, 0, L.s>>>(off, adj, n, d.fp, d.cr, d.lastp, d.dirb, d.uf, d.err); break;
        default: k_lcc_sample<OffT, 4><<<gv, kThreads, 0, L.s>>>(off, adj, n, d.fp, d.cr, d.lastp, d.dirb, d.uf, d.err); break;
        }
        L.mark("k_lcc_sample");
        k_pos_compress<<<gv, kThreads, 0, L.s>>>(d.uf, n);
        L.mark("k_pos_compress");
        k_pos_pick_big<<<1, kThreads, 0, L.s>>>(d.uf, d.tile_v, ntiles, d.fp, d.cr, big);
        L.mark("k_pos_pick_big");
        k_mark_big<<<gv, kThreads, 0, L.s>>>(d.uf, n, big, d.bigb);
        L.mark("k_mark_big");
        // the long lists' chunks go to the key list's space (used only by the outputs)
        long long *nlq = d.counters + 3;
        CK(cudaMemsetAsync(nlq, 0, sizeof(long long), L.s));
        k_last_cc_cross_rest<OffT><<<gv, kThreads, 0, L.s>>>(off, adj, n, d.fp, d.cr, d.lastp, d.dirb, d.uf, d.bigb,
                                                             d.klist, d.klist_cap, nlq, big, d.err);
        L.mark("k_last_cc_cross_rest");
        k_last_cc_cross_chunks<OffT><<<gv, kThreads, 0, L.s>>>(off, adj, d.cr, d.lastp, d.dirb, d.klist,
                                                               d.klist_cap, nlq, d.uf, big, d.err);
        L.mark("k_last_cc_cross_chunks");
        // after a weak sample the tiled pass; otherwise it returns at once
        k_last_cc_cross<OffT><<<grid_for(L, ceil_div(ntiles, kWarpsPerCta)), kThreads, 0, L.s>>>(
            off, adj, nnz, d.tile_v, ntiles, d.cr, d.lastp, d.dirb, d.uf, d.err, vec, big);
        L.mark("k_last_cc_cross");
    } else if (nnz > 0) {
        k_last_cc_cross<OffT><<<grid_for(L, ceil_div(ntiles, kWarpsPerCta)), kThreads, 0, L.s>>>(
            off, adj, nnz, d.tile_v, ntiles, d.cr, d.lastp, d.dirb, d.uf, d.err, vec, nullptr);
        L.mark("k_last_cc_cross");
    }
    CK(launch_final_labels(d, n, d.lp, d.uf, L));
#undef CK
    return cudaGetLastError();
}

cudaError_t launch_final_labels(const Dev &d, int64_t n, const int32_t *lp, const int32_t *uf, const Launch &L)
{
    cudaError_t e = cudaMemsetAsync(d.smin, 0x7f, n * sizeof(int32_t), L.s);
    if (e == cudaSuccess) e = cudaMemsetAsync(d.nh, 0, n * sizeof(int32_t), L.s);
    if (e != cudaSuccess) return e;
    k_final_label<<<grid_for(L, ceil_div(n, kThreads)), kThreads, 0, L.s>>>(n, lp, uf, d.ord, d.porig, d.lab, d.smin,
                                                                          d.nh, d.stats, d.err);
    L.mark("k_final_label");
    return cudaGetLastError();
}

template cudaError_t launch_first_cc<int32_t>(const Dev &, const int32_t *, const int32_t *, int64_t, int64_t, int,
                                              int, int, int, bool, const Launch &);
template cudaError_t launch_first_cc<int64_t>(const Dev &, const int64_t *, const int32_t *, int64_t, int64_t, int,
                                              int, int, int, bool, const Launch &);
template cudaError_t launch_last_cc<int32_t>(const Dev &, const int32_t *, const int32_t *, int64_t, int64_t, int,
                                             bool, const Launch &);
template cudaError_t launch_last_cc<int64_t>(const Dev &, const int64_t *, const int32_t *, int64_t, int64_t, int,
                                             bool, const Launch &);

}  // namespace fbcc
