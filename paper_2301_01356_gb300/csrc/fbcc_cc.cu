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

// tile_v[t] = source of arc t*kTile; tile_v[ntiles] = source of the last arc.
// Also resets the union-find and the tree-edge record.
template <typename OffT>
__global__ void __launch_bounds__(kThreads) k_cc_init(const OffT *__restrict__ off, int64_t n, int64_t nnz,
                                                      int32_t *tile_v, int64_t ntiles, int32_t *uf,
                                                      int32_t *te_u)
{
    for (int64_t v = blockIdx.x * (int64_t)kThreads + threadIdx.x; v < n; v += (int64_t)gridDim.x * kThreads) {
        uf[v] = (int32_t)v;
        te_u[v] = -1;
        int64_t b = off[v], e = off[v + 1];
        if (e > b) {
            for (int64_t t = (b + kTile - 1) / kTile; t * kTile < e; ++t) tile_v[t] = (int32_t)v;
            if (b <= nnz - 1 && nnz - 1 < e) tile_v[ntiles] = (int32_t)v;
        }
    }
}

// Hook every edge u-v (from its arc with u < v). A successful CAS hooks root r
// and records u-v as the tree edge owned by r.
template <typename OffT>
__global__ void __launch_bounds__(kThreads) k_cc_hook(const OffT *__restrict__ off, const int32_t *__restrict__ adj,
                                                      int64_t nnz, const int32_t *__restrict__ tile_v, int64_t ntiles,
                                                      int32_t *uf, int32_t *te_u, int32_t *te_v, int *err, bool vec)
{
    __shared__ OffT win[kOffWin];
    ArcTile<OffT> at;
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        arc_tile_sources(off, nnz, tile_v, t, win, at);
        if (!at.cnt) continue;
        int32_t d[kItems];
        arc_tile_targets(adj, at.a0, at.cnt, vec, d);
#pragma unroll
        for (int j = 0; j < kItems; ++j) {
            if (j >= at.cnt || at.src[j] >= d[j]) continue;
            int32_t r = uf_unite(uf, at.src[j], d[j], err);
            if (r >= 0) {
                te_u[r] = at.src[j];
                te_v[r] = d[j];
            }
        }
    }
}

// Sampling pre-pass: hook each vertex's first `k` neighbours (vertex-parallel).
template <typename OffT>
__global__ void __launch_bounds__(kThreads) k_cc_sample(const OffT *__restrict__ off, const int32_t *__restrict__ adj,
                                                        int64_t n, int k, int32_t *uf, int32_t *te_u, int32_t *te_v,
                                                        int *err)
{
    for (int64_t v = blockIdx.x * (int64_t)kThreads + threadIdx.x; v < n; v += (int64_t)gridDim.x * kThreads) {
        int64_t b = off[v], e = off[v + 1];
        for (int64_t a = b; a < e && a < b + k; ++a) {
            int32_t w = adj[a];
            int32_t r = uf_unite(uf, (int32_t)v, w, err);
            if (r >= 0) {
                te_u[r] = (int32_t)v;
                te_v[r] = w;
            }
        }
    }
}

// Full pass after sampling: arcs whose source already sits in the component of
// `big` are skipped (the same edge is still seen from its other endpoint, unless
// both endpoints are in that component, where it cannot join anything new).
template <typename OffT>
__global__ void __launch_bounds__(kThreads) k_cc_hook_skip(const OffT *__restrict__ off, const int32_t *__restrict__ adj,
                                                           int64_t nnz, const int32_t *__restrict__ tile_v,
                                                           int64_t ntiles, int32_t *uf, int32_t *te_u, int32_t *te_v,
                                                           const int32_t *big, int *err, bool vec)
{
    __shared__ OffT win[kOffWin];
    ArcTile<OffT> at;
    const int32_t root = *big;
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        arc_tile_sources(off, nnz, tile_v, t, win, at);
        if (!at.cnt) continue;
        bool any = false;
        int32_t rs[kItems];
        int32_t last_src = -1, last_root = root;
#pragma unroll
        for (int j = 0; j < kItems; ++j) {
            if (j < at.cnt) {
                if (at.src[j] != last_src) {
                    last_src = at.src[j];
                    last_root = uf_find(uf, last_src);
                }
                rs[j] = last_root;
                any |= last_root != root;
            } else {
                rs[j] = root;
            }
        }
        if (!any) continue;
        int32_t d[kItems];
        arc_tile_targets(adj, at.a0, at.cnt, vec, d);
#pragma unroll
        for (int j = 0; j < kItems; ++j) {
            if (j >= at.cnt || rs[j] == root) continue;
            int32_t r = uf_unite(uf, at.src[j], d[j], err);
            if (r >= 0) {
                te_u[r] = at.src[j];
                te_v[r] = d[j];
            }
        }
    }
}

// Flatten every set to its root. Only roots are ever stored, so concurrent
// threads cannot leave a vertex pointing at a non-root (see uf_root).
__global__ void __launch_bounds__(kThreads) k_uf_compress(int32_t *uf, int64_t n)
{
    for (int64_t v = blockIdx.x * (int64_t)kThreads + threadIdx.x; v < n; v += (int64_t)gridDim.x * kThreads)
        uf[v] = uf_root(uf, (int32_t)v);
}

// The root of the component holding most sampled vertices: a vote over a fixed
// subset of vertices (a single CTA).
__global__ void __launch_bounds__(kThreads) k_cc_pick_big(int32_t *uf, int64_t n, int32_t *big)
{
    __shared__ int32_t cand[kThreads];
    __shared__ int32_t cnt[kThreads];
    int64_t step = n / kThreads > 0 ? n / kThreads : 1;
    int64_t v = (int64_t)threadIdx.x * step;
    cand[threadIdx.x] = v < n ? uf_find(uf, (int32_t)v) : -1;
    __syncthreads();
    int c = 0;
    for (int i = 0; i < kThreads; ++i) c += cand[i] == cand[threadIdx.x];
    cnt[threadIdx.x] = cand[threadIdx.x] >= 0 ? c : 0;
    __syncthreads();
    if (threadIdx.x == 0) {
        int best = 0;
        for (int i = 1; i < kThreads; ++i)
            if (cnt[i] > cnt[best]) best = i;
        *big = cand[best] >= 0 ? cand[best] : 0;
    }
}

template <typename OffT>
cudaError_t launch_first_cc(const Dev &d, const OffT *off, const int32_t *adj, int64_t n, int64_t nnz,
                            int cc_sample, bool vec, const Launch &L)
{
    const int64_t ntiles = ceil_div(nnz, kTile);
    const int gv = grid_for(L, ceil_div(n, kThreads));
    const int ga = grid_for(L, ntiles);
    k_cc_init<OffT><<<gv, kThreads, 0, L.s>>>(off, n, nnz, d.tile_v, ntiles, d.uf, d.te_u);
    L.mark("k_cc_init");
    if (nnz > 0) {
        if (cc_sample > 0) {
            int32_t *big = reinterpret_cast<int32_t *>(d.counters + 8);
            k_cc_sample<OffT><<<gv, kThreads, 0, L.s>>>(off, adj, n, cc_sample, d.uf, d.te_u, d.te_v, d.err);
            L.mark("k_cc_sample");
            k_uf_compress<<<gv, kThreads, 0, L.s>>>(d.uf, n);
            L.mark("k_uf_compress");
            k_cc_pick_big<<<1, kThreads, 0, L.s>>>(d.uf, n, big);
            L.mark("k_cc_pick_big");
            k_cc_hook_skip<OffT><<<ga, kThreads, 0, L.s>>>(off, adj, nnz, d.tile_v, ntiles, d.uf, d.te_u, d.te_v,
                                                          big, d.err, vec);
            L.mark("k_cc_hook_skip");
        } else {
            k_cc_hook<OffT><<<ga, kThreads, 0, L.s>>>(off, adj, nnz, d.tile_v, ntiles, d.uf, d.te_u, d.te_v, d.err,
                                                     vec);
            L.mark("k_cc_hook");
        }
    }
    k_uf_compress<<<gv, kThreads, 0, L.s>>>(d.uf, n);
    L.mark("k_uf_compress");
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Last-CC: cross edges. The tree edges are skipped by their tree bit; a non-tree
// arc u->w with first[w] > first[u] is a back edge iff first[w] <= last[u] (u is
// an ancestor of w; Algorithm 1, Back) and a cross edge otherwise. Arcs with
// first[w] < first[u] are left to the reverse arc, where the comparison is made
// from the endpoint that comes first in preorder.
// ---------------------------------------------------------------------------
template <typename OffT>
__global__ void __launch_bounds__(kThreads) k_last_cc_cross(const OffT *__restrict__ off, const int32_t *__restrict__ adj,
                                                            int64_t nnz, const int32_t *__restrict__ tile_v,
                                                            int64_t ntiles, const uint32_t *__restrict__ tree_bits,
                                                            const int32_t *__restrict__ first,
                                                            const int32_t *__restrict__ last, int32_t *uf, int *err,
                                                            bool vec)
{
    __shared__ OffT win[kOffWin];
    ArcTile<OffT> at;
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        arc_tile_sources(off, nnz, tile_v, t, win, at);
        if (!at.cnt) continue;
        uint32_t tb = arc_tile_treebits(tree_bits, at.a0);
        int32_t d[kItems];
        arc_tile_targets(adj, at.a0, at.cnt, vec, d);
        int32_t cur = -1, ls = 0;
#pragma unroll
        for (int j = 0; j < kItems; ++j) {
            if (j >= at.cnt || ((tb >> j) & 1u)) continue;
            if (at.src[j] != cur) {
                cur = at.src[j];
                ls = __ldg(last + cur);
            }
            int32_t fd = __ldg(first + d[j]);
            if (fd > ls) uf_unite(uf, cur, d[j], err);
        }
    }
}

template <typename OffT>
cudaError_t launch_last_cc(const Dev &d, const OffT *off, const int32_t *adj, int64_t n, int64_t nnz,
                           bool vec, const Launch &L)
{
    const int64_t ntiles = ceil_div(nnz, kTile);
    if (nnz > 0)
        k_last_cc_cross<OffT><<<grid_for(L, ntiles), kThreads, 0, L.s>>>(off, adj, nnz, d.tile_v, ntiles, d.tree_bits,
                                                                        d.first, d.last, d.uf, d.err, vec);
        L.mark("k_last_cc_cross");
    k_uf_compress<<<grid_for(L, ceil_div(n, kThreads)), kThreads, 0, L.s>>>(d.uf, n);
    L.mark("k_uf_compress");
    return cudaGetLastError();
}

template cudaError_t launch_first_cc<int32_t>(const Dev &, const int32_t *, const int32_t *, int64_t, int64_t, int,
                                              bool, const Launch &);
template cudaError_t launch_first_cc<int64_t>(const Dev &, const int64_t *, const int32_t *, int64_t, int64_t, int,
                                              bool, const Launch &);
template cudaError_t launch_last_cc<int32_t>(const Dev &, const int32_t *, const int32_t *, int64_t, int64_t, bool,
                                             const Launch &);
template cudaError_t launch_last_cc<int64_t>(const Dev &, const int64_t *, const int32_t *, int64_t, int64_t, bool,
                                             const Launch &);

}  // namespace fbcc
