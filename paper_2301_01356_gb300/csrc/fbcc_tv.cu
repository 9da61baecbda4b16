// The Tarjan-Vishkin skeleton, built explicitly: the space and speed foil of
// FAST-BCC's implicit one (section 3.2 and the appendix that gives the skeleton's
// three rules; the appendix on its running time and O(m) auxiliary space).
//
// With the spanning forest rooted and tagged as for FAST-BCC, the skeleton G' has
// one vertex per edge of G: a tree edge (u, p(u)) is vertex first[u] (its child's
// preorder number, in [0, n)), a non-tree edge is vertex n + a, a being its arc
// from the endpoint later in preorder (each non-tree edge has exactly one). Its
// edges, materialised as a list of pairs:
//  1. (u, p(u)) with every non-tree edge (u, v), first[v] < first[u];
//  2. (u, p(u)) with (v, p(v)) for every cross edge (u, v) (neither endpoint an
//     ancestor of the other);
//  3. (u, v = p(u)) with (v, p(v)) when v is not a root and some non-tree edge
//     leaves T_u for a vertex outside T_v: the tree edge is not a fence.
// Union-find over G' (hook the larger root under the smaller) then leaves each
// class of tree edges rooted at its smallest preorder number, its top vertex,
// which is the labelling Last-CC produces; the outputs step runs unchanged.
//
// Caller memory (tv_scratch_bytes): the union-find over n + nnz skeleton vertices,
// the pair list (at most nnz / 2 pairs of kind 1, nnz / 2 of kind 2 and n of kind
// 3), the identity plain-component pointers and a counter: 12 bytes per arc and
// 16 per vertex, against FAST-BCC's O(n) for the same step.
#include "fbcc_internal.cuh"

namespace fbcc {

namespace {

struct TvLayout {
    int32_t *uf;        // n + nnz
    int2 *pairs;        // cap
    int64_t cap;
    int32_t *lp;        // n: the identity
    long long *npairs;  // 1
    size_t bytes;
};

TvLayout tv_layout(char *base, int64_t n, int64_t nnz)
{
    TvLayout t{};
    size_t used = 0;
    auto take = [&](size_t bytes) {
        char *q = base ? base + used : nullptr;
        used += (bytes + 255) & ~size_t(255);
        return q;
    };
    t.uf = reinterpret_cast<int32_t *>(take((size_t)(n + nnz) * sizeof(int32_t)));
    t.cap = nnz + n;
    t.pairs = reinterpret_cast<int2 *>(take((size_t)t.cap * sizeof(int2)));
    t.lp = reinterpret_cast<int32_t *>(take((size_t)n * sizeof(int32_t)));
    t.npairs = reinterpret_cast<long long *>(take(sizeof(long long)));
    t.bytes = used;
    return t;
}

}  // namespace

size_t tv_scratch_bytes(int64_t n, int64_t nnz) { return tv_layout(nullptr, n, nnz).bytes; }

// Fresh union-find over the skeleton's vertices and the identity pointers.
__global__ void __launch_bounds__(kThreads) k_tv_init(int64_t n, int64_t nnz, int32_t *uf, int32_t *lp)
{
    for (int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x; i < n + nnz; i += (int64_t)gridDim.x * kThreads) {
        uf[i] = (int32_t)i;
        if (i < n) lp[i] = (int32_t)i;
    }
}

// Kinds 1 and 2, from the non-tree arcs towards earlier vertices.
template <typename OffT>
__global__ void __launch_bounds__(kThreads) k_tv_arcs(const OffT *__restrict__ off, const int32_t *__restrict__ adj,
                                                      int64_t nnz, int64_t n, const int32_t *__restrict__ tile_v,
                                                      int64_t nwt, const int2 *__restrict__ fp,
                                                      const int2 *__restrict__ fl, const uint8_t *__restrict__ dirb,
                                                      int2 *pairs, int64_t cap, long long *npairs, bool vec)
{
    __shared__ OffT win_all[kWarpsPerCta * kWarpWin];
    OffT *win = win_all + (threadIdx.x >> 5) * kWarpWin;
    ArcTile<OffT> at;
    FOR_EACH_WARP_TILE(w, nwt)
    {
        arc_tile_sources(off, nnz, tile_v, w, win, at);
        int32_t d[kItems];
        arc_tile_targets(adj, at.a0, at.cnt, vec, d);
        const uint32_t bits = at.cnt ? __ldg(dirb + (at.a0 >> 3)) : 0u;
        int32_t cur = -1;
        int2 fs = make_int2(0, -1);
#pragma unroll
        for (int j = 0; j < kItems; ++j) {
            bool k1 = false, k2 = false;
            int2 fw = make_int2(0, 0);
            if (j < at.cnt && !((bits >> j) & 1u)) {   // the target lies earlier in preorder
                if (at.src[j] != cur) {
                    cur = at.src[j];
                    fs = __ldg(fp + cur);                 // {first, parent} of the source
                }
                if (d[j] != fs.y) {                      // not the tree arc to the parent
                    fw = __ldg(fl + d[j]);               // {first, last} of the target
                    k1 = true;
                    k2 = fs.x > fw.y;                    // the source lies after T_target: a cross edge
                }
            }
            warp_append<int2>(pairs, npairs, cap, k1, make_int2(fs.x, (int32_t)(n + at.a0 + j)));
            warp_append<int2>(pairs, npairs, cap, k2, make_int2(fs.x, fw.x));
        }
    }
}

// Kind 3, by vertex: the tree edge above v and the one above its parent, unless
// v's edge is a fence or the parent is a root.
__global__ void __launch_bounds__(kThreads) k_tv_tree(int64_t n, const int2 *__restrict__ fp,
                                                      const uint8_t *__restrict__ vbits, int2 *pairs, int64_t cap,
                                                      long long *npairs)
{
    const int64_t n_pad = (n + 31) & ~31ll;
    for (int64_t v = blockIdx.x * (int64_t)kThreads + threadIdx.x; v < n_pad; v += (int64_t)gridDim.x * kThreads) {
        bool k3 = false;
        int2 f = make_int2(0, -1), fpar = make_int2(0, -1);
        if (v < n) {
            f = fp[v];
            if (f.y >= 0 && !(vbits[v] & 2)) {
                fpar = __ldg(fp + f.y);
                k3 = fpar.y >= 0;
            }
        }
        warp_append<int2>(pairs, npairs, cap, k3, make_int2(f.x, fpar.x));
    }
}

// Union-find over the pair list.
__global__ void __launch_bounds__(kThreads) k_tv_unite(const int2 *__restrict__ pairs, int64_t cap,
                                                       const long long *__restrict__ npairs, int32_t *uf, int *err)
{
    const int64_t m = *npairs < cap ? *npairs : cap;
    if (*npairs > cap && blockIdx.x == 0 && threadIdx.x == 0) atomicOr(err, kErrIndex);   // (cap bounds every kind)
    for (int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x; i < m; i += (int64_t)gridDim.x * kThreads) {
        const int2 e = pairs[i];
        uf_unite(uf, e.x, e.y, err);
    }
}

template <typename OffT>
cudaError_t launch_tv_connect(const Dev &d, const OffT *off, const int32_t *adj, int64_t n, int64_t nnz,
                              const TvScratch &tv, bool vec, const Launch &L)
{
    const TvLayout t = tv_layout(static_cast<char *>(tv.mem), n, nnz);
    if (!tv.mem || tv.bytes < t.bytes) return cudaErrorInvalidValue;
    const int gv = grid_for(L, ceil_div(n + nnz, kThreads));
    cudaError_t e = cudaMemsetAsync(t.npairs, 0, sizeof(long long), L.s);
    if (e != cudaSuccess) return e;
    k_tv_init<<<gv, kThreads, 0, L.s>>>(n, nnz, t.uf, t.lp);
    L.mark("k_tv_init");
    const int64_t nwt = ceil_div(nnz, kWTile);
    if (nnz > 0) {
        k_tv_arcs<OffT><<<grid_for(L, ceil_div(nwt, kWarpsPerCta)), kThreads, 0, L.s>>>(
            off, adj, nnz, n, d.tile_v, nwt, d.fp, d.fl, d.dirb, t.pairs, t.cap, t.npairs, vec);
        L.mark("k_tv_arcs");
    }
    k_tv_tree<<<grid_for(L, ceil_div(n, kThreads)), kThreads, 0, L.s>>>(n, d.fp, d.vbits, t.pairs, t.cap, t.npairs);
    L.mark("k_tv_tree");
    k_tv_unite<<<gv, kThreads, 0, L.s>>>(t.pairs, t.cap, t.npairs, t.uf, d.err);
    L.mark("k_tv_unite");
    return launch_final_labels(d, n, t.lp, t.uf, L);
}

template cudaError_t launch_tv_connect<int32_t>(const Dev &, const int32_t *, const int32_t *, int64_t, int64_t,
                                                const TvScratch &, bool, const Launch &);
template cudaError_t launch_tv_connect<int64_t>(const Dev &, const int64_t *, const int32_t *, int64_t, int64_t,
                                                const TvScratch &, bool, const Launch &);

}  // namespace fbcc
