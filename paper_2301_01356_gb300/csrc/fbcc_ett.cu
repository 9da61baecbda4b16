// Rooting (Algorithm 1, step 2; section 2 "Euler tour technique" and section 5
// "Euler Tour Technique"): root every tree of the spanning forest at its
// component's smallest vertex and derive, per vertex, its parent, its preorder
// number first[v] and last[v] = first[v] + |T_v| - 1.
//
//  1. tree CSR: both arcs of every forest edge, grouped by source (counting sort),
//     with the index of each arc's reverse (twin);
//  2. Euler circuit: the arc u->v is followed by the arc after v->u in v's list,
//     cyclically (the paper's linking of u_i->v to v->u_{i+1}); each circuit is cut
//     before the root's first arc, which becomes the tour's head;
//  3. list ranking: rulers (every tour head plus one arc in `stride`) each walk
//     their successors up to the next ruler, recording owner and offset; the
//     short ruler lists are ranked by pointer jumping; every arc's tour position
//     follows from its ruler's suffix length (the paper samples sqrt(n) nodes and
//     chases pointers between them; the GPU takes many more rulers so that every
//     thread has a short walk);
//  4. preorder: an arc is a down arc iff it precedes its twin in the tour; a prefix
//     count of down arcs over tour positions numbers the vertices in preorder, and
//     the distance between a vertex's down and up arcs gives its subtree size.
// Tours are laid out at positions [2*base, 2*base + 2*size) of their component
// (base = preorder number of the root); the last two slots are padding, one of
// which counts 1 so that the prefix count restarts at each component's base.
#include "fbcc_internal.cuh"

namespace fbcc {

#define GRID_STRIDE(i, n) \
    for (int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x; i < (n); i += (int64_t)gridDim.x * kThreads)

template <typename OffT>
__device__ __forceinline__ int64_t find_arc(const OffT *__restrict__ off, const int32_t *__restrict__ adj,
                                            int32_t from, int32_t to)
{
    int64_t lo = off[from], hi = off[from + 1];
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (adj[mid] < to) lo = mid + 1; else hi = mid;
    }
    return lo;  // the arc exists in a valid (symmetric, sorted) CSR
}

// Tree degrees, and the tree bit of both arcs of every forest edge.
template <typename OffT>
__global__ void __launch_bounds__(kThreads) k_tree_count(const OffT *__restrict__ off, const int32_t *__restrict__ adj,
                                                         int64_t n, const int32_t *__restrict__ te_u,
                                                         const int32_t *__restrict__ te_v, int32_t *tdeg,
                                                         uint32_t *tree_bits)
{
    GRID_STRIDE(h, n)
    {
        int32_t u = te_u[h];
        if (u < 0) continue;
        int32_t v = te_v[h];
        atomicAdd(tdeg + u, 1);
        atomicAdd(tdeg + v, 1);
        set_bit(tree_bits, find_arc(off, adj, u, v));
        set_bit(tree_bits, find_arc(off, adj, v, u));
    }
}

__global__ void __launch_bounds__(kThreads) k_tree_fill(int64_t n, const int32_t *__restrict__ te_u,
                                                        const int32_t *__restrict__ te_v, const int32_t *__restrict__ toff,
                                                        int32_t *cursor, int32_t *tadj, int32_t *twin, int *err)
{
    GRID_STRIDE(h, n)
    {
        int32_t u = te_u[h];
        if (u < 0) continue;
        int32_t v = te_v[h];
        int32_t su = toff[u] + atomicAdd(cursor + u, 1);
        int32_t sv = toff[v] + atomicAdd(cursor + v, 1);
        if (!in_range(su, toff[u + 1], err) || !in_range(sv, toff[v + 1], err)) continue;
        tadj[su] = v;
        tadj[sv] = u;
        twin[su] = sv;
        twin[sv] = su;
    }
}

// succ[s] for s = x->y: the arc after twin(s) = y->x in y's list, cyclically.
__global__ void __launch_bounds__(kThreads) k_succ(int64_t n2, const int32_t *__restrict__ toff, int64_t n,
                                                   const int32_t *__restrict__ tadj, const int32_t *__restrict__ twin,
                                                   int32_t *succ, uint8_t *is_head)
{
    const int64_t A = toff[n];
    (void)n2;
    GRID_STRIDE(s, A)
    {
        int32_t y = tadj[s];
        int32_t nx = twin[s] + 1;
        succ[s] = nx < toff[y + 1] ? nx : toff[y];
        is_head[s] = 0;
    }
}

// Per component root r (uf[r] == r) with tree arcs: its first arc heads the tour;
// the arc entering r just before that one (the twin of r's last arc) ends it.
__global__ void __launch_bounds__(kThreads) k_tour_cut(int64_t n, const int32_t *__restrict__ uf,
                                                       const int32_t *__restrict__ toff, const int32_t *__restrict__ twin,
                                                       int32_t *succ, uint8_t *is_head)
{
    GRID_STRIDE(r, n)
    {
        if (uf[r] != r || toff[r + 1] == toff[r]) continue;
        is_head[toff[r]] = 1;
        succ[twin[toff[r + 1] - 1]] = -1;
    }
}

// Rulers: tour heads and every arc whose index is a multiple of the stride.
// link[s] = {succ[s], ruler id or -1}; relem[id] = s. Ids come from one atomic
// per CTA and iteration (a per-warp atomic on a single counter serialises).
__global__ void __launch_bounds__(kThreads) k_rulers(const int32_t *__restrict__ toff, int64_t n, int stride,
                                                     const int32_t *__restrict__ succ,
                                                     const uint8_t *__restrict__ is_head, int2 *link, int32_t *relem,
                                                     long long *nr)
{
    __shared__ int32_t warp_cnt[kThreads / 32];
    __shared__ long long block_base;
    const int64_t A = toff[n];
    const int64_t A_pad = (A + kThreads - 1) / kThreads * kThreads;  // whole CTAs take part
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int64_t s = blockIdx.x * (int64_t)kThreads + threadIdx.x; s < A_pad; s += (int64_t)gridDim.x * kThreads) {
        const bool in = s < A;
        const bool ruler = in && (is_head[s] || (s & (stride - 1)) == 0);
        const unsigned mask = __ballot_sync(0xffffffffu, ruler);
        if (lane == 0) warp_cnt[wid] = __popc(mask);
        __syncthreads();
        if (threadIdx.x == 0) {
            int32_t t = 0;
            for (int w = 0; w < kThreads / 32; ++w) t += warp_cnt[w];
            block_base = t ? (long long)atomicAdd((unsigned long long *)nr, (unsigned long long)t) : 0;
        }
        __syncthreads();
        int32_t before = 0;
        for (int w = 0; w < wid; ++w) before += warp_cnt[w];
        const long long base = block_base + before;
        __syncthreads();  // warp_cnt / block_base are rewritten next iteration
        if (!in) continue;
        int32_t id = -1;
        if (ruler) {
            id = (int32_t)(base + __popc(mask & ((1u << lane) - 1u)));
            relem[id] = (int32_t)s;
        }
        link[s] = make_int2(succ[s], id);
    }
}

// Each ruler walks its successors until the next ruler or the tour's end.
__global__ void __launch_bounds__(kThreads) k_chase(const int32_t *__restrict__ toff, int64_t n,
                                                    const long long *__restrict__ nr_p, const int32_t *__restrict__ relem,
                                                    const int2 *__restrict__ link, int32_t *owner, int32_t *offs,
                                                    int32_t *rnext, int32_t *rval, int32_t *rlen, int *err)
{
    const int64_t A = toff[n];
    const int64_t nr = *nr_p;
    GRID_STRIDE(r, nr)
    {
        int32_t s = relem[r];
        owner[s] = (int32_t)r;
        offs[s] = 0;
        int32_t acc = 1, nxr = -1;
        int32_t t = link[s].x;
        int64_t steps = 0;
        while (t >= 0) {
            int2 lk = link[t];
            if (lk.y >= 0) { nxr = lk.y; break; }
            owner[t] = (int32_t)r;
            offs[t] = acc++;
            t = lk.x;
            if (++steps > A) { atomicOr(err, kErrChase); break; }
        }
        rnext[r] = nxr;
        rval[r] = acc;
        rlen[r] = acc;
    }
}

// One pointer-jumping round on the ruler lists: val = suffix weight.
__global__ void __launch_bounds__(kThreads) k_jump(const long long *__restrict__ nr_p, const int32_t *__restrict__ nx_in,
                                                   const int32_t *__restrict__ val_in, int32_t *nx_out, int32_t *val_out)
{
    const int64_t nr = *nr_p;
    GRID_STRIDE(r, nr)
    {
        int32_t x = nx_in[r];
        if (x >= 0) {
            val_out[r] = val_in[r] + val_in[x];
            nx_out[r] = nx_in[x];
        } else {
            val_out[r] = val_in[r];
            nx_out[r] = -1;
        }
    }
}

// Component size at its root: 1 for an isolated root, else tour length / 2 + 1.
__global__ void __launch_bounds__(kThreads) k_comp_size(int64_t n, const int32_t *__restrict__ uf,
                                                        const int32_t *__restrict__ toff, const int2 *__restrict__ link,
                                                        const int32_t *__restrict__ sd, const long long *nr_p,
                                                        int32_t *csize, int *err)
{
    const int64_t nr = *nr_p;
    GRID_STRIDE(v, n)
    {
        int32_t c = 0;
        if (uf[v] == v) {
            c = 1;
            if (toff[v + 1] != toff[v]) {
                const int32_t id = link[toff[v]].y;
                if (in_range(id, nr, err)) c = sd[id] / 2 + 1;
            }
        }
        csize[v] = c;
    }
}

// Tour position of every tree arc: 2*base + L - (arcs from it to the tour's end).
__global__ void __launch_bounds__(kThreads) k_place(const int32_t *__restrict__ toff, int64_t n,
                                                    const int32_t *__restrict__ tadj, const int32_t *__restrict__ uf,
                                                    const int32_t *__restrict__ csize, const int32_t *__restrict__ vbase,
                                                    const int32_t *__restrict__ owner, const int32_t *__restrict__ offs,
                                                    const int32_t *__restrict__ sd, int32_t *pos, int32_t *tour,
                                                    int *err)
{
    const int64_t A = toff[n];
    GRID_STRIDE(s, A)
    {
        int32_t r = uf[tadj[s]];
        int32_t L = 2 * (csize[r] - 1);
        int32_t dist = sd[owner[s]] - offs[s];
        int32_t p = 2 * vbase[r] + L - dist;
        pos[s] = p;
        if (in_range(dist - 1, L, err)) tour[p] = (int32_t)s;
    }
}

// Per component root: padding slots and the root's own tags.
__global__ void __launch_bounds__(kThreads) k_root_tags(int64_t n, const int32_t *__restrict__ uf,
                                                        const int32_t *__restrict__ csize,
                                                        const int32_t *__restrict__ vbase, int32_t *tour, int32_t *first,
                                                        int32_t *last, int32_t *parent, int32_t *ord, int32_t *lastp,
                                                        int32_t *porig, int32_t *w1, int32_t *w2)
{
    GRID_STRIDE(r, n)
    {
        if (uf[r] != r) continue;
        int32_t b = vbase[r], sz = csize[r];
        tour[2 * b + 2 * sz - 2] = -2;
        tour[2 * b + 2 * sz - 1] = -1;
        first[r] = b;
        last[r] = b + sz - 1;
        parent[r] = -1;
        ord[b] = (int32_t)r;
        lastp[b] = b + sz - 1;
        porig[b] = -1;
        w1[b] = b;
        w2[b] = b;
    }
}

// Preorder from the tour (single-pass scan over the 2n tour positions).
__global__ void __launch_bounds__(kThreads) k_preorder(int64_t n2, const int32_t *__restrict__ tour,
                                                       const int32_t *__restrict__ pos, const int32_t *__restrict__ tadj,
                                                       const int32_t *__restrict__ twin, int32_t *first, int32_t *last,
                                                       int32_t *parent, int32_t *ord, int32_t *lastp, int32_t *porig,
                                                       int32_t *w1, int32_t *w2, long long *ticket, uint64_t *status,
                                                       int *err)
{
    const int64_t ntiles = (n2 + kTile - 1) / kTile;
    while (true) {
        int64_t t = scan_ticket(ticket);
        if (t >= ntiles) return;
        const int64_t p0 = t * kTile + (int64_t)threadIdx.x * kItems;
        long long v[kItems];
        int32_t arc[kItems], q[kItems];
#pragma unroll
        for (int j = 0; j < kItems; ++j) {
            int64_t p = p0 + j;
            int32_t s = p < n2 ? tour[p] : -1;
            if (s >= n2) { atomicOr(err, kErrIndex); s = -1; }
            arc[j] = s;
            q[j] = 0;
            if (s >= 0) {
                q[j] = pos[twin[s]];
                v[j] = p < q[j];
            } else {
                v[j] = s == -2;
            }
        }
        scan_tile_exclusive(v, t, status, err);
#pragma unroll
        for (int j = 0; j < kItems; ++j) {
            int64_t p = p0 + j;
            int32_t s = arc[j];
            if (s < 0 || p >= q[j]) continue;  // padding or an up arc
            int32_t vtx = tadj[s], x = tadj[twin[s]];
            int32_t fv = (int32_t)v[j] + 1;
            int32_t lv = fv + (int32_t)((q[j] - p + 1) / 2) - 1;
            if (!in_range(fv, n2 / 2, err) || !in_range(lv, n2 / 2, err)) continue;
            first[vtx] = fv;
            last[vtx] = lv;
            parent[vtx] = x;
            ord[fv] = vtx;
            lastp[fv] = lv;
            porig[fv] = x;
            w1[fv] = fv;
            w2[fv] = fv;
        }
    }
}

template <typename OffT>
cudaError_t launch_rooting(const Dev &d, const OffT *off, const int32_t *adj, int64_t n, int64_t nnz,
                           int ruler_stride, const Launch &L)
{
    (void)nnz;
    const int gv = grid_for(L, ceil_div(n, kThreads));
    const int ga = grid_for(L, ceil_div(2 * n, kThreads));
    cudaError_t e;
#define CK(x) do { e = (x); if (e != cudaSuccess) return e; } while (0)
    CK(cudaMemsetAsync(d.tdeg, 0, (n + 1) * sizeof(int32_t), L.s));
    k_tree_count<OffT><<<gv, kThreads, 0, L.s>>>(off, adj, n, d.te_u, d.te_v, d.tdeg, d.tree_bits);
    L.mark("k_tree_count");
    CK(cudaGetLastError());
    CK(launch_scan_i32(d, d.tdeg, d.toff, n, L));
    CK(cudaMemsetAsync(d.tdeg, 0, (n + 1) * sizeof(int32_t), L.s));
    k_tree_fill<<<gv, kThreads, 0, L.s>>>(n, d.te_u, d.te_v, d.toff, d.tdeg, d.tadj, d.twin, d.err);
    L.mark("k_tree_fill");
    k_succ<<<ga, kThreads, 0, L.s>>>(2 * n, d.toff, n, d.tadj, d.twin, d.succ, d.is_head);
    L.mark("k_succ");
    k_tour_cut<<<gv, kThreads, 0, L.s>>>(n, d.uf, d.toff, d.twin, d.succ, d.is_head);
    L.mark("k_tour_cut");
    long long *nr = d.counters + 1;
    CK(cudaMemsetAsync(nr, 0, sizeof(long long), L.s));
    k_rulers<<<ga, kThreads, 0, L.s>>>(d.toff, n, ruler_stride, d.succ, d.is_head, d.link, d.relem, nr);
    L.mark("k_rulers");
    // upper bound on the number of rulers: every tour head plus one per stride
    const int64_t rbound = n + ceil_div(2 * n, ruler_stride) + 1;
    const int gr = grid_for(L, ceil_div(rbound, kThreads));
    k_chase<<<gr, kThreads, 0, L.s>>>(d.toff, n, nr, d.relem, d.link, d.owner, d.offs, d.rnext[0], d.rval[0],
                                      d.rlen, d.err);
    L.mark("k_chase");
    int cur = 0;
    const int rounds = jump_rounds(rbound);
    for (int i = 0; i < rounds; ++i) {
        k_jump<<<gr, kThreads, 0, L.s>>>(nr, d.rnext[cur], d.rval[cur], d.rnext[cur ^ 1], d.rval[cur ^ 1]);
        L.mark("k_jump");
        cur ^= 1;
    }
    const int32_t *sd = d.rval[cur];
    k_comp_size<<<gv, kThreads, 0, L.s>>>(n, d.uf, d.toff, d.link, sd, nr, d.csize, d.err);
    L.mark("k_comp_size");
    CK(cudaGetLastError());
    CK(launch_scan_i32(d, d.csize, d.vbase, n, L));
    CK(cudaMemsetAsync(d.tour, 0xff, 2 * n * sizeof(int32_t), L.s));
    k_place<<<ga, kThreads, 0, L.s>>>(d.toff, n, d.tadj, d.uf, d.csize, d.vbase, d.owner, d.offs, sd, d.pos, d.tour,
                                      d.err);
    L.mark("k_place");
    k_root_tags<<<gv, kThreads, 0, L.s>>>(n, d.uf, d.csize, d.vbase, d.tour, d.first, d.last, d.parent, d.ord,
                                          d.lastp, d.porig, d.w1, d.w2);
    L.mark("k_root_tags");
    CK(cudaGetLastError());
    const int64_t ntiles = ceil_div(2 * n, kTile);
    CK(cudaMemsetAsync(d.counters, 0, sizeof(long long), L.s));
    CK(cudaMemsetAsync(d.scan_status, 0, ntiles * sizeof(uint64_t), L.s));
    k_preorder<<<grid_for(L, ntiles), kThreads, 0, L.s>>>(2 * n, d.tour, d.pos, d.tadj, d.twin, d.first, d.last,
                                                           d.parent, d.ord, d.lastp, d.porig, d.w1, d.w2, d.counters,
                                                           d.scan_status, d.err);
    L.mark("k_preorder");
#undef CK
    return cudaGetLastError();
}

template cudaError_t launch_rooting<int32_t>(const Dev &, const int32_t *, const int32_t *, int64_t, int64_t, int,
                                             const Launch &);
template cudaError_t launch_rooting<int64_t>(const Dev &, const int64_t *, const int32_t *, int64_t, int64_t, int,
                                             const Launch &);

}  // namespace fbcc
