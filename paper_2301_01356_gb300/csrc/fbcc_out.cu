// Heads and outputs (Algorithm 1, the component-head loop after Last-CC; section
// 4.2 for why it is right).
//
// After Last-CC every non-root vertex v has a label l[v] (the top vertex of its
// skeleton component). For each v with l[v] != l[p(v)], p(v) is the head of
// label l[v]; every such writer of one label stores the same vertex (head lemma,
// section 4.2), the top vertex l itself among them, so head(l) = p(l) is read
// from the parent array rather than stored. Label l's BCC is {v : l[v] = l} plus
// its head.
//
// Expansion to the per-edge canonical form:
//  - articulation points: non-root heads, and roots that head two or more labels
//    (section 4.2, head/AP lemma; the root of a DFS-like argument in Theorem 1);
//  - each arc takes the label of its endpoint with the larger preorder number
//    (the child for a tree edge, the descendant for a back edge, either endpoint
//    for a cross edge, which lies in G' and so joins two equally labelled vertices);
//  - a tree edge p(v)-v is a bridge iff no edge leaves T_v (flag from tagging);
//    its BCC is {v, p(v)} and v's label class is {v}, so an arc is a bridge
//    exactly when the vertex that labels it carries the flag;
//  - canonical BCC numbers: the key of a BCC is its smallest arc id with
//    src < dst, which orders BCCs exactly like their smallest edge ids. Its source
//    is u0 = min(smin(l), head(l)) (the BCC's smallest vertex). If u0 lies in this BCC
//    only, the key is u0's first arc; otherwise u0's list is scanned for the arcs
//    of this BCC. Keys are set in a bitmap over arcs whose popcount prefix gives
//    each BCC its rank. (A label is the id of its class's top vertex; smin[l]
//    holds the class's smallest vertex id.)
#include "fbcc_internal.cuh"

namespace fbcc {

#define GRID_STRIDE(i, n) \
    for (int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x; i < (n); i += (int64_t)gridDim.x * kThreads)

// Articulation points, component count, and the keys that need no list scan.
// Each thread takes kVPer vertices per step and issues each round of their loads
// together (the pass is bound by dependent-load latency, not bandwidth).
constexpr int kVPer = 4;

template <typename OffT>
__global__ void __launch_bounds__(kThreads) k_ap_keys(int64_t n, const OffT *__restrict__ off,
                                                      const int2 *__restrict__ fp, const int32_t *__restrict__ lab,
                                                      const int32_t *__restrict__ nh,
                                                      const int32_t *__restrict__ smin,
                                                      uint8_t *is_ap, unsigned long long *key, uint8_t *scanv,
                                                      fbcc_stats *stats, int *err)
{
    long long nap = 0, ncc = 0;
    const int64_t T = (int64_t)gridDim.x * kThreads;
    for (int64_t v0 = blockIdx.x * (int64_t)kThreads + threadIdx.x; v0 < n; v0 += T * kVPer) {
        int2 f[kVPer];
        int32_t h[kVPer], l[kVPer];
#pragma unroll
        for (int k = 0; k < kVPer; ++k) {
            const int64_t v = v0 + k * T;
            f[k] = make_int2(0, -1);
            h[k] = 0;
            l[k] = -1;
            if (v < n) { f[k] = fp[v]; h[k] = nh[v]; l[k] = lab[v]; }
        }
        uint32_t lbl = 0;
        int32_t sm[kVPer];
#pragma unroll
        for (int k = 0; k < kVPer; ++k) {
            const int64_t v = v0 + k * T;
            sm[k] = 0;
            if (v >= n) continue;
            const bool root = f[k].y < 0;
            const uint8_t ap = root ? h[k] >= 2 : h[k] >= 1;
            is_ap[v] = ap;
            nap += ap;
            ncc += root;
            // a label's head is its parent
            if (!root && l[k] == v && in_range(f[k].y, n, err)) {
                lbl |= 1u << k;
                sm[k] = smin[v];
            }
        }
        int32_t u0[kVPer], hu[kVPer];
        bool pu[kVPer];
        OffT ou[kVPer];
#pragma unroll
        for (int k = 0; k < kVPer; ++k) {
            if (!((lbl >> k) & 1u)) continue;
            u0[k] = f[k].y < sm[k] ? f[k].y : sm[k];
            pu[k] = fp[u0[k]].y >= 0;
            hu[k] = nh[u0[k]];
            ou[k] = off[u0[k]];
        }
#pragma unroll
        for (int k = 0; k < kVPer; ++k) {
            if (!((lbl >> k) & 1u)) continue;
            const int64_t v = v0 + k * T;
            if ((int)pu[k] + hu[k] == 1) {   // u0 lies in this BCC only: its first arc is the key
                key[v] = (unsigned long long)ou[k];
            } else {
                key[v] = ~0ull;
                scanv[u0[k]] = 1;
            }
        }
    }
    block_count((long long *)&stats->n_ap, nap);
    block_count((long long *)&stats->n_cc, ncc);
}

// Keys of BCCs whose smallest vertex u0 lies in several BCCs: scan u0's arcs to
// larger neighbours; the smallest arc of each such BCC wins an atomicMin.
template <typename OffT>
__global__ void __launch_bounds__(kThreads) k_key_scan(const OffT *__restrict__ off, const int32_t *__restrict__ adj,
                                                       int64_t nnz, const int32_t *__restrict__ tile_v, int64_t ntiles,
                                                       const uint8_t *__restrict__ scanv,
                                                       const uint8_t *__restrict__ dirb,
                                                       const int32_t *__restrict__ lab,
                                                       const int2 *__restrict__ fp,
                                                       const int32_t *__restrict__ smin, unsigned long long *key,
                                                       bool vec)
{
    __shared__ OffT win_all[kWarpsPerCta * kWarpWin];
    OffT *win = win_all + (threadIdx.x >> 5) * kWarpWin;
    ArcTile<OffT> at;
    FOR_EACH_WARP_TILE(t, ntiles)
    {
        arc_tile_sources(off, nnz, tile_v, t, win, at);
        if (!at.cnt) continue;
        bool any = false;
        uint32_t sel = 0;
        int32_t prev = -1;
        bool ps = false;
#pragma unroll
        for (int j = 0; j < kItems; ++j) {
            if (j >= at.cnt) continue;
            if (at.src[j] != prev) {
                prev = at.src[j];
                ps = __ldg(scanv + prev) != 0;
            }
            if (ps) { sel |= 1u << j; any = true; }
        }
        if (!any) continue;
        int32_t d[kItems];
        arc_tile_targets(adj, at.a0, at.cnt, vec, d);
        const uint32_t bits = __ldg(dirb + (at.a0 >> 3));
        int32_t cur = -1, last_l = -1;
#pragma unroll
        for (int j = 0; j < kItems; ++j) {
            if (!((sel >> j) & 1u)) continue;
            const int32_t u = at.src[j], w = d[j];
            if (w < u) continue;
            if (u != cur) { cur = u; last_l = -1; }
            const int32_t x = (bits >> j) & 1u ? w : u;   // the endpoint later in preorder
            const int32_t l = __ldg(lab + x);
            if (l == last_l) continue;  // a later arc of the same BCC cannot be smaller
            last_l = l;
            const int32_t hd = __ldg(&fp[l].y), sm = __ldg(smin + l);
            if ((hd < sm ? hd : sm) == u) atomicMin(key + l, (unsigned long long)(at.a0 + j));
        }
    }
}

__global__ void __launch_bounds__(kThreads) k_key_bits(int64_t n, const int2 *__restrict__ fp,
                                                       const int32_t *__restrict__ lab,
                                                       const unsigned long long *__restrict__ key, uint32_t *key_bits,
                                                       int64_t nnz, int *err)
{
    // kVPer vertices per thread and step, each round of their loads issued together
    const int64_t T = (int64_t)gridDim.x * kThreads;
    for (int64_t v0 = blockIdx.x * (int64_t)kThreads + threadIdx.x; v0 < n; v0 += T * kVPer) {
        uint32_t lbl = 0;
#pragma unroll
        for (int k = 0; k < kVPer; ++k) {
            const int64_t v = v0 + k * T;
            if (v < n && fp[v].y >= 0 && lab[v] == v) lbl |= 1u << k;
        }
        unsigned long long ks[kVPer];
#pragma unroll
        for (int k = 0; k < kVPer; ++k)
            if ((lbl >> k) & 1u) ks[k] = key[v0 + k * T];
#pragma unroll
        for (int k = 0; k < kVPer; ++k)
            if (((lbl >> k) & 1u) && in_range((int64_t)ks[k], nnz, err)) set_bit(key_bits, (int64_t)ks[k]);
    }
}

// Rank of every label's key among all keys; heads go to their canonical slot. In
// a batch, ranks and heads are made local to the label's graph.
__global__ void __launch_bounds__(kThreads) k_rank(int64_t n, const int2 *__restrict__ fp,
                                                   const int32_t *__restrict__ lab,
                                                   const unsigned long long *__restrict__ key,
                                                   const uint32_t *__restrict__ key_bits,
                                                   const int32_t *__restrict__ key_pre,
                                                   int32_t *rank, int32_t *bcc_head,
                                                   Batch B, int64_t nnz, int *err)
{
    GRID_STRIDE(v, n)
    {
        const int32_t hd = fp[v].y;   // a label's head is its parent
        if (hd < 0 || lab[v] != v) continue;
        const int64_t k = (int64_t)key[v];
        if (!in_range(k, nnz, err)) continue;
        int32_t r = key_pre[k >> 5] + __popc(key_bits[k >> 5] & ((1u << (k & 31)) - 1u));
        if (B.G > 0) {
            const int32_t g = graph_of(B.vtx_base, B.G, v);
            const int64_t vb = B.vtx_base[g];
            r -= (int32_t)B.bcc_base[g];
            rank[v] = r;
            if (in_range(r, B.vtx_base[g + 1] - vb, err)) bcc_head[vb + r] = hd - (int32_t)vb;
        } else {
            rank[v] = r;
            if (in_range(r, n, err)) bcc_head[r] = hd;
        }
    }
}

// BCCs numbered before graph g: keys (set bits) below arc_base[g].
__global__ void __launch_bounds__(kThreads) k_bcc_base(Batch B, const uint32_t *__restrict__ key_bits,
                                                       const int32_t *__restrict__ key_pre)
{
    GRID_STRIDE(g, (int64_t)B.G + 1)
    {
        const int64_t a = B.arc_base[g];
        B.bcc_base[g] = key_pre[a >> 5] + __popc(key_bits[a >> 5] & ((1u << (a & 31)) - 1u));
    }
}

// Per vertex output word: BCC index of its label | bridge << 31.
__global__ void __launch_bounds__(kThreads) k_fo(int64_t n, const int2 *__restrict__ fp,
                                                 const int32_t *__restrict__ lab, const int32_t *__restrict__ rank,
                                                 const uint8_t *__restrict__ vbits, int32_t *word, fbcc_stats *stats)
{
    long long nb = 0;
    const int64_t T = (int64_t)gridDim.x * kThreads;
    for (int64_t v0 = blockIdx.x * (int64_t)kThreads + threadIdx.x; v0 < n; v0 += T * kVPer) {
        int32_t y[kVPer], l[kVPer];
        uint32_t br[kVPer];
#pragma unroll
        for (int k = 0; k < kVPer; ++k) {
            const int64_t v = v0 + k * T;
            y[k] = -1;
            if (v >= n) continue;
            y[k] = fp[v].y;
            l[k] = lab[v];
            br[k] = vbits[v] & 1u;
        }
#pragma unroll
        for (int k = 0; k < kVPer; ++k) {
            const int64_t v = v0 + k * T;
            if (v >= n) continue;
            int32_t w = 0;
            if (y[k] >= 0) {
                w = (int32_t)((uint32_t)rank[l[k]] | (br[k] << 31));
                nb += br[k];
            }
            word[v] = w;
        }
    }
    block_count((long long *)&stats->n_bridge, nb);
}

// Per-graph counts of a batch. A warp's vertices mostly belong to one graph:
// lanes of the same graph reduce together and one lane adds.
__global__ void __launch_bounds__(kThreads) k_batch_stats(int64_t n, Batch B, const int2 *__restrict__ fp,
                                                          const uint8_t *__restrict__ is_ap,
                                                          const uint8_t *__restrict__ vbits, const int *err)
{
    const int64_t n_pad = (n + 31) & ~31ll;
    const int lane = threadIdx.x & 31;
    for (int64_t v = blockIdx.x * (int64_t)kThreads + threadIdx.x; v < n_pad; v += (int64_t)gridDim.x * kThreads) {
        const bool in = v < n;
        const int32_t g = in ? graph_of(B.vtx_base, B.G, v) : -1;
        unsigned long long ap = 0, cc = 0, br = 0;
        if (in) {
            const bool root = fp[v].y < 0;
            ap = is_ap[v];
            cc = root;
            br = !root && (vbits[v] & 1u);
        }
        const unsigned peers = __match_any_sync(0xffffffffu, g);
        unsigned long long sap = 0, scc = 0, sbr = 0;
        for (int i = 0; i < 32; ++i) {
            unsigned long long a2 = __shfl_sync(0xffffffffu, ap, i), c2 = __shfl_sync(0xffffffffu, cc, i),
                               b2 = __shfl_sync(0xffffffffu, br, i);
            if ((peers >> i) & 1u) { sap += a2; scc += c2; sbr += b2; }
        }
        if (in && lane == __ffs(peers) - 1) {
            fbcc_stats *s = B.stats + g;
            if (sap) atomicAdd((unsigned long long *)&s->n_ap, sap);
            if (scc) atomicAdd((unsigned long long *)&s->n_cc, scc);
            if (sbr) atomicAdd((unsigned long long *)&s->n_bridge, sbr);
        }
    }
    GRID_STRIDE(g, (int64_t)B.G)
    {
        B.stats[g].n_bcc = B.bcc_base[g + 1] - B.bcc_base[g];
        B.stats[g].device_status = !*err ? FBCC_OK : (*err & kErrIndex) ? FBCC_E_INVALID : FBCC_E_ITER_LIMIT;
    }
}

// edge_bcc / is_bridge for every arc.
template <typename OffT>
__global__ void __launch_bounds__(kThreads, 6) k_edge_out(const OffT *__restrict__ off, const int32_t *__restrict__ adj,
                                                       int64_t nnz, const int32_t *__restrict__ tile_v, int64_t ntiles,
                                                       const int32_t *__restrict__ word,
                                                       const uint8_t *__restrict__ dirb, int32_t *edge_bcc,
                                                       uint8_t *is_bridge, bool vec, bool vec_out)
{
    __shared__ OffT win_all[kWarpsPerCta * kWarpWin];
    OffT *win = win_all + (threadIdx.x >> 5) * kWarpWin;
    ArcTile<OffT> at;
    FOR_EACH_WARP_TILE(t, ntiles)
    {
        arc_tile_sources(off, nnz, tile_v, t, win, at);
        if (!at.cnt) continue;
        int32_t d[kItems];
        arc_tile_targets(adj, at.a0, at.cnt, vec, d);
        const uint32_t bits = __ldg(dirb + (at.a0 >> 3));
        int32_t lab8[kItems];
        uint8_t br8[kItems];
        // x = the endpoint with the larger preorder number (the direction bit):
        // every arc's word gather is issued before any is used (a lane's sources
        // are few and neighbouring, so their repeated loads hit L1)
        int32_t wx[kItems];
#pragma unroll
        for (int j = 0; j < kItems; ++j)
            wx[j] = j < at.cnt ? __ldg(word + ((bits >> j) & 1u ? d[j] : at.src[j])) : 0;
#pragma unroll
        for (int j = 0; j < kItems; ++j) {
            lab8[j] = 0;
            br8[j] = 0;
            if (j >= at.cnt) continue;
            // If x's parent edge is a bridge, x's label class is {x} and that bridge
            // is the only edge of its BCC, so every arc labelled through x is the
            // bridge itself.
            const int32_t w = wx[j];
            lab8[j] = w & 0x7fffffff;
            br8[j] = (uint8_t)((uint32_t)w >> 31);
        }
        if (vec_out && at.cnt == kItems) {
            int4 *o = reinterpret_cast<int4 *>(edge_bcc + at.a0);
            __stcs(o, make_int4(lab8[0], lab8[1], lab8[2], lab8[3]));
            __stcs(o + 1, make_int4(lab8[4], lab8[5], lab8[6], lab8[7]));
            uint2 b;
            b.x = br8[0] | (br8[1] << 8) | (br8[2] << 16) | ((uint32_t)br8[3] << 24);
            b.y = br8[4] | (br8[5] << 8) | (br8[6] << 16) | ((uint32_t)br8[7] << 24);
            __stcs(reinterpret_cast<uint2 *>(is_bridge + at.a0), b);
        } else {
#pragma unroll
            for (int j = 0; j < kItems; ++j) {
                if (j < at.cnt) {
                    edge_bcc[at.a0 + j] = lab8[j];
                    is_bridge[at.a0 + j] = br8[j];
                }
            }
        }
    }
}

template <typename OffT>
cudaError_t launch_outputs(const Dev &d, const OffT *off, const int32_t *adj, int64_t n, int64_t nnz,
                           bool vec, int32_t *edge_bcc, int32_t *bcc_head, uint8_t *is_ap, uint8_t *is_bridge,
                           const Batch &B, const Launch &L)
{
    cudaError_t e;
#define CK(x) do { e = (x); if (e != cudaSuccess) return e; } while (0)
    const int gv = grid_for(L, ceil_div(n, kThreads));
    const int64_t ntiles = ceil_div(nnz, kWTile);
    const int64_t nwords = ceil_div(nnz, 32);
    CK(cudaMemsetAsync(d.scanv, 0, n, L.s));
    k_ap_keys<OffT><<<gv, kThreads, 0, L.s>>>(n, off, d.fp, d.lab, d.nh, d.smin, is_ap, d.key, d.scanv, d.stats, d.err);
    L.mark("k_ap_keys");
    CK(cudaGetLastError());
    if (nnz > 0) {
        k_key_scan<OffT><<<grid_for(L, ceil_div(ntiles, kWarpsPerCta)), kThreads, 0, L.s>>>(off, adj, nnz, d.tile_v, ntiles, d.scanv, d.dirb,
                                                                   d.lab, d.fp, d.smin, d.key, vec);
        L.mark("k_key_scan");
        CK(cudaMemsetAsync(d.key_bits, 0, nwords * sizeof(uint32_t), L.s));
        k_key_bits<<<gv, kThreads, 0, L.s>>>(n, d.fp, d.lab, d.key, d.key_bits, nnz, d.err);
        L.mark("k_key_bits");
        CK(cudaGetLastError());
        CK(launch_scan_popc(d, d.key_bits, d.key_pre, nwords, L));
        if (B.G > 0) {
            k_bcc_base<<<grid_for(L, ceil_div(B.G + 1, kThreads)), kThreads, 0, L.s>>>(B, d.key_bits, d.key_pre);
            L.mark("k_bcc_base");
        }
        k_rank<<<gv, kThreads, 0, L.s>>>(n, d.fp, d.lab, d.key, d.key_bits, d.key_pre, d.rank, bcc_head, B, nnz, d.err);
        L.mark("k_rank");
        k_fo<<<gv, kThreads, 0, L.s>>>(n, d.fp, d.lab, d.rank, d.vbits, d.word, d.stats);
        L.mark("k_fo");
        const bool vec_out = ((uintptr_t)edge_bcc & 15) == 0 && ((uintptr_t)is_bridge & 7) == 0;
        k_edge_out<OffT><<<grid_for(L, ceil_div(ntiles, kWarpsPerCta)), kThreads, 0, L.s>>>(off, adj, nnz, d.tile_v, ntiles,
                                                                   d.word, d.dirb, edge_bcc, is_bridge, vec, vec_out);
        L.mark("k_edge_out");
    } else if (B.G > 0) {
        CK(cudaMemsetAsync(B.bcc_base, 0, (B.G + 1) * sizeof(int64_t), L.s));
    }
    if (B.G > 0) {
        CK(cudaMemsetAsync(B.stats, 0, B.G * sizeof(fbcc_stats), L.s));
        k_batch_stats<<<gv, kThreads, 0, L.s>>>(n, B, d.fp, is_ap, d.vbits, d.err);
        L.mark("k_batch_stats");
    }
#undef CK
    return cudaGetLastError();
}

template cudaError_t launch_outputs<int32_t>(const Dev &, const int32_t *, const int32_t *, int64_t, int64_t, bool,
                                             int32_t *, int32_t *, uint8_t *, uint8_t *, const Batch &,
                                             const Launch &);
template cudaError_t launch_outputs<int64_t>(const Dev &, const int64_t *, const int32_t *, int64_t, int64_t, bool,
                                             int32_t *, int32_t *, uint8_t *, uint8_t *, const Batch &,
                                             const Launch &);

}  // namespace fbcc
