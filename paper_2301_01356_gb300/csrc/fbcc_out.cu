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
//    is u0 = min(smin(l), head(l)) (the BCC's smallest vertex), and its target the
//    smallest neighbour of u0 in the BCC. Three cases:
//      * u0 lies in this BCC only: every neighbour of u0 is in it, and the key is
//        u0's first arc;
//      * u0 is the head h, h's list is long and h heads few labels for its
//        length: the neighbours of h in the BCC are exactly the class members
//        adjacent to h (two adjacent vertices of one BCC put their edge in it),
//        so each member smaller than the top (which is adjacent: the tree edge)
//        tests its adjacency to h by a binary search of its own list, the
//        smallest wins (kmin), and one search of h's list finds the key;
//      * otherwise (u0 is a head with a short list or with many labels for its
//        list, or a class member in several BCCs) u0's list is scanned, in
//        chunks of kKeyChunk arcs, for the arcs of its BCCs.
//    Keys are set in a bitmap over arcs whose popcount prefix gives each BCC its
//    rank. (A label is the id of its class's top vertex; smin[l] holds the class's
//    smallest vertex id.)
#include "fbcc_internal.cuh"

namespace fbcc {

#define GRID_STRIDE(i, n) \
    for (int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x; i < (n); i += (int64_t)gridDim.x * kThreads)

// Articulation points, component count, and the keys that need no list scan.
// Each thread takes kVPer vertices per step and issues each round of their loads
// together (the pass is bound by dependent-load latency, not bandwidth).
constexpr int kVPer = 4;

// Key of a label whose head is its BCC's smallest vertex: found by k_key_bits.
constexpr unsigned long long kKeyHead = ~1ull;
// Heads with at most this many arcs are scanned like the other listed vertices,
// and so are heads with at most kScanPerLabel arcs per label they head: one scan
// of such a list finds all their labels' keys for fewer loads than a search of it
// per label (a hub whose leaf children are each a bridge BCC).
constexpr int kHeadScan = 32;
constexpr int kScanPerLabel = 8;

template <typename OffT>
__global__ void __launch_bounds__(kThreads) k_ap_keys(int64_t n, const OffT *__restrict__ off,
                                                      const int2 *__restrict__ fp, const int32_t *__restrict__ lab,
                                                      const int32_t *__restrict__ nh,
                                                      const int32_t *__restrict__ smin,
                                                      uint8_t *is_ap, unsigned long long *key, int32_t *kmin,
                                                      uint8_t *scanv, long long *nhead_n, fbcc_stats *stats,
                                                      int *err)
{
    long long nap = 0, ncc = 0, nhead = 0;
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
        OffT ou[kVPer], oe[kVPer];
#pragma unroll
        for (int k = 0; k < kVPer; ++k) {
            if (!((lbl >> k) & 1u)) continue;
            u0[k] = f[k].y < sm[k] ? f[k].y : sm[k];
            pu[k] = fp[u0[k]].y >= 0;
            hu[k] = nh[u0[k]];
            ou[k] = off[u0[k]];
            oe[k] = off[u0[k] + 1];
        }
#pragma unroll
        for (int k = 0; k < kVPer; ++k) {
            if (!((lbl >> k) & 1u)) continue;
            const int64_t v = v0 + k * T;
            const int64_t deg = (int64_t)oe[k] - (int64_t)ou[k];
            if ((int)pu[k] + hu[k] == 1) {   // u0 lies in this BCC only: its first arc is the key
                key[v] = (unsigned long long)ou[k];
            } else if (f[k].y < sm[k] && deg > kHeadScan && deg > (int64_t)kScanPerLabel * hu[k]) {
                // u0 is a head with a long list: the class members find their adjacency
                // to it (the top is adjacent), and a search of its list the key
                key[v] = kKeyHead;
                kmin[v] = (int32_t)v;
                ++nhead;
            } else {                         // u0's list is scanned, once for all its labels
                key[v] = ~0ull;
                scanv[u0[k]] = 1;
            }
        }
    }
    block_count((long long *)&stats->n_ap, nap);
    block_count((long long *)&stats->n_cc, ncc);
    block_count(nhead_n, nhead);
}

// The marked lists to scan, as work items of kKeyChunk arcs each: every marked
// vertex takes ceil(deg / kKeyChunk) consecutive entries of klist, reserved with
// one atomic per warp (kVPer vertices per thread, striped like the other passes).
template <typename OffT>
__global__ void __launch_bounds__(kThreads) k_key_list(int64_t n, const OffT *__restrict__ off,
                                                       const uint8_t *__restrict__ scanv, int2 *klist,
                                                       int64_t klist_cap, long long *klist_n, int *err)
{
    const int64_t T = (int64_t)gridDim.x * kThreads;
    const int lane = threadIdx.x & 31;
    // the loop test is the warp's (its first lane's): the reservation needs every lane
    for (int64_t v0 = blockIdx.x * (int64_t)kThreads + threadIdx.x; v0 - lane < n; v0 += T * kVPer) {
        int64_t nch[kVPer];
        long long mine = 0;
#pragma unroll
        for (int k = 0; k < kVPer; ++k) {
            const int64_t v = v0 + k * T;
            nch[k] = 0;
            if (v < n && scanv[v]) nch[k] = ((int64_t)off[v + 1] - (int64_t)off[v] + kKeyChunk - 1) / kKeyChunk;
            mine += nch[k];
        }
        if (!__any_sync(0xffffffffu, mine != 0)) continue;
        long long inc = mine;
        for (int o = 1; o < 32; o <<= 1) {
            const long long y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += y;
        }
        const long long wtot = __shfl_sync(0xffffffffu, inc, 31);
        long long at = 0;
        if (lane == 31) at = (long long)atomicAdd((unsigned long long *)klist_n, (unsigned long long)wtot);
        at = __shfl_sync(0xffffffffu, at, 31) + inc - mine;
#pragma unroll
        for (int k = 0; k < kVPer; ++k)
            for (int64_t c = 0; c < nch[k]; ++c, ++at)
                if (in_range(at, klist_cap, err)) klist[at] = make_int2((int32_t)(v0 + k * T), (int32_t)c);
    }
}

// Labels whose head is their BCC's smallest vertex h: every class member x smaller
// than the class's top (the top itself is adjacent to h through its tree edge)
// tests whether it is adjacent to h (its parent is h, or a binary search of its
// own sorted list finds h), and the smallest adjacent one wins.
template <typename OffT>
__global__ void __launch_bounds__(kThreads) k_key_adj(int64_t n, const OffT *__restrict__ off,
                                                      const int32_t *__restrict__ adj, const int2 *__restrict__ fp,
                                                      const int32_t *__restrict__ lab, int32_t *kmin,
                                                      const long long *__restrict__ nhead_n, int *err)
{
    if (*nhead_n == 0) return;   // no label takes this path
    const int64_t T = (int64_t)gridDim.x * kThreads;
    for (int64_t v0 = blockIdx.x * (int64_t)kThreads + threadIdx.x; v0 < n; v0 += T * kVPer) {
        int32_t l[kVPer], py[kVPer];
#pragma unroll
        for (int k = 0; k < kVPer; ++k) {
            const int64_t v = v0 + k * T;
            l[k] = -1;
            if (v < n) {
                l[k] = lab[v];
                py[k] = fp[v].y;
            }
        }
        int32_t km[kVPer];
        uint32_t cand = 0;
#pragma unroll
        for (int k = 0; k < kVPer; ++k) {
            const int64_t v = v0 + k * T;
            if (v >= n || py[k] < 0 || v >= l[k] || !in_range(l[k], n, err)) continue;
            km[k] = kmin[l[k]];
            cand |= 1u << k;
        }
#pragma unroll
        for (int k = 0; k < kVPer; ++k) {
            if (!((cand >> k) & 1u)) continue;
            const int64_t v = v0 + k * T;
            if (km[k] < 0 || v >= km[k]) continue;
            const int32_t h = fp[l[k]].y;
            bool adjc = py[k] == h;
            if (!adjc) {
                int64_t lo = off[v], hi = off[v + 1];
                while (lo < hi) {
                    const int64_t mid = (lo + hi) >> 1;
                    if (adj[mid] < h) lo = mid + 1; else hi = mid;
                }
                adjc = lo < (int64_t)off[v + 1] && adj[lo] == h;
            }
            if (adjc) atomicMin(kmin + l[k], (int32_t)v);
        }
    }
}

// Keys of BCCs whose smallest vertex u0 lies in several BCCs and is not a hub head:
// the listed chunks of u0's arcs to larger neighbours are scanned, and the
// smallest arc of each such BCC wins an atomicMin. A warp takes 32 chunks, one
// per lane: a lane scans a chunk of at most kShortScan arcs alone (consecutive
// arcs of one BCC bid once), longer chunks are then scanned by the whole warp
// one at a time (the lanes of one label reduce to their smallest arc first).
constexpr int kShortScan = 32;

template <typename OffT>
__device__ __forceinline__ int32_t key_label(const int32_t *__restrict__ adj, const uint8_t *__restrict__ dirb,
                                             const int32_t *__restrict__ lab, const int2 *__restrict__ fp,
                                             const int32_t *__restrict__ smin, int32_t u, int64_t a)
{
    const int32_t w = adj[a];
    if (w <= u) return -1;
    const int32_t x = dir_bit(dirb, a) ? w : u;   // the endpoint later in preorder
    const int32_t l = __ldg(lab + x);
    const int32_t hd = __ldg(&fp[l].y), sm = __ldg(smin + l);
    return (hd < sm ? hd : sm) == u ? l : -1;
}

template <typename OffT>
__global__ void __launch_bounds__(kThreads) k_key_scan(const OffT *__restrict__ off, const int32_t *__restrict__ adj,
                                                       const long long *__restrict__ klist_n,
                                                       const int2 *__restrict__ klist,
                                                       const uint8_t *__restrict__ dirb,
                                                       const int32_t *__restrict__ lab,
                                                       const int2 *__restrict__ fp,
                                                       const int32_t *__restrict__ smin, unsigned long long *key)
{
    const int64_t cnt = *klist_n;
    const int lane = threadIdx.x & 31;
    const int64_t cnt_pad = (cnt + 31) & ~31ll;
    for (int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x; i < cnt_pad; i += (int64_t)gridDim.x * kThreads) {
        int32_t u = -1;
        int64_t b = 0, end = 0;
        if (i < cnt) {
            const int2 e = klist[i];
            u = e.x;
            b = (int64_t)off[u] + (int64_t)e.y * kKeyChunk;
            const int64_t lend = off[u + 1];
            end = b + kKeyChunk < lend ? b + kKeyChunk : lend;
        }
        const bool lng = end - b > kShortScan;
        if (!lng) {
            int32_t last_l = -1;
            for (int64_t a = b; a < end; ++a) {
                const int32_t l = key_label<OffT>(adj, dirb, lab, fp, smin, u, a);
                if (l < 0 || l == last_l) continue;   // a later arc of the same BCC cannot be smaller
                last_l = l;
                if ((unsigned long long)a < key[l]) atomicMin(key + l, (unsigned long long)a);
            }
        }
        unsigned todo = __ballot_sync(0xffffffffu, lng);
        while (todo) {
            const int src = __ffs(todo) - 1;
            todo &= todo - 1;
            const int32_t uu = __shfl_sync(0xffffffffu, u, src);
            const int64_t bb = __shfl_sync(0xffffffffu, b, src), ee = __shfl_sync(0xffffffffu, end, src);
            for (int64_t a0 = bb; a0 < ee; a0 += 32) {
                const int64_t a = a0 + lane;
                const int32_t l = a < ee ? key_label<OffT>(adj, dirb, lab, fp, smin, uu, a) : -1;
                const unsigned peers = __match_any_sync(0xffffffffu, l);
                if (l >= 0 && lane == __ffs(peers) - 1 && (unsigned long long)a < key[l])
                    atomicMin(key + l, (unsigned long long)a);
            }
        }
    }
}

template <typename OffT>
__global__ void __launch_bounds__(kThreads) k_key_bits(int64_t n, const OffT *__restrict__ off,
                                                       const int32_t *__restrict__ adj, const int2 *__restrict__ fp,
                                                       const int32_t *__restrict__ lab,
                                                       const int32_t *__restrict__ kmin,
                                                       const int32_t *__restrict__ parc, unsigned long long *key,
                                                       uint32_t *key_bits, int64_t nnz, int *err,
                                                       const int32_t *__restrict__ maxdeg)
{
    // On graphs with heavy hubs many labels search one hub's list: the searches load
    // with the evict-last policy, so that the levels they share stay in L2.
    const bool keep = *maxdeg >= kHeavyDeg;
    const uint64_t policy = l2_keep_policy();
    // kVPer vertices per thread and step, each round of their loads issued together
    const int64_t T = (int64_t)gridDim.x * kThreads;
    for (int64_t v0 = blockIdx.x * (int64_t)kThreads + threadIdx.x; v0 < n; v0 += T * kVPer) {
        uint32_t lbl = 0;
        int32_t hd[kVPer];
#pragma unroll
        for (int k = 0; k < kVPer; ++k) {
            const int64_t v = v0 + k * T;
            hd[k] = -1;
            if (v < n) hd[k] = fp[v].y;
            if (v < n && hd[k] >= 0 && lab[v] == v) lbl |= 1u << k;
        }
        unsigned long long ks[kVPer];
#pragma unroll
        for (int k = 0; k < kVPer; ++k)
            if ((lbl >> k) & 1u) ks[k] = key[v0 + k * T];
#pragma unroll
        for (int k = 0; k < kVPer; ++k) {
            if (!((lbl >> k) & 1u) || ks[k] != kKeyHead) continue;
            // the head's arc to the smallest class member adjacent to it: the tree arc
            // head -> top when the top is that member and First-CC kept its position,
            // else a binary search of the head's list
            const int64_t v = v0 + k * T;
            const int32_t w = kmin[v], h = hd[k];
            if (w == v && parc) {
                const int32_t pa = parc[v];
                if (pa >= 0) {
                    ks[k] = (unsigned long long)pa;
                    key[v] = ks[k];
                    continue;
                }
            }
            int64_t lo = off[h], hi = off[h + 1];
            while (lo < hi) {
                const int64_t mid = (lo + hi) >> 1;
                const int32_t am = keep ? ld_nc_policy(adj + mid, policy) : __ldg(adj + mid);
                if (am < w) lo = mid + 1; else hi = mid;
            }
            if (lo >= (int64_t)off[h + 1] || adj[lo] != w) {
                atomicOr(err, kErrIndex);
                lbl &= ~(1u << k);
                continue;
            }
            ks[k] = (unsigned long long)lo;
            key[v] = ks[k];
        }
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

// edge_bcc / is_bridge for every arc. Two forms, both launched; the one that does
// not fit the graph returns at once. On graphs with heavy hubs (kKeep) the word
// gathers keep their lines in L2 ahead of the streaming adjacency and outputs,
// with the register room that the policy takes.
template <typename OffT, bool kKeep>
__global__ void __launch_bounds__(kThreads, kKeep ? 6 : 8) k_edge_out(const OffT *__restrict__ off,
                                                                     const int32_t *__restrict__ adj, int64_t nnz,
                                                                     const int32_t *__restrict__ tile_v,
                                                                     int64_t ntiles,
                                                                     const int32_t *__restrict__ word,
                                                                     const uint8_t *__restrict__ dirb,
                                                                     int32_t *edge_bcc, uint8_t *is_bridge, bool vec,
                                                                     bool vec_out,
                                                                     const int32_t *__restrict__ maxdeg)
{
    if ((*maxdeg >= kHeavyDeg) != kKeep) return;
    const uint64_t policy = kKeep ? l2_keep_policy() : 0ull;
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
        for (int j = 0; j < kItems; ++j) {
            wx[j] = 0;
            if (j < at.cnt) {
                const int32_t *a = word + ((bits >> j) & 1u ? d[j] : at.src[j]);
                wx[j] = kKeep ? ld_nc_policy(a, policy) : __ldg(a);
            }
        }
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
                           bool vec, bool hubs, int32_t *edge_bcc, int32_t *bcc_head, uint8_t *is_ap,
                           uint8_t *is_bridge, const Batch &B, const Launch &L)
{
    cudaError_t e;
#define CK(x) do { e = (x); if (e != cudaSuccess) return e; } while (0)
    const int gv = grid_for(L, ceil_div(n, kThreads));
    const int64_t ntiles = ceil_div(nnz, kWTile);
    const int64_t nwords = ceil_div(nnz, 32);
    long long *klist_n = d.counters + 10, *nhead_n = d.counters + 13;
    CK(cudaMemsetAsync(d.scanv, 0, n, L.s));
    CK(cudaMemsetAsync(d.kmin, 0xff, n * sizeof(int32_t), L.s));
    CK(cudaMemsetAsync(klist_n, 0, sizeof(long long), L.s));
    CK(cudaMemsetAsync(nhead_n, 0, sizeof(long long), L.s));
    k_ap_keys<OffT><<<gv, kThreads, 0, L.s>>>(n, off, d.fp, d.lab, d.nh, d.smin, is_ap, d.key, d.kmin, d.scanv,
                                              nhead_n, d.stats, d.err);
    L.mark("k_ap_keys");
    CK(cudaGetLastError());
    if (nnz > 0) {
        k_key_list<OffT><<<gv, kThreads, 0, L.s>>>(n, off, d.scanv, d.klist, d.klist_cap, klist_n, d.err);
        L.mark("k_key_list");
        k_key_adj<OffT><<<gv, kThreads, 0, L.s>>>(n, off, adj, d.fp, d.lab, d.kmin, nhead_n, d.err);
        L.mark("k_key_adj");
        k_key_scan<OffT><<<L.grid, kThreads, 0, L.s>>>(off, adj, klist_n, d.klist, d.dirb, d.lab, d.fp, d.smin,
                                                       d.key);
        L.mark("k_key_scan");
        CK(cudaMemsetAsync(d.key_bits, 0, nwords * sizeof(uint32_t), L.s));
        k_key_bits<OffT><<<gv, kThreads, 0, L.s>>>(n, off, adj, d.fp, d.lab, d.kmin, hubs ? d.parc : nullptr, d.key,
                                                    d.key_bits, nnz, d.err,
                                                    reinterpret_cast<const int32_t *>(d.counters + 5));
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
        const int32_t *maxdeg = reinterpret_cast<const int32_t *>(d.counters + 5);
        const int ge = grid_for(L, ceil_div(ntiles, kWarpsPerCta));
        k_edge_out<OffT, false><<<ge, kThreads, 0, L.s>>>(off, adj, nnz, d.tile_v, ntiles, d.word, d.dirb, edge_bcc,
                                                          is_bridge, vec, vec_out, maxdeg);
        L.mark("k_edge_out");
        k_edge_out<OffT, true><<<ge, kThreads, 0, L.s>>>(off, adj, nnz, d.tile_v, ntiles, d.word, d.dirb, edge_bcc,
                                                         is_bridge, vec, vec_out, maxdeg);
        L.mark("k_edge_out_keep");
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
                                             bool, int32_t *, int32_t *, uint8_t *, uint8_t *, const Batch &,
                                             const Launch &);
template cudaError_t launch_outputs<int64_t>(const Dev &, const int64_t *, const int32_t *, int64_t, int64_t, bool,
                                             bool, int32_t *, int32_t *, uint8_t *, uint8_t *, const Batch &,
                                             const Launch &);

}  // namespace fbcc
