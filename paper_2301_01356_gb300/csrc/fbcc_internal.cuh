// Internal declarations of libfbcc: workspace layout, device building blocks
// (union-find, arc tiles, block scan with decoupled look-back) and the host
// launchers each phase's translation unit provides.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/fbcc.h"

namespace fbcc {

// ---------------------------------------------------------------------------
// Launch geometry
// ---------------------------------------------------------------------------
constexpr int kThreads = 256;                       // threads per CTA everywhere
constexpr int kItems = 8;                           // consecutive items per thread
constexpr int kTile = kThreads * kItems;            // 2048 items (arcs, positions) per CTA tile
constexpr int kRmqTile = 1024;                      // positions per low/high tile
constexpr int kChunk = 32;                          // positions per in-tile RMQ chunk
constexpr int kStride2 = 16;                        // level-2 ruler sampling stride

// Device error bits (workspace error word); reported as FBCC_E_ITER_LIMIT.
constexpr int kErrUnite = 1;      // union-find retry cap
constexpr int kErrChase = 2;      // list-ranking chase longer than the list
constexpr int kErrLookback = 4;   // scan look-back wait cap
constexpr int kErrIndex = 8;      // a computed index fell outside its array (inconsistent input)
constexpr int kUniteCap = 1 << 26;
constexpr int kKeyChunk = 1024;   // arcs of a scanned list per key-scan work item
// Forest-arc lists of vertices of graph degree >= kHubDeg (hubs) are split into
// kHubSub sub-lists (by edge id), so that their pushes do not serialise on one word.
constexpr int kHubDeg = 256;      // the default threshold (fbcc_config.hub_deg)
constexpr int kHubMinDeg = 32;    // the smallest threshold a configuration may set
constexpr int kHubSub = 32;
constexpr int64_t kHubCap = 1 << 16;
constexpr int kLookbackCap = 1 << 22;

// ---------------------------------------------------------------------------
// Workspace: every O(n) / O(nnz) array of one solve (device pointers).
// ---------------------------------------------------------------------------
// One sampling level of the list ranking above the level-1 rulers: its nodes are
// a sample of the lists of the level below (their heads plus one node in
// kStride2), and every node carries the weight of the segment of the level below
// that it owns.
struct RankLevel {
    int64_t cap;              // node capacity of this level
    int2 *l;                  // per node below: {next node below, node id here; -1 none, -2 finished}
    int32_t *relem;           // node below of every node here
    int32_t *owner, *offs;    // per node below: its owning node here and its weighted offset from it
    int32_t *next, *w;        // per node here: next node of its list (-1: last), segment weight
    uint8_t *head;            // per node here: 1 if it heads its list
    int32_t *sd;              // per node here: suffix weight to the end of its list
};
constexpr int kRankLevels = 2;

struct Dev {
    // sizes the workspace was created for
    int64_t n_max, nnz_max;
    int64_t ruler_max;        // capacity of the ruler arrays
    int64_t rmq_tiles_max, st_levels;

    int *err;                 // device error word
    long long *counters;      // [0] scan tile ticket, [1] ruler count, [2..] stats accumulators
    uint64_t *scan_status;    // per-tile look-back status (largest scan: 2n positions)

    // First-CC
    int32_t *uf;              // union-find parent (First-CC, then Last-CC)
    int32_t *te_u, *te_v;     // tree edge recorded at the vertex it hooked (-1: none)
    int32_t *te_a;            // CSR position of the arc te_u -> te_v it was hooked from (-1: not known)
    int32_t *parc;            // by vertex: CSR position of the arc parent -> vertex (-1: not known)
    int32_t *te2_u, *te2_v, *te2_a;  // the forest edges renumbered component by component (cc_order)
    uint32_t *bigb;           // sampling variants: one bit per vertex (First-CC) or position
                              // (Last-CC) in the sampled largest component, fixed for the full pass
    int2 *xl;                 // local-first First-CC: edges between vertex ranges {u, w}, u < w
    int64_t xl_cap;           // (aliases the rooting scratch, which is dead during First-CC)
    int32_t *tile_v;          // source vertex of the first arc of every arc tile (+1 sentinel)
    // Rooting
    int32_t *lhead;           // first forest arc of every vertex's list (-1: none)
    int32_t *nxt;             // next arc in its source's list (2n ids; -1: last)
    int32_t *hubidx;          // per vertex: its hub slot (-1: not a hub), see kHubDeg
    int32_t *hubhead;         // per hub slot: kHubSub sub-list heads
    int32_t *hubnext;         // per hub slot and sub-list: head of the next non-empty sub-list (-1: none)
    int32_t *hubvert;         // vertex of every hub slot
    int64_t hub_cap;          // hub slots
    uint8_t *rhead;           // by ruler id: 1 if the ruler heads its tour
    int2 *link;               // {succ, ruler id or -1} per tree arc; after the walks a non-ruler
                              // arc holds {owning ruler, -distance from it}
    int32_t *relem;           // arc of ruler r
    int32_t *rlen;            // ruler segment length
    int32_t *rnx1;            // next ruler in the tour (-1: last)
    int32_t *sd1;             // suffix length (arcs to the tour's end) from every ruler
    RankLevel lv[kRankLevels];// the ruler lists sampled again (levels 2 and 3)
    int32_t *top_tmp[4];      // global double buffers of the top level's pointer jumping
    int64_t top_tmp_cap;
    int32_t *csize;           // component size at its root (other entries unspecified)
    int32_t *vbase;           // first preorder number of the component at its root
    int2 *rec;                // tour record at every position (down/up arc, padding)
    // Tagging (fp indexed by vertex; the rest by preorder number)
    int2 *fp;                 // {first, parent} by vertex (parent -1 at a root)
    int32_t *first4;          // first by vertex alone (the arc passes gather it: half of fp's bytes)
    int2 *fl;                 // {first, last} by vertex (one gather gives the fence test a parent's interval)
    uint8_t *dirb;            // one bit per arc: the target's preorder number exceeds the source's
    int32_t *ord;             // vertex at preorder number p
    int32_t *porig;           // parent vertex of the vertex at preorder number p (-1 root)
    int32_t *w1, *w2;         // w1/w2 at preorder number p
    int2 *pmm;                // in-tile prefix {min of w1, max of w2}
    int32_t *tmin, *tmax;     // sparse tables over RMQ tiles: st_levels x rmq_tiles_max
    uint8_t *vbits;           // per vertex: bit0 = tree edge to parent is a bridge
    int32_t *low, *high;      // low/high by preorder number (written by profiled solves only)
    // Last-CC by preorder number
    int32_t *lp;              // plain-component pointer (root: itself), flattened in place
    uint8_t *ext;             // position referenced across an RMQ tile
    int32_t *qlist;           // compacted positions with ext set
    int2 *cr;                 // by vertex {first, plain-component root} (Last-CC arc passes)
    int32_t *lastp;           // last[] by preorder number (written by the preorder scan)
    int32_t *lab;             // Last-CC label by vertex: its class's top vertex (a root: itself)
    int32_t *smin;            // by label vertex: smallest vertex id of its label class
    // Last-CC and outputs
    int32_t *nh;              // number of labels a vertex heads
    unsigned long long *key;  // smallest arc id (src < dst) of label L at [L]
    uint8_t *scanv;           // per vertex: its list is scanned for keys (listed in klist)
    int2 *klist;              // {u0, chunk} of every kKeyChunk-arc chunk of the scanned lists
    int64_t klist_cap;
    int32_t *kmin;            // per label whose head is its BCC's smallest vertex: the smallest
                              // class member adjacent to the head (-1: another kind of label)
    uint32_t *key_bits;       // one bit per arc: arc is the key of its BCC
    int32_t *key_pre;         // exclusive popcount prefix per 32-bit word of key_bits
    int32_t *rank;            // canonical BCC index of label L at [L]
    int32_t *word;            // per vertex: BCC index of its label | bridge << 31
    // Query index of the last solve (built by the first query after it)
    int32_t *hoff;            // labels headed by the vertices before v (n+1 entries)
    int32_t *hfill;           // fill cursor per head
    int32_t *hlist;           // ranks of the labels each vertex heads, at [hoff[v], hoff[v+1])
    fbcc_stats *stats;        // device-side counts
};

// ---------------------------------------------------------------------------
// Small device helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ int32_t ld_cg(const int32_t *p) { return __ldcg(p); }

// True when 0 <= i < n; otherwise raises kErrIndex (the access is then skipped).
__device__ __forceinline__ bool in_range(int64_t i, int64_t n, int *err)
{
    if ((uint64_t)i < (uint64_t)n) return true;
    atomicOr(err, kErrIndex);
    return false;
}

__device__ __forceinline__ bool test_bit(const uint32_t *bits, int64_t i)
{
    return (__ldg(bits + (i >> 5)) >> (i & 31)) & 1u;
}

__device__ __forceinline__ void set_bit(uint32_t *bits, int64_t i)
{
    atomicOr(bits + (i >> 5), 1u << (i & 31));
}

// Union-find root with path halving. Parents only ever point to smaller ids
// (larger roots are hooked under smaller ones), so the walk strictly decreases
// and the root of a set is its smallest member. Loads may be served from L1
// although other SMs write the array: an entry only ever moves to a higher
// ancestor, so a stale copy still names an ancestor (the walk is longer, never
// wrong), and every hook is a CAS, which L2 decides on the current value.
__device__ __forceinline__ int32_t uf_find(int32_t *uf, int32_t v)
{
    while (true) {
        int32_t p = uf[v];
        if (p == v) return v;
        int32_t gp = uf[p];
        if (gp == p) return p;
        uf[v] = gp;  // halving: gp is an ancestor of v, so the store is always safe
        v = gp;
    }
}

// Root of v without writing anything. The final flattening pass uses this: a
// halving store made there by one thread could land after another thread had
// already stored the root into the same slot and leave a non-root behind.
__device__ __forceinline__ int32_t uf_root(const int32_t *uf, int32_t v)
{
    int32_t p = uf[v];
    while (p != v) {
        v = p;
        p = uf[v];
    }
    return v;
}

// uf[v] = root of v for one vertex per lane (lanes with in == false take part
// but change nothing). Lanes whose parents agree walk once: a warp's vertices
// mostly share a set.
__device__ __forceinline__ void uf_flatten_warp(int32_t *uf, int64_t v, bool in)
{
    const int32_t p = in ? uf[v] : -1;
    const unsigned peers = __match_any_sync(0xffffffffu, p);
    const int leader = __ffs(peers) - 1;
    int32_t r = -1;
    if (in && (int)(threadIdx.x & 31) == leader) r = uf_root(uf, p);
    r = __shfl_sync(0xffffffffu, r, leader);
    if (in && r != p) uf[v] = r;
}

// Record the forest edge u-v at the root r it hooked, with the CSR position of
// the arc u->v it came from (-1 when unknown or beyond 32 bits; not kept when te_a
// is null).
__device__ __forceinline__ void tree_edge(int32_t *te_u, int32_t *te_v, int32_t *te_a, int32_t r, int32_t u,
                                          int32_t v, int64_t a)
{
    te_u[r] = u;
    te_v[r] = v;
    if (te_a) te_a[r] = (a >= 0 && a < INT32_MAX) ? (int32_t)a : -1;
}

// Union of the sets of u and v by CAS-hooking the larger root under the smaller.
// Returns the root that got hooked, or -1 when u and v were already joined.
__device__ __forceinline__ int32_t uf_unite(int32_t *uf, int32_t u, int32_t v, int *err)
{
    int32_t ru = uf_find(uf, u), rv = uf_find(uf, v);
    for (int it = 0; it < kUniteCap; ++it) {
        if (ru == rv) return -1;
        int32_t hi = ru > rv ? ru : rv, lo = ru > rv ? rv : ru;
        int32_t old = atomicCAS(uf + hi, hi, lo);
        if (old == hi) return hi;
        ru = uf_find(uf, old);  // hi was hooked meanwhile; continue from its new parent
        rv = uf_find(uf, lo);
    }
    atomicOr(err, kErrUnite);
    return -1;
}

// Lists above kRestLong arcs, in passes that go by vertex, are cut into chunks of
// kRestChunk arcs that a second launch spreads over the whole grid.
constexpr int kRestLong = 2048;
constexpr int kRestChunk = 1024;

// Queues the chunks of vertex v's list of len arcs (whole warp, v and len the same
// in every lane): {v, chunk index} entries. Without room for all of them the warp
// keeps the list (false); entries it had reserved below the capacity are marked
// empty, and the drain reads at most `cap` entries.
__device__ __forceinline__ bool rest_queue(int2 *lq, int64_t cap, long long *nq, int32_t v, int64_t len, int lane)
{
    const int64_t nch = (len + kRestChunk - 1) / kRestChunk;
    long long k = 0;
    if (lane == 0) k = (long long)atomicAdd((unsigned long long *)nq, (unsigned long long)nch);
    k = __shfl_sync(0xffffffffu, k, 0);
    if (k + nch > cap) {
        for (int64_t c = k + lane; c < cap; c += 32) lq[c] = make_int2(-1, 0);
        return false;
    }
    for (int64_t c = lane; c < nch; c += 32) lq[k + c] = make_int2(v, (int32_t)c);
    return true;
}

// One slot per wanting lane, reserved with one atomic per warp (the whole warp
// calls); slots at or above cap are counted but not written.
template <typename T>
__device__ __forceinline__ void warp_append(T *q, long long *cnt, int64_t cap, bool want, T val)
{
    const unsigned m = __ballot_sync(0xffffffffu, want);
    if (!m) return;
    const int lane = threadIdx.x & 31, leader = __ffs(m) - 1;
    long long base = 0;
    if (lane == leader) base = (long long)atomicAdd((unsigned long long *)cnt, (unsigned long long)__popc(m));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (want) {
        const long long i = base + __popc(m & ((1u << lane) - 1u));
        if (i < cap) q[i] = val;
    }
}

// Graphs whose largest degree (taken by First-CC's init pass into counters[5]) is
// at least this have heavy hubs: their arc passes see the same targets again and
// again, and some kernels take another form for them.
constexpr int kHeavyDeg = 4096;

// L2 eviction priority of a gather (a PTX cache policy, sm_80 and later): lines
// loaded with the evict_last policy stay in L2 ahead of lines loaded normally.
__device__ __forceinline__ uint64_t l2_keep_policy()
{
    uint64_t p;
    asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}

// A read-only 4-byte load through the non-coherent path with an L2 cache policy.
__device__ __forceinline__ int32_t ld_nc_policy(const int32_t *a, uint64_t policy)
{
    int32_t v;
    asm("ld.global.nc.L2::cache_hint.b32 %0, [%1], %2;" : "=r"(v) : "l"(a), "l"(policy));
    return v;
}

__device__ __forceinline__ int32_t warp_sum_i32(int32_t x)
{
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

// Block-wide sum of one value per thread, result valid in every thread.
__device__ __forceinline__ long long block_sum(long long x)
{
    __shared__ long long part[kThreads / 32];
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = x;
    __syncthreads();
    long long t = 0;
#pragma unroll
    for (int i = 0; i < kThreads / 32; ++i) t += part[i];
    return t;
}

// Add a per-thread count into a device counter with one atomic per CTA.
__device__ __forceinline__ void block_count(long long *dst, long long x)
{
    long long t = block_sum(x);
    if (threadIdx.x == 0 && t) atomicAdd((unsigned long long *)dst, (unsigned long long)t);
}

// ---------------------------------------------------------------------------
// Single-pass exclusive scan with decoupled look-back (Merrill & Garland, 2016).
// A CTA takes the next tile ticket, scans its kTile items in registers, publishes
// its aggregate, waits (bounded) for its predecessors' prefix and publishes its
// inclusive prefix. Status word: bits 62..63 flag (1 aggregate, 2 prefix),
// bits 0..61 value.
// ---------------------------------------------------------------------------
constexpr uint64_t kFlagAgg = 1ull << 62, kFlagPre = 2ull << 62, kValMask = (1ull << 62) - 1;

__device__ __forceinline__ int64_t scan_ticket(long long *ticket)
{
    __shared__ int64_t t;
    __syncthreads();
    if (threadIdx.x == 0) t = (int64_t)atomicAdd((unsigned long long *)ticket, 1ull);
    __syncthreads();
    return t;
}

// In: v[] the thread's N values (items tile*N*kThreads + threadIdx.x*N + j).
// Out: v[] their global exclusive prefixes; returns the tile's inclusive total end.
template <int N>
__device__ __forceinline__ long long scan_tile_exclusive(long long (&v)[N], int64_t tile, uint64_t *status, int *err)
{
    __shared__ long long warp_tot[kThreads / 32];
    __shared__ long long tile_excl;
    long long run = 0;
#pragma unroll
    for (int j = 0; j < N; ++j) {
        long long x = v[j];
        v[j] = run;
        run += x;
    }
    // exclusive scan of the per-thread totals across the CTA
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    long long inc = run;
    for (int o = 1; o < 32; o <<= 1) {
        long long y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) warp_tot[wid] = inc;
    __syncthreads();
    long long wexcl = 0, agg = 0;
#pragma unroll
    for (int i = 0; i < kThreads / 32; ++i) {
        if (i < wid) wexcl += warp_tot[i];
        agg += warp_tot[i];
    }
    long long texcl = wexcl + inc - run;
    // Look-back by warp 0: each step inspects 32 predecessors at once and adds
    // the aggregates up to the nearest published prefix.
    if (wid == 0) {
        long long excl = 0;
        if (tile == 0) {
            if (lane == 0)
                atomicExch((unsigned long long *)(status + tile), (unsigned long long)(kFlagPre | (uint64_t)agg));
        } else {
            if (lane == 0)
                atomicExch((unsigned long long *)(status + tile), (unsigned long long)(kFlagAgg | (uint64_t)agg));
            int64_t j = tile - 1;
            int spins = 0;
            while (true) {
                const int64_t idx = j - lane;
                uint64_t st = 2ull << 62;  // before tile 0: an empty published prefix
                if (idx >= 0) st = *(volatile uint64_t *)(status + idx);
                const uint64_t f = st & ~kValMask;
                const unsigned pre = __ballot_sync(0xffffffffu, f == kFlagPre);
                const unsigned zero = __ballot_sync(0xffffffffu, f == 0);
                // lanes 0..stop are the window: up to and including the nearest prefix
                const int stop = pre ? __ffs(pre) - 1 : 31;
                const unsigned window = stop == 31 ? 0xffffffffu : ((1u << (stop + 1)) - 1u);
                if (zero & window) {
                    if (++spins > kLookbackCap) {
                        if (lane == 0) atomicOr(err, kErrLookback);
                        break;
                    }
                    continue;
                }
                long long v = ((window >> lane) & 1u) ? (long long)(st & kValMask) : 0;
                for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                excl += v;
                if (pre) break;
                j -= 32;
            }
            if (lane == 0)
                atomicExch((unsigned long long *)(status + tile),
                           (unsigned long long)(kFlagPre | (uint64_t)(excl + agg)));
        }
        if (lane == 0) tile_excl = excl;
    }
    __syncthreads();
    long long base = tile_excl + texcl;
#pragma unroll
    for (int j = 0; j < N; ++j) v[j] += base;
    return tile_excl + agg;
}

// ---------------------------------------------------------------------------
// Arc tiles, one per warp: warp tile w covers arcs [w*kWTile, (w+1)*kWTile); lane
// i covers the kItems consecutive arcs starting at w*kWTile + i*kItems. The
// source vertex of every arc comes from the tile's window of offsets, staged in
// the warp's slice of shared memory. Warps never wait for each other, so a lane
// stuck in a long union-find walk only holds back its own warp. tile_v[w] is the
// source of the tile's first arc, tile_v[nwt] that of the graph's last arc.
// ---------------------------------------------------------------------------
constexpr int kWTile = 32 * kItems;                 // 256 arcs per warp tile
constexpr int kWarpWin = kWTile + 32;               // offsets cached per warp tile
constexpr int kWarpsPerCta = kThreads / 32;

template <typename OffT>
struct ArcTile {
    int64_t a0;        // first arc of this lane
    int cnt;           // arcs of this lane (0..kItems)
    int32_t src[kItems];
};

template <typename OffT>
__device__ __forceinline__ void arc_tile_sources(const OffT *__restrict__ off, int64_t nnz,
                                                 const int32_t *__restrict__ tile_v, int64_t w,
                                                 OffT *win, ArcTile<OffT> &at)
{
    const int lane = threadIdx.x & 31;
    const int32_t vlo = tile_v[w], vhi = tile_v[w + 1];
    const int64_t wn = (int64_t)vhi - vlo + 2;  // off[vlo .. vhi+1]
    const bool sm = wn <= kWarpWin;
    __syncwarp();
    if (sm)
        for (int64_t i = lane; i < wn; i += 32) win[i] = off[vlo + i];
    __syncwarp();
    at.a0 = w * (int64_t)kWTile + (int64_t)lane * kItems;
    at.cnt = 0;
    if (at.a0 >= nnz) return;
    at.cnt = (int)((nnz - at.a0) < kItems ? (nnz - at.a0) : kItems);
    // largest i in [0, wn-2] with off[vlo+i] <= a0
    int64_t lo = 0, hi = wn - 2;
    while (lo < hi) {
        int64_t mid = (lo + hi + 1) >> 1;
        int64_t x = sm ? (int64_t)win[mid] : (int64_t)off[vlo + mid];
        if (x <= at.a0) lo = mid; else hi = mid - 1;
    }
    int64_t end = sm ? (int64_t)win[lo + 1] : (int64_t)off[vlo + lo + 1];
#pragma unroll
    for (int j = 0; j < kItems; ++j) {
        int64_t a = at.a0 + j;
        if (j < at.cnt) {
            while (end <= a) {
                ++lo;
                end = sm ? (int64_t)win[lo + 1] : (int64_t)off[vlo + lo + 1];
            }
        }
        at.src[j] = vlo + (int32_t)lo;
    }
}

// The same for a whole CTA tile of kTile arcs (kWarpsPerCta consecutive warp
// tiles): one shared window, loaded by the CTA. The union-find passes use it.
constexpr int kCtaWin = kTile + 256;

template <typename OffT>
__device__ __forceinline__ void arc_cta_tile_sources(const OffT *__restrict__ off, int64_t nnz,
                                                     const int32_t *__restrict__ tile_v, int64_t nwt, int64_t t,
                                                     OffT *win, ArcTile<OffT> &at)
{
    const int64_t w0 = t * kWarpsPerCta, w1 = (w0 + kWarpsPerCta < nwt) ? w0 + kWarpsPerCta : nwt;
    const int32_t vlo = tile_v[w0], vhi = tile_v[w1];
    const int64_t wn = (int64_t)vhi - vlo + 2;
    const bool sm = wn <= kCtaWin;
    __syncthreads();
    if (sm)
        for (int64_t i = threadIdx.x; i < wn; i += kThreads) win[i] = off[vlo + i];
    __syncthreads();
    at.a0 = t * (int64_t)kTile + (int64_t)threadIdx.x * kItems;
    at.cnt = 0;
    if (at.a0 >= nnz) return;
    at.cnt = (int)((nnz - at.a0) < kItems ? (nnz - at.a0) : kItems);
    int64_t lo = 0, hi = wn - 2;
    while (lo < hi) {
        int64_t mid = (lo + hi + 1) >> 1;
        int64_t x = sm ? (int64_t)win[mid] : (int64_t)off[vlo + mid];
        if (x <= at.a0) lo = mid; else hi = mid - 1;
    }
    int64_t end = sm ? (int64_t)win[lo + 1] : (int64_t)off[vlo + lo + 1];
#pragma unroll
    for (int j = 0; j < kItems; ++j) {
        int64_t a = at.a0 + j;
        if (j < at.cnt) {
            while (end <= a) {
                ++lo;
                end = sm ? (int64_t)win[lo + 1] : (int64_t)off[vlo + lo + 1];
            }
        }
        at.src[j] = vlo + (int32_t)lo;
    }
}

// Loop header of an arc pass: the calling warp's tiles, and its window slice.
#define FOR_EACH_WARP_TILE(w, nwt)                                                          \
    for (int64_t w = (blockIdx.x * (int64_t)kThreads + threadIdx.x) >> 5; w < (nwt);      \
         w += ((int64_t)gridDim.x * kThreads) >> 5)

// The kItems neighbour ids of the thread's arcs (vector loads when aligned).
__device__ __forceinline__ void arc_tile_targets(const int32_t *__restrict__ adj, int64_t a0, int cnt,
                                                 bool vec, int32_t (&d)[kItems])
{
    if (vec && cnt == kItems) {
        int4 x = __ldcs(reinterpret_cast<const int4 *>(adj + a0));
        int4 y = __ldcs(reinterpret_cast<const int4 *>(adj + a0) + 1);
        d[0] = x.x; d[1] = x.y; d[2] = x.z; d[3] = x.w;
        d[4] = y.x; d[5] = y.y; d[6] = y.z; d[7] = y.w;
    } else {
#pragma unroll
        for (int j = 0; j < kItems; ++j) d[j] = j < cnt ? __ldcs(adj + a0 + j) : 0;
    }
}


// ---------------------------------------------------------------------------
// Batched solves: many graphs packed as one disjoint union with global ids.
// ---------------------------------------------------------------------------
struct Batch {
    int32_t G = 0;                       // number of graphs; 0 for a plain solve
    const int64_t *vtx_base = nullptr;   // device, G+1
    const int64_t *arc_base = nullptr;   // device, G+1
    int64_t *bcc_base = nullptr;         // device, G+1: BCCs of the graphs before g
    fbcc_stats *stats = nullptr;         // device, G
};

// Graph owning global vertex v: the largest g with vtx_base[g] <= v.
__device__ __forceinline__ int32_t graph_of(const int64_t *__restrict__ vtx_base, int32_t G, int64_t v)
{
    int32_t lo = 0, hi = G - 1;
    while (lo < hi) {
        int32_t mid = (lo + hi + 1) >> 1;
        if (__ldg(vtx_base + mid) <= v) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Direction bit of arc a: the target comes later in preorder than the source.
__device__ __forceinline__ bool dir_bit(const uint8_t *dirb, int64_t a)
{
    return (__ldg(dirb + (a >> 3)) >> (a & 7)) & 1u;
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
// Per-kernel timing of a solve (fbcc_config.profile): an event after every launch.
constexpr int kProfMax = 320;
struct Prof {
    int count = 0;
    const char *names[kProfMax];
    cudaEvent_t ev[kProfMax + 1];
    bool ready = false;
};

struct Launch {
    cudaStream_t s;
    int grid;              // persistent grid size (CTAs)
    Prof *prof = nullptr;  // set when the solve is profiled
    void mark(const char *name) const
    {
        if (prof && prof->count < kProfMax) {
            prof->names[prof->count] = name;
            cudaEventRecord(prof->ev[prof->count + 1], s);
            ++prof->count;
        }
    }
};

inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

inline int grid_for(const Launch &L, int64_t items_per_cta_units)
{
    int64_t g = items_per_cta_units < 1 ? 1 : items_per_cta_units;
    return (int)(g < L.grid ? g : L.grid);
}

// Phase launchers (each returns the first launch error or cudaSuccess).
template <typename OffT>
cudaError_t launch_first_cc(const Dev &d, const OffT *off, const int32_t *adj, int64_t n, int64_t nnz,
                            int cc_sample, int cc_local, int cc_ldd, int hub_deg, bool vec, const Launch &L);
// First-CC by LDD: the clusters' forest edges and the union of the edges between
// clusters (flag[1] = 0 when their list overflowed and a full hook pass must
// follow); after the flatten, the roots moved to each component's smallest vertex.
template <typename OffT>
cudaError_t launch_ldd_forest(const Dev &d, const OffT *off, const int32_t *adj, int64_t n, int64_t nnz,
                              int inv_beta, int32_t *te_a, int32_t *flag, const Launch &L);
cudaError_t launch_ldd_reroot(const Dev &d, int64_t n, const Launch &L);
// Allow the local-first First-CC kernel its shared memory for ranges of V vertices.
cudaError_t prepare_cc_local(int V);
template <typename OffT>
cudaError_t launch_rooting(const Dev &d, const OffT *off, const int32_t *adj, int64_t n, int64_t nnz,
                           int ruler_stride, int chase_chains, int rank_variant, int cc_order, bool hubs,
                           const Launch &L);
template <typename OffT>
cudaError_t launch_tagging(const Dev &d, const OffT *off, const int32_t *adj, int64_t n, int64_t nnz,
                           bool vec, bool keep_low_high, const Launch &L);
template <typename OffT>
cudaError_t launch_last_cc(const Dev &d, const OffT *off, const int32_t *adj, int64_t n, int64_t nnz,
                           int lcc_sample, bool vec, const Launch &L);
// Labels from a union-find over positions (uf; lp the plain-component pointers,
// the identity where uf holds every union): lab, smin, nh and the BCC count.
cudaError_t launch_final_labels(const Dev &d, int64_t n, const int32_t *lp, const int32_t *uf, const Launch &L);
// The Tarjan-Vishkin skeleton (section 3.2; its rules in the appendix on
// Tarjan-Vishkin) built explicitly in caller memory and connected in place of
// Last-CC.
struct TvScratch {
    void *mem;
    size_t bytes;
};
size_t tv_scratch_bytes(int64_t n, int64_t nnz);
template <typename OffT>
cudaError_t launch_tv_connect(const Dev &d, const OffT *off, const int32_t *adj, int64_t n, int64_t nnz,
                              const TvScratch &tv, bool vec, const Launch &L);
template <typename OffT>
cudaError_t launch_outputs(const Dev &d, const OffT *off, const int32_t *adj, int64_t n, int64_t nnz,
                           bool vec, bool hubs, int32_t *edge_bcc, int32_t *bcc_head, uint8_t *is_ap,
                           uint8_t *is_bridge, const Batch &B, const Launch &L);
template <typename OffT>
cudaError_t launch_validate(const Dev &d, const OffT *off, const int32_t *adj, int64_t n, int64_t nnz,
                            const Launch &L);

// Generic exclusive scan over int32 counts: out[i] = sum of in[0..i), out[len] = total
// (out has len+1 entries; in may alias out when in_place).
// out[i] = set bits in words[0..i), i in [0, len].
cudaError_t launch_scan_popc(const Dev &d, const uint32_t *words, int32_t *out, int64_t len, const Launch &L);
// In place: a[i] = sum of a[0..i) for i in [0, len] (a has len + 1 entries).
cudaError_t launch_scan_i32(const Dev &d, int32_t *a, int64_t len, const Launch &L);

// Biconnectivity queries over the last solve's labels and heads (fbcc_query.cu).
cudaError_t launch_query_index(const Dev &d, int64_t n, cudaStream_t s);
cudaError_t launch_query_pairs(const Dev &d, int64_t n, const int32_t *u, const int32_t *v, int64_t q, int32_t *out,
                               int grid, cudaStream_t s);
cudaError_t launch_query_count(const Dev &d, int64_t n, const int32_t *v, int64_t q, int64_t *out_off, int grid,
                               cudaStream_t s);
cudaError_t launch_query_list(const Dev &d, int64_t n, const int32_t *v, int64_t q, const int64_t *out_off,
                              int32_t *out, int grid, cudaStream_t s);

// Rounds of pointer jumping that rank lists of up to r nodes.
inline int jump_rounds(int64_t r)
{
    int k = 0;
    while ((1ll << k) < r + 1) ++k;
    return k + 1;
}

// The top level of the list ranking is ranked by one CTA in shared memory when it
// holds at most kTopCap nodes (else by the same CTA in global memory).
constexpr int kTopThreads = 1024;
constexpr int kTopPer = 16;
constexpr int kTopCap = kTopThreads * kTopPer;
cudaError_t prepare_rooting();

}  // namespace fbcc
