// Tagging (Algorithm 1, step 3; section 3.2 for w1/w2/low/high, section 5
// "Computing Tags"):
//   w1[u] = min({first[u]} U {first[u'] : u-u' a non-tree edge}), w2 the max;
//   low[v] = min of w1 over T_v, high[v] = max of w2 over T_v.
// With preorder numbers, T_v is the position range [first[v], last[v]], so w1/w2
// are stored by preorder number and low/high are range-min/max queries over that
// range (the paper uses a sparse table; here: 1024-position tiles, in-tile
// prefix/suffix and 32-position chunks in shared memory, and a sparse table only
// over the tile extrema, which keeps the extra space O(n)).
//
// The query kernel then tests the tree edge p(v)-v (Algorithm 1, Fence):
//   fence iff first[p(v)] <= low[v] and last[p(v)] >= high[v];
// a plain (non-fence) tree edge is an edge of the skeleton G' and is united in the
// Last-CC union-find right there. The edge is a bridge iff nothing leaves T_v:
// low[v] == first[v] and high[v] <= last[v].
#include "fbcc_internal.cuh"

namespace fbcc {

#define GRID_STRIDE(i, n) \
    for (int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x; i < (n); i += (int64_t)gridDim.x * kThreads)

// first by vertex as a compact array for the arc passes' gathers, and {first,
// last} by vertex for the fence test (last gathered here from the preorder-indexed
// array, in a pass with many loads in flight, so that the query kernel needs one
// independent gather per parent instead of two dependent ones).
__global__ void __launch_bounds__(kThreads) k_first_of(int64_t n, const int2 *__restrict__ fp,
                                                       const int32_t *__restrict__ lastp, int32_t *first4, int2 *fl)
{
    GRID_STRIDE(v, n)
    {
        const int32_t f = fp[v].x;
        first4[v] = f;
        fl[v] = make_int2(f, (uint32_t)f < (uint64_t)n ? __ldg(lastp + f) : -1);
    }
}

// w1/w2 over the arcs, one atomic per run of equal sources per thread, and the
// direction bit of every arc (target later in preorder than the source).
//
// Only the parent arc is left out. The arcs to children may enter: a child c of
// u has first[u] < first[c] <= last[u], so it cannot lower w1[u] (which holds
// first[u]), and although it can raise w2[u], every value it adds lies inside
// T_v for each ancestor v of u, where high[v] >= last[v] already (w2 of T_v's
// last vertex is at least its own first). low and high, the only consumers, stay
// exactly as defined, and no parent of a neighbour has to be gathered.
template <typename OffT, bool kKeep>
__global__ void __launch_bounds__(kThreads) k_w12(const OffT *__restrict__ off, const int32_t *__restrict__ adj,
                                                  int64_t nnz, const int32_t *__restrict__ tile_v, int64_t ntiles,
                                                  const int2 *__restrict__ fp, const int32_t *__restrict__ first4,
                                                  int32_t *w1, int32_t *w2, uint8_t *dirb, int64_t n, int *err,
                                                  bool vec, const int32_t *__restrict__ maxdeg)
{
    // Two forms, both launched; the one that does not fit the graph returns at once.
    // On graphs with heavy hubs (kKeep) the targets' first numbers are read again
    // and again: their lines are kept in L2 ahead of the streaming adjacency and
    // the w1/w2 updates (rmat24: 2.51 to 2.30 ms). Elsewhere it costs, and the
    // plain form keeps its lower register count.
    if ((*maxdeg >= kHeavyDeg) != kKeep) return;
    // (the policy is made once here: made at each load, it measured no effect)
    const uint64_t policy = kKeep ? l2_keep_policy() : 0ull;
    __shared__ OffT win_all[kWarpsPerCta * kWarpWin];
    OffT *win = win_all + (threadIdx.x >> 5) * kWarpWin;
    const int lane = threadIdx.x & 31;
    ArcTile<OffT> at;
    FOR_EACH_WARP_TILE(t, ntiles)
    {
        arc_tile_sources(off, nnz, tile_v, t, win, at);
        // A lane whose arcs all leave one source keeps that run for a warp-wide
        // reduction: the lanes of a long list then add one atomic per warp.
        int32_t src_last = at.src[0];   // (static indices keep at.src in registers)
#pragma unroll
        for (int j = 1; j < kItems; ++j)
            if (j < at.cnt) src_last = at.src[j];
        const bool single = at.cnt > 0 && at.src[0] == src_last;
        int32_t cur = -1, mn = INT32_MAX, mx = INT32_MIN;
        int2 fc = make_int2(0, -1);
        uint32_t bits = 0;
        if (at.cnt) {
            int32_t d[kItems];
            arc_tile_targets(adj, at.a0, at.cnt, vec, d);
#pragma unroll
            for (int j = 0; j < kItems; ++j) {
                if (j >= at.cnt) break;
                if (at.src[j] != cur) {   // a new source: the previous run adds its atomics
                    if (cur >= 0 && mn != INT32_MAX && in_range(fc.x, n, err)) {
                        if (mn < fc.x) atomicMin(w1 + fc.x, mn);
                        if (mx > fc.x) atomicMax(w2 + fc.x, mx);
                    }
                    cur = at.src[j];
                    fc = __ldg(fp + cur);
                    mn = INT32_MAX;
                    mx = INT32_MIN;
                }
                if (d[j] == fc.y) continue;   // the parent arc: earlier in preorder
                const int32_t fw = kKeep ? ld_nc_policy(first4 + d[j], policy) : __ldg(first4 + d[j]);
                if (fw > fc.x) bits |= 1u << j;
                mn = fw < mn ? fw : mn;
                mx = fw > mx ? fw : mx;
            }
            // the last run adds its atomics here, unless the lane has a single
            // source (flushed below, with the warp)
            if (!single && cur >= 0 && mn != INT32_MAX && in_range(fc.x, n, err)) {
                if (mn < fc.x) atomicMin(w1 + fc.x, mn);
                if (mx > fc.x) atomicMax(w2 + fc.x, mx);
            }
            dirb[at.a0 >> 3] = (uint8_t)bits;   // a0 is a multiple of kItems = 8
        }
        // segmented min/max over runs of lanes with the same single source (such
        // lanes are consecutive: arcs are in CSR order); the run's first lane adds
        const int32_t key = single ? cur : -1 - lane;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int32_t ko = __shfl_down_sync(0xffffffffu, key, o);
            const int32_t a = __shfl_down_sync(0xffffffffu, mn, o), b = __shfl_down_sync(0xffffffffu, mx, o);
            if (lane + o < 32 && ko == key) {
                mn = a < mn ? a : mn;
                mx = b > mx ? b : mx;
            }
        }
        const int32_t kp = __shfl_up_sync(0xffffffffu, key, 1);
        if (single && (lane == 0 || kp != key) && mn != INT32_MAX && in_range(fc.x, n, err)) {
            if (mn < fc.x) atomicMin(w1 + fc.x, mn);
            if (mx > fc.x) atomicMax(w2 + fc.x, mx);
        }
    }
}

// Per RMQ tile: inclusive prefix min of w1 and max of w2 from the tile start (one
// 8-byte pair per position: the query gathers both at once), and the tile's
// min/max (level 0 of the tile sparse table).
__global__ void __launch_bounds__(kThreads) k_rmq_prefix(int64_t n, const int32_t *__restrict__ w1,
                                                         const int32_t *__restrict__ w2, int2 *pmm,
                                                         int32_t *tmin, int32_t *tmax)
{
    constexpr int kPer = kRmqTile / kThreads;  // 4 positions per thread
    __shared__ int32_t smin[kThreads / 32], smax[kThreads / 32];
    const int64_t ntiles = (n + kRmqTile - 1) / kRmqTile;
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int64_t p0 = t * kRmqTile + (int64_t)threadIdx.x * kPer;
        static_assert(kPer == 4, "one 16-byte load per array and thread");
        const bool whole = p0 + kPer <= n;   // the arrays' pieces are 256-byte aligned
        int32_t x4[kPer], y4[kPer];
        if (whole) {
            const int4 xv = *reinterpret_cast<const int4 *>(w1 + p0), yv = *reinterpret_cast<const int4 *>(w2 + p0);
            x4[0] = xv.x; x4[1] = xv.y; x4[2] = xv.z; x4[3] = xv.w;
            y4[0] = yv.x; y4[1] = yv.y; y4[2] = yv.z; y4[3] = yv.w;
        } else {
#pragma unroll
            for (int j = 0; j < kPer; ++j) {
                x4[j] = p0 + j < n ? w1[p0 + j] : INT32_MAX;
                y4[j] = p0 + j < n ? w2[p0 + j] : INT32_MIN;
            }
        }
        int32_t a[kPer], b[kPer];
        int32_t rmn = INT32_MAX, rmx = INT32_MIN;
#pragma unroll
        for (int j = 0; j < kPer; ++j) {
            const int32_t x = x4[j], y = y4[j];
            rmn = x < rmn ? x : rmn;
            rmx = y > rmx ? y : rmx;
            a[j] = rmn;
            b[j] = rmx;
        }
        // exclusive scan of the thread extrema across the CTA
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
        int32_t imn = rmn, imx = rmx;
        for (int o = 1; o < 32; o <<= 1) {
            int32_t y1 = __shfl_up_sync(0xffffffffu, imn, o), y2 = __shfl_up_sync(0xffffffffu, imx, o);
            if (lane >= o) {
                imn = y1 < imn ? y1 : imn;
                imx = y2 > imx ? y2 : imx;
            }
        }
        __syncthreads();
        if (lane == 31) { smin[wid] = imn; smax[wid] = imx; }
        __syncthreads();
        int32_t emn = INT32_MAX, emx = INT32_MIN, tmn = INT32_MAX, tmx = INT32_MIN;
#pragma unroll
        for (int i = 0; i < kThreads / 32; ++i) {
            if (i < wid) { emn = smin[i] < emn ? smin[i] : emn; emx = smax[i] > emx ? smax[i] : emx; }
            tmn = smin[i] < tmn ? smin[i] : tmn;
            tmx = smax[i] > tmx ? smax[i] : tmx;
        }
        int32_t xmn = __shfl_up_sync(0xffffffffu, imn, 1), xmx = __shfl_up_sync(0xffffffffu, imx, 1);
        if (lane > 0) {
            emn = xmn < emn ? xmn : emn;
            emx = xmx > emx ? xmx : emx;
        }
#pragma unroll
        for (int j = 0; j < kPer; ++j) {
            a[j] = a[j] < emn ? a[j] : emn;
            b[j] = b[j] > emx ? b[j] : emx;
        }
        if (whole) {
            int4 *o = reinterpret_cast<int4 *>(pmm + p0);
            o[0] = make_int4(a[0], b[0], a[1], b[1]);
            o[1] = make_int4(a[2], b[2], a[3], b[3]);
        } else {
#pragma unroll
            for (int j = 0; j < kPer; ++j)
                if (p0 + j < n) pmm[p0 + j] = make_int2(a[j], b[j]);
        }
        if (threadIdx.x == 0) {
            tmin[t] = tmn;
            tmax[t] = tmx;
        }
    }
}

// Sparse-table levels j0 .. j0+cnt-1 over the tile extrema (level j covers 2^j
// tiles), all from level j0-1 in one launch: level j0+q is the extremum of
// 2^(q+1) entries of level j0-1, h = 2^(j0-1) apart.
constexpr int kLevelsPerLaunch = 3;

__global__ void __launch_bounds__(kThreads) k_rmq_level(int64_t ntiles, int j0, int cnt, int64_t stride,
                                                        int32_t *tmin, int32_t *tmax)
{
    const int32_t *pm = tmin + (int64_t)(j0 - 1) * stride, *pM = tmax + (int64_t)(j0 - 1) * stride;
    const int64_t h = 1ll << (j0 - 1);
    GRID_STRIDE(t, ntiles)
    {
        int32_t a = pm[t], b = pM[t];
        int k = 1;
#pragma unroll
        for (int q = 0; q < kLevelsPerLaunch; ++q) {
            if (q >= cnt) break;
            for (; k < (2 << q); ++k) {   // fold in the entries k*h, up to 2^(q+1) of them
                const int64_t u = t + (int64_t)k * h;
                if (u < ntiles) {
                    a = pm[u] < a ? pm[u] : a;
                    b = pM[u] > b ? pM[u] : b;
                }
            }
            tmin[(int64_t)(j0 + q) * stride + t] = a;
            tmax[(int64_t)(j0 + q) * stride + t] = b;
        }
    }
}

// low/high for every position, the fence and bridge tests, and the start of
// Last-CC: every plain tree edge v-p(v) becomes the pointer lp[pos(v)] = pos(p(v))
// (fence edges and roots point to themselves), so each plain component is a tree
// of pointers to smaller preorder numbers whose root is its top vertex. Chains
// inside the tile are flattened in shared memory (pointer doubling); a pointer that
// leaves the tile marks its target in `ext` for the cross-tile resolution.
__global__ void __launch_bounds__(kThreads, 4) k_rmq_query(int64_t n, const int32_t *__restrict__ w1,
                                                        const int32_t *__restrict__ w2, const int2 *__restrict__ pmm,
                                                        const int32_t *__restrict__ tmin,
                                                        const int32_t *__restrict__ tmax, int64_t st_stride,
                                                        const int32_t *__restrict__ ord,
                                                        const int32_t *__restrict__ porig,
                                                        const int2 *__restrict__ fl,
                                                        const int32_t *__restrict__ lastp, uint8_t *vbits, int32_t *lp,
                                                        uint8_t *ext, int32_t *low_out, int32_t *high_out, int *err)
{
    constexpr int kPer = kRmqTile / kThreads;
    constexpr int kNChunk = kRmqTile / kChunk;
    constexpr int kCLv = 5;                                 // sparse-table levels over the 32 chunks
    __shared__ int32_t s1[kRmqTile], s2[kRmqTile];          // w1, w2
    __shared__ int32_t pre1[kRmqTile], pre2[kRmqTile];      // prefix within the chunk
    __shared__ int32_t suf1[kRmqTile], suf2[kRmqTile];      // suffix within the chunk
    __shared__ int32_t c1[kCLv][kNChunk], c2[kCLv][kNChunk];// sparse table of chunk extrema (level 0: chunks)
    __shared__ int32_t cs1[kNChunk], cs2[kNChunk];          // suffix over chunks (tile suffix helper)
    __shared__ int32_t sp[kRmqTile];                        // plain pointers of the tile
    const int64_t ntiles = (n + kRmqTile - 1) / kRmqTile;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int64_t base = t * kRmqTile;
        __syncthreads();
        for (int i = threadIdx.x; i < kRmqTile; i += kThreads) {
            int64_t p = base + i;
            s1[i] = p < n ? w1[p] : INT32_MAX;
            s2[i] = p < n ? w2[p] : INT32_MIN;
        }
        __syncthreads();
        // chunk prefix/suffix: warp w handles chunks w, w+8, ... one position per lane
        for (int c = wid; c < kNChunk; c += kThreads / 32) {
            int i = c * kChunk + lane;
            int32_t x = s1[i], y = s2[i], px = x, py = y, sx = x, sy = y;
            for (int o = 1; o < 32; o <<= 1) {
                int32_t a = __shfl_up_sync(0xffffffffu, px, o), b = __shfl_up_sync(0xffffffffu, py, o);
                int32_t a2 = __shfl_down_sync(0xffffffffu, sx, o), b2 = __shfl_down_sync(0xffffffffu, sy, o);
                if (lane >= o) { px = a < px ? a : px; py = b > py ? b : py; }
                if (lane + o < 32) { sx = a2 < sx ? a2 : sx; sy = b2 > sy ? b2 : sy; }
            }
            pre1[i] = px; pre2[i] = py; suf1[i] = sx; suf2[i] = sy;
            if (lane == 31) { c1[0][c] = px; c2[0][c] = py; }
        }
        __syncthreads();
        if (wid == 0) {
            // levels 1..4 of the chunk sparse table (level l covers 2^l chunks), and the
            // suffix extrema over chunks
            int32_t sa = c1[0][lane], sb = c2[0][lane];
            for (int lv = 1; lv < kCLv; ++lv) {
                const int h = 1 << (lv - 1);
                const int32_t a = __shfl_down_sync(0xffffffffu, sa, h), b = __shfl_down_sync(0xffffffffu, sb, h);
                if (lane + h < kNChunk) { sa = a < sa ? a : sa; sb = b > sb ? b : sb; }
                c1[lv][lane] = sa;
                c2[lv][lane] = sb;
            }
            int32_t x = c1[0][lane], y = c2[0][lane];
            for (int o = 1; o < 32; o <<= 1) {
                int32_t a = __shfl_down_sync(0xffffffffu, x, o), b = __shfl_down_sync(0xffffffffu, y, o);
                if (lane + o < 32) { x = a < x ? a : x; y = b > y ? b : y; }
            }
            cs1[lane] = x;
            cs2[lane] = y;
        }
        __syncthreads();
        // every position's range end, vertex and parent, and then the parent's
        // preorder interval and the range end's prefix extrema, all in flight
        // before the range queries
        int32_t ev[kPer], vv[kPer], xv[kPer], fxv[kPer], lxv[kPer];
        int2 pe[kPer];
#pragma unroll
        for (int k = 0; k < kPer; ++k) {
            const int64_t p = base + threadIdx.x + k * kThreads;
            ev[k] = (int32_t)p;
            vv[k] = -1;
            xv[k] = -1;
            if (p < n) {
                ev[k] = lastp[p];
                vv[k] = ord[p];
                xv[k] = porig[p];
            }
        }
#pragma unroll
        for (int k = 0; k < kPer; ++k) {
            const int64_t p = base + threadIdx.x + k * kThreads;
            fxv[k] = -1;
            lxv[k] = -1;
            pe[k] = make_int2(INT32_MAX, INT32_MIN);
            if (p >= n) continue;
            if ((uint32_t)xv[k] < (uint64_t)n) {
                const int2 f = __ldg(fl + xv[k]);
                fxv[k] = f.x;
                lxv[k] = f.y;
            }
            if (ev[k] >= base + kRmqTile && ev[k] < n) pe[k] = __ldg(pmm + ev[k]);
        }
#pragma unroll
        for (int k = 0; k < kPer; ++k) {
            // this warp holds one chunk (lane = position in it): a sparse table of
            // the chunk in registers answers ranges inside the chunk with two
            // shuffles per level, the same work for every lane
            const int i = threadIdx.x + k * kThreads;
            const int64_t p = base + i;
            const bool valid = p < n;
            int32_t e = ev[k];
            if (valid && (e < p || e >= n)) { atomicOr(err, kErrIndex); e = (int32_t)p; }
            const int ci = i / kChunk;
            const int jl = (int)(e - base) - ci * kChunk;          // e's lane when inside the chunk
            const bool in_chunk = jl < kChunk;
            int32_t ra = s1[i], rb = s2[i], lo = INT32_MAX, hi = INT32_MIN;
            const int len = in_chunk ? jl - lane + 1 : 1;
            const int kl = 31 - __clz(len);                          // 0..5
#pragma unroll
            for (int lv = 0; lv < 5; ++lv) {
                if (lv > 0) {   // ra/rb: extremum of the 2^lv positions from this lane on
                    const int h = 1 << (lv - 1);
                    const int32_t xa = __shfl_down_sync(0xffffffffu, ra, h), xb = __shfl_down_sync(0xffffffffu, rb, h);
                    if (lane + h < kChunk) { ra = xa < ra ? xa : ra; rb = xb > rb ? xb : rb; }
                }
                int src = (in_chunk ? jl : lane) - (1 << lv) + 1;
                src = src < 0 ? 0 : src;
                const int32_t ya = __shfl_sync(0xffffffffu, ra, src), yb = __shfl_sync(0xffffffffu, rb, src);
                if (lv == kl) { lo = ya < ra ? ya : ra; hi = yb > rb ? yb : rb; }
            }
            if (kl == 5) { lo = c1[0][ci]; hi = c2[0][ci]; }         // the whole chunk
            if (!valid) continue;
            if (e < base + kRmqTile) {
                const int je = (int)(e - base), ce = je / kChunk;
                if (ci != ce) {
                    lo = suf1[i] < pre1[je] ? suf1[i] : pre1[je];
                    hi = suf2[i] > pre2[je] ? suf2[i] : pre2[je];
                    if (ce > ci + 1) {   // whole chunks ci+1 .. ce-1: two overlapping table ranges
                        const int cl = ce - ci - 1, lv = 31 - __clz(cl), b = ce - (1 << lv);
                        const int32_t x = c1[lv][ci + 1] < c1[lv][b] ? c1[lv][ci + 1] : c1[lv][b];
                        const int32_t y = c2[lv][ci + 1] > c2[lv][b] ? c2[lv][ci + 1] : c2[lv][b];
                        lo = x < lo ? x : lo;
                        hi = y > hi ? y : hi;
                    }
                }
            } else {
                lo = suf1[i];
                hi = suf2[i];
                if (ci + 1 < kNChunk) {
                    lo = cs1[ci + 1] < lo ? cs1[ci + 1] : lo;
                    hi = cs2[ci + 1] > hi ? cs2[ci + 1] : hi;
                }
                const int64_t te = e / kRmqTile;
                if (te > t + 1) {  // whole tiles t+1 .. te-1: two overlapping sparse-table ranges
                    const int64_t a = t + 1, len = te - 1 - a + 1;
                    const int lv = 63 - __clzll(len);
                    const int64_t b = te - 1 - (1ll << lv) + 1;
                    const int32_t *lm = tmin + (int64_t)lv * st_stride, *lM = tmax + (int64_t)lv * st_stride;
                    int32_t x = lm[a] < lm[b] ? lm[a] : lm[b], y = lM[a] > lM[b] ? lM[a] : lM[b];
                    lo = x < lo ? x : lo;
                    hi = y > hi ? y : hi;
                }
                lo = pe[k].x < lo ? pe[k].x : lo;
                hi = pe[k].y > hi ? pe[k].y : hi;
            }
            if (low_out) {
                low_out[p] = lo;
                high_out[p] = hi;
            }
            const int32_t v = vv[k], x = xv[k];
            int32_t ptr = (int32_t)p;
            if (in_range(v, n, err) && x < n) {
                uint8_t bits = 0;
                if (x >= 0) {
                    if (lo == (int32_t)p && hi <= e) bits |= 1;  // bridge: nothing leaves T_v
                    const int32_t fx = fxv[k];
                    const bool fence = !in_range(fx, n, err) || (fx <= lo && lxv[k] >= hi);
                    if (fence) bits |= 2;
                    else ptr = fx;                                // plain tree edge: in G'
                }
                vbits[v] = bits;
            }
            sp[i] = ptr;
        }
        for (int i = threadIdx.x; i < kRmqTile; i += kThreads)
            if (base + i >= n) sp[i] = (int32_t)(base + i);
        __syncthreads();
        // pointer doubling inside the tile (10 rounds cover 1024 positions); pointers
        // only move towards their root, so updating in place is safe
        for (int r = 0; r < 10; ++r) {
#pragma unroll
            for (int k = 0; k < kPer; ++k) {
                const int i = threadIdx.x + k * kThreads;
                const int32_t q = sp[i];
                if (q >= base) sp[i] = sp[q - base];
            }
            __syncthreads();
        }
#pragma unroll
        for (int k = 0; k < kPer; ++k) {
            const int i = threadIdx.x + k * kThreads;
            const int64_t p = base + i;
            if (p >= n) continue;
            const int32_t t = sp[i];
            lp[p] = t;
            if (t < base) ext[t] = 1;
        }
    }
}

template <typename OffT>
cudaError_t launch_tagging(const Dev &d, const OffT *off, const int32_t *adj, int64_t n, int64_t nnz,
                           bool vec, bool keep_low_high, const Launch &L)
{
    k_first_of<<<grid_for(L, ceil_div(n, kThreads)), kThreads, 0, L.s>>>(n, d.fp, d.lastp, d.first4, d.fl);
    L.mark("k_first_of");
    const int64_t ntiles = ceil_div(nnz, kWTile);
    if (nnz > 0) {
        const int32_t *maxdeg = reinterpret_cast<const int32_t *>(d.counters + 5);
        k_w12<OffT, false><<<grid_for(L, ceil_div(ntiles, kWarpsPerCta)), kThreads, 0, L.s>>>(
            off, adj, nnz, d.tile_v, ntiles, d.fp, d.first4, d.w1, d.w2, d.dirb, n, d.err, vec, maxdeg);
        L.mark("k_w12");
        k_w12<OffT, true><<<grid_for(L, ceil_div(ntiles, kWarpsPerCta)), kThreads, 0, L.s>>>(
            off, adj, nnz, d.tile_v, ntiles, d.fp, d.first4, d.w1, d.w2, d.dirb, n, d.err, vec, maxdeg);
        L.mark("k_w12_keep");
    }
    const int64_t rt = ceil_div(n, kRmqTile);
    k_rmq_prefix<<<grid_for(L, rt), kThreads, 0, L.s>>>(n, d.w1, d.w2, d.pmm, d.tmin, d.tmax);
    L.mark("k_rmq_prefix");
    int top = 0;   // levels 1 .. top are needed: 2^top <= rt
    while ((2ll << top) <= rt) ++top;
    for (int j = 1; j <= top; j += kLevelsPerLaunch) {
        const int cnt = top - j + 1 < kLevelsPerLaunch ? top - j + 1 : kLevelsPerLaunch;
        k_rmq_level<<<grid_for(L, ceil_div(rt, kThreads)), kThreads, 0, L.s>>>(rt, j, cnt, d.rmq_tiles_max, d.tmin,
                                                                                 d.tmax);
        L.mark("k_rmq_level");
    }
    // Last-CC starts here: plain-edge pointers by preorder number
    cudaError_t e = cudaMemsetAsync(d.ext, 0, n, L.s);
    if (e != cudaSuccess) return e;
    k_rmq_query<<<grid_for(L, rt), kThreads, 0, L.s>>>(n, d.w1, d.w2, d.pmm, d.tmin, d.tmax,
                                                       d.rmq_tiles_max, d.ord, d.porig, d.fl, d.lastp,
                                                       d.vbits, d.lp, d.ext, keep_low_high ? d.low : nullptr,
                                                       keep_low_high ? d.high : nullptr, d.err);
    L.mark("k_rmq_query");
    return cudaGetLastError();
}

template cudaError_t launch_tagging<int32_t>(const Dev &, const int32_t *, const int32_t *, int64_t, int64_t, bool,
                                             bool, const Launch &);
template cudaError_t launch_tagging<int64_t>(const Dev &, const int64_t *, const int32_t *, int64_t, int64_t, bool,
                                             bool, const Launch &);

}  // namespace fbcc
