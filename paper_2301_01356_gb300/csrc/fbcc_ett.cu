// Rooting (Algorithm 1, step 2; section 2 "Euler tour technique" and section 5
// "Euler Tour Technique"): root every tree of the spanning forest at its
// component's smallest vertex and derive, per vertex, its parent, its preorder
// number first[v] and last[v] = first[v] + |T_v| - 1.
//
//  1. forest arcs: the edge recorded at hooked vertex h gives arcs 2h and 2h+1
//     (reverse = a ^ 1, no sort needed), and each vertex's arcs are chained into a
//     list (the paper semisorts the arcs by source instead); the arc passes later
//     recognise tree arcs by the parent relation, so the CSR is never marked;
//  2. Euler circuit: the arc u->v is followed by the arc after v->u in v's list,
//     cyclically (the paper's linking of u_i->v to v->u_{i+1}); each circuit is cut
//     before the root's first arc, which becomes the tour's head;
//  3. list ranking: rulers (every tour head plus one arc in `stride`) each walk
//     their successors up to the next ruler, recording owner and offset in the
//     link entries they pass; the ruler lists are sampled again and the top
//     level is ranked by pointer jumping; every arc's tour position follows from
//     its ruler's suffix length (the paper samples sqrt(n) nodes and chases
//     pointers between them; the GPU takes many more rulers so that every thread
//     has a short walk);
//  4. preorder: an arc is a down arc iff it precedes its reverse in the tour; a
//     prefix count of down arcs over tour positions numbers the vertices in
//     preorder: the down arc into v gives first[v], the up arc leaving v gives
//     last[v].
// Tours are laid out at positions [2*base, 2*base + 2*size) of their component
// (base = preorder number of the root; components take their ranges in any
// order); the last two slots are padding, one of which counts 1 so that the
// prefix count restarts at each component's base.
#include "fbcc_internal.cuh"

namespace fbcc {

#define GRID_STRIDE(i, n) \
    for (int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x; i < (n); i += (int64_t)gridDim.x * kThreads)

// Forest arcs: the edge recorded at hooked vertex h gives arcs 2h = u->v and
// 2h+1 = v->u, so an arc's reverse is a ^ 1 and ids need no scan; ids of vertices
// that hooked nothing are unused. Each vertex's arcs form a list threaded through
// nxt[] (pushed with atomicExch, in arbitrary order), headed by lhead[].
__device__ __forceinline__ int32_t arc_src(const int32_t *te_u, const int32_t *te_v, int64_t a)
{
    return (a & 1) ? te_v[a >> 1] : te_u[a >> 1];
}

__device__ __forceinline__ int32_t arc_dst(const int32_t *te_u, const int32_t *te_v, int64_t a)
{
    return (a & 1) ? te_u[a >> 1] : te_v[a >> 1];
}

// Forest edges renumbered component by component (fbcc_config.cc_order; the paper
// reorders the CSR after First-CC so that each connected component is contiguous):
// vertex v, whose slot holds the edge that hooked v (if any), moves to position
// base(root) + its rank among its component's vertices (in no particular order),
// so that each Euler tour's arcs 2h, 2h+1 and their link entries are contiguous.
// Counts and ranks per component: the lanes of a warp with the same root reduce
// and take their slots with one atomic per group.
__global__ void __launch_bounds__(kThreads) k_cc_count(int64_t n, const int32_t *__restrict__ uf, int32_t *cnt)
{
    const int64_t n_pad = (n + 31) & ~31ll;
    for (int64_t v = blockIdx.x * (int64_t)kThreads + threadIdx.x; v < n_pad; v += (int64_t)gridDim.x * kThreads) {
        const int32_t r = v < n ? uf[v] : -1;
        const unsigned peers = __match_any_sync(0xffffffffu, r);
        if (r >= 0 && (int)(threadIdx.x & 31) == __ffs(peers) - 1) atomicAdd(cnt + r, __popc(peers));
    }
}

__global__ void __launch_bounds__(kThreads) k_cc_place(int64_t n, const int32_t *__restrict__ uf,
                                                       const int32_t *__restrict__ base, int32_t *fill,
                                                       int32_t *pos)
{
    const int64_t n_pad = (n + 31) & ~31ll;
    const int lane = threadIdx.x & 31;
    for (int64_t v = blockIdx.x * (int64_t)kThreads + threadIdx.x; v < n_pad; v += (int64_t)gridDim.x * kThreads) {
        const int32_t r = v < n ? uf[v] : -1;
        const unsigned peers = __match_any_sync(0xffffffffu, r);
        const int leader = __ffs(peers) - 1;
        int32_t at = 0;
        if (r >= 0 && lane == leader) at = base[r] + atomicAdd(fill + r, __popc(peers));
        at = __shfl_sync(0xffffffffu, at, leader);
        if (r >= 0) pos[v] = at + __popc(peers & ((1u << lane) - 1u));
    }
}

__global__ void __launch_bounds__(kThreads) k_permute_te(int64_t n, const int32_t *__restrict__ pos,
                                                         const int32_t *__restrict__ te_u,
                                                         const int32_t *__restrict__ te_v,
                                                         const int32_t *__restrict__ te_a, int32_t *u2, int32_t *v2,
                                                         int32_t *a2, int *err)
{
    GRID_STRIDE(h, n)
    {
        const int32_t p = pos[h], u = te_u[h];
        if (!in_range(p, n, err)) continue;
        u2[p] = u;
        if (u >= 0) {
            v2[p] = te_v[h];
            if (te_a) a2[p] = te_a[h];
        }
    }
}

// Sub-list of edge h at a hub: a multiplicative hash of h, so that the sub-lists do
// not follow the low bits of the arc ids, which pick the rulers of the ranking (with
// h mod kHubSub, all of a hub's sampled arcs would fall into two sub-lists and the
// walks through the others would be as long as the sub-lists).
__device__ __forceinline__ int hub_sub(int64_t h)
{
    return (int)(((uint32_t)h * 2654435761u) >> 27);
}

// Forest-arc lists: each vertex's arcs chained through nxt by atomicExch on its list
// head. A hub (hubidx >= 0, found by First-CC; null when hubs are off) pushes onto
// one of kHubSub sub-lists chosen by a hash of the edge id instead, so that the
// exchanges of its many forest edges spread over kHubSub words; sub-list s of hub
// slot i has its head at hubhead[s * hub_cap + i], so that a hub's heads lie in
// different cache lines (atomics on one line are processed one at a time).
// Pushes of arcs onto lists, aggregated over the warp: the lanes that push onto
// the same list chain their arcs in lane order, and the first of them exchanges
// the list head once. Every lane takes part; a lane with head == nullptr pushes
// nothing. A push is split in two so that a thread's exchanges are all in flight
// together: push_group finds the lane's group (the first lane, which exchanges,
// and the next lane of the group, or -1 for the last, whose successor is the old
// head), the caller issues the exchanges, and push_resolve turns them into each
// arc's successor.
//  - runs: only runs of neighbouring lanes with the same list are joined (a
//    shuffle and a ballot find them: a hub's tree arcs often come in runs of edge
//    ids), which costs next to nothing where no list repeats;
//  - match: every lane of the warp with the same list (__match_any_sync), for
//    graphs with heavy hubs, whose list heads otherwise take a serialised
//    exchange per arc.
__device__ __forceinline__ void push_group(const int32_t *head, bool match, int &first, int &next)
{
    const int lane = threadIdx.x & 31;
    const unsigned long long key =
        head ? (unsigned long long)head : ~0ull - (unsigned long long)lane;   // an idle lane is alone
    if (match) {
        const unsigned peers = __match_any_sync(0xffffffffu, key);
        first = __ffs(peers) - 1;
        const unsigned above = peers & ~((2u << lane) - 1u);   // peers above this lane (2u << 31 wraps to 0)
        next = above ? __ffs(above) - 1 : -1;
    } else {
        const unsigned long long prev = __shfl_up_sync(0xffffffffu, key, 1);
        const unsigned starts = __ballot_sync(0xffffffffu, lane == 0 || prev != key);
        first = 31 - __clz(starts & ((2u << lane) - 1u));       // the run's start at or below this lane
        next = (lane == 31 || ((starts >> (lane + 1)) & 1u)) ? -1 : lane + 1;
    }
}

__device__ __forceinline__ int32_t push_resolve(int32_t old, int32_t a, int first, int next)
{
    const int lane = threadIdx.x & 31;
    const int32_t head_old = __shfl_sync(0xffffffffu, old, first);
    const int32_t next_a = __shfl_sync(0xffffffffu, a, next >= 0 ? next : lane);
    return next >= 0 ? next_a : head_old;
}


__global__ void __launch_bounds__(kThreads) k_link(int64_t n, const int32_t *__restrict__ te_u,
                                                   const int32_t *__restrict__ te_v,
                                                   const int32_t *__restrict__ hubidx, int32_t *lhead,
                                                   int32_t *hubhead, int64_t hub_cap, int32_t *nxt,
                                                   const int32_t *__restrict__ maxdeg)
{
    const bool match = *maxdeg >= kHeavyDeg;   // the same in every thread
    const int lane = threadIdx.x & 31;
    // four edges per thread and step: their loads, and then their eight exchanges,
    // in flight together
    constexpr int kPer = 4;
    const int64_t T = (int64_t)gridDim.x * kThreads;
    const int64_t n_pad = (n + 31) & ~31ll;
    for (int64_t h0 = blockIdx.x * (int64_t)kThreads + threadIdx.x; h0 < n_pad; h0 += T * kPer) {
        int32_t u[kPer], v[kPer];
#pragma unroll
        for (int k = 0; k < kPer; ++k) {
            const int64_t h = h0 + k * T;
            u[k] = h < n ? te_u[h] : -1;
            v[k] = u[k] >= 0 ? te_v[h] : -1;
        }
        int32_t hu[kPer], hv[kPer];
#pragma unroll
        for (int k = 0; k < kPer; ++k) {
            hu[k] = hv[k] = -1;
            if (u[k] < 0 || !hubidx) continue;
            hu[k] = __ldg(hubidx + u[k]);
            hv[k] = __ldg(hubidx + v[k]);
        }
        int first[2 * kPer], next[2 * kPer];
        int32_t old[2 * kPer];
#pragma unroll
        for (int j = 0; j < 2 * kPer; ++j) {
            const int k = j >> 1;
            const int64_t h = h0 + k * T;
            const int s = hub_sub(h);   // the sub-list of both arcs of edge h
            int32_t *p = nullptr;
            if (u[k] >= 0) {
                if (j & 1) p = hv[k] >= 0 ? hubhead + (int64_t)s * hub_cap + hv[k] : lhead + v[k];
                else p = hu[k] >= 0 ? hubhead + (int64_t)s * hub_cap + hu[k] : lhead + u[k];
            }
            push_group(p, match, first[j], next[j]);
            old[j] = (p && lane == first[j]) ? atomicExch(p, (int32_t)(2 * h + (j & 1))) : 0;
        }
#pragma unroll
        for (int k = 0; k < kPer; ++k) {
            const int64_t h = h0 + k * T;
            int2 o;
            o.x = push_resolve(old[2 * k], (int32_t)(2 * h), first[2 * k], next[2 * k]);
            o.y = push_resolve(old[2 * k + 1], (int32_t)(2 * h + 1), first[2 * k + 1], next[2 * k + 1]);
            if (u[k] >= 0) *reinterpret_cast<int2 *>(nxt + 2 * h) = o;
        }
    }
}

// A hub's sub-lists in one cyclic order: each non-empty sub-list is followed by the
// next non-empty one (hubnext, -1 after the last), and the hub's list starts with
// the first (lhead), so that the successor pass sees one list per vertex. A warp
// per hub slot, a lane per sub-list.
__global__ void __launch_bounds__(kThreads) k_hub_order(const long long *__restrict__ nhub_p, int64_t hub_cap,
                                                        const int32_t *__restrict__ hubvert,
                                                        const int32_t *__restrict__ hubhead, int32_t *hubnext,
                                                        int32_t *lhead)
{
    const long long nh = *nhub_p;
    const int64_t cnt = nh < hub_cap ? nh : hub_cap;
    const int lane = threadIdx.x & 31;
    static_assert(kHubSub == 32, "a lane per sub-list");
    for (int64_t i = (blockIdx.x * (int64_t)kThreads + threadIdx.x) >> 5; i < cnt;
         i += ((int64_t)gridDim.x * kThreads) >> 5) {
        const int32_t hd = hubhead[(int64_t)lane * hub_cap + i];
        const unsigned m = __ballot_sync(0xffffffffu, hd >= 0);
        const unsigned later = lane == 31 ? 0u : m & ~((2u << lane) - 1u);
        const int nx = later ? __ffs(later) - 1 : -1;
        const int32_t nh2 = __shfl_sync(0xffffffffu, hd, nx < 0 ? 0 : nx);
        hubnext[i * kHubSub + lane] = nx < 0 ? -1 : nh2;
        const int32_t first = __shfl_sync(0xffffffffu, hd, m ? __ffs(m) - 1 : 0);
        if (lane == 0) lhead[hubvert[i]] = m ? first : -1;
    }
}

// Euler successor of every arc and the rulers of the list ranking, in one pass.
// succ(a) for a = x->y is the arc after a^1 in y's list, cyclically; when y is a
// component root the wrap-around ends the tour instead, and the first arc of the
// root's list heads it. Rulers: tour heads plus every arc id divisible by the
// stride. link[a] = {succ, ruler id or -1} ({-1, -1} for the unused ids of
// vertices that hooked nothing); relem[id] = a; rhead[id] = 1 if the ruler heads
// its tour. A thread takes four consecutive forest edges (eight arcs, loaded and
// stored as 16-byte vectors); ids come from one atomic per CTA and step of kTile
// arcs.
__global__ void __launch_bounds__(kThreads) k_succ_rulers(int64_t n, const int32_t *__restrict__ te_u,
                                                          const int32_t *__restrict__ te_v,
                                                          const int32_t *__restrict__ uf,
                                                          const int32_t *__restrict__ lhead,
                                                          const int32_t *__restrict__ nxt,
                                                          const int32_t *__restrict__ hubidx,
                                                          const int32_t *__restrict__ hubnext, int stride, int2 *link,
                                                          uint8_t *rhead, int32_t *relem, long long *nr)
{
    constexpr int kE = kItems / 2;   // forest edges per thread and step
    static_assert(kE == 4, "one 16-byte load of te_u and te_v per thread");
    __shared__ int32_t warp_cnt[kThreads / 32];
    __shared__ long long block_base;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t ntiles = (n + kThreads * kE - 1) / (kThreads * kE);
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {   // whole CTAs take part
        const int64_t h0 = (t * kThreads + threadIdx.x) * kE;
        // the workspace's pieces are 256-byte aligned and h0 is a multiple of 4
        const bool whole = h0 + kE <= n;
        int32_t eu[kE], ev[kE], nx[2 * kE];
        if (whole) {
            const int4 a = *reinterpret_cast<const int4 *>(te_u + h0), b = *reinterpret_cast<const int4 *>(te_v + h0);
            const int4 c = *reinterpret_cast<const int4 *>(nxt + 2 * h0);
            const int4 d = *reinterpret_cast<const int4 *>(nxt + 2 * h0 + 4);
            eu[0] = a.x; eu[1] = a.y; eu[2] = a.z; eu[3] = a.w;
            ev[0] = b.x; ev[1] = b.y; ev[2] = b.z; ev[3] = b.w;
            nx[0] = c.x; nx[1] = c.y; nx[2] = c.z; nx[3] = c.w; nx[4] = d.x; nx[5] = d.y; nx[6] = d.z; nx[7] = d.w;
        } else {
#pragma unroll
            for (int k = 0; k < kE; ++k) {
                const bool in = h0 + k < n;
                eu[k] = in ? te_u[h0 + k] : -1;
                ev[k] = in ? te_v[h0 + k] : -1;
                nx[2 * k] = in ? nxt[2 * (h0 + k)] : -1;
                nx[2 * k + 1] = in ? nxt[2 * (h0 + k) + 1] : -1;
            }
        }
        int32_t sc[2 * kE];
        unsigned head = 0, ruler = 0;
#pragma unroll
        for (int j = 0; j < 2 * kE; ++j) {
            const int k = j >> 1;
            const int64_t a = 2 * h0 + j;
            sc[j] = -1;
            if (eu[k] < 0) continue;
            const int32_t x = (j & 1) ? ev[k] : eu[k], y = (j & 1) ? eu[k] : ev[k];
            int32_t nxr = nx[j ^ 1];   // nxt of the reverse arc
            if (nxr < 0 && hubidx) {   // the reverse arc ends a (sub-)list of y
                const int32_t hy = hubidx[y];
                if (hy >= 0) nxr = hubnext[(int64_t)hy * kHubSub + hub_sub(h0 + k)];
            }
            sc[j] = nxr >= 0 ? nxr : (uf[y] == y ? -1 : lhead[y]);
            if (uf[x] == x && lhead[x] == a) head |= 1u << j;
            if (((head >> j) & 1u) || (a & (stride - 1)) == 0) ruler |= 1u << j;
        }
        const int cnt = __popc(ruler);
        int inc = cnt;
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += y;
        }
        if (lane == 31) warp_cnt[wid] = inc;
        __syncthreads();
        if (threadIdx.x == 0) {
            int32_t tot = 0;
            for (int w = 0; w < kThreads / 32; ++w) tot += warp_cnt[w];
            block_base = tot ? (long long)atomicAdd((unsigned long long *)nr, (unsigned long long)tot) : 0;
        }
        __syncthreads();
        long long id = block_base + inc - cnt;
        for (int w = 0; w < wid; ++w) id += warp_cnt[w];
        __syncthreads();  // warp_cnt / block_base are rewritten next step
        int32_t rid[2 * kE];
#pragma unroll
        for (int j = 0; j < 2 * kE; ++j) {
            rid[j] = -1;
            if ((ruler >> j) & 1u) {
                rid[j] = (int32_t)id++;
                relem[rid[j]] = (int32_t)(2 * h0 + j);
                rhead[rid[j]] = (head >> j) & 1u;
            }
        }
        if (whole) {
            int4 *o = reinterpret_cast<int4 *>(link + 2 * h0);
#pragma unroll
            for (int q = 0; q < kE; ++q) o[q] = make_int4(sc[2 * q], rid[2 * q], sc[2 * q + 1], rid[2 * q + 1]);
        } else {
#pragma unroll
            for (int j = 0; j < 2 * kE; ++j)
                if (h0 + (j >> 1) < n) link[2 * h0 + j] = make_int2(sc[j], rid[j]);
        }
    }
}

// Each ruler walks its successors until the next ruler or the tour's end. A
// thread advances kChains rulers' walks in lock step, so it keeps that many
// independent loads in flight (the walk is bound by load latency). Every
// non-ruler arc is visited by exactly one walk, which overwrites its link entry
// (just read) with {owning ruler, -distance from it}: a ruler's entry keeps
// {successor, ruler id >= 0}, so the sign of .y tells the two apart afterwards,
// and the write lands in a line the walk has just loaded.
template <int kChains>
__global__ void __launch_bounds__(kThreads) k_chase(int64_t n,
                                                    const long long *__restrict__ nr_p, const int32_t *__restrict__ relem,
                                                    int2 *link, int32_t *rnext, int32_t *rlen, int *err)
{
    const int64_t A = 2 * n;
    const int64_t nr = *nr_p;
    const int64_t T = (int64_t)gridDim.x * kThreads;
    for (int64_t r0 = blockIdx.x * (int64_t)kThreads + threadIdx.x; r0 < nr; r0 += T * kChains) {
        int32_t t[kChains], acc[kChains], nxr[kChains];
        int64_t steps = 0;
        unsigned live = 0;
#pragma unroll
        for (int k = 0; k < kChains; ++k) {
            const int64_t r = r0 + k * T;
            acc[k] = 1;
            nxr[k] = -1;
            t[k] = -1;
            if (r < nr) {
                t[k] = link[relem[r]].x;
                if (t[k] >= 0) live |= 1u << k;
            }
        }
        while (live) {
            int2 lk[kChains];
#pragma unroll
            for (int k = 0; k < kChains; ++k)
                if ((live >> k) & 1u) lk[k] = link[t[k]];
#pragma unroll
            for (int k = 0; k < kChains; ++k) {
                if (!((live >> k) & 1u)) continue;
                if (lk[k].y >= 0) {
                    nxr[k] = lk[k].y;
                    live &= ~(1u << k);
                    continue;
                }
                link[t[k]] = make_int2((int32_t)(r0 + k * T), -(acc[k]++));
                t[k] = lk[k].x;
                if (t[k] < 0) live &= ~(1u << k);
            }
            if (++steps > A) {
                atomicOr(err, kErrChase);
                break;
            }
        }
#pragma unroll
        for (int k = 0; k < kChains; ++k) {
            const int64_t r = r0 + k * T;
            if (r < nr) {
                rnext[r] = nxr[k];
                rlen[r] = acc[k];
            }
        }
    }
}

// One more level of the ranking: the lists of the level below (next_lo, with
// head flags head_lo) are sampled again. A list of one node (a short tour) is
// finished already (marked -2); the others' heads and every stride-th node become
// nodes of this level, which inherit the head flag.
__global__ void __launch_bounds__(kThreads) k_lvl_rulers(const long long *__restrict__ cnt_lo_p, int stride,
                                                         const int32_t *__restrict__ next_lo,
                                                         const uint8_t *__restrict__ head_lo, int2 *l,
                                                         int32_t *relem, uint8_t *head_up, long long *cnt_up,
                                                         int64_t cap_up, int *err)
{
    __shared__ int32_t warp_cnt[kThreads / 32];
    __shared__ long long block_base;
    const int64_t nr = *cnt_lo_p;
    const int64_t pad = (nr + kThreads - 1) / kThreads * kThreads;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int64_t r = blockIdx.x * (int64_t)kThreads + threadIdx.x; r < pad; r += (int64_t)gridDim.x * kThreads) {
        const bool in = r < nr;
        bool single = false, ruler = false, head = false;
        int32_t nx = -1;
        if (in) {
            head = head_lo[r];
            nx = next_lo[r];
            single = head && nx < 0;
            ruler = !single && (head || (r & (stride - 1)) == 0);
        }
        const unsigned mask = __ballot_sync(0xffffffffu, ruler);
        if (lane == 0) warp_cnt[wid] = __popc(mask);
        __syncthreads();
        if (threadIdx.x == 0) {
            int32_t c = 0;
            for (int w = 0; w < kThreads / 32; ++w) c += warp_cnt[w];
            block_base = c ? (long long)atomicAdd((unsigned long long *)cnt_up, (unsigned long long)c) : 0;
        }
        __syncthreads();
        int32_t before = 0;
        for (int w = 0; w < wid; ++w) before += warp_cnt[w];
        const long long base = block_base + before;
        __syncthreads();
        if (!in) continue;
        int32_t id = single ? -2 : -1;
        if (ruler) {
            const long long at = base + __popc(mask & ((1u << lane) - 1u));
            if (in_range(at, cap_up, err)) {
                id = (int32_t)at;
                relem[id] = (int32_t)r;
                head_up[id] = head;
            }
        }
        l[r] = make_int2(nx, id);
    }
}

// Walks of this level over the lists below, weighted by the segment weights below:
// every node below learns its owner here and its weighted offset from it; every
// node here its next node and its segment weight.
__global__ void __launch_bounds__(kThreads) k_lvl_chase(const long long *__restrict__ cnt_lo_p,
                                                        const long long *__restrict__ cnt_up_p,
                                                        const int32_t *__restrict__ relem, const int2 *__restrict__ l,
                                                        const int32_t *__restrict__ w_lo, int32_t *owner,
                                                        int32_t *offs, int32_t *next_up, int32_t *w_up, int *err)
{
    const int64_t nr = *cnt_lo_p, nr2 = *cnt_up_p;
    GRID_STRIDE(R, nr2)
    {
        const int32_t r0 = relem[R];
        owner[r0] = (int32_t)R;
        offs[r0] = 0;
        int32_t acc = w_lo[r0], nxr = -1;
        int32_t t = l[r0].x;
        int64_t steps = 0;
        while (t >= 0) {
            const int2 lk = l[t];
            if (lk.y >= 0) { nxr = lk.y; break; }
            owner[t] = (int32_t)R;
            offs[t] = acc;
            acc += w_lo[t];
            t = lk.x;
            if (++steps > nr) { atomicOr(err, kErrChase); break; }
        }
        next_up[R] = nxr;
        w_up[R] = acc;
    }
}

// Suffix weights of the nodes below from those of this level.
__global__ void __launch_bounds__(kThreads) k_lvl_expand(const long long *__restrict__ cnt_lo_p,
                                                         const int2 *__restrict__ l, const int32_t *__restrict__ w_lo,
                                                         const int32_t *__restrict__ owner,
                                                         const int32_t *__restrict__ offs,
                                                         const int32_t *__restrict__ sd_up, int32_t *sd_lo)
{
    const int64_t nr = *cnt_lo_p;
    GRID_STRIDE(r, nr)
    {
        sd_lo[r] = l[r].y == -2 ? w_lo[r] : sd_up[owner[r]] - offs[r];
    }
}

// One grid-wide round of pointer jumping over the ruler lists: val = suffix weight.
__global__ void __launch_bounds__(kThreads) k_jump(const long long *__restrict__ nr_p, const int32_t *__restrict__ nx_in,
                                                   const int32_t *__restrict__ val_in, int32_t *nx_out, int32_t *val_out)
{
    const int64_t nr = *nr_p;
    GRID_STRIDE(r, nr)
    {
        const int32_t x = nx_in[r];
        if (x >= 0) {
            val_out[r] = val_in[r] + val_in[x];
            nx_out[r] = nx_in[x];
        } else {
            val_out[r] = val_in[r];
            nx_out[r] = -1;
        }
    }
}

// The top level: suffix weights of every node by pointer jumping, in one CTA. Up
// to kTopCap nodes live in shared memory (each round reads every pointer and
// value, synchronises, writes, and stops when no pointer moved); more nodes take
// the same rounds over global double buffers.
__global__ void __launch_bounds__(kTopThreads) k_top(const long long *__restrict__ cnt_p,
                                                     const int32_t *__restrict__ next, const int32_t *__restrict__ w,
                                                     int32_t *sd, int32_t *g0n, int32_t *g0v, int32_t *g1n,
                                                     int32_t *g1v, int64_t gcap, int *err)
{
    extern __shared__ __align__(16) int32_t top_smem[];
    const int64_t cnt = *cnt_p;
    const int tid = threadIdx.x;
    if (cnt <= kTopCap) {
        const int n = (int)cnt;
        int32_t *s_nx = top_smem, *s_v = top_smem + kTopCap;
        for (int i = tid; i < n; i += kTopThreads) {
            s_nx[i] = next[i];
            s_v[i] = w[i];
        }
        __syncthreads();
        bool done = false;
        for (int round = 0; round < 40 && !done; ++round) {
            int32_t nn[kTopPer], nv[kTopPer];
            int moved = 0;
#pragma unroll
            for (int k = 0; k < kTopPer; ++k) {
                const int i = tid + k * kTopThreads;
                nn[k] = -1;
                if (i < n) {
                    const int32_t x = s_nx[i];
                    nv[k] = s_v[i];
                    if (x >= 0) {
                        nv[k] += s_v[x];
                        nn[k] = s_nx[x];
                        moved = 1;
                    }
                }
            }
            __syncthreads();
#pragma unroll
            for (int k = 0; k < kTopPer; ++k) {
                const int i = tid + k * kTopThreads;
                if (i < n) {
                    s_nx[i] = nn[k];
                    s_v[i] = nv[k];
                }
            }
            done = !__syncthreads_or(moved);
        }
        if (!done && tid == 0) atomicOr(err, kErrChase);
        for (int i = tid; i < n; i += kTopThreads) sd[i] = s_v[i];
        return;
    }
    if (cnt > gcap) {
        if (tid == 0) atomicOr(err, kErrIndex);
        return;
    }
    const int32_t *rn = next, *rv = w;
    int32_t *on = g0n, *ov = g0v, *sn = g1n, *sv = g1v;   // written this round, the round after
    bool done = false;
    for (int round = 0; round < 40 && !done; ++round) {
        int moved = 0;
        for (int64_t i = tid; i < cnt; i += kTopThreads) {
            const int32_t x = rn[i];
            int32_t v = rv[i], nx = -1;
            if (x >= 0) {
                v += rv[x];
                nx = rn[x];
                moved = 1;
            }
            on[i] = nx;
            ov[i] = v;
        }
        done = !__syncthreads_or(moved);
        rn = on;
        rv = ov;
        int32_t *tn = on, *tv = ov;
        on = sn;
        ov = sv;
        sn = tn;
        sv = tv;
    }
    if (!done && tid == 0) atomicOr(err, kErrChase);
    for (int64_t i = tid; i < cnt; i += kTopThreads) sd[i] = rv[i];
}

cudaError_t prepare_rooting()
{
    return cudaFuncSetAttribute(k_top, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)(2 * kTopCap * sizeof(int32_t)));
}

// Component size at its root (1 for an isolated root, else tour length / 2 + 1)
// and the component's first preorder number. The components may take the
// preorder range in any order (only the order inside a component matters), so
// each CTA reserves one block of the range with one atomic per step of kTile
// vertices (kItems consecutive ones per thread, loaded as 16-byte vectors) and
// hands it out to its roots by a block scan: no separate scan pass over all
// vertices. Only roots are written. The root also writes its own tags (preorder
// number b, last b + size - 1, no parent) and the two padding records that end
// its tour's slot in the record array (the arcs fill the slot's first
// 2 (size - 1) positions): a counting one, so that the count restarts right at
// the next component's base, and a neutral one.
__global__ void __launch_bounds__(kThreads) k_comp_size(int64_t n, const int32_t *__restrict__ uf,
                                                        const int32_t *__restrict__ lhead,
                                                        const int2 *__restrict__ link, const int32_t *__restrict__ sd,
                                                        const long long *nr_p, int32_t *csize, int32_t *vbase,
                                                        long long *next_base, int2 *rec, int2 *fp, int32_t *lastp,
                                                        int32_t *ord, int32_t *porig, int32_t *w1, int32_t *w2,
                                                        int *err)
{
    static_assert(kItems == 8, "two 16-byte loads per thread");
    __shared__ long long warp_tot[kThreads / 32];
    __shared__ long long block_base;
    __shared__ int32_t s_c[kTile + kTile / 32], s_b[kTile + kTile / 32];   // padded against bank conflicts
    const int64_t nr = *nr_p;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t ntiles = (n + kTile - 1) / kTile;
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {     // whole CTAs take part
        const int64_t v0 = t * kTile + (int64_t)threadIdx.x * kItems;
        int32_t p[kItems];
        if (v0 + kItems <= n) {   // uf is a 256-byte aligned workspace piece
            const int4 a = *reinterpret_cast<const int4 *>(uf + v0), b = *reinterpret_cast<const int4 *>(uf + v0 + 4);
            p[0] = a.x; p[1] = a.y; p[2] = a.z; p[3] = a.w; p[4] = b.x; p[5] = b.y; p[6] = b.z; p[7] = b.w;
        } else {
#pragma unroll
            for (int j = 0; j < kItems; ++j) p[j] = v0 + j < n ? uf[v0 + j] : -1;
        }
        int32_t c[kItems];
        long long run = 0;
#pragma unroll
        for (int j = 0; j < kItems; ++j) {
            const int64_t v = v0 + j;
            c[j] = 0;
            if (p[j] == v) {
                c[j] = 1;
                const int32_t h = lhead[v];
                if (h >= 0) {
                    const int32_t id = link[h].y;
                    if (in_range(id, nr, err)) c[j] = sd[id] / 2 + 1;
                }
            }
            run += c[j];
        }
        long long inc = run;
        for (int o = 1; o < 32; o <<= 1) {
            const long long y = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += y;
        }
        if (lane == 31) warp_tot[wid] = inc;
        __syncthreads();
        if (threadIdx.x == 0) {
            long long tot = 0;
            for (int w = 0; w < kThreads / 32; ++w) tot += warp_tot[w];
            block_base = tot ? (long long)atomicAdd((unsigned long long *)next_base, (unsigned long long)tot) : 0;
        }
        __syncthreads();
        long long b = block_base + inc - run;
        for (int w = 0; w < wid; ++w) b += warp_tot[w];
        // the roots' writes go out in vertex order across the lanes (slot e holds
        // vertex t * kTile + e), so that neighbouring lanes write neighbouring words
#pragma unroll
        for (int j = 0; j < kItems; ++j) {
            const int e = threadIdx.x * kItems + j;
            s_c[e + (e >> 5)] = c[j];
            s_b[e + (e >> 5)] = (int32_t)b;
            b += c[j];
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < kItems; ++k) {
            const int e = k * kThreads + threadIdx.x;
            const int32_t cc = s_c[e + (e >> 5)];
            if (!cc) continue;
            const int64_t v = t * kTile + e;
            const int32_t bb = s_b[e + (e >> 5)];
            csize[v] = cc;
            vbase[v] = bb;
            rec[2 * (int64_t)bb + 2 * cc - 2] = make_int2(-2, 0);
            rec[2 * (int64_t)bb + 2 * cc - 1] = make_int2(-3, 0);
            fp[v] = make_int2(bb, -1);
            lastp[bb] = bb + cc - 1;
            ord[bb] = (int32_t)v;
            porig[bb] = -1;
            w1[bb] = bb;
            w2[bb] = bb;
        }
        __syncthreads();   // warp_tot, block_base and the staging are rewritten next step
    }
}

// Up-arc records hold kUpRec - child (below the padding markers -2 and -3).
constexpr int32_t kUpRec = -4;

// Tour positions of both arcs of every forest edge, and their tour records. The
// position of arc s is its tour's base (2 * vbase at the root r) plus the tour
// length L = 2 (size(r) - 1) minus its distance to the tour's end, which is the
// owning ruler's suffix length minus the arc's distance from that ruler. The
// earlier of the two arcs is the down arc: it stores {child, parent}; the up
// arc stores {kUpRec - child, its distance back to the down arc}. parc[child] is
// the CSR position of the arc parent -> child when First-CC hooked the edge from
// that arc, else -1.
__global__ void __launch_bounds__(kThreads) k_place_records(int64_t n, const int32_t *__restrict__ te_u,
                                                            const int32_t *__restrict__ te_v,
                                                            const int32_t *__restrict__ te_a, int32_t *parc,
                                                            const int32_t *__restrict__ uf,
                                                            const int32_t *__restrict__ csize,
                                                            const int32_t *__restrict__ vbase,
                                                            const int2 *__restrict__ link,
                                                            const int32_t *__restrict__ sd, int2 *rec, int *err)
{
    GRID_STRIDE(h, n)
    {
        const int32_t u = te_u[h];
        if (u < 0) continue;
        const int32_t v = te_v[h];
        const int32_t r = uf[u];
        const int32_t L = 2 * (csize[r] - 1);
        const int32_t base = 2 * vbase[r] + L;
        const int4 lk = *reinterpret_cast<const int4 *>(link + 2 * h);   // arcs 2h (u->v) and 2h+1 (v->u)
        const int32_t d0 = lk.y >= 0 ? sd[lk.y] : sd[lk.x] + lk.y;
        const int32_t d1 = lk.w >= 0 ? sd[lk.w] : sd[lk.z] + lk.w;
        if (!in_range(d0 - 1, L, err) || !in_range(d1 - 1, L, err)) continue;
        const int32_t p0 = base - d0, p1 = base - d1;
        // the child learns the CSR position of the arc from its parent when the edge
        // was hooked from that arc (u -> v)
        if (p0 < p1) {
            rec[p0] = make_int2(v, u);
            rec[p1] = make_int2(kUpRec - v, p1 - p0);
            if (parc) parc[v] = te_a[h];
        } else {
            rec[p1] = make_int2(u, v);
            rec[p0] = make_int2(kUpRec - u, p0 - p1);
            if (parc) parc[u] = -1;
        }
    }
}

// Preorder from the tour (single-pass scan over the 2n tour positions). With S(p)
// the number of counting positions before p: a down arc into v gives
// first[v] = S(p) + 1, and the up arc leaving v gives last[v] = S(q). The tour
// of T_v spans positions p..q, two per vertex, so size(v) = (q - p + 1) / 2 and
// the up arc also knows first[v] = S(q) - (q - p - 1) / 2: it stores last by
// preorder number. Only fp is written by vertex id.
__global__ void __launch_bounds__(kThreads, 5) k_preorder(int64_t n2, const int2 *__restrict__ rec, int2 *fp,
                                                       int32_t *lastp, int32_t *ord, int32_t *porig, int32_t *w1,
                                                       int32_t *w2, long long *ticket, uint64_t *status, int *err)
{
    // the tile's records pass through shared memory: coalesced loads, then each
    // thread takes its kItems consecutive records (slot e at e + e / 8 keeps the
    // 8-byte reads of a warp free of bank conflicts)
    __shared__ int2 srec[kTile + kTile / 8];
    __shared__ long long s_base;
    static_assert(2 * kTile * sizeof(int32_t) <= sizeof(srec), "staging fits in the record buffer");
    const int64_t ntiles = (n2 + kTile - 1) / kTile;
    const int64_t n = n2 / 2;
    while (true) {
        int64_t t = scan_ticket(ticket);
        if (t >= ntiles) return;
#pragma unroll
        for (int k = 0; k < kItems; ++k) {
            const int e = k * kThreads + threadIdx.x;
            const int64_t p = t * kTile + e;
            srec[e + (e >> 3)] = p < n2 ? __ldcs(rec + p) : make_int2(-3, 0);
        }
        __syncthreads();
        long long v[kItems];
        int2 r[kItems];
#pragma unroll
        for (int j = 0; j < kItems; ++j) {
            const int e = threadIdx.x * kItems + j;
            r[j] = srec[e + (e >> 3)];
            v[j] = r[j].x >= 0 || r[j].x == -2;
        }
        scan_tile_exclusive(v, t, status, err);
        // The tile's counting positions take consecutive preorder numbers from
        // the tile's base on, so the arrays indexed by preorder number are staged
        // in shared memory (srec is free again: the scan synchronised the CTA)
        // and written out coalesced; slot i holds preorder number base + i + 1.
        int32_t *s_ord = reinterpret_cast<int32_t *>(srec), *s_porig = s_ord + kTile;
        if (threadIdx.x == 0) s_base = v[0];
#pragma unroll
        for (int k = 0; k < kItems; ++k) s_ord[k * kThreads + threadIdx.x] = -1;
        __syncthreads();
        const long long base = s_base;
#pragma unroll
        for (int j = 0; j < kItems; ++j) {
            if (r[j].x >= 0) {
                const int32_t vtx = r[j].x, x = r[j].y, fv = (int32_t)v[j] + 1;
                if (!in_range(fv, n, err) || !in_range(vtx, n, err)) continue;
                fp[vtx] = make_int2(fv, x);
                s_ord[v[j] - base] = vtx;
                s_porig[v[j] - base] = x;
            } else if (r[j].x <= kUpRec) {
                const int32_t e = (int32_t)v[j], fv = e - (r[j].y - 1) / 2;
                if (in_range(fv, n, err) && fv <= e) lastp[fv] = e;
            }
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < kItems; ++k) {
            const int i = k * kThreads + threadIdx.x;
            const int32_t o = s_ord[i];
            if (o < 0) continue;
            const int32_t fv = (int32_t)(base + i + 1);
            ord[fv] = o;
            porig[fv] = s_porig[i];
            w1[fv] = fv;
            w2[fv] = fv;
        }
        __syncthreads();   // the next tile's records overwrite the staging
    }
}

template <typename OffT>
cudaError_t launch_rooting(const Dev &d, const OffT *off, const int32_t *adj, int64_t n, int64_t nnz,
                           int ruler_stride, int chase_chains, int rank_variant, int cc_order, bool hubs,
                           const Launch &L)
{
    (void)off;
    const int32_t *te_u = d.te_u, *te_v = d.te_v, *te_a = d.te_a;
    if (cc_order) {
        // counts, bases and positions live in the link array, which is free until the
        // successor pass (4n int32 slots; 3n + 1 are needed)
        int32_t *cnt = reinterpret_cast<int32_t *>(d.link), *fill = cnt + n + 1, *pos = fill + n;
        cudaError_t e0 = cudaMemsetAsync(cnt, 0, (2 * n + 1) * sizeof(int32_t), L.s);
        if (e0 != cudaSuccess) return e0;
        const int gn = grid_for(L, ceil_div(n, kThreads));
        k_cc_count<<<gn, kThreads, 0, L.s>>>(n, d.uf, cnt);
        L.mark("k_cc_count");
        e0 = launch_scan_i32(d, cnt, n, L);
        if (e0 != cudaSuccess) return e0;
        k_cc_place<<<gn, kThreads, 0, L.s>>>(n, d.uf, cnt, fill, pos);
        L.mark("k_cc_place");
        k_permute_te<<<gn, kThreads, 0, L.s>>>(n, pos, d.te_u, d.te_v, hubs ? d.te_a : nullptr, d.te2_u, d.te2_v,
                                               d.te2_a, d.err);
        L.mark("k_permute_te");
        te_u = d.te2_u;
        te_v = d.te2_v;
        te_a = d.te2_a;
    }
    (void)nnz;
    const int gv = grid_for(L, ceil_div(n, kThreads));
    const int ga = grid_for(L, ceil_div(2 * n, kThreads));
    cudaError_t e;
#define CK(x) do { e = (x); if (e != cudaSuccess) return e; } while (0)
    long long *nhub = d.counters + 14;   // hub slots taken by First-CC
    const int32_t *hubidx = hubs ? d.hubidx : nullptr;
    CK(cudaMemsetAsync(d.lhead, 0xff, n * sizeof(int32_t), L.s));
    if (hubs) CK(cudaMemsetAsync(d.hubhead, 0xff, d.hub_cap * kHubSub * sizeof(int32_t), L.s));
    k_link<<<gv, kThreads, 0, L.s>>>(n, te_u, te_v, hubidx, d.lhead, d.hubhead, d.hub_cap, d.nxt,
                                     reinterpret_cast<const int32_t *>(d.counters + 5));
    L.mark("k_link");
    if (hubs) {
        k_hub_order<<<grid_for(L, ceil_div(d.hub_cap * 32, kThreads)), kThreads, 0, L.s>>>(
            nhub, d.hub_cap, d.hubvert, d.hubhead, d.hubnext, d.lhead);
        L.mark("k_hub_order");
    }
    long long *nr = d.counters + 1;
    CK(cudaMemsetAsync(nr, 0, sizeof(long long), L.s));
    k_succ_rulers<<<grid_for(L, ceil_div(n, kTile / 2)), kThreads, 0, L.s>>>(n, te_u, te_v, d.uf, d.lhead, d.nxt,
                                                                             hubidx, d.hubnext, ruler_stride,
                                                                             d.link, d.rhead, d.relem, nr);
    L.mark("k_succ_rulers");
    // upper bound on the number of rulers: a head per tour (a tour spans at least
    // two vertices) plus one per stride
    const int64_t rbound = n / 2 + ceil_div(2 * n, ruler_stride) + 1;
    // the walk's grid: one ruler per thread (up to 16 resident waves), so that the
    // block scheduler balances the long walks
    const int64_t gwant = ceil_div(ceil_div(rbound, kThreads), chase_chains);
    const int gr = (int)(gwant < 16ll * L.grid ? (gwant < 1 ? 1 : gwant) : 16ll * L.grid);
    if (chase_chains >= 4)
        k_chase<4><<<gr, kThreads, 0, L.s>>>(n, nr, d.relem, d.link, d.rnx1, d.rlen, d.err);
    else if (chase_chains == 2)
        k_chase<2><<<gr, kThreads, 0, L.s>>>(n, nr, d.relem, d.link, d.rnx1, d.rlen, d.err);
    else
        k_chase<1><<<gr, kThreads, 0, L.s>>>(n, nr, d.relem, d.link, d.rnx1, d.rlen, d.err);
    L.mark("k_chase");
    if (rank_variant == 1) {
        // Wyllie: pointer jumping over the level-1 ruler lists, a fixed number of
        // grid-wide rounds (enough for the longest possible list), double-buffered in
        // the level-2 arrays, which this variant leaves unused
        int32_t *nb[2] = {d.lv[0].owner, reinterpret_cast<int32_t *>(d.lv[0].l)};
        int32_t *vb[2] = {d.lv[0].offs, reinterpret_cast<int32_t *>(d.lv[0].l) + d.ruler_max};
        const int gj = grid_for(L, ceil_div(rbound, kThreads));
        const int rounds = jump_rounds(rbound);
        const int32_t *nx = d.rnx1, *vl = d.rlen;
        for (int i = 0; i < rounds; ++i) {
            int32_t *onx = nb[i & 1], *ovl = i + 1 == rounds ? d.sd1 : vb[i & 1];
            k_jump<<<gj, kThreads, 0, L.s>>>(nr, nx, vl, onx, ovl);
            L.mark("k_jump");
            nx = onx;
            vl = ovl;
        }
    } else {
    // Levels above the rulers: each samples the lists below again (heads of lists of
    // several nodes, at most the stride samples two levels down, plus one node in
    // kStride2); a third level is added when the second may exceed what one CTA
    // ranks in shared memory. The top level is ranked by k_top.
    int64_t bnd[kRankLevels + 1];
    bnd[0] = rbound;
    int64_t below2 = ceil_div(2 * n, ruler_stride);
    int levels = 0;
    for (int k = 0; k < kRankLevels; ++k) {
        bnd[k + 1] = below2 + ceil_div(bnd[k], kStride2) + 1;
        below2 = ceil_div(bnd[k], kStride2);
        ++levels;
        if (bnd[k + 1] <= kTopCap) break;
    }
    const long long *cnt[kRankLevels + 1];
    cnt[0] = nr;
    const int32_t *next_lo = d.rnx1, *w_lo = d.rlen;
    const uint8_t *head_lo = d.rhead;
    for (int k = 0; k < levels; ++k) {
        const RankLevel &v = d.lv[k];
        long long *c = d.counters + 11 + k;
        CK(cudaMemsetAsync(c, 0, sizeof(long long), L.s));
        k_lvl_rulers<<<grid_for(L, ceil_div(bnd[k], kThreads)), kThreads, 0, L.s>>>(
            cnt[k], kStride2, next_lo, head_lo, v.l, v.relem, v.head, c, v.cap, d.err);
        L.mark("k_lvl_rulers");
        k_lvl_chase<<<grid_for(L, ceil_div(bnd[k + 1], kThreads)), kThreads, 0, L.s>>>(
            cnt[k], c, v.relem, v.l, w_lo, v.owner, v.offs, v.next, v.w, d.err);
        L.mark("k_lvl_chase");
        cnt[k + 1] = c;
        next_lo = v.next;
        w_lo = v.w;
        head_lo = v.head;
    }
    const RankLevel &top = d.lv[levels - 1];
    k_top<<<1, kTopThreads, 2 * kTopCap * sizeof(int32_t), L.s>>>(cnt[levels], top.next, top.w, top.sd,
                                                                   d.top_tmp[0], d.top_tmp[1], d.top_tmp[2],
                                                                   d.top_tmp[3], d.top_tmp_cap, d.err);
    L.mark("k_top");
    for (int k = levels - 1; k >= 0; --k) {
        const RankLevel &v = d.lv[k];
        const int32_t *wl = k == 0 ? d.rlen : d.lv[k - 1].w;
        int32_t *sdl = k == 0 ? d.sd1 : d.lv[k - 1].sd;
        k_lvl_expand<<<grid_for(L, ceil_div(bnd[k], kThreads)), kThreads, 0, L.s>>>(cnt[k], v.l, wl, v.owner,
                                                                                    v.offs, v.sd, sdl);
        L.mark("k_lvl_expand");
    }
    }
    const int32_t *sd = d.sd1;
    long long *next_base = d.counters + 6;
    CK(cudaMemsetAsync(next_base, 0, sizeof(long long), L.s));
    k_comp_size<<<grid_for(L, ceil_div(n, kTile)), kThreads, 0, L.s>>>(n, d.uf, d.lhead, d.link, sd, nr, d.csize, d.vbase, next_base, d.rec,
                                          d.fp, d.lastp, d.ord, d.porig, d.w1, d.w2, d.err);
    L.mark("k_comp_size");
    CK(cudaGetLastError());
    k_place_records<<<gv, kThreads, 0, L.s>>>(n, te_u, te_v, te_a, hubs ? d.parc : nullptr, d.uf, d.csize, d.vbase, d.link, sd, d.rec, d.err);
    L.mark("k_place_records");
    CK(cudaGetLastError());
    const int64_t ntiles = ceil_div(2 * n, kTile);
    CK(cudaMemsetAsync(d.counters, 0, sizeof(long long), L.s));
    CK(cudaMemsetAsync(d.scan_status, 0, ntiles * sizeof(uint64_t), L.s));
    k_preorder<<<grid_for(L, ntiles), kThreads, 0, L.s>>>(2 * n, d.rec, d.fp, d.lastp, d.ord, d.porig, d.w1, d.w2,
                                                           d.counters, d.scan_status, d.err);
    L.mark("k_preorder");
#undef CK
    return cudaGetLastError();
}

template cudaError_t launch_rooting<int32_t>(const Dev &, const int32_t *, const int32_t *, int64_t, int64_t, int,
                                             int, int, int, bool, const Launch &);
template cudaError_t launch_rooting<int64_t>(const Dev &, const int64_t *, const int32_t *, int64_t, int64_t, int,
                                             int, int, int, bool, const Launch &);

}  // namespace fbcc
