/*
 * libfbcc: FAST-BCC biconnected components on one GPU (sm_103a), C ABI.
 *
 * The operation is the one the paper (Dong, Wang, Gu, Sun, "Provably Fast and
 * Space-Efficient Parallel Biconnectivity", PPoPP'23) states in Algorithm 1: given
 * an undirected graph G = (V, E), find its biconnected components (BCCs). The four
 * steps of Algorithm 1 (First-CC, Rooting, Tagging, Last-CC plus heads; section
 * 4.1) all run as CUDA kernels on the caller's stream. Where the paper outputs
 * vertex labels plus a head per label (section 3.4, "space-efficient BCC
 * representation"), this library expands them into the per-edge form below.
 *
 * Graph format (all calls): symmetric CSR. offsets has n+1 entries (int32 or
 * int64, chosen by `offsets_64`), offsets[0] = 0, offsets[n] = 2m; adj has 2m int32
 * vertex ids. Every undirected edge {u,v} appears as the two arcs u->v and v->u;
 * each adjacency list is sorted strictly ascending; no self-loops (a simple graph).
 * fbcc_validate checks this; the solvers assume it.
 *
 * Canonical output (identical, bit for bit, to the Hopcroft-Tarjan oracle):
 *  - edge id of {u,v}: the rank, in CSR order, of its arc with src < dst among all
 *    arcs with src < dst;
 *  - BCC k (k = 0 .. n_bcc-1) is the BCC with the k-th smallest smallest-edge-id;
 *  - edge_bcc[a]: the BCC index k of arc a (both arcs of an edge agree);
 *  - bcc_head[k]: the head of BCC k, its shallowest vertex when every connected
 *    component is rooted at its smallest vertex id (section 4.2);
 *  - is_ap[v] = 1 iff v is an articulation point; is_bridge[a] = 1 iff arc a's
 *    edge is a bridge (section 2: removal increases the number of components);
 *  - isolated vertices belong to no BCC and count as connected components.
 *
 * Memory: the caller owns every input and output buffer. Device buffers are
 * plain device pointers (e.g. from PyTorch). The library owns only the workspace,
 * allocated once by fbcc_workspace_create. `stream` is a cudaStream_t passed as
 * void* (NULL = the legacy default stream). Calls are asynchronous on the stream
 * unless stated; host-checked argument errors return immediately without
 * launching anything. No C++ exception crosses this interface.
 */
#ifndef FBCC_H
#define FBCC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    FBCC_OK = 0,
    FBCC_E_INVALID = 1,     /* bad argument: null pointer, negative size, offsets[n] != 2m, ... */
    FBCC_E_NOT_SIMPLE = 2,  /* fbcc_validate: self-loop, duplicate, unsorted or asymmetric CSR */
    FBCC_E_OOM = 3,         /* device memory for the workspace could not be allocated */
    FBCC_E_CUDA = 4,        /* a CUDA runtime call failed (message: fbcc_last_cuda_error) */
    FBCC_E_ITER_LIMIT = 5,  /* a bounded device loop hit its cap (reported in stats.device_status) */
    FBCC_E_WORKSPACE = 6    /* the graph exceeds the workspace's n_max / nnz_max */
} fbcc_status;

typedef struct fbcc_workspace fbcc_workspace; /* opaque; library-owned device memory */

/* Counts of one solve. device_status is 0 or an fbcc_status a kernel raised. */
typedef struct {
    int64_t n_bcc;     /* number of BCCs */
    int64_t n_ap;      /* number of articulation points */
    int64_t n_bridge;  /* number of bridges (undirected edges) */
    int64_t n_cc;      /* connected components, isolated vertices included */
    int32_t device_status;
    int32_t reserved;
} fbcc_stats;

/* Tuning knobs; zero in a field means "library default". */
typedef struct {
    int32_t ruler_stride;  /* list ranking: one ruler per this many tree arcs (power of 2, >= 8) */
    int32_t cc_sample;     /* First-CC: first neighbours per vertex hooked before the full pass (0 = off).
                              The full pass then goes by vertex and skips the largest sampled
                              component, or, when that component holds under half of a
                              degree-weighted vote, runs over all arcs as without sampling */
    int32_t grid_ctas;     /* CTAs of the persistent grid-stride kernels; -k = k per SM (default 8 per SM) */
    int32_t use_graph;     /* 1 = replay a captured CUDA graph for repeated identical calls (default), -1 = never */
    int32_t profile;       /* 1 = record a CUDA event after every kernel (no graph); see fbcc_profile_get */
    int32_t chase_chains;  /* list ranking: walks a thread advances together (1, 2 or 4) */
    int32_t cc_local;      /* First-CC: unite inside ranges of this many consecutive vertex ids in
                              shared memory first (power of 2, 1024..16384; 0 = off); a range
                              whose lists hold 2^31 arcs or more makes the solve report
                              FBCC_E_INVALID in device_status */
    int32_t lcc_sample;    /* Last-CC: first arcs per vertex (the tree arc to its parent not
                              counted) tested and united before the full pass (0 = off, 1..4);
                              the full pass then chooses as for cc_sample */
    int32_t rank_variant;  /* list ranking above the rulers: 0 = sample the ruler lists again and rank
                              the top level in one CTA (default); 1 = pointer jumping (Wyllie) over
                              the ruler lists, a fixed number of grid-wide rounds */
    int32_t cc_order;      /* rooting: 1 = renumber the spanning forest's edges component by component
                              before the Euler tours are built, so that each tour's arcs are
                              contiguous (0 = off) */
    int32_t hub_deg;       /* rooting and keys: vertices of at least this many arcs are hubs, whose
                              forest-arc lists are split to spread their atomic pushes, and the
                              forest records each tree edge's CSR position (which lets a hub head
                              name its BCC's key without searching its list); 0 = 256, -1 = off
                              (graphs without hubs), else >= 32 */
    int32_t cc_ldd;        /* First-CC by low-diameter decomposition, then union-find (section 5,
                              "Connectivity"): 0 = off, else 1/beta of the exponential shifts
                              (1..64; the decomposition takes ceil(cc_ldd * ln n) rounds, at most
                              63). cc_local takes precedence over it, it over cc_sample */
} fbcc_config;

/* Device bytes a workspace for graphs of up to n vertices and nnz arcs holds.
 * The workspace is the algorithm's auxiliary space, which section 4.3 (cost
 * bounds, the theorem's space part) bounds by O(n) beyond the input: every tag
 * and union-find array is per vertex; the per-arc part is one direction bit and
 * a 4-byte index per 256 arcs (about 132 bytes per vertex plus 0.14 per arc).
 * Used for admission by HBM footprint. No device call; never fails. */
size_t fbcc_workspace_bytes(int64_t n, int64_t nnz);

/* Allocate a workspace (one cudaMalloc of fbcc_workspace_bytes(n_max, nnz_max)
 * bytes, plus a private capture stream) for graphs with n <= n_max and
 * 2m <= nnz_max: the O(n) auxiliary space of section 4.3. The library owns it
 * until fbcc_workspace_destroy. Returns FBCC_OK and *ws, FBCC_E_INVALID for bad
 * sizes (n_max >= 2^30, nnz_max >= 2^40, negative, ws NULL), FBCC_E_OOM or
 * FBCC_E_CUDA (*ws is then NULL). */
fbcc_status fbcc_workspace_create(int64_t n_max, int64_t nnz_max, fbcc_workspace **ws);

/* A workspace carved from device memory the caller owns (for callers that pool
 * device memory themselves, e.g. a server admitting requests by HBM footprint):
 * `mem` (256-byte aligned) holds at least fbcc_batch_workspace_bytes(n_max,
 * nnz_max, max_graphs) bytes when max_graphs > 0 (fbcc_solve_batch of up to
 * max_graphs graphs), else fbcc_workspace_bytes(n_max, nnz_max). The library
 * allocates no device memory for it: fbcc_solve and fbcc_solve_batch run in
 * `mem`; fbcc_solve_host / _async, which need staging of their own, return
 * FBCC_E_INVALID on it, and fbcc_solve_batch returns FBCC_E_WORKSPACE for more
 * than max_graphs graphs. The memory must outlive the workspace and every solve
 * on it; fbcc_workspace_destroy releases only the library's host-side state and
 * does not synchronise. Returns FBCC_E_INVALID (NULL, unaligned or bad sizes) or
 * FBCC_E_WORKSPACE (bytes too small). Same O(n) auxiliary space as above. */
fbcc_status fbcc_workspace_create_in(void *mem, size_t bytes, int64_t n_max, int64_t nnz_max, int32_t max_graphs,
                                     fbcc_workspace **ws);

/* Release a workspace (synchronises the device first, unless it lives in caller
 * memory). NULL is ignored. */
void fbcc_workspace_destroy(fbcc_workspace *ws);

/* Set tuning knobs of a workspace (copied). NULL restores the defaults. */
fbcc_status fbcc_workspace_configure(fbcc_workspace *ws, const fbcc_config *cfg);

/*
 * Biconnected components of one graph (Algorithm 1), device-resident.
 *   csr_offsets  device, n+1 entries, int64 if offsets_64 else int32
 *   csr_adj      device, 2m int32 (format above)
 *   edge_bcc     device out, 2m int32: BCC index per arc
 *   bcc_head     device out, capacity >= max(n,1) int32: head of BCC k at [k]
 *   is_ap        device out, n uint8
 *   is_bridge    device out, 2m uint8
 *   stats        host out (may be NULL); written by an async copy on `stream`,
 *                valid after the stream is synchronised
 * Returns FBCC_OK once every kernel is enqueued; kernel-side failures appear in
 * stats->device_status. Calls on one workspace must not overlap on the device.
 */
fbcc_status fbcc_solve(const void *csr_offsets, int offsets_64, const int32_t *csr_adj,
                       int64_t n, int64_t m,
                       int32_t *edge_bcc, int32_t *bcc_head, uint8_t *is_ap, uint8_t *is_bridge,
                       fbcc_stats *stats, fbcc_workspace *ws, void *stream);

/*
 * The Tarjan-Vishkin foil (section 3.2; the skeleton's three rules are in the
 * appendix on Tarjan-Vishkin, its O(m) space in the appendix on its performance):
 * the same outputs as fbcc_solve, with Last-CC's implicit skeleton replaced by
 * Tarjan-Vishkin's explicit one. The skeleton has one vertex per edge of G, and a
 * list of up to m + n vertex pairs is materialised in `scratch` and united. The
 * forest, rooting and tags are FAST-BCC's, on `ws`; the labels it produces equal
 * Last-CC's, so every output equals fbcc_solve's.
 *   scratch        device, 256-byte aligned, at least fbcc_tv_scratch_bytes(n, 2m)
 *                  bytes (12 per arc and 16 per vertex: the O(m) auxiliary space
 *                  that FAST-BCC avoids), owned by the caller, untouched after the
 *                  stream is synchronised
 * The solve is enqueued with direct launches (no CUDA graph). Returns
 * FBCC_E_WORKSPACE when scratch is too small, FBCC_E_INVALID for n + 2m >= 2^31
 * (the skeleton's 32-bit vertex ids) or an unaligned scratch; otherwise as
 * fbcc_solve. Calls on one workspace must not overlap on the device.
 */
size_t fbcc_tv_scratch_bytes(int64_t n, int64_t nnz);
fbcc_status fbcc_solve_tv(const void *csr_offsets, int offsets_64, const int32_t *csr_adj,
                          int64_t n, int64_t m,
                          int32_t *edge_bcc, int32_t *bcc_head, uint8_t *is_ap, uint8_t *is_bridge,
                          fbcc_stats *stats, void *scratch, size_t scratch_bytes, fbcc_workspace *ws, void *stream);

/*
 * Same as fbcc_solve with every buffer in HOST memory (pinned memory makes the
 * copies asynchronous-capable). The inputs are copied into workspace-owned device
 * staging buffers, solved, and the outputs copied back; the call returns after the
 * stream has been synchronised, so stats is valid on return.
 */
fbcc_status fbcc_solve_host(const void *csr_offsets, int offsets_64, const int32_t *csr_adj,
                            int64_t n, int64_t m,
                            int32_t *edge_bcc, int32_t *bcc_head, uint8_t *is_ap, uint8_t *is_bridge,
                            fbcc_stats *stats, fbcc_workspace *ws, void *stream);

/*
 * fbcc_solve_host without waiting: the copies in, the solve and the copies out
 * are all enqueued on `stream` and the call returns at once. Every host buffer
 * must be page-locked (cudaHostAlloc / cudaHostRegister) and stay untouched until
 * the stream has been synchronised; stats (page-locked too, or NULL) is valid
 * then. bcc_head receives all n entries (those at n_bcc and beyond are left
 * unspecified), since n_bcc is not known when the copy is enqueued. Solves on
 * several workspaces, each with its own stream, overlap: one's copies run during
 * the others' kernels. Three in flight keep the GPU busy; with two, a workspace's
 * next input copy waits for its own output copy and the kernels idle meanwhile.
 * Calls on one workspace must not overlap (its staging buffers are reused).
 */
fbcc_status fbcc_solve_host_async(const void *csr_offsets, int offsets_64, const int32_t *csr_adj,
                                  int64_t n, int64_t m,
                                  int32_t *edge_bcc, int32_t *bcc_head, uint8_t *is_ap, uint8_t *is_bridge,
                                  fbcc_stats *stats, fbcc_workspace *ws, void *stream);

/*
 * Many independent graphs in one call. Section 4.1 (First-CC) observes that the
 * connected components of a graph are simply processed in parallel; a batch is
 * solved as the disjoint union of its graphs, whose components are exactly the
 * graphs' components, so every kernel launch covers all of them and each graph's
 * outputs equal those of fbcc_solve on that graph alone (numbered per graph).
 *   vtx_base   device, n_graphs+1 int64: graph g owns global vertices
 *              [vtx_base[g], vtx_base[g+1]); vtx_base[0] = 0, vtx_base[G] = n_total
 *   arc_base   device, n_graphs+1 int64: graph g owns arcs [arc_base[g], arc_base[g+1])
 *   local_off  device, n_total int32: for vertex i of graph g, the start of its list
 *              relative to arc_base[g] is local_off[vtx_base[g] + i] (its end is the
 *              next vertex's start, or arc_base[g+1] - arc_base[g] for the last vertex)
 *   local_adj  device, nnz_total int32 neighbour ids local to their graph
 *   outputs    at the same global positions as their inputs: edge_bcc / is_bridge per
 *              arc (BCC indices numbered within each graph), is_ap per vertex, and
 *              bcc_head[vtx_base[g] + k] = local head id of graph g's BCC k
 *   stats      device out, n_graphs fbcc_stats (device_status is set in every entry)
 *   host_vtx_base / host_arc_base  the same two arrays in host memory (sizes only)
 */
fbcc_status fbcc_solve_batch(int32_t n_graphs, const int64_t *vtx_base, const int64_t *arc_base,
                             const int64_t *host_vtx_base, const int64_t *host_arc_base,
                             const int32_t *local_off, const int32_t *local_adj,
                             int32_t *edge_bcc, int32_t *bcc_head, uint8_t *is_ap, uint8_t *is_bridge,
                             fbcc_stats *stats, fbcc_workspace *ws, void *stream);

/*
 * fbcc_solve for small graphs without allocating anything (the paper has no
 * counterpart: this serves callers that cannot call cudaMalloc, such as code
 * under an allocator or memory pool that forbids it, plugin hosts that own all
 * device memory, or paths that cannot afford an allocation's synchronisation).
 * The scratch is a fixed 12 MiB static device array inside the library, which
 * every GPU that loads the library holds until the process exits.
 *   Limits: n <= 32768 vertices and 2m <= 262144 arcs; larger graphs return
 *   FBCC_E_WORKSPACE without launching anything.
 *   Arguments: as fbcc_solve, except `stats_dev`, a DEVICE pointer to one
 *   fbcc_stats (or NULL) filled by a device-to-device copy on `stream`.
 *   Set-up: the first call on each device looks up that device's copy of the
 *   array (cudaGetSymbolAddress) with the device current; make that first call
 *   before any stream capture. The address is cached with the id of the context
 *   it came from: after a cudaDeviceReset the next call looks it up again.
 *   Sharing: all calls use the same array and every call re-initialises what it
 *   needs; calls that overlap on the GPU (other streams, other threads) race on
 *   it and must be serialised by the caller.
 */
fbcc_status fbcc_solve_noalloc(const void *csr_offsets, int offsets_64, const int32_t *csr_adj,
                               int64_t n, int64_t m,
                               int32_t *edge_bcc, int32_t *bcc_head, uint8_t *is_ap, uint8_t *is_bridge,
                               fbcc_stats *stats_dev, void *stream);

/*
 * Biconnectivity queries over the last solve on `ws` (section 3.4, the
 * space-efficient BCC representation: a label per vertex plus one head per label;
 * a label's BCC is its class plus its head, section 4.2). They read the
 * workspace's labels, parents, label ranks and head counts, which stay valid
 * until the next solve on the same workspace, and answer in the canonical BCC
 * numbering of that solve's outputs (for a batch: the vertex ids are global,
 * vtx_base[g] + local id, and the BCC indices are those of the vertex's graph).
 * The first query after a solve also enqueues a per-head index of the labels
 * (two O(n) passes). All arrays are device memory, owned by the caller; the calls
 * are asynchronous on `stream` (order them after the solve, e.g. the same
 * stream). Returns FBCC_E_INVALID when no solve has run on ws or for a NULL array
 * with q > 0; vertex ids outside [0, n) are answered as having no BCC.
 *
 * fbcc_query_biconnected: bcc[i] = the BCC index that u[i] and v[i] share, or -1
 *   when they share none (also for u[i] == v[i]); two BCCs share at most one
 *   vertex, so the answer is unique.
 */
fbcc_status fbcc_query_biconnected(fbcc_workspace *ws, const int32_t *u, const int32_t *v, int64_t q,
                                   int32_t *bcc, void *stream);

/*
 * fbcc_query_bcc_count: out_off[i] = the number of BCCs holding the vertices
 *   v[0..i) (exclusive prefix, q+1 entries, int64), out_off[q] = the total; an
 *   isolated vertex is in none, an articulation point in several. q <= 2 n_max
 *   (else FBCC_E_WORKSPACE).
 * fbcc_query_bccs_of: with out_off from fbcc_query_bcc_count on the same v, writes
 *   the BCC indices of v[i] to out[out_off[i] .. out_off[i+1]) (out holds
 *   out_off[q] entries): first the BCC of v[i]'s own label (when v[i] is not a
 *   component root), then those of the labels v[i] heads, in no fixed order.
 */
fbcc_status fbcc_query_bcc_count(fbcc_workspace *ws, const int32_t *v, int64_t q, int64_t *out_off, void *stream);
fbcc_status fbcc_query_bccs_of(fbcc_workspace *ws, const int32_t *v, int64_t q, const int64_t *out_off,
                               int32_t *out, void *stream);

/* Device bytes fbcc_solve_batch needs beyond the inputs and outputs (for admission). */
size_t fbcc_batch_workspace_bytes(int64_t n_total, int64_t nnz_total, int32_t n_graphs);

/*
 * Check the graph format on the device: ids in range, lists sorted strictly
 * ascending, no self-loops, every arc has its reverse, offsets monotone with
 * offsets[n] = 2m. Section 2 (preliminaries) states the problem on an undirected
 * graph G = (V, E) with edges x--y and is silent on self-loops and parallel
 * edges; this library reads the input as a simple graph (the solvers recognise
 * the tree arc to a parent by its endpoint, which needs simplicity), and this call
 * is the check of that reading. Synchronous on `stream`. Returns FBCC_OK,
 * FBCC_E_INVALID (bad sizes, pointers, offsets or ids) or FBCC_E_NOT_SIMPLE.
 */
fbcc_status fbcc_validate(const void *csr_offsets, int offsets_64, const int32_t *csr_adj,
                          int64_t n, int64_t m, fbcc_workspace *ws, void *stream);

/* Number of kernels timed in the last solve made with fbcc_config.profile = 1. */
int32_t fbcc_profile_count(const fbcc_workspace *ws);

/* Name and device time (ms, from CUDA events on the solve's stream) of timed
 * kernel i of the last profiled solve; waits for that solve to finish. */
fbcc_status fbcc_profile_get(const fbcc_workspace *ws, int32_t i, const char **name, float *ms);

/*
 * Copy the named internal per-vertex array of the workspace's last solve into
 * host memory (synchronous; for tests of the intermediate phases). Names and
 * element types (int32 unless stated), all of length n:
 *   "first", "last", "parent"  preorder number, last preorder number in the
 *                              subtree, tree parent (-1 for a root), by vertex
 *   "label"                    Last-CC label by vertex (a root is its own label)
 *   "w1", "w2"                 w1/w2 by preorder number; w2 may also hold the
 *                              preorder numbers of tree children (they leave
 *                              high unchanged), w1 is exactly its definition
 *   "low", "high"              low/high by preorder number (only when the solve
 *                              ran with fbcc_config.profile = 1)
 *   "ord", "porig"             vertex and parent vertex (-1: root) by preorder number
 *   "vbits" (uint8)            bit 0: the tree edge to the parent is a bridge;
 *                              bit 1: it is a fence edge
 *   "err" (count 1)            the device error bits of the last solve
 *   "sampled" (count up to 4)  the sampling votes of the last solves that sampled:
 *                              First-CC's largest root and whether it won at least
 *                              half of the votes (1) or the tiled pass ran (0), then
 *                              the same two for Last-CC (a plain-component root by
 *                              preorder number, -1 when no arc voted); after an LDD
 *                              First-CC the second value is 1 when its list of edges
 *                              between clusters held them all, 0 when the full hook
 *                              pass ran
 *   "dirb" (uint8, count up to ceil(nnz_max / 8))  one bit per arc, least
 *                              significant first: the target's preorder number
 *                              exceeds the source's
 * Returns FBCC_E_INVALID for an unknown name or a count above those limits
 * (n_max for the per-vertex arrays).
 */
fbcc_status fbcc_debug_read(const fbcc_workspace *ws, const char *name, void *host_dst, int64_t count);

/* Static description of a status code. */
const char *fbcc_status_string(fbcc_status s);

/* Text of the last CUDA error this thread saw inside the library ("" if none). */
const char *fbcc_last_cuda_error(void);

#ifdef __cplusplus
}
#endif

#endif /* FBCC_H */
