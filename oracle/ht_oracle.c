/*
 * Hopcroft-Tarjan biconnected components: the ORACLE.
 *
 * TEST INFRASTRUCTURE ONLY. The test suite, the smoke check and the CPU-baseline
 * leg of the benchmark load this file; the GPU library never calls it and shares no
 * code, header or table with it.
 *
 * It is a plain, slow, single-threaded restatement of what the paper defines:
 *
 *  - Articulation point / bridge (section 2, "Notation"): a vertex / an edge whose
 *    removal increases the number of connected components.
 *  - Hopcroft-Tarjan (section 3.1): a DFS tree T; first[v] is v's preorder number;
 *    w1[u] = min({first[u]} U {first[u'] : (u,u') a non-tree edge});
 *    low[v] = min of w1 over the subtree T_v. When the DFS returns from child c to
 *    u and low[c] >= first[u], the edges pushed on the edge stack since the tree
 *    edge u-c (inclusive) form one biconnected component (BCC), and u separates it.
 *  - BCC head (section 4.2): the unique shallowest vertex of a BCC in the spanning
 *    tree. Each connected component's DFS is rooted at its smallest vertex id, so
 *    the vertex u above is that head. A non-root head is an articulation point; the
 *    root is one iff it heads two or more BCCs (section 4.2, head/AP lemma).
 *  - A bridge is a BCC with exactly one edge (it lies on no cycle, so removing it
 *    disconnects its endpoints).
 *
 * Canonical numbering (the output contract shared with the GPU library):
 *  - The edge id of an undirected edge {u,v} is the rank, in CSR order, of its arc
 *    with src < dst among all arcs with src < dst.
 *  - BCCs are numbered k = 0 .. n_bcc-1 in increasing order of their smallest edge id.
 *  - edge_bcc[a] = k for both arcs of every edge; bcc_head[k] = head of BCC k;
 *    is_bridge[a] = 1 on both arcs of a bridge; is_ap[v] = 1 for articulation points.
 *  - Isolated vertices belong to no BCC and are counted as connected components.
 *
 * Input contract: symmetric CSR with int64 offsets (n+1) and int32 adjacency
 * (offsets[n] = 2m arcs); every adjacency list sorted strictly ascending (so no
 * duplicate edges), no self-loops. Return 0 on success, 1 for a malformed CSR
 * (offsets or ids out of range), 2 for a graph that is not simple or not symmetric,
 * 3 when host memory runs out.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* Index of the arc from -> to (binary search in from's sorted list), or -1. */
static int64_t find_arc(const int64_t *off, const int32_t *adj, int32_t from, int32_t to)
{
    int64_t lo = off[from], hi = off[from + 1];
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (adj[mid] < to) lo = mid + 1; else hi = mid;
    }
    return (lo < off[from + 1] && adj[lo] == to) ? lo : -1;
}

int fbcc_oracle_check_csr(int64_t n, int64_t m, const int64_t *off, const int32_t *adj)
{
    if (n < 0 || m < 0) return 1;
    if (off[0] != 0 || off[n] != 2 * m) return 1;
    for (int64_t v = 0; v < n; v++)
        if (off[v + 1] < off[v]) return 1;
    for (int64_t a = 0; a < 2 * m; a++)
        if (adj[a] < 0 || (int64_t)adj[a] >= n) return 1;
    for (int64_t v = 0; v < n; v++) {
        for (int64_t a = off[v]; a < off[v + 1]; a++) {
            if (adj[a] == v) return 2;                                /* self-loop */
            if (a > off[v] && adj[a] <= adj[a - 1]) return 2;         /* unsorted or duplicate */
            if (find_arc(off, adj, adj[a], (int32_t)v) < 0) return 2; /* missing twin */
        }
    }
    return 0;
}

typedef struct { int64_t key; int32_t blk; } keyed_block;

static int cmp_keyed(const void *x, const void *y)
{
    const keyed_block *a = (const keyed_block *)x, *b = (const keyed_block *)y;
    return (a->key > b->key) - (a->key < b->key);
}

int fbcc_oracle_solve(int64_t n, int64_t m, const int64_t *off, const int32_t *adj,
                      int32_t *edge_bcc, int32_t *bcc_head, uint8_t *is_ap,
                      uint8_t *is_bridge, int64_t *stats /* n_bcc, n_ap, n_bridge, n_cc */)
{
    int rc = fbcc_oracle_check_csr(n, m, off, adj);
    if (rc) return rc;
    const int64_t nnz = 2 * m;
    int64_t nn = n > 0 ? n : 1, mm = m > 0 ? m : 1, zz = nnz > 0 ? nnz : 1;

    int32_t *first = malloc(nn * sizeof(int32_t));     /* preorder number, -1 = unvisited */
    int32_t *low = malloc(nn * sizeof(int32_t));
    int32_t *parent = malloc(nn * sizeof(int32_t));    /* DFS-tree parent, -1 for a root */
    int64_t *tree_arc = malloc(nn * sizeof(int64_t));  /* arc parent -> v */
    int64_t *cursor = malloc(nn * sizeof(int64_t));    /* next arc to scan */
    uint8_t *skipped = malloc(nn);                     /* parent arc already skipped once */
    int32_t *vstack = malloc(nn * sizeof(int32_t));
    int64_t *estack = malloc(mm * sizeof(int64_t));    /* arcs, one per undirected edge */
    int32_t *esrc = malloc(mm * sizeof(int32_t));      /* their source vertices */
    int32_t *blk_of = malloc(zz * sizeof(int32_t));    /* block of an edge, at its src<dst arc */
    int32_t *head = malloc(nn * sizeof(int32_t));      /* head of block b (#blocks <= n-1) */
    int64_t *nedge = malloc(nn * sizeof(int64_t));     /* edges in block b */
    if (!first || !low || !parent || !tree_arc || !cursor || !skipped || !vstack || !estack ||
        !esrc || !blk_of || !head || !nedge) {
        rc = 3;
        goto done;
    }
    for (int64_t v = 0; v < n; v++) { first[v] = -1; is_ap[v] = 0; }

    int32_t t = 0, nblk = 0;
    int64_t etop = 0, n_cc = 0;
    for (int32_t s = 0; s < n; s++) {
        if (first[s] != -1) continue;
        n_cc++;
        first[s] = low[s] = t++;
        if (off[s] == off[s + 1]) continue; /* isolated vertex: in no BCC */
        parent[s] = -1;
        cursor[s] = off[s];
        skipped[s] = 0;
        int64_t vtop = 0;
        vstack[vtop++] = s;
        int root_blocks = 0;
        while (vtop > 0) {
            int32_t u = vstack[vtop - 1];
            if (cursor[u] < off[u + 1]) {
                int64_t a = cursor[u]++;
                int32_t w = adj[a];
                if (w == parent[u] && !skipped[u]) { skipped[u] = 1; continue; }
                if (first[w] == -1) {                 /* tree edge u -> w: descend */
                    estack[etop] = a; esrc[etop] = u; etop++;
                    parent[w] = u; tree_arc[w] = a; skipped[w] = 0;
                    first[w] = low[w] = t++;
                    cursor[w] = off[w];
                    vstack[vtop++] = w;
                } else if (first[w] < first[u]) {     /* back edge to an ancestor */
                    estack[etop] = a; esrc[etop] = u; etop++;
                    if (first[w] < low[u]) low[u] = first[w];
                }
                /* first[w] > first[u]: a finished descendant; pushed from w's side */
            } else {
                vtop--;
                if (parent[u] == -1) continue;        /* the root is done */
                int32_t p = parent[u];
                if (low[u] < low[p]) low[p] = low[u];
                if (low[u] >= first[p]) {             /* p separates T_u: pop one BCC */
                    int32_t b = nblk++;
                    head[b] = p;
                    nedge[b] = 0;
                    int64_t e;
                    do {
                        etop--;
                        e = estack[etop];
                        int32_t x = esrc[etop], y = adj[e];
                        int64_t key_arc = x < y ? e : find_arc(off, adj, y, x);
                        blk_of[key_arc] = b;
                        nedge[b]++;
                    } while (e != tree_arc[u]);
                    if (parent[p] == -1) root_blocks++; else is_ap[p] = 1;
                }
            }
        }
        if (root_blocks >= 2) is_ap[s] = 1;
    }

    /* Smallest edge id of every block: scan arcs with src < dst in CSR order. */
    keyed_block *kb = malloc((nblk > 0 ? nblk : 1) * sizeof(keyed_block));
    int32_t *rank = malloc((nblk > 0 ? nblk : 1) * sizeof(int32_t));
    if (!kb || !rank) { free(kb); free(rank); rc = 3; goto done; }
    for (int32_t b = 0; b < nblk; b++) { kb[b].key = INT64_MAX; kb[b].blk = b; }
    int64_t eid = 0;
    for (int64_t u = 0; u < n; u++)
        for (int64_t a = off[u]; a < off[u + 1]; a++)
            if (u < adj[a]) {
                int32_t b = blk_of[a];
                if (eid < kb[b].key) kb[b].key = eid;
                eid++;
            }
    qsort(kb, nblk, sizeof(keyed_block), cmp_keyed);
    for (int32_t k = 0; k < nblk; k++) rank[kb[k].blk] = k;

    int64_t n_bridge = 0, n_ap = 0;
    for (int32_t b = 0; b < nblk; b++) {
        bcc_head[rank[b]] = head[b];
        if (nedge[b] == 1) n_bridge++;
    }
    for (int64_t u = 0; u < n; u++) {
        n_ap += is_ap[u];
        for (int64_t a = off[u]; a < off[u + 1]; a++) {
            int32_t v = adj[a];
            int64_t key_arc = u < v ? a : find_arc(off, adj, v, (int32_t)u);
            int32_t b = blk_of[key_arc];
            edge_bcc[a] = rank[b];
            is_bridge[a] = nedge[b] == 1;
        }
    }
    stats[0] = nblk;
    stats[1] = n_ap;
    stats[2] = n_bridge;
    stats[3] = n_cc;
    free(kb);
    free(rank);

done:
    free(first); free(low); free(parent); free(tree_arc); free(cursor); free(skipped);
    free(vstack); free(estack); free(esrc); free(blk_of); free(head); free(nedge);
    return rc;
}
