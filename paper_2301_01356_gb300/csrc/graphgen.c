/*
 * Seeded synthetic graph generators (host C, OpenMP).
 *
 * These make the inputs only: they contain none of the biconnectivity method's
 * arithmetic and are shared, as plain CSR arrays, by the oracle and the GPU path.
 *
 * Randomness: every draw is a pure function of (seed, stream, counter), the
 * SplitMix64 output function of Steele, Lea and Flood ("Fast splittable
 * pseudorandom number generators", OOPSLA 2014) applied to a counter, so results
 * do not depend on the number of threads.
 *
 * Output CSR: symmetric, every list sorted ascending, no self-loops, no duplicates,
 * int64 offsets (n+1) and int32 adjacency. Results are malloc'ed and returned in a
 * gg_csr; release them with gg_free.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    int64_t n, nnz;
    int64_t *off;
    int32_t *adj;
    int64_t truth_bcc, truth_ap; /* ground truth where the family fixes it, else -1 */
} gg_csr;

static inline uint64_t sm64(uint64_t z)
{
    z += 0x9e3779b97f4a7c15ULL;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

/* 64 random bits for draw i of a (seed, stream) sequence. */
static inline uint64_t rnd(uint64_t seed, uint64_t stream, uint64_t i)
{
    return sm64(sm64(seed * 0x9e3779b97f4a7c15ULL + stream) ^ sm64(i));
}

static inline double unif(uint64_t seed, uint64_t stream, uint64_t i)
{
    return (double)(rnd(seed, stream, i) >> 11) * 0x1.0p-53;
}

static inline uint64_t below(uint64_t seed, uint64_t stream, uint64_t i, uint64_t bound)
{
    /* multiply-shift mapping of 64 random bits to [0, bound) */
    return (uint64_t)(((unsigned __int128)rnd(seed, stream, i) * bound) >> 64);
}

void gg_free(void *p) { free(p); }

static int cmp_i32(const void *a, const void *b)
{
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

static void sort_i32(int32_t *a, int64_t len)
{
    if (len < 32) {
        for (int64_t i = 1; i < len; i++) {
            int32_t x = a[i];
            int64_t j = i - 1;
            while (j >= 0 && a[j] > x) { a[j + 1] = a[j]; j--; }
            a[j + 1] = x;
        }
    } else {
        qsort(a, (size_t)len, sizeof(int32_t), cmp_i32);
    }
}

/*
 * Symmetric simple CSR from an undirected edge list (u[i], v[i]). Self-loops and
 * repeated edges are dropped. Returns 0, or 3 when memory runs out.
 */
int gg_build_csr(int64_t n, int64_t ne, const int32_t *u, const int32_t *v, gg_csr *out)
{
    memset(out, 0, sizeof(*out));
    out->truth_bcc = out->truth_ap = -1;
    int64_t *deg = calloc((size_t)n + 1, sizeof(int64_t));
    int64_t *off = malloc(((size_t)n + 1) * sizeof(int64_t));
    if (!deg || !off) { free(deg); free(off); return 3; }
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < ne; i++) {
        if (u[i] == v[i]) continue;
#pragma omp atomic
        deg[u[i]]++;
#pragma omp atomic
        deg[v[i]]++;
    }
    off[0] = 0;
    for (int64_t x = 0; x < n; x++) off[x + 1] = off[x] + deg[x];
    int64_t tot = off[n];
    int32_t *raw = malloc((size_t)(tot > 0 ? tot : 1) * sizeof(int32_t));
    if (!raw) { free(deg); free(off); return 3; }
    memcpy(deg, off, (size_t)n * sizeof(int64_t)); /* deg[] becomes a fill cursor */
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < ne; i++) {
        if (u[i] == v[i]) continue;
        int64_t p, q;
#pragma omp atomic capture
        p = deg[u[i]]++;
#pragma omp atomic capture
        q = deg[v[i]]++;
        raw[p] = v[i];
        raw[q] = u[i];
    }
    /* sort and deduplicate each list in place; deg[x] = its new length */
#pragma omp parallel for schedule(dynamic, 1024)
    for (int64_t x = 0; x < n; x++) {
        int32_t *l = raw + off[x];
        int64_t len = off[x + 1] - off[x], k = 0;
        sort_i32(l, len);
        for (int64_t i = 0; i < len; i++)
            if (k == 0 || l[i] != l[k - 1]) l[k++] = l[i];
        deg[x] = k;
    }
    int64_t *noff = malloc(((size_t)n + 1) * sizeof(int64_t));
    if (!noff) { free(deg); free(off); free(raw); return 3; }
    noff[0] = 0;
    for (int64_t x = 0; x < n; x++) noff[x + 1] = noff[x] + deg[x];
    int32_t *adj = malloc((size_t)(noff[n] > 0 ? noff[n] : 1) * sizeof(int32_t));
    if (!adj) { free(deg); free(off); free(raw); free(noff); return 3; }
#pragma omp parallel for schedule(dynamic, 1024)
    for (int64_t x = 0; x < n; x++)
        memcpy(adj + noff[x], raw + off[x], (size_t)deg[x] * sizeof(int32_t));
    free(deg);
    free(off);
    free(raw);
    out->n = n;
    out->nnz = noff[n];
    out->off = noff;
    out->adj = adj;
    return 0;
}

/* ---- uniform random: m distinct edges u != v, drawn uniformly ------------------ */

typedef struct { uint64_t *keys; uint64_t mask; } hset;

static int hset_init(hset *h, int64_t cap)
{
    uint64_t sz = 16;
    while (sz < (uint64_t)cap * 2) sz <<= 1;
    h->keys = malloc(sz * sizeof(uint64_t));
    if (!h->keys) return 3;
    memset(h->keys, 0xff, sz * sizeof(uint64_t));
    h->mask = sz - 1;
    return 0;
}

/* insert; returns 1 if the key was new */
static int hset_add(hset *h, uint64_t key)
{
    uint64_t i = sm64(key) & h->mask;
    while (h->keys[i] != UINT64_MAX) {
        if (h->keys[i] == key) return 0;
        i = (i + 1) & h->mask;
    }
    h->keys[i] = key;
    return 1;
}

static inline uint64_t ekey(int64_t a, int64_t b)
{
    return a < b ? ((uint64_t)a << 32) | (uint64_t)b : ((uint64_t)b << 32) | (uint64_t)a;
}

/* Candidate pairs are taken in counter order and kept if not a self-loop and new. */
int gg_uniform(int64_t n, int64_t m, uint64_t seed, gg_csr *out)
{
    memset(out, 0, sizeof(*out));
    if (n < 2 && m > 0) return 1;
    if (m > n * (n - 1) / 2) return 1;
    int32_t *u = malloc((size_t)(m > 0 ? m : 1) * sizeof(int32_t));
    int32_t *v = malloc((size_t)(m > 0 ? m : 1) * sizeof(int32_t));
    hset h;
    if (!u || !v || hset_init(&h, m + 1)) { free(u); free(v); return 3; }
    int64_t k = 0;
    for (uint64_t i = 0; k < m; i++) {
        int64_t a = (int64_t)below(seed, 11, 2 * i, (uint64_t)n);
        int64_t b = (int64_t)below(seed, 11, 2 * i + 1, (uint64_t)n);
        if (a == b || !hset_add(&h, ekey(a, b))) continue;
        u[k] = (int32_t)a;
        v[k] = (int32_t)b;
        k++;
    }
    free(h.keys);
    int rc = gg_build_csr(n, m, u, v, out);
    free(u);
    free(v);
    return rc;
}

/* ---- thinned 2-D grid plus short-range extra edges ----------------------------- */

/*
 * R x C grid, vertex id r*C + c, open boundary (torus != 0 wraps rows and columns).
 * Each grid edge is kept independently with probability p. Then
 * round(extra_frac * kept) extra edges are added: a uniform vertex plus a uniform
 * offset (dr, dc) with 1 <= |dr| + |dc| <= max_l1, in bounds, not already present.
 */
int gg_grid(int64_t R, int64_t C, int torus, double p, double extra_frac, int64_t max_l1,
            uint64_t seed, gg_csr *out)
{
    memset(out, 0, sizeof(*out));
    int64_t n = R * C;
    int64_t nh = torus ? R * C : R * (C - 1);   /* horizontal edges */
    int64_t nv = torus ? R * C : (R - 1) * C;   /* vertical edges */
    if (torus && (R < 3 || C < 3)) return 1;
    if (torus && extra_frac > 0) return 1; /* extra edges are defined on the open grid */
    int64_t ng = nh + nv;
    uint8_t *keep = malloc((size_t)(ng > 0 ? ng : 1));
    if (!keep) return 3;
    int64_t kept = 0;
#pragma omp parallel for reduction(+ : kept) schedule(static)
    for (int64_t e = 0; e < ng; e++) {
        keep[e] = p >= 1.0 || unif(seed, 21, (uint64_t)e) < p;
        kept += keep[e];
    }
    int64_t nextra = (int64_t)llround(extra_frac * (double)kept);
    int32_t *u = malloc((size_t)(kept + nextra + 1) * sizeof(int32_t));
    int32_t *v = malloc((size_t)(kept + nextra + 1) * sizeof(int32_t));
    if (!u || !v) { free(keep); free(u); free(v); return 3; }
    int64_t k = 0;
    for (int64_t e = 0; e < ng; e++) {
        if (!keep[e]) continue;
        int64_t a, b;
        if (e < nh) {
            int64_t r = e / (torus ? C : C - 1), c = e % (torus ? C : C - 1);
            a = r * C + c;
            b = r * C + (c + 1) % C;
        } else {
            int64_t f = e - nh, r = f / C, c = f % C;
            a = r * C + c;
            b = ((r + 1) % R) * C + c;
        }
        u[k] = (int32_t)a;
        v[k] = (int32_t)b;
        k++;
    }
    if (nextra > 0) {
        /* offsets with 1 <= |dr|+|dc| <= max_l1, in a fixed order */
        int64_t no = 2 * max_l1 * (max_l1 + 1);
        int32_t *odr = malloc((size_t)no * sizeof(int32_t)), *odc = malloc((size_t)no * sizeof(int32_t));
        hset h;
        if (!odr || !odc || hset_init(&h, nextra + 1)) {
            free(keep); free(u); free(v); free(odr); free(odc); return 3;
        }
        int64_t q = 0;
        for (int64_t dr = -max_l1; dr <= max_l1; dr++)
            for (int64_t dc = -max_l1; dc <= max_l1; dc++) {
                int64_t l1 = (dr < 0 ? -dr : dr) + (dc < 0 ? -dc : dc);
                if (l1 >= 1 && l1 <= max_l1) { odr[q] = (int32_t)dr; odc[q] = (int32_t)dc; q++; }
            }
        int64_t added = 0;
        for (uint64_t i = 0; added < nextra; i++) {
            int64_t a = (int64_t)below(seed, 22, 2 * i, (uint64_t)n);
            int64_t o = (int64_t)below(seed, 22, 2 * i + 1, (uint64_t)no);
            int64_t r = a / C + odr[o], c = a % C + odc[o];
            if (r < 0 || r >= R || c < 0 || c >= C) continue;
            int64_t b = r * C + c;
            int64_t l1 = (odr[o] < 0 ? -odr[o] : odr[o]) + (odc[o] < 0 ? -odc[o] : odc[o]);
            if (l1 == 1) { /* a grid neighbour: skip if that grid edge was kept */
                int64_t lo = a < b ? a : b, hi = a < b ? b : a, e;
                if (hi - lo == 1) e = (lo / C) * (C - 1) + lo % C;
                else e = nh + lo;
                if (keep[e]) continue;
            }
            if (!hset_add(&h, ekey(a, b))) continue;
            u[k] = (int32_t)a;
            v[k] = (int32_t)b;
            k++;
            added++;
        }
        free(h.keys);
        free(odr);
        free(odc);
    }
    free(keep);
    int rc = gg_build_csr(n, k, u, v, out);
    free(u);
    free(v);
    return rc;
}

/* ---- R-MAT ----------------------------------------------------------------------- */

/*
 * ne = edge_factor * 2^scale directed draws; each descends `scale` levels of the
 * adjacency matrix choosing quadrant (0,0), (0,1), (1,0), (1,1) with probability
 * a, b, c, 1-a-b-c (most significant bit first). No noise, no vertex permutation.
 * The draws are symmetrised; self-loops and duplicates are dropped; isolated
 * vertices stay.
 */
int gg_rmat(int scale, int64_t edge_factor, double a, double b, double c, uint64_t seed,
            gg_csr *out)
{
    memset(out, 0, sizeof(*out));
    int64_t n = (int64_t)1 << scale, ne = edge_factor * n;
    int32_t *u = malloc((size_t)ne * sizeof(int32_t)), *v = malloc((size_t)ne * sizeof(int32_t));
    if (!u || !v) { free(u); free(v); return 3; }
    double ab = a + b, abc = a + b + c;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < ne; i++) {
        int64_t x = 0, y = 0;
        for (int l = 0; l < scale; l++) {
            double r = unif(seed, 31, (uint64_t)i * (uint64_t)scale + (uint64_t)l);
            int bx = r >= ab, by = (r >= a && r < ab) || r >= abc;
            x = (x << 1) | bx;
            y = (y << 1) | by;
        }
        u[i] = (int32_t)x;
        v[i] = (int32_t)y;
    }
    int rc = gg_build_csr(n, ne, u, v, out);
    free(u);
    free(v);
    return rc;
}

/* ---- chain of cycles with pendant trees ------------------------------------------ */

/*
 * k cycles (k >= 1) with lengths drawn uniformly from [lmin, lmax] and capped so the
 * chain fits in n vertices; cycle i+1 shares exactly one vertex with cycle i (a vertex
 * of cycle i other than the one it shares with cycle i-1). Every remaining vertex is
 * attached by one edge to a uniformly chosen earlier vertex (random pendant trees).
 * Ground truth: #BCC = (cycles) + (pendant vertices); the articulation points are the
 * shared vertices plus every vertex with a pendant child.
 */
int gg_cycle_chain(int64_t n, int64_t k, int64_t lmin, int64_t lmax, uint64_t seed, gg_csr *out)
{
    memset(out, 0, sizeof(*out));
    if (k < 1 || lmin < 3 || lmax < lmin || n < 3) return 1;
    int32_t *u = malloc((size_t)(2 * n + 8) * sizeof(int32_t));
    int32_t *v = malloc((size_t)(2 * n + 8) * sizeof(int32_t));
    uint8_t *ap = calloc((size_t)n, 1);
    if (!u || !v || !ap) { free(u); free(v); free(ap); return 3; }
    /* start/len_prev: the fresh ids of the previous cycle, from which the next
       shared vertex is drawn (this excludes the vertex it shares with its own
       predecessor, which is not fresh) */
    int64_t used = 0, ne = 0, cycles = 0, start = 0, len_prev = 0;
    uint64_t ctr = 0;
    for (int64_t i = 0; i < k && used < n; i++) {
        int64_t L = lmin + (int64_t)below(seed, 41, ctr++, (uint64_t)(lmax - lmin + 1));
        int64_t fresh = i == 0 ? L : L - 1;
        if (used + fresh > n) fresh = n - used;
        if ((i == 0 && fresh < 3) || (i > 0 && fresh < 2)) break;
        int64_t join = -1;
        if (i > 0) {
            join = start + (int64_t)below(seed, 42, ctr++, (uint64_t)len_prev);
            ap[join] = 1;
        }
        int64_t first_new = used;
        int64_t s0 = join >= 0 ? join : first_new, prevv = s0;
        for (int64_t j = (join >= 0 ? 0 : 1); j < fresh; j++) {
            int64_t w = first_new + j;
            u[ne] = (int32_t)prevv; v[ne] = (int32_t)w; ne++;
            prevv = w;
        }
        u[ne] = (int32_t)prevv; v[ne] = (int32_t)s0; ne++;
        used += fresh;
        cycles++;
        start = first_new;
        len_prev = fresh;
    }
    int64_t pendants = 0;
    for (int64_t w = used; w < n; w++) {
        int64_t p = (int64_t)below(seed, 43, (uint64_t)w, (uint64_t)w);
        u[ne] = (int32_t)p; v[ne] = (int32_t)w; ne++;
        ap[p] = 1;
        pendants++;
    }
    int rc = gg_build_csr(n, ne, u, v, out);
    if (!rc) {
        int64_t nap = 0;
        for (int64_t w = 0; w < n; w++) nap += ap[w];
        out->truth_bcc = cycles + pendants;
        out->truth_ap = nap;
    }
    free(u);
    free(v);
    free(ap);
    return rc;
}

/* ---- k nearest neighbours of uniform points in the unit cube --------------------- */

/*
 * n points uniform in [0,1)^3; each point is joined to its k nearest other points
 * (Euclidean; ties broken by smaller id), then the edges are symmetrised. Uses a
 * uniform bucket grid with about 2 points per cell and an expanding shell search.
 */
int gg_knn3(int64_t n, int64_t k, uint64_t seed, gg_csr *out)
{
    memset(out, 0, sizeof(*out));
    if (n < 2 || k < 1 || k >= n) return 1;
    float *px = malloc((size_t)n * 3 * sizeof(float));
    int64_t g = (int64_t)cbrt((double)n / 2.0);
    if (g < 1) g = 1;
    int64_t ncell = g * g * g;
    int64_t *cstart = calloc((size_t)ncell + 1, sizeof(int64_t));
    int32_t *cidx = malloc((size_t)n * sizeof(int32_t));
    int64_t *cell = malloc((size_t)n * sizeof(int64_t));
    int32_t *eu = malloc((size_t)(n * k) * sizeof(int32_t)), *ev = malloc((size_t)(n * k) * sizeof(int32_t));
    if (!px || !cstart || !cidx || !cell || !eu || !ev) {
        free(px); free(cstart); free(cidx); free(cell); free(eu); free(ev); return 3;
    }
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; i++) {
        for (int d = 0; d < 3; d++) px[3 * i + d] = (float)unif(seed, 51, (uint64_t)(3 * i + d));
        int64_t cx = (int64_t)(px[3 * i] * g), cy = (int64_t)(px[3 * i + 1] * g), cz = (int64_t)(px[3 * i + 2] * g);
        if (cx >= g) cx = g - 1;
        if (cy >= g) cy = g - 1;
        if (cz >= g) cz = g - 1;
        cell[i] = (cx * g + cy) * g + cz;
    }
    for (int64_t i = 0; i < n; i++) cstart[cell[i] + 1]++;
    for (int64_t c = 0; c < ncell; c++) cstart[c + 1] += cstart[c];
    {
        int64_t *cur = malloc((size_t)ncell * sizeof(int64_t));
        if (!cur) { free(px); free(cstart); free(cidx); free(cell); free(eu); free(ev); return 3; }
        memcpy(cur, cstart, (size_t)ncell * sizeof(int64_t));
        for (int64_t i = 0; i < n; i++) cidx[cur[cell[i]]++] = (int32_t)i;
        free(cur);
    }
    int fail = 0;
#pragma omp parallel
    {
        float *bd = malloc((size_t)k * sizeof(float));
        int32_t *bi = malloc((size_t)k * sizeof(int32_t));
        if (!bd || !bi) {
#pragma omp atomic write
            fail = 1;
        }
#pragma omp for schedule(dynamic, 256)
        for (int64_t i = 0; i < n; i++) {
            if (!bd || !bi) continue;
            int64_t cnt = 0;
            float x = px[3 * i], y = px[3 * i + 1], z = px[3 * i + 2];
            int64_t cx = cell[i] / (g * g), cy = (cell[i] / g) % g, cz = cell[i] % g;
            for (int64_t r = 0;; r++) {
                /* visit the shell of cells at Chebyshev distance r */
                for (int64_t ax = cx - r; ax <= cx + r; ax++) {
                    if (ax < 0 || ax >= g) continue;
                    for (int64_t ay = cy - r; ay <= cy + r; ay++) {
                        if (ay < 0 || ay >= g) continue;
                        for (int64_t az = cz - r; az <= cz + r; az++) {
                            if (az < 0 || az >= g) continue;
                            int64_t dx = ax - cx, dy = ay - cy, dz = az - cz;
                            int64_t ch = dx < 0 ? -dx : dx;
                            if ((dy < 0 ? -dy : dy) > ch) ch = dy < 0 ? -dy : dy;
                            if ((dz < 0 ? -dz : dz) > ch) ch = dz < 0 ? -dz : dz;
                            if (ch != r) continue;
                            int64_t c = (ax * g + ay) * g + az;
                            for (int64_t t = cstart[c]; t < cstart[c + 1]; t++) {
                                int32_t j = cidx[t];
                                if (j == i) continue;
                                float ddx = px[3 * j] - x, ddy = px[3 * j + 1] - y, ddz = px[3 * j + 2] - z;
                                float d2 = ddx * ddx + ddy * ddy + ddz * ddz;
                                /* insert into the sorted top-k by (distance, id) */
                                if (cnt == k && (d2 > bd[k - 1] || (d2 == bd[k - 1] && j > bi[k - 1]))) continue;
                                int64_t pos = cnt < k ? cnt : k - 1;
                                while (pos > 0 && (bd[pos - 1] > d2 || (bd[pos - 1] == d2 && bi[pos - 1] > j))) {
                                    bd[pos] = bd[pos - 1];
                                    bi[pos] = bi[pos - 1];
                                    pos--;
                                }
                                bd[pos] = d2;
                                bi[pos] = j;
                                if (cnt < k) cnt++;
                            }
                        }
                    }
                }
                /* every unvisited point is at least r/g away along some axis */
                float reach = (float)r / (float)g;
                if ((cnt == k && bd[k - 1] <= reach * reach) || r > g) break;
            }
            for (int64_t q = 0; q < k; q++) {
                eu[i * k + q] = (int32_t)i;
                ev[i * k + q] = bi[q];
            }
        }
        free(bd);
        free(bi);
    }
    free(px);
    free(cstart);
    free(cidx);
    free(cell);
    int rc = fail ? 3 : gg_build_csr(n, n * k, eu, ev, out);
    free(eu);
    free(ev);
    return rc;
}

/* ---- packed batches of many graphs ------------------------------------------------ */

typedef struct {
    int64_t G;
    int64_t *vtx_base, *arc_base;   /* G+1 each */
    int32_t *loff;                  /* n_total: list starts relative to the graph's arc base */
    int32_t *ladj;                  /* nnz_total: local neighbour ids */
    int32_t *family;                /* G: 0 uniform, 1 grid, 2 cycle chain, 3 k-NN */
    int64_t *truth_bcc, *truth_ap;  /* G: ground truth where the family fixes it, else -1 */
} gg_batch;

/*
 * G graphs, vertex counts log-uniform on [nmin, nmax], families taken round-robin from
 * the `fam_mask` bits (bit f = family f):
 *   0 uniform random, average degree uniform on [4, 12];
 *   1 thinned open grid floor(sqrt(n)) x ceil(n / floor(sqrt(n))), p uniform on [0.55, 0.75];
 *   2 chain of k (2..64) cycles of lengths 3..5000, pendant trees for the rest;
 *   3 k-NN (k = 5) of uniform points in the unit cube.
 * Graph g uses seed `seed * 1000003 + g`. Returns 0, 1 for bad arguments, 3 on OOM.
 */
int gg_batch_make(int64_t G, uint64_t seed, int64_t nmin, int64_t nmax, int fam_mask, gg_batch *out)
{
    memset(out, 0, sizeof(*out));
    if (G < 1 || nmin < 3 || nmax < nmin || !(fam_mask & 15)) return 1;
    int fams[4], nf = 0;
    for (int f = 0; f < 4; f++)
        if (fam_mask >> f & 1) fams[nf++] = f;
    int64_t *ns = malloc((size_t)G * sizeof(int64_t));
    gg_csr *gs = calloc((size_t)G, sizeof(gg_csr));
    int *fam = malloc((size_t)G * sizeof(int));
    if (!ns || !gs || !fam) { free(ns); free(gs); free(fam); return 3; }
    double lmin = log((double)nmin), lmax = log((double)nmax);
    for (int64_t g = 0; g < G; g++) {
        double x = lmin + (lmax - lmin) * unif(seed, 61, (uint64_t)g);
        int64_t n = (int64_t)llround(exp(x));
        ns[g] = n < nmin ? nmin : (n > nmax ? nmax : n);
        fam[g] = fams[g % nf];
    }
    int fail = 0;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t g = 0; g < G; g++) {
        uint64_t sg = seed * 1000003ULL + (uint64_t)g;
        int64_t n = ns[g];
        int rc = 0;
        switch (fam[g]) {
        case 0: {
            double d = 4.0 + 8.0 * unif(sg, 71, 0);
            int64_t m = (int64_t)llround(n * d / 2);
            if (m > n * (n - 1) / 2) m = n * (n - 1) / 2;
            rc = gg_uniform(n, m, sg, &gs[g]);
            break;
        }
        case 1: {
            int64_t R = (int64_t)floor(sqrt((double)n));
            if (R < 2) R = 2;
            int64_t C = (n + R - 1) / R;
            if (C < 2) C = 2;
            double p = 0.55 + 0.20 * unif(sg, 72, 0);
            rc = gg_grid(R, C, 0, p, 0.0, 1, sg, &gs[g]);
            break;
        }
        case 2: {
            int64_t k = 2 + (int64_t)below(sg, 73, 0, 63);
            rc = gg_cycle_chain(n, k, 3, 5000, sg, &gs[g]);
            break;
        }
        default:
            rc = gg_knn3(n, 5, sg, &gs[g]);
        }
        if (rc) {
#pragma omp atomic write
            fail = rc;
        }
    }
    if (fail) {
        for (int64_t g = 0; g < G; g++) { free(gs[g].off); free(gs[g].adj); }
        free(ns); free(gs); free(fam);
        return fail;
    }
    out->G = G;
    out->vtx_base = malloc((size_t)(G + 1) * sizeof(int64_t));
    out->arc_base = malloc((size_t)(G + 1) * sizeof(int64_t));
    out->family = malloc((size_t)G * sizeof(int32_t));
    out->truth_bcc = malloc((size_t)G * sizeof(int64_t));
    out->truth_ap = malloc((size_t)G * sizeof(int64_t));
    if (!out->vtx_base || !out->arc_base || !out->family || !out->truth_bcc || !out->truth_ap) fail = 3;
    if (!fail) {
        out->vtx_base[0] = out->arc_base[0] = 0;
        for (int64_t g = 0; g < G; g++) {
            out->vtx_base[g + 1] = out->vtx_base[g] + gs[g].n;
            out->arc_base[g + 1] = out->arc_base[g] + gs[g].nnz;
            out->family[g] = fam[g];
            out->truth_bcc[g] = gs[g].truth_bcc;
            out->truth_ap[g] = gs[g].truth_ap;
        }
        out->loff = malloc((size_t)(out->vtx_base[G] > 0 ? out->vtx_base[G] : 1) * sizeof(int32_t));
        out->ladj = malloc((size_t)(out->arc_base[G] > 0 ? out->arc_base[G] : 1) * sizeof(int32_t));
        if (!out->loff || !out->ladj) fail = 3;
    }
    if (!fail) {
#pragma omp parallel for schedule(dynamic, 1)
        for (int64_t g = 0; g < G; g++) {
            int32_t *lo = out->loff + out->vtx_base[g];
            for (int64_t v = 0; v < gs[g].n; v++) lo[v] = (int32_t)gs[g].off[v];
            memcpy(out->ladj + out->arc_base[g], gs[g].adj, (size_t)gs[g].nnz * sizeof(int32_t));
        }
    }
    for (int64_t g = 0; g < G; g++) { free(gs[g].off); free(gs[g].adj); }
    free(ns); free(gs); free(fam);
    if (fail) {
        free(out->vtx_base); free(out->arc_base); free(out->family); free(out->truth_bcc); free(out->truth_ap);
        free(out->loff); free(out->ladj);
        memset(out, 0, sizeof(*out));
    }
    return fail;
}
