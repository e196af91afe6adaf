/*
 * CPU oracle for all pairs of geodesic distances on a grey image.
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product path may link, load or
 * call this file: only the tests, the smoke check and the benchmark's CPU
 * baseline use it. It shares no code, header, table or helper with the CUDA
 * library.
 *
 * It is written to be read against Noyel, Angulo & Jeulin, "Fast computation
 * of all pairs of geodesic distances":
 *   - the image graph (Sec. 2, eqs. "voisinage 1/2"): pixels are vertices,
 *     4- or 8-neighbours are edges, a pixel is not its own neighbour;
 *   - the path time and geodesic distance (Sec. 2, eqs. "temps",
 *     "distance"): the infimum over paths of the summed edge weights;
 *   - the sum-of-grey-levels pseudo-metric (Sec. 2, eq. "distance somme"),
 *     taken here as w(p,q) = f(p) + f(q) + 1 so that every edge costs at
 *     least 1; the obstacle-mask variant uses w = 2 between free pixels;
 *   - Property 1 (Sec. 2): along a geodesic path d(pi,pj) = d(p0,pj) -
 *     d(p0,pi), applied to every ancestor of every vertex of the geodesic
 *     tree (Sec. 2, "geodesic tree");
 *   - the marks D_mrk, the per-point filling rate and "filled" (Sec. 2, eqs.
 *     "a", "filling rate pt");
 *   - the source orders of Sec. 3: naive, spiral (Algorithm "spiral
 *     method"), and minimum filling rate (Algorithm "method based on the
 *     filling rate") with its geodesic-extrema pre-pass (Sec. 3.3).
 *
 * The distance array is the plain definition: a textbook binary-heap
 * Dijkstra from every source. The orders are simulated step by step, in the
 * paper's order of operations, with no blocking, fusion or reordering.
 *
 * Parity status of each function is stated beside it.
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_UNREACH 0xFFFFFFFFu
#define OR_UNSET 0xFFFFFFFEu /* "not written yet" marker for the simulated array */

/* ------------------------------------------------------------------------ */
/* Image graph (Sec. 2, eqs. "voisinage 1/2" and the 4/8-neighbourhoods).    */
/* ------------------------------------------------------------------------ */

typedef struct {
    const uint8_t *f;    /* grey values, H*W, row-major; for kind 3, nch planes of H*W */
    const uint8_t *mask; /* 1 = free pixel; NULL means every pixel is free */
    int H, W, conn, kind; /* kind 0 = sum of grey levels, 1 = mask (w = 2), 2 = L1,
                             3 = sum over the channels of a multichannel image */
    int nch;              /* channels (kind 3) */
} or_graph;

/* The exported functions take the kind as a code: 0, 1, 2, or 3 | (L << 8)
 * for a multichannel image of L channels (Sec. 2: values in T^L), whose f
 * then holds the L planes one after the other. */
static or_graph or_make(const uint8_t *f, const uint8_t *mask, int H, int W, int conn, int code) {
    or_graph g = {f, mask, H, W, conn, code & 0xFF, code >> 8};
    return g;
}

static int or_code(const or_graph *g) { return g->kind | (g->nch << 8); }

static int or_free(const or_graph *g, int p) {
    return g->kind != 1 || g->mask == NULL || g->mask[p] != 0;
}

/* Neighbours of p in increasing linear index. Only free neighbours of a free
 * pixel are edges. Returns the count. */
static int or_neighbours(const or_graph *g, int p, int *out) {
    static const int d8r[8] = {-1, -1, -1, 0, 0, 1, 1, 1};
    static const int d8c[8] = {-1, 0, 1, -1, 1, -1, 0, 1};
    static const int d4r[4] = {-1, 0, 0, 1};
    static const int d4c[4] = {0, -1, 1, 0};
    int r = p / g->W, c = p % g->W, n = 0;
    if (!or_free(g, p)) return 0;
    int k, K = g->conn == 8 ? 8 : 4;
    for (k = 0; k < K; k++) {
        int rr = r + (K == 8 ? d8r[k] : d4r[k]);
        int cc = c + (K == 8 ? d8c[k] : d4c[k]);
        if (rr < 0 || rr >= g->H || cc < 0 || cc >= g->W) continue;
        int q = rr * g->W + cc;
        if (!or_free(g, q)) continue;
        out[n++] = q;
    }
    return n;
}

/* Edge weight: sum of grey levels plus one (Sec. 2, eq. "distance somme",
 * with +1), 2 between free pixels of a mask, the absolute difference of
 * grey levels plus one (Sec. 2, pseudo-metric L1, eq. "distance abs
 * difference", with +1 so that every edge costs at least 1), or, for a
 * multichannel image (Sec. 2, values in T^L), the sum pseudo-metric added
 * over its channels plus one. Parity status of the channel sum: pinned by
 * brute force, Floyd-Warshall, the one-channel case, constant channels and
 * the 1 x W closed form. */
static uint32_t or_weight(const or_graph *g, int p, int q) {
    if (g->kind == 1) return 2u;
    if (g->kind == 3) {
        /* the sum pseudo-metric summed over the channels, plus one */
        size_t N = (size_t)g->H * g->W;
        uint32_t w = 1u;
        for (int l = 0; l < g->nch; l++) w += (uint32_t)g->f[l * N + p] + (uint32_t)g->f[l * N + q];
        return w;
    }
    if (g->kind == 2) return (uint32_t)(g->f[p] > g->f[q] ? g->f[p] - g->f[q] : g->f[q] - g->f[p]) + 1u;
    return (uint32_t)g->f[p] + (uint32_t)g->f[q] + 1u;
}

/* ------------------------------------------------------------------------ */
/* Dijkstra with a binary heap (the geodesic distance of Sec. 2, eq.        */
/* "distance", as the infimum of path times).                                */
/* ------------------------------------------------------------------------ */

typedef struct { uint32_t d; int v; } or_item;

typedef struct { or_item *a; int n, cap; } or_heap;

static void or_heap_push(or_heap *h, uint32_t d, int v) {
    if (h->n == h->cap) {
        h->cap = h->cap ? 2 * h->cap : 1024;
        h->a = (or_item *)realloc(h->a, (size_t)h->cap * sizeof(or_item));
    }
    int i = h->n++;
    while (i > 0) {
        int par = (i - 1) / 2;
        if (h->a[par].d <= d) break;
        h->a[i] = h->a[par];
        i = par;
    }
    h->a[i].d = d;
    h->a[i].v = v;
}

static or_item or_heap_pop(or_heap *h) {
    or_item top = h->a[0], last = h->a[--h->n];
    int i = 0;
    for (;;) {
        int l = 2 * i + 1, r = l + 1, m = i;
        uint32_t dm = last.d;
        if (l < h->n && h->a[l].d < dm) { m = l; dm = h->a[l].d; }
        if (r < h->n && h->a[r].d < dm) { m = r; }
        if (m == i) break;
        h->a[i] = h->a[m];
        i = m;
    }
    if (h->n > 0) h->a[i] = last;
    return top;
}

/* Multi-source Dijkstra: every source starts at 0. dist has H*W entries;
 * unreached vertices keep OR_UNREACH. */
static void or_dijkstra(const or_graph *g, const int *src, int nsrc, uint32_t *dist) {
    int N = g->H * g->W, nb[8];
    or_heap h = {0};
    for (int p = 0; p < N; p++) dist[p] = OR_UNREACH;
    for (int i = 0; i < nsrc; i++) {
        if (!or_free(g, src[i])) continue;
        dist[src[i]] = 0;
        or_heap_push(&h, 0, src[i]);
    }
    while (h.n > 0) {
        or_item it = or_heap_pop(&h);
        if (it.d != dist[it.v]) continue; /* stale entry */
        int k = or_neighbours(g, it.v, nb);
        for (int j = 0; j < k; j++) {
            uint32_t nd = it.d + or_weight(g, it.v, nb[j]);
            if (nd < dist[nb[j]]) {
                dist[nb[j]] = nd;
                or_heap_push(&h, nd, nb[j]);
            }
        }
    }
    free(h.a);
}

/* Single-source geodesic distance row d(s, .). An obstacle source reaches
 * only itself. Parity: pinned by Floyd-Warshall, brute-force path
 * enumeration, the 1-D closed form and the constant-image closed forms. */
void or_sssp(const uint8_t *f, const uint8_t *mask, int H, int W, int conn, int kind,
             int s, uint32_t *row) {
    or_graph g = or_make(f, mask, H, W, conn, kind);
    if (!or_free(&g, s)) {
        for (int p = 0; p < H * W; p++) row[p] = OR_UNREACH;
        row[s] = 0;
        return;
    }
    or_dijkstra(&g, &s, 1, row);
}

/* Multi-source distance (used by the geodesic-extrema pre-pass). */
void or_msssp(const uint8_t *f, const uint8_t *mask, int H, int W, int conn, int kind,
              const int32_t *src, int nsrc, uint32_t *row) {
    or_graph g = or_make(f, mask, H, W, conn, kind);
    or_dijkstra(&g, (const int *)src, nsrc, row);
}

typedef struct {
    const or_graph *g;
    uint32_t *D;
    const int32_t *rows; /* which sources; NULL = all */
    int nrows, t, T;
} or_apsp_job;

static void *or_apsp_worker(void *arg) {
    or_apsp_job *j = (or_apsp_job *)arg;
    int N = j->g->H * j->g->W;
    for (int i = j->t; i < j->nrows; i += j->T) {
        int s = j->rows ? j->rows[i] : i;
        or_sssp(j->g->f, j->g->mask, j->g->H, j->g->W, j->g->conn, or_code(j->g), s,
                j->D + (size_t)i * N);
    }
    return NULL;
}

/* Rows d(s, .) for a list of sources (all sources when src == NULL, giving
 * the full N x N array), spread over nthreads host threads. The naive
 * method of Sec. 1: one propagation per source. */
void or_rows(const uint8_t *f, const uint8_t *mask, int H, int W, int conn, int kind,
             const int32_t *src, int nsrc, uint32_t *out, int nthreads) {
    or_graph g = or_make(f, mask, H, W, conn, kind);
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    pthread_t th[256];
    or_apsp_job jobs[256];
    int n = src ? nsrc : H * W;
    for (int t = 0; t < nthreads; t++) {
        jobs[t].g = &g; jobs[t].D = out; jobs[t].rows = src; jobs[t].nrows = n;
        jobs[t].t = t; jobs[t].T = nthreads;
        pthread_create(&th[t], NULL, or_apsp_worker, &jobs[t]);
    }
    for (int t = 0; t < nthreads; t++) pthread_join(th[t], NULL);
}

/* Floyd-Warshall over the same graph, for tiny images only (N <= 256). An
 * independent route to the same array. */
void or_floyd(const uint8_t *f, const uint8_t *mask, int H, int W, int conn, int kind,
              uint32_t *D) {
    or_graph g = or_make(f, mask, H, W, conn, kind);
    int N = H * W, nb[8];
    uint64_t *M = (uint64_t *)malloc((size_t)N * N * sizeof(uint64_t));
    const uint64_t INF = (uint64_t)1 << 62;
    for (int i = 0; i < N; i++)
        for (int j = 0; j < N; j++) M[(size_t)i * N + j] = (i == j) ? 0 : INF;
    for (int p = 0; p < N; p++) {
        int k = or_neighbours(&g, p, nb);
        for (int j = 0; j < k; j++) M[(size_t)p * N + nb[j]] = or_weight(&g, p, nb[j]);
    }
    for (int k = 0; k < N; k++)
        for (int i = 0; i < N; i++)
            for (int j = 0; j < N; j++) {
                uint64_t c = M[(size_t)i * N + k] + M[(size_t)k * N + j];
                if (c < M[(size_t)i * N + j]) M[(size_t)i * N + j] = c;
            }
    for (size_t i = 0; i < (size_t)N * N; i++) D[i] = M[i] >= INF ? OR_UNREACH : (uint32_t)M[i];
    free(M);
}

/* ------------------------------------------------------------------------ */
/* Geodesic tree (Sec. 2, "geodesic tree": root, nodes, leaves).              */
/* The paper leaves the choice of tree open; the canonical tree here gives   */
/* every reached vertex b != s the smallest-index neighbour q that is tight: */
/* d(s,q) + w(q,b) == d(s,b).                                                 */
/* ------------------------------------------------------------------------ */

void or_parents(const uint8_t *f, const uint8_t *mask, int H, int W, int conn, int kind,
                const uint32_t *drow, int s, int32_t *parent) {
    or_graph g = or_make(f, mask, H, W, conn, kind);
    int N = H * W, nb[8];
    for (int b = 0; b < N; b++) {
        parent[b] = -1;
        if (b == s || drow[b] == OR_UNREACH) continue;
        int k = or_neighbours(&g, b, nb); /* increasing index */
        for (int j = 0; j < k; j++) {
            int q = nb[j];
            if (drow[q] == OR_UNREACH) continue;
            if ((uint64_t)drow[q] + or_weight(&g, q, b) == (uint64_t)drow[b]) {
                parent[b] = q;
                break;
            }
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Connected components of free pixels (used for the mask variant: pairs in  */
/* different components are unreachable and count as filled from the start; */
/* the paper assumes a connected image and is silent here).                  */
/* ------------------------------------------------------------------------ */

static int or_components(const or_graph *g, int *comp, int *size /* N */) {
    int N = g->H * g->W, ncomp = 0, nb[8];
    int *stack = (int *)malloc((size_t)N * sizeof(int));
    for (int p = 0; p < N; p++) comp[p] = -1;
    for (int p = 0; p < N; p++) {
        if (!or_free(g, p) || comp[p] >= 0) continue;
        int top = 0, cnt = 0;
        stack[top++] = p;
        comp[p] = ncomp;
        while (top > 0) {
            int v = stack[--top];
            cnt++;
            int k = or_neighbours(g, v, nb);
            for (int j = 0; j < k; j++)
                if (comp[nb[j]] < 0) { comp[nb[j]] = ncomp; stack[top++] = nb[j]; }
        }
        size[ncomp++] = cnt;
    }
    free(stack);
    return ncomp;
}

/* ------------------------------------------------------------------------ */
/* Spiral order (Sec. 3.1, Algorithm "spiral method"): concentric one-pixel  */
/* frames, outermost first; within a frame a uniform random unfilled pixel.  */
/* The random draws come from SplitMix64 (Steele, Lea & Flood, OOPSLA 2014), */
/* one stream per frame, driving a Fisher-Yates shuffle of the frame.         */
/* ------------------------------------------------------------------------ */

static uint64_t or_splitmix64(uint64_t *state) {
    uint64_t z = (*state += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* Fills seq with the free pixels, frame by frame, each frame shuffled.
 * Returns the count. */
int or_spiral_sequence(const uint8_t *mask, int kind, int H, int W, uint64_t seed,
                       int32_t *seq) {
    int nframes = ((H < W ? H : W) + 1) / 2, n = 0;
    for (int k = 0; k < nframes; k++) {
        int start = n;
        for (int p = 0; p < H * W; p++) {
            int r = p / W, c = p % W;
            int m = r;
            if (c < m) m = c;
            if (H - 1 - r < m) m = H - 1 - r;
            if (W - 1 - c < m) m = W - 1 - c;
            if (m != k) continue;
            if (kind == 1 && mask && !mask[p]) continue;
            seq[n++] = p;
        }
        uint64_t st = seed ^ ((uint64_t)k * 0x9E3779B97F4A7C15ull);
        int len = n - start;
        for (int i = len - 1; i >= 1; i--) {
            int j = (int)(or_splitmix64(&st) % (uint64_t)(i + 1));
            int32_t t = seq[start + i];
            seq[start + i] = seq[start + j];
            seq[start + j] = t;
        }
    }
    return n;
}

/* ------------------------------------------------------------------------ */
/* Geodesic extrema (Sec. 3.3): a propagation from the image edges gives the */
/* geodesic centroid c (a farthest point from the edges); a propagation from */
/* c gives the list Ext of pixels by decreasing distance from c. On a mask,  */
/* the "edges" are the boundary vertices of the general-graph extension      */
/* (Sec. 5): free pixels with fewer free neighbours than the connectivity;   */
/* each component gets its own centroid. Ties: smallest index first.         */
/* rank[p] = position of p in Ext (0 = greatest extremum).                   */
/* ------------------------------------------------------------------------ */

static const uint32_t *or_sort_key;
static int or_rank_cmp(const void *a, const void *b) {
    int p = *(const int *)a, q = *(const int *)b;
    uint32_t gp = or_sort_key[p], gq = or_sort_key[q];
    if (gp != gq) return gp > gq ? -1 : 1; /* decreasing distance */
    return p < q ? -1 : (p > q ? 1 : 0);
}

/* Outputs: e (distance from the boundary), gdist (distance from the
 * centroids), centroids (per component, capacity N), rank. Returns the
 * number of components. */
int or_extrema(const uint8_t *f, const uint8_t *mask, int H, int W, int conn, int kind,
               uint32_t *e, uint32_t *gdist, int32_t *centroids, int32_t *rank) {
    or_graph g = or_make(f, mask, H, W, conn, kind);
    int N = H * W, nb[8];
    int *comp = (int *)malloc((size_t)N * sizeof(int));
    int *csize = (int *)malloc((size_t)N * sizeof(int));
    int32_t *bd = (int32_t *)calloc((size_t)N, sizeof(int32_t));
    int ncomp = or_components(&g, comp, csize), nb_count = 0;
    for (int p = 0; p < N; p++)
        if (or_free(&g, p) && or_neighbours(&g, p, nb) < conn) bd[nb_count++] = p;
    or_dijkstra(&g, bd, nb_count, e);
    for (int c = 0; c < ncomp; c++) centroids[c] = -1;
    for (int p = 0; p < N; p++) {
        if (comp[p] < 0) continue;
        int c = comp[p];
        if (centroids[c] < 0 || e[p] > e[centroids[c]]) centroids[c] = p;
    }
    or_dijkstra(&g, centroids, ncomp, gdist);
    int *order = (int *)malloc((size_t)N * sizeof(int));
    int nfree = 0;
    for (int p = 0; p < N; p++)
        if (or_free(&g, p)) order[nfree++] = p;
    or_sort_key = gdist;
    qsort(order, (size_t)nfree, sizeof(int), or_rank_cmp);
    for (int p = 0; p < N; p++) rank[p] = -1;
    for (int i = 0; i < nfree; i++) rank[order[i]] = i;
    free(order); free(bd); free(csize); free(comp);
    return ncomp;
}

/* ------------------------------------------------------------------------ */
/* The method: fill D from geodesic trees, choosing sources by an order.     */
/*                                                                            */
/* Marks D_mrk and the per-point count cnt (Sec. 2, eqs. "a" and "filling    */
/* rate pt": tau(x) = (cnt(x) - 1)/(N - 1), filled <=> cnt == N). A round     */
/* picks B sources from the state at the start of the round (B = 1 is the    */
/* paper's loop), then for each source, in selection order, computes the      */
/* geodesic tree and fills every (ancestor, vertex) pair by Property 1.       */
/* ------------------------------------------------------------------------ */

enum { OR_NAIVE = 0, OR_SPIRAL = 1, OR_MINFILL = 2, OR_EXTREMA = 3, OR_REPULSION = 4 };

/* Spiral turns as rings (Sec. 3.2, Algorithm "spiral method with
 * repulsion"): frame k = {min(r, c, H-1-r, W-1-c) = k}, its free pixels in
 * clockwise order from (k, k). A frame with at least two rows and two
 * columns is a closed ring; a single row or column is an open line. Fills
 * ring (all frames in turn), fstart[k] .. fstart[k+1] and fcyc[k]; returns
 * the number of frames. */
int or_rings(const uint8_t *mask, int kind, int H, int W, int32_t *ring, int32_t *fstart,
             uint8_t *fcyc) {
    int nframes = ((H < W ? H : W) + 1) / 2, n = 0;
    for (int k = 0; k < nframes; k++) {
        int r0 = k, r1 = H - 1 - k, c0 = k, c1 = W - 1 - k;
        fstart[k] = n;
        fcyc[k] = (uint8_t)(r1 > r0 && c1 > c0);
#define OR_PUSH(rr, cc)                                            \
    do {                                                           \
        int p_ = (rr) * W + (cc);                                  \
        if (!(kind == 1 && mask && !mask[p_])) ring[n++] = p_;     \
    } while (0)
        for (int c = c0; c <= c1; c++) OR_PUSH(r0, c);
        if (r1 > r0) {
            for (int r = r0 + 1; r <= r1; r++) OR_PUSH(r, c1);
            if (c1 > c0) {
                for (int c = c1 - 1; c >= c0; c--) OR_PUSH(r1, c);
                for (int r = r1 - 1; r > r0; r--) OR_PUSH(r, c0);
            }
        }
#undef OR_PUSH
    }
    fstart[nframes] = n;
    return nframes;
}

/* stats[0] propagations, [1] pre-pass propagations, [2] distance operations
 * (sum over propagations of the depth of every reached vertex), [3] new
 * pairs, [4] rounds, [5] pairs filled before the first round (different
 * components), [6] number of components.
 *
 * seq_out (capacity N) receives the sources in selection order;
 * round_new (capacity N) the new pairs of each round; D_out (N*N, may be
 * NULL) the array filled by the method itself. Returns 0, or -1 if the loop
 * did not end within N rounds (cannot happen: a source's own row is filled
 * by its propagation). */
int or_fill(const uint8_t *f, const uint8_t *mask, int H, int W, int conn, int kind,
            int order, int B, uint64_t seed, uint64_t *stats, int32_t *seq_out,
            uint64_t *round_new, uint32_t *D_out) {
    or_graph g = or_make(f, mask, H, W, conn, kind);
    int N = H * W;
    size_t words = ((size_t)N * N + 63) / 64;
    uint64_t *mrk = (uint64_t *)calloc(words, sizeof(uint64_t));
    uint32_t *cnt = (uint32_t *)malloc((size_t)N * sizeof(uint32_t));
    int *comp = (int *)malloc((size_t)N * sizeof(int));
    int *csize = (int *)malloc((size_t)N * sizeof(int));
    uint32_t *d = (uint32_t *)malloc((size_t)N * sizeof(uint32_t));
    int32_t *parent = (int32_t *)malloc((size_t)N * sizeof(int32_t));
    int32_t *seq = (int32_t *)malloc((size_t)N * sizeof(int32_t));
    int32_t *rank = (int32_t *)malloc((size_t)N * sizeof(int32_t));
    uint32_t *gcen = (uint32_t *)malloc((size_t)N * sizeof(uint32_t));
    int32_t *S = (int32_t *)malloc((size_t)(B > 0 ? B : 1) * sizeof(int32_t));
    uint8_t *taken = (uint8_t *)calloc((size_t)N, 1);
    /* repulsion order: rings, the current frame and its list S of ring
     * positions (inS), and one SplitMix64 stream for the draws */
    int32_t *ring = (int32_t *)malloc((size_t)N * sizeof(int32_t));
    int32_t *fstart = (int32_t *)malloc((size_t)(N + 2) * sizeof(int32_t));
    uint8_t *fcyc = (uint8_t *)malloc((size_t)(N + 1));
    uint8_t *inS = (uint8_t *)calloc((size_t)N, 1);
    int nframes = 0, cur = -1;
    uint64_t rst = seed;
    for (int i = 0; i < 8; i++) stats[i] = 0;

    int ncomp = or_components(&g, comp, csize);
    stats[6] = (uint64_t)ncomp;

    /* Initial marks: the diagonal (D_mrk(i,i) = 1), and every pair that no
     * path joins (obstacles, different components), which is known and
     * filled with "unreachable" before any propagation. */
    uint64_t pre = 0;
    for (int p = 0; p < N; p++) {
        if (comp[p] < 0) cnt[p] = (uint32_t)N;
        else cnt[p] = 1u + (uint32_t)(N - csize[comp[p]]);
    }
    for (int p = 0; p < N; p++)
        for (int q = p + 1; q < N; q++)
            if (comp[p] < 0 || comp[q] < 0 || comp[p] != comp[q]) pre++;
    stats[5] = pre;
    if (D_out) {
        for (int p = 0; p < N; p++)
            for (int q = 0; q < N; q++) {
                uint32_t v;
                if (p == q) v = 0;
                else if (comp[p] < 0 || comp[q] < 0 || comp[p] != comp[q]) v = OR_UNREACH;
                else v = OR_UNSET;
                D_out[(size_t)p * N + q] = v;
            }
    }

    /* Order set-up. */
    int nseq = 0, cursor = 0;
    if (order == OR_NAIVE) {
        for (int p = 0; p < N; p++)
            if (comp[p] >= 0) seq[nseq++] = p;
    } else if (order == OR_SPIRAL) {
        nseq = or_spiral_sequence(mask, kind, H, W, seed, seq);
    } else if (order == OR_REPULSION) {
        nframes = or_rings(mask, kind, H, W, ring, fstart, fcyc);
    } else {
        uint32_t *e = (uint32_t *)malloc((size_t)N * sizeof(uint32_t));
        int32_t *cen = (int32_t *)malloc((size_t)N * sizeof(int32_t));
        or_extrema(f, mask, H, W, conn, kind, e, gcen, cen, rank);
        stats[1] = 2;
        free(e); free(cen);
    }

    int nsel_total = 0, rounds = 0, status = 0;
    for (;;) {
        /* Select from the state at the start of the round. */
        int ns = 0;
        if (order == OR_NAIVE || order == OR_SPIRAL) {
            while (cursor < nseq && ns < B) {
                int p = seq[cursor++];
                if (cnt[p] < (uint32_t)N) S[ns++] = p;
            }
        } else if (order == OR_REPULSION) {
            /* Spiral method with repulsion (Algorithm "spiral method with
             * repulsion", h = 3): S holds the current turn's points not yet
             * filled; a source is drawn uniformly from S, and its two left
             * and two right neighbours on the turn leave S with it. When S
             * is empty the outermost turn not yet filled starts again. The B
             * sources of a round are drawn one after the other from the
             * round-start state. */
            if (cur >= 0)
                for (int i = fstart[cur]; i < fstart[cur + 1]; i++)
                    if (inS[i - fstart[cur]] && cnt[ring[i]] >= (uint32_t)N) inS[i - fstart[cur]] = 0;
            while (ns < B) {
                int len = cur >= 0 ? fstart[cur + 1] - fstart[cur] : 0, size = 0;
                for (int i = 0; i < len; i++) size += inS[i];
                if (size == 0) {
                    cur = -1;
                    for (int k = 0; k < nframes && cur < 0; k++)
                        for (int i = fstart[k]; i < fstart[k + 1]; i++)
                            if (cnt[ring[i]] < (uint32_t)N && !taken[ring[i]]) { cur = k; break; }
                    if (cur < 0) break;
                    len = fstart[cur + 1] - fstart[cur];
                    for (int i = 0; i < len; i++) {
                        int p = ring[fstart[cur] + i];
                        inS[i] = (uint8_t)(cnt[p] < (uint32_t)N && !taken[p]);
                        size += inS[i];
                    }
                }
                int jth = (int)(or_splitmix64(&rst) % (uint64_t)size), at = -1;
                for (int i = 0; i < len; i++)
                    if (inS[i] && jth-- == 0) { at = i; break; }
                int s = ring[fstart[cur] + at];
                S[ns++] = s;
                taken[s] = 1;
                for (int dlt = -2; dlt <= 2; dlt++) {
                    int i = at + dlt;
                    if (fcyc[cur]) i = ((i % len) + len) % len;
                    if (i >= 0 && i < len) inS[i] = 0;
                }
            }
            for (int t = 0; t < ns; t++) taken[S[t]] = 0;
        } else if (order == OR_EXTREMA) {
            /* Geodesic extrema method (Sec. 3.3, Algorithm "geodesic extrema
             * method"): the unfilled points farthest from the centroid; among
             * points at the same distance the least filled, then the
             * smallest index. Plain repeated minimum search. */
            for (int k = 0; k < B; k++) {
                int best = -1;
                for (int p = 0; p < N; p++) {
                    if (comp[p] < 0 || cnt[p] >= (uint32_t)N || taken[p]) continue;
                    if (best < 0 || gcen[p] > gcen[best] ||
                        (gcen[p] == gcen[best] && cnt[p] < cnt[best]))
                        best = p;
                }
                if (best < 0) break;
                taken[best] = 1;
                S[ns++] = best;
            }
            for (int t = 0; t < ns; t++) taken[S[t]] = 0;
        } else {
            /* The B unfilled points of least filling rate; ties go to the
             * greatest geodesic extremum (smallest rank). Plain repeated
             * minimum search. */
            for (int k = 0; k < B; k++) {
                int best = -1;
                for (int p = 0; p < N; p++) {
                    if (comp[p] < 0 || cnt[p] >= (uint32_t)N || taken[p]) continue;
                    if (best < 0 || cnt[p] < cnt[best] ||
                        (cnt[p] == cnt[best] && rank[p] < rank[best]))
                        best = p;
                }
                if (best < 0) break;
                taken[best] = 1;
                S[ns++] = best;
            }
            for (int t = 0; t < ns; t++) taken[S[t]] = 0;
        }
        if (ns == 0) break;
        if (rounds >= N) { status = -1; break; }
        uint64_t new_this_round = 0;
        for (int i = 0; i < ns; i++) {
            int s = S[i];
            seq_out[nsel_total++] = s;
            stats[0]++;
            or_sssp(f, mask, H, W, conn, kind, s, d);
            or_parents(f, mask, H, W, conn, kind, d, s, parent);
            for (int b = 0; b < N; b++) {
                if (b == s || d[b] == OR_UNREACH) continue;
                for (int a = parent[b]; a >= 0; a = parent[a]) {
                    stats[2]++;
                    size_t ab = (size_t)a * N + b, ba = (size_t)b * N + a;
                    if (mrk[ab >> 6] & (1ull << (ab & 63))) continue;
                    mrk[ab >> 6] |= 1ull << (ab & 63);
                    mrk[ba >> 6] |= 1ull << (ba & 63);
                    cnt[a]++;
                    cnt[b]++;
                    new_this_round++;
                    if (D_out) {
                        uint32_t v = d[b] - d[a]; /* Property 1 */
                        D_out[ab] = v;
                        D_out[ba] = v;
                    }
                }
            }
        }
        round_new[rounds++] = new_this_round;
        stats[3] += new_this_round;
    }
    stats[4] = (uint64_t)rounds;
    free(ring); free(fstart); free(fcyc); free(inS);
    free(gcen); free(taken); free(S); free(rank); free(seq); free(parent); free(d);
    free(csize); free(comp); free(cnt); free(mrk);
    return status;
}
