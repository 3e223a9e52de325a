/*
 * Seeded synthetic graph generators shared by the test suite, the benchmark
 * and the oracle checks.  This file builds input graphs only: it contains no
 * step of the hybrid transfer method (no partitioning, no cost model, no
 * relaxation).  Every random number comes from a counter-based generator, so
 * the bytes produced do not depend on the number of threads.
 *
 * Graph families (the paper evaluates on R-MAT graphs, Sec. VII-A and Table 4,
 * and on real web/social graphs that are stood in for by these shapes):
 *   - R-MAT (Chakrabarti et al., 2004) with parameters (a, b, c, d), no vertex
 *     scrambling, so the hubs sit near vertex 0;
 *   - a W x H 4-neighbour grid with a fraction of local shortcuts (a
 *     high-diameter, road-like mesh);
 *   - Chung-Lu power-law graphs with expected degree (i + i0)^(-1/(beta-1)),
 *     both endpoints drawn by inverse CDF of the continuous weight density.
 *
 * Output format: CSR with uint64 row offsets (V + 1 entries), uint32
 * destinations and uint32 weights.  Rows are sorted by (dst, weight) so that
 * the CSR is a pure function of (family, parameters, seed).  Duplicates and
 * self-loops are kept.
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

/* ---------------------------------------------------------------- RNG ---- */
/* splitmix64 (Steele, Lea, Flood, "Fast splittable pseudorandom number
 * generators", OOPSLA 2014): golden-gamma increment followed by the
 * published 64-bit finaliser. */
static inline uint64_t sm64(uint64_t x) {
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}
/* Counter-based draw: value i of stream `stream` under `seed`. */
static inline uint64_t ctr_draw(uint64_t seed, uint64_t stream, uint64_t i) {
    return sm64(sm64(seed ^ (stream * 0xD6E8FEB86659FD93ull)) + i);
}
uint64_t gg_draw(uint64_t seed, uint64_t stream, uint64_t i) { return ctr_draw(seed, stream, i); }

enum { ST_RMAT = 1, ST_W = 2, ST_SC = 3, ST_CL = 4 };

/* ----------------------------------------------------------- threads ---- */
typedef void (*range_fn)(void *ctx, uint64_t lo, uint64_t hi);
typedef struct { range_fn fn; void *ctx; uint64_t lo, hi; } job_t;
static void *job_run(void *p) { job_t *j = (job_t *)p; j->fn(j->ctx, j->lo, j->hi); return NULL; }

static void parallel_for(uint64_t n, int nthreads, range_fn fn, void *ctx) {
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    if ((uint64_t)nthreads > n) nthreads = n ? (int)n : 1;
    pthread_t th[256];
    job_t jobs[256];
    for (int t = 0; t < nthreads; ++t) {
        jobs[t].fn = fn; jobs[t].ctx = ctx;
        jobs[t].lo = n * (uint64_t)t / nthreads;
        jobs[t].hi = n * (uint64_t)(t + 1) / nthreads;
    }
    for (int t = 1; t < nthreads; ++t) pthread_create(&th[t], NULL, job_run, &jobs[t]);
    job_run(&jobs[0]);
    for (int t = 1; t < nthreads; ++t) pthread_join(th[t], NULL);
}

/* ------------------------------------------------- row sort (dst, w) ---- */
static void sort_row(uint32_t *d, uint32_t *w, uint64_t n) {
    if (n < 2) return;
    if (n <= 32) {
        for (uint64_t i = 1; i < n; ++i) {
            uint32_t kd = d[i], kw = w ? w[i] : 0;
            uint64_t j = i;
            while (j > 0 && (d[j - 1] > kd || (d[j - 1] == kd && w && w[j - 1] > kw))) {
                d[j] = d[j - 1];
                if (w) w[j] = w[j - 1];
                --j;
            }
            d[j] = kd;
            if (w) w[j] = kw;
        }
        return;
    }
    /* pack to 64-bit keys and use an LSD radix sort on the packed key */
    uint64_t *k = (uint64_t *)malloc(n * sizeof(uint64_t));
    uint64_t *t = (uint64_t *)malloc(n * sizeof(uint64_t));
    for (uint64_t i = 0; i < n; ++i) k[i] = ((uint64_t)d[i] << 32) | (w ? w[i] : 0u);
    for (int pass = 0; pass < 8; ++pass) {
        int sh = pass * 8;
        uint64_t cnt[257];
        memset(cnt, 0, sizeof(cnt));
        for (uint64_t i = 0; i < n; ++i) cnt[((k[i] >> sh) & 255) + 1]++;
        int trivial = 0;
        for (int b = 0; b < 256; ++b) if (cnt[b + 1] == n) trivial = 1;
        if (trivial) continue;
        for (int b = 0; b < 256; ++b) cnt[b + 1] += cnt[b];
        for (uint64_t i = 0; i < n; ++i) t[cnt[(k[i] >> sh) & 255]++] = k[i];
        uint64_t *s = k; k = t; t = s;
    }
    for (uint64_t i = 0; i < n; ++i) { d[i] = (uint32_t)(k[i] >> 32); if (w) w[i] = (uint32_t)k[i]; }
    free(k); free(t);
}

typedef struct { const uint64_t *off; uint32_t *dst, *w; } rowsort_ctx;
static void rowsort_range(void *p, uint64_t lo, uint64_t hi) {
    rowsort_ctx *c = (rowsort_ctx *)p;
    for (uint64_t v = lo; v < hi; ++v)
        sort_row(c->dst + c->off[v], c->w ? c->w + c->off[v] : NULL, c->off[v + 1] - c->off[v]);
}

/* exclusive prefix sum of counts[0..V) into off[0..V], off[V] = total */
static uint64_t exclusive_scan(const uint64_t *counts, uint64_t *off, uint64_t V) {
    uint64_t s = 0;
    for (uint64_t v = 0; v < V; ++v) { off[v] = s; s += counts[v]; }
    off[V] = s;
    return s;
}

/* ------------------------------------------------------------- R-MAT ---- */
typedef struct {
    uint64_t seed; int scale; uint32_t thr_a, thr_ab, thr_abc;
    uint64_t *deg;       /* counting pass: atomic per-source counts */
    uint64_t *cursor;    /* scatter pass: atomic per-source cursors */
    uint32_t *dst, *w; uint32_t wmax;
} rmat_ctx;

static inline void rmat_edge(const rmat_ctx *c, uint64_t e, uint64_t *s, uint64_t *d) {
    uint64_t src = 0, dst = 0;
    uint64_t r = 0;
    for (int l = 0; l < c->scale; ++l) {
        uint32_t u;
        if ((l & 1) == 0) { r = ctr_draw(c->seed, ST_RMAT, e * (uint64_t)((c->scale + 1) / 2) + (uint64_t)(l / 2)); u = (uint32_t)r; }
        else u = (uint32_t)(r >> 32);
        uint64_t bit = 1ull << (c->scale - 1 - l);
        if (u < c->thr_a) { }
        else if (u < c->thr_ab) dst |= bit;
        else if (u < c->thr_abc) src |= bit;
        else { src |= bit; dst |= bit; }
    }
    *s = src; *d = dst;
}
static void rmat_count(void *p, uint64_t lo, uint64_t hi) {
    rmat_ctx *c = (rmat_ctx *)p;
    for (uint64_t e = lo; e < hi; ++e) {
        uint64_t s, d; rmat_edge(c, e, &s, &d);
        __atomic_fetch_add(&c->deg[s], 1, __ATOMIC_RELAXED);
    }
}
static void rmat_scatter(void *p, uint64_t lo, uint64_t hi) {
    rmat_ctx *c = (rmat_ctx *)p;
    for (uint64_t e = lo; e < hi; ++e) {
        uint64_t s, d; rmat_edge(c, e, &s, &d);
        uint64_t pos = __atomic_fetch_add(&c->cursor[s], 1, __ATOMIC_RELAXED);
        c->dst[pos] = (uint32_t)d;
        if (c->w) c->w[pos] = 1u + (uint32_t)(ctr_draw(c->seed, ST_W, e) % c->wmax);
    }
}

/* Number of edges: E = edge_factor * 2^scale.  off must hold V+1 entries,
 * dst and w (w may be NULL) E entries.  Weights uniform in [1, wmax]. */
int gg_rmat(int scale, uint64_t E, double a, double b, double c, uint64_t seed, uint32_t wmax,
            int nthreads, uint64_t *off, uint32_t *dst, uint32_t *w) {
    if (scale < 1 || scale > 31 || a < 0 || b < 0 || c < 0 || a + b + c > 1.0 || wmax == 0) return -1;
    uint64_t V = 1ull << scale;
    rmat_ctx ctx;
    ctx.seed = seed; ctx.scale = scale;
    double two32 = 4294967296.0;
    double ta = a * two32, tab = (a + b) * two32, tabc = (a + b + c) * two32;
    ctx.thr_a = ta >= two32 ? 0xFFFFFFFFu : (uint32_t)ta;
    ctx.thr_ab = tab >= two32 ? 0xFFFFFFFFu : (uint32_t)tab;
    ctx.thr_abc = tabc >= two32 ? 0xFFFFFFFFu : (uint32_t)tabc;
    ctx.deg = (uint64_t *)calloc(V, sizeof(uint64_t));
    if (!ctx.deg) return -2;
    ctx.dst = dst; ctx.w = w; ctx.wmax = wmax;
    parallel_for(E, nthreads, rmat_count, &ctx);
    exclusive_scan(ctx.deg, off, V);
    memcpy(ctx.deg, off, V * sizeof(uint64_t));
    ctx.cursor = ctx.deg;
    parallel_for(E, nthreads, rmat_scatter, &ctx);
    free(ctx.deg);
    rowsort_ctx rs = { off, dst, w };
    parallel_for(V, nthreads, rowsort_range, &rs);
    return 0;
}

/* --------------------------------------------------------- grid mesh ---- */
/* Vertex id = r * W + c.  Grid edges in both directions to the 4 neighbours
 * inside the grid.  n_short vertices, drawn with replacement, each get one
 * undirected shortcut (both directions) to a vertex whose row and column are
 * each within +-radius, chosen uniformly among the in-grid offsets other than
 * (0, 0).  Weights uniform in [1, wmax], one draw per final CSR position. */
typedef struct {
    uint64_t W, H, seed; uint64_t n_short; int radius;
    uint64_t *sc_u, *sc_v;        /* shortcut endpoints */
    uint64_t *deg;
    const uint64_t *off; uint32_t *dst, *w; uint32_t wmax;
} mesh_ctx;

static void mesh_pick_shortcuts(void *p, uint64_t lo, uint64_t hi) {
    mesh_ctx *c = (mesh_ctx *)p;
    uint64_t V = c->W * c->H, span = 2 * (uint64_t)c->radius + 1;
    for (uint64_t j = lo; j < hi; ++j) {
        uint64_t u = ctr_draw(c->seed, ST_SC, 4 * j) % V;
        uint64_t r = u / c->W, col = u % c->W;
        uint64_t v = u;
        for (uint64_t t = 0; v == u; ++t) {
            uint64_t x = ctr_draw(c->seed, ST_SC, 4 * j + 1 + 2 * t);
            uint64_t y = ctr_draw(c->seed ^ 0x5bd1e995ull, ST_SC, 4 * j + 1 + 2 * t);
            int64_t dr = (int64_t)(x % span) - c->radius, dc = (int64_t)(y % span) - c->radius;
            int64_t rr = (int64_t)r + dr, cc = (int64_t)col + dc;
            if (rr < 0 || cc < 0 || rr >= (int64_t)c->H || cc >= (int64_t)c->W) continue;
            v = (uint64_t)rr * c->W + (uint64_t)cc;
        }
        c->sc_u[j] = u; c->sc_v[j] = v;
    }
}
static void mesh_grid_degree(void *p, uint64_t lo, uint64_t hi) {
    mesh_ctx *c = (mesh_ctx *)p;
    for (uint64_t u = lo; u < hi; ++u) {
        uint64_t r = u / c->W, col = u % c->W;
        c->deg[u] = (r > 0) + (col > 0) + (col + 1 < c->W) + (r + 1 < c->H);
    }
}
static void mesh_grid_fill(void *p, uint64_t lo, uint64_t hi) {
    mesh_ctx *c = (mesh_ctx *)p;
    for (uint64_t u = lo; u < hi; ++u) {
        uint64_t r = u / c->W, col = u % c->W, pos = c->off[u];
        if (r > 0) c->dst[pos++] = (uint32_t)(u - c->W);
        if (col > 0) c->dst[pos++] = (uint32_t)(u - 1);
        if (col + 1 < c->W) c->dst[pos++] = (uint32_t)(u + 1);
        if (r + 1 < c->H) c->dst[pos++] = (uint32_t)(u + c->W);
        c->deg[u] = pos;   /* becomes the shortcut cursor */
    }
}
static void weights_fill(void *p, uint64_t lo, uint64_t hi) {
    mesh_ctx *c = (mesh_ctx *)p;
    for (uint64_t e = lo; e < hi; ++e) c->w[e] = 1u + (uint32_t)(ctr_draw(c->seed, ST_W, e) % c->wmax);
}

/* Returns the edge count through *E_out.  Call once with dst == NULL to get
 * the offsets and E, then again with buffers of E entries. */
int gg_mesh(uint64_t W, uint64_t H, uint64_t n_short, int radius, uint64_t seed, uint32_t wmax,
            int nthreads, uint64_t *off, uint32_t *dst, uint32_t *w, uint64_t *E_out) {
    if (W < 1 || H < 1 || W * H > 0xFFFFFFFFull || radius < 1 || wmax == 0) return -1;
    if (W * H == 1) n_short = 0;
    uint64_t V = W * H;
    mesh_ctx c;
    memset(&c, 0, sizeof(c));
    c.W = W; c.H = H; c.seed = seed; c.n_short = n_short; c.radius = radius; c.wmax = wmax;
    c.sc_u = (uint64_t *)malloc((n_short + 1) * sizeof(uint64_t));
    c.sc_v = (uint64_t *)malloc((n_short + 1) * sizeof(uint64_t));
    c.deg = (uint64_t *)malloc(V * sizeof(uint64_t));
    if (!c.sc_u || !c.sc_v || !c.deg) return -2;
    parallel_for(n_short, nthreads, mesh_pick_shortcuts, &c);
    parallel_for(V, nthreads, mesh_grid_degree, &c);
    for (uint64_t j = 0; j < n_short; ++j) { c.deg[c.sc_u[j]]++; c.deg[c.sc_v[j]]++; }
    uint64_t E = exclusive_scan(c.deg, off, V);
    *E_out = E;
    if (dst) {
        c.off = off; c.dst = dst; c.w = w;
        parallel_for(V, nthreads, mesh_grid_fill, &c);
        for (uint64_t j = 0; j < n_short; ++j) {
            uint64_t u = c.sc_u[j], v = c.sc_v[j];
            dst[c.deg[u]++] = (uint32_t)v;
            dst[c.deg[v]++] = (uint32_t)u;
        }
        rowsort_ctx rs = { off, dst, NULL };
        parallel_for(V, nthreads, rowsort_range, &rs);
        if (w) parallel_for(E, nthreads, weights_fill, &c);
    }
    free(c.sc_u); free(c.sc_v); free(c.deg);
    return 0;
}

/* ---------------------------------------------------------- Chung-Lu ---- */
/* Weight density f(x) = (x + i0)^(-alpha) on x in [0, V), alpha = 1/(beta-1).
 * Inverse CDF in closed form: with g(x) = (x + i0)^(1-alpha),
 * x = (g(0) + u (g(V) - g(0)))^(1/(1-alpha)) - i0, vertex = floor(x). */
typedef struct {
    uint64_t V, seed; double alpha, i0, g0, g1;
    uint64_t *deg, *cursor; uint32_t *dst, *w; uint32_t wmax;
} cl_ctx;
static inline uint64_t cl_vertex(const cl_ctx *c, uint64_t r) {
    double u = (double)(r >> 11) * (1.0 / 9007199254740992.0);
    double g = c->g0 + u * (c->g1 - c->g0);
    double x = pow(g, 1.0 / (1.0 - c->alpha)) - c->i0;
    if (x < 0) x = 0;
    uint64_t v = (uint64_t)x;
    return v >= c->V ? c->V - 1 : v;
}
static void cl_count(void *p, uint64_t lo, uint64_t hi) {
    cl_ctx *c = (cl_ctx *)p;
    for (uint64_t e = lo; e < hi; ++e) {
        uint64_t s = cl_vertex(c, ctr_draw(c->seed, ST_CL, 2 * e));
        __atomic_fetch_add(&c->deg[s], 1, __ATOMIC_RELAXED);
    }
}
static void cl_scatter(void *p, uint64_t lo, uint64_t hi) {
    cl_ctx *c = (cl_ctx *)p;
    for (uint64_t e = lo; e < hi; ++e) {
        uint64_t s = cl_vertex(c, ctr_draw(c->seed, ST_CL, 2 * e));
        uint64_t d = cl_vertex(c, ctr_draw(c->seed, ST_CL, 2 * e + 1));
        uint64_t pos = __atomic_fetch_add(&c->cursor[s], 1, __ATOMIC_RELAXED);
        c->dst[pos] = (uint32_t)d;
        if (c->w) c->w[pos] = 1u + (uint32_t)(ctr_draw(c->seed, ST_W, e) % c->wmax);
    }
}
int gg_chung_lu(uint64_t V, uint64_t E, double beta, double i0, uint64_t seed, uint32_t wmax,
                int nthreads, uint64_t *off, uint32_t *dst, uint32_t *w) {
    if (V < 1 || V > 0xFFFFFFFFull || beta <= 2.0 || i0 <= 0 || wmax == 0) return -1;
    cl_ctx c;
    c.V = V; c.seed = seed; c.alpha = 1.0 / (beta - 1.0); c.i0 = i0; c.wmax = wmax;
    c.g0 = pow(i0, 1.0 - c.alpha);
    c.g1 = pow((double)V + i0, 1.0 - c.alpha);
    c.deg = (uint64_t *)calloc(V, sizeof(uint64_t));
    if (!c.deg) return -2;
    c.dst = dst; c.w = w;
    parallel_for(E, nthreads, cl_count, &c);
    exclusive_scan(c.deg, off, V);
    memcpy(c.deg, off, V * sizeof(uint64_t));
    c.cursor = c.deg;
    parallel_for(E, nthreads, cl_scatter, &c);
    free(c.deg);
    rowsort_ctx rs = { off, dst, w };
    parallel_for(V, nthreads, rowsort_range, &rs);
    return 0;
}

/* ------------------------------------------------------- symmetrise ---- */
/* For every edge u->v emit u->v and v->u (2E edges; a self-loop appears
 * twice).  Weights are not carried (connected components ignore them). */
typedef struct { uint64_t V; const uint64_t *off; const uint32_t *dst; uint64_t *deg; uint64_t *off2; uint32_t *dst2; } sym_ctx;
static void sym_count_in(void *p, uint64_t lo, uint64_t hi) {
    sym_ctx *c = (sym_ctx *)p;
    for (uint64_t u = lo; u < hi; ++u)
        for (uint64_t e = c->off[u]; e < c->off[u + 1]; ++e)
            __atomic_fetch_add(&c->deg[c->dst[e]], 1, __ATOMIC_RELAXED);
}
static void sym_fill(void *p, uint64_t lo, uint64_t hi) {
    sym_ctx *c = (sym_ctx *)p;
    for (uint64_t u = lo; u < hi; ++u) {
        uint64_t n = c->off[u + 1] - c->off[u];
        uint64_t pos = __atomic_fetch_add(&c->deg[u], n, __ATOMIC_RELAXED);
        memcpy(c->dst2 + pos, c->dst + c->off[u], n * sizeof(uint32_t));
        for (uint64_t e = c->off[u]; e < c->off[u + 1]; ++e) {
            uint64_t q = __atomic_fetch_add(&c->deg[c->dst[e]], 1, __ATOMIC_RELAXED);
            c->dst2[q] = (uint32_t)u;
        }
    }
}
int gg_symmetrize(uint64_t V, const uint64_t *off, const uint32_t *dst, int nthreads,
                  uint64_t *off2, uint32_t *dst2) {
    sym_ctx c;
    c.V = V; c.off = off; c.dst = dst; c.off2 = off2; c.dst2 = dst2;
    c.deg = (uint64_t *)calloc(V, sizeof(uint64_t));
    if (!c.deg) return -2;
    for (uint64_t u = 0; u < V; ++u) c.deg[u] = off[u + 1] - off[u];
    parallel_for(V, nthreads, sym_count_in, &c);
    exclusive_scan(c.deg, off2, V);
    memcpy(c.deg, off2, V * sizeof(uint64_t));
    parallel_for(V, nthreads, sym_fill, &c);
    free(c.deg);
    rowsort_ctx rs = { off2, dst2, NULL };
    parallel_for(V, nthreads, rowsort_range, &rs);
    return 0;
}
