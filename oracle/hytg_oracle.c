/*
 * ORACLE -- test infrastructure only.  Plain, slow, single-threaded CPU code
 * that states what the hybrid-transfer graph engine must compute.  Only the
 * test suite, the smoke check and the benchmark's CPU-baseline leg may load
 * this library; the product path never does.  It shares no code with the
 * CUDA library.
 *
 * The hybrid transfer method (Sec. I, Sec. IV) only changes how active edges
 * reach the GPU, never what is computed, so each algorithm's oracle is the
 * textbook definition of its result:
 *   BFS   (Sec. VII-A): hop distance from the source along out-edges, FIFO queue.
 *   SSSP  (Sec. II-A, Fig. 1): shortest path distance, Dijkstra with a binary
 *         heap and lazy deletion, 64-bit accumulation.
 *   CC    (Sec. VII-A): weakly connected components by union-find; the label
 *         of a vertex is the smallest vertex id in its component.
 *   PageRank / personalised PageRank (Sec. VI-A, delta-based PageRank): the
 *         fixed point x = (1-d) t + d A^T D_o^-1 x by FP64 power iteration,
 *         where t is all-ones (PageRank) or the seed indicator (PPR).
 *         Vertices with no out-edges push nothing (their mass leaks).
 * Alternates (Bellman-Ford, BFS-labelled components) and O(E) certificates
 * pin the oracle against something other than itself.
 *
 * The cost-model counts (Sec. V-A, Eq. 1-3 and the footnote to Eq. 3) are
 * also computed here from their definitions: per partition, the number of
 * active vertices, the active out-edges, and the exact number of 128-byte
 * lines that the active vertices' edge lists span.
 *
 * Unreached vertices hold 0xFFFFFFFF.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

#define UNREACHED 0xFFFFFFFFu

/* ---------------------------------------------------------------- BFS ---- */
/* level[v] = number of edges on a shortest directed path source -> v. */
int or_bfs(uint64_t V, const uint64_t *off, const uint32_t *dst, uint32_t src,
           uint32_t *level, uint64_t *edges_scanned) {
    if (src >= V) return -1;
    for (uint64_t v = 0; v < V; ++v) level[v] = UNREACHED;
    uint32_t *queue = (uint32_t *)malloc((V ? V : 1) * sizeof(uint32_t));
    if (!queue) return -2;
    uint64_t head = 0, tail = 0, scanned = 0;
    level[src] = 0;
    queue[tail++] = src;
    while (head < tail) {
        uint32_t u = queue[head++];
        for (uint64_t e = off[u]; e < off[u + 1]; ++e) {
            uint32_t v = dst[e];
            if (level[v] == UNREACHED) {
                level[v] = level[u] + 1;
                queue[tail++] = v;
            }
        }
        scanned += off[u + 1] - off[u];
    }
    free(queue);
    if (edges_scanned) *edges_scanned = scanned;
    return 0;
}

/* --------------------------------------------------------------- SSSP ---- */
typedef struct { uint64_t d; uint32_t v; } heap_item;

static void heap_push(heap_item *h, uint64_t *n, heap_item x) {
    uint64_t i = (*n)++;
    while (i > 0) {
        uint64_t p = (i - 1) / 2;
        if (h[p].d <= x.d) break;
        h[i] = h[p];
        i = p;
    }
    h[i] = x;
}
static heap_item heap_pop(heap_item *h, uint64_t *n) {
    heap_item top = h[0], last = h[--(*n)];
    uint64_t i = 0;
    for (;;) {
        uint64_t l = 2 * i + 1, r = l + 1, m = i;
        heap_item best = last;
        if (l < *n && h[l].d < best.d) { m = l; best = h[l]; }
        if (r < *n && h[r].d < best.d) { m = r; best = h[r]; }
        if (m == i) break;
        h[i] = h[m];
        i = m;
    }
    if (*n > 0) h[i] = last;
    return top;
}

/* dist[v] = min over directed paths source -> v of the sum of weights.
 * Returns 1 if some reached distance is >= 0xFFFFFFFE (it would not fit the
 * 32-bit result with 0xFFFFFFFF reserved for "unreached"); 0 otherwise. */
int or_sssp_dijkstra(uint64_t V, const uint64_t *off, const uint32_t *dst, const uint32_t *w,
                     uint32_t src, uint32_t *dist, uint64_t *edges_scanned) {
    if (src >= V) return -1;
    uint64_t E = off[V];
    uint64_t *d = (uint64_t *)malloc((V ? V : 1) * sizeof(uint64_t));
    unsigned char *done = (unsigned char *)calloc(V ? V : 1, 1);
    heap_item *h = (heap_item *)malloc((E + 1) * sizeof(heap_item));
    if (!d || !done || !h) { free(d); free(done); free(h); return -2; }
    for (uint64_t v = 0; v < V; ++v) d[v] = UINT64_MAX;
    uint64_t n = 0, scanned = 0;
    d[src] = 0;
    heap_push(h, &n, (heap_item){0, src});
    while (n > 0) {
        heap_item it = heap_pop(h, &n);
        uint32_t u = it.v;
        if (done[u] || it.d != d[u]) continue;
        done[u] = 1;
        for (uint64_t e = off[u]; e < off[u + 1]; ++e) {
            uint64_t nd = d[u] + w[e];
            if (nd < d[dst[e]]) {
                d[dst[e]] = nd;
                heap_push(h, &n, (heap_item){nd, dst[e]});
            }
        }
        scanned += off[u + 1] - off[u];
    }
    int overflow = 0;
    for (uint64_t v = 0; v < V; ++v) {
        if (d[v] == UINT64_MAX) dist[v] = UNREACHED;
        else if (d[v] >= 0xFFFFFFFEull) { dist[v] = UNREACHED; overflow = 1; }
        else dist[v] = (uint32_t)d[v];
    }
    free(d); free(done); free(h);
    if (edges_scanned) *edges_scanned = scanned;
    return overflow;
}

/* Alternate: Bellman-Ford, relaxing every edge until a full pass changes
 * nothing (at most V passes).  O(V E): small graphs only. */
int or_sssp_bellman_ford(uint64_t V, const uint64_t *off, const uint32_t *dst, const uint32_t *w,
                         uint32_t src, uint32_t *dist) {
    if (src >= V) return -1;
    uint64_t *d = (uint64_t *)malloc((V ? V : 1) * sizeof(uint64_t));
    if (!d) return -2;
    for (uint64_t v = 0; v < V; ++v) d[v] = UINT64_MAX;
    d[src] = 0;
    for (uint64_t pass = 0; pass <= V; ++pass) {
        int changed = 0;
        for (uint64_t u = 0; u < V; ++u) {
            if (d[u] == UINT64_MAX) continue;
            for (uint64_t e = off[u]; e < off[u + 1]; ++e) {
                uint64_t nd = d[u] + (w ? w[e] : 1u);
                if (nd < d[dst[e]]) { d[dst[e]] = nd; changed = 1; }
            }
        }
        if (!changed) break;
    }
    int overflow = 0;
    for (uint64_t v = 0; v < V; ++v) {
        if (d[v] == UINT64_MAX) dist[v] = UNREACHED;
        else if (d[v] >= 0xFFFFFFFEull) { dist[v] = UNREACHED; overflow = 1; }
        else dist[v] = (uint32_t)d[v];
    }
    free(d);
    return overflow;
}

/* ----------------------------------------------------------------- CC ---- */
static uint32_t uf_find(uint32_t *parent, uint32_t x) {
    while (parent[x] != x) {
        parent[x] = parent[parent[x]];   /* path halving */
        x = parent[x];
    }
    return x;
}

/* Weakly connected components: edges are taken as undirected.  The root of
 * every set is kept at its smallest member, so find(v) is the label. */
int or_cc_unionfind(uint64_t V, const uint64_t *off, const uint32_t *dst, uint32_t *label) {
    for (uint64_t v = 0; v < V; ++v) label[v] = (uint32_t)v;
    for (uint64_t u = 0; u < V; ++u) {
        for (uint64_t e = off[u]; e < off[u + 1]; ++e) {
            uint32_t a = uf_find(label, (uint32_t)u), b = uf_find(label, dst[e]);
            if (a < b) label[b] = a;
            else if (b < a) label[a] = b;
        }
    }
    for (uint64_t v = 0; v < V; ++v) label[v] = uf_find(label, (uint32_t)v);
    return 0;
}

/* Alternate for symmetric graphs: scan ids upwards, and BFS from each vertex
 * not yet labelled, giving its whole component the start id (the smallest
 * id of that component, since every smaller id was labelled earlier). */
int or_cc_bfs(uint64_t V, const uint64_t *off, const uint32_t *dst, uint32_t *label) {
    uint32_t *queue = (uint32_t *)malloc((V ? V : 1) * sizeof(uint32_t));
    if (!queue) return -2;
    for (uint64_t v = 0; v < V; ++v) label[v] = UNREACHED;
    for (uint64_t s = 0; s < V; ++s) {
        if (label[s] != UNREACHED) continue;
        uint64_t head = 0, tail = 0;
        label[s] = (uint32_t)s;
        queue[tail++] = (uint32_t)s;
        while (head < tail) {
            uint32_t u = queue[head++];
            for (uint64_t e = off[u]; e < off[u + 1]; ++e)
                if (label[dst[e]] == UNREACHED) { label[dst[e]] = (uint32_t)s; queue[tail++] = dst[e]; }
        }
    }
    free(queue);
    return 0;
}

/* 1 if for every edge u->v the graph also has v->u with the same multiplicity. */
int or_is_symmetric(uint64_t V, const uint64_t *off, const uint32_t *dst) {
    uint64_t E = off[V];
    uint64_t *cnt_in = (uint64_t *)calloc(V + 1, sizeof(uint64_t));
    uint32_t *rev = (uint32_t *)malloc((E ? E : 1) * sizeof(uint32_t));
    if (!cnt_in || !rev) { free(cnt_in); free(rev); return -2; }
    for (uint64_t e = 0; e < E; ++e) cnt_in[dst[e] + 1]++;
    for (uint64_t v = 0; v < V; ++v) cnt_in[v + 1] += cnt_in[v];
    int sym = 1;
    for (uint64_t v = 0; v < V && sym; ++v) if (cnt_in[v + 1] - cnt_in[v] != off[v + 1] - off[v]) sym = 0;
    if (sym) {
        /* reverse adjacency, sources in increasing order, then compare sorted rows */
        uint64_t *cur = (uint64_t *)malloc((V ? V : 1) * sizeof(uint64_t));
        memcpy(cur, cnt_in, V * sizeof(uint64_t));
        for (uint64_t u = 0; u < V; ++u)
            for (uint64_t e = off[u]; e < off[u + 1]; ++e) rev[cur[dst[e]]++] = (uint32_t)u;
        free(cur);
        for (uint64_t v = 0; v < V && sym; ++v) {
            /* rows of dst are sorted by the generators; sort a copy to be safe */
            uint64_t n = off[v + 1] - off[v];
            uint32_t *a = (uint32_t *)malloc((n ? n : 1) * sizeof(uint32_t));
            memcpy(a, dst + off[v], n * sizeof(uint32_t));
            for (uint64_t i = 1; i < n; ++i) {
                uint32_t k = a[i]; uint64_t j = i;
                while (j > 0 && a[j - 1] > k) { a[j] = a[j - 1]; --j; }
                a[j] = k;
            }
            for (uint64_t i = 0; i < n; ++i) if (a[i] != rev[cnt_in[v] + i]) { sym = 0; break; }
            free(a);
        }
    }
    free(cnt_in); free(rev);
    return sym;
}

/* ----------------------------------------------------------- PageRank ---- */
/* Power iteration x_{t+1}[v] = (1-d) t[v] + d * sum_{u->v} x_t[u] / D_o(u),
 * from x_0 = t, in FP64, until ||x_{t+1} - x_t||_1 < tol * sum(t) or maxit
 * iterations.  t[v] = 1 for every v (seed == UINT32_MAX) or t = e_seed.
 * x_out receives x / sum(x); raw_sum the sum of the unnormalised fixed point. */
int or_pagerank(uint64_t V, const uint64_t *off, const uint32_t *dst, double d, double tol,
                int maxit, uint32_t seed, double *x_out, double *raw_sum, int *iters) {
    if (V == 0) return -1;
    if (seed != UNREACHED && seed >= V) return -1;
    double *x = (double *)malloc(V * sizeof(double));
    double *y = (double *)malloc(V * sizeof(double));
    if (!x || !y) { free(x); free(y); return -2; }
    double tsum = (seed == UNREACHED) ? (double)V : 1.0;
    for (uint64_t v = 0; v < V; ++v) x[v] = (seed == UNREACHED || v == seed) ? 1.0 : 0.0;
    int it = 0;
    for (; it < maxit; ++it) {
        for (uint64_t v = 0; v < V; ++v) y[v] = (seed == UNREACHED || v == seed) ? (1.0 - d) : 0.0;
        for (uint64_t u = 0; u < V; ++u) {
            uint64_t deg = off[u + 1] - off[u];
            if (deg == 0) continue;
            double share = d * x[u] / (double)deg;
            for (uint64_t e = off[u]; e < off[u + 1]; ++e) y[dst[e]] += share;
        }
        double diff = 0.0;
        for (uint64_t v = 0; v < V; ++v) diff += fabs(y[v] - x[v]);
        double *s = x; x = y; y = s;
        if (diff < tol * tsum) { ++it; break; }
    }
    double sum = 0.0;
    for (uint64_t v = 0; v < V; ++v) sum += x[v];
    for (uint64_t v = 0; v < V; ++v) x_out[v] = sum > 0 ? x[v] / sum : 0.0;
    if (raw_sum) *raw_sum = sum;
    if (iters) *iters = it;
    free(x); free(y);
    return 0;
}

/* Residual of a candidate rank vector r (unnormalised scale):
 * res = || (1-d) t + d A^T D_o^-1 r - r ||_1.  For the contraction
 * x -> (1-d) t + d A^T D_o^-1 x (factor d in the L1 norm, since every column
 * of A^T D_o^-1 sums to 1 or 0), ||r - x*||_1 <= res / (1 - d). */
int or_pagerank_residual(uint64_t V, const uint64_t *off, const uint32_t *dst, double d,
                         uint32_t seed, const double *r, double *res) {
    double *y = (double *)malloc((V ? V : 1) * sizeof(double));
    if (!y) return -2;
    for (uint64_t v = 0; v < V; ++v) y[v] = (seed == UNREACHED || v == seed) ? (1.0 - d) : 0.0;
    for (uint64_t u = 0; u < V; ++u) {
        uint64_t deg = off[u + 1] - off[u];
        if (deg == 0) continue;
        double share = d * r[u] / (double)deg;
        for (uint64_t e = off[u]; e < off[u + 1]; ++e) y[dst[e]] += share;
    }
    double s = 0.0;
    for (uint64_t v = 0; v < V; ++v) s += fabs(y[v] - r[v]);
    *res = s;
    free(y);
    return 0;
}

/* ------------------------------------------------------- certificates ---- */
/* Each returns 0 if the candidate is exactly the algorithm's result, else a
 * positive code; *bad receives the offending vertex. */

/* BFS: level[src] = 0; every edge u->v with u reached has level[v] <=
 * level[u] + 1; every reached v != src has an in-edge from a u with
 * level[u] = level[v] - 1; an unreached vertex has no reached in-neighbour
 * (covered by the edge rule, since level[v] <= level[u] + 1 < UNREACHED). */
int or_bfs_certify(uint64_t V, const uint64_t *off, const uint32_t *dst, uint32_t src,
                   const uint32_t *level, uint64_t *bad) {
    if (level[src] != 0) { *bad = src; return 1; }
    unsigned char *tight = (unsigned char *)calloc(V ? V : 1, 1);
    int rc = 0;
    for (uint64_t u = 0; u < V && !rc; ++u) {
        if (level[u] == UNREACHED) continue;
        for (uint64_t e = off[u]; e < off[u + 1]; ++e) {
            uint32_t v = dst[e];
            if ((uint64_t)level[v] > (uint64_t)level[u] + 1) { *bad = v; rc = 2; break; }
            if ((uint64_t)level[v] == (uint64_t)level[u] + 1) tight[v] = 1;
        }
    }
    for (uint64_t v = 0; v < V && !rc; ++v)
        if (v != src && level[v] != UNREACHED && !tight[v]) { *bad = v; rc = 3; }
    free(tight);
    return rc;
}

/* SSSP with non-negative weights: dist[src] = 0; dist[v] <= dist[u] + w on
 * every edge from a reached u; every reached v != src has a tight in-edge
 * (dist[v] = dist[u] + w).  Together these make dist the exact distances
 * when every weight is >= 1: inducting along a shortest path, the edge rule
 * gives dist[v] <= true distance; following tight in-edges backwards strictly
 * lowers dist, so the chain ends at the source and is a path of length
 * dist[v], giving dist[v] >= true distance. */
int or_sssp_certify(uint64_t V, const uint64_t *off, const uint32_t *dst, const uint32_t *w,
                    uint32_t src, const uint32_t *dist, uint64_t *bad) {
    if (dist[src] != 0) { *bad = src; return 1; }
    unsigned char *tight = (unsigned char *)calloc(V ? V : 1, 1);
    int rc = 0;
    for (uint64_t u = 0; u < V && !rc; ++u) {
        if (dist[u] == UNREACHED) continue;
        for (uint64_t e = off[u]; e < off[u + 1]; ++e) {
            uint32_t v = dst[e];
            uint64_t nd = (uint64_t)dist[u] + w[e];
            if ((uint64_t)dist[v] > nd) { *bad = v; rc = 2; break; }
            if ((uint64_t)dist[v] == nd) tight[v] = 1;
        }
    }
    for (uint64_t v = 0; v < V && !rc; ++v)
        if (v != src && dist[v] != UNREACHED && !tight[v]) { *bad = v; rc = 3; }
    free(tight);
    return rc;
}

/* CC on a symmetric graph: the label is equal across every edge, label[v]
 * <= v, label[label[v]] = label[v] (so each label is a member of its own
 * class), and the number of distinct labels equals the component count. */
int or_cc_certify(uint64_t V, const uint64_t *off, const uint32_t *dst, const uint32_t *label,
                  uint64_t n_components, uint64_t *bad) {
    uint64_t roots = 0;
    for (uint64_t v = 0; v < V; ++v) {
        if (label[v] > v) { *bad = v; return 1; }
        if (label[label[v]] != label[v]) { *bad = v; return 2; }
        if (label[v] == v) ++roots;
        for (uint64_t e = off[v]; e < off[v + 1]; ++e)
            if (label[dst[e]] != label[v]) { *bad = v; return 3; }
    }
    if (roots != n_components) { *bad = roots; return 4; }
    return 0;
}

/* ----------------------------------------------- cost-model counting ---- */
/* Number of m-byte lines spanned by bytes [start, start + len): the request
 * count ceil(len/m) + am(v) of the footnote to Eq. 3, computed from the
 * physical start position and the length. */
static uint64_t lines_spanned(uint64_t start, uint64_t len, uint64_t m) {
    if (len == 0) return 0;
    return (start + len - 1) / m - start / m + 1;
}

/* For each partition i (vertex range [vb[i], vb[i+1])) and the active set
 * given as a 0/1 byte per vertex: n_act[i] = |A_i|, act_edges[i] = sum of
 * D_o(v) over A_i, lines[i] = sum over A_i of the lines each edge array
 * segment spans.  The edge arrays hold `elem_bytes`-byte entries and start
 * on an m-byte boundary; `n_arrays` arrays are read per edge. */
int or_partition_counts(uint64_t V, const uint64_t *off, const unsigned char *active,
                        uint32_t n_parts, const uint64_t *vb, uint32_t elem_bytes, uint32_t n_arrays,
                        uint32_t m, uint64_t *n_act, uint64_t *act_edges, uint64_t *lines) {
    for (uint32_t i = 0; i < n_parts; ++i) {
        n_act[i] = act_edges[i] = lines[i] = 0;
        for (uint64_t v = vb[i]; v < vb[i + 1] && v < V; ++v) {
            if (!active[v]) continue;
            uint64_t deg = off[v + 1] - off[v];
            n_act[i] += 1;
            act_edges[i] += deg;
            lines[i] += (uint64_t)n_arrays * lines_spanned(off[v] * elem_bytes, deg * elem_bytes, m);
        }
    }
    return 0;
}
