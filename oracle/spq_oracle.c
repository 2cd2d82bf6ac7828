/*
 * Oracle for shortest-path distance queries on undirected weighted graphs.
 *
 * TEST INFRASTRUCTURE ONLY: this file is built into liboracle.so, which only the test
 * suite, the package's smoke check and the benchmark's CPU-baseline leg load.  The
 * CUDA distance-query path neither links nor calls it, and the two share no code.
 *
 * What it computes is the plain definition of the paper's Sec. 2: the length of a path
 * is the sum of its edge weights and dist(v, w) is the minimum length over all v-w
 * paths of G (infinite when none exists).  Because the paper's query method is exact
 * (its Lemma 3: Algorithm 2 returns dist(v1, v2)), this definition is the parity target
 * for every query, with no reference to the partition or to the boundary graph.
 *
 *   oracle_sssp_i64 / _f64     Dijkstra's algorithm (Dijkstra 1959, cited in Sec. 1)
 *                              from one source, binary heap, lazy deletion.
 *   oracle_pairs_i64 / _f64    the same, one run per (v, w) pair, stopping when w is
 *                              settled; OpenMP across pairs.
 *   oracle_fw_i64              plain Floyd-Warshall on a dense matrix (Sec. 4: the
 *                              distance-matrix representation, cell (i, j) = wt(i, j) or
 *                              infinity, updated in place until it holds dist(i, j)).
 *   oracle_subgraph_sssp_i64   Dijkstra restricted to the subgraph induced by a vertex
 *                              set, i.e. dist_H of Sec. 2 (used for APSP(C) checks).
 *
 * Weights must be nonnegative (the reading the paper's commented-out Sec. 2 remark and
 * its use of Dijkstra imply).  Self-loops never shorten a path and parallel edges are
 * all relaxed, so the smallest one wins, as the definition requires.
 *
 * Unreachable: ORACLE_INF_I64 (INT64_MAX) or +infinity.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_INF_I64 INT64_MAX

/* ---------------- binary min-heap of (key, vertex), lazy deletion ---------------- */

typedef struct {
    int64_t key;
    int32_t v;
} hitem_i;

typedef struct {
    hitem_i* a;
    int64_t size, cap;
} heap_i;

static int heap_i_push(heap_i* h, int64_t key, int32_t v) {
    if (h->size == h->cap) {
        int64_t nc = h->cap ? 2 * h->cap : 1024;
        hitem_i* na = (hitem_i*)realloc(h->a, (size_t)nc * sizeof(hitem_i));
        if (!na) return -1;
        h->a = na;
        h->cap = nc;
    }
    int64_t i = h->size++;
    while (i > 0) {
        int64_t p = (i - 1) / 2;
        if (h->a[p].key <= key) break;
        h->a[i] = h->a[p];
        i = p;
    }
    h->a[i].key = key;
    h->a[i].v = v;
    return 0;
}

static hitem_i heap_i_pop(heap_i* h) {
    hitem_i top = h->a[0];
    hitem_i last = h->a[--h->size];
    int64_t i = 0;
    for (;;) {
        int64_t l = 2 * i + 1;
        if (l >= h->size) break;
        int64_t c = (l + 1 < h->size && h->a[l + 1].key < h->a[l].key) ? l + 1 : l;
        if (h->a[c].key >= last.key) break;
        h->a[i] = h->a[c];
        i = c;
    }
    if (h->size > 0) h->a[i] = last;
    return top;
}

typedef struct {
    double key;
    int32_t v;
} hitem_d;

typedef struct {
    hitem_d* a;
    int64_t size, cap;
} heap_d;

static int heap_d_push(heap_d* h, double key, int32_t v) {
    if (h->size == h->cap) {
        int64_t nc = h->cap ? 2 * h->cap : 1024;
        hitem_d* na = (hitem_d*)realloc(h->a, (size_t)nc * sizeof(hitem_d));
        if (!na) return -1;
        h->a = na;
        h->cap = nc;
    }
    int64_t i = h->size++;
    while (i > 0) {
        int64_t p = (i - 1) / 2;
        if (h->a[p].key <= key) break;
        h->a[i] = h->a[p];
        i = p;
    }
    h->a[i].key = key;
    h->a[i].v = v;
    return 0;
}

static hitem_d heap_d_pop(heap_d* h) {
    hitem_d top = h->a[0];
    hitem_d last = h->a[--h->size];
    int64_t i = 0;
    for (;;) {
        int64_t l = 2 * i + 1;
        if (l >= h->size) break;
        int64_t c = (l + 1 < h->size && h->a[l + 1].key < h->a[l].key) ? l + 1 : l;
        if (h->a[c].key >= last.key) break;
        h->a[i] = h->a[c];
        i = c;
    }
    if (h->size > 0) h->a[i] = last;
    return top;
}

/* ---------------- Dijkstra, integer weights ---------------- */

/* One Dijkstra run.  dist[] must hold ORACLE_INF_I64 everywhere on entry; every vertex
 * whose entry it changes is appended to touched[] (so the caller can reset cheaply).
 * mask (may be NULL): only vertices with mask[v] == mask_val are part of the graph.
 * Stops early once `target` (>= 0) is settled.  Returns the number of touched
 * vertices, or -1 on allocation failure. */
static int64_t dijkstra_i64(int32_t n, const int64_t* row_ptr, const int32_t* col, const int64_t* w,
                            int32_t src, int32_t target, const int32_t* mask, int32_t mask_val,
                            int64_t* dist, int32_t* touched, heap_i* h) {
    (void)n;
    int64_t nt = 0;
    h->size = 0;
    dist[src] = 0;
    touched[nt++] = src;
    if (heap_i_push(h, 0, src)) return -1;
    while (h->size > 0) {
        hitem_i it = heap_i_pop(h);
        int32_t u = it.v;
        if (it.key != dist[u]) continue; /* stale entry */
        if (u == target) break;
        for (int64_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e) {
            int32_t x = col[e];
            if (mask && mask[x] != mask_val) continue;
            int64_t nd = it.key + w[e];
            if (nd < dist[x]) {
                if (dist[x] == ORACLE_INF_I64) touched[nt++] = x;
                dist[x] = nd;
                if (heap_i_push(h, nd, x)) return -1;
            }
        }
    }
    return nt;
}

static int has_negative_i64(int64_t m, const int64_t* w) {
    for (int64_t e = 0; e < m; ++e)
        if (w[e] < 0) return 1;
    return 0;
}

/* Single-source distances from src to every vertex.  Returns 0, or -1 on bad input. */
int oracle_sssp_i64(int32_t n, const int64_t* row_ptr, const int32_t* col, const int64_t* w, int32_t src,
                    int64_t* dist) {
    if (n <= 0 || src < 0 || src >= n || has_negative_i64(row_ptr[n], w)) return -1;
    for (int32_t v = 0; v < n; ++v) dist[v] = ORACLE_INF_I64;
    int32_t* touched = (int32_t*)malloc((size_t)n * sizeof(int32_t));
    heap_i h = {0, 0, 0};
    int64_t r = touched ? dijkstra_i64(n, row_ptr, col, w, src, -1, NULL, 0, dist, touched, &h) : -1;
    free(touched);
    free(h.a);
    return r < 0 ? -1 : 0;
}

/* dist_H from src, H = subgraph induced by {v : mask[v] == mask_val} (Sec. 2). */
int oracle_subgraph_sssp_i64(int32_t n, const int64_t* row_ptr, const int32_t* col, const int64_t* w,
                             const int32_t* mask, int32_t mask_val, int32_t src, int64_t* dist) {
    if (n <= 0 || src < 0 || src >= n || mask[src] != mask_val || has_negative_i64(row_ptr[n], w)) return -1;
    for (int32_t v = 0; v < n; ++v) dist[v] = ORACLE_INF_I64;
    int32_t* touched = (int32_t*)malloc((size_t)n * sizeof(int32_t));
    heap_i h = {0, 0, 0};
    int64_t r = touched ? dijkstra_i64(n, row_ptr, col, w, src, -1, mask, mask_val, dist, touched, &h) : -1;
    free(touched);
    free(h.a);
    return r < 0 ? -1 : 0;
}

/* Many single-source runs, one output row of n distances per source (OpenMP). */
int oracle_multi_sssp_i64(int32_t n, const int64_t* row_ptr, const int32_t* col, const int64_t* w,
                          int64_t ns, const int32_t* srcs, int64_t* out, int32_t nthreads) {
    if (n <= 0 || has_negative_i64(row_ptr[n], w)) return -1;
    for (int64_t i = 0; i < ns; ++i)
        if (srcs[i] < 0 || srcs[i] >= n) return -1;
    int err = 0;
#ifdef _OPENMP
    if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads)
#endif
    for (int64_t i = 0; i < ns; ++i) {
        if (oracle_sssp_i64(n, row_ptr, col, w, srcs[i], out + i * (int64_t)n)) {
#ifdef _OPENMP
#pragma omp atomic write
#endif
            err = 1;
        }
    }
    return err ? -1 : 0;
}

/* dist(v, w) for each pair, early exit at w; OpenMP across pairs. */
int oracle_pairs_i64(int32_t n, const int64_t* row_ptr, const int32_t* col, const int64_t* w, int64_t q,
                     const int32_t* pairs, int64_t* out, int32_t nthreads) {
    if (n <= 0 || has_negative_i64(row_ptr[n], w)) return -1;
    for (int64_t i = 0; i < 2 * q; ++i)
        if (pairs[i] < 0 || pairs[i] >= n) return -1;
    int err = 0;
#ifdef _OPENMP
    if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel num_threads(nthreads)
#endif
    {
        int64_t* dist = (int64_t*)malloc((size_t)n * sizeof(int64_t));
        int32_t* touched = (int32_t*)malloc((size_t)n * sizeof(int32_t));
        heap_i h = {0, 0, 0};
        if (!dist || !touched) {
            err = 1;
        } else {
            for (int32_t v = 0; v < n; ++v) dist[v] = ORACLE_INF_I64;
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 16)
#endif
            for (int64_t i = 0; i < q; ++i) {
                int32_t s = pairs[2 * i], t = pairs[2 * i + 1];
                int64_t nt = dijkstra_i64(n, row_ptr, col, w, s, t, NULL, 0, dist, touched, &h);
                if (nt < 0) {
                    err = 1;
                    out[i] = ORACLE_INF_I64;
                    continue;
                }
                out[i] = dist[t];
                for (int64_t j = 0; j < nt; ++j) dist[touched[j]] = ORACLE_INF_I64;
            }
        }
        free(dist);
        free(touched);
        free(h.a);
    }
    return err ? -1 : 0;
}

/* ---------------- Dijkstra, floating-point weights (computed in double) ---------------- */

static int64_t dijkstra_f64(const int64_t* row_ptr, const int32_t* col, const double* w, int32_t src,
                            int32_t target, double* dist, int32_t* pred_edge, int32_t* touched, heap_d* h) {
    int64_t nt = 0;
    h->size = 0;
    dist[src] = 0.0;
    touched[nt++] = src;
    if (pred_edge) pred_edge[src] = -1;
    if (heap_d_push(h, 0.0, src)) return -1;
    while (h->size > 0) {
        hitem_d it = heap_d_pop(h);
        int32_t u = it.v;
        if (it.key != dist[u]) continue;
        if (u == target) break;
        for (int64_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e) {
            int32_t x = col[e];
            double nd = it.key + w[e];
            if (nd < dist[x]) {
                if (dist[x] == INFINITY) touched[nt++] = x;
                dist[x] = nd;
                if (pred_edge) pred_edge[x] = (int32_t)e;
                if (heap_d_push(h, nd, x)) return -1;
            }
        }
    }
    return nt;
}

static int bad_weights_f64(int64_t m, const double* w) {
    for (int64_t e = 0; e < m; ++e)
        if (!(w[e] >= 0.0) || isinf(w[e])) return 1;
    return 0;
}

int oracle_sssp_f64(int32_t n, const int64_t* row_ptr, const int32_t* col, const double* w, int32_t src,
                    double* dist) {
    if (n <= 0 || src < 0 || src >= n || bad_weights_f64(row_ptr[n], w)) return -1;
    for (int32_t v = 0; v < n; ++v) dist[v] = INFINITY;
    int32_t* touched = (int32_t*)malloc((size_t)n * sizeof(int32_t));
    heap_d h = {0, 0, 0};
    int64_t r = touched ? dijkstra_f64(row_ptr, col, w, src, -1, dist, NULL, touched, &h) : -1;
    free(touched);
    free(h.a);
    return r < 0 ? -1 : 0;
}

/* dist(v, w) per pair in double.  If grad and g are given, each pair's shortest path
 * (the one Dijkstra's predecessor edges give) is walked back from w to v and g[i] is
 * added to grad[e] for every directed CSR slot e on it.  On inputs where every queried
 * shortest path is unique, grad is then the derivative of sum_i g[i] * dist(v_i, w_i)
 * with respect to each slot's weight (an undirected edge's derivative is the sum over
 * its two slots).  Single-threaded when grad is requested, so the sums are ordered. */
int oracle_pairs_f64(int32_t n, const int64_t* row_ptr, const int32_t* col, const double* w, int64_t q,
                     const int32_t* pairs, double* out, const double* g, double* grad, int32_t nthreads) {
    if (n <= 0 || bad_weights_f64(row_ptr[n], w)) return -1;
    for (int64_t i = 0; i < 2 * q; ++i)
        if (pairs[i] < 0 || pairs[i] >= n) return -1;
    int64_t m = row_ptr[n];
    int err = 0;
#ifdef _OPENMP
    if (nthreads <= 0) nthreads = omp_get_max_threads();
    if (grad) nthreads = 1; /* accumulation order fixed: one thread */
#pragma omp parallel num_threads(nthreads)
#endif
    {
        double* dist = (double*)malloc((size_t)n * sizeof(double));
        int32_t* pred = (int32_t*)malloc((size_t)n * sizeof(int32_t));
        int32_t* touched = (int32_t*)malloc((size_t)n * sizeof(int32_t));
        heap_d h = {0, 0, 0};
        if (!dist || !pred || !touched) {
            err = 1;
        } else {
            for (int32_t v = 0; v < n; ++v) dist[v] = INFINITY;
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 16)
#endif
            for (int64_t i = 0; i < q; ++i) {
                int32_t s = pairs[2 * i], t = pairs[2 * i + 1];
                int64_t nt = dijkstra_f64(row_ptr, col, w, s, t, dist, pred, touched, &h);
                if (nt < 0) {
                    err = 1;
                    out[i] = INFINITY;
                    continue;
                }
                out[i] = dist[t];
                if (grad && g && dist[t] != INFINITY) {
                    int32_t x = t;
                    while (x != s) {
                        int32_t e = pred[x];
                        grad[e] += g[i];
                        /* the source end of slot e: binary search row_ptr */
                        int64_t lo = 0, hi = n;
                        while (hi - lo > 1) {
                            int64_t mid = (lo + hi) / 2;
                            if (row_ptr[mid] <= e) lo = mid; else hi = mid;
                        }
                        x = (int32_t)lo;
                    }
                }
                for (int64_t j = 0; j < nt; ++j) dist[touched[j]] = INFINITY;
            }
        }
        free(dist);
        free(pred);
        free(touched);
        free(h.a);
    }
    (void)m;
    return err ? -1 : 0;
}

/* ---------------- Floyd-Warshall on a dense matrix (Sec. 4 representation) ---------------- */

/* d: n*n row-major, d[i*n+j] = wt(i, j) or ORACLE_INF_I64; the diagonal is set to 0.
 * In place: for each intermediate k, d[i][j] = min(d[i][j], d[i][k] + d[k][j]). */
int oracle_fw_i64(int32_t n, int64_t* d) {
    if (n <= 0) return -1;
    for (int64_t i = 0; i < n; ++i) d[i * n + i] = 0;
    for (int64_t k = 0; k < n; ++k) {
        const int64_t* dk = d + k * n;
        for (int64_t i = 0; i < n; ++i) {
            int64_t dik = d[i * n + k];
            if (dik == ORACLE_INF_I64) continue;
            int64_t* di = d + i * n;
            for (int64_t j = 0; j < n; ++j) {
                if (dk[j] == ORACLE_INF_I64) continue;
                int64_t s = dik + dk[j];
                if (s < di[j]) di[j] = s;
            }
        }
    }
    return 0;
}
