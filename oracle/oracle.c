/*
 * oracle.c -- plain, slow, obviously correct CPU oracle for the online query
 * path of GATE-style graph ANNS (arXiv 2506.15986).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is compiled into liboracle.so and is
 * used by the test suite, by the smoke check and by the CPU-baseline leg of
 * the benchmark.  The product library never links, loads or calls it, and it
 * shares no code, header or table with the CUDA path.
 *
 * Row types: uint8, float32 and float64 (the last for rows dequantized from
 * int8 codes with a per-row scale: code * scale is exact in double).
 *
 * Arithmetic: every floating-point distance is accumulated in double
 * precision (or_hbkm excepted: it decides cluster memberships in float32,
 * the precision the GPU decides them in); uint8 data give integer squared
 * distances that double holds exactly (128 * 255^2 < 2^53).  or_topo_tokens
 * ranks neighbours in float32 for the same reason as or_hbkm.  Every ordering is the lexicographic order on
 * (distance, id), smaller id first on ties.
 *
 * Functions and the passages they follow:
 *   or_knn             exact k-nearest neighbours (Sec. 2.1, Problem 1 and the
 *                      recall@k definition: R is the exact top-k set)
 *   or_search          greedy best-first graph search (Sec. 2.1, Algorithm 1),
 *                      in the sorted-candidate-pool form with the readings
 *                      listed at or_search_one
 *   or_build_graph     proximity graph (Sec. 2.1, Def. 1): exact K-NN
 *                      candidates, relative-neighbourhood pruning, and a
 *                      reachability repair from the navigating node
 *   or_medoid          navigating node of the NSG-style graph (Sec. 2.1): the
 *                      base point nearest the data mean
 *   or_kmeans          Lloyd's k-means (the flat alternative to the balanced
 *                      clustering of Sec. 4.1, Def. 2 / Algorithm 2)
 *   or_hbkm            hierarchical balanced k-means (Sec. 4.1, Def. 2,
 *                      Algorithm 2) and its hubs (Def. 3), with the readings
 *                      listed at the function; float32 (see there)
 *   or_hubs            hub nodes (Sec. 4.1, Def. 3): in each cluster, the
 *                      member nearest its centroid
 *   or_topo_tokens     per-hop topology tokens of each hub from the guided
 *                      subgraph walk of Sec. 4.2 (float32, see there)
 *   or_hub_graph       high-tier hub graph (Sec. 4.3): each hub linked to its
 *                      s most cosine-similar hubs
 *   (label generation, Sec. 4.2 Def. 4, uses or_search with a target id)
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_U8 0
#define OR_F32 1
#define OR_F64 2
#define OR_L2 0
#define OR_IP 1

#define OR_OK 0
#define OR_ERR_ARG 1
#define OR_ERR_NOMEM 2
#define OR_ERR_NOSLOT 3

/* value of coordinate j of base row i, as a double */
static double base_at(const void *base, int dtype, int64_t i, int d, int j)
{
    if (dtype == OR_U8)
        return (double)((const uint8_t *)base)[i * (int64_t)d + j];
    if (dtype == OR_F64)
        return ((const double *)base)[i * (int64_t)d + j];
    return (double)((const float *)base)[i * (int64_t)d + j];
}

/* delta(q, x_i): squared Euclidean distance, or the negated inner product for
 * the maximum-inner-product metric (so that smaller is always better). */
static double delta_q(const void *base, int dtype, int metric, int64_t i, int d,
                      const double *q)
{
    double s = 0.0;
    if (metric == OR_L2) {
        for (int j = 0; j < d; ++j) {
            double t = base_at(base, dtype, i, d, j) - q[j];
            s += t * t;
        }
        return s;
    }
    for (int j = 0; j < d; ++j)
        s += base_at(base, dtype, i, d, j) * q[j];
    return -s;
}

/* delta between two base rows */
static double delta_xx(const void *base, int dtype, int metric, int64_t a,
                       int64_t b, int d)
{
    double s = 0.0;
    for (int j = 0; j < d; ++j) {
        double xa = base_at(base, dtype, a, d, j);
        double xb = base_at(base, dtype, b, d, j);
        if (metric == OR_L2)
            s += (xa - xb) * (xa - xb);
        else
            s += xa * xb;
    }
    return metric == OR_L2 ? s : -s;
}

/* strict lexicographic (dist, id) order */
static int key_less(double da, int32_t ia, double db, int32_t ib)
{
    return da < db || (da == db && ia < ib);
}

/* ------------------------------------------------------------------------ */
/* Exact k-NN (Problem 1; recall@k uses this set as ground truth).           */
/* For every query: compute delta to all n base rows, keep the k smallest by  */
/* (dist, id).  exclude[qi] >= 0 removes that base id (used when the query is */
/* itself a base point).  Missing slots (k > n) are (-1, +inf).               */
/* ------------------------------------------------------------------------ */
int or_knn(const void *base, int64_t n, int d, int dtype, int metric,
           const double *queries, int64_t nq, int k, const int32_t *exclude,
           int32_t *out_ids, double *out_dists, int nthreads)
{
    if (!base || !queries || !out_ids || !out_dists || n <= 0 || d <= 0 || k <= 0)
        return OR_ERR_ARG;
    int err = 0;
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads > 0 ? nthreads : 1)
    for (int64_t qi = 0; qi < nq; ++qi) {
        double *bd = (double *)malloc(sizeof(double) * (size_t)k);
        int32_t *bi = (int32_t *)malloc(sizeof(int32_t) * (size_t)k);
        if (!bd || !bi) {
            free(bd);
            free(bi);
            err = 1;
            continue;
        }
        int cnt = 0;
        const double *q = queries + qi * (int64_t)d;
        int32_t ex = exclude ? exclude[qi] : -1;
        for (int64_t i = 0; i < n; ++i) {
            if (i == ex)
                continue;
            double di = delta_q(base, dtype, metric, i, d, q);
            if (cnt == k && !key_less(di, (int32_t)i, bd[k - 1], bi[k - 1]))
                continue;
            /* insertion into the sorted best list */
            int pos = cnt < k ? cnt : k - 1;
            while (pos > 0 && key_less(di, (int32_t)i, bd[pos - 1], bi[pos - 1])) {
                bd[pos] = bd[pos - 1];
                bi[pos] = bi[pos - 1];
                --pos;
            }
            bd[pos] = di;
            bi[pos] = (int32_t)i;
            if (cnt < k)
                ++cnt;
        }
        for (int j = 0; j < k; ++j) {
            out_ids[qi * k + j] = j < cnt ? bi[j] : -1;
            out_dists[qi * k + j] = j < cnt ? bd[j] : INFINITY;
        }
        free(bd);
        free(bi);
    }
    return err ? OR_ERR_NOMEM : OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Greedy best-first graph search (Sec. 2.1, Algorithm 1).                   */
/*                                                                          */
/* Algorithm 1 keeps a min-heap Q of candidates resized to l_s and a max-heap */
/* R of results resized to k.  This oracle keeps the same information as one */
/* pool P sorted by (dist, id) and truncated to L (= l_s); the first k entries */
/* of P are R.  Readings of the passages the algorithm leaves open:          */
/*  - initial pool: the single given entry node (no random sample);          */
/*  - a node joins the visited set when its distance is computed, so each    */
/*    node is evaluated at most once per query; 'evals' counts these          */
/*    evaluations, the entry included;                                       */
/*  - one step takes the first W not-yet-expanded entries of P in pool order, */
/*    marks them expanded ('hops' += their number), and evaluates every       */
/*    unvisited neighbour (entries in pool order, neighbours in stored        */
/*    order), inserting each into P and truncating P to L;                   */
/*  - the search stops when P has no unexpanded entry;                       */
/*  - a negative id in an adjacency row is padding and is skipped.           */
/* Label mode (target >= 0, Sec. 4.2 Def. 4): after the entry evaluation and */
/* after every step, if the target has been evaluated the search stops and   */
/* reports the evals and hops counted so far; if it never is, both counters  */
/* are INT32_MAX.                                                            */
/* ------------------------------------------------------------------------ */
typedef struct {
    double *pd;
    int32_t *pi;
    uint8_t *px; /* expanded flag */
    int cnt, cap;
} or_pool;

static void pool_insert(or_pool *P, double d, int32_t id)
{
    int pos = P->cnt;
    while (pos > 0 && key_less(d, id, P->pd[pos - 1], P->pi[pos - 1]))
        --pos;
    if (pos >= P->cap)
        return; /* worse than every kept entry of a full pool */
    int last = P->cnt < P->cap ? P->cnt : P->cap - 1;
    for (int j = last; j > pos; --j) {
        P->pd[j] = P->pd[j - 1];
        P->pi[j] = P->pi[j - 1];
        P->px[j] = P->px[j - 1];
    }
    P->pd[pos] = d;
    P->pi[pos] = id;
    P->px[pos] = 0;
    if (P->cnt < P->cap)
        P->cnt++;
}

static void or_search_one(const void *base, int64_t n, int d, int dtype,
                          int metric, const int32_t *graph, int R,
                          const double *q, const int32_t *seeds, int m, int L, int k, int W,
                          int32_t target, uint8_t *visited, int32_t *touched,
                          or_pool *P, int32_t *sel, int32_t *out_ids,
                          double *out_dists, int32_t *out_evals,
                          int32_t *out_hops)
{
    int64_t nt = 0;
    int64_t evals = 0, hops = 0;
    int done_target = 0;
    P->cnt = 0;
    P->cap = L;
    /* the initial pool: every distinct seed (Algorithm 1 starts from a set of
     * nodes; -1 marks an unused seed slot) */
    for (int e = 0; e < m; ++e) {
        const int32_t s = seeds[e];
        if (s < 0 || visited[s])
            continue;
        visited[s] = 1;
        touched[nt++] = s;
        pool_insert(P, delta_q(base, dtype, metric, s, d, q), s);
        evals++;
    }
    if (target >= 0 && visited[target])
        done_target = 1;
    while (!done_target) {
        int ns = 0;
        for (int i = 0; i < P->cnt && ns < W; ++i) {
            if (!P->px[i]) {
                P->px[i] = 1;
                sel[ns++] = P->pi[i];
            }
        }
        if (ns == 0)
            break;
        hops += ns;
        for (int s = 0; s < ns; ++s) {
            const int32_t *row = graph + (int64_t)sel[s] * R;
            for (int j = 0; j < R; ++j) {
                int32_t nb = row[j];
                if (nb < 0 || nb >= n || visited[nb])
                    continue;
                visited[nb] = 1;
                touched[nt++] = nb;
                evals++;
                pool_insert(P, delta_q(base, dtype, metric, nb, d, q), nb);
            }
        }
        if (target >= 0 && visited[target])
            done_target = 1;
    }
    for (int j = 0; j < k; ++j) {
        out_ids[j] = j < P->cnt ? P->pi[j] : -1;
        out_dists[j] = j < P->cnt ? P->pd[j] : INFINITY;
    }
    if (target >= 0 && !done_target) {
        evals = INT32_MAX;
        hops = INT32_MAX;
    }
    *out_evals = (int32_t)(evals > INT32_MAX ? INT32_MAX : evals);
    *out_hops = (int32_t)(hops > INT32_MAX ? INT32_MAX : hops);
    for (int64_t t = 0; t < nt; ++t)
        visited[touched[t]] = 0;
}

/*
 * Batch driver.  Per query i: seeds entries[i*m .. i*m+m) (-1 = unused, at
 * least one node id); pool size Ls ? Ls[i] : L;
 * result size ks ? ks[i] : k (rows of out_ids/out_dists have stride kstride);
 * target targets ? targets[i] : -1.  Queries run in parallel, one per thread.
 */
int or_search(const void *base, int64_t n, int d, int dtype, int metric,
              const int32_t *graph, int R, const double *queries, int64_t nq,
              const int32_t *entries, int m, int L, int k, const int32_t *Ls,
              const int32_t *ks, int kstride, int W, const int32_t *targets,
              int32_t *out_ids, double *out_dists, int32_t *out_evals,
              int32_t *out_hops, int nthreads)
{
    if (!base || !graph || !queries || !entries || !out_ids || !out_dists ||
        !out_evals || !out_hops || n <= 0 || d <= 0 || R <= 0 || W <= 0 ||
        kstride <= 0 || m <= 0)
        return OR_ERR_ARG;
    for (int64_t i = 0; i < nq; ++i) {
        int Li = Ls ? Ls[i] : L, ki = ks ? ks[i] : k;
        int valid = 0;
        for (int e = 0; e < m; ++e) {
            const int32_t s = entries[i * (int64_t)m + e];
            if (s < -1 || s >= n)
                return OR_ERR_ARG;
            valid += s >= 0;
        }
        if (!valid || Li <= 0 || ki <= 0 || ki > Li || ki > kstride)
            return OR_ERR_ARG;
    }
    int err = 0;
#pragma omp parallel num_threads(nthreads > 0 ? nthreads : 1)
    {
        uint8_t *visited = (uint8_t *)calloc((size_t)n, 1);
        int32_t *touched = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
        int Lmax = L;
        if (Ls)
            for (int64_t i = 0; i < nq; ++i)
                if (Ls[i] > Lmax)
                    Lmax = Ls[i];
        or_pool P;
        P.pd = (double *)malloc(sizeof(double) * (size_t)Lmax);
        P.pi = (int32_t *)malloc(sizeof(int32_t) * (size_t)Lmax);
        P.px = (uint8_t *)malloc((size_t)Lmax);
        int32_t *sel = (int32_t *)malloc(sizeof(int32_t) * (size_t)W);
        double *dtmp = (double *)malloc(sizeof(double) * (size_t)kstride);
        if (!visited || !touched || !P.pd || !P.pi || !P.px || !sel || !dtmp) {
#pragma omp atomic write
            err = 1;
        } else {
#pragma omp for schedule(dynamic, 1)
            for (int64_t i = 0; i < nq; ++i) {
                int Li = Ls ? Ls[i] : L, ki = ks ? ks[i] : k;
                int32_t *oi = out_ids + i * (int64_t)kstride;
                double *od = out_dists + i * (int64_t)kstride;
                or_search_one(base, n, d, dtype, metric, graph, R,
                              queries + i * (int64_t)d, entries + i * (int64_t)m, m, Li, ki, W,
                              targets ? targets[i] : -1, visited, touched, &P,
                              sel, oi, od, out_evals + i, out_hops + i);
                for (int j = ki; j < kstride; ++j) {
                    oi[j] = -1;
                    od[j] = INFINITY;
                }
            }
        }
        free(visited);
        free(touched);
        free(P.pd);
        free(P.pi);
        free(P.px);
        free(sel);
        free(dtmp);
    }
    return err ? OR_ERR_NOMEM : OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Navigating node (Sec. 2.1, NSG): argmin_i ||x_i - mean||^2, smaller id on */
/* ties.  uint8 data are handled exactly in integers as ||n x_i - sum x||^2.  */
/* ------------------------------------------------------------------------ */
int32_t or_medoid(const void *base, int64_t n, int d, int dtype)
{
    if (!base || n <= 0 || d <= 0)
        return -1;
    int32_t best = -1;
    if (dtype == OR_U8) {
        const uint8_t *x = (const uint8_t *)base;
        int64_t *sum = (int64_t *)calloc((size_t)d, sizeof(int64_t));
        if (!sum)
            return -1;
        for (int64_t i = 0; i < n; ++i)
            for (int j = 0; j < d; ++j)
                sum[j] += x[i * d + j];
        unsigned __int128 bestv = 0;
        for (int64_t i = 0; i < n; ++i) {
            unsigned __int128 s = 0;
            for (int j = 0; j < d; ++j) {
                int64_t t = n * (int64_t)x[i * d + j] - sum[j];
                s += (unsigned __int128)((__int128)t * t);
            }
            if (best < 0 || s < bestv) {
                bestv = s;
                best = (int32_t)i;
            }
        }
        free(sum);
        return best;
    }
    double *mean = (double *)calloc((size_t)d, sizeof(double));
    if (!mean)
        return -1;
    for (int64_t i = 0; i < n; ++i)
        for (int j = 0; j < d; ++j)
            mean[j] += base_at(base, dtype, i, d, j);
    for (int j = 0; j < d; ++j)
        mean[j] /= (double)n;
    double bestv = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        double s = delta_q(base, dtype, OR_L2, i, d, mean);
        if (best < 0 || s < bestv) {
            bestv = s;
            best = (int32_t)i;
        }
    }
    free(mean);
    return best;
}

/* ------------------------------------------------------------------------ */
/* Proximity graph (Sec. 2.1, Def. 1), squared L2 only.                      */
/*  1. candidates of node p: its K exact nearest other nodes by (dist, id);  */
/*  2. relative-neighbourhood pruning in candidate order: c is kept unless a */
/*     node s kept before it has alpha * delta(s, c) <= delta(p, c); stop at */
/*     R kept; the row is padded with -1;                                    */
/*  3. reachability repair from the navigating node 'root': nodes are      */
/*     taken in id order; a node u that is not reachable from root at its    */
/*     turn gets the edge w -> u from the node w nearest to u, by (dist, id), */
/*     among the reachable nodes whose row has a free slot; the edge goes to */
/*     w's first free slot, and everything reachable from u becomes          */
/*     reachable before the next node is taken.  Afterwards every node is    */
/*     reachable from root.                                                  */
/* Steps 1-2 alone run when root < 0.  pre_repair (optional, n*R) receives   */
/* the rows after step 2.  Returns the number of repair edges (>= 0) or      */
/* -OR_ERR_*.                                                                */
/* ------------------------------------------------------------------------ */
int64_t or_build_graph(const void *base, int64_t n, int d, int dtype, int K,
                       int R, double alpha, int32_t root, int32_t *graph,
                       int32_t *pre_repair, int nthreads)
{
    if (!base || !graph || n <= 1 || d <= 0 || K <= 0 || R <= 0)
        return -OR_ERR_ARG;
    if (K > n - 1)
        K = (int)(n - 1);
    int err = 0;
#pragma omp parallel num_threads(nthreads > 0 ? nthreads : 1)
    {
        double *q = (double *)malloc(sizeof(double) * (size_t)d);
        double *cd = (double *)malloc(sizeof(double) * (size_t)K);
        int32_t *ci = (int32_t *)malloc(sizeof(int32_t) * (size_t)K);
        if (!q || !cd || !ci) {
#pragma omp atomic write
            err = 1;
        } else {
#pragma omp for schedule(dynamic, 16)
            for (int64_t p = 0; p < n; ++p) {
                for (int j = 0; j < d; ++j)
                    q[j] = base_at(base, dtype, p, d, j);
                int32_t ex = (int32_t)p;
                or_knn(base, n, d, dtype, OR_L2, q, 1, K, &ex, ci, cd, 1);
                int32_t *row = graph + p * (int64_t)R;
                int kept = 0;
                for (int c = 0; c < K && kept < R; ++c) {
                    if (ci[c] < 0)
                        break;
                    int ok = 1;
                    for (int s = 0; s < kept; ++s) {
                        double dsc = delta_xx(base, dtype, OR_L2, row[s], ci[c], d);
                        if (alpha * dsc <= cd[c]) {
                            ok = 0;
                            break;
                        }
                    }
                    if (ok)
                        row[kept++] = ci[c];
                }
                for (int j = kept; j < R; ++j)
                    row[j] = -1;
            }
        }
        free(q);
        free(cd);
        free(ci);
    }
    if (err)
        return -OR_ERR_NOMEM;
    if (pre_repair)
        memcpy(pre_repair, graph, sizeof(int32_t) * (size_t)(n * R));
    if (root < 0)
        return 0;
    /* breadth-first reachability from root */
    uint8_t *reached = (uint8_t *)calloc((size_t)n, 1);
    int32_t *queue = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int32_t *deg = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    if (!reached || !queue || !deg) {
        free(reached);
        free(queue);
        free(deg);
        return -OR_ERR_NOMEM;
    }
    int64_t head = 0, tail = 0;
    reached[root] = 1;
    queue[tail++] = root;
    while (head < tail) {
        int32_t v = queue[head++];
        for (int j = 0; j < R; ++j) {
            int32_t u = graph[(int64_t)v * R + j];
            if (u >= 0 && !reached[u]) {
                reached[u] = 1;
                queue[tail++] = u;
            }
        }
    }
    for (int64_t v = 0; v < n; ++v) {
        int c = 0;
        while (c < R && graph[v * R + c] >= 0)
            ++c;
        deg[v] = c;
    }
    int64_t added = 0;
    for (int64_t u = 0; u < n; ++u) {
        if (reached[u])
            continue;
        int32_t bw = -1;
        double bd = 0.0;
        for (int64_t w = 0; w < n; ++w) {
            if (!reached[w] || deg[w] >= R)
                continue;
            double dw = delta_xx(base, dtype, OR_L2, w, u, d);
            if (bw < 0 || key_less(dw, (int32_t)w, bd, bw)) {
                bw = (int32_t)w;
                bd = dw;
            }
        }
        if (bw < 0) {
            free(reached);
            free(queue);
            free(deg);
            return -OR_ERR_NOSLOT;
        }
        graph[(int64_t)bw * R + deg[bw]] = (int32_t)u;
        deg[bw]++;
        added++;
        /* extend the reachable set by everything reachable from u */
        head = tail = 0;
        reached[u] = 1;
        queue[tail++] = (int32_t)u;
        while (head < tail) {
            int32_t v = queue[head++];
            for (int j = 0; j < R; ++j) {
                int32_t x = graph[(int64_t)v * R + j];
                if (x >= 0 && !reached[x]) {
                    reached[x] = 1;
                    queue[tail++] = x;
                }
            }
        }
    }
    free(reached);
    free(queue);
    free(deg);
    return added;
}

/* ------------------------------------------------------------------------ */
/* Lloyd's k-means on m sample rows (a flat stand-in for Algorithm 2):       */
/*   centroids start at the sample rows init[0..k-1] (drawn by the caller);  */
/*   each of T iterations assigns every row to its nearest centroid by       */
/*   (squared L2, centroid index), then moves each centroid to the mean of   */
/*   its rows; a centroid left with no row is moved onto the row farthest    */
/*   from its own centroid (larger distance first, smaller row on ties),     */
/*   each row used at most once per iteration.                               */
/* objective[t] = sum of squared distances of the assignment of iteration t. */
/* ------------------------------------------------------------------------ */
static int32_t nearest_centroid(const double *cent, int k, int d,
                                const void *x, int dtype, int64_t i,
                                double *out_d)
{
    int32_t bj = -1;
    double bd = 0.0;
    for (int j = 0; j < k; ++j) {
        double s = 0.0;
        for (int t = 0; t < d; ++t) {
            double v = base_at(x, dtype, i, d, t) - cent[(int64_t)j * d + t];
            s += v * v;
        }
        if (bj < 0 || s < bd) {
            bj = j;
            bd = s;
        }
    }
    *out_d = bd;
    return bj;
}

int or_kmeans(const void *x, int64_t m, int d, int dtype, int k,
              const int32_t *init, int T, double *centroids, int32_t *assign,
              double *objective, int nthreads)
{
    if (!x || !init || !centroids || !assign || m <= 0 || d <= 0 || k <= 0 || k > m)
        return OR_ERR_ARG;
    for (int j = 0; j < k; ++j)
        for (int t = 0; t < d; ++t)
            centroids[(int64_t)j * d + t] = base_at(x, dtype, init[j], d, t);
    double *dist = (double *)malloc(sizeof(double) * (size_t)m);
    int64_t *cnt = (int64_t *)malloc(sizeof(int64_t) * (size_t)k);
    uint8_t *used = (uint8_t *)malloc((size_t)m);
    if (!dist || !cnt || !used) {
        free(dist);
        free(cnt);
        free(used);
        return OR_ERR_NOMEM;
    }
    for (int it = 0; it < T; ++it) {
#pragma omp parallel for schedule(static) num_threads(nthreads > 0 ? nthreads : 1)
        for (int64_t i = 0; i < m; ++i)
            assign[i] = nearest_centroid(centroids, k, d, x, dtype, i, &dist[i]);
        double obj = 0.0;
        for (int64_t i = 0; i < m; ++i)
            obj += dist[i];
        if (objective)
            objective[it] = obj;
        memset(centroids, 0, sizeof(double) * (size_t)k * d);
        memset(cnt, 0, sizeof(int64_t) * (size_t)k);
        for (int64_t i = 0; i < m; ++i) {
            cnt[assign[i]]++;
            for (int t = 0; t < d; ++t)
                centroids[(int64_t)assign[i] * d + t] += base_at(x, dtype, i, d, t);
        }
        memset(used, 0, (size_t)m);
        for (int j = 0; j < k; ++j) {
            if (cnt[j] > 0) {
                for (int t = 0; t < d; ++t)
                    centroids[(int64_t)j * d + t] /= (double)cnt[j];
                continue;
            }
            int64_t far = -1;
            for (int64_t i = 0; i < m; ++i)
                if (!used[i] && (far < 0 || dist[i] > dist[far]))
                    far = i;
            used[far] = 1;
            for (int t = 0; t < d; ++t)
                centroids[(int64_t)j * d + t] = base_at(x, dtype, far, d, t);
        }
    }
    free(dist);
    free(cnt);
    free(used);
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Hub nodes (Sec. 4.1, Def. 3): assign every base row to its nearest        */
/* centroid (squared L2, smaller centroid index on ties); the hub of cluster */
/* j is argmin over its members of ||x - mu_j||^2 (smaller id on ties), or   */
/* -1 when the cluster has no member.  assign (optional, n) receives the     */
/* final assignment.                                                         */
/* ------------------------------------------------------------------------ */
int or_hubs(const void *base, int64_t n, int d, int dtype,
            const double *centroids, int k, int32_t *hubs, int32_t *assign,
            int nthreads)
{
    if (!base || !centroids || !hubs || n <= 0 || d <= 0 || k <= 0)
        return OR_ERR_ARG;
    int32_t *a = assign ? assign : (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    double *dist = (double *)malloc(sizeof(double) * (size_t)n);
    double *bestd = (double *)malloc(sizeof(double) * (size_t)k);
    if (!a || !dist || !bestd) {
        if (!assign)
            free(a);
        free(dist);
        free(bestd);
        return OR_ERR_NOMEM;
    }
#pragma omp parallel for schedule(static) num_threads(nthreads > 0 ? nthreads : 1)
    for (int64_t i = 0; i < n; ++i)
        a[i] = nearest_centroid(centroids, k, d, base, dtype, i, &dist[i]);
    for (int j = 0; j < k; ++j)
        hubs[j] = -1;
    for (int64_t i = 0; i < n; ++i) {
        int j = a[i];
        if (hubs[j] < 0 || dist[i] < bestd[j]) {
            hubs[j] = (int32_t)i;
            bestd[j] = dist[i];
        }
    }
    if (!assign)
        free(a);
    free(dist);
    free(bestd);
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* High-tier hub graph (Sec. 4.3): each hub i is linked to the s hubs j != i */
/* with the largest cosine similarity of their embeddings (smaller index on  */
/* ties).  entry receives the hub with the largest cosine to the mean        */
/* embedding (smaller index on ties).                                        */
/* ------------------------------------------------------------------------ */
int or_hub_graph(const double *emb, int H, int e, int s, int32_t *adj,
                 int32_t *entry)
{
    if (!emb || !adj || H <= 1 || e <= 0 || s <= 0 || s > H - 1)
        return OR_ERR_ARG;
    double *nrm = (double *)malloc(sizeof(double) * (size_t)H);
    double *cs = (double *)malloc(sizeof(double) * (size_t)H);
    double *mean = (double *)calloc((size_t)e, sizeof(double));
    if (!nrm || !cs || !mean) {
        free(nrm);
        free(cs);
        free(mean);
        return OR_ERR_NOMEM;
    }
    for (int i = 0; i < H; ++i) {
        double t = 0.0;
        for (int c = 0; c < e; ++c)
            t += emb[(int64_t)i * e + c] * emb[(int64_t)i * e + c];
        nrm[i] = sqrt(t);
    }
    for (int i = 0; i < H; ++i) {
        for (int j = 0; j < H; ++j) {
            double t = 0.0;
            for (int c = 0; c < e; ++c)
                t += emb[(int64_t)i * e + c] * emb[(int64_t)j * e + c];
            cs[j] = t / (nrm[i] * nrm[j]);
        }
        for (int r = 0; r < s; ++r) {
            int bj = -1;
            for (int j = 0; j < H; ++j) {
                if (j == i)
                    continue;
                int taken = 0;
                for (int t = 0; t < r; ++t)
                    if (adj[(int64_t)i * s + t] == j)
                        taken = 1;
                if (taken)
                    continue;
                if (bj < 0 || cs[j] > cs[bj])
                    bj = j;
            }
            adj[(int64_t)i * s + r] = bj;
        }
    }
    if (entry) {
        for (int i = 0; i < H; ++i)
            for (int c = 0; c < e; ++c)
                mean[c] += emb[(int64_t)i * e + c] / (double)H;
        double mn = 0.0;
        for (int c = 0; c < e; ++c)
            mn += mean[c] * mean[c];
        mn = sqrt(mn);
        int be = 0;
        double bv = -INFINITY;
        for (int i = 0; i < H; ++i) {
            double t = 0.0;
            for (int c = 0; c < e; ++c)
                t += emb[(int64_t)i * e + c] * mean[c];
            t /= nrm[i] * mn;
            if (t > bv) {
                bv = t;
                be = i;
            }
        }
        *entry = be;
    }
    free(nrm);
    free(cs);
    free(mean);
    return OR_OK;
}

int or_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* Hierarchical balanced k-means, HBKM (Sec. 4.1, Def. 2 and Algorithm 2),   */
/* and the hub of every final cluster (Def. 3).                              */
/*                                                                           */
/* Each of `levels` levels splits every cluster C of the level above        */
/* (level 0: the whole data set) into k children, so k^levels clusters come */
/* out.  A split runs T iterations; each iteration empties the children,     */
/* then visits C's members in increasing id and puts member x into           */
/*   j = argmin_j ||x - mu_j||^2 + lam * (2 (c_j - m) + 1)                   */
/* (ties to the smaller j), c_j the child's current size and m = |C| / k;    */
/* the penalty is the increase of Def. 2's size-variance objective           */
/* (c_j + 1 - m)^2 - (c_j - m)^2 that adding x to child j causes, and        */
/* lam = lambda * sigma^2 / m with sigma^2 the mean squared distance of C's  */
/* members to C's centroid, so that lambda carries no units.  After the      */
/* visit every non-empty child's centroid becomes the mean of its members    */
/* (an empty child keeps its centroid).  The children start at the members  */
/* with the min(k, |C|) smallest (key, id), in that order; children past |C| */
/* stay empty.  Child j of cluster c is cluster c * k + j of the next level. */
/*                                                                           */
/* Arithmetic is float32 with every operation rounded on its own (the        */
/* file's build keeps floating-point contraction off), in these orders:      */
/* distance = sum over coordinates 0..d-1 of (x_t - mu_t)^2; sigma^2 and     */
/* the centroid sums run over members in increasing id; division last.      */
/* Float32 is the precision in which the assignment (an integer) is decided. */
/*                                                                           */
/* Outputs: label[n] final cluster of every row; centroids[k^levels * d];    */
/* hubs[k^levels], the member nearest its cluster's centroid (smaller id on  */
/* ties), -1 for an empty cluster; sizes (optional) the final cluster sizes. */
/* ------------------------------------------------------------------------ */
static float hb_dist(const float *x, const float *mu, int d)
{
    float acc = 0.0f;
    for (int t = 0; t < d; ++t) {
        const float df = x[t] - mu[t];
        const float sq = df * df;
        acc = acc + sq;
    }
    return acc;
}

int or_hbkm(const float *x, int64_t n, int d, int k, int levels, double lambda, int T,
            const uint32_t *keys, int32_t *label, float *centroids, int32_t *hubs, int64_t *sizes)
{
    if (!x || !keys || !label || !centroids || !hubs || n <= 0 || d <= 0 || k < 2 || levels < 1 || T < 1 ||
        lambda < 0.0)
        return OR_ERR_ARG;
    int64_t nc = 1;
    for (int l = 0; l < levels; ++l) {
        nc *= k;
        if (nc > (int64_t)1 << 30)
            return OR_ERR_ARG;
    }
    float *cur = (float *)malloc(sizeof(float) * (size_t)d);  /* level-0 centroid */
    float *pc = NULL;                                        /* parents' centroids */
    float *cc = NULL;                                        /* children's centroids */
    int32_t *own = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int32_t *nown = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int32_t *mem = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);  /* a cluster's members */
    int32_t *chl = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);  /* their child index */
    int64_t *cnt = (int64_t *)malloc(sizeof(int64_t) * (size_t)k);
    int32_t *ini = (int32_t *)malloc(sizeof(int32_t) * (size_t)k);
    float *sum = (float *)malloc(sizeof(float) * (size_t)k * d);
    if (!cur || !own || !nown || !mem || !chl || !cnt || !ini || !sum) {
        free(cur); free(own); free(nown); free(mem); free(chl); free(cnt); free(ini); free(sum);
        return OR_ERR_NOMEM;
    }
    /* level 0: one cluster, the data set, with its mean */
    for (int t = 0; t < d; ++t) {
        float s = 0.0f;
        for (int64_t i = 0; i < n; ++i)
            s = s + x[i * (int64_t)d + t];
        cur[t] = s / (float)n;
    }
    for (int64_t i = 0; i < n; ++i)
        own[i] = 0;
    pc = cur;
    int64_t np = 1;
    int err = OR_OK;
    for (int l = 1; l <= levels && err == OR_OK; ++l) {
        cc = (float *)malloc(sizeof(float) * (size_t)(np * k) * d);
        if (!cc) {
            err = OR_ERR_NOMEM;
            break;
        }
        for (int64_t c = 0; c < np; ++c) {
            const float *mu_p = pc + c * d;
            float *mu = cc + c * k * d;
            /* members of cluster c in increasing id */
            int64_t s = 0;
            for (int64_t i = 0; i < n; ++i)
                if (own[i] == c)
                    mem[s++] = (int32_t)i;
            /* every child starts at the parent's centroid (what an empty child keeps) */
            for (int j = 0; j < k; ++j)
                memcpy(mu + (int64_t)j * d, mu_p, sizeof(float) * (size_t)d);
            if (s == 0)
                continue;
            /* penalty scale */
            float sig = 0.0f;
            for (int64_t a = 0; a < s; ++a)
                sig = sig + hb_dist(x + (int64_t)mem[a] * d, mu_p, d);
            sig = sig / (float)s;
            const float m = (float)s / (float)k;
            const float lam = ((float)lambda * sig) / m;
            /* initial centroids: the members with the smallest (key, id) */
            const int kk = s < k ? (int)s : k;
            for (int j = 0; j < kk; ++j) {
                int32_t best = -1;
                for (int64_t a = 0; a < s; ++a) {
                    const int32_t id = mem[a];
                    int taken = 0;
                    for (int q = 0; q < j; ++q)
                        taken |= ini[q] == id;
                    if (taken)
                        continue;
                    if (best < 0 || keys[id] < keys[best] || (keys[id] == keys[best] && id < best))
                        best = id;
                }
                ini[j] = best;
                memcpy(mu + (int64_t)j * d, x + (int64_t)best * d, sizeof(float) * (size_t)d);
            }
            for (int it = 0; it < T; ++it) {
                for (int j = 0; j < k; ++j)
                    cnt[j] = 0;
                for (int64_t a = 0; a < s; ++a) {
                    const float *xa = x + (int64_t)mem[a] * d;
                    int bj = -1;
                    float bc = 0.0f;
                    for (int j = 0; j < kk; ++j) {
                        const float pen = lam * (2.0f * ((float)cnt[j] - m) + 1.0f);
                        const float cost = hb_dist(xa, mu + (int64_t)j * d, d) + pen;
                        if (bj < 0 || cost < bc) {
                            bj = j;
                            bc = cost;
                        }
                    }
                    chl[a] = bj;
                    cnt[bj]++;
                }
                for (int64_t q = 0; q < (int64_t)k * d; ++q)
                    sum[q] = 0.0f;
                for (int64_t a = 0; a < s; ++a)
                    for (int t = 0; t < d; ++t)
                        sum[(int64_t)chl[a] * d + t] = sum[(int64_t)chl[a] * d + t] + x[(int64_t)mem[a] * d + t];
                for (int j = 0; j < kk; ++j)
                    if (cnt[j] > 0)
                        for (int t = 0; t < d; ++t)
                            mu[(int64_t)j * d + t] = sum[(int64_t)j * d + t] / (float)cnt[j];
            }
            for (int64_t a = 0; a < s; ++a)
                nown[mem[a]] = (int32_t)(c * k + chl[a]);
        }
        memcpy(own, nown, sizeof(int32_t) * (size_t)n);
        if (pc != cur)
            free(pc);
        pc = cc;
        cc = NULL;
        np *= k;
    }
    if (err == OR_OK) {
        memcpy(centroids, pc, sizeof(float) * (size_t)nc * d);
        for (int64_t c = 0; c < nc; ++c) {
            hubs[c] = -1;
            if (sizes)
                sizes[c] = 0;
        }
        float *hd = (float *)malloc(sizeof(float) * (size_t)nc);
        if (!hd) {
            err = OR_ERR_NOMEM;
        } else {
            for (int64_t i = 0; i < n; ++i) {
                const int64_t c = own[i];
                label[i] = (int32_t)c;
                if (sizes)
                    sizes[c]++;
                const float di = hb_dist(x + i * (int64_t)d, pc + c * d, d);
                if (hubs[c] < 0 || di < hd[c]) {  /* increasing id: the first of equals stays */
                    hubs[c] = (int32_t)i;
                    hd[c] = di;
                }
            }
            free(hd);
        }
    }
    if (pc != cur)
        free(pc);
    free(cc); free(cur); free(own); free(nown); free(mem); free(chl); free(cnt); free(ini); free(sum);
    return err;
}

/* ------------------------------------------------------------------------ */
/* Topology tokens of a hub (Sec. 4.2, subgraph sampling, with a fixed-size  */
/* per-hop summary standing in for Graph2Vec).                               */
/*                                                                           */
/* The guided walk: MinDeg and MaxDeg are the smallest and largest numbers   */
/* of valid neighbours over all nodes of G.  A FIFO queue starts with the   */
/* hub at hop 0.  A dequeued node u at hop < h ranks its deg(u) valid        */
/* neighbours by (squared L2 to u, id) and samples the ceil(x/2) nearest and */
/* the floor(x/2) farthest, x = ceil(MinDeg * deg(u) / MaxDeg); each sampled */
/* neighbour not yet in the subgraph joins it (in rank order) at hop(u) + 1  */
/* with parent u, and is queued.  Nodes at hop h join but are not expanded;  */
/* the subgraph stops growing at max_nodes nodes.                            */
/*                                                                           */
/* Token l (0..h) summarises the nodes at hop l, with s the hub's mean       */
/* squared distance to its valid neighbours (1 if it has none or it is 0):   */
/*   u0 = count / total nodes          u4 = mean d2(w, parent) / s           */
/*   u1 = mean deg / MaxDeg            u5 = share sampled as farthest        */
/*   u2 = mean d2(w, hub) / s          u6 = l / h                            */
/*   u3 = max d2(w, hub) / s           u7 = 1                                */
/* (u0..u5 are 0 for an empty hop).  float32 as in or_hbkm: distances summed */
/* over coordinates 0..d-1, means over the hop's nodes in joining order, one */
/* division at the end; the ranking (an integer decision) uses the same     */
/* float32 distances the GPU ranks by.                                       */
/*                                                                           */
/* tokens: H * (h+1) * 8 floats; nodes (optional): H subgraph sizes.         */
/* ------------------------------------------------------------------------ */
#define OR_TOKEN_DIM 8

static float tp_dist(const float *x, int d, int64_t a, int64_t b)
{
    return hb_dist(x + a * (int64_t)d, x + b * (int64_t)d, d);
}

int or_topo_tokens(const float *x, int64_t n, int d, const int32_t *graph, int R, const int32_t *hubs, int H,
                   int h, int max_nodes, float *tokens, int32_t *nodes)
{
    if (!x || !graph || !hubs || !tokens || n <= 0 || d <= 0 || R <= 0 || H <= 0 || h < 1 || max_nodes < 1)
        return OR_ERR_ARG;
    int mindeg = R, maxdeg = 0;
    for (int64_t u = 0; u < n; ++u) {
        int dg = 0;
        for (int r = 0; r < R; ++r)
            dg += graph[u * R + r] >= 0;
        mindeg = dg < mindeg ? dg : mindeg;
        maxdeg = dg > maxdeg ? dg : maxdeg;
    }
    int32_t *node = (int32_t *)malloc(sizeof(int32_t) * (size_t)max_nodes);
    int32_t *hop = (int32_t *)malloc(sizeof(int32_t) * (size_t)max_nodes);
    int32_t *par = (int32_t *)malloc(sizeof(int32_t) * (size_t)max_nodes);
    uint8_t *far = (uint8_t *)malloc((size_t)max_nodes);
    int32_t *nb = (int32_t *)malloc(sizeof(int32_t) * (size_t)R);
    float *nd = (float *)malloc(sizeof(float) * (size_t)R);
    if (!node || !hop || !par || !far || !nb || !nd) {
        free(node); free(hop); free(par); free(far); free(nb); free(nd);
        return OR_ERR_NOMEM;
    }
    for (int v = 0; v < H; ++v) {
        const int32_t hub = hubs[v];
        float *tok = tokens + (int64_t)v * (h + 1) * OR_TOKEN_DIM;
        if (hub < 0 || hub >= n) {
            free(node); free(hop); free(par); free(far); free(nb); free(nd);
            return OR_ERR_ARG;
        }
        int cnt = 1, head = 0;
        node[0] = hub; hop[0] = 0; par[0] = -1; far[0] = 0;
        while (head < cnt) {
            const int32_t u = node[head];
            const int hu = hop[head];
            ++head;
            if (hu >= h)
                continue;
            int dg = 0;
            for (int r = 0; r < R; ++r)
                if (graph[(int64_t)u * R + r] >= 0) {
                    nb[dg] = graph[(int64_t)u * R + r];
                    nd[dg] = tp_dist(x, d, u, nb[dg]);
                    ++dg;
                }
            /* rank by (distance, id): insertion sort */
            for (int a = 1; a < dg; ++a) {
                const int32_t ib = nb[a];
                const float db = nd[a];
                int b = a;
                while (b > 0 && (nd[b - 1] > db || (nd[b - 1] == db && nb[b - 1] > ib))) {
                    nb[b] = nb[b - 1];
                    nd[b] = nd[b - 1];
                    --b;
                }
                nb[b] = ib;
                nd[b] = db;
            }
            const int xs = maxdeg > 0 ? (mindeg * dg + maxdeg - 1) / maxdeg : 0;
            const int near_n = (xs + 1) / 2, far_n = xs / 2;
            for (int a = 0; a < dg && cnt < max_nodes; ++a) {
                const int is_far = a >= dg - far_n;
                if (a >= near_n && !is_far)
                    continue;
                int seen = 0;
                for (int q = 0; q < cnt && !seen; ++q)
                    seen = node[q] == nb[a];
                if (seen)
                    continue;
                node[cnt] = nb[a]; hop[cnt] = hu + 1; par[cnt] = u; far[cnt] = (uint8_t)is_far;
                ++cnt;
            }
        }
        if (nodes)
            nodes[v] = cnt;
        /* scale: the hub's mean squared distance to its valid neighbours */
        float ssum = 0.0f;
        int sdeg = 0;
        for (int r = 0; r < R; ++r) {
            const int32_t w = graph[(int64_t)hub * R + r];
            if (w >= 0) {
                ssum = ssum + tp_dist(x, d, hub, w);
                ++sdeg;
            }
        }
        float s = sdeg > 0 ? ssum / (float)sdeg : 1.0f;
        if (!(s > 0.0f))
            s = 1.0f;
        for (int l = 0; l <= h; ++l) {
            float *t = tok + l * OR_TOKEN_DIM;
            int c = 0, fars = 0;
            int64_t degsum = 0;
            float dh = 0.0f, dmax = 0.0f, dpar = 0.0f;
            for (int q = 0; q < cnt; ++q) {
                if (hop[q] != l)
                    continue;
                const float a = tp_dist(x, d, node[q], hub) / s;
                const float b = par[q] >= 0 ? tp_dist(x, d, node[q], par[q]) / s : 0.0f;
                int dg = 0;
                for (int r = 0; r < R; ++r)
                    dg += graph[(int64_t)node[q] * R + r] >= 0;
                ++c;
                degsum += dg;
                fars += far[q];
                dh = dh + a;
                dmax = a > dmax ? a : dmax;
                dpar = dpar + b;
            }
            for (int f = 0; f < OR_TOKEN_DIM; ++f)
                t[f] = 0.0f;
            if (c > 0) {
                t[0] = (float)c / (float)cnt;
                t[1] = maxdeg > 0 ? (float)degsum / ((float)c * (float)maxdeg) : 0.0f;
                t[2] = dh / (float)c;
                t[3] = dmax;
                t[4] = dpar / (float)c;
                t[5] = (float)fars / (float)c;
            }
            t[6] = (float)l / (float)h;
            t[7] = 1.0f;
        }
    }
    free(node); free(hop); free(par); free(far); free(nb); free(nd);
    return OR_OK;
}
