/*
 * htd_oracle.c -- plain, slow, single-threaded CPU oracle for higher-order (k,h)-truss
 * decomposition (Chen et al., "Parallel Higher-order Truss Decomposition", 2024).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the benchmark's CPU
 * baseline leg load this library.  It shares no code, header or table with the CUDA
 * path and must never be used as a fallback for it.
 *
 * Everything here follows the paper's definitions literally:
 *   - N_G(v,h): vertices within distance h of v, v itself excluded (Sec. 2).
 *   - common h-neighbours and h-support sup_G(e,h) = |N_G(u,h) ∩ N_G(v,h)| (Def. 2, Def. 3).
 *   - (k,h)-truss: maximal edge set S with sup_S(e,h) >= k-2 for every e in S (Def. 4);
 *     t(e,h) = largest such k.
 *   - peeling from k = 2 upward, removing edges whose h-support is <= k-2 (Sec. 3,
 *     Lemma 1, Algorithm 1).
 * Readings where the paper is silent or garbled (the build's design notes list them):
 *   - a subgraph is an edge set; distances inside it use only its edges (Algorithm 1
 *     deletes single edges);
 *   - a path through the edge e itself counts when measuring sup_S(e,h) (e is in S);
 *   - "within distance h" means dist <= h;
 *   - input hygiene: self-loops dropped, duplicates and reverse pairs merged;
 *   - edge id = rank of (u,v), u < v, in lexicographic order.
 * No blocking, fusion or incremental update: every h-support is a fresh pair of BFS runs.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct htdo_graph {
    int32_t n;
    int64_t m;
    int32_t *eu, *ev;   /* m canonical edges, eu < ev, lexicographic order */
    int64_t *adj_off;   /* n+1 offsets into adj_v / adj_e */
    int32_t *adj_v;     /* 2m neighbour ids */
    int64_t *adj_e;     /* 2m edge ids */
    int32_t *dist_a;    /* n BFS distances, -1 = unvisited */
    int32_t *dist_b;
    int32_t *queue_a;   /* n BFS queues (also the list of visited vertices) */
    int32_t *queue_b;
} htdo_graph;

static int cmp_u64(const void *a, const void *b) {
    uint64_t x = *(const uint64_t *)a, y = *(const uint64_t *)b;
    return (x > y) - (x < y);
}

/* Input hygiene (Sec. 2 assumes a simple undirected graph): drop self-loops, store each
 * pair as (min,max), sort lexicographically, merge duplicates.  eu/ev must hold m_in
 * entries.  Returns the number of distinct edges, or -1 if n < 0 or an id is outside
 * [0,n). */
int64_t htdo_normalise(int32_t n, const int32_t *src, const int32_t *dst, int64_t m_in,
                       int32_t *eu, int32_t *ev) {
    if (n < 0 || m_in < 0) return -1;
    uint64_t *keys = (uint64_t *)malloc((size_t)(m_in > 0 ? m_in : 1) * sizeof(uint64_t));
    if (!keys) return -2;
    int64_t k = 0;
    for (int64_t i = 0; i < m_in; i++) {
        int32_t a = src[i], b = dst[i];
        if (a < 0 || a >= n || b < 0 || b >= n) { free(keys); return -1; }
        if (a == b) continue;
        uint32_t lo = (uint32_t)(a < b ? a : b), hi = (uint32_t)(a < b ? b : a);
        keys[k++] = ((uint64_t)lo << 32) | hi;
    }
    qsort(keys, (size_t)k, sizeof(uint64_t), cmp_u64);
    int64_t m = 0;
    for (int64_t i = 0; i < k; i++) {
        if (i > 0 && keys[i] == keys[i - 1]) continue;
        eu[m] = (int32_t)(keys[i] >> 32);
        ev[m] = (int32_t)(keys[i] & 0xffffffffu);
        m++;
    }
    free(keys);
    return m;
}

void htdo_graph_free(htdo_graph *g) {
    if (!g) return;
    free(g->eu); free(g->ev); free(g->adj_off); free(g->adj_v); free(g->adj_e);
    free(g->dist_a); free(g->dist_b); free(g->queue_a); free(g->queue_b);
    free(g);
}

/* Builds adjacency lists for a graph given by canonical edges (eu < ev, sorted, distinct,
 * as returned by htdo_normalise).  Returns NULL on allocation failure. */
htdo_graph *htdo_graph_new(int32_t n, int64_t m, const int32_t *eu, const int32_t *ev) {
    htdo_graph *g = (htdo_graph *)calloc(1, sizeof(htdo_graph));
    if (!g) return NULL;
    g->n = n;
    g->m = m;
    size_t nn = (size_t)(n > 0 ? n : 1), mm = (size_t)(m > 0 ? m : 1);
    g->eu = (int32_t *)malloc(mm * sizeof(int32_t));
    g->ev = (int32_t *)malloc(mm * sizeof(int32_t));
    g->adj_off = (int64_t *)calloc(nn + 1, sizeof(int64_t));
    g->adj_v = (int32_t *)malloc(2 * mm * sizeof(int32_t));
    g->adj_e = (int64_t *)malloc(2 * mm * sizeof(int64_t));
    g->dist_a = (int32_t *)malloc(nn * sizeof(int32_t));
    g->dist_b = (int32_t *)malloc(nn * sizeof(int32_t));
    g->queue_a = (int32_t *)malloc(nn * sizeof(int32_t));
    g->queue_b = (int32_t *)malloc(nn * sizeof(int32_t));
    if (!g->eu || !g->ev || !g->adj_off || !g->adj_v || !g->adj_e || !g->dist_a ||
        !g->dist_b || !g->queue_a || !g->queue_b) {
        htdo_graph_free(g);
        return NULL;
    }
    if (m > 0) {
        memcpy(g->eu, eu, (size_t)m * sizeof(int32_t));
        memcpy(g->ev, ev, (size_t)m * sizeof(int32_t));
    }
    for (int64_t e = 0; e < m; e++) {
        g->adj_off[eu[e] + 1]++;
        g->adj_off[ev[e] + 1]++;
    }
    for (int32_t x = 0; x < n; x++) g->adj_off[x + 1] += g->adj_off[x];
    int64_t *fill = (int64_t *)malloc(nn * sizeof(int64_t));
    if (!fill) { htdo_graph_free(g); return NULL; }
    for (int32_t x = 0; x < n; x++) fill[x] = g->adj_off[x];
    for (int64_t e = 0; e < m; e++) {
        int32_t u = eu[e], v = ev[e];
        g->adj_v[fill[u]] = v; g->adj_e[fill[u]++] = e;
        g->adj_v[fill[v]] = u; g->adj_e[fill[v]++] = e;
    }
    free(fill);
    for (int32_t x = 0; x < n; x++) { g->dist_a[x] = -1; g->dist_b[x] = -1; }
    return g;
}

/* Breadth-first search from src to depth h (Sec. 2: N_G(v,h) = vertices within distance h)
 * inside the edge subgraph {e : key == NULL or key[e] >= thr}.  Fills dist[] for every
 * vertex reached (src gets 0) and lists them in queue[]; returns how many were reached. */
static int64_t ball_bfs(const htdo_graph *g, int32_t src, int32_t h, const int32_t *key,
                        int32_t thr, int32_t *dist, int32_t *queue) {
    int64_t head = 0, tail = 0;
    dist[src] = 0;
    queue[tail++] = src;
    while (head < tail) {
        int32_t x = queue[head++];
        if (dist[x] >= h) continue;
        for (int64_t s = g->adj_off[x]; s < g->adj_off[x + 1]; s++) {
            int64_t e = g->adj_e[s];
            if (key && key[e] < thr) continue;
            int32_t y = g->adj_v[s];
            if (dist[y] < 0) {
                dist[y] = dist[x] + 1;
                queue[tail++] = y;
            }
        }
    }
    return tail;
}

static void ball_reset(int32_t *dist, const int32_t *queue, int64_t cnt) {
    for (int64_t i = 0; i < cnt; i++) dist[queue[i]] = -1;
}

/* h-support of edge e (Def. 2 and Def. 3): the number of vertices w, w not an endpoint,
 * with dist(u,w) <= h and dist(v,w) <= h, distances measured in the edge subgraph
 * {e' : key == NULL or key[e'] >= thr} (which must contain e). */
int32_t htdo_edge_h_support(htdo_graph *g, int32_t h, const int32_t *key, int32_t thr,
                            int64_t e) {
    int32_t u = g->eu[e], v = g->ev[e];
    int64_t na = ball_bfs(g, u, h, key, thr, g->dist_a, g->queue_a);
    int64_t nb = ball_bfs(g, v, h, key, thr, g->dist_b, g->queue_b);
    int32_t cnt = 0;
    for (int64_t i = 0; i < na; i++) {
        int32_t w = g->queue_a[i];
        if (w == u || w == v) continue;
        if (g->dist_b[w] >= 0) cnt++;
    }
    ball_reset(g->dist_a, g->queue_a, na);
    ball_reset(g->dist_b, g->queue_b, nb);
    return cnt;
}

/* h-support of every edge of the subgraph {key[e] >= thr} (all edges when key is NULL);
 * sup_out[e] = -1 for edges outside it.  This is the initial h-support loop of
 * Algorithm 2 and of Algorithm 1, run one edge after the other. */
void htdo_h_support(htdo_graph *g, int32_t h, const int32_t *key, int32_t thr,
                    int32_t *sup_out) {
    for (int64_t e = 0; e < g->m; e++) {
        if (key && key[e] < thr) { sup_out[e] = -1; continue; }
        sup_out[e] = htdo_edge_h_support(g, h, key, thr, e);
    }
}

/* Level-synchronous peeling (Sec. 3, Lemma 1, Algorithm 1 with every edge of the current
 * level removed at once): starting at k = 2, remove all alive edges whose h-support in
 * the alive subgraph is <= k-2, assigning them t = k; recompute every alive edge's
 * h-support from scratch after each removal round; when no alive edge qualifies, k grows
 * by one.  stamp_out[e] (nullable) receives the round in which e was removed.  Returns
 * the number of removal rounds, or -1 on allocation failure. */
int64_t htdo_truss_decompose(htdo_graph *g, int32_t h, int32_t *t_out, int32_t *stamp_out) {
    int64_t m = g->m;
    size_t mm = (size_t)(m > 0 ? m : 1);
    int32_t *alive = (int32_t *)malloc(mm * sizeof(int32_t));
    int32_t *sup = (int32_t *)malloc(mm * sizeof(int32_t));
    int64_t *frontier = (int64_t *)malloc(mm * sizeof(int64_t));
    if (!alive || !sup || !frontier) { free(alive); free(sup); free(frontier); return -1; }
    for (int64_t e = 0; e < m; e++) alive[e] = 1;
    htdo_h_support(g, h, alive, 1, sup);
    int64_t remaining = m, round = 0;
    int32_t k = 2;
    while (remaining > 0) {
        int64_t nf = 0;
        for (int64_t e = 0; e < m; e++)
            if (alive[e] && sup[e] <= k - 2) frontier[nf++] = e;
        if (nf == 0) { k++; continue; }
        for (int64_t i = 0; i < nf; i++) {
            int64_t e = frontier[i];
            t_out[e] = k;
            if (stamp_out) stamp_out[e] = (int32_t)round;
            alive[e] = 0;
        }
        remaining -= nf;
        round++;
        htdo_h_support(g, h, alive, 1, sup);
    }
    free(alive); free(sup); free(frontier);
    return round;
}

/* Algorithm 1 taken literally, one edge at a time: bins indexed by sup+2, k from 2 to
 * ubtruss = max sup + 2; pick the smallest-id edge of bin[k], assign t = k, delete it,
 * then for every remaining edge whose h-support is above k-2 recompute its h-support and
 * move it to bin[max(sup+2, k)].  The affected set E_G(e,h) of Algorithm 1 is taken as every remaining
 * edge (a superset of any reading of it).  Returns 0, or -1 on allocation failure. */
int32_t htdo_truss_sequential(htdo_graph *g, int32_t h, int32_t *t_out) {
    int64_t m = g->m;
    size_t mm = (size_t)(m > 0 ? m : 1);
    int32_t *alive = (int32_t *)malloc(mm * sizeof(int32_t));
    int32_t *sup = (int32_t *)malloc(mm * sizeof(int32_t));
    int32_t *bin = (int32_t *)malloc(mm * sizeof(int32_t));
    if (!alive || !sup || !bin) { free(alive); free(sup); free(bin); return -1; }
    for (int64_t e = 0; e < m; e++) alive[e] = 1;
    htdo_h_support(g, h, alive, 1, sup);
    int32_t ub = 2;
    for (int64_t e = 0; e < m; e++) {
        bin[e] = sup[e] + 2;
        if (bin[e] > ub) ub = bin[e];
    }
    for (int32_t k = 2; k <= ub; k++) {
        for (;;) {
            int64_t pick = -1;
            for (int64_t e = 0; e < m; e++)
                if (alive[e] && bin[e] == k) { pick = e; break; }
            if (pick < 0) break;
            t_out[pick] = k;
            alive[pick] = 0;
            for (int64_t e = 0; e < m; e++) {
                if (!alive[e] || sup[e] <= k - 2) continue;
                sup[e] = htdo_edge_h_support(g, h, alive, 1, e);
                bin[e] = (sup[e] + 2 > k) ? sup[e] + 2 : k;
            }
        }
    }
    free(alive); free(sup); free(bin);
    return 0;
}

/* Peeling certificate for a claimed decomposition (t, stamp), checked edge by edge for
 * the listed edges (all when edges == NULL):
 *   (validity)    sup_{T}(e,h) >= t(e)-2 in T = {e' : t(e') >= t(e)}  (Def. 4 (i));
 *   (removability) sup_{G_s}(e,h) <= t(e)-2 in G_s = {e' : stamp(e') >= stamp(e)},
 *                  i.e. e qualified for removal at level t(e) in the graph left when it
 *                  was removed (Algorithm 1, its removal step).
 * Together with stamps ordered like t (htdo_check_stamp_order) these imply t is the exact
 * h-trussness.  fail_out[i] gets 0 (ok), 1 (validity fails) or 2 (removability fails).
 * Returns the number of failing edges. */
int64_t htdo_certify(htdo_graph *g, int32_t h, const int32_t *t, const int32_t *stamp,
                     const int64_t *edges, int64_t ne, int32_t *fail_out) {
    int64_t cnt = edges ? ne : g->m, bad = 0;
    for (int64_t i = 0; i < cnt; i++) {
        int64_t e = edges ? edges[i] : i;
        int32_t f = 0;
        int32_t s_valid = htdo_edge_h_support(g, h, t, t[e], e);
        if (s_valid < t[e] - 2) f = 1;
        else {
            int32_t s_rem = htdo_edge_h_support(g, h, stamp, stamp[e], e);
            if (s_rem > t[e] - 2) f = 2;
        }
        if (fail_out) fail_out[i] = f;
        if (f) bad++;
    }
    return bad;
}

/* Stamps must be ordered like t: stamp(a) < stamp(b) implies t(a) <= t(b).  Returns the
 * number of stamp values whose smallest t is below the largest t of an earlier stamp
 * (0 means ordered), or -1 on a negative stamp or allocation failure. */
int64_t htdo_check_stamp_order(int64_t m, const int32_t *t, const int32_t *stamp) {
    int32_t smax = -1;
    for (int64_t e = 0; e < m; e++) if (stamp[e] > smax) smax = stamp[e];
    if (smax < 0) return 0;
    int32_t *tmin = (int32_t *)malloc((size_t)(smax + 1) * sizeof(int32_t));
    int32_t *tmax = (int32_t *)malloc((size_t)(smax + 1) * sizeof(int32_t));
    if (!tmin || !tmax) { free(tmin); free(tmax); return -1; }
    for (int32_t s = 0; s <= smax; s++) { tmin[s] = INT32_MAX; tmax[s] = INT32_MIN; }
    for (int64_t e = 0; e < m; e++) {
        int32_t s = stamp[e];
        if (s < 0) { free(tmin); free(tmax); return -1; }
        if (t[e] < tmin[s]) tmin[s] = t[e];
        if (t[e] > tmax[s]) tmax[s] = t[e];
    }
    int64_t bad = 0;
    int32_t run = INT32_MIN;
    for (int32_t s = 0; s <= smax; s++) {
        if (tmin[s] == INT32_MAX) continue;
        if (tmin[s] < run) bad++;
        if (tmax[s] > run) run = tmax[s];
    }
    free(tmin); free(tmax);
    return bad;
}

/* ---- The H-index iteration of Sec. 4 (Definition of the h-hop reachable path key,
 * Theorems 3 and 4, Algorithm 2; asynchronous updating) ------------------------------
 *
 * H(S) is the H-index of a multiset S: the largest y such that at least y members of S
 * are >= y.  With H^(0)(e) = sup_G(e,h), order n computes for e = (u,v)
 *     H^(n)(e) = H({ min(P(u,w), P(v,w)) : w in N_G(u,h) ∩ N_G(v,h) }),
 * where P(a,b), the h-hop reachable path key, is the largest over paths from a to b of at
 * most h edges of the smallest H^(n-1) on the path.  Readings: the paths have at most h
 * edges (with unbounded paths the proof of Theorem 4 (ii) does not hold), they may use e
 * itself, and the common h-neighbourhood is that of the whole graph G.  The iteration
 * stops at the first order n with H^(n) = H^(n-1) on every edge; t(e,h) = H^(n)(e) + 2
 * (Theorem 4).  Asynchronous updating (Sec. 4) takes the edges in id order and uses every
 * value already updated in the current sweep. */

/* H-index of vals[0..cnt) (reorders vals). */
static int32_t h_index(int32_t *vals, int64_t cnt) {
    /* counting by value: c[y] = members equal to y, capped at cnt */
    int64_t *c = (int64_t *)calloc((size_t)cnt + 2, sizeof(int64_t));
    if (!c) return -1;
    for (int64_t i = 0; i < cnt; i++) {
        int64_t v = vals[i] < 0 ? 0 : vals[i];
        c[v > cnt ? cnt : v]++;
    }
    int64_t at_least = 0;
    int32_t y = 0;
    for (int64_t v = cnt; v >= 0; v--) {
        at_least += c[v];
        if (at_least >= v) { y = (int32_t)v; break; }
    }
    free(c);
    return y;
}

/* P(src, w) for every vertex w: hop-limited widest paths by h rounds of relaxation over
 * all edges (round r extends the paths of at most r-1 edges by one edge).  key = H per
 * edge.  best[w] = -1 where no path of at most h edges exists; best[src] = INT32_MAX (the
 * empty path). */
static void path_keys(const htdo_graph *g, int32_t src, int32_t h, const int32_t *key,
                      int32_t *best, int32_t *prev) {
    for (int32_t x = 0; x < g->n; x++) best[x] = -1;
    best[src] = INT32_MAX;
    for (int32_t r = 1; r <= h; r++) {
        memcpy(prev, best, (size_t)g->n * sizeof(int32_t));
        for (int64_t e = 0; e < g->m; e++) {
            int32_t a = g->eu[e], b = g->ev[e];
            if (prev[a] >= 0) {
                int32_t c = prev[a] < key[e] ? prev[a] : key[e];
                if (c > best[b]) best[b] = c;
            }
            if (prev[b] >= 0) {
                int32_t c = prev[b] < key[e] ? prev[b] : key[e];
                if (c > best[a]) best[a] = c;
            }
        }
    }
}

/* One order of the iteration for edge e from the keys `key`: H({min(P(u,w),P(v,w))}). */
static int32_t hindex_edge(htdo_graph *g, int32_t h, const int32_t *key, int64_t e,
                           int32_t *pu, int32_t *pv, int32_t *tmp, int32_t *vals) {
    int32_t u = g->eu[e], v = g->ev[e];
    path_keys(g, u, h, key, pu, tmp);
    path_keys(g, v, h, key, pv, tmp);
    /* the common h-neighbours of e in G */
    int64_t na = ball_bfs(g, u, h, NULL, 0, g->dist_a, g->queue_a);
    int64_t nb = ball_bfs(g, v, h, NULL, 0, g->dist_b, g->queue_b);
    int64_t cnt = 0;
    for (int64_t i = 0; i < na; i++) {
        int32_t w = g->queue_a[i];
        if (w == u || w == v || g->dist_b[w] < 0) continue;
        vals[cnt++] = pu[w] < pv[w] ? pu[w] : pv[w];
    }
    ball_reset(g->dist_a, g->queue_a, na);
    ball_reset(g->dist_b, g->queue_b, nb);
    return h_index(vals, cnt);
}

/* The H-index iteration from H^(0) = sup_G(e,h) for at most max_iter orders (max_iter < 0:
 * until stable).  asynchronous = 0: order n uses only H^(n-1) (Algorithm 2);
 * asynchronous = 1: Gauss-Seidel sweeps in edge id order.  hv_out receives the last H
 * values; iters_out the orders computed (the last one changed nothing when converged).
 * Returns 1 if converged, 0 if stopped at max_iter (or, which Theorem 3 rules out, after
 * more orders than the values can decrease), -1 on allocation failure. */
int32_t htdo_hindex(htdo_graph *g, int32_t h, int32_t asynchronous, int32_t max_iter,
                    int32_t *hv_out, int32_t *iters_out) {
    int64_t m = g->m;
    size_t mm = (size_t)(m > 0 ? m : 1), nn = (size_t)(g->n > 0 ? g->n : 1);
    int32_t *cur = (int32_t *)malloc(mm * sizeof(int32_t));
    int32_t *nxt = (int32_t *)malloc(mm * sizeof(int32_t));
    int32_t *pu = (int32_t *)malloc(nn * sizeof(int32_t));
    int32_t *pv = (int32_t *)malloc(nn * sizeof(int32_t));
    int32_t *tmp = (int32_t *)malloc(nn * sizeof(int32_t));
    int32_t *vals = (int32_t *)malloc(nn * sizeof(int32_t));
    int32_t rc = 0, n = 0;
    if (!cur || !nxt || !pu || !pv || !tmp || !vals) { rc = -1; goto done; }
    htdo_h_support(g, h, NULL, 0, cur);
    /* every order before the fixed point lowers at least one value by at least one
     * (Theorem 3), so 1 + sum of H^(0) orders always suffice */
    int64_t cap = 1;
    for (int64_t e = 0; e < m; e++) cap += cur[e];
    for (;;) {
        if (max_iter >= 0 && n >= max_iter) break;
        if (n >= cap) break;
        int changed = 0;
        if (asynchronous) {
            for (int64_t e = 0; e < m; e++) {
                int32_t v = hindex_edge(g, h, cur, e, pu, pv, tmp, vals);
                if (v < 0) { rc = -1; goto done; }
                if (v != cur[e]) { cur[e] = v; changed = 1; }
            }
        } else {
            for (int64_t e = 0; e < m; e++) {
                nxt[e] = hindex_edge(g, h, cur, e, pu, pv, tmp, vals);
                if (nxt[e] < 0) { rc = -1; goto done; }
                if (nxt[e] != cur[e]) changed = 1;
            }
            int32_t *t = cur; cur = nxt; nxt = t;
        }
        n++;
        if (!changed) { rc = 1; break; }
    }
    if (m > 0) memcpy(hv_out, cur, (size_t)m * sizeof(int32_t));
done:
    if (iters_out) *iters_out = n;
    free(cur); free(nxt); free(pu); free(pv); free(tmp); free(vals);
    return rc;
}

/* Synchronous H-index iteration with the redundant-computation pruning of Sec. 4 (Lemma 4):
 * from order 2 on, H^(n)(e) is not computed but set to H^(n-1)(e) when no edge e' of
 * E_G(e,h) fell across T = H^(n-1)(e) in the previous order, i.e. when every e' has
 * H^(n-2)(e') = H^(n-1)(e') (case i), H^(n-2)(e') < T (case ii) or H^(n-1)(e') >= T
 * (case iii).  Reading of E_G(e,h), which the paper leaves undefined here: every edge with
 * an endpoint within distance h-1 of u or of v in G, which holds every edge of a path of
 * at most h edges from u or from v (the paths the keys of H^(n)(e) come from).  Outputs as
 * htdo_hindex; evals_out (nullable) receives the number of H^(n)(e) actually computed.
 * Returns 1 if converged, 0 if stopped at max_iter, -1 on allocation failure. */
int32_t htdo_hindex_pruned(htdo_graph *g, int32_t h, int32_t max_iter, int32_t *hv_out,
                           int32_t *iters_out, int64_t *evals_out) {
    int64_t m = g->m;
    size_t mm = (size_t)(m > 0 ? m : 1), nn = (size_t)(g->n > 0 ? g->n : 1);
    int32_t *old = (int32_t *)malloc(mm * sizeof(int32_t));   /* H^(n-2) */
    int32_t *cur = (int32_t *)malloc(mm * sizeof(int32_t));   /* H^(n-1) */
    int32_t *nxt = (int32_t *)malloc(mm * sizeof(int32_t));   /* H^(n)   */
    int32_t *pu = (int32_t *)malloc(nn * sizeof(int32_t));
    int32_t *pv = (int32_t *)malloc(nn * sizeof(int32_t));
    int32_t *tmp = (int32_t *)malloc(nn * sizeof(int32_t));
    int32_t *vals = (int32_t *)malloc(nn * sizeof(int32_t));
    int32_t rc = 0, n = 0;
    int64_t evals = 0;
    if (!old || !cur || !nxt || !pu || !pv || !tmp || !vals) { rc = -1; goto done; }
    htdo_h_support(g, h, NULL, 0, cur);
    int64_t cap = 1;
    for (int64_t e = 0; e < m; e++) cap += cur[e];
    for (;;) {
        if (max_iter >= 0 && n >= max_iter) break;
        if (n >= cap) break;
        int changed = 0;
        for (int64_t e = 0; e < m; e++) {
            int needed = 1;
            if (n >= 1) {
                /* was any edge of E_G(e,h) across T = H^(n-1)(e) in the previous order? */
                int32_t T = cur[e], u = g->eu[e], v = g->ev[e];
                int64_t na = ball_bfs(g, u, h - 1, NULL, 0, g->dist_a, g->queue_a);
                int64_t nb = ball_bfs(g, v, h - 1, NULL, 0, g->dist_b, g->queue_b);
                needed = 0;
                for (int64_t f = 0; f < m && !needed; f++) {
                    int32_t a = g->eu[f], b = g->ev[f];
                    int in = g->dist_a[a] >= 0 || g->dist_a[b] >= 0 || g->dist_b[a] >= 0 ||
                             g->dist_b[b] >= 0;
                    if (in && old[f] >= T && cur[f] < T) needed = 1;
                }
                ball_reset(g->dist_a, g->queue_a, na);
                ball_reset(g->dist_b, g->queue_b, nb);
            }
            if (needed) {
                nxt[e] = hindex_edge(g, h, cur, e, pu, pv, tmp, vals);
                if (nxt[e] < 0) { rc = -1; goto done; }
                evals++;
            } else {
                nxt[e] = cur[e];
            }
            if (nxt[e] != cur[e]) changed = 1;
        }
        int32_t *t = old; old = cur; cur = nxt; nxt = t;
        n++;
        if (!changed) { rc = 1; break; }
    }
    if (m > 0) memcpy(hv_out, cur, (size_t)m * sizeof(int32_t));
done:
    if (iters_out) *iters_out = n;
    if (evals_out) *evals_out = evals;
    free(old); free(cur); free(nxt); free(pu); free(pv); free(tmp); free(vals);
    return rc;
}
