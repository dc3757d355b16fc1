/*
 * htd_cert.c -- all-edge peeling certificate for a claimed (k,h)-truss decomposition
 * (Chen et al., "Parallel Higher-order Truss Decomposition", 2024).
 *
 * TEST INFRASTRUCTURE ONLY, like the rest of this directory: the tests and the smoke check
 * load it to check the CUDA path's output.  It shares no code, header or table with the
 * CUDA path.
 *
 * What is checked, for a claimed trussness t(e) and removal round stamp(e) of every edge:
 *   (order)        stamp(a) <= stamp(b) implies t(a) <= t(b);
 *   (validity)     sup_T(e,h) >= t(e) - 2 in T = {e' : t(e') >= t(e)}          (Def. 4);
 *   (removability) sup_G(e,h) <= t(e) - 2 in G = {e' : stamp(e') >= stamp(e)},  i.e. e
 *                  qualified for removal at level t(e) in the graph left when it was
 *                  removed (Sec. 3, Algorithm 1, its removal step).
 * Validity makes every T_k = {t >= k} satisfy Def. 4, so t(e) is at most the true
 * trussness.  If some e had a larger true trussness K, the edge e* of the (K,h)-truss with
 * the smallest stamp would have h-support >= K - 2 in its removal graph; removability gives
 * t(e*) >= K, and the order (stamp(e*) <= stamp(e)) gives t(e*) <= t(e) < K.  So the three
 * conditions together prove that t is exactly the h-trussness of every edge.
 *
 * How the h-supports are obtained: the graphs G_s = {stamp >= s} grow as s decreases, so
 * the edges are inserted in decreasing stamp order and every closed ball
 * B(x,r) = {w : dist(x,w) <= r}, r = 1..h, is kept as an n-bit set.  Inserting an edge set
 * can only add members: a pair {p,q} comes within distance r exactly when some path of at
 * most r edges between them uses a new edge (a,b), i.e. p in B(a,i) and q in B(b,r-1-i)
 * for some i in [0, r-1], both balls taken in the new graph (a shorter walk is a path too,
 * so taking the new balls adds only true pairs).  The radii are therefore brought up to
 * date one after the other: adjacency first, then radius 2 from radius <= 1, and so on.
 * After the edges of stamp s are in, every h-support of G_s is |B(u,h) ∩ B(v,h)| - 2
 * (Def. 2, Def. 3: u and v lie in both closed balls).  Under the order condition,
 * T_k = G_{s_min(k)} with s_min(k) the smallest stamp of level k, so the validity supports
 * of level k are read when that stamp's edges are in.
 *
 * The work of one stamp (adjacency, then each radius, then the support reads) is split
 * over threads (pthreads); the phases are separated by barriers, and bits are set with
 * atomic ORs, so the result does not depend on the thread count.
 */
#include <pthread.h>
#include <sched.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define CERT_MAX_H 8

typedef struct cert {
    int32_t n, h, nthreads;
    int64_t m, W;               /* W = 64-bit words of an n-bit set */
    const int32_t *eu, *ev, *t, *stamp;
    uint64_t *ball[CERT_MAX_H + 1];  /* ball[r] = n x W words: B(x,r), r = 1..h (r = 1
                                        only when needed: h == 1 or h >= 3) */
    int64_t *adj_off;           /* n+1: adjacency capacity of every vertex */
    int32_t *adj_fill;          /* n: neighbours inserted so far */
    int32_t *adj;               /* 2m */
    int64_t *order;             /* m edge ids by decreasing stamp */
    int64_t next[4];            /* work counters of phases seq, seq+1, seq+2 (mod 4) */
    /* barrier between phases: arrivals counted down, the last one flips the sense */
    int32_t bar_left, bar_sense;
    pthread_mutex_t gate;       /* workers start once the thread count is final */
    pthread_cond_t gate_cv;
    int32_t go;
    int32_t *sup_rem, *sup_val; /* nullable outputs */
    int32_t *fail;
    int32_t **buf;              /* per thread: 2 member lists of n entries */
    int32_t nbuf;
} cert;

static inline void set_bit(uint64_t *row, int32_t q) {
    uint64_t *w = row + (q >> 6);
    const uint64_t mask = 1ull << (q & 63);
    if (!(__atomic_load_n(w, __ATOMIC_RELAXED) & mask)) __atomic_fetch_or(w, mask, __ATOMIC_RELAXED);
}

static inline void row_or(uint64_t *dst, const uint64_t *src, int64_t W) {
    for (int64_t i = 0; i < W; i++) {
        const uint64_t v = src[i];
        if (v & ~__atomic_load_n(dst + i, __ATOMIC_RELAXED)) __atomic_fetch_or(dst + i, v, __ATOMIC_RELAXED);
    }
}

/* Bit count by the usual shift-and-add reduction, written portably so that the loop below
 * vectorises on any target. */
static inline uint64_t popc64(uint64_t x) {
    x = x - ((x >> 1) & 0x5555555555555555ull);
    x = (x & 0x3333333333333333ull) + ((x >> 2) & 0x3333333333333333ull);
    x = (x + (x >> 4)) & 0x0f0f0f0f0f0f0f0full;
    x += x >> 8;
    x += x >> 16;
    x += x >> 32;
    return x & 0x7f;
}

static int64_t and_count(const uint64_t *a, const uint64_t *b, int64_t W) {
    uint64_t c = 0;
    for (int64_t i = 0; i < W; i++) c += popc64(a[i] & b[i]);
    return (int64_t)c;
}

/* Members of the closed ball B(x,i) in the current graph, into out[]; returns the count. */
static int64_t members(const cert *C, int32_t i, int32_t x, int32_t *out) {
    if (i == 0) {
        out[0] = x;
        return 1;
    }
    if (i == 1) {
        const int64_t b = C->adj_off[x];
        const int32_t f = C->adj_fill[x];
        out[0] = x;
        for (int32_t j = 0; j < f; j++) out[1 + j] = C->adj[b + j];
        return 1 + (int64_t)f;
    }
    const uint64_t *row = C->ball[i] + (int64_t)x * C->W;
    int64_t c = 0;
    for (int64_t w = 0; w < C->W; w++) {
        uint64_t v = row[w];
        while (v) {
            const int bit = __builtin_ctzll(v);
            out[c++] = (int32_t)(w * 64 + bit);
            v &= v - 1;
        }
    }
    return c;
}

/* Pairs {p,q}, p in B(a,i), q in B(b,j), i + j = r - 1, are put within distance r. */
static void ball_term(cert *C, int tid, int32_t r, int32_t i, int32_t a, int32_t b) {
    const int32_t j = r - 1 - i;
    int32_t *P = C->buf[tid], *Q = C->buf[tid] + C->n;
    const int64_t np = members(C, i, a, P), nq = members(C, j, b, Q);
    uint64_t *Br = C->ball[r];
    const int64_t W = C->W;
    const int rows_ok = i >= 1 && j >= 1 && C->ball[i] && C->ball[j];
    if (!rows_ok || np * nq <= (np + nq) * W) {
        for (int64_t x = 0; x < np; x++) {
            uint64_t *row = Br + (int64_t)P[x] * W;
            for (int64_t y = 0; y < nq; y++) set_bit(row, Q[y]);
        }
        for (int64_t y = 0; y < nq; y++) {
            uint64_t *row = Br + (int64_t)Q[y] * W;
            for (int64_t x = 0; x < np; x++) set_bit(row, P[x]);
        }
    } else {
        const uint64_t *rb = C->ball[j] + (int64_t)b * W, *ra = C->ball[i] + (int64_t)a * W;
        for (int64_t x = 0; x < np; x++) row_or(Br + (int64_t)P[x] * W, rb, W);
        for (int64_t y = 0; y < nq; y++) row_or(Br + (int64_t)Q[y] * W, ra, W);
    }
}

/* One phase of the check: every thread derives the same sequence of phases itself. */
typedef struct phase_t {
    const int64_t *items;  /* edge ids of the phase */
    int64_t nitems, nterms;
    int32_t radius;        /* radius of a ball phase */
    int32_t mode;          /* 0 adjacency, 1 ball radius, 2 removability, 3 validity */
    int64_t seq;           /* phase number: selects the work counter */
} phase_t;

static void unit(cert *C, const phase_t *ph, int tid, int64_t u) {
    const int64_t e = ph->items[u / ph->nterms];
    const int32_t a = C->eu[e], b = C->ev[e];
    switch (ph->mode) {
    case 0: { /* adjacency (and radius-1 sets) */
        const int32_t fa = __atomic_fetch_add(&C->adj_fill[a], 1, __ATOMIC_RELAXED);
        C->adj[C->adj_off[a] + fa] = b;
        const int32_t fb = __atomic_fetch_add(&C->adj_fill[b], 1, __ATOMIC_RELAXED);
        C->adj[C->adj_off[b] + fb] = a;
        for (int32_t r = 1; r <= C->h; r++) {
            if (!C->ball[r]) continue;
            set_bit(C->ball[r] + (int64_t)a * C->W, b);
            set_bit(C->ball[r] + (int64_t)b * C->W, a);
        }
        break;
    }
    case 1: /* radius r >= 2, term i = u % nterms */
        ball_term(C, tid, ph->radius, (int32_t)(u % ph->nterms), a, b);
        break;
    default: { /* h-support of e in the current graph */
        const int64_t W = C->W;
        const uint64_t *bh = C->ball[C->h];
        const int32_t s = (int32_t)(and_count(bh + (int64_t)a * W, bh + (int64_t)b * W, W) - 2);
        if (ph->mode == 2) {
            if (C->sup_rem) C->sup_rem[e] = s;
            if (s > C->t[e] - 2) __atomic_fetch_or(&C->fail[e], 2, __ATOMIC_RELAXED);
        } else {
            if (C->sup_val) C->sup_val[e] = s;
            if (s < C->t[e] - 2) __atomic_fetch_or(&C->fail[e], 1, __ATOMIC_RELAXED);
        }
        break;
    }
    }
}

/* Runs the current phase's units on thread tid (work taken from a shared counter). */
static void run_phase(cert *C, const phase_t *ph, int tid) {
    int64_t *ctr = &C->next[ph->seq & 3];
    const int64_t total = ph->nitems * ph->nterms;
    const int64_t chunk = ph->mode == 0 ? 64 : 1;
    for (;;) {
        const int64_t u0 = __atomic_fetch_add(ctr, chunk, __ATOMIC_RELAXED);
        if (u0 >= total) break;
        const int64_t u1 = u0 + chunk < total ? u0 + chunk : total;
        for (int64_t u = u0; u < u1; u++) unit(C, ph, tid, u);
    }
}

/* Phase barrier: the phases are short (a few edges), so waiting threads spin (yielding
 * the core after a while) instead of sleeping. */
static void spin_barrier(cert *C, int32_t *local_sense) {
    const int32_t s = *local_sense ^ 1;
    *local_sense = s;
    if (__atomic_sub_fetch(&C->bar_left, 1, __ATOMIC_ACQ_REL) == 0) {
        __atomic_store_n(&C->bar_left, C->nthreads, __ATOMIC_RELAXED);
        __atomic_store_n(&C->bar_sense, s, __ATOMIC_RELEASE);
        return;
    }
    for (uint64_t spins = 0; __atomic_load_n(&C->bar_sense, __ATOMIC_ACQUIRE) != s; spins++)
        if (spins > 4096) sched_yield();
}

typedef struct worker_arg {
    cert *C;
    int tid;
} worker_arg;

/* Phase sequence of the whole check; every thread runs it, thread 0 sets up each phase
 * between two barriers. */
static void drive(cert *C, int tid) {
    const int T = C->nthreads;
    int64_t pos = 0;
    int64_t level_lo = 0;  /* first edge (in order[]) of the current level */
    int32_t sense = 0;
#define SYNC() do { if (T > 1) spin_barrier(C, &sense); } while (0)
    phase_t ph;
    ph.seq = 0;
    /* phase seq runs on counter seq & 3; thread 0 clears the counter of phase seq + 2,
     * which the barriers at the ends of phases seq and seq + 1 separate from its use */
#define PHASE(MODE, ITEMS, NITEMS, NTERMS, R)                                            \
    do {                                                                                 \
        ph.mode = (MODE); ph.items = (ITEMS); ph.nitems = (NITEMS);                       \
        ph.nterms = (NTERMS); ph.radius = (R);                                           \
        if (tid == 0) C->next[(ph.seq + 2) & 3] = 0;                                     \
        run_phase(C, &ph, tid);                                                          \
        SYNC();                                                                          \
        ph.seq++;                                                                        \
    } while (0)
    while (pos < C->m) {
        const int32_t s = C->stamp[C->order[pos]];
        int64_t end = pos;
        while (end < C->m && C->stamp[C->order[end]] == s) end++;
        const int64_t *grp = C->order + pos;
        const int64_t cnt = end - pos;
        PHASE(0, grp, cnt, 1, 1);
        for (int32_t r = 2; r <= C->h; r++) PHASE(1, grp, cnt, r, r);
        PHASE(2, grp, cnt, 1, 0);
        /* the last stamp of a level in this order is its smallest: T_k is complete */
        const int32_t k = C->t[C->order[pos]];
        if (end == C->m || C->t[C->order[end]] != k) {
            PHASE(3, C->order + level_lo, end - level_lo, 1, 0);
            level_lo = end;
        }
        pos = end;
    }
#undef PHASE
#undef SYNC
}

static void *worker(void *p) {
    worker_arg *w = (worker_arg *)p;
    cert *C = w->C;
    pthread_mutex_lock(&C->gate);
    while (!C->go) pthread_cond_wait(&C->gate_cv, &C->gate);
    pthread_mutex_unlock(&C->gate);
    drive(C, w->tid);
    return NULL;
}

/* Certifies every edge of a claimed decomposition (see the top of this file).
 *   n, m, eu, ev     the normalised graph (eu < ev, m edges);
 *   h                hop threshold, 1..CERT_MAX_H;
 *   t, stamp         the claim: trussness and removal round of every edge;
 *   nthreads         threads to use (< 1: 1);
 *   fail_out         m codes: 0 ok, bit 1 validity fails, bit 2 removability fails;
 *   sup_rem, sup_val nullable, m each: sup(e,h) in {stamp >= stamp(e)} and in
 *                    {t >= t(e)} (the latter is -1 for every edge if the order fails);
 *   order_bad        receives the number of stamps whose smallest t lies below the
 *                    largest t of a smaller stamp (0 = ordered).
 * Returns the number of failing edges, -1 on allocation failure, -2 on a bad argument
 * (negative stamp, h out of range) and -3 when the order fails (nothing else checked). */
int64_t htdo_certify_all(int32_t n, int64_t m, const int32_t *eu, const int32_t *ev, int32_t h,
                         const int32_t *t, const int32_t *stamp, int32_t nthreads,
                         int32_t *fail_out, int32_t *sup_rem, int32_t *sup_val,
                         int64_t *order_bad) {
    if (order_bad) *order_bad = 0;
    if (h < 1 || h > CERT_MAX_H || n < 0 || m < 0) return -2;
    for (int64_t e = 0; e < m; e++) {
        fail_out[e] = 0;
        if (sup_rem) sup_rem[e] = -1;
        if (sup_val) sup_val[e] = -1;
        if (stamp[e] < 0 || stamp[e] > m) return -2;
    }
    if (m == 0) return 0;
    cert C;
    memset(&C, 0, sizeof(C));
    C.n = n; C.m = m; C.h = h; C.eu = eu; C.ev = ev; C.t = t; C.stamp = stamp;
    C.nthreads = nthreads < 1 ? 1 : nthreads;
    C.next[0] = C.next[1] = 0;
    C.W = ((int64_t)n + 63) / 64;
    C.fail = fail_out; C.sup_rem = sup_rem; C.sup_val = sup_val;
    pthread_mutex_init(&C.gate, NULL);
    pthread_cond_init(&C.gate_cv, NULL);
    int64_t rc = -1;
    /* edges by decreasing stamp (counting sort), then the order condition */
    int64_t *cnt = (int64_t *)calloc((size_t)m + 2, sizeof(int64_t));
    C.order = (int64_t *)malloc((size_t)m * sizeof(int64_t));
    C.adj_off = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    C.adj_fill = (int32_t *)calloc((size_t)(n > 0 ? n : 1), sizeof(int32_t));
    C.adj = (int32_t *)malloc((size_t)(2 * m) * sizeof(int32_t));
    C.buf = (int32_t **)calloc((size_t)C.nthreads, sizeof(int32_t *));
    C.nbuf = C.buf ? C.nthreads : 0;
    if (!cnt || !C.order || !C.adj_off || !C.adj_fill || !C.adj || !C.buf) goto done;
    for (int64_t e = 0; e < m; e++) cnt[m - stamp[e]]++;
    for (int64_t i = 1; i <= m + 1; i++) cnt[i] += cnt[i - 1];
    for (int64_t e = m - 1; e >= 0; e--) C.order[--cnt[m - stamp[e]]] = e;
    {
        int64_t bad = 0;
        int32_t run_min = INT32_MAX;  /* smallest t among larger stamps */
        int64_t p = 0;
        while (p < m) {
            const int32_t s = stamp[C.order[p]];
            int64_t q = p;
            int32_t tmax = INT32_MIN, tmin = INT32_MAX;
            while (q < m && stamp[C.order[q]] == s) {
                const int32_t tv = t[C.order[q]];
                if (tv > tmax) tmax = tv;
                if (tv < tmin) tmin = tv;
                q++;
            }
            if (tmax > run_min || tmin != tmax) bad++;
            if (tmin < run_min) run_min = tmin;
            p = q;
        }
        if (order_bad) *order_bad = bad;
        if (bad) { rc = -3; goto done; }
    }
    for (int64_t e = 0; e < m; e++) { C.adj_off[eu[e] + 1]++; C.adj_off[ev[e] + 1]++; }
    for (int32_t x = 0; x < n; x++) C.adj_off[x + 1] += C.adj_off[x];
    for (int32_t r = 1; r <= h; r++) {
        if (r == 1 && h == 2) continue;  /* radius 2 is built from the adjacency lists */
        /* zeroed up front: faulting the pages in lazily from many threads at once
         * serialises them in the kernel */
        const size_t bytes = (size_t)n * (size_t)C.W * sizeof(uint64_t);
        C.ball[r] = (uint64_t *)malloc(bytes);
        if (!C.ball[r]) goto done;
        memset(C.ball[r], 0, bytes);
        for (int32_t x = 0; x < n; x++) C.ball[r][(int64_t)x * C.W + (x >> 6)] |= 1ull << (x & 63);
    }
    for (int i = 0; i < C.nthreads; i++) {
        C.buf[i] = (int32_t *)malloc((size_t)(2 * (int64_t)n + 2) * sizeof(int32_t));
        if (!C.buf[i]) goto done;
    }
    if (C.nthreads > 1) {
        pthread_t *th = (pthread_t *)malloc((size_t)C.nthreads * sizeof(pthread_t));
        worker_arg *wa = (worker_arg *)malloc((size_t)C.nthreads * sizeof(worker_arg));
        if (!th || !wa) { free(th); free(wa); goto done; }
        /* threads that could not be started simply run no share: the barrier counts the
         * threads that did start */
        int started = 1;
        pthread_mutex_lock(&C.gate);
        for (int i = 1; i < C.nthreads; i++) {
            wa[i].C = &C; wa[i].tid = i;
            if (pthread_create(&th[i], NULL, worker, &wa[i]) != 0) break;
            started++;
        }
        C.nthreads = started;
        C.bar_left = started;
        C.go = 1;
        pthread_cond_broadcast(&C.gate_cv);
        pthread_mutex_unlock(&C.gate);
        drive(&C, 0);
        for (int i = 1; i < started; i++) pthread_join(th[i], NULL);
        free(th); free(wa);
    } else {
        drive(&C, 0);
    }
    rc = 0;
    for (int64_t e = 0; e < m; e++) rc += fail_out[e] != 0;
done:
    for (int r = 0; r <= CERT_MAX_H; r++) free(C.ball[r]);
    for (int i = 0; i < C.nbuf; i++) free(C.buf[i]);
    free(C.buf); free(cnt); free(C.order); free(C.adj_off); free(C.adj_fill); free(C.adj);
    pthread_mutex_destroy(&C.gate);
    pthread_cond_destroy(&C.gate_cv);
    return rc;
}
