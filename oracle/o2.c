/*
 * Scalable sequential CPU oracle for greedy all-switches strategy improvement
 * with one-player best responses (Fearnley, "Efficient Parallel Strategy
 * Improvement for Parity Games", arXiv 1705.02313).
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product path may call, link or
 * load this file; only tests, the smoke check and the CPU-baseline leg of the
 * benchmark use it. It shares no code with the CUDA path.
 *
 * Scope: games whose priorities are pairwise distinct (every count in a
 * valuation is then 0 or 1). Plain C, single thread, int32/int64 only.
 *
 * Conventions (each is a reading of a passage the paper leaves open):
 *  - the sink has id n (n = vertex count of the preprocessed game G');
 *  - strat[v] is sigma(v) for Even v (n = the sink) and tau(v) for Odd v;
 *  - switches are taken only when strictly better, and among equally good
 *    successors the lowest CSR position wins; for Even the sink is considered
 *    before the edge list (Section 3, "Switching rules"; Section 4,
 *    All_Odd);
 *  - the initial Odd strategy is the first edge of each list (Algorithm 1
 *    leaves it arbitrary).
 *
 * Valuation encoding (the order of Section 3, "Valuations"): with distinct
 * priorities a finite valuation is the set P(v) of vertices on the play from
 * v to the sink. The oracle reports, for every vertex, its class (finite or
 * top), depth |P(v)|, and its rank: the position of Val(v) in the total order
 * of all finite valuations together with the empty valuation of the sink.
 * Ranks are built by Kruskal's merge order (tree edges taken in increasing
 * priority of their lower endpoint, the child side placed above the parent
 * side when that priority is even and below it when odd). Tests pin this
 * order against the literal Maxdiff comparison of Section 3 and against a
 * closed form; o2_compare gives the literal comparison by walking both paths.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define O2_OK 0
#define O2_EINVAL 1
#define O2_ENOMEM 2
#define O2_ETIMEOUT 3
#define O2_ENOTADMISSIBLE 4
#define O2_ECHECK 5

#define CLS_FIN 0
#define CLS_TOP 1
#define CLS_ODDCYCLE 2

typedef struct {
    int32_t n;
    const int32_t *off, *tgt;
    const uint8_t *own;
    const int32_t *pri;
} o2_game;

/* ------------------------------------------------------------------------ */
/* P0: admissibility preprocessing (Section 3, "The algorithm", the sentence
 * on dummy Even vertices). U is the greatest set of Odd vertices each having
 * an edge into U (Odd can avoid Even vertices forever from U). Every w in U
 * that is the target of an edge from U gets a dummy Even vertex d_w with the
 * single edge d_w -> w; edges U -> w are redirected to d_w. Dummy j (for the
 * j-th such w in increasing id order) has id n+j and priority 2j; every
 * original priority p becomes p + 2k. With dummy_zero (games whose
 * priorities repeat, ranked by count vectors) every dummy has priority 0
 * instead and every original priority becomes p + 2: the dummies then add
 * one priority, not k. Both keep parities and put the dummies below every
 * original priority. Outputs must be sized for the worst case:
 * out_off[2n+1], out_tgt[m+n], out_own[2n], out_pri[2n], dummy_of[n].
 */
int o2_preprocess(int32_t n, const int32_t *off, const int32_t *tgt, const uint8_t *own,
                  const int32_t *pri, int32_t *out_off, int32_t *out_tgt, uint8_t *out_own,
                  int32_t *out_pri, int32_t *dummy_of, int32_t *k_out, uint8_t *in_u_out, int dummy_zero)
{
    int64_t m = off[n];
    /* count, for every Odd vertex, its edges into the current U (initially all Odd) */
    int32_t *cnt = (int32_t *)calloc((size_t)n + 1, sizeof(int32_t));
    int32_t *roff = (int32_t *)calloc((size_t)n + 2, sizeof(int32_t));
    int32_t *radj = (int32_t *)malloc(sizeof(int32_t) * (size_t)(m > 0 ? m : 1));
    int32_t *queue = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n + 1));
    uint8_t *inU = (uint8_t *)calloc((size_t)n + 1, 1);
    int32_t *widx = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n + 1));
    if (!cnt || !roff || !radj || !queue || !inU || !widx) {
        free(cnt); free(roff); free(radj); free(queue); free(inU); free(widx);
        return O2_ENOMEM;
    }
    for (int32_t v = 0; v < n; v++) inU[v] = own[v] == 1;
    /* reverse adjacency */
    for (int64_t e = 0; e < m; e++) roff[tgt[e] + 1]++;
    for (int32_t v = 0; v < n; v++) roff[v + 1] += roff[v];
    {
        int32_t *fill = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n + 1));
        if (!fill) { free(cnt); free(roff); free(radj); free(queue); free(inU); free(widx); return O2_ENOMEM; }
        memcpy(fill, roff, sizeof(int32_t) * (size_t)n);
        for (int32_t v = 0; v < n; v++)
            for (int32_t e = off[v]; e < off[v + 1]; e++) radj[fill[tgt[e]]++] = v;
        free(fill);
    }
    int32_t qh = 0, qt = 0;
    for (int32_t v = 0; v < n; v++) {
        if (!inU[v]) continue;
        for (int32_t e = off[v]; e < off[v + 1]; e++) cnt[v] += inU[tgt[e]];
        if (cnt[v] == 0) queue[qt++] = v;
    }
    /* peel Odd vertices with no edge left into U (greatest fixpoint) */
    while (qh < qt) {
        int32_t x = queue[qh++];
        inU[x] = 0;
        for (int32_t r = roff[x]; r < roff[x + 1]; r++) {
            int32_t y = radj[r];
            if (inU[y] && cnt[y] > 0) {
                if (--cnt[y] == 0) queue[qt++] = y;
            }
        }
    }
    /* W: vertices of U entered by an edge from U, indexed in increasing id order */
    uint8_t *isW = (uint8_t *)calloc((size_t)n + 1, 1);
    if (!isW) { free(cnt); free(roff); free(radj); free(queue); free(inU); free(widx); return O2_ENOMEM; }
    for (int32_t v = 0; v < n; v++)
        if (inU[v])
            for (int32_t e = off[v]; e < off[v + 1]; e++)
                if (inU[tgt[e]]) isW[tgt[e]] = 1;
    int32_t k = 0;
    for (int32_t w = 0; w < n; w++) {
        widx[w] = -1;
        if (isW[w]) { dummy_of[k] = w; widx[w] = k; k++; }
    }
    /* G' */
    int32_t np_ = n + k;
    out_off[0] = 0;
    for (int32_t v = 0; v < n; v++) {
        int32_t base = out_off[v];
        for (int32_t e = off[v]; e < off[v + 1]; e++) {
            int32_t t = tgt[e];
            if (inU[v] && inU[t]) t = n + widx[t];
            out_tgt[base + (e - off[v])] = t;
        }
        out_off[v + 1] = base + (off[v + 1] - off[v]);
        out_own[v] = own[v];
        out_pri[v] = pri[v] + (dummy_zero ? 2 : 2 * k);
    }
    for (int32_t j = 0; j < k; j++) {
        int32_t d = n + j;
        out_tgt[out_off[d]] = dummy_of[j];
        out_off[d + 1] = out_off[d] + 1;
        out_own[d] = 0;
        out_pri[d] = dummy_zero ? 0 : 2 * j;
    }
    (void)np_;
    if (in_u_out) memcpy(in_u_out, inU, (size_t)n);
    *k_out = k;
    free(cnt); free(roff); free(radj); free(queue); free(inU); free(widx); free(isW);
    return O2_OK;
}

/* ------------------------------------------------------------------------ */
/* Kruskal merge order over the finite tree: a union-find whose roots carry
 * the head and tail of a linked list holding their component in ascending
 * valuation order. */
typedef struct {
    int32_t *par, *head, *tail, *next, *sz;
} o2_uf;

static int32_t uf_find(int32_t *par, int32_t x)
{
    while (par[x] != x) {
        par[x] = par[par[x]];
        x = par[x];
    }
    return x;
}

static int cmp64(const void *a, const void *b)
{
    int64_t x = *(const int64_t *)a, y = *(const int64_t *)b;
    return (x > y) - (x < y);
}

/* order[] lists vertex ids by increasing priority (computed once per game). */
static int o2_order_by_priority(int32_t n, const int32_t *pri, int32_t *order)
{
    /* counting placement when priorities are small, otherwise sort */
    int32_t pmax = -1;
    for (int32_t v = 0; v < n; v++) {
        if (pri[v] < 0) return O2_EINVAL;
        if (pri[v] > pmax) pmax = pri[v];
    }
    if ((int64_t)pmax < 4 * (int64_t)n + 16) {
        int32_t *slot = (int32_t *)malloc(sizeof(int32_t) * ((size_t)pmax + 1));
        if (!slot) return O2_ENOMEM;
        for (int32_t p = 0; p <= pmax; p++) slot[p] = -1;
        for (int32_t v = 0; v < n; v++) {
            if (slot[pri[v]] != -1) { free(slot); return O2_EINVAL; } /* repeated priority */
            slot[pri[v]] = v;
        }
        int32_t i = 0;
        for (int32_t p = 0; p <= pmax; p++)
            if (slot[p] >= 0) order[i++] = slot[p];
        free(slot);
        return O2_OK;
    }
    /* sparse priorities: sort (pri, id) pairs */
    int64_t *pairs = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    if (!pairs) return O2_ENOMEM;
    for (int32_t v = 0; v < n; v++) pairs[v] = ((int64_t)pri[v] << 32) | (uint32_t)v;
    qsort(pairs, (size_t)n, sizeof(int64_t), cmp64);
    for (int32_t i = 0; i < n; i++) {
        order[i] = (int32_t)(pairs[i] & 0xffffffff);
        if (i > 0 && (pairs[i] >> 32) == (pairs[i - 1] >> 32)) { free(pairs); return O2_EINVAL; }
    }
    free(pairs);
    return O2_OK;
}


/* ------------------------------------------------------------------------ */
/* Valuation of the profile strat (Section 3, "Valuations"; Section 5 on the
 * pseudoforest): the play from v follows strat until it reaches the sink
 * (finite valuation) or repeats a vertex (top). For top vertices dom[v] is the
 * largest priority on the cycle the play ends in; an odd one means sigma was
 * not admissible. Writes cls, depth (|P(v)|, -1 for top), rank (position
 * among finite valuations and the sink's empty valuation; INT32_MAX for top)
 * and the sink's rank. Scratch is allocated here. */
int o2_valuate(int32_t n, const int32_t *pri, const int32_t *order, const int32_t *strat,
               int8_t *cls, int32_t *depth, int32_t *rank, int32_t *dom, int32_t *sink_rank,
               int32_t *n_fin_out, int32_t *n_oddcycle_out)
{
    int32_t S = n; /* sink id */
    int8_t *state = (int8_t *)malloc((size_t)n + 1); /* 0 new, 1 on stack, 2 done */
    int32_t *stack = (int32_t *)malloc(sizeof(int32_t) * ((size_t)n + 1));
    int32_t *pos = (int32_t *)malloc(sizeof(int32_t) * ((size_t)n + 1));
    if (!state || !stack || !pos) { free(state); free(stack); free(pos); return O2_ENOMEM; }
    memset(state, 0, (size_t)n + 1);
    state[S] = 2;
    int32_t n_fin = 0, n_odd = 0;
    for (int32_t v0 = 0; v0 < n; v0++) {
        if (state[v0]) continue;
        int32_t sp = 0, x = v0;
        while (x != S && state[x] == 0) {
            state[x] = 1;
            pos[x] = sp;
            stack[sp++] = x;
            x = strat[x];
        }
        int32_t stop = sp; /* stack[0..stop) receive values from x */
        if (x != S && state[x] == 1) {
            /* the play closes a cycle: stack[pos[x]..sp) */
            int32_t mx = -1;
            for (int32_t i = pos[x]; i < sp; i++)
                if (pri[stack[i]] > mx) mx = pri[stack[i]];
            for (int32_t i = pos[x]; i < sp; i++) {
                int32_t y = stack[i];
                cls[y] = (mx % 2 == 0) ? CLS_TOP : CLS_ODDCYCLE;
                dom[y] = mx;
                depth[y] = -1;
                state[y] = 2;
            }
            stop = pos[x];
        }
        /* propagate backwards from the point reached */
        for (int32_t i = stop - 1; i >= 0; i--) {
            int32_t y = stack[i], z = strat[y];
            if (z == S) {
                cls[y] = CLS_FIN; depth[y] = 1; dom[y] = -1;
            } else if (cls[z] == CLS_FIN) {
                cls[y] = CLS_FIN; depth[y] = depth[z] + 1; dom[y] = -1;
            } else {
                cls[y] = cls[z]; depth[y] = -1; dom[y] = dom[z];
            }
            state[y] = 2;
        }
    }
    for (int32_t v = 0; v < n; v++) {
        if (cls[v] == CLS_FIN) n_fin++;
        else if (cls[v] == CLS_ODDCYCLE) n_odd++;
    }
    free(state); free(stack); free(pos);

    /* ranks: Kruskal merge order on the finite tree (including the sink) */
    int32_t *par = (int32_t *)malloc(sizeof(int32_t) * ((size_t)n + 1));
    int32_t *head = (int32_t *)malloc(sizeof(int32_t) * ((size_t)n + 1));
    int32_t *tail = (int32_t *)malloc(sizeof(int32_t) * ((size_t)n + 1));
    int32_t *next = (int32_t *)malloc(sizeof(int32_t) * ((size_t)n + 1));
    int32_t *sz = (int32_t *)malloc(sizeof(int32_t) * ((size_t)n + 1));
    if (!par || !head || !tail || !next || !sz) {
        free(par); free(head); free(tail); free(next); free(sz);
        return O2_ENOMEM;
    }
    for (int32_t v = 0; v <= n; v++) { par[v] = v; head[v] = v; tail[v] = v; next[v] = -1; sz[v] = 1; }
    for (int32_t i = 0; i < n; i++) {
        int32_t x = order[i];
        if (cls[x] != CLS_FIN) continue;
        int32_t a = uf_find(par, x), b = uf_find(par, strat[x]);
        /* a: child side (vertices reaching x through lower priorities);
         * b: parent side. The child side goes above when pri(x) is even. */
        int32_t lo_h, lo_t, hi_h, hi_t;
        if (pri[x] % 2 == 0) { lo_h = head[b]; lo_t = tail[b]; hi_h = head[a]; hi_t = tail[a]; }
        else { lo_h = head[a]; lo_t = tail[a]; hi_h = head[b]; hi_t = tail[b]; }
        next[lo_t] = hi_h;
        int32_t r = sz[a] >= sz[b] ? a : b, o = (r == a) ? b : a;
        par[o] = r;
        sz[r] += sz[o];
        head[r] = lo_h;
        tail[r] = hi_t;
    }
    int32_t root = uf_find(par, S), k = 0;
    for (int32_t y = head[root]; y != -1; y = next[y]) {
        if (y == S) *sink_rank = k;
        else rank[y] = k;
        k++;
    }
    for (int32_t v = 0; v < n; v++)
        if (cls[v] != CLS_FIN) rank[v] = INT32_MAX;
    free(par); free(head); free(tail); free(next); free(sz);
    if (k != n_fin + 1) return O2_ECHECK;
    if (n_fin_out) *n_fin_out = n_fin;
    if (n_oddcycle_out) *n_oddcycle_out = n_odd;
    return O2_OK;
}

/* Literal comparison of Val(u) and Val(w) for finite u, w (or the sink),
 * by walking both plays to their meeting point (Section 3, Maxdiff): returns
 * -1 if Val(u) is below Val(w), 0 if equal, +1 if above. */
int o2_compare(int32_t n, const int32_t *pri, const int32_t *strat, const int32_t *depth, int32_t u, int32_t w)
{
    int32_t du = (u == n) ? 0 : depth[u], dw = (w == n) ? 0 : depth[w];
    int32_t mu = -1, mw = -1, xu = -1, xw = -1; /* max priority (and its vertex) on each arm */
    while (du > dw) { if (pri[u] > mu) { mu = pri[u]; xu = u; } u = strat[u]; du--; }
    while (dw > du) { if (pri[w] > mw) { mw = pri[w]; xw = w; } w = strat[w]; dw--; }
    while (u != w) {
        if (pri[u] > mu) { mu = pri[u]; xu = u; }
        if (pri[w] > mw) { mw = pri[w]; xw = w; }
        u = strat[u]; w = strat[w];
    }
    (void)xu; (void)xw;
    if (mu < 0 && mw < 0) return 0;
    if (mu > mw) return (mu % 2 == 0) ? 1 : -1;
    return (mw % 2 == 0) ? -1 : 1;
}

/* key for switching: rank for finite vertices and the sink, above all for top */
static inline int64_t o2_key(int32_t n, const int32_t *rank, const int8_t *cls, int32_t sink_rank, int32_t x)
{
    if (x == n) return sink_rank;
    return cls[x] == CLS_FIN ? (int64_t)rank[x] : (int64_t)INT32_MAX + 1;
}

/* One round of switching for one player (Section 3, "Switching rules" for
 * Even; Section 4, All_Odd for Odd). Returns the number of switched vertices.
 * With check != 0 every decision between two finite candidates is recomputed
 * by o2_compare and a disagreement makes the count negative. */
static int64_t o2_switch(const o2_game *g, int player, const int32_t *strat, int32_t *next_strat,
                         const int8_t *cls, const int32_t *depth, const int32_t *rank, int32_t sink_rank,
                         int check)
{
    int32_t n = g->n;
    int64_t nsw = 0;
    memcpy(next_strat, strat, sizeof(int32_t) * (size_t)n);
    int bad = 0;
    for (int32_t v = 0; v < n; v++) {
        if (g->own[v] != player) continue;
        int32_t best;
        int64_t bk;
        int32_t e0 = g->off[v], e1 = g->off[v + 1];
        if (player == 0) { best = n; bk = o2_key(n, rank, cls, sink_rank, n); }
        else { best = g->tgt[e0]; bk = o2_key(n, rank, cls, sink_rank, best); e0++; }
        for (int32_t e = e0; e < e1; e++) {
            int32_t u = g->tgt[e];
            int64_t ku = o2_key(n, rank, cls, sink_rank, u);
            int better = (player == 0) ? (ku > bk) : (ku < bk);
            if (check && ku <= INT32_MAX && bk <= INT32_MAX) {
                int c = o2_compare(n, g->pri, strat, depth, u, best);
                int expect = (ku > bk) - (ku < bk);
                if (c != expect) bad = 1;
            }
            if (better) { best = u; bk = ku; }
        }
        int64_t cur = o2_key(n, rank, cls, sink_rank, strat[v]);
        int improves = (player == 0) ? (bk > cur) : (bk < cur);
        if (improves) {
            next_strat[v] = best;
            nsw++;
        }
    }
    return bad ? -1 : nsw;
}

/* Algorithm 1 (Section 4): the inner loop computes a best response to sigma
 * by one-player strategy improvement for Odd; the outer loop switches Even
 * with the greedy all-switches rule using the last inner valuation.
 * strat holds the initial profile on entry (callers pass sigma_init and the
 * first-edge tau for a cold start) and the final profile on exit.
 * mode 0: full solve; mode 1: best response only (inner loop); mode 2: full
 * solve in which every best-response computation starts again from the
 * initial Odd strategy (the first edge of each list), the "SI-Reset" variant
 * of Section 6.
 * stats (nullable): per inner iteration {n_fin, max_depth, sum_depth_lo32, n_odd_switch}.
 */
int o2_run(int32_t n, const int32_t *off, const int32_t *tgt, const uint8_t *own, const int32_t *pri,
           int32_t *strat, int mode, int64_t max_inner, int check,
           int8_t *cls, int32_t *depth, int32_t *rank, int32_t *dom, int32_t *sink_rank,
           int64_t *major_out, int64_t *inner_out, int64_t *stats, int64_t stats_cap)
{
    o2_game g = {n, off, tgt, own, pri};
    int32_t *order = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int32_t *nstrat = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    if (!order || !nstrat) { free(order); free(nstrat); return O2_ENOMEM; }
    int rc = o2_order_by_priority(n, pri, order);
    if (rc) { free(order); free(nstrat); return rc; }
    int64_t major = 0, inner = 0;
    rc = O2_OK;
    for (;;) {
        for (;;) {
            if (inner >= max_inner) { rc = O2_ETIMEOUT; goto done; }
            int32_t nfin = 0, nodd = 0;
            rc = o2_valuate(n, pri, order, strat, cls, depth, rank, dom, sink_rank, &nfin, &nodd);
            if (rc) goto done;
            if (nodd) { rc = O2_ENOTADMISSIBLE; goto done; }
            int64_t nsw = o2_switch(&g, 1, strat, nstrat, cls, depth, rank, *sink_rank, check);
            if (nsw < 0) { rc = O2_ECHECK; goto done; }
            memcpy(strat, nstrat, sizeof(int32_t) * (size_t)n);
            if (stats && inner < stats_cap) {
                int64_t md = 0, sd = 0;
                for (int32_t v = 0; v < n; v++)
                    if (cls[v] == CLS_FIN) { sd += depth[v]; if (depth[v] > md) md = depth[v]; }
                stats[4 * inner + 0] = nfin;
                stats[4 * inner + 1] = md;
                stats[4 * inner + 2] = sd;
                stats[4 * inner + 3] = nsw;
            }
            inner++;
            if (nsw == 0) break;
        }
        if (mode == 1) break;
        int64_t nsw = o2_switch(&g, 0, strat, nstrat, cls, depth, rank, *sink_rank, check);
        if (nsw < 0) { rc = O2_ECHECK; goto done; }
        memcpy(strat, nstrat, sizeof(int32_t) * (size_t)n);
        if (nsw == 0) break;
        major++;
        if (mode == 2)
            for (int32_t v = 0; v < n; v++)
                if (own[v]) strat[v] = tgt[off[v]];
    }
done:
    *major_out = major;
    *inner_out = inner;
    free(order);
    free(nstrat);
    return rc;
}

/* Valuation of a given profile only (no switching). */
int o2_valuate_profile(int32_t n, const int32_t *pri, const int32_t *strat, int8_t *cls, int32_t *depth,
                       int32_t *rank, int32_t *dom, int32_t *sink_rank)
{
    int32_t *order = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    if (!order) return O2_ENOMEM;
    int rc = o2_order_by_priority(n, pri, order);
    if (!rc) rc = o2_valuate(n, pri, order, strat, cls, depth, rank, dom, sink_rank, NULL, NULL);
    free(order);
    return rc;
}
