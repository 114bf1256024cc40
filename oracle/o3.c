/*
 * Count-vector CPU oracle (O-3) for greedy all-switches strategy improvement
 * on games whose priorities may repeat (Fearnley, "Efficient Parallel
 * Strategy Improvement for Parity Games", arXiv 1705.02313).
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product path may call, link or
 * load this file; only tests, the smoke check and the CPU-baseline leg of the
 * benchmark use it. It shares no code with the CUDA path.
 *
 * It is the definition written out: a finite valuation is the count vector
 * L(p) of Section 3 ("Valuations": how often each priority occurs on the play
 * from v to the sink, v included, the sink not), a play that never reaches
 * the sink is top, and two finite valuations are compared by Maxdiff (same
 * paragraph): at the largest priority where the counts differ, more is
 * better if it is even, fewer is better if it is odd. The switching rules
 * (Section 3 for Even, All_Odd of Section 4 for Odd) and Algorithm 1 follow,
 * with the conventions of the other oracle tiers: strictly better only, the
 * lowest edge-list position among equals, the sink looked at first by Even,
 * the first edge as the initial Odd strategy. Plain C, one thread; memory
 * n x d counts, so intended for few distinct priorities (or small n).
 *
 * The game passed in is already preprocessed (G'); the sink has id n.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define O3_OK 0
#define O3_EINVAL 1
#define O3_ENOMEM 2
#define O3_ETIMEOUT 3
#define O3_ENOTADMISSIBLE 4

#define CLS_FIN 0
#define CLS_TOP 1
#define CLS_ODDCYCLE 2

typedef struct {
    int32_t n, d;
    const int32_t *off, *tgt;
    const uint8_t *own;
    const int32_t *lvl;    /* level of each vertex: index of its priority among the distinct priorities, ascending */
    const uint8_t *lodd;   /* parity of each level's priority */
    const int32_t *pri;
} o3_game;

/* Levels: the distinct priorities in ascending order. */
static int cmp_i32(const void *a, const void *b)
{
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return x < y ? -1 : x > y;
}

int o3_levels(int32_t n, const int32_t *pri, int32_t *lvl, int32_t *level_pri, int32_t *d_out)
{
    int32_t *s = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    if (!s) return O3_ENOMEM;
    memcpy(s, pri, sizeof(int32_t) * (size_t)n);
    qsort(s, (size_t)n, sizeof(int32_t), cmp_i32);
    int32_t d = 0;
    for (int32_t i = 0; i < n; i++)
        if (i == 0 || s[i] != s[i - 1]) s[d++] = s[i];
    for (int32_t v = 0; v < n; v++) {
        int32_t lo = 0, hi = d - 1;
        while (lo < hi) {
            int32_t mid = (lo + hi) / 2;
            if (s[mid] < pri[v]) lo = mid + 1;
            else hi = mid;
        }
        lvl[v] = lo;
    }
    if (level_pri) memcpy(level_pri, s, sizeof(int32_t) * (size_t)d);
    *d_out = d;
    free(s);
    return O3_OK;
}

/* Maxdiff comparison of Section 3 on two count vectors: -1 if a is worse for
 * Even than b, 0 if equal, 1 if better. Top (NULL) is above every vector. */
static int cmp_val(const o3_game *g, const int32_t *a, const int32_t *b)
{
    if (!a || !b) return (!a && !b) ? 0 : (!a ? 1 : -1);
    for (int32_t l = g->d - 1; l >= 0; l--) {
        if (a[l] == b[l]) continue;
        int more = a[l] > b[l];
        return g->lodd[l] ? (more ? -1 : 1) : (more ? 1 : -1);
    }
    return 0;
}

/* Valuation of every vertex under strat: class, dominant priority of the
 * cycle reached (top) or -1, depth (vertices on the play to the sink) and
 * the count vector (cnt[v * d + level]). Returns the number of vertices whose
 * play reaches a cycle of odd largest priority. */
static int64_t valuate(const o3_game *g, const int32_t *strat, int8_t *cls, int32_t *dom, int32_t *depth,
                       int32_t *cnt, int32_t *state, int32_t *path)
{
    const int32_t n = g->n, d = g->d;
    int64_t nodd = 0;
    for (int32_t v = 0; v < n; v++) state[v] = 0; /* 0 unseen, 1 on the current path, 2 done */
    for (int32_t v0 = 0; v0 < n; v0++) {
        if (state[v0]) continue;
        int32_t len = 0, x = v0;
        while (x != n && state[x] == 0) {
            state[x] = 1;
            path[len++] = x;
            x = strat[x];
        }
        int32_t stop = len;  /* path[0 .. stop) take their values from x */
        if (x != n && state[x] == 1) {
            /* a new cycle: from x to the end of the path */
            int32_t first = 0;
            while (path[first] != x) first++;
            int32_t best = -1;
            for (int32_t i = first; i < len; i++)
                if (best < 0 || g->pri[path[i]] > best) best = g->pri[path[i]];
            const int8_t c = (best & 1) ? CLS_ODDCYCLE : CLS_TOP;
            for (int32_t i = first; i < len; i++) {
                cls[path[i]] = c;
                dom[path[i]] = best;
                depth[path[i]] = -1;
                state[path[i]] = 2;
            }
            stop = first;
        }
        for (int32_t i = stop - 1; i >= 0; i--) {
            const int32_t y = path[i], s = strat[y];
            state[y] = 2;
            if (s != n && cls[s] != CLS_FIN) {
                cls[y] = cls[s];
                dom[y] = dom[s];
                depth[y] = -1;
                continue;
            }
            cls[y] = CLS_FIN;
            dom[y] = -1;
            int32_t *cy = cnt + (int64_t)y * d;
            if (s == n) {
                memset(cy, 0, sizeof(int32_t) * (size_t)d);
                depth[y] = 1;
            } else {
                memcpy(cy, cnt + (int64_t)s * d, sizeof(int32_t) * (size_t)d);
                depth[y] = depth[s] + 1;
            }
            cy[g->lvl[y]] += 1;
        }
    }
    for (int32_t v = 0; v < n; v++) nodd += cls[v] == CLS_ODDCYCLE;
    return nodd;
}

static const int32_t *val_of(const o3_game *g, const int8_t *cls, const int32_t *cnt, const int32_t *zero,
                             int32_t u)
{
    if (u == g->n) return zero;  /* the sink: the empty valuation */
    return cls[u] == CLS_FIN ? cnt + (int64_t)u * g->d : NULL;
}

/* One switching pass for player (0 Even, 1 Odd) into next; returns the number of switches. */
static int64_t switch_pass(const o3_game *g, int player, const int32_t *strat, int32_t *next, const int8_t *cls,
                           const int32_t *cnt, const int32_t *zero)
{
    int64_t nsw = 0;
    for (int32_t v = 0; v < g->n; v++) {
        next[v] = strat[v];
        if (g->own[v] != player) continue;
        int32_t best = -1;
        const int32_t *bv = NULL;
        int have = 0;
        if (player == 0) {
            best = g->n;
            bv = zero;
            have = 1;
        }
        for (int32_t e = g->off[v]; e < g->off[v + 1]; e++) {
            const int32_t u = g->tgt[e];
            const int32_t *uv = val_of(g, cls, cnt, zero, u);
            const int c = have ? cmp_val(g, uv, bv) : 0;
            if (!have || (player == 0 ? c > 0 : c < 0)) {
                best = u;
                bv = uv;
                have = 1;
            }
        }
        const int32_t *cur = val_of(g, cls, cnt, zero, strat[v]);
        const int c = cmp_val(g, bv, cur);
        if (player == 0 ? c > 0 : c < 0) {
            next[v] = best;
            nsw++;
        }
    }
    return nsw;
}

/* Algorithm 1 (Section 4). mode 0: solve; 1: best response (inner loop
 * only); 2: solve with SI-Reset (Section 6: every best response starts
 * again from the first edge of each Odd list). strat holds the initial
 * profile on entry and the final one on exit; the outputs describe the
 * valuation of the final profile (as of its last computation). level_pri
 * (d entries) and cnt (n x d) are outputs; d_out receives d. */
int o3_run(int32_t n, const int32_t *off, const int32_t *tgt, const uint8_t *own, const int32_t *pri, int32_t *strat,
           int mode, int64_t max_inner, int8_t *cls, int32_t *depth, int32_t *dom, int32_t *cnt, int32_t *level_pri,
           int32_t *d_out, int64_t *major_out, int64_t *inner_out)
{
    int32_t *lvl = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int32_t *lp = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int32_t *state = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int32_t *path = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int32_t *next = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    uint8_t *lodd = (uint8_t *)malloc((size_t)(n > 0 ? n : 1));
    int rc = O3_OK;
    int32_t d = 0;
    int32_t *zero = NULL;
    int64_t major = 0, inner = 0;
    if (!lvl || !lp || !state || !path || !next || !lodd) { rc = O3_ENOMEM; goto done; }
    rc = o3_levels(n, pri, lvl, lp, &d);
    if (rc) goto done;
    for (int32_t l = 0; l < d; l++) lodd[l] = (uint8_t)(lp[l] & 1);
    zero = (int32_t *)calloc((size_t)(d > 0 ? d : 1), sizeof(int32_t));
    if (!zero) { rc = O3_ENOMEM; goto done; }
    o3_game g = {n, d, off, tgt, own, lvl, lodd, pri};
    for (;;) {
        for (;;) {
            if (inner >= max_inner) { rc = O3_ETIMEOUT; goto done; }
            if (valuate(&g, strat, cls, dom, depth, cnt, state, path)) { rc = O3_ENOTADMISSIBLE; goto done; }
            inner++;
            const int64_t nsw = switch_pass(&g, 1, strat, next, cls, cnt, zero);
            memcpy(strat, next, sizeof(int32_t) * (size_t)n);
            if (nsw == 0) break;
        }
        if (mode == 1) break;
        const int64_t nsw = switch_pass(&g, 0, strat, next, cls, cnt, zero);
        memcpy(strat, next, sizeof(int32_t) * (size_t)n);
        if (nsw == 0) break;
        major++;
        if (mode == 2)
            for (int32_t v = 0; v < n; v++)
                if (own[v]) strat[v] = tgt[off[v]];
    }
done:
    if (rc == O3_OK || rc == O3_ETIMEOUT || rc == O3_ENOTADMISSIBLE) {
        if (level_pri) memcpy(level_pri, lp, sizeof(int32_t) * (size_t)d);
        *d_out = d;
    }
    *major_out = major;
    *inner_out = inner;
    free(lvl); free(lp); free(state); free(path); free(next); free(lodd); free(zero);
    return rc;
}

/* The valuation of one profile (no switching). */
int o3_valuate_profile(int32_t n, const int32_t *off, const int32_t *tgt, const uint8_t *own, const int32_t *pri,
                       const int32_t *strat, int8_t *cls, int32_t *depth, int32_t *dom, int32_t *cnt,
                       int32_t *level_pri, int32_t *d_out)
{
    int32_t *lvl = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int32_t *state = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int32_t *path = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    uint8_t *lodd = (uint8_t *)malloc((size_t)(n > 0 ? n : 1));
    int rc = O3_OK;
    int32_t d = 0;
    if (!lvl || !state || !path || !lodd) { rc = O3_ENOMEM; goto done; }
    rc = o3_levels(n, pri, lvl, level_pri, &d);
    if (rc) goto done;
    for (int32_t l = 0; l < d; l++) lodd[l] = (uint8_t)(level_pri[l] & 1);
    o3_game g = {n, d, off, tgt, own, lvl, lodd, pri};
    if (valuate(&g, strat, cls, dom, depth, cnt, state, path)) rc = O3_ENOTADMISSIBLE;
    *d_out = d;
done:
    free(lvl); free(state); free(path); free(lodd);
    return rc;
}
