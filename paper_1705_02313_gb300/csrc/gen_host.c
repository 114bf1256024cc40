/* Multithreaded host generator for random parity games.
 *
 * Produces exactly the games of gen.random_game (same SplitMix64 counter-based
 * draws, same redraw rule for repeated targets, same priority permutation),
 * but in C with one worker thread per core, so that batches of thousands of
 * games (billions of edges) can be generated in seconds. It holds none of the
 * solver's arithmetic: it only writes inputs.
 *
 * SplitMix64 is the generator of Steele, Lea and Flood ("Fast splittable
 * pseudorandom number generators", OOPSLA 2014), output function as published
 * by Vigna; draw(seed, stream, index, j) keys it by a counter as gen.draw does.
 *
 * Layout of a packed batch (the pg_solve_batch input layout): game i has
 * vertices vtx_base[i] .. vtx_base[i+1] of owner and pri, edges edge_base[i] ..
 * edge_base[i+1] of targets (local ids), and n_i + 1 local CSR offsets starting
 * at offsets[vtx_base[i] + i].
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define S_DEGREE 1
#define S_TARGET 2
#define S_OWNER 3
#define S_PRIORITY 4

static inline uint64_t sm64(uint64_t z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static inline uint64_t stream_key(uint64_t seed, uint64_t stream) { return sm64(seed ^ (stream << 56)); }

/* draw(seed, stream, index, j) with k = stream_key(seed, stream) */
static inline uint64_t draw_k(uint64_t k, uint64_t index, uint64_t j) { return sm64(sm64(k ^ index) ^ j); }

static inline uint64_t below(uint64_t bits, uint64_t n) { return ((bits >> 32) * n) >> 32; }

typedef struct {
    int64_t n;
    int64_t dmin, dmax; /* already capped at n */
    uint64_t seed;
} game_spec;

static game_spec make_spec(int64_t n, int64_t dmin, int64_t dmax, uint64_t seed) {
    game_spec s;
    s.n = n;
    s.dmin = dmin < n ? dmin : n;
    s.dmax = dmax < n ? dmax : n;
    s.seed = seed;
    return s;
}

static inline int64_t degree_of(const game_spec* s, uint64_t kdeg, int64_t v) {
    return s->dmin + (int64_t)below(draw_k(kdeg, (uint64_t)v, 0), (uint64_t)(s->dmax - s->dmin + 1));
}

static int64_t edge_count(const game_spec* s) {
    const uint64_t kdeg = stream_key(s->seed, S_DEGREE);
    int64_t m = 0;
    for (int64_t v = 0; v < s->n; ++v) m += degree_of(s, kdeg, v);
    return m;
}

/* Stable LSD radix sort of (key, index) pairs by key, 16-bit digits. */
typedef struct {
    uint64_t key;
    int64_t v;
} kv;

static int radix_sort(kv* a, int64_t n) {
    kv* b = (kv*)malloc((size_t)(n > 0 ? n : 1) * sizeof(kv));
    int64_t* cnt = (int64_t*)malloc(65536 * sizeof(int64_t));
    if (!b || !cnt) {
        free(b);
        free(cnt);
        return -1;
    }
    for (int pass = 0; pass < 4; ++pass) {
        const int sh = 16 * pass;
        memset(cnt, 0, 65536 * sizeof(int64_t));
        for (int64_t i = 0; i < n; ++i) ++cnt[(a[i].key >> sh) & 0xFFFF];
        int64_t run = 0;
        for (int d = 0; d < 65536; ++d) {
            int64_t c = cnt[d];
            cnt[d] = run;
            run += c;
        }
        for (int64_t i = 0; i < n; ++i) b[cnt[(a[i].key >> sh) & 0xFFFF]++] = a[i];
        kv* t = a;
        a = b;
        b = t;
    }
    /* four passes: the sorted data is back in the caller's array */
    free(b);
    free(cnt);
    return 0;
}

static void insertion_sort_i64(int64_t* x, int64_t d) {
    for (int64_t i = 1; i < d; ++i) {
        int64_t y = x[i], j = i - 1;
        while (j >= 0 && x[j] > y) {
            x[j + 1] = x[j];
            --j;
        }
        x[j + 1] = y;
    }
}

/* Vertex range [v0, v1) of one game: degrees, targets, owners. off must hold
 * the game's local CSR offsets for the range already. */
static void fill_vertices(const game_spec* s, uint64_t owner_thr, int64_t v0, int64_t v1, const int32_t* off,
                          int32_t* tgt, uint8_t* owner) {
    const uint64_t kt = stream_key(s->seed, S_TARGET), ko = stream_key(s->seed, S_OWNER);
    int64_t slots[64];
    for (int64_t v = v0; v < v1; ++v) {
        const int64_t d = (int64_t)off[v + 1] - off[v];
        const uint64_t a = sm64(kt ^ (uint64_t)v);
        for (int64_t j = 0; j < d; ++j) {
            for (uint64_t r = 0;; ++r) {
                const int64_t cand = (int64_t)below(sm64(a ^ ((uint64_t)j + 64 * r)), (uint64_t)s->n);
                int dup = 0;
                for (int64_t i = 0; i < j; ++i) dup |= slots[i] == cand;
                if (!dup) {
                    slots[j] = cand;
                    break;
                }
            }
        }
        insertion_sort_i64(slots, d);
        for (int64_t j = 0; j < d; ++j) tgt[off[v] + j] = (int32_t)slots[j];
        owner[v] = draw_k(ko, (uint64_t)v, 0) < owner_thr;
    }
}

static int fill_priorities(const game_spec* s, int32_t* pri) {
    kv* a = (kv*)malloc((size_t)(s->n > 0 ? s->n : 1) * sizeof(kv));
    if (!a) return -1;
    const uint64_t kp = stream_key(s->seed, S_PRIORITY);
    for (int64_t v = 0; v < s->n; ++v) {
        a[v].key = draw_k(kp, (uint64_t)v, 0);
        a[v].v = v;
    }
    if (radix_sort(a, s->n)) {
        free(a);
        return -1;
    }
    for (int64_t r = 0; r < s->n; ++r) pri[a[r].v] = (int32_t)r;
    free(a);
    return 0;
}

static int fill_game(const game_spec* s, uint64_t owner_thr, int32_t* off, int32_t* tgt, uint8_t* owner,
                     int32_t* pri) {
    const uint64_t kdeg = stream_key(s->seed, S_DEGREE);
    int64_t run = 0;
    off[0] = 0;
    for (int64_t v = 0; v < s->n; ++v) {
        run += degree_of(s, kdeg, v);
        off[v + 1] = (int32_t)run;
    }
    fill_vertices(s, owner_thr, 0, s->n, off, tgt, owner);
    return fill_priorities(s, pri);
}

/* ---- threads ------------------------------------------------------------ */

typedef struct {
    int64_t count;
    const int64_t* sizes;
    const uint64_t* seeds;
    int64_t dmin, dmax;
    uint64_t owner_thr;
    const int64_t* vtx_base;
    const int64_t* edge_base;
    int64_t* edge_counts; /* phase 0 output */
    int32_t* offsets;
    int32_t* targets;
    uint8_t* owner;
    int32_t* pri;
    int phase; /* 0: edge counts, 1: fill */
    int64_t next;
    int err;
    pthread_mutex_t mu;
} batch_job;

static void* batch_worker(void* p) {
    batch_job* J = (batch_job*)p;
    for (;;) {
        pthread_mutex_lock(&J->mu);
        const int64_t i = J->next++;
        pthread_mutex_unlock(&J->mu);
        if (i >= J->count) break;
        game_spec s = make_spec(J->sizes[i], J->dmin, J->dmax, J->seeds[i]);
        if (J->phase == 0) {
            J->edge_counts[i] = edge_count(&s);
        } else {
            const int64_t vb = J->vtx_base[i], eb = J->edge_base[i];
            if (fill_game(&s, J->owner_thr, J->offsets + vb + i, J->targets + eb, J->owner + vb, J->pri + vb)) {
                pthread_mutex_lock(&J->mu);
                J->err = 1;
                pthread_mutex_unlock(&J->mu);
            }
        }
    }
    return NULL;
}

static int run_batch(batch_job* J, int nthreads) {
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    if (nthreads > J->count) nthreads = J->count > 0 ? (int)J->count : 1;
    pthread_t th[256];
    J->next = 0;
    J->err = 0;
    pthread_mutex_init(&J->mu, NULL);
    int started = 0;
    for (int t = 1; t < nthreads; ++t) {
        if (pthread_create(&th[t], NULL, batch_worker, J) != 0) break;
        ++started;
    }
    batch_worker(J);
    for (int t = 1; t <= started; ++t) pthread_join(th[t], NULL);
    pthread_mutex_destroy(&J->mu);
    return J->err ? -1 : 0;
}

/* ---- exported ------------------------------------------------------------ */

/* Edge count of each game (sizes[i] vertices, out-degree uniform in [dmin,
 * dmax] capped at the size, seed seeds[i]). Returns 0, or -1 on bad input. */
int pggen_edge_counts(int64_t count, const int64_t* sizes, const uint64_t* seeds, int64_t dmin, int64_t dmax,
                      int64_t* edge_counts, int nthreads) {
    if (count < 0 || dmin < 1 || dmax < dmin || dmax > 64) return -1;
    for (int64_t i = 0; i < count; ++i)
        if (sizes[i] < 1 || sizes[i] >= ((int64_t)1 << 31)) return -1;
    batch_job J;
    memset(&J, 0, sizeof(J));
    J.count = count;
    J.sizes = sizes;
    J.seeds = seeds;
    J.dmin = dmin;
    J.dmax = dmax;
    J.edge_counts = edge_counts;
    J.phase = 0;
    return run_batch(&J, nthreads);
}

/* Fills a packed batch (layout at the top of this file); vtx_base and
 * edge_base (count + 1 entries each) must come from the sizes and from
 * pggen_edge_counts. Vertex v of game i is Odd when its owner draw is below
 * owner_thr. Returns 0, or -1 on bad input or allocation failure. */
int pggen_fill_batch(int64_t count, const int64_t* sizes, const uint64_t* seeds, int64_t dmin, int64_t dmax,
                     uint64_t owner_thr, const int64_t* vtx_base, const int64_t* edge_base, int32_t* offsets,
                     int32_t* targets, uint8_t* owner, int32_t* pri, int nthreads) {
    if (count < 0 || dmin < 1 || dmax < dmin || dmax > 64) return -1;
    for (int64_t i = 0; i < count; ++i) {
        if (sizes[i] < 1 || sizes[i] >= ((int64_t)1 << 31)) return -1;
        if (vtx_base[i + 1] - vtx_base[i] != sizes[i]) return -1;
        if (edge_base[i + 1] - edge_base[i] > INT32_MAX) return -1;
    }
    batch_job J;
    memset(&J, 0, sizeof(J));
    J.count = count;
    J.sizes = sizes;
    J.seeds = seeds;
    J.dmin = dmin;
    J.dmax = dmax;
    J.owner_thr = owner_thr;
    J.vtx_base = vtx_base;
    J.edge_base = edge_base;
    J.offsets = offsets;
    J.targets = targets;
    J.owner = owner;
    J.pri = pri;
    J.phase = 1;
    return run_batch(&J, nthreads);
}

/* One large game with the vertex loop split across threads (targets and
 * owners); offsets[n + 1], targets[edge count], owner[n], pri[n]. */
typedef struct {
    const game_spec* s;
    uint64_t owner_thr;
    int64_t v0, v1;
    const int32_t* off;
    int32_t* tgt;
    uint8_t* owner;
} range_job;

static void* range_worker(void* p) {
    range_job* R = (range_job*)p;
    fill_vertices(R->s, R->owner_thr, R->v0, R->v1, R->off, R->tgt, R->owner);
    return NULL;
}

/* levels > 0: priorities uniform over 0 .. levels-1 instead of a permutation. */
int pggen_fill_game(int64_t n, int64_t dmin, int64_t dmax, uint64_t seed, uint64_t owner_thr, int32_t* offsets,
                    int32_t* targets, uint8_t* owner, int32_t* pri, int nthreads, int64_t levels) {
    if (n < 1 || n >= ((int64_t)1 << 31) || dmin < 1 || dmax < dmin || dmax > 64) return -1;
    game_spec s = make_spec(n, dmin, dmax, seed);
    const uint64_t kdeg = stream_key(seed, S_DEGREE);
    int64_t run = 0;
    offsets[0] = 0;
    for (int64_t v = 0; v < n; ++v) {
        run += degree_of(&s, kdeg, v);
        if (run > INT32_MAX) return -1;
        offsets[v + 1] = (int32_t)run;
    }
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    pthread_t th[256];
    range_job R[256];
    for (int t = 0; t < nthreads; ++t) {
        R[t].s = &s;
        R[t].owner_thr = owner_thr;
        R[t].v0 = n * t / nthreads;
        R[t].v1 = n * (t + 1) / nthreads;
        R[t].off = offsets;
        R[t].tgt = targets;
        R[t].owner = owner;
    }
    int created[256] = {0};
    for (int t = 1; t < nthreads; ++t) created[t] = pthread_create(&th[t], NULL, range_worker, &R[t]) == 0;
    for (int t = 1; t < nthreads; ++t)
        if (!created[t]) range_worker(&R[t]);
    /* priorities (one sort) on this thread while the workers fill edges */
    int perr = 0;
    if (levels > 0) {
        const uint64_t kp = stream_key(seed, S_PRIORITY);
        for (int64_t v = 0; v < n; ++v) pri[v] = (int32_t)below(draw_k(kp, (uint64_t)v, 0), (uint64_t)levels);
    } else {
        perr = fill_priorities(&s, pri);
    }
    range_worker(&R[0]);
    for (int t = 1; t < nthreads; ++t)
        if (created[t]) pthread_join(th[t], NULL);
    return perr;
}
