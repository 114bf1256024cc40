// Batches: many games solved together in one id space (pg_solve_batch).
//
// Every game is loaded as usual (validation, the admissibility preprocessing
// of Section 3, relabelling), then copied into the packed layout: game i's
// relabelled vertices occupy ids [B_i, B_i + n_i'), its sink slot is
// B_i + n_i', and its edges [E_i, E_i + m_i'). Each pass of Algorithm 1 then
// runs once over all games; each game keeps its own state on the device and
// follows exactly the trajectory it would follow alone.
#include <string.h>

#include <atomic>
#include <chrono>
#include <thread>

#include "pg_internal.cuh"

// Loader threads of a batch (each with its own stream).
#ifndef PG_LOADERS
#define PG_LOADERS 8
#endif

namespace pg {
namespace {

template <typename OffT>
__global__ void k_pack(int32_t np, int64_t mp, int32_t B, int64_t E, int32_t gi, int64_t o0, int32_t n0, int32_t k,
                       int32_t d0, const int32_t* __restrict__ off_i, const int32_t* __restrict__ tgt_i,
                       const uint8_t* __restrict__ flags_i, const int32_t* __restrict__ pri_i,
                       const int32_t* __restrict__ orig_i, const int32_t* __restrict__ nid0_i,
                       const int32_t* __restrict__ dnid_i, const int32_t* __restrict__ dummy_i, OffT* off, int32_t* tgt,
                       uint8_t* flags, int32_t* pri, int32_t* orig, int32_t* nid0, int32_t* dnid, int32_t* dummy,
                       int32_t* vgame, int32_t* strat) {
    int64_t span = (int64_t)np + 1;
    if (mp > span) span = mp;
    if (n0 > span) span = n0;
    if (k > span) span = k;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < span; t += (int64_t)gridDim.x * blockDim.x) {
        if (t <= np) {
            off[B + t] = (OffT)(E + off_i[t]);
            flags[B + t] = flags_i[t];
            pri[B + t] = pri_i[t];
            orig[B + t] = orig_i[t];
            vgame[B + t] = gi;
            if (t == np) strat[B + t] = B + np;  // the sink slot points at itself (never read)
        }
        if (t < mp) tgt[E + t] = B + tgt_i[t];
        if (t < n0) nid0[o0 + t] = B + nid0_i[t];
        if (t < k) {
            dnid[d0 + t] = B + dnid_i[t];
            dummy[d0 + t] = dummy_i[t];
        }
    }
}

template <typename OffT>
__global__ void k_pack_last(OffT* off, int64_t N, int64_t M) {
    off[N] = (OffT)M;
}

inline unsigned grid_of(int64_t n) {
    int64_t b = (n + kBlock - 1) / kBlock;
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(b, 152 * 32));
}

}  // namespace

pg_status pack_games(pg_ctx* ctx, pg_game** games, int32_t ngames, pg_game** out) {
    *out = nullptr;
    cudaStream_t s = ctx->stream;
    int64_t N = 0, M = 0, n0 = 0;
    int64_t K = 0;
    for (int32_t i = 0; i < ngames; ++i) {
        N += games[i]->n;  // G' vertices plus the sink slot
        M += games[i]->m;
        n0 += games[i]->n0;
        K += games[i]->k;
    }
    if (N >= (1ll << 30) - 1) return fail(ctx, PG_EUNSUPPORTED, "pg_solve_batch: more than 2^30 vertices in the batch");
    if (K > INT32_MAX) return fail(ctx, PG_EUNSUPPORTED, "pg_solve_batch: too many dummy vertices");
    pg_game* g = new pg_game();
    g->ctx = ctx;
    g->device = ctx->device;
    g->ngames = ngames;
    g->n = (int32_t)N;
    g->m = M;
    g->n0 = n0;
    g->k = (int32_t)K;
    for (int32_t i = 0; i < ngames; ++i) g->m0 += games[i]->m0;
    const bool wide = ctx->wide_offsets || M > INT32_MAX - 1;
    auto A = [&](void** p, size_t bytes) { return dev_alloc(ctx, p, bytes, ctx->stream); };
#define PK_TRY(expr)                                                 \
    do {                                                             \
        cudaError_t _e = (expr);                                     \
        if (_e != cudaSuccess) {                                     \
            free_game(g);                                            \
            return cuda_fail(ctx, _e, #expr);                        \
        }                                                            \
    } while (0)
    if (wide) PK_TRY(A((void**)&g->off64, sizeof(int64_t) * (N + 1)));
    else PK_TRY(A((void**)&g->off, sizeof(int32_t) * (N + 1)));
    PK_TRY(A((void**)&g->tgt, sizeof(int32_t) * M));
    PK_TRY(A((void**)&g->flags, N));
    PK_TRY(A((void**)&g->pri, sizeof(int32_t) * N));
    PK_TRY(A((void**)&g->orig_of, sizeof(int32_t) * N));
    PK_TRY(A((void**)&g->nid0, sizeof(int32_t) * n0));
    PK_TRY(A((void**)&g->dnid, sizeof(int32_t) * K));
    PK_TRY(A((void**)&g->dummy_of, sizeof(int32_t) * K));
    PK_TRY(A((void**)&g->vgame, sizeof(int32_t) * N));
    PK_TRY(A((void**)&g->strat, sizeof(int32_t) * N));
    PK_TRY(A((void**)&g->gsink, sizeof(int32_t) * ngames));
    std::vector<int32_t> hsink(ngames);
    g->h_base0.assign(ngames + 1, 0);
    g->h_dbase.assign(ngames + 1, 0);
    int64_t B = 0, E = 0, o0 = 0;
    int32_t d0 = 0;
    for (int32_t i = 0; i < ngames; ++i) {
        pg_game* gi = games[i];
        const int32_t np = gi->n - 1;  // G' vertices of game i
        if (wide)
            k_pack<int64_t><<<grid_of(std::max<int64_t>(std::max<int64_t>(gi->n, gi->m), gi->n0)), kBlock, 0, s>>>(
                np, gi->m, (int32_t)B, E, i, o0, (int32_t)gi->n0, gi->k, d0, gi->off, gi->tgt, gi->flags, gi->pri,
                gi->orig_of, gi->nid0, gi->dnid, gi->dummy_of, g->off64, g->tgt, g->flags, g->pri, g->orig_of, g->nid0,
                g->dnid, g->dummy_of, g->vgame, g->strat);
        else
            k_pack<int32_t><<<grid_of(std::max<int64_t>(std::max<int64_t>(gi->n, gi->m), gi->n0)), kBlock, 0, s>>>(
                np, gi->m, (int32_t)B, E, i, o0, (int32_t)gi->n0, gi->k, d0, gi->off, gi->tgt, gi->flags, gi->pri,
                gi->orig_of, gi->nid0, gi->dnid, gi->dummy_of, g->off, g->tgt, g->flags, g->pri, g->orig_of, g->nid0,
                g->dnid, g->dummy_of, g->vgame, g->strat);
        ctx->launches += 1;
        PK_TRY(cudaGetLastError());
        hsink[i] = (int32_t)(B + np);
        B += gi->n;
        E += gi->m;
        o0 += gi->n0;
        d0 += gi->k;
        g->h_base0[i + 1] = o0;
        g->h_dbase[i + 1] = d0;
    }
    if (wide) k_pack_last<int64_t><<<1, 1, 0, s>>>(g->off64, N, M);
    else k_pack_last<int32_t><<<1, 1, 0, s>>>(g->off, N, M);
    ctx->launches += 1;
    PK_TRY(cudaMemcpyAsync(g->gsink, hsink.data(), sizeof(int32_t) * ngames, cudaMemcpyHostToDevice, s));
    PK_TRY(cudaStreamSynchronize(s));
    g->sink0 = hsink[0];
#undef PK_TRY
    for (int32_t i = 0; i < ngames; ++i) {
        free_game(games[i]);
        games[i] = nullptr;
    }
    pg_status st = alloc_scratch(g);
    if (st) {
        free_game(g);
        return st;
    }
    *out = g;
    return PG_OK;
}

}  // namespace pg

using namespace pg;

namespace {

pg_status batch_solve(pg_ctx* ctx, int32_t ngames, const int64_t* vb, const int64_t* eb, const int32_t* offsets,
                      const int32_t* targets, const uint8_t* owner, const int32_t* pri, int32_t mem_kind,
                      int64_t max_inner, pg_result_batch* out) {
    auto wall = []() { return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count(); };
    const double t0 = wall();
    std::vector<pg_game*> games(ngames, nullptr);
    auto cleanup = [&]() {
        for (pg_game* gi : games)
            if (gi) free_game(gi);
    };
    // Loading (validation, preprocessing, relabelling) is a chain of small
    // kernels and host synchronisations per game: up to kLoaders threads,
    // each with its own stream, load games concurrently so that their work
    // overlaps on the device. The first failing game (in index order) decides
    // the status.
    constexpr int kLoaders = PG_LOADERS;
    const int nload = std::max(1, std::min<int>(kLoaders, ngames));
    std::vector<pg_ctx*> lctx(nload, nullptr);
    std::vector<pg_status> gst_load(ngames, PG_OK);
    std::vector<std::string> gerr(ngames);
    for (int t = 0; t < nload; ++t) {
        pg_status st = pg_ctx_create(&lctx[t], ctx->device);
        if (st == PG_OK && cudaStreamCreateWithFlags(&lctx[t]->stream, cudaStreamNonBlocking) != cudaSuccess)
            st = PG_ECUDA;
        if (st) {
            for (pg_ctx* c : lctx)
                if (c) {
                    if (c->stream) cudaStreamDestroy(c->stream);
                    pg_ctx_destroy(c);
                }
            return fail(ctx, st, "pg_solve_batch: could not create loader streams");
        }
    }
    std::atomic<int32_t> next(0);
    auto loader = [&](int t) {
        cudaSetDevice(ctx->device);
        for (;;) {
            const int32_t i = next.fetch_add(1);
            if (i >= ngames) break;
            const int64_t ni = vb[i + 1] - vb[i], mi = eb[i + 1] - eb[i];
            pg_status st = load_game(lctx[t], (int32_t)ni, mi, offsets + vb[i] + i, targets + eb[i], owner + vb[i],
                                     pri + vb[i], mem_kind, &games[i], false);
            if (st == PG_OK && games[i]->cv) {
                st = fail(lctx[t], PG_EUNSUPPORTED,
                          "pg_solve_batch: games with repeated priorities are solved one at a time");
            }
            if (st) {
                gst_load[i] = st;
                gerr[i] = lctx[t]->err;
                next.store(ngames);  // stop the other loaders early
            }
        }
    };
    std::vector<std::thread> th;
    for (int t = 1; t < nload; ++t) th.emplace_back(loader, t);
    loader(0);
    for (auto& x : th) x.join();
    for (pg_ctx* c : lctx) {
        cudaStreamDestroy(c->stream);
        pg_ctx_destroy(c);
    }
    int64_t nmax = 0;
    for (int32_t i = 0; i < ngames; ++i) {
        if (gst_load[i] != PG_OK) {
            cleanup();
            ctx->err = gerr[i];
            return gst_load[i];
        }
        if (!games[i]) {  // not reached because another game failed first
            cleanup();
            return fail(ctx, PG_ECUDA, "pg_solve_batch: a game was not loaded");
        }
        nmax = std::max<int64_t>(nmax, games[i]->n);
    }
    const double t1 = wall();
    pg_game* g = nullptr;
    pg_status st = pack_games(ctx, games.data(), ngames, &g);
    if (st) {
        cleanup();
        return st;
    }
    struct Guard {
        pg_game* g;
        ~Guard() { free_game(g); }
    } guard{g};
    const int64_t cap = max_inner > 0 ? max_inner : 64 * (nmax + 64);
    st = apply_profile(g, nullptr, nullptr, nullptr, PG_MEM_HOST);
    if (!st) st = reset_scratch(g);
    if (st) return st;
    Timer tm(g);
    tm.mark(3);
    const double t2 = wall();
    st = run_loop(g, cap, true, tm);
    if (st) return st;
    out->load_ms = t1 - t0;
    out->pack_ms = t2 - t1;
    out->loop_ms = wall() - t2;
    std::vector<GameState> gs(ngames);
    PG_CUDA_TRY(ctx, cudaMemcpy(gs.data(), g->gst, sizeof(GameState) * ngames, cudaMemcpyDeviceToHost));
    bool any_timeout = false, any_odd = false;
    for (const GameState& x : gs) {
        any_timeout |= x.phase == kPhaseTimeout;
        any_odd |= x.phase == kPhaseOddCycle;
    }
    if (any_timeout || g->last_cmp) {  // the full valuation of the profiles being returned
        st = full_valuation(g, false);
        if (st) return st;
        g->last_cmp = false;
    }
    tm.mark(2);
    g->t_total = tm.since(3, 2);
    for (int32_t i = 0; i < ngames; ++i) {
        if (out->major) out->major[i] = gs[i].major;
        if (out->inner) out->inner[i] = gs[i].inner;
        if (out->status)
            out->status[i] = gs[i].phase == kPhaseDone ? PG_OK
                             : gs[i].phase == kPhaseTimeout ? PG_ETIMEOUT
                                                            : PG_ENOTADMISSIBLE;
    }
    if (out->dummy_base)
        for (int32_t i = 0; i <= ngames; ++i) out->dummy_base[i] = g->h_dbase[i];
    out->iterations = g->t_vals;
    st = write_outputs(g, out->mem_kind, out->win, out->sigma, out->tau, out->val_class, out->val_depth,
                       out->val_rank, nullptr, out->dummy_sigma);
    if (st) return st;
    if (any_odd) return fail(ctx, PG_ENOTADMISSIBLE, "pg_solve_batch: a game reached an odd cycle");
    if (any_timeout) return fail(ctx, PG_ETIMEOUT, "pg_solve_batch: iteration cap reached");
    return PG_OK;
}

}  // namespace

extern "C" pg_status pg_solve_batch(pg_ctx* ctx, int32_t ngames, const int64_t* vtx_base, const int64_t* edge_base,
                                    const int32_t* offsets, const int32_t* targets, const uint8_t* owner,
                                    const int32_t* pri, int32_t mem_kind, int64_t max_inner, pg_result_batch* out) {
    if (!ctx) return PG_EINVAL;
    if (ngames < 1 || !vtx_base || !edge_base || !offsets || !targets || !owner || !pri || !out)
        return fail(ctx, PG_EINVAL, "pg_solve_batch: bad arguments");
    if (mem_kind != PG_MEM_HOST && mem_kind != PG_MEM_DEVICE) return fail(ctx, PG_EINVAL, "pg_solve_batch: bad mem_kind");
    if (vtx_base[0] != 0 || edge_base[0] != 0) return fail(ctx, PG_EINVAL, "pg_solve_batch: bases must start at 0");
    for (int32_t i = 0; i < ngames; ++i) {
        if (vtx_base[i + 1] <= vtx_base[i] || edge_base[i + 1] < edge_base[i])
            return fail(ctx, PG_EINVAL, "pg_solve_batch: every game needs at least one vertex");
        if (vtx_base[i + 1] - vtx_base[i] >= (1 << 29))
            return fail(ctx, PG_EINVAL, "pg_solve_batch: a game has more than 2^29 vertices");
    }
    if (cudaSetDevice(ctx->device) != cudaSuccess) return fail(ctx, PG_ECUDA, "cudaSetDevice failed");
    return batch_solve(ctx, ngames, vtx_base, edge_base, offsets, targets, owner, pri, mem_kind, max_inner, out);
}
