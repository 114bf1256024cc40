// Serving: a request loop with continuous batching (pg_server_*).
//
// Two threads, each with its own CUDA stream. The loader takes submitted
// games (host copies of their arrays) from a FIFO queue and loads them
// (validation, the preprocessing of Section 3, relabelling, the initial
// profile) while the worker is solving: their work overlaps on the device.
// The worker owns a packed batch allocated once at the server's capacity
// (ids, edges, games). Between rounds it retires finished games and admits
// loaded ones in arrival order while they fit; every game keeps its strategy
// profile and its loop state (Algorithm 1, Section 4: inner and major counts,
// phase) across rounds, so its trajectory, and therefore its result, is
// exactly the one pg_solve gives for it alone. A round is the device-side
// loop over all resident games for at most round_iters iterations.
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>

#include "pg_internal.cuh"

namespace pg {
namespace {

double now_us() {
    return std::chrono::duration<double, std::micro>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

inline unsigned grid_of(int64_t n) {
    int64_t b = (n + kBlock - 1) / kBlock;
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(b, 152 * 32));
}

// The default profile of Algorithm 1 on one loaded game: Even vertices and
// dummies to the sink slot, Odd vertices to their first edge.
__global__ void k_init_profile(int32_t np, const int32_t* __restrict__ off, const int32_t* __restrict__ tgt,
                               const uint8_t* __restrict__ flags, int32_t* __restrict__ strat) {
    for (int32_t v = blockIdx.x * blockDim.x + threadIdx.x; v <= np; v += gridDim.x * blockDim.x)
        strat[v] = v == np ? np : ((flags[v] & kOwnerOdd) ? tgt[off[v]] : np);
}

// One game into the packed batch at id base B, edge base E, original-vertex
// base o0 and dummy base d0; its profile comes along (local ids + B).
template <typename OffT>
__global__ void k_pack_game(int32_t np, int64_t mp, int32_t B, int64_t E, int32_t gi, int64_t o0, int32_t n0,
                            int32_t k, int64_t d0, const int32_t* __restrict__ off_i, const int32_t* __restrict__ tgt_i,
                            const uint8_t* __restrict__ flags_i, const int32_t* __restrict__ pri_i,
                            const int32_t* __restrict__ orig_i, const int32_t* __restrict__ nid0_i,
                            const int32_t* __restrict__ dnid_i, const int32_t* __restrict__ dummy_i,
                            const int32_t* __restrict__ strat_i, OffT* off, int32_t* tgt, uint8_t* flags, int32_t* pri,
                            int32_t* orig, int32_t* nid0, int32_t* dnid, int32_t* dummy, int32_t* vgame,
                            int32_t* strat) {
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
            strat[B + t] = B + strat_i[t];
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
__global__ void k_pack_end(OffT* off, int64_t N, int64_t M) {
    off[N] = (OffT)M;
}

// A game's profile back out of the packed batch (local ids).
__global__ void k_unpack_profile(int32_t np, int32_t B, const int32_t* __restrict__ strat, int32_t* __restrict__ strat_i) {
    for (int32_t t = blockIdx.x * blockDim.x + threadIdx.x; t <= np; t += gridDim.x * blockDim.x)
        strat_i[t] = strat[B + t] - B;
}

struct Pending {
    uint64_t tag;
    int32_t n;
    int64_t m;
    std::vector<int32_t> off, tgt, pri;
    std::vector<uint8_t> own;
    double t_submit;
};

struct Resident {
    uint64_t tag;
    pg_game* g;  // the game's own G' arrays; its strat holds the profile while the game is not packed
    GameState st;
    double t_submit, t_admit;
    int32_t slot;  // index in the packed batch (valid while packed)
};

struct Done {
    pg_status status;
    int32_t n, k;
    int64_t major, inner;
    double t_submit, t_admit, t_done;
    std::vector<uint8_t> win;
    std::vector<int32_t> sigma, tau, depth, rank;
    std::vector<int8_t> cls, dsig;
};

}  // namespace
}  // namespace pg

using namespace pg;

struct pg_server {
    pg_ctx* ctx = nullptr;   // the worker's
    pg_ctx* lctx = nullptr;  // the loader's
    pg_server_opts opts{};
    std::thread worker, loader;
    std::mutex mu;
    std::condition_variable cv_work, cv_done, cv_load;
    std::deque<Pending> queue;       // submitted, not loaded
    std::deque<Resident> ready;      // loaded, not admitted
    int64_t ready_ids = 0;
    std::map<uint64_t, int> inflight;  // tags of resident games (for duplicate checks)
    std::map<uint64_t, Done> done;
    std::deque<uint64_t> done_order;  // completion order, not yet reported by pg_server_poll
    bool stop = false;
    pg_status fatal = PG_OK;
    std::string fatal_msg;
    pg_server_stats stats{};
    // worker-only state
    std::vector<Resident> res;
    size_t packed_count = 0;  // res[0 .. packed_count) are laid out in the packed batch
    pg_game* B = nullptr;  // packed batch at capacity
    int64_t capN = 0, capM = 0;
    int32_t capG = 0;
    void* stage = nullptr;  // device staging of finished games' outputs (grown as needed)
    size_t stage_size = 0;
};

namespace {

pg_status alloc_batch(pg_server* sv) {
    pg_ctx* ctx = sv->ctx;
    pg_game* g = new pg_game();
    g->ctx = ctx;
    g->device = ctx->device;
    g->ngames = sv->capG;
    g->n = (int32_t)sv->capN;
    g->m = sv->capM;
    sv->B = g;
    auto A = [&](void** p, size_t bytes) { return dev_alloc(ctx, p, bytes, ctx->stream); };
    const int64_t N = sv->capN, M = sv->capM;
    if (sv->opts.wide_offsets || M > INT32_MAX - 1) PG_CUDA_TRY(ctx, A((void**)&g->off64, sizeof(int64_t) * (N + 1)));
    else PG_CUDA_TRY(ctx, A((void**)&g->off, sizeof(int32_t) * (N + 1)));
    PG_CUDA_TRY(ctx, A((void**)&g->tgt, sizeof(int32_t) * M));
    PG_CUDA_TRY(ctx, A((void**)&g->flags, N));
    PG_CUDA_TRY(ctx, A((void**)&g->pri, sizeof(int32_t) * N));
    PG_CUDA_TRY(ctx, A((void**)&g->orig_of, sizeof(int32_t) * N));
    PG_CUDA_TRY(ctx, A((void**)&g->nid0, sizeof(int32_t) * N));
    PG_CUDA_TRY(ctx, A((void**)&g->dnid, sizeof(int32_t) * N));
    PG_CUDA_TRY(ctx, A((void**)&g->dummy_of, sizeof(int32_t) * N));
    PG_CUDA_TRY(ctx, A((void**)&g->vgame, sizeof(int32_t) * N));
    PG_CUDA_TRY(ctx, A((void**)&g->strat, sizeof(int32_t) * N));
    PG_CUDA_TRY(ctx, A((void**)&g->gsink, sizeof(int32_t) * sv->capG));
    return alloc_scratch(g);
}

void set_fatal(pg_server* sv, pg_status st, pg_ctx* from) {
    std::lock_guard<std::mutex> lk(sv->mu);
    if (sv->fatal == PG_OK) {
        sv->fatal = st;
        sv->fatal_msg = from->err;
    }
    sv->cv_done.notify_all();
    sv->cv_work.notify_all();
    sv->cv_load.notify_all();
}

void finish_pending_error(pg_server* sv, const Pending& p, pg_status st) {
    Done d{};
    d.status = st;
    d.n = p.n;
    d.t_submit = p.t_submit;
    d.t_admit = d.t_done = now_us();
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->inflight.erase(p.tag);
    sv->done[p.tag] = std::move(d);
    sv->done_order.push_back(p.tag);
    sv->stats.completed += 1;
    sv->cv_done.notify_all();
}

// Packs the resident games into the batch (their profiles and states included).
pg_status repack(pg_server* sv) {
    pg_ctx* ctx = sv->ctx;
    pg_game* g = sv->B;
    cudaStream_t s = ctx->stream;
    const bool wide = g->off64 != nullptr;
    int64_t Bb = 0, E = 0, o0 = 0, d0 = 0;
    std::vector<int32_t> hsink(sv->res.size());
    std::vector<GameState> hst(sv->res.size());
    g->h_base0.assign(sv->res.size() + 1, 0);
    g->h_dbase.assign(sv->res.size() + 1, 0);
    for (size_t i = 0; i < sv->res.size(); ++i) {
        Resident& r = sv->res[i];
        pg_game* gi = r.g;
        const int32_t np = gi->n - 1;
        const unsigned grid = grid_of(std::max<int64_t>(std::max<int64_t>(gi->n, gi->m), gi->n0));
        ctx->launches += 1;
        if (wide)
            k_pack_game<int64_t><<<grid, kBlock, 0, s>>>(
                np, gi->m, (int32_t)Bb, E, (int32_t)i, o0, (int32_t)gi->n0, gi->k, d0, gi->off, gi->tgt, gi->flags,
                gi->pri, gi->orig_of, gi->nid0, gi->dnid, gi->dummy_of, gi->strat, g->off64, g->tgt, g->flags, g->pri,
                g->orig_of, g->nid0, g->dnid, g->dummy_of, g->vgame, g->strat);
        else
            k_pack_game<int32_t><<<grid, kBlock, 0, s>>>(
                np, gi->m, (int32_t)Bb, E, (int32_t)i, o0, (int32_t)gi->n0, gi->k, d0, gi->off, gi->tgt, gi->flags,
                gi->pri, gi->orig_of, gi->nid0, gi->dnid, gi->dummy_of, gi->strat, g->off, g->tgt, g->flags, g->pri,
                g->orig_of, g->nid0, g->dnid, g->dummy_of, g->vgame, g->strat);
        PG_CUDA_TRY(ctx, cudaGetLastError());
        r.slot = (int32_t)i;
        hsink[i] = (int32_t)(Bb + np);
        hst[i] = r.st;
        Bb += gi->n;
        E += gi->m;
        o0 += gi->n0;
        d0 += gi->k;
        g->h_base0[i + 1] = o0;
        g->h_dbase[i + 1] = (int32_t)d0;
    }
    ctx->launches += 1;
    if (wide) k_pack_end<int64_t><<<1, 1, 0, s>>>(g->off64, Bb, E);
    else k_pack_end<int32_t><<<1, 1, 0, s>>>(g->off, Bb, E);
    g->ngames = (int32_t)sv->res.size();
    g->n = (int32_t)Bb;
    g->m = E;
    g->n0 = o0;
    g->k = (int32_t)d0;
    g->sink0 = hsink.empty() ? 0 : hsink[0];
    g->ntiles = std::max<int64_t>(1, (Bb + kCoopTile - 1) / kCoopTile);
    PG_CUDA_TRY(ctx, cudaMemcpyAsync(g->gsink, hsink.data(), sizeof(int32_t) * hsink.size(), cudaMemcpyHostToDevice, s));
    PG_CUDA_TRY(ctx, cudaMemcpyAsync(g->gst, hst.data(), sizeof(GameState) * hst.size(), cudaMemcpyHostToDevice, s));
    drop_loop_graphs(g);
    g->pl_ok = false;  // the switching players' views follow the new layout
    pg_status st = reset_scratch(g);
    if (st) return st;
    // reset_scratch clears the loop states: put them back
    PG_CUDA_TRY(ctx, cudaMemcpyAsync(g->gst, hst.data(), sizeof(GameState) * hst.size(), cudaMemcpyHostToDevice, s));
    PG_CUDA_TRY(ctx, cudaStreamSynchronize(s));
    return PG_OK;
}

// Profiles of the games that stay resident back into their own arrays
// (keep covers the games of the current layout, a prefix of res).
pg_status unpack_profiles(pg_server* sv, const std::vector<bool>& keep) {
    pg_ctx* ctx = sv->ctx;
    pg_game* g = sv->B;
    cudaStream_t s = ctx->stream;
    int64_t Bb = 0;
    for (size_t i = 0; i < keep.size(); ++i) {
        pg_game* gi = sv->res[i].g;
        if (keep[i]) {
            ctx->launches += 1;
            k_unpack_profile<<<grid_of(gi->n), kBlock, 0, s>>>(gi->n - 1, (int32_t)Bb, g->strat, gi->strat);
            PG_CUDA_TRY(ctx, cudaGetLastError());
        }
        Bb += gi->n;
    }
    PG_CUDA_TRY(ctx, cudaStreamSynchronize(s));
    return PG_OK;
}

// Writes the results of game i of the packed batch into a Done record.
pg_status collect(pg_server* sv, size_t i, Done* d) {
    pg_ctx* ctx = sv->ctx;
    pg_game* g = sv->B;
    const int64_t o0 = g->h_base0[i], n0 = g->h_base0[i + 1] - o0;
    const int32_t d0 = g->h_dbase[i], k = g->h_dbase[i + 1] - d0;
    // a view of the packed batch restricted to game i's original vertices and dummies
    const size_t need = stage_bytes_for(n0, k);
    if (need > sv->stage_size) {
        if (sv->stage) cudaFree(sv->stage);
        sv->stage = nullptr;
        sv->stage_size = 0;
        PG_CUDA_TRY(ctx, cudaMalloc(&sv->stage, need + need / 2));
        sv->stage_size = need + need / 2;
    }
    pg_game view = *g;
    view.nid0 = g->nid0 + o0;
    view.dnid = g->dnid + d0;
    view.n0 = n0;
    view.k = k;
    view.stage = sv->stage;
    d->n = (int32_t)n0;
    d->k = k;
    d->win.resize(n0);
    d->sigma.resize(n0);
    d->tau.resize(n0);
    d->cls.resize(n0);
    d->depth.resize(n0);
    d->rank.resize(n0);
    d->dsig.resize(std::max(k, 1));
    pg_status st = write_outputs(&view, PG_MEM_HOST, d->win.data(), d->sigma.data(), d->tau.data(), d->cls.data(),
                                 d->depth.data(), d->rank.data(), nullptr, d->dsig.data(), true);
    return st;
}

// Loads queued games on the loader's stream while the worker solves, up to
// the capacity's worth of loaded games waiting for admission.
void loader_main(pg_server* sv) {
    pg_ctx* ctx = sv->lctx;
    if (cudaSetDevice(ctx->device) != cudaSuccess) {
        set_fatal(sv, PG_ECUDA, ctx);
        return;
    }
    for (;;) {
        Pending p;
        {
            std::unique_lock<std::mutex> lk(sv->mu);
            sv->cv_load.wait(lk, [&] {
                return sv->stop || sv->fatal ||
                       (!sv->queue.empty() && sv->ready_ids < sv->capN && (int64_t)sv->ready.size() < sv->capG);
            });
            if (sv->stop || sv->fatal) return;
            p = std::move(sv->queue.front());
            sv->queue.pop_front();
            sv->inflight[p.tag] = 1;
        }
        pg_game* gi = nullptr;
        pg_status st = load_game(ctx, p.n, p.m, p.off.data(), p.tgt.data(), p.own.data(), p.pri.data(), PG_MEM_HOST,
                                 &gi, false);
        if (st == PG_OK && gi->cv) {  // the packed batch ranks distinct priorities only
            free_game(gi);
            st = PG_EUNSUPPORTED;
        }
        if (st != PG_OK) {
            if (st == PG_ECUDA) {
                set_fatal(sv, st, ctx);
                return;
            }
            finish_pending_error(sv, p, st);
            continue;
        }
        ctx->launches += 1;
        k_init_profile<<<grid_of(gi->n), kBlock, 0, ctx->stream>>>(gi->n - 1, gi->off, gi->tgt, gi->flags, gi->strat);
        if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(ctx->stream) != cudaSuccess) {
            free_game(gi);
            set_fatal(sv, PG_ECUDA, ctx);
            return;
        }
        Resident r{};
        r.tag = p.tag;
        r.g = gi;
        r.t_submit = p.t_submit;
        r.slot = -1;
        {
            std::lock_guard<std::mutex> lk(sv->mu);
            sv->ready_ids += gi->n;
            sv->ready.push_back(r);
        }
        sv->cv_work.notify_all();
    }
}

void worker_main(pg_server* sv) {
    pg_ctx* ctx = sv->ctx;
    if (cudaSetDevice(ctx->device) != cudaSuccess) {
        set_fatal(sv, PG_ECUDA, ctx);
        return;
    }
    const int64_t round_iters = sv->opts.round_iters > 0 ? sv->opts.round_iters : 8;
    bool changed = false;
    for (;;) {
        // admission: loaded games in arrival order while they fit
        for (;;) {
            Resident r;
            {
                std::unique_lock<std::mutex> lk(sv->mu);
                if (sv->stop || sv->fatal) return;
                if (sv->ready.empty()) {
                    if (!sv->res.empty()) break;
                    sv->cv_work.wait(lk, [&] { return sv->stop || sv->fatal || !sv->ready.empty(); });
                    if (sv->stop || sv->fatal) return;
                }
                int64_t N = 0, M = 0;
                for (const Resident& x : sv->res) {
                    N += x.g->n;
                    M += x.g->m;
                }
                const Resident& q = sv->ready.front();
                const bool fits = N + q.g->n <= sv->capN && M + q.g->m <= sv->capM &&
                                  (int64_t)sv->res.size() < sv->capG;
                if (!fits && !sv->res.empty()) break;
                r = sv->ready.front();
                sv->ready.pop_front();
                sv->ready_ids -= r.g->n;
                if (fits) {
                    sv->stats.admitted += 1;
                    if (!sv->res.empty()) sv->stats.admitted_while_busy += 1;
                }
            }
            sv->cv_load.notify_all();
            if (!(r.g->n <= sv->capN && r.g->m <= sv->capM)) {  // larger than the whole capacity
                Pending p;
                p.tag = r.tag;
                p.n = (int32_t)r.g->n0;
                p.t_submit = r.t_submit;
                free_game(r.g);
                finish_pending_error(sv, p, PG_ENOMEM);
                continue;
            }
            r.t_admit = now_us();
            sv->res.push_back(r);
            changed = true;
        }
        if (sv->res.empty()) continue;
        pg_status st = PG_OK;
        double t_rep = now_us();
        if (changed) {
            // profiles of the games already in the batch come out first: the new layout starts from them
            if (sv->packed_count > 0) {
                std::vector<bool> all(sv->packed_count, true);
                st = unpack_profiles(sv, all);
                if (st) {
                    set_fatal(sv, st, ctx);
                    return;
                }
            }
            st = repack(sv);
            sv->packed_count = sv->res.size();
            changed = false;
            if (st) {
                set_fatal(sv, st, ctx);
                return;
            }
        }
        const double t_loop = now_us();
        {
            std::lock_guard<std::mutex> lk(sv->mu);
            sv->stats.max_resident = std::max<int64_t>(sv->stats.max_resident, (int64_t)sv->res.size());
            sv->stats.repack_ms += (t_loop - t_rep) / 1e3;
        }
        // one round over all resident games
        int64_t nmax = 0;
        for (const Resident& r : sv->res) nmax = std::max<int64_t>(nmax, r.g->n);
        const int64_t cap = sv->opts.max_inner > 0 ? sv->opts.max_inner : 64 * (nmax + 64);
        Timer tm(sv->B);
        st = run_loop(sv->B, cap, true, tm, round_iters);
        if (st) {
            set_fatal(sv, st, ctx);
            return;
        }
        std::vector<GameState> gs(sv->res.size());
        if (cudaMemcpyAsync(gs.data(), sv->B->gst, sizeof(GameState) * gs.size(), cudaMemcpyDeviceToHost,
                            ctx->stream) != cudaSuccess ||
            cudaStreamSynchronize(ctx->stream) != cudaSuccess) {
            set_fatal(sv, PG_ECUDA, ctx);
            return;
        }
        bool any_done = false, any_timeout = false;
        std::vector<bool> keep(sv->res.size(), true);
        for (size_t i = 0; i < gs.size(); ++i) {
            sv->res[i].st = gs[i];
            if (gs[i].phase != kPhaseActive) {
                keep[i] = false;
                any_done = true;
                any_timeout |= gs[i].phase == kPhaseTimeout;
            }
        }
        const double t_col = now_us();
        {
            std::lock_guard<std::mutex> lk(sv->mu);
            sv->stats.rounds += 1;
            sv->stats.iterations += sv->B->t_vals;
            sv->stats.loop_ms += (t_col - t_loop) / 1e3;
        }
        if (!any_done) continue;
        if (any_timeout || sv->B->last_cmp) {  // results describe the profile being returned (full valuation)
            st = full_valuation(sv->B, false);
            if (st) {
                set_fatal(sv, st, ctx);
                return;
            }
            sv->B->last_cmp = false;
        }
        st = enqueue_depth(sv->B);  // once for every finished game of this round
        if (st) {
            set_fatal(sv, st, ctx);
            return;
        }
        std::vector<std::pair<uint64_t, Done>> fin;
        for (size_t i = 0; i < gs.size(); ++i) {
            if (keep[i]) continue;
            Done d{};
            st = collect(sv, i, &d);
            if (st) {
                set_fatal(sv, st, ctx);
                return;
            }
            d.status = gs[i].phase == kPhaseDone ? PG_OK
                       : gs[i].phase == kPhaseTimeout ? PG_ETIMEOUT
                                                      : PG_ENOTADMISSIBLE;
            d.major = gs[i].major;
            d.inner = gs[i].inner;
            d.t_submit = sv->res[i].t_submit;
            d.t_admit = sv->res[i].t_admit;
            d.t_done = now_us();
            fin.emplace_back(sv->res[i].tag, std::move(d));
        }
        st = unpack_profiles(sv, keep);
        if (st) {
            set_fatal(sv, st, ctx);
            return;
        }
        std::vector<Resident> rest;
        for (size_t i = 0; i < sv->res.size(); ++i) {
            if (keep[i]) rest.push_back(sv->res[i]);
            else free_game(sv->res[i].g);
        }
        sv->res.swap(rest);
        sv->packed_count = 0;  // the kept profiles are out of the batch already
        changed = true;
        {
            std::lock_guard<std::mutex> lk(sv->mu);
            for (auto& f : fin) {
                sv->inflight.erase(f.first);
                sv->done[f.first] = std::move(f.second);
                sv->done_order.push_back(f.first);
                sv->stats.completed += 1;
            }
            sv->stats.collect_ms += (now_us() - t_col) / 1e3;
            sv->cv_done.notify_all();
        }
    }
}

}  // namespace

extern "C" {

pg_status pg_server_create(int device, const pg_server_opts* opts, pg_server** out) {
    if (!out) return PG_EINVAL;
    *out = nullptr;
    pg_ctx* ctx = nullptr;
    pg_status st = pg_ctx_create(&ctx, device);
    if (st) return st;
    pg_server* sv = new pg_server();
    sv->ctx = ctx;
    if (opts) sv->opts = *opts;
    if (cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking) != cudaSuccess) {
        pg_ctx_destroy(ctx);
        delete sv;
        return PG_ECUDA;
    }
    size_t freeb = 0, totalb = 0;
    if (cudaMemGetInfo(&freeb, &totalb) != cudaSuccess) freeb = 0;
    // Default capacity from free device memory: about 200 bytes per id of the
    // packed batch and its scratch, plus the resident games' own arrays, and
    // 24 bytes per edge; a quarter of the free memory in all.
    const int64_t budget = (int64_t)(freeb / 4);
    sv->capN = sv->opts.max_vertices > 0 ? sv->opts.max_vertices : std::max<int64_t>(1 << 20, budget / 2 / 200);
    sv->capM = sv->opts.max_edges > 0 ? sv->opts.max_edges : std::max<int64_t>(1 << 22, budget / 2 / 24);
    if (sv->capN >= (1ll << 30) - 1) sv->capN = (1ll << 30) - 2;
    sv->capG = sv->opts.max_games > 0 ? sv->opts.max_games : 4096;
    sv->stats.capacity_vertices = sv->capN;
    sv->stats.capacity_edges = sv->capM;
    st = alloc_batch(sv);
    if (st) {
        if (sv->B) free_game(sv->B);
        cudaStreamDestroy(ctx->stream);
        pg_ctx_destroy(ctx);
        delete sv;
        return st;
    }
    st = pg_ctx_create(&sv->lctx, device);
    if (st == PG_OK && cudaStreamCreateWithFlags(&sv->lctx->stream, cudaStreamNonBlocking) != cudaSuccess) st = PG_ECUDA;
    if (st) {
        if (sv->lctx) pg_ctx_destroy(sv->lctx);
        free_game(sv->B);
        cudaStreamDestroy(ctx->stream);
        pg_ctx_destroy(ctx);
        delete sv;
        return st;
    }
    sv->worker = std::thread(worker_main, sv);
    sv->loader = std::thread(loader_main, sv);
    *out = sv;
    return PG_OK;
}

void pg_server_destroy(pg_server* sv) {
    if (!sv) return;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->stop = true;
    }
    sv->cv_work.notify_all();
    sv->cv_load.notify_all();
    if (sv->worker.joinable()) sv->worker.join();
    if (sv->loader.joinable()) sv->loader.join();
    cudaSetDevice(sv->ctx->device);
    cudaStreamSynchronize(sv->ctx->stream);
    cudaStreamSynchronize(sv->lctx->stream);
    for (Resident& r : sv->res) free_game(r.g);
    for (Resident& r : sv->ready) free_game(r.g);
    if (sv->B) free_game(sv->B);
    if (sv->stage) cudaFree(sv->stage);
    cudaStreamDestroy(sv->ctx->stream);
    cudaStreamDestroy(sv->lctx->stream);
    pg_ctx_destroy(sv->ctx);
    pg_ctx_destroy(sv->lctx);
    delete sv;
}

pg_status pg_server_submit(pg_server* sv, int32_t n, int64_t m, const int32_t* offsets, const int32_t* targets,
                           const uint8_t* owner, const int32_t* pri, uint64_t tag) {
    if (!sv) return PG_EINVAL;
    if (n < 1 || m < n || !offsets || !targets || !owner || !pri) return PG_EINVAL;
    Pending p;
    p.tag = tag;
    p.n = n;
    p.m = m;
    p.off.assign(offsets, offsets + (size_t)n + 1);
    p.tgt.assign(targets, targets + (size_t)m);
    p.own.assign(owner, owner + (size_t)n);
    p.pri.assign(pri, pri + (size_t)n);
    p.t_submit = now_us();
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        if (sv->fatal) return sv->fatal;
        if (sv->done.count(tag)) return PG_EINVAL;
        for (const Pending& q : sv->queue)
            if (q.tag == tag) return PG_EINVAL;
        for (const Resident& q : sv->ready)
            if (q.tag == tag) return PG_EINVAL;
        if (sv->inflight.count(tag)) return PG_EINVAL;
        sv->queue.push_back(std::move(p));
        sv->stats.submitted += 1;
    }
    sv->cv_load.notify_all();
    return PG_OK;
}

pg_status pg_server_poll(pg_server* sv, pg_served* out, int32_t max, int32_t timeout_ms, int32_t* count) {
    if (!sv || !count || max < 0 || (max > 0 && !out)) return PG_EINVAL;
    *count = 0;
    std::unique_lock<std::mutex> lk(sv->mu);
    if (sv->done_order.empty() && timeout_ms > 0 && !sv->fatal)
        sv->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms),
                             [&] { return !sv->done_order.empty() || sv->fatal; });
    int32_t c = 0;
    while (c < max && !sv->done_order.empty()) {
        const uint64_t tag = sv->done_order.front();
        sv->done_order.pop_front();
        const Done& d = sv->done[tag];
        pg_served& o = out[c++];
        o.tag = tag;
        o.status = d.status;
        o.n = d.n;
        o.k = d.k;
        o.major = d.major;
        o.inner = d.inner;
        o.queue_us = d.t_admit - d.t_submit;
        o.latency_us = d.t_done - d.t_submit;
    }
    *count = c;
    return c == 0 && sv->fatal ? sv->fatal : PG_OK;
}

pg_status pg_server_fetch(pg_server* sv, uint64_t tag, uint8_t* win, int32_t* sigma, int32_t* tau, int8_t* val_class,
                          int32_t* val_depth, int32_t* val_rank, int8_t* dummy_sigma) {
    if (!sv) return PG_EINVAL;
    Done d;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        auto it = sv->done.find(tag);
        if (it == sv->done.end()) return PG_EINVAL;
        for (uint64_t t : sv->done_order)
            if (t == tag) return PG_EINVAL;  // not reported by pg_server_poll yet
        d = std::move(it->second);
        sv->done.erase(it);
    }
    const size_t n = d.win.size();
    if (win) memcpy(win, d.win.data(), n);
    if (sigma) memcpy(sigma, d.sigma.data(), 4 * n);
    if (tau) memcpy(tau, d.tau.data(), 4 * n);
    if (val_class) memcpy(val_class, d.cls.data(), n);
    if (val_depth) memcpy(val_depth, d.depth.data(), 4 * n);
    if (val_rank) memcpy(val_rank, d.rank.data(), 4 * n);
    if (dummy_sigma && d.k > 0) memcpy(dummy_sigma, d.dsig.data(), (size_t)d.k);
    return PG_OK;
}

pg_status pg_server_get_stats(pg_server* sv, pg_server_stats* out) {
    if (!sv || !out) return PG_EINVAL;
    std::lock_guard<std::mutex> lk(sv->mu);
    *out = sv->stats;
    out->queued = (int64_t)(sv->queue.size() + sv->ready.size());
    return PG_OK;
}

const char* pg_server_error(pg_server* sv) {
    if (!sv) return "NULL server";
    std::lock_guard<std::mutex> lk(sv->mu);
    return sv->fatal ? sv->fatal_msg.c_str() : "no error";
}

}  // extern "C"
