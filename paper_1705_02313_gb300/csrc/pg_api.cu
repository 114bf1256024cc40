// C ABI of libpg: contexts, games, and the loops of Algorithm 1 (Section 4).
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include <mutex>

#include "pg_internal.cuh"

namespace pg {

pg_status fail(pg_ctx* ctx, pg_status code, const char* msg) {
    if (ctx && !ctx->quiet) ctx->err = msg;
    return code;
}

pg_status cuda_fail(pg_ctx* ctx, cudaError_t e, const char* where) {
    pg_status code = e == cudaErrorMemoryAllocation ? PG_ENOMEM : PG_ECUDA;
    if (!ctx || ctx->quiet) return code;
    ctx->err = std::string("CUDA error ") + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ") at " + where;
    return code;
}

void drop_loop_graphs(pg_game* g) {
    for (int i = 0; i < 2; ++i) {
        if (g->loop_exec[i]) cudaGraphExecDestroy(g->loop_exec[i]);
        g->loop_exec[i] = nullptr;
        g->loop_cap[i] = g->loop_limit[i] = 0;
    }
}

namespace {
constexpr int kPoolDevices = 64;
std::mutex g_pool_mu;
cudaMemPool_t g_pool[kPoolDevices] = {};

cudaError_t game_pool(int device, cudaMemPool_t* out) {
    if (device < 0 || device >= kPoolDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_pool_mu);
    if (!g_pool[device]) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = device;
        cudaMemPool_t p = nullptr;
        cudaError_t e = cudaMemPoolCreate(&p, &props);
        if (e != cudaSuccess) return e;
        cudaDeviceProp prop;
        e = cudaGetDeviceProperties(&prop, device);
        uint64_t keep = e == cudaSuccess ? (uint64_t)prop.totalGlobalMem / 4 : 0;
        e = cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &keep);
        if (e != cudaSuccess) {
            cudaMemPoolDestroy(p);
            return e;
        }
        g_pool[device] = p;
    }
    *out = g_pool[device];
    return cudaSuccess;
}
}  // namespace

cudaError_t dev_alloc(pg_ctx* ctx, void** p, size_t bytes, cudaStream_t s) {
    cudaMemPool_t pool = nullptr;
    cudaError_t e = game_pool(ctx->device, &pool);
    if (e != cudaSuccess) return e;
    return cudaMallocFromPoolAsync(p, bytes ? bytes : 1, pool, s);
}

cudaError_t dev_trim(int device) {
    cudaMemPool_t pool = nullptr;
    cudaError_t e = game_pool(device, &pool);
    if (e != cudaSuccess) return e;
    e = cudaDeviceSynchronize();
    return e == cudaSuccess ? cudaMemPoolTrimTo(pool, 0) : e;
}

// Work of any stream may still read the game (batch loaders, the server's
// worker): the device is synchronised once, as cudaFree would, and then every
// buffer goes back to the pool.
void free_game(pg_game* g) {
    if (!g) return;
    void* ptrs[] = {g->off,  g->off64,   g->vgame, g->gsink, g->gst,   g->gactive, g->gscan,
                    g->tgt,     g->flags, g->pri,   g->nid0,  g->orig_of, g->dnid,    g->dummy_of,
                    g->strat, g->gd,     g->gd32,  g->kind,  g->plist, g->slot,  g->ccnt,  g->coff,    g->cl_ks,   g->sz,
                    g->sinkval, g->wgt,  g->oddsz, g->key,   g->cls,   g->depth,   g->dom,     g->hugelist,
                    g->tiles, g->tsum,   g->cnt,    g->scan_tmp, g->stage, g->loop_iters, g->ws, g->wsB, g->gdB, g->key128,
                    g->d_anc, g->d_sc, g->d_podd, g->d_peven, g->d_oddL, g->d_evenL, g->d_nxt, g->d_wt, g->d_loc,
                    g->d_own, g->d_rid, g->d_rl, g->d_val, g->d_rnx, g->pl_vid[0], g->pl_vid[1], g->pl_off[0],
                    g->pl_off[1], g->pl_tgt[0], g->pl_tgt[1], g->rv_off, g->rv_src, g->omark};
    int prev = -1;
    const bool switched =
        cudaGetDevice(&prev) == cudaSuccess && prev != g->device && cudaSetDevice(g->device) == cudaSuccess;
    cudaDeviceSynchronize();
    for (void* p : ptrs)
        if (p) cudaFreeAsync(p, 0);
    if (g->hcnt) cudaFreeHost(g->hcnt);
    for (auto& x : g->loop_exec)
        if (x) cudaGraphExecDestroy(x);
    for (auto& e : g->ev)
        if (e) cudaEventDestroy(e);
    for (auto& e : g->kev)
        if (e) cudaEventDestroy(e);
    if (switched) cudaSetDevice(prev);
    delete g;
}

namespace {

inline unsigned grid_of(int64_t n) {
    int64_t b = (n + kBlock - 1) / kBlock;
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(b, 152 * 64));
}

// Sets g->strat from a profile given in original ids (NULL arrays take the
// defaults: Even and dummies to the sink, Odd to its first edge).
__device__ inline int32_t sink_id(int32_t i, const int32_t* vgame, const int32_t* gsink, int32_t sink0) {
    return vgame ? gsink[vgame[i]] : sink0;
}

// The initial profile of Algorithm 1 (no profile given): every Odd vertex to
// the first edge of its list, every Even vertex and dummy to its game's sink;
// sink slots keep their own id. In relabelled id order, coalesced.
template <typename OffT>
__global__ void k_default_profile(int32_t n, const OffT* __restrict__ off, const int32_t* __restrict__ tgt,
                                  const uint8_t* __restrict__ flags, const int32_t* __restrict__ vgame,
                                  const int32_t* __restrict__ gsink, int32_t sink0, int32_t* strat) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint8_t f = flags[i];
        if (f & kSinkSlot) continue;
        strat[i] = (f & kOwnerOdd) ? tgt[off[i]] : sink_id((int32_t)i, vgame, gsink, sink0);
    }
}

template <typename OffT>
__global__ void k_apply_profile(int64_t n0, int32_t k, const int32_t* __restrict__ nid0,
                                const OffT* __restrict__ off, const int32_t* __restrict__ tgt,
                                const uint8_t* __restrict__ flags, const int32_t* __restrict__ orig_of,
                                const int32_t* __restrict__ dnid, const int32_t* __restrict__ vgame,
                                const int32_t* __restrict__ gsink, int32_t sink0, const int32_t* sigma,
                                const int32_t* tau, const int8_t* dsig, int32_t* strat, int32_t* err) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n0 + (int64_t)k;
         v += (int64_t)gridDim.x * blockDim.x) {
        if (v >= n0) {
            int32_t d = dnid[v - n0];
            strat[d] = (dsig && dsig[v - n0]) ? tgt[off[d]] : sink_id(d, vgame, gsink, sink0);
            continue;
        }
        int32_t i = nid0[v];
        const int32_t n = sink_id(i, vgame, gsink, sink0);
        bool odd = (flags[i] & kOwnerOdd) != 0;
        const int32_t* src = odd ? tau : sigma;
        if (!src) {
            strat[i] = odd ? tgt[off[i]] : n;
            continue;
        }
        int32_t t = src[v];
        if (!odd && t == -1) {
            strat[i] = n;
            continue;
        }
        int32_t pick = -1;
        for (OffT e = off[i]; e < off[i + 1]; ++e)
            if (orig_of[tgt[e]] == t) {
                pick = tgt[e];
                break;
            }
        if (pick < 0) {
            atomicOr(err, 1);
            strat[i] = odd ? tgt[off[i]] : n;
        } else {
            strat[i] = pick;
        }
    }
}

struct OutPtrs {
    int32_t cv;  // count-vector mode: valuations are count vectors, there is no rank (written as -1)
    uint8_t* win;
    int32_t* sigma;
    int32_t* tau;
    int8_t* vclass;
    int32_t* vdepth;
    int32_t* vrank;
    int32_t* vdom;
    int8_t* dsig;
};

__global__ void k_results(int64_t n0, int32_t k, const int32_t* __restrict__ nid0,
                          const int32_t* __restrict__ dnid, const uint8_t* __restrict__ flags,
                          const int32_t* __restrict__ strat, const uint8_t* __restrict__ cls,
                          const int32_t* __restrict__ depth, const int32_t* __restrict__ key,
                          const int32_t* __restrict__ orig_of, const int32_t* __restrict__ dom,
                          const int32_t* __restrict__ vgame, const int32_t* __restrict__ gsink, int32_t sink0,
                          OutPtrs o) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n0 + (int64_t)k;
         v += (int64_t)gridDim.x * blockDim.x) {
        if (v >= n0) {
            const int32_t d = dnid[v - n0];
            if (o.dsig) o.dsig[v - n0] = strat[d] != sink_id(d, vgame, gsink, sink0);
            continue;
        }
        int32_t i = nid0[v];
        const int32_t n = sink_id(i, vgame, gsink, sink0);
        bool fin = cls[i] == kFin;
        bool odd = (flags[i] & kOwnerOdd) != 0;
        int32_t s = strat[i];
        if (o.win) o.win[v] = fin ? 1 : 0;
        if (o.sigma) o.sigma[v] = odd ? -1 : (s == n ? -1 : orig_of[s]);
        if (o.tau) o.tau[v] = odd ? orig_of[s] : -1;
        if (o.vclass) o.vclass[v] = fin ? 0 : 1;
        if (o.vdepth) o.vdepth[v] = fin ? depth[i] : -1;
        if (o.vrank) o.vrank[v] = o.cv ? -1 : (fin ? key[i] : INT32_MAX);
        if (o.vdom) o.vdom[v] = dom[i];
    }
}

// staging layout for host outputs
struct Stage {
    size_t off_win, off_sigma, off_tau, off_class, off_depth, off_rank, off_dom, off_dsig, bytes;
};
inline size_t al(size_t x) { return (x + 255) & ~(size_t)255; }
Stage stage_layout(int64_t n0, int64_t k) {
    Stage s;
    size_t p = 0;
    s.off_win = p; p = al(p + n0);
    s.off_sigma = p; p = al(p + 4 * n0);
    s.off_tau = p; p = al(p + 4 * n0);
    s.off_class = p; p = al(p + n0);
    s.off_depth = p; p = al(p + 4 * n0);
    s.off_rank = p; p = al(p + 4 * n0);
    s.off_dom = p; p = al(p + 4 * n0);
    s.off_dsig = p; p = al(p + k);
    s.bytes = p;
    return s;
}

}  // namespace

size_t stage_bytes_for(int64_t n0, int64_t k) { return stage_layout(n0, k).bytes; }

pg_status write_outputs(pg_game* g, int32_t mem_kind, uint8_t* win, int32_t* sigma, int32_t* tau, int8_t* vclass,
                        int32_t* vdepth, int32_t* vrank, int32_t* vdom, int8_t* dsig, bool depth_ready) {
    pg_ctx* ctx = g->ctx;
    cudaStream_t s = ctx->stream;
    OutPtrs o = {g->cv ? 1 : 0, win, sigma, tau, vclass, vdepth, vrank, vdom, dsig};
    Stage L = stage_layout(g->n0, g->k);
    if (mem_kind == PG_MEM_HOST) {
        if (!g->stage) PG_CUDA_TRY(ctx, dev_alloc(ctx, &g->stage, L.bytes, s));
        char* b = (char*)g->stage;
        o = {g->cv ? 1 : 0,
             win ? (uint8_t*)(b + L.off_win) : nullptr,     sigma ? (int32_t*)(b + L.off_sigma) : nullptr,
             tau ? (int32_t*)(b + L.off_tau) : nullptr,     vclass ? (int8_t*)(b + L.off_class) : nullptr,
             vdepth ? (int32_t*)(b + L.off_depth) : nullptr, vrank ? (int32_t*)(b + L.off_rank) : nullptr,
             vdom ? (int32_t*)(b + L.off_dom) : nullptr,     dsig ? (int8_t*)(b + L.off_dsig) : nullptr};
    }
    if (vdepth && !depth_ready) {
        pg_status st = enqueue_depth(g);
        if (st) return st;
    }
    ctx->launches += 1;
    k_results<<<grid_of((int64_t)g->n0 + g->k), kBlock, 0, s>>>(g->n0, g->k, g->nid0, g->dnid, g->flags, g->strat,
                                                                g->cls, g->depth, g->key, g->orig_of, g->dom,
                                                                g->vgame, g->gsink, g->sink0, o);
    PG_CUDA_TRY(ctx, cudaGetLastError());
    if (mem_kind == PG_MEM_HOST) {
        size_t n0 = (size_t)g->n0;
        auto cp = [&](void* dst, const void* src, size_t bytes) {
            return dst ? cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, s) : cudaSuccess;
        };
        PG_CUDA_TRY(ctx, cp(win, o.win, n0));
        PG_CUDA_TRY(ctx, cp(sigma, o.sigma, 4 * n0));
        PG_CUDA_TRY(ctx, cp(tau, o.tau, 4 * n0));
        PG_CUDA_TRY(ctx, cp(vclass, o.vclass, n0));
        PG_CUDA_TRY(ctx, cp(vdepth, o.vdepth, 4 * n0));
        PG_CUDA_TRY(ctx, cp(vrank, o.vrank, 4 * n0));
        PG_CUDA_TRY(ctx, cp(vdom, o.vdom, 4 * n0));
        PG_CUDA_TRY(ctx, cp(dsig, o.dsig, (size_t)g->k));
    }
    PG_CUDA_TRY(ctx, cudaStreamSynchronize(s));
    return PG_OK;
}

// Copies caller profile arrays to the device when needed and applies them.
pg_status apply_profile(pg_game* g, const int32_t* sigma, const int32_t* tau, const int8_t* dsig, int32_t mem_kind) {
    pg_ctx* ctx = g->ctx;
    cudaStream_t s = ctx->stream;
    if (mem_kind != PG_MEM_HOST && mem_kind != PG_MEM_DEVICE) return fail(ctx, PG_EINVAL, "bad mem_kind");
    const int32_t *ds = sigma, *dt = tau;
    const int8_t* dd = dsig;
    int32_t* buf = nullptr;
    cudaError_t e = cudaSuccess;
    if (mem_kind == PG_MEM_HOST && (sigma || tau || dsig)) {
        size_t bytes = 8 * (size_t)g->n0 + (size_t)g->k + 16;
        PG_CUDA_TRY(ctx, dev_alloc(ctx, (void**)&buf, bytes, s));
        char* b = (char*)buf;
        if (sigma) {
            e = cudaMemcpyAsync(b, sigma, 4 * (size_t)g->n0, cudaMemcpyHostToDevice, s);
            ds = (const int32_t*)b;
        }
        if (tau && e == cudaSuccess) {
            e = cudaMemcpyAsync(b + 4 * (size_t)g->n0, tau, 4 * (size_t)g->n0, cudaMemcpyHostToDevice, s);
            dt = (const int32_t*)(b + 4 * (size_t)g->n0);
        }
        if (dsig && g->k && e == cudaSuccess) {
            e = cudaMemcpyAsync(b + 8 * (size_t)g->n0, dsig, (size_t)g->k, cudaMemcpyHostToDevice, s);
            dd = (const int8_t*)(b + 8 * (size_t)g->n0);
        }
    }
    if (!sigma && !tau && !dsig) {  // the initial profile: nothing to check, no wait
        ctx->launches += 1;
        if (g->off64)
            k_default_profile<int64_t><<<grid_of(g->n), kBlock, 0, s>>>(g->n, g->off64, g->tgt, g->flags, g->vgame,
                                                                          g->gsink, g->sink0, g->strat);
        else
            k_default_profile<int32_t><<<grid_of(g->n), kBlock, 0, s>>>(g->n, g->off, g->tgt, g->flags, g->vgame,
                                                                          g->gsink, g->sink0, g->strat);
        PG_CUDA_TRY(ctx, cudaGetLastError());
        return PG_OK;
    }
    int32_t* err = &g->cnt->err;
    if (e == cudaSuccess) e = cudaMemsetAsync(err, 0, sizeof(int32_t), s);
    if (e == cudaSuccess) {
        ctx->launches += 1;
        if (g->off64)
            k_apply_profile<int64_t><<<grid_of((int64_t)g->n0 + g->k), kBlock, 0, s>>>(
                g->n0, g->k, g->nid0, g->off64, g->tgt, g->flags, g->orig_of, g->dnid, g->vgame, g->gsink, g->sink0, ds,
                dt, dd, g->strat, err);
        else
            k_apply_profile<int32_t><<<grid_of((int64_t)g->n0 + g->k), kBlock, 0, s>>>(
                g->n0, g->k, g->nid0, g->off, g->tgt, g->flags, g->orig_of, g->dnid, g->vgame, g->gsink, g->sink0, ds,
                dt, dd, g->strat, err);
        e = cudaMemcpyAsync(ctx->pinned, err, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (buf) cudaFreeAsync(buf, s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "apply_profile");
    if (ctx->pinned[0]) return fail(ctx, PG_EINVAL, "profile names a successor that is not an edge of its vertex");
    return PG_OK;
}



// Loop condition of the device-side loop: continue while a game is active,
// no device error was recorded and the hard cap is not reached.
__global__ void k_loop_cond(cudaGraphConditionalHandle h, const int32_t* gactive, const Counters* c, int64_t* iters,
                            int64_t hard_cap) {
    const int64_t it = *iters + 1;
    *iters = it;
    cudaGraphSetConditional(h, (gactive[0] > 0 && c->err == 0 && c->deep == 0 && it < hard_cap) ? 1u : 0u);
}

// One iteration of Algorithm 1 for every game of g (enqueued on ctx->stream).
pg_status enqueue_iteration(pg_game* g, int64_t cap, bool even) {
    const bool cmp = loop_compares(g);
    pg_status st = cmp ? enqueue_valuation_cmp(g) : enqueue_valuation(g, false);
    if (!st) st = cmp ? enqueue_switch_cmp(g, 1) : enqueue_switch(g, 1);
    if (!st && even) st = cmp ? enqueue_switch_cmp(g, 0) : enqueue_switch(g, 0);
    if (!st) st = enqueue_bookkeeping(g, cap, even);
    if (!st && even && g->reset_tau) st = enqueue_reset(g);
    return st;
}

// Builds the loop graph: a WHILE node whose body is one iteration followed
// by k_loop_cond. Returns false (nothing recorded) when the runtime refuses
// any step; the caller then runs the loop from the host.
bool build_loop_graph(pg_game* g, int64_t cap, bool even, int64_t limit) {
    pg_ctx* ctx = g->ctx;
    const int w = even ? 1 : 0;
    if (g->loop_exec[w] && g->loop_cap[w] == cap && g->loop_limit[w] == limit && g->loop_reset[w] == g->reset_tau &&
        g->loop_cmp[w] == loop_compares(g) && g->loop_deep[w] == g->deep_mode && g->loop_tune[w] == g->tune)
        return true;
    if (g->loop_exec[w]) {
        cudaGraphExecDestroy(g->loop_exec[w]);
        g->loop_exec[w] = nullptr;
    }
    if (!ctx->cap_stream && cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    cudaGraph_t graph = nullptr;
    if (cudaGraphCreate(&graph, 0) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    bool ok = false;
    cudaGraphConditionalHandle h;
    cudaGraphNodeParams cp = {};
    cudaGraphNode_t node;
    if (cudaGraphConditionalHandleCreate(&h, graph, 1, cudaGraphCondAssignDefault) == cudaSuccess) {
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = h;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        ok = cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &cp) == cudaSuccess;
    }
    const int64_t l0 = ctx->launches;
    int64_t k0[KID_COUNT];
    for (int i = 0; i < KID_COUNT; ++i) k0[i] = g->klaunch[i];
    if (ok) {
        cudaGraph_t body = cp.conditional.phGraph_out[0];
        cudaStream_t user = ctx->stream;
        ctx->stream = ctx->cap_stream;
        const bool quiet = ctx->quiet;
        ctx->quiet = true;
        ok = cudaStreamBeginCaptureToGraph(ctx->cap_stream, body, nullptr, nullptr, 0,
                                           cudaStreamCaptureModeThreadLocal) == cudaSuccess;
        if (ok) {
            bool enq = enqueue_iteration(g, cap, even) == PG_OK;
            if (enq) {
                k_loop_cond<<<1, 1, 0, ctx->cap_stream>>>(h, g->gactive, g->cnt, g->loop_iters, limit);
                enq = cudaGetLastError() == cudaSuccess;
            }
            cudaGraph_t out = nullptr;
            ok = cudaStreamEndCapture(ctx->cap_stream, &out) == cudaSuccess && enq;
        }
        ctx->stream = user;
        ctx->quiet = quiet;
    }
    // launches counted while capturing belong to the iterations the graph will run
    g->loop_launch[w] = ctx->launches - l0 + 1;
    ctx->launches = l0;
    for (int i = 0; i < KID_COUNT; ++i) {
        g->loop_klaunch[w][i] = g->klaunch[i] - k0[i];
        g->klaunch[i] = k0[i];
    }
    if (ok) ok = cudaGraphInstantiate(&g->loop_exec[w], graph, 0) == cudaSuccess;
    cudaGraphDestroy(graph);
    if (!ok) {
        g->loop_exec[w] = nullptr;
        cudaGetLastError();
        return false;
    }
    g->loop_cap[w] = cap;
    g->loop_limit[w] = limit;
    g->loop_reset[w] = g->reset_tau;
    g->loop_cmp[w] = loop_compares(g);
    g->loop_deep[w] = g->deep_mode;
    g->loop_tune[w] = g->tune;
    return true;
}

// Algorithm 1 for every game of g at once: each iteration computes the
// valuation of every game, switches Odd in active games, switches Even in
// games whose inner loop has converged (no Odd switch this iteration), and
// updates each game's state on the device (see k_bookkeep). With even = false
// only the inner loop runs (best responses). Normally the whole loop is one
// CUDA graph launch whose WHILE node repeats the iteration until no game is
// active (no host synchronisation between iterations); with timing enabled,
// or where the runtime refuses the graph, the host runs the loop and
// synchronises once per iteration. A positive limit ends the call after that
// many iterations even if games are still active (their state stays on the
// device and a later call continues them).
pg_status run_loop_once(pg_game* g, int64_t cap, bool even, Timer& tm, int64_t limit, int64_t* ran) {
    pg_ctx* ctx = g->ctx;
    g->last_graph = false;
    *ran = 0;
    const bool cmp = loop_compares(g);
    const int64_t hard = limit > 0 ? std::min<int64_t>(limit, cap + 2) : cap + 2;
    if (!tm.on && ctx->graphs && build_loop_graph(g, cap, even, hard)) {
        const int w = even ? 1 : 0;
        cudaStream_t s = ctx->stream;
        PG_CUDA_TRY(ctx, cudaMemsetAsync(g->loop_iters, 0, sizeof(int64_t), s));
        PG_CUDA_TRY(ctx, cudaGraphLaunch(g->loop_exec[w], s));
        int64_t* it = (int64_t*)ctx->pinned;
        PG_CUDA_TRY(ctx, cudaMemcpyAsync(it, g->loop_iters, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        pg_status st = sync_counters(g);
        const int64_t iters = *it;
        *ran = iters;
        g->t_vals += iters;
        ctx->launches += g->loop_launch[w] * iters;
        for (int i = 0; i < KID_COUNT; ++i) g->klaunch[i] += g->loop_klaunch[w][i] * iters;
        g->last_graph = true;
        if (st) return st;
        if (iters > hard) return fail(ctx, PG_ECUDA, "device-side loop exceeded its iteration cap");
        return PG_OK;
    }
    for (int64_t it = 1;; ++it) {
        tm.mark(0);
        pg_status st = cmp ? enqueue_valuation_cmp(g) : enqueue_valuation(g, false);
        if (st) return st;
        tm.mark(1);
        st = cmp ? enqueue_switch_cmp(g, 1) : enqueue_switch(g, 1);
        if (!st && even) st = cmp ? enqueue_switch_cmp(g, 0) : enqueue_switch(g, 0);
        if (!st) st = enqueue_bookkeeping(g, cap, even);
        if (!st && even && g->reset_tau) st = enqueue_reset(g);
        if (st) return st;
        tm.mark(2);
        PG_CUDA_TRY(ctx, cudaMemcpyAsync(ctx->pinned, g->gactive, sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->stream));
        st = sync_counters(g);
        if (st) return st;
        ++g->t_vals;
        *ran = it;
        g->t_val += tm.since(0, 1);
        g->t_switch += tm.since(1, 2);
        if (ctx->pinned[0] == 0 || it >= hard || g->hcnt->deep) return PG_OK;
    }
}

// The loop of Algorithm 1 (run_loop_once) until its end, a cap or the limit.
// When an iteration finds a g-chain longer than the cutover depth, it is
// abandoned before anything is switched or counted, the loop stops, and the
// game continues from the same profile with the ruling-set ranks (for the
// rest of this call), so the trajectory is unchanged.
pg_status run_loop(pg_game* g, int64_t cap, bool even, Timer& tm, int64_t limit) {
    if (loop_compares(g) && !g->pl_ok) {
        pg_status st = build_player_split(g);
        if (st) return st;
    }
    if (omark_of(g))  // the first Odd pass of the call evaluates every Odd vertex (a nonzero flag)
        PG_CUDA_TRY(g->ctx, cudaMemsetAsync(g->gactive + 1, 0xff, sizeof(int32_t), g->ctx->stream));
    int64_t done = 0;
    for (;;) {
        int64_t ran = 0;
        pg_status st = run_loop_once(g, cap, even, tm, limit > 0 ? limit - done : 0, &ran);
        if (st) return st;
        g->last_cmp = loop_compares(g);
        if (g->cv || g->deep_mode || !g->hcnt->deep) return PG_OK;
        g->deep_mode = true;
        st = prepare_deep(g);
        if (st) return st;
        g->t_vals -= 1;  // the abandoned iteration
        done += ran - 1;
        if (limit > 0 && done >= limit) return PG_OK;
    }
}

}  // namespace pg

namespace pg {
namespace {
// Checks t and merges its nonzero fields into out.
bool merge_tuning(const pg_tuning& t, Tune* out) {
    if (t.deep_cut < 0 || t.ruler_bits < 0 || t.ruler_bits > 16 || t.loop_ranks < 0 || t.loop_ranks > 1)
        return false;
    if (t.walk_cap && t.walk_cap != 16 && t.walk_cap != 32 && t.walk_cap != 64 && t.walk_cap != 128) return false;
    if (t.switch_block && t.switch_block != 128 && t.switch_block != 256 && t.switch_block != 512) return false;
    if (t.deep_cut) out->deep_cut = t.deep_cut;
    if (t.ruler_bits) out->ruler_bits = t.ruler_bits;
    if (t.walk_cap) out->walk_cap = t.walk_cap;
    if (t.switch_block) out->switch_block = t.switch_block;
    out->loop_ranks = t.loop_ranks;
    return true;
}
}  // namespace

Tune tune_for(const pg_ctx* ctx, int64_t n) {
    for (const Tune& t : ctx->tune_table)
        if (n <= t.max_ids) return t;
    return ctx->tune;
}

}  // namespace pg

using namespace pg;

extern "C" {

pg_status pg_ctx_create(pg_ctx** out, int device) {
    if (!out) return PG_EINVAL;
    *out = nullptr;
    int count = 0;
    if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count) return PG_ECUDA;
    if (cudaSetDevice(device) != cudaSuccess) return PG_ECUDA;
    pg_ctx* c = new pg_ctx();
    c->device = device;
    if (cudaMallocHost((void**)&c->pinned, 64) != cudaSuccess) {
        delete c;
        return PG_ENOMEM;
    }
    const char* tf = getenv("PG_TUNING_FILE");  // the autotuner's table, when the caller names one
    if (tf && *tf && pg_load_tuning(c, tf) != PG_OK) c->tune_table.clear();
    *out = c;
    return PG_OK;
}

pg_status pg_device_name(int device, char* buf, int32_t cap) {
    if (!buf || cap < 1) return PG_EINVAL;
    cudaDeviceProp p;
    if (cudaGetDeviceProperties(&p, device) != cudaSuccess) return PG_ECUDA;
    snprintf(buf, (size_t)cap, "%s", p.name);
    return PG_OK;
}

void pg_ctx_destroy(pg_ctx* ctx) {
    if (!ctx) return;
    if (ctx->pinned) cudaFreeHost(ctx->pinned);
    if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
    delete ctx;
}

pg_status pg_set_stream(pg_ctx* ctx, void* stream) {
    if (!ctx) return PG_EINVAL;
    ctx->stream = (cudaStream_t)stream;
    return PG_OK;
}

const char* pg_last_error(const pg_ctx* ctx) { return ctx ? ctx->err.c_str() : "NULL context"; }

pg_status pg_release_cached_memory(int device) {
    int count = 0;
    if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count) return PG_ECUDA;
    int prev = 0;
    if (cudaGetDevice(&prev) != cudaSuccess || cudaSetDevice(device) != cudaSuccess) return PG_ECUDA;
    cudaError_t e = dev_trim(device);
    cudaSetDevice(prev);
    return e == cudaSuccess ? PG_OK : PG_ECUDA;
}

pg_status pg_set_graphs(pg_ctx* ctx, int32_t enable) {
    if (!ctx) return PG_EINVAL;
    ctx->graphs = enable != 0;
    return PG_OK;
}

pg_status pg_set_tuning(pg_ctx* ctx, const pg_tuning* t) {
    if (!ctx || !t) return PG_EINVAL;
    Tune x = ctx->tune;
    pg_tuning u = *t;
    if (!u.loop_ranks) u.loop_ranks = ctx->tune.loop_ranks;  // zero keeps it, like the other fields
    if (!merge_tuning(u, &x)) return fail(ctx, PG_EINVAL, "pg_set_tuning: bad value");
    ctx->tune = x;
    return PG_OK;
}

pg_status pg_get_tuning(const pg_ctx* ctx, pg_tuning* t) {
    if (!ctx || !t) return PG_EINVAL;
    *t = pg_tuning{ctx->tune.deep_cut, ctx->tune.ruler_bits, ctx->tune.walk_cap, ctx->tune.switch_block,
                   ctx->tune.loop_ranks};
    return PG_OK;
}

pg_status pg_set_tuning_table(pg_ctx* ctx, const pg_tuning_entry* e, int32_t count) {
    if (!ctx || count < 0 || (count && !e)) return PG_EINVAL;
    std::vector<Tune> table;
    for (int32_t i = 0; i < count; ++i) {
        Tune x;  // the defaults, then the entry's nonzero fields
        if (e[i].max_ids < 1 || (i && e[i].max_ids <= e[i - 1].max_ids) || !merge_tuning(e[i].t, &x))
            return fail(ctx, PG_EINVAL, "pg_set_tuning_table: bad entry (max_ids must increase)");
        x.max_ids = e[i].max_ids;
        table.push_back(x);
    }
    ctx->tune_table = table;
    return PG_OK;
}

pg_status pg_load_tuning(pg_ctx* ctx, const char* path) {
    if (!ctx || !path) return PG_EINVAL;
    FILE* f = fopen(path, "r");
    if (!f) return fail(ctx, PG_EINVAL, "pg_load_tuning: cannot open the file");
    std::vector<pg_tuning_entry> es;
    char line[512];
    bool bad = false;
    while (fgets(line, sizeof line, f)) {
        const char* p = line;
        while (*p == ' ' || *p == '\t') ++p;
        if (*p == '#' || *p == '\n' || *p == '\0') continue;
        long long m = 0;
        int a = 0, b = 0, c = 0, d = 0, r = 0;
        if (sscanf(p, "%lld %d %d %d %d %d", &m, &a, &b, &c, &d, &r) != 6) {
            bad = true;
            break;
        }
        es.push_back(pg_tuning_entry{(int64_t)m, pg_tuning{a, b, c, d, r}});
    }
    fclose(f);
    if (bad) return fail(ctx, PG_EINVAL, "pg_load_tuning: a line is not 'max_ids deep_cut ruler_bits walk_cap "
                                         "switch_block loop_ranks'");
    return pg_set_tuning_table(ctx, es.data(), (int32_t)es.size());
}

pg_status pg_set_wide_offsets(pg_ctx* ctx, int32_t enable) {
    if (!ctx) return PG_EINVAL;
    ctx->wide_offsets = enable != 0;
    return PG_OK;
}

pg_status pg_set_loop_ranks(pg_ctx* ctx, int32_t enable) {
    if (!ctx) return PG_EINVAL;
    ctx->tune.loop_ranks = enable != 0;
    return PG_OK;
}

pg_status pg_last_loop(const pg_game* g, int32_t* graph, int64_t* iterations) {
    if (!g) return PG_EINVAL;
    if (graph) *graph = g->last_graph ? 1 : 0;
    if (iterations) *iterations = g->t_vals;
    return PG_OK;
}

pg_status pg_set_timing(pg_ctx* ctx, int32_t enable) {
    if (!ctx) return PG_EINVAL;
    ctx->timing = enable != 0;
    return PG_OK;
}

pg_status pg_last_timing(const pg_game* g, double* total_ms, double* valuation_ms, double* switch_ms,
                         int64_t* valuations) {
    if (!g) return PG_EINVAL;
    if (total_ms) *total_ms = g->t_total;
    if (valuation_ms) *valuation_ms = g->t_val;
    if (switch_ms) *switch_ms = g->t_switch;
    if (valuations) *valuations = g->t_vals;
    return PG_OK;
}

pg_status pg_kernel_stats(const pg_game* g, pg_kernel_stat* out, int32_t cap, int32_t* count) {
    if (!g || (!out && cap > 0)) return PG_EINVAL;
    int32_t c = 0;
    for (int id = 0; id < KID_COUNT && c < cap; ++id, ++c) {
        memset(out[c].name, 0, sizeof(out[c].name));
        strncpy(out[c].name, kKernelNames[id], sizeof(out[c].name) - 1);
        out[c].ms = g->kms[id];
        out[c].launches = g->klaunch[id];
        out[c].calls = g->kcalls[id];
    }
    if (count) *count = KID_COUNT;
    return PG_OK;
}

pg_status pg_reset_stats(pg_game* g) {
    if (!g) return PG_EINVAL;
    for (int id = 0; id < KID_COUNT; ++id) {
        g->kms[id] = 0;
        g->klaunch[id] = 0;
        g->kcalls[id] = 0;
        g->kpend[id] = false;
    }
    return PG_OK;
}

pg_status pg_launch_count(const pg_ctx* ctx, int64_t* out) {
    if (!ctx || !out) return PG_EINVAL;
    *out = ctx->launches;
    return PG_OK;
}

pg_status pg_load_csr(pg_ctx* ctx, int32_t n, int64_t m, const int32_t* offsets, const int32_t* targets,
                      const uint8_t* owner, const int32_t* pri, int32_t mem_kind, pg_game** out) {
    if (!ctx) return PG_EINVAL;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return fail(ctx, PG_ECUDA, "cudaSetDevice failed");
    return load_game(ctx, n, m, offsets, targets, owner, pri, mem_kind, out);
}

void pg_game_free(pg_game* game) { free_game(game); }

pg_status pg_game_info(const pg_game* g, int32_t* n, int64_t* m, int32_t* k) {
    if (!g) return PG_EINVAL;
    if (n) *n = g->n0;
    if (m) *m = g->m0;
    if (k) *k = g->k;
    return PG_OK;
}

pg_status pg_game_counters(const pg_game* g, pg_counters* out) {
    if (!g || !out || !g->hcnt) return PG_EINVAL;
    const Counters& c = *g->hcnt;  // copied to the host at the end of every valuation
    *out = {c.n_pending, c.jump_rounds, c.n_fin, c.n_odd, c.n_big, c.n_huge, c.n_switch,
            g->val_deep ? 1 : 0, c.n_rulers, c.deep_rounds, c.rs_rounds};
    return PG_OK;
}

pg_status pg_game_levels(const pg_game* g, int32_t* d, int32_t* level_pri) {
    if (!g || !d) return PG_EINVAL;
    *d = g->cv ? g->lev.n : 0;
    if (level_pri && g->cv)
        for (int32_t l = 0; l < g->lev.n; ++l) level_pri[l] = g->lev_pri[l];
    return PG_OK;
}

pg_status pg_game_dummies(const pg_game* g, int32_t* out) {
    if (!g || (!out && g->k)) return PG_EINVAL;
    if (g->k == 0) return PG_OK;
    cudaError_t e = cudaMemcpyAsync(out, g->dummy_of, sizeof(int32_t) * g->k, cudaMemcpyDeviceToHost, g->ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(g->ctx->stream);
    return e == cudaSuccess ? PG_OK : cuda_fail(g->ctx, e, "pg_game_dummies");
}

pg_status pg_solve(pg_game* g, const pg_solve_opts* opts, pg_result* out) {
    if (!g || !out) return g ? fail(g->ctx, PG_EINVAL, "pg_solve: out is NULL") : PG_EINVAL;
    pg_ctx* ctx = g->ctx;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return fail(ctx, PG_ECUDA, "cudaSetDevice failed");
    int64_t cap = (opts && opts->max_inner > 0) ? opts->max_inner : 64 * ((int64_t)g->n + 64);
    pg_status st = apply_profile(g, opts ? opts->sigma_init : nullptr, opts ? opts->tau_init : nullptr,
                                 opts ? opts->dummy_sigma_init : nullptr, opts ? opts->mem_kind : PG_MEM_HOST);
    if (!st) st = reset_scratch(g);
    if (st) return st;
    Timer tm(g);
    tm.mark(3);
    g->reset_tau = opts && opts->reset_tau;
    st = run_loop(g, cap, true, tm);
    g->reset_tau = false;
    if (st) return st;
    GameState gs;
    PG_CUDA_TRY(ctx, cudaMemcpy(&gs, g->gst, sizeof(gs), cudaMemcpyDeviceToHost));
    if (gs.phase == kPhaseOddCycle)
        return fail(ctx, PG_ENOTADMISSIBLE, "pg_solve: an odd cycle was reached: sigma is not admissible");
    const bool timed_out = gs.phase == kPhaseTimeout;
    if (timed_out || g->last_cmp) {
        st = full_valuation(g, false);  // the full valuation of the profile being returned
        if (st) return st;
        g->last_cmp = false;
    }
    tm.mark(2);
    g->t_total = tm.since(3, 2);
    out->major = gs.major;
    out->inner = gs.inner;
    st = write_outputs(g, out->mem_kind, out->win, out->sigma, out->tau, out->val_class, out->val_depth,
                       out->val_rank, nullptr, out->dummy_sigma);
    if (!st && g->cv && out->val_counts) st = write_counts(g, out->mem_kind, out->val_counts);
    if (st) return st;
    if (timed_out) return fail(ctx, PG_ETIMEOUT, "pg_solve: iteration cap reached");
    return PG_OK;
}

pg_status pg_best_response(pg_game* g, const int32_t* sigma, const int8_t* dummy_sigma, int32_t* tau_inout,
                           int32_t mem_kind, pg_valuation* out, int64_t* iters_out) {
    if (!g) return PG_EINVAL;
    pg_ctx* ctx = g->ctx;
    if (!sigma) return fail(ctx, PG_EINVAL, "pg_best_response: sigma is NULL");
    if (cudaSetDevice(ctx->device) != cudaSuccess) return fail(ctx, PG_ECUDA, "cudaSetDevice failed");
    pg_status st = apply_profile(g, sigma, tau_inout, dummy_sigma, mem_kind);
    if (!st) st = reset_scratch(g);
    if (st) return st;
    Timer tm(g);
    tm.mark(3);
    st = run_loop(g, 64 * ((int64_t)g->n + 64), false, tm);
    if (st) return st;
    GameState gs;
    PG_CUDA_TRY(ctx, cudaMemcpy(&gs, g->gst, sizeof(gs), cudaMemcpyDeviceToHost));
    if (iters_out) *iters_out = gs.inner;
    if (gs.phase == kPhaseOddCycle)
        return fail(ctx, PG_ENOTADMISSIBLE, "an odd cycle was reached: sigma is not admissible");
    const bool timed_out = gs.phase == kPhaseTimeout;
    st = finish_loop(g);  // ranks of the best response's valuation
    if (st) return st;
    tm.mark(2);
    g->t_total = tm.since(3, 2);
    st = write_outputs(g, mem_kind, nullptr, nullptr, tau_inout, nullptr, nullptr, nullptr, nullptr, nullptr);
    if (st) return st;
    if (out) {
        st = write_outputs(g, out->mem_kind, nullptr, nullptr, nullptr, out->val_class, out->val_depth,
                           out->val_rank, nullptr, nullptr);
        if (!st && g->cv && out->val_counts) st = write_counts(g, out->mem_kind, out->val_counts);
        if (st) return st;
        if (out->dom) {
            // dom needs a valuation that records it
            st = full_valuation(g, true);
            if (st) return st;
            st = write_outputs(g, out->mem_kind, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, out->dom,
                               nullptr);
            if (st) return st;
        }
    }
    if (timed_out) return fail(ctx, PG_ETIMEOUT, "pg_best_response: iteration cap reached");
    return PG_OK;
}

pg_status pg_best_response_bf(pg_game* g, const int32_t* sigma, const int8_t* dummy_sigma, int32_t* tau_out,
                              int32_t mem_kind, pg_valuation* out, int64_t* rounds_out) {
    if (!g) return PG_EINVAL;
    pg_ctx* ctx = g->ctx;
    if (!sigma) return fail(ctx, PG_EINVAL, "pg_best_response_bf: sigma is NULL");
    if (!g->cv) return fail(ctx, PG_EUNSUPPORTED, "pg_best_response_bf: count-vector mode only (repeated priorities)");
    if (cudaSetDevice(ctx->device) != cudaSuccess) return fail(ctx, PG_ECUDA, "cudaSetDevice failed");
    pg_status st = apply_profile(g, sigma, nullptr, dummy_sigma, mem_kind);
    if (!st) st = reset_scratch(g);
    if (st) return st;
    Timer tm(g);
    tm.mark(3);
    int64_t rounds = 0;
    st = bellman_ford_cv(g, &rounds);
    if (rounds_out) *rounds_out = rounds;
    if (st) return st;
    tm.mark(2);
    g->t_total = tm.since(3, 2);
    // the valuation of (sigma, the Bellman-Ford best response) for the outputs
    st = enqueue_valuation(g, out && out->dom);
    if (!st) st = sync_counters(g);
    if (!st) st = write_outputs(g, mem_kind, nullptr, nullptr, tau_out, nullptr, nullptr, nullptr, nullptr, nullptr);
    if (!st && out) {
        st = write_outputs(g, out->mem_kind, nullptr, nullptr, nullptr, out->val_class, out->val_depth, out->val_rank,
                           out->dom, nullptr);
        if (!st && out->val_counts) st = write_counts(g, out->mem_kind, out->val_counts);
    }
    if (st) return st;
    if (g->hcnt->n_odd > 0) return fail(ctx, PG_ENOTADMISSIBLE, "pg_best_response_bf: an odd cycle was reached");
    return PG_OK;
}

pg_status pg_valuate(pg_game* g, const int32_t* sigma, const int8_t* dummy_sigma, const int32_t* tau,
                     int32_t mem_kind, pg_valuation* out) {
    if (!g) return PG_EINVAL;
    pg_ctx* ctx = g->ctx;
    if (cudaSetDevice(ctx->device) != cudaSuccess) return fail(ctx, PG_ECUDA, "cudaSetDevice failed");
    pg_status st = apply_profile(g, sigma, tau, dummy_sigma, mem_kind);
    if (!st) st = reset_scratch(g);
    if (st) return st;
    Timer tm(g);
    tm.mark(0);
    st = full_valuation(g, true);
    if (st) return st;
    tm.mark(1);
    g->t_val = g->t_total = tm.since(0, 1);
    g->t_vals = 1;
    if (out) {
        st = write_outputs(g, out->mem_kind, nullptr, nullptr, nullptr, out->val_class, out->val_depth, out->val_rank,
                           out->dom, nullptr);
        if (!st && g->cv && out->val_counts) st = write_counts(g, out->mem_kind, out->val_counts);
        if (st) return st;
    }
    if (g->hcnt->n_odd > 0) return fail(ctx, PG_ENOTADMISSIBLE, "pg_valuate: the profile reaches an odd cycle");
    return PG_OK;
}

}  // extern "C"
