// Loading a game: validation, the admissibility preprocessing of Section 3
// ("The algorithm": dummy Even vertices in Odd's Even-free trap), and the
// relabelling of G' by priority rank. Runs once per game, entirely on the
// device; only a few scalars cross to the host (sizes and error bits).
#include <stdio.h>

#include <vector>

#include "pg_device.cuh"

namespace pg {
namespace {

constexpr int32_t kEOff = 1, kETgt = 2, kEOwn = 4, kEPri = 8, kEDup = 16;

struct LoadScalars {
    int32_t err;
    int32_t maxpri;
    int32_t frontier;
    int32_t pad;
};

inline unsigned nblocks(int64_t n, int per = kBlock) {
    int64_t b = (n + per - 1) / per;
    if (b < 1) b = 1;
    if (b > (1ll << 30)) b = 1ll << 30;
    return (unsigned)b;
}

__global__ void k_validate(int32_t n, int64_t m, const int32_t* off, const int32_t* tgt, const uint8_t* own,
                           const int32_t* pri, LoadScalars* sc) {
    int32_t err = 0, mx = -1;
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x, nthr = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = tid; v < n; v += nthr) {
        int32_t a = off[v], b = off[v + 1];
        if (b <= a || a < 0 || (int64_t)b > m) err |= kEOff;
        if (v == 0 && a != 0) err |= kEOff;
        if (v == n - 1 && (int64_t)b != m) err |= kEOff;
        if (own[v] > 1) err |= kEOwn;
        if (pri[v] < 0) err |= kEPri;
        if (pri[v] > mx) mx = pri[v];
    }
    for (int64_t e = tid; e < m; e += nthr)  // every target, in order (the array holds m whatever the offsets)
        if (tgt[e] < 0 || tgt[e] >= n) err |= kETgt;
    // one atomic of each kind per warp
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        err |= __shfl_xor_sync(0xffffffffu, err, o);
        mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    }
    if ((threadIdx.x & 31) == 0) {
        if (err) atomicOr(&sc->err, err);
        atomicMax(&sc->maxpri, mx);
    }
}

// Marks every priority in a bitmap; a bit already set means a repeated priority.
// The lanes of a warp that mark the same word combine their bits first (one
// atomic per word and warp), and a word that already holds all of them takes no
// atomic at all: with few distinct priorities every vertex marks one of a few
// words, which would otherwise serialise n atomics on them.
__global__ void k_mark_priorities(int32_t n, const int32_t* pri, int32_t shift_orig, int32_t n_orig,
                                  uint32_t* bits, LoadScalars* sc, int dummy_zero) {
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v0 = (int64_t)blockIdx.x * blockDim.x; v0 < n; v0 += stride) {  // uniform per block
        const int64_t v = v0 + threadIdx.x;
        const bool ok = v < n;
        // vertices below n_orig are original (priority shifted by shift_orig); the rest are dummies with 2j (0)
        int64_t p = !ok ? 0 : v < n_orig ? (int64_t)pri[v] + shift_orig : (dummy_zero ? 0 : 2 * (v - n_orig));
        const uint64_t word = ok ? (uint64_t)(p >> 5) : ~0ull;
        const uint32_t bit = ok ? 1u << (p & 31) : 0u;
        const unsigned peers = __match_any_sync(0xffffffffu, word);
        const uint32_t all = __reduce_or_sync(peers, bit);
        if (!ok || lane != __ffs(peers) - 1) continue;
        bool dup = __popc(all) < __popc(peers);  // two lanes of this warp share a priority
        const uint32_t cur = *(volatile uint32_t*)&bits[word];
        if ((cur & all) != 0) dup = true;
        if ((cur & all) != all) dup |= (atomicOr(&bits[word], all) & all) != 0;
        if (dup && !(*(volatile int32_t*)&sc->err & kEDup)) atomicOr(&sc->err, kEDup);
    }
}

// The reverse adjacency of the trap computation holds only the edges between
// Odd vertices: U starts as the Odd vertices, and peeling only ever lowers the
// counts of Odd predecessors of Odd vertices.
__global__ void k_indegree(int32_t n, const int32_t* off, const int32_t* tgt, const uint8_t* own, int32_t* indeg) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        if (own[v] != 1) continue;
        for (int32_t e = off[v]; e < off[v + 1]; ++e)
            if (own[tgt[e]] == 1) atomicAdd(&indeg[tgt[e]], 1);
    }
}

__global__ void k_reverse_scatter(int32_t n, const int32_t* off, const int32_t* tgt, const uint8_t* own,
                                  int32_t* fill, int32_t* radj) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        if (own[v] != 1) continue;
        for (int32_t e = off[v]; e < off[v + 1]; ++e) {
            const int32_t t = tgt[e];
            if (own[t] == 1) radj[atomicAdd(&fill[t], 1)] = (int32_t)v;
        }
    }
}

// U starts as every Odd vertex; cnt[v] = edges of v into Odd vertices. Odd
// vertices without such an edge leave U first.
__global__ void k_trap_init(int32_t n, const int32_t* off, const int32_t* tgt, const uint8_t* own, uint8_t* inU,
                            int32_t* cnt, int32_t* frontier, LoadScalars* sc) {
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    // warp-uniform rounds (the frontier is appended one atomic per warp)
    for (int64_t b = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) - lane; b < n; b += stride) {
        const int64_t v = b + lane;
        bool push = false;
        if (v < n) {
            if (own[v] != 1) {
                inU[v] = 0;
            } else {
                int32_t c = 0;
                for (int32_t e = off[v]; e < off[v + 1]; ++e) c += own[tgt[e]] == 1;
                cnt[v] = c;
                inU[v] = c > 0;
                push = c == 0;
            }
        }
        const int32_t slot = warp_append(push, &sc->frontier);
        if (push) frontier[slot] = (int32_t)v;
    }
}

// W: vertices of U entered by an edge from U.
__global__ void k_mark_w(int32_t n, const int32_t* off, const int32_t* tgt, const uint8_t* inU, uint8_t* isW) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        if (!inU[v]) continue;
        for (int32_t e = off[v]; e < off[v + 1]; ++e)
            if (inU[tgt[e]]) isW[tgt[e]] = 1;
    }
}

__global__ void k_dummy_of(int32_t n, const uint8_t* isW, const int32_t* widx, int32_t* dummy_of) {
    for (int64_t w = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; w < n; w += (int64_t)gridDim.x * blockDim.x)
        if (isW[w]) dummy_of[widx[w]] = (int32_t)w;
}

// Peeling without rounds: every vertex x that leaves U decrements the count of
// its Odd predecessors, and a predecessor whose count reaches zero leaves U
// too. Each thread takes vertices of the initial frontier and peels what they
// free depth first, keeping up to kPeelStack vertices of its own and peeling at
// most kPeelBudget per frontier vertex; a vertex freed beyond either goes to the
// overflow list (counted in c->left[0]), which k_trap_peel_coop then peels in
// rounds across the grid (a large cascade must not run in one thread). The set
// left in U does not depend on the order of the decrements.
constexpr int kPeelStack = 16;
constexpr int kPeelBudget = 64;

__global__ void __launch_bounds__(kBlock) k_trap_peel_dfs(const int32_t* __restrict__ frontier, const LoadScalars* sc,
                                                          const int32_t* __restrict__ roff,
                                                          const int32_t* __restrict__ radj,
                                                          const uint8_t* __restrict__ own, uint8_t* inU, int32_t* cnt,
                                                          int32_t* overflow, Counters* c) {
    const int32_t nf = sc->frontier;
    int32_t stack[kPeelStack];
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < nf; i += gridDim.x * blockDim.x) {
        int32_t top = 0, budget = kPeelBudget;
        stack[top++] = frontier[i];
        while (top > 0) {
            const int32_t x = stack[--top];
            if (--budget < 0) {  // the rest of this cascade is peeled in rounds
                overflow[atomicAdd(&c->left[0], 1)] = x;
                continue;
            }
            const int32_t e1 = roff[x + 1];
            for (int32_t e = roff[x]; e < e1; ++e) {
                const int32_t y = radj[e];
                if (own[y] == 1 && atomicSub(&cnt[y], 1) == 1) {
                    inU[y] = 0;
                    if (top < kPeelStack) stack[top++] = y;
                    else overflow[atomicAdd(&c->left[0], 1)] = y;
                }
            }
        }
    }
}

// Peeling in rounds: every vertex x that leaves U decrements the count of its Odd
// predecessors; a predecessor whose count reaches zero leaves U in the next
// round. Every round runs in one cooperative launch, with a grid barrier
// between rounds (the barrier gives up after a bounded wait and records
// kErrBarrier). c->left[r % 3] counts round r's frontier (left[0] is the
// initial one); round r appends the next frontier through left[(r + 1) % 3],
// which block 0 cleared in round r - 1, and clears left[(r + 2) % 3]. The set
// left in U does not depend on the order of the decrements.
__global__ void __launch_bounds__(kBlock) k_trap_peel_coop(const int32_t* __restrict__ roff,
                                                           const int32_t* __restrict__ radj,
                                                           const uint8_t* __restrict__ own, uint8_t* inU, int32_t* cnt,
                                                           int32_t* fa, int32_t* fb, Counters* c, int32_t max_rounds) {
    int32_t* cur = fa;
    int32_t* nxt = fb;
    for (int32_t r = 0; r < max_rounds; ++r) {
        if (blockIdx.x == 0 && threadIdx.x == 0) c->left[(r + 2) % 3] = 0;
        const int32_t nf = *(volatile int32_t*)&c->left[r % 3];
        if (nf == 0) return;  // every block reads the same count after the barrier
        for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < nf; i += gridDim.x * blockDim.x) {
            const int32_t x = __ldcg(cur + i);
            for (int32_t e = roff[x]; e < roff[x + 1]; ++e) {
                const int32_t y = radj[e];
                if (own[y] == 1 && atomicSub(&cnt[y], 1) == 1) {
                    inU[y] = 0;
                    __stcg(nxt + atomicAdd(&c->left[(r + 1) % 3], 1), y);
                }
            }
        }
        if (!grid_sync(c)) return;
        int32_t* t = cur;
        cur = nxt;
        nxt = t;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(&c->err, kErrJumpRounds);  // more rounds than vertices
}

// G' priority: distinct priorities (cv = 0): originals + 2k, dummy j has 2j;
// repeated priorities (cv = 1): originals + 2, every dummy 0.
__device__ inline int32_t prio_of(int64_t v, int32_t n0, const int32_t* pri, int32_t k, int cv) {
    if (cv) return v < n0 ? pri[v] + 2 : 0;
    return v < n0 ? pri[v] + 2 * k : (int32_t)(2 * (v - n0));
}

// relabelled id of every G' vertex = rank of its priority
__global__ void k_rank(int32_t np, int32_t n0, int32_t k, const int32_t* pri, const uint32_t* bits,
                       const int32_t* wprefix, int32_t* nid, int32_t* gid) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < np; v += (int64_t)gridDim.x * blockDim.x) {
        int32_t p = prio_of(v, n0, pri, k, 0);
        int32_t r = wprefix[p >> 5] + __popc(bits[p >> 5] & ((1u << (p & 31)) - 1u));
        nid[v] = r;
        gid[r] = (int32_t)v;
    }
}

// Repeated priorities: level of every G' vertex = rank of its priority value
// among the distinct values.
__global__ void k_level(int32_t np, int32_t n0, const int32_t* pri, const uint32_t* bits, const int32_t* wprefix,
                        uint8_t* lvl) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < np; v += (int64_t)gridDim.x * blockDim.x) {
        int32_t p = prio_of(v, n0, pri, 0, 1);
        lvl[v] = (uint8_t)(wprefix[p >> 5] + __popc(bits[p >> 5] & ((1u << (p & 31)) - 1u)));
    }
}

__global__ void k_is_level(int32_t np, const uint8_t* lvl, int32_t l, uint8_t* ind) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < np; v += (int64_t)gridDim.x * blockDim.x)
        ind[v] = lvl[v] == l;
}

// relabelled id = first id of the level + position among the level's vertices in G' order
__global__ void k_assign_level(int32_t np, const uint8_t* lvl, int32_t l, int32_t start, const int32_t* pos,
                               int32_t* nid, int32_t* gid) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < np; v += (int64_t)gridDim.x * blockDim.x) {
        if (lvl[v] != l) continue;
        const int32_t r = start + pos[v];
        nid[v] = r;
        gid[r] = (int32_t)v;
    }
}

// What the relabelling reads of an input vertex, packed in input order so that
// the passes in relabelled order gather one 16-byte record per vertex: x = its
// first edge, y = its out-degree, z = its G' priority, w = bit 0: owned by Odd,
// bit 1: in U.
__global__ void k_pack_vertices(int32_t n0, const int32_t* off, const uint8_t* own, const int32_t* pri,
                                const uint8_t* inU, int32_t k, int cv, int4* rec) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n0; v += (int64_t)gridDim.x * blockDim.x) {
        const int32_t e0 = off[v];
        rec[v] = make_int4(e0, off[v + 1] - e0, prio_of(v, n0, pri, k, cv), (own[v] ? 1 : 0) | (inU[v] ? 2 : 0));
    }
}

__global__ void k_relabel_degree(int32_t np, int32_t n0, const int4* rec, const int32_t* gid, int32_t* deg) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < np; i += (int64_t)gridDim.x * blockDim.x) {
        int32_t src = gid[i];
        deg[i] = src < n0 ? rec[src].y : 1;
    }
}

// New id of each input vertex as the target of an edge from U: its dummy's for
// a vertex of W (the edge is redirected to the dummy), its own otherwise.
__global__ void k_nid_u(int32_t n0, const uint8_t* isW, const int32_t* widx, const int32_t* nid, int32_t* nidu) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n0; v += (int64_t)gridDim.x * blockDim.x)
        nidu[v] = isW[v] ? nid[n0 + widx[v]] : nid[v];
}

__global__ void k_relabel_rows(int32_t np, int32_t n0, int32_t k, const int4* rec, const int32_t* tgt,
                               const int32_t* nidu, const int32_t* dummy_of, const int32_t* gid, const int32_t* nid,
                               const int32_t* roff, int32_t* rtgt, uint8_t* rflags, int32_t* rpri,
                               int32_t* orig_of, int cv) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < np; i += (int64_t)gridDim.x * blockDim.x) {
        int32_t src = gid[i];
        int32_t p = src < n0 ? 0 : prio_of(src, n0, nullptr, k, cv);
        int32_t base = roff[i];
        if (src < n0) {
            const int4 r = rec[src];
            p = r.z;
            // edges from U to W go to the dummy of their target (every target of an edge from U in U is in W)
            const int32_t* map = (r.w & 2) ? nidu : nid;
            for (int32_t j = 0; j < r.y; ++j) rtgt[base + j] = map[tgt[r.x + j]];
            rflags[i] = (uint8_t)(((r.w & 1) ? kOwnerOdd : 0) | ((p & 1) ? kPriOdd : 0));
            orig_of[i] = src;
        } else {
            int32_t w = dummy_of[src - n0];
            rtgt[base] = nid[w];
            rflags[i] = (uint8_t)((p & 1) ? kPriOdd : 0);  // dummies are Even
            orig_of[i] = w;
        }
        rpri[i] = p;
    }
}

__global__ void k_maps(int32_t n0, int32_t k, const int32_t* nid, int32_t* nid0, int32_t* dnid) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n0 + (int64_t)k;
         v += (int64_t)gridDim.x * blockDim.x) {
        if (v < n0) nid0[v] = nid[v];
        else dnid[v - n0] = nid[v];
    }
}

// The game's own arrays, stream-ordered on the load stream from the game
// pool (no global allocation lock between concurrent loads); the load
// synchronises its stream before returning, so they are valid on every stream
// afterwards.
template <typename T>
cudaError_t dalloc(pg_ctx* ctx, T** p, int64_t count, cudaStream_t s) {
    return dev_alloc(ctx, (void**)p, (size_t)(count > 0 ? count : 1) * sizeof(T), s);
}

// Temporaries of one load, stream-ordered on the load's stream (allocating
// and freeing them does not synchronise the device, so loads can overlap
// other streams' work).
struct Temps {
    pg_ctx* ctx;
    cudaStream_t s;
    std::vector<void*> ptrs;
    Temps(pg_ctx* c, cudaStream_t st) : ctx(c), s(st) {}
    ~Temps() {
        for (void* p : ptrs) cudaFreeAsync(p, s);
    }
    template <typename T>
    cudaError_t get(T** p, int64_t count) {
        cudaError_t e = dev_alloc(ctx, (void**)p, (size_t)(count > 0 ? count : 1) * sizeof(T), s);
        if (e == cudaSuccess) ptrs.push_back((void*)*p);
        return e;
    }
};

}  // namespace

// Vertices whose priorities are checked for repeats before the load chooses its
// mode: games with few distinct priorities repeat them within the first few
// hundred vertices; a repeat further on is found by the ranking pass, and the
// load then runs again in the count-vector mode.
constexpr int32_t kDupProbe = 1 << 16;

// One load; with cv_forced the count-vector mode is chosen without looking.
// *again is set (and nothing returned) when a priority repeats beyond the probe.
pg_status load_game_pass(pg_ctx* ctx, int32_t n, int64_t m, const int32_t* off_in, const int32_t* tgt_in,
                         const uint8_t* own_in, const int32_t* pri_in, int32_t mem_kind, pg_game** out,
                         bool with_scratch, bool cv_forced, bool* again) {
    if (!out) return fail(ctx, PG_EINVAL, "pg_load_csr: out is NULL");
    *out = nullptr;
    if (!off_in || !tgt_in || !own_in || !pri_in) return fail(ctx, PG_EINVAL, "pg_load_csr: NULL array");
    if (mem_kind != PG_MEM_HOST && mem_kind != PG_MEM_DEVICE) return fail(ctx, PG_EINVAL, "pg_load_csr: bad mem_kind");
    if (n < 1 || n >= (1 << 29)) return fail(ctx, PG_EINVAL, "pg_load_csr: n must be in [1, 2^29)");
    if (m < n || m > INT32_MAX - 1) return fail(ctx, PG_EINVAL, "pg_load_csr: m must be in [n, 2^31-1)");
    cudaStream_t s = ctx->stream;
    cudaMemcpyKind kind = mem_kind == PG_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    Temps T(ctx, s);
    int32_t *off, *tgt, *pri;
    uint8_t* own;
    LoadScalars* sc;
    PG_CUDA_TRY(ctx, T.get(&off, (int64_t)n + 1));
    PG_CUDA_TRY(ctx, T.get(&tgt, m));
    PG_CUDA_TRY(ctx, T.get(&own, n));
    PG_CUDA_TRY(ctx, T.get(&pri, n));
    PG_CUDA_TRY(ctx, T.get(&sc, 1));
    PG_CUDA_TRY(ctx, cudaMemcpyAsync(off, off_in, sizeof(int32_t) * ((size_t)n + 1), kind, s));
    PG_CUDA_TRY(ctx, cudaMemcpyAsync(tgt, tgt_in, sizeof(int32_t) * (size_t)m, kind, s));
    PG_CUDA_TRY(ctx, cudaMemcpyAsync(own, own_in, (size_t)n, kind, s));
    PG_CUDA_TRY(ctx, cudaMemcpyAsync(pri, pri_in, sizeof(int32_t) * (size_t)n, kind, s));
    PG_CUDA_TRY(ctx, cudaMemsetAsync(sc, 0, sizeof(LoadScalars), s));
    {
        LoadScalars init = {0, -1, 0, 0};
        PG_CUDA_TRY(ctx, cudaMemcpyAsync(sc, &init, sizeof(init), cudaMemcpyHostToDevice, s));
    }
    ++ctx->launches;
    k_validate<<<nblocks(n), kBlock, 0, s>>>(n, m, off, tgt, own, pri, sc);
    LoadScalars h;
    PG_CUDA_TRY(ctx, cudaMemcpyAsync(&h, sc, sizeof(h), cudaMemcpyDeviceToHost, s));
    PG_CUDA_TRY(ctx, cudaStreamSynchronize(s));
    if (h.err & kEOff) return fail(ctx, PG_EINVAL, "pg_load_csr: offsets must start at 0, end at m, and give every vertex at least one edge");
    if (h.err & kETgt) return fail(ctx, PG_EINVAL, "pg_load_csr: edge target out of range");
    if (h.err & kEOwn) return fail(ctx, PG_EINVAL, "pg_load_csr: owner must be 0 (Even) or 1 (Odd)");
    if (h.err & kEPri) return fail(ctx, PG_EINVAL, "pg_load_csr: negative priority");
    int32_t maxpri = h.maxpri;

    // repeated priorities select the count-vector mode (probed on a prefix here)
    bool cv = cv_forced;
    if (!cv) {
        const int32_t nprobe = n < kDupProbe ? n : kDupProbe;
        int64_t nwords = ((int64_t)maxpri >> 5) + 1;
        uint32_t* bits;
        PG_CUDA_TRY(ctx, T.get(&bits, nwords));
        PG_CUDA_TRY(ctx, cudaMemsetAsync(bits, 0, sizeof(uint32_t) * (size_t)nwords, s));
        ++ctx->launches;
        k_mark_priorities<<<nblocks(nprobe), kBlock, 0, s>>>(nprobe, pri, 0, n, bits, sc, 0);
        PG_CUDA_TRY(ctx, cudaMemcpyAsync(&h, sc, sizeof(h), cudaMemcpyDeviceToHost, s));
        PG_CUDA_TRY(ctx, cudaStreamSynchronize(s));
        cv = (h.err & kEDup) != 0;
    }

    // reverse adjacency for the trap computation
    int32_t *indeg, *roff, *radj, *fill, *cnt, *fa, *fb, *widx;
    uint8_t *inU, *isW;
    size_t stb = scan_tmp_bytes((int64_t)n + 2) + 64;
    void* stmp;
    PG_CUDA_TRY(ctx, T.get((char**)&stmp, (int64_t)stb));
    PG_CUDA_TRY(ctx, T.get(&indeg, n));
    PG_CUDA_TRY(ctx, T.get(&roff, (int64_t)n + 1));
    PG_CUDA_TRY(ctx, T.get(&radj, m));
    PG_CUDA_TRY(ctx, T.get(&fill, (int64_t)n + 1));
    PG_CUDA_TRY(ctx, cudaMemsetAsync(indeg, 0, sizeof(int32_t) * (size_t)n, s));
    ++ctx->launches;
    k_indegree<<<nblocks(n), kBlock, 0, s>>>(n, off, tgt, own, indeg);
    ctx->launches += 3;
    PG_CUDA_TRY(ctx, exclusive_scan_i32(indeg, roff, n, nullptr, stmp, stb, s));
    PG_CUDA_TRY(ctx, cudaMemcpyAsync(fill, roff, sizeof(int32_t) * ((size_t)n + 1), cudaMemcpyDeviceToDevice, s));
    ++ctx->launches;
    k_reverse_scatter<<<nblocks(n), kBlock, 0, s>>>(n, off, tgt, own, fill, radj);

    // U: greatest fixpoint by peeling
    PG_CUDA_TRY(ctx, T.get(&cnt, n));
    PG_CUDA_TRY(ctx, T.get(&fa, n));
    PG_CUDA_TRY(ctx, T.get(&fb, n));
    PG_CUDA_TRY(ctx, T.get(&inU, n));
    Counters* pc;  // the peeling rounds' frontier counts and grid barrier
    PG_CUDA_TRY(ctx, T.get(&pc, 1));
    PG_CUDA_TRY(ctx, cudaMemsetAsync(pc, 0, sizeof(Counters), s));
    ++ctx->launches;
    k_trap_init<<<nblocks(n), kBlock, 0, s>>>(n, off, tgt, own, inU, cnt, fa, sc);
    ++ctx->launches;
    k_trap_peel_dfs<<<nblocks(n), kBlock, 0, s>>>(fa, sc, roff, radj, own, inU, cnt, fb, pc);
    {  // the overflow list (in fb), if any, in rounds
        int sms = 0, per = 0;
        PG_CUDA_TRY(ctx, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device));
        PG_CUDA_TRY(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_trap_peel_coop, kBlock, 0));
        int blocks = std::max(1, sms * std::max(1, std::min(per, 4)));
        int32_t max_rounds = n + 1;
        void* args[] = {(void*)&roff, (void*)&radj, (void*)&own, (void*)&inU, (void*)&cnt,
                        (void*)&fb,   (void*)&fa,   (void*)&pc,  (void*)&max_rounds};
        ++ctx->launches;
        PG_CUDA_TRY(ctx, cudaLaunchCooperativeKernel((void*)k_trap_peel_coop, blocks, kBlock, args, 0, s));
    }
    PG_CUDA_TRY(ctx, T.get(&isW, n));
    PG_CUDA_TRY(ctx, T.get(&widx, (int64_t)n + 1));
    PG_CUDA_TRY(ctx, cudaMemsetAsync(isW, 0, (size_t)n, s));
    ++ctx->launches;
    k_mark_w<<<nblocks(n), kBlock, 0, s>>>(n, off, tgt, inU, isW);
    ctx->launches += 3;
    PG_CUDA_TRY(ctx, exclusive_scan_u8(isW, widx, n, stmp, stb, s));
    int32_t k = 0, peel_err = 0;
    PG_CUDA_TRY(ctx, cudaMemcpyAsync(&k, widx + n, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    PG_CUDA_TRY(ctx, cudaMemcpyAsync(&peel_err, &pc->err, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    PG_CUDA_TRY(ctx, cudaStreamSynchronize(s));
    if (peel_err & kErrBarrier) return fail(ctx, PG_ECUDA, "pg_load_csr: a grid barrier of the trap peeling timed out");
    if (peel_err) return fail(ctx, PG_EINVAL, "pg_load_csr: trap peeling did not converge");
    int64_t np = (int64_t)n + k, mp = m + k;
    if (np >= (1 << 29) - 1) return fail(ctx, PG_EINVAL, "pg_load_csr: more than 2^29 vertices after preprocessing");
    if (mp > INT32_MAX - 1) return fail(ctx, PG_EINVAL, "pg_load_csr: more than 2^31-2 edges after preprocessing");
    if ((int64_t)maxpri + (cv ? 2 : 2 * (int64_t)k) > INT32_MAX - 1)
        return fail(ctx, PG_EINVAL, "pg_load_csr: priorities too large for the preprocessing shift");

    pg_game* g = new pg_game();
    g->ctx = ctx;
    g->device = ctx->device;
    g->n0 = n;
    g->m0 = m;
    g->k = k;
    g->n = (int32_t)np + 1;  // G' vertices and the sink slot
    g->m = mp;
    g->sink0 = (int32_t)np;
    g->ngames = 1;
    g->h_base0 = {0, (int64_t)n};
    g->h_dbase = {0, k};
    auto bail = [&](cudaError_t e, const char* where) {
        free_game(g);
        return cuda_fail(ctx, e, where);
    };
#define LG_TRY(expr)                                  \
    do {                                              \
        cudaError_t _e = (expr);                      \
        if (_e != cudaSuccess) return bail(_e, #expr); \
    } while (0)
    LG_TRY(dalloc(ctx, &g->off, np + 2, s));
    LG_TRY(dalloc(ctx, &g->tgt, mp, s));
    LG_TRY(dalloc(ctx, &g->flags, np + 1, s));
    LG_TRY(dalloc(ctx, &g->pri, np + 1, s));
    LG_TRY(dalloc(ctx, &g->nid0, n, s));
    LG_TRY(dalloc(ctx, &g->orig_of, np + 1, s));
    LG_TRY(dalloc(ctx, &g->dnid, k, s));
    LG_TRY(dalloc(ctx, &g->dummy_of, k, s));
    LG_TRY(dalloc(ctx, &g->strat, np + 1, s));
    LG_TRY(dalloc(ctx, &g->gsink, 1, s));
    ++ctx->launches;
    k_dummy_of<<<nblocks(n), kBlock, 0, s>>>(n, isW, widx, g->dummy_of);

    // ranks of the G' priorities
    int64_t pmax = (int64_t)maxpri + (cv ? 2 : 2 * (int64_t)k);
    int64_t nw = (pmax >> 5) + 1;
    uint32_t* bits2;
    int32_t *wprefix, *nid, *gid, *deg;
    LG_TRY(T.get(&bits2, nw));
    LG_TRY(T.get(&wprefix, nw + 1));
    LG_TRY(T.get(&nid, np));
    LG_TRY(T.get(&gid, np));
    LG_TRY(T.get(&deg, np));
    size_t stb2 = scan_tmp_bytes(nw > np + 1 ? nw : np + 1) + 64;
    void* stmp2;
    LG_TRY(T.get((char**)&stmp2, (int64_t)stb2));
    LG_TRY(cudaMemsetAsync(bits2, 0, sizeof(uint32_t) * (size_t)nw, s));
    LG_TRY(cudaMemsetAsync(&sc->err, 0, sizeof(int32_t), s));
    ++ctx->launches;
    k_mark_priorities<<<nblocks(np), kBlock, 0, s>>>((int32_t)np, pri, cv ? 2 : 2 * k, n, bits2, sc, cv ? 1 : 0);
    if (!cv) {  // a priority repeated beyond the probe would give two vertices one rank: load again instead
        LG_TRY(cudaMemcpyAsync(&h, sc, sizeof(h), cudaMemcpyDeviceToHost, s));
        LG_TRY(cudaStreamSynchronize(s));
        if (h.err & kEDup) {
            free_game(g);
            *again = true;
            return PG_OK;
        }
    }
    ctx->launches += 3;
    LG_TRY(exclusive_popc_scan(bits2, wprefix, nw, stmp2, stb2, s));
    if (!cv) {
        ++ctx->launches;
        k_rank<<<nblocks(np), kBlock, 0, s>>>((int32_t)np, n, k, pri, bits2, wprefix, nid, gid);
    } else {
        // levels: the distinct priorities of G'; ids by (priority, G' order)
        int32_t nlev = 0;
        LG_TRY(cudaMemcpyAsync(&nlev, wprefix + nw, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        LG_TRY(cudaStreamSynchronize(s));
        if (nlev > kMaxLevels) {
            free_game(g);
            return fail(ctx, PG_EUNSUPPORTED, "pg_load_csr: repeated priorities support at most 5 distinct priorities "
                                              "after preprocessing (the dummies' priority counts as one)");
        }

        uint8_t *lvl8, *ind;
        int32_t* pos;
        LG_TRY(T.get(&lvl8, np));
        LG_TRY(T.get(&ind, np));
        LG_TRY(T.get(&pos, np + 1));
        ++ctx->launches;
        k_level<<<nblocks(np), kBlock, 0, s>>>((int32_t)np, n, pri, bits2, wprefix, lvl8);
        g->cv = true;
        g->lev.n = nlev;
        int32_t start = 0;
        for (int32_t l = 0; l < nlev; ++l) {
            g->lev.start[l] = start;
            ctx->launches += 5;
            k_is_level<<<nblocks(np), kBlock, 0, s>>>((int32_t)np, lvl8, l, ind);
            LG_TRY(exclusive_scan_u8(ind, pos, np, stmp2, stb2, s));
            k_assign_level<<<nblocks(np), kBlock, 0, s>>>((int32_t)np, lvl8, l, start, pos, nid, gid);
            int32_t cnt_l = 0;
            LG_TRY(cudaMemcpyAsync(&cnt_l, pos + np, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
            LG_TRY(cudaStreamSynchronize(s));
            start += cnt_l;
        }
        g->lev.start[nlev] = start;
        // digits: level l's count on a play never exceeds the level's size, so its digit takes one bit more
        // than that size's bit length; the digits of all levels share the 126 bits below the top key
        int32_t shift = 0;
        for (int32_t l = 0; l < nlev; ++l) {
            const int64_t size = (int64_t)g->lev.start[l + 1] - g->lev.start[l];
            int32_t w = 1;
            while (w < 40 && (size >> w) != 0) ++w;
            g->lev.shift[l] = shift;
            shift += w + 1;
        }
        g->lev.shift[nlev] = shift;
        if (shift > kKeyBits) {
            free_game(g);
            return fail(ctx, PG_EUNSUPPORTED, "pg_load_csr: repeated priorities: the count digits of the levels "
                                              "(each one bit more than the bit length of its level's size) exceed "
                                              "126 bits");
        }
    }
    ++ctx->launches;
    int4* rec;
    LG_TRY(T.get(&rec, n));
    ++ctx->launches;
    k_pack_vertices<<<nblocks(n), kBlock, 0, s>>>(n, off, own, pri, inU, k, cv ? 1 : 0, rec);
    k_relabel_degree<<<nblocks(np), kBlock, 0, s>>>((int32_t)np, n, rec, gid, deg);
    ctx->launches += 3;
    LG_TRY(exclusive_scan_i32(deg, g->off, np, nullptr, stmp2, stb2, s));
    int32_t* nidu;
    LG_TRY(T.get(&nidu, n));
    ctx->launches += 2;
    k_nid_u<<<nblocks(n), kBlock, 0, s>>>(n, isW, widx, nid, nidu);
    k_relabel_rows<<<nblocks(np), kBlock, 0, s>>>((int32_t)np, n, k, rec, tgt, nidu, g->dummy_of, gid, nid, g->off,
                                                  g->tgt, g->flags, g->pri, g->orig_of, cv ? 1 : 0);
    ++ctx->launches;
    k_maps<<<nblocks(np), kBlock, 0, s>>>(n, k, nid, g->nid0, g->dnid);
    // the sink slot: no edges, a flag, no priority or original vertex
    {
        const int32_t sk = (int32_t)np;
        const uint8_t sf = kSinkSlot;
        LG_TRY(cudaMemcpyAsync(g->off + np + 1, g->off + np, sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
        LG_TRY(cudaMemcpyAsync(g->flags + np, &sf, 1, cudaMemcpyHostToDevice, s));
        LG_TRY(cudaMemsetAsync(g->pri + np, 0xff, sizeof(int32_t), s));
        LG_TRY(cudaMemsetAsync(g->orig_of + np, 0xff, sizeof(int32_t), s));
        LG_TRY(cudaMemcpyAsync(g->strat + np, &sk, sizeof(int32_t), cudaMemcpyHostToDevice, s));
        LG_TRY(cudaMemcpyAsync(g->gsink, &sk, sizeof(int32_t), cudaMemcpyHostToDevice, s));
    }
    LG_TRY(cudaMemcpyAsync(&h, sc, sizeof(h), cudaMemcpyDeviceToHost, s));
    LG_TRY(cudaStreamSynchronize(s));
    LG_TRY(cudaGetLastError());
    if (cv) {  // each level's priority and parity
        g->lev.odd_mask = 0;
        for (int32_t l = 0; l < g->lev.n; ++l) {
            LG_TRY(cudaMemcpy(&g->lev_pri[l], g->pri + g->lev.start[l], sizeof(int32_t), cudaMemcpyDeviceToHost));
            if (g->lev_pri[l] & 1) g->lev.odd_mask |= 1u << l;
        }
    }
    if (!cv && (h.err & kEDup)) {
        free_game(g);
        return fail(ctx, PG_EUNSUPPORTED, "pg_load_csr: internal priority collision after preprocessing");
    }
#undef LG_TRY
    pg_status st = with_scratch ? alloc_scratch(g) : PG_OK;
    if (st != PG_OK) {
        free_game(g);
        return st;
    }
    *out = g;
    return PG_OK;
}

pg_status load_game(pg_ctx* ctx, int32_t n, int64_t m, const int32_t* off_in, const int32_t* tgt_in,
                    const uint8_t* own_in, const int32_t* pri_in, int32_t mem_kind, pg_game** out, bool with_scratch) {
    bool again = false;
    pg_status st = load_game_pass(ctx, n, m, off_in, tgt_in, own_in, pri_in, mem_kind, out, with_scratch, false, &again);
    if (st != PG_OK || !again) return st;
    return load_game_pass(ctx, n, m, off_in, tgt_in, own_in, pri_in, mem_kind, out, with_scratch, true, &again);
}

}  // namespace pg
