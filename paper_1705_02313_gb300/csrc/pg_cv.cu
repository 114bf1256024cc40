// Count-vector mode: valuations of games whose priorities repeat (Section 3,
// "Valuations": L(p) counts how often priority p occurs on the play from v to
// the sink, v included), for at most kMaxLevels distinct priorities.
//
// Ids are ranks by (priority, input order), so the ids of one priority form
// a range (a level) and the largest id on a cycle has the cycle's largest
// priority. A count vector is encoded as one signed 128-bit key
//   key(v) = sum over levels l of s_l * L_l(v) * 2^(shift_l),  s_l = +1 (even), -1 (odd),
// with the digit of level l one bit wider than the bit length of the level's
// size (L.shift), so every digit stays below half its range in magnitude and
// the digits below any level sum to less than that level's unit: keys
// compare exactly as valuations do under Maxdiff: the largest level whose
// counts differ decides, more is better when its priority is even. The key is
// a sum of per-vertex weights along the play, computed over the same
// nearest-greater decomposition as the distinct-priority path:
//   k_walk_cv      g(v) by a direct walk, with the weight of the segment [v, g(v))
//   k_jump_cv_coop pointer jumping for the walks that ran out of steps, with
//                  the weights (two buffers per round, so every read sees one
//                  consistent (word, weight) pair)
//   k_chain_cv     classification and key = sum of segment weights along the g-chain
//   k_switch_cv    the switching rules of Section 3 and Section 4 on the keys
#include "pg_internal.cuh"

namespace pg {
namespace {

using i128 = __int128;

constexpr unsigned kFullMask = 0xffffffffu;
constexpr int kIlpCv = 2;  // walks per thread (2 / 3 / 4 / 6: 129.0 / 133.9 / 136.0 / 168.5 ms per 10M 4-priority solve)

__device__ inline i128 top_key() { return (i128)(~(unsigned __int128)0 >> 1); }

__device__ inline int level_of(const Levels& L, int32_t v) {
    int l = 0;
#pragma unroll
    for (int i = 1; i < kMaxLevels; ++i) l += (i < L.n && v >= L.start[i]) ? 1 : 0;
    return l;
}

// The walks count the vertices they pass per level in 7-bit fields of one
// word (a walk passes at most kWalkCap + 1 < 128 vertices in one kernel) and
// turn the counts into the 128-bit weight once at the end.
static_assert(kWalkCap + 1 < 128 && 7 * kMaxLevels <= 64, "per-level walk counts must fit 7-bit fields");
__device__ inline uint64_t count_one(const Levels& L, int32_t v) { return 1ull << (7 * level_of(L, v)); }

__device__ inline i128 weight_of_counts(const Levels& L, uint64_t c) {
    i128 w = 0;
#pragma unroll
    for (int l = 0; l < kMaxLevels; ++l) {
        if (l >= L.n) break;
        const i128 d = (i128)((c >> (7 * l)) & 127u) << L.shift[l];
        w += ((L.odd_mask >> l) & 1u) ? -d : d;
    }
    return w;
}

__device__ inline i128 weight_of(const Levels& L, int32_t v) {
    const int l = level_of(L, v);
    const i128 w = (i128)1 << L.shift[l];
    return ((L.odd_mask >> l) & 1u) ? -w : w;
}

inline unsigned grid_n(int64_t n) {
    int64_t b = (n + kBlock - 1) / kBlock;
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(b, 152 * 64));
}

inline unsigned grid_ilp(int64_t n) {
    int64_t tiles = (n + 32 * kIlpCv - 1) / (32 * kIlpCv);
    int64_t b = (tiles + kBlock / 32 - 1) / (kBlock / 32);
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(b, 152 * 64));
}

__device__ inline uint32_t g32_word(uint64_t w) {
    return (gd_none(w) ? 0x80000000u : 0u) | (gd_sink(w) ? 0x40000000u : 0u) | (uint32_t)gd_ptr(w);
}
__device__ inline bool w32_none(uint32_t w) { return (w & 0x80000000u) != 0; }
__device__ inline bool w32_sink(uint32_t w) { return (w & 0x40000000u) != 0; }
__device__ inline int32_t w32_ptr(uint32_t w) { return (int32_t)(w & 0x3fffffffu); }

__device__ inline void block_add32(int32_t v, int32_t* counter) {
    __shared__ int32_t acc;
    if (threadIdx.x == 0) acc = 0;
    __syncthreads();
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(kFullMask, v, o);
    if ((threadIdx.x & 31) == 0 && v) atomicAdd(&acc, v);
    __syncthreads();
    if (threadIdx.x == 0 && acc) atomicAdd(counter, acc);
}

// Bounded software grid barrier (all blocks co-resident in a cooperative
// launch); records kErrBarrier and returns false when it gives up.
__device__ bool grid_sync_cv(Counters* c) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        ok = 1;
        volatile uint32_t* genp = &c->bar_gen;
        const uint32_t gen = *genp;
        __threadfence();
        const uint32_t arrived = atomicAdd(&c->bar_count, 1u);
        if (arrived == gridDim.x - 1) {
            atomicExch(&c->bar_count, 0u);
            __threadfence();
            atomicAdd(&c->bar_gen, 1u);
        } else {
            int64_t spins = 0;
            while (*genp == gen) {
                if (++spins > (1ll << 24)) {
                    atomicOr(&c->err, kErrBarrier);
                    ok = 0;
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
    }
    __syncthreads();
    return ok != 0;
}

// Nearest greater vertex by a direct walk, summing the weights of the
// vertices passed (v included, g(v) not). Both buffers get the result. As in
// the distinct-priority walk, the first pass takes at most kWalkShort steps
// and the walks still below their start continue densely in k_walk_more_cv
// up to kWalkCap steps; those still pending join the pointer-jumping list.
__device__ inline uint64_t cv_word(int32_t v, int32_t x, uint32_t d, int32_t sink0, bool* pend) {
    *pend = false;
    if (x > v) return gd_pack(true, false, d, x, x == sink0);
    if (x == v) return gd_pack(true, true, d, v);
    *pend = true;
    return gd_pack(false, false, d, x);
}

__global__ void __launch_bounds__(kBlock) k_walk_cv(int32_t n, Levels L, const int32_t* __restrict__ strat,
                                                    const uint8_t* __restrict__ flags, int32_t sink0,
                                                    uint64_t* __restrict__ gd, uint64_t* __restrict__ gdB,
                                                    uint32_t* __restrict__ gd32, i128* __restrict__ ws,
                                                    i128* __restrict__ wsB, int32_t* __restrict__ more,
                                                    Counters* cnt) {
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t tile = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; tile * 32 * kIlpCv < n;
         tile += nwarps) {
        int32_t v[kIlpCv], x[kIlpCv];
        uint32_t d[kIlpCv];
        uint64_t acc[kIlpCv];  // per-level counts of the vertices passed
        bool act[kIlpCv], slotid[kIlpCv];
#pragma unroll
        for (int j = 0; j < kIlpCv; ++j) {
            v[j] = (int32_t)(tile * 32 * kIlpCv + lane + 32 * j);
            const int32_t xr = v[j] < n ? __ldg(strat + v[j]) : INT32_MAX;  // loaded with the flags, not after
            slotid[j] = v[j] < n && (flags[v[j]] & kSinkSlot);
            x[j] = slotid[j] ? INT32_MAX : xr;
            d[j] = 1;
            acc[j] = (v[j] < n && !slotid[j]) ? count_one(L, v[j]) : 0;
            act[j] = v[j] < n && !slotid[j] && x[j] < v[j];
        }
        for (;;) {
            bool any = false;
            int32_t nx[kIlpCv];
#pragma unroll
            for (int j = 0; j < kIlpCv; ++j) {
                if (act[j] && d[j] >= (uint32_t)kWalkShort) act[j] = false;  // pending at x (not summed)
                nx[j] = act[j] ? __ldg(strat + x[j]) : x[j];
            }
#pragma unroll
            for (int j = 0; j < kIlpCv; ++j) {
                if (act[j]) {
                    acc[j] += count_one(L, x[j]);
                    x[j] = nx[j];
                    ++d[j];
                    act[j] = x[j] < v[j];
                }
                any |= act[j];
            }
            if (!any) break;
        }
#pragma unroll
        for (int j = 0; j < kIlpCv; ++j) {
            bool pend = false;
            if (v[j] < n) {
                const uint64_t w = slotid[j] ? gd_pack(true, false, 0, v[j], true) : cv_word(v[j], x[j], d[j], sink0, &pend);
                gd[v[j]] = w;
                gdB[v[j]] = w;
                gd32[v[j]] = g32_word(w);
                const i128 wt = weight_of_counts(L, acc[j]);
                ws[v[j]] = wt;
                wsB[v[j]] = wt;
            }
            const unsigned m = __ballot_sync(kFullMask, pend);
            if (m) {
                const int leader = __ffs(m) - 1;
                int32_t base = 0;
                if (lane == leader) base = atomicAdd(&cnt->n_walk2, __popc(m));
                base = __shfl_sync(kFullMask, base, leader);
                if (pend) more[base + __popc(m & ((1u << lane) - 1u))] = v[j];
            }
        }
    }
}

// Second walk pass over the list left by k_walk_cv, kIlpCv walks per thread.
__global__ void __launch_bounds__(kBlock) k_walk_more_cv(Levels L, const int32_t* __restrict__ more,
                                                         const int32_t* __restrict__ strat, int32_t sink0,
                                                         uint64_t* __restrict__ gd, uint64_t* __restrict__ gdB,
                                                         uint32_t* __restrict__ gd32, i128* __restrict__ ws,
                                                         i128* __restrict__ wsB, int32_t* __restrict__ plist,
                                                         Counters* cnt) {
    const int32_t cntm = cnt->n_walk2;
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t tile = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; tile * 32 * kIlpCv < cntm;
         tile += nwarps) {
        int32_t v[kIlpCv], x[kIlpCv];
        uint32_t d[kIlpCv];
        i128 acc[kIlpCv];
        uint64_t lc[kIlpCv];  // per-level counts of the vertices passed in this kernel
        bool act[kIlpCv], in[kIlpCv];
#pragma unroll
        for (int j = 0; j < kIlpCv; ++j) {
            const int64_t i = tile * 32 * kIlpCv + lane + 32 * j;
            in[j] = i < cntm;
            v[j] = in[j] ? more[i] : 0;
            const uint64_t w = in[j] ? gd[v[j]] : 0;
            x[j] = gd_ptr(w);
            d[j] = gd_dist(w);
            acc[j] = in[j] ? ws[v[j]] : 0;
            lc[j] = 0;
            act[j] = in[j] && x[j] < v[j];
        }
        for (;;) {
            bool any = false;
            int32_t nx[kIlpCv];
#pragma unroll
            for (int j = 0; j < kIlpCv; ++j) {
                if (act[j] && d[j] >= (uint32_t)kWalkCap) act[j] = false;
                nx[j] = act[j] ? __ldg(strat + x[j]) : x[j];
            }
#pragma unroll
            for (int j = 0; j < kIlpCv; ++j) {
                if (act[j]) {
                    lc[j] += count_one(L, x[j]);
                    x[j] = nx[j];
                    ++d[j];
                    act[j] = x[j] < v[j];
                }
                any |= act[j];
            }
            if (!any) break;
        }
#pragma unroll
        for (int j = 0; j < kIlpCv; ++j) {
            bool pend = false;
            if (in[j]) {
                const uint64_t w = cv_word(v[j], x[j], d[j], sink0, &pend);
                gd[v[j]] = w;
                gdB[v[j]] = w;
                gd32[v[j]] = g32_word(w);
                const i128 wt = acc[j] + weight_of_counts(L, lc[j]);
                ws[v[j]] = wt;
                wsB[v[j]] = wt;
            }
            const unsigned m = __ballot_sync(kFullMask, pend);
            if (m) {
                const int leader = __ffs(m) - 1;
                int32_t base = 0;
                if (lane == leader) base = atomicAdd(&cnt->n_pending, __popc(m));
                base = __shfl_sync(kFullMask, base, leader);
                if (pend) plist[base + __popc(m & ((1u << lane) - 1u))] = v[j];
            }
        }
    }
}

// Pointer jumping with weights, all rounds in one cooperative launch. Round r
// reads buffer r % 2 and writes the other for every pending-list vertex
// (copying finished ones forward), so a vertex's word and weight are always
// read from the same round. The final values end in the first buffer.
__global__ void __launch_bounds__(kBlock) k_jump_cv_coop(const int32_t* __restrict__ plist, uint64_t* gd,
                                                         uint64_t* gdB, i128* ws, i128* wsB, uint32_t* gd32,
                                                         int32_t sink0, Counters* cnt, int32_t cap) {
    const int32_t np = cnt->n_pending;
    if (np == 0) return;
    for (int32_t r = 0;; ++r) {
        uint64_t* sg = (r & 1) ? gdB : gd;
        uint64_t* dg = (r & 1) ? gd : gdB;
        i128* sw = (r & 1) ? wsB : ws;
        i128* dw = (r & 1) ? ws : wsB;
        if (blockIdx.x == 0 && threadIdx.x == 0) cnt->left[(r + 1) % 3] = 0;
        int32_t left = 0;
        for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < np; i += gridDim.x * blockDim.x) {
            const int32_t v = plist[i];
            const uint64_t w = __ldcg((const unsigned long long*)(sg + v));
            const i128 a = sw[v];
            if (gd_resolved(w)) {
                dg[v] = w;
                dw[v] = a;
                continue;
            }
            int32_t x = gd_ptr(w);
            uint64_t wx = __ldcg((const unsigned long long*)(sg + x));
            i128 ax = sw[x];
            i128 acc = a;
            uint64_t pre = gd_dist(w);
            // through up to kJumpFollow resolved vertices below v at once (their segments rise to g(x) < v)
            for (int f = 0; f < kJumpFollow && gd_resolved(wx) && !gd_none(wx) && gd_ptr(wx) < v; ++f) {
                acc += ax;
                pre += gd_dist(wx);
                x = gd_ptr(wx);
                wx = __ldcg((const unsigned long long*)(sg + x));
                ax = sw[x];
            }
            uint64_t nw;
            if (gd_resolved(wx) && gd_none(wx)) {
                nw = gd_pack(true, true, 0, gd_ptr(wx));  // v is above its whole future, in a top basin
            } else {
                const int32_t y = gd_ptr(wx);
                uint64_t nd = pre + gd_dist(wx);
                if (nd > kDistMax) nd = kDistMax;
                if (y > v) nw = gd_pack(true, false, (uint32_t)nd, y, y == sink0);
                else if (y == v) nw = gd_pack(true, true, (uint32_t)nd, v);
                else {
                    nw = gd_pack(false, false, (uint32_t)nd, y);
                    ++left;
                }
            }
            dg[v] = nw;
            dw[v] = acc + ax;
            if (gd_resolved(nw)) gd32[v] = g32_word(nw);
        }
        block_add32(left, &cnt->left[r % 3]);
        if (!grid_sync_cv(cnt)) return;
        const int32_t rem = *(volatile int32_t*)&cnt->left[r % 3];
        if (rem == 0 || r + 1 >= cap) {
            if (rem != 0 && blockIdx.x == 0 && threadIdx.x == 0) atomicOr(&cnt->err, kErrJumpRounds);
            if (blockIdx.x == 0 && threadIdx.x == 0) cnt->jump_rounds = r + 1;
            if (!(r & 1)) {  // this round wrote the second buffer: bring the results back
                for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < np; i += gridDim.x * blockDim.x) {
                    const int32_t v = plist[i];
                    gd[v] = gdB[v];
                    ws[v] = wsB[v];
                }
            }
            return;
        }
    }
}

// Classification and keys: each vertex sums the segment weights along its
// g-chain to the sink (finite) or meets a vertex above its whole future
// (top; the cycle's largest priority is that vertex's maximum's).
__global__ void __launch_bounds__(kBlock) k_chain_cv(int32_t n, const uint32_t* __restrict__ gd32,
                                                     const i128* __restrict__ ws, const uint8_t* __restrict__ flags,
                                                     const int32_t* __restrict__ pri, i128* __restrict__ key,
                                                     uint8_t* __restrict__ kind, uint8_t* __restrict__ cls,
                                                     int32_t* __restrict__ dom, int want_dom, GameState* gst,
                                                     Counters* cnt) {
    if (cnt->err) return;  // unfinished jumping: g-words may point downwards, so no chain walk would end
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    int32_t nfin = 0, nodd = 0;
    for (int64_t tile = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; tile * 32 * kIlpCv < n;
         tile += nwarps) {
        int32_t v[kIlpCv], x[kIlpCv], cyc[kIlpCv];
        i128 acc[kIlpCv];
        bool act[kIlpCv], slotid[kIlpCv];
#pragma unroll
        for (int j = 0; j < kIlpCv; ++j) {
            v[j] = (int32_t)(tile * 32 * kIlpCv + lane + 32 * j);
            const uint32_t wr = v[j] < n ? gd32[v[j]] : 0x40000000u;  // loaded with the flags, not after them
            slotid[j] = v[j] < n && (flags[v[j]] & kSinkSlot);
            const uint32_t w = slotid[j] ? 0x40000000u : wr;
            cyc[j] = w32_none(w) ? w32_ptr(w) : -1;
            acc[j] = (v[j] < n && !slotid[j] && cyc[j] < 0) ? ws[v[j]] : 0;
            x[j] = w32_ptr(w);
            act[j] = v[j] < n && !slotid[j] && !w32_none(w) && !w32_sink(w);
        }
        for (;;) {
            bool any = false;
            uint32_t wx[kIlpCv];
            i128 ax[kIlpCv];
#pragma unroll
            for (int j = 0; j < kIlpCv; ++j) {
                wx[j] = act[j] ? gd32[x[j]] : 0u;
                ax[j] = act[j] ? ws[x[j]] : 0;
            }
#pragma unroll
            for (int j = 0; j < kIlpCv; ++j) {
                if (act[j]) {
                    if (w32_none(wx[j])) {
                        cyc[j] = w32_ptr(wx[j]);
                        act[j] = false;
                    } else {
                        acc[j] += ax[j];
                        x[j] = w32_ptr(wx[j]);
                        act[j] = !w32_sink(wx[j]);
                    }
                }
                any |= act[j];
            }
            if (!any) break;
        }
#pragma unroll
        for (int j = 0; j < kIlpCv; ++j) {
            if (v[j] >= n) continue;
            if (slotid[j]) {
                key[v[j]] = 0;  // the sink: the empty valuation
                kind[v[j]] = 8;
                cls[v[j]] = kFin;
                if (want_dom) dom[v[j]] = -1;
            } else if (cyc[j] < 0) {
                key[v[j]] = acc[j];
                kind[v[j]] = 1;  // finite (read by the depth pass)
                cls[v[j]] = kFin;
                if (want_dom) dom[v[j]] = -1;
                ++nfin;
            } else {
                const bool odd = (flags[cyc[j]] & kPriOdd) != 0;
                key[v[j]] = top_key();
                kind[v[j]] = 0;
                cls[v[j]] = odd ? kOddCycle : kTop;
                if (want_dom) dom[v[j]] = pri[cyc[j]];
                if (odd) {
                    ++nodd;
                    atomicAdd(&gst[0].nodd, 1);
                }
            }
        }
    }
    block_add32(nfin, &cnt->n_fin);
    block_add32(nodd, &cnt->n_odd);
}

// The switching rules on keys (first minimiser for Odd; the sink first, then
// the first maximiser for Even; strictly better only), one thread per vertex.
template <typename OffT>
__global__ void __launch_bounds__(kBlock) k_switch_cv(int32_t n, int player, const OffT* __restrict__ off,
                                                      const int32_t* __restrict__ tgt,
                                                      const uint8_t* __restrict__ flags, const i128* __restrict__ key,
                                                      int32_t sink0, GameState* gst, int32_t* strat, Counters* cnt) {
    {
        const GameState st = gst[0];
        if (st.phase != kPhaseActive || (player == 0 && st.sw_odd != 0)) return;
    }
    int32_t nsw = 0;
    for (int32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        const uint8_t f = flags[v];
        if ((f & kSinkSlot) || (int)(f & kOwnerOdd) != player) continue;
        const int64_t e0 = off[v], e1 = off[v + 1];
        const int32_t cur = strat[v];
        int32_t best = player == 0 ? sink0 : -1;
        i128 bk = player == 0 ? key[sink0] : 0;
        const i128 curkey = key[cur];
        for (int64_t e = e0; e < e1; e += 4) {
            int32_t t[4];
            i128 kk[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) t[j] = e + j < e1 ? tgt[e + j] : -1;
#pragma unroll
            for (int j = 0; j < 4; ++j) kk[j] = t[j] >= 0 ? key[t[j]] : 0;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                if (t[j] < 0) continue;
                const bool better = player == 0 ? kk[j] > bk : (best < 0 || kk[j] < bk);
                if (better) {
                    best = t[j];
                    bk = kk[j];
                }
            }
        }
        if (player == 0 ? bk > curkey : bk < curkey) {
            strat[v] = best;
            ++nsw;
        }
    }
    block_add32(nsw, &cnt->n_switch);
    __shared__ int32_t tot;
    if (threadIdx.x == 0) tot = 0;
    __syncthreads();
    int32_t x = nsw;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(kFullMask, x, o);
    if ((threadIdx.x & 31) == 0 && x) atomicAdd(&tot, x);
    __syncthreads();
    if (threadIdx.x == 0 && tot) atomicAdd(player ? &gst[0].sw_odd : &gst[0].sw_even, tot);
}

// Count vectors of the original vertices (rows of nlev), decoded from the
// keys: balanced digits (level l's of width L.shift[l+1] - L.shift[l]), each the signed count of its level.
__global__ void k_counts(int64_t n0, const int32_t* __restrict__ nid0, const i128* __restrict__ key,
                         const uint8_t* __restrict__ cls, Levels L, int32_t* __restrict__ out) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n0; v += (int64_t)gridDim.x * blockDim.x) {
        const int32_t i = nid0[v];
        const bool fin = cls[i] == kFin;
        i128 k = fin ? key[i] : 0;
        for (int l = 0; l < L.n; ++l) {
            // the lowest digit in (-2^(b-1), 2^(b-1)): low b bits, taken negative from 2^(b-1) up
            const int b = L.shift[l + 1] - L.shift[l];
            int64_t a = (int64_t)(k & (i128)((1ll << b) - 1));
            if (a >= (1ll << (b - 1))) a -= 1ll << b;
            k = (k - (i128)a) >> b;  // exact: k - a is a multiple of 2^b
            out[v * L.n + l] = (int32_t)(((L.odd_mask >> l) & 1u) ? -a : a);
        }
    }
}

// Bellman-Ford (Section 4, "Computing Best Responses": a best response is a
// shortest path to the sink under the order of Section 3; odd priorities are
// negative weights, and an admissible sigma leaves Odd no negative cycle).
// One Jacobi round: every vertex takes its weight plus the best key of its
// successors under the previous round's keys (Odd: the least over its edges;
// Even: the one sigma names); an unreached vertex stays top.
template <typename OffT>
__global__ void __launch_bounds__(kBlock) k_bf_round(int32_t n, Levels L, const OffT* __restrict__ off,
                                                     const int32_t* __restrict__ tgt,
                                                     const uint8_t* __restrict__ flags,
                                                     const int32_t* __restrict__ strat, const i128* __restrict__ src,
                                                     i128* __restrict__ dst, int32_t* changed) {
    int32_t ch = 0;
    const i128 top = top_key();
    for (int32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        const uint8_t f = flags[v];
        if (f & kSinkSlot) {
            dst[v] = 0;
            continue;
        }
        i128 best = top;
        if (f & kOwnerOdd) {
            for (OffT e = off[v]; e < off[v + 1]; ++e) {
                const i128 k = src[tgt[e]];
                if (k < best) best = k;
            }
        } else {
            best = src[strat[v]];
        }
        const i128 nk = best == top ? top : weight_of(L, v) + best;
        ch += nk != src[v];
        dst[v] = nk;
    }
    block_add32(ch, changed);
}

__global__ void k_bf_init(int32_t n, const uint8_t* __restrict__ flags, i128* __restrict__ key) {
    for (int32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
        key[v] = (flags[v] & kSinkSlot) ? (i128)0 : top_key();
}

// Odd's strategy from the final keys: the first edge of least key.
template <typename OffT>
__global__ void k_bf_argmin(int32_t n, const OffT* __restrict__ off, const int32_t* __restrict__ tgt,
                            const uint8_t* __restrict__ flags, const i128* __restrict__ key, int32_t* strat) {
    for (int32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        const uint8_t f = flags[v];
        if ((f & kSinkSlot) || !(f & kOwnerOdd)) continue;
        int32_t best = -1;
        i128 bk = 0;
        for (OffT e = off[v]; e < off[v + 1]; ++e) {
            const i128 k = key[tgt[e]];
            if (best < 0 || k < bk) {
                best = tgt[e];
                bk = k;
            }
        }
        strat[v] = best;
    }
}

}  // namespace

// Bellman-Ford best response on g->strat's sigma: rounds until no key
// changes (checked every kCheck rounds), at most n + 2 rounds (more would
// mean a negative cycle: sigma not admissible). Leaves Odd's choice in
// g->strat; *rounds gets the rounds run.
pg_status bellman_ford_cv(pg_game* g, int64_t* rounds) {
    pg_ctx* ctx = g->ctx;
    cudaStream_t s = ctx->stream;
    const int32_t n = g->n;
    constexpr int kCheck = 8;
    int32_t* changed = nullptr;
    PG_CUDA_TRY(ctx, cudaMallocAsync((void**)&changed, sizeof(int32_t) * kCheck, s));
    int32_t hchg[kCheck];
    i128* buf[2] = {g->ws, g->wsB};
    ctx->launches += 1;
    k_bf_init<<<grid_n(n), kBlock, 0, s>>>(n, g->flags, buf[0]);
    int64_t r = 0;
    pg_status st = PG_OK;
    for (;;) {
        cudaError_t e = cudaMemsetAsync(changed, 0, sizeof(int32_t) * kCheck, s);
        for (int i = 0; i < kCheck && e == cudaSuccess; ++i, ++r) {
            ctx->launches += 1;
            k_bf_round<int32_t><<<grid_n(n), kBlock, 0, s>>>(n, g->lev, g->off, g->tgt, g->flags, g->strat,
                                                             buf[r & 1], buf[(r + 1) & 1], changed + i);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaMemcpyAsync(hchg, changed, sizeof(hchg), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) {
            st = cuda_fail(ctx, e, "bellman_ford_cv");
            break;
        }
        if (hchg[kCheck - 1] == 0) break;
        if (r > (int64_t)n + 2) {
            st = fail(ctx, PG_ENOTADMISSIBLE, "Bellman-Ford: keys still decrease (a negative cycle: sigma is not admissible)");
            break;
        }
    }
    if (st == PG_OK) {
        // the keys of the last round are in buf[r & 1]
        ctx->launches += 1;
        k_bf_argmin<int32_t><<<grid_n(n), kBlock, 0, s>>>(n, g->off, g->tgt, g->flags, buf[r & 1], g->strat);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) st = cuda_fail(ctx, e, "k_bf_argmin");
    }
    cudaFreeAsync(changed, s);
    *rounds = r;
    return st;
}

pg_status alloc_cv(pg_game* g) {
    pg_ctx* ctx = g->ctx;
    const int64_t n = g->n;
    cudaStream_t s = ctx->stream;
    PG_CUDA_TRY(ctx, dev_alloc(ctx, (void**)&g->ws, sizeof(i128) * n, s));
    PG_CUDA_TRY(ctx, dev_alloc(ctx, (void**)&g->wsB, sizeof(i128) * n, s));
    PG_CUDA_TRY(ctx, dev_alloc(ctx, (void**)&g->gdB, sizeof(uint64_t) * n, s));
    PG_CUDA_TRY(ctx, dev_alloc(ctx, (void**)&g->key128, sizeof(i128) * n, s));
    return PG_OK;
}

pg_status enqueue_valuation_cv(pg_game* g, bool want_dom) {
    pg_ctx* ctx = g->ctx;
    cudaStream_t s = ctx->stream;
    const int32_t n = g->n;
    Counters* c = g->cnt;
    PG_CUDA_TRY(ctx, cudaMemsetAsync(c, 0, sizeof(Counters), s));
    prof_begin(g, KID_WALK);
    k_walk_cv<<<grid_ilp(n), kBlock, 0, s>>>(n, g->lev, g->strat, g->flags, g->sink0, g->gd, g->gdB, g->gd32, g->ws,
                                             g->wsB, g->hugelist, c);
    k_walk_more_cv<<<g->coop_blocks, kBlock, 0, s>>>(g->lev, g->hugelist, g->strat, g->sink0, g->gd, g->gdB, g->gd32,
                                                     g->ws, g->wsB, g->plist, c);
    prof_end(g, KID_WALK, 2);
    {
        int32_t cap = 64;
        for (int64_t x = n; x > 1; x >>= 1) cap += 2;
        void* args[] = {(void*)&g->plist, (void*)&g->gd,    (void*)&g->gdB, (void*)&g->ws, (void*)&g->wsB,
                        (void*)&g->gd32,  (void*)&g->sink0, (void*)&c,      (void*)&cap};
        prof_begin(g, KID_JUMP);
        PG_CUDA_TRY(ctx, cudaLaunchCooperativeKernel((void*)k_jump_cv_coop, g->coop_blocks, kBlock, args, 0, s));
        prof_end(g, KID_JUMP, 1);
    }
    prof_begin(g, KID_CHAIN2);
    k_chain_cv<<<grid_ilp(n), kBlock, 0, s>>>(n, g->gd32, g->ws, g->flags, g->pri, g->key128, g->kind, g->cls,
                                              g->dom, want_dom ? 1 : 0, g->gst, c);
    prof_end(g, KID_CHAIN2, 1);
    PG_CUDA_TRY(ctx, cudaGetLastError());
    return PG_OK;
}

pg_status enqueue_switch_cv(pg_game* g, int player) {
    pg_ctx* ctx = g->ctx;
    cudaStream_t s = ctx->stream;
    PG_CUDA_TRY(ctx, cudaMemsetAsync(&g->cnt->n_switch, 0, sizeof(int32_t), s));
    const int kid = player ? KID_SWITCH_ODD : KID_SWITCH_EVEN;
    prof_begin(g, kid);
    k_switch_cv<int32_t><<<grid_n(g->n), kBlock, 0, s>>>(g->n, player, g->off, g->tgt, g->flags, g->key128, g->sink0,
                                                        g->gst, g->strat, g->cnt);
    prof_end(g, kid, 1);
    PG_CUDA_TRY(ctx, cudaGetLastError());
    return PG_OK;
}

pg_status write_counts(pg_game* g, int32_t mem_kind, int32_t* counts) {
    pg_ctx* ctx = g->ctx;
    cudaStream_t s = ctx->stream;
    const size_t bytes = sizeof(int32_t) * (size_t)g->n0 * (size_t)g->lev.n;
    int32_t* dst = counts;
    if (mem_kind == PG_MEM_HOST) PG_CUDA_TRY(ctx, cudaMallocAsync((void**)&dst, bytes ? bytes : 4, s));
    ctx->launches += 1;
    k_counts<<<grid_n(g->n0), kBlock, 0, s>>>(g->n0, g->nid0, g->key128, g->cls, g->lev, dst);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && mem_kind == PG_MEM_HOST)
        e = cudaMemcpyAsync(counts, dst, bytes, cudaMemcpyDeviceToHost, s);
    if (mem_kind == PG_MEM_HOST) cudaFreeAsync(dst, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "write_counts");
    return PG_OK;
}

}  // namespace pg
