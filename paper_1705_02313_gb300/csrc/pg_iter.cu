// One valuation (K1 + K2) and one switching pass (K3) of strategy improvement.
//
// Valuation (Section 3, "Valuations"; Section 5, the pseudoforest of a profile).
// Under a profile every vertex has one successor strat[v] (the sink is id n).
// Vertex ids are priority ranks, so with distinct priorities a finite
// valuation is the set of vertices on the play to the sink, and the order of
// Section 3 compares two such sets by the largest vertex in their symmetric
// difference: it decides for the side holding it when its priority is even,
// against it when odd. This build computes the exact position of every
// finite valuation in that order through the nearest-greater-ancestor
// forest: g(v) is the first vertex after v on its play with a larger id (the
// sink counts as larger than all). Two finite plays first differ below their
// lowest common g-ancestor, and there the larger of the two differing g-chain
// members decides, so the order is the in-order of the g-forest in which the
// children of a node are ordered odd-priority first (larger id first), then the
// node itself, then even-priority children (smaller id first). That in-order is
//   rank(v) = oddsz(v) + sum over c on v's g-chain below the sink of wgt(c),
//   wgt(c)  = [pri(c) even] + total size of the siblings ordered before c,
// with sizes of g-subtrees. Infinite plays (TOP) end in a cycle; the cycle's
// largest vertex is the only vertex whose walk returns to itself, which gives
// the dominant priority of the cycle (Section 5, "Modifications to the
// Helman-JaJa algorithm": pseudotree vertices are TOP; an odd dominant
// priority means sigma was not admissible).
//
// Passes of one valuation (no host synchronisation between them):
//   k_walk        nearest greater vertex by a direct walk of <= kWalkCap steps
//   k_jump_coop   pointer jumping over smaller vertices for the rest
//   k_chain1      classification, g-subtree sizes and children counts
//   scan          children counts -> contiguous child segments
//   k_scatter     children into their segments; the sink's children marked
//   k_siblings    sibling weights inside each segment (k_big_parents for
//                 large segments)
//   sink scan     id-ordered scan for the children of each game's sink
//   k_idscan_coop the same scan for parents with > kHugeChildren children
//   k_chain2      rank and class by summing weights along each g-chain
// The pointer-chasing passes give every thread several independent chains so
// that several gathers are in flight per thread.
//
// Switching (Section 3, "Switching rules"; Section 4, All_Odd): one thread
// per vertex of the switching player, edges in batches of four gathers, first
// minimiser for Odd, the sink first and then the first maximiser for Even; a
// vertex switches only when strictly better.
#include <cooperative_groups.h>
#include <string.h>

#include "pg_device.cuh"

// Vertices per thread of the loop's two chain passes (k_walk_cmp, k_classify).
#ifndef PG_CHAIN_ILP
#define PG_CHAIN_ILP 4
#endif

namespace cg = cooperative_groups;

namespace pg {
namespace {

// K1: nearest greater vertex along the play, by a direct walk of at most
// cap steps; the walks still below their start are appended to a list (the
// pointer-jumping list). A walk that returns to its start found the maximum
// of its cycle; a walk that runs out of steps leaves a jump pointer for
// k_jump_coop.
__device__ inline uint64_t walk_word(int32_t v, int32_t x, uint32_t d, const int32_t* vgame, const int32_t* gsink,
                                     int32_t sink0, bool* pend) {
    *pend = false;
    if (x > v) return gd_pack(true, false, d, x, x == sink_of(v, vgame, gsink, sink0));  // a larger vertex or the sink
    if (x == v) return gd_pack(true, true, d, v);                                        // v is its cycle's maximum
    *pend = true;
    return gd_pack(false, false, d, x);
}

template <uint32_t cap>
__global__ void __launch_bounds__(kBlock) k_walk(int32_t n, const int32_t* __restrict__ strat,
                                                 const uint8_t* __restrict__ flags, const int32_t* __restrict__ vgame,
                                                 const int32_t* __restrict__ gsink, int32_t sink0,
                                                 uint64_t* __restrict__ gd, uint32_t* __restrict__ gd32,
                                                 int32_t* __restrict__ more, int32_t* __restrict__ sz,
                                                 int32_t* __restrict__ oddsz, Counters* cnt, int32_t* more_count) {
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t tile = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; warp_tile_base(tile) < n;
         tile += nwarps) {
        int32_t v[kIlp], x[kIlp];
        uint32_t d[kIlp];
        bool act[kIlp], slotid[kIlp];
#pragma unroll
        for (int j = 0; j < kIlp; ++j) {
            v[j] = (int32_t)(warp_tile_base(tile) + lane + 32 * j);
            const int32_t xr = v[j] < n ? __ldg(strat + v[j]) : INT32_MAX;  // loaded with the flags, not after
            slotid[j] = v[j] < n && (flags[v[j]] & kSinkSlot);
            x[j] = slotid[j] ? INT32_MAX : xr;
            d[j] = 1;
        }
#pragma unroll
        for (int j = 0; j < kIlp; ++j) act[j] = v[j] < n && !slotid[j] && x[j] < v[j] && d[j] < cap;
        for (;;) {
            bool any = false;
            int32_t nx[kIlp];
#pragma unroll
            for (int j = 0; j < kIlp; ++j) nx[j] = act[j] ? __ldg(strat + x[j]) : x[j];
#pragma unroll
            for (int j = 0; j < kIlp; ++j) {
                if (act[j]) {
                    x[j] = nx[j];
                    ++d[j];
                    act[j] = x[j] < v[j] && d[j] < cap;
                }
                any |= act[j];
            }
            if (!any) break;
        }
#pragma unroll
        for (int j = 0; j < kIlp; ++j) {
            bool pend = false;
            if (v[j] < n) {
                const uint64_t w = slotid[j] ? gd_pack(true, false, 0, v[j], true)  // a sink slot: inert
                                             : walk_word(v[j], x[j], d[j], vgame, gsink, sink0, &pend);
                gd[v[j]] = w;
                gd32[v[j]] = g32_of(w);
                sz[v[j]] = 0;  // zeros for this valuation's size and odd-total accumulation
                oddsz[v[j]] = 0;
            }
            int32_t slot = warp_append(pend, more_count);
            if (pend) more[slot] = v[j];
        }
    }
}

// Pointer jumping over smaller vertices for the walks that ran out of steps,
// all rounds in one cooperative launch. Invariant of a pending word: every
// vertex strictly between v and ptr is below v, and ptr is below v. Jumping
// through x = ptr uses x's own pointer (x pending) or g(x) (x resolved): both
// skip only vertices below x < v. Rounds stop when none is left or after cap.
// Three rotating counters keep each round's count stable until every block
// has read it.
__global__ void __launch_bounds__(kBlock) k_jump_coop(const int32_t* __restrict__ plist, uint64_t* gd,
                                                      uint32_t* gd32, const int32_t* __restrict__ vgame,
                                                      const int32_t* __restrict__ gsink, int32_t sink0, Counters* cnt,
                                                      int32_t cap, int cap_deep) {
    const int32_t np = cnt->n_pending;
    if (np == 0) return;
    for (int32_t r = 0;; ++r) {
        if (blockIdx.x == 0 && threadIdx.x == 0) cnt->left[(r + 1) % 3] = 0;
        int32_t left = 0;
        for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < np; i += gridDim.x * blockDim.x) {
            int32_t v = plist[i];
            uint64_t w = ld_cg(gd + v);
            if (gd_resolved(w)) continue;
            int32_t x = gd_ptr(w);
            uint64_t wx = ld_cg(gd + x);
            uint64_t pre = gd_dist(w);  // walk length from v to x
            // through up to kJumpFollow resolved vertices below v at once: their g-chains rise, so a long
            // increasing run below v costs rounds / kJumpFollow instead of one round per vertex
            for (int f = 0; f < kJumpFollow && gd_resolved(wx) && !gd_none(wx) && gd_ptr(wx) < v; ++f) {
                pre += gd_dist(wx);
                x = gd_ptr(wx);
                wx = ld_cg(gd + x);
            }
            uint64_t nw;
            if (gd_resolved(wx) && gd_none(wx)) {
                // x is above its whole future and below v: so is v (same cycle)
                nw = gd_pack(true, true, 0, gd_ptr(wx));
            } else {
                int32_t y = gd_ptr(wx);
                uint64_t nd = pre + gd_dist(wx);
                if (nd > kDistMax) nd = kDistMax;  // only reachable around cycles, where dist is unused
                if (y > v) {
                    nw = gd_pack(true, false, (uint32_t)nd, y, y == sink_of(v, vgame, gsink, sink0));
                } else if (y == v) {
                    nw = gd_pack(true, true, (uint32_t)nd, v);
                } else {
                    nw = gd_pack(false, false, (uint32_t)nd, y);
                    ++left;
                }
            }
            st_cg(gd + v, nw);
            if (gd_resolved(nw)) gd32[v] = g32_of(nw);
        }
        block_add(left, &cnt->left[r % 3]);
        if (!grid_sync(cnt)) return;
        int32_t rem = *(volatile int32_t*)&cnt->left[r % 3];
        if (rem == 0) {
            if (blockIdx.x == 0 && threadIdx.x == 0) cnt->jump_rounds = r + 1;
            return;
        }
        if (r + 1 >= cap) {  // the ruling-set path retries with a larger cap, or the call fails
            if (blockIdx.x == 0 && threadIdx.x == 0) {
                if (cap_deep) cnt->deep = 1;
                else atomicOr(&cnt->err, kErrJumpRounds);
            }
            return;
        }
    }
}

// Compare-mode K1 (loop iterations that compare valuations): the same walks
// and jumps with 4-byte g-words only. A word with both the none and the sink
// bit set is pending: its low bits are a jump pointer (every vertex strictly
// between v and it on the play is below v, and so is the pointer). A word
// with only the sink bit (g(v) is the game's sink slot, which the word does
// not repeat) carries v's priority parity in bit 0, so that the vertex that
// ends a chain gives its top's parity with no further read.
constexpr uint32_t kG32Pend = kG32None | kG32Sink;
__device__ inline bool g32_pending(uint32_t w) { return (w & kG32Pend) == kG32Pend; }
__device__ inline uint32_t g32_sink_word(uint8_t fl) { return kG32Sink | ((fl & kPriOdd) ? 1u : 0u); }

// Packed games: a warp tile of consecutive ids inside one game that is no
// longer active is skipped by the loop's chain passes (its words are not read
// by any active game: plays stay inside their game, and the full valuation
// after the loop recomputes every game). Warp-uniform.
__device__ inline bool tile_idle(int64_t t0, int64_t t1, int32_t n, const int32_t* __restrict__ vgame,
                                 const GameState* __restrict__ gst) {
    if (!vgame) return false;
    const int32_t a = vgame[t0], b = vgame[(int32_t)(t1 < n ? t1 : n) - 1];
    return a == b && gst[a].phase != kPhaseActive;
}

template <uint32_t cap, int ILP = kIlp, bool BATCH = false>
__global__ void __launch_bounds__(kBlock, 2048 / kBlock) k_walk_cmp(int32_t n, const int32_t* __restrict__ strat,
                                                     const uint8_t* __restrict__ flags,
                                                     const int32_t* __restrict__ vgame,
                                                     const int32_t* __restrict__ gsink, int32_t sink0,
                                                     uint32_t* __restrict__ gd32, int32_t* __restrict__ more,
                                                     int32_t* more_count, const GameState* __restrict__ gst) {
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t tile = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; (tile * 32 * ILP) < n;
         tile += nwarps) {
        if (BATCH && tile_idle(tile * 32 * ILP, (tile + 1) * 32 * ILP, n, vgame, gst)) continue;
        int32_t v[ILP], x[ILP];
        uint32_t slots = 0, odd = 0, act = 0;  // bit j: slot j's id is a sink slot / has an odd priority / walks
#pragma unroll
        for (int j = 0; j < ILP; ++j) {
            v[j] = (int32_t)((tile * 32 * ILP) + lane + 32 * j);
            const uint8_t fv = v[j] < n ? flags[v[j]] : 0;
            if (fv & kSinkSlot) slots |= 1u << j;
            if (fv & kPriOdd) odd |= 1u << j;
            // read together with the flags (a sink slot's successor is itself, so its walk ends at once)
            x[j] = v[j] < n ? __ldg(strat + v[j]) : INT32_MAX;
            if (v[j] < n && !(fv & kSinkSlot) && x[j] < v[j]) act |= 1u << j;
        }
        // the walks start together, so a walk still going has read `steps` successors
        for (uint32_t steps = 1; act && steps < cap; ++steps) {
            int32_t nx[ILP];
#pragma unroll
            for (int j = 0; j < ILP; ++j) nx[j] = ((act >> j) & 1u) ? __ldg(strat + x[j]) : x[j];
#pragma unroll
            for (int j = 0; j < ILP; ++j) {
                if ((act >> j) & 1u) {
                    x[j] = nx[j];
                    if (x[j] >= v[j]) act &= ~(1u << j);
                }
            }
        }
#pragma unroll
        for (int j = 0; j < ILP; ++j) {
            bool pend = false;
            if (v[j] < n) {
                uint32_t w;
                if ((slots >> j) & 1u) w = kG32Sink;  // a sink slot: inert (its own top, even)
                else if (x[j] > v[j])
                    w = x[j] == (BATCH ? gsink[vgame[v[j]]] : sink0) ? kG32Sink | ((odd >> j) & 1u) : (uint32_t)x[j];
                else if (x[j] == v[j]) w = kG32None | (uint32_t)v[j];  // v is its cycle's maximum
                else {
                    w = kG32Pend | (uint32_t)x[j];
                    pend = true;
                }
                gd32[v[j]] = w;
            }
            int32_t slot = warp_append(pend, more_count);
            if (pend) more[slot] = v[j];
        }
    }
}

// Pointer jumping on the 4-byte words for the walks that ran out of steps,
// all rounds in one cooperative launch (as k_jump_coop, without walk lengths).
__global__ void __launch_bounds__(kBlock) k_jump32_coop(const int32_t* __restrict__ plist, uint32_t* gd32,
                                                        const uint8_t* __restrict__ flags,
                                                        const int32_t* __restrict__ vgame,
                                                        const int32_t* __restrict__ gsink, int32_t sink0,
                                                        Counters* cnt, int32_t cap, int cap_deep) {
    const int32_t np = cnt->n_pending;
    if (np == 0) return;
    for (int32_t r = 0;; ++r) {
        if (blockIdx.x == 0 && threadIdx.x == 0) cnt->left[(r + 1) % 3] = 0;
        int32_t left = 0;
        for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < np; i += gridDim.x * blockDim.x) {
            const int32_t v = plist[i];
            const uint32_t w = __ldcg(gd32 + v);
            if (!g32_pending(w)) continue;
            int32_t x = g32_ptr(w);
            uint32_t wx = __ldcg(gd32 + x);
            for (int f = 0; f < kJumpFollow && !(wx & kG32Pend) && g32_ptr(wx) < v; ++f) {  // resolved, rising
                x = g32_ptr(wx);
                wx = __ldcg(gd32 + x);
            }
            uint32_t nw;
            if (g32_none(wx) && !g32_pending(wx)) {
                // x is above its whole future and below v: so is v (same cycle)
                nw = kG32None | (uint32_t)g32_ptr(wx);
            } else {
                const int32_t sk = sink_of(v, vgame, gsink, sink0);
                const int32_t y = (g32_sink(wx) && !g32_pending(wx)) ? sk : g32_ptr(wx);
                if (y > v) nw = y == sk ? g32_sink_word(flags[v]) : (uint32_t)y;
                else if (y == v) nw = kG32None | (uint32_t)v;
                else {
                    nw = kG32Pend | (uint32_t)y;
                    ++left;
                }
            }
            __stcg(gd32 + v, nw);
        }
        block_add(left, &cnt->left[r % 3]);
        if (!grid_sync(cnt)) return;
        int32_t rem = *(volatile int32_t*)&cnt->left[r % 3];
        if (rem == 0) {
            if (blockIdx.x == 0 && threadIdx.x == 0) cnt->jump_rounds = r + 1;
            return;
        }
        if (r + 1 >= cap) {  // the iteration is abandoned and retried on the ruling-set path
            if (blockIdx.x == 0 && threadIdx.x == 0) {
                if (cap_deep) cnt->deep = 1;
                else atomicOr(&cnt->err, kErrJumpRounds);
            }
            return;
        }
    }
}

// Size additions near the roots of deep g-trees. Every vertex of a large
// g-tree has the same few vertices near the root among its ancestors, and one
// global atomic per vertex on each of them would serialise (an n-long chain: n
// additions on one word). Chains of at least kDeepChain vertices therefore add
// their top kHotTop ancestors into a per-block table in shared memory (open
// addressing, kHotProbes probes, then the global atomic), flushed once per
// block. Shorter chains (most vertices of random games) add directly: in the
// table they would only crowd out the hot entries. The launch bound keeps five
// blocks per SM.
constexpr int kHotSlots = 2048;
constexpr int kHotBits = 11;
constexpr int kHotProbes = 4;
constexpr int kHotTop = 8;
constexpr int kDeepChain = 4;

__device__ inline void hot_add(int32_t x, int32_t* tkey, int32_t* tcnt, int32_t* sz) {
    const uint32_t h = ((uint32_t)x * 2654435761u) >> (32 - kHotBits);
#pragma unroll
    for (int p = 0; p < kHotProbes; ++p) {
        const uint32_t i = (h + p) & (kHotSlots - 1);
        int32_t k = *(volatile int32_t*)&tkey[i];
        if (k == -1) k = atomicCAS(&tkey[i], -1, x);
        if (k == -1 || k == x) {
            atomicAdd(&tcnt[i], 1);
            return;
        }
    }
    atomicAdd(sz + x, 1);
}

// k_chain1 walks three chains per thread: it is bound by issuing its walk
// instructions, and a warp runs until the longest of its chains ends, so fewer
// chains per warp waste fewer issue slots (two, three, four, six: 287, 280,
// 290, 340 us per launch on the 10M game).
constexpr int kIlpChain1 = 3;

// Classification and g-subtree sizes. Each vertex walks its g-chain (4-byte
// words) to its end: the sink means a finite valuation, a "none" vertex
// means TOP (odd cycle if that cycle maximum is odd). Finite vertices then
// take a slot among their g-parent's children and add one to each g-ancestor
// below the sink (the top ones of deep chains through the block's table).
// TOP vertices touch nothing else, so large TOP components cause no atomic hot
// spots.
__global__ void __launch_bounds__(kBlock, 5) k_chain1(int32_t n, const uint32_t* __restrict__ gd32,
                                                   const uint8_t* __restrict__ flags, const int32_t* __restrict__ pri,
                                                   int32_t* sz, int32_t* ccnt, int32_t* __restrict__ slot,
                                                   uint8_t* __restrict__ kind, uint8_t* __restrict__ cls,
                                                   int32_t* __restrict__ dom, int want_dom,
                                                   const int32_t* __restrict__ vgame, GameState* gst, Counters* cnt,
                                                   int32_t deep_cut) {
    if (cnt->err || cnt->deep) return;  // unfinished jumping: g-words may point downwards, no chain walk would end
    __shared__ int32_t tkey[kHotSlots], tcnt[kHotSlots];
    for (int i = threadIdx.x; i < kHotSlots; i += blockDim.x) {
        tkey[i] = -1;
        tcnt[i] = 0;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    int32_t nfin = 0, nodd = 0;
    for (int64_t tile = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; (tile * 32 * kIlpChain1) < n;
         tile += nwarps) {
        int32_t v[kIlpChain1], g[kIlpChain1], x[kIlpChain1], cyc[kIlpChain1], len[kIlpChain1];
        bool act[kIlpChain1], sinkchild[kIlpChain1], slotid[kIlpChain1];
#pragma unroll
        for (int j = 0; j < kIlpChain1; ++j) {
            v[j] = (int32_t)((tile * 32 * kIlpChain1) + lane + 32 * j);
            const uint32_t wr = v[j] < n ? gd32[v[j]] : kG32Sink;  // loaded with the flags, not after them
            slotid[j] = v[j] < n && (flags[v[j]] & kSinkSlot);
            const uint32_t w = slotid[j] ? kG32Sink : wr;
            g[j] = g32_ptr(w);
            sinkchild[j] = g32_sink(w);
            cyc[j] = g32_none(w) ? g[j] : -1;
            x[j] = g[j];
            len[j] = 0;
            act[j] = v[j] < n && !slotid[j] && !g32_none(w) && !sinkchild[j];
        }
        // classification walks (len: the vertices from g(v) to the chain's end); a walk longer than deep_cut
        // hands the valuation to the ruling-set path and stops (its vertex takes no further part here)
        bool cut[kIlpChain1];
#pragma unroll
        for (int j = 0; j < kIlpChain1; ++j) cut[j] = false;
        for (;;) {
            bool any = false;
            uint32_t wx[kIlpChain1];
#pragma unroll
            for (int j = 0; j < kIlpChain1; ++j) wx[j] = act[j] ? gd32[x[j]] : 0u;
#pragma unroll
            for (int j = 0; j < kIlpChain1; ++j) {
                if (act[j] && len[j] >= deep_cut) {
                    cut[j] = true;
                    act[j] = false;
                    cnt->deep = 1;
                }
                if (act[j]) {
                    ++len[j];
                    if (g32_none(wx[j])) {
                        cyc[j] = g32_ptr(wx[j]);
                        act[j] = false;
                    } else {
                        x[j] = g32_ptr(wx[j]);
                        act[j] = !g32_sink(wx[j]);
                    }
                }
                any |= act[j];
            }
            if (!any) break;
        }
        // finite vertices below a vertex parent: slot, then sizes along the chain
        int32_t sl[kIlpChain1];
        bool deep[kIlpChain1];
#pragma unroll
        for (int j = 0; j < kIlpChain1; ++j) {
            act[j] = v[j] < n && !slotid[j] && cyc[j] < 0 && !sinkchild[j] && !cut[j];
            sl[j] = act[j] ? atomicAdd(ccnt + g[j], 1) : -1;
            x[j] = g[j];
            deep[j] = len[j] >= kDeepChain;
        }
        for (;;) {
            bool any = false;
            uint32_t wx[kIlpChain1];
#pragma unroll
            for (int j = 0; j < kIlpChain1; ++j) {
                if (act[j]) {  // len[j]: the additions still to come on this chain, this one included
                    if (deep[j] && len[j] <= kHotTop) hot_add(x[j], tkey, tcnt, sz);
                    else atomicAdd(sz + x[j], 1);
                    --len[j];
                }
                wx[j] = act[j] ? gd32[x[j]] : 0u;
            }
#pragma unroll
            for (int j = 0; j < kIlpChain1; ++j) {
                if (act[j]) {
                    x[j] = g32_ptr(wx[j]);
                    act[j] = !g32_sink(wx[j]);
                }
                any |= act[j];
            }
            if (!any) break;
        }
#pragma unroll
        for (int j = 0; j < kIlpChain1; ++j) {
            if (v[j] >= n) continue;
            if (slotid[j]) {
                kind[v[j]] = kKSinkSlot;
                cls[v[j]] = kFin;
                if (want_dom) dom[v[j]] = -1;
            } else if (cyc[j] < 0) {
                const bool odd_v = (flags[v[j]] & kPriOdd) != 0;
                kind[v[j]] = kKFin | (sinkchild[j] ? kKSinkChild : 0) | (odd_v ? kKOdd : 0);
                cls[v[j]] = kFin;
                if (want_dom) dom[v[j]] = -1;
                ++nfin;
            } else {
                const bool odd = (flags[cyc[j]] & kPriOdd) != 0;
                kind[v[j]] = 0;
                cls[v[j]] = odd ? kOddCycle : kTop;
                if (want_dom) dom[v[j]] = pri[cyc[j]];
                if (odd) {
                    ++nodd;
                    atomicAdd(&gst[vgame ? vgame[v[j]] : 0].nodd, 1);
                }
            }
            slot[v[j]] = sl[j];
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kHotSlots; i += blockDim.x)
        if (tcnt[i]) atomicAdd(sz + tkey[i], tcnt[i]);
    block_add(nfin, &cnt->n_fin);
    block_add(nodd, &cnt->n_odd);
}

__device__ inline int32_t order_key(int32_t c, bool odd) { return odd ? -(c + 1) : c; }

// Finite children into their segments at the slots taken in k_chain1
// (order key, subtree size); the sink's children record size and parity for
// the id-ordered scan. Also clears the children counts for the next valuation.
// kIlp vertices per thread, their parents' segment offsets gathered together.
static_assert(kCoopTile % (32 * kIlp) == 0, "k_scatter sums each warp tile into one scan tile");

__global__ void __launch_bounds__(kBlock) k_scatter(int32_t n, const uint32_t* __restrict__ gd32,
                                                    const uint8_t* __restrict__ kind, const int32_t* __restrict__ sz,
                                                    const int32_t* __restrict__ coff, const int32_t* __restrict__ slot,
                                                    int32_t* __restrict__ ccnt, int2* __restrict__ cl_ks,
                                                    int32_t* __restrict__ sinkval, int64_t* __restrict__ tsum,
                                                    const Counters* cnt) {
    if (cnt->deep) return;  // the ruling-set path takes over (and clears the children counts)
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t tile = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; warp_tile_base(tile) < n;
         tile += nwarps) {
        int32_t v[kIlp], base[kIlp], sl[kIlp], s[kIlp];
        uint8_t kd[kIlp];
        bool ent[kIlp];
#pragma unroll
        for (int j = 0; j < kIlp; ++j) {
            v[j] = (int32_t)(warp_tile_base(tile) + lane + 32 * j);
            kd[j] = v[j] < n ? kind[v[j]] : 0;
            ent[j] = (kd[j] & kKFin) && !(kd[j] & kKSinkChild);
            s[j] = (kd[j] & kKFin) ? 1 + sz[v[j]] : 0;
            sl[j] = ent[j] ? slot[v[j]] : 0;
            base[j] = ent[j] ? g32_ptr(gd32[v[j]]) : 0;
        }
#pragma unroll
        for (int j = 0; j < kIlp; ++j) base[j] = ent[j] ? coff[base[j]] : 0;
        int32_t se = 0, so = 0;  // sizes of the sink's children in this warp tile (disjoint subtrees: < 2^31)
#pragma unroll
        for (int j = 0; j < kIlp; ++j) {
            if (v[j] >= n) continue;
            const bool odd = (kd[j] & kKOdd) != 0;
            ccnt[v[j]] = 0;
            int32_t sv = 0;
            if ((kd[j] & kKFin) && (kd[j] & kKSinkChild)) {
                sv = s[j] | (odd ? INT32_MIN : 0);
                if (odd) so += s[j];
                else se += s[j];
            }
            if (ent[j]) cl_ks[base[j] + sl[j]] = make_int2(order_key(v[j], odd), s[j]);
            sinkval[v[j]] = sv;
        }
        // the tile sums of the id-ordered scan over the sink's children (a warp tile lies in one scan tile)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            se += __shfl_down_sync(kFull, se, o);
            so += __shfl_down_sync(kFull, so, o);
        }
        if (lane == 0) {
            const int64_t t = warp_tile_base(tile) / kCoopTile;
            if (se) atomicAdd((unsigned long long*)&tsum[2 * t], (unsigned long long)se);
            if (so) atomicAdd((unsigned long long*)&tsum[2 * t + 1], (unsigned long long)so);
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) ccnt[n] = 0;
}

// Sibling weights, one thread per parent (coalesced segment offsets): for
// each child in the parent's segment, the sizes of the siblings ordered
// before it, plus one for even children; the parent's odd total goes to
// oddsz. Segments of up to kSmallChildren children are done here;
// larger ones are queued for k_big_parents (up to kHugeChildren) or for the
// id-ordered scan (beyond).
constexpr int kSmallChildren = 32;

__device__ inline int32_t child_of_key(int32_t k) { return k >= 0 ? k : -k - 1; }

__global__ void __launch_bounds__(kBlock) k_siblings(int32_t n, const int32_t* __restrict__ coff,
                                                     const int2* __restrict__ cl_ks, int32_t* __restrict__ wgt,
                                                     int32_t* __restrict__ oddsz, int32_t* biglist,
                                                     int32_t* hugelist, Counters* cnt) {
    if (cnt->deep) return;
    const int lane = threadIdx.x & 31;
    for (int32_t a0 = blockIdx.x * blockDim.x; a0 < n; a0 += gridDim.x * blockDim.x) {
        const int32_t a = a0 + threadIdx.x;
        int32_t s0 = 0, k = 0;
        if (a < n) {
            s0 = coff[a];
            k = coff[a + 1] - s0;
        }
        if (k > kHugeChildren) hugelist[atomicAdd(&cnt->n_huge, 1)] = a;
        else if (k > kSmallChildren) biglist[atomicAdd(&cnt->n_big, 1)] = a;
        else if (k > 0 && k <= 4) {  // few children: this thread alone
            int32_t os = 0;
            for (int32_t i = s0; i < s0 + k; ++i) {
                const int2 ki = __ldg(cl_ks + i);
                int32_t pre = 0;
                for (int32_t j = s0; j < s0 + k; ++j) {
                    const int2 kj = __ldg(cl_ks + j);
                    if (kj.x < ki.x) pre += kj.y;
                }
                wgt[child_of_key(ki.x)] = pre + (ki.x >= 0 ? 1 : 0);
                if (ki.x < 0) os += ki.y;
            }
            oddsz[a] = os;
        }
        // 5..kSmallChildren children: the whole warp, one lane per child
        unsigned mid = __ballot_sync(kFull, k > 4 && k <= kSmallChildren);
        while (mid) {
            const int src = __ffs(mid) - 1;
            mid &= mid - 1;
            const int32_t pa = __shfl_sync(kFull, a, src), ps0 = __shfl_sync(kFull, s0, src),
                          pk = __shfl_sync(kFull, k, src);
            const int2 mine = lane < pk ? __ldg(cl_ks + ps0 + lane) : make_int2(INT32_MAX, 0);
            int32_t pre = 0;
            for (int j = 0; j < pk; ++j) {
                const int32_t kx = __shfl_sync(kFull, mine.x, j), ky = __shfl_sync(kFull, mine.y, j);
                if (kx < mine.x) pre += ky;
            }
            int32_t os = (lane < pk && mine.x < 0) ? mine.y : 0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) os += __shfl_down_sync(kFull, os, o);
            if (lane < pk) wgt[child_of_key(mine.x)] = pre + (mine.x >= 0 ? 1 : 0);
            if (lane == 0) oddsz[pa] = os;
        }
    }
}

// One block per big parent (kSmallChildren < k <= kHugeChildren): the
// segment is sorted by order key in shared memory and scanned.
__global__ void __launch_bounds__(kBlock) k_big_parents(const int32_t* __restrict__ coff,
                                                        const int2* __restrict__ cl_ks,
                                                        const int32_t* __restrict__ biglist,
                                                        int32_t* __restrict__ wgt, int32_t* __restrict__ oddsz,
                                                        const Counters* cnt) {
    if (cnt->deep) return;
    __shared__ int2 sk[kHugeChildren];
    __shared__ int32_t wsum[kBlock / 32];
    __shared__ int32_t carry_s, odd_s;
    const int32_t nb = cnt->n_big;
    for (int32_t b = blockIdx.x; b < nb; b += gridDim.x) {
        const int32_t a = biglist[b];
        const int32_t s0 = coff[a], count = coff[a + 1] - s0;
        int p2 = 1;
        while (p2 < count) p2 <<= 1;
        for (int i = threadIdx.x; i < p2; i += blockDim.x) sk[i] = i < count ? cl_ks[s0 + i] : make_int2(INT32_MAX, 0);
        __syncthreads();
        for (int kk = 2; kk <= p2; kk <<= 1) {
            for (int j = kk >> 1; j > 0; j >>= 1) {
                for (int i = threadIdx.x; i < p2; i += blockDim.x) {
                    const int ixj = i ^ j;
                    if (ixj > i) {
                        const int2 x = sk[i], y = sk[ixj];
                        const bool up = (i & kk) == 0;
                        if ((x.x > y.x) == up) {
                            sk[i] = y;
                            sk[ixj] = x;
                        }
                    }
                }
                __syncthreads();
            }
        }
        if (threadIdx.x == 0) {
            carry_s = 0;
            odd_s = 0;
        }
        __syncthreads();
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
        for (int base = 0; base < count; base += blockDim.x) {
            const int i = base + threadIdx.x;
            const int2 e = i < count ? sk[i] : make_int2(0, 0);
            const int32_t sv = i < count ? e.y : 0;
            int32_t x = sv;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int32_t y = __shfl_up_sync(kFull, x, o);
                if (lane >= o) x += y;
            }
            if (lane == 31) wsum[wid] = x;
            __syncthreads();
            if (wid == 0) {
                int32_t t = lane < kBlock / 32 ? wsum[lane] : 0;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int32_t y = __shfl_up_sync(kFull, t, o);
                    if (lane >= o) t += y;
                }
                if (lane < kBlock / 32) wsum[lane] = t;
            }
            __syncthreads();
            if (i < count) {
                wgt[child_of_key(e.x)] = carry_s + (wid > 0 ? wsum[wid - 1] : 0) + x - sv + (e.x >= 0 ? 1 : 0);
                if (e.x < 0) atomicAdd(&odd_s, sv);
            }
            __syncthreads();
            if (threadIdx.x == 0) carry_s += wsum[kBlock / 32 - 1];
            __syncthreads();
        }
        if (threadIdx.x == 0) oddsz[a] = odd_s;
        __syncthreads();
    }
}

// Children of the sink: ordered by id, so one id-ordered scan gives their
// weights. Even child c: 1 + (all odd children) + (even children with
// smaller id); odd child c: odd children with larger id. The sink's rank is
// the odd total. Three kernels: tile sums, a one-block scan of the tile sums,
// per-tile scans. Parents above kHugeChildren children use the same scan in
// k_idscan_coop below.
constexpr int kCIpt = kCoopTile / kBlock;

__device__ inline void sink_contrib(int32_t sv, int32_t* e, int32_t* o) {
    int32_t s = sv & 0x7fffffff;
    *e = sv > 0 ? s : 0;
    *o = sv < 0 ? s : 0;
}

__device__ inline void block_scan2(int32_t ve, int32_t vo, int64_t* xe, int64_t* xo, int64_t* te, int64_t* to) {
    __shared__ int64_t se[kBlock / 32], so[kBlock / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int64_t a = ve, b = vo;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        int64_t ya = __shfl_up_sync(kFull, a, d), yb = __shfl_up_sync(kFull, b, d);
        if (lane >= d) {
            a += ya;
            b += yb;
        }
    }
    if (lane == 31) {
        se[wid] = a;
        so[wid] = b;
    }
    __syncthreads();
    if (wid == 0) {
        int64_t pa = lane < kBlock / 32 ? se[lane] : 0, pb = lane < kBlock / 32 ? so[lane] : 0;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            int64_t ya = __shfl_up_sync(kFull, pa, d), yb = __shfl_up_sync(kFull, pb, d);
            if (lane >= d) {
                pa += ya;
                pb += yb;
            }
        }
        if (lane < kBlock / 32) {
            se[lane] = pa;
            so[lane] = pb;
        }
    }
    __syncthreads();
    *xe = (wid > 0 ? se[wid - 1] : 0) + a - ve;  // exclusive
    *xo = (wid > 0 ? so[wid - 1] : 0) + b - vo;
    *te = se[kBlock / 32 - 1];
    *to = so[kBlock / 32 - 1];
    __syncthreads();
}

// kCIpt consecutive sinkval entries starting at i0 (16-byte loads when full)
__device__ inline void load8(const int32_t* __restrict__ sinkval, int32_t n, int64_t i0, int32_t v[kCIpt]) {
    if (i0 + kCIpt <= n) {
#pragma unroll
        for (int q = 0; q < kCIpt / 4; ++q) {
            int4 a = __ldg(reinterpret_cast<const int4*>(sinkval + i0) + q);
            v[4 * q] = a.x;
            v[4 * q + 1] = a.y;
            v[4 * q + 2] = a.z;
            v[4 * q + 3] = a.w;
        }
    } else {
#pragma unroll
        for (int k = 0; k < kCIpt; ++k) v[k] = i0 + k < n ? sinkval[i0 + k] : 0;
    }
}


// exclusive scan of the (even, odd) tile sums (tsum, summed by k_scatter) by
// one block into tiles, totals after the last tile; tsum is cleared for the
// next valuation. A single game whose sink slot is its last id needs no
// k_game_prefix: its prefixes at its first id are zero and the odd prefix at
// its sink slot is the odd total, which ranks the sink (sink_key >= 0 names it).
constexpr int kTileScanThreads = 1024;

__global__ void __launch_bounds__(kTileScanThreads) k_tiles_scan(int64_t* __restrict__ tsum, int64_t* tiles,
                                                                 int64_t ntiles, int32_t sink_key, int64_t* gscan,
                                                                 int32_t* key, Counters* cnt) {
    if (cnt->deep) return;
    __shared__ int64_t se[kTileScanThreads / 32], so[kTileScanThreads / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int64_t ce = 0, co = 0;
    for (int64_t b = 0; b < ntiles; b += kTileScanThreads) {
        const int64_t i = b + threadIdx.x;
        const int64_t e = i < ntiles ? tsum[2 * i] : 0, o = i < ntiles ? tsum[2 * i + 1] : 0;
        if (i < ntiles) {
            tsum[2 * i] = 0;
            tsum[2 * i + 1] = 0;
        }
        int64_t xa = e, xb = o;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int64_t ya = __shfl_up_sync(kFull, xa, d), yb = __shfl_up_sync(kFull, xb, d);
            if (lane >= d) {
                xa += ya;
                xb += yb;
            }
        }
        if (lane == 31) {
            se[wid] = xa;
            so[wid] = xb;
        }
        __syncthreads();
        if (wid == 0) {
            int64_t pa = se[lane], pb = so[lane];
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const int64_t ya = __shfl_up_sync(kFull, pa, d), yb = __shfl_up_sync(kFull, pb, d);
                if (lane >= d) {
                    pa += ya;
                    pb += yb;
                }
            }
            se[lane] = pa;
            so[lane] = pb;
        }
        __syncthreads();
        if (i < ntiles) {
            tiles[2 * i] = ce + (wid > 0 ? se[wid - 1] : 0) + xa - e;
            tiles[2 * i + 1] = co + (wid > 0 ? so[wid - 1] : 0) + xb - o;
        }
        ce += se[kTileScanThreads / 32 - 1];
        co += so[kTileScanThreads / 32 - 1];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        tiles[2 * ntiles] = ce;
        tiles[2 * ntiles + 1] = co;
        if (sink_key >= 0) {
            gscan[0] = 0;
            gscan[1] = 0;
            gscan[2] = co;
            key[sink_key] = (int32_t)co;
            cnt->sink_rank = (int32_t)co;
        }
    }
}

// Per game g (one warp each): the even and odd exclusive prefixes over all ids
// at the game's first id and the odd prefix at its sink slot, from the
// scanned tile sums plus the partial tile. The game's ranks are these global
// prefixes minus the values at its first id; its sink's rank is its odd total,
// written into the sink slot's key.
__device__ inline void prefix_at(int64_t p, int32_t n, const int32_t* __restrict__ sinkval,
                                 const int64_t* __restrict__ tiles, int64_t* pe, int64_t* po) {
    const int lane = threadIdx.x & 31;
    const int64_t t = p / kCoopTile;
    int64_t e = 0, o = 0;
    for (int64_t i = t * kCoopTile + lane; i < p && i < n; i += 32) {
        int32_t ee, oo;
        sink_contrib(sinkval[i], &ee, &oo);
        e += ee;
        o += oo;
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
        e += __shfl_down_sync(kFull, e, d);
        o += __shfl_down_sync(kFull, o, d);
    }
    *pe = tiles[2 * t] + e;
    *po = tiles[2 * t + 1] + o;
}

__global__ void __launch_bounds__(kBlock) k_game_prefix(int32_t n, int32_t ngames, const int32_t* __restrict__ gsink,
                                                        const int32_t* __restrict__ sinkval,
                                                        const int64_t* __restrict__ tiles, int64_t* gscan,
                                                        int32_t* key, Counters* cnt) {
    if (cnt->deep) return;
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t gi = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; gi < ngames; gi += nw) {
        const int64_t base = gi == 0 ? 0 : (int64_t)gsink[gi - 1] + 1;
        const int64_t sk = gsink[gi];
        int64_t eb, ob, es, os;
        prefix_at(base, n, sinkval, tiles, &eb, &ob);
        prefix_at(sk, n, sinkval, tiles, &es, &os);
        if (lane == 0) {
            gscan[3 * gi] = eb;
            gscan[3 * gi + 1] = ob;
            gscan[3 * gi + 2] = os;
            key[sk] = (int32_t)(os - ob);
            if (gi == 0) cnt->sink_rank = (int32_t)(os - ob);
        }
    }
}

__global__ void __launch_bounds__(kBlock) k_sink_apply(int32_t n, const int32_t* __restrict__ sinkval,
                                                       const int64_t* __restrict__ tiles,
                                                       const int32_t* __restrict__ vgame,
                                                       const int64_t* __restrict__ gscan, int32_t* __restrict__ wgt,
                                                       const Counters* cnt) {
    if (cnt->deep) return;
    const int64_t i0 = (int64_t)blockIdx.x * kCoopTile + (int64_t)threadIdx.x * kCIpt;
    int32_t v[kCIpt];
    load8(sinkval, n, i0, v);
    int32_t es[kCIpt], os[kCIpt];
    int32_t e = 0, o = 0;
#pragma unroll
    for (int k = 0; k < kCIpt; ++k) {
        sink_contrib(v[k], &es[k], &os[k]);
        e += es[k];
        o += os[k];
    }
    int64_t xe, xo, te, to;
    block_scan2(e, o, &xe, &xo, &te, &to);
    int64_t run_e = tiles[2 * blockIdx.x] + xe, run_o = tiles[2 * blockIdx.x + 1] + xo;
#pragma unroll
    for (int k = 0; k < kCIpt; ++k) {
        if (es[k] | os[k]) {
            const int64_t gi = vgame ? vgame[i0 + k] : 0;
            const int64_t eb = gscan[3 * gi], ob = gscan[3 * gi + 1], tot_o = gscan[3 * gi + 2] - ob;
            if (es[k]) wgt[i0 + k] = (int32_t)(1 + tot_o + (run_e - eb));
            else wgt[i0 + k] = (int32_t)(tot_o - (run_o + os[k] - ob));
        }
        run_o += os[k];
        run_e += es[k];
    }
}

// Parents with more than kHugeChildren children (none in the measured
// workloads): the same id-ordered scan over every vertex, one parent after
// the other, in one cooperative launch that returns at once when there are
// none. Children of a are the vertices whose g-word points at a.
__global__ void __launch_bounds__(kBlock) k_idscan_coop(int32_t n, const uint32_t* __restrict__ gd32,
                                                        const int32_t* __restrict__ sz,
                                                        const uint8_t* __restrict__ kind,
                                                        const int32_t* __restrict__ hugelist, int64_t* tiles,
                                                        int64_t ntiles, int32_t* wgt, int32_t* oddsz, Counters* cnt) {
    if (cnt->deep) return;  // uniform over the grid: no block reaches a barrier
    const int32_t nh = cnt->n_huge;
    for (int32_t h = 0; h < nh; ++h) {
        const int32_t a = hugelist[h];
        auto contrib = [&](int64_t i, int32_t* e, int32_t* o) {
            *e = *o = 0;
            if (i >= n) return;
            const uint8_t kd = kind[i];
            if ((kd & kKFin) && !(kd & kKSinkChild) && g32_ptr(gd32[i]) == a) {
                int32_t s = 1 + sz[i];
                if (kd & kKOdd) *o = s;
                else *e = s;
            }
        };
        for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
            int32_t e = 0, o = 0;
            for (int k = 0; k < kCIpt; ++k) {
                int32_t ee, oo;
                contrib(t * kCoopTile + (int64_t)threadIdx.x * kCIpt + k, &ee, &oo);
                e += ee;
                o += oo;
            }
            int64_t xe, xo, te, to;
            block_scan2(e, o, &xe, &xo, &te, &to);
            if (threadIdx.x == 0) {
                tiles[2 * t] = te;
                tiles[2 * t + 1] = to;
            }
        }
        if (!grid_sync(cnt)) return;
        if (blockIdx.x == 0) {
            int64_t ce = 0, co = 0;
            for (int64_t b = 0; b < ntiles; b += kBlock) {
                int64_t i = b + threadIdx.x;
                int64_t e = i < ntiles ? tiles[2 * i] : 0, o = i < ntiles ? tiles[2 * i + 1] : 0;
                int64_t xe, xo, te, to;
                block_scan2((int32_t)e, (int32_t)o, &xe, &xo, &te, &to);
                if (i < ntiles) {
                    tiles[2 * i] = ce + xe;
                    tiles[2 * i + 1] = co + xo;
                }
                ce += te;
                co += to;
            }
            if (threadIdx.x == 0) {
                tiles[2 * ntiles] = ce;
                tiles[2 * ntiles + 1] = co;
            }
        }
        if (!grid_sync(cnt)) return;
        const int64_t tot_o = tiles[2 * ntiles + 1];
        for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
            int32_t es[kCIpt], os[kCIpt];
            int32_t e = 0, o = 0;
            const int64_t i0 = t * kCoopTile + (int64_t)threadIdx.x * kCIpt;
            for (int k = 0; k < kCIpt; ++k) {
                contrib(i0 + k, &es[k], &os[k]);
                e += es[k];
                o += os[k];
            }
            int64_t xe, xo, te, to;
            block_scan2(e, o, &xe, &xo, &te, &to);
            int64_t run_e = tiles[2 * t] + xe, run_o = tiles[2 * t + 1] + xo;
            for (int k = 0; k < kCIpt; ++k) {
                if (es[k]) wgt[i0 + k] = (int32_t)(1 + tot_o + run_e);
                run_o += os[k];
                if (os[k]) wgt[i0 + k] = (int32_t)(tot_o - run_o);
                run_e += es[k];
            }
        }
        if (blockIdx.x == 0 && threadIdx.x == 0) oddsz[a] = (int32_t)tot_o;
        if (!grid_sync(cnt)) return;  // the tile sums are reused by the next parent
    }
}

// Ranks: sum the weights along each finite vertex's g-chain (TOP vertices
// rank above everything).
__global__ void __launch_bounds__(kBlock) k_chain2(int32_t n, const uint32_t* __restrict__ gd32,
                                                   const uint8_t* __restrict__ kind, const int32_t* __restrict__ wgt,
                                                   const int32_t* __restrict__ oddsz, int32_t* __restrict__ key,
                                                   const Counters* cnt) {
    if (cnt->err || cnt->deep) return;  // unfinished jumping or a deep forest: no chain walk
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t tile = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; warp_tile_base(tile) < n;
         tile += nwarps) {
        int32_t v[kIlp], x[kIlp], acc[kIlp];
        bool fin[kIlp], act[kIlp], slotid[kIlp];
#pragma unroll
        for (int j = 0; j < kIlp; ++j) {
            v[j] = (int32_t)(warp_tile_base(tile) + lane + 32 * j);
            const uint8_t kd = v[j] < n ? kind[v[j]] : 0;
            slotid[j] = (kd & kKSinkSlot) != 0;
            fin[j] = (kd & kKFin) != 0;
            acc[j] = 0;
            x[j] = 0;
            act[j] = false;
            if (fin[j]) {
                acc[j] = oddsz[v[j]] + wgt[v[j]];
                const uint32_t w = gd32[v[j]];
                x[j] = g32_ptr(w);
                act[j] = !g32_sink(w);
            }
        }
        for (;;) {
            bool any = false;
            uint32_t wx[kIlp];
            int32_t wg[kIlp];
#pragma unroll
            for (int j = 0; j < kIlp; ++j) {
                wx[j] = act[j] ? gd32[x[j]] : 0u;
                wg[j] = act[j] ? wgt[x[j]] : 0;
            }
#pragma unroll
            for (int j = 0; j < kIlp; ++j) {
                if (act[j]) {
                    acc[j] += wg[j];
                    x[j] = g32_ptr(wx[j]);
                    act[j] = !g32_sink(wx[j]);
                }
                any |= act[j];
            }
            if (!any) break;
        }
#pragma unroll
        for (int j = 0; j < kIlp; ++j)
            if (v[j] < n && !slotid[j]) key[v[j]] = fin[j] ? acc[j] : INT32_MAX;
    }
}

// Depth of every finite vertex (outputs only): the number of vertices on its
// play before the sink, the sum of the walk lengths along its g-chain.
__global__ void __launch_bounds__(kBlock) k_depth(int32_t n, const uint64_t* __restrict__ gd,
                                                  const uint8_t* __restrict__ kind, int32_t* __restrict__ depth,
                                                  const Counters* cnt) {
    if (cnt->err) return;  // unfinished jumping: no chain walk
    for (int32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        int32_t dep = -1;
        if (kind[v] & kKFin) {
            uint64_t w = gd[v];
            uint32_t d = gd_dist(w);
            while (!gd_sink(w)) {
                w = gd[gd_ptr(w)];
                d += gd_dist(w);
            }
            dep = (int32_t)d;
        }
        depth[v] = dep;
    }
}

// K3: greedy all-switches for one player, one thread per vertex. Edges are
// taken in batches of four whose target reads and rank gathers are issued
// together, then compared in edge-list order (first minimiser for Odd; for
// Even the sink first, then the first maximiser). A game takes part while it
// is active; Even switches only in games where no Odd vertex switched in this
// iteration (the inner loop of Algorithm 1 has converged).
template <typename OffT>
__global__ void __launch_bounds__(kBlock) k_switch(int32_t n, int player, const OffT* __restrict__ off,
                                                   const int32_t* __restrict__ tgt,
                                                   const uint8_t* __restrict__ flags,
                                                   const int32_t* __restrict__ key, const int32_t* __restrict__ vgame,
                                                   const int32_t* __restrict__ gsink, int32_t sink0, GameState* gst,
                                                   int32_t* strat, Counters* cnt) {
    if (cnt->deep) return;  // the ranks were not computed: the loop stops and continues on the ruling-set path
    if (!vgame) {  // one game: the whole pass is skipped when the game does not switch this player now
        const GameState st = gst[0];
        if (st.phase != kPhaseActive || (player == 0 && st.sw_odd != 0)) return;
    }
    int32_t nsw = 0;
    for (int32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        const uint8_t f = flags[v];
        if ((f & kSinkSlot) || (int)(f & kOwnerOdd) != player) continue;
        const int32_t gi = vgame ? vgame[v] : 0;
        const GameState st = gst[gi];
        if (st.phase != kPhaseActive || (player == 0 && st.sw_odd != 0)) continue;
        const int64_t e0 = off[v], e1 = off[v + 1];
        const int32_t cur = strat[v];
        const int32_t sk = player == 0 ? (vgame ? gsink[gi] : sink0) : 0;
        int32_t best = player == 0 ? sk : -1;
        int32_t bk = player == 0 ? key[sk] : INT32_MAX;
        // the current successor is the sink (Even) or one of the edges: its key comes with them
        int32_t curkey = (player == 0 && cur == sk) ? bk : 0;
        for (int64_t e = e0; e < e1; e += 4) {
            int32_t t[4], kk[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) t[j] = e + j < e1 ? tgt[e + j] : -1;
#pragma unroll
            for (int j = 0; j < 4; ++j) kk[j] = t[j] >= 0 ? key[t[j]] : 0;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                if (t[j] < 0) continue;
                if (t[j] == cur) curkey = kk[j];
                bool better = player == 0 ? kk[j] > bk : (best < 0 || kk[j] < bk);
                if (better) {
                    best = t[j];
                    bk = kk[j];
                }
            }
        }
        if (player == 0 ? bk > curkey : bk < curkey) {
            strat[v] = best;
            ++nsw;
            if (vgame) {  // one count per group of lanes of the same game
                cg::coalesced_group sw = cg::coalesced_threads();
                cg::coalesced_group same = cg::labeled_partition(sw, gi);
                if (same.thread_rank() == 0)
                    atomicAdd(player ? &gst[gi].sw_odd : &gst[gi].sw_even, (int32_t)same.size());
            }
        }
    }
    block_add(nsw, &cnt->n_switch);
    if (!vgame) {  // one game: the block totals are the game's
        __shared__ int32_t tot;
        if (threadIdx.x == 0) tot = 0;
        __syncthreads();
        int32_t x = nsw;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(kFull, x, o);
        if ((threadIdx.x & 31) == 0 && x) atomicAdd(&tot, x);
        __syncthreads();
        if (threadIdx.x == 0 && tot) atomicAdd(player ? &gst[0].sw_odd : &gst[0].sw_even, tot);
    }
}

// Per-game bookkeeping of Algorithm 1 after the switching passes (one thread
// per game): count the valuation, stop at an odd cycle, finish when neither
// player switched (or, for best responses, when Odd did not), count a major
// iteration when Even switched, stop at the cap. Counts the games still active.
// With reset_mode, a game whose Even player switched is marked for k_reset_odd.
__global__ void k_bookkeep(int32_t ngames, GameState* gst, int64_t cap, int even_phase, int reset_mode,
                           int32_t* gactive, const Counters* cnt) {
    if (cnt->deep) return;  // an abandoned iteration: nothing counted, no game active (the loop stops)
    int32_t act = 0;
    for (int32_t gi = blockIdx.x * blockDim.x + threadIdx.x; gi < ngames; gi += gridDim.x * blockDim.x) {
        GameState st = gst[gi];
        st.reset = 0;
        if (st.phase == kPhaseActive) {
            st.inner += 1;
            if (st.nodd > 0) st.phase = kPhaseOddCycle;
            else if (st.sw_odd == 0) {
                if (!even_phase || st.sw_even == 0) st.phase = kPhaseDone;
                else {
                    st.major += 1;
                    st.reset = reset_mode;
                    if (reset_mode) atomicOr(gactive + 1, 1);  // Odd restarts: the next Odd pass is full
                }
            }
            if (st.phase == kPhaseActive && st.inner >= cap) st.phase = kPhaseTimeout;
        }
        st.sw_odd = st.sw_even = st.nodd = 0;
        gst[gi] = st;
        act += st.phase == kPhaseActive;
    }
    block_add(act, gactive);
}

// SI-Reset (Section 6): in games marked by k_bookkeep, every Odd vertex goes
// back to the first edge of its list (the initial strategy of Algorithm 1);
// k_bookkeep has set the flag that makes the next Odd switching pass full.
template <typename OffT>
__global__ void __launch_bounds__(kBlock) k_reset_odd(int32_t n, const OffT* __restrict__ off,
                                                      const int32_t* __restrict__ tgt,
                                                      const uint8_t* __restrict__ flags,
                                                      const int32_t* __restrict__ vgame, const GameState* gst,
                                                      int32_t* strat, const Counters* cnt) {
    if (cnt->deep) return;
    if (!vgame && !gst[0].reset) return;
    for (int32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        const uint8_t f = flags[v];
        if ((f & kSinkSlot) || !(f & kOwnerOdd)) continue;
        if (vgame && !gst[vgame[v]].reset) continue;
        strat[v] = tgt[off[v]];
    }
}

// ---------------------------------------------------------------------------
// Loop iterations without ranks. Switching (Section 3, "Switching rules")
// only compares the valuations of a vertex's successors with each other, so
// the loop does not need the position of every valuation in the order: two
// finite valuations are compared directly on the g-forest. Walk both g-chains
// upwards, always advancing the smaller id, until they meet at their lowest
// common g-ancestor (at the latest the game's sink slot). The largest vertex
// of the symmetric difference of the two plays is the larger of the last two
// vertices passed below the meeting point; its side wins for Even when its
// priority is even. TOP valuations are above every finite one and equal to
// each other. The dense ranks, depths and classes of the outputs come from a
// full valuation after the loop.

// After k_classify, bit 31 of a g-word marks a TOP vertex (its play ends in
// a cycle); finite words are unchanged (bit 30: g(v) is the game's sink slot).
constexpr uint32_t kG32Top = 0x80000000u;
// k_classify also writes one "top word" per vertex: bit 31 = TOP; for a finite
// vertex bits 0..29 = its top, the last vertex of its g-chain below the sink
// slot (a child of the sink in the g-forest), and bit 30 = that top's priority
// is odd.
constexpr uint32_t kTopOdd = 0x40000000u;
__device__ inline int32_t top_id(uint32_t t) { return (int32_t)(t & 0x3fffffffu); }

// Class and top of every vertex from its g-chain: a chain that ends at a
// "none" vertex (above its whole infinite future) or passes a vertex already
// marked TOP is TOP, and its g-word gets bit 31; a chain that reaches the sink
// is finite, its top being the chain's last vertex. g-words change only by
// gaining bit 31 on TOP vertices, and a walker that reads either the old or
// the new word of a TOP vertex stops there with the same answer, so the
// in-place marks are race-free shortcuts. A cycle maximum (a none vertex whose
// pointer is itself) with an odd priority counts toward its game's odd cycles
// (sigma not admissible).
//
// With omark, a top word is written only when it differs from the previous
// iteration's, and then every Odd vertex with an edge to v (rv_off, rv_src)
// is marked for the next Odd switching pass. An Odd vertex decides from its
// successors' top words alone, unless two finite successors with the best
// top tie (a chain comparison, which leaves its mark set): so an unmarked
// vertex, none of whose successors changed since it was last evaluated,
// would take the same decision again and is skipped. Before a full Odd pass
// (*full != 0) no marks are needed. Eight blocks per SM: the pass is bound
// by the latency of its chain gathers.
template <int ILP = kIlp>
__global__ void __launch_bounds__(kBlock, 2048 / kBlock)
    k_classify(int32_t n, uint32_t* gd32, const uint8_t* __restrict__ flags, uint32_t* __restrict__ topw,
               const int32_t* __restrict__ vgame, GameState* gst, Counters* cnt, int32_t deep_cut,
               const int32_t* __restrict__ rv_off, const int32_t* __restrict__ rv_src, uint8_t* omark,
               const int32_t* __restrict__ full) {
    if (cnt->err || cnt->deep) return;  // unfinished jumping: g-words may point downwards, no chain walk would end
    if (omark && *full) omark = nullptr;  // the next Odd pass evaluates every Odd vertex: no marks
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t tile = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; (tile * 32 * ILP) < n;
         tile += nwarps) {
        if (tile_idle(tile * 32 * ILP, (tile + 1) * 32 * ILP, n, vgame, gst)) continue;
        int32_t v[ILP], x[ILP];
        uint32_t ot[ILP];
        // bit j: slot j walks / is TOP / its top's priority is odd / its own word is "none" (not to be marked)
        uint32_t act = 0, top = 0, podd = 0, wnone = 0;
#pragma unroll
        for (int j = 0; j < ILP; ++j) {
            v[j] = (int32_t)((tile * 32 * ILP) + lane + 32 * j);
            // (a sink slot's word is the sink bit alone: its own top, even)
            const uint32_t w0 = v[j] < n ? gd32[v[j]] : kG32Sink;
            if (g32_none(w0)) top |= 1u << j, wnone |= 1u << j;
            x[j] = g32_sink(w0) ? v[j] : g32_ptr(w0);  // a child of the sink is its own top
            if (!(w0 & (kG32None | kG32Sink))) act |= 1u << j;
            if (g32_sink(w0)) podd |= (w0 & 1u) << j;
            if (v[j] < n && g32_none(w0) && x[j] == v[j] && (flags[v[j]] & kPriOdd))
                atomicAdd(&gst[vgame ? vgame[v[j]] : 0].nodd, 1);
        }
        // the chains start together, so a chain still going has taken `len` steps
        for (int32_t len = 1; act; ++len) {
            if (len > deep_cut) {  // a deep forest: the iteration is abandoned (loop stops)
                cnt->deep = 1;
                break;
            }
            uint32_t wx[ILP];
#pragma unroll
            for (int j = 0; j < ILP; ++j) wx[j] = ((act >> j) & 1u) ? gd32[x[j]] : 0u;
#pragma unroll
            for (int j = 0; j < ILP; ++j) {
                if (!((act >> j) & 1u)) continue;
                if (wx[j] & kG32Top) {  // a none vertex, or one already marked TOP
                    top |= 1u << j;
                    act &= ~(1u << j);
                } else if (g32_sink(wx[j])) {  // x is the top
                    podd |= (wx[j] & 1u) << j;
                    act &= ~(1u << j);
                } else {
                    const int32_t nx = g32_ptr(wx[j]);
                    if (nx <= x[j]) act &= ~(1u << j);  // g-chains rise (a guard, never taken here)
                    x[j] = nx;
                }
            }
        }
#pragma unroll
        for (int j = 0; j < ILP; ++j) ot[j] = (omark && v[j] < n) ? __ldcs(topw + v[j]) : 0u;  // read once: evict first
#pragma unroll
        for (int j = 0; j < ILP; ++j) {
            if (v[j] >= n) continue;
            const bool tp = (top >> j) & 1u;
            if (tp && !((wnone >> j) & 1u)) gd32[v[j]] |= kG32Top;  // only this thread writes v's word
            const uint32_t tw = tp ? kG32Top : (((podd >> j) & 1u) ? kTopOdd : 0u) | (uint32_t)x[j];
            if (!omark) {
                topw[v[j]] = tw;
            } else if (tw != ot[j]) {
                topw[v[j]] = tw;
                const int32_t e1 = rv_off[v[j] + 1];
                for (int32_t e = rv_off[v[j]]; e < e1; ++e) omark[rv_src[e]] = 1;
            }
        }
    }
}

// Compares the valuations of two finite vertices u and w of one game with the
// same top: walk both g-chains (words wu, ww) upwards, always advancing the
// smaller id, until they meet (at the top at the latest). The larger of the
// last two vertices passed below the meeting point is the largest vertex of
// the symmetric difference of the two plays; its side is better for Even
// when its priority is even. Returns > 0 if Val(u) is better for Even, < 0 if
// worse, 0 if u == w. g(x) > x for every vertex below the top, so each step
// raises a or b.
__device__ inline int cmp_walk(int32_t u, int32_t w, const uint32_t* __restrict__ gd32,
                               const uint8_t* __restrict__ flags) {
    int32_t a = u, b = w, pa = -1, pb = -1;
    uint32_t wa = 0, wb = 0;
    if (a != b) {
        wa = gd32[a];
        wb = gd32[b];
    }
    while (a != b) {
        if (a < b) {
            pa = a;
            a = g32_ptr(wa);
            if (a <= pa) return 0;  // g-chains rise (a guard that keeps every walk finite; never taken)
            wa = gd32[a];
        } else {
            pb = b;
            b = g32_ptr(wb);
            if (b <= pb) return 0;
            wb = gd32[b];
        }
    }
    if (pa == pb) return 0;  // u == w
    const bool u_side = pa > pb;
    const bool even = !(flags[u_side ? pa : pb] & kPriOdd);
    return u_side == even ? 1 : -1;
}

// Order of the valuations of u and w (vertices of one game, with their top
// words tu, tw): > 0 if Val(u) is better for Even than Val(w), < 0 if worse,
// 0 if equal. TOP is above every finite valuation and equal to TOP. Finite
// plays with different tops differ above everything else at the larger top,
// which decides by its parity; with the same top the chains are walked.
__device__ inline int cmp_val(int32_t u, uint32_t tu, int32_t w, uint32_t tw, const uint32_t* __restrict__ gd32,
                              const uint8_t* __restrict__ flags) {
    const int xu = (tu & kG32Top) ? 1 : 0, xw = (tw & kG32Top) ? 1 : 0;
    if (xu | xw) return xu - xw;
    const int32_t hu = top_id(tu), hw = top_id(tw);
    if (hu != hw) {
        const bool u_side = hu > hw;
        const bool even = !((u_side ? tu : tw) & kTopOdd);
        return u_side == even ? 1 : -1;
    }
    return cmp_walk(u, w, gd32, flags);
}

// Against the sink's empty valuation: the top of a finite play is its largest
// vertex, so Val(u) is better for Even exactly when that top is even.
__device__ inline int cmp_sink(uint32_t tu) {
    if (tu & kG32Top) return 1;
    return (tu & kTopOdd) ? -1 : 1;
}

// K3 with comparisons: as k_switch (one thread per vertex of the switching
// player, the first minimiser for Odd, the sink first and then the first
// maximiser for Even, a switch only when strictly better), with the best
// successor kept by comparing valuations. Two valuations are equal only when
// both are TOP, so Odd switches when its best successor differs from the
// current one and is finite, Even when they differ and the current one is not
// TOP (the best one is then at least as good as TOP only if equal to it).
template <typename OffT, int BS>
__global__ void __launch_bounds__(BS) k_switch_cmp(int32_t n, int player, const OffT* __restrict__ off,
                                                       const int32_t* __restrict__ tgt,
                                                       const uint8_t* __restrict__ flags,
                                                       const uint32_t* __restrict__ gd32,
                                                       const uint32_t* __restrict__ topw,
                                                       const int32_t* __restrict__ vgame,
                                                       const int32_t* __restrict__ gsink, int32_t sink0,
                                                       GameState* gst, int32_t* strat, Counters* cnt) {
    if (cnt->err || cnt->deep) return;  // unfinished jumping, or a deep forest (the loop stops)
    if (!vgame) {  // one game: the whole pass is skipped when the game does not switch this player now
        const GameState st = gst[0];
        if (st.phase != kPhaseActive || (player == 0 && st.sw_odd != 0)) return;
    }
    int32_t nsw = 0;
    for (int32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        const uint8_t f = flags[v];
        if ((f & kSinkSlot) || (int)(f & kOwnerOdd) != player) continue;
        const int32_t gi = vgame ? vgame[v] : 0;
        if (vgame) {
            const GameState st = gst[gi];
            if (st.phase != kPhaseActive || (player == 0 && st.sw_odd != 0)) continue;
        }
        const int64_t e0 = off[v], e1 = off[v + 1];
        const int32_t cur = strat[v];
        const int32_t sk = player == 0 ? (vgame ? gsink[gi] : sink0) : -1;
        int32_t best = sk;  // Even: the sink first; Odd: none yet
        uint32_t tbest = 0;
        bool cur_top = false;
        for (int64_t e = e0; e < e1; e += 4) {
            int32_t t[4];
            uint32_t tt[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) t[j] = e + j < e1 ? tgt[e + j] : -1;
#pragma unroll
            for (int j = 0; j < 4; ++j) tt[j] = t[j] >= 0 ? topw[t[j]] : 0u;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                if (t[j] < 0) continue;
                if (t[j] == cur) cur_top = (tt[j] & kG32Top) != 0;
                bool take;
                if (player == 1) take = best < 0 || cmp_val(t[j], tt[j], best, tbest, gd32, flags) < 0;
                else take = (best == sk ? cmp_sink(tt[j]) : cmp_val(t[j], tt[j], best, tbest, gd32, flags)) > 0;
                if (take) {
                    best = t[j];
                    tbest = tt[j];
                }
            }
        }
        const bool sw = best != cur && (player == 0 ? !cur_top : !(tbest & kG32Top));
        if (sw) {
            strat[v] = best;
            ++nsw;
            if (vgame) {  // one count per group of lanes of the same game
                cg::coalesced_group swg = cg::coalesced_threads();
                cg::coalesced_group same = cg::labeled_partition(swg, gi);
                if (same.thread_rank() == 0)
                    atomicAdd(player ? &gst[gi].sw_odd : &gst[gi].sw_even, (int32_t)same.size());
            }
        }
    }
    block_add(nsw, &cnt->n_switch);
    if (!vgame) {  // one game: the block totals are the game's
        __shared__ int32_t tot;
        if (threadIdx.x == 0) tot = 0;
        __syncthreads();
        int32_t x = nsw;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(kFull, x, o);
        if ((threadIdx.x & 31) == 0 && x) atomicAdd(&tot, x);
        __syncthreads();
        if (threadIdx.x == 0 && tot) atomicAdd(player ? &gst[0].sw_odd : &gst[0].sw_even, tot);
    }
}

// The switching players' views: the vertices of one player in increasing
// id order with their edge lists copied contiguously, so that a switching
// pass reads only its player's edges and every lane of a warp has a vertex.
__global__ void __launch_bounds__(kBlock) k_pl_mark(int32_t n, const uint8_t* __restrict__ flags,
                                                    uint8_t* __restrict__ m0, uint8_t* __restrict__ m1) {
    for (int32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        const uint8_t f = flags[v];
        const bool vert = !(f & kSinkSlot);
        m0[v] = vert && !(f & kOwnerOdd);
        m1[v] = vert && (f & kOwnerOdd);
    }
}

template <typename OffT>
__global__ void __launch_bounds__(kBlock) k_pl_gather(int32_t n, const uint8_t* __restrict__ m,
                                                      const int32_t* __restrict__ pos,
                                                      const OffT* __restrict__ off, int32_t* __restrict__ vid,
                                                      int32_t* __restrict__ deg) {
    for (int32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        if (!m[v]) continue;
        const int32_t i = pos[v];
        vid[i] = v;
        deg[i] = (int32_t)(off[v + 1] - off[v]);
    }
}

template <typename OffT>
__global__ void __launch_bounds__(kBlock) k_pl_copy(int32_t np, const int32_t* __restrict__ vid,
                                                    const OffT* __restrict__ off, const int32_t* __restrict__ tgt,
                                                    const int32_t* __restrict__ poff, int32_t* __restrict__ ptgt) {
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < np; i += gridDim.x * blockDim.x) {
        const int32_t v = vid[i];
        const OffT e0 = off[v];
        const int32_t k = (int32_t)(off[v + 1] - e0), d0 = poff[i];
        for (int32_t j = 0; j < k; ++j) ptgt[d0 + j] = tgt[e0 + j];
    }
}

// Odd's reverse view: the in-degree of every id from Odd's edges, then each
// edge's source (its position in Odd's view) at the next free slot of its
// target, cur[t] starting at rv_off[t] (the order within a list is arbitrary;
// the lists only mark).
__global__ void __launch_bounds__(kBlock) k_rv_count(int32_t np, const int32_t* __restrict__ poff,
                                                     const int32_t* __restrict__ ptgt, int32_t* __restrict__ cnt) {
    const int32_t m = poff[np];
    for (int32_t e = blockIdx.x * blockDim.x + threadIdx.x; e < m; e += gridDim.x * blockDim.x)
        atomicAdd(cnt + ptgt[e], 1);
}

__global__ void __launch_bounds__(kBlock) k_rv_fill(int32_t np, const int32_t* __restrict__ poff,
                                                    const int32_t* __restrict__ ptgt, int32_t* __restrict__ cur,
                                                    int32_t* __restrict__ rv_src) {
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < np; i += gridDim.x * blockDim.x) {
        const int32_t e1 = poff[i + 1];
        for (int32_t e = poff[i]; e < e1; ++e) rv_src[atomicAdd(cur + ptgt[e], 1)] = i;
    }
}

// One vertex of k_switch_cmp_pl: view position i (vertex vid[i]), with the
// rules of k_switch_cmp. Returns whether it switched; *tie tells whether the
// decision took a chain comparison (two finite successors with the best top
// so far), *gi is its game. Vertices of games that do not switch this player
// now are left alone (tie set, no switch).
template <int PLAYER, bool BATCH>
__device__ inline bool switch_at(int32_t i, const int32_t* __restrict__ vid,
                                 const int32_t* __restrict__ poff, const int32_t* __restrict__ ptgt,
                                 const uint8_t* __restrict__ flags, const uint32_t* __restrict__ gd32,
                                 const uint32_t* __restrict__ topw, const int32_t* __restrict__ vgame,
                                 const int32_t* __restrict__ gsink, int32_t sink0, const GameState* gst,
                                 int32_t* strat, bool* tie_out, int32_t* gi_out) {
    const int32_t v = vid[i];
    const int32_t gi = BATCH ? vgame[v] : 0;
    *gi_out = gi;
    *tie_out = true;
    if (BATCH) {
        const GameState st = gst[gi];
        if (st.phase != kPhaseActive || (PLAYER == 0 && st.sw_odd != 0)) return false;
    }
    const int32_t e0 = poff[i], e1 = poff[i + 1];
    const int32_t cur = strat[v];
    const int32_t sk = PLAYER == 0 ? (BATCH ? gsink[gi] : sink0) : -1;
    int32_t best = sk;  // Even: the sink first; Odd: none yet
    uint32_t tbest = 0;
    bool cur_top = false, tie = false;
    for (int32_t e = e0; e < e1; e += 4) {
        int32_t t[4];
        uint32_t tt[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) t[j] = e + j < e1 ? ptgt[e + j] : -1;
#pragma unroll
        for (int j = 0; j < 4; ++j) tt[j] = t[j] >= 0 ? topw[t[j]] : 0u;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if (t[j] < 0) continue;
            if (PLAYER == 0 && t[j] == cur) cur_top = (tt[j] & kG32Top) != 0;
            bool take;
            if (PLAYER == 1) {
                tie |= best >= 0 && !((tt[j] | tbest) & kG32Top) && top_id(tt[j]) == top_id(tbest);
                take = best < 0 || cmp_val(t[j], tt[j], best, tbest, gd32, flags) < 0;
            } else take = (best == sk ? cmp_sink(tt[j]) : cmp_val(t[j], tt[j], best, tbest, gd32, flags)) > 0;
            if (take) {
                best = t[j];
                tbest = tt[j];
            }
        }
    }
    *tie_out = tie;
    const bool sw = best != cur && (PLAYER == 0 ? !cur_top : !(tbest & kG32Top));
    if (sw) strat[v] = best;
    return sw;
}

// A switch counted into its game (packed games: one atomic per group of
// lanes of the same game; one game: the block total at the end).
template <int PLAYER, bool BATCH>
__device__ inline void count_switch(bool sw, int32_t gi, GameState* gst, int32_t* nsw) {
    if (!sw) return;
    ++*nsw;
    if (BATCH) {
        cg::coalesced_group swg = cg::coalesced_threads();
        cg::coalesced_group same = cg::labeled_partition(swg, gi);
        if (same.thread_rank() == 0) atomicAdd(PLAYER ? &gst[gi].sw_odd : &gst[gi].sw_even, (int32_t)same.size());
    }
}

// k_switch_cmp over a player's view: thread i takes the player's i-th vertex.
// With MARKS (Odd's pass; omark holds one byte per view position, zero padded
// to a multiple of 16), a pass that is not full evaluates only the marked
// positions and clears the mark of each unless its decision took a chain
// comparison; a full pass (the first of a call, or after an SI-Reset:
// *full_flag != 0) evaluates every vertex and sets each mark to that flag.
// Full occupancy (32 registers): the evaluations wait on their gathers.
template <int BS, int PLAYER, bool MARKS, bool BATCH>
__global__ void __launch_bounds__(BS, 2048 / BS) k_switch_cmp_pl(int32_t np, const int32_t* __restrict__ vid,
                                                      const int32_t* __restrict__ poff,
                                                      const int32_t* __restrict__ ptgt,
                                                      const uint8_t* __restrict__ flags,
                                                      const uint32_t* __restrict__ gd32,
                                                      const uint32_t* __restrict__ topw,
                                                      const int32_t* __restrict__ vgame,
                                                      const int32_t* __restrict__ gsink, int32_t sink0,
                                                      GameState* gst, int32_t* strat, Counters* cnt,
                                                      uint8_t* omark, const int32_t* __restrict__ full_flag) {
    if (cnt->err || cnt->deep) return;  // unfinished jumping, or a deep forest (the loop stops)
    if (!BATCH) {  // one game: the whole pass is skipped when the game does not switch this player now
        const GameState st = gst[0];
        if (st.phase != kPhaseActive || (PLAYER == 0 && st.sw_odd != 0)) return;
    }
    const bool full = !MARKS || *full_flag;
    int32_t nsw = 0;
    if (full) {
        for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < np; i += gridDim.x * blockDim.x) {
            bool tie;
            int32_t gi;
            const bool sw = switch_at<PLAYER, BATCH>(i, vid, poff, ptgt, flags, gd32, topw, vgame, gsink, sink0, gst,
                                                     strat, &tie, &gi);
            if (MARKS) omark[i] = tie;
            count_switch<PLAYER, BATCH>(sw, gi, gst, &nsw);
        }
    } else if (MARKS) {
        // warps take 512 positions at a time: each lane loads 16 marks, the marked positions are listed in
        // shared memory (a warp scan of the lanes' counts), and the lanes share the list, so a chunk costs
        // one 16-byte load per lane plus ceil(marked / 32) evaluation rounds
        __shared__ int32_t list[BS / 32][512];
        int32_t* mine = list[threadIdx.x >> 5];
        const int lane = threadIdx.x & 31;
        const int32_t nch = (np + 511) >> 9;
        const int32_t nw = (int32_t)((gridDim.x * blockDim.x) >> 5);
        for (int32_t c = (int32_t)((blockIdx.x * blockDim.x + threadIdx.x) >> 5); c < nch; c += nw) {
            const int32_t q = (c << 9) + 16 * lane;
            uint4 m = make_uint4(0u, 0u, 0u, 0u);
            if (q < np) m = *reinterpret_cast<const uint4*>(omark + q);
            const uint32_t mw[4] = {m.x, m.y, m.z, m.w};
            const int k = __popc(m.x) + __popc(m.y) + __popc(m.z) + __popc(m.w);  // marks are 0 or 1
            int incl = k;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(kFull, incl, o);
                if (lane >= o) incl += y;
            }
            const int total = __shfl_sync(kFull, incl, 31);
            if (total == 0) continue;  // no successor of these 512 changed its top word
            int pos = incl - k;
#pragma unroll
            for (int b = 0; b < 16; ++b)
                if ((mw[b >> 2] >> (8 * (b & 3))) & 1u) mine[pos++] = q + b;
            __syncwarp();
            for (int j = lane; j < total; j += 32) {
                const int32_t i = mine[j];  // < np: the padding is never marked
                bool tie;
                int32_t gi;
                const bool sw = switch_at<PLAYER, BATCH>(i, vid, poff, ptgt, flags, gd32, topw, vgame, gsink, sink0,
                                                         gst, strat, &tie, &gi);
                if (!tie) omark[i] = 0;
                count_switch<PLAYER, BATCH>(sw, gi, gst, &nsw);
            }
            __syncwarp();
        }
    }
    block_add(nsw, &cnt->n_switch);
    if (!BATCH) {  // one game: the block totals are the game's
        __shared__ int32_t tot;
        if (threadIdx.x == 0) tot = 0;
        __syncthreads();
        int32_t x = nsw;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(kFull, x, o);
        if ((threadIdx.x & 31) == 0 && x) atomicAdd(&tot, x);
        __syncthreads();
        if (threadIdx.x == 0 && tot) atomicAdd(PLAYER ? &gst[0].sw_odd : &gst[0].sw_even, tot);
    }
}

}  // namespace

const char* const kKernelNames[KID_COUNT] = {"walk",     "jump",      "chain1", "child_scan", "scatter",
                                              "siblings", "sink_scan", "chain2", "switch_odd", "switch_even",
                                              "classify", "ruling_set"};

void prof_begin(pg_game* g, int id) {
    if (g->ctx->timing) cudaEventRecord(g->kev[2 * id], g->ctx->stream);
}

void prof_end(pg_game* g, int id, int nlaunch) {
    g->ctx->launches += nlaunch;
    g->klaunch[id] += nlaunch;
    if (g->ctx->timing) {
        cudaEventRecord(g->kev[2 * id + 1], g->ctx->stream);
        g->kpend[id] = true;
    }
}

void prof_collect(pg_game* g) {
    for (int id = 0; id < KID_COUNT; ++id) {
        if (!g->kpend[id]) continue;
        float ms = 0;
        if (cudaEventElapsedTime(&ms, g->kev[2 * id], g->kev[2 * id + 1]) == cudaSuccess) {
            g->kms[id] += ms;
            g->kcalls[id] += 1;
        }
        g->kpend[id] = false;
    }
}

pg_status alloc_scratch(pg_game* g) {
    pg_ctx* ctx = g->ctx;
    const int64_t n = g->n;
    auto A = [&](void** p, size_t bytes) { return dev_alloc(ctx, p, bytes, ctx->stream); };
    PG_CUDA_TRY(ctx, A((void**)&g->gd, sizeof(uint64_t) * n));
    PG_CUDA_TRY(ctx, A((void**)&g->gd32, sizeof(uint32_t) * n));
    PG_CUDA_TRY(ctx, A((void**)&g->kind, n));
    PG_CUDA_TRY(ctx, A((void**)&g->plist, sizeof(int32_t) * n));
    PG_CUDA_TRY(ctx, A((void**)&g->slot, sizeof(int32_t) * n));
    PG_CUDA_TRY(ctx, A((void**)&g->ccnt, sizeof(int32_t) * (n + 1)));
    PG_CUDA_TRY(ctx, A((void**)&g->coff, sizeof(int32_t) * (n + 2)));
    PG_CUDA_TRY(ctx, A((void**)&g->cl_ks, sizeof(int2) * n));
    PG_CUDA_TRY(ctx, A((void**)&g->sz, sizeof(int32_t) * n));
    PG_CUDA_TRY(ctx, A((void**)&g->sinkval, sizeof(int32_t) * n));
    PG_CUDA_TRY(ctx, A((void**)&g->wgt, sizeof(int32_t) * n));
    PG_CUDA_TRY(ctx, A((void**)&g->oddsz, sizeof(int32_t) * n));
    PG_CUDA_TRY(ctx, A((void**)&g->key, sizeof(int32_t) * n));
    PG_CUDA_TRY(ctx, A((void**)&g->cls, n));
    PG_CUDA_TRY(ctx, A((void**)&g->depth, sizeof(int32_t) * n));
    PG_CUDA_TRY(ctx, A((void**)&g->dom, sizeof(int32_t) * n));
    PG_CUDA_TRY(ctx, A((void**)&g->hugelist, sizeof(int32_t) * n));
    g->ntiles = std::max<int64_t>(1, (n + kCoopTile - 1) / kCoopTile);
    PG_CUDA_TRY(ctx, A((void**)&g->tiles, sizeof(int64_t) * (2 * g->ntiles + 2)));
    PG_CUDA_TRY(ctx, A((void**)&g->tsum, sizeof(int64_t) * (2 * g->ntiles + 2)));
    PG_CUDA_TRY(ctx, A((void**)&g->gscan, sizeof(int64_t) * 3 * (size_t)g->ngames));
    PG_CUDA_TRY(ctx, A((void**)&g->gst, sizeof(GameState) * (size_t)g->ngames));
    PG_CUDA_TRY(ctx, A((void**)&g->gactive, 2 * sizeof(int32_t)));
    PG_CUDA_TRY(ctx, A((void**)&g->loop_iters, sizeof(int64_t)));
    PG_CUDA_TRY(ctx, A((void**)&g->cnt, sizeof(Counters)));
    PG_CUDA_TRY(ctx, cudaMallocHost((void**)&g->hcnt, sizeof(Counters)));
    g->scan_tmp_bytes = scan_tmp_bytes(n + 2) + 64;
    PG_CUDA_TRY(ctx, A(&g->scan_tmp, g->scan_tmp_bytes));
    pg_status st = coop_blocks_for(ctx, &g->coop_blocks);
    if (st) return st;
    st = chain1_blocks_for(ctx, &g->chain1_blocks);
    if (st) return st;
    if (g->cv) {
        pg_status st2 = alloc_cv(g);
        if (st2) return st2;
    }
    for (int i = 0; i < 4; ++i) PG_CUDA_TRY(ctx, cudaEventCreate(&g->ev[i]));
    for (int i = 0; i < 2 * KID_COUNT; ++i) PG_CUDA_TRY(ctx, cudaEventCreate(&g->kev[i]));
    return reset_scratch(g);
}

pg_status coop_blocks_for(pg_ctx* ctx, int* out) {
    int sms = 0, a = 0, b = 0;
    PG_CUDA_TRY(ctx, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device));
    PG_CUDA_TRY(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_jump_coop, kBlock, 0));
    PG_CUDA_TRY(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_idscan_coop, kBlock, 0));
    int c = 0;
    PG_CUDA_TRY(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&c, k_jump32_coop, kBlock, 0));
    *out = sms * std::max(1, std::min(std::min(std::min(a, b), c), 4));
    return PG_OK;
}

// k_chain1 runs as one wave of resident blocks whose warps stride over the
// tiles: the walks' lengths vary, and a warp with many tiles averages them out,
// where one tile per warp would hold each block until its longest walk ends.
pg_status chain1_blocks_for(pg_ctx* ctx, int* out) {
    int sms = 0, a = 0;
    PG_CUDA_TRY(ctx, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device));
    PG_CUDA_TRY(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_chain1, kBlock, 0));
    *out = sms * std::max(1, a);
    return PG_OK;
}

pg_status reset_scratch(pg_game* g) {
    pg_ctx* ctx = g->ctx;
    g->deep_mode = false;  // every call starts on the default path; a deep g-forest switches it
    g->val_deep = false;
    g->tune = tune_for(ctx, g->n);
    cudaStream_t s = ctx->stream;
    const int64_t n = g->n;
    PG_CUDA_TRY(ctx, cudaMemsetAsync(g->sz, 0, sizeof(int32_t) * n, s));
    PG_CUDA_TRY(ctx, cudaMemsetAsync(g->oddsz, 0, sizeof(int32_t) * n, s));
    PG_CUDA_TRY(ctx, cudaMemsetAsync(g->ccnt, 0, sizeof(int32_t) * (n + 1), s));
    PG_CUDA_TRY(ctx, cudaMemsetAsync(g->tsum, 0, sizeof(int64_t) * (2 * g->ntiles + 2), s));
    return reset_games(g);
}

pg_status reset_games(pg_game* g) {
    pg_ctx* ctx = g->ctx;
    PG_CUDA_TRY(ctx, cudaMemsetAsync(g->gst, 0, sizeof(GameState) * (size_t)g->ngames, ctx->stream));
    return PG_OK;
}

pg_status enqueue_k1(pg_game* g) {
    pg_ctx* ctx = g->ctx;
    cudaStream_t s = ctx->stream;
    int32_t n = g->n;
    Counters* c = g->cnt;
    PG_CUDA_TRY(ctx, cudaMemsetAsync(c, 0, sizeof(Counters), s));
    prof_begin(g, KID_WALK);
    {
        auto walk = k_walk<kWalkCap>;
        switch (g->tune.walk_cap) {
            case 16: walk = k_walk<16>; break;
            case 32: walk = k_walk<32>; break;
            case 128: walk = k_walk<128>; break;
            default: break;
        }
        walk<<<ilp_grid(n), kBlock, 0, s>>>(n, g->strat, g->flags, g->vgame, g->gsink, g->sink0, g->gd, g->gd32,
                                            g->plist, g->sz, g->oddsz, c, &c->n_pending);
    }
    prof_end(g, KID_WALK, 1);
    {
        int32_t cap = 64;
        for (int64_t x = n; x > 1; x >>= 1) cap += 2;
        // on the ruling-set path the rounds may run much longer (long increasing runs below pending walks)
        int cap_deep = (ctx->deep_fallback && !g->deep_mode) ? 1 : 0;
        if (g->deep_mode) cap += kJumpRoundsDeep;
        void* args[] = {(void*)&g->plist, (void*)&g->gd,    (void*)&g->gd32, (void*)&g->vgame,
                        (void*)&g->gsink, (void*)&g->sink0, (void*)&c,       (void*)&cap, (void*)&cap_deep};
        prof_begin(g, KID_JUMP);
        PG_CUDA_TRY(ctx, cudaLaunchCooperativeKernel((void*)k_jump_coop, g->coop_blocks, kBlock, args, 0, s));
        prof_end(g, KID_JUMP, 1);
    }
    PG_CUDA_TRY(ctx, cudaGetLastError());
    return PG_OK;
}

pg_status enqueue_valuation(pg_game* g, bool want_dom) {
    if (g->cv) return enqueue_valuation_cv(g, want_dom);
    if (g->deep_mode) return enqueue_valuation_deep(g, want_dom);
    g->val_deep = false;
    pg_ctx* ctx = g->ctx;
    cudaStream_t s = ctx->stream;
    int32_t n = g->n;
    Counters* c = g->cnt;
    const unsigned grid = grid_for(n);
    // K1: walks here are short but for a few, one pass of kWalkCap steps straight into the jumping list
    pg_status st1 = enqueue_k1(g);
    if (st1) return st1;
    prof_begin(g, KID_CHAIN1);
    // one wave of resident blocks for a single game; packed games (batches, servers) keep one block per 8 tiles,
    // which measured faster there (4,096-game batch: 5.95 s of loop against 6.52 s)
    const unsigned c1grid =
        (g->chain1_blocks > 0 && !g->vgame) ? std::min(ilp_grid(n), (unsigned)g->chain1_blocks) : ilp_grid(n);
    k_chain1<<<c1grid, kBlock, 0, s>>>(n, g->gd32, g->flags, g->pri, g->sz, g->ccnt, g->slot, g->kind, g->cls,
                                       g->dom, want_dom ? 1 : 0, g->vgame, g->gst, c, g->tune.deep_cut);
    prof_end(g, KID_CHAIN1, 1);
    prof_begin(g, KID_CSCAN);
    PG_CUDA_TRY(ctx, exclusive_scan_i32(g->ccnt, g->coff, (int64_t)n + 1, nullptr, g->scan_tmp, g->scan_tmp_bytes, s));
    prof_end(g, KID_CSCAN, 3);
    prof_begin(g, KID_SCATTER);
    k_scatter<<<ilp_grid(n), kBlock, 0, s>>>(n, g->gd32, g->kind, g->sz, g->coff, g->slot, g->ccnt, g->cl_ks, g->sinkval,
                                             g->tsum, c);
    prof_end(g, KID_SCATTER, 1);
    prof_begin(g, KID_SIBLINGS);
    k_siblings<<<grid, kBlock, 0, s>>>(n, g->coff, g->cl_ks, g->wgt, g->oddsz, g->plist, g->hugelist, c);
    k_big_parents<<<g->coop_blocks, kBlock, 0, s>>>(g->coff, g->cl_ks, g->plist, g->wgt, g->oddsz, c);
    prof_end(g, KID_SIBLINGS, 2);
    prof_begin(g, KID_SINKSCAN);
    {
        int64_t ntiles = g->ntiles;
        void* args[] = {(void*)&n,        (void*)&g->gd32,   (void*)&g->sz,  (void*)&g->kind,  (void*)&g->hugelist,
                        (void*)&g->tiles, (void*)&ntiles,    (void*)&g->wgt, (void*)&g->oddsz, (void*)&c};
        PG_CUDA_TRY(ctx, cudaLaunchCooperativeKernel((void*)k_idscan_coop, g->coop_blocks, kBlock, args, 0, s));
        // one game whose sink slot is its last id: the tile scan ranks the sink itself
        const bool single = g->ngames == 1 && !g->vgame && g->sink0 == n - 1;
        k_tiles_scan<<<1, kTileScanThreads, 0, s>>>(g->tsum, g->tiles, g->ntiles, single ? g->sink0 : -1, g->gscan,
                                                    g->key, c);
        if (!single) {
            const unsigned gp = (unsigned)std::max<int64_t>(1, std::min<int64_t>(((int64_t)g->ngames + 7) / 8, 4096));
            k_game_prefix<<<gp, kBlock, 0, s>>>(n, g->ngames, g->gsink, g->sinkval, g->tiles, g->gscan, g->key, c);
        }
        k_sink_apply<<<(unsigned)g->ntiles, kBlock, 0, s>>>(n, g->sinkval, g->tiles, g->vgame, g->gscan, g->wgt, c);
        prof_end(g, KID_SINKSCAN, single ? 3 : 4);
    }
    prof_begin(g, KID_CHAIN2);
    k_chain2<<<ilp_grid(n), kBlock, 0, s>>>(n, g->gd32, g->kind, g->wgt, g->oddsz, g->key, c);
    prof_end(g, KID_CHAIN2, 1);
    PG_CUDA_TRY(ctx, cudaGetLastError());
    return PG_OK;
}

pg_status enqueue_depth(pg_game* g) {
    if (g->val_deep) return PG_OK;  // the ruling-set path wrote the depths with the ranks
    pg_ctx* ctx = g->ctx;
    ctx->launches += 1;
    k_depth<<<grid_for(g->n), kBlock, 0, ctx->stream>>>(g->n, g->gd, g->kind, g->depth, g->cnt);
    PG_CUDA_TRY(ctx, cudaGetLastError());
    return PG_OK;
}

pg_status enqueue_switch(pg_game* g, int player) {
    if (g->cv) return enqueue_switch_cv(g, player);
    pg_ctx* ctx = g->ctx;
    cudaStream_t s = ctx->stream;
    PG_CUDA_TRY(ctx, cudaMemsetAsync(&g->cnt->n_switch, 0, sizeof(int32_t), s));
    int kid = player ? KID_SWITCH_ODD : KID_SWITCH_EVEN;
    prof_begin(g, kid);
    if (g->off64)
        k_switch<int64_t><<<grid_for(g->n), kBlock, 0, s>>>(g->n, player, g->off64, g->tgt, g->flags, g->key, g->vgame,
                                                            g->gsink, g->sink0, g->gst, g->strat, g->cnt);
    else
        k_switch<int32_t><<<grid_for(g->n), kBlock, 0, s>>>(g->n, player, g->off, g->tgt, g->flags, g->key, g->vgame,
                                                            g->gsink, g->sink0, g->gst, g->strat, g->cnt);
    prof_end(g, kid, 1);
    PG_CUDA_TRY(ctx, cudaGetLastError());
    return PG_OK;
}

pg_status enqueue_bookkeeping(pg_game* g, int64_t cap, bool even_phase) {
    pg_ctx* ctx = g->ctx;
    cudaStream_t s = ctx->stream;
    PG_CUDA_TRY(ctx, cudaMemsetAsync(g->gactive, 0, 2 * sizeof(int32_t), s));
    ctx->launches += 1;
    const unsigned b = (unsigned)std::max<int64_t>(1, std::min<int64_t>(((int64_t)g->ngames + kBlock - 1) / kBlock, 1024));
    k_bookkeep<<<b, kBlock, 0, s>>>(g->ngames, g->gst, cap, even_phase ? 1 : 0, g->reset_tau ? 1 : 0, g->gactive,
                                    g->cnt);
    PG_CUDA_TRY(ctx, cudaGetLastError());
    return PG_OK;
}

// The Odd marks when the loop compares valuations over the players' views
// (null otherwise: every Odd vertex is evaluated in every pass).
uint8_t* omark_of(const pg_game* g) {
    return g->pl_ok && g->omark && !g->cv && !g->tune.loop_ranks && !g->deep_mode ? g->omark : nullptr;
}

pg_status enqueue_reset(pg_game* g) {
    pg_ctx* ctx = g->ctx;
    cudaStream_t s = ctx->stream;
    ctx->launches += 1;
    if (g->off64)
        k_reset_odd<int64_t><<<grid_for(g->n), kBlock, 0, s>>>(g->n, g->off64, g->tgt, g->flags, g->vgame, g->gst,
                                                               g->strat, g->cnt);
    else
        k_reset_odd<int32_t><<<grid_for(g->n), kBlock, 0, s>>>(g->n, g->off, g->tgt, g->flags, g->vgame, g->gst,
                                                               g->strat, g->cnt);
    PG_CUDA_TRY(ctx, cudaGetLastError());
    return PG_OK;
}

bool loop_compares(const pg_game* g) { return !g->cv && !g->tune.loop_ranks && !g->deep_mode; }

pg_status enqueue_valuation_cmp(pg_game* g) {
    pg_ctx* ctx = g->ctx;
    cudaStream_t s = ctx->stream;
    int32_t n = g->n;
    Counters* c = g->cnt;
    PG_CUDA_TRY(ctx, cudaMemsetAsync(c, 0, sizeof(Counters), s));
    prof_begin(g, KID_WALK);
    {
        const bool batch = g->vgame != nullptr;
        auto walk = batch ? k_walk_cmp<kWalkCap, PG_CHAIN_ILP, true> : k_walk_cmp<kWalkCap, PG_CHAIN_ILP, false>;
        switch (g->tune.walk_cap) {
            case 16: walk = batch ? k_walk_cmp<16, PG_CHAIN_ILP, true> : k_walk_cmp<16, PG_CHAIN_ILP, false>; break;
            case 32: walk = batch ? k_walk_cmp<32, PG_CHAIN_ILP, true> : k_walk_cmp<32, PG_CHAIN_ILP, false>; break;
            case 128: walk = batch ? k_walk_cmp<128, PG_CHAIN_ILP, true> : k_walk_cmp<128, PG_CHAIN_ILP, false>; break;
            default: break;
        }
        walk<<<ilp_grid(n), kBlock, 0, s>>>(n, g->strat, g->flags, g->vgame, g->gsink, g->sink0, g->gd32, g->plist,
                                            &c->n_pending, g->gst);
    }
    prof_end(g, KID_WALK, 1);
    {
        int32_t cap = 64;
        for (int64_t x = n; x > 1; x >>= 1) cap += 2;
        int cap_deep = ctx->deep_fallback ? 1 : 0;
        void* args[] = {(void*)&g->plist, (void*)&g->gd32, (void*)&g->flags, (void*)&g->vgame, (void*)&g->gsink,
                        (void*)&g->sink0, (void*)&c,       (void*)&cap,      (void*)&cap_deep};
        prof_begin(g, KID_JUMP);
        PG_CUDA_TRY(ctx, cudaLaunchCooperativeKernel((void*)k_jump32_coop, g->coop_blocks, kBlock, args, 0, s));
        prof_end(g, KID_JUMP, 1);
    }
    prof_begin(g, KID_CLASSIFY);
    // the top words live in the chain-weight array, which only a full valuation uses
    k_classify<PG_CHAIN_ILP><<<ilp_grid(n), kBlock, 0, s>>>(n, g->gd32, g->flags, (uint32_t*)g->wgt, g->vgame,
                                                            g->gst, c, g->tune.deep_cut, g->rv_off, g->rv_src,
                                                            omark_of(g), g->gactive + 1);
    prof_end(g, KID_CLASSIFY, 1);
    PG_CUDA_TRY(ctx, cudaGetLastError());
    return PG_OK;
}

namespace {
template <int BS>
void launch_switch_cmp_bs(pg_game* g, int player) {
    cudaStream_t s = g->ctx->stream;
    const uint32_t* topw = (const uint32_t*)g->wgt;
    if (g->pl_ok) {  // the player's view
        const int64_t np = g->pl_n[player];
        // one wave of blocks striding over the view: the Even pass returns at once in most iterations, and a
        // grid of one block per BS vertices would spend that time scheduling blocks
        int sms = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, g->device);
        const int64_t wave = (int64_t)std::max(sms, 1) * (2048 / BS);
        const int64_t b = std::max<int64_t>(1, std::min<int64_t>((np + BS - 1) / BS, wave));
        uint8_t* om = player == 1 ? omark_of(g) : nullptr;
        const bool batch = g->vgame != nullptr;
        auto kern = player == 0 ? (batch ? k_switch_cmp_pl<BS, 0, false, true> : k_switch_cmp_pl<BS, 0, false, false>)
                    : om        ? (batch ? k_switch_cmp_pl<BS, 1, true, true> : k_switch_cmp_pl<BS, 1, true, false>)
                                : (batch ? k_switch_cmp_pl<BS, 1, false, true> : k_switch_cmp_pl<BS, 1, false, false>);
        kern<<<(unsigned)b, BS, 0, s>>>((int32_t)np, g->pl_vid[player], g->pl_off[player], g->pl_tgt[player],
                                        g->flags, g->gd32, topw, g->vgame, g->gsink, g->sink0, g->gst, g->strat,
                                        g->cnt, om, g->gactive + 1);
        return;
    }
    const int64_t b = std::max<int64_t>(1, std::min<int64_t>(((int64_t)g->n + BS - 1) / BS, 152LL * 64 * kBlock / BS));
    if (g->off64)
        k_switch_cmp<int64_t, BS><<<(unsigned)b, BS, 0, s>>>(g->n, player, g->off64, g->tgt, g->flags, g->gd32, topw,
                                                             g->vgame, g->gsink, g->sink0, g->gst, g->strat, g->cnt);
    else
        k_switch_cmp<int32_t, BS><<<(unsigned)b, BS, 0, s>>>(g->n, player, g->off, g->tgt, g->flags, g->gd32, topw,
                                                             g->vgame, g->gsink, g->sink0, g->gst, g->strat, g->cnt);
}

void launch_switch_cmp(pg_game* g, int player, int bs) {
    if (bs == 128) launch_switch_cmp_bs<128>(g, player);
    else if (bs == 512) launch_switch_cmp_bs<512>(g, player);
    else launch_switch_cmp_bs<256>(g, player);
}
}  // namespace

pg_status enqueue_switch_cmp(pg_game* g, int player) {
    pg_ctx* ctx = g->ctx;
    cudaStream_t s = ctx->stream;
    PG_CUDA_TRY(ctx, cudaMemsetAsync(&g->cnt->n_switch, 0, sizeof(int32_t), s));
    int kid = player ? KID_SWITCH_ODD : KID_SWITCH_EVEN;
    prof_begin(g, kid);
    launch_switch_cmp(g, player, g->tune.switch_block);
    prof_end(g, kid, 1);
    PG_CUDA_TRY(ctx, cudaGetLastError());
    return PG_OK;
}

pg_status finish_loop(pg_game* g) {
    if (!g->last_cmp) return PG_OK;
    pg_status st = full_valuation(g, false);
    if (!st) g->last_cmp = false;
    return st;
}

pg_status full_valuation(pg_game* g, bool want_dom) {
    pg_status st = enqueue_valuation(g, want_dom);
    if (!st) st = sync_counters(g);
    if (st || g->cv || g->val_deep || !g->hcnt->deep) return st;
    g->deep_mode = true;  // a chain walk passed the cutover: the ruling-set path, for the rest of the call
    st = enqueue_valuation_deep(g, want_dom);
    if (!st) st = sync_counters(g);
    return st;
}

pg_status build_player_split(pg_game* g) {
    if (g->pl_ok || g->cv) return PG_OK;
    pg_ctx* ctx = g->ctx;
    cudaStream_t s = ctx->stream;
    const int32_t n = g->n;
    const unsigned grid = grid_for(n);
    drop_loop_graphs(g);  // captured loops hold the old views' addresses
    for (int p = 0; p < 2; ++p) {
        if (g->pl_vid[p]) cudaFreeAsync(g->pl_vid[p], s);
        if (g->pl_off[p]) cudaFreeAsync(g->pl_off[p], s);
        if (g->pl_tgt[p]) cudaFreeAsync(g->pl_tgt[p], s);
        g->pl_vid[p] = g->pl_off[p] = g->pl_tgt[p] = nullptr;
    }
    for (void** q : {(void**)&g->rv_off, (void**)&g->rv_src, (void**)&g->omark}) {
        if (*q) cudaFreeAsync(*q, s);
        *q = nullptr;
    }
    int32_t mp_of[2] = {0, 0};
    // the valuation's scratch is free before a loop: marks in kind and cls, positions in coff, degrees in
    // hugelist
    uint8_t* mark[2] = {g->kind, g->cls};
    k_pl_mark<<<grid, kBlock, 0, s>>>(n, g->flags, mark[0], mark[1]);
    PG_CUDA_TRY(ctx, cudaGetLastError());
    int32_t* host = ctx->pinned;
    for (int p = 0; p < 2; ++p) {
        PG_CUDA_TRY(ctx, exclusive_scan_u8(mark[p], g->coff, n, g->scan_tmp, g->scan_tmp_bytes, s));
        PG_CUDA_TRY(ctx, cudaMemcpyAsync(host, g->coff + n, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        PG_CUDA_TRY(ctx, cudaStreamSynchronize(s));
        const int32_t np = host[0];
        g->pl_n[p] = np;
        PG_CUDA_TRY(ctx, dev_alloc(ctx, (void**)&g->pl_vid[p], sizeof(int32_t) * std::max(np, 1), s));
        PG_CUDA_TRY(ctx, dev_alloc(ctx, (void**)&g->pl_off[p], sizeof(int32_t) * ((size_t)np + 1), s));
        if (g->off64) k_pl_gather<int64_t><<<grid, kBlock, 0, s>>>(n, mark[p], g->coff, g->off64, g->pl_vid[p], g->hugelist);
        else k_pl_gather<int32_t><<<grid, kBlock, 0, s>>>(n, mark[p], g->coff, g->off, g->pl_vid[p], g->hugelist);
        // the view's offsets are 32-bit: the player's edges must number fewer than 2^31 (the scan's total is 64-bit)
        int64_t* total = g->loop_iters;  // free before a loop
        PG_CUDA_TRY(ctx, exclusive_scan_i32(g->hugelist, g->pl_off[p], np, total, g->scan_tmp, g->scan_tmp_bytes, s));
        PG_CUDA_TRY(ctx, cudaMemcpyAsync(host + 2, total, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        PG_CUDA_TRY(ctx, cudaStreamSynchronize(s));
        int64_t mp64 = 0;
        memcpy(&mp64, host + 2, sizeof(int64_t));
        if (mp64 > INT32_MAX - 1) {  // too many for the view: the unsplit passes, as before any view
            for (int q = 0; q < 2; ++q) {
                if (g->pl_vid[q]) cudaFreeAsync(g->pl_vid[q], s);
                if (g->pl_off[q]) cudaFreeAsync(g->pl_off[q], s);
                if (g->pl_tgt[q]) cudaFreeAsync(g->pl_tgt[q], s);
                g->pl_vid[q] = g->pl_off[q] = g->pl_tgt[q] = nullptr;
            }
            return PG_OK;
        }
        const int32_t mp = (int32_t)mp64;
        mp_of[p] = mp;
        PG_CUDA_TRY(ctx, dev_alloc(ctx, (void**)&g->pl_tgt[p], sizeof(int32_t) * std::max(mp, 1), s));
        if (g->off64)
            k_pl_copy<int64_t><<<grid_for(std::max(np, 1)), kBlock, 0, s>>>(np, g->pl_vid[p], g->off64, g->tgt,
                                                                            g->pl_off[p], g->pl_tgt[p]);
        else
            k_pl_copy<int32_t><<<grid_for(std::max(np, 1)), kBlock, 0, s>>>(np, g->pl_vid[p], g->off, g->tgt,
                                                                            g->pl_off[p], g->pl_tgt[p]);
        PG_CUDA_TRY(ctx, cudaGetLastError());
    }
    ctx->launches += 7;
    {  // Odd's reverse view, counted in hugelist (free again)
        const int32_t np = (int32_t)g->pl_n[1];
        int32_t* cnt = g->hugelist;
        PG_CUDA_TRY(ctx, dev_alloc(ctx, (void**)&g->rv_off, sizeof(int32_t) * ((size_t)n + 1), s));
        PG_CUDA_TRY(ctx, dev_alloc(ctx, (void**)&g->rv_src, sizeof(int32_t) * std::max(mp_of[1], 1), s));
        const size_t mark_bytes = ((size_t)np + 16) & ~(size_t)15;  // read 16 at a time, the padding zero
        PG_CUDA_TRY(ctx, dev_alloc(ctx, (void**)&g->omark, mark_bytes, s));
        PG_CUDA_TRY(ctx, cudaMemsetAsync(g->omark, 0, mark_bytes, s));
        PG_CUDA_TRY(ctx, cudaMemsetAsync(cnt, 0, sizeof(int32_t) * (size_t)n, s));
        k_rv_count<<<grid_for(std::max(mp_of[1], 1)), kBlock, 0, s>>>(np, g->pl_off[1], g->pl_tgt[1], cnt);
        PG_CUDA_TRY(ctx, exclusive_scan_i32(cnt, g->rv_off, n, nullptr, g->scan_tmp, g->scan_tmp_bytes, s));
        PG_CUDA_TRY(ctx, cudaMemcpyAsync(cnt, g->rv_off, sizeof(int32_t) * (size_t)n, cudaMemcpyDeviceToDevice, s));
        k_rv_fill<<<grid_for(std::max(np, 1)), kBlock, 0, s>>>(np, g->pl_off[1], g->pl_tgt[1], cnt, g->rv_src);
        PG_CUDA_TRY(ctx, cudaGetLastError());
        ctx->launches += 5;
    }
    g->pl_ok = true;
    return PG_OK;
}

pg_status sync_counters(pg_game* g) {
    pg_ctx* ctx = g->ctx;
    cudaStream_t s = ctx->stream;
    PG_CUDA_TRY(ctx, cudaMemcpyAsync(g->hcnt, g->cnt, sizeof(Counters), cudaMemcpyDeviceToHost, s));
    PG_CUDA_TRY(ctx, cudaStreamSynchronize(s));
    prof_collect(g);
    if (g->hcnt->err & kErrBarrier) return fail(ctx, PG_ECUDA, "valuation: a grid barrier timed out");
    if (g->hcnt->err & kErrJumpRounds) return fail(ctx, PG_ECUDA, "valuation: pointer jumping did not converge");
    if (g->hcnt->err & kErrRulers) return fail(ctx, PG_ECUDA, "valuation: the ruling-set list ranking failed");
    return PG_OK;
}

}  // namespace pg
