// Ranks of a deep g-forest: an Euler tour ranked by a sparse ruling set.
//
// The default valuation ranks through the nearest-greater forest (g-forest)
// by walking every vertex's g-chain (pg_iter.cu), which costs the chain's
// length per vertex: cheap when plays rise only a few times (random
// priorities), quadratic when they climb long increasing runs (an n-vertex
// path with increasing priorities has g-chains of every length up to n).
// When a chain walk exceeds the cutover depth (the context's deep_cut), the
// game switches to this path, which does the same job in work linear in n:
//
//   D1 roots of the g-forest by pointer jumping (class, dominant priority,
//      odd cycles; children counts for the segments);
//   D2 children of every finite vertex in one segment each, sorted by the
//      order of Section 3 (odd children, larger first, then even children,
//      smaller first); the children of a game's sink come in id order from
//      two stable compactions (odd, even);
//   D3 the Euler tour of every game's g-tree as a linked list of 2 elements
//      per vertex (enter, exit), with weights: one visit where the in-order
//      reaches the vertex (after its odd children), and the vertex's walk
//      length on entering and its negation on exiting (for the depth);
//   D4 list ranking by a sparse ruling set (Section 5 ranks its Euler-tour
//      list with Helman-JaJa splitters): about one element in ruler_stride is
//      a ruler (plus every list head), each ruler walks its sublist summing
//      weights, the rulers' sums are ranked by pointer jumping over the short
//      list of rulers, and every element adds its ruler's prefix;
//   D5 rank = visits before the vertex's visit, depth = the depth channel at
//      its entry, as the default valuation defines them.
//
// Nothing here walks a g-chain, so no step depends on the forest's depth
// beyond the logarithmic rounds of D1.
#include "pg_device.cuh"

namespace pg {
namespace {

// ---------------------------------------------------------------------------
// D1: roots. A root is a vertex whose g-word ends its chain: a child of the
// sink (bit 30, finite) or a vertex above its whole infinite future (bit 31,
// TOP); sink slots are inert roots. anc[v] starts at g(v) and jumps
// (anc[v] = anc[anc[v]]) until it is a root. Also clears the children counts.
__global__ void __launch_bounds__(kBlock) k_deep_init(int32_t n, const uint32_t* __restrict__ gd32,
                                                      const uint8_t* __restrict__ flags, int32_t* __restrict__ anc,
                                                      int32_t* __restrict__ ccnt, int32_t* __restrict__ dlist,
                                                      int32_t* __restrict__ vis, Counters* cnt) {
    if (cnt->err) return;
    for (int64_t v0 = (int64_t)blockIdx.x * blockDim.x; v0 < n; v0 += (int64_t)gridDim.x * blockDim.x) {
        const int32_t v = (int32_t)(v0 + threadIdx.x);
        bool nonroot = false;
        if (v < n) {
            const uint32_t w = (flags[v] & kSinkSlot) ? kG32Sink : gd32[v];
            const bool root = (w & (kG32None | kG32Sink)) != 0;
            anc[v] = root ? v : g32_ptr(w);
            nonroot = !root;
            ccnt[v] = 0;
            vis[v] = -1;
        }
        const int32_t at = warp_append(nonroot, &cnt->n_dlist);
        if (nonroot) dlist[at] = v;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) ccnt[n] = 0;
}

// Pointer jumping towards the roots, all rounds in one cooperative launch.
// In-place updates are safe: anc only moves up the vertex's own g-chain.
// Rounds stop when a round changes nothing (about log2 of the depth) or at
// the cap (kErrJumpRounds).
__global__ void __launch_bounds__(kBlock) k_deep_anc_coop(const int32_t* __restrict__ dlist, int32_t* anc,
                                                          Counters* cnt, int32_t cap) {
    if (cnt->err) return;
    const int32_t nl = cnt->n_dlist;
    for (int32_t r = 0;; ++r) {
        if (blockIdx.x == 0 && threadIdx.x == 0) cnt->left[(r + 1) % 3] = 0;
        int32_t changed = 0;
        for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < nl; i += gridDim.x * blockDim.x) {
            const int32_t v = dlist[i];
            const int32_t a = __ldcg(anc + v);
            const int32_t aa = __ldcg(anc + a);
            if (aa != a) {
                __stcg(anc + v, aa);
                ++changed;
            }
        }
        block_add(changed, &cnt->left[r % 3]);
        if (!grid_sync(cnt)) return;
        const int32_t rem = *(volatile int32_t*)&cnt->left[r % 3];
        if (rem == 0) {
            if (blockIdx.x == 0 && threadIdx.x == 0) cnt->deep_rounds = r + 1;
            return;
        }
        if (r + 1 >= cap) {
            if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(&cnt->err, kErrJumpRounds);
            return;
        }
    }
}

// kind bits (as the default valuation's first chain pass writes them)
constexpr uint8_t kDFin = 1, kDSinkChild = 2, kDOdd = 4, kDSinkSlot = 8;

// Class of every vertex from its root; finite vertices below a vertex parent
// take a slot among its children; sink children are flagged by parity for the
// two id-ordered compactions of the sink's children.
__global__ void __launch_bounds__(kBlock) k_deep_classify(int32_t n, const uint32_t* __restrict__ gd32,
                                                          const uint8_t* __restrict__ flags,
                                                          const int32_t* __restrict__ pri,
                                                          const int32_t* __restrict__ anc, int32_t* ccnt,
                                                          int32_t* __restrict__ slot, uint8_t* __restrict__ kind,
                                                          uint8_t* __restrict__ cls, int32_t* __restrict__ dom,
                                                          int want_dom, uint8_t* __restrict__ sc_odd,
                                                          uint8_t* __restrict__ sc_even,
                                                          const int32_t* __restrict__ vgame, GameState* gst,
                                                          Counters* cnt) {
    if (cnt->err) return;
    int32_t nfin = 0, nodd = 0;
    for (int32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        const uint8_t f = flags[v];
        uint8_t so = 0, se = 0;
        if (f & kSinkSlot) {
            kind[v] = kDSinkSlot;
            cls[v] = kFin;
            if (want_dom) dom[v] = -1;
        } else {
            const uint32_t w = gd32[v];
            const uint32_t wr = gd32[anc[v]];
            if (g32_none(wr)) {
                const int32_t cyc = g32_ptr(wr);  // the cycle's maximum
                const bool odd = (flags[cyc] & kPriOdd) != 0;
                kind[v] = 0;
                cls[v] = odd ? kOddCycle : kTop;
                if (want_dom) dom[v] = pri[cyc];
                if (odd) {
                    ++nodd;
                    atomicAdd(&gst[vgame ? vgame[v] : 0].nodd, 1);
                }
            } else {
                const bool sinkchild = g32_sink(w);
                const bool odd_v = (f & kPriOdd) != 0;
                kind[v] = kDFin | (sinkchild ? kDSinkChild : 0) | (odd_v ? kDOdd : 0);
                cls[v] = kFin;
                if (want_dom) dom[v] = -1;
                ++nfin;
                if (sinkchild) {
                    so = odd_v ? 1 : 0;
                    se = odd_v ? 0 : 1;
                } else {
                    slot[v] = atomicAdd(ccnt + g32_ptr(w), 1);
                }
            }
        }
        sc_odd[v] = so;
        sc_even[v] = se;
    }
    block_add(nfin, &cnt->n_fin);
    block_add(nodd, &cnt->n_odd);
}

// ---------------------------------------------------------------------------
// D2: segments. Sort key of a child c inside its parent's segment, ascending
// in the order of Section 3: odd children by decreasing id, then even ones by
// increasing id (ids are below 2^30).
__device__ inline uint32_t tkey(int32_t c, const uint8_t* __restrict__ flags) {
    return (flags[c] & kPriOdd) ? (0x3fffffffu - (uint32_t)c) : (0x40000000u + (uint32_t)c);
}
__device__ inline bool tkey_odd(uint32_t k) { return k < 0x40000000u; }

// Finite children of vertex parents into their segments (at the slots taken
// in k_deep_classify), the sink's children into two id-ordered lists (odd,
// even) at their compaction positions; clears the children counts.
__global__ void __launch_bounds__(kBlock) k_deep_scatter(int32_t n, const uint32_t* __restrict__ gd32,
                                                         const uint8_t* __restrict__ kind,
                                                         const int32_t* __restrict__ coff,
                                                         const int32_t* __restrict__ slot,
                                                         const uint8_t* __restrict__ sc_odd,
                                                         const uint8_t* __restrict__ sc_even,
                                                         const int32_t* __restrict__ podd,
                                                         const int32_t* __restrict__ peven, int32_t* __restrict__ seg,
                                                         int32_t* __restrict__ oddL, int32_t* __restrict__ evenL,
                                                         const Counters* cnt) {
    if (cnt->err) return;
    for (int32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        const uint8_t kd = kind[v];
        if (!(kd & kDFin)) continue;
        if (kd & kDSinkChild) {
            if (sc_odd[v]) oddL[podd[v]] = v;
            if (sc_even[v]) evenL[peven[v]] = v;
        } else {
            seg[coff[g32_ptr(gd32[v])] + slot[v]] = v;
        }
    }
}

// Sorts the segments of up to kDSmall children in registers (one thread per
// parent); larger segments are queued: up to kDBlock children for a
// shared-memory sort (one block each), beyond for a radix sort in global
// memory (one block each).
constexpr int kDSmall = 16;
constexpr int kDBlock = 4096;

__global__ void __launch_bounds__(kBlock) k_deep_sort_small(int32_t n, const int32_t* __restrict__ coff,
                                                            const uint8_t* __restrict__ flags, int32_t* seg,
                                                            int32_t* __restrict__ midlist, int32_t* __restrict__ biglist,
                                                            Counters* cnt) {
    if (cnt->err) return;
    for (int32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
        const int32_t a = coff[p], k = coff[p + 1] - a;
        if (k <= 1) continue;
        if (k > kDBlock) {
            biglist[atomicAdd(&cnt->n_dbig, 1)] = p;
            continue;
        }
        if (k > kDSmall) {
            midlist[atomicAdd(&cnt->n_dmid, 1)] = p;
            continue;
        }
        uint32_t key[kDSmall];
        int32_t val[kDSmall];
#pragma unroll
        for (int i = 0; i < kDSmall; ++i) {
            if (i < k) {
                val[i] = seg[a + i];
                key[i] = tkey(val[i], flags);
            }
        }
        // insertion sort (k <= 16)
        for (int i = 1; i < k; ++i) {
            const uint32_t ki = key[i];
            const int32_t vi = val[i];
            int j = i - 1;
            while (j >= 0 && key[j] > ki) {
                key[j + 1] = key[j];
                val[j + 1] = val[j];
                --j;
            }
            key[j + 1] = ki;
            val[j + 1] = vi;
        }
        for (int i = 0; i < k; ++i) seg[a + i] = val[i];
    }
}

// One block per queued segment of kDSmall < k <= kDBlock children: bitonic
// sort of (key, child) pairs in shared memory.
__global__ void __launch_bounds__(kBlock) k_deep_sort_mid(const int32_t* __restrict__ coff,
                                                          const uint8_t* __restrict__ flags, int32_t* seg,
                                                          const int32_t* __restrict__ midlist, const Counters* cnt) {
    if (cnt->err) return;
    __shared__ uint32_t sk[kDBlock];
    __shared__ int32_t sv[kDBlock];
    const int32_t nm = cnt->n_dmid;
    for (int32_t b = blockIdx.x; b < nm; b += gridDim.x) {
        const int32_t p = midlist[b];
        const int32_t a = coff[p], k = coff[p + 1] - a;
        int p2 = 1;
        while (p2 < k) p2 <<= 1;
        for (int i = threadIdx.x; i < p2; i += blockDim.x) {
            if (i < k) {
                sv[i] = seg[a + i];
                sk[i] = tkey(sv[i], flags);
            } else {
                sv[i] = -1;
                sk[i] = 0xffffffffu;
            }
        }
        __syncthreads();
        for (int kk = 2; kk <= p2; kk <<= 1) {
            for (int j = kk >> 1; j > 0; j >>= 1) {
                for (int i = threadIdx.x; i < p2; i += blockDim.x) {
                    const int ixj = i ^ j;
                    if (ixj > i) {
                        const bool up = (i & kk) == 0;
                        if ((sk[i] > sk[ixj]) == up) {
                            const uint32_t tk = sk[i];
                            sk[i] = sk[ixj];
                            sk[ixj] = tk;
                            const int32_t tv = sv[i];
                            sv[i] = sv[ixj];
                            sv[ixj] = tv;
                        }
                    }
                }
                __syncthreads();
            }
        }
        for (int i = threadIdx.x; i < k; i += blockDim.x) seg[a + i] = sv[i];
        __syncthreads();
    }
}

// One block per queued segment of more than kDBlock children: a stable
// least-significant-digit radix sort of the segment by its sort key, four
// passes of 8 bits between the segment and a scratch copy (seg2), the result
// back in seg. Stability inside each chunk of blockDim elements: ranks among
// equal digits within a warp from __match_any_sync, across the warps of the
// chunk from per-warp digit counts in shared memory.
__global__ void __launch_bounds__(kBlock) k_deep_sort_big(const int32_t* __restrict__ coff,
                                                          const uint8_t* __restrict__ flags, int32_t* seg,
                                                          int32_t* seg2, const int32_t* __restrict__ biglist,
                                                          const Counters* cnt) {
    if (cnt->err) return;
    constexpr int kW = kBlock / 32;
    __shared__ int32_t base[256];
    __shared__ int32_t wcnt[kW][257];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    const int32_t nb = cnt->n_dbig;
    for (int32_t b = blockIdx.x; b < nb; b += gridDim.x) {
        const int32_t p = biglist[b];
        const int32_t a = coff[p], k = coff[p + 1] - a;
        int32_t* src = seg + a;
        int32_t* dst = seg2 + a;
        for (int pass = 0; pass < 4; ++pass) {
            const int shift = 8 * pass;
            for (int d = threadIdx.x; d < 256; d += blockDim.x) base[d] = 0;
            __syncthreads();
            for (int32_t i = threadIdx.x; i < k; i += blockDim.x)
                atomicAdd(&base[(tkey(src[i], flags) >> shift) & 255u], 1);
            __syncthreads();
            if (threadIdx.x == 0) {
                int32_t run = 0;
                for (int d = 0; d < 256; ++d) {
                    const int32_t c = base[d];
                    base[d] = run;
                    run += c;
                }
            }
            __syncthreads();
            for (int32_t c0 = 0; c0 < k; c0 += blockDim.x) {
                for (int d = threadIdx.x; d < kW * 257; d += blockDim.x) (&wcnt[0][0])[d] = 0;
                __syncthreads();
                const int32_t i = c0 + threadIdx.x;
                const int32_t val = i < k ? src[i] : -1;
                const uint32_t dig = i < k ? ((tkey(val, flags) >> shift) & 255u) : 256u;
                const unsigned same = __match_any_sync(kFull, dig);
                const int32_t lrank = __popc(same & lt);
                if (lrank == 0) wcnt[wid][dig] = __popc(same);
                __syncthreads();
                if (i < k) {
                    int32_t before = 0;
                    for (int w = 0; w < wid; ++w) before += wcnt[w][dig];
                    dst[base[dig] + before + lrank] = val;
                }
                __syncthreads();
                for (int d = threadIdx.x; d < 256; d += blockDim.x) {
                    int32_t t = 0;
                    for (int w = 0; w < kW; ++w) t += wcnt[w][d];
                    base[d] += t;
                }
                __syncthreads();
            }
            int32_t* t = src;
            src = dst;
            dst = t;
        }
        // four passes: the sorted segment is back in seg
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// D3: the Euler tour. Element 2v enters v, 2v+1 leaves it; a game's list
// starts at its sink slot's enter element and ends at its exit element. Each
// element carries (visits, depth): the in-order visit of a vertex sits on its
// enter element when it has no odd children, else on the exit element of its
// last odd child; the depth channel adds the vertex's walk length (its
// distance to g(v) on the play) on entering and removes it on leaving.
__device__ inline int32_t walk_len(const uint64_t* __restrict__ gd, int32_t v) { return (int32_t)gd_dist(gd[v]); }

// Every finite vertex as a parent: its enter element links to its first child
// in order (or to its own exit element), its exit element starts with the
// depth weight only; clears the children counts for the next valuation.
__global__ void __launch_bounds__(kBlock) k_deep_links_parent(int32_t n, const uint8_t* __restrict__ kind,
                                                              const uint8_t* __restrict__ flags,
                                                              const uint64_t* __restrict__ gd,
                                                              const int32_t* __restrict__ coff,
                                                              const int32_t* __restrict__ seg, int32_t* ccnt,
                                                              int32_t* __restrict__ nxt, int2* __restrict__ wt,
                                                              int32_t* __restrict__ vis, const Counters* cnt) {
    if (cnt->err) return;
    for (int32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
        ccnt[p] = 0;
        if (!(kind[p] & kDFin)) continue;
        const int32_t a = coff[p], k = coff[p + 1] - a;
        const int32_t first = k > 0 ? seg[a] : -1;
        const bool visit_here = k == 0 || !(flags[first] & kPriOdd);
        const int32_t d = walk_len(gd, p);
        nxt[2 * p] = k > 0 ? 2 * first : 2 * p + 1;
        wt[2 * p] = make_int2(visit_here ? 1 : 0, d);
        wt[2 * p + 1] = make_int2(0, -d);
        if (visit_here) vis[p] = 2 * p;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) ccnt[n] = 0;
}

// Every child of a vertex parent, at its sorted position i: its exit element
// links to its next sibling's enter element (or to the parent's exit); the
// last odd child's exit element carries the parent's visit.
__global__ void __launch_bounds__(kBlock) k_deep_links_seg(int32_t n, const uint32_t* __restrict__ gd32,
                                                           const uint8_t* __restrict__ flags,
                                                           const uint64_t* __restrict__ gd,
                                                           const int32_t* __restrict__ coff,
                                                           const int32_t* __restrict__ seg, int32_t* __restrict__ nxt,
                                                           int2* __restrict__ wt, int32_t* __restrict__ vis,
                                                           const Counters* cnt) {
    if (cnt->err) return;
    const int32_t total = coff[n];
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
        const int32_t c = seg[i];
        const int32_t p = g32_ptr(gd32[c]);
        const int32_t nx = i + 1 < coff[p + 1] ? seg[i + 1] : -1;
        nxt[2 * c + 1] = nx >= 0 ? 2 * nx : 2 * p + 1;
        if ((flags[c] & kPriOdd) && (nx < 0 || !(flags[nx] & kPriOdd))) {
            wt[2 * c + 1] = make_int2(1, -walk_len(gd, c));
            vis[p] = 2 * c + 1;
        }
    }
}

__device__ inline int32_t game_first(int32_t gi, const int32_t* __restrict__ gsink) {
    return gi > 0 ? gsink[gi - 1] + 1 : 0;
}

// The sink's children of each game: odd ones by decreasing id (the list oddL
// holds them increasing), then even ones by increasing id. The last odd one
// carries the sink's visit (the rank of the empty valuation).
__global__ void __launch_bounds__(kBlock) k_deep_links_sink(int32_t n, const uint64_t* __restrict__ gd,
                                                            const int32_t* __restrict__ podd,
                                                            const int32_t* __restrict__ peven,
                                                            const int32_t* __restrict__ oddL,
                                                            const int32_t* __restrict__ evenL,
                                                            const int32_t* __restrict__ vgame,
                                                            const int32_t* __restrict__ gsink, int32_t sink0,
                                                            int32_t* __restrict__ nxt, int2* __restrict__ wt,
                                                            int32_t* __restrict__ vis, const Counters* cnt) {
    if (cnt->err) return;
    const int32_t no = podd[n], ne = peven[n];
    for (int32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < no + ne; j += gridDim.x * blockDim.x) {
        const bool odd = j < no;
        const int32_t c = odd ? oddL[j] : evenL[j - no];
        const int32_t gi = vgame ? vgame[c] : 0;
        const int32_t s = vgame ? gsink[gi] : sink0;
        const int32_t first = vgame ? game_first(gi, gsink) : 0;
        int32_t sib;
        if (odd) {
            const int32_t t = j - podd[first];
            const int32_t e0 = peven[first], ke = peven[s] - e0;
            sib = t > 0 ? oddL[j - 1] : (ke > 0 ? evenL[e0] : -1);
            if (t == 0) {
                wt[2 * c + 1] = make_int2(1, -walk_len(gd, c));
                vis[s] = 2 * c + 1;
            }
        } else {
            const int32_t je = j - no;
            sib = je + 1 < peven[s] ? evenL[je + 1] : -1;
        }
        nxt[2 * c + 1] = sib >= 0 ? 2 * sib : 2 * s + 1;
    }
}

// Each game's sink slot: the list head (enter) links to the first child in
// order, the exit element ends the list.
__global__ void k_deep_links_slot(int32_t ngames, const int32_t* __restrict__ podd,
                                  const int32_t* __restrict__ peven, const int32_t* __restrict__ oddL,
                                  const int32_t* __restrict__ evenL, const int32_t* __restrict__ gsink, int32_t sink0,
                                  int single, int32_t* __restrict__ nxt, int2* __restrict__ wt,
                                  int32_t* __restrict__ vis, const Counters* cnt) {
    if (cnt->err) return;
    for (int32_t gi = blockIdx.x * blockDim.x + threadIdx.x; gi < ngames; gi += gridDim.x * blockDim.x) {
        const int32_t s = single ? sink0 : gsink[gi];
        const int32_t first = single ? 0 : game_first(gi, gsink);
        const int32_t ko = podd[s] - podd[first], ke = peven[s] - peven[first];
        nxt[2 * s] = ko > 0 ? 2 * oddL[podd[s] - 1] : (ke > 0 ? 2 * evenL[peven[first]] : 2 * s + 1);
        wt[2 * s] = make_int2(ko == 0 ? 1 : 0, 0);
        if (ko == 0) vis[s] = 2 * s;
        nxt[2 * s + 1] = -1;
        wt[2 * s + 1] = make_int2(0, 0);
    }
}

// ---------------------------------------------------------------------------
// D4: list ranking by a sparse ruling set. An element is in a list when its
// vertex is finite or a sink slot. Rulers: every list head (a sink slot's
// enter element) and every listed element whose hash falls in the top
// 1/stride of the range (stride a power of two, log2 in stride_bits).
__device__ inline uint32_t ruler_hash(uint32_t e) { return e * 0x9E3779B1u; }

__global__ void __launch_bounds__(kBlock) k_deep_rulers(int32_t n, const uint8_t* __restrict__ kind,
                                                        int stride_bits, int32_t cap, int32_t* __restrict__ rid,
                                                        int32_t* __restrict__ rl, int32_t* __restrict__ own,
                                                        Counters* cnt) {
    if (cnt->err) return;
    const int64_t ne = 2 * (int64_t)n;
    for (int64_t e0 = (int64_t)blockIdx.x * blockDim.x; e0 < ne; e0 += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e = e0 + threadIdx.x;
        bool ruler = false;
        if (e < ne) {
            const uint8_t kd = kind[e >> 1];
            const bool listed = (kd & (kDFin | kDSinkSlot)) != 0;
            const bool head = (kd & kDSinkSlot) && !(e & 1);
            ruler = listed && (head || (ruler_hash((uint32_t)e) >> (32 - stride_bits)) == 0);
        }
        int32_t at = warp_append(ruler, &cnt->n_rulers);
        if (ruler && at >= cap) {  // more rulers than the scratch holds: recorded, nothing written
            atomicOr(&cnt->err, kErrRulers);
            ruler = false;
            at = -1;
        }
        if (e < ne) {
            rid[e] = ruler ? at : -1;
            own[e] = -1;  // set by the walk of the ruler whose sublist holds e
        }
        if (ruler) rl[at] = (int32_t)e;
    }
}

// Each ruler walks its sublist (up to the next ruler or the list's end):
// inclusive prefix of the weights within the sublist (loc) and the owning
// ruler (own) of every element, the sublist's sum and the next ruler.
__global__ void __launch_bounds__(kBlock) k_deep_rwalk(const int32_t* __restrict__ rl, const int32_t* __restrict__ rid,
                                                       const int32_t* __restrict__ nxt, const int2* __restrict__ wt,
                                                       int2* __restrict__ loc, int32_t* __restrict__ own,
                                                       int2* __restrict__ val0, int32_t* __restrict__ nx0, int64_t limit,
                                                       Counters* cnt) {
    if (cnt->err) return;
    const int32_t nr = cnt->n_rulers;
    for (int32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < nr; j += gridDim.x * blockDim.x) {
        int32_t e = rl[j];
        int2 acc = make_int2(0, 0);
        int32_t next_ruler = -1;
        for (int64_t steps = 0;; ++steps) {
            const int2 w = wt[e];
            acc.x += w.x;
            acc.y += w.y;
            loc[e] = acc;
            own[e] = j;
            const int32_t nx = nxt[e];
            if (nx < 0) break;
            const int32_t r2 = rid[nx];
            if (r2 >= 0) {
                next_ruler = r2;
                break;
            }
            if (steps > limit) {  // longer than every list: a malformed tour (never taken)
                atomicOr(&cnt->err, kErrRulers);
                break;
            }
            e = nx;
        }
        val0[j] = acc;
        nx0[j] = next_ruler;
    }
}

// Suffix sums over the list of rulers by pointer jumping (Wyllie), double
// buffered, all rounds in one cooperative launch: afterwards the buffer named
// in cnt->rs_buf holds, for each ruler, the sum from its sublist to the end of
// its list.
__global__ void __launch_bounds__(kBlock) k_deep_wyllie_coop(int2* val0, int32_t* nx0, int2* val1, int32_t* nx1,
                                                             Counters* cnt, int32_t cap) {
    if (cnt->err) return;
    const int32_t nr = cnt->n_rulers;
    for (int32_t r = 0;; ++r) {
        int2* vs = (r & 1) ? val1 : val0;
        int32_t* ns = (r & 1) ? nx1 : nx0;
        int2* vd = (r & 1) ? val0 : val1;
        int32_t* nd = (r & 1) ? nx0 : nx1;
        if (blockIdx.x == 0 && threadIdx.x == 0) cnt->left[(r + 1) % 3] = 0;
        int32_t live = 0;
        for (int32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < nr; j += gridDim.x * blockDim.x) {
            const int32_t nj = __ldcg(ns + j);
            int2 v = __ldcg(vs + j);
            if (nj >= 0) {
                const int2 u = __ldcg(vs + nj);
                v.x += u.x;
                v.y += u.y;
                const int32_t nn = __ldcg(ns + nj);
                __stcg(nd + j, nn);
                if (nn >= 0) ++live;
            } else {
                __stcg(nd + j, -1);
            }
            __stcg(vd + j, v);
        }
        block_add(live, &cnt->left[r % 3]);
        if (!grid_sync(cnt)) return;
        const int32_t rem = *(volatile int32_t*)&cnt->left[r % 3];
        if (rem == 0) {
            if (blockIdx.x == 0 && threadIdx.x == 0) {
                cnt->rs_rounds = r + 1;
                cnt->rs_buf = (r & 1) ? 0 : 1;  // the buffer written in this round
            }
            return;
        }
        if (r + 1 >= cap) {
            if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(&cnt->err, kErrJumpRounds);
            return;
        }
    }
}

// ---------------------------------------------------------------------------
// D5: ranks and depths from the ranked list. The inclusive prefix of element
// e is (its list's total - the suffix sum of its ruler) + its prefix within
// the ruler's sublist; the list's total is the suffix sum of its head.
__device__ inline int2 prefix_of(int32_t e, int32_t head, const int2* __restrict__ loc, const int32_t* __restrict__ own,
                                 const int2* __restrict__ suf) {
    const int2 tot = suf[head], sj = suf[own[e]], l = loc[e];
    return make_int2(tot.x - sj.x + l.x, tot.y - sj.y + l.y);
}

__global__ void __launch_bounds__(kBlock) k_deep_results(int32_t n, const uint8_t* __restrict__ kind,
                                                         const int32_t* __restrict__ vis,
                                                         const int32_t* __restrict__ rid,
                                                         const int2* __restrict__ loc,
                                                         const int32_t* __restrict__ own, const int2* val0,
                                                         const int2* val1, const int32_t* __restrict__ vgame,
                                                         const int32_t* __restrict__ gsink, int32_t sink0,
                                                         int32_t* __restrict__ key, int32_t* __restrict__ depth,
                                                         Counters* cnt) {
    if (cnt->err) return;
    const int2* suf = cnt->rs_buf ? val1 : val0;
    for (int32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        const uint8_t kd = kind[v];
        if (!(kd & (kDFin | kDSinkSlot))) {
            key[v] = INT32_MAX;
            depth[v] = -1;
            continue;
        }
        const int32_t s = vgame ? gsink[vgame[v]] : sink0;
        const int32_t head = rid[2 * s];
        const int32_t e = vis[v];
        if (head < 0 || e < 0 || own[e] < 0 || own[2 * v] < 0) {  // not on its list (never taken)
            atomicOr(&cnt->err, kErrRulers);
            key[v] = INT32_MIN;
            continue;
        }
        const int32_t r = prefix_of(e, head, loc, own, suf).x - 1;
        key[v] = r;
        if (kd & kDSinkSlot) {
            depth[v] = 0;
            if (v == (vgame ? gsink[0] : sink0)) cnt->sink_rank = r;
        } else {
            depth[v] = prefix_of(2 * v, head, loc, own, suf).y;
        }
    }
}

}  // namespace
}  // namespace pg

namespace pg {

// Scratch of the ruling-set path, allocated before the game's first deep
// valuation (outside any stream capture: the loops call this before they
// build their graph).
pg_status prepare_deep(pg_game* g) {
    pg_ctx* ctx = g->ctx;
    const int64_t n = g->n;
    const int bits = std::max(1, std::min(g->tune.ruler_bits, 16));
    // rulers: list heads plus about 2n / 2^bits hashed ones, with room for twice that
    const int64_t want = 2 * ((2 * n) >> bits) + g->ngames + 1024;
    const int32_t rcap = (int32_t)std::min<int64_t>(want, 2 * n + g->ngames + 1024);
    if (g->d_anc && g->d_rcap >= rcap) return PG_OK;
    auto A = [&](void** p, size_t bytes) { return dev_alloc(ctx, p, bytes, ctx->stream); };
    if (!g->d_anc) {
        PG_CUDA_TRY(ctx, A((void**)&g->d_anc, sizeof(int32_t) * n));
        PG_CUDA_TRY(ctx, A((void**)&g->d_sc, 2 * (size_t)n));
        PG_CUDA_TRY(ctx, A((void**)&g->d_podd, sizeof(int32_t) * (n + 1)));
        PG_CUDA_TRY(ctx, A((void**)&g->d_peven, sizeof(int32_t) * (n + 1)));
        PG_CUDA_TRY(ctx, A((void**)&g->d_oddL, sizeof(int32_t) * n));
        PG_CUDA_TRY(ctx, A((void**)&g->d_evenL, sizeof(int32_t) * n));
        PG_CUDA_TRY(ctx, A((void**)&g->d_nxt, sizeof(int32_t) * 2 * n));
        PG_CUDA_TRY(ctx, A((void**)&g->d_wt, sizeof(int2) * 2 * n));
        PG_CUDA_TRY(ctx, A((void**)&g->d_loc, sizeof(int2) * 2 * n));
        PG_CUDA_TRY(ctx, A((void**)&g->d_own, sizeof(int32_t) * 2 * n));
        PG_CUDA_TRY(ctx, A((void**)&g->d_rid, sizeof(int32_t) * 2 * n));
        int sms = 0, a = 0, b = 0;
        PG_CUDA_TRY(ctx, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device));
        PG_CUDA_TRY(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_deep_anc_coop, kBlock, 0));
        PG_CUDA_TRY(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_deep_wyllie_coop, kBlock, 0));
        g->d_coop = sms * std::max(1, std::min(std::min(a, b), 4));
    }
    if (g->d_rl) {  // a denser ruler setting than the scratch was made for
        cudaFreeAsync(g->d_rl, ctx->stream);
        cudaFreeAsync(g->d_val, ctx->stream);
        cudaFreeAsync(g->d_rnx, ctx->stream);
        g->d_rl = nullptr;
        g->d_val = nullptr;
        g->d_rnx = nullptr;
    }
    PG_CUDA_TRY(ctx, A((void**)&g->d_rl, sizeof(int32_t) * rcap));
    PG_CUDA_TRY(ctx, A((void**)&g->d_val, sizeof(int2) * 2 * (size_t)rcap));
    PG_CUDA_TRY(ctx, A((void**)&g->d_rnx, sizeof(int32_t) * 2 * (size_t)rcap));
    g->d_rcap = rcap;
    return PG_OK;
}

pg_status enqueue_valuation_deep(pg_game* g, bool want_dom) {
    pg_ctx* ctx = g->ctx;
    cudaStream_t s = ctx->stream;
    pg_status st = prepare_deep(g);
    if (st) return st;
    const int32_t n = g->n;
    Counters* c = g->cnt;
    const unsigned grid = grid_for(n);
    st = enqueue_k1(g);
    if (st) return st;
    prof_begin(g, KID_DEEP);
    // D1
    int32_t* vis = g->wgt;  // the chain-weight array holds each vertex's visit element
    k_deep_init<<<grid, kBlock, 0, s>>>(n, g->gd32, g->flags, g->d_anc, g->ccnt, g->plist, vis, c);
    {
        int32_t cap = 40;
        void* args[] = {(void*)&g->plist, (void*)&g->d_anc, (void*)&c, (void*)&cap};
        PG_CUDA_TRY(ctx, cudaLaunchCooperativeKernel((void*)k_deep_anc_coop, g->d_coop, kBlock, args, 0, s));
    }
    uint8_t* sc_odd = g->d_sc;
    uint8_t* sc_even = g->d_sc + n;
    k_deep_classify<<<grid, kBlock, 0, s>>>(n, g->gd32, g->flags, g->pri, g->d_anc, g->ccnt, g->slot, g->kind, g->cls,
                                            g->dom, want_dom ? 1 : 0, sc_odd, sc_even, g->vgame, g->gst, c);
    // D2
    PG_CUDA_TRY(ctx, exclusive_scan_i32(g->ccnt, g->coff, n, nullptr, g->scan_tmp, g->scan_tmp_bytes, s));
    PG_CUDA_TRY(ctx, exclusive_scan_u8(sc_odd, g->d_podd, n, g->scan_tmp, g->scan_tmp_bytes, s));
    PG_CUDA_TRY(ctx, exclusive_scan_u8(sc_even, g->d_peven, n, g->scan_tmp, g->scan_tmp_bytes, s));
    int32_t* seg = (int32_t*)g->cl_ks;  // the chain pass's [n] pairs hold the segments and their radix copy
    int32_t* seg2 = seg + n;
    int32_t* midlist = g->hugelist;
    int32_t* biglist = g->hugelist + n / 2;
    k_deep_scatter<<<grid, kBlock, 0, s>>>(n, g->gd32, g->kind, g->coff, g->slot, sc_odd, sc_even, g->d_podd,
                                           g->d_peven, seg, g->d_oddL, g->d_evenL, c);
    k_deep_sort_small<<<grid, kBlock, 0, s>>>(n, g->coff, g->flags, seg, midlist, biglist, c);
    k_deep_sort_mid<<<g->d_coop, kBlock, 0, s>>>(g->coff, g->flags, seg, midlist, c);
    k_deep_sort_big<<<g->d_coop, kBlock, 0, s>>>(g->coff, g->flags, seg, seg2, biglist, c);
    // D3
    k_deep_links_parent<<<grid, kBlock, 0, s>>>(n, g->kind, g->flags, g->gd, g->coff, seg, g->ccnt, g->d_nxt, g->d_wt,
                                                vis, c);
    k_deep_links_seg<<<grid, kBlock, 0, s>>>(n, g->gd32, g->flags, g->gd, g->coff, seg, g->d_nxt, g->d_wt, vis, c);
    k_deep_links_sink<<<grid, kBlock, 0, s>>>(n, g->gd, g->d_podd, g->d_peven, g->d_oddL, g->d_evenL, g->vgame,
                                              g->gsink, g->sink0, g->d_nxt, g->d_wt, vis, c);
    const unsigned gg = (unsigned)std::max<int64_t>(1, std::min<int64_t>(((int64_t)g->ngames + kBlock - 1) / kBlock, 4096));
    k_deep_links_slot<<<gg, kBlock, 0, s>>>(g->ngames, g->d_podd, g->d_peven, g->d_oddL, g->d_evenL, g->gsink,
                                            g->sink0, g->vgame ? 0 : 1, g->d_nxt, g->d_wt, vis, c);
    // D4
    const int bits = std::max(1, std::min(g->tune.ruler_bits, 16));
    k_deep_rulers<<<grid_for(2 * (int64_t)n), kBlock, 0, s>>>(n, g->kind, bits, g->d_rcap, g->d_rid, g->d_rl, g->d_own,
                                                              c);
    int2* val0 = g->d_val;
    int2* val1 = g->d_val + g->d_rcap;
    int32_t* nx0 = g->d_rnx;
    int32_t* nx1 = g->d_rnx + g->d_rcap;
    k_deep_rwalk<<<grid_for(g->d_rcap), kBlock, 0, s>>>(g->d_rl, g->d_rid, g->d_nxt, g->d_wt, g->d_loc, g->d_own, val0,
                                                        nx0, 2 * (int64_t)n + 2, c);
    {
        int32_t cap = 40;
        void* args[] = {(void*)&val0, (void*)&nx0, (void*)&val1, (void*)&nx1, (void*)&c, (void*)&cap};
        PG_CUDA_TRY(ctx, cudaLaunchCooperativeKernel((void*)k_deep_wyllie_coop, g->d_coop, kBlock, args, 0, s));
    }
    // D5
    k_deep_results<<<grid, kBlock, 0, s>>>(n, g->kind, vis, g->d_rid, g->d_loc, g->d_own, val0, val1, g->vgame,
                                           g->gsink, g->sink0, g->key, g->depth, c);
    prof_end(g, KID_DEEP, 20);
    PG_CUDA_TRY(ctx, cudaGetLastError());
    g->val_deep = true;
    return PG_OK;
}

}  // namespace pg
