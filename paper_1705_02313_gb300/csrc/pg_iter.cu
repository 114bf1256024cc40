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
// computed as
//   rank(v) = oddsz(v) + sum over c on v's g-chain below the sink of wgt(c),
//   wgt(c)  = [pri(c) even] + total size of the siblings ordered before c,
// with sizes of g-subtrees. Infinite plays (TOP) end in a cycle; the cycle's
// largest vertex is the only vertex whose walk returns to itself, which gives
// the dominant priority of the cycle (Section 5, "Modifications to the
// Helman-JaJa algorithm": pseudotree vertices are TOP; an odd dominant
// priority means sigma was not admissible).
//
// Switching (Section 3, "Switching rules"; Section 4, All_Odd): a segmented
// arg-best over each vertex's edge list using the ranks as keys.
#include <algorithm>
#include <vector>

#include "pg_internal.cuh"

namespace pg {
namespace {

inline unsigned grid_for(int64_t n, int per = kBlock) {
    int64_t b = (n + per - 1) / per;
    if (b < 1) b = 1;
    if (b > 152 * 64) b = 152 * 64;  // grid-stride beyond this
    return (unsigned)b;
}

__device__ inline int32_t warp_append(bool pred, int32_t* counter) {
    unsigned act = __activemask();
    unsigned m = __ballot_sync(act, pred);
    if (!m) return -1;
    int lane = threadIdx.x & 31;
    int leader = __ffs(m) - 1;
    int32_t base = 0;
    if (lane == leader) base = atomicAdd(counter, __popc(m));
    base = __shfl_sync(act, base, leader);
    return pred ? base + __popc(m & ((1u << lane) - 1u)) : -1;
}

__device__ inline void block_add(int32_t v, int32_t* counter) {
    __shared__ int32_t acc;
    if (threadIdx.x == 0) acc = 0;
    __syncthreads();
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0 && v) atomicAdd(&acc, v);
    __syncthreads();
    if (threadIdx.x == 0 && acc) atomicAdd(counter, acc);
}

__device__ inline uint64_t ld_cg(const uint64_t* p) { return __ldcg((const unsigned long long*)p); }
__device__ inline void st_cg(uint64_t* p, uint64_t v) { __stcg((unsigned long long*)p, (unsigned long long)v); }

// K1: nearest greater vertex along the play, by a direct walk of at most
// kWalkCap steps. A walk that returns to its start found the maximum of its
// cycle; a walk that runs out of steps leaves a jump pointer for k_jump.
__global__ void k_gwalk(int32_t n, const int32_t* __restrict__ strat, uint64_t* __restrict__ gd,
                        int32_t* __restrict__ plist, Counters* cnt) {
    for (int32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        int32_t x = __ldg(strat + v);
        uint32_t d = 1;
        while (x < v && d < (uint32_t)kWalkCap) {
            x = __ldg(strat + x);
            ++d;
        }
        uint64_t w;
        bool pend = false;
        if (x > v) w = gd_pack(true, false, d, x);           // a larger vertex or the sink
        else if (x == v) w = gd_pack(true, true, d, v);      // v is the maximum of its cycle
        else { w = gd_pack(false, false, d, x); pend = true; }
        gd[v] = w;
        int32_t slot = warp_append(pend, &cnt->n_pending);
        if (pend) plist[slot] = v;
    }
}

// Pointer jumping over smaller vertices for the walks that ran out of steps.
// Invariant of a pending word: every vertex strictly between v and ptr is
// below v, and ptr is below v. Jumping through x = ptr uses x's own pointer
// (x pending) or g(x) (x resolved): both skip only vertices below x < v.
__global__ void k_jump(int32_t np, const int32_t* __restrict__ plist, uint64_t* gd, Counters* cnt) {
    int32_t left = 0;
    for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < np; i += gridDim.x * blockDim.x) {
        int32_t v = plist[i];
        uint64_t w = ld_cg(gd + v);
        if (gd_resolved(w)) continue;
        int32_t x = gd_ptr(w);
        uint64_t wx = ld_cg(gd + x);
        uint64_t nw;
        if (gd_resolved(wx) && gd_none(wx)) {
            // x is above its whole future and below v: so is v (same cycle)
            nw = gd_pack(true, true, 0, gd_ptr(wx));
        } else {
            int32_t y = gd_ptr(wx);
            uint64_t nd = (uint64_t)gd_dist(w) + gd_dist(wx);
            if (nd > 0x3fffffffull) nd = 0x3fffffffull;  // only reachable around cycles, where dist is unused
            if (y > v) nw = gd_pack(true, false, (uint32_t)nd, y);
            else if (y == v) nw = gd_pack(true, true, (uint32_t)nd, v);
            else {
                nw = gd_pack(false, false, (uint32_t)nd, y);
                ++left;
            }
        }
        st_cg(gd + v, nw);
    }
    block_add(left, &cnt->n_pending);
}

// First pass over g-chains: class, depth, subtree sizes and children lists.
__global__ void k_chain1(int32_t n, const uint64_t* __restrict__ gd, const uint8_t* __restrict__ flags,
                         const int32_t* __restrict__ pri, uint8_t* __restrict__ cls, uint8_t* __restrict__ kind,
                         int32_t* __restrict__ depth, int32_t* sz, int32_t* head, int32_t* __restrict__ nxt,
                         int32_t* __restrict__ dom, int want_dom, Counters* cnt) {
    int32_t nfin = 0, nodd = 0;
    for (int32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        uint64_t w = gd[v];
        int32_t cyc = -1;
        uint32_t dep = 0;
        if (gd_none(w)) {
            cyc = gd_ptr(w);
        } else {
            dep = gd_dist(w);
            int32_t x = gd_ptr(w);
            while (x != n) {
                uint64_t wx = gd[x];
                if (gd_none(wx)) {
                    cyc = gd_ptr(wx);
                    break;
                }
                dep += gd_dist(wx);
                x = gd_ptr(wx);
            }
        }
        if (cyc < 0) {
            int32_t g = gd_ptr(w);
            cls[v] = kFin;
            depth[v] = (int32_t)dep;
            kind[v] = kKindFin | (g == n ? kKindSinkChild : 0);
            for (int32_t x = g; x != n; x = gd_ptr(gd[x])) atomicAdd(sz + x, 1);
            if (g != n) nxt[v] = atomicExch(head + g, v);
            if (want_dom) dom[v] = -1;
            ++nfin;
        } else {
            bool odd = (flags[cyc] & kPriOdd) != 0;
            cls[v] = odd ? kOddCycle : kTop;
            kind[v] = 0;
            depth[v] = -1;
            if (want_dom) dom[v] = pri[cyc];
            nodd += odd;
        }
    }
    block_add(nfin, &cnt->n_fin);
    block_add(nodd, &cnt->n_odd);
}

__device__ inline int32_t order_key(int32_t c, uint8_t f) { return (f & kPriOdd) ? -(c + 1) : c; }

// Children of non-sink parents: sort each small list by the order of
// Section 3 (odd children by decreasing id, then even children by increasing
// id) and give every child its weight; parents with more children are left
// to k_big_parents.
__global__ void k_parents(int32_t n, const int32_t* __restrict__ head, const int32_t* __restrict__ nxt,
                          const int32_t* __restrict__ sz, const uint8_t* __restrict__ flags, int32_t* wgt,
                          int32_t* oddsz, int32_t* biglist, Counters* cnt) {
    for (int32_t a = blockIdx.x * blockDim.x + threadIdx.x; a < n; a += gridDim.x * blockDim.x) {
        int32_t h = head[a];
        if (h < 0) {
            oddsz[a] = 0;
            continue;
        }
        int32_t ids[kSmallChildren];
        int32_t keys[kSmallChildren];
        int cnt_c = 0;
        bool big = false;
        for (int32_t c = h; c >= 0; c = nxt[c]) {
            if (cnt_c == kSmallChildren) {
                big = true;
                break;
            }
            int32_t kk = order_key(c, flags[c]);
            int j = cnt_c++;
            while (j > 0 && keys[j - 1] > kk) {
                keys[j] = keys[j - 1];
                ids[j] = ids[j - 1];
                --j;
            }
            keys[j] = kk;
            ids[j] = c;
        }
        if (big) {
            int32_t slot = atomicAdd(&cnt->n_big, 1);
            biglist[slot] = a;
            continue;
        }
        int32_t run = 0, os = 0;
        for (int i = 0; i < cnt_c; ++i) {
            int32_t c = ids[i];
            int32_t s = 1 + sz[c];
            bool odd = keys[i] < 0;
            wgt[c] = run + (odd ? 0 : 1);
            run += s;
            if (odd) os += s;
        }
        oddsz[a] = os;
    }
}

// Big parents (more than kSmallChildren children): instead of walking a long
// list, every child finds its parent's batch slot and appends itself to the
// slot's buffer; k_big_parents then sorts each buffer in shared memory.
__global__ void k_big_collect(int32_t n, const uint64_t* __restrict__ gd, const uint8_t* __restrict__ kind,
                              const int32_t* __restrict__ bigslot, int32_t* bigfill, int32_t* bigbuf,
                              const Counters* cnt) {
    if (cnt->n_big == 0) return;
    for (int32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        uint8_t kd = kind[v];
        if (!(kd & kKindFin) || (kd & kKindSinkChild)) continue;
        int32_t a = gd_ptr(gd[v]);
        int32_t b = bigslot[a];
        if (b < 0) continue;
        int32_t pos = atomicAdd(bigfill + b, 1);
        if (pos < kBlockChildren) bigbuf[(int64_t)b * kBlockChildren + pos] = v;
    }
}

__global__ void k_big_mark(const int32_t* __restrict__ biglist, int32_t* bigslot, const Counters* cnt) {
    int32_t nb = cnt->n_big;
    for (int32_t b = blockIdx.x * blockDim.x + threadIdx.x; b < nb; b += gridDim.x * blockDim.x)
        bigslot[biglist[b]] = b;
}

__global__ void k_big_parents(const int32_t* __restrict__ biglist, int32_t* bigslot, int32_t* bigfill,
                              const int32_t* __restrict__ bigbuf, const int32_t* __restrict__ sz,
                              const uint8_t* __restrict__ flags, int32_t* wgt, int32_t* oddsz, int32_t* hugelist,
                              Counters* cnt) {
    __shared__ int64_t sk[kBlockChildren];  // (order key << 32) | id
    __shared__ int32_t wsum[kBlock / 32];
    __shared__ int32_t carry_s, odd_s;
    int32_t nb = cnt->n_big;
    for (int32_t b = blockIdx.x; b < nb; b += gridDim.x) {
        int32_t a = biglist[b];
        int32_t count = bigfill[b];
        __syncthreads();
        if (count > kBlockChildren) {
            if (threadIdx.x == 0) {
                hugelist[atomicAdd(&cnt->pad, 1)] = a;  // pad counts huge parents
                bigslot[a] = -1;
                bigfill[b] = 0;
            }
            continue;
        }
        int p2 = 1;
        while (p2 < count) p2 <<= 1;
        for (int i = threadIdx.x; i < p2; i += blockDim.x) {
            if (i < count) {
                int32_t c = bigbuf[(int64_t)b * kBlockChildren + i];
                sk[i] = ((int64_t)order_key(c, flags[c]) << 32) | (uint32_t)c;
            } else {
                sk[i] = INT64_MAX;
            }
        }
        __syncthreads();
        // bitonic sort in shared memory
        for (int kk = 2; kk <= p2; kk <<= 1) {
            for (int j = kk >> 1; j > 0; j >>= 1) {
                for (int i = threadIdx.x; i < p2; i += blockDim.x) {
                    int ixj = i ^ j;
                    if (ixj > i) {
                        int64_t x = sk[i], y = sk[ixj];
                        bool up = (i & kk) == 0;
                        if ((x > y) == up) {
                            sk[i] = y;
                            sk[ixj] = x;
                        }
                    }
                }
                __syncthreads();
            }
        }
        // running sums in sorted order, one chunk of blockDim elements at a time
        if (threadIdx.x == 0) {
            carry_s = 0;
            odd_s = 0;
        }
        __syncthreads();
        for (int base = 0; base < count; base += blockDim.x) {
            int i = base + threadIdx.x;
            int32_t c = -1, s = 0;
            bool odd = false;
            if (i < count) {
                c = (int32_t)(uint32_t)(sk[i] & 0xffffffffll);
                s = 1 + sz[c];
                odd = (sk[i] >> 32) < 0;
            }
            // block exclusive scan of s
            int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
            int32_t x = s;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                int32_t y = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o) x += y;
            }
            if (lane == 31) wsum[wid] = x;
            __syncthreads();
            if (wid == 0) {
                int32_t t = lane < kBlock / 32 ? wsum[lane] : 0;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    int32_t y = __shfl_up_sync(0xffffffffu, t, o);
                    if (lane >= o) t += y;
                }
                if (lane < kBlock / 32) wsum[lane] = t;
            }
            __syncthreads();
            int32_t excl = carry_s + (wid > 0 ? wsum[wid - 1] : 0) + x - s;
            if (c >= 0) wgt[c] = excl + (odd ? 0 : 1);
            int32_t oddpart = odd ? s : 0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) oddpart += __shfl_down_sync(0xffffffffu, oddpart, o);
            __syncthreads();
            if (lane == 0 && oddpart) atomicAdd(&odd_s, oddpart);
            if (threadIdx.x == 0) carry_s += wsum[kBlock / 32 - 1];
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            oddsz[a] = odd_s;
            bigslot[a] = -1;
            bigfill[b] = 0;
        }
        __syncthreads();
    }
}

// Children of one parent p whose children are too many for a block (and of
// the sink, which has most vertices as children): their order is the id
// order, so a scan over ids does it. Pass 1: per-tile sums of the even and
// odd children's sizes.
constexpr int kSIpt = 8;
constexpr int kSTile = kBlock * kSIpt;

template <bool kSink>
__device__ inline bool is_child(int64_t i, int32_t p, const uint8_t* kind, const uint64_t* gd) {
    uint8_t kd = kind[i];
    if (!(kd & kKindFin)) return false;
    if (kSink) return (kd & kKindSinkChild) != 0;
    return !(kd & kKindSinkChild) && gd_ptr(gd[i]) == p;
}

template <bool kSink>
__global__ void k_idscan_reduce(int32_t n, int32_t p, const uint8_t* __restrict__ kind,
                                const uint64_t* __restrict__ gd, const int32_t* __restrict__ sz,
                                const uint8_t* __restrict__ flags, int64_t* tsum) {
    __shared__ int32_t se, so;
    if (threadIdx.x == 0) se = so = 0;
    __syncthreads();
    int64_t base = (int64_t)blockIdx.x * kSTile + (int64_t)threadIdx.x * kSIpt;
    int32_t e = 0, o = 0;
#pragma unroll
    for (int k = 0; k < kSIpt; ++k) {
        int64_t i = base + k;
        if (i < n && is_child<kSink>(i, p, kind, gd)) {
            int32_t s = 1 + sz[i];
            if (flags[i] & kPriOdd) o += s;
            else e += s;
        }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        e += __shfl_down_sync(0xffffffffu, e, off);
        o += __shfl_down_sync(0xffffffffu, o, off);
    }
    if ((threadIdx.x & 31) == 0) {
        if (e) atomicAdd(&se, e);
        if (o) atomicAdd(&so, o);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        tsum[2 * blockIdx.x] = se;
        tsum[2 * blockIdx.x + 1] = so;
    }
}

// exclusive scan of the (even, odd) tile sums by one block; totals at the end
__global__ void k_idscan_tiles(int64_t* tsum, int64_t ntiles) {
    __shared__ int64_t we[kBlock / 32], wo[kBlock / 32];
    int64_t ce = 0, co = 0;
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int64_t b = 0; b < ntiles; b += kBlock) {
        int64_t i = b + threadIdx.x;
        int64_t e = i < ntiles ? tsum[2 * i] : 0, o = i < ntiles ? tsum[2 * i + 1] : 0;
        int64_t xe = e, xo = o;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            int64_t ye = __shfl_up_sync(0xffffffffu, xe, d), yo = __shfl_up_sync(0xffffffffu, xo, d);
            if (lane >= d) {
                xe += ye;
                xo += yo;
            }
        }
        if (lane == 31) {
            we[wid] = xe;
            wo[wid] = xo;
        }
        __syncthreads();
        if (wid == 0) {
            int64_t te = lane < kBlock / 32 ? we[lane] : 0, to = lane < kBlock / 32 ? wo[lane] : 0;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                int64_t ye = __shfl_up_sync(0xffffffffu, te, d), yo = __shfl_up_sync(0xffffffffu, to, d);
                if (lane >= d) {
                    te += ye;
                    to += yo;
                }
            }
            if (lane < kBlock / 32) {
                we[lane] = te;
                wo[lane] = to;
            }
        }
        __syncthreads();
        int64_t pe = ce + (wid > 0 ? we[wid - 1] : 0) + xe - e;
        int64_t po = co + (wid > 0 ? wo[wid - 1] : 0) + xo - o;
        if (i < ntiles) {
            tsum[2 * i] = pe;
            tsum[2 * i + 1] = po;
        }
        ce += we[kBlock / 32 - 1];
        co += wo[kBlock / 32 - 1];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        tsum[2 * ntiles] = ce;
        tsum[2 * ntiles + 1] = co;
    }
}

// Pass 3: weights. Even child c: 1 + (all odd children) + (even children with
// smaller id); odd child c: odd children with larger id. The parent's own
// rank offset oddsz(p) is the odd total (the sink's rank when p is the sink).
template <bool kSink>
__global__ void k_idscan_apply(int32_t n, int32_t p, const uint8_t* __restrict__ kind,
                               const uint64_t* __restrict__ gd, const int32_t* __restrict__ sz,
                               const uint8_t* __restrict__ flags, const int64_t* __restrict__ tsum, int64_t ntiles,
                               int32_t* wgt, int32_t* oddsz_p) {
    __shared__ int32_t we[kBlock / 32], wo[kBlock / 32];
    int64_t base = (int64_t)blockIdx.x * kSTile + (int64_t)threadIdx.x * kSIpt;
    int32_t se[kSIpt], so[kSIpt];
    int32_t te = 0, to = 0;
#pragma unroll
    for (int k = 0; k < kSIpt; ++k) {
        int64_t i = base + k;
        se[k] = so[k] = 0;
        if (i < n && is_child<kSink>(i, p, kind, gd)) {
            int32_t s = 1 + sz[i];
            if (flags[i] & kPriOdd) so[k] = s;
            else se[k] = s;
        }
        te += se[k];
        to += so[k];
    }
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int32_t xe = te, xo = to;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        int32_t ye = __shfl_up_sync(0xffffffffu, xe, d), yo = __shfl_up_sync(0xffffffffu, xo, d);
        if (lane >= d) {
            xe += ye;
            xo += yo;
        }
    }
    if (lane == 31) {
        we[wid] = xe;
        wo[wid] = xo;
    }
    __syncthreads();
    if (wid == 0) {
        int32_t a = lane < kBlock / 32 ? we[lane] : 0, b = lane < kBlock / 32 ? wo[lane] : 0;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            int32_t ya = __shfl_up_sync(0xffffffffu, a, d), yb = __shfl_up_sync(0xffffffffu, b, d);
            if (lane >= d) {
                a += ya;
                b += yb;
            }
        }
        if (lane < kBlock / 32) {
            we[lane] = a;
            wo[lane] = b;
        }
    }
    __syncthreads();
    int64_t run_e = tsum[2 * blockIdx.x] + (wid > 0 ? we[wid - 1] : 0) + xe - te;
    int64_t run_o = tsum[2 * blockIdx.x + 1] + (wid > 0 ? wo[wid - 1] : 0) + xo - to;
    int64_t tot_o = tsum[2 * ntiles + 1];
#pragma unroll
    for (int k = 0; k < kSIpt; ++k) {
        int64_t i = base + k;
        if (se[k]) wgt[i] = (int32_t)(1 + tot_o + run_e);
        run_o += so[k];
        if (so[k]) wgt[i] = (int32_t)(tot_o - run_o);
        run_e += se[k];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) *oddsz_p = (int32_t)tot_o;
}

// Second pass over g-chains: the rank, and reset of the per-iteration lists.
__global__ void k_chain2(int32_t n, const uint64_t* __restrict__ gd, const uint8_t* __restrict__ kind,
                         const int32_t* __restrict__ wgt, const int32_t* __restrict__ oddsz,
                         int32_t* __restrict__ key, int32_t* __restrict__ sz, int32_t* __restrict__ head,
                         const Counters* cnt) {
    for (int32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        int32_t r = INT32_MAX;
        if (kind[v] & kKindFin) {
            int64_t acc = (int64_t)oddsz[v] + wgt[v];
            for (int32_t x = gd_ptr(gd[v]); x != n; x = gd_ptr(gd[x])) acc += wgt[x];
            r = (int32_t)acc;
        }
        key[v] = r;
        sz[v] = 0;
        head[v] = -1;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) key[n] = cnt->sink_rank;
}

// K3: greedy all-switches for one player. Odd takes the first minimiser of
// its edge list, Even the first maximiser with the sink looked at first; a
// vertex switches only if strictly better than its current choice.
__global__ void k_switch(int32_t n, int player, const int32_t* __restrict__ off, const int32_t* __restrict__ tgt,
                         const uint8_t* __restrict__ flags, const int32_t* __restrict__ key, int32_t* strat,
                         Counters* cnt) {
    int32_t nsw = 0;
    for (int32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        if ((flags[v] & kOwnerOdd) != player) continue;
        int32_t e0 = off[v], e1 = off[v + 1];
        int32_t best, bk;
        if (player == 0) {
            best = n;
            bk = key[n];
        } else {
            best = tgt[e0];
            bk = key[best];
            ++e0;
        }
        for (int32_t e = e0; e < e1; ++e) {
            int32_t u = tgt[e];
            int32_t ku = key[u];
            if (player == 0 ? ku > bk : ku < bk) {
                best = u;
                bk = ku;
            }
        }
        int32_t cur = key[strat[v]];
        if (player == 0 ? bk > cur : bk < cur) {
            strat[v] = best;
            ++nsw;
        }
    }
    block_add(nsw, &cnt->n_switch);
}

}  // namespace

const char* const kKernelNames[KID_COUNT] = {"walk", "jump", "chain1", "parents", "big_parents",
                                              "sink_scan", "chain2", "switch_odd", "switch_even"};

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
    int64_t n = g->n;
    auto A = [&](void** p, size_t bytes) { return cudaMalloc(p, bytes ? bytes : 1); };
    PG_CUDA_TRY(ctx, A((void**)&g->gd, sizeof(uint64_t) * n));
    PG_CUDA_TRY(ctx, A((void**)&g->plist, sizeof(int32_t) * n));
    PG_CUDA_TRY(ctx, A((void**)&g->cls, n));
    PG_CUDA_TRY(ctx, A((void**)&g->kind, n));
    PG_CUDA_TRY(ctx, A((void**)&g->depth, sizeof(int32_t) * n));
    PG_CUDA_TRY(ctx, A((void**)&g->sz, sizeof(int32_t) * n));
    PG_CUDA_TRY(ctx, A((void**)&g->head, sizeof(int32_t) * n));
    PG_CUDA_TRY(ctx, A((void**)&g->nxt, sizeof(int32_t) * n));
    PG_CUDA_TRY(ctx, A((void**)&g->wgt, sizeof(int32_t) * n));
    PG_CUDA_TRY(ctx, A((void**)&g->oddsz, sizeof(int32_t) * n));
    PG_CUDA_TRY(ctx, A((void**)&g->key, sizeof(int32_t) * (n + 1)));
    PG_CUDA_TRY(ctx, A((void**)&g->dom, sizeof(int32_t) * n));
    PG_CUDA_TRY(ctx, A((void**)&g->biglist, sizeof(int32_t) * n));
    PG_CUDA_TRY(ctx, A((void**)&g->cnt, sizeof(Counters)));
    g->ntiles = (n + kSTile - 1) / kSTile;
    if (g->ntiles < 1) g->ntiles = 1;
    PG_CUDA_TRY(ctx, A((void**)&g->scan_total, sizeof(int64_t) * (2 * g->ntiles + 2)));
    // big-parent scratch shares the plist-sized buffers: bigslot lives in wgt? no - own arrays
    PG_CUDA_TRY(ctx, A((void**)&g->tile_e, sizeof(int32_t) * n));  // bigslot
    PG_CUDA_TRY(ctx, A((void**)&g->tile_o, sizeof(int32_t) * n));  // bigfill
    cudaStream_t s = ctx->stream;
    PG_CUDA_TRY(ctx, cudaMemsetAsync(g->sz, 0, sizeof(int32_t) * n, s));
    PG_CUDA_TRY(ctx, cudaMemsetAsync(g->head, 0xff, sizeof(int32_t) * n, s));
    PG_CUDA_TRY(ctx, cudaMemsetAsync(g->tile_e, 0xff, sizeof(int32_t) * n, s));
    PG_CUDA_TRY(ctx, cudaMemsetAsync(g->tile_o, 0, sizeof(int32_t) * n, s));
    for (int i = 0; i < 4; ++i) PG_CUDA_TRY(ctx, cudaEventCreate(&g->ev[i]));
    for (int i = 0; i < 2 * KID_COUNT; ++i) PG_CUDA_TRY(ctx, cudaEventCreate(&g->kev[i]));
    return PG_OK;
}

pg_status valuate_device(pg_game* g, bool want_dom, Counters* h) {
    pg_ctx* ctx = g->ctx;
    cudaStream_t s = ctx->stream;
    int32_t n = g->n;
    Counters* c = g->cnt;
    unsigned grid = grid_for(n);
    PG_CUDA_TRY(ctx, cudaMemsetAsync(c, 0, sizeof(Counters), s));
    prof_begin(g, KID_WALK);
    k_gwalk<<<grid, kBlock, 0, s>>>(n, g->strat, g->gd, g->plist, c);
    prof_end(g, KID_WALK, 1);
    PG_CUDA_TRY(ctx, cudaMemcpyAsync(ctx->pinned, &c->n_pending, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    PG_CUDA_TRY(ctx, cudaStreamSynchronize(s));
    prof_collect(g);
    int32_t np = ctx->pinned[0];
    if (np > 0) {
        int rounds = 0;
        int cap = 96;
        for (int64_t x = n; x > 1; x >>= 1) cap += 2;
        for (;;) {
            PG_CUDA_TRY(ctx, cudaMemsetAsync(&c->n_pending, 0, sizeof(int32_t), s));
            prof_begin(g, KID_JUMP);
            k_jump<<<grid_for(np), kBlock, 0, s>>>(np, g->plist, g->gd, c);
            prof_end(g, KID_JUMP, 1);
            PG_CUDA_TRY(ctx, cudaMemcpyAsync(ctx->pinned, &c->n_pending, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
            PG_CUDA_TRY(ctx, cudaStreamSynchronize(s));
            prof_collect(g);
            if (ctx->pinned[0] == 0) break;
            if (++rounds > cap) return fail(ctx, PG_ECUDA, "valuation: pointer jumping did not converge");
        }
    }
    prof_begin(g, KID_CHAIN1);
    k_chain1<<<grid, kBlock, 0, s>>>(n, g->gd, g->flags, g->pri, g->cls, g->kind, g->depth, g->sz, g->head, g->nxt,
                                     g->dom, want_dom ? 1 : 0, c);
    prof_end(g, KID_CHAIN1, 1);
    prof_begin(g, KID_PARENTS);
    k_parents<<<grid, kBlock, 0, s>>>(n, g->head, g->nxt, g->sz, g->flags, g->wgt, g->oddsz, g->biglist, c);
    prof_end(g, KID_PARENTS, 1);
    int32_t* bigslot = g->tile_e;
    int32_t* bigfill = g->tile_o;
    int32_t* hugelist = g->plist;  // pending list is no longer needed
    // big parents: their children are collected into kBlockChildren-entry slots of a buffer that borrows
    // key (rewritten by k_chain2 afterwards); parents are processed in batches that fit.
    int32_t* bigbuf = g->key;
    PG_CUDA_TRY(ctx, cudaMemcpyAsync(ctx->pinned, &c->n_big, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    PG_CUDA_TRY(ctx, cudaStreamSynchronize(s));
    prof_collect(g);
    int32_t nbig = ctx->pinned[0];
    if (nbig > 0) {
        int64_t cap_parents = (int64_t)n / kBlockChildren;
        if (cap_parents < 1) cap_parents = 1;
        // process big parents in batches that fit in the buffer
        std::vector<int32_t> hb((size_t)nbig);
        PG_CUDA_TRY(ctx, cudaMemcpyAsync(hb.data(), g->biglist, sizeof(int32_t) * nbig, cudaMemcpyDeviceToHost, s));
        PG_CUDA_TRY(ctx, cudaStreamSynchronize(s));
        std::vector<int32_t> huge;
        for (int64_t b0 = 0; b0 < nbig; b0 += cap_parents) {
            int32_t cnt_b = (int32_t)std::min<int64_t>(cap_parents, nbig - b0);
            Counters hc;
            // stage this batch into biglist[0..cnt_b)
            PG_CUDA_TRY(ctx, cudaMemcpyAsync(g->biglist, hb.data() + b0, sizeof(int32_t) * cnt_b,
                                             cudaMemcpyHostToDevice, s));
            PG_CUDA_TRY(ctx, cudaMemcpyAsync(&c->n_big, &cnt_b, sizeof(int32_t), cudaMemcpyHostToDevice, s));
            PG_CUDA_TRY(ctx, cudaMemsetAsync(&c->pad, 0, sizeof(int32_t), s));
            prof_begin(g, KID_BIG);
            k_big_mark<<<grid_for(cnt_b), kBlock, 0, s>>>(g->biglist, bigslot, c);
            k_big_collect<<<grid, kBlock, 0, s>>>(n, g->gd, g->kind, bigslot, bigfill, bigbuf, c);
            k_big_parents<<<(unsigned)std::min<int64_t>(cnt_b, 152 * 4), kBlock, 0, s>>>(
                g->biglist, bigslot, bigfill, bigbuf, g->sz, g->flags, g->wgt, g->oddsz, hugelist, c);
            prof_end(g, KID_BIG, 3);
            PG_CUDA_TRY(ctx, cudaMemcpyAsync(&hc, c, sizeof(Counters), cudaMemcpyDeviceToHost, s));
            PG_CUDA_TRY(ctx, cudaStreamSynchronize(s));
            prof_collect(g);
            if (hc.pad > 0) {
                size_t old = huge.size();
                huge.resize(old + hc.pad);
                PG_CUDA_TRY(ctx, cudaMemcpyAsync(huge.data() + old, hugelist, sizeof(int32_t) * hc.pad,
                                                 cudaMemcpyDeviceToHost, s));
                PG_CUDA_TRY(ctx, cudaStreamSynchronize(s));
            }
        }
        // huge parents: one id-ordered scan each
        for (int32_t p : huge) {
            ctx->launches += 3;
            k_idscan_reduce<false><<<(unsigned)g->ntiles, kBlock, 0, s>>>(n, p, g->kind, g->gd, g->sz, g->flags,
                                                                          g->scan_total);
            k_idscan_tiles<<<1, kBlock, 0, s>>>(g->scan_total, g->ntiles);
            k_idscan_apply<false><<<(unsigned)g->ntiles, kBlock, 0, s>>>(n, p, g->kind, g->gd, g->sz, g->flags,
                                                                         g->scan_total, g->ntiles, g->wgt,
                                                                         g->oddsz + p);
        }
    }
    // the sink's children
    prof_begin(g, KID_SINKSCAN);
    k_idscan_reduce<true><<<(unsigned)g->ntiles, kBlock, 0, s>>>(n, n, g->kind, g->gd, g->sz, g->flags,
                                                                 g->scan_total);
    k_idscan_tiles<<<1, kBlock, 0, s>>>(g->scan_total, g->ntiles);
    k_idscan_apply<true><<<(unsigned)g->ntiles, kBlock, 0, s>>>(n, n, g->kind, g->gd, g->sz, g->flags,
                                                                g->scan_total, g->ntiles, g->wgt, &c->sink_rank);
    prof_end(g, KID_SINKSCAN, 3);
    prof_begin(g, KID_CHAIN2);
    k_chain2<<<grid, kBlock, 0, s>>>(n, g->gd, g->kind, g->wgt, g->oddsz, g->key, g->sz, g->head, c);
    prof_end(g, KID_CHAIN2, 1);
    PG_CUDA_TRY(ctx, cudaMemcpyAsync(h, c, sizeof(Counters), cudaMemcpyDeviceToHost, s));
    PG_CUDA_TRY(ctx, cudaStreamSynchronize(s));
    prof_collect(g);
    PG_CUDA_TRY(ctx, cudaGetLastError());
    return PG_OK;
}

pg_status switch_device(pg_game* g, int player, int32_t* nswitch) {
    pg_ctx* ctx = g->ctx;
    cudaStream_t s = ctx->stream;
    PG_CUDA_TRY(ctx, cudaMemsetAsync(&g->cnt->n_switch, 0, sizeof(int32_t), s));
    int kid = player ? KID_SWITCH_ODD : KID_SWITCH_EVEN;
    prof_begin(g, kid);
    k_switch<<<grid_for(g->n), kBlock, 0, s>>>(g->n, player, g->off, g->tgt, g->flags, g->key, g->strat, g->cnt);
    prof_end(g, kid, 1);
    PG_CUDA_TRY(ctx, cudaMemcpyAsync(ctx->pinned, &g->cnt->n_switch, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    PG_CUDA_TRY(ctx, cudaStreamSynchronize(s));
    prof_collect(g);
    PG_CUDA_TRY(ctx, cudaGetLastError());
    *nswitch = ctx->pinned[0];
    return PG_OK;
}

}  // namespace pg
