// Device helpers shared by the valuation translation units (pg_iter.cu,
// pg_deep.cu): launch shapes, warp and block reductions, the compact
// nearest-greater word, the software grid barrier of the cooperative kernels.
#pragma once

#include "pg_internal.cuh"

namespace pg {
namespace {

constexpr unsigned kFull = 0xffffffffu;

inline unsigned ilp_grid(int64_t n) {
    int64_t tiles = (n + 32 * 4 - 1) / (32 * 4);
    int64_t b = (tiles + kBlock / 32 - 1) / (kBlock / 32);
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(b, 152 * 64));
}

inline unsigned grid_for(int64_t n) {
    int64_t b = (n + kBlock - 1) / kBlock;
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(b, 152 * 64));
}

// All 32 lanes must call this (uniform control flow).
__device__ inline int32_t warp_append(bool pred, int32_t* counter) {
    unsigned m = __ballot_sync(kFull, pred);
    if (!m) return -1;
    int lane = threadIdx.x & 31;
    int leader = __ffs(m) - 1;
    int32_t base = 0;
    if (lane == leader) base = atomicAdd(counter, __popc(m));
    base = __shfl_sync(kFull, base, leader);
    return pred ? base + __popc(m & ((1u << lane) - 1u)) : -1;
}

__device__ inline void block_add(int32_t v, int32_t* counter) {
    __shared__ int32_t acc;
    if (threadIdx.x == 0) acc = 0;
    __syncthreads();
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(kFull, v, o);
    if ((threadIdx.x & 31) == 0 && v) atomicAdd(&acc, v);
    __syncthreads();
    if (threadIdx.x == 0 && acc) atomicAdd(counter, acc);
}

__device__ inline uint64_t ld_cg(const uint64_t* p) { return __ldcg((const unsigned long long*)p); }
__device__ inline void st_cg(uint64_t* p, uint64_t v) { __stcg((unsigned long long*)p, (unsigned long long)v); }

// Compact g-word read by every chain pass: bit 31 = "none" (v is above its
// whole infinite future; the low bits then name the cycle maximum), bit 30 =
// g(v) is the game's sink, low 30 bits = g(v) (ids < 2^30).
constexpr uint32_t kG32None = 0x80000000u;
constexpr uint32_t kG32Sink = 0x40000000u;
__device__ inline uint32_t g32_of(uint64_t w) {
    return (gd_none(w) ? kG32None : 0u) | (gd_sink(w) ? kG32Sink : 0u) | (uint32_t)gd_ptr(w);
}
__device__ inline bool g32_none(uint32_t w) { return (w & kG32None) != 0; }
__device__ inline bool g32_sink(uint32_t w) { return (w & kG32Sink) != 0; }
__device__ inline int32_t g32_ptr(uint32_t w) { return (int32_t)(w & 0x3fffffffu); }

// The sink slot of v's game.
__device__ inline int32_t sink_of(int32_t v, const int32_t* vgame, const int32_t* gsink, int32_t sink0) {
    return vgame ? gsink[vgame[v]] : sink0;
}

// kind[v], written by k_chain1
constexpr uint8_t kKFin = 1;        // finite valuation
constexpr uint8_t kKSinkChild = 2;  // g(v) is the sink
constexpr uint8_t kKOdd = 4;        // odd priority
constexpr uint8_t kKSinkSlot = 8;   // the id is a sink slot

// Software grid barrier for cooperative launches (all blocks co-resident).
// Gives up after a bounded number of spins, records kErrBarrier and returns
// false; the caller then returns.
__device__ bool grid_sync(Counters* c) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        ok = 1;
        volatile uint32_t* genp = &c->bar_gen;
        uint32_t gen = *genp;
        __threadfence();
        uint32_t arrived = atomicAdd(&c->bar_count, 1u);
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

// ---------------------------------------------------------------------------
// Pointer-chasing passes give each thread kIlp vertices, v + 32 j for
// j < kIlp within a warp tile of 32 kIlp vertices: per-vertex reads and writes
// stay coalesced for every j, and the walks of one thread issue their gathers
// together, so each thread keeps kIlp loads in flight.
constexpr int kIlp = 4;

__device__ inline int64_t warp_tile_base(int64_t tile) { return tile * 32 * kIlp; }

}  // namespace
}  // namespace pg
