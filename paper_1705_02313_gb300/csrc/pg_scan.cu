// Device-wide exclusive scans (reduce-then-scan over 2048-element tiles).
// Used for CSR offsets, compaction indices and priority ranks; the
// list-ranking-like passes of the valuation have their own kernels.
#include "pg_internal.cuh"

namespace pg {
namespace {

constexpr int kIpt = 8;
constexpr int kTile = kBlock * kIpt;

__device__ inline int64_t warp_sum(int64_t v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Exclusive block scan of one value per thread; returns the exclusive prefix,
// *total gets the block sum.
__device__ inline int64_t block_exclusive(int64_t v, int64_t* total) {
    __shared__ int64_t wsum[kBlock / 32];
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int64_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int64_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int64_t w = lane < kBlock / 32 ? wsum[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int64_t y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < kBlock / 32) wsum[lane] = w;
    }
    __syncthreads();
    int64_t before = (wid > 0 ? wsum[wid - 1] : 0) + x - v;
    *total = wsum[kBlock / 32 - 1];
    __syncthreads();
    return before;
}

struct LoadI32 {
    const int32_t* p;
    __device__ int64_t operator()(int64_t i) const { return p[i]; }
};
struct LoadU8 {
    const uint8_t* p;
    __device__ int64_t operator()(int64_t i) const { return p[i] != 0; }
};
struct LoadPopc {
    const uint32_t* p;
    __device__ int64_t operator()(int64_t i) const { return __popc(p[i]); }
};

template <typename L>
__global__ void k_tile_reduce(L ld, int64_t n, int64_t* tsum) {
    int64_t base = (int64_t)blockIdx.x * kTile + (int64_t)threadIdx.x * kIpt;
    int64_t s = 0;
#pragma unroll
    for (int i = 0; i < kIpt; ++i)
        if (base + i < n) s += ld(base + i);
    int64_t tot;
    block_exclusive(s, &tot);
    if (threadIdx.x == 0) tsum[blockIdx.x] = tot;
}

// Exclusive scan of the tile sums in place by one block; total in *total.
__global__ void k_scan_tiles(int64_t* tsum, int64_t ntiles, int64_t* total) {
    int64_t carry = 0;
    for (int64_t b = 0; b < ntiles; b += kBlock) {
        int64_t i = b + threadIdx.x;
        int64_t v = i < ntiles ? tsum[i] : 0;
        int64_t tot;
        int64_t ex = block_exclusive(v, &tot);
        if (i < ntiles) tsum[i] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0) *total = carry;
}

template <typename L>
__global__ void k_tile_scan(L ld, int64_t n, const int64_t* toff, int32_t* out, const int64_t* total,
                            int64_t write_total_at) {
    int64_t base = (int64_t)blockIdx.x * kTile + (int64_t)threadIdx.x * kIpt;
    int64_t vals[kIpt];
    int64_t s = 0;
#pragma unroll
    for (int i = 0; i < kIpt; ++i) {
        vals[i] = (base + i < n) ? ld(base + i) : 0;
        s += vals[i];
    }
    int64_t tot;
    int64_t run = toff[blockIdx.x] + block_exclusive(s, &tot);
#pragma unroll
    for (int i = 0; i < kIpt; ++i) {
        if (base + i < n) out[base + i] = (int32_t)run;
        run += vals[i];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0 && write_total_at >= 0) out[write_total_at] = (int32_t)*total;
}

template <typename L>
cudaError_t scan_impl(L ld, int64_t n, int32_t* out, int64_t write_total_at, int64_t* total_dev, void* tmp,
                      size_t tmp_bytes, cudaStream_t s) {
    int64_t ntiles = (n + kTile - 1) / kTile;
    if (ntiles == 0) ntiles = 1;
    if (tmp_bytes < (size_t)(ntiles + 1) * sizeof(int64_t)) return cudaErrorInvalidValue;
    int64_t* tsum = (int64_t*)tmp;
    int64_t* total = total_dev ? total_dev : tsum + ntiles;
    k_tile_reduce<<<(unsigned)ntiles, kBlock, 0, s>>>(ld, n, tsum);
    k_scan_tiles<<<1, kBlock, 0, s>>>(tsum, ntiles, total);
    k_tile_scan<<<(unsigned)ntiles, kBlock, 0, s>>>(ld, n, tsum, out, total, write_total_at);
    return cudaGetLastError();
}

}  // namespace

size_t scan_tmp_bytes(int64_t n) { return (size_t)((n + kTile - 1) / kTile + 2) * sizeof(int64_t); }

cudaError_t exclusive_scan_i32(const int32_t* in, int32_t* out, int64_t n, int64_t* total_dev, void* tmp,
                               size_t tmp_bytes, cudaStream_t s) {
    return scan_impl(LoadI32{in}, n, out, n, total_dev, tmp, tmp_bytes, s);
}

cudaError_t exclusive_scan_u8(const uint8_t* in, int32_t* out, int64_t n, void* tmp, size_t tmp_bytes,
                              cudaStream_t s) {
    return scan_impl(LoadU8{in}, n, out, n, nullptr, tmp, tmp_bytes, s);
}

cudaError_t exclusive_popc_scan(const uint32_t* words, int32_t* out, int64_t nwords, void* tmp, size_t tmp_bytes,
                                cudaStream_t s) {
    return scan_impl(LoadPopc{words}, nwords, out, nwords, nullptr, tmp, tmp_bytes, s);
}

}  // namespace pg
