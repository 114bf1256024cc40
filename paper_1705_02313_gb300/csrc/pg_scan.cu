// Device-wide exclusive scans (reduce-then-scan over 4096-element tiles).
// Used for CSR offsets, compaction indices, priority ranks and the children
// segments of every valuation. Tiles are read with 16-byte loads when the
// tile is full and aligned; the tile sums are scanned by one 1024-thread
// block.
#include "pg_internal.cuh"

namespace pg {
namespace {

constexpr int kIpt = 16;
constexpr int kTile = kBlock * kIpt;
constexpr int kTileScanThreads = 1024;

template <int NT>
__device__ inline int64_t block_exclusive(int64_t v, int64_t* total) {
    __shared__ int64_t wsum[NT / 32];
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
        int64_t w = lane < NT / 32 ? wsum[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int64_t y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < NT / 32) wsum[lane] = w;
    }
    __syncthreads();
    int64_t before = (wid > 0 ? wsum[wid - 1] : 0) + x - v;
    *total = wsum[NT / 32 - 1];
    __syncthreads();
    return before;
}

// Loaders: fill v[0..kIpt) for the kIpt consecutive elements starting at i0.
struct LoadI32 {
    const int32_t* p;
    __device__ void operator()(int64_t i0, int64_t n, int64_t v[kIpt]) const {
        if (i0 + kIpt <= n && ((reinterpret_cast<uintptr_t>(p + i0) & 15) == 0)) {
            const int4* q = reinterpret_cast<const int4*>(p + i0);
#pragma unroll
            for (int k = 0; k < kIpt / 4; ++k) {
                int4 a = __ldg(q + k);
                v[4 * k] = a.x;
                v[4 * k + 1] = a.y;
                v[4 * k + 2] = a.z;
                v[4 * k + 3] = a.w;
            }
        } else {
#pragma unroll
            for (int k = 0; k < kIpt; ++k) v[k] = i0 + k < n ? p[i0 + k] : 0;
        }
    }
};
struct LoadU8 {
    const uint8_t* p;
    __device__ void operator()(int64_t i0, int64_t n, int64_t v[kIpt]) const {
#pragma unroll
        for (int k = 0; k < kIpt; ++k) v[k] = (i0 + k < n) ? (p[i0 + k] != 0) : 0;
    }
};
struct LoadPopc {
    const uint32_t* p;
    __device__ void operator()(int64_t i0, int64_t n, int64_t v[kIpt]) const {
#pragma unroll
        for (int k = 0; k < kIpt; ++k) v[k] = (i0 + k < n) ? __popc(p[i0 + k]) : 0;
    }
};

template <typename L>
__global__ void __launch_bounds__(kBlock) k_tile_reduce(L ld, int64_t n, int64_t* tsum) {
    int64_t v[kIpt];
    ld((int64_t)blockIdx.x * kTile + (int64_t)threadIdx.x * kIpt, n, v);
    int64_t s = 0;
#pragma unroll
    for (int i = 0; i < kIpt; ++i) s += v[i];
    int64_t tot;
    block_exclusive<kBlock>(s, &tot);
    if (threadIdx.x == 0) tsum[blockIdx.x] = tot;
}

// Exclusive scan of the tile sums in place by one block; total in *total.
__global__ void __launch_bounds__(kTileScanThreads) k_scan_tiles(int64_t* tsum, int64_t ntiles, int64_t* total) {
    int64_t carry = 0;
    for (int64_t b = 0; b < ntiles; b += kTileScanThreads) {
        int64_t i = b + threadIdx.x;
        int64_t v = i < ntiles ? tsum[i] : 0;
        int64_t tot;
        int64_t ex = block_exclusive<kTileScanThreads>(v, &tot);
        if (i < ntiles) tsum[i] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0) *total = carry;
}

template <typename L>
__global__ void __launch_bounds__(kBlock) k_tile_scan(L ld, int64_t n, const int64_t* toff, int32_t* out,
                                                      const int64_t* total, int64_t write_total_at) {
    const int64_t i0 = (int64_t)blockIdx.x * kTile + (int64_t)threadIdx.x * kIpt;
    int64_t v[kIpt];
    ld(i0, n, v);
    int64_t s = 0;
#pragma unroll
    for (int i = 0; i < kIpt; ++i) s += v[i];
    int64_t tot;
    int64_t run = toff[blockIdx.x] + block_exclusive<kBlock>(s, &tot);
    if (i0 + kIpt <= n && ((reinterpret_cast<uintptr_t>(out + i0) & 15) == 0)) {
        int4* q = reinterpret_cast<int4*>(out + i0);
#pragma unroll
        for (int k = 0; k < kIpt / 4; ++k) {
            int4 a;
            a.x = (int32_t)run;
            run += v[4 * k];
            a.y = (int32_t)run;
            run += v[4 * k + 1];
            a.z = (int32_t)run;
            run += v[4 * k + 2];
            a.w = (int32_t)run;
            run += v[4 * k + 3];
            q[k] = a;
        }
    } else {
#pragma unroll
        for (int k = 0; k < kIpt; ++k) {
            if (i0 + k < n) out[i0 + k] = (int32_t)run;
            run += v[k];
        }
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
    k_scan_tiles<<<1, kTileScanThreads, 0, s>>>(tsum, ntiles, total);
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
