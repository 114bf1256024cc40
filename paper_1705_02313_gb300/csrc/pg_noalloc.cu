// pg_valuate_static: the valuation of one successor function with every
// piece of working memory taken from a fixed array compiled into the library,
// for callers that cannot allocate device memory (see include/pg.h).
//
// The working memory is one file-scope device array of kStaticBytes bytes,
// sized for kStaticMaxN vertices. Host code cannot use the array's name as a
// device address, so every call looks the address up with
// cudaGetSymbolAddress (with the call's device current; the lookup allocates
// nothing, and a context made after a device reset gets the new address). The call
// then lays out the valuation's arrays inside the static buffer, copies the
// successor function into it (a successor outside [0, n] is recorded and
// replaced by the sink, so no kernel reads out of bounds), runs the same
// kernels as pg_valuate on the copy, writes class, depth and rank into the
// caller's arrays and waits for its stream once, at the end, to read the
// error words. No device or host memory is allocated on any path; error
// messages are not recorded (only the status is returned).
#include <mutex>

#include "pg_internal.cuh"

namespace pg {
namespace {

constexpr int32_t kStaticMaxN = 1 << 18;
constexpr int kMaxDevices = 64;

constexpr size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

// Byte offsets of the arrays inside the static buffer, for kStaticMaxN vertices.
struct Layout {
    size_t succ, bad, gd, gd32, plist, slot, ccnt, coff, cl_ks, sz, sinkval, wgt, oddsz, key, cls, kind, depth, hugelist,
        flags, tiles, tsum, gst, gscan, gsink, cnt, scan, bytes;
};

constexpr Layout make_layout() {
    const size_t N = kStaticMaxN + 1;  // the vertices and the sink slot
    const size_t ntiles = (N + kCoopTile - 1) / kCoopTile;
    Layout L{};
    size_t p = 0;
    L.succ = p;     p = al256(p + 4 * N);
    L.bad = p;      p = al256(p + 4);
    L.gd = p;       p = al256(p + 8 * N);
    L.gd32 = p;     p = al256(p + 4 * N);
    L.plist = p;    p = al256(p + 4 * N);
    L.slot = p;     p = al256(p + 4 * N);
    L.ccnt = p;     p = al256(p + 4 * (N + 1));
    L.coff = p;     p = al256(p + 4 * (N + 2));
    L.cl_ks = p;    p = al256(p + 8 * N);
    L.sz = p;       p = al256(p + 4 * N);
    L.sinkval = p;  p = al256(p + 4 * N);
    L.wgt = p;      p = al256(p + 4 * N);
    L.oddsz = p;    p = al256(p + 4 * N);
    L.key = p;      p = al256(p + 4 * (N + 1));
    L.cls = p;      p = al256(p + N);
    L.kind = p;     p = al256(p + N);
    L.depth = p;    p = al256(p + 4 * N);
    L.hugelist = p; p = al256(p + 4 * N);
    L.flags = p;    p = al256(p + N);
    L.tiles = p;    p = al256(p + 8 * (2 * ntiles + 2));
    L.tsum = p;     p = al256(p + 8 * (2 * ntiles + 2));
    L.gst = p;      p = al256(p + sizeof(GameState));
    L.gscan = p;    p = al256(p + 3 * 8);
    L.gsink = p;    p = al256(p + 4);
    L.cnt = p;      p = al256(p + sizeof(Counters));
    L.scan = p;     p = al256(p + 8 * ((N + 2 + 2047) / 2048 + 2) + 64);
    L.bytes = p;
    return L;
}

constexpr Layout kLayout = make_layout();
constexpr size_t kStaticBytes = kLayout.bytes;

// Every call shares this buffer; it keeps the last call's contents.
static __device__ __align__(256) unsigned char g_static_scratch[kStaticBytes];

int g_static_coop[kMaxDevices] = {};
int g_static_chain1[kMaxDevices] = {};
std::mutex g_static_mu;
Counters g_static_hcnt;  // host copies of the counters and of the range-check word (pageable, fixed)
int32_t g_static_hbad;

// Copies the successor function into the buffer, sets the flags and checks
// the range: a successor outside [0, n] is counted in *bad and replaced by
// the sink (id n is the sink slot), so that no later kernel reads outside the
// buffer. *bad must be zero before the launch.
__global__ void k_static_prepare(int32_t n, const int32_t* __restrict__ succ, const uint8_t* __restrict__ odd,
                                 int32_t* __restrict__ succ_copy, uint8_t* __restrict__ flags, int32_t* gsink,
                                 int32_t* bad) {
    for (int32_t v = blockIdx.x * blockDim.x + threadIdx.x; v <= n; v += gridDim.x * blockDim.x) {
        if (v == n) {
            flags[v] = kSinkSlot;
            succ_copy[v] = n;
            *gsink = n;
            continue;
        }
        int32_t s = succ[v];
        if (s < 0 || s > n) {
            atomicAdd(bad, 1);
            s = n;
        }
        succ_copy[v] = s;
        flags[v] = odd[v] ? kPriOdd : 0;
    }
}

__global__ void k_static_results(int32_t n, const uint8_t* __restrict__ cls, const int32_t* __restrict__ depth,
                                 const int32_t* __restrict__ key, int8_t* val_class, int32_t* val_depth,
                                 int32_t* val_rank) {
    for (int32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        const bool fin = cls[v] == kFin;
        if (val_class) val_class[v] = fin ? 0 : 1;
        if (val_depth) val_depth[v] = fin ? depth[v] : -1;
        if (val_rank) val_rank[v] = fin ? key[v] : INT32_MAX;
    }
}

// Device address of the static buffer on the current device (looked up on
// every call), and the launch sizes (computed once per device: they depend on
// the device's SM count and the kernels' resources only).
pg_status static_setup(pg_ctx* ctx, unsigned char** base, int* coop, int* chain1) {
    std::lock_guard<std::mutex> lock(g_static_mu);
    if (ctx->device < 0 || ctx->device >= kMaxDevices) return PG_EUNSUPPORTED;
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess || p == nullptr) return PG_ECUDA;
    if (!g_static_coop[ctx->device]) {
        int cb = 0, c1 = 0;
        if (coop_blocks_for(ctx, &cb) != PG_OK || chain1_blocks_for(ctx, &c1) != PG_OK) return PG_ECUDA;
        g_static_chain1[ctx->device] = c1;
        g_static_coop[ctx->device] = cb;
    }
    *base = (unsigned char*)p;
    *coop = g_static_coop[ctx->device];
    *chain1 = g_static_chain1[ctx->device];
    return PG_OK;
}

}  // namespace
}  // namespace pg

using namespace pg;

extern "C" pg_status pg_valuate_static(int32_t n, const int32_t* succ, const uint8_t* odd, int8_t* val_class,
                                       int32_t* val_depth, int32_t* val_rank, void* stream) {
    if (n < 1 || !succ || !odd) return PG_EINVAL;
    if (n > kStaticMaxN) return PG_EUNSUPPORTED;
    int device = 0;
    if (cudaGetDevice(&device) != cudaSuccess) return PG_ECUDA;

    pg_ctx ctx;  // on the stack; quiet: no message strings are built
    ctx.device = device;
    ctx.stream = (cudaStream_t)stream;
    ctx.quiet = true;
    ctx.tune.deep_cut = INT32_MAX;  // no ruling-set path here (its scratch is not in the fixed array)
    ctx.deep_fallback = false;
    unsigned char* base = nullptr;
    int coop = 0, chain1 = 0;
    pg_status st = static_setup(&ctx, &base, &coop, &chain1);
    if (st != PG_OK) return st;

    // a game view over the static buffer: only the fields the valuation reads
    pg_game g;
    g.ctx = &ctx;
    g.n = n + 1;  // the vertices and the sink slot
    g.sink0 = n;
    g.ngames = 1;
    g.strat = (int32_t*)(base + kLayout.succ);  // the checked copy of succ
    g.gd = (uint64_t*)(base + kLayout.gd);
    g.gd32 = (uint32_t*)(base + kLayout.gd32);
    g.plist = (int32_t*)(base + kLayout.plist);
    g.slot = (int32_t*)(base + kLayout.slot);
    g.ccnt = (int32_t*)(base + kLayout.ccnt);
    g.coff = (int32_t*)(base + kLayout.coff);
    g.cl_ks = (int2*)(base + kLayout.cl_ks);
    g.sz = (int32_t*)(base + kLayout.sz);
    g.sinkval = (int32_t*)(base + kLayout.sinkval);
    g.wgt = (int32_t*)(base + kLayout.wgt);
    g.oddsz = (int32_t*)(base + kLayout.oddsz);
    g.key = (int32_t*)(base + kLayout.key);
    g.cls = (uint8_t*)(base + kLayout.cls);
    g.kind = (uint8_t*)(base + kLayout.kind);
    g.depth = (int32_t*)(base + kLayout.depth);
    g.hugelist = (int32_t*)(base + kLayout.hugelist);
    g.flags = (uint8_t*)(base + kLayout.flags);
    g.tiles = (int64_t*)(base + kLayout.tiles);
    g.tsum = (int64_t*)(base + kLayout.tsum);
    g.ntiles = std::max<int64_t>(1, ((int64_t)n + 1 + kCoopTile - 1) / kCoopTile);
    g.gst = (GameState*)(base + kLayout.gst);
    g.gscan = (int64_t*)(base + kLayout.gscan);
    g.gsink = (int32_t*)(base + kLayout.gsink);
    g.cnt = (Counters*)(base + kLayout.cnt);
    g.hcnt = &g_static_hcnt;
    g.scan_tmp = base + kLayout.scan;
    g.scan_tmp_bytes = kLayout.bytes - kLayout.scan;
    g.coop_blocks = coop;
    g.chain1_blocks = chain1;

    cudaStream_t s = ctx.stream;
    int32_t* bad = (int32_t*)(base + kLayout.bad);
    if (cudaMemsetAsync(bad, 0, sizeof(int32_t), s) != cudaSuccess) return PG_ECUDA;
    k_static_prepare<<<(unsigned)std::min<int64_t>(((int64_t)n + kBlock) / kBlock, 4096), kBlock, 0, s>>>(
        n, succ, odd, g.strat, g.flags, g.gsink, bad);
    if (cudaGetLastError() != cudaSuccess) return PG_ECUDA;

    st = reset_scratch(&g);  // the buffer keeps the previous call's contents
    if (st == PG_OK) st = enqueue_valuation(&g, false);
    if (st == PG_OK) st = enqueue_depth(&g);
    if (st != PG_OK) return st;
    k_static_results<<<(unsigned)std::min<int64_t>(((int64_t)n + kBlock - 1) / kBlock, 4096), kBlock, 0, s>>>(
        n, g.cls, g.depth, g.key, val_class, val_depth, val_rank);
    if (cudaGetLastError() != cudaSuccess) return PG_ECUDA;
    // the one wait of the call: the range-check word, then the counters (sync_counters waits for the stream)
    if (cudaMemcpyAsync(&g_static_hbad, bad, sizeof(int32_t), cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return PG_ECUDA;
    st = sync_counters(&g);
    if (st != PG_OK) return st;
    if (g_static_hbad) return PG_EINVAL;
    return g_static_hcnt.n_odd > 0 ? PG_ENOTADMISSIBLE : PG_OK;
}
