// Internal declarations of libpg (GB300, sm_103a).
//
// Device layout of a loaded game. After the admissibility preprocessing
// (Section 3) the game G' has n vertices; they are relabelled so that a
// vertex id is the rank of its priority among all n priorities (priorities
// are pairwise distinct). "Higher priority" is then "larger id", the parity
// of the priority is kept in a flag bit, and the sink is the id n, above
// every vertex, which is what the nearest-greater-ancestor walks need.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <string>
#include <vector>

#include "pg.h"

namespace pg {

constexpr int kBlock = 256;
constexpr int kWalkCap = 64;          // steps of a direct nearest-greater walk before pointer jumping takes over
constexpr int kWalkShort = 8;         // steps of the first walk pass; longer walks continue in a dense second pass
constexpr int kJumpFollow = 32;       // resolved vertices a pointer-jumping round may pass through at once
constexpr int kJumpRoundsDeep = 4096; // extra pointer-jumping rounds allowed on the ruling-set path
constexpr int kHugeChildren = 4096;   // a parent with more children is ranked by an id-ordered scan instead
constexpr int kCoopTile = 4096;       // elements per tile of the id-ordered scans
// Count-vector mode (repeated priorities): at most kMaxLevels distinct
// priorities; a count vector is one signed 128-bit key with one digit per
// level (Levels::shift), each wide enough that its signed count stays below
// half the digit's range (so the key order is the order of Section 3), all
// within kKeyBits bits (the top key stays above every finite one).
constexpr int kMaxLevels = 5;
constexpr int kKeyBits = 126;

// flags[v]
constexpr uint8_t kOwnerOdd = 1;   // owner is Odd
constexpr uint8_t kPriOdd = 2;     // priority is odd
constexpr uint8_t kSinkSlot = 4;   // the id is a game's sink slot, not a vertex

// cls[v]
constexpr uint8_t kFin = 0;
constexpr uint8_t kTop = 1;
constexpr uint8_t kOddCycle = 2;

// Packed nearest-greater-ancestor word gd[v]:
//   bits 0..31  ptr  (a vertex id, the game's sink slot, or for "none" vertices the id of the cycle maximum)
//   bits 32..60 dist (number of steps from v to ptr along the successor function)
//   bit  61     sink (ptr is the game's sink slot)
//   bit  62     none (v is above every vertex of its infinite future)
//   bit  63     resolved (ptr is final; otherwise ptr is a jump pointer: every vertex strictly between v and ptr is below v)
constexpr uint64_t kResolved = 1ull << 63;
constexpr uint64_t kNone = 1ull << 62;
constexpr uint64_t kSinkBit = 1ull << 61;
constexpr uint32_t kDistMax = 0x1fffffffu;
__host__ __device__ inline uint64_t gd_pack(bool resolved, bool none, uint32_t dist, int32_t ptr, bool sink = false) {
    return (resolved ? kResolved : 0ull) | (none ? kNone : 0ull) | (sink ? kSinkBit : 0ull) |
           ((uint64_t)(dist & kDistMax) << 32) | (uint64_t)(uint32_t)ptr;
}
__host__ __device__ inline int32_t gd_ptr(uint64_t w) { return (int32_t)(uint32_t)(w & 0xffffffffull); }
__host__ __device__ inline uint32_t gd_dist(uint64_t w) { return (uint32_t)((w >> 32) & kDistMax); }
__host__ __device__ inline bool gd_sink(uint64_t w) { return (w & kSinkBit) != 0; }
__host__ __device__ inline bool gd_resolved(uint64_t w) { return (w & kResolved) != 0; }
__host__ __device__ inline bool gd_none(uint64_t w) { return (w & kNone) != 0; }

// kind[v] written by the first chain pass
constexpr uint8_t kKindFin = 1;        // finite valuation
constexpr uint8_t kKindSinkChild = 2;  // nearest greater ancestor is the sink

// Device counters of one valuation (reset at its start).
struct Counters {
    int32_t n_pending;   // walks that ran out of steps (length of the pending list)
    int32_t n_walk2;     // walks continued by the second walk pass
    int32_t left[3];     // pending vertices left after a jump round (three rotating counters)
    int32_t n_fin;       // finite vertices
    int32_t n_odd;       // vertices reaching an odd cycle (all games)
    int32_t n_huge;      // parents ranked by the id-ordered scan
    int32_t n_big;       // parents ranked by one block each
    int32_t n_switch;    // switched vertices in the last switching pass (all games)
    int32_t err;         // device-side error bits (kErr*)
    int32_t sink_rank;   // rank of game 0's sink (its empty valuation)
    uint32_t bar_count;  // software grid barrier
    uint32_t bar_gen;
    int32_t jump_rounds;
    int32_t deep;         // a chain walk passed the cutover depth: the valuation needs the ruling-set path
    int32_t n_dlist;      // ruling-set path: vertices whose root is found by pointer jumping
    int32_t deep_rounds;  //   rounds of that pointer jumping
    int32_t n_dmid;       //   segments sorted in shared memory
    int32_t n_dbig;       //   segments sorted by the global-memory radix sort
    int32_t n_rulers;     //   rulers of the list ranking
    int32_t rs_rounds;    //   pointer-jumping rounds over the rulers
    int32_t rs_buf;       //   the buffer holding the rulers' suffix sums
};
constexpr int32_t kErrJumpRounds = 1;   // pointer jumping exceeded its round cap
constexpr int32_t kErrBarrier = 2;      // a grid barrier waited past its spin limit
constexpr int32_t kErrRulers = 4;       // the list ranking's rulers overflowed their scratch, or a sublist never ended

// Kernel classes of one iteration, for per-kernel device timing.
enum KernelId {
    KID_WALK,        // k_walk
    KID_JUMP,        // k_jump_coop (all rounds)
    KID_CHAIN1,      // k_chain1
    KID_CSCAN,       // children-count scan (3 kernels)
    KID_SCATTER,     // k_scatter
    KID_SIBLINGS,    // k_siblings
    KID_SINKSCAN,    // the sink's id-ordered scan (and k_idscan_coop for huge parents)
    KID_CHAIN2,      // k_chain2
    KID_SWITCH_ODD,  // k_switch for Odd
    KID_SWITCH_EVEN, // k_switch for Even
    KID_CLASSIFY,    // k_classify (loop iterations that compare valuations instead of ranking them)
    KID_DEEP,        // the ruling-set ranks of a deep g-forest (pg_deep.cu), after K1
    KID_COUNT
};
extern const char* const kKernelNames[KID_COUNT];

// scan helpers (pg_scan.cu)
// Exclusive scan of in[0..n) into out[0..n], out[n] = total; int64 accumulation, int32 output.
cudaError_t exclusive_scan_i32(const int32_t* in, int32_t* out, int64_t n, int64_t* total_dev, void* tmp,
                               size_t tmp_bytes, cudaStream_t s);
size_t scan_tmp_bytes(int64_t n);
// Exclusive scan of 0/1 bytes.
cudaError_t exclusive_scan_u8(const uint8_t* in, int32_t* out, int64_t n, void* tmp, size_t tmp_bytes,
                              cudaStream_t s);
// Exclusive popcount scan over 32-bit words: out[i] = popcount of words[0..i).
cudaError_t exclusive_popc_scan(const uint32_t* words, int32_t* out, int64_t nwords, void* tmp,
                                size_t tmp_bytes, cudaStream_t s);

// Work partitioning of the valuation (pg_set_tuning). Results never depend on it.
struct Tune {
    int64_t max_ids = INT64_MAX;  // a table entry applies to games (batches) of at most this many ids
    int32_t deep_cut = 64;        // a g-chain walk longer than this switches the call to the ruling-set ranks
    int32_t ruler_bits = 5;       // the ruling set takes about one list element in 2^ruler_bits as a ruler
    int32_t walk_cap = kWalkCap;  // steps of a direct nearest-greater walk before pointer jumping (16..128)
    int32_t switch_block = kBlock;// threads per block of the compare-mode switching passes (128, 256, 512)
    int32_t loop_ranks = 0;       // loop iterations rank every valuation (else they only compare them)
    bool operator==(const Tune& o) const {
        return deep_cut == o.deep_cut && ruler_bits == o.ruler_bits && walk_cap == o.walk_cap &&
               switch_block == o.switch_block && loop_ranks == o.loop_ranks;
    }
};

}  // namespace pg

// Library objects
struct pg_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    std::string err = "no error";
    bool timing = false;
    int32_t* pinned = nullptr;  // small pinned host buffer for counters
    int64_t launches = 0;       // kernels launched through this context
    bool quiet = false;         // record no error message (keeps failing calls free of host allocation)
    bool graphs = true;         // run the iteration loop as one CUDA graph with a device-side condition
    bool wide_offsets = false;  // batches take 64-bit edge offsets at any size (else from 2^31 edges)
    pg::Tune tune;              // partitioning of games beyond every table entry (pg_set_tuning)
    std::vector<pg::Tune> tune_table;  // by increasing max_ids (pg_set_tuning_table, pg_load_tuning)
    bool deep_fallback = true;  // a deep forest or unfinished jumping hands over to the ruling-set path
    cudaStream_t cap_stream = nullptr;  // private stream on which loop graphs are captured
};

// Per-game state of Algorithm 1 on the device (one entry per game of a batch).
namespace pg {
struct GameState {
    int32_t phase;    // kPhaseActive, kPhaseDone, kPhaseOddCycle, kPhaseTimeout
    int32_t sw_odd;   // Odd switches in this iteration
    int32_t sw_even;  // Even switches in this iteration
    int32_t nodd;     // vertices reaching an odd cycle in this iteration's valuation
    int32_t reset;    // Even switched and Odd restarts from its initial strategy (SI-Reset, Section 6)
    int64_t inner;    // valuations computed
    int64_t major;    // Even switching rounds that switched something
};
constexpr int32_t kPhaseActive = 0, kPhaseDone = 1, kPhaseOddCycle = 2, kPhaseTimeout = 3;
}  // namespace pg

// Levels of a count-vector game: ids [start[l], start[l+1]) have the l-th
// smallest priority; bit l of odd_mask is that priority's parity.
struct Levels {
    int32_t n;
    uint32_t odd_mask;
    int32_t start[pg::kMaxLevels + 1];
    int32_t shift[pg::kMaxLevels + 1];  // bit offset of level l's digit; shift[l+1] - shift[l] = its width, one bit
                                        // more than the bit length of the level's size, so every signed count
                                        // of level l lies in (-2^(width-1), 2^(width-1))
};

// A loaded game, or a batch of games packed into one id space. Every game's
// relabelled G' vertices occupy a contiguous id range followed by one "sink
// slot" id that stands for that game's sink (greater than every vertex of the
// game, as the nearest-greater walks need). A single game is a batch of one.
struct pg_game {
    pg_ctx* ctx = nullptr;
    int device = 0;   // the device holding the game's memory
    int32_t ngames = 1;
    int64_t n0 = 0;   // original vertices, all games
    int64_t m0 = 0;   // original edges, all games
    int32_t k = 0;    // dummies, all games
    int32_t n = 0;    // ids: G' vertices of all games plus one sink slot per game
    int64_t m = 0;    // edges of all G'
    int32_t sink0 = 0;           // the sink slot of game 0 (the only one for a single game)
    // count-vector mode (repeated priorities; single games only)
    bool cv = false;
    Levels lev{};
    int32_t lev_pri[pg::kMaxLevels] = {};  // the G' priority of each level
    __int128* ws = nullptr;      // [n] key weight of the walk segment [v, g(v))
    __int128* wsB = nullptr;     // [n] second buffer of the pointer-jumping rounds
    uint64_t* gdB = nullptr;     // [n] second buffer of the nearest-greater words
    __int128* key128 = nullptr;  // [n] count-vector key; a sink slot holds 0
    // packed relabelled G'
    int32_t* off = nullptr;      // [n+1] int32 edge offsets (when m < 2^31), else off64
    int64_t* off64 = nullptr;    // [n+1]
    int32_t* tgt = nullptr;      // [m]
    uint8_t* flags = nullptr;    // [n] owner, priority parity, sink slot
    int32_t* pri = nullptr;      // [n] priority in G' (-1 for sink slots)
    int32_t* nid0 = nullptr;     // [n0] packed original vertex -> id
    int32_t* orig_of = nullptr;  // [n] id -> original vertex within its game (a dummy reports the vertex it guards)
    int32_t* dnid = nullptr;     // [k] packed dummy index -> id
    int32_t* dummy_of = nullptr; // [k] packed dummy index -> original vertex it guards, within its game
    int32_t* vgame = nullptr;    // [n] game of each id; nullptr for a single game
    int32_t* gsink = nullptr;    // [ngames] sink slot id of each game
    pg::GameState* gst = nullptr;// [ngames]
    int32_t* gactive = nullptr;  // [1] active games after the last bookkeeping pass
    std::vector<int64_t> h_base0;  // host: original vertex base of each game (ngames + 1)
    std::vector<int32_t> h_dbase;  // host: dummy base of each game (ngames + 1)
    // solver state
    int32_t* strat = nullptr;    // [n] successor under the current profile (a sink slot for the sink)
    // per-valuation scratch
    uint64_t* gd = nullptr;      // [n] nearest-greater words (pointer, walk length, flags)
    uint32_t* gd32 = nullptr;    // [n] compact g-words read by the chain passes
    uint8_t* kind = nullptr;     // [n] finite / sink child / odd priority
    int32_t* plist = nullptr;    // [n] pending list
    int32_t* slot = nullptr;     // [n] slot of v among its g-parent's children, -1 if none
    int32_t* ccnt = nullptr;     // [n+1] children per parent (zero between valuations)
    int32_t* coff = nullptr;     // [n+2] children segment offsets
    int2* cl_ks = nullptr;       // [n] per child slot: (order key, subtree size)
    int32_t* sz = nullptr;       // [n] proper descendants in the g-forest
    int32_t* sinkval = nullptr;  // [n] sink children: subtree size | odd << 31; 0 otherwise
    int32_t* wgt = nullptr;      // [n] chain weight: [even] + sizes of siblings ordered before
    int32_t* oddsz = nullptr;    // [n] sizes of odd children
    int32_t* key = nullptr;      // [n] rank; INT32_MAX for TOP; a sink slot holds its sink's rank
    uint8_t* cls = nullptr;      // [n]
    int32_t* depth = nullptr;    // [n]
    int32_t* dom = nullptr;      // [n] dominant priority of the cycle reached (TOP), -1 finite
    int32_t* hugelist = nullptr; // [n] parents with more than kHugeChildren children
    int64_t* tiles = nullptr;    // [2 * ntiles + 2] id-ordered scan tile sums
    int64_t* tsum = nullptr;     // [2 * ntiles + 2] (even, odd) sizes of the sink's children per tile, summed by k_scatter
    int64_t ntiles = 0;
    int64_t* gscan = nullptr;    // [3 * ngames] per game: even and odd prefix at its first id, odd prefix at its sink
    pg::Counters* cnt = nullptr; // device counters
    pg::Counters* hcnt = nullptr;// pinned host copy
    void* scan_tmp = nullptr;    // children-count scan scratch
    size_t scan_tmp_bytes = 0;
    int coop_blocks = 0;         // co-resident blocks for the cooperative kernels
    int chain1_blocks = 0;       // k_chain1 blocks resident at once (0: one block per 8 tiles)
    void* stage = nullptr;       // staging for host outputs
    int64_t* loop_iters = nullptr;  // [1] iterations run by the device-side loop
    // instantiated loop graphs: [0] inner loop only, [1] both players; built for loop_cap[i]
    cudaGraphExec_t loop_exec[2] = {nullptr, nullptr};
    int64_t loop_cap[2] = {0, 0};
    int64_t loop_limit[2] = {0, 0};
    int64_t loop_launch[2] = {0, 0};                  // kernels per iteration of each graph
    int64_t loop_klaunch[2][pg::KID_COUNT] = {};      // per kernel class
    bool last_graph = false;     // the last loop ran as a graph
    bool last_cmp = false;       // the last loop compared valuations: key, cls and depth are not the current ones
    // the switching player's view (built before the first loop that compares valuations): for p = 0
    // (Even, dummies included) and 1 (Odd) the ids of p's vertices in increasing order and their edge
    // lists, contiguous (int32 offsets; a player with 2^31 or more edges keeps the unsplit passes)
    bool pl_ok = false;
    int32_t* pl_vid[2] = {nullptr, nullptr};
    int32_t* pl_off[2] = {nullptr, nullptr};
    int32_t* pl_tgt[2] = {nullptr, nullptr};
    int64_t pl_n[2] = {0, 0};
    // built with the views: Odd's reverse view (for every id t, rv_src[rv_off[t] .. rv_off[t+1]) are the
    // positions in Odd's view of the vertices with an edge to t) and omark (one byte per position of Odd's
    // view, zero padded to a multiple of 16): the vertices that the next Odd switching pass evaluates unless
    // it is full; the others keep their decision (see k_classify)
    int32_t* rv_off = nullptr;
    int32_t* rv_src = nullptr;
    uint8_t* omark = nullptr;
    // ruling-set ranks (pg_deep.cu), for games whose g-forest is deep
    bool deep_mode = false;      // every valuation of the current call takes the ruling-set path
    bool val_deep = false;       // the last valuation took it (its depths are written; no depth pass)
    int32_t* d_anc = nullptr;    // [n] root of each vertex's g-chain
    uint8_t* d_sc = nullptr;     // [2n] the sink's odd and even children (flags for the compactions)
    int32_t* d_podd = nullptr;   // [n+1] positions of the sink's odd children
    int32_t* d_peven = nullptr;  // [n+1] positions of the sink's even children
    int32_t* d_oddL = nullptr;   // [n] the sink's odd children, by id
    int32_t* d_evenL = nullptr;  // [n] the sink's even children, by id
    int32_t* d_nxt = nullptr;    // [2n] Euler tour: next element
    int2* d_wt = nullptr;        // [2n] element weights (visits, depth)
    int2* d_loc = nullptr;       // [2n] prefix within the ruler's sublist
    int32_t* d_own = nullptr;    // [2n] the element's ruler
    int32_t* d_rid = nullptr;    // [2n] ruler index of a ruler element, else -1
    int32_t* d_rl = nullptr;     // [rcap] element of each ruler
    int2* d_val = nullptr;       // [2 rcap] suffix sums of the rulers (two buffers)
    int32_t* d_rnx = nullptr;    // [2 rcap] next ruler (two buffers)
    int32_t d_rcap = 0;          // rulers the scratch holds
    int d_coop = 0;              // co-resident blocks of the ruling-set path's cooperative kernels
    bool reset_tau = false;      // SI-Reset (Section 6): Odd restarts from its first edges after every Even switch
    bool loop_reset[2] = {false, false};  // the SI-Reset setting each loop graph was built with
    bool loop_cmp[2] = {false, false};    // each loop graph compares valuations (loop_compares)
    bool loop_deep[2] = {false, false};   // each loop graph ranks through the ruling-set path
    pg::Tune loop_tune[2];                // the partitioning each loop graph was built with
    pg::Tune tune;                        // the partitioning of the current call (tune_for, at its start)
    // timing of the last call
    double t_total = 0, t_val = 0, t_switch = 0;
    int64_t t_vals = 0;
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    // per-kernel-class device time (timing enabled) and launch counts
    double kms[pg::KID_COUNT] = {};
    int64_t klaunch[pg::KID_COUNT] = {};
    int64_t kcalls[pg::KID_COUNT] = {};
    cudaEvent_t kev[2 * pg::KID_COUNT] = {};
    bool kpend[pg::KID_COUNT] = {};
};

// internal entry points shared by the translation units
namespace pg {
// The partitioning for a game (batch) of n ids: the first table entry covering n, else the context's.
Tune tune_for(const pg_ctx* ctx, int64_t n);
pg_status fail(pg_ctx* ctx, pg_status code, const char* msg);
pg_status cuda_fail(pg_ctx* ctx, cudaError_t e, const char* where);
pg_status load_game(pg_ctx* ctx, int32_t n, int64_t m, const int32_t* off, const int32_t* tgt,
                    const uint8_t* own, const int32_t* pri, int32_t mem_kind, pg_game** out,
                    bool with_scratch = true);
pg_status alloc_scratch(pg_game* g);
// Event timing of a call's phases (active when the context's timing is on).
struct Timer {
    pg_game* g;
    bool on;
    explicit Timer(pg_game* gg) : g(gg), on(gg->ctx->timing) {
        g->t_total = g->t_val = g->t_switch = 0;
        g->t_vals = 0;
    }
    void mark(int i) {
        if (on) cudaEventRecord(g->ev[i], g->ctx->stream);
    }
    double since(int a, int b) {
        if (!on) return 0;
        cudaEventSynchronize(g->ev[b]);
        float ms = 0;
        cudaEventElapsedTime(&ms, g->ev[a], g->ev[b]);
        return ms;
    }
};

// Sets g->strat from a profile in original ids (NULL arrays: the initial profile).
pg_status apply_profile(pg_game* g, const int32_t* sigma, const int32_t* tau, const int8_t* dsig, int32_t mem_kind);
// Writes results in original ids (host or device arrays; NULL skips).
// Bytes of the device staging that write_outputs uses for host outputs.
size_t stage_bytes_for(int64_t n0, int64_t k);
// depth_ready: the depth pass already ran after the last valuation.
pg_status write_outputs(pg_game* g, int32_t mem_kind, uint8_t* win, int32_t* sigma, int32_t* tau, int8_t* vclass,
                        int32_t* vdepth, int32_t* vrank, int32_t* vdom, int8_t* dsig, bool depth_ready = false);
// Algorithm 1 for all games of g (even = false: inner loop only).
// limit > 0: return after at most limit iterations (games may still be active).
pg_status run_loop(pg_game* g, int64_t cap, bool even, Timer& tm, int64_t limit = 0);
// Launches of the iteration loop graph are invalidated (sizes of g changed).
void drop_loop_graphs(pg_game* g);
// Packs loaded single games (freed by the call) into one batch game.
pg_status pack_games(pg_ctx* ctx, pg_game** games, int32_t ngames, pg_game** out);
// Per-game loop bookkeeping after the switching passes; counts active games.
pg_status enqueue_bookkeeping(pg_game* g, int64_t cap, bool even_phase);
// SI-Reset: Odd vertices of games whose Even player just switched back to their first edge.
pg_status enqueue_reset(pg_game* g);
// Resets the per-game state for a new solve.
pg_status reset_games(pg_game* g);
void free_game(pg_game* g);
// Device memory of games: stream-ordered allocations from one pool per
// device that keeps freed memory cached (up to a quarter of the device's
// memory) for the next game, instead of mapping and unmapping it each time.
// Everything free_game releases comes from here.
cudaError_t dev_alloc(pg_ctx* ctx, void** p, size_t bytes, cudaStream_t s);
// Returns the pool's cached memory to the device (pg_release_cached_memory).
cudaError_t dev_trim(int device);
// Co-resident blocks of the cooperative valuation kernels on a device.
pg_status coop_blocks_for(pg_ctx* ctx, int* out);
pg_status chain1_blocks_for(pg_ctx* ctx, int* out);
// per-kernel timing: events around a kernel class on the game's stream
void prof_begin(pg_game* g, int id);
void prof_end(pg_game* g, int id, int nlaunch);
void prof_collect(pg_game* g);  // after a stream synchronisation
// Resets the between-valuation invariants of the scratch arrays (once per call).
pg_status reset_scratch(pg_game* g);
// Enqueues one valuation of g->strat: cls, depth, key (and dom when want_dom). No host synchronisation.
pg_status enqueue_valuation(pg_game* g, bool want_dom);
// Enqueues the depth pass (outputs only; after a valuation).
pg_status enqueue_depth(pg_game* g);
// Enqueues one switching pass for player (0 Even, 1 Odd) using g->key. No host synchronisation.
pg_status enqueue_switch(pg_game* g, int player);
// The loop's iterations without ranks: the nearest-greater forest and the class of every vertex, then
// switching passes that compare the valuations of two successors by walking their g-chains.
bool loop_compares(const pg_game* g);
uint8_t* omark_of(const pg_game* g);  // the Odd marks in use by the loop, or null
pg_status enqueue_valuation_cmp(pg_game* g);
pg_status enqueue_switch_cmp(pg_game* g, int player);
// After a loop that compared valuations: the full valuation of the current profile (key, cls, depth).
pg_status finish_loop(pg_game* g);
// Builds the switching players' views (pl_*) if they are missing; not under stream capture.
pg_status build_player_split(pg_game* g);
// K1 alone (counters cleared, nearest-greater walks and pointer jumping with walk lengths).
pg_status enqueue_k1(pg_game* g);
// The valuation through the ruling-set ranks of an Euler tour (pg_deep.cu): cls, depth, key, dom.
pg_status enqueue_valuation_deep(pg_game* g, bool want_dom);
// Allocates (once, and again for denser rulers) the ruling-set path's scratch; not under stream capture.
pg_status prepare_deep(pg_game* g);
// One valuation on the host's schedule: the default path, and the ruling-set path if a chain walk
// passed the cutover depth (the game then stays on it for the rest of the call). Waits for the stream.
pg_status full_valuation(pg_game* g, bool want_dom);
// Copies the counters to g->hcnt and waits for the stream; checks device error bits.
pg_status sync_counters(pg_game* g);
// Count-vector mode (pg_cv.cu): scratch, one valuation, one switching pass, counts output.
pg_status alloc_cv(pg_game* g);
pg_status enqueue_valuation_cv(pg_game* g, bool want_dom);
pg_status enqueue_switch_cv(pg_game* g, int player);
pg_status write_counts(pg_game* g, int32_t mem_kind, int32_t* counts);
// Bellman-Ford best response against the sigma in g->strat (count-vector mode).
pg_status bellman_ford_cv(pg_game* g, int64_t* rounds);
}  // namespace pg

#define PG_CUDA_TRY(ctx, expr)                                    \
    do {                                                          \
        cudaError_t _e = (expr);                                  \
        if (_e != cudaSuccess) return pg::cuda_fail((ctx), _e, #expr); \
    } while (0)
