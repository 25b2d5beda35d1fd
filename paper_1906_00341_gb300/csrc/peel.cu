// Level-synchronous (k,Psi)-core peeling with level statistics.
//
// Algorithm 3 removes one minimum clique-degree vertex at a time and lowers
// the clique-degree of every vertex sharing a clique instance with it, never
// below the removed vertex's value.  Here every alive vertex whose
// clique-degree is <= k leaves at once (the frontier F); each clique
// instance destroyed by F is credited once, to its smallest-id frontier
// member, and lowers the count of each of its alive non-frontier members by
// one.  A vertex whose count falls to <= k joins the next frontier at the
// same level; when no vertex is left at <= k, k jumps to the minimum alive
// count.  core(v) is the k at which v leaves.  The first round of every
// level starts from the set R_k (Def. 6), whose size and clique count are
// recorded: these give the CoreApp outputs (the k_max core, Lemma 6) and the
// densest residual level (Pruning1, Sec. 5.1) without storing cliques.
//
// One persistent cooperative kernel runs every round; phases are separated
// by grid barriers whose waits are bounded in time (a wait that runs out
// records DSD_ERR_TIMEOUT and every block leaves).
//
// Large regime (many alive vertices), round r, F_r in global lists r mod 3:
//   P1  mark F_{r-1} removed (core = k); mark F_r as frontier     | barrier
//   J   (only if F_r is empty) compact the alive list and take   |
//       the minimum count; k = that minimum; record the level    | barrier
//       (k, |R_k|, mu(R_k)); F_r = alive vertices with count <= k;|
//       when the alive set has halved, drop removed vertices     |
//       from the rows of alive vertices                          | barrier
//   P2  enumerate the cliques each v in F_r destroys; decrement   | barrier
//   P2b (h >= 4) candidate sets above 32 vertices, one block each | barrier
//
// Small regime (the long tail of tiny levels: at most `asmall` vertices
// alive).  Every block holds a slice of the alive list and the whole
// frontier in shared memory and performs the bookkeeping of P1 itself
// (identical writes in every block).  A level jump is distributed: each block
// publishes its slice minimum and the slice vertices attaining it; after one
// barrier every block combines them into k and the frontier.  So a round
// needs one grid barrier after P2, plus the jump barrier (no block may
// decrement counts another block is still reading) and one when big items
// exist.  On entry every alive vertex gets a fixed local id, kept in the
// upper bits of its state word; each block then holds, for the first
// frontier vertices, a bitmap over local ids of their neighbourhoods, so that
// "x in N(v)" is one shared-memory bit instead of a binary search in global
// memory.
//
// Rows live in a private copy of the oriented CSR: row v is
// wadj[off[v] .. wend[v]) and N+(v) = wadj[wnb[v] .. wend[v]).  Compaction
// rewrites a row in place (stable, so rows stay sorted) and moves wend/wnb.
#include "cliques.cuh"
#include "graph.cuh"
#include "xl.cuh"

#include <cooperative_groups.h>
#include <string.h>

namespace dsd {
namespace {

// state word: bits 0-1 the state, bits 2-31 the local id (small regime)
enum : uint32_t { kAlive = 0, kFront = 1, kGone = 2 };
enum : uint32_t { kErrTimeout = 1, kErrBigOverflow = 2 };
constexpr uint32_t kSmallFront = 1024;
constexpr uint32_t kBitmapSlots = 16;   // frontier vertices with a shared bitmap
constexpr int kChunks = 4;              // 32-entry chunks of a row in flight per warp
constexpr uint32_t kWarpCand = 32;      // candidate sets a warp handles itself (h >= 4)
constexpr uint32_t kWarpWords = 3 * kWarpCand;   // a warp's candidates, counters, rows
constexpr uint32_t kMidWords = 3 + kWarpCand;    // a mid item: v, w, |C|, C
constexpr int kGroupWarps = 8;                    // warps of a group taking one mid item
// h >= 4: a warp lists the cliques of a candidate set of at most this many
// vertices itself (default 4, dsd_set_peel_items); larger sets go to a warp
// group or a whole block after the next grid barrier.  Items are the round's
// critical path when one warp walks the rows of many candidates in turn: on
// R-MAT scale 21 the peel took 9.4 s (h = 4) and 20.5 s (h = 5) with the limit
// at 32, 5.2 s and 13.5 s at 4.
inline uint32_t warp_cand_limit(int h) {
    uint32_t w = peel_item_warp_limit();
    return h >= 4 ? (w < kWarpCand ? w : kWarpCand) : kWarpCand;
}
constexpr uint32_t kHeavyBit = 4;       // state word: frontier vertex on the heavy list
constexpr uint32_t kSlotShift = 3;      // state word: 1 + its neighbourhood bitmap slot
constexpr uint32_t kSlotMask = 0xffu;

__device__ __forceinline__ uint32_t st_of(uint32_t w) { return w & 3u; }

struct PeelCtrl {
    unsigned long long min_deg[2];
    uint32_t new_alive[2];
    uint32_t fcnt[3];
    uint32_t big_cnt[6];            // per round slot s: big items [s], mid items [3 + s]
    unsigned long long destroyed[3];
    uint32_t hcnt[3];               // heavy frontier vertices of the round
    uint32_t grab[3];               // light frontier vertices taken by blocks
    uint32_t bgrab[6];              // big items [s] and mid items [3 + s] taken
    uint32_t hubcnt[2];             // bitmap slots asked for, by round parity
    uint32_t pad0[11];
    uint32_t bar_count;
    uint32_t pad1[31];
    uint32_t bar_gen;
    uint32_t pad2[31];
    uint32_t error;
    uint32_t err_info;
    unsigned long long kmax;
    uint32_t nlevels;
    uint32_t rounds;
    unsigned long long items;
    unsigned long long bytes;       // algorithmic bytes (meter notes below)
    unsigned long long barrier_ns;  // block 0's time inside grid barriers
    uint32_t barriers;
    uint32_t compactions;
    uint32_t small_round;           // first round of the small regime (0 = never)
    uint32_t pad3;
    unsigned long long tph[8];      // block 0's time per phase (ns)
    // hand-over to the cluster tail kernel
    uint32_t tail_n;                // alive vertices handed over (0 = none)
    uint32_t tail_round;            // round at the hand-over
    uint32_t tail_sel;              // which hand-over list holds them
    uint32_t tail_entry;            // alive vertices at the first hand-over
    uint32_t tail_entry_round;      // its round
    uint32_t pad4;
    unsigned long long mu_tail;     // mu of the alive graph at the hand-over
    unsigned long long tail_ns;     // the tail kernel's duration
    unsigned long long tail_tph[7]; // tail lead CTA: build, A+sync, jump+list, C prefix, C work, C sync, D
};

// Byte meter.  Every global-memory element the algorithm reads or writes is
// counted once per access: ids and state words 4 B, offsets 8 B, counters
// 8 B, an atomic read-modify-write 16 B, a binary search over a row of d
// entries floor(log2 d) + 1 probes of 4 B.  Shared-memory traffic is not
// counted, and bookkeeping that every block repeats in the small regime
// counts once.
__device__ __forceinline__ unsigned probes(uint64_t d) {
    return d ? 64u - (unsigned)__clzll((long long)d) : 0u;
}

struct PeelParams {
    uint32_t n;
    int h;
    const uint64_t* off;   // row starts (read-only)
    uint32_t* wadj;        // private copy of the rows
    uint64_t* wend;        // row ends
    uint64_t* wnb;         // N+ starts (h >= 3)
    unsigned long long* deg;
    uint64_t* core;
    uint32_t* rnd;
    uint32_t* sl;          // state words
    uint32_t* alive[2];
    uint32_t* front[3];
    uint32_t* jf;          // small regime: per-slice jump candidates
    ulonglong2* jblk;      // small regime: per-block (slice minimum, alive<<32 | candidates)
    uint2* big;
    uint64_t big_cap;
    uint32_t* heavy;       // large regime: frontier vertices with long rows
    uint32_t heavy_min;    // rows longer than this are heavy (0 = no heavy list)
    // Large regime: frontier vertices with rows longer than hub_min get (up
    // to hub_slots per round) a bitmap of their neighbourhood over vertex
    // ids, so that "x in N(v)" is one probe instead of a binary search.  Two
    // sets of hub_slots bitmaps of hub_words words, by round parity; hubs
    // lists the owners (2 x hub_slots).
    uint32_t* hub_bm;
    uint32_t* hubs;
    uint64_t hub_words;
    uint32_t hub_slots;    // 0 = no bitmaps
    uint32_t hub_min;
    uint64_t* lvl_k;
    uint32_t* lvl_size;
    uint64_t* lvl_mu;
    PeelCtrl* ctrl;
    uint64_t wait_ns;
    unsigned long long mu0;
    unsigned long long k0; // initial level: kstart - 1, or 0
    uint32_t cap;          // candidate sets are at most this (>= max |N+|, >= 32)
    uint32_t bcap;         // a big item's shared buffers: min(cap, kBitmapMax)
    uint32_t warp_cand;    // h >= 4: candidate sets a warp handles (<= kWarpCand); larger
                           // ones go to a warp group (mid items) or a block
    uint32_t gather_cap;   // a warp's candidate walk stops past this many
    uint32_t* mid;         // mid items: kMidWords words each (v, w, |C|, C)
    uint32_t mid_cap;      // 0: none (every set above warp_cand goes to a block)
    uint32_t* xl;          // per block (kMaxDepth + 1) * cap entries when cap > kBitmapMax
    int compact;           // drop removed vertices from rows as the graph shrinks
    uint32_t work_words;   // shared words before the small-regime lists
    uint32_t asmall;       // small-regime list capacity (0 = regime off)
    uint32_t tail_max;     // hand over to the cluster tail at <= this many alive (0 = off)
    uint64_t* snap;        // if set: each alive vertex's count at every level jump (the
                           // last one written is its count in its own (k,Psi)-core)
};

// ------------------------------------------------------------ barrier
__device__ bool grid_barrier(PeelCtrl* c, uint64_t wait_ns, unsigned long long& waited) {
    __shared__ uint32_t s_err;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint64_t t_in = globaltimer_ns();
        volatile uint32_t* genp = &c->bar_gen;
        uint32_t gen = *genp;
        __threadfence();
        uint32_t arrived = atomicAdd(&c->bar_count, 1u) + 1u;
        if (arrived == gridDim.x) {
            c->bar_count = 0;
            __threadfence();
            atomicAdd(&c->bar_gen, 1u);
        } else {
            uint32_t spins = 0;
            while (*genp == gen) {
                if (((++spins) & 255u) == 0 && globaltimer_ns() - t_in > wait_ns) {
                    atomicOr(&c->error, kErrTimeout);
                    break;
                }
                if (*(volatile uint32_t*)&c->error) break;
            }
        }
        __threadfence();
        s_err = *(volatile uint32_t*)&c->error;
        waited += globaltimer_ns() - t_in;
    }
    __syncthreads();
    // one decision per block, so that its threads leave (or stay) together
    return s_err == 0;
}

// ------------------------------------------------------------ helpers
__device__ __forceinline__ void dec_and_queue(const PeelParams& P, uint32_t u,
                                              unsigned long long c, unsigned long long k,
                                              uint32_t* next, uint32_t* next_cnt) {
    unsigned long long old = atomic_sub_u64(&P.deg[u], c);
    if (old > k && old - c <= k) {
        uint32_t at = atomicAdd(next_cnt, 1u);
        next[at] = u;
    }
}

// Warp-aggregated append of `val` where pred holds (all lanes call).
__device__ __forceinline__ void warp_append(bool pred, uint32_t val, uint32_t* counter,
                                            uint32_t* list) {
    unsigned lane = lane_id();
    unsigned b = __ballot_sync(0xffffffffu, pred);
    if (!b) return;
    uint32_t base = 0;
    if (lane == 0) base = atomicAdd(counter, (uint32_t)__popc(b));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (pred) list[base + __popc(b & ((1u << lane) - 1u))] = val;
}

// Block sum of per-thread values; result valid in thread 0.
template <int NT>
__device__ __forceinline__ unsigned long long block_sum(unsigned long long v,
                                                       unsigned long long* red) {
    v = warp_sum(v);
    if (lane_id() == 0) red[warp_id()] = v;
    __syncthreads();
    unsigned long long t = 0;
    if (threadIdx.x == 0)
        for (int w = 0; w < NT / 32; w++) t += red[w];
    __syncthreads();
    return t;
}

// Block-wide exclusive scan of small per-thread counts; returns this
// thread's prefix and the total in *tot (all threads).
template <int NT>
__device__ __forceinline__ uint32_t block_scan_count(uint32_t v, uint32_t* wtot, uint32_t* tot) {
    unsigned lane = lane_id(), wid = warp_id();
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if ((int)lane >= o) x += y;
    }
    if (lane == 31) wtot[wid] = x;
    __syncthreads();
    uint32_t before = 0, all = 0;
    for (int w = 0; w < NT / 32; w++) {
        uint32_t t = wtot[w];
        before += (w < (int)wid) ? t : 0u;
        all += t;
    }
    __syncthreads();
    *tot = all;
    return before + x - v;
}

// pre[0] = 0, pre[i+1] = sum of the current row lengths of F[0..i], for
// f <= kSmallFront entries (each thread owns kSmallFront/NT consecutive ones).
template <int NT>
__device__ __forceinline__ void block_prefix_degrees(const PeelParams& P, const uint32_t* F,
                                                     uint32_t f, unsigned long long* pre,
                                                     unsigned long long* red,
                                                     bool skip_empty = false) {
    constexpr int E = kSmallFront / NT;
    unsigned long long d[E], sum = 0;
    uint32_t i0 = threadIdx.x * E;
#pragma unroll
    for (int q = 0; q < E; q++) {
        uint32_t i = i0 + q;
        d[q] = 0;
        if (i < f) {
            uint32_t v = F[i];
            // a frontier vertex of count 0 lies in no clique: no items
            if (!skip_empty || P.deg[v] != 0) d[q] = P.wend[v] - P.off[v];
        }
        sum += d[q];
    }
    unsigned lane = lane_id();
    unsigned long long x = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
        if ((int)lane >= o) x += y;
    }
    if (lane == 31) red[warp_id()] = x;
    __syncthreads();
    unsigned long long before = 0;
    for (unsigned w = 0; w < warp_id(); w++) before += red[w];
    unsigned long long run = before + x - sum;
    if (threadIdx.x == 0) pre[0] = 0;
#pragma unroll
    for (int q = 0; q < E; q++) {
        run += d[q];
        if (i0 + q < f) pre[i0 + q + 1] = run;
    }
    __syncthreads();
}

// Candidates of frontier vertex v among N+(w), in order (one warp).  A
// candidate is alive, or a frontier vertex with a larger id than v, and is
// adjacent to v: tested on v's shared bitmap `bm` (over local ids) when
// given, else by binary search in v's row.  kChunks chunks of the row are
// loaded at once.  MODE:
//   kGatherDirect (h = 3): each candidate closes the triangle {v, w, x}; an
//     alive candidate loses it on the spot; nothing is stored;
//   kGatherWarp: the first kWarpCand candidates go to C; the walk stops as
//     soon as there are more than P.gather_cap (the item then needs a block).
// gbm (large regime, may be null): v's neighbourhood bitmap over vertex ids.
// Returns the number of candidates seen.
enum { kGatherDirect = 0, kGatherWarp = 1 };

template <int MODE>
__device__ __forceinline__ void take_candidate(const PeelParams& P, bool ok, bool alive,
                                               uint32_t x, uint32_t* C, uint32_t& nc,
                                               unsigned long long k, uint32_t* next,
                                               uint32_t* next_cnt, unsigned long long& bytes) {
    unsigned lane = lane_id();
    unsigned bal = __ballot_sync(0xffffffffu, ok);
    if (MODE == kGatherDirect) {
        if (ok && alive) {
            dec_and_queue(P, x, 1ull, k, next, next_cnt);
            bytes += 16;
        }
    } else {
        uint32_t at = nc + __popc(bal & ((1u << lane) - 1u));
        if (ok && at < kWarpCand) C[at] = x;
    }
    nc += __popc(bal);
}

template <int MODE>
__device__ __forceinline__ uint32_t gather_candidates(const PeelParams& P, uint32_t v,
                                                      uint32_t w, uint32_t* C,
                                                      const uint32_t* bm, const uint32_t* gbm,
                                                      unsigned long long k,
                                                      uint32_t* next, uint32_t* next_cnt,
                                                      unsigned long long& bytes) {
    unsigned lane = lane_id();
    const uint32_t* Nv = P.wadj + P.off[v];
    uint64_t dv = P.wend[v] - P.off[v];
    uint64_t b = P.wnb[w], e = P.wend[w];
    const uint64_t dw = e - b;
    const unsigned pr = probes(dv);
    uint32_t nc = 0;
    // Walk the shorter side: the entries of N(v) above w, each searched in
    // N+(w), when that costs fewer probes than walking N+(w).
    const uint64_t cost_w = (bm || gbm) ? dw : dw * pr;
    if (dv * probes(dw) < cost_w) {
        const uint32_t* Nw = P.wadj + b;
        uint64_t s0 = lower_bound_u32(Nv, dv, w + 1u);
        const unsigned pw = probes(dw);
        for (uint64_t p0 = s0; p0 < dv; p0 += 32 * kChunks) {
            uint32_t xs[kChunks], ws[kChunks];
#pragma unroll
            for (int u = 0; u < kChunks; u++) {
                uint64_t p = p0 + u * 32 + lane;
                xs[u] = p < dv ? Nv[p] : 0u;
            }
#pragma unroll
            for (int u = 0; u < kChunks; u++) {
                uint64_t p = p0 + u * 32 + lane;
                ws[u] = p < dv ? P.sl[xs[u]] : (uint32_t)kGone;
            }
#pragma unroll
            for (int u = 0; u < kChunks; u++) {
                uint64_t p = p0 + u * 32 + lane;
                bool ok = false;
                uint32_t x = xs[u];
                uint32_t s = st_of(ws[u]);
                if (p < dv) {
                    bytes += 8;
                    if (s == kAlive || (s == kFront && x > v)) {
                        uint64_t pos = lower_bound_u32(Nw, dw, x);
                        ok = pos < dw && Nw[pos] == x;
                        bytes += 4ull * pw;
                    }
                }
                take_candidate<MODE>(P, ok, s == kAlive, x, C, nc, k, next, next_cnt, bytes);
            }
            if (MODE == kGatherWarp && nc > P.gather_cap) return nc;
        }
        return nc;
    }
    for (uint64_t p0 = b; p0 < e; p0 += 32 * kChunks) {
        uint32_t xs[kChunks], ws[kChunks];
#pragma unroll
        for (int u = 0; u < kChunks; u++) {
            uint64_t p = p0 + u * 32 + lane;
            xs[u] = p < e ? P.wadj[p] : 0u;
        }
#pragma unroll
        for (int u = 0; u < kChunks; u++) {
            uint64_t p = p0 + u * 32 + lane;
            ws[u] = p < e ? P.sl[xs[u]] : (uint32_t)kGone;
        }
#pragma unroll
        for (int u = 0; u < kChunks; u++) {
            uint64_t p = p0 + u * 32 + lane;
            bool ok = false;
            uint32_t x = xs[u];
            uint32_t s = st_of(ws[u]);
            if (p < e) {
                bytes += 8;
                if (s == kAlive || (s == kFront && x > v)) {
                    if (bm) {
                        uint32_t l = ws[u] >> 2;
                        ok = (bm[l >> 5] >> (l & 31)) & 1u;
                    } else if (gbm) {
                        ok = (gbm[x >> 5] >> (x & 31)) & 1u;
                        bytes += 4;
                    } else {
                        uint64_t pos = lower_bound_u32(Nv, dv, x);
                        ok = pos < dv && Nv[pos] == x;
                        bytes += 4ull * pr;
                    }
                }
            }
            take_candidate<MODE>(P, ok, s == kAlive, x, C, nc, k, next, next_cnt, bytes);
        }
        if (MODE == kGatherWarp && nc > P.gather_cap) return nc;
    }
    return nc;
}

// One (v, w) work item of a frontier vertex v with h >= 3: the cliques
// {v, w, ...} whose members other than v are candidates of v and whose
// smallest such member is w.  Executed by one warp; C, cnt, rows are the
// warp's kWarpCand-entry buffers.  Candidate sets above P.warp_cand (h >= 4)
// are queued, as mid items with their candidates when at most kWarpCand
// (`big_cnt + 3` counts them), else as big items for a block.
__device__ void process_vw(const PeelParams& P, uint32_t v, uint32_t w, unsigned long long k,
                           uint32_t* next, uint32_t* next_cnt, uint32_t* C, unsigned* cnt,
                           uint32_t* rows, uint32_t* big_cnt, const uint32_t* bm,
                           const uint32_t* gbm, unsigned long long& destroyed,
                           unsigned long long& bytes) {
    unsigned lane = lane_id();
    uint32_t sw = st_of(P.sl[w]);
    if (lane == 0) bytes += 4 + 4;   // w, its state word
    if (!(sw == kAlive || (sw == kFront && w > v))) return;
    if (lane == 0) bytes += 16;      // wnb[w], wend[w]
    const int r = P.h - 2;
    unsigned long long tot = 0;
    if (r == 1) {
        tot = gather_candidates<kGatherDirect>(P, v, w, C, bm, gbm, k, next, next_cnt, bytes);
    } else {
        uint32_t nc =
            gather_candidates<kGatherWarp>(P, v, w, C, bm, gbm, k, next, next_cnt, bytes);
        __syncwarp();
        if (nc < (uint32_t)r) return;
        if (nc > P.warp_cand) {
            // mid item: its candidates go with it to a warp group; else a block
            if (nc <= kWarpCand && P.mid_cap) {
                uint32_t at = 0;
                if (lane == 0) at = atomicAdd(big_cnt + 3, 1u);
                at = __shfl_sync(0xffffffffu, at, 0);
                if (at < P.mid_cap) {
                    uint32_t* rec = P.mid + (size_t)at * kMidWords;
                    if (lane < nc) rec[3 + lane] = C[lane];
                    if (lane == 0) {
                        rec[0] = v;
                        rec[1] = w;
                        rec[2] = nc;
                        bytes += 12 + 4ull * nc;
                    }
                    return;
                }
            }
            if (lane == 0) {
                uint32_t at = atomicAdd(big_cnt, 1u);
                if (at < P.big_cap) P.big[at] = make_uint2(v, w);
                else atomicOr(&P.ctrl->error, kErrBigOverflow);
            }
            return;
        }
        for (uint32_t i = lane; i < nc; i += 32) cnt[i] = 0;
        __syncwarp();
        if (r == 2) {
            // edges of G[C]: each is a clique {v, w, x, y}
            const uint32_t cmax = C[nc - 1];
            for (uint32_t i = 0; i + 1 < nc; i++) {
                uint32_t x = C[i];
                uint64_t xb = P.wnb[x], xe = P.wend[x], xr = xe;
                unsigned hits = scan_row_hits(C, nc, cmax, P.wadj, xb, xe, cnt, &xr);
                if (lane == 0) bytes += 16 + 4ull * (xr - xb);
                hits = __reduce_add_sync(0xffffffffu, hits);
                if (lane == 0 && hits) atomicAdd(&cnt[i], hits);
                tot += hits;
            }
        } else {
            if (lane == 0)
                for (uint32_t i = 0; i < nc; i++)
                    bytes += 16 + 4ull * (P.wend[C[i]] - P.wnb[C[i]]);
            warp_build_rows32(C, nc, P.wend, P.wadj, P.wnb, rows);
            tot = warp_dfs32(rows, nc, r, cnt);
        }
        __syncwarp();
        if (tot)
            for (uint32_t i = lane; i < nc; i += 32) {
                uint32_t x = C[i];
                if (cnt[i]) {
                    bytes += 4;
                    if (st_of(P.sl[x]) == kAlive) {
                        dec_and_queue(P, x, (unsigned long long)cnt[i], k, next, next_cnt);
                        bytes += 16;
                    }
                }
            }
        __syncwarp();
    }
    if (tot && lane == 0) {
        if (sw == kAlive) {
            dec_and_queue(P, w, tot, k, next, next_cnt);
            bytes += 16;
        }
        destroyed += tot;
    }
}

// A (v, w) item whose candidate set exceeds 32 vertices (h >= 4): one block,
// bitmap rows of G[C] and a warp-level DFS per starting candidate.  When
// N+(w) holds more than kBitmapMax entries (degeneracy above 1024) the
// candidates are gathered into the block's global scratch; a set that still
// exceeds kBitmapMax is split by its next member (xl.cuh).
__device__ void process_big(const PeelParams& P, uint32_t v, uint32_t w, unsigned long long k,
                            uint32_t* next, uint32_t* next_cnt, uint32_t* smem,
                            const uint32_t* gbm, unsigned long long& destroyed,
                            unsigned long long& bytes) {
    unsigned long long* cnt = reinterpret_cast<unsigned long long*>(smem);  // bcap
    uint32_t* C = smem + 2 * P.bcap;                                          // bcap
    uint32_t* rows = C + P.bcap;                                              // bcap * W
    __shared__ uint32_t s_nc;
    __shared__ uint32_t s_next;
    __shared__ unsigned long long s_tot;
    __shared__ uint32_t s_flag[kBitmapMax / 32], s_at[kBitmapMax / 32];
    __shared__ uint32_t s_w[32], s_t2;
    const unsigned lane = lane_id(), nw = blockDim.x >> 5;
    uint32_t sw = st_of(P.sl[w]);
    const uint64_t b = P.wnb[w], e = P.wend[w];
    const uint32_t* Nv = P.wadj + P.off[v];
    const uint64_t dv = P.wend[v] - P.off[v];
    const unsigned pr = probes(dv);
    if (e - b > kBitmapMax) {
        // oversized N+(w): gather in order into the block's global scratch
        uint32_t* G0 = P.xl + (size_t)blockIdx.x * (kMaxDepth + 1) * P.cap;
        const uint32_t nc = block_filter(
            P.wadj + b, e - b, G0,
            [&](uint32_t x) {
                const uint32_t st = st_of(P.sl[x]);
                if (!(st == kAlive || (st == kFront && x > v))) return false;
                if (gbm) return ((gbm[x >> 5] >> (x & 31)) & 1u) != 0u;
                uint64_t pos = lower_bound_u32(Nv, dv, x);
                return pos < dv && Nv[pos] == x;
            },
            s_w, &s_t2);
        if (threadIdx.x == 0) bytes += (8ull + 4ull * pr) * (e - b) + 24;
        if (nc > kBitmapMax) {
            if (threadIdx.x == 0) s_tot = 0;
            __syncthreads();
            xl_cliques(
                G0, nc, P.h - 2, P.wnb, P.wend, P.wadj, G0 + P.cap, P.cap, smem,
                [&](uint32_t x, unsigned long long c) {
                    if (st_of(P.sl[x]) == kAlive) dec_and_queue(P, x, c, k, next, next_cnt);
                },
                [&](unsigned long long c) { s_tot += c; });
            __syncthreads();
            if (threadIdx.x == 0 && s_tot) {
                if (sw == kAlive) dec_and_queue(P, w, s_tot, k, next, next_cnt);
                destroyed += s_tot;
            }
            __syncthreads();
            return;
        }
        for (uint32_t i = threadIdx.x; i < nc; i += blockDim.x) C[i] = G0[i];
        if (threadIdx.x == 0) {
            s_nc = nc;
            s_next = 0;
            s_tot = 0;
        }
        __syncthreads();
        if (nc < (uint32_t)(P.h - 2)) return;
        goto bitmap;
    }
    {
    // candidates of v among N+(w), all warps at once: warp c tests the c-th
    // run of 32 entries, the runs' hit masks are compacted in order
    const uint32_t runs = (uint32_t)((e - b + 31) >> 5);   // <= kBitmapMax / 32
    for (uint32_t c = warp_id(); c < runs; c += nw) {
        const uint64_t p = b + (uint64_t)c * 32 + lane;
        bool ok = false;
        if (p < e) {
            const uint32_t x = P.wadj[p];
            const uint32_t st = st_of(P.sl[x]);
            bytes += 8;
            if (st == kAlive || (st == kFront && x > v)) {
                if (gbm) {
                    ok = (gbm[x >> 5] >> (x & 31)) & 1u;
                    bytes += 4;
                } else {
                    uint64_t pos = lower_bound_u32(Nv, dv, x);
                    ok = pos < dv && Nv[pos] == x;
                    bytes += 4ull * pr;
                }
            }
        }
        const unsigned bal = __ballot_sync(0xffffffffu, ok);
        if (lane == 0) s_flag[c] = bal;
    }
    __syncthreads();
    if (warp_id() == 0) {
        uint32_t tot = 0;
        for (uint32_t c0 = 0; c0 < runs; c0 += 32) {
            const uint32_t c = c0 + lane;
            uint32_t x = c < runs ? (uint32_t)__popc(s_flag[c]) : 0u, inc = x;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
                if ((int)lane >= o) inc += y;
            }
            if (c < runs) s_at[c] = tot + inc - x;
            tot += __shfl_sync(0xffffffffu, inc, 31);
        }
        if (lane == 0) {
            s_nc = tot;
            s_next = 0;
            s_tot = 0;
            bytes += 4 + 4 + 16;
        }
    }
    __syncthreads();
    for (uint32_t c = warp_id(); c < runs; c += nw) {
        const unsigned bal = s_flag[c];
        if ((bal >> lane) & 1u)
            C[s_at[c] + __popc(bal & ((1u << lane) - 1u))] = P.wadj[b + (uint64_t)c * 32 + lane];
    }
    __syncthreads();
    }
bitmap:
    uint32_t nc = s_nc;
    uint32_t W = (nc + 31) >> 5;
    for (uint32_t i = threadIdx.x; i < nc; i += blockDim.x) {
        cnt[i] = 0;
        bytes += 16 + 4ull * (P.wend[C[i]] - P.wnb[C[i]]);
    }
    for (uint32_t i = threadIdx.x; i < nc * W; i += blockDim.x) rows[i] = 0;
    __syncthreads();
    block_build_rows(C, nc, W, P.wend, P.wadj, P.wnb, rows);
    __syncthreads();
    unsigned long long mine = block_dfs(rows, nc, W, P.h - 2, cnt, &s_next);
    if (mine) atomicAdd(&s_tot, mine);
    __syncthreads();
    unsigned long long tot = s_tot;
    if (tot) {
        for (uint32_t i = threadIdx.x; i < nc; i += blockDim.x) {
            uint32_t x = C[i];
            if (cnt[i] && st_of(P.sl[x]) == kAlive) {
                dec_and_queue(P, x, cnt[i], k, next, next_cnt);
                bytes += 20;
            }
        }
        if (threadIdx.x == 0) {
            if (sw == kAlive) dec_and_queue(P, w, tot, k, next, next_cnt);
            destroyed += tot;
        }
    }
    __syncthreads();
}

__device__ __forceinline__ void group_bar(uint32_t id, uint32_t threads) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(threads) : "memory");
}

// Mid items (h >= 4; candidate sets of warp_cand + 1 .. 32 vertices, listed
// by the warp that found them): groups of kGroupWarps warps take them from
// *grab, several per block at once.  The group's warps build the one-word
// rows of G[C] side by side (one candidate's list each), its first warp
// lists the cliques of G[C] (warp_dfs32), and the alive members are lowered.
// Group g synchronises on named barrier 1 + g.  destroyed: the round's sum.
template <int NT>
__device__ void drain_mid(const PeelParams& P, uint32_t nm, uint32_t* grab, unsigned long long k,
                          uint32_t* next, uint32_t* next_cnt, unsigned long long* destroyed,
                          unsigned long long& bytes) {
    constexpr int NG = NT / 32 / kGroupWarps;
    struct MidBuf {
        uint32_t C[kWarpCand];
        unsigned cnt[kWarpCand];
        uint32_t rows[kWarpCand];
        uint32_t i;
        unsigned long long tot;
    };
    __shared__ MidBuf s_mb[NG];
    const unsigned lane = lane_id(), wid = warp_id();
    const uint32_t grp = wid / kGroupWarps, gw = wid % kGroupWarps;
    const uint32_t bar = 1u + grp, nth = kGroupWarps * 32u;
    MidBuf& B = s_mb[grp];
    const int r = P.h - 2;
    unsigned long long dsum = 0;
    for (;;) {
        if (gw == 0 && lane == 0) B.i = atomicAdd(grab, 1u);
        group_bar(bar, nth);
        const uint32_t i = B.i;
        if (i >= nm) break;
        const uint32_t* rec = P.mid + (size_t)i * kMidWords;
        const uint32_t v = rec[0], w = rec[1], nc = rec[2];
        (void)v;
        if (gw == 0) {
            B.C[lane] = lane < nc ? rec[3 + lane] : 0u;
            B.cnt[lane] = 0;
            B.rows[lane] = 0;
        }
        group_bar(bar, nth);
        const uint32_t cmax = B.C[nc - 1];
        for (uint32_t x = gw; x + 1 < nc; x += kGroupWarps) {
            const uint32_t y = B.C[x];
            const uint32_t bits = warp_row32(B.C, nc, cmax, y, P.wadj, P.wnb[y], P.wend[y]);
            if (lane == 0) {
                B.rows[x] = bits;
                bytes += 16 + 4ull * (P.wend[y] - P.wnb[y]);
            }
        }
        group_bar(bar, nth);
        if (gw == 0) {
            const unsigned long long t = warp_dfs32(B.rows, nc, r, B.cnt);
            if (lane == 0) B.tot = t;
        }
        group_bar(bar, nth);
        const unsigned long long tot = B.tot;
        if (tot) {
            const uint32_t t = gw * 32 + lane;
            if (t < nc && B.cnt[t]) {
                const uint32_t x = B.C[t];
                if (st_of(P.sl[x]) == kAlive) {
                    dec_and_queue(P, x, (unsigned long long)B.cnt[t], k, next, next_cnt);
                    bytes += 20;
                }
            }
            if (gw == 0 && lane == 0) {
                if (st_of(P.sl[w]) == kAlive) dec_and_queue(P, w, tot, k, next, next_cnt);
                dsum += tot;
            }
        }
        group_bar(bar, nth);   // B is rewritten by the next item
    }
    if (gw == 0 && lane == 0 && dsum) atomicAdd(destroyed, dsum);
}

// Drop removed vertices from row v in place (one warp); rows stay sorted.
__device__ __forceinline__ void compact_row(const PeelParams& P, uint32_t v,
                                            unsigned long long& bytes) {
    unsigned lane = lane_id();
    uint64_t b = P.off[v], e = P.wend[v];
    uint64_t outp = b;
    uint64_t below = 0;   // kept entries smaller than v
    for (uint64_t p0 = b; p0 < e; p0 += 32) {
        uint64_t p = p0 + lane;
        uint32_t x = 0;
        bool keep = false;
        if (p < e) {
            x = P.wadj[p];
            keep = st_of(P.sl[x]) != kGone;
        }
        unsigned bal = __ballot_sync(0xffffffffu, keep);
        unsigned lt = __ballot_sync(0xffffffffu, keep && x < v);
        // every lane has read its entry before any lane writes
        if (keep) P.wadj[outp + __popc(bal & ((1u << lane) - 1u))] = x;
        outp += __popc(bal);
        below += __popc(lt);
        __syncwarp();
    }
    bytes += 8ull * (e - b) + 4ull * (outp - b);
    if (lane == 0) {
        P.wend[v] = outp;
        P.wnb[v] = b + below;
        bytes += 16;
    }
}

// Large regime: the neighbourhood bitmap of frontier vertex v for rounds of
// parity par, or null if v has none.
__device__ __forceinline__ const uint32_t* hub_bm_of(const PeelParams& P, uint32_t v,
                                                    uint32_t par) {
    if (!P.hub_slots) return nullptr;
    uint32_t slot = (P.sl[v] >> kSlotShift) & kSlotMask;
    return slot ? P.hub_bm + ((size_t)par * P.hub_slots + (slot - 1)) * P.hub_words : nullptr;
}

// Large regime, marking v as a member of frontier F_r: its state word, with
// kHeavyBit for rows longer than heavy_min and, for rows longer than hub_min
// while slots of this parity last, 1 + its bitmap slot (the owner goes to
// the parity's hub list).
__device__ __forceinline__ uint32_t front_word(const PeelParams& P, PeelCtrl* c, uint32_t v,
                                               uint32_t par, bool& hv) {
    uint64_t d = P.wend[v] - P.off[v];
    hv = P.heavy_min && d > P.heavy_min;
    uint32_t w = kFront | (hv ? kHeavyBit : 0u);
    if (hv && P.hub_slots && d > P.hub_min) {
        uint32_t at = atomicAdd(&c->hubcnt[par], 1u);
        if (at < P.hub_slots) {
            P.hubs[par * P.hub_slots + at] = v;
            w |= (at + 1u) << kSlotShift;
        }
    }
    return w;
}

// Sets (or, clear = true, zeroes the words of) the bitmaps of the hubs of
// parity par over their rows; the rows' entries are flattened over every
// thread of the grid.  Every thread of every block calls it.
template <int NT>
__device__ __forceinline__ void hub_bitmaps(const PeelParams& P, uint32_t nhub, uint32_t par,
                                            bool clear, unsigned long long* s_pre,
                                            unsigned long long* s_red,
                                            unsigned long long& bytes) {
    const uint32_t* H = P.hubs + (size_t)par * P.hub_slots;
    block_prefix_degrees<NT>(P, H, nhub, s_pre, s_red);
    const unsigned long long T = s_pre[nhub];
    const uint64_t gtid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t gthreads = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t t = gtid; t < T; t += gthreads) {
        uint32_t lo = 0, hi = nhub;
        while (hi - lo > 1) {
            uint32_t mid = (lo + hi) >> 1;
            if (s_pre[mid] <= t) lo = mid; else hi = mid;
        }
        uint32_t v = H[lo];
        uint32_t x = P.wadj[P.off[v] + (t - s_pre[lo])];
        uint32_t* bm = P.hub_bm + ((size_t)par * P.hub_slots + lo) * P.hub_words;
        if (clear) bm[x >> 5] = 0u;   // every set bit belongs to a row entry
        else atomicOr(&bm[x >> 5], 1u << (x & 31));
        bytes += 4 + 16;
    }
    __syncthreads();   // s_pre is reused afterwards
}

// P2: the cliques destroyed by frontier F (nf vertices; F in global or
// shared memory, identical for every block).  Frontier counts do not change
// during P2 (only alive vertices are lowered), so a frontier vertex of count
// 0, which lies in no clique of the current set, is skipped.  bm: shared bitmaps of the
// neighbourhoods of F[0 .. min(nf, kBitmapSlots)) (small regime), or null.
template <int NT>
__device__ __forceinline__ void process_frontier(
    const PeelParams& P, const uint32_t* F, uint32_t nf, unsigned long long k, uint32_t* Fnext,
    uint32_t* next_cnt, uint32_t* big_cnt, uint32_t* wC, unsigned* wCnt, uint32_t* wRows,
    const uint32_t* bm, uint32_t bm_words, unsigned long long* s_pre, unsigned long long* s_red,
    const uint32_t* hl, uint32_t nh, uint32_t* grab, uint32_t* s_grab, uint32_t par,
    unsigned long long& destroyed, unsigned long long& items, unsigned long long& bytes) {
    constexpr int NW = NT / 32;
    const unsigned lane = lane_id(), wid = warp_id();
    const uint64_t gtid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t gthreads = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t gwarp = gtid >> 5;
    const uint64_t gwarps = gthreads >> 5;
    if (k == 0) return;   // every frontier vertex has count 0
    if (nf <= kSmallFront) {
        // flatten (v, neighbour index) items over the whole grid
        block_prefix_degrees<NT>(P, F, nf, s_pre, s_red, true);
        unsigned long long T = s_pre[nf];
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            items += T;
            bytes += 20ull * nf;   // frontier ids and their row bounds
        }
        if (P.h == 2) {
            for (uint64_t t = gtid; t < T; t += gthreads) {
                uint32_t lo = 0, hi = nf;  // last i with s_pre[i] <= t
                while (hi - lo > 1) {
                    uint32_t mid = (lo + hi) >> 1;
                    if (s_pre[mid] <= t) lo = mid; else hi = mid;
                }
                uint32_t v = F[lo];
                uint32_t u = P.wadj[P.off[v] + (t - s_pre[lo])];
                uint32_t su = st_of(P.sl[u]);
                bytes += 4 + 4;
                if (su == kAlive) {
                    dec_and_queue(P, u, 1ull, k, Fnext, next_cnt);
                    destroyed++;
                    bytes += 16;
                } else if (su == kFront && u > v) {
                    destroyed++;
                }
            }
        } else {
            for (uint64_t t = gwarp; t < T; t += gwarps) {
                uint32_t lo = 0, hi = nf;
                while (hi - lo > 1) {
                    uint32_t mid = (lo + hi) >> 1;
                    if (s_pre[mid] <= t) lo = mid; else hi = mid;
                }
                uint32_t v = F[lo];
                uint32_t w = P.wadj[P.off[v] + (t - s_pre[lo])];
                const uint32_t* vbm = (bm && lo < kBitmapSlots) ? bm + (size_t)lo * bm_words : nullptr;
                const uint32_t* gbm = hl ? hub_bm_of(P, v, par) : nullptr;
                process_vw(P, v, w, k, Fnext, next_cnt, wC, wCnt, wRows, big_cnt, vbm, gbm,
                           destroyed, bytes);
            }
        }
    } else if (P.h == 2) {
        for (uint64_t i = gwarp; i < nf; i += gwarps) {
            uint32_t v = F[i];
            if (P.deg[v] == 0) continue;
            uint64_t b = P.off[v], e = P.wend[v];
            for (uint64_t p = b + lane; p < e; p += 32) {
                uint32_t u = P.wadj[p];
                uint32_t su = st_of(P.sl[u]);
                bytes += 4 + 4;
                if (su == kAlive) {
                    dec_and_queue(P, u, 1ull, k, Fnext, next_cnt);
                    destroyed++;
                    bytes += 16;
                } else if (su == kFront && u > v) {
                    destroyed++;
                }
            }
            if (lane == 0) {
                items += e - b;
                bytes += 20;
            }
        }
    } else {
        // Large regime: the items of heavy vertices (hl, nh: rows longer than
        // heavy_min, flagged kHeavyBit) are flattened over every warp of the
        // grid in batches of kSmallFront vertices; every other vertex goes to
        // one block, blocks taking chunks of the frontier from *grab.  In the
        // small regime (hl null) blocks take the vertices in a fixed order.
        if (hl) {
            for (uint32_t b0 = 0; b0 < nh; b0 += kSmallFront) {
                const uint32_t nb = nh - b0 < kSmallFront ? nh - b0 : kSmallFront;
                const uint32_t* H = hl + b0;
                block_prefix_degrees<NT>(P, H, nb, s_pre, s_red, true);
                unsigned long long T = s_pre[nb];
                if (blockIdx.x == 0 && threadIdx.x == 0) {
                    items += T;
                    bytes += 20ull * nb;
                }
                for (uint64_t t = gwarp; t < T; t += gwarps) {
                    uint32_t lo = 0, hi = nb;
                    while (hi - lo > 1) {
                        uint32_t mid = (lo + hi) >> 1;
                        if (s_pre[mid] <= t) lo = mid; else hi = mid;
                    }
                    uint32_t v = H[lo];
                    uint32_t w = P.wadj[P.off[v] + (t - s_pre[lo])];
                    process_vw(P, v, w, k, Fnext, next_cnt, wC, wCnt, wRows, big_cnt, nullptr,
                               hub_bm_of(P, v, par), destroyed, bytes);
                }
                __syncthreads();   // s_pre is rewritten by the next batch
            }
            const uint32_t ch0 = nf / (4u * gridDim.x);
            const uint32_t ch = ch0 < 1u ? 1u : (ch0 > 32u ? 32u : ch0);
            for (;;) {
                if (threadIdx.x == 0) *s_grab = atomicAdd(grab, ch);
                __syncthreads();
                const uint32_t i0 = *s_grab;
                __syncthreads();
                if (i0 >= nf) break;
                const uint32_t i1 = i0 + ch < nf ? i0 + ch : nf;
                for (uint32_t i = i0; i < i1; i++) {
                    uint32_t v = F[i];
                    if ((P.sl[v] & kHeavyBit) || P.deg[v] == 0) continue;   // taken above, or none
                    uint64_t b = P.off[v], e = P.wend[v];
                    for (uint64_t p = b + wid; p < e; p += NW)
                        process_vw(P, v, P.wadj[p], k, Fnext, next_cnt, wC, wCnt, wRows, big_cnt,
                                   nullptr, nullptr, destroyed, bytes);
                    if (threadIdx.x == 0) {
                        items += e - b;
                        bytes += 24;
                    }
                }
            }
            return;
        }
        for (uint64_t i = blockIdx.x; i < nf; i += gridDim.x) {
            uint32_t v = F[i];
            if (P.deg[v] == 0) continue;
            uint64_t b = P.off[v], e = P.wend[v];
            const uint32_t* vbm = (bm && i < kBitmapSlots) ? bm + (size_t)i * bm_words : nullptr;
            for (uint64_t p = b + wid; p < e; p += NW)
                process_vw(P, v, P.wadj[p], k, Fnext, next_cnt, wC, wCnt, wRows, big_cnt, vbm,
                           nullptr, destroyed, bytes);
            if (threadIdx.x == 0) {
                items += e - b;
                bytes += 20;
            }
        }
    }
}

// Shared bitmaps over local ids of the neighbourhoods of F[0..min(nf,
// kBitmapSlots)), built by every block (small regime).
template <int NT>
__device__ __forceinline__ void build_bitmaps(const PeelParams& P, const uint32_t* F, uint32_t nf,
                                              uint32_t* bm, uint32_t bm_words) {
    uint32_t slots = nf < kBitmapSlots ? nf : kBitmapSlots;
    for (uint32_t i = threadIdx.x; i < slots * bm_words; i += NT) bm[i] = 0;
    __syncthreads();
    const unsigned nw = NT / 32;
    for (uint32_t s = warp_id(); s < slots; s += nw) {
        uint32_t v = F[s];
        uint64_t b = P.off[v], e = P.wend[v];
        uint32_t* row = bm + (size_t)s * bm_words;
        for (uint64_t p = b + lane_id(); p < e; p += 32) {
            uint32_t x = P.wadj[p];
            uint32_t w = P.sl[x];
            // removed vertices may lack a local id; they are never candidates
            if (st_of(w) != kGone) {
                uint32_t l = w >> 2;
                atomicOr(&row[l >> 5], 1u << (l & 31));
            }
        }
    }
    __syncthreads();
}

// ---------------------------------------------------------------- kernel
template <int NT>
__global__ void __launch_bounds__(NT, 1024 / NT) k_peel(PeelParams P) {
    constexpr int NW = NT / 32;
    extern __shared__ uint32_t smem[];
    __shared__ unsigned long long s_pre[kSmallFront + 1];
    __shared__ unsigned long long s_red[NW];
    __shared__ uint32_t s_wtot[NW];
    __shared__ uint32_t s_n;
    __shared__ uint32_t s_grab;
    PeelCtrl* c = P.ctrl;
    const unsigned lane = lane_id(), wid = warp_id();
    const uint64_t gtid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t gthreads = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t gwarp = gtid >> 5;
    const uint64_t gwarps = gthreads >> 5;
    uint32_t* wC = smem + (size_t)wid * kWarpWords;
    unsigned* wCnt = wC + kWarpCand;
    uint32_t* wRows = wC + 2 * kWarpCand;
    uint32_t* sA = smem + P.work_words;   // small regime: alive list
    uint32_t* sF = sA + P.asmall;         // small regime: frontier
    uint32_t* sBM = sF + P.asmall;        // small regime: neighbourhood bitmaps
    const uint32_t bm_words = (P.asmall + 31) / 32;
    const bool lead = blockIdx.x == 0 && threadIdx.x == 0;

    unsigned long long k = P.k0;           // level floor (threshold pruning when > 0)
    unsigned long long mu_alive = P.mu0;   // meaningful in block 0
    uint32_t r = 0, jumps = 0, nlev = 0, nbar = 0, ncompact = 0;
    int ap = 0;
    uint32_t alive_cnt = P.n;
    uint32_t compacted_at = P.n;           // alive count at the last row compaction
    bool small = false;
    uint32_t na_s = 0, nf_s = 0;           // small regime: alive total, frontier size
    uint32_t na_entry = 0;                 // alive vertices when the small regime began
    uint32_t slice_lo = 0, na_loc = 0;     // this block's slice of the alive list
    uint32_t cmp_loc = 0;                  // slice size at its last row compaction
    unsigned long long items = 0, bytes = 0, waited = 0;

    // Block 0's time per phase (thread 0, %globaltimer); the time inside
    // barriers is counted separately in `waited`.
    __shared__ unsigned long long tph[8];
    if (threadIdx.x < 8) tph[threadIdx.x] = 0;
    uint64_t tlast = lead ? globaltimer_ns() : 0;
#define PHASE(i)                                 \
    do {                                         \
        if (lead) {                              \
            uint64_t t_ = globaltimer_ns();      \
            tph[i] += t_ - tlast;                \
            tlast = t_;                          \
        }                                        \
    } while (0)
#define BARRIER(i)                                         \
    do {                                                   \
        PHASE(i);                                          \
        nbar++;                                            \
        if (!grid_barrier(c, P.wait_ns, waited)) goto out; \
        if (lead) tlast = globaltimer_ns();                \
    } while (0)

    for (;;) {
        bool s_jump = false;
        if (!small) {
            // ------------------------------------------------------ P1
            {
                uint32_t fprev = r ? c->fcnt[(r + 2) % 3] : 0u;
                const uint32_t* Fprev = P.front[(r + 2) % 3];
                for (uint64_t i = gtid; i < fprev; i += gthreads) {
                    uint32_t v = Fprev[i];
                    P.sl[v] = kGone;
                    P.core[v] = k;
                    if (P.rnd) P.rnd[v] = r - 1;
                    bytes += 4 + 4 + 8 + (P.rnd ? 4 : 0);
                }
            }
            uint32_t fcur = c->fcnt[r % 3];
            uint32_t* Fcur = P.front[r % 3];
            // the bitmaps of F_{r-1}'s hubs are zeroed for round r+1
            if (r && P.hub_slots) {
                uint32_t nhub = c->hubcnt[(r + 1) & 1];
                if (nhub > P.hub_slots) nhub = P.hub_slots;
                if (nhub) hub_bitmaps<NT>(P, nhub, (r + 1) & 1, true, s_pre, s_red, bytes);
            }
            // mark F_r; rows longer than heavy_min also go to the heavy list
            for (uint64_t base = gwarp * 32; base < fcur; base += gwarps * 32) {
                uint64_t i = base + lane;
                bool hv = false;
                uint32_t v = 0;
                if (i < fcur) {
                    v = Fcur[i];
                    P.sl[v] = P.heavy_min ? front_word(P, c, v, r & 1, hv) : (uint32_t)kFront;
                    bytes += 4 + 4 + (P.heavy_min ? 16 : 0);
                }
                if (P.heavy_min) warp_append(hv, v, &c->hcnt[r % 3], P.heavy);
            }
            if (lead) {
                if (r) {
                    mu_alive -= c->destroyed[(r + 2) % 3];
                    c->destroyed[(r + 2) % 3] = 0;
                    c->big_cnt[(r + 2) % 3] = 0;
                    c->bgrab[(r + 2) % 3] = 0;
                    c->big_cnt[3 + (r + 2) % 3] = 0;
                    c->bgrab[3 + (r + 2) % 3] = 0;
                }
                c->fcnt[(r + 1) % 3] = 0;
                c->hcnt[(r + 1) % 3] = 0;
                c->grab[(r + 1) % 3] = 0;
            }
            BARRIER(0);

            // ------------------------------------------------- level jump
            if (fcur == 0) {
                const uint32_t* Ain = P.alive[ap];
                uint32_t* Aout = P.alive[ap ^ 1];
                unsigned long long mn = ~0ull;
                for (uint64_t base = gwarp * 32; base < alive_cnt; base += gwarps * 32) {
                    uint64_t i = base + lane;
                    bool keep = false;
                    uint32_t v = 0;
                    if (i < alive_cnt) {
                        v = Ain[i];
                        bytes += 4 + 4;
                        if (st_of(P.sl[v]) != kGone) {
                            keep = true;
                            unsigned long long d = P.deg[v];
                            mn = d < mn ? d : mn;
                            if (P.snap) P.snap[v] = d;
                            bytes += 8 + 4;
                        }
                    }
                    warp_append(keep, v, &c->new_alive[jumps & 1], Aout);
                }
                mn = warp_min_u64(mn);
                if (lane == 0 && mn != ~0ull) atomicMin(&c->min_deg[jumps & 1], mn);
                BARRIER(1);
                uint32_t na = c->new_alive[jumps & 1];
                if (na == 0) break;
                ap ^= 1;
                alive_cnt = na;
                if (na <= P.asmall) {
                    // enter the small regime: each block keeps its slice of
                    // the alive list in shared memory and gives those vertices
                    // their local id (the position in the list)
                    na_entry = na;
                    slice_lo = (uint32_t)((uint64_t)na * blockIdx.x / gridDim.x);
                    na_loc = (uint32_t)((uint64_t)na * (blockIdx.x + 1) / gridDim.x) - slice_lo;
                    cmp_loc = na_loc;
                    for (uint32_t i = threadIdx.x; i < na_loc; i += NT) {
                        uint32_t v = Aout[slice_lo + i];
                        sA[i] = v;
                        P.sl[v] = ((slice_lo + i) << 2) | kAlive;
                    }
                    if (lead) {
                        c->small_round = r;
                        bytes += 12ull * na;
                    }
                    small = true;
                    na_s = na;
                    nf_s = 0;
                    s_jump = true;
                    __syncthreads();
                } else {
                    unsigned long long m2 = c->min_deg[jumps & 1];
                    k = m2 > k ? m2 : k;
                    if (lead) {
                        P.lvl_k[nlev] = k;
                        P.lvl_size[nlev] = na;
                        P.lvl_mu[nlev] = mu_alive;
                        c->min_deg[(jumps + 1) & 1] = ~0ull;
                        c->new_alive[(jumps + 1) & 1] = 0;
                    }
                    nlev++;
                    jumps++;
                    // Rows may be compacted in this same phase: compaction keeps
                    // every vertex that is not removed, whether or not it is
                    // being marked frontier concurrently.
                    if (P.compact && 2ull * na <= compacted_at) {
                        compacted_at = na;
                        ncompact++;
                        for (uint64_t i = gwarp; i < na; i += gwarps) compact_row(P, Aout[i], bytes);
                    }
                    for (uint64_t base = gwarp * 32; base < na; base += gwarps * 32) {
                        uint64_t i = base + lane;
                        bool in = false, hv = false;
                        uint32_t v = 0;
                        if (i < na) {
                            v = Aout[i];
                            bytes += 4 + 8;
                            if (P.deg[v] <= k) {
                                in = true;
                                P.sl[v] = P.heavy_min ? front_word(P, c, v, r & 1, hv)
                                                      : (uint32_t)kFront;
                                bytes += 4 + 4 + (P.heavy_min ? 16 : 0);
                            }
                        }
                        warp_append(in, v, &c->fcnt[r % 3], Fcur);
                        if (P.heavy_min) warp_append(hv, v, &c->hcnt[r % 3], P.heavy);
                    }
                    BARRIER(2);
                    fcur = c->fcnt[r % 3];
                }
            }
            if (!small) {
                // -------------------------------------------------- P2
                if (P.hub_slots) {
                    uint32_t nhub = c->hubcnt[r & 1];
                    if (nhub > P.hub_slots) nhub = P.hub_slots;
                    if (lead) c->hubcnt[(r + 1) & 1] = 0;   // read last in this round's P1
                    if (nhub) {
                        hub_bitmaps<NT>(P, nhub, r & 1, false, s_pre, s_red, bytes);
                        BARRIER(3);
                    }
                }
                unsigned long long destroyed = 0;
                process_frontier<NT>(P, Fcur, fcur, k, P.front[(r + 1) % 3],
                                     &c->fcnt[(r + 1) % 3], &c->big_cnt[r % 3], wC, wCnt,
                                     wRows, nullptr, 0, s_pre, s_red,
                                     P.heavy_min ? P.heavy : nullptr, c->hcnt[r % 3],
                                     &c->grab[r % 3], &s_grab, r & 1, destroyed, items, bytes);
                unsigned long long bd = block_sum<NT>(destroyed, s_red);
                if (threadIdx.x == 0 && bd) atomicAdd(&c->destroyed[r % 3], bd);
                BARRIER(3);
                // ------------------------------------------------- P2b
                if (P.big_cap) {
                    uint32_t nb = c->big_cnt[r % 3];
                    uint32_t nm = c->big_cnt[3 + r % 3];
                    if (nb || nm) {
                        if (nb > P.big_cap) nb = (uint32_t)P.big_cap;
                        if (nm > P.mid_cap) nm = P.mid_cap;
                        if (nm) {
                            drain_mid<NT>(P, nm, &c->bgrab[3 + r % 3], k, P.front[(r + 1) % 3],
                                          &c->fcnt[(r + 1) % 3], &c->destroyed[r % 3], bytes);
                            __syncthreads();
                        }
                        unsigned long long d2 = 0;
                        for (;;) {
                            if (threadIdx.x == 0) s_grab = atomicAdd(&c->bgrab[r % 3], 1u);
                            __syncthreads();
                            const uint32_t i = s_grab;
                            __syncthreads();
                            if (i >= nb) break;
                            uint2 it = P.big[i];
                            process_big(P, it.x, it.y, k, P.front[(r + 1) % 3],
                                        &c->fcnt[(r + 1) % 3], smem, hub_bm_of(P, it.x, r & 1),
                                        d2, bytes);
                        }
                        if (threadIdx.x == 0 && d2) atomicAdd(&c->destroyed[r % 3], d2);
                        BARRIER(3);
                    }
                }
                r++;
                continue;
            }
        }

        // ========================================================= small
        if (!s_jump) {
            // retire F_{r-1}: identical writes in every block
            for (uint32_t i = threadIdx.x; i < nf_s; i += NT) {
                uint32_t v = sF[i];
                P.sl[v] = (P.sl[v] & ~3u) | kGone;
                P.core[v] = k;
                if (P.rnd) P.rnd[v] = r - 1;
            }
            if (lead) bytes += (20ull + (P.rnd ? 4 : 0)) * nf_s;
            if (lead) {
                mu_alive -= c->destroyed[(r + 2) % 3];
                c->destroyed[(r + 2) % 3] = 0;
                c->big_cnt[(r + 2) % 3] = 0;
                c->bgrab[(r + 2) % 3] = 0;
                c->big_cnt[3 + (r + 2) % 3] = 0;
                c->bgrab[3 + (r + 2) % 3] = 0;
            }
            uint32_t nf_new = c->fcnt[r % 3];
            __syncthreads();
            if (nf_new) {
                const uint32_t* G = P.front[r % 3];
                for (uint32_t i = threadIdx.x; i < nf_new; i += NT) sF[i] = G[i];
                if (lead) bytes += 4ull * nf_new;
                nf_s = nf_new;
            } else {
                s_jump = true;
            }
        }
        // the counter that collects round r+2's appends was last read at the
        // start of round r-1
        if (lead) c->fcnt[(r + 2) % 3] = 0;
        PHASE(4);
        if (s_jump) {
            // Level jump over the alive set, distributed: each block compacts
            // its own slice (kept in shared memory), takes the slice minimum
            // and the slice vertices attaining it, and publishes them; after
            // the barrier every block combines the slice minima and gathers the
            // frontier from the slices that attain the global minimum.
            uint32_t kept = 0;
            unsigned long long lmin = ~0ull;
            {
                if (threadIdx.x == 0) s_n = 0;
                __syncthreads();
                for (uint32_t base = 0; base < na_loc; base += NT) {
                    uint32_t i = base + threadIdx.x;
                    uint32_t v = i < na_loc ? sA[i] : 0u;
                    uint32_t s = i < na_loc ? st_of(P.sl[v]) : (uint32_t)kGone;
                    unsigned long long d = i < na_loc ? P.deg[v] : ~0ull;
                    bool keep = s == kAlive;
                    if (keep) lmin = d < lmin ? d : lmin;
                    if (keep && P.snap) P.snap[v] = d;
                    uint32_t tot;
                    uint32_t at = block_scan_count<NT>(keep ? 1u : 0u, s_wtot, &tot);
                    uint32_t o = s_n;
                    __syncthreads();   // every read of this pass precedes any write
                    if (keep) sA[o + at] = v;
                    __syncthreads();
                    if (threadIdx.x == 0) s_n = o + tot;
                }
                __syncthreads();
                kept = s_n;
                if (lead) bytes += 16ull * na_entry;
            }
            lmin = warp_min_u64(lmin);
            if (lane == 0) s_red[wid] = lmin;
            __syncthreads();
            lmin = ~0ull;
            for (int w = 0; w < NW; w++) lmin = s_red[w] < lmin ? s_red[w] : lmin;
            __syncthreads();
            na_loc = kept;
            // the slice vertices attaining the slice minimum, published in
            // this block's part of the jump list
            {
                if (threadIdx.x == 0) s_n = 0;
                __syncthreads();
                for (uint32_t base = 0; base < na_loc; base += NT) {
                    uint32_t i = base + threadIdx.x;
                    uint32_t v = i < na_loc ? sA[i] : 0u;
                    bool in = i < na_loc && P.deg[v] == lmin;
                    uint32_t tot;
                    uint32_t at = block_scan_count<NT>(in ? 1u : 0u, s_wtot, &tot);
                    uint32_t o = s_n;
                    if (in) P.jf[slice_lo + o + at] = v;
                    __syncthreads();
                    if (threadIdx.x == 0) s_n = o + tot;
                }
                __syncthreads();
                if (threadIdx.x == 0) {
                    P.jblk[blockIdx.x] = make_ulonglong2(lmin, ((unsigned long long)na_loc << 32) | s_n);
                }
            }
            // rows of this slice lose their removed entries once the slice
            // has halved (no block reads rows during this phase)
            if (P.compact && 2ull * na_loc <= cmp_loc) {
                cmp_loc = na_loc;
                ncompact++;
                for (uint32_t i = wid; i < na_loc; i += NW) compact_row(P, sA[i], bytes);
            }
            // Every block must have read the counts for this jump before any
            // block starts the round's decrements.
            BARRIER(5);
            // combine: global minimum, alive count, and the frontier
            {
                unsigned long long gm = ~0ull;
                unsigned long long tot_alive = 0;
                uint32_t cnt_t = 0;
                unsigned long long min_t = ~0ull;
                if (threadIdx.x < gridDim.x) {
                    ulonglong2 e = P.jblk[threadIdx.x];
                    min_t = e.x;
                    tot_alive = e.y >> 32;
                    cnt_t = (uint32_t)(e.y & 0xffffffffull);
                    gm = min_t;
                }
                gm = warp_min_u64(gm);
                tot_alive = warp_sum(tot_alive);
                if (lane == 0) {
                    s_red[wid] = gm;
                    s_pre[wid] = tot_alive;
                }
                __syncthreads();
                gm = ~0ull;
                tot_alive = 0;
                for (int w = 0; w < NW; w++) {
                    gm = s_red[w] < gm ? s_red[w] : gm;
                    tot_alive += s_pre[w];
                }
                __syncthreads();
                if (tot_alive == 0) break;
                if (tot_alive <= P.tail_max) {
                    // Hand the rest to the cluster tail kernel: every block
                    // writes its compacted slice into one list (blocks in
                    // order) and gives those vertices their tail local ids.
                    uint32_t before_me = 0;
                    if (threadIdx.x < gridDim.x && threadIdx.x < blockIdx.x)
                        before_me = (uint32_t)(P.jblk[threadIdx.x].y >> 32);
                    uint32_t base;
                    block_scan_count<NT>(before_me, s_wtot, &base);
                    for (uint32_t i = threadIdx.x; i < na_loc; i += NT) {
                        uint32_t v = sA[i];
                        P.alive[0][base + i] = v;
                        P.sl[v] = ((base + i) << 2) | kAlive;
                    }
                    if (lead) {
                        c->tail_n = (uint32_t)tot_alive;
                        c->tail_round = r;
                        c->tail_entry = (uint32_t)tot_alive;
                        c->tail_entry_round = r;
                        c->mu_tail = mu_alive;
                        bytes += 12ull * tot_alive;
                    }
                    break;
                }
                k = gm > k ? gm : k;
                na_s = (uint32_t)tot_alive;
                if (lead) {
                    P.lvl_k[nlev] = k;
                    P.lvl_size[nlev] = na_s;
                    P.lvl_mu[nlev] = mu_alive;
                }
                nlev++;
                // frontier = the published vertices of slices whose minimum is gm
                uint32_t take = (threadIdx.x < gridDim.x && min_t == gm) ? cnt_t : 0u;
                uint32_t tot;
                uint32_t at = block_scan_count<NT>(take, s_wtot, &tot);
                if (threadIdx.x < gridDim.x) {
                    s_pre[threadIdx.x] = ((unsigned long long)at << 32) | take;
                }
                __syncthreads();
                for (uint32_t t = wid; t < gridDim.x; t += NW) {
                    unsigned long long e = s_pre[t];
                    uint32_t ct = (uint32_t)(e & 0xffffffffull), o = (uint32_t)(e >> 32);
                    uint64_t lo = (uint64_t)na_entry * t / gridDim.x;
                    for (uint32_t j = lane; j < ct; j += 32) sF[o + j] = P.jf[lo + j];
                }
                nf_s = tot;
                if (lead) bytes += 16ull * gridDim.x + 8ull * nf_s;
                __syncthreads();
            }
        }
        // mark the frontier (identical writes in every block)
        for (uint32_t i = threadIdx.x; i < nf_s; i += NT) {
            uint32_t v = sF[i];
            P.sl[v] = (P.sl[v] & ~3u) | kFront;
        }
        if (lead) bytes += 8ull * nf_s;
        __syncthreads();
        if (P.h >= 3) build_bitmaps<NT>(P, sF, nf_s, sBM, bm_words);
        PHASE(6);
        {
            unsigned long long destroyed = 0;
            process_frontier<NT>(P, sF, nf_s, k, P.front[(r + 1) % 3], &c->fcnt[(r + 1) % 3],
                                 &c->big_cnt[r % 3], wC, wCnt, wRows, P.h >= 3 ? sBM : nullptr,
                                 bm_words, s_pre, s_red, nullptr, 0, nullptr, nullptr, 0,
                                 destroyed, items, bytes);
            unsigned long long bd = block_sum<NT>(destroyed, s_red);
            if (threadIdx.x == 0 && bd) atomicAdd(&c->destroyed[r % 3], bd);
            BARRIER(7);
            if (P.big_cap) {
                uint32_t nb = c->big_cnt[r % 3];
                uint32_t nm = c->big_cnt[3 + r % 3];
                if (nb || nm) {
                    if (nb > P.big_cap) nb = (uint32_t)P.big_cap;
                    if (nm > P.mid_cap) nm = P.mid_cap;
                    if (nm) {
                        drain_mid<NT>(P, nm, &c->bgrab[3 + r % 3], k, P.front[(r + 1) % 3],
                                      &c->fcnt[(r + 1) % 3], &c->destroyed[r % 3], bytes);
                        __syncthreads();
                    }
                    unsigned long long d2 = 0;
                    for (;;) {
                        if (threadIdx.x == 0) s_grab = atomicAdd(&c->bgrab[r % 3], 1u);
                        __syncthreads();
                        const uint32_t i = s_grab;
                        __syncthreads();
                        if (i >= nb) break;
                        uint2 it = P.big[i];
                        process_big(P, it.x, it.y, k, P.front[(r + 1) % 3],
                                    &c->fcnt[(r + 1) % 3], smem, nullptr, d2, bytes);
                    }
                    if (threadIdx.x == 0 && d2) atomicAdd(&c->destroyed[r % 3], d2);
                    BARRIER(7);
                }
            }
        }
        r++;
    }
out:
#undef BARRIER
#undef PHASE
    if (lead) {
        for (int i = 0; i < 8; i++) c->tph[i] = tph[i];
        c->kmax = k;
        c->nlevels = nlev;
        c->rounds = r;
        c->barrier_ns = waited;
        c->barriers = nbar;
        c->compactions = ncompact;
    }
    items = warp_sum(items);
    bytes = warp_sum(bytes);
    if (lane == 0 && items) atomicAdd(&c->items, items);
    if (lane == 0 && bytes) atomicAdd(&c->bytes, bytes);
}

__global__ void k_peel_init(uint32_t n, const uint64_t* off, const uint64_t* split,
                            uint32_t* sl, uint32_t* alive0, uint64_t* wend, uint64_t* wnb,
                            PeelCtrl* c) {
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x) {
        sl[i] = kAlive;
        alive0[i] = (uint32_t)i;
        wend[i] = off[i + 1];
        wnb[i] = split ? split[i] : off[i];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        c->min_deg[0] = ~0ull;
        c->min_deg[1] = ~0ull;
    }
}

#include "peel_tail.inc"

// Tail launch shapes: the largest cluster this device co-schedules (16,
// else 8) and the largest alive set whose per-CTA state fits its shared
// memory; `grows` selects rows in global memory.
struct TailShape {
    uint32_t cs = 0, cap = 0;
    size_t smem = 0;
};

TailShape find_tail_shape(bool grows) {
    TailShape t;
    const size_t budget = 220 * 1024;
    const void* fn = grows ? (const void*)k_peel_tail<true> : (const void*)k_peel_tail<false>;
    for (uint32_t cs : {16u, 8u}) {
        uint32_t cap = 0;
        for (uint32_t cc = 32 * cs; cc <= kTailMaxAlive; cc += 32 * cs) {
            size_t scratch = grows ? SIZE_MAX : (size_t)(cc / cs) * (cc / 32) * 4;
            if (tail_smem_bytes(grows, cc, cs) <= budget && tail_np(cc) * 4 <= scratch &&
                (grows || cc <= 8192))
                cap = cc;
        }
        if (!cap) continue;
        size_t smem = tail_smem_bytes(grows, cap, cs);
        if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
                cudaSuccess ||
            (cs > 8 &&
             cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) !=
                 cudaSuccess)) {
            (void)cudaGetLastError();
            continue;
        }
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = cs;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.gridDim = dim3(cs);
        cfg.blockDim = dim3(kTailNT);
        cfg.dynamicSmemBytes = smem;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        int nc = 0;
        if (cudaOccupancyMaxActiveClusters(&nc, fn, &cfg) != cudaSuccess) {
            (void)cudaGetLastError();
            continue;
        }
        if (nc >= 1) {
            t.cs = cs;
            t.cap = cap;
            t.smem = smem;
            break;
        }
    }
    return t;
}

const TailShape& tail_shape(bool grows) {
    static TailShape cached[2];
    static bool done[2] = {false, false};
    if (!done[grows]) {
        cached[grows] = find_tail_shape(grows);
        done[grows] = true;
    }
    return cached[grows];
}

template <bool GROWS>
cudaError_t launch_tail(const TailParams& T, const TailShape& sh, cudaStream_t s) {
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = sh.cs;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(sh.cs);
    cfg.blockDim = dim3(kTailNT);
    cfg.dynamicSmemBytes = sh.smem;
    cfg.stream = s;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    note_launch();
    return cudaLaunchKernelEx(&cfg, k_peel_tail<GROWS>, T);
}

// Failure detection: the grid barrier of k_peel with one block withheld
// (absent >= 0), so that every other block's bounded wait runs out and sets
// the timeout flag; absent < 0 passes four barriers normally.
__global__ void k_barrier_probe(PeelCtrl* c, uint64_t wait_ns, int absent) {
    unsigned long long waited = 0;
    if ((int)blockIdx.x == absent) return;
    for (int i = 0; i < 4; i++)
        if (!grid_barrier(c, wait_ns, waited)) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) c->barriers = 4;
}

template <int NT>
cudaError_t launch_peel(PeelParams& P, int sms, size_t smem, cudaStream_t s, unsigned* grid_out) {
    // opt in for every launch: the 48 KB default bounds static + dynamic
    // shared memory together, and the attribute persists across calls
    cudaError_t e = cudaFuncSetAttribute(k_peel<NT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_peel<NT>, NT, smem);
    if (e != cudaSuccess) return e;
    if (per_sm <= 0) return cudaErrorInvalidConfiguration;
    // one block per SM: the fewest barrier arrivals; every block holds the
    // small-regime lists in its own shared memory
    unsigned grid = (unsigned)sms;
    *grid_out = grid;
    void* args[] = {&P};
    e = cudaLaunchCooperativeKernel((void*)k_peel<NT>, dim3(grid), dim3(NT), args, smem, s);
    note_launch();
    return e;
}

}  // namespace

dsd_status run_peel(dsd_graph* g, int h, uint32_t n, const uint64_t* off, const uint32_t* adj,
                    const uint64_t* split, uint32_t maxdplus, unsigned long long* deg,
                    uint64_t mu0, uint64_t* core, uint32_t* rnd, uint64_t* lvl_k,
                    uint32_t* lvl_size, uint64_t* lvl_mu, PeelResult* res,
                    uint64_t kstart, uint64_t* snap) {
    cudaStream_t s = g->stream;
    *res = PeelResult();
    if (n == 0) return DSD_OK;
    int sms = 152;
    DSD_TRY(num_sms(&sms));
    PeelParams P;
    memset(&P, 0, sizeof(P));
    P.n = n;
    P.h = h;
    P.off = off;
    P.deg = deg;
    P.core = core;
    P.rnd = rnd;
    P.lvl_k = lvl_k;
    P.lvl_size = lvl_size;
    P.lvl_mu = lvl_mu;
    P.wait_ns = wait_limit_ns();
    P.mu0 = mu0;
    P.k0 = kstart ? kstart - 1 : 0;
    P.snap = snap;
    P.cap = maxdplus < 32 ? 32 : maxdplus;
    P.bcap = P.cap < kBitmapMax ? P.cap : kBitmapMax;
    P.warp_cand = warp_cand_limit(h);
    P.gather_cap = P.warp_cand;
    P.compact = h >= 3 ? 1 : 0;
    // Big items (candidate sets above kWarpCand vertices, one block each)
    // for h >= 4; every candidate set fits 32-word rows.
    const bool big_items = h >= 4;
    // Shared memory: per-warp candidate buffers (h >= 3) or the big-item
    // bitmap, then the small-regime alive list, frontier and
    // neighbourhood bitmaps.
    const size_t budget = 220 * 1024;
    constexpr int NT = 1024;
    size_t work = h >= 3 ? (size_t)(NT / 32) * kWarpWords : 0;
    // large-regime frontier vertices with more items than a block's warps
    // take in four passes have their items spread over the whole grid
    P.heavy_min = h >= 3 ? 4u * (NT / 32) : 0u;
    // neighbourhood bitmaps for frontier vertices with rows above 512 (a
    // binary search there takes 10 or more probes): up to 64 per round, two
    // sets, within 64 MiB
    if (h >= 3) {
        P.hub_words = ((uint64_t)n + 31) / 32;
        uint64_t slots = (64ull << 20) / (2 * 4 * P.hub_words);
        P.hub_slots = (uint32_t)(slots > 64 ? 64 : (slots < 4 ? 0 : slots));
        P.hub_min = 4 * P.heavy_min;
    }
    if (big_items) {
        size_t W = (P.bcap + 31) / 32;
        size_t big = (size_t)3 * P.bcap + (size_t)P.bcap * W;
        // the split search of oversized sets uses the full bitmap tier layout
        if (P.cap > kBitmapMax) big = (size_t)3 * kBitmapMax + (size_t)kBitmapMax * 32;
        if (big > work) work = big;
    }
    size_t room = budget > work * 4 + 12 * 1024 ? budget - work * 4 - 12 * 1024 : 0;
    // per alive entry: list 4 B + frontier 4 B + one bit per bitmap slot
    size_t per_entry_bits = 64 + (h >= 3 ? kBitmapSlots : 0);
    size_t asmall = room * 8 / per_entry_bits;
    asmall &= ~(size_t)31;
    if (asmall > 16384) asmall = 16384;
    if (asmall > peel_small_limit()) asmall = peel_small_limit() & ~31u;
    if (asmall < 1024) asmall = 0;
    // the jump combines one entry per block in a single pass over the threads
    if (sms > NT || sms > 1024) asmall = 0;
    P.work_words = (uint32_t)work;
    P.asmall = (uint32_t)asmall;
    TailShape tsh_d, tsh_g;   // rows in distributed shared memory / in global memory
    if ((h == 2 || h == 3) && asmall > 0 && peel_tail_limit() > 0 && !snap) {
        tsh_d = tail_shape(false);
        // global rows pay for h = 3 only: an h = 2 round is too cheap for the
        // wider rows (measured on the 1M-vertex Chung-Lu graph)
        if (tsh_d.cs && h == 3) tsh_g = tail_shape(true);
        uint32_t tmax = tsh_g.cs && tsh_g.cap > tsh_d.cap ? tsh_g.cap : tsh_d.cap;
        if (tmax > peel_tail_limit()) tmax = peel_tail_limit();
        if (tmax <= tsh_d.cap) tsh_g = TailShape();   // the global-row launch is not needed
        if (tsh_d.cs) P.tail_max = tmax;
    }
    size_t bm_words = h >= 3 ? (size_t)kBitmapSlots * (asmall / 32) : 0;
    size_t smem = (work + 2 * asmall + bm_words) * 4;

    uint32_t* sl = nullptr;
    uint32_t* lists = nullptr;
    uint64_t* wmeta = nullptr;
    uint32_t* wadj = nullptr;
    PeelCtrl* ctrl = nullptr;
    uint32_t* rows_g = nullptr;
    uint2* big = nullptr;
    uint32_t* mid = nullptr;
    uint32_t* heavy = nullptr;
    uint32_t* xl = nullptr;
    uint32_t* hub_bm = nullptr;
    uint32_t* hubs = nullptr;
    ulonglong2* jblk = nullptr;
    dsd_status st = DSD_OK;
    PeelCtrl hc;
    unsigned grid = 0;
    cudaError_t e = cudaSuccess;
    const uint64_t nadj = 2 * g->m;   // both CSRs of g hold 2m entries
    if ((st = dalloc(&sl, n, s)) != DSD_OK) goto done;
    if ((st = dalloc(&lists, (size_t)6 * n, s)) != DSD_OK) goto done;
    if ((st = dalloc(&jblk, 1024, s)) != DSD_OK) goto done;
    if ((st = dalloc(&wmeta, (size_t)2 * n, s)) != DSD_OK) goto done;
    if ((st = dalloc(&wadj, nadj + 1, s)) != DSD_OK) goto done;
    if ((st = dalloc(&ctrl, 1, s)) != DSD_OK) goto done;
    if (tsh_g.cs &&
        (st = dalloc(&rows_g, (size_t)tsh_g.cap * (tsh_g.cap / 32), s)) != DSD_OK)
        goto done;
    if (big_items) {
        P.big_cap = g->m * 2 + 1;
        if ((st = dalloc(&big, P.big_cap, s)) != DSD_OK) goto done;
        // mid items (sets of warp_cand + 1 .. 32 candidates): up to 2^20 per
        // round (144 MB), the rest as big items
        uint64_t mc = P.big_cap < (1u << 20) ? P.big_cap : (1u << 20);
        if (mc > peel_item_mid_limit()) mc = peel_item_mid_limit();
        if (P.warp_cand < kWarpCand && mc > 0) {
            if ((st = dalloc(&mid, (size_t)mc * kMidWords, s)) != DSD_OK) goto done;
            P.mid = mid;
            P.mid_cap = (uint32_t)mc;
            P.gather_cap = kWarpCand;
        }
    }
    if (P.heavy_min && (st = dalloc(&heavy, n, s)) != DSD_OK) goto done;
    P.heavy = heavy;
    if (big_items && P.cap > kBitmapMax &&
        (st = dalloc(&xl, (size_t)sms * (kMaxDepth + 1) * P.cap, s)) != DSD_OK)
        goto done;
    P.xl = xl;
    if (P.hub_slots) {
        if ((st = dalloc(&hub_bm, (size_t)2 * P.hub_slots * P.hub_words, s)) != DSD_OK) goto done;
        if ((st = dalloc(&hubs, (size_t)2 * P.hub_slots, s)) != DSD_OK) goto done;
        e = cudaMemsetAsync(hub_bm, 0, (size_t)2 * P.hub_slots * P.hub_words * 4, s);
        if (e != cudaSuccess) {
            st = cuda_fail(e, "peel bitmaps", __FILE__, __LINE__);
            goto done;
        }
    }
    P.hub_bm = hub_bm;
    P.hubs = hubs;
    P.sl = sl;
    P.alive[0] = lists;
    P.alive[1] = lists + n;
    P.front[0] = lists + 2 * (size_t)n;
    P.front[1] = lists + 3 * (size_t)n;
    P.front[2] = lists + 4 * (size_t)n;
    P.jf = lists + 5 * (size_t)n;
    P.jblk = jblk;
    P.wend = wmeta;
    P.wnb = wmeta + n;
    P.wadj = wadj;
    P.big = big;
    P.ctrl = ctrl;
    e = cudaMemsetAsync(ctrl, 0, sizeof(PeelCtrl), s);
    if (e == cudaSuccess && nadj) e = cudaMemcpyAsync(wadj, adj, nadj * 4, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) {
        k_peel_init<<<sms * 4, 256, 0, s>>>(n, off, h >= 3 ? split : nullptr, sl, P.alive[0],
                                            P.wend, P.wnb, ctrl);
        note_launch();
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = launch_peel<NT>(P, sms, smem, s, &grid);
    if (e == cudaSuccess && P.tail_max) {
        // the launches run only if something was handed over (they read tail_n)
        TailParams T;
        memset(&T, 0, sizeof(T));
        T.h = h;
        T.off = off;
        T.wend = P.wend;
        T.wadj = P.wadj;
        T.sl = P.sl;
        T.deg = P.deg;
        T.list[0] = P.alive[0];
        T.list[1] = P.alive[1];
        T.core = P.core;
        T.rnd = P.rnd;
        T.lvl_k = P.lvl_k;
        T.lvl_size = P.lvl_size;
        T.lvl_mu = P.lvl_mu;
        T.ctrl = ctrl;
        if (tsh_g.cs) {
            T.cap = tsh_g.cap;
            T.rows_cap = tsh_g.cap / tsh_g.cs;
            T.W = tsh_g.cap / 32;
            T.pass_below = tsh_d.cap;
            T.rows_g = rows_g;
            e = launch_tail<true>(T, tsh_g, s);
        }
        if (e == cudaSuccess) {
            T.cap = tsh_d.cap;
            T.rows_cap = tsh_d.cap / tsh_d.cs;
            T.W = tsh_d.cap / 32;
            T.pass_below = 0;
            T.rows_g = nullptr;
            e = launch_tail<false>(T, tsh_d, s);
        }
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hc, ctrl, sizeof(PeelCtrl), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        st = cuda_fail(e, "peel", __FILE__, __LINE__);
        goto done;
    }
    if (hc.error & kErrTimeout) {
        set_error("a grid barrier wait in the peeling kernel exceeded %llu ms",
                  (unsigned long long)(P.wait_ns / 1000000ull));
        st = DSD_ERR_TIMEOUT;
        goto done;
    }
    if (hc.error) {
        set_error("peeling kernel internal error %u", hc.error);
        st = DSD_ERR_INTERNAL;
        goto done;
    }
    res->kmax = hc.kmax;
    res->nlevels = hc.nlevels;
    res->rounds = hc.rounds;
    res->items = hc.items;
    res->bytes = hc.bytes;
    res->barrier_ns = hc.barrier_ns;
    res->barriers = hc.barriers;
    res->compactions = hc.compactions;
    res->threads = NT;
    res->grid = grid;
    res->small_round = hc.small_round;
    res->tail_n = hc.tail_entry;
    res->tail_round = hc.tail_entry_round;
    res->tail_ns = hc.tail_ns;
    for (int i = 0; i < 7; i++) res->tail_tph[i] = hc.tail_tph[i];
    for (int i = 0; i < 8; i++) res->tph[i] = hc.tph[i];
done:
    dev_free(sl, s);
    dev_free(lists, s);
    dev_free(wmeta, s);
    dev_free(wadj, s);
    dev_free(ctrl, s);
    dev_free(rows_g, s);
    dev_free(big, s);
    dev_free(mid, s);
    dev_free(heavy, s);
    dev_free(xl, s);
    dev_free(hub_bm, s);
    dev_free(hubs, s);
    dev_free(jblk, s);
    return st;
}

}  // namespace dsd

extern "C" dsd_status dsd_check_barrier_timeout(int absent_block, uint32_t wait_ms,
                                                void* cuda_stream) {
    using namespace dsd;
    set_error("");
    cudaStream_t s = (cudaStream_t)cuda_stream;
    int sms = 152;
    DSD_TRY(num_sms(&sms));
    if (wait_ms == 0 || wait_ms > 60000 || absent_block >= sms) {
        set_error("dsd_check_barrier_timeout: need 0 < wait_ms <= 60000 and absent_block < %d",
                  sms);
        return DSD_ERR_INVALID;
    }
    PeelCtrl* ctrl = nullptr;
    DSD_TRY(dalloc(&ctrl, 1, s));
    PeelCtrl hc;
    memset(&hc, 0, sizeof(hc));
    uint64_t wait_ns = (uint64_t)wait_ms * 1000000ull;
    int absent = absent_block;
    void* args[] = {&ctrl, &wait_ns, &absent};
    cudaError_t e = cudaMemsetAsync(ctrl, 0, sizeof(PeelCtrl), s);
    if (e == cudaSuccess)
        e = cudaLaunchCooperativeKernel((void*)k_barrier_probe, dim3(sms), dim3(128), args, 0, s);
    note_launch();
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hc, ctrl, sizeof(hc), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    dev_free(ctrl, s);
    if (e != cudaSuccess) return cuda_fail(e, "barrier probe", __FILE__, __LINE__);
    if (hc.error & kErrTimeout) {
        set_error("grid barrier wait ran out after %u ms (block %d withheld)", wait_ms, absent);
        return DSD_ERR_TIMEOUT;
    }
    if (hc.error || hc.barriers != 4) {
        set_error("barrier probe: error %u, %u barriers", hc.error, hc.barriers);
        return DSD_ERR_INTERNAL;
    }
    return DSD_OK;
}
