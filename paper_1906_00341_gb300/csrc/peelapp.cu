// PeelApp (Algorithm 2, Sec. 3.2) on the GPU.
//
// Algorithm 2 removes one vertex of minimum current clique-degree at a time
// (ties: the smaller id) and keeps the densest of the sets it meets -- G and
// every residual -- a later set replacing the best only when strictly
// denser.  The order of its removals follows the (k,Psi)-core levels: while
// the current set S lies between R_{k+1} and R_k, every vertex of R_{k+1}
// has at least k+1 h-cliques in S, and S \ R_{k+1}, when not empty, holds a
// vertex with at most k (otherwise S would lie inside R_{k+1}, the largest
// set whose members all reach k+1).  So the minimum is always taken in
// S \ R_{k+1}: the peel passes through every R_k, and during level k it
// removes exactly L_k = R_k \ R_{k+1} = {v : core(v) = k}, starting from
// S = R_k with the counts deg_{R_k}.  Members of R_{k+1} do not leave during
// level k and their counts play no part in it.  After one decomposition that
// records deg_{R_k}(v) for every v in L_k (the count at v's level's first
// jump), the levels are independent processes.
//
// One block per level (the largest levels first).  Per step the block
//   - takes the alive member of L_k of least (count, caller id): from a
//     bucket queue when the level has one (below), else by a scan of the
//     level,
//   - compares the density of the current set with the level's best,
//   - removes it and lowers the count of every alive member of L_k that
//     shares an h-clique with it inside the current set.  The cliques through
//     v are listed from their smallest-rank other member w: C = N+(w) ∩ N(v)
//     ∩ S, then the (h-2)-cliques of G[C] with per-member credits, one warp
//     per w (one block for candidate sets above 32 vertices, h >= 4).
// Level 0 (vertices in no h-clique) is removed in id order with no change.
// A final pass takes, over the levels in order, the earliest set of
// greatest density and emits it in caller ids.
//
// Bucket queue of a level: for every count c < B (B <= k + 1), a bitmap over
// the level's positions with bit i set iff member i is alive with count c,
// two summary levels above it (bit t of a summary word: word t below may be
// non-empty), the population of every bucket and a bitmap of the buckets
// that may be non-empty.  The least (count, position) is the first set bit
// of the first non-empty bucket; with B = k + 1 that bucket always exists,
// since the minimum stays at or below k.  A count lowered from d to d - c
// toggles (XOR) its bit in buckets d and d - c: toggles commute, so the
// lowerings of one step may run in any order and the buckets are exact once
// they are all done; summaries are only ever set by the lowerings and are
// cleared lazily by the search.  Members of count 0 lie in no h-clique of
// the current set, so their removal changes no count: they leave one after
// another in position order without the clique listing.
#include "graph.cuh"
#include "xl.cuh"

#include <algorithm>
#include <string.h>
#include <vector>

namespace dsd {
namespace {

constexpr int kAppNT = 512;
constexpr uint32_t kAppWarpCand = 32;
constexpr uint32_t kNoStep = 0xffffffffu;

struct AppParams {
    uint32_t n;
    int h;
    const uint64_t* off;      // rank-space CSR: rows ascending, N+(x) from split[x]
    const uint32_t* adj;
    const uint64_t* split;
    const uint64_t* core;     // core numbers (rank space)
    const uint64_t* snap;     // count of v in R_core(v) (rank space)
    const uint32_t* posof;    // rank -> position (levels ascending, caller id inside)
    const uint32_t* rank_at;  // position -> rank
    unsigned long long* deg;  // by position: current count in the level's process
    uint32_t* step;           // by position: removal step inside its level (kNoStep alive)
    const uint64_t* lk;       // level records (k ascending, |R_k|, mu(R_k))
    const uint32_t* ls;
    const uint64_t* lm;
    uint32_t nl;
    const uint32_t* lorder;   // levels in processing order
    uint32_t* queue;          // [1] next entry of lorder
    ulonglong2* best;         // per level: (mu, size << 32 | step) of its best set
    uint32_t* bigw;           // per block: bigcap entries
    uint32_t bigcap;
    uint32_t cap;             // big candidate sets: >= max |N+|, >= 32
    uint32_t bcap;            // shared-memory candidate sets: min(cap, kBitmapMax)
    uint32_t* xl;             // per block (kMaxDepth + 1) * cap entries when cap > kBitmapMax
    uint32_t qwords;          // shared words of the bucket queue (after the scratch)
    uint32_t scratch_words;   // shared words of the warp and big-set scratch
    const uint32_t* qB;       // per level: buckets B (0 = no queue: the scan)
    const uint64_t* qoff;     // per level: word offset in qg, or kQShared
    uint32_t* qg;             // bucket queues of levels too large for shared memory
    uint32_t* err;            // [1] set when the queue and the counts disagree
};

constexpr uint64_t kQShared = ~0ull;
constexpr uint32_t kQMaxBuckets = 1024;   // the bucket bitmap is one warp's 32 words

__host__ __device__ inline uint32_t q_words_per_bucket(uint32_t sz) {
    uint32_t n1 = (sz + 31) / 32, n2 = (n1 + 31) / 32, n3 = (n2 + 31) / 32;
    return n1 + n2 + n3;
}
__host__ __device__ inline uint64_t q_words(uint32_t sz, uint32_t B) {
    return (uint64_t)B * q_words_per_bucket(sz) + B + 32;
}

// One level's bucket queue (a view; B = 0: none).
struct AppQ {
    uint32_t *M, *S, *T;      // bitmaps and summaries, bucket-major
    uint32_t *pop, *bsum;
    uint32_t B, n1, n2, n3, base;

    __device__ void toggle(unsigned long long d, uint32_t i) const {
        if (d >= B) return;
        const uint32_t c = (uint32_t)d, bit = 1u << (i & 31u);
        const uint32_t old = atomicXor(&M[(size_t)c * n1 + (i >> 5)], bit);
        if (old & bit) {
            atomicSub(&pop[c], 1u);
        } else {
            atomicAdd(&pop[c], 1u);
            atomicOr(&S[(size_t)c * n2 + (i >> 10)], 1u << ((i >> 5) & 31u));
            atomicOr(&T[(size_t)c * n3 + (i >> 15)], 1u << ((i >> 10) & 31u));
            atomicOr(&bsum[c >> 5], 1u << (c & 31u));
        }
    }
};

__device__ __forceinline__ bool ratio_gt(unsigned long long a, unsigned long long b,
                                         unsigned long long c, unsigned long long d) {
    // a/b > c/d for u64 a, c and u32-range b, d > 0: a*d > c*b in 128 bits
    unsigned long long lhi = __umul64hi(a, d), llo = a * d;
    unsigned long long rhi = __umul64hi(c, b), rlo = c * b;
    return lhi > rhi || (lhi == rhi && llo > rlo);
}

// x lies in the current set S of level k: above the level, or an alive
// member of it.
__device__ __forceinline__ bool in_set(const AppParams& P, uint32_t x, unsigned long long k) {
    unsigned long long c = P.core[x];
    return c > k || (c == k && P.step[P.posof[x]] == kNoStep);
}

__device__ __forceinline__ void lower(const AppParams& P, const AppQ& Q, uint32_t x,
                                      unsigned long long k, unsigned long long c) {
    if (c && P.core[x] == k) {
        uint32_t p = P.posof[x];
        if (P.step[p] == kNoStep) {
            unsigned long long old = atomicAdd(&P.deg[p], 0ull - c);
            if (Q.B) {
                Q.toggle(old, p - Q.base);
                Q.toggle(old - c, p - Q.base);
            }
        }
    }
}

// Candidates of v among N+(w) inside S, in order (one warp); returns how
// many there are.  DIRECT (h = 3): each candidate closes a triangle {v, w, x}
// and an alive level member loses it on the spot; else the first `keep` go
// to C, and with keep = kAppWarpCand the walk stops once there are more.
template <bool DIRECT>
__device__ __forceinline__ uint32_t app_gather(const AppParams& P, const AppQ& Q, uint32_t v,
                                               uint32_t w, unsigned long long k, uint32_t* C,
                                               uint32_t keep) {
    const unsigned lane = lane_id();
    const uint32_t* Nv = P.adj + P.off[v];
    const uint64_t dv = P.off[v + 1] - P.off[v];
    const uint64_t b = P.split[w], e = P.off[w + 1];
    uint32_t nc = 0;
    for (uint64_t p0 = b; p0 < e; p0 += 32) {
        uint64_t p = p0 + lane;
        bool ok = false;
        uint32_t x = 0;
        if (p < e) {
            x = P.adj[p];
            if (in_set(P, x, k)) {
                uint64_t pos = lower_bound_u32(Nv, dv, x);
                ok = pos < dv && Nv[pos] == x;
            }
        }
        unsigned bal = __ballot_sync(0xffffffffu, ok);
        if (DIRECT) {
            if (ok) lower(P, Q, x, k, 1ull);
        } else {
            uint32_t at = nc + __popc(bal & ((1u << lane) - 1u));
            if (ok && at < keep) C[at] = x;
        }
        nc += __popc(bal);
        if (!DIRECT && keep <= kAppWarpCand && nc > keep) return nc;   // needs the block
    }
    return nc;
}

// The cliques {v, w, ...} of S whose smallest-rank member other than v is
// w, counted by one warp when their candidate set fits kAppWarpCand; their
// alive level members lose them.  Returns false when the set is larger
// (h >= 4; the block takes it afterwards).
__device__ bool app_item(const AppParams& P, const AppQ& Q, uint32_t v, uint32_t w,
                         unsigned long long k, uint32_t* C, unsigned* cnt, uint32_t* rows) {
    const unsigned lane = lane_id();
    const int r = P.h - 2;
    if (r == 1) {
        uint32_t nc = app_gather<true>(P, Q, v, w, k, C, 0);
        if (lane == 0) lower(P, Q, w, k, nc);
        return true;
    }
    uint32_t nc = app_gather<false>(P, Q, v, w, k, C, kAppWarpCand);
    __syncwarp();
    if (nc < (uint32_t)r) return true;
    if (nc > kAppWarpCand) return false;
    unsigned long long tot = 0;
    {
        for (uint32_t i = lane; i < nc; i += 32) cnt[i] = 0;
        __syncwarp();
        if (r == 2) {
            const uint32_t cmax = C[nc - 1];
            for (uint32_t i = 0; i + 1 < nc; i++) {
                uint32_t x = C[i];
                unsigned hits = scan_row_hits(C, nc, cmax, P.adj, P.split[x], P.off[x + 1], cnt);
                hits = __reduce_add_sync(0xffffffffu, hits);
                if (lane == 0 && hits) atomicAdd(&cnt[i], hits);
                tot += hits;
            }
        } else {
            warp_build_rows32(C, nc, P.off + 1, P.adj, P.split, rows);
            tot = warp_dfs32(rows, nc, r, cnt);
        }
        __syncwarp();
        for (uint32_t i = lane; i < nc; i += 32) lower(P, Q, C[i], k, cnt[i]);
        __syncwarp();
    }
    if (lane == 0) lower(P, Q, w, k, tot);
    return true;
}

// A candidate set above kAppWarpCand vertices (h >= 4): the whole block,
// bitmap rows of G[C] and the block DFS.  When N+(w) holds more than
// kBitmapMax entries (degeneracy above 1024) the candidates are gathered in
// order into the block's global scratch, and a set that still exceeds
// kBitmapMax is split by its next member (xl.cuh), as in the peel.
__device__ void app_big(const AppParams& P, const AppQ& Q, uint32_t v, uint32_t w,
                        unsigned long long k, uint32_t* smem) {
    unsigned long long* cnt = reinterpret_cast<unsigned long long*>(smem);   // bcap
    uint32_t* C = smem + 2 * P.bcap;                                           // bcap
    uint32_t* rows = C + P.bcap;                                               // bcap * W
    __shared__ uint32_t s_nc, s_next, s_w[32], s_t2;
    __shared__ unsigned long long s_tot;
    const uint64_t wb = P.split[w], we = P.off[w + 1];
    if (we - wb > kBitmapMax) {
        uint32_t* G0 = P.xl + (size_t)blockIdx.x * (kMaxDepth + 1) * P.cap;
        const uint32_t* Nv = P.adj + P.off[v];
        const uint64_t dv = P.off[v + 1] - P.off[v];
        const uint32_t nc = block_filter(
            P.adj + wb, we - wb, G0,
            [&](uint32_t x) {
                if (!in_set(P, x, k)) return false;
                uint64_t pos = lower_bound_u32(Nv, dv, x);
                return pos < dv && Nv[pos] == x;
            },
            s_w, &s_t2);
        if (threadIdx.x == 0) s_tot = 0;
        __syncthreads();
        if (nc < (uint32_t)(P.h - 2)) return;
        if (nc > kBitmapMax) {
            xl_cliques(
                G0, nc, P.h - 2, P.split, P.off + 1, P.adj, G0 + P.cap, P.cap, smem,
                [&](uint32_t x, unsigned long long c) { lower(P, Q, x, k, c); },
                [&](unsigned long long c) { s_tot += c; });
            __syncthreads();
            if (threadIdx.x == 0) lower(P, Q, w, k, s_tot);
            __syncthreads();
            return;
        }
        for (uint32_t i = threadIdx.x; i < nc; i += blockDim.x) C[i] = G0[i];
        if (threadIdx.x == 0) {
            s_nc = nc;
            s_next = 0;
        }
        __syncthreads();
    } else {
        if (warp_id() == 0) {
            uint32_t nc = app_gather<false>(P, Q, v, w, k, C, P.bcap);
            if (lane_id() == 0) {
                s_nc = nc;
                s_next = 0;
                s_tot = 0;
            }
        }
        __syncthreads();
    }
    const uint32_t nc = s_nc, W = (nc + 31) >> 5;
    for (uint32_t i = threadIdx.x; i < nc; i += blockDim.x) cnt[i] = 0;
    for (uint32_t i = threadIdx.x; i < nc * W; i += blockDim.x) rows[i] = 0;
    __syncthreads();
    block_build_rows(C, nc, W, P.off + 1, P.adj, P.split, rows);
    __syncthreads();
    unsigned long long mine = block_dfs(rows, nc, W, P.h - 2, cnt, &s_next);
    if (mine) atomicAdd(&s_tot, mine);
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < nc; i += blockDim.x) lower(P, Q, C[i], k, cnt[i]);
    if (threadIdx.x == 0) lower(P, Q, w, k, s_tot);
    __syncthreads();
}

// Warp search of a level's queue (one warp, nothing else touching the
// queue): the least bucket with members, B if none; stale bucket bits are
// cleared on the way.  Values read by lane 0 are broadcast, so every lane
// takes the same branch.
__device__ __forceinline__ uint32_t q_least_bucket(const AppQ& Q) {
    const unsigned lane = lane_id();
    volatile uint32_t* bs = Q.bsum;
    volatile uint32_t* pop = Q.pop;
    const uint32_t nbw = (Q.B + 31) / 32;
    for (;;) {
        uint32_t w = lane < nbw ? bs[lane] : 0u;
        const unsigned bal = __ballot_sync(0xffffffffu, w != 0);
        if (!bal) return Q.B;
        const uint32_t t = __ffs(bal) - 1;
        w = __shfl_sync(0xffffffffu, w, t);
        const uint32_t b = t * 32 + __ffs(w) - 1;
        uint32_t pb = lane == 0 ? pop[b] : 0u;
        pb = __shfl_sync(0xffffffffu, pb, 0);
        if (pb) return b;
        if (lane == 0) bs[t] = w & ~(1u << (b & 31u));
        __syncwarp();
    }
}

// The first position in bucket b (~0u if the summaries lead to none); stale
// summary bits are cleared on the way.
__device__ __forceinline__ uint32_t q_first(const AppQ& Q, uint32_t b) {
    const unsigned lane = lane_id();
    volatile uint32_t* T = Q.T + (size_t)b * Q.n3;
    volatile uint32_t* S = Q.S + (size_t)b * Q.n2;
    volatile uint32_t* M = Q.M + (size_t)b * Q.n1;
    for (;;) {
        uint32_t tw = lane < Q.n3 ? T[lane] : 0u;
        const unsigned bal = __ballot_sync(0xffffffffu, tw != 0);
        if (!bal) return ~0u;
        const uint32_t t = __ffs(bal) - 1;
        tw = __shfl_sync(0xffffffffu, tw, t);
        const uint32_t si = t * 32 + __ffs(tw) - 1;
        uint32_t sw = lane == 0 ? S[si] : 0u;
        sw = __shfl_sync(0xffffffffu, sw, 0);
        if (!sw) {
            if (lane == 0) T[t] = tw & ~(1u << (si & 31u));
            __syncwarp();
            continue;
        }
        const uint32_t mi = si * 32 + __ffs(sw) - 1;
        uint32_t mw = lane == 0 ? M[mi] : 0u;
        mw = __shfl_sync(0xffffffffu, mw, 0);
        if (!mw) {
            if (lane == 0) S[si] = sw & ~(1u << (mi & 31u));
            __syncwarp();
            continue;
        }
        return mi * 32 + __ffs(mw) - 1;
    }
}

constexpr uint32_t kPickScan = 0xffffffffu;   // no queue pick: scan the level
constexpr uint32_t kPickDone = 0xfffffffeu;   // every member removed

template <int NT>
__global__ void __launch_bounds__(NT) k_peel_app(AppParams P) {
    constexpr int NW = NT / 32;
    extern __shared__ uint32_t smem[];
    __shared__ unsigned long long s_kd[NW];
    __shared__ uint32_t s_kp[NW];
    __shared__ uint32_t s_lv, s_pick, s_nbig, s_it;
    const unsigned lane = lane_id(), wid = warp_id();
    uint32_t* wC = smem + (size_t)wid * 3 * kAppWarpCand;
    unsigned* wCnt = wC + kAppWarpCand;
    uint32_t* wRows = wC + 2 * kAppWarpCand;
    uint32_t* bigw = P.bigw + (size_t)blockIdx.x * P.bigcap;
    for (;;) {
        if (threadIdx.x == 0) {
            uint32_t q = atomicAdd(P.queue, 1u);
            s_lv = q < P.nl ? P.lorder[q] : 0xffffffffu;
        }
        __syncthreads();
        const uint32_t j = s_lv;
        __syncthreads();
        if (j == 0xffffffffu) break;
        const unsigned long long k = P.lk[j];
        const uint32_t size0 = P.ls[j];
        const uint32_t next = j + 1 < P.nl ? P.ls[j + 1] : 0u;
        const uint32_t base = P.n - size0, sz = size0 - next;
        unsigned long long mu = P.lm[j];
        if (k == 0) {
            // no cliques here: removal in id order, no count changes; the
            // density only grows as the set shrinks
            for (uint32_t i = threadIdx.x; i < sz; i += NT) P.step[base + i] = i;
            if (threadIdx.x == 0) {
                uint32_t bs = mu ? sz - 1 : 0;
                P.best[j] = make_ulonglong2(mu, ((unsigned long long)(size0 - bs) << 32) | bs);
            }
            continue;
        }
        // the level's bucket queue, if it has one
        AppQ Q;
        Q.B = P.qB[j];
        Q.n1 = (sz + 31) / 32;
        Q.n2 = (Q.n1 + 31) / 32;
        Q.n3 = (Q.n2 + 31) / 32;
        Q.base = base;
        Q.M = Q.S = Q.T = Q.pop = Q.bsum = nullptr;
        if (Q.B) {
            uint32_t* R = P.qoff[j] == kQShared ? smem + P.scratch_words : P.qg + P.qoff[j];
            Q.M = R;
            Q.S = Q.M + (size_t)Q.B * Q.n1;
            Q.T = Q.S + (size_t)Q.B * Q.n2;
            Q.pop = Q.T + (size_t)Q.B * Q.n3;
            Q.bsum = Q.pop + Q.B;
            const uint64_t nw = q_words(sz, Q.B);
            for (uint64_t i = threadIdx.x; i < nw; i += NT) R[i] = 0;
            __syncthreads();
        }
        for (uint32_t i = threadIdx.x; i < sz; i += NT) {
            const unsigned long long d = P.snap[P.rank_at[base + i]];
            P.deg[base + i] = d;
            P.step[base + i] = kNoStep;
            Q.toggle(d, i);
        }
        unsigned long long bmu = mu;
        uint32_t bsize = size0, bstep = 0, it = 0;   // thread 0's (it: warp 0's)
        __syncthreads();
        for (;;) {
            // ---- the next removal: the queue's least (count, position), the
            // members of count 0 leaving at once; or a scan of the level
            if (wid == 0) {
                uint32_t pick = kPickScan;
                while (Q.B) {
                    const uint32_t b = q_least_bucket(Q);
                    if (b == Q.B) break;   // only counts >= B left (B < k + 1)
                    const uint32_t i = q_first(Q, b);
                    if (i == ~0u) {
                        if (lane == 0) atomicOr(P.err, 1u);
                        pick = kPickDone;
                        break;
                    }
                    if (lane == 0) {
                        Q.M[(size_t)b * Q.n1 + (i >> 5)] &= ~(1u << (i & 31u));
                        Q.pop[b] -= 1u;
                        if (P.deg[base + i] != b) atomicOr(P.err, 2u);
                        // the set before this removal: size0 - it vertices, mu cliques
                        if (it > 0 && ratio_gt(mu, size0 - it, bmu, bsize)) {
                            bmu = mu;
                            bsize = size0 - it;
                            bstep = it;
                        }
                        mu -= b;
                        P.step[base + i] = it;
                    }
                    it++;
                    __syncwarp();
                    if (b != 0) {
                        pick = i;
                        break;
                    }
                    if (it == sz) {
                        pick = kPickDone;
                        break;
                    }
                }
                if (lane == 0) {
                    s_pick = pick;
                    s_it = it;
                    s_nbig = 0;
                }
            }
            __syncthreads();
            uint32_t pick = s_pick;
            if (pick == kPickDone) break;
            if (pick == kPickScan) {
                // least (count, position); positions ascend with the caller id
                unsigned long long md = ~0ull;
                uint32_t mp = 0xffffffffu;
                for (uint32_t i = threadIdx.x; i < sz; i += NT) {
                    if (P.step[base + i] != kNoStep) continue;
                    unsigned long long d = P.deg[base + i];
                    if (d < md) { md = d; mp = i; }   // i ascends: ties keep the first
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    unsigned long long od = __shfl_xor_sync(0xffffffffu, md, o);
                    uint32_t op = __shfl_xor_sync(0xffffffffu, mp, o);
                    if (od < md || (od == md && op < mp)) { md = od; mp = op; }
                }
                if (lane == 0) { s_kd[wid] = md; s_kp[wid] = mp; }
                __syncthreads();
                if (threadIdx.x == 0) {
                    unsigned long long bd = s_kd[0];
                    uint32_t bp = s_kp[0];
                    for (int w2 = 1; w2 < NW; w2++)
                        if (s_kd[w2] < bd || (s_kd[w2] == bd && s_kp[w2] < bp)) {
                            bd = s_kd[w2];
                            bp = s_kp[w2];
                        }
                    if (bd < Q.B) atomicOr(P.err, 4u);   // the queue holds every count < B
                    if (it > 0 && ratio_gt(mu, size0 - it, bmu, bsize)) {
                        bmu = mu;
                        bsize = size0 - it;
                        bstep = it;
                    }
                    mu -= bd;
                    P.step[base + bp] = it;
                    s_pick = bp;
                    s_it = it + 1;
                }
                if (wid == 0) it++;
                __syncthreads();
                pick = s_pick;
            }
            // ---- the cliques through the removed vertex lower its partners
            const uint32_t v = P.rank_at[base + pick];
            const uint64_t vb = P.off[v], ve = P.off[v + 1];
            if (P.h == 2) {
                for (uint64_t p = vb + threadIdx.x; p < ve; p += NT)
                    lower(P, Q, P.adj[p], k, 1ull);
            } else {
                for (uint64_t p = vb + wid; p < ve; p += NW) {
                    uint32_t w = P.adj[p];
                    if (!in_set(P, w, k)) continue;
                    if (!app_item(P, Q, v, w, k, wC, wCnt, wRows) && lane == 0) {
                        uint32_t at = atomicAdd(&s_nbig, 1u);
                        if (at < P.bigcap) bigw[at] = w;
                    }
                }
                __syncthreads();
                const uint32_t nb = s_nbig;
                for (uint32_t b = 0; b < nb && b < P.bigcap; b++)
                    app_big(P, Q, v, bigw[b], k, smem);
            }
            __syncthreads();
            if (s_it >= sz) break;
        }
        if (threadIdx.x == 0)
            P.best[j] = make_ulonglong2(bmu, ((unsigned long long)bsize << 32) | bstep);
        __syncthreads();
    }
}

// Level of each vertex (binary search of its core number in the records),
// counted per level.
__global__ void k_app_levels(uint32_t n, const uint64_t* core, const uint64_t* lk, uint32_t nl,
                             uint32_t* lev) {
    for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t c = core[v];
        uint32_t lo = 0, hi = nl;   // first j with lk[j] >= c
        while (lo < hi) {
            uint32_t mid = (lo + hi) >> 1;
            if (lk[mid] < c) lo = mid + 1; else hi = mid;
        }
        lev[v] = lo;
    }
}

// Scatter caller ids into their level's segment (any order inside).
__global__ void k_app_place(uint32_t n, const uint32_t* lev, const uint32_t* ls, uint32_t nl,
                            const uint32_t* old_of, uint32_t* cursor, uint32_t* ids) {
    for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t j = lev[v];
        uint32_t at = atomicAdd(&cursor[j], 1u);
        ids[n - ls[j] + at] = old_of[v];
    }
}

__global__ void k_app_maps(uint32_t n, const uint32_t* ids, const uint32_t* new_of,
                           uint32_t* rank_at, uint32_t* posof) {
    for (uint64_t p = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n;
         p += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t r = new_of[ids[p]];
        rank_at[p] = r;
        posof[r] = (uint32_t)p;
    }
}

// The earliest set of greatest density over the levels in order (one thread).
__global__ void k_app_pick(uint32_t nl, const ulonglong2* best, ulonglong2* out) {
    if (blockIdx.x || threadIdx.x) return;
    unsigned long long bm = 0, bsz = 0;
    uint32_t bj = 0, bstep = 0;
    for (uint32_t j = 0; j < nl; j++) {
        unsigned long long m = best[j].x, sz = best[j].y >> 32;
        if (j == 0 || ratio_gt(m, sz, bm, bsz)) {
            bm = m;
            bsz = sz;
            bj = j;
            bstep = (uint32_t)(best[j].y & 0xffffffffull);
        }
    }
    *out = make_ulonglong2(bm, (bsz << 32) | bj);
    out[1] = make_ulonglong2(bstep, 0);
}

// flag[o] (caller id o) = 1 if o is in the chosen set: above its level, or in
// it and removed at step >= the chosen one.  order[start_j + step] = o.
__global__ void k_app_emit(uint32_t n, const uint32_t* ids, const uint32_t* rank_at,
                           const uint64_t* core, const uint32_t* step, const uint32_t* lev,
                           const uint32_t* ls, const ulonglong2* pick, const uint64_t* lk,
                           uint32_t* flag, uint32_t* order) {
    const uint32_t bj = (uint32_t)(pick[0].y & 0xffffffffull);
    const uint32_t bstep = (uint32_t)pick[1].x;
    const unsigned long long kb = lk[bj];
    for (uint64_t p = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n;
         p += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t r = rank_at[p], o = ids[p];
        const unsigned long long c = core[r];
        flag[o] = (c > kb || (c == kb && step[p] >= bstep)) ? 1u : 0u;
        if (order) order[n - ls[lev[r]] + step[p]] = o;
    }
}

__global__ void k_app_compact(uint32_t n, const uint32_t* flag, const uint64_t* pos,
                              uint32_t* out) {
    for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (uint64_t)gridDim.x * blockDim.x)
        if (flag[v]) out[pos[v]] = (uint32_t)v;
}

__global__ void k_app_maxdeg(uint32_t n, const uint64_t* off, unsigned long long* out) {
    unsigned long long m = 0;
    for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (uint64_t)gridDim.x * blockDim.x) {
        unsigned long long d = off[v + 1] - off[v];
        m = d > m ? d : m;
    }
    for (int o = 16; o > 0; o >>= 1) {
        unsigned long long t = __shfl_xor_sync(0xffffffffu, m, o);
        m = t > m ? t : m;
    }
    if ((threadIdx.x & 31) == 0 && m) atomicMax(out, m);
}

unsigned app_grid(uint64_t n) {
    uint64_t b = (n + 255) / 256;
    return (unsigned)(b < 1 ? 1 : (b > 152 * 16 ? 152 * 16 : b));
}

}  // namespace
}  // namespace dsd

using namespace dsd;

extern "C" dsd_status dsd_peel_app(dsd_graph* g, int h, uint32_t* densest, uint32_t* order,
                                   int mem, dsd_peel_app_result* res) {
    set_error("");
    if (!g || !res || h < 2 || h > DSD_MAX_H || (mem != DSD_MEM_HOST && mem != DSD_MEM_DEVICE)) {
        set_error("invalid argument to dsd_peel_app");
        return DSD_ERR_INVALID;
    }
    memset(res, 0, sizeof(*res));
    DSD_TRY(ensure_order(g));
    const uint32_t n = g->n;
    if (n == 0) return DSD_OK;
    cudaStream_t s = g->stream;
    int sms = 152;
    DSD_TRY(num_sms(&sms));
    // ---- one decomposition with the level-start counts
    unsigned long long* deg = nullptr;
    uint64_t *core = nullptr, *snap = nullptr, *lk = nullptr, *lm = nullptr, *pos = nullptr;
    uint32_t *ls = nullptr, *lev = nullptr, *cur = nullptr, *ids = nullptr, *tmp = nullptr;
    uint32_t *lenv = nullptr, *newlen = nullptr, *rank_at = nullptr, *posof = nullptr;
    uint32_t *stepv = nullptr, *lorder = nullptr, *bigw = nullptr, *flag = nullptr;
    uint32_t* obuf = nullptr;
    uint64_t* lpos = nullptr;
    ulonglong2 *best = nullptr, *pick = nullptr;
    unsigned long long* pdeg = nullptr;
    unsigned long long mu = 0;
    dsd_status st = DSD_OK;
    cudaError_t e = cudaSuccess;
    PeelResult pr;
    uint32_t nl = 0;
    std::vector<uint32_t> hls, hqB;
    std::vector<uint64_t> hk, hqoff;
    uint32_t *qBv = nullptr, *qg = nullptr, *xl = nullptr;
    uint64_t* qoffv = nullptr;
    uint32_t herr = 0;
#define APP_TRY(x)                                \
    do {                                          \
        st = (x);                                 \
        if (st != DSD_OK) goto done;              \
    } while (0)
#define APP_CU(x)                                                                    \
    do {                                                                             \
        e = (x);                                                                     \
        if (e != cudaSuccess) { st = cuda_fail(e, #x, __FILE__, __LINE__); goto done; } \
    } while (0)
    APP_TRY(dalloc(&deg, (size_t)n + 2, s));
    APP_TRY(dalloc(&core, (size_t)n + 1, s));
    APP_TRY(dalloc(&snap, (size_t)n + 1, s));
    APP_TRY(dalloc(&lk, (size_t)n + 1, s));
    APP_TRY(dalloc(&ls, (size_t)n + 1, s));
    APP_TRY(dalloc(&lm, (size_t)n + 1, s));
    APP_TRY(count_cliques(g, h, deg, deg + n + 1));
    APP_CU(cudaMemcpyAsync(&mu, deg + n + 1, 8, cudaMemcpyDeviceToHost, s));
    APP_CU(cudaStreamSynchronize(s));
    APP_TRY(run_peel(g, h, n, g->roff, g->radj, g->rsplit, g->maxdplus, deg, mu, core, nullptr,
                     lk, ls, lm, &pr, 0, snap));
    nl = pr.nlevels;
    if (nl == 0) {
        set_error("PeelApp: the decomposition recorded no level");
        st = DSD_ERR_INTERNAL;
        goto done;
    }
    // ---- positions: levels ascending, caller ids ascending inside a level
    APP_TRY(dalloc(&lev, (size_t)n + 1, s));
    APP_TRY(dalloc(&cur, (size_t)nl + 1, s));
    APP_TRY(dalloc(&ids, (size_t)n + 1, s));
    APP_TRY(dalloc(&tmp, (size_t)n + 1, s));
    APP_TRY(dalloc(&lenv, (size_t)nl + 1, s));
    APP_TRY(dalloc(&newlen, (size_t)nl + 1, s));
    APP_TRY(dalloc(&lpos, (size_t)nl + 1, s));
    APP_TRY(dalloc(&rank_at, (size_t)n + 1, s));
    APP_TRY(dalloc(&posof, (size_t)n + 1, s));
    APP_CU(cudaMemsetAsync(cur, 0, (size_t)nl * 4, s));
    k_app_levels<<<app_grid(n), 256, 0, s>>>(n, core, lk, nl, lev); note_launch();
    k_app_place<<<app_grid(n), 256, 0, s>>>(n, lev, ls, nl, g->old_of, cur, ids); note_launch();
    APP_CU(cudaGetLastError());
    hls.resize(nl);
    hk.resize(nl);
    APP_CU(cudaMemcpyAsync(hls.data(), ls, (size_t)nl * 4, cudaMemcpyDeviceToHost, s));
    APP_CU(cudaMemcpyAsync(hk.data(), lk, (size_t)nl * 8, cudaMemcpyDeviceToHost, s));
    APP_CU(cudaStreamSynchronize(s));
    {
        std::vector<uint32_t> len(nl), order(nl);
        std::vector<uint64_t> start(nl);
        for (uint32_t j = 0; j < nl; j++) {
            start[j] = n - hls[j];
            len[j] = hls[j] - (j + 1 < nl ? hls[j + 1] : 0u);
            order[j] = j;
        }
        std::stable_sort(order.begin(), order.end(),
                         [&](uint32_t a, uint32_t b) { return len[a] > len[b]; });
        APP_TRY(dalloc(&lorder, (size_t)nl + 1, s));
        APP_CU(cudaMemcpyAsync(lenv, len.data(), (size_t)nl * 4, cudaMemcpyHostToDevice, s));
        APP_CU(cudaMemcpyAsync(lpos, start.data(), (size_t)nl * 8, cudaMemcpyHostToDevice, s));
        APP_CU(cudaMemcpyAsync(lorder, order.data(), (size_t)nl * 4, cudaMemcpyHostToDevice, s));
        APP_TRY(segmented_sort_unique(ids, tmp, lpos, lenv, newlen, nl, n, s));
        APP_CU(cudaStreamSynchronize(s));   // host vectors leave scope
    }
    k_app_maps<<<app_grid(n), 256, 0, s>>>(n, ids, g->new_of, rank_at, posof); note_launch();
    APP_CU(cudaGetLastError());
    // ---- the per-level processes
    {
        AppParams P;
        memset(&P, 0, sizeof(P));
        P.n = n;
        P.h = h;
        P.off = g->roff;
        P.adj = g->radj;
        P.split = g->rsplit;
        P.core = core;
        P.snap = snap;
        P.posof = posof;
        P.rank_at = rank_at;
        P.lk = lk;
        P.ls = ls;
        P.lm = lm;
        P.nl = nl;
        P.cap = g->maxdplus < 32 ? 32 : g->maxdplus;
        P.bcap = P.cap < kBitmapMax ? P.cap : kBitmapMax;
        // the counts, steps and queue reuse buffers of the decomposition
        APP_TRY(dalloc(&pdeg, (size_t)n + 1, s));
        APP_TRY(dalloc(&stepv, (size_t)n + 2, s));
        APP_TRY(dalloc(&best, (size_t)nl + 1, s));
        APP_TRY(dalloc(&pick, 2, s));
        P.deg = pdeg;
        P.step = stepv;
        P.queue = stepv + n;
        P.lorder = lorder;
        P.best = best;
        size_t words = (size_t)(kAppNT / 32) * 3 * kAppWarpCand;
        if (h >= 4) {
            size_t W = (P.bcap + 31) / 32;
            size_t big = (size_t)3 * P.bcap + (size_t)P.bcap * W;
            // the split search of oversized sets uses the full bitmap tier layout
            if (P.cap > kBitmapMax) big = (size_t)3 * kBitmapMax + (size_t)kBitmapMax * 32;
            if (big > words) words = big;
        }
        // bucket queues: in shared memory after the scratch where they fit
        // (every count 0..k), else in global memory within a budget, else
        // the buckets that fit shared memory with the scan behind them
        const size_t qsh = std::min<size_t>(peel_app_queue_shared(),
                                            220 * 1024 / 4 > words ? 220 * 1024 / 4 - words : 0);
        P.scratch_words = (uint32_t)words;
        P.qwords = (uint32_t)qsh;
        hqB.assign(nl, 0u);
        hqoff.assign(nl, kQShared);
        uint64_t gwords = 0;
        const uint64_t gbudget = peel_app_queue_global();   // words (default 2^26: 256 MB)
        for (uint32_t j = 0; j < nl; j++) {
            const uint32_t sz = hls[j] - (j + 1 < nl ? hls[j + 1] : 0u);
            if (hk[j] == 0 || sz == 0 || sz > (1u << 20)) continue;   // the warp search: <= 32^4
            const uint32_t bf = hk[j] + 1 < kQMaxBuckets ? (uint32_t)hk[j] + 1 : kQMaxBuckets;
            const uint64_t need = q_words(sz, bf);
            if (need <= qsh) {
                hqB[j] = bf;
            } else if (gwords + need <= gbudget) {
                hqB[j] = bf;
                hqoff[j] = gwords;
                gwords += need;
            } else {
                const uint64_t wpb = q_words_per_bucket(sz) + 1;
                const uint64_t b = qsh > 32 ? (qsh - 32) / wpb : 0;
                hqB[j] = (uint32_t)(b < bf ? b : bf);
            }
        }
        APP_TRY(dalloc(&qBv, (size_t)nl, s));
        APP_TRY(dalloc(&qoffv, (size_t)nl, s));
        APP_TRY(dalloc(&qg, (size_t)gwords + 1, s));
        APP_CU(cudaMemcpyAsync(qBv, hqB.data(), (size_t)nl * 4, cudaMemcpyHostToDevice, s));
        APP_CU(cudaMemcpyAsync(qoffv, hqoff.data(), (size_t)nl * 8, cudaMemcpyHostToDevice, s));
        P.qB = qBv;
        P.qoff = qoffv;
        P.qg = qg;
        P.err = stepv + n + 1;
        size_t smem = (words + qsh) * 4;
        const void* fn = (const void*)k_peel_app<kAppNT>;
        // opt in for every launch: the 48 KB default bounds static + dynamic
        // shared memory together
        APP_CU(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        int per = 0;
        APP_CU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_peel_app<kAppNT>, kAppNT,
                                                             smem));
        if (per < 1) {
            set_error("PeelApp kernel does not fit on this device");
            st = DSD_ERR_UNSUPPORTED;
            goto done;
        }
        unsigned grid = (unsigned)(sms * per);
        if (h >= 4 && P.cap > kBitmapMax) {
            APP_TRY(dalloc(&xl, (size_t)grid * (kMaxDepth + 1) * P.cap, s));
            P.xl = xl;
        }
        // a removal lists at most deg(v) big candidate sets: the per-block
        // list holds the largest row
        unsigned long long maxrow = 0;
        if (h >= 4) {
            APP_CU(cudaMemsetAsync(best, 0, 8, s));
            k_app_maxdeg<<<app_grid(n), 256, 0, s>>>(n, g->roff, (unsigned long long*)best);
            note_launch();
            APP_CU(cudaMemcpyAsync(&maxrow, best, 8, cudaMemcpyDeviceToHost, s));
            APP_CU(cudaStreamSynchronize(s));
        }
        P.bigcap = (uint32_t)(maxrow + 1);
        APP_TRY(dalloc(&bigw, (size_t)grid * P.bigcap + 1, s));
        P.bigw = bigw;
        APP_CU(cudaMemsetAsync(P.queue, 0, 8, s));   // the level queue and the error word
        k_peel_app<kAppNT><<<grid, kAppNT, smem, s>>>(P); note_launch();
        APP_CU(cudaGetLastError());
        APP_CU(cudaMemcpyAsync(&herr, P.err, 4, cudaMemcpyDeviceToHost, s));
        APP_CU(cudaStreamSynchronize(s));   // the host plans above leave scope
        if (herr) {
            set_error("PeelApp: a level's bucket queue disagreed with its counts (%u)", herr);
            st = DSD_ERR_INTERNAL;
            goto done;
        }
        k_app_pick<<<1, 32, 0, s>>>(nl, best, pick); note_launch();
        APP_CU(cudaGetLastError());
    }
    // ---- the chosen set, in caller ids, ascending
    {
        APP_TRY(dalloc(&flag, (size_t)n + 1, s));
        APP_TRY(dalloc(&pos, (size_t)n + 1, s));
        if (order) APP_TRY(dalloc(&obuf, (size_t)n + 1, s));
        k_app_emit<<<app_grid(n), 256, 0, s>>>(n, ids, rank_at, core, stepv, lev, ls, pick, lk,
                                               flag, obuf); note_launch();
        APP_TRY(exclusive_scan_u32_to_u64(flag, pos, n, s));
        ulonglong2 hp[2];
        APP_CU(cudaMemcpyAsync(hp, pick, sizeof(hp), cudaMemcpyDeviceToHost, s));
        APP_CU(cudaStreamSynchronize(s));
        res->mu = hp[0].x;
        res->size = (uint32_t)(hp[0].y >> 32);
        res->removed = n - res->size;
        res->level_k = 0;
        {
            uint64_t kb = 0;
            APP_CU(cudaMemcpyAsync(&kb, lk + (uint32_t)(hp[0].y & 0xffffffffull), 8,
                                   cudaMemcpyDeviceToHost, s));
            APP_CU(cudaStreamSynchronize(s));
            res->level_k = kb;
        }
        const cudaMemcpyKind kind =
            mem == DSD_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
        if (densest) {
            uint32_t* dbuf = nullptr;
            APP_TRY(dalloc(&dbuf, (size_t)res->size + 1, s));
            k_app_compact<<<app_grid(n), 256, 0, s>>>(n, flag, pos, dbuf); note_launch();
            e = cudaGetLastError();
            if (e == cudaSuccess && res->size)
                e = cudaMemcpyAsync(densest, dbuf, (size_t)res->size * 4, kind, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            dev_free(dbuf, s);
            if (e != cudaSuccess) {
                st = cuda_fail(e, "PeelApp set", __FILE__, __LINE__);
                goto done;
            }
        }
        if (order) {
            APP_CU(cudaMemcpyAsync(order, obuf, (size_t)n * 4, kind, s));
            APP_CU(cudaStreamSynchronize(s));
        }
    }
#undef APP_TRY
#undef APP_CU
done:
    for (void* p : {(void*)deg, (void*)core, (void*)snap, (void*)lk, (void*)ls, (void*)lm,
                    (void*)lev, (void*)cur, (void*)ids, (void*)tmp, (void*)lenv, (void*)newlen,
                    (void*)lpos, (void*)rank_at, (void*)posof, (void*)pdeg, (void*)stepv,
                    (void*)best, (void*)pick, (void*)lorder, (void*)bigw, (void*)flag,
                    (void*)pos, (void*)obuf, (void*)qBv, (void*)qoffv, (void*)qg, (void*)xl})
        dev_free(p, s);
    return st;
}
