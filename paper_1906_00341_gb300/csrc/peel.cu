// K5/K6: level-synchronous (k,Psi)-core peeling with level statistics.
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
// One persistent cooperative kernel runs every round; the phases of a round
// are separated by grid barriers whose waits are bounded in time (a wait that
// runs out records DSD_ERR_TIMEOUT and every block leaves).
//
// Round r (F_r = frontier of round r, lists indexed r mod 3):
//   P1  mark F_{r-1} removed (core = k); mark F_r as frontier     | barrier
//   J   (only if F_r is empty) compact the alive list and take   |
//       the minimum count; k = that minimum; record the level    | barrier
//       (k, |R_k|, mu(R_k)); F_r = alive vertices with count <= k | barrier
//   P2  enumerate the cliques each v in F_r destroys; decrement   | barrier
//   P2b (h >= 5) candidate sets above 32 vertices, one block each | barrier
#include "cliques.cuh"
#include "graph.cuh"

namespace dsd {
namespace {

enum : uint8_t { kAlive = 0, kFront = 1, kGone = 2 };
enum : uint32_t { kErrTimeout = 1, kErrBigOverflow = 2 };
constexpr int kPeelThreads = 256;
constexpr int kPeelWarps = kPeelThreads / 32;
constexpr uint32_t kSmallFront = 1024;

struct PeelCtrl {
    unsigned long long min_deg[2];
    uint32_t new_alive[2];
    uint32_t fcnt[3];
    uint32_t big_cnt[3];
    unsigned long long destroyed[3];
    uint32_t pad0[16];
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
    unsigned long long bytes;   // algorithmic bytes (see meter notes below)
};

// Byte meter.  Every global-memory element the algorithm reads or writes is
// counted once per access: ids 4 B, offsets 8 B, state 1 B, counters 8 B, an
// atomic read-modify-write 16 B, a binary search over a row of d entries
// floor(log2 d) + 1 probes of 4 B.  Shared-memory traffic is not counted.
__device__ __forceinline__ unsigned probes(uint64_t d) {
    return d ? 64u - (unsigned)__clzll((long long)d) : 0u;
}

struct PeelParams {
    uint32_t n;
    int h;
    const uint64_t* off;
    const uint32_t* adj;
    const uint64_t* split;
    unsigned long long* deg;
    uint64_t* core;
    uint32_t* rnd;
    uint8_t* state;
    uint32_t* alive[2];
    uint32_t* front[3];
    uint2* big;
    uint64_t big_cap;
    uint64_t* lvl_k;
    uint32_t* lvl_size;
    uint64_t* lvl_mu;
    PeelCtrl* ctrl;
    uint64_t wait_ns;
    unsigned long long mu0;
    uint32_t cap;        // per-warp candidate buffer entries (>= max |N+|, >= 32)
};

// ------------------------------------------------------------ barrier
__device__ bool grid_barrier(PeelCtrl* c, uint64_t wait_ns) {
    __shared__ uint32_t s_err;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile uint32_t* genp = &c->bar_gen;
        uint32_t gen = *genp;
        __threadfence();
        uint32_t arrived = atomicAdd(&c->bar_count, 1u) + 1u;
        if (arrived == gridDim.x) {
            c->bar_count = 0;
            __threadfence();
            atomicAdd(&c->bar_gen, 1u);
        } else {
            uint64_t t0 = globaltimer_ns();
            uint32_t spins = 0;
            while (*genp == gen) {
                if (((++spins) & 255u) == 0 && globaltimer_ns() - t0 > wait_ns) {
                    atomicOr(&c->error, kErrTimeout);
                    break;
                }
                if (*(volatile uint32_t*)&c->error) break;
            }
        }
        __threadfence();
        s_err = *(volatile uint32_t*)&c->error;
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

__device__ __forceinline__ bool candidate(const PeelParams& P, uint32_t x, uint32_t v) {
    uint8_t s = P.state[x];
    return s == kAlive || (s == kFront && x > v);
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
__device__ __forceinline__ unsigned long long block_sum(unsigned long long v,
                                                       unsigned long long* red) {
    v = warp_sum(v);
    if (lane_id() == 0) red[warp_id()] = v;
    __syncthreads();
    unsigned long long t = 0;
    if (threadIdx.x == 0)
        for (int w = 0; w < kPeelWarps; w++) t += red[w];
    __syncthreads();
    return t;
}

// pre[0] = 0, pre[i+1] = sum of the degrees of F[0..i], for f <= 1024
// entries (each thread owns 4 consecutive entries).
__device__ __forceinline__ void block_prefix_degrees(const PeelParams& P, const uint32_t* F,
                                                     uint32_t f, unsigned long long* pre,
                                                     unsigned long long* red) {
    static_assert(kSmallFront == 4 * kPeelThreads, "one thread per 4 frontier entries");
    unsigned long long d[4], sum = 0;
    uint32_t i0 = threadIdx.x * 4;
#pragma unroll
    for (int q = 0; q < 4; q++) {
        uint32_t i = i0 + q;
        d[q] = 0;
        if (i < f) {
            uint32_t v = F[i];
            d[q] = P.off[v + 1] - P.off[v];
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
    for (int q = 0; q < 4; q++) {
        run += d[q];
        if (i0 + q < f) pre[i0 + q + 1] = run;
    }
    __syncthreads();
}

// One (v, w) work item of a frontier vertex v with h >= 3: the cliques
// {v, w, ...} whose members other than v are candidates of v and whose
// smallest such member is w.  Executed by one warp.
__device__ void process_vw(const PeelParams& P, uint32_t v, uint32_t w, unsigned long long k,
                           uint32_t* next, uint32_t* next_cnt, uint32_t* C, unsigned* cnt,
                           uint32_t* rows, uint32_t* big_cnt, unsigned long long& destroyed,
                           unsigned long long& bytes) {
    unsigned lane = lane_id();
    uint8_t sw = P.state[w];
    if (lane == 0) bytes += 4 + 1;   // w, state[w]
    if (!(sw == kAlive || (sw == kFront && w > v))) return;
    const uint32_t* Nv = P.adj + P.off[v];
    uint64_t dv = P.off[v + 1] - P.off[v];
    uint64_t b = P.split[w], e = P.off[w + 1];
    if (lane == 0) bytes += 16;
    const unsigned pr = probes(dv);
    uint32_t nc = 0;
    for (uint64_t p0 = b; p0 < e; p0 += 32) {
        uint64_t p = p0 + lane;
        bool ok = false;
        uint32_t x = 0;
        if (p < e) {
            x = P.adj[p];
            bytes += 4 + 1;
            if (candidate(P, x, v)) {
                uint64_t pos = lower_bound_u32(Nv, dv, x);
                ok = pos < dv && Nv[pos] == x;
                bytes += 4ull * pr;
            }
        }
        unsigned bal = __ballot_sync(0xffffffffu, ok);
        if (ok) C[nc + __popc(bal & ((1u << lane) - 1u))] = x;
        nc += __popc(bal);
    }
    __syncwarp();
    const int r = P.h - 2;
    unsigned long long tot = 0;
    if (r == 1) {
        tot = nc;
        for (uint32_t i = lane; i < nc; i += 32) {
            uint32_t x = C[i];
            bytes += 1;
            if (P.state[x] == kAlive) {
                dec_and_queue(P, x, 1ull, k, next, next_cnt);
                bytes += 16;
            }
        }
    } else {
        if (nc < (uint32_t)r) return;
        if (r >= 3 && nc > 32) {
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
            for (uint32_t i = 0; i < nc; i++) {
                uint32_t x = C[i];
                uint64_t xb = P.split[x], xe = P.off[x + 1];
                unsigned hits = 0;
                if (lane == 0) bytes += 16;
                for (uint64_t p = xb + lane; p < xe; p += 32) {
                    uint32_t y = P.adj[p];
                    bytes += 4;
                    uint32_t pos = (uint32_t)lower_bound_u32(C, nc, y);
                    if (pos < nc && C[pos] == y) { atomicAdd(&cnt[pos], 1u); hits++; }
                }
                hits = __reduce_add_sync(0xffffffffu, hits);
                if (lane == 0 && hits) atomicAdd(&cnt[i], hits);
                tot += hits;
            }
        } else {
            if (lane == 0)
                for (uint32_t i = 0; i < nc; i++)
                    bytes += 16 + 4ull * (P.off[C[i] + 1] - P.split[C[i]]);
            warp_build_rows32(C, nc, P.off, P.adj, P.split, rows);
            tot = warp_dfs32(rows, nc, r, cnt);
        }
        __syncwarp();
        if (tot)
            for (uint32_t i = lane; i < nc; i += 32) {
                uint32_t x = C[i];
                if (cnt[i]) {
                    bytes += 1;
                    if (P.state[x] == kAlive) {
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

// A (v, w) item whose candidate set exceeds 32 vertices (h >= 5): one block.
__device__ void process_big(const PeelParams& P, uint32_t v, uint32_t w, unsigned long long k,
                            uint32_t* next, uint32_t* next_cnt, uint32_t* smem,
                            unsigned long long& destroyed) {
    unsigned long long* cnt = reinterpret_cast<unsigned long long*>(smem);  // cap
    uint32_t* C = smem + 2 * P.cap;                                           // cap
    uint32_t* rows = C + P.cap;                                               // cap * W
    __shared__ uint32_t s_nc;
    __shared__ unsigned long long s_tot;
    unsigned lane = lane_id();
    uint8_t sw = P.state[w];
    if (warp_id() == 0) {
        const uint32_t* Nv = P.adj + P.off[v];
        uint64_t dv = P.off[v + 1] - P.off[v];
        uint64_t b = P.split[w], e = P.off[w + 1];
        uint32_t nc = 0;
        for (uint64_t p0 = b; p0 < e; p0 += 32) {
            uint64_t p = p0 + lane;
            bool ok = false;
            uint32_t x = 0;
            if (p < e) {
                x = P.adj[p];
                if (candidate(P, x, v)) {
                    uint64_t pos = lower_bound_u32(Nv, dv, x);
                    ok = pos < dv && Nv[pos] == x;
                }
            }
            unsigned bal = __ballot_sync(0xffffffffu, ok);
            if (ok) C[nc + __popc(bal & ((1u << lane) - 1u))] = x;
            nc += __popc(bal);
        }
        if (lane == 0) { s_nc = nc; s_tot = 0; }
    }
    __syncthreads();
    uint32_t nc = s_nc;
    uint32_t W = (nc + 31) >> 5;
    for (uint32_t i = threadIdx.x; i < nc; i += blockDim.x) cnt[i] = 0;
    for (uint32_t i = threadIdx.x; i < nc * W; i += blockDim.x) rows[i] = 0;
    __syncthreads();
    block_build_rows(C, nc, W, P.off, P.adj, P.split, rows);
    __syncthreads();
    unsigned long long mine = block_dfs(rows, nc, W, P.h - 2, cnt);
    if (mine) atomicAdd(&s_tot, mine);
    __syncthreads();
    unsigned long long tot = s_tot;
    if (tot) {
        for (uint32_t i = threadIdx.x; i < nc; i += blockDim.x) {
            uint32_t x = C[i];
            if (cnt[i] && P.state[x] == kAlive) dec_and_queue(P, x, cnt[i], k, next, next_cnt);
        }
        if (threadIdx.x == 0) {
            if (sw == kAlive) dec_and_queue(P, w, tot, k, next, next_cnt);
            destroyed += tot;
        }
    }
    __syncthreads();
}

// ---------------------------------------------------------------- kernel
__global__ void __launch_bounds__(kPeelThreads) k_peel(PeelParams P) {
    extern __shared__ uint32_t smem[];
    __shared__ unsigned long long s_pre[kSmallFront + 1];
    __shared__ unsigned long long s_red[kPeelWarps];
    PeelCtrl* c = P.ctrl;
    const unsigned lane = lane_id(), wid = warp_id();
    const uint64_t gtid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t gthreads = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t gwarp = gtid >> 5;
    const uint64_t gwarps = gthreads >> 5;
    uint32_t* wC = smem + (size_t)wid * (2 * P.cap + 32);
    unsigned* wCnt = wC + P.cap;
    uint32_t* wRows = wC + 2 * P.cap;

    unsigned long long k = 0;
    unsigned long long mu_alive = P.mu0;   // meaningful in block 0
    uint32_t r = 0, jumps = 0, nlev = 0;
    int ap = 0;
    uint32_t alive_cnt = P.n;
    unsigned long long items = 0;
    unsigned long long bytes = 0;

    for (;;) {
        // ---------------------------------------------------------- P1
        uint32_t fprev = r ? c->fcnt[(r + 2) % 3] : 0u;
        const uint32_t* Fprev = P.front[(r + 2) % 3];
        for (uint64_t i = gtid; i < fprev; i += gthreads) {
            uint32_t v = Fprev[i];
            P.state[v] = kGone;
            P.core[v] = k;
            if (P.rnd) P.rnd[v] = r - 1;
            bytes += 4 + 1 + 8 + (P.rnd ? 4 : 0);
        }
        uint32_t fcur = c->fcnt[r % 3];
        uint32_t* Fcur = P.front[r % 3];
        for (uint64_t i = gtid; i < fcur; i += gthreads) {
            P.state[Fcur[i]] = kFront;
            bytes += 4 + 1;
        }
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            if (r) {
                mu_alive -= c->destroyed[(r + 2) % 3];
                c->destroyed[(r + 2) % 3] = 0;
                c->big_cnt[(r + 2) % 3] = 0;
            }
            c->fcnt[(r + 1) % 3] = 0;
        }
        if (!grid_barrier(c, P.wait_ns)) break;

        // ----------------------------------------------------- level jump
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
                    bytes += 4 + 1;
                    if (P.state[v] != kGone) {
                        keep = true;
                        unsigned long long d = P.deg[v];
                        mn = d < mn ? d : mn;
                        bytes += 8 + 4;
                    }
                }
                warp_append(keep, v, &c->new_alive[jumps & 1], Aout);
            }
            mn = warp_min_u64(mn);
            if (lane == 0 && mn != ~0ull) atomicMin(&c->min_deg[jumps & 1], mn);
            if (!grid_barrier(c, P.wait_ns)) break;
            uint32_t na = c->new_alive[jumps & 1];
            if (na == 0) break;
            unsigned long long m2 = c->min_deg[jumps & 1];
            k = m2 > k ? m2 : k;
            ap ^= 1;
            alive_cnt = na;
            if (blockIdx.x == 0 && threadIdx.x == 0) {
                P.lvl_k[nlev] = k;
                P.lvl_size[nlev] = na;
                P.lvl_mu[nlev] = mu_alive;
                nlev++;
                c->min_deg[(jumps + 1) & 1] = ~0ull;
                c->new_alive[(jumps + 1) & 1] = 0;
            }
            jumps++;
            for (uint64_t base = gwarp * 32; base < na; base += gwarps * 32) {
                uint64_t i = base + lane;
                bool in = false;
                uint32_t v = 0;
                if (i < na) {
                    v = Aout[i];
                    bytes += 4 + 8;
                    if (P.deg[v] <= k) {
                        in = true;
                        P.state[v] = kFront;
                        bytes += 1 + 4;
                    }
                }
                warp_append(in, v, &c->fcnt[r % 3], Fcur);
            }
            if (!grid_barrier(c, P.wait_ns)) break;
            fcur = c->fcnt[r % 3];
        }

        // ----------------------------------------------------------- P2
        uint32_t* Fnext = P.front[(r + 1) % 3];
        uint32_t* next_cnt = &c->fcnt[(r + 1) % 3];
        unsigned long long destroyed = 0;
        if (fcur <= kSmallFront) {
            // flatten (v, neighbour index) items over the whole grid
            block_prefix_degrees(P, Fcur, fcur, s_pre, s_red);
            unsigned long long T = s_pre[fcur];
            if (blockIdx.x == 0 && threadIdx.x == 0) {
                items += T;
                bytes += 20ull * fcur;   // frontier ids and their offsets
            }
            if (P.h == 2) {
                for (uint64_t t = gtid; t < T; t += gthreads) {
                    uint32_t lo = 0, hi = fcur;  // last i with s_pre[i] <= t
                    while (hi - lo > 1) {
                        uint32_t mid = (lo + hi) >> 1;
                        if (s_pre[mid] <= t) lo = mid; else hi = mid;
                    }
                    uint32_t v = Fcur[lo];
                    uint32_t u = P.adj[P.off[v] + (t - s_pre[lo])];
                    uint8_t su = P.state[u];
                    bytes += 4 + 1;
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
                    uint32_t lo = 0, hi = fcur;
                    while (hi - lo > 1) {
                        uint32_t mid = (lo + hi) >> 1;
                        if (s_pre[mid] <= t) lo = mid; else hi = mid;
                    }
                    uint32_t v = Fcur[lo];
                    uint32_t w = P.adj[P.off[v] + (t - s_pre[lo])];
                    process_vw(P, v, w, k, Fnext, next_cnt, wC, wCnt, wRows,
                               &c->big_cnt[r % 3], destroyed, bytes);
                }
            }
        } else {
            if (P.h == 2) {
                for (uint64_t i = gwarp; i < fcur; i += gwarps) {
                    uint32_t v = Fcur[i];
                    uint64_t b = P.off[v], e = P.off[v + 1];
                    for (uint64_t p = b + lane; p < e; p += 32) {
                        uint32_t u = P.adj[p];
                        uint8_t su = P.state[u];
                        bytes += 4 + 1;
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
                for (uint64_t i = blockIdx.x; i < fcur; i += gridDim.x) {
                    uint32_t v = Fcur[i];
                    uint64_t b = P.off[v], e = P.off[v + 1];
                    for (uint64_t p = b + wid; p < e; p += kPeelWarps)
                        process_vw(P, v, P.adj[p], k, Fnext, next_cnt, wC, wCnt, wRows,
                                   &c->big_cnt[r % 3], destroyed, bytes);
                    if (threadIdx.x == 0) {
                        items += e - b;
                        bytes += 20;
                    }
                }
            }
        }
        unsigned long long bd = block_sum(destroyed, s_red);
        if (threadIdx.x == 0 && bd) atomicAdd(&c->destroyed[r % 3], bd);
        if (!grid_barrier(c, P.wait_ns)) break;

        // ---------------------------------------------------------- P2b
        if (P.h >= 5) {
            uint32_t nb = c->big_cnt[r % 3];
            if (nb) {
                if (nb > P.big_cap) nb = (uint32_t)P.big_cap;
                unsigned long long d2 = 0;
                for (uint32_t i = blockIdx.x; i < nb; i += gridDim.x) {
                    uint2 it = P.big[i];
                    process_big(P, it.x, it.y, k, Fnext, next_cnt, smem, d2);
                }
                if (threadIdx.x == 0 && d2) atomicAdd(&c->destroyed[r % 3], d2);
                if (!grid_barrier(c, P.wait_ns)) break;
            }
        }
        r++;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        c->kmax = k;
        c->nlevels = nlev;
        c->rounds = r;
    }
    items = warp_sum(items);
    bytes = warp_sum(bytes);
    if (lane == 0 && items) atomicAdd(&c->items, items);
    if (lane == 0 && bytes) atomicAdd(&c->bytes, bytes);
}

__global__ void k_peel_init(uint32_t n, uint8_t* state, uint32_t* alive0, PeelCtrl* c) {
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x) {
        state[i] = kAlive;
        alive0[i] = (uint32_t)i;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        c->min_deg[0] = ~0ull;
        c->min_deg[1] = ~0ull;
    }
}

}  // namespace

dsd_status run_peel(dsd_graph* g, int h, uint32_t n, const uint64_t* off, const uint32_t* adj,
                    const uint64_t* split, uint32_t maxdplus, unsigned long long* deg,
                    uint64_t mu0, uint64_t* core, uint32_t* rnd, uint64_t* lvl_k,
                    uint32_t* lvl_size, uint64_t* lvl_mu, PeelResult* res) {
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
    P.adj = adj;
    P.split = split;
    P.deg = deg;
    P.core = core;
    P.rnd = rnd;
    P.lvl_k = lvl_k;
    P.lvl_size = lvl_size;
    P.lvl_mu = lvl_mu;
    P.wait_ns = wait_limit_ns();
    P.mu0 = mu0;
    P.cap = maxdplus < 32 ? 32 : maxdplus;
    size_t warp_words = (size_t)2 * P.cap + 32;
    size_t smem = h >= 3 ? warp_words * kPeelWarps * 4 : 0;
    if (h >= 5) {
        uint32_t W = (P.cap + 31) / 32;
        size_t big = ((size_t)3 * P.cap + (size_t)P.cap * W) * 4;
        if (big > smem) smem = big;
        if (maxdplus > kBitmapMax) {
            set_error("h=%d peeling needs at most %u higher-ranked neighbours per vertex "
                      "(max here %u)", h, kBitmapMax, maxdplus);
            return DSD_ERR_UNSUPPORTED;
        }
    }
    if (smem > 48 * 1024)
        DSD_CU(cudaFuncSetAttribute(k_peel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem));
    int per_sm = 0;
    DSD_CU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_peel, kPeelThreads, smem));
    if (per_sm <= 0) {
        set_error("peel kernel does not fit on an SM (shared memory %zu bytes)", smem);
        return DSD_ERR_UNSUPPORTED;
    }
    if (per_sm > 4) per_sm = 4;
    unsigned grid = (unsigned)(sms * per_sm);

    uint8_t* state = nullptr;
    uint32_t* lists = nullptr;
    PeelCtrl* ctrl = nullptr;
    uint2* big = nullptr;
    dsd_status st = DSD_OK;
    PeelCtrl hc;
    cudaError_t e = cudaSuccess;
    if ((st = dalloc(&state, n, s)) != DSD_OK) goto done;
    if ((st = dalloc(&lists, (size_t)5 * n, s)) != DSD_OK) goto done;
    if ((st = dalloc(&ctrl, 1, s)) != DSD_OK) goto done;
    if (h >= 5) {
        P.big_cap = g->m * 2 + 1;
        if ((st = dalloc(&big, P.big_cap, s)) != DSD_OK) goto done;
    }
    P.state = state;
    P.alive[0] = lists;
    P.alive[1] = lists + n;
    P.front[0] = lists + 2 * (size_t)n;
    P.front[1] = lists + 3 * (size_t)n;
    P.front[2] = lists + 4 * (size_t)n;
    P.big = big;
    P.ctrl = ctrl;
    e = cudaMemsetAsync(ctrl, 0, sizeof(PeelCtrl), s);
    if (e == cudaSuccess) {
        k_peel_init<<<sms * 4, 256, 0, s>>>(n, state, P.alive[0], ctrl); note_launch();
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        void* args[] = {&P};
        e = cudaLaunchCooperativeKernel((void*)k_peel, dim3(grid), dim3(kPeelThreads), args,
                                        smem, s);
        note_launch();
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
done:
    dev_free(state, s);
    dev_free(lists, s);
    dev_free(ctrl, s);
    dev_free(big, s);
    return st;
}

}  // namespace dsd
