// Many small graphs (mixed h) in one persistent launch.
//
// Each CTA takes graphs from an atomic work queue (largest first) and runs
// the whole path of one graph by itself -- CSR build (Sec. 2 data model),
// degeneracy peel (edge k-cores, Def. 5), rank relabelling, h-clique
// clique-degrees (Def. 3) and the level-synchronous (k,Psi)-core peel
// (Algorithm 3) with its level statistics, then the CoreApp outputs (k_max
// core, Lemma 6; densest level, Pruning1).  Within a graph the phases are
// separated by __syncthreads only: no grid barrier, no host round trip.
// Per-graph scratch is a private slice of one workspace per CTA.
//
// Graph size limits: n <= 65535 vertices (keys u * n + v fit 32 bits) and,
// for h = 4, at most 512 higher-ranked neighbours per vertex.
#include "cliques.cuh"
#include "graph.cuh"

#include <string.h>

namespace dsd {
namespace {

constexpr uint32_t kBatchMaxN = 65535;
constexpr uint32_t kBatchMaxDplus = 512;
enum : uint32_t { kBOk = 0, kBInvalid = 1, kBUnsupported = 2 };
enum : uint32_t { kAl = 0, kFr = 1, kGo = 2 };

struct BatchDesc {
    uint64_t e_off;     // first edge of this graph in src/dst
    uint64_t core_off;  // first entry of its core numbers (~0: not wanted)
    uint32_t m;         // raw edges
    uint32_t n;
    int32_t h;
    uint32_t pad;
};

struct BatchRes {
    unsigned long long kmax, kmax_core_mu, best_k, densest_mu, mu, m_clean;
    uint32_t kmax_core_size, densest_size, nlevels, status;
};

// Per-CTA workspace (global memory), sized for the largest graph.
struct Work {
    uint32_t* k1;       // keys / scratch, E
    uint32_t* k2;       // keys / scratch, E
    uint32_t* adj;      // rows (caller ids), E
    uint32_t* radj;     // rows (ranks), E
    uint32_t* off;      // n + 1
    uint32_t* roff;     // n + 1
    uint32_t* rsplit;   // n
    uint32_t* rnd;      // n
    uint32_t* new_of;   // n
    uint32_t* old_of;   // n
    uint32_t* st;       // n
    uint32_t* fa;       // n  (frontier)
    uint32_t* fb;       // n  (next frontier)
    uint32_t* alive;    // n
    unsigned long long* deg;   // n
    unsigned long long* core;  // n
    unsigned long long* lk;    // n + 1
    unsigned long long* lm;    // n + 1
    uint32_t* ls;              // n + 1
};

struct BatchArgs {
    const BatchDesc* desc;
    const uint32_t* order;     // graphs, largest first
    uint32_t count;
    const uint32_t* src;
    const uint32_t* dst;
    BatchRes* res;
    unsigned long long* cores; // concatenated core numbers (may be null)
    uint32_t* queue;           // work counter
    uint8_t* ws;               // workspaces
    uint64_t ws_stride;        // bytes per CTA
    uint32_t maxn;
    uint64_t maxe;
};

__device__ __forceinline__ uint8_t* align_up(uint8_t* p) {
    return (uint8_t*)(((uintptr_t)p + 255) & ~(uintptr_t)255);
}

__device__ Work carve(uint8_t* base, uint32_t maxn, uint64_t maxe) {
    Work w;
    uint8_t* p = align_up(base);
    auto take = [&](size_t bytes) {
        uint8_t* r = p;
        p = align_up(p + bytes);
        return r;
    };
    w.k1 = (uint32_t*)take(maxe * 4);
    w.k2 = (uint32_t*)take(maxe * 4);
    w.adj = (uint32_t*)take(maxe * 4);
    w.radj = (uint32_t*)take(maxe * 4);
    w.off = (uint32_t*)take(((size_t)maxn + 1) * 4);
    w.roff = (uint32_t*)take(((size_t)maxn + 1) * 4);
    w.rsplit = (uint32_t*)take((size_t)maxn * 4 + 4);
    w.rnd = (uint32_t*)take((size_t)maxn * 4 + 4);
    w.new_of = (uint32_t*)take((size_t)maxn * 4 + 4);
    w.old_of = (uint32_t*)take((size_t)maxn * 4 + 4);
    w.st = (uint32_t*)take((size_t)maxn * 4 + 4);
    w.fa = (uint32_t*)take((size_t)maxn * 4 + 4);
    w.fb = (uint32_t*)take((size_t)maxn * 4 + 4);
    w.alive = (uint32_t*)take((size_t)maxn * 4 + 4);
    w.deg = (unsigned long long*)take((size_t)maxn * 8 + 8);
    w.core = (unsigned long long*)take((size_t)maxn * 8 + 8);
    w.lk = (unsigned long long*)take(((size_t)maxn + 1) * 8);
    w.lm = (unsigned long long*)take(((size_t)maxn + 1) * 8);
    w.ls = (uint32_t*)take(((size_t)maxn + 1) * 4);
    return w;
}

// Shared-memory layout used by the phases (they run one after another).
template <int NT>
struct Smem {
    static constexpr int NW = NT / 32;
    uint32_t wcnt[NW][256];     // radix: per-warp digit counts
    uint32_t base[256];         // radix: digit offsets
    uint32_t tcnt[256];
    uint32_t wbuf[NW][2 * kBatchMaxDplus + 64];   // per-warp candidate lists
    unsigned long long red[NW];
    uint32_t ured[NW];
    uint32_t cnt1, cnt2, flag;
    unsigned long long k, mu_alive;
};

// ------------------------------------------------ block-level building blocks

// Exclusive prefix of per-thread counts; returns this thread's prefix and the
// total (all threads).
template <int NT>
__device__ __forceinline__ uint32_t bscan(uint32_t v, uint32_t* ured, uint32_t* total) {
    unsigned lane = lane_id(), wid = warp_id();
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if ((int)lane >= o) x += y;
    }
    if (lane == 31) ured[wid] = x;
    __syncthreads();
    uint32_t before = 0, all = 0;
    for (int w = 0; w < NT / 32; w++) {
        uint32_t t = ured[w];
        before += (w < (int)wid) ? t : 0u;
        all += t;
    }
    __syncthreads();
    *total = all;
    return before + x - v;
}

template <int NT>
__device__ __forceinline__ unsigned long long bmin(unsigned long long v, unsigned long long* red) {
    v = warp_min_u64(v);
    if (lane_id() == 0) red[warp_id()] = v;
    __syncthreads();
    unsigned long long m = ~0ull;
    for (int w = 0; w < NT / 32; w++) m = red[w] < m ? red[w] : m;
    __syncthreads();
    return m;
}

template <int NT>
__device__ __forceinline__ unsigned long long bsum(unsigned long long v, unsigned long long* red) {
    v = warp_sum(v);
    if (lane_id() == 0) red[warp_id()] = v;
    __syncthreads();
    unsigned long long m = 0;
    for (int w = 0; w < NT / 32; w++) m += red[w];
    __syncthreads();
    return m;
}

// Stable LSD radix sort of a[0..cnt) (u32 keys below 2^bits) by one CTA; the
// result ends in a (b is scratch).  Digits of 8 bits; each warp ranks its
// keys in order with match masks, so equal digits keep their order.
template <int NT>
__device__ void block_radix_sort(uint32_t* a, uint32_t* b, uint32_t cnt, int bits, Smem<NT>& S) {
    constexpr int NW = NT / 32;
    constexpr int ITEMS = 8;
    constexpr uint32_t TILE = NT * ITEMS;
    const unsigned lane = lane_id(), wid = warp_id();
    uint32_t* src = a;
    uint32_t* dst = b;
    int passes = 0;
    for (int shift = 0; shift < bits; shift += 8) {
        // digit histogram of the whole array -> exclusive offsets
        for (uint32_t i = threadIdx.x; i < 256; i += NT) S.base[i] = 0;
        __syncthreads();
        for (uint32_t i = threadIdx.x; i < cnt; i += NT) atomicAdd(&S.base[(src[i] >> shift) & 255u], 1u);
        __syncthreads();
        if (threadIdx.x == 0) {
            uint32_t run = 0;
            for (int d = 0; d < 256; d++) {
                uint32_t t = S.base[d];
                S.base[d] = run;
                run += t;
            }
        }
        __syncthreads();
        for (uint32_t t0 = 0; t0 < cnt; t0 += TILE) {
            for (uint32_t i = threadIdx.x; i < NW * 256; i += NT) (&S.wcnt[0][0])[i] = 0;
            __syncthreads();
            uint32_t key[ITEMS], rk[ITEMS];
            // warp w holds tile entries [w*32*ITEMS, (w+1)*32*ITEMS), item j at j*32 + lane
#pragma unroll
            for (int j = 0; j < ITEMS; j++) {
                uint32_t idx = t0 + wid * 32 * ITEMS + j * 32 + lane;
                bool ok = idx < cnt;
                key[j] = ok ? src[idx] : 0u;
                uint32_t d = ok ? ((key[j] >> shift) & 255u) : 256u;
                unsigned peers = __match_any_sync(0xffffffffu, d);
                uint32_t before = 0;
                if (ok) {
                    int leader = __ffs(peers) - 1;
                    uint32_t prior = 0;
                    if ((int)lane == leader) prior = S.wcnt[wid][d];
                    prior = __shfl_sync(peers, prior, leader);
                    before = prior + __popc(peers & ((1u << lane) - 1u));
                    if ((int)lane == leader) S.wcnt[wid][d] = prior + __popc(peers);
                }
                rk[j] = before;
                __syncwarp();
            }
            __syncthreads();
            // per digit: prefix over warps, tile total
            for (uint32_t d = threadIdx.x; d < 256; d += NT) {
                uint32_t run = 0;
                for (int w = 0; w < NW; w++) {
                    uint32_t t = S.wcnt[w][d];
                    S.wcnt[w][d] = run;
                    run += t;
                }
                S.tcnt[d] = run;
            }
            __syncthreads();
#pragma unroll
            for (int j = 0; j < ITEMS; j++) {
                uint32_t idx = t0 + wid * 32 * ITEMS + j * 32 + lane;
                if (idx < cnt) {
                    uint32_t d = (key[j] >> shift) & 255u;
                    dst[S.base[d] + S.wcnt[wid][d] + rk[j]] = key[j];
                }
            }
            __syncthreads();
            for (uint32_t d = threadIdx.x; d < 256; d += NT) S.base[d] += S.tcnt[d];
            __syncthreads();
        }
        uint32_t* t = src;
        src = dst;
        dst = t;
        passes++;
    }
    if (passes & 1)
        for (uint32_t i = threadIdx.x; i < cnt; i += NT) a[i] = src[i];
    __syncthreads();
}

__device__ __forceinline__ uint32_t key_bits(uint64_t maxkey) {
    uint32_t b = 0;
    while (b < 32 && (maxkey >> b)) b += 8;
    return b ? b : 8;
}

// Sorted keys u * n + v (deduplicated in place) -> CSR off[0..n], adj.
// Returns the number of entries.
template <int NT>
__device__ uint32_t keys_to_csr(uint32_t* keys, uint32_t cnt, uint32_t n, uint32_t* off,
                                uint32_t* adj, Smem<NT>& S) {
    // unique (ordered compaction; each pass reads its tile before writing)
    if (threadIdx.x == 0) S.cnt1 = 0;
    __syncthreads();
    for (uint32_t t0 = 0; t0 < cnt; t0 += NT) {
        uint32_t i = t0 + threadIdx.x;
        uint32_t k = i < cnt ? keys[i] : 0u;
        bool keep = i < cnt && (i == 0 || keys[i - 1] != k);
        uint32_t tot;
        uint32_t at = bscan<NT>(keep ? 1u : 0u, S.ured, &tot);
        uint32_t o = S.cnt1;
        __syncthreads();
        if (keep) keys[o + at] = k;
        __syncthreads();
        if (threadIdx.x == 0) S.cnt1 = o + tot;
        __syncthreads();
    }
    uint32_t u = S.cnt1;
    for (uint32_t i = threadIdx.x; i < u; i += NT) adj[i] = keys[i] % n;
    for (uint32_t v = threadIdx.x; v <= n; v += NT) {
        uint32_t target = v * n;  // first key of row v (v < n; v == n gives u)
        uint32_t lo = 0, hi = u;
        if (v == n) lo = u;
        while (lo < hi) {
            uint32_t mid = (lo + hi) >> 1;
            if (keys[mid] < target) lo = mid + 1; else hi = mid;
        }
        off[v] = lo;
    }
    __syncthreads();
    return u;
}

// ------------------------------------------------------------ peeling

struct BPeel {
    const uint32_t* off;
    const uint32_t* adj;
    const uint32_t* nplus;   // start of N+ per vertex (h >= 3)
    uint32_t n;
    int h;
    unsigned long long* deg;
    unsigned long long* core;
    uint32_t* rnd;           // may be null
    uint32_t* st;
    uint32_t* alive;
    uint32_t* fa;
    uint32_t* fb;
    unsigned long long* lk;
    unsigned long long* lm;
    uint32_t* ls;
    unsigned long long mu0;
};

__device__ __forceinline__ bool bcand(const BPeel& B, uint32_t x, uint32_t v) {
    uint32_t s = B.st[x];
    return s == kAl || (s == kFr && x > v);
}

__device__ __forceinline__ void bdec(const BPeel& B, uint32_t u, unsigned long long c,
                                     unsigned long long k, uint32_t* next, uint32_t* ncnt) {
    unsigned long long old = atomic_sub_u64(&B.deg[u], c);
    if (old > k && old - c <= k) next[atomicAdd(ncnt, 1u)] = u;
}

// Lanes of this lane's group when a warp scans 32 / LPR rows at once, LPR
// lanes each (the intersection tile the launch was tuned with).
template <int LPR>
__device__ __forceinline__ unsigned group_mask() {
    if (LPR == 32) return 0xffffffffu;
    return ((1u << LPR) - 1u) << (lane_id() & ~(unsigned)(LPR - 1));
}

// (v, w) item for h >= 3, one warp: the cliques {v, w, ...} whose other
// members are candidates of v and whose smallest such member is w.
template <int LPR>
__device__ unsigned long long bitem(const BPeel& B, uint32_t v, uint32_t w, unsigned long long k,
                                    uint32_t* next, uint32_t* ncnt, uint32_t* C, uint32_t* cnt) {
    unsigned lane = lane_id();
    if (!bcand(B, w, v)) return 0;
    const uint32_t* Nv = B.adj + B.off[v];
    uint32_t dv = B.off[v + 1] - B.off[v];
    uint32_t b = B.nplus[w], e = B.off[w + 1];
    uint32_t nc = 0;
    for (uint32_t p0 = b; p0 < e; p0 += 32) {
        uint32_t p = p0 + lane;
        bool ok = false;
        uint32_t x = 0;
        if (p < e) {
            x = B.adj[p];
            if (bcand(B, x, v)) {
                uint32_t pos = (uint32_t)lower_bound_u32(Nv, dv, x);
                ok = pos < dv && Nv[pos] == x;
            }
        }
        unsigned bal = __ballot_sync(0xffffffffu, ok);
        if (ok) C[nc + __popc(bal & ((1u << lane) - 1u))] = x;
        nc += __popc(bal);
    }
    __syncwarp();
    unsigned long long tot = 0;
    if (B.h == 3) {
        tot = nc;
        for (uint32_t i = lane; i < nc; i += 32)
            if (B.st[C[i]] == kAl) bdec(B, C[i], 1ull, k, next, ncnt);
    } else {
        // h = 4: edges of G[C]; the warp scans 32 / LPR rows at once
        for (uint32_t i = lane; i < nc; i += 32) cnt[i] = 0;
        __syncwarp();
        const unsigned gl = lane & (LPR - 1), gm = group_mask<LPR>();
        unsigned long long mine = 0;
        for (uint32_t i = lane / LPR; i < nc; i += 32 / LPR) {
            uint32_t x = C[i];
            unsigned hits = 0;
            for (uint32_t p = B.nplus[x] + gl; p < B.off[x + 1]; p += LPR) {
                uint32_t y = B.adj[p];
                uint32_t pos = (uint32_t)lower_bound_u32(C, nc, y);
                if (pos < nc && C[pos] == y) { atomicAdd(&cnt[pos], 1u); hits++; }
            }
            hits = __reduce_add_sync(gm, hits);
            if (gl == 0 && hits) atomicAdd(&cnt[i], hits);
            if (gl == 0) mine += hits;
        }
        __syncwarp();
        tot = warp_sum(mine);
        if (tot)
            for (uint32_t i = lane; i < nc; i += 32)
                if (cnt[i] && B.st[C[i]] == kAl) bdec(B, C[i], cnt[i], k, next, ncnt);
        __syncwarp();
    }
    if (tot && lane == 0 && B.st[w] == kAl) bdec(B, w, tot, k, next, ncnt);
    return tot;
}

// Level-synchronous peel of one graph by one CTA; returns k_max and writes
// the level records; *nl receives their number.
template <int NT, int LPR>
__device__ unsigned long long block_peel(const BPeel& B, Smem<NT>& S, uint32_t* nl) {
    constexpr int NW = NT / 32;
    const unsigned lane = lane_id(), wid = warp_id();
    uint32_t n = B.n;
    for (uint32_t v = threadIdx.x; v < n; v += NT) {
        B.st[v] = kAl;
        B.alive[v] = v;
    }
    if (threadIdx.x == 0) {
        S.cnt1 = 0;   // current frontier size
        S.mu_alive = B.mu0;
    }
    __syncthreads();
    unsigned long long k = 0;
    uint32_t na = n, nlev = 0, r = 0;
    uint32_t* F = B.fa;
    uint32_t* G = B.fb;
    uint32_t nf = 0;
    for (;;) {
        if (nf == 0) {
            // level jump: compact the alive list, minimum count, frontier
            if (threadIdx.x == 0) S.cnt2 = 0;
            __syncthreads();
            unsigned long long mn = ~0ull;
            for (uint32_t t0 = 0; t0 < na; t0 += NT) {
                uint32_t i = t0 + threadIdx.x;
                uint32_t v = i < na ? B.alive[i] : 0u;
                bool keep = i < na && B.st[v] == kAl;
                if (keep) mn = B.deg[v] < mn ? B.deg[v] : mn;
                uint32_t tot;
                uint32_t at = bscan<NT>(keep ? 1u : 0u, S.ured, &tot);
                uint32_t o = S.cnt2;
                __syncthreads();
                if (keep) B.alive[o + at] = v;
                __syncthreads();
                if (threadIdx.x == 0) S.cnt2 = o + tot;
                __syncthreads();
            }
            na = S.cnt2;
            mn = bmin<NT>(mn, S.red);
            if (na == 0) break;
            k = mn > k ? mn : k;
            if (threadIdx.x == 0) {
                B.lk[nlev] = k;
                B.ls[nlev] = na;
                B.lm[nlev] = S.mu_alive;
                S.cnt1 = 0;
            }
            nlev++;
            __syncthreads();
            for (uint32_t i = threadIdx.x; i < na; i += NT) {
                uint32_t v = B.alive[i];
                if (B.deg[v] <= k) F[atomicAdd(&S.cnt1, 1u)] = v;
            }
            __syncthreads();
            nf = S.cnt1;
        }
        for (uint32_t i = threadIdx.x; i < nf; i += NT) B.st[F[i]] = kFr;
        if (threadIdx.x == 0) S.cnt2 = 0;   // next frontier size
        __syncthreads();
        unsigned long long destroyed = 0;
        if (B.h == 2) {
            for (uint32_t i = wid; i < nf; i += NW) {
                uint32_t v = F[i];
                for (uint32_t p = B.off[v] + lane; p < B.off[v + 1]; p += 32) {
                    uint32_t u = B.adj[p];
                    uint32_t s = B.st[u];
                    if (s == kAl) {
                        bdec(B, u, 1ull, k, G, &S.cnt2);
                        destroyed++;
                    } else if (s == kFr && u > v) {
                        destroyed++;
                    }
                }
            }
        } else {
            uint32_t* C = S.wbuf[wid];
            uint32_t* cnt = C + kBatchMaxDplus;
            for (uint32_t i = 0; i < nf; i++) {
                uint32_t v = F[i];
                for (uint32_t p = B.off[v] + wid; p < B.off[v + 1]; p += NW) {
                    unsigned long long t = bitem<LPR>(B, v, B.adj[p], k, G, &S.cnt2, C, cnt);
                    if (lane == 0) destroyed += t;
                }
            }
        }
        destroyed = bsum<NT>(destroyed, S.red);
        for (uint32_t i = threadIdx.x; i < nf; i += NT) {
            uint32_t v = F[i];
            B.st[v] = kGo;
            B.core[v] = k;
            if (B.rnd) B.rnd[v] = r;
        }
        if (threadIdx.x == 0) S.mu_alive -= destroyed;
        __syncthreads();
        nf = S.cnt2;
        uint32_t* t = F;
        F = G;
        G = t;
        r++;
    }
    *nl = nlev;
    return k;
}

// a/b >= c/d in 128-bit arithmetic.
__device__ __forceinline__ bool bratio_ge(unsigned long long a, unsigned long long b,
                                          unsigned long long c, unsigned long long d) {
    unsigned long long lhi = __umul64hi(a, d), llo = a * d;
    unsigned long long rhi = __umul64hi(c, b), rlo = c * b;
    return lhi > rhi || (lhi == rhi && llo >= rlo);
}

// ------------------------------------------------------------ the kernel
// LPR: lanes per row scan (the intersection tile; 32 / LPR rows at once per
// warp in the triangle listing and the h = 4 edge counts).
template <int NT, int LPR>
__global__ void __launch_bounds__(NT) k_batch(BatchArgs A) {
    constexpr int NW = NT / 32;
    extern __shared__ uint8_t smem_raw[];
    Smem<NT>& S = *reinterpret_cast<Smem<NT>*>(smem_raw);
    __shared__ uint32_t s_gi;
    const unsigned lane = lane_id(), wid = warp_id();
    Work W = carve(A.ws + (size_t)blockIdx.x * A.ws_stride, A.maxn, A.maxe);
    for (;;) {
        if (threadIdx.x == 0) s_gi = atomicAdd(A.queue, 1u);
        __syncthreads();
        uint32_t qi = s_gi;
        __syncthreads();
        if (qi >= A.count) break;
        const uint32_t gi = A.order[qi];
        const BatchDesc D = A.desc[gi];
        const uint32_t n = D.n;
        BatchRes R;
        memset(&R, 0, sizeof(R));
        if (n == 0 || n > kBatchMaxN || D.h < 2 || D.h > 4) {
            if (threadIdx.x == 0) {
                R.status = n == 0 ? kBOk : kBInvalid;
                A.res[gi] = R;
            }
            __syncthreads();
            continue;
        }
        // ---- CSR: keys u*n+v for both orientations, loops dropped
        if (threadIdx.x == 0) {
            S.cnt1 = 0;
            S.flag = 0;
        }
        __syncthreads();
        for (uint32_t e = threadIdx.x; e < D.m; e += NT) {
            uint32_t u = A.src[D.e_off + e], v = A.dst[D.e_off + e];
            if (u >= n || v >= n) {
                S.flag = 1;
                continue;
            }
            if (u == v) continue;
            uint32_t at = atomicAdd(&S.cnt1, 2u);
            W.k1[at] = u * n + v;
            W.k1[at + 1] = v * n + u;
        }
        __syncthreads();
        if (S.flag) {
            if (threadIdx.x == 0) {
                R.status = kBInvalid;
                A.res[gi] = R;
            }
            __syncthreads();
            continue;
        }
        const uint32_t nkeys = S.cnt1;
        const int kb = key_bits((uint64_t)n * n - 1);
        block_radix_sort<NT>(W.k1, W.k2, nkeys, kb, S);
        const uint32_t E = keys_to_csr<NT>(W.k1, nkeys, n, W.off, W.adj, S);
        R.m_clean = E / 2;
        // ---- degeneracy peel (the h = 2 decomposition)
        for (uint32_t v = threadIdx.x; v < n; v += NT) W.deg[v] = W.off[v + 1] - W.off[v];
        __syncthreads();
        BPeel B2;
        B2.off = W.off;
        B2.adj = W.adj;
        B2.nplus = nullptr;
        B2.n = n;
        B2.h = 2;
        B2.deg = W.deg;
        B2.core = W.core;
        B2.rnd = W.rnd;
        B2.st = W.st;
        B2.alive = W.alive;
        B2.fa = W.fa;
        B2.fb = W.fb;
        B2.lk = W.lk;
        B2.lm = W.lm;
        B2.ls = W.ls;
        B2.mu0 = E / 2;
        uint32_t nl = 0;
        unsigned long long kmax = block_peel<NT, LPR>(B2, S, &nl);
        unsigned long long mu = E / 2;
        const unsigned long long* corev = W.core;   // caller ids
        if (D.h >= 3) {
            // ---- rank = (round, id), relabel, sorted rows
            for (uint32_t v = threadIdx.x; v < n; v += NT) W.k2[v] = (W.rnd[v] << 16) | v;
            __syncthreads();
            block_radix_sort<NT>(W.k2, W.k1, n, 32, S);
            for (uint32_t i = threadIdx.x; i < n; i += NT) {
                uint32_t o = W.k2[i] & 0xffffu;
                W.old_of[i] = o;
                W.new_of[o] = i;
            }
            __syncthreads();
            for (uint32_t v = threadIdx.x; v < n; v += NT) {
                uint32_t nv = W.new_of[v];
                for (uint32_t p = W.off[v]; p < W.off[v + 1]; p++) W.k1[p] = nv * n + W.new_of[W.adj[p]];
            }
            __syncthreads();
            block_radix_sort<NT>(W.k1, W.k2, E, kb, S);
            keys_to_csr<NT>(W.k1, E, n, W.roff, W.radj, S);
            // N+(v): first entry above v; largest out-degree
            if (threadIdx.x == 0) S.cnt2 = 0;
            __syncthreads();
            for (uint32_t v = threadIdx.x; v < n; v += NT) {
                uint32_t b = W.roff[v], e = W.roff[v + 1];
                uint32_t s = b + (uint32_t)lower_bound_u32(W.radj + b, e - b, v + 1u);
                W.rsplit[v] = s;
                atomicMax(&S.cnt2, e - s);
            }
            __syncthreads();
            if (S.cnt2 > kBatchMaxDplus) {
                if (threadIdx.x == 0) {
                    R.status = kBUnsupported;
                    A.res[gi] = R;
                }
                __syncthreads();
                continue;
            }
            // ---- clique-degrees (warp per vertex, candidates in shared memory)
            for (uint32_t v = threadIdx.x; v < n; v += NT) W.deg[v] = 0;
            __syncthreads();
            unsigned long long mu_loc = 0;
            {
                uint32_t* C = S.wbuf[wid];
                uint32_t* cnt = C + kBatchMaxDplus;
                uint32_t* rows = cnt + kBatchMaxDplus;
                for (uint32_t u = wid; u < n; u += NW) {
                    uint32_t b = W.rsplit[u], e = W.roff[u + 1], d = e - b;
                    if (d < (uint32_t)(D.h - 1)) continue;
                    for (uint32_t i = lane; i < d; i += 32) {
                        C[i] = W.radj[b + i];
                        cnt[i] = 0;
                    }
                    __syncwarp();
                    unsigned long long tot = 0;
                    if (D.h == 3) {
                        // each hit of a row scan is a triangle {u, x, y}; the
                        // warp scans 32 / LPR rows at once
                        const unsigned gl = lane & (LPR - 1), gm = group_mask<LPR>();
                        unsigned long long mine = 0;
                        for (uint32_t i = lane / LPR; i < d; i += 32 / LPR) {
                            uint32_t x = C[i];
                            unsigned hits = 0;
                            for (uint32_t p = W.rsplit[x] + gl; p < W.roff[x + 1]; p += LPR) {
                                uint32_t y = W.radj[p];
                                uint32_t pos = (uint32_t)lower_bound_u32(C, d, y);
                                if (pos < d && C[pos] == y) { atomicAdd(&cnt[pos], 1u); hits++; }
                            }
                            hits = __reduce_add_sync(gm, hits);
                            if (gl == 0 && hits) atomicAdd(&cnt[i], hits);
                            if (gl == 0) mine += hits;
                        }
                        __syncwarp();
                        tot = warp_sum(mine);
                    } else if (d <= 32) {
                        // h = 4: triangles of G[C] by the one-word bitmap DFS
                        warp_build_rows32(C, d, W.roff + 1, W.radj, W.rsplit, rows);
                        tot = warp_dfs32(rows, d, 3, cnt);
                    } else {
                        // h = 4, |C| > 32: every edge (x, y) of G[C] with x < y,
                        // and each common higher neighbour z of x and y in C
                        for (uint32_t i = 0; i < d; i++) {
                            uint32_t x = C[i];
                            const uint32_t* Nx = W.radj + W.rsplit[x];
                            uint32_t dx = W.roff[x + 1] - W.rsplit[x];
                            for (uint32_t p = 0; p < dx; p++) {
                                uint32_t y = Nx[p];
                                uint32_t py = (uint32_t)lower_bound_u32(C, d, y);
                                if (!(py < d && C[py] == y)) continue;
                                unsigned hits = 0;
                                for (uint32_t q = W.rsplit[y] + lane; q < W.roff[y + 1]; q += 32) {
                                    uint32_t z = W.radj[q];
                                    uint32_t pz = (uint32_t)lower_bound_u32(C, d, z);
                                    if (!(pz < d && C[pz] == z)) continue;
                                    uint32_t qx = (uint32_t)lower_bound_u32(Nx, dx, z);
                                    if (qx < dx && Nx[qx] == z) { atomicAdd(&cnt[pz], 1u); hits++; }
                                }
                                hits = __reduce_add_sync(0xffffffffu, hits);
                                if (lane == 0 && hits) {
                                    atomicAdd(&cnt[i], hits);
                                    atomicAdd(&cnt[py], hits);
                                }
                                tot += hits;
                            }
                        }
                    }
                    __syncwarp();
                    if (tot)
                        for (uint32_t i = lane; i < d; i += 32)
                            if (cnt[i]) atomicAdd(&W.deg[C[i]], (unsigned long long)cnt[i]);
                    if (lane == 0 && tot) {
                        atomicAdd(&W.deg[u], tot);
                        mu_loc += tot;
                    }
                    __syncwarp();
                }
            }
            mu = bsum<NT>(mu_loc, S.red);
            // ---- (k,Psi)-core peel on the ranked graph
            BPeel B;
            B.off = W.roff;
            B.adj = W.radj;
            B.nplus = W.rsplit;
            B.n = n;
            B.h = D.h;
            B.deg = W.deg;
            B.core = W.core;
            B.rnd = nullptr;
            B.st = W.st;
            B.alive = W.alive;
            B.fa = W.fa;
            B.fb = W.fb;
            B.lk = W.lk;
            B.lm = W.lm;
            B.ls = W.ls;
            B.mu0 = mu;
            kmax = block_peel<NT, LPR>(B, S, &nl);
            // core numbers back to caller ids (k1 as 64-bit scratch is not
            // needed: write through old_of)
            for (uint32_t i = threadIdx.x; i < n; i += NT) W.deg[W.old_of[i]] = W.core[i];
            __syncthreads();
            corev = W.deg;
        }
        // ---- outputs: densest level (ties to larger k), k_max level
        {
            uint32_t best = 0xffffffffu;
            for (uint32_t j = threadIdx.x; j < nl; j += NT)
                if (best == 0xffffffffu || bratio_ge(W.lm[j], W.ls[j], W.lm[best], W.ls[best])) best = j;
            // block argmax with the same tie rule (larger index on ties)
            __shared__ uint32_t s_best[NT];
            s_best[threadIdx.x] = best;
            __syncthreads();
            if (threadIdx.x == 0) {
                uint32_t bb = 0xffffffffu;
                for (int t = 0; t < NT; t++) {
                    uint32_t j = s_best[t];
                    if (j == 0xffffffffu) continue;
                    if (bb == 0xffffffffu) { bb = j; continue; }
                    bool ge = bratio_ge(W.lm[j], W.ls[j], W.lm[bb], W.ls[bb]);
                    bool le = bratio_ge(W.lm[bb], W.ls[bb], W.lm[j], W.ls[j]);
                    if ((ge && !le) || (ge && le && j > bb)) bb = j;
                }
                R.mu = mu;
                R.nlevels = nl;
                if (nl) {
                    R.kmax = W.lk[nl - 1];
                    R.kmax_core_size = W.ls[nl - 1];
                    R.kmax_core_mu = W.lm[nl - 1];
                    R.best_k = W.lk[bb];
                    R.densest_size = W.ls[bb];
                    R.densest_mu = W.lm[bb];
                }
                R.status = kBOk;
                A.res[gi] = R;
            }
            (void)kmax;
        }
        if (A.cores && D.core_off != ~0ull)
            for (uint32_t v = threadIdx.x; v < n; v += NT) A.cores[D.core_off + v] = corev[v];
        __syncthreads();
    }
}

}  // namespace
}  // namespace dsd

#include "batch_host.inc"
