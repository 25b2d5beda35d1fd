// Pattern densities (Sec. 6) for two special patterns on the GPU: the x-star
// (a centre and x of its neighbours, x = 2..8) and the 4-vertex loop
// (4-cycle).  Instances need not be induced: every injective map of the
// pattern whose edges land on graph edges, up to the pattern's symmetries.
//
// Pattern-degrees by the closed forms of the appendix on special patterns,
// on the alive subgraph (d(.) = alive degree):
//   x-star: deg(v) = C(d(v), x) + sum_{u in N(v)} C(d(u) - 1, x - 1)
//           (v as the centre, plus v as a leaf of each neighbour u);
//   loop:   deg(v) = sum_{w != v} C(c(v, w), 2), c(v, w) = alive common
//           neighbours (a loop through v is v, w opposite, and two of their
//           common neighbours).
// mu = sum deg / |V_Psi| (|V_Psi| = x + 1 or 4).
//
// (k,Psi)-cores by level-synchronous peeling: k <- max(k, least alive
// degree); every alive vertex with degree <= k leaves at level k; the
// degrees of the alive vertices within two hops of them are recounted;
// repeat.  Pattern-degrees only fall when
// vertices leave, so the vertices leaving at level k are exactly
// R_k \ R_{k+1} and the core numbers equal Algorithm 3's; the alive set at
// the first round of a level k is R_k (level records for CoreApp's
// outputs).  Recounts use the same closed forms as the first count: exact.
// The level k and the level records live on the device; the host launches
// rounds in batches and reads back only to see whether anything is alive.
//
// Every kernel reads and writes library-owned device buffers only; results
// reach the caller through cudaMemcpyAsync.
#include "graph.cuh"

#include <string.h>
#include <vector>

namespace dsd {
namespace {

constexpr int kStar = DSD_PATTERN_STAR;
constexpr int kLoop = DSD_PATTERN_LOOP4;

unsigned pgrid(uint64_t n, unsigned per_block = 256) {
    uint64_t b = (n + per_block - 1) / per_block;
    return (unsigned)(b < 1 ? 1 : (b > 152 * 16 ? 152 * 16 : b));
}

// C(a, b) with the product kept exact step by step (a (a-1) ... / b!).
__device__ __forceinline__ unsigned long long binom(unsigned long long a, int b) {
    if (b < 0 || a < (unsigned long long)b) return 0;
    unsigned long long c = 1;
    for (int t = 1; t <= b; t++) c = c * (a - (unsigned long long)b + (unsigned long long)t) / t;
    return c;
}

// Alive degree of every vertex (0 for vertices that left).  Warp per vertex.
__global__ void k_alive_deg(uint32_t n, const uint64_t* off, const uint32_t* adj,
                            const uint8_t* alive, uint32_t* dal) {
    uint64_t gw = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    unsigned lane = lane_id();
    for (uint64_t v = gw; v < n; v += nw) {
        unsigned c = 0;
        if (alive[v])
            for (uint64_t p = off[v] + lane; p < off[v + 1]; p += 32) c += alive[adj[p]];
        c = warp_sum(c);
        if (lane == 0) dal[v] = c;
    }
}

// x-star degrees.  Warp per vertex.
__global__ void k_star_deg(uint32_t n, const uint64_t* off, const uint32_t* adj,
                           const uint8_t* alive, const uint32_t* dal, int x,
                           unsigned long long* deg) {
    uint64_t gw = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    unsigned lane = lane_id();
    for (uint64_t v = gw; v < n; v += nw) {
        unsigned long long s = 0;
        if (alive[v]) {
            for (uint64_t p = off[v] + lane; p < off[v + 1]; p += 32) {
                uint32_t u = adj[p];
                if (alive[u]) s += binom((unsigned long long)dal[u] - 1, x - 1);
            }
        }
        s = warp_sum(s);
        if (lane == 0) deg[v] = alive[v] ? s + binom(dal[v], x) : 0ull;
    }
}

// 4-loop degrees.  Block per vertex v with a private counter row cnt[0..n)
// (zero on entry and on exit): every alive 2-path v - a - w (w != v) adds
// the number of earlier 2-paths to the same w, which sums C(c(v, w), 2).
__global__ void k_loop_deg(uint32_t n, const uint64_t* off, const uint32_t* adj,
                           const uint8_t* alive, uint32_t* cnt_all,
                           unsigned long long* deg) {
    __shared__ unsigned long long s_sum[32];
    uint32_t* cnt = cnt_all + (uint64_t)blockIdx.x * n;
    const unsigned nwarp = blockDim.x >> 5, warp = warp_id(), lane = lane_id();
    for (uint64_t v = blockIdx.x; v < n; v += gridDim.x) {
        if (!alive[v]) {
            if (threadIdx.x == 0) deg[v] = 0;
            continue;
        }
        unsigned long long s = 0;
        // warps over the alive neighbours a, lanes over N(a)
        for (uint64_t p = off[v] + warp; p < off[v + 1]; p += nwarp) {
            uint32_t a = adj[p];
            if (!alive[a]) continue;
            for (uint64_t q = off[a] + lane; q < off[a + 1]; q += 32) {
                uint32_t w = adj[q];
                if (w != v && alive[w]) s += atomicAdd(&cnt[w], 1u);
            }
        }
        s = warp_sum(s);
        if (lane == 0) s_sum[warp] = s;
        __syncthreads();
        // reset the touched counters
        for (uint64_t p = off[v] + warp; p < off[v + 1]; p += nwarp) {
            uint32_t a = adj[p];
            if (!alive[a]) continue;
            for (uint64_t q = off[a] + lane; q < off[a + 1]; q += 32) cnt[adj[q]] = 0;
        }
        if (threadIdx.x == 0) {
            unsigned long long t = 0;
            for (unsigned i = 0; i < nwarp; i++) t += s_sum[i];
            deg[v] = t;
        }
        __syncthreads();
    }
}

// Per round: out[0] = least alive degree (~0 if none), out[1] = alive count,
// out[2] = sum of alive degrees.
__global__ void k_round_stats(uint32_t n, const uint8_t* alive, const unsigned long long* deg,
                              unsigned long long* out) {
    unsigned long long mn = ~0ull, cnt = 0, sum = 0;
    for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (uint64_t)gridDim.x * blockDim.x)
        if (alive[v]) {
            mn = deg[v] < mn ? deg[v] : mn;
            cnt++;
            sum += deg[v];
        }
    mn = warp_min_u64(mn);
    cnt = warp_sum(cnt);
    sum = warp_sum(sum);
    if (lane_id() == 0) {
        if (mn != ~0ull) atomicMin(&out[0], mn);
        if (cnt) atomicAdd(&out[1], cnt);
        if (sum) atomicAdd(&out[2], sum);
    }
}

__global__ void k_fill_u8(uint32_t n, uint8_t* a, uint8_t val) {
    for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (uint64_t)gridDim.x * blockDim.x)
        a[v] = val;
}

__global__ void k_flag_ge(uint32_t n, const unsigned long long* core, unsigned long long k,
                          uint32_t* flag) {
    for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (uint64_t)gridDim.x * blockDim.x)
        flag[v] = core[v] >= k ? 1u : 0u;
}

__global__ void k_compact_ids(uint32_t n, const uint32_t* flag, const uint64_t* pos,
                              uint32_t* out) {
    for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (uint64_t)gridDim.x * blockDim.x)
        if (flag[v]) out[pos[v]] = (uint32_t)v;
}

__device__ __forceinline__ void warp_push(bool add, uint32_t x, uint32_t* out, uint32_t* n) {
    unsigned b = __ballot_sync(0xffffffffu, add);
    if (!b) return;
    int leader = __ffs(b) - 1;
    uint32_t base = 0;
    if ((int)lane_id() == leader) base = atomicAdd(n, (uint32_t)__popc(b));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (add) out[base + __popc(b & ((1u << lane_id()) - 1u))] = x;
}

// Retire the level's frontier (core = k) and list it.
__global__ void k_retire_list(uint32_t n, uint8_t* alive, const unsigned long long* deg,
                              const unsigned long long* st, unsigned long long* core,
                              uint32_t* lf, uint32_t* nf) {
    const unsigned long long k = st[3];
    for (uint64_t x0 = (uint64_t)blockIdx.x * blockDim.x; x0 < n;
         x0 += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t v = x0 + threadIdx.x;
        bool r = v < n && alive[v] && deg[v] <= k;
        if (r) {
            core[v] = k;
            alive[v] = 0;
        }
        warp_push(r, (uint32_t)v, lf, nf);
    }
}

// Alive neighbours of the listed vertices, each listed once per round
// (stamp = round + 1).  Warp per listed vertex.
__global__ void k_touch(const uint32_t* lin, const uint32_t* nin, const uint64_t* off,
                        const uint32_t* adj, const uint8_t* alive, uint32_t* stamp,
                        uint32_t mark, uint32_t* lout, uint32_t* nout) {
    uint64_t gw = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    const uint32_t n = *nin;
    for (uint64_t i = gw; i < n; i += nw) {
        const uint32_t x = lin[i];
        for (uint64_t p0 = off[x]; p0 < off[x + 1]; p0 += 32) {
            uint64_t p = p0 + lane_id();
            bool add = false;
            uint32_t a = 0;
            if (p < off[x + 1]) {
                a = adj[p];
                add = alive[a] && atomicMax(&stamp[a], mark) < mark;
            }
            warp_push(add, a, lout, nout);
        }
    }
}

// The listed vertices themselves, each once per round.
__global__ void k_add(const uint32_t* lin, const uint32_t* nin, uint32_t* stamp, uint32_t mark,
                      uint32_t* lout, uint32_t* nout) {
    const uint32_t n = *nin;
    for (uint64_t x0 = (uint64_t)blockIdx.x * blockDim.x; x0 < n;
         x0 += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t i = x0 + threadIdx.x;
        uint32_t a = i < n ? lin[i] : 0u;
        bool add = i < n && atomicMax(&stamp[a], mark) < mark;
        warp_push(add, a, lout, nout);
    }
}

// Alive degree of the listed (alive) vertices.  Warp per entry.
__global__ void k_alive_deg_list(const uint32_t* list, const uint32_t* nl, const uint64_t* off,
                                 const uint32_t* adj, const uint8_t* alive, uint32_t* dal) {
    uint64_t gw = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    unsigned lane = lane_id();
    const uint32_t n = *nl;
    for (uint64_t i = gw; i < n; i += nw) {
        const uint32_t v = list[i];
        unsigned c = 0;
        for (uint64_t p = off[v] + lane; p < off[v + 1]; p += 32) c += alive[adj[p]];
        c = warp_sum(c);
        if (lane == 0) dal[v] = c;
    }
}

// x-star degrees of the listed (alive) vertices.  Warp per entry.
__global__ void k_star_deg_list(const uint32_t* list, const uint32_t* nl, const uint64_t* off,
                                const uint32_t* adj, const uint8_t* alive, const uint32_t* dal,
                                int x, unsigned long long* deg) {
    uint64_t gw = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    unsigned lane = lane_id();
    const uint32_t n = *nl;
    for (uint64_t i = gw; i < n; i += nw) {
        const uint32_t v = list[i];
        unsigned long long sum = 0;
        for (uint64_t p = off[v] + lane; p < off[v + 1]; p += 32) {
            uint32_t u = adj[p];
            if (alive[u]) sum += binom((unsigned long long)dal[u] - 1, x - 1);
        }
        sum = warp_sum(sum);
        if (lane == 0) deg[v] = sum + binom(dal[v], x);
    }
}

// 4-loop degrees of the listed (alive) vertices (see k_loop_deg).  Block per
// entry.
__global__ void k_loop_deg_list(const uint32_t* list, const uint32_t* nl, uint32_t n,
                                const uint64_t* off, const uint32_t* adj, const uint8_t* alive,
                                uint32_t* cnt_all, unsigned long long* deg) {
    __shared__ unsigned long long s_sum[32];
    uint32_t* cnt = cnt_all + (uint64_t)blockIdx.x * n;
    const unsigned nwarp = blockDim.x >> 5, warp = warp_id(), lane = lane_id();
    const uint32_t m = *nl;
    for (uint64_t i = blockIdx.x; i < m; i += gridDim.x) {
        const uint32_t v = list[i];
        unsigned long long sum = 0;
        for (uint64_t p = off[v] + warp; p < off[v + 1]; p += nwarp) {
            uint32_t a = adj[p];
            if (!alive[a]) continue;
            for (uint64_t q = off[a] + lane; q < off[a + 1]; q += 32) {
                uint32_t w = adj[q];
                if (w != v && alive[w]) sum += atomicAdd(&cnt[w], 1u);
            }
        }
        sum = warp_sum(sum);
        if (lane == 0) s_sum[warp] = sum;
        __syncthreads();
        for (uint64_t p = off[v] + warp; p < off[v + 1]; p += nwarp) {
            uint32_t a = adj[p];
            if (!alive[a]) continue;
            for (uint64_t q = off[a] + lane; q < off[a + 1]; q += 32) cnt[adj[q]] = 0;
        }
        if (threadIdx.x == 0) {
            unsigned long long t = 0;
            for (unsigned w = 0; w < nwarp; w++) t += s_sum[w];
            deg[v] = t;
        }
        __syncthreads();
    }
}

// Device-side round state: st[0..2] the round's statistics (see
// k_round_stats), st[3] the current level k, st[4] the number of level
// records, st[5] 1 while no level has started, st[6] 1 once nothing is alive.
__global__ void k_stats_reset(unsigned long long* st) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        st[0] = ~0ull;
        st[1] = 0;
        st[2] = 0;
    }
}

// After the statistics: stop when nothing is alive; else k = max(k, least
// degree) and, when a level starts, its record (k, |R_k|, mu(R_k)).
__global__ void k_level(unsigned long long* st, int vs, unsigned long long* lk,
                        uint32_t* ls, unsigned long long* lm) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    if (st[1] == 0) {
        st[6] = 1;
        return;
    }
    const unsigned long long mn = st[0];
    if (st[5] || mn > st[3]) {
        const unsigned long long k = st[5] ? mn : (mn > st[3] ? mn : st[3]);
        const unsigned long long j = st[4];
        lk[j] = k;
        ls[j] = (uint32_t)st[1];
        lm[j] = st[2] / (unsigned long long)vs;
        st[4] = j + 1;
        st[3] = k;
        st[5] = 0;
    }
}

int pattern_size(int pattern, int x) { return pattern == kStar ? x + 1 : 4; }

dsd_status check_args(const dsd_graph* g, int pattern, int x, int mem) {
    if (!g) {
        set_error("graph handle is NULL");
        return DSD_ERR_INVALID;
    }
    if (pattern == kStar ? (x < 2 || x > 8) : pattern != kLoop) {
        set_error("pattern %d with x = %d: expected the x-star (x = 2..8) or the 4-loop",
                  pattern, x);
        return DSD_ERR_INVALID;
    }
    if (mem != DSD_MEM_HOST && mem != DSD_MEM_DEVICE) {
        set_error("invalid memory kind %d", mem);
        return DSD_ERR_INVALID;
    }
    return DSD_OK;
}

// Device working set of one pattern computation.
struct PatWork {
    uint8_t* alive = nullptr;
    uint32_t* dal = nullptr;
    unsigned long long* deg = nullptr;
    unsigned long long* core = nullptr;
    unsigned long long* stats = nullptr;
    uint32_t* cnt = nullptr;          // loop counters: blocks x n
    unsigned loop_blocks = 0;
    uint32_t* stamp1 = nullptr;       // per-round marks (round + 1)
    uint32_t* stamp2 = nullptr;
    uint32_t* lf = nullptr;           // the round's frontier
    uint32_t* l1 = nullptr;           // alive vertices next to it
    uint32_t* lt = nullptr;           // alive vertices within two hops of it
    uint32_t* ln = nullptr;           // lengths of lf, l1, lt
    unsigned long long* lvk = nullptr;   // level records on the device
    uint32_t* lvs = nullptr;
    unsigned long long* lvm = nullptr;
};

void pat_free(PatWork* w, cudaStream_t s) {
    void* ptrs[] = {w->alive, w->dal, w->deg, w->core, w->stats, w->cnt,
                    w->stamp1, w->stamp2, w->lf, w->l1, w->lt, w->ln,
                    w->lvk, w->lvs, w->lvm};
    for (void* p : ptrs) dev_free(p, s);
    *w = PatWork();
}

dsd_status pat_alloc(PatWork* w, uint32_t n, int pattern, cudaStream_t s) {
    DSD_TRY(dalloc(&w->alive, (size_t)n + 1, s));
    DSD_TRY(dalloc(&w->dal, (size_t)n + 1, s));
    DSD_TRY(dalloc(&w->deg, (size_t)n + 1, s));
    DSD_TRY(dalloc(&w->core, (size_t)n + 1, s));
    DSD_TRY(dalloc(&w->stats, 8, s));
    DSD_TRY(dalloc(&w->lvk, (size_t)n + 1, s));
    DSD_TRY(dalloc(&w->lvs, (size_t)n + 1, s));
    DSD_TRY(dalloc(&w->lvm, (size_t)n + 1, s));
    DSD_TRY(dalloc(&w->stamp1, (size_t)n + 1, s));
    DSD_TRY(dalloc(&w->stamp2, (size_t)n + 1, s));
    DSD_TRY(dalloc(&w->lf, (size_t)n + 1, s));
    DSD_TRY(dalloc(&w->l1, (size_t)n + 1, s));
    DSD_TRY(dalloc(&w->lt, (size_t)n + 1, s));
    DSD_TRY(dalloc(&w->ln, 4, s));
    DSD_CU(cudaMemsetAsync(w->stamp1, 0, ((size_t)n + 1) * 4, s));
    DSD_CU(cudaMemsetAsync(w->stamp2, 0, ((size_t)n + 1) * 4, s));
    if (pattern == kLoop && n) {
        // one counter row per block, at most ~1 GiB of rows
        uint64_t rows = (1ull << 28) / ((uint64_t)n + 1);
        if (rows > 152 * 4) rows = 152 * 4;
        if (rows < 1) rows = 1;
        w->loop_blocks = (unsigned)rows;
        DSD_TRY(dalloc(&w->cnt, rows * (uint64_t)n, s));
        DSD_CU(cudaMemsetAsync(w->cnt, 0, rows * (uint64_t)n * 4, s));
    }
    return DSD_OK;
}

// Pattern-degrees of the alive vertices into w->deg.
dsd_status degrees(dsd_graph* g, int pattern, int x, PatWork* w) {
    cudaStream_t s = g->stream;
    const uint32_t n = g->n;
    if (!n) return DSD_OK;
    k_alive_deg<<<pgrid((uint64_t)n * 32), 256, 0, s>>>(n, g->off, g->adj, w->alive, w->dal);
    note_launch();
    if (pattern == kStar) {
        k_star_deg<<<pgrid((uint64_t)n * 32), 256, 0, s>>>(n, g->off, g->adj, w->alive, w->dal,
                                                          x, w->deg);
    } else {
        k_loop_deg<<<w->loop_blocks, 256, 0, s>>>(n, g->off, g->adj, w->alive, w->cnt, w->deg);
    }
    note_launch();
    DSD_LAUNCHED();
    return DSD_OK;
}

struct Levels {
    std::vector<uint64_t> k, mu;
    std::vector<uint32_t> size;
};

// Level-synchronous decomposition; w->core holds the core numbers.
dsd_status decompose(dsd_graph* g, int pattern, int x, PatWork* w, Levels* L, uint64_t* kmax) {
    cudaStream_t s = g->stream;
    const uint32_t n = g->n;
    const int vs = pattern_size(pattern, x);
    L->k.clear();
    L->mu.clear();
    L->size.clear();
    *kmax = 0;
    if (!n) return DSD_OK;
    k_fill_u8<<<pgrid(n), 256, 0, s>>>(n, w->alive, 1); note_launch();
    DSD_TRY(degrees(g, pattern, x, w));
    // st[3] = k = 0, st[4] = 0 records, st[5] = 1 (no level yet), st[6] = 0
    const unsigned long long init[8] = {0, 0, 0, 0, 0, 1, 0, 0};
    DSD_CU(cudaMemcpyAsync(w->stats, init, sizeof(init), cudaMemcpyHostToDevice, s));
    const unsigned gw = 152 * 8;
    // rounds run on the device state without a readback; the host checks
    // for the end every kBatch rounds (rounds after the end do nothing)
    constexpr uint32_t kBatch = 32;
    unsigned long long st[8];
    for (uint32_t round = 0;; round++) {
        if (round > n + kBatch) {
            set_error("pattern peel did not settle");
            return DSD_ERR_INTERNAL;
        }
        k_stats_reset<<<1, 32, 0, s>>>(w->stats);
        k_round_stats<<<pgrid(n), 256, 0, s>>>(n, w->alive, w->deg, w->stats);
        k_level<<<1, 32, 0, s>>>(w->stats, vs, w->lvk, w->lvs, w->lvm);
        // retire the frontier; only the alive vertices within two hops of it
        // can lose instances (every instance through one of them and a
        // frontier vertex spans at most two edges from it), so only they
        // are recounted: l1 = alive neighbours of the frontier, lt = l1 plus
        // their alive neighbours
        const uint32_t mark = round + 1;
        DSD_CU(cudaMemsetAsync(w->ln, 0, 16, s));
        k_retire_list<<<pgrid(n), 256, 0, s>>>(n, w->alive, w->deg, w->stats, w->core, w->lf,
                                               w->ln);
        k_touch<<<gw, 256, 0, s>>>(w->lf, w->ln, g->off, g->adj, w->alive, w->stamp1, mark, w->l1,
                                   w->ln + 1);
        k_add<<<pgrid(n), 256, 0, s>>>(w->l1, w->ln + 1, w->stamp2, mark, w->lt, w->ln + 2);
        k_touch<<<gw, 256, 0, s>>>(w->l1, w->ln + 1, g->off, g->adj, w->alive, w->stamp2, mark,
                                   w->lt, w->ln + 2);
        for (int i = 0; i < 7; i++) note_launch();
        if (pattern == kStar) {
            k_alive_deg_list<<<gw, 256, 0, s>>>(w->l1, w->ln + 1, g->off, g->adj, w->alive, w->dal);
            k_star_deg_list<<<gw, 256, 0, s>>>(w->lt, w->ln + 2, g->off, g->adj, w->alive, w->dal,
                                               x, w->deg);
            note_launch();
            note_launch();
        } else {
            k_loop_deg_list<<<w->loop_blocks, 256, 0, s>>>(w->lt, w->ln + 2, n, g->off, g->adj,
                                                           w->alive, w->cnt, w->deg);
            note_launch();
        }
        DSD_LAUNCHED();
        if ((round + 1) % kBatch == 0) {
            DSD_CU(cudaMemcpyAsync(st, w->stats, sizeof(st), cudaMemcpyDeviceToHost, s));
            DSD_CU(cudaStreamSynchronize(s));
            if (st[6]) break;
        }
    }
    const uint32_t nl = (uint32_t)st[4];
    L->k.resize(nl);
    L->size.resize(nl);
    L->mu.resize(nl);
    if (nl) {
        DSD_CU(cudaMemcpyAsync(L->k.data(), w->lvk, (size_t)nl * 8, cudaMemcpyDeviceToHost, s));
        DSD_CU(cudaMemcpyAsync(L->size.data(), w->lvs, (size_t)nl * 4, cudaMemcpyDeviceToHost, s));
        DSD_CU(cudaMemcpyAsync(L->mu.data(), w->lvm, (size_t)nl * 8, cudaMemcpyDeviceToHost, s));
        DSD_CU(cudaStreamSynchronize(s));
    }
    *kmax = st[3];
    return DSD_OK;
}

// The vertices with core >= thr, ascending, into out (host or device).
dsd_status emit_set(dsd_graph* g, const unsigned long long* core, uint64_t thr, uint32_t* out,
                    int mem, uint32_t* size_out) {
    cudaStream_t s = g->stream;
    const uint32_t n = g->n;
    uint32_t* flag = nullptr;
    uint32_t* ids = nullptr;
    uint64_t* pos = nullptr;
    uint64_t total = 0;
    dsd_status st = dalloc(&flag, (size_t)n + 1, s);
    if (st == DSD_OK) st = dalloc(&pos, (size_t)n + 1, s);
    if (st == DSD_OK) st = dalloc(&ids, (size_t)n + 1, s);
    if (st == DSD_OK) {
        k_flag_ge<<<pgrid(n), 256, 0, s>>>(n, core, thr, flag); note_launch();
        st = exclusive_scan_u32_to_u64(flag, pos, n, s);
    }
    if (st == DSD_OK) {
        k_compact_ids<<<pgrid(n), 256, 0, s>>>(n, flag, pos, ids); note_launch();
        cudaError_t e = cudaMemcpyAsync(&total, pos + n, 8, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e == cudaSuccess && out && total)
            e = cudaMemcpyAsync(out, ids, total * 4,
                                mem == DSD_MEM_HOST ? cudaMemcpyDeviceToHost
                                                    : cudaMemcpyDeviceToDevice, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) st = cuda_fail(e, "pattern set", __FILE__, __LINE__);
    }
    dev_free(flag, s);
    dev_free(pos, s);
    dev_free(ids, s);
    *size_out = (uint32_t)total;
    return st;
}

dsd_status copy_to(void* dst, const void* src, size_t bytes, int mem, cudaStream_t s) {
    if (!dst || !bytes) return DSD_OK;
    DSD_CU(cudaMemcpyAsync(dst, src, bytes,
                           mem == DSD_MEM_HOST ? cudaMemcpyDeviceToHost
                                               : cudaMemcpyDeviceToDevice, s));
    DSD_CU(cudaStreamSynchronize(s));
    return DSD_OK;
}

}  // namespace
}  // namespace dsd

using namespace dsd;

extern "C" {

dsd_status dsd_pattern_degrees(dsd_graph* g, int pattern, int x, uint64_t* deg, uint64_t* mu,
                               int mem) {
    set_error("");
    DSD_TRY(check_args(g, pattern, x, mem));
    cudaStream_t s = g->stream;
    const uint32_t n = g->n;
    PatWork w;
    dsd_status st = pat_alloc(&w, n, pattern, s);
    unsigned long long hs[3] = {0, 0, 0};
    if (st == DSD_OK && n) {
        k_fill_u8<<<pgrid(n), 256, 0, s>>>(n, w.alive, 1); note_launch();
        st = degrees(g, pattern, x, &w);
    }
    if (st == DSD_OK && n) {
        unsigned long long init[3] = {~0ull, 0ull, 0ull};
        cudaError_t e = cudaMemcpyAsync(w.stats, init, sizeof(init), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) {
            k_round_stats<<<pgrid(n), 256, 0, s>>>(n, w.alive, w.deg, w.stats); note_launch();
            e = cudaMemcpyAsync(hs, w.stats, sizeof(hs), cudaMemcpyDeviceToHost, s);
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) st = cuda_fail(e, "pattern degrees", __FILE__, __LINE__);
    }
    if (st == DSD_OK) st = copy_to(deg, w.deg, (size_t)n * 8, mem, s);
    const uint64_t m = hs[2] / (uint64_t)pattern_size(pattern, x);
    if (st == DSD_OK && mu) {
        if (mem == DSD_MEM_HOST) {
            *mu = m;
        } else {
            cudaError_t e = cudaMemcpyAsync(mu, &m, 8, cudaMemcpyHostToDevice, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) st = cuda_fail(e, "pattern mu", __FILE__, __LINE__);
        }
    }
    pat_free(&w, s);
    return st;
}

dsd_status dsd_pattern_core_decompose(dsd_graph* g, int pattern, int x, uint64_t* core,
                                      uint64_t* kmax, uint64_t* level_k, uint32_t* level_size,
                                      uint64_t* level_mu, uint32_t cap, uint32_t* nlevels,
                                      int mem) {
    set_error("");
    DSD_TRY(check_args(g, pattern, x, mem));
    cudaStream_t s = g->stream;
    PatWork w;
    Levels L;
    uint64_t km = 0;
    dsd_status st = pat_alloc(&w, g->n, pattern, s);
    if (st == DSD_OK) st = decompose(g, pattern, x, &w, &L, &km);
    if (st == DSD_OK) st = copy_to(core, w.core, (size_t)g->n * 8, mem, s);
    pat_free(&w, s);
    DSD_TRY(st);
    // small host-side records, written to the caller's memory per mem
    const uint32_t nl = (uint32_t)L.k.size();
    const uint32_t c = nl < cap ? nl : cap;
    if (mem == DSD_MEM_HOST) {
        if (kmax) *kmax = km;
        if (nlevels) *nlevels = nl;
        if (c && level_k) memcpy(level_k, L.k.data(), (size_t)c * 8);
        if (c && level_size) memcpy(level_size, L.size.data(), (size_t)c * 4);
        if (c && level_mu) memcpy(level_mu, L.mu.data(), (size_t)c * 8);
    } else {
        if (kmax) DSD_CU(cudaMemcpyAsync(kmax, &km, 8, cudaMemcpyHostToDevice, s));
        if (nlevels) DSD_CU(cudaMemcpyAsync(nlevels, &nl, 4, cudaMemcpyHostToDevice, s));
        if (c && level_k) DSD_CU(cudaMemcpyAsync(level_k, L.k.data(), (size_t)c * 8,
                                                 cudaMemcpyHostToDevice, s));
        if (c && level_size) DSD_CU(cudaMemcpyAsync(level_size, L.size.data(), (size_t)c * 4,
                                                    cudaMemcpyHostToDevice, s));
        if (c && level_mu) DSD_CU(cudaMemcpyAsync(level_mu, L.mu.data(), (size_t)c * 8,
                                                  cudaMemcpyHostToDevice, s));
        DSD_CU(cudaStreamSynchronize(s));
    }
    if (nl > cap && (level_k || level_size || level_mu)) {
        set_error("%u levels exceed the capacity %u", nl, cap);
        return DSD_ERR_OVERFLOW;
    }
    return DSD_OK;
}

dsd_status dsd_pattern_core_app(dsd_graph* g, int pattern, int x, uint32_t* kmax_core,
                                uint32_t* densest, int mem, dsd_core_app_result* r) {
    set_error("");
    DSD_TRY(check_args(g, pattern, x, mem));
    if (!r) {
        set_error("result pointer is NULL");
        return DSD_ERR_INVALID;
    }
    cudaStream_t s = g->stream;
    const uint32_t n = g->n;
    PatWork w;
    Levels L;
    uint64_t km = 0;
    memset(r, 0, sizeof(*r));
    dsd_status st = pat_alloc(&w, n, pattern, s);
    if (st == DSD_OK) st = decompose(g, pattern, x, &w, &L, &km);
    if (st == DSD_OK && n) {
        const uint32_t nl = (uint32_t)L.k.size();
        uint32_t best = 0;
        for (uint32_t j = 1; j < nl; j++)   // densest level, ties to the larger k
            if ((unsigned __int128)L.mu[j] * L.size[best] >=
                (unsigned __int128)L.mu[best] * L.size[j])
                best = j;
        r->kmax = km;
        r->kmax_core_size = L.size[nl - 1];
        r->kmax_core_mu = L.mu[nl - 1];
        r->best_k = L.k[best];
        r->densest_size = L.size[best];
        r->densest_mu = L.mu[best];
        r->nlevels = nl;
        uint32_t sz = 0;
        if (kmax_core) st = emit_set(g, w.core, km, kmax_core, mem, &sz);
        if (st == DSD_OK && kmax_core && sz != r->kmax_core_size) {
            set_error("k_max core size %u differs from its level record %u", sz,
                      r->kmax_core_size);
            st = DSD_ERR_INTERNAL;
        }
        if (st == DSD_OK && densest) st = emit_set(g, w.core, r->best_k, densest, mem, &sz);
        if (st == DSD_OK && densest && sz != r->densest_size) {
            set_error("densest level size %u differs from its level record %u", sz,
                      r->densest_size);
            st = DSD_ERR_INTERNAL;
        }
    }
    pat_free(&w, s);
    return st;
}

}  // extern "C"
