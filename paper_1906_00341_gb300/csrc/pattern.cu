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
// degrees of the alive vertices within two hops of them are updated;
// repeat.  Pattern-degrees only fall when
// vertices leave, so the vertices leaving at level k are exactly
// R_k \ R_{k+1} and the core numbers equal Algorithm 3's; the alive set at
// the first round of a level k is R_k (level records for CoreApp's
// outputs).  Recounts use the same closed forms as the first count: exact.
// All rounds run in one cooperative launch whose phases -- statistics,
// level and retirement, the degree changes -- are separated by grid barriers
// with bounded waits.  The degree changes are exact differences, not
// recounts: for the x-star from the changed alive degrees, for the loop from
// the destroyed loops, each charged to its smallest-id frontier member.
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

// ------------------------------------------------------- persistent rounds
// All rounds in one cooperative launch (one block per SM): the phases of a
// round are separated by a grid barrier whose waits are bounded in time (a
// wait past the limit sets the error flag; every block then leaves at its
// next barrier).  The device-side round state (st, see k_level) is the same
// as the launch-per-phase path's.

struct PatCtrl {
    uint32_t bar_count;
    uint32_t bar_gen;
    uint32_t error;
    uint32_t rounds;
};

struct PatRun {
    uint32_t n;
    int pattern, x, vs;
    const uint64_t* off;
    const uint32_t* adj;
    uint8_t* alive;
    uint32_t* dal;
    unsigned long long* deg;
    unsigned long long* core;
    unsigned long long* st;
    unsigned long long* lvk;
    uint32_t* lvs;
    unsigned long long* lvm;
    uint32_t* stamp1;
    uint32_t* lf;
    uint32_t* l1;
    uint32_t* ln;
    uint32_t* gone;           // star: frontier neighbours lost this round
    uint32_t* cnt;
    uint32_t cnt_rows;        // blocks with a loop counter row
    PatCtrl* ctrl;
    uint64_t wait_ns;
};

__device__ bool pat_barrier(PatCtrl* c, uint64_t wait_ns) {
    __shared__ uint32_t s_err;
    __syncthreads();
    if (threadIdx.x == 0) {
        const uint64_t t_in = globaltimer_ns();
        volatile uint32_t* genp = &c->bar_gen;
        const uint32_t gen = *genp;
        __threadfence();
        const uint32_t arrived = atomicAdd(&c->bar_count, 1u) + 1u;
        if (arrived == gridDim.x) {
            c->bar_count = 0;
            __threadfence();
            atomicAdd(&c->bar_gen, 1u);
        } else {
            uint32_t spins = 0;
            while (*genp == gen) {
                if (((++spins) & 255u) == 0 && globaltimer_ns() - t_in > wait_ns) {
                    atomicOr(&c->error, 1u);
                    break;
                }
                if (*(volatile uint32_t*)&c->error) break;
            }
        }
        __threadfence();
        s_err = *(volatile uint32_t*)&c->error;
    }
    __syncthreads();
    return s_err == 0;
}

__global__ void __launch_bounds__(256) k_pattern_rounds(PatRun R) {
    __shared__ unsigned long long s_red[3][8];
    const unsigned lane = lane_id(), warp = warp_id();
    const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t nthreads = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t gwarp = tid >> 5, nwarps = nthreads >> 5;
    const uint32_t n = R.n;
    unsigned long long* st = R.st;
    for (uint32_t round = 0; round <= n; round++) {
        // ---- statistics of the alive vertices (st[0..2] are zero / ~0 here)
        {
            unsigned long long mn = ~0ull, cnt = 0, sum = 0;
            for (uint64_t v = tid; v < n; v += nthreads)
                if (R.alive[v]) {
                    mn = R.deg[v] < mn ? R.deg[v] : mn;
                    cnt++;
                    sum += R.deg[v];
                }
            mn = warp_min_u64(mn);
            cnt = warp_sum(cnt);
            sum = warp_sum(sum);
            if (lane == 0) {
                s_red[0][warp] = mn;
                s_red[1][warp] = cnt;
                s_red[2][warp] = sum;
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                for (unsigned w = 1; w < (blockDim.x >> 5); w++) {
                    mn = s_red[0][w] < s_red[0][0] ? s_red[0][w] : s_red[0][0];
                    s_red[0][0] = mn;
                    s_red[1][0] += s_red[1][w];
                    s_red[2][0] += s_red[2][w];
                }
                if (s_red[0][0] != ~0ull) atomicMin(&st[0], s_red[0][0]);
                if (s_red[1][0]) atomicAdd(&st[1], s_red[1][0]);
                if (s_red[2][0]) atomicAdd(&st[2], s_red[2][0]);
            }
            if (blockIdx.x == 0 && threadIdx.x < 3) R.ln[threadIdx.x] = 0;
        }
        if (!pat_barrier(R.ctrl, R.wait_ns)) return;
        // ---- level (every block decides alike from st); retire the frontier
        const unsigned long long amin = *(volatile unsigned long long*)&st[0];
        const unsigned long long acnt = *(volatile unsigned long long*)&st[1];
        const unsigned long long asum = *(volatile unsigned long long*)&st[2];
        if (acnt == 0) {
            if (tid == 0) {
                st[6] = 1;
                R.ctrl->rounds = round;
            }
            return;
        }
        const unsigned long long k0 = *(volatile unsigned long long*)&st[3];
        const bool fresh = *(volatile unsigned long long*)&st[5] != 0;
        unsigned long long k = k0;
        if (fresh || amin > k0) {
            k = fresh ? amin : (amin > k0 ? amin : k0);
            if (tid == 0) {
                const unsigned long long j = st[4];
                R.lvk[j] = k;
                R.lvs[j] = (uint32_t)acnt;
                R.lvm[j] = asum / (unsigned long long)R.vs;
            }
        }
        const uint32_t mark = round + 1;
        for (uint64_t x0 = (uint64_t)blockIdx.x * blockDim.x; x0 < n; x0 += nthreads) {
            const uint64_t v = x0 + threadIdx.x;
            bool r = v < n && R.alive[v] && R.deg[v] <= k;
            if (r) {
                R.core[v] = k;
                R.alive[v] = 0;
                R.stamp1[v] = mark;   // a frontier member of this round
            }
            warp_push(r, (uint32_t)v, R.lf, R.ln);
        }
        if (!pat_barrier(R.ctrl, R.wait_ns)) return;
        // ---- level state for the next round
        if (tid == 0) {
            if (fresh || amin > k0) {
                st[4] += 1;
                st[3] = k;
                st[5] = 0;
            }
            st[0] = ~0ull;
            st[1] = 0;
            st[2] = 0;
        }
        const uint32_t nf = *(volatile uint32_t*)&R.ln[0];
        if (R.pattern == kStar) {
            // x-star: deg(v) = C(d(v), x) + sum over alive neighbours u of
            // C(d(u) - 1, x - 1) depends only on alive degrees, so the
            // round's change is applied as exact differences:
            //   (a) every alive v next to a frontier vertex f loses f's term
            //       C(d(f) - 1, x - 1), and u = v counts its lost neighbours;
            //   (b) every such u (its degree d -> d') changes its own term
            //       by C(d', x) - C(d, x) and each alive neighbour's term by
            //       C(d' - 1, x - 1) - C(d - 1, x - 1).
            // Sums wrap modulo 2^64 like the counts themselves.
            for (uint64_t i = gwarp; i < nf; i += nwarps) {
                const uint32_t f = R.lf[i];
                const unsigned long long lost = binom((unsigned long long)R.dal[f] - 1, R.x - 1);
                for (uint64_t p0 = R.off[f]; p0 < R.off[f + 1]; p0 += 32) {
                    const uint64_t p = p0 + lane;
                    bool add = false;
                    uint32_t a = 0;
                    if (p < R.off[f + 1]) {
                        a = R.adj[p];
                        if (R.alive[a]) {
                            atomicAdd(&R.deg[a], 0ull - lost);
                            atomicAdd(&R.gone[a], 1u);
                            add = atomicMax(&R.stamp1[a], mark) < mark;
                        }
                    }
                    warp_push(add, a, R.l1, R.ln + 1);
                }
            }
            if (!pat_barrier(R.ctrl, R.wait_ns)) return;
            const uint32_t n1 = *(volatile uint32_t*)&R.ln[1];
            for (uint64_t i = gwarp; i < n1; i += nwarps) {
                const uint32_t u = R.l1[i];
                const unsigned long long d0 = R.dal[u], d1 = d0 - R.gone[u];
                const unsigned long long dn = binom(d1 - 1, R.x - 1) - binom(d0 - 1, R.x - 1);
                for (uint64_t p = R.off[u] + lane; p < R.off[u + 1]; p += 32) {
                    const uint32_t v = R.adj[p];
                    if (R.alive[v] && dn) atomicAdd(&R.deg[v], dn);
                }
                if (lane == 0) {
                    atomicAdd(&R.deg[u], binom(d1, R.x) - binom(d0, R.x));
                    R.dal[u] = (uint32_t)d1;
                    R.gone[u] = 0;
                }
            }
            if (!pat_barrier(R.ctrl, R.wait_ns)) return;
            continue;
        }
        // ---- 4-loop: every destroyed loop is charged once, to its
        // smallest-id frontier member f: from f, the loops f - a - w - b
        // whose other members are alive or larger frontier members.
        // Grouping the 2-paths f - a - w by w (c(w) of them), each alive a
        // loses c(w) - 1 loops and each alive w loses C(c(w), 2) -- the
        // appendix's decrements, made exact under simultaneous removal by
        // the single charge.  A block per frontier vertex, with its private
        // counter row (zero between uses).
        if (blockIdx.x < R.cnt_rows) {
            uint32_t* cnt = R.cnt + (uint64_t)blockIdx.x * n;
            const unsigned nwarp = blockDim.x >> 5;
            auto valid = [&](uint32_t y, uint32_t f) -> bool {
                return R.alive[y] || (R.stamp1[y] == mark && y > f);
            };
            for (uint64_t i = blockIdx.x; i < nf; i += R.cnt_rows) {
                const uint32_t f = R.lf[i];
                for (int pass = 0; pass < 3; pass++) {
                    for (uint64_t p = R.off[f] + warp; p < R.off[f + 1]; p += nwarp) {
                        const uint32_t a = R.adj[p];
                        if (!valid(a, f)) continue;
                        const bool a_alive = R.alive[a];
                        for (uint64_t q = R.off[a] + lane; q < R.off[a + 1]; q += 32) {
                            const uint32_t w = R.adj[q];
                            if (w == f || !valid(w, f)) continue;
                            if (pass == 0) {
                                atomicAdd(&cnt[w], 1u);
                            } else if (pass == 1) {
                                const uint32_t c = cnt[w];
                                if (a_alive && c > 1)
                                    atomicAdd(&R.deg[a], 0ull - (unsigned long long)(c - 1));
                            } else {
                                const uint32_t c = atomicExch(&cnt[w], 0u);
                                if (c > 1 && R.alive[w])
                                    atomicAdd(&R.deg[w],
                                              0ull - (unsigned long long)c * (c - 1) / 2);
                            }
                        }
                    }
                    __syncthreads();
                }
            }
        }
        if (!pat_barrier(R.ctrl, R.wait_ns)) return;
    }
    if (tid == 0) atomicOr(&R.ctrl->error, 2u);   // more rounds than vertices
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
    uint32_t* lf = nullptr;           // the round's frontier
    uint32_t* l1 = nullptr;           // alive vertices next to it
    uint32_t* ln = nullptr;           // lengths of lf, l1
    uint32_t* gone = nullptr;         // per vertex, zero between rounds
    unsigned long long* lvk = nullptr;   // level records on the device
    uint32_t* lvs = nullptr;
    unsigned long long* lvm = nullptr;
};

void pat_free(PatWork* w, cudaStream_t s) {
    void* ptrs[] = {w->alive, w->dal, w->deg, w->core, w->stats, w->cnt,
                    w->stamp1, w->lf, w->l1, w->ln, w->gone,
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
    DSD_TRY(dalloc(&w->lf, (size_t)n + 1, s));
    DSD_TRY(dalloc(&w->l1, (size_t)n + 1, s));
    DSD_TRY(dalloc(&w->ln, 4, s));
    DSD_TRY(dalloc(&w->gone, (size_t)n + 1, s));
    DSD_CU(cudaMemsetAsync(w->gone, 0, ((size_t)n + 1) * 4, s));
    DSD_CU(cudaMemsetAsync(w->stamp1, 0, ((size_t)n + 1) * 4, s));
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
    // st[0..2] the statistics (min ~0), st[3] = k = 0, st[4] = 0 records,
    // st[5] = 1 (no level yet), st[6] = 0
    const unsigned long long init[8] = {~0ull, 0, 0, 0, 0, 1, 0, 0};
    unsigned long long st[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    PatCtrl* ctrl = nullptr;
    DSD_TRY(dalloc(&ctrl, 1, s));
    int sms = 152;
    dsd_status rs = num_sms(&sms);
    int per_sm = 0;
    cudaError_t e = cudaSuccess;
    if (rs == DSD_OK) {
        e = cudaMemcpyAsync(w->stats, init, sizeof(init), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemsetAsync(ctrl, 0, sizeof(PatCtrl), s);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pattern_rounds, 256, 0);
        if (e == cudaSuccess && per_sm < 1) e = cudaErrorInvalidConfiguration;
    }
    PatCtrl hc;
    memset(&hc, 0, sizeof(hc));
    if (rs == DSD_OK && e == cudaSuccess) {
        PatRun R;
        R.n = n;
        R.pattern = pattern;
        R.x = x;
        R.vs = vs;
        R.off = g->off;
        R.adj = g->adj;
        R.alive = w->alive;
        R.dal = w->dal;
        R.deg = w->deg;
        R.core = w->core;
        R.st = w->stats;
        R.lvk = w->lvk;
        R.lvs = w->lvs;
        R.lvm = w->lvm;
        R.stamp1 = w->stamp1;
        R.lf = w->lf;
        R.l1 = w->l1;
        R.ln = w->ln;
        R.gone = w->gone;
        R.cnt = w->cnt;
        R.ctrl = ctrl;
        R.wait_ns = wait_limit_ns();
        // x-star: one block per SM (the fewest barrier arrivals); 4-loop: up
        // to 4 (its decrements run a block per frontier vertex)
        const unsigned per = pattern == kLoop ? (unsigned)(per_sm < 4 ? per_sm : 4) : 1u;
        const unsigned grid = (unsigned)sms * per;
        R.cnt_rows = pattern == kLoop ? (w->loop_blocks < grid ? w->loop_blocks : grid) : 0;
        void* args[] = {&R};
        e = cudaLaunchCooperativeKernel((void*)k_pattern_rounds, dim3(grid), dim3(256), args, 0, s);
        note_launch();
        if (e == cudaSuccess) e = cudaMemcpyAsync(&hc, ctrl, sizeof(hc), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(st, w->stats, sizeof(st), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    }
    dev_free(ctrl, s);
    DSD_TRY(rs);
    if (e != cudaSuccess) return cuda_fail(e, "pattern rounds", __FILE__, __LINE__);
    if (hc.error & 1u) {
        set_error("pattern peel: a grid barrier wait ran past the limit");
        return DSD_ERR_TIMEOUT;
    }
    if (hc.error || !st[6]) {
        set_error("pattern peel did not settle");
        return DSD_ERR_INTERNAL;
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
