// CoreExact (Algorithm 4, Sec. 4.3) on the GPU: the h-clique densest
// subgraph, exactly.
//
// Steps, each on the device:
//  1. the (k,Psi)-core decomposition and its densest level rho' (Algorithm 3,
//     Pruning1): every densest set lies in R_k1, k1 = ceil(rho') (each of its
//     vertices is in >= rho_opt of its cliques, Sec. 4.3);
//  2. connected components of G[R_k1] (hooking to the smaller root +
//     pointer jumping) and their densities; the densest component raises the
//     lower bound (Pruning2, k2 = ceil of its density);
//  3. the search for rho_opt on the located core R_ceil(alpha): one flow
//     network of Algorithm 1 built from the listed (h-1)-cliques and their
//     common neighbourhoods, and a minimum cut by parallel push-relabel with
//     global relabelling.  A cut at alpha = p/q (capacities scaled by q)
//     costs q h (mu(W) - mu(A)) + p h |A| for the vertex set A on its source
//     side, so the largest source side A of a minimum cut maximises
//     mu(A) - alpha |A|.  If A beats alpha, alpha <- rho(A) and the core
//     shrinks to R_ceil(alpha) (the network gets smaller as alpha grows,
//     Sec. 4.3); otherwise alpha = rho_opt and A is the union of all densest
//     sets.
// The components are not searched one by one: they are disjoint, so one
// network over the whole located core is the disjoint union of their
// networks and a single cut serves them all.  The search is Dinkelbach's
// iteration on exact rationals instead of a bisection with the
// 1/(|V_C|(|V_C|-1)) stop (Pruning3); it visits a strictly increasing
// sequence of densities of actual vertex sets and ends exactly at rho_opt.
#include "graph.cuh"

#include <chrono>
#include <string.h>
#include <vector>

namespace dsd {

const uint64_t* cached_core(const dsd_graph* g, int h);

namespace {

constexpr uint32_t kUnset = 0xffffffffu;
constexpr unsigned long long kInfCap = 1ull << 62;
enum : uint8_t { kArcRev = 0, kArcS = 1, kArcT = 2, kArcQ = 3, kArcInf = 4 };
// An arc's kind byte: its own kind (low 4 bits) and the kind of the forward
// arc of its pair (high 4 bits), so the pair's total capacity -- and with it
// the twin's residual, total minus this arc's residual -- is known locally.
__host__ __device__ constexpr uint8_t arc_kind(uint8_t own, uint8_t pair) {
    return (uint8_t)(own | (pair << 4));
}
// Arcs per node above which a block, not a warp, works on the node.
constexpr uint64_t kBigArcs = 2048;
constexpr int kBigThreads = 1024;

unsigned grid_for_n(uint64_t n, unsigned per_block = 256) {
    uint64_t b = (n + per_block - 1) / per_block;
    return (unsigned)(b < 1 ? 1 : (b > 152 * 16 ? 152 * 16 : b));
}

unsigned grid_for_warps(uint64_t warps) { return grid_for_n(warps * 32); }

__device__ __forceinline__ unsigned lanemask_lt() { return (1u << lane_id()) - 1u; }

// Appends x (where add) to out[] behind the counter *n, one atomic per warp.
// Every lane of the warp must call it.
__device__ __forceinline__ void warp_append(bool add, uint32_t x, uint32_t* out, uint32_t* n) {
    unsigned b = __ballot_sync(0xffffffffu, add);
    if (!b) return;
    int leader = __ffs(b) - 1;
    uint32_t base = 0;
    if ((int)lane_id() == leader) base = atomicAdd(n, (uint32_t)__popc(b));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (add) out[base + __popc(b & lanemask_lt())] = x;
}

__device__ __forceinline__ bool in_sorted(const uint32_t* a, uint64_t len, uint32_t x) {
    uint64_t p = lower_bound_u32(a, len, x);
    return p < len && a[p] == x;
}

// ------------------------------------------------------------ located core

__global__ void k_flag_core_ge(uint32_t n, const uint64_t* core, unsigned long long k,
                               uint32_t* flag) {
    for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (uint64_t)gridDim.x * blockDim.x)
        flag[v] = core[v] >= k ? 1u : 0u;
}

// ------------------------------------------------------ connected components
// parent[x] <= x always; a root is its own parent.  Hooking links the larger
// of two roots under the smaller one (atomicMin), so parents only decrease
// and every find terminates.

__global__ void k_cc_init(uint32_t n, uint32_t* parent) {
    for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (uint64_t)gridDim.x * blockDim.x)
        parent[v] = (uint32_t)v;
}

__device__ __forceinline__ uint32_t cc_find(const uint32_t* parent, uint32_t x) {
    uint32_t p = parent[x];
    while (p != x) {
        x = p;
        p = parent[x];
    }
    return x;
}

// Warp per vertex v; each edge (v, u), u < v, hooks the two roots.
__global__ void k_cc_hook(uint32_t n, const uint64_t* off, const uint32_t* adj,
                          uint32_t* parent, uint32_t* changed) {
    uint64_t gw = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    unsigned lane = lane_id();
    for (uint64_t v = gw; v < n; v += nw) {
        bool any = false;
        for (uint64_t p = off[v] + lane; p < off[v + 1]; p += 32) {
            uint32_t u = adj[p];
            if (u >= v) break;                    // rows ascend: the rest are > v
            uint32_t ru = cc_find(parent, u), rv = cc_find(parent, (uint32_t)v);
            if (ru != rv) {
                uint32_t hi = ru > rv ? ru : rv, lo = ru > rv ? rv : ru;
                atomicMin(&parent[hi], lo);
                any = true;
            }
        }
        if (__any_sync(0xffffffffu, any) && lane == 0) *changed = 1u;
    }
}

__global__ void k_cc_compress(uint32_t n, uint32_t* parent) {
    for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (uint64_t)gridDim.x * blockDim.x)
        parent[v] = cc_find(parent, (uint32_t)v);
}

// Per component (indexed by its root): sum of clique-degrees and size.
// deg is in the rank space of H, old_of maps rank -> H id.
__global__ void k_comp_sums(uint32_t nh, const uint32_t* old_of, const unsigned long long* deg,
                            const uint32_t* parent, unsigned long long* cdeg, uint32_t* csz) {
    for (uint64_t r = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; r < nh;
         r += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t root = parent[old_of[r]];
        atomicAdd(&cdeg[root], deg[r]);
        atomicAdd(&csz[root], 1u);
    }
}

__device__ __forceinline__ bool frac_gt(unsigned long long a, unsigned long long b,
                                        unsigned long long c, unsigned long long d) {
    // a/b > c/d (b, d > 0)
    return (unsigned __int128)a * d > (unsigned __int128)c * b;
}

// One block: the component of largest cdeg/csz and the number of components.
// out[0] = cdeg, out[1] = csz of the best, out[2] = components.
__global__ void k_best_comp(uint32_t nh, const unsigned long long* cdeg, const uint32_t* csz,
                            unsigned long long* out) {
    __shared__ unsigned long long sm[1024], ss[1024], sc[1024];
    unsigned long long bm = 0, bs = 1, cnt = 0;
    for (uint32_t x = threadIdx.x; x < nh; x += blockDim.x) {
        if (csz[x] == 0) continue;
        cnt++;
        if (frac_gt(cdeg[x], csz[x], bm, bs)) {
            bm = cdeg[x];
            bs = csz[x];
        }
    }
    sm[threadIdx.x] = bm;
    ss[threadIdx.x] = bs;
    sc[threadIdx.x] = cnt;
    __syncthreads();
    for (unsigned w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            unsigned o = threadIdx.x + w;
            if (frac_gt(sm[o], ss[o], sm[threadIdx.x], ss[threadIdx.x])) {
                sm[threadIdx.x] = sm[o];
                ss[threadIdx.x] = ss[o];
            }
            sc[threadIdx.x] += sc[o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[0] = sm[0];
        out[1] = ss[0];
        out[2] = sc[0];
    }
}

// ------------------------------------------------ (h-1)-cliques of the core
// Cliques are listed level by level as ascending rank tuples: a j-tuple
// extends by every w in N+(last member) adjacent to all the other members.
// Each clique appears once (its members in increasing rank order).

__global__ void k_iota(uint32_t n, uint32_t* out) {
    for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (uint64_t)gridDim.x * blockDim.x)
        out[v] = (uint32_t)v;
}

// fill == false: cnt[t] = number of extensions of tuple t.
// fill == true:  writes the (j+1)-tuples of t from pos[t] on.
template <bool FILL>
__global__ void k_extend(uint64_t nt, int j, const uint32_t* T, const uint64_t* roff,
                         const uint32_t* radj, const uint64_t* rsplit, uint32_t* cnt,
                         const uint64_t* pos, uint32_t* T2) {
    for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nt;
         t += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t* tup = T + t * j;
        uint32_t last = tup[j - 1];
        uint32_t k = 0;
        uint64_t at = FILL ? pos[t] : 0;
        for (uint64_t p = rsplit[last]; p < roff[last + 1]; p++) {
            uint32_t w = radj[p];
            bool ok = true;
            for (int i = 0; i < j - 1 && ok; i++) {
                uint32_t x = tup[i];
                ok = in_sorted(radj + rsplit[x], roff[x + 1] - rsplit[x], w);
            }
            if (!ok) continue;
            if (FILL) {
                uint32_t* dst = T2 + (at + k) * (j + 1);
                for (int i = 0; i < j; i++) dst[i] = tup[i];
                dst[j] = w;
            }
            k++;
        }
        if (!FILL) cnt[t] = k;
    }
}

// ------------------------------------------------------------ flow network
// Nodes: 0 = s, 1 = t, 2 + v for the core's vertices (rank ids), then one per
// (h-1)-clique psi.  Arcs are stored per node (head[x] .. head[x+1]) with
// the index of the residual twin in rev[].
//   s -> v   capacity q * deg_W(v)       (its twin first in v's list)
//   v -> t   capacity p * h              (second in v's list)
//   psi -> u infinite, u in psi          (first h-1 arcs of psi)
//   w -> psi capacity q, psi + w a clique (twins after them in psi's list)
// The remaining arcs of a vertex are taken from a per-vertex cursor.

// Common neighbours of psi: every w adjacent to all members, found by
// scanning the shortest member row and binary-searching the others (a
// member never passes: it is not in its own row).  Warp per psi.
// FILL == false: c[i] = |CN(psi_i)|, vin[w] += 1 and vdeg[w] += 1 per common
// neighbour, vin[u] += 1 per member when c > 0.
// FILL == true: writes the psi -> u / w -> psi arcs and their twins.
template <bool FILL>
__global__ void k_psi(uint64_t npsi, int r, const uint32_t* P, uint32_t nW, const uint64_t* roff,
                      const uint32_t* radj, uint32_t* c, unsigned long long* vin,
                      unsigned long long* vdeg, const uint64_t* head, unsigned long long* cursor,
                      uint32_t* to, uint64_t* rev, uint8_t* kind, uint32_t* err) {
    uint64_t gw = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    unsigned lane = lane_id();
    for (uint64_t i = gw; i < npsi; i += nw) {
        const uint32_t* psi = P + i * r;
        if (FILL && c[i] == 0) continue;
        // the member with the shortest row
        uint32_t b = psi[0];
        for (int k = 1; k < r; k++) {
            uint32_t x = psi[k];
            if (roff[x + 1] - roff[x] < roff[b + 1] - roff[b]) b = x;
        }
        const uint64_t node = 2ull + nW + i;
        uint64_t base = FILL ? head[node] : 0;
        uint32_t found = 0;
        for (uint64_t p0 = roff[b]; p0 < roff[b + 1]; p0 += 32) {
            uint64_t p = p0 + lane;
            uint32_t w = 0;
            bool ok = p < roff[b + 1];
            if (ok) {
                w = radj[p];
                for (int k = 0; k < r && ok; k++) {
                    uint32_t x = psi[k];
                    if (x != b) ok = in_sorted(radj + roff[x], roff[x + 1] - roff[x], w);
                }
            }
            unsigned bal = __ballot_sync(0xffffffffu, ok);
            if (ok) {
                if (!FILL) {
                    atomicAdd(&vin[w], 1ull);
                    atomicAdd(&vdeg[w], 1ull);
                } else {
                    uint64_t a = base + r + found + __popc(bal & lanemask_lt());
                    uint64_t bpos = head[2 + w] + atomicAdd(&cursor[w], 1ull);
                    if (a < head[node + 1] && bpos < head[2 + w + 1]) {
                        to[a] = 2 + w;
                        kind[a] = arc_kind(kArcRev, kArcQ);
                        rev[a] = bpos;
                        to[bpos] = (uint32_t)node;
                        kind[bpos] = arc_kind(kArcQ, kArcQ);
                        rev[bpos] = a;
                    } else {
                        atomicOr(err, 1u);
                    }
                }
            }
            found += __popc(bal);
        }
        if (!FILL) {
            if (lane == 0) {
                c[i] = found;
                if (found)
                    for (int k = 0; k < r; k++) atomicAdd(&vin[psi[k]], 1ull);
            }
        } else if ((int)lane < r) {
            uint32_t u = psi[lane];
            uint64_t a = base + lane;
            uint64_t bpos = head[2 + u] + atomicAdd(&cursor[u], 1ull);
            if (a < head[node + 1] && bpos < head[2 + u + 1]) {
                to[a] = 2 + u;
                kind[a] = arc_kind(kArcInf, kArcInf);
                rev[a] = bpos;
                to[bpos] = (uint32_t)node;
                kind[bpos] = arc_kind(kArcRev, kArcInf);
                rev[bpos] = a;
            } else {
                atomicOr(err, 1u);
            }
        }
    }
}

// Arcs per node.
__global__ void k_node_arcs(uint32_t nW, uint64_t npsi, int r, const unsigned long long* vin,
                            const uint32_t* c, uint64_t* cnt) {
    uint64_t N = 2ull + nW + npsi;
    for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < N;
         x += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t k;
        if (x < 2) k = nW;
        else if (x < 2ull + nW) k = 2 + vin[x - 2];
        else k = c[x - 2 - nW] ? (uint64_t)r + c[x - 2 - nW] : 0;
        cnt[x] = k;
    }
}

// The source and sink arcs of vertex v and their twins; cursor[v] = 2.
__global__ void k_fixed_arcs(uint32_t nW, const uint64_t* head, uint32_t* to, uint64_t* rev,
                             uint8_t* kind, unsigned long long* cursor) {
    for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < nW;
         v += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t sa = head[0] + v, ta = head[1] + v, v0 = head[2 + v], v1 = v0 + 1;
        to[sa] = 2 + (uint32_t)v; kind[sa] = arc_kind(kArcS, kArcS);   rev[sa] = v0;
        to[v0] = 0;               kind[v0] = arc_kind(kArcRev, kArcS); rev[v0] = sa;
        to[v1] = 1;               kind[v1] = arc_kind(kArcT, kArcT);   rev[v1] = ta;
        to[ta] = 2 + (uint32_t)v; kind[ta] = arc_kind(kArcRev, kArcT); rev[ta] = v1;
        cursor[v] = 2;
    }
}

__global__ void k_check_cursor(uint32_t nW, const unsigned long long* cursor,
                               const unsigned long long* vin, uint32_t* err) {
    for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < nW;
         v += (uint64_t)gridDim.x * blockDim.x)
        if (cursor[v] != 2 + vin[v]) atomicOr(err, 2u);
}

// Capacities for alpha = p / q (scaled by q); twins start empty.
__global__ void k_caps(uint64_t E, const uint8_t* kind, const uint32_t* to,
                       const unsigned long long* vdeg, unsigned long long p,
                       unsigned long long q, int h, unsigned long long* cf) {
    for (uint64_t a = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; a < E;
         a += (uint64_t)gridDim.x * blockDim.x) {
        unsigned long long c = 0;
        switch (kind[a] & 15) {
            case kArcS: c = q * vdeg[to[a] - 2]; break;
            case kArcT: c = p * (unsigned long long)h; break;
            case kArcQ: c = q; break;
            case kArcInf: c = kInfCap; break;
            default: c = 0;
        }
        cf[a] = c;
    }
}

// ---------------------------------------------------- push-relabel min cut
// Heights obey h(x) <= h(y) + 1 on every residual arc x -> y; a node with
// excess and height < N is active.  One round: every active node pushes what
// it holds along admissible arcs (h(y) = h(x) - 1) against the heights of
// the round's start; a node whose arcs hold no admissible one any more and
// that still has excess is relabelled to 1 + the least height over its
// residual arcs, read from the same snapshot and written to a separate
// buffer.  A push on x -> y needs h(x) = h(y) + 1 and one on y -> x the
// reverse, so no arc pair is pushed from both ends in a round.
// Each node keeps a current arc: the arcs before it are saturated or not
// admissible, and stay so until the node's height changes (an arc x -> y
// turns admissible only if h(y) falls or y pushes back, which needs
// h(y) = h(x) + 1), so a push resumes there and a relabel resets it.
// Every few rounds the heights are replaced by exact residual distances to t
// (backward breadth-first search; nodes that cannot reach t get N), which
// resets all current arcs.  With no active node left the preflow is maximum,
// and the nodes that still reach t form the smallest sink side of a minimum
// cut.  Nodes with more than kBigArcs arcs (the core's vertices, each in
// many cliques) are worked on by a block, the rest by a warp.

struct PR {
    const uint64_t* head;
    const uint32_t* to;
    const uint64_t* rev;
    const uint8_t* kind;
    unsigned long long* cf;
    unsigned long long* excess;
    uint32_t* height;
    uint64_t* cur;
    const unsigned long long* vdeg;
    unsigned long long p, q;
    int h;
    uint64_t N;
};

// Capacity of the pair of arc e (owner -> x): the twin's residual is this
// minus e's residual.
__device__ __forceinline__ unsigned long long pair_cap(const PR& P, uint8_t k, uint32_t owner,
                                                       uint32_t x) {
    switch (k >> 4) {
        case kArcS: return P.q * P.vdeg[(x == 0 ? owner : x) - 2];
        case kArcT: return P.p * (unsigned long long)P.h;
        case kArcQ: return P.q;
        case kArcInf: return kInfCap;
    }
    return 0;
}

__device__ __forceinline__ bool is_big(const PR& P, uint32_t x) {
    return P.head[x + 1] - P.head[x] > kBigArcs;
}

__device__ __forceinline__ unsigned long long sat_add(unsigned long long a, unsigned long long b) {
    unsigned long long c = a + b;
    return c < a ? ~0ull : c;
}

__device__ __forceinline__ unsigned long long warp_scan_sat(unsigned long long v) {
    unsigned lane = lane_id();
    for (int o = 1; o < 32; o <<= 1) {
        unsigned long long y = __shfl_up_sync(0xffffffffu, v, o);
        if ((int)lane >= o) v = sat_add(v, y);
    }
    return v;
}

__global__ void k_preflow(uint32_t nW, const uint64_t* head, const uint64_t* rev,
                          unsigned long long* cf, unsigned long long* excess) {
    for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < nW;
         v += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t sa = head[0] + v;
        unsigned long long c = cf[sa];
        cf[sa] = 0;
        cf[rev[sa]] = c;
        excess[2 + v] = c;
    }
}

// Frontier lists: small nodes (warp each) and big nodes (block each); the
// counters c[0], c[1] hold their lengths.
__global__ void k_bfs_init(PR P, uint32_t* fs, uint32_t* fb, uint32_t* c) {
    for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < P.N;
         x += (uint64_t)gridDim.x * blockDim.x)
        P.height[x] = x == 1 ? 0u : kUnset;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        bool big = is_big(P, 1);
        (big ? fb : fs)[0] = 1;
        c[0] = big ? 0u : 1u;
        c[1] = big ? 1u : 0u;
    }
}

// Arc e of frontier node y at distance d: x = to[e] gets d + 1 when
// x -> y has residual capacity and x has no distance yet (s is never entered).
__device__ __forceinline__ void bfs_arc(const PR& P, uint32_t y, uint64_t e, uint64_t end,
                                        uint32_t d, uint32_t* os, uint32_t* ob, uint32_t* oc) {
    bool add = false;
    uint32_t x = 0;
    if (e < end) {
        x = P.to[e];
        if (x != 0 && P.height[x] == kUnset && pair_cap(P, P.kind[e], y, x) > P.cf[e])
            add = atomicCAS(&P.height[x], kUnset, d + 1) == kUnset;
    }
    bool big = add && is_big(P, x);
    warp_append(add && !big, x, os, oc);
    warp_append(big, x, ob, oc + 1);
}

__global__ void k_bfs_small(PR P, const uint32_t* fs, const uint32_t* c, uint32_t d,
                            uint32_t* os, uint32_t* ob, uint32_t* oc) {
    uint64_t gw = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    const uint32_t n = c[0];
    for (uint64_t i = gw; i < n; i += nw) {
        uint32_t y = fs[i];
        const uint64_t end = P.head[y + 1];
        for (uint64_t p0 = P.head[y]; p0 < end; p0 += 32)
            bfs_arc(P, y, p0 + lane_id(), end, d, os, ob, oc);
    }
}

__global__ void k_bfs_big(PR P, const uint32_t* fb, const uint32_t* c, uint32_t d,
                          uint32_t* os, uint32_t* ob, uint32_t* oc) {
    const uint32_t n = c[1];
    for (uint64_t i = blockIdx.x; i < n; i += gridDim.x) {
        uint32_t y = fb[i];
        const uint64_t end = P.head[y + 1];
        for (uint64_t p0 = P.head[y]; p0 < end; p0 += blockDim.x)
            bfs_arc(P, y, p0 + threadIdx.x, end, d, os, ob, oc);
    }
}

// Unreached nodes (and s) get N; every current arc goes back to the start.
__global__ void k_bfs_finish(PR P) {
    for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < P.N;
         x += (uint64_t)gridDim.x * blockDim.x) {
        if (x == 0 || P.height[x] == kUnset) P.height[x] = (uint32_t)P.N;
        P.cur[x] = P.head[x];
    }
}

// Active nodes into the small (c[0]) and big (c[1]) lists.
__global__ void k_collect(PR P, uint32_t* ls, uint32_t* lb, uint32_t* c) {
    for (uint64_t x0 = (uint64_t)blockIdx.x * blockDim.x; x0 < P.N;
         x0 += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t x = x0 + threadIdx.x;
        bool act = x >= 2 && x < P.N && P.excess[x] > 0 && P.height[x] < P.N;
        bool big = act && is_big(P, (uint32_t)x);
        warp_append(act && !big, (uint32_t)x, ls, c);
        warp_append(big, (uint32_t)x, lb, c + 1);
    }
}

// One chunk of node u's arcs from a (one arc per thread): the admissible
// residual c of this thread's arc.
__device__ __forceinline__ unsigned long long admissible(const PR& P, uint64_t a, uint64_t end,
                                                         uint32_t hu, uint32_t* v) {
    unsigned long long c = 0;
    *v = 0;
    if (a < end) {
        *v = P.to[a];
        unsigned long long ca = P.cf[a];
        if (ca > 0 && P.height[*v] + 1 == hu) c = ca;
    }
    return c;
}

__device__ __forceinline__ void push_arc(const PR& P, uint64_t a, uint32_t v,
                                         unsigned long long d) {
    atomicAdd(&P.cf[a], (unsigned long long)(-(long long)d));
    atomicAdd(&P.cf[P.rev[a]], d);
    atomicAdd(&P.excess[v], d);
}

// Warp per small active node.  The prefix of the admissible residuals is
// saturating: a saturated sum leaves the exclusive prefix above any excess
// (residuals < 2^63, excess < 2^61), so no push is made from it.
__global__ void k_push_small(PR P, const uint32_t* list, const uint32_t* c) {
    uint64_t gw = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    unsigned lane = lane_id();
    const uint32_t n = c[0];
    for (uint64_t i = gw; i < n; i += nw) {
        const uint32_t u = list[i];
        const unsigned long long e0 = P.excess[u];
        const uint32_t hu = P.height[u];
        const uint64_t end = P.head[u + 1];
        unsigned long long rem = e0;
        uint64_t p0 = P.cur[u], ncur = end;
        while (p0 < end && rem > 0) {
            uint32_t v;
            const uint64_t a = p0 + lane;
            unsigned long long cv = admissible(P, a, end, hu, &v);
            unsigned long long incl = warp_scan_sat(cv), excl = incl - cv;
            unsigned long long d = 0;
            if (cv > 0 && excl < rem) d = cv < rem - excl ? cv : rem - excl;
            if (d) push_arc(P, a, v, d);
            // first arc with admissible residual left: the new current arc
            uint64_t left = cv > d ? a : ~0ull;
            left = warp_min_u64(left);
            if (left < ncur) ncur = left;
            unsigned long long tot = __shfl_sync(0xffffffffu, incl, 31);
            rem -= tot < rem ? tot : rem;
            p0 += 32;
        }
        if (lane == 0) {
            P.cur[u] = ncur < p0 ? ncur : (p0 < end ? p0 : end);
            if (rem != e0) atomicAdd(&P.excess[u], (unsigned long long)(-(long long)(e0 - rem)));
        }
    }
}

// Block per big active node (kBigThreads threads).
__global__ void __launch_bounds__(kBigThreads) k_push_big(PR P, const uint32_t* list,
                                                          const uint32_t* c) {
    constexpr int NW = kBigThreads / 32;
    __shared__ unsigned long long s_w[NW];
    __shared__ unsigned long long s_cur;
    const unsigned lane = lane_id(), warp = warp_id();
    const uint32_t n = c[1];
    for (uint64_t i = blockIdx.x; i < n; i += gridDim.x) {
        const uint32_t u = list[i];
        const unsigned long long e0 = P.excess[u];
        const uint32_t hu = P.height[u];
        const uint64_t end = P.head[u + 1];
        unsigned long long rem = e0;
        uint64_t p0 = P.cur[u];
        if (threadIdx.x == 0) s_cur = end;
        __syncthreads();
        while (p0 < end && rem > 0) {
            uint32_t v;
            const uint64_t a = p0 + threadIdx.x;
            unsigned long long cv = admissible(P, a, end, hu, &v);
            unsigned long long incl = warp_scan_sat(cv);
            if (lane == 31) s_w[warp] = incl;
            __syncthreads();
            if (warp == 0) {
                unsigned long long t = lane < NW ? s_w[lane] : 0;
                t = warp_scan_sat(t);
                if (lane < NW) s_w[lane] = t;
            }
            __syncthreads();
            if (warp > 0) incl = sat_add(incl, s_w[warp - 1]);
            const unsigned long long tot = s_w[NW - 1];
            unsigned long long excl = incl - cv;
            unsigned long long d = 0;
            if (cv > 0 && excl < rem) d = cv < rem - excl ? cv : rem - excl;
            if (d) push_arc(P, a, v, d);
            if (cv > d) atomicMin(&s_cur, (unsigned long long)a);
            rem -= tot < rem ? tot : rem;
            p0 += kBigThreads;
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            uint64_t nc = s_cur;
            P.cur[u] = nc < p0 ? nc : (p0 < end ? p0 : end);
            if (rem != e0) atomicAdd(&P.excess[u], (unsigned long long)(-(long long)(e0 - rem)));
        }
        __syncthreads();
    }
}

// New height of a node that holds excess with its current arc at the end:
// 1 + the least height over its residual arcs (N if none), else kUnset.
__global__ void k_relabel_small(PR P, const uint32_t* list, const uint32_t* c, uint32_t* nh) {
    uint64_t gw = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    unsigned lane = lane_id();
    const uint32_t n = c[0];
    for (uint64_t i = gw; i < n; i += nw) {
        const uint32_t u = list[i];
        const uint64_t end = P.head[u + 1];
        if (P.excess[u] == 0 || P.cur[u] < end) {
            if (lane == 0) nh[i] = kUnset;
            continue;
        }
        uint32_t m = kUnset;
        for (uint64_t a = P.head[u] + lane; a < end; a += 32)
            if (P.cf[a] > 0) {
                uint32_t hv = P.height[P.to[a]];
                m = hv < m ? hv : m;
            }
        for (int o = 16; o > 0; o >>= 1) {
            uint32_t y = __shfl_xor_sync(0xffffffffu, m, o);
            m = y < m ? y : m;
        }
        if (lane == 0) {
            uint64_t nv = m == kUnset ? P.N : (uint64_t)m + 1;
            if (nv > P.N) nv = P.N;
            nh[i] = (uint32_t)nv;
        }
    }
}

__global__ void __launch_bounds__(kBigThreads) k_relabel_big(PR P, const uint32_t* list,
                                                             const uint32_t* c, uint32_t* nh) {
    __shared__ uint32_t s_m;
    const uint32_t n = c[1];
    for (uint64_t i = blockIdx.x; i < n; i += gridDim.x) {
        const uint32_t u = list[i];
        const uint64_t end = P.head[u + 1];
        if (P.excess[u] == 0 || P.cur[u] < end) {
            if (threadIdx.x == 0) nh[i] = kUnset;
            continue;
        }
        if (threadIdx.x == 0) s_m = kUnset;
        __syncthreads();
        uint32_t m = kUnset;
        for (uint64_t a = P.head[u] + threadIdx.x; a < end; a += blockDim.x)
            if (P.cf[a] > 0) {
                uint32_t hv = P.height[P.to[a]];
                m = hv < m ? hv : m;
            }
        for (int o = 16; o > 0; o >>= 1) {
            uint32_t y = __shfl_xor_sync(0xffffffffu, m, o);
            m = y < m ? y : m;
        }
        if (lane_id() == 0 && m != kUnset) atomicMin(&s_m, m);
        __syncthreads();
        if (threadIdx.x == 0) {
            uint64_t nv = s_m == kUnset ? P.N : (uint64_t)s_m + 1;
            if (nv > P.N) nv = P.N;
            nh[i] = (uint32_t)nv;
        }
        __syncthreads();
    }
}

// Relabelled nodes take their new height and restart at their first arc.
__global__ void k_apply(PR P, const uint32_t* ls, const uint32_t* lb, const uint32_t* c,
                        const uint32_t* nhs, const uint32_t* nhb) {
    const uint64_t ns = c[0], nb = c[1];
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < ns + nb;
         i += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t u = i < ns ? ls[i] : lb[i - ns];
        uint32_t v = i < ns ? nhs[i] : nhb[i - ns];
        if (v != kUnset) {
            P.height[u] = v;
            P.cur[u] = P.head[u];
        }
    }
}

// Vertex v of the core is on the source side when it cannot reach t.
__global__ void k_source_side(uint32_t nW, const uint32_t* height, uint64_t N, uint32_t* inA,
                              unsigned long long* cnt) {
    unsigned long long c = 0;
    for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < nW;
         v += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t a = height[2 + v] >= N ? 1u : 0u;
        inA[v] = a;
        c += a;
    }
    c = warp_sum(c);
    if (lane_id() == 0 && c) atomicAdd(cnt, c);
}

// flag[g id] = 1 for the core vertices (rank r) with inA[r].
__global__ void k_mark_g(uint32_t nW, const uint32_t* inA, const uint32_t* old_of,
                         const uint32_t* orig, uint32_t* flag) {
    for (uint64_t r = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; r < nW;
         r += (uint64_t)gridDim.x * blockDim.x)
        if (inA[r]) flag[orig[old_of[r]]] = 1u;
}

__global__ void k_compact_flags(uint32_t n, const uint32_t* flag, const uint64_t* pos,
                                uint32_t* out) {
    for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (uint64_t)gridDim.x * blockDim.x)
        if (flag[v]) out[pos[v]] = (uint32_t)v;
}

// ------------------------------------------------------------------- host

uint64_t now_ns() {
    return (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(
               std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

struct Net {
    uint32_t nW = 0;
    uint64_t npsi = 0, N = 0, E = 0;
    uint64_t* head = nullptr;
    uint32_t* to = nullptr;
    uint64_t* rev = nullptr;
    uint8_t* kind = nullptr;
    unsigned long long* cf = nullptr;
    unsigned long long* vdeg = nullptr;
    unsigned long long muW = 0;
};

void net_free(Net* net, cudaStream_t s) {
    void* ptrs[] = {net->head, net->to, net->rev, net->kind, net->cf, net->vdeg};
    for (void* p : ptrs) dev_free(p, s);
    *net = Net();
}

#define XSTEP(x)                     \
    do {                             \
        st = (x);                    \
        if (st != DSD_OK) goto done; \
    } while (0)
#define XCU(x)                                                                          \
    do {                                                                                \
        cudaError_t e_ = (x);                                                           \
        if (e_ != cudaSuccess) { st = cuda_fail(e_, #x, __FILE__, __LINE__); goto done; } \
    } while (0)

template <class T>
dsd_status read_back(T* host, const T* dev, cudaStream_t s) {
    DSD_CU(cudaMemcpyAsync(host, dev, sizeof(T), cudaMemcpyDeviceToHost, s));
    DSD_CU(cudaStreamSynchronize(s));
    return DSD_OK;
}

// The network of Algorithm 1 on W (its relabelled CSR), capacities unset.
dsd_status build_network(dsd_graph* W, int h, Net* net) {
    cudaStream_t s = W->stream;
    const int r = h - 1;
    const uint32_t nW = W->n;
    dsd_status st = DSD_OK;
    uint32_t *T = nullptr, *T2 = nullptr, *cnt = nullptr, *c = nullptr, *err = nullptr;
    uint64_t *pos = nullptr, *ncnt = nullptr;
    unsigned long long *vin = nullptr, *cursor = nullptr;
    uint64_t nt = nW, total = 0, sumc = 0;
    uint32_t herr = 0;
    *net = Net();
    net->nW = nW;
    XSTEP(dalloc(&T, (size_t)nW + 1, s));
    k_iota<<<grid_for_n(nW), 256, 0, s>>>(nW, T); note_launch();
    for (int j = 1; j < r; j++) {
        XSTEP(dalloc(&cnt, nt + 1, s));
        XSTEP(dalloc(&pos, nt + 1, s));
        if (nt)
            k_extend<false><<<grid_for_n(nt), 256, 0, s>>>(nt, j, T, W->roff, W->radj, W->rsplit,
                                                           cnt, nullptr, nullptr);
        note_launch();
        XSTEP(exclusive_scan_u32_to_u64(cnt, pos, nt, s));
        XSTEP(read_back(&total, pos + nt, s));
        XSTEP(dalloc(&T2, (size_t)total * (j + 1) + 1, s));
        if (nt)
            k_extend<true><<<grid_for_n(nt), 256, 0, s>>>(nt, j, T, W->roff, W->radj, W->rsplit,
                                                          nullptr, pos, T2);
        note_launch();
        XCU(cudaGetLastError());
        dev_free(T, s);
        dev_free(cnt, s);
        dev_free(pos, s);
        T = T2;
        T2 = nullptr;
        cnt = nullptr;
        pos = nullptr;
        nt = total;
    }
    net->npsi = nt;
    net->N = 2ull + nW + nt;
    if (net->N >= (1ull << 31)) {
        set_error("flow network of %llu nodes exceeds 2^31", (unsigned long long)net->N);
        st = DSD_ERR_UNSUPPORTED;
        goto done;
    }
    XSTEP(dalloc(&c, nt + 1, s));
    XSTEP(dalloc(&vin, (size_t)nW + 1, s));
    XSTEP(dalloc(&net->vdeg, (size_t)nW + 1, s));
    XSTEP(dalloc(&err, 1, s));
    XCU(cudaMemsetAsync(vin, 0, ((size_t)nW + 1) * 8, s));
    XCU(cudaMemsetAsync(net->vdeg, 0, ((size_t)nW + 1) * 8, s));
    XCU(cudaMemsetAsync(err, 0, 4, s));
    if (nt)
        k_psi<false><<<grid_for_warps(nt), 256, 0, s>>>(nt, r, T, nW, W->roff, W->radj, c, vin,
                                                        net->vdeg, nullptr, nullptr, nullptr,
                                                        nullptr, nullptr, err);
    note_launch();
    XSTEP(dalloc(&pos, nt + 1, s));
    XSTEP(exclusive_scan_u32_to_u64(c, pos, nt, s));
    XSTEP(read_back(&sumc, pos + nt, s));
    if (sumc % (uint64_t)h) {
        set_error("clique count of the flow network is not a multiple of h");
        st = DSD_ERR_INTERNAL;
        goto done;
    }
    net->muW = sumc / (uint64_t)h;
    XSTEP(dalloc(&ncnt, net->N + 1, s));
    XSTEP(dalloc(&net->head, net->N + 1, s));
    k_node_arcs<<<grid_for_n(net->N), 256, 0, s>>>(nW, nt, r, vin, c, ncnt); note_launch();
    XSTEP(exclusive_scan_u64(ncnt, net->head, net->N, s));
    XSTEP(read_back(&net->E, net->head + net->N, s));
    XSTEP(dalloc(&net->to, net->E + 1, s));
    XSTEP(dalloc(&net->rev, net->E + 1, s));
    XSTEP(dalloc(&net->kind, net->E + 1, s));
    XSTEP(dalloc(&net->cf, net->E + 1, s));
    XSTEP(dalloc(&cursor, (size_t)nW + 1, s));
    // every slot is written below (checked); zeros keep an unwritten one inert
    XCU(cudaMemsetAsync(net->to, 0, (net->E + 1) * 4, s));
    XCU(cudaMemsetAsync(net->rev, 0, (net->E + 1) * 8, s));
    XCU(cudaMemsetAsync(net->kind, 0, net->E + 1, s));
    if (nW) {
        k_fixed_arcs<<<grid_for_n(nW), 256, 0, s>>>(nW, net->head, net->to, net->rev, net->kind,
                                                    cursor);
        note_launch();
    }
    if (nt)
        k_psi<true><<<grid_for_warps(nt), 256, 0, s>>>(nt, r, T, nW, W->roff, W->radj, c, nullptr,
                                                       nullptr, net->head, cursor, net->to,
                                                       net->rev, net->kind, err);
    note_launch();
    if (nW) {
        k_check_cursor<<<grid_for_n(nW), 256, 0, s>>>(nW, cursor, vin, err);
        note_launch();
    }
    XCU(cudaGetLastError());
    XSTEP(read_back(&herr, err, s));
    if (herr) {
        set_error("flow network arc layout check failed (%u)", herr);
        st = DSD_ERR_INTERNAL;
    }
done:
    {
        void* ptrs[] = {T, T2, cnt, c, err, pos, ncnt, vin, cursor};
        for (void* p : ptrs) dev_free(p, s);
    }
    if (st != DSD_OK) net_free(net, s);
    return st;
}

struct CutStats {
    uint64_t rounds = 0, relabels = 0;
};

// Device buffers of one minimum cut.
struct CutWork {
    unsigned long long* excess = nullptr;
    uint32_t* height = nullptr;
    uint64_t* cur = nullptr;
    uint32_t* ls = nullptr;       // active lists: small, big
    uint32_t* lb = nullptr;
    uint32_t* nhs = nullptr;      // new heights for them
    uint32_t* nhb = nullptr;
    uint32_t* f[4] = {};          // frontiers: small/big, two levels
    uint32_t* ctr = nullptr;      // [0,1] active, [2..5] frontier counters
    unsigned long long* cnt = nullptr;
};

dsd_status cut_alloc(CutWork* w, uint64_t N, cudaStream_t s) {
    DSD_TRY(dalloc(&w->excess, N + 1, s));
    DSD_TRY(dalloc(&w->height, N + 1, s));
    DSD_TRY(dalloc(&w->cur, N + 1, s));
    DSD_TRY(dalloc(&w->ls, N + 1, s));
    DSD_TRY(dalloc(&w->lb, N + 1, s));
    DSD_TRY(dalloc(&w->nhs, N + 1, s));
    DSD_TRY(dalloc(&w->nhb, N + 1, s));
    for (auto& f : w->f) DSD_TRY(dalloc(&f, N + 1, s));
    DSD_TRY(dalloc(&w->ctr, 8, s));
    DSD_TRY(dalloc(&w->cnt, 1, s));
    return DSD_OK;
}

void cut_free(CutWork* w, cudaStream_t s) {
    void* ptrs[] = {w->excess, w->height, w->cur, w->ls, w->lb, w->nhs, w->nhb,
                    w->f[0], w->f[1], w->f[2], w->f[3], w->ctr, w->cnt};
    for (void* p : ptrs) dev_free(p, s);
    *w = CutWork();
}

constexpr unsigned kSmallGrid = 152 * 8;   // blocks of 256 threads (warp per node)
constexpr unsigned kBigGrid = 152 * 4;     // blocks of kBigThreads (block per node)

// Backward breadth-first search from t: exact residual distances to t, N for
// nodes that cannot reach it (and for s); resets the current arcs.  The
// levels are queued kBfsBatch at a time and the host reads the frontier size
// once per batch: a level whose input frontier is empty does nothing.
constexpr uint32_t kBfsBatch = 8;

dsd_status global_relabel(const PR& P, CutWork& w, cudaStream_t s) {
    uint32_t *fs = w.f[0], *fb = w.f[1], *os = w.f[2], *ob = w.f[3];
    uint32_t* cin = w.ctr + 2;
    uint32_t* cout = w.ctr + 4;
    k_bfs_init<<<grid_for_n(P.N), 256, 0, s>>>(P, fs, fb, cin); note_launch();
    for (uint32_t d0 = 0;; d0 += kBfsBatch) {
        for (uint32_t d = d0; d < d0 + kBfsBatch; d++) {
            DSD_CU(cudaMemsetAsync(cout, 0, 8, s));
            k_bfs_small<<<kSmallGrid, 256, 0, s>>>(P, fs, cin, d, os, ob, cout);
            k_bfs_big<<<kBigGrid, kBigThreads, 0, s>>>(P, fb, cin, d, os, ob, cout);
            note_launch();
            note_launch();
            uint32_t* t;
            t = fs; fs = os; os = t;
            t = fb; fb = ob; ob = t;
            t = cin; cin = cout; cout = t;
        }
        uint32_t nc[2] = {0, 0};   // the last level's output frontier (now cin)
        DSD_CU(cudaMemcpyAsync(nc, cin, 8, cudaMemcpyDeviceToHost, s));
        DSD_CU(cudaStreamSynchronize(s));
        if (nc[0] + nc[1] == 0) break;
        if (d0 > P.N) {
            set_error("breadth-first search did not settle");
            return DSD_ERR_INTERNAL;
        }
    }
    k_bfs_finish<<<grid_for_n(P.N), 256, 0, s>>>(P); note_launch();
    DSD_LAUNCHED();
    return DSD_OK;
}

// Maximum flow of the network at alpha = p / q; *flow = value, inA[r] = 1
// for the core vertices on the largest source side of a minimum cut,
// *sizeA their number.
dsd_status min_cut(const Net& net, int h, uint64_t p, uint64_t q, cudaStream_t s,
                   unsigned long long* flow, uint32_t* inA, uint64_t* sizeA, CutStats* cs) {
    dsd_status st = DSD_OK;
    const uint64_t N = net.N;
    CutWork w;
    PR P;
    const uint64_t t0 = now_ns();
    const uint64_t limit_rounds = 4 * N + 100000;
    const int kRoundsPerRelabel = 32;
    XSTEP(cut_alloc(&w, N, s));
    P.head = net.head;
    P.to = net.to;
    P.rev = net.rev;
    P.kind = net.kind;
    P.cf = net.cf;
    P.excess = w.excess;
    P.height = w.height;
    P.cur = w.cur;
    P.vdeg = net.vdeg;
    P.p = p;
    P.q = q;
    P.h = h;
    P.N = N;
    k_caps<<<grid_for_n(net.E), 256, 0, s>>>(net.E, net.kind, net.to, net.vdeg, p, q, h, net.cf);
    note_launch();
    XCU(cudaMemsetAsync(w.excess, 0, (N + 1) * 8, s));
    k_preflow<<<grid_for_n(net.nW), 256, 0, s>>>(net.nW, net.head, net.rev, net.cf, w.excess);
    note_launch();
    XSTEP(global_relabel(P, w, s));
    cs->relabels++;
    for (;;) {
        uint32_t na[2] = {0, 0};
        XCU(cudaMemsetAsync(w.ctr, 0, 8, s));
        k_collect<<<grid_for_n(N), 256, 0, s>>>(P, w.ls, w.lb, w.ctr); note_launch();
        XCU(cudaMemcpyAsync(na, w.ctr, 8, cudaMemcpyDeviceToHost, s));
        XCU(cudaStreamSynchronize(s));
        if (na[0] + na[1] == 0) break;
        for (int it = 0; it < kRoundsPerRelabel; it++) {
            if (it) {
                XCU(cudaMemsetAsync(w.ctr, 0, 8, s));
                k_collect<<<grid_for_n(N), 256, 0, s>>>(P, w.ls, w.lb, w.ctr);
                note_launch();
            }
            k_push_small<<<kSmallGrid, 256, 0, s>>>(P, w.ls, w.ctr);
            k_push_big<<<kBigGrid, kBigThreads, 0, s>>>(P, w.lb, w.ctr);
            k_relabel_small<<<kSmallGrid, 256, 0, s>>>(P, w.ls, w.ctr, w.nhs);
            k_relabel_big<<<kBigGrid, kBigThreads, 0, s>>>(P, w.lb, w.ctr, w.nhb);
            k_apply<<<kSmallGrid, 256, 0, s>>>(P, w.ls, w.lb, w.ctr, w.nhs, w.nhb);
            for (int k = 0; k < 5; k++) note_launch();
            cs->rounds++;
        }
        XCU(cudaGetLastError());
        XSTEP(global_relabel(P, w, s));
        cs->relabels++;
        if (cs->rounds > limit_rounds || now_ns() - t0 > wait_limit_ns()) {
            set_error("push-relabel did not finish within %llu rounds / the wait limit",
                      (unsigned long long)limit_rounds);
            st = DSD_ERR_TIMEOUT;
            goto done;
        }
    }
    XSTEP(read_back(flow, w.excess + 1, s));
    XCU(cudaMemsetAsync(w.cnt, 0, 8, s));
    if (net.nW) {
        k_source_side<<<grid_for_n(net.nW), 256, 0, s>>>(net.nW, w.height, N, inA, w.cnt);
        note_launch();
    }
    {
        unsigned long long a = 0;
        XSTEP(read_back(&a, w.cnt, s));
        *sizeA = a;
    }
done:
    cut_free(&w, s);
    return st;
}

uint64_t gcd_u64(uint64_t a, uint64_t b) {
    while (b) {
        uint64_t t = a % b;
        a = b;
        b = t;
    }
    return a;
}

uint64_t ceil_div(uint64_t a, uint64_t b) { return a / b + (a % b ? 1 : 0); }

// G[R_k] as its own relabelled graph; *orig maps its ids to g's.
dsd_status located_core(dsd_graph* g, const uint64_t* core, uint64_t k, dsd_graph** W,
                        uint32_t** orig) {
    cudaStream_t s = g->stream;
    uint32_t* flag = nullptr;
    DSD_TRY(dalloc(&flag, (size_t)g->n + 1, s));
    k_flag_core_ge<<<grid_for_n(g->n), 256, 0, s>>>(g->n, core, k, flag); note_launch();
    dsd_status st = induced_subgraph(g, flag, W, orig);
    dev_free(flag, s);
    if (st == DSD_OK) st = ensure_order(*W);
    if (st != DSD_OK && *W) {
        dsd_graph_destroy(*W);
        dev_free(*orig, s);
        *W = nullptr;
        *orig = nullptr;
    }
    return st;
}

// Pruning2: the densest connected component of G[R_k1] (mu_C, |C|) and the
// number of components.
dsd_status densest_component(dsd_graph* g, int h, const uint64_t* core, uint64_t k1,
                             uint64_t* mu_c, uint64_t* size_c, uint32_t* ncomp) {
    cudaStream_t s = g->stream;
    dsd_graph* H = nullptr;
    uint32_t* orig = nullptr;
    uint32_t *parent = nullptr, *changed = nullptr, *csz = nullptr;
    unsigned long long *deg = nullptr, *cdeg = nullptr, *best = nullptr;
    dsd_status st = located_core(g, core, k1, &H, &orig);
    if (st != DSD_OK) return st;
    const uint32_t nh = H->n;
    unsigned long long hb[3] = {0, 1, 0};
    XSTEP(dalloc(&parent, (size_t)nh + 1, s));
    XSTEP(dalloc(&changed, 1, s));
    XSTEP(dalloc(&deg, (size_t)nh + 2, s));
    XSTEP(dalloc(&cdeg, (size_t)nh + 1, s));
    XSTEP(dalloc(&csz, (size_t)nh + 1, s));
    XSTEP(dalloc(&best, 3, s));
    XSTEP(count_cliques(H, h, deg, deg + nh + 1));
    k_cc_init<<<grid_for_n(nh), 256, 0, s>>>(nh, parent); note_launch();
    for (uint32_t round = 0;; round++) {
        uint32_t ch = 0;
        XCU(cudaMemsetAsync(changed, 0, 4, s));
        k_cc_hook<<<grid_for_warps(nh), 256, 0, s>>>(nh, H->off, H->adj, parent, changed);
        k_cc_compress<<<grid_for_n(nh), 256, 0, s>>>(nh, parent);
        note_launch();
        note_launch();
        XSTEP(read_back(&ch, changed, s));
        if (!ch) break;
        if (round > nh + 1) {
            set_error("connected components did not settle");
            st = DSD_ERR_INTERNAL;
            goto done;
        }
    }
    XCU(cudaMemsetAsync(cdeg, 0, ((size_t)nh + 1) * 8, s));
    XCU(cudaMemsetAsync(csz, 0, ((size_t)nh + 1) * 4, s));
    k_comp_sums<<<grid_for_n(nh), 256, 0, s>>>(nh, H->old_of, deg, parent, cdeg, csz);
    k_best_comp<<<1, 1024, 0, s>>>(nh, cdeg, csz, best);
    note_launch();
    note_launch();
    XCU(cudaMemcpyAsync(hb, best, sizeof(hb), cudaMemcpyDeviceToHost, s));
    XCU(cudaStreamSynchronize(s));
    if (hb[0] % (unsigned long long)h) {
        set_error("component clique-degree sum is not a multiple of h");
        st = DSD_ERR_INTERNAL;
        goto done;
    }
    *mu_c = hb[0] / (unsigned long long)h;
    *size_c = hb[1];
    *ncomp = (uint32_t)hb[2];
done:
    {
        void* ptrs[] = {parent, changed, deg, cdeg, csz, best, orig};
        for (void* p : ptrs) dev_free(p, s);
    }
    dsd_graph_destroy(H);
    return st;
}

// mu(G[D]) for the vertex set flagged in flag (g ids).
dsd_status count_in(dsd_graph* g, int h, const uint32_t* flag, uint64_t* mu) {
    cudaStream_t s = g->stream;
    dsd_graph* D = nullptr;
    uint32_t* orig = nullptr;
    unsigned long long* deg = nullptr;
    dsd_status st = induced_subgraph(g, flag, &D, &orig);
    if (st != DSD_OK) return st;
    XSTEP(ensure_order(D));
    XSTEP(dalloc(&deg, (size_t)D->n + 2, s));
    XSTEP(count_cliques(D, h, deg, deg + D->n + 1));
    {
        unsigned long long m = 0;
        XSTEP(read_back(&m, deg + D->n + 1, s));
        *mu = m;
    }
done:
    dev_free(deg, s);
    dev_free(orig, s);
    dsd_graph_destroy(D);
    return st;
}

}  // namespace
}  // namespace dsd

using namespace dsd;

extern "C" {

dsd_status dsd_core_exact(dsd_graph* g, int h, uint32_t* cds, int mem, dsd_exact_info* info) {
    set_error("");
    if (!g || !info || h < 2 || h > DSD_MAX_H || (mem != DSD_MEM_HOST && mem != DSD_MEM_DEVICE)) {
        set_error("invalid argument to dsd_core_exact");
        return DSD_ERR_INVALID;
    }
    dsd_exact_info I;
    memset(&I, 0, sizeof(I));
    uint64_t tm = now_ns();
    dsd_core_app_result app;
    DSD_TRY(dsd_core_app(g, h, nullptr, nullptr, DSD_MEM_HOST, &app));
    cudaStream_t s = g->stream;
    const uint32_t n = g->n;
    const uint64_t* core = cached_core(g, h);
    dsd_status st = DSD_OK;
    dsd_graph* W = nullptr;
    uint32_t *orig = nullptr, *inA = nullptr, *flag = nullptr, *tmp = nullptr;
    uint64_t* pos = nullptr;
    Net net;
    uint64_t kcur = 0, p = 0, q = 1, muA = 0, sizeA = 0;
    if (n == 0) {
        *info = I;
        return DSD_OK;
    }
    if (!core) {
        set_error("no decomposition cached for h = %d", h);
        return DSD_ERR_INTERNAL;
    }
    XSTEP(dalloc(&flag, (size_t)n + 1, s));
    if (app.densest_mu == 0) {
        // no h-clique: every set has density 0 and the largest is V
        XCU(cudaMemsetAsync(flag, 0, ((size_t)n + 1) * 4, s));
        k_flag_core_ge<<<grid_for_n(n), 256, 0, s>>>(n, core, 0, flag); note_launch();
        I.size = n;
    } else {
        // Pruning1 and Pruning2
        I.k1 = ceil_div(app.densest_mu, app.densest_size);
        uint64_t mc = 0, sc = 1;
        XSTEP(densest_component(g, h, core, I.k1, &mc, &sc, &I.components));
        p = app.densest_mu;
        q = app.densest_size;
        if ((unsigned __int128)mc * q > (unsigned __int128)p * sc) {
            p = mc;
            q = sc;
        }
        I.k2 = ceil_div(p, q);
        I.lower_mu = p;
        I.lower_size = (uint32_t)q;
        I.locate_ns = now_ns() - tm;
        // Dinkelbach's iteration on the located core
        for (;;) {
            uint64_t gq = gcd_u64(p, q);
            p /= gq;
            q /= gq;
            uint64_t k = ceil_div(p, q);
            if (!W || k != kcur) {
                net_free(&net, s);
                if (W) {
                    dsd_graph_destroy(W);
                    W = nullptr;
                }
                dev_free(orig, s);
                orig = nullptr;
                dev_free(inA, s);
                inA = nullptr;
                tm = now_ns();
                XSTEP(located_core(g, core, k, &W, &orig));
                XSTEP(build_network(W, h, &net));
                XSTEP(dalloc(&inA, (size_t)W->n + 1, s));
                I.build_ns += now_ns() - tm;
                kcur = k;
                if (I.cuts == 0) {
                    I.net_nodes = (uint32_t)net.N;
                    I.net_arcs = net.E;
                }
            }
            const unsigned __int128 cap_s = (unsigned __int128)q * h * net.muW;
            if (cap_s >= ((unsigned __int128)1 << 61) ||
                (unsigned __int128)p * h >= ((unsigned __int128)1 << 61)) {
                set_error("flow capacities exceed 2^61 (q = %llu, mu = %llu)",
                          (unsigned long long)q, (unsigned long long)net.muW);
                st = DSD_ERR_OVERFLOW;
                goto done;
            }
            unsigned long long F = 0;
            CutStats cs;
            tm = now_ns();
            XSTEP(min_cut(net, h, p, q, s, &F, inA, &sizeA, &cs));
            I.cut_ns += now_ns() - tm;
            I.cuts++;
            I.rounds += cs.rounds;
            I.relabels += cs.relabels;
            // F = q h (mu(W) - mu(A)) + p h |A|
            const unsigned __int128 php = (unsigned __int128)p * h * sizeA;
            const unsigned __int128 qh = (unsigned __int128)q * h;
            if (sizeA == 0 || (unsigned __int128)F < php || ((unsigned __int128)F - php) % qh) {
                set_error("minimum cut inconsistent with the network (|A| = %llu)",
                          (unsigned long long)sizeA);
                st = DSD_ERR_INTERNAL;
                goto done;
            }
            muA = net.muW - (uint64_t)(((unsigned __int128)F - php) / qh);
            const unsigned __int128 lhs = (unsigned __int128)muA * q,
                                    rhs = (unsigned __int128)p * sizeA;
            if (lhs > rhs) {
                p = muA;
                q = sizeA;
                continue;
            }
            if (lhs < rhs) {
                set_error("minimum cut below the current density");
                st = DSD_ERR_INTERNAL;
                goto done;
            }
            break;
        }
        tm = now_ns();
        XCU(cudaMemsetAsync(flag, 0, ((size_t)n + 1) * 4, s));
        k_mark_g<<<grid_for_n(W->n), 256, 0, s>>>(W->n, inA, W->old_of, orig, flag);
        note_launch();
        {
            uint64_t check = 0;
            XSTEP(count_in(g, h, flag, &check));
            if (check != muA) {
                set_error("CDS clique count %llu differs from the cut's %llu",
                          (unsigned long long)check, (unsigned long long)muA);
                st = DSD_ERR_INTERNAL;
                goto done;
            }
        }
        I.mu = muA;
        I.size = (uint32_t)sizeA;
    }
    if (cds) {
        XSTEP(dalloc(&pos, (size_t)n + 1, s));
        if (mem == DSD_MEM_HOST) XSTEP(dalloc(&tmp, (size_t)n + 1, s));
        XSTEP(exclusive_scan_u32_to_u64(flag, pos, n, s));
        k_compact_flags<<<grid_for_n(n), 256, 0, s>>>(n, flag, pos, tmp ? tmp : cds);
        note_launch();
        XCU(cudaGetLastError());
        if (tmp) XCU(cudaMemcpyAsync(cds, tmp, (size_t)I.size * 4, cudaMemcpyDeviceToHost, s));
    }
    XCU(cudaStreamSynchronize(s));
    I.verify_ns = now_ns() - tm;
    *info = I;
done:
    net_free(&net, s);
    if (W) dsd_graph_destroy(W);
    {
        void* ptrs[] = {orig, inA, flag, tmp, pos};
        for (void* ptr : ptrs) dev_free(ptr, s);
    }
    return st;
}

}  // extern "C"
