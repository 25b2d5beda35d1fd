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
                        kind[a] = kArcRev;
                        rev[a] = bpos;
                        to[bpos] = (uint32_t)node;
                        kind[bpos] = kArcQ;
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
                kind[a] = kArcInf;
                rev[a] = bpos;
                to[bpos] = (uint32_t)node;
                kind[bpos] = kArcRev;
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
        to[sa] = 2 + (uint32_t)v; kind[sa] = kArcS; rev[sa] = v0;
        to[v0] = 0;               kind[v0] = kArcRev; rev[v0] = sa;
        to[v1] = 1;               kind[v1] = kArcT; rev[v1] = ta;
        to[ta] = 2 + (uint32_t)v; kind[ta] = kArcRev; rev[ta] = v1;
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
        switch (kind[a]) {
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
// the round's start, then each node still holding excess is relabelled to
// 1 + the least height over its residual arcs, read from the same snapshot
// and written to a separate buffer.  A push on x -> y needs h(x) = h(y) + 1
// and one on y -> x the reverse, so no arc pair is pushed from both ends in
// a round.  Every few rounds the heights are replaced by exact residual
// distances to t (backward breadth-first search), nodes that cannot reach t
// getting N.  With no active node left the preflow is maximum, and the nodes
// that still reach t form the smallest sink side of a minimum cut.

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

__global__ void k_bfs_init(uint64_t N, uint32_t* height, uint32_t* frontier, uint32_t* nf) {
    for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < N;
         x += (uint64_t)gridDim.x * blockDim.x)
        height[x] = x == 1 ? 0u : kUnset;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        frontier[0] = 1;
        *nf = 1;
    }
}

// Warp per frontier node y at distance d: every x with residual x -> y (the
// twin of y -> x) and no distance yet gets d + 1.  s is never entered.
__global__ void k_bfs_step(const uint32_t* fin, const uint32_t* nfin, uint32_t* fout,
                           uint32_t* nfout, uint32_t d, const uint64_t* head, const uint32_t* to,
                           const uint64_t* rev, const unsigned long long* cf, uint32_t* height) {
    uint64_t gw = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    unsigned lane = lane_id();
    const uint32_t n_in = *nfin;
    for (uint64_t i = gw; i < n_in; i += nw) {
        uint32_t y = fin[i];
        for (uint64_t p0 = head[y]; p0 < head[y + 1]; p0 += 32) {
            uint64_t e = p0 + lane;
            bool add = false;
            uint32_t x = 0;
            if (e < head[y + 1]) {
                x = to[e];
                if (x != 0 && cf[rev[e]] > 0 && height[x] == kUnset)
                    add = atomicCAS(&height[x], kUnset, d + 1) == kUnset;
            }
            warp_append(add, x, fout, nfout);
        }
    }
}

__global__ void k_bfs_finish(uint64_t N, uint32_t* height) {
    for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < N;
         x += (uint64_t)gridDim.x * blockDim.x)
        if (x == 0 || height[x] == kUnset) height[x] = (uint32_t)N;
}

__global__ void k_collect(uint64_t N, const unsigned long long* excess, const uint32_t* height,
                          uint32_t* list, uint32_t* nlist) {
    for (uint64_t x0 = (uint64_t)blockIdx.x * blockDim.x; x0 < N;
         x0 += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t x = x0 + threadIdx.x;
        bool act = x >= 2 && x < N && excess[x] > 0 && height[x] < N;
        warp_append(act, (uint32_t)x, list, nlist);
    }
}

__device__ __forceinline__ unsigned long long sat_add(unsigned long long a, unsigned long long b) {
    unsigned long long c = a + b;
    return c < a ? ~0ull : c;
}

// Warp per active node u.
__global__ void k_push(const uint32_t* list, const uint32_t* nlist, const uint64_t* head,
                       const uint32_t* to, const uint64_t* rev, unsigned long long* cf,
                       unsigned long long* excess, const uint32_t* height) {
    uint64_t gw = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    unsigned lane = lane_id();
    const uint32_t n = *nlist;
    for (uint64_t i = gw; i < n; i += nw) {
        uint32_t u = list[i];
        const unsigned long long e0 = excess[u];
        const uint32_t hu = height[u];
        unsigned long long rem = e0;
        for (uint64_t p0 = head[u]; p0 < head[u + 1] && rem > 0; p0 += 32) {
            uint64_t a = p0 + lane;
            unsigned long long c = 0;
            uint32_t v = 0;
            if (a < head[u + 1]) {
                v = to[a];
                unsigned long long ca = cf[a];
                if (ca > 0 && height[v] + 1 == hu) c = ca;
            }
            // inclusive prefix of c over the lanes (saturating)
            unsigned long long incl = c;
            for (int o = 1; o < 32; o <<= 1) {
                unsigned long long y = __shfl_up_sync(0xffffffffu, incl, o);
                if ((int)lane >= o) incl = sat_add(incl, y);
            }
            // exact unless saturated, and a saturated sum leaves excl far
            // above any excess (capacities < 2^63, excess < 2^61)
            unsigned long long excl = incl - c;
            unsigned long long d = 0;
            if (c > 0 && excl < rem) d = c < rem - excl ? c : rem - excl;
            if (d) {
                atomicAdd(&cf[a], (unsigned long long)(-(long long)d));
                atomicAdd(&cf[rev[a]], d);
                atomicAdd(&excess[v], d);
            }
            unsigned long long tot = warp_sum(d);
            rem -= tot;
        }
        if (lane == 0 && rem != e0) atomicAdd(&excess[u], (unsigned long long)(-(long long)(e0 - rem)));
    }
}

// Warp per active node: new height (into nh[i]) for nodes still holding
// excess, from the heights of the round's start.
__global__ void k_relabel(const uint32_t* list, const uint32_t* nlist, uint64_t N,
                          const uint64_t* head, const uint32_t* to,
                          const unsigned long long* cf, const unsigned long long* excess,
                          const uint32_t* height, uint32_t* nh) {
    uint64_t gw = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    unsigned lane = lane_id();
    const uint32_t n = *nlist;
    for (uint64_t i = gw; i < n; i += nw) {
        uint32_t u = list[i];
        uint32_t hu = height[u];
        if (excess[u] == 0) {
            if (lane == 0) nh[i] = hu;
            continue;
        }
        uint32_t m = kUnset;
        for (uint64_t a = head[u] + lane; a < head[u + 1]; a += 32)
            if (cf[a] > 0) {
                uint32_t hv = height[to[a]];
                m = hv < m ? hv : m;
            }
        for (int o = 16; o > 0; o >>= 1) {
            uint32_t y = __shfl_xor_sync(0xffffffffu, m, o);
            m = y < m ? y : m;
        }
        if (lane == 0) {
            uint64_t nv = m == kUnset ? N : (uint64_t)m + 1;
            if (nv > N) nv = N;
            if (nv < hu) nv = hu;
            nh[i] = (uint32_t)nv;
        }
    }
}

__global__ void k_apply(const uint32_t* list, const uint32_t* nlist, const uint32_t* nh,
                        uint32_t* height) {
    const uint32_t n = *nlist;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x)
        height[list[i]] = nh[i];
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

// Backward breadth-first search from t: exact residual distances to t,
// N for nodes that cannot reach it (and for s).
dsd_status global_relabel(const Net& net, cudaStream_t s, uint32_t* height, uint32_t* fa,
                          uint32_t* fb, uint32_t* ctr) {
    k_bfs_init<<<grid_for_n(net.N), 256, 0, s>>>(net.N, height, fa, ctr); note_launch();
    uint32_t nf = 1, d = 0;
    while (nf) {
        DSD_CU(cudaMemsetAsync(ctr + 1, 0, 4, s));
        k_bfs_step<<<grid_for_warps(nf), 256, 0, s>>>(fa, ctr, fb, ctr + 1, d, net.head, net.to,
                                                      net.rev, net.cf, height);
        note_launch();
        DSD_CU(cudaMemcpyAsync(ctr, ctr + 1, 4, cudaMemcpyDeviceToDevice, s));
        DSD_CU(cudaMemcpyAsync(&nf, ctr + 1, 4, cudaMemcpyDeviceToHost, s));
        DSD_CU(cudaStreamSynchronize(s));
        uint32_t* t = fa;
        fa = fb;
        fb = t;
        d++;
        if (d > net.N) {
            set_error("breadth-first search did not settle");
            return DSD_ERR_INTERNAL;
        }
    }
    k_bfs_finish<<<grid_for_n(net.N), 256, 0, s>>>(net.N, height); note_launch();
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
    unsigned long long* excess = nullptr;
    uint32_t *height = nullptr, *list = nullptr, *nh = nullptr, *fa = nullptr, *fb = nullptr,
             *ctr = nullptr;
    unsigned long long* cnt = nullptr;
    const uint64_t t0 = now_ns();
    const uint64_t limit_rounds = 4 * N + 100000;
    const int kRoundsPerRelabel = 8;
    XSTEP(dalloc(&excess, N + 1, s));
    XSTEP(dalloc(&height, N + 1, s));
    XSTEP(dalloc(&list, N + 1, s));
    XSTEP(dalloc(&nh, N + 1, s));
    XSTEP(dalloc(&fa, N + 1, s));
    XSTEP(dalloc(&fb, N + 1, s));
    XSTEP(dalloc(&ctr, 4, s));
    XSTEP(dalloc(&cnt, 1, s));
    k_caps<<<grid_for_n(net.E), 256, 0, s>>>(net.E, net.kind, net.to, net.vdeg, p, q, h, net.cf);
    note_launch();
    XCU(cudaMemsetAsync(excess, 0, (N + 1) * 8, s));
    k_preflow<<<grid_for_n(net.nW), 256, 0, s>>>(net.nW, net.head, net.rev, net.cf, excess);
    note_launch();
    XSTEP(global_relabel(net, s, height, fa, fb, ctr));
    cs->relabels++;
    for (;;) {
        uint32_t nact = 0;
        XCU(cudaMemsetAsync(ctr + 2, 0, 4, s));
        k_collect<<<grid_for_n(N), 256, 0, s>>>(N, excess, height, list, ctr + 2); note_launch();
        XSTEP(read_back(&nact, ctr + 2, s));
        if (nact == 0) break;
        for (int it = 0; it < kRoundsPerRelabel; it++) {
            if (it) {
                XCU(cudaMemsetAsync(ctr + 2, 0, 4, s));
                k_collect<<<grid_for_n(N), 256, 0, s>>>(N, excess, height, list, ctr + 2);
                note_launch();
            }
            const unsigned gw = grid_for_warps(nact);
            k_push<<<gw, 256, 0, s>>>(list, ctr + 2, net.head, net.to, net.rev, net.cf, excess,
                                      height);
            k_relabel<<<gw, 256, 0, s>>>(list, ctr + 2, N, net.head, net.to, net.cf, excess,
                                         height, nh);
            k_apply<<<grid_for_n(nact), 256, 0, s>>>(list, ctr + 2, nh, height);
            note_launch();
            note_launch();
            note_launch();
            cs->rounds++;
        }
        XCU(cudaGetLastError());
        XSTEP(global_relabel(net, s, height, fa, fb, ctr));
        cs->relabels++;
        if (cs->rounds > limit_rounds || now_ns() - t0 > wait_limit_ns()) {
            set_error("push-relabel did not finish within %llu rounds / the wait limit",
                      (unsigned long long)limit_rounds);
            st = DSD_ERR_TIMEOUT;
            goto done;
        }
    }
    XSTEP(read_back(flow, excess + 1, s));
    XCU(cudaMemsetAsync(cnt, 0, 8, s));
    if (net.nW) {
        k_source_side<<<grid_for_n(net.nW), 256, 0, s>>>(net.nW, height, N, inA, cnt);
        note_launch();
    }
    {
        unsigned long long a = 0;
        XSTEP(read_back(&a, cnt, s));
        *sizeA = a;
    }
done:
    {
        void* ptrs[] = {excess, height, list, nh, fa, fb, ctr, cnt};
        for (void* ptr : ptrs) dev_free(ptr, s);
    }
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
                XSTEP(located_core(g, core, k, &W, &orig));
                XSTEP(build_network(W, h, &net));
                XSTEP(dalloc(&inA, (size_t)W->n + 1, s));
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
            XSTEP(min_cut(net, h, p, q, s, &F, inA, &sizeA, &cs));
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
