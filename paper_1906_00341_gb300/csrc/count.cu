// h-clique clique-degrees (Def. 3) and mu (Def. 4) over the
// degeneracy-oriented graph.
//
// Every h-clique is listed once, from its lowest-ranked vertex u: it is u
// plus an (h-1)-clique inside N+(u) (vertices are relabelled so that rank =
// id, hence N+(u) is the tail of u's sorted row).  Per vertex u the kernel
// solves the sub-problem of cliques.cuh with root {u}, C = N+(u),
// r = h - 1, and credits the counts with one atomic per (u, x) pair.
//
// Tiers by |N+(u)|:
//   S  <= 32   : one warp per vertex, one-word bitmap rows, lane-level DFS;
//   M  <= 1024 : one block per vertex, 32-word bitmap rows in shared memory;
//   L  >  1024 : one block per vertex; h = 3 needs no bitmap (candidates
//                stay in global memory), h >= 4 splits the set by its next
//                member until it fits (xl.cuh).
// For h = 3 (r = 2) the rows are never materialised: each hit of the row
// scan is a triangle and is counted on the spot.
#include "cliques.cuh"
#include "graph.cuh"
#include "xl.cuh"

namespace dsd {
namespace {

constexpr int kCountThreads = 256;

struct CountArgs {
    uint32_t n;
    int r;  // h - 1
    const uint64_t* off;
    const uint32_t* adj;
    const uint64_t* split;
    unsigned long long* deg;
    unsigned long long* mu;
    uint32_t* listM;      // vertices of tier M
    uint32_t* listL;      // vertices of tier L
    uint32_t* cntML;      // [0] tier M, [1] tier L, [3] checked-mode overflow, [4] tier S
                          // chunks taken, [5] tier M and [6] tier L vertices taken
    uint32_t* work;       // [1] dynamic queue for tier S
    uint32_t* ovf;        // checked mode: set when a counter wraps (else null)
};

// Tier S + classification.  One warp per vertex.
__global__ void __launch_bounds__(kCountThreads) k_count_small(CountArgs A) {
    __shared__ uint32_t sC[kCountThreads / 32][32];
    __shared__ uint32_t sRows[kCountThreads / 32][32];
    __shared__ unsigned sCnt[kCountThreads / 32][32];
    unsigned lane = lane_id(), w = warp_id();
    uint32_t* C = sC[w];
    uint32_t* rows = sRows[w];
    unsigned* cnt = sCnt[w];
    unsigned long long mu_acc = 0;
    const uint32_t chunk = 32;
    for (;;) {
        uint32_t base = 0;
        if (lane == 0) base = atomicAdd(A.work, chunk);
        base = __shfl_sync(0xffffffffu, base, 0);
        if (base >= A.n) break;
        uint32_t end = base + chunk < A.n ? base + chunk : A.n;
        for (uint32_t u = base; u < end; u++) {
            uint64_t b = A.split[u], e = A.off[u + 1];
            uint32_t d = (uint32_t)(e - b);
            if (d < (uint32_t)A.r) continue;            // cannot host a clique
            if (d > 32) {
                if (lane == 0) {
                    int which = d <= kBitmapMax ? 0 : 1;
                    uint32_t at = atomicAdd(&A.cntML[which], 1u);
                    (which ? A.listL : A.listM)[at] = u;
                }
                continue;
            }
            if (lane < d) { C[lane] = A.adj[b + lane]; cnt[lane] = 0; }
            __syncwarp();
            unsigned long long tot;
            if (A.r == 2) {
                // triangles: hits of row i are the third members
                unsigned long long t = 0;
                const uint32_t cmax = C[d - 1];
                for (uint32_t i = 0; i + 1 < d; i++) {
                    uint32_t x = C[i];
                    unsigned hits = scan_row_hits(C, d, cmax, A.adj, A.split[x], A.off[x + 1], cnt);
                    hits = __reduce_add_sync(0xffffffffu, hits);
                    if (lane == 0 && hits) { atomicAdd(&cnt[i], hits); }
                    t += hits;
                }
                tot = t;
            } else {
                warp_build_rows32(C, d, A.off + 1, A.adj, A.split, rows);
                tot = warp_dfs32(rows, d, A.r, cnt);
            }
            __syncwarp();
            if (tot) {
                if (lane < d && cnt[lane])
                    add_counter(&A.deg[C[lane]], (unsigned long long)cnt[lane], A.ovf);
                if (lane == 0) {
                    add_counter(&A.deg[u], tot, A.ovf);
                    if (A.ovf && mu_acc + tot < mu_acc) atomicOr(A.ovf, 1u);
                    mu_acc += tot;
                }
            }
            __syncwarp();
        }
    }
    if (lane == 0 && mu_acc) add_counter(A.mu, mu_acc, A.ovf);
}

// Tier M: one block per vertex, |N+(u)| in (32, 1024].
template <int NT>
__global__ void __launch_bounds__(NT) k_count_medium(CountArgs A) {
    extern __shared__ uint32_t smem[];
    unsigned long long* cnt = reinterpret_cast<unsigned long long*>(smem);  // 1024
    uint32_t* C = smem + 2 * kBitmapMax;      // 1024
    uint32_t* rows = smem + 3 * kBitmapMax;   // up to 1024*32 (only if r >= 3)
    __shared__ unsigned long long s_tot;
    __shared__ uint32_t s_next, s_it;
    uint32_t nM = A.cntML[0];
    // vertices are taken one at a time from a shared counter: their work
    // varies by orders of magnitude
    for (;;) {
        if (threadIdx.x == 0) s_it = atomicAdd(&A.cntML[5], 1u);
        __syncthreads();
        const uint32_t it = s_it;
        if (it >= nM) break;
        uint32_t u = A.listM[it];
        uint64_t b = A.split[u], e = A.off[u + 1];
        uint32_t d = (uint32_t)(e - b);
        uint32_t W = (d + 31) >> 5;
        for (uint32_t i = threadIdx.x; i < d; i += blockDim.x) { C[i] = A.adj[b + i]; cnt[i] = 0; }
        if (A.r >= 3)
            for (uint32_t i = threadIdx.x; i < d * W; i += blockDim.x) rows[i] = 0;
        if (threadIdx.x == 0) {
            s_tot = 0;
            s_next = 0;
        }
        __syncthreads();
        unsigned long long mine = 0;
        if (A.r == 2) {
            unsigned lane = lane_id(), nw = blockDim.x >> 5;
            const uint32_t cmax = C[d - 1];
            for (uint32_t i = warp_id(); i + 1 < d; i += nw) {
                uint32_t x = C[i];
                unsigned hits = scan_row_hits(C, d, cmax, A.adj, A.split[x], A.off[x + 1], cnt);
                hits = __reduce_add_sync(0xffffffffu, hits);
                if (lane == 0 && hits) atomicAdd(&cnt[i], (unsigned long long)hits);
                if (lane == 0) mine += hits;
            }
        } else {
            block_build_rows(C, d, W, A.off + 1, A.adj, A.split, rows);
            __syncthreads();
            mine = block_dfs(rows, d, W, A.r, cnt, &s_next);
        }
        if (mine) atomicAdd(&s_tot, mine);
        __syncthreads();
        unsigned long long tot = s_tot;
        if (tot) {
            for (uint32_t i = threadIdx.x; i < d; i += blockDim.x)
                if (cnt[i]) add_counter(&A.deg[C[i]], cnt[i], A.ovf);
            if (threadIdx.x == 0) {
                add_counter(&A.deg[u], tot, A.ovf);
                add_counter(A.mu, tot, A.ovf);
            }
        }
        __syncthreads();
    }
}

// Tier M in decreasing |N+(u)|, so that the largest searches start first and
// the last vertices taken are short: a counting sort over d in (32, 1024]
// (order inside one d is arbitrary; the counts do not depend on it).
__global__ void k_m_hist(CountArgs A, uint32_t* hist) {
    const uint32_t nM = A.cntML[0];
    for (uint32_t it = blockIdx.x * blockDim.x + threadIdx.x; it < nM; it += gridDim.x * blockDim.x) {
        const uint32_t u = A.listM[it];
        const uint32_t d = (uint32_t)(A.off[u + 1] - A.split[u]);
        atomicAdd(&hist[kBitmapMax - d], 1u);
    }
}
// one block of kBitmapMax threads: hist -> exclusive starts
__global__ void __launch_bounds__(kBitmapMax) k_m_starts(uint32_t* hist) {
    __shared__ uint32_t s_w[kBitmapMax / 32];
    const unsigned lane = lane_id(), wid = warp_id();
    const uint32_t x = hist[threadIdx.x];
    uint32_t inc = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if ((int)lane >= o) inc += y;
    }
    if (lane == 31) s_w[wid] = inc;
    __syncthreads();
    uint32_t before = 0;
    for (unsigned w = 0; w < wid; w++) before += s_w[w];
    hist[threadIdx.x] = before + inc - x;
}
__global__ void k_m_place(CountArgs A, uint32_t* start, uint32_t* out) {
    const uint32_t nM = A.cntML[0];
    for (uint32_t it = blockIdx.x * blockDim.x + threadIdx.x; it < nM; it += gridDim.x * blockDim.x) {
        const uint32_t u = A.listM[it];
        const uint32_t d = (uint32_t)(A.off[u + 1] - A.split[u]);
        out[atomicAdd(&start[kBitmapMax - d], 1u)] = u;
    }
}

// Tier L (h = 3 only): |N+(u)| > 1024; candidates stay in global memory and
// the credits go straight to the global counters.
__global__ void __launch_bounds__(kCountThreads) k_count_large3(CountArgs A) {
    __shared__ unsigned long long s_tot;
    __shared__ uint32_t s_it;
    uint32_t nL = A.cntML[1];
    unsigned lane = lane_id(), nw = blockDim.x >> 5;
    for (;;) {
        if (threadIdx.x == 0) s_it = atomicAdd(&A.cntML[6], 1u);
        __syncthreads();
        const uint32_t it = s_it;
        if (it >= nL) break;
        uint32_t u = A.listL[it];
        uint64_t b = A.split[u], e = A.off[u + 1];
        uint32_t d = (uint32_t)(e - b);
        const uint32_t* C = A.adj + b;
        if (threadIdx.x == 0) s_tot = 0;
        __syncthreads();
        unsigned long long mine = 0;
        for (uint32_t i = warp_id(); i < d; i += nw) {
            uint32_t x = C[i];
            uint64_t xb = A.split[x], xe = A.off[x + 1];
            unsigned hits = 0;
            for (uint64_t p = xb + lane; p < xe; p += 32) {
                uint32_t y = A.adj[p];
                uint64_t pos = lower_bound_u32(C, d, y);
                if (pos < d && C[pos] == y) { add_counter(&A.deg[y], 1ull, A.ovf); hits++; }
            }
            hits = __reduce_add_sync(0xffffffffu, hits);
            if (lane == 0 && hits) {
                add_counter(&A.deg[x], (unsigned long long)hits, A.ovf);
                mine += hits;
            }
        }
        if (mine) atomicAdd(&s_tot, mine);
        __syncthreads();
        if (threadIdx.x == 0 && s_tot) {
            add_counter(&A.deg[u], s_tot, A.ovf);
            add_counter(A.mu, s_tot, A.ovf);
        }
        __syncthreads();
    }
}

// Tier L for h >= 4: |N+(u)| > 1024, one block per vertex; the candidate
// set is split by its next member until it fits the bitmap tier (xl.cuh).
// scratch: kMaxDepth * cap entries per block.
__global__ void __launch_bounds__(1024) k_count_xl(CountArgs A, uint32_t* scratch, uint32_t cap) {
    extern __shared__ uint32_t smem[];
    __shared__ unsigned long long s_root;
    __shared__ uint32_t s_it;
    uint32_t* mine = scratch + (size_t)blockIdx.x * kMaxDepth * cap;
    const uint32_t nL = A.cntML[1];
    for (;;) {
        if (threadIdx.x == 0) s_it = atomicAdd(&A.cntML[6], 1u);
        __syncthreads();
        const uint32_t it = s_it;
        if (it >= nL) break;
        const uint32_t u = A.listL[it];
        const uint64_t b = A.split[u], e = A.off[u + 1];
        if (threadIdx.x == 0) s_root = 0;
        __syncthreads();
        xl_cliques(
            A.adj + b, (uint32_t)(e - b), A.r, A.split, A.off + 1, A.adj, mine, cap, smem,
            [&](uint32_t x, unsigned long long c) { add_counter(&A.deg[x], c, A.ovf); },
            [&](unsigned long long c) { s_root += c; });
        __syncthreads();
        if (threadIdx.x == 0 && s_root) {
            add_counter(&A.deg[u], s_root, A.ovf);
            add_counter(A.mu, s_root, A.ovf);
        }
        __syncthreads();
    }
}

__global__ void k_degree_as_count(uint32_t n, const uint64_t* off, unsigned long long* deg) {
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
        deg[v] = off[v + 1] - off[v];
}

// Algorithmic bytes of the listing, two models (per launch of the count):
// out[0], the kernels' own staging: offsets and split read once per vertex,
// each N+(u) read once (it is staged in shared memory), each N+(x) read once
// per oriented edge (u, x), one 8-byte read-modify-write per counter that
// can be credited (u and every x), the 8-byte zero-fill of deg;
// out[1], a merge intersection's: both lists of every oriented edge,
// 4 (d+(u) + d+(x)), plus 8 (n+1) offsets, 4 m oriented entries and the
// 8 n counters written.  Bitmap searches below the first level (h >= 4)
// stay in shared memory and are in neither.
__global__ void k_count_bytes(uint32_t n, const uint64_t* off, const uint32_t* adj,
                              const uint64_t* split, unsigned long long* out) {
    unsigned long long acc = 0, mrg = 0;
    for (uint32_t u = blockIdx.x * blockDim.x + threadIdx.x; u < n; u += gridDim.x * blockDim.x) {
        uint64_t b = split[u], e = off[u + 1];
        acc += 16 + 4 * (e - b);              // off + split, N+(u)
        for (uint64_t p = b; p < e; p++) {
            uint32_t x = adj[p];
            uint64_t dx = off[x + 1] - split[x];
            acc += 16 + 4 * dx;               // off/split of x, N+(x)
            acc += 16;                        // counter of x
            mrg += 4 * ((e - b) + dx);
        }
        acc += 16 + 8;                        // counter of u, its zero-fill
        mrg += 8 + 4 * (e - b) + 8;
    }
    acc = warp_sum(acc);
    mrg = warp_sum(mrg);
    if (lane_id() == 0) {
        atomicAdd(out, acc);
        atomicAdd(out + 1, mrg);
    }
}

}  // namespace

dsd_status count_cliques(dsd_graph* g, int h, unsigned long long* deg_new,
                         unsigned long long* mu_dev) {
    cudaStream_t s = g->stream;
    int sms = 152;
    DSD_TRY(num_sms(&sms));
    uint32_t n = g->n;
    DSD_CU(cudaMemsetAsync(deg_new, 0, (size_t)n * 8 + 8, s));
    DSD_CU(cudaMemsetAsync(mu_dev, 0, 8, s));
    if (n == 0) return DSD_OK;
    if (h == 2) {
        k_degree_as_count<<<sms * 8, 256, 0, s>>>(n, g->roff, deg_new); note_launch();
        DSD_LAUNCHED();
        unsigned long long m2 = g->m;
        DSD_CU(cudaMemcpyAsync(mu_dev, &m2, 8, cudaMemcpyHostToDevice, s));
        DSD_CU(cudaStreamSynchronize(s));
        return DSD_OK;
    }
    CountArgs A;
    A.n = n;
    A.r = h - 1;
    A.off = g->roff;
    A.adj = g->radj;
    A.split = g->rsplit;
    A.deg = deg_new;
    A.mu = mu_dev;
    uint32_t* ws = nullptr;
    uint32_t* xl_scratch = nullptr;
    DSD_TRY(dalloc(&ws, (size_t)3 * n + 8 + kBitmapMax, s));
    A.listM = ws;
    A.listL = ws + n;
    A.cntML = ws + 2 * (size_t)n;
    A.work = A.cntML + 4;
    A.ovf = checked_mode() ? A.cntML + 3 : nullptr;
    dsd_status st = DSD_OK;
    cudaError_t e = cudaMemsetAsync(A.cntML, 0, 8 * sizeof(uint32_t), s);
    if (e == cudaSuccess) {
        k_count_small<<<sms * 8, kCountThreads, 0, s>>>(A); note_launch();
        {
            // tier M by decreasing |N+(u)|
            uint32_t* hist = A.cntML + 8;
            uint32_t* sorted = hist + kBitmapMax;
            e = cudaMemsetAsync(hist, 0, kBitmapMax * sizeof(uint32_t), s);
            if (e == cudaSuccess) {
                k_m_hist<<<sms * 4, 256, 0, s>>>(A, hist);
                k_m_starts<<<1, kBitmapMax, 0, s>>>(hist);
                k_m_place<<<sms * 4, 256, 0, s>>>(A, hist, sorted);
                for (int i = 0; i < 3; i++) note_launch();
                A.listM = sorted;
            }
        }
        size_t smemM = (size_t)3 * kBitmapMax * 4 + (h >= 4 ? (size_t)kBitmapMax * 32 * 4 : 0);
        if (h >= 4) {
            // one block per SM (the rows fill its shared memory): 32 warps
            cudaFuncSetAttribute(k_count_medium<1024>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smemM);
            k_count_medium<1024><<<sms, 1024, smemM, s>>>(A);
        } else {
            k_count_medium<kCountThreads><<<sms * 4, kCountThreads, smemM, s>>>(A);
        }
        note_launch();
        if (h == 3) {
            k_count_large3<<<sms * 4, kCountThreads, 0, s>>>(A);
            note_launch();
        } else if (g->maxdplus > kBitmapMax && e == cudaSuccess) {
            e = cudaGetLastError();
            const uint32_t cap = g->maxdplus;
            if (e == cudaSuccess && dalloc(&xl_scratch, (size_t)sms * kMaxDepth * cap, s) != DSD_OK)
                e = cudaErrorMemoryAllocation;
            if (e == cudaSuccess) {
                cudaFuncSetAttribute(k_count_xl, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smemM);
                k_count_xl<<<sms, 1024, smemM, s>>>(A, xl_scratch, cap);
                note_launch();
            }
        }
        if (e == cudaSuccess) e = cudaGetLastError();
    }
    uint32_t flags[2] = {0, 0};   // (unused), counter overflow
    if (e == cudaSuccess) e = cudaMemcpyAsync(flags, A.cntML + 2, 8, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    dev_free(ws, s);
    dev_free(xl_scratch, s);
    if (e != cudaSuccess) return cuda_fail(e, "clique count", __FILE__, __LINE__);
    if (flags[1]) {
        set_error("h=%d: a clique-degree or mu exceeds 2^64 - 1 (checked mode)", h);
        return DSD_ERR_OVERFLOW;
    }
    g->prof_launches[kPhaseCount] = h == 3 ? 6 : (g->maxdplus > kBitmapMax ? 6 : 5);
    return st;
}

namespace {
// Adds addends[0..count) one after another into a counter starting at
// start, through the checked addition of the counting kernels.
__global__ void k_checked_add_probe(unsigned long long start, const unsigned long long* addends,
                                    uint32_t count, unsigned long long* out, uint32_t* ovf) {
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    *out = start;
    for (uint32_t i = 0; i < count; i++) add_counter(out, addends[i], ovf);
}
}  // namespace

dsd_status checked_add_selftest(uint64_t start, const uint64_t* addends, uint32_t count,
                                uint64_t* sum, int* overflowed) {
    unsigned long long* d = nullptr;
    DSD_TRY(dalloc(&d, (size_t)count + 2, nullptr));
    uint32_t* ovf = reinterpret_cast<uint32_t*>(d + count + 1);
    cudaError_t e = cudaMemset(ovf, 0, 4);
    if (e == cudaSuccess && count)
        e = cudaMemcpy(d, addends, (size_t)count * 8, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        k_checked_add_probe<<<1, 32>>>(start, d, count, d + count, ovf);
        note_launch();
        e = cudaGetLastError();
    }
    unsigned long long out = 0;
    uint32_t flag = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&out, d + count, 8, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(&flag, ovf, 4, cudaMemcpyDeviceToHost);
    dev_free(d, nullptr);
    if (e != cudaSuccess) return cuda_fail(e, "checked add self-test", __FILE__, __LINE__);
    *sum = out;
    *overflowed = flag ? 1 : 0;
    return DSD_OK;
}

dsd_status count_bytes(dsd_graph* g, uint64_t* staged, uint64_t* merge) {
    DSD_TRY(ensure_order(g));
    cudaStream_t s = g->stream;
    unsigned long long* d = nullptr;
    DSD_TRY(dalloc(&d, 2, s));
    DSD_CU(cudaMemsetAsync(d, 0, 16, s));
    int sms = 152;
    num_sms(&sms);
    k_count_bytes<<<sms * 8, 256, 0, s>>>(g->n, g->roff, g->radj, g->rsplit, d); note_launch();
    unsigned long long h[2] = {0, 0};
    cudaError_t e = cudaMemcpyAsync(h, d, 16, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    dev_free(d, s);
    if (e != cudaSuccess) return cuda_fail(e, "count bytes", __FILE__, __LINE__);
    if (staged) *staged = h[0];
    if (merge) *merge = h[1] + 8;   // the final offset
    return DSD_OK;
}

}  // namespace dsd
