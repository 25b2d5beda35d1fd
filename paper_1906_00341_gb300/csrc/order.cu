// Degeneracy order and orientation.
//
// The first stage runs the level-synchronous peel with h = 2, which yields the edge
// k-core numbers (Def. 5; the h = 2 case of the decomposition) and the round
// in which each vertex left.  Vertices are then ranked by (round, id): a
// vertex removed at level k had at most k alive neighbours, all of which are
// ranked after it or in its own round, so orienting every edge from lower to
// higher rank leaves each vertex with at most degeneracy-many out-neighbours.
// The core-number bound gamma(v) = C(core_2(v), h-1) used by CoreApp
// (Sec. 5.2) rests on the same core numbers.
//
// The second stage relabels vertices by rank and rebuilds the CSR with sorted rows, so that
// N+(v) = {u in N(v) : u > v} is the tail of row v (start kept in rsplit).
#include "graph.cuh"

#include <vector>

namespace dsd {
namespace {

__global__ void k_row_lengths(uint32_t n, const uint64_t* off, unsigned long long* deg) {
    for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (uint64_t)gridDim.x * blockDim.x)
        deg[v] = off[v + 1] - off[v];
}

__global__ void k_round_hist(uint32_t n, const uint32_t* rnd, uint32_t* hist) {
    for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (uint64_t)gridDim.x * blockDim.x)
        atomicAdd(&hist[rnd[v]], 1u);
}

__global__ void k_round_scatter(uint32_t n, const uint32_t* rnd, const uint64_t* start,
                                uint32_t* cursor, uint32_t* out) {
    for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t r = rnd[v];
        out[start[r] + atomicAdd(&cursor[r], 1u)] = (uint32_t)v;
    }
}

// A round of more than kHugeRound members: flag[v] = 1 iff v left in it; the
// members then go to their place in id order through a scan of the flags
// (1M-vertex Chung-Lu graph: orientation 5.4 -> 3.1 ms at this threshold,
// 3.9 ms at 65,536; each such round costs a handful of launches).
constexpr uint32_t kHugeRound = 16384;
__global__ void k_round_flag(uint32_t n, const uint32_t* rnd, uint32_t r, uint32_t* flag) {
    for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (uint64_t)gridDim.x * blockDim.x)
        flag[v] = rnd[v] == r ? 1u : 0u;
}
__global__ void k_round_place(uint32_t n, const uint32_t* rnd, uint32_t r, const uint64_t* pos,
                              const uint64_t* start, uint32_t* out) {
    for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (uint64_t)gridDim.x * blockDim.x)
        if (rnd[v] == r) out[start[r] + pos[v]] = (uint32_t)v;
}

__global__ void k_invert(uint32_t n, const uint32_t* old_of, uint32_t* new_of,
                         const uint64_t* off, uint32_t* rdeg) {
    for (uint64_t p = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n;
         p += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t o = old_of[p];
        new_of[o] = (uint32_t)p;
        rdeg[p] = (uint32_t)(off[o + 1] - off[o]);
    }
}

// Warp per relabelled row: translate the neighbour ids.
__global__ void k_fill_rows(uint32_t n, const uint32_t* old_of, const uint32_t* new_of,
                            const uint64_t* off, const uint32_t* adj, const uint64_t* roff,
                            uint32_t* radj) {
    uint64_t gw = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    unsigned lane = lane_id();
    for (uint64_t p = gw; p < n; p += nw) {
        uint32_t o = old_of[p];
        uint64_t b = off[o], l = off[o + 1] - b, d = roff[p];
        for (uint64_t j = lane; j < l; j += 32) radj[d + j] = new_of[adj[b + j]];
    }
}

// Warp per row: split = first entry greater than the row's own id; track the
// largest out-degree.
__global__ void k_split(uint32_t n, const uint64_t* roff, const uint32_t* radj, uint64_t* split,
                        uint32_t* maxdplus) {
    uint64_t gw = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    unsigned lane = lane_id();
    uint32_t best = 0;
    for (uint64_t p = gw; p < n; p += nw) {
        uint64_t b = roff[p], e = roff[p + 1];
        uint64_t at = b + lower_bound_u32(radj + b, e - b, (uint32_t)p + 1u);
        if (lane == 0) {
            split[p] = at;
            uint32_t dp = (uint32_t)(e - at);
            best = dp > best ? dp : best;
        }
    }
    if (lane == 0 && best) atomicMax(maxdplus, best);
}

}  // namespace

dsd_status ensure_order(dsd_graph* g) {
    if (g->ordered) return DSD_OK;
    cudaStream_t s = g->stream;
    uint32_t n = g->n;
    int sms = 152;
    DSD_TRY(num_sms(&sms));
    unsigned grid = (unsigned)sms * 8;
    dsd_status st = DSD_OK;
    unsigned long long* deg = nullptr;
    uint32_t* hist = nullptr;
    uint64_t* start = nullptr;
    uint32_t* rdeg = nullptr;
    uint32_t* tmp = nullptr;
    uint32_t* dmax = nullptr;
    PeelResult pr;
    std::vector<uint32_t> hh;
    uint32_t R = 0;
    uint32_t hmax = 0;
#define STEP(x)                      \
    do {                             \
        st = (x);                    \
        if (st != DSD_OK) goto done; \
    } while (0)
#define CUSTEP(x)                                                          \
    do {                                                                   \
        cudaError_t e_ = (x);                                              \
        if (e_ != cudaSuccess) { st = cuda_fail(e_, #x, __FILE__, __LINE__); goto done; } \
    } while (0)
    STEP(dalloc(&g->core2, (size_t)n + 1, s));
    STEP(dalloc(&g->rnd, (size_t)n + 1, s));
    STEP(dalloc(&g->new_of, (size_t)n + 1, s));
    STEP(dalloc(&g->old_of, (size_t)n + 1, s));
    STEP(dalloc(&g->roff, (size_t)n + 1, s));
    STEP(dalloc(&g->radj, 2 * g->m + 1, s));
    STEP(dalloc(&g->rsplit, (size_t)n + 1, s));
    STEP(dalloc(&g->lvl2_k, (size_t)n + 1, s));
    STEP(dalloc(&g->lvl2_size, (size_t)n + 1, s));
    STEP(dalloc(&g->lvl2_mu, (size_t)n + 1, s));
    STEP(dalloc(&deg, (size_t)n + 1, s));
    if (n == 0) {
        CUSTEP(cudaMemsetAsync(g->roff, 0, 8, s));
        g->ordered = true;
        goto done;
    }
    // edge core numbers and removal rounds
    prof_begin(g, kPhaseOrderPeel);
    k_row_lengths<<<grid, 256, 0, s>>>(n, g->off, deg); note_launch();
    CUSTEP(cudaGetLastError());
    STEP(run_peel(g, 2, n, g->off, g->adj, nullptr, 0, deg, g->m, g->core2, g->rnd, g->lvl2_k,
                  g->lvl2_size, g->lvl2_mu, &pr));
    prof_end(g, kPhaseOrderPeel);
    g->prof_launches[kPhaseOrderPeel] = 3;
    g->degeneracy = (uint32_t)pr.kmax;
    g->order_kmax = pr.kmax;
    g->nlevels2 = pr.nlevels;
    g->prof_bytes[kPhaseOrderPeel] = pr.bytes;
    record_peel(g, 0, pr);
    R = pr.rounds + 1;

    // rank by (round, id), relabel, rebuild rows
    prof_begin(g, kPhaseOrient);
    STEP(dalloc(&hist, (size_t)R + 1, s));
    STEP(dalloc(&start, (size_t)R + 1, s));
    STEP(dalloc(&rdeg, (size_t)n + 1, s));
    // scratch for the per-round sort (n entries) and the row sort (2m entries)
    STEP(dalloc(&tmp, (2 * g->m > n ? 2 * g->m : (uint64_t)n) + 1, s));
    STEP(dalloc(&dmax, 1, s));
    CUSTEP(cudaMemsetAsync(hist, 0, ((size_t)R + 1) * 4, s));
    k_round_hist<<<grid, 256, 0, s>>>(n, g->rnd, hist); note_launch();
    CUSTEP(cudaGetLastError());
    STEP(exclusive_scan_u32_to_u64(hist, start, R, s));
    CUSTEP(cudaMemsetAsync(rdeg, 0, ((size_t)n + 1) * 4, s));
    k_round_scatter<<<grid, 256, 0, s>>>(n, g->rnd, start, rdeg, g->old_of); note_launch();
    CUSTEP(cudaGetLastError());
    // the largest rounds (the first ones of a large graph) in id order by a
    // flag scan over all vertices, each over the whole GPU, rather than by the
    // row sort's one block per row; their rows are then left out of the sort
    hh.resize(R);
    CUSTEP(cudaMemcpyAsync(hh.data(), hist, (size_t)R * 4, cudaMemcpyDeviceToHost, s));
    CUSTEP(cudaStreamSynchronize(s));
    for (uint32_t r = 0; r < R; r++) {
        if (hh[r] <= kHugeRound) continue;
        uint64_t* fpos = reinterpret_cast<uint64_t*>(deg);   // free after the peel
        k_round_flag<<<grid, 256, 0, s>>>(n, g->rnd, r, tmp); note_launch();
        CUSTEP(cudaGetLastError());
        STEP(exclusive_scan_u32_to_u64(tmp, fpos, n, s));
        k_round_place<<<grid, 256, 0, s>>>(n, g->rnd, r, fpos, start, g->old_of); note_launch();
        CUSTEP(cudaGetLastError());
        CUSTEP(cudaMemsetAsync(hist + r, 0, 4, s));
    }
    // rows = rounds; sort the members of each round by id (distinct ids)
    STEP(segmented_sort_unique(g->old_of, tmp, start, hist, rdeg, R, n, s));
    k_invert<<<grid, 256, 0, s>>>(n, g->old_of, g->new_of, g->off, rdeg); note_launch();
    CUSTEP(cudaGetLastError());
    STEP(exclusive_scan_u32_to_u64(rdeg, g->roff, n, s));
    k_fill_rows<<<grid, 256, 0, s>>>(n, g->old_of, g->new_of, g->off, g->adj, g->roff, g->radj); note_launch();
    CUSTEP(cudaGetLastError());
    {
        // rows have distinct entries; reuse hist as the (ignored) unique counts
        uint32_t* ulen = nullptr;
        STEP(dalloc(&ulen, (size_t)n + 1, s));
        st = segmented_sort_unique(g->radj, tmp, g->roff, rdeg, ulen, n, 2 * g->m, s);
        dev_free(ulen, s);
        if (st != DSD_OK) goto done;
    }
    CUSTEP(cudaMemsetAsync(dmax, 0, 4, s));
    k_split<<<grid, 256, 0, s>>>(n, g->roff, g->radj, g->rsplit, dmax); note_launch();
    CUSTEP(cudaGetLastError());
    CUSTEP(cudaMemcpyAsync(&hmax, dmax, 4, cudaMemcpyDeviceToHost, s));
    CUSTEP(cudaStreamSynchronize(s));
    g->maxdplus = hmax;
    prof_end(g, kPhaseOrient);
    g->prof_launches[kPhaseOrient] = 12;
    g->ordered = true;
done:
#undef STEP
#undef CUSTEP
    dev_free(deg, s);
    dev_free(hist, s);
    dev_free(start, s);
    dev_free(rdeg, s);
    dev_free(tmp, s);
    dev_free(dmax, s);
    return st;
}

}  // namespace dsd
