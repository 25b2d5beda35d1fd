// Edge list -> cleaned symmetric CSR (Sec. 2 data model: undirected,
// unweighted, simple).  Counting pass, exclusive scan, scatter by atomic
// cursors, per-row sort + unique, scan of the unique counts, row copy.
#include "graph.cuh"

namespace dsd {
namespace {

// The edge list is streamed once per pass.  When both arrays start on a
// 16-byte boundary, each thread reads four edges of each with one 128-bit
// load (the last m % 4 edges one by one); otherwise one edge at a time.
template <class F>
__device__ __forceinline__ void for_each_edge(const uint32_t* src, const uint32_t* dst,
                                              uint64_t m, F f) {
    const uint64_t t0 = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t nt = (uint64_t)gridDim.x * blockDim.x;
    const bool vec = ((reinterpret_cast<uintptr_t>(src) | reinterpret_cast<uintptr_t>(dst)) & 15) == 0;
    uint64_t done = 0;
    if (vec) {
        const uint64_t q = m >> 2;
        const uint4* s4 = reinterpret_cast<const uint4*>(src);
        const uint4* d4 = reinterpret_cast<const uint4*>(dst);
        for (uint64_t i = t0; i < q; i += nt) {
            const uint4 a = s4[i], b = d4[i];
            f(a.x, b.x);
            f(a.y, b.y);
            f(a.z, b.z);
            f(a.w, b.w);
        }
        done = q << 2;
    }
    for (uint64_t i = done + t0; i < m; i += nt) f(src[i], dst[i]);
}

__global__ void k_count_endpoints(const uint32_t* src, const uint32_t* dst, uint64_t m,
                                  uint32_t n, uint32_t* cnt, uint32_t* err) {
    for_each_edge(src, dst, m, [&](uint32_t u, uint32_t v) {
        if (u >= n || v >= n) {
            atomicOr(err, 1u);
            return;
        }
        if (u == v) return;
        atomicAdd(&cnt[u], 1u);
        atomicAdd(&cnt[v], 1u);
    });
}

__global__ void k_scatter(const uint32_t* src, const uint32_t* dst, uint64_t m, uint32_t n,
                          const uint64_t* pos, uint32_t* cursor, uint32_t* out) {
    for_each_edge(src, dst, m, [&](uint32_t u, uint32_t v) {
        if (u >= n || v >= n || u == v) return;
        out[pos[u] + atomicAdd(&cursor[u], 1u)] = v;
        out[pos[v] + atomicAdd(&cursor[v], 1u)] = u;
    });
}

// One warp per row: copy the unique prefix of each row to its final place.
__global__ void k_copy_rows(const uint32_t* tmp, const uint64_t* pos, const uint64_t* off,
                            uint32_t n, uint32_t* adj) {
    uint32_t gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    uint32_t nw = (gridDim.x * blockDim.x) >> 5;
    unsigned lane = lane_id();
    for (uint32_t r = gw; r < n; r += nw) {
        uint64_t s = pos[r], d = off[r], l = off[r + 1] - off[r];
        for (uint64_t j = lane; j < l; j += 32) adj[d + j] = tmp[s + j];
    }
}

}  // namespace

dsd_status build_csr(dsd_graph* g, uint64_t m, const uint32_t* src, const uint32_t* dst) {
    cudaStream_t s = g->stream;
    uint32_t n = g->n;
    int sms = 152;
    DSD_TRY(num_sms(&sms));
    if ((m >> 31) != 0) {
        set_error("edge lists of 2^31 or more entries are not supported by this library");
        return DSD_ERR_UNSUPPORTED;
    }
    uint32_t* cnt = nullptr;      // [n] endpoint counts, then cursors
    uint32_t* err = nullptr;
    uint64_t* pos = nullptr;      // [n+1]
    uint32_t* tmp = nullptr;      // [2m]
    uint32_t* tmp2 = nullptr;     // [2m]
    uint32_t* ulen = nullptr;     // [n]
    dsd_status st = DSD_OK;
    uint64_t total = 0;
    uint32_t herr = 0;
    unsigned grid = (unsigned)(sms * 8);
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
    STEP(dalloc(&cnt, (size_t)n + 1, s));
    STEP(dalloc(&err, 1, s));
    STEP(dalloc(&pos, (size_t)n + 1, s));
    STEP(dalloc(&ulen, (size_t)n + 1, s));
    STEP(dalloc(&g->off, (size_t)n + 1, s));
    CUSTEP(cudaMemsetAsync(cnt, 0, ((size_t)n + 1) * 4, s));
    CUSTEP(cudaMemsetAsync(err, 0, 4, s));
    if (m) {
        k_count_endpoints<<<grid, 256, 0, s>>>(src, dst, m, n, cnt, err); note_launch();
        CUSTEP(cudaGetLastError());
    }
    CUSTEP(cudaMemcpyAsync(&herr, err, 4, cudaMemcpyDeviceToHost, s));
    STEP(exclusive_scan_u32_to_u64(cnt, pos, n, s));
    CUSTEP(cudaMemcpyAsync(&total, pos + n, 8, cudaMemcpyDeviceToHost, s));
    CUSTEP(cudaStreamSynchronize(s));
    if (herr) {
        set_error("edge endpoint out of range (n = %u)", n);
        st = DSD_ERR_INVALID;
        goto done;
    }
    STEP(dalloc(&tmp, total + 1, s));
    STEP(dalloc(&tmp2, total + 1, s));
    CUSTEP(cudaMemsetAsync(cnt, 0, ((size_t)n + 1) * 4, s));
    if (m) {
        k_scatter<<<grid, 256, 0, s>>>(src, dst, m, n, pos, cnt, tmp); note_launch();
        CUSTEP(cudaGetLastError());
    }
    // cnt now equals the per-row lengths again
    STEP(segmented_sort_unique(tmp, tmp2, pos, cnt, ulen, n, total, s));
    STEP(exclusive_scan_u32_to_u64(ulen, g->off, n, s));
    {
        uint64_t tot2 = 0;
        CUSTEP(cudaMemcpyAsync(&tot2, g->off + n, 8, cudaMemcpyDeviceToHost, s));
        CUSTEP(cudaStreamSynchronize(s));
        g->m = tot2 / 2;
        STEP(dalloc(&g->adj, tot2 + 1, s));
        if (n) {
            k_copy_rows<<<grid, 256, 0, s>>>(tmp, pos, g->off, n, g->adj); note_launch();
            CUSTEP(cudaGetLastError());
        }
    }
done:
#undef STEP
#undef CUSTEP
    dev_free(cnt, s);
    dev_free(err, s);
    dev_free(pos, s);
    dev_free(tmp, s);
    dev_free(tmp2, s);
    dev_free(ulen, s);
    return st;
}

}  // namespace dsd
