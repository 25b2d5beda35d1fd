// Allocation-free triangle clique-degrees (h = 3) for callers that cannot
// allocate device memory.
//
// Some callers cannot call cudaMalloc: plug-ins that live inside a host
// framework whose allocator has already reserved the device memory (another
// allocation would fail or fragment the framework's pool), and latency-bound
// serving paths where an allocation's cost or possible failure in the middle
// of a request is not acceptable.  dsd_triangle_degrees_noalloc serves them:
// it reads the caller's CSR, writes the caller's output buffers, and keeps
// its own scratch (a work counter and a list of heavy rows) in one statically
// sized __device__ array of this translation unit.  It calls no allocator.
//
// The first call on a device looks up the array's device address (with that
// device current) and caches it; make that first call before any stream
// capture begins.
//
// Unlike dsd_clique_degrees it needs no graph handle and no degeneracy
// order: rows are oriented by vertex id (N+(u) = the entries of row u that
// exceed u), which lists every triangle exactly once, like any total order.
//
// The scratch array is shared by every call in the process on that device:
// calls whose work overlaps on the GPU (different streams, or different host
// threads) race on it.  Serialise them.
#include "common.cuh"

#include <mutex>

namespace dsd {
namespace {

// Scratch: [0] work counter, [1] heavy-row count, [2..] heavy-row list.
constexpr uint32_t kNoAllocWords = 1u << 20;           // 4 MiB
constexpr uint32_t kNoAllocMaxN = kNoAllocWords - 64;  // every row fits the list
static __device__ __align__(256) uint32_t g_noalloc_scratch[kNoAllocWords];

constexpr int kDevMax = 64;
uint32_t* g_scratch_ptr[kDevMax];
std::once_flag g_scratch_once[kDevMax];
cudaError_t g_scratch_err[kDevMax];

__device__ __forceinline__ uint64_t tail_start(const uint64_t* off, const uint32_t* adj,
                                               uint32_t u) {
    uint64_t b = off[u], e = off[u + 1];
    return b + lower_bound_u32(adj + b, e - b, u + 1u);
}

// Rows with at most 32 higher-id neighbours: one warp each (dynamic queue).
// Larger rows go to the heavy list for k_na_heavy.
__global__ void __launch_bounds__(256) k_na_light(uint32_t n, const uint64_t* off,
                                                  const uint32_t* adj,
                                                  unsigned long long* deg,
                                                  unsigned long long* mu, uint32_t* scratch) {
    __shared__ uint32_t sC[8][32];
    __shared__ unsigned sCnt[8][32];
    unsigned lane = lane_id(), w = warp_id();
    uint32_t* C = sC[w];
    unsigned* cnt = sCnt[w];
    unsigned long long acc = 0;
    for (;;) {
        uint32_t base = 0;
        if (lane == 0) base = atomicAdd(&scratch[0], 32u);
        base = __shfl_sync(0xffffffffu, base, 0);
        if (base >= n) break;
        uint32_t end = base + 32 < n ? base + 32 : n;
        for (uint32_t u = base; u < end; u++) {
            uint64_t b = tail_start(off, adj, u), e = off[u + 1];
            uint32_t d = (uint32_t)(e - b);
            if (d < 2) continue;
            if (d > 32) {
                if (lane == 0) scratch[2 + atomicAdd(&scratch[1], 1u)] = u;
                continue;
            }
            if (lane < d) { C[lane] = adj[b + lane]; cnt[lane] = 0; }
            __syncwarp();
            unsigned long long t = 0;
            for (uint32_t i = 0; i < d; i++) {
                uint32_t x = C[i];
                uint64_t xb = tail_start(off, adj, x), xe = off[x + 1];
                unsigned hits = 0;
                for (uint64_t p = xb + lane; p < xe; p += 32) {
                    uint32_t y = adj[p];
                    uint32_t pos = (uint32_t)lower_bound_u32(C, d, y);
                    if (pos < d && C[pos] == y) { atomicAdd(&cnt[pos], 1u); hits++; }
                }
                hits = __reduce_add_sync(0xffffffffu, hits);
                if (lane == 0 && hits) atomicAdd(&cnt[i], hits);
                t += hits;
            }
            __syncwarp();
            if (t) {
                if (lane < d && cnt[lane]) atomicAdd(&deg[C[lane]], (unsigned long long)cnt[lane]);
                if (lane == 0) { atomicAdd(&deg[u], t); acc += t; }
            }
            __syncwarp();
        }
    }
    if (lane == 0 && acc) atomicAdd(mu, acc);
}

// Heavy rows: one block each, candidates read in place from the CSR.
__global__ void __launch_bounds__(256) k_na_heavy(const uint64_t* off, const uint32_t* adj,
                                                  unsigned long long* deg,
                                                  unsigned long long* mu,
                                                  const uint32_t* scratch) {
    __shared__ unsigned long long s_tot;
    uint32_t nh = scratch[1];
    unsigned lane = lane_id(), nw = blockDim.x >> 5;
    for (uint32_t it = blockIdx.x; it < nh; it += gridDim.x) {
        uint32_t u = scratch[2 + it];
        uint64_t b = tail_start(off, adj, u), e = off[u + 1];
        uint32_t d = (uint32_t)(e - b);
        const uint32_t* C = adj + b;
        if (threadIdx.x == 0) s_tot = 0;
        __syncthreads();
        unsigned long long mine = 0;
        for (uint32_t i = warp_id(); i < d; i += nw) {
            uint32_t x = C[i];
            uint64_t xb = tail_start(off, adj, x), xe = off[x + 1];
            unsigned hits = 0;
            for (uint64_t p = xb + lane; p < xe; p += 32) {
                uint32_t y = adj[p];
                uint64_t pos = lower_bound_u32(C, d, y);
                if (pos < d && C[pos] == y) { atomicAdd(&deg[y], 1ull); hits++; }
            }
            hits = __reduce_add_sync(0xffffffffu, hits);
            if (lane == 0 && hits) { atomicAdd(&deg[x], (unsigned long long)hits); mine += hits; }
        }
        if (mine) atomicAdd(&s_tot, mine);
        __syncthreads();
        if (threadIdx.x == 0 && s_tot) {
            atomicAdd(&deg[u], s_tot);
            atomicAdd(mu, s_tot);
        }
        __syncthreads();
    }
}

// Device address of the scratch array for the current device, looked up
// once per device (with that device current).
dsd_status scratch_for_current_device(uint32_t** out) {
    int dev = 0;
    DSD_CU(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kDevMax) {
        set_error("device ordinal %d out of range", dev);
        return DSD_ERR_UNSUPPORTED;
    }
    std::call_once(g_scratch_once[dev], [dev]() {
        void* p = nullptr;
        g_scratch_err[dev] = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        g_scratch_ptr[dev] = static_cast<uint32_t*>(p);
    });
    if (g_scratch_err[dev] != cudaSuccess || !g_scratch_ptr[dev]) {
        set_error("cudaGetSymbolAddress for the scratch array failed: %s",
                  cudaGetErrorString(g_scratch_err[dev]));
        return DSD_ERR_CUDA;
    }
    *out = g_scratch_ptr[dev];
    return DSD_OK;
}

}  // namespace
}  // namespace dsd

using namespace dsd;

extern "C" dsd_status dsd_triangle_degrees_noalloc(uint32_t n, const uint64_t* off,
                                                   const uint32_t* adj, uint64_t* deg,
                                                   uint64_t* mu, void* cuda_stream) {
    set_error("");
    if (!off || !deg || !mu) {
        set_error("dsd_triangle_degrees_noalloc: off, deg and mu must be device pointers");
        return DSD_ERR_INVALID;
    }
    if (n > kNoAllocMaxN) {
        set_error("dsd_triangle_degrees_noalloc handles at most %u vertices (got %u): its "
                  "scratch is a fixed %u-word device array", kNoAllocMaxN, n, kNoAllocWords);
        return DSD_ERR_UNSUPPORTED;
    }
    cudaStream_t s = (cudaStream_t)cuda_stream;
    if (n && !adj) {
        // an edgeless CSR may come with a null adj (a zero-length device
        // buffer has no address); any other null adj is an error
        uint64_t edges = 0;
        DSD_CU(cudaMemcpyAsync(&edges, off + n, sizeof(edges), cudaMemcpyDeviceToHost, s));
        DSD_CU(cudaStreamSynchronize(s));
        if (edges) {
            set_error("dsd_triangle_degrees_noalloc: adj is NULL but off[n] = %llu",
                      (unsigned long long)edges);
            return DSD_ERR_INVALID;
        }
    }
    uint32_t* scratch = nullptr;
    DSD_TRY(scratch_for_current_device(&scratch));
    // the counters and the outputs start at zero on every call
    DSD_CU(cudaMemsetAsync(scratch, 0, 2 * sizeof(uint32_t), s));
    DSD_CU(cudaMemsetAsync(deg, 0, (size_t)n * sizeof(uint64_t), s));
    DSD_CU(cudaMemsetAsync(mu, 0, sizeof(uint64_t), s));
    if (n == 0) return DSD_OK;
    int sms = 152;
    DSD_TRY(num_sms(&sms));
    k_na_light<<<sms * 8, 256, 0, s>>>(n, off, adj, (unsigned long long*)deg,
                                       (unsigned long long*)mu, scratch);
    note_launch();
    k_na_heavy<<<sms * 4, 256, 0, s>>>(off, adj, (unsigned long long*)deg,
                                       (unsigned long long*)mu, scratch);
    note_launch();
    DSD_CU(cudaGetLastError());
    return DSD_OK;
}
