// Building blocks: prefix sums and the segmented sort + unique used by the
// CSR builders (graph model of Sec. 2: sorted, duplicate-free rows).
#include "common.cuh"

#include <stdarg.h>
#include <string.h>

namespace dsd {

// ---------------------------------------------------------------- errors
static thread_local char g_last_error[1024];

void set_error(const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_last_error, sizeof(g_last_error), fmt, ap);
    va_end(ap);
}

const char* last_error() { return g_last_error; }

dsd_status cuda_fail(cudaError_t e, const char* what, const char* file, int line) {
    set_error("%s failed: %s (%s:%d)", what, cudaGetErrorString(e), file, line);
    (void)cudaGetLastError();   // a non-sticky error must not surface in a later check
    if (e == cudaErrorMemoryAllocation) return DSD_ERR_NOMEM;
    return DSD_ERR_CUDA;
}

dsd_status dev_alloc(void** p, size_t bytes, cudaStream_t s) {
    *p = nullptr;
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMallocAsync(p, bytes, s);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        set_error("device allocation of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
        *p = nullptr;
        return e == cudaErrorMemoryAllocation ? DSD_ERR_NOMEM : DSD_ERR_CUDA;
    }
    return DSD_OK;
}

void dev_free(void* p, cudaStream_t s) {
    if (p) cudaFreeAsync(p, s);
}

dsd_status num_sms(int* out) {
    int dev = 0;
    DSD_CU(cudaGetDevice(&dev));
    DSD_CU(cudaDeviceGetAttribute(out, cudaDevAttrMultiProcessorCount, dev));
    return DSD_OK;
}

// ----------------------------------------------------------------- scans
namespace {

constexpr int kScanThreads = 256;
constexpr int kScanPer = 8;
constexpr int kScanTile = kScanThreads * kScanPer;  // 2048

template <class T>
__device__ __forceinline__ uint64_t load_as_u64(const T* in, uint64_t i, uint64_t n) {
    return i < n ? (uint64_t)in[i] : 0ull;
}

// Block-wide exclusive scan of one value per thread; returns the prefix and
// writes the block total into *total.
__device__ uint64_t block_exclusive_scan(uint64_t v, uint64_t* total) {
    __shared__ uint64_t warp_tot[32];
    unsigned lane = lane_id(), wid = warp_id();
    uint64_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint64_t y = __shfl_up_sync(0xffffffffu, x, o);
        if ((int)lane >= o) x += y;
    }
    if (lane == 31) warp_tot[wid] = x;
    __syncthreads();
    unsigned nw = blockDim.x >> 5;
    if (wid == 0) {
        uint64_t t = lane < nw ? warp_tot[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint64_t y = __shfl_up_sync(0xffffffffu, t, o);
            if ((int)lane >= o) t += y;
        }
        if (lane < nw) warp_tot[lane] = t;  // inclusive
    }
    __syncthreads();
    uint64_t before = wid ? warp_tot[wid - 1] : 0;
    *total = warp_tot[nw - 1];
    __syncthreads();
    return before + x - v;
}

template <class T>
__global__ void k_tile_sums(const T* in, uint64_t n, uint64_t* sums) {
    uint64_t base = (uint64_t)blockIdx.x * kScanTile;
    uint64_t acc = 0;
    for (int i = 0; i < kScanPer; i++)
        acc += load_as_u64(in, base + (uint64_t)i * kScanThreads + threadIdx.x, n);
    acc = warp_sum(acc);
    __shared__ uint64_t ws[kScanThreads / 32];
    if (lane_id() == 0) ws[warp_id()] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint64_t t = 0;
        for (int w = 0; w < kScanThreads / 32; w++) t += ws[w];
        sums[blockIdx.x] = t;
    }
}

// Exclusive scan of sums[0..nt) in place by one block; sums[nt] = total.
__global__ void k_scan_sums(uint64_t* sums, uint64_t nt) {
    uint64_t carry = 0;
    for (uint64_t base = 0; base < nt; base += blockDim.x) {
        uint64_t i = base + threadIdx.x;
        uint64_t v = i < nt ? sums[i] : 0;
        uint64_t tot;
        uint64_t ex = block_exclusive_scan(v, &tot);
        if (i < nt) sums[i] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0) sums[nt] = carry;
}

template <class T>
__global__ void k_scan_apply(const T* in, uint64_t n, const uint64_t* sums, uint64_t* out) {
    uint64_t base = (uint64_t)blockIdx.x * kScanTile + (uint64_t)threadIdx.x * kScanPer;
    uint64_t vals[kScanPer];
    uint64_t local = 0;
#pragma unroll
    for (int i = 0; i < kScanPer; i++) {
        vals[i] = load_as_u64(in, base + i, n);
        local += vals[i];
    }
    uint64_t tot;
    uint64_t ex = block_exclusive_scan(local, &tot) + sums[blockIdx.x];
#pragma unroll
    for (int i = 0; i < kScanPer; i++) {
        if (base + i < n) out[base + i] = ex;
        ex += vals[i];
    }
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) out[n] = sums[gridDim.x];
}

template <class T>
dsd_status exclusive_scan_impl(const T* in, uint64_t* out, uint64_t n, cudaStream_t s) {
    uint64_t nt = (n + kScanTile - 1) / kScanTile;
    if (nt == 0) {
        DSD_CU(cudaMemsetAsync(out, 0, sizeof(uint64_t), s));
        return DSD_OK;
    }
    uint64_t* sums = nullptr;
    DSD_TRY(dalloc(&sums, nt + 1, s));
    k_tile_sums<T><<<(unsigned)nt, kScanThreads, 0, s>>>(in, n, sums); note_launch();
    k_scan_sums<<<1, 1024, 0, s>>>(sums, nt); note_launch();
    k_scan_apply<T><<<(unsigned)nt, kScanThreads, 0, s>>>(in, n, sums, out); note_launch();
    cudaError_t e = cudaGetLastError();
    dev_free(sums, s);
    if (e != cudaSuccess) return cuda_fail(e, "scan launch", __FILE__, __LINE__);
    return DSD_OK;
}

}  // namespace

dsd_status exclusive_scan_u64(const uint64_t* in, uint64_t* out, uint64_t n, cudaStream_t s) {
    return exclusive_scan_impl<uint64_t>(in, out, n, s);
}
dsd_status exclusive_scan_u32_to_u64(const uint32_t* in, uint64_t* out, uint64_t n,
                                     cudaStream_t s) {
    return exclusive_scan_impl<uint32_t>(in, out, n, s);
}

// ------------------------------------------------ segmented sort + unique
namespace {

constexpr uint32_t kSmallMax = 32;      // warp, registers
constexpr uint32_t kWarpMax = 256;      // warp, its own 1 KB of shared memory
constexpr uint32_t kMedMax = 2048;      // 256 threads, shared memory
constexpr uint32_t kLargeMax = 16384;   // 1024 threads, 64 KB shared memory
constexpr int kClasses = 5;

struct SortLists {
    uint32_t* rows[kClasses];
    uint32_t* count;   // kClasses counters
};

// One atomic per class and warp (a warp's rows of one class are appended
// together; order inside a class does not matter).
__global__ void k_classify(const uint32_t* len, uint32_t rows, SortLists L) {
    const unsigned lane = lane_id();
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t r0 = blockIdx.x * blockDim.x; r0 < rows; r0 += stride) {
        const uint32_t r = r0 + threadIdx.x;
        int c = -1;
        if (r < rows) {
            const uint32_t l = len[r];
            c = l <= kSmallMax ? 0 : l <= kWarpMax ? 4 : l <= kMedMax ? 1 : l <= kLargeMax ? 2 : 3;
        }
#pragma unroll
        for (int q = 0; q < kClasses; q++) {
            const unsigned b = __ballot_sync(0xffffffffu, c == q);
            if (!b) continue;
            uint32_t base = 0;
            if (lane == (unsigned)(__ffs(b) - 1)) base = atomicAdd(&L.count[q], (uint32_t)__popc(b));
            base = __shfl_sync(0xffffffffu, base, __ffs(b) - 1);
            if (c == q) L.rows[q][base + __popc(b & ((1u << lane) - 1u))] = r;
        }
    }
}

// Rows of at most 32 entries: one warp each, bitonic network in registers.
__global__ void k_sort_small(uint32_t* vals, const uint64_t* pos, const uint32_t* len,
                             uint32_t* newlen, const uint32_t* list, const uint32_t* count) {
    unsigned lane = lane_id();
    uint32_t nrows = *count;
    uint32_t gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    uint32_t nw = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t i = gw; i < nrows; i += nw) {
        uint32_t r = list[i];
        uint32_t l = len[r];
        uint32_t* row = vals + pos[r];
        uint32_t x = lane < l ? row[lane] : 0xffffffffu;
#pragma unroll
        for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
            for (int j = k >> 1; j > 0; j >>= 1) {
                uint32_t y = __shfl_xor_sync(0xffffffffu, x, j);
                bool asc = (lane & k) == 0;
                bool lower = (lane & j) == 0;
                x = (lower == asc) ? min(x, y) : max(x, y);
            }
        }
        uint32_t prev = __shfl_up_sync(0xffffffffu, x, 1);
        bool keep = lane < l && (lane == 0 || x != prev);
        unsigned b = __ballot_sync(0xffffffffu, keep);
        if (keep) row[__popc(b & ((1u << lane) - 1u))] = x;
        if (lane == 0) newlen[r] = __popc(b);
    }
}

// Rows of 33..256 entries: one warp each, a bitonic network in the warp's
// own shared-memory slice (warp synchronisation only), then the unique
// entries written back in order.
__global__ void __launch_bounds__(256) k_sort_warp(uint32_t* vals, const uint64_t* pos,
                                                   const uint32_t* len, uint32_t* newlen,
                                                   const uint32_t* list, const uint32_t* count) {
    __shared__ uint32_t sm[8][kWarpMax];
    const unsigned lane = lane_id();
    uint32_t* sw = sm[threadIdx.x >> 5];
    const uint32_t nrows = *count;
    const uint32_t gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nw = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t i = gw; i < nrows; i += nw) {
        const uint32_t r = list[i];
        const uint32_t l = len[r];
        uint32_t* row = vals + pos[r];
        uint32_t N = 64;
        while (N < l) N <<= 1;
        for (uint32_t j = lane; j < N; j += 32) sw[j] = j < l ? row[j] : 0xffffffffu;
        __syncwarp();
        for (uint32_t k = 2; k <= N; k <<= 1) {
            for (uint32_t j = k >> 1; j > 0; j >>= 1) {
                for (uint32_t x = lane; x < N; x += 32) {
                    const uint32_t y = x ^ j;
                    if (y > x) {
                        const bool asc = (x & k) == 0;
                        const uint32_t a = sw[x], b = sw[y];
                        if ((a > b) == asc) {
                            sw[x] = b;
                            sw[y] = a;
                        }
                    }
                }
                __syncwarp();
            }
        }
        uint32_t base = 0;
        for (uint32_t b0 = 0; b0 < l; b0 += 32) {
            const uint32_t x = b0 + lane;
            uint32_t v = 0;
            bool keep = false;
            if (x < l) {
                v = sw[x];
                keep = x == 0 || v != sw[x - 1];
            }
            const unsigned bal = __ballot_sync(0xffffffffu, keep);
            if (keep) row[base + __popc(bal & ((1u << lane) - 1u))] = v;
            base += __popc(bal);
        }
        if (lane == 0) newlen[r] = base;
        __syncwarp();
    }
}

__device__ void smem_bitonic(uint32_t* s, uint32_t N) {
    for (uint32_t k = 2; k <= N; k <<= 1) {
        for (uint32_t j = k >> 1; j > 0; j >>= 1) {
            for (uint32_t i = threadIdx.x; i < N; i += blockDim.x) {
                uint32_t ixj = i ^ j;
                if (ixj > i) {
                    bool asc = (i & k) == 0;
                    uint32_t a = s[i], b = s[ixj];
                    if ((a > b) == asc) { s[i] = b; s[ixj] = a; }
                }
            }
            __syncthreads();
        }
    }
}

// Block-level unique of sorted src[0..l) (smem or global) into dst (global),
// dst may alias src only if src is shared memory.  Returns the count in
// every thread.
template <class P>
__device__ uint32_t block_unique_write(P src, uint32_t l, uint32_t* dst) {
    __shared__ uint32_t s_base;
    if (threadIdx.x == 0) s_base = 0;
    __syncthreads();
    for (uint32_t b0 = 0; b0 < l; b0 += blockDim.x) {
        uint32_t i = b0 + threadIdx.x;
        uint32_t x = 0;
        bool keep = false;
        if (i < l) {
            x = src[i];
            keep = (i == 0) || (x != src[i - 1]);
        }
        uint64_t tot;
        uint64_t ex = block_exclusive_scan(keep ? 1 : 0, &tot);
        uint32_t base = s_base;
        __syncthreads();
        if (keep) dst[base + (uint32_t)ex] = x;
        __syncthreads();
        if (threadIdx.x == 0) s_base = base + (uint32_t)tot;
        __syncthreads();
    }
    return s_base;
}

// Rows of 33..16384 entries: one block each, bitonic sort in shared memory.
template <uint32_t MAXN>
__global__ void k_sort_block(uint32_t* vals, const uint64_t* pos, const uint32_t* len,
                             uint32_t* newlen, const uint32_t* list, const uint32_t* count) {
    extern __shared__ uint32_t s[];
    uint32_t nrows = *count;
    for (uint32_t i = blockIdx.x; i < nrows; i += gridDim.x) {
        uint32_t r = list[i];
        uint32_t l = len[r];
        uint32_t* row = vals + pos[r];
        uint32_t N = 64;
        while (N < l) N <<= 1;
        for (uint32_t j = threadIdx.x; j < N; j += blockDim.x) s[j] = j < l ? row[j] : 0xffffffffu;
        __syncthreads();
        smem_bitonic(s, N);
        uint32_t u = block_unique_write(s, l, row);
        if (threadIdx.x == 0) newlen[r] = u;
        __syncthreads();
    }
}

// Merge sorted a[0..na) and b[0..nb) into out, one block.
__device__ void block_merge(const uint32_t* a, uint64_t na, const uint32_t* b, uint64_t nb,
                            uint32_t* out) {
    uint64_t total = na + nb;
    uint64_t per = (total + blockDim.x - 1) / blockDim.x;
    uint64_t d0 = (uint64_t)threadIdx.x * per;
    if (d0 >= total) return;
    uint64_t d1 = d0 + per < total ? d0 + per : total;
    uint64_t lo = d0 > nb ? d0 - nb : 0, hi = d0 < na ? d0 : na;
    while (lo < hi) {
        uint64_t mid = (lo + hi) >> 1;
        if (a[mid] <= b[d0 - 1 - mid]) lo = mid + 1; else hi = mid;
    }
    uint64_t ia = lo, ib = d0 - lo;
    for (uint64_t d = d0; d < d1; d++) {
        if (ib >= nb || (ia < na && a[ia] <= b[ib])) out[d] = a[ia++];
        else out[d] = b[ib++];
    }
}

// Rows above 16384 entries: sort 16384-chunks in shared memory, then merge
// runs pairwise through `tmp`, then unique into the row.
__global__ void k_sort_huge(uint32_t* vals, uint32_t* tmp, const uint64_t* pos,
                            const uint32_t* len, uint32_t* newlen, const uint32_t* list,
                            const uint32_t* count) {
    extern __shared__ uint32_t s[];
    uint32_t nrows = *count;
    for (uint32_t i = blockIdx.x; i < nrows; i += gridDim.x) {
        uint32_t r = list[i];
        uint64_t l = len[r];
        uint32_t* row = vals + pos[r];
        uint32_t* alt = tmp + pos[r];
        for (uint64_t c0 = 0; c0 < l; c0 += kLargeMax) {
            uint64_t cl = l - c0 < kLargeMax ? l - c0 : kLargeMax;
            for (uint32_t j = threadIdx.x; j < kLargeMax; j += blockDim.x)
                s[j] = j < cl ? row[c0 + j] : 0xffffffffu;
            __syncthreads();
            smem_bitonic(s, kLargeMax);
            for (uint32_t j = threadIdx.x; j < cl; j += blockDim.x) row[c0 + j] = s[j];
            __syncthreads();
        }
        uint32_t* src = row;
        uint32_t* dst = alt;
        for (uint64_t w = kLargeMax; w < l; w <<= 1) {
            for (uint64_t a0 = 0; a0 < l; a0 += 2 * w) {
                uint64_t na = l - a0 < w ? l - a0 : w;
                uint64_t b0 = a0 + na;
                uint64_t nb = b0 < l ? (l - b0 < w ? l - b0 : w) : 0;
                block_merge(src + a0, na, src + b0, nb, dst + a0);
            }
            __syncthreads();
            uint32_t* t = src; src = dst; dst = t;
        }
        uint32_t u;
        if (src == row) {
            // unique in place needs a separate destination: copy via alt
            for (uint64_t j = threadIdx.x; j < l; j += blockDim.x) alt[j] = row[j];
            __syncthreads();
            u = block_unique_write(alt, (uint32_t)l, row);
        } else {
            u = block_unique_write(src, (uint32_t)l, row);
        }
        if (threadIdx.x == 0) newlen[r] = u;
        __syncthreads();
    }
}

}  // namespace

dsd_status segmented_sort_unique(uint32_t* vals, uint32_t* tmp, const uint64_t* pos,
                                 const uint32_t* len, uint32_t* newlen, uint32_t rows,
                                 uint64_t total, cudaStream_t s) {
    (void)total;
    if (rows == 0) return DSD_OK;
    SortLists L;
    uint32_t* lists = nullptr;
    uint32_t* cnt = nullptr;
    DSD_TRY(dalloc(&lists, (size_t)rows * kClasses, s));
    dsd_status st = dalloc(&cnt, kClasses, s);
    if (st != DSD_OK) { dev_free(lists, s); return st; }
    for (int c = 0; c < kClasses; c++) L.rows[c] = lists + (size_t)c * rows;
    L.count = cnt;
    int sms = 152;
    num_sms(&sms);
    cudaError_t e = cudaMemsetAsync(cnt, 0, kClasses * sizeof(uint32_t), s);
    if (e == cudaSuccess) {
        unsigned g = (unsigned)((rows + 255) / 256);
        k_classify<<<g < 65535u ? g : 65535u, 256, 0, s>>>(len, rows, L); note_launch();
        k_sort_small<<<sms * 8, 256, 0, s>>>(vals, pos, len, newlen, L.rows[0], cnt + 0); note_launch();
        k_sort_warp<<<sms * 8, 256, 0, s>>>(vals, pos, len, newlen, L.rows[4], cnt + 4); note_launch();
        k_sort_block<kMedMax><<<sms * 4, 256, kMedMax * 4, s>>>(vals, pos, len, newlen,
                                                                  L.rows[1], cnt + 1); note_launch();
        static bool attr_done = false;
        if (!attr_done) {
            cudaFuncSetAttribute(k_sort_block<kLargeMax>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, kLargeMax * 4);
            cudaFuncSetAttribute(k_sort_huge, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 kLargeMax * 4);
            attr_done = true;
        }
        k_sort_block<kLargeMax><<<sms * 2, 1024, kLargeMax * 4, s>>>(vals, pos, len, newlen,
                                                                      L.rows[2], cnt + 2); note_launch();
        k_sort_huge<<<sms, 1024, kLargeMax * 4, s>>>(vals, tmp, pos, len, newlen, L.rows[3],
                                                     cnt + 3); note_launch();
        e = cudaGetLastError();
    }
    dev_free(lists, s);
    dev_free(cnt, s);
    if (e != cudaSuccess) return cuda_fail(e, "segmented sort", __FILE__, __LINE__);
    return DSD_OK;
}

}  // namespace dsd
