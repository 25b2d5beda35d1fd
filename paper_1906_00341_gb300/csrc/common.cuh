// Internal helpers shared by the libdsd translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>

#include "dsd.h"

namespace dsd {

// ------------------------------------------------------------ host errors
void set_error(const char* fmt, ...);
dsd_status cuda_fail(cudaError_t e, const char* what, const char* file, int line);

#define DSD_CU(expr)                                                              \
    do {                                                                          \
        cudaError_t e__ = (expr);                                                 \
        if (e__ != cudaSuccess) return ::dsd::cuda_fail(e__, #expr, __FILE__, __LINE__); \
    } while (0)

#define DSD_TRY(expr)                                                             \
    do {                                                                          \
        dsd_status s__ = (expr);                                                  \
        if (s__ != DSD_OK) return s__;                                            \
    } while (0)

// Launch-error check after <<<>>> (does not synchronise).
#define DSD_LAUNCHED() DSD_CU(cudaGetLastError())

// ------------------------------------------------------- device memory
// Stream-ordered allocations from the device's default memory pool.
struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
};
dsd_status dev_alloc(void** p, size_t bytes, cudaStream_t s);
void dev_free(void* p, cudaStream_t s);

template <class T>
inline dsd_status dalloc(T** p, size_t count, cudaStream_t s) {
    return dev_alloc(reinterpret_cast<void**>(p), count * sizeof(T) + 16, s);
}

// ------------------------------------------------------------- constants
constexpr int kWarp = 32;
constexpr uint32_t kNone = 0xffffffffu;

// Process-wide wait limit for grid barriers (nanoseconds).
uint64_t wait_limit_ns();

// Process-wide count of kernel launches issued by the library.
void note_launch();

// Largest alive set the peel replicates in every block's shared memory.
uint32_t peel_small_limit();
// Largest alive set handed to the cluster tail kernel (0 = never).
uint32_t peel_tail_limit();
uint32_t peel_app_queue_shared();   // PeelApp bucket queues: shared-memory words per block
uint64_t peel_app_queue_global();   // and global-memory words in all
uint32_t peel_item_warp_limit();    // h >= 4 peel: candidate sets a warp lists itself
uint32_t peel_item_mid_limit();     // and mid items a round may queue for warp groups

// --------------------------------------------------------- device utils
__device__ __forceinline__ uint64_t globaltimer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }
__device__ __forceinline__ unsigned warp_id() { return threadIdx.x >> 5; }

template <class T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ uint64_t warp_min_u64(uint64_t v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        uint64_t w = __shfl_xor_sync(0xffffffffu, v, o);
        v = w < v ? w : v;
    }
    return v;
}

// Lower bound of x in sorted a[0..len): first index with a[i] >= x.
template <class P>
__device__ __forceinline__ uint64_t lower_bound_u32(P a, uint64_t len, uint32_t x) {
    uint64_t lo = 0, hi = len;
    while (lo < hi) {
        uint64_t mid = (lo + hi) >> 1;
        if (a[mid] < x) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// Checked mode (dsd_set_checked): an addition into a 64-bit counter that
// wraps around sets *ovf instead of passing silently (ovf null: unchecked).
bool checked_mode();
__device__ __forceinline__ void add_counter(unsigned long long* p, unsigned long long v,
                                            uint32_t* ovf) {
    if (ovf) {
        unsigned long long old = atomicAdd(p, v);
        if (old + v < old) atomicOr(ovf, 1u);
    } else {
        atomicAdd(p, v);
    }
}

// u64 atomic subtract returning the old value.
__device__ __forceinline__ unsigned long long atomic_sub_u64(unsigned long long* p,
                                                            unsigned long long v) {
    return atomicAdd(p, (unsigned long long)(0ull - v));
}

// -------------------------------------------------- scans (host drivers)
// out[i] = sum_{j<i} in[j] for i in [0, n]; out has n+1 entries.
// Temporary storage is allocated on the stream.
dsd_status exclusive_scan_u64(const uint64_t* in, uint64_t* out, uint64_t n, cudaStream_t s);
dsd_status exclusive_scan_u32_to_u64(const uint32_t* in, uint64_t* out, uint64_t n,
                                     cudaStream_t s);

// Sort every row vals[pos[r] .. pos[r]+len[r]) ascending and drop repeats in
// place; newlen[r] receives the unique count.  rows: number of rows.
// `tmp` must have as many entries as vals.
dsd_status segmented_sort_unique(uint32_t* vals, uint32_t* tmp, const uint64_t* pos,
                                 const uint32_t* len, uint32_t* newlen, uint32_t rows,
                                 uint64_t total, cudaStream_t s);

// Device-side counters of a fill (used by builders and sizes).
dsd_status num_sms(int* out);

}  // namespace dsd
