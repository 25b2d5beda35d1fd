// The C ABI (include/dsd.h): argument checks, host/device marshalling,
// output extraction kernels, profiling.
#include "graph.cuh"

#include <atomic>
#include <new>
#include <string.h>

namespace dsd {
const char* last_error();

static uint64_t g_wait_ns = 20000ull * 1000000ull;
uint64_t wait_limit_ns() { return g_wait_ns; }

static std::atomic<uint32_t> g_small_limit{16384};
uint32_t peel_small_limit() { return g_small_limit.load(); }

static std::atomic<uint32_t> g_tail_limit{1u << 30};
uint32_t peel_tail_limit() { return g_tail_limit.load(); }

static std::atomic<uint32_t> g_app_qshared{12288};
static std::atomic<unsigned long long> g_app_qglobal{64ull << 20};
uint32_t peel_app_queue_shared() { return g_app_qshared.load(); }
uint64_t peel_app_queue_global() { return g_app_qglobal.load(); }

static std::atomic<uint32_t> g_item_warp{4};
static std::atomic<uint32_t> g_item_mid{1u << 20};
uint32_t peel_item_warp_limit() { return g_item_warp.load(); }
uint32_t peel_item_mid_limit() { return g_item_mid.load(); }

static std::atomic<int> g_checked{0};
bool checked_mode() { return g_checked.load() != 0; }

static std::atomic<unsigned long long> g_launches{0};
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

void record_peel(dsd_graph* g, int which, const PeelResult& r) {
    uint64_t* o = g->peel_stats[which];
    o[0] = r.rounds;
    o[1] = r.nlevels;
    o[2] = r.items;
    o[3] = r.bytes;
    o[4] = r.barrier_ns;
    o[5] = r.barriers;
    o[6] = r.compactions;
    o[7] = r.threads;
    o[8] = r.grid;
    o[9] = r.kmax;
    o[10] = r.small_round;
    for (int i = 0; i < 8; i++) o[11 + i] = r.tph[i];
    o[19] = r.tail_n;
    o[20] = r.tail_round;
    o[21] = r.tail_ns;
    for (int i = 0; i < 7; i++) o[22 + i] = r.tail_tph[i];
}

void prof_begin(dsd_graph* g, int phase) {
    if (!g->profiling) return;
    cudaEventRecord(g->ev[2 * phase], g->stream);
}
void prof_end(dsd_graph* g, int phase) {
    if (!g->profiling) return;
    cudaEventRecord(g->ev[2 * phase + 1], g->stream);
    g->prof_ms[phase] = -1.f;   // resolved lazily in dsd_phase_stats
}

namespace {

struct DevResult {
    unsigned long long kmax;
    unsigned long long kmax_core_mu;
    unsigned long long best_k;
    unsigned long long densest_mu;
    uint32_t kmax_core_size;
    uint32_t densest_size;
    uint32_t nlevels;
    uint32_t best_index;
};

__global__ void k_map_u64(uint32_t n, const uint32_t* old_of, const uint64_t* src, uint64_t* dst) {
    for (uint64_t p = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n;
         p += (uint64_t)gridDim.x * blockDim.x)
        dst[old_of[p]] = src[p];
}

__global__ void k_u64_to_u32(uint32_t n, const uint64_t* src, uint32_t* dst) {
    for (uint64_t p = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n;
         p += (uint64_t)gridDim.x * blockDim.x)
        dst[p] = (uint32_t)src[p];
}

__global__ void k_flags_ge(uint32_t n, const uint64_t* core, const unsigned long long* thr,
                           uint32_t* flags) {
    unsigned long long t = *thr;
    for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (uint64_t)gridDim.x * blockDim.x)
        flags[v] = core[v] >= t ? 1u : 0u;
}

__global__ void k_compact(uint32_t n, const uint32_t* flags, const uint64_t* pos, uint32_t* out) {
    for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (uint64_t)gridDim.x * blockDim.x)
        if (flags[v]) out[pos[v]] = (uint32_t)v;
}

// a/b >= c/d for a,c u64 and b,d u32 (b, d > 0): compare a*d with c*b in
// 128-bit arithmetic.
__device__ __forceinline__ bool ratio_ge(unsigned long long a, unsigned long long b,
                                         unsigned long long c, unsigned long long d) {
    unsigned long long lhi = __umul64hi(a, d), llo = a * d;
    unsigned long long rhi = __umul64hi(c, b), rlo = c * b;
    return lhi > rhi || (lhi == rhi && llo >= rlo);
}

// Densest level (ties to the larger k = later index) and the k_max level.
__global__ void k_best_level(uint32_t nl, const uint64_t* lk, const uint32_t* ls,
                             const uint64_t* lm, DevResult* out) {
    __shared__ uint32_t s_best[1024];
    uint32_t best = 0xffffffffu;
    for (uint32_t j = threadIdx.x; j < nl; j += blockDim.x) {
        if (best == 0xffffffffu || ratio_ge(lm[j], ls[j], lm[best], ls[best])) best = j;
    }
    s_best[threadIdx.x] = best;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t b = 0xffffffffu;
        for (uint32_t t = 0; t < blockDim.x; t++) {
            uint32_t j = s_best[t];
            if (j == 0xffffffffu) continue;
            if (b == 0xffffffffu) { b = j; continue; }
            // higher density wins; equal density -> larger index
            bool ge = ratio_ge(lm[j], ls[j], lm[b], ls[b]);
            bool le = ratio_ge(lm[b], ls[b], lm[j], ls[j]);
            if ((ge && !le) || (ge && le && j > b)) b = j;
        }
        DevResult r;
        memset(&r, 0, sizeof(r));
        r.nlevels = nl;
        if (nl) {
            r.kmax = lk[nl - 1];
            r.kmax_core_size = ls[nl - 1];
            r.kmax_core_mu = lm[nl - 1];
            r.best_k = lk[b];
            r.densest_size = ls[b];
            r.densest_mu = lm[b];
            r.best_index = b;
        }
        *out = r;
    }
}

bool valid_mem(int mem) { return mem == DSD_MEM_HOST || mem == DSD_MEM_DEVICE; }

dsd_status check_graph(const dsd_graph* g) {
    if (!g) {
        set_error("graph handle is NULL");
        return DSD_ERR_INVALID;
    }
    return DSD_OK;
}

dsd_status check_h(int h) {
    if (h < 2 || h > DSD_MAX_H) {
        set_error("h = %d outside [2, %d]", h, DSD_MAX_H);
        return DSD_ERR_INVALID;
    }
    return DSD_OK;
}

unsigned grid_for(uint64_t n) {
    uint64_t b = (n + 255) / 256;
    if (b < 1) b = 1;
    if (b > 152 * 16) b = 152 * 16;
    return (unsigned)b;
}

// Copy `bytes` from device src to the caller's buffer per `mem`.
dsd_status copy_out(void* dst, const void* src, size_t bytes, int mem, cudaStream_t s) {
    if (!dst || bytes == 0) return DSD_OK;
    DSD_CU(cudaMemcpyAsync(dst, src, bytes,
                           mem == DSD_MEM_DEVICE ? cudaMemcpyDeviceToDevice
                                                 : cudaMemcpyDeviceToHost, s));
    return DSD_OK;
}

dsd_status finish(int mem, cudaStream_t s) {
    if (mem == DSD_MEM_HOST) DSD_CU(cudaStreamSynchronize(s));
    return DSD_OK;
}

// Run (or reuse) the decomposition for h; leaves g->core / levels set.
dsd_status decompose(dsd_graph* g, int h) {
    DSD_TRY(ensure_order(g));
    if (h == 2) return DSD_OK;
    if (g->last_h == h) return DSD_OK;
    cudaStream_t s = g->stream;
    uint32_t n = g->n;
    g->last_h = 0;
    if (!g->core) DSD_TRY(dalloc(&g->core, (size_t)n + 1, s));
    if (!g->lvl_k) {
        DSD_TRY(dalloc(&g->lvl_k, (size_t)n + 1, s));
        DSD_TRY(dalloc(&g->lvl_size, (size_t)n + 1, s));
        DSD_TRY(dalloc(&g->lvl_mu, (size_t)n + 1, s));
    }
    unsigned long long* deg = nullptr;
    uint64_t* core_new = nullptr;
    DSD_TRY(dalloc(&deg, (size_t)n + 2, s));
    dsd_status st = dalloc(&core_new, (size_t)n + 1, s);
    if (st != DSD_OK) { dev_free(deg, s); return st; }
    unsigned long long mu = 0;
    PeelResult pr;
    prof_begin(g, kPhaseCount);
    st = count_cliques(g, h, deg, deg + n + 1);
    prof_end(g, kPhaseCount);
    if (st == DSD_OK) {
        cudaError_t e = cudaMemcpyAsync(&mu, deg + n + 1, 8, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) st = cuda_fail(e, "mu readback", __FILE__, __LINE__);
    }
    if (st == DSD_OK) {
        prof_begin(g, kPhasePeel);
        st = run_peel(g, h, n, g->roff, g->radj, g->rsplit, g->maxdplus, deg, mu, core_new,
                      nullptr, g->lvl_k, g->lvl_size, g->lvl_mu, &pr);
        prof_end(g, kPhasePeel);
        g->prof_launches[kPhasePeel] = 2;
    }
    if (st == DSD_OK && n) {
        k_map_u64<<<grid_for(n), 256, 0, s>>>(n, g->old_of, core_new, g->core); note_launch();
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) st = cuda_fail(e, "map", __FILE__, __LINE__);
    }
    dev_free(deg, s);
    dev_free(core_new, s);
    if (st != DSD_OK) return st;
    g->last_h = h;
    g->prof_bytes[kPhasePeel] = pr.bytes;
    record_peel(g, 1, pr);
    g->last_kmax = pr.kmax;
    g->last_mu = mu;
    g->nlevels = pr.nlevels;
    return DSD_OK;
}

void level_arrays(dsd_graph* g, int h, const uint64_t** lk, const uint32_t** ls,
                  const uint64_t** lm, uint32_t* nl, const uint64_t** core) {
    if (h == 2) {
        *lk = g->lvl2_k; *ls = g->lvl2_size; *lm = g->lvl2_mu; *nl = g->nlevels2;
        *core = g->core2;
    } else {
        *lk = g->lvl_k; *ls = g->lvl_size; *lm = g->lvl_mu; *nl = g->nlevels;
        *core = g->core;
    }
}

// Vertices v (ascending) with core[v] >= *thr_dev into out (device).
dsd_status extract_set(dsd_graph* g, const uint64_t* core, const unsigned long long* thr_dev,
                       uint32_t* out_dev) {
    cudaStream_t s = g->stream;
    uint32_t n = g->n;
    uint32_t* flags = nullptr;
    uint64_t* pos = nullptr;
    DSD_TRY(dalloc(&flags, (size_t)n + 1, s));
    dsd_status st = dalloc(&pos, (size_t)n + 1, s);
    if (st == DSD_OK) {
        k_flags_ge<<<grid_for(n), 256, 0, s>>>(n, core, thr_dev, flags); note_launch();
        st = exclusive_scan_u32_to_u64(flags, pos, n, s);
        if (st == DSD_OK) {
            k_compact<<<grid_for(n), 256, 0, s>>>(n, flags, pos, out_dev); note_launch();
            cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) st = cuda_fail(e, "compact", __FILE__, __LINE__);
        }
    }
    dev_free(flags, s);
    dev_free(pos, s);
    return st;
}

dsd_status make_graph(void* stream, uint32_t n, dsd_graph** out, dsd_graph** g) {
    *g = new (std::nothrow) dsd_graph();
    if (!*g) {
        set_error("host allocation failed");
        return DSD_ERR_NOMEM;
    }
    (*g)->stream = (cudaStream_t)stream;
    (*g)->n = n;
    cudaError_t e = cudaGetDevice(&(*g)->device);
    if (e != cudaSuccess) {
        delete *g;
        *g = nullptr;
        return cuda_fail(e, "cudaGetDevice", __FILE__, __LINE__);
    }
    for (int i = 0; i < 2 * DSD_NPHASES; i++) {
        e = cudaEventCreate(&(*g)->ev[i]);
        if (e != cudaSuccess) {
            for (int j = 0; j < i; j++) cudaEventDestroy((*g)->ev[j]);
            delete *g;
            *g = nullptr;
            return cuda_fail(e, "cudaEventCreate", __FILE__, __LINE__);
        }
    }
    (void)out;
    return DSD_OK;
}

// Offsets must be non-decreasing and end at `total`; checked before any
// row is expanded so that a malformed array never drives a write.
__global__ void k_check_offsets(uint32_t n, const uint64_t* off, uint64_t total, uint32_t* err) {
    for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (uint64_t)gridDim.x * blockDim.x)
        if (off[v + 1] < off[v] || off[v + 1] > total) atomicOr(err, 1u);
}

__global__ void k_expand_rows(uint32_t n, const uint64_t* off, uint32_t* src) {
    uint64_t gw = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    unsigned lane = lane_id();
    for (uint64_t v = gw; v < n; v += nw) {
        uint64_t b = off[v], e = off[v + 1];
        for (uint64_t j = b + lane; j < e; j += 32) src[j] = (uint32_t)v;
    }
}

}  // namespace

// Core numbers of the cached decomposition for h (caller ids), or null.
const uint64_t* cached_core(const dsd_graph* g, int h) {
    if (h == 2) return g->ordered ? g->core2 : nullptr;
    return g->last_h == h ? g->core : nullptr;
}

}  // namespace dsd

using namespace dsd;

extern "C" {

const char* dsd_status_string(dsd_status s) {
    switch (s) {
        case DSD_OK: return "ok";
        case DSD_ERR_INVALID: return "invalid argument";
        case DSD_ERR_NOMEM: return "out of memory";
        case DSD_ERR_CUDA: return "CUDA error";
        case DSD_ERR_TIMEOUT: return "bounded wait timed out";
        case DSD_ERR_OVERFLOW: return "overflow";
        case DSD_ERR_UNSUPPORTED: return "unsupported input";
        case DSD_ERR_INTERNAL: return "internal error";
    }
    return "unknown status";
}

const char* dsd_last_error(void) { return dsd::last_error(); }
uint64_t dsd_kernel_launches(void) { return g_launches.load(); }
const char* dsd_version(void) { return "libdsd 0.1 (sm_103a)"; }

dsd_status dsd_set_wait_limit_ms(uint32_t ms) {
    if (ms == 0) {
        set_error("wait limit must be positive");
        return DSD_ERR_INVALID;
    }
    g_wait_ns = (uint64_t)ms * 1000000ull;
    return DSD_OK;
}

dsd_status dsd_set_peel_small_limit(uint32_t max_alive) {
    g_small_limit = max_alive;
    return DSD_OK;
}

dsd_status dsd_set_peel_tail_limit(uint32_t max_alive) {
    g_tail_limit = max_alive;
    return DSD_OK;
}

dsd_status dsd_set_peel_app_queue(uint32_t shared_words, uint64_t global_words) {
    g_app_qshared = shared_words < 12288 ? shared_words : 12288;
    g_app_qglobal = global_words;
    return DSD_OK;
}

dsd_status dsd_set_peel_items(uint32_t warp_max, uint32_t mid_max) {
    if (warp_max < 2 || warp_max > 32) {
        set_error("dsd_set_peel_items: warp_max must be 2..32 (got %u)", warp_max);
        return DSD_ERR_INVALID;
    }
    g_item_warp = warp_max;
    g_item_mid = mid_max;
    return DSD_OK;
}

dsd_status dsd_set_checked(int on) {
    g_checked = on ? 1 : 0;
    return DSD_OK;
}

dsd_status dsd_checked_add_selftest(uint64_t start, const uint64_t* addends, uint32_t count,
                                    uint64_t* sum, int* overflowed) {
    set_error("");
    if ((count && !addends) || !sum || !overflowed || count > (1u << 20)) {
        set_error("invalid argument to dsd_checked_add_selftest");
        return DSD_ERR_INVALID;
    }
    return checked_add_selftest(start, addends, count, sum, overflowed);
}

dsd_status dsd_graph_from_edges(uint32_t n, uint64_t m, const uint32_t* src, const uint32_t* dst,
                                int mem, void* cuda_stream, dsd_graph** out) {
    set_error("");
    if (!out || !valid_mem(mem) || (m && (!src || !dst))) {
        set_error("invalid argument to dsd_graph_from_edges");
        return DSD_ERR_INVALID;
    }
    *out = nullptr;
    dsd_graph* g = nullptr;
    DSD_TRY(make_graph(cuda_stream, n, out, &g));
    cudaStream_t s = g->stream;
    const uint32_t* ds = src;
    const uint32_t* dd = dst;
    uint32_t* tmp = nullptr;
    dsd_status st = DSD_OK;
    prof_begin(g, kPhaseCsr);
    if (mem == DSD_MEM_HOST && m) {
        st = dalloc(&tmp, 2 * m, s);
        if (st == DSD_OK) {
            cudaError_t e = cudaMemcpyAsync(tmp, src, m * 4, cudaMemcpyHostToDevice, s);
            if (e == cudaSuccess) e = cudaMemcpyAsync(tmp + m, dst, m * 4, cudaMemcpyHostToDevice, s);
            if (e != cudaSuccess) st = cuda_fail(e, "edge upload", __FILE__, __LINE__);
            ds = tmp;
            dd = tmp + m;
        }
    }
    if (st == DSD_OK) st = build_csr(g, m, ds, dd);
    prof_end(g, kPhaseCsr);
    g->prof_launches[kPhaseCsr] = 12;
    dev_free(tmp, s);
    if (st != DSD_OK) {
        dsd_graph_destroy(g);
        return st;
    }
    *out = g;
    return DSD_OK;
}

dsd_status dsd_graph_from_csr(uint32_t n, const uint64_t* off, const uint32_t* adj, int mem,
                              void* cuda_stream, dsd_graph** out) {
    set_error("");
    if (!out || !off || !valid_mem(mem)) {
        set_error("invalid argument to dsd_graph_from_csr");
        return DSD_ERR_INVALID;
    }
    *out = nullptr;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    uint64_t first = 0, total = 0;
    if (mem == DSD_MEM_HOST) {
        first = off[0];
        total = off[n];
    } else {
        DSD_CU(cudaMemcpyAsync(&first, off, 8, cudaMemcpyDeviceToHost, s));
        DSD_CU(cudaMemcpyAsync(&total, off + n, 8, cudaMemcpyDeviceToHost, s));
        DSD_CU(cudaStreamSynchronize(s));
    }
    if (first != 0 || (total && !adj)) {
        set_error("CSR offsets must start at 0 and adj must be given");
        return DSD_ERR_INVALID;
    }
    uint64_t* doff = nullptr;
    uint32_t* buf = nullptr;   // [total] src + [total] dst
    uint32_t* err = nullptr;
    DSD_TRY(dalloc(&doff, (size_t)n + 1, s));
    dsd_status st = dalloc(&buf, 2 * total + 1, s);
    if (st == DSD_OK) st = dalloc(&err, 1, s);
    uint32_t herr = 0;
    if (st == DSD_OK) {
        cudaMemcpyKind k = mem == DSD_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
        cudaError_t e = cudaMemcpyAsync(doff, off, ((size_t)n + 1) * 8, k, s);
        if (e == cudaSuccess && total) e = cudaMemcpyAsync(buf + total, adj, total * 4, k, s);
        if (e == cudaSuccess) e = cudaMemsetAsync(err, 0, 4, s);
        if (e == cudaSuccess && n) {
            k_check_offsets<<<grid_for(n), 256, 0, s>>>(n, doff, total, err); note_launch();
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, err, 4, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e == cudaSuccess && !herr && n) {
            k_expand_rows<<<grid_for((uint64_t)n * 32), 256, 0, s>>>(n, doff, buf); note_launch();
            e = cudaGetLastError();
        }
        if (e != cudaSuccess) st = cuda_fail(e, "csr upload", __FILE__, __LINE__);
        else if (herr) {
            set_error("CSR offsets must be non-decreasing and end at off[n]");
            st = DSD_ERR_INVALID;
        }
    }
    if (st == DSD_OK) st = dsd_graph_from_edges(n, total, buf, buf + total, DSD_MEM_DEVICE, cuda_stream, out);
    dev_free(doff, s);
    dev_free(buf, s);
    dev_free(err, s);
    return st;
}

void dsd_graph_destroy(dsd_graph* g) {
    if (!g) return;
    cudaStream_t s = g->stream;
    void* ptrs[] = {g->off, g->adj, g->core2, g->rnd, g->new_of, g->old_of, g->roff, g->radj,
                    g->rsplit, g->lvl2_k, g->lvl2_size, g->lvl2_mu, g->core, g->lvl_k,
                    g->lvl_size, g->lvl_mu};
    for (void* p : ptrs) dev_free(p, s);
    cudaStreamSynchronize(s);
    for (int i = 0; i < 2 * DSD_NPHASES; i++)
        if (g->ev[i]) cudaEventDestroy(g->ev[i]);
    delete g;
}

dsd_status dsd_graph_info(const dsd_graph* g, uint32_t* n, uint64_t* m) {
    DSD_TRY(check_graph(g));
    if (n) *n = g->n;
    if (m) *m = g->m;
    return DSD_OK;
}

dsd_status dsd_graph_set_stream(dsd_graph* g, void* cuda_stream) {
    DSD_TRY(check_graph(g));
    DSD_CU(cudaStreamSynchronize(g->stream));
    g->stream = (cudaStream_t)cuda_stream;
    return DSD_OK;
}

dsd_status dsd_graph_csr(dsd_graph* g, uint64_t* off, uint32_t* adj, int mem) {
    DSD_TRY(check_graph(g));
    if (!valid_mem(mem)) return DSD_ERR_INVALID;
    DSD_TRY(copy_out(off, g->off, ((size_t)g->n + 1) * 8, mem, g->stream));
    DSD_TRY(copy_out(adj, g->adj, (size_t)g->m * 2 * 4, mem, g->stream));
    return finish(mem, g->stream);
}

dsd_status dsd_degeneracy_order(dsd_graph* g, uint32_t* core2, uint32_t* rank,
                                uint32_t* degeneracy, int mem) {
    set_error("");
    DSD_TRY(check_graph(g));
    if (!valid_mem(mem)) return DSD_ERR_INVALID;
    DSD_TRY(ensure_order(g));
    cudaStream_t s = g->stream;
    uint32_t n = g->n;
    if (core2) {
        uint32_t* tmp = nullptr;
        uint32_t* dst = core2;
        if (mem == DSD_MEM_HOST) {
            DSD_TRY(dalloc(&tmp, (size_t)n + 1, s));
            dst = tmp;
        }
        if (n) k_u64_to_u32<<<grid_for(n), 256, 0, s>>>(n, g->core2, dst); note_launch();
        DSD_LAUNCHED();
        if (tmp) {
            dsd_status st = copy_out(core2, tmp, (size_t)n * 4, mem, s);
            if (st == DSD_OK) st = finish(mem, s);
            dev_free(tmp, s);
            DSD_TRY(st);
        }
    }
    if (rank) DSD_TRY(copy_out(rank, g->new_of, (size_t)n * 4, mem, s));
    if (degeneracy) {
        if (mem == DSD_MEM_HOST) *degeneracy = g->degeneracy;
        else DSD_CU(cudaMemcpyAsync(degeneracy, &g->degeneracy, 4, cudaMemcpyHostToDevice, s));
    }
    return finish(mem, s);
}

dsd_status dsd_clique_degrees(dsd_graph* g, int h, uint64_t* deg, uint64_t* mu, int mem) {
    set_error("");
    DSD_TRY(check_graph(g));
    DSD_TRY(check_h(h));
    if (!valid_mem(mem)) return DSD_ERR_INVALID;
    DSD_TRY(ensure_order(g));
    cudaStream_t s = g->stream;
    uint32_t n = g->n;
    unsigned long long* dnew = nullptr;
    uint64_t* dout = nullptr;
    DSD_TRY(dalloc(&dnew, (size_t)n + 2, s));
    dsd_status st = DSD_OK;
    if (deg && mem == DSD_MEM_HOST) st = dalloc(&dout, (size_t)n + 1, s);
    if (st == DSD_OK) {
        prof_begin(g, kPhaseCount);
        st = count_cliques(g, h, dnew, dnew + n + 1);
        prof_end(g, kPhaseCount);
    }
    if (st == DSD_OK && deg && n) {
        uint64_t* target = dout ? dout : deg;
        k_map_u64<<<grid_for(n), 256, 0, s>>>(n, g->old_of, (const uint64_t*)dnew, target); note_launch();
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) st = cuda_fail(e, "map", __FILE__, __LINE__);
        if (st == DSD_OK && dout) st = copy_out(deg, dout, (size_t)n * 8, mem, s);
    }
    if (st == DSD_OK && mu) st = copy_out(mu, dnew + n + 1, 8, mem, s);
    if (st == DSD_OK) st = finish(mem, s);
    dev_free(dnew, s);
    dev_free(dout, s);
    return st;
}

dsd_status dsd_core_decompose(dsd_graph* g, int h, uint64_t* core, uint64_t* kmax, int mem) {
    set_error("");
    DSD_TRY(check_graph(g));
    DSD_TRY(check_h(h));
    if (!valid_mem(mem)) return DSD_ERR_INVALID;
    DSD_TRY(decompose(g, h));
    cudaStream_t s = g->stream;
    const uint64_t *lk, *lm, *cv;
    const uint32_t* ls;
    uint32_t nl;
    level_arrays(g, h, &lk, &ls, &lm, &nl, &cv);
    if (core) DSD_TRY(copy_out(core, cv, (size_t)g->n * 8, mem, s));
    if (kmax) {
        uint64_t km = h == 2 ? g->order_kmax : g->last_kmax;
        if (mem == DSD_MEM_HOST) *kmax = km;
        else DSD_CU(cudaMemcpyAsync(kmax, &km, 8, cudaMemcpyHostToDevice, s));
        if (mem == DSD_MEM_DEVICE) DSD_CU(cudaStreamSynchronize(s));
    }
    return finish(mem, s);
}

dsd_status dsd_level_stats(dsd_graph* g, int h, uint64_t* level_k, uint32_t* level_size,
                           uint64_t* level_mu, uint32_t cap, uint32_t* nlevels, int mem) {
    set_error("");
    DSD_TRY(check_graph(g));
    DSD_TRY(check_h(h));
    if (!valid_mem(mem) || !nlevels) return DSD_ERR_INVALID;
    if (h == 2 ? !g->ordered : g->last_h != h) {
        set_error("no decomposition with h = %d has run on this graph", h);
        return DSD_ERR_INVALID;
    }
    const uint64_t *lk, *lm, *cv;
    const uint32_t* ls;
    uint32_t nl;
    level_arrays(g, h, &lk, &ls, &lm, &nl, &cv);
    *nlevels = nl;
    uint32_t c = nl < cap ? nl : cap;
    cudaStream_t s = g->stream;
    DSD_TRY(copy_out(level_k, lk, (size_t)c * 8, mem, s));
    DSD_TRY(copy_out(level_size, ls, (size_t)c * 4, mem, s));
    DSD_TRY(copy_out(level_mu, lm, (size_t)c * 8, mem, s));
    DSD_TRY(finish(mem, s));
    if (nl > cap) {
        set_error("%u levels exceed the capacity %u", nl, cap);
        return DSD_ERR_OVERFLOW;
    }
    return DSD_OK;
}

dsd_status dsd_core_app(dsd_graph* g, int h, uint32_t* kmax_core, uint32_t* densest, int mem,
                        dsd_core_app_result* r) {
    set_error("");
    DSD_TRY(check_graph(g));
    DSD_TRY(check_h(h));
    if (!valid_mem(mem) || !r) {
        set_error("invalid argument to dsd_core_app");
        return DSD_ERR_INVALID;
    }
    DSD_TRY(decompose(g, h));
    cudaStream_t s = g->stream;
    uint32_t n = g->n;
    const uint64_t *lk, *lm, *cv;
    const uint32_t* ls;
    uint32_t nl;
    level_arrays(g, h, &lk, &ls, &lm, &nl, &cv);
    DevResult* dr = nullptr;
    uint32_t* tmp = nullptr;
    DSD_TRY(dalloc(&dr, 1, s));
    dsd_status st = DSD_OK;
    DevResult hr;
    memset(&hr, 0, sizeof(hr));
    prof_begin(g, kPhaseExtract);
    k_best_level<<<1, 1024, 0, s>>>(nl, lk, ls, lm, dr); note_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) st = cuda_fail(e, "best level", __FILE__, __LINE__);
    if (st == DSD_OK && mem == DSD_MEM_HOST && (kmax_core || densest)) st = dalloc(&tmp, (size_t)n + 1, s);
    if (st == DSD_OK && n && kmax_core) {
        uint32_t* target = tmp ? tmp : kmax_core;
        st = extract_set(g, cv, &dr->kmax, target);
        if (st == DSD_OK && tmp) {
            e = cudaMemcpyAsync(&hr, dr, sizeof(hr), cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) st = cuda_fail(e, "result", __FILE__, __LINE__);
            if (st == DSD_OK) st = copy_out(kmax_core, tmp, (size_t)hr.kmax_core_size * 4, mem, s);
            if (st == DSD_OK) st = finish(mem, s);
        }
    }
    if (st == DSD_OK && n && densest) {
        uint32_t* target = tmp ? tmp : densest;
        st = extract_set(g, cv, &dr->best_k, target);
        if (st == DSD_OK && tmp) {
            e = cudaMemcpyAsync(&hr, dr, sizeof(hr), cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) st = cuda_fail(e, "result", __FILE__, __LINE__);
            if (st == DSD_OK) st = copy_out(densest, tmp, (size_t)hr.densest_size * 4, mem, s);
            if (st == DSD_OK) st = finish(mem, s);
        }
    }
    prof_end(g, kPhaseExtract);
    g->prof_launches[kPhaseExtract] = 1 + (kmax_core ? 5 : 0) + (densest ? 5 : 0);
    if (st == DSD_OK) {
        e = cudaMemcpyAsync(&hr, dr, sizeof(hr), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) st = cuda_fail(e, "result", __FILE__, __LINE__);
    }
    dev_free(dr, s);
    dev_free(tmp, s);
    if (st != DSD_OK) return st;
    r->kmax = hr.kmax;
    r->kmax_core_size = hr.kmax_core_size;
    r->kmax_core_mu = hr.kmax_core_mu;
    r->best_k = hr.best_k;
    r->densest_size = hr.densest_size;
    r->densest_mu = hr.densest_mu;
    r->nlevels = hr.nlevels;
    r->seeded_accepted = 0;
    r->seed_k = 0;
    return DSD_OK;
}

dsd_status dsd_peel_stats(dsd_graph* g, int which, uint64_t* out) {
    DSD_TRY(check_graph(g));
    if (!out || (which != 0 && which != 1)) {
        set_error("dsd_peel_stats: which must be 0 or 1 and out non-NULL");
        return DSD_ERR_INVALID;
    }
    for (int i = 0; i < DSD_PEEL_STATS; i++) out[i] = g->peel_stats[which][i];
    return DSD_OK;
}

dsd_status dsd_set_profiling(dsd_graph* g, int on) {
    DSD_TRY(check_graph(g));
    g->profiling = on != 0;
    return DSD_OK;
}

dsd_status dsd_phase_stats(dsd_graph* g, float* ms, uint64_t* bytes, uint32_t* launches) {
    DSD_TRY(check_graph(g));
    DSD_CU(cudaStreamSynchronize(g->stream));
    for (int p = 0; p < DSD_NPHASES; p++) {
        if (g->profiling && g->prof_ms[p] < 0.f) {
            float t = 0.f;
            if (cudaEventElapsedTime(&t, g->ev[2 * p], g->ev[2 * p + 1]) == cudaSuccess)
                g->prof_ms[p] = t;
            else
                (void)cudaGetLastError();
        }
        if (ms) ms[p] = g->prof_ms[p];
        if (bytes) bytes[p] = g->prof_bytes[p];
        if (launches) launches[p] = g->prof_launches[p];
    }
    if (g->profiling && g->last_h >= 3 && bytes) {
        uint64_t b = 0;
        if (count_bytes(g, &b, nullptr) == DSD_OK)
            bytes[kPhaseCount] = g->prof_bytes[kPhaseCount] = b;
    }
    return DSD_OK;
}

dsd_status dsd_listing_bytes(dsd_graph* g, uint64_t* staged, uint64_t* merge) {
    DSD_TRY(check_graph(g));
    return count_bytes(g, staged, merge);
}

}  // extern "C"
