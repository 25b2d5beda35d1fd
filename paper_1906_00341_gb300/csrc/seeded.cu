// The seeded CoreApp call.
//
// A proposal rho' (learn.cu) fixes k = ceil(rho').  Every vertex of the
// (k,Psi)-core has core_2 >= x0 = min{x : C(x, h-1) >= k}: inside R_k each
// vertex lies in >= k h-cliques, which needs >= x0 neighbours in R_k, so R_k
// lies in the x0 edge-core (Sec. 5.2 bounds clique-core numbers the same way
// with gamma = C(core_2, h-1)).  The call therefore builds H = G[{core_2 >=
// x0}], counts h-cliques in H only, and peels H starting at level k (one
// cascade removes everything below k: threshold pruning to R_k).  For every
// j >= k, R_j(H) = R_j(G) because R_j(G) is the largest vertex set with the
// property and lies in H.
//
// Acceptance: some level is >= k and the densest level >= k has density at
// least k - 1 (128-bit integers).  Every level j < k has density at most
// max(rho(R_{j+1}), j) <= ... <= max(rho(R_k), k - 1) (each vertex removed
// at level j destroys at most j cliques), which the densest level >= k then
// reaches, so the densest level (ties to the larger k), k_max and the k_max
// core are all found among the levels >= k (Lemma 5 gives the same
// containment for the optimum).  Every proposal rho' <= rho(S*) passes: the
// densest level's k is at least its density (a level denser than its own k
// is beaten or tied by the next, Theorem 1 bounds the last by k_max), so
// k = ceil(rho') does not exceed it.  A rejected proposal falls back to the
// plain decomposition.
#include "graph.cuh"

#include <math.h>
#include <new>
#include <string.h>

struct dsd_model;

namespace dsd {

dsd_status compute_features(dsd_graph* g, int h, float* f_dev);
dsd_status model_propose(dsd_model* M, const float* f_dev, float* rho_dev, cudaStream_t s);
dsd_status count_cliques(dsd_graph* g, int h, unsigned long long* deg_new,
                         unsigned long long* mu_dev);

namespace {

__global__ void k_sub_flags(uint32_t n, const uint64_t* core2, uint64_t x0, uint32_t* flag) {
    for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (uint64_t)gridDim.x * blockDim.x)
        flag[v] = core2[v] >= x0 ? 1u : 0u;
}

__global__ void k_sub_map(uint32_t n, const uint32_t* flag, const uint64_t* pos, uint32_t* map,
                          uint32_t* orig) {
    for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (uint64_t)gridDim.x * blockDim.x) {
        if (flag[v]) {
            map[v] = (uint32_t)pos[v];
            orig[pos[v]] = (uint32_t)v;
        } else {
            map[v] = 0xffffffffu;
        }
    }
}

// Edges of H, each once (u < w): count per vertex, then fill.
__global__ void k_sub_count(uint32_t n, const uint64_t* off, const uint32_t* adj,
                            const uint32_t* map, uint32_t* cnt) {
    uint64_t gw = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    unsigned lane = lane_id();
    for (uint64_t v = gw; v < n; v += nw) {
        unsigned c = 0;
        if (map[v] != 0xffffffffu)
            for (uint64_t p = off[v] + lane; p < off[v + 1]; p += 32) {
                uint32_t u = adj[p];
                if (u > v && map[u] != 0xffffffffu) c++;
            }
        c = warp_sum(c);
        if (lane == 0) cnt[v] = c;
    }
}

__global__ void k_sub_fill(uint32_t n, const uint64_t* off, const uint32_t* adj,
                           const uint32_t* map, const uint64_t* epos, uint32_t* src,
                           uint32_t* dst) {
    uint64_t gw = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    unsigned lane = lane_id();
    for (uint64_t v = gw; v < n; v += nw) {
        if (map[v] == 0xffffffffu) continue;
        uint64_t at = epos[v];
        for (uint64_t p0 = off[v]; p0 < off[v + 1]; p0 += 32) {
            uint64_t p = p0 + lane;
            bool ok = false;
            uint32_t u = 0;
            if (p < off[v + 1]) {
                u = adj[p];
                ok = u > v && map[u] != 0xffffffffu;
            }
            unsigned b = __ballot_sync(0xffffffffu, ok);
            if (ok) {
                uint64_t q = at + __popc(b & ((1u << lane) - 1u));
                src[q] = map[v];
                dst[q] = map[u];
            }
            at += __popc(b);
        }
    }
}

struct SeedRes {
    unsigned long long kmax, kmax_core_mu, best_k, densest_mu;
    uint32_t kmax_core_size, densest_size, nlevels, accepted;
};

__device__ __forceinline__ bool ratio_ge2(unsigned long long a, unsigned long long b,
                                          unsigned long long c, unsigned long long d) {
    unsigned __int128 l = (unsigned __int128)a * d, r = (unsigned __int128)c * b;
    return l >= r;
}

// Among the levels >= k: the densest (ties to the larger k) and the last.
// Accepted iff a level >= k exists and that densest one has density at
// least k - 1: every level j < k then has density at most max(rho(R_k),
// k - 1) (each vertex leaving at level j holds at most j cliques when it
// leaves), so no lower level beats it and the answer lies among the levels
// >= k.  One thread; the level count is small.
__global__ void k_seed_select(uint32_t nl, const uint64_t* lk, const uint32_t* ls,
                              const uint64_t* lm, unsigned long long k, SeedRes* out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    SeedRes r;
    memset(&r, 0, sizeof(r));
    uint32_t j0 = 0;
    while (j0 < nl && lk[j0] < k) j0++;
    uint32_t best = j0;
    for (uint32_t j = j0 + 1; j < nl; j++)
        if (ratio_ge2(lm[j], ls[j], lm[best], ls[best])) best = j;
    // rho(R_best) >= k - 1  <=>  mu >= (k - 1) * |R_best|  (128-bit)
    if (j0 < nl && ratio_ge2(lm[best], ls[best], k - 1, 1)) {
        r.accepted = 1;
        r.kmax = lk[nl - 1];
        r.kmax_core_size = ls[nl - 1];
        r.kmax_core_mu = lm[nl - 1];
        r.best_k = lk[best];
        r.densest_size = ls[best];
        r.densest_mu = lm[best];
        r.nlevels = nl - j0;
    }
    *out = r;
}

// core of H vertex (H ids) from its rank-space core; flags >= threshold.
__global__ void k_sub_flags_core(uint32_t nh, const uint32_t* old_of_rank, const uint64_t* core_rank,
                                 unsigned long long t, uint32_t* flag_h) {
    for (uint64_t p = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; p < nh;
         p += (uint64_t)gridDim.x * blockDim.x)
        flag_h[old_of_rank[p]] = core_rank[p] >= t ? 1u : 0u;
}

__global__ void k_sub_emit(uint32_t nh, const uint32_t* flag, const uint64_t* pos,
                           const uint32_t* orig, uint32_t* out) {
    for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < nh;
         v += (uint64_t)gridDim.x * blockDim.x)
        if (flag[v]) out[pos[v]] = orig[v];
}

unsigned grid_n(uint64_t n) {
    uint64_t b = (n + 255) / 256;
    return (unsigned)(b < 1 ? 1 : (b > 152 * 16 ? 152 * 16 : b));
}

// C(x, r) >= k, without overflow (the running product C(x-r+t, t) is exact).
bool binom_ge(uint64_t x, int r, uint64_t k) {
    if (x < (uint64_t)r) return k == 0;
    unsigned __int128 c = 1;
    for (int t = 1; t <= r; t++) {
        c = c * (unsigned __int128)(x - r + t) / (unsigned __int128)t;
        if (c >= k) return true;
    }
    return c >= k;
}

// x0 = min{x : C(x, h-1) >= k} searched in [h-1, cap]; cap + 1 if none.
uint64_t min_x_for(uint64_t k, int h, uint64_t cap) {
    uint64_t lo = (uint64_t)(h - 1), hi = cap + 1;
    if (lo > cap) return cap + 1;
    while (lo < hi) {
        uint64_t mid = lo + (hi - lo) / 2;
        if (binom_ge(mid, h - 1, k)) hi = mid;
        else lo = mid + 1;
    }
    return lo;
}

}  // namespace

void sub_core_free(SubCore* S, cudaStream_t s) {
    if (S->H) dsd_graph_destroy(S->H);
    void* ptrs[] = {S->orig, S->core, S->lk, S->ls, S->lm};
    for (void* p : ptrs) dev_free(p, s);
    *S = SubCore();
}

dsd_status induced_subgraph(dsd_graph* g, const uint32_t* flag, dsd_graph** Hout,
                            uint32_t** orig_out) {
    *Hout = nullptr;
    *orig_out = nullptr;
    cudaStream_t s = g->stream;
    const uint32_t n = g->n;
    uint32_t *map = nullptr, *cnt = nullptr, *es = nullptr, *orig = nullptr;
    uint64_t *pos = nullptr, *epos = nullptr;
    uint64_t nh = 0, mh = 0;
    dsd_graph* H = nullptr;
    dsd_status st = DSD_OK;
    cudaError_t e = cudaSuccess;
#define SSTEP(x)                         \
    do {                                 \
        st = (x);                        \
        if (st != DSD_OK) goto done;     \
    } while (0)
#define SCU(x)                                                                          \
    do {                                                                                \
        e = (x);                                                                        \
        if (e != cudaSuccess) { st = cuda_fail(e, #x, __FILE__, __LINE__); goto done; } \
    } while (0)
    SSTEP(dalloc(&map, (size_t)n + 1, s));
    SSTEP(dalloc(&cnt, (size_t)n + 1, s));
    SSTEP(dalloc(&pos, (size_t)n + 1, s));
    SSTEP(dalloc(&epos, (size_t)n + 1, s));
    SSTEP(exclusive_scan_u32_to_u64(flag, pos, n, s));
    SCU(cudaMemcpyAsync(&nh, pos + n, 8, cudaMemcpyDeviceToHost, s));
    SCU(cudaStreamSynchronize(s));
    SSTEP(dalloc(&orig, nh + 1, s));
    if (n) {
        k_sub_map<<<grid_n(n), 256, 0, s>>>(n, flag, pos, map, orig);
        k_sub_count<<<grid_n((uint64_t)n * 32), 256, 0, s>>>(n, g->off, g->adj, map, cnt);
        note_launch();
        note_launch();
    }
    SSTEP(exclusive_scan_u32_to_u64(cnt, epos, n, s));
    SCU(cudaMemcpyAsync(&mh, epos + n, 8, cudaMemcpyDeviceToHost, s));
    SCU(cudaStreamSynchronize(s));
    SSTEP(dalloc(&es, 2 * mh + 2, s));
    if (n) {
        k_sub_fill<<<grid_n((uint64_t)n * 32), 256, 0, s>>>(n, g->off, g->adj, map, epos, es,
                                                           es + mh);
        note_launch();
    }
    SCU(cudaGetLastError());
    H = new (std::nothrow) dsd_graph();
    if (!H) {
        st = DSD_ERR_NOMEM;
        goto done;
    }
    H->stream = s;
    H->n = (uint32_t)nh;
    H->device = g->device;
    SSTEP(build_csr(H, mh, es, es + mh));
done:
#undef SSTEP
#undef SCU
    void* ptrs[] = {map, cnt, es, pos, epos};
    for (void* p : ptrs) dev_free(p, s);
    if (st != DSD_OK) {
        if (H) dsd_graph_destroy(H);
        dev_free(orig, s);
        return st;
    }
    *Hout = H;
    *orig_out = orig;
    return DSD_OK;
}

dsd_status sub_core_build(dsd_graph* g, int h, uint64_t x0, uint64_t kstart, SubCore* S) {
    *S = SubCore();
    cudaStream_t s = g->stream;
    const uint32_t n = g->n;
    uint32_t* flag = nullptr;
    unsigned long long* deg = nullptr;
    dsd_status st = DSD_OK;
    cudaError_t e = cudaSuccess;
#define SSTEP(x)                         \
    do {                                 \
        st = (x);                        \
        if (st != DSD_OK) goto done;     \
    } while (0)
#define SCU(x)                                                                          \
    do {                                                                                \
        e = (x);                                                                        \
        if (e != cudaSuccess) { st = cuda_fail(e, #x, __FILE__, __LINE__); goto done; } \
    } while (0)
    SSTEP(dalloc(&flag, (size_t)n + 1, s));
    if (n) {
        k_sub_flags<<<grid_n(n), 256, 0, s>>>(n, g->core2, x0, flag);
        note_launch();
    }
    SSTEP(induced_subgraph(g, flag, &S->H, &S->orig));
    S->nh = S->H->n;
    S->mh = S->H->m;
    SSTEP(ensure_order(S->H));
    SSTEP(dalloc(&deg, S->nh + 2, s));
    SSTEP(dalloc(&S->core, S->nh + 1, s));
    SSTEP(dalloc(&S->lk, S->nh + 1, s));
    SSTEP(dalloc(&S->lm, S->nh + 1, s));
    SSTEP(dalloc(&S->ls, S->nh + 1, s));
    SSTEP(count_cliques(S->H, h, deg, deg + S->nh + 1));
    SCU(cudaMemcpyAsync(&S->mu, deg + S->nh + 1, 8, cudaMemcpyDeviceToHost, s));
    SCU(cudaStreamSynchronize(s));
    SSTEP(run_peel(S->H, h, S->H->n, S->H->roff, S->H->radj, S->H->rsplit, S->H->maxdplus, deg,
                   S->mu, S->core, nullptr, S->lk, S->ls, S->lm, &S->pr, kstart));
done:
#undef SSTEP
#undef SCU
    dev_free(flag, s);
    dev_free(deg, s);
    if (st != DSD_OK) sub_core_free(S, s);
    return st;
}

dsd_status sub_core_emit(dsd_graph* g, const SubCore& S, uint64_t thr, uint32_t size,
                         uint32_t* out, int mem) {
    if (!out || S.nh == 0) return DSD_OK;
    cudaStream_t s = g->stream;
    uint32_t* fh = nullptr;
    uint64_t* ph = nullptr;
    uint32_t* tmp = nullptr;
    dsd_status st = dalloc(&fh, S.nh + 1, s);
    if (st == DSD_OK) st = dalloc(&ph, S.nh + 1, s);
    if (st == DSD_OK && mem == DSD_MEM_HOST) st = dalloc(&tmp, S.nh + 1, s);
    if (st == DSD_OK) {
        k_sub_flags_core<<<grid_n(S.nh), 256, 0, s>>>((uint32_t)S.nh, S.H->old_of, S.core, thr, fh);
        note_launch();
        st = exclusive_scan_u32_to_u64(fh, ph, S.nh, s);
    }
    if (st == DSD_OK) {
        k_sub_emit<<<grid_n(S.nh), 256, 0, s>>>((uint32_t)S.nh, fh, ph, S.orig, tmp ? tmp : out);
        note_launch();
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess && tmp)
            e = cudaMemcpyAsync(out, tmp, (size_t)size * 4, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) st = cuda_fail(e, "core set", __FILE__, __LINE__);
    }
    dev_free(fh, s);
    dev_free(ph, s);
    dev_free(tmp, s);
    return st;
}

}  // namespace dsd

using namespace dsd;

extern "C" {

dsd_status dsd_core_app_seeded_info(dsd_graph* g, int h, const dsd_model* Mc,
                                    uint32_t* kmax_core, uint32_t* densest, int mem,
                                    dsd_core_app_result* r, dsd_seed_info* info) {
    set_error("");
    // the proposal reads the weights; the model's device work buffers are
    // scratch that the call may overwrite
    dsd_model* M = const_cast<dsd_model*>(Mc);
    if (!g || !M || !r || h < 2 || h > DSD_MAX_H || (mem != DSD_MEM_HOST && mem != DSD_MEM_DEVICE)) {
        set_error("invalid argument to dsd_core_app_seeded");
        return DSD_ERR_INVALID;
    }
    dsd_seed_info si;
    memset(&si, 0, sizeof(si));
    cudaStream_t s = g->stream;
    DSD_TRY(ensure_order(g));
    uint32_t n = g->n;
    // ---- proposal
    float* fbuf = nullptr;
    DSD_TRY(dalloc(&fbuf, 72, s));
    dsd_status st = compute_features(g, h, fbuf);
    if (st == DSD_OK) st = model_propose(M, fbuf, fbuf + 64, s);
    float rho = 0.f;
    if (st == DSD_OK) {
        cudaError_t e = cudaMemcpyAsync(&rho, fbuf + 64, 4, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) st = cuda_fail(e, "proposal", __FILE__, __LINE__);
    }
    dev_free(fbuf, s);
    DSD_TRY(st);
    si.rho_prime = rho;
    // a proposal of 2^62 or more cannot be met by any graph with < 2^32 vertices
    bool try_seed = n > 0 && isfinite(rho) && rho > 0.f && rho < 4.6e18f;
    uint64_t k = 0, x0 = 0;
    if (try_seed) {
        k = (uint64_t)ceilf(rho);
        if (k < 1) k = 1;
        x0 = min_x_for(k, h, g->degeneracy);
        si.seed_k = k;
        si.x0 = x0;
        if (x0 > g->degeneracy) try_seed = false;   // no vertex can reach level k
    }
    if (try_seed) {
        SubCore S;
        SeedRes hs;
        memset(&hs, 0, sizeof(hs));
        SeedRes* sr = nullptr;
        st = sub_core_build(g, h, x0, k, &S);
        if (st == DSD_OK) {
            si.sub_n = (uint32_t)S.nh;
            si.sub_m = S.mh;
            record_peel(g, 1, S.pr);
            st = dalloc(&sr, 1, s);
        }
        if (st == DSD_OK) {
            k_seed_select<<<1, 32, 0, s>>>(S.pr.nlevels, S.lk, S.ls, S.lm, k, sr);
            note_launch();
            cudaError_t e = cudaMemcpyAsync(&hs, sr, sizeof(hs), cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) st = cuda_fail(e, "seed select", __FILE__, __LINE__);
        }
        if (st == DSD_OK && hs.accepted) {
            st = sub_core_emit(g, S, hs.kmax, hs.kmax_core_size, kmax_core, mem);
            if (st == DSD_OK) st = sub_core_emit(g, S, hs.best_k, hs.densest_size, densest, mem);
        }
        dev_free(sr, s);
        sub_core_free(&S, s);
        DSD_TRY(st);
        if (hs.accepted) {
            si.accepted = 1;
            memset(r, 0, sizeof(*r));
            r->kmax = hs.kmax;
            r->kmax_core_size = hs.kmax_core_size;
            r->kmax_core_mu = hs.kmax_core_mu;
            r->best_k = hs.best_k;
            r->densest_size = hs.densest_size;
            r->densest_mu = hs.densest_mu;
            r->nlevels = hs.nlevels;
            r->seeded_accepted = 1;
            r->seed_k = k;
            if (info) *info = si;
            return DSD_OK;
        }
    }
    // ---- rejected (or no usable proposal): the plain path
    st = dsd_core_app(g, h, kmax_core, densest, mem, r);
    if (st == DSD_OK) r->seed_k = si.seed_k;
    if (info) *info = si;
    return st;
}

dsd_status dsd_core_app_seeded(dsd_graph* g, int h, const dsd_model* m, uint32_t* kmax_core,
                               uint32_t* densest, int mem, dsd_core_app_result* r) {
    return dsd_core_app_seeded_info(g, h, m, kmax_core, densest, mem, r, nullptr);
}

}  // extern "C"
