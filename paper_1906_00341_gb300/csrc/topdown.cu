// CoreApp's top-down schedule (Algorithm 6, Sec. 5.2) on the GPU.
//
// CoreApp visits vertices in decreasing order of the bound gamma(v) =
// C(core_2(v), h-1) on their clique-core number and decomposes a growing
// window W of the top vertices, doubling it until no vertex outside W can
// reach the k_max core.  Sorting by gamma is sorting by core_2, so each
// window here is an edge core {core_2 >= x} (its size read from the level
// records of the degeneracy peel), and the window's decomposition is the
// (k,Psi)-core decomposition of that induced subgraph H.
//
// With gamma_out = the largest gamma outside H and K = gamma_out + 1, every
// R_j(G) with j >= K lies inside H and equals R_j(H) (R_j is the largest set
// with the property).  So:
//   * k_max(G) = k_max(H) and the k_max cores agree once k_max(H) >= K
//     (CoreApp's stopping rule);
//   * the densest level of G is the densest level of H at or above K once
//     that level's density is >= K - 1: every level j < K has density at
//     most max(rho(R_K), K - 1) (each vertex leaving at level j holds <= j
//     cliques when it leaves), and ties go to the larger k.  This second test
//     is the weaker acceptance test of the learned path, with K in place of
//     ceil(rho').
// The window doubles until both hold; when it is the whole graph both hold
// trivially.  As CoreApp restricts each window to the levels that can still
// matter, a window is peeled from level K (threshold pruning to R_K(H) in
// one cascade), not from 0.  The outputs equal dsd_core_app's.
#include "graph.cuh"

#include <string.h>
#include <vector>

namespace dsd {
namespace {

// C(x, r) saturated at 2^64 - 1.
uint64_t binom_sat(uint64_t x, int r) {
    if (x < (uint64_t)r) return 0;
    unsigned __int128 c = 1;
    for (int t = 1; t <= r; t++) {
        c = c * (unsigned __int128)(x - r + t) / (unsigned __int128)t;
        if (c >> 64) return ~0ull;
    }
    return (uint64_t)c;
}

bool ratio_ge(uint64_t a, uint64_t b, uint64_t c, uint64_t d) {   // a/b >= c/d
    return (unsigned __int128)a * d >= (unsigned __int128)c * b;
}

}  // namespace
}  // namespace dsd

using namespace dsd;

extern "C" {

dsd_status dsd_core_app_topdown(dsd_graph* g, int h, uint32_t* kmax_core, uint32_t* densest,
                                int mem, dsd_core_app_result* r, dsd_topdown_info* info) {
    set_error("");
    if (!g || !r || h < 2 || h > DSD_MAX_H || (mem != DSD_MEM_HOST && mem != DSD_MEM_DEVICE)) {
        set_error("invalid argument to dsd_core_app_topdown");
        return DSD_ERR_INVALID;
    }
    dsd_topdown_info ti;
    memset(&ti, 0, sizeof(ti));
    DSD_TRY(ensure_order(g));
    cudaStream_t s = g->stream;
    const uint32_t nl2 = g->nlevels2;
    if (h == 2 || g->n == 0 || nl2 == 0) {
        // the degeneracy peel already is the h = 2 decomposition
        dsd_status st = dsd_core_app(g, h, kmax_core, densest, mem, r);
        ti.passes = 1;
        ti.sub_n = g->n;
        ti.sub_m = g->m;
        if (info) *info = ti;
        return st;
    }
    // edge-core sizes: level j of the h = 2 peel has value k2[j] and
    // |{core_2 >= k2[j]}| = s2[j] (values ascending, sizes descending)
    std::vector<uint64_t> k2(nl2);
    std::vector<uint32_t> s2(nl2);
    DSD_CU(cudaMemcpyAsync(k2.data(), g->lvl2_k, nl2 * 8, cudaMemcpyDeviceToHost, s));
    DSD_CU(cudaMemcpyAsync(s2.data(), g->lvl2_size, nl2 * 4, cudaMemcpyDeviceToHost, s));
    DSD_CU(cudaStreamSynchronize(s));
    // initial window: the top edge core, at least 1024 vertices (the paper
    // leaves the initial size open)
    uint64_t want = s2[nl2 - 1] > 1024 ? s2[nl2 - 1] : 1024;
    for (;;) {
        ti.passes++;
        // the largest level whose edge core holds >= want vertices
        uint32_t j = nl2 - 1;
        while (j > 0 && s2[j] < want) j--;
        const bool whole = j == 0;
        const uint64_t x = k2[j];
        const uint64_t gout = whole ? 0 : binom_sat(k2[j - 1], h - 1);
        const uint64_t K = whole ? 0 : (gout == ~0ull ? ~0ull : gout + 1);
        // only the levels at or above K can be answers: the window is peeled
        // from level K (one cascade removes everything below it)
        SubCore S;
        DSD_TRY(sub_core_build(g, h, x, (whole || K == ~0ull) ? 0 : K, &S));
        const uint32_t nl = S.pr.nlevels;
        std::vector<uint64_t> lk(nl), lm(nl);
        std::vector<uint32_t> ls(nl);
        cudaError_t e = cudaSuccess;
        if (nl) {
            e = cudaMemcpyAsync(lk.data(), S.lk, (size_t)nl * 8, cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(lm.data(), S.lm, (size_t)nl * 8, cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(ls.data(), S.ls, (size_t)nl * 4, cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        }
        if (e != cudaSuccess) {
            sub_core_free(&S, s);
            return cuda_fail(e, "top-down levels", __FILE__, __LINE__);
        }
        bool done = false;
        uint32_t j0 = 0, best = 0;
        if (nl) {
            const uint64_t kmaxH = lk[nl - 1];
            while (j0 < nl && lk[j0] < K) j0++;
            if (j0 < nl && kmaxH >= K) {
                best = j0;
                for (uint32_t q = j0 + 1; q < nl; q++)
                    if (ratio_ge(lm[q], ls[q], lm[best], ls[best])) best = q;
                // densest level accepted if its density >= K - 1
                done = whole || (unsigned __int128)lm[best] >=
                                    (unsigned __int128)(K - 1) * ls[best];
            }
        }
        if (done) {
            record_peel(g, 1, S.pr);
            ti.x = x;
            ti.gamma_out = gout;
            ti.sub_n = (uint32_t)S.nh;
            ti.sub_m = S.mh;
            memset(r, 0, sizeof(*r));
            r->kmax = lk[nl - 1];
            r->kmax_core_size = ls[nl - 1];
            r->kmax_core_mu = lm[nl - 1];
            r->best_k = lk[best];
            r->densest_size = ls[best];
            r->densest_mu = lm[best];
            r->nlevels = nl - j0;
            dsd_status st = sub_core_emit(g, S, r->kmax, r->kmax_core_size, kmax_core, mem);
            if (st == DSD_OK) st = sub_core_emit(g, S, r->best_k, r->densest_size, densest, mem);
            sub_core_free(&S, s);
            if (info) *info = ti;
            return st;
        }
        sub_core_free(&S, s);
        if (whole) {
            set_error("top-down schedule did not converge on the whole graph");
            return DSD_ERR_INTERNAL;
        }
        want *= 2;
    }
}

}  // extern "C"
