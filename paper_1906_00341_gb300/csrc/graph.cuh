// The graph handle and the internal entry points of each stage.
#pragma once

#include "common.cuh"

enum {
    kPhaseCsr = 0,
    kPhaseOrderPeel = 1,
    kPhaseOrient = 2,
    kPhaseCount = 3,
    kPhasePeel = 4,
    kPhaseExtract = 5,
};

struct dsd_graph {
    int device = 0;
    cudaStream_t stream = nullptr;
    uint32_t n = 0;
    uint64_t m = 0;               // undirected edges after cleaning

    // cleaned CSR in the caller's vertex ids (rows ascending)
    uint64_t* off = nullptr;      // [n+1]
    uint32_t* adj = nullptr;      // [2m]

    // degeneracy ordering (h = 2 peel) and the relabelled CSR
    bool ordered = false;
    uint64_t* core2 = nullptr;    // [n] edge core numbers, caller ids
    uint32_t* rnd = nullptr;      // [n] peeling round, caller ids
    uint32_t* new_of = nullptr;   // [n] caller id -> rank
    uint32_t* old_of = nullptr;   // [n] rank -> caller id
    uint64_t* roff = nullptr;     // [n+1] relabelled CSR (ids = ranks)
    uint32_t* radj = nullptr;     // [2m]
    uint64_t* rsplit = nullptr;   // [n] first entry of N+(v) in radj
    uint32_t degeneracy = 0;
    uint32_t maxdplus = 0;        // max |N+(v)|
    uint64_t order_kmax = 0;

    // levels of the h = 2 peel (caller ids space; levels are id-free)
    uint32_t nlevels2 = 0;
    uint64_t* lvl2_k = nullptr;
    uint32_t* lvl2_size = nullptr;
    uint64_t* lvl2_mu = nullptr;

    // results of the last (k,Psi) decomposition with h >= 3
    int last_h = 0;
    uint64_t* core = nullptr;     // [n] caller ids
    uint64_t last_kmax = 0;
    uint64_t last_mu = 0;
    uint32_t nlevels = 0;
    uint64_t* lvl_k = nullptr;    // [n+1]
    uint32_t* lvl_size = nullptr;
    uint64_t* lvl_mu = nullptr;

    // peel statistics: [0] degeneracy peel, [1] last (k,Psi) peel
    uint64_t peel_stats[2][DSD_PEEL_STATS] = {};

    // profiling
    bool profiling = false;
    cudaEvent_t ev[2 * 6] = {};
    float prof_ms[6] = {};
    uint64_t prof_bytes[6] = {};
    uint32_t prof_launches[6] = {};
};

namespace dsd {

// CSR construction.  src/dst on the device.
dsd_status build_csr(dsd_graph* g, uint64_t m, const uint32_t* src, const uint32_t* dst);

// Degeneracy order + relabelled CSR, cached on g.
dsd_status ensure_order(dsd_graph* g);

// h-clique counting on the relabelled graph: deg_new[rank] and *mu_dev (device pointers).
dsd_status count_cliques(dsd_graph* g, int h, unsigned long long* deg_new,
                         unsigned long long* mu_dev);
// Algorithmic bytes of one listing under the kernels' staging model and
// under a merge-intersection model (k_count_bytes).
dsd_status count_bytes(dsd_graph* g, uint64_t* staged, uint64_t* merge);
// The counting kernels' checked addition on given values (dsd_checked_add_selftest).
dsd_status checked_add_selftest(uint64_t start, const uint64_t* addends, uint32_t count,
                                uint64_t* sum, int* overflowed);

// Level-synchronous (k,Psi)-core peeling.
struct PeelResult {
    uint64_t kmax = 0;
    uint32_t nlevels = 0;
    uint32_t rounds = 0;
    uint64_t items = 0;       // frontier work items processed
    uint64_t bytes = 0;       // metered algorithmic bytes
    uint64_t barrier_ns = 0;  // time block 0 spent in grid barriers
    uint32_t barriers = 0;
    uint32_t compactions = 0;
    uint32_t threads = 0;     // block size used
    uint32_t grid = 0;        // blocks launched
    uint32_t small_round = 0; // first round of the small regime (0 = never)
    uint64_t tph[8] = {};     // block 0's time per phase (ns)
    uint32_t tail_n = 0;      // alive vertices handed to the cluster tail kernel
    uint32_t tail_round = 0;  // round of the hand-over
    uint64_t tail_ns = 0;     // the tail kernel's duration
    uint64_t tail_tph[7] = {};  // the tail's time per phase (ns)
};
// off/adj/split: CSR in the working id space (split may be null for h = 2).
// deg: [n] clique-degrees in, destroyed on return.  core/rnd: [n] outputs
// (rnd may be null).  lvl_*: [n+1] level records.
dsd_status run_peel(dsd_graph* g, int h, uint32_t n, const uint64_t* off, const uint32_t* adj,
                    const uint64_t* split, uint32_t maxdplus, unsigned long long* deg,
                    uint64_t mu0, uint64_t* core, uint32_t* rnd, uint64_t* lvl_k,
                    uint32_t* lvl_size, uint64_t* lvl_mu, PeelResult* res,
                    uint64_t kstart = 0, uint64_t* snap = nullptr);
// snap (may be null; no cluster tail then): snap[v] receives v's count in
// R_core(v), its clique-degree inside its own (k,Psi)-core.
// kstart > 0: the first level removes every vertex with fewer than kstart
// cliques in one cascade (threshold pruning to the (kstart,Psi)-core); its
// level record is then (kstart - 1, |V|, mu) and the core numbers it assigns
// are not core numbers.  Levels at or above kstart are exact.

// G[{v : flag[v] != 0}] (flag: device, n entries) as a graph of its own, ids
// ascending with g's ids; *orig (device, |H| entries) maps H ids to g ids.
// The caller destroys *H and frees *orig (dev_free on g's stream).
dsd_status induced_subgraph(dsd_graph* g, const uint32_t* flag, dsd_graph** H, uint32_t** orig);

// The edge core {core_2 >= x0} of g as a graph of its own (ids ascend with
// g's ids), its h-clique counts, and its peel from level kstart (levels at or
// above kstart exact).  Used by the seeded and the top-down CoreApp calls.
struct SubCore {
    dsd_graph* H = nullptr;
    uint32_t* orig = nullptr;     // H id -> g id
    uint64_t* core = nullptr;     // H rank space
    uint64_t* lk = nullptr;       // level records [nlevels]
    uint32_t* ls = nullptr;
    uint64_t* lm = nullptr;
    uint64_t nh = 0, mh = 0;
    unsigned long long mu = 0;
    PeelResult pr;
};
dsd_status sub_core_build(dsd_graph* g, int h, uint64_t x0, uint64_t kstart, SubCore* S);
// The g ids (ascending) of the H vertices with core >= thr into out (size
// entries; host or device memory by mem).
dsd_status sub_core_emit(dsd_graph* g, const SubCore& S, uint64_t thr, uint32_t size,
                         uint32_t* out, int mem);
void sub_core_free(SubCore* S, cudaStream_t s);

// Statistics of the last peel runs: [0] degeneracy peel, [1] (k,Psi) peel.
void record_peel(dsd_graph* g, int which, const PeelResult& r);

// Profiling helpers.
void prof_begin(dsd_graph* g, int phase);
void prof_end(dsd_graph* g, int phase);

}  // namespace dsd
