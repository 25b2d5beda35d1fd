/*
 * dsd.h -- C ABI of libdsd: h-clique clique-degrees, (k,Psi)-core
 * decomposition and CoreApp outputs on one NVIDIA GB300 GPU (sm_103a).
 *
 * The operations follow Fang, Yu, Cheng, Lakshmanan, Lin, "Efficient
 * Algorithms for Densest Subgraph Discovery", PVLDB 12(11), 2019:
 *   - graph model: undirected, unweighted, simple (Sec. 2, "Data model");
 *   - clique instance, clique-degree deg(v,Psi), mu(G,Psi), density
 *     rho = mu/|V| (Sec. 2, Defs. 2-4; Problem 1);
 *   - (k,Psi)-core R_k, clique-core number core(v,Psi), k_max
 *     (Sec. 4.1, Def. 6);
 *   - (k,Psi)-core decomposition (Sec. 4.3, Algorithm 3);
 *   - IncApp / CoreApp output: the (k_max,Psi)-core (Sec. 5.2, Algorithms 5
 *     and 6, Lemma 6), and the densest residual subgraph met while peeling
 *     (Sec. 5.1, Pruning1), returned as the densest nested level set R_k;
 *   - CoreExact: the exact h-clique densest subgraph by minimum cuts
 *     (Sec. 3.1 Algorithm 1's network, Sec. 4.3 Algorithm 4);
 *   - pattern densities for the x-star and the 4-vertex loop (Sec. 6 and
 *     its appendix on special patterns).
 * Not in the paper: a learned density proposal that narrows the
 * decomposition (exact either way), a batched executor for many small
 * graphs, and an allocation-free triangle-degree entry point.
 *
 * Conventions shared by every call:
 *   - Vertex ids are uint32 in [0, n).  Per-vertex counters are uint64.
 *   - h (the clique size |V_Psi|) must satisfy 2 <= h <= DSD_MAX_H.
 *   - `mem` says where caller buffers live: DSD_MEM_HOST (pageable or pinned
 *     host memory) or DSD_MEM_DEVICE (device memory of the graph's GPU).
 *     Every output buffer is allocated and owned by the caller; the library
 *     never frees caller memory and keeps no pointer to it after returning.
 *   - Work is ordered on the graph's CUDA stream (given at creation, changed
 *     with dsd_graph_set_stream).  A call with DSD_MEM_HOST outputs returns
 *     after the results are in host memory; with DSD_MEM_DEVICE outputs it
 *     may return before the stream has finished (synchronise the stream to
 *     read them).
 *   - Errors are returned as dsd_status, never thrown; dsd_last_error()
 *     gives a message for the calling thread.  After DSD_ERR_CUDA the graph
 *     handle should be destroyed; after DSD_ERR_TIMEOUT of a peel as well
 *     (its state is partial), while a CoreExact timeout leaves the handle
 *     usable.
 *   - A handle is not thread-safe; distinct handles are independent.
 *   - Every call computes its result entirely on the GPU; there is no CPU
 *     fallback.  Without a usable CUDA device calls return DSD_ERR_CUDA.
 */
#ifndef DSD_H
#define DSD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define DSD_MAX_H 8

typedef enum {
    DSD_OK = 0,
    DSD_ERR_INVALID = 1,     /* bad argument: NULL pointer, h out of range, id >= n, ... */
    DSD_ERR_NOMEM = 2,       /* device or host allocation failed */
    DSD_ERR_CUDA = 3,        /* a CUDA runtime call or kernel failed */
    DSD_ERR_TIMEOUT = 4,     /* a bounded inter-block wait ran out (see dsd_set_wait_limit_ms) */
    DSD_ERR_OVERFLOW = 5,    /* a result does not fit the caller's buffer or a counter overflowed */
    DSD_ERR_INTERNAL = 6,    /* a self-check of the library failed (message says which) */
    DSD_ERR_UNSUPPORTED = 7  /* input outside what the library handles (message says why) */
} dsd_status;

enum { DSD_MEM_HOST = 0, DSD_MEM_DEVICE = 1 };

typedef struct dsd_graph dsd_graph;   /* opaque */

/* ------------------------------------------------------------------ meta */

const char* dsd_status_string(dsd_status s);
/* Message for the last failed call on this thread ("" if none). */
const char* dsd_last_error(void);
/* Library version string. */
const char* dsd_version(void);
/* Number of CUDA kernels the library has launched in this process so far
 * (all devices, all handles); the difference across a region counts the
 * launches inside it. */
uint64_t dsd_kernel_launches(void);

/* Upper bound, in milliseconds, on every inter-block wait inside a
 * persistent kernel (grid barriers).  A wait that runs out makes the kernel
 * record the fault, leave its loop, and the call return DSD_ERR_TIMEOUT.
 * Default 20000 ms.  Applies to calls started afterwards, process-wide. */
dsd_status dsd_set_wait_limit_ms(uint32_t ms);

/* Tuning: once at most `max_alive` vertices remain alive, the peeling kernel
 * keeps the alive list and the frontier in every block's shared memory and
 * needs one grid barrier per round (the tail of many tiny levels).  Default
 * 16384 (also capped by shared memory); 0 disables it.  Results do not
 * depend on it.  Process-wide; applies to calls started afterwards. */
dsd_status dsd_set_peel_small_limit(uint32_t max_alive);
/* Largest alive set whose remaining levels (h = 2, 3) are finished by one
 * thread-block cluster holding the alive subgraph as bitmap rows (in global
 * memory up to 16,384 vertices for h = 3, in the cluster's distributed shared
 * memory below about 4,600; the default is as large as those hold; 0 =
 * never).  Results do not depend on it.  Process-wide. */
dsd_status dsd_set_peel_tail_limit(uint32_t max_alive);
/* Where dsd_peel_app keeps each level's bucket queue (the bitmaps, one per
 * count below k + 1, over the level's positions): in a block's shared memory
 * when it fits `shared_words` 32-bit words (default and maximum 12,288), else
 * in global memory while the levels placed there total at most
 * `global_words` words (default 2^26), else only the buckets of the smallest
 * counts that fit shared memory, with a scan of the level behind them (0 and
 * 0: the scan alone).  Results do not depend on it.  Process-wide; applies
 * to calls started afterwards.  Never fails. */
dsd_status dsd_set_peel_app_queue(uint32_t shared_words, uint64_t global_words);
/* Work items of the peel for h >= 4 (the cliques through one frontier vertex
 * v whose smallest other member is w): a warp lists those of a candidate set
 * of at most `warp_max` vertices itself (2..32, default 4); sets of up to 32
 * go, with their candidates, to groups of 8 warps, at most `mid_max` per
 * round (default 2^20; 0: none); larger ones, and any beyond mid_max, to a
 * whole block.  Results do not depend on it.  Process-wide; applies to calls
 * started afterwards.  DSD_ERR_INVALID for warp_max outside 2..32. */
dsd_status dsd_set_peel_items(uint32_t warp_max, uint32_t mid_max);

/* Checked mode (off by default; process-wide, for calls started
 * afterwards).  Clique-degrees and mu are exact unsigned 64-bit integers;
 * no graph this library can hold reaches 2^64 h-cliques through a vertex in
 * practice, but in checked mode every addition into a per-vertex counter or
 * into mu also tests for wrap-around, and a wrapped counter makes the call
 * return DSD_ERR_OVERFLOW instead of a wrong count.  Costs a returned
 * atomic per addition. */
dsd_status dsd_set_checked(int on);
/* Self-test of that checked addition on the current device: starting from
 * `start`, adds addends[0..count) (host array, count <= 2^20) one by one
 * into a device counter exactly as the counting kernels do in checked mode;
 * *sum receives the (wrapped) result and *overflowed 1 if any addition
 * wrapped, else 0. */
dsd_status dsd_checked_add_selftest(uint64_t start, const uint64_t* addends, uint32_t count,
                                    uint64_t* sum, int* overflowed);

/* ---------------------------------------------------------------- graphs */

/* Build a graph from an edge list (Sec. 2 data model).  Edge i joins
 * src[i] and dst[i]; the list may hold self-loops, repeated pairs and both
 * orientations of a pair -- loops are dropped and each unordered pair is
 * kept once.  src/dst: m entries each, in host or device memory per `mem`.
 * `cuda_stream` is a cudaStream_t (NULL = the legacy default stream) on the
 * current CUDA device; the graph lives on that device.
 * Errors: DSD_ERR_INVALID if out == NULL, (m > 0 and src/dst NULL), or an
 * endpoint >= n; DSD_ERR_NOMEM; DSD_ERR_CUDA. */
dsd_status dsd_graph_from_edges(uint32_t n, uint64_t m, const uint32_t* src,
                                const uint32_t* dst, int mem, void* cuda_stream,
                                dsd_graph** out);

/* Build a graph from a CSR: off[n+1] (off[0] = 0, non-decreasing), adj[off[n]].
 * The CSR is cleaned exactly like an edge list (rows sorted, loops and
 * repeats dropped) and symmetrised: an entry v in row u makes u,v adjacent.
 * Errors: as dsd_graph_from_edges, plus DSD_ERR_INVALID for a malformed off[]. */
dsd_status dsd_graph_from_csr(uint32_t n, const uint64_t* off, const uint32_t* adj,
                              int mem, void* cuda_stream, dsd_graph** out);

/* Release a graph and all its device memory.  NULL is a no-op. */
void dsd_graph_destroy(dsd_graph* g);

/* n and the number m of undirected edges after cleaning.  Either pointer may
 * be NULL. */
dsd_status dsd_graph_info(const dsd_graph* g, uint32_t* n, uint64_t* m);

/* Change the stream later calls on g are ordered on. */
dsd_status dsd_graph_set_stream(dsd_graph* g, void* cuda_stream);

/* Copy out the cleaned symmetric CSR: off[n+1], adj[2m] (rows ascending). */
dsd_status dsd_graph_csr(dsd_graph* g, uint64_t* off, uint32_t* adj, int mem);

/* ------------------------------------------------- ordering (h = 2 core) */

/* Edge k-core numbers (Sec. 4.1, Def. 5) -- the (k,Psi)-core numbers for
 * h = 2 -- and the degeneracy rank used to orient edges for listing:
 * rank[v] in [0, n) orders vertices by (peeling round, id), where the
 * peeling round is the level-synchronous round in which v left.  Either
 * output may be NULL.  `degeneracy` (may be NULL) receives max core_2. */
dsd_status dsd_degeneracy_order(dsd_graph* g, uint32_t* core2, uint32_t* rank,
                                uint32_t* degeneracy, int mem);

/* ------------------------------------------------------ clique-degrees */

/* deg[v] = deg_G(v, Psi), the number of h-clique instances containing v
 * (Def. 3), for all n vertices; *mu = mu(G, Psi) (Def. 4).  deg: n entries
 * (may be NULL to get mu only); mu may be NULL.  Both live per `mem`.
 * Errors: DSD_ERR_INVALID (h); DSD_ERR_OVERFLOW in checked mode. */
dsd_status dsd_clique_degrees(dsd_graph* g, int h, uint64_t* deg, uint64_t* mu, int mem);

/* ------------------------------------------------- core decomposition */

/* core[v] = core_G(v, Psi) (Def. 6) for all n vertices, by level-synchronous
 * peeling (Algorithm 3 with every minimum-degree vertex removed at once);
 * *kmax = max core.  core (n entries) or kmax may be NULL.
 * A graph with no h-clique has core = 0 everywhere and kmax = 0. */
dsd_status dsd_core_decompose(dsd_graph* g, int h, uint64_t* core, uint64_t* kmax, int mem);

/* Nested level statistics of the last decomposition run on g with this h
 * (dsd_core_decompose or dsd_core_app): for each distinct core value k in
 * increasing order, level_k[j] = k, level_size[j] = |R_k| and
 * level_mu[j] = mu(R_k).  `cap` is the capacity of each array; *nlevels
 * receives the number of levels (DSD_ERR_OVERFLOW if it exceeds cap; the
 * first cap entries are still written).  Arrays may be NULL when cap = 0.
 * DSD_ERR_INVALID if no decomposition with this h has run on g. */
dsd_status dsd_level_stats(dsd_graph* g, int h, uint64_t* level_k, uint32_t* level_size,
                           uint64_t* level_mu, uint32_t cap, uint32_t* nlevels, int mem);

/* ------------------------------------------------------------- CoreApp */

typedef struct {
    uint64_t kmax;            /* maximum clique-core number k_max */
    uint32_t kmax_core_size;  /* |R_kmax| */
    uint32_t densest_size;    /* |S*| */
    uint64_t kmax_core_mu;    /* mu(R_kmax) */
    uint64_t best_k;          /* S* = R_best_k */
    uint64_t densest_mu;      /* mu(S*); rho(S*) = densest_mu / densest_size exactly */
    uint32_t nlevels;         /* number of distinct core values */
    int32_t seeded_accepted;  /* dsd_core_app_seeded: 1 if answered from the (seed_k,Psi)-core
                                 of the proposal, 0 if it fell back; 0 for every other call */
    uint64_t seed_k;          /* dsd_core_app_seeded: ceil(rho') of the proposal (0 when there
                                 was no usable proposal); 0 for every other call */
} dsd_core_app_result;

/* CoreApp / IncApp output (Algorithms 5 and 6, Lemma 6) plus Pruning1's
 * densest residual (Sec. 5.1):
 *   kmax_core: the vertices of the (k_max,Psi)-core, ascending;
 *   densest:   S* = R_k maximising rho(R_k) = mu(R_k)/|R_k| over the
 *              distinct levels k (ties: the largest k), ascending.
 * Each vertex array needs capacity n (may be NULL to skip it); r must not
 * be NULL.  With no h-clique: kmax = 0 and both sets are all of V, density
 * 0/n (the whole graph is the (0,Psi)-core, Example 3).  With n = 0 all
 * sizes are 0. */
dsd_status dsd_core_app(dsd_graph* g, int h, uint32_t* kmax_core, uint32_t* densest,
                        int mem, dsd_core_app_result* r);

/* ---------------------------------------------------- failure detection */

/* Runs the grid barrier of the peeling kernel (one block per SM, bounded
 * waits) on `cuda_stream`.  absent_block < 0: all blocks pass four barriers,
 * DSD_OK.  absent_block = b >= 0: block b leaves without arriving, every
 * other block's wait runs out after wait_ms (1..60000) and the call returns
 * DSD_ERR_TIMEOUT; the kernel ends and the context stays usable.  The same
 * limit (dsd_set_wait_limit_ms) turns a stalled peel into DSD_ERR_TIMEOUT. */
dsd_status dsd_check_barrier_timeout(int absent_block, uint32_t wait_ms, void* cuda_stream);

/* ------------------------------------------------------ learned proposal */

/* Not in the paper: a small network proposes rho', a lower bound of the
 * optimal h-clique density (Problem 1), from 64 statistics of the graph.
 * The seeded call then decomposes only the (ceil(rho'),Psi)-core (Lemma 5;
 * the clique-core bound of Sec. 5.2 limits it to an edge core) and falls
 * back to the full decomposition when the proposal fails an exact test, so
 * its outputs always equal dsd_core_app's.
 *
 * The network: 64 -> 256 -> 256 -> 256 -> 1, ReLU, BF16 weights with FP32
 * master copy and accumulation, output log(1 + rho').  Training minimises the
 * pinball (quantile) loss at quantile q with Adam (beta 0.9 / 0.999). */
typedef struct dsd_model dsd_model;
/* Number of parameters (148481). */
uint64_t dsd_model_param_count(void);
/* New model with deterministic He-uniform weights from `seed`. */
dsd_status dsd_model_create(uint64_t seed, void* cuda_stream, dsd_model** out);
void dsd_model_destroy(dsd_model* m);
/* Parameters, Adam first and second moments, then the step count:
 * state has 3 * count + 1 floats (host); count = dsd_model_param_count(). */
dsd_status dsd_model_get_state(dsd_model* m, float* state, uint64_t count);
dsd_status dsd_model_set_state(dsd_model* m, const float* state, uint64_t count);
/* Network outputs for B <= 1024 feature rows X [B x 64] (host) into out [B] (host). */
dsd_status dsd_model_forward(dsd_model* m, const float* X, uint32_t B, float* out);
/* Mean pinball loss at quantile q on labels y [B] and its gradient with
 * respect to the parameters (grad: count floats, host, may be NULL); no update. */
dsd_status dsd_model_gradient(dsd_model* m, const float* X, const float* y, uint32_t B,
                              float q, float* loss, float* grad);
/* One Adam step (learning rate lr) on a batch; *loss (host, may be NULL) is
 * the batch loss before the step. */
dsd_status dsd_model_train_step(dsd_model* m, const float* X, const float* y, uint32_t B,
                                float q, float lr, float* loss);
/* The 64 statistics of g used as network input for clique size h: sizes,
 * degree and edge-core histograms, and for three nested edge cores (all of
 * V, core number >= degeneracy/2, core number = degeneracy) their sizes and
 * clustering, triangle and h-clique estimates from neighbour pairs sampled
 * around 4096 hashed vertices each.  Deterministic.  f: 64 floats, host or
 * device memory as mem says. */
dsd_status dsd_graph_features(dsd_graph* g, int h, float* f, int mem);

typedef struct {
    float rho_prime;          /* the proposal */
    uint32_t accepted;        /* 1: answered from the (seed_k,Psi)-core */
    uint64_t seed_k;          /* ceil(rho') */
    uint64_t x0;              /* edge-core order the core was looked for in */
    uint32_t sub_n;           /* vertices of that edge core */
    uint32_t reserved;
    uint64_t sub_m;           /* its edges */
} dsd_seed_info;

/* dsd_core_app with a proposal from model m: identical outputs (kmax_core,
 * densest, r); r->nlevels counts the levels at or above seed_k when
 * accepted, r->seeded_accepted and r->seed_k say what the proposal did.
 * The model is only read. */
dsd_status dsd_core_app_seeded(dsd_graph* g, int h, const dsd_model* m, uint32_t* kmax_core,
                               uint32_t* densest, int mem, dsd_core_app_result* r);
/* The same, with the proposal's details in info (may be NULL). */
dsd_status dsd_core_app_seeded_info(dsd_graph* g, int h, const dsd_model* m,
                                    uint32_t* kmax_core, uint32_t* densest, int mem,
                                    dsd_core_app_result* r, dsd_seed_info* info);

/* ------------------------------------------------------------- PeelApp */

typedef struct {
    uint64_t mu;              /* h-cliques inside the returned set */
    uint32_t size;            /* its vertices; its density is mu / size exactly */
    uint32_t removed;         /* vertices removed when the set was met (n - size) */
    uint64_t level_k;         /* the (k,Psi)-core level the set was met in */
} dsd_peel_app_result;

/* PeelApp (Algorithm 2, Sec. 3.2): remove one vertex of minimum current
 * clique-degree at a time (ties: the smaller vertex id) and return the
 * densest of the sets met -- G and every residual -- where a later set
 * replaces the best only when strictly denser.  Its guarantee is Lemma 2
 * (density >= rho_opt / h).  The removal order passes through every
 * (k,Psi)-core R_k and removes R_k \ R_{k+1} while in it, so after one
 * decomposition every level is peeled independently on the GPU.
 *   densest (capacity n, may be NULL): the returned set, ascending;
 *   order (capacity n, may be NULL): the removal order, order[i] = the
 *       vertex removed at step i;
 *   both host or device memory per mem; res must not be NULL.
 * Candidate sets of more than 1024 vertices (degeneracy above 1024, h >= 4)
 * are split by their next member, as in the decomposition.
 * With n = 0 all fields are 0.  Errors: DSD_ERR_INVALID; DSD_ERR_NOMEM;
 * DSD_ERR_TIMEOUT (the decomposition's wait limit); DSD_ERR_CUDA. */
dsd_status dsd_peel_app(dsd_graph* g, int h, uint32_t* densest, uint32_t* order, int mem,
                        dsd_peel_app_result* res);

/* ---------------------------------------------- CoreApp's top-down schedule */

typedef struct {
    uint32_t passes;          /* windows decomposed */
    uint32_t sub_n;           /* vertices of the last window */
    uint64_t x;               /* its edge-core order: the window is {core_2 >= x} */
    uint64_t gamma_out;       /* the largest C(core_2, h-1) outside it */
    uint64_t sub_m;           /* its edges */
} dsd_topdown_info;

/* dsd_core_app through CoreApp's own schedule (Algorithm 6, Sec. 5.2):
 * windows of the vertices with the largest bound gamma(v) = C(core_2(v), h-1)
 * (edge cores, at least 1024 vertices, doubling), each peeled from level
 * K = gamma_out + 1 (gamma_out: the largest gamma outside the window; one
 * cascade prunes to R_K), until the window's k_max is >= K and its densest
 * level at or above K has density >= K - 1 (then no level below K is
 * denser).  Outputs identical to dsd_core_app; r->nlevels counts
 * the levels at or above K.  info (may be NULL) describes the schedule. */
dsd_status dsd_core_app_topdown(dsd_graph* g, int h, uint32_t* kmax_core, uint32_t* densest,
                                int mem, dsd_core_app_result* r, dsd_topdown_info* info);

/* ------------------------------------------------------------ CoreExact */

typedef struct {
    uint64_t mu;              /* h-cliques inside the CDS */
    uint32_t size;            /* |CDS|; rho_opt = mu / size exactly */
    uint32_t cuts;            /* minimum cuts solved */
    uint64_t k1;              /* Pruning1: ceil(rho') of the densest level */
    uint64_t k2;              /* Pruning2: ceil of the starting lower bound */
    uint64_t lower_mu;        /* the lower bound the search started from, */
    uint32_t lower_size;      /*   lower_mu / lower_size */
    uint32_t components;      /* connected components of the (k1,Psi)-core */
    uint32_t net_nodes;       /* the first (largest) flow network: nodes */
    uint32_t reserved;
    uint64_t net_arcs;        /*   and arcs, residual twins included */
    uint64_t rounds;          /* push/relabel rounds, all cuts */
    uint64_t relabels;        /* global relabels (searches back from t), all cuts */
    uint64_t locate_ns;       /* host wall time: decomposition lookup, Pruning2 */
    uint64_t build_ns;        /*   located cores and their networks */
    uint64_t cut_ns;          /*   minimum cuts */
    uint64_t verify_ns;       /*   recount of the answer and its output */
} dsd_exact_info;

/* CoreExact (Algorithm 4, Sec. 4.3): the h-clique densest subgraph (CDS,
 * Problem 1) exactly.  Pruning1 locates it in the (ceil(rho'),Psi)-core
 * (rho': density of the densest level, Sec. 4.3 lemma on the CDS's core);
 * Pruning2 raises the lower bound to the densest connected component of
 * that core; then minimum cuts of Algorithm 1's network (built from the
 * (h-1)-cliques of the located core, which shrinks as the bound rises) and
 * Dinkelbach's iteration on exact rationals reach rho_opt.
 *   cds (capacity n, may be NULL): the largest densest vertex set -- the
 *       union of all vertex sets of density rho_opt, itself of that density
 *       -- ascending, host or device memory per mem.
 *   info (not NULL): info->mu / info->size = rho_opt, plus search statistics.
 * With no h-clique every set has density 0 and the answer is V (0 / n).
 * Runs (or reuses) the decomposition behind dsd_core_decompose for this h.
 * Errors: DSD_ERR_INVALID; DSD_ERR_NOMEM; DSD_ERR_UNSUPPORTED (a network
 * of 2^31 nodes or more); DSD_ERR_OVERFLOW (scaled capacities reach 2^61);
 * DSD_ERR_TIMEOUT (a cut ran past 4N + 100000 push/relabel rounds or the
 * wait limit of dsd_set_wait_limit_ms); DSD_ERR_INTERNAL (a self-check of
 * the network or of the cut failed); DSD_ERR_CUDA. */
dsd_status dsd_core_exact(dsd_graph* g, int h, uint32_t* cds, int mem, dsd_exact_info* info);

/* ---------------------------------------------------- pattern densities */

/* Sec. 6 generalises the h-clique to a pattern Psi: an instance is a copy of
 * the pattern in G (pattern edges on graph edges, not necessarily induced),
 * deg(v, Psi) the instances holding v, mu(G, Psi) the number of instances,
 * and the (k,Psi)-cores, core numbers and CoreApp outputs follow as for
 * cliques.  Two patterns, with the closed forms of the appendix on special
 * patterns:
 *   DSD_PATTERN_STAR,  x = 2..8: the x-star (a centre and x leaves);
 *     deg(v) = C(d(v), x) + sum over neighbours u of C(d(u) - 1, x - 1);
 *   DSD_PATTERN_LOOP4 (x ignored): the 4-vertex loop (4-cycle);
 *     deg(v) = sum over w != v of C(c(v, w), 2), c = common neighbours.
 * Counts are 64-bit (binomials wrap beyond 2^64, as in any 64-bit count).
 * Errors: DSD_ERR_INVALID (NULL handle, unknown pattern, x out of range,
 * bad mem), DSD_ERR_NOMEM, DSD_ERR_TIMEOUT (a grid-barrier wait of the
 * peel ran past the limit of dsd_set_wait_limit_ms), DSD_ERR_CUDA. */
#define DSD_PATTERN_STAR 1
#define DSD_PATTERN_LOOP4 2

/* deg (n entries, may be NULL) and *mu (may be NULL), host or device per mem. */
dsd_status dsd_pattern_degrees(dsd_graph* g, int pattern, int x, uint64_t* deg, uint64_t* mu,
                               int mem);

/* (k,Psi)-core numbers (core, n entries, may be NULL), *kmax (may be NULL),
 * and the level records: for each distinct core value k ascending, |R_k|
 * and mu(R_k, Psi) (arrays of capacity cap, may be NULL; *nlevels = the
 * count, DSD_ERR_OVERFLOW when it exceeds cap, the first cap still written).
 * Level-synchronous peeling: every alive vertex of pattern-degree <= k
 * leaves at level k, k = max(k, least alive pattern-degree). */
dsd_status dsd_pattern_core_decompose(dsd_graph* g, int pattern, int x, uint64_t* core,
                                      uint64_t* kmax, uint64_t* level_k, uint32_t* level_size,
                                      uint64_t* level_mu, uint32_t cap, uint32_t* nlevels,
                                      int mem);

/* CoreApp's outputs for the pattern (the fields of dsd_core_app_result; mu
 * counts pattern instances): the (k_max,Psi)-core and the densest level set
 * (ties: the larger k), each ascending, capacity n, may be NULL. */
dsd_status dsd_pattern_core_app(dsd_graph* g, int pattern, int x, uint32_t* kmax_core,
                                uint32_t* densest, int mem, dsd_core_app_result* r);

/* ------------------------------------------------------------- batches */

/* Many small graphs in one launch.  The paper treats one graph at a time;
 * this runs the same path as dsd_graph_from_edges + dsd_core_app (CSR build,
 * degeneracy peel, h-clique clique-degrees, (k,Psi)-core peel, CoreApp
 * outputs) for every graph of a batch in one persistent kernel whose CTAs
 * take graphs from a work queue (largest first), each graph handled by one
 * CTA.  The launch is captured once in a CUDA graph and replayed by
 * dsd_batch_replay.
 *   count graphs; graph i has n[i] vertices (<= 65535), clique size h[i]
 *   (2..4) and m[i] edges: src/dst[e_i .. e_i + m[i]) with e_i the sum of
 *   the earlier m (same clean-up rules as dsd_graph_from_edges).
 *   mem: where src/dst live (copied at creation; the caller may free them).
 *   want_cores != 0 keeps every graph's core numbers for dsd_batch_results.
 *   autotune_cache: text file (may be NULL) remembering the launch shape
 *   chosen for a batch signature; without an entry, creation times shapes on
 *   the batch itself: threads per CTA x CTAs per SM, then the intersection
 *   tile (lanes per row scan) at the best of those.
 * Errors: DSD_ERR_INVALID, DSD_ERR_UNSUPPORTED (n, h or m out of range),
 * DSD_ERR_NOMEM, DSD_ERR_CUDA. */
typedef struct dsd_batch dsd_batch;
dsd_status dsd_batch_create(uint32_t count, const uint32_t* n, const int* h, const uint64_t* m,
                            const uint32_t* src, const uint32_t* dst, int mem, int want_cores,
                            void* cuda_stream, const char* autotune_cache, dsd_batch** out);
/* Run the whole batch once (one graph replay; asynchronous on the stream). */
dsd_status dsd_batch_replay(dsd_batch* b);
/* Results of the last run (synchronises the stream).  res: count entries
 * (the fields of dsd_core_app_result; kmax_core/densest sets are not kept);
 * status: count entries, 0 ok, 1 invalid graph (an endpoint >= n); cores:
 * sum of n[i] entries in graph order, or NULL (needs want_cores).  Any
 * pointer may be NULL.  Graphs beyond the batch kernel's limits (h = 4 with
 * more than 512 higher-ranked neighbours at a vertex) are answered by the
 * single-graph path, from the batch's device edge lists, at the first call
 * after a run (their results are kept for later calls). */
dsd_status dsd_batch_results(dsd_batch* b, dsd_core_app_result* res, int* status, uint64_t* cores);
/* Chosen launch shape -- threads per CTA, CTAs per SM, and the intersection
 * tile: lanes that scan one row (32, 16 or 8; a warp scans 32 / lanes rows
 * at once in the triangle listing and the h = 4 edge counts) -- and its
 * timed duration (ms, 0 if read from the cache or set).  Any pointer may be
 * NULL. */
dsd_status dsd_batch_info(const dsd_batch* b, uint32_t* threads, uint32_t* ctas_per_sm,
                          uint32_t* lanes_per_row, float* tuned_ms);
/* Replace the tuned shape (threads 256/512/1024, ctas_per_sm 1 or 2,
 * lanes_per_row 8/16/32) and capture the launch again; results do not depend
 * on it.  DSD_ERR_UNSUPPORTED if the shape does not fit on an SM. */
dsd_status dsd_batch_set_shape(dsd_batch* b, uint32_t threads, uint32_t ctas_per_sm,
                               uint32_t lanes_per_row);
void dsd_batch_destroy(dsd_batch* b);

/* CoreApp outputs (no vertex sets) for `count` existing graph handles in one
 * call: rs[i] gets what dsd_core_app(gs[i], hs[i], ...) returns, and
 * cores[i] (host memory, n_i entries; cores or cores[i] may be NULL) the
 * core numbers of dsd_core_decompose.  Graphs within the batch kernel's
 * limits (n <= 65535, 2 <= h <= 4) run together in one persistent launch,
 * built from the handles' cleaned CSRs (a batch created, replayed once and
 * destroyed, on the first handle's stream; the launch shape comes from
 * autotune_cache, which may be NULL, or is timed); every other graph -- and
 * any the batch kernel reports unsupported -- runs through the single-graph
 * path on its own stream.  Returns after every result is in host memory.
 * All handles must live on the current device.
 * Errors: DSD_ERR_INVALID (count < 0, NULL arrays, a NULL handle, h out of
 * range), and those of the calls above. */
dsd_status dsd_batch_run(int count, dsd_graph* const* gs, const int* hs,
                         dsd_core_app_result* rs, uint64_t* const* cores,
                         const char* autotune_cache);

/* ------------------------------------------------ allocation-free variant */

/* The paper has no counterpart to this call; it exists for callers that
 * cannot allocate device memory (a host framework whose allocator already
 * holds the device's memory, or a serving path that may not allocate in the
 * middle of a request).  It computes what dsd_clique_degrees computes for
 * h = 3 (triangle clique-degrees deg[v] and mu), directly from a caller CSR,
 * without a graph handle and without allocating anything.
 *   off: device pointer, n+1 entries; adj: device pointer, off[n] entries
 *        (may be NULL when off[n] = 0; the call then reads off[n] back and
 *        synchronises the stream to check it).  The CSR must already be
 *        symmetric with ascending, duplicate-free rows and no self-loops
 *        (e.g. the output of dsd_graph_csr).
 *   deg: device pointer, n entries (written); mu: device pointer (written).
 *   cuda_stream: the stream the work is ordered on (NULL = legacy stream).
 * Its scratch is a fixed 4 MiB __device__ array that every GPU which loads
 * the library keeps until the process exits; n must not exceed 1,048,512
 * (DSD_ERR_UNSUPPORTED otherwise).  The first call on a device looks up that
 * array's address and caches it; since CUDA may load the library's device
 * code lazily, that first call may also be what makes the driver reserve
 * the array.  Make one warm-up call per device before any stretch of work
 * that must not allocate, and before any stream capture begins.
 * All calls on a device share the array, so calls that overlap on the GPU
 * (other streams, other threads) race: serialise them.  Returns once the
 * work is queued; synchronise the stream before reading deg and mu. */
dsd_status dsd_triangle_degrees_noalloc(uint32_t n, const uint64_t* off, const uint32_t* adj,
                                        uint64_t* deg, uint64_t* mu, void* cuda_stream);

/* ---------------------------------------------------------- profiling */

/* Per-phase device timings (CUDA events on the graph's stream) of the most
 * recent calls on g.  Enable with dsd_set_profiling(g, 1).  Phases:
 *   0 csr build, 1 degeneracy peel (h = 2), 2 orientation, 3 clique count,
 *   4 (k,Psi) peel, 5 output extraction.
 * ms[p] is the time of the last run of phase p; bytes[p] the algorithmic
 * bytes that run moved (model in the project documentation; 0 if none);
 * launches[p] the number of kernels it launched. */
#define DSD_NPHASES 6
dsd_status dsd_set_profiling(dsd_graph* g, int on);
dsd_status dsd_phase_stats(dsd_graph* g, float* ms, uint64_t* bytes, uint32_t* launches);

/* Algorithmic bytes of one h-clique listing of g (any h >= 3; the global
 * reads do not depend on h, deeper levels stay in shared memory):
 *   staged: the listing kernels' own model -- offsets and N+(u) read once
 *           per vertex, N+(x) once per oriented edge (u, x), an 8-byte
 *           read-modify-write per counter that can be credited, deg zeroed;
 *   merge:  a sorted-list merge intersection's -- 4 (d+(u) + d+(x)) per
 *           oriented edge, 8 (n+1) offsets, 4 m entries, 8 n counters.
 * Either pointer may be NULL (host memory).  Runs the degeneracy order if
 * it has not run yet. */
dsd_status dsd_listing_bytes(dsd_graph* g, uint64_t* staged, uint64_t* merge);

/* Counters of the last peeling run: which = 0 the degeneracy (h = 2) peel,
 * 1 the last (k,Psi) peel with h >= 3.  out[DSD_PEEL_STATS] receives:
 * rounds, levels, frontier work items, metered algorithmic bytes, time block 0
 * spent inside grid barriers (ns), barriers passed, row compactions, block
 * size, grid size, k_max, first round run with the alive set replicated in
 * every block's shared memory (0 if none), then block 0's time (ns) in each
 * phase outside barriers: [large regime] retire/mark, alive-list scan, level
 * jump, clique enumeration; [small regime] retire/copy, level jump,
 * mark/bitmaps, clique enumeration; then the alive vertices handed to the
 * cluster tail kernel (0 if none), the round of the hand-over, the tail
 * kernel's time (ns) and its lead CTA's time (ns) in: building the rows,
 * frontier broadcast, level jumps and frontier lists, candidate numbering,
 * candidate work, the barrier after it, retiring.  Zeros if that peel has
 * not run. */
#define DSD_PEEL_STATS 29
dsd_status dsd_peel_stats(dsd_graph* g, int which, uint64_t* out);

#ifdef __cplusplus
}
#endif
#endif /* DSD_H */
