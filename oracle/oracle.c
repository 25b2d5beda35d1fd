/*
 * Plain CPU oracle for h-clique clique-degrees, (k,Psi)-core decomposition
 * and the CoreApp outputs (Fang et al., "Efficient Algorithms for Densest
 * Subgraph Discovery", PVLDB 12(11), 2019).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark load this file.  It shares no code, header,
 * table or helper with the CUDA library; it is deliberately slow and
 * written to be checked against the paper by eye.
 *
 * Every function is single-threaded, uses plain C arrays and 64-bit
 * unsigned counters, and returns 0 on success or a negative error code.
 *
 *   orc_build_csr            Sec. 2 "Data model": undirected, simple graph.
 *   orc_clique_degrees       Def. 2 (clique instance), Def. 3 (clique-degree),
 *                            Def. 4 (mu = number of instances).
 *   orc_vertex_clique_degree Def. 3 for one vertex (orc_vertex_clique_degrees:
 *                            for many, sharing one listing order).
 *   orc_core_decompose       Algorithm 3 ((k,Psi)-core decomposition), in the
 *                            paper's steps: take a minimum clique-degree
 *                            vertex v, record core[v] = deg[v], and for each
 *                            clique instance containing v decrease every other
 *                            member u whose clique-degree exceeds deg[v].
 *   orc_threshold_prune      Def. 6 read directly: the (k,Psi)-core as what is
 *                            left after repeatedly deleting every vertex with
 *                            fewer than k clique instances (Sec. 4.3, opening
 *                            paragraph).
 *   orc_induced_clique_count mu(G[S]) for a vertex subset S (Def. 4).
 *   orc_level_stats          For every distinct core value k: |R_k| and
 *                            mu(R_k), with R_k = {v : core(v) >= k} (Def. 6,
 *                            nestedness); one clique lies in R_k exactly when
 *                            its smallest member core number is >= k.
 *   orc_exact_cds            Algorithm 1 (Exact, Sec. 3.1): binary search on
 *                            alpha over [0, max clique-degree] with one
 *                            minimum st-cut of the (h-1)-clique flow network
 *                            per guess, stopping once u - l < 1/(n(n-1));
 *                            then the largest densest vertex set.
 *
 * Clique instances are unordered vertex sets (Def. 2 and the remark after
 * Def. 3).  Each set is listed exactly once as the increasing sequence
 * v1 < v2 < ... < vh under one fixed total order of V; the oracle uses the
 * order (degree, id), which only changes how long the listing takes.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_EINVAL (-1)
#define ORC_ENOMEM (-2)

/* ---------------------------------------------------------------- CSR --- */

static int cmp_u32(const void* a, const void* b) {
    uint32_t x = *(const uint32_t*)a, y = *(const uint32_t*)b;
    return (x > y) - (x < y);
}

/* Symmetric, sorted, duplicate-free CSR without self-loops.
 * off: n+1 entries; adj: capacity 2*m.  Returns the number of adjacency
 * entries written (2 * number of undirected edges) or a negative code. */
int64_t orc_build_csr(uint32_t n, uint64_t m, const uint32_t* src,
                      const uint32_t* dst, uint64_t* off, uint32_t* adj) {
    uint64_t* cnt = (uint64_t*)calloc((size_t)n + 1, sizeof(uint64_t));
    if (!cnt) return ORC_ENOMEM;
    for (uint64_t i = 0; i < m; i++) {
        if (src[i] >= n || dst[i] >= n) { free(cnt); return ORC_EINVAL; }
        if (src[i] == dst[i]) continue;
        cnt[src[i]]++;
        cnt[dst[i]]++;
    }
    uint64_t* pos = (uint64_t*)malloc(((size_t)n + 1) * sizeof(uint64_t));
    uint64_t* cur = (uint64_t*)malloc(((size_t)n + 1) * sizeof(uint64_t));
    uint64_t tot = 0;
    for (uint32_t v = 0; v < n; v++) tot += cnt[v];
    uint32_t* tmp = (uint32_t*)malloc((size_t)(tot ? tot : 1) * sizeof(uint32_t));
    if (!pos || !cur || !tmp) { free(cnt); free(pos); free(cur); free(tmp); return ORC_ENOMEM; }
    pos[0] = 0;
    for (uint32_t v = 0; v < n; v++) pos[v + 1] = pos[v] + cnt[v];
    memcpy(cur, pos, ((size_t)n + 1) * sizeof(uint64_t));
    for (uint64_t i = 0; i < m; i++) {
        uint32_t u = src[i], v = dst[i];
        if (u == v) continue;
        tmp[cur[u]++] = v;
        tmp[cur[v]++] = u;
    }
    uint64_t k = 0;
    off[0] = 0;
    for (uint32_t v = 0; v < n; v++) {
        uint32_t* row = tmp + pos[v];
        uint64_t len = pos[v + 1] - pos[v];
        qsort(row, (size_t)len, sizeof(uint32_t), cmp_u32);
        for (uint64_t j = 0; j < len; j++)
            if (j == 0 || row[j] != row[j - 1]) adj[k++] = row[j];
        off[v + 1] = k;
    }
    free(cnt); free(pos); free(cur); free(tmp);
    return (int64_t)k;
}

/* ------------------------------------------- relabelled working graph --- */

/* The working graph: vertices renamed so that new id order = (degree, id)
 * order; rows sorted by new id.  old_of[new] and new_of[old] map back. */
typedef struct {
    uint32_t n;
    uint64_t* off;
    uint32_t* adj;
    uint32_t* old_of;
    uint32_t* new_of;
    uint32_t maxdeg;
} wgraph;

static const uint64_t* g_sort_deg_off;
static int cmp_by_deg_id(const void* a, const void* b) {
    uint32_t x = *(const uint32_t*)a, y = *(const uint32_t*)b;
    uint64_t dx = g_sort_deg_off[x + 1] - g_sort_deg_off[x];
    uint64_t dy = g_sort_deg_off[y + 1] - g_sort_deg_off[y];
    if (dx != dy) return (dx > dy) - (dx < dy);
    return (x > y) - (x < y);
}

static void wg_free(wgraph* w) {
    free(w->off); free(w->adj); free(w->old_of); free(w->new_of);
    memset(w, 0, sizeof(*w));
}

static int wg_make(uint32_t n, const uint64_t* off, const uint32_t* adj, wgraph* w) {
    memset(w, 0, sizeof(*w));
    w->n = n;
    uint64_t tot = off[n];
    w->off = (uint64_t*)malloc(((size_t)n + 1) * sizeof(uint64_t));
    w->adj = (uint32_t*)malloc((size_t)(tot ? tot : 1) * sizeof(uint32_t));
    w->old_of = (uint32_t*)malloc((size_t)(n ? n : 1) * sizeof(uint32_t));
    w->new_of = (uint32_t*)malloc((size_t)(n ? n : 1) * sizeof(uint32_t));
    if (!w->off || !w->adj || !w->old_of || !w->new_of) { wg_free(w); return ORC_ENOMEM; }
    for (uint32_t v = 0; v < n; v++) w->old_of[v] = v;
    g_sort_deg_off = off;
    qsort(w->old_of, n, sizeof(uint32_t), cmp_by_deg_id);
    for (uint32_t i = 0; i < n; i++) w->new_of[w->old_of[i]] = i;
    w->off[0] = 0;
    uint32_t md = 0;
    for (uint32_t i = 0; i < n; i++) {
        uint32_t o = w->old_of[i];
        uint64_t b = off[o], e = off[o + 1];
        uint64_t base = w->off[i];
        for (uint64_t j = b; j < e; j++) w->adj[base + (j - b)] = w->new_of[adj[j]];
        qsort(w->adj + base, (size_t)(e - b), sizeof(uint32_t), cmp_u32);
        w->off[i + 1] = base + (e - b);
        if (e - b > md) md = (uint32_t)(e - b);
    }
    w->maxdeg = md;
    return ORC_OK;
}

/* ------------------------------------------------ sorted-set helpers --- */

static int bsearch_u32(const uint32_t* a, uint64_t len, uint32_t x) {
    uint64_t lo = 0, hi = len;
    while (lo < hi) {
        uint64_t mid = lo + (hi - lo) / 2;
        if (a[mid] < x) lo = mid + 1; else hi = mid;
    }
    return lo < len && a[lo] == x;
}

/* out = a intersect b (both sorted ascending); returns its size.  Iterates
 * the shorter list and binary-searches the longer one. */
static uint32_t intersect(const uint32_t* a, uint64_t na, const uint32_t* b,
                          uint64_t nb, uint32_t* out) {
    uint32_t k = 0;
    if (na <= nb) {
        for (uint64_t i = 0; i < na; i++) if (bsearch_u32(b, nb, a[i])) out[k++] = a[i];
    } else {
        for (uint64_t i = 0; i < nb; i++) if (bsearch_u32(a, na, b[i])) out[k++] = b[i];
    }
    return k;
}

/* Indexed binary min-heap over vertices keyed by (deg, tie), where tie is
 * the vertex's original id (tie_order 0) or its complement (tie_order 1):
 * the "sort"/"resort" steps of Algorithm 3 (the paper uses a bin-sort; any
 * structure that yields a minimum clique-degree vertex computes the same
 * core numbers). */
typedef struct {
    uint32_t* heap;
    uint32_t* pos;
    uint32_t size;
    const uint64_t* key;
    const uint32_t* tie;
} vheap;

static int vh_less(const vheap* H, uint32_t a, uint32_t b) {
    if (H->key[a] != H->key[b]) return H->key[a] < H->key[b];
    return H->tie[a] < H->tie[b];
}
static void vh_swap(vheap* H, uint32_t i, uint32_t j) {
    uint32_t a = H->heap[i], b = H->heap[j];
    H->heap[i] = b; H->heap[j] = a;
    H->pos[b] = i; H->pos[a] = j;
}
static void vh_up(vheap* H, uint32_t i) {
    while (i > 0) {
        uint32_t p = (i - 1) / 2;
        if (!vh_less(H, H->heap[i], H->heap[p])) break;
        vh_swap(H, i, p);
        i = p;
    }
}
static void vh_down(vheap* H, uint32_t i) {
    for (;;) {
        uint32_t l = 2 * i + 1, r = l + 1, s = i;
        if (l < H->size && vh_less(H, H->heap[l], H->heap[s])) s = l;
        if (r < H->size && vh_less(H, H->heap[r], H->heap[s])) s = r;
        if (s == i) break;
        vh_swap(H, i, s);
        i = s;
    }
}
static uint32_t vh_pop(vheap* H) {
    uint32_t top = H->heap[0];
    H->size--;
    if (H->size) {
        H->heap[0] = H->heap[H->size];
        H->pos[H->heap[0]] = 0;
        vh_down(H, 0);
    }
    H->pos[top] = UINT32_MAX;
    return top;
}

/* --------------------------------------------------- clique listing --- */

/* A visitor receives every clique instance (as h new ids) once. */
typedef struct lister lister;
typedef void (*visit_fn)(lister* L, const uint32_t* clique);

struct lister {
    const wgraph* g;
    int h;
    uint32_t* tuple;     /* h entries */
    uint32_t** cand;     /* h candidate buffers, each maxdeg+1 */
    visit_fn visit;
    /* visitor state */
    uint64_t* deg;       /* per new id */
    uint64_t mu;
    vheap* heap;         /* peeling: bucket structure of Algorithm 3 */
    const uint64_t* core;     /* level stats: core per new id */
    const uint64_t* levels;   /* sorted distinct core values */
    uint32_t nlevels;
    uint64_t* level_hist;
    uint64_t kthr;       /* threshold prune */
    uint8_t* queued;
    uint32_t* queue;
    uint64_t qtail;
    const uint8_t* mask;      /* count inside a vertex subset (new ids) */
    uint32_t* store;          /* collected tuples, h entries each */
    uint64_t nstore, capstore;
    int overflow;
};

/* tuple[0..depth-1] is a clique; cand (sorted, ncand entries) holds every
 * vertex after tuple[depth-1] adjacent to all of tuple[0..depth-1]. */
static void extend(lister* L, int depth, const uint32_t* cand, uint32_t ncand) {
    const wgraph* g = L->g;
    for (uint32_t i = 0; i < ncand; i++) {
        uint32_t x = cand[i];
        L->tuple[depth] = x;
        if (depth + 1 == L->h) {
            L->visit(L, L->tuple);
        } else {
            uint32_t* nxt = L->cand[depth + 1];
            uint32_t nn = intersect(cand + i + 1, ncand - i - 1,
                                    g->adj + g->off[x], g->off[x + 1] - g->off[x], nxt);
            if (nn + depth + 1 >= (uint32_t)L->h) extend(L, depth + 1, nxt, nn);
        }
    }
}

static int lister_init(lister* L, const wgraph* g, int h, visit_fn f) {
    memset(L, 0, sizeof(*L));
    L->g = g; L->h = h; L->visit = f;
    L->tuple = (uint32_t*)calloc((size_t)h + 1, sizeof(uint32_t));
    L->cand = (uint32_t**)calloc((size_t)h + 1, sizeof(uint32_t*));
    if (!L->tuple || !L->cand) return ORC_ENOMEM;
    for (int i = 0; i <= h; i++) {
        L->cand[i] = (uint32_t*)malloc(((size_t)g->maxdeg + 1) * sizeof(uint32_t));
        if (!L->cand[i]) return ORC_ENOMEM;
    }
    return ORC_OK;
}

static void lister_free(lister* L) {
    if (L->cand) for (int i = 0; i <= L->h; i++) free(L->cand[i]);
    free(L->cand); free(L->tuple);
}

/* Every h-clique of the whole graph, once (v1 < ... < vh in new ids). */
static void list_all(lister* L) {
    const wgraph* g = L->g;
    for (uint32_t v = 0; v < g->n; v++) {
        L->tuple[0] = v;
        const uint32_t* row = g->adj + g->off[v];
        uint64_t len = g->off[v + 1] - g->off[v];
        uint64_t j = 0;
        while (j < len && row[j] <= v) j++;        /* later neighbours only */
        if (L->h == 1) { L->visit(L, L->tuple); continue; }
        extend(L, 1, row + j, (uint32_t)(len - j));
    }
}

/* Every h-clique that contains v, among vertices with alive[] != 0 (v is
 * taken as alive): v plus an (h-1)-clique of the alive neighbours of v.
 * The visitor sees the clique with v in slot 0. */
static void list_containing(lister* L, uint32_t v, const uint8_t* alive) {
    const wgraph* g = L->g;
    uint32_t* c0 = L->cand[L->h];   /* spare buffer */
    uint32_t k = 0;
    for (uint64_t j = g->off[v]; j < g->off[v + 1]; j++) {
        uint32_t u = g->adj[j];
        if (!alive || alive[u]) c0[k++] = u;
    }
    L->tuple[0] = v;
    if (L->h == 1) { L->visit(L, L->tuple); return; }
    extend(L, 1, c0, k);
}

/* ----------------------------------------------------- Def. 3 / Def. 4 -- */

static void visit_count(lister* L, const uint32_t* c) {
    L->mu++;
    for (int i = 0; i < L->h; i++) L->deg[c[i]]++;
}

static int check_h(int h) { return (h >= 2 && h <= 16) ? ORC_OK : ORC_EINVAL; }

/* deg[v] = number of h-clique instances containing v (original ids);
 * *mu = number of h-clique instances. */
int orc_clique_degrees(uint32_t n, const uint64_t* off, const uint32_t* adj,
                       int h, uint64_t* deg, uint64_t* mu) {
    if (check_h(h)) return ORC_EINVAL;
    wgraph g;
    if (wg_make(n, off, adj, &g)) return ORC_ENOMEM;
    lister L;
    if (lister_init(&L, &g, h, visit_count)) { lister_free(&L); wg_free(&g); return ORC_ENOMEM; }
    L.deg = (uint64_t*)calloc((size_t)(n ? n : 1), sizeof(uint64_t));
    if (!L.deg) { lister_free(&L); wg_free(&g); return ORC_ENOMEM; }
    list_all(&L);
    for (uint32_t i = 0; i < n; i++) deg[g.old_of[i]] = L.deg[i];
    *mu = L.mu;
    free(L.deg); lister_free(&L); wg_free(&g);
    return ORC_OK;
}

/* deg(v, Psi) for one vertex v: the (h-1)-cliques among the neighbours. */
int orc_vertex_clique_degree(uint32_t n, const uint64_t* off, const uint32_t* adj,
                             int h, uint32_t v, uint64_t* out) {
    if (check_h(h) || v >= n) return ORC_EINVAL;
    wgraph g;
    if (wg_make(n, off, adj, &g)) return ORC_ENOMEM;
    lister L;
    if (lister_init(&L, &g, h, visit_count)) { lister_free(&L); wg_free(&g); return ORC_ENOMEM; }
    L.deg = (uint64_t*)calloc((size_t)n, sizeof(uint64_t));
    if (!L.deg) { lister_free(&L); wg_free(&g); return ORC_ENOMEM; }
    list_containing(&L, g.new_of[v], NULL);
    *out = L.mu;
    free(L.deg); lister_free(&L); wg_free(&g);
    return ORC_OK;
}

/* Def. 3 for each of count vertices vs[i] into out[i], with the listing
 * order built once (the same listing as orc_vertex_clique_degree). */
int orc_vertex_clique_degrees(uint32_t n, const uint64_t* off, const uint32_t* adj,
                              int h, const uint32_t* vs, uint32_t count, uint64_t* out) {
    if (check_h(h)) return ORC_EINVAL;
    for (uint32_t i = 0; i < count; i++)
        if (vs[i] >= n) return ORC_EINVAL;
    wgraph g;
    if (wg_make(n, off, adj, &g)) return ORC_ENOMEM;
    lister L;
    if (lister_init(&L, &g, h, visit_count)) { lister_free(&L); wg_free(&g); return ORC_ENOMEM; }
    L.deg = (uint64_t*)calloc((size_t)n, sizeof(uint64_t));
    if (!L.deg) { lister_free(&L); wg_free(&g); return ORC_ENOMEM; }
    for (uint32_t i = 0; i < count; i++) {
        L.mu = 0;
        list_containing(&L, g.new_of[vs[i]], NULL);
        out[i] = L.mu;
    }
    free(L.deg); lister_free(&L); wg_free(&g);
    return ORC_OK;
}

/* mu(G[S]) with S = {v : mask[v] != 0}. */
int orc_induced_clique_count(uint32_t n, const uint64_t* off, const uint32_t* adj,
                             int h, const uint8_t* mask, uint64_t* mu) {
    if (check_h(h)) return ORC_EINVAL;
    /* Build G[S] as a CSR on the original ids (rows of vertices outside S
     * are empty) and count its cliques. */
    uint64_t* o2 = (uint64_t*)malloc(((size_t)n + 1) * sizeof(uint64_t));
    uint32_t* a2 = (uint32_t*)malloc((size_t)(off[n] ? off[n] : 1) * sizeof(uint32_t));
    uint64_t* d2 = (uint64_t*)malloc((size_t)(n ? n : 1) * sizeof(uint64_t));
    if (!o2 || !a2 || !d2) { free(o2); free(a2); free(d2); return ORC_ENOMEM; }
    uint64_t k = 0;
    o2[0] = 0;
    for (uint32_t v = 0; v < n; v++) {
        if (mask[v])
            for (uint64_t j = off[v]; j < off[v + 1]; j++)
                if (mask[adj[j]]) a2[k++] = adj[j];
        o2[v + 1] = k;
    }
    int rc = orc_clique_degrees(n, o2, a2, h, d2, mu);
    free(o2); free(a2); free(d2);
    return rc;
}

/* ----------------------------------------------------- Algorithm 3 ----- */

/* Lines 6-9 of Algorithm 3 for one clique instance containing the pivot v
 * (slot 0): decrease each other member u whose clique-degree exceeds v's,
 * and move u to its new place in the order at once (line 11). */
static void visit_peel(lister* L, const uint32_t* c) {
    uint64_t dv = L->deg[c[0]];
    for (int i = 1; i < L->h; i++) {
        uint32_t u = c[i];
        if (L->deg[u] > dv) {
            L->deg[u]--;
            vh_up(L->heap, L->heap->pos[u]);
        }
    }
}

/* core[v] (original ids) and *kmax.  tie_order picks which of several
 * minimum clique-degree vertices goes first (0: smallest id, 1: largest);
 * the result must not depend on it. */
int orc_core_decompose(uint32_t n, const uint64_t* off, const uint32_t* adj,
                       int h, int tie_order, uint64_t* core, uint64_t* kmax) {
    if (check_h(h)) return ORC_EINVAL;
    wgraph g;
    if (wg_make(n, off, adj, &g)) return ORC_ENOMEM;
    lister L;
    int rc = ORC_ENOMEM;
    uint8_t* alive = NULL; uint32_t* tie = NULL; vheap H; memset(&H, 0, sizeof(H));
    if (lister_init(&L, &g, h, visit_count)) goto out;
    L.deg = (uint64_t*)calloc((size_t)(n ? n : 1), sizeof(uint64_t));
    alive = (uint8_t*)malloc((size_t)(n ? n : 1));
    tie = (uint32_t*)malloc((size_t)(n ? n : 1) * sizeof(uint32_t));
    H.heap = (uint32_t*)malloc((size_t)(n ? n : 1) * sizeof(uint32_t));
    H.pos = (uint32_t*)malloc((size_t)(n ? n : 1) * sizeof(uint32_t));
    if (!L.deg || !alive || !tie || !H.heap || !H.pos) goto out;
    /* line 2: clique-degree of every vertex */
    list_all(&L);
    /* line 3: order by clique-degree */
    for (uint32_t i = 0; i < n; i++) {
        alive[i] = 1;
        tie[i] = tie_order ? ~g.old_of[i] : g.old_of[i];
    }
    H.key = L.deg; H.tie = tie; H.size = n;
    for (uint32_t i = 0; i < n; i++) { H.heap[i] = i; H.pos[i] = i; }
    for (int64_t i = (int64_t)n / 2 - 1; i >= 0; i--) vh_down(&H, (uint32_t)i);
    L.visit = visit_peel;
    L.heap = &H;
    uint64_t km = 0;
    /* lines 4-11 */
    while (H.size) {
        uint32_t v = vh_pop(&H);
        core[g.old_of[v]] = L.deg[v];                 /* line 5 */
        if (L.deg[v] > km) km = L.deg[v];
        list_containing(&L, v, alive);                /* lines 6-9, 11 */
        alive[v] = 0;                                 /* line 10 */
    }
    *kmax = km;
    rc = ORC_OK;
out:
    free(L.deg); free(alive); free(tie);
    free(H.heap); free(H.pos);
    lister_free(&L); wg_free(&g);
    return rc;
}

/* -------------------------------------------- Def. 6 by pruning -------- */

static void visit_prune(lister* L, const uint32_t* c) {
    for (int i = 1; i < L->h; i++) {
        uint32_t u = c[i];
        L->deg[u]--;
        if (L->deg[u] < L->kthr && !L->queued[u]) {
            L->queued[u] = 1;
            L->queue[L->qtail++] = u;
        }
    }
}

/* in_R[v] = 1 iff v is in the (k,Psi)-core R_k: delete vertices with fewer
 * than k clique instances until none is left. */
int orc_threshold_prune(uint32_t n, const uint64_t* off, const uint32_t* adj,
                        int h, uint64_t k, uint8_t* in_R) {
    if (check_h(h)) return ORC_EINVAL;
    wgraph g;
    if (wg_make(n, off, adj, &g)) return ORC_ENOMEM;
    lister L;
    int rc = ORC_ENOMEM;
    uint8_t* alive = NULL;
    if (lister_init(&L, &g, h, visit_count)) goto out;
    L.deg = (uint64_t*)calloc((size_t)(n ? n : 1), sizeof(uint64_t));
    L.queued = (uint8_t*)calloc((size_t)(n ? n : 1), 1);
    L.queue = (uint32_t*)malloc((size_t)(n ? n : 1) * sizeof(uint32_t));
    alive = (uint8_t*)malloc((size_t)(n ? n : 1));
    if (!L.deg || !L.queued || !L.queue || !alive) goto out;
    list_all(&L);
    L.kthr = k;
    for (uint32_t v = 0; v < n; v++) {
        alive[v] = 1;
        if (L.deg[v] < k) { L.queued[v] = 1; L.queue[L.qtail++] = v; }
    }
    L.visit = visit_prune;
    for (uint64_t qh = 0; qh < L.qtail; qh++) {
        uint32_t v = L.queue[qh];
        list_containing(&L, v, alive);
        alive[v] = 0;
    }
    for (uint32_t i = 0; i < n; i++) in_R[g.old_of[i]] = alive[i];
    rc = ORC_OK;
out:
    free(L.deg); free(L.queued); free(L.queue); free(alive);
    lister_free(&L); wg_free(&g);
    return rc;
}

/* ---------------------------------------------- level statistics ------- */

static void visit_level(lister* L, const uint32_t* c) {
    uint64_t lo = L->core[c[0]];
    for (int i = 1; i < L->h; i++) if (L->core[c[i]] < lo) lo = L->core[c[i]];
    /* index of lo among the sorted distinct levels */
    uint32_t a = 0, b = L->nlevels;
    while (a < b) {
        uint32_t mid = a + (b - a) / 2;
        if (L->levels[mid] < lo) a = mid + 1; else b = mid;
    }
    L->level_hist[a]++;
}

/* Given core[] (original ids) and the sorted distinct values levels[0..nl),
 * write size[j] = |R_{levels[j]}| and mu[j] = mu(R_{levels[j]}). */
int orc_level_stats(uint32_t n, const uint64_t* off, const uint32_t* adj, int h,
                    const uint64_t* core, const uint64_t* levels, uint32_t nl,
                    uint64_t* size, uint64_t* mu) {
    if (check_h(h)) return ORC_EINVAL;
    wgraph g;
    if (wg_make(n, off, adj, &g)) return ORC_ENOMEM;
    lister L;
    int rc = ORC_ENOMEM;
    uint64_t* cw = NULL;
    if (lister_init(&L, &g, h, visit_level)) goto out;
    cw = (uint64_t*)malloc((size_t)(n ? n : 1) * sizeof(uint64_t));
    L.level_hist = (uint64_t*)calloc((size_t)nl + 1, sizeof(uint64_t));
    if (!cw || !L.level_hist) goto out;
    for (uint32_t i = 0; i < n; i++) cw[i] = core[g.old_of[i]];
    L.core = cw; L.levels = levels; L.nlevels = nl;
    list_all(&L);
    /* |R_k| counts vertices with core >= k: histogram by level, then
     * suffix sums; mu(R_k) counts cliques whose smallest core is >= k. */
    for (uint32_t j = 0; j < nl; j++) size[j] = 0;
    for (uint32_t v = 0; v < n; v++) {
        uint32_t a = 0, b = nl;
        while (a < b) {
            uint32_t mid = a + (b - a) / 2;
            if (levels[mid] < core[v]) a = mid + 1; else b = mid;
        }
        if (a < nl && levels[a] == core[v]) size[a]++;
        else { rc = ORC_EINVAL; goto out; }
    }
    uint64_t acc = 0, accv = 0;
    for (int64_t j = (int64_t)nl - 1; j >= 0; j--) {
        acc += L.level_hist[j]; mu[j] = acc;
        accv += size[j]; size[j] = accv;
    }
    rc = ORC_OK;
out:
    free(cw); free(L.level_hist);
    lister_free(&L); wg_free(&g);
    return rc;
}

/* ------------------------------------------------ pattern densities --- */
/*
 * Sec. 6 generalises the h-clique to a pattern Psi; an instance is a
 * subgraph isomorphic to Psi (Def. of subgraph isomorphism there: every
 * pattern edge maps to a graph edge, so instances need not be induced),
 * pattern-degree deg(v, Psi) = instances containing v, mu(G, Psi) = number
 * of instances.  Two special patterns, with the counts the appendix on
 * special patterns derives:
 *   ORC_STAR, x leaves (x >= 2): an instance is a centre c with x of its
 *     neighbours; deg(v) = C(d_v, x) + sum_{u in N(v)} C(d_u - 1, x - 1)
 *     (v as the centre, or as a leaf of a neighbour u); mu = sum_c C(d_c, x).
 *   ORC_LOOP4, the 4-vertex loop: an instance is a 4-cycle v-a-w-b; for
 *     fixed v its opposite vertex w and the pair {a, b} of common neighbours
 *     determine it, so deg(v) = sum_{w != v} C(|N(v) ∩ N(w)|, 2) (the
 *     appendix groups the 2-paths from v by their far end w); mu = sum deg / 4.
 * Only the vertices with alive[v] != 0 (all if alive == NULL) form the graph.
 */
#define ORC_STAR 1
#define ORC_LOOP4 2

static uint64_t binom_u64(uint64_t a, int b) {
    if (b < 0 || a < (uint64_t)b) return 0;
    uint64_t c = 1;
    for (int t = 1; t <= b; t++) c = c * (a - (uint64_t)b + (uint64_t)t) / (uint64_t)t;
    return c;
}

static uint64_t alive_degree(const uint64_t* off, const uint32_t* adj, const uint8_t* alive,
                             uint32_t v) {
    uint64_t d = 0;
    for (uint64_t p = off[v]; p < off[v + 1]; p++)
        if (!alive || alive[adj[p]]) d++;
    return d;
}

/* deg(v) of one alive vertex; cnt: n zeroed scratch counters (returned zeroed). */
static uint64_t pattern_degree_one(uint32_t n, const uint64_t* off, const uint32_t* adj,
                                   int pattern, int x, const uint8_t* alive, uint32_t v,
                                   uint32_t* cnt) {
    (void)n;
    if (pattern == ORC_STAR) {
        uint64_t dv = alive_degree(off, adj, alive, v);
        uint64_t s = binom_u64(dv, x);
        for (uint64_t p = off[v]; p < off[v + 1]; p++) {
            uint32_t u = adj[p];
            if (alive && !alive[u]) continue;
            s += binom_u64(alive_degree(off, adj, alive, u) - 1, x - 1);
        }
        return s;
    }
    /* ORC_LOOP4: c(v, w) by walking the 2-paths v-a-w */
    uint64_t s = 0;
    for (uint64_t p = off[v]; p < off[v + 1]; p++) {
        uint32_t a = adj[p];
        if (alive && !alive[a]) continue;
        for (uint64_t q = off[a]; q < off[a + 1]; q++) {
            uint32_t w = adj[q];
            if (w == v || (alive && !alive[w])) continue;
            s += cnt[w]++;          /* the new 2-path pairs with each earlier one */
        }
    }
    for (uint64_t p = off[v]; p < off[v + 1]; p++) {
        uint32_t a = adj[p];
        if (alive && !alive[a]) continue;
        for (uint64_t q = off[a]; q < off[a + 1]; q++) cnt[adj[q]] = 0;
    }
    return s;
}

static int check_pattern(int pattern, int x) {
    if (pattern == ORC_STAR) return (x >= 2 && x <= 8) ? ORC_OK : ORC_EINVAL;
    if (pattern == ORC_LOOP4) return ORC_OK;
    return ORC_EINVAL;
}

static int pattern_size(int pattern, int x) { return pattern == ORC_STAR ? x + 1 : 4; }

/* deg[v] for every vertex (0 for vertices not alive) and mu. */
int orc_pattern_degrees(uint32_t n, const uint64_t* off, const uint32_t* adj, int pattern,
                        int x, const uint8_t* alive, uint64_t* deg, uint64_t* mu) {
    if (check_pattern(pattern, x)) return ORC_EINVAL;
    uint32_t* cnt = (uint32_t*)calloc((size_t)(n ? n : 1), sizeof(uint32_t));
    if (!cnt) return ORC_ENOMEM;
    uint64_t total = 0;
    for (uint32_t v = 0; v < n; v++) {
        deg[v] = (alive && !alive[v]) ? 0 : pattern_degree_one(n, off, adj, pattern, x, alive, v, cnt);
        total += deg[v];
    }
    *mu = total / (uint64_t)pattern_size(pattern, x);
    free(cnt);
    return ORC_OK;
}

/* Algorithm 3 extended to a pattern (Sec. 4.1 remark on k-pattern-cores):
 * repeatedly take a vertex v of minimum pattern-degree (ties to the smaller
 * id), set core[v] to it, and remove v; the pattern-degree of every vertex
 * that shared an instance with v -- all lie within two hops of v -- is
 * recomputed on the remaining graph and, as Algorithm 3 never lowers a
 * degree below the removed vertex's, raised to at least core[v]. */
int orc_pattern_core_decompose(uint32_t n, const uint64_t* off, const uint32_t* adj,
                               int pattern, int x, uint64_t* core, uint64_t* kmax) {
    if (check_pattern(pattern, x)) return ORC_EINVAL;
    int rc = ORC_ENOMEM;
    size_t nn = n ? n : 1;
    uint64_t* key = (uint64_t*)malloc(nn * sizeof(uint64_t));
    uint8_t* alive = (uint8_t*)malloc(nn);
    uint32_t* cnt = (uint32_t*)calloc(nn, sizeof(uint32_t));
    uint32_t* stamp = (uint32_t*)calloc(nn, sizeof(uint32_t));
    uint32_t* tie = (uint32_t*)malloc(nn * sizeof(uint32_t));
    uint32_t* touched = (uint32_t*)malloc(nn * sizeof(uint32_t));
    vheap H;
    memset(&H, 0, sizeof(H));
    H.heap = (uint32_t*)malloc(nn * sizeof(uint32_t));
    H.pos = (uint32_t*)malloc(nn * sizeof(uint32_t));
    if (!key || !alive || !cnt || !stamp || !tie || !touched || !H.heap || !H.pos) goto out;
    for (uint32_t v = 0; v < n; v++) { alive[v] = 1; tie[v] = v; }
    for (uint32_t v = 0; v < n; v++)
        key[v] = pattern_degree_one(n, off, adj, pattern, x, alive, v, cnt);
    H.key = key; H.tie = tie; H.size = n;
    for (uint32_t i = 0; i < n; i++) { H.heap[i] = i; H.pos[i] = i; }
    for (int64_t i = (int64_t)n / 2 - 1; i >= 0; i--) vh_down(&H, (uint32_t)i);
    uint64_t km = 0;
    uint32_t round = 0;
    while (H.size) {
        uint32_t v = vh_pop(&H);
        uint64_t kv = key[v];
        core[v] = kv;
        if (kv > km) km = kv;
        alive[v] = 0;
        /* alive vertices within two hops of v */
        round++;
        uint32_t nt = 0;
        for (uint64_t p = off[v]; p < off[v + 1]; p++) {
            uint32_t a = adj[p];
            if (alive[a] && stamp[a] != round) { stamp[a] = round; touched[nt++] = a; }
            for (uint64_t q = off[a]; q < off[a + 1]; q++) {
                uint32_t w = adj[q];
                if (alive[w] && stamp[w] != round) { stamp[w] = round; touched[nt++] = w; }
            }
        }
        for (uint32_t i = 0; i < nt; i++) {
            uint32_t u = touched[i];
            uint64_t d = pattern_degree_one(n, off, adj, pattern, x, alive, u, cnt);
            if (d < kv) d = kv;
            if (d < key[u]) {
                key[u] = d;
                vh_up(&H, H.pos[u]);
            }
        }
    }
    *kmax = km;
    rc = ORC_OK;
out:
    free(key); free(alive); free(cnt); free(stamp); free(tie); free(touched);
    free(H.heap); free(H.pos);
    return rc;
}

/* For the distinct core values k (ascending, nl of them in levels[]):
 * size[j] = |R_k| and mu[j] = mu(G[R_k], Psi) with R_k = {v : core(v) >= k}. */
int orc_pattern_level_stats(uint32_t n, const uint64_t* off, const uint32_t* adj, int pattern,
                            int x, const uint64_t* core, const uint64_t* levels, uint32_t nl,
                            uint64_t* size, uint64_t* mu) {
    if (check_pattern(pattern, x)) return ORC_EINVAL;
    size_t nn = n ? n : 1;
    uint8_t* mask = (uint8_t*)malloc(nn);
    uint64_t* deg = (uint64_t*)malloc(nn * sizeof(uint64_t));
    if (!mask || !deg) { free(mask); free(deg); return ORC_ENOMEM; }
    int rc = ORC_OK;
    for (uint32_t j = 0; j < nl && rc == ORC_OK; j++) {
        uint64_t s = 0;
        for (uint32_t v = 0; v < n; v++) { mask[v] = core[v] >= levels[j]; s += mask[v]; }
        size[j] = s;
        rc = orc_pattern_degrees(n, off, adj, pattern, x, mask, deg, &mu[j]);
    }
    free(mask); free(deg);
    return rc;
}

/* ------------------------------------------ Algorithm 1 (Exact) ------ */

/* Sec. 3.1 builds, for a guess alpha, a flow network over the vertices and
 * the (h-1)-cliques Lambda: s -> v with capacity deg(v, Psi), v -> t with
 * capacity alpha * h, psi -> v with infinite capacity for every member v of
 * psi, and v -> psi with capacity 1 when psi + v is an h-clique.  A vertex
 * set A on the source side (with every psi whose members all lie in A) cuts
 *     h * mu(G) - h * mu(A) + alpha * h * |A|,
 * so the minimum cut lies below h * mu(G) exactly when some A has
 * mu(A) > alpha * |A|.  Here alpha = p / q is kept exact by scaling every
 * capacity by q (128-bit integers), and the minimum cut comes from Dinic's
 * algorithm. */

typedef unsigned __int128 u128;

enum { ARC_REV = 0, ARC_S = 1, ARC_T = 2, ARC_Q = 3, ARC_INF = 4 };

typedef struct {
    uint32_t N;               /* 0 = s, 1 = t, 2 + v vertices, then Lambda */
    uint64_t E, cap_e;
    /* arcs as added: e = from -> to, its residual twin e ^ 1 */
    uint32_t* from;
    uint32_t* to;
    uint8_t* kind;
    /* the same arcs grouped by tail node (fn_finish): slots first[x] ..
     * first[x+1]-1 of node x, head node, twin slot, kind, residual capacity */
    uint64_t* first;
    uint32_t* head;
    uint64_t* twin;
    uint8_t* skind;
    u128* cap;
    int32_t* level;
    uint64_t* it;
    uint32_t* queue;
} fnet;

static void fn_free(fnet* F) {
    free(F->from); free(F->to); free(F->kind);
    free(F->first); free(F->head); free(F->twin); free(F->skind); free(F->cap);
    free(F->level); free(F->it); free(F->queue);
    memset(F, 0, sizeof(*F));
}

static int fn_init(fnet* F, uint32_t N, uint64_t E) {
    memset(F, 0, sizeof(*F));
    F->N = N;
    F->cap_e = E;
    size_t e1 = (size_t)(E ? E : 1);
    F->from = (uint32_t*)malloc(e1 * sizeof(uint32_t));
    F->to = (uint32_t*)malloc(e1 * sizeof(uint32_t));
    F->kind = (uint8_t*)malloc(e1);
    F->level = (int32_t*)malloc((size_t)N * sizeof(int32_t));
    F->it = (uint64_t*)malloc((size_t)N * sizeof(uint64_t));
    F->queue = (uint32_t*)malloc((size_t)N * sizeof(uint32_t));
    if (!F->from || !F->to || !F->kind || !F->level || !F->it || !F->queue) {
        fn_free(F);
        return ORC_ENOMEM;
    }
    return ORC_OK;
}

/* Arc u -> v of the given kind and its residual twin v -> u (index ^ 1). */
static void fn_arc(fnet* F, uint32_t u, uint32_t v, uint8_t kind) {
    uint64_t e = F->E;
    if (e + 2 > F->cap_e) { F->E = e + 2; return; }   /* counted, caught by the caller */
    F->from[e] = u; F->to[e] = v; F->kind[e] = kind;
    F->from[e + 1] = v; F->to[e + 1] = u; F->kind[e + 1] = ARC_REV;
    F->E = e + 2;
}

/* Groups the arcs by tail node (a counting sort). */
static int fn_finish(fnet* F) {
    size_t e1 = (size_t)(F->E ? F->E : 1);
    uint64_t* pos = (uint64_t*)malloc(e1 * sizeof(uint64_t));
    F->first = (uint64_t*)calloc((size_t)F->N + 1, sizeof(uint64_t));
    F->head = (uint32_t*)malloc(e1 * sizeof(uint32_t));
    F->twin = (uint64_t*)malloc(e1 * sizeof(uint64_t));
    F->skind = (uint8_t*)malloc(e1);
    F->cap = (u128*)malloc(e1 * sizeof(u128));
    if (!pos || !F->first || !F->head || !F->twin || !F->skind || !F->cap) {
        free(pos);
        return ORC_ENOMEM;
    }
    for (uint64_t e = 0; e < F->E; e++) F->first[F->from[e] + 1]++;
    for (uint32_t x = 0; x < F->N; x++) F->first[x + 1] += F->first[x];
    for (uint64_t e = 0; e < F->E; e++) pos[e] = F->first[F->from[e]]++;
    for (uint32_t x = F->N; x > 0; x--) F->first[x] = F->first[x - 1];
    F->first[0] = 0;
    for (uint64_t e = 0; e < F->E; e++) {
        F->head[pos[e]] = F->to[e];
        F->skind[pos[e]] = F->kind[e];
        F->twin[pos[e]] = pos[e ^ 1];
    }
    free(pos);
    free(F->from); free(F->to); free(F->kind);
    F->from = F->to = NULL;
    F->kind = NULL;
    return ORC_OK;
}

/* Capacities for alpha = p / q (all scaled by q); twins start empty. */
static void fn_capacities(fnet* F, const uint64_t* deg, int h, u128 p, u128 q) {
    const u128 inf = (u128)1 << 120;
    for (uint64_t a = 0; a < F->E; a++) {
        u128 c = 0;
        switch (F->skind[a]) {
            case ARC_S: c = q * deg[F->head[a] - 2]; break;
            case ARC_T: c = p * (u128)h; break;
            case ARC_Q: c = q; break;
            case ARC_INF: c = inf; break;
        }
        F->cap[a] = c;
    }
}

/* Breadth-first levels from s over arcs with residual capacity. */
static int fn_bfs(fnet* F) {
    for (uint32_t x = 0; x < F->N; x++) F->level[x] = -1;
    uint64_t qh = 0, qt = 0;
    F->level[0] = 0;
    F->queue[qt++] = 0;
    while (qh < qt) {
        uint32_t u = F->queue[qh++];
        for (uint64_t a = F->first[u]; a < F->first[u + 1]; a++) {
            uint32_t v = F->head[a];
            if (F->cap[a] > 0 && F->level[v] < 0) {
                F->level[v] = F->level[u] + 1;
                F->queue[qt++] = v;
            }
        }
    }
    return F->level[1] >= 0;
}

/* Dinic's maximum flow from s = 0 to t = 1; the blocking flow of each level
 * graph is found by an explicit-stack depth-first search. */
static int fn_maxflow(fnet* F, u128* flow_out) {
    uint32_t* pnode = (uint32_t*)malloc((size_t)F->N * sizeof(uint32_t));
    uint64_t* parc = (uint64_t*)malloc((size_t)F->N * sizeof(uint64_t));
    if (!pnode || !parc) { free(pnode); free(parc); return ORC_ENOMEM; }
    u128 flow = 0;
    while (fn_bfs(F)) {
        for (uint32_t x = 0; x < F->N; x++) F->it[x] = F->first[x];
        for (;;) {
            uint32_t depth = 0, u = 0;
            int found = 0;
            for (;;) {
                if (u == 1) { found = 1; break; }
                uint64_t a = F->it[u], end = F->first[u + 1];
                while (a < end && !(F->cap[a] > 0 && F->level[F->head[a]] == F->level[u] + 1))
                    a++;
                F->it[u] = a;
                if (a == end) {                   /* dead end: retreat */
                    F->level[u] = -1;
                    if (depth == 0) break;
                    depth--;
                    u = pnode[depth];
                    F->it[u] = parc[depth] + 1;
                    continue;
                }
                pnode[depth] = u;
                parc[depth] = a;
                depth++;
                u = F->head[a];
            }
            if (!found) break;
            u128 b = F->cap[parc[0]];
            for (uint32_t i = 1; i < depth; i++)
                if (F->cap[parc[i]] < b) b = F->cap[parc[i]];
            for (uint32_t i = 0; i < depth; i++) {
                F->cap[parc[i]] -= b;
                F->cap[F->twin[parc[i]]] += b;
            }
            flow += b;
        }
    }
    free(pnode); free(parc);
    *flow_out = flow;
    return ORC_OK;
}

/* After a maximum flow: mark[x] = 1 for the nodes that can still reach t
 * through arcs with residual capacity.  Their complement is the largest
 * source side among all minimum cuts. */
static void fn_reach_t(fnet* F, uint8_t* mark) {
    memset(mark, 0, F->N);
    uint64_t qh = 0, qt = 0;
    mark[1] = 1;
    F->queue[qt++] = 1;
    while (qh < qt) {
        uint32_t y = F->queue[qh++];
        for (uint64_t a = F->first[y]; a < F->first[y + 1]; a++) {
            uint32_t x = F->head[a];          /* arc a: y -> x; its twin x -> y */
            if (!mark[x] && F->cap[F->twin[a]] > 0) {
                mark[x] = 1;
                F->queue[qt++] = x;
            }
        }
    }
}

static void visit_store(lister* L, const uint32_t* c) {
    if (L->nstore >= L->capstore) {
        uint64_t nc = L->capstore ? 2 * L->capstore : 1024;
        uint32_t* ns = (uint32_t*)realloc(L->store, (size_t)nc * L->h * sizeof(uint32_t));
        if (!ns) { L->overflow = 1; return; }
        L->store = ns;
        L->capstore = nc;
    }
    memcpy(L->store + L->nstore * L->h, c, (size_t)L->h * sizeof(uint32_t));
    L->nstore++;
}

static void visit_count_mask(lister* L, const uint32_t* c) {
    for (int i = 0; i < L->h; i++)
        if (!L->mask[c[i]]) return;
    L->mu++;
}

/* mu(G[A]) for A = {new ids x : mask[x]} on the working graph. */
static int wg_count_in(const wgraph* g, int h, const uint8_t* mask, uint64_t* mu) {
    lister L;
    if (lister_init(&L, g, h, visit_count_mask)) { lister_free(&L); return ORC_ENOMEM; }
    L.mask = mask;
    list_all(&L);
    *mu = L.mu;
    lister_free(&L);
    return ORC_OK;
}

static u128 gcd128(u128 a, u128 b) {
    while (b) { u128 t = a % b; a = b; b = t; }
    return a;
}

/* Algorithm 1's network for G (working graph g, mu(G) = mu): s, t, one node
 * per vertex and per (h-1)-clique psi (listed once each); arcs s -> v, v -> t,
 * psi -> v for v in psi, w -> psi for every w adjacent to all of psi. */
static int alg1_network(const wgraph* g, int h, uint64_t mu, fnet* F) {
    const uint32_t n = g->n;
    int rc = ORC_ENOMEM;
    lister C;
    memset(&C, 0, sizeof(C));
    uint32_t* cn = (uint32_t*)malloc(((size_t)g->maxdeg + 1) * sizeof(uint32_t));
    uint32_t* cn2 = (uint32_t*)malloc(((size_t)g->maxdeg + 1) * sizeof(uint32_t));
    if (!cn || !cn2) goto out;
    /* Lambda: the (h-1)-cliques, each once */
    if (lister_init(&C, g, h - 1, visit_store)) goto out;
    list_all(&C);
    if (C.overflow) goto out;
    uint64_t nl = C.nstore;
    if ((uint64_t)n + nl + 2 >= ((uint64_t)1 << 31)) { rc = ORC_EINVAL; goto out; }
    uint32_t N = (uint32_t)(2 + n + nl);
    uint64_t E = 2 * (2 * (uint64_t)n + (uint64_t)(h - 1) * nl + (uint64_t)h * mu);
    if (fn_init(F, N, E)) goto out;
    for (uint32_t v = 0; v < n; v++) {
        fn_arc(F, 0, 2 + v, ARC_S);
        fn_arc(F, 2 + v, 1, ARC_T);
    }
    for (uint64_t i = 0; i < nl; i++) {
        const uint32_t* psi = C.store + i * (h - 1);
        uint32_t node = (uint32_t)(2 + n + i);
        for (int j = 0; j < h - 1; j++) fn_arc(F, node, 2 + psi[j], ARC_INF);
        /* common neighbours of psi's members: psi + w is an h-clique */
        uint32_t x0 = psi[0];
        uint32_t k = (uint32_t)(g->off[x0 + 1] - g->off[x0]);
        memcpy(cn, g->adj + g->off[x0], (size_t)k * sizeof(uint32_t));
        for (int j = 1; j < h - 1 && k; j++) {
            uint32_t x = psi[j];
            k = intersect(cn, k, g->adj + g->off[x], g->off[x + 1] - g->off[x], cn2);
            memcpy(cn, cn2, (size_t)k * sizeof(uint32_t));
        }
        for (uint32_t j = 0; j < k; j++) fn_arc(F, 2 + cn[j], node, ARC_Q);
    }
    rc = F->E == E ? fn_finish(F) : -3;
out:
    free(C.store);
    lister_free(&C);
    free(cn); free(cn2);
    if (rc) fn_free(F);
    return rc;
}

/* The CDS of G (Problem 1) by Algorithm 1, and then the largest densest set.
 *
 * in_cds[v] (original ids) marks the union of all vertex sets of maximum
 * h-clique-density; *mu_out = mu of that set and *size_out = its size, so
 * rho_opt = *mu_out / *size_out.  *steps = binary-search iterations.  The
 * union of two densest sets is again densest (mu(A u B) + mu(A n B) >=
 * mu(A) + mu(B)), so this set is unique; it is the largest source side of a
 * minimum cut at alpha = rho_opt.  With no h-clique every set has density 0
 * and the answer is V.  Returns ORC_EINVAL when n^2 * max deg(v, Psi) does
 * not fit the exact arithmetic (2^60). */
int orc_exact_cds(uint32_t n, const uint64_t* off, const uint32_t* adj, int h,
                  uint8_t* in_cds, uint64_t* mu_out, uint64_t* size_out, uint32_t* steps) {
    if (check_h(h)) return ORC_EINVAL;
    *steps = 0;
    wgraph g;
    if (wg_make(n, off, adj, &g)) return ORC_ENOMEM;
    int rc = ORC_ENOMEM;
    lister L;
    memset(&L, 0, sizeof(L));
    fnet F;
    memset(&F, 0, sizeof(F));
    uint64_t* deg = (uint64_t*)calloc((size_t)(n ? n : 1), sizeof(uint64_t));
    uint8_t* inD = (uint8_t*)calloc((size_t)(n ? n : 1), 1);
    uint8_t* mark = NULL;
    if (!deg || !inD) goto out;
    /* clique-degrees and mu(G) */
    if (lister_init(&L, &g, h, visit_count)) goto out;
    L.deg = deg;
    list_all(&L);
    uint64_t mu = L.mu;
    if (mu == 0) {
        for (uint32_t v = 0; v < n; v++) in_cds[v] = 1;
        *mu_out = 0;
        *size_out = n;
        rc = ORC_OK;
        goto out;
    }
    uint64_t maxdeg = 0;
    for (uint32_t v = 0; v < n; v++) if (deg[v] > maxdeg) maxdeg = deg[v];
    u128 nn1 = (u128)n * (n - 1);
    if (nn1 * maxdeg >= ((u128)1 << 60)) { rc = ORC_EINVAL; goto out; }
    rc = alg1_network(&g, h, mu, &F);
    if (rc) goto out;
    rc = ORC_ENOMEM;
    mark = (uint8_t*)malloc(F.N);
    if (!mark) goto out;
    /* binary search (l, u) = (L, U) / 2^t over [0, max deg] */
    u128 Lo = 0, Up = maxdeg;
    int t = 0, haveD = 0;
    while ((Up - Lo) * nn1 >= ((u128)1 << t)) {
        u128 A = Lo + Up;               /* alpha = A / 2^(t+1) */
        u128 q = (u128)1 << (t + 1);
        fn_capacities(&F, deg, h, A, q);
        u128 flow;
        if (fn_maxflow(&F, &flow)) goto out;
        /* minimal source side: the nodes s still reaches (last BFS) */
        int any = 0;
        for (uint32_t v = 0; v < n; v++) if (F.level[2 + v] >= 0) { any = 1; break; }
        if (!any) {
            Up = A;
            Lo = 2 * Lo;
        } else {
            Lo = A;
            Up = 2 * Up;
            for (uint32_t v = 0; v < n; v++) inD[v] = F.level[2 + v] >= 0;
            haveD = 1;
        }
        t++;
        (*steps)++;
        if (t > 120) { rc = -3; goto out; }
    }
    if (!haveD) { rc = -3; goto out; }
    uint64_t muD, sD = 0;
    for (uint32_t v = 0; v < n; v++) sD += inD[v];
    if (wg_count_in(&g, h, inD, &muD)) goto out;
    /* the largest densest set: the largest minimum-cut source side at
     * alpha = rho(D) = rho_opt */
    u128 gg = gcd128(muD, sD);
    fn_capacities(&F, deg, h, (u128)muD / gg, (u128)sD / gg);
    u128 flow;
    if (fn_maxflow(&F, &flow)) goto out;
    if (flow != (u128)sD / gg * h * mu) { rc = -3; goto out; }  /* no set beats rho(D) */
    fn_reach_t(&F, mark);
    uint64_t sM = 0, muM = 0;
    for (uint32_t v = 0; v < n; v++) { inD[v] = !mark[2 + v]; sM += inD[v]; }
    if (wg_count_in(&g, h, inD, &muM)) goto out;
    if (sM < sD || (u128)muM * sD != (u128)muD * sM) { rc = -3; goto out; }
    for (uint32_t i = 0; i < n; i++) in_cds[g.old_of[i]] = inD[i];
    *mu_out = muM;
    *size_out = sM;
    rc = ORC_OK;
out:
    fn_free(&F);
    lister_free(&L);
    free(deg); free(inD); free(mark);
    wg_free(&g);
    return rc;
}

/* One minimum cut of Algorithm 1's network at alpha = p / q (q > 0): a
 * certificate check of a claimed optimum.  *beats = 1 when some vertex set A
 * has mu(A) > alpha |A| (the cut is below q h mu(G)); in_set (original ids)
 * marks the vertices of the largest source side of a minimum cut.  At
 * alpha = rho_opt, *beats = 0 and in_set is the largest densest set. */
int orc_densest_check(uint32_t n, const uint64_t* off, const uint32_t* adj, int h,
                      uint64_t p, uint64_t q, uint8_t* in_set, int* beats) {
    if (check_h(h) || q == 0) return ORC_EINVAL;
    wgraph g;
    if (wg_make(n, off, adj, &g)) return ORC_ENOMEM;
    int rc = ORC_ENOMEM;
    lister L;
    memset(&L, 0, sizeof(L));
    fnet F;
    memset(&F, 0, sizeof(F));
    uint8_t* mark = NULL;
    uint64_t* deg = (uint64_t*)calloc((size_t)(n ? n : 1), sizeof(uint64_t));
    if (!deg) goto out;
    if (lister_init(&L, &g, h, visit_count)) goto out;
    L.deg = deg;
    list_all(&L);
    rc = alg1_network(&g, h, L.mu, &F);
    if (rc) goto out;
    rc = ORC_ENOMEM;
    mark = (uint8_t*)malloc(F.N);
    if (!mark) goto out;
    fn_capacities(&F, deg, h, p, q);
    u128 flow;
    if (fn_maxflow(&F, &flow)) goto out;
    *beats = flow < (u128)q * h * L.mu;
    fn_reach_t(&F, mark);
    for (uint32_t i = 0; i < n; i++) in_set[g.old_of[i]] = !mark[2 + i];
    rc = ORC_OK;
out:
    fn_free(&F);
    lister_free(&L);
    free(deg); free(mark);
    wg_free(&g);
    return rc;
}

/* ------------------------------------------ Algorithm 2 (PeelApp) ---- */

/* One clique instance through the removed vertex v (slot 0): every other
 * member loses it (exact clique-degrees, no floor). */
static void visit_peel_exact(lister* L, const uint32_t* c) {
    for (int i = 1; i < L->h; i++) {
        uint32_t u = c[i];
        L->deg[u]--;
        vh_up(L->heap, L->heap->pos[u]);
    }
}

/* Algorithm 2 (PeelApp, Sec. 3.2): remove a vertex of minimum current
 * clique-degree (ties: the smaller original id) one at a time and keep the
 * densest of the sets met.  The sets are G itself and every residual; a
 * later set replaces the best only when strictly denser.  in_best[v]
 * (original ids) marks the best set; *mu_out and *size_out are its clique
 * count and size (with no h-clique: G, 0 cliques).  order_out (may be NULL,
 * n entries) receives the removal order in original ids. */
int orc_peel_app(uint32_t n, const uint64_t* off, const uint32_t* adj, int h,
                 uint8_t* in_best, uint64_t* mu_out, uint64_t* size_out, uint32_t* order_out) {
    if (check_h(h)) return ORC_EINVAL;
    wgraph g;
    if (wg_make(n, off, adj, &g)) return ORC_ENOMEM;
    lister L;
    int rc = ORC_ENOMEM;
    uint8_t* alive = NULL; uint32_t* tie = NULL; uint32_t* order = NULL;
    vheap H; memset(&H, 0, sizeof(H));
    if (lister_init(&L, &g, h, visit_count)) goto out;
    L.deg = (uint64_t*)calloc((size_t)(n ? n : 1), sizeof(uint64_t));
    alive = (uint8_t*)malloc((size_t)(n ? n : 1));
    tie = (uint32_t*)malloc((size_t)(n ? n : 1) * sizeof(uint32_t));
    order = (uint32_t*)malloc((size_t)(n ? n : 1) * sizeof(uint32_t));
    H.heap = (uint32_t*)malloc((size_t)(n ? n : 1) * sizeof(uint32_t));
    H.pos = (uint32_t*)malloc((size_t)(n ? n : 1) * sizeof(uint32_t));
    if (!L.deg || !alive || !tie || !order || !H.heap || !H.pos) goto out;
    list_all(&L);                                  /* clique-degrees and mu(G) */
    uint64_t mu = L.mu;
    for (uint32_t i = 0; i < n; i++) { alive[i] = 1; tie[i] = g.old_of[i]; }
    H.key = L.deg; H.tie = tie; H.size = n;
    for (uint32_t i = 0; i < n; i++) { H.heap[i] = i; H.pos[i] = i; }
    for (int64_t i = (int64_t)n / 2 - 1; i >= 0; i--) vh_down(&H, (uint32_t)i);
    L.visit = visit_peel_exact;
    L.heap = &H;
    uint64_t bmu = mu, bsize = n, bstep = 0, size = n, step = 0;
    while (H.size) {
        uint32_t v = vh_pop(&H);
        order[step++] = v;
        mu -= L.deg[v];                            /* the cliques through v */
        list_containing(&L, v, alive);
        alive[v] = 0;
        size--;
        if (size && (unsigned __int128)mu * bsize > (unsigned __int128)bmu * size) {
            bmu = mu;
            bsize = size;
            bstep = step;
        }
    }
    for (uint32_t i = 0; i < n; i++) in_best[i] = 0;
    for (uint64_t j = bstep; j < n; j++) in_best[g.old_of[order[j]]] = 1;
    if (order_out)
        for (uint32_t j = 0; j < n; j++) order_out[j] = g.old_of[order[j]];
    *mu_out = bmu;
    *size_out = bsize;
    rc = ORC_OK;
out:
    free(L.deg); free(alive); free(tie); free(order);
    free(H.heap); free(H.pos);
    lister_free(&L); wg_free(&g);
    return rc;
}
