// Oversized candidate sets for h >= 4: more than kBitmapMax candidates
// (graphs whose degeneracy exceeds 1024).
//
// The sub-problem is the one of cliques.cuh: a fixed root clique, sorted
// candidates C adjacent to every root member, and rr members still to
// choose; every rr-clique of G[C] is one h-clique.  One block splits it by
// its next member z: the cliques whose smallest candidate is z are z plus an
// (rr-1)-clique of C' = {y in C : y > z} ∩ N+(z), listed the same way, until
// a set fits the bitmap tier (at most kBitmapMax candidates), one member
// remains (every candidate closes one clique), or two remain over at most
// kXLSharedMax candidates (every edge of G[C], found by scanning N+(x) for
// each x in C against C held in shared memory).
// The open levels' candidate lists live in the block's global scratch
// (kMaxDepth levels of `cap` entries).  Credits go through the caller's
// functor: cand(x, c) for a candidate x in c cliques, root(c) for the
// caller's fixed root members; the members chosen by the splits are
// candidates of the level above and are credited through cand.
#pragma once

#include "cliques.cuh"

namespace dsd {

// Two members left: candidate lists up to this size and their counters are
// kept in shared memory (2 * kXLSharedMax words of the bitmap tier's
// buffers).
constexpr uint32_t kXLSharedMax = 8192;

// Order-preserving filter, whole block: out[0 .. *count) = the entries y of
// in[0, n_in) with keep(y), in order.  Returns the count (all threads).
template <class Keep>
__device__ __forceinline__ uint32_t block_filter(const uint32_t* in, uint64_t n_in,
                                                 uint32_t* out, Keep keep, uint32_t* s_w,
                                                 uint32_t* s_tot) {
    const unsigned lane = lane_id(), wid = warp_id(), nw = blockDim.x >> 5;
    uint32_t total = 0;
    for (uint64_t base = 0; base < n_in; base += blockDim.x) {
        const uint64_t i = base + threadIdx.x;
        uint32_t y = 0;
        bool k = false;
        if (i < n_in) {
            y = in[i];
            k = keep(y);
        }
        const unsigned bal = __ballot_sync(0xffffffffu, k);
        if (lane == 0) s_w[wid] = __popc(bal);
        __syncthreads();
        uint32_t before = 0, all = 0;
        for (unsigned w = 0; w < nw; w++) {
            uint32_t c = s_w[w];
            before += w < wid ? c : 0u;
            all += c;
        }
        if (k) out[total + before + __popc(bal & ((1u << lane) - 1u))] = y;
        total += all;
        __syncthreads();   // s_w is rewritten by the next pass
    }
    (void)s_tot;
    return total;
}

struct XLLevel {
    const uint32_t* C;
    uint32_t n;
    int rr;
    uint32_t i;       // next member to split on
    uint32_t z;       // member chosen to open this level (not for level 0)
};

// smem: kBitmapMax u64 counters, kBitmapMax candidates, kBitmapMax * 32 row
// words (the bitmap tier's buffers).  scratch: kMaxDepth * cap entries.
template <class Cand, class Root>
__device__ void xl_cliques(const uint32_t* C0, uint32_t n0, int rr0, const uint64_t* nb,
                           const uint64_t* ne, const uint32_t* adj, uint32_t* scratch,
                           uint32_t cap, uint32_t* smem, Cand cand, Root root) {
    __shared__ XLLevel s_lv[kMaxDepth + 1];
    __shared__ int s_t;
    __shared__ uint32_t s_w[32], s_tot, s_next;
    __shared__ unsigned long long s_sum;
    const unsigned lane = lane_id(), wid = warp_id(), nw = blockDim.x >> 5;
    unsigned long long* cnt = reinterpret_cast<unsigned long long*>(smem);   // kBitmapMax
    uint32_t* Cs = smem + 2 * kBitmapMax;                                    // kBitmapMax
    uint32_t* rows = Cs + kBitmapMax;                                        // kBitmapMax * 32
    if (threadIdx.x == 0) {
        s_lv[0] = XLLevel{C0, n0, rr0, 0u, 0u};
        s_t = 0;
    }
    __syncthreads();
    for (;;) {
        const int t = s_t;
        if (t < 0) break;
        const XLLevel L = s_lv[t];
        __syncthreads();
        // leaves: a set the bitmap tier holds, one member left, or two
        // members left over a set whose list and counters fit shared memory
        const bool leaf = L.n <= kBitmapMax || L.rr == 1 ||
                          (L.rr == 2 && L.n <= kXLSharedMax);
        if (leaf) {
            if (threadIdx.x == 0) s_sum = 0;
            __syncthreads();
            unsigned long long mine = 0;
            if (L.rr == 1) {
                for (uint32_t i = threadIdx.x; i < L.n; i += blockDim.x) cand(L.C[i], 1ull);
                mine = threadIdx.x == 0 ? L.n : 0;
            } else if (L.n > kBitmapMax) {
                // rr = 2: every edge (x, y) of G[C], x < y, by scanning N+(x)
                // against C in shared memory, with shared counters
                uint32_t* Cs2 = smem;
                unsigned* c2 = smem + kXLSharedMax;
                const uint32_t n = L.n;
                for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) {
                    Cs2[i] = L.C[i];
                    c2[i] = 0;
                }
                __syncthreads();
                const uint32_t cmax = Cs2[n - 1];
                for (uint32_t i = wid; i + 1 < n; i += nw) {
                    const uint32_t x = Cs2[i];
                    unsigned hits = scan_row_hits(Cs2, n, cmax, adj, nb[x], ne[x], c2);
                    hits = __reduce_add_sync(0xffffffffu, hits);
                    if (lane == 0 && hits) {
                        atomicAdd(&c2[i], hits);
                        mine += hits;
                    }
                }
                __syncthreads();
                for (uint32_t i = threadIdx.x; i < n; i += blockDim.x)
                    if (c2[i]) cand(Cs2[i], (unsigned long long)c2[i]);
            } else {
                // at most kBitmapMax candidates: the bitmap tier (rr >= 2)
                const uint32_t n = L.n, W = (n + 31) >> 5;
                for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) {
                    Cs[i] = L.C[i];
                    cnt[i] = 0;
                }
                for (uint32_t i = threadIdx.x; i < n * W; i += blockDim.x) rows[i] = 0;
                if (threadIdx.x == 0) s_next = 0;
                __syncthreads();
                block_build_rows(Cs, n, W, ne, adj, nb, rows);
                __syncthreads();
                mine = block_dfs(rows, n, W, L.rr, cnt, &s_next);
                __syncthreads();
                for (uint32_t i = threadIdx.x; i < n; i += blockDim.x)
                    if (cnt[i]) cand(Cs[i], cnt[i]);
            }
            if (mine) atomicAdd(&s_sum, mine);
            __syncthreads();
            const unsigned long long T = s_sum;
            if (threadIdx.x == 0) {
                if (T) {
                    root(T);
                    for (int d = 1; d <= t; d++) cand(s_lv[d].z, T);
                }
                s_t = t - 1;
            }
            __syncthreads();
            continue;
        }
        // split on the next member, if enough candidates remain after it
        if (L.i + (uint32_t)L.rr > L.n) {
            if (threadIdx.x == 0) s_t = t - 1;
            __syncthreads();
            continue;
        }
        const uint32_t z = L.C[L.i];
        const uint32_t* rest = L.C + L.i + 1;
        const uint32_t nrest = L.n - L.i - 1;
        const uint32_t cmax = L.C[L.n - 1];
        uint32_t* out = scratch + (size_t)t * cap;
        const uint32_t n2 = block_filter(
            adj + nb[z], ne[z] - nb[z], out,
            [&](uint32_t y) {
                if (y > cmax) return false;
                uint64_t pos = lower_bound_u32(rest, nrest, y);
                return pos < nrest && rest[pos] == y;
            },
            s_w, &s_tot);
        if (threadIdx.x == 0) {
            s_lv[t].i = L.i + 1;
            if (n2 >= (uint32_t)(L.rr - 1) && t + 1 <= kMaxDepth - 1) {
                s_lv[t + 1] = XLLevel{out, n2, L.rr - 1, 0u, z};
                s_t = t + 1;
            }
        }
        __syncthreads();
    }
}

}  // namespace dsd
