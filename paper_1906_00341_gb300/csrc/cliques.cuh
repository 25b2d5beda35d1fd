// Device routines shared by clique listing and peeling.
//
// Both reduce to one sub-problem: a fixed clique prefix ("root") and a
// sorted candidate list C of vertices adjacent to every root member; find
// the r-cliques inside G[C] and credit each member of C with the number of
// r-cliques it lies in (the root members get the total).  Each r-clique is
// listed once as an increasing sequence of positions in C, extending only
// through the oriented lists N+(x) = {y in N(x) : y > x}.  This is the
// kClist-style ordered listing the paper relies on for clique enumeration
// (Sec. 4.3), restated for warps and blocks.
//
// Local adjacency of G[C] is a bitmap: row i holds bit j (j > i) when C[j]
// is in N+(C[i]).  Up to 32 candidates a row is one word (warp routines);
// up to 1024 a row is 32 words, one per lane (block routines).
#pragma once

#include "common.cuh"

namespace dsd {

constexpr int kMaxDepth = DSD_MAX_H;     // r <= h - 1 <= 7
constexpr uint32_t kBitmapMax = 1024;   // candidates per bitmap problem

// ---------------------------------------------------------------------------
// Row construction: for candidate i, the positions j > i whose vertex is in
// N+(C[i]) = adj[nb[x] .. ne[x]).  Candidates are sorted ascending, N+ lists
// too, and every j > i automatically has C[j] > C[i]; membership is a binary
// search in C.

// Row scans read kScanChunks chunks of 32 entries per step (their loads in
// flight together) and stop at the first chunk past the largest candidate:
// the lists ascend, so nothing beyond it can be in C.
constexpr int kScanChunks = 4;

// Hits of the list adj[b, e) (ascending) in the sorted candidates C[0, nc)
// whose largest entry is cmax, by one warp: cnt[pos] += 1 for each hit
// (shared counters); returns this lane's number of hits.  Each step loads
// kScanChunks coalesced 32-entry chunks at once, lane l taking entry l of
// each, so that the lanes' binary searches look for neighbouring ids and
// follow nearly the same path through C; the scan stops after the first step
// that passes cmax.  *read_end (if given) receives the end of what was read.
template <class T>
__device__ __forceinline__ unsigned scan_row_hits(const uint32_t* C, uint32_t nc, uint32_t cmax,
                                                  const uint32_t* adj, uint64_t b, uint64_t e,
                                                  T* cnt, uint64_t* read_end = nullptr) {
    const unsigned lane = lane_id();
    unsigned hits = 0;
    uint64_t p0 = b;
    for (; p0 < e; p0 += 32 * kScanChunks) {
        uint32_t ys[kScanChunks];
#pragma unroll
        for (int u = 0; u < kScanChunks; u++) {
            uint64_t p = p0 + u * 32 + lane;
            ys[u] = p < e ? adj[p] : 0xffffffffu;
        }
#pragma unroll
        for (int u = 0; u < kScanChunks; u++) {
            const uint32_t y = ys[u];
            if (y <= cmax) {
                uint32_t pos = (uint32_t)lower_bound_u32(C, nc, y);
                if (pos < nc && C[pos] == y) {
                    atomicAdd(&cnt[pos], (T)1);
                    hits++;
                }
            }
        }
        if (__shfl_sync(0xffffffffu, ys[kScanChunks - 1], 31) > cmax) {
            p0 += 32 * kScanChunks;
            break;
        }
    }
    if (read_end) *read_end = p0 < e ? p0 : e;
    return hits;
}

// One warp: the one-word row of candidate x = C[i] for |C| <= 32, i.e. bit j
// set iff C[j] > x lies in x's list adj[b, e) (sorted ascending; the scan
// stops past cmax = C[nc - 1]).  All lanes return it.
__device__ __forceinline__ uint32_t warp_row32(const uint32_t* C, uint32_t nc, uint32_t cmax,
                                               uint32_t x, const uint32_t* adj, uint64_t b,
                                               uint64_t e) {
    const unsigned lane = lane_id();
    uint32_t bits = 0;
    for (uint64_t p0 = b; p0 < e; p0 += 32 * kScanChunks) {
        uint32_t ys[kScanChunks];
#pragma unroll
        for (int u = 0; u < kScanChunks; u++) {
            uint64_t p = p0 + u * 32 + lane;
            ys[u] = p < e ? adj[p] : 0xffffffffu;
        }
#pragma unroll
        for (int u = 0; u < kScanChunks; u++) {
            const uint32_t y = ys[u];
            if (y > x && y <= cmax) {
                uint32_t pos = (uint32_t)lower_bound_u32(C, nc, y);
                if (pos < nc && C[pos] == y) bits |= 1u << pos;
            }
        }
        if (__shfl_sync(0xffffffffu, ys[kScanChunks - 1], 31) > cmax) break;
    }
    return __reduce_or_sync(0xffffffffu, bits);
}

// Warp builds one-word rows for |C| <= 32 (rows[i] for i < nc).  The last
// candidate's row is empty (no candidate lies above it).
template <class OFF>
__device__ __forceinline__ void warp_build_rows32(const uint32_t* C, uint32_t nc,
                                                  const OFF* ne, const uint32_t* adj,
                                                  const OFF* nb, uint32_t* rows) {
    const unsigned lane = lane_id();
    if (nc == 0) return;
    const uint32_t cmax = C[nc - 1];
    for (uint32_t i = 0; i + 1 < nc; i++) {
        const uint32_t x = C[i];
        const uint32_t bits = warp_row32(C, nc, cmax, x, adj, nb[x], ne[x]);
        if (lane == 0) rows[i] = bits;
    }
    if (lane == 0) rows[nc - 1] = 0;
    __syncwarp();
}

// ---------------------------------------------------------------------------
// Per-candidate credits.  An r-clique listed as positions j1 < ... < jr of C
// adds one to each member's counter.  The last member of a clique is one bit
// of the leaf mask P & rows[j_{r-1}], so it is credited through bit-sliced
// counters held in registers: 32 counters of kSlices bits, counter b being
// bit b of S[0..kSlices-1] (S[0] least significant); adding a mask adds one
// to every counter whose bit is set, by ripple carry.  The counters are
// flushed (one shared-memory atomic per non-zero counter) before any of them
// can reach 2^kSlices.  The other members are credited once per search node
// with the number of cliques below it, instead of once per clique.
constexpr int kSlices = 8;
constexpr uint32_t kSliceAdds = (1u << kSlices) - 1;   // adds between flushes

struct BitSliced {
    uint32_t S[kSlices];
    uint32_t adds;
    __device__ __forceinline__ void clear() {
#pragma unroll
        for (int i = 0; i < kSlices; i++) S[i] = 0;
        adds = 0;
    }
    __device__ __forceinline__ void add(uint32_t m) {
        uint32_t carry = m;
#pragma unroll
        for (int i = 0; i < kSlices; i++) {
            uint32_t t = S[i] & carry;
            S[i] ^= carry;
            carry = t;
            if (!carry) break;
        }
        adds++;
    }
    // cnt[b] += counter b for every b; then zero.
    template <class T>
    __device__ __forceinline__ void flush(T* cnt) {
        uint32_t any = 0;
#pragma unroll
        for (int i = 0; i < kSlices; i++) any |= S[i];
        while (any) {
            int b = __ffs(any) - 1;
            any &= any - 1;
            uint32_t v = 0;
#pragma unroll
            for (int i = 0; i < kSlices; i++) v |= ((S[i] >> b) & 1u) << i;
            atomicAdd(&cnt[b], (T)v);
        }
        clear();
    }
};

// ---------------------------------------------------------------------------
// Warp DFS over one-word rows: lane i takes the cliques whose first member
// is candidate i.  Counts r-cliques (r >= 2) in G[C]; adds per-candidate
// counts into cnt[] (shared memory) and returns the warp total (all lanes).
// A node at depth d has chosen d members (sel[1..d]); P[d] holds the
// candidates adjacent to all of them.  Nodes at depth r - 2 enumerate their
// leaves in one loop.
__device__ __forceinline__ unsigned long long warp_dfs32(const uint32_t* rows, uint32_t nc,
                                                        int r, unsigned* cnt) {
    unsigned lane = lane_id();
    unsigned long long total = 0;
    if (lane < nc) {
        BitSliced bs;
        bs.clear();
        if (r == 2) {
            uint32_t last = rows[lane];
            unsigned c = __popc(last);
            if (c) {
                bs.add(last);
                atomicAdd(&cnt[lane], c);
                total = c;
            }
        } else {
            uint32_t P[kMaxDepth], rem[kMaxDepth], sel[kMaxDepth];
            unsigned acc[kMaxDepth];
            int depth = 1;
            P[1] = rows[lane];
            rem[1] = P[1];
            sel[1] = lane;
            acc[1] = 0;
            // need r - 1 more members after the first
            if (__popc(P[1]) < r - 1) depth = 0;
            while (depth >= 1) {
                if (depth == r - 2) {
                    // every j left in rem is member r-1, its leaf mask the last members
                    uint32_t rm = rem[depth], Pd = P[depth];
                    unsigned sub = 0;
                    while (rm) {
                        int j = __ffs(rm) - 1;
                        rm &= rm - 1;
                        uint32_t last = Pd & rows[j];
                        unsigned c = __popc(last);
                        if (c) {
                            bs.add(last);
                            if (bs.adds == kSliceAdds) bs.flush(cnt);
                            atomicAdd(&cnt[j], c);
                            sub += c;
                        }
                    }
                    acc[depth] += sub;
                } else if (rem[depth]) {
                    int j = __ffs(rem[depth]) - 1;
                    rem[depth] &= rem[depth] - 1;
                    uint32_t pn = P[depth] & rows[j];
                    if (__popc(pn) >= r - depth - 1) {
                        depth++;
                        sel[depth] = j;
                        P[depth] = pn;
                        rem[depth] = pn;
                        acc[depth] = 0;
                    }
                    continue;
                }
                // leave the node: credit its member with the cliques below it
                unsigned a = acc[depth];
                if (a) {
                    atomicAdd(&cnt[sel[depth]], a);
                    if (depth > 1) acc[depth - 1] += a;
                    else total = a;
                }
                depth--;
            }
        }
        bs.flush(cnt);
    }
    return warp_sum(total);
}

// ---------------------------------------------------------------------------
// Block-level bitmap routines for 32 < |C| <= 1024.  rows: nc * W words in
// shared memory (W = ceil(nc/32)), zeroed by the caller.
template <class OFF>
__device__ __forceinline__ void block_build_rows(const uint32_t* C, uint32_t nc, uint32_t W,
                                                 const OFF* ne, const uint32_t* adj,
                                                 const OFF* nb, uint32_t* rows) {
    const unsigned lane = lane_id();
    const unsigned nw = blockDim.x >> 5;
    if (nc == 0) return;
    const uint32_t cmax = C[nc - 1];
    for (uint32_t i = warp_id(); i + 1 < nc; i += nw) {
        const uint32_t x = C[i];
        const uint64_t b = nb[x], e = ne[x];
        for (uint64_t p0 = b; p0 < e; p0 += 32 * kScanChunks) {
            uint32_t ys[kScanChunks];
#pragma unroll
            for (int u = 0; u < kScanChunks; u++) {
                uint64_t p = p0 + u * 32 + lane;
                ys[u] = p < e ? adj[p] : 0xffffffffu;
            }
#pragma unroll
            for (int u = 0; u < kScanChunks; u++) {
                const uint32_t y = ys[u];
                if (y > x && y <= cmax) {
                    uint32_t pos = (uint32_t)lower_bound_u32(C, nc, y);
                    if (pos < nc && C[pos] == y && pos > i)
                        atomicOr(&rows[i * W + (pos >> 5)], 1u << (pos & 31));
                }
            }
            if (__shfl_sync(0xffffffffu, ys[kScanChunks - 1], 31) > cmax) break;
        }
    }
}

// Warps take first members i from the shared counter *next_i (zero on
// entry; the early candidates, with the largest searches below them, go
// first); lane l holds word l of the current sets (and the bit-sliced
// counters of candidates 32 l .. 32 l + 31).  Rows of at most 16 words leave
// lanes idle in the leaf loop, so there the warp takes G = 32 / W2 leaves at
// a time (W2 = W rounded up to a power of two): lane l works on word l % W2
// of leaf l / W2 and keeps the bit-sliced counters of that word.  Returns
// this thread's share of the total (sum over the block = total).
__device__ __forceinline__ unsigned long long block_dfs(const uint32_t* rows, uint32_t nc,
                                                       uint32_t W, int r,
                                                       unsigned long long* cnt,
                                                       uint32_t* next_i) {
    const unsigned full = 0xffffffffu;
    unsigned lane = lane_id();
    unsigned long long total = 0;
    // leaf packing: W2 lanes per leaf, G leaves per step
    uint32_t W2 = 1;
    while (W2 < W) W2 <<= 1;
    const uint32_t G = W2 <= 16 ? 32 / W2 : 1;
    const uint32_t lw = G > 1 ? lane % W2 : lane;   // the word this lane works on
    const uint32_t slot = G > 1 ? lane / W2 : 0;
    BitSliced bs;
    bs.clear();
    for (;;) {
        uint32_t i = 0;
        if (lane == 0) i = atomicAdd(next_i, 1u);
        i = __shfl_sync(full, i, 0);
        if (i >= nc) break;
        uint32_t P[kMaxDepth], rem[kMaxDepth];
        uint32_t sel[kMaxDepth];
        unsigned long long acc[kMaxDepth];
        int depth = 1;
        P[1] = lane < W ? rows[i * W + lane] : 0u;
        rem[1] = P[1];
        sel[1] = i;
        acc[1] = 0;
        unsigned pc = __reduce_add_sync(full, (unsigned)__popc(P[1]));
        if ((int)pc < r - 1) continue;
        if (r == 2) {
            bs.add(G > 1 ? __shfl_sync(full, P[1], lw) * (slot == 0) : P[1]);
            if (bs.adds == kSliceAdds) bs.flush(cnt + lw * 32);
            if (lane == 0) {
                atomicAdd(&cnt[i], (unsigned long long)pc);
                total += pc;
            }
            continue;
        }
        while (depth >= 1) {
            if (depth == r - 2 && G > 1) {
                // packed leaves: slot q of each step takes the q-th next j
                const uint32_t Pw = __shfl_sync(full, P[depth], lw);
                uint32_t rm = rem[depth];
                unsigned long long sub = 0;
                for (;;) {
                    uint32_t myj = 0xffffffffu;
                    uint32_t got = 0;
                    for (uint32_t q = 0; q < G; q++) {
                        const unsigned have = __ballot_sync(full, rm != 0);
                        if (!have) break;
                        const int fl = __ffs(have) - 1;
                        const uint32_t word = __shfl_sync(full, rm, fl);
                        const uint32_t j = (uint32_t)fl * 32 + (__ffs(word) - 1);
                        if ((int)lane == fl) rm &= rm - 1;
                        if (slot == q) myj = j;
                        got++;
                    }
                    if (!got) break;
                    const uint32_t last =
                        (myj != 0xffffffffu && lw < W) ? Pw & rows[myj * W + lw] : 0u;
                    unsigned c = __popc(last);
                    for (uint32_t o = W2 >> 1; o > 0; o >>= 1) c += __shfl_xor_sync(full, c, o);
                    bs.add(last);
                    if (bs.adds == kSliceAdds) bs.flush(cnt + lw * 32);
                    const unsigned lead_c = lw == 0 ? c : 0u;
                    if (lead_c) atomicAdd(&cnt[myj], (unsigned long long)lead_c);
                    sub += __reduce_add_sync(full, lead_c);
                }
                acc[depth] += sub;
            } else if (depth == r - 2) {
                // every j left in rem is member r-1, its leaf mask the last members
                const uint32_t Pd = P[depth];
                uint32_t rm = rem[depth];
                unsigned long long sub = 0;
                for (;;) {
                    unsigned have = __ballot_sync(full, rm != 0);
                    if (!have) break;
                    int fl = __ffs(have) - 1;
                    uint32_t word = __shfl_sync(full, rm, fl);
                    uint32_t j = (uint32_t)fl * 32 + (__ffs(word) - 1);
                    if ((int)lane == fl) rm &= rm - 1;
                    uint32_t last = Pd & (lane < W ? rows[j * W + lane] : 0u);
                    unsigned c = __reduce_add_sync(full, (unsigned)__popc(last));
                    if (c) {
                        bs.add(last);
                        if (bs.adds == kSliceAdds) bs.flush(cnt + lw * 32);
                        if (lane == 0) atomicAdd(&cnt[j], (unsigned long long)c);
                        sub += c;
                    }
                }
                acc[depth] += sub;
            } else {
                unsigned have = __ballot_sync(full, rem[depth] != 0);
                if (have) {
                    int fl = __ffs(have) - 1;
                    uint32_t word = __shfl_sync(full, rem[depth], fl);
                    uint32_t j = (uint32_t)fl * 32 + (__ffs(word) - 1);
                    if ((int)lane == fl) rem[depth] &= rem[depth] - 1;
                    uint32_t pn = P[depth] & (lane < W ? rows[j * W + lane] : 0u);
                    int c = (int)__reduce_add_sync(full, (unsigned)__popc(pn));
                    if (c >= r - depth - 1) {
                        depth++;
                        sel[depth] = j;
                        P[depth] = pn;
                        rem[depth] = pn;
                        acc[depth] = 0;
                    }
                    continue;
                }
            }
            // leave the node: credit its member with the cliques below it
            unsigned long long a = acc[depth];
            if (a) {
                if (lane == 0) atomicAdd(&cnt[sel[depth]], a);
                if (depth > 1) acc[depth - 1] += a;
                else total += a;
            }
            depth--;
        }
    }
    bs.flush(cnt + lw * 32);
    return lane == 0 ? total : 0ull;
}

}  // namespace dsd
