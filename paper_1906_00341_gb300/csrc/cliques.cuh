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

// Warp builds one-word rows for |C| <= 32 (rows[i] for i < nc).
template <class OFF>
__device__ __forceinline__ void warp_build_rows32(const uint32_t* C, uint32_t nc,
                                                  const OFF* ne, const uint32_t* adj,
                                                  const OFF* nb, uint32_t* rows) {
    unsigned lane = lane_id();
    for (uint32_t i = 0; i < nc; i++) {
        uint32_t x = C[i];
        uint64_t b = nb[x], e = ne[x];
        uint32_t bits = 0;
        for (uint64_t p = b + lane; p - lane < e; p += 32) {
            bool hit = false;
            uint32_t pos = 0;
            if (p < e) {
                uint32_t y = adj[p];
                if (y > x) {
                    pos = (uint32_t)lower_bound_u32(C, nc, y);
                    hit = pos < nc && C[pos] == y;
                }
            }
            bits |= __reduce_or_sync(0xffffffffu, hit ? (1u << pos) : 0u);
        }
        if (lane == 0) rows[i] = bits;
    }
    __syncwarp();
}

// ---------------------------------------------------------------------------
// Warp DFS over one-word rows: lane i takes the cliques whose first member
// is candidate i.  Counts r-cliques (r >= 2) in G[C]; adds per-candidate
// counts into cnt[] (shared memory) and returns the warp total (all lanes).
__device__ __forceinline__ unsigned long long warp_dfs32(const uint32_t* rows, uint32_t nc,
                                                        int r, unsigned* cnt) {
    unsigned lane = lane_id();
    unsigned long long total = 0;
    if (lane < nc) {
        uint32_t P[kMaxDepth], rem[kMaxDepth];
        uint32_t sel[kMaxDepth];
        int depth = 1;
        P[1] = rows[lane];
        rem[1] = P[1];
        sel[1] = lane;
        // need r - 1 more members after the first
        if (__popc(P[1]) >= r - 1) {
            while (depth >= 1) {
                if (depth == r - 1) {
                    uint32_t last = P[depth];
                    unsigned c = __popc(last);
                    if (c) {
                        total += c;
                        for (int d = 1; d <= depth; d++) atomicAdd(&cnt[sel[d]], c);
                        while (last) {
                            int b = __ffs(last) - 1;
                            last &= last - 1;
                            atomicAdd(&cnt[b], 1u);
                        }
                    }
                    depth--;
                    continue;
                }
                if (rem[depth] == 0) { depth--; continue; }
                int j = __ffs(rem[depth]) - 1;
                rem[depth] &= rem[depth] - 1;
                uint32_t pn = P[depth] & rows[j];
                if (__popc(pn) < r - depth - 1) continue;
                depth++;
                sel[depth] = j;
                P[depth] = pn;
                rem[depth] = pn;
            }
        }
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
    unsigned lane = lane_id();
    unsigned nw = blockDim.x >> 5;
    for (uint32_t i = warp_id(); i < nc; i += nw) {
        uint32_t x = C[i];
        uint64_t b = nb[x], e = ne[x];
        for (uint64_t p = b + lane; p < e; p += 32) {
            uint32_t y = adj[p];
            uint32_t pos = (uint32_t)lower_bound_u32(C, nc, y);
            if (pos < nc && C[pos] == y && pos > i)
                atomicOr(&rows[i * W + (pos >> 5)], 1u << (pos & 31));
        }
    }
}

// Warps take first members i; lane l holds word l of the current sets.
// Returns this thread's share of the total (sum over the block = total).
__device__ __forceinline__ unsigned long long block_dfs(const uint32_t* rows, uint32_t nc,
                                                       uint32_t W, int r,
                                                       unsigned long long* cnt) {
    unsigned lane = lane_id();
    unsigned nw = blockDim.x >> 5;
    unsigned long long total = 0;
    for (uint32_t i = warp_id(); i < nc; i += nw) {
        uint32_t P[kMaxDepth], rem[kMaxDepth];
        uint32_t sel[kMaxDepth];
        int depth = 1;
        P[1] = lane < W ? rows[i * W + lane] : 0u;
        rem[1] = P[1];
        sel[1] = i;
        int pc = __reduce_add_sync(0xffffffffu, (unsigned)__popc(P[1]));
        if (pc < r - 1) continue;
        while (depth >= 1) {
            if (depth == r - 1) {
                uint32_t last = P[depth];
                unsigned c = __reduce_add_sync(0xffffffffu, (unsigned)__popc(last));
                if (c) {
                    if (lane == 0) {
                        total += c;
                        for (int d = 1; d <= depth; d++)
                            atomicAdd(&cnt[sel[d]], (unsigned long long)c);
                    }
                    while (last) {
                        int b = __ffs(last) - 1;
                        last &= last - 1;
                        atomicAdd(&cnt[lane * 32 + b], 1ull);
                    }
                }
                depth--;
                continue;
            }
            unsigned have = __ballot_sync(0xffffffffu, rem[depth] != 0);
            if (!have) { depth--; continue; }
            int fl = __ffs(have) - 1;
            uint32_t word = __shfl_sync(0xffffffffu, rem[depth], fl);
            int bit = __ffs(word) - 1;
            uint32_t j = (uint32_t)fl * 32 + bit;
            if ((int)lane == fl) rem[depth] &= rem[depth] - 1;
            uint32_t pn = P[depth] & (lane < W ? rows[j * W + lane] : 0u);
            int c = __reduce_add_sync(0xffffffffu, (unsigned)__popc(pn));
            if (c < r - depth - 1) continue;
            depth++;
            sel[depth] = j;
            P[depth] = pn;
            rem[depth] = pn;
        }
    }
    return total;
}

}  // namespace dsd
