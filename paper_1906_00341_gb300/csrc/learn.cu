// The learned proposal.
//
// Not in the paper.  A small MLP reads 64 statistics of a graph and proposes
// rho', meant as a lower bound of the optimal h-clique density (Problem 1).
// The seeded path (seeded.cu) then extracts only the (ceil(rho'),Psi)-core: by
// Lemma 5 and the level-density argument the CoreApp outputs at or above
// that level are unchanged, and a proposal that fails the exact acceptance
// test falls back to the full decomposition, so the network can only cost
// time, never change an answer.
//
// Everything here is hand-written CUDA:
//   * k_feat_*   -- the 64 statistics (degree and edge-core histograms,
//                   and sampled clustering and clique-count estimates inside
//                   three nested edge cores), FP32;
//   * k_lin_*    -- dense layers Y = act(X W + b) with BF16 weights and FP32
//                   accumulation, their input and weight gradients;
//   * k_pinball  -- quantile (pinball) loss and its gradient;
//   * k_adam     -- Adam on FP32 master weights, refreshing the BF16 copy.
// The network is 64 -> 256 -> 256 -> 256 -> 1 with ReLU (148,481 parameters).
// Its GEMMs are 256 x 256 x 256 at most (about 33 MFLOP per batch of 256):
// launch-bound, so they run on CUDA cores with shared-memory tiles rather
// than tensor-core pipelines.
#include "graph.cuh"

#include <cuda_bf16.h>
#include <math.h>
#include <new>
#include <string.h>

struct dsd_model {
    float* master = nullptr;          // FP32 parameters
    __nv_bfloat16* w16 = nullptr;     // BF16 copy used by the forward pass
    float* grad = nullptr;
    float* adam_m = nullptr;
    float* adam_v = nullptr;
    float* act = nullptr;             // activations, B_MAX x (64 + 3*256 + 1)
    float* dact = nullptr;            // their gradients
    float* y = nullptr;               // labels
    float* loss = nullptr;            // [1]
    uint64_t step = 0;
    cudaStream_t stream = nullptr;
};

namespace dsd {

constexpr int kFeat = 64;
constexpr int kHid = 256;
constexpr uint32_t kBMax = 1024;
// parameter layout: W1 [64x256], b1, W2 [256x256], b2, W3, b3, W4 [256x1], b4
constexpr size_t kOffW1 = 0;
constexpr size_t kOffB1 = kOffW1 + (size_t)kFeat * kHid;
constexpr size_t kOffW2 = kOffB1 + kHid;
constexpr size_t kOffB2 = kOffW2 + (size_t)kHid * kHid;
constexpr size_t kOffW3 = kOffB2 + kHid;
constexpr size_t kOffB3 = kOffW3 + (size_t)kHid * kHid;
constexpr size_t kOffW4 = kOffB3 + kHid;
constexpr size_t kOffB4 = kOffW4 + kHid;
constexpr size_t kNParams = kOffB4 + 1;
// activation layout per sample: x (64) | h1 (256) | h2 (256) | h3 (256) | out (1)
constexpr size_t kActW = kFeat + 3 * kHid + 1;

namespace {

// --------------------------------------------------------- dense layers
constexpr int kTile = 32;

// Y[b, o] = act(sum_i X[b, i] W[i, o] + bias[o]); X rows of stride ldx,
// Y rows of stride ldy.  One 32x32 output tile per block, 32x8 threads.
template <bool RELU>
__global__ void k_lin_fwd(const float* X, int ldx, const __nv_bfloat16* W, const float* bias,
                          float* Y, int ldy, int B, int I, int O) {
    __shared__ float sx[kTile][kTile + 1];
    __shared__ float sw[kTile][kTile + 1];
    int tx = threadIdx.x, ty = threadIdx.y;   // 32 x 8
    int row0 = blockIdx.y * kTile, col0 = blockIdx.x * kTile;
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    for (int k0 = 0; k0 < I; k0 += kTile) {
        for (int r = ty; r < kTile; r += 8) {
            int b = row0 + r, i = k0 + tx;
            sx[r][tx] = (b < B && i < I) ? X[(size_t)b * ldx + i] : 0.f;
            int ii = k0 + r, o = col0 + tx;
            sw[r][tx] = (ii < I && o < O) ? __bfloat162float(W[(size_t)ii * O + o]) : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < kTile; kk++) {
            float w = sw[kk][tx];
#pragma unroll
            for (int q = 0; q < 4; q++) acc[q] += sx[ty + 8 * q][kk] * w;
        }
        __syncthreads();
    }
    int o = col0 + tx;
    if (o < O)
#pragma unroll
        for (int q = 0; q < 4; q++) {
            int b = row0 + ty + 8 * q;
            if (b < B) {
                float v = acc[q] + bias[o];
                Y[(size_t)b * ldy + o] = RELU ? fmaxf(v, 0.f) : v;
            }
        }
}

// dX[b, i] = (sum_o dY[b, o] W[i, o]) * (relu mask of Xact[b, i] if MASK)
template <bool MASK>
__global__ void k_lin_bwd_x(const float* dY, int ldy, const __nv_bfloat16* W, const float* Xact,
                            int ldx, float* dX, int B, int I, int O) {
    __shared__ float sd[kTile][kTile + 1];
    __shared__ float sw[kTile][kTile + 1];
    int tx = threadIdx.x, ty = threadIdx.y;
    int row0 = blockIdx.y * kTile, col0 = blockIdx.x * kTile;   // cols over I
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    for (int k0 = 0; k0 < O; k0 += kTile) {
        for (int r = ty; r < kTile; r += 8) {
            int b = row0 + r, o = k0 + tx;
            sd[r][tx] = (b < B && o < O) ? dY[(size_t)b * ldy + o] : 0.f;
            int i = col0 + r, oo = k0 + tx;   // sw[i_local][o_local] = W[i, o]
            sw[r][tx] = (i < I && oo < O) ? __bfloat162float(W[(size_t)i * O + oo]) : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < kTile; kk++) {
            float w = sw[tx][kk];
#pragma unroll
            for (int q = 0; q < 4; q++) acc[q] += sd[ty + 8 * q][kk] * w;
        }
        __syncthreads();
    }
    int i = col0 + tx;
    if (i < I)
#pragma unroll
        for (int q = 0; q < 4; q++) {
            int b = row0 + ty + 8 * q;
            if (b < B) {
                float v = acc[q];
                if (MASK && Xact[(size_t)b * ldx + i] <= 0.f) v = 0.f;
                dX[(size_t)b * ldx + i] = v;
            }
        }
}

// dW[i, o] = sum_b X[b, i] dY[b, o]; db[o] = sum_b dY[b, o]  (overwrite)
__global__ void k_lin_bwd_w(const float* X, int ldx, const float* dY, int ldy, float* dW,
                            float* db, int B, int I, int O) {
    __shared__ float sx[kTile][kTile + 1];
    __shared__ float sd[kTile][kTile + 1];
    int tx = threadIdx.x, ty = threadIdx.y;
    int i0 = blockIdx.y * kTile, o0 = blockIdx.x * kTile;
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    float bacc = 0.f;
    for (int b0 = 0; b0 < B; b0 += kTile) {
        for (int r = ty; r < kTile; r += 8) {
            int b = b0 + r;
            sx[r][tx] = (b < B && i0 + tx < I) ? X[(size_t)b * ldx + i0 + tx] : 0.f;
            sd[r][tx] = (b < B && o0 + tx < O) ? dY[(size_t)b * ldy + o0 + tx] : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int bb = 0; bb < kTile; bb++) {
            float d = sd[bb][tx];
#pragma unroll
            for (int q = 0; q < 4; q++) acc[q] += sx[bb][ty + 8 * q] * d;
            if (ty == 0) bacc += d;
        }
        __syncthreads();
    }
    int o = o0 + tx;
    if (o < O) {
#pragma unroll
        for (int q = 0; q < 4; q++) {
            int i = i0 + ty + 8 * q;
            if (i < I) dW[(size_t)i * O + o] = acc[q];
        }
        if (ty == 0 && blockIdx.y == 0) db[o] = bacc;
    }
}

// Pinball loss L = mean_b rho_q(y_b - p_b), rho_q(u) = u (q - [u < 0]);
// dL/dp_b = -(q - [y_b < p_b]) / B.
__global__ void k_pinball(const float* pred, int ldp, const float* y, int B, float q,
                          float* dpred, float* loss) {
    __shared__ float s[32];
    float acc = 0.f;
    for (int b = threadIdx.x; b < B; b += blockDim.x) {
        float p = pred[(size_t)b * ldp];
        float u = y[b] - p;
        float ind = u < 0.f ? 1.f : 0.f;
        acc += u * (q - ind);
        dpred[(size_t)b * ldp] = -(q - ind) / (float)B;
    }
    acc = warp_sum(acc);
    if (lane_id() == 0) s[warp_id()] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) t += s[w];
        *loss = t / (float)B;
    }
}

__global__ void k_adam(float* w, const float* g, float* m, float* v, __nv_bfloat16* w16, size_t n,
                       float lr, float b1, float b2, float eps, float c1, float c2) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x) {
        float gi = g[i];
        float mi = b1 * m[i] + (1.f - b1) * gi;
        float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
        w[i] = wi;
        w16[i] = __float2bfloat16(wi);
    }
}

__global__ void k_to_bf16(const float* w, __nv_bfloat16* w16, size_t n) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x)
        w16[i] = __float2bfloat16(w[i]);
}

// Deterministic initialisation: uniform(-a, a) with a = sqrt(6 / fan_in)
// (He-uniform) from a counter-based hash of (seed, index); biases 0.
__device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__global__ void k_init(float* w, size_t n, uint64_t seed) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x) {
        float fan_in = 0.f;
        bool bias = false;
        if (i < kOffB1) fan_in = kFeat;
        else if (i < kOffW2) bias = true;
        else if (i < kOffB2) fan_in = kHid;
        else if (i < kOffW3) bias = true;
        else if (i < kOffB3) fan_in = kHid;
        else if (i < kOffW4) bias = true;
        else if (i < kOffB4) fan_in = kHid;
        else bias = true;
        if (bias) {
            w[i] = 0.f;
            continue;
        }
        uint64_t r = mix64(seed ^ mix64(i));
        float u = (float)((r >> 40) * (1.0 / 16777216.0));   // [0, 1)
        float a = sqrtf(6.f / fan_in);
        w[i] = (2.f * u - 1.f) * a;
    }
}

dsd_status launch_forward(dsd_model* M, int B) {
    cudaStream_t s = M->stream;
    float* x = M->act;
    float* h1 = x + kFeat;
    float* h2 = h1 + kHid;
    float* h3 = h2 + kHid;
    float* out = h3 + kHid;
    dim3 thr(32, 8);
    dim3 g1(kHid / kTile, (B + kTile - 1) / kTile);
    const __nv_bfloat16* W = M->w16;
    const float* P = M->master;
    k_lin_fwd<true><<<g1, thr, 0, s>>>(x, kActW, W + kOffW1, P + kOffB1, h1, kActW, B, kFeat, kHid);
    k_lin_fwd<true><<<g1, thr, 0, s>>>(h1, kActW, W + kOffW2, P + kOffB2, h2, kActW, B, kHid, kHid);
    k_lin_fwd<true><<<g1, thr, 0, s>>>(h2, kActW, W + kOffW3, P + kOffB3, h3, kActW, B, kHid, kHid);
    dim3 g4(1, (B + kTile - 1) / kTile);
    k_lin_fwd<false><<<g4, thr, 0, s>>>(h3, kActW, W + kOffW4, P + kOffB4, out, kActW, B, kHid, 1);
    for (int i = 0; i < 4; i++) note_launch();
    DSD_LAUNCHED();
    return DSD_OK;
}

// Loss and parameter gradients for the batch already in act / y.
dsd_status launch_backward(dsd_model* M, int B, float q) {
    cudaStream_t s = M->stream;
    float* x = M->act;
    float* h1 = x + kFeat;
    float* h2 = h1 + kHid;
    float* h3 = h2 + kHid;
    float* out = h3 + kHid;
    float* dx = M->dact;
    float* dh1 = dx + kFeat;
    float* dh2 = dh1 + kHid;
    float* dh3 = dh2 + kHid;
    float* dout = dh3 + kHid;
    float* G = M->grad;
    const __nv_bfloat16* W = M->w16;
    dim3 thr(32, 8);
    k_pinball<<<1, 1024, 0, s>>>(out, kActW, M->y, B, q, dout, M->loss);
    dim3 gw4(1, kHid / kTile);
    k_lin_bwd_w<<<gw4, thr, 0, s>>>(h3, kActW, dout, kActW, G + kOffW4, G + kOffB4, B, kHid, 1);
    dim3 gx(kHid / kTile, (B + kTile - 1) / kTile);
    k_lin_bwd_x<true><<<gx, thr, 0, s>>>(dout, kActW, W + kOffW4, h3, kActW, dh3, B, kHid, 1);
    dim3 gw(kHid / kTile, kHid / kTile);
    k_lin_bwd_w<<<gw, thr, 0, s>>>(h2, kActW, dh3, kActW, G + kOffW3, G + kOffB3, B, kHid, kHid);
    k_lin_bwd_x<true><<<gx, thr, 0, s>>>(dh3, kActW, W + kOffW3, h2, kActW, dh2, B, kHid, kHid);
    k_lin_bwd_w<<<gw, thr, 0, s>>>(h1, kActW, dh2, kActW, G + kOffW2, G + kOffB2, B, kHid, kHid);
    k_lin_bwd_x<true><<<gx, thr, 0, s>>>(dh2, kActW, W + kOffW2, h1, kActW, dh1, B, kHid, kHid);
    dim3 gw1(kHid / kTile, kFeat / kTile);
    k_lin_bwd_w<<<gw1, thr, 0, s>>>(x, kActW, dh1, kActW, G + kOffW1, G + kOffB1, B, kFeat, kHid);
    for (int i = 0; i < 8; i++) note_launch();
    DSD_LAUNCHED();
    return DSD_OK;
}

// ------------------------------------------------------------ features
//
// Three nested vertex sets are sampled: C_0 = V, C_1 = {core_2 >= degen/2}
// and C_2 = {core_2 = degen} (degen = the degeneracy).  Ranks order vertices
// by their removal round in the h = 2 peel, and core_2 does not decrease with
// the round, so each C_g is a suffix [r_g, n) of the rank order, and in the
// relabelled CSR (rows sorted by rank) the neighbours of v inside C_g are the
// tail of row v from r_g on.  For kSamples vertices v of each C_g (hashed
// ranks) a warp draws 32 pairs of C_g-neighbours and tests them for an edge:
// the closed fraction c estimates the local clustering inside C_g; with
// d = |N(v) ∩ C_g|, c C(d,2) estimates v's triangle count and
// c^C(h-1,2) C(d,h-1) its h-clique count in G[C_g] (exact on cliques, 0 on
// triangle-free graphs).  Per-sample records are reduced in a fixed order,
// so the statistics are deterministic.

constexpr uint32_t kSamples = 4096;
constexpr int kGroups = 3;

struct FeatAcc {
    unsigned int deg_hist[16];
    unsigned int core_hist[16];
    unsigned int dmax;
    unsigned int cnt[kGroups];   // |C_g|
};

struct FeatRec {
    float d;        // |N(v) ∩ C_g|
    float c;        // closed fraction of the sampled pairs
    float tri;      // estimated triangles at v inside C_g
    float lclq;     // log1p(estimated h-cliques at v inside C_g)
};

__device__ __forceinline__ int bucket16(uint64_t x) {
    int b = 0;
    uint64_t y = x + 1;
    while (y > 1 && b < 15) {
        y >>= 1;
        b++;
    }
    return b;
}

__global__ void k_feat_hist(uint32_t n, const uint64_t* off, const uint64_t* core2,
                            uint32_t degen, FeatAcc* A) {
    __shared__ unsigned int sd[16], sc[16];
    if (threadIdx.x < 16) {
        sd[threadIdx.x] = 0;
        sc[threadIdx.x] = 0;
    }
    __syncthreads();
    unsigned int dmax = 0, top = 0, half = 0;
    for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n;
         v += (uint64_t)gridDim.x * blockDim.x) {
        uint64_t d = off[v + 1] - off[v];
        uint64_t c = core2[v];
        atomicAdd(&sd[bucket16(d)], 1u);
        atomicAdd(&sc[bucket16(c)], 1u);
        dmax = d > dmax ? (unsigned)d : dmax;
        if (c == degen) top++;
        if (2 * c >= degen) half++;
    }
    __syncthreads();
    if (threadIdx.x < 16) {
        atomicAdd(&A->deg_hist[threadIdx.x], sd[threadIdx.x]);
        atomicAdd(&A->core_hist[threadIdx.x], sc[threadIdx.x]);
    }
    atomicMax(&A->dmax, dmax);
    atomicAdd(&A->cnt[1], half);
    atomicAdd(&A->cnt[2], top);
}

__device__ __forceinline__ bool has_edge(const uint64_t* off, const uint32_t* adj, uint32_t a,
                                         uint32_t b) {
    uint64_t s = off[a], len = off[a + 1] - s;
    uint64_t p = lower_bound_u32(adj + s, len, b);
    return p < len && adj[s + p] == b;
}

// One warp per (group, sample); rec[g * kSamples + i].
__global__ void k_feat_sample(uint32_t n, const uint64_t* roff, const uint32_t* radj, int h,
                              uint64_t seed, const FeatAcc* A, FeatRec* rec) {
    unsigned lane = lane_id();
    uint64_t gw = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t t = gw; t < (uint64_t)kGroups * kSamples; t += nw) {
        int grp = (int)(t / kSamples);
        uint64_t sidx = t % kSamples;
        uint32_t size = grp == 0 ? n : A->cnt[grp];
        FeatRec r = {0.f, 0.f, 0.f, 0.f};
        if (size > 0) {
            uint32_t r0 = n - size;
            uint64_t z = mix64(seed ^ mix64(t * 0x2545F4914F6CDD1Dull));
            uint32_t v = r0 + (uint32_t)(z % size);
            uint64_t b = roff[v], len = roff[v + 1] - b;
            uint64_t first = lower_bound_u32(radj + b, len, r0);
            uint64_t d = len - first;
            b += first;
            r.d = (float)d;
            if (d >= 2) {
                uint64_t q = mix64(seed + 7919ull * t + 104729ull * lane);
                uint32_t i = (uint32_t)(q % d), j = (uint32_t)((q >> 32) % (d - 1));
                if (j >= i) j++;
                bool closed = has_edge(roff, radj, radj[b + i], radj[b + j]);
                unsigned cn = __popc(__ballot_sync(0xffffffffu, closed));
                float c = (float)cn / 32.f;
                float dd = (float)d;
                r.c = c;
                r.tri = c * dd * (dd - 1.f) * 0.5f;
                float lc = 0.f;   // log C(d, h-1)
                for (int k = 0; k < h - 1; k++) lc += logf(fmaxf(dd - k, 1.f)) - logf((float)(k + 1));
                if (dd < (float)(h - 1)) lc = -1e30f;
                float pe = (float)((h - 1) * (h - 2) / 2);
                float l = lc + (pe > 0.f ? (c > 0.f ? pe * logf(c) : -1e30f) : 0.f);
                r.lclq = l > -50.f ? log1pf(expf(fminf(l, 80.f))) : 0.f;
            }
        }
        if (lane == 0) rec[t] = r;
    }
}

// One warp per group reduces its records in a fixed order; thread 0 of the
// block then writes the 64 statistics.
__global__ void k_feat_final(uint32_t n, uint64_t m, uint32_t degen, int h, const FeatAcc* A,
                             const FeatRec* rec, float* f) {
    __shared__ float red[kGroups][8];
    int w = threadIdx.x >> 5;
    unsigned lane = lane_id();
    if (w < kGroups) {
        float sd = 0.f, sc = 0.f, stri = 0.f, sclq = 0.f, sl = 0.f, mx = 0.f, ok = 0.f;
        for (uint32_t i = lane; i < kSamples; i += 32) {
            FeatRec r = rec[(size_t)w * kSamples + i];
            sd += r.d;
            sc += r.c;
            stri += r.tri;
            sclq += expm1f(fminf(r.lclq, 80.f));
            sl += r.lclq;
            mx = fmaxf(mx, r.lclq);
            ok += r.d >= (float)(h - 1) ? 1.f : 0.f;
        }
        sd = warp_sum(sd);
        sc = warp_sum(sc);
        stri = warp_sum(stri);
        sclq = warp_sum(sclq);
        sl = warp_sum(sl);
        ok = warp_sum(ok);
        for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if (lane == 0) {
            float S = (float)kSamples;
            red[w][0] = sd / S;
            red[w][1] = sc / S;
            red[w][2] = stri / S;
            red[w][3] = sclq / S;
            red[w][4] = sl / S;
            red[w][5] = mx;
            red[w][6] = ok / S;
        }
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    for (int i = 0; i < kFeat; i++) f[i] = 0.f;
    float fn = (float)n, fm = (float)m;
    f[0] = log1pf(fn);
    f[1] = log1pf(fm);
    f[2] = log1pf((float)A->dmax);
    f[3] = log1pf((float)degen);
    f[4] = (float)h * 0.25f;
    f[5] = log1pf(n ? 2.f * fm / fn : 0.f);
    float lc = 0.f;
    for (int t = 0; t < h - 1; t++) lc += logf(fmaxf((float)degen - t, 1.f)) - logf((float)(t + 1));
    f[6] = (float)degen >= (float)(h - 1) ? log1pf(expf(fminf(lc, 80.f))) : 0.f;  // C(degen, h-1)
    f[7] = log1pf((float)A->cnt[2]);
    for (int i = 0; i < 16; i++) {
        f[8 + i] = n ? (float)A->deg_hist[i] / fn : 0.f;
        f[24 + i] = n ? (float)A->core_hist[i] / fn : 0.f;
    }
    for (int g = 0; g < kGroups; g++) {
        float size = g == 0 ? fn : (float)A->cnt[g];
        float* o = f + 40 + 8 * g;
        o[0] = log1pf(size);
        o[1] = log1pf(red[g][0]);                  // mean degree inside C_g
        o[2] = red[g][1];                          // mean closed fraction
        o[3] = log1pf(red[g][2]);                  // mean triangles at a vertex
        o[4] = log1pf(red[g][3]);                  // mean h-cliques at a vertex
        o[5] = log1pf(red[g][3] / (float)h);       // h-clique density estimate of G[C_g]
        o[6] = red[g][4];                          // mean log1p(h-cliques at a vertex)
        o[7] = red[g][5];                          // max of the same
    }
}

}  // namespace

dsd_status compute_features(dsd_graph* g, int h, float* f_dev) {
    DSD_TRY(ensure_order(g));
    cudaStream_t s = g->stream;
    FeatAcc* A = nullptr;
    FeatRec* rec = nullptr;
    DSD_TRY(dalloc(&A, 1, s));
    dsd_status st = dalloc(&rec, (size_t)kGroups * kSamples, s);
    if (st != DSD_OK) {
        dev_free(A, s);
        return st;
    }
    int sms = 152;
    num_sms(&sms);
    cudaError_t e = cudaMemsetAsync(A, 0, sizeof(FeatAcc), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(rec, 0, sizeof(FeatRec) * kGroups * kSamples, s);
    if (e == cudaSuccess && g->n) {
        k_feat_hist<<<sms * 4, 256, 0, s>>>(g->n, g->off, g->core2, g->degeneracy, A);
        k_feat_sample<<<sms * 4, 256, 0, s>>>(g->n, g->roff, g->radj, h, 0x5EEDull, A, rec);
        note_launch();
        note_launch();
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        k_feat_final<<<1, 32 * kGroups, 0, s>>>(g->n, g->m, g->degeneracy, h, A, rec, f_dev);
        note_launch();
        e = cudaGetLastError();
    }
    dev_free(A, s);
    dev_free(rec, s);
    if (e != cudaSuccess) return cuda_fail(e, "features", __FILE__, __LINE__);
    return DSD_OK;
}

// rho' = expm1(network output) for one feature vector (device), written to
// *rho_dev (device float).
dsd_status model_propose(dsd_model* M, const float* f_dev, float* rho_dev, cudaStream_t s);

}  // namespace dsd

using namespace dsd;

namespace dsd {
namespace {
__global__ void k_expm1_out(const float* out, float* rho) {
    float o = *out;
    *rho = fmaxf(expm1f(o), 0.f);
}
}  // namespace

dsd_status model_propose(dsd_model* M, const float* f_dev, float* rho_dev, cudaStream_t s) {
    cudaStream_t keep = M->stream;
    M->stream = s;
    DSD_CU(cudaMemcpyAsync(M->act, f_dev, kFeat * sizeof(float), cudaMemcpyDeviceToDevice, s));
    dsd_status st = launch_forward(M, 1);
    if (st == DSD_OK) {
        k_expm1_out<<<1, 1, 0, s>>>(M->act + kFeat + 3 * kHid, rho_dev);
        note_launch();
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) st = cuda_fail(e, "propose", __FILE__, __LINE__);
    }
    M->stream = keep;
    return st;
}
}  // namespace dsd

extern "C" {

uint64_t dsd_model_param_count(void) { return kNParams; }

dsd_status dsd_model_create(uint64_t seed, void* cuda_stream, dsd_model** out) {
    set_error("");
    if (!out) return DSD_ERR_INVALID;
    *out = nullptr;
    dsd_model* M = new (std::nothrow) dsd_model();
    if (!M) return DSD_ERR_NOMEM;
    M->stream = (cudaStream_t)cuda_stream;
    cudaStream_t s = M->stream;
    dsd_status st = DSD_OK;
    if ((st = dalloc(&M->master, kNParams, s)) == DSD_OK &&
        (st = dalloc(&M->w16, kNParams, s)) == DSD_OK &&
        (st = dalloc(&M->grad, kNParams, s)) == DSD_OK &&
        (st = dalloc(&M->adam_m, kNParams, s)) == DSD_OK &&
        (st = dalloc(&M->adam_v, kNParams, s)) == DSD_OK &&
        (st = dalloc(&M->act, (size_t)kBMax * kActW, s)) == DSD_OK &&
        (st = dalloc(&M->dact, (size_t)kBMax * kActW, s)) == DSD_OK &&
        (st = dalloc(&M->y, kBMax, s)) == DSD_OK && (st = dalloc(&M->loss, 1, s)) == DSD_OK) {
        k_init<<<64, 256, 0, s>>>(M->master, kNParams, seed);
        k_to_bf16<<<64, 256, 0, s>>>(M->master, M->w16, kNParams);
        note_launch();
        note_launch();
        cudaError_t e = cudaMemsetAsync(M->adam_m, 0, kNParams * 4, s);
        if (e == cudaSuccess) e = cudaMemsetAsync(M->adam_v, 0, kNParams * 4, s);
        if (e == cudaSuccess) e = cudaMemsetAsync(M->act, 0, (size_t)kBMax * kActW * 4, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) st = cuda_fail(e, "model init", __FILE__, __LINE__);
    }
    if (st != DSD_OK) {
        dsd_model_destroy(M);
        return st;
    }
    *out = M;
    return DSD_OK;
}

void dsd_model_destroy(dsd_model* M) {
    if (!M) return;
    cudaStream_t s = M->stream;
    void* ptrs[] = {M->master, M->w16, M->grad, M->adam_m, M->adam_v, M->act, M->dact, M->y, M->loss};
    for (void* p : ptrs) dev_free(p, s);
    cudaStreamSynchronize(s);
    delete M;
}

// Parameters and Adam state in host memory (FP32): params, m, v, then the
// step count in the last entry of `state` (size 3 * count + 1).
dsd_status dsd_model_get_state(dsd_model* M, float* state, uint64_t count) {
    if (!M || !state || count != kNParams) return DSD_ERR_INVALID;
    cudaStream_t s = M->stream;
    DSD_CU(cudaMemcpyAsync(state, M->master, kNParams * 4, cudaMemcpyDeviceToHost, s));
    DSD_CU(cudaMemcpyAsync(state + kNParams, M->adam_m, kNParams * 4, cudaMemcpyDeviceToHost, s));
    DSD_CU(cudaMemcpyAsync(state + 2 * kNParams, M->adam_v, kNParams * 4, cudaMemcpyDeviceToHost, s));
    DSD_CU(cudaStreamSynchronize(s));
    state[3 * kNParams] = (float)M->step;
    return DSD_OK;
}

dsd_status dsd_model_set_state(dsd_model* M, const float* state, uint64_t count) {
    if (!M || !state || count != kNParams) return DSD_ERR_INVALID;
    cudaStream_t s = M->stream;
    DSD_CU(cudaMemcpyAsync(M->master, state, kNParams * 4, cudaMemcpyHostToDevice, s));
    DSD_CU(cudaMemcpyAsync(M->adam_m, state + kNParams, kNParams * 4, cudaMemcpyHostToDevice, s));
    DSD_CU(cudaMemcpyAsync(M->adam_v, state + 2 * kNParams, kNParams * 4, cudaMemcpyHostToDevice, s));
    k_to_bf16<<<64, 256, 0, s>>>(M->master, M->w16, kNParams);
    note_launch();
    DSD_LAUNCHED();
    DSD_CU(cudaStreamSynchronize(s));
    M->step = (uint64_t)state[3 * kNParams];
    return DSD_OK;
}

// Forward pass: X [B x 64] (host), out [B] (host) = network output.
dsd_status dsd_model_forward(dsd_model* M, const float* X, uint32_t B, float* out) {
    if (!M || !X || !out || B == 0 || B > kBMax) return DSD_ERR_INVALID;
    cudaStream_t s = M->stream;
    DSD_CU(cudaMemcpy2DAsync(M->act, kActW * 4, X, kFeat * 4, kFeat * 4, B, cudaMemcpyHostToDevice, s));
    DSD_TRY(launch_forward(M, (int)B));
    DSD_CU(cudaMemcpy2DAsync(out, 4, M->act + kFeat + 3 * kHid, kActW * 4, 4, B,
                             cudaMemcpyDeviceToHost, s));
    DSD_CU(cudaStreamSynchronize(s));
    return DSD_OK;
}

// Loss and gradients (no update): grad [param_count] (host, may be NULL).
dsd_status dsd_model_gradient(dsd_model* M, const float* X, const float* y, uint32_t B, float q,
                              float* loss, float* grad) {
    if (!M || !X || !y || B == 0 || B > kBMax) return DSD_ERR_INVALID;
    cudaStream_t s = M->stream;
    DSD_CU(cudaMemcpy2DAsync(M->act, kActW * 4, X, kFeat * 4, kFeat * 4, B, cudaMemcpyHostToDevice, s));
    DSD_CU(cudaMemcpyAsync(M->y, y, B * 4, cudaMemcpyHostToDevice, s));
    DSD_TRY(launch_forward(M, (int)B));
    DSD_TRY(launch_backward(M, (int)B, q));
    if (loss) DSD_CU(cudaMemcpyAsync(loss, M->loss, 4, cudaMemcpyDeviceToHost, s));
    if (grad) DSD_CU(cudaMemcpyAsync(grad, M->grad, kNParams * 4, cudaMemcpyDeviceToHost, s));
    DSD_CU(cudaStreamSynchronize(s));
    return DSD_OK;
}

// One Adam step on the batch (X [B x 64], y [B], host memory).
dsd_status dsd_model_train_step(dsd_model* M, const float* X, const float* y, uint32_t B, float q,
                                float lr, float* loss) {
    DSD_TRY(dsd_model_gradient(M, X, y, B, q, loss, nullptr));
    M->step++;
    float b1 = 0.9f, b2 = 0.999f;
    float c1 = 1.f - powf(b1, (float)M->step), c2 = 1.f - powf(b2, (float)M->step);
    k_adam<<<128, 256, 0, M->stream>>>(M->master, M->grad, M->adam_m, M->adam_v, M->w16, kNParams,
                                       lr, b1, b2, 1e-8f, c1, c2);
    note_launch();
    DSD_LAUNCHED();
    return DSD_OK;
}

// The 64 statistics of g for clique size h (host or device output).
dsd_status dsd_graph_features(dsd_graph* g, int h, float* f, int mem) {
    set_error("");
    if (!g || !f || h < 2 || h > DSD_MAX_H) return DSD_ERR_INVALID;
    float* dev = nullptr;
    cudaStream_t s = g->stream;
    if (mem == DSD_MEM_HOST) DSD_TRY(dalloc(&dev, kFeat, s));
    dsd_status st = compute_features(g, h, mem == DSD_MEM_HOST ? dev : f);
    if (st == DSD_OK && mem == DSD_MEM_HOST) {
        cudaError_t e = cudaMemcpyAsync(f, dev, kFeat * 4, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) st = cuda_fail(e, "features", __FILE__, __LINE__);
    }
    dev_free(dev, s);
    return st;
}

}  // extern "C"
