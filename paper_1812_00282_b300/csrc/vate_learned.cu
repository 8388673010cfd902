// vate_learned.cu -- the learned estimator (include/vate_learned.h): feature
// extraction at slice close, MLP inference, MLP training, and the fused
// gather + MLP estimate with the Eq. 11 fallback.  FP32 CUDA-core arithmetic:
// the model is far too small (5.7 k parameters) for tensor cores to pay.
#include <algorithm>
#include <cmath>

#include "vate.h"
#include "vate_learned.h"
#include "vate_device_ops.cuh"
#include "vate_ages.cuh"
#include "vate_launch.cuh"

using namespace vate;

namespace {

constexpr int HID = VATE_MLP_HIDDEN;     // 64
constexpr int MAX_IN = 32;               // 2k + 2 with k <= 15
constexpr int WARPS = 8;                 // warps per block in the per-host kernels
constexpr uint32_t SPLIT_MAX_L = 8;      // vate_estimate_learned: features, then the model, for L <= 8
constexpr uint64_t SPLIT_CHUNK = 1ull << 17;   // hosts per features + model pass (scratch: 2^17 (n_in + 1) floats)
constexpr int TR_ROWS = 64;              // rows per training tile
constexpr int TR_THREADS = 256;

// W1, b1, W2, b2, w3, b3, then the gate (not trained)
__host__ __device__ inline uint64_t n_params(uint32_t n_in) {
    return (uint64_t)n_in * HID + HID + (uint64_t)HID * HID + HID + HID + 1 + 1;
}

struct Layout {                          // offsets of the parameter blocks
    uint32_t W1, b1, W2, b2, w3, b3, gate;
};
__host__ __device__ inline Layout layout(uint32_t n_in) {
    Layout L;
    L.W1 = 0;
    L.b1 = n_in * HID;
    L.W2 = L.b1 + HID;
    L.b2 = L.W2 + HID * HID;
    L.w3 = L.b2 + HID;
    L.b3 = L.w3 + HID;
    L.gate = L.b3 + 1;
    return L;
}

// Features of one host into xw[0 .. 2k+2) (shared memory of the warp); returns
// the closed-form estimate for k' = k and its flags, and the active count.
__device__ __forceinline__ float host_features(const Geom &G, uint32_t bact0, const uint64_t *hist, uint64_t N0,
                                               uint32_t aip, uint32_t lane, float *xw, uint8_t &flags, uint32_t &A) {
    const uint32_t cd = host_age_counts(G, bact0, aip, lane);
    A = __reduce_add_sync(0xFFFFFFFFu, cd);
    const float plain = estimate_eq11(G.g, G.P, N0, A, flags);
    if (lane < G.k) {
        xw[lane] = (float)cd / (float)G.g;
        xw[G.k + lane] = (float)((double)hist[lane] / (double)G.P);
    }
    if (lane == 0) {
        xw[2 * G.k] = log2f((float)G.g) / 16.0f;
        xw[2 * G.k + 1] = log1pf(fmaxf(plain, 0.0f)) / 16.0f;
    }
    __syncwarp();
    return plain;
}

// y = w3 . relu(W2 relu(W1 x + b1) + b2) + b3 for one input row x (shared
// memory), evaluated by one lane.  The lanes of a warp evaluate different rows
// with the same weights, so every weight read is a shared-memory broadcast;
// w2t holds W2 transposed (w2t[j * 64 + i] = W2[i][j]) so that unit j reads its
// 64 inputs contiguously.  Every sum runs in index order (bias first), so the
// result is deterministic and the same in every kernel that calls this.
__device__ __forceinline__ float mlp_eval_lane(const float *prm, const float *w2t, uint32_t n_in, const float *x) {
    const Layout L = layout(n_in);
    float h[HID];
#pragma unroll
    for (int j = 0; j < HID; j++) h[j] = prm[L.b1 + j];
    for (uint32_t i = 0; i < n_in; i++) {
        const float xi = x[i];
        const float4 *row = reinterpret_cast<const float4 *>(prm + L.W1 + i * HID);
#pragma unroll
        for (int j4 = 0; j4 < HID / 4; j4++) {
            const float4 w = row[j4];
            h[4 * j4] = fmaf(w.x, xi, h[4 * j4]);
            h[4 * j4 + 1] = fmaf(w.y, xi, h[4 * j4 + 1]);
            h[4 * j4 + 2] = fmaf(w.z, xi, h[4 * j4 + 2]);
            h[4 * j4 + 3] = fmaf(w.w, xi, h[4 * j4 + 3]);
        }
    }
#pragma unroll
    for (int j = 0; j < HID; j++) h[j] = fmaxf(h[j], 0.0f);
    float y = prm[L.b3];
#pragma unroll 2
    for (int j = 0; j < HID; j++) {
        const float4 *col = reinterpret_cast<const float4 *>(w2t + j * HID);
        float a = prm[L.b2 + j];
#pragma unroll
        for (int i4 = 0; i4 < HID / 4; i4++) {
            const float4 w = col[i4];
            a = fmaf(w.x, h[4 * i4], a);
            a = fmaf(w.y, h[4 * i4 + 1], a);
            a = fmaf(w.z, h[4 * i4 + 2], a);
            a = fmaf(w.w, h[4 * i4 + 3], a);
        }
        y = fmaf(prm[L.w3 + j], fmaxf(a, 0.0f), y);
    }
    return y;
}

// The model in shared memory for mlp_eval_lane: the parameters (padded to a
// multiple of 4 floats) followed by W2 transposed.  Returns w2t.
__device__ __forceinline__ float *stage_model(float *sm, const float *params, uint32_t n_in) {
    const uint64_t np = n_params(n_in), npad = (np + 3) & ~3ull;
    const Layout L = layout(n_in);
    float *w2t = sm + npad;
    for (uint64_t i = threadIdx.x; i < np; i += blockDim.x) sm[i] = params[i];
    for (uint32_t t = threadIdx.x; t < HID * HID; t += blockDim.x) {
        const uint32_t j = t / HID, i = t % HID;
        w2t[t] = params[L.W2 + i * HID + j];
    }
    return w2t;
}

__host__ __device__ inline size_t model_smem_floats(uint32_t n_in) { return ((n_params(n_in) + 3) & ~3ull) + HID * HID; }

constexpr int XS = MAX_IN + 1;           // row stride of the per-warp input rows (no bank conflicts per lane)

__device__ __forceinline__ uint64_t inactive_for_k(const uint64_t *hist, uint64_t P, uint32_t k) {
    uint64_t act = 0;
    for (uint32_t d = 0; d < k; d++) act += hist[d];
    return P - act;
}

// Warp per host: the host's feature row into x, and, where plain / pflags are
// not NULL, its Eq. 11 estimate and the closed form's flags.
__global__ void __launch_bounds__(WARPS * 32) features_kernel(Geom G, uint32_t bact0, const uint64_t *__restrict__ hist,
                                                              const uint32_t *__restrict__ aips, uint64_t n,
                                                              float *__restrict__ x, float *__restrict__ plain,
                                                              uint8_t *__restrict__ pflags) {
    __shared__ float xs[WARPS][MAX_IN];
    __shared__ uint64_t sN0;
    if (threadIdx.x == 0) sN0 = inactive_for_k(hist, G.P, G.k);
    __syncthreads();
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    const uint32_t n_in = 2 * G.k + 2;
    for (uint64_t h = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5; h < n;
         h += ((uint64_t)gridDim.x * blockDim.x) >> 5) {
        uint8_t f = 0;
        uint32_t A;
        const float p = host_features(G, bact0, hist, sN0, aips[h], lane, xs[warp], f, A);
        if (lane < n_in) x[h * n_in + lane] = xs[warp][lane];
        if (lane == 0 && plain) plain[h] = p;
        if (lane == 0 && pflags) pflags[h] = f;
        __syncwarp();
    }
}

// The output rule of the learned estimator for one host: the closed form
// `plain` (Eq. 11) is returned, flagged FALLBACK, when the host has no active
// VAT in the window or when the corrected value expm1(8 y + log1p(max(plain,
// 0))) is not finite (x_last * 16 = log1p(max(plain, 0)) is the host's last
// feature); flagged GATED when the corrected value and the closed form are
// both >= the model's gate (a host both call large, for which the closed form
// is the better estimate); otherwise the corrected value.
__device__ __forceinline__ float learned_rule(float plain, bool no_active, float y, float x_last, float gate,
                                              uint8_t &flags) {
    if (no_active) {
        flags |= (uint8_t)VATE_FLAG_FALLBACK;
        return plain;
    }
    const float e = expm1f(8.0f * y + 16.0f * x_last);
    if (!isfinite(e)) {
        flags |= (uint8_t)VATE_FLAG_FALLBACK;
        return plain;
    }
    if (e >= gate && plain >= gate) {      // both call the host large: the closed form is kept
        flags |= (uint8_t)VATE_FLAG_GATED;
        return plain;
    }
    return e;
}

// 32 hosts per warp: the warp extracts each host's features into its row of
// xs (host_features), then lane j evaluates host j's model (mlp_eval_lane)
// and the fallback.
__global__ void __launch_bounds__(WARPS * 32, 3) learned_estimate_kernel(Geom G, uint32_t bact0,
                                                                      const uint64_t *__restrict__ hist,
                                                                      const uint32_t *__restrict__ aips, uint64_t n,
                                                                      const float *__restrict__ params,
                                                                      float *__restrict__ out,
                                                                      uint8_t *__restrict__ flags) {
    extern __shared__ float4 dyn4[];
    float *prm = reinterpret_cast<float *>(dyn4);
    const uint32_t n_in = 2 * G.k + 2;
    float *w2t = stage_model(prm, params, n_in);
    float *xs = w2t + HID * HID;                       // [WARPS][32][XS]
    __shared__ uint64_t sN0;
    if (threadIdx.x == 0) sN0 = inactive_for_k(hist, G.P, G.k);
    __syncthreads();
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    float *xw = xs + (size_t)warp * 32 * XS;
    const uint64_t warp0 = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t g0 = warp0 * 32; g0 < n; g0 += nwarps * 32) {
        uint32_t myA = 0;
        float myplain = 0.0f;
        uint8_t myf = 0;
        for (uint32_t j = 0; j < 32u && g0 + j < n; j++) {
            uint8_t f;
            uint32_t A;
            const float plain = host_features(G, bact0, hist, sN0, aips[g0 + j], lane, xw + j * XS, f, A);
            if (lane == j) {
                myA = A;
                myplain = plain;
                myf = f;
            }
        }
        __syncwarp();
        if (g0 + lane < n) {
            const float *x = xw + lane * XS;
            const float y = mlp_eval_lane(prm, w2t, n_in, x);
            const float e = learned_rule(myplain, myA == 0u, y, x[n_in - 1], prm[layout(n_in).gate], myf);
            out[g0 + lane] = e;
            if (flags) flags[g0 + lane] = myf;
        }
        __syncwarp();
    }
}

// Lane per row: lane j evaluates row r0 + j.
__global__ void __launch_bounds__(WARPS * 32) mlp_forward_kernel(const float *__restrict__ params, uint32_t n_in,
                                                                 const float *__restrict__ x, uint64_t n,
                                                                 float *__restrict__ y) {
    extern __shared__ float4 dyn4[];
    float *prm = reinterpret_cast<float *>(dyn4);
    float *w2t = stage_model(prm, params, n_in);
    float *xs = w2t + HID * HID;                       // [WARPS][32][XS]
    __syncthreads();
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    float *xw = xs + (size_t)warp * 32 * XS;
    const uint64_t warp0 = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t r0 = warp0 * 32; r0 < n; r0 += nwarps * 32) {
        const uint64_t rows = n - r0 < 32 ? n - r0 : 32;
        for (uint32_t t = lane; t < rows * n_in; t += 32u) xw[(t / n_in) * XS + t % n_in] = x[r0 * n_in + t];
        __syncwarp();
        if (lane < rows) y[r0 + lane] = mlp_eval_lane(prm, w2t, n_in, xw + lane * XS);
        __syncwarp();
    }
}

// The output rule on feature rows (lane per row, as mlp_forward_kernel): a
// row has no active VAT when its first k features (the per-age counts / g)
// are all 0, k = (n_in - 2) / 2.
// Lane per row: the output rule.  or_flags = 1: the rule's bits are added to
// the flags already in `flags` (the closed form's, written by features_kernel).
__global__ void __launch_bounds__(WARPS * 32) mlp_apply_kernel(const float *__restrict__ params, uint32_t n_in,
                                                               const float *__restrict__ x,
                                                               const float *__restrict__ plain, uint64_t n,
                                                               float *__restrict__ out, uint8_t *__restrict__ flags,
                                                               uint32_t or_flags) {
    extern __shared__ float4 dyn4[];
    float *prm = reinterpret_cast<float *>(dyn4);
    float *w2t = stage_model(prm, params, n_in);
    float *xs = w2t + HID * HID;                       // [WARPS][32][XS]
    __syncthreads();
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    const uint32_t k = (n_in - 2u) / 2u;
    float *xw = xs + (size_t)warp * 32 * XS;
    const uint64_t warp0 = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t r0 = warp0 * 32; r0 < n; r0 += nwarps * 32) {
        const uint64_t rows = n - r0 < 32 ? n - r0 : 32;
        for (uint32_t t = lane; t < rows * n_in; t += 32u) xw[(t / n_in) * XS + t % n_in] = x[r0 * n_in + t];
        __syncwarp();
        if (lane < rows) {
            const float *xr = xw + lane * XS;
            bool no_active = true;
            for (uint32_t d = 0; d < k; d++) no_active = no_active && xr[d] == 0.0f;
            const float y = mlp_eval_lane(prm, w2t, n_in, xr);
            uint8_t f = (or_flags && flags) ? flags[r0 + lane] : (uint8_t)0;
            out[r0 + lane] = learned_rule(plain[r0 + lane], no_active, y, xr[n_in - 1], prm[layout(n_in).gate], f);
            if (flags) flags[r0 + lane] = f;
        }
        __syncwarp();
    }
}

// mlp_apply_kernel fed from per-age counts instead of feature rows: lane j
// builds host j's row in shared memory from its counts (16-bit fields, age d
// of host h in counts[(d / 4) stride + h] >> 16 (d mod 4)) with the
// expressions of host_features, evaluates Eq. 11 and the model, and applies
// the output rule -- what vate_estimate_learned returns for the host, bit for
// bit, without a row in global memory.
__global__ void __launch_bounds__(WARPS * 32) learned_from_counts_kernel(Geom G, const uint64_t *__restrict__ hist,
                                                                         const unsigned long long *__restrict__ counts,
                                                                         uint64_t stride, uint64_t n,
                                                                         const float *__restrict__ params,
                                                                         float *__restrict__ out,
                                                                         uint8_t *__restrict__ flags) {
    extern __shared__ float4 dyn4[];
    const uint32_t n_in = 2 * G.k + 2;
    float *prm = reinterpret_cast<float *>(dyn4);
    float *w2t = stage_model(prm, params, n_in);
    float *xs = w2t + HID * HID;                       // [WARPS][32][XS]
    __shared__ uint64_t sN0;
    if (threadIdx.x == 0) sN0 = inactive_for_k(hist, G.P, G.k);
    __syncthreads();
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    float *xr = xs + (size_t)warp * 32 * XS + lane * XS;
    const float lg = log2f((float)G.g) / 16.0f;
    for (uint64_t h = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; h < n; h += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t A = 0;
        for (uint32_t d = 0; d < G.k; d++) {
            const uint32_t c = (uint32_t)(counts[(d >> 2) * stride + h] >> (16u * (d & 3u))) & 0xFFFFu;
            A += c;
            xr[d] = (float)c / (float)G.g;
            xr[G.k + d] = (float)((double)hist[d] / (double)G.P);
        }
        uint8_t f = 0;
        const float plain = estimate_eq11(G.g, G.P, sN0, A, f);
        xr[2 * G.k] = lg;
        xr[2 * G.k + 1] = log1pf(fmaxf(plain, 0.0f)) / 16.0f;
        const float y = mlp_eval_lane(prm, w2t, n_in, xr);
        out[h] = learned_rule(plain, A == 0u, y, xr[n_in - 1], prm[layout(n_in).gate], f);
        if (flags) flags[h] = f;
    }
}

__global__ void mlp_init_kernel(float *__restrict__ params, uint32_t n_in, uint64_t seed) {
    const Layout L = layout(n_in);
    const uint64_t np = n_params(n_in);
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < np; i += (uint64_t)gridDim.x * blockDim.x) {
        float a = 0.0f;
        if (i < L.b1) a = sqrtf(6.0f / (float)(n_in + HID));
        else if (i >= L.W2 && i < L.b2) a = sqrtf(6.0f / (float)(HID + HID));
        else if (i >= L.w3 && i < L.b3) a = sqrtf(6.0f / (float)(HID + 1));
        const uint64_t r = mix64(seed ^ (i * 0x9E3779B97F4A7C15ull));
        const float u = (float)(r >> 40) * (1.0f / 16777216.0f);     // [0, 1), 24 bits
        params[i] = i == L.gate ? INFINITY : a * (2.0f * u - 1.0f);  // the gate starts closed: never
    }
}

// One tile of TR_ROWS rows: forward, MSE gradient, backward; the tile's
// gradient (and loss) sums go to partial[blockIdx.x][...] for a fixed-order
// reduction.  Shared memory: parameters, X, H1, H2, dH2, dH1, dy.
__global__ void __launch_bounds__(TR_THREADS) mlp_grad_kernel(const float *__restrict__ params, uint32_t n_in,
                                                              const float *__restrict__ x,
                                                              const float *__restrict__ target,
                                                              const float *__restrict__ weight, uint32_t loss,
                                                              uint64_t n, float *__restrict__ partial,
                                                              float *__restrict__ loss_partial) {
    extern __shared__ float sm[];
    const Layout L = layout(n_in);
    const uint32_t np = (uint32_t)n_params(n_in);
    const uint32_t npad = (np + 3u) & ~3u;
    float *prm = sm;
    float *X = sm + npad;                       // [TR_ROWS][n_in]
    float *H1 = X + TR_ROWS * n_in;             // [TR_ROWS][HID]
    float *H2 = H1 + TR_ROWS * HID;
    float *D2 = H2 + TR_ROWS * HID;
    float *D1 = D2 + TR_ROWS * HID;
    float *dy = D1 + TR_ROWS * HID;             // [TR_ROWS]
    const uint32_t t = threadIdx.x;
    const uint64_t r0 = (uint64_t)blockIdx.x * TR_ROWS;
    const uint32_t rows = (uint32_t)min((uint64_t)TR_ROWS, n - r0);
    for (uint32_t i = t; i < np; i += TR_THREADS) prm[i] = params[i];
    for (uint32_t i = t; i < TR_ROWS * n_in; i += TR_THREADS) {
        const uint32_t r = i / n_in;
        X[i] = r < rows ? x[(r0 + r) * n_in + (i - r * n_in)] : 0.0f;
    }
    __syncthreads();
    const uint32_t j = t & (HID - 1), rq = t >> 6;      // hidden unit, row quarter
    for (uint32_t r = rq; r < TR_ROWS; r += 4) {
        float a = prm[L.b1 + j];
        for (uint32_t i = 0; i < n_in; i++) a = fmaf(X[r * n_in + i], prm[L.W1 + i * HID + j], a);
        H1[r * HID + j] = fmaxf(a, 0.0f);
    }
    __syncthreads();
    for (uint32_t r = rq; r < TR_ROWS; r += 4) {
        float a = prm[L.b2 + j];
        for (uint32_t i = 0; i < HID; i++) a = fmaf(H1[r * HID + i], prm[L.W2 + i * HID + j], a);
        H2[r * HID + j] = fmaxf(a, 0.0f);
    }
    __syncthreads();
    if (t < TR_ROWS) {
        float y = prm[L.b3];
        for (uint32_t i = 0; i < HID; i++) y = fmaf(H2[t * HID + i], prm[L.w3 + i], y);
        const float e = t < rows ? y - target[r0 + t] : 0.0f;
        const float w = (t < rows && weight) ? weight[r0 + t] : 1.0f;
        if (loss == VATE_MLP_LOSS_ABSOLUTE) {
            dy[t] = w * (e > 0.0f ? 1.0f : (e < 0.0f ? -1.0f : 0.0f)) / (float)n;
            D1[t] = w * fabsf(e) / (float)n;    // temporary: this row's loss term
        } else {
            dy[t] = 2.0f * w * e / (float)n;
            D1[t] = w * e * e / (float)n;       // temporary: this row's loss term
        }
    }
    __syncthreads();
    if (t == 0) {
        float s = 0.0f;
        for (uint32_t r = 0; r < TR_ROWS; r++) s += D1[r];
        loss_partial[blockIdx.x] = s;
    }
    __syncthreads();
    for (uint32_t r = rq; r < TR_ROWS; r += 4)
        D2[r * HID + j] = H2[r * HID + j] > 0.0f ? dy[r] * prm[L.w3 + j] : 0.0f;
    __syncthreads();
    for (uint32_t r = rq; r < TR_ROWS; r += 4) {
        float a = 0.0f;
        for (uint32_t q = 0; q < HID; q++) a = fmaf(D2[r * HID + q], prm[L.W2 + j * HID + q], a);
        D1[r * HID + j] = H1[r * HID + j] > 0.0f ? a : 0.0f;
    }
    __syncthreads();
    float *out = partial + (uint64_t)blockIdx.x * np;
    for (uint32_t p = t; p < np; p += TR_THREADS) {
        float s = 0.0f;
        if (p < L.b1) {                                         // dW1[i][q]
            const uint32_t i = p / HID, q = p % HID;
            for (uint32_t r = 0; r < TR_ROWS; r++) s = fmaf(X[r * n_in + i], D1[r * HID + q], s);
        } else if (p < L.W2) {                                  // db1
            for (uint32_t r = 0; r < TR_ROWS; r++) s += D1[r * HID + (p - L.b1)];
        } else if (p < L.b2) {                                  // dW2[i][q]
            const uint32_t i = (p - L.W2) / HID, q = (p - L.W2) % HID;
            for (uint32_t r = 0; r < TR_ROWS; r++) s = fmaf(H1[r * HID + i], D2[r * HID + q], s);
        } else if (p < L.w3) {                                  // db2
            for (uint32_t r = 0; r < TR_ROWS; r++) s += D2[r * HID + (p - L.b2)];
        } else if (p < L.b3) {                                  // dw3
            for (uint32_t r = 0; r < TR_ROWS; r++) s = fmaf(dy[r], H2[r * HID + (p - L.w3)], s);
        } else if (p == L.b3) {                                 // db3
            for (uint32_t r = 0; r < TR_ROWS; r++) s += dy[r];
        }                                                       // the gate: not trained (gradient 0)
        out[p] = s;
    }
}

__global__ void mlp_adam_kernel(float *__restrict__ params, float *__restrict__ m, float *__restrict__ v,
                                const float *__restrict__ partial, const float *__restrict__ loss_partial,
                                uint32_t ntiles, uint32_t np, float lr, float bc1, float bc2,
                                float *__restrict__ grad, float *__restrict__ loss) {
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    for (uint32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < np; p += gridDim.x * blockDim.x) {
        float g = 0.0f;
        for (uint32_t b = 0; b < ntiles; b++) g += partial[(uint64_t)b * np + p];   // fixed order
        if (grad) grad[p] = g;
        const float mm = b1 * m[p] + (1.0f - b1) * g;
        const float vv = b2 * v[p] + (1.0f - b2) * g * g;
        m[p] = mm;
        v[p] = vv;
        params[p] -= lr * (mm / bc1) / (sqrtf(vv / bc2) + eps);
    }
    if (loss && blockIdx.x == 0 && threadIdx.x == 0) {
        float s = 0.0f;
        for (uint32_t b = 0; b < ntiles; b++) s += loss_partial[b];
        *loss = s;
    }
}

size_t train_smem(uint32_t n_in) {
    const uint32_t np = (uint32_t)n_params(n_in);
    return sizeof(float) * (((np + 3u) & ~3u) + TR_ROWS * n_in + 4 * TR_ROWS * HID + TR_ROWS);
}

int sms_now() {
    int dev = 0, sms = 148;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms;
}

int check_learned_handle(const vate_handle *h, HandleView *v) {
    if (int rc = handle_view(h, v)) return rc;
    if (!v->closed) return set_error(VATE_ESLICE, "the current slice has not been closed");
    if (v->G.k > 15) return set_error(VATE_EINVAL, "the learned estimator needs k <= 15 (2k + 2 <= 32 inputs)");
    if (v->G.counter != VATE_COUNTER_AT) return set_error(VATE_EINVAL, "the learned estimator runs on asynchronous timestamps");
    if (v->G.lo != 0 || v->G.hi != v->G.P) return set_error(VATE_EINVAL, "the learned estimator needs the whole pool");
    if (v->G.packed) return set_error(VATE_EINVAL, "the learned estimator needs byte ATs (at_bits 0 or 8)");
    return VATE_OK;
}

}  // namespace

namespace vate {

int learned_handle_ok(const vate_handle *h) {
    HandleView w;
    return check_learned_handle(h, &w);
}

int learned_from_age_counts(vate_handle *h, const HandleView &v, const unsigned long long *counts, uint64_t n,
                            const float *d_params, float *d_out, uint8_t *d_flags, cudaStream_t st) {
    if (int rc = learned_handle_ok(h)) return rc;
    const uint32_t n_in = 2 * v.G.k + 2;
    const size_t smem = sizeof(float) * (model_smem_floats(n_in) + (size_t)WARPS * 32 * XS);
    if (cudaError_t e = cudaFuncSetAttribute(learned_from_counts_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem))
        return set_error(VATE_ECUDA, cudaGetErrorString(e));
    const int grid = (int)std::min<uint64_t>((n + WARPS * 32 - 1) / (WARPS * 32), (uint64_t)v.sms * 8);
    learned_from_counts_kernel<<<grid, WARPS * 32, smem, st>>>(v.G, v.hist, counts, n, n, d_params, d_out, d_flags);
    count_launch();
    if (cudaError_t e = cudaGetLastError()) return set_error(VATE_ECUDA, cudaGetErrorString(e));
    return VATE_OK;
}

}  // namespace vate

extern "C" {

uint64_t vate_mlp_param_count(uint32_t n_in) { return n_params(n_in); }

uint64_t vate_mlp_train_scratch(uint32_t n_in, uint64_t n) {
    const uint64_t tiles = (n + TR_ROWS - 1) / TR_ROWS;
    return tiles * n_params(n_in) + tiles;
}

int vate_features(vate_handle *h, const uint32_t *d_aips, uint64_t n, float *d_x, void *stream) {
    HandleView v;
    if (int rc = check_learned_handle(h, &v)) return rc;
    if (n && (!d_aips || !d_x)) return set_error(VATE_EINVAL, "d_aips and d_x must not be NULL");
    if (n == 0) return VATE_OK;
    int grid = (int)std::min<uint64_t>((n + WARPS - 1) / WARPS, (uint64_t)v.sms * 16);
    cudaError_t e = launch_pool(v.G, features_kernel, grid, WARPS * 32, 0, (cudaStream_t)stream, v.G, v.bact0, v.hist,
                                d_aips, n, d_x, (float *)nullptr, (uint8_t *)nullptr);
    return e == cudaSuccess ? VATE_OK : set_error(VATE_ECUDA, cudaGetErrorString(e));
}

int vate_mlp_init(float *d_params, uint32_t n_in, uint64_t seed, void *stream) {
    if (!d_params || n_in < 1 || n_in > MAX_IN) return set_error(VATE_EINVAL, "bad parameters pointer or n_in (1..32)");
    mlp_init_kernel<<<16, 256, 0, (cudaStream_t)stream>>>(d_params, n_in, seed);
    count_launch();
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? VATE_OK : set_error(VATE_ECUDA, cudaGetErrorString(e));
}

int vate_mlp_forward(const float *d_params, uint32_t n_in, const float *d_x, uint64_t n, float *d_y, void *stream) {
    if (!d_params || n_in < 1 || n_in > MAX_IN) return set_error(VATE_EINVAL, "bad parameters pointer or n_in (1..32)");
    if (n && (!d_x || !d_y)) return set_error(VATE_EINVAL, "d_x and d_y must not be NULL");
    if (n == 0) return VATE_OK;
    const size_t smem = sizeof(float) * (model_smem_floats(n_in) + (size_t)WARPS * 32 * XS);
    if (cudaError_t e = cudaFuncSetAttribute(mlp_forward_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem))
        return set_error(VATE_ECUDA, cudaGetErrorString(e));
    int grid = (int)std::min<uint64_t>((n + WARPS * 32 - 1) / (WARPS * 32), (uint64_t)sms_now() * 8);
    mlp_forward_kernel<<<grid, WARPS * 32, smem, (cudaStream_t)stream>>>(d_params, n_in, d_x, n, d_y);
    count_launch();
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? VATE_OK : set_error(VATE_ECUDA, cudaGetErrorString(e));
}

int vate_mlp_train_step(float *d_params, float *d_m, float *d_v, uint32_t n_in, const float *d_x,
                        const float *d_target, const float *d_weight, uint32_t loss, uint64_t n, float lr,
                        uint32_t t, float *d_scratch, uint64_t scratch_floats, float *d_grad, float *d_loss,
                        void *stream) {
    if (!d_params || !d_m || !d_v || !d_x || !d_target || !d_scratch)
        return set_error(VATE_EINVAL, "NULL buffer");
    if (n_in < 1 || n_in > MAX_IN || n == 0 || t < 1) return set_error(VATE_EINVAL, "n_in in 1..32, n > 0, t >= 1");
    if (scratch_floats < vate_mlp_train_scratch(n_in, n)) return set_error(VATE_EINVAL, "scratch too small");
    if (loss > VATE_MLP_LOSS_ABSOLUTE) return set_error(VATE_EINVAL, "unknown loss");
    cudaStream_t st = (cudaStream_t)stream;
    const uint32_t tiles = (uint32_t)((n + TR_ROWS - 1) / TR_ROWS);
    const uint32_t np = (uint32_t)n_params(n_in);
    const size_t smem = train_smem(n_in);
    if (cudaError_t e = cudaFuncSetAttribute(mlp_grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem))
        return set_error(VATE_ECUDA, cudaGetErrorString(e));
    float *partial = d_scratch, *loss_partial = d_scratch + (uint64_t)tiles * np;
    mlp_grad_kernel<<<tiles, TR_THREADS, smem, st>>>(d_params, n_in, d_x, d_target, d_weight, loss, n, partial,
                                                     loss_partial);
    count_launch();
    const float bc1 = 1.0f - powf(0.9f, (float)t), bc2 = 1.0f - powf(0.999f, (float)t);
    mlp_adam_kernel<<<(np + 255) / 256, 256, 0, st>>>(d_params, d_m, d_v, partial, loss_partial, tiles, np, lr, bc1,
                                                      bc2, d_grad, d_loss);
    count_launch();
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? VATE_OK : set_error(VATE_ECUDA, cudaGetErrorString(e));
}

int vate_mlp_apply(const float *d_params, uint32_t n_in, const float *d_x, const float *d_plain, uint64_t n,
                   float *d_out, uint8_t *d_flags, void *stream) {
    if (!d_params || n_in < 4 || n_in > MAX_IN || (n_in & 1u))
        return set_error(VATE_EINVAL, "bad parameters pointer or n_in (2k + 2 for 1 <= k <= 15)");
    if (n && (!d_x || !d_plain || !d_out)) return set_error(VATE_EINVAL, "d_x, d_plain and d_out must not be NULL");
    if (n == 0) return VATE_OK;
    const size_t smem = sizeof(float) * (model_smem_floats(n_in) + (size_t)WARPS * 32 * XS);
    if (cudaError_t e = cudaFuncSetAttribute(mlp_apply_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem))
        return set_error(VATE_ECUDA, cudaGetErrorString(e));
    int grid = (int)std::min<uint64_t>((n + WARPS * 32 - 1) / (WARPS * 32), (uint64_t)sms_now() * 8);
    mlp_apply_kernel<<<grid, WARPS * 32, smem, (cudaStream_t)stream>>>(d_params, n_in, d_x, d_plain, n, d_out, d_flags,
                                                                       0u);
    count_launch();
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? VATE_OK : set_error(VATE_ECUDA, cudaGetErrorString(e));
}

int vate_estimate_learned(vate_handle *h, const uint32_t *d_aips, uint64_t n, const float *d_params, float *d_out,
                          uint8_t *d_flags, void *stream) {
    HandleView v;
    if (int rc = check_learned_handle(h, &v)) return rc;
    if (!d_params) return set_error(VATE_EINVAL, "d_params must not be NULL");
    if (n && (!d_aips || !d_out)) return set_error(VATE_EINVAL, "d_aips and d_out must not be NULL");
    if (n == 0) return VATE_OK;
    const uint32_t n_in = 2 * v.G.k + 2;
    const size_t smem = sizeof(float) * (model_smem_floats(n_in) + (size_t)WARPS * 32 * XS);
    cudaStream_t st = (cudaStream_t)stream;
    if (v.G.L <= SPLIT_MAX_L) {
        // Segments of at most 8 ATs: the reads of the host's g / L segments bound the close, and the
        // features kernel, free of the model's registers, keeps enough of them in flight to run at
        // the random-sector rate; the model then runs over the rows (same values, same order: the
        // results equal the fused kernel's bit for bit).
        void *scr = nullptr;
        const uint64_t chunk = std::min<uint64_t>(n, SPLIT_CHUNK);
        if (int rc = handle_scratch(h, chunk * (n_in + 1) * sizeof(float), &scr)) return rc;
        float *x = static_cast<float *>(scr), *plain = x + chunk * n_in;
        if (cudaError_t e = cudaFuncSetAttribute(mlp_apply_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem))
            return set_error(VATE_ECUDA, cudaGetErrorString(e));
        for (uint64_t h0 = 0; h0 < n; h0 += chunk) {
            const uint64_t m = std::min(chunk, n - h0);
            const int fgrid = (int)std::min<uint64_t>((m + WARPS - 1) / WARPS, (uint64_t)v.sms * 16);
            cudaError_t e = launch_pool(v.G, features_kernel, fgrid, WARPS * 32, 0, st, v.G, v.bact0, v.hist,
                                        d_aips + h0, m, x, plain, d_flags ? d_flags + h0 : (uint8_t *)nullptr);
            if (e != cudaSuccess) return set_error(VATE_ECUDA, cudaGetErrorString(e));
            const int agrid = (int)std::min<uint64_t>((m + WARPS * 32 - 1) / (WARPS * 32), (uint64_t)v.sms * 8);
            mlp_apply_kernel<<<agrid, WARPS * 32, smem, st>>>(d_params, n_in, x, plain, m, d_out + h0,
                                                              d_flags ? d_flags + h0 : (uint8_t *)nullptr, 1u);
            count_launch();
            if ((e = cudaGetLastError()) != cudaSuccess) return set_error(VATE_ECUDA, cudaGetErrorString(e));
        }
        return VATE_OK;
    }
    if (cudaError_t e = cudaFuncSetAttribute(learned_estimate_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem))
        return set_error(VATE_ECUDA, cudaGetErrorString(e));
    int grid = (int)std::min<uint64_t>((n + WARPS * 32 - 1) / (WARPS * 32), (uint64_t)v.sms * 8);
    cudaError_t e = launch_pool(v.G, learned_estimate_kernel, grid, WARPS * 32, smem, st, v.G,
                                v.bact0, v.hist, d_aips, n, d_params, d_out, d_flags);
    return e == cudaSuccess ? VATE_OK : set_error(VATE_ECUDA, cudaGetErrorString(e));
}

}  // extern "C"
