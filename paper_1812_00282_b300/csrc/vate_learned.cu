// vate_learned.cu -- the learned estimator (include/vate_learned.h): feature
// extraction at slice close, MLP inference, MLP training, and the fused
// gather + MLP estimate with the Eq. 11 fallback.  FP32 CUDA-core arithmetic:
// the model is far too small (5.7 k parameters) for tensor cores to pay.
#include <algorithm>
#include <cmath>

#include "vate.h"
#include "vate_learned.h"
#include "vate_device_ops.cuh"
#include "vate_launch.cuh"

using namespace vate;

namespace {

constexpr int HID = VATE_MLP_HIDDEN;     // 64
constexpr int MAX_IN = 32;               // 2k + 2 with k <= 15
constexpr int WARPS = 8;                 // warps per block in the per-host kernels
constexpr int TR_ROWS = 64;              // rows per training tile
constexpr int TR_THREADS = 256;

__host__ __device__ inline uint64_t n_params(uint32_t n_in) {
    return (uint64_t)n_in * HID + HID + (uint64_t)HID * HID + HID + HID + 1;
}

struct Layout {                          // offsets of the parameter blocks
    uint32_t W1, b1, W2, b2, w3, b3;
};
__host__ __device__ inline Layout layout(uint32_t n_in) {
    Layout L;
    L.W1 = 0;
    L.b1 = n_in * HID;
    L.W2 = L.b1 + HID;
    L.b2 = L.W2 + HID * HID;
    L.w3 = L.b2 + HID;
    L.b3 = L.w3 + HID;
    return L;
}

// Per-age counts of one host's VATs accumulated into this lane's column
// (col[d * 32], d < k) from a frame-0 pool, where every AT has ACT = BACT^0;
// 16-byte chunks when L >= 16, one byte per VAT otherwise.
__device__ __forceinline__ void host_age_columns(const Geom &G, uint32_t bact0, uint32_t aip, uint32_t lane,
                                                 uint32_t *col) {
    const uint64_t hk = host_key(G, aip);
    if (G.L >= 16) {
        const uint4 *pool16 = reinterpret_cast<const uint4 *>(G.pool);
        const uint32_t nchunks = G.g >> 4;
        for (uint32_t c = lane; c < nchunks; c += 32u) {
            const uint32_t pid = vat_pid_k(G, hk, c << 4);   // first VAT of the chunk
            const uint4 w = __ldg(pool16 + (pid >> 4));
            uint32_t words[4] = {swar_bins(w.x, bact0, G.twok), swar_bins(w.y, bact0, G.twok),
                                 swar_bins(w.z, bact0, G.twok), swar_bins(w.w, bact0, G.twok)};
#pragma unroll
            for (int b = 0; b < 16; b++) {
                uint32_t d = (words[b >> 2] >> (8 * (b & 3))) & 0xFFu;
                if (d < G.k) col[d * 32u] += 1u;
            }
        }
    } else {
        for (uint32_t i = lane; i < G.g; i += 32u) {
            uint32_t v = __ldg(G.pool + vat_pid_k(G, hk, i));
            if (v >= G.twok) continue;
            uint32_t d = bact0 + G.twok - v;
            if (d >= G.twok) d -= G.twok;
            if (d < G.k) col[d * 32u] += 1u;
        }
    }
}

// Features of one host into xw[0 .. 2k+2) (shared memory of the warp); returns
// the closed-form estimate for k' = k and its flags, and the active count.
__device__ __forceinline__ float host_features(const Geom &G, uint32_t bact0, const uint64_t *hist, uint64_t N0,
                                               uint32_t aip, uint32_t lane, uint32_t *colw, float *xw,
                                               uint8_t &flags, uint32_t &A) {
    uint32_t *col = colw + lane;
    for (uint32_t d = 0; d < G.k; d++) col[d * 32u] = 0u;
    host_age_columns(G, bact0, aip, lane, col);
    __syncwarp();
    uint32_t cd = 0;
    if (lane < G.k)
        for (uint32_t l = 0; l < 32u; l++) cd += colw[lane * 32u + l];
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

// y = w3 . relu(W2 relu(W1 x + b1) + b2) + b3 for one input row held in shared
// memory (xw), lane j computing hidden units j and j + 32.  Summation order is
// fixed, so the result is deterministic.
__device__ __forceinline__ float mlp_eval_warp(const float *prm, uint32_t n_in, const float *xw, uint32_t lane) {
    const Layout L = layout(n_in);
    float a = prm[L.b1 + lane], b = prm[L.b1 + lane + 32];
    for (uint32_t i = 0; i < n_in; i++) {
        const float xi = xw[i];
        a = fmaf(prm[L.W1 + i * HID + lane], xi, a);
        b = fmaf(prm[L.W1 + i * HID + lane + 32], xi, b);
    }
    a = fmaxf(a, 0.0f);
    b = fmaxf(b, 0.0f);
    float c = prm[L.b2 + lane], d = prm[L.b2 + lane + 32];
#pragma unroll 8
    for (uint32_t i = 0; i < 32; i++) {
        const float hi = __shfl_sync(0xFFFFFFFFu, a, i);
        c = fmaf(prm[L.W2 + i * HID + lane], hi, c);
        d = fmaf(prm[L.W2 + i * HID + lane + 32], hi, d);
    }
#pragma unroll 8
    for (uint32_t i = 0; i < 32; i++) {
        const float hi = __shfl_sync(0xFFFFFFFFu, b, i);
        c = fmaf(prm[L.W2 + (i + 32) * HID + lane], hi, c);
        d = fmaf(prm[L.W2 + (i + 32) * HID + lane + 32], hi, d);
    }
    c = fmaxf(c, 0.0f);
    d = fmaxf(d, 0.0f);
    float y = fmaf(prm[L.w3 + lane], c, prm[L.w3 + lane + 32] * d);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) y += __shfl_down_sync(0xFFFFFFFFu, y, o);
    y = __shfl_sync(0xFFFFFFFFu, y, 0);
    return y + prm[L.b3];
}

__device__ __forceinline__ uint64_t inactive_for_k(const uint64_t *hist, uint64_t P, uint32_t k) {
    uint64_t act = 0;
    for (uint32_t d = 0; d < k; d++) act += hist[d];
    return P - act;
}

__global__ void __launch_bounds__(WARPS * 32) features_kernel(Geom G, uint32_t bact0, const uint64_t *__restrict__ hist,
                                                              const uint32_t *__restrict__ aips, uint64_t n,
                                                              float *__restrict__ x) {
    __shared__ uint32_t cols[WARPS][15 * 32];
    __shared__ float xs[WARPS][MAX_IN];
    __shared__ uint64_t sN0;
    if (threadIdx.x == 0) sN0 = inactive_for_k(hist, G.P, G.k);
    __syncthreads();
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    const uint32_t n_in = 2 * G.k + 2;
    for (uint64_t h = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5; h < n;
         h += ((uint64_t)gridDim.x * blockDim.x) >> 5) {
        uint8_t f;
        uint32_t A;
        host_features(G, bact0, hist, sN0, aips[h], lane, cols[warp], xs[warp], f, A);
        if (lane < n_in) x[h * n_in + lane] = xs[warp][lane];
        __syncwarp();
    }
}

__global__ void __launch_bounds__(WARPS * 32) learned_estimate_kernel(Geom G, uint32_t bact0,
                                                                      const uint64_t *__restrict__ hist,
                                                                      const uint32_t *__restrict__ aips, uint64_t n,
                                                                      const float *__restrict__ params,
                                                                      float *__restrict__ out,
                                                                      uint8_t *__restrict__ flags) {
    extern __shared__ float prm[];           // the model
    __shared__ uint32_t cols[WARPS][15 * 32];
    __shared__ float xs[WARPS][MAX_IN];
    __shared__ uint64_t sN0;
    const uint32_t n_in = 2 * G.k + 2;
    const uint64_t np = n_params(n_in);
    for (uint64_t i = threadIdx.x; i < np; i += blockDim.x) prm[i] = params[i];
    if (threadIdx.x == 0) sN0 = inactive_for_k(hist, G.P, G.k);
    __syncthreads();
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    for (uint64_t h = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5; h < n;
         h += ((uint64_t)gridDim.x * blockDim.x) >> 5) {
        uint8_t f;
        uint32_t A;
        const float plain = host_features(G, bact0, hist, sN0, aips[h], lane, cols[warp], xs[warp], f, A);
        const float y = mlp_eval_warp(prm, n_in, xs[warp], lane);
        // the model corrects the closed form in log space: x[2k+1] * 16 = log1p(max(plain, 0))
        float e = expm1f(8.0f * y + 16.0f * xs[warp][n_in - 1]);
        if (A == 0u || !isfinite(e)) {
            e = plain;
            f |= (uint8_t)VATE_FLAG_FALLBACK;
        }
        if (lane == 0) {
            out[h] = e;
            if (flags) flags[h] = f;
        }
        __syncwarp();
    }
}

__global__ void __launch_bounds__(WARPS * 32) mlp_forward_kernel(const float *__restrict__ params, uint32_t n_in,
                                                                 const float *__restrict__ x, uint64_t n,
                                                                 float *__restrict__ y) {
    extern __shared__ float prm[];
    __shared__ float xs[WARPS][MAX_IN];
    const uint64_t np = n_params(n_in);
    for (uint64_t i = threadIdx.x; i < np; i += blockDim.x) prm[i] = params[i];
    __syncthreads();
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    for (uint64_t r = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5; r < n;
         r += ((uint64_t)gridDim.x * blockDim.x) >> 5) {
        if (lane < n_in) xs[warp][lane] = x[r * n_in + lane];
        __syncwarp();
        const float v = mlp_eval_warp(prm, n_in, xs[warp], lane);
        if (lane == 0) y[r] = v;
        __syncwarp();
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
        params[i] = a * (2.0f * u - 1.0f);
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
        } else {                                                // db3
            for (uint32_t r = 0; r < TR_ROWS; r++) s += dy[r];
        }
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
                                d_aips, n, d_x);
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
    const size_t smem = sizeof(float) * n_params(n_in);
    cudaFuncSetAttribute(mlp_forward_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int grid = (int)std::min<uint64_t>((n + WARPS - 1) / WARPS, (uint64_t)sms_now() * 8);
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
    cudaFuncSetAttribute(mlp_grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
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

int vate_estimate_learned(vate_handle *h, const uint32_t *d_aips, uint64_t n, const float *d_params, float *d_out,
                          uint8_t *d_flags, void *stream) {
    HandleView v;
    if (int rc = check_learned_handle(h, &v)) return rc;
    if (!d_params) return set_error(VATE_EINVAL, "d_params must not be NULL");
    if (n && (!d_aips || !d_out)) return set_error(VATE_EINVAL, "d_aips and d_out must not be NULL");
    if (n == 0) return VATE_OK;
    const size_t smem = sizeof(float) * n_params(2 * v.G.k + 2);
    cudaFuncSetAttribute(learned_estimate_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int grid = (int)std::min<uint64_t>((n + WARPS - 1) / WARPS, (uint64_t)v.sms * 8);
    cudaError_t e = launch_pool(v.G, learned_estimate_kernel, grid, WARPS * 32, smem, (cudaStream_t)stream, v.G,
                                v.bact0, v.hist, d_aips, n, d_params, d_out, d_flags);
    return e == cudaSuccess ? VATE_OK : set_error(VATE_ECUDA, cudaGetErrorString(e));
}

}  // extern "C"
