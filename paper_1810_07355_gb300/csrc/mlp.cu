// The per-query parameter predictor: a 16 -> 64 -> 64 -> 2 network with ReLU
// after both hidden layers, trained on the GPU in float32 and evaluated in
// bfloat16.  The paper's counterpart is the fixed policy of Eq. 1 (e_p as a
// function of eps); here the network maps features of a query's first hops to
// (log(eps + 0.01), log e_s).
//
// Parameters are one flat float32 vector: W1[64][16], b1[64], W2[64][64],
// b2[64], W3[2][64], b3[2] (5,378 values).  Loss: batch mean of
// 0.5 * sum_o (y_o - t_o)^2.
//
// One warp evaluates one sample: lane j owns hidden units j and j + 32.  The
// weights sit in shared memory transposed (input-major), so the 32 lanes read
// 32 consecutive words.  Gradients are accumulated in shared memory with
// atomics and written (or added) to global memory once per CTA.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>

#include "common.cuh"

namespace onng {
namespace {

constexpr int I = 16, H = 64, O = 2;
constexpr int NP = H * I + H + H * H + H + O * H + O;  // 5378
constexpr int kMlpWarps = 8;
constexpr unsigned FULL = 0xffffffffu;

// offsets in the flat (row-major, output-major) parameter vector
constexpr int oW1 = 0, ob1 = oW1 + H * I, oW2 = ob1 + H, ob2 = oW2 + H * H, oW3 = ob2 + H, ob3 = oW3 + O * H;

// Shared-memory image of the parameters, input-major for the weight matrices.
struct MlpShared {
    float w1t[I * H];  // [i][u]
    float b1[H];
    float w2t[H * H];  // [i][u]
    float w2[H * H];   // [u][i], read by the backward pass
    float b2[H];
    float w3[O * H];   // [o][u]
    float b3[O];
};

__device__ void load_params(MlpShared &s, const float *__restrict__ P)
{
    for (int e = threadIdx.x; e < H * I; e += blockDim.x) {
        const int u = e / I, i = e % I;
        s.w1t[i * H + u] = P[oW1 + e];
    }
    for (int e = threadIdx.x; e < H * H; e += blockDim.x) {
        const int u = e / H, i = e % H;
        s.w2t[i * H + u] = P[oW2 + e];
        s.w2[e] = P[oW2 + e];
    }
    for (int e = threadIdx.x; e < H; e += blockDim.x) {
        s.b1[e] = P[ob1 + e];
        s.b2[e] = P[ob2 + e];
    }
    for (int e = threadIdx.x; e < O * H; e += blockDim.x)
        s.w3[e] = P[oW3 + e];
    if (threadIdx.x < O)
        s.b3[threadIdx.x] = P[ob3 + threadIdx.x];
}

// Writes (or adds) a shared gradient image back to the flat layout.
__device__ void store_grad(const MlpShared &g, float *__restrict__ G, bool add)
{
    for (int e = threadIdx.x; e < NP; e += blockDim.x) {
        float v;
        if (e < ob1) {
            const int u = e / I, i = e % I;
            v = g.w1t[i * H + u];
        } else if (e < oW2) {
            v = g.b1[e - ob1];
        } else if (e < ob2) {
            const int u = (e - oW2) / H, i = (e - oW2) % H;
            v = g.w2t[i * H + u];
        } else if (e < oW3) {
            v = g.b2[e - ob2];
        } else if (e < ob3) {
            v = g.w3[e - oW3];
        } else {
            v = g.b3[e - ob3];
        }
        if (add)
            atomicAdd(&G[e], v);
        else
            G[e] = v;
    }
}

__device__ void zero_shared(MlpShared &g)
{
    float *f = reinterpret_cast<float *>(&g);
    for (int e = threadIdx.x; e < (int)(sizeof(MlpShared) / sizeof(float)); e += blockDim.x)
        f[e] = 0.f;
}

__device__ __forceinline__ float warp_sum(float v)
{
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1)
        v += __shfl_xor_sync(FULL, v, off);
    return v;
}

// Forward pass of one sample by one warp; returns y in every lane.  h1 (64
// floats of per-warp scratch) receives the first hidden layer.
__device__ void forward_warp(const MlpShared &s, const float *x, float *h1, int lane, float (&a1)[2], float (&a2)[2],
                             float (&h2)[2], float (&y)[O])
{
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        const int u = lane + 32 * r;
        float acc = s.b1[u];
#pragma unroll
        for (int i = 0; i < I; ++i)
            acc = fmaf(s.w1t[i * H + u], x[i], acc);
        a1[r] = acc;
        h1[u] = fmaxf(acc, 0.f);
    }
    __syncwarp();
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        const int u = lane + 32 * r;
        float acc = s.b2[u];
#pragma unroll 8
        for (int i = 0; i < H; ++i)
            acc = fmaf(s.w2t[i * H + u], h1[i], acc);
        a2[r] = acc;
        h2[r] = fmaxf(acc, 0.f);
    }
#pragma unroll
    for (int o = 0; o < O; ++o) {
        float p = s.w3[o * H + lane] * h2[0] + s.w3[o * H + lane + 32] * h2[1];
        y[o] = warp_sum(p) + s.b3[o];
    }
}

// Forward and backward of one sample; adds scale * dLoss/dParams into g (shared).
__device__ float fwd_bwd_warp(const MlpShared &s, MlpShared &g, const float *x, const float *t, float scale, float *h1,
                              float *da2s, int lane)
{
    float a1[2], a2[2], h2[2], y[O];
    forward_warp(s, x, h1, lane, a1, a2, h2, y);
    float dy[O], loss = 0.f;
#pragma unroll
    for (int o = 0; o < O; ++o) {
        const float e = y[o] - t[o];
        loss += 0.5f * e * e;
        dy[o] = e * scale;
    }
    if (lane < O)
        atomicAdd(&g.b3[lane], dy[lane]);
    float da2[2];
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        const int u = lane + 32 * r;
        float dh2 = 0.f;
#pragma unroll
        for (int o = 0; o < O; ++o) {
            atomicAdd(&g.w3[o * H + u], dy[o] * h2[r]);
            dh2 = fmaf(s.w3[o * H + u], dy[o], dh2);
        }
        da2[r] = a2[r] > 0.f ? dh2 : 0.f;
        atomicAdd(&g.b2[u], da2[r]);
        da2s[u] = da2[r];
    }
    // gW2[u][i] += da2[u] * h1[i]  (input-major image: w2t[i][u])
#pragma unroll 8
    for (int i = 0; i < H; ++i) {
        const float hi = h1[i];
        atomicAdd(&g.w2t[i * H + lane], da2[0] * hi);
        atomicAdd(&g.w2t[i * H + lane + 32], da2[1] * hi);
    }
    __syncwarp();
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        const int u = lane + 32 * r;  // first-layer unit
        float dh1 = 0.f;
#pragma unroll 8
        for (int j = 0; j < H; ++j)
            dh1 = fmaf(s.w2[j * H + u], da2s[j], dh1);
        const float da1 = a1[r] > 0.f ? dh1 : 0.f;
        atomicAdd(&g.b1[u], da1);
#pragma unroll
        for (int i = 0; i < I; ++i)
            atomicAdd(&g.w1t[i * H + u], da1 * x[i]);
    }
    __syncwarp();
    return loss;
}

// Loss and gradient over a batch: every CTA accumulates its samples in shared
// memory and adds them to G (which the host zeroes first).
__global__ void __launch_bounds__(kMlpWarps * 32)
    mlp_loss_grad_kernel(const float *__restrict__ P, const float *__restrict__ X, const float *__restrict__ T,
                         int64_t B, float *__restrict__ G, float *__restrict__ loss_out)
{
    extern __shared__ __align__(16) unsigned char raw[];
    MlpShared &s = *reinterpret_cast<MlpShared *>(raw);
    MlpShared &g = *reinterpret_cast<MlpShared *>(raw + sizeof(MlpShared));
    float *scratch = reinterpret_cast<float *>(raw + 2 * sizeof(MlpShared));
    __shared__ float s_loss;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    load_params(s, P);
    zero_shared(g);
    if (threadIdx.x == 0)
        s_loss = 0.f;
    __syncthreads();
    float *h1 = scratch + warp * 2 * H;
    float *da2s = h1 + H;
    const float scale = 1.f / (float)B;
    float lsum = 0.f;
    for (int64_t b = (int64_t)blockIdx.x * kMlpWarps + warp; b < B; b += (int64_t)gridDim.x * kMlpWarps) {
        float x[I], t[O];
#pragma unroll
        for (int i = 0; i < I; ++i)
            x[i] = X[b * I + i];
        t[0] = T[b * O];
        t[1] = T[b * O + 1];
        lsum += fwd_bwd_warp(s, g, x, t, scale, h1, da2s, lane);
    }
    if (lane == 0)
        atomicAdd(&s_loss, lsum);
    __syncthreads();
    store_grad(g, G, true);
    if (threadIdx.x == 0)
        atomicAdd(loss_out, s_loss * scale);
}

__global__ void __launch_bounds__(kMlpWarps * 32)
    mlp_forward_kernel(const float *__restrict__ P, const float *__restrict__ X, int64_t B, float *__restrict__ Y)
{
    extern __shared__ __align__(16) unsigned char raw[];
    MlpShared &s = *reinterpret_cast<MlpShared *>(raw);
    float *scratch = reinterpret_cast<float *>(raw + sizeof(MlpShared));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    load_params(s, P);
    __syncthreads();
    float *h1 = scratch + warp * H;
    for (int64_t b = (int64_t)blockIdx.x * kMlpWarps + warp; b < B; b += (int64_t)gridDim.x * kMlpWarps) {
        float x[I];
#pragma unroll
        for (int i = 0; i < I; ++i)
            x[i] = X[b * I + i];
        float a1[2], a2[2], h2[2], y[O];
        forward_warp(s, x, h1, lane, a1, a2, h2, y);
        if (lane < O)
            Y[b * O + lane] = y[lane];
        __syncwarp();
    }
}

// Adam (Kingma & Ba 2015) on the flat vectors, step count t >= 1.
__device__ __forceinline__ void adam1(float &p, float g, float &m, float &v, float lr, float b1, float b2, float eps,
                                      float c1, float c2)
{
    m = b1 * m + (1.f - b1) * g;
    v = b2 * v + (1.f - b2) * g * g;
    p -= lr * (m / c1) / (sqrtf(v / c2) + eps);
}

__global__ void mlp_adam_kernel(float *__restrict__ P, const float *__restrict__ G, float *__restrict__ M,
                                float *__restrict__ Vv, int64_t t, float lr, float b1, float b2, float eps)
{
    const float c1 = 1.f - powf(b1, (float)t), c2 = 1.f - powf(b2, (float)t);
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < NP; e += gridDim.x * blockDim.x)
        adam1(P[e], G[e], M[e], Vv[e], lr, b1, b2, eps, c1, c2);
}

// Whole training run in one CTA, as batched small matrix products in shared
// memory (no atomics): per step, for a mini-batch of B <= 128 consecutive rows
// (wrapping around the set) the forward pass keeps the pre-activations A1, A2
// [B][64]; the backward pass forms dA2, the gradients of W3, W2, then dA1 and the
// gradients of W1; Adam updates the parameters in place.  The weights are kept
// both row-major (flat layout, for Adam and the backward pass) and transposed
// (for the forward pass) so that the 32 lanes of a warp read consecutive words.
constexpr int kTrainMaxB = 128;
constexpr int kTrainThreads = 256;

struct TrainShared {
    float P[NP];
    float G[NP];
    float w1t[I * H];
    float w2t[H * H];
    float x[kTrainMaxB * I];
    float t[kTrainMaxB * O];
    float a1[kTrainMaxB * H];
    float a2[kTrainMaxB * H];  // pre-activations of layer 2, later dA1
    float da[kTrainMaxB * H];  // dA2
    float dy[kTrainMaxB * O];
    float loss;
};

__device__ void refresh_transposed(TrainShared &s)
{
    for (int e = threadIdx.x; e < H * I; e += blockDim.x)
        s.w1t[(e % I) * H + e / I] = s.P[oW1 + e];
    for (int e = threadIdx.x; e < H * H; e += blockDim.x)
        s.w2t[(e % H) * H + e / H] = s.P[oW2 + e];
}

__global__ void __launch_bounds__(kTrainThreads, 1)
    mlp_train_kernel(float *__restrict__ Pg, float *__restrict__ M, float *__restrict__ Vv,
                     const float *__restrict__ X, const float *__restrict__ T, int64_t N, int B, int64_t steps,
                     int64_t t0, float lr, float b1, float b2, float eps, float *__restrict__ loss_out)
{
    extern __shared__ __align__(16) unsigned char raw[];
    TrainShared &s = *reinterpret_cast<TrainShared *>(raw);
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int e = tid; e < NP; e += nt)
        s.P[e] = Pg[e];
    __syncthreads();
    refresh_transposed(s);
    const float invB = 1.f / (float)B;
    for (int64_t st = 0; st < steps; ++st) {
        for (int e = tid; e < B * I; e += nt)
            s.x[e] = X[((st * B + e / I) % N) * I + e % I];
        for (int e = tid; e < B * O; e += nt)
            s.t[e] = T[((st * B + e / O) % N) * O + e % O];
        if (tid == 0)
            s.loss = 0.f;
        __syncthreads();
        // A1[b][u] = b1[u] + sum_i W1[u][i] x[b][i]
        for (int e = tid; e < B * H; e += nt) {
            const int b = e / H, u = e % H;
            float acc = s.P[ob1 + u];
#pragma unroll
            for (int i = 0; i < I; ++i)
                acc = fmaf(s.w1t[i * H + u], s.x[b * I + i], acc);
            s.a1[e] = acc;
        }
        __syncthreads();
        // A2[b][u] = b2[u] + sum_i W2[u][i] relu(A1[b][i])
        for (int e = tid; e < B * H; e += nt) {
            const int b = e / H, u = e % H;
            float acc = s.P[ob2 + u];
#pragma unroll 8
            for (int i = 0; i < H; ++i)
                acc = fmaf(s.w2t[i * H + u], fmaxf(s.a1[b * H + i], 0.f), acc);
            s.a2[e] = acc;
        }
        __syncthreads();
        // y[b][o], dY = (y - t) / B, loss
        for (int e = tid; e < B * O; e += nt) {
            const int b = e / O, o = e % O;
            float acc = s.P[ob3 + o];
            for (int j = 0; j < H; ++j) {
                const int u = (j + (tid & 31)) & (H - 1);  // skewed so lanes hit distinct banks
                acc = fmaf(s.P[oW3 + o * H + u], fmaxf(s.a2[b * H + u], 0.f), acc);
            }
            const float err = acc - s.t[e];
            s.dy[e] = err * invB;
            atomicAdd(&s.loss, 0.5f * err * err * invB);
        }
        __syncthreads();
        // gW3[o][u], gb3[o]; dA2[b][u]
        for (int e = tid; e < O * H; e += nt) {
            const int o = e / H, u = e % H;
            float acc = 0.f;
            for (int b = 0; b < B; ++b)
                acc = fmaf(s.dy[b * O + o], fmaxf(s.a2[b * H + u], 0.f), acc);
            s.G[oW3 + e] = acc;
        }
        if (tid < O) {
            float acc = 0.f;
            for (int b = 0; b < B; ++b)
                acc += s.dy[b * O + tid];
            s.G[ob3 + tid] = acc;
        }
        for (int e = tid; e < B * H; e += nt) {
            const int b = e / H, u = e % H;
            const float g = s.P[oW3 + u] * s.dy[b * O] + s.P[oW3 + H + u] * s.dy[b * O + 1];
            s.da[e] = s.a2[e] > 0.f ? g : 0.f;
        }
        __syncthreads();
        // gW2[u][i] = sum_b dA2[b][u] relu(A1[b][i]); gb2[u]
        for (int e = tid; e < H * H; e += nt) {
            const int u = e / H, i = e % H;
            float acc = 0.f;
            for (int b = 0; b < B; ++b)
                acc = fmaf(s.da[b * H + u], fmaxf(s.a1[b * H + i], 0.f), acc);
            s.G[oW2 + e] = acc;
        }
        for (int u = tid; u < H; u += nt) {
            float acc = 0.f;
            for (int b = 0; b < B; ++b)
                acc += s.da[b * H + u];
            s.G[ob2 + u] = acc;
        }
        __syncthreads();
        // dA1[b][i] = relu'(A1[b][i]) sum_u W2[u][i] dA2[b][u]  (into a2)
        for (int e = tid; e < B * H; e += nt) {
            const int b = e / H, i = e % H;
            float acc = 0.f;
#pragma unroll 8
            for (int u = 0; u < H; ++u)
                acc = fmaf(s.P[oW2 + u * H + i], s.da[b * H + u], acc);
            s.a2[e] = s.a1[e] > 0.f ? acc : 0.f;
        }
        __syncthreads();
        // gW1[u][i] = sum_b dA1[b][u] x[b][i]; gb1[u]
        for (int e = tid; e < H * I; e += nt) {
            const int u = e / I, i = e % I;
            float acc = 0.f;
            for (int b = 0; b < B; ++b)
                acc = fmaf(s.a2[b * H + u], s.x[b * I + i], acc);
            s.G[oW1 + e] = acc;
        }
        for (int u = tid; u < H; u += nt) {
            float acc = 0.f;
            for (int b = 0; b < B; ++b)
                acc += s.a2[b * H + u];
            s.G[ob1 + u] = acc;
        }
        __syncthreads();
        const int64_t t = t0 + st + 1;
        const float c1 = 1.f - powf(b1, (float)t), c2 = 1.f - powf(b2, (float)t);
        for (int e = tid; e < NP; e += nt) {
            float p = s.P[e], m = M[e], v = Vv[e];
            adam1(p, s.G[e], m, v, lr, b1, b2, eps, c1, c2);
            s.P[e] = p;
            M[e] = m;
            Vv[e] = v;
        }
        if (tid == 0 && loss_out)
            loss_out[st] = s.loss;
        __syncthreads();
        refresh_transposed(s);
    }
    __syncthreads();
    for (int e = tid; e < NP; e += nt)
        Pg[e] = s.P[e];
}

// bfloat16 evaluation: weights and inputs rounded to bfloat16, float32
// accumulation; outputs mapped to eps = max(0, exp(y0) - 0.01) * alpha and
// e_s = clamp(round(exp(y1)), es_min, es_max).
__global__ void __launch_bounds__(kMlpWarps * 32)
    mlp_predict_kernel(const float *__restrict__ P, const float *__restrict__ X, int64_t B, float alpha, int es_min,
                       int es_max, float *__restrict__ eps_out, int32_t *__restrict__ es_out)
{
    extern __shared__ __align__(16) unsigned char raw[];
    MlpShared &s = *reinterpret_cast<MlpShared *>(raw);
    float *scratch = reinterpret_cast<float *>(raw + sizeof(MlpShared));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    load_params(s, P);
    __syncthreads();
    float *f = reinterpret_cast<float *>(&s);
    for (int e = threadIdx.x; e < (int)(sizeof(MlpShared) / sizeof(float)); e += blockDim.x)
        f[e] = __bfloat162float(__float2bfloat16_rn(f[e]));
    __syncthreads();
    float *h1 = scratch + warp * H;
    for (int64_t b = (int64_t)blockIdx.x * kMlpWarps + warp; b < B; b += (int64_t)gridDim.x * kMlpWarps) {
        float x[I];
#pragma unroll
        for (int i = 0; i < I; ++i)
            x[i] = __bfloat162float(__float2bfloat16_rn(X[b * I + i]));
        float a1[2], a2[2], h2[2], y[O];
        forward_warp(s, x, h1, lane, a1, a2, h2, y);
        if (lane == 0) {
            eps_out[b] = fmaxf(0.f, expf(y[0]) - 0.01f) * alpha;
            const float e = rintf(expf(fminf(y[1], 20.f)));
            es_out[b] = (int32_t)fminf(fmaxf(e, (float)es_min), (float)es_max);
        }
        __syncwarp();
    }
}

size_t shared_bytes(int copies, int scratch_per_warp) { return copies * sizeof(MlpShared) + kMlpWarps * scratch_per_warp * sizeof(float); }

int set_smem(const void *fn, size_t bytes)
{
    ONNG_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes), "mlp: smem attribute");
    return ONNG_OK;
}

int grid_for(int64_t B) { return (int)std::max<int64_t>(1, std::min<int64_t>((B + kMlpWarps - 1) / kMlpWarps, num_sms() * 2)); }

}  // namespace
}  // namespace onng

using namespace onng;

extern "C" int onng_mlp_nparam(void) { return NP; }

extern "C" int onng_mlp_forward(const float *P, const float *X, int64_t B, float *Y, onng_stream_t stream)
{
    ONNG_RANGE("onng_mlp_forward");
    ONNG_REQUIRE(B >= 0, ONNG_E_INVAL, "onng_mlp_forward: negative batch");
    if (B == 0)
        return ONNG_OK;
    ONNG_REQUIRE(P && X && Y, ONNG_E_INVAL, "onng_mlp_forward: NULL pointer");
    const size_t sm = shared_bytes(1, H);
    int st = set_smem(reinterpret_cast<const void *>(mlp_forward_kernel), sm);
    if (st)
        return st;
    mlp_forward_kernel<<<grid_for(B), kMlpWarps * 32, sm, to_cuda(stream)>>>(P, X, B, Y);
    return check_launch("onng_mlp_forward");
}

extern "C" int onng_mlp_loss_grad(const float *P, const float *X, const float *T, int64_t B, float *G, float *loss,
                                  onng_stream_t stream)
{
    ONNG_RANGE("onng_mlp_loss_grad");
    ONNG_REQUIRE(B >= 1, ONNG_E_INVAL, "onng_mlp_loss_grad: empty batch");
    ONNG_REQUIRE(P && X && T && G && loss, ONNG_E_INVAL, "onng_mlp_loss_grad: NULL pointer");
    cudaStream_t s = to_cuda(stream);
    ONNG_CUDA_TRY(cudaMemsetAsync(G, 0, sizeof(float) * NP, s), "onng_mlp_loss_grad: clear");
    ONNG_CUDA_TRY(cudaMemsetAsync(loss, 0, sizeof(float), s), "onng_mlp_loss_grad: clear");
    const size_t sm = shared_bytes(2, 2 * H);
    int st = set_smem(reinterpret_cast<const void *>(mlp_loss_grad_kernel), sm);
    if (st)
        return st;
    mlp_loss_grad_kernel<<<grid_for(B), kMlpWarps * 32, sm, s>>>(P, X, T, B, G, loss);
    return check_launch("onng_mlp_loss_grad");
}

extern "C" int onng_mlp_adam(float *P, const float *G, float *M, float *V, int64_t t, float lr, float beta1,
                             float beta2, float eps, onng_stream_t stream)
{
    ONNG_RANGE("onng_mlp_adam");
    ONNG_REQUIRE(t >= 1 && lr > 0.f, ONNG_E_INVAL, "onng_mlp_adam: bad step or rate");
    ONNG_REQUIRE(P && G && M && V, ONNG_E_INVAL, "onng_mlp_adam: NULL pointer");
    mlp_adam_kernel<<<(NP + 255) / 256, 256, 0, to_cuda(stream)>>>(P, G, M, V, t, lr, beta1, beta2, eps);
    return check_launch("onng_mlp_adam");
}

extern "C" int onng_mlp_train(float *P, float *M, float *V, const float *X, const float *T, int64_t N, int32_t batch,
                              int64_t steps, int64_t t0, float lr, float *G, float *losses, onng_stream_t stream)
{
    ONNG_RANGE("onng_mlp_train");
    (void)G;
    ONNG_REQUIRE(N >= 1 && batch >= 1 && steps >= 0 && t0 >= 0 && lr > 0.f, ONNG_E_INVAL, "onng_mlp_train: bad sizes");
    ONNG_REQUIRE(batch <= kTrainMaxB, ONNG_E_UNSUPPORTED, "onng_mlp_train: batch must be <= %d", kTrainMaxB);
    ONNG_REQUIRE(P && M && V && X && T, ONNG_E_INVAL, "onng_mlp_train: NULL pointer");
    if (steps == 0)
        return ONNG_OK;
    const size_t sm = sizeof(TrainShared);
    int st = set_smem(reinterpret_cast<const void *>(mlp_train_kernel), sm);
    if (st)
        return st;
    mlp_train_kernel<<<1, kTrainThreads, sm, to_cuda(stream)>>>(P, M, V, X, T, N, batch, steps, t0, lr, 0.9f, 0.999f,
                                                                1e-8f, losses);
    return check_launch("onng_mlp_train");
}

extern "C" int onng_mlp_predict(const float *P, const float *X, int64_t B, float alpha, int32_t es_min, int32_t es_max,
                                float *eps_out, int32_t *es_out, onng_stream_t stream)
{
    ONNG_RANGE("onng_mlp_predict");
    ONNG_REQUIRE(B >= 0 && es_min >= 1 && es_max >= es_min && alpha >= 0.f, ONNG_E_INVAL, "onng_mlp_predict: bad args");
    if (B == 0)
        return ONNG_OK;
    ONNG_REQUIRE(P && X && eps_out && es_out, ONNG_E_INVAL, "onng_mlp_predict: NULL pointer");
    const size_t sm = shared_bytes(1, H);
    int st = set_smem(reinterpret_cast<const void *>(mlp_predict_kernel), sm);
    if (st)
        return st;
    mlp_predict_kernel<<<grid_for(B), kMlpWarps * 32, sm, to_cuda(stream)>>>(P, X, B, alpha, es_min, es_max, eps_out,
                                                                            es_out);
    return check_launch("onng_mlp_predict");
}
