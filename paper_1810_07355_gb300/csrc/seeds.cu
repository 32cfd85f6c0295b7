// Seed selection for the search.  The paper takes seeds from NGT's vp-tree
// (Sec. 2, Table 5), which it does not specify, and also reports a random
// variant (Sec. 3).  Two deterministic rules are provided:
//   random: n_seed distinct ids per query from a SplitMix64 stream (Steele,
//           Lea and Flood 2014) that starts at global_seed + q * 2^32; a draw z
//           maps to floor(z * n / 2^64) and repeats are redrawn.
//   pivot:  the n_seed nearest (distance, id) of the P pivots floor(t * n / P).
#include <algorithm>
#include <climits>
#include <cmath>

#include "common.cuh"

namespace onng {
namespace {

constexpr int kMaxSeed = 64;
constexpr int kMaxPivot = 2048;

__device__ __forceinline__ unsigned long long splitmix64(unsigned long long &state)
{
    unsigned long long z = (state += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__global__ void seeds_random_kernel(unsigned long long global_seed, int64_t nq, int64_t n, int n_seed,
                                    int32_t *__restrict__ out)
{
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= nq)
        return;
    int32_t *o = out + q * n_seed;
    const int m = (int64_t)n_seed < n ? n_seed : (int)n;
    for (int t = m; t < n_seed; ++t)
        o[t] = -1;
    if (2 * (int64_t)m > n) {
        for (int t = 0; t < m; ++t)
            o[t] = t;
        return;
    }
    int32_t chosen[kMaxSeed];
    unsigned long long st = global_seed + ((unsigned long long)q << 32);
    int got = 0;
    while (got < m) {
        const unsigned long long z = splitmix64(st);
        const int32_t id = (int32_t)__umul64hi(z, (unsigned long long)n);
        bool dup = false;
        for (int t = 0; t < got; ++t)
            dup |= chosen[t] == id;
        if (!dup)
            chosen[got++] = id;
    }
    for (int t = 0; t < m; ++t)
        o[t] = chosen[t];
}

// Nearest-pivot seeds, one CTA per kPivQ queries.  The CTA walks the pivots in
// tiles of kPivT: each tile (in chunks of kPivD coordinates) and the CTA's
// queries are staged in shared memory, and thread (i, j) accumulates the
// squared distances of query i to pivots j, j + 16, j + 32, j + 48 of the tile
// by direct difference in float32.  All P distances of a query stay in shared
// memory; then one warp per query takes n_seed rounds of an argmin over
// (distance, pivot index).  Every pivot row is read once per CTA instead of once
// per query.
constexpr int kPivQ = 16;
constexpr int kPivT = 64;
constexpr int kPivD = 128;
constexpr int kPivThreads = 256;
constexpr int kPivRow = kPivD + 4;  // padded tile row: conflict-free 16-byte reads

size_t pivot_smem_bytes(int P)
{
    return sizeof(float) * ((size_t)kPivQ * kPivD + (size_t)kPivT * kPivRow + (size_t)kPivQ * P);
}

__global__ void __launch_bounds__(kPivThreads)
    seeds_pivot_kernel(const float *__restrict__ X, int64_t n, int d, const float *__restrict__ Q, int64_t nq, int P,
                       int n_seed, int32_t *__restrict__ out)
{
    extern __shared__ __align__(16) float psm[];
    float *qs = psm;                      // [kPivQ][kPivD]
    float *ts = qs + kPivQ * kPivD;       // [kPivT][kPivRow]
    float *dist = ts + kPivT * kPivRow;   // [kPivQ][P]
    const int tid = threadIdx.x;
    const int qi = tid >> 4, pj = tid & 15;
    const int64_t q0 = (int64_t)blockIdx.x * kPivQ;
    const int d4 = d >> 2;
    for (int t0 = 0; t0 < P; t0 += kPivT) {
        float acc[4] = {0.f, 0.f, 0.f, 0.f};
        for (int c0 = 0; c0 < d4; c0 += kPivD / 4) {
            __syncthreads();
            // stage the queries' and the tile's coordinates c0*4 .. c0*4 + kPivD (zero past d)
            for (int e = tid; e < kPivQ * (kPivD / 4); e += kPivThreads) {
                const int r = e / (kPivD / 4), c = e % (kPivD / 4);
                float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                if (q0 + r < nq && c0 + c < d4)
                    v = __ldg(reinterpret_cast<const float4 *>(Q + (q0 + r) * d) + c0 + c);
                reinterpret_cast<float4 *>(qs + r * kPivD)[c] = v;
            }
            for (int e = tid; e < kPivT * (kPivD / 4); e += kPivThreads) {
                const int r = e / (kPivD / 4), c = e % (kPivD / 4);
                float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                if (t0 + r < P && c0 + c < d4) {
                    const int64_t id = (int64_t)(t0 + r) * n / P;
                    v = __ldg(reinterpret_cast<const float4 *>(X + id * d) + c0 + c);
                }
                reinterpret_cast<float4 *>(ts + r * kPivRow)[c] = v;
            }
            __syncthreads();
            const float4 *qr = reinterpret_cast<const float4 *>(qs + qi * kPivD);
#pragma unroll 4
            for (int c = 0; c < kPivD / 4; ++c) {
                const float4 a = qr[c];
#pragma unroll
                for (int m = 0; m < 4; ++m) {
                    const float4 b = reinterpret_cast<const float4 *>(ts + (pj + 16 * m) * kPivRow)[c];
                    float u = a.x - b.x;
                    acc[m] = fmaf(u, u, acc[m]);
                    u = a.y - b.y;
                    acc[m] = fmaf(u, u, acc[m]);
                    u = a.z - b.z;
                    acc[m] = fmaf(u, u, acc[m]);
                    u = a.w - b.w;
                    acc[m] = fmaf(u, u, acc[m]);
                }
            }
        }
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            const int t = t0 + pj + 16 * m;
            if (t < P)
                dist[qi * P + t] = acc[m];
        }
    }
    __syncthreads();
    const int warp = tid >> 5, lane = tid & 31;
    const int m = n_seed < P ? n_seed : P;
    for (int i = warp; i < kPivQ; i += kPivThreads / 32) {
        const int64_t q = q0 + i;
        if (q >= nq)
            break;
        float *dw = dist + i * P;
        for (int r = 0; r < m; ++r) {
            float bd = INFINITY;
            int bt = INT_MAX;
            for (int t = lane; t < P; t += 32) {
                const float v = dw[t];
                if (v < bd || (v == bd && t < bt)) {
                    bd = v;
                    bt = t;
                }
            }
#pragma unroll
            for (int off = 16; off >= 1; off >>= 1) {
                const float od = __shfl_xor_sync(0xffffffffu, bd, off);
                const int ot = __shfl_xor_sync(0xffffffffu, bt, off);
                if (od < bd || (od == bd && ot < bt)) {
                    bd = od;
                    bt = ot;
                }
            }
            if (bt >= P) {  // only NaN distances left (non-finite input): no further seeds
                for (int e = r + lane; e < n_seed; e += 32)
                    out[q * n_seed + e] = -1;
                break;
            }
            if (lane == 0) {
                out[q * n_seed + r] = (int32_t)((int64_t)bt * n / P);
                dw[bt] = __int_as_float(0x7fc00000);  // NaN: never selected again
            }
            __syncwarp();
        }
        for (int r = m + lane; r < n_seed; r += 32)
            out[q * n_seed + r] = -1;
    }
}

}  // namespace
}  // namespace onng

using namespace onng;

extern "C" int onng_seeds_random(uint64_t global_seed, int64_t nq, int64_t n, int32_t n_seed, int32_t *out,
                                 onng_stream_t stream)
{
    ONNG_REQUIRE(nq >= 0 && n > 0 && n <= INT32_MAX, ONNG_E_INVAL, "onng_seeds_random: bad sizes");
    ONNG_REQUIRE(n_seed >= 1 && n_seed <= kMaxSeed, ONNG_E_UNSUPPORTED, "onng_seeds_random: n_seed must be in [1, %d]",
                 kMaxSeed);
    if (nq == 0)
        return ONNG_OK;
    ONNG_REQUIRE(out, ONNG_E_INVAL, "onng_seeds_random: NULL output");
    seeds_random_kernel<<<(unsigned)((nq + 127) / 128), 128, 0, to_cuda(stream)>>>(global_seed, nq, n, n_seed, out);
    return check_launch("onng_seeds_random");
}

extern "C" size_t onng_seeds_pivot_workspace_bytes(int64_t n, int32_t d, int32_t n_pivot)
{
    (void)n;
    (void)d;
    (void)n_pivot;
    return 0;
}

extern "C" int onng_seeds_pivot(const float *X, int64_t n, int32_t d, const float *Q, int64_t nq, int32_t n_pivot,
                                int32_t n_seed, int32_t *out, void *ws, size_t ws_bytes, onng_stream_t stream)
{
    (void)ws;
    (void)ws_bytes;
    ONNG_REQUIRE(nq >= 0 && n > 0 && n <= INT32_MAX, ONNG_E_INVAL, "onng_seeds_pivot: bad sizes");
    ONNG_REQUIRE(d > 0 && d % 4 == 0, ONNG_E_UNSUPPORTED, "onng_seeds_pivot: d must be a positive multiple of 4");
    ONNG_REQUIRE(n_pivot >= 1 && n_pivot <= kMaxPivot, ONNG_E_UNSUPPORTED, "onng_seeds_pivot: n_pivot in [1, %d]",
                 kMaxPivot);
    ONNG_REQUIRE(n_seed >= 1 && n_seed <= kMaxSeed, ONNG_E_UNSUPPORTED, "onng_seeds_pivot: n_seed in [1, %d]",
                 kMaxSeed);
    if (nq == 0)
        return ONNG_OK;
    ONNG_REQUIRE(X && Q && out, ONNG_E_INVAL, "onng_seeds_pivot: NULL pointer");
    ONNG_REQUIRE(aligned16(X) && aligned16(Q), ONNG_E_INVAL, "onng_seeds_pivot: X and Q must be 16-byte aligned");
    const int P = (int)std::min<int64_t>(n_pivot, n);
    const size_t sm = pivot_smem_bytes(P);
    ONNG_CUDA_TRY(cudaFuncSetAttribute(reinterpret_cast<const void *>(seeds_pivot_kernel),
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm),
                  "onng_seeds_pivot: smem attribute");
    seeds_pivot_kernel<<<(unsigned)((nq + kPivQ - 1) / kPivQ), kPivThreads, sm, to_cuda(stream)>>>(X, n, d, Q, nq, P,
                                                                                                  n_seed, out);
    return check_launch("onng_seeds_pivot");
}
