// Seed selection for the search.  The paper takes seeds from NGT's vp-tree
// (Sec. 2, Table 5), which it does not specify, and also reports a random
// variant (Sec. 3.2, Fig. 5(a)).  Two deterministic rules are provided:
//   random: n_seed distinct ids per query from a SplitMix64 stream (Steele,
//           Lea and Flood 2014) that starts at global_seed + q * 2^32; a draw z
//           maps to floor(z * n / 2^64) and repeats are redrawn.
//   pivot:  the n_seed nearest (distance, id) of the P pivots floor(t * n / P).
#include <algorithm>
#include <climits>
#include <cmath>

#include "common.cuh"
#include "warp_sort.cuh"

namespace onng {
namespace {

constexpr int kMaxSeed = 64;

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
// by direct difference in float32, coordinate by coordinate.  After each tile a
// warp per query folds the tile's 64 (distance, pivot index) keys into the
// query's sorted list of its 64 best so far.  Only keys below the list's
// n_seed-th take part: a few of them are inserted one at a time; when many
// qualify (the first tiles) the list and the tile are bitonic-sorted together.
// Every pivot row is read once per CTA instead of once per query, and shared
// memory (33 KB, so that five CTAs share an SM) does not grow with the pivot
// count.
constexpr int kPivQ = 16;
constexpr int kPivT = 64;
constexpr int kPivD = 64;
constexpr int kPivThreads = 256;
constexpr int kPivMinCta = 5;
constexpr int kPivRow = kPivD + 4;  // padded tile row: conflict-free 16-byte reads
constexpr int kPivInsertMax = 16;   // at most this many qualifying keys: insert one by one
constexpr unsigned long long kNoKey = ~0ull;

size_t pivot_smem_bytes()
{
    return sizeof(float) * ((size_t)kPivQ * kPivD + (size_t)kPivT * kPivRow + (size_t)kPivQ * kPivT) +
           sizeof(unsigned long long) * (size_t)kPivQ * kMaxSeed;
}

// Inserts `key` (warp-uniform, absent from the list) into the ascending list
// whose element e = h * 32 + lane is b[h] of lane `lane`; the last element drops.
__device__ __forceinline__ void list_insert(unsigned long long (&b)[2], unsigned long long key, int lane)
{
    const int pos = __popc(__ballot_sync(0xffffffffu, b[0] < key)) + __popc(__ballot_sync(0xffffffffu, b[1] < key));
    const unsigned long long up0 = __shfl_up_sync(0xffffffffu, b[0], 1);
    const unsigned long long up1 = __shfl_up_sync(0xffffffffu, b[1], 1);
    const unsigned long long last0 = __shfl_sync(0xffffffffu, b[0], 31);
    const int e1 = 32 + lane;
    b[0] = lane < pos ? b[0] : (lane == pos ? key : up0);
    b[1] = e1 < pos ? b[1] : (e1 == pos ? key : (lane == 0 ? last0 : up1));
}

__global__ void __launch_bounds__(kPivThreads, kPivMinCta)
    seeds_pivot_kernel(const float *__restrict__ X, int64_t n, int d, const float *__restrict__ Q, int64_t nq, int P,
                       int n_seed, int32_t *__restrict__ out)
{
    extern __shared__ __align__(16) float psm[];
    float *qs = psm;                     // [kPivQ][kPivD]
    float *ts = qs + kPivQ * kPivD;      // [kPivT][kPivRow]
    float *dist = ts + kPivT * kPivRow;  // [kPivQ][kPivT]: the tile's squared distances
    unsigned long long *best = reinterpret_cast<unsigned long long *>(dist + kPivQ * kPivT);  // [kPivQ][kMaxSeed]
    const int tid = threadIdx.x;
    const int qi = tid >> 4, pj = tid & 15;
    const int warp = tid >> 5, lane = tid & 31;
    const int64_t q0 = (int64_t)blockIdx.x * kPivQ;
    const int d4 = d >> 2;
    const int m = n_seed < P ? n_seed : P;
    for (int e = tid; e < kPivQ * kMaxSeed; e += kPivThreads)
        best[e] = kNoKey;
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
                for (int mm = 0; mm < 4; ++mm) {
                    const float4 b = reinterpret_cast<const float4 *>(ts + (pj + 16 * mm) * kPivRow)[c];
                    float u = a.x - b.x;
                    acc[mm] = fmaf(u, u, acc[mm]);
                    u = a.y - b.y;
                    acc[mm] = fmaf(u, u, acc[mm]);
                    u = a.z - b.z;
                    acc[mm] = fmaf(u, u, acc[mm]);
                    u = a.w - b.w;
                    acc[mm] = fmaf(u, u, acc[mm]);
                }
            }
        }
#pragma unroll
        for (int mm = 0; mm < 4; ++mm)
            dist[qi * kPivT + pj + 16 * mm] = acc[mm];
        __syncthreads();
        // fold the tile into each query's best list: keys (distance bits, pivot
        // index) order as (distance, index) for non-negative distances; NaN
        // distances (non-finite input) are never taken
        for (int i = warp; i < kPivQ; i += kPivThreads / 32) {
            unsigned long long *bl = best + i * kMaxSeed;
            unsigned long long b[2], v[2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int t = t0 + lane + 32 * h;
                const float dv = dist[i * kPivT + lane + 32 * h];
                v[h] = (t < P && !isnan(dv)) ? pack_key(dv, t) : kNoKey;
                b[h] = bl[lane + 32 * h];
            }
            const bool hi = m > 32;  // the n_seed-th key sits in b[1]
            unsigned long long kth = __shfl_sync(0xffffffffu, hi ? b[1] : b[0], (m - 1) & 31);
            unsigned in0 = __ballot_sync(0xffffffffu, v[0] < kth);
            unsigned in1 = __ballot_sync(0xffffffffu, v[1] < kth);
            const int cnt = __popc(in0) + __popc(in1);
            if (cnt > kPivInsertMax) {
                unsigned long long s[4] = {b[0], b[1], v[0], v[1]};
                warp_bitonic_sort<4>(s, lane);
                b[0] = s[0];
                b[1] = s[1];
            } else {
                while (in0 | in1) {
                    const bool first = in0 != 0;
                    const unsigned mk = first ? in0 : in1;
                    const int src = __ffs(mk) - 1;
                    if (first)
                        in0 &= in0 - 1;
                    else
                        in1 &= in1 - 1;
                    const unsigned long long key = __shfl_sync(0xffffffffu, first ? v[0] : v[1], src);
                    if (key < kth) {
                        list_insert(b, key, lane);
                        kth = __shfl_sync(0xffffffffu, hi ? b[1] : b[0], (m - 1) & 31);
                    }
                }
            }
            if (cnt) {
                bl[lane] = b[0];
                bl[32 + lane] = b[1];
            }
            __syncwarp();
        }
    }
    __syncthreads();
    for (int i = warp; i < kPivQ; i += kPivThreads / 32) {
        const int64_t q = q0 + i;
        if (q >= nq)
            break;
        for (int r = lane; r < n_seed; r += 32) {
            const unsigned long long key = r < m ? best[i * kMaxSeed + r] : kNoKey;
            out[q * n_seed + r] = key == kNoKey ? -1 : (int32_t)((int64_t)(unsigned)(key & 0xFFFFFFFFull) * n / P);
        }
    }
}
}  // namespace
}  // namespace onng

using namespace onng;

extern "C" int onng_seeds_random(uint64_t global_seed, int64_t nq, int64_t n, int32_t n_seed, int32_t *out,
                                 onng_stream_t stream)
{
    ONNG_RANGE("onng_seeds_random");
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
    ONNG_RANGE("onng_seeds_pivot");
    (void)ws;
    (void)ws_bytes;
    ONNG_REQUIRE(nq >= 0 && n > 0 && n <= INT32_MAX, ONNG_E_INVAL, "onng_seeds_pivot: bad sizes");
    ONNG_REQUIRE(d > 0 && d % 4 == 0, ONNG_E_UNSUPPORTED, "onng_seeds_pivot: d must be a positive multiple of 4");
    ONNG_REQUIRE(n_pivot >= 1, ONNG_E_UNSUPPORTED, "onng_seeds_pivot: n_pivot must be >= 1");
    ONNG_REQUIRE(n_seed >= 1 && n_seed <= kMaxSeed, ONNG_E_UNSUPPORTED, "onng_seeds_pivot: n_seed in [1, %d]",
                 kMaxSeed);
    if (nq == 0)
        return ONNG_OK;
    ONNG_REQUIRE(X && Q && out, ONNG_E_INVAL, "onng_seeds_pivot: NULL pointer");
    ONNG_REQUIRE(aligned16(X) && aligned16(Q), ONNG_E_INVAL, "onng_seeds_pivot: X and Q must be 16-byte aligned");
    const int P = (int)std::min<int64_t>(n_pivot, n);
    const size_t sm = pivot_smem_bytes();
    ONNG_CUDA_TRY(cudaFuncSetAttribute(reinterpret_cast<const void *>(seeds_pivot_kernel),
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm),
                  "onng_seeds_pivot: smem attribute");
    seeds_pivot_kernel<<<(unsigned)((nq + kPivQ - 1) / kPivQ), kPivThreads, sm, to_cuda(stream)>>>(X, n, d, Q, nq, P,
                                                                                                  n_seed, out);
    return check_launch("onng_seeds_pivot");
}
