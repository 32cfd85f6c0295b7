// Exact k-nearest-neighbour lists (the exact kNN graph that replaces the
// paper's approximate graph, Sec. 2.5) without materialising the n x n matrix.
//
// knn_tile_kernel: a CTA owns 128 query rows and sweeps all base columns in
// tiles of 128.  The tile of squared distances |q|^2 + |x|^2 - 2 q.x is formed
// in registers (8 x 8 per thread, float32 FMA).  Entries below the row's
// running threshold are appended to a per-row candidate buffer in global
// memory (mostly L2); when a buffer may not absorb another tile it is merged
// with the row's best list (a warp-wide bitonic sort in registers) and the
// threshold drops to the list's last entry.  The best list keeps KC >= k + 16
// entries so that rounding in the expanded form cannot push a true neighbour
// out of it.
//
// knn_final_kernel: rescoring of the KC survivors of each row by direct
// difference sum (q_j - x_j)^2 in float32, ordering by (distance, id) and
// output of the first k as ids and Euclidean lengths.
//
// Integer-valued inputs whose squared norms stay below 2^23 are ranked exactly:
// every product, partial sum and the expanded form are exact in float32.
#include <algorithm>
#include <cmath>

#include "common.cuh"
#include "warp_sort.cuh"

namespace onng {
namespace {

constexpr int BM = 128, BN = 128, BK = 16, NT = 256;
constexpr int BUF = 256;  // candidate buffer entries per row (>= 2 * BN)
constexpr unsigned long long EMPTY_KEY = 0x7F800000FFFFFFFFull;  // (+inf, id -1)

__device__ __forceinline__ float key_dist(unsigned long long k) { return __uint_as_float((unsigned)(k >> 32)); }
__device__ __forceinline__ int key_id(unsigned long long k) { return (int)(unsigned)(k & 0xFFFFFFFFull); }

__global__ void norms_kernel(const float *__restrict__ X, int64_t n, int d, float *__restrict__ out)
{
    const int lane = threadIdx.x & 31;
    const int64_t row = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (row >= n)
        return;
    const float4 *p = reinterpret_cast<const float4 *>(X + row * d);
    float s = 0.f;
    for (int c = lane; c < (d >> 2); c += 32) {
        float4 v = __ldg(p + c);
        s = fmaf(v.x, v.x, s);
        s = fmaf(v.y, v.y, s);
        s = fmaf(v.z, v.z, s);
        s = fmaf(v.w, v.w, s);
    }
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1)
        s += __shfl_xor_sync(0xffffffffu, s, off);
    if (lane == 0)
        out[row] = s;
}

// Loads a BK-wide slab of 128 rows (rows >= nrows and dims >= d read as 0) and
// stores it transposed: S[k][m].
__device__ __forceinline__ void load_slab(const float *__restrict__ M, int64_t row0, int64_t nrows, int d, int k0,
                                          float (*S)[BM + 4], int tid)
{
#pragma unroll
    for (int t = 0; t < (BM * BK / 4) / NT; ++t) {
        const int f = tid + t * NT;
        const int m = f >> 2;
        const int kq = (f & 3) << 2;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (row0 + m < nrows && k0 + kq < d)
            v = __ldg(reinterpret_cast<const float4 *>(M + (row0 + m) * d + k0 + kq));
        S[kq + 0][m] = v.x;
        S[kq + 1][m] = v.y;
        S[kq + 2][m] = v.z;
        S[kq + 3][m] = v.w;
    }
}

template <int KC>
__device__ void merge_row(int r, int64_t grow, unsigned long long *__restrict__ best, unsigned long long *__restrict__ buf,
                          float *s_thr, int *s_cnt, int lane)
{
    const int cnt = s_cnt[r];
    unsigned long long v[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        const int e = i * 32 + lane;
        if (e < KC)
            v[i] = best[grow * KC + e];
        else if (e - KC < cnt)
            v[i] = buf[grow * BUF + (e - KC)];
        else
            v[i] = EMPTY_KEY;
    }
    warp_bitonic_sort<16>(v, lane);
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        const int e = i * 32 + lane;
        if (e < KC)
            best[grow * KC + e] = v[i];
    }
    const unsigned long long last = __shfl_sync(0xffffffffu, v[(KC - 1) >> 5], (KC - 1) & 31);
    __syncwarp();
    if (lane == 0) {
        s_thr[r] = key_dist(last);
        s_cnt[r] = 0;
    }
}

template <int KC>
__global__ void __launch_bounds__(NT, 2)
    knn_tile_kernel(const float *__restrict__ X, int64_t n, int d, const float *__restrict__ Q, int64_t nq,
                    int64_t self_offset, const float *__restrict__ xn, const float *__restrict__ qn,
                    unsigned long long *__restrict__ best, unsigned long long *__restrict__ buf)
{
    static_assert(KC + BUF <= 512, "merge sorts 512 keys");
    __shared__ __align__(16) float As[BK][BM + 4];
    __shared__ __align__(16) float Bs[BK][BN + 4];
    __shared__ float s_thr[BM];
    __shared__ int s_cnt[BM];
    __shared__ float s_qn[BM];

    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    const int lane = tid & 31, warp = tid >> 5;
    const int64_t row0 = (int64_t)blockIdx.x * BM;

    for (int r = tid; r < BM; r += NT) {
        s_thr[r] = INFINITY;
        s_cnt[r] = 0;
        s_qn[r] = row0 + r < nq ? qn[row0 + r] : 0.f;
    }
    for (int e = tid; e < BM * KC; e += NT) {
        const int64_t gr = row0 + e / KC;
        if (gr < nq)
            best[gr * KC + e % KC] = EMPTY_KEY;
    }
    __syncthreads();

    for (int64_t col0 = 0; col0 < n; col0 += BN) {
        float acc[8][8];
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
            for (int j = 0; j < 8; ++j)
                acc[i][j] = 0.f;
        for (int k0 = 0; k0 < d; k0 += BK) {
            load_slab(Q, row0, nq, d, k0, As, tid);
            load_slab(X, col0, n, d, k0, Bs, tid);
            __syncthreads();
#pragma unroll
            for (int kk = 0; kk < BK; ++kk) {
                float a[8], b[8];
                *reinterpret_cast<float4 *>(&a[0]) = *reinterpret_cast<const float4 *>(&As[kk][ty * 4]);
                *reinterpret_cast<float4 *>(&a[4]) = *reinterpret_cast<const float4 *>(&As[kk][64 + ty * 4]);
                *reinterpret_cast<float4 *>(&b[0]) = *reinterpret_cast<const float4 *>(&Bs[kk][tx * 4]);
                *reinterpret_cast<float4 *>(&b[4]) = *reinterpret_cast<const float4 *>(&Bs[kk][64 + tx * 4]);
#pragma unroll
                for (int i = 0; i < 8; ++i)
#pragma unroll
                    for (int j = 0; j < 8; ++j)
                        acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
            }
            __syncthreads();
        }
        // epilogue: squared distances, threshold filter, append to row buffers
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int r = (i < 4) ? ty * 4 + i : 64 + ty * 4 + (i - 4);
            const int64_t grow = row0 + r;
            if (grow >= nq)
                continue;
            const float thr = s_thr[r];
            const int64_t self = self_offset >= 0 ? self_offset + grow : -1;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int cl = (j < 4) ? tx * 4 + j : 64 + tx * 4 + (j - 4);
                const int64_t c = col0 + cl;
                if (c >= n || c == self)
                    continue;
                const float d2 = fmaxf(s_qn[r] + __ldg(xn + c) - 2.f * acc[i][j], 0.f);
                if (d2 < thr) {
                    const int pos = atomicAdd(&s_cnt[r], 1);
                    buf[grow * BUF + pos] = pack_key(d2, (int)c);
                }
            }
        }
        __syncthreads();
        const bool last_tile = col0 + BN >= n;
        for (int r = warp; r < BM; r += NT / 32) {
            const int64_t grow = row0 + r;
            if (grow >= nq)
                break;
            const int c = s_cnt[r];
            if (c > BUF - BN || (last_tile && c > 0))
                merge_row<KC>(r, grow, best, buf, s_thr, s_cnt, lane);
        }
        __syncthreads();
    }
}

// Rescores the KC survivors of each row by direct difference and writes the best k.
template <int KC>
__global__ void knn_final_kernel(const float *__restrict__ X, int d, const float *__restrict__ Q, int64_t nq,
                                 const unsigned long long *__restrict__ best, int k, int32_t *__restrict__ nbr,
                                 float *__restrict__ len)
{
    constexpr int PER = KC / 32;
    const int lane = threadIdx.x & 31;
    const int64_t row = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (row >= nq)
        return;
    unsigned long long v[PER];
    const float4 *q4 = reinterpret_cast<const float4 *>(Q + row * d);
#pragma unroll
    for (int i = 0; i < PER; ++i) {
        const unsigned long long key = best[row * KC + i * 32 + lane];
        const int id = key_id(key);
        // every lane walks the 32 candidates of this slice in turn
        float mine = INFINITY;
        for (int t = 0; t < 32; ++t) {
            const int cid = __shfl_sync(0xffffffffu, id, t);
            if (cid < 0)
                continue;
            const float4 *x4 = reinterpret_cast<const float4 *>(X + (int64_t)cid * d);
            float s = 0.f;
            for (int c = lane; c < (d >> 2); c += 32) {
                float4 a = __ldg(q4 + c), b = __ldg(x4 + c);
                float u = a.x - b.x;
                s = fmaf(u, u, s);
                u = a.y - b.y;
                s = fmaf(u, u, s);
                u = a.z - b.z;
                s = fmaf(u, u, s);
                u = a.w - b.w;
                s = fmaf(u, u, s);
            }
#pragma unroll
            for (int off = 16; off >= 1; off >>= 1)
                s += __shfl_xor_sync(0xffffffffu, s, off);
            if (lane == t)
                mine = s;
        }
        v[i] = id < 0 ? EMPTY_KEY : pack_key(mine, id);
    }
    if constexpr (PER >= 1) {
        if constexpr ((PER & (PER - 1)) == 0)
            warp_bitonic_sort<PER>(v, lane);
    }
#pragma unroll
    for (int i = 0; i < PER; ++i) {
        const int e = i * 32 + lane;
        if (e < k) {
            const int id = key_id(v[i]);
            nbr[row * k + e] = id;
            len[row * k + e] = id < 0 ? INFINITY : sqrtf(key_dist(v[i]));
        }
    }
}

int pick_kc(int k)
{
    for (int kc = 32; kc <= 256; kc <<= 1)
        if (k + 16 <= kc)
            return kc;
    return 0;
}

template <int KC>
int launch(const float *X, int64_t n, int d, const float *Q, int64_t nq, int k, int64_t self_offset, int32_t *nbr,
           float *len, float *xn, float *qn, unsigned long long *best, unsigned long long *bufp, cudaStream_t s)
{
    knn_tile_kernel<KC><<<(unsigned)((nq + BM - 1) / BM), NT, 0, s>>>(X, n, d, Q, nq, self_offset, xn, qn, best, bufp);
    int st = check_launch("onng_knn: tile kernel");
    if (st)
        return st;
    knn_final_kernel<KC><<<(unsigned)((nq * 32 + 255) / 256), 256, 0, s>>>(X, d, Q, nq, best, k, nbr, len);
    return check_launch("onng_knn: final kernel");
}

}  // namespace
}  // namespace onng

using namespace onng;

extern "C" size_t onng_knn_workspace_bytes(int64_t n, int32_t d, int64_t nq, int32_t k)
{
    (void)d;
    int kc = pick_kc(k);
    WsCarver c(nullptr);
    c.take<float>((size_t)std::max<int64_t>(n, 1));
    c.take<float>((size_t)std::max<int64_t>(nq, 1));
    c.take<unsigned long long>((size_t)std::max<int64_t>(nq, 1) * (kc ? kc : 32));
    c.take<unsigned long long>((size_t)std::max<int64_t>(nq, 1) * BUF);
    return c.used;
}

extern "C" int onng_knn(const float *X, int64_t n, int32_t d, const float *Q, int64_t nq, int32_t k,
                        int64_t self_offset, int32_t *nbr, float *len, void *ws, size_t ws_bytes, onng_stream_t stream)
{
    ONNG_REQUIRE(n >= 0 && nq >= 0 && n <= INT32_MAX, ONNG_E_INVAL, "onng_knn: bad sizes");
    ONNG_REQUIRE(d > 0 && d % 4 == 0, ONNG_E_UNSUPPORTED, "onng_knn: d must be a positive multiple of 4");
    ONNG_REQUIRE(k >= 1, ONNG_E_INVAL, "onng_knn: k must be >= 1");
    ONNG_REQUIRE(pick_kc(k) > 0, ONNG_E_UNSUPPORTED, "onng_knn: k must be <= 240");
    ONNG_REQUIRE(self_offset < 0 || self_offset + nq <= n, ONNG_E_INVAL, "onng_knn: self rows outside the base");
    if (nq == 0)
        return ONNG_OK;
    ONNG_REQUIRE(X && Q && nbr && len, ONNG_E_INVAL, "onng_knn: NULL pointer");
    ONNG_REQUIRE(aligned16(X) && aligned16(Q), ONNG_E_INVAL, "onng_knn: X and Q must be 16-byte aligned");
    const size_t need = onng_knn_workspace_bytes(n, d, nq, k);
    ONNG_REQUIRE(ws && ws_bytes >= need, ONNG_E_WORKSPACE, "onng_knn: workspace %zu < %zu bytes", ws_bytes, need);
    const int kc = pick_kc(k);
    WsCarver c(ws);
    float *xn = c.take<float>((size_t)std::max<int64_t>(n, 1));
    float *qn = c.take<float>((size_t)nq);
    unsigned long long *best = c.take<unsigned long long>((size_t)nq * kc);
    unsigned long long *bufp = c.take<unsigned long long>((size_t)nq * BUF);
    cudaStream_t s = to_cuda(stream);
    if (n > 0)
        norms_kernel<<<(unsigned)((n * 32 + 255) / 256), 256, 0, s>>>(X, n, d, xn);
    norms_kernel<<<(unsigned)((nq * 32 + 255) / 256), 256, 0, s>>>(Q, nq, d, qn);
    int st = check_launch("onng_knn: norms");
    if (st)
        return st;
    switch (kc) {
    case 32: return launch<32>(X, n, d, Q, nq, k, self_offset, nbr, len, xn, qn, best, bufp, s);
    case 64: return launch<64>(X, n, d, Q, nq, k, self_offset, nbr, len, xn, qn, best, bufp, s);
    case 128: return launch<128>(X, n, d, Q, nq, k, self_offset, nbr, len, xn, qn, best, bufp, s);
    default: return launch<256>(X, n, d, Q, nq, k, self_offset, nbr, len, xn, qn, best, bufp, s);
    }
}

extern "C" int onng_build_knng(const float *X, int64_t n, int32_t d, int32_t k, int32_t *nbr, float *len, void *ws,
                               size_t ws_bytes, onng_stream_t stream)
{
    ONNG_REQUIRE(k <= n - 1 || n == 0, ONNG_E_INVAL, "onng_build_knng: k must be <= n - 1");
    return onng_knn(X, n, d, X, n, k, 0, nbr, len, ws, ws_bytes, stream);
}
