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

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

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

template <int KC, int NBUF = BUF>
__device__ void merge_row(int r, int64_t grow, unsigned long long *__restrict__ best, unsigned long long *__restrict__ buf,
                          float *s_thr, int *s_cnt, int lane)
{
    static_assert(KC + NBUF <= 512, "merge sorts 512 keys");
    const int cnt = s_cnt[r];
    unsigned long long v[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        const int e = i * 32 + lane;
        if (e < KC)
            v[i] = best[grow * KC + e];
        else if (e - KC < cnt)
            v[i] = buf[grow * NBUF + (e - KC)];
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

// ---------------------------------------------------------------- tensor cores
//
// knn_tc_kernel: the same sweep with the dot products on the 5th-generation
// tensor cores, for byte-valued inputs (integers in [0, 255], e.g. 8-bit image
// descriptors) at d = 64 or 128: they are exact in bfloat16, every product and
// partial sum is an integer below 2^23, so the float32 accumulation, and with it
// the ranking, is exact.
//
// One CTA owns 128 query rows (the A operand, loaded once by TMA) and sweeps the
// base in tiles of 256 rows (the B operand, a two-stage TMA ring).  Shared
// memory holds both operands K-major in 128-byte-swizzled atoms (8 rows x 64
// bfloat16).  Warp 9 allocates 512 TMEM columns (two 128 x 256 float32
// accumulators); its lane 0 issues tcgen05.mma (M = 128, N = 256, K = 16 per
// instruction) and commits to mbarriers that free the smem stage and hand the
// accumulator to the epilogue.  Warp 8 lane 0 issues the TMA loads.  Warps 0-7
// read the accumulators with tcgen05.ld (warp w sees TMEM lanes 32 (w % 4) ..
// +31, i.e. one query row per thread, and columns 128 (w / 4) .. +127), form
// |q|^2 + |x|^2 - 2 q.x, filter against the row's threshold and append to the
// row's candidate buffer; rows whose buffer may not absorb another tile are
// merged between tiles.  Every mbarrier wait gives up after 2 s, records an
// error code and lets all roles reach the teardown, where TMEM is freed.
constexpr int TC_M = 128, TC_N = 256, TC_BUF = 384, TC_STAGES = 2;
constexpr int TC_EPI = 256;                 // epilogue threads (8 warps)
constexpr int TC_THREADS = TC_EPI + 64;     // + TMA warp + MMA warp
constexpr unsigned long long TC_TIMEOUT_NS = 2000000000ull;

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
                 : "=r"(ok)
                 : "r"(smem_u32(bar)), "r"(parity)
                 : "memory");
    return ok != 0;
}
__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Bounded wait on a phase; false (and *err set) after TC_TIMEOUT_NS or when
// another role has already given up.
__device__ bool mbar_wait(uint64_t *bar, uint32_t parity, int *err, int code)
{
    if (mbar_try_wait(bar, parity))
        return true;
    const uint64_t t0 = global_ns();
    for (uint32_t it = 0;; ++it) {
        if (mbar_try_wait(bar, parity))
            return true;
        if ((it & 63) == 0) {
            if (*reinterpret_cast<volatile int *>(err) != 0)
                return false;
            if (global_ns() - t0 > TC_TIMEOUT_NS) {
                atomicCAS(err, 0, code);
                return false;
            }
        }
    }
}
// Bounded wait for a role's own work in flight before teardown: unlike
// mbar_wait it keeps waiting when another role has already given up; on its
// own timeout it records `code` in *err (global memory) and returns.
__device__ void mbar_drain(uint64_t *bar, uint32_t parity, int *err, int code)
{
    const uint64_t t0 = global_ns();
    for (uint32_t it = 0;; ++it) {
        if (mbar_try_wait(bar, parity))
            return;
        if ((it & 63) == 0 && global_ns() - t0 > TC_TIMEOUT_NS) {
            atomicCAS(err, 0, code);
            return;
        }
    }
}
__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int c0, int c1, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(smem_u32(bar))
        : "memory");
}
// Shared-memory matrix descriptor: K-major operand in 128-byte-swizzled atoms of
// 8 rows x 128 bytes stacked 1024 bytes apart (start address >> 4, leading
// offset unused, stride offset 1024 >> 4, descriptor version 1, swizzle 128B).
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr)
{
    uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)(1024 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}
// Instruction descriptor, kind::f16: float32 accumulator, bfloat16 A and B, both
// K-major, N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t umma_idesc(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
__device__ __forceinline__ void umma_bf16(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc)
{
    asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                 " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(dtmem),
                 "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
                 : "memory");
}
__device__ __forceinline__ void umma_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32])
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
                 "%13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, "
                 "[%32];"
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                   "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
                   "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]),
                   "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]),
                   "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void epi_sync() { asm volatile("bar.sync 1, %0;" ::"n"(TC_EPI) : "memory"); }

template <int KA> struct TcSmem {
    static constexpr int A_ATOM = TC_M * 128;   // bytes of one 64-wide K atom of A
    static constexpr int B_ATOM = TC_N * 128;
    static constexpr int A_BYTES = KA * A_ATOM;
    static constexpr int B_STAGE = KA * B_ATOM;
    // alignment slack, operands, then barriers, TMEM address, flags, thresholds,
    // counts and the base norms of two tiles
    static constexpr int BYTES = 1024 + A_BYTES + TC_STAGES * B_STAGE + 4096;
};

template <int KC, int KA>
__global__ void __launch_bounds__(TC_THREADS, 1)
    knn_tc_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, int64_t n,
                  int64_t nq, int64_t self_offset, const float *__restrict__ xn, const float *__restrict__ qn,
                  unsigned long long *__restrict__ best, unsigned long long *__restrict__ buf, int *err)
{
    using L = TcSmem<KA>;
    extern __shared__ unsigned char tc_raw[];
    unsigned char *base = reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(tc_raw) + 1023) & ~uintptr_t(1023));
    unsigned char *sA = base;
    unsigned char *sB = base + L::A_BYTES;
    uint64_t *bars = reinterpret_cast<uint64_t *>(sB + TC_STAGES * L::B_STAGE);
    uint64_t *full = bars, *empty = bars + TC_STAGES, *accf = bars + 2 * TC_STAGES, *acce = accf + 2, *abar = acce + 2;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(abar + 1);
    int *s_ok = reinterpret_cast<int *>(tmem_slot + 1);
    float *s_thr = reinterpret_cast<float *>(s_ok + 4);
    int *s_cnt = reinterpret_cast<int *>(s_thr + TC_M);
    float *s_xn = reinterpret_cast<float *>(s_cnt + TC_M);  // [2][TC_N], +inf past n

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t row0 = (int64_t)blockIdx.x * TC_M;
    const int64_t tiles = (n + TC_N - 1) / TC_N;

    if (tid == 0) {
        for (int s = 0; s < TC_STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&accf[b], 1);
            mbar_init(&acce[b], TC_EPI);
        }
        mbar_init(abar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 9) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_u32(tmem_slot))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    for (int r = tid; r < TC_M; r += blockDim.x) {
        s_thr[r] = INFINITY;
        s_cnt[r] = 0;
    }
    for (int e = tid; e < TC_M * KC; e += blockDim.x) {
        const int64_t gr = row0 + e / KC;
        if (gr < nq)
            best[gr * KC + e % KC] = EMPTY_KEY;
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 8) {
        // ------------------------------------------------ TMA producer
        if (lane == 0) {
            int64_t issued = 0;
            mbar_expect_tx(abar, L::A_BYTES);
            for (int a = 0; a < KA; ++a)
                tma_load_2d(sA + a * L::A_ATOM, &tmA, a * 64, (int)row0, abar);
            for (int64_t t = 0; t < tiles; ++t) {
                const int s = (int)(t % TC_STAGES);
                if (t >= TC_STAGES && !mbar_wait(&empty[s], (uint32_t)(((t / TC_STAGES) & 1) ^ 1), err, 1))
                    break;
                mbar_expect_tx(&full[s], L::B_STAGE);
                for (int a = 0; a < KA; ++a)
                    tma_load_2d(sB + s * L::B_STAGE + a * L::B_ATOM, &tmB, a * 64, (int)(t * TC_N), &full[s]);
                issued = t + 1;
            }
            // our copies in flight complete before the CTA may exit (bounded)
            mbar_drain(abar, 0, err, 6);
            for (int64_t t = issued > TC_STAGES ? issued - TC_STAGES : 0; t < issued; ++t)
                mbar_drain(&full[t % TC_STAGES], (uint32_t)((t / TC_STAGES) & 1), err, 6);
        }
    } else if (warp == 9) {
        // ------------------------------------------------ MMA issuer
        if (lane == 0) {
            constexpr uint32_t idesc = umma_idesc(TC_M, TC_N);
            int64_t done = 0;
            bool ok = mbar_wait(abar, 0, err, 2);
            for (int64_t t = 0; ok && t < tiles; ++t) {
                const int s = (int)(t % TC_STAGES), b = (int)(t & 1);
                if (!mbar_wait(&full[s], (uint32_t)((t / TC_STAGES) & 1), err, 3))
                    break;
                if (t >= 2 && !mbar_wait(&acce[b], (uint32_t)(((t >> 1) & 1) ^ 1), err, 4))
                    break;
                tc_fence_after();
                const uint32_t aa = smem_u32(sA), bb = smem_u32(sB + s * L::B_STAGE);
#pragma unroll
                for (int kk = 0; kk < 4 * KA; ++kk) {
                    const uint32_t off = (uint32_t)((kk & 3) * 32);  // 16 bf16 = 32 bytes inside the atom
                    const uint64_t ad = umma_desc(aa + (kk >> 2) * L::A_ATOM + off);
                    const uint64_t bd = umma_desc(bb + (kk >> 2) * L::B_ATOM + off);
                    umma_bf16(tmem + (uint32_t)(b * TC_N), ad, bd, idesc, kk > 0 ? 1u : 0u);
                }
                umma_commit(&empty[s]);
                umma_commit(&accf[b]);
                done = t + 1;
            }
            // the MMAs issued so far complete before TMEM is freed (bounded)
            if (done > 0)
                mbar_drain(&accf[(done - 1) & 1], (uint32_t)(((done - 1) >> 1) & 1), err, 7);
        }
    } else {
        // ------------------------------------------------ epilogue (warps 0-7)
        // Thread (warp w, lane l) owns query row r = 32 (w % 4) + l and columns
        // 128 (w / 4) .. +127 of each tile.  The tile's base norms are staged in
        // shared memory one tile ahead (+inf past n, so no bounds test is needed);
        // the self column is cleared from a chunk's hit mask, and only hits leave
        // the fast path.
        const int qd = warp & 3, half = warp >> 2;
        const int r = qd * 32 + lane;
        const int64_t grow = row0 + r;
        const bool row_ok = grow < nq;
        const float qnr = row_ok ? qn[grow] : 0.f;
        const int64_t self = (self_offset >= 0 && row_ok) ? self_offset + grow : -1;
        float thr = row_ok ? INFINITY : -INFINITY;
        s_xn[tid] = tid < n ? 0.5f * xn[tid] : INFINITY;
        // the half norm this thread stages for the next tile, loaded one tile ahead
        // so that its latency never sits in front of a barrier
        float xn_next = TC_N + tid < n ? 0.5f * xn[TC_N + tid] : INFINITY;
        epi_sync();
        for (int64_t t = 0; t < tiles; ++t) {
            const int b = (int)(t & 1);
            if (tid == 0)
                s_ok[0] = mbar_wait(&accf[b], (uint32_t)((t >> 1) & 1), err, 5) ? 1 : 0;
            epi_sync();
            if (!s_ok[0])
                break;
            tc_fence_after();
            const int64_t col0 = t * TC_N + half * 128;
            const float *hs = s_xn + b * TC_N + half * 128;  // |x|^2 / 2 of the tile's columns
            const int64_t self_local = self - col0;  // in [0, 128) when the self column is here
            // d^2 = |q|^2 + |x|^2 - 2 q.x < thr  <=>  q.x - |x|^2 / 2 > (|q|^2 - thr) / 2, every term
            // an exact integer or half-integer here; the running maximum of the left side
            // decides a chunk, and only a chunk with a hit forms distances
            const float tr = 0.5f * (qnr - thr);
#pragma unroll 1
            for (int c = 0; c < 4; ++c) {
                uint32_t v[32];
                tmem_ld32(tmem + ((uint32_t)(qd * 32) << 16) + (uint32_t)(b * TC_N + half * 128 + c * 32), v);
                float mx = -INFINITY;
#pragma unroll
                for (int j = 0; j < 32; ++j)
                    mx = fmaxf(mx, __uint_as_float(v[j]) - hs[c * 32 + j]);
                if (!(mx > tr))
                    continue;
                uint32_t hit = 0;
#pragma unroll
                for (int j = 0; j < 32; ++j)
                    hit |= (__uint_as_float(v[j]) - hs[c * 32 + j] > tr ? 1u : 0u) << j;
                const int64_t sj = self_local - c * 32;
                if (sj >= 0 && sj < 32)
                    hit &= ~(1u << (int)sj);
                while (hit) {
                    const int j = __ffs(hit) - 1;
                    hit &= hit - 1;
                    float aj = __uint_as_float(v[0]) - hs[c * 32];
#pragma unroll
                    for (int u = 1; u < 32; ++u)
                        aj = u == j ? __uint_as_float(v[u]) - hs[c * 32 + u] : aj;
                    const float dj = fmaxf(qnr - 2.f * aj, 0.f);
                    const int pos = atomicAdd(&s_cnt[r], 1);
                    buf[grow * TC_BUF + pos] = pack_key(dj, (int)(col0 + c * 32 + j));
                }
            }
            tc_fence_before();
            mbar_arrive(&acce[b]);
            // stage the next tile's half norms into the other half of s_xn, and load
            // those of the tile after it
            s_xn[(b ^ 1) * TC_N + tid] = xn_next;
            {
                const int64_t nc = (t + 2) * TC_N + tid;
                xn_next = nc < n ? 0.5f * xn[nc] : INFINITY;
            }
            epi_sync();
            const bool last = t + 1 == tiles;
            for (int rr = warp; rr < TC_M; rr += TC_EPI / 32) {
                const int64_t gr = row0 + rr;
                if (gr >= nq)
                    break;
                const int cnt = s_cnt[rr];
                if (cnt > TC_BUF - TC_N || (last && cnt > 0))
                    merge_row<KC, TC_BUF>(rr, gr, best, buf, s_thr, s_cnt, lane);
            }
            epi_sync();
            if (row_ok)
                thr = s_thr[r];
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 9) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem) : "memory");
    }
}

// Sets *flag if any of the values is not an integer in [0, 255] (byte-valued
// descriptors: exact in bfloat16, and at d <= 128 every squared norm, dot product,
// |x|^2 / 2 and distance of the tensor-core path is an exact float32 below 2^23).
__global__ void bf16_exact_kernel(const float *__restrict__ x, int64_t count, int *flag)
{
    int bad = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
        const float v = x[i];
        bad |= !(v == rintf(v) && v >= 0.f && v <= 255.f);
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0)
        atomicOr(flag, 1);
}

__global__ void f32_to_bf16_kernel(const float *__restrict__ x, int64_t count, __nv_bfloat16 *__restrict__ y)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
        y[i] = __float2bfloat16_rn(x[i]);
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

// 2-D bf16 tensor map over rows x d (row-major), box 64 x box_rows, 128B swizzle,
// zero fill outside the matrix.
int make_map(CUtensorMap *m, const void *ptr, int64_t rows, int d, int box_rows)
{
    auto fn = encode_fn();
    if (!fn)
        return set_error(ONNG_E_CUDA, "onng_knn: cuTensorMapEncodeTiled unavailable");
    cuuint64_t dims[2] = {(cuuint64_t)d, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)d * 2};
    cuuint32_t box[2] = {64, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(ptr), dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS)
        return set_error(ONNG_E_CUDA, "onng_knn: tensor map encode failed (%d)", (int)r);
    return ONNG_OK;
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

template <int KC, int KA>
int launch_tc_kc(const CUtensorMap &ma, const CUtensorMap &mb, int64_t n, int64_t nq, int64_t self_offset,
                 const float *xn, const float *qn, unsigned long long *best, unsigned long long *bufp, int *err,
                 cudaStream_t s)
{
    const size_t smem = TcSmem<KA>::BYTES;
    ONNG_CUDA_TRY(cudaFuncSetAttribute(reinterpret_cast<const void *>(knn_tc_kernel<KC, KA>),
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
                  "onng_knn: tensor kernel smem attribute");
    knn_tc_kernel<KC, KA><<<(unsigned)((nq + TC_M - 1) / TC_M), TC_THREADS, smem, s>>>(ma, mb, n, nq, self_offset, xn,
                                                                                     qn, best, bufp, err);
    return check_launch("onng_knn: tensor kernel");
}

int launch_tc(const float *X, int64_t n, int d, const float *Q, int64_t nq, int k, int kc, int64_t self_offset,
              int32_t *nbr, float *len, float *xn, float *qn, unsigned long long *best, unsigned long long *bufp,
              int *err, __nv_bfloat16 *xb, __nv_bfloat16 *qb, cudaStream_t s)
{
    const int gb = num_sms() * 8;
    f32_to_bf16_kernel<<<gb, 256, 0, s>>>(X, n * d, xb);
    f32_to_bf16_kernel<<<gb, 256, 0, s>>>(Q, nq * d, qb);
    int st = check_launch("onng_knn: bf16 copies");
    if (st)
        return st;
    CUtensorMap ma, mb;
    if ((st = make_map(&ma, qb, nq, d, TC_M)) || (st = make_map(&mb, xb, n, d, TC_N)))
        return st;
    const int ka = d / 64;
    if (kc == 32)
        st = ka == 1 ? launch_tc_kc<32, 1>(ma, mb, n, nq, self_offset, xn, qn, best, bufp, err, s)
                     : launch_tc_kc<32, 2>(ma, mb, n, nq, self_offset, xn, qn, best, bufp, err, s);
    else if (kc == 64)
        st = ka == 1 ? launch_tc_kc<64, 1>(ma, mb, n, nq, self_offset, xn, qn, best, bufp, err, s)
                     : launch_tc_kc<64, 2>(ma, mb, n, nq, self_offset, xn, qn, best, bufp, err, s);
    else
        st = ka == 1 ? launch_tc_kc<128, 1>(ma, mb, n, nq, self_offset, xn, qn, best, bufp, err, s)
                     : launch_tc_kc<128, 2>(ma, mb, n, nq, self_offset, xn, qn, best, bufp, err, s);
    if (st)
        return st;
    int code = 0;
    ONNG_CUDA_TRY(cudaMemcpyAsync(&code, err, sizeof(int), cudaMemcpyDeviceToHost, s), "onng_knn: error flag");
    ONNG_CUDA_TRY(cudaStreamSynchronize(s), "onng_knn: tensor kernel");
    if (code)
        return set_error(ONNG_E_LIMIT, "onng_knn: tensor-core pipeline wait timed out (role %d)", code);
    switch (kc) {
    case 32:
        knn_final_kernel<32><<<(unsigned)((nq * 32 + 255) / 256), 256, 0, s>>>(X, d, Q, nq, best, k, nbr, len);
        break;
    case 64:
        knn_final_kernel<64><<<(unsigned)((nq * 32 + 255) / 256), 256, 0, s>>>(X, d, Q, nq, best, k, nbr, len);
        break;
    default:
        knn_final_kernel<128><<<(unsigned)((nq * 32 + 255) / 256), 256, 0, s>>>(X, d, Q, nq, best, k, nbr, len);
    }
    return check_launch("onng_knn: final kernel");
}

}  // namespace
}  // namespace onng

using namespace onng;

extern "C" size_t onng_knn_workspace_bytes(int64_t n, int32_t d, int64_t nq, int32_t k)
{
    int kc = pick_kc(k);
    WsCarver c(nullptr);
    c.take<float>((size_t)std::max<int64_t>(n, 1));
    c.take<float>((size_t)std::max<int64_t>(nq, 1));
    c.take<unsigned long long>((size_t)std::max<int64_t>(nq, 1) * (kc ? kc : 32));
    c.take<unsigned long long>((size_t)std::max<int64_t>(nq, 1) * std::max(BUF, TC_BUF));
    c.take<int>(64);
    c.take<__nv_bfloat16>((size_t)std::max<int64_t>(n, 1) * std::max(d, 1));
    c.take<__nv_bfloat16>((size_t)std::max<int64_t>(nq, 1) * std::max(d, 1));
    return c.used;
}

extern "C" int onng_knn(const float *X, int64_t n, int32_t d, const float *Q, int64_t nq, int32_t k,
                        int64_t self_offset, int32_t *nbr, float *len, void *ws, size_t ws_bytes, onng_stream_t stream)
{
    ONNG_RANGE("onng_knn");
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
    unsigned long long *bufp = c.take<unsigned long long>((size_t)nq * std::max(BUF, TC_BUF));
    int *flags = c.take<int>(64);
    __nv_bfloat16 *xb = c.take<__nv_bfloat16>((size_t)std::max<int64_t>(n, 1) * d);
    __nv_bfloat16 *qb = c.take<__nv_bfloat16>((size_t)nq * d);
    cudaStream_t s = to_cuda(stream);
    if (n > 0)
        norms_kernel<<<(unsigned)((n * 32 + 255) / 256), 256, 0, s>>>(X, n, d, xn);
    norms_kernel<<<(unsigned)((nq * 32 + 255) / 256), 256, 0, s>>>(Q, nq, d, qn);
    int st = check_launch("onng_knn: norms");
    if (st)
        return st;
    // tensor-core path: d of 64 or 128, k + 16 <= 128, byte-valued inputs
    if (n > 0 && (d == 64 || d == 128) && kc <= 128 && n <= INT32_MAX - TC_N) {
        ONNG_CUDA_TRY(cudaMemsetAsync(flags, 0, 64 * sizeof(int), s), "onng_knn: clear flags");
        const int gb = num_sms() * 8;
        bf16_exact_kernel<<<gb, 256, 0, s>>>(X, n * d, flags);
        bf16_exact_kernel<<<gb, 256, 0, s>>>(Q, nq * d, flags);
        int inexact = 1;
        ONNG_CUDA_TRY(cudaMemcpyAsync(&inexact, flags, sizeof(int), cudaMemcpyDeviceToHost, s), "onng_knn: flag");
        ONNG_CUDA_TRY(cudaStreamSynchronize(s), "onng_knn: exactness check");
        if (!inexact)
            return launch_tc(X, n, d, Q, nq, k, kc, self_offset, nbr, len, xn, qn, best, bufp, flags + 1, xb, qb, s);
    }
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
    ONNG_RANGE("onng_build_knng");
    ONNG_REQUIRE(k <= n - 1 || n == 0, ONNG_E_INVAL, "onng_build_knng: k must be <= n - 1");
    return onng_knn(X, n, d, X, n, k, 0, nbr, len, ws, ws_bytes, stream);
}
