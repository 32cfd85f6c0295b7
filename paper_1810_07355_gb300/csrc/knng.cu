// Exact k-nearest-neighbour lists (the exact kNN graph that replaces the
// paper's approximate graph, Sec. 2.6) without materialising the n x n matrix.
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
//
// Which sweep runs (onng_knn): byte-valued inputs at d = 64 / 128 take the
// tensor cores exactly (knn_tc_kernel); other non-integer inputs at d >= 32 take
// the tensor cores in a split bfloat16 form (knn_tcs_kernel) whose survivors are
// rescored; everything else, and problems smaller than one tile, the SIMT sweep.
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

// Rescores the survivors of each row by direct difference and writes the best k:
// NL lists of KC keys per row (list l of row r at best[l * lstride + r * KC]).
template <int KC, int NL = 1>
__global__ void knn_final_kernel(const float *__restrict__ X, int d, const float *__restrict__ Q, int64_t nq,
                                 const unsigned long long *__restrict__ best, int k, int32_t *__restrict__ nbr,
                                 float *__restrict__ len, int64_t lstride = 0)
{
    constexpr int PER = KC * NL / 32;
    const int lane = threadIdx.x & 31;
    const int64_t row = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (row >= nq)
        return;
    unsigned long long v[PER];
    const float4 *q4 = reinterpret_cast<const float4 *>(Q + row * d);
#pragma unroll
    for (int i = 0; i < PER; ++i) {
        const int e = i * 32 + lane;
        const unsigned long long key = best[(int64_t)(e / KC) * lstride + row * KC + e % KC];
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

// The byte-valued tensor-core form ranks exactly: its best lists are already in
// (squared distance, id) order with the exact integer squared distances a float32
// direct-difference rescore would recompute, so the first k entries are written
// as they are.
__global__ void knn_emit_kernel(int64_t nq, const unsigned long long *__restrict__ best, int kc, int k,
                                int32_t *__restrict__ nbr, float *__restrict__ len)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nq * k; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t row = e / k;
        const unsigned long long key = best[row * kc + e % k];
        const int id = key_id(key);
        nbr[e] = id;
        len[e] = id < 0 ? INFINITY : sqrtf(key_dist(key));
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
// One CTA owns 256 query rows, two blocks of 128 (the A operands, loaded once by
// TMA), and sweeps the base in tiles of 128 rows (the B operand, a three-stage
// TMA ring) that both row blocks share.  Shared memory holds the operands
// K-major in 128-byte-swizzled atoms (8 rows x 64 bfloat16).  Warp 9 allocates
// the 512 TMEM columns: for each row block two 128 x 128 float32 accumulators
// (tiles alternate between them).  Its lane 0 issues tcgen05.mma (M = 128,
// N = 128, K = 16 per instruction, both row blocks per K step) and commits to
// mbarriers that free the smem stage and hand the accumulators to the epilogue.
// Warp 8 lane 0 issues the TMA loads.
//
// Epilogue (warps 0-7): thread (w, l) owns query row 128 (w / 4) + 32 (w % 4) + l
// outright, reading it from TMEM lanes 32 (w % 4) .. +31 with tcgen05.ld.  Per
// 32-column chunk it takes the running maximum of q.x - |x|^2 / 2 (the half
// norms come from a padded global array, the same address for the whole warp);
// a chunk whose maximum passes the row's threshold appends its hits (|q|^2 +
// |x|^2 - 2 q.x below the threshold) to the row's candidate buffer.  A row whose
// buffer may not absorb another tile is merged into its sorted best list by its
// warp: the buffer is sorted (bitonic, in registers) and a half-cleaner against
// the reversed best list plus a bitonic merge keep the KC smallest.  No barrier
// couples the epilogue warps: each arrives on the accumulator's "empty" barrier
// when its TMEM reads are done and merges afterwards.  Every mbarrier wait gives
// up after 2 s, records an error code and lets all roles reach the teardown,
// where TMEM is freed.
constexpr int TC_M = 128, TC_N = 128, TC_BUF = 256;
constexpr int TC_RB = 2;                    // 128-row blocks per CTA
constexpr int TC_EAGER = 64;                // buffered keys that trigger a merge
constexpr int TC_ROWS = TC_M * TC_RB;       // query rows per CTA
constexpr int TC_EPI = 256;                 // epilogue threads (8 warps), one per row
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
// KA atoms per row: KA - 1 of data and the spare atom.  A holds the data atoms of
// both row blocks and one spare atom (1.0 in its first three columns for every
// row) that both blocks share; only its first K = 16 step is non-zero, so the MMA
// takes that step alone.
template <int KA> struct TcSmem {
    static constexpr int A_ATOM = TC_M * 128;   // bytes of one 64-wide K atom of a 128-row block
    static constexpr int B_ATOM = TC_N * 128;
    static constexpr int A_BYTES = (TC_RB * (KA - 1) + 1) * A_ATOM;
    static constexpr int B_STAGE = KA * B_ATOM;
    static constexpr int STAGES = 3;
    // alignment slack, operands, then barriers and the TMEM address
    static constexpr int BYTES = 1024 + A_BYTES + STAGES * B_STAGE + 256;
    static_assert(BYTES <= 232448, "more than 227 KB of shared memory");
};

// Compact warp sorts for the tensor-core epilogue: the stage loops run at run
// time (only the loop over a lane's registers is unrolled), so the code stays
// small enough for the instruction cache next to the epilogue's hot loop.
// Element e = i * 32 + lane lives in v[i] of lane `lane`.

// compare-exchange of registers i and i ^ JR (partners 32 JR elements apart),
// ascending where bit `size` of the element index is clear
template <int JR, int N>
__device__ __forceinline__ void cas_regs(unsigned long long (&v)[N], int lane, int size)
{
#pragma unroll
    for (int i = 0; i < N; ++i) {
        const int ii = i ^ JR;
        if (ii > i) {
            const bool asc = (((i << 5) | lane) & size) == 0;
            const unsigned long long a = v[i], b = v[ii];
            const bool sw = asc ? (a > b) : (a < b);
            v[i] = sw ? b : a;
            v[ii] = sw ? a : b;
        }
    }
}

// one bitonic step at distance j elements for sequences of length `size`
template <int N>
__device__ __forceinline__ void bitonic_step(unsigned long long (&v)[N], int lane, int size, int j)
{
    if (j >= 32) {
        const int jr = j >> 5;
        if constexpr (N >= 2)
            if (jr == 1)
                cas_regs<1>(v, lane, size);
        if constexpr (N >= 4)
            if (jr == 2)
                cas_regs<2>(v, lane, size);
        if constexpr (N >= 8)
            if (jr == 4)
                cas_regs<4>(v, lane, size);
    } else {
        const bool lower = (lane & j) == 0;
#pragma unroll
        for (int i = 0; i < N; ++i) {
            const bool asc = (((i << 5) | lane) & size) == 0;
            const unsigned long long o = __shfl_xor_sync(0xffffffffu, v[i], j);
            const bool take_min = lower == asc;
            v[i] = take_min ? (o < v[i] ? o : v[i]) : (o > v[i] ? o : v[i]);
        }
    }
}

// ascending sort of 32 N keys
template <int N> __device__ void warp_sort_compact(unsigned long long (&v)[N], int lane)
{
    static_assert(N == 1 || N == 2 || N == 4 || N == 8, "N in {1, 2, 4, 8}");
#pragma unroll 1
    for (int size = 2; size <= 32 * N; size <<= 1)
#pragma unroll 1
        for (int j = size >> 1; j > 0; j >>= 1)
            bitonic_step<N>(v, lane, size, j);
}

// ascending merge of a bitonic sequence of 32 N keys (one bitonic merge pass with
// every element's direction ascending)
template <int N> __device__ void warp_merge_compact(unsigned long long (&v)[N], int lane)
{
#pragma unroll 1
    for (int j = 16 * N; j > 0; j >>= 1)
        bitonic_step<N>(v, lane, 64 * N, j);
}

// The warp merges row gr's cnt buffered keys into its sorted best list of KC
// keys and returns the new threshold: the distance of list entry kth (< KC).
template <int KC>
__device__ __noinline__ float tc_merge_row(int64_t gr, int cnt, int kth, unsigned long long *__restrict__ best,
                                           const unsigned long long *__restrict__ buf, int lane)
{
    static_assert(KC <= TC_BUF && TC_BUF == 256, "the buffer sort holds 256 keys");
    constexpr int PB = KC / 32;
    unsigned long long a[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int e = i * 32 + lane;
        a[i] = e < cnt ? buf[gr * TC_BUF + e] : EMPTY_KEY;
    }
    // sort the smallest power-of-two prefix holding the cnt keys (the rest is +inf)
    if (cnt <= 64) {
        unsigned long long t[2] = {a[0], a[1]};
        warp_sort_compact<2>(t, lane);
        a[0] = t[0];
        a[1] = t[1];
    } else if (cnt <= 128) {
        unsigned long long t[4] = {a[0], a[1], a[2], a[3]};
        warp_sort_compact<4>(t, lane);
#pragma unroll
        for (int i = 0; i < 4; ++i)
            a[i] = t[i];
    } else {
        warp_sort_compact<8>(a, lane);
    }
    unsigned long long bv[PB], m[PB];
#pragma unroll
    for (int i = 0; i < PB; ++i)
        bv[i] = best[gr * KC + i * 32 + lane];
    // half-cleaner of (a[0 .. KC), reversed best): the smaller of each pair is a
    // bitonic sequence holding the KC smallest keys
#pragma unroll
    for (int i = 0; i < PB; ++i) {
        const unsigned long long br = __shfl_sync(0xffffffffu, bv[PB - 1 - i], 31 - lane);
        m[i] = a[i] < br ? a[i] : br;
    }
    warp_merge_compact<PB>(m, lane);
#pragma unroll
    for (int i = 0; i < PB; ++i)
        best[gr * KC + i * 32 + lane] = m[i];
    unsigned long long kv = m[0];
#pragma unroll
    for (int i = 1; i < PB; ++i)
        kv = (kth >> 5) == i ? m[i] : kv;
    return key_dist(__shfl_sync(0xffffffffu, kv, kth & 31));
}

// tcgen05.ld of 32 columns without the wait; tmem_wait32 completes it (its
// operands tie the registers to the wait, so nothing reads them earlier)
__device__ __forceinline__ void tmem_ld32_async(uint32_t taddr, uint32_t (&v)[32])
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
}
__device__ __forceinline__ void tmem_wait32(uint32_t (&v)[32])
{
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(v[0]), "+r"(v[1]), "+r"(v[2]), "+r"(v[3]), "+r"(v[4]), "+r"(v[5]), "+r"(v[6]), "+r"(v[7]),
                   "+r"(v[8]), "+r"(v[9]), "+r"(v[10]), "+r"(v[11]), "+r"(v[12]), "+r"(v[13]), "+r"(v[14]),
                   "+r"(v[15]), "+r"(v[16]), "+r"(v[17]), "+r"(v[18]), "+r"(v[19]), "+r"(v[20]), "+r"(v[21]),
                   "+r"(v[22]), "+r"(v[23]), "+r"(v[24]), "+r"(v[25]), "+r"(v[26]), "+r"(v[27]), "+r"(v[28]),
                   "+r"(v[29]), "+r"(v[30]), "+r"(v[31])
                 :
                 : "memory");
}

// the half norms of a chunk's 32 columns (loaded right before their use: a load
// one chunk ahead costs registers the kernel does not have at one CTA per SM)
__device__ __forceinline__ void load_h(float4 (&h)[8], const float4 *__restrict__ p)
{
#pragma unroll
    for (int i = 0; i < 8; ++i)
        h[i] = __ldg(p + i);
}

// tcgen05.ld of one column (each lane its own TMEM lane) and its wait
__device__ __forceinline__ uint32_t tmem_ld1(uint32_t taddr)
{
    uint32_t x;
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x1.b32 {%0}, [%1];\n\ttcgen05.wait::ld.sync.aligned;"
                 : "=r"(x)
                 : "r"(taddr)
                 : "memory");
    return x;
}

// One 32-column chunk of a row in the split float form: the running maximum of
// q.x - |x|^2 / 2 decides whether any column passes; then the whole warp visits
// the passing columns of all its rows once each, reading each back from TMEM
// (taddr = the chunk's first column; hc = the chunk's half norms).
__device__ __forceinline__ void tc_chunk(const uint32_t (&v)[32], const float4 (&hq)[8], uint32_t taddr,
                                         const float *__restrict__ hc, float tr, float qnr, int64_t cb, int64_t self,
                                         unsigned long long *__restrict__ brow, int &cnt)
{
    float a[32];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const float4 x = hq[i];
        a[4 * i] = __uint_as_float(v[4 * i]) - x.x;
        a[4 * i + 1] = __uint_as_float(v[4 * i + 1]) - x.y;
        a[4 * i + 2] = __uint_as_float(v[4 * i + 2]) - x.z;
        a[4 * i + 3] = __uint_as_float(v[4 * i + 3]) - x.w;
    }
    float m0 = a[0], m1 = a[1], m2 = a[2], m3 = a[3];
#pragma unroll
    for (int j = 4; j < 32; j += 4) {
        m0 = fmaxf(m0, a[j]);
        m1 = fmaxf(m1, a[j + 1]);
        m2 = fmaxf(m2, a[j + 2]);
        m3 = fmaxf(m3, a[j + 3]);
    }
    if (!__any_sync(0xffffffffu, fmaxf(fmaxf(m0, m1), fmaxf(m2, m3)) > tr))
        return;
    unsigned hit = 0;
#pragma unroll
    for (int j = 0; j < 32; ++j)
        hit |= (a[j] > tr ? 1u : 0u) << j;
    const int64_t sj = self - cb;
    if (sj >= 0 && sj < 32)
        hit &= ~(1u << (int)sj);
    unsigned cols = __reduce_or_sync(0xffffffffu, hit);
    while (cols) {
        const int j = __ffs(cols) - 1;
        cols &= cols - 1;
        const float x = __uint_as_float(tmem_ld1(taddr + (uint32_t)j)) - __ldg(hc + j);
        if ((hit >> j) & 1u)
            brow[cnt++] = pack_key(fmaxf(qnr - 2.f * x, 0.f), (int)(cb + j));
    }
}

// The byte-valued form of a chunk: the accumulator already holds
// v = q.x - floor(|x|^2 / 2) (the MMA adds the spare K atom's pieces), an integer,
// and v >= q.x - |x|^2 / 2, so v >= tr selects a superset of the hits; a candidate
// is corrected by the parity of |x|^2 (one bit per column in par, loaded only
// here) to a = q.x - |x|^2 / 2 and kept when a >= tr, i.e. d^2 <= thr.  The
// comparison is not strict because thr is the k-th distance so far here (ranking
// is exact, so the list needs no slack): a later column at that distance may still
// win its tie by id.  Columns past n (zero rows of the last tile) are skipped.
// Called by the whole warp: the candidate columns of all 32 rows are visited
// once each, reading that column back from TMEM (taddr = the chunk's first
// column), so no lane indexes its registers at run time.
__device__ __forceinline__ void tc_chunk_aug(const uint32_t (&v)[32], uint32_t taddr, float tr, float qnr, int64_t cb,
                                             int64_t self, int64_t n, const unsigned *__restrict__ par,
                                             unsigned long long *__restrict__ brow, int &cnt)
{
    const float *f = reinterpret_cast<const float *>(v);
    float m[8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
        m[i] = f[i];
#pragma unroll
    for (int j = 8; j < 32; j += 8)
#pragma unroll
        for (int i = 0; i < 8; ++i)
            m[i] = fmaxf(m[i], f[j + i]);
    const float mx = fmaxf(fmaxf(fmaxf(m[0], m[1]), fmaxf(m[2], m[3])), fmaxf(fmaxf(m[4], m[5]), fmaxf(m[6], m[7])));
    if (!__any_sync(0xffffffffu, mx >= tr))
        return;
    unsigned hit = 0;
#pragma unroll
    for (int j = 0; j < 32; ++j)
        hit |= (f[j] >= tr ? 1u : 0u) << j;
    const int64_t sj = self - cb;
    if (sj >= 0 && sj < 32)
        hit &= ~(1u << (int)sj);
    if (n - cb < 32)
        hit &= n - cb > 0 ? (1u << (int)(n - cb)) - 1u : 0u;
    unsigned cols = __reduce_or_sync(0xffffffffu, hit);
    if (!cols)
        return;
    const unsigned odd = __ldg(par + (cb >> 5));
    while (cols) {
        const int j = __ffs(cols) - 1;
        cols &= cols - 1;
        const float x = __uint_as_float(tmem_ld1(taddr + (uint32_t)j));
        if ((hit >> j) & 1u) {
            const float aj = x - ((odd >> j) & 1u ? 0.5f : 0.f);
            if (aj >= tr)
                brow[cnt++] = pack_key(fmaxf(qnr - 2.f * aj, 0.f), (int)(cb + j));
        }
    }
}

// Which base tiles a CTA sweeps, in order: its u-th tile is (t0 + g + u G) mod
// `all`, for u < count.  G CTAs share a row set and take every G-th tile (g = this
// CTA's share); t0 rotates a self-join's sweep to start at its own rows.
struct TileMap {
    int64_t all, t0, count;
    int G, g;
    __device__ TileMap(int64_t all_, int64_t t0_, int G_, int g_)
        : all(all_), t0(t0_), count((all_ - g_ + G_ - 1) / G_), G(G_), g(g_)
    {
    }
    __device__ __forceinline__ int64_t tile(int64_t u) const { return (t0 + g + u * G) % all; }
};

// The epilogue of the tensor-core kernels (warps 0-7; see knn_tc_kernel): one
// query row per thread, tile by tile from the TMEM accumulators (row block rb =
// warp / 4 at columns (2 rb + b) * TC_N, b = tile & 1).
// AUG: the byte-valued form (tc_chunk_aug with the parity bits `par`); otherwise
// the split float form (tc_chunk with the padded half norms `xh`).
template <int KC, bool AUG>
__device__ void tc_epilogue(uint64_t *accf, uint64_t *acce, uint32_t tmem, int warp, int lane, int64_t row0,
                            int64_t nq, int64_t n, const TileMap tm, int kth, int64_t self_offset,
                            const float *__restrict__ xh,
                            const unsigned *__restrict__ par, const float *__restrict__ qn,
                            unsigned long long *__restrict__ best, unsigned long long *__restrict__ buf, int *err)
{
    const int rb = warp >> 2, qd = warp & 3;
    const int64_t grow = row0 + rb * TC_M + qd * 32 + lane;
    const bool row_ok = grow < nq;
    const float qnr = row_ok ? qn[grow] : 0.f;
    const int64_t self = (self_offset >= 0 && row_ok) ? self_offset + grow : -1;
    float thr = row_ok ? INFINITY : -INFINITY;
    int cnt = 0;
    unsigned long long *brow = buf + (row_ok ? grow : 0) * TC_BUF;
    const uint32_t lane_base = tmem + ((uint32_t)(qd * 32) << 16) + (uint32_t)(rb * 2 * TC_N);
    for (int64_t t = 0; t < tm.count; ++t) {
        const int b = (int)(t & 1);
        const bool ok = mbar_wait(&accf[b], (uint32_t)((t >> 1) & 1), err, 5);
        if (!__all_sync(0xffffffffu, ok))
            break;
        tc_fence_after();
        const int64_t col0 = tm.tile(t) * TC_N;
        // d^2 = |q|^2 + |x|^2 - 2 q.x < thr  <=>  q.x - |x|^2 / 2 > (|q|^2 - thr) / 2, every
        // term an exact integer or half-integer for byte-valued inputs (approximate in
        // the split float form, whose survivors are rescored)
        const float tr = 0.5f * (qnr - thr);
        const float4 *h4 = reinterpret_cast<const float4 *>(xh + col0);
        const uint32_t tb = lane_base + (uint32_t)(b * TC_N);
        // TMEM loads run one chunk ahead of the filter (chunk pairs: va even, vb odd)
        uint32_t va[32], vb[32];
        float4 hq[8];
        tmem_ld32_async(tb, va);
        tmem_wait32(va);
#pragma unroll 1
        for (int c = 0; c < TC_N / 32; c += 2) {
            tmem_ld32_async(tb + (uint32_t)((c + 1) * 32), vb);
            if constexpr (AUG) {
                tc_chunk_aug(va, tb + (uint32_t)(c * 32), tr, qnr, col0 + c * 32, self, n, par, brow, cnt);
            } else {
                load_h(hq, h4 + c * 8);
                tc_chunk(va, hq, tb + (uint32_t)(c * 32), xh + col0 + c * 32, tr, qnr, col0 + c * 32, self, brow,
                         cnt);
            }
            tmem_wait32(vb);
            if (c + 2 < TC_N / 32)
                tmem_ld32_async(tb + (uint32_t)((c + 2) * 32), va);
            if constexpr (AUG) {
                tc_chunk_aug(vb, tb + (uint32_t)((c + 1) * 32), tr, qnr, col0 + (c + 1) * 32, self, n, par, brow,
                             cnt);
            } else {
                load_h(hq, h4 + (c + 1) * 8);
                tc_chunk(vb, hq, tb + (uint32_t)((c + 1) * 32), xh + col0 + (c + 1) * 32, tr, qnr,
                         col0 + (c + 1) * 32, self, brow, cnt);
            }
            if (c + 2 < TC_N / 32)
                tmem_wait32(va);
        }
        tc_fence_before();
        mbar_arrive(&acce[b]);
        // rows whose buffer may not absorb another tile, or holds TC_EAGER keys (an
        // earlier merge lowers the threshold, which saves later appends: cheaper
        // than the smaller sorts it costs), and all rows after the last tile
        const bool last = t + 1 == tm.count;
        unsigned need = __ballot_sync(0xffffffffu, row_ok && (cnt > TC_BUF - TC_N || cnt >= TC_EAGER ||
                                                              (last && cnt > 0)));
        while (need) {
            const int src = __ffs(need) - 1;
            need &= need - 1;
            const int64_t gr = __shfl_sync(0xffffffffu, grow, src);
            const int c = __shfl_sync(0xffffffffu, cnt, src);
            const float nt = tc_merge_row<KC>(gr, c, kth, best, buf, lane);
            if (lane == src) {
                thr = nt;
                cnt = 0;
            }
        }
    }
}

template <int KC, int KA>
__global__ void __launch_bounds__(TC_THREADS, 1)
    knn_tc_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, int64_t n,
                  int64_t nq, int k, int64_t self_offset, const unsigned *__restrict__ par, const float *__restrict__ qn,
                  unsigned long long *__restrict__ best, unsigned long long *__restrict__ buf, int *err)
{
    using L = TcSmem<KA>;
    extern __shared__ unsigned char tc_raw[];
    unsigned char *base = reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(tc_raw) + 1023) & ~uintptr_t(1023));
    unsigned char *sA = base;
    unsigned char *sB = base + L::A_BYTES;
    uint64_t *bars = reinterpret_cast<uint64_t *>(sB + L::STAGES * L::B_STAGE);
    uint64_t *full = bars, *empty = bars + L::STAGES, *accf = bars + 2 * L::STAGES, *acce = accf + 2, *abar = acce + 2;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(abar + 1);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t row0 = (int64_t)blockIdx.x * TC_ROWS;
    const int64_t tiles = (n + TC_N - 1) / TC_N;
    const int nrb = row0 + TC_M < nq ? TC_RB : 1;  // row blocks holding any query row
    // a self-join starts its sweep at the tile of its own rows and wraps around:
    // where nearby rows sit together, the thresholds fall within the first tiles
    const int64_t t0 = self_offset >= 0 ? ((self_offset + row0) / TC_N) % tiles : 0;

    if (tid == 0) {
        for (int s = 0; s < L::STAGES; ++s) {
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
    for (int e = tid; e < TC_ROWS * KC; e += blockDim.x) {
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
            mbar_expect_tx(abar, (nrb * (KA - 1) + 1) * L::A_ATOM);
            for (int rb = 0; rb < nrb; ++rb)
                for (int a = 0; a < KA - 1; ++a)
                    tma_load_2d(sA + (rb * (KA - 1) + a) * L::A_ATOM, &tmA, a * 64, (int)(row0 + rb * TC_M), abar);
            // the spare atom from block 0's rows: a valid row of block 1 sits 128 rows
            // past a valid row of block 0, and all valid rows carry the same 1.0s
            tma_load_2d(sA + TC_RB * (KA - 1) * L::A_ATOM, &tmA, (KA - 1) * 64, (int)row0, abar);
            for (int64_t t = 0; t < tiles; ++t) {
                const int s = (int)(t % L::STAGES);
                if (t >= L::STAGES && !mbar_wait(&empty[s], (uint32_t)(((t / L::STAGES) & 1) ^ 1), err, 1))
                    break;
                mbar_expect_tx(&full[s], L::B_STAGE);
                for (int a = 0; a < KA; ++a)
                    tma_load_2d(sB + s * L::B_STAGE + a * L::B_ATOM, &tmB, a * 64, (int)(((t + t0) % tiles) * TC_N),
                                &full[s]);
                issued = t + 1;
            }
            // our copies in flight complete before the CTA may exit (bounded)
            mbar_drain(abar, 0, err, 6);
            for (int64_t t = issued > L::STAGES ? issued - L::STAGES : 0; t < issued; ++t)
                mbar_drain(&full[t % L::STAGES], (uint32_t)((t / L::STAGES) & 1), err, 6);
        }
    } else if (warp == 9) {
        // ------------------------------------------------ MMA issuer
        if (lane == 0) {
            constexpr uint32_t idesc = umma_idesc(TC_M, TC_N);
            int64_t done = 0;
            bool ok = mbar_wait(abar, 0, err, 2);
            for (int64_t t = 0; ok && t < tiles; ++t) {
                const int s = (int)(t % L::STAGES), b = (int)(t & 1);
                if (!mbar_wait(&full[s], (uint32_t)((t / L::STAGES) & 1), err, 3))
                    break;
                if (t >= 2 && !mbar_wait(&acce[b], (uint32_t)(((t >> 1) & 1) ^ 1), err, 4))
                    break;
                tc_fence_after();
                const uint32_t bb = smem_u32(sB + s * L::B_STAGE);
#pragma unroll
                for (int rb = 0; rb < TC_RB; ++rb) {
                    if (rb >= nrb)
                        break;
                    const uint32_t aa = smem_u32(sA + rb * (KA - 1) * L::A_ATOM);
                    const uint32_t dt = tmem + (uint32_t)((rb * 2 + b) * TC_N);
#pragma unroll
                    for (int kk = 0; kk < 4 * (KA - 1); ++kk) {
                        const uint32_t off = (uint32_t)((kk & 3) * 32);  // 16 bf16 = 32 bytes inside the atom
                        const uint64_t ad = umma_desc(aa + (kk >> 2) * L::A_ATOM + off);
                        const uint64_t bd = umma_desc(bb + (kk >> 2) * L::B_ATOM + off);
                        umma_bf16(dt, ad, bd, idesc, kk > 0 ? 1u : 0u);
                    }
                    // the spare atom's first K step adds -floor(|x|^2 / 2)
                    umma_bf16(dt, umma_desc(smem_u32(sA + TC_RB * (KA - 1) * L::A_ATOM)),
                              umma_desc(bb + (KA - 1) * L::B_ATOM), idesc, 1u);
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
        tc_epilogue<KC, true>(accf, acce, tmem, warp, lane, row0, nq, n, TileMap(tiles, t0, 1, 0), k - 1, self_offset, nullptr, par, qn,
                              best, buf, err);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 9) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem) : "memory");
    }
}

// ---------------------------------------------------------------- float inputs
//
// knn_tcs_kernel: the tensor-core sweep for float inputs.  Both vector sets are
// first centred on the mean of the base (distances do not change) and split into
// bfloat16 pairs c = hi + lo with hi = bf16(c), lo = bf16(c - hi); a dot product
// is then qh.xh + qh.xl + ql.xh in float32 (three tcgen05.mma per K step; the
// dropped ql.xl and the rounding of lo are below 2^-16 |q| |x|).  The ranking of
// this expanded form only selects the KC survivors of a row, which
// knn_final_kernel rescores by direct difference in float32 from the original
// vectors, as for the SIMT sweep.  Rows are zero-padded to dp = 64 ceil(d / 64),
// so K runs in chunks of one 64-wide atom: A (both row blocks, hi and lo) and B
// (hi and lo) stream through a two-stage ring of 96 KB, the accumulators stay in
// TMEM across the chunks of a tile, and the epilogue is tc_epilogue.
constexpr int TCS_STAGES = 2;
struct TcsSmem {
    static constexpr int ATOM = TC_M * 128;  // 128 rows x 64 bfloat16 (TC_N == TC_M)
    static constexpr int STAGE = 6 * ATOM;   // A hi (2 blocks), A lo (2 blocks), B hi, B lo
    static constexpr int BYTES = 1024 + TCS_STAGES * STAGE + 256;
};
static_assert(TC_N == TC_M, "the split kernel's atoms are 128 rows for A and B alike");

template <int KC>
__global__ void __launch_bounds__(TC_THREADS, 1)
    knn_tcs_kernel(const __grid_constant__ CUtensorMap tmAh, const __grid_constant__ CUtensorMap tmAl,
                   const __grid_constant__ CUtensorMap tmBh, const __grid_constant__ CUtensorMap tmBl, int64_t n,
                   int64_t nq, int nk, int G, int64_t self_offset, const float *__restrict__ xh,
                   const float *__restrict__ qn, unsigned long long *__restrict__ best,
                   unsigned long long *__restrict__ buf, int *err)
{
    using L = TcsSmem;
    extern __shared__ unsigned char tc_raw[];
    unsigned char *base = reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(tc_raw) + 1023) & ~uintptr_t(1023));
    uint64_t *bars = reinterpret_cast<uint64_t *>(base + TCS_STAGES * L::STAGE);
    uint64_t *full = bars, *empty = bars + TCS_STAGES, *accf = bars + 2 * TCS_STAGES, *acce = accf + 2;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(acce + 2);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t row0 = (int64_t)(blockIdx.x / G) * TC_ROWS;
    const int64_t tiles = (n + TC_N - 1) / TC_N;
    const int nrb = row0 + TC_M < nq ? TC_RB : 1;  // row blocks holding any query row
    // a self-join starts its sweep at the tile of its own rows and wraps around:
    // where nearby rows sit together, the thresholds fall within the first tiles
    const int64_t t0 = self_offset >= 0 ? ((self_offset + row0) / TC_N) % tiles : 0;
    const TileMap tm(tiles, t0, G, (int)(blockIdx.x % G));
    const int64_t steps = tm.count * nk;
    // this CTA's lists: share g of the row set keeps its own best list and buffers
    best += (int64_t)tm.g * nq * KC;
    buf += (int64_t)tm.g * nq * TC_BUF;

    if (tid == 0) {
        for (int s = 0; s < TCS_STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&accf[b], 1);
            mbar_init(&acce[b], TC_EPI);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 9) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_u32(tmem_slot))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    for (int e = tid; e < TC_ROWS * KC; e += blockDim.x) {
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
            const uint32_t bytes = (uint32_t)((2 * nrb + 2) * L::ATOM);
            int64_t issued = 0;
            for (int64_t step = 0; step < steps; ++step) {
                const int s = (int)(step % TCS_STAGES);
                const int64_t t = step / nk;
                const int kc = (int)(step % nk);
                if (step >= TCS_STAGES &&
                    !mbar_wait(&empty[s], (uint32_t)(((step / TCS_STAGES) & 1) ^ 1), err, 1))
                    break;
                unsigned char *st = base + s * L::STAGE;
                mbar_expect_tx(&full[s], bytes);
                for (int rb = 0; rb < nrb; ++rb) {
                    tma_load_2d(st + rb * L::ATOM, &tmAh, kc * 64, (int)(row0 + rb * TC_M), &full[s]);
                    tma_load_2d(st + (2 + rb) * L::ATOM, &tmAl, kc * 64, (int)(row0 + rb * TC_M), &full[s]);
                }
                tma_load_2d(st + 4 * L::ATOM, &tmBh, kc * 64, (int)(tm.tile(t) * TC_N), &full[s]);
                tma_load_2d(st + 5 * L::ATOM, &tmBl, kc * 64, (int)(tm.tile(t) * TC_N), &full[s]);
                issued = step + 1;
            }
            // our copies in flight complete before the CTA may exit (bounded)
            for (int64_t step = issued > TCS_STAGES ? issued - TCS_STAGES : 0; step < issued; ++step)
                mbar_drain(&full[step % TCS_STAGES], (uint32_t)((step / TCS_STAGES) & 1), err, 6);
        }
    } else if (warp == 9) {
        // ------------------------------------------------ MMA issuer
        if (lane == 0) {
            constexpr uint32_t idesc = umma_idesc(TC_M, TC_N);
            int64_t last = -1;  // the last step whose MMAs were issued (and committed to empty)
            for (int64_t step = 0; step < steps; ++step) {
                const int s = (int)(step % TCS_STAGES);
                const int64_t t = step / nk;
                const int kc = (int)(step % nk), b = (int)(t & 1);
                if (!mbar_wait(&full[s], (uint32_t)((step / TCS_STAGES) & 1), err, 3))
                    break;
                if (kc == 0 && t >= 2 && !mbar_wait(&acce[b], (uint32_t)(((t >> 1) & 1) ^ 1), err, 4))
                    break;
                tc_fence_after();
                const uint32_t st = smem_u32(base + s * L::STAGE);
#pragma unroll
                for (int rb = 0; rb < TC_RB; ++rb) {
                    if (rb >= nrb)
                        break;
                    const uint32_t dt = tmem + (uint32_t)((rb * 2 + b) * TC_N);
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk) {
                        const uint32_t off = (uint32_t)(kk * 32);  // 16 bf16 = 32 bytes inside the atom
                        const uint64_t ah = umma_desc(st + rb * L::ATOM + off);
                        const uint64_t al = umma_desc(st + (2 + rb) * L::ATOM + off);
                        const uint64_t bh = umma_desc(st + 4 * L::ATOM + off);
                        const uint64_t bl = umma_desc(st + 5 * L::ATOM + off);
                        umma_bf16(dt, ah, bh, idesc, (kc > 0 || kk > 0) ? 1u : 0u);
                        umma_bf16(dt, ah, bl, idesc, 1u);
                        umma_bf16(dt, al, bh, idesc, 1u);
                    }
                }
                umma_commit(&empty[s]);
                if (kc == nk - 1)
                    umma_commit(&accf[b]);
                last = step;
            }
            // the MMAs issued so far complete before TMEM is freed (bounded)
            if (last >= 0)
                mbar_drain(&empty[last % TCS_STAGES], (uint32_t)((last / TCS_STAGES) & 1), err, 7);
        }
    } else {
        // ------------------------------------------------ epilogue (warps 0-7)
        tc_epilogue<KC, false>(accf, acce, tmem, warp, lane, row0, nq, n, tm, KC - 1, self_offset, xh, nullptr, qn,
                               best, buf, err);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 9) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem) : "memory");
    }
}

// sums[j] += the base's coordinates j (float64), for the centring mean
__global__ void col_sums_kernel(const float *__restrict__ X, int64_t n, int d, double *__restrict__ sums)
{
    const int64_t per = (n + gridDim.x - 1) / gridDim.x;
    const int64_t r0 = (int64_t)blockIdx.x * per, r1 = r0 + per < n ? r0 + per : n;
    for (int j = threadIdx.x; j < d; j += blockDim.x) {
        double acc = 0.0;
        for (int64_t r = r0; r < r1; ++r)
            acc += (double)X[r * d + j];
        if (r1 > r0)
            atomicAdd(&sums[j], acc);
    }
}

__global__ void mean_kernel(const double *__restrict__ sums, int64_t n, int d, float *__restrict__ mu)
{
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < d; j += gridDim.x * blockDim.x)
        mu[j] = (float)(sums[j] / (double)n);
}

// Row r of M [rows, d] centred on mu, split into bfloat16 hi / lo rows of
// length dp (zeros past d), and its centred squared norm (half of it when
// `half`; +inf for the padded rows rows .. padded_rows of a half-norm array).
__global__ void split_rows_kernel(const float *__restrict__ M, int64_t rows, int d, int dp,
                                  const float *__restrict__ mu, __nv_bfloat16 *__restrict__ hi,
                                  __nv_bfloat16 *__restrict__ lo, float *__restrict__ norm, bool half,
                                  int64_t padded_rows)
{
    const int lane = threadIdx.x & 31;
    for (int64_t r = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; r < padded_rows;
         r += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        if (r >= rows) {
            if (lane == 0)
                norm[r] = INFINITY;
            continue;
        }
        float s = 0.f;
        for (int j = lane; j < dp; j += 32) {
            const float c = j < d ? M[r * d + j] - mu[j] : 0.f;
            const __nv_bfloat16 h = __float2bfloat16_rn(c);
            hi[r * dp + j] = h;
            lo[r * dp + j] = __float2bfloat16_rn(c - __bfloat162float(h));
            s = fmaf(c, c, s);
        }
#pragma unroll
        for (int off = 16; off >= 1; off >>= 1)
            s += __shfl_xor_sync(0xffffffffu, s, off);
        if (lane == 0)
            norm[r] = half ? 0.5f * s : s;
    }
}

// Sets bit 0 of *flag if any value is not an integer in [0, 255] (byte-valued
// descriptors: exact in bfloat16, and at d <= 128 every squared norm, dot product,
// |x|^2 / 2 and distance of the tensor-core path is an exact float32 below 2^23),
// and bit 1 if any value is not an integer at all.
__global__ void value_kind_kernel(const float *__restrict__ x, int64_t count, int *flag)
{
    unsigned bad = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
        const float v = x[i];
        const bool integer = v == rintf(v);
        bad |= (integer && v >= 0.f && v <= 255.f) ? 0u : 1u;
        bad |= integer ? 0u : 2u;
    }
    bad = __reduce_or_sync(0xffffffffu, bad);
    if ((threadIdx.x & 31) == 0 && bad)
        atomicOr(flag, (int)bad);
}

// The byte-valued form's operands: row r of M in bfloat16 in columns [0, d) of a
// row of dpa = d + 64 (an extra K atom), then in columns d, d + 1, d + 2 either
// 1.0 (queries: s == nullptr) or the three pieces of -floor(s_r / 2) (base rows;
// s_r = |x_r|^2, an integer below 2^23): its 8-bit fields times 2^16, 2^8 and 1,
// each exact in bfloat16; zeros elsewhere.  The MMA then accumulates
// q.x - floor(|x|^2 / 2) exactly.
__global__ void aug_rows_kernel(const float *__restrict__ M, int64_t rows, int d, int dpa,
                                const float *__restrict__ s, __nv_bfloat16 *__restrict__ out)
{
    const int lane = threadIdx.x & 31;
    for (int64_t r = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; r < rows;
         r += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        const unsigned h = s ? ((unsigned)s[r]) >> 1 : 0u;
        for (int j = lane; j < dpa; j += 32) {
            float v = 0.f;
            if (j < d)
                v = M[r * d + j];
            else if (j < d + 3) {
                const int p = j - d;
                v = !s ? 1.f : -(float)(p == 0 ? (h >> 16) << 16 : p == 1 ? ((h >> 8) & 255u) << 8 : h & 255u);
            }
            out[r * dpa + j] = __float2bfloat16_rn(v);
        }
    }
}

// Bit i of par = the parity of the integer s_i (0 past n), one word per 32 columns.
__global__ void parity_kernel(const float *__restrict__ s, int64_t n, int64_t words, unsigned *__restrict__ par)
{
    const int lane = threadIdx.x & 31;
    for (int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; w < words;
         w += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        const int64_t i = w * 32 + lane;
        const unsigned bit = i < n ? ((unsigned)s[i] & 1u) : 0u;
        const unsigned b = __ballot_sync(0xffffffffu, bit != 0);
        if (lane == 0)
            par[w] = b;
    }
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

// CTAs sharing one row set in the split sweep: above d = 128 a CTA's A chunks
// (256 rows x dp x 4 bytes) over all resident CTAs would exceed L2, so two CTAs take
// alternate tiles of the same rows (half the A data in flight) and keep a best list
// each, merged by the rescore.
int split_share(int d) { return d > 128 ? 2 : 1; }

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
int launch_tc_kc(const CUtensorMap &ma, const CUtensorMap &mb, int64_t n, int64_t nq, int k, int64_t self_offset,
                 const unsigned *par, const float *qn, unsigned long long *best, unsigned long long *bufp, int *err,
                 cudaStream_t s)
{
    const size_t smem = TcSmem<KA>::BYTES;
    ONNG_CUDA_TRY(cudaFuncSetAttribute(reinterpret_cast<const void *>(knn_tc_kernel<KC, KA>),
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
                  "onng_knn: tensor kernel smem attribute");
    knn_tc_kernel<KC, KA><<<(unsigned)((nq + TC_ROWS - 1) / TC_ROWS), TC_THREADS, smem, s>>>(
        ma, mb, n, nq, k, self_offset, par, qn, best, bufp, err);
    return check_launch("onng_knn: tensor kernel");
}

int launch_tc(const float *X, int64_t n, int d, const float *Q, int64_t nq, int k, int kc, int64_t self_offset,
              int32_t *nbr, float *len, const float *xn, unsigned *par, float *qn, unsigned long long *best,
              unsigned long long *bufp, int *err, __nv_bfloat16 *xb, __nv_bfloat16 *qb, cudaStream_t s)
{
    const int gb = num_sms() * 8;
    const int dpa = d + 64;  // the extra K atom carries -floor(|x|^2 / 2)
    aug_rows_kernel<<<gb, 256, 0, s>>>(X, n, d, dpa, xn, xb);
    aug_rows_kernel<<<gb, 256, 0, s>>>(Q, nq, d, dpa, nullptr, qb);
    parity_kernel<<<gb, 256, 0, s>>>(xn, n, (n + TC_N - 1) / TC_N * (TC_N / 32), par);
    int st = check_launch("onng_knn: bf16 operands");
    if (st)
        return st;
    CUtensorMap ma, mb;
    if ((st = make_map(&ma, qb, nq, dpa, TC_M)) || (st = make_map(&mb, xb, n, dpa, TC_N)))
        return st;
    const int ka = dpa / 64;
    if (kc == 32)
        st = ka == 2 ? launch_tc_kc<32, 2>(ma, mb, n, nq, k, self_offset, par, qn, best, bufp, err, s)
                     : launch_tc_kc<32, 3>(ma, mb, n, nq, k, self_offset, par, qn, best, bufp, err, s);
    else if (kc == 64)
        st = ka == 2 ? launch_tc_kc<64, 2>(ma, mb, n, nq, k, self_offset, par, qn, best, bufp, err, s)
                     : launch_tc_kc<64, 3>(ma, mb, n, nq, k, self_offset, par, qn, best, bufp, err, s);
    else
        st = ka == 2 ? launch_tc_kc<128, 2>(ma, mb, n, nq, k, self_offset, par, qn, best, bufp, err, s)
                     : launch_tc_kc<128, 3>(ma, mb, n, nq, k, self_offset, par, qn, best, bufp, err, s);
    if (st)
        return st;
    int code = 0;
    ONNG_CUDA_TRY(cudaMemcpyAsync(&code, err, sizeof(int), cudaMemcpyDeviceToHost, s), "onng_knn: error flag");
    ONNG_CUDA_TRY(cudaStreamSynchronize(s), "onng_knn: tensor kernel");
    if (code)
        return set_error(ONNG_E_LIMIT, "onng_knn: tensor-core pipeline wait timed out (role %d)", code);
    knn_emit_kernel<<<gb, 256, 0, s>>>(nq, best, kc, k, nbr, len);
    return check_launch("onng_knn: output");
}

template <int KC>
int launch_tcs_kc(const CUtensorMap *m, int64_t n, int64_t nq, int nk, int G, int64_t self_offset, const float *xh,
                  const float *qn, unsigned long long *best, unsigned long long *bufp, int *err, cudaStream_t s)
{
    const size_t smem = TcsSmem::BYTES;
    ONNG_CUDA_TRY(cudaFuncSetAttribute(reinterpret_cast<const void *>(knn_tcs_kernel<KC>),
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
                  "onng_knn: split tensor kernel smem attribute");
    knn_tcs_kernel<KC><<<(unsigned)((nq + TC_ROWS - 1) / TC_ROWS * G), TC_THREADS, smem, s>>>(
        m[0], m[1], m[2], m[3], n, nq, nk, G, self_offset, xh, qn, best, bufp, err);
    return check_launch("onng_knn: split tensor kernel");
}

// Float inputs on the tensor cores: centre, split into bfloat16 hi / lo, sweep
// (knn_tcs_kernel), rescore the survivors from the original vectors.
int launch_tcs(const float *X, int64_t n, int d, const float *Q, int64_t nq, int k, int kc, int64_t self_offset,
               int32_t *nbr, float *len, float *xh, float *qn, unsigned long long *best, unsigned long long *bufp,
               int *err, __nv_bfloat16 *xs, __nv_bfloat16 *qs, double *sums, float *mu, cudaStream_t s)
{
    const int dp = (d + 63) / 64 * 64;
    const int gb = num_sms() * 8;
    __nv_bfloat16 *xhi = xs, *xlo = xs + (size_t)n * dp;
    __nv_bfloat16 *qhi = qs, *qlo = qs + (size_t)nq * dp;
    ONNG_CUDA_TRY(cudaMemsetAsync(sums, 0, sizeof(double) * (size_t)d, s), "onng_knn: clear sums");
    col_sums_kernel<<<(unsigned)std::min<int64_t>(n, 1024), 256, 0, s>>>(X, n, d, sums);
    mean_kernel<<<(d + 255) / 256, 256, 0, s>>>(sums, n, d, mu);
    split_rows_kernel<<<gb, 256, 0, s>>>(X, n, d, dp, mu, xhi, xlo, xh, true, (n + TC_N - 1) / TC_N * TC_N);
    split_rows_kernel<<<gb, 256, 0, s>>>(Q, nq, d, dp, mu, qhi, qlo, qn, false, nq);
    int st = check_launch("onng_knn: split copies");
    if (st)
        return st;
    CUtensorMap m[4];
    if ((st = make_map(&m[0], qhi, nq, dp, TC_M)) || (st = make_map(&m[1], qlo, nq, dp, TC_M)) ||
        (st = make_map(&m[2], xhi, n, dp, TC_N)) || (st = make_map(&m[3], xlo, n, dp, TC_N)))
        return st;
    const int nk = dp / 64;
    const int G = split_share(d);
    st = kc == 32 ? launch_tcs_kc<32>(m, n, nq, nk, G, self_offset, xh, qn, best, bufp, err, s)
         : kc == 64 ? launch_tcs_kc<64>(m, n, nq, nk, G, self_offset, xh, qn, best, bufp, err, s)
                    : launch_tcs_kc<128>(m, n, nq, nk, G, self_offset, xh, qn, best, bufp, err, s);
    if (st)
        return st;
    int code = 0;
    ONNG_CUDA_TRY(cudaMemcpyAsync(&code, err, sizeof(int), cudaMemcpyDeviceToHost, s), "onng_knn: error flag");
    ONNG_CUDA_TRY(cudaStreamSynchronize(s), "onng_knn: split tensor kernel");
    if (code)
        return set_error(ONNG_E_LIMIT, "onng_knn: tensor-core pipeline wait timed out (role %d)", code);
    const unsigned grid = (unsigned)((nq * 32 + 255) / 256);
    const int64_t ls = nq * kc;  // the G lists of a row
    if (G == 1) {
        if (kc == 32)
            knn_final_kernel<32><<<grid, 256, 0, s>>>(X, d, Q, nq, best, k, nbr, len);
        else if (kc == 64)
            knn_final_kernel<64><<<grid, 256, 0, s>>>(X, d, Q, nq, best, k, nbr, len);
        else
            knn_final_kernel<128><<<grid, 256, 0, s>>>(X, d, Q, nq, best, k, nbr, len);
    } else {
        if (kc == 32)
            knn_final_kernel<32, 2><<<grid, 256, 0, s>>>(X, d, Q, nq, best, k, nbr, len, ls);
        else if (kc == 64)
            knn_final_kernel<64, 2><<<grid, 256, 0, s>>>(X, d, Q, nq, best, k, nbr, len, ls);
        else
            knn_final_kernel<128, 2><<<grid, 256, 0, s>>>(X, d, Q, nq, best, k, nbr, len, ls);
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
    c.take<unsigned long long>((size_t)std::max<int64_t>(nq, 1) * (kc ? kc : 32) * split_share(d));
    c.take<unsigned long long>((size_t)std::max<int64_t>(nq, 1) * std::max(BUF, TC_BUF) * split_share(d));
    c.take<int>(64);
    // bfloat16 copies: hi and lo rows of dp = 64 ceil(d / 64) (the byte path's rows of d + 64 fit)
    const size_t dp = (size_t)(std::max(d, 1) + 63) / 64 * 64;
    c.take<__nv_bfloat16>((size_t)std::max<int64_t>(n, 1) * dp * 2);
    c.take<__nv_bfloat16>((size_t)std::max<int64_t>(nq, 1) * dp * 2);
    c.take<float>((size_t)(std::max<int64_t>(n, 1) + TC_N - 1) / TC_N * TC_N);
    c.take<double>((size_t)std::max(d, 1));
    c.take<float>((size_t)std::max(d, 1));
    c.take<unsigned>((size_t)(std::max<int64_t>(n, 1) + TC_N - 1) / TC_N * (TC_N / 32));
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
    unsigned long long *best = c.take<unsigned long long>((size_t)nq * kc * split_share(d));
    unsigned long long *bufp = c.take<unsigned long long>((size_t)nq * std::max(BUF, TC_BUF) * split_share(d));
    int *flags = c.take<int>(64);
    const size_t dp = (size_t)(d + 63) / 64 * 64;
    __nv_bfloat16 *xb = c.take<__nv_bfloat16>((size_t)std::max<int64_t>(n, 1) * dp * 2);
    __nv_bfloat16 *qb = c.take<__nv_bfloat16>((size_t)nq * dp * 2);
    float *xh = c.take<float>((size_t)(std::max<int64_t>(n, 1) + TC_N - 1) / TC_N * TC_N);
    double *sums = c.take<double>((size_t)d);
    float *mu = c.take<float>((size_t)d);
    unsigned *par = c.take<unsigned>((size_t)(std::max<int64_t>(n, 1) + TC_N - 1) / TC_N * (TC_N / 32));
    cudaStream_t s = to_cuda(stream);
    if (n > 0)
        norms_kernel<<<(unsigned)((n * 32 + 255) / 256), 256, 0, s>>>(X, n, d, xn);
    norms_kernel<<<(unsigned)((nq * 32 + 255) / 256), 256, 0, s>>>(Q, nq, d, qn);
    int st = check_launch("onng_knn: norms");
    if (st)
        return st;
    // tensor-core paths (at least one full tile of base rows and one row block of
    // queries, k + 16 <= 128): byte-valued inputs at d = 64 / 128 exactly; other
    // non-integer inputs at d >= 32 by the split bfloat16 form.  Integer-valued
    // inputs otherwise take the SIMT sweep, which ranks them exactly.
    if (n >= TC_N && nq >= TC_M && kc <= 128 && n <= INT32_MAX - TC_N) {
        ONNG_CUDA_TRY(cudaMemsetAsync(flags, 0, 64 * sizeof(int), s), "onng_knn: clear flags");
        const int gb = num_sms() * 8;
        value_kind_kernel<<<gb, 256, 0, s>>>(X, n * d, flags);
        value_kind_kernel<<<gb, 256, 0, s>>>(Q, nq * d, flags);
        int kind = 3;
        ONNG_CUDA_TRY(cudaMemcpyAsync(&kind, flags, sizeof(int), cudaMemcpyDeviceToHost, s), "onng_knn: flag");
        ONNG_CUDA_TRY(cudaStreamSynchronize(s), "onng_knn: value check");
        if (!(kind & 1) && (d == 64 || d == 128))
            return launch_tc(X, n, d, Q, nq, k, kc, self_offset, nbr, len, xn, par, qn, best, bufp, flags + 1, xb,
                             qb, s);
        if ((kind & 2) && d >= 32)
            return launch_tcs(X, n, d, Q, nq, k, kc, self_offset, nbr, len, xh, qn, best, bufp, flags + 1, xb, qb,
                              sums, mu, s);
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
