// KnnSearch (Algorithm 1) on the GPU: one warp per query.  Device code of the
// search kernels; search_inst.cu instantiates it once per (vector type, chunks
// per lane) so the instantiations compile in parallel, and search.cu holds the
// host entry points.
//
// Per warp:
//   - the visited set C, in shared memory, as buckets of 8 ids with two bucket
//     choices per id (the paper's Set/IsSet table, Sec. 2.5, chains collisions
//     off one inline id; here a batch of 32 ids reads both buckets of each id and
//     claims free slots in lane order, with no probe loop).  An id that finds
//     both of its buckets full moves the query to a per-warp bitmap over all n
//     ids in global memory (one atomicOr per new id); the ids set there are
//     logged and cleared when the query ends.
//   - the candidate set S in three levels of (distance, id) keys: a sorted head
//     of up to 32 keys in registers (one per lane: the pop is a shift, an
//     insertion a ballot plus a shift), an unsorted overflow in shared memory
//     whose keys are all >= every head key, and a per-warp spill pool in global
//     memory whose keys are all >= tau > every key above it.  So the head's
//     first key is the minimum of S; a level refills the one above only when
//     that one runs empty.  An entry beyond r(1+eps) can never be expanded (r
//     only shrinks, and popping it ends the search), so such entries are
//     dropped whenever a level is rebuilt.  S stays exact.
//   - the result set R, in registers, as a sorted list of at most k keys.
// The up-to-e_s neighbours of the expanded node are tested and the new ones'
// vectors gathered together (their ids go to shared gather slots in lane order;
// coalesced 16-byte loads, several vectors in flight per lane, one transposed
// butterfly reduction for all of them).  R then takes the k
// best of R and the batch, and S takes the batch members within the new
// r(1+eps).  Applying a batch at once yields the same R, the same r after the
// batch and, since S only loses entries that can never be expanded, the same
// expansion order as the one-at-a-time loop of Algorithm 1.
//
// The node expanded next is known as soon as the batch's distances are: it is
// the nearer of S's head and the batch's nearest member if that one will be
// pushed (its distance is within the bound before the batch).  Its adjacency
// row is loaded right then, so the load overlaps the R and S updates, and once
// the row is in, its neighbours' vectors are prefetched into L2.
//
// Adjacency is read from the CSR lists, or from an optional padded table
// adj [n, width] (-1 padded) that holds each node's first `width` entries, which
// saves the row-pointer indirection per expansion.
//
// Distances are squared float32 sums of (q - x)^2; the bound r^2 (1 + eps)^2 is
// formed in double whenever r changes and kept rounded down to float32, which
// for a float32 d^2 decides d^2 <= r^2 (1 + eps)^2 exactly as the double
// comparison does.  For integer-valued inputs with squared distances below 2^24
// every decision then equals the float64 algorithm's.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <type_traits>

#include "common.cuh"
#include "warp_sort.cuh"

// Visited set in shared memory: 1 = buckets of 8 ids with two choices per id,
// 0 = one open-addressing table with linear probing.
#ifndef ONNG_SEARCH_VISIT
#define ONNG_SEARCH_VISIT 1
#endif
// 1: once the adjacency row of the node expanded next has arrived, ask L2 for
// its neighbours' vectors (the next round's gathers then start from L2).
#ifndef ONNG_SEARCH_PREFETCH
#define ONNG_SEARCH_PREFETCH 1
#endif
// Gather slots of a batch: 1 = the new ids go through shared memory in lane
// order; 0 = each slot finds its lane by a find-first-set on the mask.
#ifndef ONNG_SEARCH_COMPACT
#define ONNG_SEARCH_COMPACT 1
#endif
#ifndef ONNG_SEARCH_MAXV
#define ONNG_SEARCH_MAXV 8  // kernels are built for d <= 128 * ONNG_SEARCH_MAXV (1, 2, 4 or 8)
#endif
// Per vector type, for d <= 256 and k <= 32: visited-table slots per warp (a
// multiple of 8), shared-memory overflow keys per warp (a power of two >= 64),
// the most vectors gathered per round (a power of two) and the resident CTAs per
// SM the registers are sized for.  The search is latency-bound, so resident
// warps set its speed: float32 vectors (512 B at d = 128) want 16 gathers in
// flight per lane and run 5 CTAs (20 warps) per SM; bfloat16 vectors are half
// the size and run 8 gathers per round at 6 CTAs per SM.
#ifndef ONNG_SEARCH_F32_HV
#define ONNG_SEARCH_F32_HV 2048
#endif
#ifndef ONNG_SEARCH_F32_OVF
#define ONNG_SEARCH_F32_OVF 128
#endif
#ifndef ONNG_SEARCH_F32_GMAX
#define ONNG_SEARCH_F32_GMAX 16
#endif
#ifndef ONNG_SEARCH_F32_MINB
#define ONNG_SEARCH_F32_MINB 5
#endif
#ifndef ONNG_SEARCH_BF16_HV
#define ONNG_SEARCH_BF16_HV 2048
#endif
#ifndef ONNG_SEARCH_BF16_OVF
#define ONNG_SEARCH_BF16_OVF 128
#endif
#ifndef ONNG_SEARCH_BF16_GMAX
#define ONNG_SEARCH_BF16_GMAX 8
#endif
#ifndef ONNG_SEARCH_BF16_MINB
#define ONNG_SEARCH_BF16_MINB 6
#endif
#ifndef ONNG_SEARCH_FP8_HV
#define ONNG_SEARCH_FP8_HV 2048
#endif
#ifndef ONNG_SEARCH_FP8_OVF
#define ONNG_SEARCH_FP8_OVF 128
#endif
#ifndef ONNG_SEARCH_FP8_GMAX
#define ONNG_SEARCH_FP8_GMAX 8
#endif
#ifndef ONNG_SEARCH_FP8_MINB
#define ONNG_SEARCH_FP8_MINB 6
#endif

namespace onng {
namespace sk {

typedef unsigned long long u64;

constexpr unsigned FULL = 0xffffffffu;
constexpr int kWarpsPerCta = 4;
constexpr int kMaxK = 128;
constexpr int kMaxSeed = 64;
template <class T> struct Tune {
    static constexpr int hv = ONNG_SEARCH_F32_HV, ovf = ONNG_SEARCH_F32_OVF, gmax = ONNG_SEARCH_F32_GMAX,
                         minb = ONNG_SEARCH_F32_MINB;
};
template <> struct Tune<__nv_bfloat16> {
    static constexpr int hv = ONNG_SEARCH_BF16_HV, ovf = ONNG_SEARCH_BF16_OVF, gmax = ONNG_SEARCH_BF16_GMAX,
                         minb = ONNG_SEARCH_BF16_MINB;
};
template <> struct Tune<__nv_fp8_e4m3> {
    static constexpr int hv = ONNG_SEARCH_FP8_HV, ovf = ONNG_SEARCH_FP8_OVF, gmax = ONNG_SEARCH_FP8_GMAX,
                         minb = ONNG_SEARCH_FP8_MINB;
};
constexpr int kVisitLog = 16384;     // ids logged per warp for clearing its bitmap
constexpr int kGlobalPool = 16384;   // default per-warp candidate spill pool entries
constexpr u64 kMaxKey = ~0ull;
constexpr int kFeat = 16;

struct SearchArgs {
    const int64_t *row_ptr;
    const int32_t *col;
    const int32_t *adj;
    int adj_w;
    const float *X;
    const uint16_t *Xb;
    const uint8_t *X8;     // e4m3 codes, dequantised as scale8[j] * e4m3
    const float *scale8;
    int64_t n;
    int d;
    const float *Q;
    int64_t nq;
    int k;      // results kept by the search (k_rerank for bf16)
    int k_out;  // results written
    int e_s;
    float eps;
    const float *eps_q;
    const int32_t *es_q;
    const int32_t *seeds;
    int n_seed;
    int max_exp;
    int32_t *out_ids;  // may be NULL (probe only)
    float *out_dist;
    int32_t *stats;
    float *feat;       // [nq, kFeat] probe features, or NULL
    float target;      // feature 0 (the recall the prediction is for)
    int *counter;
    unsigned *gbits;  // [slots, bits_words]: visited bitmap past the shared table
    int64_t bits_words;
    int *glog;        // [slots, kVisitLog]: ids set in the bitmap
    u64 *gpool;       // [slots, gpool_cap]
    int gpool_cap;    // spill pool entries per warp
};

template <int HV, int OVF> struct WarpSmem {
    int vis[HV];
    u64 ovf[OVF];
    int slot[32];  // ids of a batch's new nodes in lane order (gather slots)
#ifdef ONNG_CHECK
    unsigned canary[4];  // between this warp's arrays and the next warp's
#endif
};

#ifdef ONNG_CHECK
constexpr unsigned kCanary = 0x0C4A7A10u;
#endif

__host__ __device__ constexpr int log2i(int v) { return v <= 1 ? 0 : 1 + log2i(v >> 1); }

__device__ __forceinline__ unsigned lanemask_lt(int lane) { return (1u << lane) - 1u; }

__device__ __forceinline__ unsigned hash_id(int id) { return static_cast<unsigned>(id) * 0x9E3779B1u; }
__device__ __forceinline__ unsigned hash2_id(int id) { return (static_cast<unsigned>(id) ^ 0x5BD1E995u) * 0x7FEB352Du; }

__device__ __forceinline__ float key_d2(u64 k) { return __uint_as_float((unsigned)(k >> 32)); }
__device__ __forceinline__ int key_id(u64 k) { return (int)(unsigned)(k & 0xFFFFFFFFull); }

__device__ __forceinline__ u64 warp_min_u64(u64 v)
{
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) {
        u64 o = __shfl_xor_sync(FULL, v, off);
        v = o < v ? o : v;
    }
    return v;
}

// Ascending list of 32*N keys striped over the warp: element e sits in v[e / 32]
// of lane e % 32.  Empty slots hold kMaxKey.
template <int N> struct RegList {
    u64 v[N];

    __device__ void clear()
    {
#pragma unroll
        for (int i = 0; i < N; ++i)
            v[i] = kMaxKey;
    }
    // number of elements smaller than key
    __device__ int rank(u64 key) const
    {
        int r = 0;
#pragma unroll
        for (int i = 0; i < N; ++i)
            r += __popc(__ballot_sync(FULL, v[i] < key));
        return r;
    }
    // element e (uniform e < 32*N), broadcast to all lanes
    __device__ u64 get(int e) const
    {
        u64 x = kMaxKey;
#pragma unroll
        for (int i = 0; i < N; ++i)
            if (i == (e >> 5))
                x = v[i];
        return __shfl_sync(FULL, x, e & 31);
    }
    // inserts key at position pos (uniform); elements at positions >= limit are emptied
    __device__ void insert_at(int pos, u64 key, int lane, int limit)
    {
        u64 carry = kMaxKey;  // old element i*32 - 1
#pragma unroll
        for (int i = 0; i < N; ++i) {
            const u64 up = __shfl_up_sync(FULL, v[i], 1);
            const u64 last = __shfl_sync(FULL, v[i], 31);
            const u64 before = lane == 0 ? carry : up;
            const int e = i * 32 + lane;
            u64 nv = e < pos ? v[i] : (e == pos ? key : before);
            v[i] = e < limit ? nv : kMaxKey;
            carry = last;
        }
    }
    // removes element 0
    __device__ void pop_front(int lane)
    {
#pragma unroll
        for (int i = 0; i < N; ++i) {
            const u64 down = __shfl_down_sync(FULL, v[i], 1);
            const u64 next0 = (i + 1 < N) ? __shfl_sync(FULL, v[i + 1], 0) : kMaxKey;
            v[i] = lane == 31 ? next0 : down;
        }
    }
    // empties every element at position >= m
    __device__ void truncate(int m, int lane)
    {
#pragma unroll
        for (int i = 0; i < N; ++i)
            if (i * 32 + lane >= m)
                v[i] = kMaxKey;
    }
};

// Loads 4 consecutive coordinates of a stored vector as float4.
template <class T> struct Loader;
template <> struct Loader<float> {
    static __device__ __forceinline__ float4 load(const void *base, int64_t id, int d, int c)
    {
        const float4 *p = reinterpret_cast<const float4 *>(static_cast<const float *>(base) + id * d) + c;
        return __ldg(p);
    }
};
template <> struct Loader<__nv_bfloat16> {
    static __device__ __forceinline__ float4 load(const void *base, int64_t id, int d, int c)
    {
        const uint2 *p = reinterpret_cast<const uint2 *>(static_cast<const uint16_t *>(base) + id * d) + c;
        uint2 u = __ldg(p);
        float4 f;
        f.x = __uint_as_float(u.x << 16);
        f.y = __uint_as_float(u.x & 0xFFFF0000u);
        f.z = __uint_as_float(u.y << 16);
        f.w = __uint_as_float(u.y & 0xFFFF0000u);
        return f;
    }
};
// e4m3 codes, 4 per 32-bit load; the per-dimension scale is applied by the caller
template <> struct Loader<__nv_fp8_e4m3> {
    static __device__ __forceinline__ float4 load(const void *base, int64_t id, int d, int c)
    {
        const unsigned *p = reinterpret_cast<const unsigned *>(static_cast<const uint8_t *>(base) + id * d) + c;
        const unsigned u = __ldg(p);
        const __half2 lo(__nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(u & 0xFFFFu), __NV_E4M3));
        const __half2 hi(__nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(u >> 16), __NV_E4M3));
        const float2 a = __half22float2(lo), b = __half22float2(hi);
        return make_float4(a.x, a.y, b.x, b.y);
    }
};

__device__ __forceinline__ float sqdiff4(float4 a, float4 b, float acc)
{
    float t = a.x - b.x;
    acc = fmaf(t, t, acc);
    t = a.y - b.y;
    acc = fmaf(t, t, acc);
    t = a.z - b.z;
    acc = fmaf(t, t, acc);
    t = a.w - b.w;
    return fmaf(t, t, acc);
}

// Sums v[g] over the warp for G values at once (G a power of two <= 16): each
// butterfly stage halves the values a lane holds by swapping halves with its
// partner, then plain butterflies finish.  Afterwards every lane holds the full
// sum of one value index: value g sits in the lanes whose bits 4 .. 5 - log2 G
// spell g, lane g << (5 - log2 G) among them.
template <int G, int OFF> __device__ __forceinline__ void tr_stage(float (&v)[G], int lane, int held)
{
    const int half = held >> 1;
    const bool hi = lane & OFF;
#pragma unroll
    for (int i = 0; i < G / 2; ++i) {
        if (i < half) {
            float send = hi ? v[i] : v[i + half];
            float keep = hi ? v[i + half] : v[i];
            v[i] = keep + __shfl_xor_sync(FULL, send, OFF);
        }
    }
}

template <int G> __device__ __forceinline__ float transpose_reduce(float (&v)[G], int lane)
{
    static_assert(G == 1 || G == 2 || G == 4 || G == 8 || G == 16, "G");
    constexpr int m = log2i(G);
    if constexpr (m >= 1)
        tr_stage<G, 16>(v, lane, G);
    if constexpr (m >= 2)
        tr_stage<G, 8>(v, lane, G >> 1);
    if constexpr (m >= 3)
        tr_stage<G, 4>(v, lane, G >> 2);
    if constexpr (m >= 4)
        tr_stage<G, 2>(v, lane, G >> 3);
    float s = v[0];
#pragma unroll
    for (int off = 16 >> m; off >= 1; off >>= 1)
        s += __shfl_xor_sync(FULL, s, off);
    return s;
}

template <int V, class T, int HV, int KR> struct Warp {
    // vectors per gather round: 16 loads in flight per lane at d <= 128
    static constexpr int G0 = V >= 8 ? 2 : V >= 4 ? 4 : V >= 2 ? 8 : 16;
    static constexpr int G = G0 < Tune<T>::gmax ? G0 : Tune<T>::gmax;
    static constexpr int kOvf = Tune<T>::ovf;  // shared-memory overflow keys
    static_assert(kOvf >= 64 && (kOvf & (kOvf - 1)) == 0, "the overflow holds a power of two >= 64 keys");
    static_assert(HV % 8 == 0, "the visited table holds whole buckets of 8 ids");
    WarpSmem<HV, kOvf> &sm;
    const SearchArgs &a;
    const void *xs;  // vectors the search reads (float32 or bfloat16)
    int lane;
    unsigned *gbits;
    int *glog;
    u64 *gpool;
    float4 qv[V];
    float4 sv[V];  // e4m3 form: the per-dimension scales of this lane's coordinates
    RegList<1> head;  // the nearest candidates, sorted
    RegList<KR> res;
    // per-query state, uniform across the warp
    int nh, no, ng, cnt, ndc, nexp, nvis, nlog, kk, nscan, es;
    int pf_node, pf_id;  // adjacency row already loaded for the next expansion
    unsigned flags;
#ifdef ONNG_CHECK
    int64_t nnz_chk;  // row_ptr[n]: every row must lie inside col
#endif
    bool spill, rset, stop, padded, capped;
    int seed_cnt, rins;  // probe features: seeds evaluated, result insertions
    float seed_sum;
    u64 seed1, seed2;
    float r2;
    u64 tau;  // every key in the global pool is >= tau (kMaxKey when it is empty)
    double f2, bound2;
    // bound2 rounded down to float32: for a float32 d^2, d^2 <= bound2 exactly when
    // d^2 <= bnd (bound2 lies in [bnd, next float above bnd), so no float lies
    // strictly between), which keeps the double comparison's decisions in float32
    float bnd;

    __device__ Warp(WarpSmem<HV, kOvf> &s, const SearchArgs &args, const void *x, int ln, unsigned *gb, int *gl, u64 *gp)
        : sm(s), a(args), xs(x), lane(ln), gbits(gb), glog(gl), gpool(gp)
    {
    }

    __device__ bool in_bound(u64 key) const { return key_d2(key) <= bnd; }

    // ---------------------------------------------------------------- visited set

    // Test-and-set of one id by the calling lane; true if newly visited.
    __device__ bool visit(int id)
    {
        static_assert(ONNG_SEARCH_VISIT == 1 || (HV & (HV - 1)) == 0, "the probing table holds a power of two");
        unsigned h = hash_id(id) >> (32 - log2i(HV));
        for (int t = 0; t < HV; ++t) {
            int v = sm.vis[h];
            if (v == id)
                return false;
            if (v == -1) {
                if (spill)
                    break;
                int old = atomicCAS(&sm.vis[h], -1, id);
                if (old == -1)
                    return true;
                if (old == id)
                    return false;
            }
            h = (h + 1) & (HV - 1);
        }
        const unsigned bit = 1u << (id & 31);
        return (atomicOr(&gbits[id >> 5], bit) & bit) == 0;
    }

    // Past half load of the shared table, new ids go to the bitmap.
    __device__ void begin_batch()
    {
        if (!spill && nvis >= HV / 2 - 32)
            spill = true;
    }

    // Appends the ids of the lanes with `set` (bits this warp set) to the bitmap's log.
    __device__ void log_bits(bool set, int id)
    {
        const unsigned m = __ballot_sync(FULL, set);
        if (set) {
            const int pos = nlog + __popc(m & lanemask_lt(lane));
            if (pos < kVisitLog)
                glog[pos] = id;
        }
        nlog += __popc(m);
    }

    // Test-and-set of a batch (one id per lane, -1 = none) in the bucketed table:
    // HV / 8 buckets of 8 ids, filled in slot order, two bucket choices per id.
    // Every lane first looks its id up in both buckets; new ids then take free
    // slots of their first bucket (lanes aiming at one bucket in lane order),
    // the rest of their second; an id that finds both full goes to the bitmap,
    // and so does every later new id of the query.  True if newly visited.
    __device__ bool visit_batch(int id)
    {
        constexpr unsigned NB = HV / 8;
        // an id held by several lanes (repeated seeds) counts once, at its lowest lane
        if (__match_any_sync(FULL, id) & lanemask_lt(lane))
            id = -1;
        const bool has = id >= 0;
        const unsigned b1 = has ? __umulhi(hash_id(id), NB) : 0u;
        const unsigned b2 = has ? __umulhi(hash2_id(id), NB) : 0u;
        const int4 *bk = reinterpret_cast<const int4 *>(sm.vis);
        const int4 p0 = bk[2 * b1], p1 = bk[2 * b1 + 1], q0 = bk[2 * b2], q1 = bk[2 * b2 + 1];
        const bool found = has && (p0.x == id || p0.y == id || p0.z == id || p0.w == id || p1.x == id ||
                                   p1.y == id || p1.z == id || p1.w == id || q0.x == id || q0.y == id ||
                                   q0.z == id || q0.w == id || q1.x == id || q1.y == id || q1.z == id || q1.w == id);
        const bool want = has && !found;
        if (spill) {
            const unsigned bit = 1u << (id & 31);
            const bool isnew = want && (atomicOr(&gbits[id >> 5], bit) & bit) == 0;
            log_bits(isnew, id);
            return isnew;
        }
        const unsigned wm = __ballot_sync(FULL, want);
        if (!wm)
            return false;
        const int used1 = (p0.x != -1) + (p0.y != -1) + (p0.z != -1) + (p0.w != -1) + (p1.x != -1) +
                          (p1.y != -1) + (p1.z != -1) + (p1.w != -1);
        const unsigned g1 = __match_any_sync(FULL, want ? b1 : 0xFFFFFFFFu);
        const int r1 = __popc(g1 & wm & lanemask_lt(lane));
        const bool ok1 = want && used1 + r1 < 8;
        if (ok1)
            sm.vis[b1 * 8 + used1 + r1] = id;
        __syncwarp();
        const bool want2 = want && !ok1;
        const unsigned wm2 = __ballot_sync(FULL, want2);
        if (wm2) {
            const int4 s0 = bk[2 * b2], s1 = bk[2 * b2 + 1];  // after the first-choice stores
            const int used2 = (s0.x != -1) + (s0.y != -1) + (s0.z != -1) + (s0.w != -1) + (s1.x != -1) +
                              (s1.y != -1) + (s1.z != -1) + (s1.w != -1);
            const unsigned g2 = __match_any_sync(FULL, want2 ? b2 : 0xFFFFFFFFu);
            const int r2 = __popc(g2 & wm2 & lanemask_lt(lane));
            const bool ok2 = want2 && used2 + r2 < 8;
            if (ok2)
                sm.vis[b2 * 8 + used2 + r2] = id;
            __syncwarp();
            const bool want3 = want2 && !ok2;
            if (__ballot_sync(FULL, want3)) {
                // both buckets full: this id and every later new one go to the bitmap
                spill = true;
                if (want3)
                    atomicOr(&gbits[id >> 5], 1u << (id & 31));
                log_bits(want3, id);
            }
        }
        return want;
    }

    // Leaves the bitmap all zero for the next query: clears the logged words,
    // or the whole bitmap if the log overflowed.
    __device__ void clear_bits()
    {
        if (!spill)
            return;
        if (nlog <= kVisitLog) {
            for (int i = lane; i < nlog; i += 32)
                gbits[glog[i] >> 5] = 0u;
        } else {
            for (int64_t i = lane; i < a.bits_words; i += 32)
                gbits[i] = 0u;
        }
        __syncwarp();
    }

    // ---------------------------------------------------------------- distances

    // Squared distances of the ids held by the lanes in `mask`; returns this lane's.
    // The ids go to shared slots in lane order; gather round b takes slots
    // b .. b + G - 1, every slot loads (empty slots read row 0 and are masked),
    // so all loads of a round issue back to back.
    template <class L> __device__ float distances(const void *base, int id, unsigned mask)
    {
        const int chunks = a.d >> 2;
        const int m = __popc(mask);
        const bool mine_in = (mask >> lane) & 1u;
        const int rank = __popc(mask & lanemask_lt(lane));
#if ONNG_SEARCH_COMPACT
        if (mine_in)
            sm.slot[rank] = id;
        __syncwarp();
#endif
        float mine = 0.0f;
        for (int b0 = 0; b0 < m; b0 += G) {
            int gid[G];
#if ONNG_SEARCH_COMPACT
#pragma unroll
            for (int g = 0; g < G; ++g) {
                const int sid = b0 + g < m ? sm.slot[b0 + g] : 0;
                gid[g] = sid < 0 ? 0 : sid;
            }
#else
            {
                unsigned rest = mask;  // lanes of slots b0 .. : drop the first b0 set bits
                for (int t = 0; t < b0; ++t)
                    rest &= rest - 1;
#pragma unroll
                for (int g = 0; g < G; ++g) {
                    const int src = rest ? __ffs(rest) - 1 : 0;
                    rest &= rest - 1;
                    const int sid = __shfl_sync(FULL, id, src);
                    gid[g] = (b0 + g < m && sid >= 0) ? sid : 0;
                }
            }
#endif
            float4 xv[G][V];
#pragma unroll
            for (int g = 0; g < G; ++g)
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    const int c = lane + 32 * v;
                    xv[g][v] = L::load(base, gid[g], a.d, c < chunks ? c : 0);
                    if constexpr (std::is_same<L, Loader<__nv_fp8_e4m3>>::value) {
                        // dequantise with a rounded product (never fused into the difference)
                        xv[g][v] = make_float4(__fmul_rn(sv[v].x, xv[g][v].x), __fmul_rn(sv[v].y, xv[g][v].y),
                                               __fmul_rn(sv[v].z, xv[g][v].z), __fmul_rn(sv[v].w, xv[g][v].w));
                    }
                }
            float acc[G];
#pragma unroll
            for (int g = 0; g < G; ++g) {
                acc[g] = 0.0f;
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    int c = lane + 32 * v;
                    if (b0 + g < m && c < chunks)
                        acc[g] = sqdiff4(qv[v], xv[g][v], acc[g]);
                }
            }
            const float red = transpose_reduce<G>(acc, lane);
            // value g of the round sits in lane g << (5 - log2 G)
            const int r = rank - b0;
            const float s = __shfl_sync(FULL, red, (r & (G - 1)) << (5 - log2i(G)));
            if (mine_in && r >= 0 && r < G)
                mine = s;
        }
        __syncwarp();
        return mine;
    }

    // ---------------------------------------------------------------- result list

    // Inserts key into R; false if R keeps its k entries (key would be evicted).
    __device__ bool r_insert(u64 key)
    {
        const int pos = res.rank(key);
        if (pos >= kk)
            return false;
        res.insert_at(pos, key, lane, kk);
        cnt = min(cnt + 1, kk);
        return true;
    }

    // Bounds-checked builds (-DONNG_CHECK): an id read from the graph outside
    // [-1, n) becomes -1 (no access) and flags the query ONNG_FLAG_CHECK.  Called
    // by the whole warp.  Other builds trust the graph.
    __device__ __forceinline__ int graph_id(int id)
    {
#ifdef ONNG_CHECK
        const bool bad = id < -1 || id >= a.n;
        if (__any_sync(FULL, bad))
            flags |= ONNG_FLAG_CHECK;
        return bad ? -1 : id;
#else
        return id;
#endif
    }

    __device__ void update_bound()
    {
        bound2 = (rset && !isinf(f2)) ? (double)r2 * f2 : INFINITY;
        bnd = __double2float_rd(bound2);
    }

    // ---------------------------------------------------------------- candidate pool

    // Appends the keys of the lanes with `put` to the global pool.
    __device__ void gpool_append(bool put, u64 key)
    {
        unsigned m = __ballot_sync(FULL, put);
        if (!m)
            return;
        if (put) {
            int dst = ng + __popc(m & lanemask_lt(lane));
            if (dst < a.gpool_cap)
                gpool[dst] = key;
        }
        if (ng + __popc(m) > a.gpool_cap)
            flags |= ONNG_FLAG_S_OVERFLOW;
        ng = min(ng + __popc(m), a.gpool_cap);
    }

    // Makes room for `need` (<= 32) more keys in the overflow: drops its
    // out-of-bound keys; if they still do not fit, sorts it and moves the
    // farther half to the global pool (so at most kOvf / 2 keys remain).
    __device__ void make_room(int need)
    {
        int w = 0;
        for (int base = 0; base < no; base += 32) {
            const int e = base + lane;
            const u64 kv = e < no ? sm.ovf[e] : kMaxKey;
            const bool keep = e < no && in_bound(kv);
            const unsigned km = __ballot_sync(FULL, keep);
            __syncwarp();
            if (keep)
                sm.ovf[w + __popc(km & lanemask_lt(lane))] = kv;
            w += __popc(km);
            __syncwarp();
        }
        no = w;
        if (no + need <= kOvf)
            return;
        // no > kOvf - need >= kOvf / 2, so the element at kOvf / 2 is a real key
        constexpr int N = kOvf / 32;
        u64 v[N];
#pragma unroll
        for (int i = 0; i < N; ++i)
            v[i] = i * 32 + lane < no ? sm.ovf[i * 32 + lane] : kMaxKey;
        warp_bitonic_sort<N>(v, lane);
        __syncwarp();
#pragma unroll
        for (int i = 0; i < N / 2; ++i)
            sm.ovf[i * 32 + lane] = v[i];
        const u64 first_moved = __shfl_sync(FULL, v[N / 2], 0);
#pragma unroll
        for (int i = N / 2; i < N; ++i)
            gpool_append(v[i] != kMaxKey, v[i]);
        __syncwarp();
        tau = first_moved;
        no = kOvf / 2;
    }

    __device__ void ovf_append(u64 key)
    {
        if (no == kOvf)
            make_room(1);
        if (key >= tau) {
            gpool_append(lane == 0, key);
            return;
        }
        if (lane == 0)
            sm.ovf[no] = key;
        ++no;
        __syncwarp();
    }

    // Refills the empty overflow with the 64 nearest in-bound global keys.
    __device__ void refill_ovf()
    {
        u64 v[8];  // v[0..1]: best 64 so far; v[2..5]: next 128 global keys
#pragma unroll
        for (int i = 0; i < 8; ++i)
            v[i] = kMaxKey;
        u64 worst = kMaxKey;  // the 64th best so far: a chunk with nothing below it changes nothing
        for (int base = 0; base < ng; base += 128) {
#pragma unroll
            for (int i = 2; i < 6; ++i) {
                int e = base + (i - 2) * 32 + lane;
                u64 kv = e < ng ? gpool[e] : kMaxKey;
                v[i] = (kv < worst && in_bound(kv)) ? kv : kMaxKey;
            }
            if (!__any_sync(FULL, v[2] != kMaxKey || v[3] != kMaxKey || v[4] != kMaxKey || v[5] != kMaxKey))
                continue;
            v[6] = v[7] = kMaxKey;
            warp_bitonic_sort<8>(v, lane);
            worst = __shfl_sync(FULL, v[1], 31);
        }
        const u64 kth = __shfl_sync(FULL, v[1], 31);
        sm.ovf[lane] = v[0];
        sm.ovf[32 + lane] = v[1];
        no = __popc(__ballot_sync(FULL, v[0] != kMaxKey)) + __popc(__ballot_sync(FULL, v[1] != kMaxKey));
        // keep the global entries beyond kth that are still in bound
        int w = 0;
        u64 mn = kMaxKey;
        for (int base = 0; base < ng; base += 32) {
            int e = base + lane;
            u64 kv = e < ng ? gpool[e] : kMaxKey;
            bool keep = e < ng && kv > kth && in_bound(kv);
            unsigned km = __ballot_sync(FULL, keep);
            __syncwarp();
            if (keep) {
                gpool[w + __popc(km & lanemask_lt(lane))] = kv;
                mn = kv < mn ? kv : mn;
            }
            w += __popc(km);
            __syncwarp();
        }
        ng = w;
        tau = warp_min_u64(mn);
        __syncwarp();
    }

    // Refills the empty head with the 32 nearest in-bound overflow keys.
    __device__ void refill_head()
    {
        if (no == 0) {
            if (ng == 0)
                return;
            refill_ovf();
        }
        constexpr int N = kOvf / 32;
        u64 v[N];
#pragma unroll
        for (int i = 0; i < N; ++i) {
            const int e = i * 32 + lane;
            const u64 kv = e < no ? sm.ovf[e] : kMaxKey;
            v[i] = (kv != kMaxKey && in_bound(kv)) ? kv : kMaxKey;
        }
        warp_bitonic_sort<N>(v, lane);
        head.v[0] = v[0];
        nh = __popc(__ballot_sync(FULL, v[0] != kMaxKey));
        int m = 0;
#pragma unroll
        for (int i = 1; i < N; ++i)
            m += __popc(__ballot_sync(FULL, v[i] != kMaxKey));
        __syncwarp();
#pragma unroll
        for (int i = 1; i < N; ++i)
            if ((i - 1) * 32 + lane < m)
                sm.ovf[(i - 1) * 32 + lane] = v[i];
        no = m;
        __syncwarp();
    }

    // Appends the keys of the lanes with `put` (all < tau) to the shared overflow,
    // making room first if they do not fit; keys that end up >= tau after that
    // go to the global pool.
    __device__ void ovf_append_many(bool put, u64 key)
    {
        unsigned m = __ballot_sync(FULL, put);
        if (!m)
            return;
        if (no + __popc(m) > kOvf) {
            make_room(__popc(m));  // tau may drop
            const bool far = put && key >= tau;
            gpool_append(far, key);
            put = put && !far;
            m = __ballot_sync(FULL, put);
        }
        if (put)
            sm.ovf[no + __popc(m & lanemask_lt(lane))] = key;
        no += __popc(m);
        __syncwarp();
    }

    // Adds the batch members marked `push` to S.  Keys >= tau go to the global
    // pool and keys >= the head's maximum to the overflow, each in one step;
    // only keys that enter the sorted head are inserted one at a time.  While S
    // is the head alone (no overflow, empty pool) every key is inserted in turn.
    __device__ void pool_push(bool push, u64 key)
    {
        unsigned pm = __ballot_sync(FULL, push);
        if (!pm)
            return;
        if (no > 0 || ng > 0) {
            const bool far = push && key >= tau;
            gpool_append(far, key);
            push = push && !far;
            const u64 hmax = nh > 0 ? __shfl_sync(FULL, head.v[0], nh - 1) : kMaxKey;
            const bool to_ovf = push && key >= hmax;
            ovf_append_many(to_ovf, key);
            push = push && !to_ovf;
            pm = __ballot_sync(FULL, push);
        }
        while (pm) {
            const int src = __ffs(pm) - 1;
            pm &= pm - 1;
            const u64 ck = __shfl_sync(FULL, key, src);
            if (ck >= tau) {
                gpool_append(lane == 0, ck);
                continue;
            }
            const u64 hmax = nh > 0 ? __shfl_sync(FULL, head.v[0], nh - 1) : kMaxKey;
            const bool only_head = no == 0 && ng == 0;
            if (ck < hmax || (only_head && nh < 32)) {
                if (nh == 32)
                    ovf_append(hmax);  // the evicted maximum stays >= the rest of the head
                head.insert_at(head.rank(ck), ck, lane, 32);
                nh = min(nh + 1, 32);
            } else {
                ovf_append(ck);
            }
        }
    }

    // Removes and returns the minimum of S (the head's first key); refills the
    // head when it runs empty.
    __device__ u64 pool_pop()
    {
        const u64 top = __shfl_sync(FULL, head.v[0], 0);
        head.pop_front(lane);
        --nh;
        if (nh == 0 && (no > 0 || ng > 0))
            refill_head();
        return top;
    }

    // ---------------------------------------------------------------- one batch

    // Tests a batch of up to 32 ids (one per lane, -1 = none) and applies it.
    // With `predict`, loads the adjacency row of the node expanded next.
    __device__ void batch(int id, bool init, bool predict)
    {
#if ONNG_SEARCH_VISIT == 1
        const bool isnew = visit_batch(id);
        const unsigned mask = __ballot_sync(FULL, isnew);
        if (!mask)
            return;
        const int nnew = __popc(mask);
        ndc += nnew;
#else
        begin_batch();
        bool isnew = id >= 0 && visit(id);
        unsigned mask = __ballot_sync(FULL, isnew);
        if (!mask)
            return;
        int nnew = __popc(mask);
        ndc += nnew;
        if (spill) {
            const int pos = nlog + __popc(mask & lanemask_lt(lane));
            if (isnew && pos < kVisitLog)
                glog[pos] = id;
            nlog += nnew;
        } else {
            nvis += nnew;
        }
#endif
        __syncwarp();
        float d2 = distances<Loader<T>>(xs, id, mask);
        u64 key = pack_key(d2, id);
        if (init && a.feat) {
            float sd = isnew ? sqrtf(d2) : 0.f;
#pragma unroll
            for (int off = 16; off >= 1; off >>= 1)
                sd += __shfl_xor_sync(FULL, sd, off);
            seed_sum += sd;
            seed_cnt += nnew;
        }
        if (predict) {
            // next pop = min(S head, nearest batch member if it is pushed); the
            // batch minimum by (distance bits, id) from two warp reductions
            const unsigned dmin = __reduce_min_sync(FULL, isnew ? __float_as_uint(d2) : 0xFFFFFFFFu);
            const unsigned imin = __reduce_min_sync(FULL, isnew && __float_as_uint(d2) == dmin ? (unsigned)id
                                                                                               : 0xFFFFFFFFu);
            const u64 bmin = dmin == 0xFFFFFFFFu ? kMaxKey : ((u64)dmin << 32) | imin;
            const u64 top = __shfl_sync(FULL, head.v[0], 0);
            const u64 next = (key_d2(bmin) <= bnd && bmin < top) ? bmin : top;
            if (next != kMaxKey) {
                pf_node = key_id(next);
                pf_id = graph_id(lane < es ? a.adj[(int64_t)pf_node * a.adj_w + lane] : -1);
            }
        }
        // R <- the best kk of R and the batch
        unsigned cm = __ballot_sync(FULL, isnew && (init || !rset || d2 <= r2));
        while (cm) {
            int src = __ffs(cm) - 1;
            cm &= cm - 1;
            u64 ck = __shfl_sync(FULL, key, src);
            if (init || !rset || key_d2(ck) <= r2) {
                if (r_insert(ck) && !init)
                    ++rins;
                if (!init && cnt == kk) {
                    rset = true;
                    r2 = key_d2(res.get(kk - 1));
                }
            }
        }
        update_bound();
        // S <- S + batch members within r(1+eps)
        pool_push(isnew && d2 <= bnd, key);
#if ONNG_SEARCH_PREFETCH
        if (predict && pf_node >= 0 && pf_id >= 0) {
            // the row of the next node is in: its neighbours' vectors into L2
            const int bytes = a.d * (int)sizeof(T);  // float32 4, bfloat16 2, e4m3 1 byte per coordinate
            const char *row = static_cast<const char *>(xs) + (int64_t)pf_id * bytes;
            for (int off = 0; off < bytes; off += 128)
                asm volatile("prefetch.global.L2 [%0];" ::"l"(row + off));
        }
#endif
    }

    __device__ void run(int64_t q)
    {
        const int d = a.d;
        const float *qp = a.Q + q * d;
#pragma unroll
        for (int v = 0; v < V; ++v) {
            int c = lane + 32 * v;
            qv[v] = c < (d >> 2) ? __ldg(reinterpret_cast<const float4 *>(qp) + c) : make_float4(0.f, 0.f, 0.f, 0.f);
            if constexpr (std::is_same<T, __nv_fp8_e4m3>::value)
                sv[v] = c < (d >> 2) ? __ldg(reinterpret_cast<const float4 *>(a.scale8) + c)
                                     : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        const float eps = a.eps_q ? a.eps_q[q] : a.eps;
        es = a.es_q ? a.es_q[q] : a.e_s;
        if (es <= 0)
            es = INT_MAX;
        padded = a.adj != nullptr && es <= a.adj_w;
        const bool predict = padded && es <= 32;
        f2 = isinf(eps) ? INFINITY : (1.0 + (double)eps) * (1.0 + (double)eps);
        for (int i = lane; i < HV / 4; i += 32)
            reinterpret_cast<int4 *>(sm.vis)[i] = make_int4(-1, -1, -1, -1);
        head.clear();
        res.clear();
        nh = no = ng = cnt = ndc = nexp = nvis = nlog = nscan = 0;
        pf_node = -1;
        kk = a.k;
        flags = 0;
#ifdef ONNG_CHECK
        nnz_chk = a.row_ptr[a.n];
#endif
        spill = rset = stop = capped = false;
        seed_cnt = rins = 0;
        seed_sum = 0.f;
        r2 = INFINITY;
        tau = kMaxKey;
        bound2 = INFINITY;
        bnd = INFINITY;
        __syncwarp();
        for (int c0 = 0; c0 < a.n_seed; c0 += 32) {
            int id = -1;
            if (c0 + lane < a.n_seed) {
                id = a.seeds[q * a.n_seed + c0 + lane];
                if (id >= a.n)
                    id = -1;
            }
            batch(id < 0 ? -1 : id, true, false);
        }
        seed1 = head.get(0);
        seed2 = head.get(1);
        while (!stop) {
            if (nh == 0) {
                refill_head();
                if (nh == 0)
                    break;
            }
            if (a.max_exp > 0 && nexp >= a.max_exp) {
                // capped with a candidate still to expand (not merely pending termination)
                capped = key_d2(__shfl_sync(FULL, head.v[0], 0)) <= bnd;
                if (capped)
                    flags |= ONNG_FLAG_LIMIT;
                break;
            }
            const u64 sk = pool_pop();
            if (key_d2(sk) > bnd)
                break;
            ++nexp;
            const int s = key_id(sk);
            if (predict) {
                const int id = s == pf_node ? pf_id : graph_id(lane < es ? a.adj[(int64_t)s * a.adj_w + lane] : -1);
                pf_node = -1;
                nscan += __popc(__ballot_sync(FULL, id >= 0));
                batch(id, false, true);
            } else if (padded) {
                for (int c0 = 0; c0 < es && !stop; c0 += 32) {
                    const int id = graph_id(c0 + lane < es ? a.adj[(int64_t)s * a.adj_w + c0 + lane] : -1);
                    const unsigned got = __ballot_sync(FULL, id >= 0);
                    if (!got)
                        break;
                    nscan += __popc(got);
                    batch(id, false, false);
                }
            } else {
                const int64_t beg = a.row_ptr[s];
                int64_t deg = a.row_ptr[s + 1] - beg;
#ifdef ONNG_CHECK
                if (beg < 0 || deg < 0 || beg + deg > nnz_chk) {
                    flags |= ONNG_FLAG_CHECK;
                    deg = 0;
                }
#endif
                const int m = deg < (int64_t)es ? (int)deg : es;
                nscan += m;
                for (int c0 = 0; c0 < m && !stop; c0 += 32) {
                    int id = graph_id(c0 + lane < m ? a.col[beg + c0 + lane] : -1);
                    batch(id, false, false);
                }
            }
        }
    }

    // Rescores the kept list in float32 against X and keeps the best k_out.
    __device__ void rerank()
    {
        u64 nk[KR];
#pragma unroll
        for (int i = 0; i < KR; ++i) {
            const int id = res.v[i] == kMaxKey ? -1 : key_id(res.v[i]);
            const unsigned mask = __ballot_sync(FULL, id >= 0);
            const float dv = distances<Loader<float>>(a.X, id, mask);
            nk[i] = id >= 0 ? pack_key(dv, id) : kMaxKey;
        }
        res.clear();
        cnt = 0;
        kk = a.k_out;
#pragma unroll
        for (int i = 0; i < KR; ++i) {
            unsigned m = __ballot_sync(FULL, nk[i] != kMaxKey);
            while (m) {
                const int src = __ffs(m) - 1;
                m &= m - 1;
                r_insert(__shfl_sync(FULL, nk[i], src));
            }
        }
    }

    // Probe features after the capped search (all logs natural, distances Euclidean).
    __device__ void features(int64_t q)
    {
        const u64 rbk = res.get(0);
        const u64 rkk = res.get(cnt > 0 ? cnt - 1 : 0);
        const u64 hk = __shfl_sync(FULL, head.v[0], 0);
        if (lane != 0)
            return;
        const float e6 = 1e-6f;
        const float ds1 = seed1 == kMaxKey ? 0.f : sqrtf(key_d2(seed1));
        const float ds2 = seed2 == kMaxKey ? ds1 : sqrtf(key_d2(seed2));
        const float dmean = seed_cnt > 0 ? seed_sum / (float)seed_cnt : ds1;
        const float rb = cnt > 0 ? sqrtf(key_d2(rbk)) : ds1;
        const float rk = cnt > 0 ? sqrtf(key_d2(rkk)) : ds1;
        const float bound = (rset && !isinf(f2)) ? (float)sqrt(bound2) : INFINITY;
        float top = capped ? fminf(sqrtf(key_d2(hk)), bound) : bound;
        if (isinf(top))
            top = rk;
        float *f = a.feat + q * kFeat;
        f[0] = a.target;
        f[1] = logf(ds1 + e6);
        f[2] = logf((ds2 + e6) / (ds1 + e6));
        f[3] = logf((dmean + e6) / (ds1 + e6));
        f[4] = logf((rb + e6) / (ds1 + e6));
        f[5] = logf((rk + e6) / (rb + e6));
        f[6] = logf((top + e6) / (rb + e6));
        f[7] = (float)ndc / (float)max(1, seed_cnt + nscan);
        f[8] = (float)nexp / (float)max(1, a.max_exp);
        f[9] = log1pf((float)ndc);
        f[10] = (float)rins / (float)max(1, ndc);
        f[11] = rset ? 1.f : 0.f;
        f[12] = logf((rk + e6) / (ds1 + e6));
        f[13] = log1pf((float)nscan);
        f[14] = capped ? 1.f : 0.f;
        f[15] = logf((float)a.d) / 8.f;
    }

    __device__ void write(int64_t q)
    {
        if (a.feat)
            features(q);
        const int k = a.k_out;
#pragma unroll
        for (int i = 0; i < KR; ++i) {
            const int e = i * 32 + lane;
            if (e < k && a.out_ids) {
                a.out_ids[q * k + e] = e < cnt ? key_id(res.v[i]) : -1;
                a.out_dist[q * k + e] = e < cnt ? sqrtf(key_d2(res.v[i])) : INFINITY;
            }
        }
#ifdef ONNG_CHECK
        if (__any_sync(FULL, lane < 4 && sm.canary[lane] != kCanary + lane))
            flags |= ONNG_FLAG_CHECK;
#endif
        if (a.stats && lane == 0) {
            a.stats[q * 4 + 0] = ndc;
            a.stats[q * 4 + 1] = nexp;
            a.stats[q * 4 + 2] = nscan;
            a.stats[q * 4 + 3] = (int)flags;
        }
    }
};

// Resident CTAs per SM the register budget is sized for.  Shared memory holds
// 6 CTAs of warps with a 2048-slot table and 128 overflow keys (37 KB a CTA).
template <class T> __host__ __device__ constexpr int min_blocks(int V, int KR)
{
    return V <= 2 && KR == 1 ? Tune<T>::minb : 3;
}

template <int V, class T, int HV, int KR>
__global__ void __launch_bounds__(kWarpsPerCta * 32, min_blocks<T>(V, KR)) search_kernel(SearchArgs a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    auto *smem = reinterpret_cast<WarpSmem<HV, Tune<T>::ovf> *>(smem_raw);
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int64_t slot = (int64_t)blockIdx.x * kWarpsPerCta + warp;
    const void *xs = std::is_same<T, float>::value           ? static_cast<const void *>(a.X)
                     : std::is_same<T, __nv_bfloat16>::value ? static_cast<const void *>(a.Xb)
                                                              : static_cast<const void *>(a.X8);
    Warp<V, T, HV, KR> w(smem[warp], a, xs, lane, a.gbits + slot * a.bits_words, a.glog + slot * kVisitLog,
                         a.gpool + slot * a.gpool_cap);
#ifdef ONNG_CHECK
    if (lane < 4)
        smem[warp].canary[lane] = kCanary + lane;
    __syncwarp();
#endif
    for (;;) {
        int q = 0;
        if (lane == 0)
            q = atomicAdd(a.counter, 1);
        q = __shfl_sync(FULL, q, 0);
        if (q >= a.nq)
            break;
        w.run(q);
        w.clear_bits();
        if constexpr (!std::is_same<T, float>::value)
            w.rerank();
        w.write(q);
        __syncwarp();
    }
}

struct Launch {
    void (*fn)(SearchArgs);
    size_t smem;
};

// The search kernel for vector type T with V float4 chunks per lane (d <= 128 V)
// and a kept list of at most 32 KR keys (KR = 1 or kMaxK / 32); defined in
// search_inst.cu.
template <class T, int V, int KR> Launch pick();
#define ONNG_SEARCH_DECLARE_PICK(T, V)   \
    template <> Launch pick<T, V, 1>(); \
    template <> Launch pick<T, V, kMaxK / 32>();
#define ONNG_SEARCH_DECLARE_PICKS(T)    \
    ONNG_SEARCH_DECLARE_PICK(T, 1)      \
    ONNG_SEARCH_DECLARE_PICK(T, 2)      \
    ONNG_SEARCH_DECLARE_PICK(T, 4)      \
    ONNG_SEARCH_DECLARE_PICK(T, 8)
ONNG_SEARCH_DECLARE_PICKS(float)
ONNG_SEARCH_DECLARE_PICKS(__nv_bfloat16)
ONNG_SEARCH_DECLARE_PICKS(__nv_fp8_e4m3)
#undef ONNG_SEARCH_DECLARE_PICKS
#undef ONNG_SEARCH_DECLARE_PICK

}  // namespace sk
}  // namespace onng
