// KnnSearch (Algorithm 1) on the GPU: one warp per query.
//
// Per warp, in shared memory:
//   - the visited set C as an exact open-addressing hash (linear probing).  The
//     paper's Set/IsSet table (Sec. 2.5) keeps the first id of a bucket inline and
//     chains collisions; on the GPU a flat table probed by 32 lanes at once is
//     cheaper.  Past 3/4 load, new ids go to a per-warp table in global memory.
//   - the candidate set S as an unsorted pool of (distance, id) keys popped by a
//     warp-wide min.  An entry beyond r(1+eps) can never be expanded (r only
//     shrinks, and popping it ends the search), so such entries are dropped
//     whenever room is needed.  If the in-bound entries still do not fit, the
//     farther half moves to a per-warp pool in global memory; every key there
//     is >= tau > every key in shared memory, so the shared pool's minimum is
//     the minimum of S, and the global pool refills the shared one only when the
//     latter runs empty.  S stays exact.
//   - the result set R as a (distance, id)-sorted list of at most k entries.
// The up-to-e_s neighbours of the expanded node are tested and their vectors
// gathered together (coalesced 16-byte loads, several vectors in flight per
// lane, one transposed butterfly reduction for all of them).  R then takes the k
// best of R and the batch, and S takes the batch members within the new
// r(1+eps).  Applying a batch at once yields the same R, the same r after the
// batch and, since S only loses entries that can never be expanded, the same
// expansion order as the one-at-a-time loop of Algorithm 1.
//
// Adjacency is read from the CSR lists, or from an optional padded table
// adj [n, width] (-1 padded) that holds each node's first `width` entries, which
// saves the row-pointer indirection per expansion.
//
// Distances are squared float32 sums of (q - x)^2; bounds are compared in
// double: d^2 <= r^2 (1 + eps)^2.  For integer-valued inputs with squared
// distances below 2^24 every decision then equals the float64 algorithm's.
#include <cuda_bf16.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <type_traits>

#include "common.cuh"
#include "warp_sort.cuh"

#ifndef ONNG_SEARCH_HV
#define ONNG_SEARCH_HV 2048
#endif

namespace onng {
namespace {

typedef unsigned long long u64;

constexpr int kWarpsPerCta = 4;
constexpr int kMaxK = 128;
constexpr int kMaxSeed = 64;
constexpr int kPool = 256;           // shared-memory candidate pool entries
constexpr int kGlobalVisit = 65536;  // per-warp visited spill region (ints): tables of 4K, 8K, 16K, 32K
constexpr int kSpillFirst = 4096;    // first spill table size; each growth doubles it
constexpr int kGlobalPool = 16384;   // per-warp candidate spill pool entries
constexpr u64 kMaxKey = ~0ull;

struct SearchArgs {
    const int64_t *row_ptr;
    const int32_t *col;
    const int32_t *adj;
    int adj_w;
    const float *X;
    const uint16_t *Xb;
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
    int32_t *out_ids;
    float *out_dist;
    int32_t *stats;
    int *counter;
    int *gvis;  // [slots, kGlobalVisit]
    u64 *gpool; // [slots, kGlobalPool]
};

template <int HV> struct WarpSmem {
    int vis[HV];
    u64 pool[kPool];
    u64 res[kMaxK];
};

__host__ __device__ constexpr int log2i(int v) { return v <= 1 ? 0 : 1 + log2i(v >> 1); }

__device__ __forceinline__ unsigned lanemask_lt(int lane) { return (1u << lane) - 1u; }

__device__ __forceinline__ unsigned hash_id(int id) { return static_cast<unsigned>(id) * 0x9E3779B1u; }

__device__ __forceinline__ float key_d2(u64 k) { return __uint_as_float((unsigned)(k >> 32)); }
__device__ __forceinline__ int key_id(u64 k) { return (int)(unsigned)(k & 0xFFFFFFFFull); }

__device__ __forceinline__ u64 warp_min_u64(u64 v)
{
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) {
        u64 o = __shfl_xor_sync(0xffffffffu, v, off);
        v = o < v ? o : v;
    }
    return v;
}

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

// Sums v[g] over the warp for G values at once.  Afterwards every lane holds
// the full sum of one value index; holder_lane(g) names a lane holding value g.
template <int G> __device__ __forceinline__ float transpose_reduce(float (&v)[G], int lane)
{
    static_assert(G == 1 || G == 2 || G == 4 || G == 8, "G");
    if constexpr (G >= 2) {
        const bool hi = lane & 16;
#pragma unroll
        for (int i = 0; i < G / 2; ++i) {
            float send = hi ? v[i] : v[i + G / 2];
            float keep = hi ? v[i + G / 2] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
        }
    }
    if constexpr (G >= 4) {
        const bool hi = lane & 8;
#pragma unroll
        for (int i = 0; i < G / 4; ++i) {
            float send = hi ? v[i] : v[i + G / 4];
            float keep = hi ? v[i + G / 4] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
        }
    }
    if constexpr (G >= 8) {
        const bool hi = lane & 4;
        float send = hi ? v[0] : v[1];
        float keep = hi ? v[1] : v[0];
        v[0] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
    }
    float s = v[0];
    constexpr int first = G == 1 ? 16 : G == 2 ? 8 : G == 4 ? 4 : 2;
#pragma unroll
    for (int off = first; off >= 1; off >>= 1)
        s += __shfl_xor_sync(0xffffffffu, s, off);
    return s;
}

template <int G> __device__ __forceinline__ int holder_lane(int g)
{
    if constexpr (G == 1)
        return 0;
    else if constexpr (G == 2)
        return g << 4;
    else if constexpr (G == 4)
        return ((g >> 1) & 1) << 4 | (g & 1) << 3;
    else
        return ((g >> 2) & 1) << 4 | ((g >> 1) & 1) << 3 | (g & 1) << 2;
}

template <int V, class T, int HV> struct Warp {
    static constexpr int G = V >= 8 ? 1 : V >= 4 ? 2 : V >= 2 ? 4 : 8;  // vectors per gather round
    WarpSmem<HV> &sm;
    const SearchArgs &a;
    const void *xs;  // vectors the search reads (float32 or bfloat16)
    int lane;
    int *gvis;
    u64 *gpool;
    float4 qv[V];
    // per-query state, uniform across the warp
    int ns, ng, cnt, ndc, nexp, nvis, nvis_g, kk, nscan, gcap;
    unsigned flags;
    bool spill, rset, stop;
    float r2;
    u64 tau;  // every key in the global pool is >= tau (kMaxKey when it is empty)
    double f2, bound2;

    __device__ Warp(WarpSmem<HV> &s, const SearchArgs &args, const void *x, int ln, int *gv, u64 *gp)
        : sm(s), a(args), xs(x), lane(ln), gvis(gv), gpool(gp)
    {
    }

    __device__ bool in_bound(u64 key) const { return (double)key_d2(key) <= bound2; }

    // ---------------------------------------------------------------- visited set

    // Test-and-set of one id by the calling lane; true if newly visited.
    __device__ bool visit(int id)
    {
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
        return gvisit(gvis + gcap, gcap, id) == 1;
    }

    // Insert into a spill table of `cap` slots at `tab`: 1 inserted, 0 present.
    __device__ int gvisit(int *tab, int cap, int id)
    {
        unsigned hg = hash_id(id) >> (32 - __ffs(cap) + 1);
        for (int t = 0; t < cap; ++t) {
            int old = atomicCAS(&tab[hg], -1, id);
            if (old == -1)
                return 1;
            if (old == id)
                return 0;
            hg = (hg + 1) & (cap - 1);
        }
        return 1;  // unreachable: tables are kept below half load
    }

    // Clears a spill table of `cap` slots at offset cap of the region.
    __device__ void gclear(int cap)
    {
        int4 m1 = make_int4(-1, -1, -1, -1);
        int4 *g4 = reinterpret_cast<int4 *>(gvis + cap);
        for (int i = lane; i < cap / 4; i += 32)
            g4[i] = m1;
        __syncwarp();
    }

    // Starts the spill table when the shared table nears 3/4 load, and doubles
    // the spill table (tables of size c live at offset c, so they never overlap)
    // before a batch could take it past half load.
    __device__ void begin_batch()
    {
        if (!spill && nvis >= HV / 4 * 3 - 32) {
            spill = true;
            gcap = kSpillFirst;
            gclear(gcap);
        }
        if (spill && nvis_g + 32 >= gcap / 2 && gcap * 2 <= kGlobalVisit / 2) {
            const int ncap = gcap * 2;
            gclear(ncap);
            const int *old = gvis + gcap;
            for (int i = lane; i < gcap; i += 32) {
                int v = old[i];
                if (v != -1)
                    gvisit(gvis + ncap, ncap, v);
            }
            __syncwarp();
            gcap = ncap;
        }
    }

    // ---------------------------------------------------------------- distances

    // Squared distances of the ids held by the lanes in `mask`; returns this lane's.
    template <class L> __device__ float distances(const void *base, int id, unsigned mask)
    {
        float mine = 0.0f;
        const int chunks = a.d >> 2;
        while (mask) {
            int src[G];
            int gid[G];
#pragma unroll
            for (int g = 0; g < G; ++g) {
                src[g] = mask ? __ffs(mask) - 1 : -1;
                if (mask)
                    mask &= mask - 1;
                gid[g] = __shfl_sync(0xffffffffu, id, src[g] < 0 ? 0 : src[g]);
            }
            float4 xv[G][V];
#pragma unroll
            for (int g = 0; g < G; ++g)
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    int c = lane + 32 * v;
                    xv[g][v] = (src[g] >= 0 && c < chunks) ? L::load(base, gid[g], a.d, c)
                                                           : make_float4(0.f, 0.f, 0.f, 0.f);
                }
            float acc[G];
#pragma unroll
            for (int g = 0; g < G; ++g) {
                acc[g] = 0.0f;
#pragma unroll
                for (int v = 0; v < V; ++v) {
                    int c = lane + 32 * v;
                    if (src[g] >= 0 && c < chunks)
                        acc[g] = sqdiff4(qv[v], xv[g][v], acc[g]);
                }
            }
            float red = transpose_reduce<G>(acc, lane);
#pragma unroll
            for (int g = 0; g < G; ++g) {
                float s = __shfl_sync(0xffffffffu, red, holder_lane<G>(g));
                if (lane == src[g])
                    mine = s;
            }
        }
        return mine;
    }

    // ---------------------------------------------------------------- result list

    // Inserts key into the sorted result list, keeping at most kk entries.
    __device__ void r_insert(u64 key)
    {
        int pos = 0;
#pragma unroll
        for (int s = 0; s < kMaxK / 32; ++s) {
            int i = s * 32 + lane;
            pos += __popc(__ballot_sync(0xffffffffu, i < cnt && sm.res[i] < key));
        }
        if (pos >= kk)
            return;
        int last = min(cnt, kk - 1);  // entries [pos, last) move up by one
        u64 t[kMaxK / 32];
#pragma unroll
        for (int s = 0; s < kMaxK / 32; ++s) {
            int i = s * 32 + lane;
            if (i >= pos && i < last)
                t[s] = sm.res[i];
        }
        __syncwarp();
#pragma unroll
        for (int s = 0; s < kMaxK / 32; ++s) {
            int i = s * 32 + lane;
            if (i >= pos && i < last)
                sm.res[i + 1] = t[s];
        }
        if (lane == 0)
            sm.res[pos] = key;
        __syncwarp();
        cnt = min(cnt + 1, kk);
    }

    __device__ void update_bound()
    {
        bound2 = (rset && !isinf(f2)) ? (double)r2 * f2 : INFINITY;
    }

    // ---------------------------------------------------------------- candidate pool

    // Drops shared-pool entries beyond the bound.
    __device__ void pool_compact()
    {
        int w = 0;
        for (int base = 0; base < ns; base += 32) {
            int i = base + lane;
            u64 kv = i < ns ? sm.pool[i] : kMaxKey;
            bool keep = i < ns && in_bound(kv);
            unsigned km = __ballot_sync(0xffffffffu, keep);
            __syncwarp();
            if (keep)
                sm.pool[w + __popc(km & lanemask_lt(lane))] = kv;
            w += __popc(km);
            __syncwarp();
        }
        ns = w;
    }

    // Appends `count` keys (one per lane in `mask`) to the global pool.
    __device__ void gpool_append(bool put, u64 key)
    {
        unsigned m = __ballot_sync(0xffffffffu, put);
        if (!m)
            return;
        if (put) {
            int dst = ng + __popc(m & lanemask_lt(lane));
            if (dst < kGlobalPool)
                gpool[dst] = key;
        }
        if (ng + __popc(m) > kGlobalPool)
            flags |= ONNG_FLAG_S_OVERFLOW;
        ng = min(ng + __popc(m), kGlobalPool);
    }

    // Moves the farther half of the (full) shared pool to the global pool.
    __device__ void spill_half()
    {
        constexpr int N = kPool / 32;
        u64 v[N];
#pragma unroll
        for (int i = 0; i < N; ++i) {
            int e = i * 32 + lane;
            v[i] = e < ns ? sm.pool[e] : kMaxKey;
        }
        warp_bitonic_sort<N>(v, lane);
        constexpr int keep = kPool / 2;
        __syncwarp();
#pragma unroll
        for (int i = 0; i < N; ++i) {
            int e = i * 32 + lane;
            if (e < keep && e < ns)
                sm.pool[e] = v[i];
        }
        u64 first_moved = __shfl_sync(0xffffffffu, v[keep / 32], 0);
#pragma unroll
        for (int i = keep / 32; i < N; ++i) {
            int e = i * 32 + lane;
            gpool_append(e < ns, v[i]);
        }
        __syncwarp();
        if (ns > keep) {
            tau = first_moved;
            ns = keep;
        }
    }

    // Refills the empty shared pool with the nearest in-bound global entries.
    __device__ void refill()
    {
        constexpr int M = kPool / 2;  // entries brought back
        u64 v[16];
#pragma unroll
        for (int i = 0; i < 16; ++i)
            v[i] = kMaxKey;
        for (int base = 0; base < ng; base += 256) {
#pragma unroll
            for (int i = 4; i < 12; ++i) {
                int e = base + (i - 4) * 32 + lane;
                u64 kv = e < ng ? gpool[e] : kMaxKey;
                v[i] = (kv != kMaxKey && in_bound(kv)) ? kv : kMaxKey;
            }
#pragma unroll
            for (int i = 12; i < 16; ++i)
                v[i] = kMaxKey;
            warp_bitonic_sort<16>(v, lane);  // the M smallest end up in v[0..3]
        }
        const u64 kth = __shfl_sync(0xffffffffu, v[(M - 1) / 32], 31);
        int m = 0;
#pragma unroll
        for (int i = 0; i < M / 32; ++i) {
            int e = i * 32 + lane;
            bool has = v[i] != kMaxKey;
            if (has)
                sm.pool[e] = v[i];
            m += __popc(__ballot_sync(0xffffffffu, has));
        }
        // keep the global entries that are beyond kth and still in bound
        int w = 0;
        u64 mn = kMaxKey;
        for (int base = 0; base < ng; base += 32) {
            int e = base + lane;
            u64 kv = e < ng ? gpool[e] : kMaxKey;
            bool keep = e < ng && kv > kth && in_bound(kv);
            unsigned km = __ballot_sync(0xffffffffu, keep);
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
        ns = m;
        __syncwarp();
    }

    // Adds the batch members marked `push` to S.
    __device__ void pool_push(bool push, u64 key)
    {
        bool to_s = push && key < tau;
        unsigned sm_mask = __ballot_sync(0xffffffffu, to_s);
        int nps = __popc(sm_mask);
        if (ns + nps > kPool) {
            pool_compact();
            if (ns + nps > kPool) {
                spill_half();
                to_s = push && key < tau;
                sm_mask = __ballot_sync(0xffffffffu, to_s);
                nps = __popc(sm_mask);
            }
        }
        if (to_s)
            sm.pool[ns + __popc(sm_mask & lanemask_lt(lane))] = key;
        ns += nps;
        gpool_append(push && !to_s, key);
        __syncwarp();
    }

    // Warp-wide min of the shared pool; removes and returns it.
    __device__ u64 pool_pop()
    {
        u64 best = kMaxKey;
        int bx = -1;
        for (int i = lane; i < ns; i += 32) {
            u64 kv = sm.pool[i];
            if (kv < best) {
                best = kv;
                bx = i;
            }
        }
#pragma unroll
        for (int off = 16; off >= 1; off >>= 1) {
            u64 ob = __shfl_xor_sync(0xffffffffu, best, off);
            int ox = __shfl_xor_sync(0xffffffffu, bx, off);
            if (ob < best) {
                best = ob;
                bx = ox;
            }
        }
        __syncwarp();
        if (lane == 0)
            sm.pool[bx] = sm.pool[ns - 1];
        --ns;
        __syncwarp();
        return best;
    }

    // ---------------------------------------------------------------- one batch

    // Tests a batch of up to 32 ids (one per lane, -1 = none) and applies it.
    __device__ void batch(int id, bool init)
    {
        begin_batch();
        bool isnew = id >= 0 && visit(id);
        unsigned mask = __ballot_sync(0xffffffffu, isnew);
        if (!mask)
            return;
        int nnew = __popc(mask);
        ndc += nnew;
        if (spill)
            nvis_g += nnew;
        else
            nvis += nnew;
        __syncwarp();
        float d2 = distances<Loader<T>>(xs, id, mask);
        u64 key = pack_key(d2, id);
        // R <- the best kk of R and the batch
        unsigned cm = __ballot_sync(0xffffffffu, isnew && (init || !rset || d2 <= r2));
        while (cm) {
            int src = __ffs(cm) - 1;
            cm &= cm - 1;
            u64 ck = __shfl_sync(0xffffffffu, key, src);
            if (init || !rset || key_d2(ck) <= r2) {
                r_insert(ck);
                if (!init && cnt == kk) {
                    rset = true;
                    r2 = key_d2(sm.res[kk - 1]);
                }
            }
        }
        update_bound();
        // S <- S + batch members within r(1+eps)
        pool_push(isnew && (double)d2 <= bound2, key);
        if (nvis_g + 32 >= gcap / 2 && gcap * 2 > kGlobalVisit / 2) {
            flags |= ONNG_FLAG_VISIT_OVERFLOW;
            stop = true;
        }
    }

    __device__ void run(int64_t q)
    {
        const int d = a.d;
        const float *qp = a.Q + q * d;
#pragma unroll
        for (int v = 0; v < V; ++v) {
            int c = lane + 32 * v;
            qv[v] = c < (d >> 2) ? __ldg(reinterpret_cast<const float4 *>(qp) + c) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        const float eps = a.eps_q ? a.eps_q[q] : a.eps;
        int es = a.es_q ? a.es_q[q] : a.e_s;
        if (es <= 0)
            es = INT_MAX;
        const bool padded = a.adj != nullptr && es <= a.adj_w;
        f2 = isinf(eps) ? INFINITY : (1.0 + (double)eps) * (1.0 + (double)eps);
        for (int i = lane; i < HV; i += 32)
            sm.vis[i] = -1;
        ns = ng = cnt = ndc = nexp = nvis = nvis_g = nscan = 0;
        gcap = kSpillFirst;
        kk = a.k;
        flags = 0;
        spill = rset = stop = false;
        r2 = INFINITY;
        tau = kMaxKey;
        bound2 = INFINITY;
        __syncwarp();
        for (int c0 = 0; c0 < a.n_seed; c0 += 32) {
            int id = -1;
            if (c0 + lane < a.n_seed) {
                id = a.seeds[q * a.n_seed + c0 + lane];
                if (id >= a.n)
                    id = -1;
            }
            batch(id < 0 ? -1 : id, true);
        }
        while (!stop) {
            if (ns == 0) {
                if (ng == 0)
                    break;
                refill();
                if (ns == 0)
                    break;
            }
            const u64 sk = pool_pop();
            if ((double)key_d2(sk) > bound2)
                break;
            if (a.max_exp > 0 && nexp >= a.max_exp) {
                flags |= ONNG_FLAG_LIMIT;
                break;
            }
            ++nexp;
            const int s = key_id(sk);
            if (padded) {
                // first `es` entries of the padded row; -1 marks the end of a short row
                int id = lane < es ? a.adj[(int64_t)s * a.adj_w + lane] : -1;
                nscan += __popc(__ballot_sync(0xffffffffu, id >= 0));
                batch(id, false);
                for (int c0 = 32; c0 < es && !stop; c0 += 32) {
                    id = c0 + lane < es ? a.adj[(int64_t)s * a.adj_w + c0 + lane] : -1;
                    unsigned got = __ballot_sync(0xffffffffu, id >= 0);
                    if (!got)
                        break;
                    nscan += __popc(got);
                    batch(id, false);
                }
            } else {
                const int64_t beg = a.row_ptr[s];
                const int64_t deg = a.row_ptr[s + 1] - beg;
                const int m = deg < (int64_t)es ? (int)deg : es;
                nscan += m;
                for (int c0 = 0; c0 < m && !stop; c0 += 32) {
                    int id = c0 + lane < m ? a.col[beg + c0 + lane] : -1;
                    batch(id, false);
                }
            }
        }
    }

    // Rescores the kept list in float32 against X and keeps the best k_out.
    __device__ void rerank()
    {
        const int m = cnt;
        for (int c0 = 0; c0 < m; c0 += 32) {
            int i = c0 + lane;
            int id = i < m ? key_id(sm.res[i]) : -1;
            unsigned mask = __ballot_sync(0xffffffffu, id >= 0);
            float dv = distances<Loader<float>>(a.X, id, mask);
            if (id >= 0)
                sm.pool[i] = pack_key(dv, id);
        }
        __syncwarp();
        cnt = 0;
        kk = a.k_out;
        for (int i = 0; i < m; ++i)
            r_insert(sm.pool[i]);
    }

    __device__ void write(int64_t q)
    {
        const int k = a.k_out;
        for (int i = lane; i < k; i += 32) {
            a.out_ids[q * k + i] = i < cnt ? key_id(sm.res[i]) : -1;
            a.out_dist[q * k + i] = i < cnt ? sqrtf(key_d2(sm.res[i])) : INFINITY;
        }
        if (a.stats && lane == 0) {
            a.stats[q * 4 + 0] = ndc;
            a.stats[q * 4 + 1] = nexp;
            a.stats[q * 4 + 2] = nscan;
            a.stats[q * 4 + 3] = (int)flags;
        }
    }
};

template <int V, class T, int HV>
__global__ void __launch_bounds__(kWarpsPerCta * 32) search_kernel(SearchArgs a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    auto *smem = reinterpret_cast<WarpSmem<HV> *>(smem_raw);
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int64_t slot = (int64_t)blockIdx.x * kWarpsPerCta + warp;
    const void *xs = std::is_same<T, float>::value ? static_cast<const void *>(a.X) : static_cast<const void *>(a.Xb);
    Warp<V, T, HV> w(smem[warp], a, xs, lane, a.gvis + slot * kGlobalVisit, a.gpool + slot * kGlobalPool);
    for (;;) {
        int q = 0;
        if (lane == 0)
            q = atomicAdd(a.counter, 1);
        q = __shfl_sync(0xffffffffu, q, 0);
        if (q >= a.nq)
            break;
        w.run(q);
        if (!std::is_same<T, float>::value)
            w.rerank();
        w.write(q);
        __syncwarp();
    }
}

__global__ void pad_adjacency_kernel(const int64_t *__restrict__ row_ptr, const int32_t *__restrict__ col, int64_t n,
                                     int width, int32_t *__restrict__ adj)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n * width;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / width;
        const int t = (int)(e % width);
        const int64_t beg = row_ptr[i];
        adj[e] = beg + t < row_ptr[i + 1] ? col[beg + t] : -1;
    }
}

struct Launch {
    void (*fn)(SearchArgs);
    size_t smem;
};

template <int V, class T> Launch pick()
{
    return {search_kernel<V, T, ONNG_SEARCH_HV>, sizeof(WarpSmem<ONNG_SEARCH_HV>) * kWarpsPerCta};
}

template <class T> Launch pick_v(int d)
{
    const int V = (d + 127) / 128;
    if (V <= 1)
        return pick<1, T>();
    if (V <= 2)
        return pick<2, T>();
    if (V <= 4)
        return pick<4, T>();
    if (V <= 8)
        return pick<8, T>();
    return {nullptr, 0};
}

int resident_blocks(const Launch &L, int *per_sm)
{
    ONNG_CUDA_TRY(cudaFuncSetAttribute(reinterpret_cast<const void *>(L.fn),
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.smem),
                  "search: smem attribute");
    ONNG_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, reinterpret_cast<const void *>(L.fn),
                                                                 kWarpsPerCta * 32, L.smem),
                  "search: occupancy");
    if (*per_sm < 1)
        *per_sm = 1;
    return ONNG_OK;
}

constexpr size_t kSlotBytes = (size_t)kGlobalVisit * sizeof(int) + (size_t)kGlobalPool * sizeof(u64);

}  // namespace
}  // namespace onng

using namespace onng;

extern "C" size_t onng_search_workspace_bytes(int64_t nq, const onng_index *idx, const onng_search_params *p)
{
    (void)p;
    Launch L = pick_v<float>(idx ? idx->d : 128);
    int per_sm = 16;
    if (!L.fn || resident_blocks(L, &per_sm) != ONNG_OK)
        per_sm = 16;
    const int64_t blocks = std::min<int64_t>(std::max<int64_t>(1, (nq + kWarpsPerCta - 1) / kWarpsPerCta),
                                             (int64_t)per_sm * num_sms());
    return 256 + (size_t)blocks * kWarpsPerCta * kSlotBytes;
}

extern "C" int onng_pad_adjacency(const int64_t *row_ptr, const int32_t *col, int64_t n, int32_t width, int32_t *adj,
                                  onng_stream_t stream)
{
    ONNG_REQUIRE(n >= 0 && width >= 1, ONNG_E_INVAL, "onng_pad_adjacency: bad sizes");
    if (n == 0)
        return ONNG_OK;
    ONNG_REQUIRE(row_ptr && adj, ONNG_E_INVAL, "onng_pad_adjacency: NULL pointer");
    const int64_t total = n * width;
    const int blocks = (int)std::min<int64_t>((total + 255) / 256, (int64_t)num_sms() * 16);
    pad_adjacency_kernel<<<blocks, 256, 0, to_cuda(stream)>>>(row_ptr, col, n, width, adj);
    return check_launch("onng_pad_adjacency");
}

extern "C" int onng_search(const onng_index *idx, const float *Q, int64_t nq, const onng_search_params *p,
                           const int32_t *seeds, int32_t n_seed, const float *eps_q, const int32_t *es_q,
                           int32_t *out_ids, float *out_dist, int32_t *stats, void *ws, size_t ws_bytes,
                           onng_stream_t stream)
{
    ONNG_REQUIRE(idx && p, ONNG_E_INVAL, "onng_search: NULL index or params");
    ONNG_REQUIRE(nq >= 0 && idx->n > 0 && idx->n <= INT32_MAX, ONNG_E_INVAL, "onng_search: bad sizes");
    ONNG_REQUIRE(idx->d > 0 && idx->d % 4 == 0, ONNG_E_UNSUPPORTED, "onng_search: d must be a positive multiple of 4");
    ONNG_REQUIRE(idx->d <= 1024, ONNG_E_UNSUPPORTED, "onng_search: d > 1024");
    ONNG_REQUIRE(p->k >= 1 && p->k <= kMaxK, ONNG_E_UNSUPPORTED, "onng_search: k must be in [1, %d]", kMaxK);
    ONNG_REQUIRE(n_seed >= 1 && n_seed <= kMaxSeed, ONNG_E_UNSUPPORTED, "onng_search: n_seed must be in [1, %d]",
                 kMaxSeed);
    ONNG_REQUIRE(!std::isnan(p->eps) && p->eps >= 0, ONNG_E_INVAL, "onng_search: eps must be >= 0");
    ONNG_REQUIRE(idx->adj == nullptr || idx->adj_width >= 1, ONNG_E_INVAL, "onng_search: adj_width must be >= 1");
    const bool bf16 = p->precision == ONNG_PREC_BF16;
    ONNG_REQUIRE(p->precision == ONNG_PREC_FP32 || bf16, ONNG_E_INVAL, "onng_search: unknown precision");
    int kr = p->k;
    if (bf16) {
        kr = std::max(p->k, p->k_rerank);
        ONNG_REQUIRE(kr <= kMaxK, ONNG_E_UNSUPPORTED, "onng_search: k_rerank > %d", kMaxK);
        ONNG_REQUIRE(idx->X_bf16 && aligned16(idx->X_bf16), ONNG_E_INVAL, "onng_search: bf16 needs aligned X_bf16");
    }
    if (nq == 0)
        return ONNG_OK;
    ONNG_REQUIRE(idx->row_ptr && idx->col && idx->X && Q && seeds && out_ids && out_dist, ONNG_E_INVAL,
                 "onng_search: NULL pointer");
    ONNG_REQUIRE(aligned16(idx->X) && aligned16(Q), ONNG_E_INVAL, "onng_search: X and Q must be 16-byte aligned");
    ONNG_REQUIRE(ws, ONNG_E_WORKSPACE, "onng_search: NULL workspace");

    Launch L = bf16 ? pick_v<__nv_bfloat16>(idx->d) : pick_v<float>(idx->d);
    ONNG_REQUIRE(L.fn, ONNG_E_UNSUPPORTED, "onng_search: no kernel for d=%d", idx->d);
    int per_sm = 0;
    int st = resident_blocks(L, &per_sm);
    if (st)
        return st;
    int64_t blocks = std::min<int64_t>((nq + kWarpsPerCta - 1) / kWarpsPerCta, (int64_t)per_sm * num_sms());
    // the workspace bounds the number of warps (each needs its own spill tables)
    const int64_t fit = ws_bytes > 256 ? (int64_t)((ws_bytes - 256) / (kSlotBytes * kWarpsPerCta)) : 0;
    blocks = std::min(blocks, fit);
    ONNG_REQUIRE(blocks >= 1, ONNG_E_WORKSPACE, "onng_search: workspace of %zu bytes holds no CTA (%zu needed per CTA)",
                 ws_bytes, kSlotBytes * kWarpsPerCta + 256);

    WsCarver c(ws);
    SearchArgs a;
    a.counter = c.take<int>(64);
    a.gvis = c.take<int>((size_t)blocks * kWarpsPerCta * kGlobalVisit);
    a.gpool = c.take<u64>((size_t)blocks * kWarpsPerCta * kGlobalPool);
    a.row_ptr = idx->row_ptr;
    a.col = idx->col;
    a.adj = idx->adj;
    a.adj_w = idx->adj_width;
    a.X = idx->X;
    a.Xb = idx->X_bf16;
    a.n = idx->n;
    a.d = idx->d;
    a.Q = Q;
    a.nq = nq;
    a.k = kr;
    a.k_out = p->k;
    a.e_s = p->e_s;
    a.eps = p->eps;
    a.eps_q = eps_q;
    a.es_q = es_q;
    a.seeds = seeds;
    a.n_seed = n_seed;
    a.max_exp = p->max_expansions;
    a.out_ids = out_ids;
    a.out_dist = out_dist;
    a.stats = stats;
    cudaStream_t s = to_cuda(stream);
    ONNG_CUDA_TRY(cudaMemsetAsync(a.counter, 0, sizeof(int), s), "onng_search: reset counter");
    L.fn<<<(unsigned)blocks, kWarpsPerCta * 32, L.smem, s>>>(a);
    return check_launch("onng_search");
}
