// KnnSearch (Algorithm 1) on the GPU: one warp per query.
//
// Per warp, in shared memory:
//   - the visited set C as an exact open-addressing hash (linear probing).  The
//     paper's Set/IsSet table (Sec. 2.5) keeps the first id of a bucket inline and
//     chains collisions; on the GPU a flat table probed by 32 lanes at once is
//     cheaper.  Past 3/4 load, new ids go to a per-warp table in global memory.
//   - the candidate set S as an unsorted pool popped by a warp-wide argmin.  An
//     entry beyond r(1+eps) can never be expanded (r only shrinks, and popping it
//     ends the search), so such entries may be dropped whenever room is needed.
//   - the result set R as a (distance, id)-sorted list of at most k entries.
// The up-to-e_s neighbours of the expanded node are tested and their vectors
// gathered together (coalesced 16-byte loads, several vectors in flight per
// lane, one transposed butterfly reduction for all of them).  R then takes the k
// best of R and the batch, and S takes the batch members within the new
// r(1+eps).  Applying a batch at once yields the same R, the same r after the
// batch and, since S only loses entries that can never be expanded, the same
// expansion order as the one-at-a-time loop of Algorithm 1.
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

namespace onng {
namespace {

constexpr int kWarpsPerCta = 4;
constexpr int kMaxK = 128;
constexpr int kMaxSeed = 64;
constexpr int kGlobalVisit = 32768;  // per-warp spill table entries (power of two)

struct SearchArgs {
    const int64_t *row_ptr;
    const int32_t *col;
    const float *X;
    const uint16_t *Xb;
    int64_t n;
    int d;
    const float *Q;
    int64_t nq;
    int k;        // results kept by the search (k_rerank for bf16)
    int k_out;    // results written
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
};

template <int HV, int CS> struct WarpSmem {
    int vis[HV];
    float sd[CS];
    int si[CS];
    float rd[kMaxK];
    int ri[kMaxK];
};

__host__ __device__ constexpr int log2i(int v) { return v <= 1 ? 0 : 1 + log2i(v >> 1); }

__device__ __forceinline__ unsigned lanemask_lt(int lane) { return (1u << lane) - 1u; }

__device__ __forceinline__ unsigned hash_id(int id) { return static_cast<unsigned>(id) * 0x9E3779B1u; }

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

// Sums v[g] over the warp for G values at once.  Returns, in every lane, the
// full sum of the value index holder_g(lane); see holder_lane().
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

// Lane that holds the sum of value g after transpose_reduce<G>.
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

template <int V, class T, int HV, int CS> struct Warp {
    static constexpr int G = V >= 8 ? 1 : V >= 4 ? 2 : V >= 2 ? 4 : 8;  // vectors per gather round
    WarpSmem<HV, CS> &sm;
    const SearchArgs &a;
    const void *xs;  // vectors the search reads (float32 or bfloat16)
    int lane;
    int *gvis;
    float4 qv[V];
    // per-query state (uniform across the warp)
    int ns, cnt, ndc, nexp, nvis, nvis_g, kk;
    unsigned flags;
    bool spill, rset, stop;
    float r2;
    double f2, bound2;

    __device__ Warp(WarpSmem<HV, CS> &s, const SearchArgs &args, const void *x, int ln, int *gv)
        : sm(s), a(args), xs(x), lane(ln), gvis(gv)
    {
    }

    // Visited test-and-set of one id by the calling lane; true if newly visited.
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
        unsigned hg = (hash_id(id) ^ 0x5bd1e995u) & (kGlobalVisit - 1);
        for (int t = 0; t < kGlobalVisit / 4 * 3; ++t) {
            int old = atomicCAS(&gvis[hg], -1, id);
            if (old == -1)
                return true;
            if (old == id)
                return false;
            hg = (hg + 1) & (kGlobalVisit - 1);
        }
        return true;  // unreachable while the spill table stays below 3/4 load
    }

    __device__ void begin_batch()
    {
        if (!spill && nvis >= HV / 4 * 3 - 32) {
            spill = true;
            int4 m1 = make_int4(-1, -1, -1, -1);
            int4 *g4 = reinterpret_cast<int4 *>(gvis);
            for (int i = lane; i < kGlobalVisit / 4; i += 32)
                g4[i] = m1;
            __syncwarp();
        }
    }

    // Distances of the ids held by the lanes in `mask`; returns this lane's d^2.
    __device__ float distances(int id, unsigned mask)
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
                    xv[g][v] = (src[g] >= 0 && c < chunks) ? Loader<T>::load(xs, gid[g], a.d, c)
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

    // Inserts (cd, cid) into the sorted result list, keeping at most kk entries.
    __device__ void r_insert(float cd, int cid)
    {
        int pos = 0;
#pragma unroll
        for (int s = 0; s < kMaxK / 32; ++s) {
            int i = s * 32 + lane;
            bool lt = i < cnt && pair_lt(sm.rd[i], sm.ri[i], cd, cid);
            pos += __popc(__ballot_sync(0xffffffffu, lt));
        }
        if (pos >= kk)
            return;
        int last = min(cnt, kk - 1);  // entries [pos, last) move up by one
        float td[kMaxK / 32];
        int ti[kMaxK / 32];
#pragma unroll
        for (int s = 0; s < kMaxK / 32; ++s) {
            int i = s * 32 + lane;
            if (i >= pos && i < last) {
                td[s] = sm.rd[i];
                ti[s] = sm.ri[i];
            }
        }
        __syncwarp();
#pragma unroll
        for (int s = 0; s < kMaxK / 32; ++s) {
            int i = s * 32 + lane;
            if (i >= pos && i < last) {
                sm.rd[i + 1] = td[s];
                sm.ri[i + 1] = ti[s];
            }
        }
        if (lane == 0) {
            sm.rd[pos] = cd;
            sm.ri[pos] = cid;
        }
        __syncwarp();
        cnt = min(cnt + 1, kk);
    }

    __device__ void update_bound()
    {
        bound2 = (rset && !isinf(f2)) ? (double)r2 * f2 : INFINITY;
    }

    // Drops pool entries beyond the bound (they can never be expanded).
    __device__ void pool_compact()
    {
        int w = 0;
        for (int base = 0; base < ns; base += 32) {
            int i = base + lane;
            float dv = i < ns ? sm.sd[i] : 0.f;
            int iv = i < ns ? sm.si[i] : 0;
            bool keep = i < ns && (double)dv <= bound2;
            unsigned km = __ballot_sync(0xffffffffu, keep);
            __syncwarp();
            if (keep) {
                int dst = w + __popc(km & lanemask_lt(lane));
                sm.sd[dst] = dv;
                sm.si[dst] = iv;
            }
            w += __popc(km);
            __syncwarp();
        }
        ns = w;
    }

    // Pool argmin by (d, id): returns index (or -1 when empty) and the entry.
    __device__ int pool_argmin(float &bd, int &bi)
    {
        bd = INFINITY;
        bi = INT_MAX;
        int bx = -1;
        for (int i = lane; i < ns; i += 32) {
            float dv = sm.sd[i];
            int iv = sm.si[i];
            if (bx < 0 || pair_lt(dv, iv, bd, bi)) {
                bd = dv;
                bi = iv;
                bx = i;
            }
        }
#pragma unroll
        for (int off = 16; off >= 1; off >>= 1) {
            float od = __shfl_xor_sync(0xffffffffu, bd, off);
            int oi = __shfl_xor_sync(0xffffffffu, bi, off);
            int ox = __shfl_xor_sync(0xffffffffu, bx, off);
            if (ox >= 0 && (bx < 0 || pair_lt(od, oi, bd, bi))) {
                bd = od;
                bi = oi;
                bx = ox;
            }
        }
        return bx;
    }

    // Pool argmax by (d, id) (used only when the pool is full).
    __device__ int pool_argmax(float &bd, int &bi)
    {
        bd = -1.f;
        bi = -1;
        int bx = -1;
        for (int i = lane; i < ns; i += 32) {
            float dv = sm.sd[i];
            int iv = sm.si[i];
            if (bx < 0 || pair_lt(bd, bi, dv, iv)) {
                bd = dv;
                bi = iv;
                bx = i;
            }
        }
#pragma unroll
        for (int off = 16; off >= 1; off >>= 1) {
            float od = __shfl_xor_sync(0xffffffffu, bd, off);
            int oi = __shfl_xor_sync(0xffffffffu, bi, off);
            int ox = __shfl_xor_sync(0xffffffffu, bx, off);
            if (ox >= 0 && (bx < 0 || pair_lt(bd, bi, od, oi))) {
                bd = od;
                bi = oi;
                bx = ox;
            }
        }
        return bx;
    }

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
        float d2 = distances(id, mask);
        // R <- the best kk of R and the batch
        unsigned cm = __ballot_sync(0xffffffffu, isnew && (init || !rset || d2 <= r2));
        while (cm) {
            int src = __ffs(cm) - 1;
            cm &= cm - 1;
            float cd = __shfl_sync(0xffffffffu, d2, src);
            int cid = __shfl_sync(0xffffffffu, id, src);
            if (init || !rset || cd <= r2) {
                r_insert(cd, cid);
                if (!init && cnt == kk) {
                    rset = true;
                    r2 = sm.rd[kk - 1];
                }
            }
        }
        update_bound();
        // S <- S + batch members within r(1+eps)
        bool push = isnew && (double)d2 <= bound2;
        unsigned pm = __ballot_sync(0xffffffffu, push);
        int np = __popc(pm);
        if (ns + np > CS)
            pool_compact();
        if (ns + np <= CS) {
            if (push) {
                int dst = ns + __popc(pm & lanemask_lt(lane));
                sm.sd[dst] = d2;
                sm.si[dst] = id;
            }
            ns += np;
            __syncwarp();
        } else {
            // full even after compaction: keep the nearest entries
            flags |= ONNG_FLAG_S_OVERFLOW;
            while (pm) {
                int src = __ffs(pm) - 1;
                pm &= pm - 1;
                float cd = __shfl_sync(0xffffffffu, d2, src);
                int cid = __shfl_sync(0xffffffffu, id, src);
                if (ns < CS) {
                    if (lane == 0) {
                        sm.sd[ns] = cd;
                        sm.si[ns] = cid;
                    }
                    ++ns;
                } else {
                    float md;
                    int mi;
                    int mx = pool_argmax(md, mi);
                    if (pair_lt(cd, cid, md, mi) && lane == 0) {
                        sm.sd[mx] = cd;
                        sm.si[mx] = cid;
                    }
                }
                __syncwarp();
            }
        }
        if (nvis_g >= kGlobalVisit / 2) {
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
        f2 = isinf(eps) ? INFINITY : (1.0 + (double)eps) * (1.0 + (double)eps);
        for (int i = lane; i < HV; i += 32)
            sm.vis[i] = -1;
        ns = cnt = ndc = nexp = nvis = nvis_g = 0;
        kk = a.k;
        flags = 0;
        spill = rset = stop = false;
        r2 = INFINITY;
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
        while (ns > 0 && !stop) {
            float sd;
            int s;
            int ix = pool_argmin(sd, s);
            __syncwarp();
            if (lane == 0) {
                sm.sd[ix] = sm.sd[ns - 1];
                sm.si[ix] = sm.si[ns - 1];
            }
            --ns;
            __syncwarp();
            if ((double)sd > bound2)
                break;
            if (a.max_exp > 0 && nexp >= a.max_exp) {
                flags |= ONNG_FLAG_LIMIT;
                break;
            }
            ++nexp;
            const int64_t beg = a.row_ptr[s];
            const int64_t deg = a.row_ptr[s + 1] - beg;
            const int m = deg < (int64_t)es ? (int)deg : es;
            for (int c0 = 0; c0 < m && !stop; c0 += 32) {
                int id = c0 + lane < m ? a.col[beg + c0 + lane] : -1;
                batch(id, false);
            }
        }
    }

    // Rescores the kept list in float32 against X and keeps the best k_out.
    __device__ void rerank()
    {
        const int m = cnt;
        // exact distances of the kept ids, staged in the pool arrays
        for (int c0 = 0; c0 < m; c0 += 32) {
            int i = c0 + lane;
            int id = i < m ? sm.ri[i] : -1;
            unsigned mask = __ballot_sync(0xffffffffu, id >= 0);
            float dv = exact_distances(id, mask);
            if (id >= 0) {
                sm.sd[i] = dv;
                sm.si[i] = id;
            }
        }
        __syncwarp();
        cnt = 0;
        kk = a.k_out;
        for (int i = 0; i < m; ++i)
            r_insert(sm.sd[i], sm.si[i]);
    }

    __device__ float exact_distances(int id, unsigned mask)
    {
        float mine = 0.0f;
        const int chunks = a.d >> 2;
        while (mask) {
            int src = __ffs(mask) - 1;
            mask &= mask - 1;
            int gid = __shfl_sync(0xffffffffu, id, src);
            float acc[1] = {0.0f};
#pragma unroll
            for (int v = 0; v < V; ++v) {
                int c = lane + 32 * v;
                if (c < chunks)
                    acc[0] = sqdiff4(qv[v], Loader<float>::load(a.X, gid, a.d, c), acc[0]);
            }
            float s = transpose_reduce<1>(acc, lane);
            if (lane == src)
                mine = s;
        }
        return mine;
    }

    __device__ void write(int64_t q)
    {
        const int k = a.k_out;
        for (int i = lane; i < k; i += 32) {
            a.out_ids[q * k + i] = i < cnt ? sm.ri[i] : -1;
            a.out_dist[q * k + i] = i < cnt ? sqrtf(sm.rd[i]) : INFINITY;
        }
        if (a.stats && lane == 0) {
            a.stats[q * 4 + 0] = ndc;
            a.stats[q * 4 + 1] = nexp;
            a.stats[q * 4 + 2] = nvis + nvis_g;
            a.stats[q * 4 + 3] = (int)flags;
        }
    }
};

template <int V, class T, int HV, int CS>
__global__ void __launch_bounds__(kWarpsPerCta * 32) search_kernel(SearchArgs a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    auto *smem = reinterpret_cast<WarpSmem<HV, CS> *>(smem_raw);
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int64_t slot = (int64_t)blockIdx.x * kWarpsPerCta + warp;
    const void *xs = std::is_same<T, float>::value ? static_cast<const void *>(a.X) : static_cast<const void *>(a.Xb);
    Warp<V, T, HV, CS> w(smem[warp], a, xs, lane, a.gvis + slot * kGlobalVisit);
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

struct Launch {
    void (*fn)(SearchArgs);
    size_t smem;
};

template <int V, class T, int HV, int CS> Launch pick()
{
    return {search_kernel<V, T, HV, CS>, sizeof(WarpSmem<HV, CS>) * kWarpsPerCta};
}

template <class T> Launch pick_v(int d, int k)
{
    const int V = (d + 127) / 128;
    const bool big = k > 32;
#define ONNG_PICK(v)                                                                  \
    if (V <= v)                                                                       \
        return big ? pick<v, T, 4096, 512>() : pick<v, T, 2048, 256>();
    ONNG_PICK(1)
    ONNG_PICK(2)
    ONNG_PICK(4)
    ONNG_PICK(8)
#undef ONNG_PICK
    return {nullptr, 0};
}

int grid_for(const Launch &L, int64_t nq, int *blocks_out)
{
    ONNG_CUDA_TRY(cudaFuncSetAttribute(reinterpret_cast<const void *>(L.fn),
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.smem),
                  "search: smem attribute");
    int per_sm = 0;
    ONNG_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, reinterpret_cast<const void *>(L.fn),
                                                                 kWarpsPerCta * 32, L.smem),
                  "search: occupancy");
    if (per_sm < 1)
        per_sm = 1;
    int64_t want = (nq + kWarpsPerCta - 1) / kWarpsPerCta;
    *blocks_out = (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)per_sm * num_sms()));
    return ONNG_OK;
}

int max_blocks()
{
    // upper bound on resident CTAs used to size the spill tables: smallest
    // configuration (d <= 128, k <= 32) at full occupancy
    Launch L = pick_v<float>(128, 10);
    int per_sm = 0;
    cudaFuncSetAttribute(reinterpret_cast<const void *>(L.fn), cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)L.smem);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, reinterpret_cast<const void *>(L.fn),
                                                      kWarpsPerCta * 32, L.smem) != cudaSuccess ||
        per_sm < 1)
        per_sm = 16;
    return per_sm * num_sms();
}

}  // namespace
}  // namespace onng

using namespace onng;

extern "C" size_t onng_search_workspace_bytes(int64_t nq, const onng_index *idx, const onng_search_params *p)
{
    (void)idx;
    (void)p;
    int64_t blocks = std::min<int64_t>(std::max<int64_t>(1, (nq + kWarpsPerCta - 1) / kWarpsPerCta),
                                       (int64_t)max_blocks());
    WsCarver c(nullptr);
    c.take<int>(64);
    c.take<int>((size_t)blocks * kWarpsPerCta * kGlobalVisit);
    return c.used;
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
    size_t need = onng_search_workspace_bytes(nq, idx, p);
    ONNG_REQUIRE(ws && ws_bytes >= need, ONNG_E_WORKSPACE, "onng_search: workspace %zu < %zu bytes", ws_bytes, need);

    WsCarver c(ws);
    SearchArgs a;
    a.counter = c.take<int>(64);
    a.gvis = c.take<int>(0);
    a.row_ptr = idx->row_ptr;
    a.col = idx->col;
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

    Launch L = bf16 ? pick_v<__nv_bfloat16>(idx->d, kr) : pick_v<float>(idx->d, kr);
    ONNG_REQUIRE(L.fn, ONNG_E_UNSUPPORTED, "onng_search: no kernel for d=%d", idx->d);
    int blocks = 0;
    int st = grid_for(L, nq, &blocks);
    if (st)
        return st;
    int64_t slots_avail = (int64_t)(ws_bytes - (reinterpret_cast<char *>(a.gvis) - static_cast<char *>(ws))) /
                          ((int64_t)kGlobalVisit * sizeof(int));
    blocks = (int)std::min<int64_t>(blocks, slots_avail / kWarpsPerCta);
    ONNG_REQUIRE(blocks >= 1, ONNG_E_WORKSPACE, "onng_search: workspace too small for one CTA");
    cudaStream_t s = to_cuda(stream);
    ONNG_CUDA_TRY(cudaMemsetAsync(a.counter, 0, sizeof(int), s), "onng_search: reset counter");
    L.fn<<<blocks, kWarpsPerCta * 32, L.smem, s>>>(a);
    return check_launch("onng_search");
}
