// Graph adjustment on the GPU.
//
// Static degree adjustment (Algorithm 2, set form):
//   N_e(y) = first_{e_o}(N_k(y))  united with  { o : y in first_{e_i}(N_k(o)) }.
// The reversed edge y->o carries the length stored for o->y; it is skipped when
// y->o is already one of y's forward edges (the forward length wins).  The
// count pass computes every row's exact size (forward edges plus non-duplicate
// reversed edges), a device scan turns the sizes into row_ptr, the fill pass
// writes (length, id) keys, and each row is sorted by (length, id): a warp
// register bitonic sort for rows up to 512 edges, an in-place CTA sort for
// longer rows (hubs).
//
// Degree adjustment with constraints (Algorithm 3, "SAC"): its greedy pass reads
// in a closed form.  N(G_t, o) = { n : o in first_{e_i}(N_k(n)) } (Algorithm 2
// with (0, e_i)), so a node n is considered only by the nodes of its own first
// e_i kNN entries, at most e_i of them: the in-degree test |N(G_i, n)| < e_i
// always holds when n is met.  Taking the nodes o in increasing
// (|N(G_t, o)|, o) and each list in increasing (length, id), o therefore adds
// its first e_o members unconditionally and a later member n exactly when no
// earlier node has added n, i.e. when o is the first of n's considerers in that
// order (that one always adds n).  Both rules are per-edge, so the pass runs in
// parallel and equals the sequential one edge for edge.  The last loop then
// gives every node with fewer than e_o edges its nearest kNN neighbours not yet
// in its list.
//
// Algorithm 4 taken literally (rounds over the partial output; a variant beside
// the order-free rule below): in round p every node s with more than p input
// edges decides its p-th edge (s, t) (input rows are in (length, id) order), in
// ascending s, and keeps it unless HasPath (Algorithm 5) finds, in the partial
// output G_p, a kept edge (s, m) and a kept edge (m, t) shorter than (s, t).
// (s, m) was decided in an earlier round; (m, t) sits at m's position r of t:
// decided when r < p, or earlier in this round when r = p and m < s.  A round
// first decides every edge whose answer needs no same-round edge, then repeats
// a resolution pass: an edge waiting on same-round edges of smaller nodes is
// removed once one of them is kept and kept once all are removed; the smallest
// waiting node can always be decided, so each pass makes progress.  Positions
// of t in m's row come from a per-row copy sorted by id (binary search).
//
// Path adjustment (Algorithms 4/5, order-free reading): edge (i, j) is dropped
// if the input graph holds i->m and m->j with len(i,m) < len(i,j) and
// len(m,j) < len(i,j).  A warp owns a node i at a time (persistent warps stride
// over the nodes): N(i) goes into a shared-memory hash (id -> position); for
// every m in N(i) shorter than i's longest edge, the prefix of m's list shorter
// than that edge (a binary search: rows are sorted by length) is streamed with
// the others as one flattened sequence across the lanes, and every hit j that
// satisfies both strict comparisons records the smallest witness position.
// Nodes with more than 256 edges use a CTA and a hash in global scratch.  A
// count / scan / compact sequence then writes the kept edges in their input
// order.
#include <algorithm>
#include <cmath>
#include <vector>

#include "common.cuh"
#include "scan.cuh"
#include "warp_sort.cuh"

namespace onng {
namespace {

constexpr unsigned long long EMPTY_KEY = 0x7F800000FFFFFFFFull;

__device__ __forceinline__ bool in_first(const int32_t *__restrict__ nbr, int64_t row, int k, int f, int32_t id)
{
    const int32_t *p = nbr + row * k;
    for (int t = 0; t < f; ++t)
        if (p[t] == id)
            return true;
    return false;
}

__device__ __forceinline__ int valid_prefix(const int32_t *__restrict__ nbr, int64_t row, int k, int f)
{
    int c = 0;
    for (int t = 0; t < f; ++t)
        c += nbr[row * k + t] >= 0;
    return c;
}

// deg[y] = valid forward edges of y; incnt[y] += non-duplicate reversed edges.
__global__ void degree_count_kernel(const int32_t *__restrict__ nbr, int64_t n, int k, int fo, int fi,
                                    int64_t *__restrict__ deg, int *__restrict__ incnt)
{
    for (int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; o < n; o += (int64_t)gridDim.x * blockDim.x) {
        for (int p = 0; p < fi; ++p) {
            const int32_t y = nbr[o * k + p];
            if (y < 0 || y >= n)
                continue;
            if (!in_first(nbr, y, k, fo, (int32_t)o))
                atomicAdd(&incnt[y], 1);
        }
    }
}

__global__ void degree_total_kernel(const int32_t *__restrict__ nbr, int64_t n, int k, int fo,
                                    const int *__restrict__ incnt, int64_t *__restrict__ deg)
{
    for (int64_t y = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; y < n; y += (int64_t)gridDim.x * blockDim.x)
        deg[y] = valid_prefix(nbr, y, k, fo) + incnt[y];
}

__global__ void degree_fill_kernel(const int32_t *__restrict__ nbr, const float *__restrict__ len, int64_t n, int k,
                                   int fo, int fi, const int64_t *__restrict__ row_ptr, int *__restrict__ cursor,
                                   unsigned long long *__restrict__ keys)
{
    for (int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; o < n; o += (int64_t)gridDim.x * blockDim.x) {
        // forward edges of o occupy the head of its row
        int w = 0;
        for (int p = 0; p < fo; ++p) {
            const int32_t x = nbr[o * k + p];
            if (x >= 0)
                keys[row_ptr[o] + w++] = pack_key(len[o * k + p], x);
        }
        // reversed edges y->o go after y's forward edges
        for (int p = 0; p < fi; ++p) {
            const int32_t y = nbr[o * k + p];
            if (y < 0 || y >= n)
                continue;
            if (in_first(nbr, y, k, fo, (int32_t)o))
                continue;
            const int pos = atomicAdd(&cursor[y], 1);
            keys[row_ptr[y] + valid_prefix(nbr, y, k, fo) + pos] = pack_key(len[o * k + p], (int32_t)o);
        }
    }
}

// Sorts rows of up to 512 keys, one warp per row; longer rows are listed for the CTA sort.
__global__ void sort_small_rows(const int64_t *__restrict__ row_ptr, int64_t n, unsigned long long *__restrict__ keys,
                                int64_t *__restrict__ big_rows, int *__restrict__ n_big)
{
    const int lane = threadIdx.x & 31;
    const int64_t row = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (row >= n)
        return;
    const int64_t beg = row_ptr[row], m = row_ptr[row + 1] - beg;
    if (m <= 1)
        return;
    if (m > 512) {
        if (lane == 0)
            big_rows[atomicAdd(n_big, 1)] = row;
        return;
    }
    unsigned long long v[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        const int e = i * 32 + lane;
        v[i] = e < m ? keys[beg + e] : EMPTY_KEY;
    }
    warp_bitonic_sort<16>(v, lane);
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        const int e = i * 32 + lane;
        if (e < m)
            keys[beg + e] = v[i];
    }
}

// In-place ascending sort of a[0..m) by one CTA: bitonic network in the form
// whose comparators all point upward (first stage of each merge compares
// mirrored positions), so positions >= m act as +inf and are never touched.
__device__ void cta_sort(unsigned long long *a, int64_t m)
{
    int64_t P = 1;
    while (P < m)
        P <<= 1;
    for (int64_t size = 2; size <= P; size <<= 1) {
        for (int64_t t = threadIdx.x; t < P / 2; t += blockDim.x) {
            const int64_t blk = t / (size / 2), off = t % (size / 2);
            const int64_t i = blk * size + off, j = blk * size + size - 1 - off;
            if (j < m && a[j] < a[i]) {
                unsigned long long x = a[i];
                a[i] = a[j];
                a[j] = x;
            }
        }
        __syncthreads();
        for (int64_t h = size / 4; h >= 1; h >>= 1) {
            for (int64_t t = threadIdx.x; t < P / 2; t += blockDim.x) {
                const int64_t blk = t / h, off = t % h;
                const int64_t i = blk * 2 * h + off, j = i + h;
                if (j < m && a[j] < a[i]) {
                    unsigned long long x = a[i];
                    a[i] = a[j];
                    a[j] = x;
                }
            }
            __syncthreads();
        }
    }
}

__global__ void sort_big_rows(const int64_t *__restrict__ row_ptr, unsigned long long *__restrict__ keys,
                              const int64_t *__restrict__ big_rows, const int *__restrict__ n_big)
{
    for (int b = blockIdx.x; b < *n_big; b += gridDim.x) {
        const int64_t row = big_rows[b];
        cta_sort(keys + row_ptr[row], row_ptr[row + 1] - row_ptr[row]);
        __syncthreads();
    }
}

__global__ void unpack_keys(const unsigned long long *__restrict__ keys, const int64_t *__restrict__ nnz,
                            int32_t *__restrict__ col, float *__restrict__ len)
{
    const int64_t m = *nnz;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long k = keys[e];
        col[e] = (int32_t)(unsigned)(k & 0xFFFFFFFFull);
        len[e] = __uint_as_float((unsigned)(k >> 32));
    }
}

// ------------------------------------------------------------------ path

constexpr int kPathSmall = 256;       // rows up to this many edges: one warp, shared-memory hash
constexpr int kPathHash = 512;        // hash slots for small rows
constexpr int kPathWarps = 4;
constexpr int kPathUnroll = 4;  // list entries per lane in flight

struct PathSmem {
    int hkey[kPathHash];
    int hpos[kPathHash];
    float li[kPathSmall];
    int wit[kPathSmall];
    int64_t pre[32];
    int64_t mb[32];
    int mu[32];
};

__device__ __forceinline__ unsigned phash(int id) { return static_cast<unsigned>(id) * 0x9E3779B1u; }

// Looks id up in an open-addressing table of `cap` slots; returns its position or -1.
__device__ __forceinline__ int hash_find(const int *hkey, const int *hpos, int cap, int lg, int id)
{
    unsigned h = phash(id) >> (32 - lg);
    for (int t = 0; t < cap; ++t) {
        const int k = hkey[h];
        if (k == id)
            return hpos[h];
        if (k == -1)
            return -1;
        h = (h + 1) & (cap - 1);
    }
    return -1;
}

__device__ __forceinline__ void hash_put(int *hkey, int *hpos, int cap, int lg, int id, int pos)
{
    unsigned h = phash(id) >> (32 - lg);
    for (int t = 0; t < cap; ++t) {
        const int old = atomicCAS(&hkey[h], -1, id);
        if (old == -1 || old == id) {
            hpos[h] = pos;
            return;
        }
        h = (h + 1) & (cap - 1);
    }
}

// Marks removals of the edges of node i (deg <= kPathSmall) by one warp.
__device__ void path_row_warp(int64_t i, const int64_t *__restrict__ rp, const int32_t *__restrict__ col,
                              const float *__restrict__ len, PathSmem &sm, int *__restrict__ wit_out, int lane)
{
    const int64_t beg = rp[i];
    const int deg = (int)(rp[i + 1] - beg);
    constexpr int lg = 9;  // log2(kPathHash)
    for (int t = lane; t < kPathHash; t += 32)
        sm.hkey[t] = -1;
    __syncwarp();
    for (int t = lane; t < deg; t += 32) {
        const int j = col[beg + t];
        sm.li[t] = len[beg + t];
        sm.wit[t] = INT_MAX;
        hash_put(sm.hkey, sm.hpos, kPathHash, lg, j, t);
    }
    __syncwarp();
    float lmax = 0.f;
    for (int t = lane; t < deg; t += 32)
        lmax = fmaxf(lmax, sm.li[t]);
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1)
        lmax = fmaxf(lmax, __shfl_xor_sync(0xffffffffu, lmax, off));
    for (int u0 = 0; u0 < deg; u0 += 32) {
        const int u = u0 + lane;
        int64_t cnt = 0, mb = 0;
        if (u < deg && sm.li[u] < lmax) {
            // only the prefix of m's list shorter than lmax can witness (rows are
            // sorted by length): its size by binary search
            const int m = col[beg + u];
            mb = rp[m];
            int64_t lo = 0, hi = rp[m + 1] - mb;
            while (lo < hi) {
                const int64_t mid = (lo + hi) >> 1;
                if (len[mb + mid] < lmax)
                    lo = mid + 1;
                else
                    hi = mid;
            }
            cnt = lo;
        }
        int64_t x = cnt;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int64_t y = __shfl_up_sync(0xffffffffu, x, off);
            if (lane >= off)
                x += y;
        }
        sm.pre[lane] = x;  // inclusive prefix
        sm.mb[lane] = mb;
        sm.mu[lane] = u;
        __syncwarp();
        const int64_t total = sm.pre[31];
        // kPathUnroll entries per lane and round: their list loads are all issued
        // before any is used, so several gathers are in flight per lane
        for (int64_t e0 = lane; e0 < total; e0 += 32 * kPathUnroll) {
            int own[kPathUnroll];
            int64_t idx[kPathUnroll];
#pragma unroll
            for (int r = 0; r < kPathUnroll; ++r) {
                const int64_t e = e0 + 32 * r;
                int lo = 0, hi = 31;  // first lane whose inclusive prefix exceeds e
                while (lo < hi) {
                    const int mid = (lo + hi) >> 1;
                    if (sm.pre[mid] > e)
                        hi = mid;
                    else
                        lo = mid + 1;
                }
                own[r] = e < total ? lo : -1;
                const int64_t start = sm.pre[lo] - (lo ? sm.pre[lo - 1] : 0);
                idx[r] = sm.mb[lo] + (e - (sm.pre[lo] - start));
            }
            float lmj[kPathUnroll];
            int cj[kPathUnroll];
#pragma unroll
            for (int r = 0; r < kPathUnroll; ++r) {
                lmj[r] = own[r] >= 0 ? len[idx[r]] : INFINITY;
                cj[r] = own[r] >= 0 ? col[idx[r]] : -1;
            }
#pragma unroll
            for (int r = 0; r < kPathUnroll; ++r) {
                if (own[r] < 0 || !(lmj[r] < lmax))
                    continue;
                const int t = hash_find(sm.hkey, sm.hpos, kPathHash, lg, cj[r]);
                if (t < 0)
                    continue;
                const int uu = sm.mu[own[r]];
                const float lij = sm.li[t];
                if (sm.li[uu] < lij && lmj[r] < lij)
                    atomicMin(&sm.wit[t], uu);
            }
        }
        __syncwarp();
    }
    for (int t = lane; t < deg; t += 32)
        wit_out[beg + t] = sm.wit[t] == INT_MAX ? -1 : sm.wit[t];
    __syncwarp();
}

// Warps stride over the rows (the grid is what stays resident), so a warp whose
// row ends early takes the next one instead of idling until the slowest row of
// its CTA is done.
__global__ void __launch_bounds__(kPathWarps * 32)
    path_small_kernel(const int64_t *__restrict__ rp, const int32_t *__restrict__ col, const float *__restrict__ len,
                      int64_t n, int *__restrict__ wit, int64_t *__restrict__ big_rows, int *__restrict__ n_big)
{
    __shared__ PathSmem sm[kPathWarps];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * kPathWarps;
    for (int64_t i = (int64_t)blockIdx.x * kPathWarps + warp; i < n; i += stride) {
        const int64_t deg = rp[i + 1] - rp[i];
        if (deg > kPathSmall) {
            if (lane == 0)
                big_rows[atomicAdd(n_big, 1)] = i;
            continue;
        }
        if (deg >= 2)
            path_row_warp(i, rp, col, len, sm[warp], wit, lane);
        else if (deg == 1 && lane == 0)
            wit[rp[i]] = -1;
    }
}

// Open-addressing table of any size `cap` (range reduction by multiply-high).
__device__ __forceinline__ int ghash_find(const int *hkey, const int *hpos, int cap, int id)
{
    unsigned h = __umulhi(phash(id), (unsigned)cap);
    for (int t = 0; t < cap; ++t) {
        const int k = hkey[h];
        if (k == id)
            return hpos[h];
        if (k == -1)
            return -1;
        h = h + 1 == (unsigned)cap ? 0 : h + 1;
    }
    return -1;
}

__device__ __forceinline__ void ghash_put(int *hkey, int *hpos, int cap, int id, int pos)
{
    unsigned h = __umulhi(phash(id), (unsigned)cap);
    for (int t = 0; t < cap; ++t) {
        const int old = atomicCAS(&hkey[h], -1, id);
        if (old == -1 || old == id) {
            hpos[h] = pos;
            return;
        }
        h = h + 1 == (unsigned)cap ? 0 : h + 1;
    }
}

// Rows with more than kPathSmall edges: one CTA per row; the row's hash lives in
// global scratch at offset 2 * row_ptr[i] (2 * degree slots, so rows never overlap).
__global__ void path_big_kernel(const int64_t *__restrict__ rp, const int32_t *__restrict__ col,
                                const float *__restrict__ len, int *__restrict__ wit,
                                const int64_t *__restrict__ big_rows, const int *__restrict__ n_big,
                                int *__restrict__ skey, int *__restrict__ spos)
{
    __shared__ float s_lmax;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int b = blockIdx.x; b < *n_big; b += gridDim.x) {
        const int64_t i = big_rows[b];
        const int64_t beg = rp[i];
        const int deg = (int)(rp[i + 1] - beg);
        const int cap = 2 * deg;
        int *hkey = skey + 2 * beg;
        int *hpos = spos + 2 * beg;
        for (int t = threadIdx.x; t < cap; t += blockDim.x)
            hkey[t] = -1;
        if (threadIdx.x == 0)
            s_lmax = 0.f;
        __syncthreads();
        for (int t = threadIdx.x; t < deg; t += blockDim.x) {
            wit[beg + t] = INT_MAX;
            ghash_put(hkey, hpos, cap, col[beg + t], t);
        }
        if (threadIdx.x == 0)
            s_lmax = len[beg + deg - 1];  // rows are sorted by length
        __syncthreads();
        const float lmax = s_lmax;
        for (int u = warp; u < deg; u += nw) {
            const float liu = len[beg + u];
            if (!(liu < lmax))
                continue;
            const int m = col[beg + u];
            const int64_t mb = rp[m];
            // the prefix of m's list shorter than lmax (rows are sorted by length)
            int64_t lo = 0, hi = rp[m + 1] - mb;
            while (lo < hi) {
                const int64_t mid = (lo + hi) >> 1;
                if (len[mb + mid] < lmax)
                    lo = mid + 1;
                else
                    hi = mid;
            }
            const int64_t me = mb + lo;
            // kPathUnroll entries per lane in flight
            for (int64_t i0 = mb + lane; i0 < me; i0 += 32 * kPathUnroll) {
                float lmj[kPathUnroll];
                int cj[kPathUnroll];
#pragma unroll
                for (int r = 0; r < kPathUnroll; ++r) {
                    const int64_t idx = i0 + 32 * r;
                    lmj[r] = idx < me ? len[idx] : INFINITY;
                    cj[r] = idx < me ? col[idx] : -1;
                }
#pragma unroll
                for (int r = 0; r < kPathUnroll; ++r) {
                    if (cj[r] < 0)
                        continue;
                    const int t = ghash_find(hkey, hpos, cap, cj[r]);
                    if (t < 0)
                        continue;
                    const float lij = len[beg + t];
                    if (liu < lij && lmj[r] < lij)
                        atomicMin(&wit[beg + t], u);
                }
            }
        }
        __syncthreads();
        for (int t = threadIdx.x; t < deg; t += blockDim.x)
            if (wit[beg + t] == INT_MAX)
                wit[beg + t] = -1;
        __syncthreads();
    }
}

__global__ void path_count_kernel(const int64_t *__restrict__ rp, int64_t n, const int *__restrict__ wit,
                                  int64_t *__restrict__ kept)
{
    const int lane = threadIdx.x & 31;
    const int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (i >= n)
        return;
    int64_t c = 0;
    for (int64_t e = rp[i] + lane; e < rp[i + 1]; e += 32)
        c += wit[e] < 0;
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1)
        c += __shfl_xor_sync(0xffffffffu, c, off);
    if (lane == 0)
        kept[i] = c;
}

__global__ void path_compact_kernel(const int64_t *__restrict__ rp, const int32_t *__restrict__ col,
                                    const float *__restrict__ len, int64_t n, const int *__restrict__ wit,
                                    const int64_t *__restrict__ rp_out, int32_t *__restrict__ col_out,
                                    float *__restrict__ len_out, int32_t *__restrict__ removed_by)
{
    const int lane = threadIdx.x & 31;
    const int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (i >= n)
        return;
    const int64_t beg = rp[i], end = rp[i + 1];
    int64_t w = rp_out[i];
    for (int64_t e0 = beg; e0 < end; e0 += 32) {
        const int64_t e = e0 + lane;
        const bool keep = e < end && wit[e] < 0;
        const unsigned km = __ballot_sync(0xffffffffu, keep);
        if (keep) {
            const int64_t dst = w + __popc(km & ((1u << lane) - 1u));
            col_out[dst] = col[e];
            len_out[dst] = len[e];
        }
        if (removed_by && e < end)
            removed_by[e] = wit[e] < 0 ? -1 : col[beg + wit[e]];
        w += __popc(km);
    }
}

// ------------------------------------------------------------------ Algorithm 4, literal

// byid[e] = (id << 32 | position) of every edge, per row; sorted per row afterwards
__global__ void alg4_byid_kernel(const int64_t *__restrict__ rp, const int32_t *__restrict__ col, int64_t n,
                                 unsigned long long *__restrict__ byid)
{
    const int lane = threadIdx.x & 31;
    const int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (i >= n)
        return;
    for (int64_t e = rp[i] + lane; e < rp[i + 1]; e += 32)
        byid[e] = ((unsigned long long)(unsigned)col[e] << 32) | (unsigned)(e - rp[i]);
}

// position of t in row m (its id-sorted copy), or -1
__device__ __forceinline__ int alg4_find(const int64_t *__restrict__ rp, const unsigned long long *__restrict__ byid,
                                         int32_t m, int32_t t)
{
    int64_t lo = rp[m], hi = rp[m + 1];
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        const int32_t id = (int32_t)(byid[mid] >> 32);
        if (id < t)
            lo = mid + 1;
        else
            hi = mid;
    }
    if (lo < rp[m + 1] && (int32_t)(byid[lo] >> 32) == t)
        return (int)(unsigned)(byid[lo] & 0xFFFFFFFFull);
    return -1;
}

// Edge states: 0 undecided, 1 kept, 2 removed.
// One warp per node s = order[w] (nodes by degree, descending: the nodes with
// more than p edges are a prefix).  Decides s's p-th edge if it can; counts the
// edges still waiting in *waiting.
__global__ void alg4_round_kernel(const int64_t *__restrict__ rp, const int32_t *__restrict__ col,
                                  const float *__restrict__ len, const unsigned long long *__restrict__ byid,
                                  const int32_t *__restrict__ order, int64_t active, int p,
                                  unsigned char *__restrict__ state, int *__restrict__ waiting)
{
    const int lane = threadIdx.x & 31;
    const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (w >= active)
        return;
    const int32_t s = order[w];
    const int64_t beg = rp[s];
    if (state[beg + p] != 0)
        return;
    const int32_t t = col[beg + p];
    const float lst = len[beg + p];
    bool path = false, wait = false;
    for (int q0 = 0; q0 < p; q0 += 32) {
        const int q = q0 + lane;
        if (q < p && state[beg + q] == 1) {
            const int32_t m = col[beg + q];
            const int r = alg4_find(rp, byid, m, t);
            if (r >= 0 && len[rp[m] + r] < lst) {
                if (r < p) {
                    path |= state[rp[m] + r] == 1;
                } else if (r == p && m < s) {
                    const unsigned char sm = state[rp[m] + r];
                    path |= sm == 1;
                    wait |= sm == 0;
                }
            }
        }
    }
    path = __any_sync(0xffffffffu, path);
    wait = __any_sync(0xffffffffu, wait);
    if (lane == 0) {
        if (path)
            state[beg + p] = 2;
        else if (!wait)
            state[beg + p] = 1;
        else
            atomicAdd(waiting, 1);
    }
}

__global__ void alg4_hist_kernel(const int64_t *__restrict__ rp, int64_t n, int *__restrict__ hist)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(&hist[rp[i + 1] - rp[i]], 1);
}

// order[] = nodes grouped by degree, largest first (offset[d] = nodes of degree > d)
__global__ void alg4_order_kernel(const int64_t *__restrict__ rp, int64_t n, const int64_t *__restrict__ offset,
                                  int *__restrict__ cursor, int32_t *__restrict__ order)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t d = rp[i + 1] - rp[i];
        order[offset[d] + atomicAdd(&cursor[d], 1)] = (int32_t)i;
    }
}

__global__ void alg4_wit_kernel(const unsigned char *__restrict__ state, int64_t nnz, int *__restrict__ wit)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x)
        wit[e] = state[e] == 2 ? 0 : -1;
}

// ------------------------------------------------------------------ SAC

// first[n] = the first node, in the order (|N(G_t, o)|, o), among the valid ids
// of first_{fi}(N_k(n)) (-1 if none): the node of Algorithm 3 that meets n first.
__global__ void sac_first_kernel(const int32_t *__restrict__ nbr, int64_t n, int k, int fi,
                                 const int64_t *__restrict__ gt_ptr, int32_t *__restrict__ first)
{
    for (int64_t y = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; y < n; y += (int64_t)gridDim.x * blockDim.x) {
        int64_t best_deg = INT64_MAX;
        int32_t best = -1;
        for (int p = 0; p < fi; ++p) {
            const int32_t o = nbr[y * k + p];
            if (o < 0 || o >= n)
                continue;
            const int64_t dg = gt_ptr[o + 1] - gt_ptr[o];
            if (dg < best_deg || (dg == best_deg && o < best)) {
                best_deg = dg;
                best = o;
            }
        }
        first[y] = best;
    }
}

// One warp per node o.  Row = the members of N(G_t, o) (keys sorted by (length,
// id)) at positions < e_o or first-met at o, then, if fewer than e_o, o's kNN
// neighbours in order that are not in N(G_t, o), up to e_o in all.  Count mode
// (keys == NULL) writes the row sizes; fill mode writes the keys at row_ptr[o].
__global__ void sac_row_kernel(const int32_t *__restrict__ nbr, const float *__restrict__ len, int64_t n, int k,
                               int e_o, const int64_t *__restrict__ gt_ptr,
                               const unsigned long long *__restrict__ gt_keys, const int32_t *__restrict__ first,
                               int64_t *__restrict__ cnt, const int64_t *__restrict__ row_ptr,
                               unsigned long long *__restrict__ keys)
{
    const int lane = threadIdx.x & 31;
    const int64_t o = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (o >= n)
        return;
    const int64_t beg = gt_ptr[o];
    const int64_t m = gt_ptr[o + 1] - beg;
    const int64_t out = keys ? row_ptr[o] : 0;
    int64_t w = 0;
    for (int64_t c0 = 0; c0 < m; c0 += 32) {
        const int64_t p = c0 + lane;
        unsigned long long key = 0;
        bool take = false;
        if (p < m) {
            key = gt_keys[beg + p];
            take = p < e_o || first[(int32_t)(unsigned)(key & 0xFFFFFFFFull)] == (int32_t)o;
        }
        const unsigned tm = __ballot_sync(0xffffffffu, take);
        if (keys && take)
            keys[out + w + __popc(tm & ((1u << lane) - 1u))] = key;
        w += __popc(tm);
    }
    if (m < e_o) {
        // every member was taken; the nearest kNN neighbours not among them follow
        for (int p0 = 0; p0 < k && w < e_o; p0 += 32) {
            const int p = p0 + lane;
            const int32_t x = p < k ? nbr[o * k + p] : -1;
            bool cand = x >= 0 && x < n;
            for (int64_t t = 0; cand && t < m; ++t)
                cand = (int32_t)(unsigned)(gt_keys[beg + t] & 0xFFFFFFFFull) != x;
            const unsigned cm = __ballot_sync(0xffffffffu, cand);
            const int rank = __popc(cm & ((1u << lane) - 1u));
            if (keys && cand && w + rank < e_o)
                keys[out + w + rank] = pack_key(len[o * k + p], x);
            w = min((int64_t)e_o, w + __popc(cm));
            // kNN rows are padded with -1 at their end: the list stops there
            if (__ballot_sync(0xffffffffu, p < k && x < 0))
                break;
        }
    }
    if (!keys && lane == 0)
        cnt[o] = w;
}

int grid1d(int64_t work, int threads)
{
    return (int)std::max<int64_t>(1, std::min<int64_t>((work + threads - 1) / threads, (int64_t)num_sms() * 16));
}

}  // namespace
}  // namespace onng

using namespace onng;

// ------------------------------------------------------------------ degree ABI

extern "C" size_t onng_adjust_degree_workspace_bytes(int64_t n, int32_t k)
{
    WsCarver c(nullptr);
    c.take<int>((size_t)std::max<int64_t>(n, 1));  // in-counts / cursors
    c.take<int64_t>((size_t)std::max<int64_t>(n, 1));  // row sizes
    c.take<int64_t>((size_t)std::max<int64_t>(n, 1));  // long rows
    c.take<int>(64);
    c.take<char>(scan_workspace_bytes(std::max<int64_t>(n, 1)));
    c.take<unsigned long long>((size_t)std::max<int64_t>(n, 1) * (size_t)std::max(k, 1) * 2);  // keys
    return c.used;
}

static int degree_args(const int32_t *nbr, const float *len, int64_t n, int32_t k, int32_t e_o, int32_t e_i,
                       void *ws, size_t ws_bytes, const char *who)
{
    ONNG_REQUIRE(n >= 0 && n <= INT32_MAX && k >= 1 && e_o >= 0 && e_i >= 0, ONNG_E_INVAL, "%s: bad sizes", who);
    ONNG_REQUIRE(n == 0 || (nbr && len), ONNG_E_INVAL, "%s: NULL input", who);
    const size_t need = onng_adjust_degree_workspace_bytes(n, k);
    ONNG_REQUIRE(ws && ws_bytes >= need, ONNG_E_WORKSPACE, "%s: workspace %zu < %zu bytes", who, ws_bytes, need);
    return ONNG_OK;
}

extern "C" int onng_adjust_degree_count(const int32_t *nbr, const float *len, int64_t n, int32_t k, int32_t e_o,
                                        int32_t e_i, int64_t *row_ptr, int64_t *nnz_host, void *ws, size_t ws_bytes,
                                        onng_stream_t stream)
{
    ONNG_RANGE("onng_adjust_degree_count");
    int st = degree_args(nbr, len, n, k, e_o, e_i, ws, ws_bytes, "onng_adjust_degree_count");
    if (st)
        return st;
    ONNG_REQUIRE(row_ptr, ONNG_E_INVAL, "onng_adjust_degree_count: NULL row_ptr");
    cudaStream_t s = to_cuda(stream);
    const int fo = std::min(e_o, k), fi = std::min(e_i, k);
    WsCarver c(ws);
    int *incnt = c.take<int>((size_t)std::max<int64_t>(n, 1));
    int64_t *deg = c.take<int64_t>((size_t)std::max<int64_t>(n, 1));
    c.take<int64_t>((size_t)std::max<int64_t>(n, 1));
    c.take<int>(64);
    char *scan_ws = c.take<char>(scan_workspace_bytes(std::max<int64_t>(n, 1)));
    if (n > 0) {
        ONNG_CUDA_TRY(cudaMemsetAsync(incnt, 0, sizeof(int) * n, s), "adjust_degree: clear");
        degree_count_kernel<<<grid1d(n, 256), 256, 0, s>>>(nbr, n, k, fo, fi, deg, incnt);
        degree_total_kernel<<<grid1d(n, 256), 256, 0, s>>>(nbr, n, k, fo, incnt, deg);
        st = check_launch("onng_adjust_degree_count");
        if (st)
            return st;
    }
    st = exclusive_scan(deg, row_ptr, n, scan_ws, scan_workspace_bytes(std::max<int64_t>(n, 1)), s);
    if (st)
        return st;
    if (nnz_host) {
        ONNG_CUDA_TRY(cudaMemcpyAsync(nnz_host, row_ptr + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s),
                      "adjust_degree: nnz");
        ONNG_CUDA_TRY(cudaStreamSynchronize(s), "adjust_degree: sync");
    }
    return ONNG_OK;
}

extern "C" int onng_adjust_degree(const int32_t *nbr, const float *len, int64_t n, int32_t k, int32_t e_o, int32_t e_i,
                                  const int64_t *row_ptr, int32_t *col, float *len_out, void *ws, size_t ws_bytes,
                                  onng_stream_t stream)
{
    ONNG_RANGE("onng_adjust_degree");
    int st = degree_args(nbr, len, n, k, e_o, e_i, ws, ws_bytes, "onng_adjust_degree");
    if (st)
        return st;
    if (n == 0)
        return ONNG_OK;
    ONNG_REQUIRE(row_ptr && col && len_out, ONNG_E_INVAL, "onng_adjust_degree: NULL output");
    cudaStream_t s = to_cuda(stream);
    const int fo = std::min(e_o, k), fi = std::min(e_i, k);
    WsCarver c(ws);
    int *cursor = c.take<int>((size_t)n);
    c.take<int64_t>((size_t)n);
    int64_t *big = c.take<int64_t>((size_t)n);
    int *n_big = c.take<int>(64);
    c.take<char>(scan_workspace_bytes(n));
    unsigned long long *keys = c.take<unsigned long long>((size_t)n * k * 2);
    ONNG_CUDA_TRY(cudaMemsetAsync(cursor, 0, sizeof(int) * n, s), "adjust_degree: clear");
    ONNG_CUDA_TRY(cudaMemsetAsync(n_big, 0, sizeof(int), s), "adjust_degree: clear");
    degree_fill_kernel<<<grid1d(n, 256), 256, 0, s>>>(nbr, len, n, k, fo, fi, row_ptr, cursor, keys);
    sort_small_rows<<<(unsigned)((n * 32 + 255) / 256), 256, 0, s>>>(row_ptr, n, keys, big, n_big);
    sort_big_rows<<<num_sms() * 2, 1024, 0, s>>>(row_ptr, keys, big, n_big);
    st = check_launch("onng_adjust_degree: fill/sort");
    if (st)
        return st;
    // the edge count row_ptr[n] is read on the device: no host round trip
    unpack_keys<<<grid1d(n * (int64_t)(fo + fi), 256), 256, 0, s>>>(keys, row_ptr + n, col, len_out);
    return check_launch("onng_adjust_degree: unpack");
}

// ------------------------------------------------------------------ SAC ABI

namespace onng {
namespace {

struct SacWs {
    int *incnt;
    int64_t *cnt, *big, *gt_ptr;
    int *n_big;
    char *scan_ws;
    size_t scan_bytes;
    unsigned long long *gt_keys, *keys;
    int32_t *first;
    size_t used;
};

SacWs sac_carve(void *ws, int64_t n, int k)
{
    const int64_t nn = std::max<int64_t>(n, 1);
    WsCarver c(ws);
    SacWs w;
    w.incnt = c.take<int>((size_t)nn);
    w.cnt = c.take<int64_t>((size_t)nn);
    w.big = c.take<int64_t>((size_t)nn);
    w.n_big = c.take<int>(64);
    w.scan_bytes = scan_workspace_bytes(nn + 1);
    w.scan_ws = c.take<char>(w.scan_bytes);
    w.gt_ptr = c.take<int64_t>((size_t)nn + 1);
    w.gt_keys = c.take<unsigned long long>((size_t)nn * std::max(k, 1));
    w.first = c.take<int32_t>((size_t)nn);
    w.keys = c.take<unsigned long long>((size_t)nn * std::max(k, 1) * 2);  // rows hold <= n k + n k edges
    w.used = c.used;
    return w;
}

// G_t of Algorithm 3 (Algorithm 2 with (0, e_i)) as sorted (length, id) keys,
// then every node's first considerer.
int sac_prepare(const int32_t *nbr, const float *len, int64_t n, int k, int fi, const SacWs &w, cudaStream_t s)
{
    ONNG_CUDA_TRY(cudaMemsetAsync(w.incnt, 0, sizeof(int) * n, s), "adjust_degree_sac: clear");
    ONNG_CUDA_TRY(cudaMemsetAsync(w.n_big, 0, sizeof(int), s), "adjust_degree_sac: clear");
    degree_count_kernel<<<grid1d(n, 256), 256, 0, s>>>(nbr, n, k, 0, fi, w.cnt, w.incnt);
    degree_total_kernel<<<grid1d(n, 256), 256, 0, s>>>(nbr, n, k, 0, w.incnt, w.cnt);
    int st = check_launch("onng_adjust_degree_sac: G_t count");
    if (st)
        return st;
    st = exclusive_scan(w.cnt, w.gt_ptr, n, w.scan_ws, w.scan_bytes, s);
    if (st)
        return st;
    ONNG_CUDA_TRY(cudaMemsetAsync(w.incnt, 0, sizeof(int) * n, s), "adjust_degree_sac: clear");
    degree_fill_kernel<<<grid1d(n, 256), 256, 0, s>>>(nbr, len, n, k, 0, fi, w.gt_ptr, w.incnt, w.gt_keys);
    sort_small_rows<<<(unsigned)((n * 32 + 255) / 256), 256, 0, s>>>(w.gt_ptr, n, w.gt_keys, w.big, w.n_big);
    sort_big_rows<<<num_sms() * 2, 1024, 0, s>>>(w.gt_ptr, w.gt_keys, w.big, w.n_big);
    sac_first_kernel<<<grid1d(n, 256), 256, 0, s>>>(nbr, n, k, fi, w.gt_ptr, w.first);
    return check_launch("onng_adjust_degree_sac: G_t");
}

}  // namespace
}  // namespace onng

extern "C" size_t onng_adjust_degree_sac_workspace_bytes(int64_t n, int32_t k)
{
    return sac_carve(nullptr, n, k).used;
}

extern "C" int onng_adjust_degree_sac_count(const int32_t *nbr, const float *len, int64_t n, int32_t k, int32_t e_o,
                                            int32_t e_i, int64_t *row_ptr, int64_t *nnz_host, void *ws,
                                            size_t ws_bytes, onng_stream_t stream)
{
    ONNG_RANGE("onng_adjust_degree_sac_count");
    ONNG_REQUIRE(n >= 0 && n <= INT32_MAX && k >= 1 && e_o >= 0 && e_i >= 0, ONNG_E_INVAL,
                 "onng_adjust_degree_sac_count: bad sizes");
    ONNG_REQUIRE(n == 0 || (nbr && len), ONNG_E_INVAL, "onng_adjust_degree_sac_count: NULL input");
    ONNG_REQUIRE(row_ptr, ONNG_E_INVAL, "onng_adjust_degree_sac_count: NULL row_ptr");
    const size_t need = onng_adjust_degree_sac_workspace_bytes(n, k);
    ONNG_REQUIRE(ws && ws_bytes >= need, ONNG_E_WORKSPACE, "onng_adjust_degree_sac_count: workspace %zu < %zu bytes",
                 ws_bytes, need);
    cudaStream_t s = to_cuda(stream);
    const SacWs w = sac_carve(ws, n, k);
    int st;
    if (n > 0) {
        st = sac_prepare(nbr, len, n, k, std::min(e_i, k), w, s);
        if (st)
            return st;
        sac_row_kernel<<<(unsigned)((n * 32 + 255) / 256), 256, 0, s>>>(nbr, len, n, k, e_o, w.gt_ptr, w.gt_keys,
                                                                       w.first, w.cnt, nullptr, nullptr);
        st = check_launch("onng_adjust_degree_sac_count: rows");
        if (st)
            return st;
    }
    st = exclusive_scan(w.cnt, row_ptr, n, w.scan_ws, w.scan_bytes, s);
    if (st)
        return st;
    if (nnz_host) {
        ONNG_CUDA_TRY(cudaMemcpyAsync(nnz_host, row_ptr + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s),
                      "adjust_degree_sac: nnz");
        ONNG_CUDA_TRY(cudaStreamSynchronize(s), "adjust_degree_sac: sync");
    }
    return ONNG_OK;
}

extern "C" int onng_adjust_degree_sac(const int32_t *nbr, const float *len, int64_t n, int32_t k, int32_t e_o,
                                      int32_t e_i, const int64_t *row_ptr, int32_t *col, float *len_out, void *ws,
                                      size_t ws_bytes, onng_stream_t stream)
{
    ONNG_RANGE("onng_adjust_degree_sac");
    ONNG_REQUIRE(n >= 0 && n <= INT32_MAX && k >= 1 && e_o >= 0 && e_i >= 0, ONNG_E_INVAL,
                 "onng_adjust_degree_sac: bad sizes");
    ONNG_REQUIRE(n == 0 || (nbr && len), ONNG_E_INVAL, "onng_adjust_degree_sac: NULL input");
    const size_t need = onng_adjust_degree_sac_workspace_bytes(n, k);
    ONNG_REQUIRE(ws && ws_bytes >= need, ONNG_E_WORKSPACE, "onng_adjust_degree_sac: workspace %zu < %zu bytes",
                 ws_bytes, need);
    if (n == 0)
        return ONNG_OK;
    ONNG_REQUIRE(row_ptr && col && len_out, ONNG_E_INVAL, "onng_adjust_degree_sac: NULL output");
    cudaStream_t s = to_cuda(stream);
    const SacWs w = sac_carve(ws, n, k);
    int st = sac_prepare(nbr, len, n, k, std::min(e_i, k), w, s);
    if (st)
        return st;
    sac_row_kernel<<<(unsigned)((n * 32 + 255) / 256), 256, 0, s>>>(nbr, len, n, k, e_o, w.gt_ptr, w.gt_keys, w.first,
                                                                   nullptr, row_ptr, w.keys);
    ONNG_CUDA_TRY(cudaMemsetAsync(w.n_big, 0, sizeof(int), s), "adjust_degree_sac: clear");
    sort_small_rows<<<(unsigned)((n * 32 + 255) / 256), 256, 0, s>>>(row_ptr, n, w.keys, w.big, w.n_big);
    sort_big_rows<<<num_sms() * 2, 1024, 0, s>>>(row_ptr, w.keys, w.big, w.n_big);
    st = check_launch("onng_adjust_degree_sac: fill/sort");
    if (st)
        return st;
    unpack_keys<<<grid1d(n * (int64_t)2 * k, 256), 256, 0, s>>>(w.keys, row_ptr + n, col, len_out);
    return check_launch("onng_adjust_degree_sac: unpack");
}

// ------------------------------------------------------------------ literal Algorithm 4 ABI

extern "C" size_t onng_adjust_path_literal_workspace_bytes(int64_t n, int64_t nnz)
{
    const int64_t nn = std::max<int64_t>(n, 1), mm = std::max<int64_t>(nnz, 1);
    WsCarver c(nullptr);
    c.take<unsigned long long>((size_t)mm);  // id-sorted rows
    c.take<unsigned char>((size_t)mm);       // edge states
    c.take<int>((size_t)mm);                 // removal marks
    c.take<int64_t>((size_t)nn);             // kept counts / long rows
    c.take<int64_t>((size_t)nn + 1);         // degree offsets
    c.take<int>((size_t)nn + 1);             // degree histogram / cursors
    c.take<int32_t>((size_t)nn);             // nodes by degree
    c.take<int>(64);
    c.take<char>(scan_workspace_bytes(nn + 1));
    return c.used;
}

extern "C" int onng_adjust_path_literal(const int64_t *row_ptr, const int32_t *col, const float *len, int64_t n,
                                        int64_t *row_ptr_out, int32_t *col_out, float *len_out, int64_t *nnz_host,
                                        void *ws, size_t ws_bytes, onng_stream_t stream)
{
    ONNG_RANGE("onng_adjust_path_literal");
    // ids are sorted as (id << 32 | position) keys below the sorters' padding key
    ONNG_REQUIRE(n >= 0 && n < 0x7F800000LL, ONNG_E_INVAL, "onng_adjust_path_literal: bad n");
    ONNG_REQUIRE(row_ptr && row_ptr_out, ONNG_E_INVAL, "onng_adjust_path_literal: NULL row_ptr");
    cudaStream_t s = to_cuda(stream);
    int64_t nnz = 0;
    ONNG_CUDA_TRY(cudaMemcpyAsync(&nnz, row_ptr + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s),
                  "adjust_path_literal: nnz");
    ONNG_CUDA_TRY(cudaStreamSynchronize(s), "adjust_path_literal: sync");
    const size_t need = onng_adjust_path_literal_workspace_bytes(n, nnz);
    ONNG_REQUIRE(ws && ws_bytes >= need, ONNG_E_WORKSPACE, "onng_adjust_path_literal: workspace %zu < %zu bytes",
                 ws_bytes, need);
    ONNG_REQUIRE(nnz == 0 || (col && len && col_out && len_out), ONNG_E_INVAL,
                 "onng_adjust_path_literal: NULL arrays");
    const int64_t nn = std::max<int64_t>(n, 1), mm = std::max<int64_t>(nnz, 1);
    WsCarver c(ws);
    unsigned long long *byid = c.take<unsigned long long>((size_t)mm);
    unsigned char *state = c.take<unsigned char>((size_t)mm);
    int *wit = c.take<int>((size_t)mm);
    int64_t *kept = c.take<int64_t>((size_t)nn);
    int64_t *offset = c.take<int64_t>((size_t)nn + 1);
    int *hist = c.take<int>((size_t)nn + 1);
    int32_t *order = c.take<int32_t>((size_t)nn);
    int *flags = c.take<int>(64);
    char *scan_ws = c.take<char>(scan_workspace_bytes(nn + 1));
    int st;
    if (n > 0 && nnz > 0) {
        // rows by id for the position lookups of Algorithm 5
        ONNG_CUDA_TRY(cudaMemsetAsync(flags, 0, sizeof(int) * 64, s), "adjust_path_literal: clear");
        alg4_byid_kernel<<<(unsigned)((n * 32 + 255) / 256), 256, 0, s>>>(row_ptr, col, n, byid);
        sort_small_rows<<<(unsigned)((n * 32 + 255) / 256), 256, 0, s>>>(row_ptr, n, byid, kept, flags);
        sort_big_rows<<<num_sms() * 2, 1024, 0, s>>>(row_ptr, byid, kept, flags);
        // nodes by degree, largest first
        ONNG_CUDA_TRY(cudaMemsetAsync(hist, 0, sizeof(int) * (n + 1), s), "adjust_path_literal: clear");
        alg4_hist_kernel<<<grid1d(n, 256), 256, 0, s>>>(row_ptr, n, hist);
        ONNG_CUDA_TRY(cudaMemsetAsync(state, 0, (size_t)nnz, s), "adjust_path_literal: clear");
        st = check_launch("onng_adjust_path_literal: prepare");
        if (st)
            return st;
        std::vector<int> h((size_t)n + 1);
        ONNG_CUDA_TRY(cudaMemcpyAsync(h.data(), hist, sizeof(int) * (n + 1), cudaMemcpyDeviceToHost, s),
                      "adjust_path_literal: histogram");
        ONNG_CUDA_TRY(cudaStreamSynchronize(s), "adjust_path_literal: sync");
        int64_t maxdeg = 0;
        for (int64_t d = n; d >= 0; --d)
            if (h[d]) {
                maxdeg = d;
                break;
            }
        std::vector<int64_t> off((size_t)n + 1, 0), active((size_t)maxdeg + 1, 0);
        int64_t acc = 0;
        for (int64_t d = maxdeg; d >= 0; --d) {
            off[d] = acc;  // nodes of degree > d come first
            acc += h[d];
        }
        for (int64_t p = 0; p <= maxdeg; ++p)
            active[p] = off[p];  // nodes with more than p edges
        ONNG_CUDA_TRY(cudaMemcpyAsync(offset, off.data(), sizeof(int64_t) * (n + 1), cudaMemcpyHostToDevice, s),
                      "adjust_path_literal: offsets");
        ONNG_CUDA_TRY(cudaMemsetAsync(hist, 0, sizeof(int) * (n + 1), s), "adjust_path_literal: clear");
        alg4_order_kernel<<<grid1d(n, 256), 256, 0, s>>>(row_ptr, n, offset, hist, order);
        st = check_launch("onng_adjust_path_literal: order");
        if (st)
            return st;
        int *waiting = flags + 32;
        for (int64_t p = 0; p < maxdeg; ++p) {
            const int64_t act = active[p];
            // every pass decides at least the smallest waiting node, so act + 1 passes suffice
            for (int64_t pass = 0;; ++pass) {
                ONNG_REQUIRE(pass <= act, ONNG_E_LIMIT, "onng_adjust_path_literal: round %lld did not settle",
                             (long long)p);
                ONNG_CUDA_TRY(cudaMemsetAsync(waiting, 0, sizeof(int), s), "adjust_path_literal: clear");
                alg4_round_kernel<<<(unsigned)((act * 32 + 255) / 256), 256, 0, s>>>(row_ptr, col, len, byid, order,
                                                                                  act, (int)p, state, waiting);
                st = check_launch("onng_adjust_path_literal: round");
                if (st)
                    return st;
                int left = 0;
                ONNG_CUDA_TRY(cudaMemcpyAsync(&left, waiting, sizeof(int), cudaMemcpyDeviceToHost, s),
                              "adjust_path_literal: waiting");
                ONNG_CUDA_TRY(cudaStreamSynchronize(s), "adjust_path_literal: sync");
                if (left == 0)
                    break;
            }
        }
        alg4_wit_kernel<<<grid1d(nnz, 256), 256, 0, s>>>(state, nnz, wit);
        path_count_kernel<<<(unsigned)((n * 32 + 255) / 256), 256, 0, s>>>(row_ptr, n, wit, kept);
        st = check_launch("onng_adjust_path_literal: count");
        if (st)
            return st;
    } else if (n > 0) {
        ONNG_CUDA_TRY(cudaMemsetAsync(kept, 0, sizeof(int64_t) * n, s), "adjust_path_literal: clear");
    }
    st = exclusive_scan(kept, row_ptr_out, n, scan_ws, scan_workspace_bytes(nn + 1), s);
    if (st)
        return st;
    if (n > 0 && nnz > 0) {
        path_compact_kernel<<<(unsigned)((n * 32 + 255) / 256), 256, 0, s>>>(row_ptr, col, len, n, wit, row_ptr_out,
                                                                           col_out, len_out, nullptr);
        st = check_launch("onng_adjust_path_literal: compact");
        if (st)
            return st;
    }
    if (nnz_host) {
        ONNG_CUDA_TRY(cudaMemcpyAsync(nnz_host, row_ptr_out + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s),
                      "adjust_path_literal: nnz");
        ONNG_CUDA_TRY(cudaStreamSynchronize(s), "adjust_path_literal: sync");
    }
    return ONNG_OK;
}

// ------------------------------------------------------------------ path ABI

extern "C" size_t onng_adjust_path_workspace_bytes(int64_t n, int64_t nnz)
{
    WsCarver c(nullptr);
    c.take<int>((size_t)std::max<int64_t>(nnz, 1));        // witness positions
    c.take<int>((size_t)std::max<int64_t>(nnz, 1) * 2);    // hub hash keys
    c.take<int>((size_t)std::max<int64_t>(nnz, 1) * 2);    // hub hash positions
    c.take<int64_t>((size_t)std::max<int64_t>(n, 1));      // kept counts / long rows
    c.take<int64_t>((size_t)std::max<int64_t>(n, 1));
    c.take<int>(64);
    c.take<unsigned long long>(4);
    c.take<char>(scan_workspace_bytes(std::max<int64_t>(n, 1)));
    return c.used;
}

extern "C" int onng_adjust_path(const int64_t *row_ptr, const int32_t *col, const float *len, int64_t n,
                                int64_t *row_ptr_out, int32_t *col_out, float *len_out, int64_t *nnz_host,
                                int32_t *removed_by, void *ws, size_t ws_bytes, onng_stream_t stream)
{
    ONNG_RANGE("onng_adjust_path");
    ONNG_REQUIRE(n >= 0 && n <= INT32_MAX, ONNG_E_INVAL, "onng_adjust_path: bad n");
    ONNG_REQUIRE(row_ptr && row_ptr_out, ONNG_E_INVAL, "onng_adjust_path: NULL row_ptr");
    cudaStream_t s = to_cuda(stream);
    int64_t nnz = 0;
    ONNG_CUDA_TRY(cudaMemcpyAsync(&nnz, row_ptr + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s), "adjust_path: nnz");
    ONNG_CUDA_TRY(cudaStreamSynchronize(s), "adjust_path: sync");
    const size_t need = onng_adjust_path_workspace_bytes(n, nnz);
    ONNG_REQUIRE(ws && ws_bytes >= need, ONNG_E_WORKSPACE, "onng_adjust_path: workspace %zu < %zu bytes", ws_bytes,
                 need);
    ONNG_REQUIRE(nnz == 0 || (col && len && col_out && len_out), ONNG_E_INVAL, "onng_adjust_path: NULL arrays");
    WsCarver c(ws);
    int *wit = c.take<int>((size_t)std::max<int64_t>(nnz, 1));
    int *skey = c.take<int>((size_t)std::max<int64_t>(nnz, 1) * 2);
    int *spos = c.take<int>((size_t)std::max<int64_t>(nnz, 1) * 2);
    int64_t *kept = c.take<int64_t>((size_t)std::max<int64_t>(n, 1));
    int64_t *big = c.take<int64_t>((size_t)std::max<int64_t>(n, 1));
    int *n_big = c.take<int>(64);
    c.take<unsigned long long>(4);
    char *scan_ws = c.take<char>(scan_workspace_bytes(std::max<int64_t>(n, 1)));
    int st;
    if (n > 0) {
        ONNG_CUDA_TRY(cudaMemsetAsync(n_big, 0, sizeof(int), s), "adjust_path: clear");
        int per_sm = 0;
        ONNG_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, path_small_kernel, kPathWarps * 32, 0),
                      "adjust_path: occupancy");
        const int64_t resident = (int64_t)num_sms() * std::max(per_sm, 1);
        const int64_t ctas = std::min<int64_t>((n + kPathWarps - 1) / kPathWarps, resident);
        path_small_kernel<<<(unsigned)ctas, kPathWarps * 32, 0, s>>>(row_ptr, col, len, n, wit, big, n_big);
        // hub rows: the kernel reads the count of listed rows on the device
        path_big_kernel<<<num_sms() * 2, 512, 0, s>>>(row_ptr, col, len, wit, big, n_big, skey, spos);
        st = check_launch("onng_adjust_path: mark");
        if (st)
            return st;
        path_count_kernel<<<(unsigned)((n * 32 + 255) / 256), 256, 0, s>>>(row_ptr, n, wit, kept);
        st = check_launch("onng_adjust_path: count");
        if (st)
            return st;
    }
    st = exclusive_scan(kept, row_ptr_out, n, scan_ws, scan_workspace_bytes(std::max<int64_t>(n, 1)), s);
    if (st)
        return st;
    if (n > 0) {
        path_compact_kernel<<<(unsigned)((n * 32 + 255) / 256), 256, 0, s>>>(row_ptr, col, len, n, wit, row_ptr_out,
                                                                           col_out, len_out, removed_by);
        st = check_launch("onng_adjust_path: compact");
        if (st)
            return st;
    }
    if (nnz_host) {
        ONNG_CUDA_TRY(cudaMemcpyAsync(nnz_host, row_ptr_out + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s),
                      "adjust_path: nnz");
        ONNG_CUDA_TRY(cudaStreamSynchronize(s), "adjust_path: sync");
    }
    return ONNG_OK;
}
