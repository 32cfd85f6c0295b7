// Graph statistics of Table 4 (Sec. 3.1): mean outdegree of the top 5 % of the
// nodes by outdegree, mean indegree of the bottom 5 % by indegree, and the mean
// indegree distance (edges of the transposed graph, each node's list cut to its
// 10 shortest); plus the maximum indegree and the count of unreachable nodes
// (indegree 0) that Sec. 3 and Fig. 3(c) discuss.
//
// Degrees are 32-bit.  The m-th largest (or smallest) degree is found by an
// 8-bit radix select: four histogram passes over the nodes, each followed by a
// one-warp kernel that picks the digit and narrows the prefix, so the host never
// waits between passes.  The sum of the m extreme degrees is then
// sum(v beyond the m-th value) + (m - count beyond) * m-th value.
//
// The indegree distance builds the transposed lengths by counting sort (indegree
// scan, atomic cursors), then a warp per node keeps each lane's 10 shortest in
// registers and takes the 10 shortest of the node by ten warp-wide minimum
// rounds.  Lengths are non-negative, so their float bits order as unsigned
// integers.
#include <cmath>

#include "common.cuh"
#include "scan.cuh"

namespace onng {
namespace {

constexpr int ST_NT = 256;
constexpr int TOPL = 10;  // incoming edges kept per node

struct SelState {
    unsigned prefix, mask;
    long long kleft;  // elements still to take at the current prefix
    unsigned long long sum_beyond;
    long long cnt_beyond;
};

__device__ __forceinline__ unsigned deg_out(const int64_t *row_ptr, int64_t i)
{
    return (unsigned)(row_ptr[i + 1] - row_ptr[i]);
}

__global__ void indeg_kernel(const int32_t *__restrict__ col, int64_t nnz, int64_t n, unsigned *__restrict__ indeg,
                             int *bad)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x) {
        const int c = col[e];
        if (c < 0 || c >= n)
            atomicOr(bad, 1);
        else
            atomicAdd(&indeg[c], 1u);
    }
}

// out_deg[i] = row_ptr[i+1] - row_ptr[i]; maxima and the count of indegree-0 nodes
__global__ void degree_kernel(const int64_t *__restrict__ row_ptr, const unsigned *__restrict__ indeg, int64_t n,
                              unsigned *__restrict__ outdeg, unsigned *max_out, unsigned *max_in,
                              unsigned long long *zero_in)
{
    unsigned mo = 0, mi = 0, z = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const unsigned o = deg_out(row_ptr, i), d = indeg[i];
        outdeg[i] = o;
        mo = max(mo, o);
        mi = max(mi, d);
        z += d == 0;
    }
    mo = __reduce_max_sync(0xffffffffu, mo);
    mi = __reduce_max_sync(0xffffffffu, mi);
    z = __reduce_add_sync(0xffffffffu, z);
    if ((threadIdx.x & 31) == 0) {
        atomicMax(max_out, mo);
        atomicMax(max_in, mi);
        atomicAdd(zero_in, (unsigned long long)z);
    }
}

// key of a degree for the selection: largest first (top) or smallest first
__device__ __forceinline__ unsigned sel_key(unsigned v, bool smallest) { return smallest ? ~v : v; }

__global__ void sel_init(SelState *st, long long m)
{
    st->prefix = 0;
    st->mask = 0;
    st->kleft = m;
    st->sum_beyond = 0;
    st->cnt_beyond = 0;
}

__global__ void sel_hist(const unsigned *__restrict__ v, int64_t n, bool smallest, const SelState *st, int shift,
                         unsigned long long *__restrict__ hist)
{
    __shared__ unsigned h[256];
    for (int b = threadIdx.x; b < 256; b += blockDim.x)
        h[b] = 0;
    __syncthreads();
    const unsigned prefix = st->prefix, mask = st->mask;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const unsigned key = sel_key(v[i], smallest);
        if ((key & mask) == prefix)
            atomicAdd(&h[(key >> shift) & 255u], 1u);
    }
    __syncthreads();
    for (int b = threadIdx.x; b < 256; b += blockDim.x)
        if (h[b])
            atomicAdd(&hist[b], (unsigned long long)h[b]);
}

// One warp: the digit (from 255 down) that holds the kleft-th key of the
// current prefix; clears the histogram for the next pass.
__global__ void sel_pick(SelState *st, int shift, unsigned long long *hist)
{
    const int lane = threadIdx.x;
    if (lane == 0 && st->kleft > 0) {
        long long above = 0;
        int b = 255;
        for (; b > 0; --b) {
            const long long c = (long long)hist[b];
            if (above + c >= st->kleft)
                break;
            above += c;
        }
        st->kleft -= above;
        st->prefix |= (unsigned)b << shift;
        st->mask |= 255u << shift;
    }
    __syncwarp();
    for (int b = lane; b < 256; b += 32)
        hist[b] = 0;
}

// sum and count of the values whose key lies beyond (above) the selected key
__global__ void sel_sum(const unsigned *__restrict__ v, int64_t n, bool smallest, SelState *st)
{
    const unsigned t = st->prefix;
    unsigned long long s = 0, c = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const unsigned x = v[i];
        if (sel_key(x, smallest) > t) {
            s += x;
            ++c;
        }
    }
#pragma unroll
    for (int off = 16; off; off >>= 1) {
        s += __shfl_xor_sync(0xffffffffu, s, off);
        c += __shfl_xor_sync(0xffffffffu, c, off);
    }
    if ((threadIdx.x & 31) == 0 && c) {
        atomicAdd(&st->sum_beyond, s);
        atomicAdd(reinterpret_cast<unsigned long long *>(&st->cnt_beyond), c);
    }
}

__global__ void in_ptr_kernel(const unsigned *__restrict__ indeg, int64_t n, int64_t *__restrict__ cnt)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        cnt[i] = indeg[i];
}

__global__ void transpose_lengths(const int64_t *__restrict__ row_ptr, const int32_t *__restrict__ col,
                                  const float *__restrict__ len, int64_t n, unsigned long long *__restrict__ cursor,
                                  float *__restrict__ in_len)
{
    // warp per source row
    const int lane = threadIdx.x & 31;
    for (int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; i < n;
         i += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        for (int64_t e = row_ptr[i] + lane; e < row_ptr[i + 1]; e += 32) {
            const int c = col[e];
            if (c < 0 || c >= n)
                continue;  // reported by indeg_kernel
            const unsigned long long pos = atomicAdd(&cursor[c], 1ull);
            in_len[pos] = len[e];
        }
    }
}

// warp per node: sum of its (up to) 10 shortest incoming lengths
__global__ void in_dist_kernel(const int64_t *__restrict__ in_ptr, const float *__restrict__ in_len, int64_t n,
                               double *sum, unsigned long long *count)
{
    const int lane = threadIdx.x & 31;
    double s = 0.0;
    unsigned long long c = 0;
    for (int64_t j = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; j < n;
         j += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        const int64_t b = in_ptr[j], e = in_ptr[j + 1];
        unsigned loc[TOPL];  // this lane's shortest, ascending (float bits)
#pragma unroll
        for (int t = 0; t < TOPL; ++t)
            loc[t] = 0xFFFFFFFFu;
        for (int64_t p = b + lane; p < e; p += 32) {
            unsigned x = __float_as_uint(in_len[p]);
#pragma unroll
            for (int t = 0; t < TOPL; ++t) {
                const unsigned lo = min(loc[t], x);
                x = max(loc[t], x);
                loc[t] = lo;
            }
        }
        const int take = e - b < TOPL ? (int)(e - b) : TOPL;
        for (int r = 0; r < take; ++r) {
            const unsigned m = __reduce_min_sync(0xffffffffu, loc[0]);
            const unsigned who = __ballot_sync(0xffffffffu, loc[0] == m);
            if (lane == __ffs(who) - 1) {
#pragma unroll
                for (int t = 0; t + 1 < TOPL; ++t)
                    loc[t] = loc[t + 1];
                loc[TOPL - 1] = 0xFFFFFFFFu;
            }
            s += (double)__uint_as_float(m);
        }
        c += (unsigned long long)take;
    }
    if (lane == 0 && c) {
        atomicAdd(sum, s);
        atomicAdd(count, c);
    }
}

struct StatsWs {
    unsigned *indeg, *outdeg, *maxes;
    unsigned long long *zero_in, *hist, *cursor, *count;
    double *sum;
    SelState *sel;
    int *bad;
    int64_t *in_ptr, *cnt;
    float *in_len;
    char *scan_ws;
    size_t scan_bytes;
    size_t used;
};

StatsWs carve(void *ws, int64_t n, int64_t nnz)
{
    WsCarver c(ws);
    StatsWs w;
    w.indeg = c.take<unsigned>((size_t)n + 1);
    w.outdeg = c.take<unsigned>((size_t)n + 1);
    w.maxes = c.take<unsigned>(2);
    w.zero_in = c.take<unsigned long long>(1);
    w.hist = c.take<unsigned long long>(256);
    w.count = c.take<unsigned long long>(1);
    w.sum = c.take<double>(1);
    w.sel = c.take<SelState>(2);
    w.bad = c.take<int>(1);
    w.in_ptr = c.take<int64_t>((size_t)n + 1);
    w.cnt = c.take<int64_t>((size_t)n + 1);
    w.cursor = c.take<unsigned long long>((size_t)n + 1);
    w.in_len = c.take<float>((size_t)nnz + 1);
    w.scan_bytes = scan_workspace_bytes(n);
    w.scan_ws = c.take<char>(w.scan_bytes);
    w.used = c.used;
    return w;
}

// sum of the m largest (or smallest) values of v [n], into sel
void select_sum(const unsigned *v, int64_t n, long long m, bool smallest, SelState *sel, unsigned long long *hist,
                int grid, cudaStream_t s)
{
    sel_init<<<1, 1, 0, s>>>(sel, m);
    for (int pass = 0; pass < 4; ++pass) {
        const int shift = 24 - 8 * pass;
        sel_hist<<<grid, ST_NT, 0, s>>>(v, n, smallest, sel, shift, hist);
        sel_pick<<<1, 32, 0, s>>>(sel, shift, hist);
    }
    sel_sum<<<grid, ST_NT, 0, s>>>(v, n, smallest, sel);
}

}  // namespace
}  // namespace onng

using namespace onng;

extern "C" size_t onng_graph_stats_workspace_bytes(int64_t n, int64_t nnz)
{
    return carve(nullptr, n < 0 ? 0 : n, nnz < 0 ? 0 : nnz).used;
}

extern "C" int onng_graph_stats(const int64_t *row_ptr, const int32_t *col, const float *len, int64_t n,
                                onng_graph_stats_t *out, void *ws, size_t ws_bytes, onng_stream_t stream)
{
    ONNG_RANGE("onng_graph_stats");
    ONNG_REQUIRE(n >= 1 && n <= INT32_MAX, ONNG_E_INVAL, "onng_graph_stats: n must be in [1, 2^31)");
    ONNG_REQUIRE(row_ptr && out, ONNG_E_INVAL, "onng_graph_stats: NULL pointer");
    cudaStream_t s = to_cuda(stream);
    int64_t nnz = 0;
    ONNG_CUDA_TRY(cudaMemcpyAsync(&nnz, row_ptr + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s),
                  "onng_graph_stats: read nnz");
    ONNG_CUDA_TRY(cudaStreamSynchronize(s), "onng_graph_stats: read nnz");
    ONNG_REQUIRE(nnz >= 0, ONNG_E_INVAL, "onng_graph_stats: row_ptr[n] < 0");
    ONNG_REQUIRE(nnz == 0 || (col && len), ONNG_E_INVAL, "onng_graph_stats: NULL col or len");
    const size_t need = onng_graph_stats_workspace_bytes(n, nnz);
    ONNG_REQUIRE(ws && ws_bytes >= need, ONNG_E_WORKSPACE, "onng_graph_stats: workspace %zu < %zu bytes", ws_bytes,
                 need);
    StatsWs w = carve(ws, n, nnz);
    const int grid = num_sms() * 8;
    // everything from indeg up to bad is zeroed: counts, maxima, accumulators
    ONNG_CUDA_TRY(cudaMemsetAsync(w.indeg, 0, sizeof(unsigned) * ((size_t)n + 1), s), "onng_graph_stats: clear");
    ONNG_CUDA_TRY(cudaMemsetAsync(w.maxes, 0, reinterpret_cast<char *>(w.in_ptr) - reinterpret_cast<char *>(w.maxes),
                                  s),
                  "onng_graph_stats: clear");
    if (nnz)
        indeg_kernel<<<grid, ST_NT, 0, s>>>(col, nnz, n, w.indeg, w.bad);
    degree_kernel<<<grid, ST_NT, 0, s>>>(row_ptr, w.indeg, n, w.outdeg, w.maxes, w.maxes + 1, w.zero_in);
    int st = check_launch("onng_graph_stats: degrees");
    if (st)
        return st;
    const long long m = (n + 19) / 20;  // ceil(5 % of n)
    select_sum(w.outdeg, n, m, false, w.sel, w.hist, grid, s);
    select_sum(w.indeg, n, m, true, w.sel + 1, w.hist, grid, s);
    if ((st = check_launch("onng_graph_stats: selection")))
        return st;
    if (nnz) {
        in_ptr_kernel<<<grid, ST_NT, 0, s>>>(w.indeg, n, w.cnt);
        if ((st = check_launch("onng_graph_stats: indegree copy")) ||
            (st = exclusive_scan(w.cnt, w.in_ptr, n, w.scan_ws, w.scan_bytes, s)))
            return st;
        ONNG_CUDA_TRY(cudaMemcpyAsync(w.cursor, w.in_ptr, sizeof(int64_t) * (size_t)n, cudaMemcpyDeviceToDevice, s),
                      "onng_graph_stats: cursors");
        transpose_lengths<<<grid, ST_NT, 0, s>>>(row_ptr, col, len, n, w.cursor, w.in_len);
        in_dist_kernel<<<grid, ST_NT, 0, s>>>(w.in_ptr, w.in_len, n, w.sum, w.count);
        if ((st = check_launch("onng_graph_stats: indegree distance")))
            return st;
    }
    unsigned maxes[2];
    unsigned long long zero = 0, cnt = 0;
    double sum = 0.0;
    SelState sel[2];
    int bad = 0;
    ONNG_CUDA_TRY(cudaMemcpyAsync(maxes, w.maxes, sizeof(maxes), cudaMemcpyDeviceToHost, s), "onng_graph_stats");
    ONNG_CUDA_TRY(cudaMemcpyAsync(&zero, w.zero_in, sizeof(zero), cudaMemcpyDeviceToHost, s), "onng_graph_stats");
    ONNG_CUDA_TRY(cudaMemcpyAsync(&cnt, w.count, sizeof(cnt), cudaMemcpyDeviceToHost, s), "onng_graph_stats");
    ONNG_CUDA_TRY(cudaMemcpyAsync(&sum, w.sum, sizeof(sum), cudaMemcpyDeviceToHost, s), "onng_graph_stats");
    ONNG_CUDA_TRY(cudaMemcpyAsync(sel, w.sel, sizeof(sel), cudaMemcpyDeviceToHost, s), "onng_graph_stats");
    ONNG_CUDA_TRY(cudaMemcpyAsync(&bad, w.bad, sizeof(bad), cudaMemcpyDeviceToHost, s), "onng_graph_stats");
    ONNG_CUDA_TRY(cudaStreamSynchronize(s), "onng_graph_stats");
    ONNG_REQUIRE(!bad, ONNG_E_INVAL, "onng_graph_stats: a column id lies outside [0, n)");
    out->n = n;
    out->nnz = nnz;
    out->max_out = maxes[0];
    out->max_in = maxes[1];
    out->zero_in = (int64_t)zero;
    out->mean_out = (double)nnz / (double)n;
    // the m-th key's value: the prefix itself (top) or its complement (bottom)
    const double t_top = (double)sel[0].prefix, t_bot = (double)(~sel[1].prefix);
    out->top5_out = ((double)sel[0].sum_beyond + (double)(m - sel[0].cnt_beyond) * t_top) / (double)m;
    out->bottom5_in = ((double)sel[1].sum_beyond + (double)(m - sel[1].cnt_beyond) * t_bot) / (double)m;
    out->in_dist10 = cnt ? sum / (double)cnt : NAN;
    return ONNG_OK;
}
