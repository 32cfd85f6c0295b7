// Device-wide exclusive prefix sum: per-block scans of 4096 values, a recursive
// scan of the block totals, then a pass that adds each block's offset.
#include "scan.cuh"

namespace onng {
namespace {

constexpr int kThreads = 1024, kPer = 4, kTile = kThreads * kPer;

__device__ int64_t block_excl_scan(int64_t v, int64_t *sh, int64_t *total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int64_t x = v;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        int64_t y = __shfl_up_sync(0xffffffffu, x, off);
        if (lane >= off)
            x += y;
    }
    if (lane == 31)
        sh[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int64_t w = sh[lane];
        int64_t z = w;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            int64_t y = __shfl_up_sync(0xffffffffu, z, off);
            if (lane >= off)
                z += y;
        }
        sh[lane] = z - w;
        if (lane == 31)
            sh[32] = z;
    }
    __syncthreads();
    int64_t r = x - v + sh[warp];
    *total = sh[32];
    __syncthreads();
    return r;
}

// out[i] = exclusive prefix within the block; sums[b] = block total.
__global__ void scan_blocks(const int64_t *__restrict__ in, int64_t *__restrict__ out, int64_t n,
                            int64_t *__restrict__ sums)
{
    __shared__ int64_t sh[33];
    const int64_t base = (int64_t)blockIdx.x * kTile + (int64_t)threadIdx.x * kPer;
    int64_t v[kPer];
    int64_t s = 0;
#pragma unroll
    for (int i = 0; i < kPer; ++i) {
        v[i] = base + i < n ? in[base + i] : 0;
        s += v[i];
    }
    int64_t total;
    int64_t pre = block_excl_scan(s, sh, &total);
#pragma unroll
    for (int i = 0; i < kPer; ++i) {
        if (base + i < n)
            out[base + i] = pre;
        pre += v[i];
    }
    if (threadIdx.x == 0)
        sums[blockIdx.x] = total;
}

__global__ void add_offsets(int64_t *__restrict__ out, int64_t n, const int64_t *__restrict__ offs)
{
    const int64_t base = (int64_t)blockIdx.x * kTile + (int64_t)threadIdx.x * kPer;
    const int64_t o = offs[blockIdx.x];
#pragma unroll
    for (int i = 0; i < kPer; ++i)
        if (base + i < n)
            out[base + i] += o;
}

// Exclusive scan of n values into out[0..n) plus the total in out[n] (recursive).
int scan_rec(const int64_t *in, int64_t *out, int64_t n, char *ws, cudaStream_t s)
{
    const int64_t blocks = (n + kTile - 1) / kTile;
    int64_t *sums = reinterpret_cast<int64_t *>(ws);
    int64_t *sums_scan = sums + align_up((size_t)blocks, 32);
    char *next = reinterpret_cast<char *>(sums_scan + align_up((size_t)blocks + 1, 32));
    scan_blocks<<<(unsigned)blocks, kThreads, 0, s>>>(in, out, n, sums);
    int st = check_launch("scan: blocks");
    if (st)
        return st;
    if (blocks == 1) {
        // total of the single block lands in out[n]
        ONNG_CUDA_TRY(cudaMemcpyAsync(out + n, sums, sizeof(int64_t), cudaMemcpyDeviceToDevice, s), "scan: total");
        return ONNG_OK;
    }
    st = scan_rec(sums, sums_scan, blocks, next, s);
    if (st)
        return st;
    add_offsets<<<(unsigned)blocks, kThreads, 0, s>>>(out, n, sums_scan);
    st = check_launch("scan: offsets");
    if (st)
        return st;
    ONNG_CUDA_TRY(cudaMemcpyAsync(out + n, sums_scan + blocks, sizeof(int64_t), cudaMemcpyDeviceToDevice, s),
                  "scan: total");
    return ONNG_OK;
}

}  // namespace

size_t scan_workspace_bytes(int64_t n)
{
    size_t bytes = 0;
    int64_t m = n;
    do {
        const int64_t blocks = (m + kTile - 1) / kTile;
        bytes += (align_up((size_t)blocks, 32) + align_up((size_t)blocks + 1, 32)) * sizeof(int64_t);
        m = blocks;
    } while (m > 1);
    return bytes + 256;
}

int exclusive_scan(const int64_t *in, int64_t *out, int64_t n, void *ws, size_t ws_bytes, cudaStream_t s)
{
    if (n == 0) {
        ONNG_CUDA_TRY(cudaMemsetAsync(out, 0, sizeof(int64_t), s), "scan: empty");
        return ONNG_OK;
    }
    if (ws_bytes < scan_workspace_bytes(n))
        return set_error(ONNG_E_WORKSPACE, "scan: workspace too small");
    return scan_rec(in, out, n, static_cast<char *>(ws), s);
}

}  // namespace onng
