// Host entry points of the search (Algorithm 1): argument checks, workspace
// layout, grid sizing and launch of the kernels in search_kernel.cuh.
#include <algorithm>
#include <climits>
#include <cmath>

#include "search_kernel.cuh"

namespace onng {
namespace {

using namespace sk;

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

using sk::Launch;

template <class T, int V> Launch pick_kr(int k)
{
    return k <= 32 ? sk::pick<T, V, 1>() : sk::pick<T, V, kMaxK / 32>();
}

template <class T> Launch pick_v(int d, int k)
{
#ifdef ONNG_CHECK
    // the bounds-checked build carries the float32 kernels only
    if constexpr (!std::is_same<T, float>::value) {
        return {nullptr, 0};
    } else
#endif
    {
        const int V = (d + 127) / 128;
        if (V <= 1)
            return pick_kr<T, 1>(k);
        if constexpr (ONNG_SEARCH_MAXV >= 2)
            if (V <= 2)
                return pick_kr<T, 2>(k);
        if constexpr (ONNG_SEARCH_MAXV >= 4)
            if (V <= 4)
                return pick_kr<T, 4>(k);
        if constexpr (ONNG_SEARCH_MAXV >= 8)
            if (V <= 8)
                return pick_kr<T, 8>(k);
        return {nullptr, 0};
    }
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

// per-warp workspace: visited bitmap (rounded to 256 bytes), id log, candidate spill pool
int64_t bits_words(int64_t n) { return (n + 8191) / 8192 * 256; }
int pool_cap(const onng_search_params *p) { return p && p->pool_cap > 0 ? p->pool_cap : kGlobalPool; }
size_t slot_bytes(int64_t n, int cap)
{
    return (size_t)bits_words(n) * sizeof(unsigned) + (size_t)kVisitLog * sizeof(int) + (size_t)cap * sizeof(u64);
}

}  // namespace
}  // namespace onng

using namespace onng;

extern "C" size_t onng_search_workspace_bytes(int64_t nq, const onng_index *idx, const onng_search_params *p)
{
    // sized for the grid of the kernel that will run (the reduced-precision kernels hold more CTAs per SM)
    const int d = idx ? idx->d : 128;
    const int prec = p ? p->precision : ONNG_PREC_FP32;
    const int kr = p ? (prec != ONNG_PREC_FP32 ? std::max(p->k, p->k_rerank) : p->k) : 10;
    Launch L = prec == ONNG_PREC_BF16 ? pick_v<__nv_bfloat16>(d, kr)
               : prec == ONNG_PREC_FP8 ? pick_v<__nv_fp8_e4m3>(d, kr)
                                       : pick_v<float>(d, kr);
    int per_sm = 16;
    if (!L.fn || resident_blocks(L, &per_sm) != ONNG_OK)
        per_sm = 16;
    const int64_t blocks = std::min<int64_t>(std::max<int64_t>(1, (nq + kWarpsPerCta - 1) / kWarpsPerCta),
                                             (int64_t)per_sm * num_sms());
    return 1024 + (size_t)blocks * kWarpsPerCta * slot_bytes(idx ? idx->n : 1, pool_cap(p));
}

extern "C" int onng_pad_adjacency(const int64_t *row_ptr, const int32_t *col, int64_t n, int32_t width, int32_t *adj,
                                  onng_stream_t stream)
{
    ONNG_RANGE("onng_pad_adjacency");
    ONNG_REQUIRE(n >= 0 && width >= 1, ONNG_E_INVAL, "onng_pad_adjacency: bad sizes");
    if (n == 0)
        return ONNG_OK;
    ONNG_REQUIRE(row_ptr && adj, ONNG_E_INVAL, "onng_pad_adjacency: NULL pointer");
    const int64_t total = n * width;
    const int blocks = (int)std::min<int64_t>((total + 255) / 256, (int64_t)num_sms() * 16);
    pad_adjacency_kernel<<<blocks, 256, 0, to_cuda(stream)>>>(row_ptr, col, n, width, adj);
    return check_launch("onng_pad_adjacency");
}

static int search_impl(const onng_index *idx, const float *Q, int64_t nq, const onng_search_params *p,
                       const int32_t *seeds, int32_t n_seed, const float *eps_q, const int32_t *es_q, int32_t *out_ids,
                       float *out_dist, int32_t *stats, float *feat, float target, void *ws, size_t ws_bytes,
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
    ONNG_REQUIRE(p->pool_cap >= 0 && p->pool_cap <= (1 << 24), ONNG_E_INVAL, "onng_search: pool_cap must be in [0, 2^24]");
    ONNG_REQUIRE(idx->adj == nullptr || idx->adj_width >= 1, ONNG_E_INVAL, "onng_search: adj_width must be >= 1");
    const bool bf16 = p->precision == ONNG_PREC_BF16;
    const bool fp8 = p->precision == ONNG_PREC_FP8;
    ONNG_REQUIRE(p->precision == ONNG_PREC_FP32 || bf16 || fp8, ONNG_E_INVAL, "onng_search: unknown precision");
    int kr = p->k;
    if (bf16 || fp8) {
        kr = std::max(p->k, p->k_rerank);
        ONNG_REQUIRE(kr <= kMaxK, ONNG_E_UNSUPPORTED, "onng_search: k_rerank > %d", kMaxK);
    }
    if (bf16)
        ONNG_REQUIRE(idx->X_bf16 && aligned16(idx->X_bf16), ONNG_E_INVAL, "onng_search: bf16 needs aligned X_bf16");
    if (fp8)
        ONNG_REQUIRE(idx->X_fp8 && aligned16(idx->X_fp8) && idx->fp8_scale && aligned16(idx->fp8_scale),
                     ONNG_E_INVAL, "onng_search: fp8 needs aligned X_fp8 and fp8_scale");
    if (nq == 0)
        return ONNG_OK;
    ONNG_REQUIRE(idx->row_ptr && idx->col && idx->X && Q && seeds && (feat || (out_ids && out_dist)), ONNG_E_INVAL,
                 "onng_search: NULL pointer");
    ONNG_REQUIRE(aligned16(idx->X) && aligned16(Q), ONNG_E_INVAL, "onng_search: X and Q must be 16-byte aligned");
    ONNG_REQUIRE(ws, ONNG_E_WORKSPACE, "onng_search: NULL workspace");

    Launch L = bf16  ? pick_v<__nv_bfloat16>(idx->d, kr)
               : fp8 ? pick_v<__nv_fp8_e4m3>(idx->d, kr)
                     : pick_v<float>(idx->d, kr);
    ONNG_REQUIRE(L.fn, ONNG_E_UNSUPPORTED, "onng_search: no kernel for d=%d", idx->d);
    int per_sm = 0;
    int st = resident_blocks(L, &per_sm);
    if (st)
        return st;
    int64_t blocks = std::min<int64_t>((nq + kWarpsPerCta - 1) / kWarpsPerCta, (int64_t)per_sm * num_sms());
    // the workspace bounds the number of warps (each needs its own spill tables)
    const int cap = pool_cap(p);
    const size_t per_cta = slot_bytes(idx->n, cap) * kWarpsPerCta;
    const int64_t fit = ws_bytes > 1024 ? (int64_t)((ws_bytes - 1024) / per_cta) : 0;
    blocks = std::min(blocks, fit);
    ONNG_REQUIRE(blocks >= 1, ONNG_E_WORKSPACE, "onng_search: workspace of %zu bytes holds no CTA (%zu needed per CTA)",
                 ws_bytes, per_cta + 1024);

    WsCarver c(ws);
    SearchArgs a;
    a.counter = c.take<int>(64);
    const int64_t slots = blocks * kWarpsPerCta;
    a.bits_words = bits_words(idx->n);
    a.gbits = c.take<unsigned>((size_t)slots * a.bits_words);
    a.glog = c.take<int>((size_t)slots * kVisitLog);
    a.gpool = c.take<u64>((size_t)slots * cap);
    a.gpool_cap = cap;
    a.row_ptr = idx->row_ptr;
    a.col = idx->col;
    a.adj = idx->adj;
    a.adj_w = idx->adj_width;
    a.X = idx->X;
    a.Xb = idx->X_bf16;
    a.X8 = idx->X_fp8;
    a.scale8 = idx->fp8_scale;
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
    a.feat = feat;
    a.target = target;
    cudaStream_t s = to_cuda(stream);
    ONNG_CUDA_TRY(cudaMemsetAsync(a.counter, 0, sizeof(int), s), "onng_search: reset counter");
    // the bitmaps start empty; every query leaves its bitmap empty again
    ONNG_CUDA_TRY(cudaMemsetAsync(a.gbits, 0, sizeof(unsigned) * (size_t)slots * a.bits_words, s),
                  "onng_search: clear visited bitmaps");
    L.fn<<<(unsigned)blocks, kWarpsPerCta * 32, L.smem, s>>>(a);
    return check_launch("onng_search");
}

extern "C" int onng_search(const onng_index *idx, const float *Q, int64_t nq, const onng_search_params *p,
                           const int32_t *seeds, int32_t n_seed, const float *eps_q, const int32_t *es_q,
                           int32_t *out_ids, float *out_dist, int32_t *stats, void *ws, size_t ws_bytes,
                           onng_stream_t stream)
{
    ONNG_RANGE("onng_search");
    return search_impl(idx, Q, nq, p, seeds, n_seed, eps_q, es_q, out_ids, out_dist, stats, nullptr, 0.f, ws,
                       ws_bytes, stream);
}

extern "C" int onng_search_probe(const onng_index *idx, const float *Q, int64_t nq, const onng_search_params *p,
                                 const int32_t *seeds, int32_t n_seed, float target, float *features, int32_t *stats,
                                 void *ws, size_t ws_bytes, onng_stream_t stream)
{
    ONNG_RANGE("onng_search_probe");
    ONNG_REQUIRE(p && p->max_expansions >= 1, ONNG_E_INVAL, "onng_search_probe: max_expansions must be >= 1");
    ONNG_REQUIRE(features || nq == 0, ONNG_E_INVAL, "onng_search_probe: NULL features");
    return search_impl(idx, Q, nq, p, seeds, n_seed, nullptr, nullptr, nullptr, nullptr, stats, features, target, ws,
                       ws_bytes, stream);
}

// ---------------------------------------------------------------------------
// onng_search without allocation.  Some callers cannot allocate device memory
// per call: a query loop that must not stall (cudaMalloc and cudaFree may
// synchronise the whole device), a process whose memory is already committed
// to the index and its batch buffers, or C code with no allocator of its own.
// For them the search's scratch lives in one fixed array per device.  The
// array is reserved when this module is loaded and held until the process
// exits, so its size is kept modest; search_impl sizes the grid to it.
//
// Host code must not hand `g_noalloc_scratch` to a kernel: here that name is a
// host-side stand-in for the symbol, not its device address.  The address is
// looked up on every call, with the caller's device current, so a device reset
// or a reloaded module never leaves a stale pointer behind.
static __device__ __align__(256) unsigned char g_noalloc_scratch[ONNG_SEARCH_NOALLOC_SCRATCH_BYTES];

namespace onng {
namespace {

int noalloc_scratch(void **out)
{
    void *ptr = nullptr;
    ONNG_CUDA_TRY(cudaGetSymbolAddress(&ptr, g_noalloc_scratch), "onng_search_noalloc: scratch address");
    ONNG_REQUIRE(ptr, ONNG_E_CUDA, "onng_search_noalloc: scratch address is NULL");
    *out = ptr;
    return ONNG_OK;
}

}  // namespace
}  // namespace onng

extern "C" int onng_search_noalloc(const onng_index *idx, const float *Q, int64_t nq, const onng_search_params *p,
                                   const int32_t *seeds, int32_t n_seed, const float *eps_q, const int32_t *es_q,
                                   int32_t *out_ids, float *out_dist, int32_t *stats, onng_stream_t stream)
{
    ONNG_RANGE("onng_search_noalloc");
    ONNG_REQUIRE(idx && p, ONNG_E_INVAL, "onng_search_noalloc: NULL index or params");
    ONNG_REQUIRE(idx->n > 0 && idx->n <= INT32_MAX, ONNG_E_INVAL, "onng_search_noalloc: bad index size");
    // one CTA's share: the query counter's slot plus kWarpsPerCta per-warp slots
    const size_t cap = (size_t)ONNG_SEARCH_NOALLOC_SCRATCH_BYTES;
    ONNG_REQUIRE(p->pool_cap >= 0 && p->pool_cap <= (1 << 24), ONNG_E_INVAL,
                 "onng_search_noalloc: pool_cap must be in [0, 2^24]");
    const size_t need = 1024 + (size_t)kWarpsPerCta * slot_bytes(idx->n, pool_cap(p));
    ONNG_REQUIRE(need <= cap, ONNG_E_WORKSPACE,
                 "onng_search_noalloc: an index of n = %lld needs %zu scratch bytes for one CTA, more than the "
                 "fixed %zu (use onng_search with a caller workspace)",
                 (long long)idx->n, need, cap);
    if (nq == 0)
        return search_impl(idx, Q, nq, p, seeds, n_seed, eps_q, es_q, out_ids, out_dist, stats, nullptr, 0.f,
                           nullptr, 0, stream);
    void *ws = nullptr;
    const int st = noalloc_scratch(&ws);
    if (st)
        return st;
    // search_impl clears the counter and the bitmaps on `stream` before its launch
    return search_impl(idx, Q, nq, p, seeds, n_seed, eps_q, es_q, out_ids, out_dist, stats, nullptr, 0.f, ws, cap,
                       stream);
}
