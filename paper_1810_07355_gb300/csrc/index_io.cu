// Index files: a built graph and its vectors written to disk and read back
// (the paper keeps its indexes as NGT files and quotes their memory in Table 7;
// this is the library's own format).  Host code only.
//
// Layout, little-endian, a 64-byte header then the payload:
//   0  char[8]  magic "ONNGIDX" + NUL
//   8  u32      version (1)
//  12  u32      flags: bit 0 = edge lengths present
//  16  i64      n
//  24  i32      d
//  28  u32      CRC-32 of the payload
//  32  i64      nnz
//  40  u8[24]   zero
//  payload: row_ptr [n+1] i64, col [nnz] i32, len [nnz] f32 (if flag bit 0),
//           X [n, d] f32
// The CRC is the common reflected CRC-32 (polynomial 0xEDB88320, initial value
// and final xor 0xFFFFFFFF), table-driven.  Device arrays are streamed through
// a host buffer in chunks; a load checks the header and the CRC of the whole
// payload before it writes any device memory.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <vector>

#include "common.cuh"

namespace onng {
namespace {

constexpr char kMagic[8] = {'O', 'N', 'N', 'G', 'I', 'D', 'X', 0};
constexpr uint32_t kVersion = 1;
constexpr size_t kHeader = 64;
constexpr size_t kChunk = size_t(64) << 20;

struct Header {
    uint32_t flags = 0, crc = 0;
    int64_t n = 0, nnz = 0;
    int32_t d = 0;
};

struct Crc32Table {
    uint32_t t[256];
    Crc32Table()
    {
        for (uint32_t i = 0; i < 256; ++i) {
            uint32_t c = i;
            for (int b = 0; b < 8; ++b)
                c = (c & 1u) ? (c >> 1) ^ 0xEDB88320u : c >> 1;
            t[i] = c;
        }
    }
};

uint32_t crc32_update(uint32_t crc, const void *data, size_t len)
{
    static const Crc32Table table;
    const unsigned char *p = static_cast<const unsigned char *>(data);
    uint32_t c = ~crc;
    for (size_t i = 0; i < len; ++i)
        c = table.t[(c ^ p[i]) & 0xFFu] ^ (c >> 8);
    return ~c;
}

void put_u32(unsigned char *p, uint32_t v)
{
    for (int i = 0; i < 4; ++i)
        p[i] = (unsigned char)(v >> (8 * i));
}
void put_i64(unsigned char *p, int64_t v)
{
    for (int i = 0; i < 8; ++i)
        p[i] = (unsigned char)((uint64_t)v >> (8 * i));
}
uint32_t get_u32(const unsigned char *p)
{
    uint32_t v = 0;
    for (int i = 0; i < 4; ++i)
        v |= (uint32_t)p[i] << (8 * i);
    return v;
}
int64_t get_i64(const unsigned char *p)
{
    uint64_t v = 0;
    for (int i = 0; i < 8; ++i)
        v |= (uint64_t)p[i] << (8 * i);
    return (int64_t)v;
}

void encode(const Header &h, unsigned char *b)
{
    std::memset(b, 0, kHeader);
    std::memcpy(b, kMagic, 8);
    put_u32(b + 8, kVersion);
    put_u32(b + 12, h.flags);
    put_i64(b + 16, h.n);
    put_u32(b + 24, (uint32_t)h.d);
    put_u32(b + 28, h.crc);
    put_i64(b + 32, h.nnz);
}

// sizes in bytes of the payload sections
struct Sections {
    size_t ptr, col, len, x;
    size_t total() const { return ptr + col + len + x; }
};

Sections sections(const Header &h)
{
    Sections s;
    s.ptr = sizeof(int64_t) * (size_t)(h.n + 1);
    s.col = sizeof(int32_t) * (size_t)h.nnz;
    s.len = (h.flags & 1u) ? sizeof(float) * (size_t)h.nnz : 0;
    s.x = sizeof(float) * (size_t)h.n * (size_t)h.d;
    return s;
}

struct File {
    FILE *f = nullptr;
    ~File()
    {
        if (f)
            std::fclose(f);
    }
};

// Reads and checks the header; ONNG_E_INVAL with a message on any mismatch.
int read_header(FILE *f, const char *path, Header *h)
{
    unsigned char b[kHeader];
    if (std::fread(b, 1, kHeader, f) != kHeader)
        return set_error(ONNG_E_INVAL, "onng_index: %s: shorter than the header", path);
    if (std::memcmp(b, kMagic, 8) != 0)
        return set_error(ONNG_E_INVAL, "onng_index: %s: not an index file (magic)", path);
    const uint32_t ver = get_u32(b + 8);
    if (ver != kVersion)
        return set_error(ONNG_E_INVAL, "onng_index: %s: version %u, this library reads %u", path, ver, kVersion);
    h->flags = get_u32(b + 12);
    h->n = get_i64(b + 16);
    h->d = (int32_t)get_u32(b + 24);
    h->crc = get_u32(b + 28);
    h->nnz = get_i64(b + 32);
    for (size_t i = 40; i < kHeader; ++i)
        if (b[i] != 0)
            return set_error(ONNG_E_INVAL, "onng_index: %s: reserved header bytes are not zero", path);
    if (h->n < 0 || h->n > INT32_MAX || h->d <= 0 || h->d % 4 != 0 || h->nnz < 0 || (h->flags & ~1u) != 0)
        return set_error(ONNG_E_INVAL, "onng_index: %s: bad header (n %lld, d %d, nnz %lld, flags %u)", path,
                         (long long)h->n, h->d, (long long)h->nnz, h->flags);
    return ONNG_OK;
}

// CRC of the whole payload, checking that the file holds exactly that many bytes.
int check_payload(FILE *f, const char *path, const Header &h)
{
    const size_t want = sections(h).total();
    std::vector<unsigned char> buf(std::min(kChunk, std::max<size_t>(want, 1)));
    uint32_t crc = 0;
    size_t got = 0;
    for (;;) {
        const size_t r = std::fread(buf.data(), 1, buf.size(), f);
        if (r == 0)
            break;
        crc = crc32_update(crc, buf.data(), r);
        got += r;
        if (got > want)
            break;
    }
    if (got != want)
        return set_error(ONNG_E_INVAL, "onng_index: %s: payload of %zu bytes, header implies %zu", path, got, want);
    if (crc != h.crc)
        return set_error(ONNG_E_INVAL, "onng_index: %s: CRC mismatch (file %08x, computed %08x)", path, h.crc, crc);
    return ONNG_OK;
}

// device -> file through the host buffer, updating the CRC
int write_section(FILE *f, const void *dev, size_t bytes, std::vector<unsigned char> &buf, uint32_t *crc,
                  cudaStream_t s)
{
    const char *p = static_cast<const char *>(dev);
    for (size_t off = 0; off < bytes; off += buf.size()) {
        const size_t m = std::min(buf.size(), bytes - off);
        ONNG_CUDA_TRY(cudaMemcpyAsync(buf.data(), p + off, m, cudaMemcpyDeviceToHost, s), "onng_index_save: copy");
        ONNG_CUDA_TRY(cudaStreamSynchronize(s), "onng_index_save: copy");
        *crc = crc32_update(*crc, buf.data(), m);
        if (std::fwrite(buf.data(), 1, m, f) != m)
            return set_error(ONNG_E_INVAL, "onng_index_save: write failed");
    }
    return ONNG_OK;
}

// file -> device (dev NULL: skip the bytes)
int read_section(FILE *f, void *dev, size_t bytes, std::vector<unsigned char> &buf, cudaStream_t s)
{
    char *p = static_cast<char *>(dev);
    for (size_t off = 0; off < bytes; off += buf.size()) {
        const size_t m = std::min(buf.size(), bytes - off);
        if (std::fread(buf.data(), 1, m, f) != m)
            return set_error(ONNG_E_INVAL, "onng_index_load: short read");
        if (p) {
            ONNG_CUDA_TRY(cudaMemcpyAsync(p + off, buf.data(), m, cudaMemcpyHostToDevice, s), "onng_index_load: copy");
            ONNG_CUDA_TRY(cudaStreamSynchronize(s), "onng_index_load: copy");
        }
    }
    return ONNG_OK;
}

}  // namespace
}  // namespace onng

using namespace onng;

extern "C" uint32_t onng_crc32(uint32_t crc, const void *data, size_t len)
{
    return crc32_update(crc, data, len);
}

extern "C" int onng_index_save(const char *path, const int64_t *row_ptr, const int32_t *col, const float *len,
                               const float *X, int64_t n, int32_t d, onng_stream_t stream)
{
    ONNG_RANGE("onng_index_save");
    ONNG_REQUIRE(path && row_ptr && X, ONNG_E_INVAL, "onng_index_save: NULL pointer");
    ONNG_REQUIRE(n >= 0 && n <= INT32_MAX && d > 0 && d % 4 == 0, ONNG_E_INVAL, "onng_index_save: bad sizes");
    cudaStream_t s = to_cuda(stream);
    Header h;
    ONNG_CUDA_TRY(cudaMemcpyAsync(&h.nnz, row_ptr + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s),
                  "onng_index_save: read nnz");
    ONNG_CUDA_TRY(cudaStreamSynchronize(s), "onng_index_save: read nnz");
    ONNG_REQUIRE(h.nnz >= 0 && (h.nnz == 0 || col), ONNG_E_INVAL, "onng_index_save: bad row_ptr[n] or NULL col");
    h.n = n;
    h.d = d;
    h.flags = len ? 1u : 0u;
    File out;
    out.f = std::fopen(path, "wb");
    ONNG_REQUIRE(out.f, ONNG_E_INVAL, "onng_index_save: cannot open %s for writing", path);
    unsigned char hb[kHeader];
    encode(h, hb);  // CRC written after the payload
    ONNG_REQUIRE(std::fwrite(hb, 1, kHeader, out.f) == kHeader, ONNG_E_INVAL, "onng_index_save: write failed");
    const Sections sz = sections(h);
    std::vector<unsigned char> buf(std::min(kChunk, std::max<size_t>(sz.total(), 1)));
    uint32_t crc = 0;
    int st;
    if ((st = write_section(out.f, row_ptr, sz.ptr, buf, &crc, s)) ||
        (st = write_section(out.f, col, sz.col, buf, &crc, s)) ||
        (st = write_section(out.f, len, sz.len, buf, &crc, s)) ||
        (st = write_section(out.f, X, sz.x, buf, &crc, s)))
        return st;
    h.crc = crc;
    encode(h, hb);
    ONNG_REQUIRE(std::fseek(out.f, 0, SEEK_SET) == 0 && std::fwrite(hb, 1, kHeader, out.f) == kHeader, ONNG_E_INVAL,
                 "onng_index_save: header rewrite failed");
    ONNG_REQUIRE(std::fclose(out.f) == 0, ONNG_E_INVAL, "onng_index_save: close failed");
    out.f = nullptr;
    return ONNG_OK;
}

extern "C" int onng_index_check(const char *path, int64_t *n, int32_t *d, int64_t *nnz, int32_t *has_len)
{
    ONNG_REQUIRE(path, ONNG_E_INVAL, "onng_index_check: NULL path");
    File in;
    in.f = std::fopen(path, "rb");
    ONNG_REQUIRE(in.f, ONNG_E_INVAL, "onng_index_check: cannot open %s", path);
    Header h;
    int st;
    if ((st = read_header(in.f, path, &h)) || (st = check_payload(in.f, path, h)))
        return st;
    if (n)
        *n = h.n;
    if (d)
        *d = h.d;
    if (nnz)
        *nnz = h.nnz;
    if (has_len)
        *has_len = (int32_t)(h.flags & 1u);
    return ONNG_OK;
}

extern "C" int onng_index_load(const char *path, int64_t n, int32_t d, int64_t nnz, int64_t *row_ptr,
                               int32_t *col, float *len, float *X, onng_stream_t stream)
{
    ONNG_RANGE("onng_index_load");
    ONNG_REQUIRE(path && row_ptr && X && (nnz == 0 || col), ONNG_E_INVAL, "onng_index_load: NULL pointer");
    File in;
    in.f = std::fopen(path, "rb");
    ONNG_REQUIRE(in.f, ONNG_E_INVAL, "onng_index_load: cannot open %s", path);
    Header h;
    int st;
    if ((st = read_header(in.f, path, &h)))
        return st;
    ONNG_REQUIRE(h.n == n && h.d == d && h.nnz == nnz, ONNG_E_INVAL,
                 "onng_index_load: %s holds n %lld, d %d, nnz %lld; the call expects n %lld, d %d, nnz %lld", path,
                 (long long)h.n, h.d, (long long)h.nnz, (long long)n, d, (long long)nnz);
    ONNG_REQUIRE(!len || (h.flags & 1u), ONNG_E_INVAL, "onng_index_load: %s holds no edge lengths", path);
    if ((st = check_payload(in.f, path, h)))
        return st;
    ONNG_REQUIRE(std::fseek(in.f, (long)kHeader, SEEK_SET) == 0, ONNG_E_INVAL, "onng_index_load: seek failed");
    const Sections sz = sections(h);
    std::vector<unsigned char> buf(std::min(kChunk, std::max<size_t>(sz.total(), 1)));
    cudaStream_t s = to_cuda(stream);
    if ((st = read_section(in.f, row_ptr, sz.ptr, buf, s)) || (st = read_section(in.f, col, sz.col, buf, s)) ||
        (st = read_section(in.f, len, sz.len, buf, s)) || (st = read_section(in.f, X, sz.x, buf, s)))
        return st;
    return ONNG_OK;
}
