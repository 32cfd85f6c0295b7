// Device-wide exclusive prefix sum of int64 values (CSR row pointers).
#pragma once

#include "common.cuh"

namespace onng {

// Workspace bytes for exclusive_scan over n values.
size_t scan_workspace_bytes(int64_t n);

// out[0] = 0, out[i + 1] = in[0] + ... + in[i]; out has n + 1 entries.  `in`
// and `out` may not alias.
int exclusive_scan(const int64_t *in, int64_t *out, int64_t n, void *ws, size_t ws_bytes, cudaStream_t s);

}  // namespace onng
