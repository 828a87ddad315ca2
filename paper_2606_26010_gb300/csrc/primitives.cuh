#pragma once
#include "far_internal.cuh"

namespace far {

// Number of partial sums scan_exclusive needs for n items (allocate scan_blocks(n) + 1).
u32 scan_blocks(u32 n);
// out[i] = sum in[0..i) over min(n, *n_dev) items (n_dev may be null); *total_dev = total
// (may be null). In-place (in == out) is allowed. n <= 2^27.
cudaError_t scan_exclusive(const u32* in, u32* out, u32 n, const u32* n_dev, u32* total_dev, u32* partials,
                           cudaStream_t s);

}  // namespace far
