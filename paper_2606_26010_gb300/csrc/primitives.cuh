#pragma once
#include "far_internal.cuh"

namespace far {

// Number of partial sums scan_exclusive needs for n items (allocate scan_blocks(n) + 1;
// scan_exclusive2 needs twice as many).
u32 scan_blocks(u32 n);
// out[i] = sum in[0..i) over min(n, *n_dev) items (n_dev may be null); *total_dev = total
// (may be null). In-place (in == out) is allowed. n <= 2^27.
cudaError_t scan_exclusive(const u32* in, u32* out, u32 n, const u32* n_dev, u32* total_dev, u32* partials,
                           cudaStream_t s);

// Two independent scans of n items each in one pair of launches (job 0: in0 -> out0, job 1:
// in1 -> out1, each bounded by its own n_dev and writing its own total).
cudaError_t scan_exclusive2(const u32* in0, u32* out0, const u32* n_dev0, u32* total0, const u32* in1, u32* out1,
                            const u32* n_dev1, u32* total1, u32 n, u32* partials, cudaStream_t s);

}  // namespace far
