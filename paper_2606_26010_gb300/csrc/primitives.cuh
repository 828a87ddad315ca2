#pragma once
#include "far_internal.cuh"

namespace far {

// Number of partial sums scan_exclusive needs for n items (allocate scan_blocks(n) + 1).
u32 scan_blocks(u32 n);
// out[i] = sum in[0..i) over min(n, *n_dev) items (n_dev may be null); *total_dev = total
// (may be null). In-place (in == out) is allowed. n <= 2^27.
cudaError_t scan_exclusive(const u32* in, u32* out, u32 n, const u32* n_dev, u32* total_dev, u32* partials,
                           cudaStream_t s);

// Tiles of the radix sort for n items; `hist` needs 256 * radix_blocks(n) entries and
// `scan_partials` scan_blocks(256 * radix_blocks(n)) + 1 entries.
u32 radix_blocks(u32 n);
// Stable sort of (keys, vals) by the low `bits` bits of the keys (8 bits per pass).
// The result is in (keys, vals) or, when *result_in_alt, in (keys_alt, vals_alt).
cudaError_t radix_sort_pairs(u32* keys, u32* vals, u32* keys_alt, u32* vals_alt, u32 n, int bits, u32* hist,
                             u32* scan_partials, cudaStream_t s, bool* result_in_alt);

}  // namespace far
