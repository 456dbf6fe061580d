// Histogram copies of the cell sort.  A bin holds tens to thousands of
// queries of a 2^22 batch (most near the surface), and the histogram atomics
// of one bin, issued from every SM, queue at one L2 address.  On grids of at
// most kCopiesBins bins (R <= 47) the histogram has room for kCoarseCopies
// copies (measured at 32^3 x 2^22: the in-line bin kernel 0.096 -> 0.063 ms;
// the narrow sort beside a fit kernel uses them on coarse grids only),
// copy-major (entry
// copy * nbins + bin: the copies of a bin lie a whole histogram apart, in
// different L2 lines and slices), and a query takes its rank in one copy;
// the rank array keeps (copy << kRankBits) | rank (J <= 2^30, so a rank fits
// in 30 bits).  The scan runs over bins and assigns each bin's copies
// consecutive ranges, so a bin's queries stay contiguous (copy 0 first) and
// its work items are cut from the bin's total, as with one counter per bin.
#pragma once

#include <stdint.h>

namespace efunc {

constexpr int64_t kCoarseBins = 12288;        // coarse grids (R <= 19): shared-memory counting in line
constexpr int64_t kCopiesBins = (int64_t)1 << 17;
constexpr int kCoarseCopies = 4;
constexpr uint32_t kRankBits = 30;
constexpr uint32_t kRankMask = (1u << kRankBits) - 1u;

// histogram copies for a grid of nbins bins (1 or kCoarseCopies)
__host__ __device__ inline int hist_copies(int64_t nbins) { return nbins <= kCopiesBins ? kCoarseCopies : 1; }

// histogram entries (4-byte counters) of a grid of nbins bins
__host__ __device__ inline int64_t hist_entries(int64_t nbins) { return nbins * hist_copies(nbins); }

}  // namespace efunc
