// Plain layout types shared by host-only and device code (no CUDA headers).
#pragma once

#include <stdint.h>

namespace lpop {

constexpr int kBlock = 256;      // threads per block of every row kernel
constexpr int kMaxBins = 64;     // row-length classes per matrix
constexpr int kSellMaxLen = 48;  // rows of at most this many entries take one lane, from the sliced copy
constexpr int kPairMaxLen = 2;   // sliced rows of at most this many entries: two rows per thread
constexpr int kMaxPartials = 20; // fields of a partial-sum record (an A-row kernel's own + the folded A^T-row ones)
constexpr int kPrimalTimed = 0;  // kernel ids for the event timers
constexpr int kDualTimed = 1;

enum Sense : uint8_t { kEq = 0, kLe = 1, kGe = 2 };
enum Mode : int { kPlain = 0, kPdlp = 1 };
enum Sched : int { kAdagrad = 0, kAdagradNorm = 1, kConst = 2 };

// One row-length class: rows [row_begin, row_end) of a permuted CSR matrix,
// handled with `width` lanes per row (1..32), a whole block per row when
// width == 0, cut into segments of seg_len entries that different blocks
// reduce concurrently when width == kSegmented, or, when width == kSell, rows
// of exactly `len` entries (len <= kSellMaxLen) read from a sliced copy: slices of 32
// consecutive rows stored column-major (entry k of the slice's row t at
// base + slice * 32 len + 32 k + t), so every load of a warp is contiguous
// and an entry's position needs no row pointer.  Work units: one row per unit
// for width 0, kBlock/width rows per unit for 1..32, one segment per unit for
// kSegmented, kBlock rows per unit for kSell (2 kBlock, two rows per thread,
// when len <= kPairMaxLen); units of all bins are numbered consecutively.
constexpr int kSegmented = -1;
constexpr int kSell = -2;

struct Bin {
  int row_begin;
  int row_end;
  int width;
  int unit_begin;
  int len;         // kSell: entries per row
  long long base;  // kSell: position of the bin's first entry in the sliced copy
};

// Rows per work unit of a bin.
inline int rows_per_unit(const Bin& b) {
  if (b.width == 0 || b.width == kSegmented) return 1;
  if (b.width == kSell) return b.len <= kPairMaxLen ? 2 * kBlock : kBlock;
  return kBlock / b.width;
}

struct BinTable {
  int nbins;
  int nunits;
  Bin bin[kMaxBins];
  // segmented bin (at most one, always bin 0 when present)
  int seg_len;             // entries per segment (0: no segmented bin)
  int seg_rows;            // rows in the segmented bin
  const int* seg_unit;     // device [2 * segment units]: (row, segment index); a row's segments are consecutive
  double* seg_sum;         // device [2 * segment units]: block sums of the segments (up to two vectors)
  unsigned int* ticket;    // device [seg_rows]: segments of the row finished in the running launch
  // sliced copy of the kSell bins (device; null until the values are final,
  // and then the kSell rows are read from the CSR arrays instead)
  const int* sell_ci;
  const double* sell_v;
  const float* sell_v32;
};

}  // namespace lpop
