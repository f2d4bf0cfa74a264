// Plain layout types shared by host-only and device code (no CUDA headers).
#pragma once

#include <stdint.h>

#if defined(__CUDACC__)
#define LPOP_HD __host__ __device__
#else
#define LPOP_HD
#endif

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
// when len <= kPairMaxLen, or unit_rows rows when a matrix sets it); units of
// all bins are numbered consecutively.
constexpr int kSegmented = -1;
constexpr int kSell = -2;

struct Bin {
  int row_begin;
  int row_end;
  int width;
  int unit_begin;
  int len;         // kSell: entries per row
  int unit_rows;   // kSell: rows per unit when set (0: the default below), a multiple of 32 (64 for pairs)
  long long base;  // kSell: position of the bin's first entry in the sliced copy
};

// Rows per work unit of a bin.
LPOP_HD inline int rows_per_unit(const Bin& b) {
  if (b.width == 0 || b.width == kSegmented) return 1;
  if (b.width == kSell) return b.unit_rows > 0 ? b.unit_rows : (b.len <= kPairMaxLen ? 2 * kBlock : kBlock);
  return kBlock / b.width;
}

constexpr long long kBlockRowThreshold = 2048;  // rows longer than this get a whole block
constexpr int kCountMax = 4096;                 // rows up to this long are ordered by a counting key

// Lanes per row for a row of length len: 1 up to kSellMaxLen entries (one
// lane per row needs no shuffle adds to combine lane sums and runs the row's
// epilogue on every lane: on GB300 the FP64 pipe limits these kernels), 4, 16
// or 32 for longer rows, 0 (a block per row) beyond kBlockRowThreshold.
// `widen` (a power of two >= 1) asks for up to that many lanes on short rows
// when a matrix has too few rows to occupy the GPU with one lane each.
LPOP_HD inline int width_for_length(long long len, int widen = 1) {
  int w;
  if (len <= kSellMaxLen) w = 1;
  else if (len <= 64) w = 4;
  else if (len <= 256) w = 16;
  else if (len <= kBlockRowThreshold) w = 32;
  else return 0;
  // a short row gains nothing from more lanes than entries
  int cap = 1;
  while (cap < len && cap < 32) cap <<= 1;
  const int wide = widen < cap ? widen : cap;
  return w > wide ? w : wide;
}

// Work order of the row classes: whole-block rows first (they are the
// longest, so they start early), then 32, 16, ... 1 lanes.
LPOP_HD inline int bin_rank(int width) {
  switch (width) {
    case 0: return 0;
    case 32: return 1;
    case 16: return 2;
    case 8: return 3;
    case 4: return 4;
    case 2: return 5;
    default: return 6;
  }
}

// Position key of a row in the bin order of a matrix whose longest row has
// lmax entries: ascending keys put the rows longer than kCountMax first
// (longest first), then class by class in work order, longest first within a
// class.  Sorting the rows stably by this key gives the bin order.
LPOP_HD inline unsigned order_key(long long len, int widen, long long lmax) {
  const long long base = (lmax > kCountMax ? lmax : kCountMax) - kCountMax;
  if (len > kCountMax) return (unsigned)(base + kCountMax - len);
  return (unsigned)(base + (long long)bin_rank(width_for_length(len, widen)) * (kCountMax + 1) + (kCountMax - len));
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
