// Host-side data layout of a problem: input validation, duplicate merging,
// and the permuted ("bin order") CSR copies of A and A^T.  Pure C++: no CUDA
// calls, so it runs (and is tested) without a GPU.
#pragma once

#include <stdint.h>

#include <string>
#include <vector>

#include "layout_types.h"

namespace lpop {

struct HostLayout {
  int m = 0, n = 0;
  long long nnz = 0;  // after merging repeated entries
  std::vector<int> prow, pcol;  // permuted index -> caller's index
  std::vector<int> A_rp, A_ci, At_rp, At_ci;
  std::vector<double> A_v, At_v;
  BinTable binsA{}, binsAt{};
};

// Lanes per row for a row of length len: 1, 2, 4, ..., 32, or 0 (a block per
// row).  `widen` (a power of two >= 1) asks for up to that many lanes on short
// rows when a matrix has too few rows to occupy the GPU with one lane each.
int width_for_length(long long len, int widen = 1);

// Validate the CSR input and build the layout.  Returns 0 on success, or a
// negative lp_err code with a message in err.  target_threads: threads that
// fill the GPU (SMs x resident threads); matrices with fewer rows get wider
// row groups.
int build_layout(int32_t m, int32_t n, int64_t nnz, const int64_t* row_ptr, const int32_t* col_idx,
                 const double* val, HostLayout& out, std::string& err, long long target_threads = 0);

// Bin table for rows already sorted by bin (widths in "work" order, longest
// rows first within a width).  One-lane rows form kSell bins of one exact
// length each (no kSell bins when lengths_sorted is empty).
BinTable make_bins(const std::vector<int>& widths_sorted, const std::vector<int>& lengths_sorted);

// Entries of the sliced copy of a table's kSell bins (padding included); the
// copy itself is filled on the device.
long long sliced_entries(const BinTable& bt);

// Segment length for a matrix of nnz entries processed by `grid` blocks.
int segment_length(long long nnz, int grid);

// Cut the rows of the whole-block bin longer than seg_len into segments: they
// become a leading kSegmented bin and the unit numbering of every bin is
// redone.  Returns the (row, segment index) pair of each segment unit (empty,
// with bt unchanged, when no row is that long).
std::vector<int> segment_long_rows(BinTable& bt, const std::vector<int>& rp, int seg_len);

}  // namespace lpop
