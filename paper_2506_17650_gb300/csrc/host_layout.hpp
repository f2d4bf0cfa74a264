// Host-side data layout of a problem: input validation, duplicate merging,
// and the permuted ("bin order") CSR copies of A and A^T.  Pure C++: no CUDA
// calls, so it runs (and is tested) without a GPU.
#pragma once

#include <stdint.h>

#include <algorithm>
#include <functional>
#include <mutex>
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

// fn(begin, end) over [0, count) in contiguous pieces, on the layout's host
// threads when the work (count, or `work` when given) is large.
void for_each_range(long long count, const std::function<void(long long, long long)>& fn, long long work = -1);

// Smallest i in [0, count) with bad(i), or count if there is none; on the
// layout's host threads when count is large.  A piece is first tested whole
// (bad ORed over it without an early exit, so the loop has no branch to
// mispredict) and walked for its first bad index only when it holds one.
template <class Bad>
long long first_bad_index(long long count, Bad bad) {
  std::mutex mu;
  long long first = count;
  for_each_range(count, [&](long long b, long long e) {
    bool any = false;
    for (long long i = b; i < e; ++i) any |= bad(i);
    if (!any) return;
    long long i = b;
    while (!bad(i)) ++i;
    std::lock_guard<std::mutex> lock(mu);
    first = std::min(first, i);
  });
  return first;
}

// Check a caller's CSR matrix: sizes and pointers, row_ptr (0 first, nnz
// last, non-decreasing), then every entry (column in range, finite value),
// on host threads.  Returns 0, or a negative lp_err code with a message
// naming the first offending index in err; sets canonical when every row is
// in strictly increasing column order.
int validate_csr(int32_t m, int32_t n, int64_t nnz, const int64_t* row_ptr, const int32_t* col_idx,
                 const double* val, bool& canonical, std::string& err);

// The rows of a valid CSR matrix sorted by column with repeated entries
// summed (rows already in strictly increasing order are copied as they are),
// on host threads.
void merge_rows(int32_t m, const int64_t* row_ptr, const int32_t* col_idx, const double* val,
                std::vector<int64_t>& rp, std::vector<int>& ci, std::vector<double>& cv);

// Validate the CSR input and build the layout on the host.  Returns 0 on
// success, or a negative lp_err code with a message in err.  target_threads:
// threads that fill the GPU (SMs x resident threads); matrices with fewer
// rows get wider row groups.
int build_layout(int32_t m, int32_t n, int64_t nnz, const int64_t* row_ptr, const int32_t* col_idx,
                 const double* val, HostLayout& out, std::string& err, long long target_threads = 0);

// Bin table for rows already sorted by bin (widths in "work" order, longest
// rows first within a width).  One-lane rows form kSell bins of one exact
// length each (no kSell bins when lengths_sorted is empty).
BinTable make_bins(const std::vector<int>& widths_sorted, const std::vector<int>& lengths_sorted);

// One maximal run of rows of one width (and, for kSell, of one length).
struct BinRun {
  int row_begin, row_end, width, len;
};

// Bin table from the runs of a matrix in bin order (width kSell for sliced
// runs): unit numbering and sliced-copy offsets.
BinTable bins_from_runs(const std::vector<BinRun>& runs);

// Widen factor of build_layout for a matrix of `rows` rows: a power of two
// >= target_threads / rows, capped at 8 (1 when the rows fill the GPU).
int widen_factor(long long rows, long long target_threads);

// Rows per thread column of a table's kSell bins: units of `rows` rows (a
// multiple of 32 up to kBlock; kBlock is the default), 2 rows for the bins of
// at most kPairMaxLen entries per row, with the units renumbered (a
// segmented bin keeps its units).
void set_sliced_unit_rows(BinTable& bt, int rows);

// Entries of the sliced copy of a table's kSell bins (padding included); the
// copy itself is filled on the device.
long long sliced_entries(const BinTable& bt);

// Segment length for a matrix of nnz entries processed by `grid` blocks (a
// quarter of a block's mean share, at least 4096).
int segment_length(long long nnz, int grid);

// Cut the rows of the whole-block bin longer than seg_len into segments: they
// become a leading kSegmented bin and the unit numbering of every bin is
// redone.  Returns the (row, segment index) pair of each segment unit (empty,
// with bt unchanged, when no row is that long).
std::vector<int> segment_long_rows(BinTable& bt, const std::vector<int>& rp, int seg_len);

}  // namespace lpop
