// The layout of a problem built on the device from the caller's CSR arrays:
// the bin order of the rows of A and of A^T, the permuted CSR copies of both
// and the bin tables, equal entry for entry to what build_layout makes on the
// host.  The host keeps only the permutations, the bin tables and a few row
// pointers; the matrices never exist on the host in permuted form.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <functional>
#include <string>
#include <vector>

#include "host_layout.hpp"

namespace lpop {

// Device arrays of a layout, allocated by the caller: the permuted CSR of A
// (m + 1 row pointers, nnz entries) and of A^T (n + 1, nnz), and optionally
// (null: not kept) the permutations themselves (permuted index -> caller's
// index, m and n entries).
struct LayoutArrays {
  int* A_rp;
  int* A_ci;
  double* A_v;
  int* At_rp;
  int* At_ci;
  double* At_v;
  int* prow;
  int* pcol;
};

// Optional: the caller's b, c, lb, ub and senses (host) and their device
// copies in bin order (b and the senses permuted like the rows of A, c, lb
// and ub like its columns; senses as Sense codes).  Null host pointers skip
// them.
struct LayoutVectors {
  const double *b, *c, *lb, *ub;
  const char* sense;
  double *d_b, *d_c, *d_l, *d_u;
  uint8_t* d_sense;
};

// What the host keeps of a layout built on the device.
struct LayoutInfo {
  std::vector<int> prow, pcol;       // permuted index -> caller's index
  BinTable binsA{}, binsAt{};
  std::vector<int> A_head, At_head;  // row pointers 0..e of the leading whole-block bin (rows 0..e-1), if any
  int split[2] = {0, 0};             // first row of A / A^T with at most 32 entries (or the row count)
};

// Device scratch for the build: sets *ptr to `bytes` bytes of device memory
// (256-byte aligned) and returns 0, or returns a negative lp_err code.  The
// build frees nothing; the caller releases the scratch after the call returns
// (the stream is synchronized by then).
using ScratchAlloc = std::function<int(void** ptr, size_t bytes)>;

// Build the layout of a valid CSR matrix whose rows are in strictly
// increasing column order (what validate_csr accepts as canonical, or what
// merge_rows returns) on the device, on stream s: the caller's arrays are
// copied up once, then row and column lengths, the bin orders (stable radix
// sorts by order_key), and the permuted CSR of A^T and of A (two stable
// radix sorts of the entries, by permuted column and then by permuted row,
// so that the rows of both come out in increasing index order) are computed
// there.  `widen` as in width_for_length (1: no widening).  Returns 0, or a
// negative lp_err code with a message in err.
int build_layout_device(int32_t m, int32_t n, int64_t nnz, const int64_t* row_ptr, const int32_t* col_idx,
                        const double* val, int widen_a, int widen_at, const LayoutArrays& out,
                        const LayoutVectors* vec, LayoutInfo& info, const ScratchAlloc& alloc, cudaStream_t s,
                        std::string& err);

}  // namespace lpop
