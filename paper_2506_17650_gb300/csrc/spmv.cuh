// Binned CSR row products with a per-row epilogue.
//
// A kernel built on for_each_row() walks the work units of a BinTable in a
// grid-stride loop.  For every row r it forms NV dot products
//     s[q] = sum_k M.v[k] * x_q[M.ci[k]],   k in [M.rp[r], M.rp[r+1])
// in the accumulator type Acc (matrix and vectors of type V) and hands them to
// op.row(r, s); op.prefetch(r) is called first, before the row's loads, so an
// op can start loading its own per-row operands early.  Rows up to 16 entries use one lane, longer rows 4..32 lanes
// that stride through the row so that one warp's loads of M.v and M.ci are
// contiguous, very long rows a whole block.  Lane sums are combined by a fixed
// shuffle tree, so results do not depend on scheduling.
#pragma once

#include "common.cuh"

namespace lpop {

template <int NV, class V>
struct Gather {
  const V* x[NV];
};

template <int W, int NV, class V, class Acc, class Op>
__device__ __forceinline__ void vec_rows(int first, int row_end, const CsrT<V>& M, const Gather<NV, V>& g,
                                         Op& op) {
  const int row = first + (int)threadIdx.x / W;
  const int lane = (int)threadIdx.x % W;
  Acc s[NV];
#pragma unroll
  for (int q = 0; q < NV; ++q) s[q] = Acc(0);
  if (row < row_end) {
    if (lane == 0) op.prefetch(row);  // epilogue operands load while the row is gathered
    const int beg = __ldg(M.rp + row);
    const int end = __ldg(M.rp + row + 1);
#pragma unroll 4
    for (int k = beg + lane; k < end; k += W) {
      const Acc a = (Acc)__ldg(M.v + k);
      const int c = __ldg(M.ci + k);
#pragma unroll
      for (int q = 0; q < NV; ++q) s[q] = fma(a, (Acc)__ldg(g.x[q] + c), s[q]);
    }
  }
  if (W > 1) {
#pragma unroll
    for (int q = 0; q < NV; ++q) {
#pragma unroll
      for (int off = W / 2; off > 0; off >>= 1) s[q] += __shfl_down_sync(0xffffffffu, s[q], off, W);
    }
  }
  if (lane == 0 && row < row_end) op.row(row, s);
}

template <int NV, class V, class Acc, class Op>
__device__ __forceinline__ void block_row(int row, const CsrT<V>& M, const Gather<NV, V>& g, Op& op,
                                          double* smem) {
  if (threadIdx.x == 0) op.prefetch(row);
  const int beg = __ldg(M.rp + row);
  const int end = __ldg(M.rp + row + 1);
  double s[NV];  // the block-wide sum of a long row is formed in FP64
#pragma unroll
  for (int q = 0; q < NV; ++q) s[q] = 0.0;
  for (int k = beg + (int)threadIdx.x; k < end; k += (int)blockDim.x) {
    const double a = (double)__ldg(M.v + k);
    const int c = __ldg(M.ci + k);
#pragma unroll
    for (int q = 0; q < NV; ++q) s[q] = fma(a, (double)__ldg(g.x[q] + c), s[q]);
  }
  block_sum<NV>(s, smem);
  if (threadIdx.x == 0) {
    Acc r[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) r[q] = (Acc)s[q];
    op.row(row, r);
  }
}

// smem must hold 32 * NV doubles.
template <int NV, class V, class Acc, class Op>
__device__ __forceinline__ void for_each_row(const BinTable& bt, const CsrT<V>& M, const Gather<NV, V>& g, Op& op,
                                             double* smem) {
  for (int u = blockIdx.x; u < bt.nunits; u += gridDim.x) {
    int b = 0;
    while (b + 1 < bt.nbins && u >= bt.bin[b + 1].unit_begin) ++b;
    const int row_begin = bt.bin[b].row_begin;
    const int row_end = bt.bin[b].row_end;
    const int local = u - bt.bin[b].unit_begin;
    switch (bt.bin[b].width) {
      case 0: block_row<NV, V, Acc>(row_begin + local, M, g, op, smem); break;
      case 1: vec_rows<1, NV, V, Acc>(row_begin + local * kBlock, row_end, M, g, op); break;
      case 2: vec_rows<2, NV, V, Acc>(row_begin + local * (kBlock / 2), row_end, M, g, op); break;
      case 4: vec_rows<4, NV, V, Acc>(row_begin + local * (kBlock / 4), row_end, M, g, op); break;
      case 8: vec_rows<8, NV, V, Acc>(row_begin + local * (kBlock / 8), row_end, M, g, op); break;
      case 16: vec_rows<16, NV, V, Acc>(row_begin + local * (kBlock / 16), row_end, M, g, op); break;
      default: vec_rows<32, NV, V, Acc>(row_begin + local * (kBlock / 32), row_end, M, g, op); break;
    }
  }
}

// Rows per work unit for a bin width (0 = block per row).
__host__ __device__ inline int rows_per_unit(int width) { return width == 0 ? 1 : kBlock / width; }

}  // namespace lpop
