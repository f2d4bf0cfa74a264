// Binned CSR row products with a per-row epilogue.
//
// A kernel built on for_each_row() walks the work units of a BinTable in a
// grid-stride loop.  For every row r it forms NV dot products
//     s[q] = sum_k M.v[k] * x_q[M.ci[k]],   k in [M.rp[r], M.rp[r+1])
// in the accumulator type Acc (matrix and vectors of type V) and hands them to
// op.row(r, s); op.prefetch(r) is called first, before the row's loads, so an
// op can start loading its own per-row operands early.  Rows up to 48 entries
// use one lane (two rows per thread up to 2 entries) and read a sliced copy,
// longer rows 4..32 lanes that stride through the row so that one warp's loads
// of M.v and M.ci are contiguous, long rows a whole block, and the longest rows
// several blocks (segments).  Lane sums are combined by a fixed shuffle tree,
// so results do not depend on scheduling.
#pragma once

#include <type_traits>

#include "common.cuh"

namespace lpop {

template <int NV, class V>
struct Gather {
  const V* x[NV];
  int n = 0x7fffffff;            // entries of each x (checked builds reject indices beyond)
  unsigned int* bad = nullptr;   // checked builds: count of rejected indices
};

// x[q][c].  Built with LPOP_CHECK_BOUNDS (the debug build the tests use), an
// index outside [0, n) is counted in *bad and reads 0 instead of memory.
template <int NV, class V>
__device__ __forceinline__ V gather(const Gather<NV, V>& g, int q, int c) {
#ifdef LPOP_CHECK_BOUNDS
  if ((unsigned)c >= (unsigned)g.n) {
    if (g.bad) atomicAdd(g.bad, 1u);
    return V(0);
  }
#endif
  return __ldg(g.x[q] + c);
}

// Ops that keep per-block reduction accumulators (member `acc`).
template <class Op, class = void>
struct HasAcc : std::false_type {};
template <class Op>
struct HasAcc<Op, std::void_t<decltype(std::declval<Op&>().acc)>> : std::true_type {};

// Ops that take short sliced rows two per thread (all but those that declare kNoPair).
template <class Op, class = void>
struct AllowsPair : std::true_type {};
template <class Op>
struct AllowsPair<Op, std::void_t<decltype(Op::kNoPair)>> : std::false_type {};

// Entries handled per lane per round: all their index/value loads are issued,
// then all gathers, then the FMAs, so each lane keeps kChunk independent
// loads in flight instead of one dependent load chain per entry.
constexpr int kChunk = 8;

// s[q] += sum over this lane's entries k = k0 + u * stride (u < kChunk, k < end), in order of k.
template <int NV, class V, class Acc>
__device__ __forceinline__ void chunk_dot(int k0, int end, int stride, const CsrT<V>& M, const Gather<NV, V>& g,
                                          Acc (&s)[NV]) {
  int c[kChunk];
  Acc a[kChunk];
#pragma unroll
  for (int u = 0; u < kChunk; ++u) {
    const int k = k0 + u * stride;
    const bool ok = k < end;
    c[u] = ok ? __ldg(M.ci + k) : -1;
    a[u] = ok ? (Acc)__ldg(M.v + k) : Acc(0);
  }
  // entries of this lane in the chunk, and their maximum over the warp's active
  // lanes: FMAs past it are skipped by a warp-uniform branch (on GB300 a
  // predicated-off FP64 instruction still costs its issue slots)
  const int mine = end > k0 ? min(kChunk, (end - k0 + stride - 1) / stride) : 0;
  const int most = __reduce_max_sync(__activemask(), mine);
#pragma unroll
  for (int q = 0; q < NV; ++q) {
    Acc xv[kChunk];
#pragma unroll
    for (int u = 0; u < kChunk; ++u) xv[u] = c[u] >= 0 ? (Acc)gather(g, q, c[u]) : Acc(0);
#pragma unroll
    for (int u = 0; u < kChunk; ++u) {
      if (u >= most) break;
      if (u < mine) s[q] = fma(a[u], xv[u], s[q]);
    }
  }
}

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
    for (int k0 = beg + lane; k0 < end; k0 += kChunk * W) chunk_dot<NV, V, Acc>(k0, end, W, M, g, s);
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

template <class V>
__device__ __forceinline__ const V* sell_values(const BinTable& bt);
template <>
__device__ __forceinline__ const double* sell_values<double>(const BinTable& bt) { return bt.sell_v; }
template <>
__device__ __forceinline__ const float* sell_values<float>(const BinTable& bt) { return bt.sell_v32; }

// Row i of a kSell bin (row B.row_begin + i), of exactly B.len entries, from
// the sliced copy.  Called by consecutive threads for consecutive rows, so the
// loop bound is the same for the whole warp and the loads of a warp are
// contiguous; the entries are added in row order, as in the CSR path.
template <int NV, class V, class Acc, class Op>
__device__ __forceinline__ void sell_rows_at(const BinTable& bt, const Bin& B, int i, const Gather<NV, V>& g,
                                             Op& op) {
  const int row = B.row_begin + i;
  if (row >= B.row_end) return;
  op.prefetch(row);
  const int L = B.len;
  const int* sci = bt.sell_ci + B.base + (long long)(i >> 5) * (32LL * L) + (i & 31);
  const V* sv = sell_values<V>(bt) + B.base + (long long)(i >> 5) * (32LL * L) + (i & 31);
  Acc s[NV];
#pragma unroll
  for (int q = 0; q < NV; ++q) s[q] = Acc(0);
  for (int k0 = 0; k0 < L; k0 += kChunk) {
    const int nk = min(kChunk, L - k0);  // warp-uniform
    int c[kChunk];
    Acc a[kChunk];
#pragma unroll
    for (int u = 0; u < kChunk; ++u) {
      c[u] = u < nk ? __ldg(sci + 32 * (k0 + u)) : 0;
      a[u] = u < nk ? (Acc)__ldg(sv + 32 * (k0 + u)) : Acc(0);
    }
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      Acc xv[kChunk];
#pragma unroll
      for (int u = 0; u < kChunk; ++u) xv[u] = u < nk ? (Acc)gather(g, q, c[u]) : Acc(0);
#pragma unroll
      for (int u = 0; u < kChunk; ++u) {
        if (u >= nk) break;
        s[q] = fma(a[u], xv[u], s[q]);
      }
    }
  }
  op.row(row, s);
}

// A unit of a kSell bin: thread t < R takes row local * R + t of the bin (R
// rows per unit: kBlock, or fewer when the matrix spreads its rows thinner).
template <int NV, class V, class Acc, class Op>
__device__ __forceinline__ void sell_rows(const BinTable& bt, const Bin& B, int local, const Gather<NV, V>& g,
                                          Op& op) {
  const int R = rows_per_unit(B);
  if ((int)threadIdx.x < R) sell_rows_at<NV, V, Acc>(bt, B, local * R + (int)threadIdx.x, g, op);
}

// A unit of a kSell bin of at most kPairMaxLen entries per row: thread t
// takes rows i and i + kBlock of the unit's 2 kBlock rows, and every load of
// both rows (operands, entries, gathers) is issued before either row's
// arithmetic, so that the two rows' FP64 chains interleave.  The second row's
// reduction terms are kept apart and added to the thread's accumulators after
// the pair (a fixed order).
template <int NV, class V, class Acc, class Op>
__device__ __forceinline__ void sell_rows_pair(const BinTable& bt, const Bin& B, int local, const Gather<NV, V>& g,
                                               Op& op) {
  constexpr int C = kPairMaxLen;
  const int H = rows_per_unit(B) / 2;  // rows per half unit: thread t < H takes rows t and H + t
  if ((int)threadIdx.x >= H) return;
  const int i0 = local * (2 * H) + (int)threadIdx.x;
  const int i1 = i0 + H;
  const int r0 = B.row_begin + i0, r1 = B.row_begin + i1;
  if (r0 >= B.row_end) return;
  const bool v1 = r1 < B.row_end;
  Op op2 = op;
  if constexpr (HasAcc<Op>::value) {
    constexpr int NA = (int)(sizeof(op.acc) / sizeof(op.acc[0]));
#pragma unroll
    for (int q = 0; q < NA; ++q) op2.acc[q] = 0;
  }
  op.prefetch(r0);
  if (v1) op2.prefetch(r1);
  const int L = B.len;
  const long long o0 = B.base + (long long)(i0 >> 5) * (32LL * L) + (i0 & 31);
  const long long o1 = B.base + (long long)(i1 >> 5) * (32LL * L) + (i1 & 31);
  const int* sci = bt.sell_ci;
  const V* sv = sell_values<V>(bt);
  int c0[C], c1[C];
  Acc a0[C], a1[C];
#pragma unroll
  for (int u = 0; u < C; ++u) {
    const bool ok = u < L;
    c0[u] = ok ? __ldg(sci + o0 + 32 * u) : 0;
    a0[u] = ok ? (Acc)__ldg(sv + o0 + 32 * u) : Acc(0);
    c1[u] = ok && v1 ? __ldg(sci + o1 + 32 * u) : 0;
    a1[u] = ok && v1 ? (Acc)__ldg(sv + o1 + 32 * u) : Acc(0);
  }
  Acc s0[NV], s1[NV];
#pragma unroll
  for (int q = 0; q < NV; ++q) {
    Acc x0[C], x1[C];
#pragma unroll
    for (int u = 0; u < C; ++u) {
      x0[u] = u < L ? (Acc)gather(g, q, c0[u]) : Acc(0);
      x1[u] = u < L && v1 ? (Acc)gather(g, q, c1[u]) : Acc(0);
    }
    s0[q] = Acc(0);
    s1[q] = Acc(0);
#pragma unroll
    for (int u = 0; u < C; ++u) {
      if (u >= L) break;
      s0[q] = fma(a0[u], x0[u], s0[q]);
      s1[q] = fma(a1[u], x1[u], s1[q]);
    }
  }
  op.row(r0, s0);
  if (v1) op2.row(r1, s1);
  if constexpr (HasAcc<Op>::value) {
    constexpr int NA = (int)(sizeof(op.acc) / sizeof(op.acc[0]));
#pragma unroll
    for (int q = 0; q < NA; ++q) op.acc[q] += op2.acc[q];
  }
}

// Block-wide FP64 sums of the entries [beg, end) of one row (valid in warp 0).
template <int NV, class V, class Acc>
__device__ __forceinline__ void block_dot(int beg, int end, const CsrT<V>& M, const Gather<NV, V>& g, double (&s)[NV],
                                          double* smem) {
#pragma unroll
  for (int q = 0; q < NV; ++q) s[q] = 0.0;
  const int stride = (int)blockDim.x;
  for (int k0 = beg + (int)threadIdx.x; k0 < end; k0 += kChunk * stride) {
    Acc t[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) t[q] = Acc(0);
    chunk_dot<NV, V, Acc>(k0, end, stride, M, g, t);
#pragma unroll
    for (int q = 0; q < NV; ++q) s[q] += (double)t[q];
  }
  block_sum<NV>(s, smem);
}

template <int NV, class V, class Acc, class Op>
__device__ __forceinline__ void block_row(int row, const CsrT<V>& M, const Gather<NV, V>& g, Op& op,
                                          double* smem) {
  if (threadIdx.x == 0) op.prefetch(row);
  double s[NV];  // the block-wide sum of a long row is formed in FP64
  block_dot<NV, V, Acc>(__ldg(M.rp + row), __ldg(M.rp + row + 1), M, g, s, smem);
  if (threadIdx.x == 0) {
    Acc r[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) r[q] = (Acc)s[q];
    op.row(row, r);
  }
}

// Run op.row with the op's reduction accumulators diverted into slot[0..): the
// contribution of a segmented row is kept apart from the block's own partial
// sums, so the totals do not depend on which block finishes the row.
template <class Acc, class Op, int NV>
__device__ __forceinline__ void row_into_slot(Op& op, int row, const Acc (&r)[NV], double* slot) {
  constexpr int NA = (int)(sizeof(op.acc) / sizeof(op.acc[0]));
  using A = typename std::remove_reference<decltype(op.acc[0])>::type;
  A saved[NA];
#pragma unroll
  for (int q = 0; q < NA; ++q) {
    saved[q] = op.acc[q];
    op.acc[q] = A(0);
  }
  op.row(row, r);
#pragma unroll
  for (int q = 0; q < NA; ++q) {
    slot[q] = (double)op.acc[q];
    op.acc[q] = saved[q];
  }
  for (int q = NA; q < kMaxPartials; ++q) slot[q] = 0.0;  // fields read by wider sums
}


// One segment of a segmented row, published for the row's other segments;
// the block that completes the row's last segment adds the segment sums in
// segment order and runs the epilogue into the row's slot.
template <int NV, class V, class Acc, class Op>
__device__ __forceinline__ void segment_reduce(const BinTable& bt, int local, int row, int seg, const CsrT<V>& M,
                                               const Gather<NV, V>& g, Op& op, double* smem, double* row_slots) {
  static_assert(NV <= 2, "segment sums hold up to two vectors");
  const int r0 = __ldg(M.rp + row), r1 = __ldg(M.rp + row + 1);
  const int beg = r0 + seg * bt.seg_len;
  const int end = min(beg + bt.seg_len, r1);
  double s[NV];
  block_dot<NV, V, Acc>(beg, end, M, g, s, smem);
  if (threadIdx.x != 0) return;
#pragma unroll
  for (int q = 0; q < NV; ++q) bt.seg_sum[2 * local + q] = s[q];
  __threadfence();
  const int id = row - bt.bin[0].row_begin;
  const unsigned int nseg = (unsigned int)((r1 - r0 + bt.seg_len - 1) / bt.seg_len);
  if (atomicAdd(bt.ticket + id, 1u) != nseg - 1) return;
  __threadfence();
  const int first = local - seg;
  double tot[NV];
#pragma unroll
  for (int q = 0; q < NV; ++q) tot[q] = 0.0;
  for (int t = 0; t < (int)nseg; ++t) {
#pragma unroll
    for (int q = 0; q < NV; ++q) tot[q] += __ldcg(bt.seg_sum + 2 * (first + t) + q);
  }
  bt.ticket[id] = 0u;  // ready for the next launch
  Acc r[NV];
#pragma unroll
  for (int q = 0; q < NV; ++q) r[q] = (Acc)tot[q];
  op.prefetch(row);
  row_into_slot<Acc>(op, row, r, row_slots + (size_t)id * kMaxPartials);
}

// A unit of the segmented bin.  With row_slots (one row of kMaxPartials
// doubles per segmented row, for ops with reduction accumulators) segments
// are reduced by separate blocks (segment_reduce).  Without, the unit of
// segment 0 reduces the whole row and the others do nothing.
template <int NV, class V, class Acc, class Op>
__device__ __forceinline__ void segment_unit(const BinTable& bt, int local, const CsrT<V>& M, const Gather<NV, V>& g,
                                             Op& op, double* smem, double* row_slots) {
  const int row = __ldg(bt.seg_unit + 2 * local);
  const int seg = __ldg(bt.seg_unit + 2 * local + 1);
  if constexpr (HasAcc<Op>::value) {
    if (row_slots) {
      segment_reduce<NV, V, Acc>(bt, local, row, seg, M, g, op, smem, row_slots);
      return;
    }
  }
  if (seg == 0) block_row<NV, V, Acc>(row, M, g, op, smem);
}

// Work units first_unit, first_unit + unit_stride, ... of the table (one block
// per unit at a time).  smem must hold 32 * NV doubles.  row_slots: see
// segment_unit.
template <int NV, class V, class Acc, class Op>
__device__ __forceinline__ void for_each_row_range(const BinTable& bt, const CsrT<V>& M, const Gather<NV, V>& g,
                                                   Op& op, double* smem, int first_unit, int unit_stride,
                                                   double* row_slots = nullptr) {
  int b = 0;  // units only increase, so the bin search resumes where it stopped
  for (int u = first_unit; u < bt.nunits; u += unit_stride) {
    while (b + 1 < bt.nbins && u >= bt.bin[b + 1].unit_begin) ++b;
    const int row_begin = bt.bin[b].row_begin;
    const int row_end = bt.bin[b].row_end;
    const int local = u - bt.bin[b].unit_begin;
    switch (bt.bin[b].width) {
      case kSegmented: segment_unit<NV, V, Acc>(bt, local, M, g, op, smem, row_slots); break;
      case kSell:
        if (bt.bin[b].len <= kPairMaxLen) {  // units of two halves of H rows (H = kBlock by default)
          const int H = rows_per_unit(bt.bin[b]) / 2;
          if (bt.sell_ci) {
            if constexpr (AllowsPair<Op>::value) {
              sell_rows_pair<NV, V, Acc>(bt, bt.bin[b], local, g, op);
            } else if ((int)threadIdx.x < H) {  // the unit's two halves one after the other
              const int i0 = local * 2 * H + (int)threadIdx.x;
              sell_rows_at<NV, V, Acc>(bt, bt.bin[b], i0, g, op);
              sell_rows_at<NV, V, Acc>(bt, bt.bin[b], i0 + H, g, op);
            }
          } else {
            const int h0 = row_begin + local * 2 * H;
            vec_rows<1, NV, V, Acc>(h0, min(row_end, h0 + H), M, g, op);
            vec_rows<1, NV, V, Acc>(h0 + H, min(row_end, h0 + 2 * H), M, g, op);
          }
        } else if (bt.sell_ci) {
          sell_rows<NV, V, Acc>(bt, bt.bin[b], local, g, op);
        } else {
          const int R = rows_per_unit(bt.bin[b]);
          vec_rows<1, NV, V, Acc>(row_begin + local * R, min(row_end, row_begin + (local + 1) * R), M, g, op);
        }
        break;
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

// All work units, spread over the grid's blocks in a grid-stride loop (the
// longest rows are numbered first, so they start first).
template <int NV, class V, class Acc, class Op>
__device__ __forceinline__ void for_each_row(const BinTable& bt, const CsrT<V>& M, const Gather<NV, V>& g, Op& op,
                                             double* smem, double* row_slots = nullptr) {
  for_each_row_range<NV, V, Acc>(bt, M, g, op, smem, blockIdx.x, gridDim.x, row_slots);
}

}  // namespace lpop
