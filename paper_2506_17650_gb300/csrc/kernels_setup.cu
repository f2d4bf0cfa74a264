// Preprocessing kernels (run once per problem by lp_create, and by lp_reset
// for the initial state):
//   - Ruiz equilibration (Section 2): row / column infinity norms, factors
//     1/sqrt(norm), applied to both CSR copies;
//   - Pock-Chambolle rescaling (Section 2): factors 1/sqrt(sum |a|^beta) for
//     rows and 1/sqrt(sum |a|^(2-beta)) for columns;
//   - L2 rescaling (Section 4.2): factors 1/sqrt(||row||_2), 1/sqrt(||col||_2);
//   - rescaling of b, c, l, u; norms; max |a_ij|; power iteration for ||A~||_2;
//   - the initial iterate x_0 = proj_[l,u](0), y_0 = 0, T_0 = Sigma_0 = I (Section 3.2).
// Reductions use per-block partials summed by one block in a fixed order.
#include "common.cuh"
#include "spmv.cuh"

namespace lpop {

namespace {

constexpr int kSetupGrid = 1024;

__global__ void fill_kernel(double* v, double val, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    v[i] = val;
}

__device__ __forceinline__ double pow_term(double v, double beta) {
  const double a = fabs(v);
  return beta == 1.0 ? a : (beta == 2.0 ? a * a : (beta == 0.0 ? 1.0 : pow(a, beta)));
}

// out[r] = sum_k |v_k|^beta (beta == 1 and beta == 2 exact), optionally sqrt:
// the whole-block rows [0, nlong) a block each (four strided partial sums
// per thread, so that four loads are in flight, then the block's fixed
// tree), rows [nlong, split) a warp each, the rows of at most 32 entries
// [split, rows) eight lanes each (four rows per warp at a time); a lane's
// terms are summed in order, then the lanes' sums by a butterfly.
__global__ void row_powsum_kernel(Csr M, int rows, int nlong, int split, double beta, int square_root, double* out) {
  __shared__ double smem[32];
  for (int r = blockIdx.x; r < nlong; r += gridDim.x) {
    double s4[4] = {0.0, 0.0, 0.0, 0.0};
    const int k1 = M.rp[r + 1];
    int k = M.rp[r] + threadIdx.x;
    for (; k + 3 * kBlock < k1; k += 4 * kBlock) {
#pragma unroll
      for (int q = 0; q < 4; ++q) s4[q] += pow_term(M.v[k + q * kBlock], beta);
    }
    if (k < k1) s4[0] += pow_term(M.v[k], beta);  // at most three left
    if (k + kBlock < k1) s4[1] += pow_term(M.v[k + kBlock], beta);
    if (k + 2 * kBlock < k1) s4[2] += pow_term(M.v[k + 2 * kBlock], beta);
    double s[1] = {(s4[0] + s4[1]) + (s4[2] + s4[3])};
    block_sum<1>(s, smem);
    if (threadIdx.x == 0) out[r] = square_root ? sqrt(s[0]) : s[0];
  }
  const int lane = threadIdx.x & 31;
  const int warps = (gridDim.x * blockDim.x) >> 5;
  const int wid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  for (int r = nlong + wid; r < split; r += warps) {
    double s = 0.0;
#pragma unroll 4
    for (int k = M.rp[r] + lane; k < M.rp[r + 1]; k += 32) s += pow_term(M.v[k], beta);
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if (lane == 0) out[r] = square_root ? sqrt(s) : s;
  }
  for (long long r0 = split + 4LL * wid; r0 < rows; r0 += 4LL * warps) {
    const long long r = r0 + (lane >> 3);
    double s = 0.0;
    if (r < rows) {
#pragma unroll 4
      for (int k = M.rp[r] + (lane & 7); k < M.rp[r + 1]; k += 8) s += pow_term(M.v[k], beta);
    }
    for (int off = 4; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if ((lane & 7) == 0 && r < rows) out[r] = square_root ? sqrt(s) : s;
  }
}

// Rows of one matrix in a Ruiz round (rows sorted longest first): the
// whole-block rows [0, nlong) in chunks of kRuizChunk entries, rows
// [nlong, split) a warp each, rows [split, rows) (at most 32 entries) four
// lanes each, so that a warp's loads cover eight runs of consecutive
// entries.  Units (one per warp): chunk units [0, nchunks), then one per warp
// row, then one per eight short rows.
struct RuizRows {
  const int* rp;
  const int* ci;
  double* v;
  int rows;
  RuizSplit sp;
  __host__ __device__ __forceinline__ long long units() const {
    return sp.nchunks + (sp.split - sp.nlong) + (rows - sp.split + 7) / 8;
  }
  // unit w -> (row, first entry, end entry, step) for this lane; false if the lane has no row
  __device__ __forceinline__ bool range(long long w, int lane, long long& r, long long& k0, long long& k1,
                                        int& step) const {
    r = k0 = k1 = 0;
    step = 1;
    if (w < sp.nchunks) {  // the row whose chunks include w: the last r with chunk_pre[r] <= w
      int lo = 0, hi = sp.nlong;
      while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (sp.chunk_pre[mid] <= w) lo = mid;
        else hi = mid;
      }
      r = lo;
      const long long c0 = rp[r] + (w - sp.chunk_pre[lo]) * (long long)kRuizChunk;
      k0 = c0 + lane;
      k1 = min((long long)rp[r + 1], c0 + kRuizChunk);
      step = 32;
      return true;
    }
    w -= sp.nchunks;
    if (w < sp.split - sp.nlong) {
      r = sp.nlong + w;
      k0 = rp[r] + lane;
      k1 = rp[r + 1];
      step = 32;
      return true;
    }
    step = 4;
    r = sp.split + (w - (sp.split - sp.nlong)) * 8 + (lane >> 2);
    if (r >= rows) return false;
    k0 = rp[r] + (lane & 3);
    k1 = rp[r + 1];
    return true;
  }
};

// out[r] = max_k |v_k| for the rows of unit w (max is exact: the result does
// not depend on the order, so the chunks of a row combine by atomic max on
// the bit patterns of their non-negative maxima, into an out[r] zeroed
// before the launch).
__device__ __forceinline__ void absmax_unit(const RuizRows& R, long long w, int lane, double* out) {
  long long r, k0, k1;
  int step;
  const bool has = R.range(w, lane, r, k0, k1, step);
  double mx = 0.0;
  if (has) {
#pragma unroll 4
    for (long long k = k0; k < k1; k += step) mx = fmax(mx, fabs(R.v[k]));
  }
  // step is uniform across the warp: 32 for chunk and warp rows, 4 for eight short rows
  for (int off = step == 32 ? 16 : 2; off > 0; off >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, off));
  if (step == 32) {
    if (lane == 0) {
      if (w < R.sp.nchunks)
        atomicMax(reinterpret_cast<unsigned long long*>(out + r), (unsigned long long)__double_as_longlong(mx));
      else
        out[r] = mx;
    }
  } else if (has && (lane & 3) == 0) {
    out[r] = mx;
  }
}

// v_k <- (v_k * frow_i) * fcol_j for entry (i, j) of A.  For the A copy the
// row is i and ci is j; for the A^T copy the row is j and ci is i.  Both
// copies evaluate the same expression, so they stay bitwise equal.
__device__ __forceinline__ void scale_unit(const RuizRows& R, long long w, int lane, const double* frow,
                                           const double* fcol, bool a_rows) {
  long long r, k0, k1;
  int step;
  if (!R.range(w, lane, r, k0, k1, step)) return;
#pragma unroll 4
  for (long long k = k0; k < k1; k += step) {
    const int c = R.ci[k];
    const long long i = a_rows ? r : c;
    const long long j = a_rows ? c : r;
    R.v[k] = (R.v[k] * frow[i]) * fcol[j];
  }
}

// Row infinity norms of A (into fr) and of A^T (column norms of A, into fc),
// one launch for both.
__global__ void ruiz_norms_kernel(RuizRows A, RuizRows At, double* fr, double* fc) {
  const int lane = threadIdx.x & 31;
  const long long ua = A.units(), total = ua + At.units();
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long w = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < total; w += nw) {
    if (w < ua) absmax_unit(A, w, lane, fr);
    else absmax_unit(At, w - ua, lane, fc);
  }
}

// Both CSR copies scaled by the row factors fr and column factors fc.
__global__ void ruiz_scale_kernel(RuizRows A, RuizRows At, const double* fr, const double* fc) {
  const int lane = threadIdx.x & 31;
  const long long ua = A.units(), total = ua + At.units();
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long w = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < total; w += nw) {
    if (w < ua) scale_unit(A, w, lane, fr, fc, true);
    else scale_unit(At, w - ua, lane, fr, fc, false);
  }
}

// Norms -> factors f = 1 / sqrt(norm) (1 for an empty row or column), and the
// accumulated scalings dr *= f_row, dc *= f_col.
__global__ void factor_mul_kernel(double* fr, double* dr, int m, double* fc, double* dc, int n) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < (long long)m + n;
       t += (long long)gridDim.x * blockDim.x) {
    double* f = t < m ? fr + t : fc + (t - m);
    double* acc = t < m ? dr + t : dc + (t - m);
    const double v = *f;
    const double g = v > 0.0 ? 1.0 / sqrt(v) : 1.0;
    *f = g;
    *acc *= g;
  }
}

__global__ void scale_vectors_kernel(Dev d) {
  const Vecs<double>& v = d.f64;
  const int stride = gridDim.x * blockDim.x;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < d.m; i += stride) {
    v.b[i] = d.dr[i] * v.b[i];
    d.inv_dr[i] = 1.0 / d.dr[i];
  }
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < d.n; j += stride) {
    const double f = d.dc[j];
    v.c[j] = f * v.c[j];
    v.l[j] = v.l[j] / f;
    v.u[j] = v.u[j] / f;
    d.inv_dc[j] = 1.0 / f;
  }
}

__global__ void sumsq_partial_kernel(const double* v, long long n, double* part) {
  __shared__ double smem[32];
  double s[1] = {0.0};
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    s[0] += v[i] * v[i];
  block_sum<1>(s, smem);
  if (threadIdx.x == 0) part[blockIdx.x] = s[0];
}

__global__ void absmax_partial_kernel(const double* v, long long n, double* part) {
  __shared__ double smem[32];
  double mx = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    mx = fmax(mx, fabs(v[i]));
  for (int off = 16; off > 0; off >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, off));
  if ((threadIdx.x & 31) == 0) smem[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t = fmax(t, smem[w]);
    part[blockIdx.x] = t;
  }
}

// out[0] = sqrt(sum part) (mode 0) or max part (mode 1); one block, fixed order
__global__ void finish_kernel(const double* part, int np, double* out, int mode) {
  __shared__ double smem[32];
  double s[1] = {0.0};
  for (int i = threadIdx.x; i < np; i += blockDim.x) s[0] = mode == 0 ? s[0] + part[i] : fmax(s[0], part[i]);
  if (mode == 0) {
    block_sum<1>(s, smem);
    if (threadIdx.x == 0) out[0] = sqrt(s[0]);
  } else {
    for (int off = 16; off > 0; off >>= 1) s[0] = fmax(s[0], __shfl_xor_sync(0xffffffffu, s[0], off));
    if ((threadIdx.x & 31) == 0) smem[threadIdx.x >> 5] = s[0];
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t = fmax(t, smem[w]);
      out[0] = t;
    }
  }
}

__global__ void scale_by_inv_kernel(double* v, int n, const double* denom) {
  const double dv = denom[0];
  if (dv == 0.0) return;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) v[i] = v[i] / dv;
}

struct StoreOp {
  double* y;
  __device__ __forceinline__ void prefetch(int) {}
  __device__ __forceinline__ void row(int r, const double (&s)[1]) { y[r] = s[0]; }
};

__global__ void __launch_bounds__(kBlock) spmv_kernel(Csr M, BinTable bt, const double* x, double* y) {
  __shared__ double smem[32];
  StoreOp op{y};
  Gather<1, double> g;
  g.x[0] = x;
  for_each_row<1, double, double>(bt, M, g, op, smem);
}

__global__ void init_vectors_kernel(Dev d) {
  const Vecs<double>& v = d.f64;
  const int stride = gridDim.x * blockDim.x;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < d.n; j += stride) {
    const double x0 = fmin(fmax(0.0, v.l[j]), v.u[j]);
    v.x[0][j] = x0; v.x[1][j] = x0;
    v.xbar[0][j] = 0.0; v.xbar[1][j] = 0.0;
    v.T[j] = 1.0; v.invT[j] = 1.0; v.GT[j] = 0.0; v.q[j] = 0.0;
    v.x_last[j] = x0;
  }
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < d.m; i += stride) {
    v.y[0][i] = 0.0; v.y[1][i] = 0.0;
    v.ybar[0][i] = 0.0; v.ybar[1][i] = 0.0;
    v.S[i] = 1.0; v.invS[i] = 1.0; v.GS[i] = 0.0; v.p[i] = 0.0;
    v.y_last[i] = 0.0;
    v.ax_avg[i] = 0.0;
  }
}

// FP32 copies of the preprocessed matrix values and problem vectors.
__global__ void make_fp32_kernel(Dev d, long long nnz) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < nnz; k += stride) {
    d.f32.Av[k] = (float)d.f64.Av[k];
    d.f32.Atv[k] = (float)d.f64.Atv[k];
  }
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < d.m; i += stride) d.f32.b[i] = (float)d.f64.b[i];
  for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < d.n; j += stride) {
    d.f32.c[j] = (float)d.f64.c[j];
    d.f32.l[j] = (float)d.f64.l[j];
    d.f32.u[j] = (float)d.f64.u[j];
  }
}

// Copy the iteration state between the precisions: `up` = FP32 -> FP64
// (start of the refinement phase), else FP64 -> FP32.  Only the current half
// of the double buffers carries state; the other half is rewritten before use.
template <class S, class D>
__global__ void convert_state_kernel(Dev d, Vecs<S> src, Vecs<D> dst) {
  const int cur = d.st->cur;
  const int stride = gridDim.x * blockDim.x;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < d.n; j += stride) {
    dst.x[cur][j] = (D)src.x[cur][j];
    dst.xbar[cur][j] = (D)src.xbar[cur][j];
    dst.T[j] = (D)src.T[j];
    dst.invT[j] = D(1) / dst.T[j];
    dst.GT[j] = (D)src.GT[j];
    dst.q[j] = (D)src.q[j];
    dst.x_last[j] = (D)src.x_last[j];
  }
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < d.m; i += stride) {
    dst.y[cur][i] = (D)src.y[cur][i];
    dst.ybar[cur][i] = (D)src.ybar[cur][i];
    dst.ax[cur][i] = (D)src.ax[cur][i];
    dst.S[i] = (D)src.S[i];
    dst.invS[i] = D(1) / dst.S[i];
    dst.GS[i] = (D)src.GS[i];
    dst.p[i] = (D)src.p[i];
    dst.y_last[i] = (D)src.y_last[i];
    dst.ax_avg[i] = (D)src.ax_avg[i];
  }
}

// A x of the current iterate, recomputed in FP64 after a promotion.
struct StoreCurOp {
  double* y;
  __device__ __forceinline__ void prefetch(int) {}
  __device__ __forceinline__ void row(int r, const double (&s)[1]) { y[r] = s[0]; }
};

__global__ void __launch_bounds__(kBlock) recompute_ax_kernel(Dev d) {
  __shared__ double smem[32];
  const int cur = d.st->cur;
  StoreCurOp op{d.f64.ax[cur]};
  Gather<1, double> g;
  g.x[0] = d.f64.x[cur];
  g.n = d.n;
  g.bad = d.bad_gathers;
  for_each_row<1, double, double>(d.binsA, d.A, g, op, smem);
}

// Entry p of the sliced copy: in the kSell bin with the largest base <= p,
// off = p - base = slice * 32 len + 32 k + t is entry k of row slice * 32 + t
// of the bin; rows past the bin's end (padding of its last slice) get
// column 0 and value 0.
__global__ void fill_sliced_kernel(BinTable bt, const int* rp, const int* ci, const double* v, int* sell_ci,
                                   double* sell_v, long long total) {
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < total; p += (long long)gridDim.x * blockDim.x) {
    int b = -1;
    for (int q = 0; q < bt.nbins; ++q)
      if (bt.bin[q].width == kSell && bt.bin[q].base <= p) b = q;
    int c = 0;
    double x = 0.0;
    if (b >= 0) {
      const Bin& B = bt.bin[b];
      const long long off = p - B.base, per = 32LL * B.len;
      const long long slice = off / per;
      const int rem = (int)(off - slice * per);
      const long long row = B.row_begin + slice * 32 + (rem & 31);
      if (row < B.row_end) {
        const long long src = (long long)rp[row] + (rem >> 5);
        c = ci[src];
        x = v[src];
      }
    }
    sell_ci[p] = c;
    sell_v[p] = x;
  }
}

__global__ void narrow_kernel(const double* in, float* out, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = (float)in[i];
}

__global__ void widen_kernel(double* out, const float* in, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) out[i] = (double)in[i];
}

int grid_for(long long n) {
  long long g = (n + kBlock - 1) / kBlock;
  if (g > kSetupGrid) g = kSetupGrid;
  if (g < 1) g = 1;
  return (int)g;
}

int warp_grid_for(long long rows) {
  long long g = (rows * 32 + kBlock - 1) / kBlock;
  if (g > 4 * kSetupGrid) g = 4 * kSetupGrid;
  if (g < 1) g = 1;
  return (int)g;
}

}  // namespace

void launch_fill(double* v, double val, long long n, cudaStream_t s) {
  if (n > 0) fill_kernel<<<grid_for(n), kBlock, 0, s>>>(v, val, n);
}


void launch_row_powsum(const Csr& M, int rows, int nlong, int split, double beta, int square_root, double* out,
                       cudaStream_t s) {
  if (rows > 0)
    row_powsum_kernel<<<warp_grid_for(nlong + (split - nlong) + (rows - split + 3) / 4), kBlock, 0, s>>>(
        M, rows, nlong, split, beta, square_root, out);
}

namespace {
int ruiz_grid(const RuizRows& a, const RuizRows& at) {
  const long long units = a.units() + at.units();
  return warp_grid_for(units);
}
}  // namespace

void launch_ruiz_norms(const Dev& d, const RuizSplit& a, const RuizSplit& at, double* fr, double* fc, cudaStream_t s) {
  const RuizRows A{d.A_rp, d.A_ci, d.A_v, d.m, a}, At{d.At_rp, d.At_ci, d.At_v, d.n, at};
  // the chunked rows' maxima are combined by atomic max from zero
  if (a.nlong > 0) cudaMemsetAsync(fr, 0, sizeof(double) * a.nlong, s);
  if (at.nlong > 0) cudaMemsetAsync(fc, 0, sizeof(double) * at.nlong, s);
  ruiz_norms_kernel<<<ruiz_grid(A, At), kBlock, 0, s>>>(A, At, fr, fc);
}

void launch_ruiz_apply(const Dev& d, const RuizSplit& a, const RuizSplit& at, double* fr, double* fc, cudaStream_t s) {
  const RuizRows A{d.A_rp, d.A_ci, d.A_v, d.m, a}, At{d.At_rp, d.At_ci, d.At_v, d.n, at};
  factor_mul_kernel<<<grid_for((long long)d.m + d.n), kBlock, 0, s>>>(fr, d.dr, d.m, fc, d.dc, d.n);
  ruiz_scale_kernel<<<ruiz_grid(A, At), kBlock, 0, s>>>(A, At, fr, fc);
}

void launch_scale_problem_vectors(const Dev& d, cudaStream_t s) {
  scale_vectors_kernel<<<grid_for(d.n > d.m ? d.n : d.m), kBlock, 0, s>>>(d);
}

// out[0] = ||v||_2 ; uses out[1 .. 1 + kSetupGrid) as partials
void launch_norm2(const double* v, int n, double* out, cudaStream_t s) {
  const int g = grid_for(n);
  sumsq_partial_kernel<<<g, kBlock, 0, s>>>(v, n, out + 1);
  finish_kernel<<<1, kBlock, 0, s>>>(out + 1, g, out, 0);
}

void launch_absmax(const double* v, long long n, double* out, cudaStream_t s) {
  const int g = grid_for(n);
  absmax_partial_kernel<<<g, kBlock, 0, s>>>(v, n, out + 1);
  finish_kernel<<<1, kBlock, 0, s>>>(out + 1, g, out, 1);
}

void launch_scale_by_inv(double* v, int n, const double* denom, cudaStream_t s) {
  if (n > 0) scale_by_inv_kernel<<<grid_for(n), kBlock, 0, s>>>(v, n, denom);
}

void launch_spmv_binned(const Csr& M, const BinTable& bt, int grid, const double* x, double* y, cudaStream_t s) {
  if (bt.nunits > 0) spmv_kernel<<<grid, kBlock, 0, s>>>(M, bt, x, y);
}

void launch_init_vectors(const Dev& d, cudaStream_t s) {
  init_vectors_kernel<<<grid_for(d.n > d.m ? d.n : d.m), kBlock, 0, s>>>(d);
}

}  // namespace lpop

namespace lpop {

void launch_fill_sliced(const BinTable& bt, const int* rp, const int* ci, const double* v, int* sell_ci,
                        double* sell_v, long long total, cudaStream_t s) {
  if (total > 0) fill_sliced_kernel<<<grid_for(total), kBlock, 0, s>>>(bt, rp, ci, v, sell_ci, sell_v, total);
}

void launch_narrow(const double* in, float* out, long long n, cudaStream_t s) {
  if (n > 0) narrow_kernel<<<grid_for(n), kBlock, 0, s>>>(in, out, n);
}

void launch_make_fp32(const Dev& d, cudaStream_t s) {
  long long big = d.nnz > d.n ? d.nnz : d.n;
  if (d.m > big) big = d.m;
  make_fp32_kernel<<<grid_for(big), kBlock, 0, s>>>(d, d.nnz);
}

void launch_promote_state(const Dev& d, cudaStream_t s) {
  convert_state_kernel<float, double><<<grid_for(d.n > d.m ? d.n : d.m), kBlock, 0, s>>>(d, d.f32, d.f64);
  if (d.binsA.nunits > 0) recompute_ax_kernel<<<d.gridA, kBlock, 0, s>>>(d);
}

void launch_demote_state(const Dev& d, cudaStream_t s) {
  convert_state_kernel<double, float><<<grid_for(d.n > d.m ? d.n : d.m), kBlock, 0, s>>>(d, d.f64, d.f32);
}

void launch_widen(double* out, const float* in, int n, cudaStream_t s) {
  if (n > 0) widen_kernel<<<grid_for(n), kBlock, 0, s>>>(out, in, n);
}

}  // namespace lpop
