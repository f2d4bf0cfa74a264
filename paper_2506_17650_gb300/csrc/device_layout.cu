// Layout build on the device (see device_layout.hpp): lengths, bin orders,
// and the permuted CSR of A^T and of A by stable least-significant-digit
// radix sorts.  Every step is deterministic (no order decided by atomics), so
// the result equals the host's build_layout entry for entry.
#include "device_layout.hpp"

#include <algorithm>
#include <climits>
#include <type_traits>

#include "../../include/lpop.h"

namespace lpop {

namespace {

constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kSortItems = 16;                    // items per thread of one radix tile
constexpr int kTile = kSortThreads * kSortItems;  // items per tile (and per block of the scans)
constexpr int kMaxDigitBits = 8;
constexpr int kClassBounds = 6 + kSellMaxLen + 1;  // class boundaries of a bin order (see runs_from_bounds)

struct SortSet {
  unsigned* key;
  int* idx;
  double* val;  // null: no value payload
};

struct BoundKeys {
  unsigned k[64];
};

__device__ __forceinline__ unsigned warp_max(unsigned v) {
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xFFFFFFFFu, v, o));
  return v;
}

__device__ __forceinline__ unsigned warp_min(unsigned v) {
  for (int o = 16; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(0xFFFFFFFFu, v, o));
  return v;
}

__device__ __forceinline__ int warp_sum(int v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
  return v;
}

__device__ __forceinline__ int warp_inclusive_scan(int v, int lane) {
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xFFFFFFFFu, v, o);
    if (lane >= o) v += y;
  }
  return v;
}

// misc[0..1] longest row of A / A^T, [2..3] and [4..5] smallest and largest
// order key of A / A^T, [6..7] first row of A / A^T with at most 32 entries
__global__ void init_misc_kernel(unsigned* misc, int m, int n) {
  if (threadIdx.x == 0) {
    misc[0] = misc[1] = 0u;
    misc[2] = misc[4] = UINT_MAX;
    misc[3] = misc[5] = 0u;
    misc[6] = (unsigned)m;
    misc[7] = (unsigned)n;
  }
}

// len[i] = rp[i + 1] - rp[i] when rp is given (else len is read), and the
// largest length into *lmax
__global__ void lengths_kernel(const long long* __restrict__ rp, int* __restrict__ len, int rows, unsigned* lmax) {
  unsigned mx = 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < rows; i += (long long)gridDim.x * blockDim.x) {
    int l;
    if (rp) {
      l = (int)(rp[i + 1] - rp[i]);
      len[i] = l;
    } else {
      l = len[i];
    }
    mx = max(mx, (unsigned)l);
  }
  mx = warp_max(mx);
  if ((threadIdx.x & 31) == 0 && mx) atomicMax(lmax, mx);
}

__global__ void col_counts_kernel(const int* __restrict__ ci, long long nnz, int* __restrict__ clen) {
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < nnz; k += (long long)gridDim.x * blockDim.x)
    atomicAdd(&clen[ci[k]], 1);
}

// order key of every row, the identity as payload, and the key range into mm[0], mm[1]
__global__ void order_keys_kernel(const int* __restrict__ len, int rows, int widen, const unsigned* __restrict__ lmax,
                                  unsigned* __restrict__ key, int* __restrict__ idx, unsigned* mm) {
  const long long L = *lmax;
  unsigned lo = UINT_MAX, hi = 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < rows; i += (long long)gridDim.x * blockDim.x) {
    const unsigned k = order_key(len[i], widen, L);
    key[i] = k;
    idx[i] = (int)i;
    lo = min(lo, k);
    hi = max(hi, k);
  }
  lo = warp_min(lo);
  hi = warp_max(hi);
  if ((threadIdx.x & 31) == 0) {
    if (lo != UINT_MAX) atomicMin(&mm[0], lo);
    if (hi) atomicMax(&mm[1], hi);
  }
}

// Digit counts of one tile of kTile items: counts[d * ntiles + tile].
__global__ void __launch_bounds__(kSortThreads) radix_hist_kernel(const unsigned* __restrict__ key, long long N,
                                                                  unsigned kmin, int shift, int bits,
                                                                  int* __restrict__ counts, int ntiles) {
  __shared__ int c[1 << kMaxDigitBits];
  const int t = threadIdx.x, lane = t & 31;
  const int D = 1 << bits;
  c[t] = 0;
  __syncthreads();
  const long long t0 = (long long)blockIdx.x * kTile;
  for (int r = 0; r < kSortItems; ++r) {
    const long long i = t0 + (long long)r * kSortThreads + t;
    const bool act = i < N;
    const unsigned d = act ? ((key[i] - kmin) >> shift) & (unsigned)(D - 1) : 0xFFFFFFFFu;
    const unsigned peers = __match_any_sync(0xFFFFFFFFu, d);
    if (act && lane == __ffs(peers) - 1) atomicAdd(&c[d], __popc(peers));
  }
  __syncthreads();
  if (t < D) counts[(long long)t * ntiles + blockIdx.x] = c[t];
}

// Stable scatter of one tile: the tile's items in input order (round r,
// thread t holds item r * kSortThreads + t) go to offs[d * ntiles + tile] plus
// the number of earlier items of the tile with the same digit: earlier
// rounds (base), earlier warps of the round (wpre) and lower lanes (rank).
template <bool kVal>
__global__ void __launch_bounds__(kSortThreads) radix_scatter_kernel(SortSet src, SortSet dst, long long N,
                                                                     unsigned kmin, int shift, int bits,
                                                                     int write_keys, const int* __restrict__ offs,
                                                                     int ntiles) {
  __shared__ int base[1 << kMaxDigitBits];
  __shared__ int wcnt[kSortWarps][1 << kMaxDigitBits];
  __shared__ int wpre[kSortWarps][1 << kMaxDigitBits];
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  const int D = 1 << bits;
  const unsigned mask = (unsigned)D - 1u;
  base[t] = t < D ? offs[(long long)t * ntiles + blockIdx.x] : 0;
  for (int q = 0; q < kSortWarps; ++q) wcnt[q][t] = 0;
  __syncthreads();
  const long long t0 = (long long)blockIdx.x * kTile;
  const unsigned lower = (1u << lane) - 1u;
  for (int r = 0; r < kSortItems; ++r) {
    const long long i = t0 + (long long)r * kSortThreads + t;
    const bool act = i < N;
    unsigned k = 0, d = 0xFFFFFFFFu;
    int x = 0;
    double v = 0.0;
    if (act) {
      k = src.key[i];
      x = src.idx[i];
      if (kVal) v = src.val[i];
      d = ((k - kmin) >> shift) & mask;
    }
    const unsigned peers = __match_any_sync(0xFFFFFFFFu, d);
    const int rank = __popc(peers & lower);
    if (act && rank == 0) wcnt[w][d] = __popc(peers);
    __syncthreads();
    if (t < D) {
      int acc = base[t];
      for (int q = 0; q < kSortWarps; ++q) {
        const int c = wcnt[q][t];
        wpre[q][t] = acc;
        acc += c;
        wcnt[q][t] = 0;
      }
      base[t] = acc;
    }
    __syncthreads();
    if (act) {
      const int pos = wpre[w][d] + rank;
      if (write_keys) dst.key[pos] = k;
      dst.idx[pos] = x;
      if (kVal) dst.val[pos] = v;
    }
  }
}

// Scans: sums of chunks of kTile elements, an exclusive scan of those sums in
// one block, then each chunk scanned with its offset.
__global__ void __launch_bounds__(kSortThreads) scan_sums_kernel(const int* __restrict__ a, long long count,
                                                                 int* __restrict__ sums) {
  __shared__ int ws[kSortWarps];
  const long long c0 = (long long)blockIdx.x * kTile;
  int s = 0;
  for (int r = 0; r < kSortItems; ++r) {
    const long long i = c0 + (long long)r * kSortThreads + threadIdx.x;
    if (i < count) s += a[i];
  }
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    int v = threadIdx.x < kSortWarps ? ws[threadIdx.x] : 0;
    v = warp_sum(v);
    if (threadIdx.x == 0) sums[blockIdx.x] = v;
  }
}

__global__ void __launch_bounds__(1024) scan_top_kernel(int* sums, int parts) {
  __shared__ int wt[32];
  __shared__ int carry;
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  if (t == 0) carry = 0;
  __syncthreads();
  for (int b = 0; b < parts; b += 1024) {
    const int i = b + t;
    const int v = i < parts ? sums[i] : 0;
    const int x = warp_inclusive_scan(v, lane);
    if (lane == 31) wt[w] = x;
    __syncthreads();
    if (w == 0) wt[lane] = warp_inclusive_scan(wt[lane], lane);
    __syncthreads();
    const int excl = carry + (w > 0 ? wt[w - 1] : 0) + x - v;
    if (i < parts) sums[i] = excl;
    __syncthreads();
    if (t == 1023) carry = excl + v;
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kSortThreads) scan_apply_kernel(int* __restrict__ a, long long count,
                                                                  const int* __restrict__ sums) {
  // padded so that thread t's run of kSortItems consecutive elements is conflict-free
  __shared__ int s[kTile + kTile / 32];
  __shared__ int wt[kSortWarps];
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  auto P = [](int i) { return i + (i >> 5); };
  const long long c0 = (long long)blockIdx.x * kTile;
  for (int r = 0; r < kSortItems; ++r) {
    const int i = r * kSortThreads + t;
    s[P(i)] = c0 + i < count ? a[c0 + i] : 0;
  }
  __syncthreads();
  int tot = 0;
  for (int k = 0; k < kSortItems; ++k) tot += s[P(t * kSortItems + k)];
  const int x = warp_inclusive_scan(tot, lane);
  if (lane == 31) wt[w] = x;
  __syncthreads();
  if (w == 0) {
    const int y = warp_inclusive_scan(lane < kSortWarps ? wt[lane] : 0, lane);
    __syncwarp();
    if (lane < kSortWarps) wt[lane] = y;
  }
  __syncthreads();
  int run = sums[blockIdx.x] + (w > 0 ? wt[w - 1] : 0) + x - tot;
  for (int k = 0; k < kSortItems; ++k) {
    const int q = P(t * kSortItems + k);
    const int v = s[q];
    s[q] = run;
    run += v;
  }
  __syncthreads();
  for (int r = 0; r < kSortItems; ++r) {
    const int i = r * kSortThreads + t;
    if (c0 + i < count) a[c0 + i] = s[P(i)];
  }
}

__global__ void inverse_kernel(const int* __restrict__ perm, int rows, int* __restrict__ inv) {
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < rows; p += (long long)gridDim.x * blockDim.x)
    inv[perm[p]] = (int)p;
}

// out[p] = len[perm[p]] for p < rows, out[rows] = 0 (an exclusive scan then gives row pointers)
__global__ void perm_lengths_kernel(const int* __restrict__ perm, const int* __restrict__ len, int rows,
                                    int* __restrict__ out) {
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < rows; p += (long long)gridDim.x * blockDim.x)
    out[p] = len[perm[p]];
  if (blockIdx.x == 0 && threadIdx.x == 0) out[rows] = 0;
}

// Entries of A in permuted-row order, one warp per row: key = permuted
// column, payload = permuted row and value.
__global__ void gather_entries_kernel(int m, const int* __restrict__ prow, const long long* __restrict__ rp,
                                      const int* __restrict__ ci, const double* __restrict__ v,
                                      const int* __restrict__ icol, const int* __restrict__ A_rp,
                                      unsigned* __restrict__ kout, int* __restrict__ iout, double* __restrict__ vout) {
  const int lane = threadIdx.x & 31;
  const long long warps = (long long)gridDim.x * blockDim.x / 32;
  for (long long ip = (blockIdx.x * (long long)blockDim.x + threadIdx.x) / 32; ip < m; ip += warps) {
    const int i = prow[ip];
    const long long src = rp[i];
    const int len = (int)(rp[i + 1] - src);
    const int dst = A_rp[ip];
    for (int k = lane; k < len; k += 32) {
      kout[dst + k] = (unsigned)icol[ci[src + k]];
      iout[dst + k] = (int)ip;
      vout[dst + k] = v[src + k];
    }
  }
}

// pos[c] = first position whose key is >= K.k[c] in the sorted keys
__global__ void bounds_kernel(const unsigned* __restrict__ sorted, int rows, BoundKeys K, int nk, int* __restrict__ pos) {
  const int c = threadIdx.x;
  if (c >= nk) return;
  const unsigned key = K.k[c];
  int lo = 0, hi = rows;
  while (lo < hi) {
    const int mid = (int)(((unsigned)lo + (unsigned)hi) >> 1);
    if (sorted[mid] < key) lo = mid + 1;
    else hi = mid;
  }
  pos[c] = lo;
}

// first row with at most 32 entries into *out (initialised to the row count)
__global__ void split_kernel(const int* __restrict__ rp, int rows, unsigned* out) {
  unsigned first = UINT_MAX;
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < rows; r += (long long)gridDim.x * blockDim.x)
    if (rp[r + 1] - rp[r] <= 32) first = min(first, (unsigned)r);
  first = warp_min(first);
  if ((threadIdx.x & 31) == 0 && first != UINT_MAX) atomicMin(out, first);
}

__global__ void permute_vectors_kernel(int m, int n, const int* __restrict__ prow, const int* __restrict__ pcol,
                                       const double* __restrict__ b, const char* __restrict__ sense,
                                       const double* __restrict__ c, const double* __restrict__ lb,
                                       const double* __restrict__ ub, double* __restrict__ db,
                                       uint8_t* __restrict__ ds, double* __restrict__ dc, double* __restrict__ dl,
                                       double* __restrict__ du) {
  const int rows = m > n ? m : n;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < rows; i += (long long)gridDim.x * blockDim.x) {
    if (i < m) {
      const int r = prow[i];
      db[i] = b[r];
      const char s = sense[r];
      ds[i] = s == 'E' ? kEq : (s == 'L' ? kLe : kGe);
    }
    if (i < n) {
      const int j = pcol[i];
      dc[i] = c[j];
      dl[i] = lb[j];
      du[i] = ub[j];
    }
  }
}

int bit_length(unsigned long long x) {
  int b = 0;
  while (x) {
    ++b;
    x >>= 1;
  }
  return b;
}

// An odd number of passes of at most kMaxDigitBits bits each (odd, so that a
// ping-pong from set 0 ends in set 1).
int odd_passes(int bits) {
  int p = (bits + kMaxDigitBits - 1) / kMaxDigitBits;
  if (p < 1) p = 1;
  if (p % 2 == 0) ++p;
  return p;
}

int grid_for(long long work, int per_block = 256) {
  long long g = (work + per_block - 1) / per_block;
  if (g > 4096) g = 4096;
  if (g < 1) g = 1;
  return (int)g;
}

void exclusive_scan(int* a, long long count, int* sums, cudaStream_t s) {
  const long long parts = (count + kTile - 1) / kTile;
  if (parts < 1) return;
  scan_sums_kernel<<<(unsigned)parts, kSortThreads, 0, s>>>(a, count, sums);
  scan_top_kernel<<<1, 1024, 0, s>>>(sums, (int)parts);
  scan_apply_kernel<<<(unsigned)parts, kSortThreads, 0, s>>>(a, count, sums);
}

void radix_pass(const SortSet& src, const SortSet& dst, long long N, unsigned kmin, int shift, int bits,
                bool write_keys, int* counts, int* sums, cudaStream_t s) {
  const int ntiles = (int)((N + kTile - 1) / kTile);
  radix_hist_kernel<<<ntiles, kSortThreads, 0, s>>>(src.key, N, kmin, shift, bits, counts, ntiles);
  exclusive_scan(counts, (long long)ntiles << bits, sums, s);
  if (src.val)
    radix_scatter_kernel<true><<<ntiles, kSortThreads, 0, s>>>(src, dst, N, kmin, shift, bits, write_keys ? 1 : 0,
                                                                counts, ntiles);
  else
    radix_scatter_kernel<false><<<ntiles, kSortThreads, 0, s>>>(src, dst, N, kmin, shift, bits, write_keys ? 1 : 0,
                                                                 counts, ntiles);
}

// Stable sort of N items by the `bits` low bits of key - kmin, in an odd
// number of passes alternating a -> b -> a ... -> b (the result is in b).
void radix_sort_pingpong(const SortSet& a, const SortSet& b, long long N, unsigned kmin, int bits, int* counts,
                         int* sums, cudaStream_t s) {
  const int p = odd_passes(bits);
  const int w = (bits + p - 1) / p;
  for (int k = 0; k < p; ++k) radix_pass(k % 2 ? b : a, k % 2 ? a : b, N, kmin, k * w, w > 0 ? w : 1, true, counts, sums, s);
}

// Class boundaries of a bin order: the first row with a key >= each of
// (rank r + 1) * (kCountMax + 1) + base for r < 6 (the ends of the classes
// of width 0, 32, 16, 8, 4, 2), then the ends of the one-lane rows of length
// kSellMaxLen, kSellMaxLen - 1, ..., 0.
BoundKeys class_bound_keys(unsigned lmax) {
  BoundKeys K{};
  const long long base = (lmax > (unsigned)kCountMax ? (long long)lmax : kCountMax) - kCountMax;
  for (int r = 0; r < 6; ++r) K.k[r] = (unsigned)(base + (long long)(r + 1) * (kCountMax + 1));
  for (int l = kSellMaxLen; l >= 0; --l)
    K.k[6 + (kSellMaxLen - l)] = (unsigned)(base + 6LL * (kCountMax + 1) + (kCountMax - l) + 1);
  return K;
}

std::vector<BinRun> runs_from_bounds(const int* pos) {
  static const int kWidth[6] = {0, 32, 16, 8, 4, 2};
  std::vector<BinRun> runs;
  int begin = 0;
  for (int k = 0; k < kClassBounds; ++k) {
    const int end = pos[k];
    if (end > begin) {
      if (k < 6) runs.push_back(BinRun{begin, end, kWidth[k], 0});
      else runs.push_back(BinRun{begin, end, kSell, kSellMaxLen - (k - 6)});
    }
    begin = end > begin ? end : begin;
  }
  return runs;
}

}  // namespace

int build_layout_device(int32_t m, int32_t n, int64_t nnz, const int64_t* row_ptr, const int32_t* col_idx,
                        const double* val, int widen_a, int widen_at, const LayoutArrays& out,
                        const LayoutVectors* vec, LayoutInfo& info, const ScratchAlloc& alloc, cudaStream_t s,
                        std::string& err) {
  static_assert(kClassBounds <= 64, "class boundaries exceed the key table");
  static_assert(kSortThreads == (1 << kMaxDigitBits), "one thread per digit in the radix kernels");
#define CKD(call)                                                                              \
  do {                                                                                         \
    cudaError_t e_ = (call);                                                                   \
    if (e_ != cudaSuccess) {                                                                   \
      err = std::string(#call) + " failed: " + cudaGetErrorString(e_);                         \
      return e_ == cudaErrorMemoryAllocation ? LP_ERR_OOM : LP_ERR_CUDA;                       \
    }                                                                                          \
  } while (0)
#define TRYD(x)                   \
  do {                            \
    const int rc_ = (x);          \
    if (rc_ != LP_OK) return rc_; \
  } while (0)
  auto get = [&](auto** ptr, long long count) -> int {
    using T = std::remove_pointer_t<std::remove_pointer_t<decltype(ptr)>>;
    size_t bytes = (size_t)(count < 1 ? 1 : count) * sizeof(T);
    void* v = nullptr;
    const int rc = alloc(&v, bytes < 8 ? 8 : bytes);
    if (rc != LP_OK) {
      err = "layout scratch of " + std::to_string(bytes) + " bytes: allocation failed";
      return rc;
    }
    *ptr = static_cast<T*>(v);
    return LP_OK;
  };
  const long long nz = nnz;
  const int rows_max = m > n ? m : n;
  const long long sort_max = nz > rows_max ? nz : rows_max;
  const long long tiles_max = (sort_max + kTile - 1) / kTile;
  const long long scan_max = std::max<long long>(tiles_max << kMaxDigitBits, (long long)rows_max + 1);

  long long* d_rp = nullptr;
  int *rlen = nullptr, *clen = nullptr, *icol = nullptr, *counts = nullptr, *sums = nullptr, *pos = nullptr;
  unsigned *keyA[2] = {nullptr, nullptr}, *keyT[2] = {nullptr, nullptr}, *misc = nullptr;
  int *idxA[2] = {nullptr, nullptr}, *idxT[2] = {nullptr, nullptr};
  unsigned *Kp = nullptr, *Kq = nullptr, *Kr = nullptr;
  int* Ir = nullptr;
  double* Vr = nullptr;
  TRYD(get(&d_rp, (long long)m + 1));
  TRYD(get(&rlen, m));
  TRYD(get(&clen, n));
  TRYD(get(&icol, n));
  for (int k = 0; k < 2; ++k) {  // the sorted permutations end in idxA[1] / idxT[1]
    TRYD(get(&keyA[k], m));
    TRYD(get(&keyT[k], n));
    if (k == 1 && out.prow) idxA[1] = out.prow;
    else TRYD(get(&idxA[k], m));
    if (k == 1 && out.pcol) idxT[1] = out.pcol;
    else TRYD(get(&idxT[k], n));
  }
  TRYD(get(&Kp, nz));
  TRYD(get(&Kq, nz));
  TRYD(get(&Kr, nz));
  TRYD(get(&Ir, nz));
  TRYD(get(&Vr, nz));
  TRYD(get(&counts, scan_max));
  TRYD(get(&sums, (scan_max + kTile - 1) / kTile));
  TRYD(get(&misc, 16));
  TRYD(get(&pos, 128));
  double *rb = nullptr, *rc = nullptr, *rl = nullptr, *ru = nullptr;
  char* rs = nullptr;
  if (vec) {
    TRYD(get(&rb, m));
    TRYD(get(&rs, m));
    TRYD(get(&rc, n));
    TRYD(get(&rl, n));
    TRYD(get(&ru, n));
  }

  // the caller's arrays, once; the raw entries sit in the A^T arrays until the gather has read them
  CKD(cudaMemcpyAsync(d_rp, row_ptr, sizeof(long long) * ((size_t)m + 1), cudaMemcpyHostToDevice, s));
  if (nz > 0) {
    CKD(cudaMemcpyAsync(out.At_ci, col_idx, sizeof(int) * (size_t)nz, cudaMemcpyHostToDevice, s));
    CKD(cudaMemcpyAsync(out.At_v, val, sizeof(double) * (size_t)nz, cudaMemcpyHostToDevice, s));
  }
  if (vec) {
    if (m > 0) {
      CKD(cudaMemcpyAsync(rb, vec->b, sizeof(double) * m, cudaMemcpyHostToDevice, s));
      CKD(cudaMemcpyAsync(rs, vec->sense, m, cudaMemcpyHostToDevice, s));
    }
    CKD(cudaMemcpyAsync(rc, vec->c, sizeof(double) * n, cudaMemcpyHostToDevice, s));
    CKD(cudaMemcpyAsync(rl, vec->lb, sizeof(double) * n, cudaMemcpyHostToDevice, s));
    CKD(cudaMemcpyAsync(ru, vec->ub, sizeof(double) * n, cudaMemcpyHostToDevice, s));
  }

  // lengths, longest rows, order keys and their ranges
  init_misc_kernel<<<1, 32, 0, s>>>(misc, m, n);
  CKD(cudaMemsetAsync(clen, 0, sizeof(int) * (size_t)n, s));
  if (m > 0) lengths_kernel<<<grid_for(m), 256, 0, s>>>(d_rp, rlen, m, &misc[0]);
  if (nz > 0) col_counts_kernel<<<grid_for(nz), 256, 0, s>>>(out.At_ci, nz, clen);
  lengths_kernel<<<grid_for(n), 256, 0, s>>>(nullptr, clen, n, &misc[1]);
  if (m > 0) order_keys_kernel<<<grid_for(m), 256, 0, s>>>(rlen, m, widen_a, &misc[0], keyA[0], idxA[0], &misc[2]);
  order_keys_kernel<<<grid_for(n), 256, 0, s>>>(clen, n, widen_at, &misc[1], keyT[0], idxT[0], &misc[4]);
  CKD(cudaGetLastError());
  unsigned hm[8];
  CKD(cudaMemcpyAsync(hm, misc, sizeof(hm), cudaMemcpyDeviceToHost, s));
  CKD(cudaStreamSynchronize(s));

  // bin orders of the rows of A and of A^T
  if (m > 0)
    radix_sort_pingpong(SortSet{keyA[0], idxA[0], nullptr}, SortSet{keyA[1], idxA[1], nullptr}, m, hm[2],
                        bit_length(hm[3] - hm[2]), counts, sums, s);
  radix_sort_pingpong(SortSet{keyT[0], idxT[0], nullptr}, SortSet{keyT[1], idxT[1], nullptr}, n, hm[4],
                      bit_length(hm[5] - hm[4]), counts, sums, s);
  const int* prow = idxA[1];
  const int* pcol = idxT[1];
  inverse_kernel<<<grid_for(n), 256, 0, s>>>(pcol, n, icol);
  perm_lengths_kernel<<<grid_for(m), 256, 0, s>>>(prow, rlen, m, out.A_rp);
  exclusive_scan(out.A_rp, (long long)m + 1, sums, s);
  perm_lengths_kernel<<<grid_for(n), 256, 0, s>>>(pcol, clen, n, out.At_rp);
  exclusive_scan(out.At_rp, (long long)n + 1, sums, s);

  if (nz > 0) {
    // entries in permuted-row order keyed by permuted column; a stable sort by
    // column gives A^T with increasing row indices, and a stable sort of that
    // by row gives A with increasing column indices
    const SortSet P{Kp, out.A_ci, out.A_v};
    const SortSet Q{Kq, out.At_ci, out.At_v};
    gather_entries_kernel<<<grid_for((long long)m * 32), 256, 0, s>>>(m, prow, d_rp, out.At_ci, out.At_v, icol,
                                                                     out.A_rp, Kp, out.A_ci, out.A_v);
    radix_sort_pingpong(P, Q, nz, 0u, bit_length((unsigned)(n - 1)), counts, sums, s);
    // by row: Q (rows as keys, columns as payload) -> S -> R -> S ...
    const SortSet Qr{reinterpret_cast<unsigned*>(out.At_ci), reinterpret_cast<int*>(Kq), out.At_v};
    const SortSet S{Kp, out.A_ci, out.A_v};
    const SortSet R{Kr, Ir, Vr};
    const int bits = bit_length((unsigned)(m - 1));
    const int p = odd_passes(bits);
    const int w = bits > 0 ? (bits + p - 1) / p : 1;
    for (int k = 0; k < p; ++k) {
      const SortSet& from = k == 0 ? Qr : (k % 2 ? S : R);
      const SortSet& to = k % 2 ? R : S;
      radix_pass(from, to, nz, 0u, k * w, w, k + 1 < p, counts, sums, s);
    }
  }
  if (vec)
    permute_vectors_kernel<<<grid_for(rows_max), 256, 0, s>>>(m, n, prow, pcol, rb, rs, rc, rl, ru, vec->d_b,
                                                              vec->d_sense, vec->d_c, vec->d_l, vec->d_u);

  // class boundaries and the first rows of at most 32 entries
  if (m > 0) bounds_kernel<<<1, 64, 0, s>>>(keyA[1], m, class_bound_keys(hm[0]), kClassBounds, pos);
  bounds_kernel<<<1, 64, 0, s>>>(keyT[1], n, class_bound_keys(hm[1]), kClassBounds, pos + 64);
  split_kernel<<<grid_for(m), 256, 0, s>>>(out.A_rp, m, &misc[6]);
  split_kernel<<<grid_for(n), 256, 0, s>>>(out.At_rp, n, &misc[7]);
  CKD(cudaGetLastError());
  info.prow.assign((size_t)m, 0);
  info.pcol.assign((size_t)n, 0);
  int hpos[128] = {0};
  if (m > 0) CKD(cudaMemcpyAsync(info.prow.data(), prow, sizeof(int) * (size_t)m, cudaMemcpyDeviceToHost, s));
  CKD(cudaMemcpyAsync(info.pcol.data(), pcol, sizeof(int) * (size_t)n, cudaMemcpyDeviceToHost, s));
  CKD(cudaMemcpyAsync(hpos, pos, sizeof(hpos), cudaMemcpyDeviceToHost, s));
  CKD(cudaMemcpyAsync(hm, misc, sizeof(hm), cudaMemcpyDeviceToHost, s));
  CKD(cudaStreamSynchronize(s));
  info.split[0] = (int)hm[6];
  info.split[1] = (int)hm[7];
  info.binsA = m > 0 ? bins_from_runs(runs_from_bounds(hpos)) : bins_from_runs({});
  info.binsAt = bins_from_runs(runs_from_bounds(hpos + 64));

  // row pointers of the whole-block rows (the rows segmentation may cut)
  for (int which = 0; which < 2; ++which) {
    const BinTable& bt = which ? info.binsAt : info.binsA;
    std::vector<int>& head = which ? info.At_head : info.A_head;
    head.clear();
    if (bt.nbins == 0 || bt.bin[0].width != 0) continue;
    head.assign((size_t)bt.bin[0].row_end + 1, 0);
    CKD(cudaMemcpyAsync(head.data(), which ? out.At_rp : out.A_rp, sizeof(int) * head.size(), cudaMemcpyDeviceToHost,
                        s));
  }
  CKD(cudaStreamSynchronize(s));
  return LP_OK;
#undef CKD
#undef TRYD
}

}  // namespace lpop
