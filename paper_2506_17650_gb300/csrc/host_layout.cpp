#include "host_layout.hpp"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <numeric>
#include <thread>

#include "../../include/lpop.h"

namespace lpop {

namespace {

// Host threads for the layout's parallel phases: every hardware thread, up to 32.
int layout_threads() {
  const unsigned hw = std::thread::hardware_concurrency();
  return (int)std::min<unsigned>(hw == 0 ? 1u : hw, 32u);
}

// Run fn(begin, end) over [0, count) split into contiguous pieces, on the
// layout's host threads when the work (count by default; e.g. the entries of
// the rows when a range is rows) is large.
template <class Fn>
void parallel_ranges(long long count, Fn fn, long long work = -1) {
  int t = layout_threads();
  if ((work < 0 ? count : work) < (1 << 16)) t = 1;
  if (t <= 1) {
    fn(0LL, count);
    return;
  }
  std::vector<std::thread> pool;
  for (int i = 0; i < t; ++i) {
    const long long b = count * i / t, e = count * (i + 1) / t;
    pool.emplace_back([=]() { fn(b, e); });
  }
  for (auto& th : pool) th.join();
}

// Run fn(t) for t in [0, T) on T host threads (T = 1: inline).
template <class Fn>
void parallel_ranges_n(int T, Fn fn) {
  if (T <= 1) {
    fn(0);
    return;
  }
  std::vector<std::thread> pool;
  for (int t = 0; t < T; ++t) pool.emplace_back([=]() { fn(t); });
  for (auto& th : pool) th.join();
}

// Stable permutation of rows by bin rank, longest first within a bin.
std::vector<int> bin_permutation(const std::vector<long long>& len, std::vector<int>& widths_sorted,
                                 std::vector<int>& lengths_sorted, long long target_threads) {
  const int rows = (int)len.size();
  const int widen = widen_factor(rows, target_threads);
  std::vector<int> width(rows);
  for (int r = 0; r < rows; ++r) width[r] = width_for_length(len[r], widen);
  std::vector<int> perm(rows);
  // a warp's rows get similar lengths and the heaviest units come first.
  // Counting sort on (rank, length) for rows up to kCountMax entries; the few
  // longer rows (all in the whole-block bin) are sorted directly and go first.
  std::vector<int> longer;
  std::vector<long long> start(7 * (kCountMax + 1) + 1, 0);
  auto key = [&](int r) { return bin_rank(width[r]) * (kCountMax + 1) + (kCountMax - (int)len[r]); };
  for (int r = 0; r < rows; ++r) {
    if (len[r] > kCountMax) longer.push_back(r);
    else start[key(r) + 1]++;
  }
  std::stable_sort(longer.begin(), longer.end(), [&](int a, int b) { return len[a] > len[b]; });
  int pos = 0;
  for (int r : longer) perm[pos++] = r;
  start[0] = pos;
  for (size_t k = 1; k < start.size(); ++k) start[k] += start[k - 1];
  for (int r = 0; r < rows; ++r)
    if (len[r] <= kCountMax) perm[start[key(r)]++] = r;
  widths_sorted.resize(rows);
  lengths_sorted.resize(rows);
  for (int r = 0; r < rows; ++r) {
    widths_sorted[r] = width[perm[r]];
    lengths_sorted[r] = (int)len[perm[r]];
  }
  return perm;
}

}  // namespace

int widen_factor(long long rows, long long target_threads) {
  int f = 1;
  while (f < 8 && (long long)f * rows < target_threads) f <<= 1;
  return f;
}

BinTable bins_from_runs(const std::vector<BinRun>& runs) {
  BinTable t{};
  t.nbins = 0;
  t.nunits = 0;
  long long sell = 0;
  for (const BinRun& x : runs) {
    Bin& b = t.bin[t.nbins++];
    b.row_begin = x.row_begin;
    b.row_end = x.row_end;
    b.width = x.width;
    b.unit_begin = t.nunits;
    b.len = x.width == kSell ? x.len : 0;
    b.base = x.width == kSell ? sell : 0;
    if (x.width == kSell) sell += (long long)(x.row_end - x.row_begin + 31) / 32 * 32 * x.len;
    const int per = rows_per_unit(b);
    t.nunits += (x.row_end - x.row_begin + per - 1) / per;
  }
  return t;
}

BinTable make_bins(const std::vector<int>& widths_sorted, const std::vector<int>& lengths_sorted) {
  std::vector<BinRun> runs;
  const int rows = (int)widths_sorted.size();
  int r = 0;
  while (r < rows) {
    const int w = widths_sorted[r];
    // one-lane rows (at most kSellMaxLen entries) go to sliced bins of one exact length
    const bool sliced = w == 1 && !lengths_sorted.empty();
    int e = r;
    while (e < rows && widths_sorted[e] == w && (!sliced || lengths_sorted[e] == lengths_sorted[r])) ++e;
    runs.push_back(BinRun{r, e, sliced ? kSell : w, sliced ? lengths_sorted[r] : 0});
    r = e;
  }
  // at most kSellMaxLen + 1 sliced lengths and six other classes: within kMaxBins
  static_assert(kSellMaxLen + 1 + 6 + 1 <= kMaxBins, "bin table too small");
  return bins_from_runs(runs);
}

void set_sliced_unit_rows(BinTable& bt, int rows) {
  int unit = 0;
  for (int b = 0; b < bt.nbins; ++b) {
    Bin& x = bt.bin[b];
    const int old_count = (b + 1 < bt.nbins ? bt.bin[b + 1].unit_begin : bt.nunits) - x.unit_begin;
    if (x.width == kSell) x.unit_rows = rows == kBlock ? 0 : (x.len <= kPairMaxLen ? 2 * rows : rows);
    x.unit_begin = unit;
    if (x.width == kSegmented) {
      unit += old_count;
    } else {
      const int per = rows_per_unit(x);
      unit += (x.row_end - x.row_begin + per - 1) / per;
    }
  }
  bt.nunits = unit;
}

long long sliced_entries(const BinTable& bt) {
  long long total = 0;
  for (int b = 0; b < bt.nbins; ++b) {
    const Bin& x = bt.bin[b];
    if (x.width == kSell) total = x.base + (long long)(x.row_end - x.row_begin + 31) / 32 * 32 * x.len;
  }
  return total;
}

void for_each_range(long long count, const std::function<void(long long, long long)>& fn, long long work) {
  parallel_ranges(count, fn, work);
}

int validate_csr(int32_t m, int32_t n, int64_t nnz, const int64_t* row_ptr, const int32_t* col_idx,
                 const double* val, bool& canonical, std::string& err) {
  if (m < 0 || n < 1 || nnz < 0) {
    err = "need m >= 0, n >= 1 and nnz >= 0";
    return LP_ERR_INVALID_ARG;
  }
  if (nnz >= (int64_t)1 << 31) {
    err = "nnz must be below 2^31";
    return LP_ERR_INVALID_ARG;
  }
  if (!row_ptr || (nnz > 0 && (!col_idx || !val))) {
    err = "row_ptr, col_idx and val must not be NULL";
    return LP_ERR_INVALID_ARG;
  }
  if (row_ptr[0] != 0 || row_ptr[m] != nnz) {
    err = "row_ptr[0] must be 0 and row_ptr[m] must equal nnz";
    return LP_ERR_INVALID_INPUT;
  }
  const long long dec = first_bad_index(m, [&](long long i) { return row_ptr[i + 1] < row_ptr[i]; });
  if (dec < m) {
    err = "row_ptr must be non-decreasing (row " + std::to_string(dec) + ")";
    return LP_ERR_INVALID_INPUT;
  }
  // entries (on host threads, by ranges of rows): the first one with a column
  // out of range or a value that is not finite, and whether every row is in
  // strictly increasing column order.  A range is first passed without
  // branches (columns and exponent bits tested, column descents counted, the
  // descents across row starts taken off again); only a range with a bad
  // entry is walked again for its first one.
  canonical = true;
  {
    std::mutex mu;
    int64_t bad = nnz;
    auto scan = [&](long long r0, long long r1) {
      const int64_t k0 = row_ptr[r0], k1 = row_ptr[r1];
      unsigned any_bad = 0;
      long long desc = 0;
      for (int64_t k = k0; k < k1; ++k) {
        uint64_t bits;
        std::memcpy(&bits, val + k, sizeof(bits));
        any_bad |= (unsigned)((uint32_t)col_idx[k] >= (uint32_t)n) |
                   (unsigned)((bits & 0x7ff0000000000000ULL) == 0x7ff0000000000000ULL);
      }
      for (int64_t k = k0 + 1; k < k1; ++k) desc += col_idx[k - 1] >= col_idx[k];
      for (long long i = r0 + 1; i < r1; ++i) {  // each distinct row start inside the range once
        const int64_t st = row_ptr[i];
        if (st > k0 && st < k1 && st != row_ptr[i - 1]) desc -= col_idx[st - 1] >= col_idx[st];
      }
      int64_t first_bad = nnz;
      for (int64_t k = k0; any_bad && k < k1; ++k) {
        if (col_idx[k] < 0 || col_idx[k] >= n || !std::isfinite(val[k])) {
          first_bad = k;
          break;
        }
      }
      std::lock_guard<std::mutex> lock(mu);
      bad = std::min(bad, first_bad);
      canonical = canonical && desc == 0;
    };
    parallel_ranges(m, scan, nnz);
    if (bad < nnz) {
      err = col_idx[bad] < 0 || col_idx[bad] >= n ? "col_idx[" + std::to_string(bad) + "] out of range"
                                                  : "val[" + std::to_string(bad) + "] is not finite";
      return LP_ERR_INVALID_INPUT;
    }
  }
  return LP_OK;
}

void merge_rows(int32_t m, const int64_t* row_ptr, const int32_t* col_idx, const double* val,
                std::vector<int64_t>& rp, std::vector<int>& ci, std::vector<double>& cv) {
  const int64_t nnz = row_ptr[m];
  rp.assign(m + 1, 0);
  struct Part {
    long long r0 = 0, r1 = 0;
    std::vector<int> ci;
    std::vector<double> cv;
    std::vector<int64_t> len;
  };
  const int T = nnz < (1 << 16) ? 1 : layout_threads();
  std::vector<Part> parts(T);
  for (int t = 0; t < T; ++t) {
    parts[t].r0 = (long long)m * t / T;
    parts[t].r1 = (long long)m * (t + 1) / T;
  }
  auto work = [&](Part& P) {
    std::vector<std::pair<int, double>> row;
    P.ci.reserve(row_ptr[P.r1] - row_ptr[P.r0]);
    P.cv.reserve(row_ptr[P.r1] - row_ptr[P.r0]);
    P.len.reserve(P.r1 - P.r0);
    for (long long i = P.r0; i < P.r1; ++i) {
      const size_t before = P.ci.size();
      bool sorted = true;
      for (int64_t k = row_ptr[i] + 1; k < row_ptr[i + 1]; ++k) sorted = sorted && col_idx[k - 1] < col_idx[k];
      if (sorted) {  // the common case: copy as is
        P.ci.insert(P.ci.end(), col_idx + row_ptr[i], col_idx + row_ptr[i + 1]);
        P.cv.insert(P.cv.end(), val + row_ptr[i], val + row_ptr[i + 1]);
      } else {
        row.clear();
        for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) row.emplace_back(col_idx[k], val[k]);
        std::stable_sort(row.begin(), row.end(), [](const auto& a, const auto& b) { return a.first < b.first; });
        for (size_t t = 0; t < row.size();) {
          const int c = row[t].first;
          double sum = row[t].second;
          size_t e = t + 1;
          while (e < row.size() && row[e].first == c) sum += row[e++].second;
          P.ci.push_back(c);
          P.cv.push_back(sum);
          t = e;
        }
      }
      P.len.push_back((int64_t)(P.ci.size() - before));
    }
  };
  if (T == 1) {
    work(parts[0]);
  } else {
    std::vector<std::thread> pool;
    for (int t = 0; t < T; ++t) pool.emplace_back([&, t]() { work(parts[t]); });
    for (auto& th : pool) th.join();
  }
  long long total = 0;
  for (const Part& P : parts) total += (long long)P.ci.size();
  ci.resize(total);
  cv.resize(total);
  long long off = 0;
  for (const Part& P : parts) {
    std::copy(P.ci.begin(), P.ci.end(), ci.begin() + off);
    std::copy(P.cv.begin(), P.cv.end(), cv.begin() + off);
    for (long long i = P.r0; i < P.r1; ++i) rp[i + 1] = rp[i] + P.len[i - P.r0];
    off += (long long)P.ci.size();
  }
}

int build_layout(int32_t m, int32_t n, int64_t nnz, const int64_t* row_ptr, const int32_t* col_idx,
                 const double* val, HostLayout& out, std::string& err, long long target_threads) {
  bool canonical = true;
  if (const int rc = validate_csr(m, n, nnz, row_ptr, col_idx, val, canonical, err)) return rc;
  // rows in strictly increasing column order (the common case) are used in
  // place; otherwise each row is sorted by column and repeated entries are
  // merged (summed)
  std::vector<int64_t> rp_m;
  std::vector<int> ci_m;
  std::vector<double> cv_m;
  if (!canonical) merge_rows(m, row_ptr, col_idx, val, rp_m, ci_m, cv_m);
  const int64_t* rp = canonical ? row_ptr : rp_m.data();
  const int32_t* ci = canonical ? col_idx : ci_m.data();
  const double* cv = canonical ? val : cv_m.data();
  const long long nz = canonical ? (long long)nnz : (long long)ci_m.size();

  // row and column orders (independent: the columns on a second thread)
  std::vector<long long> rlen(m), clen(n, 0);
  std::vector<int> wA, wAt, lA, lAt;
  out.m = m;
  out.n = n;
  out.nnz = nz;
  {
    auto columns = [&]() {
      // column lengths: ranges of entries on the layout's threads, relaxed atomic increments
      parallel_ranges(nz, [&](long long b, long long e) {
        for (long long k = b; k < e; ++k) __atomic_fetch_add(&clen[ci[k]], 1LL, __ATOMIC_RELAXED);
      });
      out.pcol = bin_permutation(clen, wAt, lAt, target_threads);
      out.binsAt = make_bins(wAt, lAt);
    };
    std::thread th;
    if (nz >= (1 << 16)) th = std::thread(columns);
    for (int i = 0; i < m; ++i) rlen[i] = rp[i + 1] - rp[i];
    out.prow = bin_permutation(rlen, wA, lA, target_threads);
    out.binsA = make_bins(wA, lA);
    if (th.joinable()) th.join();
    else columns();
  }
  std::vector<int> icol(n);
  for (int j = 0; j < n; ++j) icol[out.pcol[j]] = j;

  // permuted CSR of A, rows in bin order, column indices permuted and sorted
  out.A_rp.assign(m + 1, 0);
  for (int ip = 0; ip < m; ++ip) out.A_rp[ip + 1] = out.A_rp[ip] + (int)rlen[out.prow[ip]];
  out.A_ci.resize(nz);
  out.A_v.resize(nz);
  auto permute_rows = [&](long long b, long long e) {
    std::vector<std::pair<int, double>> tmp;
    for (long long ip = b; ip < e; ++ip) {
      const int i = out.prow[ip];
      const int64_t src = rp[i], len = rp[i + 1] - rp[i];
      const int dst = out.A_rp[ip];
      bool sorted = true;
      for (int64_t k = 0; k < len; ++k) {
        out.A_ci[dst + k] = icol[ci[src + k]];
        out.A_v[dst + k] = cv[src + k];
        if (k > 0 && out.A_ci[dst + k - 1] > out.A_ci[dst + k]) sorted = false;
      }
      if (!sorted) {
        tmp.clear();
        for (int64_t k = 0; k < len; ++k) tmp.emplace_back(out.A_ci[dst + k], out.A_v[dst + k]);
        std::sort(tmp.begin(), tmp.end(), [](const auto& x, const auto& y) { return x.first < y.first; });
        for (int64_t k = 0; k < len; ++k) {
          out.A_ci[dst + k] = tmp[k].first;
          out.A_v[dst + k] = tmp[k].second;
        }
      }
    }
  };
  parallel_ranges(m, permute_rows, nz);  // ranges of rows, sized by their entries

  // permuted CSR of A^T by counting sort (row indices come out sorted): rows
  // of A in T contiguous chunks, per-chunk column counts give every chunk its
  // own start in each column, so the chunks fill in parallel
  out.At_rp.assign(n + 1, 0);
  for (int j = 0; j < n; ++j) out.At_rp[j + 1] = out.At_rp[j] + (int)clen[out.pcol[j]];
  out.At_ci.resize(nz);
  out.At_v.resize(nz);
  {
    int T = nz < (1 << 17) ? 1 : layout_threads();
    while (T > 1 && (long long)T * n > (64LL << 20)) --T;  // bound the count table (256 MB)
    std::vector<int> fill((size_t)T * n);
    parallel_ranges_n(T, [&](int t) {
      int* f = fill.data() + (size_t)t * n;
      std::fill(f, f + n, 0);
      const long long r0 = (long long)m * t / T, r1 = (long long)m * (t + 1) / T;
      for (long long k = out.A_rp[r0]; k < out.A_rp[r1]; ++k) f[out.A_ci[k]]++;
    });
    parallel_ranges(n, [&](long long b, long long e) {
      for (long long j = b; j < e; ++j) {
        int at = out.At_rp[j];
        for (int t = 0; t < T; ++t) {
          int& f = fill[(size_t)t * n + j];
          const int c = f;
          f = at;
          at += c;
        }
      }
    });
    parallel_ranges_n(T, [&](int t) {
      int* f = fill.data() + (size_t)t * n;
      const long long r0 = (long long)m * t / T, r1 = (long long)m * (t + 1) / T;
      for (long long ip = r0; ip < r1; ++ip) {
        for (int k = out.A_rp[ip]; k < out.A_rp[ip + 1]; ++k) {
          const int j = out.A_ci[k];
          out.At_ci[f[j]] = (int)ip;
          out.At_v[f[j]] = out.A_v[k];
          f[j]++;
        }
      }
    });
  }
  return LP_OK;
}

}  // namespace lpop

namespace lpop {

int segment_length(long long nnz, int grid) {
  // a quarter of the mean work of a block, so that a long row spreads over at
  // least four blocks' worth of the grid and no unit holds much more than a
  // block's share (measured on the power-law LP against a half: FP32 primal
  // kernel 4% faster, FP64 1%); never below twice the whole-block threshold
  const long long per_block = grid > 0 ? nnz / grid : nnz;
  long long len = (per_block / 4 + 1023) / 1024 * 1024;
  if (len < 2 * kBlockRowThreshold) len = 2 * kBlockRowThreshold;
  if (len > (1LL << 30)) len = 1LL << 30;
  return (int)len;
}

std::vector<int> segment_long_rows(BinTable& bt, const std::vector<int>& rp, int seg_len) {
  std::vector<int> units;
  bt.seg_len = 0;
  bt.seg_rows = 0;
  if (bt.nbins == 0 || bt.bin[0].width != 0 || seg_len <= 0) return units;
  // rows of the whole-block bin are sorted longest first: the segmented rows are a prefix
  const Bin blk = bt.bin[0];
  int r = blk.row_begin;
  while (r < blk.row_end && rp[r + 1] - rp[r] > seg_len) {
    const int segs = (rp[r + 1] - rp[r] + seg_len - 1) / seg_len;
    for (int t = 0; t < segs; ++t) {
      units.push_back(r);
      units.push_back(t);
    }
    ++r;
  }
  const int rows = r - blk.row_begin;
  if (rows == 0 || bt.nbins + (r < blk.row_end ? 1 : 0) > kMaxBins) return std::vector<int>();
  const int nseg_units = (int)units.size() / 2;
  BinTable out = bt;
  out.nbins = 0;
  out.bin[out.nbins++] = Bin{blk.row_begin, r, kSegmented, 0, 0, 0, 0};
  int unit = nseg_units;
  if (r < blk.row_end) {
    out.bin[out.nbins++] = Bin{r, blk.row_end, 0, unit, 0, 0, 0};
    unit += blk.row_end - r;
  }
  for (int b = 1; b < bt.nbins; ++b) {
    Bin x = bt.bin[b];
    x.unit_begin = unit;
    const int per = rows_per_unit(x);
    unit += (x.row_end - x.row_begin + per - 1) / per;
    out.bin[out.nbins++] = x;
  }
  out.nunits = unit;
  out.seg_len = seg_len;
  out.seg_rows = rows;
  bt = out;
  return units;
}

}  // namespace lpop
