// Test program for the library's host-side layout code (csrc/host_layout.cpp):
// reads a CSR matrix from three raw files, runs build_layout (and optionally
// segment_long_rows on both bin tables, then set_sliced_unit_rows), and writes
// everything it produced to one raw file that tests/test_host_layout.py reads
// back and checks.
//
//   host_layout_runner m n nnz in_prefix out_path target_threads seg_len [sliced_rows]
//
// Input files: <in_prefix>rp.bin (int64 [m+1]), ci.bin (int32 [nnz]),
// v.bin (float64 [nnz]).  seg_len <= 0 skips the segmentation.  sliced_rows
// = -1 runs validate_csr alone and writes rc, the message and the canonical
// flag (int32 each, the message as its length and bytes).
#include <cstdio>
#include <cstdlib>
#include <string>
#include <vector>

#include "host_layout.hpp"

namespace {

template <class T>
std::vector<T> read_all(const std::string& path, size_t count) {
  std::vector<T> v(count);
  FILE* f = std::fopen(path.c_str(), "rb");
  if (!f) {
    std::fprintf(stderr, "cannot open %s\n", path.c_str());
    std::exit(2);
  }
  if (count && std::fread(v.data(), sizeof(T), count, f) != count) {
    std::fprintf(stderr, "short read from %s\n", path.c_str());
    std::exit(2);
  }
  std::fclose(f);
  return v;
}

template <class T>
void put(FILE* f, const T& x) {
  std::fwrite(&x, sizeof(T), 1, f);
}

template <class T>
void put_vec(FILE* f, const std::vector<T>& v) {
  put<long long>(f, (long long)v.size());
  if (!v.empty()) std::fwrite(v.data(), sizeof(T), v.size(), f);
}

void put_bins(FILE* f, const lpop::BinTable& bt) {
  put<int>(f, bt.nbins);
  put<int>(f, bt.nunits);
  put<int>(f, bt.seg_len);
  put<int>(f, bt.seg_rows);
  for (int b = 0; b < bt.nbins; ++b) {
    const lpop::Bin& x = bt.bin[b];
    put<long long>(f, x.row_begin);
    put<long long>(f, x.row_end);
    put<long long>(f, x.width);
    put<long long>(f, x.unit_begin);
    put<long long>(f, x.len);
    put<long long>(f, x.base);
  }
  put<long long>(f, lpop::sliced_entries(bt));
}

}  // namespace

int main(int argc, char** argv) {
  if (argc != 8 && argc != 9) {
    std::fprintf(stderr, "usage: %s m n nnz in_prefix out_path target_threads seg_len [sliced_rows]\n", argv[0]);
    return 2;
  }
  const int sliced_rows = argc == 9 ? std::atoi(argv[8]) : 0;
  const int m = std::atoi(argv[1]), n = std::atoi(argv[2]);
  const long long nnz = std::atoll(argv[3]);
  const std::string pre = argv[4];
  const long long target = std::atoll(argv[6]);
  const int seg_len = std::atoi(argv[7]);
  const auto rp = read_all<long long>(pre + "rp.bin", (size_t)m + 1);
  const auto ci = read_all<int>(pre + "ci.bin", (size_t)nnz);
  const auto v = read_all<double>(pre + "v.bin", (size_t)nnz);
  if (sliced_rows == -1) {
    bool canonical = false;
    std::string err;
    const int rc = lpop::validate_csr(m, n, nnz, reinterpret_cast<const int64_t*>(rp.data()), ci.data(), v.data(),
                                      canonical, err);
    FILE* o = std::fopen(argv[5], "wb");
    if (!o) return 2;
    put<int>(o, rc);
    put<int>(o, (int)err.size());
    std::fwrite(err.data(), 1, err.size(), o);
    put<int>(o, canonical ? 1 : 0);
    std::fclose(o);
    return 0;
  }

  lpop::HostLayout lay;
  std::string err;
  const int rc = lpop::build_layout(m, n, nnz, reinterpret_cast<const int64_t*>(rp.data()), ci.data(), v.data(), lay,
                                    err, target);
  std::vector<int> segA, segAt;
  if (rc == 0 && seg_len > 0) {
    segA = lpop::segment_long_rows(lay.binsA, lay.A_rp, seg_len);
    segAt = lpop::segment_long_rows(lay.binsAt, lay.At_rp, seg_len);
  }
  if (rc == 0 && sliced_rows > 0) {
    lpop::set_sliced_unit_rows(lay.binsA, sliced_rows);
    lpop::set_sliced_unit_rows(lay.binsAt, sliced_rows);
  }
  FILE* o = std::fopen(argv[5], "wb");
  if (!o) return 2;
  put<int>(o, rc);
  put<int>(o, (int)err.size());
  std::fwrite(err.data(), 1, err.size(), o);
  put<long long>(o, lay.nnz);
  put_vec(o, lay.prow);
  put_vec(o, lay.pcol);
  put_vec(o, lay.A_rp);
  put_vec(o, lay.A_ci);
  put_vec(o, lay.A_v);
  put_vec(o, lay.At_rp);
  put_vec(o, lay.At_ci);
  put_vec(o, lay.At_v);
  put_bins(o, lay.binsA);
  put_bins(o, lay.binsAt);
  put_vec(o, segA);
  put_vec(o, segAt);
  std::fclose(o);
  return 0;
}
