// Test program for the library's device-side layout build
// (csrc/device_layout.cu): reads a CSR matrix from the three raw files that
// tests/host_layout_runner.cpp reads, validates (and if needed merges) it as
// lp_create does, builds the layout on the device, and writes what it
// produced in the host runner's format, followed by the first rows of at
// most 32 entries and the permuted copies of index-derived vectors:
//
//   device_layout_runner m n nnz in_prefix out_path target_threads seg_len
//
// so that tests/test_gpu_device_layout.py can compare the two byte for byte.
#include <cuda_runtime.h>

#include <cstdio>
#include <cstdlib>
#include <string>
#include <vector>

#include "device_layout.hpp"
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

template <class T>
std::vector<T> down(const T* d, size_t count) {
  std::vector<T> h(count);
  if (count && cudaMemcpy(h.data(), d, sizeof(T) * count, cudaMemcpyDeviceToHost) != cudaSuccess) {
    std::fprintf(stderr, "copy back failed\n");
    std::exit(3);
  }
  return h;
}

template <class T>
T* dev(size_t count, std::vector<void*>& owned) {
  void* p = nullptr;
  if (cudaMalloc(&p, sizeof(T) * (count < 1 ? 1 : count)) != cudaSuccess) {
    std::fprintf(stderr, "cudaMalloc failed\n");
    std::exit(3);
  }
  owned.push_back(p);
  return static_cast<T*>(p);
}

}  // namespace

int main(int argc, char** argv) {
  if (argc != 8) {
    std::fprintf(stderr, "usage: %s m n nnz in_prefix out_path target_threads seg_len\n", argv[0]);
    return 2;
  }
  const int m = std::atoi(argv[1]), n = std::atoi(argv[2]);
  const long long nnz = std::atoll(argv[3]);
  const std::string pre = argv[4];
  const long long target = std::atoll(argv[6]);
  const int seg_len = std::atoi(argv[7]);
  const auto rp0 = read_all<long long>(pre + "rp.bin", (size_t)m + 1);
  const auto ci0 = read_all<int>(pre + "ci.bin", (size_t)nnz);
  const auto v0 = read_all<double>(pre + "v.bin", (size_t)nnz);

  bool canonical = true;
  std::string err;
  int rc = lpop::validate_csr(m, n, nnz, reinterpret_cast<const int64_t*>(rp0.data()), ci0.data(), v0.data(), canonical,
                              err);
  std::vector<int64_t> rp_m;
  std::vector<int> ci_m;
  std::vector<double> cv_m;
  if (rc == 0 && !canonical)
    lpop::merge_rows(m, reinterpret_cast<const int64_t*>(rp0.data()), ci0.data(), v0.data(), rp_m, ci_m, cv_m);
  const int64_t* rp = canonical ? reinterpret_cast<const int64_t*>(rp0.data()) : rp_m.data();
  const int* ci = canonical ? ci0.data() : ci_m.data();
  const double* cv = canonical ? v0.data() : cv_m.data();
  const long long nz = rc != 0 ? 0 : (canonical ? nnz : (long long)ci_m.size());

  std::vector<double> b(m), c(n), lb(n), ub(n);
  std::vector<char> sense(m);
  for (int i = 0; i < m; ++i) {
    b[i] = i + 0.5;
    sense[i] = "ELG"[i % 3];
  }
  for (int j = 0; j < n; ++j) {
    c[j] = -1.0 - j;
    lb[j] = 2.0 * j;
    ub[j] = 2.0 * j + 1.0;
  }

  std::vector<void*> owned;
  lpop::LayoutArrays arr{dev<int>((size_t)m + 1, owned), dev<int>(nz, owned), dev<double>(nz, owned),
                         dev<int>((size_t)n + 1, owned), dev<int>(nz, owned), dev<double>(nz, owned),
                         dev<int>(m, owned), dev<int>(n, owned)};
  lpop::LayoutVectors vec{b.data(), c.data(), lb.data(), ub.data(), sense.data(),
                          dev<double>(m, owned), dev<double>(n, owned), dev<double>(n, owned),
                          dev<double>(n, owned), dev<uint8_t>(m, owned)};
  lpop::LayoutInfo info;
  cudaStream_t s = nullptr;
  if (cudaStreamCreate(&s) != cudaSuccess) return 3;
  std::vector<void*> scratch;
  const lpop::ScratchAlloc alloc = [&scratch](void** ptr, size_t bytes) {
    *ptr = nullptr;
    if (cudaMalloc(ptr, bytes) != cudaSuccess) return -3;
    scratch.push_back(*ptr);
    return 0;
  };
  if (rc == 0)
    rc = lpop::build_layout_device(m, n, nz, rp, ci, cv, lpop::widen_factor(m, target), lpop::widen_factor(n, target),
                                   arr, &vec, info, alloc, s, err);
  for (void* q : scratch) cudaFree(q);

  std::vector<int> segA, segAt;
  if (rc == 0 && seg_len > 0) {
    segA = lpop::segment_long_rows(info.binsA, info.A_head, seg_len);
    segAt = lpop::segment_long_rows(info.binsAt, info.At_head, seg_len);
  }
  FILE* o = std::fopen(argv[5], "wb");
  if (!o) return 2;
  put<int>(o, rc);
  put<int>(o, (int)err.size());
  std::fwrite(err.data(), 1, err.size(), o);
  put<long long>(o, rc == 0 ? nz : 0);
  const bool ok = rc == 0;
  put_vec(o, info.prow);
  put_vec(o, info.pcol);
  put_vec(o, ok ? down(arr.A_rp, (size_t)m + 1) : std::vector<int>());
  put_vec(o, ok ? down(arr.A_ci, (size_t)nz) : std::vector<int>());
  put_vec(o, ok ? down(arr.A_v, (size_t)nz) : std::vector<double>());
  put_vec(o, ok ? down(arr.At_rp, (size_t)n + 1) : std::vector<int>());
  put_vec(o, ok ? down(arr.At_ci, (size_t)nz) : std::vector<int>());
  put_vec(o, ok ? down(arr.At_v, (size_t)nz) : std::vector<double>());
  put_bins(o, info.binsA);
  put_bins(o, info.binsAt);
  put_vec(o, segA);
  put_vec(o, segAt);
  // beyond the host runner's format
  put<int>(o, info.split[0]);
  put<int>(o, info.split[1]);
  put_vec(o, ok ? down(arr.prow, (size_t)m) : std::vector<int>());
  put_vec(o, ok ? down(arr.pcol, (size_t)n) : std::vector<int>());
  put_vec(o, ok ? down(vec.d_b, (size_t)m) : std::vector<double>());
  put_vec(o, ok ? down(vec.d_sense, (size_t)m) : std::vector<uint8_t>());
  put_vec(o, ok ? down(vec.d_c, (size_t)n) : std::vector<double>());
  put_vec(o, ok ? down(vec.d_l, (size_t)n) : std::vector<double>());
  put_vec(o, ok ? down(vec.d_u, (size_t)n) : std::vector<double>());
  std::fclose(o);
  for (void* q : owned) cudaFree(q);
  cudaStreamDestroy(s);
  return 0;
}
