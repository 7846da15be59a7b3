// Resumable elimination (the paper's stop-and-resume by step, Sec. 5): the
// state of the in-place elimination after k steps is the matrix itself, so a
// run can stop between steps, save (A, k) and continue later, here or in
// another process. blockinv_invert_steps applies a range of FP64 steps;
// the checkpoint functions move that state to and from a file.
//
// File layout (little-endian): "BLKINVC1", int64 n, int32 p, int32 k_done,
// int32 sizes[p], uint64 FNV-1a hash of the matrix bytes, then the n x n
// doubles row by row (the leading dimension is not stored).
#include <cstdio>
#include <cstring>
#include <vector>

#include "internal.h"

namespace blockinv {

namespace {

constexpr char kMagic[8] = {'B', 'L', 'K', 'I', 'N', 'V', 'C', '1'};

uint64_t fnv1a(const void* data, size_t bytes) {
  const unsigned char* p = static_cast<const unsigned char*>(data);
  uint64_t h = 1469598103934665603ull;
  for (size_t i = 0; i < bytes; ++i) {
    h ^= p[i];
    h *= 1099511628211ull;
  }
  return h;
}

struct File {
  FILE* f = nullptr;
  File(const char* path, const char* mode) : f(std::fopen(path, mode)) {}
  ~File() {
    if (f) std::fclose(f);
  }
};

}  // namespace

}  // namespace blockinv

using namespace blockinv;

extern "C" {

int blockinv_checkpoint_write(const char* path, int64_t n, int32_t p, const int32_t* block_sizes, const double* A,
                              int64_t lda, int32_t k_done, void* stream) {
  Plan pl;
  int st = plan_for(n, p, block_sizes, lda, &pl);
  if (st != BLOCKINV_OK || !path || !A || k_done < 0 || k_done > (int32_t)pl.sizes.size())
    return BLOCKINV_ERR_INVALID;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  std::vector<double> host((size_t)n * n);
  const size_t row = sizeof(double) * (size_t)n;
  cudaError_t e = copy_matrix(host.data(), n, A, lda, n, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_status(e);
  const int32_t np = (int32_t)pl.sizes.size();
  const uint64_t h = fnv1a(host.data(), row * (size_t)n);
  File out(path, "wb");
  if (!out.f) return BLOCKINV_ERR_INVALID;
  const int64_t nn = n;
  bool ok = std::fwrite(kMagic, 1, 8, out.f) == 8 && std::fwrite(&nn, 8, 1, out.f) == 1 &&
            std::fwrite(&np, 4, 1, out.f) == 1 && std::fwrite(&k_done, 4, 1, out.f) == 1 &&
            std::fwrite(pl.sizes.data(), 4, (size_t)np, out.f) == (size_t)np && std::fwrite(&h, 8, 1, out.f) == 1 &&
            std::fwrite(host.data(), row, (size_t)n, out.f) == (size_t)n;
  return ok ? BLOCKINV_OK : BLOCKINV_ERR_INVALID;
}

int blockinv_checkpoint_read(const char* path, int64_t n, int32_t p, const int32_t* block_sizes, double* A,
                             int64_t lda, int32_t* k_done, void* stream) {
  Plan pl;
  int st = plan_for(n, p, block_sizes, lda, &pl);
  if (st != BLOCKINV_OK || !path || !A || !k_done) return BLOCKINV_ERR_INVALID;
  // everything is checked on the host before A is touched
  File in(path, "rb");
  if (!in.f) return BLOCKINV_ERR_INVALID;
  char magic[8];
  int64_t fn = 0;
  int32_t fp = 0, fk = 0;
  uint64_t h = 0;
  if (std::fread(magic, 1, 8, in.f) != 8 || std::memcmp(magic, kMagic, 8) != 0) return BLOCKINV_ERR_INVALID;
  if (std::fread(&fn, 8, 1, in.f) != 1 || std::fread(&fp, 4, 1, in.f) != 1 || std::fread(&fk, 4, 1, in.f) != 1)
    return BLOCKINV_ERR_INVALID;
  if (fn != n || fp != (int32_t)pl.sizes.size() || fk < 0 || fk > fp) return BLOCKINV_ERR_INVALID;
  std::vector<int32_t> fs((size_t)fp);
  if (std::fread(fs.data(), 4, (size_t)fp, in.f) != (size_t)fp) return BLOCKINV_ERR_INVALID;
  for (int32_t i = 0; i < fp; ++i)
    if (fs[i] != pl.sizes[i]) return BLOCKINV_ERR_INVALID;
  if (std::fread(&h, 8, 1, in.f) != 1) return BLOCKINV_ERR_INVALID;
  std::vector<double> host((size_t)n * n);
  const size_t row = sizeof(double) * (size_t)n;
  if (std::fread(host.data(), row, (size_t)n, in.f) != (size_t)n) return BLOCKINV_ERR_INVALID;
  if (std::fgetc(in.f) != EOF || fnv1a(host.data(), row * (size_t)n) != h) return BLOCKINV_ERR_INVALID;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = copy_matrix(A, lda, host.data(), n, n, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_status(e);
  *k_done = fk;
  return BLOCKINV_OK;
}

int blockinv_invert_steps(int64_t n, int32_t p, const int32_t* block_sizes, double* A, int64_t lda, int32_t k0,
                          int32_t k1, void* stream) {
  Plan pl;
  int st = plan_for(n, p, block_sizes, lda, &pl);
  if (st != BLOCKINV_OK || !A || k0 < 0 || k1 < k0 || k1 > (int32_t)pl.sizes.size()) return BLOCKINV_ERR_INVALID;
  return invert_steps(pl, A, lda, k0, k1, static_cast<cudaStream_t>(stream));
}

}  // extern "C"
