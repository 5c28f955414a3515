// Krylov workspace and internal entry points shared by expmv and the correlators.
#pragma once
#include <complex>

#include "syk_internal.h"

namespace syk {

// Device scratch of one Lanczos process over a batch of B states of dimension D.
struct KrylovWS {
  int m = 0;            // maximum Krylov dimension
  int64_t B = 0, D = 0;
  int dtype = 0;
  int G = 0;            // blocks of the reduction kernels
  int bdim = 0;         // threads per block of the vector kernels (multiple of B)
  char* V = nullptr;    // (m+1) basis vectors, D*B elements each
  char* w = nullptr;    // work vector
  double2* part = nullptr;   // G * (m+1) * B partial dots
  double2* h1 = nullptr;     // (m+1) * B
  double2* h2 = nullptr;
  double* npart = nullptr;   // G * B partial squared norms
  double* alpha = nullptr;   // m * B
  double* beta = nullptr;    // m * B
  double* beta0 = nullptr;   // B
  double* inv = nullptr;     // B
  double* theta = nullptr;   // m * B
  double* Q = nullptr;       // B * m * m
  double* sb = nullptr;      // B
  double* sacc = nullptr;    // 1
  double2* c = nullptr;      // m * B
  int* status = nullptr;     // 4 ints
  void* host_stage = nullptr;  // host buffer (>= 64 B) for status reads; NULL: pinned scratch
  size_t vec_bytes() const { return size_t(D) * B * dtype_size(dtype); }
  char* vec(int k) const { return V + size_t(k) * vec_bytes(); }
};

size_t krylov_ws_bytes(int64_t D, int dtype, int m, int64_t B);
int krylov_ws_carve(KrylovWS* ws, void* base, size_t bytes, int64_t D, int dtype, int m, int64_t B);

// out = e^{z H} psi (see syk_expmv).  psi and out may alias.
int expmv_impl(const ApplyParams& P, int dtype, std::complex<double> z, const void* psi, void* out,
               int64_t B, double tol, KrylovWS& ws, cudaStream_t st, int* nsteps);

// result[b] = sum_x conj(x[x][b]) y[x][b] (FP64), written to device memory `res` (B double2).
int dot_columns(const void* x, const void* y, int64_t D, int64_t B, int dtype, KrylovWS& ws,
                double2* res, cudaStream_t st);

// Host helpers: pinned staging buffer for small device->host reads.
void* pinned_scratch(size_t bytes);

}  // namespace syk
