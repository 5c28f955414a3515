// Krylov workspace and internal entry points shared by expmv and the correlators.
#pragma once
#include <complex>
#include <vector>

#include "syk_internal.h"

namespace syk {

// Device-side control of an evolution run as one CUDA graph (see expmv_chain): the job (z,
// tol, input and output vectors), the step state, error bits and work counters.
struct ExpJob {
  double zr, zi, tol;
  const void* in;
  void* out;
};
struct DevCtl {
  double s_rem, s_done, ds, s_acc;
  int m_eff, err, jsteps, done;
  long long bases, applies, launches;
  long long mv[3];  // matvec launches by kernel family (rows, tiled, coset)
};

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
  char* split = nullptr;     // complex128 only: double-float copy of the matvec input (D*B float4)
  // The basis is stored unnormalised: V_k = u_k with v_k = sc[k*B + b] u_k (sc[0] = 1; the
  // Lanczos step folds 1/beta_j into the next matvec's output instead of rescaling u_{j+1}).
  double* sc = nullptr;      // (m+1) * B
  double2* ep_part = nullptr;  // per-CTA partial dots of the matvec epilogue (ep_cap * B)
  int* ep_nblk = nullptr;
  int64_t ep_cap = 0;
  ExpJob* job = nullptr;     // the evolution a device-driven graph runs next
  DevCtl* ctl = nullptr;
  void* host_stage = nullptr;  // host buffer (>= 64 B) for status reads; NULL: pinned scratch
  size_t vec_bytes() const { return size_t(D) * B * dtype_size(dtype); }
  char* vec(int k) const { return V + size_t(k) * vec_bytes(); }
  // the matvec parameters with this workspace's split buffer (complex128 in double-float)
  ApplyParams with_split(const ApplyParams& P) const {
    ApplyParams q = P;
    if (split) {
      q.df_split = split;
      q.df_split_bytes = size_t(D) * B * 16;
    }
    q.ep_cap = ep_cap;
    return q;
  }
};

// Orthogonalisation of expmv's Lanczos basis (syk_lanczos_orth): full classical Gram-Schmidt
// against the whole basis, or the local three-term recurrence.
enum { kOrthFull = 0, kOrthLocal = 1 };
int lanczos_orth(int dtype);

size_t krylov_ws_bytes(int64_t D, int dtype, int m, int64_t B);
int krylov_ws_carve(KrylovWS* ws, void* base, size_t bytes, int64_t D, int dtype, int m, int64_t B);

// out = e^{z H} psi (see syk_expmv).  psi and out may alias.
int expmv_impl(const ApplyParams& P, int dtype, std::complex<double> z, const void* psi, void* out,
               int64_t B, double tol, KrylovWS& ws, cudaStream_t st, int* nsteps);

// The evolutions of a correlator chain: out = e^{zH} in (in and out may alias), as expmv_impl.
// With CUDA graphs enabled and profiling off, each is one launch of a graph that runs the
// whole Krylov loop with its step control on the device (conditional WHILE and IF nodes):
// the host only enqueues, with no synchronisation until the chain ends.  chain_begin clears
// the device-side error bits and counters; chain_end (called after the caller has
// synchronised the stream) reports the first device-side error and adds the counters.
int chain_begin(KrylovWS& ws, cudaStream_t st);
int expmv_chain(const ApplyParams& P, int dtype, std::complex<double> z, const void* in, void* out, int64_t B,
                double tol, KrylovWS& ws, cudaStream_t st);
int chain_end(KrylovWS& ws, cudaStream_t st);

// outs[k] = e^{fr[k] z H} psi for increasing fractions 0 < fr[0] < ... < fr[nf-1], each output
// combined from the Krylov basis whose step covers it (no extra matvecs per output).  psi may
// alias outs[nf-1] only; the other outputs must be distinct buffers.
int expmv_points(const ApplyParams& P, int dtype, std::complex<double> z, const void* psi, const double* fr, int nf,
                 void* const* outs, int64_t B, double tol, KrylovWS& ws, cudaStream_t st);

// result[b] = sum_x conj(x[x][b]) y[x][b] (FP64), written to device memory `res` (B double2).
int dot_columns(const void* x, const void* y, int64_t D, int64_t B, int dtype, KrylovWS& ws,
                double2* res, cudaStream_t st);

// Host helpers: pinned staging buffer for small device->host reads.
void* pinned_scratch(size_t bytes);

// Lanczos for eigenvalues (syk_lowest_eigenvalues): lanczos_begin stores v_0 = psi/||psi||
// (one column, B = 1); lanczos_steps runs steps [j0, j1) of the three-term recurrence with
// full two-pass classical Gram-Schmidt reorthogonalisation, writing alpha_j, beta_j to the
// workspace (ws.alpha, ws.beta; beta_j = 0 marks a breakdown) and v_{j+1} for j + 1 < ws.m.
int lanczos_begin(int dtype, const void* psi, KrylovWS& ws, cudaStream_t st);
int lanczos_steps(const ApplyParams& P, int dtype, KrylovWS& ws, int j0, int j1, cudaStream_t st);

// Persistent batched OTOC (syk_batch.cu).  batch_item_persistent_states: how many of an item's
// states one CTA of the persistent kernel takes (1, 2, 4, 8 or 16: the largest power of two
// that divides the item's state count and whose sector vectors and launch scalars fit one
// CTA's shared memory; at least 2 unless the item has one state), or 0 when the item takes
// the per-item path (complex128, full Gram-Schmidt for complex64, or too large a sector).
// otoc_batch_persistent runs the items in idx, each split into sub-items of Bs states (one
// CTA each; the states of a chain are independent), as ONE launch on stream st and fills their
// host results and statuses (synchronises st); report gets, added: items, -, CTAs, clock
// cycles in matvecs, convergence checks, full eigendecompositions and whole sub-items, H
// applications (states x matvecs), convergence checks, full eigendecompositions, sub-items,
// and the matvecs' algorithmic flops (8 per nonzero of H_s per state).
constexpr int kBatchReportWords = 12;
bool batch_persistent_enabled();
bool batch_persistent_split_always();  // syk_batch_persistent(2): split items regardless of count
int batch_item_persistent_states(const syk_terms* t, int64_t B, const void* psi0, int dtype, int m);
int otoc_batch_persistent(const syk_otoc_item* items, const std::vector<int>& idx, int64_t Bs, int i, int j,
                          const double* t, int nt, int m, double tol, int* item_status, cudaStream_t st,
                          long long* report);
void batch_report_store(const long long* r);

// Device buffers owned by one library call (freed, stream-ordered, when it returns).
struct Scratch {
  cudaStream_t st;
  std::vector<void*> ptrs;
  explicit Scratch(cudaStream_t s) : st(s) {}
  ~Scratch() {
    for (void* p : ptrs) cudaFreeAsync(p, st);
  }
  int alloc(void** p, size_t bytes) {
    cudaError_t e = cudaMallocAsync(p, bytes, st);
    if (e != cudaSuccess) {
      set_error("cannot allocate %zu bytes of device memory: %s", bytes, cudaGetErrorString(e));
      *p = nullptr;
      return SYK_ENOMEM;
    }
    ptrs.push_back(*p);
    return SYK_OK;
  }
};

// Returns a device copy of psi0 if it is host memory, else psi0 itself.
inline int device_input(const void* psi0, size_t bytes, Scratch& sc, const void** out) {
  cudaPointerAttributes at;
  cudaError_t e = cudaPointerGetAttributes(&at, psi0);
  if (e != cudaSuccess) cudaGetLastError();
  if (e == cudaSuccess && (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged)) {
    *out = psi0;
    return SYK_OK;
  }
  void* d = nullptr;
  SYK_TRY(sc.alloc(&d, bytes));
  SYK_CUDA_CHECK(cudaMemcpyAsync(d, psi0, bytes, cudaMemcpyHostToDevice, sc.st));
  *out = d;
  return SYK_OK;
}


}  // namespace syk
