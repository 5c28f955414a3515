// Internal declarations shared by the translation units of libsyk_gb300.
#pragma once

#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdint>
#include <map>
#include <mutex>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/syk.h"

namespace syk {

// Names a span of host-side library work for profilers (NVTX ranges: a call into a stub that
// does nothing unless a profiler is attached).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

void set_error(const char* fmt, ...);
void clear_error();

#define SYK_CUDA_CHECK(expr)                                                                   \
  do {                                                                                         \
    cudaError_t e_ = (expr);                                                                   \
    if (e_ != cudaSuccess) {                                                                   \
      syk::set_error("%s failed: %s (%s:%d)", #expr, cudaGetErrorString(e_), __FILE__, __LINE__); \
      return SYK_ECUDA;                                                                        \
    }                                                                                          \
  } while (0)

#define SYK_TRY(expr)          \
  do {                         \
    int rc_ = (expr);          \
    if (rc_ != SYK_OK) return rc_; \
  } while (0)

// Row-flip patterns of a popcount-4 mask record (.w): 5 bits (4 table-index support bits and
// the sign bit) per compact row bit kFlipBit0 .. kFlipBit0 + 5; a kernel whose row slots are
// the compact bits b .. b+2 reads them at shift 5 * (b - kFlipBit0).
constexpr int kFlipBit0 = 5;
constexpr int flip_shift(int b) { return 5 * (b - kFlipBit0); }

// Device copies of the grouped coefficient tables (see syk_terms.cpp for the math).
struct DeviceTables {
  int device = -1;
  uint4* m4_rec = nullptr;    // popcount-4 X-masks: {compact xor, zeta0, packed support, row-flip patterns}
  double2* m4_t64 = nullptr;  // 32 entries per mask: T[u], then -T[u]
  float2* m4_t32 = nullptr;
  uint4* m2_rec = nullptr;    // popcount-2 X-masks: {compact xor, zeta_f, a | b<<8, 0}
  double2* m2_t64 = nullptr;  // n x 4 entries per mask: W_c[u]
  float2* m2_t32 = nullptr;
  double* wd64 = nullptr;     // n x n upper triangle: diagonal couplings w_cd
  float* wd32 = nullptr;
  // double-float copies of the FP64 tables for the complex128 matvec: every double d is
  // stored as floats (hi, lo) = (fl(d), fl(d - hi)); complex entries as (re_hi, im_hi, re_lo, im_lo)
  float4* m4_tdf = nullptr;
  float4* m2_tdf = nullptr;
  float2* wd_df = nullptr;
  int* status = nullptr;      // device status word of the matvec (bounded-wait timeouts)
};

// Everything apply_H needs, by value, for one launch.
struct ApplyParams {
  int n;        // spins
  int sector;   // 0 even, 1 odd
  int64_t D;    // sector dimension 2^(n-1)
  int n4, n2;
  const uint4* m4_rec;
  const uint4* m2_rec;
  const void* m4_tab;
  const void* m2_tab;
  const void* wd;
  int* status;
  const float4* m4_tdf;    // double-float tables (complex128 matvec in FP32 arithmetic)
  const float4* m2_tdf;
  const float2* wd_df;
  double rho;              // host-side: spectral half-width estimate of H (term set's rho_est)
  const syk_terms* terms;  // host-side: tile-group lists
  bool no_alloc;           // host-side: never allocate (use only cached tile-group lists)
  void* df_split;          // host-side: device buffer (>= D x batch x 16 bytes) for the split
  size_t df_split_bytes;   // copy of a complex128 input, or NULL (then allocated per call)
  // Lanczos epilogue (ep_part NULL: plain y = H psi).  With it the launch computes
  //   y[x][b] = ep_scale[b] * (H psi)[x][b]   (ep_scale NULL: scale 1), and
  //   ep_part[cta * batch + b] = sum over the CTA's rows of conj(ep_u[x][b]) y[x][b]   (FP64),
  // one partial per CTA and column (fixed-order sums), and *ep_nblk = the number of CTAs.
  // ep_u has psi's layout and dtype (complex128 for the double-float kernel too).
  const double* ep_scale;
  const void* ep_u;
  double2* ep_part;
  int* ep_nblk;
  int64_t ep_cap;          // host-side: capacity of ep_part in CTAs
};

// Chunks of X-masks sharing the compact-mask bits h above a tile of 2^tb rows, at
// most gmax popcount-4 masks per chunk: {h | first-chunk-of-h << 31, first
// popcount-4 mask, end, first popcount-2 mask | end << 16} (popcount-2 masks and
// the diagonal go with the first chunk of their h).
int tile_groups(const syk_terms* t, int tb, int gmax, const int4** dev, int* count);
// Lookup only: returns false if that list has not been built on this device yet.
bool tile_groups_cached(const syk_terms* t, int tb, int gmax, const int4** dev, int* count);

// Coset layout of the popcount-4 masks for a tile of 2^tb rows whose threads own rows that
// differ in the top `rbits` row bits (offsets d): masks m and m ^ (d << (tb - rbits)) read the
// same partner row for the thread's row slots 0 and d.  Per chunk (<= gmax masks):
//   chunks[c] = {h | first << 31, first mask, end mask, popcount-2 range as in tile_groups},
//   counts[c] = number of cosets of each multi-mask shape (byte per shape, in the fixed shape
//               order of the row-bit count); the chunk's masks are those cosets' members in
//               shape order, each coset's members by increasing offset, then single masks,
// with the mask records and 32-entry tables (fp32 and fp64) permuted into that order.
struct CosetLayout {
  int4* chunks = nullptr;
  uint32_t* counts = nullptr;
  uint4* rec = nullptr;
  float2* t32 = nullptr;
  double2* t64 = nullptr;
  int nchunks = 0;
};
int coset_layout(const syk_terms* t, int tb, int rbits, int gmax, bool may_alloc, const CosetLayout** out);
// The same layout in host memory (no device needed).
struct CosetHost {
  std::vector<int4> chunks;
  std::vector<uint32_t> counts;
  std::vector<uint4> rec;
  std::vector<float> t32;
  std::vector<double> t64;
};
int coset_layout_host(const syk_terms* t, int tb, int rbits, int gmax, CosetHost* out);

// complex64 coset matvec (syk_apply_coset.cu).  var = log2(rows per thread): 1 or 2 for 16
// columns, 2 or 3 for 4 and 8 columns.  launch_coset_var returns 1 when that variant does
// not apply to this launch (the caller then uses k_apply_tiled).
bool coset_var_ok(int dtype, int64_t batch, int var);
bool coset_fits(int64_t batch, int var, int ntb);  // CTA width 2^ntb (6 or 7) within shared memory
int launch_coset_var(const ApplyParams& p, int64_t batch, const void* psi, void* y, cudaStream_t st, int var, int ntb,
                     int cs);

// complex64 matvec of one state (syk_apply_one.cu) on the tiles of k_apply_tiled<float, 1>
// (8 rows per thread, CTA width 2^ntb, ntb in 6..8, cluster of cs CTAs; groups: the chunk list
// of that tile size).
int launch_one_state(const ApplyParams& p, const int4* groups, int ng, int ntb, int cs, const void* psi, void* y,
                     cudaStream_t st);

int ensure_device_tables(const syk_terms* t);
int ensure_grad_groups(const syk_terms* t);  // builds and uploads the gradient term groups
int make_apply_params(const syk_terms* t, int parity, int dtype, ApplyParams* p);

// Kernel launchers (stream-ordered, no synchronisation).
int launch_apply_H(const ApplyParams& p, int dtype, const void* psi, void* y, int64_t batch,
                   cudaStream_t st);
int launch_apply_chi(int N, int i, int parity_in, int dtype, const void* psi, void* y,
                     int64_t batch, cudaStream_t st);

// Profiling of apply_H launches (CUDA events) and work counters.
void prof_before_apply(cudaStream_t st);
void prof_after_apply(cudaStream_t st);
void prof_collect();
void count_applies(int64_t states);
void count_bases(int64_t n);
void count_launch(int64_t n = 1);
// While a thread captures a CUDA graph its counts go to thread-local tallies (returned by
// capture_counts_end) so that every replay can add them.
void capture_counts_begin();
void capture_counts_end(int64_t* launches, int64_t* applies, int64_t* kinds);
// Matvec launches by kernel family (kMvRows: k_apply_rows, kMvTiled: k_apply_tiled, kMvCoset:
// k_apply_coset), counted like the launches above (a replayed graph adds its recorded ones).
enum { kMvRows = 0, kMvTiled = 1, kMvCoset = 2, kMvKinds = 3 };
void count_matvec(int kind);
void count_matvec_replay(const int64_t* kinds);
bool prof_enabled();
uint64_t graph_epoch();  // changes whenever captured graphs may hold stale parameters
void bump_graph_epoch();
bool graphs_enabled();
bool device_chains_enabled();  // syk_use_graphs(2)

// Arithmetic of the complex128 matvec: double-float (FP32 error-free transformations, the
// default) or native FP64 (syk_c128_arith).
enum { kC128DoubleFloat = 0, kC128Fp64 = 1 };
int c128_arith();

// Raises func's dynamic shared-memory limit to at least `bytes` on the current device (the
// attribute is per device; done once per kernel and device, thread-safe).
int ensure_smem_limit(const void* func, int bytes);
// Streaming multiprocessors of the current device (cached per device; 1 if the query fails).
int sm_count();

inline size_t dtype_size(int dtype) { return dtype == SYK_C64 ? 8 : 16; }
inline bool dtype_ok(int dtype) { return dtype == SYK_C64 || dtype == SYK_C128; }

}  // namespace syk

struct syk_terms {
  int N = 0, n = 0;
  int64_t nterms = 0, D = 0;
  std::vector<uint64_t> xm, zm;  // per term, lexicographic order
  std::vector<uint8_t> ph;
  std::vector<double> J;
  double rho_est = 0.0;  // 2 sqrt(sum J^2 / 16): half-width of the spectrum (RMS level x 2)
  int n4 = 0, n2 = 0;
  std::vector<uint32_t> m4_rec;  // 4 words per mask
  std::vector<double> m4_tab;    // n4 * 32 * 2
  std::vector<uint32_t> m2_rec;  // 4 words per mask
  std::vector<double> m2_tab;    // n2 * n * 4 * 2
  std::vector<double> wdiag;     // n * n
  mutable syk::DeviceTables dev;
  mutable std::map<int, std::pair<int4*, int>> groups_dev;  // tile bits -> device group list
  mutable std::map<int, syk::CosetLayout> coset_dev;         // (tb, rbits, gmax) -> coset layout
  // Term groups of the per-term inner products (gradients), built on first use: terms sharing
  // an X-mask and a Z-mask off their support bits; device copies on dev.device.
  mutable int ngg = 0;
  mutable std::vector<uint32_t> gg_rec;   // 4 words per group: compact xor, zeta, support shifts, k
  mutable std::vector<int32_t> term_group;
  mutable std::vector<uint8_t> term_s;
  mutable std::vector<double> term_phase;  // 2 per term: i^p (-1)^popcount(z & m) / 4
  mutable uint4* d_gg_rec = nullptr;
  mutable int* d_term_group = nullptr;
  mutable uint8_t* d_term_s = nullptr;
  mutable double2* d_term_phase = nullptr;
  mutable std::mutex mtx;
};
