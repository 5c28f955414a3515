// Persistent batched OTOC: the disorder and random-state average of Supp. Sec. I.C as ONE
// kernel launch over many small-sector work items.  Each CTA takes items from a device-side
// queue (an atomic counter) and evaluates an item's whole regularized-OTOC chain (Eq. F_reg
// by Eq. q_typicality, the chain of syk_otoc) by itself: every Krylov evolution (Supp. Sec.
// I.B: Lanczos with the three-term recurrence, FP64 scalars, FP64 tridiagonal
// eigendecompositions, Saad's error estimate and the step control of syk_expmv), the
// Majorana applications and the final dots.  A work item is a sub-item: some of a coupling
// draw's states (all of them, or a share of 2 or more when D x states would not fit), whose
// sector vector fits in shared memory, so every matvec gathers its partner rows psi[x ^ m]
// from the staged input; the Krylov basis and the chain's vectors live in the CTA's own slice
// of global memory (L2).  CTAs share nothing but the queue counter: there is no grid-wide
// synchronisation, no spin-wait (only CTA barriers) and no host round trip until the launch
// ends.  complex64 vectors (FP32 arithmetic), as the batched workload specifies; larger
// sectors and complex128 items take the per-item path of syk_otoc_batch.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <vector>

#include "syk_krylov.cuh"
#include "syk_tile.cuh"
#include "syk_tridiag.cuh"

namespace syk {
namespace {

constexpr int kPNT = 512;              // threads per CTA
constexpr int kPWarps = kPNT / 32;     // >= the largest batch of an item (16)
constexpr int kPG = 64;                // popcount-4 masks staged in shared memory per chunk
// Bounds on the Krylov bases of one evolution and of one item (a sane chain needs a few per
// evolution): past them the item stops with error bit 4, so no input keeps a CTA busy for long.
constexpr int kMaxBasesPerEvolution = 1000;
constexpr long long kMaxBasesPerItem = 4000;
// Bisection steps of the step selection: the accepted step is within 2^-12 of the largest
// admissible one (the per-item path takes 24; each costs an FP64 evaluation of the estimate).
constexpr int kBisect = 12;

// One work item: a coupling draw's tables (complex64 copies), its states and beta.
struct PItem {
  const uint4* m4_rec;
  const float2* m4_t32;
  const uint4* m2_rec;
  const float2* m2_t32;
  const float* wd32;
  const float2* psi0;  // D x B (device)
  double2* F;          // F[k * Fld + c]: result of state c at time k (device)
  double beta, rho;
  int n, D, n4, n2;
  int every;           // Lanczos vectors between two convergence checks after the first
  int first8;          // the first check comes at first8/8 of the predicted Krylov dimension
  int Fld;             // row stride of F (the parent item's state count)
};

// Per-item record written by the kernel.
enum { kStStatus = 0, kStMatvecs = 1, kStBases = 2, kStCyMatvec = 3, kStCyCheck = 4, kStCyEig = 5, kStCyAll = 6,
       kStChecks = 7, kStEigs = 8, kStWords = 10 };

// Work and clock counters of one item.
struct PCount {
  long long cy[3];  // clock cycles: matvecs, convergence checks, full eigendecompositions
  long long mv, nb, nck, neig;
};

// Shared-memory layout of a launch (byte offsets, computed on the host).
struct PLayout {
  int A;        // region A: staged matvec input | convergence-check scratch | eigenvector matrices
  int rec, tab;  // staged popcount-4 records and 32-entry tables
  int alpha, beta, sc, beta0, h, n2, cc, red, sb, fc, ctl;
  int total;
  int ncol;     // columns per round of the full eigendecomposition
};

struct PArgs {
  const PItem* items;
  int nitems;
  int* next;          // queue counter, 0 at launch
  long long* stat;    // kStWords per item
  const double* t;    // nt output times (device)
  int nt, i, j;       // Majoranas i (W), j (V)
  int m;              // Krylov dimension
  double tol, bt;     // step tolerance, breakdown threshold of beta_j
  float2* ws;         // per CTA: (m + 5) vectors of vmax elements, then cmax float2 of coefficients
  long long vmax, cmax;
  PLayout L;
};

struct PCtl {
  int item, status, first;
  double s_acc;
};

// ---------------------------------------------------------------- row access
// Rows are B contiguous complex64 values (16-byte aligned for B >= 2), accessed as column
// pairs: pair q holds columns 2q and 2q + 1 (B >= 2) or column 0 alone (B == 1).
constexpr int npairs(int B) { return B >= 2 ? B / 2 : 1; }
template <int B>
__device__ __forceinline__ void ld_pair(const float2* row, int q, float2& v0, float2& v1) {
  if constexpr (B == 1) {
    v0 = row[0];
    v1 = make_float2(0.f, 0.f);
  } else {
    const float4 t = reinterpret_cast<const float4*>(row)[q];
    v0 = make_float2(t.x, t.y);
    v1 = make_float2(t.z, t.w);
  }
}
template <int B>
__device__ __forceinline__ void st_pair(float2* row, int q, float2 v0, float2 v1) {
  if constexpr (B == 1) row[0] = v0;
  else reinterpret_cast<float4*>(row)[q] = make_float4(v0.x, v0.y, v1.x, v1.y);
}
// p += conj(a) b
__device__ __forceinline__ void cdot_acc(float2& p, const float2 a, const float2 b) {
  p.x = fmaf(a.x, b.x, fmaf(a.y, b.y, p.x));
  p.y = fmaf(a.x, b.y, fmaf(-a.y, b.x, p.y));
}
__device__ __forceinline__ void norm_acc(float2& p, const float2 a) { p.x = fmaf(a.x, a.x, fmaf(a.y, a.y, p.x)); }

// ---------------------------------------------------------------- reductions
// Compensated FP32 sum over the warp (Knuth's TwoSum at every level of the butterfly): the
// pair (hi, lo) carries the sum to about 2^-44 relative, the same in every lane.
__device__ __forceinline__ void df_warp_sum(float& hi, float& lo) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float oh = __shfl_xor_sync(0xffffffffu, hi, o);
    const float ol = __shfl_xor_sync(0xffffffffu, lo, o);
    const float s = __fadd_rn(hi, oh);
    const float bp = __fsub_rn(s, hi);
    const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bp)), __fsub_rn(oh, bp));
    hi = s;
    lo = __fadd_rn(__fadd_rn(lo, ol), err);
  }
}

// out[c] = sum over the CTA of the threads' v[c] (c < B): per-thread FP32 partial sums (of at
// most 16 rows), a compensated sum per warp, then FP64 over the warps in increasing order
// (deterministic).  Ends with a barrier, so out is visible to every thread.
template <int B>
__device__ void cta_sum_cols(const float2 (&v)[B], double2* red, double2* out) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int c = 0; c < B; ++c) {
    float xh = v[c].x, xl = 0.f, yh = v[c].y, yl = 0.f;
    df_warp_sum(xh, xl);
    df_warp_sum(yh, yl);
    if (lane == 0) red[w * B + c] = make_double2((double)xh + (double)xl, (double)yh + (double)yl);
  }
  __syncthreads();
  if (threadIdx.x < B) {
    double sx = 0.0, sy = 0.0;
    for (int k = 0; k < kPWarps; ++k) {
      sx += red[k * B + threadIdx.x].x;
      sy += red[k * B + threadIdx.x].y;
    }
    out[threadIdx.x] = make_double2(sx, sy);
  }
  __syncthreads();
}

// Shared-memory views of a launch.
struct PSmem {
  unsigned char* A;
  uint4* rec;
  float2* tab;
  double *alpha, *beta, *sc, *beta0, *sb;
  double2 *h, *n2, *cc, *red;
  // FP32 coefficients of the vector passes, per column c: fc[c] = (sc_j, 0) of the staged
  // input, fc[B + c] = -h_j, fc[2B + c] = (-beta_{j-1} sc_{j-1}, 0), fc[(3 + k) B + c] =
  // cc_k sc_k of the combination (written once by a few threads: the FP64 pipe is 1/64 of
  // the FP32 rate, so no pass converts FP64 scalars per element)
  float2* fc;
  PCtl* ctl;
  __device__ PSmem(unsigned char* base, const PLayout& L)
      : A(base + L.A),
        rec(reinterpret_cast<uint4*>(base + L.rec)),
        tab(reinterpret_cast<float2*>(base + L.tab)),
        alpha(reinterpret_cast<double*>(base + L.alpha)),
        beta(reinterpret_cast<double*>(base + L.beta)),
        sc(reinterpret_cast<double*>(base + L.sc)),
        beta0(reinterpret_cast<double*>(base + L.beta0)),
        sb(reinterpret_cast<double*>(base + L.sb)),
        h(reinterpret_cast<double2*>(base + L.h)),
        n2(reinterpret_cast<double2*>(base + L.n2)),
        cc(reinterpret_cast<double2*>(base + L.cc)),
        red(reinterpret_cast<double2*>(base + L.red)),
        fc(reinterpret_cast<float2*>(base + L.fc)),
        ctl(reinterpret_cast<PCtl*>(base + L.ctl)) {}
};

// ---------------------------------------------------------------- vector passes
// Thread t handles rows t, t + kPNT, ... (all B columns of each).

// out[c] = sum_x conj(x[x][c]) y[x][c]
template <int B>
__device__ __noinline__ void cta_dot(const float2* x, const float2* y, int D, PSmem& S, double2* out) {
  float2 p[B];
#pragma unroll
  for (int c = 0; c < B; ++c) p[c] = make_float2(0.f, 0.f);
  for (int r = threadIdx.x; r < D; r += kPNT) {
#pragma unroll
    for (int q = 0; q < npairs(B); ++q) {
      float2 a0, a1, b0, b1;
      ld_pair<B>(x + (size_t)r * B, q, a0, a1);
      ld_pair<B>(y + (size_t)r * B, q, b0, b1);
      cdot_acc(p[B >= 2 ? 2 * q : 0], a0, b0);
      if constexpr (B >= 2) cdot_acc(p[2 * q + 1], a1, b1);
    }
  }
  cta_sum_cols<B>(p, S.red, out);
}

// y = x (elementwise copy)
template <int B>
__device__ void cta_copy(const float2* x, float2* y, int D) {
  for (int r = threadIdx.x; r < D; r += kPNT) {
#pragma unroll
    for (int q = 0; q < npairs(B); ++q) {
      float2 a0, a1;
      ld_pair<B>(x + (size_t)r * B, q, a0, a1);
      st_pair<B>(y + (size_t)r * B, q, a0, a1);
    }
  }
  __syncthreads();
}

// y = chi_maj x (Supp. Sec. I.A): x in sector 1 - sector_out, y in sector_out; as k_apply_chi
template <int B>
__device__ __noinline__ void cta_chi(int n, int D, int maj, int sector_out, const float2* x, float2* y) {
  const int k = maj >> 1;
  const float hh = 0.70710678118654752440f;
  for (int r = threadIdx.x; r < D; r += kPNT) {
    const uint32_t co = (uint32_t)r;
    const uint32_t xo = co | ((uint32_t)((__popc(co) + sector_out) & 1) << (n - 1));
    const uint32_t xs = xo ^ (1u << k);
    const float sg = (__popc(xs & ((1u << k) - 1u)) & 1) ? -hh : hh;
    const float2* src = x + (size_t)(xs & (uint32_t)(D - 1)) * B;
    const float si = ((xs >> k) & 1u) ? -sg : sg;  // odd maj: +i (x_k = 0) or -i (x_k = 1)
#pragma unroll
    for (int q = 0; q < npairs(B); ++q) {
      float2 v0, v1;
      ld_pair<B>(src, q, v0, v1);
      if (maj & 1) {
        v0 = make_float2(-si * v0.y, si * v0.x);
        v1 = make_float2(-si * v1.y, si * v1.x);
      } else {
        v0 = make_float2(sg * v0.x, sg * v0.y);
        v1 = make_float2(sg * v1.x, sg * v1.y);
      }
      st_pair<B>(y + (size_t)r * B, q, v0, v1);
    }
  }
  __syncthreads();
}

// ---------------------------------------------------------------- matvec
// The diagonal and popcount-2 coefficients of a row depend only on the row and the sector, so
// they are evaluated once per item (each is an O(n) sum over the spins) and stored in the
// CTA's workspace: dg[s * D + x] = c_0(x) and pc[(s * n2 + k) * D + x] = c_{m_k}(x) for the
// popcount-2 masks m_k, sector s.
__device__ __noinline__ void cta_coef(const PItem& it, float* dg, float2* pc) {
  const int n = it.n, D = it.D;
  for (int s = 0; s < 2; ++s)
    for (int r = threadIdx.x; r < D; r += kPNT) {
      const uint32_t xc = (uint32_t)r;
      const uint32_t xf = xc | ((uint32_t)((__popc(xc) + s) & 1) << (n - 1));
      dg[(size_t)s * D + r] = diag_coef<float>(it.wd32, n, xf);
      for (int k = 0; k < it.n2; ++k) {
        float cr, ci;
        pc2_coef<float2, float>(it.m2_t32, k, n, __ldg(&it.m2_rec[k]), xf, cr, ci);
        pc[((size_t)s * it.n2 + k) * D + r] = make_float2(cr, ci);
      }
    }
  __syncthreads();
}

// y = H xs in sector `sector` (Supp. Sec. I.B; the sums of k_apply_rows), xs staged in shared
// memory (D x B).  A thread owns RPT rows r0 + tid + i kPNT of each pass (they differ in the
// compact bits 9 and 10 only) and all B columns; rows wider than 16 bytes are read in 16-byte
// chunks in a lane-rotated order (chunk (q + lane) mod Q into accumulator q) so that the 32
// lanes of a warp hit distinct banks.  Popcount-4 records and tables are staged in chunks of
// kPG masks; a mask's table index for rows 1 .. RPT-1 is row 0's XOR the record's row-flip
// patterns of compact bits 9 and 10 (one extraction of the support bits per mask).
// dg, pc: this sector's precomputed diagonal and popcount-2 coefficients (cta_coef).
template <int B, int RPT>
__device__ __noinline__ void cta_matvec(const PItem& it, int sector, const float2* __restrict__ xs,
                                        float2* __restrict__ y, PSmem& S, const float* __restrict__ dg,
                                        const float2* __restrict__ pc) {
  static_assert(RPT == 1 || RPT == 2 || RPT == 4, "row slots are the compact bits 9 and 10");
  constexpr int Q = B >= 2 ? B / 2 : 1;
  constexpr int fsh = flip_shift(9);
  using V = typename std::conditional<(B >= 2), float4, float2>::type;
  const int tid = threadIdx.x;
  const int rot = (tid & 31) & (Q - 1);
  const int n = it.n, D = it.D;
  const V* __restrict__ x4 = reinterpret_cast<const V*>(xs);
  auto mac = [](V& a, float cr, float ci, const V v) {
    if constexpr (B >= 2) {
      Slot<float>::mac(a, cr, ci, v);
    } else {
      cmac(a, cr, ci, v);
    }
  };
  for (int r0 = 0; r0 < D; r0 += kPNT * RPT) {
    uint32_t xr[RPT];
    bool ok[RPT];
    V acc[RPT][Q];
    const uint32_t xr0 = (uint32_t)(r0 + tid);
    const uint32_t xf0 = xr0 | ((uint32_t)((__popc(xr0) + sector) & 1) << (n - 1));
#pragma unroll
    for (int i = 0; i < RPT; ++i) {
      xr[i] = xr0 + (uint32_t)(i * kPNT);
      ok[i] = (int)xr[i] < D;
      if (!ok[i]) continue;
      const float c0 = dg[xr[i]];
#pragma unroll
      for (int q = 0; q < Q; ++q) {
        const V v = x4[xr[i] * Q + ((q + rot) & (Q - 1))];
        if constexpr (B >= 2) acc[i][q] = make_float4(c0 * v.x, c0 * v.y, c0 * v.z, c0 * v.w);
        else acc[i][q] = make_float2(c0 * v.x, c0 * v.y);
      }
      for (int k = 0; k < it.n2; ++k) {
        const uint32_t mx = __ldg(&it.m2_rec[k].x);
        const float2 cf = pc[(size_t)k * D + xr[i]];
        const uint32_t pr = xr[i] ^ mx;
#pragma unroll
        for (int q = 0; q < Q; ++q) mac(acc[i][q], cf.x, cf.y, x4[pr * Q + ((q + rot) & (Q - 1))]);
      }
    }
    for (int c0 = 0; c0 < it.n4; c0 += kPG) {
      const int cnt = min(kPG, it.n4 - c0);
      __syncthreads();  // the previous chunk's records and tables are no longer read
      for (int e = tid; e < cnt; e += kPNT) S.rec[e] = __ldg(&it.m4_rec[c0 + e]);
      const float4* src = reinterpret_cast<const float4*>(it.m4_t32 + (size_t)c0 * 32);
      float4* dst = reinterpret_cast<float4*>(S.tab);
      for (int e = tid; e < cnt * 16; e += kPNT) dst[e] = __ldg(&src[e]);
      __syncthreads();
      if (!ok[0]) continue;  // rows 1 .. RPT-1 lie above row 0
      for (int k = 0; k < cnt; ++k) {
        const uint4 rec = S.rec[k];
        const float2* T = S.tab + k * 32;
        const uint32_t idx0 = supp_bits(xf0, rec.z) | ((__popc(rec.y & xf0) & 1u) << 4);
        const uint32_t fl = rec.w >> fsh;
        const uint32_t pr0 = xr0 ^ rec.x;
#pragma unroll
        for (int i = 0; i < RPT; ++i) {
          if (!ok[i]) continue;
          uint32_t f = 0u;
          if (i & 1) f ^= fl;
          if (i & 2) f ^= fl >> 5;
          const float2 cf = T[idx0 ^ (f & 31u)];
          const uint32_t pr = pr0 ^ (uint32_t)(i * kPNT);
#pragma unroll
          for (int q = 0; q < Q; ++q) mac(acc[i][q], cf.x, cf.y, x4[pr * Q + ((q + rot) & (Q - 1))]);
        }
      }
    }
    V* y4 = reinterpret_cast<V*>(y);
#pragma unroll
    for (int i = 0; i < RPT; ++i) {
      if (!ok[i]) continue;
#pragma unroll
      for (int q = 0; q < Q; ++q) y4[xr[i] * Q + ((q + rot) & (Q - 1))] = acc[i][q];
    }
  }
  __syncthreads();
}

__device__ __forceinline__ long long clk() { return clock64(); }

// ---------------------------------------------------------------- one evolution
// out = e^{z H} in in sector `sector` (in and out may alias), with the step control of
// syk_expmv for one output (expmv_T with a single fraction 1): Krylov bases of up to m vectors,
// convergence checks by the plan of check_plan (first check at 3/4 of the predicted
// dimension, later ones every it.every vectors; restarts from 4 vectors on), the largest step
// per basis whose estimate is <= tol for every column, restarts from the end state.
// basis: slots 1..m of the Krylov basis (slot k at basis + (k-1) vmax); slot 0 is `in` or the
// restart state.  dgs, pcs: the item's precomputed diagonal and popcount-2 coefficients.  Error bits go to S.ctl->status (1 non-finite scalar, 2 eigensolver, 4 step
// collapse or too many bases).
template <int B, int RPT>
__device__ __noinline__ void cta_expmv(const PArgs& a, const PItem& it, int sector, double zr, double zi, const float2* in,
                          float2* out, float2* basis, PSmem& S, PCount& pc, const float* dgs,
                          const float2* pcs) {
  const int D = it.D, m = a.m, tid = threadIdx.x;
  const double tol = a.tol;
  const size_t fstride = (size_t)m * m + 4 * (size_t)m + 2;  // doubles per column: Q, d, e, fg, rot
  const bool fused = a.L.ncol >= B;
  if (zr == 0.0 && zi == 0.0) {
    if (out != in) cta_copy<B>(in, out, D);
    return;
  }
  if (tid == 0) {  // predicted Krylov dimension: smallest k with (e rho |z| / 2k)^k <= tol
    const double rt = hypot(zr, zi) * it.rho;
    int k = m + 1;
    for (int kk = 1; kk <= m; ++kk)
      if (rt <= 0.0 || double(kk) * log(2.718281828459045 * rt / (2.0 * kk)) <= log(tol)) {
        k = kk;
        break;
      }
    S.ctl->first = min(m, max(4, (it.first8 * k) / 8));
  }
  __syncthreads();
  const int first = S.ctl->first;
  double s_rem = 1.0, s_done = 0.0;
  const float2* cur = in;
  float2* xs = reinterpret_cast<float2*>(S.A);
  int bases = 0;
  while (s_rem > 0.0) {
    if (++bases > kMaxBasesPerEvolution || pc.nb >= kMaxBasesPerItem) {
      if (tid == 0) S.ctl->status |= 4;
      __syncthreads();
      return;
    }
    ++pc.nb;
    auto U = [&](int k) -> const float2* { return k == 0 ? cur : basis + (size_t)(k - 1) * a.vmax; };
    // beta0 = ||cur||, sc_0 = 1/beta0
    {
      float2 p[B];
#pragma unroll
      for (int c = 0; c < B; ++c) p[c] = make_float2(0.f, 0.f);
      for (int r = tid; r < D; r += kPNT) {
#pragma unroll
        for (int q = 0; q < npairs(B); ++q) {
          float2 v0, v1;
          ld_pair<B>(cur + (size_t)r * B, q, v0, v1);
          norm_acc(p[B >= 2 ? 2 * q : 0], v0);
          if constexpr (B >= 2) norm_acc(p[2 * q + 1], v1);
        }
      }
      cta_sum_cols<B>(p, S.red, S.n2);
      if (tid < B) {
        const double nb0 = sqrt(fmax(S.n2[tid].x, 0.0));
        if (!isfinite(nb0)) atomicOr(&S.ctl->status, 1);
        S.beta0[tid] = nb0;
        S.sc[tid] = nb0 > 0.0 ? 1.0 / nb0 : 0.0;
        S.fc[tid] = make_float2((float)S.sc[tid], 0.f);
      }
      __syncthreads();
    }
    int j0 = 0, m_eff = m;
    int j1 = bases == 1 ? first : min(m, 4);
    double s_acc = 0.0;
    for (;;) {
      for (int j = j0; j < j1; ++j) {
        // stage v_j = sc_j u_j
        {
          const float2* u = U(j);
          for (int r = tid; r < D; r += kPNT) {
#pragma unroll
            for (int q = 0; q < npairs(B); ++q) {
              float2 v0, v1;
              ld_pair<B>(u + (size_t)r * B, q, v0, v1);
              const float s0 = S.fc[B >= 2 ? 2 * q : 0].x;
              const float s1 = B >= 2 ? S.fc[2 * q + 1].x : 0.f;
              st_pair<B>(xs + (size_t)r * B, q, make_float2(v0.x * s0, v0.y * s0), make_float2(v1.x * s1, v1.y * s1));
            }
          }
          __syncthreads();
        }
        float2* w = basis + (size_t)j * a.vmax;  // slot j+1
        const long long t0 = clk();
        cta_matvec<B, RPT>(it, sector, xs, w, S, dgs + (size_t)sector * D, pcs + (size_t)sector * it.n2 * D);
        pc.cy[0] += clk() - t0;
        ++pc.mv;
        // h_j = <v_j, w>
        cta_dot<B>(xs, w, D, S, S.h);
        if (tid < B) {
          S.fc[B + tid] = make_float2((float)(-S.h[tid].x), (float)(-S.h[tid].y));
          S.fc[2 * B + tid] =
              make_float2(j > 0 ? (float)(-S.beta[(j - 1) * B + tid] * S.sc[(j - 1) * B + tid]) : 0.f, 0.f);
        }
        __syncthreads();
        // u_{j+1} = w - h_j v_j - beta_{j-1} v_{j-1}, |u_{j+1}|^2
        {
          const float2* vm = j > 0 ? U(j - 1) : nullptr;
          float2 p[B];
#pragma unroll
          for (int c = 0; c < B; ++c) p[c] = make_float2(0.f, 0.f);
          for (int r = tid; r < D; r += kPNT) {
#pragma unroll
            for (int q = 0; q < npairs(B); ++q) {
              float2 w0, w1, v0, v1;
              ld_pair<B>(w + (size_t)r * B, q, w0, w1);
              ld_pair<B>(xs + (size_t)r * B, q, v0, v1);
              const int c0 = B >= 2 ? 2 * q : 0, c1 = B >= 2 ? 2 * q + 1 : 0;
              const float2 h0 = S.fc[B + c0], h1 = S.fc[B + c1];
              cmac(w0, h0.x, h0.y, v0);
              cmac(w1, h1.x, h1.y, v1);
              if (vm) {
                float2 p0, p1;
                ld_pair<B>(vm + (size_t)r * B, q, p0, p1);
                const float f0 = S.fc[2 * B + c0].x, f1 = S.fc[2 * B + c1].x;
                w0 = make_float2(fmaf(f0, p0.x, w0.x), fmaf(f0, p0.y, w0.y));
                w1 = make_float2(fmaf(f1, p1.x, w1.x), fmaf(f1, p1.y, w1.y));
              }
              st_pair<B>(w + (size_t)r * B, q, w0, w1);
              norm_acc(p[c0], w0);
              if constexpr (B >= 2) norm_acc(p[c1], w1);
            }
          }
          cta_sum_cols<B>(p, S.red, S.n2);
        }
        // alpha_j, beta_j (breakdown: beta_j = 0), sc_{j+1} = 1/beta_j, as k_lanczos_scalars
        if (tid < B) {
          const int c = tid;
          const double al = S.h[c].x;
          double be = sqrt(fmax(S.n2[c].x, 0.0));
          if (!isfinite(al) || !isfinite(be)) {
            atomicOr(&S.ctl->status, 1);
            be = 0.0;
          }
          const double prev = j > 0 ? S.beta[(j - 1) * B + c] : 0.0;
          if (be <= a.bt * (fabs(al) + prev)) be = 0.0;
          S.alpha[j * B + c] = isfinite(al) ? al : 0.0;
          S.beta[j * B + c] = be;
          S.sc[(j + 1) * B + c] = be > 0.0 ? 1.0 / be : 0.0;
          S.fc[c] = make_float2((float)S.sc[(j + 1) * B + c], 0.f);  // the next step's staging
        }
        __syncthreads();
      }
      // convergence check on T of dimension j1: warp b checks column b.  Fused (every column's
      // eigenvector matrix fits region A at once): the check runs the full eigendecomposition,
      // and the accepted basis takes its coefficients from it (on GB300 the FP64-bound
      // rows-only and full eigensolves cost about the same); otherwise rows 0 and j1-1 only.
      {
        const long long t0 = clk();
        const int wp = tid >> 5, lane = tid & 31;
        if (wp < B) {
          const int b = wp;
          double *d, *e, *q0, *qm;
          bool ok = true;
          if (fused) {
            double* Qm = reinterpret_cast<double*>(S.A) + (size_t)b * fstride;
            d = Qm + (size_t)m * m;
            e = d + m;
            for (int k = lane; k < j1; k += 32) {
              d[k] = S.alpha[k * B + b];
              e[k] = k + 1 < j1 ? S.beta[k * B + b] : 0.0;
            }
            __syncwarp();
            ok = tridiag_eig_warp(j1, d, e, Qm, e + 3 * m);
            q0 = Qm;
            qm = Qm + (size_t)(j1 - 1) * j1;
          } else {
            d = reinterpret_cast<double*>(S.A) + (size_t)b * 4 * m;
            e = d + m;
            q0 = e + m;
            qm = q0 + m;
            for (int k = lane; k < j1; k += 32) {
              d[k] = S.alpha[k * B + b];
              e[k] = k + 1 < j1 ? S.beta[k * B + b] : 0.0;
            }
            __syncwarp();
            if (lane == 0) ok = tridiag_eig_rows(j1, d, e, q0, qm);
            ok = __shfl_sync(0xffffffffu, ok, 0);
            __syncwarp();
          }
          if (!ok && lane == 0) atomicOr(&S.ctl->status, 2);
          const double bl = S.beta[(j1 - 1) * B + b];
          const double s = select_step(j1, d, q0, qm, bl, s_rem, tol, zr, zi, kBisect);
          if (lane == 0) S.sb[b] = s;
        }
        __syncthreads();
        if (tid == 0) {
          double s = S.sb[0];
          for (int b = 1; b < B; ++b) s = fmin(s, S.sb[b]);
          S.ctl->s_acc = s;
        }
        __syncthreads();
        s_acc = S.ctl->s_acc;
        pc.cy[1] += clk() - t0;
        ++pc.nck;
      }
      if (S.ctl->status & 3) return;
      if (j1 == m || s_acc >= s_rem) {
        m_eff = j1;
        break;
      }
      j0 = j1;
      j1 = min(m, j1 + it.every);
    }
    s_acc = fmin(s_acc, s_rem);
    if (!(s_acc > 1e-13 * s_rem) && !(s_acc >= s_rem)) {
      if (tid == 0) S.ctl->status |= 4;
      __syncthreads();
      return;
    }
    const bool final_basis = s_acc >= s_rem || s_done + s_acc * (1.0 + 1e-13) >= 1.0;
    // full eigendecomposition of the accepted basis (unless the last check made it) and the
    // combination coefficients
    //   cc[k][b] = beta0_b sum_l Q_b[k][l] e^{s_acc z theta_l} Q_b[0][l]   (as k_tridiag_coef)
    {
      const long long t0 = clk();
      const int wp = tid >> 5, lane = tid & 31;
      for (int r0 = 0; r0 < B; r0 += a.L.ncol) {
        const int b = r0 + wp;
        if (wp < a.L.ncol && b < B) {
          double* Qm = reinterpret_cast<double*>(S.A) + (size_t)wp * fstride;
          double* d = Qm + (size_t)m * m;
          double* e = d + m;
          double* fg = e + m;     // 2 m doubles
          double* rot = fg + 2 * m;
          if (!fused) {
            for (int k = lane; k < m_eff; k += 32) {
              d[k] = S.alpha[k * B + b];
              e[k] = k + 1 < m_eff ? S.beta[k * B + b] : 0.0;
            }
            __syncwarp();
            const bool ok = tridiag_eig_warp(m_eff, d, e, Qm, rot);
            if (!ok && lane == 0) atomicOr(&S.ctl->status, 2);
          }
          for (int l = lane; l < m_eff; l += 32) {
            const double2 f = cexp_scaled(s_acc, zr, zi, d[l]);
            const double g = Qm[l];  // row 0
            fg[2 * l] = f.x * g;
            fg[2 * l + 1] = f.y * g;
          }
          __syncwarp();
          const double b0 = S.beta0[b];
          for (int k = lane; k < m_eff; k += 32) {
            double re = 0.0, im = 0.0;
            for (int l = 0; l < m_eff; ++l) {
              const double q = Qm[(size_t)k * m_eff + l];
              re = fma(q, fg[2 * l], re);
              im = fma(q, fg[2 * l + 1], im);
            }
            S.cc[k * B + b] = make_double2(b0 * re, b0 * im);
          }
        }
        __syncthreads();
      }
      pc.cy[2] += clk() - t0;
      if (!fused) ++pc.neig;
    }
    if (S.ctl->status & 3) return;
    for (int e = tid; e < m_eff * B; e += kPNT) {
      const double2 ck = S.cc[e];
      const double f = S.sc[e];
      S.fc[3 * B + e] = make_float2((float)(ck.x * f), (float)(ck.y * f));
    }
    __syncthreads();
    // out = sum_{k < m_eff} cc_k sc_k u_k (in place when out aliases the current state: each
    // element is read and then written by the same thread)
    for (int r = tid; r < D; r += kPNT) {
#pragma unroll
      for (int q = 0; q < npairs(B); ++q) {
        const int c0 = B >= 2 ? 2 * q : 0, c1 = B >= 2 ? 2 * q + 1 : 0;
        float2 a0 = make_float2(0.f, 0.f), a1 = make_float2(0.f, 0.f);
        for (int k = 0; k < m_eff; ++k) {
          float2 v0, v1;
          ld_pair<B>(U(k) + (size_t)r * B, q, v0, v1);
          const float2 k0 = S.fc[(3 + k) * B + c0], k1 = S.fc[(3 + k) * B + c1];
          cmac(a0, k0.x, k0.y, v0);
          cmac(a1, k1.x, k1.y, v1);
        }
        st_pair<B>(out + (size_t)r * B, q, a0, a1);
      }
    }
    __syncthreads();
    if (final_basis) {
      s_rem = 0.0;
    } else {
      s_done += s_acc;
      s_rem -= s_acc;
      cur = out;
    }
  }
}

// ---------------------------------------------------------------- the persistent kernel
// Chain of syk_otoc with rho split into quarters (Eq. F_reg):
//   ua = rho^{1/8} psi~, ub = rho^{1/4} chi_j ua; per time t_k: ua, ub advanced by U(t_k - t_{k-1}),
//   pr = rho^{1/4} U(t_k)^dag chi_i ua, qs = rho^{1/4} U(t_k)^dag chi_i ub, F_k = <pr | chi_j qs>.
template <int B, int RPT>
__global__ void __launch_bounds__(kPNT, 1) k_otoc_items(const __grid_constant__ PArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  PSmem S(smem, a.L);
  const int tid = threadIdx.x;
  const size_t vmax = (size_t)a.vmax;
  float2* base = a.ws + (size_t)blockIdx.x * ((size_t)(a.m + 5) * vmax + (size_t)a.cmax);
  float2* basis = base;
  float2* ua = base + (size_t)a.m * vmax;
  float2* ub = ua + vmax;
  float2* pr = ub + vmax;
  float2* qs = pr + vmax;
  float2* tmp = qs + vmax;
  float* dgs = reinterpret_cast<float*>(tmp + vmax);  // 2 D floats, then 2 n2 D float2 (cta_coef)
  float2* pcs = nullptr;
  for (;;) {
    if (tid == 0) {
      S.ctl->item = atomicAdd(a.next, 1);
      S.ctl->status = 0;
    }
    __syncthreads();
    const int q = S.ctl->item;
    if (q >= a.nitems) break;
    const PItem it = a.items[q];
    const long long t_all = clk();
    PCount pc = {{0, 0, 0}, 0, 0, 0, 0};
    pcs = tmp + vmax + (size_t)it.D;  // after the 2 D diagonal floats
    cta_coef(it, dgs, pcs);
    const double be = it.beta;
    const int n = it.n, D = it.D;
    bool failed = false;
    auto bad = [&]() -> bool { return (S.ctl->status) != 0; };
    cta_expmv<B, RPT>(a, it, 0, -be / 8.0, 0.0, it.psi0, ua, basis, S, pc, dgs, pcs);
    failed = bad();
    if (!failed) {
      cta_chi<B>(n, D, a.j, 1, ua, tmp);
      cta_expmv<B, RPT>(a, it, 1, -be / 4.0, 0.0, tmp, ub, basis, S, pc, dgs, pcs);
      failed = bad();
    }
    double tcur = 0.0;
    for (int k = 0; k < a.nt && !failed; ++k) {
      const double tk = a.t[k], dt = tk - tcur;
      if (dt > 0.0) {
        cta_expmv<B, RPT>(a, it, 0, 0.0, -dt, ua, ua, basis, S, pc, dgs, pcs);
        if ((failed = bad())) break;
        cta_expmv<B, RPT>(a, it, 1, 0.0, -dt, ub, ub, basis, S, pc, dgs, pcs);
        if ((failed = bad())) break;
        tcur = tk;
      }
      cta_chi<B>(n, D, a.i, 1, ua, pr);  // p (odd)
      cta_chi<B>(n, D, a.i, 0, ub, qs);  // q (even)
      cta_expmv<B, RPT>(a, it, 1, -be / 4.0, tk, pr, pr, basis, S, pc, dgs, pcs);
      if ((failed = bad())) break;
      cta_expmv<B, RPT>(a, it, 0, -be / 4.0, tk, qs, qs, basis, S, pc, dgs, pcs);
      if ((failed = bad())) break;
      cta_chi<B>(n, D, a.j, 1, qs, tmp);  // chi_j s (odd)
      cta_dot<B>(pr, tmp, D, S, S.h);
      if (tid < B) it.F[(size_t)k * it.Fld + tid] = S.h[tid];
      __syncthreads();
    }
    if (tid == 0) {
      long long* st = a.stat + (size_t)q * kStWords;
      st[kStStatus] = S.ctl->status;
      st[kStMatvecs] = pc.mv;
      st[kStBases] = pc.nb;
      st[kStCyMatvec] = pc.cy[0];
      st[kStCyCheck] = pc.cy[1];
      st[kStCyEig] = pc.cy[2];
      st[kStCyAll] = clk() - t_all;
      st[kStChecks] = pc.nck;
      st[kStEigs] = pc.neig;
    }
    __syncthreads();  // ctl is rewritten by the next item
  }
}

using KFn = void (*)(PArgs);
KFn kernel_for(int B) {
  switch (B) {
    case 1: return k_otoc_items<1, 4>;
    case 2: return k_otoc_items<2, 4>;
    case 4: return k_otoc_items<4, 2>;
    case 8: return k_otoc_items<8, 2>;
    case 16: return k_otoc_items<16, 1>;
    default: return nullptr;
  }
}

size_t a16(size_t v) { return (v + 15) & ~size_t(15); }

// Shared-memory layout for items of at most vmax elements per vector, batch B, Krylov m;
// returns false if it exceeds `limit` bytes.
bool make_layout(long long vmax, int B, int m, int limit, PLayout* L) {
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off += a16(bytes);
    return (int)o;
  };
  const size_t vec = (size_t)vmax * sizeof(float2);
  const size_t chk = (size_t)B * 4 * m * sizeof(double);
  const size_t fcol = ((size_t)m * m + 4 * (size_t)m + 2) * sizeof(double);
  // everything but region A
  size_t rest = 0;
  {
    const size_t parts[] = {kPG * sizeof(uint4),           kPG * 32 * sizeof(float2),   (size_t)m * B * 8,
                            (size_t)m * B * 8,              (size_t)(m + 1) * B * 8,     (size_t)B * 8,
                            (size_t)B * 16,                 (size_t)B * 16,              (size_t)m * B * 16,
                            (size_t)kPWarps * B * 16,       (size_t)B * 8,               (size_t)(m + 3) * B * 8,
                            sizeof(PCtl)};
    for (size_t p : parts) rest += a16(p);
  }
  int ncol = std::min(B, kPWarps);
  const size_t a0 = std::max(vec, chk);
  while (ncol > 1 && rest + a16(std::max(a0, ncol * fcol)) > (size_t)limit) --ncol;
  const size_t A = a16(std::max(a0, ncol * fcol));
  if (rest + A > (size_t)limit) return false;
  L->A = take(A);
  L->rec = take(kPG * sizeof(uint4));
  L->tab = take(kPG * 32 * sizeof(float2));
  L->alpha = take((size_t)m * B * 8);
  L->beta = take((size_t)m * B * 8);
  L->sc = take((size_t)(m + 1) * B * 8);
  L->beta0 = take((size_t)B * 8);
  L->h = take((size_t)B * 16);
  L->n2 = take((size_t)B * 16);
  L->cc = take((size_t)m * B * 16);
  L->red = take((size_t)kPWarps * B * 16);
  L->sb = take((size_t)B * 8);
  L->fc = take((size_t)(m + 3) * B * 8);
  L->ctl = take(sizeof(PCtl));
  L->total = (int)off;
  L->ncol = ncol;
  return true;
}

std::atomic<int> g_persistent{1};
std::mutex g_report_mtx;
long long g_report[kBatchReportWords] = {};

}  // namespace

bool batch_persistent_enabled() { return g_persistent.load() != 0; }
bool batch_persistent_split_always() { return g_persistent.load() == 2; }

int smem_optin_limit() {
  int dev = 0, v = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 48 * 1024;
  if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess || v <= 0)
    return 48 * 1024;
  return v;
}

// States per CTA of the persistent launch for an item of n spins (sector dimension D) with B
// states, Krylov dimension m and `limit` bytes of shared memory per CTA: the largest power of
// two bs <= 16 dividing B whose layout fits (bs = 1 only for one-state items); 0 if none.
// *smem gets that layout's bytes.  Host arithmetic only.
int persistent_states_for(int64_t D, int n, int64_t B, int m, int limit, int* smem) {
  if (B < 1 || n < 2) return 0;
  for (int bs = 16; bs >= 1; bs >>= 1) {
    if (B % bs != 0 || (bs == 1 && B > 1)) continue;
    PLayout L;
    if (make_layout((long long)D * bs, bs, m, limit, &L)) {
      if (smem) *smem = L.total;
      return bs;
    }
  }
  return 0;
}

int batch_item_persistent_states(const syk_terms* t, int64_t B, const void* psi0, int dtype, int m) {
  if (!batch_persistent_enabled() || dtype != SYK_C64 || lanczos_orth(SYK_C64) != kOrthLocal) return 0;
  (void)psi0;  // every sub-item gets its own aligned device copy of its columns
  return persistent_states_for(t->D, t->n, B, m, smem_optin_limit(), nullptr);
}

// Runs the items of idx, each split into sub-items of Bs states (columns b0 .. b0 + Bs - 1 of
// its D x nstates input, copied into an aligned device buffer of their own), as one
// persistent launch on stream st; fills each item's host F_re_im and status.  Synchronises st.
int otoc_batch_persistent(const syk_otoc_item* items, const std::vector<int>& idx, int64_t Bs, int i, int j,
                          const double* t, int nt, int m, double tol, int* item_status, cudaStream_t st,
                          long long* report) {
  if (idx.empty()) return SYK_OK;
  KFn fn = kernel_for((int)Bs);
  if (!fn) {
    set_error("persistent batch: unsupported states per CTA %lld", (long long)Bs);
    return SYK_EINVAL;
  }
  // sub-items (item, first column), largest sectors first so that the long ones do not form the tail
  struct Sub {
    int k;
    int64_t b0;
  };
  std::vector<Sub> subs;
  for (int k : idx)
    for (int64_t b0 = 0; b0 < items[k].nstates; b0 += Bs) subs.push_back({k, b0});
  std::stable_sort(subs.begin(), subs.end(),
                   [&](const Sub& x, const Sub& y) { return items[x.k].terms->D > items[y.k].terms->D; });
  const int ni = (int)subs.size();
  long long vmax = 0, cmax = 0;
  for (const Sub& u : subs) {
    const syk_terms* T = items[u.k].terms;
    vmax = std::max<long long>(vmax, (long long)T->D * Bs);
    cmax = std::max<long long>(cmax, (long long)T->D * (1 + 2LL * T->n2));
  }
  PLayout L;
  if (!make_layout(vmax, (int)Bs, m, smem_optin_limit(), &L)) {
    set_error("persistent batch: items do not fit in shared memory");
    return SYK_EINVAL;
  }
  const int grid = std::min(ni, sm_count());
  Scratch sc(st);
  void *d_items, *d_stat, *d_next, *d_t, *d_F, *d_ws;
  size_t fsize = 0;  // device results: nt x nstates per item, in idx order
  std::vector<size_t> foff(idx.size());
  for (size_t q = 0; q < idx.size(); ++q) {
    foff[q] = fsize;
    fsize += (size_t)nt * items[idx[q]].nstates;
  }
  auto item_slot = [&](int k) {
    return (size_t)(std::find(idx.begin(), idx.end(), k) - idx.begin());
  };
  SYK_TRY(sc.alloc(&d_items, sizeof(PItem) * ni));
  SYK_TRY(sc.alloc(&d_stat, sizeof(long long) * kStWords * ni));
  SYK_TRY(sc.alloc(&d_next, sizeof(int)));
  SYK_TRY(sc.alloc(&d_t, sizeof(double) * nt));
  SYK_TRY(sc.alloc(&d_F, sizeof(double2) * fsize));
  SYK_TRY(sc.alloc(&d_ws, sizeof(float2) * ((size_t)vmax * (m + 5) + (size_t)cmax) * grid));
  std::vector<PItem> h(ni);
  std::vector<size_t> sub_slot(ni);
  for (int q = 0; q < ni; ++q) {
    const syk_otoc_item& itm = items[subs[q].k];
    const syk_terms* T = itm.terms;
    const int64_t B = itm.nstates, b0 = subs[q].b0;
    ApplyParams P;
    SYK_TRY(make_apply_params(T, 0, SYK_C64, &P));
    void* psi = nullptr;
    SYK_TRY(sc.alloc(&psi, sizeof(float2) * (size_t)T->D * Bs));
    SYK_CUDA_CHECK(cudaMemcpy2DAsync(psi, sizeof(float2) * Bs, static_cast<const float2*>(itm.psi0) + b0,
                                     sizeof(float2) * B, sizeof(float2) * Bs, (size_t)T->D, cudaMemcpyDefault, st));
    sub_slot[q] = item_slot(subs[q].k);
    PItem& p = h[q];
    p.m4_rec = P.m4_rec;
    p.m4_t32 = static_cast<const float2*>(P.m4_tab);
    p.m2_rec = P.m2_rec;
    p.m2_t32 = static_cast<const float2*>(P.m2_tab);
    p.wd32 = static_cast<const float*>(P.wd);
    p.psi0 = static_cast<const float2*>(psi);
    p.F = static_cast<double2*>(d_F) + foff[sub_slot[q]] + b0;
    p.Fld = (int)B;
    p.beta = itm.beta;
    p.rho = T->rho_est;
    p.n = T->n;
    p.D = (int)T->D;
    p.n4 = T->n4;
    p.n2 = T->n2;
    // Check plan from the measured costs in this kernel: a convergence check (FP64 eigensolves
    // of Bs columns sharing the SM's FP64 pipe) ~0.6 + 0.05 Bs ms; a matvec ~(0.10 + 0.035 Bs)
    // ns per row x mask pair.  The later checks come every ~sqrt(16 ratio) vectors (the
    // expected overshoot of a few vectors against the checks saved), the first at 3/4 of the
    // predicted dimension when checks are cheap, 7/8 or all of it when they are not.
    const double mv_ms = double(T->D) * double(T->n4 + T->n2 + 1) * (0.10 + 0.035 * double(Bs)) * 1e-6;
    const double ratio = (0.6 + 0.05 * double(Bs)) / std::max(mv_ms, 1e-6);
    p.every = std::max(2, std::min(8, (int)std::lround(std::sqrt(16.0 * ratio))));
    p.first8 = ratio < 1.0 ? 6 : ratio < 4.0 ? 7 : 8;
  }
  SYK_CUDA_CHECK(cudaMemcpyAsync(d_items, h.data(), sizeof(PItem) * ni, cudaMemcpyHostToDevice, st));
  SYK_CUDA_CHECK(cudaMemcpyAsync(d_t, t, sizeof(double) * nt, cudaMemcpyHostToDevice, st));
  PArgs a;
  a.items = static_cast<const PItem*>(d_items);
  a.nitems = ni;
  a.next = static_cast<int*>(d_next);
  a.stat = static_cast<long long*>(d_stat);
  a.t = static_cast<const double*>(d_t);
  a.nt = nt;
  a.i = i;
  a.j = j;
  a.m = m;
  a.tol = tol;
  a.bt = 64.0 * 5.96e-8;
  a.ws = static_cast<float2*>(d_ws);
  a.vmax = vmax;
  a.cmax = cmax;
  a.L = L;
  SYK_TRY(ensure_smem_limit(reinterpret_cast<const void*>(fn), L.total));
  // the queue reset and the persistent launch, as one CUDA graph
  cudaGraph_t g = nullptr;
  cudaGraphExec_t ge = nullptr;
  SYK_CUDA_CHECK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
  cudaMemsetAsync(d_next, 0, sizeof(int), st);
  fn<<<grid, kPNT, L.total, st>>>(a);
  const cudaError_t el = cudaGetLastError();
  const cudaError_t ec = cudaStreamEndCapture(st, &g);
  if (el != cudaSuccess || ec != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    set_error("persistent batch: capture failed: %s", cudaGetErrorString(el != cudaSuccess ? el : ec));
    return SYK_ECUDA;
  }
  const cudaError_t ei = cudaGraphInstantiate(&ge, g, 0);
  cudaGraphDestroy(g);
  if (ei != cudaSuccess) {
    set_error("persistent batch: graph instantiation failed: %s", cudaGetErrorString(ei));
    return SYK_ECUDA;
  }
  const cudaError_t eg = cudaGraphLaunch(ge, st);
  count_launch(1);
  std::vector<long long> hst((size_t)kStWords * ni);
  std::vector<double2> hF(fsize);
  cudaError_t e1 = eg;
  if (e1 == cudaSuccess) e1 = cudaMemcpyAsync(hst.data(), d_stat, sizeof(long long) * hst.size(), cudaMemcpyDeviceToHost, st);
  if (e1 == cudaSuccess) e1 = cudaMemcpyAsync(hF.data(), d_F, sizeof(double2) * hF.size(), cudaMemcpyDeviceToHost, st);
  const cudaError_t e2 = cudaStreamSynchronize(st);
  cudaGraphExecDestroy(ge);
  if (e1 != cudaSuccess || e2 != cudaSuccess) {
    set_error("persistent batch: %s", cudaGetErrorString(e1 != cudaSuccess ? e1 : e2));
    return SYK_ECUDA;
  }
  // per item: the OR of its sub-items' error bits
  std::vector<int> bits(idx.size(), 0);
  long long tot[kStWords] = {};
  long long mv_flops = 0;  // algorithmic matvec work: 8 flops per nonzero of H_s per state
  for (int q = 0; q < ni; ++q) {
    const long long* w = &hst[(size_t)q * kStWords];
    bits[sub_slot[q]] |= (int)w[kStStatus];
    for (int e = 1; e < kStWords; ++e) tot[e] += w[e];
    const syk_terms* T = items[subs[q].k].terms;
    mv_flops += w[kStMatvecs] * 8LL * T->D * (long long)(T->n4 + T->n2 + 1) * Bs;
  }
  int rc = SYK_OK;
  for (size_t q = 0; q < idx.size(); ++q) {
    const int k = idx[q];
    int irc = SYK_OK;
    if (bits[q]) {
      irc = SYK_ENUMERIC;
      if (rc == SYK_OK) {
        set_error("persistent batch: item %d: %s", k,
                  (bits[q] & 1) ? "non-finite Lanczos scalar"
                                : (bits[q] & 2) ? "tridiagonal eigensolver did not converge"
                                                : "Krylov step collapsed or too many bases; raise krylov_dim or tol");
        rc = irc;
      }
    }
    if (item_status) item_status[k] = irc;
    double* F = items[k].F_re_im;
    const size_t ne = (size_t)nt * items[k].nstates;
    for (size_t e = 0; e < ne; ++e) {
      F[2 * e] = hF[foff[q] + e].x;
      F[2 * e + 1] = hF[foff[q] + e].y;
    }
  }
  count_applies(tot[kStMatvecs] * Bs);
  count_bases(tot[kStBases]);
  if (report) {
    report[0] += (long long)idx.size();
    report[10] += ni;
    report[11] += mv_flops;
    report[2] += grid;
    report[3] += tot[kStCyMatvec];
    report[4] += tot[kStCyCheck];
    report[5] += tot[kStCyEig];
    report[6] += tot[kStCyAll];
    report[7] += tot[kStMatvecs] * Bs;
    report[8] += tot[kStChecks];
    report[9] += tot[kStEigs];
  }
  return rc;
}

void batch_report_store(const long long* r) {
  std::lock_guard<std::mutex> lk(g_report_mtx);
  for (int k = 0; k < kBatchReportWords; ++k) g_report[k] = r[k];
}

void batch_report_load(long long* r) {
  std::lock_guard<std::mutex> lk(g_report_mtx);
  for (int k = 0; k < kBatchReportWords; ++k) r[k] = g_report[k];
}

}  // namespace syk

extern "C" int syk_batch_persistent(int on) {
  if (on < 0 || on > 2) {
    syk::set_error("syk_batch_persistent: mode must be 0, 1 or 2 (got %d)", on);
    return SYK_EINVAL;
  }
  return syk::g_persistent.exchange(on);
}

extern "C" int syk_batch_plan(int N, int64_t nstates, int krylov_dim, int smem_limit, int* states_per_cta,
                              int* smem_per_cta) {
  if (N < 4 || N > 62 || (N & 1) || nstates < 1 || krylov_dim < 2 || krylov_dim > SYK_MAX_KRYLOV ||
      !states_per_cta) {
    syk::set_error("syk_batch_plan: need even 4 <= N <= 62, nstates >= 1, 2 <= krylov_dim <= %d and an output",
                   SYK_MAX_KRYLOV);
    return SYK_EINVAL;
  }
  const int n = N / 2;
  const int limit = smem_limit > 0 ? smem_limit : syk::smem_optin_limit();
  int smem = 0;
  *states_per_cta = syk::persistent_states_for(int64_t(1) << (n - 1), n, nstates, krylov_dim, limit, &smem);
  if (smem_per_cta) *smem_per_cta = *states_per_cta > 0 ? smem : 0;
  return SYK_OK;
}

extern "C" int syk_batch_report(long long* out, int n) {
  if (!out || n < 1) {
    syk::set_error("syk_batch_report: need an output array");
    return SYK_EINVAL;
  }
  long long r[syk::kBatchReportWords];
  syk::batch_report_load(r);
  for (int k = 0; k < n && k < syk::kBatchReportWords; ++k) out[k] = r[k];
  return SYK_OK;
}
