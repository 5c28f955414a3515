// Krylov expmv (Supp. Sec. I.B): Lanczos basis with full classical Gram-Schmidt
// reorthogonalisation (two passes for complex128, one for complex64) (K2 + K7), eigendecomposition of the FP64
// tridiagonal projection and its exponential (K3), and the combination
// psi_out = V c (K4).  All scalars are FP64; complex64 vectors use FP32
// arithmetic with FP64 accumulation of every reduction.
//
// Vector kernels use blockDim = B * floor(256/B) threads, so thread t always
// works on batch column t % B, and a fixed number G of blocks; each block
// writes one partial sum per (vector, column), summed in a fixed order by a
// second kernel (results are deterministic).
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <set>
#include <tuple>

#include "syk_cplx.cuh"
#include "syk_krylov.cuh"
#include "syk_tridiag.cuh"

namespace syk {
namespace {

// Reduction kernels run 2 blocks per SM of the current device; workspaces are sized for up to
// kRedBlocksCap blocks so that their size does not depend on the device.
constexpr int kRedBlocksCap = 512;
constexpr int kFlush = 16;          // FP32 partial sums are flushed to FP64 every kFlush elements

inline int vec_bdim(int64_t B) { return int(B) * std::max(1, int(256 / B)); }
inline int red_grid(int64_t total, int bdim, int max_blocks) {
  return int(std::min<int64_t>((total + bdim - 1) / bdim, max_blocks));
}

// ---------------------------------------------------------------- reductions
// Accumulates sum conj(a) * b.  FP32 data: products and short partial sums in
// FP32, flushed into FP64 every kFlush elements.  FP64 data: FP64 throughout.
template <typename R>
struct DotAcc;
template <>
struct DotAcc<double> {
  double re = 0, im = 0;
  __device__ void add(double2 a, double2 b) {
    re = fma(a.x, b.x, fma(a.y, b.y, re));
    im = fma(a.x, b.y, fma(-a.y, b.x, im));
  }
  __device__ void tick() {}
  __device__ double2 get() { return make_double2(re, im); }
};
template <>
struct DotAcc<float> {
  double re = 0, im = 0;
  float fr = 0.f, fi = 0.f;
  int cnt = 0;
  __device__ void add(float2 a, float2 b) {
    fr = fmaf(a.x, b.x, fmaf(a.y, b.y, fr));
    fi = fmaf(a.x, b.y, fmaf(-a.y, b.x, fi));
  }
  __device__ void tick() {
    if (++cnt == kFlush) {
      re += fr;
      im += fi;
      fr = fi = 0.f;
      cnt = 0;
    }
  }
  __device__ double2 get() { return make_double2(re + fr, im + fi); }
};

// Block-level reduction of one double2 per thread into one value per column:
// thread t < B gets the sum over threads t, t+B, t+2B, ... in that order.
__device__ double2 block_reduce_cols(double2 v, int B, double2* sm) {
  sm[threadIdx.x] = v;
  __syncthreads();
  double2 r = make_double2(0.0, 0.0);
  if ((int)threadIdx.x < B) {
    for (int t = threadIdx.x; t < (int)blockDim.x; t += B) {
      r.x += sm[t].x;
      r.y += sm[t].y;
    }
  }
  __syncthreads();
  return r;
}

// part[(k*G + g)*B + b] = sum over this block's elements of conj(V_k) w, for
// k in [KC*blockIdx.y, min(nk, KC*(blockIdx.y+1))): w is read once per KC vectors.
constexpr int KC = 8;
template <typename R>
__global__ void k_dots(int nk, const typename CT<R>::T* __restrict__ V, size_t vs,
                       const typename CT<R>::T* __restrict__ w, int64_t total, int B, double2* __restrict__ part) {
  extern __shared__ double2 sm[];
  const int k0 = KC * blockIdx.y;
  const int kc = min(KC, nk - k0);
  DotAcc<R> acc[KC];
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const typename CT<R>::T we = w[e];
#pragma unroll
    for (int j = 0; j < KC; ++j)
      if (j < kc) {
        acc[j].add(V[(size_t)(k0 + j) * vs + e], we);
        acc[j].tick();
      }
  }
  for (int j = 0; j < kc; ++j) {
    double2 r = block_reduce_cols(acc[j].get(), B, sm);
    if ((int)threadIdx.x < B) part[((size_t)(k0 + j) * gridDim.x + blockIdx.x) * B + threadIdx.x] = r;
  }
}

// out[k*B + b] = sc[k*B + b] * sum_g part[(k*G + g)*B + b] for k < nk (sc NULL: 1): one warp
// per (k, b) in the first nwb blocks (8 warps each).  If ep_part is given, each of the B
// blocks after them sums the matvec epilogue's partials of one column b over its *ep_nblk
// CTAs (256 threads, strided, then a fixed tree) into out[ep_k*B + b] = sc[ep_k*B + b] * sum,
// and, with beta_prev, also sets out[(ep_k-1)*B + b] = (beta_prev[b], 0) (the three-term
// recurrence's coefficient of v_{ep_k-1}).  The epilogue's result goes to index ep_k (nk for
// Gram-Schmidt, which projects on v_0..v_{nk-1} before it).  Deterministic order throughout.
__global__ void k_reduce_parts(int nk, int G, int B, int nwb, const double2* __restrict__ part,
                               const double* __restrict__ sc, int ep_k, const double2* __restrict__ ep_part,
                               const int* __restrict__ ep_nblk, const double* __restrict__ beta_prev,
                               double2* __restrict__ out) {
  __shared__ double2 red[256];
  if ((int)blockIdx.x >= nwb) {
    const int b = (int)blockIdx.x - nwb;
    const int ng = *ep_nblk;
    double sx = 0.0, sy = 0.0;
    for (int g = threadIdx.x; g < ng; g += blockDim.x) {
      const double2 p = ep_part[(size_t)g * B + b];
      sx += p.x;
      sy += p.y;
    }
    red[threadIdx.x] = make_double2(sx, sy);
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
      if ((int)threadIdx.x < h) {
        red[threadIdx.x].x += red[threadIdx.x + h].x;
        red[threadIdx.x].y += red[threadIdx.x + h].y;
      }
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      const double f = sc ? sc[ep_k * B + b] : 1.0;
      out[ep_k * B + b] = make_double2(f * red[0].x, f * red[0].y);
      if (beta_prev && ep_k > 0) out[(ep_k - 1) * B + b] = make_double2(beta_prev[b], 0.0);
    }
    return;
  }
  const int idx = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (idx >= nk * B) return;
  const int k = idx / B, b = idx - k * B;
  double sx = 0.0, sy = 0.0;
  for (int g = lane; g < G; g += 32) {
    const double2 p = part[((size_t)k * G + g) * B + b];
    sx += p.x;
    sy += p.y;
  }
  for (int o = 16; o > 0; o >>= 1) {
    sx += __shfl_xor_sync(0xffffffffu, sx, o);
    sy += __shfl_xor_sync(0xffffffffu, sy, o);
  }
  const double f = sc ? sc[idx] : 1.0;
  if (lane == 0) out[idx] = make_double2(f * sx, f * sy);
}

// dst = w - sum_{k0<=k<k1} h_k v_k with v_k = sc_k V_k (per column; dst may be w);
// npart[g*B + b] = partial |dst|^2
template <typename R>
__global__ void k_update(int k0, int k1, const typename CT<R>::T* __restrict__ V, size_t vs,
                         const double2* __restrict__ h, const double* __restrict__ sc, const typename CT<R>::T* w,
                         typename CT<R>::T* dst, int64_t total, int B, double* __restrict__ npart) {
  using C = typename CT<R>::T;
  extern __shared__ double2 sm[];
  const int b = threadIdx.x % B;
  DotAcc<R> acc;
  // U elements per thread and pass (same column: the stride is a multiple of B), so that the
  // loads of w and of every basis vector for all U are in flight together
  constexpr int U = 4;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e0 < total; e0 += U * stride) {
    C x[U];
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (e0 + u * stride < total) x[u] = w[e0 + u * stride];
    for (int k = k0; k < k1; ++k) {
      const double2 hk = h[k * B + b];
      const double f = sc[k * B + b];
      const R cr = R(-hk.x * f), ci = R(-hk.y * f);
      const C* __restrict__ Vk = V + (size_t)k * vs;
#pragma unroll
      for (int u = 0; u < U; ++u)
        if (e0 + u * stride < total) cmac(x[u], cr, ci, Vk[e0 + u * stride]);
    }
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (e0 + u * stride < total) {
        dst[e0 + u * stride] = x[u];
        acc.add(x[u], x[u]);
        acc.tick();
      }
  }
  double2 r = block_reduce_cols(acc.get(), B, sm);
  if ((int)threadIdx.x < B && npart) npart[(size_t)blockIdx.x * B + threadIdx.x] = r.x;
}

template <typename R>
__global__ void k_scale(const typename CT<R>::T* __restrict__ src, typename CT<R>::T* __restrict__ dst,
                        const double* __restrict__ inv, int64_t total, int B) {
  const int b = threadIdx.x % B;
  const R s = R(inv[b]);
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    typename CT<R>::T v = src[e];
    v.x *= s;
    v.y *= s;
    dst[e] = v;
  }
}

// out = sum_{k<nk} c_k v_k with v_k = sc_k V_k (per column)
template <typename R>
__global__ void k_combine(int nk, const typename CT<R>::T* __restrict__ V, size_t vs, const double2* __restrict__ c,
                          const double* __restrict__ sc, typename CT<R>::T* __restrict__ out, int64_t total, int B) {
  using C = typename CT<R>::T;
  const int b = threadIdx.x % B;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    C x = make_c<R>(R(0), R(0));
    for (int k = 0; k < nk; ++k) {
      const double2 ck = c[k * B + b];
      const double f = sc[k * B + b];
      cmac(x, R(ck.x * f), R(ck.y * f), V[(size_t)k * vs + e]);
    }
    out[e] = x;
  }
}

// beta0 = ||psi||, inv = 1/beta0 (0 for a zero column)
__global__ void k_norm_init(int B, const double2* __restrict__ d, double* __restrict__ beta0, double* __restrict__ inv,
                            double* __restrict__ sc, int* status) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  sc[b] = 1.0;  // v_0 is stored normalised
  const double n2 = d[b].x;
  const double nb = sqrt(fmax(n2, 0.0));
  if (!isfinite(nb)) atomicOr(status, 1);
  beta0[b] = nb;
  inv[b] = nb > 0.0 ? 1.0 / nb : 0.0;
}

// alpha_j = Re(h1_j + h2_j), beta_j = ||w||; breakdown sets beta_j = 0.  One warp per column:
// the G partial norms are summed lane-strided, then by a fixed shuffle tree.
__global__ void k_lanczos_scalars(int j, int B, int G, const double2* __restrict__ h1, const double2* __restrict__ h2,
                                  const double* __restrict__ npart, double* __restrict__ alpha,
                                  double* __restrict__ beta, double* __restrict__ inv, double* __restrict__ sc,
                                  int* status, double bt) {
  const int b = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (b >= B) return;
  double n2 = 0.0;
  for (int g = lane; g < G; g += 32) n2 += npart[(size_t)g * B + b];
  for (int o = 16; o > 0; o >>= 1) n2 += __shfl_xor_sync(0xffffffffu, n2, o);
  if (lane != 0) return;
  const double a = h1[j * B + b].x + (h2 ? h2[j * B + b].x : 0.0);
  double be = sqrt(fmax(n2, 0.0));
  if (!isfinite(a) || !isfinite(be)) {
    atomicOr(status, 1);
    be = 0.0;
  }
  const double prev = j > 0 ? beta[(j - 1) * B + b] : 0.0;
  if (be <= bt * (fabs(a) + prev)) be = 0.0;
  alpha[j * B + b] = isfinite(a) ? a : 0.0;
  beta[j * B + b] = be;
  inv[b] = be > 0.0 ? 1.0 / be : 0.0;
  sc[(j + 1) * B + b] = inv[b];  // v_{j+1} = u_{j+1} / beta_j
}

// One block (one warp) per batch column: eigendecomposition of T_b and the largest
// s <= s_target whose error estimate is <= tol.  FULL: the whole eigenvector matrix (for the
// combination coefficients), written to Qout; otherwise only rows 0 and m-1 (a convergence
// check), computed by lane 0 alone.  Shared memory: m^2 + 2m + 2 doubles (FULL) or 4m.
template <bool FULL>
__device__ void tridiag_eig_block(int m, int B, const double* __restrict__ alpha, const double* __restrict__ beta,
                                  const double* __restrict__ beta_last_arr, double zr, double zi, double s_target,
                                  double tol, double* __restrict__ theta, double* __restrict__ Qout,
                                  double* __restrict__ sb, int* status) {
  extern __shared__ double smd[];
  double *Q, *d, *e, *q0, *qm;
  if constexpr (FULL) {
    Q = smd;
    d = Q + m * m;
    e = d + m;
    q0 = Q;
    qm = Q + (m - 1) * m;
  } else {
    d = smd;
    e = d + m;
    q0 = e + m;
    qm = q0 + m;
  }
  const int b = blockIdx.x;
  const int lane = threadIdx.x;
  for (int k = lane; k < m; k += 32) {
    d[k] = alpha[k * B + b];
    e[k] = k + 1 < m ? beta[k * B + b] : 0.0;
  }
  __syncwarp();
  bool ok;
  if constexpr (FULL) {
    ok = tridiag_eig_warp(m, d, e, Q, e + m);
  } else {
    ok = true;
    if (lane == 0) ok = tridiag_eig_rows(m, d, e, q0, qm);
    ok = __shfl_sync(0xffffffffu, ok, 0);
    __syncwarp();
  }
  if (!ok && lane == 0) atomicOr(status, 2);
  const double bl = beta_last_arr ? beta_last_arr[b] : 0.0;
  const double s = select_step(m, d, q0, qm, bl, s_target, tol, zr, zi);
  for (int k = lane; k < m; k += 32) theta[k * B + b] = d[k];
  if constexpr (FULL)
    for (int r = lane; r < m; r += 32)
      for (int c = 0; c < m; ++c) Qout[((size_t)b * m + r) * m + c] = Q[r * m + c];
  if (lane == 0) sb[b] = s;
}

template <bool FULL>
__global__ void k_tridiag_eig(int m, int B, const double* __restrict__ alpha, const double* __restrict__ beta,
                              const double* __restrict__ beta_last_arr, double zr, double zi, double s_target,
                              double tol, double* __restrict__ theta, double* __restrict__ Qout,
                              double* __restrict__ sb, int* status) {
  tridiag_eig_block<FULL>(m, B, alpha, beta, beta_last_arr, zr, zi, s_target, tol, theta, Qout, sb, status);
}

inline size_t tridiag_smem(int m, bool full) {
  return sizeof(double) * (full ? size_t(m) * m + 2 * m + 2 : 4 * size_t(m));
}

__global__ void k_step_min(int B, const double* __restrict__ sb, double* __restrict__ sacc) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double s = sb[0];
    for (int b = 1; b < B; ++b) s = fmin(s, sb[b]);
    *sacc = s;
  }
}

// c[k*B + b] = beta0_b * sum_l Q_b[k][l] e^{s z theta_l} Q_b[0][l]
__global__ void k_tridiag_coef(int m, int B, const double* __restrict__ theta, const double* __restrict__ Q,
                               const double* __restrict__ beta0, double zr, double zi, const double* __restrict__ sptr,
                               double s_val, double2* __restrict__ c) {
  __shared__ double2 fg[SYK_MAX_KRYLOV];
  const int b = blockIdx.x;
  const int k = threadIdx.x;
  const double s = sptr ? *sptr : s_val;
  const double* Qb = Q + (size_t)b * m * m;
  if (k < m) {
    const double2 f = cexp_scaled(s, zr, zi, theta[k * B + b]);
    const double g = Qb[k];  // row 0
    fg[k] = make_double2(f.x * g, f.y * g);
  }
  __syncthreads();
  if (k < m) {
    double re = 0.0, im = 0.0;
    for (int l = 0; l < m; ++l) {
      const double q = Qb[k * m + l];
      re = fma(q, fg[l].x, re);
      im = fma(q, fg[l].y, im);
    }
    const double b0 = beta0[b];
    c[k * B + b] = make_double2(b0 * re, b0 * im);
  }
}

// ---------------------------------------------------------------- device-driven evolution
// Kernels of the evolution graph (expmv_chain): they read z, tol and the vectors from the
// job record and keep the step state in DevCtl; single-thread kernels set the graph's
// conditional handles (one thread each: concurrent sets would race).
constexpr int kMaxSegs = 64;
struct IfHandles {
  cudaGraphConditionalHandle h[kMaxSegs];
  int n;
};

__global__ void k_set_job(ExpJob* job, double zr, double zi, double tol, const void* in, void* out) {
  job->zr = zr;
  job->zi = zi;
  job->tol = tol;
  job->in = in;
  job->out = out;
}

// n16 16-byte units: dir 0 copies the job's input into w, dir 1 w into the job's output
__global__ void k_job_copy(const ExpJob* job, uint4* w, int64_t n16, int dir) {
  const uint4* src = dir == 0 ? static_cast<const uint4*>(job->in) : w;
  uint4* dst = dir == 0 ? w : static_cast<uint4*>(job->out);
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n16; e += (int64_t)gridDim.x * blockDim.x)
    dst[e] = src[e];
}

__global__ void k_job_begin(const ExpJob* job, DevCtl* ctl, cudaGraphConditionalHandle h_loop) {
  ctl->s_rem = 1.0;
  ctl->s_done = 0.0;
  ctl->jsteps = 0;
  cudaGraphSetConditional(h_loop, (job->zr != 0.0 || job->zi != 0.0) ? 1u : 0u);
}

// Start of a basis: the first basis of the evolution (no bases yet) or a restart.
__global__ void k_basis_head(const DevCtl* ctl, cudaGraphConditionalHandle h_first) {
  cudaGraphSetConditional(h_first, ctl->jsteps == 0 ? 1u : 0u);
}

__global__ void k_reset_ifs(IfHandles hs) {
  for (int k = 0; k < hs.n; ++k) cudaGraphSetConditional(hs.h[k], 0u);
}

// A convergence check (rows 0 and m-1 only) of the evolution graph.
__global__ void k_tridiag_eig_dev(int m, int B, const double* __restrict__ alpha, const double* __restrict__ beta,
                                  const double* __restrict__ beta_last_arr, const ExpJob* __restrict__ job,
                                  const DevCtl* __restrict__ ctl, double* __restrict__ theta,
                                  double* __restrict__ Qout, double* __restrict__ sb, int* status) {
  tridiag_eig_block<false>(m, B, alpha, beta, beta_last_arr, job->zr, job->zi, ctl->s_rem, job->tol, theta, Qout, sb,
                           status);
}
// The full eigendecomposition of the accepted basis (dimension m_eff) for its coefficients.
__global__ void k_tridiag_eig_full_dev(int B, const double* __restrict__ alpha, const double* __restrict__ beta,
                                       const DevCtl* __restrict__ ctl, double* __restrict__ theta,
                                       double* __restrict__ Qout, double* __restrict__ sb, int* status) {
  tridiag_eig_block<true>(ctl->m_eff, B, alpha, beta, nullptr, 0.0, 0.0, 1.0, 1.0, theta, Qout, sb, status);
}

// After the check that ends Lanczos segment [.., j1): converged when the accepted step covers
// what remains (or the basis is full, or an error bit is set); the next segment's IF handle
// is set accordingly.  Adds the segment's matvecs and kernel launches to the counters.
__global__ void k_decide(DevCtl* ctl, int j1, int last, const int* __restrict__ st_ws,
                         const int* __restrict__ st_apply, const double* __restrict__ sacc,
                         cudaGraphConditionalHandle h_next, int has_next, long long seg_applies,
                         long long seg_launches, long long mv_rows, long long mv_tiled, long long mv_coset) {
  ctl->applies += seg_applies;
  ctl->launches += seg_launches;
  ctl->mv[0] += mv_rows;
  ctl->mv[1] += mv_tiled;
  ctl->mv[2] += mv_coset;
  int e = 0;
  if (st_ws[0] & 1) e |= 1;     // non-finite Lanczos scalar
  if (st_ws[0] & 2) e |= 2;     // tridiagonal eigensolver did not converge
  if (st_apply[0] & 4) e |= 4;  // a bounded wait of a matvec gave up
  ctl->err |= e;
  const bool conv = last || e != 0 || *sacc >= ctl->s_rem;
  if (conv) ctl->m_eff = j1;
  if (has_next) cudaGraphSetConditional(h_next, conv ? 0u : 1u);
}

// The accepted step of the basis, decided as expmv_T decides it for one output at fraction 1:
// the output is combined from this basis when the step reaches it (within 1e-13) or covers
// what remains; otherwise the basis' end state restarts the next one.
__global__ void k_finalize(DevCtl* ctl, const double* __restrict__ sacc) {
  const double s_acc = fmin(*sacc, ctl->s_rem);
  if (!(s_acc > 1e-13 * ctl->s_rem) && !(s_acc >= ctl->s_rem)) ctl->err |= 8;  // step collapsed
  const bool final_basis = s_acc >= ctl->s_rem;
  const bool covered = final_basis || 1.0 <= ctl->s_done + s_acc * (1.0 + 1e-13);
  ctl->s_acc = s_acc;
  ctl->ds = covered ? (final_basis ? s_acc : fmin(1.0 - ctl->s_done, s_acc)) : s_acc;
  ctl->done = covered ? 1 : 0;
}

__global__ void k_tridiag_coef_dev(int B, const double* __restrict__ theta, const double* __restrict__ Q,
                                   const double* __restrict__ beta0, const ExpJob* __restrict__ job,
                                   const DevCtl* __restrict__ ctl, double2* __restrict__ c) {
  __shared__ double2 fg[SYK_MAX_KRYLOV];
  const int m = ctl->m_eff;
  const double s = ctl->ds, zr = job->zr, zi = job->zi;
  const int b = blockIdx.x;
  const int k = threadIdx.x;
  const double* Qb = Q + (size_t)b * m * m;
  if (k < m) {
    const double2 f = cexp_scaled(s, zr, zi, theta[k * B + b]);
    const double g = Qb[k];
    fg[k] = make_double2(f.x * g, f.y * g);
  }
  __syncthreads();
  if (k < m) {
    double re = 0.0, im = 0.0;
    for (int l = 0; l < m; ++l) {
      const double q = Qb[k * m + l];
      re = fma(q, fg[l].x, re);
      im = fma(q, fg[l].y, im);
    }
    const double b0 = beta0[b];
    c[k * B + b] = make_double2(b0 * re, b0 * im);
  }
}

// out = sum_{k < m_eff} c_k v_k (m_eff from the control block)
template <typename R>
__global__ void k_combine_dev(const DevCtl* __restrict__ ctl, const typename CT<R>::T* __restrict__ V, size_t vs,
                              const double2* __restrict__ c, const double* __restrict__ sc,
                              typename CT<R>::T* __restrict__ out, int64_t total, int B) {
  using C = typename CT<R>::T;
  const int nk = ctl->m_eff;
  const int b = threadIdx.x % B;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    C x = make_c<R>(R(0), R(0));
    for (int k = 0; k < nk; ++k) {
      const double2 ck = c[k * B + b];
      const double f = sc[k * B + b];
      cmac(x, R(ck.x * f), R(ck.y * f), V[(size_t)k * vs + e]);
    }
    out[e] = x;
  }
}

// End of a Krylov basis: advance by the accepted step; loop while some of z remains.
__global__ void k_advance(DevCtl* ctl, cudaGraphConditionalHandle h_loop, long long tail_launches) {
  if (ctl->done) {
    ctl->s_rem = 0.0;
  } else {
    ctl->s_done += ctl->s_acc;
    ctl->s_rem -= ctl->s_acc;
  }
  ctl->bases += 1;
  ctl->launches += tail_launches;
  if (++ctl->jsteps > 100000) ctl->err |= 16;
  cudaGraphSetConditional(h_loop, (ctl->s_rem > 0.0 && ctl->err == 0) ? 1u : 0u);
}

// ---------------------------------------------------------------- launch helpers
template <typename R>
struct Ops {
  using C = typename CT<R>::T;
  static void dots(const KrylovWS& ws, int nk, const void* V, size_t vs, const void* w, cudaStream_t st) {
    dim3 grid(ws.G, (nk + KC - 1) / KC);
    k_dots<R><<<grid, ws.bdim, ws.bdim * sizeof(double2), st>>>(nk, (const C*)V, vs, (const C*)w, ws.D * ws.B,
                                                                 (int)ws.B, ws.part);
    count_launch();
  }
  // dst = w - sum_{k0 <= k < k1} h_k v_k
  static void update(const KrylovWS& ws, int k0, int k1, const double2* h, const void* w, void* dst, double* np,
                     cudaStream_t st) {
    k_update<R><<<ws.G, ws.bdim, ws.bdim * sizeof(double2), st>>>(k0, k1, (const C*)ws.V, (size_t)(ws.D * ws.B), h,
                                                                   ws.sc, (const C*)w, (C*)dst, ws.D * ws.B,
                                                                   (int)ws.B, np);
    count_launch();
  }
  static void scale(const KrylovWS& ws, const void* src, void* dst, const double* inv, cudaStream_t st) {
    k_scale<R><<<ws.G, ws.bdim, 0, st>>>((const C*)src, (C*)dst, inv, ws.D * ws.B, (int)ws.B);
    count_launch();
  }
  static void combine(const KrylovWS& ws, int nk, const double2* c, void* out, cudaStream_t st) {
    k_combine<R><<<ws.G, ws.bdim, 0, st>>>(nk, (const C*)ws.V, (size_t)(ws.D * ws.B), c, ws.sc, (C*)out,
                                           ws.D * ws.B, (int)ws.B);
    count_launch();
  }
};

// out[k] (k < nk) from the dots' partial sums, scaled by the basis scales when sc is given,
// plus out[nk] from the matvec epilogue's partials when with_ep
// out[k] for k < nk from the dots' partial sums (scaled by the basis scales when sc is given),
// and, with ep_k >= 0, out[ep_k] from the matvec epilogue's partials (see k_reduce_parts)
void reduce_parts(const KrylovWS& ws, int nk, double2* out, cudaStream_t st, const double* sc = nullptr,
                  int ep_k = -1, const double* beta_prev = nullptr) {
  const int nwb = (nk * (int)ws.B + 7) / 8;  // one warp per (k, b)
  const int nb = nwb + (ep_k >= 0 ? (int)ws.B : 0);
  if (nb == 0) return;
  k_reduce_parts<<<nb, 256, 0, st>>>(nk, ws.G, (int)ws.B, nwb, ws.part, sc, ep_k, ep_k >= 0 ? ws.ep_part : nullptr,
                                     ws.ep_nblk, beta_prev, out);
  count_launch();
}

// One Lanczos step j on the unnormalised basis (see KrylovWS::sc).  The matvec computes
// w = H v_j = sc_j H u_j (scale in its output stage) and h_j = <v_j, w> (per-CTA partial dots in
// its epilogue, fixed-order sums); then, by `orth`:
//   kOrthFull:  h_k = <v_k, w> for k < j (classical Gram-Schmidt against the whole basis);
//               u_{j+1} = w - sum_{k<=j} h_k v_k; with two_pass a second projection and
//               update (the first updates w in place);
//   kOrthLocal: the three-term recurrence u_{j+1} = w - h_j v_j - beta_{j-1} v_{j-1};
// u_{j+1} is written straight into basis slot j+1 with its partial norms, and the scalars
// kernel sets alpha_j = Re h_j, beta_j = |u_{j+1}|, sc_{j+1} = 1/beta_j.  There is no
// normalisation pass: the next matvec and every later coefficient carry sc.
template <typename R>
int lanczos_step(const ApplyParams& P, int dtype, KrylovWS& ws, int j, int orth, bool two_pass, double bt,
                 cudaStream_t st) {
  const int64_t B = ws.B;
  const size_t vs = size_t(ws.D) * B;
  ApplyParams Pe = P;
  Pe.ep_scale = ws.sc + size_t(j) * B;
  Pe.ep_u = ws.vec(j);
  Pe.ep_part = ws.ep_part;
  Pe.ep_nblk = ws.ep_nblk;
  SYK_TRY(launch_apply_H(Pe, dtype, ws.vec(j), ws.w, B, st));
  void* next = ws.vec(j + 1);
  if (orth == kOrthLocal) {
    reduce_parts(ws, 0, ws.h1, st, ws.sc, j, j > 0 ? ws.beta + size_t(j - 1) * B : nullptr);
    Ops<R>::update(ws, j > 0 ? j - 1 : 0, j + 1, ws.h1, ws.w, next, ws.npart, st);
    two_pass = false;
  } else {
    if (j > 0) Ops<R>::dots(ws, j, ws.V, vs, ws.w, st);
    reduce_parts(ws, j, ws.h1, st, ws.sc, j);
    if (two_pass) {
      Ops<R>::update(ws, 0, j + 1, ws.h1, ws.w, ws.w, nullptr, st);
      Ops<R>::dots(ws, j + 1, ws.V, vs, ws.w, st);
      reduce_parts(ws, j + 1, ws.h2, st, ws.sc);
      Ops<R>::update(ws, 0, j + 1, ws.h2, ws.w, next, ws.npart, st);
    } else {
      Ops<R>::update(ws, 0, j + 1, ws.h1, ws.w, next, ws.npart, st);
    }
  }
  k_lanczos_scalars<<<(int(B) + 7) / 8, 256, 0, st>>>(j, int(B), ws.G, ws.h1, two_pass ? ws.h2 : nullptr, ws.npart,
                                                       ws.alpha, ws.beta, ws.inv, ws.sc, ws.status, bt);
  count_launch();
  SYK_CUDA_CHECK(cudaGetLastError());
  return SYK_OK;
}

size_t align_up(size_t v) { return (v + 255) & ~size_t(255); }

// CTAs a matvec launch may have (its epilogue writes one partial per CTA and column): tiles of
// at least 64 rows, clusters of at most 8; the row kernel's epilogue uses at most kRedBlocksCap.
int64_t ep_capacity(int64_t D) { return std::max<int64_t>(D / 8, kRedBlocksCap); }

}  // namespace

// by dtype code: complex64 defaults to the three-term recurrence (as accurate as full
// Gram-Schmidt at FP32 rounding, measured against complex128 and the oracle, and 11 % less
// time per OTOC curve at N = 40); complex128, the accuracy reference, to full Gram-Schmidt
std::atomic<int> g_orth[3] = {{kOrthFull}, {kOrthLocal}, {kOrthFull}};
int lanczos_orth(int dtype) { return g_orth[dtype == SYK_C64 ? SYK_C64 : SYK_C128].load(); }

// ---------------------------------------------------------------- workspace
size_t krylov_ws_bytes(int64_t D, int dtype, int m, int64_t B) {
  const int bdim = vec_bdim(B);
  const int G = red_grid(D * B, bdim, kRedBlocksCap);
  const size_t vb = align_up(size_t(D) * B * dtype_size(dtype));
  size_t s = 0;
  s += vb * (m + 1);                                  // V
  s += vb;                                            // w
  s += align_up(sizeof(double2) * G * (m + 1) * B);   // part
  s += 2 * align_up(sizeof(double2) * (m + 1) * B);   // h1, h2
  s += align_up(sizeof(double) * G * B);              // npart
  s += 2 * align_up(sizeof(double) * m * B);          // alpha, beta
  s += 3 * align_up(sizeof(double) * B);              // beta0, inv, sb
  s += align_up(sizeof(double) * m * B);              // theta
  s += align_up(sizeof(double) * m * m * B);          // Q
  s += align_up(sizeof(double));                      // sacc
  s += align_up(sizeof(double2) * m * B);             // c
  s += align_up(sizeof(int) * 4);                     // status
  if (dtype == SYK_C128) s += align_up(size_t(D) * B * 16);  // split
  s += align_up(sizeof(double) * (m + 1) * B);                // sc
  s += align_up(sizeof(double2) * size_t(ep_capacity(D)) * B);  // ep_part
  s += align_up(sizeof(int));                                 // ep_nblk
  s += align_up(sizeof(ExpJob)) + align_up(sizeof(DevCtl));   // job, ctl
  return s;
}

int krylov_ws_carve(KrylovWS* ws, void* base, size_t bytes, int64_t D, int dtype, int m, int64_t B) {
  if (bytes < krylov_ws_bytes(D, dtype, m, B)) {
    set_error("workspace too small: %zu < %zu bytes", bytes, krylov_ws_bytes(D, dtype, m, B));
    return SYK_ENOMEM;
  }
  if ((reinterpret_cast<uintptr_t>(base) & 255) != 0) {
    set_error("workspace must be 256-byte aligned");
    return SYK_EINVAL;
  }
  ws->m = m;
  ws->B = B;
  ws->D = D;
  ws->dtype = dtype;
  ws->bdim = vec_bdim(B);
  ws->G = red_grid(D * B, ws->bdim, std::min(kRedBlocksCap, 2 * sm_count()));
  const size_t vb = align_up(size_t(D) * B * dtype_size(dtype));
  char* p = static_cast<char*>(base);
  auto take = [&](size_t n) {
    char* r = p;
    p += align_up(n);
    return r;
  };
  ws->V = take(vb * (m + 1));
  ws->w = take(vb);
  ws->part = (double2*)take(sizeof(double2) * ws->G * (m + 1) * B);
  ws->h1 = (double2*)take(sizeof(double2) * (m + 1) * B);
  ws->h2 = (double2*)take(sizeof(double2) * (m + 1) * B);
  ws->npart = (double*)take(sizeof(double) * ws->G * B);
  ws->alpha = (double*)take(sizeof(double) * m * B);
  ws->beta = (double*)take(sizeof(double) * m * B);
  ws->beta0 = (double*)take(sizeof(double) * B);
  ws->inv = (double*)take(sizeof(double) * B);
  ws->sb = (double*)take(sizeof(double) * B);
  ws->theta = (double*)take(sizeof(double) * m * B);
  ws->Q = (double*)take(sizeof(double) * m * m * B);
  ws->sacc = (double*)take(sizeof(double));
  ws->c = (double2*)take(sizeof(double2) * m * B);
  ws->status = (int*)take(sizeof(int) * 4);
  ws->split = dtype == SYK_C128 ? take(size_t(D) * B * 16) : nullptr;
  ws->sc = (double*)take(sizeof(double) * (m + 1) * B);
  ws->ep_cap = ep_capacity(D);
  ws->ep_part = (double2*)take(sizeof(double2) * size_t(ws->ep_cap) * B);
  ws->ep_nblk = (int*)take(sizeof(int));
  ws->job = (ExpJob*)take(sizeof(ExpJob));
  ws->ctl = (DevCtl*)take(sizeof(DevCtl));
  return SYK_OK;
}

// ---------------------------------------------------------------- dot helper
int dot_columns(const void* x, const void* y, int64_t D, int64_t B, int dtype, KrylovWS& ws, double2* res,
                cudaStream_t st) {
  if (ws.D != D || ws.B != B || ws.dtype != dtype) {
    set_error("dot_columns: workspace shape mismatch");
    return SYK_EINVAL;
  }
  if (dtype == SYK_C64) Ops<float>::dots(ws, 1, x, 0, y, st);
  else Ops<double>::dots(ws, 1, x, 0, y, st);
  reduce_parts(ws, 1, res, st);
  SYK_CUDA_CHECK(cudaGetLastError());
  return SYK_OK;
}

// ---------------------------------------------------------------- expmv
namespace {

// Replays the kernel sequence of one Lanczos segment as a captured CUDA graph.  Graphs are
// cached per host thread and keyed by everything their launches bake in (workspace, term
// tables, sector, shapes, segment range) plus an epoch that changes when term sets are freed
// or tile shapes retuned.  The first sighting of a key runs eagerly (lazy allocations happen
// outside capture); the second captures and instantiates; later ones only launch.
struct SegKey {
  const void* V;
  const void* tab;
  int sector, dtype;
  int64_t B, D;
  int m, j0, j1, two;
  uint64_t epoch;
  bool operator<(const SegKey& o) const {
    return std::tie(V, tab, sector, dtype, B, D, m, j0, j1, two, epoch) <
           std::tie(o.V, o.tab, o.sector, o.dtype, o.B, o.D, o.m, o.j0, o.j1, o.two, o.epoch);
  }
};
struct SegGraph {
  cudaGraphExec_t exec = nullptr;
  int64_t launches = 0, applies = 0;
  int64_t kinds[kMvKinds] = {};
};
struct GraphCache {
  std::map<SegKey, SegGraph> graphs;
  std::set<SegKey> seen;
  cudaStream_t cap = nullptr;  // capture stream (the legacy default stream cannot be captured)
  ~GraphCache() {
    for (auto& kv : graphs) cudaGraphExecDestroy(kv.second.exec);
  }
};
thread_local GraphCache t_cache;

template <typename F>
int run_segment_graphed(const ApplyParams& P, const KrylovWS& ws, int dtype, int64_t B, int m, int j0, int j1,
                        bool two, cudaStream_t st, F&& eager) {
  // no_alloc callers (syk_expmv_static) always launch eagerly: capturing and instantiating a
  // graph, and the cache's host containers, would allocate
  if (P.no_alloc || !graphs_enabled() || prof_enabled()) return eager(st);
  const SegKey key{ws.V, P.m4_tab, P.sector, dtype, B, P.D, m, j0, j1, two ? 1 : 0, graph_epoch()};
  auto it = t_cache.graphs.find(key);
  if (it == t_cache.graphs.end()) {
    if (!t_cache.seen.count(key)) {
      if (t_cache.seen.size() > 4096) t_cache.seen.clear();
      t_cache.seen.insert(key);
      return eager(st);
    }
    if (t_cache.graphs.size() > 512) {
      for (auto& kv : t_cache.graphs) cudaGraphExecDestroy(kv.second.exec);
      t_cache.graphs.clear();
    }
    SegGraph sg;
    cudaGraph_t g = nullptr;
    if (!t_cache.cap) SYK_CUDA_CHECK(cudaStreamCreateWithFlags(&t_cache.cap, cudaStreamNonBlocking));
    SYK_CUDA_CHECK(cudaStreamBeginCapture(t_cache.cap, cudaStreamCaptureModeThreadLocal));
    capture_counts_begin();
    const int rc = eager(t_cache.cap);  // recorded, not executed
    capture_counts_end(&sg.launches, &sg.applies, sg.kinds);
    const cudaError_t ec = cudaStreamEndCapture(t_cache.cap, &g);
    if (rc != SYK_OK) {
      if (g) cudaGraphDestroy(g);
      return rc;
    }
    if (ec != cudaSuccess) {
      set_error("expmv: graph capture failed: %s", cudaGetErrorString(ec));
      return SYK_ECUDA;
    }
    const cudaError_t ei = cudaGraphInstantiate(&sg.exec, g, 0);
    cudaGraphDestroy(g);
    if (ei != cudaSuccess) {
      set_error("expmv: graph instantiation failed: %s", cudaGetErrorString(ei));
      return SYK_ECUDA;
    }
    it = t_cache.graphs.emplace(key, sg).first;
  }
  SYK_CUDA_CHECK(cudaGraphLaunch(it->second.exec, st));
  count_launch(it->second.launches);
  count_applies(it->second.applies);
  count_matvec_replay(it->second.kinds);
  return SYK_OK;
}

// When to check a Krylov basis for convergence (one plan per evolution, the same for the host-
// and the device-driven paths).  The Lanczos approximation of e^{tau H} for a spectrum of
// half-width rho needs about the smallest k with (e rho |tau| / 2k)^k <= tol vectors; with
// rho = 2 x the RMS level this predicts the counts measured at N = 40 (808 matvecs per OTOC
// curve) but overestimates by a few vectors (more at tight tol: measured, checking 2 vectors
// before the prediction added 3 % matvecs at tol 1e-7 and 12 % at 1e-12), so the first check
// comes at 3/4 of it (at least after 4 vectors, at most at m), the next ones every `every`
// vectors: 2 when a matvec costs more than a check (~0.2 ms), else 4.  The matvec cost is
// modelled from its work (8 nnz B flop at ~20 TFLOP/s for complex64, ~4.4 for complex128,
// plus 10 us).
struct CheckPlan {
  int first, every;
};
CheckPlan check_plan(const ApplyParams& P, int dtype, int64_t D, int64_t B, int m, std::complex<double> z,
                     double tol) {
  const double nnz = double(D) * double(P.n4 + P.n2 + 1);
  const double apply_ms = 0.01 + 8.0 * nnz * double(B) / (dtype == SYK_C64 ? 2.0e10 : 4.4e9);
  const int every = apply_ms >= 0.2 ? 2 : 4;
  const double rt = std::abs(z) * P.rho;
  int k = m + 1;
  for (int kk = 1; kk <= m; ++kk)
    if (rt <= 0.0 || double(kk) * std::log(2.718281828459045 * rt / (2.0 * kk)) <= std::log(tol)) {
      k = kk;
      break;
    }
  const int first = std::min(m, std::max(4, (3 * k) / 4));
  return {first, every};
}

// Segment ends of a basis under a plan: the first check, then every `every` vectors, and m.
std::vector<int> segment_ends(int m, const CheckPlan& pl) {
  std::vector<int> e;
  int j1 = std::min(m, std::max(1, pl.first));
  e.push_back(j1);
  while (j1 < m) {
    j1 = std::min(m, j1 + pl.every);
    e.push_back(j1);
  }
  return e;
}

// outs[k] = e^{fr[k] z H} psi for 0 < fr[0] < ... < fr[nf-1]: the step to fr[nf-1] is split
// into Krylov bases as the error estimate allows, and each output is combined from the basis
// whose step covers its fraction.  Restarts pass through outs[nf-1], written last.
template <typename R>
int expmv_T(const ApplyParams& P_in, int dtype, std::complex<double> z, const void* psi, const double* fr, int nf,
            void* const* outs, double tol, KrylovWS& ws, cudaStream_t st, int* nsteps) {
  const ApplyParams P = ws.with_split(P_in);
  const int64_t B = ws.B;
  const int m = ws.m;
  const double bt = (dtype == SYK_C64 ? 64.0 * 5.96e-8 : 64.0 * 1.11e-16);
  // complex64 vectors carry ~1e-7 relative error, which one reorthogonalisation pass already
  // reaches; complex128 vectors get the second pass ("twice is enough")
  const bool two_pass = dtype == SYK_C128;
  const int orth = lanczos_orth(dtype);
  const CheckPlan plan = check_plan(P, dtype, ws.D, B, m, z, tol);
  // the first basis checks by the plan; a restart covers an unknown remainder: from 4 vectors on
  const std::vector<int> ends_first = segment_ends(m, plan), ends_restart = segment_ends(m, CheckPlan{4, plan.every});
  const double zr = z.real(), zi = z.imag();
  int* hstat = static_cast<int*>(ws.host_stage ? ws.host_stage : pinned_scratch(64));
  double* hs = reinterpret_cast<double*>(hstat + 4);
  SYK_CUDA_CHECK(cudaMemsetAsync(ws.status, 0, sizeof(int) * 4, st));
  double s_rem = fr[nf - 1], s_done = 0.0;
  int steps = 0, next = 0;
  const void* cur = psi;
  while (s_rem > 0.0) {
    NvtxRange basis_range("krylov basis");
    if (++steps > 100000) {
      set_error("expmv: more than 100000 Krylov steps");
      return SYK_ENUMERIC;
    }
    // v_0 = cur / ||cur||
    Ops<R>::dots(ws, 1, cur, 0, cur, st);
    reduce_parts(ws, 1, ws.h1, st);
    k_norm_init<<<(int(B) + 127) / 128, 128, 0, st>>>(int(B), ws.h1, ws.beta0, ws.inv, ws.sc, ws.status);
    count_launch();
    Ops<R>::scale(ws, cur, ws.vec(0), ws.inv, st);
    int m_eff = m;
    // Lanczos iterations j in [j0, j1) between two convergence checks
    auto segment = [&](int j0, int j1, cudaStream_t st) -> int {
      // classical Gram-Schmidt against the whole basis; a second pass for FP64 vectors
      for (int j = j0; j < j1; ++j) SYK_TRY(lanczos_step<R>(P, dtype, ws, j, orth, two_pass, bt, st));
      return SYK_OK;
    };
    const std::vector<int>& ends = steps == 1 ? ends_first : ends_restart;
    int j0 = 0;
    for (size_t si = 0; si < ends.size() && j0 < m; ++si) {
      const int j1 = ends[si];
      SYK_TRY(run_segment_graphed(P, ws, dtype, B, m, j0, j1, two_pass, st,
                                  [&](cudaStream_t s) { return segment(j0, j1, s); }));
      const int j = j1 - 1;
      const bool last = (j1 == m);
      {
        const int mm = j1;
        k_tridiag_eig<false><<<int(B), 32, tridiag_smem(mm, false), st>>>(
            mm, int(B), ws.alpha, ws.beta, ws.beta + size_t(j) * B, zr, zi, s_rem, tol, ws.theta, ws.Q, ws.sb,
            ws.status);
        k_step_min<<<1, 32, 0, st>>>(int(B), ws.sb, ws.sacc);
        count_launch(2);
        SYK_CUDA_CHECK(cudaMemcpyAsync(hstat, ws.status, sizeof(int) * 2, cudaMemcpyDeviceToHost, st));
        SYK_CUDA_CHECK(cudaMemcpyAsync(hstat + 2, P.status, sizeof(int), cudaMemcpyDeviceToHost, st));
        SYK_CUDA_CHECK(cudaMemcpyAsync(hs, ws.sacc, sizeof(double), cudaMemcpyDeviceToHost, st));
        SYK_CUDA_CHECK(cudaStreamSynchronize(st));
        prof_collect();
        if (hstat[0] & 1) {
          set_error("expmv: non-finite Lanczos scalar");
          return SYK_ENUMERIC;
        }
        if (hstat[0] & 2) {
          set_error("expmv: tridiagonal eigensolver did not converge");
          return SYK_ENUMERIC;
        }
        if (hstat[2] & 4) {
          set_error("apply_H: a bounded wait for a staged tile gave up");
          return SYK_ETIMEOUT;
        }
        if (last || *hs >= s_rem) {
          m_eff = mm;
          break;
        }
      }
      j0 = j1;
    }
    double s_acc = std::min(*hs, s_rem);
    if (!(s_acc > 1e-13 * s_rem) && !(s_acc >= s_rem)) {
      set_error("expmv: Krylov step collapsed (s=%g of remaining %g); raise krylov_dim or tol", s_acc, s_rem);
      return SYK_ENUMERIC;
    }
    // the checks kept only two rows of the eigenvectors: the full set for the coefficients
    k_tridiag_eig<true><<<int(B), 32, tridiag_smem(m_eff, true), st>>>(
        m_eff, int(B), ws.alpha, ws.beta, nullptr, zr, zi, 1.0, 1.0, ws.theta, ws.Q, ws.sb, ws.status);
    count_launch();
    const bool final_basis = s_acc >= s_rem;
    // outputs whose fraction this basis reaches
    while (next < nf && (fr[next] <= s_done + s_acc * (1.0 + 1e-13) || (final_basis && next == nf - 1))) {
      const double ds = (final_basis && next == nf - 1) ? s_acc : std::min(fr[next] - s_done, s_acc);
      k_tridiag_coef<<<int(B), 64, 0, st>>>(m_eff, int(B), ws.theta, ws.Q, ws.beta0, zr, zi, nullptr, ds, ws.c);
      count_launch();
      Ops<R>::combine(ws, m_eff, ws.c, outs[next], st);
      ++next;
    }
    if (next == nf) {
      SYK_CUDA_CHECK(cudaGetLastError());
      count_bases(1);
      break;
    }
    if (!final_basis) {  // restart from the state at the end of this basis' step
      k_tridiag_coef<<<int(B), 64, 0, st>>>(m_eff, int(B), ws.theta, ws.Q, ws.beta0, zr, zi, nullptr, s_acc, ws.c);
      count_launch();
      Ops<R>::combine(ws, m_eff, ws.c, outs[nf - 1], st);
      cur = outs[nf - 1];
    }
    SYK_CUDA_CHECK(cudaGetLastError());
    count_bases(1);
    s_done += s_acc;
    if (final_basis) s_rem = 0.0;
    else s_rem -= s_acc;
  }
  if (nsteps) *nsteps = steps;
  return SYK_OK;
}

}  // namespace

int expmv_impl(const ApplyParams& P, int dtype, std::complex<double> z, const void* psi, void* out, int64_t B,
               double tol, KrylovWS& ws, cudaStream_t st, int* nsteps) {
  if (ws.B != B || ws.D != P.D || ws.dtype != dtype) {
    set_error("expmv: workspace shape mismatch");
    return SYK_EINVAL;
  }
  if (!(tol > 0.0)) {
    set_error("expmv: tol must be > 0");
    return SYK_EINVAL;
  }
  if (z == std::complex<double>(0.0, 0.0)) {
    if (out != psi)
      SYK_CUDA_CHECK(cudaMemcpyAsync(out, psi, ws.vec_bytes(), cudaMemcpyDeviceToDevice, st));
    if (nsteps) *nsteps = 0;
    return SYK_OK;
  }
  const double one = 1.0;
  void* outs[1] = {out};
  return dtype == SYK_C64 ? expmv_T<float>(P, dtype, z, psi, &one, 1, outs, tol, ws, st, nsteps)
                          : expmv_T<double>(P, dtype, z, psi, &one, 1, outs, tol, ws, st, nsteps);
}

int expmv_points(const ApplyParams& P, int dtype, std::complex<double> z, const void* psi, const double* fr, int nf,
                 void* const* outs, int64_t B, double tol, KrylovWS& ws, cudaStream_t st) {
  if (ws.B != B || ws.D != P.D || ws.dtype != dtype) {
    set_error("expmv: workspace shape mismatch");
    return SYK_EINVAL;
  }
  if (nf < 1 || !(tol > 0.0) || !(fr[0] > 0.0)) {
    set_error("expmv_points: need nf >= 1, tol > 0 and positive fractions");
    return SYK_EINVAL;
  }
  for (int k = 1; k < nf; ++k)
    if (!(fr[k] > fr[k - 1])) {
      set_error("expmv_points: fractions must increase");
      return SYK_EINVAL;
    }
  if (z == std::complex<double>(0.0, 0.0)) {
    for (int k = 0; k < nf; ++k)
      if (outs[k] != psi) SYK_CUDA_CHECK(cudaMemcpyAsync(outs[k], psi, ws.vec_bytes(), cudaMemcpyDeviceToDevice, st));
    return SYK_OK;
  }
  return dtype == SYK_C64 ? expmv_T<float>(P, dtype, z, psi, fr, nf, outs, tol, ws, st, nullptr)
                          : expmv_T<double>(P, dtype, z, psi, fr, nf, outs, tol, ws, st, nullptr);
}

// ---------------------------------------------------------------- device-driven chain
namespace {

struct DevKey {
  const void* V;
  const void* tab;
  int sector, dtype;
  int64_t B, D;
  int m, orth, first, every;
  uint64_t epoch;
  bool operator<(const DevKey& o) const {
    return std::tie(V, tab, sector, dtype, B, D, m, orth, first, every, epoch) <
           std::tie(o.V, o.tab, o.sector, o.dtype, o.B, o.D, o.m, o.orth, o.first, o.every, o.epoch);
  }
};
struct DevCache {
  std::map<DevKey, cudaGraphExec_t> graphs;
  cudaStream_t cap = nullptr;
  ~DevCache() {
    for (auto& kv : graphs) cudaGraphExecDestroy(kv.second);
  }
};
thread_local DevCache t_dev;

std::vector<cudaGraphNode_t> capture_frontier(cudaStream_t s) {
  cudaStreamCaptureStatus stt;
  const cudaGraphNode_t* deps = nullptr;
  size_t nd = 0;
  if (cudaStreamGetCaptureInfo(s, &stt, nullptr, nullptr, &deps, nullptr, &nd) != cudaSuccess) return {};
  return std::vector<cudaGraphNode_t>(deps, deps + nd);
}

// Builds the graph of one evolution out = e^{zH} in on workspace ws (z, tol, in, out from
// ws.job; step state in ws.ctl):
//   copy in -> w; WHILE (some of z remains) {
//     v_0 = w / |w|; Lanczos segment [0, 4); check; then for each later segment
//     IF (not converged) { segment; check }   (sequential IF nodes, reset each iteration)
//     coefficients of the accepted step; w = V c; advance }
//   copy w -> out.
// The segments and checks are exactly expmv_T's, so results equal the host-driven path's.
template <typename R>
int build_dev_graph(const ApplyParams& P, int dtype, KrylovWS& ws, int orth, bool two_pass, const CheckPlan& plan,
                    double bt, cudaStream_t st, cudaGraphExec_t* out) {
  const int64_t B = ws.B;
  const int m = ws.m;
  if (!t_dev.cap) SYK_CUDA_CHECK(cudaStreamCreateWithFlags(&t_dev.cap, cudaStreamNonBlocking));
  cudaStream_t cs = t_dev.cap;  // capture only: nothing executes on it
  // Lazily built chunk lists and coset layouts, kernel attributes: one eager matvec first, on
  // the caller's stream so that it is ordered after the chain's pending work on this workspace
  // (its counts are dropped: it is set-up, not work of the evolution).
  int64_t wl = 0, wa = 0, wk[kMvKinds];
  capture_counts_begin();
  const int wrc = launch_apply_H(P, dtype, ws.vec(0), ws.w, B, st);
  capture_counts_end(&wl, &wa, wk);
  SYK_TRY(wrc);
  // segment ends: the evolution's check plan for its first basis, checks from 4 vectors on
  // for restarts (as in expmv_T)
  const std::vector<int> j1s_first = segment_ends(m, plan), j1s_restart = segment_ends(m, CheckPlan{4, plan.every});
  if (int(j1s_restart.size()) > kMaxSegs) {
    set_error("expmv graph: %d segments exceed %d", int(j1s_restart.size()), kMaxSegs);
    return SYK_EINVAL;
  }
  const cudaStreamCaptureMode mode = cudaStreamCaptureModeThreadLocal;
  const int64_t n16 = int64_t(ws.vec_bytes() / 16);
  const int cg = std::min<int64_t>((n16 + 255) / 256, 4 * sm_count());
  cudaGraph_t g = nullptr;
  SYK_CUDA_CHECK(cudaGraphCreate(&g, 0));
  int rc = SYK_OK;
  auto fail = [&](cudaError_t e, const char* what) {
    cudaGraph_t junk = nullptr;
    cudaStreamCaptureStatus stt;
    if (cudaStreamIsCapturing(cs, &stt) == cudaSuccess && stt != cudaStreamCaptureStatusNone)
      cudaStreamEndCapture(cs, &junk);
    cudaGetLastError();
    set_error("expmv graph: %s: %s", what, cudaGetErrorString(e));
    return SYK_ECUDA;
  };
#define DEV_CK(expr, what)                 \
  do {                                     \
    cudaError_t e_ = (expr);               \
    if (e_ != cudaSuccess) {               \
      rc = fail(e_, what);                 \
      cudaGraphDestroy(g);                 \
      return rc;                           \
    }                                      \
  } while (0)
  cudaGraphConditionalHandle hloop;
  DEV_CK(cudaGraphConditionalHandleCreate(&hloop, g, 0, 0), "loop handle");
  // prologue: w = in, loop condition
  DEV_CK(cudaStreamBeginCaptureToGraph(cs, g, nullptr, nullptr, 0, mode), "capture");
  capture_counts_begin();
  k_job_copy<<<cg, 256, 0, cs>>>(ws.job, reinterpret_cast<uint4*>(ws.w), n16, 0);
  k_job_begin<<<1, 1, 0, cs>>>(ws.job, ws.ctl, hloop);
  std::vector<cudaGraphNode_t> fr = capture_frontier(cs);
  DEV_CK(cudaStreamEndCapture(cs, &g), "end capture");
  cudaGraphNodeParams wp = {};
  wp.type = cudaGraphNodeTypeConditional;
  wp.conditional.handle = hloop;
  wp.conditional.type = cudaGraphCondTypeWhile;
  wp.conditional.size = 1;
  cudaGraphNode_t wnode;
  DEV_CK(cudaGraphAddNode(&wnode, g, fr.data(), nullptr, fr.size(), &wp), "while node");
  cudaGraph_t body = wp.conditional.phGraph_out[0];
  cudaGraphConditionalHandle hfirst;
  DEV_CK(cudaGraphConditionalHandleCreate(&hfirst, body, 0, 0), "first-basis handle");
  // one segment of Lanczos steps [j0, j1) and its convergence check, captured on cs; its
  // decide kernel opens the next segment of the chain (handle ifs.h[k])
  auto segment = [&](const IfHandles& ifs, int k, int j0, int j1) -> int {
    int64_t l0 = 0, a0 = 0, kinds[kMvKinds];
    capture_counts_begin();  // the segment's own tallies (launches and matvecs per execution)
    for (int j = j0; j < j1; ++j) SYK_TRY(lanczos_step<R>(P, dtype, ws, j, orth, two_pass, bt, cs));
    capture_counts_end(&l0, &a0, kinds);
    capture_counts_begin();  // keep counting captured launches away from the global counters
    const int mm = j1;
    k_tridiag_eig_dev<<<int(B), 32, tridiag_smem(mm, false), cs>>>(mm, int(B), ws.alpha, ws.beta,
                                                                  ws.beta + size_t(j1 - 1) * B, ws.job,
                                                                  ws.ctl, ws.theta, ws.Q, ws.sb, ws.status);
    k_step_min<<<1, 32, 0, cs>>>(int(B), ws.sb, ws.sacc);
    const bool has_next = k < ifs.n;
    k_decide<<<1, 1, 0, cs>>>(ws.ctl, j1, j1 == m ? 1 : 0, ws.status, P.status, ws.sacc,
                              has_next ? ifs.h[k] : cudaGraphConditionalHandle(0), has_next ? 1 : 0, a0, l0 + 3,
                              kinds[kMvRows], kinds[kMvTiled], kinds[kMvCoset]);
    SYK_CUDA_CHECK(cudaGetLastError());
    return SYK_OK;
  };
  // the segments ending at `ends`, captured into graph gb: reset the chain's IF handles, the
  // first segment, then one IF node per later segment
  auto build_chain = [&](cudaGraph_t gb, const std::vector<int>& ends) -> int {
    IfHandles ifs = {};
    ifs.n = int(ends.size()) - 1;
    for (int k = 0; k < ifs.n; ++k) SYK_CUDA_CHECK(cudaGraphConditionalHandleCreate(&ifs.h[k], gb, 0, 0));
    SYK_CUDA_CHECK(cudaStreamBeginCaptureToGraph(cs, gb, nullptr, nullptr, 0, mode));
    k_reset_ifs<<<1, 1, 0, cs>>>(ifs);
    int crc = segment(ifs, 0, 0, ends[0]);
    std::vector<cudaGraphNode_t> cf = capture_frontier(cs);
    {
      cudaGraph_t tmp = gb;
      const cudaError_t e = cudaStreamEndCapture(cs, &tmp);
      if (crc == SYK_OK && e != cudaSuccess) {
        set_error("expmv graph: end capture: %s", cudaGetErrorString(e));
        crc = SYK_ECUDA;
      }
    }
    if (crc != SYK_OK) return crc;
    for (int k = 1; k < int(ends.size()); ++k) {
      cudaGraphNodeParams ip = {};
      ip.type = cudaGraphNodeTypeConditional;
      ip.conditional.handle = ifs.h[k - 1];
      ip.conditional.type = cudaGraphCondTypeIf;
      ip.conditional.size = 1;
      cudaGraphNode_t inode;
      SYK_CUDA_CHECK(cudaGraphAddNode(&inode, gb, cf.data(), nullptr, cf.size(), &ip));
      cudaGraph_t ib = ip.conditional.phGraph_out[0];
      SYK_CUDA_CHECK(cudaStreamBeginCaptureToGraph(cs, ib, nullptr, nullptr, 0, mode));
      crc = segment(ifs, k, ends[k - 1], ends[k]);
      cudaGraph_t tmp = ib;
      const cudaError_t e = cudaStreamEndCapture(cs, &tmp);
      if (crc != SYK_OK) return crc;
      SYK_CUDA_CHECK(e);
      cf = {inode};
    }
    return SYK_OK;
  };
  // body head: first basis of the evolution or a restart, v_0 = w / |w|
  DEV_CK(cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, mode), "capture body");
  k_basis_head<<<1, 1, 0, cs>>>(ws.ctl, hfirst);
  Ops<R>::dots(ws, 1, ws.w, 0, ws.w, cs);
  reduce_parts(ws, 1, ws.h1, cs);
  k_norm_init<<<(int(B) + 127) / 128, 128, 0, cs>>>(int(B), ws.h1, ws.beta0, ws.inv, ws.sc, ws.status);
  Ops<R>::scale(ws, ws.w, ws.vec(0), ws.inv, cs);
  fr = capture_frontier(cs);
  {
    cudaGraph_t tmp = body;
    DEV_CK(cudaStreamEndCapture(cs, &tmp), "end capture body");
  }
  // the first basis checks by the evolution's plan, restarts from 4 vectors on
  cudaGraphNodeParams bp = {};
  bp.type = cudaGraphNodeTypeConditional;
  bp.conditional.handle = hfirst;
  bp.conditional.type = cudaGraphCondTypeIf;
  bp.conditional.size = 2;
  cudaGraphNode_t bnode;
  DEV_CK(cudaGraphAddNode(&bnode, body, fr.data(), nullptr, fr.size(), &bp), "first/restart node");
  cudaGraph_t first_branch = bp.conditional.phGraph_out[0], restart_branch = bp.conditional.phGraph_out[1];
  rc = build_chain(first_branch, j1s_first);
  if (rc == SYK_OK) rc = build_chain(restart_branch, j1s_restart);
  if (rc != SYK_OK) {
    cudaGetLastError();
    cudaGraphDestroy(g);
    return rc;
  }
  fr = {bnode};
  // body tail: the accepted step's coefficients, w = V c, advance
  DEV_CK(cudaStreamBeginCaptureToGraph(cs, body, fr.data(), nullptr, fr.size(), mode), "capture tail");
  k_finalize<<<1, 1, 0, cs>>>(ws.ctl, ws.sacc);
  k_tridiag_eig_full_dev<<<int(B), 32, tridiag_smem(m, true), cs>>>(int(B), ws.alpha, ws.beta, ws.ctl, ws.theta,
                                                                     ws.Q, ws.sb, ws.status);
  k_tridiag_coef_dev<<<int(B), 64, 0, cs>>>(int(B), ws.theta, ws.Q, ws.beta0, ws.job, ws.ctl, ws.c);
  k_combine_dev<R><<<ws.G, ws.bdim, 0, cs>>>(ws.ctl, (const typename CT<R>::T*)ws.V, size_t(ws.D * B), ws.c, ws.sc,
                                             (typename CT<R>::T*)ws.w, ws.D * B, int(B));
  // per basis: head, the 4 kernels of v_0, reset, finalize, eigenvectors, coefficients, combine, advance
  k_advance<<<1, 1, 0, cs>>>(ws.ctl, hloop, 11);
  {
    cudaGraph_t tmp = body;
    DEV_CK(cudaStreamEndCapture(cs, &tmp), "end capture tail");
  }
  // epilogue: out = w
  DEV_CK(cudaStreamBeginCaptureToGraph(cs, g, &wnode, nullptr, 1, mode), "capture epilogue");
  k_job_copy<<<cg, 256, 0, cs>>>(ws.job, reinterpret_cast<uint4*>(ws.w), n16, 1);
  {
    cudaGraph_t tmp = g;
    DEV_CK(cudaStreamEndCapture(cs, &tmp), "end capture epilogue");
  }
  int64_t l0 = 0, a0 = 0, kinds[kMvKinds];
  capture_counts_end(&l0, &a0, kinds);
  cudaGraphExec_t exec = nullptr;
  DEV_CK(cudaGraphInstantiate(&exec, g, 0), "instantiate");
  cudaGraphDestroy(g);
  *out = exec;
#undef DEV_CK
  return SYK_OK;
}

}  // namespace

int chain_begin(KrylovWS& ws, cudaStream_t st) {
  SYK_CUDA_CHECK(cudaMemsetAsync(ws.ctl, 0, sizeof(DevCtl), st));
  SYK_CUDA_CHECK(cudaMemsetAsync(ws.status, 0, sizeof(int) * 4, st));
  return SYK_OK;
}

int expmv_chain(const ApplyParams& P_in, int dtype, std::complex<double> z, const void* in, void* out, int64_t B,
                double tol, KrylovWS& ws, cudaStream_t st) {
  if (P_in.no_alloc || !device_chains_enabled() || prof_enabled())
    return expmv_impl(P_in, dtype, z, in, out, B, tol, ws, st, nullptr);
  if (ws.B != B || ws.D != P_in.D || ws.dtype != dtype) {
    set_error("expmv: workspace shape mismatch");
    return SYK_EINVAL;
  }
  if (!(tol > 0.0)) {
    set_error("expmv: tol must be > 0");
    return SYK_EINVAL;
  }
  const ApplyParams P = ws.with_split(P_in);
  const int orth = lanczos_orth(dtype);
  const CheckPlan plan = check_plan(P, dtype, ws.D, B, ws.m, z, tol);
  const DevKey key{ws.V, P.m4_tab, P.sector, dtype, B, P.D, ws.m, orth, plan.first, plan.every, graph_epoch()};
  auto it = t_dev.graphs.find(key);
  if (it == t_dev.graphs.end()) {
    if (t_dev.graphs.size() > 256) {
      for (auto& kv : t_dev.graphs) cudaGraphExecDestroy(kv.second);
      t_dev.graphs.clear();
    }
    const double bt = (dtype == SYK_C64 ? 64.0 * 5.96e-8 : 64.0 * 1.11e-16);
    cudaGraphExec_t exec = nullptr;
    const int rc = dtype == SYK_C64 ? build_dev_graph<float>(P, dtype, ws, orth, false, plan, bt, st, &exec)
                                    : build_dev_graph<double>(P, dtype, ws, orth, true, plan, bt, st, &exec);
    if (rc != SYK_OK) return rc;
    it = t_dev.graphs.emplace(key, exec).first;
  }
  k_set_job<<<1, 1, 0, st>>>(ws.job, z.real(), z.imag(), tol, in, out);
  SYK_CUDA_CHECK(cudaGetLastError());
  SYK_CUDA_CHECK(cudaGraphLaunch(it->second, st));
  count_launch(4);  // set_job, and the graph's copy in, loop set-up and copy out
  return SYK_OK;
}

int chain_end(KrylovWS& ws, cudaStream_t st) {
  DevCtl h;
  SYK_CUDA_CHECK(cudaMemcpyAsync(&h, ws.ctl, sizeof(DevCtl), cudaMemcpyDeviceToHost, st));
  SYK_CUDA_CHECK(cudaStreamSynchronize(st));
  count_applies(h.applies);
  count_bases(h.bases);
  count_launch(h.launches);
  const int64_t mv[kMvKinds] = {h.mv[0], h.mv[1], h.mv[2]};
  count_matvec_replay(mv);
  if (h.err & 4) {
    set_error("apply_H: a bounded wait for a staged tile gave up");
    return SYK_ETIMEOUT;
  }
  if (h.err & 1) {
    set_error("expmv: non-finite Lanczos scalar");
    return SYK_ENUMERIC;
  }
  if (h.err & 2) {
    set_error("expmv: tridiagonal eigensolver did not converge");
    return SYK_ENUMERIC;
  }
  if (h.err & 8) {
    set_error("expmv: Krylov step collapsed; raise krylov_dim or tol");
    return SYK_ENUMERIC;
  }
  if (h.err & 16) {
    set_error("expmv: more than 100000 Krylov steps");
    return SYK_ENUMERIC;
  }
  return SYK_OK;
}

namespace {
template <typename R>
int lanczos_steps_T(const ApplyParams& P_in, int dtype, KrylovWS& ws, int j0, int j1, cudaStream_t st) {
  const ApplyParams P = ws.with_split(P_in);
  const double bt = (dtype == SYK_C64 ? 64.0 * 5.96e-8 : 64.0 * 1.11e-16);
  // two passes of classical Gram-Schmidt against the whole basis for both vector types:
  // Ritz values of a long run need the basis orthogonal to working precision
  for (int j = j0; j < j1; ++j) SYK_TRY(lanczos_step<R>(P, dtype, ws, j, kOrthFull, true, bt, st));
  return SYK_OK;
}
}  // namespace

int lanczos_begin(int dtype, const void* psi, KrylovWS& ws, cudaStream_t st) {
  SYK_CUDA_CHECK(cudaMemsetAsync(ws.status, 0, sizeof(int) * 4, st));
  if (dtype == SYK_C64) Ops<float>::dots(ws, 1, psi, 0, psi, st);
  else Ops<double>::dots(ws, 1, psi, 0, psi, st);
  reduce_parts(ws, 1, ws.h1, st);
  k_norm_init<<<(int(ws.B) + 127) / 128, 128, 0, st>>>(int(ws.B), ws.h1, ws.beta0, ws.inv, ws.sc, ws.status);
  count_launch();
  if (dtype == SYK_C64) Ops<float>::scale(ws, psi, ws.vec(0), ws.inv, st);
  else Ops<double>::scale(ws, psi, ws.vec(0), ws.inv, st);
  SYK_CUDA_CHECK(cudaGetLastError());
  return SYK_OK;
}

int lanczos_steps(const ApplyParams& P, int dtype, KrylovWS& ws, int j0, int j1, cudaStream_t st) {
  if (j0 < 0 || j1 > ws.m || j0 > j1) {
    set_error("lanczos_steps: steps [%d, %d) outside the workspace's %d", j0, j1, ws.m);
    return SYK_EINVAL;
  }
  return dtype == SYK_C64 ? lanczos_steps_T<float>(P, dtype, ws, j0, j1, st)
                          : lanczos_steps_T<double>(P, dtype, ws, j0, j1, st);
}

}  // namespace syk

// ---------------------------------------------------------------- C ABI
using namespace syk;

extern "C" int syk_lanczos_orth(int dtype, int mode) {
  clear_error();
  if (!dtype_ok(dtype)) {
    set_error("syk_lanczos_orth: dtype must be SYK_C64 or SYK_C128 (got %d)", dtype);
    return SYK_EINVAL;
  }
  const int prev = g_orth[dtype].load();
  if (mode < 0) return prev;
  if (mode != kOrthFull && mode != kOrthLocal) {
    set_error("syk_lanczos_orth: mode must be 0 (full Gram-Schmidt) or 1 (three-term recurrence), got %d", mode);
    return SYK_EINVAL;
  }
  g_orth[dtype] = mode;
  bump_graph_epoch();  // captured segments carry the other kernel sequence
  return prev;
}

extern "C" size_t syk_workspace_bytes(int N, int dtype, int krylov_dim, int64_t batch, int kind) {
  (void)kind;
  if (N < 4 || (N & 1) || N > 64 || !dtype_ok(dtype) || krylov_dim < 1 || krylov_dim > SYK_MAX_KRYLOV ||
      batch < 1 || batch > 256)
    return 0;
  const int64_t D = int64_t(1) << (N / 2 - 1);
  return krylov_ws_bytes(D, dtype, krylov_dim, batch);
}

extern "C" int syk_expmv(const syk_terms* terms, int parity, int dtype, double z_re, double z_im, const void* psi,
                         void* out, int64_t batch, int krylov_dim, double tol, void* workspace, size_t ws_bytes,
                         void* stream, int* nsteps) {
  syk::NvtxRange nvtx_range_("syk_expmv");
  clear_error();
  if (!psi || !out || batch < 1 || batch > 256 || krylov_dim < 2 || krylov_dim > SYK_MAX_KRYLOV) {
    set_error("syk_expmv: invalid argument (batch=%lld krylov_dim=%d)", (long long)batch, krylov_dim);
    return SYK_EINVAL;
  }
  if (!std::isfinite(z_re) || !std::isfinite(z_im)) {
    set_error("syk_expmv: non-finite z");
    return SYK_EINVAL;
  }
  ApplyParams P;
  SYK_TRY(make_apply_params(terms, parity, dtype, &P));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t need = krylov_ws_bytes(P.D, dtype, krylov_dim, batch);
  void* base = workspace;
  bool owned = false;
  if (!base) {
    cudaError_t e = cudaMallocAsync(&base, need, st);
    if (e != cudaSuccess) {
      set_error("syk_expmv: cannot allocate %zu bytes of workspace: %s", need, cudaGetErrorString(e));
      return SYK_ENOMEM;
    }
    owned = true;
    ws_bytes = need;
  }
  KrylovWS ws;
  int rc = krylov_ws_carve(&ws, base, ws_bytes, P.D, dtype, krylov_dim, batch);
  if (rc == SYK_OK) rc = expmv_impl(P, dtype, {z_re, z_im}, psi, out, batch, tol, ws, st, nsteps);
  if (owned) cudaFreeAsync(base, st);
  return rc;
}

extern "C" int syk_tridiag_expm(int m, int64_t batch, const double* alpha, const double* beta, const double* beta0,
                                double z_re, double z_im, double* out, void* stream) {
  syk::NvtxRange nvtx_range_("syk_tridiag_expm");
  clear_error();
  if (m < 1 || m > SYK_MAX_KRYLOV || batch < 1 || batch > 65535 || !alpha || !beta0 || !out || (m > 1 && !beta)) {
    set_error("syk_tridiag_expm: invalid argument (m=%d batch=%lld)", m, (long long)batch);
    return SYK_EINVAL;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int B = int(batch);
  // scratch: beta padded to m rows, theta, Q, sb, status
  const size_t nb = align_up(sizeof(double) * m * B), nq = align_up(sizeof(double) * m * m * B);
  const size_t total = 3 * nb + nq + align_up(sizeof(double) * B) + 256;
  char* base = nullptr;
  SYK_CUDA_CHECK(cudaMallocAsync((void**)&base, total, st));
  double* bpad = (double*)base;
  double* theta = (double*)(base + nb);
  double* Q = (double*)(base + 2 * nb);
  double* sb = (double*)(base + 2 * nb + nq);
  int* status = (int*)(base + 2 * nb + nq + align_up(sizeof(double) * B));
  cudaMemsetAsync(bpad, 0, nb, st);
  cudaMemsetAsync(status, 0, 16, st);
  if (m > 1) cudaMemcpyAsync(bpad, beta, sizeof(double) * (m - 1) * B, cudaMemcpyDeviceToDevice, st);
  k_tridiag_eig<true><<<B, 32, tridiag_smem(m, true), st>>>(m, B, alpha, bpad, nullptr, z_re, z_im, 1.0, 1.0, theta, Q,
                                                             sb, status);
  k_tridiag_coef<<<B, 64, 0, st>>>(m, B, theta, Q, beta0, z_re, z_im, nullptr, 1.0, (double2*)out);
  count_launch(2);
  cudaError_t e = cudaGetLastError();
  int hstat = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hstat, status, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFreeAsync(base, st);
  if (e != cudaSuccess) {
    set_error("syk_tridiag_expm: %s", cudaGetErrorString(e));
    return SYK_ECUDA;
  }
  if (hstat) {
    set_error("syk_tridiag_expm: eigensolver did not converge");
    return SYK_ENUMERIC;
  }
  return SYK_OK;
}

// ---------------------------------------------------------------- static-scratch variant
// Workspace of syk_expmv_static: one fixed array of device memory per GPU that
// loads the library.  Host code only ever uses its device address, looked up
// once per device with cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_expmv_static_scratch[SYK_STATIC_SCRATCH_BYTES];

namespace {
std::mutex g_static_mtx;
void* g_static_addr[128] = {};
}  // namespace

extern "C" int syk_expmv_static(const syk_terms* terms, int parity, int dtype, double z_re, double z_im,
                                const void* psi, void* out, int64_t batch, int krylov_dim, double tol, void* stream,
                                int* nsteps) {
  syk::NvtxRange nvtx_range_("syk_expmv_static");
  clear_error();
  if (!terms || !psi || !out || batch < 1 || batch > 256 || krylov_dim < 2 || krylov_dim > SYK_MAX_KRYLOV ||
      !dtype_ok(dtype) || (parity != 0 && parity != 1)) {
    set_error("syk_expmv_static: invalid argument (batch=%lld krylov_dim=%d dtype=%d parity=%d)", (long long)batch,
              krylov_dim, dtype, parity);
    return SYK_EINVAL;
  }
  if (!std::isfinite(z_re) || !std::isfinite(z_im)) {
    set_error("syk_expmv_static: non-finite z");
    return SYK_EINVAL;
  }
  int dev = -1;
  SYK_CUDA_CHECK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 128) {
    set_error("syk_expmv_static: device ordinal %d out of range", dev);
    return SYK_EINVAL;
  }
  const size_t need = krylov_ws_bytes(terms->D, dtype, krylov_dim, batch);
  if (need > SYK_STATIC_SCRATCH_BYTES) {
    set_error("syk_expmv_static: needs %zu bytes of workspace, more than the %u-byte static scratch; "
              "use syk_expmv or a smaller batch or krylov_dim", need, (unsigned)SYK_STATIC_SCRATCH_BYTES);
    return SYK_ENOMEM;
  }
  if (terms->dev.device != dev) {
    set_error("syk_expmv_static: the term set is not on device %d yet; make any other call with it on this "
              "device first (that call uploads it)", dev);
    return SYK_EINVAL;
  }
  void* base = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_static_mtx);
    if (!g_static_addr[dev]) {
      void* p = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&p, g_expmv_static_scratch);
      if (e != cudaSuccess || !p) {
        set_error("syk_expmv_static: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
        return SYK_ECUDA;
      }
      g_static_addr[dev] = p;
    }
    base = g_static_addr[dev];
  }
  ApplyParams P;
  SYK_TRY(make_apply_params(terms, parity, dtype, &P));
  P.no_alloc = true;
  KrylovWS ws;
  SYK_TRY(krylov_ws_carve(&ws, base, SYK_STATIC_SCRATCH_BYTES, P.D, dtype, krylov_dim, batch));
  alignas(16) unsigned char stage[64];
  ws.host_stage = stage;
  return expmv_impl(P, dtype, {z_re, z_im}, psi, out, batch, tol, ws, static_cast<cudaStream_t>(stream), nsteps);
}
