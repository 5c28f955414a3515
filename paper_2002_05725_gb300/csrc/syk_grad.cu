// Gradients of the correlators with respect to every coupling J_ijkl and beta
// (reverse mode through the Krylov evolutions).
//
// A correlator is a sesquilinear form <a|b> of two chains of operators applied to
// the random states: a = A_K..A_1 psi~, b = B_L..B_1 psi~, each operator either an
// exponential e^{zH} (z = -c_beta beta - i c_t t) or one Majorana chi_i (Eq. F_reg,
// Eq. G, Eq. q_typicality).  For an exponential M = e^{zH} with input x and the
// adjoint vector lam at its output, Duhamel's formula gives
//   <lam| dM/dJ_T |x> = z int_0^1 <e^{(1-v) conj(z) H} lam| P_T |e^{v z H} x> dv,
// P_T = dH/dJ_T = chi_i chi_j chi_k chi_l (Eq. 1).  The integral is split into S
// sub-intervals with 4 Gauss-Legendre nodes each.  The adjoint lam(v) marches from
// v = 1 down to 0 while the forward state psi(v) is needed in the same decreasing
// order, so psi is checkpointed every ceil(sqrt(S)) sub-intervals on a forward
// sweep and each segment is recomputed from its checkpoint (O(sqrt S) stored states).
// At every node one pass over the state (K6, k_term_grad) accumulates
// <lam|P_T|psi> for all C(N,4) terms at once: terms sharing an X-mask and the
// Z-mask bits off their support form one group, and each row adds
// conj(lam[x]) psi[x^m] (-1)^popcount(zeta & x) with the signs (-1)^popcount(s & u(x))
// of the group's 2^k terms.  d/dbeta of e^{-c beta H} is -c H e^{-c beta H}.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <complex>
#include <condition_variable>
#include <functional>
#include <mutex>
#include <string>
#include <thread>
#include <type_traits>
#include <vector>

#include "syk_cplx.cuh"
#include "syk_krylov.cuh"

namespace syk {
namespace {

// v's bits deposited, lowest first, at the set bits of mask
__device__ __forceinline__ uint32_t deposit_bits(uint32_t v, uint32_t mask) {
  uint32_t r = 0;
  for (uint32_t bit = 1; mask; bit <<= 1) {
    const uint32_t low = mask & (0u - mask);
    if (v & bit) r |= low;
    mask ^= low;
  }
  return r;
}

// Blocks of 2^G rows xb + o_q of one thread (term kernel below): the G lowest walked bits in
// Gray order (o_q = their deposit of q ^ (q >> 1)), the other walked bits (hmask) in
// increasing order.  Within a block the row parity alternates (pb, pb^1, ...) and the zeta sign
// is the block's sign times a per-thread constant f_q, so only xb needs popcounts; lam rows sit
// at xb + o_q and psi rows at (xb ^ m) + d_q, because xb has no bits at the Gray bits.
template <int G, typename R, typename C>
__device__ __forceinline__ void term_blocks(const C* __restrict__ lam, const C* __restrict__ psi, size_t bs, int col,
                                            uint32_t x0, uint32_t jmask, uint4 rec, int nb, int sector, R& a0r,
                                            R& a0i, R& a1r, R& a1i) {
  constexpr int NQ = 1 << G;
  uint32_t e[G], low = 0, rest = jmask;
#pragma unroll
  for (int i = 0; i < G; ++i) {
    e[i] = rest & (0u - rest);
    rest ^= e[i];
    low |= e[i];
  }
  const uint32_t hmask = rest, mj = rec.x & low;
  const uint32_t zc = rec.y & ((1u << nb) - 1u), zt = (rec.y >> nb) & 1u;
  ptrdiff_t lo[NQ], po[NQ];
  R f[NQ];
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    const uint32_t gq = (uint32_t)(q ^ (q >> 1));
    uint32_t o = 0;
#pragma unroll
    for (int i = 0; i < G; ++i)
      if ((gq >> i) & 1u) o |= e[i];
    lo[q] = (ptrdiff_t)o * (ptrdiff_t)bs;
    po[q] = ((ptrdiff_t)(mj ^ o) - (ptrdiff_t)mj) * (ptrdiff_t)bs;
    f[q] = ((__popc(zc & o) ^ (zt & (uint32_t)(q & 1))) & 1) ? R(-1) : R(1);
  }
  uint32_t hi = 0;
  do {
    const uint32_t xb = x0 | hi;
    const C* lb = lam + (size_t)xb * bs + col;
    const C* pb_ = psi + (size_t)(xb ^ rec.x) * bs + col;
    C l[NQ], p[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      l[q] = lb[lo[q]];
      p[q] = pb_[po[q]];
    }
    const uint32_t pb = (uint32_t)((__popc(xb) + sector) & 1);
    const uint32_t sg = (uint32_t)(__popc(zc & xb) & 1) ^ (zt & pb);
    // even rows (parity pb) and odd rows (parity pb ^ 1), signs applied: conj(l) p
    R er = R(0), ei = R(0), orr = R(0), oi = R(0);
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      const R xr = f[q] * (l[q].x * p[q].x + l[q].y * p[q].y);
      const R xi = f[q] * (l[q].x * p[q].y - l[q].y * p[q].x);
      if (q & 1) {
        orr += xr;
        oi += xi;
      } else {
        er += xr;
        ei += xi;
      }
    }
    if (sg) {
      er = -er;
      ei = -ei;
      orr = -orr;
      oi = -oi;
    }
    if (pb) {
      a1r += er;
      a1i += ei;
      a0r += orr;
      a0i += oi;
    } else {
      a0r += er;
      a0i += ei;
      a1r += orr;
      a1i += oi;
    }
    hi = ((hi | ~hmask) + 1u) & hmask;
  } while (hi != 0u);
}

// partial[((g*RC + chunk)*16 + s)*Bt + c0 + b] = sum over the rows x of the chunk of
// conj(lam[x][c0+b]) psi[x^m][c0+b] (-1)^popcount(zeta & xf) (-1)^popcount(s & u(xf)), u(xf) = the
// bits of the full index xf at the group's k support positions.
// The rows of the nb-bit compact index are enumerated per group: the LB lane bits of a thread
// (r = tid / Bc) are the support positions below the top spin plus the lowest other bits, the
// CB chunk bits the highest of the rest, and the thread walks the remaining bits.  So u is the
// same for all rows of a thread except for the top spin (the parity bit, set by the row), and
// the thread sums its products in two register pairs (parity 0 and 1), without a per-row
// shared-memory update.  Then each thread forms the 2^k-point Walsh transform of its (at most
// two) nonzero bins, and the threads of each column are summed in a fixed order
// (deterministic).  Lanes r >= 2^LB (sectors smaller than the lane count) hold no rows.
template <typename R>
__global__ void k_term_grad(const uint4* __restrict__ grec, int n, int sector, int LB, int CB, int Bt, int c0, int Bc,
                            const typename CT<R>::T* __restrict__ lam, const typename CT<R>::T* __restrict__ psi,
                            double2* __restrict__ partial) {
  using C = typename CT<R>::T;
  extern __shared__ __align__(16) unsigned char tg_smem[];
  R* bins = reinterpret_cast<R*>(tg_smem);  // [32][NT]: real parts of s = 0..15, then imaginary parts
  const int g = blockIdx.x, chunk = blockIdx.y, RC = gridDim.y;
  const int tid = threadIdx.x, NT = blockDim.x;
  const int b = tid % Bc, r = tid / Bc;
  const int rows_per_pass = NT / Bc;
  const uint4 rec = __ldg(&grec[g]);
  const int k = (int)rec.w, ns = 1 << k;
  const int nb = n - 1;  // compact bits; full-index bit nb is the parity (top) spin
  auto supp_pos = [&](int kk) { return (int)((rec.z >> (8 * kk)) & 0xffu) + kk; };  // ascending
  uint32_t smask = 0;
  int ktop = -1;
  for (int kk = 0; kk < k; ++kk) {
    if (supp_pos(kk) < nb) smask |= 1u << supp_pos(kk);
    else ktop = kk;
  }
  uint32_t lmask = smask;
  for (int bit = 0; __popc(lmask) < LB; ++bit) lmask |= 1u << bit;
  uint32_t rest = ((1u << nb) - 1u) & ~lmask, cmask = 0;
  for (int i = 0; i < CB; ++i) {
    const uint32_t hb = 1u << (31 - __clz(rest));
    cmask |= hb;
    rest ^= hb;
  }
  const uint32_t jmask = rest;
  R a0r = R(0), a0i = R(0), a1r = R(0), a1i = R(0);
  const uint32_t x0 = deposit_bits((uint32_t)r, lmask) | deposit_bits((uint32_t)chunk, cmask);
  // one row: conj(lam) psi with the sign (-1)^popcount(zeta & xf), into the bin of its parity
  auto add_row = [&](uint32_t xc) {
    const uint32_t par = (uint32_t)((__popc(xc) + sector) & 1);
    const uint32_t xf = xc | (par << nb);
    const C l = lam[(size_t)xc * Bt + c0 + b];
    const C p = psi[(size_t)(xc ^ rec.x) * Bt + c0 + b];
    R cr = l.x * p.x + l.y * p.y;  // conj(l) * p
    R ci = l.x * p.y - l.y * p.x;
    if (__popc(rec.y & xf) & 1) {
      cr = -cr;
      ci = -ci;
    }
    if (par) {
      a1r += cr;
      a1i += ci;
    } else {
      a0r += cr;
      a0i += ci;
    }
  };
  if (r < (1 << LB)) {
    const int nj = __popc(jmask);  // 2^nj rows per thread
    // blocks of 8 rows for complex128, 4 for complex64 (measured at N = 28, 8 states: 8-row
    // blocks 160 against 148 us per complex64 launch, 10.5 against 11.1 s per complex128 call)
    constexpr bool wide = std::is_same<R, double>::value;
    if (wide && nj >= 3) {
      term_blocks<3, R, C>(lam, psi, (size_t)Bt, c0 + b, x0, jmask, rec, nb, sector, a0r, a0i, a1r, a1i);
    } else if (nj >= 2) {
      term_blocks<2, R, C>(lam, psi, (size_t)Bt, c0 + b, x0, jmask, rec, nb, sector, a0r, a0i, a1r, a1i);
    } else {
      uint32_t xj = 0;
      do {
        add_row(x0 | xj);
        xj = ((xj | ~jmask) + 1u) & jmask;
      } while (xj != 0u);
    }
  }
  // bins of this thread: u0 (parity 0) and u1 (parity 1), equal unless the top spin is a support bit
  uint32_t uc = 0;
  for (int kk = 0; kk < k; ++kk)
    if (kk != ktop) uc |= ((x0 >> supp_pos(kk)) & 1u) << kk;
  const uint32_t u0 = uc, u1 = ktop >= 0 ? (uc | (1u << ktop)) : uc;
  // Walsh transform of the two bins: W_s = sum_u (-1)^popcount(s & u) bin_u
#pragma unroll
  for (int sidx = 0; sidx < 16; ++sidx)
    if (sidx < ns) {
      const R s0 = (__popc((uint32_t)sidx & u0) & 1) ? R(-1) : R(1);
      const R s1 = (__popc((uint32_t)sidx & u1) & 1) ? R(-1) : R(1);
      bins[sidx * NT + tid] = s0 * a0r + s1 * a1r;
      bins[(16 + sidx) * NT + tid] = s0 * a0i + s1 * a1i;
    }
  __syncthreads();
  // column b's sum over its threads b, b + Bc, b + 2 Bc, ... in increasing order
  for (int o = tid; o < ns * Bc; o += NT) {
    const int sidx = o / Bc, bb = o - sidx * Bc;
    R sx = R(0), sy = R(0);
    for (int j = 0; j < rows_per_pass; ++j) {
      sx += bins[sidx * NT + bb + j * Bc];
      sy += bins[(16 + sidx) * NT + bb + j * Bc];
    }
    partial[(((size_t)g * RC + chunk) * 16 + sidx) * Bt + c0 + bb] = make_double2((double)sx, (double)sy);
  }
}

// acc[T*B + b] += coef * phase_T * sum_chunks partial[group(T), chunk, s(T), b]
__global__ void k_term_grad_accum(int64_t nterms, int B, int RC, const int* __restrict__ tgroup,
                                  const uint8_t* __restrict__ ts, const double2* __restrict__ tphase,
                                  const double2* __restrict__ partial, double cre, double cim,
                                  double2* __restrict__ acc) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= nterms * B) return;
  const int64_t T = idx / B;
  const int b = (int)(idx - T * B);
  const int g = tgroup[T], s = ts[T];
  double vx = 0.0, vy = 0.0;
  for (int c = 0; c < RC; ++c) {
    const double2 p = partial[(((size_t)g * RC + c) * 16 + s) * B + b];
    vx += p.x;
    vy += p.y;
  }
  const double2 ph = tphase[T];
  const double wx = ph.x * vx - ph.y * vy, wy = ph.x * vy + ph.y * vx;  // phase * v
  double2 a = acc[idx];
  a.x += cre * wx - cim * wy;
  a.y += cre * wy + cim * wx;
  acc[idx] = a;
}

// out[T*B + b] += coef[b] * (gb[T*B + b] + conj(ga[T*B + b]))   (T < nrows)
__global__ void k_grad_combine(int64_t nrows, int B, const double2* __restrict__ gb, const double2* __restrict__ ga,
                               const double2* __restrict__ coef, double2* __restrict__ out) {
  const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (idx >= nrows * B) return;
  const int b = (int)(idx % B);
  const double vx = gb[idx].x + ga[idx].x, vy = gb[idx].y - ga[idx].y;
  const double2 c = coef[b];
  double2 o = out[idx];
  o.x += c.x * vx - c.y * vy;
  o.y += c.x * vy + c.y * vx;
  out[idx] = o;
}

// acc[b] += coef * d[b]
__global__ void k_axpy_cols(int B, const double2* __restrict__ d, double cre, double cim, double2* __restrict__ acc) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  const double2 v = d[b];
  acc[b].x += cre * v.x - cim * v.y;
  acc[b].y += cre * v.y + cim * v.x;
}

struct Op {
  int kind;   // 0: e^{zH}, z = -cb*beta - i*ct*t;  1: chi_maj
  double cb, ct;
  int maj;
};

// Gauss-Legendre nodes and weights on [-1, 1] (4 points)
const double kGLx[4] = {-0.8611363115940526, -0.3399810435848563, 0.3399810435848563, 0.8611363115940526};
const double kGLw[4] = {0.3478548451374538, 0.6521451548625461, 0.6521451548625461, 0.3478548451374538};

// One host thread that runs submitted jobs (here: forward Krylov evolutions on the engine's
// second stream) one at a time.  It lives as long as its engine, so the evolutions' graph
// cache, which is kept per host thread, survives from one segment to the next.
struct Worker {
  std::thread th;
  std::mutex m;
  std::condition_variable cv;
  std::function<int()> job;
  bool has = false, done = true, quit = false;
  int rc = SYK_OK;
  std::string err;

  void start(int dev) {
    th = std::thread([this, dev] {
      cudaSetDevice(dev);
      for (;;) {
        std::unique_lock<std::mutex> lk(m);
        cv.wait(lk, [&] { return has || quit; });
        if (quit) return;
        std::function<int()> f = std::move(job);
        has = false;
        lk.unlock();
        const int r = f();
        std::string e = r != SYK_OK ? std::string(syk_last_error()) : std::string();
        lk.lock();
        rc = r;
        err = std::move(e);
        done = true;
        cv.notify_all();
      }
    });
  }
  void submit(std::function<int()> f) {
    std::lock_guard<std::mutex> lk(m);
    job = std::move(f);
    has = true;
    done = false;
    cv.notify_all();
  }
  // waits for the submitted job; returns its code (message in *e)
  int wait(std::string* e) {
    std::unique_lock<std::mutex> lk(m);
    cv.wait(lk, [&] { return done; });
    *e = err;
    return rc;
  }
  void stop() {
    {
      std::lock_guard<std::mutex> lk(m);
      quit = true;
    }
    cv.notify_all();
    if (th.joinable()) th.join();
  }
};

struct GradEngine {
  const syk_terms* terms = nullptr;
  int dtype = 0, krylov = 0;
  int64_t B = 0, D = 0;
  double beta = 0, t = 0, tol = 0, rho = 1.0, dz = 0.05;  // dz: max |z| per sub-interval
  cudaStream_t st = nullptr;
  // the forward evolutions of the backward sweep run on st2 (own workspace ws2, driven from a
  // second host thread) while the adjoint evolution of the same segment runs on st
  cudaStream_t st2 = nullptr;
  cudaEvent_t ev_main = nullptr, ev_fwd = nullptr;
  int device = 0;
  Worker worker;
  ApplyParams P[2];
  KrylovWS ws, ws2;
  std::vector<void*> owned;
  size_t vb = 0;
  // term kernel shape: columns in blocks of Bc <= 16, 2^LB row lanes, RC = 2^CB row chunks
  int RC = 1, CB = 0, LB = 0, Bc = 1, bdim = 0;
  double2* partial = nullptr;
  double2* dots = nullptr;  // B

  ~GradEngine() {
    worker.stop();
    if (st2) {
      cudaStreamSynchronize(st2);  // ws2 and node vectors are freed on st below
      cudaStreamDestroy(st2);
    }
    if (ev_main) cudaEventDestroy(ev_main);
    if (ev_fwd) cudaEventDestroy(ev_fwd);
    for (void* p : owned) cudaFreeAsync(p, st);
  }
  int alloc(void** p, size_t bytes) {
    cudaError_t e = cudaMallocAsync(p, bytes, st);
    if (e != cudaSuccess) {
      set_error("gradient: cannot allocate %zu bytes: %s", bytes, cudaGetErrorString(e));
      *p = nullptr;
      return SYK_ENOMEM;
    }
    owned.push_back(*p);
    return SYK_OK;
  }
  int vec(void** p) { return alloc(p, vb); }
  // reusable state vectors (returned with put)
  std::vector<void*> free_vecs;
  int get(void** p) {
    if (!free_vecs.empty()) {
      *p = free_vecs.back();
      free_vecs.pop_back();
      return SYK_OK;
    }
    return vec(p);
  }
  void put(void* p) {
    if (p) free_vecs.push_back(p);
  }

  int init() {
    SYK_TRY(make_apply_params(terms, 0, dtype, &P[0]));
    SYK_TRY(make_apply_params(terms, 1, dtype, &P[1]));
    SYK_TRY(ensure_grad_groups(terms));
    D = terms->D;
    vb = size_t(D) * B * dtype_size(dtype);
    void* w = nullptr;
    const size_t wsb = krylov_ws_bytes(D, dtype, krylov, B);
    SYK_TRY(alloc(&w, wsb));
    SYK_TRY(krylov_ws_carve(&ws, w, wsb, D, dtype, krylov, B));
    SYK_TRY(alloc(&w, wsb));
    SYK_TRY(krylov_ws_carve(&ws2, w, wsb, D, dtype, krylov, B));
    SYK_CUDA_CHECK(cudaGetDevice(&device));
    SYK_CUDA_CHECK(cudaStreamCreateWithFlags(&st2, cudaStreamNonBlocking));
    SYK_CUDA_CHECK(cudaEventCreateWithFlags(&ev_main, cudaEventDisableTiming));
    SYK_CUDA_CHECK(cudaEventCreateWithFlags(&ev_fwd, cudaEventDisableTiming));
    worker.start(device);
    // 256 threads: Bc columns x 256 / Bc row lanes (at least 16, so that the <= 4 support bits
    // below the top spin fit in the lane bits); row chunks of at least 64 rows per thread, so
    // the per-block epilogue (Walsh transform of the bins, column sums) costs a fraction of the
    // row loop
    Bc = int(std::min<int64_t>(B, 16));
    int lanes = 1;
    while (lanes * 2 * Bc <= 256) lanes *= 2;
    bdim = Bc * lanes;
    const int nb = terms->n - 1;
    LB = 0;
    while ((1 << LB) < lanes && LB < nb) ++LB;
    CB = std::max(0, std::min(6, nb - LB - 6));
    RC = 1 << CB;
    void* p = nullptr;
    SYK_TRY(alloc(&p, sizeof(double2) * size_t(terms->ngg) * RC * 16 * B));
    partial = static_cast<double2*>(p);
    SYK_TRY(alloc(&p, sizeof(double2) * B));
    dots = static_cast<double2*>(p);
    // spectral-radius scale of H for the quadrature step: 3 x sqrt(Tr H^2 / dim) = 3 sqrt(sum J^2 / 16)
    double s2 = 0.0;
    for (double j : terms->J) s2 += j * j;
    rho = 3.0 * std::sqrt(s2 / 16.0);
    return SYK_OK;
  }

  std::complex<double> z_of(const Op& o) const { return {-o.cb * beta, -o.ct * t}; }

  int expmv(int sector, std::complex<double> z, const void* in, void* out) {
    return expmv_impl(P[sector], dtype, z, in, out, B, tol, ws, st, nullptr);
  }
  // outs[k] = e^{fr[k] z H} in from the Krylov bases of one evolution (no matvecs per output)
  int expmv_points(int sector, std::complex<double> z, const void* in, const double* fr, int nf, void* const* outs) {
    return syk::expmv_points(P[sector], dtype, z, in, fr, nf, outs, B, tol, ws, st);
  }
  int copy(void* dst, const void* src) {
    SYK_CUDA_CHECK(cudaMemcpyAsync(dst, src, vb, cudaMemcpyDeviceToDevice, st));
    return SYK_OK;
  }

  // acc[T][b] += coef * <lam|P_T|psi>
  int term_grad(int sector, const void* lam, const void* psi, std::complex<double> coef, double2* acc) {
    dim3 grid(terms->ngg, RC);
    // bins: 32 x (at most 256 threads) values of the vector type
    SYK_TRY(ensure_smem_limit((const void*)k_term_grad<float>, 32 * 256 * (int)sizeof(float)));
    SYK_TRY(ensure_smem_limit((const void*)k_term_grad<double>, 32 * 256 * (int)sizeof(double)));
    for (int c0 = 0; c0 < int(B); c0 += Bc) {
      const int bc = std::min<int>(Bc, int(B) - c0);
      const int nt = bc * (bdim / Bc);
      if (dtype == SYK_C64)
        k_term_grad<float><<<grid, nt, 32 * nt * sizeof(float), st>>>(
            terms->d_gg_rec, terms->n, sector, LB, CB, int(B), c0, bc, (const float2*)lam, (const float2*)psi, partial);
      else
        k_term_grad<double><<<grid, nt, 32 * nt * sizeof(double), st>>>(
            terms->d_gg_rec, terms->n, sector, LB, CB, int(B), c0, bc, (const double2*)lam, (const double2*)psi,
            partial);
      count_launch();
    }
    const int64_t n = terms->nterms * B;
    k_term_grad_accum<<<unsigned((n + 255) / 256), 256, 0, st>>>(terms->nterms, int(B), RC, terms->d_term_group,
                                                                 terms->d_term_s, terms->d_term_phase, partial,
                                                                 coef.real(), coef.imag(), acc);
    count_launch();
    SYK_CUDA_CHECK(cudaGetLastError());
    return SYK_OK;
  }

  // Forward pass of a chain: xs[k] = input of op k (xs[0] = psi), returns output sectors.
  int forward(const std::vector<Op>& ops, const void* psi, std::vector<void*>& xs, std::vector<int>& sec) {
    xs.assign(ops.size() + 1, nullptr);
    sec.assign(ops.size() + 1, 0);
    xs[0] = const_cast<void*>(psi);
    for (size_t k = 0; k < ops.size(); ++k) {
      SYK_TRY(get(&xs[k + 1]));
      const Op& o = ops[k];
      if (o.kind == 1) {
        SYK_TRY(launch_apply_chi(terms->N, o.maj, sec[k], dtype, xs[k], xs[k + 1], B, st));
        sec[k + 1] = 1 - sec[k];
      } else {
        SYK_TRY(expmv(sec[k], z_of(o), xs[k], xs[k + 1]));
        sec[k + 1] = sec[k];
      }
    }
    return SYK_OK;
  }

  // lam: adjoint at the output of the exponential (overwritten with the adjoint at its input);
  // x: input; y: output.  Adds <lam|dM/dJ_T|x> to gJ and <lam|dM/dbeta|x> to gb.
  int exp_adjoint(const Op& o, int sector, const void* x, const void* y, void* lam, double2* gJ, double2* gb) {
    const std::complex<double> z = z_of(o);
    if (z == std::complex<double>(0.0, 0.0)) return SYK_OK;  // identity
    if (o.cb != 0.0) {
      // d/dbeta e^{-cb beta H} = -cb H e^{-cb beta H}:  <lam| -cb H y>
      void* hy = nullptr;
      SYK_TRY(get(&hy));
      SYK_TRY(launch_apply_H(P[sector], dtype, y, hy, B, st));
      SYK_TRY(dot_columns(lam, hy, D, B, dtype, ws, dots, st));
      k_axpy_cols<<<unsigned((B + 127) / 128), 128, 0, st>>>(int(B), dots, -o.cb, 0.0, gb);
      count_launch();
      put(hy);
    }
    const int S = std::max(1, int(std::ceil(std::abs(z) * rho / dz)));
    const int c = std::max(1, int(std::ceil(std::sqrt(double(S)))));
    const int nseg = (S + c - 1) / c;
    const std::complex<double> zs = z / double(S), zbar = std::conj(z);
    // per segment of up to c sub-intervals: the forward states at its 4c Gauss-Legendre nodes
    // from one evolution of its checkpoint, and the adjoint at those nodes and at the segment's
    // start from one evolution of the adjoint (states read off the Krylov bases at fractions of
    // the step: no matvecs per node)
    std::vector<void*> ckpt(nseg), nodeF(4 * c), nodeA(4 * c);
    for (auto& p : ckpt) SYK_TRY(get(&p));
    for (auto& p : nodeF) SYK_TRY(get(&p));
    for (auto& p : nodeA) SYK_TRY(get(&p));
    std::vector<double> frf(4 * c), fra(4 * c + 1);
    std::vector<void*> outa(4 * c + 1);
    // forward sweep: checkpoints psi(s/S) for s = 0, c, 2c, ...
    SYK_TRY(copy(ckpt[0], x));
    for (int sg = 1; sg < nseg; ++sg) {
      SYK_TRY(copy(ckpt[sg], ckpt[sg - 1]));
      SYK_TRY(expmv(sector, zs * double(c), ckpt[sg], ckpt[sg]));  // c sub-intervals in one evolution
    }
    // backward: the adjoint marches from v = 1 to 0, one segment at a time
    for (int sg = nseg - 1; sg >= 0; --sg) {
      const int s0 = sg * c, s1 = std::min(S, s0 + c), L = s1 - s0;
      // forward nodes, ascending: sub-interval s, node q at fraction ((s - s0) + (1 + x_q)/2) / L
      for (int s = s0; s < s1; ++s)
        for (int q = 0; q < 4; ++q) frf[(s - s0) * 4 + q] = ((s - s0) + 0.5 * (1.0 + kGLx[q])) / L;
      // forward nodes on st2, after everything st has queued (the checkpoint, and the previous
      // segment's term kernels that read nodeF), from a second host thread: its convergence
      // checks then do not hold up the adjoint evolution below
      SYK_CUDA_CHECK(cudaEventRecord(ev_main, st));
      SYK_CUDA_CHECK(cudaStreamWaitEvent(st2, ev_main, 0));
      const std::complex<double> zf = zs * double(L);
      void* const ck = ckpt[sg];
      worker.submit([this, sector, zf, ck, L, &frf, &nodeF] {
        return syk::expmv_points(P[sector], dtype, zf, ck, frf.data(), 4 * L, nodeF.data(), B, tol, ws2, st2);
      });
      // adjoint nodes by increasing distance from s1/S (s = s1-1 .. s0, q = 3 .. 0), then v = s0/S
      int k = 0;
      for (int s = s1 - 1; s >= s0; --s)
        for (int q = 3; q >= 0; --q) {
          fra[k] = ((s1 - s) - 0.5 * (1.0 + kGLx[q])) / L;
          outa[k] = nodeA[(s - s0) * 4 + q];
          ++k;
        }
      fra[k] = 1.0;
      outa[k] = lam;
      const int rc_a = expmv_points(sector, zbar * (double(L) / S), lam, fra.data(), k + 1, outa.data());
      std::string err_f;
      const int rc_f = worker.wait(&err_f);
      if (rc_f != SYK_OK) {
        set_error("%s", err_f.c_str());
        return rc_f;
      }
      SYK_TRY(rc_a);
      SYK_CUDA_CHECK(cudaEventRecord(ev_fwd, st2));
      SYK_CUDA_CHECK(cudaStreamWaitEvent(st, ev_fwd, 0));
      for (int s = s1 - 1; s >= s0; --s)
        for (int q = 3; q >= 0; --q)
          SYK_TRY(term_grad(sector, nodeA[(s - s0) * 4 + q], nodeF[(s - s0) * 4 + q], z * (0.5 * kGLw[q] / S), gJ));
    }
    for (auto p : ckpt) put(p);
    for (auto p : nodeF) put(p);
    for (auto p : nodeA) put(p);
    return SYK_OK;
  }

  // Raw gradient of <left| chain psi>: gJ[T][b] += <left|d chain/dJ_T|psi>, gb[b] likewise.
  int chain_grad(const std::vector<Op>& ops, const void* psi, const void* left, double2* gJ, double2* gb) {
    std::vector<void*> xs;
    std::vector<int> sec;
    SYK_TRY(forward(ops, psi, xs, sec));
    void* lam = nullptr;
    SYK_TRY(get(&lam));
    SYK_TRY(copy(lam, left));
    for (int k = int(ops.size()) - 1; k >= 0; --k) {
      const Op& o = ops[k];
      if (o.kind == 1) {
        void* tmp = nullptr;
        SYK_TRY(get(&tmp));
        SYK_TRY(launch_apply_chi(terms->N, o.maj, sec[k + 1], dtype, lam, tmp, B, st));
        put(lam);
        lam = tmp;
      } else {
        SYK_TRY(exp_adjoint(o, sec[k], xs[k], xs[k + 1], lam, gJ, gb));
      }
    }
    put(lam);
    for (size_t k = 1; k < xs.size(); ++k) put(xs[k]);
    return SYK_OK;
  }

  // Value <a|b> (device, B entries) of two chains.
  int value(const std::vector<Op>& A, const std::vector<Op>& Bc, const void* psi, double2* out, void** a_out,
            void** b_out) {
    std::vector<void*> xa, xb;
    std::vector<int> sa, sb;
    SYK_TRY(forward(A, psi, xa, sa));
    SYK_TRY(forward(Bc, psi, xb, sb));
    SYK_TRY(dot_columns(xa.back(), xb.back(), D, B, dtype, ws, out, st));
    *a_out = xa.back();
    *b_out = xb.back();
    return SYK_OK;
  }

  // out_J[T][b] += coef[b] * d<a|b>/dJ_T, out_b[b] += coef[b] * d<a|b>/dbeta
  int form_grad(const std::vector<Op>& A, const std::vector<Op>& Bc, const void* psi, const void* a, const void* b,
                const double2* coef, double2* out_J, double2* out_b) {
    const size_t nJ = sizeof(double2) * size_t(terms->nterms) * B;
    void *gJa, *gJb, *gba, *gbb;
    SYK_TRY(alloc(&gJa, nJ));
    SYK_TRY(alloc(&gJb, nJ));
    SYK_TRY(alloc(&gba, sizeof(double2) * B));
    SYK_TRY(alloc(&gbb, sizeof(double2) * B));
    cudaMemsetAsync(gJa, 0, nJ, st);
    cudaMemsetAsync(gJb, 0, nJ, st);
    cudaMemsetAsync(gba, 0, sizeof(double2) * B, st);
    cudaMemsetAsync(gbb, 0, sizeof(double2) * B, st);
    SYK_TRY(chain_grad(Bc, psi, a, (double2*)gJb, (double2*)gbb));  // <a|db>
    SYK_TRY(chain_grad(A, psi, b, (double2*)gJa, (double2*)gba));   // <b|da> = conj(<da|b>)
    const int64_t n = terms->nterms * B;
    k_grad_combine<<<unsigned((n + 255) / 256), 256, 0, st>>>(terms->nterms, int(B), (double2*)gJb, (double2*)gJa,
                                                              coef, out_J);
    k_grad_combine<<<1, 256, 0, st>>>(1, int(B), (double2*)gbb, (double2*)gba, coef, out_b);
    count_launch(2);
    SYK_CUDA_CHECK(cudaGetLastError());
    return SYK_OK;
  }
};

std::vector<Op> otoc_A(int i) {
  return {{0, 1.0 / 8, 0, 0}, {0, 0, 1.0, 0}, {1, 0, 0, i}, {0, 0, -1.0, 0}, {0, 1.0 / 4, 0, 0}};
}
std::vector<Op> otoc_B(int i, int j) {
  return {{0, 1.0 / 8, 0, 0}, {1, 0, 0, j}, {0, 1.0 / 4, 0, 0}, {0, 0, 1.0, 0},
          {1, 0, 0, i},       {0, 0, -1.0, 0}, {0, 1.0 / 4, 0, 0}, {1, 0, 0, j}};
}

int grad_common_checks(const syk_terms* terms, double beta, double t, const void* psi0, int64_t ns, int dtype, int kd,
                       double tol, double dz) {
  if (!terms || !psi0) {
    set_error("NULL argument");
    return SYK_EINVAL;
  }
  if (!std::isfinite(beta) || beta < 0.0 || !std::isfinite(t) || t < 0.0) {
    set_error("beta and t must be finite and >= 0");
    return SYK_EINVAL;
  }
  if (ns < 1 || ns > 256 || kd < 2 || kd > SYK_MAX_KRYLOV || !dtype_ok(dtype) || !(tol > 0.0) || !(dz > 0.0)) {
    set_error("invalid sizes (nstates=%lld krylov_dim=%d dtype=%d tol=%g quad_dz=%g)", (long long)ns, kd, dtype, tol,
              dz);
    return SYK_EINVAL;
  }
  return SYK_OK;
}

int device_input_copy(GradEngine& E, const void* psi0, const void** out) {
  cudaPointerAttributes at;
  cudaError_t e = cudaPointerGetAttributes(&at, psi0);
  if (e != cudaSuccess) cudaGetLastError();
  if (e == cudaSuccess && (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged)) {
    *out = psi0;
    return SYK_OK;
  }
  void* d = nullptr;
  SYK_TRY(E.vec(&d));
  SYK_CUDA_CHECK(cudaMemcpyAsync(d, psi0, E.vb, cudaMemcpyHostToDevice, E.st));
  *out = d;
  return SYK_OK;
}

int finish_outputs(GradEngine& E, const double2* val, const double2* gJ, const double2* gb, double* v_re_im,
                   double* dJ, double* db) {
  const size_t B = size_t(E.B), nt = size_t(E.terms->nterms);
  std::vector<double2> hv(B), hb(B);
  SYK_CUDA_CHECK(cudaMemcpyAsync(hv.data(), val, sizeof(double2) * B, cudaMemcpyDeviceToHost, E.st));
  SYK_CUDA_CHECK(cudaMemcpyAsync(hb.data(), gb, sizeof(double2) * B, cudaMemcpyDeviceToHost, E.st));
  if (dJ) SYK_CUDA_CHECK(cudaMemcpyAsync(dJ, gJ, sizeof(double2) * nt * B, cudaMemcpyDeviceToHost, E.st));
  SYK_CUDA_CHECK(cudaStreamSynchronize(E.st));
  prof_collect();
  for (size_t b = 0; b < B; ++b) {
    if (v_re_im) {
      v_re_im[2 * b] = hv[b].x;
      v_re_im[2 * b + 1] = hv[b].y;
    }
    if (db) {
      db[2 * b] = hb[b].x;
      db[2 * b + 1] = hb[b].y;
    }
  }
  return SYK_OK;
}

}  // namespace
}  // namespace syk

using namespace syk;

extern "C" int syk_otoc_grad(const syk_terms* terms, double beta, int i, int j, double t, const void* psi0,
                             int64_t nstates, int dtype, int krylov_dim, double tol, double quad_dz,
                             double* Ft_re_im, double* dFt_dJ, double* dFt_dbeta, void* stream) {
  syk::NvtxRange nvtx_range_("syk_otoc_grad");
  clear_error();
  SYK_TRY(grad_common_checks(terms, beta, t, psi0, nstates, dtype, krylov_dim, tol, quad_dz));
  if (i < 0 || i >= terms->N || j < 0 || j >= terms->N || i == j) {
    set_error("syk_otoc_grad: need 0 <= i != j < N");
    return SYK_EINVAL;
  }
  GradEngine E;
  E.terms = terms;
  E.dtype = dtype;
  E.krylov = krylov_dim;
  E.B = nstates;
  E.beta = beta;
  E.tol = tol;
  E.dz = quad_dz;
  E.st = static_cast<cudaStream_t>(stream);
  SYK_TRY(E.init());
  const void* psi = nullptr;
  SYK_TRY(device_input_copy(E, psi0, &psi));
  const std::vector<Op> A = otoc_A(i), Bc = otoc_B(i, j);
  const size_t B = size_t(nstates);
  // values F(t) and F(0)
  void *vt, *v0, *a_t, *b_t, *a_0, *b_0;
  SYK_TRY(E.alloc(&vt, sizeof(double2) * B));
  SYK_TRY(E.alloc(&v0, sizeof(double2) * B));
  E.t = t;
  SYK_TRY(E.value(A, Bc, psi, (double2*)vt, &a_t, &b_t));
  E.t = 0.0;
  SYK_TRY(E.value(A, Bc, psi, (double2*)v0, &a_0, &b_0));
  std::vector<double2> ht(B), h0(B);
  SYK_CUDA_CHECK(cudaMemcpyAsync(ht.data(), vt, sizeof(double2) * B, cudaMemcpyDeviceToHost, E.st));
  SYK_CUDA_CHECK(cudaMemcpyAsync(h0.data(), v0, sizeof(double2) * B, cudaMemcpyDeviceToHost, E.st));
  SYK_CUDA_CHECK(cudaStreamSynchronize(E.st));
  // F~ = F_t / F_0;  dF~ = dF_t / F_0 - F~ dF_0 / F_0
  std::vector<double2> ctv(B), c0v(B), ft(B);
  for (size_t b = 0; b < B; ++b) {
    const std::complex<double> Ft(ht[b].x, ht[b].y), F0(h0[b].x, h0[b].y);
    if (std::abs(F0) == 0.0) {
      set_error("syk_otoc_grad: F(0) = 0 for state %zu", b);
      return SYK_ENUMERIC;
    }
    const std::complex<double> Ftil = Ft / F0, c1 = 1.0 / F0, c0 = -Ftil / F0;
    ft[b] = make_double2(Ftil.real(), Ftil.imag());
    ctv[b] = make_double2(c1.real(), c1.imag());
    c0v[b] = make_double2(c0.real(), c0.imag());
  }
  void *ct, *c0, *gJ, *gb, *ftd;
  const size_t nJ = sizeof(double2) * size_t(terms->nterms) * B;
  SYK_TRY(E.alloc(&ct, sizeof(double2) * B));
  SYK_TRY(E.alloc(&c0, sizeof(double2) * B));
  SYK_TRY(E.alloc(&ftd, sizeof(double2) * B));
  SYK_TRY(E.alloc(&gJ, nJ));
  SYK_TRY(E.alloc(&gb, sizeof(double2) * B));
  SYK_CUDA_CHECK(cudaMemcpyAsync(ct, ctv.data(), sizeof(double2) * B, cudaMemcpyHostToDevice, E.st));
  SYK_CUDA_CHECK(cudaMemcpyAsync(c0, c0v.data(), sizeof(double2) * B, cudaMemcpyHostToDevice, E.st));
  SYK_CUDA_CHECK(cudaMemcpyAsync(ftd, ft.data(), sizeof(double2) * B, cudaMemcpyHostToDevice, E.st));
  cudaMemsetAsync(gJ, 0, nJ, E.st);
  cudaMemsetAsync(gb, 0, sizeof(double2) * B, E.st);
  E.t = t;
  SYK_TRY(E.form_grad(A, Bc, psi, a_t, b_t, (double2*)ct, (double2*)gJ, (double2*)gb));
  E.t = 0.0;
  SYK_TRY(E.form_grad(A, Bc, psi, a_0, b_0, (double2*)c0, (double2*)gJ, (double2*)gb));
  return finish_outputs(E, (double2*)ftd, (double2*)gJ, (double2*)gb, Ft_re_im, dFt_dJ, dFt_dbeta);
}

extern "C" int syk_correlator_G_grad(const syk_terms* terms, double beta, int i, double t, const void* psi0,
                                     int64_t nstates, int dtype, int krylov_dim, double tol, double quad_dz,
                                     double* G_re_im, double* dG_dJ, double* dG_dbeta, void* stream) {
  syk::NvtxRange nvtx_range_("syk_correlator_G_grad");
  clear_error();
  SYK_TRY(grad_common_checks(terms, beta, t, psi0, nstates, dtype, krylov_dim, tol, quad_dz));
  if (i < 0 || i >= terms->N) {
    set_error("syk_correlator_G_grad: Majorana index out of range");
    return SYK_EINVAL;
  }
  GradEngine E;
  E.terms = terms;
  E.dtype = dtype;
  E.krylov = krylov_dim;
  E.B = nstates;
  E.beta = beta;
  E.t = t;
  E.tol = tol;
  E.dz = quad_dz;
  E.st = static_cast<cudaStream_t>(stream);
  SYK_TRY(E.init());
  const void* psi = nullptr;
  SYK_TRY(device_input_copy(E, psi0, &psi));
  const std::vector<Op> A = {{0, 0.5, 0, 0}, {0, 0, 1.0, 0}};
  const std::vector<Op> Bc = {{0, 0.5, 0, 0}, {1, 0, 0, i}, {0, 0, 1.0, 0}, {1, 0, 0, i}};
  const std::vector<Op> Zc = {{0, 0.5, 0, 0}};
  const size_t B = size_t(nstates);
  void *vn, *vz, *a, *b, *za, *zb;
  SYK_TRY(E.alloc(&vn, sizeof(double2) * B));
  SYK_TRY(E.alloc(&vz, sizeof(double2) * B));
  SYK_TRY(E.value(A, Bc, psi, (double2*)vn, &a, &b));
  SYK_TRY(E.value(Zc, Zc, psi, (double2*)vz, &za, &zb));
  std::vector<double2> hn(B), hz(B);
  SYK_CUDA_CHECK(cudaMemcpyAsync(hn.data(), vn, sizeof(double2) * B, cudaMemcpyDeviceToHost, E.st));
  SYK_CUDA_CHECK(cudaMemcpyAsync(hz.data(), vz, sizeof(double2) * B, cudaMemcpyDeviceToHost, E.st));
  SYK_CUDA_CHECK(cudaStreamSynchronize(E.st));
  // G = num / Z;  dG = dnum / Z - G dZ / Z
  std::vector<double2> cn(B), cz(B), gv(B);
  for (size_t k = 0; k < B; ++k) {
    const std::complex<double> num(hn[k].x, hn[k].y);
    const double Z = hz[k].x;
    if (!(Z > 0.0)) {
      set_error("syk_correlator_G_grad: Z <= 0 for state %zu", k);
      return SYK_ENUMERIC;
    }
    const std::complex<double> G = num / Z, c1 = 1.0 / Z, c0 = -G / Z;
    gv[k] = make_double2(G.real(), G.imag());
    cn[k] = make_double2(c1.real(), c1.imag());
    cz[k] = make_double2(c0.real(), c0.imag());
  }
  void *dcn, *dcz, *gJ, *gb, *gvd;
  const size_t nJ = sizeof(double2) * size_t(terms->nterms) * B;
  SYK_TRY(E.alloc(&dcn, sizeof(double2) * B));
  SYK_TRY(E.alloc(&dcz, sizeof(double2) * B));
  SYK_TRY(E.alloc(&gvd, sizeof(double2) * B));
  SYK_TRY(E.alloc(&gJ, nJ));
  SYK_TRY(E.alloc(&gb, sizeof(double2) * B));
  SYK_CUDA_CHECK(cudaMemcpyAsync(dcn, cn.data(), sizeof(double2) * B, cudaMemcpyHostToDevice, E.st));
  SYK_CUDA_CHECK(cudaMemcpyAsync(dcz, cz.data(), sizeof(double2) * B, cudaMemcpyHostToDevice, E.st));
  SYK_CUDA_CHECK(cudaMemcpyAsync(gvd, gv.data(), sizeof(double2) * B, cudaMemcpyHostToDevice, E.st));
  cudaMemsetAsync(gJ, 0, nJ, E.st);
  cudaMemsetAsync(gb, 0, sizeof(double2) * B, E.st);
  SYK_TRY(E.form_grad(A, Bc, psi, a, b, (double2*)dcn, (double2*)gJ, (double2*)gb));
  SYK_TRY(E.form_grad(Zc, Zc, psi, za, zb, (double2*)dcz, (double2*)gJ, (double2*)gb));
  return finish_outputs(E, (double2*)gvd, (double2*)gJ, (double2*)gb, G_re_im, dG_dJ, dG_dbeta);
}
