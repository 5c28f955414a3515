// Lowest eigenvalues of H in one parity sector, by Lanczos with full reorthogonalisation.
// The finite-size rescaling of the supplement (Sec. "Finite-size rescaling method") keeps the
// system sizes whose lowest 20 eigenstates lie within the thermal window of the ground state;
// this supplies those eigenvalues on the GPU with the same matvec as the dynamics.
//
// The Lanczos process (syk_krylov.cu: one column, two-pass classical Gram-Schmidt against the
// whole basis) runs on the device; every `kCheck` steps the tridiagonal projection T_j is
// diagonalised on the host in FP64 and the Ritz values theta_i with residual bounds
// beta_j |y_i(j)| (the last component of the Ritz vector times the last beta) are tested.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <numeric>
#include <vector>

#include "syk_krylov.cuh"

namespace syk {
namespace {

constexpr int kCheck = 16;  // Lanczos steps between Ritz-value checks

// Eigenvalues d of the symmetric tridiagonal T = tridiag(e, d, e) (d: m diagonal, e: m-1
// off-diagonal entries; both overwritten) by implicit QR with Wilkinson shifts (Golub & Van
// Loan, Sec. 8.3), accumulating only the last row of the rotation product Q (T = Q D Q^T):
// last[i] = Q[m-1][i], the last component of the i-th eigenvector.  Returns false if some
// eigenvalue fails to converge within 64 m sweeps.
bool tridiag_eig_lastrow(int m, std::vector<double>& d, std::vector<double>& e, std::vector<double>& last) {
  last.assign(m, 0.0);
  last[m - 1] = 1.0;
  const double eps = 2.220446049250313e-16;
  int q = m - 1, iter = 0;
  while (q > 0) {
    if (std::fabs(e[q - 1]) <= eps * (std::fabs(d[q - 1]) + std::fabs(d[q]))) {
      --q;
      continue;
    }
    if (++iter > 64 * m) return false;
    int l = q - 1;
    while (l > 0 && std::fabs(e[l - 1]) > eps * (std::fabs(d[l - 1]) + std::fabs(d[l]))) --l;
    // Wilkinson shift from the trailing 2x2 block of the unreduced part [l, q]
    const double dd = 0.5 * (d[q - 1] - d[q]), ee = e[q - 1];
    const double mu = d[q] - ee * ee / (dd + std::copysign(std::hypot(dd, ee), dd));
    double x = d[l] - mu, y = e[l];
    for (int k = l; k < q; ++k) {
      const double r = std::hypot(x, y);
      const double c = r > 0.0 ? x / r : 1.0, s = r > 0.0 ? y / r : 0.0;
      if (k > l) e[k - 1] = r;
      const double a = d[k], b = e[k], cc = d[k + 1];
      d[k] = c * c * a + 2.0 * c * s * b + s * s * cc;
      d[k + 1] = s * s * a - 2.0 * c * s * b + c * c * cc;
      e[k] = c * s * (cc - a) + (c * c - s * s) * b;
      if (k + 1 < q) {
        y = s * e[k + 1];
        e[k + 1] = c * e[k + 1];
        x = e[k];
      }
      const double qa = last[k], qb = last[k + 1];
      last[k] = c * qa + s * qb;
      last[k + 1] = -s * qa + c * qb;
    }
  }
  return true;
}

}  // namespace
}  // namespace syk

using namespace syk;

extern "C" int syk_lowest_eigenvalues(const syk_terms* terms, int parity, int dtype, const void* psi0, int k,
                                      int max_steps, double tol, double* evals, double* resid, int* nsteps,
                                      void* stream) {
  syk::NvtxRange nvtx_range_("syk_lowest_eigenvalues");
  clear_error();
  if (!terms || !psi0 || !evals || k < 1 || !(tol > 0.0) || !dtype_ok(dtype) || (parity != 0 && parity != 1)) {
    set_error("syk_lowest_eigenvalues: invalid argument (k=%d tol=%g dtype=%d parity=%d)", k, tol, dtype, parity);
    return SYK_EINVAL;
  }
  const int64_t D = terms->D;
  const int m = int(std::min<int64_t>(max_steps, D));
  if (k > m || max_steps > SYK_MAX_EIG_STEPS) {
    set_error("syk_lowest_eigenvalues: need k <= min(max_steps, sector dimension %lld) and max_steps <= %d "
              "(k=%d max_steps=%d)", (long long)D, SYK_MAX_EIG_STEPS, k, max_steps);
    return SYK_EINVAL;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  ApplyParams P;
  SYK_TRY(make_apply_params(terms, parity, dtype, &P));
  Scratch sc(st);
  const size_t vb = size_t(D) * dtype_size(dtype);
  const size_t wsb = krylov_ws_bytes(D, dtype, m, 1);
  void* wsp = nullptr;
  SYK_TRY(sc.alloc(&wsp, wsb));
  const void* psi = nullptr;
  SYK_TRY(device_input(psi0, vb, sc, &psi));
  KrylovWS ws;
  SYK_TRY(krylov_ws_carve(&ws, wsp, wsb, D, dtype, m, 1));
  SYK_TRY(lanczos_begin(dtype, psi, ws, st));
  std::vector<double> ha(m), hb(m), d, e, last;
  int hstat[4] = {0, 0, 0, 0};
  int j0 = 0, mm = 0;
  bool converged = false, invariant = false;
  while (j0 < m && !converged) {
    const int j1 = std::min(m, j0 + kCheck);
    SYK_TRY(lanczos_steps(P, dtype, ws, j0, j1, st));
    SYK_CUDA_CHECK(cudaMemcpyAsync(ha.data(), ws.alpha, sizeof(double) * j1, cudaMemcpyDeviceToHost, st));
    SYK_CUDA_CHECK(cudaMemcpyAsync(hb.data(), ws.beta, sizeof(double) * j1, cudaMemcpyDeviceToHost, st));
    SYK_CUDA_CHECK(cudaMemcpyAsync(hstat, ws.status, sizeof(int) * 2, cudaMemcpyDeviceToHost, st));
    SYK_CUDA_CHECK(cudaMemcpyAsync(hstat + 2, P.status, sizeof(int), cudaMemcpyDeviceToHost, st));
    SYK_CUDA_CHECK(cudaStreamSynchronize(st));
    if (hstat[0] & 1) {
      set_error("syk_lowest_eigenvalues: non-finite Lanczos scalar");
      return SYK_ENUMERIC;
    }
    if (hstat[2] & 4) {
      set_error("apply_H: a bounded wait for a staged tile gave up");
      return SYK_ETIMEOUT;
    }
    // a zero beta_j means the Krylov space is invariant: T_{j+1} holds exact eigenvalues
    mm = j1;
    for (int j = j0; j < j1; ++j)
      if (hb[j] == 0.0) {
        mm = j + 1;
        invariant = true;
        break;
      }
    d.assign(ha.begin(), ha.begin() + mm);
    e.assign(hb.begin(), hb.begin() + mm);  // e[mm-1] (the last beta) is unused by the solver
    if (!tridiag_eig_lastrow(mm, d, e, last)) {
      set_error("syk_lowest_eigenvalues: tridiagonal eigensolver did not converge");
      return SYK_ENUMERIC;
    }
    const double beta_last = invariant ? 0.0 : hb[mm - 1];
    std::vector<int> ord(mm);
    std::iota(ord.begin(), ord.end(), 0);
    std::sort(ord.begin(), ord.end(), [&](int a, int b) { return d[a] < d[b]; });
    double scale = 0.0;
    for (int i = 0; i < mm; ++i) scale = std::max(scale, std::fabs(d[i]));
    scale = std::max(1.0, scale);
    // distinct levels: rounding eventually lets one start vector find both members of a
    // degenerate pair, whose Ritz values then agree far below the merge gap
    const double gap = 10.0 * tol * scale;
    int kk = 0;
    converged = true;
    for (int i = 0; i < mm && kk < k; ++i) {
      const double th = d[ord[i]];
      if (kk > 0 && th - evals[kk - 1] <= gap) continue;
      evals[kk] = th;
      const double r = beta_last * std::fabs(last[ord[i]]);
      if (resid) resid[kk] = r;
      if (!(r <= tol * scale)) converged = false;
      ++kk;
    }
    if (kk < k) converged = false;
    if (invariant) break;
    j0 = j1;
  }
  if (nsteps) *nsteps = mm;
  if (!converged && invariant) {
    set_error("syk_lowest_eigenvalues: the Krylov space of the start vector holds fewer than k = %d distinct levels "
              "(dimension %d)", k, mm);
    return SYK_ENUMERIC;
  }
  if (!converged) {
    set_error("syk_lowest_eigenvalues: %d lowest Ritz values not converged to tol %g in %d steps", k, tol, mm);
    return SYK_ENUMERIC;
  }
  return SYK_OK;
}
