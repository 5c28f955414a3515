// FP64 device routines on the Krylov projection T (Supp. Sec. I.B): eigendecomposition of the
// symmetric tridiagonal matrix, the exponential of its eigenvalues and Saad's a-posteriori
// error estimate of a step, shared by the Krylov driver (syk_krylov.cu) and the persistent
// batched kernel (syk_batch.cu).
#pragma once
#include <cuda_runtime.h>

namespace syk {

// ---------------------------------------------------------------- tridiagonal
// Implicit symmetric QR with Wilkinson shift (Golub & Van Loan, Sec. 8.3) on
// T = tridiag(beta, alpha, beta) of dimension m, one warp per matrix.  Lane 0
// computes every Givens rotation (the scalar recurrence), all lanes apply it
// to their rows of the accumulated eigenvector matrix Q (row-major m x m in
// shared memory).  On return d holds the eigenvalues and T = Q diag(d) Q^T.
// Givens rotation (c, s) with c x + s y = r, -s x + c y = 0; r^2 = x^2 + y^2 (the entries of
// T are O(1) to O(10^2), so the squares neither overflow nor underflow) and one reciprocal
// square root instead of a hypot and two divisions: the chain of dependent FP64 operations
// of the bulge chase is the eigensolver's latency.
__device__ __forceinline__ void givens(double x, double y, double& c, double& s, double& r) {
  const double r2 = fma(x, x, y * y);
  if (r2 > 0.0) {
    const double ri = rsqrt(r2);
    c = x * ri;
    s = y * ri;
    r = r2 * ri;
  } else {
    c = 1.0;
    s = 0.0;
    r = 0.0;
  }
}

static __device__ bool tridiag_eig_warp(int m, double* d, double* e, double* Q, double* rot) {
  const int lane = threadIdx.x & 31;
  for (int r = lane; r < m; r += 32)
    for (int c = 0; c < m; ++c) Q[r * m + c] = (r == c) ? 1.0 : 0.0;
  __syncwarp();
  const double eps = 2.220446049250313e-16;
  int q = m - 1;
  int iter = 0;
  bool ok = true;
  while (q > 0) {
    if (fabs(e[q - 1]) <= eps * (fabs(d[q - 1]) + fabs(d[q]))) {
      --q;
      continue;
    }
    if (++iter > 64 * m) {
      ok = false;
      break;
    }
    int l = q - 1;
    while (l > 0 && fabs(e[l - 1]) > eps * (fabs(d[l - 1]) + fabs(d[l]))) --l;
    double x = 0.0, y = 0.0;
    if (lane == 0) {
      const double dd = 0.5 * (d[q - 1] - d[q]);
      const double ee = e[q - 1];
      const double mu = d[q] - ee * ee / (dd + copysign(hypot(dd, ee), dd));
      x = d[l] - mu;
      y = e[l];
    }
    for (int k = l; k < q; ++k) {
      if (lane == 0) {
        double c, s, r;
        givens(x, y, c, s, r);
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
        rot[0] = c;
        rot[1] = s;
      }
      __syncwarp();
      const double c = rot[0], s = rot[1];
      for (int r = lane; r < m; r += 32) {
        const double qa = Q[r * m + k], qb = Q[r * m + k + 1];
        Q[r * m + k] = c * qa + s * qb;
        Q[r * m + k + 1] = -s * qa + c * qb;
      }
      __syncwarp();
    }
  }
  __syncwarp();
  return ok;
}

// The same implicit QR, run by the calling thread alone, accumulating only rows 0 and m-1 of
// Q (q0, qm): all the convergence check's error estimate needs, with no warp synchronisation
// per rotation.  Same rotations as tridiag_eig_warp, so d ends up with the same eigenvalues.
static __device__ bool tridiag_eig_rows(int m, double* d, double* e, double* q0, double* qm) {
  for (int c = 0; c < m; ++c) {
    q0[c] = c == 0 ? 1.0 : 0.0;
    qm[c] = c == m - 1 ? 1.0 : 0.0;
  }
  const double eps = 2.220446049250313e-16;
  int q = m - 1;
  int iter = 0;
  while (q > 0) {
    if (fabs(e[q - 1]) <= eps * (fabs(d[q - 1]) + fabs(d[q]))) {
      --q;
      continue;
    }
    if (++iter > 64 * m) return false;
    int l = q - 1;
    while (l > 0 && fabs(e[l - 1]) > eps * (fabs(d[l - 1]) + fabs(d[l]))) --l;
    const double dd = 0.5 * (d[q - 1] - d[q]);
    const double ee = e[q - 1];
    const double mu = d[q] - ee * ee / (dd + copysign(hypot(dd, ee), dd));
    double x = d[l] - mu, y = e[l];
    for (int k = l; k < q; ++k) {
      double c, s, r;
      givens(x, y, c, s, r);
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
      const double a0 = q0[k], b0 = q0[k + 1], am = qm[k], bm = qm[k + 1];
      q0[k] = c * a0 + s * b0;
      q0[k + 1] = -s * a0 + c * b0;
      qm[k] = c * am + s * bm;
      qm[k + 1] = -s * am + c * bm;
    }
  }
  return true;
}

__device__ __forceinline__ double2 cexp_scaled(double s, double zr, double zi, double th) {
  const double mag = exp(s * zr * th);
  double sn, cs;
  sincos(s * zi * th, &sn, &cs);
  return make_double2(mag * cs, mag * sn);
}

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Saad's estimate of the relative error of the step s: beta_last |e_m^T e^{szT} e_1| / ||e^{szT} e_1||
// (q0, qm: rows 0 and m-1 of the eigenvector matrix)
static __device__ double step_error(int m, const double* d, const double* q0, const double* qm, double beta_last, double s,
                             double zr, double zi) {
  if (beta_last == 0.0) return 0.0;
  const int lane = threadIdx.x & 31;
  double nr = 0.0, ni = 0.0, den = 0.0;
  for (int k = lane; k < m; k += 32) {
    const double2 f = cexp_scaled(s, zr, zi, d[k]);
    const double g = q0[k], h = qm[k];
    nr += h * g * f.x;
    ni += h * g * f.y;
    den += (f.x * f.x + f.y * f.y) * g * g;
  }
  nr = warp_sum(nr);
  ni = warp_sum(ni);
  den = warp_sum(den);
  if (!(den > 0.0)) return 0.0;
  return beta_last * sqrt(nr * nr + ni * ni) / sqrt(den);
}

// The largest step s <= s_target whose estimate step_error is <= tol: halve s until the
// estimate passes (at most 80 times), then bisect nbis times between the last failing and the
// first passing step.  Every lane of the warp calls it (step_error sums over the lanes).
static __device__ double select_step(int m, const double* d, const double* q0, const double* qm, double bl,
                                     double s_target, double tol, double zr, double zi, int nbis = 24) {
  double s = s_target;
  if (step_error(m, d, q0, qm, bl, s, zr, zi) > tol) {
    double lo = 0.0, hi = s;
    s *= 0.5;
    int it = 0;
    while (step_error(m, d, q0, qm, bl, s, zr, zi) > tol && it < 80) {
      hi = s;
      s *= 0.5;
      ++it;
    }
    lo = s;
    for (int k = 0; k < nbis; ++k) {  // largest admissible step within [lo, hi)
      const double mid = 0.5 * (lo + hi);
      if (step_error(m, d, q0, qm, bl, mid, zr, zi) <= tol) lo = mid;
      else hi = mid;
    }
    s = lo;
  }
  return s;
}

}  // namespace syk
