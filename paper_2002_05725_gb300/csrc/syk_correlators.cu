// Correlators by random-state typicality (Eq. q_typicality):
//   G(t)  (Eq. G)      real-time two-point function,
//   F(t)  (Eq. F_reg)  regularized OTOC with rho^{1/4} between the operators.
// Each is a host-driven chain of expmv, chi and dot calls on the device; the
// batch dimension carries the random states of one coupling draw.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <complex>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "syk_krylov.cuh"

namespace syk {
namespace {

int check_common(const syk_terms* t, double beta, const double* times, int nt, const void* psi0, int64_t ns,
                 int dtype, int kd, double tol, const void* out) {
  if (!t || !times || !psi0 || !out) {
    set_error("NULL argument");
    return SYK_EINVAL;
  }
  if (!std::isfinite(beta) || beta < 0.0) {
    set_error("beta must be finite and >= 0");
    return SYK_EINVAL;
  }
  if (nt < 1 || ns < 1 || ns > 256 || kd < 2 || kd > SYK_MAX_KRYLOV || !dtype_ok(dtype) || !(tol > 0.0)) {
    set_error("invalid sizes (nt=%d nstates=%lld krylov_dim=%d dtype=%d tol=%g)", nt, (long long)ns, kd, dtype, tol);
    return SYK_EINVAL;
  }
  double prev = 0.0;
  for (int k = 0; k < nt; ++k) {
    if (!std::isfinite(times[k]) || times[k] < prev) {
      set_error("times must be finite, >= 0 and non-decreasing");
      return SYK_EINVAL;
    }
    prev = times[k];
  }
  return SYK_OK;
}

}  // namespace
}  // namespace syk

using namespace syk;

extern "C" int syk_correlator_G(const syk_terms* terms, double beta, int i, const double* t, int nt, const void* psi0,
                                int64_t nstates, int dtype, int krylov_dim, double tol, double* G_re_im, double* Z,
                                void* stream) {
  syk::NvtxRange nvtx_range_("syk_correlator_G");
  clear_error();
  SYK_TRY(check_common(terms, beta, t, nt, psi0, nstates, dtype, krylov_dim, tol, G_re_im));
  if (i < 0 || i >= terms->N) {
    set_error("syk_correlator_G: Majorana index %d out of range", i);
    return SYK_EINVAL;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int64_t B = nstates;
  ApplyParams P0, P1;
  SYK_TRY(make_apply_params(terms, 0, dtype, &P0));
  SYK_TRY(make_apply_params(terms, 1, dtype, &P1));
  Scratch sc(st);
  const size_t vb = size_t(terms->D) * B * dtype_size(dtype);
  const size_t wsb = krylov_ws_bytes(terms->D, dtype, krylov_dim, B);
  void *wsp, *a, *b, *tmp, *res;
  SYK_TRY(sc.alloc(&wsp, wsb));
  SYK_TRY(sc.alloc(&a, vb));
  SYK_TRY(sc.alloc(&b, vb));
  SYK_TRY(sc.alloc(&tmp, vb));
  SYK_TRY(sc.alloc(&res, sizeof(double2) * B * (nt + 1)));
  const void* psi = nullptr;
  SYK_TRY(device_input(psi0, vb, sc, &psi));
  KrylovWS ws;
  SYK_TRY(krylov_ws_carve(&ws, wsp, wsb, terms->D, dtype, krylov_dim, B));
  SYK_TRY(chain_begin(ws, st));
  double2* r = static_cast<double2*>(res);
  // phi = e^{-beta H/2} psi~ (even sector), Z = <phi|phi>
  SYK_TRY(expmv_chain(P0, dtype, {-0.5 * beta, 0.0}, psi, a, B, tol, ws, st));
  SYK_TRY(dot_columns(a, a, terms->D, B, dtype, ws, r + size_t(nt) * B, st));
  SYK_TRY(launch_apply_chi(terms->N, i, 0, dtype, a, b, B, st));  // b = chi_i phi (odd)
  double tcur = 0.0;
  for (int k = 0; k < nt; ++k) {
    const double dt = t[k] - tcur;
    if (dt > 0.0) {
      SYK_TRY(expmv_chain(P0, dtype, {0.0, -dt}, a, a, B, tol, ws, st));
      SYK_TRY(expmv_chain(P1, dtype, {0.0, -dt}, b, b, B, tol, ws, st));
      tcur = t[k];
    }
    SYK_TRY(launch_apply_chi(terms->N, i, 1, dtype, b, tmp, B, st));  // chi_i U chi_i phi (even)
    SYK_TRY(dot_columns(a, tmp, terms->D, B, dtype, ws, r + size_t(k) * B, st));
  }
  std::vector<double2> h(size_t(nt + 1) * B);
  SYK_CUDA_CHECK(cudaMemcpyAsync(h.data(), r, sizeof(double2) * h.size(), cudaMemcpyDeviceToHost, st));
  SYK_TRY(chain_end(ws, st));  // synchronises st; device-side errors of the evolutions
  prof_collect();
  for (int64_t s = 0; s < B; ++s) {
    const double z = h[size_t(nt) * B + s].x;
    if (Z) Z[s] = z;
    for (int k = 0; k < nt; ++k) {
      const double2 v = h[size_t(k) * B + s];
      G_re_im[(size_t(k) * B + s) * 2] = z > 0 ? v.x / z : NAN;
      G_re_im[(size_t(k) * B + s) * 2 + 1] = z > 0 ? v.y / z : NAN;
    }
  }
  return SYK_OK;
}

namespace syk {
// OTOC of one coupling draw on stream st (arguments already validated), with rho split as
// Tr[W(t) rho^{x1} V rho^{x2} W(t) rho^{x3} V rho^{x4}] (x = 1/4 each: Eq. F_reg):
//   phi = rho^{x4/2} psi~, a0 = rho^{x3} chi_j phi, p = chi_i U(t) phi, q = chi_i U(t) a0,
//   F = < rho^{x1} U(t)^dag p | chi_j | rho^{x2} U(t)^dag q >.
int otoc_impl(const syk_terms* terms, double beta, const double* x, int i, int j, const double* t, int nt,
              const void* psi0, int64_t nstates, int dtype, int krylov_dim, double tol, double* F_re_im,
              cudaStream_t st) {
  const int64_t B = nstates;
  ApplyParams P0, P1;
  SYK_TRY(make_apply_params(terms, 0, dtype, &P0));
  SYK_TRY(make_apply_params(terms, 1, dtype, &P1));
  Scratch sc(st);
  const size_t vb = size_t(terms->D) * B * dtype_size(dtype);
  const size_t wsb = krylov_ws_bytes(terms->D, dtype, krylov_dim, B);
  void *wsp, *ua, *ub, *pr, *qs, *tmp, *res;
  SYK_TRY(sc.alloc(&wsp, wsb));
  SYK_TRY(sc.alloc(&ua, vb));
  SYK_TRY(sc.alloc(&ub, vb));
  SYK_TRY(sc.alloc(&pr, vb));
  SYK_TRY(sc.alloc(&qs, vb));
  SYK_TRY(sc.alloc(&tmp, vb));
  SYK_TRY(sc.alloc(&res, sizeof(double2) * B * nt));
  const void* psi = nullptr;
  SYK_TRY(device_input(psi0, vb, sc, &psi));
  KrylovWS ws;
  SYK_TRY(krylov_ws_carve(&ws, wsp, wsb, terms->D, dtype, krylov_dim, B));
  SYK_TRY(chain_begin(ws, st));
  double2* r = static_cast<double2*>(res);
  // ua = phi = rho^{x4/2} psi~ (even); ub = a0 = rho^{x3} chi_j phi (odd)
  SYK_TRY(expmv_chain(P0, dtype, {-beta * x[3] / 2.0, 0.0}, psi, ua, B, tol, ws, st));
  SYK_TRY(launch_apply_chi(terms->N, j, 0, dtype, ua, tmp, B, st));
  SYK_TRY(expmv_chain(P1, dtype, {-beta * x[2], 0.0}, tmp, ub, B, tol, ws, st));
  double tcur = 0.0;
  for (int k = 0; k < nt; ++k) {
    const double tk = t[k], dt = tk - tcur;
    if (dt > 0.0) {
      SYK_TRY(expmv_chain(P0, dtype, {0.0, -dt}, ua, ua, B, tol, ws, st));  // U(t) phi
      SYK_TRY(expmv_chain(P1, dtype, {0.0, -dt}, ub, ub, B, tol, ws, st));  // U(t) a0
      tcur = tk;
    }
    SYK_TRY(launch_apply_chi(terms->N, i, 0, dtype, ua, pr, B, st));  // p (odd)
    SYK_TRY(launch_apply_chi(terms->N, i, 1, dtype, ub, qs, B, st));  // q (even)
    // r = rho^{x1} U^dag p and s = rho^{x2} U^dag q: the exponentials commute, so each is one
    // Krylov evolution with z = -beta x + i t
    SYK_TRY(expmv_chain(P1, dtype, {-beta * x[0], tk}, pr, pr, B, tol, ws, st));  // r (odd)
    SYK_TRY(expmv_chain(P0, dtype, {-beta * x[1], tk}, qs, qs, B, tol, ws, st));  // s (even)
    SYK_TRY(launch_apply_chi(terms->N, j, 0, dtype, qs, tmp, B, st));     // chi_j s (odd)
    SYK_TRY(dot_columns(pr, tmp, terms->D, B, dtype, ws, r + size_t(k) * B, st));
  }
  std::vector<double2> h(size_t(nt) * B);
  SYK_CUDA_CHECK(cudaMemcpyAsync(h.data(), r, sizeof(double2) * h.size(), cudaMemcpyDeviceToHost, st));
  SYK_TRY(chain_end(ws, st));  // synchronises st; device-side errors of the evolutions
  prof_collect();
  for (size_t e = 0; e < h.size(); ++e) {
    F_re_im[2 * e] = h[e].x;
    F_re_im[2 * e + 1] = h[e].y;
  }
  return SYK_OK;
}
}  // namespace syk

extern "C" int syk_otoc(const syk_terms* terms, double beta, int i, int j, const double* t, int nt, const void* psi0,
                        int64_t nstates, int dtype, int krylov_dim, double tol, double* F_re_im, void* stream) {
  syk::NvtxRange nvtx_range_("syk_otoc");
  clear_error();
  SYK_TRY(check_common(terms, beta, t, nt, psi0, nstates, dtype, krylov_dim, tol, F_re_im));
  if (i < 0 || i >= terms->N || j < 0 || j >= terms->N || i == j) {
    set_error("syk_otoc: need 0 <= i != j < N (i=%d j=%d)", i, j);
    return SYK_EINVAL;
  }
  static const double quarter[4] = {0.25, 0.25, 0.25, 0.25};
  return otoc_impl(terms, beta, quarter, i, j, t, nt, psi0, nstates, dtype, krylov_dim, tol, F_re_im,
                   static_cast<cudaStream_t>(stream));
}

extern "C" int syk_otoc_split(const syk_terms* terms, double beta, const double* x, int i, int j, const double* t,
                              int nt, const void* psi0, int64_t nstates, int dtype, int krylov_dim, double tol,
                              double* F_re_im, void* stream) {
  syk::NvtxRange nvtx_range_("syk_otoc_split");
  clear_error();
  SYK_TRY(check_common(terms, beta, t, nt, psi0, nstates, dtype, krylov_dim, tol, F_re_im));
  if (i < 0 || i >= terms->N || j < 0 || j >= terms->N || i == j) {
    set_error("syk_otoc_split: need 0 <= i != j < N (i=%d j=%d)", i, j);
    return SYK_EINVAL;
  }
  if (!x) {
    set_error("syk_otoc_split: NULL split");
    return SYK_EINVAL;
  }
  double sum = 0.0;
  for (int k = 0; k < 4; ++k) {
    if (!(x[k] >= 0.0) || !std::isfinite(x[k])) {
      set_error("syk_otoc_split: split fractions must be finite and >= 0");
      return SYK_EINVAL;
    }
    sum += x[k];
  }
  if (std::abs(sum - 1.0) > 1e-12) {
    set_error("syk_otoc_split: split fractions must sum to 1 (got %.17g)", sum);
    return SYK_EINVAL;
  }
  return otoc_impl(terms, beta, x, i, j, t, nt, psi0, nstates, dtype, krylov_dim, tol, F_re_im,
                   static_cast<cudaStream_t>(stream));
}

extern "C" int syk_correlator_G_imag(const syk_terms* terms, double beta, int i, const double* tau, int ntau,
                                     const void* psi0, int64_t nstates, int dtype, int krylov_dim, double tol,
                                     double* G_re_im, double* Z, void* stream) {
  syk::NvtxRange nvtx_range_("syk_correlator_G_imag");
  clear_error();
  SYK_TRY(check_common(terms, beta, tau, ntau, psi0, nstates, dtype, krylov_dim, tol, G_re_im));
  if (i < 0 || i >= terms->N) {
    set_error("syk_correlator_G_imag: Majorana index %d out of range", i);
    return SYK_EINVAL;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int64_t B = nstates;
  ApplyParams P0, P1;
  SYK_TRY(make_apply_params(terms, 0, dtype, &P0));
  SYK_TRY(make_apply_params(terms, 1, dtype, &P1));
  Scratch sc(st);
  const size_t vb = size_t(terms->D) * B * dtype_size(dtype);
  const size_t wsb = krylov_ws_bytes(terms->D, dtype, krylov_dim, B);
  void *wsp, *x, *w, *y, *tmp, *res;
  SYK_TRY(sc.alloc(&wsp, wsb));
  SYK_TRY(sc.alloc(&x, vb));
  SYK_TRY(sc.alloc(&w, vb));
  SYK_TRY(sc.alloc(&y, vb));
  SYK_TRY(sc.alloc(&tmp, vb));
  SYK_TRY(sc.alloc(&res, sizeof(double2) * B * (ntau + 1)));
  const void* psi = nullptr;
  SYK_TRY(device_input(psi0, vb, sc, &psi));
  KrylovWS ws;
  SYK_TRY(krylov_ws_carve(&ws, wsp, wsb, terms->D, dtype, krylov_dim, B));
  SYK_TRY(chain_begin(ws, st));
  double2* r = static_cast<double2*>(res);
  // x = e^{-beta H/2} psi~ (even), Z = <x|x>; w(tau) = e^{tau H} x (even), y(tau) = e^{-tau H} chi_i x (odd)
  SYK_TRY(expmv_chain(P0, dtype, {-0.5 * beta, 0.0}, psi, x, B, tol, ws, st));
  SYK_TRY(dot_columns(x, x, terms->D, B, dtype, ws, r + size_t(ntau) * B, st));
  SYK_CUDA_CHECK(cudaMemcpyAsync(w, x, vb, cudaMemcpyDeviceToDevice, st));
  SYK_TRY(launch_apply_chi(terms->N, i, 0, dtype, x, y, B, st));
  double tcur = 0.0;
  for (int k = 0; k < ntau; ++k) {
    const double dt = tau[k] - tcur;
    if (dt > 0.0) {
      SYK_TRY(expmv_chain(P0, dtype, {dt, 0.0}, w, w, B, tol, ws, st));
      SYK_TRY(expmv_chain(P1, dtype, {-dt, 0.0}, y, y, B, tol, ws, st));
      tcur = tau[k];
    }
    SYK_TRY(launch_apply_chi(terms->N, i, 1, dtype, y, tmp, B, st));  // chi_i e^{-tau H} chi_i x (even)
    SYK_TRY(dot_columns(w, tmp, terms->D, B, dtype, ws, r + size_t(k) * B, st));
  }
  std::vector<double2> h(size_t(ntau + 1) * B);
  SYK_CUDA_CHECK(cudaMemcpyAsync(h.data(), r, sizeof(double2) * h.size(), cudaMemcpyDeviceToHost, st));
  SYK_TRY(chain_end(ws, st));  // synchronises st; device-side errors of the evolutions
  prof_collect();
  for (int64_t s2 = 0; s2 < B; ++s2) {
    const double z = h[size_t(ntau) * B + s2].x;
    if (Z) Z[s2] = z;
    for (int k = 0; k < ntau; ++k) {
      const double2 v = h[size_t(k) * B + s2];
      G_re_im[(size_t(k) * B + s2) * 2] = z > 0 ? v.x / z : NAN;
      G_re_im[(size_t(k) * B + s2) * 2 + 1] = z > 0 ? v.y / z : NAN;
    }
  }
  return SYK_OK;
}

// ---------------------------------------------------------------- batched workload
// Items whose whole chain fits one CTA run as one persistent launch (syk_batch.cu), driven by
// one host thread on its own stream.  The other independent work items (coupling draws of any
// N, with their beta and states) are taken, largest first, from a shared counter by `nworkers`
// host threads, each driving its own non-blocking CUDA stream, so items of small sectors run
// concurrently and fill the GPU together.  Each distinct (N, dtype, batch) of those is
// autotuned first on the calling thread.
extern "C" int syk_otoc_batch(const syk_otoc_item* items, int nitems, int i, int j, const double* t, int nt,
                              int dtype, int krylov_dim, double tol, int nworkers, int* item_status) {
  syk::NvtxRange nvtx_range_("syk_otoc_batch");
  clear_error();
  if (!items || nitems < 1 || nworkers < 1) {
    set_error("syk_otoc_batch: need items, nitems >= 1 and nworkers >= 1");
    return SYK_EINVAL;
  }
  for (int k = 0; k < nitems; ++k) {
    const syk_otoc_item& it = items[k];
    SYK_TRY(check_common(it.terms, it.beta, t, nt, it.psi0, it.nstates, dtype, krylov_dim, tol, it.F_re_im));
    if (i < 0 || i >= it.terms->N || j < 0 || j >= it.terms->N || i == j) {
      set_error("syk_otoc_batch: item %d: need 0 <= i != j < N", k);
      return SYK_EINVAL;
    }
  }
  int dev = 0;
  SYK_CUDA_CHECK(cudaGetDevice(&dev));
  // items for the persistent launch, by batch size (1, 2, 4, 8, 16); the rest go to the workers
  std::vector<char> persistent(nitems, 0);
  std::vector<std::vector<int>> pgroups(5);
  // Items whose states must be split over several CTAs (sector vectors too large for one CTA
  // at their full state count) run 2 states per CTA, where a CTA's matvec is several times
  // slower per state than the per-item path's full-GPU kernels; they pay off when their
  // sub-items fill at least half the GPU, otherwise they stay on the streams.
  std::vector<int> bsv(nitems, 0);
  long long split_subitems = 0;
  for (int k = 0; k < nitems; ++k) {
    bsv[k] = batch_item_persistent_states(items[k].terms, items[k].nstates, items[k].psi0, dtype, krylov_dim);
    if (bsv[k] > 0 && bsv[k] < items[k].nstates) split_subitems += items[k].nstates / bsv[k];
  }
  const bool take_split = 2 * split_subitems >= sm_count() || batch_persistent_split_always();
  for (int k = 0; k < nitems; ++k) {
    const int bs = bsv[k];
    if (bs > 0 && (bs == items[k].nstates || take_split)) {
      persistent[k] = 1;
      int g = 0;
      while ((1 << g) < bs) ++g;
      pgroups[g].push_back(k);
    }
  }
  long long report[kBatchReportWords] = {};
  // tune the matvec shape of every distinct (N, batch) once
  {
    std::vector<std::pair<int, int64_t>> done;
    for (int k = 0; k < nitems; ++k) {
      if (persistent[k]) continue;
      const auto key = std::make_pair(items[k].terms->N, items[k].nstates);
      if (std::find(done.begin(), done.end(), key) != done.end()) continue;
      done.push_back(key);
      const int64_t b = items[k].nstates;
      if ((b == 1 || b == 2 || b == 4 || b == 8 || b == 16) && items[k].terms->D >= 4096)
        SYK_TRY(syk_autotune_apply(items[k].terms, 0, dtype, b, 2, nullptr, nullptr));
    }
  }
  // largest items first (state size x states), so the long ones do not form the tail
  std::vector<int> order;
  for (int k = 0; k < nitems; ++k)
    if (!persistent[k]) order.push_back(k);
  const int nrest = (int)order.size();
  report[1] = nrest;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    return double(items[a].terms->D) * items[a].nstates > double(items[b].terms->D) * items[b].nstates;
  });
  std::atomic<int> next{0};
  std::mutex err_mtx;
  int first_rc = SYK_OK;
  std::string first_msg;
  // the persistent launch(es), one per batch size, on their own stream and host thread
  auto persistent_driver = [&]() {
    cudaSetDevice(dev);
    cudaStream_t st = nullptr;
    int rc = SYK_OK;
    std::string msg;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
      rc = SYK_ECUDA;
      msg = "cannot create a stream";
    }
    // statuses start at a positive "not run" mark; a launch that returns them overwrites it
    if (item_status)
      for (int g = 0; g < 5; ++g)
        for (int k : pgroups[g]) item_status[k] = 1;
    for (int g = 0; g < 5 && rc == SYK_OK; ++g) {
      if (pgroups[g].empty()) continue;
      NvtxRange range("syk_otoc_batch persistent launch");
      rc = otoc_batch_persistent(items, pgroups[g], int64_t(1) << g, i, j, t, nt, krylov_dim, tol, item_status, st,
                                 report);
      if (rc != SYK_OK) msg = syk_last_error();
    }
    if (rc != SYK_OK && item_status)
      for (int g = 0; g < 5; ++g)
        for (int k : pgroups[g])
          if (item_status[k] == 1) item_status[k] = rc;
    if (st) {
      cudaStreamSynchronize(st);
      cudaStreamDestroy(st);
    }
    if (rc != SYK_OK) {
      std::lock_guard<std::mutex> lk(err_mtx);
      if (first_rc == SYK_OK) {
        first_rc = rc;
        first_msg = "persistent launch: " + msg;
      }
    }
  };
  auto worker = [&]() {
    cudaSetDevice(dev);
    cudaStream_t st = nullptr;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
      std::lock_guard<std::mutex> lk(err_mtx);
      if (first_rc == SYK_OK) {
        first_rc = SYK_ECUDA;
        first_msg = "syk_otoc_batch: cannot create a stream";
      }
      return;
    }
    for (int q = next++; q < nrest; q = next++) {
      const int k = order[q];
      const syk_otoc_item& it = items[k];
      NvtxRange item_range("syk_otoc_batch item");
      static const double quarter[4] = {0.25, 0.25, 0.25, 0.25};
      const int rc = otoc_impl(it.terms, it.beta, quarter, i, j, t, nt, it.psi0, it.nstates, dtype, krylov_dim,
                               tol, it.F_re_im, st);
      if (item_status) item_status[k] = rc;
      if (rc != SYK_OK) {
        std::lock_guard<std::mutex> lk(err_mtx);
        if (first_rc == SYK_OK) {
          first_rc = rc;
          first_msg = std::string("item ") + std::to_string(k) + ": " + syk_last_error();
        }
      }
    }
    cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
  };
  std::vector<std::thread> pool;
  const bool any_persistent = nrest < nitems;
  if (any_persistent) pool.emplace_back(persistent_driver);
  const int nw = std::min(nworkers, nrest);
  for (int w = 0; w < nw; ++w) pool.emplace_back(worker);
  for (auto& th : pool) th.join();
  batch_report_store(report);
  if (first_rc != SYK_OK) set_error("syk_otoc_batch: %s", first_msg.c_str());
  return first_rc;
}
