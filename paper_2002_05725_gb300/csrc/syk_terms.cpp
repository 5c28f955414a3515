// Host side of the SYK term set: Jordan-Wigner Pauli strings of every term of
// Eq. 1, grouped by X-mask into the coefficient tables the matvec evaluates.
//
// Pauli algebra (Supp. Sec. I.A).  A Pauli string is i^p X^m Z^z with
// X^m Z^z |x> = (-1)^popcount(z & x) |x ^ m>.  Majorana a on spin k = a/2:
//   even a: (prod_{j<k} Z_j) X_k    -> m = 1<<k, z = (1<<k)-1,            p = 0
//   odd a:  (prod_{j<k} Z_j) Y_k    -> m = 1<<k, z = ((1<<k)-1) | (1<<k), p = 1
// (Y = i X Z), each times 1/sqrt(2).  The product of two strings is
//   (i^p1 X^m1 Z^z1)(i^p2 X^m2 Z^z2) = i^(p1+p2+2 popcount(z1&m2)) X^(m1^m2) Z^(z1^z2).
// So chi_i chi_j chi_k chi_l = (1/4) i^p X^m Z^z, and term T contributes
// w_T X^m Z^z with w_T = J_T i^p / 4.
//
// Matvec in grouped form.  For output index x (full spin index):
//   (H psi)[x] = sum_m c_m(x) psi[x ^ m],
//   c_m(x) = sum_{T in m} w_T (-1)^popcount(z_T & (x^m))
//          = sum_{T in m} w'_T (-1)^popcount(z_T & x),   w'_T = w_T (-1)^popcount(z_T & m).
// * popcount(m) = 4 (spins a<b<c<d, one Majorana each): z_T = zeta0 ^ s_T where
//   s_T runs over all 16 subsets of supp(m) and zeta0 = z_T & ~m is common, so
//   c_m(x) = (-1)^popcount(zeta0 & x) * Tm[u(x)], u(x) = bits of x at supp(m),
//   Tm[u] = sum_T w'_T (-1)^popcount(s_T & u)   (a 16-point Walsh transform).
// * popcount(m) = 2 (spins a<b plus a third spin c carrying both Majoranas):
//   z_T = zeta_f ^ s_T ^ e_c, so
//   c_m(x) = (-1)^popcount(zeta_f & x) * sum_c (-1)^x_c W_c[u(x)],
//   W_c[u] = sum_{T with spin c} w'_T (-1)^popcount(s_T & u).
// * m = 0 (two spins c<d, both Majoranas each): z_T = e_c ^ e_d and
//   c_0(x) = sum_{c<d} w_cd (-1)^(x_c + x_d), w_cd real.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstring>
#include <map>
#include <new>
#include <stdexcept>
#include <string>

#include "syk_internal.h"

namespace syk {

static thread_local std::string g_err;

void set_error(const char* fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
}
void clear_error() { g_err.clear(); }

namespace {

struct Pauli {
  int p;
  uint64_t m, z;
};

Pauli majorana(int a) {
  const int k = a / 2;
  const uint64_t below = (uint64_t(1) << k) - 1;
  Pauli r;
  r.m = uint64_t(1) << k;
  r.z = below | ((a & 1) ? (uint64_t(1) << k) : 0);
  r.p = a & 1;
  return r;
}

Pauli mul(const Pauli& A, const Pauli& B) {
  Pauli r;
  r.p = (A.p + B.p + 2 * __builtin_popcountll(A.z & B.m)) & 3;
  r.m = A.m ^ B.m;
  r.z = A.z ^ B.z;
  return r;
}

// bits of v at the set positions of mask, packed from the lowest position up
uint32_t extract_bits(uint64_t v, uint64_t mask) {
  uint32_t out = 0;
  int o = 0;
  for (int k = 0; k < 64; ++k)
    if ((mask >> k) & 1) out |= uint32_t((v >> k) & 1) << (o++);
  return out;
}

std::complex<double> ipow(int p) {
  static const std::complex<double> t[4] = {{1, 0}, {0, 1}, {-1, 0}, {0, -1}};
  return t[p & 3];
}

}  // namespace

}  // namespace syk

using syk::set_error;

extern "C" int syk_build_terms(int N, const double* J, syk_terms** out) {
  syk::clear_error();
  if (!out || !J) {
    set_error("syk_build_terms: NULL argument");
    return SYK_EINVAL;
  }
  *out = nullptr;
  if (N < 4 || (N & 1) || N > 64) {
    set_error("syk_build_terms: N=%d must be even, 4 <= N <= 64", N);
    return SYK_EINVAL;
  }
  syk_terms* t = new (std::nothrow) syk_terms;
  if (!t) {
    set_error("syk_build_terms: out of host memory");
    return SYK_ENOMEM;
  }
  try {
    const int n = N / 2;
    t->N = N;
    t->n = n;
    t->D = int64_t(1) << (n - 1);
    const int64_t nt = int64_t(N) * (N - 1) * (N - 2) * (N - 3) / 24;
    t->nterms = nt;
    t->xm.resize(nt);
    t->zm.resize(nt);
    t->ph.resize(nt);
    t->J.assign(J, J + nt);

    // Pauli string of every term; group term indices by X-mask.
    std::map<uint64_t, std::vector<int64_t>> groups;
    std::vector<int> dbl(nt, -1);  // popcount-2 terms: the spin carrying two Majoranas
    int64_t idx = 0;
    for (int a = 0; a < N; ++a)
      for (int b = a + 1; b < N; ++b)
        for (int c = b + 1; c < N; ++c)
          for (int d = c + 1; d < N; ++d, ++idx) {
            using namespace syk;
            Pauli P = mul(mul(mul(majorana(a), majorana(b)), majorana(c)), majorana(d));
            t->xm[idx] = P.m;
            t->zm[idx] = P.z;
            t->ph[idx] = uint8_t(P.p);
            const int sa = a / 2, sb = b / 2, sc = c / 2, sd = d / 2;
            if (sa == sb) dbl[idx] = sa;
            else if (sb == sc) dbl[idx] = sb;
            else if (sc == sd) dbl[idx] = sc;
            groups[P.m].push_back(idx);
          }
    const uint64_t Dmask = uint64_t(t->D) - 1;
    t->wdiag.assign(size_t(n) * n, 0.0);
    struct Rec4 {
      uint32_t mc, zeta, supp, flips;
      std::complex<double> tab[16];
    };
    struct Rec2 {
      uint32_t mc, zeta, ab;
      std::vector<std::complex<double>> W;
    };
    std::vector<Rec4> r4;
    std::vector<Rec2> r2;
    for (auto& kv : groups) {
      const uint64_t m = kv.first;
      const auto& terms = kv.second;
      const int pc = __builtin_popcountll(m);
      if (pc == 0) {
        for (int64_t T : terms) {
          const uint64_t z = t->zm[T];
          if (__builtin_popcountll(z) != 2) throw std::runtime_error("diagonal term z is not e_c^e_d");
          std::complex<double> w = t->J[T] * syk::ipow(t->ph[T]) / 4.0;
          if (std::abs(w.imag()) > 1e-300 && std::abs(w.imag()) > 1e-15 * std::abs(w.real()))
            throw std::runtime_error("diagonal coefficient is not real");
          const int c = __builtin_ctzll(z), d = 63 - __builtin_clzll(z);
          t->wdiag[size_t(c) * n + d] += w.real();
        }
      } else if (pc == 4) {
        Rec4 r{};
        const uint64_t zeta0 = t->zm[terms[0]] & ~m;
        for (int64_t T : terms) {
          const uint64_t z = t->zm[T];
          if ((z & ~m) != zeta0) throw std::runtime_error("popcount-4 group: zeta0 differs");
          const uint32_t s = syk::extract_bits(z, m);
          std::complex<double> w = t->J[T] * syk::ipow(t->ph[T]) / 4.0;
          if (__builtin_popcountll(z & m) & 1) w = -w;
          for (int u = 0; u < 16; ++u) r.tab[u] += (__builtin_popcount(s & u) & 1) ? -w : w;
        }
        int pos[4], o = 0;
        for (int k = 0; k < n; ++k)
          if ((m >> k) & 1) pos[o++] = k;
        r.mc = uint32_t(m & Dmask);
        r.zeta = uint32_t(zeta0);
        // support bit k of the full index lands on bit k of the table index after a right
        // shift by pos[k] - k (pos is ascending, so every shift is >= 0)
        r.supp = uint32_t(pos[0]) | uint32_t(pos[1] - 1) << 8 | uint32_t(pos[2] - 2) << 16 |
                 uint32_t(pos[3] - 3) << 24;
        // Table-index change when compact row bit j flips (j = syk::kFlipBit0 .. +5): bit j
        // of the full index flips and so does the top bit n-1 (the parity of the compact index).
        const int top = n - 1;
        for (int b = 0; b < 6; ++b) {
          const int j = syk::kFlipBit0 + b;
          uint32_t f = 0;
          if (j < top) {
            for (int k = 0; k < 4; ++k)
              if (pos[k] == j || pos[k] == top) f |= 1u << k;
            if (((zeta0 >> j) & 1) ^ ((zeta0 >> top) & 1)) f |= 16u;
          }
          r.flips |= f << (5 * b);
        }
        r4.push_back(r);
      } else if (pc == 2) {
        Rec2 r{};
        r.W.assign(size_t(n) * 4, 0.0);
        uint64_t zetaf = 0;
        bool first = true;
        for (int64_t T : terms) {
          const int c = dbl[T];
          if (c < 0) throw std::runtime_error("popcount-2 term without a doubled spin");
          const uint64_t z = t->zm[T];
          const uint64_t rr = z ^ (uint64_t(1) << c);
          if (first) {
            zetaf = rr & ~m;
            first = false;
          } else if ((rr & ~m) != zetaf) {
            throw std::runtime_error("popcount-2 group: zeta_f differs");
          }
          const uint32_t s = syk::extract_bits(rr, m);
          std::complex<double> w = t->J[T] * syk::ipow(t->ph[T]) / 4.0;
          if (__builtin_popcountll(z & m) & 1) w = -w;
          for (int u = 0; u < 4; ++u) r.W[size_t(c) * 4 + u] += (__builtin_popcount(s & u) & 1) ? -w : w;
        }
        const int a = __builtin_ctzll(m), b = 63 - __builtin_clzll(m);
        r.mc = uint32_t(m & Dmask);
        r.zeta = uint32_t(zetaf);
        r.ab = uint32_t(a) | (uint32_t(b) << 8);
        r2.push_back(std::move(r));
      } else {
        throw std::runtime_error("X-mask with odd popcount or popcount > 4");
      }
    }
    // Tables are sorted by the compact XOR mask, so masks sharing the bits above any
    // tile size form contiguous ranges (the tiled matvec walks them group by group).
    std::sort(r4.begin(), r4.end(), [](const Rec4& a, const Rec4& b) { return a.mc < b.mc; });
    std::sort(r2.begin(), r2.end(), [](const Rec2& a, const Rec2& b) { return a.mc < b.mc; });
    for (const Rec4& r : r4) {
      t->m4_rec.insert(t->m4_rec.end(), {r.mc, r.zeta, r.supp, r.flips});
      for (int u = 0; u < 32; ++u) {
        const std::complex<double> v = u < 16 ? r.tab[u] : -r.tab[u - 16];
        t->m4_tab.push_back(v.real());
        t->m4_tab.push_back(v.imag());
      }
    }
    for (const Rec2& r : r2) {
      t->m2_rec.insert(t->m2_rec.end(), {r.mc, r.zeta, r.ab, 0u});
      for (const auto& v : r.W) {
        t->m2_tab.push_back(v.real());
        t->m2_tab.push_back(v.imag());
      }
    }
    t->n4 = int(r4.size());
    t->n2 = int(r2.size());
    double sum2 = 0.0;
    for (double v : t->J) {
      if (!std::isfinite(v)) throw std::runtime_error("non-finite coupling");
      sum2 += v * v;
    }
    // Tr H^2 / 2^n = sum J^2 / 16: the RMS eigenvalue; twice it bounds the bulk of the spectrum
    t->rho_est = 2.0 * std::sqrt(sum2 / 16.0);
  } catch (const std::bad_alloc&) {
    delete t;
    set_error("syk_build_terms: out of host memory");
    return SYK_ENOMEM;
  } catch (const std::exception& e) {
    delete t;
    set_error("syk_build_terms: %s", e.what());
    return SYK_EINVAL;
  }
  *out = t;
  return SYK_OK;
}

extern "C" void syk_free_terms(syk_terms* t) {
  if (!t) return;
  syk::bump_graph_epoch();  // graphs may hold this term set's device pointers
  if (t->dev.device >= 0) {
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(t->dev.device);
    void* ptrs[] = {t->dev.m4_rec, t->dev.m4_t64, t->dev.m4_t32, t->dev.m2_rec, t->dev.m2_t64,
                    t->dev.m2_t32, t->dev.wd64,   t->dev.wd32,   t->dev.status,
                    t->dev.m4_tdf, t->dev.m2_tdf, t->dev.wd_df};
    for (void* p : ptrs)
      if (p) cudaFree(p);
    for (auto& kv : t->groups_dev)
      if (kv.second.first) cudaFree(kv.second.first);
    void* gp[] = {t->d_gg_rec, t->d_term_group, t->d_term_s, t->d_term_phase};
    for (void* p : gp)
      if (p) cudaFree(p);
    for (auto& kv : t->coset_dev) {
      void* cp[] = {kv.second.chunks, kv.second.counts, kv.second.rec, kv.second.t32, kv.second.t64};
      for (void* p : cp)
        if (p) cudaFree(p);
    }
    if (prev >= 0) cudaSetDevice(prev);
  }
  delete t;
}

extern "C" int syk_terms_info(const syk_terms* t, int* N, int64_t* nterms, int64_t* nmasks,
                              int64_t* dim) {
  if (!t) {
    set_error("syk_terms_info: NULL terms");
    return SYK_EINVAL;
  }
  if (N) *N = t->N;
  if (nterms) *nterms = t->nterms;
  if (nmasks) *nmasks = int64_t(t->n4) + t->n2 + 1;
  if (dim) *dim = t->D;
  return SYK_OK;
}

extern "C" int syk_term_table(const syk_terms* t, uint64_t* xmask, uint64_t* zmask, uint8_t* phase) {
  if (!t) {
    set_error("syk_term_table: NULL terms");
    return SYK_EINVAL;
  }
  if (xmask) std::memcpy(xmask, t->xm.data(), t->xm.size() * sizeof(uint64_t));
  if (zmask) std::memcpy(zmask, t->zm.data(), t->zm.size() * sizeof(uint64_t));
  if (phase) std::memcpy(phase, t->ph.data(), t->ph.size());
  return SYK_OK;
}

extern "C" const char* syk_last_error(void) { return syk::g_err.c_str(); }

namespace syk {

template <typename T>
static int upload(T** dst, const void* src, size_t bytes) {
  if (bytes == 0) bytes = 16;
  SYK_CUDA_CHECK(cudaMalloc((void**)dst, bytes));
  if (src) SYK_CUDA_CHECK(cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice));
  return SYK_OK;
}

int ensure_device_tables(const syk_terms* t) {
  int cur = -1;
  SYK_CUDA_CHECK(cudaGetDevice(&cur));
  std::lock_guard<std::mutex> lock(t->mtx);
  if (t->dev.device == cur) return SYK_OK;
  if (t->dev.device >= 0) {
    set_error("term tables were uploaded to device %d; current device is %d", t->dev.device, cur);
    return SYK_EINVAL;
  }
  DeviceTables& d = t->dev;
  std::vector<float> f4(t->m4_tab.begin(), t->m4_tab.end());
  std::vector<float> f2(t->m2_tab.begin(), t->m2_tab.end());
  std::vector<float> fd(t->wdiag.begin(), t->wdiag.end());
  SYK_TRY(upload(&d.m4_rec, t->m4_rec.data(), t->m4_rec.size() * 4));
  SYK_TRY(upload(&d.m4_t64, t->m4_tab.data(), t->m4_tab.size() * 8));
  SYK_TRY(upload(&d.m4_t32, f4.data(), f4.size() * 4));
  SYK_TRY(upload(&d.m2_rec, t->m2_rec.data(), t->m2_rec.size() * 4));
  SYK_TRY(upload(&d.m2_t64, t->m2_tab.data(), t->m2_tab.size() * 8));
  SYK_TRY(upload(&d.m2_t32, f2.data(), f2.size() * 4));
  SYK_TRY(upload(&d.wd64, t->wdiag.data(), t->wdiag.size() * 8));
  SYK_TRY(upload(&d.wd32, fd.data(), fd.size() * 4));
  // double-float copies: each double d as (hi, lo) = (fl(d), fl(d - hi)); complex tables
  // interleave (re_hi, im_hi, re_lo, im_lo)
  auto split = [](double v, float* hi, float* lo) {
    *hi = (float)v;
    *lo = (float)(v - (double)*hi);
  };
  auto split_complex = [&](const std::vector<double>& src) {
    std::vector<float> out(src.size() * 2);
    for (size_t e = 0; e < src.size() / 2; ++e) {
      split(src[2 * e], &out[4 * e], &out[4 * e + 2]);
      split(src[2 * e + 1], &out[4 * e + 1], &out[4 * e + 3]);
    }
    return out;
  };
  const std::vector<float> d4 = split_complex(t->m4_tab), d2 = split_complex(t->m2_tab);
  std::vector<float> dd(t->wdiag.size() * 2);
  for (size_t e = 0; e < t->wdiag.size(); ++e) split(t->wdiag[e], &dd[2 * e], &dd[2 * e + 1]);
  SYK_TRY(upload(&d.m4_tdf, d4.data(), d4.size() * 4));
  SYK_TRY(upload(&d.m2_tdf, d2.data(), d2.size() * 4));
  SYK_TRY(upload(&d.wd_df, dd.data(), dd.size() * 4));
  SYK_TRY(upload(&d.status, nullptr, 16));
  SYK_CUDA_CHECK(cudaMemset(d.status, 0, 16));
  d.device = cur;
  return SYK_OK;
}

int make_apply_params(const syk_terms* t, int parity, int dtype, ApplyParams* p) {
  if (!t || !p) {
    set_error("NULL terms");
    return SYK_EINVAL;
  }
  if (parity != 0 && parity != 1) {
    set_error("parity must be 0 or 1 (got %d)", parity);
    return SYK_EINVAL;
  }
  if (!dtype_ok(dtype)) {
    set_error("dtype must be SYK_C64 or SYK_C128 (got %d)", dtype);
    return SYK_EINVAL;
  }
  SYK_TRY(ensure_device_tables(t));
  p->n = t->n;
  p->sector = parity;
  p->D = t->D;
  p->n4 = t->n4;
  p->n2 = t->n2;
  p->m4_rec = t->dev.m4_rec;
  p->m2_rec = t->dev.m2_rec;
  const bool f = dtype == SYK_C64;
  p->m4_tab = f ? (const void*)t->dev.m4_t32 : (const void*)t->dev.m4_t64;
  p->m2_tab = f ? (const void*)t->dev.m2_t32 : (const void*)t->dev.m2_t64;
  p->wd = f ? (const void*)t->dev.wd32 : (const void*)t->dev.wd64;
  p->status = t->dev.status;
  p->rho = t->rho_est;
  p->m4_tdf = t->dev.m4_tdf;
  p->m2_tdf = t->dev.m2_tdf;
  p->wd_df = t->dev.wd_df;
  p->terms = t;
  p->no_alloc = false;
  p->df_split = nullptr;
  p->df_split_bytes = 0;
  p->ep_scale = nullptr;
  p->ep_u = nullptr;
  p->ep_part = nullptr;
  p->ep_nblk = nullptr;
  p->ep_cap = 0;
  return SYK_OK;
}

bool tile_groups_cached(const syk_terms* t, int tb, int gmax, const int4** out, int* count) {
  std::lock_guard<std::mutex> lock(t->mtx);
  auto it = t->groups_dev.find(tb << 16 | gmax);
  if (it == t->groups_dev.end()) return false;
  *out = it->second.first;
  *count = it->second.second;
  return true;
}
int tile_groups(const syk_terms* t, int tb, int gmax, const int4** out, int* count) {
  SYK_TRY(ensure_device_tables(t));
  std::lock_guard<std::mutex> lock(t->mtx);
  const int key = tb << 16 | gmax;
  auto it = t->groups_dev.find(key);
  if (it == t->groups_dev.end()) {
    std::vector<int4> g;
    size_t i4 = 0, i2 = 0;
    const size_t n4 = size_t(t->n4), n2 = size_t(t->n2);
    bool diag = false;
    while (i4 < n4 || i2 < n2 || !diag) {
      uint32_t h = 0xffffffffu;
      if (i4 < n4) h = std::min(h, t->m4_rec[4 * i4] >> tb);
      if (i2 < n2) h = std::min(h, t->m2_rec[4 * i2] >> tb);
      if (!diag) h = 0;
      const size_t b4 = i4, b2 = i2;
      while (i4 < n4 && (t->m4_rec[4 * i4] >> tb) == h) ++i4;
      while (i2 < n2 && (t->m2_rec[4 * i2] >> tb) == h) ++i2;
      if (h == 0) diag = true;
      size_t c0 = b4;
      bool first = true;
      do {
        const size_t c1 = std::min(i4, c0 + size_t(gmax));
        const int k2 = first ? int(b2 | (i2 << 16)) : 0;
        g.push_back(make_int4(int(h | (first ? 0x80000000u : 0u)), int(c0), int(c1), k2));
        first = false;
        c0 = c1;
      } while (c0 < i4);
    }
    int4* d = nullptr;
    SYK_CUDA_CHECK(cudaMalloc(&d, g.size() * sizeof(int4)));
    SYK_CUDA_CHECK(cudaMemcpy(d, g.data(), g.size() * sizeof(int4), cudaMemcpyHostToDevice));
    it = t->groups_dev.emplace(key, std::make_pair(d, int(g.size()))).first;
  }
  *out = it->second.first;
  *count = it->second.second;
  return SYK_OK;
}


// Gradient term groups.  For term T with X-mask m and Z-mask z_T the matrix element is
// (P_T psi)[x] = (i^p/4) (-1)^popcount(z_T & (x^m)) psi[x^m].  Terms are grouped so that
// z_T = zeta ^ spread(s_T) with s_T the bits of z_T at k "support" positions:
//   popcount-4 masks: the 4 spins of m (k = 4, 16 terms);
//   popcount-2 masks: one group per (m, doubled spin c) (k = 2, 4 terms);
//   diagonal: one group per term (k = 0).
// Then <lam|P_T|psi> = phase_T * sum_x conj(lam[x]) psi[x^m] (-1)^popcount(zeta & x)
//                      (-1)^popcount(s_T & u(x)), u(x) = bits of x at the support.
int ensure_grad_groups(const syk_terms* t) {
  SYK_TRY(ensure_device_tables(t));
  std::lock_guard<std::mutex> lock(t->mtx);
  if (t->d_gg_rec) return SYK_OK;
  const int n = t->n, N = t->N;
  const uint64_t Dmask = uint64_t(t->D) - 1;
  std::map<std::pair<uint64_t, uint64_t>, int> key2g;
  t->gg_rec.clear();
  t->term_group.assign(t->nterms, -1);
  t->term_s.assign(t->nterms, 0);
  t->term_phase.assign(2 * t->nterms, 0.0);
  int64_t T = 0;
  for (int a = 0; a < N; ++a)
    for (int b = a + 1; b < N; ++b)
      for (int c = b + 1; c < N; ++c)
        for (int d = c + 1; d < N; ++d, ++T) {
          const uint64_t m = t->xm[T], z = t->zm[T];
          const int pc = __builtin_popcountll(m);
          uint64_t zeta, supp, keyz;
          if (pc == 4) {
            supp = m;
            zeta = z & ~m;
            keyz = 0;
          } else if (pc == 2) {
            const int sa = a / 2, sb = b / 2, sc = c / 2, sd = d / 2;
            const int dbl = sa == sb ? sa : sb == sc ? sb : sd;
            supp = m;
            zeta = z & ~m;  // shared by the 4 terms of (m, dbl), including the doubled spin's Z bit
            keyz = uint64_t(1) << dbl;
          } else {
            supp = 0;
            zeta = z;
            keyz = z;
          }
          const auto key = std::make_pair(m, keyz);
          auto it = key2g.find(key);
          int g;
          if (it == key2g.end()) {
            g = int(key2g.size());
            key2g.emplace(key, g);
            int pos[4] = {0, 0, 0, 0}, o = 0;
            for (int k = 0; k < n; ++k)
              if ((supp >> k) & 1) pos[o++] = k;
            uint32_t shifts = 0;
            for (int k = 0; k < 4; ++k) shifts |= uint32_t(k < o ? pos[k] - k : 31) << (8 * k);
            t->gg_rec.insert(t->gg_rec.end(), {uint32_t(m & Dmask), uint32_t(zeta), shifts, uint32_t(o)});
          } else {
            g = it->second;
          }
          t->term_group[T] = g;
          t->term_s[T] = uint8_t(syk::extract_bits(z, supp));
          std::complex<double> ph = syk::ipow(t->ph[T]) / 4.0;
          if (__builtin_popcountll(z & m) & 1) ph = -ph;
          t->term_phase[2 * T] = ph.real();
          t->term_phase[2 * T + 1] = ph.imag();
        }
  t->ngg = int(key2g.size());
  SYK_TRY(upload(&t->d_gg_rec, t->gg_rec.data(), t->gg_rec.size() * 4));
  SYK_TRY(upload(&t->d_term_group, t->term_group.data(), t->term_group.size() * 4));
  SYK_TRY(upload(&t->d_term_s, t->term_s.data(), t->term_s.size()));
  SYK_TRY(upload(&t->d_term_phase, t->term_phase.data(), t->term_phase.size() * 8));
  return SYK_OK;
}



// Member sets (bit d: row-slot offset d) of the multi-mask cosets that popcount-4 masks
// form for 1, 2 or 3 row bits; any other coset is split into single masks.
static const uint32_t* coset_shapes(int rbits, int* count) {
  static const uint32_t s1[] = {0x3u};
  static const uint32_t s2[] = {0x7u, 0xEu};
  static const uint32_t s3[] = {0x17u, 0xE8u, 0x7Eu};
  *count = rbits == 1 ? 1 : rbits == 2 ? 2 : 3;
  return rbits == 1 ? s1 : rbits == 2 ? s2 : s3;
}

int coset_layout_host(const syk_terms* t, int tb, int rbits, int gmax, CosetHost* out) {
  if (rbits < 1 || rbits > 3 || tb < rbits || gmax < 8 || gmax > 255) {
    set_error("coset_layout: unsupported shape (tb=%d rbits=%d gmax=%d)", tb, rbits, gmax);
    return SYK_EINVAL;
  }
  const int n4 = t->n4, n2 = t->n2;
  const int shift = tb - rbits;
  const uint32_t dmask = ((1u << rbits) - 1u) << shift;
  int nshape = 0;
  const uint32_t* shapes = coset_shapes(rbits, &nshape);
  CosetHost& L = *out;
  L = CosetHost();
  // masks are sorted by compact XOR, so one h = m >> tb is a contiguous range
  int i4 = 0, i2 = 0;
  bool diag = false;
  while (i4 < n4 || i2 < n2 || !diag) {
    uint32_t h = 0xffffffffu;
    if (i4 < n4) h = std::min(h, t->m4_rec[4 * i4] >> tb);
    if (i2 < n2) h = std::min(h, t->m2_rec[4 * i2] >> tb);
    if (!diag) h = 0;
    const int b4 = i4, b2 = i2;
    while (i4 < n4 && (t->m4_rec[4 * i4] >> tb) == h) ++i4;
    while (i2 < n2 && (t->m2_rec[4 * i2] >> tb) == h) ++i2;
    if (h == 0) diag = true;
    // cosets of this h: key = compact mask with the row-slot bits cleared; members by offset d
    std::map<uint32_t, std::map<uint32_t, int>> cmap;
    for (int k = b4; k < i4; ++k) cmap[t->m4_rec[4 * k] & ~dmask][(t->m4_rec[4 * k] & dmask) >> shift] = k;
    // units in chunk order: the cosets of each listed shape, then single masks
    std::vector<std::pair<int, std::vector<int>>> units;  // (shape slot or -1, masks in offset order)
    for (int sh = 0; sh < nshape; ++sh)
      for (auto& c : cmap) {
        uint32_t shape = 0;
        for (auto& md : c.second) shape |= 1u << md.first;
        if (shape != shapes[sh]) continue;
        std::vector<int> ks;
        for (auto& md : c.second) ks.push_back(md.second);
        units.emplace_back(sh, ks);
      }
    for (auto& c : cmap) {
      uint32_t shape = 0;
      for (auto& md : c.second) shape |= 1u << md.first;
      bool listed = false;
      for (int sh = 0; sh < nshape; ++sh) listed |= shape == shapes[sh];
      if (!listed)
        for (auto& md : c.second) units.emplace_back(-1, std::vector<int>{md.second});
    }
    std::stable_sort(units.begin(), units.end(), [](const std::pair<int, std::vector<int>>& a,
                                                    const std::pair<int, std::vector<int>>& b) {
      return (a.first < 0 ? 1000 : a.first) < (b.first < 0 ? 1000 : b.first);
    });
    size_t u = 0;
    bool first = true;
    do {
      const int mbeg = int(L.rec.size());
      int used = 0;
      uint32_t counts = 0;
      while (u < units.size() && used + int(units[u].second.size()) <= gmax) {
        if (units[u].first >= 0) counts += 1u << (8 * units[u].first);
        for (int k : units[u].second) {
          L.rec.push_back(make_uint4(t->m4_rec[4 * k], t->m4_rec[4 * k + 1], t->m4_rec[4 * k + 2], t->m4_rec[4 * k + 3]));
          for (int e = 0; e < 64; ++e) {
            L.t64.push_back(t->m4_tab[size_t(k) * 64 + e]);
            L.t32.push_back(float(t->m4_tab[size_t(k) * 64 + e]));
          }
          ++used;
        }
        ++u;
      }
      const int k2 = first ? (b2 | (i2 << 16)) : 0;
      L.chunks.push_back(make_int4(int(h | (first ? 0x80000000u : 0u)), mbeg, int(L.rec.size()), k2));
      L.counts.push_back(counts);
      first = false;
    } while (u < units.size());
  }
  return SYK_OK;
}

int coset_layout(const syk_terms* t, int tb, int rbits, int gmax, bool may_alloc, const CosetLayout** out) {
  if (may_alloc) SYK_TRY(ensure_device_tables(t));
  std::lock_guard<std::mutex> lock(t->mtx);
  const int key = (tb << 16) | (rbits << 8) | gmax;
  auto it = t->coset_dev.find(key);
  if (it != t->coset_dev.end()) {
    *out = &it->second;
    return SYK_OK;
  }
  if (!may_alloc) return 1;  // not built yet
  CosetHost H;
  SYK_TRY(coset_layout_host(t, tb, rbits, gmax, &H));
  CosetLayout L;
  L.nchunks = int(H.chunks.size());
  SYK_TRY(upload(&L.chunks, H.chunks.data(), H.chunks.size() * sizeof(int4)));
  SYK_TRY(upload(&L.counts, H.counts.data(), H.counts.size() * sizeof(uint32_t)));
  SYK_TRY(upload(&L.rec, H.rec.data(), H.rec.size() * sizeof(uint4)));
  SYK_TRY(upload(&L.t32, H.t32.data(), H.t32.size() * sizeof(float)));
  SYK_TRY(upload(&L.t64, H.t64.data(), H.t64.size() * sizeof(double)));
  it = t->coset_dev.emplace(key, L).first;
  *out = &it->second;
  return SYK_OK;
}

}  // namespace syk
