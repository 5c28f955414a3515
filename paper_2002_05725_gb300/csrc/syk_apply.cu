// K1: y = H psi in one parity sector, matrix-free (Supp. Sec. I.B), and
// K5: y = chi_i psi (Supp. Sec. I.A).
//
// One thread owns one output row x (compact index) and BT batch columns.  It
// evaluates every X-mask coefficient c_m(x) from the grouped tables built on
// the host (see syk_terms.cpp) and gathers psi[x ^ m] for the BT columns:
//   y[x][b] = c_0(x) psi[x][b] + sum_{popcount(m)=2} c_m(x) psi[x^m][b]
//                              + sum_{popcount(m)=4} c_m(x) psi[x^m][b].
// The full spin index of x (needed for the sign parities) is
//   xf = x | ((popcount(x) + sector) & 1) << (n-1);
// the gather index is x ^ (m & (D-1)) because every X-mask has even popcount.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "syk_cplx.cuh"
#include "syk_internal.h"

namespace syk {
namespace {

template <typename R, int BT>
__global__ void __launch_bounds__(128) k_apply_H(ApplyParams p, const typename CT<R>::T* __restrict__ psi,
                                                 typename CT<R>::T* __restrict__ y, int64_t ld, int64_t b0) {
  using C = typename CT<R>::T;
  const C* __restrict__ t4 = static_cast<const C*>(p.m4_tab);
  const C* __restrict__ t2 = static_cast<const C*>(p.m2_tab);
  const R* __restrict__ wd = static_cast<const R*>(p.wd);
  const int n = p.n;
  for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < p.D;
       x += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t xc = (uint32_t)x;
    const uint32_t xf = xc | ((uint32_t)((__popc(xc) + p.sector) & 1) << (n - 1));
    C acc[BT];
    // diagonal: c_0(x) = sum_{c<d} w_cd s_c s_d, s_c = (-1)^{x_c}
    {
      R dsum = R(0);
      for (int c = 0; c < n - 1; ++c) {
        R inner = R(0);
        for (int d = c + 1; d < n; ++d) {
          const R w = __ldg(&wd[c * n + d]);
          inner += ((xf >> d) & 1u) ? -w : w;
        }
        dsum += ((xf >> c) & 1u) ? -inner : inner;
      }
      const C* src = psi + x * ld + b0;
#pragma unroll
      for (int b = 0; b < BT; ++b) {
        const C v = src[b];
        acc[b] = make_c<R>(dsum * v.x, dsum * v.y);
      }
    }
    // popcount-2 masks
    for (int k = 0; k < p.n2; ++k) {
      const uint4 rec = __ldg(&p.m2_rec[k]);
      const uint32_t a = rec.z & 0xffu, bb = (rec.z >> 8) & 0xffu;
      const uint32_t u = ((xf >> a) & 1u) | (((xf >> bb) & 1u) << 1);
      const C* W = t2 + (size_t)k * n * 4 + u;
      R cr = R(0), ci = R(0);
      for (int c = 0; c < n; ++c) {
        const C w = __ldg(&W[4 * c]);
        if ((xf >> c) & 1u) {
          cr -= w.x;
          ci -= w.y;
        } else {
          cr += w.x;
          ci += w.y;
        }
      }
      if (__popc(rec.y & xf) & 1) {
        cr = -cr;
        ci = -ci;
      }
      const C* src = psi + (int64_t)(xc ^ rec.x) * ld + b0;
#pragma unroll
      for (int b = 0; b < BT; ++b) cmac(acc[b], cr, ci, src[b]);
    }
    // popcount-4 masks: c_m(x) = T[(sign << 4) | u(x)]
    for (int k = 0; k < p.n4; ++k) {
      const uint4 rec = __ldg(&p.m4_rec[k]);
      const uint32_t s = rec.z;
      const uint32_t u = ((xf >> (s & 0xffu)) & 1u) | (((xf >> ((s >> 8) & 0xffu)) & 1u) << 1) |
                         (((xf >> ((s >> 16) & 0xffu)) & 1u) << 2) | (((xf >> (s >> 24)) & 1u) << 3);
      const uint32_t idx = u | ((__popc(rec.y & xf) & 1u) << 4);
      const C cf = __ldg(&t4[(size_t)k * 32 + idx]);
      const C* src = psi + (int64_t)(xc ^ rec.x) * ld + b0;
#pragma unroll
      for (int b = 0; b < BT; ++b) cmac(acc[b], cf.x, cf.y, src[b]);
    }
    C* dst = y + x * ld + b0;
#pragma unroll
    for (int b = 0; b < BT; ++b) dst[b] = acc[b];
  }
}

template <typename R, int BT>
void launch_one(const ApplyParams& p, const void* psi, void* y, int64_t ld, int64_t b0, cudaStream_t st) {
  using C = typename CT<R>::T;
  const int threads = 128;
  int64_t blocks = (p.D + threads - 1) / threads;
  blocks = std::min<int64_t>(blocks, 152 * 64);
  k_apply_H<R, BT><<<(unsigned)blocks, threads, 0, st>>>(p, static_cast<const C*>(psi), static_cast<C*>(y), ld, b0);
}

template <typename R>
int launch_apply_T(const ApplyParams& p, const void* psi, void* y, int64_t batch, cudaStream_t st) {
  int64_t b0 = 0;
  while (b0 < batch) {
    const int64_t rem = batch - b0;
    if (rem >= 16) { launch_one<R, 16>(p, psi, y, batch, b0, st); b0 += 16; }
    else if (rem >= 8) { launch_one<R, 8>(p, psi, y, batch, b0, st); b0 += 8; }
    else if (rem >= 4) { launch_one<R, 4>(p, psi, y, batch, b0, st); b0 += 4; }
    else if (rem >= 2) { launch_one<R, 2>(p, psi, y, batch, b0, st); b0 += 2; }
    else { launch_one<R, 1>(p, psi, y, batch, b0, st); b0 += 1; }
  }
  SYK_CUDA_CHECK(cudaGetLastError());
  return SYK_OK;
}

// chi_i |x> = (1/sqrt 2) (-1)^{popcount(x & ((1<<k)-1))} f_i(x_k) |x ^ (1<<k)>,
// f = 1 for even i (sigma^x), f = i (x_k = 0) or -i (x_k = 1) for odd i (sigma^y).
template <typename R>
__global__ void k_apply_chi(int n, int maj, int sector_out, int64_t D, int64_t batch,
                            const typename CT<R>::T* __restrict__ psi, typename CT<R>::T* __restrict__ y) {
  using C = typename CT<R>::T;
  const int k = maj >> 1;
  const R h = R(0.70710678118654752440);
  const int64_t total = D * batch;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c_out = e / batch, b = e - c_out * batch;
    const uint32_t co = (uint32_t)c_out;
    const uint32_t xo = co | ((uint32_t)((__popc(co) + sector_out) & 1) << (n - 1));
    const uint32_t x = xo ^ (1u << k);                    // source spin state
    const uint32_t below = x & ((1u << k) - 1u);
    const R sg = (__popc(below) & 1) ? -h : h;
    const C v = psi[(int64_t)(x & (uint32_t)(D - 1)) * batch + b];
    C r;
    if (maj & 1) {
      // multiply by +i (x_k = 0) or -i (x_k = 1)
      const R si = ((x >> k) & 1u) ? -sg : sg;
      r = make_c<R>(-si * v.y, si * v.x);
    } else {
      r = make_c<R>(sg * v.x, sg * v.y);
    }
    y[e] = r;
  }
}

}  // namespace

int launch_apply_H(const ApplyParams& p, int dtype, const void* psi, void* y, int64_t batch, cudaStream_t st) {
  prof_before_apply(st);
  int rc = dtype == SYK_C64 ? launch_apply_T<float>(p, psi, y, batch, st)
                            : launch_apply_T<double>(p, psi, y, batch, st);
  prof_after_apply(st);
  count_applies(batch);
  return rc;
}

int launch_apply_chi(int N, int i, int parity_in, int dtype, const void* psi, void* y, int64_t batch,
                     cudaStream_t st) {
  const int n = N / 2;
  const int64_t D = int64_t(1) << (n - 1);
  const int threads = 256;
  int64_t blocks = std::min<int64_t>((D * batch + threads - 1) / threads, 152 * 32);
  if (dtype == SYK_C64)
    k_apply_chi<float><<<(unsigned)blocks, threads, 0, st>>>(n, i, 1 - parity_in, D, batch,
                                                             static_cast<const float2*>(psi), static_cast<float2*>(y));
  else
    k_apply_chi<double><<<(unsigned)blocks, threads, 0, st>>>(n, i, 1 - parity_in, D, batch,
                                                              static_cast<const double2*>(psi), static_cast<double2*>(y));
  SYK_CUDA_CHECK(cudaGetLastError());
  return SYK_OK;
}

}  // namespace syk

extern "C" int syk_apply_H(const syk_terms* terms, int parity, int dtype, const void* psi, void* y,
                           int64_t batch, void* stream) {
  syk::clear_error();
  if (!psi || !y || batch < 1) {
    syk::set_error("syk_apply_H: NULL vector or batch < 1");
    return SYK_EINVAL;
  }
  syk::ApplyParams p;
  SYK_TRY(syk::make_apply_params(terms, parity, dtype, &p));
  return syk::launch_apply_H(p, dtype, psi, y, batch, static_cast<cudaStream_t>(stream));
}

extern "C" int syk_apply_chi(int N, int i, int parity_in, int dtype, const void* psi, void* y, int64_t batch,
                             void* stream) {
  syk::clear_error();
  if (N < 4 || (N & 1) || N > 64 || i < 0 || i >= N || (parity_in != 0 && parity_in != 1) ||
      !syk::dtype_ok(dtype) || !psi || !y || batch < 1) {
    syk::set_error("syk_apply_chi: invalid argument (N=%d i=%d parity=%d dtype=%d batch=%lld)", N, i,
                   parity_in, dtype, (long long)batch);
    return SYK_EINVAL;
  }
  return syk::launch_apply_chi(N, i, parity_in, dtype, psi, y, batch, static_cast<cudaStream_t>(stream));
}
