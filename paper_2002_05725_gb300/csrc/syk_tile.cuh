// Device helpers shared by the tiled matvec kernels (syk_apply.cu, syk_apply_coset.cu):
// table-index extraction, bulk-copy / mbarrier / cluster PTX wrappers, 16-byte row-chunk
// multiply-adds, and the diagonal and popcount-2 coefficients (Supp. Sec. I.B).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>

#include "syk_cplx.cuh"
#include "syk_df.cuh"
#include "syk_internal.h"

namespace syk {

// opt-in dynamic shared memory per CTA on sm_100-class GPUs
constexpr size_t kMaxSmemPerCta = 227 * 1024;

// Table index bits of a popcount-4 mask: bit k = bit pos_k of the full index xf.
// s packs the right-shift pos_k - k of support bit k into byte k (funnel shifts use
// only the low 5 bits of the amount).
__device__ __forceinline__ uint32_t supp_bits(uint32_t xf, uint32_t s) {
  return (__funnelshift_r(xf, 0u, s) & 1u) | (__funnelshift_r(xf, 0u, s >> 8) & 2u) |
         (__funnelshift_r(xf, 0u, s >> 16) & 4u) | (__funnelshift_r(xf, 0u, s >> 24) & 8u);
}


namespace tma {
__device__ __forceinline__ uint32_t saddr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void expect_tx(uint64_t* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(saddr(b)), "r"(bytes) : "memory");
}
// bulk global -> shared copy; completion is signalled on mbarrier b as transaction bytes
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* b) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   saddr(dst)),
               "l"(src), "r"(bytes), "r"(saddr(b))
               : "memory");
}
__device__ __forceinline__ bool try_wait(uint64_t* b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(saddr(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Waits for phase `parity` of b; gives up after `polls` polls (each try_wait may itself block
// for a short hardware-defined time).
__device__ __forceinline__ bool wait_bounded(uint64_t* b, uint32_t parity, uint32_t polls) {
  for (uint32_t it = 0; it < polls; ++it)
    if (try_wait(b, parity)) return true;
  return false;
}
// Poll budget of the main-loop waits for staged tiles (a build-time knob: a build with 0 makes
// every such wait give up at once, which exercises the timeout path), and of the drain that
// lets in-flight copies land before a CTA that gave up exits (always the full budget).
#ifndef SYK_WAIT_POLLS
#define SYK_WAIT_POLLS (1u << 22)
#endif
constexpr uint32_t kWaitPolls = SYK_WAIT_POLLS;
constexpr uint32_t kDrainPolls = 1u << 22;
// thread-block cluster helpers
__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ uint32_t cluster_size() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// shared-memory address of the same offset in CTA `rank` of the cluster
__device__ __forceinline__ uint32_t map_rank(uint32_t saddr_local, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(saddr_local), "r"(rank));
  return r;
}
__device__ __forceinline__ float4 ld_cluster(uint32_t a, float4) {
  float4 v;
  asm volatile("ld.shared::cluster.v4.f32 {%0, %1, %2, %3}, [%4];"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
               : "r"(a)
               : "memory");
  return v;
}
__device__ __forceinline__ double2 ld_cluster(uint32_t a, double2) {
  double2 v;
  asm volatile("ld.shared::cluster.v2.f64 {%0, %1}, [%2];" : "=d"(v.x), "=d"(v.y) : "r"(a) : "memory");
  return v;
}
}  // namespace tma

// 16-byte chunk of a row: T is the chunk (and accumulator) type, Out what the output row
// stores, mac adds coefficient x chunk, renorm is called after every mask chunk.
template <typename R>
struct Slot;
template <>
struct Slot<float> {
  using T = float4;  // two complex64
  using Out = float4;
  static __device__ __forceinline__ void mac(float4& a, float cr, float ci, const float4 v) {
    a.x = fmaf(cr, v.x, fmaf(-ci, v.y, a.x));
    a.y = fmaf(cr, v.y, fmaf(ci, v.x, a.y));
    a.z = fmaf(cr, v.z, fmaf(-ci, v.w, a.z));
    a.w = fmaf(cr, v.w, fmaf(ci, v.z, a.w));
  }
  static __device__ __forceinline__ void mac(float4& a, const float2 c, const float4 v) { mac(a, c.x, c.y, v); }
  static __device__ __forceinline__ float4 zero() { return make_float4(0.f, 0.f, 0.f, 0.f); }
  static __device__ __forceinline__ Out out(const float4 a) { return a; }
  static __device__ __forceinline__ void renorm(float4&) {}
};
template <>
struct Slot<double> {
  using T = double2;  // one complex128
  using Out = double2;
  static __device__ __forceinline__ void mac(double2& a, double cr, double ci, const double2 v) { cmac(a, cr, ci, v); }
  static __device__ __forceinline__ void mac(double2& a, const double2 c, const double2 v) { cmac(a, c.x, c.y, v); }
  static __device__ __forceinline__ double2 zero() { return make_double2(0.0, 0.0); }
  static __device__ __forceinline__ Out out(const double2 a) { return a; }
  static __device__ __forceinline__ void renorm(double2&) {}
};
template <>
struct Slot<DF> {
  using T = float4;  // one complex128 as a double-float pair
  using Out = double2;
  static __device__ __forceinline__ void mac(float4& a, const float4 c, const float4 v) { df_cmac(a, c, v); }
  static __device__ __forceinline__ float4 zero() { return make_float4(0.f, 0.f, 0.f, 0.f); }
  static __device__ __forceinline__ Out out(const float4 a) { return df_to_double2(a); }
  static __device__ __forceinline__ void renorm(float4& a) { df_renorm4(a); }
};

// Table pointers of a launch for arithmetic R (the double-float kernel reads the split tables).
template <typename R>
__device__ __forceinline__ const typename CT<R>::T* tab4(const ApplyParams& p) {
  if constexpr (std::is_same<R, DF>::value) return p.m4_tdf;
  else return static_cast<const typename CT<R>::T*>(p.m4_tab);
}
template <typename R>
__device__ __forceinline__ const typename CT<R>::T* tab2(const ApplyParams& p) {
  if constexpr (std::is_same<R, DF>::value) return p.m2_tdf;
  else return static_cast<const typename CT<R>::T*>(p.m2_tab);
}

// diagonal coefficient c_0(x) = sum_{c<d} w_cd (-1)^{x_c + x_d}
template <typename R>
__device__ __forceinline__ R diag_coef(const R* __restrict__ wd, int n, uint32_t xf) {
  R dsum = R(0);
  for (int c = 0; c < n - 1; ++c) {
    R inner = R(0);
    for (int d = c + 1; d < n; ++d) {
      const R w = __ldg(&wd[c * n + d]);
      inner += ((xf >> d) & 1u) ? -w : w;
    }
    dsum += ((xf >> c) & 1u) ? -inner : inner;
  }
  return dsum;
}

// the diagonal coefficient as a complex value of the kernel's coefficient type
template <typename R>
__device__ __forceinline__ typename CT<R>::T diag_c(const ApplyParams& p, int n, uint32_t xf) {
  if constexpr (std::is_same<R, DF>::value) {
    // sum_{c<d} w_cd (-1)^{x_c + x_d} in double-float (w_cd stored as (hi, lo))
    float hi = 0.f, lo = 0.f;
    for (int c = 0; c < n - 1; ++c)
      for (int d = c + 1; d < n; ++d) {
        const float2 w = __ldg(&p.wd_df[c * n + d]);
        df_add_signed(hi, lo, w.x, w.y, ((xf >> c) ^ (xf >> d)) & 1u);
      }
    df_renorm(hi, lo);
    return make_float4(hi, 0.f, lo, 0.f);
  } else {
    return make_c<R>(diag_coef<R>(static_cast<const R*>(p.wd), n, xf), R(0));
  }
}

// popcount-2 coefficient c_m(x) = (-1)^{popcount(zeta_f & x)} sum_c (-1)^{x_c} W_c[u(x)]
template <typename C, typename R>
__device__ __forceinline__ void pc2_coef(const C* __restrict__ t2, int k, int n, uint4 rec, uint32_t xf, R& cr,
                                         R& ci) {
  const uint32_t a = rec.z & 0xffu, bb = (rec.z >> 8) & 0xffu;
  const uint32_t u = ((xf >> a) & 1u) | (((xf >> bb) & 1u) << 1);
  const C* W = t2 + (size_t)k * n * 4 + u;
  cr = R(0);
  ci = R(0);
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
}


// the popcount-2 coefficient as a complex value of the kernel's coefficient type
template <typename R>
__device__ __forceinline__ typename CT<R>::T pc2_c(const typename CT<R>::T* __restrict__ t2, int k, int n, uint4 rec,
                                                  uint32_t xf) {
  if constexpr (std::is_same<R, DF>::value) {
    const uint32_t a = rec.z & 0xffu, bb = (rec.z >> 8) & 0xffu;
    const uint32_t u = ((xf >> a) & 1u) | (((xf >> bb) & 1u) << 1);
    const float4* W = t2 + (size_t)k * n * 4 + u;
    const bool flip = __popc(rec.y & xf) & 1;
    float rh = 0.f, ih = 0.f, rl = 0.f, il = 0.f;
    for (int c = 0; c < n; ++c) {
      const float4 w = __ldg(&W[4 * c]);
      const bool neg = (((xf >> c) & 1u) != 0u) != flip;
      df_add_signed(rh, rl, w.x, w.z, neg);
      df_add_signed(ih, il, w.y, w.w, neg);
    }
    df_renorm(rh, rl);
    df_renorm(ih, il);
    return make_float4(rh, ih, rl, il);
  } else {
    typename CT<R>::T c;
    pc2_coef<typename CT<R>::T, R>(t2, k, n, rec, xf, c.x, c.y);
    return c;
  }
}

// ---------------------------------------------------------------- output stage
// The tiled matvecs write a CTA's outputs as 16-byte units: unit u lies at byte offset
// goff + 16 u of the vector (goff = the CTA's first unit, always at the start of a row).  A
// thread handles units tid, tid + NT, ...; their stride 16 NT is a multiple of the row size
// ROWB (columns x element size <= 256 <= 16 x 64), so a thread's units always hold the same
// columns: element slot e of unit u (e = 0, 1 for complex64 pairs, 0 for complex128) is column
//   col(tid, e) = ((16 tid + esz e) mod ROWB) / esz.
// With the Lanczos epilogue (p.ep_part set) every element is multiplied by its column's
// ep_scale and the CTA's conj(ep_u) . y sums per column are written to p.ep_part[cta][column]:
// per-thread sums (FP32 products and sums for complex64, FP64 for complex128) over the
// thread's units, then per column over the threads in increasing order (deterministic).
template <typename V16>
struct EpiVec;
template <>
struct EpiVec<float4> {  // two complex64 per unit
  static constexpr int NE = 2, ESZ = 8;
  struct Acc {
    float r[2] = {0.f, 0.f}, i[2] = {0.f, 0.f};
  };
  static __device__ __forceinline__ float4 scale(float4 v, const double (&s)[2]) {
    const float s0 = (float)s[0], s1 = (float)s[1];
    return make_float4(v.x * s0, v.y * s0, v.z * s1, v.w * s1);
  }
  static __device__ __forceinline__ void dot(Acc& a, const float4 u, const float4 v) {
    a.r[0] = fmaf(u.x, v.x, fmaf(u.y, v.y, a.r[0]));
    a.i[0] = fmaf(u.x, v.y, fmaf(-u.y, v.x, a.i[0]));
    a.r[1] = fmaf(u.z, v.z, fmaf(u.w, v.w, a.r[1]));
    a.i[1] = fmaf(u.z, v.w, fmaf(-u.w, v.z, a.i[1]));
  }
  static __device__ __forceinline__ double2 get(const Acc& a, int e) { return make_double2(a.r[e], a.i[e]); }
};
template <>
struct EpiVec<double2> {  // one complex128 per unit
  static constexpr int NE = 1, ESZ = 16;
  struct Acc {
    double r = 0.0, i = 0.0;
  };
  static __device__ __forceinline__ double2 scale(double2 v, const double (&s)[1]) {
    return make_double2(v.x * s[0], v.y * s[0]);
  }
  static __device__ __forceinline__ void dot(Acc& a, const double2 u, const double2 v) {
    a.r = fma(u.x, v.x, fma(u.y, v.y, a.r));
    a.i = fma(u.x, v.y, fma(-u.y, v.x, a.i));
  }
  static __device__ __forceinline__ double2 get(const Acc& a, int) { return make_double2(a.r, a.i); }
};

// Stores units [0, units) (fetch(u) gives unit u) to y at byte offset goff, with the Lanczos
// epilogue if p.ep_part is set.  red: shared scratch of 32 NT bytes.  Every thread calls it.
template <typename V16, int ROWB, typename Fetch>
__device__ __forceinline__ void store_units(const ApplyParams& p, int units, int NT, size_t goff, void* y,
                                            Fetch&& fetch, unsigned char* red) {
  using E = EpiVec<V16>;
  constexpr int NE = E::NE, ESZ = E::ESZ, NB = ROWB / ESZ > 0 ? ROWB / ESZ : 1;
  const int tid = threadIdx.x;
  unsigned char* yt = static_cast<unsigned char*>(y) + goff;
  if (p.ep_part == nullptr) {
    for (int u = tid; u < units; u += NT) *reinterpret_cast<V16*>(yt + 16u * u) = fetch(u);
    return;
  }
  double s[NE];
#pragma unroll
  for (int e = 0; e < NE; ++e) {
    const int c = ((16 * tid + ESZ * e) % ROWB) / ESZ;
    s[e] = p.ep_scale ? p.ep_scale[c] : 1.0;
  }
  typename E::Acc acc;
  const unsigned char* ut = static_cast<const unsigned char*>(p.ep_u) + goff;
  for (int u = tid; u < units; u += NT) {
    const V16 v = E::scale(fetch(u), s);
    *reinterpret_cast<V16*>(yt + 16u * u) = v;
    E::dot(acc, *reinterpret_cast<const V16*>(ut + 16u * u), v);
  }
  double2* r = reinterpret_cast<double2*>(red);
#pragma unroll
  for (int e = 0; e < NE; ++e) r[tid * NE + e] = E::get(acc, e);
  __syncthreads();
  if (tid < NB) {
    // column tid: units with slot q = (tid esz) / 16 mod P of every row (P units per row), or
    // every unit when a unit spans more than one row (one column)
    double2 sum = make_double2(0.0, 0.0);
    if constexpr (ROWB >= 16) {
      constexpr int P = ROWB / 16;
      const int q = (tid * ESZ / 16) % P, e = (tid * ESZ % 16) / ESZ;
      for (int t = q; t < NT; t += P) {
        sum.x += r[t * NE + e].x;
        sum.y += r[t * NE + e].y;
      }
    } else {
      for (int t = 0; t < NT * NE; ++t) {
        sum.x += r[t].x;
        sum.y += r[t].y;
      }
    }
    p.ep_part[(size_t)blockIdx.x * NB + tid] = sum;
  }
  if (blockIdx.x == 0 && tid == 0) *p.ep_nblk = (int)gridDim.x;
}

}  // namespace syk
