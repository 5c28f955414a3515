// K1 variant: y = H psi in one parity sector (Supp. Sec. I.B) for complex64 batches of 4, 8
// or 16 columns, with partner-row reuse across the cosets of X-masks.
//
// Same tiles, chunks and staging as k_apply_tiled (syk_apply.cu), but the popcount-4 masks
// of a chunk come in cosets: masks that differ only in the RB row-slot bits (ntb ..
// ntb+RB-1) of the compact index.  For row slot i, member d of a coset reads partner row
// slot i ^ d, so the thread loads each of its RPT partner rows ONCE per coset and
// accumulates it into every row slot that a member maps onto it: one shared-memory read
// feeds up to RPT complex multiply-adds per column instead of one.  Popcount-4 masks form
// cosets of only a few member sets (offsets {1,2,3} or {0,1,2} for two row bits, ...); the
// host orders each chunk's masks by member set (syk_terms.cpp), so the kernel runs one tight
// loop per set, and the masks left single go through a per-mask loop.  At N = 40 the
// cosets hold 1.2 masks on average for one row bit, 1.51 for two and 1.92 for three.  The
// CTA width is a template parameter, so the row-slot stride is an immediate load offset.
#include <cuda_runtime.h>

#include <cstdint>

#include "syk_coset.cuh"
#include "syk_tile.cuh"

#ifndef SYK_GMAX
#define SYK_GMAX 16
#endif

namespace syk {
namespace {

template <int BT, int RB>
struct CosetCfg {
  static constexpr int RPT = 1 << RB;
  static constexpr int ROWB = BT * 8;
  static constexpr int CH = ROWB / 16;  // 16-byte chunks per row (BT >= 2)
  static constexpr int GMAX = SYK_GMAX;
  static constexpr int TABB = 32 * 8;
  static constexpr int AUXB = GMAX * (TABB + 16);  // tables and mask records
  static size_t buf_bytes(int T) { return (size_t)T * ROWB + AUXB; }
  static size_t smem(int T) { return 2 * buf_bytes(T) + 64; }
};

// One coset of member set SH whose records start at srec[mb]: members j = 0.. in offset order.
template <int BT, int RB, int NTB, uint32_t SH>
__device__ __forceinline__ void coset_body(float4 (&acc)[1 << RB][BT / 2], const unsigned char* tb, int tid,
                                           const uint32_t (&soff)[BT / 2], const float2* stab, const uint4* srec,
                                           int mb, uint32_t xf0, int fsh) {
  constexpr int RPT = 1 << RB, NS = BT / 2, NM = __builtin_popcount(SH);
  constexpr int ROWB = BT * 8;
  uint32_t idx0[NM], fl[NM];
#pragma unroll
  for (int j = 0; j < NM; ++j) {
    const uint4 rec = srec[mb + j];
    idx0[j] = supp_bits(xf0, rec.z) | ((__popc(rec.y & xf0) & 1u) << 4);
    fl[j] = rec.w >> fsh;
  }
  const uint32_t klo = srec[mb].x & ((1u << NTB) - 1u);  // key: row-slot bits cleared
  const unsigned char* row0 = tb + (size_t)((uint32_t)tid ^ klo) * ROWB;
  constexpr int rstep = ROWB << NTB;  // row-slot stride: immediate load offsets
  const float2* tab = stab + mb * 32;
  // coefficient of member j (offset d) for the row slot i = s ^ d it feeds from source slot s
  float2 cf[RPT][NM];
#pragma unroll
  for (int s = 0; s < RPT; ++s)
#pragma unroll
    for (int d = 0; d < RPT; ++d) {
      if (!((SH >> d) & 1u)) continue;
      const int j = __builtin_popcount(SH & ((1u << d) - 1u));  // member index of offset d
      const int i = s ^ d;
      uint32_t idx = idx0[j];
      if (i & 1) idx ^= fl[j] & 31u;
      if (i & 2) idx ^= (fl[j] >> 5) & 31u;
      if (i & 4) idx ^= (fl[j] >> 10) & 31u;
      cf[s][j] = tab[j * 32 + (int)idx];
    }
  // chunk-outer: chunk k of every source row, then every multiply-add that reads it
#pragma unroll
  for (int k = 0; k < NS; ++k) {
    const unsigned char* rk = row0 + soff[k];
    float4 v[RPT];
#pragma unroll
    for (int s = 0; s < RPT; ++s) v[s] = *reinterpret_cast<const float4*>(rk + s * rstep);
#pragma unroll
    for (int s = 0; s < RPT; ++s)
#pragma unroll
      for (int d = 0; d < RPT; ++d) {
        if (!((SH >> d) & 1u)) continue;
        const int j = __builtin_popcount(SH & ((1u << d) - 1u));
        Slot<float>::mac(acc[s ^ d][k], cf[s][j].x, cf[s][j].y, v[s]);
      }
  }
}

template <int BT, int RB, bool CL, int NTB>
__global__ void __launch_bounds__(1 << NTB) k_apply_coset(ApplyParams p, const int4* __restrict__ chunks,
                                                     const uint32_t* __restrict__ counts, int nchunks,
                                                     const uint4* __restrict__ crec, const float2* __restrict__ ctab,
                                                     const float2* __restrict__ psi, float2* __restrict__ y) {
  using Cfg = CosetCfg<BT, RB>;
  using Sh = CosetShapes<RB>;
  using C = float2;
  using S = float4;
  constexpr int RPT = Cfg::RPT, ROWB = Cfg::ROWB, CH = Cfg::CH, NS = CH;
  constexpr int GMAX = Cfg::GMAX, TABB = Cfg::TABB;
  static_assert(CH >= 1 && RB >= 1 && RB <= 3, "coset variant: rows of >= 16 bytes, 2..8 rows per thread");
  constexpr int NT = 1 << NTB, T = RPT << NTB, TILEB = T * ROWB, BUFB = TILEB + Cfg::AUXB;
  extern __shared__ __align__(128) unsigned char sm[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm + 2 * BUFB);
  const C* __restrict__ t2 = static_cast<const C*>(p.m2_tab);
  const int tid = threadIdx.x, lane = tid & 31;
  const uint32_t crank = CL ? tma::cluster_rank() : 0u, csize = CL ? tma::cluster_size() : 1u;
  const uint32_t tile = blockIdx.x / csize;
  const int nmine = (int)crank < nchunks ? (nchunks - (int)crank + (int)csize - 1) / (int)csize : 0;
  const int n = p.n;
  const int rho = CH >= 8 ? (lane & 7) : (CH >= 2 ? ((lane * CH / 8) % CH) : 0);
  uint32_t soff[NS];
#pragma unroll
  for (int k = 0; k < NS; ++k) soff[k] = (uint32_t)(((k + rho) & (CH - 1)) * 16);
  constexpr int fsh = flip_shift(NTB);
  uint32_t xf[RPT];
#pragma unroll
  for (int i = 0; i < RPT; ++i) {
    const uint32_t xc = tile * (uint32_t)T + (uint32_t)(tid + i * NT);
    xf[i] = xc | ((uint32_t)((__popc(xc) + p.sector) & 1) << (n - 1));
  }
  S acc[RPT][NS];
#pragma unroll
  for (int i = 0; i < RPT; ++i)
#pragma unroll
    for (int k = 0; k < NS; ++k) acc[i][k] = Slot<float>::zero();
  auto mac_row = [&](S* a, float cr, float ci, const unsigned char* tb, uint32_t sr) {
    const unsigned char* row = tb + (size_t)sr * ROWB;
#pragma unroll
    for (int k = 0; k < NS; ++k) Slot<float>::mac(a[k], cr, ci, *reinterpret_cast<const S*>(row + soff[k]));
  };

  if (tid == 0) {
    tma::mbar_init(&bar[0], 1);
    tma::mbar_init(&bar[1], 1);
    tma::fence_mbar_init();
  }
  __syncthreads();
  const unsigned char* src = reinterpret_cast<const unsigned char*>(psi);
  auto issue = [&](int q) {
    if (tid == 0) {
      const int b = q & 1;
      const int4 gr = __ldg(&chunks[(int)crank + q * (int)csize]);
      const uint32_t part = tile ^ ((uint32_t)gr.x & 0x7fffffffu);
      const uint32_t nm = (uint32_t)(gr.z - gr.y);
      unsigned char* buf = sm + b * BUFB;
      tma::expect_tx(&bar[b], (uint32_t)TILEB + nm * (uint32_t)(TABB + 16));
      tma::bulk_load(buf, src + (size_t)part * TILEB, (uint32_t)TILEB, &bar[b]);
      if (nm) {
        tma::bulk_load(buf + TILEB, ctab + (size_t)gr.y * 32, nm * TABB, &bar[b]);
        tma::bulk_load(buf + TILEB + GMAX * TABB, crec + gr.y, nm * 16u, &bar[b]);
      }
    }
  };
  if (nmine > 0) issue(0);
  bool failed = false;
  int g = 0;
  for (; g < nmine; ++g) {
    if (g + 1 < nmine) issue(g + 1);
    const bool ok = tma::wait_bounded(&bar[g & 1], (g >> 1) & 1, tma::kWaitPolls);
    const int c = (int)crank + g * (int)csize;
    const int4 gr = __ldg(&chunks[c]);
    const unsigned char* tb = sm + (g & 1) * BUFB;
    if (ok) {
      const C* stab = reinterpret_cast<const C*>(tb + TILEB);
      const uint4* srec = reinterpret_cast<const uint4*>(tb + TILEB + GMAX * TABB);
      const uint32_t cn = __ldg(&counts[c]);
      const int nm = gr.z - gr.y;
      int mb = 0;
      for (uint32_t q = 0; q < (cn & 0xffu); ++q, mb += __builtin_popcount(Sh::s0))
        coset_body<BT, RB, NTB, Sh::s0>(acc, tb, tid, soff, stab, srec, mb, xf[0], fsh);
      if constexpr (Sh::n > 1)
        for (uint32_t q = 0; q < ((cn >> 8) & 0xffu); ++q, mb += __builtin_popcount(Sh::s1))
          coset_body<BT, RB, NTB, Sh::s1>(acc, tb, tid, soff, stab, srec, mb, xf[0], fsh);
      if constexpr (Sh::n > 2)
        for (uint32_t q = 0; q < ((cn >> 16) & 0xffu); ++q, mb += __builtin_popcount(Sh::s2))
          coset_body<BT, RB, NTB, Sh::s2>(acc, tb, tid, soff, stab, srec, mb, xf[0], fsh);
      // single masks: one partner row per row slot
      for (; mb < nm; ++mb) {
        const uint4 rec = srec[mb];
        const uint32_t lo = rec.x & (uint32_t)(T - 1);
        const uint32_t idx0 = supp_bits(xf[0], rec.z) | ((__popc(rec.y & xf[0]) & 1u) << 4);
        const uint32_t fl = rec.w >> fsh;
        const C* tab = stab + mb * 32;
#pragma unroll
        for (int i = 0; i < RPT; ++i) {
          uint32_t idx = idx0;
          if (i & 1) idx ^= fl & 31u;
          if (i & 2) idx ^= (fl >> 5) & 31u;
          if (i & 4) idx ^= (fl >> 10) & 31u;
          const C cf = tab[idx];
          mac_row(acc[i], cf.x, cf.y, tb, (uint32_t)(tid + i * NT) ^ lo);
        }
      }
      const int k2e = gr.w >> 16;
      for (int k = gr.w & 0xffff; k < k2e; ++k) {
        const uint4 rec = __ldg(&p.m2_rec[k]);
        const uint32_t lo = rec.x & (uint32_t)(T - 1);
#pragma unroll
        for (int i = 0; i < RPT; ++i) {
          float cr2, ci2;
          pc2_coef<C, float>(t2, k, n, rec, xf[i], cr2, ci2);
          mac_row(acc[i], cr2, ci2, tb, (uint32_t)(tid + i * NT) ^ lo);
        }
      }
      if ((uint32_t)gr.x == 0x80000000u) {
#pragma unroll
        for (int i = 0; i < RPT; ++i)
          mac_row(acc[i], diag_coef<float>(static_cast<const float*>(p.wd), n, xf[i]), 0.f, tb, (uint32_t)(tid + i * NT));
      }
    }
    if (__syncthreads_or(!ok)) {
      failed = true;
      break;
    }
  }
  if (failed) {
    if (tid == 0) {
      atomicOr(p.status, 4);
      tma::wait_bounded(&bar[g & 1], (g >> 1) & 1, tma::kDrainPolls);
      if (g + 1 < nmine) tma::wait_bounded(&bar[(g + 1) & 1], ((g + 1) >> 1) & 1, tma::kDrainPolls);
    }
    __syncthreads();
  }
  // straight to y, or staged in shared memory for the cluster reduction or the Lanczos epilogue
  const bool stage = CL || p.ep_part != nullptr;
  unsigned char* dst = stage ? sm : reinterpret_cast<unsigned char*>(y) + (size_t)tile * TILEB;
#pragma unroll
  for (int i = 0; i < RPT; ++i) {
    unsigned char* out = dst + (size_t)(tid + i * NT) * ROWB;
#pragma unroll
    for (int k = 0; k < NS; ++k) *reinterpret_cast<S*>(out + soff[k]) = acc[i][k];
  }
  if constexpr (CL) {
    tma::cluster_sync();
    const int units = TILEB / 16 / (int)csize;
    const uint32_t base = tma::saddr(sm) + crank * (uint32_t)units * 16u;
    store_units<float4, ROWB>(
        p, units, NT, (size_t)tile * TILEB + (size_t)crank * units * 16, y,
        [&](int u) {
          float4 sum = tma::ld_cluster(tma::map_rank(base + 16u * u, 0), float4{});
          for (uint32_t r = 1; r < csize; ++r) {
            const float4 v = tma::ld_cluster(tma::map_rank(base + 16u * u, r), float4{});
            sum.x += v.x; sum.y += v.y; sum.z += v.z; sum.w += v.w;
          }
          return sum;
        },
        sm + BUFB);
    tma::cluster_sync();
  } else if (stage) {
    __syncthreads();
    store_units<float4, ROWB>(p, TILEB / 16, NT, (size_t)tile * TILEB, y,
                              [&](int u) { return reinterpret_cast<const float4*>(sm)[u]; }, sm + BUFB);
  }
}

template <int BT, int RB, int NTB>
int launch_coset_ntb(const ApplyParams& p, const CosetLayout* L, const void* psi, void* y, cudaStream_t st, int cs) {
  using Cfg = CosetCfg<BT, RB>;
  constexpr int T = Cfg::RPT << NTB;
  const int64_t ntiles = p.D / T;
  const size_t smem = Cfg::smem(T);
  if (smem > kMaxSmemPerCta) return 1;
  if (p.ep_part && ntiles * cs > p.ep_cap) {
    set_error("apply_H: %lld CTAs exceed the epilogue buffer (%lld)", (long long)(ntiles * cs), (long long)p.ep_cap);
    return SYK_EINVAL;
  }
  SYK_TRY(ensure_smem_limit((const void*)k_apply_coset<BT, RB, false, NTB>, (int)smem));
  SYK_TRY(ensure_smem_limit((const void*)k_apply_coset<BT, RB, true, NTB>, (int)smem));
  const float2* x = static_cast<const float2*>(psi);
  float2* out = static_cast<float2*>(y);
  if (cs == 1) {
    k_apply_coset<BT, RB, false, NTB><<<(unsigned)ntiles, 1u << NTB, smem, st>>>(p, L->chunks, L->counts, L->nchunks,
                                                                             L->rec, L->t32, x, out);
  } else {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(ntiles * cs), 1, 1);
    cfg.blockDim = dim3(1u << NTB, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)cs;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    SYK_CUDA_CHECK(cudaLaunchKernelEx(&cfg, k_apply_coset<BT, RB, true, NTB>, p, (const int4*)L->chunks,
                                      (const uint32_t*)L->counts, L->nchunks, (const uint4*)L->rec,
                                      (const float2*)L->t32, x, out));
  }
  count_launch();
  count_matvec(kMvCoset);
  SYK_CUDA_CHECK(cudaGetLastError());
  return SYK_OK;
}

// Launches k_apply_coset<BT, RB> with 2^ntb-thread CTAs (ntb 6 or 7) in clusters of cs;
// returns 1 if it does not apply (tile larger than the sector or than shared memory, or
// the layout is not built and no_alloc forbids building it).
template <int BT, int RB>
int launch_coset(const ApplyParams& p, const void* psi, void* y, cudaStream_t st, int ntb, int cs) {
  using Cfg = CosetCfg<BT, RB>;
  const int T = Cfg::RPT << ntb;
  if (p.D < T || ntb < 6 || ntb > 7 || !coset_fits(BT, RB, ntb)) return 1;
  int tb = 0;
  while ((1 << tb) < T) ++tb;
  const CosetLayout* L = nullptr;
  const int lr = coset_layout(p.terms, tb, RB, Cfg::GMAX, !p.no_alloc, &L);
  if (lr != SYK_OK) return lr > 0 ? 1 : lr;
  return ntb == 6 ? launch_coset_ntb<BT, RB, 6>(p, L, psi, y, st, cs) : launch_coset_ntb<BT, RB, 7>(p, L, psi, y, st, cs);
}

}  // namespace

bool coset_var_ok(int dtype, int64_t batch, int var) {
  if (dtype != SYK_C64) return var == 0;
  if (batch == 16) return var <= 2;
  if (batch == 8 || batch == 4) return var == 0 || var == 2 || var == 3;
  return var == 0;
}

bool coset_fits(int64_t batch, int var, int ntb) {
  if (ntb < 6 || ntb > 7) return false;
  const size_t T = size_t(1) << (var + ntb);
  return 2 * (T * size_t(batch) * 8 + CosetCfg<16, 1>::AUXB) + 64 <= kMaxSmemPerCta;
}

int launch_coset_var(const ApplyParams& p, int64_t batch, const void* psi, void* y, cudaStream_t st, int var, int ntb,
                     int cs) {
  if (reinterpret_cast<uintptr_t>(psi) & 15 || reinterpret_cast<uintptr_t>(y) & 15) return 1;
  switch (batch * 8 + var) {
    case 16 * 8 + 1: return launch_coset<16, 1>(p, psi, y, st, ntb, cs);
    case 16 * 8 + 2: return launch_coset<16, 2>(p, psi, y, st, ntb, cs);
    case 8 * 8 + 2: return launch_coset<8, 2>(p, psi, y, st, ntb, cs);
    case 8 * 8 + 3: return launch_coset<8, 3>(p, psi, y, st, ntb, cs);
    case 4 * 8 + 2: return launch_coset<4, 2>(p, psi, y, st, ntb, cs);
    case 4 * 8 + 3: return launch_coset<4, 3>(p, psi, y, st, ntb, cs);
    default: return 1;
  }
}

}  // namespace syk
