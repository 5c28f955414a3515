// K1 variant for ONE complex64 state: y = H psi in one parity sector (Supp. Sec. I.B).
//
// Tiles, chunks, staging and the cluster split are those of k_apply_tiled (syk_apply.cu): a
// thread owns RPT = 8 rows r_i = tid + i NT of its tile, and a popcount-4 mask with low part
// lo sends row slot i to partner row (tid ^ lo_t) + ((i ^ H) << ntb), lo_t = lo mod NT,
// H = lo >> ntb.  With one state a row x mask pair carries only 4 FFMA, so the integer work
// around it decides the speed.  Here H (the same for the whole warp: it comes from the mask)
// selects one of 8 fully unrolled bodies in which every partner-row load has a compile-time
// offset from one per-mask base, and the 8 table indices are idx0 ^ F_i with the F_i formed
// once per mask from the three row-bit flip patterns.  Per row x mask: one XOR, two shared
// loads, 4 FFMA.
#include <cuda_runtime.h>

#include <cstdint>

#include "syk_tile.cuh"

#ifndef SYK_GMAX
#define SYK_GMAX 16
#endif

namespace syk {
namespace {

struct OneCfg {
  static constexpr int RPT = 8;
  static constexpr int GMAX = SYK_GMAX;
  static constexpr int TABB = 32 * 8;
  static constexpr int AUXB = GMAX * (TABB + 16);
  static size_t smem(int T) { return 2 * ((size_t)T * 8 + AUXB) + 64; }
};

// the 8 row slots of one mask whose low part maps slot i to partner slot i ^ H
template <int H, int NTB>
__device__ __forceinline__ void one_body(float2 (&acc)[8], const float2* __restrict__ rb, const float2* __restrict__ tab,
                                         uint32_t idx0, const uint32_t (&F)[8]) {
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const float2 v = rb[(i ^ H) << NTB];
    const float2 c = tab[idx0 ^ F[i]];
    acc[i].x = fmaf(c.x, v.x, fmaf(-c.y, v.y, acc[i].x));
    acc[i].y = fmaf(c.x, v.y, fmaf(c.y, v.x, acc[i].y));
  }
}

template <int NTB>
__device__ __forceinline__ void one_mask(float2 (&acc)[8], const float2* rb, const float2* tab, uint32_t idx0,
                                         const uint32_t (&F)[8], uint32_t H) {
  switch (H) {
    case 0: one_body<0, NTB>(acc, rb, tab, idx0, F); break;
    case 1: one_body<1, NTB>(acc, rb, tab, idx0, F); break;
    case 2: one_body<2, NTB>(acc, rb, tab, idx0, F); break;
    case 3: one_body<3, NTB>(acc, rb, tab, idx0, F); break;
    case 4: one_body<4, NTB>(acc, rb, tab, idx0, F); break;
    case 5: one_body<5, NTB>(acc, rb, tab, idx0, F); break;
    case 6: one_body<6, NTB>(acc, rb, tab, idx0, F); break;
    default: one_body<7, NTB>(acc, rb, tab, idx0, F); break;
  }
}

// CL: the CTAs of a cluster share one tile and split its mask chunks round-robin; their
// partial sums are reduced in a fixed rank order through distributed shared memory.
template <int NTB, bool CL>
__global__ void __launch_bounds__(1 << NTB) k_apply_one(ApplyParams p, const int4* __restrict__ groups, int ngroups,
                                                    const float2* __restrict__ psi, float2* __restrict__ y) {
  constexpr int RPT = OneCfg::RPT, GMAX = OneCfg::GMAX, TABB = OneCfg::TABB;
  constexpr int NT = 1 << NTB, T = RPT << NTB, TILEB = T * 8, BUFB = TILEB + OneCfg::AUXB;
  constexpr int fsh = flip_shift(NTB);  // flip patterns of row bits ntb, ntb+1, ntb+2
  extern __shared__ __align__(128) unsigned char sm[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm + 2 * BUFB);
  const float2* __restrict__ t4 = static_cast<const float2*>(p.m4_tab);
  const float2* __restrict__ t2 = static_cast<const float2*>(p.m2_tab);
  const int tid = threadIdx.x;
  const uint32_t crank = CL ? tma::cluster_rank() : 0u, csize = CL ? tma::cluster_size() : 1u;
  const uint32_t tile = blockIdx.x / csize;
  const int nmine = (int)crank < ngroups ? (ngroups - (int)crank + (int)csize - 1) / (int)csize : 0;
  const int n = p.n;
  uint32_t xf[RPT];
#pragma unroll
  for (int i = 0; i < RPT; ++i) {
    const uint32_t xc = tile * (uint32_t)T + (uint32_t)(tid + i * NT);
    xf[i] = xc | ((uint32_t)((__popc(xc) + p.sector) & 1) << (n - 1));
  }
  float2 acc[RPT];
#pragma unroll
  for (int i = 0; i < RPT; ++i) acc[i] = make_float2(0.f, 0.f);

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
      const int4 gr = __ldg(&groups[(int)crank + q * (int)csize]);
      const uint32_t part = tile ^ ((uint32_t)gr.x & 0x7fffffffu);
      const uint32_t nm = (uint32_t)(gr.z - gr.y);
      unsigned char* buf = sm + b * BUFB;
      tma::expect_tx(&bar[b], (uint32_t)TILEB + nm * (uint32_t)(TABB + 16));
      tma::bulk_load(buf, src + (size_t)part * TILEB, (uint32_t)TILEB, &bar[b]);
      if (nm) {
        tma::bulk_load(buf + TILEB, t4 + (size_t)gr.y * 32, nm * TABB, &bar[b]);
        tma::bulk_load(buf + TILEB + GMAX * TABB, p.m4_rec + gr.y, nm * 16u, &bar[b]);
      }
    }
  };
  if (nmine > 0) issue(0);
  bool failed = false;
  int g = 0;
  for (; g < nmine; ++g) {
    if (g + 1 < nmine) issue(g + 1);
    const bool ok = tma::wait_bounded(&bar[g & 1], (g >> 1) & 1, tma::kWaitPolls);
    const int4 gr = __ldg(&groups[(int)crank + g * (int)csize]);
    const unsigned char* tb = sm + (g & 1) * BUFB;
    if (ok) {
      const float2* stab = reinterpret_cast<const float2*>(tb + TILEB);
      const uint4* srec = reinterpret_cast<const uint4*>(tb + TILEB + GMAX * TABB);
      const float2* rows = reinterpret_cast<const float2*>(tb);
      const int nm = gr.z - gr.y;
      for (int kk = 0; kk < nm; ++kk) {
        const uint4 rec = srec[kk];
        const uint32_t lo = rec.x & (uint32_t)(T - 1);
        const uint32_t idx0 = supp_bits(xf[0], rec.z) | ((__popc(rec.y & xf[0]) & 1u) << 4);
        const uint32_t fl = rec.w >> fsh;
        uint32_t F[8];
        F[0] = 0u;
        F[1] = fl & 31u;
        F[2] = (fl >> 5) & 31u;
        F[3] = F[1] ^ F[2];
        F[4] = (fl >> 10) & 31u;
        F[5] = F[4] ^ F[1];
        F[6] = F[4] ^ F[2];
        F[7] = F[4] ^ F[3];
        one_mask<NTB>(acc, rows + ((uint32_t)tid ^ (lo & (NT - 1))), stab + kk * 32, idx0, F, lo >> NTB);
      }
      // popcount-2 masks and the diagonal: general row addresses (few per tile)
      const int k2e = gr.w >> 16;
      for (int k = gr.w & 0xffff; k < k2e; ++k) {
        const uint4 rec = __ldg(&p.m2_rec[k]);
        const uint32_t lo = rec.x & (uint32_t)(T - 1);
#pragma unroll
        for (int i = 0; i < RPT; ++i) {
          float cr, ci;
          pc2_coef<float2, float>(t2, k, n, rec, xf[i], cr, ci);
          const float2 v = rows[(uint32_t)(tid + i * NT) ^ lo];
          cmac(acc[i], cr, ci, v);
        }
      }
      if ((uint32_t)gr.x == 0x80000000u) {
#pragma unroll
        for (int i = 0; i < RPT; ++i) {
          const float d = diag_coef<float>(static_cast<const float*>(p.wd), n, xf[i]);
          const float2 v = rows[tid + i * NT];
          acc[i].x = fmaf(d, v.x, acc[i].x);
          acc[i].y = fmaf(d, v.y, acc[i].y);
        }
      }
    }
    // every thread is done with buffer g&1 before it is refilled; agree on failure
    if (__syncthreads_or(!ok)) {
      failed = true;
      break;
    }
  }
  if (failed) {
    // drain: let any copy still in flight land before the buffers are reused or the CTA exits
    if (tid == 0) {
      atomicOr(p.status, 4);
      tma::wait_bounded(&bar[g & 1], (g >> 1) & 1, tma::kDrainPolls);
      if (g + 1 < nmine) tma::wait_bounded(&bar[(g + 1) & 1], ((g + 1) >> 1) & 1, tma::kDrainPolls);
    }
    __syncthreads();
  }
  // straight to y, or staged in shared memory for the cluster reduction or the Lanczos epilogue
  const bool stage = CL || p.ep_part != nullptr;
  float2* dst = stage ? reinterpret_cast<float2*>(sm) : y + (size_t)tile * T;
#pragma unroll
  for (int i = 0; i < RPT; ++i) dst[tid + i * NT] = acc[i];
  if constexpr (CL) {
    tma::cluster_sync();
    const int units = TILEB / 16 / (int)csize;
    const uint32_t base = tma::saddr(sm) + crank * (uint32_t)units * 16u;
    store_units<float4, 8>(
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
    tma::cluster_sync();  // no CTA leaves while others still read its shared memory
  } else if (stage) {
    __syncthreads();
    store_units<float4, 8>(p, TILEB / 16, NT, (size_t)tile * TILEB, y,
                           [&](int u) { return reinterpret_cast<const float4*>(sm)[u]; }, sm + BUFB);
  }
}

template <int NTB>
int launch_one_ntb(const ApplyParams& p, const int4* groups, int ng, int cs, const void* psi, void* y,
                   cudaStream_t st) {
  constexpr int T = OneCfg::RPT << NTB;
  const int64_t ntiles = p.D / T;
  const size_t smem = OneCfg::smem(T);
  SYK_TRY(ensure_smem_limit((const void*)k_apply_one<NTB, false>, (int)smem));
  SYK_TRY(ensure_smem_limit((const void*)k_apply_one<NTB, true>, (int)smem));
  const float2* x = static_cast<const float2*>(psi);
  float2* out = static_cast<float2*>(y);
  if (cs == 1) {
    k_apply_one<NTB, false><<<(unsigned)ntiles, 1u << NTB, smem, st>>>(p, groups, ng, x, out);
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
    SYK_CUDA_CHECK(cudaLaunchKernelEx(&cfg, k_apply_one<NTB, true>, p, groups, ng, x, out));
  }
  count_launch();
  count_matvec(kMvTiled);
  SYK_CUDA_CHECK(cudaGetLastError());
  return SYK_OK;
}

}  // namespace

int launch_one_state(const ApplyParams& p, const int4* groups, int ng, int ntb, int cs, const void* psi, void* y,
                     cudaStream_t st) {
  switch (ntb) {
    case 6: return launch_one_ntb<6>(p, groups, ng, cs, psi, y, st);
    case 7: return launch_one_ntb<7>(p, groups, ng, cs, psi, y, st);
    case 8: return launch_one_ntb<8>(p, groups, ng, cs, psi, y, st);
    default:
      set_error("apply_H: one-state kernel: CTA width 2^%d not built", ntb);
      return SYK_EINVAL;
  }
}

}  // namespace syk
