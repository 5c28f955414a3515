// K1: y = H psi in one parity sector, matrix-free (Supp. Sec. I.B), and
// K5: y = chi_i psi (Supp. Sec. I.A).
//
// Every output row x (compact index) sums over all X-masks, with each mask
// coefficient c_m(x) evaluated on the fly from the grouped tables built on the
// host (see syk_terms.cpp):
//   y[x][b] = c_0(x) psi[x][b] + sum_{popcount(m)=2} c_m(x) psi[x^m][b]
//                              + sum_{popcount(m)=4} c_m(x) psi[x^m][b].
// The full spin index of x (needed for the sign parities) is
//   xf = x | ((popcount(x) + sector) & 1) << (n-1);
// the gather index is x ^ (m & (D-1)) because every X-mask has even popcount.
//
// k_apply_tiled (main path, batch of 1, 2, 4, 8 or 16 columns): a CTA owns a
// tile of T = 256 * RPT consecutive rows.  Masks are walked in groups sharing
// the compact-mask bits above the tile, so each group reads ONE partner tile
// psi[tile ^ h]; that tile (T * BT contiguous elements) is staged in shared
// memory by a bulk asynchronous copy (cp.async.bulk + mbarrier), double
// buffered so the next group's tile streams in during the current group's
// arithmetic.  A thread owns RPT rows that differ in the compact bits just above
// the thread index (bits 6..10 depending on the CTA width); the table index of a
// popcount-4 mask for those rows follows from the first row's by XOR with
// per-mask flip patterns, so the bit extraction is done once per mask.  Small
// sectors or single states would leave SMs idle, so the mask chunks of one tile are
// then split round-robin over a thread-block cluster of up to 8 CTAs, whose
// partial sums are reduced in a fixed order through distributed shared memory.  Rows wider than 16 bytes are read in 16-byte chunks in a lane-rotated
// order so that the 32 lanes of a warp hit distinct shared-memory banks.
// k_apply_rows (fallback: any batch, any alignment, small sectors): one thread
// per row, gathers straight from global memory.
#include <cuda_runtime.h>

#include <atomic>
#include <type_traits>
#include <map>
#include <mutex>
#include <string>
#include <cstdio>
#include <cstring>

#include <algorithm>
#include <vector>

#include "syk_tile.cuh"

// Unroll factor of the per-chunk mask loop of the tiled matvec (build-time knob).
#ifndef SYK_MASK_UNROLL
#define SYK_MASK_UNROLL 1
#endif
// Masks staged per chunk, and rows per thread of the 8- and 16-state complex64 kernels.
#ifndef SYK_GMAX
#define SYK_GMAX 16
#endif
#ifndef SYK_RPT_C64_B8
#define SYK_RPT_C64_B8 4
#endif
#ifndef SYK_RPT_C64_B16
#define SYK_RPT_C64_B16 2
#endif
// One table lookup per mask for one-state rows when the row-slot bits miss the support.
#ifndef SYK_SHARED_COEF
#define SYK_SHARED_COEF 1
#endif
// One-state complex64 launches use k_apply_one (syk_apply_one.cu); 0 keeps k_apply_tiled<float, 1>.
#ifndef SYK_ONE_STATE_KERNEL
#define SYK_ONE_STATE_KERNEL 1
#endif
#define SYK_PRAGMA(x) _Pragma(#x)
#define SYK_UNROLL(n) SYK_PRAGMA(unroll n)

namespace syk {

// Tile configuration chosen by the autotuner per (N, dtype, batch): CTA width 2^ntb,
// cluster size cs and kernel variant var (0: k_apply_tiled; 1..3: k_apply_coset with
// 2^var rows per thread).  Absent entries use the built-in heuristic.
struct TileChoice {
  int ntb, cs;
  double ms;
  int var = 0;
};
static std::atomic<int> g_c128_arith{kC128DoubleFloat};
static std::mutex g_tune_mtx;
static std::map<uint64_t, TileChoice> g_tune;
static uint64_t tune_key(int N, int dtype, int64_t batch) {
  return (uint64_t)N | ((uint64_t)dtype << 8) | ((uint64_t)batch << 16);
}
static bool tile_choice_lookup(int N, int dtype, int64_t batch, TileChoice* out) {
  std::lock_guard<std::mutex> lk(g_tune_mtx);
  auto it = g_tune.find(tune_key(N, dtype, batch));
  if (it == g_tune.end()) return false;
  *out = it->second;
  return true;
}
static void tile_choice_set(int N, int dtype, int64_t batch, TileChoice c) {
  std::lock_guard<std::mutex> lk(g_tune_mtx);
  g_tune[tune_key(N, dtype, batch)] = c;
  bump_graph_epoch();  // captured matvec launches carry the old tile shape
}

namespace {

template <typename R, int BT>
__global__ void __launch_bounds__(128) k_apply_rows(ApplyParams p, const typename CT<R>::T* __restrict__ psi,
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
      const uint32_t idx = supp_bits(xf, rec.z) | ((__popc(rec.y & xf) & 1u) << 4);
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
  blocks = std::min<int64_t>(blocks, (int64_t)sm_count() * 64);
  k_apply_rows<R, BT><<<(unsigned)blocks, threads, 0, st>>>(p, static_cast<const C*>(psi), static_cast<C*>(y), ld, b0);
  count_launch();
  count_matvec(kMvRows);
}

template <typename R>
int try_tiled(const ApplyParams& p, const void* psi, void* y, int64_t batch, cudaStream_t st);

// The Lanczos epilogue (see ApplyParams) for launches without one (the row kernel):
// y[e] *= ep_scale[b]; per-block conj(ep_u) . y sums per column.  blockDim = B * k, so thread
// t always handles column t % B; complex64 products and short sums in FP32, flushed to FP64.
template <typename R>
__global__ void k_epilogue(ApplyParams p, typename CT<R>::T* __restrict__ y, int64_t total, int B) {
  using C = typename CT<R>::T;
  extern __shared__ double2 red[];
  const int b = threadIdx.x % B;
  const R s = p.ep_scale ? R(p.ep_scale[b]) : R(1);
  const C* __restrict__ u = static_cast<const C*>(p.ep_u);
  double re = 0.0, im = 0.0;
  R fr = R(0), fi = R(0);
  int cnt = 0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    C v = y[e];
    v.x *= s;
    v.y *= s;
    y[e] = v;
    const C w = u[e];
    fr = fma(w.x, v.x, fma(w.y, v.y, fr));
    fi = fma(w.x, v.y, fma(-w.y, v.x, fi));
    if (++cnt == 16) {
      re += fr;
      im += fi;
      fr = fi = R(0);
      cnt = 0;
    }
  }
  red[threadIdx.x] = make_double2(re + fr, im + fi);
  __syncthreads();
  if ((int)threadIdx.x < B) {
    double2 r = make_double2(0.0, 0.0);
    for (int t = threadIdx.x; t < (int)blockDim.x; t += B) {
      r.x += red[t].x;
      r.y += red[t].y;
    }
    p.ep_part[(size_t)blockIdx.x * B + threadIdx.x] = r;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) *p.ep_nblk = (int)gridDim.x;
}

template <typename R>
int launch_epilogue(const ApplyParams& p, void* y, int64_t batch, cudaStream_t st) {
  const int bdim = int(batch) * std::max(1, int(256 / batch));
  const int64_t total = p.D * batch;
  const int64_t blocks = std::min<int64_t>(std::min<int64_t>((total + bdim - 1) / bdim, 2 * sm_count()), p.ep_cap);
  k_epilogue<R><<<(unsigned)blocks, bdim, bdim * sizeof(double2), st>>>(p, static_cast<typename CT<R>::T*>(y), total,
                                                                        int(batch));
  count_launch();
  SYK_CUDA_CHECK(cudaGetLastError());
  return SYK_OK;
}

template <typename R>
int launch_apply_T(const ApplyParams& p, const void* psi, void* y, int64_t batch, cudaStream_t st) {
  const int rc = try_tiled<R>(p, psi, y, batch, st);
  if (rc <= 0) return rc;  // launched (0) or failed (< 0)
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
  if (p.ep_part) return launch_epilogue<R>(p, y, batch, st);
  return SYK_OK;
}

// ---------------------------------------------------------------- tiled matvec
template <typename R, int BT>
struct TileCfg {
  using C = typename CT<R>::T;
  // rows per thread: more rows share one table-index computation, fewer leave room
  // for more resident warps
  static constexpr int RPT = std::is_same<R, float>::value
                                 ? (BT == 1 ? 8 : BT <= 4 ? 4 : BT == 8 ? SYK_RPT_C64_B8 : SYK_RPT_C64_B16)
                                 : (BT == 1 ? 4 : BT <= 4 ? 2 : 1);
  static constexpr int ROWB = BT * (int)sizeof(C);
  static constexpr int CH = ROWB >= 16 ? ROWB / 16 : 0;  // 16-byte chunks per row
  static constexpr int NS = CH ? CH : 1;
  // each buffer stages the partner tile plus the records and 32-entry coefficient
  // tables of up to GMAX popcount-4 masks
  static constexpr int GMAX = SYK_GMAX;
  static constexpr int TABB = 32 * (int)sizeof(C);
  static constexpr int AUXB = GMAX * (TABB + 16);
  static size_t buf_bytes(int T) { return (size_t)T * ROWB + AUXB; }
  static size_t smem(int T) { return 2 * buf_bytes(T) + 64; }
};

// ntb = log2(threads per CTA) in 6..8; a CTA owns T = RPT << ntb rows.  CL: launched
// as clusters that split a tile's mask chunks (otherwise one CTA per tile).
template <typename R, int BT, bool CL>
__global__ void __launch_bounds__(256) k_apply_tiled(ApplyParams p, const int4* __restrict__ groups, int ngroups,
                                                     int ntb, const void* __restrict__ psi, void* __restrict__ y) {
  using Cfg = TileCfg<R, BT>;
  using C = typename CT<R>::T;
  using S = typename std::conditional<Cfg::CH == 0, C, typename Slot<R>::T>::type;
  using Out = typename std::conditional<Cfg::CH == 0, C, typename Slot<R>::Out>::type;
  static_assert(sizeof(Out) == sizeof(S), "output rows have the layout of the staged rows");
  constexpr int RPT = Cfg::RPT, ROWB = Cfg::ROWB, CH = Cfg::CH, NS = Cfg::NS;
  constexpr int GMAX = Cfg::GMAX, TABB = Cfg::TABB;
  const int NT = 1 << ntb, T = RPT << ntb, TILEB = T * ROWB, BUFB = TILEB + Cfg::AUXB;
  extern __shared__ __align__(128) unsigned char sm[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm + 2 * BUFB);
  const C* __restrict__ t4 = tab4<R>(p);
  const C* __restrict__ t2 = tab2<R>(p);
  const int tid = threadIdx.x, lane = tid & 31;
  // the CTAs of a cluster share one tile and split its mask chunks round-robin
  const uint32_t crank = CL ? tma::cluster_rank() : 0u, csize = CL ? tma::cluster_size() : 1u;
  const uint32_t tile = blockIdx.x / csize;
  const int nmine = (int)crank < ngroups ? (ngroups - (int)crank + (int)csize - 1) / (int)csize : 0;
  const int n = p.n;
  // lane-rotated chunk order: lanes reading the same slot of different rows hit distinct banks
  const int rho = CH >= 8 ? (lane & 7) : (CH >= 2 ? ((lane * CH / 8) % CH) : 0);
  uint32_t soff[NS];
#pragma unroll
  for (int k = 0; k < NS; ++k) soff[k] = CH ? (uint32_t)(((k + rho) & (CH - 1)) * 16) : 0u;
  const int fsh = flip_shift(ntb);  // flip patterns of row bits ntb, ntb+1, ntb+2
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
    for (int k = 0; k < NS; ++k) {
      if constexpr (CH == 0) acc[i][k] = make_c<R>(R(0), R(0));
      else acc[i][k] = Slot<R>::zero();
    }

  // y_row += c * psi_tile[sr] for this thread's row slot i
  auto mac_row = [&](S* a, const C c, const unsigned char* tb, uint32_t sr) {
    if constexpr (CH == 0) {
      const C v = reinterpret_cast<const C*>(tb)[sr];
      cmac(a[0], c.x, c.y, v);
    } else {
      const unsigned char* row = tb + (size_t)sr * ROWB;
#pragma unroll
      for (int k = 0; k < NS; ++k) Slot<R>::mac(a[k], c, *reinterpret_cast<const S*>(row + soff[k]));
    }
  };

  if (tid == 0) {
    tma::mbar_init(&bar[0], 1);
    tma::mbar_init(&bar[1], 1);
    tma::fence_mbar_init();
  }
  __syncthreads();
  const unsigned char* src = reinterpret_cast<const unsigned char*>(psi);
  // one transaction per chunk: partner tile psi[tile ^ h], then the chunk's tables and records
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
  int g = 0;  // index among this CTA's chunks
  for (; g < nmine; ++g) {
    if (g + 1 < nmine) issue(g + 1);
    const bool ok = tma::wait_bounded(&bar[g & 1], (g >> 1) & 1, tma::kWaitPolls);
    const int4 gr = __ldg(&groups[(int)crank + g * (int)csize]);
    const unsigned char* tb = sm + (g & 1) * BUFB;
    if (ok) {
      // popcount-4 masks of this chunk: records and tables are in shared memory
      const C* stab = reinterpret_cast<const C*>(tb + TILEB);
      const uint4* srec = reinterpret_cast<const uint4*>(tb + TILEB + GMAX * TABB);
      const int nm = gr.z - gr.y;
      SYK_UNROLL(SYK_MASK_UNROLL)
      for (int kk = 0; kk < nm; ++kk) {
        const uint4 rec = srec[kk];
        const uint32_t lo = rec.x & (uint32_t)(T - 1);
        const uint32_t idx0 = supp_bits(xf[0], rec.z) | ((__popc(rec.y & xf[0]) & 1u) << 4);
        const uint32_t fl = rec.w >> fsh;
        const C* tab = stab + kk * 32;
        if constexpr (CH == 0 && SYK_SHARED_COEF && std::is_same<R, float>::value) {
          // one-state rows (8 bytes): the table lookup costs as much shared-memory traffic as
          // the row itself.  When no row-slot bit of this thread touches the mask's support
          // (flip bits 0..3 of every row bit clear; the same for the whole warp), every row
          // slot uses the same table entry up to the sign (flip bit 4), so look it up once.
          constexpr uint32_t used = RPT >= 8 ? 0x7fffu : RPT >= 4 ? 0x3ffu : RPT >= 2 ? 0x1fu : 0u;
          if ((fl & used & 0x3def) == 0u) {  // 0x3def: bits 0..3 of each 5-bit flip group
            const C cf = tab[idx0];
#pragma unroll
            for (int i = 0; i < RPT; ++i) {
              uint32_t sg = 0u;
              if (i & 1) sg ^= fl << 27;
              if (i & 2) sg ^= fl << 22;
              if (i & 4) sg ^= fl << 17;
              sg &= 0x80000000u;  // flip bit 4 of the row bits' groups, moved to the sign bit
              const float cr = __int_as_float(__float_as_int(cf.x) ^ (int)sg);
              const float ci = __int_as_float(__float_as_int(cf.y) ^ (int)sg);
              mac_row(acc[i], make_float2(cr, ci), tb, (uint32_t)(tid + i * NT) ^ lo);
            }
            continue;
          }
        }
#pragma unroll
        for (int i = 0; i < RPT; ++i) {
          uint32_t idx = idx0;
          if (i & 1) idx ^= fl & 31u;
          if (i & 2) idx ^= (fl >> 5) & 31u;
          if (i & 4) idx ^= (fl >> 10) & 31u;
          mac_row(acc[i], tab[idx], tb, (uint32_t)(tid + i * NT) ^ lo);
        }
      }
      // popcount-2 masks
      const int k2e = gr.w >> 16;
      for (int k = gr.w & 0xffff; k < k2e; ++k) {
        const uint4 rec = __ldg(&p.m2_rec[k]);
        const uint32_t lo = rec.x & (uint32_t)(T - 1);
#pragma unroll
        for (int i = 0; i < RPT; ++i) mac_row(acc[i], pc2_c<R>(t2, k, n, rec, xf[i]), tb, (uint32_t)(tid + i * NT) ^ lo);
      }
      // diagonal (the own tile: first chunk of h = 0)
      if ((uint32_t)gr.x == 0x80000000u) {
#pragma unroll
        for (int i = 0; i < RPT; ++i) mac_row(acc[i], diag_c<R>(p, n, xf[i]), tb, (uint32_t)(tid + i * NT));
      }
      if constexpr (CH != 0) {  // double-float accumulators: renormalise once per chunk
#pragma unroll
        for (int i = 0; i < RPT; ++i)
#pragma unroll
          for (int k = 0; k < NS; ++k) Slot<R>::renorm(acc[i][k]);
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
  // rows are written in the natural layout (logical chunk k of a row at soff[k]): straight to
  // y, or staged in shared memory for the cluster reduction or the Lanczos epilogue
  using V16 = typename Slot<R>::Out;
  const bool stage = CL || p.ep_part != nullptr;
  unsigned char* dst = stage ? sm : reinterpret_cast<unsigned char*>(y) + (size_t)tile * TILEB;
#pragma unroll
  for (int i = 0; i < RPT; ++i) {
    const size_t row = (size_t)(tid + i * NT);
    if constexpr (CH == 0) {
      reinterpret_cast<C*>(dst)[row] = acc[i][0];
    } else {
      unsigned char* out = dst + row * ROWB;
#pragma unroll
      for (int k = 0; k < NS; ++k) *reinterpret_cast<Out*>(out + soff[k]) = Slot<R>::out(acc[i][k]);
    }
  }
  if constexpr (CL) {
    // every CTA of the cluster reduces 1/csize of the tile's rows over the partial sums
    // held in the cluster's shared memories (fixed rank order: deterministic)
    tma::cluster_sync();
    const int units = TILEB / 16 / (int)csize;
    const uint32_t base = tma::saddr(sm) + crank * (uint32_t)units * 16u;
    store_units<V16, ROWB>(
        p, units, NT, (size_t)tile * TILEB + (size_t)crank * units * 16, y,
        [&](int u) {
          V16 sum = tma::ld_cluster(tma::map_rank(base + 16u * u, 0), V16{});
          for (uint32_t r = 1; r < csize; ++r) {
            const V16 v = tma::ld_cluster(tma::map_rank(base + 16u * u, r), V16{});
            if constexpr (std::is_same<V16, float4>::value) {
              sum.x += v.x; sum.y += v.y; sum.z += v.z; sum.w += v.w;
            } else {
              sum.x += v.x; sum.y += v.y;
            }
          }
          return sum;
        },
        sm + BUFB);
    tma::cluster_sync();  // no CTA leaves while others still read its shared memory
  } else if (stage) {
    __syncthreads();
    store_units<V16, ROWB>(p, TILEB / 16, NT, (size_t)tile * TILEB, y,
                           [&](int u) { return reinterpret_cast<const V16*>(sm)[u]; }, sm + BUFB);
  }
}

template <typename R, int BT>
int launch_tiled(const ApplyParams& p, const void* psi, void* y, cudaStream_t st) {
  using Cfg = TileCfg<R, BT>;
  int ntb = 8, cs = 1;
  TileChoice tc;
  const bool tuned = tile_choice_lookup(p.n * 2, std::is_same<R, float>::value ? SYK_C64 : SYK_C128, BT, &tc);
  if constexpr (std::is_same<R, float>::value && (BT == 4 || BT == 8 || BT == 16)) {
    if (tuned && tc.var > 0) {
      const int rc = launch_coset_var(p, BT, psi, y, st, tc.var, tc.ntb, tc.cs);
      if (rc <= 0) return rc;  // launched or failed; 1: not applicable, plain tiles below
    } else if (!tuned) {
      // untuned default: the coset kernel (faster than the plain one at every N = 28..40 and
      // 4/8/16 columns measured), one row bit for 16 columns and two for 4 and 8, 128-thread
      // CTAs from sector 2^18 up, cluster split while the grid has fewer than 32 warps per SM
      const int var = BT == 16 ? 1 : 2;
      const int vntb = p.D >= (int64_t(1) << 18) ? 7 : 6;
      if ((int64_t(1) << (var + vntb)) <= p.D) {
        const int64_t nt = p.D >> (var + vntb);
        int vcs = 1;
        while (vcs < 8 && nt * vcs * ((1 << vntb) / 32) < sm_count() * 32) vcs *= 2;
        const int rc = launch_coset_var(p, BT, psi, y, st, var, vntb, vcs);
        if (rc <= 0) return rc;
      }
    }
  }
  if (tuned && tc.var == 0 && (Cfg::RPT << tc.ntb) <= p.D) {
    ntb = tc.ntb;  // autotuned
    cs = tc.cs;
  } else {
    // 256-thread CTAs, narrower if the sector is smaller than a tile or a CTA would need more
    // than ~80 KB of shared memory (fewer than 2 resident CTAs per SM); if the grid has too
    // few warps, the mask chunks of a tile are split across a cluster of CTAs
    while (ntb > 6 && (p.D < ((int64_t)Cfg::RPT << ntb) || Cfg::smem(Cfg::RPT << ntb) > 80 * 1024)) --ntb;
    const int64_t nt = p.D / ((int64_t)Cfg::RPT << ntb);
    while (cs < 8 && nt * cs * ((1 << ntb) / 32) < sm_count() * 32) cs *= 2;
  }
  const int T = Cfg::RPT << ntb;
  if (p.D < T) return 1;
  const int64_t ntiles = p.D / T;
  int tb = 0;
  while ((1 << tb) < T) ++tb;
  const int4* groups = nullptr;
  int ng = 0;
  if (p.no_alloc) {
    if (!tile_groups_cached(p.terms, tb, Cfg::GMAX, &groups, &ng)) return 1;  // row kernel instead
  } else {
    SYK_TRY(tile_groups(p.terms, tb, Cfg::GMAX, &groups, &ng));
  }
  if (p.ep_part && ntiles * cs > p.ep_cap) {
    set_error("apply_H: %lld CTAs exceed the epilogue buffer (%lld)", (long long)(ntiles * cs), (long long)p.ep_cap);
    return SYK_EINVAL;
  }
  if constexpr (std::is_same<R, float>::value && BT == 1 && SYK_ONE_STATE_KERNEL)
    return launch_one_state(p, groups, ng, ntb, cs, psi, y, st);
  const size_t smem = Cfg::smem(T);
  SYK_TRY(ensure_smem_limit((const void*)k_apply_tiled<R, BT, false>, (int)Cfg::smem(Cfg::RPT << 8)));
  SYK_TRY(ensure_smem_limit((const void*)k_apply_tiled<R, BT, true>, (int)Cfg::smem(Cfg::RPT << 8)));
  if (cs == 1) {
    k_apply_tiled<R, BT, false><<<(unsigned)ntiles, 1u << ntb, smem, st>>>(p, groups, ng, ntb, psi, y);
    count_launch();
    count_matvec(kMvTiled);
    SYK_CUDA_CHECK(cudaGetLastError());
    return SYK_OK;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(ntiles * cs), 1, 1);
  cfg.blockDim = dim3(1u << ntb, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)cs;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  SYK_CUDA_CHECK(cudaLaunchKernelEx(&cfg, k_apply_tiled<R, BT, true>, p, groups, ng, ntb, psi, y));
  count_launch();
  count_matvec(kMvTiled);
  SYK_CUDA_CHECK(cudaGetLastError());
  return SYK_OK;
}

// Tiled path for a whole batch of 1, 2, 4, 8 or 16 columns; returns 1 if not applicable.
template <typename R>
int try_tiled(const ApplyParams& p, const void* psi, void* y, int64_t batch, cudaStream_t st) {
  if ((reinterpret_cast<uintptr_t>(psi) & 15) || (reinterpret_cast<uintptr_t>(y) & 15)) return 1;
  switch (batch) {
    case 1: return launch_tiled<R, 1>(p, psi, y, st);
    case 2: return launch_tiled<R, 2>(p, psi, y, st);
    case 4: return launch_tiled<R, 4>(p, psi, y, st);
    case 8: return launch_tiled<R, 8>(p, psi, y, st);
    case 16: return launch_tiled<R, 16>(p, psi, y, st);
    default: return 1;
  }
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

// Double-float copy of a complex128 vector: element e becomes (re_hi, im_hi, re_lo, im_lo)
// with hi = fl32(d) and lo = fl32(d - hi).
__global__ void k_split_df(const double2* __restrict__ x, float4* __restrict__ out, int64_t n) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const double2 v = x[e];
    const float rh = __double2float_rn(v.x), ih = __double2float_rn(v.y);
    const float rl = __double2float_rn(__dsub_rn(v.x, (double)rh));
    const float il = __double2float_rn(__dsub_rn(v.y, (double)ih));
    out[e] = make_float4(rh, ih, rl, il);
  }
}

// complex128 matvec in double-float arithmetic on the tiled kernel (batches of 1, 2, 4, 8, 16):
// the input is first split into its double-float copy (p.df_split, or a buffer allocated on
// the stream for this call); returns 1 if the tiled kernel does not apply to this launch.
int launch_apply_df(const ApplyParams& p, const void* psi, void* y, int64_t batch, cudaStream_t st) {
  if (batch != 1 && batch != 2 && batch != 4 && batch != 8 && batch != 16) return 1;
  if ((reinterpret_cast<uintptr_t>(y) & 15) || p.D < 64) return 1;
  const size_t need = size_t(p.D) * batch * sizeof(float4);
  void* split = p.df_split;
  bool owned = false;
  if (!split || p.df_split_bytes < need) {
    if (p.no_alloc) return 1;
    SYK_CUDA_CHECK(cudaMallocAsync(&split, need, st));
    owned = true;
  }
  const int64_t n = p.D * batch;
  const int threads = 256;
  const int64_t blocks = std::min<int64_t>((n + threads - 1) / threads, (int64_t)sm_count() * 16);
  k_split_df<<<(unsigned)blocks, threads, 0, st>>>(static_cast<const double2*>(psi), static_cast<float4*>(split), n);
  count_launch();
  int rc;
  switch (batch) {
    case 1: rc = launch_tiled<DF, 1>(p, split, y, st); break;
    case 2: rc = launch_tiled<DF, 2>(p, split, y, st); break;
    case 4: rc = launch_tiled<DF, 4>(p, split, y, st); break;
    case 8: rc = launch_tiled<DF, 8>(p, split, y, st); break;
    default: rc = launch_tiled<DF, 16>(p, split, y, st); break;
  }
  if (owned) cudaFreeAsync(split, st);
  return rc;
}

}  // namespace

int c128_arith() { return g_c128_arith.load(); }

int launch_apply_H(const ApplyParams& p, int dtype, const void* psi, void* y, int64_t batch, cudaStream_t st) {
  prof_before_apply(st);
  int rc = 1;
  if (dtype == SYK_C128 && c128_arith() == kC128DoubleFloat) rc = launch_apply_df(p, psi, y, batch, st);
  if (rc > 0)
    rc = dtype == SYK_C64 ? launch_apply_T<float>(p, psi, y, batch, st) : launch_apply_T<double>(p, psi, y, batch, st);
  prof_after_apply(st);
  count_applies(batch);
  return rc;
}

int launch_apply_chi(int N, int i, int parity_in, int dtype, const void* psi, void* y, int64_t batch,
                     cudaStream_t st) {
  const int n = N / 2;
  const int64_t D = int64_t(1) << (n - 1);
  const int threads = 256;
  int64_t blocks = std::min<int64_t>((D * batch + threads - 1) / threads, (int64_t)sm_count() * 32);
  if (dtype == SYK_C64)
    k_apply_chi<float><<<(unsigned)blocks, threads, 0, st>>>(n, i, 1 - parity_in, D, batch,
                                                             static_cast<const float2*>(psi), static_cast<float2*>(y));
  else
    k_apply_chi<double><<<(unsigned)blocks, threads, 0, st>>>(n, i, 1 - parity_in, D, batch,
                                                              static_cast<const double2*>(psi), static_cast<double2*>(y));
  count_launch();
  SYK_CUDA_CHECK(cudaGetLastError());
  return SYK_OK;
}

}  // namespace syk

extern "C" int syk_apply_H(const syk_terms* terms, int parity, int dtype, const void* psi, void* y,
                           int64_t batch, void* stream) {
  syk::NvtxRange nvtx_range_("syk_apply_H");
  syk::clear_error();
  if (!psi || !y || batch < 1) {
    syk::set_error("syk_apply_H: NULL vector or batch < 1");
    return SYK_EINVAL;
  }
  syk::ApplyParams p;
  SYK_TRY(syk::make_apply_params(terms, parity, dtype, &p));
  return syk::launch_apply_H(p, dtype, psi, y, batch, static_cast<cudaStream_t>(stream));
}

extern "C" int syk_status(const syk_terms* terms, int reset, void* stream) {
  syk::clear_error();
  if (!terms) {
    syk::set_error("syk_status: NULL terms");
    return SYK_EINVAL;
  }
  int cur = -1;
  SYK_CUDA_CHECK(cudaGetDevice(&cur));
  if (terms->dev.device != cur || !terms->dev.status) return SYK_OK;  // nothing launched on this device
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int word = 0;
  SYK_CUDA_CHECK(cudaMemcpyAsync(&word, terms->dev.status, sizeof(int), cudaMemcpyDeviceToHost, st));
  SYK_CUDA_CHECK(cudaStreamSynchronize(st));
  if (reset) SYK_CUDA_CHECK(cudaMemsetAsync(terms->dev.status, 0, sizeof(int), st));
  if (word & 4) {
    syk::set_error("syk_status: a bounded wait of a matvec for a staged tile gave up (its result is incomplete)");
    return SYK_ETIMEOUT;
  }
  return SYK_OK;
}

extern "C" int syk_c128_arith(int mode) {
  syk::clear_error();
  const int prev = syk::g_c128_arith.load();
  if (mode < 0) return prev;
  if (mode != syk::kC128DoubleFloat && mode != syk::kC128Fp64) {
    syk::set_error("syk_c128_arith: mode must be 0 (double-float) or 1 (FP64), got %d", mode);
    return SYK_EINVAL;
  }
  syk::g_c128_arith = mode;
  syk::bump_graph_epoch();  // captured matvec launches carry the other kernel
  return prev;
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

// ---------------------------------------------------------------- autotuner
// Sweeps the tile configurations of the tiled matvec (CTA width 64/128/256 x cluster
// size 1/2/4/8) for one (N, dtype, batch) on zero-filled scratch vectors, times each
// with CUDA events on `stream` and records the fastest for later launches.
extern "C" int syk_autotune_apply(const syk_terms* terms, int parity, int dtype, int64_t batch, int reps,
                                  void* stream, double* best_ms) {
  syk::NvtxRange nvtx_range_("syk_autotune_apply");
  using namespace syk;
  clear_error();
  if (batch != 1 && batch != 2 && batch != 4 && batch != 8 && batch != 16) {
    set_error("syk_autotune_apply: only batches of 1, 2, 4, 8 or 16 use the tiled matvec");
    return SYK_EINVAL;
  }
  if (reps < 1) reps = 2;
  ApplyParams P;
  SYK_TRY(make_apply_params(terms, parity, dtype, &P));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t vb = size_t(P.D) * batch * dtype_size(dtype);
  void *x = nullptr, *y = nullptr;
  SYK_CUDA_CHECK(cudaMallocAsync(&x, vb, st));
  cudaError_t e = cudaMallocAsync(&y, vb, st);
  if (e != cudaSuccess) {
    cudaFreeAsync(x, st);
    set_error("syk_autotune_apply: %s", cudaGetErrorString(e));
    return SYK_ENOMEM;
  }
  cudaMemsetAsync(x, 0, vb, st);
  void* split = nullptr;  // double-float copy of the input (complex128)
  if (dtype == SYK_C128) {
    if (cudaMallocAsync(&split, vb, st) != cudaSuccess) {
      cudaFreeAsync(x, st);
      cudaFreeAsync(y, st);
      set_error("syk_autotune_apply: cannot allocate %zu bytes", vb);
      return SYK_ENOMEM;
    }
    P.df_split = split;
    P.df_split_bytes = vb;
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const int N = terms->N;
  const int rows_per_thread =
      dtype == SYK_C64
          ? (batch == 1 ? TileCfg<float, 1>::RPT : batch == 2 ? TileCfg<float, 2>::RPT : batch == 4 ? TileCfg<float, 4>::RPT
             : batch == 8 ? TileCfg<float, 8>::RPT : TileCfg<float, 16>::RPT)
          : (batch == 1 ? TileCfg<double, 1>::RPT : batch == 2 ? TileCfg<double, 2>::RPT
             : batch == 4 ? TileCfg<double, 4>::RPT : batch == 8 ? TileCfg<double, 8>::RPT : TileCfg<double, 16>::RPT);
  TileChoice best{0, 0, 1e300};
  int rc = SYK_OK;
  for (int var = 0; var <= 3 && rc == SYK_OK; ++var)
  for (int ntb = 6; ntb <= 8 && rc == SYK_OK; ++ntb)
    for (int cs = 1; cs <= 8 && rc == SYK_OK; cs *= 2) {
      if (!coset_var_ok(dtype, batch, var) || (var && !coset_fits(batch, var, ntb))) continue;
      const int rpt = var ? 1 << var : rows_per_thread;
      if ((int64_t(rpt) << ntb) > P.D) continue;  // tile larger than the sector
      tile_choice_set(N, dtype, batch, TileChoice{ntb, cs, 0.0, var});
      rc = launch_apply_H(P, dtype, x, y, batch, st);  // warm-up (also builds the chunk list)
      cudaEventRecord(e0, st);
      for (int r = 0; r < reps && rc == SYK_OK; ++r) rc = launch_apply_H(P, dtype, x, y, batch, st);
      cudaEventRecord(e1, st);
      if (cudaEventSynchronize(e1) != cudaSuccess) rc = SYK_ECUDA;
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      ms /= reps;
      if (rc == SYK_OK && ms < best.ms) best = TileChoice{ntb, cs, ms, var};
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFreeAsync(x, st);
  cudaFreeAsync(y, st);
  if (split) cudaFreeAsync(split, st);
  if (rc != SYK_OK || best.ntb == 0) {
    std::lock_guard<std::mutex> lk(g_tune_mtx);
    g_tune.erase(tune_key(N, dtype, batch));
    if (rc == SYK_OK) set_error("syk_autotune_apply: the sector is smaller than every tile");
    return rc != SYK_OK ? rc : SYK_EINVAL;
  }
  tile_choice_set(N, dtype, batch, best);
  if (best_ms) *best_ms = best.ms;
  return SYK_OK;
}

// JSON form of the tuned table: {"apply_tiles": [{"N":40,"dtype":1,"batch":8,"ntb":8,"cluster":1,"ms":6.5}, ...]}
extern "C" int syk_autotune_export(char* buf, size_t len) {
  using namespace syk;
  std::string js = "{\"apply_tiles\": [";
  {
    std::lock_guard<std::mutex> lk(g_tune_mtx);
    bool first = true;
    for (auto& kv : g_tune) {
      char item[192];
      snprintf(item, sizeof(item),
               "%s{\"N\": %d, \"dtype\": %d, \"batch\": %d, \"ntb\": %d, \"cluster\": %d, \"variant\": %d, "
               "\"ms\": %.6g}",
               first ? "" : ", ", int(kv.first & 0xff), int((kv.first >> 8) & 0xff), int(kv.first >> 16),
               kv.second.ntb, kv.second.cs, kv.second.var, kv.second.ms);
      js += item;
      first = false;
    }
  }
  js += "]}";
  if (!buf || len < js.size() + 1) {
    set_error("syk_autotune_export: buffer needs %zu bytes", js.size() + 1);
    return SYK_EINVAL;
  }
  std::memcpy(buf, js.c_str(), js.size() + 1);
  return SYK_OK;
}

extern "C" int syk_autotune_reset(void) {
  using namespace syk;
  {
    std::lock_guard<std::mutex> lk(g_tune_mtx);
    g_tune.clear();
  }
  bump_graph_epoch();  // captured matvec launches carry the old tile shapes
  return SYK_OK;
}

// Reads entries written by syk_autotune_export (keys in any order; unknown keys ignored).
extern "C" int syk_autotune_import(const char* json) {
  using namespace syk;
  if (!json) {
    set_error("syk_autotune_import: NULL");
    return SYK_EINVAL;
  }
  const char* p = std::strstr(json, "\"apply_tiles\"");
  if (!p) {
    set_error("syk_autotune_import: no apply_tiles array");
    return SYK_EINVAL;
  }
  int count = 0;
  while ((p = std::strchr(p, '{')) != nullptr) {
    const char* end = std::strchr(p, '}');
    if (!end) break;
    std::string obj(p, end - p);
    auto num = [&](const char* key, double* v) {
      const std::string k = std::string("\"") + key + "\"";
      size_t at = obj.find(k);
      if (at == std::string::npos) return false;
      at = obj.find(':', at);
      if (at == std::string::npos) return false;
      *v = std::strtod(obj.c_str() + at + 1, nullptr);
      return true;
    };
    double N, dt, b, ntb, cs, ms = 0.0, var = 0.0;
    if (num("N", &N) && num("dtype", &dt) && num("batch", &b) && num("ntb", &ntb) && num("cluster", &cs)) {
      num("ms", &ms);
      num("variant", &var);
      if (ntb < 6 || ntb > 8 || (cs != 1 && cs != 2 && cs != 4 && cs != 8) ||
          !coset_var_ok(int(dt), int64_t(b), int(var))) {
        set_error("syk_autotune_import: invalid entry (ntb=%g cluster=%g variant=%g)", ntb, cs, var);
        return SYK_EINVAL;
      }
      tile_choice_set(int(N), int(dt), int64_t(b), TileChoice{int(ntb), int(cs), ms, int(var)});
      ++count;
    }
    p = end + 1;
  }
  return count > 0 ? SYK_OK : SYK_EINVAL;
}
