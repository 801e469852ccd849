// Per-bin weighted means of the pair separations and of the pair distance,
// and pixel-pair counts: the columns a PICCA/Vega fit reads next to xi (the
// paper exports its results for Vega, Appendix A):
//     rpar_mean_A = sum_A w_i w_j r_par / W_A,  rperp_mean_A = sum_A w_i w_j r_perp / W_A,
//     dist_mean_A = sum_A w_i w_j (d_i + d_j) / 2 / W_A,  count_A,
// over the pixel pairs of Eq. (2.4) with the bisector split of Section 2.1.
//
// The forest pairs (a < b) of the cached list are grouped by a (counting
// sort of pair indices); the kernel is described at means_kernel.  Bins are
// the FP32 ones of the mixed path's arithmetic (|d_i - d_j| from the packed
// distances and reference offsets, times cos(theta/2)/D_par).  Run sums are
// FP32 (a run is a few pixels), accumulated as double-float pairs per block
// and in FP64 across blocks.
#include <math.h>

#include <algorithm>

#include "dfloat.cuh"

namespace lya {
namespace {

constexpr int kMW = 16;   // warps per block
constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ int below(const float* a, int n, float v) {
  int lo = 0, hi = n;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (a[mid] < v) lo = mid + 1; else hi = mid;
  }
  return lo;
}

__global__ void first_count_kernel(const int2* p, int64_t n, int32_t* count) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
    if (p[k].x >= 0) atomicAdd(&count[p[k].x], 1);
}

__global__ void first_scatter_kernel(const int2* p, int64_t n, const int64_t* start, int32_t* cursor,
                                     int32_t* list) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    const int a = p[k].x;
    if (a >= 0) list[start[a] + atomicAdd(&cursor[a], 1)] = static_cast<int32_t>(k);
  }
}

struct Acc {
  double* W;
  double* WX;
  double* WY;
  double* WD;
  double* WZ;   // sum w_i w_j (z_i + z_j) / 2 (with pixel redshifts)
  unsigned long long* C;
};

// Segmented inclusive scan of four (five with Z) FP32 sums over lanes with
// equal bins (equal bins are contiguous); returns the first lane of the run on
// its last lane, -1 elsewhere.
template <bool Z>
__device__ __forceinline__ int run_sums(int bin, int lane, float& v0, float& v1, float& v2, float& v3, float& v4) {
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const int ob = __shfl_up_sync(kFull, bin, d);
    const float o0 = __shfl_up_sync(kFull, v0, d);
    const float o1 = __shfl_up_sync(kFull, v1, d);
    const float o2 = __shfl_up_sync(kFull, v2, d);
    const float o3 = __shfl_up_sync(kFull, v3, d);
    const float o4 = Z ? __shfl_up_sync(kFull, v4, d) : 0.f;
    if (lane >= d && ob == bin) {
      v0 += o0;
      v1 += o1;
      v2 += o2;
      v3 += o3;
      if (Z) v4 += o4;
    }
  }
  const int prev = __shfl_up_sync(kFull, bin, 1);
  const int nxt = __shfl_down_sync(kFull, bin, 1);
  const bool head = bin >= 0 && (lane == 0 || prev != bin);
  const bool tail = bin >= 0 && (lane == 31 || nxt != bin);
  const unsigned hm = __ballot_sync(kFull, head);
  if (!tail) return -1;
  return 31 - __clz(hm & (0xffffffffu >> (31 - lane)));
}

// One block per first forest a (grid-stride; a's packed distances and weights
// staged in shared memory), one warp per partner b.  A warp takes 32 pixels j
// of b at a time, one window of a's pixels per lane (binary search), then walks
// each window together with lanes over i, in two parts: d_i < d_j and
// d_i >= d_j.  In each part r_par/D_par and r_perp/D_perp are monotone in i,
// so equal bins are contiguous and a segmented warp scan sums each run of
// w_i w_j, w_i w_j r_par/D_par, w_i w_j r_perp/D_perp and w_i w_j x_i; the
// run's last lane adds them to the block's double-float histograms and its
// length to the count histogram.  With Z the runs also sum w_i w_j z_i, and
// the pair's mean redshift (z_i + z_j) / 2 goes to a fifth histogram.
template <bool Z>
__global__ void __launch_bounds__(kMW * 32, 2) means_kernel(MeansArgs A, const int64_t* poff, const int32_t* plist,
                                                             Acc acc) {
  // h1[nb] = (W, WX) | h2[nb] = (WY, WD) | hc[nb] u32 | [h3[nb] = WZ] | per team: xa[cap], wa[cap], [za[cap]]
  extern __shared__ float4 msh[];
  const int nb = A.n_par * A.n_perp;
  const int cap = A.max_len;
  float4* h1 = msh;
  float4* h2 = msh + nb;
  unsigned* hc = reinterpret_cast<unsigned*>(msh + 2 * nb);
  float2* h3 = reinterpret_cast<float2*>(hc + ((nb + 1) & ~1));
  for (int k = threadIdx.x; k < nb; k += blockDim.x) {
    h1[k] = make_float4(0.f, 0.f, 0.f, 0.f);
    h2[k] = make_float4(0.f, 0.f, 0.f, 0.f);
    hc[k] = 0u;
    if (Z) h3[k] = make_float2(0.f, 0.f);
  }
  __syncthreads();
  // two teams of kMW / 2 warps on their own first forests (own staging and
  // barrier), adding to the block's histograms
  constexpr int kTeamWarps = kMW / 2;
  const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
  const int team = wi / kTeamWarps, tw = wi % kTeamWarps, tt = threadIdx.x % (kTeamWarps * 32);
  float* stage0 = Z ? reinterpret_cast<float*>(h3 + nb) : reinterpret_cast<float*>(hc + nb);
  float* xa = stage0 + static_cast<size_t>(team) * (Z ? 3 : 2) * cap;
  float* wa = xa + cap;
  float* za = wa + cap;   // used only with Z
  const float fnpar = static_cast<float>(A.n_par), fnperp = static_cast<float>(A.n_perp);
  for (int64_t f = 2 * static_cast<int64_t>(blockIdx.x) + team; f < A.F.n; f += 2 * static_cast<int64_t>(gridDim.x)) {
    const int64_t k0 = poff[f], k1 = poff[f + 1];
    const int n = A.F.len[f];
    if (k1 <= k0 || n <= 0 || n > cap) continue;   // uniform over the team
    team_sync(1 + team, kTeamWarps * 32);
    const Pix* pa = A.pix + A.F.off[f];
    for (int k = tt; k < n; k += kTeamWarps * 32) {
      const Pix P = pa[k];
      xa[k] = P.x;
      wa[k] = P.y;
      if (Z) za[k] = static_cast<float>(A.zpix[A.F.off[f] + k]);
    }
    team_sync(1 + team, kTeamWarps * 32);
    const float dref_a = A.F.dref[f];
    for (int64_t kk = k0 + tw; kk < k1; kk += kTeamWarps) {
      const int k = plist[kk];
      const int b = A.pairs[k].y;
      if (b < 0) continue;
      const int nbp = A.F.len[b];
      if (nbp <= 0) continue;
      const float2 cs = A.cs[k];
      const float cP = cs.x, sP = cs.y;
      const float dd = dref_a - A.F.dref[b];   // exact: multiples of 2^-10 below 8192
      const float ss = dref_a + A.F.dref[b];
      const Pix* pb = A.pix + A.F.off[b];
      const float half = fnpar / cP;
      const float tmax = (sP > 0.f) ? fnperp / sP : INFINITY;
      for (int jb = 0; jb < nbp; jb += 32) {
        // lane setup: pixel j = jb + lane of b and its window [i0, i1) of a, split at im (d_i >= d_j)
        const int j = jb + lane;
        float D = 0.f, S = 0.f, wj = 0.f, zj = 0.f;
        int i0 = 0, im = 0, i1 = 0;
        if (j < nbp) {
          const Pix P = pb[j];
          D = dd - P.x;          // d_i - d_j = xa_i + D
          S = ss + P.x;          // d_i + d_j = xa_i + S
          wj = P.y;
          if (Z) zj = static_cast<float>(A.zpix[A.F.off[b] + j]);
          const float lo = -D - half - 0.5f;
          const float hi = fminf(-D + half, tmax - S) + 0.5f;
          i0 = below(xa, n, lo);
          i1 = (hi > lo) ? below(xa, n, hi) : i0;
          im = min(max(below(xa, n, -D), i0), i1);
        }
        const int nj = min(32, nbp - jb);
        for (int t = 0; t < nj; ++t) {
          const float Dt = __shfl_sync(kFull, D, t), St = __shfl_sync(kFull, S, t), wt = __shfl_sync(kFull, wj, t);
          const float Zt = Z ? __shfl_sync(kFull, zj, t) : 0.f;
          const int a0 = __shfl_sync(kFull, i0, t), am = __shfl_sync(kFull, im, t), a1 = __shfl_sync(kFull, i1, t);
#pragma unroll 1
          for (int part = 0; part < 2; ++part) {
            const int lo_i = part ? am : a0, hi_i = part ? a1 : am;
            for (int base = lo_i; base < hi_i; base += 32) {
              const int i = base + lane;
              int bin = -1;
              float v0 = 0.f, v1 = 0.f, v2 = 0.f, v3 = 0.f, v4 = 0.f;
              if (i < hi_i) {
                const float xi = xa[i];
                const float xv = fabsf(xi + Dt) * cP;
                const float yv = (xi + St) * sP;
                if (xv < fnpar && yv < fnperp) {
                  bin = static_cast<int>(xv) * A.n_perp + static_cast<int>(yv);
                  const float w = wa[i] * wt;
                  v0 = w;
                  v1 = w * xv;
                  v2 = w * yv;
                  v3 = w * xi;
                  if (Z) v4 = w * za[i];
                }
              }
              const int r0 = run_sums<Z>(bin, lane, v0, v1, v2, v3, v4);
              if (r0 >= 0) {
                df_atomic_add(reinterpret_cast<float2*>(&h1[bin]), v0, 0.f, A.err);
                df_atomic_add(reinterpret_cast<float2*>(&h1[bin]) + 1, v1, 0.f, A.err);
                df_atomic_add(reinterpret_cast<float2*>(&h2[bin]), v2, 0.f, A.err);
                df_atomic_add(reinterpret_cast<float2*>(&h2[bin]) + 1, 0.5f * fmaf(St, v0, v3), 0.f, A.err);
                if (Z) df_atomic_add(&h3[bin], 0.5f * fmaf(Zt, v0, v4), 0.f, A.err);
                atomicAdd(&hc[bin], static_cast<unsigned>(lane - r0 + 1));
              }
            }
          }
        }
      }
    }
  }
  __syncthreads();
  for (int k = threadIdx.x; k < nb; k += blockDim.x) {
    const float4 u = h1[k], v = h2[k];
    const double w = static_cast<double>(u.x) + u.y;
    if (w != 0.0) {
      red_add_f64_global(acc.W + k, w);
      red_add_f64_global(acc.WX + k, static_cast<double>(u.z) + u.w);
      red_add_f64_global(acc.WY + k, static_cast<double>(v.x) + v.y);
      red_add_f64_global(acc.WD + k, static_cast<double>(v.z) + v.w);
      if (Z) red_add_f64_global(acc.WZ + k, static_cast<double>(h3[k].x) + h3[k].y);
    }
    if (hc[k]) atomicAdd(acc.C + k, static_cast<unsigned long long>(hc[k]));
  }
}

__global__ void means_finalize_kernel(Acc acc, int nb, double d_par, double d_perp, double* wsum, double* rp,
                                      double* rt, double* dm, double* zm, int64_t* count) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nb; k += gridDim.x * blockDim.x) {
    const double w = acc.W[k];
    const bool on = w != 0.0;
    if (wsum) wsum[k] = w;
    rp[k] = on ? d_par * acc.WX[k] / w : 0.0;
    rt[k] = on ? d_perp * acc.WY[k] / w : 0.0;
    dm[k] = on ? acc.WD[k] / w : 0.0;
    if (zm) zm[k] = on ? acc.WZ[k] / w : 0.0;
    count[k] = static_cast<int64_t>(acc.C[k]);
  }
}

int grid_for(int64_t n, int threads) {
  int64_t b = (n + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > 1 << 16) b = 1 << 16;
  return static_cast<int>(b);
}

size_t al256(size_t v) { return (v + 255) & ~size_t(255); }

}  // namespace

size_t means_scratch_bytes(int64_t n_forests, int64_t n_pairs, int nb) {
  return al256(6 * static_cast<size_t>(nb) * 8) + al256((n_forests + 1) * 8) + al256(2 * n_forests * 4 + 4) +
         al256(std::max<int64_t>(n_pairs, 1) * 4);
}

int means_smem_bytes(int nb, int max_len, bool with_z) {
  const int base = 32 * nb + 4 * ((nb + 1) & ~1);
  return with_z ? base + 8 * nb + 2 * 12 * std::max(max_len, 1) : base + 2 * 8 * std::max(max_len, 1);
}

cudaError_t launch_bin_means(const MeansArgs& a, const DevInfo& dev, void* scratch, double* wsum, double* rpar_mean,
                             double* rperp_mean, double* dist_mean, double* z_mean, int64_t* count, cudaStream_t s) {
  const int nb = a.n_par * a.n_perp;
  const bool with_z = a.zpix != nullptr && z_mean != nullptr;
  char* p = static_cast<char*>(scratch);
  Acc acc;
  acc.W = reinterpret_cast<double*>(p);
  acc.WX = acc.W + nb;
  acc.WY = acc.WX + nb;
  acc.WD = acc.WY + nb;
  acc.WZ = acc.WD + nb;
  acc.C = reinterpret_cast<unsigned long long*>(acc.WZ + nb);
  p += al256(6 * static_cast<size_t>(nb) * 8);
  int64_t* poff = reinterpret_cast<int64_t*>(p);
  p += al256((a.F.n + 1) * 8);
  int32_t* cnt = reinterpret_cast<int32_t*>(p);
  int32_t* cursor = cnt + a.F.n;
  p += al256(2 * a.F.n * 4 + 4);
  int32_t* plist = reinterpret_cast<int32_t*>(p);
  cudaError_t e = cudaMemsetAsync(acc.W, 0, 6 * static_cast<size_t>(nb) * 8, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(cnt, 0, 2 * a.F.n * 4 + 4, s);
  if (e != cudaSuccess) return e;
  if (a.n_pairs > 0 && a.F.n > 0) {
    LYA_COUNT(1), first_count_kernel<<<grid_for(a.n_pairs, 256), 256, 0, s>>>(a.pairs, a.n_pairs, cnt);
    e = launch_exclusive_scan(cnt, a.F.n, poff, s);
    if (e != cudaSuccess) return e;
    LYA_COUNT(1), first_scatter_kernel<<<grid_for(a.n_pairs, 256), 256, 0, s>>>(a.pairs, a.n_pairs, poff, cursor,
                                                                                 plist);
    const int smem = means_smem_bytes(nb, a.max_len, with_z);
    const void* fn = with_z ? reinterpret_cast<const void*>(means_kernel<true>)
                            : reinterpret_cast<const void*>(means_kernel<false>);
    e = set_max_dynamic_smem(fn, smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = with_z ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, means_kernel<true>, kMW * 32, smem)
               : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, means_kernel<false>, kMW * 32, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const int blocks = static_cast<int>(std::min<int64_t>(static_cast<int64_t>(dev.sms) * per_sm, (a.F.n + 1) / 2));
    if (with_z) LYA_COUNT(1), means_kernel<true><<<blocks, kMW * 32, smem, s>>>(a, poff, plist, acc);
    else LYA_COUNT(1), means_kernel<false><<<blocks, kMW * 32, smem, s>>>(a, poff, plist, acc);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  LYA_COUNT(1), means_finalize_kernel<<<grid_for(nb, 256), 256, 0, s>>>(acc, nb, a.d_par, a.d_perp, wsum, rpar_mean,
                                                                          rperp_mean, dist_mean,
                                                                          with_z ? z_mean : nullptr, count);
  return cudaGetLastError();
}

}  // namespace lya
