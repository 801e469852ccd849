// Per-forest preparation (input checks, moments, packed pixels) and the
// continuum projection of Eq. (2.7).  One warp per forest; FP64 reductions.
#include <math.h>

#include "lya_internal.cuh"

namespace lya {
namespace {

constexpr int kPrepThreads = 256;

__global__ void __launch_bounds__(kPrepThreads) prep_kernel(lya_catalog cat, int64_t forest_base,
                                                            int64_t pix_base, int32_t mock, Forests F,
                                                            Pix* pix, unsigned* err,
                                                            unsigned long long* fp) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5;
  for (int64_t f = warp; f < cat.n_forests; f += nwarps) {
    const int64_t o0 = cat.offsets[f], o1 = cat.offsets[f + 1];
    unsigned flags = 0;
    bool ok_off = (o0 >= 0) && (o1 >= o0) && (o1 <= cat.n_pix);
    if (f == 0 && o0 != 0) ok_off = false;
    if (f == cat.n_forests - 1 && o1 != cat.n_pix) ok_off = false;
    int64_t n = ok_off ? (o1 - o0) : 0;
    if (!ok_off) flags |= FLAG_OFFSETS;
    if (n > (1 << 20)) { flags |= FLAG_TOO_LONG; n = 0; }
    const double ra = cat.ra[f], dec = cat.dec[f];
    if (!isfinite(ra) || !isfinite(dec)) { flags |= FLAG_NONFINITE; n = 0; }
    const int64_t gf = forest_base + f;
    // pass 1: sums, checks
    double sw = 0.0, swl = 0.0;
    unsigned lflags = 0;
    for (int64_t k = lane; k < n; k += 32) {
      const double d = cat.dist[o0 + k];
      const double L = cat.loglam[o0 + k];
      const float w = cat.weight[o0 + k];
      const float dl = cat.delta[o0 + k];
      if (!isfinite(d) || !(d > 0.0) || !isfinite(L) || !isfinite(w) || !isfinite(dl))
        lflags |= FLAG_NONFINITE;
      if (w < 0.0f) lflags |= FLAG_NEGATIVE_W;
      if (k + 1 < n && !(cat.dist[o0 + k + 1] > d)) lflags |= FLAG_UNSORTED;
      sw += static_cast<double>(w);
      swl += static_cast<double>(w) * L;
    }
    sw = warp_sum_f64(sw);
    swl = warp_sum_f64(swl);
    lflags = __reduce_or_sync(0xffffffffu, lflags);
    flags |= lflags;
    // a forest that fails a check takes no part in any sum (len = 0), which
    // also keeps every kernel's index arithmetic in bounds
    if (lflags & (FLAG_UNSORTED | FLAG_NONFINITE)) n = 0;
    const double lbar = (sw > 0.0) ? swl / sw : 0.0;
    const double d0 = (n > 0) ? cat.dist[o0] : 0.0;
    // Reference distance: a multiple of 2^-10 (exact in FP32 for d < 8192 Mpc/h,
    // so that differences and sums of two references are exact FP32 values).
    const float dref_f = (n > 0 && isfinite(d0)) ? static_cast<float>(floor(d0 * 1024.0) / 1024.0) : 0.0f;
    const double dref = static_cast<double>(dref_f);
    // pass 2: slope normaliser, packed pixels, bounds used for fixed-point scaling
    double ss = 0.0;
    float wmx = 0.f, wdmx = 0.f, hmn = INFINITY, xmx = 0.f;
    for (int64_t k = lane; k < n; k += 32) {
      const double d = cat.dist[o0 + k];
      const double x = cat.loglam[o0 + k] - lbar;
      const float w = cat.weight[o0 + k];
      const float dl = cat.delta[o0 + k];
      ss += static_cast<double>(w) * x * x;
      Pix p;
      p.x = static_cast<float>(d - dref);
      p.y = w;
      p.z = static_cast<float>(static_cast<double>(w) * static_cast<double>(dl));
      p.w = static_cast<float>(x);
      pix[pix_base + o0 + k] = p;
      wmx = fmaxf(wmx, fabsf(p.y));
      wdmx = fmaxf(wdmx, fabsf(p.z));
      xmx = fmaxf(xmx, fabsf(p.w));
      if (k + 1 < n) {
        const float nx = static_cast<float>(cat.dist[o0 + k + 1] - dref);
        hmn = fminf(hmn, nx - p.x);
      }
    }
    ss = warp_sum_f64(ss);
    for (int o = 16; o > 0; o >>= 1) {
      wmx = fmaxf(wmx, __shfl_xor_sync(0xffffffffu, wmx, o));
      wdmx = fmaxf(wdmx, __shfl_xor_sync(0xffffffffu, wdmx, o));
      hmn = fminf(hmn, __shfl_xor_sync(0xffffffffu, hmn, o));
      xmx = fmaxf(xmx, __shfl_xor_sync(0xffffffffu, xmx, o));
    }
    if (lane == 0) {
      if (flags) atomicOr(err, flags);
      double sr, cr, sd, cd;
      sincos(ra, &sr, &cr);
      sincos(dec, &sd, &cd);
      F.off[gf] = pix_base + (ok_off ? o0 : 0);
      F.len[gf] = static_cast<int32_t>(n);
      F.ux[gf] = cd * cr;
      F.uy[gf] = cd * sr;
      F.uz[gf] = sd;
      F.dmin[gf] = d0;
      F.dmax[gf] = (n > 0) ? cat.dist[o1 - 1] : 0.0;
      F.wsum[gf] = (sw > 0.0) ? sw : 0.0;
      F.lbar[gf] = lbar;
      F.ssum[gf] = (sw > 0.0) ? ss : 0.0;
      F.dref[gf] = dref_f;
      F.mock[gf] = mock;
      F.wmax[gf] = wmx;
      F.wdmax[gf] = wdmx;
      // packed distances of a sorted forest may repeat after rounding; a gap
      // of 0 (or a single pixel) is recorded as a tiny positive number, which
      // only makes the fixed-point bound more conservative
      F.hmin[gf] = (hmn > 1e-6f && hmn < INFINITY) ? hmn : 1e-6f;
      F.xmax[gf] = xmx;
      if (fp) {
        auto bits = [](double v) { return static_cast<uint64_t>(__double_as_longlong(v)); };
        uint64_t x = splitmix64(static_cast<uint64_t>(gf) * 0x9E3779B97F4A7C15ull ^ static_cast<uint64_t>(n));
        x = splitmix64(x ^ bits(ra));
        x = splitmix64(x ^ bits(dec));
        x = splitmix64(x ^ bits(d0));
        x = splitmix64(x ^ bits(F.dmax[gf]));
        atomicAdd(fp, static_cast<unsigned long long>(x));
      }
    }
  }
}

// delta' = delta - sum(w delta)/W - x sum(w x delta)/S  (Eq. 2.7 applied to delta)
__global__ void __launch_bounds__(kPrepThreads) project_kernel(lya_catalog cat, Forests F,
                                                               int64_t forest_base, float* out) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5;
  for (int64_t f = warp; f < cat.n_forests; f += nwarps) {
    const int64_t gf = forest_base + f;
    const int64_t n = F.len[gf];
    const int64_t o0 = cat.offsets[f];
    if (n == 0) continue;
    const double W = F.wsum[gf], S = F.ssum[gf], lbar = F.lbar[gf];
    double swd = 0.0, swxd = 0.0;
    for (int64_t k = lane; k < n; k += 32) {
      const double w = cat.weight[o0 + k];
      const double dl = cat.delta[o0 + k];
      const double x = cat.loglam[o0 + k] - lbar;
      swd += w * dl;
      swxd += w * x * dl;
    }
    swd = warp_sum_f64(swd);
    swxd = warp_sum_f64(swxd);
    const double m = (W > 0.0) ? swd / W : 0.0;
    const double k1 = (W > 0.0 && S > 0.0) ? swxd / S : 0.0;
    __syncwarp();
    for (int64_t k = lane; k < n; k += 32) {
      const double x = cat.loglam[o0 + k] - lbar;
      const double dl = cat.delta[o0 + k];
      out[o0 + k] = static_cast<float>(dl - m - x * k1);
    }
  }
}

__global__ void max_len_kernel(Forests F, int32_t* out) {
  int m = 0;
  for (int64_t f = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; f < F.n;
       f += static_cast<int64_t>(gridDim.x) * blockDim.x)
    m = max(m, F.len[f]);
  m = __reduce_max_sync(0xffffffffu, m);
  if ((threadIdx.x & 31) == 0) atomicMax(out, m);
}

int blocks_for(int64_t n_forests) {
  int64_t warps = n_forests;
  int64_t b = (warps * 32 + kPrepThreads - 1) / kPrepThreads;
  if (b < 1) b = 1;
  if (b > 65535) b = 65535;
  return static_cast<int>(b);
}

}  // namespace

cudaError_t launch_prep(const lya_catalog& cat, int64_t forest_base, int64_t pix_base, int32_t mock,
                        Forests F, Pix* pix, unsigned* err, unsigned long long* fp, cudaStream_t s) {
  if (cat.n_forests == 0) return cudaSuccess;
  LYA_COUNT(1), prep_kernel<<<blocks_for(cat.n_forests), kPrepThreads, 0, s>>>(cat, forest_base, pix_base, mock, F,
                                                                 pix, err, fp);
  return cudaGetLastError();
}

cudaError_t launch_project(const lya_catalog& cat, Forests F, int64_t forest_base, float* out,
                           cudaStream_t s) {
  if (cat.n_forests == 0) return cudaSuccess;
  LYA_COUNT(1), project_kernel<<<blocks_for(cat.n_forests), kPrepThreads, 0, s>>>(cat, F, forest_base, out);
  return cudaGetLastError();
}

cudaError_t launch_max_len(Forests F, int32_t* out, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(out, 0, sizeof(int32_t), s);
  if (e != cudaSuccess) return e;
  if (F.n == 0) return cudaSuccess;
  int64_t b = (F.n + 255) / 256;
  if (b > 4096) b = 4096;
  LYA_COUNT(1), max_len_kernel<<<static_cast<int>(b), 256, 0, s>>>(F, out);
  return cudaGetLastError();
}

}  // namespace lya
