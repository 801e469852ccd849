// lya_xi_pairs_static: the xi/W pair sum over an explicit forest-pair list
// with all scratch memory in a fixed device array of this library, for
// callers that cannot allocate device memory (see include/lya.h).
//
// The array is a file-scope __device__ object: every device that loads the
// library holds it until the process exits.  Host code must not use the
// array's name as a device address (it is a host-side stand-in); the device
// address is obtained once per device with cudaGetSymbolAddress and cached.
#include <algorithm>
#include <cmath>
#include <mutex>

#include "lya_internal.cuh"

namespace lya {
namespace {

constexpr int64_t kStaticForests = 65536;
constexpr int64_t kStaticPix = 1 << 20;
constexpr int64_t kStaticPairs = 1 << 20;
constexpr int64_t kStaticBins = 65536;

constexpr size_t al256(size_t v) { return (v + 255) & ~size_t(255); }

// byte offsets inside the static array
constexpr size_t kOffForest = 0;                                      // 16 arrays of kStaticForests
constexpr size_t kForestBytes = al256(kStaticForests * 8) * 9 + al256(kStaticForests * 4) * 7;
constexpr size_t kOffPix = kOffForest + kForestBytes;                  // float4 pixels
constexpr size_t kOffPairs = kOffPix + al256(kStaticPix * 16);         // int2 pairs
constexpr size_t kOffCs = kOffPairs + al256(kStaticPairs * 8);         // float2 pair geometry
constexpr size_t kOffOut = kOffCs + al256(kStaticPairs * 8);           // num, wsum when not given
constexpr size_t kOffMisc = kOffOut + al256(kStaticBins * 16);         // error word, counter
constexpr size_t kStaticBytes = kOffMisc + 256;

__device__ __align__(256) unsigned char g_static_scratch[kStaticBytes];

std::mutex g_mu;
void* g_base[128] = {};

// Rejects pairs that name a forest outside [0, n) or the same forest twice
// (written as (-1, -1), which every later kernel skips) and flags them.
__global__ void static_check_pairs(int2* p, int64_t n, int64_t nf, unsigned* err) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int2 q = p[k];
    if (q.x < 0 || q.y < 0 || q.x >= nf || q.y >= nf || q.x == q.y) {
      p[k] = make_int2(-1, -1);
      atomicOr(err, FLAG_OFFSETS);
    }
  }
}

int status_from_flags(unsigned f) {
  if (f == 0) return LYA_OK;
  if (f & FLAG_UNSORTED) return LYA_ERR_UNSORTED;
  if (f & (FLAG_NONFINITE | FLAG_NEGATIVE_W)) return LYA_ERR_NONFINITE;
  if (f & FLAG_TOO_LONG) return LYA_ERR_TOO_LARGE;
  return LYA_ERR_DEVICE_CHECK;
}

}  // namespace
}  // namespace lya

using namespace lya;

extern "C" int lya_xi_pairs_static(const lya_catalog* cat, const lya_bins* bins, const int32_t* pair_a,
                                   const int32_t* pair_b, int64_t n_pairs, double* num, double* wsum,
                                   double* xi, void* stream) {
  if (!cat || !bins || n_pairs < 0 || (n_pairs > 0 && (!pair_a || !pair_b))) return LYA_ERR_INVALID_ARG;
  if (!num && !wsum && !xi) return LYA_ERR_INVALID_ARG;
  if (cat->n_forests < 0 || cat->n_pix < 0 || !cat->offsets) return LYA_ERR_INVALID_ARG;
  if (cat->n_forests > 0 && (!cat->ra || !cat->dec)) return LYA_ERR_INVALID_ARG;
  if (cat->n_pix > 0 && (!cat->dist || !cat->loglam || !cat->delta || !cat->weight))
    return LYA_ERR_INVALID_ARG;
  // the limits of lya_xi_pairs (MIXED), then the static array's
  if (bins->n_par < 1 || bins->n_par > xi_mixed_max_npar() || bins->n_perp < 1 || bins->n_perp > 4096 ||
      static_cast<int64_t>(bins->n_par) * bins->n_perp > kStaticBins)
    return LYA_ERR_TOO_LARGE;
  if (!(bins->r_par_max > 0) || !(bins->r_perp_max > 0) || !std::isfinite(bins->r_par_max) ||
      !std::isfinite(bins->r_perp_max))
    return LYA_ERR_INVALID_ARG;
  if (cat->n_forests > kStaticForests || cat->n_pix > kStaticPix || n_pairs > kStaticPairs)
    return LYA_ERR_TOO_LARGE;
  cudaStream_t s = static_cast<cudaStream_t>(stream);

  // once per device: the device address of the static array
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 128) return LYA_ERR_CUDA;
  char* base = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_base[dev]) {
      void* ptr = nullptr;
      if (cudaGetSymbolAddress(&ptr, g_static_scratch) != cudaSuccess || !ptr) return LYA_ERR_CUDA;
      g_base[dev] = ptr;
    }
    base = static_cast<char*>(g_base[dev]);
  }
  DevInfo info{};
  if (cudaDeviceGetAttribute(&info.sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&info.smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
    return LYA_ERR_CUDA;

  Forests F{};
  F.n = cat->n_forests;
  {
    char* p = base + kOffForest;
    auto take = [&](size_t b) { char* q = p; p += al256(b); return q; };
    F.off = reinterpret_cast<int64_t*>(take(kStaticForests * 8));
    F.ux = reinterpret_cast<double*>(take(kStaticForests * 8));
    F.uy = reinterpret_cast<double*>(take(kStaticForests * 8));
    F.uz = reinterpret_cast<double*>(take(kStaticForests * 8));
    F.dmin = reinterpret_cast<double*>(take(kStaticForests * 8));
    F.dmax = reinterpret_cast<double*>(take(kStaticForests * 8));
    F.wsum = reinterpret_cast<double*>(take(kStaticForests * 8));
    F.lbar = reinterpret_cast<double*>(take(kStaticForests * 8));
    F.ssum = reinterpret_cast<double*>(take(kStaticForests * 8));
    F.len = reinterpret_cast<int32_t*>(take(kStaticForests * 4));
    F.dref = reinterpret_cast<float*>(take(kStaticForests * 4));
    F.mock = reinterpret_cast<int32_t*>(take(kStaticForests * 4));
    F.wmax = reinterpret_cast<float*>(take(kStaticForests * 4));
    F.wdmax = reinterpret_cast<float*>(take(kStaticForests * 4));
    F.hmin = reinterpret_cast<float*>(take(kStaticForests * 4));
    F.xmax = reinterpret_cast<float*>(take(kStaticForests * 4));
  }
  Pix* pix = reinterpret_cast<Pix*>(base + kOffPix);
  int2* pairs = reinterpret_cast<int2*>(base + kOffPairs);
  float2* cs = reinterpret_cast<float2*>(base + kOffCs);
  double* N = num ? num : reinterpret_cast<double*>(base + kOffOut);
  double* W = wsum ? wsum : reinterpret_cast<double*>(base + kOffOut) + kStaticBins;
  unsigned* err = reinterpret_cast<unsigned*>(base + kOffMisc);
  unsigned long long* counter = reinterpret_cast<unsigned long long*>(base + kOffMisc + 64);

  const int nb = bins->n_par * bins->n_perp;
  // state left by an earlier call is cleared here: error word, outputs; the
  // work counter is cleared by launch_xi_mixed
  if (cudaMemsetAsync(err, 0, sizeof(unsigned), s) != cudaSuccess) return LYA_ERR_CUDA;
  if (cudaMemsetAsync(N, 0, nb * 8, s) != cudaSuccess) return LYA_ERR_CUDA;
  if (cudaMemsetAsync(W, 0, nb * 8, s) != cudaSuccess) return LYA_ERR_CUDA;
  if (launch_prep(*cat, 0, 0, 0, F, pix, err, nullptr, s) != cudaSuccess) return LYA_ERR_CUDA;
  if (launch_pack_pairs(pair_a, pair_b, n_pairs, pairs, s) != cudaSuccess) return LYA_ERR_CUDA;
  if (n_pairs > 0) {
    const int64_t blocks = std::min<int64_t>((n_pairs + 255) / 256, 65535);
    LYA_COUNT(1), static_check_pairs<<<static_cast<int>(blocks), 256, 0, s>>>(pairs, n_pairs, cat->n_forests, err);
    if (cudaGetLastError() != cudaSuccess) return LYA_ERR_CUDA;
  }
  if (launch_pair_geometry(pairs, n_pairs, F, bins->n_par / bins->r_par_max,
                           bins->n_perp / bins->r_perp_max, cs, s) != cudaSuccess)
    return LYA_ERR_CUDA;
  XiArgs A{};
  A.pairs = pairs;
  A.cs = cs;
  A.n_pairs = n_pairs;
  A.pix = pix;
  A.F = F;
  A.n_par = bins->n_par;
  A.n_perp = bins->n_perp;
  A.num = N;
  A.wsum = W;
  A.nb = nb;
  A.counter = counter;
  XiLaunch L{};
  // staging buffers sized for forests of up to 1024 pixels; longer forests
  // are processed in 1024-pixel segments by the same kernel
  if (plan_xi_mixed(info, bins->n_par, 1024, 8, 4, &L) != cudaSuccess) return LYA_ERR_CUDA;
  if (launch_xi_mixed(A, L, s) != cudaSuccess) return LYA_ERR_CUDA;
  if (xi && launch_finalize(N, W, xi, nb, s) != cudaSuccess) return LYA_ERR_CUDA;
  unsigned flags = 0;
  if (cudaMemcpyAsync(&flags, err, sizeof(unsigned), cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return LYA_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return LYA_ERR_CUDA;
  return status_from_flags(flags);
}
