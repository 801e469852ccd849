// Covariance of xi from sub-samples of the catalogue (HEALPix pixels of the
// first forest of each pair): with per sub-sample sums N^s_A, W^s_A of
// Eq. (2.4) and the full sums N_A = sum_s N^s_A, W_A = sum_s W^s_A,
// xi_A = N_A / W_A,
//     C_AB = sum_s W^s_A W^s_B (xi^s_A - xi_A)(xi^s_B - xi_B) / (W_A W_B)
//          = sum_s a^s_A a^s_B / (W_A W_B),   a^s_A = N^s_A - W^s_A xi_A,
// the weighted sub-sample covariance (zero rows and columns where W_A = 0).
// FP64 throughout; only sub-samples with pairs enter the sum (list built in
// sub-sample order, so the result does not depend on scheduling).
#include <algorithm>

#include "lya_internal.cuh"

namespace lya {
namespace {

constexpr int kTile = 64;     // output tile edge
constexpr int kSt = 16;       // sub-samples per shared-memory stage

// full sums, xi, and the ordered list of sub-samples with any weight
__global__ void cov_totals_kernel(const double* num_s, const double* wsum_s, int n_sub, int nb, double* W,
                                  double* N, double* xi) {
  for (int A = blockIdx.x * blockDim.x + threadIdx.x; A < nb; A += gridDim.x * blockDim.x) {
    double w = 0.0, n = 0.0;
    for (int s = 0; s < n_sub; ++s) {
      w += wsum_s[static_cast<int64_t>(s) * nb + A];
      n += num_s[static_cast<int64_t>(s) * nb + A];
    }
    W[A] = w;
    N[A] = n;
    xi[A] = (w != 0.0) ? n / w : 0.0;
  }
}

__global__ void cov_list_kernel(const double* wsum_s, int n_sub, int nb, int32_t* list) {
  // one block: sub-sample s is listed if any of its bins has weight
  __shared__ int any;
  int m = 0;
  for (int s = 0; s < n_sub; ++s) {
    if (threadIdx.x == 0) any = 0;
    __syncthreads();
    for (int A = threadIdx.x; A < nb; A += blockDim.x)
      if (wsum_s[static_cast<int64_t>(s) * nb + A] != 0.0) any = 1;
    __syncthreads();
    if (any) {
      if (threadIdx.x == 0) list[1 + m] = s;
      ++m;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) list[0] = m;
}

// C tile (64 x 64) per block of 16 x 16 threads, 4 x 4 outputs per thread
__global__ void __launch_bounds__(256) cov_kernel(const double* num_s, const double* wsum_s, int nb,
                                                  const double* W, const double* xi, const int32_t* list,
                                                  double* cov) {
  __shared__ double ar[kSt][kTile];
  __shared__ double ac[kSt][kTile];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int r0 = blockIdx.y * kTile, c0 = blockIdx.x * kTile;
  const int m = list[0];
  double acc[4][4] = {};
  for (int k0 = 0; k0 < m; k0 += kSt) {
    for (int e = threadIdx.x; e < kSt * kTile; e += blockDim.x) {
      const int kk = e / kTile, t = e - kk * kTile;
      double vr = 0.0, vc = 0.0;
      if (k0 + kk < m) {
        const int64_t base = static_cast<int64_t>(list[1 + k0 + kk]) * nb;
        const int A = r0 + t, B = c0 + t;
        if (A < nb) vr = num_s[base + A] - wsum_s[base + A] * xi[A];
        if (B < nb) vc = num_s[base + B] - wsum_s[base + B] * xi[B];
      }
      ar[kk][t] = vr;
      ac[kk][t] = vc;
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < kSt; ++kk) {
      double a[4], b[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        a[u] = ar[kk][ty * 4 + u];
        b[u] = ac[kk][tx * 4 + u];
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = fma(a[u], b[v], acc[u][v]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int A = r0 + ty * 4 + u;
    if (A >= nb) continue;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int B = c0 + tx * 4 + v;
      if (B >= nb) continue;
      const double den = W[A] * W[B];
      cov[static_cast<int64_t>(A) * nb + B] = (den != 0.0) ? acc[u][v] / den : 0.0;
    }
  }
}

}  // namespace

size_t covariance_scratch_bytes(int n_sub, int nb) {
  auto al = [](size_t v) { return (v + 255) & ~size_t(255); };
  return 3 * al(static_cast<size_t>(nb) * 8) + al((static_cast<size_t>(n_sub) + 1) * 4);
}

cudaError_t launch_covariance(const double* num_s, const double* wsum_s, int n_sub, int nb, double* cov,
                              double* xi_out, void* scratch, cudaStream_t s) {
  if (nb == 0) return cudaSuccess;
  auto al = [](size_t v) { return (v + 255) & ~size_t(255); };
  char* sc = static_cast<char*>(scratch);
  double* W = reinterpret_cast<double*>(sc);
  double* N = reinterpret_cast<double*>(sc + al(static_cast<size_t>(nb) * 8));
  double* xi = reinterpret_cast<double*>(sc + 2 * al(static_cast<size_t>(nb) * 8));
  int32_t* list = reinterpret_cast<int32_t*>(sc + 3 * al(static_cast<size_t>(nb) * 8));
  const int tb = std::min((nb + 255) / 256, 1024);
  LYA_COUNT(1), cov_totals_kernel<<<tb, 256, 0, s>>>(num_s, wsum_s, n_sub, nb, W, N, xi);
  LYA_COUNT(1), cov_list_kernel<<<1, 256, 0, s>>>(wsum_s, n_sub, nb, list);
  const int nt = (nb + kTile - 1) / kTile;
  LYA_COUNT(1), cov_kernel<<<dim3(nt, nt), 256, 0, s>>>(num_s, wsum_s, nb, W, xi, list, cov);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess && xi_out) e = cudaMemcpyAsync(xi_out, xi, static_cast<size_t>(nb) * 8, cudaMemcpyDeviceToDevice, s);
  return e;
}

}  // namespace lya
