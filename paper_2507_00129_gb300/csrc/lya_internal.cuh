// Internal declarations shared by the CUDA translation units of liblya.so.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "lya.h"

namespace lya {

// Device-side input-check flags (OR-ed into the handle's error word).
enum : unsigned {
  FLAG_UNSORTED = 1u,
  FLAG_NONFINITE = 2u,
  FLAG_OFFSETS = 4u,
  FLAG_NEGATIVE_W = 8u,
  FLAG_TOO_LONG = 16u,
  FLAG_X3_CAP = 32u,      // a 3PCF main vertex had more neighbours than the kernel's capacity
  FLAG_RETRY = 64u,       // a shared-memory compare-and-swap update gave up after its retry limit
};

// Per-forest data derived by the preparation kernel (structure of arrays).
// Lengths of forests that fail the offset checks are set to 0 so that no
// kernel ever reads outside the pixel arrays.
struct Forests {
  int64_t n;          // forests
  int64_t* off;       // first pixel (global pixel index)
  int32_t* len;       // pixel count (0 = ignored)
  double* ux;         // unit vector of the line of sight
  double* uy;
  double* uz;
  double* dmin;       // distance of the first pixel
  double* dmax;       // distance of the last pixel
  double* wsum;       // W = sum w
  double* lbar;       // weighted mean of Lambda
  double* ssum;       // S = sum w (Lambda - Lbar)^2
  float* dref;        // reference distance, a multiple of 2^-10 (exact in FP32)
  int32_t* mock;      // catalogue (mock) index of the forest
  float* wmax;        // largest weight of the forest
  float* wdmax;       // largest |w delta| of the forest
  float* hmin;        // smallest gap between consecutive packed distances (> 0)
  float* xmax;        // largest |Lambda - Lbar| of the forest
};

// Packed pixel record used by every FP32 kernel:
//   x = fl32(d - dref), y = w, z = fl32(w * delta), w = fl32(Lambda - Lbar)
using Pix = float4;

// FP32 magic constant: fl_rd(x + 2^23) holds floor(x) in its low mantissa bits
// for 0 <= x < 2^23.
constexpr float kMagic = 8388608.0f;
constexpr uint32_t kMagicBits = 0x4B000000u;

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void red_add_f32_shared(uint32_t addr, float v) {
  asm volatile("red.shared.add.f32 [%0], %1;" ::"r"(addr), "f"(v));
}

template <int OFF>
__device__ __forceinline__ void red_add_f32_shared_off(uint32_t addr, float v) {
  asm volatile("red.shared.add.f32 [%0+%2], %1;" ::"r"(addr), "f"(v), "n"(OFF));
}

__device__ __forceinline__ void red_add_f64_global(double* p, double v) {
  asm volatile("red.global.add.f64 [%0], %1;" ::"l"(p), "d"(v) : "memory");
}

__device__ __forceinline__ double warp_sum_f64(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ double warp_max_f64(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// First output of the SplitMix64 generator (Steele, Lea, Flood 2014) for state x.
__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Subsample rule of the distortion matrix: keep forest pair (a, b) iff
// all != 0 or SplitMix64(seed ^ (min(a,b) * 2^32 + max(a,b))) < thr.
__device__ __forceinline__ bool keep_pair(int a, int b, uint64_t seed, uint64_t thr, int all) {
  const uint64_t lo = static_cast<uint64_t>(min(a, b)), hi = static_cast<uint64_t>(max(a, b));
  return all || (splitmix64(seed ^ ((lo << 32) | hi)) < thr);
}

// Number of elements of the sorted array a[0..n) strictly below v (v NaN -> n).
__device__ __forceinline__ int count_below(const Pix* a, int n, float v) {
  int lo = 0, hi = n;
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if (a[mid].x < v) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// ---------------------------------------------------------------------------
// host-side launchers (defined in the .cu files, called from api.cu)
// ---------------------------------------------------------------------------
struct DevInfo {
  int sms;
  int smem_optin;   // max dynamic shared memory per block (bytes)
  int smem_per_sm;
};

// prep.cu
// fp (optional) accumulates a 64-bit fingerprint of the catalogue geometry
// (sum over forests of a hash of index, position, length and distance range).
cudaError_t launch_prep(const lya_catalog& cat, int64_t forest_base, int64_t pix_base, int32_t mock,
                        Forests F, Pix* pix, unsigned* err, unsigned long long* fp, cudaStream_t s);
cudaError_t launch_project(const lya_catalog& cat, Forests F, int64_t forest_base, float* out,
                           cudaStream_t s);
cudaError_t launch_max_len(Forests F, int32_t* out, cudaStream_t s);

// pairs.cu
struct PairBuild {
  int nside;
  double rperp_max;
  double theta_max;
};
// Builds the (a < b) pair list of forests [f0, f1) into *pairs (device buffer
// grown with cudaMalloc as needed).  Synchronises.  forder (optional, [f0, f1)
// slots) receives the non-empty forests in HEALPix-cell order, then -1.
cudaError_t build_pairs(const Forests& F, int64_t f0, int64_t f1, const PairBuild& pb, int2** pairs,
                        int64_t* cap, int64_t pair_base, int64_t* n_out, void** scratch,
                        size_t* scratch_cap, int32_t* forder, cudaStream_t s);
cudaError_t launch_pair_geometry(const int2* pairs, int64_t n, Forests F, double inv_dpar,
                                 double inv_dperp, float2* cs, cudaStream_t s);
cudaError_t launch_pack_pairs(const int32_t* a, const int32_t* b, int64_t n, int2* out,
                              cudaStream_t s);
// Reorder pairs (and their geometry) by (mock, first r_perp row of the band)
// so that consecutive pairs share the pair kernel's accumulator.
cudaError_t sort_pairs_by_band(int2* pairs, float2* cs, int64_t n, Forests F, const Pix* pix, int n_perp,
                               int n_mocks, void** scratch, size_t* scratch_cap, cudaStream_t s);
cudaError_t launch_unpack_pairs(const int2* p, int64_t n, int32_t* a, int32_t* b, cudaStream_t s);
// id[f] = nested HEALPix pixel (resolution nside) of forest f's line of sight (0 for empty forests)
cudaError_t launch_subsample_ids(const Forests& F, int nside, int32_t* id, cudaStream_t s);

// cov.cu: weighted sub-sample covariance from per sub-sample sums [n_sub][nb]
// (scratch: 3 nb doubles + n_sub + 1 ints, 256-byte aligned)
size_t covariance_scratch_bytes(int n_sub, int nb);
cudaError_t launch_covariance(const double* num_s, const double* wsum_s, int n_sub, int nb, double* cov,
                              double* xi_out, void* scratch, cudaStream_t s);

// xi.cu
struct XiLaunch {
  int warps;       // warps per block
  int blocks;      // persistent grid size
  int hcap;        // histogram capacity (floats per array per warp)
  int seg;         // pixel buffer per warp (pixels)
  int grab;        // pairs per work grab
  int smem;        // dynamic shared memory bytes
};
struct XiArgs {
  const int2* pairs;
  const float2* cs;
  int64_t n_pairs;
  const Pix* pix;
  Forests F;
  int n_par, n_perp;
  double* num;
  double* wsum;
  int nb;
  unsigned long long* counter;
};
// largest n_par the mixed pair kernel's shared-memory layout holds
int xi_mixed_max_npar();
cudaError_t plan_xi_mixed(const DevInfo& dev, int n_par, int max_len, int warps, int grab,
                          XiLaunch* L);
cudaError_t launch_xi_mixed(const XiArgs& a, const XiLaunch& L, cudaStream_t s);
cudaError_t launch_xi_fp64(const XiArgs& a, const lya_catalog* cats, int n_cats, const DevInfo& dev,
                           int max_len, double r_par_max, double r_perp_max, XiLaunch* used,
                           cudaStream_t s);
cudaError_t launch_finalize(const double* num, const double* wsum, double* xi, int64_t n,
                            cudaStream_t s);

// dmat.cu
struct DmArgs {
  const int2* pairs;
  const float2* cs;
  int64_t n_pairs;
  const Pix* pix;
  Forests F;
  int n_par, n_perp;
  int eta_mean_slope;
  double p_subsample;
  uint64_t seed;
  double* G;        // [n_mocks][nb*nb] upper-triangle accumulators (A <= B)
  double* wdm;      // [n_mocks][nb]
  int max_len;
  int n_mocks;      // catalogues in the batch (forest f belongs to F.mock[f])
  const int32_t* fbase;   // [n_mocks] first forest of each catalogue (set by run_dmat)
  int tensor_tiles;       // rank-1 tiles: 0 = FP32 FMA, 1 = TF32x3 tensor cores (mma.sync)
};
cudaError_t run_dmat(const DmArgs& a, const DevInfo& dev, void** scratch, size_t* scratch_cap,
                     cudaStream_t s);
cudaError_t launch_dm_finalize(const double* G, const double* wdm, double* D, double* wdm_out,
                               int nb, int n_mocks, cudaStream_t s);
// work counts of the closed form over the kept pairs (single catalogue)
struct DmWork {
  unsigned long long pairs;   // kept forest pairs with an in-grid band
  unsigned long long pix;     // their in-grid pixel pairs
  double sv2;                 // sum over rank-1 vectors (rows of a, columns of b) of |S_v|^2
  double sp2;                 // sum over pairs of |S_pair|^2
};
cudaError_t launch_dm_work(const DmArgs& a, const DevInfo& dev, DmWork* out, cudaStream_t s);

// adjoint.cu
struct AdjArgs {
  const int2* pairs;
  const float2* cs;
  int64_t n_pairs;
  const Pix* pix;
  Forests F;
  int n_par, n_perp;
  const double* grad_xi;
  const double* grad_wsum;   // dL/dW_A (NULL = 0)
  const double* xi;
  const double* wsum;
  const float* delta;   // caller's delta (for dL/dw = delta * ...)
  const float* weight;
  int64_t pix_base;
  int64_t n_pix;
  float* grad_delta;
  float* grad_weight;
  int max_len;
  const int32_t* forder;   // [F.n] forests in sky order for the work items (-1 = none); NULL = index order
};
cudaError_t run_adjoint(const AdjArgs& a, const DevInfo& dev, void** scratch, size_t* scratch_cap,
                        cudaStream_t s);

// xi3.cu: three-point estimator, Eq. (2.8)
struct X3Args {
  const int2* pairs;     // forest pairs (a < b) that can hold pixels within r_max
  int64_t n_pairs;
  const Pix* pix;
  Forests F;
  const double* dist;    // caller's FP64 distances (single catalogue: packed index = pixel index)
  int64_t n_pix;
  int n_r, n_theta, n_alpha;
  double r_max;
  double* num;           // [n_r^2 n_alpha n_theta^2]
  double* wsum;
  double* xi;            // optional
};
cudaError_t run_xi3(const X3Args& a, const DevInfo& dev, void** scratch, size_t* scratch_cap, unsigned* err,
                    cudaStream_t s);

// pairs.cu: (forest, quasar) pairs that can hold an in-grid pixel, forest
// f's own quasar own[f] excluded (own may be NULL), grouped by forest:
// forest f's pairs are (*pairs)[qoff[f] .. qoff[f+1]) (qoff: device [F.n+1]).
// Q is a point set in the Forests layout (ux, uy, uz, dmin = dmax = distance,
// len = 1 or 0 = invalid).  *pairs is grown with cudaMalloc as needed.
// Synchronises.
cudaError_t build_cross_pairs(const Forests& F, const Forests& Q, int nside, double rpar_max, double rperp_max,
                              const int64_t* own, int2** pairs, int64_t* cap, int64_t* qoff, int64_t* n_out,
                              cudaStream_t s);

// xcf.cu: forest x quasar cross-correlation, its distortion matrix, and the
// same-forest (1D) correlation
struct XcfArgs {
  const int2* pairs;     // (forest, quasar), grouped by forest
  const int64_t* qoff;   // [F.n + 1] forest f's pairs: qoff[f] .. qoff[f+1]
  int64_t n_pairs;
  const float* delta;    // caller's pixel arrays (single catalogue: packed index = pixel index)
  const float* weight;
  const Pix* pix;
  Forests F;
  Forests Q;
  const float* wq;       // quasar weights
  int n_par, n_perp;     // r_par over [-r_par_max, r_par_max) in n_par bins
  double r_par_max, r_perp_max;
  double* num;           // [nb] cross-correlation sums
  double* wsum;
  unsigned* err;         // device flags
  int eta_mean_slope;    // distortion matrix
  double p_subsample;
  uint64_t seed;
  double* G;             // [nb*nb] upper triangle (A <= B) of D~
  double* wdm;           // [nb]
  int max_len;
};
// fp accumulates a fingerprint of the quasars' geometry (index, position, distance, validity)
cudaError_t launch_qso_prep(const lya_quasars& q, Forests Q, unsigned* err, unsigned long long* fp,
                            cudaStream_t s);
// adds a fingerprint of own[0..n) (own-quasar indices; nothing for NULL) to *fp
cudaError_t launch_own_hash(const int64_t* own, int64_t n, unsigned long long* fp, cudaStream_t s);
cudaError_t launch_xcf(const XcfArgs& a, const DevInfo& dev, cudaStream_t s);
cudaError_t launch_xdm(const XcfArgs& a, const DevInfo& dev, cudaStream_t s);
// shared memory the kernels need: 0 when the grid or forest length is beyond their limits
int xcf_smem_bytes(int nb, int max_len);
int xdm_warps(const DevInfo& dev, int max_len);
struct X1Args {
  Forests F;
  const double* dist;    // caller's arrays (single catalogue: packed index = pixel index)
  const float* delta;
  const float* weight;
  int n_bins;
  double r_max;
  double* num;
  double* wsum;
  int max_len;
};
int xi1d_smem_bytes(int n_bins, int max_len);
cudaError_t launch_xi1d(const X1Args& a, const Pix* pix, const DevInfo& dev, cudaStream_t s);

// pairs.cu: out[k] = sum_{j<k} in[j] for k <= n (one block; n up to a few million)
cudaError_t launch_exclusive_scan(const int32_t* in, int64_t n, int64_t* out, cudaStream_t s);

// means.cu: per-bin weighted means of r_par, r_perp and the pair distance, and
// pixel-pair counts, over the cached forest-pair list
struct MeansArgs {
  const int2* pairs;     // (a < b)
  const float2* cs;      // (cos(theta/2)/D_par, sin(theta/2)/D_perp) per pair
  int64_t n_pairs;
  const Pix* pix;
  Forests F;
  int n_par, n_perp;
  double d_par, d_perp;  // bin widths
  unsigned* err;
  int max_len;
  const double* zpix;    // per-pixel redshift (single catalogue: packed index = pixel index), or NULL
};
size_t means_scratch_bytes(int64_t n_forests, int64_t n_pairs, int nb);
int means_smem_bytes(int nb, int max_len, bool with_z);
// outputs: wsum, rpar_mean, rperp_mean, dist_mean [nb] float64 (wsum may be NULL), z_mean [nb] (needs
// a.zpix; NULL = not computed), count [nb] int64
cudaError_t launch_bin_means(const MeansArgs& a, const DevInfo& dev, void* scratch, double* wsum, double* rpar_mean,
                             double* rperp_mean, double* dist_mean, double* z_mean, int64_t* count, cudaStream_t s);

// scratch helper (api.cu).  While the calling thread captures a CUDA graph
// (lya_capture_begin) it allocates nothing and fails with
// cudaErrorNotPermitted if the buffer is too small.
cudaError_t grow(void** p, size_t* cap, size_t need);
bool capturing_thread();

// cudaFuncSetAttribute(MaxDynamicSharedMemorySize) for `func` on the current
// device, skipped when a value at least as large was set before (so that a
// launch captured into a graph needs no attribute call).
cudaError_t set_max_dynamic_smem(const void* func, int bytes);

// process-wide count of kernel launches (api.cu); LYA_COUNT(n) adds n
void count_launches(long long n);
#define LYA_COUNT(n) ::lya::count_launches(n)

// xi.cu: per-pair in-grid pixel-pair counts of the kept pairs
struct StatsOut {
  unsigned long long pairs;
  unsigned long long pix;
  unsigned long long pix_sq;
};
// xi.cu: FP32-vs-FP64 bin-edge flips over the kept pairs
struct FlipOut {
  unsigned long long pix;     // in-grid pixel pairs under FP64 binning
  unsigned long long flips;   // pixel pairs whose FP32 bin differs (in grid or not)
  double w;                   // their weights
  double wflip;
};
cudaError_t launch_flip_tally(const XiArgs& a, const double* dist, double inv_dpar, double inv_dperp,
                              double p_subsample, uint64_t seed, FlipOut* out, const DevInfo& dev,
                              cudaStream_t s);
cudaError_t launch_pair_stats(const XiArgs& a, double p_subsample, uint64_t seed, StatsOut* out,
                              const DevInfo& dev, cudaStream_t s);

}  // namespace lya
