// Forest x quasar cross-correlation, its distortion matrix, and the
// same-forest (1D) correlation -- the extensions the paper names as future
// work (Section 4), built on the estimator of Eq. (2.4), the bisector split of
// Section 2.1 and the projection of Eqs. (2.6)-(2.7).
//
// Cross-correlation.  A quasar q (distance d_q, weight w_q) plays the second
// pixel of Eq. (2.4) with delta = 1:
//     N_A = sum_{(i,q) in A} (w delta)_i w_q,   W_A = sum_{(i,q) in A} w_i w_q,
// r_par = (d_i - d_q) cos(theta/2) signed and binned over [-r_par_max, r_par_max),
// r_perp = (d_i + d_q) sin(theta/2).  The (forest, quasar) list is grouped by
// forest; a block holds two teams of warps, each staging one forest's packed
// pixels in shared memory.  A warp takes 32 of the forest's quasars, one
// pair's geometry per lane (FP64, then the window of pixels that can land in
// the grid by binary search in shared memory), and walks each window with all
// lanes: a lane bins one pixel in FP32 as x = fma(x_i, c/D_par, X0),
// y = fma(x_i, s/D_perp, Y0) (X0, Y0 formed in FP64).  Both grow with the pixel
// distance, so the bin never decreases along the window and equal bins sit in
// adjacent lanes: a segmented warp scan sums each run (error-free FP32
// products w_q w_i and w_q (w delta)_i, TwoSum-compensated additions) and the
// run's last lane adds it to the block's double-float histogram (bounded
// compare-and-swap), flushed to the FP64 sums once per block.
//
// Distortion matrix.  With eta = I - 1 u^T - x v^T the pair (a, q) adds
// w_q (diag(alpha) - alpha alpha^T / W_a - beta beta^T / S_a) on the bins its
// window touches, alpha[B] = sum_{k in B} w_k, beta[B] = sum_{k in B} w_k x_k.
// One warp per kept pair: the same segmented scan yields (bin, alpha, beta)
// per run, kept as the pair's run list in shared memory; the warp adds the
// upper triangle (bins ascend along the list) to D~ with FP64 global
// reductions; D = D~ / W_A row by row.
//
// 1D correlation.  One block per forest stages the forest's packed and FP64
// distances and FP64 prefix sums of w and w delta; a warp takes one pixel i,
// its lanes the pixels j > i.  The bin floor((d_j - d_i) / D) is taken from
// FP32 values unless they lie within a guard band of an edge, where the FP64
// division of the definition decides, so every bin decision is the
// definition's; each run of equal bins adds (w delta)_i (P[j1+1] - P[j0]) to
// the block's FP64 histogram.
#include <math.h>

#include <algorithm>

#include "dfloat.cuh"

namespace lya {
namespace {

constexpr int kXW = 8;    // warps per block (distortion matrix)
constexpr int kXCW = 16;  // warps per block of the cross-correlation (two blocks per SM share the shared memory)
constexpr unsigned kFull = 0xffffffffu;

// FP32 bin coordinates of a (forest, quasar) pair:
//   x = (r_par + r_par_max) / D_par = fma(x_i, cP, X0),  y = r_perp / D_perp = fma(x_i, sP, Y0)
// for the packed pixel distance x_i = fl32(d_i - dref), and the window [i0, i1)
// of pixels that can fall in the grid (0.5 Mpc/h wider than the FP32 rounding).
struct XGeo {
  float cP, sP, X0, Y0;
  int i0, i1;
};

__device__ __forceinline__ XGeo pair_geo(const XcfArgs& A, int a, int q, const Pix* fp, int n) {
  const double ax = A.F.ux[a], ay = A.F.uy[a], az = A.F.uz[a];
  const double qx = A.Q.ux[q], qy = A.Q.uy[q], qz = A.Q.uz[q];
  const double dx = ax - qx, dy = ay - qy, dz = az - qz;
  const double sx = ax + qx, sy = ay + qy, sz = az + qz;
  const double s = 0.5 * sqrt(dx * dx + dy * dy + dz * dz);
  const double c = 0.5 * sqrt(sx * sx + sy * sy + sz * sz);
  const double inv_dpar = A.n_par / (2.0 * A.r_par_max), inv_dperp = A.n_perp / A.r_perp_max;
  const double dref = static_cast<double>(A.F.dref[a]), dq = A.Q.dmin[q];
  XGeo g;
  g.cP = static_cast<float>(c * inv_dpar);
  g.sP = static_cast<float>(s * inv_dperp);
  g.X0 = static_cast<float>((dref - dq) * c * inv_dpar + 0.5 * A.n_par);
  g.Y0 = static_cast<float>((dref + dq) * s * inv_dperp);
  const double xq = dq - dref;
  const double half = A.r_par_max / c;
  const double lo = xq - half - 0.5;
  double hi = xq + half + 0.5;
  if (s > 0.0) hi = fmin(hi, A.r_perp_max / s - dref - dq + 0.5);
  g.i0 = count_below(fp, n, static_cast<float>(lo));
  g.i1 = (hi > lo) ? count_below(fp, n, static_cast<float>(hi)) : g.i0;
  if (g.i1 < g.i0) g.i1 = g.i0;
  return g;
}

// Bin of one pixel (-1 outside the grid).  Bins never decrease with x_i.
__device__ __forceinline__ int pixel_bin(const XGeo& g, float x, int n_par, int n_perp) {
  const float xv = fmaf(x, g.cP, g.X0);
  const float yv = fmaf(x, g.sP, g.Y0);
  if (!(xv >= 0.0f) || !(xv < static_cast<float>(n_par)) || !(yv < static_cast<float>(n_perp))) return -1;
  return static_cast<int>(xv) * n_perp + static_cast<int>(yv);
}

// Segmented inclusive scan of two compensated sums (hi, lo) over lanes with
// equal bins (runs are contiguous); returns true on the last lane of a run.
__device__ __forceinline__ bool run_scan(int bin, int lane, float& h1, float& l1, float& h2, float& l2) {
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const int ob = __shfl_up_sync(kFull, bin, d);
    const float oh1 = __shfl_up_sync(kFull, h1, d);
    const float ol1 = __shfl_up_sync(kFull, l1, d);
    const float oh2 = __shfl_up_sync(kFull, h2, d);
    const float ol2 = __shfl_up_sync(kFull, l2, d);
    if (lane >= d && ob == bin) {
      float s, e;
      two_sum(h1, oh1, s, e);
      h1 = s;
      l1 += ol1 + e;
      two_sum(h2, oh2, s, e);
      h2 = s;
      l2 += ol2 + e;
    }
  }
  const int nxt = __shfl_down_sync(kFull, bin, 1);
  return bin >= 0 && (lane == 31 || nxt != bin);
}

__global__ void own_hash_kernel(const int64_t* own, int64_t n, unsigned long long* fp) {
  for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < n; f += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(fp, static_cast<unsigned long long>(
                      splitmix64(static_cast<uint64_t>(f) * 0xD1B54A32D192ED03ull ^ static_cast<uint64_t>(own[f]))));
}

__global__ void qso_prep_kernel(lya_quasars q, Forests Q, unsigned* err, unsigned long long* fp) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < q.n;
       k += (int64_t)gridDim.x * blockDim.x) {
    const double ra = q.ra[k], dec = q.dec[k], d = q.dist[k];
    const float w = q.weight[k];
    const bool fin = isfinite(ra) && isfinite(dec) && isfinite(d) && d > 0.0 && isfinite(w);
    if (!fin) atomicOr(err, FLAG_NONFINITE);
    if (fin && w < 0.0f) atomicOr(err, FLAG_NEGATIVE_W);
    double sr = 0, cr = 1, sd = 0, cd = 1;
    if (fin) {
      sincos(ra, &sr, &cr);
      sincos(dec, &sd, &cd);
    }
    Q.ux[k] = cd * cr;
    Q.uy[k] = cd * sr;
    Q.uz[k] = sd;
    Q.dmin[k] = fin ? d : 1.0;
    Q.len[k] = (fin && w >= 0.0f) ? 1 : 0;
    auto bits = [](double v) { return static_cast<uint64_t>(__double_as_longlong(v)); };
    uint64_t x = splitmix64(static_cast<uint64_t>(k) * 0x9E3779B97F4A7C15ull ^ static_cast<uint64_t>(Q.len[k]));
    x = splitmix64(x ^ bits(ra));
    x = splitmix64(x ^ bits(dec));
    x = splitmix64(x ^ bits(d));
    atomicAdd(fp, static_cast<unsigned long long>(x));
  }
}

// Number of entries of the sorted shared array a[0..n) strictly below v.
__device__ __forceinline__ int count_below_s(const float* a, int n, float v) {
  int lo = 0, hi = n;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (a[mid] < v) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// Window geometry of one (forest, quasar) pair against the forest's staged
// packed distances xs[0..n): as pair_geo, searched in shared memory.
__device__ __forceinline__ XGeo pair_geo_s(const XcfArgs& A, int a, int q, const float* xs, int n) {
  const double ax = A.F.ux[a], ay = A.F.uy[a], az = A.F.uz[a];
  const double qx = A.Q.ux[q], qy = A.Q.uy[q], qz = A.Q.uz[q];
  const double dx = ax - qx, dy = ay - qy, dz = az - qz;
  const double sx = ax + qx, sy = ay + qy, sz = az + qz;
  const double s = 0.5 * sqrt(dx * dx + dy * dy + dz * dz);
  const double c = 0.5 * sqrt(sx * sx + sy * sy + sz * sz);
  const double inv_dpar = A.n_par / (2.0 * A.r_par_max), inv_dperp = A.n_perp / A.r_perp_max;
  const double dref = static_cast<double>(A.F.dref[a]), dq = A.Q.dmin[q];
  XGeo g;
  g.cP = static_cast<float>(c * inv_dpar);
  g.sP = static_cast<float>(s * inv_dperp);
  g.X0 = static_cast<float>((dref - dq) * c * inv_dpar + 0.5 * A.n_par);
  g.Y0 = static_cast<float>((dref + dq) * s * inv_dperp);
  const double xq = dq - dref;
  const double half = A.r_par_max / c;
  const double lo = xq - half - 0.5;
  double hi = xq + half + 0.5;
  if (s > 0.0) hi = fmin(hi, A.r_perp_max / s - dref - dq + 0.5);
  g.i0 = count_below_s(xs, n, static_cast<float>(lo));
  g.i1 = (hi > lo) ? count_below_s(xs, n, static_cast<float>(hi)) : g.i0;
  if (g.i1 < g.i0) g.i1 = g.i0;
  return g;
}

// Stage forest f for a block: packed distances xs[0..n) and the FP64 prefix
// sums P1[k] = sum_{j<k} v1_j, P2[k] = sum_{j<k} v2_j (P[0] = 0), v given by
// load(j) -> (v1, v2).  Ends with __syncthreads.
template <class Load>
__device__ __forceinline__ void stage_prefix(const Pix* fp, int n, float* xs, double* P1, double* P2, Load load) {
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    xs[k] = fp[k].x;
    const double2 v = load(k);
    P1[k + 1] = v.x;
    P2[k + 1] = v.y;
  }
  if (threadIdx.x == 0) {
    P1[0] = 0.0;
    P2[0] = 0.0;
  }
  __syncthreads();
  const int wi = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (wi < 2) {
    double* P = (wi == 0) ? P1 + 1 : P2 + 1;
    double carry = 0.0;
    for (int base = 0; base < n; base += 32) {
      const int k = base + lane;
      double v = (k < n) ? P[k] : 0.0;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const double o = __shfl_up_sync(kFull, v, d);
        if (lane >= d) v += o;
      }
      v += carry;
      if (k < n) P[k] = v;
      carry = __shfl_sync(kFull, v, 31);
    }
  }
  __syncthreads();
}

// Runs of equal bins in a chunk: for the last lane of a run, the first index
// of the run in this chunk (returns -1 for other lanes).
__device__ __forceinline__ int run_start(int bin, int lane) {
  const int prev = __shfl_up_sync(kFull, bin, 1);
  const int nxt = __shfl_down_sync(kFull, bin, 1);
  const bool head = bin >= 0 && (lane == 0 || prev != bin);
  const bool tail = bin >= 0 && (lane == 31 || nxt != bin);
  const unsigned hm = __ballot_sync(kFull, head);
  if (!tail) return -1;
  return 31 - __clz(hm & (0xffffffffu >> (31 - lane)));
}

// One block per forest (grid-stride): the forest's packed pixels are staged in
// shared memory; warps take 32 of the forest's quasars at a time, one pair's
// geometry per lane (FP64), then walk each pair's window together.  Per lane
// the products w_q w_j and w_q (w delta)_j are exact FP32 pairs (TwoProduct),
// a segmented TwoSum scan forms each run's sum, and the run's last lane adds
// it to the block's double-float histogram: no FP64 arithmetic per pixel.
__global__ void __launch_bounds__(kXCW * 32, 2) xcf_kernel(XcfArgs A, int cap) {
  // [nb] (num hi, num lo, w hi, w lo) | per team: staged pixels [cap], xs [cap]
  extern __shared__ float4 xs4[];
  const int nb = A.n_par * A.n_perp;
  float4* hist = xs4;
  for (int k = threadIdx.x; k < nb; k += blockDim.x) hist[k] = make_float4(0.f, 0.f, 0.f, 0.f);
  __syncthreads();
  // two teams of kXCW / 2 warps, each on its own forests with its own staging
  // buffer and barrier, so that one team's wait for its slowest warp leaves
  // the other team issuing; both add to the block's histogram
  constexpr int kTeamWarps = kXCW / 2;
  const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
  const int team = wi / kTeamWarps, tw = wi % kTeamWarps, tt = threadIdx.x % (kTeamWarps * 32);
  Pix* sp = reinterpret_cast<Pix*>(xs4 + nb) + static_cast<size_t>(team) * cap;
  float* xs = reinterpret_cast<float*>(reinterpret_cast<Pix*>(xs4 + nb) + 2 * static_cast<size_t>(cap)) +
              static_cast<size_t>(team) * cap;
  for (int64_t f = 2 * static_cast<int64_t>(blockIdx.x) + team; f < A.F.n; f += 2 * static_cast<int64_t>(gridDim.x)) {
    const int64_t q0 = A.qoff[f], q1 = A.qoff[f + 1];
    const int n = A.F.len[f];
    if (q1 <= q0 || n <= 0 || n > cap) continue;   // uniform over the team
    team_sync(1 + team, kTeamWarps * 32);          // the team's previous forest's readers are done
    const Pix* fp = A.pix + A.F.off[f];
    for (int k = tt; k < n; k += kTeamWarps * 32) {
      const Pix P = fp[k];
      sp[k] = P;
      xs[k] = P.x;
    }
    team_sync(1 + team, kTeamWarps * 32);
    for (int64_t qb = q0 + static_cast<int64_t>(tw) * 32; qb < q1; qb += kTeamWarps * 32) {
      XGeo g{0.f, 0.f, 0.f, 0.f, 0, 0};
      float wq = 0.f;
      const int64_t k = qb + lane;
      if (k < q1) {
        const int q = A.pairs[k].y;
        if (q >= 0 && A.Q.len[q] > 0) {
          g = pair_geo_s(A, static_cast<int>(f), q, xs, n);
          wq = A.wq[q];
        }
      }
      const int nq = static_cast<int>((q1 - qb < 32) ? (q1 - qb) : 32);
      for (int t = 0; t < nq; ++t) {
        const int i0 = __shfl_sync(kFull, g.i0, t), i1 = __shfl_sync(kFull, g.i1, t);
        if (i1 <= i0) continue;
        XGeo h;
        h.cP = __shfl_sync(kFull, g.cP, t);
        h.sP = __shfl_sync(kFull, g.sP, t);
        h.X0 = __shfl_sync(kFull, g.X0, t);
        h.Y0 = __shfl_sync(kFull, g.Y0, t);
        const float wqt = __shfl_sync(kFull, wq, t);
        for (int base = i0; base < i1; base += 32) {
          const int j = base + lane;
          int bin = -1;
          float hn = 0.f, ln = 0.f, hw = 0.f, lw = 0.f;
          if (j < i1) {
            const Pix P = sp[j];
            bin = pixel_bin(h, P.x, A.n_par, A.n_perp);
            if (bin >= 0) {
              hn = wqt * P.z;
              ln = fmaf(wqt, P.z, -hn);
              hw = wqt * P.y;
              lw = fmaf(wqt, P.y, -hw);
            }
          }
          if (run_scan(bin, lane, hn, ln, hw, lw)) {
            df_atomic_add(reinterpret_cast<float2*>(&hist[bin]), hn, ln, A.err);
            df_atomic_add(reinterpret_cast<float2*>(&hist[bin]) + 1, hw, lw, A.err);
          }
        }
      }
    }
  }
  __syncthreads();
  for (int k = threadIdx.x; k < nb; k += blockDim.x) {
    const float4 v = hist[k];
    const double sn = static_cast<double>(v.x) + static_cast<double>(v.y);
    const double sw = static_cast<double>(v.z) + static_cast<double>(v.w);
    if (sn != 0.0) red_add_f64_global(A.num + k, sn);
    if (sw != 0.0) red_add_f64_global(A.wsum + k, sw);
  }
}

// one warp per kept (forest, quasar) pair; per warp: run list of `cap` entries
__global__ void __launch_bounds__(kXW * 32) xdm_kernel(XcfArgs A, int cap) {
  extern __shared__ double dsh[];
  const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5, nwb = blockDim.x >> 5;
  double* lal = dsh + static_cast<size_t>(wi) * 2 * cap;
  double* lbe = lal + cap;
  int* lA = reinterpret_cast<int*>(dsh + static_cast<size_t>(nwb) * 2 * cap) + static_cast<size_t>(wi) * cap;
  const int nb = A.n_par * A.n_perp;
  const int all = A.p_subsample >= 1.0;
  const uint64_t thr = static_cast<uint64_t>(A.p_subsample * 18446744073709551616.0);
  const int64_t nw = static_cast<int64_t>(gridDim.x) * nwb;
  for (int64_t k = blockIdx.x * (int64_t)nwb + wi; k < A.n_pairs; k += nw) {
    const int2 pr = A.pairs[k];
    const int a = pr.x, q = pr.y;
    if (a < 0 || q < 0) continue;
    if (!all && !(splitmix64(A.seed ^ ((static_cast<uint64_t>(a) << 32) | static_cast<uint64_t>(q))) < thr)) continue;
    const int n = A.F.len[a];
    if (n <= 0 || A.Q.len[q] <= 0) continue;
    const Pix* fp = A.pix + A.F.off[a];
    const XGeo g = pair_geo(A, a, q, fp, n);
    int L = 0, lastA = -1;
    for (int base = g.i0; base < g.i1; base += 32) {
      const int i = base + lane;
      int bin = -1;
      float ha = 0.f, la = 0.f, hb = 0.f, lb = 0.f;
      if (i < g.i1) {
        const Pix P = fp[i];
        bin = pixel_bin(g, P.x, A.n_par, A.n_perp);
        if (bin >= 0) {
          ha = P.y;
          hb = P.y * P.w;
          lb = fmaf(P.y, P.w, -hb);
        }
      }
      const bool tail = run_scan(bin, lane, ha, la, hb, lb);
      const unsigned tm = __ballot_sync(kFull, tail);
      if (tm) {
        const int fbin = __shfl_sync(kFull, bin, __ffs(tm) - 1);
        const int merged = (fbin == lastA) ? 1 : 0;   // run continued from the previous chunk
        if (tail) {
          const int r = __popc(tm & ((1u << lane) - 1u));
          const double va = static_cast<double>(ha) + static_cast<double>(la);
          const double vb = static_cast<double>(hb) + static_cast<double>(lb);
          if (r == 0 && merged) {
            lal[L - 1] += va;
            lbe[L - 1] += vb;
          } else {
            const int slot = L + r - merged;
            lA[slot] = bin;
            lal[slot] = va;
            lbe[slot] = vb;
          }
        }
        lastA = __shfl_sync(kFull, bin, 31 - __clz(tm));
        L += __popc(tm) - merged;
      }
      __syncwarp();
    }
    if (L == 0) continue;
    const double wq = static_cast<double>(A.wq[q]);
    const double Wa = A.F.wsum[a], Sa = A.F.ssum[a];
    const bool use_w = A.eta_mean_slope && Wa > 0.0;
    const bool use_s = use_w && Sa > 0.0;
    const double iW = use_w ? wq / Wa : 0.0, iS = use_s ? wq / Sa : 0.0;
    for (int r = lane; r < L; r += 32) red_add_f64_global(A.wdm + lA[r], wq * lal[r]);
    for (int r = 0; r < L; ++r) {
      const double ar = lal[r], br = lbe[r];
      double* row = A.G + static_cast<int64_t>(lA[r]) * nb;
      for (int c = r + lane; c < L; c += 32) {
        double v = -(ar * lal[c]) * iW - (br * lbe[c]) * iS;
        if (c == r) v += wq * ar;
        if (v != 0.0) red_add_f64_global(row + lA[c], v);
      }
    }
    __syncwarp();
  }
}

// One block per forest (grid-stride), one warp per pixel i, lanes over j > i.
// p = floor((d_j - d_i) / D) is taken from the FP32 packed distances when that
// value lies farther than `guard` from an integer (the FP32 error is below
// guard / 2), else from the FP64 division of the definition, so every bin is
// the definition's.  Runs [j0, j1] of equal bins add (w d)_i (P[j1+1] - P[j0]).
__global__ void __launch_bounds__(256) xi1d_kernel(X1Args A, const Pix* pix) {
  extern __shared__ double ssh[];   // [2 n_bins] | P_w [cap+1] | P_wd [cap+1] | d [cap] | xs [cap] (float)
  const int cap = A.max_len;
  double* hn = ssh;
  double* hw = ssh + A.n_bins;
  double* Pw = hw + A.n_bins;
  double* Pwd = Pw + cap + 1;
  double* sd = Pwd + cap + 1;
  float* xs = reinterpret_cast<float*>(sd + cap);
  for (int k = threadIdx.x; k < 2 * A.n_bins; k += blockDim.x) ssh[k] = 0.0;
  const double dr = A.r_max / A.n_bins;
  const float inv_dr = static_cast<float>(A.n_bins / A.r_max);
  const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5, nwb = blockDim.x >> 5;
  for (int64_t f = blockIdx.x; f < A.F.n; f += gridDim.x) {
    const int n = A.F.len[f];
    if (n < 2 || n > cap) continue;   // uniform over the block
    __syncthreads();
    const int64_t o = A.F.off[f];
    for (int k = threadIdx.x; k < n; k += blockDim.x) sd[k] = A.dist[o + k];
    stage_prefix(pix + o, n, xs, Pw, Pwd, [&](int k) {
      const double w = static_cast<double>(A.weight[o + k]);
      return make_double2(w, w * static_cast<double>(A.delta[o + k]));
    });
    // |FP32 value - exact quotient| < 2^-22 (2 xs_max + r_max) / D + 2^-22 n_bins  (half of the guard)
    const float guard = 2.384185791015625e-7f * ((2.0f * xs[n - 1] + static_cast<float>(A.r_max)) * inv_dr +
                                                 static_cast<float>(A.n_bins)) + 1e-6f;
    for (int i = wi; i < n - 1; i += nwb) {
      const float xi = xs[i];
      const double di = sd[i];
      const double wgt = static_cast<double>(A.weight[o + i]);
      const double wdi = wgt * static_cast<double>(A.delta[o + i]);
      for (int base = i + 1; base < n; base += 32) {
        const int j = base + lane;
        int bin = -1;
        bool beyond = false;
        if (j < n) {
          const float t = (xs[j] - xi) * inv_dr;
          const float fl = floorf(t);
          double pe = fl;
          if (t - fl < guard || fl + 1.0f - t < guard) pe = floor((sd[j] - di) / dr);
          if (pe < static_cast<double>(A.n_bins)) bin = static_cast<int>(pe); else beyond = true;
        }
        const int r0 = run_start(bin, lane);
        if (r0 >= 0) {
          const int j0 = base + r0;
          atomicAdd(&hn[bin], wdi * (Pwd[j + 1] - Pwd[j0]));
          atomicAdd(&hw[bin], wgt * (Pw[j + 1] - Pw[j0]));
        }
        if (__any_sync(kFull, beyond)) break;
      }
    }
  }
  __syncthreads();
  for (int k = threadIdx.x; k < A.n_bins; k += blockDim.x) {
    if (hn[k] != 0.0) red_add_f64_global(A.num + k, hn[k]);
    if (hw[k] != 0.0) red_add_f64_global(A.wsum + k, hw[k]);
  }
}

int grid_for(int64_t n, int threads) {
  int64_t b = (n + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > 1 << 16) b = 1 << 16;
  return static_cast<int>(b);
}

}  // namespace

int xcf_smem_bytes(int nb, int max_len) {
  const int cap = std::max(max_len, 1);
  return 16 * nb + 2 * 20 * cap;
}

int xdm_warps(const DevInfo& dev, int max_len) {
  const int64_t per_warp = 20LL * std::max(max_len, 1);
  int w = static_cast<int>(std::min<int64_t>(kXW, dev.smem_optin / per_warp));
  return w;   // 0: forests too long for the run lists
}

int xi1d_smem_bytes(int n_bins, int max_len) {
  const int cap = std::max(max_len, 1);
  return 16 * n_bins + 16 * (cap + 1) + 12 * cap;
}

cudaError_t launch_qso_prep(const lya_quasars& q, Forests Q, unsigned* err, unsigned long long* fp,
                            cudaStream_t s) {
  if (q.n <= 0) return cudaSuccess;
  LYA_COUNT(1), qso_prep_kernel<<<grid_for(q.n, 256), 256, 0, s>>>(q, Q, err, fp);
  return cudaGetLastError();
}

cudaError_t launch_own_hash(const int64_t* own, int64_t n, unsigned long long* fp, cudaStream_t s) {
  if (!own || n <= 0) return cudaSuccess;
  LYA_COUNT(1), own_hash_kernel<<<grid_for(n, 256), 256, 0, s>>>(own, n, fp);
  return cudaGetLastError();
}

cudaError_t launch_xcf(const XcfArgs& a, const DevInfo& dev, cudaStream_t s) {
  if (a.n_pairs == 0) return cudaSuccess;
  const int cap = std::max(a.max_len, 1);
  const int smem = xcf_smem_bytes(a.n_par * a.n_perp, cap);
  cudaError_t e = set_max_dynamic_smem(reinterpret_cast<const void*>(xcf_kernel), smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, xcf_kernel, kXCW * 32, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  const int blocks = static_cast<int>(std::min<int64_t>(static_cast<int64_t>(dev.sms) * per_sm, (a.F.n + 1) / 2));
  LYA_COUNT(1), xcf_kernel<<<blocks, kXCW * 32, smem, s>>>(a, cap);
  return cudaGetLastError();
}

cudaError_t launch_xdm(const XcfArgs& a, const DevInfo& dev, cudaStream_t s) {
  if (a.n_pairs == 0 || a.p_subsample <= 0.0) return cudaSuccess;
  const int warps = xdm_warps(dev, a.max_len);
  if (warps < 1) return cudaErrorInvalidConfiguration;
  const int cap = std::max(a.max_len, 1);
  const int smem = warps * 20 * cap;
  cudaError_t e = set_max_dynamic_smem(reinterpret_cast<const void*>(xdm_kernel), smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, xdm_kernel, warps * 32, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  const int64_t want = (a.n_pairs + warps - 1) / warps;
  const int blocks = static_cast<int>(std::min<int64_t>(static_cast<int64_t>(dev.sms) * per_sm, want));
  LYA_COUNT(1), xdm_kernel<<<blocks, warps * 32, smem, s>>>(a, cap);
  return cudaGetLastError();
}

cudaError_t launch_xi1d(const X1Args& a, const Pix* pix, const DevInfo& dev, cudaStream_t s) {
  if (a.F.n == 0) return cudaSuccess;
  const int smem = xi1d_smem_bytes(a.n_bins, a.max_len);
  cudaError_t e = set_max_dynamic_smem(reinterpret_cast<const void*>(xi1d_kernel), smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, xi1d_kernel, 256, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  const int blocks = static_cast<int>(std::min<int64_t>(static_cast<int64_t>(dev.sms) * per_sm, a.F.n));
  LYA_COUNT(1), xi1d_kernel<<<blocks, 256, smem, s>>>(a, pix);
  return cudaGetLastError();
}

}  // namespace lya
