// Anisotropic three-point estimator, Eq. (2.8) (Section 2.3):
//   xi3_A = sum_A (w d)_i (w d)_j (w d)_k / sum_A w_i w_j w_k
// over pixel triplets of three distinct forests.  A record is a main vertex i
// with r1 = x_j - x_i, r2 = x_k - x_i (x = d n), binned in (|r1|, |r2|,
// cos alpha, theta1, theta2) and flattened as
//   A = (((i_r1 n_r + i_r2) n_alpha + i_alpha) n_theta + i_theta1) n_theta + i_theta2,
// theta the angle to the main vertex's line of sight, alpha the angle between
// r1 and r2.  Every pixel is a main vertex, the other two pixels take
// (r1, r2) in both orders, and a record needs |r1|, |r2| < r_max.
//
// One block per main-vertex pixel (work taken from an atomic counter):
//  1. gather: for every forest in the vertex forest's neighbour list, the
//     pixels within r_max of the vertex (a contiguous range of the sorted
//     distances, cut by binary search, then tested exactly) go to shared
//     memory with r in FP32 and their |r| and theta bins computed in FP64;
//  2. pairs: each warp holds 32 candidates q in registers and walks the
//     candidates p < q (one shared-memory read per p for the whole warp);
//     pixels of the same forest are skipped; cos alpha is FP32; the record and its
//     mirror (sides swapped) are added once, to the bin whose (r, theta) key
//     of side 1 is not above side 2's, with weight 2 when both keys are equal;
//     sums are FP32 products added to FP64 bin sums with global atomics;
//  3. a finalize kernel copies each canonical bin to its mirror and forms xi.
// A counting pass first finds the largest neighbour list, and the block's
// shared-memory capacity is sized to it (fewer blocks per SM when lists are
// long); a vertex beyond what one block can hold raises a device flag
// (reported as LYA_ERR_TOO_LARGE) instead of being truncated silently.
#include <algorithm>
#include <math.h>

#include "lya_internal.cuh"

namespace lya {
namespace {

constexpr int kX3Threads = 256;

__global__ void x3_degree_kernel(const int2* pairs, int64_t n, int32_t* deg) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int2 p = pairs[k];
    if (p.x < 0) continue;
    atomicAdd(&deg[p.x], 1);
    atomicAdd(&deg[p.y], 1);
  }
}

__global__ void x3_fill_kernel(const int2* pairs, int64_t n, const int64_t* start, int32_t* cursor,
                               int32_t* nbr) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int2 p = pairs[k];
    if (p.x < 0) continue;
    nbr[start[p.x] + atomicAdd(&cursor[p.x], 1)] = p.y;
    nbr[start[p.y] + atomicAdd(&cursor[p.y], 1)] = p.x;
  }
}

__global__ void x3_scan_kernel(const int32_t* in, int64_t n, int64_t* out) {
  __shared__ int64_t part[1024];
  const int t = threadIdx.x;
  const int64_t chunk = (n + blockDim.x - 1) / blockDim.x;
  const int64_t b = t * chunk, e = min(n, b + chunk);
  int64_t s = 0;
  for (int64_t k = b; k < e; ++k) s += in[k];
  part[t] = s;
  __syncthreads();
  if (t == 0) {
    int64_t run = 0;
    for (int k = 0; k < (int)blockDim.x; ++k) {
      const int64_t v = part[k];
      part[k] = run;
      run += v;
    }
    out[n] = run;
  }
  __syncthreads();
  int64_t run = part[t];
  for (int64_t k = b; k < e; ++k) {
    out[k] = run;
    run += in[k];
  }
}

// forest of packed pixel g: the last forest whose first pixel is <= g
__device__ __forceinline__ int forest_of(const Forests& F, int64_t g) {
  int lo = 0, hi = static_cast<int>(F.n) - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (F.off[mid] <= g) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__global__ void __launch_bounds__(kX3Threads) xi3_kernel(X3Args A, const int32_t* nbr, const int64_t* nstart,
                                                         int cap, unsigned long long* counter, unsigned* err) {
  extern __shared__ __align__(16) unsigned char sm[];
  float4* cr = reinterpret_cast<float4*>(sm);                  // r (FP32) and 1 / |r|
  float2* cw = reinterpret_cast<float2*>(cr + cap);            // (w d, w)
  int2* ck = reinterpret_cast<int2*>(cw + cap);                // ((radial bin << 16) | theta bin, forest)
  __shared__ int s_n;
  __shared__ long long s_item;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nwarps = blockDim.x >> 5;
  const double rmax = A.r_max, rmax2 = rmax * rmax;
  const double inv_dr = A.n_r / rmax, inv_dt = A.n_theta / M_PI;
  const float half_na = 0.5f * static_cast<float>(A.n_alpha);
  const int nr = A.n_r, nt = A.n_theta, na = A.n_alpha;
  for (;;) {
    if (tid == 0) {
      s_item = static_cast<long long>(atomicAdd(counter, 1ull));
      s_n = 0;
    }
    __syncthreads();
    const long long g = s_item;
    if (g >= A.n_pix) break;
    const int f = forest_of(A.F, g);
    const int64_t i_in = g - A.F.off[f];
    if (i_in >= A.F.len[f]) {    // pixel of a forest that failed the input checks
      __syncthreads();
      continue;
    }
    const double nax = A.F.ux[f], nay = A.F.uy[f], naz = A.F.uz[f];
    const double di = A.dist[g];
    const double xi = di * nax, yi = di * nay, zi = di * naz;
    const Pix pv = A.pix[g];
    const float w_i = pv.y, wd_i = pv.z;
    // 1. gather the vertex's neighbours within r_max
    for (int64_t e = nstart[f] + wid; e < nstart[f + 1]; e += nwarps) {
      const int o = nbr[e];
      const int no = A.F.len[o];
      if (no == 0) continue;
      const double c = nax * A.F.ux[o] + nay * A.F.uy[o] + naz * A.F.uz[o];
      const double disc = rmax2 - di * di * fmax(0.0, 1.0 - c * c);
      if (!(disc > 0.0)) continue;
      const double sq = sqrt(disc);
      const Pix* po = A.pix + A.F.off[o];
      const double ref = A.F.dref[o];
      const float lo = static_cast<float>(di * c - sq - ref) - 1e-2f;
      const float hi = static_cast<float>(di * c + sq - ref) + 1e-2f;
      const int jlo = count_below(po, no, lo), jhi = count_below(po, no, hi);
      for (int j = jlo + lane; j < jhi; j += 32) {
        const double dj = A.dist[A.F.off[o] + j];
        const double dx = dj * A.F.ux[o] - xi, dy = dj * A.F.uy[o] - yi, dz = dj * A.F.uz[o] - zi;
        const double r2 = dx * dx + dy * dy + dz * dz;
        if (!(r2 < rmax2) || !(r2 > 0.0)) continue;
        const int slot = atomicAdd(&s_n, 1);
        if (slot >= cap) continue;
        const double r = sqrt(r2);
        const double ct = (dx * nax + dy * nay + dz * naz) / r;
        const int ir = min(static_cast<int>(r * inv_dr), nr - 1);
        const int it = min(static_cast<int>(acos(fmin(1.0, fmax(-1.0, ct))) * inv_dt), nt - 1);
        const Pix q = po[j];
        cr[slot] = make_float4(static_cast<float>(dx), static_cast<float>(dy), static_cast<float>(dz),
                               static_cast<float>(1.0 / r));
        cw[slot] = make_float2(q.z, q.y);
        ck[slot] = make_int2((ir << 16) | it, o);
      }
    }
    __syncthreads();
    const int P = s_n;
    if (P > cap && tid == 0) atomicOr(err, FLAG_X3_CAP);
    // 2. unordered pairs (p < q) of neighbours from two distinct forests: a
    //    warp holds a tile of 32 candidates q in registers (one per lane) and
    //    walks the candidates p below them, each read once for the whole warp
    if (P <= cap) {
      for (int q0 = wid * 32; q0 < P; q0 += nwarps * 32) {
        const int q = q0 + lane;
        const bool qv = q < P;
        const float4 rq = qv ? cr[q] : make_float4(0.f, 0.f, 0.f, 0.f);
        const float2 wq = qv ? cw[q] : make_float2(0.f, 0.f);
        const int2 kq = qv ? ck[q] : make_int2(0, -1);
        const float wdq = wq.x * wd_i, wwq = wq.y * w_i;
        const int qr = kq.x >> 16, qt = kq.x & 0xffff;
        const int pend = min(q0 + 32, P);
        for (int p = 0; p < pend; ++p) {
          const float4 rp = cr[p];
          const int2 kp = ck[p];
          if (!qv || p >= q || kp.y == kq.y) continue;
          const float2 wp = cw[p];
          const float ca = (rp.x * rq.x + rp.y * rq.y + rp.z * rq.z) * (rp.w * rq.w);
          const int ia = min(max(static_cast<int>(floorf((ca + 1.0f) * half_na)), 0), na - 1);
          const int pr = kp.x >> 16, pt = kp.x & 0xffff;
          int r1, t1, r2, t2;
          if (kp.x <= kq.x) { r1 = pr; t1 = pt; r2 = qr; t2 = qt; } else { r1 = qr; t1 = qt; r2 = pr; t2 = pt; }
          const float mult = (kp.x == kq.x) ? 2.f : 1.f;
          const int64_t bin = (((static_cast<int64_t>(r1) * nr + r2) * na + ia) * nt + t1) * nt + t2;
          red_add_f64_global(A.num + bin, static_cast<double>(wp.x * wdq * mult));
          red_add_f64_global(A.wsum + bin, static_cast<double>(wp.y * wwq * mult));
        }
      }
    }
    __syncthreads();
  }
}

// largest number of neighbours within r_max of any main vertex (the same
// exact FP64 test as the gather of xi3_kernel), one warp per vertex pixel
__global__ void xi3_count_kernel(X3Args A, const int32_t* nbr, const int64_t* nstart, int* max_count) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const double rmax2 = A.r_max * A.r_max;
  int best = 0;
  for (int64_t g = warp; g < A.n_pix; g += nw) {
    const int f = forest_of(A.F, g);
    if (g - A.F.off[f] >= A.F.len[f]) continue;
    const double nax = A.F.ux[f], nay = A.F.uy[f], naz = A.F.uz[f];
    const double di = A.dist[g];
    const double xi = di * nax, yi = di * nay, zi = di * naz;
    int cnt = 0;
    for (int64_t e = nstart[f]; e < nstart[f + 1]; ++e) {
      const int o = nbr[e];
      const int no = A.F.len[o];
      if (no == 0) continue;
      const double c = nax * A.F.ux[o] + nay * A.F.uy[o] + naz * A.F.uz[o];
      const double disc = rmax2 - di * di * fmax(0.0, 1.0 - c * c);
      if (!(disc > 0.0)) continue;
      const double sq = sqrt(disc);
      const Pix* po = A.pix + A.F.off[o];
      const double ref = A.F.dref[o];
      const float lo = static_cast<float>(di * c - sq - ref) - 1e-2f;
      const float hi = static_cast<float>(di * c + sq - ref) + 1e-2f;
      const int jlo = count_below(po, no, lo), jhi = count_below(po, no, hi);
      for (int j = jlo + lane; j < jhi; j += 32) {
        const double dj = A.dist[A.F.off[o] + j];
        const double dx = dj * A.F.ux[o] - xi, dy = dj * A.F.uy[o] - yi, dz = dj * A.F.uz[o] - zi;
        const double r2 = dx * dx + dy * dy + dz * dz;
        cnt += (r2 < rmax2 && r2 > 0.0) ? 1 : 0;
      }
    }
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    best = max(best, cnt);
  }
  if (lane == 0 && best > 0) atomicMax(max_count, best);
}

// copy each canonical bin (side-1 key <= side-2 key) to its mirror; xi = N / W
__global__ void xi3_finalize_kernel(double* num, double* wsum, double* xi, int nr, int nt, int na) {
  const int64_t n = static_cast<int64_t>(nr) * nr * na * nt * nt;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x) {
    int64_t rest = k;
    const int t2 = static_cast<int>(rest % nt); rest /= nt;
    const int t1 = static_cast<int>(rest % nt); rest /= nt;
    const int ia = static_cast<int>(rest % na); rest /= na;
    const int r2 = static_cast<int>(rest % nr); rest /= nr;
    const int r1 = static_cast<int>(rest);
    if (r1 * nt + t1 > r2 * nt + t2) {
      const int64_t m = (((static_cast<int64_t>(r2) * nr + r1) * na + ia) * nt + t2) * nt + t1;
      num[k] = num[m];
      wsum[k] = wsum[m];
    }
  }
}

__global__ void xi3_ratio_kernel(const double* num, const double* wsum, double* xi, int64_t n) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x)
    xi[k] = (wsum[k] != 0.0) ? num[k] / wsum[k] : 0.0;
}

int grid_for(int64_t n, int threads) {
  int64_t b = (n + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > 1 << 16) b = 1 << 16;
  return static_cast<int>(b);
}

#define LYA_TRY(x)                    \
  do {                                \
    cudaError_t e_ = (x);             \
    if (e_ != cudaSuccess) return e_; \
  } while (0)

}  // namespace

cudaError_t run_xi3(const X3Args& a, const DevInfo& dev, void** scratch, size_t* scratch_cap, unsigned* err,
                    cudaStream_t s) {
  const int64_t nf = a.F.n, np = a.n_pairs;
  const int64_t nbins = static_cast<int64_t>(a.n_r) * a.n_r * a.n_alpha * a.n_theta * a.n_theta;
  LYA_TRY(cudaMemsetAsync(a.num, 0, nbins * 8, s));
  LYA_TRY(cudaMemsetAsync(a.wsum, 0, nbins * 8, s));
  auto al = [](size_t v) { return (v + 255) & ~size_t(255); };
  size_t o = 0;
  const size_t o_deg = o; o += al((nf + 1) * 4);
  const size_t o_cur = o; o += al((nf + 1) * 4);
  const size_t o_start = o; o += al((nf + 1) * 8);
  const size_t o_nbr = o; o += al(std::max<int64_t>(2 * np, 1) * 4);
  const size_t o_misc = o; o += 256;
  LYA_TRY(grow(scratch, scratch_cap, o));
  char* sc = static_cast<char*>(*scratch);
  int32_t* deg = reinterpret_cast<int32_t*>(sc + o_deg);
  int32_t* cur = reinterpret_cast<int32_t*>(sc + o_cur);
  int64_t* start = reinterpret_cast<int64_t*>(sc + o_start);
  int32_t* nbr = reinterpret_cast<int32_t*>(sc + o_nbr);
  unsigned long long* counter = reinterpret_cast<unsigned long long*>(sc + o_misc);
  LYA_TRY(cudaMemsetAsync(deg, 0, (nf + 1) * 4, s));
  LYA_TRY(cudaMemsetAsync(cur, 0, (nf + 1) * 4, s));
  LYA_TRY(cudaMemsetAsync(counter, 0, 8, s));
  if (np > 0) LYA_COUNT(1), x3_degree_kernel<<<grid_for(np, 256), 256, 0, s>>>(a.pairs, np, deg);
  LYA_COUNT(1), x3_scan_kernel<<<1, 1024, 0, s>>>(deg, nf, start);
  if (np > 0) LYA_COUNT(1), x3_fill_kernel<<<grid_for(np, 256), 256, 0, s>>>(a.pairs, np, start, cur, nbr);
  LYA_TRY(cudaGetLastError());
  // neighbour capacity per block: the largest neighbour list of any vertex
  // (counting pass, synchronising), at least what leaves three blocks per SM;
  // a list beyond one block's shared memory is reported, not truncated
  const int per_cand = 32;
  int* dmax = reinterpret_cast<int*>(sc + o_misc + 64);
  LYA_TRY(cudaMemsetAsync(dmax, 0, 4, s));
  if (a.n_pix > 0 && nf > 0)
    LYA_COUNT(1), xi3_count_kernel<<<dev.sms * 8, 256, 0, s>>>(a, nbr, start, dmax);
  int hmax = 0;
  LYA_TRY(cudaMemcpyAsync(&hmax, dmax, 4, cudaMemcpyDeviceToHost, s));
  LYA_TRY(cudaStreamSynchronize(s));
  const int cap_max = (dev.smem_optin - 1024) / per_cand;
  int cap = std::max(std::min(cap_max, (dev.smem_per_sm / 3 - 2048) / per_cand), std::min(hmax, cap_max));
  cap = std::max(cap, 256);
  const int smem = cap * per_cand;
  if (smem > dev.smem_optin) return cudaErrorInvalidValue;
  LYA_TRY(set_max_dynamic_smem(reinterpret_cast<const void*>(xi3_kernel), smem));
  int per_sm = 0;
  LYA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, xi3_kernel, kX3Threads, smem));
  if (per_sm < 1) return cudaErrorInvalidValue;
  if (a.n_pix > 0 && nf > 0)
    LYA_COUNT(1), xi3_kernel<<<per_sm * dev.sms, kX3Threads, smem, s>>>(a, nbr, start, cap, counter, err);
  LYA_TRY(cudaGetLastError());
  LYA_COUNT(1), xi3_finalize_kernel<<<grid_for(nbins, 256), 256, 0, s>>>(a.num, a.wsum, a.xi, a.n_r, a.n_theta,
                                                                        a.n_alpha);
  if (a.xi) LYA_COUNT(1), xi3_ratio_kernel<<<grid_for(nbins, 256), 256, 0, s>>>(a.num, a.wsum, a.xi, nbins);
  return cudaGetLastError();
}

}  // namespace lya
