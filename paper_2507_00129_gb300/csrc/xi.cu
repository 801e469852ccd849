// Pixel-pair histogram of Eq. (2.4): for every forest pair (a, b) and every
// pixel pair (i in a, j in b), bin (r_par, r_perp) and add (w d)_i (w d)_j and
// w_i w_j to the bin (Section 2.1).
//
// Mixed kernel (LYA_PREC_MIXED), persistent, one forest pair per warp at a time:
//  * forest b is staged in the warp's shared-memory buffer with coalesced
//    16-byte loads; 32 pixels of forest a sit in registers (one per lane);
//  * separations are FP32 fused multiply-adds on distances relative to a
//    per-forest reference (multiple of 2^-10, so the reference differences and
//    sums entering the pair constants are exact FP32 numbers):
//        r_par/D  = | d~_j * (-c/D) + ((d~_i * c/D) + (ref_a - ref_b) c/D) |
//        r_perp/D =   d~_j *   s/D  + ((d~_i * s/D) + (ref_a + ref_b) s/D)
//  * floor() is an FP32 add rounded toward -inf of 2^23 (the integer lands in
//    the low mantissa bits), so the bin index needs no float->int conversion;
//  * each lane walks j and keeps the current bin's run sums in registers; a
//    run that ends (the bin changed) is held in registers, and the warp adds
//    the held runs to its chunk histogram, which covers only the rows of the
//    pair's r_perp band, when a lane that holds one ends another: exact
//    two-word fixed point summed with native 32-bit shared-memory reductions
//    (a lane without a held run aims them at its own dummy word);
//  * every two 32-pixel chunks of forest a the integer sums are folded into a
//    warp-private compensated FP32 (TwoSum) band accumulator, which survives
//    across consecutive pairs with the same first band row (the pair list is
//    ordered for this) and is added to the FP64 bin sums in global memory when
//    the band changes;
//  * the j loop of each 32-pixel chunk of a is restricted to the pixels that
//    can be in range (distances are sorted; two binary searches).
// FP64 kernel (LYA_PREC_FP64): the same decomposition with FP64 distances,
// separations, products and shared-memory sums, mirroring the oracle's
// operation order: r = |d_i - d_j| * c, x = r * (1/D).
#include <algorithm>
#include <math.h>

#include "lya_internal.cuh"

namespace lya {
namespace {

constexpr int kHcap = 440;       // words per chunk-histogram array per warp: bins (K+1) x (n_par+1)
                                 // below kHcap - 32, then one dummy word per lane
constexpr uint32_t kM15Bits = 0x4B400000u;   // bits of 1.5 * 2^23
constexpr float kM15 = 12582912.0f;
constexpr int kAcap = 352;       // accumulator entries per warp: rows x n_par (7 rows of 50 bins;
                                 // sized with kHcap so that 14 warps fit in shared memory)
constexpr int kHcap64 = 256;     // doubles per histogram array per warp (FP64)
constexpr int kMaxSeg = 1024;    // pixel buffer cap per warp

// Knuth's TwoSum: (hi, lo) += x with the rounding error of hi + x kept in lo.
__device__ __forceinline__ void two_sum(float& hi, float& lo, float x) {
  const float s = hi + x;
  const float bp = s - hi;
  lo += (hi - (s - bp)) + (x - bp);
  hi = s;
}

// Exact two-word fixed point.  v (|v| < B) is represented as
// (hi * 2^16 + lo) * 2^-k with q = v * 2^(k-16), hi = floor(q), lo =
// round((q - hi) * 2^16) in [0, 2^16]; sc16 = 2^(k-16) is chosen per forest
// pair so that |q| < 2^21 for every run of in-grid pairs.  Sums of hi and of lo
// are kept in separate 32-bit words (no carries between them), which shared
// memory adds natively; FP32 shared-memory reductions are emulated on this
// part and far slower.
__device__ __forceinline__ void split_fixed(float v, float sc16, uint32_t& hi, uint32_t& lo) {
  // q = v * sc16 is exact (sc16 is a power of two) and |q| < 2^21
  const float hm = __fmaf_rd(v, sc16, kM15);      // 1.5 * 2^23 + floor(q)
  const float fr = fmaf(v, sc16, kM15 - hm);      // q - floor(q), exact
  const float lm = fmaf(fr, 65536.f, kM15);       // 1.5 * 2^23 + round(fr * 2^16)
  hi = __float_as_uint(hm) - kM15Bits;
  lo = __float_as_uint(lm) - kM15Bits;
}

// A lane's ended run, held in registers until the warp adds the held runs to
// the chunk histogram.
struct Held {
  uint32_t key;
  float n, w;
  bool on;
};

// Adds every lane's held run to the chunk histogram (four 32-bit reductions
// per lane; a lane without a held run adds to its own dummy word).
__device__ __forceinline__ void add_held(Held& h, uint32_t base, float scN, float scW, uint32_t dummy) {
  uint32_t nh, nl, wh, wl;
  split_fixed(h.n, scN, nh, nl);
  split_fixed(h.w, scW, wh, wl);
  const uint32_t addr = h.on ? base + (h.key << 2) : dummy;
  asm volatile(
      "{\n\t"
      "red.shared.add.u32 [%0], %1;\n\t"
      "red.shared.add.u32 [%0+%5], %2;\n\t"
      "red.shared.add.u32 [%0+%6], %3;\n\t"
      "red.shared.add.u32 [%0+%7], %4;\n\t}"
      ::"r"(addr), "r"(nh), "r"(nl), "r"(wh), "r"(wl), "n"(kHcap * 4), "n"(kHcap * 8), "n"(kHcap * 12));
  h.on = false;
}

// One pixel pair of a run walk (see chunk_runs).  A run that ends here is
// held in the lane's registers; the warp adds its held runs to the histogram
// only when some lane that already holds one ends another.  On the DESI-like
// grid a run is about seven pixels long, so the reductions come once per ~6
// steps instead of every step.
template <bool WINDOW>
__device__ __forceinline__ void run_step(const Pix& q, float cp, float sp, float uc, float us, float wdi,
                                         float wi, float pmax, float tmax, uint32_t stride, uint32_t base,
                                         float scN, float scW, uint32_t guard, uint32_t twin,
                                         uint32_t tspan, uint32_t dummy, uint32_t& cur, float& aN, float& aW,
                                         Held& held) {
  const float rp = fabsf(fmaf(-q.x, cp, uc));
  const float rt = fmaf(q.x, sp, us);
  const float pf = fminf(__fadd_rd(rp, kMagic), pmax);
  const float tf = fminf(__fadd_rd(rt, kMagic), tmax);
  uint32_t key = __float_as_uint(tf) * stride + __float_as_uint(pf);
  if (WINDOW) key = ((__float_as_uint(tf) - kMagicBits - twin) <= tspan) ? key : guard;
  const bool chg = key != cur;
  if (__any_sync(0xffffffffu, chg && held.on)) add_held(held, base, scN, scW, dummy);
  held.key = chg ? cur : held.key;
  held.n = chg ? aN : held.n;
  held.w = chg ? aW : held.w;
  held.on = held.on || chg;
  cur = key;
  aN = fmaf(wdi, q.z, chg ? 0.f : aN);
  aW = fmaf(wi, q.y, chg ? 0.f : aW);
}

// One 32-pixel chunk of forest a against pixels [jlo, jhi) of the staged
// forest b.  Each lane keeps the current bin and its running sums in
// registers; a run (consecutive j in one bin) that ends is held (see
// run_step) and later added to the shared chunk histogram.  Out-of-grid pairs
// land in the guard row / column (floor clamped with fminf); WINDOW
// additionally sends rows outside [twin, twin + tspan] to the guard.  Pixels
// are read eight at a time before the eight steps: the reductions write
// shared memory, so a later load cannot be hoisted above them.
template <bool WINDOW>
__device__ __forceinline__ void chunk_runs(const Pix* __restrict__ buf, int jlo, int jhi, float cp,
                                           float sp, float uc, float us, float wdi, float wi,
                                           float pmax, float tmax, uint32_t stride, uint32_t base,
                                           float scN, float scW, uint32_t guard, uint32_t twin,
                                           uint32_t tspan, uint32_t dummy) {
  uint32_t cur = guard;
  float aN = 0.f, aW = 0.f;
  Held held{guard, 0.f, 0.f, false};
  int j = jlo;
  for (; j + 8 <= jhi; j += 8) {
    Pix q[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) q[u] = buf[j + u];
#pragma unroll
    for (int u = 0; u < 8; ++u)
      run_step<WINDOW>(q[u], cp, sp, uc, us, wdi, wi, pmax, tmax, stride, base, scN, scW, guard, twin, tspan,
                       dummy, cur, aN, aW, held);
  }
  for (; j < jhi; ++j)
    run_step<WINDOW>(buf[j], cp, sp, uc, us, wdi, wi, pmax, tmax, stride, base, scN, scW, guard, twin, tspan,
                     dummy, cur, aN, aW, held);
  // the held runs, then the last run of every lane
  if (__any_sync(0xffffffffu, held.on)) add_held(held, base, scN, scW, dummy);
  held = Held{cur, aN, aW, true};
  add_held(held, base, scN, scW, dummy);
}

// Per-pair scale sc16 = 2^(20 - e) with 2^e <= B < 2^(e+1): every |v| < B
// maps to |q| < 2^21.
__device__ __forceinline__ float fixed_scale(float B) {
  if (!(B > 0.f) || !(B < 1e37f)) return 1.f;
  const int e = static_cast<int>((__float_as_uint(B) >> 23) & 0xFFu) - 127;
  const int ex = 20 - e + 127;
  return __uint_as_float(static_cast<uint32_t>(min(max(ex, 1), 254)) << 23);
}

struct WarpSm {
  uint32_t* h;      // chunk histogram: N hi, N lo, W hi, W lo (kHcap words each)
  float* acc;       // accumulator: N hi, N lo, W hi, W lo (kAcap each)
  Pix* buf;         // staged pixels of forest b
  uint32_t sN;      // shared address of hN
};

// chunk rows [0, nrows) x columns [0, npar) -> accumulator rows [r0, r0+nrows)
// (fixed point -> FP32 with the pair's scales); clears the whole chunk
// histogram including the guard row and column
__device__ __forceinline__ void fold_chunk(const WarpSm& w, int nrows, int npar, int r0, float inv_scN,
                                           float inv_scW, int lane) {
  __syncwarp();
  const int stride = npar + 1;
  uint32_t* nh = w.h;
  uint32_t* nl = w.h + kHcap;
  uint32_t* wh = w.h + 2 * kHcap;
  uint32_t* wl = w.h + 3 * kHcap;
  float* nhi = w.acc;
  float* nlo = w.acc + kAcap;
  float* whi = w.acc + 2 * kAcap;
  float* wlo = w.acc + 3 * kAcap;
  for (int r = 0; r <= nrows; ++r) {
    for (int p = lane; p < stride; p += 32) {
      const int k = r * stride + p;
      const uint32_t a1 = nh[k], a2 = nl[k], b1 = wh[k], b2 = wl[k];
      if ((a1 | a2 | b1 | b2) != 0u) {
        if (r < nrows && p < npar) {
          const int a = (r0 + r) * npar + p;
          const float vn = fmaf(static_cast<float>(a2), 1.f / 65536.f, static_cast<float>(static_cast<int32_t>(a1))) * inv_scN;
          const float vw = fmaf(static_cast<float>(b2), 1.f / 65536.f, static_cast<float>(static_cast<int32_t>(b1))) * inv_scW;
          two_sum(nhi[a], nlo[a], vn);
          two_sum(whi[a], wlo[a], vw);
        }
        nh[k] = 0u;
        nl[k] = 0u;
        wh[k] = 0u;
        wl[k] = 0u;
      }
    }
  }
  __syncwarp();
}

// accumulator rows [0, rows) with origin t0 -> FP64 bin sums in global memory
__device__ __forceinline__ void flush_acc(const WarpSm& w, const XiArgs& A, int rows, int t0,
                                          int64_t out_off, int lane) {
  __syncwarp();
  const int npar = A.n_par;
  float* nhi = w.acc;
  float* nlo = w.acc + kAcap;
  float* whi = w.acc + 2 * kAcap;
  float* wlo = w.acc + 3 * kAcap;
  for (int r = 0; r < rows; ++r) {
    for (int p = lane; p < npar; p += 32) {
      const int a = r * npar + p;
      const float h1 = nhi[a], h2 = whi[a];
      if (h1 != 0.f || h2 != 0.f) {
        const int64_t bin = out_off + static_cast<int64_t>(p) * A.n_perp + t0 + r;
        red_add_f64_global(A.num + bin, static_cast<double>(h1) + static_cast<double>(nlo[a]));
        red_add_f64_global(A.wsum + bin, static_cast<double>(h2) + static_cast<double>(wlo[a]));
        nhi[a] = 0.f;
        nlo[a] = 0.f;
        whi[a] = 0.f;
        wlo[a] = 0.f;
      }
    }
  }
  __syncwarp();
}

// Bin rows t0 .. t0 + K - 1 of forest pair (a, b) into the chunk histogram
// (origin t0) and fold them into accumulator rows r0 ..; WINDOW restricts to
// rows [t0, t0 + K) of a wider band whose top is t_hi.
template <bool WINDOW>
__device__ void pair_rows(const XiArgs& A, const WarpSm& w, int aidx, int bidx, const Pix* __restrict__ pa,
                          const Pix* __restrict__ pb, int na, int nb, float cp, float sp, float Dc,
                          float Ds, int t0, int K, int t_hi, int r0, int seg, int lane) {
  const int npar = A.n_par;
  const float fnpar = static_cast<float>(npar), fnperp = static_cast<float>(A.n_perp);
  const uint32_t stride = static_cast<uint32_t>(npar + 1);
  // key (M+t)*(npar+1) + (M+p) -> local index (t - t0)*(npar+1) + p
  const uint32_t C = kMagicBits * (stride + 1u) + static_cast<uint32_t>(t0) * stride;
  const uint32_t base = w.sN - 4u * C;
  // fixed-point scales: a run of in-grid pairs (fixed i, one bin) spans less
  // than 2 / cp in distance, so it holds at most 2 / (cp hmin_b) + 1 pixels of b
  const float nrun = 2.f / (cp * A.F.hmin[bidx]) + 1.f;
  const float scN = fixed_scale(A.F.wdmax[aidx] * A.F.wdmax[bidx] * nrun);
  const float scW = fixed_scale(A.F.wmax[aidx] * A.F.wmax[bidx] * nrun);
  const float inv_scN = 1.f / scN, inv_scW = 1.f / scW;
  const uint32_t guard = C + static_cast<uint32_t>(npar);   // row 0, guard column
  const float pmax = __uint_as_float(kMagicBits + static_cast<uint32_t>(npar));
  const float tmax = __uint_as_float(kMagicBits + static_cast<uint32_t>(t_hi + 1));
  int pending = 0;
  for (int j0 = 0; j0 < nb; j0 += seg) {
    const int segn = min(seg, nb - j0);
    __syncwarp();
    for (int k = lane; k < segn; k += 32) w.buf[k] = pb[j0 + k];
    __syncwarp();
    for (int i0 = 0; i0 < na; i0 += 32) {
      const int i = i0 + lane;
      // lanes past the end carry a NaN distance: they only ever hit the guard
      const Pix pi = (i < na) ? pa[i] : make_float4(__int_as_float(0x7fffffff), 0.f, 0.f, 0.f);
      const float uc = fmaf(pi.x, cp, Dc);
      const float us = fmaf(pi.x, sp, Ds);
      const int last = min(31, na - 1 - i0);
      const float uc_first = __shfl_sync(0xffffffffu, uc, 0);
      const float us_first = __shfl_sync(0xffffffffu, us, 0);
      const float uc_last = __shfl_sync(0xffffffffu, uc, last);
      float dlo = (uc_first - fnpar) / cp;
      float dhi = (uc_last + fnpar) / cp;
      if (sp > 0.f) dhi = fminf(dhi, (fnperp - us_first) / sp);
      dlo -= fabsf(dlo) * 1e-5f + 1e-2f;
      dhi += fabsf(dhi) * 1e-5f + 1e-2f;
      const int jlo = count_below(w.buf, segn, dlo);
      const int jhi = count_below(w.buf, segn, dhi);
      if (jlo >= jhi) continue;
      chunk_runs<WINDOW>(w.buf, jlo, jhi, cp, sp, uc, us, pi.z, pi.y, pmax, tmax, stride, base, scN, scW,
                         guard, static_cast<uint32_t>(t0), static_cast<uint32_t>(K - 1),
                         w.sN + 4u * static_cast<uint32_t>(kHcap - 32 + lane));
      if (++pending == 2) {
        fold_chunk(w, K, npar, r0, inv_scN, inv_scW, lane);
        pending = 0;
      }
    }
  }
  if (pending) fold_chunk(w, K, npar, r0, inv_scN, inv_scW, lane);
}

__global__ void __launch_bounds__(512, 1) xi_mixed_kernel(XiArgs A, int seg, int kmax, int grab) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  // per warp: accumulator (4 x kAcap floats), chunk histogram (4 x kHcap
  // words), pixel buffer (seg float4)
  const int per_warp = kAcap * 16 + kHcap * 16 + seg * 16;
  unsigned char* wb = smem + wid * per_warp;
  WarpSm w;
  w.acc = reinterpret_cast<float*>(wb);
  w.h = reinterpret_cast<uint32_t*>(wb + kAcap * 16);
  w.buf = reinterpret_cast<Pix*>(wb + kAcap * 16 + kHcap * 16);
  w.sN = smem_addr(w.h);
  for (int k = lane; k < 4 * kAcap; k += 32) w.acc[k] = 0.f;
  for (int k = lane; k < 4 * kHcap; k += 32) w.h[k] = 0u;
  __syncwarp();
  const int npar = A.n_par, nperp = A.n_perp;
  const float fnperp = static_cast<float>(nperp);
  // the accumulator holds rows [acc_t0, acc_t0 + kmax) of catalogue acc_off
  int acc_t0 = -1;
  int64_t acc_off = -1;
  for (;;) {
    unsigned long long it0 = 0;
    if (lane == 0) it0 = atomicAdd(A.counter, static_cast<unsigned long long>(grab));
    it0 = __shfl_sync(0xffffffffu, it0, 0);
    if (it0 >= static_cast<unsigned long long>(A.n_pairs)) break;
    const int64_t it1 = min(static_cast<int64_t>(it0) + grab, A.n_pairs);
    for (int64_t it = static_cast<int64_t>(it0); it < it1; ++it) {
      const int2 ab = A.pairs[it];
      if (ab.x < 0) continue;   // rejected pair
      const int a = ab.x, b = ab.y;
      const int na = A.F.len[a], nb = A.F.len[b];
      if (na == 0 || nb == 0) continue;
      const float2 cs = A.cs[it];
      const float cp = cs.x, sp = cs.y;
      const Pix* __restrict__ pa = A.pix + A.F.off[a];
      const Pix* __restrict__ pb = A.pix + A.F.off[b];
      const float refa = A.F.dref[a], refb = A.F.dref[b];
      const float Dc = (refa - refb) * cp;
      const float Ds = (refa + refb) * sp;
      // r_perp band from the extreme pixels (r_perp is monotone in both distances)
      const float rt_min = fmaf(pb[0].x, sp, fmaf(pa[0].x, sp, Ds));
      const float rt_max = fmaf(pb[nb - 1].x, sp, fmaf(pa[na - 1].x, sp, Ds));
      if (!(rt_min < fnperp)) continue;
      const int t_lo = static_cast<int>(rt_min);
      const int t_hi = (rt_max < fnperp) ? static_cast<int>(rt_max) : nperp - 1;
      const int K = t_hi - t_lo + 1;
      const int64_t out_off = static_cast<int64_t>(A.F.mock[a]) * A.nb;
      if (K <= kmax) {
        if (t_lo != acc_t0 || out_off != acc_off) {
          if (acc_t0 >= 0) flush_acc(w, A, kmax, acc_t0, acc_off, lane);
          acc_t0 = t_lo;
          acc_off = out_off;
        }
        pair_rows<false>(A, w, a, b, pa, pb, na, nb, cp, sp, Dc, Ds, t_lo, K, t_hi, 0, seg, lane);
      } else {
        // wide band: windows of kmax rows, each flushed on its own
        if (acc_t0 >= 0) flush_acc(w, A, kmax, acc_t0, acc_off, lane);
        acc_t0 = -1;
        for (int tw = t_lo; tw <= t_hi; tw += kmax) {
          const int Kw = min(kmax, t_hi - tw + 1);
          pair_rows<true>(A, w, a, b, pa, pb, na, nb, cp, sp, Dc, Ds, tw, Kw, t_hi, 0, seg, lane);
          flush_acc(w, A, Kw, tw, out_off, lane);
        }
      }
    }
  }
  if (acc_t0 >= 0) flush_acc(w, A, kmax, acc_t0, acc_off, lane);
}

// ----------------------------------------------------------------------------
// FP64 path
// ----------------------------------------------------------------------------
struct Fp64Args {
  XiArgs A;
  const double4_32a* pix64;   // {d, w, w*delta, 0}
  double inv_dpar, inv_dperp;
};

__device__ __forceinline__ int count_below64(const double4_32a* a, int n, double v) {
  int lo = 0, hi = n;
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if (a[mid].x < v) lo = mid + 1; else hi = mid;
  }
  return lo;
}

__global__ void __launch_bounds__(128) xi_fp64_kernel(Fp64Args P, int seg, int kmax, int grab) {
  extern __shared__ __align__(16) unsigned char smem[];
  const XiArgs& A = P.A;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int per_warp = kHcap64 * 16 + seg * 32;
  double* hN = reinterpret_cast<double*>(smem + wid * per_warp);
  double* hW = hN + kHcap64;
  double4_32a* buf = reinterpret_cast<double4_32a*>(smem + wid * per_warp + kHcap64 * 16);
  for (int k = lane; k < 2 * kHcap64; k += 32) hN[k] = 0.0;
  __syncwarp();
  const int npar = A.n_par, nperp = A.n_perp;
  const double fnpar = npar, fnperp = nperp;
  for (;;) {
    unsigned long long it0 = 0;
    if (lane == 0) it0 = atomicAdd(A.counter, static_cast<unsigned long long>(grab));
    it0 = __shfl_sync(0xffffffffu, it0, 0);
    if (it0 >= static_cast<unsigned long long>(A.n_pairs)) break;
    const int64_t it1 = min(static_cast<int64_t>(it0) + grab, A.n_pairs);
    for (int64_t it = static_cast<int64_t>(it0); it < it1; ++it) {
      const int2 ab = A.pairs[it];
      if (ab.x < 0) continue;   // rejected pair
      const int a = ab.x, b = ab.y;
      const int na = A.F.len[a], nb = A.F.len[b];
      if (na == 0 || nb == 0) continue;
      const double4_32a* pa = P.pix64 + A.F.off[a];
      const double4_32a* pb = P.pix64 + A.F.off[b];
      const double sx = A.F.ux[a] + A.F.ux[b], sy = A.F.uy[a] + A.F.uy[b], sz = A.F.uz[a] + A.F.uz[b];
      const double dx = A.F.ux[a] - A.F.ux[b], dy = A.F.uy[a] - A.F.uy[b], dz = A.F.uz[a] - A.F.uz[b];
      const double c = 0.5 * sqrt(sx * sx + sy * sy + sz * sz);
      const double s = 0.5 * sqrt(dx * dx + dy * dy + dz * dz);
      const double cp = c * P.inv_dpar, sp = s * P.inv_dperp;
      const double rt_min = (pa[0].x + pb[0].x) * sp;
      const double rt_max = (pa[na - 1].x + pb[nb - 1].x) * sp;
      if (!(rt_min < fnperp)) continue;
      const int t_lo = static_cast<int>(rt_min);
      const int t_hi = (rt_max < fnperp) ? static_cast<int>(rt_max) : nperp - 1;
      const int64_t out_off = static_cast<int64_t>(A.F.mock[a]) * A.nb;
      for (int tw = t_lo; tw <= t_hi; tw += kmax) {
        const int tw_hi = min(t_hi, tw + kmax - 1);
        for (int j0 = 0; j0 < nb; j0 += seg) {
          const int segn = min(seg, nb - j0);
          __syncwarp();
          for (int k = lane; k < segn; k += 32) buf[k] = pb[j0 + k];
          __syncwarp();
          for (int i0 = 0; i0 < na; i0 += 32) {
            const int i = i0 + lane;
            const double4_32a pi = (i < na) ? pa[i] : make_double4_32a(3.0e300, 0, 0, 0);
            const int last = min(31, na - 1 - i0);
            const double d_first = __shfl_sync(0xffffffffu, pi.x, 0);
            const double d_last = __shfl_sync(0xffffffffu, pi.x, last);
            double dlo = d_first - fnpar / cp;
            double dhi = d_last + fnpar / cp;
            if (sp > 0.0) dhi = fmin(dhi, fnperp / sp - d_first);
            dlo -= fabs(dlo) * 1e-9 + 1e-6;
            dhi += fabs(dhi) * 1e-9 + 1e-6;
            const int jlo = count_below64(buf, segn, dlo);
            const int jhi = count_below64(buf, segn, dhi);
            for (int j = jlo; j < jhi; ++j) {
              const double4_32a q = buf[j];
              const double x = fabs(pi.x - q.x) * cp;
              const double y = (pi.x + q.x) * sp;
              if (x < fnpar && y < fnperp) {
                const int p = static_cast<int>(x);
                const int t = static_cast<int>(y);
                if (t >= tw && t <= tw_hi) {
                  const int k = (t - tw) * npar + p;
                  atomicAdd(&hN[k], pi.z * q.z);
                  atomicAdd(&hW[k], pi.y * q.y);
                }
              }
            }
          }
        }
        __syncwarp();
        const int Lw = (tw_hi - tw + 1) * npar;
        for (int k = lane; k < Lw; k += 32) {
          const double vw = hW[k], vn = hN[k];
          if (vw != 0.0 || vn != 0.0) {
            const int tt = k / npar;
            const int p = k - tt * npar;
            const int64_t bin = out_off + static_cast<int64_t>(p) * nperp + tw + tt;
            red_add_f64_global(A.wsum + bin, vw);
            red_add_f64_global(A.num + bin, vn);
            hW[k] = 0.0;
            hN[k] = 0.0;
          }
        }
        __syncwarp();
      }
    }
  }
}

__global__ void pack64_kernel(lya_catalog cat, Forests F, int64_t forest_base, double4_32a* out) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t f = warp; f < cat.n_forests; f += nw) {
    const int64_t gf = forest_base + f;
    const int n = F.len[gf];
    const int64_t o = cat.offsets[f];
    const int64_t g = F.off[gf];
    for (int k = lane; k < n; k += 32) {
      const double w = cat.weight[o + k];
      out[g + k] = make_double4_32a(cat.dist[o + k], w, w * static_cast<double>(cat.delta[o + k]), 0.0);
    }
  }
}

// In-grid pixel-pair count of every kept pair (same FP32 binning as the
// mixed kernel); one warp per forest pair.
__global__ void pair_stats_kernel(XiArgs A, uint64_t seed, uint64_t thr, int all, StatsOut* out) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const float fnpar = static_cast<float>(A.n_par), fnperp = static_cast<float>(A.n_perp);
  unsigned long long my_pairs = 0, my_pix = 0, my_sq = 0;
  for (int64_t k = warp; k < A.n_pairs; k += nw) {
    const int2 ab = A.pairs[k];
    if (ab.x < 0 || !keep_pair(ab.x, ab.y, seed, thr, all)) continue;
    const int na = A.F.len[ab.x], nb = A.F.len[ab.y];
    const float cp = A.cs[k].x, sp = A.cs[k].y;
    const float refa = A.F.dref[ab.x], refb = A.F.dref[ab.y];
    const float Dc = (refa - refb) * cp, Ds = (refa + refb) * sp;
    const Pix* pa = A.pix + A.F.off[ab.x];
    const Pix* pb = A.pix + A.F.off[ab.y];
    unsigned long long cnt = 0;
    for (int i = lane; i < na; i += 32) {
      const float di = pa[i].x;
      const float uc = fmaf(di, cp, Dc), us = fmaf(di, sp, Ds);
      for (int j = 0; j < nb; ++j) {
        const float dj = pb[j].x;
        const float rp = fabsf(fmaf(-dj, cp, uc));
        const float rt = fmaf(dj, sp, us);
        cnt += (rp < fnpar && rt < fnperp) ? 1ull : 0ull;
      }
    }
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    my_pairs += 1;
    my_pix += cnt;
    my_sq += cnt * cnt;
  }
  if (lane == 0 && my_pairs) {
    atomicAdd(&out->pairs, my_pairs);
    atomicAdd(&out->pix, my_pix);
    atomicAdd(&out->pix_sq, my_sq);
  }
}

// Bin-edge flips of the mixed path: for every pixel pair of the kept forest
// pairs, the bin from the mixed kernel's FP32 arithmetic against the bin from
// the FP64 path's arithmetic (FP64 distances of the caller's catalogue, FP64
// half-angle from the unit vectors).  One warp per forest pair.
__global__ void flip_tally_kernel(XiArgs A, const double* dist, double inv_dpar, double inv_dperp,
                                  uint64_t seed, uint64_t thr, int all, FlipOut* out) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int npar = A.n_par, nperp = A.n_perp;
  const float fnpar = static_cast<float>(npar), fnperp = static_cast<float>(nperp);
  unsigned long long n64 = 0, nflip = 0;
  double w64 = 0.0, wflip = 0.0;
  for (int64_t k = warp; k < A.n_pairs; k += nw) {
    const int2 ab = A.pairs[k];
    if (ab.x < 0 || !keep_pair(ab.x, ab.y, seed, thr, all)) continue;
    const int a = ab.x, b = ab.y;
    const int na = A.F.len[a], nb = A.F.len[b];
    if (na == 0 || nb == 0) continue;
    const float cp = A.cs[k].x, sp = A.cs[k].y;
    const float refa = A.F.dref[a], refb = A.F.dref[b];
    const float Dc = (refa - refb) * cp, Ds = (refa + refb) * sp;
    const Pix* pa = A.pix + A.F.off[a];
    const Pix* pb = A.pix + A.F.off[b];
    const double* da = dist + A.F.off[a];
    const double* db = dist + A.F.off[b];
    const double sx = A.F.ux[a] + A.F.ux[b], sy = A.F.uy[a] + A.F.uy[b], sz = A.F.uz[a] + A.F.uz[b];
    const double dx = A.F.ux[a] - A.F.ux[b], dy = A.F.uy[a] - A.F.uy[b], dz = A.F.uz[a] - A.F.uz[b];
    const double cp64 = 0.5 * sqrt(sx * sx + sy * sy + sz * sz) * inv_dpar;
    const double sp64 = 0.5 * sqrt(dx * dx + dy * dy + dz * dz) * inv_dperp;
    for (int i = lane; i < na; i += 32) {
      const Pix pi = pa[i];
      const double di = da[i];
      const float uc = fmaf(pi.x, cp, Dc), us = fmaf(pi.x, sp, Ds);
      for (int j = 0; j < nb; ++j) {
        const Pix q = pb[j];
        const float rp = fabsf(fmaf(-q.x, cp, uc));
        const float rt = fmaf(q.x, sp, us);
        const int bin32 = (rp < fnpar && rt < fnperp)
                              ? static_cast<int>(__float_as_uint(__fadd_rd(rp, kMagic)) - kMagicBits) * nperp +
                                    static_cast<int>(__float_as_uint(__fadd_rd(rt, kMagic)) - kMagicBits)
                              : -1;
        const double x = fabs(di - db[j]) * cp64;
        const double y = (di + db[j]) * sp64;
        const int bin64 = (x < npar && y < nperp) ? static_cast<int>(x) * nperp + static_cast<int>(y) : -1;
        const double w = static_cast<double>(pi.y) * static_cast<double>(q.y);
        if (bin64 >= 0) {
          n64 += 1;
          w64 += w;
        }
        if (bin32 != bin64) {
          nflip += 1;
          wflip += w;
        }
      }
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    n64 += __shfl_xor_sync(0xffffffffu, n64, o);
    nflip += __shfl_xor_sync(0xffffffffu, nflip, o);
    w64 += __shfl_xor_sync(0xffffffffu, w64, o);
    wflip += __shfl_xor_sync(0xffffffffu, wflip, o);
  }
  if (lane == 0 && n64 + nflip > 0) {
    atomicAdd(&out->pix, n64);
    atomicAdd(&out->flips, nflip);
    atomicAdd(&out->w, w64);
    atomicAdd(&out->wflip, wflip);
  }
}

__global__ void finalize_kernel(const double* num, const double* wsum, double* xi, int64_t n) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x) {
    const double w = wsum[k];
    xi[k] = (w != 0.0) ? num[k] / w : 0.0;
  }
}

}  // namespace

int xi_mixed_max_npar() {
  // two chunk-histogram rows (band row and guard row) of n_par + 1 words below the 32 dummy words
  return std::min((kHcap - 32) / 2 - 1, kAcap);
}

cudaError_t plan_xi_mixed(const DevInfo& dev, int n_par, int max_len, int warps, int grab,
                          XiLaunch* L) {
  if (n_par > xi_mixed_max_npar()) return cudaErrorInvalidValue;
  int seg = ((std::max(max_len, 1) + 31) / 32) * 32;
  if (seg > kMaxSeg) seg = kMaxSeg;
  // longer forests are staged in segments: shrink the segment until the block fits
  while (seg > 32 && warps * (kAcap * 16 + kHcap * 16 + seg * 16) > dev.smem_optin) seg -= 32;
  L->warps = warps;
  L->hcap = kHcap;
  L->seg = seg;
  L->grab = grab;
  L->smem = warps * (kAcap * 16 + kHcap * 16 + seg * 16);
  if (L->smem > dev.smem_optin) return cudaErrorInvalidValue;
  cudaError_t e = set_max_dynamic_smem(reinterpret_cast<const void*>(xi_mixed_kernel), L->smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, xi_mixed_kernel, warps * 32, L->smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidValue;
  L->blocks = per_sm * dev.sms;
  return cudaSuccess;
}

cudaError_t launch_xi_mixed(const XiArgs& a, const XiLaunch& L, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(a.counter, 0, sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  if (a.n_pairs == 0) return cudaSuccess;
  // band rows per window: the chunk histogram needs (kmax + 1) x (n_par + 1)
  // entries (guard row and column), the accumulator kmax x n_par
  const int kmax = std::max(1, std::min({a.n_perp, (kHcap - 32) / (a.n_par + 1) - 1, kAcap / a.n_par}));
  LYA_COUNT(1), xi_mixed_kernel<<<L.blocks, L.warps * 32, L.smem, s>>>(a, L.seg, kmax, L.grab);
  return cudaGetLastError();
}

cudaError_t launch_xi_fp64(const XiArgs& a, const lya_catalog* cats, int n_cats, const DevInfo& dev,
                           int max_len, double r_par_max, double r_perp_max, XiLaunch* used,
                           cudaStream_t s) {
  if (a.n_par > kHcap64) return cudaErrorInvalidValue;
  // FP64 packed pixels, built on demand in a temporary buffer
  int64_t npix = 0;
  for (int m = 0; m < n_cats; ++m) npix += cats[m].n_pix;
  double4_32a* pix64 = nullptr;
  cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&pix64), std::max<int64_t>(npix, 1) * 32, s);
  if (e != cudaSuccess) return e;
  int64_t fb = 0;
  for (int m = 0; m < n_cats; ++m) {
    if (cats[m].n_forests > 0) {
      int64_t blocks = std::min<int64_t>((cats[m].n_forests * 32 + 255) / 256, 65535);
      LYA_COUNT(1), pack64_kernel<<<static_cast<int>(blocks), 256, 0, s>>>(cats[m], a.F, fb, pix64);
    }
    fb += cats[m].n_forests;
  }
  Fp64Args P;
  P.A = a;
  P.pix64 = pix64;
  P.inv_dpar = static_cast<double>(a.n_par) / r_par_max;
  P.inv_dperp = static_cast<double>(a.n_perp) / r_perp_max;
  int seg = ((std::max(max_len, 1) + 31) / 32) * 32;
  if (seg > 512) seg = 512;
  const int warps = 4;
  const int smem = warps * (kHcap64 * 16 + seg * 32);
  e = set_max_dynamic_smem(reinterpret_cast<const void*>(xi_fp64_kernel), smem);
  int per_sm = 0;
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, xi_fp64_kernel, warps * 32, smem);
  if (e == cudaSuccess && per_sm < 1) e = cudaErrorInvalidValue;
  if (e == cudaSuccess) e = cudaMemsetAsync(a.counter, 0, sizeof(unsigned long long), s);
  const int kmax = std::max(1, std::min(a.n_perp, kHcap64 / a.n_par));
  if (e == cudaSuccess && a.n_pairs > 0) {
    LYA_COUNT(1), xi_fp64_kernel<<<per_sm * dev.sms, warps * 32, smem, s>>>(P, seg, kmax, 4);
    e = cudaGetLastError();
  }
  if (used) {
    used->warps = warps;
    used->blocks = per_sm * dev.sms;
    used->seg = seg;
    used->smem = smem;
    used->hcap = kHcap64;
    used->grab = 4;
  }
  cudaFreeAsync(pix64, s);
  return e;
}

cudaError_t launch_pair_stats(const XiArgs& a, double p_subsample, uint64_t seed, StatsOut* out,
                              const DevInfo& dev, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(out, 0, sizeof(StatsOut), s);
  if (e != cudaSuccess || a.n_pairs == 0 || p_subsample <= 0.0) return e;
  const int all = p_subsample >= 1.0 ? 1 : 0;
  const uint64_t thr = all ? 0 : static_cast<uint64_t>(p_subsample * 18446744073709551616.0);
  LYA_COUNT(1), pair_stats_kernel<<<dev.sms * 8, 256, 0, s>>>(a, seed, thr, all, out);
  return cudaGetLastError();
}

cudaError_t launch_flip_tally(const XiArgs& a, const double* dist, double inv_dpar, double inv_dperp,
                              double p_subsample, uint64_t seed, FlipOut* out, const DevInfo& dev,
                              cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(out, 0, sizeof(FlipOut), s);
  if (e != cudaSuccess || a.n_pairs == 0 || p_subsample <= 0.0) return e;
  const int all = p_subsample >= 1.0 ? 1 : 0;
  const uint64_t thr = all ? 0 : static_cast<uint64_t>(p_subsample * 18446744073709551616.0);
  LYA_COUNT(1), flip_tally_kernel<<<dev.sms * 8, 256, 0, s>>>(a, dist, inv_dpar, inv_dperp, seed, thr, all, out);
  return cudaGetLastError();
}

cudaError_t launch_finalize(const double* num, const double* wsum, double* xi, int64_t n,
                            cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  int64_t b = std::min<int64_t>((n + 255) / 256, 4096);
  LYA_COUNT(1), finalize_kernel<<<static_cast<int>(b), 256, 0, s>>>(num, wsum, xi, n);
  return cudaGetLastError();
}

}  // namespace lya
