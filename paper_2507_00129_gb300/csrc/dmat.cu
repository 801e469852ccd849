// Distortion matrix of Eq. (2.6) over the seeded forest-pair subsample
// (Section 2.2), without the O(N^4) contraction.
//
// With eta = I - 1 u^T - x v^T per forest (u = w/W, v = w x/S, Eq. 2.7), one
// forest pair (a, b) adds to D~_AB = sum_{(i,j) in A} w_i w_j sum_{(k,l) in B} eta_ik eta_jl:
//
//   diag(T1)
//   - sum_j w_j (alpha_j alpha_j^T / W_a + beta_j beta_j^T / S_a)         (columns j of b)
//   - sum_i w_i (alpha'_i alpha'_i^T / W_b + beta'_i beta'_i^T / S_b)     (rows i of a)
//   + T1 T1^T/(W_a W_b) + Ty Ty^T/(W_a S_b) + Tx Tx^T/(S_a W_b) + Txy Txy^T/(S_a S_b)
//
// alpha_j[A] = sum_{i:(i,j) in A} w_i, beta_j[A] = sum w_i x_i, alpha'_i, beta'_i
// likewise over j with y = Lambda - Lbar of forest b, T1 = sum_A w_i w_j,
// Tx = sum w_i w_j x_i, Ty = sum w_i w_j y_j, Txy = sum w_i w_j x_i y_j.
//
// Work layout.  All bins a pair touches lie in its r_perp band of K rows
// (r_perp is monotone in both distances), i.e. L = K n_par local bins.  The
// kept pairs are grouped by (first band row, K); a block takes a chunk of
// pairs of one group and keeps the upper triangle of the L x L block of D~
// in shared memory (FP32): each pair's contribution is built there and added
// to the FP64 accumulator G (entries A <= B) with FP64 atomics at the end of
// the pair, so that the sum over pairs is FP64.  The rank-1 terms are applied a
// batch of up to CB vectors (consecutive columns, then rows) at a time:
//  (a1) every thread bins pixel pairs and marks the local bins the batch
//       touches; (b) one warp compacts the marks into the batch's sorted union
//       support S (|S| is a little above one vector's support, because
//       neighbouring columns visit nearly the same bins);
//  (a2) the batch's histograms are summed densely on S with shared atomics;
//       column histograms also feed the T vectors;
//  (d)  each thread owns a 4 x 4 tile of the S x S upper triangle and adds
//       sum_v (a_v a_v^T + b_v b_v^T) over the batch in registers (FP32 FMA,
//       float4 loads), then updates its 16 triangle entries -- no atomics.
// Pairs whose band is too wide for shared memory take the same code with the
// triangle replaced by FP64 atomics into G.  Binning uses exactly the FP32
// arithmetic of the xi kernel, so W^DM equals the xi weights of the kept
// pairs up to summation order.
#include <algorithm>
#include <math.h>

#include "lya_internal.cuh"

namespace lya {
namespace {

constexpr int kDmThreads = 512;
constexpr int kChunk = 32;   // pairs per work unit (each pair is flushed on its own; small units balance the SMs)


// band of a pair: same FP32 arithmetic as the xi kernel
__device__ __forceinline__ bool pair_band(const DmArgs& A, int a, int b, float sp, int* t_lo, int* K) {
  const int na = A.F.len[a], nb = A.F.len[b];
  if (na == 0 || nb == 0) return false;
  const Pix* pa = A.pix + A.F.off[a];
  const Pix* pb = A.pix + A.F.off[b];
  const float Ds = (A.F.dref[a] + A.F.dref[b]) * sp;
  const float fnperp = static_cast<float>(A.n_perp);
  const float rt_min = fmaf(pb[0].x, sp, fmaf(pa[0].x, sp, Ds));
  const float rt_max = fmaf(pb[nb - 1].x, sp, fmaf(pa[na - 1].x, sp, Ds));
  if (!(rt_min < fnperp)) return false;
  const int lo = static_cast<int>(rt_min);
  const int hi = (rt_max < fnperp) ? static_cast<int>(rt_max) : A.n_perp - 1;
  *t_lo = lo;
  *K = hi - lo + 1;
  return true;
}

__global__ void dm_select_kernel(DmArgs A, uint64_t thr, int all, int kfit, int32_t* key,
                                 int32_t* count, int32_t* wide, int32_t* n_wide) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < A.n_pairs;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int2 p = A.pairs[k];
    int32_t kk = -1;
    // the subsample rule sees forest indices local to the pair's catalogue,
    // so a mock's D does not depend on the other mocks of the batch
    const int m = (p.x >= 0) ? A.F.mock[p.x] : 0;
    const int base = (p.x >= 0) ? A.fbase[m] : 0;
    const bool keep = p.x >= 0 && keep_pair(p.x - base, p.y - base, A.seed, thr, all);
    int t_lo, K;
    if (keep && pair_band(A, p.x, p.y, A.cs[k].y, &t_lo, &K)) {
      if (K <= kfit) {
        kk = (m * A.n_perp + t_lo) * kfit + (K - 1);
        atomicAdd(&count[kk], 1);
      } else {
        const int w = atomicAdd(n_wide, 1);
        wide[w] = static_cast<int32_t>(k);
      }
    }
    key[k] = kk;
  }
}

__global__ void dm_scatter_kernel(int64_t n, const int32_t* key, const int64_t* start, int32_t* cursor,
                                  int32_t* order) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int32_t kk = key[k];
    if (kk < 0) continue;
    const int pos = atomicAdd(&cursor[kk], 1);
    order[start[kk] + pos] = static_cast<int32_t>(k);
  }
}

__global__ void chunk_count_kernel(const int32_t* count, int ngroups, int32_t* nchunks) {
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < ngroups; g += gridDim.x * blockDim.x)
    nchunks[g] = (count[g] + kChunk - 1) / kChunk;
}

struct Chunk {
  int32_t begin;   // into order[]
  int32_t n;
  int32_t t0;
  int32_t K;
  int32_t mock;    // catalogue whose accumulator the chunk adds to
};

__global__ void chunk_fill_kernel(const int32_t* count, const int64_t* start, const int64_t* coff,
                                  int ngroups, int kfit, int n_perp, Chunk* chunks) {
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < ngroups; g += gridDim.x * blockDim.x) {
    const int c = count[g];
    for (int q = 0; q * kChunk < c; ++q) {
      Chunk ch;
      ch.begin = static_cast<int32_t>(start[g] + q * kChunk);
      ch.n = min(kChunk, c - q * kChunk);
      ch.t0 = (g / kfit) % n_perp;
      ch.K = g % kfit + 1;
      ch.mock = g / (kfit * n_perp);
      chunks[coff[g] + q] = ch;
    }
  }
}

// vectors per batch: 32 where the band fits in shared memory with them (half
// the block-wide phases per pair), else 16
constexpr int kCB = 16;
constexpr int kCB2 = 32;

// Shared-memory layout of one block (offsets in bytes)
struct Lay {
  int U, T4, Va, Vb, mark, inv, S, ucs, pixa, pixb, tv, cf, gbin, misc, end;
};

__host__ __device__ inline int scap_for(int L, int npar, int K, int cb) {
  // union-support capacity: at least one vector's support bound 2 (n_par + K) + 2,
  // with room for the batch's neighbouring vectors
  int c = 2 * (npar + K) + 2;
  c = (cb > kCB) ? 2 * c : c + c / 2;
  if (c > L) c = L;
  return (c + 3) & ~3;
}

// Row stride of the batch vectors V[cb][.]: at least the support capacity
// rounded up to 16 (the tensor-core tiles read 16-row blocks) and 8 modulo 32,
// so that the fragment loads of the tensor-core tiles (rows t and t + 4 of a
// k step, 8 consecutive support entries) hit 32 different banks.
__host__ __device__ inline int ldv_for(int scap) {
  int v = (scap + 15) & ~15;
  while ((v & 31) != 8) v += 8;
  return v;
}

__host__ __device__ inline Lay layout(int L, int scap, int max_len, bool global_sink, int cb) {
  auto al = [](int v) { return (v + 15) & ~15; };
  Lay y;
  int o = 0;
  y.U = o;
  if (!global_sink) o += al(static_cast<int>((static_cast<int64_t>(L) * (L + 1) / 2) * 4));
  y.T4 = o; o += al(L * 16);
  y.Va = o; o += al(cb * ldv_for(scap) * 4);
  y.Vb = o; o += al(cb * ldv_for(scap) * 4);
  y.mark = o; o += al(L);
  y.inv = o; o += al(L * 2);
  y.S = o; o += al(scap * 4);
  y.ucs = o; o += al(max_len * 8);
  y.pixa = o; o += al(max_len * 16);
  y.pixb = o; o += al(max_len * 16);
  y.tv = o; o += al(max_len * 8);
  y.cf = o; o += al(max_len * 16);
  y.gbin = o; o += al(L * 4);
  y.misc = o; o += 64;
  y.end = o;
  return y;
}

__device__ __forceinline__ int tri_rowbase(int r, int L) {
  // index of (r, c), c >= r, in the packed upper triangle is rowbase(r) + c
  return r * (2 * L - r + 1) / 2 - r;
}

// Power of two sc = 2^(29 - e), 2^e <= B < 2^(e+1): sums bounded by B map below 2^30.
__device__ __forceinline__ float word_scale(float B) {
  if (!(B > 0.f) || !(B < 1e37f)) return 1.f;
  const int e = static_cast<int>((__float_as_uint(B) >> 23) & 0xFFu) - 127;
  return __uint_as_float(static_cast<uint32_t>(min(max(29 - e + 127, 1), 254)) << 23);
}

// Bin of pixel pair (i of a, j of b); returns the local bin or -1 if off-grid.
// The floors are FP32 adds of 2^23 rounded toward -inf, as in the xi kernel.
__device__ __forceinline__ int local_bin(float2 u, float dj, float cp, float sp, float fnpar, float fnperp,
                                         int npar, int t0) {
  const float rp = fabsf(fmaf(-dj, cp, u.x));
  const float rt = fmaf(dj, sp, u.y);
  if (rp < fnpar && rt < fnperp) return (static_cast<int>(rt) - t0) * npar + static_cast<int>(rp);
  return -1;
}

// Tile q of the packed upper triangle of 4 x 4 blocks of the union support:
// acc = sum over vectors [vlo, vhi) of a a^T + b b^T on that block.
__device__ __forceinline__ void dm_tile(const float* Va, const float* Vb, int ldv, int q, int vlo, int vhi,
                                        float (&acc)[4][4], int* rblk_out, int* cblk_out) {
  int rr = static_cast<int>((sqrtf(8.f * q + 1.f) - 1.f) * 0.5f);
  while (rr * (rr + 1) / 2 > q) --rr;
  while ((rr + 1) * (rr + 2) / 2 <= q) ++rr;
  const int cblk = rr;                      // column block (>= row block)
  const int rblk = q - rr * (rr + 1) / 2;   // row block
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) acc[u][v] = 0.f;
  for (int vv = vlo; vv < vhi; ++vv) {
    const float4 ar = *reinterpret_cast<const float4*>(Va + vv * ldv + 4 * rblk);
    const float4 ac = *reinterpret_cast<const float4*>(Va + vv * ldv + 4 * cblk);
    const float4 br = *reinterpret_cast<const float4*>(Vb + vv * ldv + 4 * rblk);
    const float4 bc = *reinterpret_cast<const float4*>(Vb + vv * ldv + 4 * cblk);
    const float arv[4] = {ar.x, ar.y, ar.z, ar.w}, acv[4] = {ac.x, ac.y, ac.z, ac.w};
    const float brv[4] = {br.x, br.y, br.z, br.w}, bcv[4] = {bc.x, bc.y, bc.z, bc.w};
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int v = 0; v < 4; ++v) acc[u][v] = fmaf(brv[u], bcv[v], fmaf(arv[u], acv[v], acc[u][v]));
  }
  *rblk_out = rblk;
  *cblk_out = cblk;
}

// Tensor-core form of the rank-1 tiles: C = V^T V over the union support,
// V the batch's [32 x S] matrix (rows: the a vectors, then the b vectors),
// with mma.sync m16n8k8 in TF32 and the 3xTF32 split (x = hi + lo, hi and lo
// TF32; C += lo.hi + hi.lo + hi.hi), which keeps the products at about FP32
// accuracy.  Warp tiles of 16 x 8 entries of the upper triangle (c >= r); each
// lane subtracts its four accumulators from the triangle (entries r <= c only,
// each unordered pair of support entries once).
__device__ __forceinline__ uint32_t tf32_bits(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ void mma_tf32(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                         uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__device__ __forceinline__ void split_tf32(float x, uint32_t& hi, uint32_t& lo) {
  hi = tf32_bits(x);
  lo = tf32_bits(x - __uint_as_float(hi));
}

__device__ void dm_tiles_tc(const float* Va, const float* Vb, int ldv, int ns, int cbn, const int32_t* S, float* U,
                            int L, int wid, int nwarps, int lane) {
  const int g = lane >> 2, t = lane & 3;
  const int R = (ns + 15) >> 4, C8 = (ns + 7) >> 3;
  const int ksteps = (cbn + 7) >> 3;   // vectors [0, cbn) in k steps of 8 (rows past cbn are zero)
  int q = 0;
  for (int rb = 0; rb < R; ++rb) {
    for (int cb = 2 * rb; cb < C8; ++cb, ++q) {
      if (q % nwarps != wid) continue;
      const int r0 = rb * 16, c0 = cb * 8;
      float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int half = 0; half < 2; ++half) {
        const float* V = half ? Vb : Va;
        for (int ks = 0; ks < ksteps; ++ks) {
          const float* v0 = V + (ks * 8 + t) * ldv;
          const float* v4 = v0 + 4 * ldv;
          uint32_t ah[4], al[4], bh[2], bl[2];
          split_tf32(v0[r0 + g], ah[0], al[0]);
          split_tf32(v0[r0 + g + 8], ah[1], al[1]);
          split_tf32(v4[r0 + g], ah[2], al[2]);
          split_tf32(v4[r0 + g + 8], ah[3], al[3]);
          split_tf32(v0[c0 + g], bh[0], bl[0]);
          split_tf32(v4[c0 + g], bh[1], bl[1]);
          mma_tf32(acc, al[0], al[1], al[2], al[3], bh[0], bh[1]);
          mma_tf32(acc, ah[0], ah[1], ah[2], ah[3], bl[0], bl[1]);
          mma_tf32(acc, ah[0], ah[1], ah[2], ah[3], bh[0], bh[1]);
        }
      }
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int r = r0 + g + ((e & 2) ? 8 : 0);
        const int c = c0 + 2 * t + (e & 1);
        if (r <= c && c < ns) {
          const int lr = S[r], lc = S[c];
          const int lo = min(lr, lc), hi = max(lr, lc);
          U[tri_rowbase(lo, L) + hi] -= acc[e];
        }
      }
    }
  }
}

// Subtract a tile from the triangle, or from G with FP64 atomics for wide
// pairs.  Positions r <= c of the union support S (which is in no particular
// order) cover each unordered pair of its bins once; the symmetric entry goes
// to (min, max) of the two local bins.
template <bool GLOBAL>
__device__ __forceinline__ void dm_tile_store(double* G, float* U, const int32_t* S, const int32_t* gbin,
                                              int ns, int L, int nbins, int rblk, int cblk,
                                              const float (&acc)[4][4]) {
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int r = 4 * rblk + u;
    if (r >= ns) continue;
    const int lr = S[r];
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int c = 4 * cblk + v;
      if (c >= ns || c < r) continue;
      const int lc = S[c];
      if (!GLOBAL) {
        const int lo = min(lr, lc), hi = max(lr, lc);
        U[tri_rowbase(lo, L) + hi] -= acc[u][v];
      } else {
        const int Ar = gbin[lr], Ac = gbin[lc];
        red_add_f64_global(G + static_cast<int64_t>(min(Ar, Ac)) * nbins + max(Ar, Ac),
                           -static_cast<double>(acc[u][v]));
      }
    }
  }
}

// One forest pair: accumulate its contribution into the triangle (or G).
template <bool GLOBAL, int CB>
__device__ void dm_pair(const DmArgs& A, double* G, double* wdm, int item, int t0, int K, int L, int scap,
                        unsigned char* sm, const Lay& y) {
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int2 pr = A.pairs[item];
  const float2 cs = A.cs[item];
  const int a = pr.x, b = pr.y;
  const int na = A.F.len[a], nb = A.F.len[b];
  // staging buffers hold max_len pixels (the longest forest when the pair list
  // was built); a longer forest means the offsets changed in place without a
  // rebuild, and the pair is skipped rather than overrun shared memory
  if (na > A.max_len || nb > A.max_len || na == 0 || nb == 0) return;
  const float cp = cs.x, sp = cs.y;
  const float refa = A.F.dref[a], refb = A.F.dref[b];
  const float Dc = (refa - refb) * cp, Ds = (refa + refb) * sp;
  const double Wa = A.F.wsum[a], Sa = A.F.ssum[a], Wb = A.F.wsum[b], Sb = A.F.ssum[b];
  const bool eta = A.eta_mean_slope != 0;
  const int npar = A.n_par, nbins = A.n_par * A.n_perp;
  const int ldv = ldv_for(scap);
  const float fnpar = static_cast<float>(npar), fnperp = static_cast<float>(A.n_perp);

  float* U = reinterpret_cast<float*>(sm + y.U);
  float4* T4 = reinterpret_cast<float4*>(sm + y.T4);
  float* Va = reinterpret_cast<float*>(sm + y.Va);
  float* Vb = reinterpret_cast<float*>(sm + y.Vb);
  int32_t* Vai = reinterpret_cast<int32_t*>(sm + y.Va);   // same storage, fixed point while filling
  int32_t* Vbi = reinterpret_cast<int32_t*>(sm + y.Vb);
  int2* tv = reinterpret_cast<int2*>(sm + y.tv);
  float4* cf = reinterpret_cast<float4*>(sm + y.cf);
  unsigned char* mark = sm + y.mark;
  int16_t* inv = reinterpret_cast<int16_t*>(sm + y.inv);
  int32_t* S = reinterpret_cast<int32_t*>(sm + y.S);
  float2* ucs = reinterpret_cast<float2*>(sm + y.ucs);
  Pix* pxa = reinterpret_cast<Pix*>(sm + y.pixa);
  Pix* pxb = reinterpret_cast<Pix*>(sm + y.pixb);
  const int32_t* gbin = reinterpret_cast<const int32_t*>(sm + y.gbin);
  int* misc = reinterpret_cast<int*>(sm + y.misc);   // [0] = |S|

  const Pix* ga = A.pix + A.F.off[a];
  const Pix* gb = A.pix + A.F.off[b];
  for (int k = tid; k < na; k += blockDim.x) {
    const Pix p = ga[k];
    pxa[k] = p;
    ucs[k] = make_float2(fmaf(p.x, cp, Dc), fmaf(p.x, sp, Ds));
  }
  for (int k = tid; k < nb; k += blockDim.x) pxb[k] = gb[k];
  __syncthreads();

  // side 0: columns j of b (histograms over i of a, weights w_i, x_i)
  // side 1: rows i of a (histograms over j of b, weights w_j, y_j)
  for (int side = 0; side < 2; ++side) {
    if (side == 1 && !eta) break;
    const int nvec = side == 0 ? nb : na;
    const int nother = side == 0 ? na : nb;
    // rank-1 coefficients sqrt(w_v / W) and sqrt(w_v / S) of this side's
    // vectors, from FP32 reciprocals computed once per pair (FP64 division is
    // slow on this part)
    const double Wn = side == 0 ? Wa : Wb;
    const double Sn = side == 0 ? Sa : Sb;
    const float inv_w = (eta && Wn > 0.0) ? static_cast<float>(1.0 / Wn) : 0.f;
    const float inv_s = (eta && Sn > 0.0) ? static_cast<float>(1.0 / Sn) : 0.f;
    // Histogram terms of the summed-over forest (w, w x) in fixed point, one
    // 32-bit word each: shared memory adds integers natively.  A (vector, bin)
    // sum holds at most 2 / (cp hmin) + 2 pixels (two windows of width 1/cp).
    {
      const int fs = side == 0 ? a : b;
      const Pix* ps = side == 0 ? pxa : pxb;
      const int ns_ = side == 0 ? na : nb;
      const float nrun = 2.f / (cp * A.F.hmin[fs]) + 2.f;
      const float scA = word_scale(nrun * A.F.wmax[fs]);
      const float scB = word_scale(nrun * A.F.wmax[fs] * A.F.xmax[fs]);
      if (tid == 0) {
        reinterpret_cast<float*>(misc)[1] = 1.f / scA;
        reinterpret_cast<float*>(misc)[2] = 1.f / scB;
      }
      for (int k = tid; k < ns_; k += blockDim.x)
        tv[k] = make_int2(__float2int_rn(ps[k].y * scA), __float2int_rn(ps[k].y * ps[k].w * scB));
      // per vector of this side: rank-1 coefficients and the T weights w_v, w_v y_v
      const Pix* pv = side == 0 ? pxb : pxa;
      for (int k = tid; k < nvec; k += blockDim.x) {
        const Pix me = pv[k];
        cf[k] = make_float4(sqrtf(me.y * inv_w), sqrtf(me.y * inv_s), me.y, me.y * me.w);
      }
      __syncthreads();
    }
    const float inv_scA = reinterpret_cast<float*>(misc)[1];
    const float inv_scB = reinterpret_cast<float*>(misc)[2];
    int v0 = 0;
    int cb = CB;
    while (v0 < nvec) {
      const int cbn = min(cb, nvec - v0);
      // (a1) mark the local bins the batch touches (and reset the slot counter of (b))
      if (tid == 0) misc[3] = 0;
      const int vv_t = tid % cbn;
      const int ostep = blockDim.x / cbn;
      // independent items: unrolled so that several items' loads are in flight
#pragma unroll 4
      for (int o = tid / cbn; o < nother && tid < ostep * cbn; o += ostep) {
        const int i = side == 0 ? o : v0 + vv_t;
        const int j = side == 0 ? v0 + vv_t : o;
        const int l = local_bin(ucs[i], pxb[j].x, cp, sp, fnpar, fnperp, npar, t0);
        if (l >= 0) mark[l] = 1;
      }
      __syncthreads();
      // (b) compaction of the marks into S and the inverse map, all warps: a
      // warp takes 32 local bins, ballots, and reserves its slots in S with
      // one shared atomic (S is in no particular order; every output entry
      // still sums its vectors in a fixed order).  V is cleared meanwhile.
      {
        const int nwarps = blockDim.x >> 5;
        for (int l0 = wid * 32; l0 < L; l0 += nwarps * 32) {
          const int l = l0 + lane;
          const bool on = (l < L) && mark[l];
          const unsigned msk = __ballot_sync(0xffffffffu, on);
          int base = 0;
          if (lane == 0 && msk) base = atomicAdd(&misc[3], __popc(msk));
          base = __shfl_sync(0xffffffffu, base, 0);
          if (on) {
            const int pos = base + __popc(msk & ((1u << lane) - 1u));
            if (pos < scap) S[pos] = l;
            inv[l] = static_cast<int16_t>(pos);
            mark[l] = 0;
          }
        }
        for (int k = tid; k < CB * ldv; k += blockDim.x) {
          Va[k] = 0.f;
          Vb[k] = 0.f;
        }
      }
      __syncthreads();
      const int ns = misc[3];
      if (ns > scap) {
        // union too large for the staging arrays: retry with half the batch
        __syncthreads();
        cb = max(1, cbn / 2);
        continue;
      }
      // (a2) dense histograms on S
      // independent items: unrolled so that several items' loads are in flight
#pragma unroll 4
      for (int o = tid / cbn; o < nother && tid < ostep * cbn; o += ostep) {
        const int i = side == 0 ? o : v0 + vv_t;
        const int j = side == 0 ? v0 + vv_t : o;
        const int l = local_bin(ucs[i], pxb[j].x, cp, sp, fnpar, fnperp, npar, t0);
        if (l >= 0) {
          const int2 t = tv[side == 0 ? i : j];   // the summed-over pixel's terms
          const int k = vv_t * ldv + inv[l];
          atomicAdd(reinterpret_cast<unsigned*>(&Vai[k]), static_cast<unsigned>(t.x));
          atomicAdd(reinterpret_cast<unsigned*>(&Vbi[k]), static_cast<unsigned>(t.y));
        }
      }
      __syncthreads();
      // T vectors (from unscaled column histograms) and scaling by the
      // rank-1 coefficients sqrt(w_v / W), sqrt(w_v / S).  Item (k, vv) =
      // (bin of S, vector of the batch); the 16 vectors of a bin sit in 16
      // consecutive lanes, which sum the bin's T terms with shuffles.
      for (int base = 0; base < ns * CB; base += blockDim.x) {
        const int idx = base + tid;
        const int k = idx / CB, vv = idx % CB;
        const bool act = (k < ns) && (vv < cbn);
        float t1 = 0.f, tx = 0.f, ty = 0.f, txy = 0.f;
        if (act) {
          const float4 c = cf[v0 + vv];
          const float va = static_cast<float>(Vai[vv * ldv + k]) * inv_scA;
          const float vb = static_cast<float>(Vbi[vv * ldv + k]) * inv_scB;
          t1 = c.z * va;
          tx = c.z * vb;
          ty = c.w * va;
          txy = c.w * vb;
          Va[vv * ldv + k] = va * c.x;
          Vb[vv * ldv + k] = vb * c.y;
        }
        if (side == 0) {
#pragma unroll
          for (int o = CB / 2; o > 0; o >>= 1) {
            t1 += __shfl_xor_sync(0xffffffffu, t1, o);
            tx += __shfl_xor_sync(0xffffffffu, tx, o);
            ty += __shfl_xor_sync(0xffffffffu, ty, o);
            txy += __shfl_xor_sync(0xffffffffu, txy, o);
          }
          if (act && vv == 0) {
            float4 t = T4[S[k]];
            t.x += t1;
            t.y += tx;
            t.z += ty;
            t.w += txy;
            T4[S[k]] = t;
          }
        }
      }
      __syncthreads();
      // (d) rank-1 updates of the batch: 4 x 4 register tiles of S x S,
      // one tile per thread, each adding its 16 entries to the triangle.
      if (eta) {
        if (!GLOBAL && A.tensor_tiles) {
          dm_tiles_tc(Va, Vb, ldv, ns, cbn, S, U, L, wid, blockDim.x >> 5, lane);
        } else {
          const int nt = (ns + 3) >> 2;
          const int ntiles = nt * (nt + 1) / 2;
          for (int q = tid; q < ntiles; q += blockDim.x) {
            float acc[4][4];
            int rblk, cblk;
            dm_tile(Va, Vb, ldv, q, 0, cbn, acc, &rblk, &cblk);
            dm_tile_store<GLOBAL>(G, U, S, gbin, ns, L, nbins, rblk, cblk, acc);
          }
        }
      }
      __syncthreads();
      v0 += cbn;
      cb = CB;
    }
  }

  // T terms, diagonal and W: one warp per row r, lanes over c >= r.  The
  // pair's whole contribution (its rank-1 terms, already in the triangle, plus
  // these) goes to the FP64 accumulator here, and the triangle is cleared, so
  // that D~ and W are summed over pairs in FP64 only.  Rows and columns with
  // T = 0 hold nothing: every rank-1 term of a bin carries the weights of the
  // pixel pairs in it.
  const int nwarps = blockDim.x >> 5;
  const float c11 = (eta && Wa > 0 && Wb > 0) ? static_cast<float>(1.0 / (Wa * Wb)) : 0.f;
  const float cyy = (eta && Wa > 0 && Sb > 0) ? static_cast<float>(1.0 / (Wa * Sb)) : 0.f;
  const float cxx = (eta && Sa > 0 && Wb > 0) ? static_cast<float>(1.0 / (Sa * Wb)) : 0.f;
  const float cxy = (eta && Sa > 0 && Sb > 0) ? static_cast<float>(1.0 / (Sa * Sb)) : 0.f;
  for (int r = wid; r < L; r += nwarps) {
    const float4 tr = T4[r];
    if (tr.x == 0.f && tr.y == 0.f && tr.z == 0.f && tr.w == 0.f) continue;
    const float f1 = c11 * tr.x, fy = cyy * tr.z, fx = cxx * tr.y, fxy = cxy * tr.w;
    const int rb = tri_rowbase(r, L);
    // two columns per lane per iteration (independent chains)
    for (int c = r + lane; c < L; c += 64) {
      const int c2 = c + 32;
      const float4 tc = T4[c];
      const float4 tc2 = (c2 < L) ? T4[c2] : make_float4(0.f, 0.f, 0.f, 0.f);
      float v = f1 * tc.x + fy * tc.z + fx * tc.y + fxy * tc.w;
      const float v2 = f1 * tc2.x + fy * tc2.z + fx * tc2.y + fxy * tc2.w;
      if (c == r) v += tr.x;
      if (!GLOBAL) {
        // (r, c), (r, c2) owned by this lane: flush and clear
        const int Ar = gbin[r];
        const float t1 = U[rb + c] + v;
        if (t1 != 0.f) {
          const int Ac = gbin[c];
          red_add_f64_global(G + static_cast<int64_t>(min(Ar, Ac)) * nbins + max(Ar, Ac), static_cast<double>(t1));
          U[rb + c] = 0.f;
        }
        if (c2 < L) {
          const float t2 = U[rb + c2] + v2;
          if (t2 != 0.f) {
            const int Ac = gbin[c2];
            red_add_f64_global(G + static_cast<int64_t>(min(Ar, Ac)) * nbins + max(Ar, Ac), static_cast<double>(t2));
            U[rb + c2] = 0.f;
          }
        }
      } else {
        const int Ar = gbin[r];
        if (v != 0.f) {
          const int Ac = gbin[c];
          red_add_f64_global(G + static_cast<int64_t>(min(Ar, Ac)) * nbins + max(Ar, Ac),
                             static_cast<double>(v));
        }
        if (v2 != 0.f) {
          const int Ac = gbin[c2];
          red_add_f64_global(G + static_cast<int64_t>(min(Ar, Ac)) * nbins + max(Ar, Ac),
                             static_cast<double>(v2));
        }
      }
    }
    if (lane == 0) red_add_f64_global(wdm + gbin[r], static_cast<double>(tr.x));
  }
  __syncthreads();
  for (int k = tid; k < L; k += blockDim.x) T4[k] = make_float4(0.f, 0.f, 0.f, 0.f);
  __syncthreads();
}

template <bool GLOBAL, int CB>
__global__ void __launch_bounds__(kDmThreads, 1) dm_kernel(DmArgs A, const Chunk* chunks,
                                                           const int32_t* n_chunks_dev,
                                                           const int32_t* order, const int32_t* wide,
                                                           const int32_t* n_wide_dev, int scap, int Lalloc,
                                                           int kmin, int kmax, unsigned long long* counter) {
  extern __shared__ __align__(16) unsigned char sm[];
  __shared__ long long s_item;
  const int tid = threadIdx.x;
  const int nbins = A.n_par * A.n_perp;
  const int n_items = GLOBAL ? *n_wide_dev : *n_chunks_dev;
  const Lay y = layout(Lalloc, scap, A.max_len, GLOBAL, CB);
  float* U = reinterpret_cast<float*>(sm + y.U);
  float4* T4 = reinterpret_cast<float4*>(sm + y.T4);
  unsigned char* mark = sm + y.mark;
  int32_t* gbin = reinterpret_cast<int32_t*>(sm + y.gbin);
  // clear all accumulators once
  if (!GLOBAL) {
    const int nt = Lalloc * (Lalloc + 1) / 2;
    for (int k = tid; k < nt; k += blockDim.x) U[k] = 0.f;
  }
  for (int k = tid; k < Lalloc; k += blockDim.x) {
    T4[k] = make_float4(0.f, 0.f, 0.f, 0.f);
    mark[k] = 0;
  }
  __syncthreads();
  for (;;) {
    if (tid == 0) s_item = static_cast<long long>(atomicAdd(counter, 1ull));
    __syncthreads();
    const long long item = s_item;
    __syncthreads();
    if (item >= n_items) break;
    int t0, K, first, cnt, mock;
    if (!GLOBAL) {
      const Chunk ch = chunks[item];
      if (ch.K < kmin || ch.K > kmax) continue;   // another launch's band widths (uniform over the block)
      t0 = ch.t0; K = ch.K; first = ch.begin; cnt = ch.n; mock = ch.mock;
    } else {
      const int pi = wide[item];
      const int2 p = A.pairs[pi];
      if (!pair_band(A, p.x, p.y, A.cs[pi].y, &t0, &K)) continue;
      first = 0; cnt = 1; mock = A.F.mock[p.x];
    }
    // accumulators of the chunk's catalogue
    double* G = A.G + static_cast<int64_t>(mock) * nbins * nbins;
    double* wdm = A.wdm + static_cast<int64_t>(mock) * nbins;
    const int L = K * A.n_par;
    for (int k = tid; k < L; k += blockDim.x) {
      const int tt = k / A.n_par, p = k - tt * A.n_par;
      gbin[k] = p * A.n_perp + t0 + tt;
    }
    __syncthreads();
    for (int q = 0; q < cnt; ++q) {
      const int pi = GLOBAL ? wide[item] : order[first + q];
      dm_pair<GLOBAL, CB>(A, G, wdm, pi, t0, K, L, scap, sm, y);
    }
  }
}

__global__ void dm_finalize_kernel(const double* G, const double* wdm, double* D, double* wout, int nb,
                                   int n_mocks) {
  const int64_t nb2 = static_cast<int64_t>(nb) * nb;
  const int64_t n = nb2 * n_mocks;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int64_t m = k / nb2, e = k - m * nb2;
    const int r = static_cast<int>(e / nb), c = static_cast<int>(e - static_cast<int64_t>(r) * nb);
    const int lo = min(r, c), hi = max(r, c);
    const double w = wdm[m * nb + r];
    D[k] = (w != 0.0) ? G[m * nb2 + static_cast<int64_t>(lo) * nb + hi] / w : 0.0;
    if (wout && c == 0) wout[m * nb + r] = w;
  }
}

// first (global) forest index of each catalogue: forests are stored catalogue
// by catalogue, so it is the forest whose predecessor belongs to another one
__global__ void fbase_kernel(Forests F, int32_t* fbase) {
  for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < F.n;
       f += (int64_t)gridDim.x * blockDim.x)
    if (f == 0 || F.mock[f] != F.mock[f - 1]) fbase[F.mock[f]] = static_cast<int32_t>(f);
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

// Work counts of the closed form (one warp per kept forest pair, the D
// kernel's FP32 binning): for every rank-1 vector (column j of b over i of a,
// row i of a over j of b) the number |S_v| of distinct bins it touches, for
// the pair the number |S_pair| of distinct bins of all its pixel pairs, and
// the in-grid pixel pairs.  Bins are marked in lane-private bitmaps of the
// pair's band (word w of lane l at w * 32 + l: no bank conflicts).
__global__ void dm_work_kernel(DmArgs A, uint64_t thr, int all, int words_cap, DmWork* out) {
  extern __shared__ uint32_t wbm[];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  uint32_t* mine = wbm + static_cast<size_t>(wid) * 33 * words_cap;
  uint32_t* pbm = mine + 32 * words_cap;
  const int npar = A.n_par;
  const float fnpar = static_cast<float>(npar), fnperp = static_cast<float>(A.n_perp);
  unsigned long long n_pairs = 0, n_pix = 0;
  double sv2 = 0.0, sp2 = 0.0;
  for (int64_t k = warp; k < A.n_pairs; k += nw) {
    const int2 pr = A.pairs[k];
    if (pr.x < 0 || !keep_pair(pr.x, pr.y, A.seed, thr, all)) continue;
    const float2 cs = A.cs[k];
    int t0, K;
    if (!pair_band(A, pr.x, pr.y, cs.y, &t0, &K)) continue;
    const int words = (K * npar + 31) >> 5;
    if (words > words_cap) continue;   // (a band wider than the grid cannot occur)
    const int na = A.F.len[pr.x], nb = A.F.len[pr.y];
    const Pix* pa = A.pix + A.F.off[pr.x];
    const Pix* pb = A.pix + A.F.off[pr.y];
    const float cp = cs.x, sp = cs.y;
    const float Dc = (A.F.dref[pr.x] - A.F.dref[pr.y]) * cp, Ds = (A.F.dref[pr.x] + A.F.dref[pr.y]) * sp;
    for (int w = lane; w < words; w += 32) pbm[w] = 0u;
    __syncwarp();
    for (int side = 0; side < 2; ++side) {
      const int nvec = side == 0 ? nb : na;
      const int nother = side == 0 ? na : nb;
      for (int v0 = 0; v0 < nvec; v0 += 32) {
        const int v = v0 + lane;
        if (v < nvec) {
          for (int w = 0; w < words; ++w) mine[w * 32 + lane] = 0u;
          for (int o = 0; o < nother; ++o) {
            const int i = side == 0 ? o : v;
            const int j = side == 0 ? v : o;
            const float xi = pa[i].x;
            const int l = local_bin(make_float2(fmaf(xi, cp, Dc), fmaf(xi, sp, Ds)), pb[j].x, cp, sp, fnpar,
                                    fnperp, npar, t0);
            if (l >= 0) {
              mine[(l >> 5) * 32 + lane] |= 1u << (l & 31);
              if (side == 0) ++n_pix;
            }
          }
          int cnt = 0;
          for (int w = 0; w < words; ++w) {
            const uint32_t m = mine[w * 32 + lane];
            if (m) {
              cnt += __popc(m);
              atomicOr(&pbm[w], m);
            }
          }
          sv2 += static_cast<double>(cnt) * cnt;
        }
      }
    }
    __syncwarp();
    int c = 0;
    for (int w = lane; w < words; w += 32) c += __popc(pbm[w]);
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if (lane == 0) {
      sp2 += static_cast<double>(c) * c;
      n_pairs += 1;
    }
    __syncwarp();
  }
  for (int o = 16; o > 0; o >>= 1) {
    n_pix += __shfl_xor_sync(0xffffffffu, n_pix, o);
    sv2 += __shfl_xor_sync(0xffffffffu, sv2, o);
  }
  if (lane == 0) {
    atomicAdd(&out->pairs, n_pairs);
    atomicAdd(&out->pix, n_pix);
    atomicAdd(&out->sv2, sv2);
    atomicAdd(&out->sp2, sp2);
  }
}

}  // namespace

// single-block exclusive scan (defined in pairs.cu's namespace would be private)
namespace {
__global__ void dm_scan_kernel(const int32_t* in, int64_t n, int64_t* out) {
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
      int64_t v = part[k];
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

__global__ void to_int32_kernel(const int64_t* in, int32_t* out) { *out = static_cast<int32_t>(*in); }
}  // namespace

cudaError_t run_dmat(const DmArgs& a, const DevInfo& dev, void** scratch, size_t* scratch_cap,
                     cudaStream_t s) {
  const int nbins = a.n_par * a.n_perp;
  const int max_len = std::max(a.max_len, 1);
  // largest band that fits in shared memory with batches of 16 vectors (kfit)
  // and with batches of 32 (kfit2 <= kfit)
  int kfit = 0, scap = 0, kfit2 = 0, scap2 = 0;
  for (int K = a.n_perp; K >= 1; --K) {
    const int L = K * a.n_par;
    const int sc = scap_for(L, a.n_par, K, kCB);
    if (layout(L, sc, max_len, false, kCB).end + 64 <= dev.smem_optin) {
      kfit = K;
      scap = sc;
      break;
    }
  }
  for (int K = kfit; K >= 1; --K) {
    const int L = K * a.n_par;
    const int sc = scap_for(L, a.n_par, K, kCB2);
    if (layout(L, sc, max_len, false, kCB2).end + 64 <= dev.smem_optin) {
      kfit2 = K;
      scap2 = sc;
      break;
    }
  }
  // wide-pair configuration (triangle in global memory)
  const int Lw = a.n_perp * a.n_par;
  const int scapw = scap_for(Lw, a.n_par, a.n_perp, kCB);
  if (layout(Lw, scapw, max_len, true, kCB).end + 64 > dev.smem_optin) return cudaErrorInvalidValue;
  if (kfit == 0) {  // everything goes wide
    kfit = 1;
    scap = scap_for(a.n_par, a.n_par, 1, kCB);
  }

  const int n_mocks = std::max(a.n_mocks, 1);
  if (static_cast<int64_t>(n_mocks) * a.n_perp * kfit > (1 << 30)) return cudaErrorInvalidValue;
  const int ngroups = n_mocks * a.n_perp * kfit;   // (catalogue, first band row, K)
  auto al = [](size_t v) { return (v + 255) & ~size_t(255); };
  const int64_t n = a.n_pairs;
  size_t o = 0;
  const size_t o_key = o; o += al(std::max<int64_t>(n, 1) * 4);
  const size_t o_order = o; o += al(std::max<int64_t>(n, 1) * 4);
  const size_t o_wide = o; o += al(std::max<int64_t>(n, 1) * 4);
  const size_t o_count = o; o += al(ngroups * 4);
  const size_t o_cursor = o; o += al(ngroups * 4);
  const size_t o_start = o; o += al((ngroups + 1) * 8);
  const size_t o_nch = o; o += al(ngroups * 4);
  const size_t o_coff = o; o += al((ngroups + 1) * 8);
  const size_t o_chunks = o; o += al((n / kChunk + ngroups + 1) * sizeof(Chunk));
  const size_t o_fbase = o; o += al(static_cast<size_t>(n_mocks) * 4);
  const size_t o_misc = o; o += al(64);
  LYA_TRY(grow(scratch, scratch_cap, o));
  char* sc = static_cast<char*>(*scratch);
  int32_t* key = reinterpret_cast<int32_t*>(sc + o_key);
  int32_t* order = reinterpret_cast<int32_t*>(sc + o_order);
  int32_t* wide = reinterpret_cast<int32_t*>(sc + o_wide);
  int32_t* count = reinterpret_cast<int32_t*>(sc + o_count);
  int32_t* cursor = reinterpret_cast<int32_t*>(sc + o_cursor);
  int64_t* start = reinterpret_cast<int64_t*>(sc + o_start);
  int32_t* nch = reinterpret_cast<int32_t*>(sc + o_nch);
  int64_t* coff = reinterpret_cast<int64_t*>(sc + o_coff);
  Chunk* chunks = reinterpret_cast<Chunk*>(sc + o_chunks);
  int32_t* fbase = reinterpret_cast<int32_t*>(sc + o_fbase);
  int32_t* misc = reinterpret_cast<int32_t*>(sc + o_misc);   // [0] n_wide, [1] n_chunks
  unsigned long long* counter = reinterpret_cast<unsigned long long*>(sc + o_misc + 16);

  LYA_TRY(cudaMemsetAsync(count, 0, ngroups * 4, s));
  LYA_TRY(cudaMemsetAsync(cursor, 0, ngroups * 4, s));
  LYA_TRY(cudaMemsetAsync(misc, 0, 64, s));
  LYA_TRY(cudaMemsetAsync(a.G, 0, sizeof(double) * nbins * (size_t)nbins * n_mocks, s));
  LYA_TRY(cudaMemsetAsync(a.wdm, 0, sizeof(double) * nbins * (size_t)n_mocks, s));
  LYA_TRY(cudaMemsetAsync(fbase, 0, static_cast<size_t>(n_mocks) * 4, s));
  if (a.F.n > 0) LYA_COUNT(1), fbase_kernel<<<grid_for(a.F.n, 256), 256, 0, s>>>(a.F, fbase);
  DmArgs a2 = a;
  a2.fbase = fbase;
  const int all = a.p_subsample >= 1.0 ? 1 : 0;
  uint64_t thr = 0;
  if (!all && a.p_subsample > 0.0) thr = static_cast<uint64_t>(a.p_subsample * 18446744073709551616.0);
  if (a.p_subsample <= 0.0) return cudaSuccess;  // nothing kept: D = 0, W = 0
  if (n > 0) {
    LYA_COUNT(1), dm_select_kernel<<<grid_for(n, 256), 256, 0, s>>>(a2, thr, all, kfit, key, count, wide, misc);
    LYA_COUNT(1), dm_scan_kernel<<<1, 1024, 0, s>>>(count, ngroups, start);
    LYA_COUNT(1), dm_scatter_kernel<<<grid_for(n, 256), 256, 0, s>>>(n, key, start, cursor, order);
    LYA_COUNT(1), chunk_count_kernel<<<grid_for(ngroups, 256), 256, 0, s>>>(count, ngroups, nch);
    LYA_COUNT(1), dm_scan_kernel<<<1, 1024, 0, s>>>(nch, ngroups, coff);
    LYA_COUNT(1), chunk_fill_kernel<<<grid_for(ngroups, 256), 256, 0, s>>>(count, start, coff, ngroups, kfit,
                                                                           a.n_perp, chunks);
    LYA_COUNT(1), to_int32_kernel<<<1, 1, 0, s>>>(coff + ngroups, misc + 1);
    LYA_TRY(cudaGetLastError());
  }
  // shared-memory triangle: bands of up to kfit2 rows with batches of 32
  // vectors, the wider ones (up to kfit) with batches of 16
  if (kfit2 > 0) {
    const int L = kfit2 * a.n_par;
    const Lay y = layout(L, scap2, max_len, false, kCB2);
    LYA_TRY(set_max_dynamic_smem(reinterpret_cast<const void*>(dm_kernel<false, kCB2>), y.end));
    LYA_TRY(cudaMemsetAsync(counter, 0, 8, s));
    LYA_COUNT(1), dm_kernel<false, kCB2><<<dev.sms, kDmThreads, y.end, s>>>(a2, chunks, misc + 1, order, wide,
                                                                            misc, scap2, L, 1, kfit2, counter);
    LYA_TRY(cudaGetLastError());
  }
  if (kfit2 < kfit) {
    const int L = kfit * a.n_par;
    const Lay y = layout(L, scap, max_len, false, kCB);
    LYA_TRY(set_max_dynamic_smem(reinterpret_cast<const void*>(dm_kernel<false, kCB>), y.end));
    LYA_TRY(cudaMemsetAsync(counter, 0, 8, s));
    LYA_COUNT(1), dm_kernel<false, kCB><<<dev.sms, kDmThreads, y.end, s>>>(a2, chunks, misc + 1, order, wide, misc,
                                                                           scap, L, kfit2 + 1, kfit, counter);
    LYA_TRY(cudaGetLastError());
  }
  // wide pairs
  {
    const Lay y = layout(Lw, scapw, max_len, true, kCB);
    LYA_TRY(set_max_dynamic_smem(reinterpret_cast<const void*>(dm_kernel<true, kCB>), y.end));
    LYA_TRY(cudaMemsetAsync(counter, 0, 8, s));
    LYA_COUNT(1), dm_kernel<true, kCB><<<dev.sms, kDmThreads, y.end, s>>>(a2, chunks, misc + 1, order, wide, misc,
                                                                          scapw, Lw, 1, a.n_perp, counter);
    LYA_TRY(cudaGetLastError());
  }
  return cudaSuccess;
}

cudaError_t launch_dm_finalize(const double* G, const double* wdm, double* D, double* wdm_out, int nb,
                               int n_mocks, cudaStream_t s) {
  const int64_t n = static_cast<int64_t>(nb) * nb * n_mocks;
  if (n == 0) return cudaSuccess;
  LYA_COUNT(1), dm_finalize_kernel<<<grid_for(n, 256), 256, 0, s>>>(G, wdm, D, wdm_out, nb, n_mocks);
  return cudaGetLastError();
}

cudaError_t launch_dm_work(const DmArgs& a, const DevInfo& dev, DmWork* out, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(out, 0, sizeof(DmWork), s);
  if (e != cudaSuccess || a.n_pairs == 0 || a.p_subsample <= 0.0) return e;
  const int all = a.p_subsample >= 1.0 ? 1 : 0;
  const uint64_t thr = all ? 0 : static_cast<uint64_t>(a.p_subsample * 18446744073709551616.0);
  const int words_cap = (a.n_par * a.n_perp + 31) / 32;
  int warps = 8;
  while (warps > 1 && warps * 33 * words_cap * 4 > dev.smem_optin) warps >>= 1;
  const int smem = warps * 33 * words_cap * 4;
  if (smem > dev.smem_optin) return cudaErrorInvalidValue;
  e = set_max_dynamic_smem(reinterpret_cast<const void*>(dm_work_kernel), smem);
  if (e != cudaSuccess) return e;
  LYA_COUNT(1), dm_work_kernel<<<dev.sms * 4, warps * 32, smem, s>>>(a, thr, all, words_cap, out);
  return cudaGetLastError();
}

}  // namespace lya
