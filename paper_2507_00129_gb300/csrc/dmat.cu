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
// in shared memory (FP32), flushing it to the FP64 accumulator G (entries
// A <= B) with FP64 atomics once per chunk.  Per pair and per batch of CB
// columns (then rows): (a) every thread bins pixel pairs into dense per-column
// histograms, (b) one warp per column compacts its histogram into a sorted
// list of non-zero bins (and adds the column to the T vectors), (c) warps
// apply the rank-1 updates of the lists to the triangle.  Pairs whose band is
// too wide for shared memory take the same code with the triangle replaced by
// FP64 atomics into G.  Binning uses exactly the FP32 arithmetic of the xi
// kernel, so W^DM equals the xi weights of the kept pairs up to summation order.
#include <algorithm>
#include <math.h>

#include "lya_internal.cuh"

namespace lya {
namespace {

constexpr int kDmThreads = 512;
constexpr int kChunk = 128;

struct DmPlan {
  int kfit;      // largest band (rows) held in shared memory
  int cb;        // columns per batch
  int lcap;      // list capacity per column
  int max_len;
  int smem;      // bytes
  int L;         // local bins allocated = kfit * n_par (or full band for wide)
};

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
    const bool keep = keep_pair(p.x, p.y, A.seed, thr, all);
    int t_lo, K;
    if (keep && pair_band(A, p.x, p.y, A.cs[k].y, &t_lo, &K)) {
      if (K <= kfit) {
        kk = t_lo * kfit + (K - 1);
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
};

__global__ void chunk_fill_kernel(const int32_t* count, const int64_t* start, const int64_t* coff,
                                  int ngroups, int kfit, Chunk* chunks) {
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < ngroups; g += gridDim.x * blockDim.x) {
    const int c = count[g];
    for (int q = 0; q * kChunk < c; ++q) {
      Chunk ch;
      ch.begin = static_cast<int32_t>(start[g] + q * kChunk);
      ch.n = min(kChunk, c - q * kChunk);
      ch.t0 = g / kfit;
      ch.K = g % kfit + 1;
      chunks[coff[g] + q] = ch;
    }
  }
}

// Shared-memory layout of one block (offsets in bytes)
struct Lay {
  int U, Wacc, T4, dense, list, lcount, ucs, pixa, pixb, gbin, end;
};

__host__ __device__ inline Lay layout(int L, int cb, int lcap, int max_len, bool global_sink) {
  auto al = [](int v) { return (v + 15) & ~15; };
  Lay y;
  int o = 0;
  y.U = o;
  if (!global_sink) o += al(static_cast<int>((static_cast<int64_t>(L) * (L + 1) / 2) * 4));
  y.Wacc = o; o += al(L * 4);
  y.T4 = o; o += al(L * 16);
  y.dense = o; o += al(cb * L * 8);
  y.list = o; o += al(cb * lcap * 16);
  y.lcount = o; o += al(cb * 4);
  y.ucs = o; o += al(max_len * 8);
  y.pixa = o; o += al(max_len * 16);
  y.pixb = o; o += al(max_len * 16);
  y.gbin = o; o += al(L * 4);
  y.end = o;
  return y;
}

struct Entry {
  int32_t l;
  float a;
  float b;
  float pad;
};

template <bool GLOBAL>
__device__ __forceinline__ void sink_add(float* U, double* G, const int32_t* gbin, int nb, int r, int c,
                                         int64_t rowbase, float v) {
  if (!GLOBAL) {
    atomicAdd(&U[rowbase + c], v);
  } else {
    const int A = gbin[r], B = gbin[c];
    const int lo = min(A, B), hi = max(A, B);
    red_add_f64_global(G + static_cast<int64_t>(lo) * nb + hi, static_cast<double>(v));
  }
}

__device__ __forceinline__ int64_t tri_rowbase(int r, int L) {
  // index of (r, c) for c >= r is rowbase(r) + c
  return static_cast<int64_t>(r) * (2 * L - r + 1) / 2 - r;
}

// One forest pair: accumulate its contribution into the triangle (or G).
template <bool GLOBAL>
__device__ void dm_pair(const DmArgs& A, int item, int t0, int K, int L, int cb, int lcap,
                        unsigned char* sm, const Lay& y) {
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nwarps = blockDim.x >> 5;
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
  const float fnpar = static_cast<float>(npar), fnperp = static_cast<float>(A.n_perp);

  float* U = reinterpret_cast<float*>(sm + y.U);
  float4* T4 = reinterpret_cast<float4*>(sm + y.T4);
  float* dense = reinterpret_cast<float*>(sm + y.dense);
  Entry* list = reinterpret_cast<Entry*>(sm + y.list);
  int32_t* lcount = reinterpret_cast<int32_t*>(sm + y.lcount);
  float2* ucs = reinterpret_cast<float2*>(sm + y.ucs);
  Pix* pxa = reinterpret_cast<Pix*>(sm + y.pixa);
  Pix* pxb = reinterpret_cast<Pix*>(sm + y.pixb);
  const int32_t* gbin = reinterpret_cast<const int32_t*>(sm + y.gbin);

  const Pix* ga = A.pix + A.F.off[a];
  const Pix* gb = A.pix + A.F.off[b];
  for (int k = tid; k < na; k += blockDim.x) {
    const Pix p = ga[k];
    pxa[k] = p;
    ucs[k] = make_float2(fmaf(p.x, cp, Dc), fmaf(p.x, sp, Ds));
  }
  for (int k = tid; k < nb; k += blockDim.x) pxb[k] = gb[k];
  __syncthreads();

  // two passes: side 0 = columns j of b (histograms over i of a),
  //             side 1 = rows i of a (histograms over j of b)
  for (int side = 0; side < 2; ++side) {
    if (side == 1 && !eta) break;
    const int nvec = side == 0 ? nb : na;
    const int nother = side == 0 ? na : nb;
    // coefficients of the rank-1 terms of this side
    const double Wn = side == 0 ? Wa : Wb;   // normaliser of the summed-over forest
    const double Sn = side == 0 ? Sa : Sb;
    for (int v0 = 0; v0 < nvec; v0 += cb) {
      const int cbn = min(cb, nvec - v0);
      // (a) dense histograms: thread -> (vector vv = tid % cb, partners o)
      const int vv_t = tid % cb;
      const int ostep = blockDim.x / cb;
      for (int o = tid / cb; o < nother && vv_t < cbn; o += ostep) {
        const int vv = vv_t;
        const int i = side == 0 ? o : v0 + vv;   // pixel of a
        const int j = side == 0 ? v0 + vv : o;   // pixel of b
        const float2 u = ucs[i];
        const float dj = pxb[j].x;
        const float rp = fabsf(fmaf(-dj, cp, u.x));
        const float rt = fmaf(dj, sp, u.y);
        if (rp < fnpar && rt < fnperp) {
          const int p = static_cast<int>(rp);
          const int t = static_cast<int>(rt);
          const int l = (t - t0) * npar + p;
          // summed-over pixel: i of a (side 0) or j of b (side 1)
          const Pix q = side == 0 ? pxa[i] : pxb[j];
          atomicAdd(&dense[(vv * L + l) * 2 + 0], q.y);
          atomicAdd(&dense[(vv * L + l) * 2 + 1], q.y * q.w);
        }
      }
      __syncthreads();
      // (b) compaction, one warp per vector
      for (int vv = wid; vv < cbn; vv += nwarps) {
        const Pix me = side == 0 ? pxb[v0 + vv] : pxa[v0 + vv];   // the vector's own pixel
        const float wv = me.y;
        const float ca = (eta && Wn > 0.0) ? sqrtf(static_cast<float>(wv / Wn)) : 0.f;
        const float cbeta = (eta && Sn > 0.0) ? sqrtf(static_cast<float>(wv / Sn)) : 0.f;
        int m = 0;
        for (int l0 = 0; l0 < L; l0 += 32) {
          const int l = l0 + lane;
          float va = 0.f, vb = 0.f;
          if (l < L) {
            va = dense[(vv * L + l) * 2 + 0];
            vb = dense[(vv * L + l) * 2 + 1];
          }
          const bool nz = (va != 0.f) || (vb != 0.f);
          const unsigned msk = __ballot_sync(0xffffffffu, nz);
          if (nz) {
            const int pos = m + __popc(msk & ((1u << lane) - 1u));
            if (pos < lcap) {
              Entry e;
              e.l = l;
              e.a = va * ca;
              e.b = vb * cbeta;
              e.pad = 0.f;
              list[vv * lcap + pos] = e;
            }
            dense[(vv * L + l) * 2 + 0] = 0.f;
            dense[(vv * L + l) * 2 + 1] = 0.f;
            if (side == 0) {
              // T vectors from the column histograms of b's pixel j = v0 + vv
              const float wj = wv, yj = me.w;
              atomicAdd(&T4[l].x, wj * va);
              atomicAdd(&T4[l].y, wj * vb);
              atomicAdd(&T4[l].z, wj * yj * va);
              atomicAdd(&T4[l].w, wj * yj * vb);
            }
          }
          m += __popc(msk);
        }
        if (lane == 0) lcount[vv] = min(m, lcap);
      }
      __syncthreads();
      // (c) rank-1 updates: warps split over vectors and over k
      if (eta) {
        const int per = max(1, nwarps / max(cbn, 1));
        for (int w = wid; w < cbn * per; w += nwarps) {
          const int vv = w % cbn;
          const int part = w / cbn;
          const int m = lcount[vv];
          const Entry* li = list + vv * lcap;
          for (int k = lane + 32 * part; k < m; k += 32 * per) {
            const Entry ek = li[k];
            const int64_t rb = tri_rowbase(ek.l, L);
            for (int l = k; l < m; ++l) {
              const Entry el = li[l];
              const float v = -(ek.a * el.a + ek.b * el.b);
              sink_add<GLOBAL>(U, A.G, gbin, nbins, ek.l, el.l, rb, v);
            }
          }
        }
      }
      // the next batch's (a) writes only dense (already cleared); its barrier
      // separates these list reads from the next (b)
    }
    __syncthreads();
  }

  // T terms, diagonal and W: one warp per row r, lanes over c >= r
  const float c11 = (eta && Wa > 0 && Wb > 0) ? static_cast<float>(1.0 / (Wa * Wb)) : 0.f;
  const float cyy = (eta && Wa > 0 && Sb > 0) ? static_cast<float>(1.0 / (Wa * Sb)) : 0.f;
  const float cxx = (eta && Sa > 0 && Wb > 0) ? static_cast<float>(1.0 / (Sa * Wb)) : 0.f;
  const float cxy = (eta && Sa > 0 && Sb > 0) ? static_cast<float>(1.0 / (Sa * Sb)) : 0.f;
  float* Wacc = reinterpret_cast<float*>(sm + y.Wacc);
  for (int r = wid; r < L; r += nwarps) {
    const float4 tr = T4[r];
    if (tr.x == 0.f && tr.y == 0.f && tr.z == 0.f && tr.w == 0.f) continue;
    const float f1 = c11 * tr.x, fy = cyy * tr.z, fx = cxx * tr.y, fxy = cxy * tr.w;
    const int64_t rb = tri_rowbase(r, L);
    for (int c = r + lane; c < L; c += 32) {
      const float4 tc = T4[c];
      float v = f1 * tc.x + fy * tc.z + fx * tc.y + fxy * tc.w;
      if (c == r) v += tr.x;
      if (v != 0.f) {
        if (!GLOBAL) U[rb + c] += v;   // (r, c) owned by this lane
        else sink_add<true>(U, A.G, gbin, nbins, r, c, rb, v);
      }
    }
    if (lane == 0) {
      if (!GLOBAL) Wacc[r] += tr.x;
      else red_add_f64_global(A.wdm + gbin[r], static_cast<double>(tr.x));
    }
  }
  __syncthreads();
  for (int k = tid; k < L; k += blockDim.x) T4[k] = make_float4(0.f, 0.f, 0.f, 0.f);
  __syncthreads();
}

template <bool GLOBAL>
__global__ void __launch_bounds__(kDmThreads, 1) dm_kernel(DmArgs A, const Chunk* chunks,
                                                           const int32_t* n_chunks_dev,
                                                           const int32_t* order, const int32_t* wide,
                                                           const int32_t* n_wide_dev, int cb, int lcap,
                                                           int Lalloc, unsigned long long* counter) {
  extern __shared__ __align__(16) unsigned char sm[];
  __shared__ long long s_item;
  const int tid = threadIdx.x;
  const int nbins = A.n_par * A.n_perp;
  const int n_items = GLOBAL ? *n_wide_dev : *n_chunks_dev;
  const Lay y = layout(Lalloc, cb, lcap, A.max_len, GLOBAL);
  float* U = reinterpret_cast<float*>(sm + y.U);
  float* Wacc = reinterpret_cast<float*>(sm + y.Wacc);
  float* dense = reinterpret_cast<float*>(sm + y.dense);
  float4* T4 = reinterpret_cast<float4*>(sm + y.T4);
  int32_t* gbin = reinterpret_cast<int32_t*>(sm + y.gbin);
  // clear all accumulators once
  if (!GLOBAL) {
    const int64_t nt = static_cast<int64_t>(Lalloc) * (Lalloc + 1) / 2;
    for (int64_t k = tid; k < nt; k += blockDim.x) U[k] = 0.f;
  }
  for (int k = tid; k < Lalloc; k += blockDim.x) {
    Wacc[k] = 0.f;
    T4[k] = make_float4(0.f, 0.f, 0.f, 0.f);
  }
  for (int k = tid; k < cb * Lalloc * 2; k += blockDim.x) dense[k] = 0.f;
  __syncthreads();
  for (;;) {
    if (tid == 0) s_item = static_cast<long long>(atomicAdd(counter, 1ull));
    __syncthreads();
    const long long item = s_item;
    __syncthreads();
    if (item >= n_items) break;
    int t0, K, first, cnt;
    if (!GLOBAL) {
      const Chunk ch = chunks[item];
      t0 = ch.t0; K = ch.K; first = ch.begin; cnt = ch.n;
    } else {
      const int pi = wide[item];
      const int2 p = A.pairs[pi];
      if (!pair_band(A, p.x, p.y, A.cs[pi].y, &t0, &K)) continue;
      first = 0; cnt = 1;
    }
    const int L = K * A.n_par;
    for (int k = tid; k < L; k += blockDim.x) {
      const int tt = k / A.n_par, p = k - tt * A.n_par;
      gbin[k] = p * A.n_perp + t0 + tt;
    }
    __syncthreads();
    for (int q = 0; q < cnt; ++q) {
      const int pi = GLOBAL ? wide[item] : order[first + q];
      dm_pair<GLOBAL>(A, pi, t0, K, L, cb, lcap, sm, y);
    }
    if (!GLOBAL) {
      // flush the triangle and W of this chunk
      const int64_t nt = static_cast<int64_t>(L) * (L + 1) / 2;
      const int nwarps = blockDim.x >> 5, wid = tid >> 5, lane = tid & 31;
      for (int r = wid; r < L; r += nwarps) {
        const int64_t rb = tri_rowbase(r, L);
        const int Ar = gbin[r];
        for (int c = r + lane; c < L; c += 32) {
          const float v = U[rb + c];
          if (v != 0.f) {
            const int Ac = gbin[c];
            red_add_f64_global(A.G + static_cast<int64_t>(min(Ar, Ac)) * nbins + max(Ar, Ac),
                               static_cast<double>(v));
            U[rb + c] = 0.f;
          }
        }
      }
      for (int k = tid; k < L; k += blockDim.x) {
        if (Wacc[k] != 0.f) {
          red_add_f64_global(A.wdm + gbin[k], static_cast<double>(Wacc[k]));
          Wacc[k] = 0.f;
        }
      }
      (void)nt;
      __syncthreads();
    }
  }
}

__global__ void dm_finalize_kernel(const double* G, const double* wdm, double* D, double* wout, int nb) {
  const int64_t n = static_cast<int64_t>(nb) * nb;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int r = static_cast<int>(k / nb), c = static_cast<int>(k - static_cast<int64_t>(r) * nb);
    const int lo = min(r, c), hi = max(r, c);
    const double w = wdm[r];
    D[k] = (w != 0.0) ? G[static_cast<int64_t>(lo) * nb + hi] / w : 0.0;
    if (wout && c == 0) wout[r] = w;
  }
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
  // largest band that fits in shared memory
  int cb = 8, kfit = 0, lcap = 0;
  for (int K = a.n_perp; K >= 1; --K) {
    const int L = K * a.n_par;
    const int lc = std::min(L, 2 * (a.n_par + K) + 2);
    const Lay y = layout(L, cb, lc, max_len, false);
    if (y.end + 64 <= dev.smem_optin) {
      kfit = K;
      lcap = lc;
      break;
    }
  }
  // wide-pair configuration (triangle in global memory)
  int cbw = 8, Lw = a.n_perp * a.n_par, lcapw = std::min(Lw, 2 * (a.n_par + a.n_perp) + 2);
  while (cbw > 1 && layout(Lw, cbw, lcapw, max_len, true).end + 64 > dev.smem_optin) cbw >>= 1;
  if (layout(Lw, cbw, lcapw, max_len, true).end + 64 > dev.smem_optin) return cudaErrorInvalidValue;
  if (kfit == 0) kfit = 1;  // everything goes wide

  const int ngroups = a.n_perp * kfit;
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
  int32_t* misc = reinterpret_cast<int32_t*>(sc + o_misc);   // [0] n_wide, [1] n_chunks
  unsigned long long* counter = reinterpret_cast<unsigned long long*>(sc + o_misc + 16);

  LYA_TRY(cudaMemsetAsync(count, 0, ngroups * 4, s));
  LYA_TRY(cudaMemsetAsync(cursor, 0, ngroups * 4, s));
  LYA_TRY(cudaMemsetAsync(misc, 0, 64, s));
  LYA_TRY(cudaMemsetAsync(a.G, 0, sizeof(double) * nbins * (size_t)nbins, s));
  LYA_TRY(cudaMemsetAsync(a.wdm, 0, sizeof(double) * nbins, s));
  const int all = a.p_subsample >= 1.0 ? 1 : 0;
  uint64_t thr = 0;
  if (!all && a.p_subsample > 0.0) thr = static_cast<uint64_t>(a.p_subsample * 18446744073709551616.0);
  if (a.p_subsample <= 0.0) return cudaSuccess;  // nothing kept: D = 0, W = 0
  if (n > 0) {
    LYA_COUNT(1), dm_select_kernel<<<grid_for(n, 256), 256, 0, s>>>(a, thr, all, kfit, key, count, wide, misc);
    LYA_COUNT(1), dm_scan_kernel<<<1, 1024, 0, s>>>(count, ngroups, start);
    LYA_COUNT(1), dm_scatter_kernel<<<grid_for(n, 256), 256, 0, s>>>(n, key, start, cursor, order);
    LYA_COUNT(1), chunk_count_kernel<<<grid_for(ngroups, 256), 256, 0, s>>>(count, ngroups, nch);
    LYA_COUNT(1), dm_scan_kernel<<<1, 1024, 0, s>>>(nch, ngroups, coff);
    LYA_COUNT(1), chunk_fill_kernel<<<grid_for(ngroups, 256), 256, 0, s>>>(count, start, coff, ngroups, kfit, chunks);
    LYA_COUNT(1), to_int32_kernel<<<1, 1, 0, s>>>(coff + ngroups, misc + 1);
    LYA_TRY(cudaGetLastError());
  }
  // main launch: shared-memory triangle
  {
    const int L = kfit * a.n_par;
    const Lay y = layout(L, cb, lcap, max_len, false);
    LYA_TRY(cudaFuncSetAttribute(dm_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, y.end));
    LYA_TRY(cudaMemsetAsync(counter, 0, 8, s));
    LYA_COUNT(1), dm_kernel<false><<<dev.sms, kDmThreads, y.end, s>>>(a, chunks, misc + 1, order, wide, misc, cb,
                                                        lcap, L, counter);
    LYA_TRY(cudaGetLastError());
  }
  // wide pairs
  {
    const Lay y = layout(Lw, cbw, lcapw, max_len, true);
    LYA_TRY(cudaFuncSetAttribute(dm_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, y.end));
    LYA_TRY(cudaMemsetAsync(counter, 0, 8, s));
    LYA_COUNT(1), dm_kernel<true><<<dev.sms, kDmThreads, y.end, s>>>(a, chunks, misc + 1, order, wide, misc, cbw,
                                                       lcapw, Lw, counter);
    LYA_TRY(cudaGetLastError());
  }
  return cudaSuccess;
}

cudaError_t launch_dm_finalize(const double* G, const double* wdm, double* D, double* wdm_out, int nb,
                               cudaStream_t s) {
  const int64_t n = static_cast<int64_t>(nb) * nb;
  if (n == 0) return cudaSuccess;
  LYA_COUNT(1), dm_finalize_kernel<<<grid_for(n, 256), 256, 0, s>>>(G, wdm, D, wdm_out, nb);
  return cudaGetLastError();
}

}  // namespace lya
