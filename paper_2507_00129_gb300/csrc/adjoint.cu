// Gradient of L = sum_A g_A xi_A with respect to delta and w (chain rule of
// Eq. 2.4):
//   dL/d delta_i = w_i sum_j gamma_A (w d)_j
//   dL/d w_i     = delta_i sum_j gamma_A (w d)_j - sum_j rho_A w_j
// with gamma_A = g_A / W_A, rho_A = gamma_A xi_A - e_A, j over the in-grid partners
// of i, for L = sum_A g_A xi_A + sum_A e_A W_A (e = 0 unless given).
//
// Each pixel is owned by one warp (work item = 32 consecutive pixels of one
// forest), which walks the forest's full neighbour list (both orientations of
// every stored pair) and gathers gamma/rho from a shared-memory table: no
// atomics, deterministic.  Each pixel pair is binned with the same FP32
// operations, in the same operand roles, as the forward kernel (first forest
// of the stored pair on the "i" side), so forward and backward agree on every
// bin.  The table has a zero guard row and column; out-of-grid pairs are
// clamped into them, so the inner loop has no branch.  Per-neighbour FP32
// partial sums are added into two-term (hi, lo) accumulators (Knuth's TwoSum).
#include <algorithm>

#include "lya_internal.cuh"

namespace lya {
namespace {

constexpr int kAdjWarps = 8;

__device__ __forceinline__ void two_sum_add(float& hi, float& lo, float x) {
  const float s = hi + x;
  const float bp = s - hi;
  const float e = (hi - (s - bp)) + (x - bp);
  hi = s;
  lo += e;
}

__device__ __forceinline__ int count_below_x(const float4* a, int n, float v) {
  int lo = 0, hi = n;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (a[mid].x < v) lo = mid + 1; else hi = mid;
  }
  return lo;
}
__device__ __forceinline__ int count_below_y(const float4* a, int n, float v) {
  int lo = 0, hi = n;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (a[mid].y < v) lo = mid + 1; else hi = mid;
  }
  return lo;
}

__global__ void degree_kernel(const int2* pairs, int64_t n, int32_t* deg) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int2 p = pairs[k];
    atomicAdd(&deg[p.x], 1);
    atomicAdd(&deg[p.y], 1);
  }
}

__global__ void adj_fill_kernel(const int2* pairs, int64_t n, const int64_t* start, int32_t* cursor,
                                int2* adj) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int2 p = pairs[k];
    const int pa = atomicAdd(&cursor[p.x], 1);
    adj[start[p.x] + pa] = make_int2(static_cast<int>(k), 1);   // owner is the first forest
    const int pb = atomicAdd(&cursor[p.y], 1);
    adj[start[p.y] + pb] = make_int2(static_cast<int>(k), 0);
  }
}

// Work items (forest, 32-pixel chunk) are laid out in the order of `order`
// (forests in HEALPix-cell order, so consecutive items read overlapping
// neighbour sets from L2), or in index order if it is NULL.
__device__ __forceinline__ int64_t item_forest(const int32_t* order, int64_t k) {
  return order ? static_cast<int64_t>(order[k]) : k;
}

__global__ void chunks_per_forest(Forests F, const int32_t* order, int32_t* nch) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < F.n;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int64_t f = item_forest(order, k);
    nch[k] = (f >= 0) ? (F.len[f] + 31) / 32 : 0;
  }
}

__global__ void item_fill_kernel(Forests F, const int32_t* order, const int64_t* coff, int2* items) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < F.n;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int64_t f = item_forest(order, k);
    if (f < 0) continue;
    const int n = (F.len[f] + 31) / 32;
    for (int c = 0; c < n; ++c) items[coff[k] + c] = make_int2(static_cast<int>(f), c);
  }
}

__global__ void scan1_kernel(const int32_t* in, int64_t n, int64_t* out) {
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

__global__ void __launch_bounds__(kAdjWarps * 32) adjoint_kernel(AdjArgs A, const int2* adj,
                                                                 const int64_t* adj_start,
                                                                 const int2* items,
                                                                 const int64_t* n_items_dev, int seg,
                                                                 unsigned long long* counter) {
  extern __shared__ __align__(16) unsigned char sm[];
  const int npar = A.n_par, nperp = A.n_perp;
  // table entry (p, t) at p * (n_perp + 1) + t; row p = n_par and column
  // t = n_perp are the zero guard
  const int tstride = nperp + 1;
  const int tab_n = (npar + 1) * tstride;
  float2* table = reinterpret_cast<float2*>(sm);
  const int tab_bytes = ((tab_n * 8) + 15) & ~15;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  float4* buf = reinterpret_cast<float4*>(sm + tab_bytes + wid * seg * 16);
  for (int k = threadIdx.x; k < tab_n; k += blockDim.x) {
    const int p = k / tstride, t = k - p * tstride;
    float2 e = make_float2(0.f, 0.f);
    if (p < npar && t < nperp) {
      const int bin = p * nperp + t;
      const double w = A.wsum[bin];
      const double g = (w != 0.0) ? A.grad_xi[bin] / w : 0.0;
      // rho = gamma xi - dL/dW (the weight sum's own dependence on w)
      const double r = g * A.xi[bin] - (A.grad_wsum ? A.grad_wsum[bin] : 0.0);
      e = make_float2(static_cast<float>(g), static_cast<float>(r));
    }
    table[k] = e;
  }
  __syncthreads();
  // key (M + p) * tstride + (M + t), M = bits of 2^23, minus this offset is p * tstride + t
  const uint32_t tbase = smem_addr(table) -
                         8u * (kMagicBits * static_cast<uint32_t>(tstride) + kMagicBits);
  const float fnpar = static_cast<float>(npar), fnperp = static_cast<float>(nperp);
  const float pmax = __uint_as_float(kMagicBits + static_cast<uint32_t>(npar));
  const float tmax = __uint_as_float(kMagicBits + static_cast<uint32_t>(nperp));
  const int64_t n_items = *n_items_dev;
  for (;;) {
    unsigned long long it = 0;
    if (lane == 0) it = atomicAdd(counter, 1ull);
    it = __shfl_sync(0xffffffffu, it, 0);
    if (it >= static_cast<unsigned long long>(n_items)) break;
    const int2 item = items[it];
    const int f = item.x;
    const int nf = A.F.len[f];
    const int i = item.y * 32 + lane;
    const bool valid = i < nf;
    const Pix me = valid ? A.pix[A.F.off[f] + i] : make_float4(0.f, 0.f, 0.f, 0.f);
    const float ref_f = A.F.dref[f];
    float g1h = 0.f, g1l = 0.f, g2h = 0.f, g2l = 0.f;
    const int64_t e0 = adj_start[f], e1 = adj_start[f + 1];
    for (int64_t e = e0; e < e1; ++e) {
      const int2 ent = adj[e];
      const int2 pr = A.pairs[ent.x];
      const float2 cs = A.cs[ent.x];
      const float cp = cs.x, sp = cs.y;
      const bool first = ent.y != 0;
      const int o = first ? pr.y : pr.x;
      const int no = A.F.len[o];
      if (no == 0 || nf == 0) continue;
      const Pix* po = A.pix + A.F.off[o];
      const float ref_o = A.F.dref[o];
      // pair constants with the stored (first, second) roles
      const float ref1 = first ? ref_f : ref_o, ref2 = first ? ref_o : ref_f;
      const float Dc = (ref1 - ref2) * cp, Ds = (ref1 + ref2) * sp;
      float a1 = 0.f, a2 = 0.f;
      for (int j0 = 0; j0 < no; j0 += seg) {
        const int segn = min(seg, no - j0);
        __syncwarp();
        if (first) {
          for (int k = lane; k < segn; k += 32) buf[k] = po[j0 + k];
        } else {
          for (int k = lane; k < segn; k += 32) {
            const Pix q = po[j0 + k];
            buf[k] = make_float4(fmaf(q.x, cp, Dc), fmaf(q.x, sp, Ds), q.y, q.z);
          }
        }
        __syncwarp();
        if (first) {
          // lanes are first-forest pixels; loop over second-forest pixels (d~ in .x)
          const float uc = fmaf(me.x, cp, Dc), us = fmaf(me.x, sp, Ds);
          const int last = max(0, min(31, nf - 1 - item.y * 32));
          const float ucf = __shfl_sync(0xffffffffu, uc, 0);
          const float usf = __shfl_sync(0xffffffffu, us, 0);
          const float ucl = __shfl_sync(0xffffffffu, uc, last);
          float dlo = (ucf - fnpar) / cp, dhi = (ucl + fnpar) / cp;
          if (sp > 0.f) dhi = fminf(dhi, (fnperp - usf) / sp);
          dlo -= fabsf(dlo) * 1e-5f + 1e-2f;
          dhi += fabsf(dhi) * 1e-5f + 1e-2f;
          const int jlo = count_below_x(buf, segn, dlo), jhi = count_below_x(buf, segn, dhi);
#pragma unroll 4
          for (int j = jlo; j < jhi; ++j) {
            const float4 q = buf[j];
            const float rp = fabsf(fmaf(-q.x, cp, uc));
            const float rt = fmaf(q.x, sp, us);
            const float pf = fminf(__fadd_rd(rp, kMagic), pmax), tf = fminf(__fadd_rd(rt, kMagic), tmax);
            const uint32_t idx = __float_as_uint(pf) * static_cast<uint32_t>(tstride) + __float_as_uint(tf);
            float2 gr;
            asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(gr.x), "=f"(gr.y) : "r"(tbase + (idx << 3)));
            a1 = fmaf(gr.x, q.z, a1);
            a2 = fmaf(gr.y, q.y, a2);
          }
        } else {
          // lanes are second-forest pixels; loop over first-forest pixels
          // (buf: .x = uc_i, .y = us_i, .z = w_i, .w = (w d)_i)
          const float dme = me.x;
          const float dmin_l = __shfl_sync(0xffffffffu, dme, 0);
          const int last = max(0, min(31, nf - 1 - item.y * 32));
          const float dmax_l = __shfl_sync(0xffffffffu, dme, last);
          // |uc_i - d cp| < npar  ->  uc_i in (dmin cp - npar, dmax cp + npar)
          float ulo = fmaf(dmin_l, cp, -fnpar), uhi = fmaf(dmax_l, cp, fnpar);
          ulo -= fabsf(ulo) * 1e-5f + 1e-3f;
          uhi += fabsf(uhi) * 1e-5f + 1e-3f;
          // rt = d sp + us_i < nperp  ->  us_i < nperp - dmin sp
          float vhi = fmaf(-dmin_l, sp, fnperp);
          vhi += fabsf(vhi) * 1e-5f + 1e-3f;
          const int ilo = count_below_x(buf, segn, ulo);
          const int ihi = min(count_below_x(buf, segn, uhi), count_below_y(buf, segn, vhi));
#pragma unroll 4
          for (int j = ilo; j < ihi; ++j) {
            const float4 q = buf[j];
            const float rp = fabsf(fmaf(-dme, cp, q.x));
            const float rt = fmaf(dme, sp, q.y);
            const float pf = fminf(__fadd_rd(rp, kMagic), pmax), tf = fminf(__fadd_rd(rt, kMagic), tmax);
            const uint32_t idx = __float_as_uint(pf) * static_cast<uint32_t>(tstride) + __float_as_uint(tf);
            float2 gr;
            asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(gr.x), "=f"(gr.y) : "r"(tbase + (idx << 3)));
            a1 = fmaf(gr.x, q.w, a1);
            a2 = fmaf(gr.y, q.z, a2);
          }
        }
      }
      two_sum_add(g1h, g1l, a1);
      two_sum_add(g2h, g2l, a2);
    }
    if (valid) {
      const int64_t gi = A.F.off[f] + i - A.pix_base;
      const float s1 = g1h + g1l, s2 = g2h + g2l;
      A.grad_delta[gi] = me.y * s1;
      A.grad_weight[gi] = A.delta[gi] * s1 - s2;
    }
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

cudaError_t run_adjoint(const AdjArgs& a, const DevInfo& dev, void** scratch, size_t* scratch_cap,
                        cudaStream_t s) {
  const int64_t nf = a.F.n;
  const int64_t np = a.n_pairs;
  auto al = [](size_t v) { return (v + 255) & ~size_t(255); };
  // work items (forest, 32-pixel chunk): at most n_pix/32 + n_forests
  const int64_t max_items = a.n_pix / 32 + nf + 1;
  size_t o = 0;
  const size_t o_deg = o; o += al((nf + 1) * 4);
  const size_t o_start = o; o += al((nf + 1) * 8);
  const size_t o_cursor = o; o += al((nf + 1) * 4);
  const size_t o_adj = o; o += al(std::max<int64_t>(2 * np, 1) * 8);
  const size_t o_nch = o; o += al((nf + 1) * 4);
  const size_t o_coff = o; o += al((nf + 1) * 8);
  const size_t o_items = o; o += al(max_items * 8);
  const size_t o_misc = o; o += 256;
  LYA_TRY(grow(scratch, scratch_cap, o));
  char* sc = static_cast<char*>(*scratch);
  int32_t* deg = reinterpret_cast<int32_t*>(sc + o_deg);
  int64_t* start = reinterpret_cast<int64_t*>(sc + o_start);
  int32_t* cursor = reinterpret_cast<int32_t*>(sc + o_cursor);
  int2* adj = reinterpret_cast<int2*>(sc + o_adj);
  int32_t* nch = reinterpret_cast<int32_t*>(sc + o_nch);
  int64_t* coff = reinterpret_cast<int64_t*>(sc + o_coff);
  int2* items = reinterpret_cast<int2*>(sc + o_items);
  unsigned long long* counter = reinterpret_cast<unsigned long long*>(sc + o_misc);
  LYA_TRY(cudaMemsetAsync(deg, 0, (nf + 1) * 4, s));
  LYA_TRY(cudaMemsetAsync(cursor, 0, (nf + 1) * 4, s));
  LYA_TRY(cudaMemsetAsync(counter, 0, 8, s));
  if (np > 0) LYA_COUNT(1), degree_kernel<<<grid_for(np, 256), 256, 0, s>>>(a.pairs, np, deg);
  LYA_COUNT(1), scan1_kernel<<<1, 1024, 0, s>>>(deg, nf, start);
  if (np > 0) LYA_COUNT(1), adj_fill_kernel<<<grid_for(np, 256), 256, 0, s>>>(a.pairs, np, start, cursor, adj);
  LYA_COUNT(1), chunks_per_forest<<<grid_for(nf, 256), 256, 0, s>>>(a.F, a.forder, nch);
  LYA_COUNT(1), scan1_kernel<<<1, 1024, 0, s>>>(nch, nf, coff);
  LYA_COUNT(1), item_fill_kernel<<<grid_for(nf, 256), 256, 0, s>>>(a.F, a.forder, coff, items);
  LYA_TRY(cudaGetLastError());
  const int tab_n = (a.n_par + 1) * (a.n_perp + 1);
  int seg = ((std::max(a.max_len, 1) + 31) / 32) * 32;
  if (seg > 1024) seg = 1024;
  const int smem = ((tab_n * 8 + 15) & ~15) + kAdjWarps * seg * 16;
  if (smem > dev.smem_optin) return cudaErrorInvalidValue;
  LYA_TRY(set_max_dynamic_smem(reinterpret_cast<const void*>(adjoint_kernel), smem));
  int per_sm = 0;
  LYA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, adjoint_kernel, kAdjWarps * 32, smem));
  if (per_sm < 1) return cudaErrorInvalidValue;
  LYA_COUNT(1), adjoint_kernel<<<per_sm * dev.sms, kAdjWarps * 32, smem, s>>>(a, adj, start, items, coff + nf, seg,
                                                                counter);
  return cudaGetLastError();
}

}  // namespace lya
