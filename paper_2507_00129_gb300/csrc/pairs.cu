// Forest-pair neighbour list (Section 2.1: only forests inside a
// neighbourhood set by the maximum separation; Section 3.1: HEALPix cells).
//
// 1. every forest gets its HEALPix NESTED cell (ang2pix written from the
//    projection formulas of Gorski et al. 2005, ApJ 622, 759, Section 4);
// 2. forests are counting-sorted by cell and each occupied cell gets a centre
//    (normalised mean unit vector), an angular radius (largest member offset)
//    and the smallest member distance;
// 3. cell pairs survive when the closest two members could still hold an
//    in-grid pixel pair:  (dmin_1 + dmin_2) sin(max(0, theta_c - r_1 - r_2)/2) < r_perp_max;
// 4. member pairs of surviving cell pairs are kept when
//    (dmin_a + dmin_b) sin(theta_ab / 2) < r_perp_max  (exact: r_perp >= that bound).
// Counts and fills use the same iteration order, so the list is deterministic.
#include <math.h>

#include <algorithm>

#include "lya_internal.cuh"

namespace lya {
namespace {

constexpr int kT = 256;

__device__ __forceinline__ uint32_t spread_bits(uint32_t v) {
  // interleave: bit k of v goes to bit 2k
  v &= 0xFFFFu;
  v = (v | (v << 8)) & 0x00FF00FFu;
  v = (v | (v << 4)) & 0x0F0F0F0Fu;
  v = (v | (v << 2)) & 0x33333333u;
  v = (v | (v << 1)) & 0x55555555u;
  return v;
}

// HEALPix NESTED pixel of the direction with z = cos(colatitude) and
// longitude phi in [0, 2 pi).  nside is a power of two, <= 8192.
__device__ int64_t ang2pix_nest(int nside, double z, double phi) {
  const double za = fabs(z);
  const double tt = phi * (2.0 / M_PI);  // in [0, 4)
  int face, ix, iy;
  if (za <= 2.0 / 3.0) {
    const double t1 = nside * (0.5 + tt);
    const double t2 = nside * (0.75 * z);
    int jp = static_cast<int>(t1 - t2);  // ascending edge line index
    int jm = static_cast<int>(t1 + t2);  // descending edge line index
    const int ifp = jp / nside;
    const int ifm = jm / nside;
    if (ifp == ifm) face = ifp | 4;
    else if (ifp < ifm) face = ifp;
    else face = ifm + 8;
    ix = jm & (nside - 1);
    iy = nside - (jp & (nside - 1)) - 1;
  } else {
    int ntt = static_cast<int>(tt);
    if (ntt > 3) ntt = 3;
    const double tp = tt - ntt;
    const double tmp = nside * sqrt(3.0 * (1.0 - za));
    int jp = static_cast<int>(tp * tmp);
    int jm = static_cast<int>((1.0 - tp) * tmp);
    if (jp > nside - 1) jp = nside - 1;
    if (jm > nside - 1) jm = nside - 1;
    if (z >= 0) {
      face = ntt;
      ix = nside - jm - 1;
      iy = nside - jp - 1;
    } else {
      face = ntt + 8;
      ix = jp;
      iy = jm;
    }
  }
  if (face < 0) face = 0;
  if (face > 11) face = 11;
  ix = min(max(ix, 0), nside - 1);
  iy = min(max(iy, 0), nside - 1);
  return static_cast<int64_t>(face) * nside * nside + (spread_bits(ix) | (spread_bits(iy) << 1));
}

__global__ void cell_kernel(Forests F, int64_t f0, int64_t nf, int nside, int32_t* cell,
                            int32_t* count) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nf;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int64_t f = f0 + k;
    int32_t c = -1;
    if (F.len[f] > 0) {
      double phi = atan2(F.uy[f], F.ux[f]);
      if (phi < 0) phi += 2.0 * M_PI;
      if (phi >= 2.0 * M_PI) phi = 0.0;
      double z = F.uz[f];
      z = fmin(1.0, fmax(-1.0, z));
      c = static_cast<int32_t>(ang2pix_nest(nside, z, phi));
      atomicAdd(&count[c], 1);
    }
    cell[k] = c;
  }
}

// sub-sample of each forest: the nested HEALPix pixel of its line of sight
__global__ void subsample_id_kernel(Forests F, int nside, int32_t* id) {
  for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < F.n;
       f += (int64_t)gridDim.x * blockDim.x) {
    double phi = atan2(F.uy[f], F.ux[f]);
    if (phi < 0) phi += 2.0 * M_PI;
    if (phi >= 2.0 * M_PI) phi = 0.0;
    const double z = fmin(1.0, fmax(-1.0, F.uz[f]));
    id[f] = (F.len[f] > 0) ? static_cast<int32_t>(ang2pix_nest(nside, z, phi)) : 0;
  }
}

// exclusive scan of n int32 counts into n+1 int64 offsets, one block
__global__ void scan_kernel(const int32_t* in, int64_t n, int64_t* out) {
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

__global__ void scatter_kernel(const int32_t* cell, int64_t f0, int64_t nf, const int64_t* start,
                               int32_t* cursor, int32_t* members) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nf;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int32_t c = cell[k];
    if (c < 0) continue;
    const int pos = atomicAdd(&cursor[c], 1);
    members[start[c] + pos] = static_cast<int32_t>(f0 + k);
  }
}

__global__ void cell_sort_kernel(const int64_t* start, int64_t ncells, int32_t* members) {
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < ncells;
       c += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = start[c], e = start[c + 1];
    for (int64_t i = b + 1; i < e; ++i) {
      const int32_t v = members[i];
      int64_t j = i - 1;
      while (j >= b && members[j] > v) {
        members[j + 1] = members[j];
        --j;
      }
      members[j + 1] = v;
    }
  }
}

// order[k] = k-th non-empty forest in cell order (members[0 .. *n_members)), -1 past the end
__global__ void forder_kernel(const int32_t* members, const int64_t* n_members, int64_t nf, int32_t* order) {
  const int64_t m = *n_members;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nf;
       k += (int64_t)gridDim.x * blockDim.x)
    order[k] = (k < m) ? members[k] : -1;
}

__global__ void occupied_flags(const int32_t* count, int64_t ncells, int32_t* flag) {
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < ncells;
       c += (int64_t)gridDim.x * blockDim.x)
    flag[c] = count[c] > 0 ? 1 : 0;
}

__global__ void occupied_list(const int32_t* count, const int64_t* fpos, int64_t ncells, int32_t* occ) {
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < ncells;
       c += (int64_t)gridDim.x * blockDim.x)
    if (count[c] > 0) occ[fpos[c]] = static_cast<int32_t>(c);
}

struct CellStat {
  double cx, cy, cz;   // unit centre
  double radius;       // angular radius (rad), rounded up
  double dmin;         // smallest member distance
  int64_t begin;       // member range
  int32_t n;
};

__global__ void cell_stat_kernel(Forests F, const int32_t* occ, int64_t K, const int64_t* start,
                                 const int32_t* members, CellStat* st) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t k = warp; k < K; k += nw) {
    const int32_t c = occ[k];
    const int64_t b = start[c], e = start[c + 1];
    double sx = 0, sy = 0, sz = 0, dm = INFINITY;
    for (int64_t i = b + lane; i < e; i += 32) {
      const int32_t f = members[i];
      sx += F.ux[f];
      sy += F.uy[f];
      sz += F.uz[f];
      dm = fmin(dm, F.dmin[f]);
    }
    sx = warp_sum_f64(sx);
    sy = warp_sum_f64(sy);
    sz = warp_sum_f64(sz);
    dm = -warp_max_f64(-dm);
    const double nrm = sqrt(sx * sx + sy * sy + sz * sz);
    double cx = 1, cy = 0, cz = 0;
    if (nrm > 0) { cx = sx / nrm; cy = sy / nrm; cz = sz / nrm; }
    double ch = 0;
    for (int64_t i = b + lane; i < e; i += 32) {
      const int32_t f = members[i];
      const double dx = F.ux[f] - cx, dy = F.uy[f] - cy, dz = F.uz[f] - cz;
      ch = fmax(ch, sqrt(dx * dx + dy * dy + dz * dz));
    }
    ch = warp_max_f64(ch);
    if (lane == 0) {
      CellStat s;
      s.cx = cx; s.cy = cy; s.cz = cz;
      s.radius = 2.0 * asin(fmin(1.0, 0.5 * ch)) * (1.0 + 1e-12) + 1e-12;
      s.dmin = dm;
      s.begin = b;
      s.n = static_cast<int32_t>(e - b);
      st[k] = s;
    }
  }
}

__device__ __forceinline__ bool cells_may_pair(const CellStat& p, const CellStat& q, double rperp_max) {
  const double dx = p.cx - q.cx, dy = p.cy - q.cy, dz = p.cz - q.cz;
  const double ch = sqrt(dx * dx + dy * dy + dz * dz);
  const double th = 2.0 * asin(fmin(1.0, 0.5 * ch)) * (1.0 - 1e-12);
  const double gap = th - p.radius - q.radius;
  if (gap <= 0.0) return true;
  return (p.dmin + q.dmin) * sin(0.5 * gap) * (1.0 - 1e-12) < rperp_max;
}

// one warp per row c1: cell pairs (c1, c2 >= c1); MODE 0 counts, MODE 1 fills
template <int MODE>
__global__ void cell_pair_kernel(const CellStat* st, int64_t K, double rperp_max, int32_t* row_count,
                                 const int64_t* row_off, int2* out) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t c1 = warp; c1 < K; c1 += nw) {
    const CellStat p = st[c1];
    int64_t run = (MODE == 1) ? row_off[c1] : 0;
    int32_t cnt = 0;
    for (int64_t base = c1; base < K; base += 32) {
      const int64_t c2 = base + lane;
      bool ok = false;
      if (c2 < K) ok = cells_may_pair(p, st[c2], rperp_max);
      const unsigned m = __ballot_sync(0xffffffffu, ok);
      if (MODE == 1 && ok) {
        const int r = __popc(m & ((1u << lane) - 1u));
        out[run + r] = make_int2(static_cast<int>(c1), static_cast<int>(c2));
      }
      run += __popc(m);
      cnt += __popc(m);
    }
    if (MODE == 0 && lane == 0) row_count[c1] = cnt;
  }
}

__device__ __forceinline__ bool forests_pair(const Forests& F, int32_t a, int32_t b, double rperp_max) {
  const double dx = F.ux[a] - F.ux[b], dy = F.uy[a] - F.uy[b], dz = F.uz[a] - F.uz[b];
  const double s = 0.5 * sqrt(dx * dx + dy * dy + dz * dz);
  return (F.dmin[a] + F.dmin[b]) * s < rperp_max;
}

// one warp per cell pair; MODE 0 counts, MODE 1 fills
template <int MODE>
__global__ void forest_pair_kernel(Forests F, const CellStat* st, const int2* cp, int64_t ncp,
                                   const int32_t* members, double rperp_max, int32_t* cnt_out,
                                   const int64_t* off, int2* out) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t k = warp; k < ncp; k += nw) {
    const int2 c = cp[k];
    const CellStat p = st[c.x], q = st[c.y];
    const bool same = (c.x == c.y);
    int64_t run = (MODE == 1) ? off[k] : 0;
    int32_t cnt = 0;
    for (int ia = 0; ia < p.n; ++ia) {
      const int32_t fa = members[p.begin + ia];
      for (int ib0 = same ? ia + 1 : 0; ib0 < q.n; ib0 += 32) {
        const int ib = ib0 + lane;
        bool ok = false;
        int32_t fb = 0;
        if (ib < q.n) {
          fb = members[q.begin + ib];
          ok = forests_pair(F, fa, fb, rperp_max);
        }
        const unsigned m = __ballot_sync(0xffffffffu, ok);
        if (MODE == 1 && ok) {
          const int r = __popc(m & ((1u << lane) - 1u));
          out[run + r] = make_int2(min(fa, fb), max(fa, fb));
        }
        run += __popc(m);
        cnt += __popc(m);
      }
    }
    if (MODE == 0 && lane == 0) cnt_out[k] = cnt;
  }
}

__global__ void pair_geometry_kernel(const int2* pairs, int64_t n, Forests F, double inv_dpar,
                                     double inv_dperp, float2* cs) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int2 p = pairs[k];
    if (p.x < 0 || p.y < 0) {   // rejected pair (see check_pairs_kernel)
      cs[k] = make_float2(0.f, 0.f);
      continue;
    }
    const double ax = F.ux[p.x], ay = F.uy[p.x], az = F.uz[p.x];
    const double bx = F.ux[p.y], by = F.uy[p.y], bz = F.uz[p.y];
    const double sx = ax + bx, sy = ay + by, sz = az + bz;
    const double dx = ax - bx, dy = ay - by, dz = az - bz;
    const double c = 0.5 * sqrt(sx * sx + sy * sy + sz * sz);
    const double s = 0.5 * sqrt(dx * dx + dy * dy + dz * dz);
    cs[k] = make_float2(static_cast<float>(c * inv_dpar), static_cast<float>(s * inv_dperp));
  }
}

__global__ void pack_pairs_kernel(const int32_t* a, const int32_t* b, int64_t n, int2* out) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x)
    out[k] = make_int2(a[k], b[k]);
}

__global__ void unpack_pairs_kernel(const int2* p, int64_t n, int32_t* a, int32_t* b) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x) {
    a[k] = p[k].x;
    b[k] = p[k].y;
  }
}

// key = mock * (n_perp + 1) + first r_perp row of the pair's band (n_perp if
// the pair has nothing in the grid); same FP32 arithmetic as the pair kernel
__global__ void band_key_kernel(const int2* pairs, const float2* cs, int64_t n, Forests F, const Pix* pix,
                                int n_perp, int32_t* key, int32_t* count) {
  const float fnperp = static_cast<float>(n_perp);
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int2 p = pairs[k];
    int t = n_perp;
    const int na = F.len[p.x], nb = F.len[p.y];
    if (na > 0 && nb > 0) {
      const float sp = cs[k].y;
      const float Ds = (F.dref[p.x] + F.dref[p.y]) * sp;
      const float rt_min = fmaf(pix[F.off[p.y]].x, sp, fmaf(pix[F.off[p.x]].x, sp, Ds));
      if (rt_min < fnperp) t = static_cast<int>(rt_min);
    }
    const int kk = F.mock[p.x] * (n_perp + 1) + t;
    key[k] = kk;
    atomicAdd(&count[kk], 1);
  }
}

__global__ void band_scatter_kernel(const int2* pairs, const float2* cs, int64_t n, const int32_t* key,
                                    const int64_t* start, int32_t* cursor, int2* pairs_out,
                                    float2* cs_out) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int32_t kk = key[k];
    const int64_t pos = start[kk] + atomicAdd(&cursor[kk], 1);
    pairs_out[pos] = pairs[k];
    cs_out[pos] = cs[k];
  }
}

// ---- forest x quasar pairs: cells of the forests against cells of the quasars

// one warp per forest cell c1, all quasar cells c2; MODE 0 counts, MODE 1 fills
template <int MODE>
__global__ void cross_cell_pair_kernel(const CellStat* sf, int64_t KF, const CellStat* sq, int64_t KQ,
                                       double rperp_max, int32_t* row_count, const int64_t* row_off, int2* out) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t c1 = warp; c1 < KF; c1 += nw) {
    const CellStat p = sf[c1];
    int64_t run = (MODE == 1) ? row_off[c1] : 0;
    int32_t cnt = 0;
    for (int64_t base = 0; base < KQ; base += 32) {
      const int64_t c2 = base + lane;
      const bool ok = (c2 < KQ) && cells_may_pair(p, sq[c2], rperp_max);
      const unsigned m = __ballot_sync(0xffffffffu, ok);
      if (MODE == 1 && ok) out[run + __popc(m & ((1u << lane) - 1u))] = make_int2(static_cast<int>(c1), static_cast<int>(c2));
      run += __popc(m);
      cnt += __popc(m);
    }
    if (MODE == 0 && lane == 0) row_count[c1] = cnt;
  }
}

// Forest a and quasar q can hold an in-grid pixel: r_perp >= (d_first + d_q) sin(theta/2) and
// |r_par| >= (distance from d_q to the forest's distance range) cos(theta/2), both exact bounds.
// Compared as squares (all terms are non-negative): sin^2(theta/2) = |n_a - n_q|^2 / 4 and
// cos^2(theta/2) = |n_a + n_q|^2 / 4, so no square root is taken (FP64 is slow on this part).
__device__ __forceinline__ bool forest_quasar_pair(const Forests& F, int32_t a, const Forests& Q, int32_t q,
                                                   double rpar_max, double rperp_max) {
  const double ax = F.ux[a], ay = F.uy[a], az = F.uz[a];
  const double qx = Q.ux[q], qy = Q.uy[q], qz = Q.uz[q];
  const double dx = ax - qx, dy = ay - qy, dz = az - qz;
  const double sx = ax + qx, sy = ay + qy, sz = az + qz;
  const double s2 = 0.25 * (dx * dx + dy * dy + dz * dz);
  const double c2 = 0.25 * (sx * sx + sy * sy + sz * sz);
  const double dsum = F.dmin[a] + Q.dmin[q];
  if (dsum * dsum * s2 >= rperp_max * rperp_max) return false;
  const double gap = fmax(0.0, fmax(Q.dmin[q] - F.dmax[a], F.dmin[a] - Q.dmin[q]));
  return gap * gap * c2 < rpar_max * rpar_max;
}

// one warp per (forest cell, quasar cell) pair; MODE 0 counts, MODE 1 fills (forest, quasar)
template <int MODE>
__global__ void cross_member_kernel(Forests F, Forests Q, const CellStat* sf, const CellStat* sq, const int2* cp,
                                    int64_t ncp, const int32_t* mf, const int32_t* mq, double rpar_max,
                                    double rperp_max, const int64_t* own, int32_t* cnt_out, const int64_t* off,
                                    int2* out) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t k = warp; k < ncp; k += nw) {
    const int2 c = cp[k];
    const CellStat p = sf[c.x], q = sq[c.y];
    int64_t run = (MODE == 1) ? off[k] : 0;
    int32_t cnt = 0;
    for (int ia = 0; ia < p.n; ++ia) {
      const int32_t fa = mf[p.begin + ia];
      const int64_t own_q = own ? own[fa] : -1;
      for (int ib0 = 0; ib0 < q.n; ib0 += 32) {
        const int ib = ib0 + lane;
        bool ok = false;
        int32_t fq = 0;
        if (ib < q.n) {
          fq = mq[q.begin + ib];
          ok = (fq != own_q) && forest_quasar_pair(F, fa, Q, fq, rpar_max, rperp_max);
        }
        const unsigned m = __ballot_sync(0xffffffffu, ok);
        if (MODE == 1 && ok) out[run + __popc(m & ((1u << lane) - 1u))] = make_int2(fa, fq);
        run += __popc(m);
        cnt += __popc(m);
      }
    }
    if (MODE == 0 && lane == 0) cnt_out[k] = cnt;
  }
}

__global__ void xcount_kernel(const int2* p, int64_t n, int32_t* count) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(&count[p[k].x], 1);
}

__global__ void xscatter_kernel(const int2* p, int64_t n, const int64_t* start, int32_t* cursor, int2* out) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    const int2 v = p[k];
    out[start[v.x] + atomicAdd(&cursor[v.x], 1)] = v;
  }
}

int grid_for(int64_t n, int threads) {
  int64_t b = (n + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > 1 << 16) b = 1 << 16;
  return static_cast<int>(b);
}

#define LYA_TRY(x)                          \
  do {                                      \
    cudaError_t e_ = (x);                   \
    if (e_ != cudaSuccess) return e_;       \
  } while (0)

}  // namespace

cudaError_t build_pairs(const Forests& F, int64_t f0, int64_t f1, const PairBuild& pb, int2** pairs,
                        int64_t* cap, int64_t pair_base, int64_t* n_out, void** scratch,
                        size_t* scratch_cap, int32_t* forder, cudaStream_t s) {
  *n_out = 0;
  const int64_t nf = f1 - f0;
  // a single forest has no pairs: no order is needed (-1 = no work)
  if (forder && nf > 0 && nf <= 1) LYA_TRY(cudaMemsetAsync(forder + f0, 0xff, nf * 4, s));
  if (nf <= 1) return cudaSuccess;
  const int64_t ncells = 12LL * pb.nside * pb.nside;
  // scratch layout (bytes, 16-aligned)
  auto al = [](size_t v) { return (v + 255) & ~size_t(255); };
  const size_t o_cell = 0;
  const size_t o_count = o_cell + al(nf * 4);
  const size_t o_cursor = o_count + al(ncells * 4);
  const size_t o_start = o_cursor + al(ncells * 4);
  const size_t o_members = o_start + al((ncells + 1) * 8);
  const size_t o_flag = o_members + al(nf * 4);
  const size_t o_fpos = o_flag + al(ncells * 4);
  const size_t o_occ = o_fpos + al((ncells + 1) * 8);
  const size_t o_stat = o_occ + al(ncells * 4);
  const size_t o_end = o_stat + al(sizeof(CellStat) * (size_t)std::min<int64_t>(ncells, nf));
  LYA_TRY(grow(scratch, scratch_cap, o_end));
  char* sc = static_cast<char*>(*scratch);
  int32_t* cell = reinterpret_cast<int32_t*>(sc + o_cell);
  int32_t* count = reinterpret_cast<int32_t*>(sc + o_count);
  int32_t* cursor = reinterpret_cast<int32_t*>(sc + o_cursor);
  int64_t* start = reinterpret_cast<int64_t*>(sc + o_start);
  int32_t* members = reinterpret_cast<int32_t*>(sc + o_members);
  int32_t* flag = reinterpret_cast<int32_t*>(sc + o_flag);
  int64_t* fpos = reinterpret_cast<int64_t*>(sc + o_fpos);
  int32_t* occ = reinterpret_cast<int32_t*>(sc + o_occ);
  CellStat* st = reinterpret_cast<CellStat*>(sc + o_stat);

  LYA_TRY(cudaMemsetAsync(count, 0, ncells * 4, s));
  LYA_TRY(cudaMemsetAsync(cursor, 0, ncells * 4, s));
  LYA_COUNT(1), cell_kernel<<<grid_for(nf, kT), kT, 0, s>>>(F, f0, nf, pb.nside, cell, count);
  LYA_TRY(cudaGetLastError());
  LYA_COUNT(1), scan_kernel<<<1, 1024, 0, s>>>(count, ncells, start);
  LYA_COUNT(1), scatter_kernel<<<grid_for(nf, kT), kT, 0, s>>>(cell, f0, nf, start, cursor, members);
  LYA_COUNT(1), cell_sort_kernel<<<grid_for(ncells, kT), kT, 0, s>>>(start, ncells, members);
  // the non-empty forests in cell order (nested HEALPix: neighbours on the sky stay close), kept for
  // kernels that walk forests and read their neighbours; the rest of the slot stays -1
  if (forder) LYA_COUNT(1), forder_kernel<<<grid_for(nf, kT), kT, 0, s>>>(members, start + ncells, nf, forder + f0);
  LYA_COUNT(1), occupied_flags<<<grid_for(ncells, kT), kT, 0, s>>>(count, ncells, flag);
  LYA_COUNT(1), scan_kernel<<<1, 1024, 0, s>>>(flag, ncells, fpos);
  LYA_COUNT(1), occupied_list<<<grid_for(ncells, kT), kT, 0, s>>>(count, fpos, ncells, occ);
  LYA_TRY(cudaGetLastError());
  int64_t K = 0;
  LYA_TRY(cudaMemcpyAsync(&K, fpos + ncells, 8, cudaMemcpyDeviceToHost, s));
  LYA_TRY(cudaStreamSynchronize(s));
  if (K == 0) return cudaSuccess;
  LYA_COUNT(1), cell_stat_kernel<<<grid_for(K * 32, kT), kT, 0, s>>>(F, occ, K, start, members, st);
  LYA_TRY(cudaGetLastError());

  // cell pairs: count rows, scan, fill
  int32_t* row_count = nullptr;
  int64_t* row_off = nullptr;
  int2* cpairs = nullptr;
  LYA_TRY(cudaMallocAsync(reinterpret_cast<void**>(&row_count), K * 4, s));
  LYA_TRY(cudaMallocAsync(reinterpret_cast<void**>(&row_off), (K + 1) * 8, s));
  LYA_COUNT(1), cell_pair_kernel<0><<<grid_for(K * 32, kT), kT, 0, s>>>(st, K, pb.rperp_max, row_count, nullptr,
                                                           nullptr);
  LYA_COUNT(1), scan_kernel<<<1, 1024, 0, s>>>(row_count, K, row_off);
  int64_t M = 0;
  LYA_TRY(cudaMemcpyAsync(&M, row_off + K, 8, cudaMemcpyDeviceToHost, s));
  LYA_TRY(cudaStreamSynchronize(s));
  cudaError_t err = cudaSuccess;
  int32_t* pc = nullptr;
  int64_t* poff = nullptr;
  int64_t P = 0;
  if (M > 0) {
    err = cudaMallocAsync(reinterpret_cast<void**>(&cpairs), M * sizeof(int2), s);
    if (err == cudaSuccess) {
      LYA_COUNT(1), cell_pair_kernel<1><<<grid_for(K * 32, kT), kT, 0, s>>>(st, K, pb.rperp_max, nullptr, row_off,
                                                               cpairs);
      err = cudaMallocAsync(reinterpret_cast<void**>(&pc), M * 4, s);
    }
    if (err == cudaSuccess) err = cudaMallocAsync(reinterpret_cast<void**>(&poff), (M + 1) * 8, s);
    if (err == cudaSuccess) {
      LYA_COUNT(1), forest_pair_kernel<0><<<grid_for(M * 32, kT), kT, 0, s>>>(F, st, cpairs, M, members,
                                                                pb.rperp_max, pc, nullptr, nullptr);
      LYA_COUNT(1), scan_kernel<<<1, 1024, 0, s>>>(pc, M, poff);
      err = cudaGetLastError();
    }
    if (err == cudaSuccess) err = cudaMemcpyAsync(&P, poff + M, 8, cudaMemcpyDeviceToHost, s);
    if (err == cudaSuccess) err = cudaStreamSynchronize(s);
    if (err == cudaSuccess && pair_base + P > *cap) {
      // grow, keeping earlier content
      int64_t ncap = std::max<int64_t>(pair_base + P, (*cap) * 3 / 2);
      int2* np = nullptr;
      err = cudaMalloc(reinterpret_cast<void**>(&np), ncap * sizeof(int2));
      if (err == cudaSuccess && *pairs && pair_base > 0)
        err = cudaMemcpyAsync(np, *pairs, pair_base * sizeof(int2), cudaMemcpyDeviceToDevice, s);
      if (err == cudaSuccess) {
        cudaStreamSynchronize(s);
        if (*pairs) cudaFree(*pairs);
        *pairs = np;
        *cap = ncap;
      } else if (np) {
        cudaFree(np);
      }
    }
    if (err == cudaSuccess && P > 0) {
      LYA_COUNT(1), forest_pair_kernel<1><<<grid_for(M * 32, kT), kT, 0, s>>>(F, st, cpairs, M, members,
                                                                pb.rperp_max, nullptr, poff,
                                                                *pairs + pair_base);
      err = cudaGetLastError();
    }
  }
  if (cpairs) cudaFreeAsync(cpairs, s);
  if (pc) cudaFreeAsync(pc, s);
  if (poff) cudaFreeAsync(poff, s);
  cudaFreeAsync(row_count, s);
  cudaFreeAsync(row_off, s);
  if (err == cudaSuccess) err = cudaStreamSynchronize(s);
  *n_out = P;
  return err;
}

cudaError_t launch_pair_geometry(const int2* pairs, int64_t n, Forests F, double inv_dpar,
                                 double inv_dperp, float2* cs, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  LYA_COUNT(1), pair_geometry_kernel<<<grid_for(n, kT), kT, 0, s>>>(pairs, n, F, inv_dpar, inv_dperp, cs);
  return cudaGetLastError();
}

cudaError_t sort_pairs_by_band(int2* pairs, float2* cs, int64_t n, Forests F, const Pix* pix, int n_perp,
                               int n_mocks, void** scratch, size_t* scratch_cap, cudaStream_t s) {
  if (n <= 1) return cudaSuccess;
  const int64_t nkeys = static_cast<int64_t>(n_mocks) * (n_perp + 1);
  auto al = [](size_t v) { return (v + 255) & ~size_t(255); };
  const size_t o_key = 0;
  const size_t o_count = o_key + al(n * 4);
  const size_t o_cursor = o_count + al(nkeys * 4);
  const size_t o_start = o_cursor + al(nkeys * 4);
  const size_t o_pairs = o_start + al((nkeys + 1) * 8);
  const size_t o_cs = o_pairs + al(n * 8);
  const size_t o_end = o_cs + al(n * 8);
  LYA_TRY(grow(scratch, scratch_cap, o_end));
  char* sc = static_cast<char*>(*scratch);
  int32_t* key = reinterpret_cast<int32_t*>(sc + o_key);
  int32_t* count = reinterpret_cast<int32_t*>(sc + o_count);
  int32_t* cursor = reinterpret_cast<int32_t*>(sc + o_cursor);
  int64_t* start = reinterpret_cast<int64_t*>(sc + o_start);
  int2* p2 = reinterpret_cast<int2*>(sc + o_pairs);
  float2* c2 = reinterpret_cast<float2*>(sc + o_cs);
  LYA_TRY(cudaMemsetAsync(count, 0, nkeys * 4, s));
  LYA_TRY(cudaMemsetAsync(cursor, 0, nkeys * 4, s));
  LYA_COUNT(1), band_key_kernel<<<grid_for(n, kT), kT, 0, s>>>(pairs, cs, n, F, pix, n_perp, key, count);
  LYA_COUNT(1), scan_kernel<<<1, 1024, 0, s>>>(count, nkeys, start);
  LYA_COUNT(1), band_scatter_kernel<<<grid_for(n, kT), kT, 0, s>>>(pairs, cs, n, key, start, cursor, p2, c2);
  LYA_TRY(cudaGetLastError());
  LYA_TRY(cudaMemcpyAsync(pairs, p2, n * 8, cudaMemcpyDeviceToDevice, s));
  LYA_TRY(cudaMemcpyAsync(cs, c2, n * 8, cudaMemcpyDeviceToDevice, s));
  return cudaSuccess;
}

cudaError_t launch_subsample_ids(const Forests& F, int nside, int32_t* id, cudaStream_t s) {
  if (F.n == 0) return cudaSuccess;
  LYA_COUNT(1), subsample_id_kernel<<<grid_for(F.n, kT), kT, 0, s>>>(F, nside, id);
  return cudaGetLastError();
}

cudaError_t launch_pack_pairs(const int32_t* a, const int32_t* b, int64_t n, int2* out,
                              cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  LYA_COUNT(1), pack_pairs_kernel<<<grid_for(n, kT), kT, 0, s>>>(a, b, n, out);
  return cudaGetLastError();
}

cudaError_t launch_unpack_pairs(const int2* p, int64_t n, int32_t* a, int32_t* b, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  LYA_COUNT(1), unpack_pairs_kernel<<<grid_for(n, kT), kT, 0, s>>>(p, n, a, b);
  return cudaGetLastError();
}

}  // namespace lya

namespace lya {
namespace {

// HEALPix cell index of one point set (forests or quasars): members sorted by
// cell and the statistics of the occupied cells.  One device allocation.
struct CellIndex {
  void* buf = nullptr;
  int32_t* members = nullptr;
  CellStat* st = nullptr;
  int64_t K = 0;
};

cudaError_t index_cells(const Forests& F, int nside, CellIndex* ci, cudaStream_t s) {
  const int64_t nf = F.n;
  const int64_t ncells = 12LL * nside * nside;
  auto al = [](size_t v) { return (v + 255) & ~size_t(255); };
  const size_t o_cell = 0;
  const size_t o_count = o_cell + al(nf * 4);
  const size_t o_cursor = o_count + al(ncells * 4);
  const size_t o_start = o_cursor + al(ncells * 4);
  const size_t o_members = o_start + al((ncells + 1) * 8);
  const size_t o_flag = o_members + al(nf * 4);
  const size_t o_fpos = o_flag + al(ncells * 4);
  const size_t o_occ = o_fpos + al((ncells + 1) * 8);
  const size_t o_stat = o_occ + al(ncells * 4);
  const size_t o_end = o_stat + al(sizeof(CellStat) * (size_t)std::max<int64_t>(1, std::min<int64_t>(ncells, nf)));
  LYA_TRY(cudaMallocAsync(&ci->buf, o_end, s));
  char* sc = static_cast<char*>(ci->buf);
  int32_t* cell = reinterpret_cast<int32_t*>(sc + o_cell);
  int32_t* count = reinterpret_cast<int32_t*>(sc + o_count);
  int32_t* cursor = reinterpret_cast<int32_t*>(sc + o_cursor);
  int64_t* start = reinterpret_cast<int64_t*>(sc + o_start);
  ci->members = reinterpret_cast<int32_t*>(sc + o_members);
  int32_t* flag = reinterpret_cast<int32_t*>(sc + o_flag);
  int64_t* fpos = reinterpret_cast<int64_t*>(sc + o_fpos);
  int32_t* occ = reinterpret_cast<int32_t*>(sc + o_occ);
  ci->st = reinterpret_cast<CellStat*>(sc + o_stat);
  LYA_TRY(cudaMemsetAsync(count, 0, ncells * 4, s));
  LYA_TRY(cudaMemsetAsync(cursor, 0, ncells * 4, s));
  LYA_COUNT(1), cell_kernel<<<grid_for(nf, kT), kT, 0, s>>>(F, 0, nf, nside, cell, count);
  LYA_COUNT(1), scan_kernel<<<1, 1024, 0, s>>>(count, ncells, start);
  LYA_COUNT(1), scatter_kernel<<<grid_for(nf, kT), kT, 0, s>>>(cell, 0, nf, start, cursor, ci->members);
  LYA_COUNT(1), cell_sort_kernel<<<grid_for(ncells, kT), kT, 0, s>>>(start, ncells, ci->members);
  LYA_COUNT(1), occupied_flags<<<grid_for(ncells, kT), kT, 0, s>>>(count, ncells, flag);
  LYA_COUNT(1), scan_kernel<<<1, 1024, 0, s>>>(flag, ncells, fpos);
  LYA_COUNT(1), occupied_list<<<grid_for(ncells, kT), kT, 0, s>>>(count, fpos, ncells, occ);
  LYA_TRY(cudaGetLastError());
  LYA_TRY(cudaMemcpyAsync(&ci->K, fpos + ncells, 8, cudaMemcpyDeviceToHost, s));
  LYA_TRY(cudaStreamSynchronize(s));
  if (ci->K > 0) {
    LYA_COUNT(1), cell_stat_kernel<<<grid_for(ci->K * 32, kT), kT, 0, s>>>(F, occ, ci->K, start, ci->members, ci->st);
    LYA_TRY(cudaGetLastError());
  }
  return cudaSuccess;
}

}  // namespace

cudaError_t build_cross_pairs(const Forests& F, const Forests& Q, int nside, double rpar_max, double rperp_max,
                              const int64_t* own, int2** pairs, int64_t* cap, int64_t* qoff, int64_t* n_out,
                              cudaStream_t s) {
  *n_out = 0;
  LYA_TRY(cudaMemsetAsync(qoff, 0, (F.n + 1) * 8, s));
  if (F.n == 0 || Q.n == 0) return cudaSuccess;
  int2* unsorted = nullptr;
  int32_t* fcount = nullptr;
  CellIndex cf, cq;
  int32_t* row_count = nullptr;
  int64_t* row_off = nullptr;
  int2* cpairs = nullptr;
  int32_t* pc = nullptr;
  int64_t* poff = nullptr;
  int64_t M = 0, P = 0;
  cudaError_t err = index_cells(F, nside, &cf, s);
  if (err == cudaSuccess) err = index_cells(Q, nside, &cq, s);
  if (err == cudaSuccess && cf.K > 0 && cq.K > 0) {
    err = cudaMallocAsync(reinterpret_cast<void**>(&row_count), cf.K * 4, s);
    if (err == cudaSuccess) err = cudaMallocAsync(reinterpret_cast<void**>(&row_off), (cf.K + 1) * 8, s);
    if (err == cudaSuccess) {
      LYA_COUNT(1), cross_cell_pair_kernel<0><<<grid_for(cf.K * 32, kT), kT, 0, s>>>(cf.st, cf.K, cq.st, cq.K,
                                                                           rperp_max, row_count, nullptr, nullptr);
      LYA_COUNT(1), scan_kernel<<<1, 1024, 0, s>>>(row_count, cf.K, row_off);
      err = cudaGetLastError();
    }
    if (err == cudaSuccess) err = cudaMemcpyAsync(&M, row_off + cf.K, 8, cudaMemcpyDeviceToHost, s);
    if (err == cudaSuccess) err = cudaStreamSynchronize(s);
    if (err == cudaSuccess && M > 0) {
      err = cudaMallocAsync(reinterpret_cast<void**>(&cpairs), M * sizeof(int2), s);
      if (err == cudaSuccess) err = cudaMallocAsync(reinterpret_cast<void**>(&pc), M * 4, s);
      if (err == cudaSuccess) err = cudaMallocAsync(reinterpret_cast<void**>(&poff), (M + 1) * 8, s);
      if (err == cudaSuccess) {
        LYA_COUNT(1), cross_cell_pair_kernel<1><<<grid_for(cf.K * 32, kT), kT, 0, s>>>(cf.st, cf.K, cq.st, cq.K,
                                                                             rperp_max, nullptr, row_off, cpairs);
        LYA_COUNT(1), cross_member_kernel<0><<<grid_for(M * 32, kT), kT, 0, s>>>(
            F, Q, cf.st, cq.st, cpairs, M, cf.members, cq.members, rpar_max, rperp_max, own, pc, nullptr, nullptr);
        LYA_COUNT(1), scan_kernel<<<1, 1024, 0, s>>>(pc, M, poff);
        err = cudaGetLastError();
      }
      if (err == cudaSuccess) err = cudaMemcpyAsync(&P, poff + M, 8, cudaMemcpyDeviceToHost, s);
      if (err == cudaSuccess) err = cudaStreamSynchronize(s);
      if (err == cudaSuccess && P > *cap) {
        int64_t ncap = std::max<int64_t>(P, (*cap) * 3 / 2);
        if (*pairs) { cudaFree(*pairs); *pairs = nullptr; *cap = 0; }
        err = cudaMalloc(reinterpret_cast<void**>(pairs), ncap * sizeof(int2));
        if (err == cudaSuccess) *cap = ncap; else *pairs = nullptr;
      }
      if (err == cudaSuccess && P > 0) err = cudaMallocAsync(reinterpret_cast<void**>(&unsorted), P * sizeof(int2), s);
      if (err == cudaSuccess && P > 0) err = cudaMallocAsync(reinterpret_cast<void**>(&fcount), F.n * 8, s);
      if (err == cudaSuccess && P > 0) {
        LYA_COUNT(1), cross_member_kernel<1><<<grid_for(M * 32, kT), kT, 0, s>>>(
            F, Q, cf.st, cq.st, cpairs, M, cf.members, cq.members, rpar_max, rperp_max, own, nullptr, poff, unsorted);
        // group by forest: counting sort into *pairs, qoff[f] .. qoff[f+1] = forest f's quasars
        int32_t* cursor = fcount + F.n;
        err = cudaMemsetAsync(fcount, 0, F.n * 8, s);
        if (err == cudaSuccess) {
          LYA_COUNT(1), xcount_kernel<<<grid_for(P, kT), kT, 0, s>>>(unsorted, P, fcount);
          LYA_COUNT(1), scan_kernel<<<1, 1024, 0, s>>>(fcount, F.n, qoff);
          LYA_COUNT(1), xscatter_kernel<<<grid_for(P, kT), kT, 0, s>>>(unsorted, P, qoff, cursor, *pairs);
          err = cudaGetLastError();
        }
      }
    }
  }
  if (unsorted) cudaFreeAsync(unsorted, s);
  if (fcount) cudaFreeAsync(fcount, s);
  if (cpairs) cudaFreeAsync(cpairs, s);
  if (pc) cudaFreeAsync(pc, s);
  if (poff) cudaFreeAsync(poff, s);
  if (row_count) cudaFreeAsync(row_count, s);
  if (row_off) cudaFreeAsync(row_off, s);
  if (cf.buf) cudaFreeAsync(cf.buf, s);
  if (cq.buf) cudaFreeAsync(cq.buf, s);
  cudaError_t e2 = cudaStreamSynchronize(s);
  if (err == cudaSuccess) err = e2;
  *n_out = (err == cudaSuccess) ? P : 0;
  return err;
}

}  // namespace lya

namespace lya {

cudaError_t launch_exclusive_scan(const int32_t* in, int64_t n, int64_t* out, cudaStream_t s) {
  LYA_COUNT(1), scan_kernel<<<1, 1024, 0, s>>>(in, n, out);
  return cudaGetLastError();
}

}  // namespace lya
