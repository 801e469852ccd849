// C ABI of liblya.so (declared in include/lya.h): handle, scratch memory,
// argument checks and the orchestration of the kernels of prep.cu, pairs.cu,
// xi.cu, dmat.cu and adjoint.cu.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "lya_internal.cuh"

#include <atomic>
#include <memory>
#include <mutex>

namespace lya {

static std::atomic<long long> g_launches{0};
void count_launches(long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

static thread_local bool t_capturing = false;
bool capturing_thread() { return t_capturing; }

cudaError_t set_max_dynamic_smem(const void* func, int bytes) {
  // (device, function) -> largest value set; a handful of kernels, one device in practice
  struct Entry { int dev; const void* f; int bytes; };
  static Entry tab[64];
  static int n = 0;
  static std::mutex mu;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(mu);
  for (int k = 0; k < n; ++k)
    if (tab[k].dev == dev && tab[k].f == func && tab[k].bytes >= bytes) return cudaSuccess;
  if (t_capturing) return cudaErrorNotPermitted;
  e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e != cudaSuccess) return e;
  for (int k = 0; k < n; ++k)
    if (tab[k].dev == dev && tab[k].f == func) { tab[k].bytes = bytes; return cudaSuccess; }
  if (n < 64) tab[n++] = Entry{dev, func, bytes};
  return cudaSuccess;
}

cudaError_t grow(void** p, size_t* cap, size_t need) {
  if (need <= *cap && *p) return cudaSuccess;
  if (t_capturing) return cudaErrorNotPermitted;
  if (*p) {
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return e;
    cudaFree(*p);
    *p = nullptr;
    *cap = 0;
  }
  size_t n = need + need / 4 + 256;
  cudaError_t e = cudaMalloc(p, n);
  if (e != cudaSuccess) {
    *p = nullptr;
    return e;
  }
  *cap = n;
  return cudaSuccess;
}

namespace {

__global__ void min_dmin_kernel(Forests F, unsigned long long* out) {
  // distances are positive: their IEEE bit patterns order like the values
  unsigned long long m = ~0ull;
  for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < F.n;
       f += (int64_t)gridDim.x * blockDim.x)
    if (F.len[f] > 0 && F.dmin[f] > 0.0)
      m = min(m, static_cast<unsigned long long>(__double_as_longlong(F.dmin[f])));
  for (int o = 16; o > 0; o >>= 1) m = min(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMin(out, m);
}

__global__ void check_pairs_kernel(int2* p, int64_t n, int64_t nf, unsigned* err) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int2 q = p[k];
    if (q.x < 0 || q.y < 0 || q.x >= nf || q.y >= nf || q.x == q.y) {
      p[k] = make_int2(-1, -1);
      atomicOr(err, FLAG_OFFSETS);
    }
  }
}

}  // namespace
}  // namespace lya

using namespace lya;

struct CatKey {
  std::vector<const void*> ptrs;
  std::vector<int64_t> sizes;
  int32_t n_par = 0, n_perp = 0;
  double rpar = 0, rperp = 0;
  bool operator==(const CatKey& o) const {
    return ptrs == o.ptrs && sizes == o.sizes && n_par == o.n_par && n_perp == o.n_perp &&
           rpar == o.rpar && rperp == o.rperp;
  }
};

struct lya_handle {
  int device = 0;
  DevInfo dev{};
  std::string err;
  unsigned* d_err = nullptr;
  unsigned long long* d_counter = nullptr;
  int32_t* d_i32 = nullptr;
  unsigned long long* d_u64 = nullptr;
  // workspace catalogue (union of all mocks)
  void* fbuf = nullptr;
  size_t fbuf_cap = 0;
  Forests F{};
  int64_t F_capacity = 0;
  void* pixbuf = nullptr;
  size_t pix_cap = 0;
  // pair list cache
  void* pairbuf = nullptr;     // int2 pairs (grown by build_pairs)
  int64_t pair_cap = 0;
  int64_t n_pairs = 0;
  void* csbuf = nullptr;
  size_t cs_cap = 0;
  void* forder = nullptr;      // forests in HEALPix-cell order (from the pair build), -1 = none
  size_t forder_cap = 0;
  bool pairs_valid = false;
  CatKey key;
  unsigned long long* d_fp = nullptr;   // geometry fingerprint of the last prepare()
  unsigned long long fp_cached = 0;     // fingerprint the cached pair list was built for
  int max_len = 0;
  int n_mocks = 1;
  // scratch
  void* scratch = nullptr;
  size_t scratch_cap = 0;
  void* scratch2 = nullptr;
  size_t scratch2_cap = 0;
  void* outbuf = nullptr;      // num/wsum when the caller passes NULL
  size_t out_cap = 0;
  void* gbuf = nullptr;        // D accumulator
  size_t g_cap = 0;
  // quasars of the cross-correlation and the (forest, quasar) pair list
  void* qbuf = nullptr;
  size_t qbuf_cap = 0;
  Forests Q{};
  int2* xpairs = nullptr;
  int64_t xpair_cap = 0;
  int64_t n_xpairs = 0;
  void* xqoff = nullptr;       // [n_forests + 1] start of each forest's quasars in xpairs
  size_t xqoff_cap = 0;
  bool xpairs_valid = false;   // cached (forest, quasar) list: key + forest and quasar fingerprints
  CatKey xkey;
  unsigned long long x_fp = 0, x_qfp = 0;
  unsigned long long* d_qfp = nullptr;
  // rank-1 tiles of the distortion-matrix kernel (lya_set_dmat_tiles)
  int dm_tensor_tiles = 0;
  // tuning and diagnostics
  int tuned_warps = 8;
  int tuned_grab = 4;
  int tuned_for_npar = -1;
  XiLaunch last{};
  int64_t last_pairs = 0;
  // stage timing events: [stage][begin, end]
  cudaEvent_t ev[4][2] = {};
  bool ev_used[4] = {false, false, false, false};
  // graph capture (lya_capture_begin .. lya_capture_end)
  bool capturing = false;
  bool cap_failed = false;
  cudaStream_t cap_stream = nullptr;
  long long cap_launches0 = 0;
  std::shared_ptr<bool> alive = std::make_shared<bool>(true);
};

// A captured launch sequence and the handle buffers it reads and writes.
struct lya_graph {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  lya_handle* h = nullptr;
  std::shared_ptr<bool> alive;
  std::vector<const void*> bufs;
  long long kernels = 0;
};

namespace {

void stage_begin(lya_handle* h, int k, cudaStream_t s) {
  if (!h->capturing) cudaEventRecord(h->ev[k][0], s);
}
void stage_end(lya_handle* h, int k, cudaStream_t s) {
  if (h->capturing) return;
  cudaEventRecord(h->ev[k][1], s);
  h->ev_used[k] = true;
}

int fail(lya_handle* h, int code, const std::string& msg) {
  if (h) {
    h->err = msg;
    if (h->capturing) h->cap_failed = true;
  }
  return code;
}

// Entry points that synchronise, read back or may rebuild the pair list are
// refused while the handle captures a graph; the others must use the
// capturing stream.
int refuse_in_capture(lya_handle* h, const char* what) {
  if (!h->capturing) return LYA_OK;
  return fail(h, LYA_ERR_INVALID_ARG, std::string(what) + " synchronises: not allowed during graph capture");
}
int check_capture_stream(lya_handle* h, cudaStream_t s) {
  if (h->capturing && s != h->cap_stream)
    return fail(h, LYA_ERR_INVALID_ARG, "during graph capture every call must use the capturing stream");
  return LYA_OK;
}

std::vector<const void*> handle_buffers(const lya_handle* h) {
  return {h->fbuf, h->pixbuf, h->pairbuf, h->csbuf, h->scratch, h->scratch2, h->outbuf, h->gbuf, h->forder,
          reinterpret_cast<const void*>(static_cast<uintptr_t>(h->F_capacity)),
          reinterpret_cast<const void*>(static_cast<uintptr_t>(h->pix_cap)),
          reinterpret_cast<const void*>(static_cast<uintptr_t>(h->scratch_cap)),
          reinterpret_cast<const void*>(static_cast<uintptr_t>(h->scratch2_cap)),
          reinterpret_cast<const void*>(static_cast<uintptr_t>(h->out_cap)),
          reinterpret_cast<const void*>(static_cast<uintptr_t>(h->g_cap))};
}

int cuda_fail(lya_handle* h, cudaError_t e, const char* where) {
  return fail(h, LYA_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define CK(call, where)                                   \
  do {                                                    \
    cudaError_t e_ = (call);                              \
    if (e_ != cudaSuccess) return cuda_fail(h, e_, where); \
  } while (0)

int check_bins(lya_handle* h, const lya_bins* b) {
  if (!b) return fail(h, LYA_ERR_INVALID_ARG, "bins is NULL");
  if (b->n_par < 1 || b->n_par > 512 || b->n_perp < 1 || b->n_perp > 4096 ||
      static_cast<int64_t>(b->n_par) * b->n_perp > 65536)
    return fail(h, LYA_ERR_TOO_LARGE, "bin grid outside 1..512 x 1..4096 (<= 65536 bins)");
  if (!(b->r_par_max > 0) || !(b->r_perp_max > 0) || !std::isfinite(b->r_par_max) ||
      !std::isfinite(b->r_perp_max))
    return fail(h, LYA_ERR_INVALID_ARG, "r_par_max and r_perp_max must be finite and > 0");
  return LYA_OK;
}

int check_cat(lya_handle* h, const lya_catalog* c) {
  if (!c) return fail(h, LYA_ERR_INVALID_ARG, "catalogue is NULL");
  if (c->n_forests < 0 || c->n_pix < 0) return fail(h, LYA_ERR_INVALID_ARG, "negative size");
  if (c->n_forests >= (1LL << 31) - 1) return fail(h, LYA_ERR_TOO_LARGE, "more than 2^31-2 forests");
  if (!c->offsets) return fail(h, LYA_ERR_INVALID_ARG, "offsets is NULL");
  if (c->n_forests > 0 && (!c->ra || !c->dec))
    return fail(h, LYA_ERR_INVALID_ARG, "ra/dec is NULL");
  if (c->n_pix > 0 && (!c->dist || !c->loglam || !c->delta || !c->weight))
    return fail(h, LYA_ERR_INVALID_ARG, "pixel array is NULL");
  return LYA_OK;
}

int flags_to_status(lya_handle* h, unsigned f) {
  if (f == 0) return LYA_OK;
  std::string m = "input check failed:";
  int code = LYA_ERR_DEVICE_CHECK;
  if (f & FLAG_OFFSETS) { m += " inconsistent offsets or pair indices;"; code = LYA_ERR_DEVICE_CHECK; }
  if (f & FLAG_TOO_LONG) { m += " forest longer than 2^20 pixels;"; code = LYA_ERR_TOO_LARGE; }
  if (f & FLAG_RETRY) { m += " a shared-memory update exceeded its retry limit;"; code = LYA_ERR_TIMEOUT; }
  if (f & FLAG_X3_CAP) { m += " a 3PCF main vertex has more neighbours within r_max than the kernel holds;"; code = LYA_ERR_TOO_LARGE; }
  if (f & FLAG_NEGATIVE_W) { m += " negative weight;"; code = LYA_ERR_NONFINITE; }
  if (f & FLAG_NONFINITE) { m += " non-finite or non-positive value;"; code = LYA_ERR_NONFINITE; }
  if (f & FLAG_UNSORTED) { m += " distances not strictly increasing within a forest;"; code = LYA_ERR_UNSORTED; }
  return fail(h, code, m);
}

int read_flags(lya_handle* h, cudaStream_t s, unsigned* out) {
  CK(cudaMemcpyAsync(out, h->d_err, sizeof(unsigned), cudaMemcpyDeviceToHost, s), "read flags");
  CK(cudaStreamSynchronize(s), "sync");
  CK(cudaMemsetAsync(h->d_err, 0, sizeof(unsigned), s), "clear flags");
  return LYA_OK;
}

// Forest and pixel workspace for n forests / p pixels.  Reallocates (losing
// the cached pair list) only when capacity is short.
int ensure_workspace(lya_handle* h, int64_t nf, int64_t np) {
  if (h->capturing && (nf > h->F_capacity || !h->fbuf))
    return fail(h, LYA_ERR_INVALID_ARG, "graph capture: forest workspace too small (run the call once before capturing)");
  if (nf > h->F_capacity || !h->fbuf) {
    const int64_t cap = std::max<int64_t>(nf, 1) + std::max<int64_t>(nf, 1) / 4;
    const size_t bytes = static_cast<size_t>(cap) * (8 * 9 + 4 * 7) + 16 * 256;
    if (h->fbuf) { cudaDeviceSynchronize(); cudaFree(h->fbuf); h->fbuf = nullptr; }
    cudaError_t e = cudaMalloc(&h->fbuf, bytes);
    if (e != cudaSuccess) { h->F_capacity = 0; return fail(h, LYA_ERR_NO_MEMORY, "forest workspace"); }
    h->fbuf_cap = bytes;
    char* p = static_cast<char*>(h->fbuf);
    auto take = [&](size_t b) { char* q = p; p += (b + 255) & ~size_t(255); return q; };
    h->F.off = reinterpret_cast<int64_t*>(take(cap * 8));
    h->F.ux = reinterpret_cast<double*>(take(cap * 8));
    h->F.uy = reinterpret_cast<double*>(take(cap * 8));
    h->F.uz = reinterpret_cast<double*>(take(cap * 8));
    h->F.dmin = reinterpret_cast<double*>(take(cap * 8));
    h->F.dmax = reinterpret_cast<double*>(take(cap * 8));
    h->F.wsum = reinterpret_cast<double*>(take(cap * 8));
    h->F.lbar = reinterpret_cast<double*>(take(cap * 8));
    h->F.ssum = reinterpret_cast<double*>(take(cap * 8));
    h->F.len = reinterpret_cast<int32_t*>(take(cap * 4));
    h->F.dref = reinterpret_cast<float*>(take(cap * 4));
    h->F.mock = reinterpret_cast<int32_t*>(take(cap * 4));
    h->F.wmax = reinterpret_cast<float*>(take(cap * 4));
    h->F.wdmax = reinterpret_cast<float*>(take(cap * 4));
    h->F.hmin = reinterpret_cast<float*>(take(cap * 4));
    h->F.xmax = reinterpret_cast<float*>(take(cap * 4));
    h->F_capacity = cap;
    h->pairs_valid = false;
  }
  h->F.n = nf;
  cudaError_t e = grow(&h->pixbuf, &h->pix_cap, static_cast<size_t>(std::max<int64_t>(np, 1)) * 16);
  if (e != cudaSuccess) return fail(h, LYA_ERR_NO_MEMORY, "pixel workspace");
  return LYA_OK;
}

CatKey make_key(const lya_catalog* cats, int n, const lya_bins* b) {
  CatKey k;
  for (int m = 0; m < n; ++m) {
    k.ptrs.push_back(cats[m].ra);
    k.ptrs.push_back(cats[m].dec);
    k.ptrs.push_back(cats[m].dist);
    k.ptrs.push_back(cats[m].offsets);
    k.sizes.push_back(cats[m].n_forests);
    k.sizes.push_back(cats[m].n_pix);
  }
  k.n_par = b->n_par;
  k.n_perp = b->n_perp;
  k.rpar = b->r_par_max;
  k.rperp = b->r_perp_max;
  return k;
}

// Prepare all catalogues (input checks, moments, packed pixels).  Async.
int prepare(lya_handle* h, const lya_catalog* cats, int n, cudaStream_t s) {
  int64_t nf = 0, np = 0;
  for (int m = 0; m < n; ++m) {
    int st = check_cat(h, &cats[m]);
    if (st) return st;
    nf += cats[m].n_forests;
    np += cats[m].n_pix;
  }
  if (nf >= (1LL << 31) - 1) return fail(h, LYA_ERR_TOO_LARGE, "more than 2^31-2 forests");
  int st = ensure_workspace(h, nf, np);
  if (st) return st;
  int64_t fb = 0, pb = 0;
  CK(cudaMemsetAsync(h->d_fp, 0, sizeof(unsigned long long), s), "clear fingerprint");
  for (int m = 0; m < n; ++m) {
    CK(launch_prep(cats[m], fb, pb, m, h->F, static_cast<Pix*>(h->pixbuf), h->d_err, h->d_fp, s), "prep");
    fb += cats[m].n_forests;
    pb += cats[m].n_pix;
  }
  return LYA_OK;
}

int build_all_pairs(lya_handle* h, const lya_catalog* cats, int n, const lya_bins* b, cudaStream_t s) {
  h->pairs_valid = false;
  stage_begin(h, 3, s);
  // catalogue-wide angle bound from the smallest distance
  CK(cudaMemsetAsync(h->d_u64, 0xff, 8, s), "memset");
  if (h->F.n > 0) {
    int64_t blocks = std::min<int64_t>((h->F.n + 255) / 256, 4096);
    LYA_COUNT(1), min_dmin_kernel<<<static_cast<int>(blocks), 256, 0, s>>>(h->F, h->d_u64);
    CK(cudaGetLastError(), "min_dmin");
  }
  unsigned long long bits = 0;
  CK(cudaMemcpyAsync(&bits, h->d_u64, 8, cudaMemcpyDeviceToHost, s), "read dmin");
  CK(launch_max_len(h->F, h->d_i32, s), "max_len");
  int32_t ml = 0;
  CK(cudaMemcpyAsync(&ml, h->d_i32, 4, cudaMemcpyDeviceToHost, s), "read max_len");
  unsigned flags = 0;
  int st = read_flags(h, s, &flags);
  if (st) return st;
  st = flags_to_status(h, flags);
  if (st) return st;
  h->max_len = ml;
  double dmin = 1.0;
  if (bits != ~0ull) std::memcpy(&dmin, &bits, 8);
  const double th = 2.0 * std::asin(std::min(1.0, b->r_perp_max / (2.0 * dmin)));
  const double th_deg = th * 180.0 / M_PI;
  int nside = 1;
  while (nside < 256 && 117.0 / th_deg >= 2.0 * nside) nside *= 2;
  PairBuild pbld{nside, b->r_perp_max, th};
  int64_t total = 0, fb = 0;
  int2* pairs = static_cast<int2*>(h->pairbuf);
  {
    cudaError_t e = grow(&h->forder, &h->forder_cap, static_cast<size_t>(std::max<int64_t>(h->F.n, 1)) * 4);
    if (e != cudaSuccess) return fail(h, LYA_ERR_NO_MEMORY, "forest order");
  }
  for (int m = 0; m < n; ++m) {
    int64_t got = 0;
    CK(build_pairs(h->F, fb, fb + cats[m].n_forests, pbld, &pairs, &h->pair_cap, total, &got,
                   &h->scratch, &h->scratch_cap, static_cast<int32_t*>(h->forder), s),
       "pair list");
    total += got;
    fb += cats[m].n_forests;
  }
  h->pairbuf = pairs;
  h->n_pairs = total;
  cudaError_t e = grow(&h->csbuf, &h->cs_cap, static_cast<size_t>(std::max<int64_t>(total, 1)) * 8);
  if (e != cudaSuccess) return fail(h, LYA_ERR_NO_MEMORY, "pair geometry");
  CK(launch_pair_geometry(pairs, total, h->F, b->n_par / b->r_par_max, b->n_perp / b->r_perp_max,
                          static_cast<float2*>(h->csbuf), s),
     "pair geometry");
  CK(sort_pairs_by_band(pairs, static_cast<float2*>(h->csbuf), total, h->F, static_cast<const Pix*>(h->pixbuf),
                        b->n_perp, n, &h->scratch, &h->scratch_cap, s),
     "pair order");
  stage_end(h, 3, s);
  unsigned long long fp = 0;
  CK(cudaMemcpyAsync(&fp, h->d_fp, 8, cudaMemcpyDeviceToHost, s), "read fingerprint");
  CK(cudaStreamSynchronize(s), "sync");
  h->fp_cached = fp;
  h->key = make_key(cats, n, b);
  h->n_mocks = n;
  h->pairs_valid = true;
  return LYA_OK;
}

// Reuse the cached pair list only if the pointers, sizes and bins match AND
// the geometry fingerprint of this call's prepare() equals the one the list
// was built for (freed device memory is often handed out again at the same
// address, so pointers alone do not identify a catalogue).  The fingerprint
// read synchronises the stream.
int ensure_pairs(lya_handle* h, const lya_catalog* cats, int n, const lya_bins* b, cudaStream_t s) {
  if (h->capturing) {
    // the geometry must not change between replays; the list cannot be rebuilt inside a graph
    if (h->pairs_valid && h->key == make_key(cats, n, b)) return LYA_OK;
    return fail(h, LYA_ERR_INVALID_ARG, "graph capture needs the pair list of these inputs cached (run the call once first)");
  }
  if (h->pairs_valid && h->key == make_key(cats, n, b)) {
    unsigned long long fp = 0;
    CK(cudaMemcpyAsync(&fp, h->d_fp, 8, cudaMemcpyDeviceToHost, s), "read fingerprint");
    CK(cudaStreamSynchronize(s), "sync");
    if (fp == h->fp_cached) return LYA_OK;
  }
  return build_all_pairs(h, cats, n, b, s);
}

int run_xi(lya_handle* h, const lya_catalog* cats, int ncat, const lya_bins* b, lya_precision prec,
           const int2* pairs, const float2* cs, int64_t npairs, double* num, double* wsum, double* xi,
           cudaStream_t s) {
  const int nb = b->n_par * b->n_perp;
  const int64_t nout = static_cast<int64_t>(nb) * ncat;
  double* N = num;
  double* W = wsum;
  if (!N || !W) {
    cudaError_t e = grow(&h->outbuf, &h->out_cap, static_cast<size_t>(nout) * 16);
    if (e != cudaSuccess) return fail(h, LYA_ERR_NO_MEMORY, "output scratch");
    if (!N) N = static_cast<double*>(h->outbuf);
    if (!W) W = static_cast<double*>(h->outbuf) + nout;
  }
  CK(cudaMemsetAsync(N, 0, nout * 8, s), "zero num");
  CK(cudaMemsetAsync(W, 0, nout * 8, s), "zero wsum");
  XiArgs A;
  A.pairs = pairs;
  A.cs = cs;
  A.n_pairs = npairs;
  A.pix = static_cast<const Pix*>(h->pixbuf);
  A.F = h->F;
  A.n_par = b->n_par;
  A.n_perp = b->n_perp;
  A.num = N;
  A.wsum = W;
  A.nb = nb;
  A.counter = h->d_counter;
  if (prec == LYA_PREC_MIXED && b->n_par > xi_mixed_max_npar())
    return fail(h, LYA_ERR_TOO_LARGE, "the mixed path supports n_par <= " + std::to_string(xi_mixed_max_npar()));
  if (prec == LYA_PREC_FP64 && b->n_par > 256)
    return fail(h, LYA_ERR_TOO_LARGE, "the FP64 path supports n_par <= 256");
  if (prec == LYA_PREC_MIXED) {
    XiLaunch L;
    const int warps = (h->tuned_for_npar == b->n_par) ? h->tuned_warps : 8;
    const int grab = (h->tuned_for_npar == b->n_par) ? h->tuned_grab : 4;
    CK(plan_xi_mixed(h->dev, b->n_par, h->max_len, warps, grab, &L), "plan xi");
    stage_begin(h, 0, s);
    CK(launch_xi_mixed(A, L, s), "xi kernel");
    stage_end(h, 0, s);
    h->last = L;
  } else if (prec == LYA_PREC_FP64) {
    if (h->capturing) return fail(h, LYA_ERR_INVALID_ARG, "the FP64 path allocates: not allowed during graph capture");
    XiLaunch L{};
    stage_begin(h, 0, s);
    CK(launch_xi_fp64(A, cats, ncat, h->dev, h->max_len, b->r_par_max, b->r_perp_max, &L, s),
       "xi fp64 kernel");
    stage_end(h, 0, s);
    h->last = L;
  } else {
    return fail(h, LYA_ERR_INVALID_ARG, "unknown precision");
  }
  h->last_pairs = npairs;
  if (xi) CK(launch_finalize(N, W, xi, nout, s), "finalize");
  return LYA_OK;
}

}  // namespace

extern "C" {

int lya_create(lya_handle** out) {
  if (!out) return LYA_ERR_INVALID_ARG;
  *out = nullptr;
  lya_handle* h = new lya_handle();
  cudaError_t e = cudaGetDevice(&h->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&h->dev.sms, cudaDevAttrMultiProcessorCount, h->device);
  if (e == cudaSuccess)
    e = cudaDeviceGetAttribute(&h->dev.smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device);
  if (e == cudaSuccess)
    e = cudaDeviceGetAttribute(&h->dev.smem_per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, h->device);
  void* small = nullptr;
  if (e == cudaSuccess) e = cudaMalloc(&small, 512);
  if (e == cudaSuccess) e = cudaMemset(small, 0, 512);
  if (e != cudaSuccess) {
    if (small) cudaFree(small);
    delete h;
    return LYA_ERR_CUDA;
  }
  for (int k = 0; k < 4 && e == cudaSuccess; ++k)
    for (int q = 0; q < 2 && e == cudaSuccess; ++q) e = cudaEventCreate(&h->ev[k][q]);
  if (e != cudaSuccess) {
    cudaFree(small);
    delete h;
    return LYA_ERR_CUDA;
  }
  char* p = static_cast<char*>(small);
  h->d_err = reinterpret_cast<unsigned*>(p);
  h->d_counter = reinterpret_cast<unsigned long long*>(p + 64);
  h->d_i32 = reinterpret_cast<int32_t*>(p + 128);
  h->d_u64 = reinterpret_cast<unsigned long long*>(p + 192);
  h->d_fp = reinterpret_cast<unsigned long long*>(p + 256);
  h->d_qfp = reinterpret_cast<unsigned long long*>(p + 320);
  *out = h;
  return LYA_OK;
}

int lya_destroy(lya_handle* h) {
  if (!h) return LYA_ERR_INVALID_ARG;
  if (h->capturing) {
    cudaGraph_t g = nullptr;
    cudaStreamEndCapture(h->cap_stream, &g);
    if (g) cudaGraphDestroy(g);
    t_capturing = false;
  }
  *h->alive = false;   // graphs captured on this handle refuse to launch from now on
  cudaDeviceSynchronize();
  void* bufs[] = {h->fbuf, h->pixbuf, h->pairbuf, h->csbuf, h->scratch, h->scratch2, h->outbuf, h->gbuf,
                  h->forder, h->d_err, h->qbuf, h->xpairs, h->xqoff};
  for (void* b : bufs)
    if (b) cudaFree(b);
  for (int k = 0; k < 4; ++k)
    for (int q = 0; q < 2; ++q)
      if (h->ev[k][q]) cudaEventDestroy(h->ev[k][q]);
  delete h;
  return LYA_OK;
}

int lya_last_error(const lya_handle* h, char* buf, size_t n) {
  if (!h || !buf || n == 0) return LYA_ERR_INVALID_ARG;
  std::snprintf(buf, n, "%s", h->err.c_str());
  return LYA_OK;
}

const char* lya_status_string(int s) {
  switch (s) {
    case LYA_OK: return "LYA_OK";
    case LYA_ERR_INVALID_ARG: return "LYA_ERR_INVALID_ARG";
    case LYA_ERR_UNSORTED: return "LYA_ERR_UNSORTED";
    case LYA_ERR_NONFINITE: return "LYA_ERR_NONFINITE";
    case LYA_ERR_NO_MEMORY: return "LYA_ERR_NO_MEMORY";
    case LYA_ERR_CUDA: return "LYA_ERR_CUDA";
    case LYA_ERR_TIMEOUT: return "LYA_ERR_TIMEOUT";
    case LYA_ERR_DEVICE_CHECK: return "LYA_ERR_DEVICE_CHECK";
    case LYA_ERR_TOO_LARGE: return "LYA_ERR_TOO_LARGE";
    default: return "LYA_ERR_UNKNOWN";
  }
}

int lya_sync_status(lya_handle* h, void* stream) {
  if (!h) return LYA_ERR_INVALID_ARG;
  if (int st = refuse_in_capture(h, "lya_sync_status")) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  unsigned flags = 0;
  int st = read_flags(h, s, &flags);
  if (st) return st;
  return flags_to_status(h, flags);
}

int lya_pairs_build(lya_handle* h, const lya_catalog* cat, const lya_bins* bins, int64_t* n_pairs,
                    void* stream) {
  if (!h) return LYA_ERR_INVALID_ARG;
  if (int st0 = refuse_in_capture(h, "lya_pairs_build")) return st0;
  int st = check_bins(h, bins);
  if (st) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  st = prepare(h, cat, 1, s);
  if (st) return st;
  st = build_all_pairs(h, cat, 1, bins, s);
  if (st) return st;
  if (n_pairs) *n_pairs = h->n_pairs;
  return LYA_OK;
}

int lya_pairs_get(lya_handle* h, int32_t* pair_a, int32_t* pair_b, int64_t cap, int64_t* n_pairs,
                  void* stream) {
  if (!h) return LYA_ERR_INVALID_ARG;
  if (int st = refuse_in_capture(h, "lya_pairs_get")) return st;
  if (!h->pairs_valid) return fail(h, LYA_ERR_INVALID_ARG, "no pair list cached");
  if (n_pairs) *n_pairs = h->n_pairs;
  if (cap < h->n_pairs) return fail(h, LYA_ERR_INVALID_ARG, "capacity too small");
  if (h->n_pairs > 0 && (!pair_a || !pair_b)) return fail(h, LYA_ERR_INVALID_ARG, "NULL output");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  CK(launch_unpack_pairs(static_cast<const int2*>(h->pairbuf), h->n_pairs, pair_a, pair_b, s), "unpack");
  CK(cudaStreamSynchronize(s), "sync");
  return LYA_OK;
}

int lya_project(lya_handle* h, const lya_catalog* cat, float* delta_out, void* stream) {
  if (!h) return LYA_ERR_INVALID_ARG;
  if (!delta_out && cat && cat->n_pix > 0) return fail(h, LYA_ERR_INVALID_ARG, "delta_out is NULL");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (int st0 = check_capture_stream(h, s)) return st0;
  int st = prepare(h, cat, 1, s);
  if (st) return st;
  CK(launch_project(*cat, h->F, 0, delta_out, s), "project");
  return LYA_OK;
}

int lya_xi(lya_handle* h, const lya_catalog* cat, const lya_bins* bins, lya_precision prec, double* num,
           double* wsum, double* xi, void* stream) {
  if (!h) return LYA_ERR_INVALID_ARG;
  int st = check_bins(h, bins);
  if (st) return st;
  if (!num && !wsum && !xi) return fail(h, LYA_ERR_INVALID_ARG, "no output requested");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if ((st = check_capture_stream(h, s))) return st;
  st = prepare(h, cat, 1, s);
  if (st) return st;
  st = ensure_pairs(h, cat, 1, bins, s);
  if (st) return st;
  return run_xi(h, cat, 1, bins, prec, static_cast<const int2*>(h->pairbuf),
                static_cast<const float2*>(h->csbuf), h->n_pairs, num, wsum, xi, s);
}

int lya_xi_pairs(lya_handle* h, const lya_catalog* cat, const lya_bins* bins, lya_precision prec,
                 const int32_t* pair_a, const int32_t* pair_b, int64_t n_pairs, double* num, double* wsum,
                 double* xi, void* stream) {
  if (!h) return LYA_ERR_INVALID_ARG;
  if (int st0 = refuse_in_capture(h, "lya_xi_pairs")) return st0;
  int st = check_bins(h, bins);
  if (st) return st;
  if (n_pairs < 0 || (n_pairs > 0 && (!pair_a || !pair_b)))
    return fail(h, LYA_ERR_INVALID_ARG, "bad pair arrays");
  if (!num && !wsum && !xi) return fail(h, LYA_ERR_INVALID_ARG, "no output requested");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  st = prepare(h, cat, 1, s);
  if (st) return st;
  // the explicit list is used as given; the cached list (if any) is left alone
  CK(launch_max_len(h->F, h->d_i32, s), "max_len");
  int32_t ml = 0;
  CK(cudaMemcpyAsync(&ml, h->d_i32, 4, cudaMemcpyDeviceToHost, s), "read max_len");
  CK(cudaStreamSynchronize(s), "sync");
  const int saved = h->max_len;
  h->max_len = ml;
  cudaError_t e = grow(&h->scratch2, &h->scratch2_cap, static_cast<size_t>(std::max<int64_t>(n_pairs, 1)) * 16);
  if (e != cudaSuccess) return fail(h, LYA_ERR_NO_MEMORY, "pair scratch");
  int2* pp = static_cast<int2*>(h->scratch2);
  float2* cs = reinterpret_cast<float2*>(pp + std::max<int64_t>(n_pairs, 1));
  CK(launch_pack_pairs(pair_a, pair_b, n_pairs, pp, s), "pack pairs");
  if (n_pairs > 0) {
    int64_t blocks = std::min<int64_t>((n_pairs + 255) / 256, 65535);
    LYA_COUNT(1), check_pairs_kernel<<<static_cast<int>(blocks), 256, 0, s>>>(pp, n_pairs, cat->n_forests, h->d_err);
    CK(cudaGetLastError(), "check pairs");
  }
  // invalid pairs were replaced by (-1,-1); the geometry and xi kernels skip them
  CK(launch_pair_geometry(pp, n_pairs, h->F, bins->n_par / bins->r_par_max,
                                  bins->n_perp / bins->r_perp_max, cs, s),
     "pair geometry");
  st = run_xi(h, cat, 1, bins, prec, pp, cs, n_pairs, num, wsum, xi, s);
  h->max_len = std::max(saved, ml);
  return st;
}

}  // extern "C"

namespace {

int run_dmat_cats(lya_handle* h, const lya_catalog* cats, int n, const lya_bins* bins, lya_eta eta,
                  double p_subsample, uint64_t seed, double* dmat, double* wsum_dm, cudaStream_t s) {
  int st = check_bins(h, bins);
  if (st) return st;
  if (!dmat) return fail(h, LYA_ERR_INVALID_ARG, "dmat is NULL");
  if (!(p_subsample >= 0.0) || !std::isfinite(p_subsample))
    return fail(h, LYA_ERR_INVALID_ARG, "p_subsample must be finite and >= 0");
  if (eta != LYA_ETA_IDENTITY && eta != LYA_ETA_MEAN_SLOPE) return fail(h, LYA_ERR_INVALID_ARG, "eta");
  if ((st = check_capture_stream(h, s))) return st;
  st = prepare(h, cats, n, s);
  if (st) return st;
  st = ensure_pairs(h, cats, n, bins, s);
  if (st) return st;
  const int nb = bins->n_par * bins->n_perp;
  const size_t gbytes = (static_cast<size_t>(nb) * nb * 8 + static_cast<size_t>(nb) * 8) * n;
  cudaError_t e = grow(&h->gbuf, &h->g_cap, gbytes);
  if (e != cudaSuccess) return fail(h, LYA_ERR_NO_MEMORY, "D accumulator");
  double* G = static_cast<double*>(h->gbuf);
  double* wdm = G + static_cast<size_t>(nb) * nb * n;
  DmArgs A;
  A.pairs = static_cast<const int2*>(h->pairbuf);
  A.cs = static_cast<const float2*>(h->csbuf);
  A.n_pairs = h->n_pairs;
  A.pix = static_cast<const Pix*>(h->pixbuf);
  A.F = h->F;
  A.n_par = bins->n_par;
  A.n_perp = bins->n_perp;
  A.eta_mean_slope = eta == LYA_ETA_MEAN_SLOPE ? 1 : 0;
  A.p_subsample = p_subsample;
  A.seed = seed;
  A.G = G;
  A.wdm = wdm;
  A.max_len = h->max_len;
  A.n_mocks = n;
  A.tensor_tiles = h->dm_tensor_tiles;
  A.fbase = nullptr;
  stage_begin(h, 1, s);
  CK(run_dmat(A, h->dev, &h->scratch2, &h->scratch2_cap, s), "dmat");
  stage_end(h, 1, s);
  CK(launch_dm_finalize(G, wdm, dmat, wsum_dm, nb, n, s), "dmat finalize");
  return LYA_OK;
}

}  // namespace

extern "C" {

int lya_dmat(lya_handle* h, const lya_catalog* cat, const lya_bins* bins, lya_eta eta, double p_subsample,
             uint64_t seed, double* dmat, double* wsum_dm, void* stream) {
  if (!h) return LYA_ERR_INVALID_ARG;
  return run_dmat_cats(h, cat, 1, bins, eta, p_subsample, seed, dmat, wsum_dm, static_cast<cudaStream_t>(stream));
}

int lya_dmat_batched(lya_handle* h, const lya_catalog* mocks, int32_t n_mocks, const lya_bins* bins, lya_eta eta,
                     double p_subsample, uint64_t seed, double* dmat, double* wsum_dm, void* stream) {
  if (!h) return LYA_ERR_INVALID_ARG;
  if (!mocks || n_mocks < 1) return fail(h, LYA_ERR_INVALID_ARG, "no mocks");
  return run_dmat_cats(h, mocks, n_mocks, bins, eta, p_subsample, seed, dmat, wsum_dm,
                       static_cast<cudaStream_t>(stream));
}

int lya_xi_backward(lya_handle* h, const lya_catalog* cat, const lya_bins* bins, const double* grad_xi,
                    const double* xi, const double* wsum, float* grad_delta, float* grad_weight,
                    void* stream) {
  return lya_xi_backward_full(h, cat, bins, grad_xi, nullptr, xi, wsum, grad_delta, grad_weight, stream);
}

int lya_xi_backward_full(lya_handle* h, const lya_catalog* cat, const lya_bins* bins, const double* grad_xi,
                         const double* grad_wsum, const double* xi, const double* wsum, float* grad_delta,
                         float* grad_weight, void* stream) {
  if (!h) return LYA_ERR_INVALID_ARG;
  int st = check_bins(h, bins);
  if (st) return st;
  if (!grad_xi || !xi || !wsum) return fail(h, LYA_ERR_INVALID_ARG, "grad_xi/xi/wsum is NULL");
  if (cat && cat->n_pix > 0 && (!grad_delta || !grad_weight))
    return fail(h, LYA_ERR_INVALID_ARG, "gradient output is NULL");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if ((st = check_capture_stream(h, s))) return st;
  st = prepare(h, cat, 1, s);
  if (st) return st;
  st = ensure_pairs(h, cat, 1, bins, s);
  if (st) return st;
  AdjArgs A;
  A.pairs = static_cast<const int2*>(h->pairbuf);
  A.cs = static_cast<const float2*>(h->csbuf);
  A.n_pairs = h->n_pairs;
  A.pix = static_cast<const Pix*>(h->pixbuf);
  A.F = h->F;
  A.n_par = bins->n_par;
  A.n_perp = bins->n_perp;
  A.grad_xi = grad_xi;
  A.grad_wsum = grad_wsum;
  A.xi = xi;
  A.wsum = wsum;
  A.delta = cat->delta;
  A.weight = cat->weight;
  A.pix_base = 0;
  A.n_pix = cat->n_pix;
  A.grad_delta = grad_delta;
  A.grad_weight = grad_weight;
  A.max_len = h->max_len;
  A.forder = static_cast<const int32_t*>(h->forder);
  if (cat->n_pix > 0) {
    CK(cudaMemsetAsync(grad_delta, 0, cat->n_pix * 4, s), "zero grad");
    CK(cudaMemsetAsync(grad_weight, 0, cat->n_pix * 4, s), "zero grad");
  }
  stage_begin(h, 2, s);
  CK(run_adjoint(A, h->dev, &h->scratch2, &h->scratch2_cap, s), "adjoint");
  stage_end(h, 2, s);
  return LYA_OK;
}

int lya_xi_batched(lya_handle* h, const lya_catalog* mocks, int32_t n_mocks, const lya_bins* bins,
                   lya_precision prec, double* num, double* wsum, double* xi, void* stream) {
  if (!h) return LYA_ERR_INVALID_ARG;
  if (!mocks || n_mocks < 1) return fail(h, LYA_ERR_INVALID_ARG, "no mocks");
  int st = check_bins(h, bins);
  if (st) return st;
  if (!num && !wsum && !xi) return fail(h, LYA_ERR_INVALID_ARG, "no output requested");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if ((st = check_capture_stream(h, s))) return st;
  st = prepare(h, mocks, n_mocks, s);
  if (st) return st;
  st = ensure_pairs(h, mocks, n_mocks, bins, s);
  if (st) return st;
  return run_xi(h, mocks, n_mocks, bins, prec, static_cast<const int2*>(h->pairbuf),
                static_cast<const float2*>(h->csbuf), h->n_pairs, num, wsum, xi, s);
}

int lya_autotune(lya_handle* h, const lya_catalog* cat, const lya_bins* bins, int32_t* choice,
                 void* stream) {
  if (!h) return LYA_ERR_INVALID_ARG;
  if (int st0 = refuse_in_capture(h, "lya_autotune")) return st0;
  int st = check_bins(h, bins);
  if (st) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  st = prepare(h, cat, 1, s);
  if (st) return st;
  st = ensure_pairs(h, cat, 1, bins, s);
  if (st) return st;
  // candidate (warps per block, pairs per work grab)
  static const int cand[][2] = {{8, 1}, {8, 4}, {8, 16}, {4, 4}, {16, 4}, {12, 4}, {13, 4}, {14, 4}, {13, 2}};
  const int nc = sizeof(cand) / sizeof(cand[0]);
  const int nb = bins->n_par * bins->n_perp;
  cudaError_t e = grow(&h->outbuf, &h->out_cap, static_cast<size_t>(nb) * 16);
  if (e != cudaSuccess) return fail(h, LYA_ERR_NO_MEMORY, "output scratch");
  double* N = static_cast<double*>(h->outbuf);
  double* W = N + nb;
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0), "event");
  CK(cudaEventCreate(&e1), "event");
  float best = 1e30f;
  int besti = 1;
  for (int c = 0; c < nc; ++c) {
    XiLaunch L;
    if (plan_xi_mixed(h->dev, bins->n_par, h->max_len, cand[c][0], cand[c][1], &L) != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    XiArgs A;
    A.pairs = static_cast<const int2*>(h->pairbuf);
    A.cs = static_cast<const float2*>(h->csbuf);
    A.n_pairs = h->n_pairs;
    A.pix = static_cast<const Pix*>(h->pixbuf);
    A.F = h->F;
    A.n_par = bins->n_par;
    A.n_perp = bins->n_perp;
    A.num = N;
    A.wsum = W;
    A.nb = nb;
    A.counter = h->d_counter;
    float tbest = 1e30f;
    for (int rep = 0; rep < 3; ++rep) {
      CK(cudaMemsetAsync(N, 0, nb * 16, s), "zero");
      CK(cudaEventRecord(e0, s), "event");
      CK(launch_xi_mixed(A, L, s), "xi kernel");
      CK(cudaEventRecord(e1, s), "event");
      CK(cudaEventSynchronize(e1), "event sync");
      float ms = 0;
      cudaEventElapsedTime(&ms, e0, e1);
      if (rep > 0) tbest = std::min(tbest, ms);
    }
    if (tbest < best) {
      best = tbest;
      besti = c;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  h->tuned_warps = cand[besti][0];
  h->tuned_grab = cand[besti][1];
  h->tuned_for_npar = bins->n_par;
  if (choice) *choice = besti;
  return LYA_OK;
}

int lya_pair_stats(lya_handle* h, const lya_catalog* cat, const lya_bins* bins, double p_subsample,
                   uint64_t seed, int64_t* n_pairs, int64_t* pixel_pairs, double* pixel_pairs_sq,
                   void* stream) {
  if (!h) return LYA_ERR_INVALID_ARG;
  if (int st0 = refuse_in_capture(h, "lya_pair_stats")) return st0;
  int st = check_bins(h, bins);
  if (st) return st;
  if (!(p_subsample >= 0.0) || !std::isfinite(p_subsample))
    return fail(h, LYA_ERR_INVALID_ARG, "p_subsample must be finite and >= 0");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  st = prepare(h, cat, 1, s);
  if (st) return st;
  st = ensure_pairs(h, cat, 1, bins, s);
  if (st) return st;
  XiArgs A{};
  A.pairs = static_cast<const int2*>(h->pairbuf);
  A.cs = static_cast<const float2*>(h->csbuf);
  A.n_pairs = h->n_pairs;
  A.pix = static_cast<const Pix*>(h->pixbuf);
  A.F = h->F;
  A.n_par = bins->n_par;
  A.n_perp = bins->n_perp;
  StatsOut* dout = reinterpret_cast<StatsOut*>(h->d_u64 + 1);
  CK(launch_pair_stats(A, p_subsample, seed, dout, h->dev, s), "pair stats");
  StatsOut host{};
  CK(cudaMemcpyAsync(&host, dout, sizeof(StatsOut), cudaMemcpyDeviceToHost, s), "read stats");
  CK(cudaStreamSynchronize(s), "sync");
  if (n_pairs) *n_pairs = static_cast<int64_t>(host.pairs);
  if (pixel_pairs) *pixel_pairs = static_cast<int64_t>(host.pix);
  if (pixel_pairs_sq) *pixel_pairs_sq = static_cast<double>(host.pix_sq);
  return LYA_OK;
}

int lya_set_dmat_tiles(lya_handle* h, int32_t mode) {
  if (!h) return LYA_ERR_INVALID_ARG;
  if (mode != 0 && mode != 1) return fail(h, LYA_ERR_INVALID_ARG, "tile mode must be 0 (FP32) or 1 (TF32x3)");
  h->dm_tensor_tiles = mode;
  return LYA_OK;
}

int lya_dmat_work(lya_handle* h, const lya_catalog* cat, const lya_bins* bins, double p_subsample, uint64_t seed,
                  int64_t* n_pairs, int64_t* pixel_pairs, double* sum_vec_support_sq, double* sum_pair_support_sq,
                  void* stream) {
  if (!h) return LYA_ERR_INVALID_ARG;
  if (int st0 = refuse_in_capture(h, "lya_dmat_work")) return st0;
  int st = check_bins(h, bins);
  if (st) return st;
  if (!(p_subsample >= 0.0) || !std::isfinite(p_subsample))
    return fail(h, LYA_ERR_INVALID_ARG, "p_subsample must be finite and >= 0");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  st = prepare(h, cat, 1, s);
  if (st) return st;
  st = ensure_pairs(h, cat, 1, bins, s);
  if (st) return st;
  DmArgs A{};
  A.pairs = static_cast<const int2*>(h->pairbuf);
  A.cs = static_cast<const float2*>(h->csbuf);
  A.n_pairs = h->n_pairs;
  A.pix = static_cast<const Pix*>(h->pixbuf);
  A.F = h->F;
  A.n_par = bins->n_par;
  A.n_perp = bins->n_perp;
  A.p_subsample = p_subsample;
  A.seed = seed;
  A.max_len = h->max_len;
  A.n_mocks = 1;
  // the small device block's last 128 bytes (after d_qfp at +320) hold the counts
  DmWork* dout = reinterpret_cast<DmWork*>(reinterpret_cast<char*>(h->d_err) + 384);
  CK(launch_dm_work(A, h->dev, dout, s), "distortion-matrix work count");
  DmWork host{};
  CK(cudaMemcpyAsync(&host, dout, sizeof(DmWork), cudaMemcpyDeviceToHost, s), "read work count");
  CK(cudaStreamSynchronize(s), "sync");
  if (n_pairs) *n_pairs = static_cast<int64_t>(host.pairs);
  if (pixel_pairs) *pixel_pairs = static_cast<int64_t>(host.pix);
  if (sum_vec_support_sq) *sum_vec_support_sq = host.sv2;
  if (sum_pair_support_sq) *sum_pair_support_sq = host.sp2;
  return LYA_OK;
}

int lya_flip_tally(lya_handle* h, const lya_catalog* cat, const lya_bins* bins, double p_subsample, uint64_t seed,
                   int64_t* pixel_pairs, int64_t* flipped, double* weight, double* flipped_weight, void* stream) {
  if (!h) return LYA_ERR_INVALID_ARG;
  if (int st0 = refuse_in_capture(h, "lya_flip_tally")) return st0;
  int st = check_bins(h, bins);
  if (st) return st;
  if (!(p_subsample >= 0.0) || !std::isfinite(p_subsample))
    return fail(h, LYA_ERR_INVALID_ARG, "p_subsample must be finite and >= 0");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  st = prepare(h, cat, 1, s);
  if (st) return st;
  st = ensure_pairs(h, cat, 1, bins, s);
  if (st) return st;
  XiArgs A{};
  A.pairs = static_cast<const int2*>(h->pairbuf);
  A.cs = static_cast<const float2*>(h->csbuf);
  A.n_pairs = h->n_pairs;
  A.pix = static_cast<const Pix*>(h->pixbuf);
  A.F = h->F;
  A.n_par = bins->n_par;
  A.n_perp = bins->n_perp;
  FlipOut* dout = reinterpret_cast<FlipOut*>(h->d_u64 + 1);
  CK(launch_flip_tally(A, cat->dist, bins->n_par / bins->r_par_max, bins->n_perp / bins->r_perp_max, p_subsample,
                       seed, dout, h->dev, s),
     "flip tally");
  FlipOut host{};
  CK(cudaMemcpyAsync(&host, dout, sizeof(FlipOut), cudaMemcpyDeviceToHost, s), "read tally");
  CK(cudaStreamSynchronize(s), "sync");
  if (pixel_pairs) *pixel_pairs = static_cast<int64_t>(host.pix);
  if (flipped) *flipped = static_cast<int64_t>(host.flips);
  if (weight) *weight = host.w;
  if (flipped_weight) *flipped_weight = host.wflip;
  return LYA_OK;
}

int lya_xi_subsamples(lya_handle* h, const lya_catalog* cat, const lya_bins* bins, int32_t nside, double* num,
                      double* wsum, double* xi, int32_t* sub_of_forest, void* stream) {
  if (!h) return LYA_ERR_INVALID_ARG;
  int st = check_bins(h, bins);
  if (st) return st;
  if (nside < 1 || nside > 64 || (nside & (nside - 1)))
    return fail(h, LYA_ERR_INVALID_ARG, "nside must be a power of two in 1..64");
  if (!num || !wsum) return fail(h, LYA_ERR_INVALID_ARG, "num and wsum are required");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if ((st = check_capture_stream(h, s))) return st;
  st = prepare(h, cat, 1, s);
  if (st) return st;
  st = ensure_pairs(h, cat, 1, bins, s);
  if (st) return st;
  // the pair kernel adds forest pair (a, b) at offset F.mock[a] * nb: the
  // sub-sample of the first forest (prepare() resets F.mock on the next call)
  CK(launch_subsample_ids(h->F, nside, h->F.mock, s), "sub-sample ids");
  if (sub_of_forest && cat->n_forests > 0)
    CK(cudaMemcpyAsync(sub_of_forest, h->F.mock, static_cast<size_t>(cat->n_forests) * 4, cudaMemcpyDeviceToDevice,
                       s),
       "sub-sample ids out");
  const int n_sub = 12 * nside * nside;
  return run_xi(h, cat, n_sub, bins, LYA_PREC_MIXED, static_cast<const int2*>(h->pairbuf),
                static_cast<const float2*>(h->csbuf), h->n_pairs, num, wsum, xi, s);
}

int lya_xi_covariance(lya_handle* h, const double* num_sub, const double* wsum_sub, int32_t n_sub, int32_t n_bins,
                      double* cov, double* xi, void* stream) {
  if (!h) return LYA_ERR_INVALID_ARG;
  if (n_sub < 1 || n_bins < 1 || n_bins > 65536 || n_sub > (1 << 20))
    return fail(h, LYA_ERR_INVALID_ARG, "n_sub in 1..2^20 and n_bins in 1..65536 required");
  if (!num_sub || !wsum_sub || !cov) return fail(h, LYA_ERR_INVALID_ARG, "NULL array");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (int st = check_capture_stream(h, s)) return st;
  cudaError_t e = grow(&h->outbuf, &h->out_cap, covariance_scratch_bytes(n_sub, n_bins));
  if (e != cudaSuccess) return fail(h, LYA_ERR_NO_MEMORY, "covariance scratch");
  CK(launch_covariance(num_sub, wsum_sub, n_sub, n_bins, cov, xi, h->outbuf, s), "covariance");
  return LYA_OK;
}

int lya_xi3(lya_handle* h, const lya_catalog* cat, const lya_bins3* bins, double* num, double* wsum, double* xi,
            void* stream) {
  if (!h) return LYA_ERR_INVALID_ARG;
  if (!bins) return fail(h, LYA_ERR_INVALID_ARG, "bins is NULL");
  if (bins->n_r < 1 || bins->n_r > 256 || bins->n_theta < 1 || bins->n_theta > 256 || bins->n_alpha < 1 ||
      bins->n_alpha > 1024)
    return fail(h, LYA_ERR_TOO_LARGE, "3PCF grid outside n_r, n_theta <= 256, n_alpha <= 1024");
  const int64_t nbins = static_cast<int64_t>(bins->n_r) * bins->n_r * bins->n_alpha * bins->n_theta * bins->n_theta;
  if (nbins > (1LL << 28)) return fail(h, LYA_ERR_TOO_LARGE, "3PCF grid above 2^28 bins");
  if (!(bins->r_max > 0) || !std::isfinite(bins->r_max)) return fail(h, LYA_ERR_INVALID_ARG, "r_max must be > 0");
  if (!num || !wsum) return fail(h, LYA_ERR_INVALID_ARG, "num and wsum are required");
  if (int st0 = refuse_in_capture(h, "lya_xi3")) return st0;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int st = prepare(h, cat, 1, s);
  if (st) return st;
  // forest pairs that can hold two pixels closer than r_max: the 2PCF list for r_par_max = r_perp_max = r_max
  const lya_bins nb2{1, 1, bins->r_max, bins->r_max};
  st = ensure_pairs(h, cat, 1, &nb2, s);
  if (st) return st;
  X3Args A;
  A.pairs = static_cast<const int2*>(h->pairbuf);
  A.n_pairs = h->n_pairs;
  A.pix = static_cast<const Pix*>(h->pixbuf);
  A.F = h->F;
  A.dist = cat->dist;
  A.n_pix = cat->n_pix;
  A.n_r = bins->n_r;
  A.n_theta = bins->n_theta;
  A.n_alpha = bins->n_alpha;
  A.r_max = bins->r_max;
  A.num = num;
  A.wsum = wsum;
  A.xi = xi;
  stage_begin(h, 0, s);
  CK(run_xi3(A, h->dev, &h->scratch2, &h->scratch2_cap, h->d_err, s), "xi3");
  stage_end(h, 0, s);
  return LYA_OK;
}

int lya_xi_bin_means_z(lya_handle* h, const lya_catalog* cat, const lya_bins* bins, const double* z_pix,
                       double* wsum, double* rpar_mean, double* rperp_mean, double* dist_mean, double* z_mean,
                       int64_t* npairs, void* stream) {
  if (!h) return LYA_ERR_INVALID_ARG;
  int st = check_bins(h, bins);
  if (st) return st;
  if (!rpar_mean || !rperp_mean || !dist_mean || !npairs)
    return fail(h, LYA_ERR_INVALID_ARG, "rpar_mean, rperp_mean, dist_mean and npairs are required");
  if ((z_pix == nullptr) != (z_mean == nullptr))
    return fail(h, LYA_ERR_INVALID_ARG, "z_pix and z_mean go together");
  if ((st = refuse_in_capture(h, "lya_xi_bin_means"))) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if ((st = prepare(h, cat, 1, s))) return st;
  if ((st = ensure_pairs(h, cat, 1, bins, s))) return st;
  const int nb = bins->n_par * bins->n_perp;
  if (means_smem_bytes(nb, h->max_len, z_pix != nullptr) > h->dev.smem_optin)
    return fail(h, LYA_ERR_TOO_LARGE, "bin means: 36 (44 with redshifts) bytes per bin + 8 (12) per pixel of the "
                                      "longest forest above shared memory");
  cudaError_t e = grow(&h->scratch2, &h->scratch2_cap, means_scratch_bytes(h->F.n, h->n_pairs, nb));
  if (e != cudaSuccess) return fail(h, LYA_ERR_NO_MEMORY, "bin-means scratch");
  MeansArgs A{};
  A.pairs = static_cast<const int2*>(h->pairbuf);
  A.cs = static_cast<const float2*>(h->csbuf);
  A.n_pairs = h->n_pairs;
  A.pix = static_cast<const Pix*>(h->pixbuf);
  A.F = h->F;
  A.n_par = bins->n_par;
  A.n_perp = bins->n_perp;
  A.d_par = bins->r_par_max / bins->n_par;
  A.d_perp = bins->r_perp_max / bins->n_perp;
  A.err = h->d_err;
  A.max_len = h->max_len;
  A.zpix = z_pix;
  stage_begin(h, 0, s);
  CK(launch_bin_means(A, h->dev, h->scratch2, wsum, rpar_mean, rperp_mean, dist_mean, z_mean, npairs, s),
     "bin means");
  stage_end(h, 0, s);
  return LYA_OK;
}

int lya_xi_bin_means(lya_handle* h, const lya_catalog* cat, const lya_bins* bins, double* wsum, double* rpar_mean,
                     double* rperp_mean, double* dist_mean, int64_t* npairs, void* stream) {
  return lya_xi_bin_means_z(h, cat, bins, nullptr, wsum, rpar_mean, rperp_mean, dist_mean, nullptr, npairs, stream);
}

// ---------------------------------------------------------------------------
// forest x quasar cross-correlation, its distortion matrix, 1D correlation
// ---------------------------------------------------------------------------
}  // extern "C"

namespace {

int prepare_quasars(lya_handle* h, const lya_quasars* q, cudaStream_t s) {
  if (!q) return fail(h, LYA_ERR_INVALID_ARG, "quasars is NULL");
  if (q->n < 0) return fail(h, LYA_ERR_INVALID_ARG, "negative quasar count");
  if (q->n >= (1LL << 31) - 1) return fail(h, LYA_ERR_TOO_LARGE, "more than 2^31-2 quasars");
  if (q->n > 0 && (!q->ra || !q->dec || !q->dist || !q->weight))
    return fail(h, LYA_ERR_INVALID_ARG, "quasar array is NULL");
  const int64_t n = std::max<int64_t>(q->n, 1);
  const size_t bytes = static_cast<size_t>(n) * (8 * 4 + 4) + 8 * 256;
  cudaError_t e = grow(&h->qbuf, &h->qbuf_cap, bytes);
  if (e != cudaSuccess) return fail(h, LYA_ERR_NO_MEMORY, "quasar workspace");
  char* p = static_cast<char*>(h->qbuf);
  auto take = [&](size_t b) { char* r = p; p += (b + 255) & ~size_t(255); return r; };
  Forests Q{};
  Q.n = q->n;
  Q.ux = reinterpret_cast<double*>(take(n * 8));
  Q.uy = reinterpret_cast<double*>(take(n * 8));
  Q.uz = reinterpret_cast<double*>(take(n * 8));
  Q.dmin = reinterpret_cast<double*>(take(n * 8));
  Q.dmax = Q.dmin;
  Q.len = reinterpret_cast<int32_t*>(take(n * 4));
  h->Q = Q;
  CK(launch_qso_prep(*q, Q, h->d_err, h->d_qfp, s), "quasar prep");
  return LYA_OK;
}

unsigned long long dmin_bits(lya_handle* h, const Forests& F, cudaStream_t s) {
  unsigned long long bits = ~0ull;
  if (cudaMemsetAsync(h->d_u64, 0xff, 8, s) != cudaSuccess) return bits;
  if (F.n > 0) {
    const int64_t blocks = std::min<int64_t>((F.n + 255) / 256, 4096);
    LYA_COUNT(1), min_dmin_kernel<<<static_cast<int>(blocks), 256, 0, s>>>(F, h->d_u64);
  }
  if (cudaMemcpyAsync(&bits, h->d_u64, 8, cudaMemcpyDeviceToHost, s) != cudaSuccess) return ~0ull;
  cudaStreamSynchronize(s);
  return bits;
}

// Prepare forests and quasars, check their flags, build the (forest, quasar) pair list.
int build_xpairs(lya_handle* h, const lya_catalog* cat, const lya_quasars* q, const int64_t* forest_qso,
                 const lya_bins* b, int* max_len, cudaStream_t s) {
  int st = prepare(h, cat, 1, s);
  if (st) return st;
  CK(cudaMemsetAsync(h->d_qfp, 0, 8, s), "clear quasar fingerprint");
  if ((st = prepare_quasars(h, q, s))) return st;
  CK(launch_own_hash(forest_qso, cat->n_forests, h->d_qfp, s), "own-quasar hash");
  CK(launch_max_len(h->F, h->d_i32, s), "max_len");
  int32_t ml = 0;
  unsigned long long fp = 0, qfp = 0;
  CK(cudaMemcpyAsync(&ml, h->d_i32, 4, cudaMemcpyDeviceToHost, s), "read max_len");
  CK(cudaMemcpyAsync(&fp, h->d_fp, 8, cudaMemcpyDeviceToHost, s), "read fingerprint");
  CK(cudaMemcpyAsync(&qfp, h->d_qfp, 8, cudaMemcpyDeviceToHost, s), "read quasar fingerprint");
  unsigned flags = 0;
  if ((st = read_flags(h, s, &flags))) return st;
  if ((st = flags_to_status(h, flags))) return st;
  *max_len = ml;
  // reuse the list built for the same pointers, sizes, bins and geometry (see ensure_pairs)
  CatKey key = make_key(cat, 1, b);
  key.ptrs.push_back(q->ra);
  key.ptrs.push_back(q->dec);
  key.ptrs.push_back(q->dist);
  key.ptrs.push_back(forest_qso);
  key.sizes.push_back(q->n);
  if (h->xpairs_valid && h->xkey == key && h->x_fp == fp && h->x_qfp == qfp) {
    h->last_pairs = h->n_xpairs;
    return LYA_OK;
  }
  h->xpairs_valid = false;
  double dmf = 1.0, dmq = 1.0;
  const unsigned long long bf = dmin_bits(h, h->F, s), bq = dmin_bits(h, h->Q, s);
  if (bf != ~0ull) std::memcpy(&dmf, &bf, 8);
  if (bq != ~0ull) std::memcpy(&dmq, &bq, 8);
  const double th = 2.0 * std::asin(std::min(1.0, b->r_perp_max / (dmf + dmq)));
  const double th_deg = th * 180.0 / M_PI;
  int nside = 1;
  while (nside < 256 && 117.0 / th_deg >= 2.0 * nside) nside *= 2;
  stage_begin(h, 3, s);
  cudaError_t e = grow(&h->xqoff, &h->xqoff_cap, static_cast<size_t>(h->F.n + 1) * 8);
  if (e != cudaSuccess) return fail(h, LYA_ERR_NO_MEMORY, "forest-quasar offsets");
  CK(build_cross_pairs(h->F, h->Q, nside, b->r_par_max, b->r_perp_max, forest_qso, &h->xpairs, &h->xpair_cap,
                       static_cast<int64_t*>(h->xqoff), &h->n_xpairs, s),
     "forest-quasar pairs");
  stage_end(h, 3, s);
  h->last_pairs = h->n_xpairs;
  h->xkey = key;
  h->x_fp = fp;
  h->x_qfp = qfp;
  h->xpairs_valid = true;
  return LYA_OK;
}

XcfArgs xcf_args(lya_handle* h, const lya_catalog* cat, const lya_quasars* q, const lya_bins* b, int max_len) {
  XcfArgs A{};
  A.pairs = h->xpairs;
  A.qoff = static_cast<const int64_t*>(h->xqoff);
  A.n_pairs = h->n_xpairs;
  A.pix = static_cast<const Pix*>(h->pixbuf);
  A.F = h->F;
  A.Q = h->Q;
  A.wq = q->weight;
  A.delta = cat->delta;
  A.weight = cat->weight;
  A.n_par = b->n_par;
  A.n_perp = b->n_perp;
  A.r_par_max = b->r_par_max;
  A.r_perp_max = b->r_perp_max;
  A.max_len = max_len;
  A.err = h->d_err;
  return A;
}

}  // namespace

extern "C" {

int lya_xcf(lya_handle* h, const lya_catalog* cat, const lya_quasars* qso, const int64_t* forest_qso,
            const lya_bins* bins, double* num, double* wsum, double* xi, void* stream) {
  if (!h) return LYA_ERR_INVALID_ARG;
  int st = check_bins(h, bins);
  if (st) return st;
  if (!num || !wsum) return fail(h, LYA_ERR_INVALID_ARG, "num and wsum are required");
  const int nb = bins->n_par * bins->n_perp;
  if (xcf_smem_bytes(nb, 1) > h->dev.smem_optin)
    return fail(h, LYA_ERR_TOO_LARGE, "cross-correlation grid above the shared-memory histogram (16 bytes per bin)");
  if ((st = refuse_in_capture(h, "lya_xcf"))) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int ml = 0;
  if ((st = build_xpairs(h, cat, qso, forest_qso, bins, &ml, s))) return st;
  if (xcf_smem_bytes(nb, ml) > h->dev.smem_optin)
    return fail(h, LYA_ERR_TOO_LARGE, "cross-correlation: 16 bytes per bin + 20 per pixel of the longest forest above shared memory");
  CK(cudaMemsetAsync(num, 0, static_cast<size_t>(nb) * 8, s), "zero num");
  CK(cudaMemsetAsync(wsum, 0, static_cast<size_t>(nb) * 8, s), "zero wsum");
  XcfArgs A = xcf_args(h, cat, qso, bins, ml);
  A.num = num;
  A.wsum = wsum;
  stage_begin(h, 0, s);
  CK(launch_xcf(A, h->dev, s), "cross-correlation kernel");
  stage_end(h, 0, s);
  if (xi) CK(launch_finalize(num, wsum, xi, nb, s), "finalize");
  return LYA_OK;
}

int lya_xdmat(lya_handle* h, const lya_catalog* cat, const lya_quasars* qso, const int64_t* forest_qso,
              const lya_bins* bins, lya_eta eta, double p_subsample, uint64_t seed, double* dmat, double* wsum_dm,
              void* stream) {
  if (!h) return LYA_ERR_INVALID_ARG;
  int st = check_bins(h, bins);
  if (st) return st;
  if (!dmat) return fail(h, LYA_ERR_INVALID_ARG, "dmat is NULL");
  if (eta != LYA_ETA_IDENTITY && eta != LYA_ETA_MEAN_SLOPE) return fail(h, LYA_ERR_INVALID_ARG, "unknown eta");
  if (!(p_subsample >= 0.0 && p_subsample <= 1.0))
    return fail(h, LYA_ERR_INVALID_ARG, "p_subsample must lie in [0, 1]");
  if ((st = refuse_in_capture(h, "lya_xdmat"))) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int ml = 0;
  if ((st = build_xpairs(h, cat, qso, forest_qso, bins, &ml, s))) return st;
  if (xdm_warps(h->dev, ml) < 1)
    return fail(h, LYA_ERR_TOO_LARGE, "forests too long for the cross distortion matrix (20 bytes per pixel per warp)");
  const int nb = bins->n_par * bins->n_perp;
  const size_t nb2 = static_cast<size_t>(nb) * nb;
  cudaError_t e = grow(&h->gbuf, &h->g_cap, (nb2 + nb) * 8);
  if (e != cudaSuccess) return fail(h, LYA_ERR_NO_MEMORY, "distortion-matrix accumulator");
  double* G = static_cast<double*>(h->gbuf);
  double* wdm = G + nb2;
  CK(cudaMemsetAsync(G, 0, (nb2 + nb) * 8, s), "zero accumulator");
  XcfArgs A = xcf_args(h, cat, qso, bins, ml);
  A.eta_mean_slope = (eta == LYA_ETA_MEAN_SLOPE);
  A.p_subsample = p_subsample;
  A.seed = seed;
  A.G = G;
  A.wdm = wdm;
  stage_begin(h, 1, s);
  CK(launch_xdm(A, h->dev, s), "cross distortion-matrix kernel");
  stage_end(h, 1, s);
  CK(launch_dm_finalize(G, wdm, dmat, wsum_dm, nb, 1, s), "finalize");
  return LYA_OK;
}

int lya_xi1d(lya_handle* h, const lya_catalog* cat, int32_t n_bins, double r_max, double* num, double* wsum,
             double* xi, void* stream) {
  if (!h) return LYA_ERR_INVALID_ARG;
  if (n_bins < 1 || n_bins > 4096) return fail(h, LYA_ERR_TOO_LARGE, "1D grid outside 1..4096 bins");
  if (!(r_max > 0) || !std::isfinite(r_max)) return fail(h, LYA_ERR_INVALID_ARG, "r_max must be finite and > 0");
  if (!num || !wsum) return fail(h, LYA_ERR_INVALID_ARG, "num and wsum are required");
  int st = refuse_in_capture(h, "lya_xi1d");
  if (st) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if ((st = prepare(h, cat, 1, s))) return st;
  CK(launch_max_len(h->F, h->d_i32, s), "max_len");
  int32_t ml = 0;
  CK(cudaMemcpyAsync(&ml, h->d_i32, 4, cudaMemcpyDeviceToHost, s), "read max_len");
  unsigned flags = 0;
  if ((st = read_flags(h, s, &flags))) return st;
  if ((st = flags_to_status(h, flags))) return st;
  if (xi1d_smem_bytes(n_bins, ml) > h->dev.smem_optin)
    return fail(h, LYA_ERR_TOO_LARGE, "1D correlation: 16 bytes per bin + 24 per pixel of the longest forest above shared memory");
  CK(cudaMemsetAsync(num, 0, static_cast<size_t>(n_bins) * 8, s), "zero num");
  CK(cudaMemsetAsync(wsum, 0, static_cast<size_t>(n_bins) * 8, s), "zero wsum");
  X1Args A{};
  A.F = h->F;
  A.dist = cat->dist;
  A.delta = cat->delta;
  A.weight = cat->weight;
  A.n_bins = n_bins;
  A.r_max = r_max;
  A.num = num;
  A.wsum = wsum;
  A.max_len = ml;
  stage_begin(h, 0, s);
  CK(launch_xi1d(A, static_cast<const Pix*>(h->pixbuf), h->dev, s), "1D correlation kernel");
  stage_end(h, 0, s);
  if (xi) CK(launch_finalize(num, wsum, xi, n_bins, s), "finalize");
  return LYA_OK;
}

int lya_stage_ms(lya_handle* h, int32_t stage, float* ms) {
  if (!h || !ms || stage < 0 || stage > 3) return LYA_ERR_INVALID_ARG;
  if (int st = refuse_in_capture(h, "lya_stage_ms")) return st;
  if (!h->ev_used[stage]) return fail(h, LYA_ERR_INVALID_ARG, "stage has not run");
  CK(cudaEventSynchronize(h->ev[stage][1]), "event sync");
  CK(cudaEventElapsedTime(ms, h->ev[stage][0], h->ev[stage][1]), "elapsed");
  return LYA_OK;
}

int64_t lya_kernel_launches(void) { return static_cast<int64_t>(g_launches.load()); }

int lya_last_launch(lya_handle* h, int64_t* n_pairs, int32_t* grid, int32_t* block, int32_t* smem_bytes) {
  if (!h) return LYA_ERR_INVALID_ARG;
  if (int st = refuse_in_capture(h, "lya_last_launch")) return st;
  cudaDeviceSynchronize();
  if (n_pairs) *n_pairs = h->last_pairs;
  if (grid) *grid = h->last.blocks;
  if (block) *block = h->last.warps * 32;
  if (smem_bytes) *smem_bytes = h->last.smem;
  return LYA_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// CUDA graph capture of a sequence of calls
// ---------------------------------------------------------------------------
extern "C" {

int lya_capture_begin(lya_handle* h, void* stream) {
  if (!h) return LYA_ERR_INVALID_ARG;
  if (h->capturing) return fail(h, LYA_ERR_INVALID_ARG, "a capture is already open on this handle");
  if (t_capturing) return fail(h, LYA_ERR_INVALID_ARG, "this thread already captures on another handle");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (!s) return fail(h, LYA_ERR_INVALID_ARG, "the legacy default stream cannot be captured");
  CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal), "begin capture");
  h->capturing = true;
  h->cap_failed = false;
  h->cap_stream = s;
  h->cap_launches0 = g_launches.load();
  t_capturing = true;
  return LYA_OK;
}

int lya_capture_end(lya_handle* h, lya_graph** out) {
  if (!h) return LYA_ERR_INVALID_ARG;
  if (out) *out = nullptr;
  if (!h->capturing) return fail(h, LYA_ERR_INVALID_ARG, "no capture open on this handle");
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(h->cap_stream, &g);
  const bool failed = h->cap_failed;
  h->capturing = false;
  h->cap_failed = false;
  t_capturing = false;
  const long long kernels = g_launches.load() - h->cap_launches0;
  if (e != cudaSuccess || failed || !out) {
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(h, e, "end capture");
    if (failed) return fail(h, LYA_ERR_INVALID_ARG, "a call inside the capture failed: " + h->err);
    return fail(h, LYA_ERR_INVALID_ARG, "out is NULL");
  }
  cudaGraphExec_t ex = nullptr;
  const cudaError_t e2 = cudaGraphInstantiate(&ex, g, 0);
  if (e2 != cudaSuccess) {
    cudaGraphDestroy(g);
    return cuda_fail(h, e2, "instantiate graph");
  }
  lya_graph* G = new lya_graph();
  G->graph = g;
  G->exec = ex;
  G->h = h;
  G->alive = h->alive;
  G->bufs = handle_buffers(h);
  G->kernels = kernels;
  *out = G;
  return LYA_OK;
}

int lya_graph_launch(lya_graph* g, void* stream) {
  if (!g) return LYA_ERR_INVALID_ARG;
  if (!*g->alive) return LYA_ERR_INVALID_ARG;   // the handle was destroyed
  lya_handle* h = g->h;
  if (h->capturing) return fail(h, LYA_ERR_INVALID_ARG, "the handle is capturing");
  if (handle_buffers(h) != g->bufs)
    return fail(h, LYA_ERR_INVALID_ARG, "graph is stale: the handle's buffers were reallocated after capture");
  CK(cudaGraphLaunch(g->exec, static_cast<cudaStream_t>(stream)), "graph launch");
  count_launches(g->kernels);
  return LYA_OK;
}

int lya_graph_destroy(lya_graph* g) {
  if (!g) return LYA_ERR_INVALID_ARG;
  if (g->exec) cudaGraphExecDestroy(g->exec);
  if (g->graph) cudaGraphDestroy(g->graph);
  delete g;
  return LYA_OK;
}

}  // extern "C"
