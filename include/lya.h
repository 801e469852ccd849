/*
 * lya.h -- C ABI of the GB300 Lyman-alpha pixel-pair library (liblya.so).
 *
 * The library computes, for a catalogue of Lyman-alpha forests, the binned
 * two-point estimator of arxiv 2507.00129 Eq. (2.4)
 *
 *     xi_A = sum_{(i,j) in A} (w_i d_i)(w_j d_j) / sum_{(i,j) in A} w_i w_j ,
 *
 * its distortion matrix (Eq. 2.6, with the continuum projection eta of
 * Eq. 2.7), the projection itself, and the gradient of xi with respect to the
 * deltas and weights.  Pixel pairs (i, j) come from different forests
 * (Section 2.1); a pair falls in bin A = p * n_perp + t when
 *
 *     p = floor(r_par / D_par),  t = floor(r_perp / D_perp),  p < n_par, t < n_perp,
 *     r_par = |d_i - d_j| cos(theta/2),  r_perp = (d_i + d_j) sin(theta/2),
 *
 * with D = r_max / n and theta the angle between the two lines of sight.
 * Every unordered forest pair is counted once.
 *
 * Conventions for every entry point:
 *  - All array pointers are DEVICE pointers owned by the caller; the library
 *    never frees or retains them past the call.  Scratch memory (pair lists,
 *    packed pixels, accumulators) is owned by the handle, allocated on first
 *    use, reused by later calls and released by lya_destroy.
 *  - Work is enqueued on the given stream (a cudaStream_t passed as void*,
 *    NULL = legacy default stream) and is asynchronous unless stated.
 *  - Outputs are overwritten, never accumulated into.
 *  - Return value: LYA_OK (0) or a negative LYA_ERR_* code; lya_last_error()
 *    gives a message.  Checks that need the data (sorted distances, finite
 *    values, non-negative weights, consistent offsets) run on the device and
 *    raise a flag that the next synchronising call (lya_pairs_build,
 *    lya_sync_status) reports; kernels stay in bounds whatever the data.
 *  - One handle serves one device and one stream at a time (not thread-safe).
 */
#ifndef LYA_H
#define LYA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  LYA_OK = 0,
  LYA_ERR_INVALID_ARG = -1,   /* bad pointer, size or bin grid */
  LYA_ERR_UNSORTED = -2,      /* distances not strictly increasing in a forest */
  LYA_ERR_NONFINITE = -3,     /* NaN/Inf input, or a negative weight */
  LYA_ERR_NO_MEMORY = -4,     /* device allocation failed */
  LYA_ERR_CUDA = -5,          /* a CUDA runtime call failed */
  LYA_ERR_TIMEOUT = -6,       /* a bounded device retry loop gave up (shared-memory compare-and-swap) */
  LYA_ERR_DEVICE_CHECK = -7,  /* inconsistent offsets seen on the device */
  LYA_ERR_TOO_LARGE = -8      /* size beyond a documented limit */
};

typedef struct lya_handle lya_handle;

/* A forest catalogue as flat pixel arrays.  Forest f owns pixels
 * offsets[f] .. offsets[f+1]-1 (offsets[0] = 0, offsets[n_forests] = n_pix).
 * Within a forest dist must be strictly increasing (pixels sorted by
 * wavelength), the source data layout of Section 3.1 with NaN pixels removed. */
typedef struct {
  int64_t n_forests;
  int64_t n_pix;
  const int64_t* offsets; /* [n_forests+1] */
  const double* ra;       /* [n_forests] right ascension, radians */
  const double* dec;      /* [n_forests] declination, radians */
  const double* dist;     /* [n_pix] comoving distance, Mpc/h */
  const double* loglam;   /* [n_pix] Lambda = log(lambda), any base */
  const float* delta;     /* [n_pix] flux-transmission fluctuation, Eq. (2.3) */
  const float* weight;    /* [n_pix] weight w >= 0 (w = 0 pixels allowed) */
} lya_catalog;

/* Bin grid of Section 2.1: n_par x n_perp rectangles, D = r_max / n.
 * Limits: 1 <= n_par <= 512, 1 <= n_perp <= 4096, n_par * n_perp <= 65536. */
typedef struct {
  int32_t n_par;
  int32_t n_perp;
  double r_par_max;
  double r_perp_max;
} lya_bins;

typedef enum {
  LYA_PREC_FP64 = 0,  /* separations, binning, products and sums in FP64 */
  LYA_PREC_MIXED = 1  /* FP32 separations/binning/products, FP64 bin sums */
} lya_precision;

typedef enum {
  LYA_ETA_IDENTITY = 0,   /* eta = I: D reduces to the identity (a check) */
  LYA_ETA_MEAN_SLOPE = 1  /* eta of Eq. (2.7): weighted mean and log-lambda slope removed */
} lya_eta;

/* Create a handle on the current CUDA device.  No device memory is taken
 * until the first call that needs it.  *out = NULL on failure. */
int lya_create(lya_handle** out);

/* Release the handle and all its scratch memory.  Synchronises the device. */
int lya_destroy(lya_handle* h);

/* Copy the last error message (NUL-terminated, truncated to n bytes). */
int lya_last_error(const lya_handle* h, char* buf, size_t n);

/* Human-readable name of a status code (static string). */
const char* lya_status_string(int status);

/* Wait for all work on `stream` and report the device-side input checks
 * raised since the last synchronising call (then clear them). */
int lya_sync_status(lya_handle* h, void* stream);

/* Forest-pair neighbour list (Section 2.1: only forests within a
 * neighbourhood set by the maximum separation, found with HEALPix cells,
 * Section 3.1).  Keeps every unordered pair (a < b) of non-empty forests with
 * (d_min,a + d_min,b) sin(theta/2) < r_perp_max -- a test that drops only
 * pairs with no in-grid pixel pair.  The list is cached in the handle for the
 * (catalogue pointers, sizes, bins) triple and reused by later calls; this
 * call rebuilds it.  Synchronises `stream`; returns input-check failures.
 * *n_pairs (host, optional) receives the pair count. */
int lya_pairs_build(lya_handle* h, const lya_catalog* cat, const lya_bins* bins,
                    int64_t* n_pairs, void* stream);

/* Copy the cached pair list (each pair once with a < b, in the library's
 * internal order: grouped by catalogue and first r_perp row) into caller device arrays of
 * capacity `cap`; *n_pairs (host) receives the count.  Synchronises.
 * Fails with LYA_ERR_INVALID_ARG if no list is cached or cap is too small. */
int lya_pairs_get(lya_handle* h, int32_t* pair_a, int32_t* pair_b, int64_t cap,
                  int64_t* n_pairs, void* stream);

/* Continuum projection of Eq. (2.7) applied to delta, forest by forest:
 * delta' = delta - sum(w delta)/W - x sum(w x delta)/S with x = Lambda - Lbar,
 * Lbar = sum(w Lambda)/W, W = sum w, S = sum w x^2 (sums in FP64).  S = 0
 * drops the slope term; W = 0 leaves the forest unchanged.
 * delta_out: [n_pix] device, may alias cat->delta. */
int lya_project(lya_handle* h, const lya_catalog* cat, float* delta_out, void* stream);

/* Two-point estimator, Eq. (2.4), over the cached (or freshly built) pair
 * list.  num[A] = sum (w d)_i (w d)_j, wsum[A] = sum w_i w_j, xi = num/wsum
 * (0 where wsum = 0), each [n_par*n_perp] float64, A = p*n_perp + t.
 * Any of num/wsum/xi may be NULL except that xi needs num and wsum.
 * Builds the pair list (synchronising) if none is cached for these inputs.
 * Bin-grid limit of the pair kernels: n_par <= 203 (MIXED), <= 256 (FP64);
 * beyond it LYA_ERR_TOO_LARGE. */
int lya_xi(lya_handle* h, const lya_catalog* cat, const lya_bins* bins, lya_precision prec,
           double* num, double* wsum, double* xi, void* stream);

/* Same sums over an explicit forest-pair list (device int32 arrays of n_pairs
 * pairs; any order; each pair counted once).  Used to evaluate xi on a
 * sample of the pairs of a large catalogue. */
int lya_xi_pairs(lya_handle* h, const lya_catalog* cat, const lya_bins* bins, lya_precision prec,
                 const int32_t* pair_a, const int32_t* pair_b, int64_t n_pairs,
                 double* num, double* wsum, double* xi, void* stream);

/* Distortion matrix, Eq. (2.6):
 *   D_AB = W_A^-1 sum_{(i,j) in A} w_i w_j sum_{(k,l) in B} eta_ik eta_jl
 * over a seeded subsample of the forest pairs (Section 2.2 "a small subset"):
 * pair (a<b) is kept iff p_subsample >= 1 or
 * SplitMix64(seed XOR (a*2^32 + b)) < floor(p_subsample * 2^64), SplitMix64
 * being the first output of the Steele-Lea-Flood generator for that state.
 * W_A (wsum_dm, [nb] float64, optional) sums w_i w_j over the kept pairs.
 * dmat: [nb*nb] float64, row A, column B.  Computed from the expansion of
 * eta = I - rank 2 into per-bin sums (no O(N^4) contraction); FP32 products
 * with FP64 accumulation.  Limits: nb <= 65536 (dmat is nb^2 doubles). */
int lya_dmat(lya_handle* h, const lya_catalog* cat, const lya_bins* bins, lya_eta eta,
             double p_subsample, uint64_t seed, double* dmat, double* wsum_dm, void* stream);

/* Distortion matrices of n_mocks independent catalogues in one launch (the
 * mock batch used for covariances): mock m gets exactly what lya_dmat gives
 * for that catalogue alone with the same eta, p_subsample and seed -- the
 * subsample rule sees forest indices local to each catalogue.  mocks is a
 * host array of catalogue descriptors (device data each).  dmat:
 * [n_mocks * nb * nb] float64, mock m at offset m * nb * nb (row A, column B);
 * wsum_dm (optional): [n_mocks * nb].  The handle's accumulator holds
 * n_mocks * (nb^2 + nb) doubles.  Pair lists as for lya_xi_batched. */
int lya_dmat_batched(lya_handle* h, const lya_catalog* mocks, int32_t n_mocks, const lya_bins* bins,
                     lya_eta eta, double p_subsample, uint64_t seed, double* dmat, double* wsum_dm,
                     void* stream);

/* Gradient of L = sum_A grad_xi[A] xi_A (chain rule of Eq. 2.4):
 *   dL/d delta_i = w_i sum_j gamma_A (w d)_j,
 *   dL/d w_i     = delta_i sum_j gamma_A (w d)_j - sum_j gamma_A xi_A w_j,
 * gamma_A = grad_xi[A] / wsum[A] (0 where wsum = 0), j over in-grid partners.
 * xi and wsum are the forward outputs for the same inputs (MIXED binning).
 * grad_delta, grad_weight: [n_pix] float32 device, overwritten. */
int lya_xi_backward(lya_handle* h, const lya_catalog* cat, const lya_bins* bins,
                    const double* grad_xi, const double* xi, const double* wsum,
                    float* grad_delta, float* grad_weight, void* stream);

/* Gradient of L = sum_A grad_xi[A] xi_A + sum_A grad_wsum[A] W_A: as
 * lya_xi_backward, with the weight sum's own dependence on w added,
 *   dL/d w_i += sum_j grad_wsum[A] w_j   (dW_A/dw_i = sum_{j in A} w_j),
 * i.e. gamma_A xi_A is replaced by gamma_A xi_A - grad_wsum[A] in the w
 * gradient.  dL/d delta is unchanged (W does not depend on delta).
 * grad_wsum: [nb] float64 device, or NULL for 0 (then this is
 * lya_xi_backward).  The chain rule of Eq. (2.4) for both outputs of the
 * estimator; the paper has no adjoint. */
int lya_xi_backward_full(lya_handle* h, const lya_catalog* cat, const lya_bins* bins, const double* grad_xi,
                         const double* grad_wsum, const double* xi, const double* wsum, float* grad_delta,
                         float* grad_weight, void* stream);

/* xi for n_mocks independent catalogues in one persistent launch.  mocks is a
 * host array of n_mocks catalogue descriptors (device data each); outputs are
 * [n_mocks * nb] float64, mock m at offset m*nb.  Pair lists are built per
 * mock (synchronising) and cached until the inputs change. */
int lya_xi_batched(lya_handle* h, const lya_catalog* mocks, int32_t n_mocks, const lya_bins* bins,
                   lya_precision prec, double* num, double* wsum, double* xi, void* stream);

/* Tuning: pick launch parameters of the pair kernel by timing candidates on
 * the cached pair list of `cat` (synchronising); the choice is kept in the
 * handle for later lya_xi calls with the same bin grid.  *choice (optional,
 * host) receives an index into the candidate table. */
int lya_autotune(lya_handle* h, const lya_catalog* cat, const lya_bins* bins, int32_t* choice,
                 void* stream);

/* Diagnostics of the last lya_xi launch (host outputs, synchronising):
 * the number of forest pairs processed and the launch shape used. */
int lya_last_launch(lya_handle* h, int64_t* n_pairs, int32_t* grid, int32_t* block,
                    int32_t* smem_bytes);

/* Work counts of the estimator over the cached pair list, for throughput
 * reporting (synchronising): over the forest pairs kept by the subsample rule
 * of lya_dmat (p_subsample >= 1 keeps all), *n_pairs receives the number of
 * forest pairs, *pixel_pairs the number of in-grid pixel pairs (the terms of
 * Eq. 2.4, MIXED binning) and *pixel_pairs_sq the sum over forest pairs of
 * (in-grid pixel pairs)^2 -- the number of terms of the quadruple sum of
 * Eq. (2.6).  Outputs are host pointers; any may be NULL. */
int lya_pair_stats(lya_handle* h, const lya_catalog* cat, const lya_bins* bins, double p_subsample,
                   uint64_t seed, int64_t* n_pairs, int64_t* pixel_pairs, double* pixel_pairs_sq,
                   void* stream);

/* How lya_dmat and lya_dmat_batched apply the rank-1 terms of the expanded
 * eta (Eq. 2.6 with Eq. 2.7) on the shared-memory triangle: mode 0 (default)
 * with FP32 fused multiply-adds in 4 x 4 register tiles per thread, mode 1
 * with the tensor cores (mma.sync m16n8k8, TF32 operands split as
 * x = hi + lo and three products per term, about FP32 accuracy).  Bands
 * wider than shared memory always use mode 0.  Host-only; LYA_ERR_INVALID_ARG
 * for another mode. */
int lya_set_dmat_tiles(lya_handle* h, int32_t mode);

/* Work counts of the closed-form distortion matrix of lya_dmat (Eq. 2.6
 * with eta of Eq. 2.7 expanded), for its roofline (synchronising): over the
 * forest pairs kept by the subsample rule of lya_dmat, with lya_dmat's FP32
 * binning, *n_pairs = kept forest pairs whose r_perp band reaches the grid,
 * *pixel_pairs = their in-grid pixel pairs, *sum_vec_support_sq = the sum over
 * every rank-1 vector (each column j of the second forest, a histogram over
 * the first forest's pixels, and each row i of the first forest) of |S_v|^2,
 * |S_v| being the number of distinct bins the vector touches, and
 * *sum_pair_support_sq = the sum over pairs of |S_pair|^2, the distinct bins
 * of all the pair's pixel pairs.  The closed form's algorithmic flops are
 * about 20 per in-grid pixel pair (T vectors and histograms) + 4 per entry of
 * the vectors' outer products (two rank-1 terms per vector, a multiply and an
 * add each) + 8 |S_pair|^2 (the four T outer products).  Host outputs, any may
 * be NULL.  LYA_ERR_CUDA if 33 * ceil(n_par n_perp / 32) words do not fit in
 * one block's shared memory. */
int lya_dmat_work(lya_handle* h, const lya_catalog* cat, const lya_bins* bins, double p_subsample, uint64_t seed,
                  int64_t* n_pairs, int64_t* pixel_pairs, double* sum_vec_support_sq, double* sum_pair_support_sq,
                  void* stream);

/* Per sub-sample sums for a covariance of xi (the paper takes its
 * uncertainties from sub-samples of the forests in HEALPix pixels, Sections
 * 3.2 and 3.4): forest pair (a < b) is added to the sub-sample of its first
 * forest a, the nested HEALPix pixel at resolution nside (a power of two,
 * 1..64) containing a's line of sight.  Outputs [12 nside^2 * nb] float64,
 * sub-sample s at offset s * nb: num and wsum (required; the sums of lya_xi
 * over the sub-sample's pairs, MIXED precision), xi (optional, num / wsum).
 * sub_of_forest (optional, device [n_forests] int32) receives each forest's
 * sub-sample.  Summing over sub-samples gives lya_xi's num and wsum. */
int lya_xi_subsamples(lya_handle* h, const lya_catalog* cat, const lya_bins* bins, int32_t nside,
                      double* num, double* wsum, double* xi, int32_t* sub_of_forest, void* stream);

/* Weighted sub-sample covariance of xi from per sub-sample sums (device
 * [n_sub * n_bins] float64 each, sub-sample s at offset s * n_bins):
 *   C_AB = sum_s W^s_A W^s_B (xi^s_A - xi_A)(xi^s_B - xi_B) / (W_A W_B),
 * xi^s = N^s / W^s, W = sum_s W^s, xi = (sum_s N^s) / W; rows and columns
 * with W_A = 0 are zero.  cov: [n_bins * n_bins] float64 (row A, column B);
 * xi (optional): [n_bins] full-sample xi.  FP64; sub-samples without weight
 * are skipped.  Limits: n_bins <= 65536, n_sub <= 2^20. */
int lya_xi_covariance(lya_handle* h, const double* num_sub, const double* wsum_sub, int32_t n_sub,
                      int32_t n_bins, double* cov, double* xi, void* stream);

/* Grid of the anisotropic three-point estimator (Section 2.3): n_r bins of
 * the side lengths over [0, r_max), n_theta bins of the angles of the sides
 * to the line of sight over [0, pi], n_alpha bins of the cosine of the inner
 * angle over [-1, 1].  The paper's figure uses r_max = 80 Mpc/h with
 * n_r = 20, n_theta = 10, n_alpha = 20. */
typedef struct {
  int32_t n_r;
  int32_t n_theta;
  int32_t n_alpha;
  double r_max;
} lya_bins3;

/* Three-point estimator, Eq. (2.8):
 *   xi3_A = sum_A (w d)_i (w d)_j (w d)_k / sum_A w_i w_j w_k
 * over pixel triplets of three distinct forests.  A record is a main vertex
 * i with r1 = x_j - x_i, r2 = x_k - x_i (x = d n); every pixel of a triplet is
 * the main vertex once and the other two take (r1, r2) in both orders; a
 * record needs |r1|, |r2| < r_max; theta is measured from the main vertex's
 * line of sight.  Triangle index
 *   A = (((i_r1 n_r + i_r2) n_alpha + i_alpha) n_theta + i_theta1) n_theta + i_theta2.
 * num, wsum (required), xi (optional): [n_r^2 n_alpha n_theta^2] float64.
 * The |r| and theta bins are computed in FP64, cos alpha in FP32; products
 * in FP32 are added to FP64 bin sums.  Builds (and caches) the forest-pair
 * list for r_par_max = r_perp_max = r_max.  Synchronises (a counting pass
 * sizes the kernel's neighbour capacity to the largest list); not allowed
 * during graph capture.  A main vertex with more neighbours within r_max
 * than one block holds (about 6,400 on GB300) is reported as
 * LYA_ERR_TOO_LARGE by the next synchronising call.  Limits: n_r, n_theta
 * <= 256, n_alpha <= 1024, at most 2^28 bins. */
int lya_xi3(lya_handle* h, const lya_catalog* cat, const lya_bins3* bins, double* num, double* wsum,
            double* xi, void* stream);

/* Per-bin weighted means of the separations and of the pair distance, and
 * pixel-pair counts, over the pixel pairs of Eq. (2.4) (the per-bin columns a
 * PICCA/Vega fit reads next to xi; the paper exports its results for Vega,
 * Appendix A):
 *   rpar_mean[A]  = sum_A w_i w_j r_par / W_A,   rperp_mean[A] = sum_A w_i w_j r_perp / W_A,
 *   dist_mean[A]  = sum_A w_i w_j (d_i + d_j)/2 / W_A  (Mpc/h; the bin's redshift
 *                   follows from the caller's d(z)),   npairs[A] = pixel pairs in A,
 * 0 where W_A = 0; wsum (optional) receives W_A.  Each [n_par*n_perp]
 * (float64; npairs int64).  Same pair list and FP32 bin arithmetic as the
 * mixed path of lya_xi; run sums in FP32, accumulation in double-float then
 * FP64.  Builds the pair list if none is cached (synchronises); refused
 * during graph capture.  Limit: 36 bytes per bin + 8 per pixel of the longest
 * forest of shared memory. */
int lya_xi_bin_means(lya_handle* h, const lya_catalog* cat, const lya_bins* bins, double* wsum, double* rpar_mean,
                     double* rperp_mean, double* dist_mean, int64_t* npairs, void* stream);

/* lya_xi_bin_means plus the bin's mean redshift (the redshift column of the
 * PICCA/Vega export, Appendix A):
 *   z_mean[A] = sum_A w_i w_j (z_i + z_j)/2 / W_A   (0 where W_A = 0),
 * the weighted mean of the pixel pairs' mean redshifts.  z_pix: [n_pix]
 * float64 device array of the catalogue's pixel redshifts, supplied by the
 * caller (the library holds no cosmology or rest-frame wavelength), read as
 * FP32 in the run sums.  z_pix and z_mean are both NULL (then this is
 * lya_xi_bin_means) or both given.  Limit: 44 bytes per bin + 12 per pixel of
 * the longest forest of shared memory. */
int lya_xi_bin_means_z(lya_handle* h, const lya_catalog* cat, const lya_bins* bins, const double* z_pix,
                       double* wsum, double* rpar_mean, double* rperp_mean, double* dist_mean, double* z_mean,
                       int64_t* npairs, void* stream);

/* Point tracers (quasars) for the forest x quasar cross-correlation.  Entries
 * with a non-finite or non-positive distance, non-finite position or weight,
 * or a negative weight are skipped and flagged (LYA_ERR_NONFINITE at the
 * call's own check). */
typedef struct {
  int64_t n;
  const double* ra;       /* [n] right ascension, radians */
  const double* dec;      /* [n] declination, radians */
  const double* dist;     /* [n] comoving distance, Mpc/h */
  const float* weight;    /* [n] quasar weight w_q >= 0 */
} lya_quasars;

/* Forest x quasar cross-correlation (the extension of Section 4; Eq. (2.4)
 * with the quasar as second point, weight w_q and no delta):
 *   num[A] = sum_{(i,q) in A} (w delta)_i w_q,  wsum[A] = sum w_i w_q,  xi = num/wsum,
 * r_par = (d_i - d_q) cos(theta/2) (signed), r_perp = (d_i + d_q) sin(theta/2),
 * A = p*n_perp + t with p = floor((r_par + r_par_max) / D_par),
 * D_par = 2 r_par_max / n_par (the grid spans [-r_par_max, r_par_max)), and
 * t = floor(r_perp / D_perp), D_perp = r_perp_max / n_perp.
 * Every pixel of every forest pairs with every quasar except the forest's own:
 * forest_qso ([n_forests] device int64, may be NULL) gives the index of each
 * forest's quasar in qso (-1 = none).  num, wsum required, xi optional, each
 * [n_par*n_perp] float64.  FP32 separations (bin decisions within about
 * 6e-5 bin widths of an edge may differ from FP64 ones), exact per-run sums,
 * FP64 accumulation.  Builds the (forest, quasar) pair list each call
 * (synchronises); refused during graph capture.  Limits: check of lya_bins,
 * and 16 bytes per bin of shared memory (n_par*n_perp <= 14,000 or so on
 * GB300; else LYA_ERR_TOO_LARGE). */
int lya_xcf(lya_handle* h, const lya_catalog* cat, const lya_quasars* qso, const int64_t* forest_qso,
            const lya_bins* bins, double* num, double* wsum, double* xi, void* stream);

/* Distortion matrix of the cross-correlation (Eq. (2.6) with the projection
 * eta of Eq. (2.7) acting on the forest only):
 *   D_AB = W_A^-1 sum_{(a,q)} sum_{i: (i,q) in A} w_i w_q sum_{k: (k,q) in B} eta_ik,
 * W_A (wsum_dm, [nb] float64, optional) the weight sum over the kept
 * (forest, quasar) pairs: (a, q) is kept iff p_subsample >= 1 or
 * SplitMix64(seed XOR (a*2^32 + q)) < floor(p_subsample * 2^64) (the rule of
 * lya_dmat on the ordered pair).  dmat: [nb*nb] float64, row A, column B.
 * Computed from eta = I - rank 2: the pair adds
 * w_q (diag(alpha) - alpha alpha^T / W_a - beta beta^T / S_a) with the
 * per-bin sums alpha = sum w_k, beta = sum w_k (Lambda_k - Lbar_a).
 * Refused during graph capture.  Limits: nb^2 doubles of scratch; forests up
 * to ~11,000 pixels (20 bytes of shared memory per pixel per warp). */
int lya_xdmat(lya_handle* h, const lya_catalog* cat, const lya_quasars* qso, const int64_t* forest_qso,
              const lya_bins* bins, lya_eta eta, double p_subsample, uint64_t seed, double* dmat,
              double* wsum_dm, void* stream);

/* Same-forest (one-dimensional) correlation: Eq. (2.4) over the pixel pairs
 * i < j of one forest that the three-dimensional estimator excludes
 * (Section 2.1), binned in p = floor(|d_i - d_j| / (r_max / n_bins)),
 * p < n_bins.  num, wsum required, xi optional, each [n_bins] float64.
 * FP64 throughout (bin decisions identical to the definition's).
 * Synchronises; refused during graph capture.  Limits: 1 <= n_bins <= 4096;
 * 16 bytes per bin + 24 per pixel of the longest forest of shared memory. */
int lya_xi1d(lya_handle* h, const lya_catalog* cat, int32_t n_bins, double r_max, double* num, double* wsum,
             double* xi, void* stream);

/* Tally of the mixed path's bin-edge flips (Section 2.1 binning done with FP32
 * separations): over the forest pairs kept by the subsample rule of lya_dmat
 * (p_subsample >= 1 keeps all), every pixel pair is binned with the mixed
 * kernel's FP32 arithmetic and with the FP64 path's (FP64 distances from
 * cat->dist, FP64 half-angle).  Host outputs (any may be NULL):
 * *pixel_pairs = in-grid pixel pairs under FP64 binning, *weight their
 * sum w_i w_j, *flipped = pixel pairs whose two bins differ (including pairs
 * in the grid under one binning only), *flipped_weight their sum w_i w_j.
 * Runs at the device's FP64 rate; use a subsample on large catalogues.
 * Synchronises. */
int lya_flip_tally(lya_handle* h, const lya_catalog* cat, const lya_bins* bins, double p_subsample,
                   uint64_t seed, int64_t* pixel_pairs, int64_t* flipped, double* weight,
                   double* flipped_weight, void* stream);

/* Device time (ms, CUDA events on the launching stream) of the last run of a
 * stage: 0 = pair kernel of lya_xi / lya_xi_pairs / lya_xi_batched,
 * 1 = distortion-matrix kernels of lya_dmat, 2 = adjoint kernel of
 * lya_xi_backward, 3 = pair-list build.  Synchronises.  LYA_ERR_INVALID_ARG
 * if the stage has not run on this handle. */
int lya_stage_ms(lya_handle* h, int32_t stage, float* ms);

/* The xi/W sums of lya_xi_pairs (MIXED precision) for callers that cannot
 * allocate device memory.  The paper has no counterpart to this entry point.
 *
 * Who needs it: code that must not call cudaMalloc at run time -- for
 * instance while another stream of the device is being captured into a CUDA
 * graph in the global capture mode (cudaMalloc is refused there), inside a
 * host whose device memory is entirely owned by a pool allocator, or in a
 * real-time pipeline that reserves all memory at start-up.  It takes no
 * handle (creating one allocates) and calls no cudaMalloc, cudaFree or
 * allocating library routine.
 *
 * Scratch: one file-scope device array of this library, 39.3 MiB, held on
 * every device where the library's module holding it is loaded (with CUDA's
 * lazy module loading: from the first call of this function on that device)
 * until the process exits.  The first call on a device looks up the array's
 * device address (cudaGetSymbolAddress) and caches it; make that first call
 * before any stream capture begins.  Every call shares the array and leaves
 * its contents behind; each call clears what must start at zero.  Calls that
 * overlap on the GPU (other streams, other host threads) race on the array:
 * serialise them.
 *
 * Limits: n_forests <= 65536, n_pix <= 1048576, n_pairs <= 1048576,
 * n_par <= 203 (the mixed pair kernel's limit), n_perp <= 4096 and
 * n_par * n_perp <= 65536; beyond them LYA_ERR_TOO_LARGE is returned before
 * any GPU work.  Arguments as for lya_xi_pairs (num/wsum may be NULL; xi needs
 * neither).
 *
 * Status codes.  Before any GPU work: LYA_ERR_INVALID_ARG for NULL pointers,
 * negative sizes, or r_par_max / r_perp_max not finite and > 0;
 * LYA_ERR_TOO_LARGE for the limits above.  After the work, which this call
 * waits for (it synchronises `stream`), it reports the device-side input
 * checks itself, where lya_xi_pairs leaves them to lya_sync_status:
 * LYA_ERR_UNSORTED, LYA_ERR_NONFINITE (also for a negative weight),
 * LYA_ERR_TOO_LARGE (a forest above 2^20 pixels) and LYA_ERR_DEVICE_CHECK
 * (inconsistent offsets, or a pair naming a forest outside [0, n_forests) or
 * the same forest twice; such pairs are skipped).  LYA_ERR_CUDA if a CUDA call
 * fails. */
int lya_xi_pairs_static(const lya_catalog* cat, const lya_bins* bins, const int32_t* pair_a,
                        const int32_t* pair_b, int64_t n_pairs, double* num, double* wsum, double* xi,
                        void* stream);

/* Number of CUDA kernels this library has launched in the calling process
 * since it was loaded (all handles).  Host-only; never fails.  A graph replay
 * (lya_graph_launch) counts the kernels it holds. */
int64_t lya_kernel_launches(void);

/* ---- CUDA-graph capture of a sequence of calls --------------------------
 * Repeated evaluations on one catalogue geometry with new deltas or weights
 * (field-level inference, many noise realisations of one mock footprint)
 * can replay a captured launch sequence instead of paying per-call launch and
 * host-synchronisation costs.  This batching of launches has no counterpart in
 * the paper, which launches one kernel per forest from Python (Section 3.1).
 *
 * lya_capture_begin starts a stream capture (thread-local mode) on `stream`,
 * which must not be the legacy default stream (NULL).  Until lya_capture_end,
 * calls of lya_project, lya_xi (MIXED only), lya_xi_batched (MIXED only),
 * lya_dmat, lya_dmat_batched and lya_xi_backward on this handle and this
 * stream are recorded,
 * not run.  While capturing they:
 *  - need the pair list of the same inputs cached (run each call once before
 *    capturing) and skip the geometry check, so ra, dec, dist and offsets
 *    must keep their values between replays; delta and weight are re-read by
 *    every replay (their pointers are fixed at capture);
 *  - allocate nothing: a buffer that would have to grow fails the call with
 *    LYA_ERR_INVALID_ARG (again: run the same calls once before capturing);
 *  - fail with LYA_ERR_INVALID_ARG if they would synchronise (lya_sync_status,
 *    lya_pairs_build, lya_pairs_get, lya_xi_pairs, lya_autotune,
 *    lya_pair_stats, lya_flip_tally, lya_xi3, lya_stage_ms, lya_last_launch)
 *    or use another stream.
 * Input checks still run on the device at every replay; read them with
 * lya_sync_status after a replay.  Outputs (caller pointers and the handle's
 * scratch) are fixed at capture.
 *
 * lya_capture_end ends the capture and instantiates it; *out receives the
 * graph (NULL on failure).  It fails if any call inside the capture failed.
 * lya_graph_launch replays it on any stream (asynchronous).  It refuses to run
 * (LYA_ERR_INVALID_ARG) if the handle has been destroyed, is capturing, or has
 * reallocated one of its buffers since the capture (a call on larger inputs,
 * or a different bin grid), because the graph would use freed memory.
 * lya_graph_destroy releases the graph (not the handle). */
typedef struct lya_graph lya_graph;
int lya_capture_begin(lya_handle* h, void* stream);
int lya_capture_end(lya_handle* h, lya_graph** out);
int lya_graph_launch(lya_graph* g, void* stream);
int lya_graph_destroy(lya_graph* g);

#ifdef __cplusplus
}
#endif
#endif /* LYA_H */
