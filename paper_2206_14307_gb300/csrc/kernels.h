// kernels.h -- launchers of the device kernels (internal to the library).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "common.cuh"

namespace nnqs {

int mpl_slot(int M);

// `nsm`: streaming multiprocessors of the device; grids are sized from it and
// the kernels' occupancy.
template <typename T>
cudaError_t launch_log_psi(const DevModel<T> &md, const uint64_t *cfg, int64_t n, double *out, int nsm,
                           cudaStream_t st);

// mode 0: h1 only (E_loc); mode 1: h1 and h2 (Lanczos)
template <typename T>
cudaError_t launch_ratio(const DevModel<T> &md, const uint64_t *cfg, int64_t n, int mode, double *h1, double *h2,
                         int nsm, cudaStream_t st);

// one tile variant (see variant_width) of the connected-configuration engine
template <typename T>
cudaError_t launch_ratio_variant(const DevModel<T> &md, int v, const uint64_t *cfg, int64_t n, int mode, double *h1,
                                 double *h2, int nsm, cudaStream_t st);

// FP64 per-block partial sums of the moment reduction: n, Re h1, |h1|^2,
// Re(conj h1 h2), Im h1, Im(conj h1 h2), |h2|^2
constexpr int kMomentSums = 7;

// observables: structure factor partial sums [grid][N + 1] and the p = 1 variance
int sq_grid(int64_t n, int nsm);
cudaError_t launch_structure_factor(const uint64_t *cfg, int64_t n, int L, int nwords, const double *weights,
                                    double *partial, int grid, double *sq_out, cudaStream_t st);
cudaError_t launch_lanczos_variance(const double *moments, const double *lanczos, double *out, cudaStream_t st);

// p = 2 Lanczos step: first-level neighbours, h3, moments about c and the 3x3 pencil
constexpr int kShiftBlocks = 64;
template <typename T>
cudaError_t launch_expand_nb(const DevModel<T> &md, const uint64_t *cfg, int64_t n, int64_t *cnt, int64_t *off,
                             cudaStream_t st);
template <typename T>
cudaError_t launch_fill_nb(const DevModel<T> &md, const uint64_t *cfg, int64_t n, const int64_t *off,
                           uint64_t *nb_cfg, double *nb_coef, cudaStream_t st);
template <typename T>
cudaError_t launch_h3(const DevModel<T> &md, const uint64_t *cfg, int64_t n, const int64_t *off,
                      const double *nb_coef, const double *lp, const double *lpn, const double *h2,
                      const double *h2n, double *h3, cudaStream_t st);
cudaError_t launch_krylov2(const double *h1, const double *h2, const double *h3, int64_t n, const double *c_ptr,
                           double *partial, int nb, double *mu_out, double *out, cudaStream_t st);

// Mixed batch (Lanczos mode): one persistent launch over (instance, sample)
// items; each instance runs with its own tile shape (GL lanes per row, MPL
// hidden units per lane).
constexpr int kNumTileShapes = 16;
constexpr int kTileGL[kNumTileShapes] = {8, 8, 16, 8, 8, 16, 8, 16, 16, 16, 32, 16, 32, 32, 32, 32};
constexpr int kTileMPL[kNumTileShapes] = {2, 4, 2, 5, 8, 4, 9, 5, 7, 8, 4, 9, 7, 8, 13, 16};
struct BatchItem { int model, sample, out; };
// sets the kernel's shared-memory limit; returns the number of resident CTAs (0 on error)
int mixed_grid(int nsm);
cudaError_t launch_mixed(int grid, const DevModel<float> *models, const int *shape, const BatchItem *items,
                         int nitems, int *counter, const uint64_t *cfg_all, const int64_t *cfg_off, double *h1_all,
                         double *h2_all, cudaStream_t st);
cudaError_t launch_moments_batched(const double *h1_all, const double *h2_all, const int64_t *out_off, int nmodels,
                                   double *moments, double *lanczos, cudaStream_t st);

// Bytes of per-chain cache the sampler needs, and the number of chains that
// run concurrently (the cache is needed for those only).
template <typename T> size_t sampler_cache_bytes(const DevModel<T> &md);
template <typename T> int sampler_grid(const DevModel<T> &md, int n_chains, int nsm);

template <typename T>
cudaError_t launch_sample(const DevModel<T> &md, uint64_t seed, int n_chains, int n_per_chain, int n_skip, int n_burn,
                          uint64_t *cfg_out, float *acc_out, void *cache, int nsm, cudaStream_t st);
// FP32 sampler with each chain's cache in the shared memory of a thread-block
// cluster; returns false (launching nothing) when the cache does not fit a
// cluster of at most 8 CTAs, else the launch status in *err.
bool launch_sample_cl(const DevModel<float> &md, uint64_t seed, int n_chains, int n_per_chain, int n_skip, int n_burn,
                      uint64_t *cfg_out, float *acc_out, int nsm, cudaStream_t st, cudaError_t *err);

// Per-CTA scratch of the gradient kernel (U, V rows) and its grid size.
template <typename T> size_t grad_scratch_bytes(const DevModel<T> &md);
template <typename T> int grad_grid(const DevModel<T> &md, int64_t n, int nsm);

// th (FP32 only, may be NULL): theta' = W.(T_g s) of every row of the n
// configurations, [n][K][G][M] (launch_log_psi_tc's theta output), read
// instead of computed
template <typename T>
cudaError_t launch_grad(const DevModel<T> &md, const uint64_t *cfg, int64_t n, double *O, void *scratch, int grid,
                        cudaStream_t st, const float2 *th = nullptr);

// configurations annihilated by the projection: mode 0 sets log psi = -inf,
// mode 1 sets h1/h2 (either may be NULL) to NaN and flags NNQS_ERANGE
template <typename T>
cudaError_t launch_mark_vanishing(const DevModel<T> &md, const uint64_t *cfg, int64_t n, int mode, double *o1,
                                  double *o2, cudaStream_t st);

// FP32 E_loc with the per-bond tables in shared memory (one CTA per SM) and
// packed FP32x2 arithmetic; supported when a model's tables fit one SM.
// tables: device buffer of eloc_fast_table_bytes, filled by launch_tables_paired
// from the model's connection tables.
bool eloc_fast_supported(const DevModel<float> &md);
size_t eloc_fast_table_bytes(const DevModel<float> &md);
cudaError_t launch_tables_paired(const DevModel<float> &md, void *tables, cudaStream_t st);
cudaError_t launch_eloc_fast(const DevModel<float> &md, const void *tables, const uint64_t *cfg, int64_t n,
                             double *h1, int nsm, cudaStream_t st);

// FP32 h1 and h2 (the Lanczos quantities) with the per-site factor tables in
// shared memory (one CTA per SM): second-level flip sets as exchanges in the
// once-exchanged configuration.  Supported when a model's site tables fit one
// SM next to the flip-set lists; tables: device buffer of
// lanczos_fast_table_bytes, filled by launch_tables_site_paired from the
// model's per-site tables.
bool lanczos_fast_supported(const DevModel<float> &md);
size_t lanczos_fast_table_bytes(const DevModel<float> &md);
cudaError_t launch_tables_site_paired(const DevModel<float> &md, void *tables, cudaStream_t st);
cudaError_t launch_lanczos_fast(const DevModel<float> &md, const void *tables, const uint64_t *cfg, int64_t n,
                                double *h1, double *h2, int nsm, cudaStream_t st);

// checked mode: first_bad <- lowest index of a configuration outside Sz = 0
// (UINT64_MAX if none)
cudaError_t launch_check_sz0(const uint64_t *cfg, int64_t n, int nwords, int N, unsigned long long *first_bad,
                             cudaStream_t st);

// FP64 reductions.  launch_moments: per-block partials -> raw sums (sums_out
// [kMomentSums], may be NULL), moments and the p = 1 step; launch_moments_finish:
// moments and the p = 1 step from raw sums (e.g. summed over processes).
cudaError_t launch_moments(const double *h1, const double *h2, int64_t n, double *partial, int nblocks,
                           double *moments, double *lanczos, cudaStream_t st, double *sums_out = nullptr);
cudaError_t launch_moments_finish(const double *sums, double *moments, double *lanczos, cudaStream_t st);
cudaError_t launch_eloc_sums(const double *eloc, int64_t n, double *partial, int nblocks, double *sums,
                             cudaStream_t st);
// SR pieces (Eq. 12), all in FP64; weights may be NULL (plain sample means)
size_t sr_scratch_doubles(int64_t n, int64_t P);
size_t egrad_scratch_doubles(int64_t n, int64_t P);
cudaError_t launch_energy_grad(const double *O, const double *eloc, const double *w, int64_t n, int64_t P, double *F,
                               double *scratch, cudaStream_t st);
cudaError_t launch_sr_matvec(const double *O, const double *w, int64_t n, int64_t P, const double *x, double lambda,
                             double *y, double *scratch, cudaStream_t st);
cudaError_t launch_sr_solve(const double *O, const double *w, int64_t n, int64_t P, const double *F, double lambda,
                            double dtau, int max_iter, double tol, double *x, double *info, double *params_inout,
                            double *scratch, cudaStream_t st);

// parameter-derived tables
template <typename T>
cudaError_t launch_build_tables(const double *params, int N, int M, int K, cx<T> *Wt, cx<T> *b, cx<T> *a, cx<T> *logc,
                                cx2<T> *X, cx2<T> *XA, cudaStream_t st);

template <typename T>
cudaError_t launch_tables_conn(const double *params, int N, int M, int Mp, int K, int nb, int use_bias,
                               const int16_t *bi, const int16_t *bj, cx<T> *Tb, cx<T> *Cb, cx<T> *S4, cx<T> *CS,
                               sc<T> *ES, cudaStream_t st);

// tensor-core (tcgen05) log psi with BF16-split weights: NS = 2 or 3 terms.
// The device image (tc_bimg_bytes) holds the split weights of every (RBM,
// hidden tile) and the bias table; pinv is [G][round16(N)] uint16 (tc_pinv_table).
bool tc_supported(int N, int M, int G, int K, int nsign, int NS);
size_t tc_bimg_bytes(int N, int M, int G, int K, int nsign, int NS);
size_t tc_pinv_bytes(int N, int G);
void tc_pinv_table(const uint8_t *perm, int N, int G, uint16_t *out);
cudaError_t launch_bimg(const double *params, int N, int M, int G, int K, int nsign, int NS, int use_bias,
                        uint16_t *img, cudaStream_t st);
// theta_out non-NULL: writes theta' = W.(T_g s) (no bias) of every row,
// [n][K][G][M] float2, instead of log psi (out unused)
cudaError_t launch_log_psi_tc(const DevModel<float> &md, const uint16_t *bimg, const uint16_t *pinv, int NS,
                              const uint64_t *cfg, int64_t n, double *out, int nsm, cudaStream_t st,
                              float2 *theta_out = nullptr);

}  // namespace nnqs
