/*
 * nnqs.h -- C ABI of the GB300 (sm_103a) library for batched variational Monte
 * Carlo of the spin-1/2 J1-J2 Heisenberg model with symmetry-projected sums of
 * complex restricted Boltzmann machines (Chen, Hendry, Weinberg, Feiguin,
 * "Systematic improvement of neural network quantum states using a Lanczos
 * recursion").
 *
 * Conventions shared by every call
 * --------------------------------
 *  - Lattice: L x L periodic square lattice, L even, 4 <= L <= 16; site
 *    i = x + L*y; N = L*L (Sec. 3.4).
 *  - Spins: s_i = 2 S^z_i = +-1.  The paper's RBM uses sigma = +-1/2
 *    (Sec. 3.1, Eq. 2); with s = 2 sigma the weights and visible biases here
 *    are half the paper's.
 *  - Configuration encoding ("cfg"): ceil(N/64) little-endian uint64 words per
 *    configuration, bit i set <=> s_i = +1.  Configurations passed to the
 *    energy and Lanczos calls must lie in the Sz = 0 sector (N/2 bits set).
 *  - Bonds (Eq. 1): for each site in increasing index, J1 (+x), J1 (+y),
 *    J2 (+x+y), J2 (+x-y); 4N bonds.  H = sum_b J_b S_i.S_j with diagonal
 *    J_b s_i s_j / 4 and off-diagonal J_b / 2 between configurations related
 *    by exchanging an anti-aligned pair.
 *  - Parameters: complex, K blocks of [log c_r, a_r[N], b_r[M], W_r[M][N]
 *    row-major]; P = K (1 + N + M + M N).  The wave function is
 *      psi(s) = sum_r c_r sum_{g in G} chi(g) [phi_r(T_g s) + chi_P phi_r(-T_g s)]
 *    with phi_r(t) = exp(a_r . t) prod_m 2 cosh(b_rm + W_rm . t) (Eq. 2; the
 *    bias-free Eq. 3 when use_bias = 0), G the translations (Eqs. 4-5) and/or
 *    the C4v operations about site 0 (Eq. 6), chi(g) = exp(-i K.R) chi_I(L),
 *    and the chi_P term present only with spin inversion.  The sum over r
 *    (K > 1) forms the linear combination of RBMs of Sec. 3.1.
 *  - Memory: every array argument is a DEVICE pointer owned by the caller
 *    (unless stated otherwise), and every call is asynchronous on the given
 *    CUDA stream (a cudaStream_t passed as void*; NULL = legacy default
 *    stream).  The library owns only the opaque model: parameters, lookup
 *    tables and a grow-only workspace.
 *  - Errors: every call returns NNQS_OK (0) or a negative code; the message
 *    of the last failure on the calling thread is nnqs_last_error().  No C++
 *    exception crosses this boundary.  Device-side range faults (a non-finite
 *    amplitude) are recorded in the model and reported by nnqs_status().
 */
#ifndef NNQS_H
#define NNQS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    NNQS_OK = 0,
    NNQS_EINVAL = -1,       /* invalid argument or model description */
    NNQS_ENOMEM = -2,       /* device allocation refused */
    NNQS_ECUDA = -3,        /* CUDA runtime error (message in nnqs_last_error) */
    NNQS_ETIMEOUT = -4,     /* a bounded device-side wait ran out */
    NNQS_EUNSUPPORTED = -5, /* valid but unsupported size or combination */
    NNQS_ERANGE = -6        /* a non-finite amplitude was produced on the device */
};

enum {
    NNQS_FP64 = 0,   /* every step in double precision (the plain FP64 GPU form) */
    NNQS_FP32 = 1,   /* FP32 arithmetic with exact binary exponent tracking */
    NNQS_BF16X2 = 2, /* FP32, theta GEMM of fresh amplitudes on tcgen05 tensor
                        cores with W split into two bf16 terms (hi + lo) */
    NNQS_BF16X3 = 3  /* as BF16X2 with a three-term split (hi + mid + lo) */
};

enum { NNQS_A1 = 0, NNQS_A2 = 1, NNQS_B1 = 2, NNQS_B2 = 3 };
enum { NNQS_K00 = 0, NNQS_KPIPI = 1, NNQS_KPI0 = 2, NNQS_K0PI = 3 };

/* Model description (plain old data). */
typedef struct nnqs_desc {
    int32_t L;                    /* even, 4..16 */
    double J1, J2;                /* Eq. 1 couplings */
    int32_t K;                    /* number of RBMs in the linear combination, 1..8 */
    int32_t M;                    /* hidden units per RBM, 1..512 */
    int32_t project_translations; /* Eqs. 4-5: sum over all N translations */
    int32_t project_point_group;  /* Eq. 6: sum over C4v (or its little group) */
    int32_t momentum;             /* NNQS_K00 .. NNQS_K0PI; (pi,0),(0,pi) use the
                                     little group {E, C2, sigma_x, sigma_y} */
    int32_t irrep;                /* NNQS_A1 .. NNQS_B2 (B1: even under axis mirrors,
                                     odd under diagonal mirrors) */
    int32_t spin_inversion;       /* 0 = off, +1 / -1 = character chi_P */
    int32_t use_bias;             /* 1: Eq. 2 with a, b; 0: bias-free Eq. 3 */
    int32_t precision;            /* NNQS_FP64 .. NNQS_BF16X3 */
    int32_t check_inputs;         /* 1: checked mode -- every call that takes
                                     configurations first verifies that each lies
                                     in the Sz = 0 sector the method samples
                                     (Sec. 3.2: N/2 bits set, none past site
                                     N - 1) and returns NNQS_EINVAL, naming the
                                     first offending index, otherwise.  The check
                                     runs on the device and synchronises the
                                     stream once per call.  0: no check (the
                                     default; results for such inputs are
                                     undefined). */
} nnqs_desc;

typedef struct nnqs_model nnqs_model;

/* Creates a model on the current CUDA device: validates the description,
 * builds the bond, permutation and character tables (Eqs. 1, 4-6) and
 * allocates parameter storage (zero parameters).  Errors: NNQS_EINVAL for an
 * invalid field or for spin_inversion = -1 without biases (the projection
 * would vanish identically, Eq. 3); NNQS_EUNSUPPORTED for sizes beyond the
 * limits above; NNQS_ENOMEM. */
int nnqs_create(const nnqs_desc *desc, nnqs_model **out);

/* Releases the model and its device memory (synchronises the device). */
int nnqs_destroy(nnqs_model *model);

/* Number of complex parameters P = K (1 + N + M + M N); -1 for NULL. */
int64_t nnqs_num_params(const nnqs_model *model);

/* Size of the symmetry group |G| used by the projection (Eqs. 4-6). */
int32_t nnqs_group_size(const nnqs_model *model);

/* Uploads parameters.  params: HOST pointer to P complex numbers stored as
 * (re, im) double pairs in the layout above.  Derived device tables
 * (transposed W, exp(+-2W), exp(+-2a), the bf16 split of W) are rebuilt on
 * the stream.  The host buffer may be reused when the call returns. */
int nnqs_set_params(nnqs_model *model, const double *params, int64_t P, void *stream);

/* Same, from a DEVICE buffer of P (re, im) double pairs (e.g. after an
 * SR update on the GPU). */
int nnqs_set_params_device(nnqs_model *model, const double *params, int64_t P, void *stream);

/* Metropolis-Hastings sampling of |psi|^2 with exchanges of anti-aligned
 * spin pairs (Sec. 3.2).  One persistent chain per (n_chains); each chain
 * keeps its per-hidden-unit amplitude cache on the device and updates it
 * incrementally on every accepted exchange.
 *   Random numbers: Philox4x32-10 (Salmon et al., SC'11) with key
 *   (seed_lo, seed_hi ^ chain).  Initial state: Fisher-Yates shuffle of
 *   N/2 up and N/2 down spins, driven by counters (q, 1, 0, 0).  Step t
 *   (t = 0, 1, ... counting burn-in) uses counter (t, 0, 0, 0): words x0, x1
 *   select the (x0 * N/2 >> 32)-th up site and the (x1 * N/2 >> 32)-th down
 *   site in increasing site order; u = (x2 >> 8) * 2^-24 and the exchange is
 *   accepted iff u < |psi(s')/psi(s)|^2.
 *   After n_burn steps, a configuration is written after every n_skip steps.
 * cfg_out: [n_chains * n_per_chain][ceil(N/64)] uint64, chain-major.
 * acc_out: [n_chains] float, accepted fraction of the post-burn-in steps
 *          (may be NULL).
 * The FP32 form keeps each chain's cache in the shared memory of one CTA (or
 * of a thread-block cluster, for caches larger than one CTA holds); a cache
 * entry outside its FP32 range (an entry e^{-2 theta} beyond 2^100 or, with
 * spin inversion, a hidden bias with |Re b| > 20) sets NNQS_ERANGE in the
 * status word.
 * Errors: NNQS_EINVAL (non-positive counts), NNQS_ENOMEM (chain caches). */
int nnqs_sample(nnqs_model *model, uint64_t seed, int32_t n_chains, int32_t n_per_chain,
                int32_t n_skip, int32_t n_burn, uint64_t *cfg_out, float *acc_out, void *stream);

/* log psi(s) for n configurations (Eqs. 2-6): logpsi_out [n][2] doubles
 * (re, im), Im in (-pi, pi].  cfg: [n][ceil(N/64)].  With NNQS_BF16X2/X3 the
 * theta products of all n*K*|G| transformed configurations run on the
 * tcgen05 tensor cores (bf16 split weights, fp32 accumulation in TMEM) for
 * every M up to the model limit of 512: the hidden units are taken in tiles of
 * at most 128, whose products multiply into each row's running product; the
 * log-cosh and projection sums are fused into the epilogue.  A shape whose
 * tiles do not fit the shared memory of one SM uses the FP32 form.  Accuracy
 * of theta: 2^-17 (two terms) or 2^-25 (three terms) relative to
 * sum_j |W_mj|.  A configuration whose amplitude vanishes by symmetry returns
 * re = -inf. */
int nnqs_log_psi(nnqs_model *model, const uint64_t *cfg, int64_t n, double *logpsi_out, void *stream);

/* Local energy (Sec. 3.2, Eq. 10): E_loc(s) = sum_s' H_{s s'} psi(s')/psi(s)
 * over the anti-aligned J1 and J2 bonds.  eloc_out: [n][2] (re, im).
 * sums_out (may be NULL): [4] doubles {sum Re E_loc, sum Im E_loc,
 * sum |E_loc|^2, n}, accumulated in FP64 on the device. */
int nnqs_local_energy(nnqs_model *model, const uint64_t *cfg, int64_t n, double *eloc_out,
                      double *sums_out, void *stream);

/* One Lanczos step (Sec. 3.3, Eqs. 13-18).  Per configuration
 *   h1 = (H psi)(s)/psi(s)   and   h2 = (H^2 psi)(s)/psi(s)
 * (h1_out, h2_out: [n][2], either may be NULL), and over all n samples of
 * |psi|^2 the FP64 moments
 *   moments_out[0..7] = {m0 = 1, m1 = <Re h1>, m2 = <|h1|^2>,
 *                        m3 = <Re(conj(h1) h2)>, n, <Im h1>,
 *                        <Im(conj(h1) h2)>, m4 = <|h2|^2>}
 * and the p = 1 energy lanczos_out[0..2] = {E_p1, v, alpha} of the 2x2
 * problem in span{psi0, psi1}:  v^2 = m2 - m1^2,
 * d = (m3 - 3 m1 m2 + 2 m1^3) / (2 v^3), alpha = d - sqrt(d^2 + 1),
 * E_p1 = m1 + v alpha (E_p1 = m1, alpha = 0 when v^2 <= 1e-14 m1^2).
 * moments_out and lanczos_out are device buffers (either may be NULL). */
int nnqs_lanczos_moments(nnqs_model *model, const uint64_t *cfg, int64_t n, double *h1_out,
                         double *h2_out, double *moments_out, double *lanczos_out, void *stream);

/* The Lanczos step of nnqs_lanczos_moments split for samples spread over
 * several processes (one GPU each; the samples of |psi|^2 are independent,
 * Sec. 3.2, so each process draws and evaluates its own chains).
 *
 * nnqs_lanczos_partial: h1 and h2 of this process's n configurations (h1_out,
 * h2_out: [n][2], either may be NULL) and their raw FP64 sums
 *   sums_out[0..6] = {n, sum Re h1, sum |h1|^2, sum Re(conj(h1) h2),
 *                     sum Im h1, sum Im(conj(h1) h2), sum |h2|^2}
 * (device [7]; n = 0 gives zeros).  Add sums_out element-wise over all
 * processes (an all-reduce of 7 doubles, e.g. NCCL on the same stream), then
 * nnqs_lanczos_finish: from the summed sums (device [7]) the moments_out [8]
 * and lanczos_out [3] of nnqs_lanczos_moments over the union of all samples
 * (either output may be NULL).  On one process the two calls give the result
 * of nnqs_lanczos_moments to FP64 rounding. */
int nnqs_lanczos_partial(nnqs_model *model, const uint64_t *cfg, int64_t n, double *h1_out, double *h2_out,
                         double *sums_out, void *stream);
int nnqs_lanczos_finish(const double *sums, double *moments_out, double *lanczos_out, void *stream);

/* The p = 2 Lanczos step (Sec. 3.3: |Psi_2> = (1 + beta_1 H + beta_2 H^2)|psi0>).
 * Per configuration
 *   h3 = (H^3 psi)(s)/psi(s) = diag(s) h2(s) + sum_b (J_b/2) [psi(s^b)/psi(s)] h2(s^b)
 * over the anti-aligned bonds b of s (h3_out: [n][2], may be NULL); over the n
 * samples of |psi|^2 the FP64 moments about c = <Re h1>
 *   mu_out[0..7] = {mu_0 = 1, mu_1, ..., mu_6, c},
 *   mu_k = <psi|(H - c)^k|psi>/<psi|psi>  (from a_i = ((H - c)^i psi)/psi:
 *   mu_{i+j} = <Re(conj(a_i) a_j)>),
 * and the lowest eigenpair of the 3x3 Krylov pencil A_ij = mu_{i+j+1},
 * B_ij = mu_{i+j} (i, j = 0..2):
 *   out[0..4] = {E_p2, x0 = 1, x1, x2, var_p2},  Psi_2 = sum_i x_i (H - c)^i psi0.
 * mu_out and out may be NULL.  Cost: one Lanczos-mode pass over every
 * first-level neighbour (about 2N per sample), i.e. about 2N p = 1 steps.
 * The neighbours' own amplitudes divide out of the formula, so a neighbour
 * whose projected amplitude vanishes (possible only for characters other than
 * +1, e.g. B1 or K != (0,0)) makes h3 undefined and raises NNQS_ERANGE in
 * nnqs_status.  Needs workspace for n x 4N neighbour configurations;
 * synchronises the stream once (to read the number of neighbours).  n >= 1. */
int nnqs_lanczos2(nnqs_model *model, const uint64_t *cfg, int64_t n, double *h3_out, double *mu_out, double *out,
                  void *stream);

/* Energy variance of the p = 0 and p = 1 states and the variance
 * extrapolation (Sec. 3.3 Eq. 16; Sec. 4.3), in FP64 on the device.  The p = 1
 * state is phi = psi0 + alpha psi1, psi1 = (H - m1) psi0 / v, i.e.
 * a psi0 + b H psi0 with b = alpha / v, a = 1 - alpha m1 / v, so that
 * <phi|H^k|phi> = a^2 m_k + 2ab m_{k+1} + b^2 m_{k+2} (k = 0, 1, 2):
 *   out[0..3] = {var0 = m2 - m1^2, E1 = <H>_phi, var1 = <H^2>_phi - E1^2,
 *                E_extrap},
 * E_extrap being the straight line through (var0, m1) and (var1, E1) at zero
 * variance (E1 if the variances are equal).  moments: the [8] output of
 * nnqs_lanczos_moments (m0..m3 and m4 = moments[7]); lanczos: its [3]
 * output; out: [4].  All device buffers; no model is needed. */
int nnqs_lanczos_variance(const double *moments, const double *lanczos, double *out, void *stream);

/* Static spin structure factor (Sec. 4.1):
 *   S(q) = (1/N^2) sum_{i,j} <sz_i sz_j> e^{i q.(r_i - r_j)},  sz = s/2,
 * for all N wave vectors q = 2 pi (qx, qy) / L, sq_out[qx + L qy] (FP64), as
 * the mean over the n configurations of the diagonal estimator
 * (1/N^2) |sum_j sz_j e^{i q.r_j}|^2 (weights: optional device [n], a
 * weighted mean; NULL = plain mean of |psi|^2 samples).  n >= 1. */
int nnqs_structure_factor(nnqs_model *model, const uint64_t *cfg, int64_t n, const double *weights,
                          double *sq_out, void *stream);

/* Log-derivatives O_k(s) = d log psi(s) / d alpha_k (holomorphic; Sec. 3.2,
 * after Eq. 12), in parameter order.  O_out: [n][P][2] doubles. */
int nnqs_grad_logpsi(nnqs_model *model, const uint64_t *cfg, int64_t n, double *O_out, void *stream);

/* Energy gradient F_k = <conj(O_k) (E_loc - <E_loc>)> over n samples (the
 * right-hand side of Eq. 12 without -dtau); for real coordinates
 * dE/dRe alpha_k = 2 Re F_k and dE/dIm alpha_k = 2 Im F_k.
 * O: [n][P][2], eloc: [n][2], F_out: [P][2] (all device, FP64; O 16-byte
 * aligned, else NNQS_EINVAL).  weights: [n] device doubles, or NULL for plain
 * means over samples drawn from |psi|^2 (with weights |psi|^2 over a complete
 * basis the result is the exact gradient).  Uses the model's workspace
 * (2 P doubles per chunk of samples, at most 128 chunks). */
int nnqs_energy_grad(const nnqs_model *model, const double *O, const double *eloc, const double *weights, int64_t n,
                     double *F_out, void *stream);

/* Matrix-free SR product (Eq. 12): y = (S + lambda I) x with
 * S_kk' = <conj(O_k) O_k'> - <conj(O_k)><O_k'>, accumulated in FP64.
 * O: [n][P][2], x, y: [P][2] (device; O and x 16-byte aligned, else
 * NNQS_EINVAL); weights as for nnqs_energy_grad. */
int nnqs_sr_matvec(const nnqs_model *model, const double *O, const double *weights, int64_t n, const double *x,
                   double lambda, double *y, void *stream);

/* Stochastic-reconfiguration step (Eq. 12 with the ridge lambda of Sec. 3.4):
 * solves (S + lambda I) delta = -dtau F by conjugate gradients in FP64,
 * matrix-free, entirely on the device (no host synchronisation; at most
 * max_iter iterations, stopping once |r| <= tol |dtau F|).
 * O: [n][P][2] (16-byte aligned, else NNQS_EINVAL), F: [P][2], delta_out: [P][2]
 * (device).
 * info_out (device [2] doubles, may be NULL): {iterations, |r| / |b|}.
 * params_inout (device [P][2], may be NULL): if given, delta is added to it
 * (the parameter update alpha += delta; follow with nnqs_set_params_device). */
int nnqs_sr_solve(const nnqs_model *model, const double *O, const double *weights, int64_t n, const double *F,
                  double lambda, double dtau, int32_t max_iter, double tol, double *delta_out, double *info_out,
                  double *params_inout, void *stream);

/* Lanczos moments without any device allocation.
 *
 * Same result as nnqs_lanczos_moments(model, cfg, n, NULL, NULL, moments_out,
 * lanczos_out, stream), for callers that cannot allocate device memory at the
 * point of the call: for example a caller whose device memory is owned up
 * front by another allocator (a framework's caching pool that holds the whole
 * budget), or a latency-sensitive loop that must not hit the device-wide
 * synchronisation that growing the model's workspace with cudaFree/cudaMalloc
 * implies.  The per-sample h1, h2 and the FP64 partial sums live in one
 * fixed-size, statically allocated device array of this library
 * (NNQS_NOALLOC_MAX_SAMPLES samples, about 2 MB), which every GPU that loads
 * the library holds until the process exits; this call never allocates.
 * The paper has no counterpart: it is a deployment variant of the call above.
 *   n must not exceed NNQS_NOALLOC_MAX_SAMPLES (NNQS_EINVAL otherwise).
 *   moments_out [8], lanczos_out [3]: caller-owned device buffers as above.
 *   The first call on a device looks up the array's device address (once per
 *   device, with that device current); make that first call before any
 *   stream capture.
 *   Every call shares the one array and overwrites it completely before it
 *   reads it back, so nothing carries over between calls; calls whose work
 *   overlaps on the GPU (different streams or threads at the same time) race
 *   on it and must be serialised by the caller. */
#define NNQS_NOALLOC_MAX_SAMPLES 65536
int nnqs_lanczos_moments_noalloc(nnqs_model *model, const uint64_t *cfg, int64_t n, double *moments_out,
                                 double *lanczos_out, void *stream);

/* ---------------------------------------------------------------------------
 * Mixed batch: instances of uneven size in one persistent launch.
 *
 * A batch owns n_models independent models (each with its own L, J1, J2, K, M,
 * projection and parameters).  nnqs_batch_lanczos computes, for every
 * instance, h1 = (H psi)/psi and h2 = (H^2 psi)/psi at its configurations and
 * the FP64 moments and p = 1 Lanczos step of nnqs_lanczos_moments (Sec. 3.3,
 * Eqs. 13-17), all instances in ONE persistent kernel launch plus one
 * reduction launch, replayed from a captured CUDA graph.  Each instance runs
 * with its own tile shape of the connected-configuration engine (GL lanes
 * per row of the projected sum x MPL hidden units per lane), chosen by
 * nnqs_batch_autotune or set by nnqs_batch_set_shape.  The paper has no
 * counterpart (it runs one model at a time): this is the batched form of the
 * Lanczos step.
 *
 * Layout shared by the batch calls: n_per_model is a HOST array [n_models] of
 * sample counts n_i >= 0; cfg holds the configurations of instance 0, then
 * instance 1, ..., each n_i x ceil(N_i/64) words; h1_out / h2_out are
 * [sum n_i][2] in the same order; moments_out is [n_models][8] and
 * lanczos_out [n_models][3] with the per-model layout of
 * nnqs_lanczos_moments.  The FP32 engine only: an FP64 instance gives
 * NNQS_EUNSUPPORTED.
 * ------------------------------------------------------------------------- */
typedef struct nnqs_batch nnqs_batch;

/* Number of tile shapes, and shape v's GL (lanes per row) and MPL (hidden
 * units per lane); its width is GL * MPL >= M of an instance that uses it. */
int32_t nnqs_num_tile_shapes(void);
int nnqs_tile_shape(int32_t v, int32_t *gl, int32_t *mpl);

/* Creates n_models >= 1 instances from descs (host array) on the current
 * device; parameters start at zero (set them through nnqs_batch_model).  Each
 * instance starts with the narrowest tile shape that holds its M. */
int nnqs_batch_create(const nnqs_desc *descs, int32_t n_models, nnqs_batch **out);
int nnqs_batch_destroy(nnqs_batch *batch);
int32_t nnqs_batch_size(const nnqs_batch *batch);

/* Borrowed handle of instance i (owned by the batch; never destroy it): use
 * it with every single-model call, e.g. nnqs_set_params or nnqs_sample. */
nnqs_model *nnqs_batch_model(nnqs_batch *batch, int32_t i);

/* Tile shape of instance i (-1 if i is out of range); setting one that does
 * not fit the instance's width gives NNQS_EINVAL.  Synchronises the device. */
int32_t nnqs_batch_get_shape(const nnqs_batch *batch, int32_t i);
int nnqs_batch_set_shape(nnqs_batch *batch, int32_t i, int32_t v);

/* Autotuner: for every instance with more than one candidate shape (widths up
 * to 15% above the narrowest that holds M), times the persistent kernel on
 * one full wave of that instance's first min(n_i, probe) configurations with
 * each candidate (CUDA events on stream) and keeps the fastest; instances of
 * the same size (N, M, |G|, inversion, bias) share one result.  Host outputs
 * (may be NULL): shape_out [n_models], ms_out [n_models] (the winning wave
 * time, 0 where nothing was timed).  Blocks until done. */
int nnqs_batch_autotune(nnqs_batch *batch, const uint64_t *cfg, const int64_t *n_per_model, int32_t probe,
                        int32_t *shape_out, double *ms_out, void *stream);

/* One Lanczos step of every instance (layout above).  h1_out, h2_out,
 * moments_out, lanczos_out may each be NULL (h1/h2 then live in the batch's
 * workspace).  The first call with a given set of pointers and counts builds
 * the work list (instances in decreasing per-sample work), copies it to the
 * device (synchronising the stream) and captures the launches as a CUDA
 * graph; later calls with the same arguments only replay the graph on
 * stream.  Calls on one batch must not overlap on the GPU. */
int nnqs_batch_lanczos(nnqs_batch *batch, const uint64_t *cfg, const int64_t *n_per_model, double *h1_out,
                       double *h2_out, double *moments_out, double *lanczos_out, void *stream);

/* nnqs_status over every instance: the first non-OK status, else NNQS_OK. */
int nnqs_batch_status(nnqs_batch *batch, void *stream);

/* Device status word: NNQS_OK, or NNQS_ERANGE if a kernel produced a
 * non-finite amplitude since the last call.  Synchronises the stream and
 * clears the word. */
int nnqs_status(nnqs_model *model, void *stream);

/* Message of the last error on the calling thread ("" if none). */
const char *nnqs_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* NNQS_H */
